"""Extended-precision evaluation of the dense oracle (test infrastructure only).

The same definition as oracle.mot -- Q_k of Section V-B composed densely,
Eq. (MOT) marched with Q_0^{-1} -- with every matrix product, projector,
inverse and solve carried out in numpy's long double (64-bit significand on
x86-64) by plain Gauss-Jordan elimination, so that the march of a given set of
FP64 input operators is obtained to ~1e-16 of its peak. It serves as the
reference where the FP64 oracle's own rounding is amplified by the march (a
mesh whose recursion magnifies operator-level rounding): the right-hand side
is formed in FP64 by oracle.mot (its rounding is not amplified) and promoted.

Projectors: P^S = Sigma (Sigma^T Sigma + 11^T/N_f)^{-1} Sigma^T and likewise
P^L with Lambda; since Sigma 1 = 0 and Lambda 1 = 0 exactly, this equals the
pseudo-inverse form of Section IV-B.
"""
from __future__ import annotations

import numpy as np

from . import mot as O

LD = np.longdouble


def inv_ld(A) -> np.ndarray:
    """Inverse by Gauss-Jordan elimination with partial pivoting in long double."""
    A = np.array(A, dtype=LD)
    n = A.shape[0]
    M = np.concatenate([A, np.eye(n, dtype=LD)], axis=1)
    for j in range(n):
        p = j + int(np.argmax(np.abs(M[j:, j])))
        if M[p, j] == 0:
            raise np.linalg.LinAlgError("singular matrix")
        if p != j:
            M[[j, p]] = M[[p, j]]
        M[j] /= M[j, j]
        f = M[:, j].copy()
        f[j] = 0
        M -= np.outer(f, M[j])
    return M[:, n:]


def _incidence(mesh):
    ne = mesh.ne
    rows = np.arange(ne)
    Lam = np.zeros((ne, mesh.nv), dtype=LD)
    Lam[rows, mesh.ev[:, 1]] = 1
    Lam[rows, mesh.ev[:, 0]] = -1
    Sig = np.zeros((ne, mesh.nf), dtype=LD)
    Sig[rows, mesh.ef[:, 0]] = 1
    Sig[rows, mesh.ef[:, 1]] = -1
    return Lam, Sig


def _projector(X) -> np.ndarray:
    n = X.shape[1]
    return X @ inv_ld(X.T @ X + np.ones((n, n), dtype=LD) / n) @ X.T


def _bd(M):
    z = np.zeros_like(M)
    return np.block([[M, z], [z, M]])


class ExtendedSystem:
    """Q_0 .. Q_{k_max+1}, [M1 | M2] and Q_0^{-1} in long double (Section V-B)."""

    def __init__(self, ops):
        self.ops = ops
        ne = ops.ne
        Lam, Sig = _incidence(ops.mesh)
        PS, PL = _projector(Sig), _projector(Lam)
        I = np.eye(ne, dtype=LD)
        PSH, PLH = I - PL, I - PS
        Ginv = inv_ld(ops.G.toarray())
        M1 = PSH @ ops.T0s.astype(LD) @ PSH @ Ginv        # T^{Sigma H} G^{-1}
        M2 = PL @ ops.T0h.astype(LD) @ PL @ Ginv @ PLH    # T^Lambda G^{-1} P^{Lambda H}
        self.M1b, self.M2b = _bd(M1), _bd(M2)
        PLHb, PSb = _bd(PLH), _bd(PS)
        self.Q = []
        for k in range(ops.kmax + 2):
            XA = O.pmchwt_block(ops, "A", k).astype(LD)
            XH = O.pmchwt_block(ops, "H", k).astype(LD)
            XT = O.pmchwt_block(ops, "T", k).astype(LD)
            self.Q.append(self.M1b @ XA @ PLHb + self.M1b @ XH @ PSb + self.M2b @ XT @ PLHb + self.M2b @ XA @ PSb)
        self.Q0inv = inv_ld(self.Q[0])

    def march(self, exc, n_steps: int, b: int = 0) -> np.ndarray:
        """w_i = Q_0^{-1} (r_i - sum_{k=1}^{i-1} Q_k w_{i-k}), i = 1..n_steps (long double)."""
        ne = self.ops.ne
        W = np.zeros((n_steps, 2 * ne), dtype=LD)
        for i in range(1, n_steps + 1):
            rho1, rho2 = O.rhs_parts(self.ops, exc, b, i)
            r = self.M1b @ rho1.astype(LD) + self.M2b @ rho2.astype(LD)
            for k in range(1, min(i, len(self.Q))):
                r = r - self.Q[k] @ W[i - k - 1]
            W[i - 1] = self.Q0inv @ r
        return W
