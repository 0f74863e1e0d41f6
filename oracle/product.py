"""Product-form FP64 oracle for meshes too large for explicit dense Q_k
(test infrastructure only; pinned against oracle.mot on small meshes).

Same definition as oracle.mot (paper Section V-B, Eq. (MOT)) but Q_k is never
formed: sum_k Q_k w_{i-k} = M1 sum_k (A_k l_{i-k} + A^_k s_{i-k})
                            + M2 sum_k (A~_k l_{i-k} + A_k s_{i-k}),
with l = P^{LH} w, s = P^S w, M1 = T^{SH} G^-1, M2 = T^L G^-1 P^{LH} formed
densely from pseudo-inverses and a dense inverse of G, the lag sums taken
entry by entry from the lag-window matrices, and Q_0 w_i = b_i solved by the
oracle's own GMRES.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp

from . import mot as O


class ProductSystem:
    def __init__(self, ops):
        self.ops = ops
        mesh = ops.mesh
        ne = ops.ne
        self.ne = ne
        rows = np.arange(ne)
        Lam = sp.csr_matrix((np.r_[np.ones(ne), -np.ones(ne)], (np.r_[rows, rows], np.r_[mesh.ev[:, 1], mesh.ev[:, 0]])),
                            shape=(ne, mesh.nv))
        Sig = sp.csr_matrix((np.r_[np.ones(ne), -np.ones(ne)], (np.r_[rows, rows], np.r_[mesh.ef[:, 0], mesh.ef[:, 1]])),
                            shape=(ne, mesh.nf))
        # P^S = Sigma (Sigma^T Sigma)^+ Sigma^T, P^L = Lambda (Lambda^T Lambda)^+ Lambda^T (Section IV-B)
        Ls = np.linalg.pinv((Sig.T @ Sig).toarray(), hermitian=True)
        Lv = np.linalg.pinv((Lam.T @ Lam).toarray(), hermitian=True)
        PS = np.asarray(Sig @ (Sig @ Ls).T).T
        PL = np.asarray(Lam @ (Lam @ Lv).T).T
        I = np.eye(ne)
        self.PS, self.PLH = PS, I - PS
        PSH = I - PL
        Ginv = np.linalg.inv(ops.G.toarray())
        self.M1 = (PSH @ ops.T0s @ PSH) @ Ginv
        self.M2 = (PL @ ops.T0h @ PL) @ Ginv @ self.PLH
        self.K = ops.kmax + 1
        self.R = self.K + 1
        # per-value index arrays of every lag-window matrix
        self.kinds = []
        fam_of = {"A": (ops.kmax, ((0, 0), (1, 1))), "H": (ops.kmax + 1, ((1, 0),)), "T": (ops.kmax - 1, ((0, 1),))}
        for name, m in ops.mats.items():
            fam = name[0]
            lim, uses = fam_of[fam]
            interior = name.endswith("p")
            typ = name[1]
            r = np.repeat(np.repeat(np.arange(ne), np.diff(m.rowptr)), m.cnt)
            c = np.repeat(m.col, m.cnt)
            first = np.repeat(np.cumsum(m.cnt) - m.cnt, m.cnt)
            lag = np.repeat(m.k0, m.cnt) + (np.arange(m.val.size) - first)
            v = m.val[np.repeat(m.voff, m.cnt) + (np.arange(m.val.size) - first)]
            keep = lag <= lim
            r, c, lag, v = r[keep], c[keep], lag[keep], v[keep]
            entry = dict(typ=typ, interior=interior, uses=uses, tail=None, lim=lim)
            # Z_0 of the family as a sparse N_e x N_e matrix, and its lags
            # 1..lim side by side, [Z_1 | Z_2 | ... | Z_lim] (N_e x lim N_e), so
            # that sum_k Z_k x_{i-k} is one product with the stacked
            # [x_{i-1}; x_{i-2}; ...]; repeated (row, column) pairs are summed
            l0 = lag == 0
            entry["Z0"] = sp.csr_matrix((v[l0], (r[l0], c[l0])), shape=(ne, ne))
            h = lag >= 1
            entry["Zh"] = (sp.csr_matrix((v[h], (r[h], (lag[h] - 1).astype(np.int64) * ne + c[h])),
                                         shape=(ne, lim * ne)) if lim >= 1 else None)
            del r, c, lag, v
            if m.ta is not None:
                tr = np.repeat(np.arange(ne), np.diff(m.rowptr))
                ok = m.ta <= ops.kmax - 1
                entry["tail"] = (tr[ok].astype(np.int32), m.col[ok].astype(np.int32), m.ta[ok].astype(np.int32),
                                 m.tc[ok])
            self.kinds.append(entry)

    # -- sums over the stored families --------------------------------------
    def _block(self, e, zu, zv, out_u, out_v):
        """Adds the 2 x 2 block of a family to (out_u, out_v), given zu = X pu
        and zv = X pv for the stored matrix X (T type: [[eta X, 0], [0, X / eta]];
        K type: [[0, -X], [X, 0]]; eta of the entry's medium)."""
        eta = self.ops.etap if e["interior"] else self.ops.eta
        if e["typ"] == "T":
            out_u += eta * zu
            out_v += zv / eta
        else:
            out_u -= zv
            out_v += zu

    def _apply(self, e, part_u, part_v, out_u, out_v, contrib_u, contrib_v):
        ops = self.ops
        eta = ops.etap if e["interior"] else ops.eta
        if e["typ"] == "T":
            out_u += eta * np.bincount(e["rows"], weights=contrib_u, minlength=self.ne)
            out_v += np.bincount(e["rows"], weights=contrib_v, minlength=self.ne) / eta
        else:  # K block: [[0, -K], [K, 0]]
            out_u -= np.bincount(e["rows"], weights=contrib_v, minlength=self.ne)
            out_v += np.bincount(e["rows"], weights=contrib_u, minlength=self.ne)

    def history(self, L, S, i):
        """s1 = sum_{k>=1} A_k l_{i-k} + A^_k s_{i-k}, s2 = sum_k A~_k l_{i-k} + A_k s_{i-k}
        with L[j], S[j] the loop/star parts (u; v) of step j (index 0 = step 0 = zero)."""
        ne = self.ne
        s = [np.zeros(ne), np.zeros(ne), np.zeros(ne), np.zeros(ne)]  # s1u, s1v, s2u, s2v
        # stacked coefficients [x_{i-1}; x_{i-2}; ...; x_{i-kmax-1}] of each part
        # (steps before the first are zero), u and v parts apart
        nl = self.ops.kmax + 1
        stacks = []
        for P in (L, S):
            X = np.zeros((nl, 2 * ne))
            for k in range(1, nl + 1):
                if i - k >= 1:
                    X[k - 1] = P[i - k]
            stacks.append((X[:, :ne].reshape(-1), X[:, ne:].reshape(-1)))
        for e in self.kinds:
            if e["Zh"] is not None:
                n = e["lim"] * ne
                for part, outi in e["uses"]:
                    xu, xv = stacks[part]
                    self._block(e, e["Zh"] @ xu[:n], e["Zh"] @ xv[:n], s[2 * outi], s[2 * outi + 1])
            if e["tail"] is not None:
                tr, tcol, ta, tc = e["tail"]
                # constant tail: sum_{k=a}^{kmax-1} l_{i-k} (steps >= 1)
                win = np.zeros((self.ops.kmax + 1, 2 * ne))
                acc = np.zeros(2 * ne)
                for k in range(self.ops.kmax - 1, 0, -1):
                    if i - k >= 1:
                        acc = acc + L[i - k]
                    win[k] = acc
                cu = tc * win[ta, tcol]
                cv = tc * win[ta, ne + tcol]
                sub = dict(e, rows=tr)
                self._apply(sub, None, None, s[2], s[3], cu, cv)
        return np.concatenate([s[0], s[1]]), np.concatenate([s[2], s[3]])

    def lag0(self, l, sg):
        """y1 = A_0 l + A^_0 s, y2 = A~_0 l + A_0 s (the lag-0 terms of Q_0 w)."""
        ne = self.ne
        s = [np.zeros(ne), np.zeros(ne), np.zeros(ne), np.zeros(ne)]
        parts = (l, sg)
        for e in self.kinds:
            Z = e["Z0"]
            for part, outi in e["uses"]:
                P = parts[part]
                self._block(e, Z @ P[:ne], Z @ P[ne:], s[2 * outi], s[2 * outi + 1])
        return np.concatenate([s[0], s[1]]), np.concatenate([s[2], s[3]])

    def split(self, w):
        ne = self.ne
        sg = np.concatenate([self.PS @ w[:ne], self.PS @ w[ne:]])
        return w - sg, sg

    def left(self, y1, y2):
        ne = self.ne
        return np.concatenate([self.M1 @ y1[:ne] + self.M2 @ y2[:ne], self.M1 @ y1[ne:] + self.M2 @ y2[ne:]])

    def q0(self, w):
        l, sg = self.split(w)
        y1, y2 = self.lag0(l, sg)
        return self.left(y1, y2)

    def march(self, exc, n_steps, b=0, tol=1e-13):
        ne = self.ne
        L = np.zeros((n_steps + 1, 2 * ne))
        S = np.zeros((n_steps + 1, 2 * ne))
        W = np.zeros((n_steps, 2 * ne))
        for i in range(1, n_steps + 1):
            W[i - 1] = self.step(exc, b, i, L, S, tol)
            L[i], S[i] = self.split(W[i - 1])
        return W

    def step(self, exc, b, i, L, S, tol=1e-13):
        rho1, rho2 = O.rhs_parts(self.ops, exc, b, i)
        s1, s2 = self.history(L, S, i)
        rhs = self.left(rho1 - s1, rho2 - s2)
        x, it, res = O.gmres(self.q0, rhs, tol=tol, restart=300, maxiter=3000)
        return x
