"""Dense FP64 oracle of the qHP TD-PMCHWT MOT scheme (test infrastructure only).

Every function cites the paper passage it follows. Notation: N_e edges,
w_i = (u_i, v_i) the auxiliary unknowns of step i (paper Eq. (xy)), Q_k the
block Toeplitz matrices of Eq. (fulldis_PMCHWT).
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np
import scipy.linalg as sla
from scipy.special import erf

# ---------------------------------------------------------------------------
# topology and projectors (Section IV-B)
# ---------------------------------------------------------------------------


def incidence(ev: np.ndarray, ef: np.ndarray, nv: int, nf: int):
    """Lambda (N_e x N_v): +1 at v^+_m, -1 at v^-_m. Sigma (N_e x N_f): +1 at
    c^+_m, -1 at c^-_m (Section IV-B, definitions of Lambda and Sigma)."""
    ne = ev.shape[0]
    Lam = np.zeros((ne, nv))
    Sig = np.zeros((ne, nf))
    for m in range(ne):
        Lam[m, ev[m, 1]] += 1.0
        Lam[m, ev[m, 0]] -= 1.0
        Sig[m, ef[m, 0]] += 1.0
        Sig[m, ef[m, 1]] -= 1.0
    return Lam, Sig


def projectors(Lam: np.ndarray, Sig: np.ndarray):
    """P^Sigma = Sigma (Sigma^T Sigma)^+ Sigma^T, P^{Lambda H} = I - P^Sigma
    (RWG space); P^Lambda = Lambda (Lambda^T Lambda)^+ Lambda^T,
    P^{Sigma H} = I - P^Lambda (BC space). Section IV-B, definition of the
    quasi-Helmholtz projectors."""
    ne = Lam.shape[0]
    PS = Sig @ np.linalg.pinv(Sig.T @ Sig) @ Sig.T
    PL = Lam @ np.linalg.pinv(Lam.T @ Lam) @ Lam.T
    I = np.eye(ne)
    return dict(PS=PS, PLH=I - PS, PL=PL, PSH=I - PL)


# ---------------------------------------------------------------------------
# lagged interaction matrices
# ---------------------------------------------------------------------------


def lag_dense(mat, k: int, kmax_tail: int) -> np.ndarray:
    """Dense N_e x N_e value of a lag-window matrix at lag k. A constant tail
    (K~ of Section V-B-3) applies for ta <= k <= kmax_tail."""
    ne = mat.ne
    out = np.zeros((ne, ne))
    for m in range(ne):
        for e in range(mat.rowptr[m], mat.rowptr[m + 1]):
            k0, cnt = mat.k0[e], mat.cnt[e]
            if k0 <= k < k0 + cnt:
                out[m, mat.col[e]] = mat.val[mat.voff[e] + k - k0]
            elif mat.ta is not None and mat.ta[e] <= k <= kmax_tail:
                out[m, mat.col[e]] = mat.tc[e]
    return out


def lag_dense_fast(mat, k: int, kmax_tail: int) -> np.ndarray:
    """Vectorised lag_dense (same values)."""
    ne = mat.ne
    rows = np.repeat(np.arange(ne), np.diff(mat.rowptr))
    out = np.zeros((ne, ne))
    inwin = (mat.k0 <= k) & (k < mat.k0 + mat.cnt)
    idx = np.nonzero(inwin)[0]
    out[rows[idx], mat.col[idx]] = mat.val[mat.voff[idx] + k - mat.k0[idx]]
    if mat.ta is not None and k <= kmax_tail:
        t = np.nonzero((mat.ta <= k) & ~inwin)[0]
        out[rows[t], mat.col[t]] = mat.tc[t]
    return out


def pmchwt_block(ops, fam: str, k: int) -> np.ndarray:
    """2x2 block [[eta T + eta' T', -(K + K')], [K + K', T/eta + T'/eta']]
    (Eq. (PMCHWT) and the Q_i^{ll}, Q_i^{ls}, Q_i^{sl}, Q_i^{ss} formulas of
    Section V-B) for family fam in {'A', 'H', 'T'} at lag k, with the family's
    truncation (A: k <= k_max, H: k <= k_max + 1, T: k <= k_max - 1)."""
    kmax = ops.kmax
    lim = {"A": kmax, "H": kmax + 1, "T": kmax - 1}[fam]
    ne = ops.ne
    if k > lim or k < 0:
        return np.zeros((2 * ne, 2 * ne))
    T = lag_dense_fast(ops.mats[fam + "T"], k, kmax - 1)
    Tp = lag_dense_fast(ops.mats[fam + "Tp"], k, kmax - 1)
    K = lag_dense_fast(ops.mats[fam + "K"], k, kmax - 1)
    Kp = lag_dense_fast(ops.mats[fam + "Kp"], k, kmax - 1)
    eta, etap = ops.eta, ops.etap
    return np.block([[eta * T + etap * Tp, -(K + Kp)], [K + Kp, T / eta + Tp / etap]])


def _bd(M):
    z = np.zeros_like(M)
    return np.block([[M, z], [z, M]])


@dataclass
class DenseSystem:
    ops: object
    P: dict
    M1: np.ndarray      # T^{Sigma H} G^{-1}
    M2: np.ndarray      # T^Lambda G^{-1} P^{Lambda H}
    Q: list             # Q_0 .. Q_{kmax+1}
    lu: tuple


def build_system(ops) -> DenseSystem:
    """Explicit dense Q_k (Section V-B):
      Q_k = T^{SH} G^-1 A_k P^{LH} + T^{SH} G^-1 A^_k P^S
          + T^L G^-1 P^{LH} A~_k P^{LH} + T^L G^-1 P^{LH} A_k P^S,
    with T^{SH} = P^{SH} T_0^s P^{SH}, T^L = P^L T_0^h P^L (Eq. (CP))."""
    mesh = ops.mesh
    Lam, Sig = incidence(mesh.ev, mesh.ef, mesh.nv, mesh.nf)
    P = projectors(Lam, Sig)
    Ginv = np.linalg.inv(ops.G.toarray())
    TSH = P["PSH"] @ ops.T0s @ P["PSH"]
    TL = P["PL"] @ ops.T0h @ P["PL"]
    M1 = TSH @ Ginv
    M2 = TL @ Ginv @ P["PLH"]
    M1b, M2b = _bd(M1), _bd(M2)
    PLHb, PSb = _bd(P["PLH"]), _bd(P["PS"])
    Q = []
    for k in range(ops.kmax + 2):
        XA = pmchwt_block(ops, "A", k)
        XH = pmchwt_block(ops, "H", k)
        XT = pmchwt_block(ops, "T", k)
        Qk = M1b @ XA @ PLHb + M1b @ XH @ PSb + M2b @ XT @ PLHb + M2b @ XA @ PSb
        Q.append(Qk)
    lu = sla.lu_factor(Q[0])
    return DenseSystem(ops, P, M1, M2, Q, lu)


# ---------------------------------------------------------------------------
# right-hand side (Section V-C, Eq. (rhs) and Eq. (hin))
# ---------------------------------------------------------------------------


def incident_integral(exc, b: int, x: np.ndarray, t: float, c: float = 1.0, eta: float = 1.0):
    """(d/dt^-1 e, d/dt^-1 h) at points x (n, 3), time t, for plane wave b of
    Eq. (hin): the time integral of the Gaussian is
    (A / (2c)) [1 + erf((4/w)(c (t - t0) - k.x))] p, saturating at (A/c) p."""
    A, p, k, w, t0 = exc.A[b], exc.p[b], exc.k[b], exc.w[b], exc.t0[b]
    arg = (4.0 / w) * (c * (t - t0) - x @ k)
    s = (A / (2.0 * c)) * (1.0 + erf(arg))
    E = s[:, None] * p[None, :]
    H = np.cross(k[None, :], E) / eta
    return E, H


def rhs_parts(ops, exc, b: int, i: int):
    """rho1_i = (1/dt) int p_i(t) (e, h)(t) dt and
    rho2_i = (1/T_max) (d/dt^-1 (e, h))(i dt), both tested with n x f_m:
    <n x f_m, a x n> = -<f_m, a>. rho2 is forced to zero after the pulse has
    passed (Section V-C, truncation of r^s)."""
    x = ops.rwg.x.reshape(-1, 3)
    wf = ops.rwg.wf
    ne = ops.ne
    dt = ops.dt
    E1, H1 = incident_integral(exc, b, x, i * dt)
    E0, H0 = incident_integral(exc, b, x, (i - 1) * dt)

    def test(F):
        return -np.einsum("eqd,eqd->e", wf, F.reshape(wf.shape))

    rho1 = np.concatenate([test(E1 - E0), test(H1 - H0)]) / dt
    if i * dt > exc.t_trunc[b]:
        rho2 = np.zeros(2 * ne)
    else:
        rho2 = np.concatenate([test(E1), test(H1)]) / ops.tmax
    return rho1, rho2


def rhs(sys_: DenseSystem, exc, b: int, i: int) -> np.ndarray:
    """r_i = r_i^l + r_i^s = T^{SH} G^-1 rho1_i + T^L G^-1 P^{LH} rho2_i (Eq. (rhs))."""
    rho1, rho2 = rhs_parts(sys_.ops, exc, b, i)
    return _bd(sys_.M1) @ rho1 + _bd(sys_.M2) @ rho2


# ---------------------------------------------------------------------------
# marching on in time (Eq. (MOT)) and current recovery (Eq. (dis_jm))
# ---------------------------------------------------------------------------


def march(sys_: DenseSystem, exc, n_steps: int, b: int = 0, solver: str = "lu", rhs_list=None):
    """w_i = Q_0^{-1} (r_i - sum_{k=1}^{i-1} Q_k w_{i-k}), i = 1..n_steps."""
    Q = sys_.Q
    K = len(Q) - 1
    W = []
    for i in range(1, n_steps + 1):
        r = rhs(sys_, exc, b, i) if rhs_list is None else rhs_list[i - 1]
        acc = r.copy()
        for k in range(1, min(i - 1, K) + 1):
            acc -= Q[k] @ W[i - k - 1]
        if solver == "lu":
            W.append(sla.lu_solve(sys_.lu, acc))
        else:
            W.append(gmres(lambda v: Q[0] @ v, acc, tol=1e-13, restart=400, maxiter=2000)[0])
    return np.array(W)


def recover(sys_: DenseSystem, W: np.ndarray):
    """Physical currents with loop and star parts kept apart (Eq. (dis_jm)):
    j_i = P^{LH} u_i + (T_max/dt) P^S (u_i - u_{i-1}); m_i likewise with v."""
    ops = sys_.ops
    ne = ops.ne
    P = sys_.P
    U = W[:, :ne]
    V = W[:, ne:]
    Up = np.vstack([np.zeros((1, ne)), U[:-1]])
    Vp = np.vstack([np.zeros((1, ne)), V[:-1]])
    s = ops.tmax / ops.dt
    return dict(j_loop=U @ P["PLH"].T, j_star=s * (U - Up) @ P["PS"].T,
                m_loop=V @ P["PLH"].T, m_star=s * (V - Vp) @ P["PS"].T)


# ---------------------------------------------------------------------------
# GMRES (for the Q_0 solve cross-check; Section V-A says GMRES solves Eq. (MOT))
# ---------------------------------------------------------------------------


def gmres(A, b: np.ndarray, tol: float = 1e-10, restart: int = 200, maxiter: int = 1000, x0=None):
    """Restarted GMRES with modified Gram-Schmidt Arnoldi and Givens rotations.
    Returns (x, iterations, relative residual)."""
    n = b.size
    x = np.zeros(n) if x0 is None else x0.copy()
    bn = np.linalg.norm(b)
    if bn == 0:
        return x, 0, 0.0
    it = 0
    while it < maxiter:
        r = b - A(x)
        beta = np.linalg.norm(r)
        if beta / bn <= tol:
            return x, it, beta / bn
        m = min(restart, maxiter - it)
        V = np.zeros((m + 1, n))
        H = np.zeros((m + 1, m))
        cs = np.zeros(m)
        sn = np.zeros(m)
        g = np.zeros(m + 1)
        g[0] = beta
        V[0] = r / beta
        j_end = 0
        for j in range(m):
            w = A(V[j])
            for i in range(j + 1):
                H[i, j] = V[i] @ w
                w = w - H[i, j] * V[i]
            H[j + 1, j] = np.linalg.norm(w)
            if H[j + 1, j] > 0:
                V[j + 1] = w / H[j + 1, j]
            for i in range(j):
                t = cs[i] * H[i, j] + sn[i] * H[i + 1, j]
                H[i + 1, j] = -sn[i] * H[i, j] + cs[i] * H[i + 1, j]
                H[i, j] = t
            d = math.hypot(H[j, j], H[j + 1, j])
            cs[j], sn[j] = H[j, j] / d, H[j + 1, j] / d
            H[j, j] = d
            H[j + 1, j] = 0.0
            g[j + 1] = -sn[j] * g[j]
            g[j] = cs[j] * g[j]
            it += 1
            j_end = j + 1
            if abs(g[j + 1]) / bn <= tol:
                break
        y = np.linalg.solve(np.triu(H[:j_end, :j_end]), g[:j_end])
        x = x + V[:j_end].T @ y
        if abs(g[j_end]) / bn <= tol:
            r = b - A(x)
            return x, it, np.linalg.norm(r) / bn
    r = b - A(x)
    return x, it, np.linalg.norm(r) / bn


# ---------------------------------------------------------------------------
# companion matrix (Section VI-A stability analysis)
# ---------------------------------------------------------------------------


def companion(sys_: DenseSystem) -> np.ndarray:
    """Companion matrix of the recursion w_i = -sum_k Q_0^{-1} Q_k w_{i-k}:
    first block row [-Q_0^{-1} Q_1, ..., -Q_0^{-1} Q_K], identity below."""
    Q = sys_.Q
    K = len(Q) - 1
    n = Q[0].shape[0]
    C = np.zeros((K * n, K * n))
    for k in range(1, K + 1):
        C[:n, (k - 1) * n:k * n] = -sla.lu_solve(sys_.lu, Q[k])
    for k in range(1, K):
        C[k * n:(k + 1) * n, (k - 1) * n:k * n] = np.eye(n)
    return C


def companion_top_eigenvalues(sys_: DenseSystem, k: int = 2, ncv: int = 300, tol: float = 1e-6) -> np.ndarray:
    """The k eigenvalues of largest magnitude of the same companion matrix
    (Section VI-A companion analysis) by Arnoldi on the operator applied
    without forming it: (x_1 .. x_K) -> (-sum_k Q_0^{-1} Q_k x_k, x_1 .. x_{K-1}),
    for meshes whose companion matrix is too large to decompose densely."""
    from scipy.sparse.linalg import LinearOperator, eigs
    Q = sys_.Q
    K = len(Q) - 1
    n = Q[0].shape[0]
    top = -sla.lu_solve(sys_.lu, np.concatenate(Q[1:], axis=1))  # first block row, n x K n

    def mv(x):
        y = np.empty_like(x)
        y[:n] = top @ x
        y[n:] = x[:-n]
        return y

    op = LinearOperator((K * n, K * n), matvec=mv, dtype=np.float64)
    return eigs(op, k=k, ncv=min(ncv, K * n - 1), which="LM", return_eigenvectors=False, tol=tol, maxiter=20000)
