"""Driver of the CPU FP64 operator assembly (input generator shared by the CUDA
path and the oracle).

Produces, for a closed mesh, material (eps_r, mu_r) and time step dt:
  * the 12 lagged interaction families of paper Section V-B, per medium
    (exterior '', interior 'p'): A.T, A.K (h_0 basis), Ah.T, Ah.K (T_max d/dt of
    q_0), At.T, At.K ((1/T_max) d/dt^-1 of p_0). Each is a lag-window CSR matrix:
    row m, entries (n, first lag k0, window length cnt, values). At.K also has a
    constant tail per entry (value tc from lag ta on, up to lag k_max - 1).
  * the static BC-space operators T_0^s, T_0^h (dense) and the mixed Gram
    matrix G (sparse) of Section III;
  * quadrature tables of the RWG (and BC) functions for right-hand sides, far
    fields and the exact-solution projection.
"""
from __future__ import annotations

import ctypes
import math
import os
import subprocess
from dataclasses import dataclass, field

import numpy as np
import scipy.sparse as sp

from .dual import BCTable, DualBasis, RWGTable, bc_table, dual_basis, gram_matrix, rwg_table
from .meshes import Mesh, diameter

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "asm.c")
_LIB = os.path.join(_HERE, "_libasm.so")

KINDS = ["AT", "AK", "HT", "HK", "TT", "TK"]   # per medium, order of the C enum
FAMILY_MAX_LAG = {"A": 0, "H": 1, "T": -1}      # relative to k_max


def build_host_library(force: bool = False) -> str:
    """Compile the host assembler (plain C + pthreads)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O3", "-fPIC", "-shared", "-o", tmp, _SRC, "-lpthread", "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


_lib = None


def _load():
    global _lib
    if _lib is None:
        _lib = ctypes.CDLL(build_host_library())
        _lib.asm_td_run.restype = ctypes.c_void_p
        _lib.asm_td_run.argtypes = [ctypes.c_int, ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p, ctypes.c_int,
                                    ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_double,
                                    ctypes.c_double, ctypes.c_double, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                    ctypes.c_int, ctypes.c_int, ctypes.c_int]
        _lib.asm_td_sizes.argtypes = [ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p]
        _lib.asm_td_copy.argtypes = [ctypes.c_void_p, ctypes.c_int] + [ctypes.c_void_p] * 8
        _lib.asm_td_free.argtypes = [ctypes.c_void_p]
        _lib.asm_time_weights.argtypes = [ctypes.c_double, ctypes.c_void_p]
        _lib.asm_time_weights.restype = None
        _lib.asm_static.restype = ctypes.c_int
        _lib.asm_static.argtypes = ([ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p,
                                     ctypes.c_int, ctypes.c_void_p] + [ctypes.c_void_p] * 6 +
                                    [ctypes.c_double, ctypes.c_double, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                     ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p])
    return _lib


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


@dataclass
class LagMat:
    """Lag-window CSR: for row m, entries e in [rowptr[m], rowptr[m+1]) hold
    column col[e] and values val[voff[e] : voff[e] + cnt[e]] for lags
    k0[e] .. k0[e] + cnt[e] - 1. Optional constant tail tc[e] for lags
    ta[e] .. kmax - 1."""
    ne: int
    rowptr: np.ndarray
    col: np.ndarray
    k0: np.ndarray
    cnt: np.ndarray
    voff: np.ndarray
    val: np.ndarray
    ta: np.ndarray | None = None
    tc: np.ndarray | None = None

    @property
    def nbytes(self) -> int:
        return int(sum(a.nbytes for a in (self.rowptr, self.col, self.k0, self.cnt, self.voff, self.val)))

    def max_lag(self) -> int:
        if self.col.size == 0:
            return -1
        return int((self.k0 + self.cnt - 1).max())


@dataclass
class Operators:
    mesh: Mesh
    eps_r: float
    mu_r: float
    dt: float
    c: float
    cp: float
    eta: float
    etap: float
    D: float
    tmax: float
    kmax: int
    mats: dict               # name -> LagMat, names KINDS (exterior) and KINDS+'p' (interior)
    T0s: np.ndarray
    T0h: np.ndarray
    G: sp.csr_matrix
    rwg: RWGTable
    dual: DualBasis | None = None
    bc: BCTable | None = None
    meta: dict = field(default_factory=dict)

    @property
    def ne(self) -> int:
        return self.mesh.ne

    @property
    def K(self) -> int:
        """Number of history lags: Q_k vanishes for k > k_max + 1."""
        return self.kmax + 1


def time_weights(phi: float) -> np.ndarray:
    """The assembler's temporal factors for R / (c dt) = j + phi (asm_time_weights):
    [dt h_0'(lags j, j+1), dt^2 q_0''(lags j..j+2), q_0(lags j..j+2), p_0(lag j),
     h_0(lags j, j+1), dt q_0'(lags j..j+2), ramp int p_0 / dt (lags j, j+1)]."""
    w = np.zeros(16)
    _load().asm_time_weights(float(phi), w.ctypes.data_as(ctypes.c_void_p))
    return w


def k_max_of(tmax: float, dt: float) -> int:
    """k_max = ceil(T_max / dt), with T_max/dt within 1e-12 of an integer taken as that integer."""
    r = tmax / dt
    n = round(r)
    if abs(r - n) < 1e-12 * max(1.0, r):
        return int(n)
    return int(math.ceil(r))


def _run_medium(mesh: Mesh, c: float, dt: float, tmax: float, kmax: int, nq: int, ntheta: int, nrad: int,
                nthreads: int, far_plain: int = 0) -> dict:
    lib = _load()
    V = np.ascontiguousarray(mesh.verts, dtype=np.float64)
    F = np.ascontiguousarray(mesh.tris, dtype=np.int32)
    EV = np.ascontiguousarray(mesh.ev, dtype=np.int32)
    EF = np.ascontiguousarray(mesh.ef, dtype=np.int32)
    EO = np.ascontiguousarray(mesh.eo, dtype=np.int32)
    h = lib.asm_td_run(mesh.nv, _ptr(V), mesh.nf, _ptr(F), mesh.ne, _ptr(EV), _ptr(EF), _ptr(EO),
                       c, dt, tmax, kmax, nq, ntheta, nrad, nthreads, far_plain)
    out = {}
    try:
        for kind, name in enumerate(KINDS):
            nent = ctypes.c_int64()
            nval = ctypes.c_int64()
            lib.asm_td_sizes(h, kind, ctypes.byref(nent), ctypes.byref(nval))
            rowptr = np.zeros(mesh.ne + 1, dtype=np.int64)
            col = np.zeros(nent.value, dtype=np.int32)
            k0 = np.zeros(nent.value, dtype=np.int32)
            cnt = np.zeros(nent.value, dtype=np.int32)
            voff = np.zeros(nent.value, dtype=np.int64)
            val = np.zeros(nval.value, dtype=np.float64)
            ta = tc = None
            if name == "TK":
                ta = np.zeros(nent.value, dtype=np.int32)
                tc = np.zeros(nent.value, dtype=np.float64)
            lib.asm_td_copy(h, kind, _ptr(rowptr), _ptr(col), _ptr(k0), _ptr(cnt), _ptr(voff), _ptr(val),
                            _ptr(ta) if ta is not None else None, _ptr(tc) if tc is not None else None)
            out[name] = LagMat(mesh.ne, rowptr, col, k0, cnt, voff, val, ta, tc)
    finally:
        lib.asm_td_free(h)
    return out


def _static(mesh: Mesh, dual: DualBasis, D: float, nq: int, ntheta: int, nrad: int, nthreads: int,
            kappa: float = 0.0):
    """T_0^s and T_0^h of the static EFIO on the BC dual basis (Section IV-A);
    kappa > 0: those of the EFIO with the imaginary wavenumber -i kappa
    (kernel exp(-kappa R) / (4 pi R), same normalisation)."""
    lib = _load()
    nref = dual.nref
    order = np.argsort(dual.bc_t, kind="stable")
    bt = dual.bc_t[order]
    bptr = np.zeros(nref + 1, dtype=np.int64)
    np.add.at(bptr, bt + 1, 1)
    bptr = np.cumsum(bptr).astype(np.int64)
    bn = np.ascontiguousarray(dual.bc_n[order], dtype=np.int32)
    ba = np.ascontiguousarray(dual.bc_alpha[order], dtype=np.float64)
    bb = np.ascontiguousarray(dual.bc_beta[order], dtype=np.float64)
    corder = np.argsort(dual.ref_vert, kind="stable")
    cptr = np.zeros(mesh.nv + 1, dtype=np.int64)
    np.add.at(cptr, dual.ref_vert + 1, 1)
    cptr = np.cumsum(cptr).astype(np.int64)
    ctri = np.ascontiguousarray(corder, dtype=np.int32)
    pts = np.ascontiguousarray(dual.ref_pts, dtype=np.float64)
    rvert = np.ascontiguousarray(dual.ref_vert, dtype=np.int32)
    deg = np.ascontiguousarray(dual.degree, dtype=np.int32)
    ev = np.ascontiguousarray(mesh.ev, dtype=np.int32)
    T0s = np.zeros((mesh.ne, mesh.ne))
    S = np.zeros((mesh.nv, mesh.nv))
    lib.asm_static(nref, _ptr(pts), _ptr(rvert), mesh.nv, _ptr(deg), mesh.ne, _ptr(ev), _ptr(bptr), _ptr(bn),
                   _ptr(ba), _ptr(bb), _ptr(cptr), _ptr(ctri), D, float(kappa), nq, ntheta, nrad, nthreads,
                   _ptr(T0s), _ptr(S))
    T0s = 0.5 * (T0s + T0s.T)
    S = 0.5 * (S + S.T)
    ne = mesh.ne
    Lam = sp.csr_matrix((np.concatenate([np.ones(ne), -np.ones(ne)]),
                         (np.concatenate([np.arange(ne)] * 2), np.concatenate([mesh.ev[:, 1], mesh.ev[:, 0]]))),
                        shape=(ne, mesh.nv))
    T0h = np.asarray((Lam @ (Lam @ S).T).T)
    T0h = 0.5 * (T0h + T0h.T)
    return T0s, T0h


def assemble(mesh: Mesh, eps_r: float, mu_r: float, dt: float, *, nq: int = 7, ntheta: int = 4, nrad: int = 4,
             nq_static: int = 3, nthreads: int | None = None, with_bc_table: bool = False,
             kmax: int | None = None, far_plain: int = 0, kappa: float = 0.0) -> Operators:
    """Assemble every input of the MOT step for one scatterer (c = 1 outside).

    nq is the outer (test) triangle rule; ntheta / nrad the Gauss orders of the
    polar inner integration per smooth piece. far_plain > 0 replaces the
    shell-split polar rule by a plain far_plain-point triangle rule for source
    triangles farther than three diameters (fast, less accurate assembly).
    kappa > 0 builds the Calderon preconditioner from the EFIO T_{-i kappa}
    (imaginary wavenumber) instead of the static T_0 (Section IV-A remark)."""
    if kappa < 0:
        raise ValueError("kappa must be >= 0")
    if nthreads is None:
        nthreads = os.cpu_count() or 1
    c = 1.0
    eta = 1.0
    cp = 1.0 / math.sqrt(eps_r * mu_r)
    etap = math.sqrt(mu_r / eps_r)
    D = diameter(mesh)
    tmax = D / min(c, cp)
    if kmax is None:
        kmax = k_max_of(tmax, dt)
    mats = {}
    for suffix, cc in (("", c), ("p", cp)):
        res = _run_medium(mesh, cc, dt, tmax, kmax, nq, ntheta, nrad, nthreads, far_plain)
        for name, m in res.items():
            mats[name + suffix] = m
    dual = dual_basis(mesh)
    T0s, T0h = _static(mesh, dual, D, nq_static, ntheta, nrad, nthreads, kappa)
    r, cidx, v = gram_matrix(mesh, dual)
    G = sp.coo_matrix((v, (r, cidx)), shape=(mesh.ne, mesh.ne)).tocsr()
    G.sum_duplicates()
    ops = Operators(mesh=mesh, eps_r=eps_r, mu_r=mu_r, dt=dt, c=c, cp=cp, eta=eta, etap=etap, D=D, tmax=tmax,
                    kmax=kmax, mats=mats, T0s=T0s, T0h=T0h, G=G, rwg=rwg_table(mesh, 7), dual=dual,
                    bc=bc_table(dual) if with_bc_table else None,
                    meta=dict(nq=nq, ntheta=ntheta, nrad=nrad, nq_static=nq_static, far_plain=far_plain,
                              kappa=kappa))
    return ops
