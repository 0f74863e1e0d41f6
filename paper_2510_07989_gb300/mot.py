"""Python binding of libmot.so (argument marshalling only; every step of the
MOT path runs in the library's CUDA kernels). Function names follow the C ABI
declared in include/mot.h.

Arrays may be numpy arrays (host) or torch CUDA tensors (device); streams are
torch.cuda.Stream objects, raw cudaStream_t integers, or None.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libmot.so")

MOT_OK, MOT_EINVAL, MOT_EOOM, MOT_ENOCONV, MOT_ECUDA, MOT_ESTATE = 0, -1, -2, -3, -4, -5
MOT_PREC_FP64, MOT_PREC_MIXED = 0, 1
MOT_MIX_HIST32, MOT_MIX_LF32, MOT_MIX_Q032, MOT_MIX_REFINE, MOT_MIX_PRECOND = 1, 2, 4, 8, 16
MOT_MIX_TC, MOT_MIX_EMU64, MOT_MIX_TCBULK = 32, 64, 128
MOT_MIX_DEFAULT = MOT_MIX_HIST32 | MOT_MIX_Q032 | MOT_MIX_REFINE | MOT_MIX_PRECOND | MOT_MIX_TC | MOT_MIX_EMU64
_NAMES = {0: "MOT_OK", -1: "MOT_EINVAL", -2: "MOT_EOOM", -3: "MOT_ENOCONV", -4: "MOT_ECUDA", -5: "MOT_ESTATE"}


class MotError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"{_NAMES.get(code, code)}: {msg}")
        self.code = code


class mot_mesh(ctypes.Structure):
    _fields_ = [("nv", ctypes.c_int32), ("verts", ctypes.c_void_p), ("nf", ctypes.c_int32), ("tris", ctypes.c_void_p)]


class mot_options(ctypes.Structure):
    _fields_ = [("precision", ctypes.c_int32), ("device", ctypes.c_int32), ("gmres_tol", ctypes.c_double),
                ("gmres_maxit", ctypes.c_int32), ("cg_tol", ctypes.c_double), ("cg_maxit", ctypes.c_int32),
                ("timing", ctypes.c_int32), ("mixed_flags", ctypes.c_int32), ("refine_sweeps", ctypes.c_int32),
                ("fp64_precond", ctypes.c_int32), ("hist_stall_test", ctypes.c_int32),
                ("fp64_direct", ctypes.c_int32)]


class mot_lagmat(ctypes.Structure):
    _fields_ = [("nent", ctypes.c_int64), ("rowptr", ctypes.c_void_p), ("col", ctypes.c_void_p),
                ("k0", ctypes.c_void_p), ("cnt", ctypes.c_void_p), ("voff", ctypes.c_void_p),
                ("val", ctypes.c_void_p), ("tail_lag", ctypes.c_void_p), ("tail_val", ctypes.c_void_p)]


class mot_operators(ctypes.Structure):
    _fields_ = [("mat", mot_lagmat * 12), ("T0s", ctypes.c_void_p), ("T0h", ctypes.c_void_p),
                ("g_rowptr", ctypes.c_void_p), ("g_col", ctypes.c_void_p), ("g_val", ctypes.c_void_p),
                ("nq", ctypes.c_int32), ("rhs_x", ctypes.c_void_p), ("rhs_wf", ctypes.c_void_p)]


class mot_wave(ctypes.Structure):
    _fields_ = [("A", ctypes.c_double), ("p", ctypes.c_double * 3), ("k", ctypes.c_double * 3),
                ("w", ctypes.c_double), ("t0", ctypes.c_double), ("t_trunc", ctypes.c_double)]


class mot_info(ctypes.Structure):
    _fields_ = [("ne", ctypes.c_int32), ("nv", ctypes.c_int32), ("nf", ctypes.c_int32), ("kmax", ctypes.c_int32),
                ("K", ctypes.c_int32), ("B", ctypes.c_int32), ("step", ctypes.c_int64), ("D", ctypes.c_double),
                ("tmax", ctypes.c_double), ("dt", ctypes.c_double), ("last_gmres_iters", ctypes.c_int32),
                ("last_gmres_resid", ctypes.c_double), ("last_cg_iters", ctypes.c_int32),
                ("device_bytes", ctypes.c_int64), ("gpu_launches", ctypes.c_int64), ("tile_fill", ctypes.c_double),
                ("tile_count", ctypes.c_int64), ("hist_flops_per_step", ctypes.c_double),
                ("hist_bytes_per_step", ctypes.c_double), ("hist_timed_launches", ctypes.c_int64),
                ("hist_timed_ms", ctypes.c_double), ("phase_ms", ctypes.c_double * 8),
                ("hist_kernel", ctypes.c_int32), ("hist_tc_tasks", ctypes.c_int64),
                ("gmres_iters_total", ctypes.c_int64), ("tc_chunk_cap", ctypes.c_int32),
                ("tc_lag_frac", ctypes.c_double), ("tc_stages", ctypes.c_int32), ("tc_tuned", ctypes.c_int32),
                ("tc_tune_ms", ctypes.c_double), ("tc_launches", ctypes.c_int64),
                ("tc_epilogue_warps", ctypes.c_int32), ("tc_tasks_per_stage", ctypes.c_int32)]

    def as_dict(self):
        d = {k: getattr(self, k) for k, _ in self._fields_}
        d["phase_ms"] = list(d["phase_ms"])
        return d


EXPORTED = ["mot_create", "mot_load_operators", "mot_set_frequencies", "mot_step", "mot_run", "mot_run_many",
            "mot_tune", "mot_set_tc_config", "mot_get_currents",
            "mot_fields", "mot_fields_noalloc", "mot_reset", "mot_save_state", "mot_load_state", "mot_get_info",
            "mot_get_edges", "mot_last_error", "mot_destroy"]

_lib = None


def load_library(path: str = LIB_PATH):
    """Load libmot.so; raises if it has not been built (there is no fallback)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError(f"{path} is missing: build it with __graft_entry__.build() "
                           "(the MOT path has no CPU fallback)")
    lib = ctypes.CDLL(path)
    vp, i32, dbl = ctypes.c_void_p, ctypes.c_int, ctypes.c_double
    lib.mot_create.argtypes = [ctypes.POINTER(mot_mesh), dbl, dbl, dbl, i32, ctypes.POINTER(mot_options),
                               ctypes.POINTER(vp)]
    lib.mot_load_operators.argtypes = [vp, ctypes.POINTER(mot_operators)]
    lib.mot_set_frequencies.argtypes = [vp, i32, vp]
    lib.mot_step.argtypes = [vp, vp, i32, vp, vp]
    lib.mot_run.argtypes = [vp, i32, vp, i32, vp, vp]
    lib.mot_run_many.argtypes = [vp, i32, i32, vp, vp, vp, vp]
    lib.mot_tune.argtypes = [vp, i32, vp]
    lib.mot_set_tc_config.argtypes = [vp, i32, dbl, i32, i32, i32]
    lib.mot_get_currents.argtypes = [vp, vp]
    lib.mot_fields.argtypes = [vp, vp, i32, vp, vp]
    lib.mot_fields_noalloc.argtypes = [vp, vp, i32, vp, vp]
    lib.mot_reset.argtypes = [vp]
    lib.mot_save_state.argtypes = [vp, vp, ctypes.POINTER(ctypes.c_size_t)]
    lib.mot_load_state.argtypes = [vp, vp, ctypes.c_size_t]
    lib.mot_get_info.argtypes = [vp, ctypes.POINTER(mot_info)]
    lib.mot_get_edges.argtypes = [vp, vp, vp]
    lib.mot_last_error.argtypes = [vp]
    lib.mot_last_error.restype = ctypes.c_char_p
    lib.mot_destroy.argtypes = [vp]
    lib.mot_destroy.restype = None
    for name in EXPORTED:
        if name not in ("mot_last_error", "mot_destroy"):
            getattr(lib, name).restype = ctypes.c_int
    _lib = lib
    return lib


def _ptr(a):
    """Raw pointer of a numpy array or torch tensor (None -> NULL)."""
    if a is None:
        return None
    if isinstance(a, np.ndarray):
        return a.ctypes.data
    return a.data_ptr()


def _stream(s):
    if s is None:
        return None
    if isinstance(s, int):
        return s
    return s.cuda_stream


def _check(h, code, allow_noconv=False):
    if code == MOT_OK or (allow_noconv and code == MOT_ENOCONV):
        return code
    msg = load_library().mot_last_error(h).decode() if h else ""
    raise MotError(code, msg)


def _c(a, dtype):
    return np.ascontiguousarray(a, dtype=dtype)


def mot_waves(exc) -> ctypes.Array:
    """mot_wave[B] from an Excitation (inputs.meshes.Excitation)."""
    arr = (mot_wave * exc.B)()
    for b in range(exc.B):
        arr[b].A = float(exc.A[b])
        for d in range(3):
            arr[b].p[d] = float(exc.p[b, d])
            arr[b].k[d] = float(exc.k[b, d])
        arr[b].w = float(exc.w[b])
        arr[b].t0 = float(exc.t0[b])
        arr[b].t_trunc = float(exc.t_trunc[b])
    return arr


class Handle:
    """Owner of a mot_handle* and of the host arrays passed to the library."""

    def __init__(self, ptr):
        self.ptr = ptr
        self._keep = []

    def __del__(self):
        try:
            mot_destroy(self)
        except Exception:
            pass


def mot_create(verts, tris, eps_r, mu_r, dt, K, precision=MOT_PREC_FP64, device=0, gmres_tol=0.0,
               gmres_maxit=200, cg_tol=1e-14, cg_maxit=5000, timing=0, mixed_flags=0, refine_sweeps=0,
               fp64_precond=0, hist_stall_test=0, fp64_direct=0) -> Handle:
    """gmres_tol <= 0 selects the library default (1e-13 FP64, 1e-11 mixed)."""
    lib = load_library()
    V = _c(verts, np.float64)
    Tr = _c(tris, np.int32)
    mesh = mot_mesh(V.shape[0], V.ctypes.data, Tr.shape[0], Tr.ctypes.data)
    opt = mot_options(precision, device, gmres_tol, gmres_maxit, cg_tol, cg_maxit, int(timing), int(mixed_flags),
                      int(refine_sweeps), int(fp64_precond), int(hist_stall_test), int(fp64_direct))
    out = ctypes.c_void_p()
    code = lib.mot_create(ctypes.byref(mesh), float(eps_r), float(mu_r), float(dt), int(K), ctypes.byref(opt),
                          ctypes.byref(out))
    if code != MOT_OK:
        msg = lib.mot_last_error(out).decode() if out.value else ""
        if out.value:
            lib.mot_destroy(out)
        raise MotError(code, msg)
    return Handle(out)


def mot_load_operators(h: Handle, ops) -> None:
    """ops: inputs.assemble.Operators."""
    from .inputs.assemble import KINDS
    o = mot_operators()
    keep = []
    names = KINDS + [k + "p" for k in KINDS]
    for i, name in enumerate(names):
        m = ops.mats[name]
        arrs = [_c(m.rowptr, np.int64), _c(m.col, np.int32), _c(m.k0, np.int32), _c(m.cnt, np.int32),
                _c(m.voff, np.int64), _c(m.val, np.float64)]
        keep += arrs
        lm = mot_lagmat(int(m.col.size), *[a.ctypes.data for a in arrs], None, None)
        if m.ta is not None:
            ta, tc = _c(m.ta, np.int32), _c(m.tc, np.float64)
            keep += [ta, tc]
            lm.tail_lag = ta.ctypes.data
            lm.tail_val = tc.ctypes.data
        o.mat[i] = lm
    T0s, T0h = _c(ops.T0s, np.float64), _c(ops.T0h, np.float64)
    G = ops.G.tocsr()
    grp, gcol, gval = _c(G.indptr, np.int64), _c(G.indices, np.int32), _c(G.data, np.float64)
    rx = _c(ops.rwg.x, np.float64)
    rw = _c(ops.rwg.wf, np.float64)
    keep += [T0s, T0h, grp, gcol, gval, rx, rw]
    o.T0s, o.T0h = T0s.ctypes.data, T0h.ctypes.data
    o.g_rowptr, o.g_col, o.g_val = grp.ctypes.data, gcol.ctypes.data, gval.ctypes.data
    o.nq = rx.shape[1]
    o.rhs_x, o.rhs_wf = rx.ctypes.data, rw.ctypes.data
    _check(h.ptr, load_library().mot_load_operators(h.ptr, ctypes.byref(o)))


def mot_set_frequencies(h: Handle, omega) -> None:
    w = _c(omega, np.float64)
    _check(h.ptr, load_library().mot_set_frequencies(h.ptr, int(w.size), w.ctypes.data if w.size else None))


def mot_step(h: Handle, waves, B: int, w_out=None, stream=None) -> int:
    """One MOT step; w_out (numpy or torch CUDA, [B][2][ne] float64) or None.
    Returns MOT_OK or MOT_ENOCONV; raises on other errors."""
    return _check(h.ptr, load_library().mot_step(h.ptr, ctypes.cast(waves, ctypes.c_void_p), int(B), _ptr(w_out),
                                                 _stream(stream)), allow_noconv=True)


def mot_run(h: Handle, n_steps: int, waves, B: int, w_out=None, stream=None) -> int:
    return _check(h.ptr, load_library().mot_run(h.ptr, int(n_steps), ctypes.cast(waves, ctypes.c_void_p), int(B),
                                                _ptr(w_out), _stream(stream)), allow_noconv=True)


def mot_run_many(handles, n_steps: int, waves_list, B_list, w_out_list=None, stream=None) -> int:
    """mot_run_many: march len(handles) scatterers n_steps each, concurrently.
    waves_list[i] is a mot_wave array of B_list[i] waves; w_out_list (None, or
    one array or None per handle, [n_steps][B][2][ne] float64, numpy or torch
    CUDA) receives the steps. Returns MOT_OK or MOT_ENOCONV; raises on other
    errors with the messages of the handles that report one."""
    n = len(handles)
    lib = load_library()
    hs = (ctypes.c_void_p * max(n, 1))(*[h.ptr for h in handles])
    wv = (ctypes.c_void_p * max(n, 1))(*[ctypes.cast(w, ctypes.c_void_p).value for w in waves_list])
    bs = (ctypes.c_int * max(n, 1))(*[int(b) for b in B_list])
    outs = None
    if w_out_list is not None:
        outs = (ctypes.c_void_p * max(n, 1))(*[_ptr(o) for o in w_out_list])
    code = lib.mot_run_many(hs if n else None, n, int(n_steps), wv if n else None, bs if n else None, outs,
                            _stream(stream))
    if code in (MOT_OK, MOT_ENOCONV):
        return code
    msgs = [f"[{i}] {lib.mot_last_error(h.ptr).decode()}" for i, h in enumerate(handles)
            if lib.mot_last_error(h.ptr)]
    raise MotError(code, "; ".join(msgs))


def mot_tune(handles, stream=None) -> None:
    """mot_tune: pick, by timing, the tensor-core history configuration of
    the handles marched together (one handle: alone)."""
    n = len(handles)
    lib = load_library()
    hs = (ctypes.c_void_p * max(n, 1))(*[h.ptr for h in handles])
    _check(handles[0].ptr if n else None, lib.mot_tune(hs, n, _stream(stream)))


def mot_set_tc_config(h: Handle, cap: int, lag_frac: float, stages: int, tasks_per_stage: int,
                      epilogue_warps: int) -> None:
    """mot_set_tc_config: apply one tensor-core history configuration as given."""
    _check(h.ptr, load_library().mot_set_tc_config(h.ptr, int(cap), float(lag_frac), int(stages),
                                                   int(tasks_per_stage), int(epilogue_warps)))


def mot_get_currents(h: Handle, out) -> None:
    _check(h.ptr, load_library().mot_get_currents(h.ptr, _ptr(out)))


def mot_fields(h: Handle, waves, dirs, n_freq: int, B: int) -> np.ndarray:
    d = _c(dirs, np.float64).reshape(-1, 3)
    out = np.zeros((B, n_freq, d.shape[0], 3, 2))
    _check(h.ptr, load_library().mot_fields(h.ptr, ctypes.cast(waves, ctypes.c_void_p), d.shape[0], d.ctypes.data,
                                            out.ctypes.data))
    return out[..., 0] + 1j * out[..., 1]


def mot_fields_noalloc(h: Handle, waves, dirs, n_freq: int, B: int) -> np.ndarray:
    """Same result as mot_fields without any device allocation in the call: the
    library stages directions and result in a fixed 2 MiB device array (for
    callers that must not call cudaMalloc at this point). Calls must not
    overlap on the GPU; 3*n_dir + 6*B*n_freq*n_dir <= 262144."""
    d = _c(dirs, np.float64).reshape(-1, 3)
    out = np.zeros((B, n_freq, d.shape[0], 3, 2))
    _check(h.ptr, load_library().mot_fields_noalloc(h.ptr, ctypes.cast(waves, ctypes.c_void_p), d.shape[0],
                                                    d.ctypes.data, out.ctypes.data))
    return out[..., 0] + 1j * out[..., 1]


def mot_reset(h: Handle) -> None:
    _check(h.ptr, load_library().mot_reset(h.ptr))


def mot_save_state(h: Handle) -> bytes:
    lib = load_library()
    n = ctypes.c_size_t(0)
    _check(h.ptr, lib.mot_save_state(h.ptr, None, ctypes.byref(n)))
    buf = ctypes.create_string_buffer(n.value)
    _check(h.ptr, lib.mot_save_state(h.ptr, buf, ctypes.byref(n)))
    return buf.raw[:n.value]


def mot_load_state(h: Handle, blob: bytes) -> None:
    buf = ctypes.create_string_buffer(blob, len(blob))
    _check(h.ptr, load_library().mot_load_state(h.ptr, buf, len(blob)))


def mot_get_info(h: Handle) -> dict:
    info = mot_info()
    _check(h.ptr, load_library().mot_get_info(h.ptr, ctypes.byref(info)))
    return info.as_dict()


def mot_get_edges(h: Handle):
    ne = mot_get_info(h)["ne"]
    ev = np.zeros((ne, 2), dtype=np.int32)
    ef = np.zeros((ne, 2), dtype=np.int32)
    _check(h.ptr, load_library().mot_get_edges(h.ptr, ev.ctypes.data, ef.ctypes.data))
    return ev, ef


def mot_last_error(h: Handle) -> str:
    return load_library().mot_last_error(h.ptr).decode()


def mot_destroy(h: Handle) -> None:
    if h.ptr is not None and h.ptr.value:
        load_library().mot_destroy(h.ptr)
        h.ptr = ctypes.c_void_p()


# ----------------------------------------------------------------------------
# convenience wrapper
# ----------------------------------------------------------------------------


class Solver:
    """mot_create + mot_load_operators for an assembled Operators object."""

    def __init__(self, ops, **kw):
        self.ops = ops
        mesh = ops.mesh
        self.h = mot_create(mesh.verts, mesh.tris, ops.eps_r, ops.mu_r, ops.dt, ops.kmax + 1, **kw)
        mot_load_operators(self.h, ops)
        self.ne = mesh.ne
        self.noconv = 0  # steps that returned MOT_ENOCONV (a GMRES or CG iteration limit)

    def run(self, exc, n_steps: int, keep: bool = True):
        """March n_steps for the excitation batch; returns W [n_steps][B][2][ne] (host)."""
        waves = mot_waves(exc)
        B = exc.B
        W = np.zeros((n_steps, B, 2, self.ne)) if keep else None
        out = np.zeros((B, 2, self.ne))
        for i in range(n_steps):
            if mot_step(self.h, waves, B, out if keep else None) == MOT_ENOCONV:
                self.noconv += 1
            if keep:
                W[i] = out
        return W

    def info(self):
        return mot_get_info(self.h)
