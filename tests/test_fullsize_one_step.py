"""Parity at the bench's full size: torus 64 x 24 (4608 edges, 53 history
lags), 64 plane waves, the configuration bench.py times. The mixed path (the
tensor-core history) is compared with the FP64 path on the GPU for every wave
and element over steps 240-260, on the pulse, from a common state; both are
compared with the product-form FP64 oracle on sampled waves, one step computed
by the oracle from the GPU's own previous steps (a one-step check cannot
accumulate error, so it isolates the full-size step). The helper's step
alignment is checked on the CPU against the oracle's own march."""
import numpy as np
import pytest

from oracle import product as P
from paper_2510_07989_gb300.inputs import meshes as MS


def oracle_step_from_history(sysP, exc, b, i, history):
    """w_i of wave b by the product-form oracle (Eq. (MOT)) from
    history[j] = w_j for the steps j < i it reads (j >= i - K)."""
    ne = sysP.ne
    L = np.zeros((i + 1, 2 * ne))
    S = np.zeros((i + 1, 2 * ne))
    for j, w in history.items():
        assert 1 <= j < i
        L[j], S[j] = sysP.split(w)
    return sysP.step(exc, b, i, L, S)


def test_one_step_helper_reproduces_the_oracle_march(pr1_ops):
    """From the oracle's own steps i - K - 1 .. i - 1 the helper returns the
    oracle's step i (PR1, second of two waves, pulse inside the run)."""
    sysP = P.ProductSystem(pr1_ops)
    exc = MS.fibonacci_batch(2, pr1_ops.dt, w_steps=30, t0_steps=60)
    n, b = 70, 1
    W = sysP.march(exc, n, b=b)
    K = pr1_ops.kmax + 1
    hist = {j: W[j - 1] for j in range(max(1, n - K - 1), n)}
    w = oracle_step_from_history(sysP, exc, b, n, hist)
    assert np.abs(w - W[n - 1]).max() <= 1e-12 * np.abs(W).max()
    # a history shifted by one step (the plausible off-by-one) is detected
    shifted = {j: W[j - 2] for j in range(max(2, n - K - 1), n)}
    w2 = oracle_step_from_history(sysP, exc, b, n, shifted)
    assert np.abs(w2 - W[n - 1]).max() > 1e-3 * np.abs(W).max()


@pytest.mark.gpu
def test_bench_workload_parity():
    """The bench configuration at full size, on the pulse (steps 240-260 of the
    paper's pulse, t0 = 240 dt, every lag live):
      * mixed against FP64 on the GPU for all 64 waves and every element:
        both march steps 240-260 from the same state after step 239
        (mot_save_state of the mixed handle loaded into an FP64 handle); per
        wave, max over the steps of the 2-norm of the difference over the
        window's largest FP64 step norm <= 1e-6 (the metric of the readings:
        normalised by the run's peak); the loop-tested (u) and second (v)
        parts are reported apart;
      * each GPU path against the product-form FP64 oracle, one step (250) from
        that path's own history, for waves 0 and 63: FP64 <= 1e-10 and mixed
        <= 1e-6 of the step's norm. A one-step check cannot accumulate error,
        so it isolates the full-size step."""
    from paper_2510_07989_gb300.build import build
    build()
    import bench
    from paper_2510_07989_gb300 import mot as M
    ops, exc, _ = bench.make_workload("torus64x24")
    B = exc.B
    K = ops.kmax + 1
    i0, i1, ic = 240, 260, 250
    samples = (0, B - 1)
    waves = M.mot_waves(exc)
    out = np.zeros((B, 2, ops.ne))
    sm = M.Solver(ops, precision=M.MOT_PREC_MIXED)
    common = {b: {} for b in samples}  # steps read by the oracle's step ic that precede i0
    for j in range(1, i0):
        if j >= ic - K - 1:
            M.mot_step(sm.h, waves, B, out)
            for b in samples:
                common[b][j] = out[b].reshape(-1).copy()
        else:
            M.mot_step(sm.h, waves, B, None)
    assert M.mot_get_info(sm.h)["hist_kernel"] == 2  # tensor-core history, as in the bench
    state = M.mot_save_state(sm.h)
    sf = M.Solver(ops, precision=M.MOT_PREC_FP64, fp64_precond=1)
    M.mot_load_state(sf.h, state)
    Wm = np.zeros((i1 - i0 + 1, B, 2, ops.ne))
    Wf = np.zeros_like(Wm)
    for n in range(i1 - i0 + 1):
        M.mot_step(sm.h, waves, B, out)
        Wm[n] = out
        assert M.mot_step(sf.h, waves, B, out) == M.MOT_OK
        Wf[n] = out
    # per wave and per part (u: loop-tested, v: the second block row), the
    # metric of the readings: max over steps of |x_i - x_i^ref|_2 over the
    # largest |x_i^ref|_2 of the window (it holds the pulse's peak)
    def peak_rel(a, b):
        return np.linalg.norm(a - b, axis=-1).max(axis=0) / np.linalg.norm(b, axis=-1).max(axis=0)
    err = peak_rel(Wm.reshape(i1 - i0 + 1, B, -1), Wf.reshape(i1 - i0 + 1, B, -1))
    eu, ev = peak_rel(Wm[:, :, 0], Wf[:, :, 0]), peak_rel(Wm[:, :, 1], Wf[:, :, 1])
    elem = (np.abs(Wm - Wf).max(axis=(0, 2, 3)) / np.abs(Wf).max(axis=(0, 2, 3))).max()
    print(f"torus64x24 steps {i0}-{i1}, mixed vs FP64 GPU, 64 waves: max {err.max():.3e} (wave {err.argmax()}); "
          f"u {eu.max():.3e}, v {ev.max():.3e}; largest element error / largest element {elem:.3e}")
    assert err.max() <= 1e-6
    # one oracle step from each path's own history
    hist = {"mixed": {b: dict(common[b]) for b in samples}, "fp64": {b: dict(common[b]) for b in samples}}
    for name, W in (("mixed", Wm), ("fp64", Wf)):
        for n in range(i1 - i0 + 1):
            for b in samples:
                hist[name][b][i0 + n] = W[n, b].reshape(-1).copy()
    sysP = P.ProductSystem(ops)
    for name, tol in (("fp64", 1e-10), ("mixed", 1e-6)):
        for b in samples:
            # steps before i0 come from the common mixed march (the FP64 handle's ring holds them too)
            h = {j: w for j, w in hist[name][b].items() if ic - K - 1 <= j < ic}
            assert len(h) == K + 1
            w_ref = oracle_step_from_history(sysP, exc, b, ic, h)
            e = np.linalg.norm(hist[name][b][ic] - w_ref) / np.linalg.norm(w_ref)
            print(f"torus64x24 {name} wave {b} step {ic}: |w_gpu - w_oracle| / |w_oracle| = {e:.3e}")
            assert e <= tol
