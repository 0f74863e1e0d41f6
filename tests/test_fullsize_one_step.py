"""Parity at the bench's full size, on sampled outputs the oracle computes one
by one: torus 64 x 24 (4608 edges, 53 history lags), mixed path, B = 64 on the
tensor-core history -- the configuration bench.py times. The GPU marches to
step 250 (near the pulse peak, every lag live); for sampled waves the
product-form FP64 oracle computes that step from the GPU's own previous
steps, and the GPU's step must agree to 1e-6 of its norm. A one-step check
cannot accumulate error, so it isolates the full-size step. The helper's step
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
def test_bench_workload_one_step_parity():
    from paper_2510_07989_gb300.build import build
    build()
    import bench
    from paper_2510_07989_gb300 import mot as M
    ops, exc, _ = bench.make_workload("torus64x24")
    K = ops.kmax + 1
    i = 250
    samples = (0, 41)
    s = M.Solver(ops, precision=M.MOT_PREC_MIXED)
    waves = M.mot_waves(exc)
    out = np.zeros((exc.B, 2, ops.ne))
    hist = {b: {} for b in samples}
    for j in range(1, i + 1):
        M.mot_step(s.h, waves, exc.B, out)
        if j >= i - K - 1:
            for b in samples:
                hist[b][j] = out[b].reshape(-1).copy()
    assert M.mot_get_info(s.h)["hist_kernel"] == 2  # tensor-core history, as in the bench
    sysP = P.ProductSystem(ops)
    for b in samples:
        w_gpu = hist[b].pop(i)
        w_ref = oracle_step_from_history(sysP, exc, b, i, hist[b])
        err = np.linalg.norm(w_gpu - w_ref) / np.linalg.norm(w_ref)
        print(f"torus64x24 wave {b} step {i}: |w_gpu - w_oracle| / |w_oracle| = {err:.3e}")
        assert err <= 1e-6
