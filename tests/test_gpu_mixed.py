"""Mixed-precision CUDA path against the FP64 oracle: error <= 1e-6 relative to
the run's peak over every step (the accuracy target of the batched mixed
path), and agreement with the FP64 GPU path."""
import numpy as np
import pytest

from oracle import mot as O
from paper_2510_07989_gb300.inputs import meshes as MS
from paper_2510_07989_gb300.inputs.assemble import assemble

pytestmark = pytest.mark.gpu
TOL_MIXED = 1e-6


@pytest.fixture(scope="module")
def M():
    from paper_2510_07989_gb300.build import build
    build()
    from paper_2510_07989_gb300 import mot
    return mot


def rel(a, b):
    return np.abs(a - b).max() / np.abs(b).max()


def test_mixed_pr1_matches_oracle(M, pr1_ops, pr1_system):
    exc = MS.single_wave(pr1_ops.dt, 30, 60)
    n = 200
    s = M.Solver(pr1_ops, precision=M.MOT_PREC_MIXED)
    W = s.run(exc, n)[:, 0].reshape(n, -1)
    ref = O.march(pr1_system, exc, n)
    err = rel(W, ref)
    print(f"mixed PR1 max rel err {err:.3e}")
    assert err < TOL_MIXED


def test_mixed_full_batch_pr1(M, pr1_ops, pr1_system):
    """B = 64 (the batched-kernel width of the bench), PR1, sampled columns vs the oracle."""
    exc = MS.fibonacci_batch(64, pr1_ops.dt, w_steps=30, t0_steps=60)
    n = 150
    W = M.Solver(pr1_ops, precision=M.MOT_PREC_MIXED).run(exc, n)
    errs = []
    for b in (0, 1, 17, 31, 32, 50, 63):
        ref = O.march(pr1_system, exc, n, b=b)
        errs.append(rel(W[:, b].reshape(n, -1), ref))
    print("mixed PR1 B=64 max rel errs", ["%.3e" % e for e in errs])
    assert max(errs) < TOL_MIXED


def test_mixed_ragged_batch_l2(M):
    ops = assemble(MS.icosphere(2), 3.0, 1.0, 0.3)
    S = O.build_system(ops)
    exc = MS.fibonacci_batch(3, 0.3, w_steps=40, t0_steps=80)
    n = 150
    W = M.Solver(ops, precision=M.MOT_PREC_MIXED).run(exc, n)
    errs = []
    for b in range(3):
        ref = O.march(S, exc, n, b=b)
        errs.append(rel(W[:, b].reshape(n, -1), ref))
    print("mixed L2 B=3 max rel errs", ["%.3e" % e for e in errs])
    assert max(errs) < TOL_MIXED


@pytest.fixture(scope="module")
def torus_small():
    """Torus 12 x 6 (216 edges: seven 32-edge row blocks, the last one ragged),
    eps_r = 4, c dt = 0.1 (k_max = 52): many lags, several tiles per row block."""
    ops = assemble(MS.torus(1.0, 0.3, 12, 6), 4.0, 1.0, 0.1)
    return ops, O.build_system(ops)


def test_tensor_core_history_matches_oracle(M, torus_small):
    """B = 64 selects the tcgen05 history kernel (bf16 x 3 slices, FP32
    accumulation, compensated sums); sampled columns against the FP64 oracle
    over every step, and against the FP32 CUDA-core kernel on the same inputs."""
    ops, S = torus_small
    exc = MS.fibonacci_batch(64, ops.dt, w_steps=30, t0_steps=60)
    n = 130
    s_tc = M.Solver(ops, precision=M.MOT_PREC_MIXED)
    W = s_tc.run(exc, n)
    assert s_tc.info()["hist_kernel"] == 2
    errs = []
    for b in (0, 9, 33, 63):
        ref = O.march(S, exc, n, b=b)
        errs.append(rel(W[:, b].reshape(n, -1), ref))
    print("tensor-core history, torus 12x6 B=64 max rel errs", ["%.3e" % e for e in errs])
    assert max(errs) < TOL_MIXED
    s_cc = M.Solver(ops, precision=M.MOT_PREC_MIXED, mixed_flags=M.MOT_MIX_DEFAULT & ~M.MOT_MIX_TC)
    W_cc = s_cc.run(exc, n)
    assert s_cc.info()["hist_kernel"] == 1
    # the FP32 CUDA-core kernel sums its FP32 tile products in FP64 every four
    # tiles; the tensor-core kernel's compensated sums are at least as accurate
    errs_cc = [rel(W_cc[:, b].reshape(n, -1), O.march(S, exc, n, b=b)) for b in (0, 33)]
    print("CUDA-core history, same columns", ["%.3e" % e for e in errs_cc])
    assert max(errs[0], errs[2]) <= max(errs_cc)


@pytest.mark.parametrize("B", [32, 16, 8])
def test_tensor_core_history_smaller_batches(M, torus_small, B):
    """A batch that is a multiple of 8 below 64 (the cube configuration's 32,
    the uneven batch's 16) also runs the tensor-core history, filling the first
    2B of the 128 MMA rows: the first and last waves against the FP64 oracle
    over every step, on the torus 12 x 6 with its 53 lags."""
    ops, S = torus_small
    exc = MS.fibonacci_batch(B, ops.dt, w_steps=30, t0_steps=60)
    n = 130
    s = M.Solver(ops, precision=M.MOT_PREC_MIXED)
    W = s.run(exc, n)
    assert s.info()["hist_kernel"] == 2 and s.noconv == 0
    errs = [rel(W[:, b].reshape(n, -1), O.march(S, exc, n, b=b)) for b in (0, B - 1)]
    print(f"tensor-core history, torus 12x6 B={B} max rel errs", ["%.3e" % e for e in errs])
    assert max(errs) < TOL_MIXED


@pytest.mark.parametrize("B", [64, 32])
def test_tensor_core_history_bulk_form(M, torus_small, B):
    """The bulk form of the tensor-core history (one global column order,
    pre-swizzled 32-row coefficient blocks moved by bulk copies): against the
    FP64 oracle over every step on the torus 12 x 6 (53 lags, ragged last row
    block), and against the gathered form on the same waves."""
    ops, S = torus_small
    exc = MS.fibonacci_batch(B, ops.dt, w_steps=30, t0_steps=60)
    n = 130
    s = M.Solver(ops, precision=M.MOT_PREC_MIXED, mixed_flags=M.MOT_MIX_DEFAULT | M.MOT_MIX_TCBULK)
    W = s.run(exc, n)
    assert s.info()["hist_kernel"] == 2 and s.noconv == 0
    errs = [rel(W[:, b].reshape(n, -1), O.march(S, exc, n, b=b)) for b in (0, B // 2 + 1, B - 1)]
    print(f"tensor-core history, bulk form, torus 12x6 B={B} max rel errs", ["%.3e" % e for e in errs])
    assert max(errs) < TOL_MIXED
    Wg = M.Solver(ops, precision=M.MOT_PREC_MIXED, mixed_flags=M.MOT_MIX_DEFAULT & ~M.MOT_MIX_TCBULK).run(exc, n)
    assert np.abs(W - Wg).max() < TOL_MIXED * np.abs(Wg).max()


def test_tune_keeps_the_march(M, torus_small):
    """mot_tune on one handle at full depth (step 54 of the 53-lag torus):
    a configuration is chosen and reported, and the march it continues meets
    the oracle as before (its trial launches leave the march state alone)."""
    ops, S = torus_small
    exc = MS.fibonacci_batch(64, ops.dt, w_steps=30, t0_steps=60)
    waves = M.mot_waves(exc)
    n = 130
    s = M.Solver(ops, precision=M.MOT_PREC_MIXED)
    out = np.zeros((64, 2, ops.ne))
    W = np.zeros((n, 64, 2, ops.ne))
    for i in range(n):
        if i == ops.kmax + 1:
            M.mot_tune([s.h])
        M.mot_step(s.h, waves, 64, out)
        W[i] = out
    info = s.info()
    assert info["tc_tuned"] == 1 and info["tc_chunk_cap"] in (256, 512, 1024) and info["tc_stages"] in (2, 3, 4, 5) and info["tc_tasks_per_stage"] in (1, 2)
    assert info["tc_epilogue_warps"] in (4, 8) and info["tc_tune_ms"] > 0
    errs = [rel(W[:, b].reshape(n, -1), O.march(S, exc, n, b=b)) for b in (0, 63)]
    print(f"tuned march (cap {info['tc_chunk_cap']}, lag fraction {info['tc_lag_frac']}, {info['tc_stages']} stages of {info['tc_tasks_per_stage']}, "
          f"{info['tc_epilogue_warps']} epilogue warps): rel errs", ["%.3e" % e for e in errs])
    assert max(errs) < TOL_MIXED


@pytest.mark.parametrize("bulk", [False, True])
def test_pipeline_configurations_agree(M, torus_small, bulk):
    """Every pipeline of the tensor-core history -- 4 or 5 stages of one task,
    2 or 3 stages of two tasks behind one barrier pair, 4 or 8 epilogue warps
    -- runs the same MMAs and folds in the same order for one chunking, so the
    marches agree to rounding (bitwise where the rest of the step is
    deterministic); the first one meets the oracle. Set after step 1 with
    mot_set_tc_config, gathered and bulk form, torus 12 x 6, B = 64."""
    ops, S = torus_small
    exc = MS.fibonacci_batch(64, ops.dt, w_steps=30, t0_steps=60)
    waves = M.mot_waves(exc)
    n = 130
    flags = M.MOT_MIX_DEFAULT | (M.MOT_MIX_TCBULK if bulk else 0)
    runs = {}
    for cfg in [(4, 1, 4), (5, 1, 8), (2, 2, 4), (2, 2, 8), (3, 2, 4)]:
        s = M.Solver(ops, precision=M.MOT_PREC_MIXED, mixed_flags=flags)
        out = np.zeros((64, 2, ops.ne))
        W = np.zeros((n, 64, 2, ops.ne))
        for i in range(n):
            if i == 1:
                M.mot_set_tc_config(s.h, 512, 0.4, *cfg)
            M.mot_step(s.h, waves, 64, out)
            W[i] = out
        info = s.info()
        assert info["hist_kernel"] == 2 and info["tc_tuned"] == 0
        assert (info["tc_stages"], info["tc_tasks_per_stage"], info["tc_epilogue_warps"]) == cfg
        runs[cfg] = W.reshape(n, 64, -1)
        del s
    W0 = runs[(4, 1, 4)]
    errs = [rel(W0[:, b], O.march(S, exc, n, b=b)) for b in (0, 63)]
    diffs = {c: float(np.abs(W - W0).max() / np.abs(W0).max()) for c, W in runs.items()}
    print(f"pipelines ({'bulk' if bulk else 'gathered'} form): oracle rel errs", ["%.3e" % e for e in errs],
          "; max rel difference to 4 x 1 stages:", {str(c): "%.1e" % d for c, d in diffs.items()})
    assert max(errs) < TOL_MIXED
    assert max(diffs.values()) < 1e-12


def test_mixed_save_load_state_resumes_exactly(M, torus_small):
    """mot_save_state / mot_load_state on the mixed path (reduced-precision ring
    copies rebuilt from the FP64 ring): the resumed run repeats the original."""
    ops, _ = torus_small
    exc = MS.fibonacci_batch(64, ops.dt, w_steps=30, t0_steps=60)
    a = M.Solver(ops, precision=M.MOT_PREC_MIXED)
    a.run(exc, 70, keep=False)
    state = M.mot_save_state(a.h)
    W1 = a.run(exc, 15)
    b = M.Solver(ops, precision=M.MOT_PREC_MIXED)
    M.mot_load_state(b.h, state)
    W2 = b.run(exc, 15)
    assert np.array_equal(W1, W2)


def test_small_cube_regime(M):
    """The cube configuration's regime at a size the oracle marches in
    seconds: non-smooth cube (side 2, 6 cells per edge: 432 triangles, 648
    edges), eps_r = 6, c dt = 0.25 (k_max = 34, 35 history lags). FP64, one
    wave, within 1e-10; mixed with the configuration's 32 waves (tensor-core
    history), sampled waves within 1e-6 -- both against the oracle over 160
    steps (pulse inside)."""
    import math
    ops = assemble(MS.cube(2.0, 6), 6.0, 1.0, 0.25)
    assert ops.kmax == 34
    S = O.build_system(ops)
    r = math.sqrt(3.0)
    n = 160
    one = MS.single_wave(0.25, 30, 60, r_obj=r)
    W1 = M.Solver(ops).run(one, n)[:, 0].reshape(n, -1)
    e64 = rel(W1, O.march(S, one, n))
    batch = MS.fibonacci_batch(32, 0.25, w_steps=30, t0_steps=60, r_obj=r)
    s = M.Solver(ops, precision=M.MOT_PREC_MIXED)
    W = s.run(batch, n)
    assert s.info()["hist_kernel"] == 2
    errs = [rel(W[:, b].reshape(n, -1), O.march(S, batch, n, b=b)) for b in (0, 13, 31)]
    print(f"cube 6/edge: FP64 rel err {e64:.3e}; mixed B=32 rel errs", ["%.3e" % e for e in errs])
    assert e64 < 1e-10
    assert max(errs) < TOL_MIXED
