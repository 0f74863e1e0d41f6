"""mot_run_many (several scatterers of uneven size, precision and batch
marched concurrently, one stream and host thread each) against the same
scatterers marched one at a time with mot_step: every step of every
scatterer agrees to 1e-14 of its peak (the kernels and their order per
scatterer are the same, so the results are expected to be bitwise equal)."""
import numpy as np
import pytest

from paper_2510_07989_gb300.inputs import meshes as MS
from paper_2510_07989_gb300.inputs.assemble import assemble

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def M():
    from paper_2510_07989_gb300.build import build
    build()
    from paper_2510_07989_gb300 import mot
    return mot


def test_run_many_uneven_batch_matches_single_runs(M):
    cases = [
        # icosphere L1 (120 edges), FP64 path, one wave
        (assemble(MS.icosphere(1), 2.0, 1.0, 0.2), M.MOT_PREC_FP64, MS.single_wave(0.2, 30, 60)),
        # icosphere L2 (480 edges), mixed path, three waves (CUDA-core history)
        (assemble(MS.icosphere(2), 3.0, 1.0, 0.3), M.MOT_PREC_MIXED,
         MS.fibonacci_batch(3, 0.3, w_steps=40, t0_steps=80)),
        # torus 12 x 6 (216 edges, 53 lags), mixed path, 64 waves (tensor-core history)
        (assemble(MS.torus(1.0, 0.3, 12, 6), 4.0, 1.0, 0.1), M.MOT_PREC_MIXED,
         MS.fibonacci_batch(64, 0.1, w_steps=30, t0_steps=60, r_obj=1.3)),
    ]
    n = 80
    refs = [M.Solver(ops, precision=p).run(exc, n) for ops, p, exc in cases]
    solvers = [M.Solver(ops, precision=p) for ops, p, _ in cases]
    waves = [M.mot_waves(exc) for _, _, exc in cases]
    outs = [np.full((n, exc.B, 2, s.ne), np.nan) for (_, _, exc), s in zip(cases, solvers)]
    code = M.mot_run_many([s.h for s in solvers], n, waves, [exc.B for _, _, exc in cases], outs)
    assert code == M.MOT_OK
    for i, (o, r) in enumerate(zip(outs, refs)):
        err = np.abs(o - r).max() / np.abs(r).max()
        print(f"scatterer {i}: max |run_many - single| / peak = {err:.3e}, bitwise equal: {np.array_equal(o, r)}")
        assert err <= 1e-14
    # the handles keep marching normally afterwards
    for s, (_, _, exc) in zip(solvers, cases):
        assert M.mot_get_info(s.h)["step"] == n


def test_run_many_merged_history_and_tuner(M):
    """Three scatterers on the tensor-core history (torus 12 x 6 with 53 lags
    and 64 waves, icosphere L2 with 13 lags and 16 waves, the non-smooth cube
    of 6 cells per edge with 35 lags and 32 waves): mot_run_many runs their
    history contractions as one launch per step and tunes that launch at the
    first step that contracts every full history (step 54). Every scatterer
    against the FP64 oracle over all 90 steps (two waves each) within 1e-6,
    and against its own single march within 1e-6 of the peak."""
    from oracle import mot as O
    cases = [
        (assemble(MS.torus(1.0, 0.3, 12, 6), 4.0, 1.0, 0.1), MS.fibonacci_batch(64, 0.1, w_steps=30, t0_steps=60,
                                                                                  r_obj=1.3)),
        (assemble(MS.icosphere(2), 3.0, 1.0, 0.3), MS.fibonacci_batch(16, 0.3, w_steps=40, t0_steps=80)),
        (assemble(MS.cube(2.0, 6), 6.0, 1.0, 0.25), MS.fibonacci_batch(32, 0.25, w_steps=30, t0_steps=60,
                                                                       r_obj=3 ** 0.5)),
    ]
    n = 90
    prec = M.MOT_PREC_MIXED
    solvers = [M.Solver(ops, precision=prec) for ops, _ in cases]
    waves = [M.mot_waves(exc) for _, exc in cases]
    outs = [np.full((n, exc.B, 2, s.ne), np.nan) for (_, exc), s in zip(cases, solvers)]
    code = M.mot_run_many([s.h for s in solvers], n, waves, [exc.B for _, exc in cases], outs)
    assert code == M.MOT_OK
    for i, ((ops, exc), s, o) in enumerate(zip(cases, solvers, outs)):
        info = M.mot_get_info(s.h)
        assert info["hist_kernel"] == 2 and info["tc_tuned"] == 1 and info["step"] == n
        S = O.build_system(ops)
        errs = [np.abs(o[:, b].reshape(n, -1) - O.march(S, exc, n, b=b)).max() /
                np.abs(O.march(S, exc, n, b=b)).max() for b in (0, exc.B - 1)]
        single = M.Solver(ops, precision=prec).run(exc, n)
        d = np.abs(o - single).max() / np.abs(single).max()
        print(f"scatterer {i}: tuned cap {info['tc_chunk_cap']}, lag fraction {info['tc_lag_frac']}, "
              f"stages {info['tc_stages']}; oracle rel errs {['%.3e' % e for e in errs]}; vs single {d:.3e}")
        assert max(errs) < 1e-6 and d < 1e-6
