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
