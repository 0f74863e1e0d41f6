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
