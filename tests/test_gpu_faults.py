"""Failures made on the host -- nothing here faults, traps or hangs the GPU:
a non-finite operator is refused at load; GMRES or CG held to one iteration
returns MOT_ENOCONV with the step counted and its iterate kept, the march
going on; the same inputs without the limits are never flagged."""
import copy

import numpy as np
import pytest

from paper_2510_07989_gb300.inputs import meshes as MS

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def M():
    from paper_2510_07989_gb300.build import build
    build()
    from paper_2510_07989_gb300 import mot
    return mot


def _march(M, s, ops, n):
    waves = M.mot_waves(MS.single_wave(ops.dt, 30, 60))
    return [M.mot_step(s.h, waves, 1) for _ in range(n)]


def test_non_finite_operator_refused(M, pr1_ops):
    bad = copy.copy(pr1_ops)
    bad.T0s = pr1_ops.T0s.copy()
    bad.T0s[3, 5] = np.nan
    m = pr1_ops.mesh
    h = M.mot_create(m.verts, m.tris, pr1_ops.eps_r, pr1_ops.mu_r, pr1_ops.dt, pr1_ops.kmax + 1)
    with pytest.raises(M.MotError) as e:
        M.mot_load_operators(h, bad)
    assert e.value.code == M.MOT_EINVAL and "non-finite" in str(e.value)


def test_gmres_iteration_limit_flags_and_continues(M, pr1_ops):
    n = 45  # the pulse (t0 = 60 dt, w = 30 c dt) is under way from about step 30
    s = M.Solver(pr1_ops, gmres_maxit=1)
    codes = _march(M, s, pr1_ops, n)
    assert M.MOT_ENOCONV in codes and set(codes) <= {M.MOT_OK, M.MOT_ENOCONV}
    info = s.info()
    assert info["step"] == n and info["last_gmres_iters"] == 1
    assert "GMRES" in M.mot_last_error(s.h)
    assert all(c == M.MOT_OK for c in _march(M, M.Solver(pr1_ops), pr1_ops, n))


def test_cg_iteration_limit_flags_and_continues(M, pr1_ops):
    n = 45
    s = M.Solver(pr1_ops, cg_maxit=1)
    codes = _march(M, s, pr1_ops, n)
    assert M.MOT_ENOCONV in codes and set(codes) <= {M.MOT_OK, M.MOT_ENOCONV}
    assert s.info()["step"] == n
    assert "CG" in M.mot_last_error(s.h)


@pytest.mark.parametrize("tasks_per_stage", [1, 2])
def test_history_wait_bound_ends_in_error_status(M, tasks_per_stage):
    """The device side of failure detection, in the allowed form: with
    hist_stall_test the first CTA of every tensor-core history launch withholds
    one stage's copies and arrivals (a barrier phase nothing completes; stages
    of one task, and of two tasks behind one barrier pair) and its
    waits give up after 1 ms. The CTA takes its abort path (stops issuing,
    drains the copies in flight, releases TMEM, raises the error word) and
    mot_step returns MOT_ECUDA; the context stays usable: a fresh handle then
    marches to the oracle's result."""
    from oracle import mot as O
    from paper_2510_07989_gb300.inputs.assemble import assemble
    ops = assemble(MS.torus(1.0, 0.3, 12, 6), 4.0, 1.0, 0.1)
    exc = MS.fibonacci_batch(64, ops.dt, w_steps=30, t0_steps=60)
    waves = M.mot_waves(exc)
    s = M.Solver(ops, precision=M.MOT_PREC_MIXED, hist_stall_test=4)
    M.mot_step(s.h, waves, 64)  # step 1 has no history (every lag >= 1): nothing stalls
    if tasks_per_stage == 2:  # two tasks behind each barrier pair
        M.mot_set_tc_config(s.h, 512, 0.4, 2, 2, 4)
    with pytest.raises(M.MotError) as e:
        for _ in range(ops.kmax + 8):
            M.mot_step(s.h, waves, 64)
    assert e.value.code == M.MOT_ECUDA and "ran out of time" in str(e.value)
    assert M.mot_get_info(s.h)["hist_kernel"] == 2
    del s
    n = 100
    s2 = M.Solver(ops, precision=M.MOT_PREC_MIXED)
    W = s2.run(exc, n)
    assert s2.noconv == 0
    ref = O.march(O.build_system(ops), exc, n, b=5)
    assert np.abs(W[:, 5].reshape(n, -1) - ref).max() < 1e-6 * np.abs(ref).max()
