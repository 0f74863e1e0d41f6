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
