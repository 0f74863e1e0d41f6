"""mot_fields_noalloc against mot_fields, through the C ABI.

mot_fields_noalloc serves callers that may not allocate device memory during
the call (a foreign memory pool owns the device, or allocation would
synchronise a latency-critical loop): it stages its data in a fixed device
array built into the library. This file is collected last so that a run that
stops at the first failure has already run every other test."""
import numpy as np
import pytest

from paper_2510_07989_gb300.inputs import meshes as MS
from paper_2510_07989_gb300.inputs.assemble import assemble

pytestmark = pytest.mark.gpu
TOL = 1e-10


@pytest.fixture(scope="module")
def marched():
    from paper_2510_07989_gb300.build import build
    build()
    from paper_2510_07989_gb300 import mot as M
    ops = assemble(MS.icosphere(1), 2.0, 1.0, 0.2)
    s = M.Solver(ops)
    exc = MS.fibonacci_batch(2, 0.2, w_steps=30, t0_steps=60)
    waves = M.mot_waves(exc)
    M.mot_set_frequencies(s.h, np.array([0.4, 0.9]))
    for _ in range(50):
        M.mot_step(s.h, waves, 2)
    return M, s, waves


def test_fields_noalloc_matches_fields_twice(marched):
    M, s, waves = marched
    dirs = np.array([[0.0, 0.0, 1.0], [0.6, 0.0, 0.8], [0.0, -1.0, 0.0], [-0.48, 0.6, -0.64]])
    ref = M.mot_fields(s.h, waves, dirs, 2, 2)
    assert np.abs(ref).max() > 0
    for _ in range(2):  # the fixed array keeps the previous call's contents
        got = M.mot_fields_noalloc(s.h, waves, dirs, 2, 2)
        assert np.abs(got - ref).max() <= TOL * np.abs(ref).max()
    # a different request in between must not leak into the next one
    other = M.mot_fields_noalloc(s.h, waves, dirs[:1], 2, 2)
    assert np.abs(other - ref[:, :, :1]).max() <= TOL * np.abs(ref).max()


def test_fields_noalloc_rejects_oversized_request(marched):
    M, s, waves = marched
    dirs = np.tile(np.array([[0.0, 0.0, 1.0]]), (20000, 1))
    with pytest.raises(M.MotError) as e:
        M.mot_fields_noalloc(s.h, waves, dirs, 2, 2)
    assert e.value.code == M.MOT_EINVAL and "exceeds the fixed scratch" in str(e.value)


def test_fields_noalloc_limit_is_exact(marched):
    """The stated limit 3*n_dir + 6*B*n_freq*n_dir <= 262144 holds to the
    double: with B = 2 and two frequencies, 9709 directions fit (262143
    doubles) and 9710 do not (262170)."""
    M, s, waves = marched
    rng = np.random.default_rng(5)
    d = rng.standard_normal((9710, 3))
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    got = M.mot_fields_noalloc(s.h, waves, d[:9709], 2, 2)
    ref = M.mot_fields(s.h, waves, d[:9709], 2, 2)
    assert np.abs(got - ref).max() <= TOL * np.abs(ref).max()
    with pytest.raises(M.MotError) as e:
        M.mot_fields_noalloc(s.h, waves, d, 2, 2)
    assert e.value.code == M.MOT_EINVAL
