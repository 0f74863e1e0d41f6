"""The plain-FP64 configuration of the paper's sphere experiments on the GPU:
dielectric sphere of radius 1 as an icosphere of level 3 (1280 triangles,
1920 edges, 3840 unknowns), eps_r = 2, the paper's pulse (w = 120 c dt,
t0 = 240 dt).

* Parity at c dt = 0.05 (k_max = 57, 58 history lags) and c dt = 0.5
  (k_max = 6): the FP64 GPU march against the product-form FP64 oracle, one
  step computed by the oracle from the GPU's own previous steps at steps 200,
  300 and 400 (the window around the pulse), within 1e-10 of the run's peak
  step norm (the metric of the readings; at c dt = 0.5 the solution at step
  400 has decayed to ~1e-12 of that peak).
* Late-time stability (Section VI-A): 10^4 steps at c dt = 0.5; the solution
  decays far below its peak and does not grow over the last 10^3 steps."""
import numpy as np
import pytest

from oracle import product as P
from paper_2510_07989_gb300.inputs import meshes as MS
from paper_2510_07989_gb300.inputs.assemble import assemble

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def M():
    from paper_2510_07989_gb300.build import build
    build()
    from paper_2510_07989_gb300 import mot
    return mot


def oracle_step(sysP, exc, b, i, history):
    """w_i of wave b by the product-form oracle from history[j] = w_j, j < i."""
    ne = sysP.ne
    L = np.zeros((i + 1, 2 * ne))
    S = np.zeros((i + 1, 2 * ne))
    for j, w in history.items():
        if j < i:
            L[j], S[j] = sysP.split(w)
    return sysP.step(exc, b, i, L, S)


@pytest.mark.parametrize("cdt", [0.05, 0.5])
def test_icosphere_l3_fp64_parity(M, cdt):
    ops = assemble(MS.icosphere(3), 2.0, 1.0, cdt)
    assert ops.ne == 1920 and ops.kmax == {0.05: 57, 0.5: 6}[cdt]
    exc = MS.single_wave(cdt)
    K = ops.kmax + 1
    checks = (200, 300, 400)
    s = M.Solver(ops)
    waves = M.mot_waves(exc)
    out = np.zeros((1, 2, ops.ne))
    hist = {}
    peak = 0.0
    for i in range(1, checks[-1] + 1):
        M.mot_step(s.h, waves, 1, out)
        peak = max(peak, np.linalg.norm(out))
        if any(c - K - 1 <= i <= c for c in checks):
            hist[i] = out[0].reshape(-1).copy()
    assert s.noconv == 0
    sysP = P.ProductSystem(ops)
    for c in checks:
        w_ref = oracle_step(sysP, exc, 0, c, {j: w for j, w in hist.items() if c - K - 1 <= j < c})
        err = np.linalg.norm(hist[c] - w_ref) / peak
        print(f"icosphere L3 c dt = {cdt}: step {c}, |w_gpu - w_oracle| / peak = {err:.3e}, "
              f"|w_oracle| / peak = {np.linalg.norm(w_ref) / peak:.3e}")
        assert err <= 1e-10


def test_icosphere_l3_late_time_stability(M):
    ops = assemble(MS.icosphere(3), 2.0, 1.0, 0.5)
    exc = MS.single_wave(0.5)
    n = 10000
    s = M.Solver(ops, fp64_precond=1)
    waves = M.mot_waves(exc)
    out = np.zeros((1, 2, ops.ne))
    norms = np.zeros(n)
    for i in range(n):
        M.mot_step(s.h, waves, 1, out)
        norms[i] = np.linalg.norm(out)
    assert s.noconv == 0
    peak = norms.max()
    print(f"icosphere L3 c dt = 0.5, 10^4 steps: peak at step {norms.argmax() + 1}, "
          f"|w| / peak at steps 1000, 5000, 10000: {norms[999] / peak:.2e}, {norms[4999] / peak:.2e}, "
          f"{norms[-1] / peak:.2e}")
    assert norms[-1] < 1e-12 * peak
    assert norms[-1000:].max() <= norms[-2000:-1000].max() + 1e-30 * peak
