"""Values the paper prints (tests/golden/, each file citing its passage)
against the mathematics, the input generators and the oracle."""
import numpy as np

from conftest import golden_table, golden_values
from oracle import mot as O
from paper_2510_07989_gb300.inputs import meshes as MS

C_M_PER_NS = 0.299792458  # speed of light in vacuum, metres per nanosecond


def test_paper_meshes_are_closed_surfaces_of_their_genus():
    """Section VI-A mesh counts: every edge borders two triangles (E = 3F/2),
    Euler's formula V - E + F = 2 - 2g, and the loop-space dimension the
    projectors must reproduce, N_e - N_f + 1 = (N_v - 1) + 2g (local loops plus
    the 2g global loops of Section IV-B)."""
    rows = golden_table("section6a_meshes.txt")
    assert [r[0] for r in rows] == ["sphere", "torus", "star_pyramid"]
    for name, f, v, e, g in rows:
        f, v, e, g = int(f), int(v), int(e), int(g)
        assert 2 * e == 3 * f, name
        assert v - e + f == 2 - 2 * g, name
        assert e - f + 1 == (v - 1) + 2 * g, name


def test_uv_sphere_is_the_paper_sphere_and_oracle_ranks():
    """The 32 x 25 latitude-longitude sphere has the counts of the paper's
    sphere, and the oracle's projectors on it have ranks N_f - 1 (star),
    N_v - 1 (BC loop) and N_e - N_f + 1 (RWG loop), Section IV-B."""
    name, f, v, e, g = golden_table("section6a_meshes.txt")[0]
    m = MS.uv_sphere(32, 25)
    assert (m.nf, m.nv, m.ne) == (int(f), int(v), int(e))
    assert abs(MS.diameter(m) - 2.0) < 1e-12
    L, S = O.incidence(m.ev, m.ef, m.nv, m.nf)
    assert np.abs(S.T @ L).max() == 0
    P = O.projectors(L, S)
    rk = lambda A: int(round(np.trace(A)))
    assert rk(P["PS"]) == m.nf - 1
    assert rk(P["PL"]) == m.nv - 1
    assert rk(P["PLH"]) == m.ne - m.nf + 1 == (m.nv - 1) + 2 * int(g)


def test_sphere_experiment_parameters_and_excitation():
    """Section VI-A: the printed time step in ns is the printed c dt in metres,
    and the input generator's excitation for that c dt is the paper's
    (A = 1, p = x, k = z, w = 120 c dt, t0 = 240 dt)."""
    gv = golden_values("section6a_sphere_experiment.txt")
    assert abs(gv["dt_ns"] * C_M_PER_NS - gv["c_dt_m"]) / gv["c_dt_m"] < 1e-3
    cdt = gv["c_dt_m"]
    exc = MS.single_wave(cdt, gv["w_over_c_dt"], gv["t0_over_dt"], r_obj=gv["radius_m"])
    assert exc.B == 1 and exc.A[0] == gv["A_V"]
    assert tuple(exc.p[0]) == gv["p"] and tuple(exc.k[0]) == gv["k"]
    assert abs(exc.w[0] - 120 * cdt) < 1e-12 and abs(exc.t0[0] - 240 * cdt) < 1e-12
