"""Pins of the oracle against what the paper and the mathematics fix: projector
algebra, closed forms of the excitation, the exact solution for eps' = eps,
the Mie series and its Rayleigh limit, late-time decay, the companion-matrix
spectrum, Delta-t independent conditioning and loop/star balance."""
import math

import numpy as np
import pytest
import scipy.linalg as sla
from scipy.integrate import quad

from oracle import farfield as FF
from oracle import mot as O
from paper_2510_07989_gb300.inputs import meshes as MS
from paper_2510_07989_gb300.inputs.assemble import assemble
from conftest import golden_values

# ---------------------------------------------------------------- projectors


@pytest.mark.parametrize("make,genus", [(lambda: MS.icosphere(2), 0), (lambda: MS.torus(1.0, 0.3, 16, 8), 1)])
def test_projector_algebra(make, genus):
    """P^2 = P, P^T = P, P^S + P^LH = I, P^L + P^SH = I, P^SH P^L = 0, rank
    P^S = N_f - 1, rank P^L = N_v - 1, dim range P^LH = N_e - N_f + 1 (local
    plus 2g global loops), Section IV-B."""
    m = make()
    L, S = O.incidence(m.ev, m.ef, m.nv, m.nf)
    P = O.projectors(L, S)
    I = np.eye(m.ne)
    for key in ("PS", "PLH", "PL", "PSH"):
        A = P[key]
        assert np.abs(A @ A - A).max() < 1e-12
        assert np.abs(A - A.T).max() < 1e-12
    assert np.abs(P["PS"] + P["PLH"] - I).max() < 1e-12
    assert np.abs(P["PSH"] @ P["PL"]).max() < 1e-12
    rk = lambda A: int(round(np.trace(A)))
    assert rk(P["PS"]) == m.nf - 1
    assert rk(P["PL"]) == m.nv - 1
    assert rk(P["PLH"]) == m.ne - m.nf + 1 == (m.nv - 1) + 2 * genus
    # Lambda columns are loops: P^S Lambda = 0
    assert np.abs(P["PS"] @ L).max() < 1e-12


def test_projector_planted_mistake_detected():
    """A transposed incidence (Lambda built with v^- and v^+ swapped on half the
    edges) breaks Sigma^T Lambda = 0 and the complementarity P^S P^L != 0."""
    m = MS.icosphere(1)
    ev = m.ev.copy()
    ev[::2] = ev[::2, ::-1]
    L, S = O.incidence(ev, m.ef, m.nv, m.nf)
    assert np.abs(S.T @ L).max() > 0.5

# ---------------------------------------------------------------- excitation


def test_gaussian_time_integral_closed_form():
    """int e(x, t) dt = (A/c) p (Section V-C) and the erf primitive used for
    d/dt^-1 e matches numerical quadrature of Eq. (hin)."""
    exc = MS.single_wave(0.1)
    A, w, t0 = exc.A[0], exc.w[0], exc.t0[0]
    x = np.array([[0.3, -0.2, 0.5]])
    g = lambda t: (4 * A / (w * math.sqrt(math.pi))) * math.exp(-((4 / w) * (t - t0 - 0.5)) ** 2)
    total = quad(g, t0 - 10 * w, t0 + 10 * w, points=[t0 + 0.5], limit=200)[0]
    assert abs(total - A) < 1e-10
    for t in (t0 - 0.3 * w, t0 + 0.1 * w, t0 + 0.7 * w):
        num = quad(g, t0 - 10 * w, t, limit=200)[0]
        E, H = O.incident_integral(exc, 0, x, t)
        assert abs(E[0, 0] - num) < 1e-10
        assert np.allclose(H[0], np.cross(exc.k[0], E[0]))


def test_rhs_loop_average_and_truncation(pr1_ops):
    """rho1 is the dt-average of the tested field over p_i's support, rho2 the
    tested time integral / T_max, forced to zero after t_trunc."""
    ops = pr1_ops
    exc = MS.single_wave(ops.dt, 30, 60)
    i = 60
    r1, r2 = O.rhs_parts(ops, exc, 0, i)
    r1a, r2a = O.rhs_parts(ops, exc, 0, i - 1)
    assert np.allclose(r1, (r2 - r2a) * ops.tmax / ops.dt, rtol=0, atol=1e-14 * np.abs(r1).max())
    late = int(exc.t_trunc[0] / ops.dt) + 2
    assert np.all(O.rhs_parts(ops, exc, 0, late)[1] == 0)

# ---------------------------------------------------------------- Q_0 solve


def test_gmres_matches_lu(pr1_system):
    """GMRES (tol 1e-13) on Q_0 w = b equals the LU solve to 1e-10 (Eq. (MOT))."""
    S = pr1_system
    rng = np.random.default_rng(3)
    b = rng.standard_normal(S.Q[0].shape[0])
    x_lu = sla.lu_solve(S.lu, b)
    x_g, it, res = O.gmres(lambda v: S.Q[0] @ v, b, tol=1e-13, restart=300)
    assert np.linalg.norm(x_g - x_lu) / np.linalg.norm(x_lu) < 1e-10
    assert it < 150


def test_truncation_of_matrix_blocks(pr1_system):
    """Q_k = 0 for k > k_max + 1 (the oracle keeps Q_0..Q_{k_max+1}); the Q^sl
    part (left factor T^L G^-1 P^LH, right factor P^LH, family A~) vanishes for
    k >= k_max (explicit truncation, Section V-B-3)."""
    S = pr1_system
    ops = S.ops
    assert len(S.Q) == ops.kmax + 2
    for k in (ops.kmax, ops.kmax + 1):
        assert np.abs(O.pmchwt_block(ops, "T", k)).max() == 0
    assert np.abs(O.pmchwt_block(ops, "T", ops.kmax - 1)).max() > 0
    assert np.abs(O.pmchwt_block(ops, "H", ops.kmax + 2)).max() == 0


def test_spectral_property_of_static_double_layer(pr1_ops):
    """T^L G^-1 P^LH K_0 P^LH = 0 (Eq. (spec_prop)) up to quadrature error,
    while dropping the right P^LH leaves an O(1) residual."""
    ops = pr1_ops
    m = ops.mesh
    ne = ops.ne
    K0 = np.zeros((ne, ne))
    rows = np.repeat(np.arange(ne), np.diff(ops.mats["TK"].rowptr))
    K0[rows, ops.mats["TK"].col] = ops.mats["TK"].tc * ops.tmax / ops.dt
    L, S = O.incidence(m.ev, m.ef, m.nv, m.nf)
    P = O.projectors(L, S)
    A = P["PL"] @ ops.T0h @ P["PL"] @ np.linalg.inv(ops.G.toarray()) @ P["PLH"]
    den = np.linalg.norm(A, 2) * np.linalg.norm(K0, 2)
    assert np.linalg.norm(A @ K0 @ P["PLH"], 2) / den < 0.02
    assert np.linalg.norm(A @ K0, 2) / den > 0.1

# ---------------------------------------------------------------- physics


@pytest.fixture(scope="module")
def vacuum_sphere_run():
    """eps' = eps sphere (Section VI-A first example) with the printed
    parameters of tests/golden/section6a_sphere_experiment.txt (c dt, pulse
    width and delay, materials), on icosphere L2 (480 edges; the dense oracle
    on the paper's 2304-edge mesh would take minutes)."""
    gv = golden_values("section6a_sphere_experiment.txt")
    m = MS.icosphere(2, gv["radius_m"])
    ops = assemble(m, gv["eps_r"], gv["mu_r"], gv["c_dt_m"], with_bc_table=True)
    S = O.build_system(ops)
    exc = MS.single_wave(gv["c_dt_m"], gv["w_over_c_dt"], gv["t0_over_dt"], r_obj=gv["radius_m"])
    W = O.march(S, exc, 600)
    return ops, S, exc, W


def test_exact_solution_vacuum_interior(vacuum_sphere_run):
    """For eps' = eps the incident traces j = n x h, m = e x n solve the problem;
    projected as -G^{-T}(h_i, e_i) with [h]_m = <g_m, h>, [e]_m = -<g_m, e>
    (Section VI-A). Match to discretisation error (< 2 % of the peak)."""
    ops, S, exc, W = vacuum_sphere_run
    cur = O.recover(S, W)
    J = cur["j_loop"] + cur["j_star"]
    M = cur["m_loop"] + cur["m_star"]
    bc = ops.bc
    ne = ops.ne
    Gt = ops.G.toarray().T
    A, p, k, w, t0 = exc.A[0], exc.p[0], exc.k[0], exc.w[0], exc.t0[0]
    ej, em, nj, nm = [], [], [], []
    for i in range(1, W.shape[0] + 1):
        tt = (i - 0.5) * ops.dt
        g = (4 * A / (w * math.sqrt(math.pi))) * np.exp(-((4 / w) * (tt - t0 - bc.x @ k)) ** 2)
        E = g[:, None] * p[None, :]
        H = np.cross(k[None, :], E)
        hv = np.zeros(ne)
        ev = np.zeros(ne)
        np.add.at(hv, bc.n, np.einsum("id,id->i", bc.wg, H))
        np.add.at(ev, bc.n, -np.einsum("id,id->i", bc.wg, E))
        jex = -np.linalg.solve(Gt, hv)
        mex = -np.linalg.solve(Gt, ev)
        ej.append(np.linalg.norm(J[i - 1] - jex))
        em.append(np.linalg.norm(M[i - 1] - mex))
        nj.append(np.linalg.norm(jex))
        nm.append(np.linalg.norm(mex))
    assert max(ej) / max(nj) < 0.02
    assert max(em) / max(nm) < 0.02


def test_planted_sign_error_breaks_exact_solution(vacuum_sphere_run):
    """Flipping the sign of the double-layer blocks (a plausible mistake in
    Eq. (PMCHWT)) makes the eps' = eps solution miss the exact one by O(1)."""
    ops, S, exc, W = vacuum_sphere_run
    orig = O.pmchwt_block

    def flipped(ops_, fam, k):
        X = orig(ops_, fam, k)
        ne = ops_.ne
        X[:ne, ne:] *= -1
        X[ne:, :ne] *= -1
        return X

    O.pmchwt_block = flipped
    try:
        S2 = O.build_system(ops)
    finally:
        O.pmchwt_block = orig
    W2 = O.march(S2, exc, 300)
    assert np.abs(W2 - W[:300]).max() > 0.1 * np.abs(W).max()


def test_late_time_decay_and_no_growth(pr1_system):
    """PR1 with a pulse that passes within the run (w = 30 c dt, t0 = 60 dt):
    the solution decays to <= 1e-13 of its peak and does not grow over 10^4
    steps (Section VI-A: decay to machine precision)."""
    S = pr1_system
    exc = MS.single_wave(S.ops.dt, 30, 60)
    W = O.march(S, exc, 10000)
    n = np.linalg.norm(W, axis=1)
    assert n[-1] < 1e-13 * n.max()
    assert n[-1000:].max() <= max(n[-2000:-1000].max(), 1e-300) + 1e-30


def test_companion_spectrum_inside_unit_circle():
    """All companion-matrix eigenvalues strictly inside the unit circle, none
    near 1 + 0i (Section VI-A companion analysis); PR1 mesh at c dt = 0.5."""
    ops = assemble(MS.icosphere(1), 2.0, 1.0, 0.5)
    S = O.build_system(ops)
    ev = np.linalg.eigvals(O.companion(S))
    assert np.abs(ev).max() < 0.95
    assert np.abs(ev - 1).min() > 1e-2


def test_conditioning_independent_of_dt():
    """cond(Q_0) stays essentially constant over the paper's range of time
    steps, c dt from 1 m to 512 m (Section VI-B; tests/golden/
    section6b_conditioning.txt), sampled at 1, 8, 64, 512 m."""
    gv = golden_values("section6b_conditioning.txt")
    lo, hi = gv["c_dt_min_m"], gv["c_dt_max_m"]
    cdts = [lo * (hi / lo) ** (j / 3) for j in range(4)]
    m = MS.icosphere(1)
    conds = [np.linalg.cond(O.build_system(assemble(m, 2.0, 1.0, cdt)).Q[0]) for cdt in cdts]
    assert max(conds) / min(conds) < 3.0
    assert max(conds) < 30


def test_loop_star_balance_large_dt():
    """In u the star part stays O(1) relative to the loop part for every dt
    (rescaled unknowns, Section IV-B), while the recovered current's star part
    scales as O(omega) = O(1/dt) (Eq. (dis_jm))."""
    m = MS.icosphere(1)
    ratios_u, ratios_j = [], []
    for cdt in (5.0, 50.0, 5000.0):
        ops = assemble(m, 2.0, 1.0, cdt)
        S = O.build_system(ops)
        W = O.march(S, MS.single_wave(cdt), 500)
        u = W[:, :ops.ne]
        pl = np.linalg.norm(u @ S.P["PLH"].T, axis=1)
        ps = np.linalg.norm(u @ S.P["PS"].T, axis=1)
        i = int(np.argmax(pl))
        cur = O.recover(S, W)
        ratios_u.append(ps[i] / pl[i])
        ratios_j.append(np.linalg.norm(cur["j_star"][i]) / np.linalg.norm(cur["j_loop"][i]))
    assert max(ratios_u) / min(ratios_u) < 1.5 and min(ratios_u) > 0.01
    assert ratios_j[0] / ratios_j[1] == pytest.approx(10.0, rel=0.1)
    assert ratios_j[1] / ratios_j[2] == pytest.approx(100.0, rel=0.1)


def test_mie_series_far_field():
    """Far field of the Fourier-transformed currents against the Mie series for a
    dielectric sphere (eps_r = 2), icosphere L2, c dt = 0.1, at ka = 0.5 and 1
    (Section VI-C). |E_theta| in the E-plane vs |S2|/k, |E_phi| in the H-plane
    vs |S1|/k, within 6 % of the peak."""
    m = MS.icosphere(2)
    ops = assemble(m, 2.0, 1.0, 0.1)
    S = O.build_system(ops)
    exc = MS.single_wave(0.1)
    n = 800
    W = O.march(S, exc, n)
    cur = O.recover(S, W)
    th = np.linspace(0.02, np.pi - 0.02, 25)
    for ka in (0.5, 1.0):
        dw = FF.dft_weights(ka, ops.dt, n)
        J = (cur["j_loop"].T @ dw) + (cur["j_star"].T @ dw)
        M = (cur["m_loop"].T @ dw) + (cur["m_star"].T @ dw)
        spec = FF.pulse_spectrum(exc, 0, ka)
        d1 = np.stack([np.sin(th), 0 * th, np.cos(th)], 1)
        t1 = np.stack([np.cos(th), 0 * th, -np.sin(th)], 1)
        Eth = np.abs(np.einsum("ad,ad->a", FF.far_field(ops.rwg, J, M, ka, 1.0, d1) / spec, t1))
        d2 = np.stack([0 * th, np.sin(th), np.cos(th)], 1)
        Eph = np.abs(FF.far_field(ops.rwg, J, M, ka, 1.0, d2)[:, 0] / spec)
        S1, S2 = FF.mie_amplitudes(ka, math.sqrt(2.0), th)
        assert np.abs(Eth - np.abs(S2) / ka).max() < 0.06 * (np.abs(S2) / ka).max()
        assert np.abs(Eph - np.abs(S1) / ka).max() < 0.06 * (np.abs(S1) / ka).max()


def test_mie_coefficients_rayleigh_limit():
    """Small-x Mie: S1 -> (3/2) a_1 with a_1 ~ -(2i/3) x^3 (m^2-1)/(m^2+2)."""
    x, mr = 1e-3, math.sqrt(3.0)
    S1, S2 = FF.mie_amplitudes(x, mr, np.array([0.3]))
    assert abs(abs(S1[0]) - x ** 3 * (mr ** 2 - 1) / (mr ** 2 + 2)) < 1e-6 * x ** 3


def test_rayleigh_limit_far_field():
    """Large time step (c dt = 50, k_max = 1): the low-frequency far field of a
    dielectric sphere is the Rayleigh dipole |E_theta| = k^2 a^3 (eps-1)/(eps+2)
    |cos theta|, symmetric about 90 degrees (Section VI-C, 1e-5 Hz case); a is
    the volume-equivalent radius of the mesh."""
    m = MS.icosphere(2)
    ops = assemble(m, 2.0, 1.0, 50.0)
    S = O.build_system(ops)
    exc = MS.single_wave(50.0)
    n = 700
    W = O.march(S, exc, n)
    cur = O.recover(S, W)
    v = m.verts[m.tris]
    vol = np.einsum("fi,fi->f", v[:, 0], np.cross(v[:, 1], v[:, 2])).sum() / 6
    a = (3 * vol / (4 * math.pi)) ** (1 / 3)
    w = 1e-3
    dw = FF.dft_weights(w, ops.dt, n)
    J = (cur["j_loop"].T @ dw) + (cur["j_star"].T @ dw)
    M = (cur["m_loop"].T @ dw) + (cur["m_star"].T @ dw)
    th = np.linspace(0.05, math.pi - 0.05, 13)
    d1 = np.stack([np.sin(th), 0 * th, np.cos(th)], 1)
    t1 = np.stack([np.cos(th), 0 * th, -np.sin(th)], 1)
    Eth = np.abs(np.einsum("ad,ad->a", FF.far_field(ops.rwg, J, M, w, 1.0, d1) / FF.pulse_spectrum(exc, 0, w), t1))
    ref = w ** 2 * a ** 3 * (2 - 1) / (2 + 2) * np.abs(np.cos(th))
    assert np.abs(Eth - ref).max() < 0.05 * ref.max()
    assert np.abs(Eth - Eth[::-1]).max() < 0.02 * ref.max()


def test_product_form_oracle_matches_dense(pr1_ops, pr1_system):
    """The product-form oracle (used for meshes too large for dense Q_k) follows
    the same definition: it reproduces the dense oracle on PR1 to 1e-10."""
    from oracle import product as P
    exc = MS.single_wave(pr1_ops.dt, 30, 60)
    ref = O.march(pr1_system, exc, 60)
    W = P.ProductSystem(pr1_ops).march(exc, 60)
    assert np.abs(W - ref).max() < 1e-10 * np.abs(ref).max()


@pytest.mark.parametrize("case", ["torus12x6", "cube6"])
def test_product_form_oracle_matches_dense_where_used(case):
    """The product-form oracle is the checker of the full-size runs (torus,
    cube); pinned against the dense oracle in those regimes: the genus-1 torus
    (loop space with two global loops, 53 history lags, the K~ tail over many
    lags) for 130 steps and the non-smooth cube (35 lags) for 100 steps, both
    with the pulse inside the run, to 1e-10 of the run's peak."""
    from oracle import product as P
    from paper_2510_07989_gb300.inputs.assemble import assemble
    if case == "torus12x6":
        ops = assemble(MS.torus(1.0, 0.3, 12, 6), 4.0, 1.0, 0.1)
        assert ops.kmax == 52
        exc, n = MS.fibonacci_batch(2, 0.1, w_steps=30, t0_steps=60, r_obj=1.3), 130
    else:
        ops = assemble(MS.cube(2.0, 6), 6.0, 1.0, 0.25)
        assert ops.kmax == 34
        exc, n = MS.fibonacci_batch(2, 0.25, w_steps=30, t0_steps=60, r_obj=3 ** 0.5), 100
    S = O.build_system(ops)
    b = 1  # the second Fibonacci wave: oblique incidence, seeded polarisation
    ref = O.march(S, exc, n, b=b)
    W = P.ProductSystem(ops).march(exc, n, b=b)
    assert np.abs(W - ref).max() < 1e-10 * np.abs(ref).max()


def test_calderon_kernel_changes_q0_not_the_march(pr1_ops, pr1_system):
    """Section IV-A remark: the static EFIO T_0 of the Calderon preconditioner
    may be replaced by the EFIO T_{-i kappa} with an imaginary wavenumber.
    The preconditioner enters only the left factor [M1 | M2] (Section V-B),
    whose two terms map onto complementary ranges (P^{Sigma H} and P^Lambda)
    through invertible T^{Sigma H}, T^Lambda, so the equations it combines --
    and hence the discrete solution -- do not depend on the kernel: the march
    with T_{-i kappa} (kappa = 1/m on PR1) equals the one with T_0 to rounding
    while Q_0 itself differs by percents, its condition number stays ~34,
    and the companion spectrum keeps its radius."""
    from paper_2510_07989_gb300.inputs.assemble import assemble
    ops_k = assemble(MS.icosphere(1), 2.0, 1.0, 0.2, kappa=1.0)
    Sk = O.build_system(ops_k)
    dq = np.abs(Sk.Q[0] - pr1_system.Q[0]).max() / np.abs(pr1_system.Q[0]).max()
    assert dq > 1e-2
    c0, ck = np.linalg.cond(pr1_system.Q[0]), np.linalg.cond(Sk.Q[0])
    assert ck < 40 and abs(ck - c0) < 0.1 * c0
    exc = MS.single_wave(pr1_ops.dt, 30, 60)
    n = 400
    W0 = O.march(pr1_system, exc, n)
    Wk = O.march(Sk, exc, n)
    peak = np.abs(W0).max()
    assert np.abs(Wk - W0).max() < 1e-12 * peak
    assert np.abs(Wk[-50:]).max() < 1e-14 * peak  # decays as the static case (Section VI-A)
    r0 = np.abs(np.linalg.eigvals(O.companion(pr1_system))).max()
    rk = np.abs(np.linalg.eigvals(O.companion(Sk))).max()
    assert rk < 1 and abs(rk - r0) < 1e-8


def test_star_pyramid_late_time_stability():
    """Section VI-A, third example: on the non-smooth star-based pyramid
    (sharp tips and edges; eps_r = 5 as in the paper; stand-in geometry with
    80 triangles, c dt = 0.2, k_max = 22) the qHP march decays without bound
    -- below 1e-14 of its peak after 400 steps -- and the companion spectrum
    lies strictly inside the unit circle with no eigenvalue near 1 + 0i."""
    from paper_2510_07989_gb300.inputs.assemble import assemble
    M = MS.star_pyramid(5, m=2)
    ops = assemble(M, 5.0, 1.0, 0.2)
    S = O.build_system(ops)
    exc = MS.single_wave(ops.dt, 30, 60, r_obj=MS.diameter(M) / 2)
    W = O.march(S, exc, 600)
    peak = np.abs(W).max()
    tail = [np.abs(W[k:k + 50]).max() / peak for k in (300, 400, 550)]
    assert tail[0] > tail[1] > tail[2] and tail[1] < 1e-14
    ev = np.linalg.eigvals(O.companion(S))
    assert np.abs(ev).max() < 0.95
    assert np.abs(ev - 1).min() > 0.1


def test_extended_precision_oracle_matches_the_oracle(pr1_ops, pr1_system):
    """oracle.extended evaluates the same definition in long double; where the
    FP64 oracle is accurate (PR1, 200 steps through the pulse) the two agree
    to FP64 rounding."""
    from oracle import extended as X
    exc = MS.single_wave(pr1_ops.dt, 30, 60)
    n = 200
    ref = O.march(pr1_system, exc, n)
    W = X.ExtendedSystem(pr1_ops).march(exc, n).astype(np.float64)
    assert np.abs(W - ref).max() < 1e-12 * np.abs(ref).max()


def test_star_pyramid80_reference_is_reproduced():
    """The stored extended-precision march of the 80-triangle pyramid
    (tests/golden/star_pyramid80_extended.txt) is what its generator computes
    from the seeded inputs with oracle.extended (to 1e-13 of the peak)."""
    import importlib.util
    import os
    here = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")
    spec = importlib.util.spec_from_file_location("mk", os.path.join(here, "make_star_pyramid80.py"))
    mk = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mk)
    _, W = mk.compute()
    rows = [ln.split() for ln in open(os.path.join(here, "star_pyramid80_extended.txt")) if ln[:1] in ("p", "w")]
    peak = float(rows[0][1])
    assert abs(float(np.abs(W).max()) - peak) < 1e-13 * peak
    vals = [(int(i), int(j), float(v)) for _, i, j, v in rows[1:]]
    assert len(vals) == len(mk.STEPS) * len(mk.UNKNOWNS)
    assert max(abs(float(W[i - 1, j]) - v) for i, j, v in vals) < 1e-13 * peak


def test_companion_arnoldi_matches_the_dense_spectrum():
    """The matrix-free Arnoldi evaluation of the companion spectrum (for
    meshes too large for a dense eigendecomposition) gives the dense
    spectral radius (PR1 mesh at c dt = 0.5)."""
    ops = assemble(MS.icosphere(1), 2.0, 1.0, 0.5)
    S = O.build_system(ops)
    dense = np.abs(np.linalg.eigvals(O.companion(S))).max()
    top = np.abs(O.companion_top_eigenvalues(S, k=2, tol=1e-10)).max()
    assert abs(top - dense) < 1e-8 * dense


def test_torus_companion_spectrum_inside_unit_circle():
    """Section VI-A, second example: the multiply-connected torus is stable
    under the qHP formulation. Torus 10 x 5 (genus 1: two global loops in
    the loop space), eps_r = 4, c dt = 0.1 (k_max = 52, companion dimension
    53 x 300): the largest eigenvalues stay strictly inside the unit circle
    (radius ~0.987) and away from 1 + 0i, so no eigenvalue lies within
    1 - radius of 1."""
    ops = assemble(MS.torus(1.0, 0.3, 10, 5), 4.0, 1.0, 0.1)
    assert ops.kmax == 52
    top = O.companion_top_eigenvalues(O.build_system(ops), k=2)
    radius = np.abs(top).max()
    assert radius < 0.995
    assert np.abs(top - 1).min() > 0.1

