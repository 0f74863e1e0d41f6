"""Pins of the input generators (meshes, canonical topology, BC dual basis,
operator assembly) against what the paper and the mathematics fix."""
import numpy as np
import pytest
import scipy.sparse as sp

from paper_2510_07989_gb300.inputs import meshes as MS
from paper_2510_07989_gb300.inputs.dual import dual_basis, gram_matrix, triangle_rule


@pytest.mark.parametrize("make,counts,chi", [
    (lambda: MS.icosphere(1), (42, 80, 120), 2),
    (lambda: MS.icosphere(3), (642, 1280, 1920), 2),
    (lambda: MS.torus(1.0, 0.3, 64, 24), (1536, 3072, 4608), 0),
    (lambda: MS.cube(2.0, 24), (3458, 6912, 10368), 2),
    (lambda: MS.geodesic_sphere(5), (252, 500, 750), 2),
    (lambda: MS.star_pyramid(5, m=11), (1212, 2420, 3630), 2),
    (lambda: MS.star_pyramid(5, m=2), (42, 80, 120), 2),
])
def test_mesh_counts_euler(make, counts, chi):
    """Counts of the configured workloads; V - E + F = 2 (sphere) or 0 (torus); E = 3F/2."""
    m = make()
    assert (m.nv, m.nf, m.ne) == counts
    assert m.nv - m.ne + m.nf == chi
    assert 2 * m.ne == 3 * m.nf


@pytest.mark.parametrize("n_points,m", [(5, 2), (5, 11), (3, 4), (7, 3)])
def test_star_pyramid_geometry(n_points, m):
    """The star-based pyramid is closed and outward oriented: its signed volume
    (sum of v0 . (v1 x v2) / 6) equals the analytic n r_tip r_inner
    sin(pi / n) h / 3 (base of 2n triangles (origin, c_j, c_j+1), cone of
    height h); its area equals the 4n flat faces' areas from their corners
    (the uniform split loses nothing); every vertex lies on one of those
    faces; the base is flat at z = 0 and the apex is the highest point."""
    r_tip, r_in, h = 1.0, 0.4, 1.0
    M = MS.star_pyramid(n_points, r_tip, r_in, h, m)
    v0, v1, v2 = (M.verts[M.tris[:, k]] for k in range(3))
    vol = np.einsum("ij,ij->i", v0, np.cross(v1, v2)).sum() / 6
    assert vol == pytest.approx(n_points * r_tip * r_in * np.sin(np.pi / n_points) * h / 3, rel=1e-12)
    area = 0.5 * np.linalg.norm(np.cross(v1 - v0, v2 - v0), axis=1).sum()
    nc = 2 * n_points
    ang = np.pi * np.arange(nc) / n_points
    rad = np.where(np.arange(nc) % 2 == 0, r_tip, r_in)
    C = np.stack([rad * np.cos(ang), rad * np.sin(ang), np.zeros(nc)], axis=1)
    apex = np.array([0.0, 0.0, h])
    big = 0.0
    for j in range(nc):
        c0, c1 = C[j], C[(j + 1) % nc]
        big += 0.5 * np.linalg.norm(np.cross(c0 - apex, c1 - apex)) + 0.5 * np.linalg.norm(np.cross(c0, c1))
    assert area == pytest.approx(big, rel=1e-12)
    assert M.verts[:, 2].min() == pytest.approx(0.0, abs=1e-15) and M.verts[:, 2].max() == pytest.approx(h)
    assert M.nf == 4 * n_points * m * m and M.nv == 2 * n_points * m * m + 2


def test_canonical_edge_rule():
    """v^- < v^+; c^+ traverses v^- -> v^+ counter-clockwise (lies left of the
    edge seen from outside); x^+/x^- are the opposite vertices."""
    m = MS.torus(1.0, 0.3, 12, 8)
    assert np.all(m.ev[:, 0] < m.ev[:, 1])
    for e in range(m.ne):
        a, b = m.ev[e]
        fp, fm = m.ef[e]
        tp, tm = list(m.tris[fp]), list(m.tris[fm])
        i = tp.index(a)
        assert tp[(i + 1) % 3] == b and tp[(i + 2) % 3] == m.eo[e, 0]
        j = tm.index(b)
        assert tm[(j + 1) % 3] == a and tm[(j + 2) % 3] == m.eo[e, 1]
    # outward orientation: signed volume > 0
    v = m.verts[m.tris]
    vol = np.einsum("fi,fi->f", v[:, 0], np.cross(v[:, 1], v[:, 2])).sum() / 6
    assert vol > 0


@pytest.mark.parametrize("make", [lambda: MS.icosphere(2), lambda: MS.torus(1.0, 0.3, 16, 8), lambda: MS.cube(2.0, 4)])
def test_incidence_orthogonality(make):
    """Sigma^T Lambda = 0 exactly, in integers (Section IV-B)."""
    m = make()
    ne = m.ne
    L = sp.csr_matrix((np.r_[np.ones(ne), -np.ones(ne)], (np.r_[np.arange(ne), np.arange(ne)], np.r_[m.ev[:, 1], m.ev[:, 0]])),
                      shape=(ne, m.nv), dtype=np.int64)
    S = sp.csr_matrix((np.r_[np.ones(ne), -np.ones(ne)], (np.r_[np.arange(ne), np.arange(ne)], np.r_[m.ef[:, 0], m.ef[:, 1]])),
                      shape=(ne, m.nf), dtype=np.int64)
    assert (S.T @ L).count_nonzero() == 0


def test_triangle_rules_exactness():
    """Each rule integrates monomials up to its degree exactly on the reference
    triangle (int x^a y^b = a! b! / (a+b+2)!)."""
    from math import factorial
    for n, deg in ((1, 1), (3, 2), (4, 3), (6, 4), (7, 5)):
        bary, w = triangle_rule(n)
        x, y = bary[:, 1], bary[:, 2]
        for a in range(deg + 1):
            for b in range(deg + 1 - a):
                exact = factorial(a) * factorial(b) / factorial(a + b + 2)
                assert abs(0.5 * np.sum(w * x ** a * y ** b) - exact) < 1e-13


@pytest.mark.parametrize("level", [1, 2, 3])
def test_gram_well_conditioned(level):
    """G = <n x f_m, g_n> is sparse, has a positive diagonal and is well
    conditioned independently of the mesh level (Section III)."""
    m = MS.icosphere(level)
    d = dual_basis(m)
    r, c, v = gram_matrix(m, d)
    G = sp.coo_matrix((v, (r, c)), shape=(m.ne, m.ne)).toarray()
    s = np.linalg.svd(G, compute_uv=False)
    assert np.all(np.diag(G) > 0)
    assert s[0] / s[-1] < 4.0


def test_bc_loops_divergence_free_and_charge():
    """Sigma-combinations of BC functions are divergence free (BC loops) and the
    divergence of every BC function integrates to zero (Section IV-A)."""
    m = MS.torus(1.0, 0.3, 12, 8)
    d = dual_basis(m)
    div = sp.coo_matrix((2 * d.bc_alpha * d.ref_area[d.bc_t], (d.bc_n, d.bc_t)), shape=(m.ne, d.nref)).toarray()
    S = np.zeros((m.ne, m.nf))
    S[np.arange(m.ne), m.ef[:, 0]] = 1
    S[np.arange(m.ne), m.ef[:, 1]] = -1
    assert np.abs(S.T @ div).max() < 1e-12
    assert np.abs(div.sum(axis=1)).max() < 1e-12


def test_static_operators_definiteness(pr1_ops):
    """T_0^s SPD; T_0^h PSD of rank N_v - 1 on the BC space (Section III)."""
    ops = pr1_ops
    es = np.linalg.eigvalsh(ops.T0s)
    eh = np.linalg.eigvalsh(ops.T0h)
    assert es[0] > 0
    assert eh[0] > -1e-12 * eh[-1]
    assert int((eh > 1e-10 * eh[-1]).sum()) == ops.mesh.nv - 1


@pytest.fixture(scope="module")
def yukawa_static():
    """T_0^s, T_0^h of the icosphere L2 (480 edges, D = 2) with the static
    kernel 1/R and with exp(-kappa R)/R for kappa = 0.5 and 2 (the EFIO with
    the imaginary wavenumber -i kappa of the Section IV-A remark)."""
    from paper_2510_07989_gb300.inputs.assemble import _static
    from paper_2510_07989_gb300.inputs.meshes import diameter
    m = MS.icosphere(2)
    dual = dual_basis(m)
    D = diameter(m)
    ops = {k: _static(m, dual, D, 3, 4, 4, 8, kappa=k) for k in (0.0, 0.5, 2.0)}
    return m, ops


def test_yukawa_kappa_zero_is_the_static_operator(yukawa_static):
    """kappa = 0 reproduces the static operators bit for bit."""
    from paper_2510_07989_gb300.inputs.assemble import _static
    from paper_2510_07989_gb300.inputs.meshes import diameter
    m, ops = yukawa_static
    T0s, T0h = _static(m, dual_basis(m), diameter(m), 3, 4, 4, 8)
    assert np.array_equal(T0s, ops[0.0][0]) and np.array_equal(T0h, ops[0.0][1])


def test_yukawa_operators_definite_and_below_the_static_ones(yukawa_static):
    """exp(-kappa R)/(4 pi R) is a positive definite kernel (Fourier transform
    1/(k^2 + kappa^2) > 0), and so is the difference to the static kernel
    (1/k^2 - 1/(k^2 + kappa^2) > 0): T^s_kappa is SPD and T_0^s - T^s_kappa
    PSD; T^h_kappa is PSD of rank N_v - 1 and T_0^h - T^h_kappa PSD. The
    differences are smoothing operators whose small eigenvalues sit at the
    quadrature error (~2e-5 of their largest for T^s; T^h's dual-cell single
    layer is exact to rounding here). A kernel with the wrong sign of the
    exponent makes the differences negative definite."""
    m, ops = yukawa_static
    T0s, T0h = ops[0.0]

    def psd(A, rel):
        e = np.linalg.eigvalsh(A)
        return e[-1] > 0 and e[0] > -rel * e[-1]

    for kappa in (0.5, 2.0):
        Ts, Th = ops[kappa]
        es, eh = np.linalg.eigvalsh(Ts), np.linalg.eigvalsh(Th)
        assert es[0] > 0
        assert eh[0] > -1e-12 * eh[-1] and int((eh > 1e-10 * eh[-1]).sum()) == m.nv - 1
        assert psd(T0s - Ts, 1e-4)
        assert psd(T0h - Th, 1e-12)
    # the larger the decay, the smaller the operator
    assert psd(ops[0.5][0] - ops[2.0][0], 1e-4) and psd(ops[0.5][1] - ops[2.0][1], 1e-12)


def test_yukawa_far_pairs_decay_as_the_kernel(yukawa_static):
    """For BC functions far apart (midpoint distance R > 0.9 D) the
    interaction is (integral of g_m) . (integral of g_n) times the kernel at
    R, so T^s_kappa / T_0^s -> exp(-kappa R): within 1 % (median 0.5 %) for
    kappa = 0.5 on the large entries. exp(-2 kappa R), exp(-kappa R / 4 pi) or
    exp(+kappa R) miss by 30 % or more."""
    m, ops = yukawa_static
    mid = 0.5 * (m.verts[m.ev[:, 0]] + m.verts[m.ev[:, 1]])
    R = np.linalg.norm(mid[:, None, :] - mid[None, :, :], axis=2)
    T0, T1 = ops[0.0][0], ops[0.5][0]
    far = R > 1.8
    sel = far & (np.abs(T0) > 0.3 * np.abs(T0[far]).max())
    assert sel.sum() > 1000
    dev = np.abs(T1[sel] / T0[sel] / np.exp(-0.5 * R[sel]) - 1)
    assert np.median(dev) < 5e-3 and dev.max() < 1e-2


def _lag_sum(mat, kmax_tail=None):
    ne = mat.ne
    out = np.zeros((ne, ne))
    rows = np.repeat(np.arange(ne), np.diff(mat.rowptr))
    for e in range(mat.col.size):
        out[rows[e], mat.col[e]] += mat.val[mat.voff[e]:mat.voff[e] + mat.cnt[e]].sum()
    return out


def _tail_dense(mat):
    ne = mat.ne
    out = np.zeros((ne, ne))
    rows = np.repeat(np.arange(ne), np.diff(mat.rowptr))
    out[rows, mat.col] = mat.tc
    return out


@pytest.mark.parametrize("med", ["", "p"])
def test_temporal_partition_identities(pr1_ops, med):
    """Sums over lags fixed by the temporal bases (Section V-A, V-B):
    sum_k h_0'(tau_k) = 0 -> sum_k T_k = 0; sum_k q_0'' = sum_k q_0' = 0 ->
    sum_k K^_k = 0; sum_k h_0(tau_k) = 1 -> sum_k K_k = K_0, which also equals
    (T_max/dt) times the constant tail of K~ (Section V-B-3)."""
    ops = pr1_ops
    sAT = _lag_sum(ops.mats["AT" + med])
    sHK = _lag_sum(ops.mats["HK" + med])
    sAK = _lag_sum(ops.mats["AK" + med])
    tail = _tail_dense(ops.mats["TK" + med]) * ops.tmax / ops.dt
    scale_T = np.abs(_lag_sum(ops.mats["TT" + med])).max() * ops.tmax / ops.dt
    assert np.abs(sAT).max() < 1e-12 * scale_T
    assert np.abs(sHK).max() < 1e-11 * np.abs(sAK).max() * ops.tmax / ops.dt
    assert np.abs(sAK - tail).max() < 1e-12 * np.abs(tail).max()


def test_lag_support_truncation(pr1_ops):
    """A_k vanishes for k > k_max, A^_k for k > k_max + 1, A~_k for k > k_max - 1
    (Section V-B); the K~ tail lies within lags <= k_max - 1."""
    ops = pr1_ops
    km = ops.kmax
    for med in ("", "p"):
        assert ops.mats["AT" + med].max_lag() <= km
        assert ops.mats["AK" + med].max_lag() <= km
        assert ops.mats["HT" + med].max_lag() <= km + 1
        assert ops.mats["HK" + med].max_lag() <= km + 1
        assert ops.mats["TT" + med].max_lag() <= km - 1
        assert ops.mats["TK" + med].max_lag() <= km - 1
    assert ops.kmax == 15 and ops.K == 16


def test_static_single_layer_symmetry(pr1_ops):
    """The lag sum of T~ is the static single layer (p_0 sums to one), which is
    symmetric in (m, n): a check of the quadrature accuracy."""
    s = _lag_sum(pr1_ops.mats["TT"])
    assert np.abs(s - s.T).max() < 2e-3 * np.abs(s).max()


def test_time_bases_against_the_paper_definitions():
    """The assembler's temporal factors (asm_time_weights, every temporal factor
    of its lag moments) against the definitions of Section V-A evaluated numerically:
    p_0 the unit pulse on (-dt, 0), h_0 the hat of half-width dt, q_0 the
    window average of h_0 over one step (Eq. (hq)); the lag-(j+i) factor of a
    basis b is b((i - phi) dt). Also q_0's peak 3/4 at dt/2, its C1 continuity
    at the knots, and the compatibility Eq. (ph) linking p_0 and h_0."""
    from paper_2510_07989_gb300.inputs.assemble import time_weights
    dt = 0.7
    p0 = lambda t: 1.0 if -dt < t < 0 else 0.0
    h0 = lambda t: max(0.0, 1.0 - abs(t) / dt)

    def integral(f, a, b, knots):
        """int_a^b f for f constant or linear between knots: midpoint rule per piece (exact)."""
        x = [a] + sorted(k for k in knots if a < k < b) + [b]
        return sum(f(0.5 * (x0 + x1)) * (x1 - x0) for x0, x1 in zip(x[:-1], x[1:]))

    q0 = lambda s: integral(h0, s - dt, s, (-dt, 0.0, dt)) / dt
    eps = 1e-4 * dt
    for phi in (0.05, 0.2, 0.37, 0.5, 0.63, 0.8, 0.95):
        w = time_weights(phi)
        xs = [(i - phi) * dt for i in range(3)]
        for i in range(3):  # q_0 values
            assert abs(w[5 + i] - q0(xs[i])) < 1e-13
        for i in range(2):  # dt h_0' (one-sided inside the linear piece)
            d = (h0(xs[i] + eps) - h0(xs[i] - eps)) / (2 * eps)
            assert abs(w[i] - dt * d) < 1e-9
        for i in range(3):  # dt^2 q_0'' (inside the quadratic piece)
            d2 = (q0(xs[i] + eps) - 2 * q0(xs[i]) + q0(xs[i] - eps)) / eps ** 2
            assert abs(w[2 + i] - dt * dt * d2) < 1e-4
        assert w[8] == p0(xs[0]) == 1.0 and p0(xs[1]) == 0.0
        for i in range(2):  # h_0 values
            assert abs(w[9 + i] - h0(xs[i])) < 1e-14
        for i in range(3):  # dt q_0'
            d = (q0(xs[i] + eps) - q0(xs[i] - eps)) / (2 * eps)
            assert abs(w[11 + i] - dt * d) < 1e-8
        for i in range(2):  # the ramp of the K~ tail, (1/dt) int_{-inf}^{x} p_0
            assert abs(w[14 + i] - integral(p0, -3 * dt, xs[i], (-dt, 0.0)) / dt) < 1e-14
    # peak of q_0: 3/4 at dt/2 (lag j+1 of phi = 1/2)
    assert abs(time_weights(0.5)[6] - 0.75) < 1e-15
    assert max(time_weights(phi)[6] for phi in np.linspace(0, 1, 201)) <= 0.75 + 1e-15
    # C1 at the knots: the factors at phi -> 1 continue those of the next lag at phi = 0
    lo, hi = time_weights(1 - 1e-9), time_weights(0.0)
    assert abs(lo[6] - hi[5]) < 1e-8 and abs(lo[7] - hi[6]) < 1e-8 and abs(lo[5]) < 1e-8
    dlo = (time_weights(1 - 1e-6) - time_weights(1 - 2e-6)) / 1e-6
    dhi = (time_weights(1e-6) - time_weights(0.0)) / 1e-6
    assert abs(dlo[6] - dhi[5]) < 1e-4 and abs(dlo[7] - dhi[6]) < 1e-4
    # Eq. (ph): (1/dt) int p_i(t) p_0(t + xi) dt = h_0(i dt + xi)
    for i in (0, 1, 2):
        for xi in (-1.3 * dt, -0.6 * dt, 0.0, 0.25 * dt, 0.9 * dt):
            lhs = integral(lambda t: p0(t - i * dt) * p0(t + xi), (i - 1) * dt, i * dt, (-xi, -dt - xi)) / dt
            assert abs(lhs - h0(i * dt + xi)) < 1e-12


def test_uneven_batch_recipe():
    """The uneven 24-scatterer batch: icospheres L1-L3 first, then 21
    ellipsoids with 540..7260 unknowns (geodesic frequency 3..11), semi-axes
    within [0.5, 1.5] (the diameter at most 3), eps_r within [1.5, 8];
    deterministic for a seed, different for another."""
    from paper_2510_07989_gb300.inputs import meshes as MS
    b = MS.uneven_batch(24)
    assert len(b) == 24
    assert [2 * m.ne for m, _ in b[:3]] == [240, 960, 3840]
    for m, eps in b:
        assert 1.5 <= eps <= 8.0
        assert m.nv - m.ne + m.nf == 2  # closed genus-0 surfaces
    for m, _ in b[3:]:
        n2 = 2 * m.ne
        assert 540 <= n2 <= 7260 and (n2 // 60) in {k * k for k in range(3, 12)}
        assert MS.diameter(m) <= 3.0 + 1e-9
    again = MS.uneven_batch(24)
    assert all(np.array_equal(m.verts, m2.verts) and e == e2 for (m, e), (m2, e2) in zip(b, again))
    other = MS.uneven_batch(24, seed=1)
    assert any(not np.array_equal(m.verts, m2.verts) for (m, _), (m2, _) in zip(b[3:], other[3:]) if m.nv == m2.nv) \
        or [m.nv for m, _ in b] != [m.nv for m, _ in other]


def test_widening_inputs_reject_bad_parameters():
    """The star pyramid needs n >= 3 tips, m >= 1, 0 < r_inner < r_tip and a
    positive height; the Yukawa decay must be >= 0 (kappa = 0 is T_0)."""
    from paper_2510_07989_gb300.inputs.assemble import assemble
    for kw in (dict(n_points=2), dict(m=0), dict(r_inner=1.0), dict(r_inner=0.0), dict(height=0.0)):
        with pytest.raises(ValueError):
            MS.star_pyramid(**kw)
    with pytest.raises(ValueError):
        assemble(MS.icosphere(1), 2.0, 1.0, 0.2, kappa=-1.0)
