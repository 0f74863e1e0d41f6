"""Barycentric refinement, Buffa-Christiansen (BC) dual basis, triangle
quadrature tables and the mixed Gram matrix G (paper Section III).

Input-generator module: geometry and basis bookkeeping, shared by the CUDA path
and the oracle.

BC functions. The paper (Section III, Fig. 2) takes the BC functions as linear
combinations of RWG functions on the barycentric refinement without printing
the coefficients. They are built here from a flux balance:
  * every RWG used below carries unit total flux across its edge (the paper's RWG
    has no edge-length factor, Section II);
  * the BC function g_n of edge e_n = (v^-, v^+) carries flux 1 from the dual cell
    D(v^-) into the dual cell D(v^+), half across each of the two refined edges
    (edge midpoint, centroid of c^+/c^-) that make up the dual edge;
  * inside D(v) (the 2 d_v refined triangles touching v) every refined triangle
    is a source (v = v^-) or sink (v = v^+) of 1/(2 d_v);
  * the two refined half-edges of e_n carry no flux.
Walking around v from the half-edge of e_n, the radiating refined edge number k
(k = 1 .. 2 d_v - 1) then carries (d_v - k) / (2 d_v), the classical BC weights.
Consequences used by the method: div g_n = -sum_v Lambda_{nv} phi_v with a fixed
density phi_v per dual cell, so Sigma-combinations of BC functions are
divergence free (BC loops) and Lambda-combinations carry the charge (BC stars).
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np

from .meshes import Mesh


# ----------------------------------------------------------------------------
# symmetric triangle rules: barycentric points and weights summing to 1
# ----------------------------------------------------------------------------

def triangle_rule(npts: int):
    """Symmetric Gauss rules on a triangle: 1 (degree 1), 3 (degree 2),
    4 (degree 3), 6 (degree 4, Dunavant), 7 (degree 5, Radon)."""
    if npts == 1:
        return np.array([[1 / 3, 1 / 3, 1 / 3]]), np.array([1.0])
    if npts == 3:
        a, b = 2 / 3, 1 / 6
        return np.array([[a, b, b], [b, a, b], [b, b, a]]), np.full(3, 1 / 3)
    if npts == 4:
        return (np.array([[1 / 3, 1 / 3, 1 / 3], [0.6, 0.2, 0.2], [0.2, 0.6, 0.2], [0.2, 0.2, 0.6]]),
                np.array([-27 / 48, 25 / 48, 25 / 48, 25 / 48]))
    if npts == 6:
        a, wa = 0.445948490915965, 0.223381589678011
        b, wb = 0.091576213509771, 0.109951743655322
        pts = [[a, a, 1 - 2 * a], [a, 1 - 2 * a, a], [1 - 2 * a, a, a],
               [b, b, 1 - 2 * b], [b, 1 - 2 * b, b], [1 - 2 * b, b, b]]
        return np.array(pts), np.array([wa] * 3 + [wb] * 3)
    if npts == 7:
        s15 = math.sqrt(15.0)
        a1, w1 = (6 - s15) / 21, (155 - s15) / 1200
        a2, w2 = (6 + s15) / 21, (155 + s15) / 1200
        pts = [[1 / 3, 1 / 3, 1 / 3],
               [a1, a1, 1 - 2 * a1], [a1, 1 - 2 * a1, a1], [1 - 2 * a1, a1, a1],
               [a2, a2, 1 - 2 * a2], [a2, 1 - 2 * a2, a2], [1 - 2 * a2, a2, a2]]
        return np.array(pts), np.array([9 / 40] + [w1] * 3 + [w2] * 3)
    raise ValueError(f"no {npts}-point triangle rule")


def tri_geometry(P: np.ndarray):
    """P (n, 3, 3): areas (n,), unit normals (n, 3)."""
    cr = np.cross(P[:, 1] - P[:, 0], P[:, 2] - P[:, 0])
    nrm = np.linalg.norm(cr, axis=1)
    return 0.5 * nrm, cr / nrm[:, None]


@dataclass
class RWGTable:
    """Quadrature table of the RWG test functions (paper Section II):
    x (ne, 2 nq, 3) points on c^+ then c^-, wf (ne, 2 nq, 3) = weight * area *
    f_m(x); [<f_m, a>] ~ sum_q wf_q . a(x_q)."""
    x: np.ndarray
    wf: np.ndarray


def rwg_table(mesh: Mesh, nq: int = 7) -> RWGTable:
    bary, w = triangle_rule(nq)
    V, T = mesh.verts, mesh.tris
    xs, wfs = [], []
    for side in (0, 1):
        f = mesh.ef[:, side]
        P = V[T[f]]                       # (ne, 3, 3)
        A, _ = tri_geometry(P)
        X = np.einsum("qk,ekd->eqd", bary, P)
        o = V[mesh.eo[:, side]]           # opposite vertex x^+ or x^-
        sgn = 1.0 if side == 0 else -1.0  # (x - x^+)/(2A) on c^+, (x^- - x)/(2A) on c^-
        fval = sgn * (X - o[:, None, :]) / (2 * A)[:, None, None]
        xs.append(X)
        wfs.append(fval * (w[None, :, None] * A[:, None, None]))
    return RWGTable(np.concatenate(xs, axis=1), np.concatenate(wfs, axis=1))


# ----------------------------------------------------------------------------
# barycentric refinement and BC functions
# ----------------------------------------------------------------------------

@dataclass
class DualBasis:
    ref_pts: np.ndarray    # (nr, 3, 3) refined triangle corners (v, a, b)
    ref_face: np.ndarray   # (nr,) parent primal face
    ref_vert: np.ndarray   # (nr,) dual cell (primal vertex) the triangle belongs to
    ref_area: np.ndarray   # (nr,)
    ref_normal: np.ndarray  # (nr, 3)
    degree: np.ndarray     # (nv,) number of faces around each primal vertex
    # BC function restricted to refined triangle: g_n(x) = alpha x + beta
    bc_n: np.ndarray       # (nb,) BC function (edge) index
    bc_t: np.ndarray       # (nb,) refined triangle index
    bc_alpha: np.ndarray   # (nb,)
    bc_beta: np.ndarray    # (nb, 3)

    @property
    def nref(self) -> int:
        return int(self.ref_pts.shape[0])


def _one_rings(mesh: Mesh):
    """For every vertex: neighbours u_0..u_{d-1} and faces F_i = (v, u_i, u_{i+1})
    in counter-clockwise order seen from outside."""
    nxt = [dict() for _ in range(mesh.nv)]
    for f, (a, b, c) in enumerate(mesh.tris):
        for (v, x, y) in ((a, b, c), (b, c, a), (c, a, b)):
            nxt[v][int(x)] = (int(y), f)
    rings = []
    for v in range(mesh.nv):
        d = nxt[v]
        start = next(iter(d))
        us, fs = [start], []
        u = start
        while True:
            y, f = d[u]
            fs.append(f)
            if y == start:
                break
            us.append(y)
            u = y
        if len(us) != len(d):
            raise ValueError(f"vertex {v} is not a manifold vertex")
        rings.append((us, fs))
    return rings


def dual_basis(mesh: Mesh) -> DualBasis:
    V = mesh.verts
    T = mesh.tris
    cen = V[T].mean(axis=1)
    edge_id = {}
    for e, (a, b) in enumerate(mesh.ev):
        edge_id[(int(a), int(b))] = e
        edge_id[(int(b), int(a))] = e
    mid = 0.5 * (V[mesh.ev[:, 0]] + V[mesh.ev[:, 1]])
    rings = _one_rings(mesh)
    ref_pts, ref_face, ref_vert = [], [], []
    cell_tris = []          # per vertex: refined triangle ids t_0 .. t_{2d-1}
    cell_ends = []          # per vertex: far ends of radiating edges r_0 .. r_{2d-1}
    for v, (us, fs) in enumerate(rings):
        d = len(us)
        ends = []
        for i in range(d):
            ends.append(mid[edge_id[(v, us[i])]])
            ends.append(cen[fs[i]])
        ids = []
        for k in range(2 * d):
            f = fs[k // 2]
            ref_pts.append([V[v], ends[k], ends[(k + 1) % (2 * d)]])
            ref_face.append(f)
            ref_vert.append(v)
            ids.append(len(ref_pts) - 1)
        cell_tris.append(ids)
        cell_ends.append(ends)
    ref_pts = np.array(ref_pts)
    ref_area, ref_normal = tri_geometry(ref_pts)
    deg = np.array([len(r[0]) for r in rings])

    bc_n, bc_t, bc_a, bc_b = [], [], [], []
    for n, (vm, vp) in enumerate(mesh.ev):
        for v, other, sgn in ((int(vm), int(vp), 1.0), (int(vp), int(vm), -1.0)):
            us, _ = rings[v]
            d = len(us)
            j = us.index(other)
            ids = cell_tris[v]
            ends = cell_ends[v]
            # radiating-edge fluxes in the cycle started at the half-edge of e_n
            G = np.array([0.0] + [sgn * (d - k) / (2 * d) for k in range(1, 2 * d)] + [0.0])
            for k in range(2 * d):
                kk = (2 * j + k) % (2 * d)
                t = ids[kk]
                Pk = ends[kk]
                Pk1 = ends[(kk + 1) % (2 * d)]
                out_b = sgn * 0.5 if k in (0, 2 * d - 1) else 0.0
                out_r0 = G[k]          # through (v, P_k), opposite corner P_{k+1}
                out_r1 = -G[k + 1]     # through (v, P_{k+1}), opposite corner P_k
                A2 = 2 * ref_area[t]
                alpha = (out_b + out_r0 + out_r1) / A2
                beta = -(out_b * V[v] + out_r0 * Pk1 + out_r1 * Pk) / A2
                bc_n.append(n)
                bc_t.append(t)
                bc_a.append(alpha)
                bc_b.append(beta)
    return DualBasis(ref_pts=ref_pts, ref_face=np.array(ref_face), ref_vert=np.array(ref_vert),
                     ref_area=ref_area, ref_normal=ref_normal, degree=deg,
                     bc_n=np.array(bc_n, dtype=np.int64), bc_t=np.array(bc_t, dtype=np.int64),
                     bc_alpha=np.array(bc_a), bc_beta=np.array(bc_b))


def gram_matrix(mesh: Mesh, dual: DualBasis):
    """Mixed Gram matrix [G]_mn = <n x f_m, g_n> (paper Section III), as
    (rows, cols, vals) COO with duplicates summed by the caller. Exact: the
    integrand is quadratic on each refined triangle (3-point degree-2 rule)."""
    bary, w = triangle_rule(3)
    V, T = mesh.verts, mesh.tris
    # edges of each primal face with their RWG sign and opposite vertex
    face_edges = [[] for _ in range(mesh.nf)]
    for e in range(mesh.ne):
        for side, sgn in ((0, 1.0), (1, -1.0)):
            face_edges[mesh.ef[e, side]].append((e, sgn, mesh.eo[e, side]))
    prim_area, prim_n = tri_geometry(V[T])
    rows, cols, vals = [], [], []
    X = np.einsum("qk,tkd->tqd", bary, dual.ref_pts)      # (nr, 3, 3)
    for b in range(dual.bc_n.size):
        t = dual.bc_t[b]
        F = dual.ref_face[t]
        g = dual.bc_alpha[b] * X[t] + dual.bc_beta[b][None, :]   # (3 pts, 3)
        wA = w * dual.ref_area[t]
        for (m, sgn, o) in face_edges[F]:
            f = sgn * (X[t] - V[o][None, :]) / (2 * prim_area[F])
            nxf = np.cross(prim_n[F][None, :], f)
            rows.append(m)
            cols.append(dual.bc_n[b])
            vals.append(float(np.sum(wA * np.einsum("qd,qd->q", nxf, g))))
    return np.array(rows), np.array(cols), np.array(vals)


@dataclass
class BCTable:
    """Quadrature table of the BC functions: for entry i, point x[i], weight *
    area * g_{n[i]}(x[i]); <g_n, a> ~ sum over entries with that n."""
    n: np.ndarray
    x: np.ndarray
    wg: np.ndarray


def bc_table(dual: DualBasis, nq: int = 3) -> BCTable:
    bary, w = triangle_rule(nq)
    X = np.einsum("qk,tkd->tqd", bary, dual.ref_pts)
    xs = X[dual.bc_t]                                   # (nb, nq, 3)
    g = dual.bc_alpha[:, None, None] * xs + dual.bc_beta[:, None, :]
    wg = g * (w[None, :, None] * dual.ref_area[dual.bc_t][:, None, None])
    return BCTable(np.repeat(dual.bc_n, nq), xs.reshape(-1, 3), wg.reshape(-1, 3))
