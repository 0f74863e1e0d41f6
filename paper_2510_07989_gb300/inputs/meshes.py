"""Seeded synthetic workloads: closed triangle meshes, their canonical edge table,
and plane-wave excitation batches.

This module is an input generator. It holds geometry and bookkeeping only, none
of the MOT method's arithmetic, and is shared by the CUDA path and the oracle.

Geometries (paper Section VI, scatterers (a)-(c), stood in by the configured
synthetic shapes): icosphere of subdivision level L, geodesic frequency-n sphere
(for seeded ellipsoids), torus quad grid split along one diagonal, cube with an
n x n grid per face.

Canonical edge rule (paper Section IV-B defines Lambda and Sigma through an edge
orientation v^- -> v^+ and the RWG flow c^+ -> c^-, Section II / Fig. 1):
  * edges are the unique vertex pairs (a, b) with a < b, sorted lexicographically;
  * v^- = a, v^+ = b;
  * c^+ is the triangle lying to the left of a -> b seen from outside (its
    counter-clockwise traversal visits a then b), c^- is the other one;
  * x^+ / x^- are the vertices of c^+ / c^- opposite to the edge.
With this rule Sigma^T Lambda = 0 holds exactly in integers.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np


@dataclass
class Mesh:
    verts: np.ndarray          # (nv, 3) float64
    tris: np.ndarray           # (nf, 3) int32, counter-clockwise seen from outside
    name: str = "mesh"
    # canonical edge table, filled by build_edges()
    ev: np.ndarray = field(default=None)    # (ne, 2) int32: v^-, v^+
    ef: np.ndarray = field(default=None)    # (ne, 2) int32: c^+, c^-
    eo: np.ndarray = field(default=None)    # (ne, 2) int32: x^+, x^- (opposite vertex ids)

    @property
    def nv(self) -> int:
        return int(self.verts.shape[0])

    @property
    def nf(self) -> int:
        return int(self.tris.shape[0])

    @property
    def ne(self) -> int:
        return int(self.ev.shape[0])


def build_edges(mesh: Mesh) -> Mesh:
    """Fill mesh.ev / ef / eo by the canonical rule; raise if not a closed,
    consistently oriented 2-manifold."""
    tris = mesh.tris.astype(np.int64)
    nf = tris.shape[0]
    # directed edges (a->b) with their face and opposite vertex
    a = tris[:, [0, 1, 2]].reshape(-1)
    b = tris[:, [1, 2, 0]].reshape(-1)
    o = tris[:, [2, 0, 1]].reshape(-1)
    f = np.repeat(np.arange(nf), 3)
    nvv = int(mesh.verts.shape[0])
    key = a * nvv + b
    if np.unique(key).size != key.size:
        raise ValueError("mesh has a repeated directed edge (non-manifold or inconsistent orientation)")
    order = np.argsort(key)
    key_sorted = key[order]
    rev = b * nvv + a
    pos = np.searchsorted(key_sorted, rev)
    ok = (pos < key.size) & (key_sorted[np.minimum(pos, key.size - 1)] == rev)
    if not np.all(ok):
        raise ValueError("mesh is open or inconsistently oriented: a directed edge has no reverse")
    partner = order[pos]
    fwd = a < b  # keep the direction a<b: that face is c^+ (face left of a->b)
    idx = np.nonzero(fwd)[0]
    ev = np.stack([a[idx], b[idx]], axis=1)
    srt = np.lexsort((ev[:, 1], ev[:, 0]))
    idx = idx[srt]
    ev = ev[srt]
    ef = np.stack([f[idx], f[partner[idx]]], axis=1)
    eo = np.stack([o[idx], o[partner[idx]]], axis=1)
    mesh.ev = ev.astype(np.int32)
    mesh.ef = ef.astype(np.int32)
    mesh.eo = eo.astype(np.int32)
    if 2 * mesh.ev.shape[0] != 3 * nf:
        raise ValueError("edge count is not 3F/2")
    return mesh


def _orient_outward(verts, tris, center_fn):
    """Flip triangles whose normal points toward center_fn(centroid)."""
    v0, v1, v2 = verts[tris[:, 0]], verts[tris[:, 1]], verts[tris[:, 2]]
    nrm = np.cross(v1 - v0, v2 - v0)
    cen = (v0 + v1 + v2) / 3.0
    out = cen - center_fn(cen)
    flip = np.einsum("ij,ij->i", nrm, out) < 0
    tris = tris.copy()
    tris[flip] = tris[flip][:, [0, 2, 1]]
    return tris


def _icosahedron():
    phi = (1.0 + math.sqrt(5.0)) / 2.0
    v = []
    for s1 in (-1, 1):
        for s2 in (-1, 1):
            v.append((0, s1, s2 * phi))
            v.append((s1, s2 * phi, 0))
            v.append((s2 * phi, 0, s1))
    v = np.array(v, dtype=np.float64)
    v /= np.linalg.norm(v, axis=1, keepdims=True)
    d = np.linalg.norm(v[:, None, :] - v[None, :, :], axis=2)
    emin = d[d > 1e-9].min()
    adj = np.abs(d - emin) < 1e-6
    faces = []
    n = v.shape[0]
    for i in range(n):
        for j in range(i + 1, n):
            if not adj[i, j]:
                continue
            for k in range(j + 1, n):
                if adj[i, k] and adj[j, k]:
                    faces.append((i, j, k))
    tris = np.array(faces, dtype=np.int64)
    tris = _orient_outward(v, tris, lambda c: np.zeros_like(c))
    return v, tris


def icosphere(level: int, radius: float = 1.0) -> Mesh:
    """Icosahedron subdivided `level` times (4-to-1), projected on a sphere:
    20*4^L triangles, 10*4^L+2 vertices, 30*4^L edges."""
    v, t = _icosahedron()
    verts = [tuple(x) for x in v]
    tris = [tuple(x) for x in t]
    for _ in range(level):
        cache = {}

        def mid(i, j):
            k = (i, j) if i < j else (j, i)
            if k in cache:
                return cache[k]
            p = np.add(verts[i], verts[j]) * 0.5
            p = p / np.linalg.norm(p)
            verts.append(tuple(p))
            cache[k] = len(verts) - 1
            return cache[k]

        nt = []
        for (a, b, c) in tris:
            ab, bc, ca = mid(a, b), mid(b, c), mid(c, a)
            nt += [(a, ab, ca), (ab, b, bc), (ca, bc, c), (ab, bc, ca)]
        tris = nt
    m = Mesh(np.array(verts) * radius, np.array(tris, dtype=np.int32), name=f"icosphere{level}")
    return build_edges(m)


def geodesic_sphere(freq: int) -> Mesh:
    """Class-I geodesic sphere: each icosahedron face split into freq^2
    triangles, projected on the unit sphere (20 n^2 triangles)."""
    v, t = _icosahedron()
    pts = []
    keymap = {}
    tris = []

    def pid(p):
        p = p / np.linalg.norm(p)
        key = tuple(np.round(p, 9))
        if key not in keymap:
            keymap[key] = len(pts)
            pts.append(p)
        return keymap[key]

    n = freq
    for (a, b, c) in t:
        A, B, C = v[a], v[b], v[c]
        ids = {}
        for i in range(n + 1):
            for j in range(n + 1 - i):
                ids[(i, j)] = pid(A + (B - A) * i / n + (C - A) * j / n)
        for i in range(n):
            for j in range(n - i):
                tris.append((ids[(i, j)], ids[(i + 1, j)], ids[(i, j + 1)]))
                if i + j + 1 < n:
                    tris.append((ids[(i + 1, j)], ids[(i + 1, j + 1)], ids[(i, j + 1)]))
    m = Mesh(np.array(pts), np.array(tris, dtype=np.int32), name=f"geodesic{freq}")
    return build_edges(m)


def ellipsoid(freq: int, semi_axes, rotation: np.ndarray) -> Mesh:
    """Geodesic frequency-n sphere scaled to the semi-axes, then rotated."""
    m = geodesic_sphere(freq)
    verts = (m.verts * np.asarray(semi_axes)[None, :]) @ np.asarray(rotation).T
    out = Mesh(verts, m.tris.copy(), name=f"ellipsoid{freq}")
    return build_edges(out)


def uneven_batch(count: int = 24, seed: int = 20251007):
    """The uneven batch of scatterers: icosphere levels 1, 2, 3 (radius 1)
    and count - 3 ellipsoids, geodesic frequency-n spheres (20 n^2
    triangles) with n drawn from {3, ..., 11}, semi-axes from U[0.5, 1.5]^3
    and a random rotation; eps_r from U[1.5, 8] for every scatterer.
    Scatterer s draws from numpy default_rng(seed + s). Returns a list of
    (mesh, eps_r)."""
    out = []
    for s in range(count):
        rng = np.random.default_rng(seed + s)
        if s < 3:
            mesh = icosphere(s + 1)
        else:
            n = int(rng.integers(3, 12))
            axes = rng.uniform(0.5, 1.5, size=3)
            q, r = np.linalg.qr(rng.standard_normal((3, 3)))
            q = q * np.sign(np.diag(r))[None, :]
            if np.linalg.det(q) < 0:
                q[:, 0] = -q[:, 0]
            mesh = ellipsoid(n, axes, q)
        out.append((mesh, float(rng.uniform(1.5, 8.0))))
    return out


def torus(R: float = 1.0, r: float = 0.3, nu: int = 64, nv: int = 24) -> Mesh:
    """Torus grid of nu (major) x nv (minor) vertices; every quad is split along
    the same diagonal (2 nu nv triangles)."""
    iu, jv = np.meshgrid(np.arange(nu), np.arange(nv), indexing="ij")
    u = 2 * np.pi * iu / nu
    w = 2 * np.pi * jv / nv
    x = (R + r * np.cos(w)) * np.cos(u)
    y = (R + r * np.cos(w)) * np.sin(u)
    z = r * np.sin(w)
    verts = np.stack([x, y, z], axis=-1).reshape(-1, 3)

    def vid(i, j):
        return (i % nu) * nv + (j % nv)

    tris = []
    for i in range(nu):
        for j in range(nv):
            a, b, c, d = vid(i, j), vid(i + 1, j), vid(i + 1, j + 1), vid(i, j + 1)
            tris.append((a, b, c))
            tris.append((a, c, d))
    tris = np.array(tris, dtype=np.int64)

    def tube_center(cen):
        ang = np.arctan2(cen[:, 1], cen[:, 0])
        return np.stack([R * np.cos(ang), R * np.sin(ang), np.zeros_like(ang)], axis=1)

    tris = _orient_outward(verts, tris, tube_center)
    m = Mesh(verts, tris.astype(np.int32), name=f"torus{nu}x{nv}")
    return build_edges(m)


def uv_sphere(n_lon: int = 32, n_bands: int = 25, radius: float = 1.0) -> Mesh:
    """Latitude-longitude sphere: n_lon meridians, n_bands bands between the
    poles (n_bands - 1 vertex rings plus the two poles), the polar bands as
    fans and every other band's quads split along the same diagonal:
    2 n_lon (n_bands - 1) triangles, n_lon (n_bands - 1) + 2 vertices. With
    32 x 25 these are the counts of the unit-sphere mesh of the paper's
    late-time experiment (1536 triangles, 770 vertices, 2304 edges)."""
    th = np.pi * np.arange(1, n_bands) / n_bands          # colatitudes of the rings
    ph = 2 * np.pi * np.arange(n_lon) / n_lon
    ring = np.stack([np.outer(np.sin(th), np.cos(ph)), np.outer(np.sin(th), np.sin(ph)),
                     np.outer(np.cos(th), np.ones(n_lon))], axis=-1).reshape(-1, 3)
    verts = np.vstack([[0.0, 0.0, 1.0], ring, [0.0, 0.0, -1.0]]) * radius
    north, south = 0, len(verts) - 1

    def vid(b, j):  # vertex j of ring b (b = 0 .. n_bands - 2)
        return 1 + b * n_lon + (j % n_lon)

    tris = []
    for j in range(n_lon):
        tris.append((north, vid(0, j), vid(0, j + 1)))
        tris.append((south, vid(n_bands - 2, j + 1), vid(n_bands - 2, j)))
        for b in range(n_bands - 2):
            a, bb, c, d = vid(b, j), vid(b + 1, j), vid(b + 1, j + 1), vid(b, j + 1)
            tris.append((a, bb, c))
            tris.append((a, c, d))
    tris = _orient_outward(verts, np.array(tris, dtype=np.int64), lambda cen: np.zeros_like(cen))
    m = Mesh(verts, tris.astype(np.int32), name=f"uvsphere{n_lon}x{n_bands}")
    return build_edges(m)


def cube(side: float = 2.0, n: int = 24) -> Mesh:
    """Axis-aligned cube centred at the origin with an n x n quad grid per face,
    every quad split along a fixed diagonal (12 n^2 triangles)."""
    ids = {}
    pts = []

    def pid(ijk):
        if ijk not in ids:
            ids[ijk] = len(pts)
            pts.append(ijk)
        return ids[ijk]

    tris = []
    for axis in range(3):
        for sgn in (0, n):
            a1, a2 = [ax for ax in range(3) if ax != axis]
            for i in range(n):
                for j in range(n):
                    def P(ii, jj):
                        c = [0, 0, 0]
                        c[axis] = sgn
                        c[a1] = ii
                        c[a2] = jj
                        return pid(tuple(c))
                    a, b, c, d = P(i, j), P(i + 1, j), P(i + 1, j + 1), P(i, j + 1)
                    tris.append((a, b, c))
                    tris.append((a, c, d))
    verts = (np.array(pts, dtype=np.float64) / n - 0.5) * side
    tris = np.array(tris, dtype=np.int64)
    # outward: compare the normal with the face's outward axis direction
    v0, v1, v2 = verts[tris[:, 0]], verts[tris[:, 1]], verts[tris[:, 2]]
    nrm = np.cross(v1 - v0, v2 - v0)
    cen = (v0 + v1 + v2) / 3.0
    flip = np.einsum("ij,ij->i", nrm, cen) < 0
    tris[flip] = tris[flip][:, [0, 2, 1]]
    m = Mesh(verts, tris.astype(np.int32), name=f"cube{n}")
    return build_edges(m)


def star_pyramid(n_points: int = 5, r_tip: float = 1.0, r_inner: float = 0.4, height: float = 1.0,
                 m: int = 11) -> Mesh:
    """Star-based pyramid: a pyramid over a star polygon with n_points tips
    (the paper's non-smooth third scatterer, Section VI-A, whose exact shape
    comes from another paper: this is a stand-in with the same character --
    sharp tips, re-entrant base corners, sharp edges). The base corners c_j
    (j = 0 .. 2 n_points - 1) sit at angle pi j / n_points, radius r_tip (even
    j) or r_inner (odd j), in the plane z = 0 around the origin; the apex at
    (0, 0, height). The surface is 4 n_points flat triangles -- (apex, c_j,
    c_{j+1}) on the sides, (origin, c_{j+1}, c_j) on the base -- each split
    uniformly into m^2 triangles (m segments per side), so F = 4 n_points m^2,
    V = 2 n_points m^2 + 2 (n_points = 5, m = 11: 1212 vertices, 2420
    triangles, 3630 edges against the paper's 1227, 2450, 3675)."""
    if n_points < 3 or m < 1 or not (0 < r_inner < r_tip) or height <= 0:
        raise ValueError("star_pyramid: needs n_points >= 3, m >= 1, 0 < r_inner < r_tip, height > 0")
    nc = 2 * n_points
    ang = np.pi * np.arange(nc) / n_points
    rad = np.where(np.arange(nc) % 2 == 0, r_tip, r_inner)
    corners = np.stack([rad * np.cos(ang), rad * np.sin(ang), np.zeros(nc)], axis=1)
    apex = np.array([0.0, 0.0, height])
    origin = np.zeros(3)
    big = []
    for j in range(nc):
        c0, c1 = corners[j], corners[(j + 1) % nc]
        big.append((apex, c0, c1))      # side: counter-clockwise seen from outside
        big.append((origin, c1, c0))    # base: seen from below
    ids = {}
    pts = []

    def pid(x):
        k = tuple(np.round(x, 12))
        if k not in ids:
            ids[k] = len(pts)
            pts.append(x)
        return ids[k]

    tris = []
    for A, B, C in big:
        # grid point (i, j): A + (i / m)(B - A) + (j / m)(C - A), i + j <= m
        P = [[pid(A + (i / m) * (B - A) + (j / m) * (C - A)) if i + j <= m else -1 for j in range(m + 1)]
             for i in range(m + 1)]
        for i in range(m):
            for j in range(m - i):
                tris.append((P[i][j], P[i + 1][j], P[i][j + 1]))
                if i + j + 1 < m:
                    tris.append((P[i + 1][j], P[i + 1][j + 1], P[i][j + 1]))
    mesh = Mesh(np.array(pts, dtype=np.float64), np.array(tris, dtype=np.int32), name=f"starpyr{n_points}_{m}")
    return build_edges(mesh)


def diameter(mesh: Mesh) -> float:
    """Scatterer diameter D: the largest vertex-to-vertex distance."""
    v = mesh.verts
    best = 0.0
    for s in range(0, v.shape[0], 1024):
        d = np.linalg.norm(v[s:s + 1024, None, :] - v[None, :, :], axis=2)
        best = max(best, float(d.max()))
    return best


# ----------------------------------------------------------------------------
# excitation batches (paper Eq. (hin): Gaussian-in-time plane waves)
# ----------------------------------------------------------------------------

@dataclass
class Excitation:
    """B plane waves: amplitude A, polarisation p, direction k, width w,
    arrival time t0, and the time after which the star RHS is forced to 0."""
    A: np.ndarray       # (B,)
    p: np.ndarray       # (B, 3)
    k: np.ndarray       # (B, 3)
    w: np.ndarray       # (B,)
    t0: np.ndarray      # (B,)
    t_trunc: np.ndarray  # (B,)

    @property
    def B(self) -> int:
        return int(self.A.shape[0])

    def packed(self) -> np.ndarray:
        """(B, 10) float64 rows: A, p[3], k[3], w, t0, t_trunc."""
        return np.concatenate([self.A[:, None], self.p, self.k, self.w[:, None],
                               self.t0[:, None], self.t_trunc[:, None]], axis=1).astype(np.float64)


def star_truncation_time(t0, w, r_obj, c=1.0):
    """Time after which the Gaussian argument exceeds 6 on the whole scatterer
    (the pulse and its derivative are below e^-36): t0 + (r_obj + 1.5 w)/c."""
    return t0 + (r_obj + 1.5 * w) / c


def single_wave(dt: float, w_steps: float = 120.0, t0_steps: float = 240.0, r_obj: float = 1.0,
                c: float = 1.0) -> Excitation:
    """The paper's excitation: A = 1, p = x, k = z, w = w_steps c dt, t0 = t0_steps dt."""
    w = w_steps * c * dt
    t0 = t0_steps * dt
    return Excitation(A=np.ones(1), p=np.array([[1.0, 0, 0]]), k=np.array([[0, 0, 1.0]]),
                      w=np.array([w]), t0=np.array([t0]),
                      t_trunc=np.array([star_truncation_time(t0, w, r_obj, c)]))


def fibonacci_batch(B: int, dt: float, seed: int = 20251007, w_steps: float = 120.0,
                    t0_steps: float = 240.0, r_obj: float = 1.0, c: float = 1.0) -> Excitation:
    """B plane waves with Fibonacci-sphere directions z_j = 1-(2j+1)/B,
    phi_j = j pi (3 - sqrt 5), polarisation angle theta_j ~ U[0, 2 pi) from
    numpy default_rng(seed)."""
    j = np.arange(B)
    z = 1.0 - (2 * j + 1) / B
    ph = j * np.pi * (3.0 - math.sqrt(5.0))
    s = np.sqrt(np.maximum(0.0, 1.0 - z * z))
    k = np.stack([s * np.cos(ph), s * np.sin(ph), z], axis=1)
    rng = np.random.default_rng(seed)
    th = rng.uniform(0.0, 2 * np.pi, size=B)
    ref = np.where(np.abs(k[:, 2:3]) < 0.9, np.array([[0, 0, 1.0]]), np.array([[1.0, 0, 0]]))
    e1 = np.cross(ref, k)
    e1 /= np.linalg.norm(e1, axis=1, keepdims=True)
    e2 = np.cross(k, e1)
    p = np.cos(th)[:, None] * e1 + np.sin(th)[:, None] * e2
    w = np.full(B, w_steps * c * dt)
    t0 = np.full(B, t0_steps * dt)
    return Excitation(A=np.ones(B), p=p, k=k, w=w, t0=t0,
                      t_trunc=star_truncation_time(t0, w, r_obj, c))
