"""Seeded synthetic inputs: surface meshes and load histories.

This module holds no arithmetic of the boundary element method itself. It only
builds triangulated closed surfaces (vertex coordinates plus vertex-index
triples) and sampled load histories, so both the CUDA path and the CPU oracle
can be fed the very same inputs.

Orientation convention (Sec. 2.1): the normal of a triangle is
(v1 - v0) x (v2 - v0) and must point OUT of the elastic solid Omega. For the
outer surface of a solid body that is the usual outward normal; for a cavity
inside a solid it points into the cavity (toward the cavity centre), so
cavity surfaces are emitted with reversed vertex order (``inward=True``).

Workload shapes (the paper's meshes are not published, so each of these is a
synthetic stand-in with the sizes and structure the text describes):

* ``geodesic_sphere(n)``: class-I geodesic sphere, 20 n^2 triangles. n=4 gives
  320 triangles (960 unknowns), n=16 gives 5,120 (15,360 unknowns).
* ``box_mesh``: closed box, each face structured into right triangles.
* ``ellipsoid_mesh``: geodesic sphere mapped to an ellipsoid.
* ``cube_with_cavities``: the large example of Sec. 5.3 (cube with spherical
  cavities, bottom fixed, top loaded), built at a chosen resolution.
* ``rod_problem``: the prismatic rod of Sec. 5.1 (3 x 1 x 1, one end fixed,
  a step traction on the other, sides free); h = 1/21 gives 12,348 triangles.
* ``ball_with_void``: a solid ball with an off-centre spherical void, outer
  surface under pressure (geodesic n=28 outside and n=15 inside give
  15,680 + 4,500 = 20,180 triangles).
* ``heaviside_history``: P(n dt) for a step load, with P(0) = 1/2.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

# Element boundary-condition kinds (Sec. 2.1: Gamma_sigma / Gamma_u).
BC_TRACTION = 0      # traction prescribed, displacement unknown
BC_DISPLACEMENT = 1  # displacement prescribed, traction unknown


@dataclasses.dataclass
class Mesh:
    """A closed triangulated surface with per-element boundary data.

    xyz:     (nv, 3) float64 vertex coordinates.
    tri:     (ne, 3) int32 vertex indices; normal (v1-v0)x(v2-v0) points out
             of the solid.
    bc_type: (ne,) int8, BC_TRACTION or BC_DISPLACEMENT per element.
    pattern: (ne, 3) float64 prescribed spatial values (traction on
             Gamma_sigma elements, displacement on Gamma_u elements); the full
             prescribed data is pattern * P(t).
    """

    xyz: np.ndarray
    tri: np.ndarray
    bc_type: np.ndarray
    pattern: np.ndarray
    name: str = ""

    def __post_init__(self):
        self.xyz = np.ascontiguousarray(self.xyz, dtype=np.float64)
        self.tri = np.ascontiguousarray(self.tri, dtype=np.int32)
        self.bc_type = np.ascontiguousarray(self.bc_type, dtype=np.int8)
        self.pattern = np.ascontiguousarray(self.pattern, dtype=np.float64)

    @property
    def ne(self) -> int:
        return int(self.tri.shape[0])

    @property
    def nv(self) -> int:
        return int(self.xyz.shape[0])


def _icosahedron():
    t = (1.0 + math.sqrt(5.0)) / 2.0
    v = np.array([
        [-1, t, 0], [1, t, 0], [-1, -t, 0], [1, -t, 0],
        [0, -1, t], [0, 1, t], [0, -1, -t], [0, 1, -t],
        [t, 0, -1], [t, 0, 1], [-t, 0, -1], [-t, 0, 1],
    ], dtype=np.float64)
    f = np.array([
        [0, 11, 5], [0, 5, 1], [0, 1, 7], [0, 7, 10], [0, 10, 11],
        [1, 5, 9], [5, 11, 4], [11, 10, 2], [10, 7, 6], [7, 1, 8],
        [3, 9, 4], [3, 4, 2], [3, 2, 6], [3, 6, 8], [3, 8, 9],
        [4, 9, 5], [2, 4, 11], [6, 2, 10], [8, 6, 7], [9, 8, 1],
    ], dtype=np.int64)
    v /= np.linalg.norm(v, axis=1, keepdims=True)
    return v, f


class _VertexPool:
    """Deduplicates vertices by their rounded coordinates."""

    def __init__(self):
        self.key = {}
        self.pts = []

    def add(self, p):
        k = tuple(np.round(p, 10))
        idx = self.key.get(k)
        if idx is None:
            idx = len(self.pts)
            self.key[k] = idx
            self.pts.append(np.asarray(p, dtype=np.float64))
        return idx

    def array(self):
        return np.array(self.pts, dtype=np.float64)


def _orient_outward(xyz, tri, center):
    """Flip triangles whose normal points toward ``center`` (star-shaped)."""
    p0, p1, p2 = xyz[tri[:, 0]], xyz[tri[:, 1]], xyz[tri[:, 2]]
    nrm = np.cross(p1 - p0, p2 - p0)
    c = (p0 + p1 + p2) / 3.0 - center
    flip = np.einsum("ij,ij->i", nrm, c) < 0
    tri = tri.copy()
    tri[flip] = tri[flip][:, [0, 2, 1]]
    return tri


def geodesic_sphere(n: int, radius: float = 1.0, center=(0.0, 0.0, 0.0),
                    inward: bool = False):
    """Class-I geodesic sphere with 20*n^2 flat triangles.

    Each icosahedron face is cut into n^2 triangles on a regular barycentric
    grid; grid points are projected onto the sphere. Returns (xyz, tri) with
    outward normals, or inward ones when ``inward`` (a cavity surface).
    """
    if n < 1:
        raise ValueError("n must be >= 1")
    v, f = _icosahedron()
    pool = _VertexPool()
    tris = []
    for a, b, c in f:
        A, B, C = v[a], v[b], v[c]
        idx = {}
        for i in range(n + 1):
            for j in range(n + 1 - i):
                p = A + (B - A) * (i / n) + (C - A) * (j / n)
                p = p / np.linalg.norm(p)
                idx[(i, j)] = pool.add(p)
        for i in range(n):
            for j in range(n - i):
                tris.append((idx[(i, j)], idx[(i + 1, j)], idx[(i, j + 1)]))
                if i + j + 1 < n:
                    tris.append((idx[(i + 1, j)], idx[(i + 1, j + 1)], idx[(i, j + 1)]))
    xyz = pool.array()
    tri = np.array(tris, dtype=np.int64)
    tri = _orient_outward(xyz, tri, np.zeros(3))
    if inward:
        tri = tri[:, [0, 2, 1]]
    xyz = xyz * radius + np.asarray(center, dtype=np.float64)
    return np.ascontiguousarray(xyz), np.ascontiguousarray(tri, dtype=np.int32)


def box_mesh(lx: float, ly: float, lz: float, h: float, center=(0.0, 0.0, 0.0)):
    """Closed axis-aligned box; each face a structured grid of right triangles.

    The number of cells along an edge is max(1, round(edge / h)). Normals point
    out of the box.
    """
    L = np.array([lx, ly, lz], dtype=np.float64)
    c0 = np.asarray(center, dtype=np.float64) - L / 2
    pool = _VertexPool()
    tris = []
    for axis in range(3):
        u_ax, v_ax = [a for a in range(3) if a != axis]
        nu = max(1, int(round(L[u_ax] / h)))
        nv = max(1, int(round(L[v_ax] / h)))
        for side in (0, 1):
            idx = {}
            for i in range(nu + 1):
                for j in range(nv + 1):
                    p = c0.copy()
                    p[axis] += side * L[axis]
                    p[u_ax] += L[u_ax] * i / nu
                    p[v_ax] += L[v_ax] * j / nv
                    idx[(i, j)] = pool.add(p)
            for i in range(nu):
                for j in range(nv):
                    a, b = idx[(i, j)], idx[(i + 1, j)]
                    c, d = idx[(i + 1, j + 1)], idx[(i, j + 1)]
                    if (i + j) % 2 == 0:
                        tris += [(a, b, c), (a, c, d)]
                    else:
                        tris += [(a, b, d), (b, c, d)]
    xyz = pool.array()
    tri = np.array(tris, dtype=np.int64)
    tri = _orient_outward(xyz, tri, np.asarray(center, dtype=np.float64))
    return np.ascontiguousarray(xyz), np.ascontiguousarray(tri, dtype=np.int32)


def ellipsoid_mesh(n: int, semi_axes, center=(0.0, 0.0, 0.0)):
    """Geodesic sphere (20 n^2 triangles) scaled to an ellipsoid."""
    xyz, tri = geodesic_sphere(n)
    xyz = xyz * np.asarray(semi_axes, dtype=np.float64) + np.asarray(center, dtype=np.float64)
    return xyz, tri


def heaviside_history(n_omega: int, amplitude: float = 1.0) -> np.ndarray:
    """Samples P(n dt), n = 0..n_omega-1, of a step load; P(0) = amplitude/2.

    The midpoint value at the jump makes the sampled transform the trapezoid
    rule of the Laplace transform of the step.
    """
    p = np.full(n_omega, float(amplitude))
    p[0] = 0.5 * amplitude
    return p


def _centroids(xyz, tri):
    return (xyz[tri[:, 0]] + xyz[tri[:, 1]] + xyz[tri[:, 2]]) / 3.0


def _normals(xyz, tri):
    p0, p1, p2 = xyz[tri[:, 0]], xyz[tri[:, 1]], xyz[tri[:, 2]]
    nrm = np.cross(p1 - p0, p2 - p0)
    return nrm / np.linalg.norm(nrm, axis=1, keepdims=True)


def cavity_problem(n: int = 4, radius: float = 1.0, pressure: float = 1.0) -> Mesh:
    """Spherical cavity in an infinite solid under uniform internal pressure.

    The surface is a geodesic sphere with normals pointing into the cavity
    (out of the solid); every element is on Gamma_sigma with prescribed
    traction t = -p n (pressure pushes the solid away from the cavity).
    n=4: 320 triangles; n=16: 5,120 triangles.
    """
    xyz, tri = geodesic_sphere(n, radius=radius, inward=True)
    nrm = _normals(xyz, tri)
    return Mesh(xyz=xyz, tri=tri,
                bc_type=np.zeros(tri.shape[0], dtype=np.int8),
                pattern=-pressure * nrm,
                name=f"cavity_sphere_{tri.shape[0]}")


def pressurised_surface(xyz, tri, pressure: float = 1.0, name: str = "") -> Mesh:
    """All-traction problem with uniform pressure on a closed surface."""
    nrm = _normals(xyz, tri)
    return Mesh(xyz=xyz, tri=tri.astype(np.int32),
                bc_type=np.zeros(tri.shape[0], dtype=np.int8),
                pattern=-pressure * nrm, name=name)


def batched_meshes(count: int = 16, seed: int = 3032, tri_min: int = 2000,
                   tri_max: int = 40000):
    """Uneven batch of closed boxes and ellipsoids (cavity problems).

    Half boxes with aspect ratios U[1, 4], half ellipsoids with semi-axes
    U[0.5, 2]; target triangle counts log-uniform in [tri_min, tri_max].
    Every surface is a cavity (normals reversed) under uniform pressure.
    """
    rng = np.random.default_rng(seed)
    out = []
    for m in range(count):
        target = math.exp(rng.uniform(math.log(tri_min), math.log(tri_max)))
        if m % 2 == 0:
            dims = np.array([1.0, rng.uniform(1, 4), rng.uniform(1, 4)])
            area = 2 * (dims[0] * dims[1] + dims[1] * dims[2] + dims[0] * dims[2])
            h = math.sqrt(2 * area / target)
            xyz, tri = box_mesh(*dims, h=h)
        else:
            axes = rng.uniform(0.5, 2.0, size=3)
            n = max(2, int(round(math.sqrt(target / 20.0))))
            xyz, tri = ellipsoid_mesh(n, axes)
        tri = tri[:, [0, 2, 1]]  # cavity: normals into the void
        out.append(pressurised_surface(xyz, tri, name=f"batch{m}_{tri.shape[0]}"))
    return out


def cube_with_cavities(n_face: int = 118, n_cav: int = 8, cav_radius: float = 0.15,
                       cav_n: int = 20, min_gap: float = 0.05, seed: int = 3032,
                       traction: float = -1.0) -> Mesh:
    """Unit cube [-.5,.5]^3 with spherical cavities (the large example, Sec. 5.3).

    Bottom face (z = -0.5) fixed (Gamma_u, u = 0), top face (z = 0.5) under a
    uniform normal traction ``traction`` (negative = compression), every other
    face and all cavity walls traction free. Cavity centres are drawn from
    ``seed`` with at least ``min_gap`` between cavities and to the cube faces.
    n_face=118, cav_n=20, n_cav=8 gives 167,088 + 64,000 = 231,088 triangles.
    """
    rng = np.random.default_rng(seed)
    xyz_c, tri_c = box_mesh(1.0, 1.0, 1.0, h=1.0 / n_face)
    centres = []
    lim = 0.5 - cav_radius - min_gap
    tries = 0
    while len(centres) < n_cav:
        tries += 1
        if tries > 100000:
            raise RuntimeError("could not place cavities")
        c = rng.uniform(-lim, lim, size=3)
        if all(np.linalg.norm(c - q) >= 2 * cav_radius + min_gap for q in centres):
            centres.append(c)
    parts_xyz = [xyz_c]
    parts_tri = [tri_c]
    off = xyz_c.shape[0]
    for c in centres:
        xs, ts = geodesic_sphere(cav_n, radius=cav_radius, center=c, inward=True)
        parts_xyz.append(xs)
        parts_tri.append(ts + off)
        off += xs.shape[0]
    xyz = np.concatenate(parts_xyz)
    tri = np.concatenate(parts_tri).astype(np.int32)
    cen = _centroids(xyz, tri)
    ne = tri.shape[0]
    bc = np.zeros(ne, dtype=np.int8)
    pattern = np.zeros((ne, 3))
    n_box = tri_c.shape[0]
    box_cen = cen[:n_box]
    bottom = np.zeros(ne, dtype=bool)
    top = np.zeros(ne, dtype=bool)
    bottom[:n_box] = np.abs(box_cen[:, 2] + 0.5) < 1e-12
    top[:n_box] = np.abs(box_cen[:, 2] - 0.5) < 1e-12
    bc[bottom] = BC_DISPLACEMENT
    pattern[top, 2] = traction
    return Mesh(xyz=xyz, tri=tri, bc_type=bc, pattern=pattern,
                name=f"cube_{n_cav}cav_{ne}")


def ball_with_void(n_outer: int = 28, n_inner: int = 15, radius: float = 1.0,
                   void_radius: float = 0.3, void_center=(0.35, 0.2, -0.1),
                   pressure: float = 1.0) -> Mesh:
    """Solid ball of ``radius`` with a spherical void, both geodesic spheres.

    The solid is the ball minus the void: the outer sphere's normals point
    away from the centre, the void's into the void. Every element is on
    Gamma_sigma; the outer surface carries t = -p n (a uniform pressure), the
    void wall is traction free.
    """
    xo, to = geodesic_sphere(n_outer, radius=radius)
    xi, ti = geodesic_sphere(n_inner, radius=void_radius, center=void_center, inward=True)
    xyz = np.concatenate([xo, xi])
    tri = np.concatenate([to, ti + xo.shape[0]]).astype(np.int32)
    ne = tri.shape[0]
    pattern = np.zeros((ne, 3))
    pattern[:to.shape[0]] = -pressure * _normals(xo, to)
    return Mesh(xyz=xyz, tri=tri, bc_type=np.zeros(ne, dtype=np.int8), pattern=pattern,
                name=f"ball_void_{ne}")


def rod_problem(length: float = 3.0, h: float = 1.0 / 21, pressure: float = 1.0) -> Mesh:
    """Prismatic rod [0, length] x [-1/2, 1/2]^2 (the rod example, Sec. 5.1).

    The end x = 0 is fixed (Gamma_u, u = 0); the end x = length carries the
    traction t = -pressure n (a compressive step when multiplied by H(t));
    the four sides are traction free.
    """
    xyz, tri = box_mesh(length, 1.0, 1.0, h, center=(length / 2, 0.0, 0.0))
    cen = _centroids(xyz, tri)
    nrm = _normals(xyz, tri)
    ne = tri.shape[0]
    bc = np.zeros(ne, dtype=np.int8)
    pattern = np.zeros((ne, 3))
    fixed = np.abs(cen[:, 0]) < 1e-9 * length
    loaded = np.abs(cen[:, 0] - length) < 1e-9 * length
    bc[fixed] = BC_DISPLACEMENT
    pattern[loaded] = -pressure * nrm[loaded]
    return Mesh(xyz=xyz, tri=tri, bc_type=bc, pattern=pattern, name=f"rod_{ne}")
