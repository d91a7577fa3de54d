"""Dense collocation BEM with constant triangles (oracle).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

Sec. 2.1: the boundary integral equation (Eq. bie) is collocated at the
centroid of every element with piecewise-constant u and t, giving
T u = U t (Eq. Tu_Ut) with N = 3 N_e unknowns and the free term
c_ij = delta_ij / 2 absorbed in T. Enforcing the boundary conditions
(Eq. Aa_b) moves the known data to the right-hand side:

  column block of element e in A:  T[:, e]   if e is on Gamma_sigma (u unknown)
                                  -U[:, e]   if e is on Gamma_u     (t unknown)
  b = sum_{e in Gamma_sigma} U[:, e] tbar_e - sum_{e in Gamma_u} T[:, e] ubar_e

Unknown/row numbering: dof 3*e + j (element-major, component-minor).
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

from . import kernels, quadrature as qd


@dataclasses.dataclass
class Geometry:
    p0: np.ndarray
    p1: np.ndarray
    p2: np.ndarray
    n: np.ndarray        # unit normals (out of the solid)
    area: np.ndarray
    c: np.ndarray        # centroids = collocation points
    h: np.ndarray        # longest edge

    @property
    def ne(self):
        return self.c.shape[0]


def geometry(xyz, tri) -> Geometry:
    xyz = np.asarray(xyz, dtype=np.float64)
    tri = np.asarray(tri)
    p0, p1, p2 = xyz[tri[:, 0]], xyz[tri[:, 1]], xyz[tri[:, 2]]
    cr = np.cross(p1 - p0, p2 - p0)
    nn = np.linalg.norm(cr, axis=-1)
    h = np.maximum(np.maximum(np.linalg.norm(p1 - p0, axis=-1), np.linalg.norm(p2 - p1, axis=-1)),
                   np.linalg.norm(p0 - p2, axis=-1))
    return Geometry(p0=p0, p1=p1, p2=p2, n=cr / nn[:, None], area=0.5 * nn,
                    c=(p0 + p1 + p2) / 3.0, h=h)


def _integrate(x, pts, wts, nrm, s, mat):
    """sum_q w_q U(x, y_q), sum_q w_q T(x, y_q; n) for pair batches."""
    U, T = kernels.kernel_pair(x[:, None, :], pts, nrm[:, None, :], s, mat)
    return np.einsum("pq,pqij->pij", wts, U), np.einsum("pq,pqij->pij", wts, T)


def self_static(g: Geometry, elems, mat: kernels.Material):
    """Static (Kelvin) self integrals: closed-form ray integrals, 16 angles per triangle.

    U*: along a ray, int_0^R U* r dr = R [(3-4nu) I + d d^T] / (16 pi mu (1-nu)).
    T*: on a flat element the static traction kernel is c0(theta)/r^2 with
    c0 = (1-2nu)/(8 pi (1-nu)) (rhat_i n_j - rhat_j n_i); its principal value
    along a ray against r dr is c0 ln R (the ln(eps) parts cancel around the
    full circle).
    """
    elems = np.asarray(elems)
    c, n = g.c[elems], g.n[elems]
    nu, mu = mat.nu, mat.mu
    _, _, dirs, logR, wth = qd.self_rule(c, g.p0[elems], g.p1[elems], g.p2[elems], n,
                                         nt=qd.SELF_NT_STATIC, nr=1)
    R = np.exp(logR)
    dd = dirs[..., :, None] * dirs[..., None, :]
    Uang = ((3 - 4 * nu) * np.eye(3) + dd) / (16 * math.pi * mu * (1 - nu))
    Ui = np.einsum("pq,pqij->pij", wth * R, Uang)
    nb = np.broadcast_to(n[:, None, :], dirs.shape)
    c0 = (1 - 2 * nu) / (8 * math.pi * (1 - nu)) * (dirs[..., :, None] * nb[..., None, :]
                                                     - nb[..., :, None] * dirs[..., None, :])
    Ti = np.einsum("pq,pqij->pij", wth * logR, c0)
    return Ui, Ti


def self_remainder(g: Geometry, elems, s, mat: kernels.Material):
    """Polar Gauss (8 angles x 6 radii per triangle) of U - U*, T - T* over the own element."""
    elems = np.asarray(elems)
    c, n = g.c[elems], g.n[elems]
    pts, wts, _, _, _ = qd.self_rule(c, g.p0[elems], g.p1[elems], g.p2[elems], n,
                                     nt=qd.SELF_NT, nr=qd.SELF_NR)
    Ud, Td = kernels.kernel_pair(c[:, None, :], pts, n[:, None, :], s, mat)
    Us = kernels.kelvin_displacement(c[:, None, :], pts, mat)
    Ts = kernels.kelvin_traction(c[:, None, :], pts, n[:, None, :], mat)
    return np.einsum("pq,pqij->pij", wts, Ud - Us), np.einsum("pq,pqij->pij", wts, Td - Ts)


def near_static(g: Geometry, rows, cols, mat: kernels.Material):
    """Static (Kelvin) integrals of NEAR pairs on the 1024-point subdivided rule."""
    x, n = g.c[rows], g.n[cols]
    pts, wts = qd.near_rule(g.p0[cols], g.p1[cols], g.p2[cols])
    Us = kernels.kelvin_displacement(x[:, None, :], pts, mat)
    Ts = kernels.kelvin_traction(x[:, None, :], pts, n[:, None, :], mat)
    return np.einsum("pq,pqij->pij", wts, Us), np.einsum("pq,pqij->pij", wts, Ts)


def near_remainder(g: Geometry, rows, cols, s, mat: kernels.Material):
    """Collapsed 4x4 rule of U - U*, T - T* for NEAR pairs."""
    x, n = g.c[rows], g.n[cols]
    pts, wts = qd.collapsed_rule(g.p0[cols], g.p1[cols], g.p2[cols], qd.NEAR_Q_REM)
    Ud, Td = kernels.kernel_pair(x[:, None, :], pts, n[:, None, :], s, mat)
    Us = kernels.kelvin_displacement(x[:, None, :], pts, mat)
    Ts = kernels.kelvin_traction(x[:, None, :], pts, n[:, None, :], mat)
    return np.einsum("pq,pqij->pij", wts, Ud - Us), np.einsum("pq,pqij->pij", wts, Td - Ts)


def _static_cached(g: Geometry, band, rows, cols, mat):
    """Frequency-independent static blocks, computed once per (mesh, pair set, material)."""
    cache = g.__dict__.setdefault("_static_cache", {})
    key = (band, rows.tobytes(), cols.tobytes(), mat)
    if key not in cache:
        if band == qd.BAND_SELF:
            cache[key] = self_static(g, cols, mat)
        else:
            cache[key] = near_static(g, rows, cols, mat)
    return cache[key]


def pair_integrals(g: Geometry, rows, cols, s, mat: kernels.Material):
    """3x3 blocks int_e U(x_i, y) dy and (PV) int_e T(x_i, y) dy for pairs.

    rows, cols: equal-length element index arrays (collocation element i,
    integration element e). Returns U, T of shape (P, 3, 3). The free term is
    NOT included here.
    """
    rows = np.asarray(rows, dtype=np.int64).ravel()
    cols = np.asarray(cols, dtype=np.int64).ravel()
    P = rows.size
    U = np.zeros((P, 3, 3), dtype=np.complex128)
    T = np.zeros((P, 3, 3), dtype=np.complex128)
    band = qd.classify(g.c[rows], g.c[cols], g.h[cols], rows == cols)
    for b in (qd.BAND_SELF, qd.BAND_NEAR, qd.BAND_Q4, qd.BAND_Q2, qd.BAND_Q1):
        sel = np.nonzero(band == b)[0]
        if sel.size == 0:
            continue
        chunk = {qd.BAND_SELF: 256, qd.BAND_NEAR: 128, qd.BAND_Q4: 8192,
                 qd.BAND_Q2: 32768, qd.BAND_Q1: 131072}[b]
        for lo in range(0, sel.size, chunk):
            idx = sel[lo:lo + chunk]
            ri, ce = rows[idx], cols[idx]
            if b == qd.BAND_SELF:
                Us, Ts = _static_cached(g, b, ri, ce, mat)
                Ur, Tr = self_remainder(g, ce, s, mat)
                Ub, Tb = Us + Ur, Ts + Tr
            elif b == qd.BAND_NEAR:
                Us, Ts = _static_cached(g, b, ri, ce, mat)
                Ur, Tr = near_remainder(g, ri, ce, s, mat)
                Ub, Tb = Us + Ur, Ts + Tr
            else:
                a, bb, cc = g.p0[ce], g.p1[ce], g.p2[ce]
                if b == qd.BAND_Q4:
                    pts, wts = qd.collapsed_rule(a, bb, cc, 4)
                elif b == qd.BAND_Q2:
                    pts, wts = qd.collapsed_rule(a, bb, cc, 2)
                else:
                    pts, wts = qd.centroid_rule(a, bb, cc)
                Ub, Tb = _integrate(g.c[ri], pts, wts, g.n[ce], s, mat)
            U[idx] = Ub
            T[idx] = Tb
    return U, T


def dense_blocks(g: Geometry, s, mat, rows=None):
    """All 3x3 blocks for the given collocation elements: U, T of shape (R, Ne, 3, 3)."""
    ne = g.ne
    rows = np.arange(ne) if rows is None else np.asarray(rows, dtype=np.int64)
    I, E = np.meshgrid(rows, np.arange(ne), indexing="ij")
    U, T = pair_integrals(g, I.ravel(), E.ravel(), s, mat)
    return U.reshape(rows.size, ne, 3, 3), T.reshape(rows.size, ne, 3, 3)


def _to_matrix(B):
    R, ne = B.shape[:2]
    return B.transpose(0, 2, 1, 3).reshape(3 * R, 3 * ne)


def system_rows(g: Geometry, bc_type, known, s, mat, rows=None):
    """Rows of A and b (Eq. Aa_b) for collocation elements ``rows``.

    bc_type: (Ne,) 0 = Gamma_sigma, 1 = Gamma_u. known: (Ne, 3) complex
    prescribed traction (Gamma_sigma) or displacement (Gamma_u).
    Returns A (3R, 3Ne) and b (3R,), complex128.
    """
    ne = g.ne
    rows = np.arange(ne) if rows is None else np.asarray(rows, dtype=np.int64)
    U, T = dense_blocks(g, s, mat, rows)
    # free term c_ij = delta_ij / 2 on the collocation element's own block
    for r_local, e in enumerate(rows):
        T[r_local, e] += 0.5 * np.eye(3)
    bc = np.asarray(bc_type).astype(bool)           # True = Gamma_u
    Acol = np.where(bc[None, :, None, None], -U, T)
    Bcol = np.where(bc[None, :, None, None], -T, U)
    A = _to_matrix(Acol)
    b = _to_matrix(Bcol) @ np.asarray(known, dtype=np.complex128).reshape(-1)
    return A, b


def full_matrices(g: Geometry, s, mat):
    """Dense T (free term included) and U, each (N, N) complex128."""
    U, T = dense_blocks(g, s, mat)
    for e in range(g.ne):
        T[e, e] += 0.5 * np.eye(3)
    return _to_matrix(T), _to_matrix(U)


def interior_field(g: Geometry, bc_type, known, a, points, s, mat):
    """Displacement at points inside the solid from the boundary solution.

    The representation formula (Somigliana's identity, the interior form of
    Eq. bie with c = I): u_i(x) = sum_e [int_e U_ij(x, y) dy t_j(e)
    - int_e T_ij(x, y) dy u_j(e)], with u, t constant per element: on
    Gamma_sigma elements t is the prescribed ``known`` and u the solved ``a``,
    on Gamma_u elements the reverse. Each (point, element) pair takes the rule
    of its distance band (as the matrix entries); the NEAR band takes the
    1024-point subdivided rule on the full kernel (the point is off the
    boundary, so the integrand is only nearly singular). Points must not lie
    on the boundary. Returns (P, 3) complex.
    """
    x = np.asarray(points, dtype=np.float64).reshape(-1, 3)
    a = np.asarray(a, dtype=np.complex128).reshape(-1, 3)
    known = np.asarray(known, dtype=np.complex128).reshape(-1, 3)
    fixed = np.asarray(bc_type).astype(bool)
    u = np.where(fixed[:, None], known, a)
    t = np.where(fixed[:, None], a, known)
    out = np.zeros((x.shape[0], 3), dtype=np.complex128)
    ne = g.c.shape[0]
    for p in range(x.shape[0]):
        xp = np.broadcast_to(x[p], (ne, 3))
        band = qd.classify(xp, g.c, g.h, np.zeros(ne, dtype=bool))
        for b in (qd.BAND_NEAR, qd.BAND_Q4, qd.BAND_Q2, qd.BAND_Q1):
            e = np.nonzero(band == b)[0]
            if e.size == 0:
                continue
            if b == qd.BAND_NEAR:
                pts, wts = qd.near_rule(g.p0[e], g.p1[e], g.p2[e])
            elif b == qd.BAND_Q4:
                pts, wts = qd.collapsed_rule(g.p0[e], g.p1[e], g.p2[e], 4)
            elif b == qd.BAND_Q2:
                pts, wts = qd.collapsed_rule(g.p0[e], g.p1[e], g.p2[e], 2)
            else:
                pts, wts = qd.centroid_rule(g.p0[e], g.p1[e], g.p2[e])
            Ui, Ti = _integrate(xp[e], pts, wts, g.n[e], s, mat)
            out[p] += np.einsum("eij,ej->i", Ui, t[e]) - np.einsum("eij,ej->i", Ti, u[e])
    return out


def interior_strain(g: Geometry, bc_type, known, a, points, s, mat, h):
    """Strain at interior points: eps = (grad u + grad u^T) / 2 with grad u by
    central differences of ``interior_field`` at x +- h e_a (step h; the six
    points must lie inside the solid). Returns (P, 6) complex, components
    xx, yy, zz, xy, yz, xz (tensor, not engineering, shear).
    """
    x = np.asarray(points, dtype=np.float64).reshape(-1, 3)
    grad = np.zeros((x.shape[0], 3, 3), dtype=np.complex128)  # grad[p, i, a] = d u_i / d x_a
    for ax in range(3):
        step = np.zeros(3)
        step[ax] = h
        up = interior_field(g, bc_type, known, a, x + step, s, mat)
        um = interior_field(g, bc_type, known, a, x - step, s, mat)
        grad[:, :, ax] = (up - um) / (2 * h)
    eps = 0.5 * (grad + grad.transpose(0, 2, 1))
    ii, jj = [0, 1, 2, 0, 1, 0], [0, 1, 2, 1, 2, 2]
    return eps[:, ii, jj]
