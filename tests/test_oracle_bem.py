"""Pins for the oracle's element integration and collocation system.

* quadrature rules integrate polynomials exactly to their stated degree;
* every 3x3 block of a small mesh is compared with an independent brute-force
  integral (fine subdivision for regular pairs; Duffy rule for the weakly
  singular self U block; epsilon-excluded polar integration of the full
  kernel for the principal-value self T block);
* the static rigid-body identity 1/2 I + sum_e int_e T = 0 (outward normals)
  or I (reversed normals) on a closed polyhedron (Sec. 2.1, free term);
* the whole discrete system converges to the closed-form cavity response as
  the mesh is refined (which fixes signs, scaling and the BC handling);
* the closed form itself solves the radial Navier ODE and the wall condition.
"""
import math

import numpy as np
import pytest

from oracle import bem, kernels, quadrature as qd, solvers
from paper_1212_3032_gb300 import inputs
from tests import analytic

MAT = kernels.Material(1.0, 0.25, 1.0)


def _ref_tri():
    return (np.array([[0.0, 0, 0]]), np.array([[1.0, 0, 0]]), np.array([[0.0, 1, 0]]))


@pytest.mark.parametrize("q", [1, 2, 3, 4, 6])
def test_collapsed_rule_exact(q):
    p0, p1, p2 = _ref_tri()
    pts, w = qd.collapsed_rule(p0, p1, p2, q)
    for a in range(0, 2 * q - 1):
        for b in range(0, 2 * q - 1 - a):
            f = pts[0, :, 0] ** a * pts[0, :, 1] ** b
            exact = math.factorial(a) * math.factorial(b) / math.factorial(a + b + 2)
            assert np.sum(w[0] * f) == pytest.approx(exact, rel=1e-12, abs=1e-15)


def test_near_and_centroid_rules():
    rng = np.random.default_rng(0)
    P = rng.normal(size=(3, 1, 3))
    area = 0.5 * np.linalg.norm(np.cross(P[1] - P[0], P[2] - P[0]))
    pts, w = qd.near_rule(P[0], P[1], P[2])
    assert pts.shape == (1, 1024, 3)
    assert w.sum() == pytest.approx(area, rel=1e-13)
    # linear functions integrate to area * value at the centroid
    cen = (P[0] + P[1] + P[2])[0] / 3
    lin = np.array([0.3, -1.1, 2.0])
    assert np.sum(w[0] * (pts[0] @ lin)) == pytest.approx(area * cen @ lin, rel=1e-12)
    pc, wc = qd.centroid_rule(P[0], P[1], P[2])
    assert np.allclose(pc[0, 0], cen) and wc[0, 0] == pytest.approx(area)


def test_self_rule_area_and_moments():
    mesh = inputs.cavity_problem(2)
    g = bem.geometry(mesh.xyz, mesh.tri)
    e = np.arange(g.ne)
    # the static rule (16 angles) is near exact, the remainder rule (8) less so
    p8, w8, _, _, _ = qd.self_rule(g.c[e], g.p0[e], g.p1[e], g.p2[e], g.n[e])
    assert np.allclose(w8.sum(axis=1), g.area, rtol=2e-4)
    pts, w, dirs, logR, wth = qd.self_rule(g.c[e], g.p0[e], g.p1[e], g.p2[e], g.n[e], nt=16)
    assert np.allclose(w.sum(axis=1), g.area, rtol=1e-9)
    # angular weights cover the full turn about the centroid
    assert np.allclose(wth.sum(axis=1), 2 * math.pi, rtol=1e-12)
    # second moment |y - c|^2 against the collapsed rule (exact for degree 2)
    cp, cw = qd.collapsed_rule(g.p0, g.p1, g.p2, 2)
    m2_ref = np.sum(cw * np.sum((cp - g.c[:, None, :]) ** 2, axis=-1), axis=1)
    m2 = np.sum(w * np.sum((pts - g.c[:, None, :]) ** 2, axis=-1), axis=1)
    assert np.allclose(m2, m2_ref, rtol=1e-8)


def _brute_regular(g, i, e, s):
    """Four levels of subdivision x collapsed 6x6 of the full kernels."""
    tris = [(g.p0[e:e + 1], g.p1[e:e + 1], g.p2[e:e + 1])]
    for _ in range(4):
        nxt = []
        for t in tris:
            nxt += qd.subdivide(*t)
        tris = nxt
    U = np.zeros((3, 3), complex)
    T = np.zeros((3, 3), complex)
    for a, b, c in tris:
        pts, w = qd.collapsed_rule(a, b, c, 6)
        Uk, Tk = kernels.kernel_pair(g.c[i], pts[0], g.n[e], s, MAT)
        U += np.einsum("q,qij->ij", w[0], Uk)
        T += np.einsum("q,qij->ij", w[0], Tk)
    return U, T


def _brute_self(g, e, s):
    """Self blocks by methods independent of the polar/analytic split.

    U: Duffy rule on the three triangles (c, p_a, p_b) with c at the collapsed
    vertex (the Jacobian cancels the 1/r singularity), 40x40 points each.
    T: polar integration of the FULL kernel from r = eps to the edge with
    graded radial nodes (uniform in ln r), 48 angles per triangle; the disk
    of radius eps contributes nothing to the principal value of the static
    part (odd in direction) and O(eps^2) to the rest.
    """
    c, n = g.c[e], g.n[e]
    V = [g.p0[e], g.p1[e], g.p2[e]]
    U = np.zeros((3, 3), complex)
    for k in range(3):
        a, b = V[k], V[(k + 1) % 3]
        # collapsed vertex of the rule is its second vertex
        pts, w = qd.collapsed_rule(a[None], c[None], b[None], 40)
        U += np.einsum("q,qij->ij", w[0], kernels.displacement_kernel(c, pts[0], s, MAT))
    T = np.zeros((3, 3), complex)
    eps = 1e-4 * g.h[e]
    tn, tw = qd.gauss_legendre_01(48)
    xn, xw = qd.gauss_legendre_01(64)
    for k in range(3):
        a, b = V[k], V[(k + 1) % 3]
        t = b - a
        foot = a + np.dot(c - a, t) / np.dot(t, t) * t
        d = np.linalg.norm(foot - c)
        fh = (foot - c) / d
        gh = np.cross(n, fh)
        tha = math.atan2(np.dot(a - c, gh), np.dot(a - c, fh))
        thb = math.atan2(np.dot(b - c, gh), np.dot(b - c, fh))
        for th, wt in zip(tha + (thb - tha) * tn, (thb - tha) * tw):
            R = d / math.cos(th)
            dr = math.cos(th) * fh + math.sin(th) * gh
            L = math.log(R / eps)
            r = eps * np.exp(L * xn)             # r dr = r^2 d(ln r)
            wr = xw * L * r * r
            Tk = kernels.traction_kernel(c, c + r[:, None] * dr, n, s, MAT)
            T += wt * np.einsum("q,qij->ij", wr, Tk)
    return U, T


@pytest.mark.parametrize("s,tol", [
    (0.625, {qd.BAND_NEAR: 5e-4, qd.BAND_Q4: 5e-5}),
    # |s| h / c_s ~ 4 on this coarse mesh: under-resolved, so looser
    (0.625 + 4.0j, {qd.BAND_NEAR: 1e-2, qd.BAND_Q4: 1e-4}),
])
def test_blocks_against_brute_force(s, tol):
    mesh = inputs.cavity_problem(2)   # 80 triangles: SELF, NEAR and Q4 bands
    g = bem.geometry(mesh.xyz, mesh.tri)
    rng = np.random.default_rng(7)
    i_all = np.repeat(np.arange(g.ne), g.ne)
    e_all = np.tile(np.arange(g.ne), g.ne)
    band = qd.classify(g.c[i_all], g.c[e_all], g.h[e_all], i_all == e_all)
    for b, rt in tol.items():
        sel = np.nonzero(band == b)[0]
        if sel.size == 0:
            continue
        pick = rng.choice(sel, size=min(6, sel.size), replace=False)
        U, T = bem.pair_integrals(g, i_all[pick], e_all[pick], s, MAT)
        for m, p in enumerate(pick):
            Ur, Tr = _brute_regular(g, i_all[p], e_all[p], s)
            assert np.abs(U[m] - Ur).max() <= rt * np.abs(Ur).max(), (b, "U")
            assert np.abs(T[m] - Tr).max() <= rt * np.abs(Tr).max(), (b, "T")
    for e in (0, 17, 55):
        U, T = bem.pair_integrals(g, [e], [e], s, MAT)
        Ur, Tr = _brute_self(g, e, s)
        assert np.abs(U[0] - Ur).max() <= 1e-5 * np.abs(Ur).max()
        assert np.abs(T[0] - Tr).max() <= 1e-6


@pytest.mark.parametrize("inward", [False, True])
def test_rigid_body_identity(inward):
    """1/2 I + sum_e int_e T(x_i, y) dy = 0 (outward) or I (reversed), s -> 0."""
    xyz, tri = inputs.geodesic_sphere(3, inward=inward)
    g = bem.geometry(xyz, tri)
    s = 1e-3
    rows = np.array([0, 40, 101, 150])
    U, T = bem.dense_blocks(g, s, MAT, rows)
    tot = T.sum(axis=1) + 0.5 * np.eye(3)
    target = np.eye(3) if inward else np.zeros((3, 3))
    assert np.abs(tot - target).max() <= 1e-4


def test_cavity_closed_form_pins_itself():
    """The closed form solves the radial Navier ODE with sigma_rr(a) = -p."""
    mu, lam, rho, a = MAT.mu, MAT.lam, MAT.rho, 1.0
    for s in (0.5, 0.5 + 2.0j, 1.0 + 7.0j):
        h = 1e-4
        r = 1.3
        f = lambda rr: analytic.cavity_field(rr, s, a, mu, lam, rho)
        u, up, upp = f(r), (f(r + h) - f(r - h)) / (2 * h), (f(r + h) - 2 * f(r) + f(r - h)) / h**2
        lhs = (lam + 2 * mu) * (upp + 2 * up / r - 2 * u / r**2)
        assert abs(lhs - rho * s * s * u) <= 1e-5 * abs(rho * s * s * u)
        ua, upa = f(a), (f(a + h) - f(a - h)) / (2 * h)
        srr = (lam + 2 * mu) * upa + 2 * lam * ua / a
        assert abs(srr + 1.0) <= 1e-6
    assert analytic.cavity_wall_response(0.0, 1.0, mu, lam, rho) == pytest.approx(1.0 / (4 * mu))


def _cavity_error(n, s):
    mesh = inputs.cavity_problem(n)
    g = bem.geometry(mesh.xyz, mesh.tri)
    A, b = bem.system_rows(g, mesh.bc_type, mesh.pattern.astype(complex), s, MAT)
    a = solvers.direct_solve(A, b).reshape(-1, 3)
    rhat = g.c / np.linalg.norm(g.c, axis=1, keepdims=True)
    ur = np.einsum("ij,ij->i", a, rhat)
    H = analytic.cavity_wall_response(s, 1.0, MAT.mu, MAT.lam, MAT.rho)
    return np.sqrt(np.mean(np.abs(ur - H) ** 2)) / abs(H)


def test_cavity_converges_to_closed_form():
    for s in (0.625, 0.625 + 3.0j):
        e4 = _cavity_error(4, s)
        e6 = _cavity_error(6, s)
        assert e6 < 0.8 * e4
        assert e6 < 0.03


def test_rod_closed_form_pins_itself():
    """The rod's 1-D field solves E u'' = rho s^2 u, u(0) = 0, E u'(L) = -p."""
    L, E, rho = 3.0, 1.0, 1.0
    for s in (0.3 + 0.4j, 0.2 + 1.0j):
        h = 1e-4
        f = lambda x: analytic.rod_field(x, s, L, E, rho)
        x = 1.7
        upp = (f(x + h) - 2 * f(x) + f(x - h)) / h**2
        assert abs(E * upp - rho * s * s * f(x)) <= 1e-5 * abs(rho * s * s * f(x))
        assert abs(f(0.0)) == 0.0
        assert abs(E * (f(L) - f(L - h)) / h + 1.0) <= 1e-3
        assert analytic.rod_end_displacement(s, L, E, rho) == pytest.approx(f(L))
        # traction on the fixed end (outward normal -x): -E u'(0)
        assert analytic.rod_fixed_traction(s, L, E, rho) == pytest.approx(-E * (f(h) - f(-h)) / (2 * h), rel=1e-6)


def _rod_errors(h, s):
    mat = kernels.Material(1.0, 0.0, 1.0)
    m = inputs.rod_problem(h=h)
    g = bem.geometry(m.xyz, m.tri)
    A, b = bem.system_rows(g, m.bc_type, m.pattern.astype(complex), s, mat)
    a = solvers.direct_solve(A, b).reshape(-1, 3)
    right = np.abs(g.c[:, 0] - 3.0) < 1e-9
    left = np.abs(g.c[:, 0]) < 1e-9
    uL = analytic.rod_end_displacement(s, 3.0, 1.0, 1.0)
    t0 = analytic.rod_fixed_traction(s, 3.0, 1.0, 1.0)
    return abs(a[right, 0].mean() - uL) / abs(uL), abs(a[left, 0].mean() - t0) / abs(t0)


def test_rod_mixed_bc_converges_to_1d_solution():
    """Mixed boundary conditions (fixed end: traction unknowns, -U columns)
    against the exact 1-D rod solution: the free-end displacement and the
    fixed-end traction converge as the mesh is refined."""
    s = 0.3 + 0.4j
    e_coarse = _rod_errors(0.5, s)
    e_fine = _rod_errors(1.0 / 3, s)
    for ec, ef in zip(e_coarse, e_fine):
        assert ef < 0.8 * ec
        assert ef < 0.03


def _manufactured_errors(xyz, tri, fixed, s):
    """Point force e at x0 outside the solid: u = e U(x0, .), t = e T(x0, .; n)
    solve the Navier equation inside, so prescribing them (u on the fixed
    elements, t elsewhere, sampled at the centroids) must return the other
    half as the mesh is refined."""
    x0, e = np.array([2.2, 0.9, -0.6]), np.array([0.3, -0.5, 0.8])
    g = bem.geometry(xyz, tri)
    bc = fixed(g.c).astype(np.int8)
    U, T = kernels.kernel_pair(x0, g.c, g.n, s, MAT)
    u, t = np.einsum("i,eij->ej", e, U), np.einsum("i,eij->ej", e, T)
    known = np.where(bc[:, None] == 1, u, t)
    want = np.where(bc[:, None] == 1, t, u)
    A, b = bem.system_rows(g, bc, known, s, MAT)
    a = solvers.direct_solve(A, b).reshape(-1, 3)
    free = bc == 0
    return (np.linalg.norm((a - want)[free]) / np.linalg.norm(want[free]),
            np.linalg.norm((a - want)[~free]) / np.linalg.norm(want[~free]))


def test_traction_kernel_is_the_traction_of_the_displacement_kernel():
    """e_i T_ij(x0, y; n) equals sigma(u) n for the field u_j = e_i U_ij(x0, y)
    (Hooke's law on central differences of U), the convention the
    manufactured solution below relies on."""
    x0, e, s = np.array([1.3, 0.2, -0.1]), np.array([0.3, -0.5, 0.8]), 0.5 + 1.0j
    y, n = np.array([0.5, -0.1, 0.2]), np.array([0.6, 0.0, 0.8])
    f = lambda yy: e @ kernels.displacement_kernel(x0, yy, s, MAT)
    h = 1e-5
    G = np.stack([(f(y + h * d) - f(y - h * d)) / (2 * h) for d in np.eye(3)], axis=1)
    eps = 0.5 * (G + G.T)
    sig = MAT.lam * np.trace(eps) * np.eye(3) + 2 * MAT.mu * eps
    assert np.allclose(e @ kernels.traction_kernel(x0, y, n, s, MAT), sig @ n, rtol=1e-6, atol=1e-9)


def test_manufactured_point_force_converges():
    """Mixed boundary conditions on a ball (lower cap fixed) and a box (bottom
    face fixed): the errors against the exact field fall at least at first
    order under refinement."""
    s = 0.5 + 1.0j
    eb = [_manufactured_errors(*inputs.geodesic_sphere(n), lambda c: c[:, 2] < -0.3, s) for n in (3, 5)]
    ex = [_manufactured_errors(*inputs.box_mesh(1.0, 1.0, 1.0, h), lambda c: np.abs(c[:, 2] + 0.5) < 1e-9, s)
          for h in (1 / 3, 1 / 5)]
    for coarse, fine, ratio in ((eb[0], eb[1], 0.6), (ex[0], ex[1], 0.6)):
        for ec, ef in zip(coarse, fine):
            assert ef < (ratio + 0.1) * ec
    assert eb[1][0] < 0.05 and eb[1][1] < 0.1


def test_interior_field_manufactured():
    """Representation formula at interior points of a box with the exact
    boundary data of a point force outside: the field converges to the point
    force's field; with the boundary solution of the mixed problem the error
    follows the boundary solution's."""
    x0, e, s = np.array([2.2, 0.9, -0.6]), np.array([0.3, -0.5, 0.8]), 0.5 + 1.0j
    P = np.array([[0.1, -0.2, 0.05], [0.3, 0.3, -0.3], [-0.35, 0.1, 0.4]])
    exact = np.einsum("i,pij->pj", e, kernels.displacement_kernel(x0, P, s, MAT))
    errs = []
    for h in (1 / 3, 1 / 5):
        xyz, tri = inputs.box_mesh(1.0, 1.0, 1.0, h)
        g = bem.geometry(xyz, tri)
        bc = (np.abs(g.c[:, 2] + 0.5) < 1e-9).astype(np.int8)
        U, T = kernels.kernel_pair(x0, g.c, g.n, s, MAT)
        u, t = np.einsum("i,eij->ej", e, U), np.einsum("i,eij->ej", e, T)
        known = np.where(bc[:, None] == 1, u, t)
        other = np.where(bc[:, None] == 1, t, u)
        f = bem.interior_field(g, bc, known, other, P, s, MAT)
        errs.append(np.linalg.norm(f - exact) / np.linalg.norm(exact))
    assert errs[0] < 0.015 and errs[1] < 0.7 * errs[0]


def test_interior_field_rod():
    """Interior displacement of the rod against its exact 1-D field."""
    mat = kernels.Material(1.0, 0.0, 1.0)
    rod = inputs.rod_problem(h=1 / 3)
    g = bem.geometry(rod.xyz, rod.tri)
    s = 0.3 + 0.4j
    A, b = bem.system_rows(g, rod.bc_type, rod.pattern.astype(complex), s, mat)
    a = solvers.direct_solve(A, b)
    xs = np.array([[0.5, 0.05, -0.1], [1.5, 0.0, 0.0], [2.5, -0.2, 0.1]])
    f = bem.interior_field(g, rod.bc_type, rod.pattern.astype(complex), a, xs, s, mat)
    ref = analytic.rod_field(xs[:, 0], s, 3.0, 1.0, 1.0)
    assert np.linalg.norm(f[:, 0] - ref) <= 0.03 * np.linalg.norm(ref)
    assert np.max(np.abs(f[:, 1:])) <= 0.01 * np.max(np.abs(ref))


def test_far_bands_against_brute_force():
    """Q2 and Q1 bands on a finer sphere (well-resolved frequency)."""
    mesh = inputs.cavity_problem(8)
    g = bem.geometry(mesh.xyz, mesh.tri)
    rng = np.random.default_rng(8)
    i = np.full(g.ne, 3)
    e = np.arange(g.ne)
    band = qd.classify(g.c[i], g.c[e], g.h[e], i == e)
    s = 0.625 + 1.0j
    for b, rt in ((qd.BAND_Q2, 2e-3), (qd.BAND_Q1, 2e-2)):
        sel = np.nonzero(band == b)[0]
        assert sel.size > 0
        pick = rng.choice(sel, size=6, replace=False)
        U, T = bem.pair_integrals(g, i[pick], e[pick], s, MAT)
        for m, p in enumerate(pick):
            Ur, Tr = _brute_regular(g, i[p], e[p], s)
            assert np.abs(U[m] - Ur).max() <= rt * np.abs(Ur).max()
            assert np.abs(T[m] - Tr).max() <= rt * np.abs(Tr).max()


def test_interior_strain_rod():
    """Interior strain of the rod (central differences of the representation
    formula) against the exact 1-D strain eps_xx = -(p / E) cosh(s x / c) /
    cosh(s L / c); the other components vanish (nu = 0). The error falls under
    refinement (252 -> 448 triangles: 2.2% -> 1.6% at the worst point)."""
    mat = kernels.Material(1.0, 0.0, 1.0)
    s = 0.3 + 0.4j
    xs = np.array([[0.5, 0.05, -0.1], [1.5, 0.0, 0.0], [2.5, -0.2, 0.1]])
    exact = -np.cosh(s * xs[:, 0]) / np.cosh(s * 3.0)
    errs = []
    for h in (1 / 3, 1 / 4):
        rod = inputs.rod_problem(h=h)
        g = bem.geometry(rod.xyz, rod.tri)
        A, b = bem.system_rows(g, rod.bc_type, rod.pattern.astype(complex), s, mat)
        a = solvers.direct_solve(A, b)
        eps = bem.interior_strain(g, rod.bc_type, rod.pattern.astype(complex), a, xs, s, mat, 0.02)
        errs.append(np.abs(eps[:, 0] - exact).max() / np.abs(exact).max())
        assert np.abs(eps[:, 1:]).max() <= 0.04 * np.abs(exact).max()
    assert errs[0] < 0.03 and errs[1] < 0.85 * errs[0]
