"""Pins for the oracle's solvers (Sec. 4.2 and Sec. 5).

* GMRES with the 3x3 block-Jacobi right preconditioner reaches the LU
  solution on random systems and on a small BEM system;
* the SEM guess (Eqs. a0, lsem, a0-solution) is exact when b_k lies in
  A_k span(X), its residual never exceeds that of a_{k-1} (a_{k-1} is in
  span(X)), and dependent columns are dropped.
"""
import numpy as np
import pytest

from oracle import bem, kernels, solvers
from paper_1212_3032_gb300 import inputs


def _rand_system(n, rng, diag=3.0):
    A = rng.normal(size=(n, n)) + 1j * rng.normal(size=(n, n))
    A = A / np.sqrt(n) + diag * np.eye(n)
    b = rng.normal(size=n) + 1j * rng.normal(size=n)
    return A, b


@pytest.mark.parametrize("restart", [5, 50])
def test_gmres_matches_lu(restart):
    rng = np.random.default_rng(11)
    A, b = _rand_system(60, rng)
    x_ref = solvers.direct_solve(A, b)
    x, its, rel = solvers.gmres(A, b, tol=1e-12, restart=restart)
    assert rel <= 1e-12
    assert np.linalg.norm(x - x_ref) <= 1e-10 * np.linalg.norm(x_ref)
    assert its > 0


def test_gmres_on_bem_system():
    mat = kernels.Material(1.0, 0.25, 1.0)
    mesh = inputs.cavity_problem(2)
    g = bem.geometry(mesh.xyz, mesh.tri)
    A, b = bem.system_rows(g, mesh.bc_type, mesh.pattern.astype(complex), 0.625 + 2.0j, mat)
    x_ref = solvers.direct_solve(A, b)
    x, its, rel = solvers.gmres(A, b, tol=1e-11, restart=30)
    assert rel <= 1e-11
    assert np.linalg.norm(x - x_ref) <= 1e-9 * np.linalg.norm(x_ref)
    # an exact initial guess needs no iteration
    _, its0, _ = solvers.gmres(A, b, x0=x_ref, tol=1e-10)
    assert its0 == 0


def test_sem_exact_in_span():
    rng = np.random.default_rng(12)
    A, _ = _rand_system(40, rng)
    X = rng.normal(size=(40, 3)) + 1j * rng.normal(size=(40, 3))
    c = np.array([0.5 - 1j, 2.0, -0.3j])
    b = A @ (X @ c)
    a0, s = solvers.sem_guess(A, b, X)
    assert np.allclose(s, c, rtol=1e-10, atol=1e-12)
    assert np.linalg.norm(A @ a0 - b) <= 1e-12 * np.linalg.norm(b)


def test_sem_residual_bound_and_rank_drop():
    rng = np.random.default_rng(13)
    A, b = _rand_system(50, rng)
    X = rng.normal(size=(50, 4)) + 1j * rng.normal(size=(50, 4))
    a0, _ = solvers.sem_guess(A, b, X)
    r0 = np.linalg.norm(A @ a0 - b)
    for j in range(4):
        # least squares over span(X) beats every single column's best multiple
        y = A @ X[:, j]
        best = np.linalg.norm(b - y * (np.vdot(y, b) / np.vdot(y, y)))
        assert r0 <= best * (1 + 1e-12)
    Xd = np.concatenate([X[:, :2], X[:, :1] * 2.0, X[:, 2:]], axis=1)
    a1, s1 = solvers.sem_guess(A, b, Xd)
    assert s1.size == 4
    assert np.linalg.norm(a1 - a0) <= 1e-10 * np.linalg.norm(a0)
    a_none, s_none = solvers.sem_guess(A, b, np.zeros((50, 0)))
    assert s_none.size == 0 and np.all(a_none == 0)


def test_bisection_clusters_partition():
    rng = np.random.default_rng(5)
    c = rng.normal(size=(1000, 3))
    groups = solvers.bisection_clusters(c, 64)
    allidx = np.sort(np.concatenate(groups))
    assert np.array_equal(allidx, np.arange(1000))
    assert max(g.size for g in groups) <= 64 and min(g.size for g in groups) >= 32


def test_cluster_preconditioner_on_the_rod():
    """Larger diagonal blocks (element groups of 64) on the mixed-boundary rod:
    the same solution with far fewer iterations than the 3x3 blocks (the
    fixed end's traction unknowns make part of the operator first kind)."""
    from oracle import transforms as tr
    mat = kernels.Material(1.0, 0.0, 1.0)
    rod = inputs.rod_problem(h=0.25)
    g = bem.geometry(rod.xyz, rod.tri)
    s = tr.eta_from_kappa(4, 26.8 * 3.0) + 4.71j
    A, b = bem.system_rows(g, rod.bc_type, rod.pattern.astype(complex), s, mat)
    x_ref = solvers.direct_solve(A, b)
    x3, it3, r3 = solvers.gmres(A, b, tol=1e-8)
    xg, itg, rg = solvers.gmres(A, b, tol=1e-8, groups=solvers.bisection_clusters(g.c, 64))
    assert r3 <= 1e-8 and rg <= 1e-8
    for x in (x3, xg):
        assert np.linalg.norm(x - x_ref) <= 1e-6 * np.linalg.norm(x_ref)
    assert itg < 0.7 * it3


def test_paper_iteration_trends_on_the_rod():
    """The paper's qualitative trends (Sec. 5.1, Table 1) on the oracle: on the
    rod (252 triangles, T = 26.8 L/c, the first 9 of 16 samples), a larger
    damping (kappa 4 against 2) does not need more GMRES steps, and the
    solution extrapolation (K = 4) cuts them by over a quarter."""
    import math
    from oracle import transforms as tr
    mat = kernels.Material(1.0, 0.0, 1.0)
    rod = inputs.rod_problem(h=1 / 3)
    g = bem.geometry(rod.xyz, rod.tri)
    T, N = 26.8 * 3.0, 16
    hist = inputs.heaviside_history(N)
    its = {}
    for kappa in (2, 4):
        eta = tr.eta_from_kappa(kappa, T)
        Pk = tr.dft_mft(hist, T, eta)
        zero = sem = 0
        prev = []
        for k in range(N // 2 + 1):
            s = eta + 1j * k * 2 * math.pi / T
            A, b = bem.system_rows(g, rod.bc_type, rod.pattern * Pk[k], s, mat)
            x, it, rel = solvers.gmres(A, b, tol=1e-5)
            assert rel <= 1e-5
            zero += it
            if kappa == 4:
                K = min(k, 4)
                X = np.stack(prev[-K:][::-1], axis=1) if K else np.zeros((b.size, 0))
                a0, _ = solvers.sem_guess(A, b, X)
                _, it2, _ = solvers.gmres(A, b, x0=a0, tol=1e-5)
                sem += it2
            prev.append(x)
        its[kappa] = (zero, sem)
    assert its[4][0] <= its[2][0]
    assert its[4][1] <= 0.75 * its[4][0]
