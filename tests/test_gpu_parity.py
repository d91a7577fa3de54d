"""Parity of the CUDA path with the CPU oracle, step by step, through the C-ABI.

Tolerances (written from the arithmetic):
* mixed precision (c64 storage, FP32 kernel evaluation): single entries carry
  a few FP32 roundings (~1e-6 relative); rows/vectors are compared at 2e-5;
* plain (c128 everywhere): 1e-8 -- the oracle evaluates the radial
  functions by their closed forms, whose 1/z^3 terms cancel to O(1), so at
  |z| ~ 1e-3 (innermost polar nodes of the self element at low frequency) it
  keeps only ~8 digits; the GPU path sums the Taylor series there;
* low-rank blocks add the ACA tolerance (rows compared at 30 x aca_tol);
* solutions: the target 1e-4 relative L2 in the frequency domain
  and 1e-3 for time traces (mixed); plain form 1e-8 / 1e-7.
"""
import math

import numpy as np
import pytest

from oracle import bem, kernels, solvers, sweep as osweep, transforms
from paper_1212_3032_gb300 import inputs

pytestmark = pytest.mark.gpu

MAT = kernels.Material(1.0, 0.25, 1.0)


@pytest.fixture(scope="module")
def B():
    from paper_1212_3032_gb300 import binding, build
    build.build()
    return binding


@pytest.fixture(scope="module")
def ctx(B):
    c = B.Context(0)
    c.set_material(MAT.E, MAT.nu, MAT.rho)
    yield c
    c.close()


def _rel(a, b):
    return np.linalg.norm(np.asarray(a) - np.asarray(b)) / max(np.linalg.norm(b), 1e-300)


# ---------------------------------------------------------------------------
# transforms
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("N", [2, 32, 256, 1000])
def test_load_dft(ctx, N):
    T = 8.0
    eta = 5.0 / T
    rng = np.random.default_rng(N)
    P = rng.normal(size=N)
    P[0] = 0.5
    got = ctx.load_dft(T, N, eta, P)
    ref = transforms.dft_mft(P, T, eta)
    assert _rel(got, ref) <= 1e-13


@pytest.mark.parametrize("win", [0, 1, 2])
@pytest.mark.parametrize("N,ndof", [(32, 7), (128, 100), (4096, 3)])
def test_idft(ctx, win, N, ndof):
    T = 3.0
    eta = transforms.eta_from_kappa(4.0, T)
    rng = np.random.default_rng(win * 1000 + N)
    Rk = rng.normal(size=(N // 2 + 1, ndof)) + 1j * rng.normal(size=(N // 2 + 1, ndof))
    got = ctx.idft(T, N, eta, win, Rk)
    ref = transforms.idft_mft(Rk, T, eta, win, N)
    assert np.abs(got - ref).max() <= 1e-11 * np.abs(ref).max()


def test_idft_empty_and_invalid(ctx, B):
    out = ctx.idft(1.0, 8, 0.1, 1, np.zeros((5, 0)))
    assert out.shape == (8, 0)
    with pytest.raises(B.BemError):
        ctx.idft(1.0, 7, 0.1, 1, np.zeros((4, 1)))
    with pytest.raises(B.BemError):
        ctx.load_dft(1.0, 9, 0.1, np.zeros(9))


# ---------------------------------------------------------------------------
# operator entries
# ---------------------------------------------------------------------------
def _mesh_ctx(ctx, B, mesh, **kw):
    o = B.default_opts(**kw)
    ctx.mesh(mesh.xyz, mesh.tri, mesh.bc_type, o)
    return o


@pytest.mark.parametrize("prec,tol", [(0, 2e-5), (1, 1e-8)])
@pytest.mark.parametrize("s", [0.625, 0.625 + 5.0j, 0.3 + 40.0j])
def test_dense_rows_match_oracle(ctx, B, prec, tol, s):
    mesh = inputs.cavity_problem(4)                       # 320 elements
    o = _mesh_ctx(ctx, B, mesh, dense=1, precision=prec)
    ctx.assemble(s, o)
    g = bem.geometry(mesh.xyz, mesh.tri)
    rows_e = np.array([0, 1, 77, 160, 319])
    A_ref, _ = bem.system_rows(g, mesh.bc_type, np.zeros((mesh.ne, 3)), s, MAT, rows=rows_e)
    rows = np.concatenate([3 * rows_e + a for a in range(3)])
    order = np.argsort(rows)
    got = ctx.operator_rows(rows[order])
    ref = np.concatenate([A_ref[a::3] for a in range(3)])[order]
    for r in range(got.shape[0]):
        assert _rel(got[r], ref[r]) <= tol


def _mixed_bc_mesh():
    # small cube with two cavities: bottom fixed (Gamma_u), top loaded
    return inputs.cube_with_cavities(n_face=8, n_cav=2, cav_radius=0.12, cav_n=3, seed=5)


@pytest.mark.parametrize("prec,tol", [(0, 2e-5), (1, 1e-8)])
def test_mixed_bc_rows_and_rhs(ctx, B, prec, tol):
    mesh = _mixed_bc_mesh()
    o = _mesh_ctx(ctx, B, mesh, dense=1, precision=prec)
    s = 2.0 + 3.0j
    ctx.assemble(s, o)
    g = bem.geometry(mesh.xyz, mesh.tri)
    pk = 0.3 - 0.2j
    rows_e = np.array([0, 5, 64, 127, 300, mesh.ne - 1])
    A_ref, b_ref = bem.system_rows(g, mesh.bc_type, mesh.pattern * pk, s, MAT, rows=rows_e)
    for m, e in enumerate(rows_e):
        got = ctx.operator_rows(3 * e + np.arange(3))
        for a in range(3):
            assert _rel(got[a], A_ref[3 * m + a]) <= tol
    b = ctx.rhs(pk, mesh.pattern)
    b_sel = np.concatenate([b[3 * e:3 * e + 3] for e in rows_e])
    assert _rel(b_sel, b_ref) <= tol


@pytest.mark.parametrize("prec", [0, 1])
def test_hmatrix_rows_match_oracle(ctx, B, prec):
    # 980 elements, leaf 32: 708 dense near blocks, 316 ACA blocks, ragged leaves
    mesh = inputs.cavity_problem(7)
    aca_tol = 1e-5
    o = _mesh_ctx(ctx, B, mesh, dense=0, precision=prec, aca_tol=aca_tol, leaf_size=32)
    s = 0.625 + 3.0j
    ctx.set_profiling(True)
    ctx.assemble(s, o)
    assert ctx.get_profile()["aca_blocks"] > 300
    ctx.set_profiling(False)
    g = bem.geometry(mesh.xyz, mesh.tri)
    rows_e = np.array([0, 333, 979])
    A_ref, _ = bem.system_rows(g, mesh.bc_type, np.zeros((mesh.ne, 3)), s, MAT, rows=rows_e)
    for m, e in enumerate(rows_e):
        got = ctx.operator_rows(3 * e + np.arange(3))
        for a in range(3):
            assert _rel(got[a], A_ref[3 * m + a]) <= 30 * aca_tol
    # the product through the hierarchical kernels equals the stored operator
    rng = np.random.default_rng(3)
    x = rng.normal(size=3 * mesh.ne) + 1j * rng.normal(size=3 * mesh.ne)
    y = ctx.apply(x)
    rows = ctx.operator_rows(np.arange(0, 3 * mesh.ne, 97))
    assert _rel(y[::97], rows @ x) <= (2e-6 if prec == 0 else 1e-12)


@pytest.mark.parametrize("prec", [0, 1])
def test_hmatrix_rows_after_pivot_reuse(ctx, B, prec):
    """Assemblies that start from the previous frequency's ACA pivots meet the
    same accuracy as a fresh ACA, for a neighbouring frequency and after a
    large jump in s (where most reused pivots fail the pivot test)."""
    mesh = inputs.cavity_problem(7)
    aca_tol = 1e-5
    o = _mesh_ctx(ctx, B, mesh, dense=0, precision=prec, aca_tol=aca_tol, leaf_size=32)
    g = bem.geometry(mesh.xyz, mesh.tri)
    rows_e = np.array([0, 333, 979])
    ctx.set_aca_reuse(True)
    ctx.assemble(0.625 + 2.8j, o)                         # cold: first assembly on this mesh
    for s in (0.625 + 3.0j, 0.3 + 9.0j):
        ctx.set_profiling(True)
        ctx.assemble(s, o)                                # warm
        prof = ctx.get_profile()
        ctx.set_profiling(False)
        assert prof["aca_blocks"] > 0
        if s == 0.625 + 3.0j:
            # a neighbouring frequency: reuse settles a good share of the blocks
            assert prof["aca_stepped"] < 0.75 * prof["aca_blocks"]
        A_ref, _ = bem.system_rows(g, mesh.bc_type, np.zeros((mesh.ne, 3)), s, MAT, rows=rows_e)
        for m, e in enumerate(rows_e):
            got = ctx.operator_rows(3 * e + np.arange(3))
            for a in range(3):
                assert _rel(got[a], A_ref[3 * m + a]) <= 30 * aca_tol, (s, e, a)
        rng = np.random.default_rng(4)
        x = rng.normal(size=3 * mesh.ne) + 1j * rng.normal(size=3 * mesh.ne)
        y = ctx.apply(x)
        rows = ctx.operator_rows(np.arange(0, 3 * mesh.ne, 97))
        assert _rel(y[::97], rows @ x) <= (2e-6 if prec == 0 else 1e-12)


def test_pivot_reuse_switch(ctx, B):
    """With reuse off every assembly is a fresh ACA (all blocks stepped)."""
    mesh = inputs.cavity_problem(7)
    o = _mesh_ctx(ctx, B, mesh, dense=0, precision=0, aca_tol=1e-5, leaf_size=32)
    ctx.set_aca_reuse(False)
    try:
        ctx.assemble(0.625 + 2.8j, o)
        ctx.set_profiling(True)
        ctx.assemble(0.625 + 3.0j, o)
        prof = ctx.get_profile()
        ctx.set_profiling(False)
        assert prof["aca_stepped"] == prof["aca_blocks"] > 0
    finally:
        ctx.set_aca_reuse(True)


@pytest.mark.parametrize("k", [64, 128])
def test_hmatrix_full_size_sampled_rows(ctx, B, k):
    """The 5,120-element cavity at the benchmark's settings (leaf 64, ACA
    1e-5, complex64 mixed precision): 4,874 admissible blocks, 246 of them
    above 256 elements (one CTA each), the rest one warp each. Sampled rows
    match the oracle at frequency k (fresh ACA) and at k + 1 (pivot reuse)."""
    mesh = inputs.cavity_problem(16)
    aca_tol = 1e-5
    o = _mesh_ctx(ctx, B, mesh, dense=0, precision=0, aca_tol=aca_tol, leaf_size=64)
    T = 64.0
    g = bem.geometry(mesh.xyz, mesh.tri)
    rows_e = np.array([0, 1, 777, 2500, 2501, 4095, 5000, 5119])
    for kk, warm in ((k, False), (k + 1, True)):
        s = 5.0 / T + 1j * kk * 2 * math.pi / T
        ctx.set_profiling(True)
        ctx.assemble(s, o)
        prof = ctx.get_profile()
        ctx.set_profiling(False)
        assert prof["aca_blocks"] == 4874
        if warm:
            assert prof["aca_stepped"] < prof["aca_blocks"]
        A_ref, b_ref = bem.system_rows(g, mesh.bc_type, mesh.pattern.astype(complex), s, MAT, rows=rows_e)
        got = ctx.operator_rows((3 * rows_e[:, None] + np.arange(3)).ravel())
        for q in range(3 * len(rows_e)):
            assert _rel(got[q], A_ref[q]) <= 30 * aca_tol, (kk, q)
        # right-hand side: near, singular and far (on-the-fly) contributions
        b = ctx.rhs(1.0, mesh.pattern)
        b_sel = b[(3 * rows_e[:, None] + np.arange(3)).ravel()]
        assert _rel(b_sel, b_ref) <= 2e-5, kk


# ---------------------------------------------------------------------------
# solves
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("prec,tol,ptol", [(0, 1e-7, 1e-4), (1, 1e-11, 1e-8)])
def test_solve_matches_direct(ctx, B, prec, tol, ptol):
    mesh = inputs.cavity_problem(4)
    o = _mesh_ctx(ctx, B, mesh, dense=1, precision=prec, tol=tol)
    s = 0.625 + 2.0j
    ctx.assemble(s, o)
    g = bem.geometry(mesh.xyz, mesh.tri)
    A, b = bem.system_rows(g, mesh.bc_type, mesh.pattern.astype(complex), s, MAT)
    x_ref = solvers.direct_solve(A, b)
    bg = ctx.rhs(1.0, mesh.pattern)
    assert _rel(bg, b) <= (2e-5 if prec == 0 else 1e-8)
    x, st = ctx.solve_assembled(bg, opts=o)
    assert st["converged"] == 1 and st["rel_residual"] <= tol
    assert _rel(x, x_ref) <= ptol


def test_sem_guess_matches_oracle(ctx, B):
    mesh = inputs.cavity_problem(4)
    o = _mesh_ctx(ctx, B, mesh, dense=1, precision=1)
    T, N = 8.0, 32
    eta = 5.0 / T
    ref = osweep.solve_sweep(mesh, MAT, T, N, eta, inputs.heaviside_history(N), ks=np.arange(6))
    k = 5
    s = ref["s"][k]
    ctx.assemble(s, o)
    g = bem.geometry(mesh.xyz, mesh.tri)
    A, b = bem.system_rows(g, mesh.bc_type, mesh.pattern * ref["Pk"][k], s, MAT)
    X = ref["a"][k - 4:k][::-1]                           # a_{k-1}, ..., a_{k-4}
    a0_ref, _ = solvers.sem_guess(A, b, X.T)
    a0 = ctx.sem_guess(X, b)
    assert _rel(a0, a0_ref) <= 1e-8
    r_ref = np.linalg.norm(A @ a0_ref - b) / np.linalg.norm(b)
    r_k1 = np.linalg.norm(A @ X[0] - b) / np.linalg.norm(b)
    assert r_ref <= r_k1
    # dependent columns are dropped, not divided by
    a0d = ctx.sem_guess(np.stack([X[0], X[0] * 2.0, X[1]]), b)
    a0d_ref, _ = solvers.sem_guess(A, b, np.stack([X[0], X[0] * 2.0, X[1]]).T)
    assert _rel(a0d, a0d_ref) <= 1e-8


# ---------------------------------------------------------------------------
# the sweep (320-element cavity, 32 samples: 17 solves)
# ---------------------------------------------------------------------------
@pytest.fixture(scope="module")
def oracle_sweep():
    mesh = inputs.cavity_problem(4)
    T, N = 8.0, 32
    eta = 5.0 / T
    ref = osweep.solve_sweep(mesh, MAT, T, N, eta, inputs.heaviside_history(N))
    return mesh, T, N, eta, ref


@pytest.mark.parametrize("prec,guess,ftol,ttol", [(1, 0, 1e-8, 1e-7), (0, 1, 1e-4, 1e-3), (0, 0, 1e-4, 1e-3)])
def test_sweep_matches_oracle(ctx, B, oracle_sweep, prec, guess, ftol, ttol):
    mesh, T, N, eta, ref = oracle_sweep
    # residual one decade below the solution tolerance (error <= condition x residual)
    o = _mesh_ctx(ctx, B, mesh, dense=1, precision=prec, guess=guess, tol=1e-9 if prec == 1 else 1e-7)
    for win in (0, 1):
        ctx.set_window(eta, win)
        stats = ctx.solve_sweep(T, N, inputs.heaviside_history(N), mesh.pattern, o)
        assert len(stats) == N // 2 + 1
        assert all(s["converged"] == 1 for s in stats)
        for k in range(N // 2 + 1):
            a = ctx.get_frequency_solution(k)
            assert _rel(a, ref["a"][k]) <= ftol, k
            assert stats[k]["s_im"] == pytest.approx(k * 2 * math.pi / T)
        dofs = np.array([0, 1, 2, 500, 959])
        tr = ctx.time_response(dofs)
        tr_ref = osweep.time_response(ref["a"], T, eta, win, N, dofs)
        assert np.linalg.norm(tr - tr_ref) <= ttol * np.linalg.norm(tr_ref)


def test_sem_reduces_iterations(ctx, B, oracle_sweep):
    mesh, T, N, eta, _ = oracle_sweep
    ctx.set_window(eta, 1)
    its = {}
    for guess in (0, 1):
        o = _mesh_ctx(ctx, B, mesh, dense=1, precision=0, guess=guess, tol=1e-5)
        stats = ctx.solve_sweep(T, N, inputs.heaviside_history(N), mesh.pattern, o)
        its[guess] = sum(s["iters"] for s in stats)
        if guess == 1:
            # the extrapolated guess is never worse than the zero guess after k >= 1
            assert all(s["guess_residual"] < 1.0 for s in stats[1:])
    assert its[1] < its[0]


# ---------------------------------------------------------------------------
# edge cases and errors (host-side validation: nothing reaches a kernel)
# ---------------------------------------------------------------------------
def test_invalid_inputs(ctx, B):
    mesh = inputs.cavity_problem(2)
    with pytest.raises(B.BemError):
        ctx.mesh(mesh.xyz, mesh.tri + 1000, mesh.bc_type)
    bad = mesh.tri.copy()
    bad[0, 1] = bad[0, 0]
    with pytest.raises(B.BemError):
        ctx.mesh(mesh.xyz, bad, mesh.bc_type)
    with pytest.raises(B.BemError):
        ctx.set_material(-1.0, 0.25, 1.0)
    with pytest.raises(B.BemError):
        ctx.set_material(1.0, 0.5, 1.0)
    with pytest.raises(B.BemError):
        ctx.set_window(-1.0, 0)
    ctx.mesh(mesh.xyz, mesh.tri, mesh.bc_type)
    with pytest.raises(B.BemError):
        ctx.solve_sweep(8.0, 31, np.ones(31), mesh.pattern)
    ctx.set_material(MAT.E, MAT.nu, MAT.rho)


def test_single_element_and_tiny_sweep(ctx, B):
    # smallest closed surface (a tetrahedron); N = 2 samples: k = 0, 1
    xyz = np.array([[0, 0, 0], [1, 0, 0], [0, 1, 0], [0, 0, 1.0]])
    tri = np.array([[0, 2, 1], [0, 1, 3], [0, 3, 2], [1, 2, 3]], dtype=np.int32)
    m = inputs.pressurised_surface(xyz, tri)
    o = B.default_opts(dense=1, precision=1, tol=1e-12)
    ctx.mesh(m.xyz, m.tri, m.bc_type, o)
    ctx.set_window(0.5, 0)
    stats = ctx.solve_sweep(4.0, 2, inputs.heaviside_history(2), m.pattern, o)
    ref = osweep.solve_sweep(m, MAT, 4.0, 2, 0.5, inputs.heaviside_history(2))
    for k in range(2):
        assert _rel(ctx.get_frequency_solution(k), ref["a"][k]) <= 1e-9
    assert len(stats) == 2


def test_device_pointer_entry_points(ctx, B):
    """The _dev variants give the same sweep as the host-pointer API."""
    import torch
    mesh = inputs.cavity_problem(3)
    T, N = 8.0, 16
    o = B.default_opts(dense=0, leaf_size=16, precision=0, tol=1e-7)
    ctx.set_window(5.0 / T, 1)
    ctx.mesh(mesh.xyz, mesh.tri, mesh.bc_type, o)
    ctx.solve_sweep(T, N, inputs.heaviside_history(N), mesh.pattern, o)
    a_host = [ctx.get_frequency_solution(k) for k in range(N // 2 + 1)]
    tr_host = ctx.time_response(np.arange(3 * mesh.ne))
    dev = torch.device("cuda", 0)
    xyz = torch.tensor(mesh.xyz, device=dev)
    tri = torch.tensor(mesh.tri, device=dev)
    bc = torch.tensor(mesh.bc_type, device=dev)
    with pytest.raises(ValueError):
        ctx.mesh_dev(xyz, tri.t().contiguous().t(), bc, o)      # non-contiguous layout is refused
    ctx.mesh_dev(xyz, tri, bc, o)
    ctx.solve_sweep_dev(T, N, torch.tensor(inputs.heaviside_history(N), device=dev),
                        torch.tensor(mesh.pattern, device=dev), o)
    # the right-hand side is summed with atomics (FP32 partial sums on the mixed
    # path), so two runs agree to FP32 rounding, not bitwise
    for k in range(N // 2 + 1):
        assert _rel(ctx.get_frequency_solution(k), a_host[k]) <= 2e-6
    out = torch.empty((N, 3 * mesh.ne), dtype=torch.float64, device=dev)
    ctx.time_response_dev(torch.arange(3 * mesh.ne, device=dev), out)
    assert np.abs(out.cpu().numpy() - tr_host).max() <= 2e-6 * np.abs(tr_host).max()
    with pytest.raises(B.BemError):
        ctx.time_response_dev(torch.tensor([0, 3 * mesh.ne], device=dev), torch.empty((N, 2), dtype=torch.float64,
                                                                                       device=dev))
