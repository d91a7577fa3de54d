"""Far-field factor storage, and the large cube with cavities at full size.

* Compact storage (ACA batch by batch in a workspace, factors packed at their
  ranks into pools that grow on overflow) gives the same operator, bit for
  bit, as full storage (capped factors written in place): products and
  stored rows, in complex64 and complex128, through fresh ACA, pivot reuse
  and a pool overflow in either. Sweeps agree to the solver tolerance (the
  right-hand side sums with atomics, so its last bits vary run to run).
* The unit cube with 8 cavities (231,088 triangles, 693,264 unknowns,
  bottom fixed, top loaded: mixed boundary conditions) at ACA tolerance 1e-4
  in complex64 selects compact storage by itself, stays under 180 GB of
  device memory, matches the oracle on sampled operator rows and right-hand
  side entries, and its GMRES solution leaves no sampled stored row with a
  residual above the residual norm the solver reports.
"""
import math

import numpy as np
import pytest

from oracle import bem, kernels
from paper_1212_3032_gb300 import inputs

pytestmark = pytest.mark.gpu

MAT = kernels.Material(1.0, 0.25, 1.0)


@pytest.fixture(scope="module")
def B():
    from paper_1212_3032_gb300 import binding, build
    build.build()
    return binding


def _ctx(B, mode, ws=0):
    c = B.Context(0)
    c.set_material(MAT.E, MAT.nu, MAT.rho)
    c.set_far_storage(mode, ws)
    return c


def _mesh(c, B, mesh, prec, aca_tol=1e-5, leaf=64, **kw):
    o = B.default_opts(dense=0, precision=prec, aca_tol=aca_tol, leaf_size=leaf, **kw)
    c.mesh(mesh.xyz, mesh.tri, mesh.bc_type, o)
    return o


def _rel(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


@pytest.mark.parametrize("prec", [0, 1])
def test_compact_equals_full(B, prec):
    mesh = inputs.cavity_problem(16)
    T = 64.0
    full = _ctx(B, B.FAR_FULL)
    comp = _ctx(B, B.FAR_COMPACT, 64 << 20)  # many batches
    try:
        of = _mesh(full, B, mesh, prec)
        oc = _mesh(comp, B, mesh, prec)
        assert full.far_storage()["compact"] == 0 and full.far_storage()["batches"] == 1
        assert comp.far_storage()["compact"] == 1 and comp.far_storage()["batches"] > 4
        rng = np.random.default_rng(7)
        x = rng.normal(size=3 * mesh.ne) + 1j * rng.normal(size=3 * mesh.ne)
        # fresh ACA near s = eta (the pools start below the need: overflow,
        # regrowth and a redo), pivot reuse, then a jump to a high frequency
        # whose ranks outgrow the pools again (a redo from the reused pivots)
        regrows = []
        for k in (0, 1, 120):
            s = 5.0 / T + 1j * k * 2 * math.pi / T
            full.assemble(s, of)
            comp.assemble(s, oc)
            assert np.array_equal(full.apply(x), comp.apply(x)), k
            fs, cs = full.far_storage(), comp.far_storage()
            assert cs["used_bytes"] == fs["used_bytes"], k
            assert cs["used_bytes"] <= cs["factor_bytes"] < fs["factor_bytes"], k
            assert cs["workspace_bytes"] > 0 and fs["workspace_bytes"] == 0
            regrows.append(cs["regrows"])
        assert regrows[0] >= 1 and regrows[2] > regrows[1], regrows
        rows = np.array([0, 1, 7000, 3 * mesh.ne - 1])
        assert np.array_equal(comp.operator_rows(rows), full.operator_rows(rows))
        np.testing.assert_array_equal(comp.far_block_info(), full.far_block_info())
    finally:
        full.close()
        comp.close()


def test_compact_sweep_equals_pipelined_sweep(B):
    # compact storage keeps one operator set and assembles frequency k + 1
    # after solving k; full storage overlaps the two: same arithmetic
    mesh = inputs.cavity_problem(7)
    T, N = 8.0, 16
    hist = inputs.heaviside_history(N)
    sols = []
    for mode in (B.FAR_FULL, B.FAR_COMPACT):
        c = _ctx(B, mode, 1 << 20)
        try:
            o = _mesh(c, B, mesh, 0, leaf=32, tol=1e-6)
            c.set_window(5.0 / T, 1)
            stats = c.solve_sweep(T, N, hist, mesh.pattern, o)
            assert all(s["converged"] == 1 for s in stats)
            sols.append(np.stack([c.get_frequency_solution(k) for k in range(N // 2 + 1)]))
            if mode == B.FAR_COMPACT:
                assert c.far_storage()["batches"] > 1
        finally:
            c.close()
    for k in range(N // 2 + 1):
        assert _rel(sols[1][k], sols[0][k]) <= 2e-5, k


@pytest.mark.parametrize("prec,aca_tol", [(1, 1e-6), (0, 1e-5)])
def test_flat_face_blocks(B, prec, aca_tol):
    # cube faces: coplanar admissible blocks couple normal rows only to
    # tangential columns and tangential rows only to normal columns; ACA must
    # approximate both parts (its per-component check rows), also when the
    # previous frequency's pivots are reused. k = 16 (|s| = 12.6): the ranks
    # of the largest flat-face blocks go above 128; none may stop at the cap
    mesh = inputs.cube_with_cavities(n_face=24, n_cav=2, cav_radius=0.15, cav_n=8, seed=3032)
    c = _ctx(B, B.FAR_AUTO)
    try:
        o = _mesh(c, B, mesh, prec, aca_tol=aca_tol)
        T = 8.0
        g = bem.geometry(mesh.xyz, mesh.tri)
        rows_e = np.array([10, 500, 1500, 3000, 4000, 6000, mesh.ne - 5])
        sel = (3 * rows_e[:, None] + np.arange(3)).ravel()
        for k in (16, 17):  # fresh ACA, then pivot reuse
            s = 4.0 / T + 1j * k * 2 * math.pi / T
            c.set_profiling(True)
            c.assemble(s, o)
            prof = c.get_profile()
            c.set_profiling(False)
            assert prof["aca_failures"] == 0, k
            A_ref, _ = bem.system_rows(g, mesh.bc_type, mesh.pattern.astype(complex), s, MAT, rows=rows_e)
            got = c.operator_rows(sel)
            err = np.array([_rel(got[q], A_ref[q]) for q in range(len(sel))])
            # ACA's stopping test bounds a block's Frobenius error by about
            # aca_tol; a block missing its second part is off by 1e3 aca_tol
            assert err.max() <= 30 * aca_tol, (k, err)
    finally:
        c.close()


def test_storage_arguments(B):
    c = B.Context(0)
    try:
        with pytest.raises(B.BemError):
            c.set_far_storage(3)
        with pytest.raises(B.BemError):
            c.set_far_storage(B.FAR_COMPACT, -1)
        with pytest.raises(B.BemError):
            c.far_storage()  # no mesh
    finally:
        c.close()


def test_cube_with_cavities_full_size(B):
    import torch
    mesh = inputs.cube_with_cavities()
    assert mesh.ne == 231088
    aca_tol, tol = 1e-4, 1e-5
    c = _ctx(B, B.FAR_AUTO)
    try:
        o = _mesh(c, B, mesh, 0, aca_tol=aca_tol, tol=tol)
        assert c.far_storage()["compact"] == 1
        T = 8.0
        s = 4.0 / T + 1j * 16 * 2 * math.pi / T
        c.set_profiling(True)
        c.assemble(s, o)
        assert c.get_profile()["aca_failures"] == 0
        c.set_profiling(False)
        free, total = torch.cuda.mem_get_info()
        assert total - free < 180e9
        st = c.far_storage()
        assert st["used_bytes"] <= st["factor_bytes"]
        # sampled rows: bottom (fixed) face, top (loaded) face, side faces and cavities
        zc = mesh.xyz[mesh.tri].mean(axis=1)[:, 2]
        bottom = np.flatnonzero(mesh.bc_type == 1)
        top = np.flatnonzero(np.abs(zc - 0.5) < 1e-6)
        rows_e = np.unique(np.concatenate([bottom[[0, len(bottom) // 2]], top[[3, len(top) - 1]],
                                           [1000, 90000, 167087, 167088, 200000, mesh.ne - 1]]))
        g = bem.geometry(mesh.xyz, mesh.tri)
        A_ref, b_ref = bem.system_rows(g, mesh.bc_type, mesh.pattern.astype(complex), s, MAT, rows=rows_e)
        sel = (3 * rows_e[:, None] + np.arange(3)).ravel()
        got = c.operator_rows(sel)
        err = np.array([_rel(got[q], A_ref[q]) for q in range(len(sel))])
        assert err.max() <= 30 * aca_tol, err
        b = c.rhs(1.0, mesh.pattern)
        assert _rel(b[sel], b_ref) <= 1e-4
        x, stats = c.solve_assembled(b, opts=o)
        assert stats["converged"] == 1 and stats["rel_residual"] <= tol
        # the solution against the stored rows, reconstructed on the host in
        # FP64: no row's residual exceeds the residual norm (tol |b|, with a
        # factor 2 for the FP32 products of the residual test)
        r = b[sel] - got @ x
        assert np.max(np.abs(r)) <= 2 * tol * np.linalg.norm(b)
    finally:
        c.close()
