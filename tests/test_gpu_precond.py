"""The leaf-block preconditioner (Sec. 3.1 / Sec. 5: block diagonal, block size
unstated) against the oracle, through the C-ABI.

* M^-1 x with the leaves' diagonal blocks against ``oracle.solvers``'
  cluster_block_inverse over the same element groups (the GPU tree's
  leaves), the oracle's blocks taken from its own dense rows: FP32
  Gauss-Jordan on complex64 blocks (condition numbers ~1e2: 1e-4), FP64 on
  complex128 blocks (1e-9);
* M^-1 x with the 3 x 3 blocks against the oracle's block_jacobi_inverse;
* on the mixed-boundary rod the leaf blocks take far fewer GMRES steps than
  the 3 x 3 blocks (the oracle: 30 against 72 at omega = 4.71) and reach the
  same solution as the oracle's LU;
* BEM_PRECOND_AUTO keeps the leaf blocks on the rod.
"""
import numpy as np
import pytest

from oracle import bem, kernels, pool, solvers
from paper_1212_3032_gb300 import inputs

pytestmark = pytest.mark.gpu

ROD_MAT = kernels.Material(1.0, 0.0, 1.0)


@pytest.fixture(scope="module")
def B():
    from paper_1212_3032_gb300 import binding, build
    build.build()
    return binding


def _rel(a, b):
    return np.linalg.norm(np.asarray(a) - np.asarray(b)) / max(np.linalg.norm(b), 1e-300)


def _leaf_groups(B, mesh, leaf):
    g = bem.geometry(mesh.xyz, mesh.tri)
    perm, near, _ = B.block_tree(g.c, g.h, leaf_size=leaf)
    return [perm[r0:r0 + nr] for r0, nr, c0, nc in near if r0 == c0 and nr == nc]


@pytest.mark.parametrize("prec,tol", [(0, 1e-4), (1, 1e-9)])
def test_leaf_inverse_matches_oracle(B, prec, tol):
    rod = inputs.rod_problem(h=1 / 6)                      # 1,008 triangles, leaves of 33-63 elements
    s = 0.3 + 4.71j
    groups = _leaf_groups(B, rod, 64)
    assert len(groups) > 10 and sum(len(q) for q in groups) == rod.ne
    with pool.RowPool(rod, ROD_MAT) as P:
        A_ref, _ = P.rows(np.zeros((rod.ne, 3)), s)
    inv_ref = solvers.cluster_block_inverse(A_ref, groups)
    b3_ref = solvers.block_jacobi_inverse(A_ref)
    rng = np.random.default_rng(5)
    with B.Context(0) as ctx:
        ctx.set_material(ROD_MAT.E, ROD_MAT.nu, ROD_MAT.rho)
        o = B.default_opts(dense=0, leaf_size=64, precision=prec, precond=B.PRECOND_LEAF,
                           aca_tol=1e-5 if prec == 0 else 1e-8)
        ctx.mesh(rod.xyz, rod.tri, rod.bc_type, o)
        ctx.assemble(s, o)
        for _ in range(2):
            x = rng.normal(size=3 * rod.ne) + 1j * rng.normal(size=3 * rod.ne)
            y = ctx.apply_preconditioner(x, B.PRECOND_LEAF)
            y_ref = np.empty_like(x)
            for d, Bi in inv_ref:
                y_ref[d] = Bi @ x[d]
            assert _rel(y, y_ref) <= tol
            y3 = ctx.apply_preconditioner(x, B.PRECOND_BLOCK3)
            y3_ref = np.einsum("eij,ej->ei", b3_ref, x.reshape(-1, 3)).ravel()
            assert _rel(y3, y3_ref) <= (2e-5 if prec == 0 else 1e-9)
        # without leaf inverses assembled, asking for them is refused
        o3 = B.default_opts(dense=0, leaf_size=64, precision=prec)
        ctx.assemble(s, o3)
        with pytest.raises(B.BemError):
            ctx.apply_preconditioner(x, B.PRECOND_LEAF)


def test_leaf_preconditioner_on_the_rod(B):
    rod = inputs.rod_problem(h=1 / 8)                      # 1,792 triangles
    s = 0.3 + 4.71j
    with pool.RowPool(rod, ROD_MAT) as P:
        A_ref, b_ref = P.rows(rod.pattern.astype(complex), s)
    x_ref = solvers.direct_solve(A_ref, b_ref)
    its = {}
    with B.Context(0) as ctx:
        ctx.set_material(ROD_MAT.E, ROD_MAT.nu, ROD_MAT.rho)
        for pc in (B.PRECOND_BLOCK3, B.PRECOND_LEAF):
            o = B.default_opts(dense=0, leaf_size=64, precision=0, aca_tol=1e-6, tol=1e-6, precond=pc)
            ctx.mesh(rod.xyz, rod.tri, rod.bc_type, o)
            ctx.assemble(s, o)
            b = ctx.rhs(1.0, rod.pattern)
            x, st = ctx.solve_assembled(b, opts=o)
            assert st["converged"] == 1 and st["precond"] == pc
            assert _rel(x, x_ref) <= 1e-4, pc
            its[pc] = st["iters"]
    print(f"rod 1792 at s = {s}: GMRES steps 3x3 {its[B.PRECOND_BLOCK3]}, leaf {its[B.PRECOND_LEAF]}")
    assert its[B.PRECOND_LEAF] < 0.6 * its[B.PRECOND_BLOCK3]


def test_auto_preconditioner_keeps_leaf_blocks_on_the_rod(B):
    rod = inputs.rod_problem(h=1 / 8)
    T, N = 26.8 * 3.0, 32
    with B.Context(0) as ctx:
        ctx.set_material(ROD_MAT.E, ROD_MAT.nu, ROD_MAT.rho)
        ctx.set_window(4 * np.log(10) / T, B.WIN_HANNING)
        o = B.default_opts(dense=0, leaf_size=64, precision=0, precond=B.PRECOND_AUTO)
        ctx.mesh(rod.xyz, rod.tri, rod.bc_type, o)
        st = ctx.solve_sweep(T, N, inputs.heaviside_history(N), rod.pattern, o)
        assert all(s["converged"] == 1 for s in st)
        assert st[1]["trial_iters"] > 0 and all(s["trial_iters"] == 0 for s in st[2:])
        assert all(s["precond"] == B.PRECOND_LEAF for s in st[1:])
        # the trial solve is counted in the iterations of its frequency
        assert st[1]["iters"] > st[1]["trial_iters"]
