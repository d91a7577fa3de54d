"""The process pool of the oracle returns exactly the serial oracle's rows,
in order, for full systems, row subsets and a sweep (it adds no arithmetic)."""
import numpy as np

from oracle import bem, kernels, pool, sweep as osweep
from paper_1212_3032_gb300 import inputs

MAT = kernels.Material(1.0, 0.25, 1.0)


def test_pool_rows_equal_serial_rows():
    mesh = inputs.cube_with_cavities(n_face=3, n_cav=1, cav_radius=0.12, cav_n=2, seed=5)
    g = bem.geometry(mesh.xyz, mesh.tri)
    known = mesh.pattern * (0.3 - 0.2j)
    s = 0.7 + 2.5j
    with pool.RowPool(mesh, MAT, workers=3) as P:
        A, b = P.rows(known, s)
        A_ref, b_ref = bem.system_rows(g, mesh.bc_type, known, s, MAT)
        assert np.array_equal(A, A_ref) and np.array_equal(b, b_ref)
        rows = np.array([mesh.ne - 1, 0, 7])
        A2, b2 = P.rows(known, s, rows=rows)
        A2_ref, b2_ref = bem.system_rows(g, mesh.bc_type, known, s, MAT, rows=rows)
        assert np.array_equal(A2, A2_ref) and np.array_equal(b2, b2_ref)
        A0, b0 = P.rows(known, s, rows=np.zeros(0, dtype=np.int64))
        assert A0.shape == (0, 3 * mesh.ne) and b0.shape == (0,)


def test_pool_sweep_equals_serial_sweep():
    mesh = inputs.cavity_problem(2)
    T, N = 8.0, 8
    load = inputs.heaviside_history(N)
    ref = osweep.solve_sweep(mesh, MAT, T, N, 5.0 / T, load)
    with pool.RowPool(mesh, MAT, workers=2) as P:
        got = pool.solve_sweep(P, T, N, 5.0 / T, load)
    assert np.allclose(got["a"], ref["a"], rtol=0, atol=1e-12 * np.abs(ref["a"]).max())
    assert got["res"].max() <= 1e-12
