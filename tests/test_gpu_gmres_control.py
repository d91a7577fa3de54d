"""GMRES driven by the device (Sec. 3.1: right preconditioning; Sec. 5:
GMRES to a relative residual): the Givens rotations, the convergence test
and the update that closes a restart cycle run in kernels, and the host only
reads the solver state a few steps later. Pinned against the oracle's GMRES
(``oracle.solvers.gmres``) on the same FP64 operator (the dense 320-element
cavity, whose rows match the oracle's to 1e-8):

* restart lengths 1 and 2 (shorter than the host's read-back lag, so the host
  checks the state before a step is that far behind), 5 and 50: the solution
  matches the LU solution and the step count the oracle's within one step
  (the device ends a cycle at 0.9 tol, the oracle at tol);
* the step limit: with restart 2 and 5 steps (cycles of 2, 2 and 1 steps) the
  iterate equals the oracle's after the same 5 steps, not converged;
* a zero right-hand side gives x = 0 without a step.
"""
import math

import numpy as np
import pytest

from oracle import bem, kernels, solvers
from paper_1212_3032_gb300 import inputs

pytestmark = pytest.mark.gpu

MAT = kernels.Material(1.0, 0.25, 1.0)
S = 0.625 + 2.0j


@pytest.fixture(scope="module")
def B():
    from paper_1212_3032_gb300 import binding, build
    build.build()
    return binding


@pytest.fixture(scope="module")
def case(B):
    mesh = inputs.cavity_problem(4)                       # 320 elements
    g = bem.geometry(mesh.xyz, mesh.tri)
    A, b = bem.system_rows(g, mesh.bc_type, mesh.pattern.astype(complex), S, MAT)
    c = B.Context(0)
    c.set_material(MAT.E, MAT.nu, MAT.rho)
    o = B.default_opts(dense=1, precision=1)
    c.mesh(mesh.xyz, mesh.tri, mesh.bc_type, o)
    c.assemble(S, o)
    bg = c.rhs(1.0, mesh.pattern)
    yield c, A, b, bg
    c.close()


def _rel(a, b):
    return np.linalg.norm(np.asarray(a) - np.asarray(b)) / max(np.linalg.norm(b), 1e-300)


@pytest.mark.parametrize("restart", [1, 2, 5, 50])
def test_restart_lengths_match_oracle(B, case, restart):
    c, A, b, bg = case
    tol = 1e-10
    x_ref = solvers.direct_solve(A, b)
    _, its_ref, _ = solvers.gmres(A, b, tol=tol, restart=restart)
    o = B.default_opts(dense=1, precision=1, tol=tol, restart=restart, max_iters=400)
    x, st = c.solve_assembled(bg, opts=o)
    assert st["converged"] == 1 and st["rel_residual"] <= tol
    assert _rel(x, x_ref) <= 1e-8
    assert abs(st["iters"] - its_ref) <= 1, (st["iters"], its_ref)
    assert st["cycles"] >= math.ceil(st["iters"] / restart)
    if restart == 1:
        assert st["cycles"] == st["iters"]


def test_step_limit_iterate_matches_oracle(B, case):
    c, A, b, bg = case
    x_ref, its_ref, rel_ref = solvers.gmres(A, b, tol=1e-14, restart=2, maxiter=5)
    assert its_ref == 5 and rel_ref > 1e-8
    o = B.default_opts(dense=1, precision=1, tol=1e-14, restart=2, max_iters=5)
    x, st = c.solve_assembled(bg, opts=o, allow_unconverged=True)
    assert st["converged"] == 0 and st["iters"] == 5 and st["cycles"] == 3
    assert _rel(x, x_ref) <= 1e-7
    assert abs(st["rel_residual"] - rel_ref) <= 1e-3 * rel_ref


def test_zero_right_hand_side(B, case):
    c, A, b, bg = case
    o = B.default_opts(dense=1, precision=1, tol=1e-10)
    x0 = np.full(bg.shape, 1.0 + 2.0j)
    x, st = c.solve_assembled(np.zeros_like(bg), x0=x0, opts=o)
    assert st["converged"] == 1 and st["iters"] == 0 and st["cycles"] == 0
    assert np.all(x == 0)
