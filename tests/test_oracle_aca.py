"""ACA with partial pivoting (oracle/aca.py) and the check-row rule.

* A matrix of exact low rank is recovered to rounding.
* On a generic block (two distant patches of a sphere) ACA meets its
  tolerance, and the check rows change nothing.
* On a coplanar block (two patches of one flat box face) plain partial
  pivoting converges on one of the two nonzero parts of the traction kernel
  (normal rows x tangential columns, tangential rows x normal columns) and
  misses the other; with one check row per displacement component it meets
  the tolerance.
"""
import numpy as np
import pytest

from oracle import aca, bem, kernels
from paper_1212_3032_gb300 import inputs

MAT = kernels.Material(1.0, 0.25, 1.0)
S = 0.5 + 3.0j


def _rel(A, U, V):
    return np.linalg.norm(A - U @ V.T) / np.linalg.norm(A)


def _block(mesh, sel_r, sel_c):
    g = bem.geometry(mesh.xyz, mesh.tri)
    r = np.flatnonzero(sel_r(g.c))
    c = np.flatnonzero(sel_c(g.c))
    A, _ = bem.system_rows(g, mesh.bc_type, np.zeros((mesh.ne, 3)), S, MAT, rows=r)
    return A[:, (3 * c[:, None] + np.arange(3)).ravel()]


def test_exact_low_rank():
    rng = np.random.default_rng(3)
    X = rng.normal(size=(60, 4)) + 1j * rng.normal(size=(60, 4))
    Y = rng.normal(size=(90, 4)) + 1j * rng.normal(size=(90, 4))
    A = X @ Y.T
    for chk in (False, True):
        U, V, r = aca.aca(A, 1e-10, check_rows=chk)
        assert r <= 5 and _rel(A, U, V) <= 1e-12


def test_check_row_rule():
    for m in (1, 2, 7, 64):
        rows = [aca.check_row(m, a) for a in range(3)]
        assert all(0 <= r < 3 * m for r in rows)
        assert [r % 3 for r in rows] == [0, 1, 2]


def test_generic_block_unchanged_by_check_rows():
    mesh = inputs.cavity_problem(8)
    A = _block(mesh, lambda c: c[:, 0] > 0.6, lambda c: c[:, 0] < -0.6)
    U0, V0, r0 = aca.aca(A, 1e-5)
    U1, V1, r1 = aca.aca(A, 1e-5, check_rows=True)
    assert _rel(A, U0, V0) <= 30e-5 and r1 == r0
    assert np.array_equal(U0, U1)


def test_coplanar_block_needs_check_rows():
    xyz, tri = inputs.box_mesh(1.0, 1.0, 1.0, 1.0 / 12)
    mesh = inputs.pressurised_surface(xyz, tri)
    top = lambda c: np.abs(c[:, 2] - 0.5) < 1e-9
    A = _block(mesh, lambda c: top(c) & (c[:, 0] < -0.25), lambda c: top(c) & (c[:, 0] > 0.25))
    # the block's structure: normal (z) rows vanish on the normal columns and
    # the tangential rows vanish on the tangential columns
    assert np.max(np.abs(A[2::3, 2::3])) <= 1e-12 * np.max(np.abs(A))
    assert np.max(np.abs(A[0::3, 0::3])) <= 1e-12 * np.max(np.abs(A))
    U0, V0, _ = aca.aca(A, 1e-5)
    assert _rel(A, U0, V0) >= 0.3
    U1, V1, _ = aca.aca(A, 1e-5, check_rows=True)
    assert _rel(A, U1, V1) <= 30e-5
