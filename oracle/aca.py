"""Adaptive cross approximation of one admissible block (oracle).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

The paper accelerates the far-field interactions with pFFT and names
hierarchical matrices as the alternative (Sec. 4.1); this library's operator
is an H-matrix whose admissible blocks are approximated by ACA with partial
pivoting (Bebendorf's method, written here from its definition):

* step k takes the residual row i_k, R_k(i_k, :) = A(i_k, :) - sum_{l<k}
  u_l(i_k) v_l; its largest entry j_k is the pivot, v_k = R_k(i_k, :) /
  R_k(i_k, j_k), u_k = R_k(:, j_k) (the residual column);
* the next row is the largest entry of u_k outside the rows used so far;
* it stops when |u_k| |v_k| <= eps ||S_k||_F, with ||S_k||_F^2 estimated by
  sum_{l<=k} |u_l|^2 |v_l|^2, or at the rank cap.

``check_rows``: partial pivoting follows the nonzero pattern of the rows and
columns it has visited. On a flat face the traction kernel couples the
normal-component rows only to the tangential columns and the tangential rows
only to the normal columns, so ACA can meet its stopping test on one of the
two parts without ever seeing the other. With ``check_rows``, when the test
holds, one residual row per displacement component (rows 3 e + a of the
element e = floor(a m_e / 3) + floor(m_e / 6), m_e the row elements) is
formed, and the first whose norm exceeds eps ||S_k||_F restarts the steps
from it. This is the rule the library uses.
"""
from __future__ import annotations

import numpy as np


def check_row(m_elems: int, a: int) -> int:
    """Row of the check for displacement component a (0, 1, 2)."""
    return 3 * ((a * m_elems) // 3 + m_elems // 6) + a


def aca(A, eps: float, rmax: int | None = None, check_rows: bool = False, start_row: int = 0):
    """ACA of the dense block A (m x n, rows and columns in element triples).

    Returns U (m x r), V (n x r) with A ~ U V^T, and the rank r.
    """
    A = np.asarray(A, dtype=np.complex128)
    m, n = A.shape
    rmax = min(m, n) if rmax is None else min(rmax, m, n)
    us, vs = [], []
    used = []
    norm2 = 0.0
    checks = 0
    i = start_row
    row = None
    while len(us) < rmax:
        if row is None:
            row = A[i].copy()
            for u, v in zip(us, vs):
                row -= u[i] * v
        j = int(np.argmax(np.abs(row)))
        stop = False
        if abs(row[j]) == 0.0:
            stop = True
        else:
            v = row / row[j]
            u = A[:, j].copy()
            for uu, vv in zip(us, vs):
                u -= uu * vv[j]
            us.append(u)
            vs.append(v)
            used.append(i)
            t = float(np.sum(np.abs(u) ** 2) * np.sum(np.abs(v) ** 2))
            norm2 += t
            if t <= eps * eps * norm2:
                stop = True
            else:
                cand = np.abs(u).copy()
                cand[used] = -1.0
                i = int(np.argmax(cand))
                if cand[i] <= 0.0:
                    stop = True
        row = None
        if not stop:
            continue
        if not check_rows:
            break
        again = False
        while checks < 3 and len(us) < rmax:
            c = check_row(m // 3, checks)
            checks += 1
            if c in used:
                continue
            r = A[c].copy()
            for u, v in zip(us, vs):
                r -= u[c] * v
            if np.sum(np.abs(r) ** 2) > eps * eps * norm2:
                i, row, again = c, r, True
                break
        if not again:
            break
    U = np.array(us).T if us else np.zeros((m, 0), dtype=np.complex128)
    V = np.array(vs).T if vs else np.zeros((n, 0), dtype=np.complex128)
    return U, V, len(us)
