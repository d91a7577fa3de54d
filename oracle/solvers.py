"""Linear solves for one frequency system, and solution extrapolation (oracle).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

* ``direct_solve``: the exact discrete solution of A a = b (Eq. Aa_b) by LU.
* ``gmres``: restarted GMRES (Saad & Schultz, the solver named in Sec. 5) with
  the block-diagonal preconditioner of Sec. 3.1 / Sec. 5, applied on the
  right. Block = the 3x3 diagonal block of A belonging to one element (the
  paper does not state the block size). Stops on the true relative residual
  ||b - A a|| / ||b|| <= tol.
* ``sem_guess``: solution extrapolation method (Sec. 4.2, Eqs. a0, lsem,
  a0-solution): a0 = X s with s minimising ||A X s - b||_2 through the QR
  factorisation Y = A X = Q R, s = R^{-1} Q^H b (the printed Q is read as its
  conjugate transpose, the least-squares solution). Columns of X that make R
  numerically rank deficient are dropped.
"""
from __future__ import annotations

import numpy as np


def direct_solve(A, b):
    return np.linalg.solve(np.asarray(A, dtype=np.complex128), np.asarray(b, dtype=np.complex128))


def block_jacobi_inverse(A):
    """Inverses of the 3x3 diagonal blocks of A: (Ne, 3, 3)."""
    n = A.shape[0] // 3
    blocks = np.stack([A[3 * e:3 * e + 3, 3 * e:3 * e + 3] for e in range(n)])
    return np.linalg.inv(blocks)


def _apply_block(Minv, v):
    return np.einsum("eij,ej->ei", Minv, v.reshape(-1, 3)).reshape(-1)


def bisection_clusters(centroids, leaf: int):
    """Element groups of at most ``leaf`` elements: recursive halving at the
    median along the longest extent of the group's centroids."""
    c = np.asarray(centroids, dtype=np.float64)
    todo, out = [np.arange(c.shape[0])], []
    while todo:
        I = todo.pop()
        if I.size <= leaf:
            out.append(I)
            continue
        ax = int(np.argmax(c[I].max(axis=0) - c[I].min(axis=0)))
        o = np.argsort(c[I, ax], kind="stable")
        h = I.size // 2
        todo += [I[o[:h]], I[o[h:]]]
    return out


def cluster_block_inverse(A, groups):
    """Inverses of the diagonal blocks of A over element groups (3 rows and
    columns per element): a block-Jacobi preconditioner with larger blocks."""
    out = []
    for I in groups:
        d = (3 * np.asarray(I)[:, None] + np.arange(3)).ravel()
        out.append((d, np.linalg.inv(A[np.ix_(d, d)])))
    return out


def _apply_groups(inv, v):
    o = np.empty_like(v)
    for d, Bi in inv:
        o[d] = Bi @ v[d]
    return o


def gmres(A, b, x0=None, tol=1e-10, restart=50, maxiter=5000, precondition=True, groups=None):
    """Right-preconditioned restarted GMRES; returns (x, iterations, rel_residual).

    The preconditioner is the inverse of the 3x3 diagonal blocks, or of the
    diagonal blocks over element ``groups`` when given."""
    A = np.asarray(A, dtype=np.complex128)
    b = np.asarray(b, dtype=np.complex128)
    N = b.size
    if precondition and groups is not None:
        ginv = cluster_block_inverse(A, groups)
        M = lambda v: _apply_groups(ginv, v)
    elif precondition:
        Minv = block_jacobi_inverse(A)
        M = lambda v: _apply_block(Minv, v)
    else:
        M = lambda v: v
    x = np.zeros(N, dtype=np.complex128) if x0 is None else np.asarray(x0, dtype=np.complex128).copy()
    bnorm = np.linalg.norm(b)
    if bnorm == 0.0:
        return np.zeros(N, dtype=np.complex128), 0, 0.0
    its = 0
    r = b - A @ x
    rel = np.linalg.norm(r) / bnorm
    while rel > tol and its < maxiter:
        beta = np.linalg.norm(r)
        V = np.zeros((restart + 1, N), dtype=np.complex128)
        H = np.zeros((restart + 1, restart), dtype=np.complex128)
        cs = np.zeros(restart, dtype=np.complex128)
        sn = np.zeros(restart, dtype=np.complex128)
        g = np.zeros(restart + 1, dtype=np.complex128)
        g[0] = beta
        V[0] = r / beta
        j_done = 0
        for j in range(restart):
            w = A @ M(V[j])
            for _ in range(2):                     # classical Gram-Schmidt, twice
                h = V[:j + 1].conj() @ w
                w = w - V[:j + 1].T @ h
                H[:j + 1, j] += h
            H[j + 1, j] = np.linalg.norm(w)
            if H[j + 1, j] != 0:
                V[j + 1] = w / H[j + 1, j]
            for i in range(j):                     # apply previous rotations
                # G_i = [[conj(c), conj(s)], [-s, c]] (unitary)
                t = np.conj(cs[i]) * H[i, j] + np.conj(sn[i]) * H[i + 1, j]
                H[i + 1, j] = -sn[i] * H[i, j] + cs[i] * H[i + 1, j]
                H[i, j] = t
            a, c = H[j, j], H[j + 1, j]
            den = np.sqrt(abs(a) ** 2 + abs(c) ** 2)
            cs[j] = a / den if den else 1.0
            sn[j] = c / den if den else 0.0
            H[j, j] = den
            H[j + 1, j] = 0
            g[j + 1] = -sn[j] * g[j]
            g[j] = np.conj(cs[j]) * g[j]
            its += 1
            j_done = j + 1
            if abs(g[j + 1]) / bnorm <= tol or its >= maxiter:
                break
        y = np.linalg.solve(np.triu(H[:j_done, :j_done]), g[:j_done])
        x = x + M(V[:j_done].T @ y)
        r = b - A @ x
        rel = np.linalg.norm(r) / bnorm
    return x, its, rel


def sem_guess(A, b, X, drop_tol=1e-12):
    """Solution extrapolation (Sec. 4.2): a0 = X R^{-1} Q^H b with A X = Q R.

    X: (N, K) previous solutions (a_{k-1}, ..., a_{k-K}); K may be 0.
    Returns (a0, s) with s the coefficients of the kept columns.
    """
    X = np.asarray(X, dtype=np.complex128)
    N = b.size
    if X.ndim != 2 or X.shape[1] == 0:
        return np.zeros(N, dtype=np.complex128), np.zeros(0, dtype=np.complex128)
    Y = A @ X
    keep = []
    for j in range(X.shape[1]):
        cand = keep + [j]
        _, R = np.linalg.qr(Y[:, cand])
        d = np.abs(np.diag(R))
        if d[-1] > drop_tol * d[0]:
            keep = cand
    Q, R = np.linalg.qr(Y[:, keep])
    s = np.linalg.solve(R, Q.conj().T @ b)
    return X[:, keep] @ s, s
