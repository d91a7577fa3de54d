"""Dense collocation rows over several processes (oracle).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

The rows of A and b (Eq. Aa_b) are independent of one another: row block i
is the collocation of the boundary integral equation (Eq. bie) at the centroid
of element i. This module only splits the row indices into contiguous slices, lets
``bem.system_rows`` compute each slice in a worker process and stacks the
slices in order; it adds no arithmetic. The direct solve (LU) then runs in
the calling process. The workers are started with the ``spawn`` method, so a
pool may be created after the process has used a GPU.
"""
from __future__ import annotations

import multiprocessing as mp
import os

import numpy as np

from . import bem, kernels, solvers, transforms


def _worker(conn, xyz, tri, bc_type, mat_args):
    """Computes the requested rows until told to stop (None)."""
    g = bem.geometry(xyz, tri)
    bc = np.asarray(bc_type)
    mat = kernels.Material(*mat_args)
    while True:
        msg = conn.recv()
        if msg is None:
            break
        known, s, rows = msg
        conn.send(bem.system_rows(g, bc, known, s, mat, rows=rows))
    conn.close()


class RowPool:
    """Worker processes computing rows of one mesh's system.

    Worker w always receives the w-th of ``workers`` contiguous slices of the
    requested rows, so that its cache of frequency-independent static parts
    serves it again at the next frequency of a sweep.
    """

    def __init__(self, mesh, mat: kernels.Material, workers: int | None = None):
        self.mesh = mesh
        self.ne = int(mesh.ne)
        self.workers = max(1, min(int(workers or os.cpu_count() or 1), self.ne))
        ctx = mp.get_context("spawn")
        # one BLAS thread per worker; the parent keeps its own setting
        saved = {k: os.environ.get(k) for k in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS")}
        for k in saved:
            os.environ[k] = "1"
        self._conns, self._procs = [], []
        try:
            for _ in range(self.workers):
                a, b = ctx.Pipe()
                p = ctx.Process(target=_worker, args=(b, mesh.xyz, mesh.tri, mesh.bc_type,
                                                      (mat.E, mat.nu, mat.rho)), daemon=True)
                p.start()
                b.close()
                self._conns.append(a)
                self._procs.append(p)
        finally:
            for k, v in saved.items():
                if v is None:
                    os.environ.pop(k, None)
                else:
                    os.environ[k] = v

    def rows(self, known, s, rows=None):
        """A[rows-blocks], b[rows-blocks] as ``bem.system_rows`` returns them."""
        rows = np.arange(self.ne) if rows is None else np.asarray(rows, dtype=np.int64)
        if rows.size == 0:
            return np.zeros((0, 3 * self.ne), dtype=np.complex128), np.zeros(0, dtype=np.complex128)
        known = np.asarray(known, dtype=np.complex128)
        chunks = np.array_split(rows, self.workers)
        busy = []
        for conn, c in zip(self._conns, chunks):
            if c.size:
                conn.send((known, complex(s), c))
                busy.append(conn)
        parts = [conn.recv() for conn in busy]
        return np.concatenate([p[0] for p in parts]), np.concatenate([p[1] for p in parts])

    def close(self):
        for conn in self._conns:
            try:
                conn.send(None)
                conn.close()
            except (OSError, BrokenPipeError):
                pass
        for p in self._procs:
            p.join(timeout=30)
            if p.is_alive():
                p.terminate()
        self._conns, self._procs = [], []

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()


def solve_sweep(pool: RowPool, T: float, n_omega: int, eta: float, load_hist, ks=None):
    """``sweep.solve_sweep`` with method "direct", rows from the pool.

    Returns dict with s, Pk, k, a (len(ks), N) and res (true relative residuals).
    """
    s_all = transforms.sampling_frequencies(T, n_omega, eta)
    Pk_all = transforms.dft_mft(load_hist, T, eta)
    ks = np.arange(s_all.size) if ks is None else np.asarray(ks)
    N = 3 * pool.ne
    sol = np.zeros((ks.size, N), dtype=np.complex128)
    res = np.zeros(ks.size)
    for m, k in enumerate(ks):
        A, b = pool.rows(pool.mesh.pattern * Pk_all[k], s_all[k])
        a = solvers.direct_solve(A, b)
        sol[m] = a
        res[m] = np.linalg.norm(b - A @ a) / max(np.linalg.norm(b), 1e-300)
    return dict(s=s_all[ks], Pk=Pk_all[ks], k=ks, a=sol, res=res)
