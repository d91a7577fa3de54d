"""The frequency sweep and the time response (oracle).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

Sec. 2.2 procedure with the MFT substitutions of Sec. 3.3:
  1. sample the prescribed history P(n dt) and transform it (Eq. DFT-MFT);
  2. for k = 0..N/2 solve A_k a_k = b_k (Eq. Aa_b-sequence) at s_k = eta + i k dw,
     with b_k built from the prescribed pattern times P_k;
  3. transform the responses back with the window (Eq. IDFT-MFT).
"""
from __future__ import annotations

import numpy as np

from . import bem, kernels, solvers, transforms


def solve_sweep(mesh, mat: kernels.Material, T: float, n_omega: int, eta: float,
                load_hist, method: str = "direct", tol: float = 1e-12, guess: str = "zero",
                K: int = 4, restart: int = 50, ks=None):
    """Solve every frequency system; returns dict with s, Pk, a (Nf, N), its, res.

    method: "direct" (LU) or "gmres". guess (gmres only): "zero" or "sem".
    ks: optional subset of frequency indices (default all k = 0..N/2).
    """
    g = bem.geometry(mesh.xyz, mesh.tri)
    s_all = transforms.sampling_frequencies(T, n_omega, eta)
    Pk_all = transforms.dft_mft(load_hist, T, eta)
    ks = np.arange(s_all.size) if ks is None else np.asarray(ks)
    N = 3 * g.ne
    sol = np.zeros((ks.size, N), dtype=np.complex128)
    its = np.zeros(ks.size, dtype=np.int64)
    res = np.zeros(ks.size)
    guess_res = np.zeros(ks.size)
    for m, k in enumerate(ks):
        known = mesh.pattern * Pk_all[k]
        A, b = bem.system_rows(g, mesh.bc_type, known, s_all[k], mat)
        if method == "direct":
            a = solvers.direct_solve(A, b)
            its[m] = 0
        else:
            x0 = None
            if guess == "sem" and m > 0:
                X = sol[max(0, m - K):m][::-1].T
                x0, _ = solvers.sem_guess(A, b, X)
            if x0 is not None:
                guess_res[m] = np.linalg.norm(b - A @ x0) / np.linalg.norm(b)
            else:
                guess_res[m] = 1.0
            a, its[m], _ = solvers.gmres(A, b, x0=x0, tol=tol, restart=restart)
        sol[m] = a
        res[m] = np.linalg.norm(b - A @ a) / max(np.linalg.norm(b), 1e-300)
    return dict(s=s_all[ks], Pk=Pk_all[ks], k=ks, a=sol, its=its, res=res, guess_res=guess_res)


def time_response(a_k, T: float, eta: float, win: int, n_omega: int, dofs=None):
    """R(n dt) at the requested dofs from the solved spectrum a_k (Nf, N)."""
    a_k = np.asarray(a_k)
    if dofs is not None:
        a_k = a_k[:, np.asarray(dofs)]
    return transforms.idft_mft(a_k, T, eta, win, n_omega)
