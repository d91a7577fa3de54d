"""Modified Fourier transform: exponential window and frequency windows (oracle).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

Sec. 2.2 and Sec. 3:
  T = 2 pi / dw, dt = T / N                         (Sec. 2.2)
  eta = kappa ln(10) / T                            (Eq. ewm-k)
  s_k = eta + i k dw, k = 0..N/2                    (Sec. 3.1: omega_k = k dw - i eta, s = i omega)
  P_k = (1/N) sum_n e^{-eta n dt} P(n dt) e^{-2 pi i n k / N}         (Eq. DFT-MFT)
  R(n dt) = e^{eta n dt} sum_{k=0}^{N-1} W_k R_k e^{2 pi i n k / N}    (Eq. IDFT-MFT)
  R_k = conj(R_{N-k}) for k > N/2                   (Sec. 2.2, step 3)
  Hanning  W_k = 0.5 (1 + cos(2 pi k / N))          (Sec. 3.2)
  Blackman W_k = 0.42 + 0.5 cos(2 pi k / N) + 0.08 cos(4 pi k / N)

Reading for the unpaired terms: the solved responses are complex at every k
(the sampling frequencies are complex), so the k = 0 and k = N/2 samples are
taken by their real parts, which is what conjugate symmetry of a real signal
requires; every other k pairs with N - k.
"""
from __future__ import annotations

import math

import numpy as np

WIN_NONE, WIN_HANNING, WIN_BLACKMAN = 0, 1, 2


def eta_from_kappa(kappa: float, T: float) -> float:
    """Damping parameter of the exponential window (Eq. ewm-k)."""
    return kappa * math.log(10.0) / T


def sampling_frequencies(T: float, n_omega: int, eta: float):
    """s_k = eta + i k dw for k = 0..n_omega/2."""
    dw = 2.0 * math.pi / T
    k = np.arange(n_omega // 2 + 1)
    return eta + 1j * k * dw


def window(kind: int, n_omega: int):
    """W(omega_k) for k = 0..n_omega-1 (Sec. 3.2)."""
    k = np.arange(n_omega)
    if kind == WIN_NONE:
        return np.ones(n_omega)
    if kind == WIN_HANNING:
        return 0.5 * (1.0 + np.cos(2 * math.pi * k / n_omega))
    if kind == WIN_BLACKMAN:
        return 0.42 + 0.5 * np.cos(2 * math.pi * k / n_omega) + 0.08 * np.cos(4 * math.pi * k / n_omega)
    raise ValueError(f"unknown window {kind}")


def dft_mft(P, T: float, eta: float):
    """Eq. DFT-MFT for k = 0..N/2 from samples P(n dt), n = 0..N-1."""
    P = np.asarray(P, dtype=np.float64)
    N = P.size
    dt = T / N
    n = np.arange(N)
    out = np.zeros(N // 2 + 1, dtype=np.complex128)
    for k in range(N // 2 + 1):
        out[k] = np.sum(np.exp(-eta * n * dt) * P * np.exp(-2j * math.pi * n * k / N)) / N
    return out


def idft_mft(Rk, T: float, eta: float, win: int, n_omega: int):
    """Eq. IDFT-MFT: time samples R(n dt), n = 0..N-1, from R_k, k = 0..N/2.

    Rk: (N/2+1, ...) complex. The spectrum is extended to k = 0..N-1 by
    conjugate symmetry before the sum; the k = 0 and k = N/2 samples enter
    through their real parts.
    """
    Rk = np.asarray(Rk, dtype=np.complex128)
    N = n_omega
    if Rk.shape[0] != N // 2 + 1:
        raise ValueError("expected N/2+1 spectral samples")
    full = np.zeros((N,) + Rk.shape[1:], dtype=np.complex128)
    full[0] = Rk[0].real
    full[1:N // 2] = Rk[1:N // 2]
    full[N // 2] = Rk[N // 2].real
    for k in range(N // 2 + 1, N):
        full[k] = np.conj(Rk[N - k])
    W = window(win, N)
    dt = T / N
    out = np.zeros((N,) + Rk.shape[1:], dtype=np.float64)
    k = np.arange(N)
    for n in range(N):
        ph = np.exp(2j * math.pi * n * k / N)
        acc = np.tensordot(W * ph, full, axes=(0, 0))
        out[n] = math.exp(eta * n * dt) * acc.real
    return out
