"""Pins for the oracle's modified Fourier transform (Sec. 2.2, Sec. 3).

* DFT-MFT of the sampled step equals its geometric-series closed form;
* IDFT-MFT(DFT-MFT(P)) = P with W = 1 for any real history (conjugate
  symmetry, Sec. 2.2 step 3);
* window values at k = 0 and N/2 and their symmetry (Sec. 3.2);
* the damping rule (Eq. ewm-k);
* pushing the closed-form cavity response H(s_k) P_k through the IDFT-MFT
  reproduces the exact step response (by residues) at early times, and the
  Hanning window reduces the late-time Gibbs error (Sec. 3.2, Sec. 5.1).
"""
import math

import numpy as np
import pytest

from oracle import kernels, transforms
from paper_1212_3032_gb300 import inputs
from tests import analytic


def test_dft_of_step_closed_form():
    N, T = 64, 8.0
    eta = 5.0 / T
    P = inputs.heaviside_history(N)
    Pk = transforms.dft_mft(P, T, eta)
    dt = T / N
    for k in range(N // 2 + 1):
        q = np.exp(-eta * dt - 2j * math.pi * k / N)
        expect = (0.5 + q * (1 - q ** (N - 1)) / (1 - q)) / N
        assert Pk[k] == pytest.approx(expect, rel=1e-12, abs=1e-15)


@pytest.mark.parametrize("N", [16, 32, 128])
def test_idft_inverts_dft(N):
    rng = np.random.default_rng(N)
    T = 3.0
    eta = transforms.eta_from_kappa(4.0, T)
    P = rng.normal(size=N)
    Pk = transforms.dft_mft(P, T, eta)
    R = transforms.idft_mft(Pk, T, eta, transforms.WIN_NONE, N)
    assert np.allclose(R, P, rtol=0, atol=1e-10 * np.abs(P).max() * math.exp(eta * T))


def test_windows():
    N = 32
    for kind in (transforms.WIN_HANNING, transforms.WIN_BLACKMAN):
        W = transforms.window(kind, N)
        assert W[0] == pytest.approx(1.0)
        assert W[N // 2] == pytest.approx(0.0, abs=1e-15)
        assert np.allclose(W[1:], W[1:][::-1])         # W_k = W_{N-k}
        assert np.all(W >= -1e-15) and np.all(W <= 1 + 1e-15)
    assert np.all(transforms.window(transforms.WIN_NONE, N) == 1.0)
    assert transforms.window(transforms.WIN_HANNING, 4)[1] == pytest.approx(0.5)
    assert transforms.window(transforms.WIN_BLACKMAN, 4)[1] == pytest.approx(0.42 - 0.08)


def test_eta_rule_and_frequencies():
    T = 0.0155
    assert transforms.eta_from_kappa(4.0, T) == pytest.approx(4.0 * math.log(10) / T)
    s = transforms.sampling_frequencies(8.0, 32, 0.625)
    assert s.size == 17
    assert s[0] == 0.625 and s[3] == pytest.approx(0.625 + 3j * 2 * math.pi / 8.0)


def _cavity_trace(N, T, win, eta):
    mat = kernels.Material(1.0, 0.25, 1.0)
    s = transforms.sampling_frequencies(T, N, eta)
    Pk = transforms.dft_mft(inputs.heaviside_history(N), T, eta)
    H = analytic.cavity_wall_response(s, 1.0, mat.mu, mat.lam, mat.rho)
    R = transforms.idft_mft(H * Pk, T, eta, win, N)
    t = np.arange(N) * T / N
    exact = analytic.cavity_step_response(t, 1.0, mat.mu, mat.lam, mat.rho)
    return t, R, exact


def test_mft_reproduces_exact_step_response():
    N, T = 256, 8.0
    eta = 5.0 / T
    t, R, exact = _cavity_trace(N, T, transforms.WIN_NONE, eta)
    early = (t > 0.5) & (t < 0.5 * T)
    err = np.abs(R - exact)[early].max() / np.abs(exact).max()
    assert err < 0.05


def test_hanning_reduces_late_gibbs():
    N, T = 128, 8.0
    eta = transforms.eta_from_kappa(4.0, T)
    t, R0, exact = _cavity_trace(N, T, transforms.WIN_NONE, eta)
    _, R1, _ = _cavity_trace(N, T, transforms.WIN_HANNING, eta)
    # the last samples mix in the wrapped-around start of the period (the
    # window is a 3-tap circular filter in time), so stop short of T
    late = (t > 0.6 * T) & (t < 0.95 * T)
    e0 = np.abs(R0 - exact)[late].max()
    e1 = np.abs(R1 - exact)[late].max()
    assert e1 < 0.5 * e0
