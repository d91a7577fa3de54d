"""Pins for the oracle's fundamental solutions (Sec. 2.1, Eqs. Uij, Tij, Gikj).

Each check is independent of the formula it tests:
* U must solve the Laplace-domain Navier equation away from the source
  (finite differences of U only);
* T must equal the traction of U's displacement field by Hooke's law
  (finite differences of U only; pins reading 3, the sign of r_i);
* U, T must reach the static Kelvin kernels (textbook closed forms) as
  s -> 0 (pins reading 2, the (c_s/c_p)^2 factor), with the first-order
  correction obtained from the exponential series;
* symmetries: U_ij = U_ji, U(x,y) = U(y,x), U(conj s) = conj U(s).
"""
import math

import numpy as np
import pytest

from oracle import kernels

MATS = [kernels.Material(1.0, 0.25, 1.0), kernels.Material(69e9, 0.3, 2.7e3),
        kernels.Material(2.0, 0.0, 1.5)]


def _rand_pair(rng, scale=1.0):
    x = rng.normal(size=3) * scale
    y = x + rng.normal(size=3) * scale
    n = rng.normal(size=3)
    return x, y, n / np.linalg.norm(n)


@pytest.mark.parametrize("mat", MATS[:1] + MATS[2:])
@pytest.mark.parametrize("s", [0.6, 0.6 + 2.5j, 1.3 + 7.0j])
def test_U_solves_navier(mat, s):
    """mu Lap U + (lam+mu) grad div U = rho s^2 U (Laplace-domain Navier)."""
    rng = np.random.default_rng(1)
    x, y, _ = _rand_pair(rng)
    h = 5e-4
    lam, mu, rho = mat.lam, mat.mu, mat.rho

    def Ui(yy):
        return kernels.displacement_kernel(x, yy, s, mat)  # row i = force dir

    # fourth-order central second derivatives d2 U / dy_a dy_b
    def d2(a, b):
        ea = np.eye(3)[a] * h
        eb = np.eye(3)[b] * h
        if a == b:
            return (-Ui(y + 2 * ea) + 16 * Ui(y + ea) - 30 * Ui(y) + 16 * Ui(y - ea) - Ui(y - 2 * ea)) / (12 * h * h)
        return (Ui(y + ea + eb) - Ui(y + ea - eb) - Ui(y - ea + eb) + Ui(y - ea - eb)) / (4 * h * h)

    H = {(a, b): d2(a, b) for a in range(3) for b in range(3)}
    U0 = Ui(y)
    for i in range(3):
        lap = sum(H[(a, a)][i] for a in range(3))                     # vector over j
        graddiv = np.array([sum(H[(j, l)][i, l] for l in range(3)) for j in range(3)])
        res = mu * lap + (lam + mu) * graddiv - rho * s * s * U0[i]
        scale = mu * np.abs(lap).max() + abs(rho * s * s) * np.abs(U0[i]).max()
        assert np.abs(res).max() <= 1e-5 * scale


@pytest.mark.parametrize("mat", MATS)
@pytest.mark.parametrize("s", [0.6, 0.6 + 2.5j, 2.0 + 9.0j])
def test_T_is_hooke_traction_of_U(mat, s):
    """T_ij(x,y;n) = sigma^(i)_jk(y) n_k with sigma from U_i. by Hooke's law."""
    rng = np.random.default_rng(2)
    cs = mat.cs
    s_phys = s * cs  # keep |s r / c| of order one for every material
    for _ in range(4):
        x, y, n = _rand_pair(rng)
        h = 1e-5
        dU = np.zeros((3, 3, 3), dtype=complex)
        for l in range(3):
            e = np.eye(3)[l] * h
            dU[:, :, l] = (kernels.displacement_kernel(x, y + e, s_phys, mat)
                           - kernels.displacement_kernel(x, y - e, s_phys, mat)) / (2 * h)
        Tref = np.zeros((3, 3), dtype=complex)
        for i in range(3):
            div = np.trace(dU[i])
            sig = mat.lam * div * np.eye(3) + mat.mu * (dU[i] + dU[i].T)
            Tref[i] = sig @ n
        T = kernels.traction_kernel(x, y, n, s_phys, mat)
        assert np.abs(T - Tref).max() <= 1e-6 * np.abs(Tref).max()
        U2, T2 = kernels.kernel_pair(x, y, n, s_phys, mat)
        assert np.allclose(T2, T, rtol=1e-13, atol=0)
        assert np.allclose(U2, kernels.displacement_kernel(x, y, s_phys, mat), rtol=1e-13, atol=0)


@pytest.mark.parametrize("mat", MATS)
def test_static_limit_is_kelvin(mat):
    """As s -> 0, U -> U* and T -> T* (Kelvin), with an O(s) correction."""
    rng = np.random.default_rng(3)
    for _ in range(5):
        x, y, n = _rand_pair(rng)
        r = np.linalg.norm(y - x)
        s = 1e-4 * mat.cs / r
        Us = kernels.kelvin_displacement(x, y, mat)
        Ts = kernels.kelvin_traction(x, y, n, mat)
        U = kernels.displacement_kernel(x, y, s, mat)
        T = kernels.traction_kernel(x, y, n, s, mat)
        assert np.abs(U - Us).max() <= 1e-3 * np.abs(Us).max()
        assert np.abs(T - Ts).max() <= 1e-3 * np.abs(Ts).max()


@pytest.mark.parametrize("mat", MATS)
def test_first_order_correction(mat):
    """U(s) - U* = -s/(4 pi mu) [2/(3 c_s) + (c_s/c_p)^2/(3 c_p)] I + O(s^2).

    From the exponential series: r phi = 1/2 + beta2/2 - (2/3) z_s
    - beta2 (1/3) z_p + O(z^2) and r psi has no linear term.
    """
    rng = np.random.default_rng(4)
    x, y, _ = _rand_pair(rng)
    r = np.linalg.norm(y - x)
    cs, cp, mu = mat.cs, mat.cp, mat.mu
    b2 = (cs / cp) ** 2
    s1 = 2e-3 * cs / r
    Us = kernels.kelvin_displacement(x, y, mat)
    d1 = (kernels.displacement_kernel(x, y, s1, mat) - Us) / s1
    d2 = (kernels.displacement_kernel(x, y, 2 * s1, mat) - Us) / (2 * s1)
    slope = 2 * d1 - d2          # Richardson: removes the O(s) part of the quotient
    expect = -(1 / (4 * math.pi * mu)) * (2 / (3 * cs) + b2 / (3 * cp)) * np.eye(3)
    assert np.abs(slope - expect).max() <= 1e-4 * np.abs(expect).max()


def test_symmetries():
    mat = MATS[0]
    rng = np.random.default_rng(5)
    for s in (0.7 + 3.1j, 1.5 - 0.4j):
        x, y, n = _rand_pair(rng)
        U = kernels.displacement_kernel(x, y, s, mat)
        assert np.allclose(U, U.T, rtol=1e-14, atol=0)
        assert np.allclose(U, kernels.displacement_kernel(y, x, s, mat), rtol=1e-14, atol=0)
        assert np.allclose(kernels.displacement_kernel(x, y, np.conj(s), mat), np.conj(U), rtol=1e-14, atol=0)
        T = kernels.traction_kernel(x, y, n, s, mat)
        assert np.allclose(kernels.traction_kernel(x, y, n, np.conj(s), mat), np.conj(T), rtol=1e-13, atol=0)
        # the traction kernel is odd in the separation vector
        assert np.allclose(kernels.traction_kernel(y, x, n, s, mat), -T, rtol=1e-13, atol=0)


def test_decay_under_damping():
    """Reading 1: entries decay at least like exp(-Re(s) r / c_p) at large r.

    The growing branch exp(+s r / c) (the literal e^{i k r} under
    omega -> omega - i eta) would make the ratio below negative.
    """
    mat = MATS[0]
    x = np.zeros(3)
    s = 2.0 + 0.5j
    d = np.array([1.0, 0.0, 0.0])
    U1 = np.abs(kernels.displacement_kernel(x, 5 * d, s, mat)).max()
    U2 = np.abs(kernels.displacement_kernel(x, 6 * d, s, mat)).max()
    rate = math.log(U1 / U2)
    assert rate >= 2.0 / mat.cp
    assert rate <= 2.0 / mat.cs + 1.0
