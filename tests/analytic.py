"""Closed-form solutions used as pins (independent of the oracle and the GPU path).

Spherical cavity of radius a in an infinite isotropic solid, uniform pressure
p on the wall, Laplace variable s (time dependence e^{s t}): the radial
displacement is the P-wave field u_r = C e^{-q r} (1 + q r) / r^2 with
q = s / c_p, and the wall condition sigma_rr(a) = -p fixes C. At r = a

    u_r(a, s) = p a (1 + a s / c_p) / (rho a^2 s^2 + 4 mu a s / c_p + 4 mu).

At s = 0 this is the Lame result p a / (4 mu). ``cavity_field`` returns the
whole radial field so a test can check the ODE and the wall condition.

Prismatic rod (Sec. 5.1) with Poisson's ratio 0: the 3-D problem is exactly
1-D (uniaxial stress is uniaxial strain when nu = 0), u_x(x, s) solves
E u'' = rho s^2 u with u(0) = 0 (fixed end) and E u'(L) = -p (the
compressive traction -p n on the end x = L), c = sqrt(E / rho):

    u_x(x, s) = -(p c / (E s)) sinh(s x / c) / cosh(s L / c),

so u_x(L, s) = -(p c / (E s)) tanh(s L / c), and the traction on the fixed
end (normal -x) is t_x(0, s) = -E u'(0) = p / cosh(s L / c).
"""
import math

import numpy as np


def cavity_wall_response(s, a, mu, lam, rho, p=1.0):
    cp = math.sqrt((lam + 2 * mu) / rho)
    s = np.asarray(s, dtype=np.complex128)
    return p * a * (1 + a * s / cp) / (rho * a * a * s * s + 4 * mu * a * s / cp + 4 * mu)


def cavity_field(r, s, a, mu, lam, rho, p=1.0):
    """u_r(r, s) for r >= a."""
    cp = math.sqrt((lam + 2 * mu) / rho)
    q = s / cp
    ua = cavity_wall_response(s, a, mu, lam, rho, p)
    C = ua * a * a / (np.exp(-q * a) * (1 + q * a))
    return C * np.exp(-q * r) * (1 + q * r) / r**2


def cavity_step_response(t, a, mu, lam, rho, p=1.0):
    """Exact u_r(a, t) for a pressure step p H(t), by residues of H(s)/s."""
    cp = math.sqrt((lam + 2 * mu) / rho)
    # H(s)/s = N(s) / (s D(s)),  N = p a (1 + a s/cp),  D = rho a^2 s^2 + 4 mu a s/cp + 4 mu
    Dc = [rho * a * a, 4 * mu * a / cp, 4 * mu]
    poles = np.roots(Dc)
    t = np.asarray(t, dtype=np.float64)
    out = np.full(t.shape, p * a / (4 * mu), dtype=np.complex128)  # residue at s = 0
    for pk in poles:
        dD = 2 * Dc[0] * pk + Dc[1]
        Nk = p * a * (1 + a * pk / cp)
        out = out + Nk / (pk * dD) * np.exp(pk * t)
    return out.real


def rod_field(x, s, L, E, rho, p=1.0):
    """u_x(x, s) of the rod, 0 <= x <= L."""
    c = math.sqrt(E / rho)
    s = np.asarray(s, dtype=np.complex128)
    return -(p * c / (E * s)) * np.sinh(s * x / c) / np.cosh(s * L / c)


def rod_end_displacement(s, L, E, rho, p=1.0):
    c = math.sqrt(E / rho)
    s = np.asarray(s, dtype=np.complex128)
    return -(p * c / (E * s)) * np.tanh(s * L / c)


def rod_fixed_traction(s, L, E, rho, p=1.0):
    c = math.sqrt(E / rho)
    s = np.asarray(s, dtype=np.complex128)
    return p / np.cosh(s * L / c)
