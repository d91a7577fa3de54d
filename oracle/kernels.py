"""Elastodynamic fundamental solutions in the Laplace domain (oracle).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

Sec. 2.1, Eqs. Uij, Tij, Gikj with the radial functions phi, psi. The complex
frequency of the exponential window (Sec. 3.1, Eq. scaled-u-TD and the text
after it) is written s = eta + i k dw, i.e. s = i omega_k with
omega_k = k dw - i eta. The paper's exp(i k r) is read as exp(-s r / c), the
branch that decays under the artificial damping (reading 1), and its P-wave
terms carry (c_s/c_p)^2 so that the static limit exists (reading 2).

All inputs/outputs are float64 / complex128 numpy arrays; the last axis of a
point array is the coordinate axis.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np


@dataclasses.dataclass(frozen=True)
class Material:
    """Isotropic elastic solid (Sec. 2.1): Young's modulus, Poisson, density."""

    E: float
    nu: float
    rho: float

    @property
    def mu(self) -> float:
        return self.E / (2.0 * (1.0 + self.nu))

    @property
    def lam(self) -> float:
        return self.E * self.nu / ((1.0 + self.nu) * (1.0 - 2.0 * self.nu))

    @property
    def cs(self) -> float:
        """S-wave speed c_s = sqrt(mu / rho)."""
        return math.sqrt(self.mu / self.rho)

    @property
    def cp(self) -> float:
        """P-wave speed c_p = sqrt((lambda + 2 mu) / rho)."""
        return math.sqrt((self.lam + 2.0 * self.mu) / self.rho)


def radial_functions(r, s, mat: Material):
    """phi(r), psi(r) and their r-derivatives (Sec. 2.1, after Eq. Gikj).

    With z = s r / c and beta2 = (c_s / c_p)^2:
      r phi = (1 + 1/z_s + 1/z_s^2) e^{-z_s} - beta2 (1/z_p + 1/z_p^2) e^{-z_p}
      r psi = (1 + 3/z_s + 3/z_s^2) e^{-z_s} - beta2 (1 + 3/z_p + 3/z_p^2) e^{-z_p}
    The derivatives are not printed in the paper; they follow from
    d/dr = (s/c) d/dz applied to the bracketed functions of z.
    """
    r = np.asarray(r, dtype=np.float64)
    s = complex(s)
    cs, cp = mat.cs, mat.cp
    beta2 = (cs / cp) ** 2
    zs = s * r / cs
    zp = s * r / cp
    es = np.exp(-zs)
    ep = np.exp(-zp)
    qs = 1.0 / zs
    qp = 1.0 / zp
    qs2, qp2 = qs * qs, qp * qp
    qs3, qp3 = qs2 * qs, qp2 * qp
    # bracketed functions of z and their z-derivatives
    A = (1 + qs + qs2) * es
    dA = -(1 + qs + 2 * qs2 + 2 * qs3) * es
    B = (qp + qp2) * ep
    dB = -(qp + 2 * qp2 + 2 * qp3) * ep
    Cs = (1 + 3 * qs + 3 * qs2) * es
    dCs = -(1 + 3 * qs + 6 * qs2 + 6 * qs3) * es
    Cp = (1 + 3 * qp + 3 * qp2) * ep
    dCp = -(1 + 3 * qp + 6 * qp2 + 6 * qp3) * ep
    Phi = A - beta2 * B
    dPhi = (s / cs) * dA - beta2 * (s / cp) * dB
    Psi = Cs - beta2 * Cp
    dPsi = (s / cs) * dCs - beta2 * (s / cp) * dCp
    ir = 1.0 / r
    phi = Phi * ir
    psi = Psi * ir
    dphi = (dPhi - phi) * ir
    dpsi = (dPsi - psi) * ir
    return phi, psi, dphi, dpsi


def displacement_kernel(x, y, s, mat: Material):
    """U_ij(x, y; s) (Eq. Uij): displacement j at y from a unit force i at x.

    U_ij = (1 / 4 pi mu) [phi delta_ij - psi rhat_i rhat_j], rhat = (x-y)/r
    (the sign of rhat does not matter here). Shape (..., 3, 3).
    """
    x = np.asarray(x, dtype=np.float64)
    y = np.asarray(y, dtype=np.float64)
    rv = x - y
    r = np.linalg.norm(rv, axis=-1)
    rh = rv / r[..., None]
    phi, psi, _, _ = radial_functions(r, s, mat)
    eye = np.eye(3)
    U = phi[..., None, None] * eye - psi[..., None, None] * rh[..., :, None] * rh[..., None, :]
    return U / (4.0 * math.pi * mat.mu)


def traction_kernel(x, y, n, s, mat: Material):
    """T_ij(x, y; s) = G_ikj n_k(y) (Eqs. Tij, Gikj).

    G_ikj = 1/(4 pi r) [ (phi' - psi/r)(delta_ij r_k + delta_ik r_j)
                         + (2/r^2)(2 psi/r - psi') r_i r_j r_k
                         + ((c_p/c_s)^2 (phi' - psi' - 2 psi/r)
                            - 2 (phi' - psi' - psi/r)) delta_jk r_i ]
    with r_i = y_i - x_i (reading 3). ``n`` is the unit normal at y, out of
    the solid. Shape (..., 3, 3).
    """
    x = np.asarray(x, dtype=np.float64)
    y = np.asarray(y, dtype=np.float64)
    n = np.asarray(n, dtype=np.float64)
    rv = y - x
    r = np.linalg.norm(rv, axis=-1)
    phi, psi, dphi, dpsi = radial_functions(r, s, mat)
    k2 = (mat.cp / mat.cs) ** 2
    a = dphi - psi / r
    b = (2.0 / r**2) * (2.0 * psi / r - dpsi)
    c = k2 * (dphi - dpsi - 2.0 * psi / r) - 2.0 * (dphi - dpsi - psi / r)
    rn = np.einsum("...k,...k->...", rv, np.broadcast_to(n, rv.shape))
    nb = np.broadcast_to(n, rv.shape)
    eye = np.eye(3)
    # G_ikj n_k term by term:
    #   (delta_ij r_k + delta_ik r_j) n_k = delta_ij (r.n) + n_i r_j
    #   r_i r_j r_k n_k = r_i r_j (r.n)
    #   delta_jk r_i n_k = r_i n_j
    T = (a[..., None, None] * (rn[..., None, None] * eye + nb[..., :, None] * rv[..., None, :])
         + (b * rn)[..., None, None] * rv[..., :, None] * rv[..., None, :]
         + c[..., None, None] * rv[..., :, None] * nb[..., None, :])
    return T / (4.0 * math.pi * r[..., None, None])


def kernel_pair(x, y, n, s, mat: Material):
    """U_ij and T_ij together (one evaluation of the radial functions).

    Same definitions as ``displacement_kernel`` and ``traction_kernel``.
    """
    x = np.asarray(x, dtype=np.float64)
    y = np.asarray(y, dtype=np.float64)
    rv = y - x
    r = np.linalg.norm(rv, axis=-1)
    phi, psi, dphi, dpsi = radial_functions(r, s, mat)
    nb = np.broadcast_to(np.asarray(n, dtype=np.float64), rv.shape)
    rr = rv[..., :, None] * rv[..., None, :]
    eye = np.eye(3)
    U = (phi[..., None, None] * eye - (psi / r**2)[..., None, None] * rr) / (4.0 * math.pi * mat.mu)
    k2 = (mat.cp / mat.cs) ** 2
    a = dphi - psi / r
    b = (2.0 / r**2) * (2.0 * psi / r - dpsi)
    c = k2 * (dphi - dpsi - 2.0 * psi / r) - 2.0 * (dphi - dpsi - psi / r)
    rn = np.einsum("...k,...k->...", rv, nb)
    T = (a[..., None, None] * (rn[..., None, None] * eye + nb[..., :, None] * rv[..., None, :])
         + (b * rn)[..., None, None] * rr
         + c[..., None, None] * rv[..., :, None] * nb[..., None, :])
    return U, T / (4.0 * math.pi * r[..., None, None])


def kelvin_displacement(x, y, mat: Material):
    """Static Kelvin displacement kernel (textbook closed form).

    U*_ij = [(3 - 4 nu) delta_ij + rhat_i rhat_j] / (16 pi mu (1 - nu) r).
    """
    x = np.asarray(x, dtype=np.float64)
    y = np.asarray(y, dtype=np.float64)
    rv = y - x
    r = np.linalg.norm(rv, axis=-1)
    rh = rv / r[..., None]
    nu = mat.nu
    U = (3 - 4 * nu) * np.eye(3) + rh[..., :, None] * rh[..., None, :]
    return U / (16.0 * math.pi * mat.mu * (1 - nu) * r[..., None, None])


def kelvin_traction(x, y, n, mat: Material):
    """Static Kelvin traction kernel (textbook closed form), rhat = (y-x)/r.

    T*_ij = -1/(8 pi (1-nu) r^2) [ (rhat.n)((1-2nu) delta_ij + 3 rhat_i rhat_j)
                                   - (1-2nu)(rhat_i n_j - rhat_j n_i) ].
    """
    x = np.asarray(x, dtype=np.float64)
    y = np.asarray(y, dtype=np.float64)
    n = np.asarray(n, dtype=np.float64)
    rv = y - x
    r = np.linalg.norm(rv, axis=-1)
    rh = rv / r[..., None]
    nb = np.broadcast_to(n, rh.shape)
    nu = mat.nu
    drdn = np.einsum("...k,...k->...", rh, nb)
    T = (drdn[..., None, None] * ((1 - 2 * nu) * np.eye(3) + 3 * rh[..., :, None] * rh[..., None, :])
         - (1 - 2 * nu) * (rh[..., :, None] * nb[..., None, :] - nb[..., :, None] * rh[..., None, :]))
    return -T / (8.0 * math.pi * (1 - nu) * r[..., None, None] ** 2)
