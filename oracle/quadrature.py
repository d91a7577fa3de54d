"""Element integration rules for constant flat triangles (oracle).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

The paper discretises with piecewise-constant triangles and collocation at
each element (Sec. 2.1, Eq. Tu_Ut) but does not state how the element
integrals are evaluated. The rule below is this library's reading; the GPU
path implements the same rule independently.

Element e: vertices p0, p1, p2 in mesh order, unit normal
n = (p1-p0)x(p2-p0)/|.|, area A, centroid c (the collocation point),
size h = longest edge. For collocation point x_i = c_i and element e the band
is chosen from rho2 = |c_i - c_e|^2 / h_e^2:

  SELF  e == i        polar coordinates about c_i over the three triangles
                      (c_i, p0, p1), (c_i, p1, p2), (c_i, p2, p0). The static
                      Kelvin parts are integrated along each ray in closed
                      form (U*: integral of U* r dr = R U*_ang; T*: Cauchy
                      principal value c0 ln R) with 16 Gauss-Legendre angles
                      per triangle; the bounded remainders U - U*, T - T*
                      with 8 angles x 6 radii per triangle.
  NEAR  rho2 < 2.2    static parts U*, T* on three levels of midpoint
                      subdivision (64 children) with the 4x4 collapsed rule
                      each (1024 points); remainders U - U*, T - T* with the
                      4x4 collapsed rule on the element (16 points).
  Q4    rho2 < 9.7    full kernels, collapsed 4x4 rule (16 points).
  Q2    rho2 < 63.3   full kernels, collapsed 2x2 rule (4 points).
  Q1    otherwise     full kernels at the centroid, weight A.

The static parts do not depend on the frequency, so they are computed once
per mesh; only the remainders and the regular bands change with s.

Collapsed q x q rule: Gauss-Legendre nodes u_a, v_b on [0, 1] with weights
w_a, w_b; point p0 + u_a (p1-p0) + (1-u_a) v_b (p2-p0); weight
2 A w_a w_b (1 - u_a).

Midpoint subdivision of (a, b, c) with m_ab, m_bc, m_ca the edge midpoints:
children (a, m_ab, m_ca), (m_ab, b, m_bc), (m_ca, m_bc, c), (m_bc, m_ca, m_ab).
"""
from __future__ import annotations

import numpy as np

BAND_SELF, BAND_NEAR, BAND_Q4, BAND_Q2, BAND_Q1 = 0, 1, 2, 3, 4
RHO2_NEAR = 2.2
RHO2_Q4 = 9.7
RHO2_Q2 = 63.3
SELF_NT_STATIC = 16
SELF_NT = 8
SELF_NR = 6
NEAR_LEVELS = 3   # midpoint subdivision levels for the static part (64 children)
NEAR_Q = 4        # collapsed rule on each child (static part)
NEAR_Q_REM = 4    # collapsed rule on the element (remainder)


def gauss_legendre_01(q: int):
    """Gauss-Legendre nodes and weights on [0, 1]."""
    x, w = np.polynomial.legendre.leggauss(q)
    return 0.5 * (x + 1.0), 0.5 * w


def classify(ci, ce, he, same):
    """Band code per pair from the collocation/element centroid distance."""
    d = np.asarray(ci, dtype=np.float64) - np.asarray(ce, dtype=np.float64)
    rho2 = np.einsum("...k,...k->...", d, d) / np.asarray(he, dtype=np.float64) ** 2
    band = np.full(rho2.shape, BAND_Q1, dtype=np.int8)
    band[rho2 < RHO2_Q2] = BAND_Q2
    band[rho2 < RHO2_Q4] = BAND_Q4
    band[rho2 < RHO2_NEAR] = BAND_NEAR
    band[np.asarray(same)] = BAND_SELF
    return band


def collapsed_rule(p0, p1, p2, q: int):
    """q x q collapsed Gauss rule on triangles (P, 3) -> points (P, q*q, 3), weights (P, q*q)."""
    p0 = np.asarray(p0, dtype=np.float64)
    e1 = np.asarray(p1, dtype=np.float64) - p0
    e2 = np.asarray(p2, dtype=np.float64) - p0
    area2 = np.linalg.norm(np.cross(e1, e2), axis=-1)  # 2A
    u, wu = gauss_legendre_01(q)
    v, wv = gauss_legendre_01(q)
    U, V = np.meshgrid(u, v, indexing="ij")
    WU, WV = np.meshgrid(wu, wv, indexing="ij")
    U, V = U.ravel(), V.ravel()
    W = (WU * WV).ravel() * (1.0 - U)
    pts = p0[:, None, :] + U[None, :, None] * e1[:, None, :] + ((1.0 - U) * V)[None, :, None] * e2[:, None, :]
    wts = area2[:, None] * W[None, :]
    return pts, wts


def centroid_rule(p0, p1, p2):
    """One-point rule at the centroid with weight A."""
    p0 = np.asarray(p0, dtype=np.float64)
    p1 = np.asarray(p1, dtype=np.float64)
    p2 = np.asarray(p2, dtype=np.float64)
    area = 0.5 * np.linalg.norm(np.cross(p1 - p0, p2 - p0), axis=-1)
    return ((p0 + p1 + p2) / 3.0)[:, None, :], area[:, None]


def subdivide(p0, p1, p2):
    """One level of midpoint subdivision; returns a list of 4 (a, b, c) triples."""
    mab = 0.5 * (p0 + p1)
    mbc = 0.5 * (p1 + p2)
    mca = 0.5 * (p2 + p0)
    return [(p0, mab, mca), (mab, p1, mbc), (mca, mbc, p2), (mbc, mca, mab)]


def near_rule(p0, p1, p2):
    """Three subdivision levels x collapsed 4x4: points (P, 1024, 3), weights (P, 1024)."""
    tris = [(np.asarray(p0, float), np.asarray(p1, float), np.asarray(p2, float))]
    for _ in range(NEAR_LEVELS):
        nxt = []
        for t in tris:
            nxt += subdivide(*t)
        tris = nxt
    pts, wts = [], []
    for a, b, c in tris:
        p, w = collapsed_rule(a, b, c, NEAR_Q)
        pts.append(p)
        wts.append(w)
    return np.concatenate(pts, axis=1), np.concatenate(wts, axis=1)


def self_rule(c, p0, p1, p2, n, nt: int = SELF_NT, nr: int = SELF_NR):
    """Polar rule about the collocation point c on its own element.

    Returns (pts, wts, dirs, logR, wth):
      pts  (P, 3*nt*nr, 3) points c + r dir(theta)
      wts  (P, 3*nt*nr)    weights for  integral f dA  (includes the Jacobian r)
      dirs (P, 3*nt, 3)    ray directions at the angular nodes
      logR (P, 3*nt)       ln R(theta), R = distance from c to the edge
      wth  (P, 3*nt)       angular weights (for the principal-value term)
    """
    c = np.asarray(c, dtype=np.float64)
    n = np.asarray(n, dtype=np.float64)
    verts = [np.asarray(p0, float), np.asarray(p1, float), np.asarray(p2, float)]
    tn, tw = gauss_legendre_01(nt)
    rn, rw = gauss_legendre_01(nr)
    all_pts, all_w, all_dir, all_logR, all_wth = [], [], [], [], []
    for k in range(3):
        pa, pb = verts[k], verts[(k + 1) % 3]
        t = pb - pa
        lam = np.einsum("ij,ij->i", c - pa, t) / np.einsum("ij,ij->i", t, t)
        foot = pa + lam[:, None] * t
        fv = foot - c
        d = np.linalg.norm(fv, axis=-1)
        fh = fv / d[:, None]
        gh = np.cross(n, fh)
        tha = np.arctan2(np.einsum("ij,ij->i", pa - c, gh), np.einsum("ij,ij->i", pa - c, fh))
        thb = np.arctan2(np.einsum("ij,ij->i", pb - c, gh), np.einsum("ij,ij->i", pb - c, fh))
        dth = thb - tha
        th = tha[:, None] + dth[:, None] * tn[None, :]          # (P, nt)
        wth = dth[:, None] * tw[None, :]                        # (P, nt)
        R = d[:, None] / np.cos(th)                             # (P, nt)
        dirs = np.cos(th)[..., None] * fh[:, None, :] + np.sin(th)[..., None] * gh[:, None, :]
        r = R[..., None] * rn[None, None, :]                    # (P, nt, nr)
        wr = R[..., None] * rw[None, None, :]
        pts = c[:, None, None, :] + r[..., None] * dirs[:, :, None, :]
        w = wth[..., None] * wr * r
        P = c.shape[0]
        all_pts.append(pts.reshape(P, nt * nr, 3))
        all_w.append(w.reshape(P, nt * nr))
        all_dir.append(dirs)
        all_logR.append(np.log(R))
        all_wth.append(wth)
    return (np.concatenate(all_pts, axis=1), np.concatenate(all_w, axis=1),
            np.concatenate(all_dir, axis=1), np.concatenate(all_logR, axis=1),
            np.concatenate(all_wth, axis=1))
