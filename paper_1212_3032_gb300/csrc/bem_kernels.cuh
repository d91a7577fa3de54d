// Device evaluation of the elastodynamic fundamental solutions and of the
// element integration rules.
//
// U_ij = (1/4 pi mu) [phi delta_ij - psi rh_i rh_j]                 (Sec. 2.1, Eq. Uij)
// T_ij = G_ikj n_k, G_ikj from Eq. Gikj with r_i = y_i - x_i          (Eqs. Tij, Gikj)
// r phi = A(z_s) - beta2 B(z_p),  r psi = C(z_s) - beta2 C(z_p),  z = s r / c,
//   A = (1 + 1/z + 1/z^2) e^-z,  B = (1/z + 1/z^2) e^-z,  C = (1 + 3/z + 3/z^2) e^-z
// (Laplace form of the printed radial functions; the P-wave terms carry
// beta2 = (c_s/c_p)^2).
//
// Precision: the singular parts of A, B, C (1/z^2, 3/z^2) cancel exactly in
// phi and psi, so for small |z_s| the regular remainders
//   Ah = A - 1/z^2,  Bh = B - 1/z^2,  Ch = C - 3/z^2
// are summed from their Taylor series (coefficients from the exponential
// series, uploaded once per translation unit); for larger |z| the closed
// forms are used directly.
#pragma once

#include "bem_common.cuh"

namespace bem {

// One copy per translation unit; filled by that unit's upload function.
static __constant__ RuleTables c_rules;

template <typename R> __device__ __forceinline__ R gl_x(int q, int i) { return R(c_rules.gl_x[q][i]); }
template <typename R> __device__ __forceinline__ R gl_w(int q, int i) { return R(c_rules.gl_w[q][i]); }

// Horner sums of f(z) = sum_m c[m] z^m and f'(z) = sum_m (m+1) c[m+1] z^m.
template <typename R, int M>
__device__ __forceinline__ void series_fd(const double* c, const double* cd, cplx<R> z, cplx<R>& f,
                                          cplx<R>& fd) {
  cplx<R> a = mk<R>(R(c[M]), R(0));
  cplx<R> b = mk<R>(R(cd[M - 1]), R(0));
#pragma unroll
  for (int m = M - 1; m >= 0; --m) {
    a = a * z + R(c[m]);
  }
#pragma unroll
  for (int m = M - 2; m >= 0; --m) {
    b = b * z + R(cd[m]);
  }
  f = a;
  fd = b;
}

// Phi = r phi, dPhi = d(r phi)/dr, Psi = r psi, dPsi = d(r psi)/dr
template <typename R>
__device__ __forceinline__ void radial(R r, const KParams<R>& P, cplx<R>& Phi, cplx<R>& dPhi,
                                       cplx<R>& Psi, cplx<R>& dPsi) {
  constexpr int M = sizeof(R) == 4 ? SERIES_M_F32 : SERIES_M_F64;
  cplx<R> zs = P.ks * r;
  cplx<R> zp = P.kp * r;
  if (abs2(zs) < R(Z_SERIES * Z_SERIES)) {
    cplx<R> Ah, dAh, Bh, dBh, Chs, dChs, Chp, dChp;
    series_fd<R, M>(c_rules.ser[0], c_rules.ser[3], zs, Ah, dAh);
    series_fd<R, M>(c_rules.ser[1], c_rules.ser[4], zp, Bh, dBh);
    series_fd<R, M>(c_rules.ser[2], c_rules.ser[5], zs, Chs, dChs);
    series_fd<R, M>(c_rules.ser[2], c_rules.ser[5], zp, Chp, dChp);
    Phi = Ah - P.beta2 * Bh;
    dPhi = P.ks * dAh - P.beta2 * (P.kp * dBh);
    Psi = Chs - P.beta2 * Chp;
    dPsi = P.ks * dChs - P.beta2 * (P.kp * dChp);
  } else {
    cplx<R> Es = cexp_neg(zs), Ep = cexp_neg(zp);
    cplx<R> qs = inv(zs), qp = inv(zp);
    cplx<R> qs2 = qs * qs, qp2 = qp * qp;
    cplx<R> qs3 = qs2 * qs, qp3 = qp2 * qp;
    cplx<R> A = (qs + qs2 + R(1)) * Es;
    cplx<R> dA = -((qs + R(2) * qs2 + R(2) * qs3 + R(1)) * Es);
    cplx<R> B = (qp + qp2) * Ep;
    cplx<R> dB = -((qp + R(2) * qp2 + R(2) * qp3) * Ep);
    cplx<R> Cs = (R(3) * qs + R(3) * qs2 + R(1)) * Es;
    cplx<R> dCs = -((R(3) * qs + R(6) * qs2 + R(6) * qs3 + R(1)) * Es);
    cplx<R> Cp = (R(3) * qp + R(3) * qp2 + R(1)) * Ep;
    cplx<R> dCp = -((R(3) * qp + R(6) * qp2 + R(6) * qp3 + R(1)) * Ep);
    Phi = A - P.beta2 * B;
    dPhi = P.ks * dA - P.beta2 * (P.kp * dB);
    Psi = Cs - P.beta2 * Cp;
    dPsi = P.ks * dCs - P.beta2 * (P.kp * dCp);
  }
}

// Accumulators of one 3x3 block pair: U is symmetric (6 entries), T full.
template <typename R> struct UTAcc {
  cplx<R> u[6];  // 00 01 02 11 12 22
  cplx<R> t[9];  // row-major
  __device__ __forceinline__ void zero() {
#pragma unroll
    for (int i = 0; i < 6; ++i) u[i] = mk<R>(0, 0);
#pragma unroll
    for (int i = 0; i < 9; ++i) t[i] = mk<R>(0, 0);
  }
  __device__ __forceinline__ cplx<R> U(int i, int j) const {
    const int idx[3][3] = {{0, 1, 2}, {1, 3, 4}, {2, 4, 5}};
    return u[idx[i][j]];
  }
};

// Adds w * U(x, y), w * T(x, y; n) with rv = y - x.
template <typename R>
__device__ __forceinline__ void accumulate_point(UTAcc<R>& acc, R rx, R ry, R rz, R nx, R ny, R nz,
                                                 R w, const KParams<R>& P) {
  R r2 = rx * rx + ry * ry + rz * rz;
  R r = sqrt(r2);
  R ir = R(1) / r;
  R h[3] = {rx * ir, ry * ir, rz * ir};
  R n[3] = {nx, ny, nz};
  R rn = h[0] * nx + h[1] * ny + h[2] * nz;
  cplx<R> Phi, dPhi, Psi, dPsi;
  radial<R>(r, P, Phi, dPhi, Psi, dPsi);
  cplx<R> phi = Phi * ir, psi = Psi * ir;
  cplx<R> dphi = (dPhi - phi) * ir, dpsi = (dPsi - psi) * ir;
  cplx<R> psir = psi * ir;
  // U = cd I + cr h h^T
  cplx<R> cd = phi * (P.u_scale * w);
  cplx<R> cr = psi * (-P.u_scale * w);
  acc.u[0] = acc.u[0] + cd;
  acc.u[3] = acc.u[3] + cd;
  acc.u[5] = acc.u[5] + cd;
  cfmr(acc.u[0], cr, h[0] * h[0]);
  cfmr(acc.u[1], cr, h[0] * h[1]);
  cfmr(acc.u[2], cr, h[0] * h[2]);
  cfmr(acc.u[3], cr, h[1] * h[1]);
  cfmr(acc.u[4], cr, h[1] * h[2]);
  cfmr(acc.u[5], cr, h[2] * h[2]);
  // T = (1/4 pi) [a (rn I + n h^T) + bb rn h h^T + c h n^T]
  R tw = P.t_scale * w;
  cplx<R> a = (dphi - psir) * tw;
  cplx<R> bb = (R(4) * psir - R(2) * dpsi) * tw;
  cplx<R> dd = dphi - dpsi;
  cplx<R> c = (P.k2 * (dd - R(2) * psir) - R(2) * (dd - psir)) * tw;
  cplx<R> arn = a * rn;
  cplx<R> brn = bb * rn;
#pragma unroll
  for (int i = 0; i < 3; ++i) {
#pragma unroll
    for (int j = 0; j < 3; ++j) {
      cplx<R>& t = acc.t[3 * i + j];
      if (i == j) t = t + arn;
      cfmr(t, a, n[i] * h[j]);
      cfmr(t, brn, h[i] * h[j]);
      cfmr(t, c, h[i] * n[j]);
    }
  }
}

// Subtracts w * (static Kelvin U*, T*) at rv = y - x (FP64 remainder rules).
__device__ __forceinline__ void subtract_kelvin(UTAcc<double>& acc, double rx, double ry, double rz,
                                                double nx, double ny, double nz, double w,
                                                const KParams<double>& P) {
  double r2 = rx * rx + ry * ry + rz * rz;
  double r = sqrt(r2);
  double ir = 1.0 / r;
  double h[3] = {rx * ir, ry * ir, rz * ir};
  double n[3] = {nx, ny, nz};
  double rn = h[0] * nx + h[1] * ny + h[2] * nz;
  double nu = P.nu;
  double su = P.kel_u * ir * w;           // U* = kel_u / r [(3-4nu) I + h h^T]
  double st = -P.kel_t * ir * ir * w;     // T* = -kel_t / r^2 [...]
  double a34 = 3.0 - 4.0 * nu, a12 = 1.0 - 2.0 * nu;
  const int iu[6][2] = {{0, 0}, {0, 1}, {0, 2}, {1, 1}, {1, 2}, {2, 2}};
#pragma unroll
  for (int m = 0; m < 6; ++m) {
    int i = iu[m][0], j = iu[m][1];
    acc.u[m].re -= su * ((i == j ? a34 : 0.0) + h[i] * h[j]);
  }
#pragma unroll
  for (int i = 0; i < 3; ++i) {
#pragma unroll
    for (int j = 0; j < 3; ++j) {
      double v = rn * ((i == j ? a12 : 0.0) + 3.0 * h[i] * h[j]) - a12 * (h[i] * n[j] - h[j] * n[i]);
      acc.t[3 * i + j].re -= st * v;
    }
  }
}

// Adds w * (static Kelvin U*, T*) into real accumulators (18 doubles).
__device__ __forceinline__ void add_kelvin(double* us, double* ts, double rx, double ry, double rz,
                                           double nx, double ny, double nz, double w,
                                           const KParams<double>& P) {
  double r2 = rx * rx + ry * ry + rz * rz;
  double r = sqrt(r2);
  double ir = 1.0 / r;
  double h[3] = {rx * ir, ry * ir, rz * ir};
  double n[3] = {nx, ny, nz};
  double rn = h[0] * nx + h[1] * ny + h[2] * nz;
  double nu = P.nu;
  double su = P.kel_u * ir * w;
  double st = -P.kel_t * ir * ir * w;
  double a34 = 3.0 - 4.0 * nu, a12 = 1.0 - 2.0 * nu;
#pragma unroll
  for (int i = 0; i < 3; ++i) {
#pragma unroll
    for (int j = 0; j < 3; ++j) {
      us[3 * i + j] += su * ((i == j ? a34 : 0.0) + h[i] * h[j]);
      double v = rn * ((i == j ? a12 : 0.0) + 3.0 * h[i] * h[j]) - a12 * (h[i] * n[j] - h[j] * n[i]);
      ts[3 * i + j] += st * v;
    }
  }
}

// Band of a pair from rho2 = d2 / h_e^2 (the SELF case is handled by the caller).
template <typename R> __device__ __forceinline__ int band_of(R d2, R he2) {
  if (d2 < R(RHO2_NEAR) * he2) return BAND_NEAR;
  if (d2 < R(RHO2_Q4) * he2) return BAND_Q4;
  if (d2 < R(RHO2_Q2) * he2) return BAND_Q2;
  return BAND_Q1;
}

// FP32 band decision that agrees with the FP64 one: near a threshold the
// decision is redone in FP64.
__device__ __forceinline__ int band_f32_exact(float d2, float he2, double d2d, double he2d) {
  const float thr[3] = {float(RHO2_NEAR), float(RHO2_Q4), float(RHO2_Q2)};
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    float t = thr[k] * he2;
    if (fabsf(d2 - t) <= 1e-4f * t) return band_of<double>(d2d, he2d);
  }
  return band_of<float>(d2, he2);
}

// Collapsed q x q rule on a triangle given by p0-relative offset o0 (the
// position of p0 relative to the collocation point) and edges e1, e2.
template <typename R, int Q>
__device__ __forceinline__ void integrate_collapsed(UTAcc<R>& acc, const R* o0, const R* e1,
                                                    const R* e2, R area2, const R* n,
                                                    const KParams<R>& P) {
#pragma unroll
  for (int a = 0; a < Q; ++a) {
    R u = gl_x<R>(Q, a), wu = gl_w<R>(Q, a);
    R omu = R(1) - u;
#pragma unroll
    for (int b = 0; b < Q; ++b) {
      R v = omu * gl_x<R>(Q, b);
      R w = area2 * wu * gl_w<R>(Q, b) * omu;
      R rx = o0[0] + u * e1[0] + v * e2[0];
      R ry = o0[1] + u * e1[1] + v * e2[1];
      R rz = o0[2] + u * e1[2] + v * e2[2];
      accumulate_point<R>(acc, rx, ry, rz, n[0], n[1], n[2], w, P);
    }
  }
}

}  // namespace bem
