// Device evaluation of the elastodynamic fundamental solutions and of the
// element integration rules.
//
// U_ij = (1/4 pi mu) [phi delta_ij - psi rh_i rh_j]                 (Sec. 2.1, Eq. Uij)
// T_ij = G_ikj n_k, G_ikj from Eq. Gikj with r_i = y_i - x_i          (Eqs. Tij, Gikj)
//      = (1/4 pi r^2) [A (rn delta_ij + n_i rh_j) + B rn rh_i rh_j + C rh_i n_j]
// with r phi = Phi(z_s), r psi = Psi(z_s) and A, B, C the combinations of
// KParams (Laplace form of the printed radial functions, z = s r / c; the
// P-wave terms carry beta2 = (c_s/c_p)^2).
//
// Two evaluation branches:
//   |z_s| <  Z_SERIES : Taylor series of Phi, Psi, A, B, C in z_s
//                       (coefficients per material, m-th term), free of the
//                       1/z^k cancellations of the closed forms;
//   |z_s| >= Z_SERIES : closed forms A(z) = (1 + 1/z + 1/z^2) e^-z,
//                       B(z) = (1/z + 1/z^2) e^-z, C(z) = (1 + 3/z + 3/z^2) e^-z
//                       and z A'(z), z B'(z), z C'(z).
// FULL = false gives the dynamic remainder (kernel minus its static Kelvin
// limit): the series without the m = 0 term, the closed forms minus the
// static constants.
#pragma once

#include "bem_common.cuh"

namespace bem {

// One copy per translation unit; filled by that unit's upload function.
static __constant__ RuleTables c_rules;

template <typename R> __device__ __forceinline__ R gl_x(int q, int i);
template <typename R> __device__ __forceinline__ R gl_w(int q, int i);
template <> __device__ __forceinline__ float gl_x<float>(int q, int i) { return c_rules.gl_xf[q][i]; }
template <> __device__ __forceinline__ float gl_w<float>(int q, int i) { return c_rules.gl_wf[q][i]; }
template <> __device__ __forceinline__ double gl_x<double>(int q, int i) { return c_rules.gl_x[q][i]; }
template <> __device__ __forceinline__ double gl_w<double>(int q, int i) { return c_rules.gl_w[q][i]; }

// Phi, Psi, A, B, C at r (FULL) or their dynamic remainders (!FULL).
template <typename R, bool FULL>
__device__ __forceinline__ void radial5(R r, const KParams<R>& P, cplx<R>& Phi, cplx<R>& Psi, cplx<R>& A,
                                        cplx<R>& B, cplx<R>& C) {
  constexpr int M = sizeof(R) == 4 ? SERIES_M_F32 : SERIES_M_F64;
  cplx<R> z = P.ks * r;
  if (abs2(z) < R(Z_SERIES * Z_SERIES)) {
    cplx<R> s0 = mk<R>(P.ser[0][M], R(0)), s1 = mk<R>(P.ser[1][M], R(0)), s2 = mk<R>(P.ser[2][M], R(0));
    cplx<R> s3 = mk<R>(P.ser[3][M], R(0)), s4 = mk<R>(P.ser[4][M], R(0));
#pragma unroll
    for (int m = M - 1; m >= (FULL ? 0 : 1); --m) {
      s0 = s0 * z + P.ser[0][m];
      s1 = s1 * z + P.ser[1][m];
      s2 = s2 * z + P.ser[2][m];
      s3 = s3 * z + P.ser[3][m];
      s4 = s4 * z + P.ser[4][m];
    }
    if (!FULL) {  // the loop stopped at m = 1: one more factor z
      s0 = s0 * z;
      s1 = s1 * z;
      s2 = s2 * z;
      s3 = s3 * z;
      s4 = s4 * z;
    }
    Phi = s0;
    Psi = s1;
    A = s2;
    B = s3;
    C = s4;
  } else {
    cplx<R> zp = P.kp * r;
    cplx<R> Es = cexp_neg(z), Ep = cexp_neg(zp);
    cplx<R> qs = inv(z), qp = inv(zp);
    cplx<R> qs2 = qs * qs, qp2 = qp * qp;
    cplx<R> As = (qs + qs2 + R(1)) * Es;
    cplx<R> zAs = -((z + R(2) * qs + R(2) * qs2 + R(1)) * Es);
    cplx<R> Bp = (qp + qp2) * Ep;
    cplx<R> zBp = -((R(2) * qp + R(2) * qp2 + R(1)) * Ep);
    cplx<R> Cs = (R(3) * qs + R(3) * qs2 + R(1)) * Es;
    cplx<R> zCs = -((z + R(6) * qs + R(6) * qs2 + R(3)) * Es);
    cplx<R> Cp = (R(3) * qp + R(3) * qp2 + R(1)) * Ep;
    cplx<R> zCp = -((zp + R(6) * qp + R(6) * qp2 + R(3)) * Ep);
    cplx<R> Ph = As - P.beta2 * Bp;
    cplx<R> Ps = Cs - P.beta2 * Cp;
    cplx<R> DPh = zAs - P.beta2 * zBp;
    cplx<R> DPs = zCs - P.beta2 * zCp;
    cplx<R> t1 = DPh - Ph;
    Phi = Ph;
    Psi = Ps;
    A = t1 - Ps;
    B = R(2) * (R(3) * Ps - DPs);
    C = P.k2 * (t1 - DPs - Ps) - R(2) * (t1 - DPs);
    if (!FULL) {
      Phi.re -= P.ser[0][0];
      Psi.re -= P.ser[1][0];
      A.re -= P.ser[2][0];
      B.re -= P.ser[3][0];
      C.re -= P.ser[4][0];
    }
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

// Adds w * U(x, y), w * T(x, y; n) (or their dynamic remainders) at rv = y - x.
template <typename R, bool FULL = true>
__device__ __forceinline__ void accumulate_point(UTAcc<R>& acc, R rx, R ry, R rz, R nx, R ny, R nz,
                                                 R w, const KParams<R>& P) {
  R r2 = rx * rx + ry * ry + rz * rz;
  R r = sqrt(r2);
  R ir = R(1) / r;
  R h[3] = {rx * ir, ry * ir, rz * ir};
  R n[3] = {nx, ny, nz};
  R rn = h[0] * nx + h[1] * ny + h[2] * nz;
  cplx<R> Phi, Psi, A, B, C;
  radial5<R, FULL>(r, P, Phi, Psi, A, B, C);
  // U = (1/4 pi mu r) [Phi I - Psi h h^T]
  R uw = P.u_scale * w * ir;
  cplx<R> cd = Phi * uw;
  cplx<R> cr = Psi * (-uw);
  acc.u[0] = acc.u[0] + cd;
  acc.u[3] = acc.u[3] + cd;
  acc.u[5] = acc.u[5] + cd;
  cfmr(acc.u[0], cr, h[0] * h[0]);
  cfmr(acc.u[1], cr, h[0] * h[1]);
  cfmr(acc.u[2], cr, h[0] * h[2]);
  cfmr(acc.u[3], cr, h[1] * h[1]);
  cfmr(acc.u[4], cr, h[1] * h[2]);
  cfmr(acc.u[5], cr, h[2] * h[2]);
  // T = (1/4 pi r^2) [A (rn I + n h^T) + B rn h h^T + C h n^T]
  R tw = P.t_scale * w * ir * ir;
  cplx<R> a = A * tw;
  cplx<R> brn = B * (tw * rn);
  cplx<R> c = C * tw;
  cplx<R> arn = a * rn;
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

// One line of the 3x3 pair block at one quadrature point: row idx (col = false:
// entries (idx, c), c < 3) or column idx (col = true: entries (a, idx)) of T
// (useT) or of U. ACA steps need one scalar row or column of the system
// matrix, i.e. one line of each pair's block; the radial functions are shared,
// the rest of the tensor is not formed.
template <typename R>
__device__ __forceinline__ void accumulate_point_line(cplx<R> out[3], R rx, R ry, R rz, R nx, R ny, R nz, R w,
                                                      const KParams<R>& P, bool useT, bool col, int idx) {
  R r2 = rx * rx + ry * ry + rz * rz;
  R r = sqrt(r2);
  R ir = R(1) / r;
  R h[3] = {rx * ir, ry * ir, rz * ir};
  R n[3] = {nx, ny, nz};
  cplx<R> Phi, Psi, A, B, C;
  radial5<R, true>(r, P, Phi, Psi, A, B, C);
  const R hi = idx == 0 ? h[0] : (idx == 1 ? h[1] : h[2]);
  if (useT) {
    R rn = h[0] * nx + h[1] * ny + h[2] * nz;
    R tw = P.t_scale * w * ir * ir;
    cplx<R> a = A * tw;
    cplx<R> brn = B * (tw * rn);
    cplx<R> c = C * tw;
    cplx<R> arn = a * rn;
    const R ni = idx == 0 ? n[0] : (idx == 1 ? n[1] : n[2]);
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      // (i, j) = (idx, k) for a row, (k, idx) for a column
      const R hI = col ? h[k] : hi, hJ = col ? hi : h[k];
      const R nI = col ? n[k] : ni, nJ = col ? ni : n[k];
      cplx<R>& t = out[k];
      if (k == idx) t = t + arn;
      cfmr(t, a, nI * hJ);
      cfmr(t, brn, hI * hJ);
      cfmr(t, c, hI * nJ);
    }
  } else {
    R uw = P.u_scale * w * ir;
    cplx<R> cd = Phi * uw;
    cplx<R> cr = Psi * (-uw);
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      cplx<R>& u = out[k];
      if (k == idx) u = u + cd;
      cfmr(u, cr, hi * h[k]);  // U is symmetric: row and column lines agree
    }
  }
}

// U only (6 entries), full kernel: for right-hand sides of traction-loaded
// elements, where T is not needed.
template <typename R>
__device__ __forceinline__ void accumulate_point_u(cplx<R>* u, R rx, R ry, R rz, R w, const KParams<R>& P) {
  constexpr int M = sizeof(R) == 4 ? SERIES_M_F32 : SERIES_M_F64;
  R r2 = rx * rx + ry * ry + rz * rz;
  R r = sqrt(r2);
  R ir = R(1) / r;
  R h[3] = {rx * ir, ry * ir, rz * ir};
  cplx<R> z = P.ks * r;
  cplx<R> Phi, Psi;
  if (abs2(z) < R(Z_SERIES * Z_SERIES)) {
    cplx<R> s0 = mk<R>(P.ser[0][M], R(0)), s1 = mk<R>(P.ser[1][M], R(0));
#pragma unroll
    for (int m = M - 1; m >= 0; --m) {
      s0 = s0 * z + P.ser[0][m];
      s1 = s1 * z + P.ser[1][m];
    }
    Phi = s0;
    Psi = s1;
  } else {
    cplx<R> zp = P.kp * r;
    cplx<R> Es = cexp_neg(z), Ep = cexp_neg(zp);
    cplx<R> qs = inv(z), qp = inv(zp);
    cplx<R> qs2 = qs * qs, qp2 = qp * qp;
    Phi = (qs + qs2 + R(1)) * Es - P.beta2 * ((qp + qp2) * Ep);
    Psi = (R(3) * qs + R(3) * qs2 + R(1)) * Es - P.beta2 * ((R(3) * qp + R(3) * qp2 + R(1)) * Ep);
  }
  R uw = P.u_scale * w * ir;
  cplx<R> cd = Phi * uw;
  cplx<R> cr = Psi * (-uw);
  u[0] = u[0] + cd;
  u[3] = u[3] + cd;
  u[5] = u[5] + cd;
  cfmr(u[0], cr, h[0] * h[0]);
  cfmr(u[1], cr, h[0] * h[1]);
  cfmr(u[2], cr, h[0] * h[2]);
  cfmr(u[3], cr, h[1] * h[1]);
  cfmr(u[4], cr, h[1] * h[2]);
  cfmr(u[5], cr, h[2] * h[2]);
}

// Adds w * (static Kelvin U*, T*) into real accumulators (9 + 9 entries),
// evaluated in R (FP64, or FP32 for the complex64 operator).
template <typename R>
__device__ __forceinline__ void add_kelvin(R* us, R* ts, R rx, R ry, R rz, R nx, R ny, R nz, R w,
                                           const KParams<double>& P) {
  R r2 = rx * rx + ry * ry + rz * rz;
  R r = sqrt(r2);
  R ir = R(1) / r;
  R h[3] = {rx * ir, ry * ir, rz * ir};
  R n[3] = {nx, ny, nz};
  R rn = h[0] * nx + h[1] * ny + h[2] * nz;
  R nu = R(P.nu);
  R su = R(P.kel_u) * ir * w;
  R st = -R(P.kel_t) * ir * ir * w;
  R a34 = R(3) - R(4) * nu, a12 = R(1) - R(2) * nu;
#pragma unroll
  for (int i = 0; i < 3; ++i) {
#pragma unroll
    for (int j = 0; j < 3; ++j) {
      us[3 * i + j] += su * ((i == j ? a34 : R(0)) + h[i] * h[j]);
      R v = rn * ((i == j ? a12 : R(0)) + R(3) * h[i] * h[j]) - a12 * (h[i] * n[j] - h[j] * n[i]);
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

// Collapsed q x q rule on a triangle given by p0-relative offset o0 (the
// position of p0 relative to the collocation point) and edges e1, e2.
template <typename R, int Q, bool FULL = true>
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
      accumulate_point<R, FULL>(acc, rx, ry, rz, n[0], n[1], n[2], w, P);
    }
  }
}

}  // namespace bem
