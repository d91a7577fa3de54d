// Shared device/host definitions of the GB300 EWM elastodynamic BEM library.
//
// Complex types, status codes, the material/frequency parameter block passed
// to every kernel-evaluation kernel, and the quadrature constants (band
// thresholds and rule sizes of the element integration rule).
#pragma once

#include <cuda_runtime.h>
#include <cstdint>
#include <cmath>

#include "../../include/bem.h"

#define BEM_HD __host__ __device__ __forceinline__

namespace bem {

template <typename R> struct alignas(2 * sizeof(R)) cplx {
  R re, im;
};
using c64 = cplx<float>;
using c128 = cplx<double>;

template <typename R> BEM_HD cplx<R> mk(R a, R b) { return cplx<R>{a, b}; }
template <typename R> BEM_HD cplx<R> operator+(cplx<R> a, cplx<R> b) { return {a.re + b.re, a.im + b.im}; }
template <typename R> BEM_HD cplx<R> operator-(cplx<R> a, cplx<R> b) { return {a.re - b.re, a.im - b.im}; }
template <typename R> BEM_HD cplx<R> operator-(cplx<R> a) { return {-a.re, -a.im}; }
template <typename R> BEM_HD cplx<R> operator*(cplx<R> a, cplx<R> b) {
  return {a.re * b.re - a.im * b.im, a.re * b.im + a.im * b.re};
}
template <typename R> BEM_HD cplx<R> operator*(cplx<R> a, R b) { return {a.re * b, a.im * b}; }
template <typename R> BEM_HD cplx<R> operator*(R b, cplx<R> a) { return {a.re * b, a.im * b}; }
template <typename R> BEM_HD cplx<R> operator+(cplx<R> a, R b) { return {a.re + b, a.im}; }
template <typename R> BEM_HD cplx<R> conj(cplx<R> a) { return {a.re, -a.im}; }
template <typename R> BEM_HD R abs2(cplx<R> a) { return a.re * a.re + a.im * a.im; }
template <typename R> BEM_HD cplx<R> inv(cplx<R> a) {
  R d = R(1) / (a.re * a.re + a.im * a.im);
  return {a.re * d, -a.im * d};
}
// a += b * c (complex fused)
template <typename R> BEM_HD void cfma(cplx<R>& a, cplx<R> b, cplx<R> c) {
  a.re = fma(b.re, c.re, fma(-b.im, c.im, a.re));
  a.im = fma(b.re, c.im, fma(b.im, c.re, a.im));
}
// a += b * r (complex times real)
template <typename R> BEM_HD void cfmr(cplx<R>& a, cplx<R> b, R r) {
  a.re = fma(b.re, r, a.re);
  a.im = fma(b.im, r, a.im);
}

template <typename To, typename From> BEM_HD cplx<To> ccast(cplx<From> a) {
  return {To(a.re), To(a.im)};
}

__device__ __forceinline__ void sincos_r(float x, float* s, float* c) { sincosf(x, s, c); }
__device__ __forceinline__ void sincos_r(double x, double* s, double* c) { sincos(x, s, c); }

// exp(-z) for complex z
__device__ __forceinline__ cplx<float> cexp_neg(cplx<float> z) {
  float sn, cs;
  sincosf(z.im, &sn, &cs);
  float m = expf(-z.re);
  return {m * cs, -m * sn};
}
__device__ __forceinline__ cplx<double> cexp_neg(cplx<double> z) {
  double sn, cs;
  sincos(z.im, &sn, &cs);
  double m = exp(-z.re);
  return {m * cs, -m * sn};
}

// ---------------------------------------------------------------------------
// Element integration rule (identical specification to the CPU oracle):
//   band from rho2 = |c_i - c_e|^2 / h_e^2
//   SELF  : polar about c_i; static parts closed form (16 angles / triangle),
//           remainders 8 angles x 6 radii / triangle            (FP64)
//   NEAR  : rho2 < 2.2; static on 64 children x 4x4 collapsed, remainder 4x4 (FP64)
//   Q4    : rho2 < 9.7  collapsed 4x4                           (FP32)
//   Q2    : rho2 < 63.3 collapsed 2x2                           (FP32)
//   Q1    : centroid                                            (FP32)
// ---------------------------------------------------------------------------
constexpr double RHO2_NEAR = 2.2;
constexpr double RHO2_Q4 = 9.7;
constexpr double RHO2_Q2 = 63.3;
constexpr int SELF_NT_STATIC = 16;
constexpr int SELF_NT = 8;
constexpr int SELF_NR = 6;
constexpr int NEAR_LEVELS = 3;
constexpr int NEAR_Q = 4;
constexpr int NEAR_Q_REM = 4;
constexpr int BAND_SELF = 0, BAND_NEAR = 1, BAND_Q4 = 2, BAND_Q2 = 3, BAND_Q1 = 4;

constexpr int GL_MAX = 16;        // Gauss-Legendre tables for q = 1..16

// Radius (in |z_s|) below which the radial functions use Taylor series.
constexpr double Z_SERIES = 1.0;
constexpr int SERIES_M_F32 = 12;  // terms used in FP32 (1/13! < 2e-10 at |z| = 1)
constexpr int SERIES_M_F64 = 20;  // terms used in FP64 (1/21! < 2e-20)
constexpr int SER_MAX = 21;

// Material and frequency parameters of one kernel evaluation (Sec. 2.1).
//
// With z = s r / c_s and gamma = c_s / c_p (so z_p = gamma z), the radial
// functions enter U and T only through
//   Phi = r phi, Psi = r psi,
//   A = r^2 (phi' - psi/r)            = r Phi' - Phi - Psi,
//   B = r^2 (4 psi/r - 2 psi')        = 2 (3 Psi - r Psi'),
//   C = r^2 (k2 (phi' - psi' - 2psi/r) - 2 (phi' - psi' - psi/r))
//     = k2 (r Phi' - Phi - r Psi' - Psi) - 2 (r Phi' - Phi - r Psi').
// Each is an entire function of z with Taylor coefficients (m-th):
//   phi_m = a_m - beta2 gamma^m b_m,  psi_m = c_m (1 - beta2 gamma^m),
//   A_m = (m-1) phi_m - psi_m,  B_m = 2 (3-m) psi_m,
//   C_m = k2 ((m-1) phi_m - (m+1) psi_m) - 2 ((m-1) phi_m - m psi_m),
// where a_m, b_m, c_m are those of A(z) - 1/z^2, B(z) - 1/z^2, C(z) - 3/z^2
// (exponential series). The m = 0 terms are the static (Kelvin) values; the
// dynamic remainder is the sum over m >= 1 (m >= 2 for A, C), free of
// cancellation.
template <typename R> struct KParams {
  cplx<R> s;      // complex frequency s = eta + i omega_k
  cplx<R> ks;     // s / c_s  (= d z_s / d r)
  cplx<R> kp;     // s / c_p
  R beta2;        // (c_s / c_p)^2
  R k2;           // (c_p / c_s)^2
  R u_scale;      // 1 / (4 pi mu)
  R t_scale;      // 1 / (4 pi)
  R nu;           // Poisson ratio (Kelvin parts)
  R kel_u;        // 1 / (16 pi mu (1 - nu))
  R kel_t;        // 1 / (8 pi (1 - nu))
  R ser[5][SER_MAX];  // Taylor coefficients of Phi, Psi, A, B, C (index m)
};
// Device-side tables (one copy per translation unit that includes
// bem_kernels.cuh; each is filled by its own upload function).
struct RuleTables {
  double gl_x[GL_MAX + 1][GL_MAX];  // nodes on [0, 1]
  double gl_w[GL_MAX + 1][GL_MAX];
  // FP32 copies for the FP32 evaluation path (no FP64 conversions in inner loops)
  float gl_xf[GL_MAX + 1][GL_MAX];
  float gl_wf[GL_MAX + 1][GL_MAX];
};

}  // namespace bem

#define BEM_CUDA_TRY(expr)                                                       \
  do {                                                                           \
    cudaError_t _e = (expr);                                                     \
    if (_e != cudaSuccess) return ::bem::fail_cuda(ctx, _e, #expr, __FILE__, __LINE__); \
  } while (0)
