// Interior field by the representation formula (Somigliana's identity, the
// interior form of Eq. bie with c = I):
//
//   u_i(x) = sum_e [ int_e U_ij(x, y) dy t_j(e) - int_e T_ij(x, y) dy u_j(e) ]
//
// with u and t constant per element: on Gamma_sigma elements t is the
// prescribed traction and u the solved displacement, on Gamma_u elements the
// reverse (Sec. 2.1, Eq. Aa_b). Each (point, element) pair takes the rule of
// its distance band, as the operator entries do; in the NEAR band the point
// is off the boundary, so the full kernel is integrated on the subdivided
// 1,024-point rule (three midpoint levels x collapsed 4 x 4).
//
//   k_interior       one warp per evaluation point; pass 1 over the elements
//                    (lanes over elements) takes the regular bands, pass 2
//                    takes each NEAR element with the whole warp (lanes over
//                    its 1,024 points). Every lane accumulates its share of
//                    the three displacement components directly (the formula
//                    is linear in the element integrals), then one warp sum.
//                    Geometry relative to the point in FP64, kernel
//                    evaluation in R (FP32 on the mixed path), sums in FP64.
//   k_offset_points  the six points x +- h e_a around each point (strain)
//   k_strain         eps = sym(grad u) by central differences of those
#include "bem_internal.h"
#include "bem_kernels.cuh"
#include "bem_launch.h"

namespace bem {

cudaError_t upload_rules_interior(const RuleTables& t, cudaStream_t st) {
  return cudaMemcpyToSymbolAsync(c_rules, &t, sizeof(RuleTables), 0, cudaMemcpyHostToDevice, st);
}

namespace {

constexpr int INTERIOR_WARPS = 4;

// out += U t - T u for one element's accumulated integrals (FP64 sums)
template <typename R>
__device__ __forceinline__ void add_contribution(cplx<double> out[3], const UTAcc<R>& acc, const cplx<double> u[3],
                                                 const cplx<double> t[3]) {
#pragma unroll
  for (int i = 0; i < 3; ++i) {
#pragma unroll
    for (int j = 0; j < 3; ++j) {
      const cplx<R> Uij = acc.U(i, j);
      const cplx<R> Tij = acc.t[3 * i + j];
      const double ur = Uij.re, ui = Uij.im, tr = Tij.re, ti = Tij.im;
      out[i].re += ur * t[j].re - ui * t[j].im - (tr * u[j].re - ti * u[j].im);
      out[i].im += ur * t[j].im + ui * t[j].re - (tr * u[j].im + ti * u[j].re);
    }
  }
}

// u (displacement) and t (traction) of element e: the solved values a_e and
// the prescribed ones pattern_e * pk, placed by the element's condition
__device__ __forceinline__ void element_data(int e, const signed char* __restrict__ bc, const c128* __restrict__ a,
                                             const double* __restrict__ pattern, c128 pk, cplx<double> u[3],
                                             cplx<double> t[3]) {
  const bool fixed = bc[e] == BEM_BC_DISPLACEMENT;
#pragma unroll
  for (int j = 0; j < 3; ++j) {
    const double p = pattern[3LL * e + j];
    const cplx<double> known{p * pk.re, p * pk.im};
    const cplx<double> sol{a[3LL * e + j].re, a[3LL * e + j].im};
    u[j] = fixed ? known : sol;
    t[j] = fixed ? sol : known;
  }
}

template <typename R>
__global__ void __launch_bounds__(32 * INTERIOR_WARPS) k_interior(
    const double* __restrict__ pts, int npts, const ElemD* __restrict__ ed, int ne,
    const signed char* __restrict__ bc, const c128* __restrict__ a, const double* __restrict__ pattern, c128 pk,
    KParams<R> P, c128* __restrict__ out) {
  const int warp = blockIdx.x * INTERIOR_WARPS + (threadIdx.x >> 5);
  const int lane = threadIdx.x & 31;
  if (warp >= npts) return;  // whole warps only: the shuffles below see full warps
  const double x[3] = {pts[3LL * warp], pts[3LL * warp + 1], pts[3LL * warp + 2]};
  cplx<double> acc_out[3] = {{0, 0}, {0, 0}, {0, 0}};
  cplx<double> u[3], t[3];
  // pass 1: regular bands, one element per lane
  for (int e = lane; e < ne; e += 32) {
    const ElemD& E = ed[e];
    double d2 = 0;
#pragma unroll
    for (int k = 0; k < 3; ++k) d2 += (E.c[k] - x[k]) * (E.c[k] - x[k]);
    const int band = band_of<double>(d2, E.h2);
    if (band == BAND_NEAR) continue;
    UTAcc<R> acc;
    acc.zero();
    const R n0 = R(E.n[0]), n1 = R(E.n[1]), n2 = R(E.n[2]);
    if (band == BAND_Q1) {
      accumulate_point<R>(acc, R(E.c[0] - x[0]), R(E.c[1] - x[1]), R(E.c[2] - x[2]), n0, n1, n2,
                          R(0.5 * E.area2), P);
    } else {
      const int Q = band == BAND_Q4 ? 4 : 2;
      const R o0[3] = {R(E.p0[0] - x[0]), R(E.p0[1] - x[1]), R(E.p0[2] - x[2])};
      const R e1[3] = {R(E.p1[0] - E.p0[0]), R(E.p1[1] - E.p0[1]), R(E.p1[2] - E.p0[2])};
      const R e2[3] = {R(E.p2[0] - E.p0[0]), R(E.p2[1] - E.p0[1]), R(E.p2[2] - E.p0[2])};
      const R area2 = R(E.area2);
#pragma unroll 1
      for (int p = 0; p < Q * Q; ++p) {
        const int ia = p / Q, ib = p - ia * Q;
        const R uu = gl_x<R>(Q, ia);
        const R omu = R(1) - uu;
        const R vv = omu * gl_x<R>(Q, ib);
        const R w = area2 * gl_w<R>(Q, ia) * gl_w<R>(Q, ib) * omu;
        accumulate_point<R>(acc, o0[0] + uu * e1[0] + vv * e2[0], o0[1] + uu * e1[1] + vv * e2[1],
                            o0[2] + uu * e1[2] + vv * e2[2], n0, n1, n2, w, P);
      }
    }
    element_data(e, bc, a, pattern, pk, u, t);
    add_contribution<R>(acc_out, acc, u, t);
  }
  // pass 2: NEAR elements, the whole warp over each one's 1,024 points
  for (int e0 = 0; e0 < ne; e0 += 32) {
    const int e = e0 + lane;
    bool near = false;
    if (e < ne) {
      const ElemD& E = ed[e];
      double d2 = 0;
#pragma unroll
      for (int k = 0; k < 3; ++k) d2 += (E.c[k] - x[k]) * (E.c[k] - x[k]);
      near = band_of<double>(d2, E.h2) == BAND_NEAR;
    }
    unsigned m = __ballot_sync(0xffffffffu, near);
    while (m) {
      const int src = __ffs(m) - 1;
      m &= m - 1;
      const int en = e0 + src;
      const ElemD& E = ed[en];
      UTAcc<R> acc;
      acc.zero();
      const R n0 = R(E.n[0]), n1 = R(E.n[1]), n2 = R(E.n[2]);
#pragma unroll 1
      for (int q = lane; q < 64 * NEAR_Q * NEAR_Q; q += 32) {
        const int child = q / (NEAR_Q * NEAR_Q), pt = q % (NEAR_Q * NEAR_Q);
        R va[3], vb[3], vc[3];
#pragma unroll
        for (int k = 0; k < 3; ++k) {
          va[k] = R(E.p0[k] - x[k]);
          vb[k] = R(E.p1[k] - x[k]);
          vc[k] = R(E.p2[k] - x[k]);
        }
        // child index in base 4, most significant digit = first level
#pragma unroll
        for (int l = NEAR_LEVELS - 1; l >= 0; --l) {
          const int dig = (child >> (2 * l)) & 3;
#pragma unroll
          for (int k = 0; k < 3; ++k) {
            const R mab = R(0.5) * (va[k] + vb[k]), mbc = R(0.5) * (vb[k] + vc[k]), mca = R(0.5) * (vc[k] + va[k]);
            R na, nb, nc;
            switch (dig) {
              case 0: na = va[k]; nb = mab; nc = mca; break;
              case 1: na = mab; nb = vb[k]; nc = mbc; break;
              case 2: na = mca; nb = mbc; nc = vc[k]; break;
              default: na = mbc; nb = mca; nc = mab; break;
            }
            va[k] = na;
            vb[k] = nb;
            vc[k] = nc;
          }
        }
        R e1[3], e2[3];
#pragma unroll
        for (int k = 0; k < 3; ++k) {
          e1[k] = vb[k] - va[k];
          e2[k] = vc[k] - va[k];
        }
        const R cr0 = e1[1] * e2[2] - e1[2] * e2[1], cr1 = e1[2] * e2[0] - e1[0] * e2[2],
                cr2 = e1[0] * e2[1] - e1[1] * e2[0];
        const R area2 = sqrt(cr0 * cr0 + cr1 * cr1 + cr2 * cr2);
        const int ia = pt / NEAR_Q, ib = pt % NEAR_Q;
        const R uu = gl_x<R>(NEAR_Q, ia), vv = (R(1) - uu) * gl_x<R>(NEAR_Q, ib);
        const R w = area2 * gl_w<R>(NEAR_Q, ia) * gl_w<R>(NEAR_Q, ib) * (R(1) - uu);
        accumulate_point<R>(acc, va[0] + uu * e1[0] + vv * e2[0], va[1] + uu * e1[1] + vv * e2[1],
                            va[2] + uu * e1[2] + vv * e2[2], n0, n1, n2, w, P);
      }
      element_data(en, bc, a, pattern, pk, u, t);
      add_contribution<R>(acc_out, acc, u, t);
    }
  }
#pragma unroll
  for (int i = 0; i < 3; ++i) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      acc_out[i].re += __shfl_xor_sync(0xffffffffu, acc_out[i].re, o);
      acc_out[i].im += __shfl_xor_sync(0xffffffffu, acc_out[i].im, o);
    }
  }
  if (lane == 0)
    for (int i = 0; i < 3; ++i) out[3LL * warp + i] = c128{acc_out[i].re, acc_out[i].im};
}

// points (npts x 3) -> 6 npts points, point p's six at 6p + 2a (+h e_a), 6p + 2a + 1 (-h e_a)
__global__ void k_offset_points(const double* __restrict__ pts, int npts, double h, double* __restrict__ out) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= 6 * npts) return;
  const int p = i / 6, a = (i % 6) / 2;
  const double sg = (i & 1) ? -1.0 : 1.0;
#pragma unroll
  for (int k = 0; k < 3; ++k) out[3LL * i + k] = pts[3LL * p + k] + (k == a ? sg * h : 0.0);
}

// displacements at the offset points (6 npts x 3) -> strain (npts x 6:
// xx, yy, zz, xy, yz, xz; tensor components) by central differences
__global__ void k_strain(const c128* __restrict__ uoff, int npts, double h, c128* __restrict__ eps) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= npts) return;
  // g[i][a] = d u_i / d x_a
  c128 g[3][3];
  const double s = 0.5 / h;
  for (int a = 0; a < 3; ++a)
    for (int i = 0; i < 3; ++i) {
      const c128 up = uoff[3LL * (6LL * p + 2 * a) + i], um = uoff[3LL * (6LL * p + 2 * a + 1) + i];
      g[i][a] = c128{(up.re - um.re) * s, (up.im - um.im) * s};
    }
  const int ii[6] = {0, 1, 2, 0, 1, 0}, jj[6] = {0, 1, 2, 1, 2, 2};
  for (int c = 0; c < 6; ++c) {
    const c128 x = g[ii[c]][jj[c]], y = g[jj[c]][ii[c]];
    eps[6LL * p + c] = c128{0.5 * (x.re + y.re), 0.5 * (x.im + y.im)};
  }
}

}  // namespace

template <typename R>
void launch_interior(const double* pts, int npts, const ElemD* ed, int ne, const signed char* bc, const c128* a,
                     const double* pattern, c128 pk, const KParams<R>& P, c128* out, cudaStream_t st) {
  if (!count_if(npts > 0)) return;
  const int grid = (npts + INTERIOR_WARPS - 1) / INTERIOR_WARPS;
  k_interior<R><<<grid, 32 * INTERIOR_WARPS, 0, st>>>(pts, npts, ed, ne, bc, a, pattern, pk, P, out);
}

void launch_offset_points(const double* pts, int npts, double h, double* out, cudaStream_t st) {
  if (!count_if(npts > 0)) return;
  k_offset_points<<<(6 * npts + 127) / 128, 128, 0, st>>>(pts, npts, h, out);
}

void launch_strain(const c128* uoff, int npts, double h, c128* eps, cudaStream_t st) {
  if (!count_if(npts > 0)) return;
  k_strain<<<(npts + 127) / 128, 128, 0, st>>>(uoff, npts, h, eps);
}

template void launch_interior<float>(const double*, int, const ElemD*, int, const signed char*, const c128*,
                                     const double*, c128, const KParams<float>&, c128*, cudaStream_t);
template void launch_interior<double>(const double*, int, const ElemD*, int, const signed char*, const c128*,
                                      const double*, c128, const KParams<double>&, c128*, cudaStream_t);

}  // namespace bem
