// Operator assembly kernels (Sec. 2.1: collocation with constant triangles,
// Eqs. Uij, Tij, Gikj, Tu_Ut, Aa_b).
//
//   k_centroids      element centroids and sizes (caller order)
//   k_geometry       tree-ordered FP32/FP64 element records
//   k_sing_count /
//   k_sing_fill      singular (self) and near-singular pairs of near blocks
//   k_static         frequency-independent Kelvin parts of those pairs (FP64)
//   k_near_regular   regular near-field entries (FP32 mixed / FP64 plain)
//   k_sing           singular + near-singular entries: FP64 remainder plus
//                    static part, block-Jacobi inverses, their RHS share
//   k_rhs            b = B(s) pattern over regular pairs, on the fly
//   k_aca            adaptive cross approximation of admissible blocks
#include "bem_internal.h"
#include "bem_kernels.cuh"
#include "bem_launch.h"

namespace bem {

cudaError_t upload_rules_assemble(const RuleTables& t, cudaStream_t st) {
  return cudaMemcpyToSymbolAsync(c_rules, &t, sizeof(RuleTables), 0, cudaMemcpyHostToDevice, st);
}

// ---------------------------------------------------------------------------
// geometry
// ---------------------------------------------------------------------------
__global__ void k_centroids(const double* __restrict__ xyz, long long nv, const int* __restrict__ tri,
                            int ne, double* __restrict__ cen, double* __restrict__ h,
                            int* __restrict__ bad) {
  int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= ne) return;
  int v[3] = {tri[3 * e], tri[3 * e + 1], tri[3 * e + 2]};
  for (int k = 0; k < 3; ++k)
    if (v[k] < 0 || v[k] >= nv) {
      atomicExch(bad, 1);
      return;
    }
  double p[3][3];
  for (int k = 0; k < 3; ++k)
    for (int a = 0; a < 3; ++a) p[k][a] = xyz[3 * (long long)v[k] + a];
  double e1[3], e2[3], e3[3];
  for (int a = 0; a < 3; ++a) {
    e1[a] = p[1][a] - p[0][a];
    e2[a] = p[2][a] - p[0][a];
    e3[a] = p[2][a] - p[1][a];
  }
  double cx = e1[1] * e2[2] - e1[2] * e2[1];
  double cy = e1[2] * e2[0] - e1[0] * e2[2];
  double cz = e1[0] * e2[1] - e1[1] * e2[0];
  double a2 = sqrt(cx * cx + cy * cy + cz * cz);
  double l1 = e1[0] * e1[0] + e1[1] * e1[1] + e1[2] * e1[2];
  double l2 = e2[0] * e2[0] + e2[1] * e2[1] + e2[2] * e2[2];
  double l3 = e3[0] * e3[0] + e3[1] * e3[1] + e3[2] * e3[2];
  double hm = sqrt(fmax(l1, fmax(l2, l3)));
  if (!(a2 > 1e-12 * hm * hm) || !(hm > 0)) atomicExch(bad, 2);
  for (int a = 0; a < 3; ++a) cen[3 * e + a] = (p[0][a] + p[1][a] + p[2][a]) / 3.0;
  h[e] = hm;
}

__global__ void k_geometry(const double* __restrict__ xyz, const int* __restrict__ tri,
                           const int* __restrict__ perm, const signed char* __restrict__ bc_in,
                           int ne, ElemF* __restrict__ ef, ElemD* __restrict__ ed,
                           signed char* __restrict__ bc) {
  int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= ne) return;
  int e = perm[k];
  double p[3][3];
  for (int v = 0; v < 3; ++v)
    for (int a = 0; a < 3; ++a) p[v][a] = xyz[3 * (long long)tri[3 * e + v] + a];
  ElemD D;
  ElemF F;
  double e1[3], e2[3], e3[3];
  for (int a = 0; a < 3; ++a) {
    D.c[a] = (p[0][a] + p[1][a] + p[2][a]) / 3.0;
    D.p0[a] = p[0][a];
    D.p1[a] = p[1][a];
    D.p2[a] = p[2][a];
    e1[a] = p[1][a] - p[0][a];
    e2[a] = p[2][a] - p[0][a];
    e3[a] = p[2][a] - p[1][a];
  }
  double cr[3] = {e1[1] * e2[2] - e1[2] * e2[1], e1[2] * e2[0] - e1[0] * e2[2],
                  e1[0] * e2[1] - e1[1] * e2[0]};
  double a2 = sqrt(cr[0] * cr[0] + cr[1] * cr[1] + cr[2] * cr[2]);
  double l1 = e1[0] * e1[0] + e1[1] * e1[1] + e1[2] * e1[2];
  double l2 = e2[0] * e2[0] + e2[1] * e2[1] + e2[2] * e2[2];
  double l3 = e3[0] * e3[0] + e3[1] * e3[1] + e3[2] * e3[2];
  D.area2 = a2;
  D.h2 = fmax(l1, fmax(l2, l3));
  for (int a = 0; a < 3; ++a) {
    D.n[a] = cr[a] / a2;
    float hi = (float)D.c[a];
    F.c_hi[a] = hi;
    F.c_lo[a] = (float)(D.c[a] - (double)hi);
    F.o0[a] = (float)(p[0][a] - D.c[a]);
    F.e1[a] = (float)e1[a];
    F.e2[a] = (float)e2[a];
    F.n[a] = (float)D.n[a];
  }
  F.area2 = (float)a2;
  F.h2 = (float)D.h2;
  ed[k] = D;
  ef[k] = F;
  bc[k] = bc_in[e];
}

// ---------------------------------------------------------------------------
// pair geometry helpers: d = c_e - c_i, o0 = p0_e - c_i (offsets of the
// integration element relative to the collocation point)
// ---------------------------------------------------------------------------
template <typename R> struct PairGeo {
  R d[3], o0[3], e1[3], e2[3], n[3];
  R area2, he2, d2;
};

__device__ __forceinline__ void pair_geo(const ElemF* ef, const ElemD* ed, int i, int e,
                                         PairGeo<float>& g, int& band) {
  const ElemF& I = ef[i];
  const ElemF& E = ef[e];
  float d2 = 0.f;
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    g.d[a] = (E.c_hi[a] - I.c_hi[a]) + (E.c_lo[a] - I.c_lo[a]);
    d2 += g.d[a] * g.d[a];
    g.o0[a] = g.d[a] + E.o0[a];
    g.e1[a] = E.e1[a];
    g.e2[a] = E.e2[a];
    g.n[a] = E.n[a];
  }
  g.area2 = E.area2;
  g.he2 = E.h2;
  g.d2 = d2;
  if (i == e) {
    band = BAND_SELF;
    return;
  }
  // exact-consistent band: FP64 decision near a threshold
  const float thr[3] = {float(RHO2_NEAR), float(RHO2_Q4), float(RHO2_Q2)};
  bool close = false;
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    float t = thr[k] * g.he2;
    close |= fabsf(d2 - t) <= 1e-4f * t;
  }
  if (close) {
    const ElemD& Id = ed[i];
    const ElemD& Ed = ed[e];
    double dd = 0;
    for (int a = 0; a < 3; ++a) dd += (Ed.c[a] - Id.c[a]) * (Ed.c[a] - Id.c[a]);
    band = band_of<double>(dd, Ed.h2);
  } else {
    band = band_of<float>(d2, g.he2);
  }
}

__device__ __forceinline__ void pair_geo(const ElemF* ef, const ElemD* ed, int i, int e,
                                         PairGeo<double>& g, int& band) {
  const ElemD& I = ed[i];
  const ElemD& E = ed[e];
  double d2 = 0;
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    g.d[a] = E.c[a] - I.c[a];
    d2 += g.d[a] * g.d[a];
    g.o0[a] = E.p0[a] - I.c[a];
    g.e1[a] = E.p1[a] - E.p0[a];
    g.e2[a] = E.p2[a] - E.p0[a];
    g.n[a] = E.n[a];
  }
  g.area2 = E.area2;
  g.he2 = E.h2;
  g.d2 = d2;
  band = (i == e) ? BAND_SELF : band_of<double>(d2, E.h2);
}

// Regular-band integral of a pair (bands Q4, Q2, Q1): one loop over the
// points of the band's rule, so the point evaluator is inlined once (keeps
// the kernels' instruction footprint small).
template <typename R>
__device__ __forceinline__ void regular_pair(UTAcc<R>& acc, const PairGeo<R>& g, int band,
                                             const KParams<R>& P) {
  acc.zero();
  const int Q = band == BAND_Q4 ? 4 : (band == BAND_Q2 ? 2 : 1);
#pragma unroll 1
  for (int p = 0; p < Q * Q; ++p) {
    R rx, ry, rz, w;
    if (Q == 1) {
      rx = g.d[0];
      ry = g.d[1];
      rz = g.d[2];
      w = R(0.5) * g.area2;
    } else {
      const int a = p / Q, b = p - (p / Q) * Q;
      const R u = gl_x<R>(Q, a);
      const R omu = R(1) - u;
      const R v = omu * gl_x<R>(Q, b);
      w = g.area2 * gl_w<R>(Q, a) * gl_w<R>(Q, b) * omu;
      rx = g.o0[0] + u * g.e1[0] + v * g.e2[0];
      ry = g.o0[1] + u * g.e1[1] + v * g.e2[1];
      rz = g.o0[2] + u * g.e1[2] + v * g.e2[2];
    }
    accumulate_point<R>(acc, rx, ry, rz, g.n[0], g.n[1], g.n[2], w, P);
  }
}

template <typename Op, typename R> __device__ __forceinline__ Op to_op(cplx<R> v) {
  Op o;
  o.re = decltype(o.re)(v.re);
  o.im = decltype(o.im)(v.im);
  return o;
}

// ---------------------------------------------------------------------------
// singular pair detection (two passes for a deterministic list)
// ---------------------------------------------------------------------------
__device__ __forceinline__ bool is_sing(const ElemD* ed, int i, int e) {
  if (i == e) return true;
  const ElemD& I = ed[i];
  const ElemD& E = ed[e];
  double dd = 0;
  for (int a = 0; a < 3; ++a) dd += (E.c[a] - I.c[a]) * (E.c[a] - I.c[a]);
  return dd < RHO2_NEAR * E.h2;
}

__global__ void k_sing_count(const NearBlk* __restrict__ blks, const ElemD* __restrict__ ed,
                             int* __restrict__ count) {
  NearBlk B = blks[blockIdx.x];
  int np = B.nr * B.nc;
  int c = 0;
  for (int p = threadIdx.x; p < np; p += blockDim.x) {
    int i = B.r0 + p % B.nr, e = B.c0 + p / B.nr;
    c += is_sing(ed, i, e) ? 1 : 0;
  }
  c = __reduce_add_sync(0xffffffffu, c);
  __shared__ int s[32];
  if ((threadIdx.x & 31) == 0) s[threadIdx.x >> 5] = c;
  __syncthreads();
  if (threadIdx.x == 0) {
    int t = 0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += s[w];
    count[blockIdx.x] = t;
  }
}

__global__ void k_sing_fill(const NearBlk* __restrict__ blks, const ElemD* __restrict__ ed,
                            const int* __restrict__ offs, SingPair* __restrict__ out) {
  NearBlk B = blks[blockIdx.x];
  int np = B.nr * B.nc;
  int ld = B.ld;
  __shared__ int warp_tot[32];
  __shared__ int base;
  if (threadIdx.x == 0) base = offs[blockIdx.x];
  __syncthreads();
  int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
  for (int p0 = 0; p0 < np; p0 += blockDim.x) {
    int p = p0 + threadIdx.x;
    bool f = false;
    int i = 0, e = 0;
    if (p < np) {
      i = B.r0 + p % B.nr;
      e = B.c0 + p / B.nr;
      f = is_sing(ed, i, e);
    }
    unsigned m = __ballot_sync(0xffffffffu, f);
    if (lane == 0) warp_tot[wid] = __popc(m);
    __syncthreads();
    int before = 0, tot = 0;
    for (int w = 0; w < nw; ++w) {
      if (w < wid) before += warp_tot[w];
      tot += warp_tot[w];
    }
    if (f) {
      int pos = base + before + __popc(m & ((1u << lane) - 1));
      SingPair sp;
      sp.i = i;
      sp.e = e;
      sp.entry = B.off + (long long)(3 * (e - B.c0)) * ld + 3 * (i - B.r0);
      sp.ld = ld;
      sp.self = (i == e);
      out[pos] = sp;
    }
    __syncthreads();
    if (threadIdx.x == 0) base += tot;
    __syncthreads();
  }
}

// ---------------------------------------------------------------------------
// static Kelvin parts (FP64, once per mesh): one warp per pair
// ---------------------------------------------------------------------------
__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}
__device__ __forceinline__ float warp_sumf(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Polar parameters of the triangle (c, pa, pb) about c (normal n).
struct PolarSub {
  double d, fh[3], gh[3], tha, dth;
};
__device__ __forceinline__ PolarSub polar_sub(const double* c, const double* pa, const double* pb,
                                              const double* n) {
  PolarSub S;
  double t[3], cpa[3];
  for (int a = 0; a < 3; ++a) {
    t[a] = pb[a] - pa[a];
    cpa[a] = c[a] - pa[a];
  }
  double lam = (cpa[0] * t[0] + cpa[1] * t[1] + cpa[2] * t[2]) / (t[0] * t[0] + t[1] * t[1] + t[2] * t[2]);
  double fv[3];
  for (int a = 0; a < 3; ++a) fv[a] = pa[a] + lam * t[a] - c[a];
  S.d = sqrt(fv[0] * fv[0] + fv[1] * fv[1] + fv[2] * fv[2]);
  for (int a = 0; a < 3; ++a) S.fh[a] = fv[a] / S.d;
  S.gh[0] = n[1] * S.fh[2] - n[2] * S.fh[1];
  S.gh[1] = n[2] * S.fh[0] - n[0] * S.fh[2];
  S.gh[2] = n[0] * S.fh[1] - n[1] * S.fh[0];
  double va[3], vb[3];
  for (int a = 0; a < 3; ++a) {
    va[a] = pa[a] - c[a];
    vb[a] = pb[a] - c[a];
  }
  double tha = atan2(va[0] * S.gh[0] + va[1] * S.gh[1] + va[2] * S.gh[2],
                     va[0] * S.fh[0] + va[1] * S.fh[1] + va[2] * S.fh[2]);
  double thb = atan2(vb[0] * S.gh[0] + vb[1] * S.gh[1] + vb[2] * S.gh[2],
                     vb[0] * S.fh[0] + vb[1] * S.fh[1] + vb[2] * S.fh[2]);
  S.tha = tha;
  S.dth = thb - tha;
  return S;
}

__device__ __forceinline__ const double* vtx(const ElemD& E, int k) {
  return k == 0 ? E.p0 : (k == 1 ? E.p1 : E.p2);
}

// Static (Kelvin) parts of the singular and near-singular pairs, once per
// mesh: the self rule in FP64; the near-singular rule (64 children x 4 x 4)
// in RN (FP64 for the complex128 operator; FP32 for the complex64 operator,
// with the geometry taken relative to the collocation point in FP64 first).
template <typename RN>
__global__ void k_static(const SingPair* __restrict__ pairs, int npairs, const ElemD* __restrict__ ed,
                         KParams<double> P, double* __restrict__ out) {
  int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  int lane = threadIdx.x & 31;
  if (warp >= npairs) return;
  SingPair sp = pairs[warp];
  const ElemD& E = ed[sp.e];
  const ElemD& I = ed[sp.i];
  double us[9], ts[9];
  for (int k = 0; k < 9; ++k) us[k] = ts[k] = 0.0;
  if (sp.self) {
    // 3 triangles x 16 angles; closed-form ray integrals
    double nu = P.nu;
    double a34 = 3.0 - 4.0 * nu, a12 = 1.0 - 2.0 * nu;
    for (int q = lane; q < 3 * SELF_NT_STATIC; q += 32) {
      int sub = q / SELF_NT_STATIC, m = q % SELF_NT_STATIC;
      PolarSub S = polar_sub(E.c, vtx(E, sub), vtx(E, (sub + 1) % 3), E.n);
      double th = S.tha + S.dth * gl_x<double>(SELF_NT_STATIC, m);
      double wth = S.dth * gl_w<double>(SELF_NT_STATIC, m);
      double sn, cs;
      sincos(th, &sn, &cs);
      double R = S.d / cs;
      double dir[3];
      for (int a = 0; a < 3; ++a) dir[a] = cs * S.fh[a] + sn * S.gh[a];
      double lr = log(R);
      for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) {
          us[3 * i + j] += wth * R * P.kel_u * ((i == j ? a34 : 0.0) + dir[i] * dir[j]);
          ts[3 * i + j] += wth * lr * a12 * P.kel_t * (dir[i] * E.n[j] - dir[j] * E.n[i]);
        }
    }
  } else {
    // 64 children (3 midpoint-subdivision levels) x collapsed 4x4; vertices
    // relative to the collocation point
    RN usr[9], tsr[9];
    for (int k = 0; k < 9; ++k) usr[k] = tsr[k] = RN(0);
    for (int q = lane; q < 64 * NEAR_Q * NEAR_Q; q += 32) {
      int child = q / (NEAR_Q * NEAR_Q), pt = q % (NEAR_Q * NEAR_Q);
      RN a[3], b[3], c[3];
      for (int k = 0; k < 3; ++k) {
        a[k] = RN(E.p0[k] - I.c[k]);
        b[k] = RN(E.p1[k] - I.c[k]);
        c[k] = RN(E.p2[k] - I.c[k]);
      }
      int digits = child;
      int dig[NEAR_LEVELS];
      for (int l = NEAR_LEVELS - 1; l >= 0; --l) {
        dig[l] = digits & 3;
        digits >>= 2;
      }
      for (int l = 0; l < NEAR_LEVELS; ++l) {
        RN mab[3], mbc[3], mca[3];
        for (int k = 0; k < 3; ++k) {
          mab[k] = RN(0.5) * (a[k] + b[k]);
          mbc[k] = RN(0.5) * (b[k] + c[k]);
          mca[k] = RN(0.5) * (c[k] + a[k]);
        }
        for (int k = 0; k < 3; ++k) {
          RN na, nb, nc;
          switch (dig[l]) {
            case 0: na = a[k]; nb = mab[k]; nc = mca[k]; break;
            case 1: na = mab[k]; nb = b[k]; nc = mbc[k]; break;
            case 2: na = mca[k]; nb = mbc[k]; nc = c[k]; break;
            default: na = mbc[k]; nb = mca[k]; nc = mab[k]; break;
          }
          a[k] = na;
          b[k] = nb;
          c[k] = nc;
        }
      }
      RN e1[3], e2[3];
      for (int k = 0; k < 3; ++k) {
        e1[k] = b[k] - a[k];
        e2[k] = c[k] - a[k];
      }
      RN cr0 = e1[1] * e2[2] - e1[2] * e2[1], cr1 = e1[2] * e2[0] - e1[0] * e2[2],
         cr2 = e1[0] * e2[1] - e1[1] * e2[0];
      RN area2 = sqrt(cr0 * cr0 + cr1 * cr1 + cr2 * cr2);
      int ia = pt / NEAR_Q, ib = pt % NEAR_Q;
      RN u = gl_x<RN>(NEAR_Q, ia), v = (RN(1) - u) * gl_x<RN>(NEAR_Q, ib);
      RN w = area2 * gl_w<RN>(NEAR_Q, ia) * gl_w<RN>(NEAR_Q, ib) * (RN(1) - u);
      RN rv[3];
      for (int k = 0; k < 3; ++k) rv[k] = a[k] + u * e1[k] + v * e2[k];
      add_kelvin<RN>(usr, tsr, rv[0], rv[1], rv[2], RN(E.n[0]), RN(E.n[1]), RN(E.n[2]), w, P);
    }
    for (int k = 0; k < 9; ++k) {
      us[k] = double(usr[k]);
      ts[k] = double(tsr[k]);
    }
  }
  for (int k = 0; k < 9; ++k) {
    us[k] = warp_sum(us[k]);
    ts[k] = warp_sum(ts[k]);
  }
  if (lane == 0) {
    double* o = out + 18 * (long long)warp;
    for (int k = 0; k < 9; ++k) {
      o[k] = us[k];
      o[9 + k] = ts[k];
    }
  }
}

// ---------------------------------------------------------------------------
// geometry of a pair without the band decision
// ---------------------------------------------------------------------------
__device__ __forceinline__ void pair_geom(const ElemF* ef, const ElemD* ed, int i, int e, PairGeo<float>& g) {
  const ElemF& I = ef[i];
  const ElemF& E = ef[e];
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    g.d[a] = (E.c_hi[a] - I.c_hi[a]) + (E.c_lo[a] - I.c_lo[a]);
    g.o0[a] = g.d[a] + E.o0[a];
    g.e1[a] = E.e1[a];
    g.e2[a] = E.e2[a];
    g.n[a] = E.n[a];
  }
  g.area2 = E.area2;
}
__device__ __forceinline__ void pair_geom(const ElemF* ef, const ElemD* ed, int i, int e, PairGeo<double>& g) {
  const ElemD& I = ed[i];
  const ElemD& E = ed[e];
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    g.d[a] = E.c[a] - I.c[a];
    g.o0[a] = E.p0[a] - I.c[a];
    g.e1[a] = E.p1[a] - E.p0[a];
    g.e2[a] = E.p2[a] - E.p0[a];
    g.n[a] = E.n[a];
  }
  g.area2 = E.area2;
}

// ---------------------------------------------------------------------------
// per near block, its regular pairs sorted by (band, distance) once per mesh,
// so that the warps of the per-frequency kernel take the same quadrature
// branch. Entry: il | el << 12 | band << 24 (SELF/NEAR pairs are left out;
// the FP32 band decision falls back to FP64 next to a threshold, as in the
// rest of the library).
// ---------------------------------------------------------------------------
constexpr int SORT_MAX = 4096;

__global__ void __launch_bounds__(1024) k_pair_sort(const NearBlk* __restrict__ blks, const ElemF* __restrict__ ef,
                                                    const ElemD* __restrict__ ed, const long long* __restrict__ poff,
                                                    unsigned* __restrict__ plist, int* __restrict__ pcount) {
  __shared__ unsigned long long key[SORT_MAX];
  __shared__ int cnt;
  const NearBlk B = blks[blockIdx.x];
  const int np = B.nr * B.nc;
  const long long base = poff[blockIdx.x];
  if (threadIdx.x == 0) cnt = 0;
  __syncthreads();
  if (np > SORT_MAX) {
    // large block (leaf size above 64): natural order, band stored per pair
    for (int p = threadIdx.x; p < np; p += blockDim.x) {
      int il = p % B.nr, el = p / B.nr;
      PairGeo<float> g;
      int band;
      pair_geo(ef, ed, B.r0 + il, B.c0 + el, g, band);
      if (band == BAND_SELF || band == BAND_NEAR) continue;
      int pos = atomicAdd(&cnt, 1);
      plist[base + pos] = (unsigned)il | ((unsigned)el << 12) | ((unsigned)band << 24);
    }
    __syncthreads();
    if (threadIdx.x == 0) pcount[blockIdx.x] = cnt;
    return;
  }
  int P2 = 1;
  while (P2 < np) P2 <<= 1;
  for (int p = threadIdx.x; p < P2; p += blockDim.x) {
    unsigned long long k = ~0ULL;
    if (p < np) {
      int il = p % B.nr, el = p / B.nr;
      PairGeo<float> g;
      int band;
      pair_geo(ef, ed, B.r0 + il, B.c0 + el, g, band);
      if (band != BAND_SELF && band != BAND_NEAR) {
        k = ((unsigned long long)band << 61) | ((unsigned long long)__float_as_uint(g.d2) << 24) |
            (unsigned long long)p;
        atomicAdd(&cnt, 1);
      }
    }
    key[p] = k;
  }
  __syncthreads();
  // bitonic sort of P2 keys
  for (int size = 2; size <= P2; size <<= 1) {
    for (int stride = size >> 1; stride > 0; stride >>= 1) {
      for (int t = threadIdx.x; t < P2 / 2; t += blockDim.x) {
        int lo = 2 * t - (t & (stride - 1));
        int hi = lo + stride;
        bool up = ((lo & size) == 0);
        unsigned long long a = key[lo], b = key[hi];
        if ((a > b) == up) {
          key[lo] = b;
          key[hi] = a;
        }
      }
      __syncthreads();
    }
  }
  const int c = cnt;
  for (int q = threadIdx.x; q < c; q += blockDim.x) {
    unsigned long long k = key[q];
    int p = (int)(k & 0xFFFFFFULL);
    unsigned band = (unsigned)(k >> 61);
    int il = p % B.nr, el = p / B.nr;
    plist[base + q] = (unsigned)il | ((unsigned)el << 12) | (band << 24);
  }
  if (threadIdx.x == 0) pcount[blockIdx.x] = c;
}

// ---------------------------------------------------------------------------
// regular near-field entries and their share of the right-hand side:
// one CTA per near block, pairs taken from the sorted list
// ---------------------------------------------------------------------------
template <typename R, typename Op>
__global__ void __launch_bounds__(256) k_near_regular(const NearBlk* __restrict__ blks,
                                                      const unsigned* __restrict__ plist,
                                                      const long long* __restrict__ poff,
                                                      const int* __restrict__ pcount, const ElemF* __restrict__ ef,
                                                      const ElemD* __restrict__ ed,
                                                      const signed char* __restrict__ bc, KParams<R> P,
                                                      Op* __restrict__ near, const float* __restrict__ patf,
                                                      const double* __restrict__ patd, c128 pk,
                                                      c128* __restrict__ b) {
  extern __shared__ __align__(16) unsigned char rsum_raw[];
  R* rsum = reinterpret_cast<R*>(rsum_raw);  // 3 nr complex row sums of B pattern
  const NearBlk B = blks[blockIdx.x];
  const int cnt = pcount[blockIdx.x];
  const long long base = poff[blockIdx.x];
  const long long ld = B.ld;
  if (b)
    for (int r = threadIdx.x; r < 6 * B.nr; r += blockDim.x) rsum[r] = R(0);
  __syncthreads();
  for (int q = threadIdx.x; q < cnt; q += blockDim.x) {
    const unsigned code = plist[base + q];
    const int il = code & 0xFFF, el = (code >> 12) & 0xFFF, band = code >> 24;
    const int i = B.r0 + il, e = B.c0 + el;
    PairGeo<R> g;
    pair_geom(ef, ed, i, e, g);
    UTAcc<R> acc;
    regular_pair<R>(acc, g, band, P);
    const bool trac = bc[e] == BEM_BC_TRACTION;
    if (near) {
      Op* dst = near + B.off + (3 * el) * ld + 3 * il;
#pragma unroll
      for (int c = 0; c < 3; ++c)
#pragma unroll
        for (int a = 0; a < 3; ++a) {
          cplx<R> v = trac ? acc.t[3 * a + c] : -acc.U(a, c);
          dst[c * ld + a] = to_op<Op>(v);
        }
    }
    if (b) {
      R pt[3];
      if (sizeof(R) == 4) {
        pt[0] = R(patf[3 * e]);
        pt[1] = R(patf[3 * e + 1]);
        pt[2] = R(patf[3 * e + 2]);
      } else {
        pt[0] = R(patd[3 * e]);
        pt[1] = R(patd[3 * e + 1]);
        pt[2] = R(patd[3 * e + 2]);
      }
      if (pt[0] != R(0) || pt[1] != R(0) || pt[2] != R(0)) {
#pragma unroll
        for (int a = 0; a < 3; ++a) {
          cplx<R> sa = mk<R>(0, 0);
#pragma unroll
          for (int c = 0; c < 3; ++c) cfmr(sa, trac ? acc.U(a, c) : -acc.t[3 * a + c], pt[c]);
          atomicAdd(&rsum[2 * (3 * il + a)], sa.re);
          atomicAdd(&rsum[2 * (3 * il + a) + 1], sa.im);
        }
      }
    }
  }
  if (!b) return;
  __syncthreads();
  for (int r = threadIdx.x; r < 3 * B.nr; r += blockDim.x) {
    c128 v = c128{(double)rsum[2 * r], (double)rsum[2 * r + 1]} * pk;
    if (v.re != 0.0 || v.im != 0.0) {
      atomicAdd(&b[3LL * B.r0 + r].re, v.re);
      atomicAdd(&b[3LL * B.r0 + r].im, v.im);
    }
  }
}

// ---------------------------------------------------------------------------
// far-field share of the right-hand side, on the fly: one warp per row of an
// admissible block (items of 8 rows); traction-loaded columns need U only
// ---------------------------------------------------------------------------

// ---------------------------------------------------------------------------
// polar parameters of the self rule: per element, per triangle (c, p_k, p_k+1):
// d, fh[3], gh[3], theta_a, dtheta (once per mesh, FP64)
// ---------------------------------------------------------------------------
__global__ void k_polar(const ElemD* __restrict__ ed, int ne, double* __restrict__ out) {
  int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= ne) return;
  const ElemD& E = ed[e];
  for (int sub = 0; sub < 3; ++sub) {
    PolarSub S = polar_sub(E.c, vtx(E, sub), vtx(E, (sub + 1) % 3), E.n);
    double* o = out + 27LL * e + 9 * sub;
    o[0] = S.d;
    for (int a = 0; a < 3; ++a) {
      o[1 + a] = S.fh[a];
      o[4 + a] = S.gh[a];
    }
    o[7] = S.tha;
    o[8] = S.dth;
  }
}

// ---------------------------------------------------------------------------
// singular + near-singular entries: one warp per pair.
//   entry = static Kelvin part (FP64, once per mesh) + dynamic remainder
//   (self: polar 8 x 6 per triangle; near: collapsed 4x4), the remainder
//   evaluated cancellation-free in R (FP32 on the mixed path, FP64 plain).
// Also: block-Jacobi inverses (FP64) and the pairs' right-hand-side share.
// ---------------------------------------------------------------------------
__device__ __forceinline__ bool inv3(const c128* A, c128* Ai) {
  // cofactor inverse of a complex 3x3 (row-major)
  c128 c00 = A[4] * A[8] - A[5] * A[7];
  c128 c01 = A[5] * A[6] - A[3] * A[8];
  c128 c02 = A[3] * A[7] - A[4] * A[6];
  c128 det = A[0] * c00 + A[1] * c01 + A[2] * c02;
  if (abs2(det) == 0.0) return false;
  c128 id = inv(det);
  Ai[0] = c00 * id;
  Ai[1] = (A[2] * A[7] - A[1] * A[8]) * id;
  Ai[2] = (A[1] * A[5] - A[2] * A[4]) * id;
  Ai[3] = c01 * id;
  Ai[4] = (A[0] * A[8] - A[2] * A[6]) * id;
  Ai[5] = (A[2] * A[3] - A[0] * A[5]) * id;
  Ai[6] = c02 * id;
  Ai[7] = (A[1] * A[6] - A[0] * A[7]) * id;
  Ai[8] = (A[0] * A[4] - A[1] * A[3]) * id;
  return true;
}

template <typename R> __device__ __forceinline__ R wred(R v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// One half-warp (16 lanes) per singular or near-singular pair: the 16 points
// of the near-singular remainder rule one per lane, the 144 of the self rule
// nine per lane. The 15 complex accumulators (U: 6, T: 9) are reduced with a
// butterfly reduce-scatter (lane l ends with accumulator l), the FP64
// epilogue (static parts, free term, storage, right-hand side) is spread over
// the lanes. Self pairs come first in the list so that half-warps of one warp
// mostly follow the same branch.
template <typename R>
__device__ __forceinline__ cplx<R> shfl_xor_c(cplx<R> v, int o) {
  return mk<R>(__shfl_xor_sync(0xffffffffu, v.re, o), __shfl_xor_sync(0xffffffffu, v.im, o));
}

template <typename R, typename Op>
__global__ void __launch_bounds__(256) k_sing(const SingPair* __restrict__ pairs, int npairs,
                                              const ElemD* __restrict__ ed, const double* __restrict__ polar,
                                              const signed char* __restrict__ bc, const double* __restrict__ stat,
                                              KParams<R> P, Op* __restrict__ near, c128* __restrict__ pinv,
                                              const double* __restrict__ pattern, c128 pk, c128* __restrict__ b,
                                              int* __restrict__ status) {
  __shared__ c128 sh[16][16];
  const int pid = (blockIdx.x * blockDim.x + threadIdx.x) >> 4;
  const int hl = threadIdx.x & 15, slot = threadIdx.x >> 4;
  const bool active = pid < npairs;
  SingPair sp{0, 0, 0, 0, 0};
  UTAcc<R> acc;
  acc.zero();
  if (active) {
    sp = pairs[pid];
    const ElemD& E = ed[sp.e];
    const ElemD& I = ed[sp.i];
    R n[3] = {R(E.n[0]), R(E.n[1]), R(E.n[2])};
    if (sp.self) {
      for (int q = hl; q < 3 * SELF_NT * SELF_NR; q += 16) {
        int sub = q / (SELF_NT * SELF_NR);
        int m = (q / SELF_NR) % SELF_NT, l = q % SELF_NR;
        const double* ps = polar + 27LL * sp.e + 9 * sub;
        R d = R(ps[0]), tha = R(ps[7]), dth = R(ps[8]);
        R th = tha + dth * gl_x<R>(SELF_NT, m);
        R wth = dth * gl_w<R>(SELF_NT, m);
        R sn, cs;
        sincos_r(th, &sn, &cs);
        R Rr = d / cs;
        R r = Rr * gl_x<R>(SELF_NR, l);
        R w = wth * Rr * gl_w<R>(SELF_NR, l) * r;
        R rv[3];
        for (int a = 0; a < 3; ++a) rv[a] = r * (cs * R(ps[1 + a]) + sn * R(ps[4 + a]));
        accumulate_point<R, false>(acc, rv[0], rv[1], rv[2], n[0], n[1], n[2], w, P);
      }
    } else {
      int ia = hl / NEAR_Q_REM, ib = hl % NEAR_Q_REM;
      R u = gl_x<R>(NEAR_Q_REM, ia), v = (R(1) - u) * gl_x<R>(NEAR_Q_REM, ib);
      R w = R(E.area2) * gl_w<R>(NEAR_Q_REM, ia) * gl_w<R>(NEAR_Q_REM, ib) * (R(1) - u);
      R rv[3];
      for (int k = 0; k < 3; ++k)
        rv[k] = R(E.p0[k] - I.c[k]) + u * R(E.p1[k] - E.p0[k]) + v * R(E.p2[k] - E.p0[k]);
      accumulate_point<R, false>(acc, rv[0], rv[1], rv[2], n[0], n[1], n[2], w, P);
    }
  }
  // butterfly reduce-scatter over the half-warp: value index = lane
  cplx<R> v16[16];
#pragma unroll
  for (int k = 0; k < 6; ++k) v16[k] = acc.u[k];
#pragma unroll
  for (int k = 0; k < 9; ++k) v16[6 + k] = acc.t[k];
  v16[15] = mk<R>(0, 0);
  cplx<R> w8[8], w4[4], w2[2];
  {
    const bool hi = hl & 8;
#pragma unroll
    for (int k = 0; k < 8; ++k) {
      cplx<R> keep = hi ? v16[8 + k] : v16[k], give = hi ? v16[k] : v16[8 + k];
      w8[k] = keep + shfl_xor_c(give, 8);
    }
  }
  {
    const bool hi = hl & 4;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      cplx<R> keep = hi ? w8[4 + k] : w8[k], give = hi ? w8[k] : w8[4 + k];
      w4[k] = keep + shfl_xor_c(give, 4);
    }
  }
  {
    const bool hi = hl & 2;
#pragma unroll
    for (int k = 0; k < 2; ++k) {
      cplx<R> keep = hi ? w4[2 + k] : w4[k], give = hi ? w4[k] : w4[2 + k];
      w2[k] = keep + shfl_xor_c(give, 2);
    }
  }
  cplx<R> mine;
  {
    const bool hi = hl & 1;
    cplx<R> keep = hi ? w2[1] : w2[0], give = hi ? w2[0] : w2[1];
    mine = keep + shfl_xor_c(give, 1);
  }
  // FP64: add the static (Kelvin) part of accumulator hl and stage it
  const double* st = stat + 18LL * (active ? pid : 0);
  if (active && hl < 15) {
    const int uac[6] = {0, 1, 2, 4, 5, 8};  // (a, c) of the symmetric U entries: 3a + c
    double sre = hl < 6 ? st[uac[hl < 6 ? hl : 0]] : st[9 + (hl - 6)];
    c128 val = c128{(double)mine.re + sre, (double)mine.im};
    if (sp.self && hl >= 6 && ((hl - 6) % 4) == 0) val.re += 0.5;  // free term c_ij = delta_ij / 2
    sh[slot][hl] = val;
  }
  __syncwarp();
  if (!active) return;
  const bool trac = bc[sp.e] == BEM_BC_TRACTION;
  const int uidx[9] = {0, 1, 2, 1, 3, 4, 2, 4, 5};  // (a, c) -> symmetric U accumulator
  if (near && hl < 9) {
    const int a = hl / 3, c = hl % 3;
    c128 A = trac ? sh[slot][6 + hl] : -sh[slot][uidx[hl]];
    near[sp.entry + (long long)c * sp.ld + a] = to_op<Op>(A);
  }
  if (sp.self && pinv && hl == 0) {
    c128 Ablk[9], Ai[9];
    for (int k = 0; k < 9; ++k) Ablk[k] = trac ? sh[slot][6 + k] : -sh[slot][uidx[k]];
    if (!inv3(Ablk, Ai)) atomicExch(status, 3);
    for (int k = 0; k < 9; ++k) pinv[9 * (long long)sp.i + k] = Ai[k];
  }
  if (b && hl < 3) {
    const double* pt = pattern + 3 * (long long)sp.e;
    if (pt[0] != 0.0 || pt[1] != 0.0 || pt[2] != 0.0) {
      const int a = hl;
      c128 sacc = mk<double>(0, 0);
      for (int c = 0; c < 3; ++c) {
        c128 Bv = trac ? sh[slot][uidx[3 * a + c]] : -sh[slot][6 + 3 * a + c];
        cfmr(sacc, Bv, pt[c]);
      }
      sacc = sacc * pk;
      atomicAdd(&b[3 * (long long)sp.i + a].re, sacc.re);
      atomicAdd(&b[3 * (long long)sp.i + a].im, sacc.im);
    }
  }
}

// ---------------------------------------------------------------------------
// right-hand side over regular pairs, on the fly: one warp per row element.
// Traction-loaded columns need U only (B = U); displacement-loaded columns
// need T (B = -T).
// ---------------------------------------------------------------------------
// U-only integral of a pair over its band's rule (one inlined evaluator).
template <typename R>
__device__ __forceinline__ void regular_pair_u(cplx<R>* u, const PairGeo<R>& g, int band, const KParams<R>& P) {
  const int Q = band == BAND_Q4 ? 4 : (band == BAND_Q2 ? 2 : 1);
#pragma unroll 1
  for (int p = 0; p < Q * Q; ++p) {
    R rx, ry, rz, w;
    if (Q == 1) {
      rx = g.d[0];
      ry = g.d[1];
      rz = g.d[2];
      w = R(0.5) * g.area2;
    } else {
      const int a = p / Q, b = p - (p / Q) * Q;
      const R uu = gl_x<R>(Q, a);
      const R omu = R(1) - uu;
      const R v = omu * gl_x<R>(Q, b);
      w = g.area2 * gl_w<R>(Q, a) * gl_w<R>(Q, b) * omu;
      rx = g.o0[0] + uu * g.e1[0] + v * g.e2[0];
      ry = g.o0[1] + uu * g.e1[1] + v * g.e2[1];
      rz = g.o0[2] + uu * g.e1[2] + v * g.e2[2];
    }
    accumulate_point_u<R>(u, rx, ry, rz, w, P);
  }
}

// One warp per row element i: every far column element of i's leaf (the
// column ranges of the admissible blocks whose row cluster holds the leaf),
// lanes striding over the concatenated ranges; one reduction and one
// (non-atomic) update of b per row. b must not be written concurrently: the
// kernel runs first after b is zeroed.
template <typename R>
__global__ void __launch_bounds__(256) k_rhs_far(const int* __restrict__ rng, const int* __restrict__ rptr,
                                                 const int* __restrict__ elem_leaf, int ne,
                                                 const ElemF* __restrict__ ef, const ElemD* __restrict__ ed,
                                                 const signed char* __restrict__ bc, const float* __restrict__ patf,
                                                 const double* __restrict__ patd, KParams<R> P, c128 pk,
                                                 c128* __restrict__ b) {
  const int i = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (i >= ne) return;
  const int leaf = elem_leaf[i];
  const int q0 = rptr[leaf], q1 = rptr[leaf + 1];
  cplx<R> s[3] = {mk<R>(0, 0), mk<R>(0, 0), mk<R>(0, 0)};
  // lane-strided walk over the concatenation of the ranges [c0, c0 + nc)
  int q = q0, base = 0;
  int c0 = q < q1 ? rng[2 * q] : 0, nc = q < q1 ? rng[2 * q + 1] : 0;
  for (int v = lane;; v += 32) {
    while (q < q1 && v >= base + nc) {
      base += nc;
      ++q;
      if (q < q1) {
        c0 = rng[2 * q];
        nc = rng[2 * q + 1];
      }
    }
    if (q >= q1) break;
    const int e = c0 + (v - base);
    R p3[3];
    if (sizeof(R) == 4) {
      p3[0] = R(patf[3 * e]);
      p3[1] = R(patf[3 * e + 1]);
      p3[2] = R(patf[3 * e + 2]);
    } else {
      p3[0] = R(patd[3 * e]);
      p3[1] = R(patd[3 * e + 1]);
      p3[2] = R(patd[3 * e + 2]);
    }
    if (p3[0] == R(0) && p3[1] == R(0) && p3[2] == R(0)) continue;
    PairGeo<R> g;
    int band;
    pair_geo(ef, ed, i, e, g, band);
    if (bc[e] == BEM_BC_TRACTION) {
      cplx<R> u[6];
#pragma unroll
      for (int k = 0; k < 6; ++k) u[k] = mk<R>(0, 0);
      regular_pair_u<R>(u, g, band, P);
      const int idx[3][3] = {{0, 1, 2}, {1, 3, 4}, {2, 4, 5}};
#pragma unroll
      for (int a = 0; a < 3; ++a)
#pragma unroll
        for (int c = 0; c < 3; ++c) cfmr(s[a], u[idx[a][c]], p3[c]);
    } else {
      UTAcc<R> acc;
      regular_pair<R>(acc, g, band, P);
#pragma unroll
      for (int a = 0; a < 3; ++a)
#pragma unroll
        for (int c = 0; c < 3; ++c) cfmr(s[a], -acc.t[3 * a + c], p3[c]);
    }
  }
  R red[6];
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    red[2 * a] = wred(s[a].re);
    red[2 * a + 1] = wred(s[a].im);
  }
  if (lane < 3) {
    R re = lane == 0 ? red[0] : (lane == 1 ? red[2] : red[4]);
    R im = lane == 0 ? red[1] : (lane == 1 ? red[3] : red[5]);
    c128 v = c128{(double)re, (double)im} * pk;
    c128& t = b[3LL * i + lane];
    t = c128{t.re + v.re, t.im + v.im};
  }
}

// ---------------------------------------------------------------------------
// Entries of an admissible block as they enter the system matrix: the column
// element's boundary condition selects T (traction prescribed: unknown
// displacement) or -U (displacement prescribed: unknown traction).
// aca_row3: row component ia of collocation element ie against element e
// (three columns); aca_col3: column component jc of element je against
// collocation element i (three rows).
// ---------------------------------------------------------------------------
// One line of a pair's block over the band's rule (one inlined evaluator).
template <typename R>
__device__ __forceinline__ void regular_pair_line(cplx<R> out[3], const PairGeo<R>& g, int band, const KParams<R>& P,
                                                  bool useT, bool col, int idx) {
  out[0] = out[1] = out[2] = mk<R>(0, 0);
  const int Q = band == BAND_Q4 ? 4 : (band == BAND_Q2 ? 2 : 1);
#pragma unroll 1
  for (int p = 0; p < Q * Q; ++p) {
    R rx, ry, rz, w;
    if (Q == 1) {
      rx = g.d[0];
      ry = g.d[1];
      rz = g.d[2];
      w = R(0.5) * g.area2;
    } else {
      const int a = p / Q, b = p - (p / Q) * Q;
      const R u = gl_x<R>(Q, a);
      const R omu = R(1) - u;
      const R v = omu * gl_x<R>(Q, b);
      w = g.area2 * gl_w<R>(Q, a) * gl_w<R>(Q, b) * omu;
      rx = g.o0[0] + u * g.e1[0] + v * g.e2[0];
      ry = g.o0[1] + u * g.e1[1] + v * g.e2[1];
      rz = g.o0[2] + u * g.e1[2] + v * g.e2[2];
    }
    accumulate_point_line<R>(out, rx, ry, rz, g.n[0], g.n[1], g.n[2], w, P, useT, col, idx);
  }
}

template <typename R, typename T>
__device__ __forceinline__ void aca_row3(const ElemF* ef, const ElemD* ed, const signed char* bc,
                                         const KParams<R>& P, int ie, int ia, int e, cplx<T> out[3]) {
  PairGeo<R> g;
  int band;
  pair_geo(ef, ed, ie, e, g, band);
  const bool trac = bc[e] == BEM_BC_TRACTION;
  cplx<R> v[3];
  regular_pair_line<R>(v, g, band, P, trac, false, ia);
#pragma unroll
  for (int c = 0; c < 3; ++c) out[c] = trac ? mk<T>(T(v[c].re), T(v[c].im)) : mk<T>(T(-v[c].re), T(-v[c].im));
}
template <typename R, typename T>
__device__ __forceinline__ void aca_col3(const ElemF* ef, const ElemD* ed, const signed char* bc,
                                         const KParams<R>& P, int i, int je, int jc, cplx<T> out[3]) {
  PairGeo<R> g;
  int band;
  pair_geo(ef, ed, i, je, g, band);
  const bool trac = bc[je] == BEM_BC_TRACTION;
  cplx<R> v[3];
  regular_pair_line<R>(v, g, band, P, trac, true, jc);
#pragma unroll
  for (int a = 0; a < 3; ++a) out[a] = trac ? mk<T>(T(v[a].re), T(v[a].im)) : mk<T>(T(-v[a].re), T(-v[a].im));
}

// ---------------------------------------------------------------------------
// ACA with partial pivoting: one CTA per admissible block
//   residual row i* -> v_k (scaled by the pivot), residual column j* -> u_k,
//   ||S_k||_F^2 estimated by sum_{l<=k} |u_l|^2 |v_l|^2 (the usual diagonal
//   estimate; the cross terms are dropped), stop when
//   |u_k| |v_k| <= eps ||S_k||_F or at the rank cap.
// Norms are accumulated in the storage precision (FP32 on the mixed path).
// ---------------------------------------------------------------------------
constexpr int ACA_THREADS = 128;
constexpr int ACA_WARPS = ACA_THREADS / 32;
constexpr int ACA_RMAX = ACA_RANK_CAP;
constexpr int ACA_EXTRA = 2;  // pivots recorded past the stopping point (spares for the next frequency)

template <typename T> struct AcaShared {
  T dot[2][1][ACA_WARPS];  // per-warp partial norms
  T amax[ACA_WARPS];
  int aidx[ACA_WARPS];
  T scal[4];
  int rows_used[ACA_RMAX];
};

template <typename T> __device__ __forceinline__ T wsumT(T v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// block-wide max with index (ties -> smaller index); result valid in all threads
template <typename T> __device__ __forceinline__ void aca_argmax(T& v, int& idx, AcaShared<T>& sh) {
  int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    T ov = __shfl_xor_sync(0xffffffffu, v, o);
    int oi = __shfl_xor_sync(0xffffffffu, idx, o);
    if (ov > v || (ov == v && oi < idx)) {
      v = ov;
      idx = oi;
    }
  }
  __syncthreads();
  if (lane == 0) {
    sh.amax[wid] = v;
    sh.aidx[wid] = idx;
  }
  __syncthreads();
  v = sh.amax[0];
  idx = sh.aidx[0];
  for (int w = 1; w < ACA_WARPS; ++w)
    if (sh.amax[w] > v || (sh.amax[w] == v && sh.aidx[w] < idx)) {
      v = sh.amax[w];
      idx = sh.aidx[w];
    }
}

// Residual row irow of a block into V[:, k]: A(irow, :) - sum_{l<k} U(irow, l) V(:, l)^T,
// the block's column elements split over the threads t0, t0 + tstride, ...
template <typename R, typename T, typename Op>
__device__ __forceinline__ void aca_residual_row(const ElemF* ef, const ElemD* ed, const signed char* bc,
                                                 const KParams<R>& P, const FarBlk& B, const Op* Ub, Op* Vb, int m,
                                                 int n, int k, int irow, int t0, int tstride) {
  const int ie = B.r0 + irow / 3, ia = irow % 3;
  for (int el = t0; el < B.nc; el += tstride) {
    int e = B.c0 + el;
    cplx<T> vv[3];
    aca_row3<R, T>(ef, ed, bc, P, ie, ia, e, vv);
    const Op* vrow = Vb + 3 * el;
#pragma unroll 4
    for (int l = 0; l < k; ++l) {
      Op ul = Ub[(long long)l * m + irow];
      const Op* vl = vrow + (long long)l * n;
      Op v0 = vl[0], v1 = vl[1], v2 = vl[2];
      cplx<T> cu = mk<T>(ul.re, ul.im);
      vv[0] = vv[0] - cu * mk<T>(v0.re, v0.im);
      vv[1] = vv[1] - cu * mk<T>(v1.re, v1.im);
      vv[2] = vv[2] - cu * mk<T>(v2.re, v2.im);
    }
#pragma unroll
    for (int c = 0; c < 3; ++c) Vb[(long long)k * n + 3 * el + c] = to_op<Op>(vv[c]);
  }
}

// Check rows of the convergence test, one per displacement component a,
// from elements spread over the row cluster. Partial pivoting only follows
// the nonzero pattern of the rows and columns it has visited: on a flat face
// the normal-component rows of a coplanar block couple only to the
// tangential columns and the tangential rows only to the normal columns, so
// a block that converged on one of the two parts has not seen the other.
// A check row whose residual is not small restarts the ACA steps from it.
__device__ __forceinline__ int aca_check_row(int nr, int a) { return 3 * ((a * nr) / 3 + nr / 6) + a; }

template <typename R, typename Op>
__global__ void __launch_bounds__(ACA_THREADS) k_aca(const int* __restrict__ list, const FarBlk* __restrict__ blks,
                                                     const ElemF* __restrict__ ef,
                                                     const ElemD* __restrict__ ed,
                                                     const signed char* __restrict__ bc, KParams<R> P,
                                                     Op* __restrict__ Ustore, Op* __restrict__ Vstore,
                                                     int* __restrict__ rank, int* __restrict__ fails, double eps_d,
                                                     AcaState st) {
  using T = decltype(Op{}.re);
  const T eps = T(eps_d);
  const int bi = list[blockIdx.x];
  const int dstate = st.done ? st.done[bi] : 0;
  if (dstate == 1) return;
  FarBlk B = blks[bi];
  const int m = 3 * B.nr, n = 3 * B.nc;
  Op* Ub = Ustore + B.uoff;
  Op* Vb = Vstore + B.voff;
  int* piv_i = st.piv_i + B.toff;
  int* piv_j = st.piv_j + B.toff;
  __shared__ AcaShared<T> sh;
  const int rmax = min(B.rmax, ACA_RMAX);
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  int k = st.kstart ? min(st.kstart[bi], rmax) : 0;
  const int k0 = k;
  int istar = 0;
  T normS2 = k ? T(st.norm0[bi]) : T(0);
  int kconv = -1;  // rank at which the stopping test first held
  // dstate 2: the reused steps met the stopping test (rank set by the reuse);
  // only the check rows remain, as after any converged ACA
  bool check_only = dstate == 2 && k > 0;
  if (check_only) {
    for (int l = threadIdx.x; l < k; l += blockDim.x) sh.rows_used[l] = piv_i[l];
    kconv = rank[bi];
    __syncthreads();
  } else if (k > 0) {
    // continue from a reused cross approximation of rank k: its pivot rows
    // are used, the next row is the largest entry of u_{k-1} outside them
    for (int l = threadIdx.x; l < k; l += blockDim.x) sh.rows_used[l] = piv_i[l];
    const int prev = piv_i[k - 1];
    T bu = T(-1);
    int inext = 0;
    for (int i = threadIdx.x; i < m; i += blockDim.x) {
      if (i == prev) continue;
      Op u = Ub[(long long)(k - 1) * m + i];
      T a = u.re * u.re + u.im * u.im;
      if (a > bu) {
        bu = a;
        inext = i;
      }
    }
    aca_argmax(bu, inext, sh);
    if (!(bu > T(0))) {
      if (threadIdx.x == 0) {
        rank[bi] = k;
        st.npiv[bi] = k;
      }
      return;
    }
    istar = inext;
    __syncthreads();
  }
  int vnext = 0;          // components whose check row has been examined
  bool have_row = false;  // V[:, k] already holds the residual row of istar
  while (k < rmax) {
   bool stop = false;
   if (check_only) {
    check_only = false;
    stop = true;
   } else {
    // --- residual row istar -> V[:, k]
    if (!have_row) aca_residual_row<R, T, Op>(ef, ed, bc, P, B, Ub, Vb, m, n, k, istar, threadIdx.x, blockDim.x);
    have_row = false;
    __syncthreads();
    T best = T(-1);
    int jstar = 0;
    for (int j = threadIdx.x; j < n; j += blockDim.x) {
      Op v = Vb[(long long)k * n + j];
      T a = v.re * v.re + v.im * v.im;
      if (a > best) {
        best = a;
        jstar = j;
      }
    }
    aca_argmax(best, jstar, sh);
    if (!(best > T(0))) {
      if (kconv < 0) kconv = k;  // zero residual row
      stop = true;
    } else {
      Op pv = Vb[(long long)k * n + jstar];
      cplx<T> ipiv = inv(mk<T>(pv.re, pv.im));
      __syncthreads();
      for (int j = threadIdx.x; j < n; j += blockDim.x) {
        Op v = Vb[(long long)k * n + j];
        Vb[(long long)k * n + j] = to_op<Op>(mk<T>(v.re, v.im) * ipiv);
      }
      if (threadIdx.x == 0) {
        piv_i[k] = istar;
        piv_j[k] = jstar;
      }
      __syncthreads();
      // --- residual column jstar -> U[:, k]
      int je = B.c0 + jstar / 3, jc = jstar % 3;
      for (int il = threadIdx.x; il < B.nr; il += blockDim.x) {
        int i = B.r0 + il;
        cplx<T> uu[3];
        aca_col3<R, T>(ef, ed, bc, P, i, je, jc, uu);
        const Op* ucol = Ub + 3 * il;
#pragma unroll 4
        for (int l = 0; l < k; ++l) {
          Op vl = Vb[(long long)l * n + jstar];
          const Op* ul = ucol + (long long)l * m;
          Op u0 = ul[0], u1 = ul[1], u2 = ul[2];
          cplx<T> cv = mk<T>(vl.re, vl.im);
          uu[0] = uu[0] - mk<T>(u0.re, u0.im) * cv;
          uu[1] = uu[1] - mk<T>(u1.re, u1.im) * cv;
          uu[2] = uu[2] - mk<T>(u2.re, u2.im) * cv;
        }
#pragma unroll
        for (int a = 0; a < 3; ++a) Ub[(long long)k * m + 3 * il + a] = to_op<Op>(uu[a]);
      }
      if (threadIdx.x == 0) sh.rows_used[k] = istar;
      __syncthreads();
      // earlier pivot rows are exactly represented already: their residual is zero
      for (int l = threadIdx.x; l < k; l += blockDim.x) Ub[(long long)k * m + sh.rows_used[l]] = Op{};
      __syncthreads();
      // Frobenius norm of the approximant estimated by its diagonal terms:
      // ||S_k||^2 ~ sum_l |u_l|^2 |v_l|^2
      {
        T nu2 = 0, nv2 = 0;
        for (int i = threadIdx.x; i < m; i += blockDim.x) {
          Op a = Ub[(long long)k * m + i];
          nu2 += a.re * a.re + a.im * a.im;
        }
        for (int j = threadIdx.x; j < n; j += blockDim.x) {
          Op a = Vb[(long long)k * n + j];
          nv2 += a.re * a.re + a.im * a.im;
        }
        nu2 = wsumT(nu2);
        nv2 = wsumT(nv2);
        if (lane == 0) {
          sh.dot[0][0][wid] = nu2;
          sh.dot[1][0][wid] = nv2;
        }
        __syncthreads();
        if (threadIdx.x == 0) {
          T a = 0, b2 = 0;
          for (int w = 0; w < ACA_WARPS; ++w) {
            a += sh.dot[0][0][w];
            b2 += sh.dot[1][0][w];
          }
          normS2 += a * b2;
          sh.scal[0] = normS2;
          sh.scal[1] = a * b2;
        }
        __syncthreads();
      }
      normS2 = sh.scal[0];
      T term = sh.scal[1];
      ++k;
      if (kconv < 0 && term <= eps * eps * normS2) kconv = k;
      // ACA_EXTRA steps past the stopping point record spare pivots for reuse
      if (kconv >= 0 && k >= kconv + ACA_EXTRA) {
        stop = true;
      } else {
        // --- next pivot row: largest entry of u_k outside the rows used so far
        T bu = T(-1);
        int inext = 0;
        for (int i = threadIdx.x; i < m; i += blockDim.x) {
          if (i == istar) continue;
          Op u = Ub[(long long)(k - 1) * m + i];
          T a = u.re * u.re + u.im * u.im;
          if (a > bu) {
            bu = a;
            inext = i;
          }
        }
        aca_argmax(bu, inext, sh);
        if (!(bu > T(0))) {
          if (kconv < 0) kconv = k;
          stop = true;
        } else {
          istar = inext;
        }
      }
    }
   }
    __syncthreads();
    if (!stop) continue;
    // --- the test held: check rows (residual into V[:, k]) before stopping
    bool again = false;
    while (vnext < 3 && k < rmax) {
      const int irow = aca_check_row(B.nr, vnext++);
      bool used = false;
      for (int l = 0; l < k; ++l) used |= sh.rows_used[l] == irow;
      if (used) continue;
      aca_residual_row<R, T, Op>(ef, ed, bc, P, B, Ub, Vb, m, n, k, irow, threadIdx.x, blockDim.x);
      __syncthreads();
      T r2 = 0;
      for (int j = threadIdx.x; j < n; j += blockDim.x) {
        Op v = Vb[(long long)k * n + j];
        r2 += v.re * v.re + v.im * v.im;
      }
      r2 = wsumT(r2);
      if (lane == 0) sh.dot[0][0][wid] = r2;
      __syncthreads();
      T tot = 0;
      for (int w = 0; w < ACA_WARPS; ++w) tot += sh.dot[0][0][w];
      __syncthreads();
      if (tot > eps * eps * normS2) {
        istar = irow;
        again = true;
        break;
      }
    }
    if (!again) break;
    kconv = -1;
    have_row = true;
  }
  if (threadIdx.x == 0) {
    rank[bi] = kconv >= 0 ? kconv : k;
    st.npiv[bi] = k;
    if (kconv < 0) atomicAdd(fails, 1);
    if (dstate == 2) st.done[bi] = k == k0 ? 1 : 0;  // settled by the reuse, or ACA steps were needed
  }
}

// ---------------------------------------------------------------------------
// ACA, one warp per (small) admissible block: same algorithm as k_aca with
// warp-synchronous reductions (no block barriers), so thousands of small
// blocks run concurrently.
// ---------------------------------------------------------------------------
constexpr int ACAW_WARPS = 4;

template <typename T> __device__ __forceinline__ void warp_argmax(T& v, int& idx) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    T ov = __shfl_xor_sync(0xffffffffu, v, o);
    int oi = __shfl_xor_sync(0xffffffffu, idx, o);
    if (ov > v || (ov == v && oi < idx)) {
      v = ov;
      idx = oi;
    }
  }
}

template <typename R, typename Op>
__global__ void __launch_bounds__(32 * ACAW_WARPS) k_aca_warp(const int* __restrict__ list, int count,
                                                              const FarBlk* __restrict__ blks,
                                                              const ElemF* __restrict__ ef,
                                                              const ElemD* __restrict__ ed,
                                                              const signed char* __restrict__ bc, KParams<R> P,
                                                              Op* __restrict__ Ustore, Op* __restrict__ Vstore,
                                                              int* __restrict__ rank, int* __restrict__ fails,
                                                              double eps_d, AcaState st) {
  using T = decltype(Op{}.re);
  const int wid = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int item = blockIdx.x * ACAW_WARPS + wid;
  if (item >= count) return;
  const int bi = list[item];
  const int dstate = st.done ? st.done[bi] : 0;
  if (dstate == 1) return;
  __shared__ int rows_used_all[ACAW_WARPS][ACA_RMAX];
  int* rows_used = rows_used_all[wid];
  const T eps = T(eps_d);
  const FarBlk B = blks[bi];
  const int m = 3 * B.nr, n = 3 * B.nc;
  Op* Ub = Ustore + B.uoff;
  Op* Vb = Vstore + B.voff;
  int* piv_i = st.piv_i + B.toff;
  int* piv_j = st.piv_j + B.toff;
  const int rmax = min(B.rmax, ACA_RMAX);
  int k = st.kstart ? min(st.kstart[bi], rmax) : 0;
  const int k0 = k;
  int istar = 0;
  T normS2 = k ? T(st.norm0[bi]) : T(0);
  int kconv = -1;
  bool check_only = dstate == 2 && k > 0;  // only the check rows remain (see k_aca)
  if (check_only) {
    for (int l = lane; l < k; l += 32) rows_used[l] = piv_i[l];
    kconv = rank[bi];
    __syncwarp();
  } else if (k > 0) {
    // continue from a reused cross approximation of rank k (see k_aca)
    for (int l = lane; l < k; l += 32) rows_used[l] = piv_i[l];
    const int prev = piv_i[k - 1];
    T bu = T(-1);
    int inext = 0;
    for (int i = lane; i < m; i += 32) {
      if (i == prev) continue;
      Op u = Ub[(long long)(k - 1) * m + i];
      T a = u.re * u.re + u.im * u.im;
      if (a > bu) {
        bu = a;
        inext = i;
      }
    }
    warp_argmax(bu, inext);
    if (!(bu > T(0))) {
      if (lane == 0) {
        rank[bi] = k;
        st.npiv[bi] = k;
      }
      return;
    }
    istar = inext;
    __syncwarp();
  }
  int vnext = 0;          // components whose check row has been examined (see k_aca)
  bool have_row = false;  // V[:, k] already holds the residual row of istar
  while (k < rmax) {
   bool stop = false;
   if (check_only) {
    check_only = false;
    stop = true;
   } else {
    if (!have_row) aca_residual_row<R, T, Op>(ef, ed, bc, P, B, Ub, Vb, m, n, k, istar, lane, 32);
    have_row = false;
    __syncwarp();
    T best = T(-1);
    int jstar = 0;
    for (int j = lane; j < n; j += 32) {
      Op v = Vb[(long long)k * n + j];
      T a = v.re * v.re + v.im * v.im;
      if (a > best) {
        best = a;
        jstar = j;
      }
    }
    warp_argmax(best, jstar);
    if (!(best > T(0))) {
      if (kconv < 0) kconv = k;
      stop = true;
    } else {
      Op pv = Vb[(long long)k * n + jstar];
      cplx<T> ipiv = inv(mk<T>(pv.re, pv.im));
      __syncwarp();
      for (int j = lane; j < n; j += 32) {
        Op v = Vb[(long long)k * n + j];
        Vb[(long long)k * n + j] = to_op<Op>(mk<T>(v.re, v.im) * ipiv);
      }
      if (lane == 0) {
        piv_i[k] = istar;
        piv_j[k] = jstar;
      }
      __syncwarp();
      int je = B.c0 + jstar / 3, jc = jstar % 3;
      for (int il = lane; il < B.nr; il += 32) {
        int i = B.r0 + il;
        cplx<T> uu[3];
        aca_col3<R, T>(ef, ed, bc, P, i, je, jc, uu);
        const Op* ucol = Ub + 3 * il;
#pragma unroll 4
        for (int l = 0; l < k; ++l) {
          Op vl = Vb[(long long)l * n + jstar];
          const Op* ul = ucol + (long long)l * m;
          Op u0 = ul[0], u1 = ul[1], u2 = ul[2];
          cplx<T> cv = mk<T>(vl.re, vl.im);
          uu[0] = uu[0] - mk<T>(u0.re, u0.im) * cv;
          uu[1] = uu[1] - mk<T>(u1.re, u1.im) * cv;
          uu[2] = uu[2] - mk<T>(u2.re, u2.im) * cv;
        }
#pragma unroll
        for (int a = 0; a < 3; ++a) Ub[(long long)k * m + 3 * il + a] = to_op<Op>(uu[a]);
      }
      if (lane == 0) rows_used[k] = istar;
      __syncwarp();
      for (int l = lane; l < k; l += 32) Ub[(long long)k * m + rows_used[l]] = Op{};
      __syncwarp();
      // Frobenius norm of the approximant estimated by its diagonal terms:
      // ||S_k||^2 ~ sum_l |u_l|^2 |v_l|^2
      T nu2 = 0, nv2 = 0;
      for (int i = lane; i < m; i += 32) {
        Op a = Ub[(long long)k * m + i];
        nu2 += a.re * a.re + a.im * a.im;
      }
      for (int j = lane; j < n; j += 32) {
        Op a = Vb[(long long)k * n + j];
        nv2 += a.re * a.re + a.im * a.im;
      }
      nu2 = wsumT(nu2);
      nv2 = wsumT(nv2);
      normS2 += nu2 * nv2;
      ++k;
      if (kconv < 0 && nu2 * nv2 <= eps * eps * normS2) kconv = k;
      if (kconv >= 0 && k >= kconv + ACA_EXTRA) {
        stop = true;
      } else {
        T bu = T(-1);
        int inext = 0;
        for (int i = lane; i < m; i += 32) {
          if (i == istar) continue;
          Op u = Ub[(long long)(k - 1) * m + i];
          T a = u.re * u.re + u.im * u.im;
          if (a > bu) {
            bu = a;
            inext = i;
          }
        }
        warp_argmax(bu, inext);
        if (!(bu > T(0))) {
          if (kconv < 0) kconv = k;
          stop = true;
        } else {
          istar = inext;
        }
      }
    }
   }
    __syncwarp();
    if (!stop) continue;
    // the test held: check rows before stopping (see k_aca)
    bool again = false;
    while (vnext < 3 && k < rmax) {
      const int irow = aca_check_row(B.nr, vnext++);
      bool used = false;
      for (int l = 0; l < k; ++l) used |= rows_used[l] == irow;
      if (used) continue;
      aca_residual_row<R, T, Op>(ef, ed, bc, P, B, Ub, Vb, m, n, k, irow, lane, 32);
      __syncwarp();
      T r2 = 0;
      for (int j = lane; j < n; j += 32) {
        Op v = Vb[(long long)k * n + j];
        r2 += v.re * v.re + v.im * v.im;
      }
      r2 = wsumT(r2);
      if (r2 > eps * eps * normS2) {
        istar = irow;
        again = true;
        break;
      }
    }
    if (!again) break;
    kconv = -1;
    have_row = true;
  }
  if (lane == 0) {
    rank[bi] = kconv >= 0 ? kconv : k;
    st.npiv[bi] = k;
    if (kconv < 0) atomicAdd(fails, 1);
    if (dstate == 2) st.done[bi] = k == k0 ? 1 : 0;
  }
}

// ---------------------------------------------------------------------------
// Cross-frequency reuse of the ACA pivots (not in the paper; its Sec. 5 names
// the per-frequency assembly as the cost to cut).
//
// With the pivot rows I = (i_1..i_r) and columns J = (j_1..j_r) that ACA chose
// for a block at the previous frequency, the cross approximation through the
// same pivots at the new s is
//     A ~ C P^{-1} R,  C = A(:, J), R = A(I, :), P = A(I, J) = L Uh
// (LU without pivoting, in the pivot order), which is exactly what ACA
// produces when it visits those pivots in that order. Stored as
//     U = C Uh^{-1},  V^T = L^{-1} R,
// step l of which equals ACA's step l (u_l v_l^T). Evaluating C and R is one
// fully parallel pass; the two triangular solves run per block from shared
// memory. Pivot l is kept only while it is still near-maximal in its residual
// row (|Uh_ll| >= tau max_j |(L^{-1} R)_lj|); the usual stopping test
// |u_l| |v_l| <= eps ||S_l|| then picks the rank. Blocks that do not meet it
// continue with ordinary ACA steps from there (k_aca / k_aca_warp).
// ---------------------------------------------------------------------------
constexpr int WARM_THREADS = 256;

// Pivot rows into V[:, l] and pivot columns into U[:, l], l < the pivot count
// of the previous frequency (its rank plus spares).
template <typename R, typename Op>
__global__ void __launch_bounds__(WARM_THREADS) k_aca_warm_eval(const FarBlk* __restrict__ blks, int b0,
                                                                const ElemF* __restrict__ ef,
                                                                const ElemD* __restrict__ ed,
                                                                const signed char* __restrict__ bc, KParams<R> P,
                                                                Op* __restrict__ Ustore, Op* __restrict__ Vstore,
                                                                const int* __restrict__ npiv,
                                                                const int* __restrict__ piv_i,
                                                                const int* __restrict__ piv_j) {
  using T = decltype(Op{}.re);
  const int bi = b0 + blockIdx.x;
  const int r = npiv[bi];
  if (r <= 0 || r > WARM_RMAX) return;
  const FarBlk B = blks[bi];
  const int m = 3 * B.nr, n = 3 * B.nc;
  Op* Ub = Ustore + B.uoff;
  Op* Vb = Vstore + B.voff;
  const int* pi = piv_i + B.toff;
  const int* pj = piv_j + B.toff;
  const int nrow = r * B.nc, total = nrow + r * B.nr;  // r <= rmax: within the block's U, V storage
  for (int idx = threadIdx.x; idx < total; idx += blockDim.x) {
    cplx<T> v[3];
    if (idx < nrow) {
      int l = idx / B.nc, el = idx - l * B.nc;
      int istar = pi[l];
      aca_row3<R, T>(ef, ed, bc, P, B.r0 + istar / 3, istar % 3, B.c0 + el, v);
      Op* dst = Vb + (long long)l * n + 3 * el;
#pragma unroll
      for (int c = 0; c < 3; ++c) dst[c] = to_op<Op>(v[c]);
    } else {
      int q = idx - nrow;
      int l = q / B.nr, il = q - l * B.nr;
      int jstar = pj[l];
      aca_col3<R, T>(ef, ed, bc, P, B.r0 + il, B.c0 + jstar / 3, jstar % 3, v);
      Op* dst = Ub + (long long)l * m + 3 * il;
#pragma unroll
      for (int a = 0; a < 3; ++a) dst[a] = to_op<Op>(v[a]);
    }
  }
}

constexpr int WARM_CW = 2;  // columns (rows) of the right-hand sides per thread

template <typename T> __device__ __forceinline__ void smem_max(T* a, T v);
template <> __device__ __forceinline__ void smem_max<float>(float* a, float v) {
  atomicMax(reinterpret_cast<int*>(a), __float_as_int(v));  // v >= 0: integer order = float order
}
template <> __device__ __forceinline__ void smem_max<double>(double* a, double v) {
  atomicMax(reinterpret_cast<unsigned long long*>(a), (unsigned long long)__double_as_longlong(v));
}

template <typename T> __device__ __forceinline__ T wmaxT(T v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = max(v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;
}

// In-place triangular solve of the rows [0, nrow) of X (row l at X + l * ldx,
// columns [0, ncol)) against the r x r matrix in shared memory Ps:
//   LOWER: X <- L^{-1} X, L unit lower (Ps[l r + q], q < l), one column of X
//          per thread lane of work;
//   else:  X <- X Uh^{-1} with X stored transposed (column l at X + l * ldx,
//          rows [0, ncol)), Uh upper (Ps[p r + l], p <= l).
// Per row l: max over the columns of |x_l|^2 into rowmax[l] (if given) and the
// sum into sum_w[l * NW + warp] (fixed order within a warp). A thread holds a
// CH x WARM_CW tile in registers; earlier rows are re-read from X.
template <typename Op, int NT, int CH, bool LOWER>
__device__ __forceinline__ void warm_trsm(Op* X, long long ldx, int ncol, int nrow, const cplx<decltype(Op{}.re)>* Ps,
                                          int r, decltype(Op{}.re)* rowmax, decltype(Op{}.re)* sum_w) {
  using T = decltype(Op{}.re);
  using C = cplx<T>;
  constexpr int NW = NT / 32;
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
  for (int j0 = 0; j0 < ncol; j0 += NT * WARM_CW) {
    if (j0 + wid * 32 >= ncol) continue;  // warp-uniform: this warp has no column in this pass
    int jc[WARM_CW];
    bool act[WARM_CW];
#pragma unroll
    for (int c = 0; c < WARM_CW; ++c) {
      jc[c] = j0 + tid + c * NT;
      act[c] = jc[c] < ncol;
    }
    const bool any2 = j0 + NT + wid * 32 < ncol;  // warp-uniform: second column set in use
    for (int c0 = 0; c0 < nrow; c0 += CH) {
      const int nv = min(CH, nrow - c0);
      // row (LOWER) or column (upper) of the factor used for chunk row t,
      // clamped into the r x r block: rows t >= nv are computed but not kept
      int ft[CH];
#pragma unroll
      for (int t = 0; t < CH; ++t) ft[t] = min(c0 + t, r - 1);
      C acc[CH][WARM_CW];
#pragma unroll
      for (int t = 0; t < CH; ++t)
#pragma unroll
        for (int c = 0; c < WARM_CW; ++c) {
          Op v = (act[c] && t < nv) ? X[(long long)(c0 + t) * ldx + jc[c]] : Op{};
          acc[t][c] = mk<T>(v.re, v.im);
        }
      if (any2) {
#pragma unroll 2
        for (int q = 0; q < c0; ++q) {
          C x[WARM_CW];
#pragma unroll
          for (int c = 0; c < WARM_CW; ++c) {
            Op xv = act[c] ? X[(long long)q * ldx + jc[c]] : Op{};
            x[c] = mk<T>(xv.re, xv.im);
          }
#pragma unroll
          for (int t = 0; t < CH; ++t) {
            const C f = LOWER ? Ps[ft[t] * r + q] : Ps[q * r + ft[t]];
#pragma unroll
            for (int c = 0; c < WARM_CW; ++c) acc[t][c] = acc[t][c] - f * x[c];
          }
        }
      } else {
#pragma unroll 2
        for (int q = 0; q < c0; ++q) {
          Op xv = act[0] ? X[(long long)q * ldx + jc[0]] : Op{};
          const C x0 = mk<T>(xv.re, xv.im);
#pragma unroll
          for (int t = 0; t < CH; ++t) {
            const C f = LOWER ? Ps[ft[t] * r + q] : Ps[q * r + ft[t]];
            acc[t][0] = acc[t][0] - f * x0;
          }
        }
      }
      // rows t >= nv are not stored; their factor reads are skipped below
#pragma unroll
      for (int t = 0; t < CH; ++t) {
        const bool rv = t < nv;
#pragma unroll
        for (int u = 0; u < t; ++u) {
          const C f = rv ? (LOWER ? Ps[(c0 + t) * r + c0 + u] : Ps[(c0 + u) * r + c0 + t]) : mk<T>(0, 0);
#pragma unroll
          for (int c = 0; c < WARM_CW; ++c) acc[t][c] = acc[t][c] - f * acc[u][c];
        }
        if (!LOWER) {
          const C id = rv ? inv(Ps[(c0 + t) * r + c0 + t]) : mk<T>(0, 0);
#pragma unroll
          for (int c = 0; c < WARM_CW; ++c) acc[t][c] = acc[t][c] * id;
        }
      }
      // stores and per-row reductions, CH rows at a time
      T a2[CH], mx[CH];
#pragma unroll
      for (int t = 0; t < CH; ++t) {
        a2[t] = 0;
        mx[t] = 0;
#pragma unroll
        for (int c = 0; c < WARM_CW; ++c)
          if (act[c] && t < nv) {
            X[(long long)(c0 + t) * ldx + jc[c]] = to_op<Op>(acc[t][c]);
            T e = abs2(acc[t][c]);
            a2[t] += e;
            mx[t] = max(mx[t], e);
          }
      }
#pragma unroll
      for (int o = 16; o > 0; o >>= 1)
#pragma unroll
        for (int t = 0; t < CH; ++t) {
          a2[t] += __shfl_xor_sync(0xffffffffu, a2[t], o);
          if (rowmax) mx[t] = max(mx[t], __shfl_xor_sync(0xffffffffu, mx[t], o));
        }
      if (lane < CH && lane < nv) {
        T sa = a2[0], sx = mx[0];
#pragma unroll
        for (int t = 1; t < CH; ++t)
          if (lane == t) {
            sa = a2[t];
            sx = mx[t];
          }
        if (rowmax) smem_max(&rowmax[c0 + lane], sx);
        sum_w[(c0 + lane) * NW + wid] += sa;
      }
    }
  }
}

// Per block: LU of P, V^T = L^{-1} R and U = C Uh^{-1} in place, the pivot
// test, and the ACA stopping test over the reused steps. Writes the state the
// ACA kernels continue from. One launch per rank class: this one handles the
// blocks with RLO < r <= RCAP with NT threads, its shared memory sized for
// RCAP. Blocks with nothing to reuse (r <= 0) are written as cold starts by
// the launch with RLO = 0, blocks above the last class's RCAP by the LAST one.
template <typename Op, int RLO, int RCAP, bool LAST, int NT, int CH>
__global__ void __launch_bounds__(NT) k_aca_warm_solve(const FarBlk* __restrict__ blks, int b0, Op* __restrict__ Ustore,
                                                       Op* __restrict__ Vstore, int* __restrict__ rank,
                                                       int* __restrict__ npiv, const int* __restrict__ piv_i,
                                                       const int* __restrict__ piv_j, int* __restrict__ kstart,
                                                       double* __restrict__ norm0, int* __restrict__ done,
                                                       double eps_d, double tau_d) {
  using T = decltype(Op{}.re);
  using C = cplx<T>;
  constexpr int NW = NT / 32;
  extern __shared__ __align__(16) unsigned char warm_smem[];
  C* Ps = reinterpret_cast<C*>(warm_smem);                 // r x r, row-major
  T* rowmax = reinterpret_cast<T*>(Ps + RCAP * RCAP);
  T* nv2w = rowmax + RCAP;                                 // [l][warp]
  T* nu2w = nv2w + RCAP * NW;
  __shared__ int sh_rp, sh_ls;
  const int bi = b0 + blockIdx.x;
  const int tid = threadIdx.x;
  const int r = npiv[bi];
  if (r <= RLO || r > RCAP) {
    if (((RLO == 0 && r <= 0) || (LAST && r > RCAP)) && tid == 0) {
      kstart[bi] = 0;
      norm0[bi] = 0.0;
      done[bi] = 0;
    }
    return;
  }
  const FarBlk B = blks[bi];
  const int m = 3 * B.nr, n = 3 * B.nc;
  Op* Ub = Ustore + B.uoff;
  Op* Vb = Vstore + B.voff;
  const int* pi = piv_i + B.toff;
  const int* pj = piv_j + B.toff;
  for (int idx = tid; idx < r * r; idx += NT) {
    int l = idx / r, q = idx - l * r;
    Op v = Vb[(long long)l * n + pj[q]];
    Ps[idx] = mk<T>(v.re, v.im);
  }
  for (int l = tid; l < RCAP; l += NT) {
    rowmax[l] = T(0);
    for (int w = 0; w < NW; ++w) nv2w[l * NW + w] = nu2w[l * NW + w] = T(0);
  }
  if (tid == 0) sh_rp = r;
  __syncthreads();
  // LU without pivoting, stopped at the first zero (or non-finite) pivot
  for (int l = 0; l < r; ++l) {
    C d = Ps[l * r + l];
    if (!(abs2(d) > T(0))) {  // uniform: every thread reads the same value
      if (tid == 0) sh_rp = l;
      break;
    }
    C id = inv(d);
    for (int p = l + 1 + tid; p < r; p += NT) Ps[p * r + l] = Ps[p * r + l] * id;
    __syncthreads();
    // trailing update: warps over rows, lanes over columns
    for (int p = l + 1 + (tid >> 5); p < r; p += NW) {
      const C lp = Ps[p * r + l];
      for (int q = l + 1 + (tid & 31); q < r; q += 32) Ps[p * r + q] = Ps[p * r + q] - lp * Ps[l * r + q];
    }
    __syncthreads();
  }
  __syncthreads();
  const int rp = sh_rp;
  // V^T <- L^{-1} R (rows of R are the columns of V)
  warm_trsm<Op, NT, CH, true>(Vb, n, n, rp, Ps, r, rowmax, nv2w);
  __syncthreads();
  if (tid == 0) {
    const T tau2 = T(tau_d * tau_d);
    int ls = rp;
    for (int l = 0; l < rp; ++l)
      if (abs2(Ps[l * r + l]) < tau2 * rowmax[l]) {
        ls = l;
        break;
      }
    sh_ls = ls;
  }
  __syncthreads();
  const int ls = sh_ls;
  // U <- C Uh^{-1} (columns of C stored as the columns of U)
  warm_trsm<Op, NT, CH, false>(Ub, m, m, ls, Ps, r, nullptr, nu2w);
  __syncthreads();
  // earlier pivot rows are represented exactly: zero them as ACA does
  for (int idx = tid; idx < ls * ls; idx += NT) {
    int q = idx / ls, p = idx % ls;
    if (p < q) Ub[(long long)q * m + pi[p]] = Op{};
  }
  if (tid == 0) {
    // the rank is the first step at which the stopping test holds after the
    // last step at which it fails: the reused pivots may cover parts of the
    // block that ACA reached only through its check rows (see k_aca)
    const T eps2 = T(eps_d * eps_d);
    T S = 0;
    int lastfail = -1;
    for (int l = 0; l < ls; ++l) {
      T nu = 0, nv = 0;
      for (int w = 0; w < NW; ++w) {
        nu += nu2w[l * NW + w];
        nv += nv2w[l * NW + w];
      }
      T term = nu * nv;
      S += term;
      if (!(term <= eps2 * S)) lastfail = l;
    }
    const int conv = lastfail + 1 < ls ? 1 : 0;
    const int kc = conv ? lastfail + 2 : ls;
    // converged: every validated step stays (the ones past the rank as
    // spares); on a block with flat faces, where partial pivoting can miss
    // the part of the block it has not visited, the ACA kernels evaluate the
    // check rows against all of them first
    kstart[bi] = ls;
    norm0[bi] = double(S);
    done[bi] = conv ? (B.flat ? 2 : 1) : 0;
    if (conv) {
      rank[bi] = kc;
      npiv[bi] = ls;
    }
  }
}

// ---------------------------------------------------------------------------
// launchers
// ---------------------------------------------------------------------------
void launch_centroids(const double* xyz, long long nv, const int* tri, int ne, double* cen, double* h,
                      int* bad, cudaStream_t st) {
  count_if(true);
  k_centroids<<<(ne + 127) / 128, 128, 0, st>>>(xyz, nv, tri, ne, cen, h, bad);
}
void launch_geometry(const double* xyz, const int* tri, const int* perm, const signed char* bc_in, int ne,
                     ElemF* ef, ElemD* ed, signed char* bc, cudaStream_t st) {
  count_if(true);
  k_geometry<<<(ne + 127) / 128, 128, 0, st>>>(xyz, tri, perm, bc_in, ne, ef, ed, bc);
}
void launch_sing_count(const NearBlk* blks, int nblk, const ElemD* ed, int* count, cudaStream_t st) {
  if (count_if(nblk)) k_sing_count<<<nblk, 256, 0, st>>>(blks, ed, count);
}
void launch_sing_fill(const NearBlk* blks, int nblk, const ElemD* ed, const int* offs, SingPair* out,
                      cudaStream_t st) {
  if (count_if(nblk)) k_sing_fill<<<nblk, 256, 0, st>>>(blks, ed, offs, out);
}
void launch_static(const SingPair* pairs, int n, const ElemD* ed, const KParams<double>& P, double* out, bool fp32,
                   cudaStream_t st) {
  if (!count_if(n)) return;
  if (fp32) k_static<float><<<(n + 3) / 4, 128, 0, st>>>(pairs, n, ed, P, out);
  else k_static<double><<<(n + 3) / 4, 128, 0, st>>>(pairs, n, ed, P, out);
}
void launch_pair_sort(const NearBlk* blks, int nblk, const ElemF* ef, const ElemD* ed, const long long* poff,
                      unsigned* plist, int* pcount, cudaStream_t st) {
  if (count_if(nblk)) k_pair_sort<<<nblk, 1024, 0, st>>>(blks, ef, ed, poff, plist, pcount);
}
template <typename R, typename Op>
void launch_near_regular(const NearBlk* blks, int nblk, int max_nr, const unsigned* plist, const long long* poff,
                         const int* pcount, const ElemF* ef, const ElemD* ed, const signed char* bc,
                         const KParams<R>& P, Op* near, const float* patf, const double* patd, c128 pk, c128* b,
                         cudaStream_t st) {
  size_t sm = b ? 6 * sizeof(R) * max_nr : 0;
  if (count_if(nblk))
    k_near_regular<R, Op><<<nblk, 256, sm, st>>>(blks, plist, poff, pcount, ef, ed, bc, P, near, patf, patd, pk, b);
}
void launch_polar(const ElemD* ed, int ne, double* out, cudaStream_t st) {
  count_if(true);
  k_polar<<<(ne + 127) / 128, 128, 0, st>>>(ed, ne, out);
}
template <typename R, typename Op>
void launch_sing(const SingPair* pairs, int n, const ElemD* ed, const double* polar, const signed char* bc,
                 const double* stat, const KParams<R>& P, Op* near, c128* pinv, const double* pattern, c128 pk,
                 c128* b, int* status, cudaStream_t st) {
  if (count_if(n))
    k_sing<R, Op><<<(n + 15) / 16, 256, 0, st>>>(pairs, n, ed, polar, bc, stat, P, near, pinv, pattern, pk, b, status);
}
template <typename R>
void launch_rhs_far(const int* rng, const int* rptr, const int* elem_leaf, int ne, const ElemF* ef, const ElemD* ed,
                    const signed char* bc, const float* patf, const double* patd, const KParams<R>& P, c128 pk,
                    c128* b, cudaStream_t st) {
  if (count_if(ne)) k_rhs_far<R><<<(ne + 7) / 8, 256, 0, st>>>(rng, rptr, elem_leaf, ne, ef, ed, bc, patf, patd, P, pk, b);
}
template <typename R, typename Op>
void launch_aca(const FarBlk* blks, const int* small_list, int nsmall, const int* large_list, int nlarge,
                const ElemF* ef, const ElemD* ed, const signed char* bc, const KParams<R>& P, Op* U, Op* V, int* rank,
                int* fails, double eps, const AcaState& state, cudaStream_t st) {
  if (count_if(nlarge))
    k_aca<R, Op><<<nlarge, ACA_THREADS, 0, st>>>(large_list, blks, ef, ed, bc, P, U, V, rank, fails, eps, state);
  if (!nsmall) return;
  count_if(true);
  if (state.done) {
    // continuation after pivot reuse: few blocks, a few steps each; one CTA
    // per block shortens each step (blocks already settled exit at once)
    k_aca<R, Op><<<nsmall, ACA_THREADS, 0, st>>>(small_list, blks, ef, ed, bc, P, U, V, rank, fails, eps, state);
  } else {
    k_aca_warp<R, Op><<<(nsmall + ACAW_WARPS - 1) / ACAW_WARPS, 32 * ACAW_WARPS, 0, st>>>(
        small_list, nsmall, blks, ef, ed, bc, P, U, V, rank, fails, eps, state);
  }
}

template <typename Op> size_t warm_solve_smem(int rcap, int nt) {
  using T = decltype(Op{}.re);
  return sizeof(cplx<T>) * rcap * rcap + sizeof(T) * rcap * (1 + 2 * (nt / 32));
}

template <typename Op, int RLO, int RCAP, bool LAST, int NT, int CH>
cudaError_t launch_warm_solve(const FarBlk* blks, int b0, int nfar, Op* U, Op* V, int* rank, int* npiv, const int* piv_i,
                              const int* piv_j, int* kstart, double* norm0, int* done, double eps, double tau,
                              cudaStream_t st) {
  const size_t sm = warm_solve_smem<Op>(RCAP, NT);
  static_assert(sizeof(Op) * RCAP * RCAP <= 200 * 1024, "pivot block must fit in shared memory");
  cudaError_t e = cudaFuncSetAttribute(k_aca_warm_solve<Op, RLO, RCAP, LAST, NT, CH>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
  if (e != cudaSuccess) return e;
  count_if(true);
  k_aca_warm_solve<Op, RLO, RCAP, LAST, NT, CH><<<nfar, NT, sm, st>>>(blks, b0, U, V, rank, npiv, piv_i, piv_j,
                                                                      kstart, norm0, done, eps, tau);
  return cudaGetLastError();
}

template <typename R, typename Op>
cudaError_t launch_aca_warm(const FarBlk* blks, int b0, int nfar, const ElemF* ef, const ElemD* ed,
                            const signed char* bc, const KParams<R>& P, Op* U, Op* V, int* rank, int* npiv,
                            int* piv_i, int* piv_j, int* kstart, double* norm0, int* done, double eps, double tau,
                            cudaStream_t st) {
  if (!nfar) return cudaSuccess;
  count_if(true);
  k_aca_warm_eval<R, Op><<<nfar, WARM_THREADS, 0, st>>>(blks, b0, ef, ed, bc, P, U, V, npiv, piv_i, piv_j);
  // rank classes (0, 64] and (64, 128]; complex128 pivot blocks above rank
  // 112 do not fit in shared memory and restart ACA
  constexpr int RTOP = sizeof(Op) == 8 ? WARM_RMAX : 112;
  cudaError_t e = launch_warm_solve<Op, 0, WARM_SPLIT, false, 128, 8>(blks, b0, nfar, U, V, rank, npiv, piv_i, piv_j,
                                                                      kstart, norm0, done, eps, tau, st);
  if (e != cudaSuccess) return e;
  return launch_warm_solve<Op, WARM_SPLIT, RTOP, true, 256, 16>(blks, b0, nfar, U, V, rank, npiv, piv_i, piv_j, kstart,
                                                                norm0, done, eps, tau, st);
}

// ---------------------------------------------------------------------------
// far-field factor storage
// ---------------------------------------------------------------------------
// Full storage: the factors stay where ACA wrote them.
__global__ void k_fbase_full(const FarBlk* __restrict__ blks, int nfar, long long* __restrict__ fbase) {
  int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= nfar) return;
  fbase[2 * b] = blks[b].uoff;
  fbase[2 * b + 1] = blks[b].voff;
}

// Compact storage: block b0 + blockIdx.x takes 3 nr rank and 3 nc rank
// entries from the pool cursors and copies the first rank columns of its U
// and V (contiguous, column-major) out of the workspace. The cursors count
// the full need even past the pools' capacity; a block that does not fit is
// not copied (the host sees the overflow and redoes the assembly).
template <typename Op>
__global__ void __launch_bounds__(256) k_far_pack(const FarBlk* __restrict__ blks, int b0, const int* __restrict__ rank,
                                                  const Op* __restrict__ wsU, const Op* __restrict__ wsV,
                                                  Op* __restrict__ U, Op* __restrict__ V, long long capU,
                                                  long long capV, long long* __restrict__ fbase,
                                                  unsigned long long* __restrict__ cursor) {
  const int b = b0 + blockIdx.x;
  const FarBlk B = blks[b];
  const int r = rank[b];
  const long long nu = 3LL * B.nr * r, nv = 3LL * B.nc * r;
  __shared__ long long ou, ov;
  if (threadIdx.x == 0) {
    ou = (long long)atomicAdd(&cursor[0], (unsigned long long)nu);
    ov = (long long)atomicAdd(&cursor[1], (unsigned long long)nv);
    fbase[2 * b] = ou;
    fbase[2 * b + 1] = ov;
  }
  __syncthreads();
  if (ou + nu > capU || ov + nv > capV) return;
  const Op* su = wsU + B.uoff;
  const Op* sv = wsV + B.voff;
  Op* du = U + ou;
  Op* dv = V + ov;
  for (long long i = threadIdx.x; i < nu; i += blockDim.x) du[i] = su[i];
  for (long long i = threadIdx.x; i < nv; i += blockDim.x) dv[i] = sv[i];
}

void launch_fbase_full(const FarBlk* blks, int nfar, long long* fbase, cudaStream_t st) {
  if (count_if(nfar)) k_fbase_full<<<(nfar + 255) / 256, 256, 0, st>>>(blks, nfar, fbase);
}

template <typename Op>
void launch_far_pack(const FarBlk* blks, int b0, int nblk, const int* rank, const Op* wsU, const Op* wsV, Op* U,
                     Op* V, long long capU, long long capV, long long* fbase, unsigned long long* cursor,
                     cudaStream_t st) {
  if (count_if(nblk))
    k_far_pack<Op><<<nblk, 256, 0, st>>>(blks, b0, rank, wsU, wsV, U, V, capU, capV, fbase, cursor);
}

template void launch_far_pack<c64>(const FarBlk*, int, int, const int*, const c64*, const c64*, c64*, c64*,
                                   long long, long long, long long*, unsigned long long*, cudaStream_t);
template void launch_far_pack<c128>(const FarBlk*, int, int, const int*, const c128*, const c128*, c128*, c128*,
                                    long long, long long, long long*, unsigned long long*, cudaStream_t);

template void launch_near_regular<float, c64>(const NearBlk*, int, int, const unsigned*, const long long*,
                                              const int*, const ElemF*, const ElemD*, const signed char*,
                                              const KParams<float>&, c64*, const float*, const double*, c128, c128*,
                                              cudaStream_t);
template void launch_near_regular<double, c128>(const NearBlk*, int, int, const unsigned*, const long long*,
                                                const int*, const ElemF*, const ElemD*, const signed char*,
                                                const KParams<double>&, c128*, const float*, const double*, c128,
                                                c128*, cudaStream_t);
template void launch_sing<float, c64>(const SingPair*, int, const ElemD*, const double*, const signed char*,
                                      const double*, const KParams<float>&, c64*, c128*, const double*, c128,
                                      c128*, int*, cudaStream_t);
template void launch_sing<double, c128>(const SingPair*, int, const ElemD*, const double*, const signed char*,
                                        const double*, const KParams<double>&, c128*, c128*, const double*, c128,
                                        c128*, int*, cudaStream_t);
template void launch_rhs_far<float>(const int*, const int*, const int*, int, const ElemF*, const ElemD*,
                                     const signed char*, const float*, const double*, const KParams<float>&, c128,
                                     c128*, cudaStream_t);
template void launch_rhs_far<double>(const int*, const int*, const int*, int, const ElemF*, const ElemD*,
                                      const signed char*, const float*, const double*, const KParams<double>&, c128,
                                      c128*, cudaStream_t);
template void launch_aca<float, c64>(const FarBlk*, const int*, int, const int*, int, const ElemF*, const ElemD*,
                                     const signed char*, const KParams<float>&, c64*, c64*, int*, int*, double,
                                     const AcaState&, cudaStream_t);
template void launch_aca<double, c128>(const FarBlk*, const int*, int, const int*, int, const ElemF*,
                                       const ElemD*, const signed char*, const KParams<double>&, c128*, c128*, int*,
                                       int*, double, const AcaState&, cudaStream_t);
template cudaError_t launch_aca_warm<float, c64>(const FarBlk*, int, int, const ElemF*, const ElemD*, const signed char*,
                                                 const KParams<float>&, c64*, c64*, int*, int*, int*, int*, int*,
                                                 double*, int*, double, double, cudaStream_t);
template cudaError_t launch_aca_warm<double, c128>(const FarBlk*, int, int, const ElemF*, const ElemD*,
                                                   const signed char*, const KParams<double>&, c128*, c128*, int*,
                                                   int*, int*, int*, int*, double*, int*, double, double,
                                                   cudaStream_t);

}  // namespace bem
