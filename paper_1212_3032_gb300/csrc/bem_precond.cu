// Leaf-block preconditioner: the inverses of the operator's diagonal blocks
// over the cluster tree's leaves (up to 64 elements, 192 x 192 complex), a
// block-Jacobi preconditioner with larger blocks than the 3 x 3 one of
// Sec. 3.1 / Sec. 5 (the paper does not state the block size).
//
//   k_leaf_inverse  one thread-block cluster per leaf (C CTAs): in-place
//                   Gauss-Jordan elimination with partial pivoting (row
//                   interchanges, undone as column interchanges at the end).
//                   The block does not fit one CTA's shared memory (288 KB
//                   in complex64), so each CTA holds ceil(m / C) rows; the
//                   pivot search, the pivot row and the displaced row move
//                   between the CTAs through distributed shared memory.
//                   Complex64 blocks: FP32 arithmetic, C = 2; complex128:
//                   FP64, C = 4. A singular pivot (never seen on boundary
//                   element blocks with eta > 0) makes the leaf fall back to
//                   its 3 x 3 block-diagonal inverses.
//   k_leaf_apply    z = M^-1 v: one CTA per leaf, pairs of rows per thread,
//                   column groups added in shared memory.
#include <type_traits>

#include <cooperative_groups.h>

#include "bem_internal.h"
#include "bem_launch.h"

namespace bem {

namespace cg = cooperative_groups;

namespace {

constexpr int LI_THREADS = 512;
constexpr int LI_MAXM = 3 * LEAF_PRE_MAX_ELEMS;  // rows of the largest leaf block

template <typename R> __device__ __forceinline__ cplx<R> cmul(cplx<R> a, cplx<R> b) {
  return cplx<R>{a.re * b.re - a.im * b.im, a.re * b.im + a.im * b.re};
}
template <typename R> __device__ __forceinline__ cplx<R> crecip(cplx<R> a) {
  const R d = a.re * a.re + a.im * a.im;
  return cplx<R>{a.re / d, -a.im / d};
}

template <typename R, int C>
__global__ void __cluster_dims__(C, 1, 1) __launch_bounds__(LI_THREADS) k_leaf_inverse(
    const LeafPre* __restrict__ leaves, const cplx<R>* __restrict__ near, const c128* __restrict__ pinv3,
    cplx<R>* __restrict__ out) {
  cg::cluster_group cl = cg::this_cluster();
  const int crank = (int)cl.block_rank();
  const LeafPre L = leaves[blockIdx.x / C];
  const int m = L.m;
  const int h = (m + C - 1) / C;
  const int i0 = crank * h, i1 = min(m, i0 + h), hr = max(0, i1 - i0);
  const int S = m + 1;  // row stride in shared memory (odd: rows fall in different banks)
  extern __shared__ unsigned char smem_raw[];
  cplx<R>* A = reinterpret_cast<cplx<R>*>(smem_raw);  // hr x S, row-major
  cplx<R>* prow = A + (size_t)h * S;                    // the pivot row (m)
  cplx<R>* swp = prow + m;                              // a displaced row k arriving here (m)
  cplx<R>* fcol = swp + m;                              // column k of the owned rows (h)
  __shared__ R cand_v;
  __shared__ int cand_i;
  __shared__ R wv[LI_THREADS / 32];
  __shared__ int wi[LI_THREADS / 32];
  __shared__ int piv[LI_MAXM];
  __shared__ int singular;
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
  if (tid == 0) singular = 0;
  for (int idx = tid; idx < hr * m; idx += LI_THREADS) {
    const int j = idx / hr, i = idx - j * hr;
    A[(size_t)i * S + j] = near[L.off + (long long)j * L.ld + i0 + i];
  }
  __syncthreads();
  for (int k = 0; k < m; ++k) {
    // 1. the largest |a_ik|, i >= k, among the owned rows
    R best = R(-1);
    int bi = -1;
    for (int i = max(i0, k) + tid; i < i1; i += LI_THREADS) {
      const cplx<R> a = A[(size_t)(i - i0) * S + k];
      const R v = a.re * a.re + a.im * a.im;
      if (v > best) {
        best = v;
        bi = i;
      }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      const R ov = __shfl_xor_sync(0xffffffffu, best, o);
      const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
      if (ov > best || (ov == best && oi >= 0 && (bi < 0 || oi < bi))) {
        best = ov;
        bi = oi;
      }
    }
    if (lane == 0) {
      wv[wid] = best;
      wi[wid] = bi;
    }
    __syncthreads();
    if (tid == 0) {
      R b = R(-1);
      int ib = -1;
      for (int w = 0; w < LI_THREADS / 32; ++w)
        if (wv[w] > b || (wv[w] == b && wi[w] >= 0 && (ib < 0 || wi[w] < ib))) {
          b = wv[w];
          ib = wi[w];
        }
      cand_v = b;
      cand_i = ib;
    }
    cl.sync();  // every CTA's candidate is posted
    // 2. the pivot: the largest candidate (ties: the smaller row), the same in every CTA
    R pv = R(-1);
    int p = -1;
    for (int c = 0; c < C; ++c) {
      const R v = *cl.map_shared_rank(&cand_v, c);
      const int i = *cl.map_shared_rank(&cand_i, c);
      if (v > pv || (v == pv && i >= 0 && (p < 0 || i < p))) {
        pv = v;
        p = i;
      }
    }
    if (!(pv > R(0))) {  // singular (or not finite): every CTA takes the same exit
      if (tid == 0) singular = 1;
      break;
    }
    if (tid == 0) piv[k] = p;
    const int own_p = p / h, own_k = k / h;
    // 3. the pivot row to every CTA; the displaced row k to the owner of row p
    if (crank == own_p) {
      for (int j = tid; j < m; j += LI_THREADS) {
        const cplx<R> v = A[(size_t)(p - i0) * S + j];
        for (int c = 0; c < C; ++c) cl.map_shared_rank(prow, c)[j] = v;
      }
    }
    if (crank == own_k && p != k) {
      cplx<R>* dst = cl.map_shared_rank(swp, own_p);
      for (int j = tid; j < m; j += LI_THREADS) dst[j] = A[(size_t)(k - i0) * S + j];
    }
    cl.sync();
    if (p != k) {
      if (crank == own_p)
        for (int j = tid; j < m; j += LI_THREADS) A[(size_t)(p - i0) * S + j] = swp[j];
      if (crank == own_k)
        for (int j = tid; j < m; j += LI_THREADS) A[(size_t)(k - i0) * S + j] = prow[j];
    }
    // 4. column k of the owned rows, then the normalised pivot row
    for (int i = tid; i < hr; i += LI_THREADS) fcol[i] = A[(size_t)i * S + k];
    const cplx<R> ip = crecip(prow[k]);
    __syncthreads();
    for (int j = tid; j < m; j += LI_THREADS) prow[j] = (j == k) ? ip : cmul(prow[j], ip);
    __syncthreads();
    // 5. eliminate column k from every other row; row k becomes the normalised pivot row
    for (int idx = tid; idx < hr * m; idx += LI_THREADS) {
      const int i = idx / m, j = idx - i * m;
      cplx<R>& a = A[(size_t)i * S + j];
      if (i0 + i == k) {
        a = prow[j];
      } else {
        const cplx<R> f = fcol[i];
        if (j == k) {
          a = cplx<R>{-(f.re * ip.re - f.im * ip.im), -(f.re * ip.im + f.im * ip.re)};
        } else {
          const cplx<R> q = prow[j];
          a.re -= f.re * q.re - f.im * q.im;
          a.im -= f.re * q.im + f.im * q.re;
        }
      }
    }
    __syncthreads();
  }
  cl.sync();  // no CTA leaves while another may still read its shared memory
  const long long o = L.ooff;
  if (singular) {
    // fall back to the 3 x 3 block-diagonal inverses of the leaf's elements
    for (int idx = tid; idx < hr * m; idx += LI_THREADS) {
      const int j = idx / hr, r = i0 + idx - j * hr;
      cplx<R> v{R(0), R(0)};
      if (r / 3 == j / 3) {
        const c128 w = pinv3[9LL * (L.e0 + r / 3) + 3 * (r % 3) + (j % 3)];
        v = cplx<R>{R(w.re), R(w.im)};
      }
      out[o + (long long)j * L.ldo + r] = v;
    }
    return;
  }
  // undo the row interchanges as column interchanges, last first
  for (int k = m - 1; k >= 0; --k) {
    const int p = piv[k];
    if (p != k)
      for (int i = tid; i < hr; i += LI_THREADS) {
        const cplx<R> t = A[(size_t)i * S + k];
        A[(size_t)i * S + k] = A[(size_t)i * S + p];
        A[(size_t)i * S + p] = t;
      }
    __syncthreads();
  }
  for (int idx = tid; idx < hr * m; idx += LI_THREADS) {
    const int j = idx / hr, i = idx - j * hr;
    out[o + (long long)j * L.ldo + i0 + i] = A[(size_t)i * S + j];
  }
}

// z[rows of leaf] = M_leaf^-1 v[rows of leaf] (column-major inverse, ldo even);
// run / joff as for the 3 x 3 blocks (a launch that does nothing unless *run,
// v read from v + (*joff) ldv)
constexpr int LA_THREADS = 256;
template <typename Pm, typename V, typename Z>
__global__ void __launch_bounds__(LA_THREADS) k_leaf_apply(const LeafPre* __restrict__ leaves,
                                                           const Pm* __restrict__ minv, const V* __restrict__ v,
                                                           Z* __restrict__ z, const int* __restrict__ run,
                                                           const int* __restrict__ joff, long long ldv) {
  if (run && !*run) return;
  if (joff) v += (long long)(*joff) * ldv;
  using Acc = std::conditional_t<(sizeof(Pm) == 16 || sizeof(V) == 16), double, float>;
  __shared__ cplx<Acc> red[LA_THREADS];
  const LeafPre L = leaves[blockIdx.x];
  const int m = L.m;
  const long long row0 = 3LL * L.e0;
  const int G = max(1, LA_THREADS / m);
  for (int rbase = 0; rbase < m; rbase += LA_THREADS) {
    const int rc = min(m - rbase, LA_THREADS);
    const int Gr = max(1, LA_THREADS / rc);
    const int g = threadIdx.x / rc, r = threadIdx.x % rc + rbase;
    const bool active = g < Gr;
    cplx<Acc> acc{Acc(0), Acc(0)};
    if (active) {
      const Pm* col = minv + L.ooff + r;
      int j = g;
      for (; j + 3 * Gr < m; j += 4 * Gr) {
        Pm a[4];
        V x[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          a[u] = col[(long long)(j + u * Gr) * L.ldo];
          x[u] = v[row0 + j + u * Gr];
        }
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          const Acc ar = a[u].re, ai = a[u].im, xr = x[u].re, xi = x[u].im;
          acc.re = fma(ar, xr, fma(-ai, xi, acc.re));
          acc.im = fma(ar, xi, fma(ai, xr, acc.im));
        }
      }
      for (; j < m; j += Gr) {
        const Pm a = col[(long long)j * L.ldo];
        const V x = v[row0 + j];
        const Acc ar = a.re, ai = a.im, xr = x.re, xi = x.im;
        acc.re = fma(ar, xr, fma(-ai, xi, acc.re));
        acc.im = fma(ar, xi, fma(ai, xr, acc.im));
      }
    }
    red[threadIdx.x] = acc;
    __syncthreads();
    if (active && g == 0) {
      for (int gg = 1; gg < Gr; ++gg) {
        acc.re += red[gg * rc + (r - rbase)].re;
        acc.im += red[gg * rc + (r - rbase)].im;
      }
      Z o;
      o.re = decltype(o.re)(acc.re);
      o.im = decltype(o.im)(acc.im);
      z[row0 + r] = o;
    }
    __syncthreads();
  }
  (void)G;
}

template <typename R, int C> size_t leaf_inverse_smem() {
  const int m = LI_MAXM, h = (m + C - 1) / C;
  return ((size_t)h * (m + 1) + 2 * (size_t)m + h) * sizeof(cplx<R>);
}

}  // namespace

template <typename R>
cudaError_t launch_leaf_inverse(const LeafPre* leaves, int nleaves, const cplx<R>* near, const c128* pinv3,
                                cplx<R>* out, cudaStream_t st) {
  if (!count_if(nleaves > 0)) return cudaSuccess;
  constexpr int C = sizeof(R) == 4 ? 2 : 4;
  const size_t sm = leaf_inverse_smem<R, C>();
  static bool attr_set[64] = {};
  int dev = 0;
  cudaGetDevice(&dev);
  if (dev < 0 || dev >= 64 || !attr_set[dev]) {
    cudaError_t e = cudaFuncSetAttribute(k_leaf_inverse<R, C>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (e != cudaSuccess) return e;
    if (dev >= 0 && dev < 64) attr_set[dev] = true;
  }
  k_leaf_inverse<R, C><<<nleaves * C, LI_THREADS, sm, st>>>(leaves, near, pinv3, out);
  return cudaGetLastError();
}

template <typename Pm, typename V, typename Z>
void launch_leaf_apply(const LeafPre* leaves, int nleaves, const Pm* minv, const V* v, Z* z, cudaStream_t st,
                       const int* run, const int* joff, long long ldv) {
  if (!count_if(nleaves > 0)) return;
  k_leaf_apply<Pm, V, Z><<<nleaves, LA_THREADS, 0, st>>>(leaves, minv, v, z, run, joff, ldv);
}

template cudaError_t launch_leaf_inverse<float>(const LeafPre*, int, const cplx<float>*, const c128*, cplx<float>*,
                                               cudaStream_t);
template cudaError_t launch_leaf_inverse<double>(const LeafPre*, int, const cplx<double>*, const c128*,
                                                cplx<double>*, cudaStream_t);
template void launch_leaf_apply<c64, c64, c64>(const LeafPre*, int, const c64*, const c64*, c64*, cudaStream_t,
                                               const int*, const int*, long long);
template void launch_leaf_apply<c64, c128, c128>(const LeafPre*, int, const c64*, const c128*, c128*, cudaStream_t,
                                                 const int*, const int*, long long);
template void launch_leaf_apply<c128, c128, c128>(const LeafPre*, int, const c128*, const c128*, c128*,
                                                  cudaStream_t, const int*, const int*, long long);

}  // namespace bem
