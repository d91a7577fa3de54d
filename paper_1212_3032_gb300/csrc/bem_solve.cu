// Solver kernels: hierarchical matrix-vector product, block-Jacobi
// preconditioner, Arnoldi pieces with FP64 accumulation, and the modified
// Fourier transforms (Sec. 3.3, Eqs. DFT-MFT and IDFT-MFT).
//
// H-matrix product (HBM-bound): y = D_near x + sum_b U_b (V_b^T x)
//   k_hmv_fused  the product of the solver: one launch, one CTA per work item
//                (near panels of a leaf row, or the admissible blocks of one
//                row cluster), 16-byte loads, per-item partial rows summed in
//                a fixed order by the item that completes a leaf
//   k_hmv_t, k_hmv_tasks, k_hmv_reduce  the same product in three launches
//                with caller-provided scratch (bem_apply_noalloc):
//     k_hmv_t     t_b = V_b^T x for every admissible block (one CTA per block,
//                 one warp per factor column, coalesced column reads)
//     k_hmv_tasks one CTA per task (a run of panels of one leaf row: dense near
//                 blocks and slices of the U_b factors), every stored entry
//                 read once, coalesced across rows (column-major storage),
//                 partial row sums to a per-task slot; no atomics
//     k_hmv_reduce per leaf row, the task slots summed in a fixed order
#include <algorithm>

#include <cooperative_groups.h>

#include "bem_internal.h"
#include "bem_launch.h"

namespace bem {

namespace cg = cooperative_groups;

template <typename A, typename B> struct Promote;
template <> struct Promote<float, float> { using type = float; };
template <> struct Promote<float, double> { using type = double; };
template <> struct Promote<double, float> { using type = double; };
template <> struct Promote<double, double> { using type = double; };

template <typename Acc, typename T> __device__ __forceinline__ cplx<Acc> up(const cplx<T>& v) {
  return cplx<Acc>{Acc(v.re), Acc(v.im)};
}

// streaming (evict-first) loads of operator entries, read once per product
__device__ __forceinline__ c64 ld_stream(const c64* p) {
  float2 v = __ldcs(reinterpret_cast<const float2*>(p));
  return c64{v.x, v.y};
}
__device__ __forceinline__ c128 ld_stream(const c128* p) {
  double2 v = __ldcs(reinterpret_cast<const double2*>(p));
  return c128{v.x, v.y};
}

// loads that bypass L1 (data written by other CTAs of the same launch)
__device__ __forceinline__ cplx<float> ld_global_cg(const cplx<float>* p) {
  float2 v = __ldcg(reinterpret_cast<const float2*>(p));
  return cplx<float>{v.x, v.y};
}
__device__ __forceinline__ cplx<double> ld_global_cg(const cplx<double>* p) {
  double2 v = __ldcg(reinterpret_cast<const double2*>(p));
  return cplx<double>{v.x, v.y};
}

template <typename Acc>
__device__ __forceinline__ void cmac(cplx<Acc>& acc, const cplx<Acc>& a, const cplx<Acc>& b) {
  acc.re = fma(a.re, b.re, fma(-a.im, b.im, acc.re));
  acc.im = fma(a.re, b.im, fma(a.im, b.re, acc.im));
}

template <typename Acc> __device__ __forceinline__ Acc wsum(Acc v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// ---------------------------------------------------------------------------
// phase 1: t_b = V_b^T x_sigma
// ---------------------------------------------------------------------------
template <typename Op, typename X, typename Acc, int NRHS>
__device__ __forceinline__ void hmv_t_block(int bi, const FarBlk* __restrict__ blks, const int* __restrict__ rank,
                                            const long long* __restrict__ fbase, const Op* __restrict__ V,
                                            const X* __restrict__ x, long long N,
                                            cplx<Acc>* __restrict__ t, int tstride) {
  // one warp per 4 factor columns: 4 independent coalesced column streams in flight
  constexpr int C = 4;
  FarBlk B = blks[bi];
  int r = rank[bi];
  int n = 3 * B.nc;
  const X* xs = x + 3LL * B.c0;
  int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
  for (int l0 = warp * C; l0 < r; l0 += nw * C) {
    const int nc = min(C, r - l0);
    const Op* col = V + fbase[2 * bi + 1] + (long long)l0 * n;
    cplx<Acc> acc[C][NRHS];
#pragma unroll
    for (int c = 0; c < C; ++c)
#pragma unroll
      for (int q = 0; q < NRHS; ++q) acc[c][q] = cplx<Acc>{0, 0};
    for (int j = lane; j < n; j += 32) {
      cplx<Acc> xv[NRHS];
#pragma unroll
      for (int q = 0; q < NRHS; ++q) xv[q] = up<Acc>(xs[q * N + j]);
#pragma unroll
      for (int c = 0; c < C; ++c) {
        if (c < nc) {
          cplx<Acc> v = up<Acc>(col[(long long)c * n + j]);
#pragma unroll
          for (int q = 0; q < NRHS; ++q) cmac(acc[c][q], v, xv[q]);
        }
      }
    }
#pragma unroll
    for (int c = 0; c < C; ++c) {
#pragma unroll
      for (int q = 0; q < NRHS; ++q) {
        Acc re = wsum(acc[c][q].re), im = wsum(acc[c][q].im);
        if (lane == 0 && c < nc) t[(long long)q * tstride + B.toff + l0 + c] = cplx<Acc>{re, im};
      }
    }
  }
}

template <typename Op, typename X, typename Acc, int NRHS>
__global__ void __launch_bounds__(256) k_hmv_t(const FarBlk* __restrict__ blks, const int* __restrict__ rank,
                                               const long long* __restrict__ fbase, const Op* __restrict__ V,
                                               const X* __restrict__ x, long long N, cplx<Acc>* __restrict__ t,
                                               int tstride) {
  hmv_t_block<Op, X, Acc, NRHS>(blockIdx.x, blks, rank, fbase, V, x, N, t, tstride);
}

// ---------------------------------------------------------------------------
// phase 2: one CTA per task (a run of column panels of one leaf row). Each
// thread owns one row of the leaf and one of G column groups; every column
// of a panel is read once, coalesced across the rows (column-major blocks),
// 8 independent loads in flight per thread. Partial row sums go to the task's
// slot of the partial buffer (no atomics).
// ---------------------------------------------------------------------------
constexpr int HMV_THREADS = 384;

template <typename Op, typename X, typename Acc, int NRHS>
__device__ __forceinline__ void hmv_task(
    const Task tk, const int* __restrict__ leaf_nr, const Panel* __restrict__ panels,
    const FarBlk* __restrict__ far, const int* __restrict__ rank, const long long* __restrict__ fbase,
    const Op* __restrict__ near,
    const Op* __restrict__ U, const cplx<Acc>* __restrict__ t, int tstride, const X* __restrict__ x, long long N,
    cplx<Acc>* __restrict__ part, long long pstride, cplx<Acc>* red) {
  const int rows = 3 * leaf_nr[tk.leaf];
  for (int rbase = 0; rbase < rows; rbase += blockDim.x) {
    const int rcount = min(rows - rbase, (int)blockDim.x);
    const int G = max(1, (int)blockDim.x / rcount);
    const int g = threadIdx.x / rcount;
    const int r = threadIdx.x % rcount + rbase;
    const bool active = g < G;
    cplx<Acc> acc[NRHS];
#pragma unroll
    for (int q = 0; q < NRHS; ++q) acc[q] = cplx<Acc>{0, 0};
    if (active) {
      for (int p = tk.p0; p < tk.p1; ++p) {
        const Panel P = panels[p];
        const long long ld = P.ld;
        if (P.kind == 0) {
          const Op* d = near + P.data + r;
          const X* xs = x + P.xoff;
          const int nc = P.ncols;
          const long long step = (long long)G * ld;
          int j = g;
          const Op* dp = d + (long long)g * ld;
          for (; j + 7 * G < nc; j += 8 * G, dp += 8 * step) {
            // all 8 column entries and x values of this group in flight before any FMA
            Op av[8];
#pragma unroll
            for (int u = 0; u < 8; ++u) av[u] = ld_stream(dp + u * step);
            X xv[NRHS][8];
#pragma unroll
            for (int q = 0; q < NRHS; ++q)
#pragma unroll
              for (int u = 0; u < 8; ++u) xv[q][u] = xs[q * N + j + u * G];
#pragma unroll
            for (int q = 0; q < NRHS; ++q)
#pragma unroll
              for (int u = 0; u < 8; ++u) cmac(acc[q], up<Acc>(av[u]), up<Acc>(xv[q][u]));
          }
          for (; j < nc; j += G) {
            cplx<Acc> a0 = up<Acc>(d[(long long)j * ld]);
#pragma unroll
            for (int q = 0; q < NRHS; ++q) cmac(acc[q], a0, up<Acc>(xs[q * N + j]));
          }
        } else {
          const int b = P.xoff;
          const int nc = rank[b];
          const Op* d = U + fbase[2 * b] + P.data + r;
          const cplx<Acc>* ts = t + far[b].toff;
          int j = g;
          for (; j + 3 * G < nc; j += 4 * G) {
            cplx<Acc> a[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) a[u] = up<Acc>(d[(long long)(j + u * G) * ld]);
#pragma unroll
            for (int q = 0; q < NRHS; ++q)
#pragma unroll
              for (int u = 0; u < 4; ++u) cmac(acc[q], a[u], ts[(long long)q * tstride + j + u * G]);
          }
          for (; j < nc; j += G) {
            cplx<Acc> a0 = up<Acc>(d[(long long)j * ld]);
#pragma unroll
            for (int q = 0; q < NRHS; ++q) cmac(acc[q], a0, ts[(long long)q * tstride + j]);
          }
        }
      }
    }
    if (G > 1) {
      if (active) {
#pragma unroll
        for (int q = 0; q < NRHS; ++q) red[(q * G + g) * rcount + (r - rbase)] = acc[q];
      }
      __syncthreads();
      if (active && g == 0) {
        for (int gg = 1; gg < G; ++gg)
#pragma unroll
          for (int q = 0; q < NRHS; ++q) {
            cplx<Acc> o = red[(q * G + gg) * rcount + (r - rbase)];
            acc[q].re += o.re;
            acc[q].im += o.im;
          }
      }
      __syncthreads();
    }
    if (active && g == 0) {
#pragma unroll
      for (int q = 0; q < NRHS; ++q) part[q * pstride + tk.slot + r] = acc[q];
    }
  }
}

template <typename Op, typename X, typename Acc, int NRHS>
__global__ void __launch_bounds__(HMV_THREADS, 2) k_hmv_tasks(
    const Task* __restrict__ tasks, const int* __restrict__ leaf_nr, const Panel* __restrict__ panels,
    const FarBlk* __restrict__ far, const int* __restrict__ rank, const long long* __restrict__ fbase,
    const Op* __restrict__ near, const Op* __restrict__ U, const cplx<Acc>* __restrict__ t, int tstride,
    const X* __restrict__ x, long long N, cplx<Acc>* __restrict__ part, long long pstride) {
  extern __shared__ unsigned char smem_raw[];
  cplx<Acc>* red = reinterpret_cast<cplx<Acc>*>(smem_raw);
  hmv_task<Op, X, Acc, NRHS>(tasks[blockIdx.x], leaf_nr, panels, far, rank, fbase, near, U, t, tstride, x, N, part,
                             pstride, red);
}

// phase 3: y[rows of leaf] = sum over the leaf's tasks, in task order
template <typename Acc, typename Y, int NRHS>
__global__ void __launch_bounds__(256) k_hmv_reduce(const int* __restrict__ leaf_r0, const int* __restrict__ leaf_nr,
                                                    const int* __restrict__ task_ptr, const Task* __restrict__ tasks,
                                                    const cplx<Acc>* __restrict__ part, long long pstride,
                                                    long long N, Y* __restrict__ y) {
  const int leaf = blockIdx.x;
  const int rows = 3 * leaf_nr[leaf];
  const long long row0 = 3LL * leaf_r0[leaf];
  const int t0 = task_ptr[leaf], t1 = task_ptr[leaf + 1];
  for (int r = threadIdx.x; r < rows; r += blockDim.x) {
#pragma unroll
    for (int q = 0; q < NRHS; ++q) {
      cplx<double> s{0, 0};  // task partials added in FP64
      for (int k = t0; k < t1; ++k) {
        cplx<Acc> v = part[q * pstride + tasks[k].slot + r];
        s.re += v.re;
        s.im += v.im;
      }
      Y o;
      o.re = decltype(o.re)(s.re);
      o.im = decltype(o.im)(s.im);
      y[q * N + row0 + r] = o;
    }
  }
}

// ---------------------------------------------------------------------------
// The fused product: one launch, one CTA per work item (HItem), items in
// decreasing order of estimated cost (CTAs are dispatched in index order).
//   near item: dense near panels of one leaf row, as hmv_task, but each
//              thread owns a PAIR of rows and reads both entries of a column
//              with one 16-byte load (near panels: even ld, even offsets)
//   far item:  one admissible block b: t = V_b^T x with 16-byte loads that
//              stream the block's factor columns two at a time as one flat
//              range (t kept in shared memory), then U_b t over the block's
//              row cluster (row pairs, 16-byte loads where aligned)
// Items write their rows to their own slot of the partial buffer; the item
// that completes a leaf's last contribution (a per-leaf arrival counter)
// adds the leaf's contributions in a fixed order (FP64) and writes y.
// ---------------------------------------------------------------------------
constexpr int HF_THREADS = 384;
// loads in flight per thread: near panels (columns of two rows), U columns,
// and 16-byte V loads per lane; CTAs per SM of the GMRES product
#ifndef HF_NEAR_DEPTH
#define HF_NEAR_DEPTH 8
#endif
#ifndef HF_U_DEPTH
#define HF_U_DEPTH 8
#endif
#ifndef HF_V_DEPTH
#define HF_V_DEPTH 2
#endif
#ifndef HF_CTAS
#define HF_CTAS 3
#endif
constexpr int HF_WARPS = HF_THREADS / 32;

__device__ __forceinline__ void ld_pair(const c64* p, c64& a, c64& b) {
  const float4 v = __ldcs(reinterpret_cast<const float4*>(p));
  a = c64{v.x, v.y};
  b = c64{v.z, v.w};
}
__device__ __forceinline__ bool aligned16(const void* p) { return (reinterpret_cast<uintptr_t>(p) & 15) == 0; }

template <typename Acc> __device__ __forceinline__ cplx<Acc> czero() { return cplx<Acc>{Acc(0), Acc(0)}; }

// (V^T x) for the columns l0 (and l0 + 1 if len = 2 n) of one factor V, whose
// columns of n entries are contiguous: the pair is streamed as one flat range
// of len entries with 16-byte loads (complex64: two entries per load, one
// entry before the first 16-byte boundary and one after the last); per-lane
// partial sums a0 (column l0) and a1 (column l0 + 1)
template <typename Op, typename X, typename Acc, int NRHS>
__device__ __forceinline__ void hf_vtx_pair(const Op* __restrict__ base, int len, int n, const X* __restrict__ xs,
                                            long long N, cplx<Acc> (&a0)[NRHS], cplx<Acc> (&a1)[NRHS]) {
  const int lane = threadIdx.x & 31;
#pragma unroll
  for (int q = 0; q < NRHS; ++q) a0[q] = a1[q] = czero<Acc>();
  // entry f of the range: column l0 + (f >= n), row f - n (f >= n)
  auto add = [&](int f, const Op& v) {
    const bool c1 = f >= n;
    const int row = c1 ? f - n : f;
    const cplx<Acc> vv = up<Acc>(v);
#pragma unroll
    for (int q = 0; q < NRHS; ++q) {
      const cplx<Acc> xv = up<Acc>(xs[q * N + row]);
      if (c1) cmac(a1[q], vv, xv);
      else cmac(a0[q], vv, xv);
    }
  };
  if constexpr (sizeof(Op) == 8) {
    const int head = aligned16(base) ? 0 : 1;
    if (head && lane == 0) add(0, ld_stream(base));
    const int body = (len - head) >> 1;
    const Op* bp = base + head;
    int c = lane;
    for (; c + 32 * (HF_V_DEPTH - 1) < body; c += 32 * HF_V_DEPTH) {
      Op v[2 * HF_V_DEPTH];
#pragma unroll
      for (int u = 0; u < HF_V_DEPTH; ++u) ld_pair(bp + 2 * (c + 32 * u), v[2 * u], v[2 * u + 1]);
#pragma unroll
      for (int u = 0; u < HF_V_DEPTH; ++u) {
        add(head + 2 * (c + 32 * u), v[2 * u]);
        add(head + 2 * (c + 32 * u) + 1, v[2 * u + 1]);
      }
    }
    for (; c < body; c += 32) {
      Op v0, v1;
      ld_pair(bp + 2 * c, v0, v1);
      add(head + 2 * c, v0);
      add(head + 2 * c + 1, v1);
    }
    if (((len - head) & 1) && lane == 0) add(len - 1, ld_stream(base + len - 1));
  } else {
    int f = lane;
    for (; f + 96 < len; f += 128) {
      Op v[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) v[u] = ld_stream(base + f + 32 * u);
#pragma unroll
      for (int u = 0; u < 4; ++u) add(f + 32 * u, v[u]);
    }
    for (; f < len; f += 32) add(f, ld_stream(base + f));
  }
}

// The admissible blocks of one far item (all with the same row cluster),
// as read by hf_item_rows: factor offsets, column-cluster sizes and starts,
// and the prefix sums of their ranks (columns) and of their column pairs.
struct HfBlocks {
  long long u[HITEM_MAX_BLOCKS], v[HITEM_MAX_BLOCKS];
  int n[HITEM_MAX_BLOCKS], c0[HITEM_MAX_BLOCKS];
  int cpre[HITEM_MAX_BLOCKS + 1], ppre[HITEM_MAX_BLOCKS + 1];
  int nb;
};

// E consecutive rows of one column at p (E = 2 for complex64, 1 for complex128)
__device__ __forceinline__ void ld_rows(const c64* p, bool pair_ok, c64 (&v)[2]) {
  if (pair_ok && aligned16(p)) {
    ld_pair(p, v[0], v[1]);
  } else {
    v[0] = ld_stream(p);
    v[1] = pair_ok ? ld_stream(p + 1) : c64{0.f, 0.f};
  }
}
__device__ __forceinline__ void ld_rows(const c128* p, bool, c128 (&v)[1]) { v[0] = ld_stream(p); }

// Rows [0, m) of one item: kind 0 sums its near panels against x, kind 1
// sums the r columns of U (column stride m) against ts; each thread owns E
// consecutive rows and one of G column groups (the groups are added in
// shared memory). Writes rows [0, m) (and the pad row m for m odd) to the
// item's slot.
template <typename Op, typename X, typename Acc, int NRHS>
__device__ __forceinline__ void hf_item_rows(const HItem& it, int m, const Panel* __restrict__ panels,
                                             const Op* __restrict__ near, const Op* __restrict__ U,
                                             const HfBlocks& fb, int tsn, const X* __restrict__ x, long long N,
                                             const cplx<Acc>* ts, cplx<Acc>* __restrict__ part, long long pstride,
                                             cplx<Acc>* red) {
  constexpr int E = 16 / (int)sizeof(Op);
  const int RP = (m + E - 1) / E;
  for (int rbase = 0; rbase < RP; rbase += HF_THREADS) {
    const int rc = min(RP - rbase, HF_THREADS);
    const int G = max(1, HF_THREADS / rc);
    const int g = threadIdx.x / rc;
    const int rl = threadIdx.x % rc;
    const int row = (rl + rbase) * E;
    const bool active = g < G;
    cplx<Acc> acc[E][NRHS];
#pragma unroll
    for (int e = 0; e < E; ++e)
#pragma unroll
      for (int q = 0; q < NRHS; ++q) acc[e][q] = czero<Acc>();
    if (active) {
      if (it.kind == 0) {
        for (int p = it.p0; p < it.p1; ++p) {
          const Panel P = panels[p];
          const long long ld = P.ld;
          const Op* d = near + P.data + row;  // pairs of rows: even ld and offsets, pad row stored
          const X* xs = x + P.xoff;
          const int nc = P.ncols;
          int j = g;
          for (; j + (HF_NEAR_DEPTH - 1) * G < nc; j += HF_NEAR_DEPTH * G) {
            Op av[HF_NEAR_DEPTH][E];
#pragma unroll
            for (int u = 0; u < HF_NEAR_DEPTH; ++u) ld_rows(d + (long long)(j + u * G) * ld, true, av[u]);
            X xv[NRHS][HF_NEAR_DEPTH];
#pragma unroll
            for (int q = 0; q < NRHS; ++q)
#pragma unroll
              for (int u = 0; u < HF_NEAR_DEPTH; ++u) xv[q][u] = xs[q * N + j + u * G];
#pragma unroll
            for (int q = 0; q < NRHS; ++q)
#pragma unroll
              for (int u = 0; u < HF_NEAR_DEPTH; ++u)
#pragma unroll
                for (int e = 0; e < E; ++e) cmac(acc[e][q], up<Acc>(av[u][e]), up<Acc>(xv[q][u]));
          }
          for (; j < nc; j += G) {
            Op av[E];
            ld_rows(d + (long long)j * ld, true, av);
#pragma unroll
            for (int q = 0; q < NRHS; ++q) {
              const cplx<Acc> xq = up<Acc>(xs[q * N + j]);
#pragma unroll
              for (int e = 0; e < E; ++e) cmac(acc[e][q], up<Acc>(av[e]), xq);
            }
          }
        }
      } else {
        // the columns of all the item's factors U_b, c < C, in block order;
        // column c of block i (cpre[i] <= c < cpre[i + 1]) is its column c - cpre[i]
        const bool pair_ok = row + E - 1 < m;
        const int C = fb.cpre[fb.nb];
        int cur = 0;
        int c = g;
        for (; c + (HF_U_DEPTH - 1) * G < C; c += HF_U_DEPTH * G) {
          Op av[HF_U_DEPTH][E];
#pragma unroll
          for (int u = 0; u < HF_U_DEPTH; ++u) {
            const int cc = c + u * G;
            while (cc >= fb.cpre[cur + 1]) ++cur;
            ld_rows(U + fb.u[cur] + (long long)(cc - fb.cpre[cur]) * m + row, pair_ok, av[u]);
          }
#pragma unroll
          for (int q = 0; q < NRHS; ++q)
#pragma unroll
            for (int u = 0; u < HF_U_DEPTH; ++u) {
              const cplx<Acc> tq = ts[q * tsn + c + u * G];
#pragma unroll
              for (int e = 0; e < E; ++e) cmac(acc[e][q], up<Acc>(av[u][e]), tq);
            }
        }
        for (; c < C; c += G) {
          while (c >= fb.cpre[cur + 1]) ++cur;
          Op av[E];
          ld_rows(U + fb.u[cur] + (long long)(c - fb.cpre[cur]) * m + row, pair_ok, av);
#pragma unroll
          for (int q = 0; q < NRHS; ++q) {
            const cplx<Acc> tq = ts[q * tsn + c];
#pragma unroll
            for (int e = 0; e < E; ++e) cmac(acc[e][q], up<Acc>(av[e]), tq);
          }
        }
      }
    }
    if (G > 1) {
      if (active && g > 0) {
#pragma unroll
        for (int q = 0; q < NRHS; ++q)
#pragma unroll
          for (int e = 0; e < E; ++e) red[((q * G + g) * rc + rl) * E + e] = acc[e][q];
      }
      __syncthreads();
      if (active && g == 0) {
        for (int gg = 1; gg < G; ++gg)
#pragma unroll
          for (int q = 0; q < NRHS; ++q)
#pragma unroll
            for (int e = 0; e < E; ++e) {
              const cplx<Acc> o = red[((q * G + gg) * rc + rl) * E + e];
              acc[e][q].re += o.re;
              acc[e][q].im += o.im;
            }
      }
      __syncthreads();
    }
    if (active && g == 0) {
#pragma unroll
      for (int q = 0; q < NRHS; ++q)
#pragma unroll
        for (int e = 0; e < E; ++e)
          if (row + e <= m) part[q * pstride + it.slot + row + e] = acc[e][q];
    }
  }
}

template <typename Op, typename X, typename Y, typename Acc, int NRHS>
__global__ void __launch_bounds__(HF_THREADS, (NRHS == 1 && sizeof(Acc) == 4) ? HF_CTAS : 2) k_hmv_fused(
    const HItem* __restrict__ items, const int* __restrict__ far_list, const int* __restrict__ leaf_r0,
    const int* __restrict__ leaf_nr, const Panel* __restrict__ panels, const FarBlk* __restrict__ far,
    const int* __restrict__ rank, const long long* __restrict__ fbase, const Op* __restrict__ near,
    const Op* __restrict__ U, const Op* __restrict__ V, const X* __restrict__ x, long long N, int tsn,
    cplx<Acc>* __restrict__ part, long long pstride, const int* __restrict__ hc_ptr,
    const long long* __restrict__ hc_off, int* __restrict__ leaf_cnt, Y* __restrict__ y,
    const int* __restrict__ run) {
  if (run && !*run) return;  // every CTA of the launch reads the same flag
  extern __shared__ unsigned char smem_raw[];
  cplx<Acc>* ts = reinterpret_cast<cplx<Acc>*>(smem_raw);  // NRHS x tsn: the items' V^T x values
  cplx<Acc>* red = ts + NRHS * tsn;                        // NRHS x HF_THREADS x E
  __shared__ HfBlocks fb;
  __shared__ int last;
  const HItem it = items[blockIdx.x];
  if (it.kind == 0) {
    if (threadIdx.x == 0) fb.nb = 0;
    __syncthreads();
    hf_item_rows<Op, X, Acc, NRHS>(it, 3 * leaf_nr[it.l0], panels, near, U, fb, tsn, x, N, ts, part, pstride, red);
  } else {
    int nrows = 0;
    if (threadIdx.x == 0) {
      int c = 0, pp = 0, nb = 0;
      for (int i = it.p0; i < it.p1; ++i, ++nb) {
        const int b = far_list[i];
        const FarBlk Bk = far[b];
        const int r = min(rank[b], Bk.rmax);
        fb.u[nb] = fbase[2 * b];
        fb.v[nb] = fbase[2 * b + 1];
        fb.n[nb] = 3 * Bk.nc;
        fb.c0[nb] = Bk.c0;
        fb.cpre[nb] = c;
        fb.ppre[nb] = pp;
        c += r;
        pp += (r + 1) / 2;
      }
      fb.cpre[nb] = c;
      fb.ppre[nb] = pp;
      fb.nb = nb;
    }
    nrows = 3 * far[far_list[it.p0]].nr;
    __syncthreads();
    // t = V_b^T x of every block, column pairs over the warps
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    int cur = 0;
    for (int pp = warp; pp < fb.ppre[fb.nb]; pp += HF_WARPS) {
      while (pp >= fb.ppre[cur + 1]) ++cur;
      const int r = fb.cpre[cur + 1] - fb.cpre[cur];
      const int l0 = 2 * (pp - fb.ppre[cur]);
      const int n = fb.n[cur];
      cplx<Acc> a0[NRHS], a1[NRHS];
      hf_vtx_pair<Op, X, Acc, NRHS>(V + fb.v[cur] + (long long)l0 * n, min(2, r - l0) * n, n, x + 3LL * fb.c0[cur],
                                    N, a0, a1);
#pragma unroll
      for (int q = 0; q < NRHS; ++q) {
        const Acc r0 = wsum(a0[q].re), i0 = wsum(a0[q].im), r1 = wsum(a1[q].re), i1 = wsum(a1[q].im);
        if (lane == 0) {
          ts[q * tsn + fb.cpre[cur] + l0] = cplx<Acc>{r0, i0};
          if (l0 + 1 < r) ts[q * tsn + fb.cpre[cur] + l0 + 1] = cplx<Acc>{r1, i1};
        }
      }
    }
    __syncthreads();
    hf_item_rows<Op, X, Acc, NRHS>(it, nrows, panels, near, U, fb, tsn, x, N, ts, part, pstride, red);
  }
  __threadfence();  // this item's partials are visible before its arrivals are counted
  __syncthreads();
  for (int l = it.l0; l < it.l1; ++l) {
    const int c0 = hc_ptr[l], c1 = hc_ptr[l + 1];
    if (threadIdx.x == 0) last = atomicAdd(&leaf_cnt[l], 1) == c1 - c0 - 1;
    __syncthreads();
    if (last) {
      __threadfence();
      const int rows = 3 * leaf_nr[l];
      const long long row0 = 3LL * leaf_r0[l];
      for (int rr = threadIdx.x; rr < rows; rr += blockDim.x) {
#pragma unroll
        for (int q = 0; q < NRHS; ++q) {
          cplx<double> sum{0, 0};
          for (int k = c0; k < c1; ++k) {
            const cplx<Acc> v = ld_global_cg(part + q * pstride + hc_off[k] + rr);
            sum.re += v.re;
            sum.im += v.im;
          }
          Y o;
          o.re = decltype(o.re)(sum.re);
          o.im = decltype(o.im)(sum.im);
          y[q * N + row0 + rr] = o;
        }
      }
      if (threadIdx.x == 0) leaf_cnt[l] = 0;
    }
    __syncthreads();
  }
}

template <typename Op, typename X, typename Y, typename Acc, int NRHS>
static void hmv_impl(const bem_ctx* ctx, const Op* near, const Op* U, const Op* V, cplx<Acc>* t,
                     const X* x, Y* y, cudaStream_t st, const int* run) {
  (void)t;
  if (!ctx->nhitems) return;
  constexpr int E = 16 / (int)sizeof(Op);
  const int tsn = std::max(1, ctx->hitem_tcols);
  const size_t sm = (size_t)NRHS * (tsn + (size_t)HF_THREADS * E) * sizeof(cplx<Acc>);
  // the attribute is per function and device: set once per device, to the
  // largest size any mesh can ask for
  const size_t sm_max = (size_t)NRHS * (HITEM_MAX_TCOLS + (size_t)HF_THREADS * E) * sizeof(cplx<Acc>);
  if (sm_max > 48 * 1024) {
    static bool attr_set[64] = {};
    int dev = 0;
    cudaGetDevice(&dev);
    if (dev < 0 || dev >= 64 || !attr_set[dev]) {
      cudaFuncSetAttribute(k_hmv_fused<Op, X, Y, Acc, NRHS>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)sm_max);
      if (dev >= 0 && dev < 64) attr_set[dev] = true;
    }
  }
  cplx<Acc>* part = reinterpret_cast<cplx<Acc>*>(ctx->part.p);
  count_if(true);
  k_hmv_fused<Op, X, Y, Acc, NRHS><<<ctx->nhitems, HF_THREADS, sm, st>>>(
      ctx->hitems.p, ctx->hfar_list.p, ctx->leaf_r0.p, ctx->leaf_nr.p, ctx->panels.p, ctx->far_d.p, ctx->rank.p,
      ctx->fbase.p, near, U, V, x, ctx->N, tsn, part, ctx->hpart_rows, ctx->hc_ptr.p, ctx->hc_off.p,
      ctx->leaf_cnt.p, y, run);
}

template <typename Op, typename X, typename Y, typename Acc>
void launch_hmatvec(const bem_ctx* ctx, const Op* near, const Op* U, const Op* V, cplx<Acc>* t, const X* x,
                    Y* y, int nrhs, cudaStream_t st, const int* run) {
  switch (nrhs) {
    case 1: hmv_impl<Op, X, Y, Acc, 1>(ctx, near, U, V, t, x, y, st, run); break;
    case 2: hmv_impl<Op, X, Y, Acc, 2>(ctx, near, U, V, t, x, y, st, run); break;
    case 3: hmv_impl<Op, X, Y, Acc, 3>(ctx, near, U, V, t, x, y, st, run); break;
    default: hmv_impl<Op, X, Y, Acc, 4>(ctx, near, U, V, t, x, y, st, run); break;
  }
}

// Same product (c64 operator, FP32 accumulation, one right-hand side) with
// caller-provided scratch for the t = V^T x values and the per-task partial
// row sums (sizes t_entries and part_rows complex64).
void launch_hmatvec_scratch_c64(const bem_ctx* ctx, const c64* near, const c64* U, const c64* V, cplx<float>* t,
                                cplx<float>* part, const c64* x, c64* y, cudaStream_t st) {
  int nfar = (int)ctx->far_h.size();
  if (count_if(nfar))
    k_hmv_t<c64, c64, float, 1><<<nfar, 256, 0, st>>>(ctx->far_d.p, ctx->rank.p, ctx->fbase.p, V, x, ctx->N, t,
                                                      ctx->t_entries);
  size_t sm = (size_t)2 * HMV_THREADS * sizeof(cplx<float>);
  count_if(true);
  k_hmv_tasks<c64, c64, float, 1><<<ctx->ntasks, HMV_THREADS, sm, st>>>(
      ctx->tasks.p, ctx->leaf_nr.p, ctx->panels.p, ctx->far_d.p, ctx->rank.p, ctx->fbase.p, near, U, t,
      ctx->t_entries, x, ctx->N, part, ctx->part_rows);
  count_if(true);
  k_hmv_reduce<float, c64, 1><<<ctx->nleaves, 256, 0, st>>>(ctx->leaf_r0.p, ctx->leaf_nr.p, ctx->task_ptr.p,
                                                           ctx->tasks.p, part, ctx->part_rows, ctx->N, y);
}

template void launch_hmatvec<c64, c64, c64, float>(const bem_ctx*, const c64*, const c64*, const c64*,
                                                   cplx<float>*, const c64*, c64*, int, cudaStream_t, const int*);
template void launch_hmatvec<c64, c64, c128, float>(const bem_ctx*, const c64*, const c64*, const c64*,
                                                    cplx<float>*, const c64*, c128*, int, cudaStream_t,
                                                    const int*);
template void launch_hmatvec<c64, c128, c128, double>(const bem_ctx*, const c64*, const c64*, const c64*,
                                                      cplx<double>*, const c128*, c128*, int, cudaStream_t,
                                                      const int*);
template void launch_hmatvec<c128, c128, c128, double>(const bem_ctx*, const c128*, const c128*,
                                                       const c128*, cplx<double>*, const c128*, c128*, int,
                                                       cudaStream_t, const int*);

// ---------------------------------------------------------------------------
// block-Jacobi preconditioner
// ---------------------------------------------------------------------------
// run (optional): the launch does nothing unless *run is nonzero; joff
// (optional): v is read from v + (*joff) ldv (the device-driven solver's
// basis vector V_j).
template <typename Pm, typename V, typename Z>
__global__ void k_precond(const Pm* __restrict__ pinv, const V* __restrict__ v, Z* __restrict__ z, int ne,
                          const int* __restrict__ run, const int* __restrict__ joff, long long ldv) {
  if (run && !*run) return;
  if (joff) v += (long long)(*joff) * ldv;
  int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= ne) return;
  using Acc = typename Promote<decltype(Pm{}.re), decltype(V{}.re)>::type;
  cplx<Acc> ve[3];
  for (int a = 0; a < 3; ++a) ve[a] = up<Acc>(v[3LL * e + a]);
  for (int a = 0; a < 3; ++a) {
    cplx<Acc> s{0, 0};
    for (int b = 0; b < 3; ++b) cmac(s, up<Acc>(pinv[9LL * e + 3 * a + b]), ve[b]);
    Z o;
    o.re = decltype(o.re)(s.re);
    o.im = decltype(o.im)(s.im);
    z[3LL * e + a] = o;
  }
}
template <typename Pm, typename V, typename Z>
void launch_precond(const Pm* pinv, const V* v, Z* z, int ne, cudaStream_t st, const int* run, const int* joff,
                    long long ldv) {
  count_if(true);
  k_precond<Pm, V, Z><<<(ne + 127) / 128, 128, 0, st>>>(pinv, v, z, ne, run, joff, ldv);
}
template void launch_precond<c64, c64, c64>(const c64*, const c64*, c64*, int, cudaStream_t, const int*,
                                            const int*, long long);
template void launch_precond<c128, c128, c128>(const c128*, const c128*, c128*, int, cudaStream_t, const int*,
                                               const int*, long long);
template void launch_precond<c128, c128, c64>(const c128*, const c128*, c64*, int, cudaStream_t, const int*,
                                              const int*, long long);

// ---------------------------------------------------------------------------
// Arnoldi pieces (FP64 accumulation)
// ---------------------------------------------------------------------------
template <typename Vb, typename W>
__global__ void k_dots(const Vb* __restrict__ V, long long ldv, const W* __restrict__ w, long long n,
                       c128* __restrict__ part) {
  const int l = blockIdx.y;
  const Vb* v = V + l * ldv;
  double re = 0, im = 0;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    Vb a = v[i];
    W b = w[i];
    double ar = a.re, ai = a.im, br = b.re, bi = b.im;
    re = fma(ar, br, fma(ai, bi, re));   // conj(a) * b
    im = fma(ar, bi, fma(-ai, br, im));
  }
  re = wsum(re);
  im = wsum(im);
  __shared__ double s[2][32];
  int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  if (lane == 0) {
    s[0][wid] = re;
    s[1][wid] = im;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double tr = 0, ti = 0;
    for (int k = 0; k < (int)(blockDim.x >> 5); ++k) {
      tr += s[0][k];
      ti += s[1][k];
    }
    part[(long long)l * gridDim.x + blockIdx.x] = c128{tr, ti};
  }
}
template <typename Vb, typename W>
int launch_dots(const Vb* V, long long ldv, int nvec, const W* w, long long n, c128* part, cudaStream_t st) {
  // enough blocks in total (nblk x nvec) to cover the GPU, two elements per thread
  int nblk = (int)std::min<long long>(std::max<long long>(1, (n + 511) / 512), 64);
  dim3 grid(nblk, nvec);
  count_if(true);
  k_dots<Vb, W><<<grid, 256, 0, st>>>(V, ldv, w, n, part);
  return nblk;
}
template int launch_dots<c64, c64>(const c64*, long long, int, const c64*, long long, c128*, cudaStream_t);
template int launch_dots<c128, c128>(const c128*, long long, int, const c128*, long long, c128*, cudaStream_t);

__global__ void k_dots_final(const c128* __restrict__ part, int nblk, c128* __restrict__ out) {
  int l = blockIdx.x;
  double re = 0, im = 0;
  for (int k = threadIdx.x; k < nblk; k += 32) {
    re += part[(long long)l * nblk + k].re;
    im += part[(long long)l * nblk + k].im;
  }
  re = wsum(re);
  im = wsum(im);
  if (threadIdx.x == 0) out[l] = c128{re, im};
}
void launch_dots_final(const c128* part, int nblk, int nvec, c128* out, cudaStream_t st) {
  count_if(true);
  k_dots_final<<<nvec, 32, 0, st>>>(part, nblk, out);
}



// ---------------------------------------------------------------------------
// One Arnoldi orthogonalisation step in one cooperative launch: classical
// Gram-Schmidt twice against V_0..V_j, the norm, and V_{j+1} = w / ||w||.
// Block b owns a slice of the rows; partial sums per block go to part and are
// added in block order by every block after a grid barrier (the same result
// in every block and on every run).
// Arithmetic: with a complex64 basis, the products and each lane's short run
// of sums (the slice / 32 elements it owns) are FP32, everything above that
// FP64; with a complex128 basis, FP64 throughout. (FP64 throughput is a small
// fraction of FP32 here; FP32 products of FP32 data keep the error at the
// basis's own rounding level.)
//   hcol: [h1 (m+1) | h2 (m+1) | ||w||^2], written by block 0
// ---------------------------------------------------------------------------
template <typename Vb>
__device__ __forceinline__ void orth_partials(const Vb* __restrict__ V, long long ldv, int nvec,
                                              const Vb* __restrict__ w, long long i0, long long i1,
                                              c128* __restrict__ part) {
  using T = decltype(Vb{}.re);
  // warp k handles vectors l = k, k + nwarps, ...; lanes stride over the slice
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
  for (int l = wid; l < nvec; l += nw) {
    const Vb* v = V + l * ldv;
    T re = 0, im = 0;
    for (long long i = i0 + lane; i < i1; i += 32) {
      const Vb a = v[i], b = w[i];
      re = fma(a.re, b.re, fma(a.im, b.im, re));  // conj(a) * b
      im = fma(a.re, b.im, fma(-a.im, b.re, im));
    }
    double dre = wsum((double)re), dim = wsum((double)im);
    if (lane == 0) part[(long long)l * gridDim.x + blockIdx.x] = c128{dre, dim};
  }
}
// part[slot * nblk + block] = ||w||^2 over the slice (warp 0)
template <typename Vb>
__device__ __forceinline__ void orth_partials_self(const Vb* __restrict__ w, int slot, long long i0, long long i1,
                                                   c128* __restrict__ part) {
  using T = decltype(Vb{}.re);
  if ((threadIdx.x >> 5) != 0) return;
  const int lane = threadIdx.x & 31;
  T s = 0;
  for (long long i = i0 + lane; i < i1; i += 32) {
    const Vb a = w[i];
    s = fma(a.re, a.re, fma(a.im, a.im, s));
  }
  const double d = wsum((double)s);
  if (lane == 0) part[(long long)slot * gridDim.x + blockIdx.x] = c128{d, 0.0};
}
// out[l] = sum_b part[l * nblk + b] for l < nvec, in block order (into shared memory)
__device__ __forceinline__ void orth_sums(const c128* __restrict__ part, int nvec, c128* out) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
  const int nb = gridDim.x;
  for (int l = wid; l < nvec; l += nw) {
    double re = 0, im = 0;
    for (int b = lane; b < nb; b += 32) {
      re += part[(long long)l * nb + b].re;
      im += part[(long long)l * nb + b].im;
    }
    re = wsum(re);
    im = wsum(im);
    if (lane == 0) out[l] = c128{re, im};
  }
}
// w -= sum_l V_l h_l over the slice (h in the basis's precision: hT)
template <typename Vb>
__device__ __forceinline__ void orth_update(const Vb* __restrict__ V, long long ldv, int nvec,
                                            const cplx<decltype(Vb{}.re)>* h, Vb* __restrict__ w, long long i0,
                                            long long i1) {
  using T = decltype(Vb{}.re);
  for (long long i = i0 + threadIdx.x; i < i1; i += blockDim.x) {
    T re = 0, im = 0;
    for (int l = 0; l < nvec; ++l) {
      const Vb a = V[l * ldv + i];
      const cplx<T> c = h[l];
      re = fma(a.re, c.re, fma(-a.im, c.im, re));
      im = fma(a.re, c.im, fma(a.im, c.re, im));
    }
    Vb o = w[i];
    o.re = o.re - re;
    o.im = o.im - im;
    w[i] = o;
  }
}

constexpr int ORTH_THREADS = 256;
constexpr int ORTH_MAXVEC = 513;  // shared-memory coefficient slots (restart + 1 <= 512)

// The host copy of the solver state (the fields the host reads).
__device__ __forceinline__ void gm_publish(const GmCtl* c, GmCtl* mirror) {
  volatile GmCtl* h = mirror;
  h->active = c->active;
  h->j = c->j;
  h->update = c->update;
  h->live = c->live;
  h->its = c->its;
  h->cycles = c->cycles;
  h->converged = c->converged;
  h->bnorm = c->bnorm;
  h->rel = c->rel;
  h->guess_rel = c->guess_rel;
  h->target = c->target;
}

// Step j of the cycle on the host's behalf (one thread): column j of the
// Hessenberg matrix (the two projections summed, ||w|| below them), the
// rotations of the earlier steps applied to it, the rotation that zeroes its
// subdiagonal, and the residual estimate |g_{j+1}|. The cycle ends when that
// estimate meets the inner target, on breakdown (||w|| = 0), after m steps or
// at the step limit.
__device__ void gm_givens(const GmDev& d, int j, const c128* __restrict__ hcol, double nrm2) {
  GmCtl* c = d.ctl;
  const int m = d.m;
  c128* Rj = d.R + (long long)j * (m + 1);
  for (int i = 0; i <= j; ++i) Rj[i] = c128{hcol[i].re + hcol[m + 1 + i].re, hcol[i].im + hcol[m + 1 + i].im};
  const double hn = sqrt(fmax(0.0, nrm2));
  c128 b = Rj[0];
  for (int i = 0; i < j; ++i) {
    // G_i = [[conj c, conj s], [-s, c]] on rows i, i + 1
    const c128 a = b, nx = Rj[i + 1], ci = d.cs[i], si = d.sn[i];
    Rj[i] = c128{ci.re * a.re + ci.im * a.im + si.re * nx.re + si.im * nx.im,
                 ci.re * a.im - ci.im * a.re + si.re * nx.im - si.im * nx.re};
    b = c128{-(si.re * a.re - si.im * a.im) + (ci.re * nx.re - ci.im * nx.im),
             -(si.re * a.im + si.im * a.re) + (ci.re * nx.im + ci.im * nx.re)};
  }
  const double den = sqrt(b.re * b.re + b.im * b.im + hn * hn);
  const c128 cj = den > 0 ? c128{b.re / den, b.im / den} : c128{1.0, 0.0};
  const c128 sj = den > 0 ? c128{hn / den, 0.0} : c128{0.0, 0.0};
  d.cs[j] = cj;
  d.sn[j] = sj;
  Rj[j] = c128{den, 0.0};
  const c128 gj = d.g[j];
  d.g[j + 1] = c128{-(sj.re * gj.re - sj.im * gj.im), -(sj.re * gj.im + sj.im * gj.re)};
  d.g[j] = c128{cj.re * gj.re + cj.im * gj.im, cj.re * gj.im - cj.im * gj.re};
  const int its = c->its + 1, jn = j + 1;
  const double gcur = sqrt(d.g[jn].re * d.g[jn].re + d.g[jn].im * d.g[jn].im);
  c->its = its;
  c->j = jn;
  if (gcur <= c->target || its >= d.max_iters || hn == 0.0 || jn == m) {
    c->active = 0;
    c->update = 1;
    const int cy = c->cycles - 1;
    if (cy >= 0 && cy < GM_MAX_CYCLES) {
      c->jdone[cy] = jn;
      reinterpret_cast<volatile int*>(d.mirror->jdone)[cy] = jn;
    }
  }
  gm_publish(c, d.mirror);
}

// With gm.ctl set (the device-driven solver) the step index j and the column
// slot come from the solver state, the launch does nothing outside a cycle,
// and block 0 takes the step's Givens rotation after the last grid barrier
// (every block has read the state before the first one).
template <typename Vb>
__global__ void __launch_bounds__(ORTH_THREADS) k_arnoldi_orth(Vb* __restrict__ V, long long ldv, int j,
                                                               Vb* __restrict__ w, long long n,
                                                               c128* __restrict__ part, c128* __restrict__ hcol,
                                                               int m, GmDev gm) {
  using T = decltype(Vb{}.re);
  if (gm.ctl) {
    if (!gm.ctl->active) return;  // the same in every block: no grid barrier is reached
    j = gm.ctl->j;
    hcol = gm.hcol + (long long)j * gm.slot_len;
  }
  cg::grid_group grid = cg::this_grid();
  __shared__ c128 h[ORTH_MAXVEC];
  __shared__ cplx<T> hT[ORTH_MAXVEC];
  const int nvec = j + 1;
  const long long per = (n + gridDim.x - 1) / gridDim.x;
  const long long i0 = min(n, (long long)blockIdx.x * per), i1 = min(n, i0 + per);
  c128* p1 = part;
  c128* p2 = part + (long long)nvec * gridDim.x;
  c128* p3 = p2 + (long long)(nvec + 1) * gridDim.x;
  orth_partials<Vb>(V, ldv, nvec, w, i0, i1, p1);
  grid.sync();
  orth_sums(p1, nvec, h);
  __syncthreads();
  for (int l = threadIdx.x; l < nvec; l += blockDim.x) {
    hT[l] = mk<T>(T(h[l].re), T(h[l].im));
    if (blockIdx.x == 0) hcol[l] = h[l];
  }
  __syncthreads();
  orth_update<Vb>(V, ldv, nvec, hT, w, i0, i1);
  __syncthreads();  // this block's slice of w is complete before its second pass reads it
  // second projection's partials and ||w1||^2 of the slice (slot nvec of p2)
  orth_partials<Vb>(V, ldv, nvec, w, i0, i1, p2);
  orth_partials_self<Vb>(w, nvec, i0, i1, p2);
  grid.sync();
  orth_sums(p2, nvec + 1, h);
  __syncthreads();
  const double n1 = h[nvec].re;
  double h2sq = 0;
  for (int l = 0; l < nvec; ++l) h2sq += h[l].re * h[l].re + h[l].im * h[l].im;  // same order in every block
  for (int l = threadIdx.x; l < nvec; l += blockDim.x) {
    hT[l] = mk<T>(T(h[l].re), T(h[l].im));
    if (blockIdx.x == 0) hcol[m + 1 + l] = h[l];
  }
  __syncthreads();
  orth_update<Vb>(V, ldv, nvec, hT, w, i0, i1);
  __syncthreads();
  // ||w2||^2 = ||w1||^2 - ||h2||^2 (w1 = w2 + V h2 with w2 orthogonal to V);
  // where that cancels (w nearly in the span of V) the norm is summed anew,
  // a decision every block takes alike from the same sums
  double nrm2 = n1 - h2sq;
  if (!(nrm2 > 1e-2 * n1)) {
    orth_partials<Vb>(w, 0, 1, w, i0, i1, p3);  // ||w||^2 of the slice
    grid.sync();
    orth_sums(p3, 1, h);
    __syncthreads();
    nrm2 = h[0].re;
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) hcol[2 * (m + 1)] = c128{nrm2, 0.0};
  const T sc = T(nrm2 > 0 ? 1.0 / sqrt(nrm2) : 0.0);
  Vb* vn = V + (long long)(j + 1) * ldv;
  for (long long i = i0 + threadIdx.x; i < i1; i += blockDim.x) {
    const Vb a = w[i];
    Vb o;
    o.re = a.re * sc;
    o.im = a.im * sc;
    vn[i] = o;
  }
  if (gm.ctl && blockIdx.x == 0) {
    __syncthreads();  // block 0's column writes are visible to its thread 0
    if (threadIdx.x == 0) gm_givens(gm, j, hcol, nrm2);
  }
}

template <typename Vb>
int orth_grid(long long n) {
  // resident blocks (per process and instantiation; one device), computed
  // once under the thread-safe initialisation of a local static
  static const int c = [] {
    int dev = 0, sms = 0, per = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_arnoldi_orth<Vb>, ORTH_THREADS, 0);
    return std::max(1, sms * std::max(1, per));
  }();
  // about 256 rows per block, at most one wave of resident blocks
  return (int)std::max<long long>(1, std::min<long long>(c, (n + 255) / 256));
}

template <typename Vb>
cudaError_t launch_arnoldi_orth(Vb* V, long long ldv, int j, Vb* w, long long n, c128* part, c128* hcol, int m,
                                cudaStream_t st, const GmDev* gm) {
  if (j + 1 > ORTH_MAXVEC || m + 1 > ORTH_MAXVEC) return cudaErrorInvalidValue;
  const int nb = orth_grid<Vb>(n);
  GmDev g{};
  if (gm) g = *gm;
  void* args[] = {&V, &ldv, &j, &w, &n, &part, &hcol, &m, &g};
  count_if(true);
  return cudaLaunchCooperativeKernel((const void*)k_arnoldi_orth<Vb>, dim3(nb), dim3(ORTH_THREADS), args, 0, st);
}
template cudaError_t launch_arnoldi_orth<c64>(c64*, long long, int, c64*, long long, c128*, c128*, int,
                                              cudaStream_t, const GmDev*);
template cudaError_t launch_arnoldi_orth<c128>(c128*, long long, int, c128*, long long, c128*, c128*, int,
                                               cudaStream_t, const GmDev*);

// ---------------------------------------------------------------------------
// The rest of the device-driven GMRES control
// ---------------------------------------------------------------------------
// Start of a solve: ||b|| from its squared norm (bb, device), counters reset.
__global__ void k_gm_init(GmDev d, const c128* __restrict__ bb) {
  GmCtl* c = d.ctl;
  c->active = 0;
  c->j = 0;
  c->update = 0;
  c->live = 1;
  c->its = 0;
  c->cycles = 0;
  c->converged = 0;
  c->arrive = 0;
  c->bnorm = sqrt(fmax(0.0, bb->re));
  c->rel = 1.0;
  c->guess_rel = 1.0;
  c->target = 0.0;
  gm_publish(c, d.mirror);
}
void launch_gm_init(const GmDev& d, const c128* bb, cudaStream_t st) {
  count_if(true);
  k_gm_init<<<1, 1, 0, st>>>(d, bb);
}

// The true-residual test after r = b - A x (rr = ||r||^2 on the device):
// the solve ends if ||r|| <= tol ||b|| (or r = 0) or the step limit is
// reached; otherwise a cycle starts from V_0 = r / ||r|| with g = (||r||, 0,
// ...) and the inner target max(0.9 tol ||b||, floor ||r||). A zero
// right-hand side gives x = 0. The blocks read the state first; the last
// block to arrive writes it, so that no block sees a half-updated state.
template <typename Vb>
__global__ void k_gm_begin(GmDev d, const c128* __restrict__ rr, const c128* __restrict__ r, Vb* __restrict__ V0,
                           c128* __restrict__ x, long long n) {
  GmCtl* c = d.ctl;
  const int live = c->live, its = c->its, cycles = c->cycles;
  const double bnorm = c->bnorm;
  const double rnorm = sqrt(fmax(0.0, rr->re));
  const double rel = bnorm > 0 ? rnorm / bnorm : 0.0;
  const bool conv = rel <= d.tol || rnorm == 0.0;
  const bool start = live && !conv && its < d.max_iters;
  const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (i < n) {
    if (live && bnorm == 0.0) x[i] = c128{0.0, 0.0};
    if (start) {
      const double sc = 1.0 / rnorm;
      Vb o;
      o.re = decltype(o.re)(r[i].re * sc);
      o.im = decltype(o.im)(r[i].im * sc);
      V0[i] = o;
    }
  }
  __shared__ int last;
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    last = atomicAdd(&c->arrive, 1) == (int)gridDim.x - 1;
  }
  __syncthreads();
  if (!last || threadIdx.x != 0) return;
  __threadfence();
  c->arrive = 0;
  if (!live) return;
  c->update = 0;
  c->rel = rel;
  if (cycles == 0) c->guess_rel = rel;
  if (!start) {
    c->live = 0;
    c->active = 0;
    c->converged = conv ? 1 : 0;
  } else {
    c->active = 1;
    c->j = 0;
    c->cycles = cycles + 1;
    d.g[0] = c128{rnorm, 0.0};
    c->target = fmax(0.9 * d.tol * bnorm, d.floor * rnorm);
  }
  gm_publish(c, d.mirror);
}
template <typename Vb>
void launch_gm_begin(const GmDev& d, const c128* rr, const c128* r, Vb* V0, c128* x, long long n, cudaStream_t st) {
  count_if(true);
  k_gm_begin<Vb><<<(unsigned)((n + 255) / 256), 256, 0, st>>>(d, rr, r, V0, x, n);
}
template void launch_gm_begin<c64>(const GmDev&, const c128*, const c128*, c64*, c128*, long long, cudaStream_t);
template void launch_gm_begin<c128>(const GmDev&, const c128*, const c128*, c128*, c128*, long long,
                                    cudaStream_t);

// The update that closes a cycle (only when one has ended): y = R^{-1} g
// over the cycle's steps (back substitution by one warp, in every block),
// then out = V y.
template <typename Vb>
__global__ void k_gm_combine(const Vb* __restrict__ V, long long ldv, GmDev d, c128* __restrict__ out,
                             long long n) {
  if (!d.ctl->update) return;
  const int jd = d.ctl->j, m = d.m;
  __shared__ c128 y[ORTH_MAXVEC];
  if (threadIdx.x < 32) {
    const int lane = threadIdx.x;
    for (int i = jd - 1; i >= 0; --i) {
      double sre = 0, sim = 0;
      for (int k = i + 1 + lane; k < jd; k += 32) {
        const c128 a = d.R[(long long)k * (m + 1) + i], b = y[k];
        sre = fma(a.re, b.re, fma(-a.im, b.im, sre));
        sim = fma(a.re, b.im, fma(a.im, b.re, sim));
      }
      sre = wsum(sre);
      sim = wsum(sim);
      if (lane == 0) {
        const c128 gi = d.g[i], a = d.R[(long long)i * (m + 1) + i];
        const double tr = gi.re - sre, ti = gi.im - sim, den = a.re * a.re + a.im * a.im;
        y[i] = den > 0 ? c128{(tr * a.re + ti * a.im) / den, (ti * a.re - tr * a.im) / den} : c128{0.0, 0.0};
      }
      __syncwarp();
    }
  }
  __syncthreads();
  const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (i >= n) return;
  double re = 0, im = 0;
  for (int l = 0; l < jd; ++l) {
    const Vb a = V[l * ldv + i];
    const c128 c = y[l];
    re = fma((double)a.re, c.re, fma(-(double)a.im, c.im, re));
    im = fma((double)a.re, c.im, fma((double)a.im, c.re, im));
  }
  out[i] = c128{re, im};
}
template <typename Vb>
void launch_gm_combine(const Vb* V, long long ldv, const GmDev& d, c128* out, long long n, cudaStream_t st) {
  count_if(true);
  k_gm_combine<Vb><<<(unsigned)((n + 255) / 256), 256, 0, st>>>(V, ldv, d, out, n);
}
template void launch_gm_combine<c64>(const c64*, long long, const GmDev&, c128*, long long, cudaStream_t);
template void launch_gm_combine<c128>(const c128*, long long, const GmDev&, c128*, long long, cudaStream_t);
int arnoldi_orth_max_blocks() { return std::max(orth_grid<c64>(1LL << 40), orth_grid<c128>(1LL << 40)); }

// ---------------------------------------------------------------------------
// Solution extrapolation (Sec. 4.2) after the products Y = A X, in one
// cooperative launch: CGS2 QR of Y (FP64; a column whose norm after
// orthogonalisation is <= 1e-12 of the first one's is dropped), s = R^{-1} Q^H b,
// a0 = X s. Every block holds the same R, Q^H b and s (sums in block order).
// res[0] = ||b - A a0|| / ||b|| over the columns before the extra one,
// res[1] = over every column (from ||b||^2 - sum |q_i^H b|^2), by block 0.
// ---------------------------------------------------------------------------
struct SemCols {
  const c128* x[SEM_MAXC];
};

__global__ void __launch_bounds__(ORTH_THREADS) k_sem_fit(SemCols X, int C, int K, const c128* __restrict__ Y,
                                                          const c128* __restrict__ b, c128* __restrict__ Q,
                                                          c128* __restrict__ part, c128* __restrict__ a0,
                                                          double* __restrict__ res, long long n) {
  cg::grid_group grid = cg::this_grid();
  __shared__ c128 R[SEM_MAXC][SEM_MAXC];
  __shared__ c128 h[SEM_MAXC + 1], hsum[SEM_MAXC], sv[SEM_MAXC];
  __shared__ int keep[SEM_MAXC];
  __shared__ int kept;
  __shared__ double r00;
  const long long per = (n + gridDim.x - 1) / gridDim.x;
  const long long i0 = min(n, (long long)blockIdx.x * per), i1 = min(n, i0 + per);
  // three partial-sum buffers used in rotation (a buffer is rewritten only
  // after every block has passed the grid barrier that follows its sums)
  c128* pb[3] = {part, part + (long long)(SEM_MAXC + 1) * gridDim.x, part + 2LL * (SEM_MAXC + 1) * gridDim.x};
  int rot = 0;
  if (threadIdx.x == 0) {
    kept = 0;
    r00 = 0;
  }
  __syncthreads();
  for (int c = 0; c < C; ++c) {
    const int kk = kept;
    c128* qc = Q + (long long)kk * n;
    for (long long i = i0 + threadIdx.x; i < i1; i += blockDim.x) qc[i] = Y[(long long)c * n + i];
    if (threadIdx.x < SEM_MAXC) hsum[threadIdx.x] = c128{0, 0};
    __syncthreads();
    for (int pass = 0; pass < 2 && kk > 0; ++pass) {
      c128* p = pb[rot];
      rot = (rot + 1) % 3;
      orth_partials<c128>(Q, n, kk, qc, i0, i1, p);
      grid.sync();
      orth_sums(p, kk, h);
      __syncthreads();
      if (threadIdx.x < kk) {
        hsum[threadIdx.x].re += h[threadIdx.x].re;
        hsum[threadIdx.x].im += h[threadIdx.x].im;
      }
      orth_update<c128>(Q, n, kk, h, qc, i0, i1);
      __syncthreads();
    }
    c128* p = pb[rot];
    rot = (rot + 1) % 3;
    orth_partials<c128>(qc, 0, 1, qc, i0, i1, p);
    grid.sync();
    orth_sums(p, 1, h);
    __syncthreads();
    const double nrm = sqrt(fmax(0.0, h[0].re));
    const double ref = kk == 0 ? nrm : r00;
    if (nrm > 1e-12 * ref && nrm != 0.0) {  // uniform: every block has the same sums
      const double sc = 1.0 / nrm;
      for (long long i = i0 + threadIdx.x; i < i1; i += blockDim.x) qc[i] = c128{qc[i].re * sc, qc[i].im * sc};
      if (threadIdx.x == 0) {
        for (int l = 0; l < kk; ++l) R[l][kk] = hsum[l];
        R[kk][kk] = c128{nrm, 0.0};
        keep[kk] = c;
        if (kk == 0) r00 = nrm;
        kept = kk + 1;
      }
    }
    __syncthreads();
  }
  const int kk = kept;
  if (kk == 0) {
    for (long long i = i0 + threadIdx.x; i < i1; i += blockDim.x) a0[i] = c128{0, 0};
    if (blockIdx.x == 0 && threadIdx.x == 0) res[0] = res[1] = 1.0;
    return;
  }
  // Q^H b (vectors 0..kk-1) and ||b||^2 (slot kk) in one pass
  c128* p = pb[rot];
  orth_partials<c128>(Q, n, kk, b, i0, i1, p);
  orth_partials<c128>(b, 0, 1, b, i0, i1, p + (long long)kk * gridDim.x);
  grid.sync();
  orth_sums(p, kk + 1, h);
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int i = kk - 1; i >= 0; --i) {
      c128 v = h[i];
      for (int j2 = i + 1; j2 < kk; ++j2) {
        const c128 rr = R[i][j2], sj = sv[j2];
        v.re -= rr.re * sj.re - rr.im * sj.im;
        v.im -= rr.re * sj.im + rr.im * sj.re;
      }
      const c128 d = R[i][i];  // real, positive
      sv[i] = c128{v.re / d.re, v.im / d.re};
    }
    if (blockIdx.x == 0) {
      const double bb = h[kk].re;
      double rem_x = bb, rem_all = bb;
      for (int i = 0; i < kk; ++i) {
        const double q2 = h[i].re * h[i].re + h[i].im * h[i].im;
        rem_all -= q2;
        if (keep[i] < K) rem_x -= q2;
      }
      res[0] = bb > 0 ? sqrt(fmax(0.0, rem_x) / bb) : 1.0;
      res[1] = bb > 0 ? sqrt(fmax(0.0, rem_all) / bb) : 1.0;
    }
  }
  __syncthreads();
  for (long long i = i0 + threadIdx.x; i < i1; i += blockDim.x) {
    double re = 0, im = 0;
    for (int l = 0; l < kk; ++l) {
      const c128 xv = X.x[keep[l]][i], s2 = sv[l];
      re += xv.re * s2.re - xv.im * s2.im;
      im += xv.re * s2.im + xv.im * s2.re;
    }
    a0[i] = c128{re, im};
  }
}

cudaError_t launch_sem_fit(const c128* const* X, int C, int K, const c128* Y, const c128* b, c128* Q, c128* part,
                           c128* a0, double* res, long long n, cudaStream_t st) {
  if (C < 1 || C > SEM_MAXC) return cudaErrorInvalidValue;
  SemCols cols{};
  for (int c = 0; c < C; ++c) cols.x[c] = X[c];
  // resident blocks of this kernel (its shared memory differs from the
  // Arnoldi kernel's), about 256 rows per block, at most one wave
  static const int resident = [] {
    int dev = 0, sms = 0, per = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_sem_fit, ORTH_THREADS, 0);
    return std::max(1, sms * std::max(1, per));
  }();
  const int nb = (int)std::max<long long>(1, std::min<long long>(resident, (n + 255) / 256));
  void* args[] = {&cols, &C, &K, &Y, &b, &Q, &part, &a0, &res, &n};
  count_if(true);
  return cudaLaunchCooperativeKernel((const void*)k_sem_fit, dim3(nb), dim3(ORTH_THREADS), args, 0, st);
}

__global__ void k_residual(const c128* __restrict__ b, const c128* __restrict__ y, c128* __restrict__ r, long long n) {
  long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (i >= n) return;
  r[i] = c128{b[i].re - y[i].re, b[i].im - y[i].im};
}
void launch_residual(const c128* b, const c128* y, c128* r, long long n, cudaStream_t st) {
  count_if(true);
  k_residual<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(b, y, r, n);
}


__global__ void k_axpy(c128 a, const c128* __restrict__ x, c128* __restrict__ y, long long n,
                       const int* __restrict__ run) {
  if (run && !*run) return;
  long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (i >= n) return;
  c128 v = x[i];
  y[i] = c128{y[i].re + a.re * v.re - a.im * v.im, y[i].im + a.re * v.im + a.im * v.re};
}
void launch_axpy(c128 a, const c128* x, c128* y, long long n, cudaStream_t st, const int* run) {
  count_if(true);
  k_axpy<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(a, x, y, n, run);
}

template <typename O>
__global__ void k_copy_cast(const c128* __restrict__ x, O* __restrict__ y, long long n, double s) {
  long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (i >= n) return;
  O o;
  o.re = decltype(o.re)(x[i].re * s);
  o.im = decltype(o.im)(x[i].im * s);
  y[i] = o;
}
void launch_copy_cast(const c128* x, c64* y, long long n, double scale, cudaStream_t st) {
  count_if(true);
  k_copy_cast<c64><<<(unsigned)((n + 255) / 256), 256, 0, st>>>(x, y, n, scale);
}
void launch_copy_cast(const c128* x, c128* y, long long n, double scale, cudaStream_t st) {
  count_if(true);
  k_copy_cast<c128><<<(unsigned)((n + 255) / 256), 256, 0, st>>>(x, y, n, scale);
}

// ---------------------------------------------------------------------------
// modified Fourier transforms (FP64)
// ---------------------------------------------------------------------------
__global__ void k_load_dft(const double* __restrict__ P, int N, double T, double eta, c128* __restrict__ out) {
  int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k > N / 2) return;
  double dt = T / N;
  double re = 0, im = 0;
  for (int n = 0; n < N; ++n) {
    long long m = ((long long)n * k) % N;
    double sn, cs;
    sincospi(2.0 * (double)m / N, &sn, &cs);
    double a = exp(-eta * n * dt) * P[n];
    re += a * cs;
    im -= a * sn;
  }
  out[k] = c128{re / N, im / N};
}
void launch_load_dft(const double* P, int n_omega, double T, double eta, c128* out, cudaStream_t st) {
  int nf = n_omega / 2 + 1;
  count_if(true);
  k_load_dft<<<(nf + 127) / 128, 128, 0, st>>>(P, n_omega, T, eta, out);
}

// R(n dt) = e^{eta n dt} [W_0 Re R_0 + 2 Re sum_{k=1}^{N/2-1} W_k R_k e^{2 pi i n k/N}
//                         + W_{N/2} Re(R_{N/2}) (-1)^n]
__global__ void k_idft(const c128* __restrict__ spec, long long ldspec, const long long* __restrict__ idx,
                       long long ndof, int N, double T, double eta, int window, double* __restrict__ out) {
  extern __shared__ double tab[];  // cos, sin of 2 pi m / N, m < N
  for (int m = threadIdx.x + threadIdx.y * blockDim.x; m < N; m += blockDim.x * blockDim.y) {
    double sn, cs;
    sincospi(2.0 * (double)m / N, &sn, &cs);
    tab[2 * m] = cs;
    tab[2 * m + 1] = sn;
  }
  __syncthreads();
  long long d = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (d >= ndof) return;
  long long col = idx ? idx[d] : d;
  const double dt = T / N;
  auto W = [&](int k) -> double {
    if (window == BEM_WIN_HANNING) return 0.5 * (1.0 + tab[2 * k]);
    if (window == BEM_WIN_BLACKMAN) return 0.42 + 0.5 * tab[2 * k] + 0.08 * tab[2 * ((2 * k) % N)];
    return 1.0;
  };
  for (int n = blockIdx.y * blockDim.y + threadIdx.y; n < N; n += gridDim.y * blockDim.y) {
    double acc = W(0) * spec[col].re;
    double sgn = (n & 1) ? -1.0 : 1.0;
    acc += W(N / 2) * spec[(long long)(N / 2) * ldspec + col].re * sgn;
    double s2 = 0;
    int m = 0;
    for (int k = 1; k < N / 2; ++k) {
      m += n;
      if (m >= N) m -= N;
      c128 v = spec[(long long)k * ldspec + col];
      s2 += W(k) * (v.re * tab[2 * m] - v.im * tab[2 * m + 1]);
    }
    acc += 2.0 * s2;
    out[(long long)n * ndof + d] = exp(eta * n * dt) * acc;
  }
}
void launch_idft(const c128* spec, long long ldspec, const long long* idx, long long ndof, int n_omega, double T,
                 double eta, int window, double* out, cudaStream_t st) {
  dim3 block(32, 8);
  dim3 grid((unsigned)((ndof + 31) / 32), (unsigned)std::min(64, (n_omega + 7) / 8));
  size_t sm = 2 * sizeof(double) * n_omega;
  if (sm > 48 * 1024) cudaFuncSetAttribute(k_idft, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
  count_if(true);
  k_idft<<<grid, block, sm, st>>>(spec, ldspec, idx, ndof, n_omega, T, eta, window, out);
}

}  // namespace bem
