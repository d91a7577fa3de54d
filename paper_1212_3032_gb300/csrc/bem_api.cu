// C-ABI entry points and host orchestration of the frequency sweep.
//
// bem_solve_sweep follows Sec. 2.2 with the substitutions of Sec. 3.3:
//   1. P_k by Eq. DFT-MFT (device kernel)
//   2. for k = 0..N/2 (Eq. Aa_b-sequence) at s_k = eta + i k dw (Sec. 3.1):
//        right-hand side b_k (Eq. Aa_b), operator A_k (near blocks + ACA),
//        initial guess (zero or Sec. 4.2 extrapolation),
//        block-Jacobi GMRES (Sec. 5) whose restarts start from the true
//        residual accumulated in FP64 (iterative refinement of the c64 solve)
//   3. bem_time_response: Eq. IDFT-MFT with the window of Sec. 3.2.
#include <algorithm>
#include <atomic>
#include <chrono>
#include <cmath>
#include <complex>
#include <cstdio>
#include <cstring>
#include <string>
#include <thread>
#include <vector>

#include "bem_internal.h"
#include "bem_launch.h"

using bem::c128;
using bem::c64;

namespace bem {

int fail(bem_ctx* ctx, int code, const std::string& msg) {
  if (ctx) ctx->err = msg;
  return code;
}

int fail_cuda(bem_ctx* ctx, cudaError_t e, const char* what, const char* file, int line) {
  char buf[512];
  snprintf(buf, sizeof(buf), "CUDA error %s (%s) in %s at %s:%d", cudaGetErrorName(e), cudaGetErrorString(e),
           what, file, line);
  if (ctx) ctx->err = buf;
  return e == cudaErrorMemoryAllocation ? BEM_ERR_OOM : BEM_ERR_CUDA;
}

// Gauss-Legendre nodes/weights on [0, 1] by Newton iteration on P_q.
void make_rule_tables(RuleTables& t) {
  memset(&t, 0, sizeof(t));
  for (int q = 1; q <= GL_MAX; ++q) {
    for (int i = 0; i < q; ++i) {
      long double x = cosl(3.14159265358979323846264338327950288L * (i + 0.75L) / (q + 0.5L));
      long double dp = 0;
      for (int it = 0; it < 100; ++it) {
        long double p0 = 1, p1 = x;
        for (int k = 2; k <= q; ++k) {
          long double p2 = ((2 * k - 1) * x * p1 - (k - 1) * p0) / k;
          p0 = p1;
          p1 = p2;
        }
        dp = q * (x * p1 - p0) / (x * x - 1);
        long double dx = p1 / dp;
        x -= dx;
        if (fabsl(dx) < 1e-19L) break;
      }
      long double p0 = 1, p1 = x;
      for (int k = 2; k <= q; ++k) {
        long double p2 = ((2 * k - 1) * x * p1 - (k - 1) * p0) / k;
        p0 = p1;
        p1 = p2;
      }
      dp = q * (x * p1 - p0) / (x * x - 1);
      long double w = 2 / ((1 - x * x) * dp * dp);
      t.gl_x[q][q - 1 - i] = (double)((x + 1) / 2);
      t.gl_w[q][q - 1 - i] = (double)(w / 2);
    }
    // sort ascending
    std::vector<std::pair<double, double>> v;
    for (int i = 0; i < q; ++i) v.push_back({t.gl_x[q][i], t.gl_w[q][i]});
    std::sort(v.begin(), v.end());
    for (int i = 0; i < q; ++i) {
      t.gl_x[q][i] = v[i].first;
      t.gl_w[q][i] = v[i].second;
    }
  }
  for (int q = 0; q <= GL_MAX; ++q)
    for (int i = 0; i < GL_MAX; ++i) {
      t.gl_xf[q][i] = (float)t.gl_x[q][i];
      t.gl_wf[q][i] = (float)t.gl_w[q][i];
    }
}

// Taylor coefficients of Phi, Psi, A, B, C (see KParams). From the
// exponential series, the regular parts of the bracketed functions are
//   A(z) - 1/z^2 : a_m = (-1)^m [1/m! - 1/(m+1)! + 1/(m+2)!]
//   B(z) - 1/z^2 : b_m = (-1)^m [1/(m+2)! - 1/(m+1)!]
//   C(z) - 3/z^2 : c_m = (-1)^m [1/m! - 3/(m+1)! + 3/(m+2)!]
// and with gamma = c_s / c_p, beta2 = gamma^2, k2 = 1 / gamma^2:
//   phi_m = a_m - gamma^(m+2) b_m,  psi_m = c_m (1 - gamma^(m+2)).
template <typename R> KParams<R> make_params(const bem_ctx* ctx, double sre, double sim) {
  KParams<R> P;
  std::complex<double> s(sre, sim);
  std::complex<double> ks = s / ctx->cs, kp = s / ctx->cp;
  P.s = {R(sre), R(sim)};
  P.ks = {R(ks.real()), R(ks.imag())};
  P.kp = {R(kp.real()), R(kp.imag())};
  P.beta2 = R((ctx->cs / ctx->cp) * (ctx->cs / ctx->cp));
  P.k2 = R((ctx->cp / ctx->cs) * (ctx->cp / ctx->cs));
  P.u_scale = R(1.0 / (4.0 * M_PI * ctx->mu));
  P.t_scale = R(1.0 / (4.0 * M_PI));
  P.nu = R(ctx->nu);
  P.kel_u = R(1.0 / (16.0 * M_PI * ctx->mu * (1.0 - ctx->nu)));
  P.kel_t = R(1.0 / (8.0 * M_PI * (1.0 - ctx->nu)));
  long double g = (long double)ctx->cs / (long double)ctx->cp;
  long double k2 = 1.0L / (g * g);
  long double fact[SER_MAX + 3];
  fact[0] = 1;
  for (int k = 1; k < SER_MAX + 3; ++k) fact[k] = fact[k - 1] * k;
  long double gp = g * g;  // gamma^(m+2)
  for (int m = 0; m < SER_MAX; ++m) {
    long double sg = (m % 2) ? -1 : 1;
    long double am = sg * (1 / fact[m] - 1 / fact[m + 1] + 1 / fact[m + 2]);
    long double bm = sg * (1 / fact[m + 2] - 1 / fact[m + 1]);
    long double cm = sg * (1 / fact[m] - 3 / fact[m + 1] + 3 / fact[m + 2]);
    long double ph = am - gp * bm;
    long double ps = cm * (1 - gp);
    P.ser[0][m] = R(ph);
    P.ser[1][m] = R(ps);
    P.ser[2][m] = R((m - 1) * ph - ps);
    P.ser[3][m] = R(2 * (3 - m) * ps);
    P.ser[4][m] = R(k2 * ((m - 1) * ph - (m + 1) * ps) - 2 * ((m - 1) * ph - m * ps));
    gp *= g;
  }
  return P;
}

}  // namespace bem

using namespace bem;

// ---------------------------------------------------------------------------
// small kernels local to the orchestration
// ---------------------------------------------------------------------------
__global__ void k_permute_pattern(const double* __restrict__ in, const int* __restrict__ perm, int ne,
                                  double* __restrict__ out) {
  int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= ne) return;
  int e = perm[k];
  for (int a = 0; a < 3; ++a) out[3 * k + a] = in[3 * e + a];
}

// deterministic compaction of elements with a nonzero pattern (one CTA)
__global__ void k_loaded(const double* __restrict__ pat, int ne, int* __restrict__ list, int* __restrict__ count) {
  __shared__ int wt[32];
  __shared__ int base;
  if (threadIdx.x == 0) base = 0;
  __syncthreads();
  int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
  for (int c0 = 0; c0 < ne; c0 += blockDim.x) {
    int e = c0 + threadIdx.x;
    bool f = e < ne && (pat[3 * e] != 0.0 || pat[3 * e + 1] != 0.0 || pat[3 * e + 2] != 0.0);
    unsigned m = __ballot_sync(0xffffffffu, f);
    if (lane == 0) wt[wid] = __popc(m);
    __syncthreads();
    int before = 0, tot = 0;
    for (int w = 0; w < nw; ++w) {
      if (w < wid) before += wt[w];
      tot += wt[w];
    }
    if (f) list[base + before + __popc(m & ((1u << lane) - 1))] = e;
    __syncthreads();
    if (threadIdx.x == 0) base += tot;
    __syncthreads();
  }
  if (threadIdx.x == 0) *count = base;
}

__global__ void k_pinv_cast(const c128* __restrict__ a, c64* __restrict__ b, long long n) {
  long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (i < n) b[i] = c64{(float)a[i].re, (float)a[i].im};
}

// ---------------------------------------------------------------------------
// helpers
// ---------------------------------------------------------------------------
namespace {

struct Timer {
  cudaEvent_t a = nullptr, b = nullptr;
  Timer() {
    cudaEventCreate(&a);
    cudaEventCreate(&b);
  }
  ~Timer() {
    cudaEventDestroy(a);
    cudaEventDestroy(b);
  }
};

int check_launch(bem_ctx* ctx, const char* what) {
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return fail_cuda(ctx, e, what, __FILE__, __LINE__);
  return BEM_OK;
}

#define CK(what)                                 \
  do {                                           \
    int _r = check_launch(ctx, what);            \
    if (_r != BEM_OK) return _r;                 \
  } while (0)

#define TRY(expr)                \
  do {                           \
    int _r = (expr);             \
    if (_r != BEM_OK) return _r; \
  } while (0)

int set_device(bem_ctx* ctx) {
  BEM_CUDA_TRY(cudaSetDevice(ctx->device));
  return BEM_OK;
}

int ensure_static(bem_ctx* ctx, bool need_fp64);

bool is_mixed(const bem_ctx* ctx) { return ctx->prec == BEM_PREC_C64_MIXED; }

cudaEvent_t take_event(bem_ctx* ctx) {
  if (ctx->event_pool.empty()) {
    cudaEvent_t e;
    cudaEventCreate(&e);
    return e;
  }
  cudaEvent_t e = ctx->event_pool.back();
  ctx->event_pool.pop_back();
  return e;
}

// Records the start of a timed region (returns the event or null).
cudaEvent_t prof_begin(bem_ctx* ctx, cudaStream_t st = nullptr) {
  if (!ctx->profiling) return nullptr;
  cudaEvent_t a = take_event(ctx);
  cudaEventRecord(a, st ? st : ctx->stream);
  return a;
}
void prof_end(bem_ctx* ctx, cudaEvent_t a, int kind, double base = 0.0, double mult = 0.0, cudaStream_t st = nullptr) {
  if (!a) return;
  cudaEvent_t b = take_event(ctx);
  cudaEventRecord(b, st ? st : ctx->stream);
  ctx->pending.push_back({a, b, base, mult, kind == 0 ? ctx->prof_slot : 0, kind});
}

// Cooperative (grid-synchronising) launches of a context that shares the GPU
// with other contexts' streams (the meshes of a batched sweep) go through one
// stream common to those contexts, ordered against the context's own stream
// by events: two such grids then never wait for residency at the same time.
// A lone context (and the parent of a batch) launches on its own stream.
class CoopLane {
 public:
  CoopLane(bem_ctx* ctx, cudaStream_t st) : ctx_(ctx), st_(st) {
    if (!ctx->coop_stream) return;  // set only together with coop_in, coop_out (bem_add_mesh)
    e_ = cudaEventRecord(ctx->coop_in, st);
    if (e_ == cudaSuccess) e_ = cudaStreamWaitEvent(ctx->coop_stream, ctx->coop_in, 0);
  }
  cudaError_t status() const { return e_; }
  cudaStream_t stream() const { return ctx_->coop_stream ? ctx_->coop_stream : st_; }
  cudaError_t join() {
    if (!ctx_->coop_stream) return cudaSuccess;
    cudaError_t e = cudaEventRecord(ctx_->coop_out, ctx_->coop_stream);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(st_, ctx_->coop_out, 0);
    return e;
  }

 private:
  bem_ctx* ctx_;
  cudaStream_t st_;
  cudaError_t e_ = cudaSuccess;
};

// Exchanges the operator set in use with the set back[i] (host pointers
// only: work already enqueued keeps the buffers it was given).
template <typename T> void swap_buf(DevBuf<T>& a, DevBuf<T>& b) {
  std::swap(a.p, b.p);
  std::swap(a.n, b.n);
}
void swap_ops(bem_ctx* ctx, int i) {
  OpSet& o = ctx->back[i];
  swap_buf(ctx->near32, o.near32);
  swap_buf(ctx->u32, o.u32);
  swap_buf(ctx->v32, o.v32);
  swap_buf(ctx->prec_inv32, o.prec_inv32);
  swap_buf(ctx->near64, o.near64);
  swap_buf(ctx->u64, o.u64);
  swap_buf(ctx->v64, o.v64);
  swap_buf(ctx->prec_inv, o.prec_inv);
  swap_buf(ctx->minv32, o.minv32);
  swap_buf(ctx->minv64, o.minv64);
  std::swap(ctx->minv_ready, o.minv_ready);
  swap_buf(ctx->b64, o.b64);
  swap_buf(ctx->rank, o.rank);
  swap_buf(ctx->aca_fail, o.aca_fail);
  swap_buf(ctx->status, o.status);
  swap_buf(ctx->fbase, o.fbase);
  std::swap(ctx->fbase_ready, o.fbase_ready);
  std::swap(ctx->near_zero_pending, o.near_zero_pending);
  std::swap(ctx->prof_slot, o.prof_slot);
}
// Folds completed timings into the counters; timings whose end event has not
// completed yet stay pending (after a stream sync every one has completed).
void prof_harvest(bem_ctx* ctx) {
  size_t keep = 0;
  for (size_t k = 0; k < ctx->pending.size(); ++k) {
    auto& p = ctx->pending[k];
    if (cudaEventQuery(p.b) == cudaErrorNotReady) {
      ctx->pending[keep++] = p;
      continue;
    }
    float ms = 0;
    if (cudaEventElapsedTime(&ms, p.a, p.b) == cudaSuccess) {
      if (p.kind == 0) {
        ctx->prof_hmv_ms += ms;
        ctx->prof_products.push_back({p.base, p.mult, p.slot});
        ctx->prof_hmv_launches += 1;
      } else {
        ctx->prof_asm_ms += ms;
        ctx->prof_asm_calls += 1;
      }
    }
    ctx->event_pool.push_back(p.a);
    ctx->event_pool.push_back(p.b);
  }
  ctx->pending.resize(keep);
  cudaGetLastError();  // a not-ready query leaves no sticky error; clear the last-error slot
}

// Algorithmic bytes of one H-matrix product: every stored operator entry in
// use (near blocks, U and V columns up to the rank), x read once, y written
// once; the low-rank entries are known on the device only (counted after each
// assembly into prof_dev), so the product records base + mult x entries.
void prof_end_hmv(bem_ctx* ctx, cudaEvent_t a, int op_bytes, int x_bytes, int y_bytes, int nrhs) {
  prof_end(ctx, a, 0, (double)op_bytes * ctx->near_entries + (double)nrhs * ctx->N * (x_bytes + y_bytes),
           (double)op_bytes);
}

constexpr int PROF_SLOTS = 1 << 16;

__global__ void k_count_zero(const int* __restrict__ v, int n, long long* __restrict__ out) {
  int c = 0;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) c += v[i] == 0;
  c = __reduce_add_sync(0xffffffffu, c);
  if ((threadIdx.x & 31) == 0 && c) atomicAdd(reinterpret_cast<unsigned long long*>(out), (unsigned long long)c);
}
__global__ void k_lowrank_entries(const int* __restrict__ rank, const FarBlk* __restrict__ far, int n,
                                  long long* __restrict__ out) {
  long long c = 0;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
    c += (long long)rank[i] * 3 * (far[i].nr + far[i].nc);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) c += __shfl_xor_sync(0xffffffffu, c, o);
  if ((threadIdx.x & 31) == 0 && c) atomicAdd(reinterpret_cast<unsigned long long*>(out), (unsigned long long)c);
}

}  // namespace

// ---------------------------------------------------------------------------
// context
// ---------------------------------------------------------------------------
extern "C" void bem_default_opts(bem_opts* o) {
  if (!o) return;
  o->tol = 1e-5;
  o->restart = 50;
  o->max_iters = 5000;
  o->aca_tol = 1e-5;
  o->leaf_size = 64;
  o->eta_adm = 1.0;
  o->precision = BEM_PREC_C64_MIXED;
  o->guess = BEM_GUESS_SEM;
  o->sem_k = 4;
  o->dense = 0;
  o->precond = BEM_PRECOND_BLOCK3;
}

extern "C" void bem_destroy(bem_ctx* ctx);

extern "C" int bem_create(bem_ctx** out, int device, void* stream) {
  if (!out) return BEM_ERR_INVALID_ARG;
  *out = nullptr;
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev) return BEM_ERR_CUDA;
  bem_ctx* ctx = new bem_ctx();
  ctx->device = device;
  ctx->stream = (cudaStream_t)stream;
  bem_default_opts(&ctx->mesh_opts);
  if (cudaSetDevice(device) != cudaSuccess) {
    delete ctx;
    return BEM_ERR_CUDA;
  }
  RuleTables t;
  make_rule_tables(t);
  if (upload_rules_assemble(t, ctx->stream) != cudaSuccess || upload_rules_interior(t, ctx->stream) != cudaSuccess ||
      cudaStreamSynchronize(ctx->stream) != cudaSuccess) {
    delete ctx;
    return BEM_ERR_CUDA;
  }
  if (cudaMallocHost(&ctx->host_red, 4096 * sizeof(double)) != cudaSuccess) {
    delete ctx;
    return BEM_ERR_OOM;
  }
  // the solver state's host copy: mapped, written by the solver kernels
  if (cudaHostAlloc(&ctx->gm_mirror, sizeof(GmCtl), cudaHostAllocMapped) != cudaSuccess ||
      cudaHostGetDevicePointer(&ctx->gm_mirror_dev, ctx->gm_mirror, 0) != cudaSuccess) {
    bem_destroy(ctx);
    return BEM_ERR_OOM;
  }
  std::memset(ctx->gm_mirror, 0, sizeof(GmCtl));
  int prio_least = 0, prio_greatest = 0;
  if (cudaDeviceGetStreamPriorityRange(&prio_least, &prio_greatest) != cudaSuccess) prio_least = prio_greatest = 0;
  if (cudaStreamCreateWithPriority(&ctx->aux_stream, cudaStreamNonBlocking, prio_least) != cudaSuccess ||
      cudaStreamCreateWithPriority(&ctx->asm_stream, cudaStreamNonBlocking, prio_least) != cudaSuccess ||
      cudaStreamCreateWithPriority(&ctx->solve_stream, cudaStreamNonBlocking, prio_greatest) != cudaSuccess ||
      cudaEventCreateWithFlags(&ctx->ev_solve_in, cudaEventDisableTiming) != cudaSuccess ||
      cudaEventCreateWithFlags(&ctx->ev_solve_out, cudaEventDisableTiming) != cudaSuccess ||
      cudaEventCreateWithFlags(&ctx->ev_far_cursor, cudaEventDisableTiming) != cudaSuccess ||
      cudaEventCreateWithFlags(&ctx->ev_fork, cudaEventDisableTiming) != cudaSuccess ||
      cudaEventCreateWithFlags(&ctx->ev_join, cudaEventDisableTiming) != cudaSuccess ||
      cudaEventCreateWithFlags(&ctx->ev_asm_ring[0], cudaEventDisableTiming) != cudaSuccess ||
      cudaEventCreateWithFlags(&ctx->ev_asm_ring[1], cudaEventDisableTiming) != cudaSuccess ||
      cudaEventCreateWithFlags(&ctx->ev_asm_ring[2], cudaEventDisableTiming) != cudaSuccess ||
      cudaEventCreateWithFlags(&ctx->ev_free_ring[0], cudaEventDisableTiming) != cudaSuccess ||
      cudaEventCreateWithFlags(&ctx->ev_free_ring[1], cudaEventDisableTiming) != cudaSuccess ||
      cudaEventCreateWithFlags(&ctx->ev_free_ring[2], cudaEventDisableTiming) != cudaSuccess) {
    bem_destroy(ctx);
    return BEM_ERR_CUDA;
  }
  *out = ctx;
  return BEM_OK;
}

extern "C" void bem_destroy(bem_ctx* ctx) {
  if (!ctx) return;
  cudaSetDevice(ctx->device);
  cudaStreamSynchronize(ctx->stream);
  if (ctx->host_red) cudaFreeHost(ctx->host_red);
  for (cudaEvent_t e : ctx->col_events) cudaEventDestroy(e);
  if (ctx->aux_stream) {
    cudaStreamSynchronize(ctx->aux_stream);
    cudaStreamDestroy(ctx->aux_stream);
  }
  if (ctx->asm_stream) {
    cudaStreamSynchronize(ctx->asm_stream);
    cudaStreamDestroy(ctx->asm_stream);
  }
  if (ctx->solve_stream) {
    cudaStreamSynchronize(ctx->solve_stream);
    cudaStreamDestroy(ctx->solve_stream);
  }
  if (ctx->ev_solve_in) cudaEventDestroy(ctx->ev_solve_in);
  if (ctx->ev_solve_out) cudaEventDestroy(ctx->ev_solve_out);
  if (ctx->ev_far_cursor) cudaEventDestroy(ctx->ev_far_cursor);
  if (ctx->ev_fork) cudaEventDestroy(ctx->ev_fork);
  if (ctx->ev_join) cudaEventDestroy(ctx->ev_join);
  for (int r = 0; r < 3; ++r) {
    if (ctx->ev_asm_ring[r]) cudaEventDestroy(ctx->ev_asm_ring[r]);
    if (ctx->ev_free_ring[r]) cudaEventDestroy(ctx->ev_free_ring[r]);
  }
  for (auto& p : ctx->pending) {
    cudaEventDestroy(p.a);
    cudaEventDestroy(p.b);
  }
  for (cudaEvent_t e : ctx->event_pool) cudaEventDestroy(e);
  for (size_t i = 0; i < ctx->batch.size(); ++i) {
    cudaStream_t bs = ctx->batch[i]->stream;
    bem_destroy(ctx->batch[i]);
    cudaStreamDestroy(bs);
  }
  if (ctx->coop_in) cudaEventDestroy(ctx->coop_in);
  if (ctx->coop_out) cudaEventDestroy(ctx->coop_out);
  if (ctx->batch_coop) {
    cudaStreamSynchronize(ctx->batch_coop);
    cudaStreamDestroy(ctx->batch_coop);
  }
  mlp_free(ctx);
  if (ctx->gm_mirror) cudaFreeHost(ctx->gm_mirror);
  if (ctx->sweep_pin) cudaFreeHost(ctx->sweep_pin);  // the streams writing it are synchronised above
  delete ctx;
}

extern "C" const char* bem_last_error(const bem_ctx* ctx) { return ctx ? ctx->err.c_str() : "null context"; }

extern "C" int bem_set_material(bem_ctx* ctx, double E, double nu, double rho) {
  if (!ctx) return BEM_ERR_INVALID_ARG;
  if (!(E > 0) || !(rho > 0) || !(nu > -1.0) || !(nu < 0.5))
    return fail(ctx, BEM_ERR_INVALID_ARG, "material needs E > 0, rho > 0, -1 < nu < 0.5");
  bool changed = !ctx->have_mat || E != ctx->E || nu != ctx->nu || rho != ctx->rho;
  ctx->E = E;
  ctx->nu = nu;
  ctx->rho = rho;
  ctx->mu = E / (2.0 * (1.0 + nu));
  ctx->lam = E * nu / ((1.0 + nu) * (1.0 - 2.0 * nu));
  ctx->cs = std::sqrt(ctx->mu / rho);
  ctx->cp = std::sqrt((ctx->lam + 2.0 * ctx->mu) / rho);
  ctx->have_mat = true;
  if (changed) ctx->sing_static.release();  // Kelvin parts depend on mu, nu
  ctx->assembled = false;
  return BEM_OK;
}

extern "C" int bem_set_window(bem_ctx* ctx, double eta, int window) {
  if (!ctx) return BEM_ERR_INVALID_ARG;
  if (!(eta >= 0) || !std::isfinite(eta)) return fail(ctx, BEM_ERR_INVALID_ARG, "eta must be finite and >= 0");
  if (window < BEM_WIN_NONE || window > BEM_WIN_BLACKMAN) return fail(ctx, BEM_ERR_INVALID_ARG, "unknown window");
  ctx->eta = eta;
  ctx->window = window;
  return BEM_OK;
}

// ---------------------------------------------------------------------------
// mesh
// ---------------------------------------------------------------------------
// Admissible blocks assembled one warp each (the others one CTA each).
static bool far_small_class(const FarBlk& fb) { return fb.nr + fb.nc <= 256; }

static int mesh_impl(bem_ctx* ctx, const double* xyz_d, long long nv, const int* tri_d, int ne,
                     const signed char* bc_d, const bem_opts* opts) {
  cudaStream_t st = ctx->stream;
  bem_opts o;
  bem_default_opts(&o);
  if (opts) o = *opts;
  if (o.leaf_size < 1 || o.leaf_size > 1024) return fail(ctx, BEM_ERR_INVALID_ARG, "leaf_size out of range");
  if (!(o.eta_adm > 0)) return fail(ctx, BEM_ERR_INVALID_ARG, "eta_adm must be > 0");
  ctx->have_mesh = false;
  ctx->assembled = false;
  ctx->aca_warm_ok = false;
  ctx->nf = 0;
  ctx->mesh_opts = o;
  ctx->ne = ne;
  ctx->N = 3LL * ne;

  DevBuf<double> cen, hh;
  DevBuf<int> bad;
  BEM_CUDA_TRY(cen.alloc(3LL * ne));
  BEM_CUDA_TRY(hh.alloc(ne));
  BEM_CUDA_TRY(bad.alloc(1));
  BEM_CUDA_TRY(cudaMemsetAsync(bad.p, 0, sizeof(int), st));
  launch_centroids(xyz_d, nv, tri_d, ne, cen.p, hh.p, bad.p, st);
  CK("centroids");
  std::vector<double> cen_h(3LL * ne), h_h(ne);
  int bad_h = 0;
  BEM_CUDA_TRY(cudaMemcpyAsync(cen_h.data(), cen.p, 3LL * ne * sizeof(double), cudaMemcpyDeviceToHost, st));
  BEM_CUDA_TRY(cudaMemcpyAsync(h_h.data(), hh.p, ne * sizeof(double), cudaMemcpyDeviceToHost, st));
  BEM_CUDA_TRY(cudaMemcpyAsync(&bad_h, bad.p, sizeof(int), cudaMemcpyDeviceToHost, st));
  BEM_CUDA_TRY(cudaStreamSynchronize(st));
  if (bad_h == 1) return fail(ctx, BEM_ERR_INVALID_ARG, "triangle vertex index out of range");
  if (bad_h == 2) return fail(ctx, BEM_ERR_INVALID_ARG, "degenerate triangle");

  build_cluster_tree(cen_h.data(), h_h.data(), ne, o.leaf_size, o.eta_adm, RHO2_NEAR, o.dense != 0, ctx->tree);
  const ClusterTree& tr = ctx->tree;
  BEM_CUDA_TRY(ctx->perm.alloc(ne));
  BEM_CUDA_TRY(ctx->iperm.alloc(ne));
  BEM_CUDA_TRY(cudaMemcpyAsync(ctx->perm.p, tr.perm.data(), ne * sizeof(int), cudaMemcpyHostToDevice, st));
  BEM_CUDA_TRY(cudaMemcpyAsync(ctx->iperm.p, tr.iperm.data(), ne * sizeof(int), cudaMemcpyHostToDevice, st));
  BEM_CUDA_TRY(ctx->ef.alloc(ne));
  BEM_CUDA_TRY(ctx->ed.alloc(ne));
  BEM_CUDA_TRY(ctx->bc.alloc(ne));
  launch_geometry(xyz_d, tri_d, ctx->perm.p, bc_d, ne, ctx->ef.p, ctx->ed.p, ctx->bc.p, st);
  CK("geometry");
  ctx->bc_host.resize(ne);
  BEM_CUDA_TRY(cudaMemcpyAsync(ctx->bc_host.data(), ctx->bc.p, ne, cudaMemcpyDeviceToHost, st));

  // element normals (tree order), for the flat-face test of the far blocks
  std::vector<ElemD> ed_h(ne);
  BEM_CUDA_TRY(cudaMemcpyAsync(ed_h.data(), ctx->ed.p, (size_t)ne * sizeof(ElemD), cudaMemcpyDeviceToHost, st));
  BEM_CUDA_TRY(cudaStreamSynchronize(st));
  // a cluster [b0, b0 + nb) is faceted when at least half of its elements
  // share their normal with its first, middle or last element (flat faces of
  // boxes and cubes; on a curved surface every element has its own normal)
  auto faceted = [&](int b0, int nb) {
    const int ref[3] = {b0, b0 + nb / 2, b0 + nb - 1};
    int same = 0;
    for (int e = b0; e < b0 + nb; ++e) {
      const ElemD& E = ed_h[e];
      for (int q = 0; q < 3; ++q) {
        const ElemD& R = ed_h[ref[q]];
        if (E.n[0] * R.n[0] + E.n[1] * R.n[1] + E.n[2] * R.n[2] > 1.0 - 1e-9) {
          ++same;
          break;
        }
      }
    }
    return 2 * same >= nb && nb > 3;
  };

  // near / far block descriptors
  ctx->near_h.clear();
  ctx->far_h.clear();
  long long noff = 0;
  for (const BlockPair& bp : tr.near) {
    const Cluster& t = tr.nodes[bp.tau];
    const Cluster& s = tr.nodes[bp.sigma];
    NearBlk nb;
    nb.off = noff;
    nb.r0 = t.begin;
    nb.nr = t.size();
    nb.c0 = s.begin;
    nb.nc = s.size();
    nb.ld = 3 * nb.nr + ((3 * nb.nr) & 1);
    noff += (long long)nb.ld * 3 * nb.nc;
    noff += noff & 1;
    ctx->near_h.push_back(nb);
  }
  ctx->near_entries = noff;
  ctx->near_zero_pending = true;
  for (OpSet& b : ctx->back) b.near_zero_pending = true;  // the other operator sets' padding rows too
  long long ucap = 0, vcap = 0, bigcap = 0, uinit = 0, vinit = 0;
  int toff = 0;
  for (const BlockPair& bp : tr.far) {
    const Cluster& t = tr.nodes[bp.tau];
    const Cluster& s = tr.nodes[bp.sigma];
    FarBlk fb;
    fb.r0 = t.begin;
    fb.nr = t.size();
    fb.c0 = s.begin;
    fb.nc = s.size();
    int mn = 3 * std::min(fb.nr, fb.nc);
    fb.rmax = std::min(mn, ACA_RANK_CAP);
    fb.toff = toff;
    fb.flat = faceted(fb.r0, fb.nr) || faceted(fb.c0, fb.nc) ? 1 : 0;
    ucap += 3LL * fb.nr * fb.rmax;
    vcap += 3LL * fb.nc * fb.rmax;
    uinit += 3LL * fb.nr * std::min(fb.rmax, POOL_INIT_RANK);
    vinit += 3LL * fb.nc * std::min(fb.rmax, POOL_INIT_RANK);
    bigcap = std::max(bigcap, 3LL * std::max(fb.nr, fb.nc) * fb.rmax);
    toff += fb.rmax;
    ctx->far_h.push_back(fb);
  }
  ctx->u_entries = ucap;
  ctx->v_entries = vcap;
  ctx->u_init = uinit;
  ctx->v_init = vinit;
  ctx->t_entries = toff;
  // factor storage: full (capped factors in place, two operator sets) unless
  // that would take over a quarter of the device memory, or compact is asked for
  {
    size_t freeb = 0, totalb = 0;
    BEM_CUDA_TRY(cudaMemGetInfo(&freeb, &totalb));
    const double esz = o.precision == BEM_PREC_C128 ? 16.0 : 8.0;
    const double full_bytes = 2.0 * (double)(ucap + vcap) * esz;
    ctx->far_compact = ctx->far_mode_req == BEM_FAR_COMPACT ||
                       (ctx->far_mode_req == BEM_FAR_AUTO && full_bytes > 0.25 * (double)totalb);
    const long long ws_total = ctx->far_ws_req > 0 ? ctx->far_ws_req / 16 : (1LL << 30);
    const long long half = ctx->far_compact ? std::max(ws_total / 2, bigcap) : 0;
    ctx->ws_entries = half;
    ctx->far_batches.clear();
    FarBatch cur{0, 0, 0, 0, 0, 0};
    long long cu = 0, cv = 0;
    int ns = 0, nl = 0;
    const int nfb = (int)ctx->far_h.size();
    for (int b = 0; b < nfb; ++b) {
      FarBlk& fb = ctx->far_h[b];
      const long long nu = 3LL * fb.nr * fb.rmax, nvv = 3LL * fb.nc * fb.rmax;
      if (ctx->far_compact && b > cur.b0 && (cu + nu > half || cv + nvv > half)) {
        cur.b1 = b;
        cur.s1 = ns;
        cur.l1 = nl;
        ctx->far_batches.push_back(cur);
        cur = FarBatch{b, 0, ns, 0, nl, 0};
        cu = cv = 0;
      }
      fb.uoff = cu;
      fb.voff = cv;
      cu += nu;
      cv += nvv;
      (far_small_class(fb) ? ns : nl) += 1;
    }
    if (nfb) {
      cur.b1 = nfb;
      cur.s1 = ns;
      cur.l1 = nl;
      ctx->far_batches.push_back(cur);
    }
    // a new mesh invalidates every set's factor offsets; the sets not in use
    // give back their operator storage (it is reallocated when next used)
    ctx->fbase_ready = false;
    for (OpSet& b : ctx->back) {
      b.fbase_ready = false;
      b.near32.release();
      b.u32.release();
      b.v32.release();
      b.near64.release();
      b.u64.release();
      b.v64.release();
    }
    if (ctx->far_compact) {
      // pools are sized by the first assembly's need
      ctx->u32.release();
      ctx->v32.release();
      ctx->u64.release();
      ctx->v64.release();
    }
    ctx->far_regrows = 0;
  }
  BEM_CUDA_TRY(ctx->near_d.alloc(std::max<size_t>(1, ctx->near_h.size())));
  BEM_CUDA_TRY(ctx->far_d.alloc(std::max<size_t>(1, ctx->far_h.size())));
  if (!ctx->near_h.empty())
    BEM_CUDA_TRY(cudaMemcpyAsync(ctx->near_d.p, ctx->near_h.data(), ctx->near_h.size() * sizeof(NearBlk),
                                 cudaMemcpyHostToDevice, st));
  if (!ctx->far_h.empty())
    BEM_CUDA_TRY(cudaMemcpyAsync(ctx->far_d.p, ctx->far_h.data(), ctx->far_h.size() * sizeof(FarBlk),
                                 cudaMemcpyHostToDevice, st));

  // leaves and matrix-vector panels (CSR by leaf row)
  ctx->leaf_nodes.clear();
  for (int id = 0; id < (int)tr.nodes.size(); ++id)
    if (tr.nodes[id].leaf()) ctx->leaf_nodes.push_back(id);
  std::sort(ctx->leaf_nodes.begin(), ctx->leaf_nodes.end(),
            [&](int a, int b) { return tr.nodes[a].begin < tr.nodes[b].begin; });
  int L = (int)ctx->leaf_nodes.size();
  ctx->nleaves = L;
  std::vector<int> leaf_idx(tr.nodes.size(), -1);
  std::vector<int> r0(L), nr(L);
  for (int l = 0; l < L; ++l) {
    leaf_idx[ctx->leaf_nodes[l]] = l;
    r0[l] = tr.nodes[ctx->leaf_nodes[l]].begin;
    nr[l] = tr.nodes[ctx->leaf_nodes[l]].size();
  }
  std::vector<std::vector<Panel>> per(L);
  for (size_t b = 0; b < ctx->near_h.size(); ++b) {
    const NearBlk& nb = ctx->near_h[b];
    int l = leaf_idx[tr.near[b].tau];
    Panel p;
    p.data = nb.off;
    p.ld = nb.ld;
    p.ncols = 3 * nb.nc;
    p.xoff = 3 * nb.c0;
    p.kind = 0;
    per[l].push_back(p);
  }
  for (size_t b = 0; b < ctx->far_h.size(); ++b) {
    const FarBlk& fb = ctx->far_h[b];
    // every leaf inside the row cluster (a run of consecutive leaves) gets
    // the matching slice of U_b
    int l = (int)(std::lower_bound(r0.begin(), r0.end(), fb.r0) - r0.begin());
    for (; l < L && r0[l] + nr[l] <= fb.r0 + fb.nr; ++l) {
      Panel p;
      p.data = 3LL * (r0[l] - fb.r0);
      p.ld = 3 * fb.nr;
      p.ncols = 0;
      p.xoff = (int)b;
      p.kind = 1;
      per[l].push_back(p);
    }
  }
  std::vector<int> pptr(L + 1, 0);
  std::vector<Panel> pan;
  for (int l = 0; l < L; ++l) {
    pptr[l] = (int)pan.size();
    pan.insert(pan.end(), per[l].begin(), per[l].end());
  }
  pptr[L] = (int)pan.size();
  // tasks: runs of at most ~TASK_COLS stored columns of one leaf row (the far
  // panels counted at their rank cap), so that there are several CTAs per SM
  const int TASK_COLS = 576;
  std::vector<Task> tk;
  std::vector<int> tptr(L + 1, 0);
  long long slot = 0;
  for (int l = 0; l < L; ++l) {
    tptr[l] = (int)tk.size();
    for (int kind = 0; kind < 2; ++kind) {
      int p = pptr[l];
      while (p < pptr[l + 1]) {
        if (pan[p].kind != kind) {
          ++p;
          continue;
        }
        Task t;
        t.leaf = l;
        t.kind = kind;
        t.slot = (int)slot;
        t.p0 = p;
        int cols = 0;
        // panels of one kind are contiguous in a leaf's list (near first, then far)
        while (p < pptr[l + 1] && pan[p].kind == kind && cols < TASK_COLS) {
          cols += kind == 0 ? pan[p].ncols : ctx->far_h[pan[p].xoff].rmax;
          ++p;
        }
        t.p1 = p;
        slot += 3LL * nr[l] + 1;  // +1: a near task writes an even number of rows
        tk.push_back(t);
      }
    }
  }
  tptr[L] = (int)tk.size();
  ctx->ntasks = (int)tk.size();
  {
    std::vector<int> order(tk.size());
    std::vector<long long> tcost(tk.size(), 0);  // stored entries read by each task
    for (int i = 0; i < (int)tk.size(); ++i) {
      order[i] = i;
      for (int p = tk[i].p0; p < tk[i].p1; ++p)
        tcost[i] += (long long)3 * nr[tk[i].leaf] *
                    (pan[p].kind == 0 ? pan[p].ncols : ctx->far_h[pan[p].xoff].rmax);
    }
    std::sort(order.begin(), order.end(),
              [&](int a, int b) { return tcost[a] != tcost[b] ? tcost[a] > tcost[b] : a < b; });
    BEM_CUDA_TRY(ctx->task_order.alloc(std::max<size_t>(1, order.size())));
    if (!order.empty())
      BEM_CUDA_TRY(cudaMemcpyAsync(ctx->task_order.p, order.data(), order.size() * sizeof(int),
                                   cudaMemcpyHostToDevice, st));
    BEM_CUDA_TRY(cudaStreamSynchronize(st));  // order outlives the copy
  }
  ctx->part_rows = slot;
  BEM_CUDA_TRY(ctx->leaf_cnt.alloc(std::max(1, L)));
  BEM_CUDA_TRY(cudaMemsetAsync(ctx->leaf_cnt.p, 0, std::max(1, L) * sizeof(int), st));
  BEM_CUDA_TRY(ctx->tasks.alloc(std::max<size_t>(1, tk.size())));
  BEM_CUDA_TRY(ctx->task_ptr.alloc(L + 1));
  // fused product items: the near tasks (their panels) and one item per
  // admissible block; each leaf's contributions in a fixed order (its near
  // tasks, then the blocks over its rows by block index)
  {
    std::vector<HItem> hi;
    std::vector<double> cost;
    std::vector<std::vector<long long>> contrib(L);
    long long hs = 0;
    for (const Task& t : tk) {
      if (t.kind != 0) continue;
      HItem it;
      it.slot = hs;
      it.kind = 0;
      it.p0 = t.p0;
      it.p1 = t.p1;
      it.l0 = t.leaf;
      it.l1 = t.leaf + 1;
      double c = 0;
      for (int p = t.p0; p < t.p1; ++p) c += 3.0 * nr[t.leaf] * pan[p].ncols;
      contrib[t.leaf].push_back(hs);
      hs += 3LL * nr[t.leaf] + 1;  // +1: rows are written in pairs
      hi.push_back(it);
      cost.push_back(c);
    }
    // far items: the admissible blocks of one row cluster, in runs bounded in
    // count, in summed rank caps (the V^T x values stay in shared memory) and
    // in estimated entries (ranks are known on the device only; a typical
    // rank of 48 stands for them)
    std::vector<int> fl(ctx->far_h.size());
    for (size_t b = 0; b < fl.size(); ++b) fl[b] = (int)b;
    std::stable_sort(fl.begin(), fl.end(), [&](int a, int b) {
      const FarBlk &A = ctx->far_h[a], &Bq = ctx->far_h[b];
      return A.r0 != Bq.r0 ? A.r0 < Bq.r0 : A.nr < Bq.nr;
    });
    const double ITEM_ENTRIES = 131072.0;
    int tcols_max = 0;
    for (size_t i = 0; i < fl.size();) {
      const FarBlk& f0 = ctx->far_h[fl[i]];
      size_t j = i;
      int tcols = 0;
      double c = 0;
      while (j < fl.size()) {
        const FarBlk& fj = ctx->far_h[fl[j]];
        if (fj.r0 != f0.r0 || fj.nr != f0.nr) break;
        const double cj = std::min(fj.rmax, 48) * 3.0 * (fj.nr + fj.nc);
        if (j > i && ((int)(j - i) >= HITEM_MAX_BLOCKS || tcols + fj.rmax > HITEM_MAX_TCOLS || c + cj > ITEM_ENTRIES))
          break;
        tcols += fj.rmax;
        c += cj;
        ++j;
      }
      HItem it;
      it.slot = hs;
      it.kind = 1;
      it.p0 = (int)i;
      it.p1 = (int)j;
      it.l0 = (int)(std::lower_bound(r0.begin(), r0.end(), f0.r0) - r0.begin());
      int l = it.l0;
      for (; l < L && r0[l] + nr[l] <= f0.r0 + f0.nr; ++l) contrib[l].push_back(hs + 3LL * (r0[l] - f0.r0));
      it.l1 = l;
      cost.push_back(c);
      hs += 3LL * f0.nr + 1;
      hi.push_back(it);
      tcols_max = std::max(tcols_max, tcols);
      i = j;
    }
    ctx->hitem_tcols = tcols_max;
    BEM_CUDA_TRY(ctx->hfar_list.alloc(std::max<size_t>(1, fl.size())));
    if (!fl.empty())
      BEM_CUDA_TRY(cudaMemcpyAsync(ctx->hfar_list.p, fl.data(), fl.size() * sizeof(int), cudaMemcpyHostToDevice, st));
    std::vector<int> ord(hi.size());
    for (size_t i = 0; i < ord.size(); ++i) ord[i] = (int)i;
    std::stable_sort(ord.begin(), ord.end(), [&](int a, int b) { return cost[a] > cost[b]; });
    std::vector<HItem> hs_sorted(hi.size());
    for (size_t i = 0; i < ord.size(); ++i) hs_sorted[i] = hi[ord[i]];
    std::vector<int> cptr(L + 1, 0);
    std::vector<long long> coff;
    for (int l = 0; l < L; ++l) {
      cptr[l] = (int)coff.size();
      coff.insert(coff.end(), contrib[l].begin(), contrib[l].end());
    }
    cptr[L] = (int)coff.size();
    ctx->nhitems = (int)hs_sorted.size();
    ctx->hpart_rows = hs;
    BEM_CUDA_TRY(ctx->hitems.alloc(std::max<size_t>(1, hs_sorted.size())));
    BEM_CUDA_TRY(ctx->hc_ptr.alloc(L + 1));
    BEM_CUDA_TRY(ctx->hc_off.alloc(std::max<size_t>(1, coff.size())));
    if (!hs_sorted.empty())
      BEM_CUDA_TRY(cudaMemcpyAsync(ctx->hitems.p, hs_sorted.data(), hs_sorted.size() * sizeof(HItem),
                                   cudaMemcpyHostToDevice, st));
    BEM_CUDA_TRY(cudaMemcpyAsync(ctx->hc_ptr.p, cptr.data(), (L + 1) * sizeof(int), cudaMemcpyHostToDevice, st));
    if (!coff.empty())
      BEM_CUDA_TRY(cudaMemcpyAsync(ctx->hc_off.p, coff.data(), coff.size() * sizeof(long long),
                                   cudaMemcpyHostToDevice, st));
    BEM_CUDA_TRY(cudaStreamSynchronize(st));  // the host vectors outlive the copies
  }
  // leaf-block preconditioner: each leaf's diagonal block is its near block
  // with itself; unavailable when a leaf exceeds LEAF_PRE_MAX_ELEMS
  {
    std::vector<LeafPre> lp(L);
    bool ok = L > 0;
    long long oo = 0;
    std::vector<int> self_blk(L, -1);
    for (size_t b = 0; b < tr.near.size(); ++b)
      if (tr.near[b].tau == tr.near[b].sigma && leaf_idx[tr.near[b].tau] >= 0) self_blk[leaf_idx[tr.near[b].tau]] = (int)b;
    for (int l = 0; l < L && ok; ++l) {
      if (nr[l] > LEAF_PRE_MAX_ELEMS || self_blk[l] < 0) {
        ok = false;
        break;
      }
      const NearBlk& nb = ctx->near_h[self_blk[l]];
      lp[l].off = nb.off;
      lp[l].ld = nb.ld;
      lp[l].m = 3 * nr[l];
      lp[l].ldo = (3 * nr[l] + 1) & ~1;
      lp[l].e0 = r0[l];
      lp[l].ooff = oo;
      oo += (long long)lp[l].ldo * lp[l].m;
    }
    ctx->nleaf_pre = ok ? L : 0;
    ctx->leaf_pre_entries = ok ? oo : 0;
    ctx->minv_ready = false;
    for (OpSet& b : ctx->back) b.minv_ready = false;
    if (ok) {
      BEM_CUDA_TRY(ctx->leaf_pre.alloc(L));
      BEM_CUDA_TRY(cudaMemcpyAsync(ctx->leaf_pre.p, lp.data(), L * sizeof(LeafPre), cudaMemcpyHostToDevice, st));
      BEM_CUDA_TRY(cudaStreamSynchronize(st));
    }
  }
  // 4 rhs x complex FP64, for the task product and the fused product
  BEM_CUDA_TRY(ctx->part.alloc(std::max<long long>(1, 8 * std::max(slot, ctx->hpart_rows))));
  if (!tk.empty())
    BEM_CUDA_TRY(cudaMemcpyAsync(ctx->tasks.p, tk.data(), tk.size() * sizeof(Task), cudaMemcpyHostToDevice, st));
  BEM_CUDA_TRY(cudaMemcpyAsync(ctx->task_ptr.p, tptr.data(), (L + 1) * sizeof(int), cudaMemcpyHostToDevice, st));
  BEM_CUDA_TRY(ctx->leaf_r0.alloc(L));
  BEM_CUDA_TRY(ctx->leaf_nr.alloc(L));
  BEM_CUDA_TRY(ctx->panel_ptr.alloc(L + 1));
  BEM_CUDA_TRY(ctx->panels.alloc(std::max<size_t>(1, pan.size())));
  BEM_CUDA_TRY(cudaMemcpyAsync(ctx->leaf_r0.p, r0.data(), L * sizeof(int), cudaMemcpyHostToDevice, st));
  BEM_CUDA_TRY(cudaMemcpyAsync(ctx->leaf_nr.p, nr.data(), L * sizeof(int), cudaMemcpyHostToDevice, st));
  BEM_CUDA_TRY(cudaMemcpyAsync(ctx->panel_ptr.p, pptr.data(), (L + 1) * sizeof(int), cudaMemcpyHostToDevice, st));
  if (!pan.empty())
    BEM_CUDA_TRY(cudaMemcpyAsync(ctx->panels.p, pan.data(), pan.size() * sizeof(Panel), cudaMemcpyHostToDevice, st));

  // admissible blocks: small ones (one warp each) and large ones (one CTA each)
  {
    std::vector<int> sm_l, lg_l;
    for (size_t b = 0; b < ctx->far_h.size(); ++b) {
      const FarBlk& fb = ctx->far_h[b];
      (far_small_class(fb) ? sm_l : lg_l).push_back((int)b);
    }
    ctx->nfar_small = (int)sm_l.size();
    ctx->nfar_large = (int)lg_l.size();
    BEM_CUDA_TRY(ctx->far_small.alloc(std::max<size_t>(1, sm_l.size())));
    BEM_CUDA_TRY(ctx->far_large.alloc(std::max<size_t>(1, lg_l.size())));
    if (!sm_l.empty())
      BEM_CUDA_TRY(cudaMemcpyAsync(ctx->far_small.p, sm_l.data(), sm_l.size() * sizeof(int), cudaMemcpyHostToDevice, st));
    if (!lg_l.empty())
      BEM_CUDA_TRY(cudaMemcpyAsync(ctx->far_large.p, lg_l.data(), lg_l.size() * sizeof(int), cudaMemcpyHostToDevice, st));
  }
  BEM_CUDA_TRY(ctx->polar.alloc(27LL * ne));
  launch_polar(ctx->ed.p, ne, ctx->polar.p, st);
  CK("polar");

  // regular pairs of every near block, sorted by (band, distance)
  {
    int nnb = (int)ctx->near_h.size();
    std::vector<long long> po(std::max(1, nnb));
    long long tot = 0;
    ctx->max_nr = 1;
    for (int b = 0; b < nnb; ++b) {
      po[b] = tot;
      tot += (long long)ctx->near_h[b].nr * ctx->near_h[b].nc;
      ctx->max_nr = std::max(ctx->max_nr, ctx->near_h[b].nr);
    }
    BEM_CUDA_TRY(ctx->poff.alloc(std::max(1, nnb)));
    BEM_CUDA_TRY(ctx->plist.alloc(std::max<long long>(1, tot)));
    BEM_CUDA_TRY(ctx->pcount.alloc(std::max(1, nnb)));
    if (nnb) BEM_CUDA_TRY(cudaMemcpyAsync(ctx->poff.p, po.data(), nnb * sizeof(long long), cudaMemcpyHostToDevice, st));
    launch_pair_sort(ctx->near_d.p, nnb, ctx->ef.p, ctx->ed.p, ctx->poff.p, ctx->plist.p, ctx->pcount.p, st);
    CK("pair_sort");
    // far right-hand side: per leaf, the column ranges of its far panels;
    // per element, its leaf
    std::vector<int> rng, rptr(L + 1, 0), eleaf(ne, 0);
    for (int l = 0; l < L; ++l) {
      rptr[l] = (int)(rng.size() / 2);
      for (int p = pptr[l]; p < pptr[l + 1]; ++p)
        if (pan[p].kind == 1) {
          const FarBlk& fb = ctx->far_h[pan[p].xoff];
          rng.push_back(fb.c0);
          rng.push_back(fb.nc);
        }
      for (int e = r0[l]; e < r0[l] + nr[l]; ++e) eleaf[e] = l;
    }
    rptr[L] = (int)(rng.size() / 2);
    BEM_CUDA_TRY(ctx->rhs_rng.alloc(std::max<size_t>(2, rng.size())));
    BEM_CUDA_TRY(ctx->rhs_rptr.alloc(L + 1));
    BEM_CUDA_TRY(ctx->elem_leaf.alloc(std::max(1, ne)));
    if (!rng.empty())
      BEM_CUDA_TRY(cudaMemcpyAsync(ctx->rhs_rng.p, rng.data(), rng.size() * sizeof(int), cudaMemcpyHostToDevice, st));
    BEM_CUDA_TRY(cudaMemcpyAsync(ctx->rhs_rptr.p, rptr.data(), (L + 1) * sizeof(int), cudaMemcpyHostToDevice, st));
    BEM_CUDA_TRY(cudaMemcpyAsync(ctx->elem_leaf.p, eleaf.data(), ne * sizeof(int), cudaMemcpyHostToDevice, st));
    // the host vectors above must outlive the copies
    BEM_CUDA_TRY(cudaStreamSynchronize(st));
  }

  // singular and near-singular pairs of the near blocks
  int nnb = (int)ctx->near_h.size();
  DevBuf<int> cnt;
  BEM_CUDA_TRY(cnt.alloc(std::max(1, nnb)));
  launch_sing_count(ctx->near_d.p, nnb, ctx->ed.p, cnt.p, st);
  CK("sing_count");
  std::vector<int> cnt_h(nnb);
  if (nnb) BEM_CUDA_TRY(cudaMemcpyAsync(cnt_h.data(), cnt.p, nnb * sizeof(int), cudaMemcpyDeviceToHost, st));
  BEM_CUDA_TRY(cudaStreamSynchronize(st));
  std::vector<int> offs(nnb + 1, 0);
  for (int b = 0; b < nnb; ++b) offs[b + 1] = offs[b] + cnt_h[b];
  ctx->nsing = offs[nnb];
  BEM_CUDA_TRY(cnt.alloc(nnb + 1));
  BEM_CUDA_TRY(cudaMemcpyAsync(cnt.p, offs.data(), (nnb + 1) * sizeof(int), cudaMemcpyHostToDevice, st));
  BEM_CUDA_TRY(ctx->sing.alloc(std::max(1, ctx->nsing)));
  launch_sing_fill(ctx->near_d.p, nnb, ctx->ed.p, cnt.p, ctx->sing.p, st);
  CK("sing_fill");
  if (ctx->nsing) {
    // self pairs first (stable), so that the half-warps of one warp mostly
    // run the same rule
    std::vector<SingPair> sp(ctx->nsing), spo;
    BEM_CUDA_TRY(cudaMemcpyAsync(sp.data(), ctx->sing.p, sp.size() * sizeof(SingPair), cudaMemcpyDeviceToHost, st));
    BEM_CUDA_TRY(cudaStreamSynchronize(st));
    spo.reserve(sp.size());
    for (const SingPair& q : sp)
      if (q.self) spo.push_back(q);
    for (const SingPair& q : sp)
      if (!q.self) spo.push_back(q);
    BEM_CUDA_TRY(cudaMemcpyAsync(ctx->sing.p, spo.data(), spo.size() * sizeof(SingPair), cudaMemcpyHostToDevice, st));
    BEM_CUDA_TRY(cudaStreamSynchronize(st));
  }
  ctx->sing_static.release();
  BEM_CUDA_TRY(cudaStreamSynchronize(st));
  ctx->have_mesh = true;
  return BEM_OK;
}

extern "C" int bem_mesh_dev(bem_ctx* ctx, const double* xyz_dev, int64_t nv, const int32_t* tri_dev, int64_t ne,
                            const int8_t* bc_dev, const bem_opts* opts) {
  if (!ctx) return BEM_ERR_INVALID_ARG;
  if (!xyz_dev || !tri_dev || !bc_dev || nv < 3 || ne < 1 || ne > (1LL << 28))
    return fail(ctx, BEM_ERR_INVALID_ARG, "bem_mesh: bad sizes or null pointers");
  TRY(set_device(ctx));
  return mesh_impl(ctx, xyz_dev, nv, tri_dev, (int)ne, (const signed char*)bc_dev, opts);
}

extern "C" int bem_mesh(bem_ctx* ctx, const double* xyz, int64_t nv, const int32_t* tri, int64_t ne,
                        const int8_t* bc, const bem_opts* opts) {
  if (!ctx) return BEM_ERR_INVALID_ARG;
  if (!xyz || !tri || !bc || nv < 3 || ne < 1 || ne > (1LL << 28))
    return fail(ctx, BEM_ERR_INVALID_ARG, "bem_mesh: bad sizes or null pointers");
  for (int64_t e = 0; e < ne; ++e)
    if (bc[e] != BEM_BC_TRACTION && bc[e] != BEM_BC_DISPLACEMENT)
      return fail(ctx, BEM_ERR_INVALID_ARG, "bem_mesh: bc_type must be 0 or 1");
  TRY(set_device(ctx));
  DevBuf<double> x;
  DevBuf<int> t;
  DevBuf<signed char> b;
  BEM_CUDA_TRY(x.alloc(3 * nv));
  BEM_CUDA_TRY(t.alloc(3 * ne));
  BEM_CUDA_TRY(b.alloc(ne));
  BEM_CUDA_TRY(cudaMemcpyAsync(x.p, xyz, 3 * nv * sizeof(double), cudaMemcpyHostToDevice, ctx->stream));
  BEM_CUDA_TRY(cudaMemcpyAsync(t.p, tri, 3 * ne * sizeof(int), cudaMemcpyHostToDevice, ctx->stream));
  BEM_CUDA_TRY(cudaMemcpyAsync(b.p, bc, ne, cudaMemcpyHostToDevice, ctx->stream));
  int r = mesh_impl(ctx, x.p, nv, t.p, (int)ne, b.p, opts);
  cudaStreamSynchronize(ctx->stream);
  return r;
}

// ---------------------------------------------------------------------------
// assembly
// ---------------------------------------------------------------------------
namespace {

// Static parts, at the precision the operator needs: FP32 near-singular
// rule for the complex64 operator, FP64 for complex128 (an FP64 set serves
// both; an FP32 set is recomputed when the FP64 operator is assembled).
int ensure_static(bem_ctx* ctx, bool need_fp64) {
  if (ctx->nsing == 0) return BEM_OK;
  if (ctx->sing_static.p && (ctx->static_fp64 || !need_fp64)) return BEM_OK;
  if (!ctx->sing_static.p) BEM_CUDA_TRY(ctx->sing_static.alloc(18LL * ctx->nsing));
  KParams<double> P = make_params<double>(ctx, 0.0, 0.0);
  launch_static(ctx->sing.p, ctx->nsing, ctx->ed.p, P, ctx->sing_static.p, !need_fp64, ctx->stream);
  CK("static");
  ctx->static_fp64 = need_fp64;
  return BEM_OK;
}

int check_ready(bem_ctx* ctx) {
  if (!ctx->have_mesh) return fail(ctx, BEM_ERR_NO_MESH, "no mesh");
  if (!ctx->have_mat) return fail(ctx, BEM_ERR_STATE, "material not set");
  return BEM_OK;
}

// Far-field blocks at the current s: reuse of the previous assembly's pivots
// where available, then ACA steps for every block not yet converged, batch by
// batch. Full storage: ACA writes the factors in place (U, V). Compact
// storage: ACA writes each batch into the workspace halves ws, ws + ws_entries
// and the batch is packed into the pools U, V (capU, capV entries).
template <typename R, typename Op>
int run_aca(bem_ctx* ctx, const KParams<R>& P, Op* U, Op* V, long long capU, long long capV, Op* ws,
            const bem_opts& o, bool count, cudaStream_t st) {
  const size_t nf = ctx->far_h.size();
  BEM_CUDA_TRY(ctx->piv_i.ensure(std::max(1, ctx->t_entries)));
  BEM_CUDA_TRY(ctx->piv_j.ensure(std::max(1, ctx->t_entries)));
  BEM_CUDA_TRY(ctx->aca_kstart.ensure(std::max<size_t>(1, nf)));
  BEM_CUDA_TRY(ctx->aca_done.ensure(std::max<size_t>(1, nf)));
  BEM_CUDA_TRY(ctx->aca_norm0.ensure(std::max<size_t>(1, nf)));
  BEM_CUDA_TRY(ctx->aca_npiv.ensure(std::max<size_t>(1, nf)));
  AcaState S{nullptr, nullptr, nullptr, ctx->piv_i.p, ctx->piv_j.p, ctx->aca_npiv.p};
  const bool warm = ctx->aca_reuse && ctx->aca_warm_ok && nf > 0;
  ctx->aca_last_warm = warm;
  if (warm) {
    S.kstart = ctx->aca_kstart.p;
    S.norm0 = ctx->aca_norm0.p;
    S.done = ctx->aca_done.p;
  }
  const bool compact = ctx->far_compact;
  unsigned long long* cursor = reinterpret_cast<unsigned long long*>(ctx->fbase.p + 2 * nf);
  if (compact && nf) BEM_CUDA_TRY(cudaMemsetAsync(cursor, 0, 2 * sizeof(unsigned long long), st));
  Op* Uw = compact ? ws : U;
  Op* Vw = compact ? ws + ctx->ws_entries : V;
  for (const FarBatch& fb : ctx->far_batches) {
    const int nb = fb.b1 - fb.b0;
    if (warm)
      BEM_CUDA_TRY((launch_aca_warm<R, Op>(ctx->far_d.p, fb.b0, nb, ctx->ef.p, ctx->ed.p, ctx->bc.p, P, Uw, Vw,
                                           ctx->rank.p, ctx->aca_npiv.p, ctx->piv_i.p, ctx->piv_j.p,
                                           ctx->aca_kstart.p, ctx->aca_norm0.p, ctx->aca_done.p, o.aca_tol,
                                           ctx->aca_tau, st)));
    launch_aca<R, Op>(ctx->far_d.p, ctx->far_small.p + fb.s0, fb.s1 - fb.s0, ctx->far_large.p + fb.l0,
                      fb.l1 - fb.l0, ctx->ef.p, ctx->ed.p, ctx->bc.p, P, Uw, Vw, ctx->rank.p, ctx->aca_fail.p,
                      o.aca_tol, S, st);
    CK("aca");
    if (compact) {
      launch_far_pack<Op>(ctx->far_d.p, fb.b0, nb, ctx->rank.p, Uw, Vw, U, V, capU, capV, ctx->fbase.p, cursor, st);
      CK("far pack");
    }
  }
  if (count && ctx->profiling && nf) {
    ctx->prof_aca_blocks += (long long)nf;
    if (warm) {
      count_if(true);
      k_count_zero<<<std::min<int>(64, ((int)nf + 255) / 256), 256, 0, st>>>(ctx->aca_done.p, (int)nf,
                                                                              ctx->prof_dev.p);
      CK("count stepped");
    } else {
      ctx->prof_aca_continued += (long long)nf;
    }
  }
  ctx->aca_warm_ok = true;
  return BEM_OK;
}

constexpr int FAR_CUR_SLOT = 4088;  // pinned host slots (two int64) of the pool cursors

// Compact storage: initial pool capacity (entries) of a factor whose capped
// size is cap; the pools grow by a quarter over the need on overflow.
static long long pool_initial(long long init) { return std::max(1LL, init); }

// Far field of one assembly in the precision Op, on the auxiliary stream:
// storage, pivot-state snapshot (compact storage), ACA.
template <typename R, typename Op>
int far_field_begin(bem_ctx* ctx, const KParams<R>& P, DevBuf<Op>& U, DevBuf<Op>& V, DevBuf<Op>& ws,
                    const bem_opts& o, cudaStream_t aux, cudaStream_t st) {
  const size_t nf = ctx->far_h.size();
  if (!ctx->far_compact) {
    BEM_CUDA_TRY(U.ensure(std::max<long long>(1, ctx->u_entries)));
    BEM_CUDA_TRY(V.ensure(std::max<long long>(1, ctx->v_entries)));
  } else {
    if (U.n == 0) BEM_CUDA_TRY(U.alloc(pool_initial(ctx->u_init)));
    if (V.n == 0) BEM_CUDA_TRY(V.alloc(pool_initial(ctx->v_init)));
    BEM_CUDA_TRY(ws.ensure(std::max<long long>(2, 2 * ctx->ws_entries)));
    // the pivot state this assembly starts from, kept for a redo
    ctx->far_was_ok = ctx->aca_warm_ok;
    const long long nt = std::max(1, ctx->t_entries);
    if (ctx->far_was_ok && nf) {
      BEM_CUDA_TRY(ctx->piv_snap.ensure(2 * nt + (long long)nf));
      BEM_CUDA_TRY(cudaMemcpyAsync(ctx->piv_snap.p, ctx->piv_i.p, nt * sizeof(int), cudaMemcpyDeviceToDevice, st));
      BEM_CUDA_TRY(
          cudaMemcpyAsync(ctx->piv_snap.p + nt, ctx->piv_j.p, nt * sizeof(int), cudaMemcpyDeviceToDevice, st));
      BEM_CUDA_TRY(cudaMemcpyAsync(ctx->piv_snap.p + 2 * nt, ctx->aca_npiv.p, nf * sizeof(int),
                                   cudaMemcpyDeviceToDevice, st));
    }
  }
  BEM_CUDA_TRY(cudaEventRecord(ctx->ev_fork, st));
  BEM_CUDA_TRY(cudaStreamWaitEvent(aux, ctx->ev_fork, 0));
  TRY((run_aca<R, Op>(ctx, P, U.p, V.p, (long long)U.n, (long long)V.n, ws.p, o, true, aux)));
  BEM_CUDA_TRY(cudaEventRecord(ctx->ev_join, aux));
  return BEM_OK;
}

template <typename R, typename Op>
int far_field_redo_if_needed(bem_ctx* ctx, const KParams<R>& P, DevBuf<Op>& U, DevBuf<Op>& V, DevBuf<Op>& ws,
                             const bem_opts& o, cudaStream_t st);

// Joins the far field into st. Compact storage: reads the pools' need; on an
// overflow the pools grow to the need plus a quarter and the far field is
// redone on st from the pivot state it started from (the same factors).
template <typename R, typename Op>
int far_field_finish(bem_ctx* ctx, const KParams<R>& P, DevBuf<Op>& U, DevBuf<Op>& V, DevBuf<Op>& ws,
                     const bem_opts& o, cudaStream_t st) {
  const size_t nf = ctx->far_h.size();
  BEM_CUDA_TRY(cudaStreamWaitEvent(st, ctx->ev_join, 0));
  if (!ctx->far_compact || !nf) return BEM_OK;
  long long* hc = reinterpret_cast<long long*>(ctx->host_red + FAR_CUR_SLOT);
  BEM_CUDA_TRY(cudaMemcpyAsync(hc, ctx->fbase.p + 2 * nf, 2 * sizeof(long long), cudaMemcpyDeviceToHost, st));
  if (ctx->far_defer) {
    // checked by far_field_verify when this operator set comes into use
    BEM_CUDA_TRY(cudaEventRecord(ctx->ev_far_cursor, st));
    ctx->far_verify_pending = true;
    ctx->far_pending_s[0] = P.s.re;
    ctx->far_pending_s[1] = P.s.im;
    return BEM_OK;
  }
  BEM_CUDA_TRY(cudaStreamSynchronize(st));
  return far_field_redo_if_needed<R, Op>(ctx, P, U, V, ws, o, st);
}

// Compact storage: if the last assembly's need exceeded the pools, grow them
// to the need plus a quarter and redo the far field on st from the pivot
// state it started from (the same factors). The need is in the pinned slot.
template <typename R, typename Op>
int far_field_redo_if_needed(bem_ctx* ctx, const KParams<R>& P, DevBuf<Op>& U, DevBuf<Op>& V, DevBuf<Op>& ws,
                             const bem_opts& o, cudaStream_t st) {
  const size_t nf = ctx->far_h.size();
  long long* hc = reinterpret_cast<long long*>(ctx->host_red + FAR_CUR_SLOT);
  if (hc[0] <= (long long)U.n && hc[1] <= (long long)V.n) return BEM_OK;
  ctx->far_regrows += 1;
  const long long nu = std::min(ctx->u_entries, hc[0] + hc[0] / 4 + 1);
  const long long nv = std::min(ctx->v_entries, hc[1] + hc[1] / 4 + 1);
  if (hc[0] > (long long)U.n) BEM_CUDA_TRY(U.alloc(std::max<long long>(nu, U.n)));
  if (hc[1] > (long long)V.n) BEM_CUDA_TRY(V.alloc(std::max<long long>(nv, V.n)));
  const long long nt = std::max(1, ctx->t_entries);
  if (ctx->far_was_ok) {
    BEM_CUDA_TRY(cudaMemcpyAsync(ctx->piv_i.p, ctx->piv_snap.p, nt * sizeof(int), cudaMemcpyDeviceToDevice, st));
    BEM_CUDA_TRY(cudaMemcpyAsync(ctx->piv_j.p, ctx->piv_snap.p + nt, nt * sizeof(int), cudaMemcpyDeviceToDevice, st));
    BEM_CUDA_TRY(cudaMemcpyAsync(ctx->aca_npiv.p, ctx->piv_snap.p + 2 * nt, nf * sizeof(int),
                                 cudaMemcpyDeviceToDevice, st));
  }
  ctx->aca_warm_ok = ctx->far_was_ok;
  BEM_CUDA_TRY(cudaMemsetAsync(ctx->aca_fail.p, 0, sizeof(int), st));
  TRY((run_aca<R, Op>(ctx, P, U.p, V.p, (long long)U.n, (long long)V.n, ws.p, o, false, st)));
  BEM_CUDA_TRY(cudaMemcpyAsync(hc, ctx->fbase.p + 2 * nf, 2 * sizeof(long long), cudaMemcpyDeviceToHost, st));
  BEM_CUDA_TRY(cudaStreamSynchronize(st));
  if (hc[0] > (long long)U.n || hc[1] > (long long)V.n)
    return fail(ctx, BEM_ERR_STATE, "far-field pools overflowed after regrowth");
  return BEM_OK;
}

// Operator at s: right-hand side contributions optional (pattern/b may be null).
int assemble_impl(bem_ctx* ctx, double sre, double sim, const bem_opts& o, const double* pattern_tree,
                  c128 pk, c128* b, cudaStream_t st) {
  TRY(ensure_static(ctx, o.precision == BEM_PREC_C128));
  ctx->prec = o.precision;
  cudaEvent_t ev = prof_begin(ctx, st);
  size_t nf = ctx->far_h.size();
  BEM_CUDA_TRY(ctx->rank.ensure(std::max<size_t>(1, nf)));
  BEM_CUDA_TRY(ctx->aca_fail.ensure(1));
  BEM_CUDA_TRY(ctx->prec_inv.ensure(9LL * ctx->ne));
  BEM_CUDA_TRY(cudaMemsetAsync(ctx->aca_fail.p, 0, sizeof(int), st));
  KParams<double> Pd = make_params<double>(ctx, sre, sim);
  BEM_CUDA_TRY(ctx->status.ensure(1));
  DevBuf<int>& status = ctx->status;
  // The far field (ACA, latency-bound in its continuation steps) runs on the
  // auxiliary stream while the right-hand side, the singular pairs and the
  // near field run on the caller's stream; they write disjoint storage and
  // join before the assembly ends.
  const bool mixed = is_mixed(ctx);
  // leaf-block inverses: asked for, or a sweep's AUTO choice still open or made for them
  const bool want_leaf = ctx->nleaf_pre > 0 && (o.precond == BEM_PRECOND_LEAF ||
                                                (o.precond == BEM_PRECOND_AUTO && ctx->pre_auto != 1));
  KParams<float> Pf = make_params<float>(ctx, sre, sim);
  if (mixed) {
    if (ctx->near32.n < (size_t)std::max<long long>(1, ctx->near_entries)) ctx->near_zero_pending = true;
    BEM_CUDA_TRY(ctx->near32.ensure(std::max<long long>(1, ctx->near_entries)));
    BEM_CUDA_TRY(ctx->t32.ensure(4LL * std::max(1, ctx->t_entries)));
    BEM_CUDA_TRY(ctx->prec_inv32.ensure(9LL * ctx->ne));
  } else {
    if (ctx->near64.n < (size_t)std::max<long long>(1, ctx->near_entries)) ctx->near_zero_pending = true;
    BEM_CUDA_TRY(ctx->near64.ensure(std::max<long long>(1, ctx->near_entries)));
  }
  BEM_CUDA_TRY(ctx->t64.ensure(4LL * std::max(1, ctx->t_entries)));
  if (ctx->fbase.n < 2 * nf + 2) {
    BEM_CUDA_TRY(ctx->fbase.alloc(2 * nf + 2));
    ctx->fbase_ready = false;
  }
  if (!ctx->far_compact && !ctx->fbase_ready) {
    launch_fbase_full(ctx->far_d.p, (int)nf, ctx->fbase.p, st);
    CK("factor offsets");
    ctx->fbase_ready = true;
  }
  cudaStream_t aux = ctx->aux_stream;
  if (mixed) TRY((far_field_begin<float, c64>(ctx, Pf, ctx->u32, ctx->v32, ctx->ws32, o, aux, st)));
  else TRY((far_field_begin<double, c128>(ctx, Pd, ctx->u64, ctx->v64, ctx->ws64, o, aux, st)));
  if (b) {
    BEM_CUDA_TRY(cudaMemsetAsync(b, 0, ctx->N * sizeof(c128), st));
    if (mixed)
      launch_rhs_far<float>(ctx->rhs_rng.p, ctx->rhs_rptr.p, ctx->elem_leaf.p, ctx->ne, ctx->ef.p, ctx->ed.p, ctx->bc.p,
                            ctx->patf.p, ctx->pattern.p, Pf, pk, b, st);
    else
      launch_rhs_far<double>(ctx->rhs_rng.p, ctx->rhs_rptr.p, ctx->elem_leaf.p, ctx->ne, ctx->ef.p, ctx->ed.p, ctx->bc.p,
                             ctx->patf.p, ctx->pattern.p, Pd, pk, b, st);
    CK("rhs_far");
  }
  if (mixed) {
    if (ctx->near_zero_pending) {
      BEM_CUDA_TRY(cudaMemsetAsync(ctx->near32.p, 0, ctx->near32.n * sizeof(c64), st));
      ctx->near_zero_pending = false;
    }
    launch_sing<float, c64>(ctx->sing.p, ctx->nsing, ctx->ed.p, ctx->polar.p, ctx->bc.p, ctx->sing_static.p, Pf,
                            ctx->near32.p, ctx->prec_inv.p, pattern_tree, pk, b, status.p, st);
    CK("sing");
    launch_near_regular<float, c64>(ctx->near_d.p, (int)ctx->near_h.size(), ctx->max_nr, ctx->plist.p, ctx->poff.p,
                                    ctx->pcount.p, ctx->ef.p, ctx->ed.p, ctx->bc.p, Pf, ctx->near32.p,
                                    b ? ctx->patf.p : nullptr, b ? ctx->pattern.p : nullptr, pk, b, st);
    CK("near_regular");
    if (want_leaf) {
      BEM_CUDA_TRY(ctx->minv32.ensure(std::max<long long>(1, ctx->leaf_pre_entries)));
      BEM_CUDA_TRY(launch_leaf_inverse<float>(ctx->leaf_pre.p, ctx->nleaf_pre, ctx->near32.p, ctx->prec_inv.p,
                                              ctx->minv32.p, st));
    }
    long long n9 = 9LL * ctx->ne;
    count_if(true);
    k_pinv_cast<<<(unsigned)((n9 + 255) / 256), 256, 0, st>>>(ctx->prec_inv.p, ctx->prec_inv32.p, n9);
    CK("pinv_cast");
  } else {
    if (ctx->near_zero_pending) {
      BEM_CUDA_TRY(cudaMemsetAsync(ctx->near64.p, 0, ctx->near64.n * sizeof(c128), st));
      ctx->near_zero_pending = false;
    }
    launch_sing<double, c128>(ctx->sing.p, ctx->nsing, ctx->ed.p, ctx->polar.p, ctx->bc.p, ctx->sing_static.p, Pd,
                              ctx->near64.p, ctx->prec_inv.p, pattern_tree, pk, b, status.p, st);
    CK("sing");
    launch_near_regular<double, c128>(ctx->near_d.p, (int)ctx->near_h.size(), ctx->max_nr, ctx->plist.p,
                                      ctx->poff.p, ctx->pcount.p, ctx->ef.p, ctx->ed.p, ctx->bc.p, Pd, ctx->near64.p,
                                      b ? ctx->patf.p : nullptr, b ? ctx->pattern.p : nullptr, pk, b, st);
    CK("near_regular");
    if (want_leaf) {
      BEM_CUDA_TRY(ctx->minv64.ensure(std::max<long long>(1, ctx->leaf_pre_entries)));
      BEM_CUDA_TRY(launch_leaf_inverse<double>(ctx->leaf_pre.p, ctx->nleaf_pre, ctx->near64.p, ctx->prec_inv.p,
                                               ctx->minv64.p, st));
    }
  }
  ctx->minv_ready = want_leaf;
  if (mixed) TRY((far_field_finish<float, c64>(ctx, Pf, ctx->u32, ctx->v32, ctx->ws32, o, st)));
  else TRY((far_field_finish<double, c128>(ctx, Pd, ctx->u64, ctx->v64, ctx->ws64, o, st)));
  prof_end(ctx, ev, 1, 0.0, 0.0, st);
  ctx->assembled = true;
  ctx->s_re = sre;
  ctx->s_im = sim;
  if (ctx->profiling) {
    // low-rank entries in use after this assembly, counted on the device
    ctx->prof_slot = std::min(ctx->prof_nslots + 1, PROF_SLOTS - 1);
    ctx->prof_nslots = ctx->prof_slot;
    BEM_CUDA_TRY(cudaMemsetAsync(ctx->prof_dev.p + ctx->prof_slot, 0, sizeof(long long), st));
    if (nf) {
      count_if(true);
      k_lowrank_entries<<<std::min<int>(64, ((int)nf + 255) / 256), 256, 0, st>>>(ctx->rank.p, ctx->far_d.p, (int)nf,
                                                                                  ctx->prof_dev.p + ctx->prof_slot);
      CK("count low-rank entries");
    }
    prof_harvest(ctx);
  }
  return BEM_OK;
}

// Compact storage in a pipelined sweep: the deferred check of the assembly
// whose operator set has just come into use (after its event), and a redo on
// the context's stream when it overflowed the pools.
int far_field_verify(bem_ctx* ctx, const bem_opts& o) {
  if (!ctx->far_verify_pending) return BEM_OK;
  ctx->far_verify_pending = false;
  BEM_CUDA_TRY(cudaEventSynchronize(ctx->ev_far_cursor));
  const double sre = ctx->far_pending_s[0], sim = ctx->far_pending_s[1];
  if (is_mixed(ctx))
    TRY((far_field_redo_if_needed<float, c64>(ctx, make_params<float>(ctx, sre, sim), ctx->u32, ctx->v32, ctx->ws32,
                                              o, ctx->stream)));
  else
    TRY((far_field_redo_if_needed<double, c128>(ctx, make_params<double>(ctx, sre, sim), ctx->u64, ctx->v64,
                                                ctx->ws64, o, ctx->stream)));
  return BEM_OK;
}

// y = A x with FP64 accumulation (x, y c128, nrhs vectors)
int apply64(bem_ctx* ctx, const c128* x, c128* y, int nrhs) {
  cudaEvent_t ev = prof_begin(ctx);
  if (is_mixed(ctx))
    launch_hmatvec<c64, c128, c128, double>(ctx, ctx->near32.p, ctx->u32.p, ctx->v32.p,
                                            reinterpret_cast<cplx<double>*>(ctx->t64.p), x, y, nrhs, ctx->stream);
  else
    launch_hmatvec<c128, c128, c128, double>(ctx, ctx->near64.p, ctx->u64.p, ctx->v64.p,
                                             reinterpret_cast<cplx<double>*>(ctx->t64.p), x, y, nrhs, ctx->stream);
  CK("hmatvec64");
  prof_end_hmv(ctx, ev, is_mixed(ctx) ? 8 : 16, 16, 16, nrhs);
  return BEM_OK;
}

__global__ void k_pattern_f32(const double* __restrict__ p, float* __restrict__ q, long long n) {
  long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (i < n) q[i] = (float)p[i];
}

// y = A x for the mixed-precision operator with FP32 products: x rounded to
// c64, FP32 sums within each task of the product, FP64 sums across tasks.
// Relative accuracy ~1e-6 of |A||x|: used for true residuals when the
// tolerance is >= 1e-6 and for the extrapolation products.
int apply_fast(bem_ctx* ctx, const c128* x, c128* y, int nrhs) {
  if (!is_mixed(ctx)) return apply64(ctx, x, y, nrhs);
  BEM_CUDA_TRY(ctx->w32.ensure((size_t)nrhs * ctx->N));
  launch_copy_cast(x, ctx->w32.p, nrhs * ctx->N, 1.0, ctx->stream);
  cudaEvent_t ev = prof_begin(ctx);
  launch_hmatvec<c64, c64, c128, float>(ctx, ctx->near32.p, ctx->u32.p, ctx->v32.p,
                                        reinterpret_cast<cplx<float>*>(ctx->t32.p), ctx->w32.p, y, nrhs, ctx->stream);
  CK("hmatvec_fast");
  prof_end_hmv(ctx, ev, 8, 8, 16, nrhs);
  return BEM_OK;
}

int prepare_loaded(bem_ctx* ctx, const double* pattern_tree) {
  BEM_CUDA_TRY(ctx->patf.ensure(3LL * ctx->ne));
  count_if(true);
  k_pattern_f32<<<(unsigned)((3LL * ctx->ne + 255) / 256), 256, 0, ctx->stream>>>(pattern_tree, ctx->patf.p,
                                                                                 3LL * ctx->ne);
  CK("pattern_f32");
  BEM_CUDA_TRY(ctx->loaded.ensure(ctx->ne + 1));
  count_if(true);
  k_loaded<<<1, 1024, 0, ctx->stream>>>(pattern_tree, ctx->ne, ctx->loaded.p, ctx->loaded.p + ctx->ne);
  CK("loaded");
  BEM_CUDA_TRY(cudaMemcpyAsync(&ctx->nloaded, ctx->loaded.p + ctx->ne, sizeof(int), cudaMemcpyDeviceToHost,
                               ctx->stream));
  BEM_CUDA_TRY(cudaStreamSynchronize(ctx->stream));
  return BEM_OK;
}

// pattern in caller order on device -> ctx->pattern in tree order + loaded list
int set_pattern_dev(bem_ctx* ctx, const double* pat_dev) {
  BEM_CUDA_TRY(ctx->pattern.ensure(3LL * ctx->ne));
  count_if(true);
  k_permute_pattern<<<(ctx->ne + 127) / 128, 128, 0, ctx->stream>>>(pat_dev, ctx->perm.p, ctx->ne, ctx->pattern.p);
  CK("permute_pattern");
  return prepare_loaded(ctx, ctx->pattern.p);
}

int set_pattern_host(bem_ctx* ctx, const double* pat) {
  std::vector<double> pt(3LL * ctx->ne);
  for (int k = 0; k < ctx->ne; ++k)
    for (int a = 0; a < 3; ++a) pt[3LL * k + a] = pat[3LL * ctx->tree.perm[k] + a];
  BEM_CUDA_TRY(ctx->pattern.ensure(3LL * ctx->ne));
  BEM_CUDA_TRY(cudaMemcpyAsync(ctx->pattern.p, pt.data(), pt.size() * sizeof(double), cudaMemcpyHostToDevice,
                               ctx->stream));
  return prepare_loaded(ctx, ctx->pattern.p);
}

// host vector (caller order, interleaved complex) <-> device tree order
void to_tree(const bem_ctx* ctx, const double* in, std::vector<c128>& out) {
  out.resize(ctx->N);
  for (int k = 0; k < ctx->ne; ++k) {
    long long e = ctx->tree.perm[k];
    for (int a = 0; a < 3; ++a) out[3LL * k + a] = c128{in[2 * (3 * e + a)], in[2 * (3 * e + a) + 1]};
  }
}
void from_tree(const bem_ctx* ctx, const std::vector<c128>& in, double* out) {
  for (int k = 0; k < ctx->ne; ++k) {
    long long e = ctx->tree.perm[k];
    for (int a = 0; a < 3; ++a) {
      out[2 * (3 * e + a)] = in[3LL * k + a].re;
      out[2 * (3 * e + a) + 1] = in[3LL * k + a].im;
    }
  }
}

template <typename Vb> DevBuf<Vb>& basis_buf(bem_ctx* ctx);
template <> DevBuf<c64>& basis_buf<c64>(bem_ctx* ctx) { return ctx->V32; }
template <> DevBuf<c128>& basis_buf<c128>(bem_ctx* ctx) { return ctx->V64; }
template <typename Pm> const Pm* basis_pinv(bem_ctx* ctx);
template <> const c64* basis_pinv<c64>(bem_ctx* ctx) { return ctx->prec_inv32.p; }
template <> const c128* basis_pinv<c128>(bem_ctx* ctx) { return ctx->prec_inv.p; }

// Pinned host slots for ncomplex values and nev timing-free events.
int ensure_col_events(bem_ctx* ctx, int nev) {
  while ((int)ctx->col_events.size() < nev) {
    cudaEvent_t e;
    BEM_CUDA_TRY(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
    ctx->col_events.push_back(e);
  }
  return BEM_OK;
}

// ---------------------------------------------------------------------------
// GMRES (Sec. 5): right preconditioning (3 x 3 or leaf blocks); each restart
// cycle starts from the true residual r = b - A x accumulated in FP64 (x in
// FP64), so restarts double as iterative refinement of the c64 Krylov solve.
//
// The solve is driven by the device (GmCtl): the host enqueues
//   init    ||b|| and the counters;
//   test    r = b - A x and ||r||: the solve ends (tolerance met, or the step
//           limit reached) or a cycle starts from V_0 = r / ||r||;
//   step j  z = M^-1 V_j, w = A z, the orthogonalisation (V_{j+1}, column j
//           of H) and the step's Givens rotation and residual estimate, which
//           end the cycle at the inner target, after m steps, on breakdown or
//           at the step limit;
//   update  x += M^-1 V R^-1 g, when a cycle has ended;
// and waits on none of them. Step kernels do nothing outside a cycle, so the
// host enqueues steps before it knows whether the cycle still runs: it reads
// the state's mapped host copy GM_LAG steps behind the newest step it has
// enqueued (the GPU has that many steps queued meanwhile), stops enqueueing
// steps once the cycle has ended, then enqueues the update and the next test.
// The steps enqueued past the end of a cycle or of the solve return at once.
// ---------------------------------------------------------------------------
constexpr int GM_LAG = 1;

template <typename Vb, typename Pm, typename Acc>
int gmres_impl(bem_ctx* ctx, const c128* b, c128* x, const bem_opts& o, bem_freq_stats* stats) {
  cudaStream_t st = ctx->stream;
  const long long N = ctx->N;
  const int m = std::max(1, o.restart);
  if (m + 1 > 512) return fail(ctx, BEM_ERR_INVALID_ARG, "restart length above 511");
  constexpr bool mixed = sizeof(Vb) == sizeof(c64);
  DevBuf<Vb>& Vbuf = basis_buf<Vb>(ctx);
  BEM_CUDA_TRY(Vbuf.ensure((m + 1) * N));
  Vb* V = Vbuf.p;
  Vb *wv, *zv;
  if constexpr (mixed) {
    BEM_CUDA_TRY(ctx->gm_w32.ensure(N));
    BEM_CUDA_TRY(ctx->gm_z32.ensure(N));
    wv = reinterpret_cast<Vb*>(ctx->gm_w32.p);
    zv = reinterpret_cast<Vb*>(ctx->gm_z32.p);
  } else {
    BEM_CUDA_TRY(ctx->gm_w64.ensure(N));
    BEM_CUDA_TRY(ctx->gm_z64.ensure(N));
    wv = reinterpret_cast<Vb*>(ctx->gm_w64.p);
    zv = reinterpret_cast<Vb*>(ctx->gm_z64.p);
  }
  BEM_CUDA_TRY(ctx->r64.ensure(N));
  BEM_CUDA_TRY(ctx->y64.ensure(N));
  BEM_CUDA_TRY(ctx->tmp64.ensure(2 * N));
  // reduction scratch: [dot partials (64) | Hessenberg column slots | ||b||^2, ||r||^2]
  const long long slot_len = 2LL * (m + 1) + 1;
  BEM_CUDA_TRY(ctx->red.ensure(2 * (64 + slot_len * (m + 1) + 2)));
  c128* part = reinterpret_cast<c128*>(ctx->red.p);
  c128* hdev = part + 64;
  c128* bb_dev = hdev + slot_len * (m + 1);
  c128* rr_dev = bb_dev + 1;
  BEM_CUDA_TRY(ctx->orth_part.ensure((size_t)(2 * (m + 1) + 2) * arnoldi_orth_max_blocks()));
  BEM_CUDA_TRY(ctx->gm_ctl.ensure(1));
  BEM_CUDA_TRY(ctx->gm_work.ensure((size_t)(m + 1) * m + 3 * (size_t)m + 1));
  TRY(ensure_col_events(ctx, m + 1));
  GmDev d{};
  d.ctl = ctx->gm_ctl.p;
  d.mirror = ctx->gm_mirror_dev;
  d.R = ctx->gm_work.p;
  d.g = d.R + (long long)(m + 1) * m;
  d.cs = d.g + (m + 1);
  d.sn = d.cs + m;
  d.hcol = hdev;
  d.slot_len = slot_len;
  d.m = m;
  d.max_iters = o.max_iters;
  d.tol = o.tol;
  d.floor = mixed ? 2e-6 : 1e-13;
  const int* act = &d.ctl->active;
  const int* jcur = &d.ctl->j;
  const int* upd = &d.ctl->update;
  const Pm* pinv = basis_pinv<Pm>(ctx);
  const bool leaf = ctx->use_leaf_pre && ctx->minv_ready;
  // true residuals: FP64 sums of FP32 products (tolerances >= 1e-6) or of
  // FP64 products. With FP32 products the residual carries an error of about
  // 1e-7 sqrt(columns per task) |A| |x| (~1.5e-6 |A||x| here), an order below
  // the tolerances it decides; FP64 products are bound by GB300's FP64 pipe
  // (1/64 of the FP32 rate), not by the bandwidth the FP32 product reaches.
  const bool exact = !(mixed && o.tol >= 1e-6);
  // timed products of the steps, kept until the cycles' step counts are known
  struct StepProf {
    cudaEvent_t a, b;
    int cycle, j;
  };
  std::vector<StepProf> sprof;
  int cyc = 0;  // cycles the host has enqueued steps for

  auto step = [&](int q) -> int {
    if (leaf) {
      if constexpr (mixed)
        launch_leaf_apply<c64, c64, c64>(ctx->leaf_pre.p, ctx->nleaf_pre, ctx->minv32.p,
                                         reinterpret_cast<const c64*>(V), reinterpret_cast<c64*>(zv), st, act,
                                         jcur, N);
      else
        launch_leaf_apply<c128, c128, c128>(ctx->leaf_pre.p, ctx->nleaf_pre, ctx->minv64.p,
                                            reinterpret_cast<const c128*>(V), reinterpret_cast<c128*>(zv), st,
                                            act, jcur, N);
    } else {
      launch_precond<Pm, Vb, Vb>(pinv, V, zv, ctx->ne, st, act, jcur, N);
    }
    cudaEvent_t ev = prof_begin(ctx);
    if constexpr (mixed)
      launch_hmatvec<c64, c64, c64, float>(ctx, ctx->near32.p, ctx->u32.p, ctx->v32.p,
                                           reinterpret_cast<cplx<float>*>(ctx->t32.p),
                                           reinterpret_cast<const c64*>(zv), reinterpret_cast<c64*>(wv), 1, st,
                                           act);
    else
      launch_hmatvec<c128, c128, c128, double>(ctx, ctx->near64.p, ctx->u64.p, ctx->v64.p,
                                               reinterpret_cast<cplx<double>*>(ctx->t64.p),
                                               reinterpret_cast<const c128*>(zv), reinterpret_cast<c128*>(wv), 1,
                                               st, act);
    CK("arnoldi matvec");
    if (ev) {
      cudaEvent_t e2 = take_event(ctx);
      cudaEventRecord(e2, st);
      sprof.push_back({ev, e2, cyc, q});
    }
    {
      CoopLane lane(ctx, st);
      BEM_CUDA_TRY(lane.status());
      BEM_CUDA_TRY(launch_arnoldi_orth<Vb>(V, N, 0, wv, N, ctx->orth_part.p, hdev, m, lane.stream(), &d));
      BEM_CUDA_TRY(lane.join());
    }
    CK("arnoldi");
    BEM_CUDA_TRY(cudaEventRecord(ctx->col_events[q], st));
    return BEM_OK;
  };
  auto test = [&]() -> int {
    if (exact) TRY(apply64(ctx, x, ctx->y64.p, 1));
    else TRY(apply_fast(ctx, x, ctx->y64.p, 1));
    launch_residual(b, ctx->y64.p, ctx->r64.p, N, st);
    const int nblk = launch_dots<c128, c128>(ctx->r64.p, N, 1, ctx->r64.p, N, part, st);
    launch_dots_final(part, nblk, 1, rr_dev, st);
    launch_gm_begin<Vb>(d, rr_dev, ctx->r64.p, V, x, N, st);
    CK("residual test");
    return BEM_OK;
  };
  auto update = [&]() -> int {
    launch_gm_combine<Vb>(V, N, d, ctx->tmp64.p, N, st);
    if (leaf && mixed)
      launch_leaf_apply<c64, c128, c128>(ctx->leaf_pre.p, ctx->nleaf_pre, ctx->minv32.p, ctx->tmp64.p,
                                         ctx->tmp64.p + N, st, upd);
    else if (leaf)
      launch_leaf_apply<c128, c128, c128>(ctx->leaf_pre.p, ctx->nleaf_pre, ctx->minv64.p, ctx->tmp64.p,
                                          ctx->tmp64.p + N, st, upd);
    else
      launch_precond<c128, c128, c128>(ctx->prec_inv.p, ctx->tmp64.p, ctx->tmp64.p + N, ctx->ne, st, upd);
    launch_axpy(c128{1.0, 0.0}, ctx->tmp64.p + N, x, N, st, upd);
    CK("update x");
    return BEM_OK;
  };

  const int nblk = launch_dots<c128, c128>(b, N, 1, b, N, part, st);
  launch_dots_final(part, nblk, 1, bb_dev, st);
  launch_gm_init(d, bb_dev, st);
  CK("solver state");
  TRY(test());
  const volatile GmCtl* hm = ctx->gm_mirror;
  for (;;) {
    // the next cycle's steps (they return at once if the test ended the solve)
    bool finished = false, ended = false;
    int q = 0;
    while (q < m && !ended) {
      TRY(step(q));
      ++q;
      const int chk = q - 1 - GM_LAG;  // the newest step GM_LAG behind
      if (chk < 0 && q < m) continue;
      BEM_CUDA_TRY(cudaEventSynchronize(ctx->col_events[std::max(chk, 0)]));
      prof_harvest(ctx);
      if (!hm->live) {
        finished = true;
        break;
      }
      if (!hm->active) ended = true;
    }
    if (finished) break;
    // the cycle has ended, or all its m steps are enqueued (the last one ends it)
    TRY(update());
    TRY(test());
    ++cyc;
    // every cycle the device starts takes at least one step, so the step
    // limit bounds the cycles; more would mean the state does not advance
    if (cyc > o.max_iters + 1) return fail(ctx, BEM_ERR_STATE, "GMRES state did not advance on the device");
  }
  const int its = hm->its, cycles = hm->cycles, converged = hm->converged;
  // the products of steps that ran (the cycle's step count is on the host copy)
  for (const StepProf& p : sprof) {
    const bool ran = p.cycle < cycles && p.cycle < GM_MAX_CYCLES && p.j < hm->jdone[p.cycle];
    if (ran) {
      ctx->pending.push_back({p.a, p.b, (double)sizeof(Vb) * ctx->near_entries + (double)N * 2 * sizeof(Vb),
                              (double)sizeof(Vb), ctx->prof_slot, 0});
    } else {
      ctx->event_pool.push_back(p.a);
      ctx->event_pool.push_back(p.b);
    }
  }
  if (stats) {
    stats->iters = its;
    stats->cycles = cycles;
    stats->rel_residual = hm->rel;
    stats->guess_residual = hm->guess_rel;
    stats->converged = converged;
    stats->precond = leaf ? BEM_PRECOND_LEAF : BEM_PRECOND_BLOCK3;
  }
  return converged ? BEM_OK : BEM_ERR_NOT_CONVERGED;
}

int gmres(bem_ctx* ctx, const c128* b, c128* x, const bem_opts& o, bem_freq_stats* st) {
  if (is_mixed(ctx)) return gmres_impl<c64, c64, float>(ctx, b, x, o, st);
  return gmres_impl<c128, c128, double>(ctx, b, x, o, st);
}

// ---------------------------------------------------------------------------
// solution extrapolation (Sec. 4.2): a0 = X R^{-1} Q^H b, A X = Q R (CGS2, FP64)
// X: K vectors (device, stride N), in the order a_{k-1}, a_{k-2}, ...
// extra (optional): one more candidate column after them (the learned
// proposal), so that the fit over the larger span can only lower the residual.
// The products A X run as one multi-right-hand-side H-matrix product, the fit
// as one cooperative kernel. With want_res, the residual estimates
// (res[0]: X columns alone, res[1]: every column; see launch_sem_fit) are
// copied to res_host (pinned, two values), valid once the stream has passed
// the fit.
// ---------------------------------------------------------------------------
int sem_impl(bem_ctx* ctx, const c128* const* X, int K, const c128* b, c128* a0, const c128* extra = nullptr,
             double* res_host = nullptr) {
  cudaStream_t st = ctx->stream;
  const long long N = ctx->N;
  const bool want_res = res_host != nullptr;
  if (want_res) res_host[0] = res_host[1] = 1.0;
  const int C = K + (extra ? 1 : 0);
  if (C <= 0) {
    BEM_CUDA_TRY(cudaMemsetAsync(a0, 0, N * sizeof(c128), st));
    return BEM_OK;
  }
  if (C > SEM_MAXC) return fail(ctx, BEM_ERR_INVALID_ARG, "too many extrapolation columns");
  std::vector<const c128*> cols(C);
  for (int c = 0; c < C; ++c) cols[c] = c < K ? X[c] : extra;
  BEM_CUDA_TRY(ctx->sem_work.ensure(3LL * C * N));
  c128* Xc = ctx->sem_work.p;
  c128* Y = Xc + (long long)C * N;
  c128* Q = Y + (long long)C * N;
  for (int q = 0; q < C; ++q)
    BEM_CUDA_TRY(cudaMemcpyAsync(Xc + q * N, cols[q], N * sizeof(c128), cudaMemcpyDeviceToDevice, st));
  for (int q = 0; q < C; q += 4) TRY(apply_fast(ctx, Xc + q * N, Y + q * N, std::min(4, C - q)));
  BEM_CUDA_TRY(ctx->sem_part.ensure((size_t)3 * (SEM_MAXC + 1) * arnoldi_orth_max_blocks()));
  BEM_CUDA_TRY(ctx->sem_res.ensure(2));
  {
    CoopLane lane(ctx, st);
    BEM_CUDA_TRY(lane.status());
    BEM_CUDA_TRY(launch_sem_fit(cols.data(), C, K, Y, b, Q, ctx->sem_part.p, a0, ctx->sem_res.p, N, lane.stream()));
    BEM_CUDA_TRY(lane.join());
  }
  CK("sem fit");
  if (want_res)
    BEM_CUDA_TRY(cudaMemcpyAsync(res_host, ctx->sem_res.p, 2 * sizeof(double),
                                 cudaMemcpyDeviceToHost, st));
  return BEM_OK;
}

}  // namespace

// ---------------------------------------------------------------------------
// step-level entry points
// ---------------------------------------------------------------------------
extern "C" int bem_assemble(bem_ctx* ctx, double s_re, double s_im, const bem_opts* opts) {
  if (!ctx) return BEM_ERR_INVALID_ARG;
  TRY(check_ready(ctx));
  TRY(set_device(ctx));
  bem_opts o = ctx->mesh_opts;
  if (opts) o = *opts;
  if (!(s_re >= 0) || !std::isfinite(s_im)) return fail(ctx, BEM_ERR_INVALID_ARG, "need Re(s) >= 0");
  TRY(assemble_impl(ctx, s_re, s_im, o, nullptr, c128{0, 0}, nullptr, ctx->stream));
  BEM_CUDA_TRY(cudaStreamSynchronize(ctx->stream));
  return BEM_OK;
}

// Entries count at base + off + i stride (i < count) of an operator array of
// complex64 (mixed) or complex128 entries, as complex128 on the host.
static int fetch_entries(bem_ctx* ctx, const void* base, bool c64s, long long off, long long count, long long stride,
                         std::vector<c128>& out) {
  out.assign(count, c128{0, 0});
  if (count == 0) return BEM_OK;
  const size_t esz = c64s ? sizeof(c64) : sizeof(c128);
  std::vector<unsigned char> tmp(count * esz);
  const unsigned char* src = static_cast<const unsigned char*>(base) + off * esz;
  cudaStream_t st = ctx->stream;
  if (stride == 1)
    BEM_CUDA_TRY(cudaMemcpyAsync(tmp.data(), src, count * esz, cudaMemcpyDeviceToHost, st));
  else
    BEM_CUDA_TRY(cudaMemcpy2DAsync(tmp.data(), esz, src, stride * esz, esz, count, cudaMemcpyDeviceToHost, st));
  BEM_CUDA_TRY(cudaStreamSynchronize(st));
  for (long long i = 0; i < count; ++i) {
    if (c64s) {
      c64 v;
      std::memcpy(&v, tmp.data() + i * esz, esz);
      out[i] = c128{v.re, v.im};
    } else {
      std::memcpy(&out[i], tmp.data() + i * esz, esz);
    }
  }
  return BEM_OK;
}

extern "C" int bem_operator_rows(bem_ctx* ctx, const int64_t* rows, int64_t nrows, double* out) {
  if (!ctx || (!rows && nrows) || (!out && nrows) || nrows < 0) return BEM_ERR_INVALID_ARG;
  if (!ctx->assembled) return fail(ctx, BEM_ERR_STATE, "operator not assembled");
  TRY(set_device(ctx));
  const long long N = ctx->N;
  for (int64_t r = 0; r < nrows; ++r)
    if (rows[r] < 0 || rows[r] >= N) return fail(ctx, BEM_ERR_INVALID_ARG, "row index out of range");
  // the stored entries of each row's blocks are read from the device; the
  // low-rank entries are formed on the host in FP64
  const bool mixed = is_mixed(ctx);
  const void* nearp = mixed ? (const void*)ctx->near32.p : (const void*)ctx->near64.p;
  const void* Up = mixed ? (const void*)ctx->u32.p : (const void*)ctx->u64.p;
  const void* Vp = mixed ? (const void*)ctx->v32.p : (const void*)ctx->v64.p;
  const size_t nf = ctx->far_h.size();
  std::vector<int> rk(nf);
  std::vector<long long> fbase(2 * nf);
  cudaStream_t st = ctx->stream;
  if (nf) {
    BEM_CUDA_TRY(cudaMemcpyAsync(rk.data(), ctx->rank.p, nf * sizeof(int), cudaMemcpyDeviceToHost, st));
    BEM_CUDA_TRY(cudaMemcpyAsync(fbase.data(), ctx->fbase.p, 2 * nf * sizeof(long long), cudaMemcpyDeviceToHost, st));
  }
  BEM_CUDA_TRY(cudaStreamSynchronize(st));
  const auto& perm = ctx->tree.perm;
  const auto& ip = ctx->tree.iperm;
  std::vector<c128> a, u, v;
  for (int64_t q = 0; q < nrows; ++q) {
    long long rc = rows[q];            // caller dof
    int ec = (int)(rc / 3), ca = (int)(rc % 3);
    int et = ip[ec];                   // tree element
    long long rt = 3LL * et + ca;      // tree row
    std::vector<c128> rowt(N, c128{0, 0});
    for (const NearBlk& nb : ctx->near_h) {
      if (et < nb.r0 || et >= nb.r0 + nb.nr) continue;
      long long lr = rt - 3LL * nb.r0;
      TRY(fetch_entries(ctx, nearp, mixed, nb.off + lr, 3LL * nb.nc, nb.ld, a));
      for (int c = 0; c < 3 * nb.nc; ++c) rowt[3LL * nb.c0 + c] = a[c];
    }
    for (size_t b = 0; b < nf; ++b) {
      const FarBlk& fb = ctx->far_h[b];
      if (et < fb.r0 || et >= fb.r0 + fb.nr) continue;
      long long m = 3LL * fb.nr, n = 3LL * fb.nc, lr = rt - 3LL * fb.r0;
      const int r = rk[b];
      TRY(fetch_entries(ctx, Up, mixed, fbase[2 * b] + lr, r, m, u));
      TRY(fetch_entries(ctx, Vp, mixed, fbase[2 * b + 1], n * r, 1, v));
      for (long long c = 0; c < n; ++c) {
        std::complex<double> sum = 0;
        for (int l = 0; l < r; ++l)
          sum += std::complex<double>(u[l].re, u[l].im) * std::complex<double>(v[l * n + c].re, v[l * n + c].im);
        rowt[3LL * fb.c0 + c] = c128{sum.real(), sum.imag()};
      }
    }
    double* o = out + 2 * q * N;
    for (int k = 0; k < ctx->ne; ++k)
      for (int c = 0; c < 3; ++c) {
        long long dc = 3LL * perm[k] + c;
        o[2 * dc] = rowt[3LL * k + c].re;
        o[2 * dc + 1] = rowt[3LL * k + c].im;
      }
  }
  return BEM_OK;
}

extern "C" int bem_apply(bem_ctx* ctx, const double* x, double* y) {
  if (!ctx || !x || !y) return BEM_ERR_INVALID_ARG;
  if (!ctx->assembled) return fail(ctx, BEM_ERR_STATE, "operator not assembled");
  TRY(set_device(ctx));
  std::vector<c128> xt;
  to_tree(ctx, x, xt);
  DevBuf<c128> xd, yd;
  BEM_CUDA_TRY(xd.alloc(ctx->N));
  BEM_CUDA_TRY(yd.alloc(ctx->N));
  BEM_CUDA_TRY(cudaMemcpyAsync(xd.p, xt.data(), ctx->N * sizeof(c128), cudaMemcpyHostToDevice, ctx->stream));
  TRY(apply64(ctx, xd.p, yd.p, 1));
  BEM_CUDA_TRY(cudaMemcpyAsync(xt.data(), yd.p, ctx->N * sizeof(c128), cudaMemcpyDeviceToHost, ctx->stream));
  BEM_CUDA_TRY(cudaStreamSynchronize(ctx->stream));
  from_tree(ctx, xt, y);
  return BEM_OK;
}

extern "C" int bem_apply_preconditioner(bem_ctx* ctx, int32_t precond, const double* x, double* y) {
  if (!ctx || !x || !y) return BEM_ERR_INVALID_ARG;
  if (!ctx->assembled) return fail(ctx, BEM_ERR_STATE, "operator not assembled");
  if (precond != BEM_PRECOND_BLOCK3 && precond != BEM_PRECOND_LEAF)
    return fail(ctx, BEM_ERR_INVALID_ARG, "precond must be BEM_PRECOND_BLOCK3 or BEM_PRECOND_LEAF");
  if (precond == BEM_PRECOND_LEAF && !ctx->minv_ready)
    return fail(ctx, BEM_ERR_STATE, "no leaf-block inverses: assemble with precond = BEM_PRECOND_LEAF");
  TRY(set_device(ctx));
  std::vector<c128> xt;
  to_tree(ctx, x, xt);
  DevBuf<c128> xd, yd;
  BEM_CUDA_TRY(xd.alloc(ctx->N));
  BEM_CUDA_TRY(yd.alloc(ctx->N));
  BEM_CUDA_TRY(cudaMemcpyAsync(xd.p, xt.data(), ctx->N * sizeof(c128), cudaMemcpyHostToDevice, ctx->stream));
  if (precond == BEM_PRECOND_BLOCK3)
    launch_precond<c128, c128, c128>(ctx->prec_inv.p, xd.p, yd.p, ctx->ne, ctx->stream);
  else if (is_mixed(ctx))
    launch_leaf_apply<c64, c128, c128>(ctx->leaf_pre.p, ctx->nleaf_pre, ctx->minv32.p, xd.p, yd.p, ctx->stream);
  else
    launch_leaf_apply<c128, c128, c128>(ctx->leaf_pre.p, ctx->nleaf_pre, ctx->minv64.p, xd.p, yd.p, ctx->stream);
  CK("apply preconditioner");
  BEM_CUDA_TRY(cudaMemcpyAsync(xt.data(), yd.p, ctx->N * sizeof(c128), cudaMemcpyDeviceToHost, ctx->stream));
  BEM_CUDA_TRY(cudaStreamSynchronize(ctx->stream));
  from_tree(ctx, xt, y);
  return BEM_OK;
}

extern "C" int bem_rhs(bem_ctx* ctx, double p_re, double p_im, const double* pattern, double* b) {
  if (!ctx || !pattern || !b) return BEM_ERR_INVALID_ARG;
  if (!ctx->assembled) return fail(ctx, BEM_ERR_STATE, "operator not assembled");
  TRY(set_device(ctx));
  TRY(set_pattern_host(ctx, pattern));
  DevBuf<c128> bd;
  BEM_CUDA_TRY(bd.alloc(ctx->N));
  c128 pk{p_re, p_im};
  KParams<double> Pd = make_params<double>(ctx, ctx->s_re, ctx->s_im);
  BEM_CUDA_TRY(cudaMemsetAsync(bd.p, 0, ctx->N * sizeof(c128), ctx->stream));
  if (is_mixed(ctx)) {
    KParams<float> Pf = make_params<float>(ctx, ctx->s_re, ctx->s_im);
    launch_rhs_far<float>(ctx->rhs_rng.p, ctx->rhs_rptr.p, ctx->elem_leaf.p, ctx->ne, ctx->ef.p, ctx->ed.p, ctx->bc.p,
                          ctx->patf.p, ctx->pattern.p, Pf, pk, bd.p, ctx->stream);
    launch_near_regular<float, c64>(ctx->near_d.p, (int)ctx->near_h.size(), ctx->max_nr, ctx->plist.p, ctx->poff.p,
                                    ctx->pcount.p, ctx->ef.p, ctx->ed.p, ctx->bc.p, Pf, (c64*)nullptr, ctx->patf.p,
                                    ctx->pattern.p, pk, bd.p, ctx->stream);
    launch_sing<float, c64>(ctx->sing.p, ctx->nsing, ctx->ed.p, ctx->polar.p, ctx->bc.p, ctx->sing_static.p, Pf,
                            nullptr, nullptr, ctx->pattern.p, pk, bd.p, ctx->status.p, ctx->stream);
  } else {
    launch_rhs_far<double>(ctx->rhs_rng.p, ctx->rhs_rptr.p, ctx->elem_leaf.p, ctx->ne, ctx->ef.p, ctx->ed.p, ctx->bc.p,
                           ctx->patf.p, ctx->pattern.p, Pd, pk, bd.p, ctx->stream);
    launch_near_regular<double, c128>(ctx->near_d.p, (int)ctx->near_h.size(), ctx->max_nr, ctx->plist.p,
                                      ctx->poff.p, ctx->pcount.p, ctx->ef.p, ctx->ed.p, ctx->bc.p, Pd,
                                      (c128*)nullptr, ctx->patf.p, ctx->pattern.p, pk, bd.p, ctx->stream);
    launch_sing<double, c128>(ctx->sing.p, ctx->nsing, ctx->ed.p, ctx->polar.p, ctx->bc.p, ctx->sing_static.p, Pd,
                              nullptr, nullptr, ctx->pattern.p, pk, bd.p, ctx->status.p, ctx->stream);
  }
  CK("rhs");
  std::vector<c128> bt(ctx->N);
  BEM_CUDA_TRY(cudaMemcpyAsync(bt.data(), bd.p, ctx->N * sizeof(c128), cudaMemcpyDeviceToHost, ctx->stream));
  BEM_CUDA_TRY(cudaStreamSynchronize(ctx->stream));
  from_tree(ctx, bt, b);
  return BEM_OK;
}

extern "C" int bem_solve_assembled(bem_ctx* ctx, const double* b, const double* x0, double* x, const bem_opts* opts,
                                   bem_freq_stats* stats) {
  if (!ctx || !b || !x) return BEM_ERR_INVALID_ARG;
  if (!ctx->assembled) return fail(ctx, BEM_ERR_STATE, "operator not assembled");
  TRY(set_device(ctx));
  bem_opts o = ctx->mesh_opts;
  if (opts) o = *opts;
  if (!(o.tol > 0) || o.restart < 1 || o.max_iters < 0) return fail(ctx, BEM_ERR_INVALID_ARG, "bad solver options");
  if (o.precision != ctx->prec) return fail(ctx, BEM_ERR_STATE, "precision differs from the assembled operator");
  std::vector<c128> bt, xt;
  to_tree(ctx, b, bt);
  if (x0) to_tree(ctx, x0, xt);
  else xt.assign(ctx->N, c128{0, 0});
  BEM_CUDA_TRY(ctx->b64.ensure(ctx->N));
  BEM_CUDA_TRY(ctx->x64.ensure(ctx->N));
  BEM_CUDA_TRY(cudaMemcpyAsync(ctx->b64.p, bt.data(), ctx->N * sizeof(c128), cudaMemcpyHostToDevice, ctx->stream));
  BEM_CUDA_TRY(cudaMemcpyAsync(ctx->x64.p, xt.data(), ctx->N * sizeof(c128), cudaMemcpyHostToDevice, ctx->stream));
  if (o.precond == BEM_PRECOND_LEAF && !ctx->minv_ready)
    return fail(ctx, BEM_ERR_STATE, "assemble with precond = BEM_PRECOND_LEAF first");
  ctx->use_leaf_pre = ctx->minv_ready && (o.precond == BEM_PRECOND_LEAF ||
                                          (o.precond == BEM_PRECOND_AUTO && ctx->pre_auto == 2));
  bem_freq_stats s{};
  auto t0 = std::chrono::steady_clock::now();
  int rc = gmres(ctx, ctx->b64.p, ctx->x64.p, o, &s);
  if (rc != BEM_OK && rc != BEM_ERR_NOT_CONVERGED) return rc;
  BEM_CUDA_TRY(cudaMemcpyAsync(xt.data(), ctx->x64.p, ctx->N * sizeof(c128), cudaMemcpyDeviceToHost, ctx->stream));
  BEM_CUDA_TRY(cudaStreamSynchronize(ctx->stream));
  s.solve_ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
  s.s_re = ctx->s_re;
  s.s_im = ctx->s_im;
  from_tree(ctx, xt, x);
  if (stats) *stats = s;
  if (rc == BEM_ERR_NOT_CONVERGED) fail(ctx, rc, "GMRES did not reach the tolerance");
  return rc;
}

extern "C" int bem_sem_guess(bem_ctx* ctx, int32_t K, const double* X, const double* b, double* a0) {
  if (!ctx || !b || !a0 || K < 0 || (K > 0 && !X)) return BEM_ERR_INVALID_ARG;
  if (!ctx->assembled) return fail(ctx, BEM_ERR_STATE, "operator not assembled");
  if (K > 4) return fail(ctx, BEM_ERR_INVALID_ARG, "K must be <= 4");
  TRY(set_device(ctx));
  const long long N = ctx->N;
  DevBuf<c128> Xd, bd, ad;
  BEM_CUDA_TRY(Xd.alloc(std::max<long long>(1, K * N)));
  BEM_CUDA_TRY(bd.alloc(N));
  BEM_CUDA_TRY(ad.alloc(N));
  std::vector<c128> t;
  std::vector<const c128*> ptrs;
  for (int q = 0; q < K; ++q) {
    to_tree(ctx, X + 2 * q * N, t);
    BEM_CUDA_TRY(cudaMemcpyAsync(Xd.p + q * N, t.data(), N * sizeof(c128), cudaMemcpyHostToDevice, ctx->stream));
    BEM_CUDA_TRY(cudaStreamSynchronize(ctx->stream));
    ptrs.push_back(Xd.p + q * N);
  }
  to_tree(ctx, b, t);
  BEM_CUDA_TRY(cudaMemcpyAsync(bd.p, t.data(), N * sizeof(c128), cudaMemcpyHostToDevice, ctx->stream));
  TRY(sem_impl(ctx, ptrs.data(), K, bd.p, ad.p));
  BEM_CUDA_TRY(cudaMemcpyAsync(t.data(), ad.p, N * sizeof(c128), cudaMemcpyDeviceToHost, ctx->stream));
  BEM_CUDA_TRY(cudaStreamSynchronize(ctx->stream));
  from_tree(ctx, t, a0);
  return BEM_OK;
}

extern "C" int bem_load_dft(bem_ctx* ctx, double T, int32_t n_omega, double eta, const double* load_hist, double* out) {
  if (!ctx || !load_hist || !out || n_omega < 2 || (n_omega & 1) || !(T > 0) || !(eta >= 0))
    return BEM_ERR_INVALID_ARG;
  TRY(set_device(ctx));
  int nf = n_omega / 2 + 1;
  DevBuf<double> P;
  DevBuf<c128> o;
  BEM_CUDA_TRY(P.alloc(n_omega));
  BEM_CUDA_TRY(o.alloc(nf));
  BEM_CUDA_TRY(cudaMemcpyAsync(P.p, load_hist, n_omega * sizeof(double), cudaMemcpyHostToDevice, ctx->stream));
  launch_load_dft(P.p, n_omega, T, eta, o.p, ctx->stream);
  CK("load_dft");
  BEM_CUDA_TRY(cudaMemcpyAsync(out, o.p, nf * sizeof(c128), cudaMemcpyDeviceToHost, ctx->stream));
  BEM_CUDA_TRY(cudaStreamSynchronize(ctx->stream));
  return BEM_OK;
}

static int idft_checks(bem_ctx* ctx, int n_omega) {
  if (n_omega < 2 || (n_omega & 1) || n_omega > 6000)
    return fail(ctx, BEM_ERR_INVALID_ARG, "n_omega must be even, 2..6000");
  return BEM_OK;
}

extern "C" int bem_idft(bem_ctx* ctx, double T, int32_t n_omega, double eta, int window, const double* Rk,
                        int64_t ndof, double* out) {
  if (!ctx || !Rk || !out || ndof < 0 || !(T > 0) || !(eta >= 0)) return BEM_ERR_INVALID_ARG;
  if (window < 0 || window > 2) return fail(ctx, BEM_ERR_INVALID_ARG, "unknown window");
  TRY(idft_checks(ctx, n_omega));
  TRY(set_device(ctx));
  if (ndof == 0) return BEM_OK;
  int nf = n_omega / 2 + 1;
  DevBuf<c128> s;
  DevBuf<double> o;
  BEM_CUDA_TRY(s.alloc(nf * ndof));
  BEM_CUDA_TRY(o.alloc(n_omega * ndof));
  BEM_CUDA_TRY(cudaMemcpyAsync(s.p, Rk, nf * ndof * sizeof(c128), cudaMemcpyHostToDevice, ctx->stream));
  launch_idft(s.p, ndof, nullptr, ndof, n_omega, T, eta, window, o.p, ctx->stream);
  CK("idft");
  BEM_CUDA_TRY(cudaMemcpyAsync(out, o.p, n_omega * ndof * sizeof(double), cudaMemcpyDeviceToHost, ctx->stream));
  BEM_CUDA_TRY(cudaStreamSynchronize(ctx->stream));
  return BEM_OK;
}

// ---------------------------------------------------------------------------
// the sweep
// ---------------------------------------------------------------------------
static int sweep_body(bem_ctx* ctx, double T, int n_omega, const double* load_dev, const bem_opts& o,
                      bem_freq_stats* stats) {
  cudaStream_t st = ctx->stream;
  const long long N = ctx->N;
  int nf = n_omega / 2 + 1;
  ctx->T = T;
  ctx->n_omega = n_omega;
  ctx->nf = 0;
  BEM_CUDA_TRY(ctx->Pk.ensure(nf));
  launch_load_dft(load_dev, n_omega, T, ctx->eta, ctx->Pk.p, st);
  CK("load_dft");
  ctx->Pk_host.resize(nf);
  BEM_CUDA_TRY(cudaMemcpyAsync(ctx->Pk_host.data(), ctx->Pk.p, nf * sizeof(c128), cudaMemcpyDeviceToHost, st));
  BEM_CUDA_TRY(ctx->sol.ensure((long long)nf * N));
  BEM_CUDA_TRY(ctx->b64.ensure(N));
  BEM_CUDA_TRY(cudaStreamSynchronize(st));
  const double dw = 2.0 * M_PI / T;
  const double dt = T / n_omega;
  int worst = BEM_OK;
  // per frequency: assembly, guess and solve events, the ACA failure count
  // and the extrapolation residuals, read once the sweep has completed (the
  // host waits on no frequency's end)
  struct FreqRec {
    cudaEvent_t a0 = nullptr, a1 = nullptr, g0 = nullptr, g1 = nullptr, s0 = nullptr, s1 = nullptr;
    bool fit = false;
  };
  std::vector<FreqRec> rec(nf);
  for (FreqRec& r : rec) {
    r.a0 = take_event(ctx);
    r.a1 = take_event(ctx);
    r.g0 = take_event(ctx);
    r.g1 = take_event(ctx);
    r.s0 = take_event(ctx);
    r.s1 = take_event(ctx);
  }
  struct RecRelease {
    bem_ctx* c;
    std::vector<FreqRec>& r;
    ~RecRelease() {
      for (FreqRec& x : r)
        for (cudaEvent_t e : {x.a0, x.a1, x.g0, x.g1, x.s0, x.s1}) c->event_pool.push_back(e);
    }
  } rec_release{ctx, rec};
  if ((size_t)(3 * nf) > ctx->sweep_pin_n) {
    if (ctx->sweep_pin) cudaFreeHost(ctx->sweep_pin);
    ctx->sweep_pin = nullptr;
    ctx->sweep_pin_n = 0;
    BEM_CUDA_TRY(cudaMallocHost(&ctx->sweep_pin, 3 * (size_t)nf * sizeof(double)));
    ctx->sweep_pin_n = 3 * (size_t)nf;
  }
  double* sem_h = ctx->sweep_pin;                              // 2 per frequency
  int* fails_h = reinterpret_cast<int*>(ctx->sweep_pin + 2 * nf);  // 1 per frequency
  std::vector<bem_freq_stats> sv(nf);
  // frequency 0 on the caller's stream; afterwards frequency k + 1 is
  // assembled on asm_stream into the other operator set while the guess and
  // GMRES of frequency k run on the caller's stream (compact storage keeps one
  // operator set: frequency k + 1 is assembled after frequency k is solved)
  ctx->pre_auto = 0;
  ctx->far_verify_pending = false;
  cudaEventRecord(rec[0].a0, st);
  TRY(assemble_impl(ctx, ctx->eta, 0.0, o, ctx->pattern.p, ctx->Pk_host[0], ctx->b64.p, st));
  cudaEventRecord(rec[0].a1, st);
  // compact storage overlaps too when a second operator set (near blocks,
  // pools at their current size, leaf inverses) fits in a fifth of the free
  // device memory (of this context's share of it in a batched sweep)
  // (full storage: a third set when one fits in that fifth as well)
  size_t freeb = 0, totalb = 0;
  BEM_CUDA_TRY(cudaMemGetInfo(&freeb, &totalb));
  const double esz = is_mixed(ctx) ? 8.0 : 16.0;
  const double pools = ctx->far_compact ? 1.25 * (is_mixed(ctx) ? (double)(ctx->u32.n + ctx->v32.n)
                                                                 : (double)(ctx->u64.n + ctx->v64.n))
                                        : (double)(ctx->u_entries + ctx->v_entries);
  const double set_bytes = esz * ((double)ctx->near_entries + pools + (double)ctx->leaf_pre_entries) + 16.0 * (double)N;
  const bool set_fits = set_bytes <= 0.2 * ctx->mem_share * (double)freeb;
  const bool pipe = !ctx->far_compact || set_fits;
  // depth: operator sets in the ring. Full storage keeps three where they
  // fit, so that the assembly stream runs up to two frequencies ahead of the
  // solve and neither stream waits for the other when one frequency takes
  // longer; compact storage keeps two (one pending pool check at a time).
  const int depth = !pipe ? 1 : (ctx->far_compact || !set_fits ? 2 : 3);
  // the sets of frequencies k + 1, k + 2 live in back[bq[0]], back[bq[1]]
  int bq[2] = {0, 1};
  BEM_CUDA_TRY(cudaEventRecord(ctx->ev_asm_ring[0], st));
  int next_asm = 1;  // the next frequency to assemble (pipelined)
  for (int k = 0; k < nf; ++k) {
    bem_freq_stats s{};
    s.k = k;
    s.s_re = ctx->eta;
    s.s_im = k * dw;
    c128* xk = ctx->sol.p + (long long)k * N;
    const bool next = k + 1 < nf;
    // the guess first, so that the solve stream has work while the host
    // enqueues assemblies
    cudaEventRecord(rec[k].g0, st);
    int K = (o.guess != BEM_GUESS_ZERO) ? std::min(k, std::max(0, std::min(o.sem_k, 4))) : 0;
    const c128* prev[4] = {};
    for (int q = 1; q <= 4 && q <= k; ++q) prev[q - 1] = ctx->sol.p + (long long)(k - q) * N;
    const c128* extra = nullptr;
    if (o.guess == BEM_GUESS_MLP && k >= 4) TRY(mlp_propose(ctx, prev, s.s_re * dt, s.s_im * dt, &extra));
    const bool fit = K > 0 || extra;
    rec[k].fit = fit;
    if (fit) {
      TRY(sem_impl(ctx, prev, K, ctx->b64.p, xk, extra, sem_h + 2 * k));
    } else {
      BEM_CUDA_TRY(cudaMemsetAsync(xk, 0, N * sizeof(c128), st));
    }
    cudaEventRecord(rec[k].g1, st);
    // assemblies of the frequencies up to k + depth - 1, each into the set
    // last used by frequency f - depth (after that solve: ev_free_ring) and
    // after the previous assembly (the pivot state passes from one to the next)
    for (; depth > 1 && next_asm < nf && next_asm <= k + depth - 1; ++next_asm) {
      const int f = next_asm, slot = f % depth, bi = bq[f - k - 1];
      swap_ops(ctx, bi);
      BEM_CUDA_TRY(ctx->b64.ensure(N));
      cudaStream_t as = ctx->asm_stream;
      BEM_CUDA_TRY(cudaStreamWaitEvent(as, ctx->ev_asm_ring[(f - 1) % depth], 0));
      BEM_CUDA_TRY(cudaStreamWaitEvent(as, ctx->ev_free_ring[slot], 0));
      cudaEventRecord(rec[f].a0, as);
      ctx->far_defer = ctx->far_compact;
      const int arc =
          assemble_impl(ctx, ctx->eta, f * dw, o, ctx->pattern.p, ctx->Pk_host[f], ctx->b64.p, as);
      ctx->far_defer = false;
      TRY(arc);
      cudaEventRecord(rec[f].a1, as);
      BEM_CUDA_TRY(cudaEventRecord(ctx->ev_asm_ring[slot], as));
      swap_ops(ctx, bi);
    }
    cudaEventRecord(rec[k].s0, st);
    int rc;
    if (o.precond == BEM_PRECOND_AUTO && ctx->pre_auto == 0 && k >= 1 && ctx->minv_ready) {
      // the first frequency with k > 0 is solved with both preconditioners
      // from the same initial guess; the one with fewer Arnoldi steps is kept
      // for the rest of the sweep (both solutions meet the tolerance)
      BEM_CUDA_TRY(ctx->w64.ensure(2 * N));
      c128* x0 = ctx->w64.p;
      c128* x3 = ctx->w64.p + N;
      BEM_CUDA_TRY(cudaMemcpyAsync(x0, xk, N * sizeof(c128), cudaMemcpyDeviceToDevice, st));
      bem_freq_stats s3 = s;
      ctx->use_leaf_pre = false;
      const int rc3 = gmres(ctx, ctx->b64.p, xk, o, &s3);
      if (rc3 != BEM_OK && rc3 != BEM_ERR_NOT_CONVERGED) return rc3;
      BEM_CUDA_TRY(cudaMemcpyAsync(x3, xk, N * sizeof(c128), cudaMemcpyDeviceToDevice, st));
      BEM_CUDA_TRY(cudaMemcpyAsync(xk, x0, N * sizeof(c128), cudaMemcpyDeviceToDevice, st));
      ctx->use_leaf_pre = true;
      rc = gmres(ctx, ctx->b64.p, xk, o, &s);
      if (rc != BEM_OK && rc != BEM_ERR_NOT_CONVERGED) return rc;
      const bool leaf_wins = rc == BEM_OK && (rc3 != BEM_OK || s.iters < s3.iters);
      ctx->pre_auto = leaf_wins ? 2 : 1;
      const int trial = leaf_wins ? s3.iters : s.iters;
      if (!leaf_wins) {
        BEM_CUDA_TRY(cudaMemcpyAsync(xk, x3, N * sizeof(c128), cudaMemcpyDeviceToDevice, st));
        s.iters = s3.iters;
        s.cycles = s3.cycles;
        s.rel_residual = s3.rel_residual;
        s.converged = s3.converged;
        s.precond = s3.precond;
        rc = rc3;
      }
      s.guess_residual = s3.guess_residual;
      s.trial_iters = trial;
      s.iters += trial;
    } else {
      ctx->use_leaf_pre = ctx->minv_ready && (o.precond == BEM_PRECOND_LEAF ||
                                              (o.precond == BEM_PRECOND_AUTO && ctx->pre_auto == 2));
      rc = gmres(ctx, ctx->b64.p, xk, o, &s);
    }
    cudaEventRecord(rec[k].s1, st);
    if (rc != BEM_OK && rc != BEM_ERR_NOT_CONVERGED) return rc;
    if (rc == BEM_ERR_NOT_CONVERGED) worst = rc;
    if (o.guess == BEM_GUESS_MLP && k >= 4)
      TRY(mlp_train(ctx, prev, xk, s.s_re * dt, s.s_im * dt, ctx->mlp_steps, ctx->mlp_lr));
    BEM_CUDA_TRY(cudaMemcpyAsync(fails_h + k, ctx->aca_fail.p, sizeof(int), cudaMemcpyDeviceToHost, st));
    // this operator set is free for the assembly of frequency k + depth after here
    BEM_CUDA_TRY(cudaEventRecord(ctx->ev_free_ring[k % depth], st));
    s.near_bytes = ctx->near_entries * (is_mixed(ctx) ? 8 : 16);
    sv[k] = s;
    ctx->nf = k + 1;
    if (next && depth > 1) {
      // frequency k + 1's operator and right-hand side become the set in use;
      // frequency k's set goes to the end of the queue
      BEM_CUDA_TRY(cudaStreamWaitEvent(st, ctx->ev_asm_ring[(k + 1) % depth], 0));
      swap_ops(ctx, bq[0]);
      if (depth == 3) std::swap(bq[0], bq[1]);
      TRY(far_field_verify(ctx, o));
    } else if (next) {
      cudaEventRecord(rec[k + 1].a0, st);
      TRY(assemble_impl(ctx, ctx->eta, (k + 1) * dw, o, ctx->pattern.p, ctx->Pk_host[k + 1], ctx->b64.p, st));
      cudaEventRecord(rec[k + 1].a1, st);
    }
  }
  BEM_CUDA_TRY(cudaStreamSynchronize(st));
  BEM_CUDA_TRY(cudaStreamSynchronize(ctx->asm_stream));
  prof_harvest(ctx);
  for (int k = 0; k < nf; ++k) {
    bem_freq_stats& s = sv[k];
    float ms = 0;
    cudaEventElapsedTime(&ms, rec[k].a0, rec[k].a1);
    s.assemble_ms = ms;
    cudaEventElapsedTime(&ms, rec[k].g0, rec[k].g1);
    s.guess_ms = ms;
    cudaEventElapsedTime(&ms, rec[k].s0, rec[k].s1);
    s.solve_ms = ms;
    s.sem_residual = rec[k].fit ? sem_h[2 * k] : 1.0;
    s.aca_failures = fails_h[k];
    if (stats) stats[k] = s;
  }
  if (stats && !ctx->far_h.empty()) {
    std::vector<int> rk(ctx->far_h.size());
    BEM_CUDA_TRY(cudaMemcpy(rk.data(), ctx->rank.p, rk.size() * sizeof(int), cudaMemcpyDeviceToHost));
    long long fb = 0;
    int mr = 0;
    for (size_t b = 0; b < rk.size(); ++b) {
      fb += (long long)rk[b] * 3 * (ctx->far_h[b].nr + ctx->far_h[b].nc);
      mr = std::max(mr, rk[b]);
    }
    stats[nf - 1].far_bytes = fb * (is_mixed(ctx) ? 8 : 16);
    stats[nf - 1].max_rank = mr;
  }
  if (worst != BEM_OK) fail(ctx, worst, "at least one frequency did not reach the tolerance");
  return worst;
}

// The sweep runs on the context's greatest-priority stream, forked from and
// joined back to the caller's stream: the block scheduler then dispatches the
// guess and GMRES work of frequency k ahead of pending blocks of the
// least-priority assembly of k + 1, which otherwise occupies the SMs the
// short solver kernels wait for.
static int sweep_impl(bem_ctx* ctx, double T, int n_omega, const double* load_dev, const bem_opts& o,
                      bem_freq_stats* stats) {
  cudaStream_t caller = ctx->stream;
  BEM_CUDA_TRY(cudaEventRecord(ctx->ev_solve_in, caller));
  BEM_CUDA_TRY(cudaStreamWaitEvent(ctx->solve_stream, ctx->ev_solve_in, 0));
  ctx->stream = ctx->solve_stream;
  int rc = sweep_body(ctx, T, n_omega, load_dev, o, stats);
  ctx->stream = caller;
  cudaError_t e = cudaEventRecord(ctx->ev_solve_out, ctx->solve_stream);
  if (e == cudaSuccess) e = cudaStreamWaitEvent(caller, ctx->ev_solve_out, 0);
  if (e != cudaSuccess && rc == BEM_OK) return fail_cuda(ctx, e, "join the solve stream", __FILE__, __LINE__);
  return rc;
}

static int sweep_checks(bem_ctx* ctx, double T, int32_t n_omega, const bem_opts& o) {
  TRY(check_ready(ctx));
  if (!(T > 0) || n_omega < 2 || (n_omega & 1) || n_omega > 6000)
    return fail(ctx, BEM_ERR_INVALID_ARG, "need T > 0 and even n_omega in 2..6000");
  if (!(o.tol > 0) || o.restart < 1 || o.max_iters < 0 || !(o.aca_tol > 0))
    return fail(ctx, BEM_ERR_INVALID_ARG, "bad solver options");
  if (o.precision != BEM_PREC_C64_MIXED && o.precision != BEM_PREC_C128)
    return fail(ctx, BEM_ERR_INVALID_ARG, "unknown precision");
  if (o.guess != BEM_GUESS_ZERO && o.guess != BEM_GUESS_SEM && o.guess != BEM_GUESS_MLP)
    return fail(ctx, BEM_ERR_INVALID_ARG, "unknown initial guess");
  if (o.precond != BEM_PRECOND_BLOCK3 && o.precond != BEM_PRECOND_LEAF && o.precond != BEM_PRECOND_AUTO)
    return fail(ctx, BEM_ERR_INVALID_ARG, "unknown preconditioner");
  if (o.precond == BEM_PRECOND_LEAF && ctx->nleaf_pre == 0)
    return fail(ctx, BEM_ERR_INVALID_ARG, "the leaf-block preconditioner needs leaves of at most 64 elements");
  return BEM_OK;
}

extern "C" int bem_solve_sweep(bem_ctx* ctx, double T, int32_t n_omega, const double* load_hist,
                               const double* bc_pattern, const bem_opts* opts, bem_freq_stats* stats) {
  if (!ctx || !load_hist || !bc_pattern) return BEM_ERR_INVALID_ARG;
  bem_opts o = ctx->mesh_opts;
  if (opts) o = *opts;
  TRY(sweep_checks(ctx, T, n_omega, o));
  TRY(set_device(ctx));
  TRY(set_pattern_host(ctx, bc_pattern));
  DevBuf<double> P;
  BEM_CUDA_TRY(P.alloc(n_omega));
  BEM_CUDA_TRY(cudaMemcpyAsync(P.p, load_hist, n_omega * sizeof(double), cudaMemcpyHostToDevice, ctx->stream));
  return sweep_impl(ctx, T, n_omega, P.p, o, stats);
}

extern "C" int bem_solve_sweep_dev(bem_ctx* ctx, double T, int32_t n_omega, const double* load_dev,
                                   const double* pattern_dev, const bem_opts* opts, bem_freq_stats* stats) {
  if (!ctx || !load_dev || !pattern_dev) return BEM_ERR_INVALID_ARG;
  bem_opts o = ctx->mesh_opts;
  if (opts) o = *opts;
  TRY(sweep_checks(ctx, T, n_omega, o));
  TRY(set_device(ctx));
  TRY(set_pattern_dev(ctx, pattern_dev));
  return sweep_impl(ctx, T, n_omega, load_dev, o, stats);
}

extern "C" int bem_get_frequency_solution(bem_ctx* ctx, int32_t k, double* out) {
  if (!ctx || !out) return BEM_ERR_INVALID_ARG;
  if (k < 0 || k >= ctx->nf) return fail(ctx, BEM_ERR_INVALID_ARG, "frequency index not solved");
  TRY(set_device(ctx));
  std::vector<c128> t(ctx->N);
  BEM_CUDA_TRY(cudaMemcpyAsync(t.data(), ctx->sol.p + (long long)k * ctx->N, ctx->N * sizeof(c128),
                               cudaMemcpyDeviceToHost, ctx->stream));
  BEM_CUDA_TRY(cudaStreamSynchronize(ctx->stream));
  from_tree(ctx, t, out);
  return BEM_OK;
}

static int time_response_impl(bem_ctx* ctx, const long long* idx_dev, long long ndof, double* out_dev) {
  if (ctx->nf != ctx->n_omega / 2 + 1 || ctx->nf == 0)
    return fail(ctx, BEM_ERR_STATE, "the sweep has not been solved");
  TRY(idft_checks(ctx, ctx->n_omega));
  launch_idft(ctx->sol.p, ctx->N, idx_dev, ndof, ctx->n_omega, ctx->T, ctx->eta, ctx->window, out_dev, ctx->stream);
  CK("idft");
  return BEM_OK;
}

extern "C" int bem_time_response(bem_ctx* ctx, const int64_t* dofs, int64_t ndof, double* out) {
  if (!ctx || (ndof > 0 && (!dofs || !out)) || ndof < 0) return BEM_ERR_INVALID_ARG;
  TRY(set_device(ctx));
  if (ndof == 0) return BEM_OK;
  std::vector<long long> idx(ndof);
  for (int64_t d = 0; d < ndof; ++d) {
    if (dofs[d] < 0 || dofs[d] >= ctx->N) return fail(ctx, BEM_ERR_INVALID_ARG, "dof out of range");
    long long e = dofs[d] / 3, a = dofs[d] % 3;
    idx[d] = 3LL * ctx->tree.iperm[e] + a;
  }
  DevBuf<long long> id;
  DevBuf<double> o;
  BEM_CUDA_TRY(id.alloc(ndof));
  BEM_CUDA_TRY(o.alloc((long long)ctx->n_omega * ndof));
  BEM_CUDA_TRY(cudaMemcpyAsync(id.p, idx.data(), ndof * sizeof(long long), cudaMemcpyHostToDevice, ctx->stream));
  TRY(time_response_impl(ctx, id.p, ndof, o.p));
  BEM_CUDA_TRY(cudaMemcpyAsync(out, o.p, (long long)ctx->n_omega * ndof * sizeof(double), cudaMemcpyDeviceToHost,
                               ctx->stream));
  BEM_CUDA_TRY(cudaStreamSynchronize(ctx->stream));
  return BEM_OK;
}

__global__ void k_map_dofs(const long long* __restrict__ in, const int* __restrict__ iperm, long long n,
                           long long ndofs, long long* __restrict__ out, int* __restrict__ bad) {
  long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (i >= n) return;
  long long d = in[i];
  if (d < 0 || d >= ndofs) {
    atomicExch(bad, 1);
    out[i] = 0;
    return;
  }
  out[i] = 3LL * iperm[d / 3] + d % 3;
}

extern "C" int bem_time_response_dev(bem_ctx* ctx, const int64_t* dofs_dev, int64_t ndof, double* out_dev) {
  if (!ctx || (ndof > 0 && (!dofs_dev || !out_dev)) || ndof < 0) return BEM_ERR_INVALID_ARG;
  TRY(set_device(ctx));
  if (ndof == 0) return BEM_OK;
  if (ctx->nf == 0) return fail(ctx, BEM_ERR_STATE, "the sweep has not been solved");
  DevBuf<long long> id;
  DevBuf<int> bad;
  BEM_CUDA_TRY(id.alloc(ndof));
  BEM_CUDA_TRY(bad.alloc(1));
  BEM_CUDA_TRY(cudaMemsetAsync(bad.p, 0, sizeof(int), ctx->stream));
  count_if(true);
  k_map_dofs<<<(unsigned)((ndof + 255) / 256), 256, 0, ctx->stream>>>((const long long*)dofs_dev, ctx->iperm.p,
                                                                      ndof, ctx->N, id.p, bad.p);
  CK("map_dofs");
  int bad_h = 0;
  BEM_CUDA_TRY(cudaMemcpyAsync(&bad_h, bad.p, sizeof(int), cudaMemcpyDeviceToHost, ctx->stream));
  BEM_CUDA_TRY(cudaStreamSynchronize(ctx->stream));
  if (bad_h) return fail(ctx, BEM_ERR_INVALID_ARG, "dof out of range");
  TRY(time_response_impl(ctx, id.p, ndof, out_dev));
  BEM_CUDA_TRY(cudaStreamSynchronize(ctx->stream));
  return BEM_OK;
}

extern "C" int bem_set_profiling(bem_ctx* ctx, int on) {
  if (!ctx) return BEM_ERR_INVALID_ARG;
  TRY(set_device(ctx));
  BEM_CUDA_TRY(cudaStreamSynchronize(ctx->stream));
  prof_harvest(ctx);
  ctx->profiling = on != 0;
  ctx->prof_hmv_launches = ctx->prof_asm_calls = 0;
  ctx->prof_hmv_ms = ctx->prof_asm_ms = 0;
  ctx->prof_aca_blocks = ctx->prof_aca_continued = 0;
  ctx->prof_products.clear();
  ctx->prof_slot = ctx->prof_nslots = 0;
  if (ctx->profiling) {
    BEM_CUDA_TRY(ctx->prof_dev.ensure(PROF_SLOTS));
    BEM_CUDA_TRY(cudaMemsetAsync(ctx->prof_dev.p, 0, PROF_SLOTS * sizeof(long long), ctx->stream));
    if (ctx->assembled) {
      // the operator assembled before profiling began is slot 1
      ctx->prof_slot = ctx->prof_nslots = 1;
      const int nf = (int)ctx->far_h.size();
      if (nf) {
        count_if(true);
        k_lowrank_entries<<<std::min<int>(64, (nf + 255) / 256), 256, 0, ctx->stream>>>(ctx->rank.p, ctx->far_d.p,
                                                                                       nf, ctx->prof_dev.p + 1);
      }
      BEM_CUDA_TRY(cudaGetLastError());
    }
  }
  ctx->launches_at_reset = launch_count();
  return BEM_OK;
}

extern "C" int bem_far_block_info(bem_ctx* ctx, int64_t nmax, int32_t* info, int64_t* count) {
  if (!ctx || !count || nmax < 0 || (nmax > 0 && !info)) return BEM_ERR_INVALID_ARG;
  const int64_t nf = (int64_t)ctx->far_h.size();
  *count = nf;
  if (nmax == 0 || nf == 0) return BEM_OK;
  if (!ctx->assembled) return fail(ctx, BEM_ERR_STATE, "operator not assembled");
  TRY(set_device(ctx));
  std::vector<int> rk(nf), ks(nf, -1), dn(nf, 0);
  cudaStream_t st = ctx->stream;
  BEM_CUDA_TRY(cudaMemcpyAsync(rk.data(), ctx->rank.p, nf * sizeof(int), cudaMemcpyDeviceToHost, st));
  const bool warm = ctx->aca_kstart.n >= (size_t)nf && ctx->aca_last_warm;
  if (warm) {
    BEM_CUDA_TRY(cudaMemcpyAsync(ks.data(), ctx->aca_kstart.p, nf * sizeof(int), cudaMemcpyDeviceToHost, st));
    BEM_CUDA_TRY(cudaMemcpyAsync(dn.data(), ctx->aca_done.p, nf * sizeof(int), cudaMemcpyDeviceToHost, st));
  }
  BEM_CUDA_TRY(cudaStreamSynchronize(st));
  for (int64_t b = 0; b < std::min(nmax, nf); ++b) {
    info[4 * b + 0] = ctx->far_h[b].nr;
    info[4 * b + 1] = ctx->far_h[b].nc;
    info[4 * b + 2] = rk[b];
    info[4 * b + 3] = warm ? (dn[b] ? rk[b] : ks[b]) : -1;
  }
  return BEM_OK;
}

extern "C" int bem_set_aca_reuse(bem_ctx* ctx, int on) {
  if (!ctx) return BEM_ERR_INVALID_ARG;
  ctx->aca_reuse = on != 0;
  return BEM_OK;
}

extern "C" int bem_block_tree(const double* centroid, const double* h, int64_t ne, int32_t leaf_size,
                              double eta_adm, int32_t dense, int32_t* perm, int64_t nmax, int32_t* near_blocks,
                              int32_t* far_blocks, int64_t* n_near, int64_t* n_far) {
  if (!centroid || !h || ne <= 0 || ne > 0x7fffffff || leaf_size < 1 || !(eta_adm > 0) || !n_near || !n_far ||
      nmax < 0 || (nmax > 0 && (!near_blocks || !far_blocks)))
    return BEM_ERR_INVALID_ARG;
  ClusterTree tr;
  build_cluster_tree(centroid, h, (int)ne, leaf_size, eta_adm, RHO2_NEAR, dense != 0, tr);
  *n_near = (int64_t)tr.near.size();
  *n_far = (int64_t)tr.far.size();
  if (perm)
    for (int64_t k = 0; k < ne; ++k) perm[k] = tr.perm[k];
  auto put = [&](const std::vector<BlockPair>& v, int32_t* out) {
    for (int64_t b = 0; b < std::min<int64_t>(nmax, (int64_t)v.size()); ++b) {
      const Cluster& t = tr.nodes[v[b].tau];
      const Cluster& s2 = tr.nodes[v[b].sigma];
      out[4 * b] = t.begin;
      out[4 * b + 1] = t.size();
      out[4 * b + 2] = s2.begin;
      out[4 * b + 3] = s2.size();
    }
  };
  if (nmax > 0) {
    put(tr.near, near_blocks);
    put(tr.far, far_blocks);
  }
  return BEM_OK;
}

extern "C" int bem_set_far_storage(bem_ctx* ctx, int32_t mode, int64_t workspace_bytes) {
  if (!ctx) return BEM_ERR_INVALID_ARG;
  if (mode < BEM_FAR_AUTO || mode > BEM_FAR_COMPACT) return fail(ctx, BEM_ERR_INVALID_ARG, "unknown storage mode");
  if (workspace_bytes < 0) return fail(ctx, BEM_ERR_INVALID_ARG, "workspace_bytes must be >= 0");
  ctx->far_mode_req = mode;
  ctx->far_ws_req = workspace_bytes;
  return BEM_OK;
}

extern "C" int bem_get_far_storage(bem_ctx* ctx, bem_far_storage* out) {
  if (!ctx || !out) return BEM_ERR_INVALID_ARG;
  *out = bem_far_storage{};
  if (!ctx->have_mesh) return fail(ctx, BEM_ERR_NO_MESH, "no mesh");
  TRY(set_device(ctx));
  const bool mixed = is_mixed(ctx);
  const long long esz = mixed ? 8 : 16;
  out->compact = ctx->far_compact ? 1 : 0;
  out->batches = (int32_t)ctx->far_batches.size();
  out->workspace_bytes = ctx->far_compact ? (long long)(mixed ? ctx->ws32.n : ctx->ws64.n) * esz : 0;
  out->factor_bytes = (long long)(mixed ? ctx->u32.n + ctx->v32.n : ctx->u64.n + ctx->v64.n) * esz;
  out->regrows = ctx->far_regrows;
  const size_t nf = ctx->far_h.size();
  if (ctx->assembled && nf) {
    std::vector<int> rk(nf);
    BEM_CUDA_TRY(cudaMemcpyAsync(rk.data(), ctx->rank.p, nf * sizeof(int), cudaMemcpyDeviceToHost, ctx->stream));
    BEM_CUDA_TRY(cudaStreamSynchronize(ctx->stream));
    long long used = 0;
    for (size_t b = 0; b < nf; ++b) used += 3LL * rk[b] * (ctx->far_h[b].nr + ctx->far_h[b].nc);
    out->used_bytes = used * esz;
  }
  return BEM_OK;
}

extern "C" int bem_get_profile(bem_ctx* ctx, bem_profile* out) {
  if (!ctx || !out) return BEM_ERR_INVALID_ARG;
  TRY(set_device(ctx));
  BEM_CUDA_TRY(cudaStreamSynchronize(ctx->stream));
  prof_harvest(ctx);
  std::vector<long long> lr(std::max(1, ctx->prof_nslots + 1), 0);
  if (ctx->prof_dev.p && ctx->prof_nslots + 1 > 0)
    BEM_CUDA_TRY(cudaMemcpy(lr.data(), ctx->prof_dev.p, lr.size() * sizeof(long long), cudaMemcpyDeviceToHost));
  double bytes = 0;
  for (const auto& d : ctx->prof_products) bytes += d.base + d.mult * (d.slot > 0 ? (double)lr[d.slot] : 0.0);
  out->hmv_launches = ctx->prof_hmv_launches;
  out->hmv_ms = ctx->prof_hmv_ms;
  out->hmv_bytes = bytes;
  out->assemble_calls = ctx->prof_asm_calls;
  out->assemble_ms = ctx->prof_asm_ms;
  out->kernel_launches = launch_count() - ctx->launches_at_reset;
  out->aca_blocks = ctx->prof_aca_blocks;
  out->aca_stepped = ctx->prof_aca_continued + (ctx->prof_dev.p ? lr[0] : 0);
  int fails = 0;
  if (ctx->assembled && ctx->aca_fail.p)
    BEM_CUDA_TRY(cudaMemcpy(&fails, ctx->aca_fail.p, sizeof(int), cudaMemcpyDeviceToHost));
  out->aca_failures = fails;
  return BEM_OK;
}

// ---------------------------------------------------------------------------
// several meshes in one context: batched sweeps
// ---------------------------------------------------------------------------
extern "C" int bem_add_mesh(bem_ctx* ctx, const double* xyz, int64_t nv, const int32_t* tri, int64_t ne,
                            const int8_t* bc_type, const bem_opts* opts, int32_t* mesh_id) {
  if (!ctx || !mesh_id) return BEM_ERR_INVALID_ARG;
  *mesh_id = -1;
  TRY(set_device(ctx));
  if (!ctx->batch_coop) BEM_CUDA_TRY(cudaStreamCreateWithFlags(&ctx->batch_coop, cudaStreamNonBlocking));
  cudaStream_t s = nullptr;
  BEM_CUDA_TRY(cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking));
  bem_ctx* child = nullptr;
  int rc = bem_create(&child, ctx->device, s);
  if (rc != BEM_OK) {
    cudaStreamDestroy(s);
    return fail(ctx, rc, "could not create the mesh's context");
  }
  rc = cudaEventCreateWithFlags(&child->coop_in, cudaEventDisableTiming) == cudaSuccess &&
               cudaEventCreateWithFlags(&child->coop_out, cudaEventDisableTiming) == cudaSuccess
           ? BEM_OK
           : BEM_ERR_CUDA;
  if (rc == BEM_OK) child->coop_stream = ctx->batch_coop;
  if (rc == BEM_OK && ctx->have_mat) rc = bem_set_material(child, ctx->E, ctx->nu, ctx->rho);
  if (rc == BEM_OK) rc = bem_set_far_storage(child, ctx->far_mode_req, ctx->far_ws_req);
  if (rc == BEM_OK) rc = bem_set_aca_reuse(child, ctx->aca_reuse ? 1 : 0);
  if (rc == BEM_OK) rc = bem_mesh(child, xyz, nv, tri, ne, bc_type, opts);
  if (rc != BEM_OK) {
    std::string msg = child->err;
    bem_destroy(child);
    cudaStreamDestroy(s);
    return fail(ctx, rc, "bem_add_mesh: " + msg);
  }
  ctx->batch.push_back(child);
  *mesh_id = (int32_t)(ctx->batch.size() - 1);
  return BEM_OK;
}

extern "C" int bem_mesh_count(const bem_ctx* ctx) { return ctx ? (int)ctx->batch.size() : BEM_ERR_INVALID_ARG; }

static int batch_child(bem_ctx* ctx, int32_t mesh_id, bem_ctx** out) {
  if (mesh_id < 0 || mesh_id >= (int32_t)ctx->batch.size()) return fail(ctx, BEM_ERR_INVALID_ARG, "unknown mesh id");
  *out = ctx->batch[mesh_id];
  return BEM_OK;
}

extern "C" int bem_solve_sweep_batched(bem_ctx* ctx, double T, int32_t n_omega, const double* load_hist,
                                       const double* const* bc_patterns, const bem_opts* opts,
                                       bem_freq_stats* stats) {
  if (!ctx || !load_hist || !bc_patterns) return BEM_ERR_INVALID_ARG;
  const int nm = (int)ctx->batch.size();
  if (!nm) return fail(ctx, BEM_ERR_NO_MESH, "no mesh added (bem_add_mesh)");
  if (!ctx->have_mat) return fail(ctx, BEM_ERR_STATE, "material not set");
  for (int i = 0; i < nm; ++i)
    if (!bc_patterns[i]) return fail(ctx, BEM_ERR_INVALID_ARG, "missing boundary pattern");
  TRY(set_device(ctx));
  for (bem_ctx* c : ctx->batch) {
    TRY(bem_set_material(c, ctx->E, ctx->nu, ctx->rho));
    TRY(bem_set_window(c, ctx->eta, ctx->window));
  }
  const int nf = n_omega / 2 + 1;
  for (bem_ctx* c : ctx->batch) c->mem_share = 1.0 / nm;  // the meshes' second operator sets share the memory
  std::vector<int> rc(nm, BEM_OK);
  // a bounded pool of host threads takes the meshes in turn
  const int hw = (int)std::thread::hardware_concurrency();
  const int nw = std::min(nm, std::max(1, std::min(16, hw > 0 ? hw : 16)));
  std::atomic<int> next{0};
  std::vector<std::thread> th;
  th.reserve(nw);
  for (int w = 0; w < nw; ++w)
    th.emplace_back([&]() {
      const bool dev_ok = cudaSetDevice(ctx->device) == cudaSuccess;
      for (int i = next.fetch_add(1); i < nm; i = next.fetch_add(1))
        rc[i] = dev_ok ? bem_solve_sweep(ctx->batch[i], T, n_omega, load_hist, bc_patterns[i], opts,
                                         stats ? stats + (long long)i * nf : nullptr)
                       : BEM_ERR_CUDA;
    });
  for (auto& t : th) t.join();
  int worst = BEM_OK;
  for (int i = 0; i < nm; ++i) {
    if (rc[i] == BEM_OK) continue;
    if (worst == BEM_OK || worst == BEM_ERR_NOT_CONVERGED) {
      worst = rc[i];
      fail(ctx, rc[i], "mesh " + std::to_string(i) + ": " + ctx->batch[i]->err);
    }
  }
  return worst;
}

extern "C" int bem_mesh_frequency_solution(bem_ctx* ctx, int32_t mesh_id, int32_t k, double* out) {
  if (!ctx) return BEM_ERR_INVALID_ARG;
  bem_ctx* c = nullptr;
  TRY(batch_child(ctx, mesh_id, &c));
  int rc = bem_get_frequency_solution(c, k, out);
  if (rc != BEM_OK) fail(ctx, rc, c->err);
  return rc;
}

extern "C" int bem_mesh_time_response(bem_ctx* ctx, int32_t mesh_id, const int64_t* dofs, int64_t ndof,
                                      double* out) {
  if (!ctx) return BEM_ERR_INVALID_ARG;
  bem_ctx* c = nullptr;
  TRY(batch_child(ctx, mesh_id, &c));
  int rc = bem_time_response(c, dofs, ndof, out);
  if (rc != BEM_OK) fail(ctx, rc, c->err);
  return rc;
}

// ---------------------------------------------------------------------------
// interior field (representation formula; the paper's Sec. 5.2 example
// reports strain at a point inside the solid)
// ---------------------------------------------------------------------------
static int interior_checks(bem_ctx* ctx, int64_t npts, int quantity, double h) {
  if (ctx->nf == 0) return fail(ctx, BEM_ERR_STATE, "the sweep has not been solved");
  if (npts < 0 || npts > (1LL << 24)) return fail(ctx, BEM_ERR_INVALID_ARG, "npts must be in 0..2^24");
  if (quantity != BEM_FIELD_DISPLACEMENT && quantity != BEM_FIELD_STRAIN)
    return fail(ctx, BEM_ERR_INVALID_ARG, "unknown interior quantity");
  if (quantity == BEM_FIELD_STRAIN && !(h > 0 && std::isfinite(h)))
    return fail(ctx, BEM_ERR_INVALID_ARG, "strain needs a difference step h > 0");
  return BEM_OK;
}

// quantity at npts device points for solved frequency k into out_dev
// (npts x 3 or npts x 6 complex)
static int interior_eval(bem_ctx* ctx, int k, const double* pts_dev, int npts, int quantity, double h,
                         c128* out_dev, DevBuf<double>& offs, DevBuf<c128>& uoff) {
  cudaStream_t st = ctx->stream;
  const c128* a = ctx->sol.p + (long long)k * ctx->N;
  const c128 pk = ctx->Pk_host[k];
  const double sre = ctx->eta, sim = k * 2.0 * M_PI / ctx->T;
  const double* p = pts_dev;
  int n = npts;
  c128* o = out_dev;
  if (quantity == BEM_FIELD_STRAIN) {
    BEM_CUDA_TRY(offs.ensure(18LL * npts));
    BEM_CUDA_TRY(uoff.ensure(18LL * npts));
    launch_offset_points(pts_dev, npts, h, offs.p, st);
    p = offs.p;
    n = 6 * npts;
    o = uoff.p;
  }
  if (is_mixed(ctx))
    launch_interior<float>(p, n, ctx->ed.p, ctx->ne, ctx->bc.p, a, ctx->pattern.p, pk,
                           make_params<float>(ctx, sre, sim), o, st);
  else
    launch_interior<double>(p, n, ctx->ed.p, ctx->ne, ctx->bc.p, a, ctx->pattern.p, pk,
                            make_params<double>(ctx, sre, sim), o, st);
  CK("interior");
  if (quantity == BEM_FIELD_STRAIN) {
    launch_strain(uoff.p, npts, h, out_dev, st);
    CK("strain");
  }
  return BEM_OK;
}

static int interior_frequency(bem_ctx* ctx, int32_t k, const double* points, int64_t npts, int quantity, double h,
                              double* out) {
  if (!ctx || (npts > 0 && (!points || !out))) return BEM_ERR_INVALID_ARG;
  TRY(interior_checks(ctx, npts, quantity, h));
  if (k < 0 || k >= ctx->nf) return fail(ctx, BEM_ERR_INVALID_ARG, "frequency index not solved");
  TRY(set_device(ctx));
  if (npts == 0) return BEM_OK;
  const int nc = quantity == BEM_FIELD_STRAIN ? 6 : 3;
  DevBuf<double> pts, offs;
  DevBuf<c128> res, uoff;
  BEM_CUDA_TRY(pts.alloc(3 * npts));
  BEM_CUDA_TRY(res.alloc(nc * npts));
  BEM_CUDA_TRY(cudaMemcpyAsync(pts.p, points, 3 * npts * sizeof(double), cudaMemcpyHostToDevice, ctx->stream));
  TRY(interior_eval(ctx, k, pts.p, (int)npts, quantity, h, res.p, offs, uoff));
  BEM_CUDA_TRY(cudaMemcpyAsync(out, res.p, nc * npts * sizeof(c128), cudaMemcpyDeviceToHost, ctx->stream));
  BEM_CUDA_TRY(cudaStreamSynchronize(ctx->stream));
  return BEM_OK;
}

extern "C" int bem_interior_field(bem_ctx* ctx, int32_t k, const double* points, int64_t npts, double* out) {
  return interior_frequency(ctx, k, points, npts, BEM_FIELD_DISPLACEMENT, 0.0, out);
}

extern "C" int bem_interior_strain(bem_ctx* ctx, int32_t k, const double* points, int64_t npts, double h,
                                   double* out) {
  return interior_frequency(ctx, k, points, npts, BEM_FIELD_STRAIN, h, out);
}

extern "C" int bem_interior_time_response(bem_ctx* ctx, const double* points, int64_t npts, int32_t quantity,
                                          double h, double* out) {
  if (!ctx || (npts > 0 && (!points || !out))) return BEM_ERR_INVALID_ARG;
  TRY(interior_checks(ctx, npts, quantity, h));
  if (ctx->nf != ctx->n_omega / 2 + 1) return fail(ctx, BEM_ERR_STATE, "the sweep has not been solved");
  TRY(set_device(ctx));
  if (npts == 0) return BEM_OK;
  const long long nc = (quantity == BEM_FIELD_STRAIN ? 6 : 3) * npts;
  DevBuf<double> pts, offs, o;
  DevBuf<c128> spec, uoff;
  BEM_CUDA_TRY(pts.alloc(3 * npts));
  BEM_CUDA_TRY(spec.alloc((long long)ctx->nf * nc));
  BEM_CUDA_TRY(o.alloc((long long)ctx->n_omega * nc));
  BEM_CUDA_TRY(cudaMemcpyAsync(pts.p, points, 3 * npts * sizeof(double), cudaMemcpyHostToDevice, ctx->stream));
  for (int k = 0; k < ctx->nf; ++k)
    TRY(interior_eval(ctx, k, pts.p, (int)npts, quantity, h, spec.p + (long long)k * nc, offs, uoff));
  launch_idft(spec.p, nc, nullptr, nc, ctx->n_omega, ctx->T, ctx->eta, ctx->window, o.p, ctx->stream);
  CK("interior idft");
  BEM_CUDA_TRY(cudaMemcpyAsync(out, o.p, (long long)ctx->n_omega * nc * sizeof(double), cudaMemcpyDeviceToHost,
                               ctx->stream));
  BEM_CUDA_TRY(cudaStreamSynchronize(ctx->stream));
  return BEM_OK;
}
