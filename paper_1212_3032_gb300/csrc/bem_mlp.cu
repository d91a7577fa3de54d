// Learned initial guess: a pointwise network that proposes the next
// frequency's solution value of every unknown from its four previous values.
//
// The paper's solution extrapolation (Sec. 4.2) fits a_k^(0) = X s in the span
// of the previous solutions; the learned proposal p_k is added to that span as
// one more column, so the least-squares guess can only get better.
//
//   features (10): a_{k-1..k-4}(d) / S (re, im), eta dt, Im(s_k) dt,
//                  S = max_d |a_{k-1}(d)|
//   x -> tanh(W1 x + b1) (256) -> tanh(W2 h1 + b2) (256) -> W3 h2 + b3 (2)
//   proposal p_k(d) = S (y0 + i y1)
//
// Weight matrices are used as BF16 (rounded from FP32 master weights after
// every update) with FP32 accumulation; training is Adam on the mean squared
// error, run on the device after each solved frequency (online).
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <random>
#include <vector>

#include <cuda_bf16.h>

#include "bem_internal.h"
#include "bem_launch.h"

namespace bem {

namespace {

constexpr int TILE = 64;
constexpr int KCH = 16;

// C[m][n] = sum_k A(m,k) B(k,n) with A(m,k) = A[m*sam + k*sak], B(k,n) =
// B[k*sbk + n*sbn] (B float or bf16), FP32 accumulation, epilogue:
//   mode 0: C = acc
//   mode 1: C = tanh(acc + bias[n])
//   mode 2: C = acc + bias[n]
//   mode 3: C = acc * (1 - H[m][n]^2)       (tanh derivative, H row-major ldh)
//
// Split-K: CTA z covers k in [z kchunk, (z + 1) kchunk) and writes its partial
// product to C + z cz (mode 0 only); k_sum_splits adds the partials in order.
template <typename TB>
__global__ void __launch_bounds__(256) k_gemm(int M, int N, int K, const float* __restrict__ A, long long sam,
                                              long long sak, const TB* __restrict__ B, long long sbk, long long sbn,
                                              float* __restrict__ C, long long ldc, const float* __restrict__ bias,
                                              const float* __restrict__ H, long long ldh, int mode, int kchunk,
                                              long long cz) {
  __shared__ float As[KCH][TILE + 1];
  __shared__ float Bs[KCH][TILE + 1];
  const int tm = blockIdx.y * TILE, tn = blockIdx.x * TILE;
  const int tx = threadIdx.x % 16, ty = threadIdx.x / 16;  // 4x4 outputs per thread
  const int kb = blockIdx.z * kchunk, ke = min(K, kb + kchunk);
  C += blockIdx.z * cz;
  float acc[4][4] = {};
  for (int k0 = kb; k0 < ke; k0 += KCH) {
    // the unit-stride index runs fastest across the threads (coalesced loads)
    for (int i = threadIdx.x; i < KCH * TILE; i += blockDim.x) {
      int kk = sak == 1 ? i % KCH : i / TILE, mm = sak == 1 ? i / KCH : i % TILE;
      long long gm = tm + mm, gk = k0 + kk;
      As[kk][mm] = (gm < M && gk < ke) ? A[gm * sam + gk * sak] : 0.f;
    }
    for (int i = threadIdx.x; i < KCH * TILE; i += blockDim.x) {
      int kk = sbk == 1 ? i % KCH : i / TILE, nn = sbk == 1 ? i / KCH : i % TILE;
      long long gn = tn + nn, gk = k0 + kk;
      Bs[kk][nn] = (gn < N && gk < ke) ? float(B[gk * sbk + gn * sbn]) : 0.f;
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < KCH; ++kk) {
      float a[4], b[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        a[i] = As[kk][ty * 4 + i];
        b[i] = Bs[kk][tx * 4 + i];
      }
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = fmaf(a[i], b[j], acc[i][j]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      int gm = tm + ty * 4 + i, gn = tn + tx * 4 + j;
      if (gm >= M || gn >= N) continue;
      float v = acc[i][j];
      if (mode == 1) v = tanhf(v + bias[gn]);
      else if (mode == 2) v = v + bias[gn];
      else if (mode == 3) {
        float h = H[(long long)gm * ldh + gn];
        v = v * (1.f - h * h);
      }
      C[(long long)gm * ldc + gn] = v;
    }
}

__global__ void k_sum_splits(long long n, int splits, const float* __restrict__ part, float* __restrict__ out) {
  long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (i >= n) return;
  float s = 0.f;
  for (int z = 0; z < splits; ++z) s += part[z * n + i];
  out[i] = s;
}

template <typename TB>
void gemm(int M, int N, int K, const float* A, long long sam, long long sak, const TB* B, long long sbk, long long sbn,
          float* C, long long ldc, const float* bias, const float* H, long long ldh, int mode, cudaStream_t st) {
  dim3 grid((N + TILE - 1) / TILE, (M + TILE - 1) / TILE, 1);
  count_if(true);
  k_gemm<TB><<<grid, 256, 0, st>>>(M, N, K, A, sam, sak, B, sbk, sbn, C, ldc, bias, H, ldh, mode, K, 0);
}

// Weight gradient C (M x N, row-major, ldc = N) = A^T-style product over a
// long K (the batch): split over K so that enough CTAs run, partials summed
// in a fixed order (run-to-run deterministic).
constexpr int SPLIT_K = 512;
void gemm_splitk(int M, int N, int K, const float* A, long long sam, long long sak, const float* B, long long sbk,
                 long long sbn, float* C, float* part, cudaStream_t st) {
  int splits = std::max(1, (K + SPLIT_K - 1) / SPLIT_K);
  dim3 grid((N + TILE - 1) / TILE, (M + TILE - 1) / TILE, splits);
  count_if(true);
  k_gemm<float><<<grid, 256, 0, st>>>(M, N, K, A, sam, sak, B, sbk, sbn, part, N, nullptr, nullptr, 0, 0, SPLIT_K,
                                      (long long)M * N);
  long long n = (long long)M * N;
  count_if(true);
  k_sum_splits<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(n, splits, part, C);
}

// column sums: out[n] = sum_m D[m][n]  (bias gradients)
__global__ void k_colsum(int M, int N, const float* __restrict__ D, float* __restrict__ out) {
  int n = blockIdx.x;
  float s = 0.f;
  for (int m = threadIdx.x; m < M; m += blockDim.x) s += D[(long long)m * N + n];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  __shared__ float w[8];
  if ((threadIdx.x & 31) == 0) w[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    float t = 0.f;
    for (int i = 0; i < (int)(blockDim.x >> 5); ++i) t += w[i];
    out[n] = t;
  }
}

// D3 = 2 (Y - T) / B ; partial squared error sums
__global__ void k_out_delta(int B, const float* __restrict__ Y, const float* __restrict__ T, float* __restrict__ D,
                            double* __restrict__ loss) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  float e = 0.f;
  if (i < 2 * B) {
    float d = Y[i] - T[i];
    D[i] = 2.f * d / B;
    e = d * d;
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) e += __shfl_xor_sync(0xffffffffu, e, o);
  if ((threadIdx.x & 31) == 0 && e != 0.f) atomicAdd(loss, (double)e / B);
}

__global__ void k_adam(long long n, float* __restrict__ th, const float* __restrict__ g, float* __restrict__ m,
                       float* __restrict__ v, float lr, float b1, float b2, float c1, float c2, float eps) {
  long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (i >= n) return;
  float gi = g[i];
  float mi = b1 * m[i] + (1.f - b1) * gi;
  float vi = b2 * v[i] + (1.f - b2) * gi * gi;
  m[i] = mi;
  v[i] = vi;
  th[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
}

__global__ void k_to_bf16(long long n, const float* __restrict__ a, __nv_bfloat16* __restrict__ b) {
  long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (i < n) b[i] = __float2bfloat16_rn(a[i]);
}

// S = max |a| over a complex128 vector (nonnegative doubles compare as integers)
__global__ void k_maxabs(const c128* __restrict__ a, long long n, unsigned long long* __restrict__ out) {
  double mx = 0;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    mx = fmax(mx, sqrt(a[i].re * a[i].re + a[i].im * a[i].im));
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, o));
  if ((threadIdx.x & 31) == 0) atomicMax(out, (unsigned long long)__double_as_longlong(mx));
}

// features of every unknown from a_{k-1..k-4} (rows of sol), and optional targets from a_k
__global__ void k_features(const c128* __restrict__ a1, const c128* __restrict__ a2, const c128* __restrict__ a3,
                           const c128* __restrict__ a4, const c128* __restrict__ ak, long long n,
                           const unsigned long long* __restrict__ smax, float sre_dt, float sim_dt,
                           float* __restrict__ X, float* __restrict__ T) {
  long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (i >= n) return;
  double S = __longlong_as_double((long long)*smax);
  double is = S > 0 ? 1.0 / S : 1.0;
  float* x = X + 10 * i;
  const c128* a[4] = {a1, a2, a3, a4};
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    x[2 * j] = float(a[j][i].re * is);
    x[2 * j + 1] = float(a[j][i].im * is);
  }
  x[8] = sre_dt;
  x[9] = sim_dt;
  if (T) {
    T[2 * i] = float(ak[i].re * is);
    T[2 * i + 1] = float(ak[i].im * is);
  }
}

__global__ void k_proposal(const float* __restrict__ Y, long long n, const unsigned long long* __restrict__ smax,
                           c128* __restrict__ p) {
  long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (i >= n) return;
  double S = __longlong_as_double((long long)*smax);
  if (!(S > 0)) S = 1.0;
  p[i] = c128{S * Y[2 * i], S * Y[2 * i + 1]};
}

constexpr int IN = 10, HID = 256, OUT = 2;
constexpr long long OW1 = 0, OB1 = OW1 + HID * IN, OW2 = OB1 + HID, OB2 = OW2 + HID * HID, OW3 = OB2 + HID,
                    OB3 = OW3 + OUT * HID, NPAR = OB3 + OUT;

}  // namespace

// ---------------------------------------------------------------------------
// device state
// ---------------------------------------------------------------------------
struct MlpState {
  DevBuf<float> theta, grad, m, v;
  DevBuf<__nv_bfloat16> w16;  // BF16 copy of the whole parameter vector (matrices used from it)
  DevBuf<float> X, H1, H2, Y, T, D3, D2, D1;
  DevBuf<float> kpart;  // split-K partial products of the weight gradients
  DevBuf<c128> prop;    // proposal of the current frequency (tree order)
  DevBuf<double> loss;
  DevBuf<unsigned long long> smax;
  long long cap = 0;
  long long step = 0;
  bool ready = false;
};

static MlpState* mlp_of(bem_ctx* ctx) {
  if (!ctx->mlp) ctx->mlp = new MlpState();
  return ctx->mlp;
}

void mlp_free(bem_ctx* ctx) {
  delete ctx->mlp;
  ctx->mlp = nullptr;
}

static int mlp_ensure(bem_ctx* ctx, long long B) {
  MlpState* s = mlp_of(ctx);
  if (B <= s->cap) return BEM_OK;
  long long c = std::max<long long>(B, 1024);
  BEM_CUDA_TRY(s->X.alloc(10 * c));
  BEM_CUDA_TRY(s->H1.alloc(HID * c));
  BEM_CUDA_TRY(s->H2.alloc(HID * c));
  BEM_CUDA_TRY(s->Y.alloc(2 * c));
  BEM_CUDA_TRY(s->T.alloc(2 * c));
  BEM_CUDA_TRY(s->D3.alloc(2 * c));
  BEM_CUDA_TRY(s->D2.alloc(HID * c));
  BEM_CUDA_TRY(s->D1.alloc(HID * c));
  BEM_CUDA_TRY(s->kpart.alloc((long long)((c + SPLIT_K - 1) / SPLIT_K) * HID * HID));
  s->cap = c;
  return BEM_OK;
}

static int mlp_sync_bf16(bem_ctx* ctx) {
  MlpState* s = mlp_of(ctx);
  count_if(true);
  k_to_bf16<<<(unsigned)((NPAR + 255) / 256), 256, 0, ctx->stream>>>(NPAR, s->theta.p, s->w16.p);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return fail_cuda(ctx, e, "mlp bf16", __FILE__, __LINE__);
  return BEM_OK;
}

static int mlp_set_host(bem_ctx* ctx, const float* th) {
  MlpState* s = mlp_of(ctx);
  BEM_CUDA_TRY(s->theta.ensure(NPAR));
  BEM_CUDA_TRY(s->grad.ensure(NPAR));
  BEM_CUDA_TRY(s->m.ensure(NPAR));
  BEM_CUDA_TRY(s->v.ensure(NPAR));
  BEM_CUDA_TRY(s->w16.ensure(NPAR));
  BEM_CUDA_TRY(s->loss.ensure(1));
  BEM_CUDA_TRY(s->smax.ensure(1));
  BEM_CUDA_TRY(cudaMemcpyAsync(s->theta.p, th, NPAR * sizeof(float), cudaMemcpyHostToDevice, ctx->stream));
  BEM_CUDA_TRY(cudaMemsetAsync(s->m.p, 0, NPAR * sizeof(float), ctx->stream));
  BEM_CUDA_TRY(cudaMemsetAsync(s->v.p, 0, NPAR * sizeof(float), ctx->stream));
  s->step = 0;
  int r = mlp_sync_bf16(ctx);
  if (r != BEM_OK) return r;
  BEM_CUDA_TRY(cudaStreamSynchronize(ctx->stream));
  s->ready = true;
  return BEM_OK;
}

static int mlp_init_seed(bem_ctx* ctx, unsigned long long seed) {
  std::vector<float> th(NPAR, 0.f);
  std::mt19937_64 rng(seed);
  auto fill = [&](long long off, int fan_out, int fan_in) {
    // Glorot-uniform initialisation
    float a = std::sqrt(6.0f / float(fan_in + fan_out));
    std::uniform_real_distribution<float> U(-a, a);
    for (long long i = 0; i < (long long)fan_out * fan_in; ++i) th[off + i] = U(rng);
  };
  fill(OW1, HID, IN);
  fill(OW2, HID, HID);
  fill(OW3, OUT, HID);
  return mlp_set_host(ctx, th.data());
}

// forward over B samples already in s->X: H1, H2, Y
static void mlp_forward_dev(bem_ctx* ctx, long long B) {
  MlpState* s = mlp_of(ctx);
  cudaStream_t st = ctx->stream;
  const __nv_bfloat16* w = s->w16.p;
  gemm<__nv_bfloat16>((int)B, HID, IN, s->X.p, IN, 1, w + OW1, 1, IN, s->H1.p, HID, s->theta.p + OB1, nullptr, 0, 1, st);
  gemm<__nv_bfloat16>((int)B, HID, HID, s->H1.p, HID, 1, w + OW2, 1, HID, s->H2.p, HID, s->theta.p + OB2, nullptr, 0, 1,
                      st);
  gemm<__nv_bfloat16>((int)B, OUT, HID, s->H2.p, HID, 1, w + OW3, 1, HID, s->Y.p, OUT, s->theta.p + OB3, nullptr, 0, 2,
                      st);
}

// backward over B samples (targets in s->T): gradient into s->grad, loss into s->loss
static void mlp_backward_dev(bem_ctx* ctx, long long B) {
  MlpState* s = mlp_of(ctx);
  cudaStream_t st = ctx->stream;
  const __nv_bfloat16* w = s->w16.p;
  cudaMemsetAsync(s->loss.p, 0, sizeof(double), st);
  count_if(true);
  k_out_delta<<<(unsigned)((2 * B + 255) / 256), 256, 0, st>>>((int)B, s->Y.p, s->T.p, s->D3.p, s->loss.p);
  float* g = s->grad.p;
  // dW3 = D3^T H2 ; db3
  gemm_splitk(OUT, HID, (int)B, s->D3.p, 1, OUT, s->H2.p, HID, 1, g + OW3, s->kpart.p, st);
  count_if(true);
  k_colsum<<<OUT, 256, 0, st>>>((int)B, OUT, s->D3.p, g + OB3);
  // D2 = (D3 W3) * (1 - H2^2)
  gemm<__nv_bfloat16>((int)B, HID, OUT, s->D3.p, OUT, 1, w + OW3, HID, 1, s->D2.p, HID, nullptr, s->H2.p, HID, 3, st);
  gemm_splitk(HID, HID, (int)B, s->D2.p, 1, HID, s->H1.p, HID, 1, g + OW2, s->kpart.p, st);
  count_if(true);
  k_colsum<<<HID, 256, 0, st>>>((int)B, HID, s->D2.p, g + OB2);
  // D1 = (D2 W2) * (1 - H1^2)
  gemm<__nv_bfloat16>((int)B, HID, HID, s->D2.p, HID, 1, w + OW2, HID, 1, s->D1.p, HID, nullptr, s->H1.p, HID, 3, st);
  gemm_splitk(HID, IN, (int)B, s->D1.p, 1, HID, s->X.p, IN, 1, g + OW1, s->kpart.p, st);
  count_if(true);
  k_colsum<<<HID, 256, 0, st>>>((int)B, HID, s->D1.p, g + OB1);
}

static void mlp_adam_dev(bem_ctx* ctx, float lr) {
  MlpState* s = mlp_of(ctx);
  s->step += 1;
  const float b1 = 0.9f, b2 = 0.999f;
  float c1 = 1.f - std::pow(b1, (float)s->step), c2 = 1.f - std::pow(b2, (float)s->step);
  count_if(true);
  k_adam<<<(unsigned)((NPAR + 255) / 256), 256, 0, ctx->stream>>>(NPAR, s->theta.p, s->grad.p, s->m.p, s->v.p, lr, b1,
                                                                  b2, c1, c2, 1e-8f);
  mlp_sync_bf16(ctx);
}

// ---------------------------------------------------------------------------
// hooks used by the sweep
// ---------------------------------------------------------------------------
int mlp_ready(bem_ctx* ctx) {
  if (!ctx->mlp || !ctx->mlp->ready) return mlp_init_seed(ctx, 3032);
  return BEM_OK;
}

// proposal for frequency k from sol rows k-1..k-4 (tree order); *out points
// to it (device, N values) until the next call
int mlp_propose(bem_ctx* ctx, const c128* const* prev, double sre_dt, double sim_dt, const c128** out) {
  const long long N = ctx->N;
  int r = mlp_ready(ctx);
  if (r == BEM_OK) r = mlp_ensure(ctx, N);
  if (r != BEM_OK) return r;
  MlpState* s = ctx->mlp;
  BEM_CUDA_TRY(s->prop.ensure(N));
  c128* p = s->prop.p;
  *out = p;
  if (r != BEM_OK) return r;
  cudaStream_t st = ctx->stream;
  BEM_CUDA_TRY(cudaMemsetAsync(s->smax.p, 0, sizeof(unsigned long long), st));
  count_if(true);
  k_maxabs<<<64, 256, 0, st>>>(prev[0], N, s->smax.p);
  count_if(true);
  k_features<<<(unsigned)((N + 255) / 256), 256, 0, st>>>(prev[0], prev[1], prev[2], prev[3], nullptr, N, s->smax.p,
                                                          (float)sre_dt, (float)sim_dt, s->X.p, nullptr);
  mlp_forward_dev(ctx, N);
  count_if(true);
  k_proposal<<<(unsigned)((N + 255) / 256), 256, 0, st>>>(s->Y.p, N, s->smax.p, p);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return fail_cuda(ctx, e, "mlp propose", __FILE__, __LINE__);
  return BEM_OK;
}

// online training on frequency k: inputs from rows k-1..k-4, target row k
int mlp_train(bem_ctx* ctx, const c128* const* prev, const c128* ak, double sre_dt, double sim_dt, int steps,
              double lr) {
  if (steps <= 0) return BEM_OK;
  const long long N = ctx->N;
  int r = mlp_ready(ctx);
  if (r == BEM_OK) r = mlp_ensure(ctx, N);
  if (r != BEM_OK) return r;
  MlpState* s = ctx->mlp;
  cudaStream_t st = ctx->stream;
  BEM_CUDA_TRY(cudaMemsetAsync(s->smax.p, 0, sizeof(unsigned long long), st));
  count_if(true);
  k_maxabs<<<64, 256, 0, st>>>(prev[0], N, s->smax.p);
  count_if(true);
  k_features<<<(unsigned)((N + 255) / 256), 256, 0, st>>>(prev[0], prev[1], prev[2], prev[3], ak, N, s->smax.p,
                                                          (float)sre_dt, (float)sim_dt, s->X.p, s->T.p);
  for (int i = 0; i < steps; ++i) {
    mlp_forward_dev(ctx, N);
    mlp_backward_dev(ctx, N);
    mlp_adam_dev(ctx, (float)lr);
  }
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return fail_cuda(ctx, e, "mlp train", __FILE__, __LINE__);
  return BEM_OK;
}

}  // namespace bem

using namespace bem;

// ---------------------------------------------------------------------------
// C-ABI
// ---------------------------------------------------------------------------
extern "C" int64_t bem_mlp_num_params(void) { return NPAR; }

extern "C" int bem_mlp_init(bem_ctx* ctx, uint64_t seed) {
  if (!ctx) return BEM_ERR_INVALID_ARG;
  BEM_CUDA_TRY(cudaSetDevice(ctx->device));
  return mlp_init_seed(ctx, seed);
}

extern "C" int bem_mlp_set_training(bem_ctx* ctx, int32_t steps_per_frequency, double lr) {
  if (!ctx || steps_per_frequency < 0 || !(lr >= 0) || !std::isfinite(lr)) return BEM_ERR_INVALID_ARG;
  ctx->mlp_steps = steps_per_frequency;
  ctx->mlp_lr = lr;
  return BEM_OK;
}

extern "C" int bem_mlp_set_weights(bem_ctx* ctx, const float* theta, int64_t n) {
  if (!ctx || !theta || n != NPAR) return BEM_ERR_INVALID_ARG;
  BEM_CUDA_TRY(cudaSetDevice(ctx->device));
  return mlp_set_host(ctx, theta);
}

extern "C" int bem_mlp_get_weights(bem_ctx* ctx, float* theta, int64_t n) {
  if (!ctx || !theta || n != NPAR) return BEM_ERR_INVALID_ARG;
  BEM_CUDA_TRY(cudaSetDevice(ctx->device));
  int r = mlp_ready(ctx);
  if (r != BEM_OK) return r;
  BEM_CUDA_TRY(cudaMemcpyAsync(theta, ctx->mlp->theta.p, NPAR * sizeof(float), cudaMemcpyDeviceToHost, ctx->stream));
  BEM_CUDA_TRY(cudaStreamSynchronize(ctx->stream));
  return BEM_OK;
}

extern "C" int bem_mlp_forward(bem_ctx* ctx, const float* x, int64_t B, float* y) {
  if (!ctx || B < 0 || (B > 0 && (!x || !y))) return BEM_ERR_INVALID_ARG;
  if (B == 0) return BEM_OK;
  BEM_CUDA_TRY(cudaSetDevice(ctx->device));
  int r = mlp_ready(ctx);
  if (r == BEM_OK) r = mlp_ensure(ctx, B);
  if (r != BEM_OK) return r;
  MlpState* s = ctx->mlp;
  BEM_CUDA_TRY(cudaMemcpyAsync(s->X.p, x, B * IN * sizeof(float), cudaMemcpyHostToDevice, ctx->stream));
  mlp_forward_dev(ctx, B);
  BEM_CUDA_TRY(cudaGetLastError());
  BEM_CUDA_TRY(cudaMemcpyAsync(y, s->Y.p, B * OUT * sizeof(float), cudaMemcpyDeviceToHost, ctx->stream));
  BEM_CUDA_TRY(cudaStreamSynchronize(ctx->stream));
  return BEM_OK;
}

static int mlp_grad_host(bem_ctx* ctx, const float* x, const float* t, int64_t B, double* loss) {
  int r = mlp_ready(ctx);
  if (r == BEM_OK) r = mlp_ensure(ctx, B);
  if (r != BEM_OK) return r;
  MlpState* s = ctx->mlp;
  BEM_CUDA_TRY(cudaMemcpyAsync(s->X.p, x, B * IN * sizeof(float), cudaMemcpyHostToDevice, ctx->stream));
  BEM_CUDA_TRY(cudaMemcpyAsync(s->T.p, t, B * OUT * sizeof(float), cudaMemcpyHostToDevice, ctx->stream));
  mlp_forward_dev(ctx, B);
  mlp_backward_dev(ctx, B);
  BEM_CUDA_TRY(cudaGetLastError());
  if (loss) BEM_CUDA_TRY(cudaMemcpyAsync(loss, s->loss.p, sizeof(double), cudaMemcpyDeviceToHost, ctx->stream));
  return BEM_OK;
}

extern "C" int bem_mlp_gradient(bem_ctx* ctx, const float* x, const float* t, int64_t B, float* grad, double* loss) {
  if (!ctx || B <= 0 || !x || !t || !grad) return BEM_ERR_INVALID_ARG;
  BEM_CUDA_TRY(cudaSetDevice(ctx->device));
  int r = mlp_grad_host(ctx, x, t, B, loss);
  if (r != BEM_OK) return r;
  BEM_CUDA_TRY(cudaMemcpyAsync(grad, ctx->mlp->grad.p, NPAR * sizeof(float), cudaMemcpyDeviceToHost, ctx->stream));
  BEM_CUDA_TRY(cudaStreamSynchronize(ctx->stream));
  return BEM_OK;
}

extern "C" int bem_mlp_train_step(bem_ctx* ctx, const float* x, const float* t, int64_t B, double lr, double* loss) {
  if (!ctx || B <= 0 || !x || !t || !(lr >= 0)) return BEM_ERR_INVALID_ARG;
  BEM_CUDA_TRY(cudaSetDevice(ctx->device));
  int r = mlp_grad_host(ctx, x, t, B, loss);
  if (r != BEM_OK) return r;
  mlp_adam_dev(ctx, (float)lr);
  BEM_CUDA_TRY(cudaGetLastError());
  BEM_CUDA_TRY(cudaStreamSynchronize(ctx->stream));
  return BEM_OK;
}
