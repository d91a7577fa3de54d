// y = A x with the assembled operator for callers that cannot allocate
// device memory during the call.
//
// Some callers own all of the device's memory through their own allocator
// (a caching pool that reserved the device up front) and cannot let a library
// call cudaMalloc behind its back; others run under hard latency bounds where
// the implicit device synchronisation of cudaMalloc/cudaFree is not
// acceptable. bem_apply_noalloc serves them: its scratch (the permuted input
// and output vectors, the V^T x values of the low-rank blocks and the partial
// row sums of the product) lives in one file-scope device array of fixed size,
// and the call allocates nothing.
//
// The array's host-side name is only a stand-in for the device object, so its
// device address is looked up once per device with cudaGetSymbolAddress (with
// that device current) on the first call made on that device.
#include <mutex>

#include "bem_internal.h"
#include "bem_launch.h"

namespace {

constexpr size_t NOALLOC_SCRATCH_BYTES = size_t(32) << 20;  // 32 MiB, held by every GPU that loads the library
constexpr int NOALLOC_MAX_DEVICES = 64;

__device__ __align__(256) unsigned char g_noalloc_scratch[NOALLOC_SCRATCH_BYTES];

std::mutex g_noalloc_mu;
void* g_noalloc_addr[NOALLOC_MAX_DEVICES] = {};

size_t round256(size_t b) { return (b + 255) & ~size_t(255); }

__global__ void k_noalloc_gather(const bem::c64* __restrict__ x, const int* __restrict__ perm, int ne,
                                 bem::c64* __restrict__ xt) {
  int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= ne) return;
  long long e = perm[k];
  for (int a = 0; a < 3; ++a) xt[3LL * k + a] = x[3 * e + a];
}

__global__ void k_noalloc_scatter(const bem::c64* __restrict__ yt, const int* __restrict__ perm, int ne,
                                  bem::c64* __restrict__ y) {
  int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= ne) return;
  long long e = perm[k];
  for (int a = 0; a < 3; ++a) y[3 * e + a] = yt[3LL * k + a];
}

}  // namespace

extern "C" int bem_apply_noalloc(bem_ctx* ctx, const float* x_dev, float* y_dev) {
  using namespace bem;
  if (!ctx || !x_dev || !y_dev) return BEM_ERR_INVALID_ARG;
  if (!ctx->assembled) return fail(ctx, BEM_ERR_STATE, "operator not assembled");
  if (ctx->prec != BEM_PREC_C64_MIXED)
    return fail(ctx, BEM_ERR_STATE, "bem_apply_noalloc needs the complex64 (mixed precision) operator");
  if (ctx->device < 0 || ctx->device >= NOALLOC_MAX_DEVICES)
    return fail(ctx, BEM_ERR_INVALID_ARG, "device ordinal beyond the supported range");
  const long long N = ctx->N;
  const size_t bx = round256(sizeof(c64) * (size_t)N);
  const size_t bt = round256(sizeof(c64) * (size_t)std::max(1, ctx->t_entries));
  const size_t bp = round256(sizeof(c64) * (size_t)std::max<long long>(1, ctx->part_rows));
  const size_t need = 2 * bx + bt + bp;
  if (need > NOALLOC_SCRATCH_BYTES) {
    char msg[256];
    snprintf(msg, sizeof(msg), "bem_apply_noalloc needs %zu bytes of scratch for this operator; the maximum is %zu",
             need, NOALLOC_SCRATCH_BYTES);
    return fail(ctx, BEM_ERR_INVALID_ARG, msg);
  }
  BEM_CUDA_TRY(cudaSetDevice(ctx->device));
  void* base = nullptr;
  {
    std::lock_guard<std::mutex> lock(g_noalloc_mu);
    if (!g_noalloc_addr[ctx->device]) {
      void* p = nullptr;
      cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
      if (e != cudaSuccess) return fail_cuda(ctx, e, "cudaGetSymbolAddress(g_noalloc_scratch)", __FILE__, __LINE__);
      g_noalloc_addr[ctx->device] = p;
    }
    base = g_noalloc_addr[ctx->device];
  }
  unsigned char* s = static_cast<unsigned char*>(base);
  c64* xt = reinterpret_cast<c64*>(s);
  c64* yt = reinterpret_cast<c64*>(s + bx);
  cplx<float>* t = reinterpret_cast<cplx<float>*>(s + 2 * bx);
  cplx<float>* part = reinterpret_cast<cplx<float>*>(s + 2 * bx + bt);
  // every scratch value read below is written earlier in this call: nothing needs clearing
  count_if(true);
  k_noalloc_gather<<<(ctx->ne + 127) / 128, 128, 0, ctx->stream>>>(reinterpret_cast<const c64*>(x_dev), ctx->perm.p,
                                                                  ctx->ne, xt);
  launch_hmatvec_scratch_c64(ctx, ctx->near32.p, ctx->u32.p, ctx->v32.p, t, part, xt, yt, ctx->stream);
  count_if(true);
  k_noalloc_scatter<<<(ctx->ne + 127) / 128, 128, 0, ctx->stream>>>(yt, ctx->perm.p, ctx->ne,
                                                                   reinterpret_cast<c64*>(y_dev));
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return fail_cuda(ctx, e, "bem_apply_noalloc launch", __FILE__, __LINE__);
  return BEM_OK;
}
