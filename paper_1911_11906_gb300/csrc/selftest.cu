// Failure detection of the bounded device-side waits, without a fault.
//
// One CTA waits, through the library's own primitives, for an event that
// nothing will produce: the grid barrier of the cooperative kernels with one
// CTA arriving where two are expected, or an mbarrier of the tensor-core
// kernels that nobody arrives on.  Both waits are bounded in SM clock cycles
// (the context's wait limit), so the kernel gives up, records
// FRACLAP_ERR_TIMEOUT in the device status word and returns; the context and
// the GPU stay usable.
#include "internal.cuh"
#include "tc_common.cuh"

namespace fraclap {
namespace {

__global__ void wait_selftest_kernel(int which, unsigned* state, long long limit, int32_t* status) {
  __shared__ __align__(8) uint64_t bar;
  if (which == 0) {
    grid_barrier(state, 2u, limit, status);  // the second CTA never comes
    return;
  }
  if (threadIdx.x == 0) tc::mbar_init(&bar, 1);
  __syncthreads();
  if (threadIdx.x == 0 && !tc::mbar_wait(&bar, 0, limit)) raise_status(status, FRACLAP_ERR_TIMEOUT);
}

}  // namespace
}  // namespace fraclap

using namespace fraclap;

extern "C" int fraclap_wait_selftest(fraclap_ctx* ctx, int which, fraclap_stream_t stream) {
  if (!ctx) return FRACLAP_ERR_INVALID_ARG;
  FL_CHECK(ctx, which == 0 || which == 1, FRACLAP_ERR_INVALID_ARG, "wait_selftest: which must be 0 or 1");
  cudaStream_t st = (cudaStream_t)stream;
  // words 2 and 3 of the barrier state: the cooperative kernels use words 0 and 1
  unsigned* state = ctx->d_barrier + 2;
  FL_CUDA(ctx, cudaMemsetAsync(state, 0, 2 * sizeof(unsigned), st));
  wait_selftest_kernel<<<1, 32, 0, st>>>(which, state, ctx->wait_cycles, ctx->d_status);
  count_launch(ctx);
  FL_CUDA(ctx, cudaGetLastError());
  return 0;
}

// ----------------------------------------------------------------------------
// FMA throughput probe: every thread runs kChains independent FMA chains of
// `iters` steps (x <- x * a + c, with a and c chosen so the values stay
// bounded), over a grid of 8 CTAs of 256 threads per SM, timed with CUDA
// events on the caller's stream.  The result is the sustained rate of the
// FP64 or FP32 FMA pipe: the peaks that the SIMT kernels of this library are
// measured against.
// ----------------------------------------------------------------------------
namespace fraclap {
namespace {

constexpr int kChains = 8;

template <class T>
__global__ void __launch_bounds__(256) fma_probe_kernel(int64_t iters, T a, T c, T* sink) {
  T x[kChains];
#pragma unroll
  for (int i = 0; i < kChains; ++i) x[i] = (T)(threadIdx.x + i) * (T)1e-3;
  for (int64_t it = 0; it < iters; ++it) {
#pragma unroll
    for (int i = 0; i < kChains; ++i) x[i] = fma(x[i], a, c);
  }
  T s = T(0);
#pragma unroll
  for (int i = 0; i < kChains; ++i) s += x[i];
  if (s == T(12345.678)) sink[0] = s;  // keeps the chains alive; never true for these inputs
}

}  // namespace
}  // namespace fraclap

extern "C" int fraclap_fma_throughput(fraclap_ctx* ctx, int precision, int64_t iters, double* flops_per_s,
                                      fraclap_stream_t stream) {
  if (!ctx || !flops_per_s) return FRACLAP_ERR_INVALID_ARG;
  FL_CHECK(ctx, (precision == 32 || precision == 64) && iters >= 1, FRACLAP_ERR_INVALID_ARG,
           "fma_throughput: precision 32 or 64, iters >= 1");
  cudaStream_t st = (cudaStream_t)stream;
  Arena ar;
  FL_TRY(get_workspace(ctx, nullptr, 0, 256, &ar));
  double* sink = ar.take<double>(1);
  const unsigned grid = (unsigned)ctx->sm_count * 8;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  FL_CUDA(ctx, cudaEventCreate(&e0));
  cudaError_t e = cudaEventCreate(&e1);
  if (e != cudaSuccess) {
    cudaEventDestroy(e0);
    return set_error(ctx, FRACLAP_ERR_CUDA, "fma_throughput: %s", cudaGetErrorString(e));
  }
  // one untimed launch, then the timed one
  for (int rep = 0; rep < 2; ++rep) {
    if (rep == 1) cudaEventRecord(e0, st);
    if (precision == 64)
      fma_probe_kernel<double><<<grid, 256, 0, st>>>(iters, 0.999999, 1e-7, sink);
    else
      fma_probe_kernel<float><<<grid, 256, 0, st>>>(iters, 0.999f, 1e-4f, reinterpret_cast<float*>(sink));
    count_launch(ctx);
  }
  cudaEventRecord(e1, st);
  e = cudaEventSynchronize(e1);
  float ms = 0.0f;
  if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (e != cudaSuccess) return set_error(ctx, FRACLAP_ERR_CUDA, "fma_throughput: %s", cudaGetErrorString(e));
  FL_CUDA(ctx, cudaGetLastError());
  const double flops = 2.0 * (double)grid * 256.0 * (double)kChains * (double)iters;
  *flops_per_s = flops / ((double)ms * 1e-3);
  return 0;
}
