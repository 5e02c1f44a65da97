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
