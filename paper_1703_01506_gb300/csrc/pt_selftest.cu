// Check of the bounded device-side wait every persistent kernel of this
// library uses: a wait on an mbarrier phase that nothing completes must give
// up after its limit, record kErrTimeout in the status word and return, leaving
// the context usable. No trap, no fault, no unbounded wait.
#include <cuda_runtime.h>

#include "pt_internal.h"
#include "pt_kernels.h"

namespace pt {
namespace {

__global__ void bounded_wait_kernel(uint32_t* status, unsigned long long limit_ns) {
  __shared__ __align__(8) uint64_t bar;
  __shared__ int abort_flag;
  if (threadIdx.x == 0) {
    mbar_init(smem_addr(&bar), 1);  // nobody arrives: phase 0 never completes
    abort_flag = 0;
    fence_mbar_init();
  }
  __syncthreads();
  if (threadIdx.x == 0) mbar_wait(smem_addr(&bar), 0u, status, &abort_flag, limit_ns);
  __syncthreads();
}

}  // namespace
}  // namespace pt

extern "C" pt_status pt_selftest_bounded_wait(pt_ctx* ctx, int32_t limit_ms) {
  if (!ctx) {
    pt::set_thread_error("pt_selftest_bounded_wait: ctx is NULL");
    return PT_ERR_INVALID;
  }
  if (limit_ms < 1 || limit_ms > 2000) {
    pt::set_error(ctx, "pt_selftest_bounded_wait: need 1 <= limit_ms <= 2000");
    return PT_ERR_INVALID;
  }
  cudaSetDevice(ctx->device);
  pt::bounded_wait_kernel<<<1, 32, 0, ctx->stream>>>(ctx->status.as<uint32_t>(),
                                                    1000000ull * uint64_t(limit_ms));
  PT_LAUNCH_CHECK(ctx);
  return PT_OK;
}
