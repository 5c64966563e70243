// Self-test of the device-side bounded waits: one CTA runs the same bounded
// mbarrier wait the pipelined kernels use (tc::mbar_wait), on a barrier whose
// phase either completes (one arrival before the wait) or never does, with a
// short iteration limit, and reports a wait that ran out as TT_STATUS_TIMEOUT.
// Nothing asynchronous (copies, tensor-core operations) is issued, so giving
// up leaves nothing in flight; the kernel returns normally either way.
#include "tc_common.cuh"
#include "ttc_device.cuh"
#include "ttc_internal.h"

namespace ttc {

__global__ void wait_selftest_kernel(int complete, long long limit, int32_t* status) {
  __shared__ __align__(8) uint64_t bar;
  __shared__ int abort_flag;
  if (threadIdx.x == 0) {
    tc::mbar_init(&bar, 1);
    tc::mbar_init_fence();
    abort_flag = 0;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    if (complete) tc::mbar_arrive(&bar);  // phase 0 completes
    const bool ok = tc::mbar_wait(&bar, 0, &abort_flag, limit);
    if (!ok) set_status(status, TT_STATUS_TIMEOUT);
  }
}

}  // namespace ttc

extern "C" int tt_selftest_wait(int complete, int64_t limit_cycles, int32_t* status_dev, tt_stream stream) {
  if (status_dev == nullptr || limit_cycles < 0 || limit_cycles > ttc::tc::kWaitLimit) return TT_ERR_ARG;
  ttc::count_launch();
  ttc::wait_selftest_kernel<<<1, 32, 0, reinterpret_cast<cudaStream_t>(stream)>>>(complete != 0, limit_cycles,
                                                                                  status_dev);
  return cudaGetLastError() == cudaSuccess ? TT_OK : TT_ERR_CUDA;
}
