// selftest.cu -- runs the library's bounded device-side waits against flags that nothing ever
// sets, so that failure detection can be tested without faulting or hanging a GPU: the wait runs
// out, the kernel records the time-out in the context's error word and returns, and the host
// sees SWS_ERR_TIMEOUT from sws_sync with the context still usable.
#include "../../include/sws.h"
#include "internal.h"
#include "mini_common.cuh"
#include "tma.cuh"

namespace sws {
namespace {

// which = 0: the look-back poll of tile 1, whose predecessor's status word stays zero.
// which = 1: an mbarrier that expects 16 bytes of a copy that is never issued.
__global__ void k_selftest_wait(int which, unsigned long long *status, int *err) {
  __shared__ __align__(8) unsigned long long bar;
  if (which == 0) {
    bool failed = false;
    (void)mini::lookback_warp(status, 1u, 1ull, err, failed);
    return;
  }
  if (threadIdx.x == 0) {
    tma::mbar_init(&bar, 1);
    tma::fence_mbar_init();
    tma::mbar_arrive_expect_tx(&bar, 16u);
    if (!tma::mbar_wait_bounded(&bar, 0u)) atomicOr(err, DEVERR_COPY_TIMEOUT);
  }
}

}  // namespace

cudaError_t launch_selftest_wait(int which, unsigned long long *status, int *err, cudaStream_t st) {
  k_selftest_wait<<<1, 32, 0, st>>>(which, status, err);
  return cudaGetLastError();
}

}  // namespace sws
