// selftest.cu — exercises the give-up path of the bounded mbarrier waits.
//
// Every kernel that waits for bulk copies (the Gram kernel) polls its
// mbarrier a bounded number of times; if the bytes never arrive it records
// ST_TIMEOUT, waits (bounded) for whatever copies it did issue and returns,
// so the context stays usable instead of hanging.  This entry point runs the
// same wait on a barrier whose expected bytes no copy will ever deliver (no
// copy is issued at all, so nothing can land in shared memory afterwards) and
// reports whether the wait gave up; with `expect_bytes` = 0 the barrier
// completes by a plain arrival and the wait must succeed.
#include "../../include/mbicg.h"
#include "internal.h"

using namespace mbicg;

namespace {

__global__ void k_wait_selftest(int limit, int expect_bytes, int* status) {
  __shared__ uint64_t bar;
  if (threadIdx.x == 0) {
    mbar_init(&bar, 1);
    mbar_fence_init();
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    if (expect_bytes > 0)
      mbar_arrive_expect_tx(&bar, (uint32_t)expect_bytes);  // bytes nothing will deliver
    else
      mbar_arrive(&bar);
  }
  __syncthreads();
  const bool arrived = mbar_wait_bounded(&bar, 0, limit);
  if (__syncthreads_or(!arrived) && threadIdx.x == 0) atomicOr(status, ST_TIMEOUT);
}

}  // namespace

extern "C" int mbicg_selftest_bounded_wait(int device, int spin_limit, int expect_bytes, int* timed_out) {
  if (!timed_out || spin_limit < 1 || spin_limit > MBAR_SPIN_LIMIT || expect_bytes < 0 || expect_bytes % 16)
    return MBICG_EINVAL;
  if (cudaSetDevice(device) != cudaSuccess) {
    cudaGetLastError();
    return MBICG_ECUDA;
  }
  int* d = nullptr;
  int h = 0;
  if (cudaMalloc(&d, sizeof(int)) != cudaSuccess) {
    cudaGetLastError();
    return MBICG_ENOMEM;
  }
  cudaError_t e = cudaMemset(d, 0, sizeof(int));
  if (e == cudaSuccess) {
    k_wait_selftest<<<1, 64>>>(spin_limit, expect_bytes, d);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaMemcpy(&h, d, sizeof(int), cudaMemcpyDeviceToHost);
  cudaFree(d);
  if (e != cudaSuccess) return MBICG_ECUDA;
  *timed_out = (h & ST_TIMEOUT) ? 1 : 0;
  return MBICG_OK;
}
