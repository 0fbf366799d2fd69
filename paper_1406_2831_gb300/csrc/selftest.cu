// Self-test of the bounded mbarrier wait (mbar.cuh) that the tensor-core
// Gram and the bulk-copy staging rely on to end instead of hanging when a
// copy or an MMA never completes.  One block initialises an mbarrier for one
// arrival and waits on its first phase through mbar_wait_for with the
// caller's limit: with `complete` set a thread arrives first and the wait
// must succeed; without it nothing ever arrives and the wait must give up
// after the limit, leave the kernel normally and report RB_ETIMEOUT, so the
// context stays usable.  Nothing in it faults, traps or spins without bound.
#include "common.cuh"
#include "kernels.h"
#include "mbar.cuh"

namespace rb {
namespace {

__global__ void k_wait_selftest(int complete, long long limit, int* status) {
  __shared__ __align__(8) uint64_t bar;
  __shared__ int abort_flag;
  if (threadIdx.x == 0) {
    mbar_init(smem_u32(&bar), 1);
    abort_flag = 0;
    fence_barrier_init();
  }
  __syncthreads();
  if (complete && threadIdx.x == 0) mbar_arrive(smem_u32(&bar));
  const bool ok = mbar_wait_for(smem_u32(&bar), 0, &abort_flag, limit);
  __syncthreads();
  if (threadIdx.x == 0) *status = (ok && !abort_flag) ? RB_OK : RB_ETIMEOUT;
}

}  // namespace
}  // namespace rb

extern "C" int rbicgstab_wait_selftest(int32_t complete, double limit_ms, double* waited_ms) {
  if (!(limit_ms > 0) || limit_ms > 1000.0) return RB_EINVAL;
  int dev = 0, khz = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&khz, cudaDevAttrClockRate, dev) != cudaSuccess)
    return RB_ECUDA;
  const long long limit = (long long)(limit_ms * (double)khz);   // SM clock cycles at the rated clock
  int* d = nullptr;
  if (cudaMalloc(&d, sizeof(int)) != cudaSuccess) return RB_ENOMEM;
  int h = RB_ECUDA;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  cudaEventRecord(e0, 0);
  rb::count_launches(1);
  rb::k_wait_selftest<<<1, 64>>>(complete, limit, d);
  cudaError_t e = cudaGetLastError();
  cudaEventRecord(e1, 0);
  if (e == cudaSuccess) e = cudaMemcpy(&h, d, sizeof(int), cudaMemcpyDeviceToHost);
  float ms = 0.f;
  if (e == cudaSuccess) cudaEventElapsedTime(&ms, e0, e1);
  if (waited_ms) *waited_ms = ms;
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaFree(d);
  return e == cudaSuccess ? h : RB_ECUDA;
}
