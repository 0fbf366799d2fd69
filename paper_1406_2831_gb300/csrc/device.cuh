// Device helpers: deterministic block + grid reductions ("last block" pattern).
//
// Every fused pass accumulates NV per-thread partial sums in FP64.  A block
// reduces them with a fixed warp-shuffle tree and a fixed cross-warp order,
// writes one row of `partials`, and takes a ticket.  The block that takes the
// last ticket reduces all rows in block order (fixed, independent of which
// block finishes last) and runs the pass's scalar step.  Results are bitwise
// reproducible run to run.
#pragma once

#include "common.cuh"

namespace rb {

template <int NV>
__device__ __forceinline__ void warp_sum(double (&a)[NV]) {
#pragma unroll
  for (int v = 0; v < NV; ++v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) a[v] += __shfl_down_sync(0xffffffffu, a[v], o);
  }
}

// Shared memory needed by block_reduce_last: NWARPS * NV + NV doubles + flag.
template <int NV>
struct ReduceSmem {
  double w[kBlock / 32][NV > 0 ? NV : 1];
  double res[NV > 0 ? NV : 1];
  int last;
};

// Reduce acc[0..nv) (nv <= NV, runtime) over the grid.  Returns true in
// every thread of the last block, with sm.res[0..nv) holding the grid totals.
// `partials` holds gridDim.x * nv doubles (block-major); `ticket` is reset to
// 0 by the last block.  The last block sums the partials with every thread
// (thread t takes blocks t, t + blockDim, ... in order), then reuses the
// fixed warp/cross-warp tree, so the result does not depend on which block
// finished last.
template <int NV>
__device__ bool block_reduce_last(double (&acc)[NV], int nv, ReduceSmem<NV>& sm, double* partials,
                                  unsigned int* ticket) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  constexpr int NW = kBlock / 32;
  warp_sum<NV>(acc);
  if (lane == 0) {
#pragma unroll
    for (int v = 0; v < NV; ++v) sm.w[warp][v] = acc[v];
  }
  __syncthreads();
  for (int v = threadIdx.x; v < nv; v += blockDim.x) {
    double s = 0.0;
#pragma unroll
    for (int w = 0; w < NW; ++w) s += sm.w[w][v];
    partials[(size_t)blockIdx.x * nv + v] = s;
  }
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) {
    unsigned int t = atomicAdd(ticket, 1u);
    sm.last = (t == gridDim.x - 1);
  }
  __syncthreads();
  if (!sm.last) return false;
  __threadfence();
#pragma unroll
  for (int v = 0; v < NV; ++v) acc[v] = 0.0;
  for (int b = threadIdx.x; b < (int)gridDim.x; b += blockDim.x) {
    const double* pb = partials + (size_t)b * nv;
#pragma unroll
    for (int v = 0; v < NV; ++v)
      if (v < nv) acc[v] += __ldcg(pb + v);
  }
  warp_sum<NV>(acc);
  __syncthreads();
  if (lane == 0) {
#pragma unroll
    for (int v = 0; v < NV; ++v) sm.w[warp][v] = acc[v];
  }
  __syncthreads();
  for (int v = threadIdx.x; v < nv; v += blockDim.x) {
    double s = 0.0;
#pragma unroll
    for (int w = 0; w < NW; ++w) s += sm.w[w][v];
    sm.res[v] = s;
  }
  __syncthreads();
  if (threadIdx.x == 0) *ticket = 0u;
  return true;
}

__device__ __forceinline__ int64_t gtid() { return blockIdx.x * (int64_t)blockDim.x + threadIdx.x; }
__device__ __forceinline__ int64_t gstride() { return (int64_t)gridDim.x * blockDim.x; }

}  // namespace rb
