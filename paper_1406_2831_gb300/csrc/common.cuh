// Internal definitions shared by the CUDA translation units of librbicgstab.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <cstdio>

#include "../../include/rbicgstab.h"

namespace rb {

// Fused multiply-add in the precision of its operands.  Templated code calls
// this instead of fma() so that FP32 arithmetic can never be promoted to the
// FP64 overload (FP64 runs on two lanes per SM per clock on this GPU).
__device__ __forceinline__ float fma_t(float a, float b, float c) { return __fmaf_rn(a, b, c); }
__device__ __forceinline__ double fma_t(double a, double b, double c) { return __fma_rn(a, b, c); }

constexpr int kSlice = 32;        // SELL slice height = warp width
constexpr int kBlock = 256;       // threads per block of the streaming kernels
constexpr int kMaxK = RB_KMAX;
constexpr int kMaxNV = kMaxK + 8; // values one fused reduction may carry per RHS
constexpr int kMaxRhs = RB_MAX_RHS; // right-hand sides one blocked solve iterates together

// SELL-32 view of a sparse matrix: slice `sl` holds rows sl*32 .. sl*32+31;
// entry j of row sl*32+lane sits at slice_ptr[sl] + j*32 + lane.  Padding
// entries have val = 0 and col = the row itself.
//
// Stencil slices.  A slice whose rows together use at most `width` distinct
// column offsets (col - row), every one of which stays inside [0, n) for all
// 32 rows, is laid out in offset order: entry j of row r has col = r + o_j,
// with an explicit zero where the row has no such entry.  Its offsets are
// stored once, offs[sl * offs_stride + j] (j < width), so a kernel may form
// the gather addresses without loading col.  Other slices keep the CSR order;
// their first offs entry is kNoStencil.  col stays valid for every slice.
constexpr int32_t kNoStencil = INT32_MIN;
constexpr int kMaxStencil = 32;
template <typename T>
struct Sell {
  const int64_t* slice_ptr;  // [nslices + 1]
  const int32_t* width;      // [nslices]
  const int32_t* col;
  const T* val;
  int64_t nslices;
  const int32_t* offs;       // [nslices * offs_stride]
  int offs_stride;           // power of two <= kMaxStencil
};

// Completion tickets of one two-level grid reduction (device.cuh,
// grid_finish): one counter per group of blocks and one for the groups.
// Every counter is back at 0 when the reducing kernel ends.
constexpr int kTicketGroups = 128;
struct GridTicket {
  unsigned int top;
  unsigned int group[kTicketGroups];
};

// Blocks per group of a grid of G blocks: 16, more when G > 16 x kTicketGroups.
__host__ __device__ inline int grid_group_size(int G) {
  return G <= 16 * kTicketGroups ? 16 : (G + kTicketGroups - 1) / kTicketGroups;
}
// Rows of nv doubles a grid reduction over G blocks needs in `partials`.
__host__ __device__ inline int64_t grid_partial_rows(int G) {
  const int gs = grid_group_size(G);
  return (int64_t)G + (G + gs - 1) / gs;
}

// Solver state that lives on the device between kernels of one solve.  The
// last block of each fused pass reduces the block partials in a fixed order
// and updates these scalars (Alg. 2).
struct IterState {
  double rho;      // (r~_0, r_{i-1})
  double alpha, omega, beta;
  double rtq;      // (r~_0, q_i)
  double snorm2, rnorm2;
  double thresh2;  // (tol ||b||)^2
  double st, tt, rts, rtt;
  double bnorm2;
  double rmax2;     // largest recursive ||r||^2 since the last reset (residual replacement)
  int32_t iter;     // completed iterations
  int32_t done;     // 1 once converged / failed: every later pass returns at once
  int32_t half;     // the current iteration ended after its half step
  int32_t status;   // RB_* code
  int32_t max_itn;
  int32_t k;
  int32_t pad0, pad1;
  double zeta[kMaxK];
  double gamma[kMaxK];
  double xc[kMaxK];
  double cr[kMaxK];    // C^T r~_0 (zero in exact arithmetic)
  double red[kMaxNV];  // scratch for generic reductions
  GridTicket ticket[8];
};

// Pass identifiers (index into IterState::ticket).
enum Pass { P1 = 0, P2 = 1, P3 = 2, P4 = 3, P5 = 4, PGEN = 5 };

}  // namespace rb

#define RB_CUDA_TRY(expr)                                                          \
  do {                                                                             \
    cudaError_t _e = (expr);                                                       \
    if (_e != cudaSuccess) {                                                       \
      if (getenv("RB_DEBUG"))                                                      \
        fprintf(stderr, "rbicgstab: %s failed at %s:%d: %s\n", #expr, __FILE__,    \
                __LINE__, cudaGetErrorString(_e));                                 \
      return (_e == cudaErrorMemoryAllocation) ? RB_ENOMEM : RB_ECUDA;             \
    }                                                                              \
  } while (0)
