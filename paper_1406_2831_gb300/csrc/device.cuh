// Device helpers: deterministic block + grid reductions ("last block" pattern).
//
// Every fused pass accumulates nv per-thread partial sums in FP64.  A block
// sums them through shared memory in a fixed order, writes one row of
// `partials`, and takes a ticket; the last block of each group of blocks sums
// its group's rows, and the last group sums the group rows and runs the
// pass's scalar step.  Results are bitwise reproducible run to run.
//
// FP64 adds are scarce on this GPU (two FP64 lanes per SM per clock), so the
// block sum is a shared-memory transpose (one add per partial) rather than a
// warp-shuffle tree (five adds per lane per value).
#pragma once

#include "common.cuh"

namespace rb {

// Per-thread dot-product accumulator.  FP64 data accumulate with FP64 FMA.
// FP32 data (the inner solve of the mixed path) accumulate with the Dot2
// scheme of Ogita, Rump and Oishi ("Accurate sum and dot product", SIAM J.
// Sci. Comput. 26, 2005): each product a*b is split exactly into p + e with an
// FMA, p is added to the running sum with Knuth's TwoSum, and the rounding
// errors are collected in a second FP32 word.  The pair (hi, lo) carries about
// twice FP32's precision, and the per-thread result is handed to the FP64 grid
// reduction as hi + lo.  This keeps FP64-class dot products on the FP32 pipes.
template <typename T>
struct Acc;

template <>
struct Acc<double> {
  double v = 0.0;
  __device__ __forceinline__ void add(double a, double b) { v = fma(a, b, v); }
  __device__ __forceinline__ void add1(double x) { v += x; }
  __device__ __forceinline__ double get() const { return v; }
};

template <>
struct Acc<float> {
  float hi = 0.0f, lo = 0.0f;
  // The _rn intrinsics are never contracted into FMAs, which would break the
  // exactness of the error-free transformations.
  __device__ __forceinline__ void add(float a, float b) {
    const float p = __fmul_rn(a, b);
    const float e = __fmaf_rn(a, b, -p);                 // a*b = p + e exactly
    const float s = __fadd_rn(hi, p);                    // TwoSum(hi, p) = s + err
    const float bb = __fsub_rn(s, hi);
    const float err = __fadd_rn(__fsub_rn(hi, __fsub_rn(s, bb)), __fsub_rn(p, bb));
    hi = s;
    lo = __fadd_rn(lo, __fadd_rn(err, e));
  }
  // Compensated add of one FP32 value (TwoSum, error into lo).
  __device__ __forceinline__ void add1(float x) {
    const float s = __fadd_rn(hi, x);
    const float bb = __fsub_rn(s, hi);
    const float err = __fadd_rn(__fsub_rn(hi, __fsub_rn(s, bb)), __fsub_rn(x, bb));
    hi = s;
    lo = __fadd_rn(lo, err);
  }
  __device__ __forceinline__ double get() const { return (double)hi + (double)lo; }
};

// Two lanes of T handled together.  For float these are the packed FP32
// instructions of this GPU (one instruction for both lanes, each lane
// rounded exactly as the scalar _rn operation); for double, two scalar
// operations.
template <typename T>
struct Pair;
template <>
struct Pair<float> {
  using V = float2;
  static __device__ __forceinline__ V mk(float a, float b) { return make_float2(a, b); }
  static __device__ __forceinline__ V fma(V a, V b, V c) { return __ffma2_rn(a, b, c); }
  static __device__ __forceinline__ V add(V a, V b) { return __fadd2_rn(a, b); }
  static __device__ __forceinline__ V mul(V a, V b) { return __fmul2_rn(a, b); }
  static __device__ __forceinline__ V neg(V a) { return make_float2(-a.x, -a.y); }
};
template <>
struct Pair<double> {
  using V = double2;
  static __device__ __forceinline__ V mk(double a, double b) { return make_double2(a, b); }
  static __device__ __forceinline__ V fma(V a, V b, V c) { return make_double2(__fma_rn(a.x, b.x, c.x), __fma_rn(a.y, b.y, c.y)); }
  static __device__ __forceinline__ V add(V a, V b) { return make_double2(__dadd_rn(a.x, b.x), __dadd_rn(a.y, b.y)); }
  static __device__ __forceinline__ V mul(V a, V b) { return make_double2(__dmul_rn(a.x, b.x), __dmul_rn(a.y, b.y)); }
  static __device__ __forceinline__ V neg(V a) { return make_double2(-a.x, -a.y); }
};

// Two dot-product accumulators side by side: for float the Dot2 scheme of
// Acc<float> on packed pairs (the same result in each lane as Acc<float>),
// for double FP64 FMAs.  lane(h) returns lane h as a scalar accumulator.
template <typename T>
struct AccP;
template <>
struct AccP<float> {
  using P = Pair<float>;
  float2 hi = make_float2(0.0f, 0.0f), lo = make_float2(0.0f, 0.0f);
  __device__ __forceinline__ void add(float2 a, float2 b) {
    const float2 p = P::mul(a, b);
    const float2 e = P::fma(a, b, P::neg(p));                 // a*b = p + e exactly
    const float2 s = P::add(hi, p);                           // TwoSum(hi, p) = s + err
    const float2 bb = P::add(s, P::neg(hi));
    const float2 err = P::add(P::add(hi, P::neg(P::add(s, P::neg(bb)))), P::add(p, P::neg(bb)));
    hi = s;
    lo = P::add(lo, P::add(err, e));
  }
  // Compensated add of one FP32 value per lane (TwoSum, error into lo).
  __device__ __forceinline__ void add1(float2 x) {
    const float2 s = P::add(hi, x);
    const float2 bb = P::add(s, P::neg(hi));
    const float2 err = P::add(P::add(hi, P::neg(P::add(s, P::neg(bb)))), P::add(x, P::neg(bb)));
    hi = s;
    lo = P::add(lo, err);
  }
  __device__ __forceinline__ Acc<float> lane(int h) const {
    Acc<float> a;
    a.hi = h ? hi.y : hi.x;
    a.lo = h ? lo.y : lo.x;
    return a;
  }
};
template <>
struct AccP<double> {
  double2 v = make_double2(0.0, 0.0);
  __device__ __forceinline__ void add(double2 a, double2 b) {
    v.x = __fma_rn(a.x, b.x, v.x);
    v.y = __fma_rn(a.y, b.y, v.y);
  }
  __device__ __forceinline__ void add1(double2 x) {
    v.x += x.x;
    v.y += x.y;
  }
  __device__ __forceinline__ Acc<double> lane(int h) const {
    Acc<double> a;
    a.v = h ? v.y : v.x;
    return a;
  }
};

constexpr int kRedCH = 8;   // values per transpose chunk

// Transpose buffer of the FP64 block sums: [warp][value][lane] (+1 pad).
typedef double RedT[kBlock / 32][kRedCH][33];

// Per-warp sums, the block/grid totals and the last-block flag.
template <int NV>
struct ReduceCore {
  double w[kBlock / 32][NV > 0 ? NV : 1];
  double res[NV > 0 ? NV : 1];
  int last;
};

template <int NV>
struct ReduceSmem : ReduceCore<NV> {
  static constexpr int CH = kRedCH;
  RedT t;
};

// Warp-level sums of per-thread accumulators into sm.w[warp][v].
// * FP32 Dot2 pairs (hi, lo): shuffle tree combining pairs with TwoSum in
//   FP32, one conversion to FP64 per warp and value.
// * FP64 values: the FP64 pipe is charged per warp instruction (about 16
//   cycles each, however many lanes are active), so few values use the
//   5-step shuffle tree (5 instructions per value) and 8 or more use a
//   shared-memory transpose (32 instructions per 8 values).
template <int NV>
__device__ __forceinline__ void warp_sums(Acc<float> (&acc)[NV], int nv, ReduceSmem<NV>& sm) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int v = 0; v < NV; ++v) {
    if (v < nv) {
      float hi = acc[v].hi, lo = acc[v].lo;
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        const float h2 = __shfl_down_sync(0xffffffffu, hi, o);
        const float l2 = __shfl_down_sync(0xffffffffu, lo, o);
        const float s = __fadd_rn(hi, h2);
        const float bb = __fsub_rn(s, hi);
        const float e = __fadd_rn(__fsub_rn(hi, __fsub_rn(s, bb)), __fsub_rn(h2, bb));
        hi = s;
        lo = __fadd_rn(__fadd_rn(lo, l2), e);
      }
      if (lane == 0) sm.w[warp][v] = (double)hi + (double)lo;
    }
  }
}

template <int NV>
__device__ __forceinline__ void warp_sums(Acc<double> (&acc)[NV], int nv, ReduceSmem<NV>& sm) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (NV < 8) {
#pragma unroll
    for (int v = 0; v < NV; ++v) {
      if (v < nv) {
        double x = acc[v].v;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) x += __shfl_down_sync(0xffffffffu, x, o);
        if (lane == 0) sm.w[warp][v] = x;
      }
    }
    return;
  }
  constexpr int CH = ReduceSmem<NV>::CH;
#pragma unroll
  for (int c0 = 0; c0 < NV; c0 += CH) {
    if (c0 < nv) {
#pragma unroll
      for (int u = 0; u < CH; ++u)
        if (c0 + u < NV) sm.t[warp][u][lane] = acc[c0 + u].v;
      __syncwarp();
      if (lane < CH && c0 + lane < nv) {
        const double* row = sm.t[warp][lane];
        double s0 = 0.0, s1 = 0.0, s2 = 0.0, s3 = 0.0;
#pragma unroll
        for (int j = 0; j < 32; j += 4) {
          s0 += row[j];
          s1 += row[j + 1];
          s2 += row[j + 2];
          s3 += row[j + 3];
        }
        sm.w[warp][c0 + lane] = (s0 + s1) + (s2 + s3);
      }
      __syncwarp();
    }
  }
}

// Sum per-thread accumulators over the block: sm.res[v] holds the block
// total of value v on return (after a __syncthreads).  Fixed order.
template <typename T, int NV>
__device__ __forceinline__ void block_sum(Acc<T> (&acc)[NV], int nv, ReduceSmem<NV>& sm) {
  constexpr int NW = kBlock / 32;
  warp_sums<NV>(acc, nv, sm);
  __syncthreads();
  for (int v = threadIdx.x; v < nv; v += blockDim.x) {
    double s = 0.0;
#pragma unroll
    for (int w = 0; w < NW; ++w) s += sm.w[w][v];
    sm.res[v] = s;
  }
  __syncthreads();
}

// Second half of a grid reduction: every warp has written its sums to
// sm.w[warp][0..nv).  Sums them across warps, publishes the block partial
// and takes a ticket; returns true in every thread of the last block with
// sm.res[0..nv) holding the grid totals.  The tickets are left at 0.
//
// Two levels, so that no single block sums every block's partials: FP64 adds
// run on few lanes per SM, and one block summing G x nv values serialised
// the end of every pass.  Blocks form groups of gs consecutive blocks; the
// last block of a group to finish sums the group's rows (in block order)
// into a group row; the last group sums the group rows (in group order).
// Fixed summation order: bitwise reproducible.  `partials` holds G + ceil(G /
// gs) rows of nv doubles.
template <int NV>
__device__ bool grid_finish(int nv, ReduceCore<NV>& sm, double* partials, GridTicket* ticket) {
  constexpr int NW = kBlock / 32;
  const int G = gridDim.x;
  const int gs = grid_group_size(G);
  const int ng = (G + gs - 1) / gs;
  const int g = blockIdx.x / gs;
  const int gsz = min(gs, G - g * gs);
  double* grows = partials + (size_t)G * nv;
  __syncthreads();
  for (int v = threadIdx.x; v < nv; v += blockDim.x) {
    double s = 0.0;
#pragma unroll
    for (int w = 0; w < NW; ++w) s += sm.w[w][v];
    partials[(size_t)blockIdx.x * nv + v] = s;
  }
  if (threadIdx.x < nv) __threadfence();   // only the writers publish before the ticket
  __syncthreads();
  if (threadIdx.x == 0) sm.last = (atomicAdd(&ticket->group[g], 1u) == (unsigned)gsz - 1u);
  __syncthreads();
  if (!sm.last) return false;
  // last block of group g
  __threadfence();
  for (int v = threadIdx.x; v < nv; v += blockDim.x) {
    const double* p = partials + (size_t)g * gs * nv + v;
    double s = 0.0;
#pragma unroll 4
    for (int i = 0; i < gsz; ++i) s += __ldcg(p + (size_t)i * nv);
    grows[(size_t)g * nv + v] = s;
  }
  if (threadIdx.x < nv) __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) {
    ticket->group[g] = 0u;
    sm.last = (atomicAdd(&ticket->top, 1u) == (unsigned)ng - 1u);
  }
  __syncthreads();
  if (!sm.last) return false;
  // last group
  __threadfence();
  for (int v = threadIdx.x; v < nv; v += blockDim.x) {
    double s = 0.0;
#pragma unroll 4
    for (int i = 0; i < ng; ++i) s += __ldcg(grows + (size_t)i * nv + v);
    sm.res[v] = s;
  }
  __syncthreads();
  if (threadIdx.x == 0) ticket->top = 0u;
  return true;
}

// Reduce per-thread accumulators acc[0..nv) (nv <= NV) over the grid.
template <typename T, int NV>
__device__ bool block_reduce_last(Acc<T> (&acc)[NV], int nv, ReduceSmem<NV>& sm, double* partials,
                                  GridTicket* ticket) {
  warp_sums<NV>(acc, nv, sm);
  return grid_finish<NV>(nv, static_cast<ReduceCore<NV>&>(sm), partials, ticket);
}

// FP64 convenience form: per-thread doubles.
template <int NV>
__device__ bool block_reduce_last(double (&vals)[NV], int nv, ReduceSmem<NV>& sm, double* partials,
                                  GridTicket* ticket) {
  Acc<double> acc[NV];
#pragma unroll
  for (int v = 0; v < NV; ++v) acc[v].v = vals[v];
  return block_reduce_last<double, NV>(acc, nv, sm, partials, ticket);
}

__device__ __forceinline__ int64_t gtid() { return blockIdx.x * (int64_t)blockDim.x + threadIdx.x; }
__device__ __forceinline__ int64_t gstride() { return (int64_t)gridDim.x * blockDim.x; }

}  // namespace rb
