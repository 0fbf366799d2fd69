// Batched solves of many independent systems of uneven sizes (the batched
// pattern of a parametric sweep: many parameter samples, each with its own
// matrix, right-hand side and recycle space), one launch per pass for all of
// them.
//
// The systems are stacked into one block-diagonal SELL-32 matrix; every
// system's rows are padded to a multiple of 32, so a slice never straddles
// two systems.  Each pass is one persistent kernel over a work list of
// tiles, a tile being a range of `tile_slices` slices inside one system.  A
// CTA takes tiles in grid-stride order; for each it forms the pass's vector
// updates and its contribution to the pass's dot products, writes one
// partial row per tile and counts the tile on its system's ticket.  The CTA
// that completes a system's last tile adds that system's tile rows with all
// its threads in a fixed order (deterministic) and runs the scalar step of
// Alg. 2 for that system (the same device functions as the single-system
// passes).  Systems that have converged or failed skip their tiles.  The
// iteration loop is captured as a CUDA graph of `poll` iterations.  The tile
// size and the number of CTAs per SM are chosen by timing the SpMV +
// projection pass on the batch (autotuner, logged on request).
//
// Each system may carry a fixed recycle space of k <= 16 columns (U~ = U,
// the right-only variant of Sec. 5), set up per system as in Sec. 3
// (C = A U, C~ = A^T U, M = C~^T C, C-hat = C~ (M^+)^T).  The inner
// iteration runs in FP64 or, in the mixed mode, in FP32 with Dot2-compensated
// dot products and FP64 residual replacement per system (folds of the FP32
// increment into the FP64 x, masked per system); a system whose FP32
// iteration stalls, breaks down or overflows is finished in FP64 rounds.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <functional>
#include <vector>

#include "device.cuh"
#include "hostla.h"
#include "kernels.h"
#include "scalars.cuh"

namespace rb {
namespace {

constexpr int kBK = 16;                 // largest recycle dimension of a batch
constexpr int kBNV = kBK + 4;           // values per tile partial row

struct PassGrids {
  int g[5];   // P1..P5
};

struct BatchTiles {
  const int32_t* sys;        // [ntiles] system of the tile
  const int64_t* sl0;        // [ntiles] first slice
  const int32_t* nsl;        // [ntiles] slices
  const int32_t* t0;         // [nsys] first tile of the system
  const int32_t* nt;         // [nsys] tiles of the system
  int ntiles;
};

template <typename T>
struct BatchArgs {
  Sell<T> A;
  const T* Chat;
  const T* C;
  int64_t ld;                // rows of the stacked vectors (all systems, padded)
  int k;
  const T* rt0;
  T *x, *r, *p, *s, *q, *t, *qraw, *traw;
  IterState* st;             // one per system
  double* partials;          // [ntiles][kBNV]
  BatchTiles tiles;
};

// Shared "does this tile's system still iterate" test: one read, broadcast.
__device__ __forceinline__ bool tile_active(const IterState* st, bool skip_half) {
  __shared__ int s_act;
  if (threadIdx.x == 0) s_act = !st->done && !(skip_half && st->half);
  __syncthreads();
  const bool a = s_act;
  __syncthreads();
  return a;
}

// After block_sum: sm.res[0..nv) are the tile's totals.  Stores the tile's
// partial row and counts it; returns true in every thread of the CTA that
// completed the system's last tile, with sm.res[0..nv) then holding the
// system's totals.  That CTA sums the system's nt partial rows with all its
// threads: thread i takes tiles i, i + blockDim, ... in order, a fixed
// shuffle tree adds the threads of a warp and the warps are added in order
// (deterministic; a system split into many tiles no longer holds one thread
// for nt dependent loads).  The ticket is back at 0 after.
template <int NV>
__device__ bool tile_commit(ReduceCore<NV>& sm, int nv, double* partials, int t, unsigned* ticket, int t0,
                            int nt) {
  __shared__ int s_last;
  if (threadIdx.x == 0) {
    for (int v = 0; v < nv; ++v) partials[(size_t)t * kBNV + v] = sm.res[v];
    __threadfence();
    const unsigned prev = atomicAdd(ticket, 1u);
    s_last = prev == (unsigned)(nt - 1);
  }
  __syncthreads();
  if (!s_last) return false;
  __threadfence();
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int v = 0; v < nv; ++v) {
    double acc = 0.0;
    for (int q = threadIdx.x; q < nt; q += blockDim.x) acc += __ldcg(partials + (size_t)(t0 + q) * kBNV + v);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
    if (lane == 0) sm.w[warp][v] = acc;
  }
  __syncthreads();
  for (int v = threadIdx.x; v < nv; v += blockDim.x) {
    double acc = 0.0;
    for (int w = 0; w < kBlock / 32; ++w) acc += sm.w[w][v];
    sm.res[v] = acc;
  }
  if (threadIdx.x == 0) *ticket = 0u;
  __syncthreads();
  return true;
}

// y = A v over the rows of one slice (lane = row), SELL-32 with column
// loads; w and sp are the slice's width and first entry.  The first kHead
// entries of every row are loaded together (values and columns), then their
// gathers, then the products: two memory latencies per slice instead of two
// per entry (a warp issues in order, so a product waiting for its gather
// would hold back the next entry's loads).  Longer rows continue entry by
// entry; the sum runs in entry order either way.
constexpr int kHead = 8;
template <typename T>
__device__ __forceinline__ T slice_row_product(const Sell<T>& A, const T* __restrict__ v, int w, int64_t sp,
                                               int lane) {
  const int64_t e0 = sp + lane;
  T val[kHead];
  int32_t col[kHead];
#pragma unroll
  for (int j = 0; j < kHead; ++j) {
    val[j] = T(0);
    col[j] = 0;
    if (j < w) {
      val[j] = __ldg(A.val + e0 + (int64_t)j * kSlice);
      col[j] = __ldg(A.col + e0 + (int64_t)j * kSlice);
    }
  }
  T g[kHead];
#pragma unroll
  for (int j = 0; j < kHead; ++j) g[j] = j < w ? __ldg(v + col[j]) : T(0);
  T y = T(0);
#pragma unroll
  for (int j = 0; j < kHead; ++j)
    if (j < w) y = fma_t(val[j], g[j], y);
  for (int j = kHead; j < w; ++j) {
    const int64_t e = e0 + (int64_t)j * kSlice;
    y = fma_t(__ldg(A.val + e), __ldg(v + __ldg(A.col + e)), y);
  }
  return y;
}

// P1 / P3 without a recycle space: q_raw = A p and (r~_0, q_raw) -> alpha
// (finish_p1); t_raw = A s and the four dots (s,t), (t,t), (r~_0,t),
// (r~_0,s) -> omega, rho, beta (finish_p4: P4 folds into P3).  One warp per
// SELL slice, row per lane, Dot2 (FP32) or FP64 accumulators.
template <typename T, bool IS_P3>
__global__ void __launch_bounds__(kBlock) kb_spmv_plain(BatchArgs<T> a) {
  constexpr int NV = 4;
  __shared__ ReduceSmem<NV> sm;
  __shared__ double scr[kBK + 1];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const T* __restrict__ v = IS_P3 ? a.s : a.p;
  T* __restrict__ out = IS_P3 ? a.traw : a.qraw;
  for (int t = blockIdx.x; t < a.tiles.ntiles; t += gridDim.x) {
    const int sys = a.tiles.sys[t];
    IterState* st = a.st + sys;
    if (!tile_active(st, IS_P3)) continue;
    Acc<T> acc[NV];
    const int64_t sl0 = a.tiles.sl0[t];
    const int nsl = a.tiles.nsl[t];
    // the next slice's width and start are loaded one step ahead
    int w_nx = 0;
    int64_t sp_nx = 0;
    if (warp < nsl) {
      w_nx = __ldg(a.A.width + sl0 + warp);
      sp_nx = __ldg(a.A.slice_ptr + sl0 + warp);
    }
    for (int q = warp; q < nsl; q += kBlock / 32) {
      const int64_t sl = sl0 + q;
      const int w = w_nx;
      const int64_t sp = sp_nx;
      if (q + kBlock / 32 < nsl) {
        w_nx = __ldg(a.A.width + sl + kBlock / 32);
        sp_nx = __ldg(a.A.slice_ptr + sl + kBlock / 32);
      }
      const int64_t row = sl * kSlice + lane;
      const T rv = __ldg(a.rt0 + row);
      const T sv = IS_P3 ? __ldg(a.s + row) : T(0);
      const T y = slice_row_product(a.A, v, w, sp, lane);
      out[row] = y;
      if (!IS_P3) {
        acc[0].add(rv, y);
      } else {
        acc[0].add(sv, y);
        acc[1].add(y, y);
        acc[2].add(rv, y);
        acc[3].add(rv, sv);
      }
    }
    const int nv = IS_P3 ? 4 : 1;
    block_sum<T, NV>(acc, nv, sm);
    if (tile_commit<NV>(sm, nv, a.partials, t, &st->ticket[IS_P3 ? P3 : P1].top, a.tiles.t0[sys], a.tiles.nt[sys])) {
      if (warp == 0) {
        if (!IS_P3) finish_p1(st, sm.res, 0, scr);
        else finish_p4(st, sm.res, 0);
      }
    }
    __syncthreads();
  }
}

// Warp total of a per-lane accumulator (valid in lane 0): FP32 Dot2 pairs
// combined by TwoSum along a fixed shuffle tree, FP64 by plain adds.
template <typename T>
__device__ __forceinline__ double warp_total(const Acc<T>& a);
template <>
__device__ __forceinline__ double warp_total<float>(const Acc<float>& a) {
  float hi = a.hi, lo = a.lo;
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
  return (double)hi + (double)lo;
}
template <>
__device__ __forceinline__ double warp_total<double>(const Acc<double>& a) {
  double x = a.v;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) x += __shfl_down_sync(0xffffffffu, x, o);
  return x;
}

// sum_l c[l] ys[l] over the 32 rows of a slice, in row order (c 16-byte
// aligned: a column of C-hat from the slice's first row).
__device__ __forceinline__ float slice_col_dot(const float* __restrict__ c, const float* ys) {
  const float4* c4 = reinterpret_cast<const float4*>(c);
  float s = 0.f;
#pragma unroll
  for (int i = 0; i < kSlice / 4; ++i) {
    const float4 v = __ldg(c4 + i);
    s = __fmaf_rn(v.x, ys[4 * i], s);
    s = __fmaf_rn(v.y, ys[4 * i + 1], s);
    s = __fmaf_rn(v.z, ys[4 * i + 2], s);
    s = __fmaf_rn(v.w, ys[4 * i + 3], s);
  }
  return s;
}
__device__ __forceinline__ double slice_col_dot(const double* __restrict__ c, const double* ys) {
  const double2* c2 = reinterpret_cast<const double2*>(c);
  double s = 0.0;
#pragma unroll
  for (int i = 0; i < kSlice / 2; ++i) {
    const double2 v = __ldg(c2 + i);
    s = __fma_rn(v.x, ys[2 * i], s);
    s = __fma_rn(v.y, ys[2 * i + 1], s);
  }
  return s;
}

// P1 / P3 with a recycle space (k > 0): the SpMV of kb_spmv_plain, and the
// projection C-hat^T y with lane j owning column j: the warp puts the
// slice's 32 products in shared memory, lane j < k sums column j's 32 rows
// against them in FP32 (row order) and carries the slice sums across slices
// in a Dot2 pair (FP64 data: FP64 throughout).  One accumulator per lane
// instead of k per thread keeps the kernel at full occupancy.  P1 also forms
// (r~_0, q_raw) row per lane.
template <typename T, bool IS_P3>
__global__ void __launch_bounds__(kBlock) kb_spmv_proj(BatchArgs<T> a) {
  constexpr int NW = kBlock / 32;
  __shared__ ReduceCore<kBK + 1> sm;
  __shared__ double scr[kBK + 1];
  __shared__ __align__(16) T ys[NW][kSlice];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const T* __restrict__ v = IS_P3 ? a.s : a.p;
  T* __restrict__ out = IS_P3 ? a.traw : a.qraw;
  const int k = a.k;
  const int off = IS_P3 ? 0 : 1;   // P1: res[0] = (r~_0, q_raw), res[1 + j] = zeta_j; P3: res[j] = gamma_j
  const int nv = k + off;
  for (int t = blockIdx.x; t < a.tiles.ntiles; t += gridDim.x) {
    const int sys = a.tiles.sys[t];
    IterState* st = a.st + sys;
    if (!tile_active(st, IS_P3)) continue;
    Acc<T> col, rq;
    const int64_t sl0 = a.tiles.sl0[t];
    const int nsl = a.tiles.nsl[t];
    int w_nx = 0;
    int64_t sp_nx = 0;
    if (warp < nsl) {
      w_nx = __ldg(a.A.width + sl0 + warp);
      sp_nx = __ldg(a.A.slice_ptr + sl0 + warp);
    }
    for (int q = warp; q < nsl; q += NW) {
      const int64_t sl = sl0 + q;
      const int w = w_nx;
      const int64_t sp = sp_nx;
      if (q + NW < nsl) {
        w_nx = __ldg(a.A.width + sl + NW);
        sp_nx = __ldg(a.A.slice_ptr + sl + NW);
      }
      const int64_t row = sl * kSlice + lane;
      const T rv = IS_P3 ? T(0) : __ldg(a.rt0 + row);
      const T y = slice_row_product(a.A, v, w, sp, lane);
      out[row] = y;
      if (!IS_P3) rq.add(rv, y);
      ys[warp][lane] = y;
      __syncwarp();
      if (lane < k) col.add1(slice_col_dot(a.Chat + (int64_t)lane * a.ld + sl * kSlice, ys[warp]));
      __syncwarp();
    }
    if (!IS_P3) {
      const double w = warp_total(rq);
      if (lane == 0) sm.w[warp][0] = w;
    }
    if (lane < k) sm.w[warp][off + lane] = col.get();
    __syncthreads();
    for (int vv = threadIdx.x; vv < nv; vv += blockDim.x) {
      double sum = 0.0;
#pragma unroll
      for (int w = 0; w < NW; ++w) sum += sm.w[w][vv];
      sm.res[vv] = sum;
    }
    __syncthreads();
    if (tile_commit<kBK + 1>(sm, nv, a.partials, t, &st->ticket[IS_P3 ? P3 : P1].top, a.tiles.t0[sys],
                             a.tiles.nt[sys])) {
      if (warp == 0) {
        if (!IS_P3) finish_p1(st, sm.res, k, scr);
        else finish_p3(st, sm.res, k);
      }
    }
    __syncthreads();
  }
}

// P2: q = q_raw - C zeta;  s = r - alpha q;  ||s||^2 (finish_p2).
template <typename T, int KB>
__global__ void __launch_bounds__(kBlock) kb_p2(BatchArgs<T> a) {
  __shared__ ReduceSmem<1> sm;
  __shared__ T zs[kBK];
  __shared__ T s_alpha;
  const int k = KB > 0 ? a.k : 0;
  for (int t = blockIdx.x; t < a.tiles.ntiles; t += gridDim.x) {
    const int sys = a.tiles.sys[t];
    IterState* st = a.st + sys;
    if (!tile_active(st, false)) continue;
    if ((int)threadIdx.x < k) zs[threadIdx.x] = (T)st->zeta[threadIdx.x];
    if (threadIdx.x == 0) s_alpha = (T)st->alpha;
    __syncthreads();
    const T alpha = s_alpha;
    Acc<T> acc[1];
    const int64_t r0 = a.tiles.sl0[t] * kSlice;
    const int rows = a.tiles.nsl[t] * kSlice;
    for (int i = threadIdx.x; i < rows; i += blockDim.x) {
      const int64_t row = r0 + i;
      T qv = a.qraw[row];
#pragma unroll
      for (int j = 0; j < KB; ++j)
        if (j < k) qv = fma_t(-__ldg(a.C + (int64_t)j * a.ld + row), zs[j], qv);
      if (KB > 0) a.q[row] = qv;
      const T sv = fma_t(-alpha, qv, a.r[row]);
      a.s[row] = sv;
      acc[0].add(sv, sv);
    }
    block_sum<T, 1>(acc, 1, sm);
    if (tile_commit<1>(sm, 1, a.partials, t, &st->ticket[P2].top, a.tiles.t0[sys], a.tiles.nt[sys]))
      if (threadIdx.x < 32) finish_p2(st, sm.res);
    __syncthreads();
  }
}

// P4 (k > 0): t = t_raw - C gamma;  (s,t), (t,t), (r~_0,t), (r~_0,s) (finish_p4).
template <typename T, int KB>
__global__ void __launch_bounds__(kBlock) kb_p4(BatchArgs<T> a) {
  __shared__ ReduceSmem<4> sm;
  __shared__ T gs[kBK];
  const int k = a.k;
  for (int t = blockIdx.x; t < a.tiles.ntiles; t += gridDim.x) {
    const int sys = a.tiles.sys[t];
    IterState* st = a.st + sys;
    if (!tile_active(st, true)) continue;
    if (threadIdx.x < k) gs[threadIdx.x] = (T)st->gamma[threadIdx.x];
    __syncthreads();
    Acc<T> acc[4];
    const int64_t r0 = a.tiles.sl0[t] * kSlice;
    const int rows = a.tiles.nsl[t] * kSlice;
    for (int i = threadIdx.x; i < rows; i += blockDim.x) {
      const int64_t row = r0 + i;
      T tv = a.traw[row];
#pragma unroll
      for (int j = 0; j < KB; ++j)
        if (j < k) tv = fma_t(-__ldg(a.C + (int64_t)j * a.ld + row), gs[j], tv);
      a.t[row] = tv;
      const T sv = a.s[row], rv = __ldg(a.rt0 + row);
      acc[0].add(sv, tv);
      acc[1].add(tv, tv);
      acc[2].add(rv, tv);
      acc[3].add(rv, sv);
    }
    block_sum<T, 4>(acc, 4, sm);
    if (tile_commit<4>(sm, 4, a.partials, t, &st->ticket[P4].top, a.tiles.t0[sys], a.tiles.nt[sys]))
      if (threadIdx.x < 32) finish_p4(st, sm.res, k);
    __syncthreads();
  }
}

// P5: x += alpha p + omega s;  r = s - omega t;  p = r + beta (p - omega q);
// ||r||^2 (finish_p5).  After a half step: x += alpha p, r = s.
template <typename T, int KB>
__global__ void __launch_bounds__(kBlock) kb_p5(BatchArgs<T> a) {
  __shared__ ReduceSmem<1> sm;
  __shared__ T s_sc[4];
  __shared__ int s_half;
  for (int t = blockIdx.x; t < a.tiles.ntiles; t += gridDim.x) {
    const int sys = a.tiles.sys[t];
    IterState* st = a.st + sys;
    if (!tile_active(st, false)) continue;
    if (threadIdx.x == 0) {
      s_sc[0] = (T)st->alpha;
      s_sc[1] = (T)st->omega;
      s_sc[2] = (T)st->beta;
      s_half = st->half;
    }
    __syncthreads();
    const T alpha = s_sc[0], omega = s_sc[1], beta = s_sc[2];
    const bool half = s_half;
    const T* __restrict__ qsrc = KB > 0 ? a.q : a.qraw;
    Acc<T> acc[1];
    const int64_t r0 = a.tiles.sl0[t] * kSlice;
    const int rows = a.tiles.nsl[t] * kSlice;
    for (int i = threadIdx.x; i < rows; i += blockDim.x) {
      const int64_t row = r0 + i;
      const T pv = a.p[row], sv = a.s[row];
      if (half) {
        a.x[row] = fma_t(alpha, pv, a.x[row]);
        a.r[row] = sv;
        acc[0].add(sv, sv);
      } else {
        const T tv = a.t[row], qv = qsrc[row];
        a.x[row] = fma_t(omega, sv, fma_t(alpha, pv, a.x[row]));
        const T rv = fma_t(-omega, tv, sv);
        a.r[row] = rv;
        a.p[row] = fma_t(beta, fma_t(-omega, qv, pv), rv);
        acc[0].add(rv, rv);
      }
    }
    block_sum<T, 1>(acc, 1, sm);
    if (tile_commit<1>(sm, 1, a.partials, t, &st->ticket[P5].top, a.tiles.t0[sys], a.tiles.nt[sys]))
      if (threadIdx.x < 32) finish_p5(st, sm.res, a.k);
    __syncthreads();
  }
}

// Per-system reductions outside the iteration (setup, refinement): for
// every system, st[sys].red[j] = M_j^T v (j < km, M column-major with
// leading dimension ld) and st[sys].red[km + q] = (a_q, b_q) (q < nd).  FP64.
struct SysDots {
  const double* M;
  int km;
  const double* v;
  const double* pa[4];
  const double* pb[4];
  int nd;
};

__global__ void __launch_bounds__(kBlock) kb_sysdots(SysDots d, int64_t ld, IterState* st, double* partials,
                                                     BatchTiles tiles) {
  __shared__ ReduceSmem<kBNV> sm;
  for (int t = blockIdx.x; t < tiles.ntiles; t += gridDim.x) {
    const int sys = tiles.sys[t];
    Acc<double> acc[kBNV];
    const int64_t r0 = tiles.sl0[t] * kSlice;
    const int rows = tiles.nsl[t] * kSlice;
    for (int i = threadIdx.x; i < rows; i += blockDim.x) {
      const int64_t row = r0 + i;
      if (d.M) {
        const double vi = d.v[row];
#pragma unroll
        for (int j = 0; j < kBK; ++j)
          if (j < d.km) acc[j].add(d.M[(int64_t)j * ld + row], vi);
      }
#pragma unroll
      for (int q = 0; q < 4; ++q)
        if (q < d.nd) acc[kBK + q].add(d.pa[q][row], d.pb[q][row]);
    }
    block_sum<double, kBNV>(acc, kBNV, sm);
    IterState* s = st + sys;
    if (tile_commit<kBNV>(sm, kBNV, partials, t, &s->ticket[PGEN].top, tiles.t0[sys], tiles.nt[sys])) {
      if (threadIdx.x < d.km) s->red[threadIdx.x] = sm.res[threadIdx.x];
      if (threadIdx.x < d.nd) s->red[d.km + threadIdx.x] = sm.res[kBK + threadIdx.x];
    }
    __syncthreads();
  }
}

// y += sign * M c_sys for every system (M column-major, k columns); the
// coefficients are the system's st.red (XC = false) or st.xc (XC = true).
// Systems with skip[sys] != 0 (when skip is given) keep y unchanged.
template <bool XC>
__global__ void __launch_bounds__(kBlock) kb_gemv(double* __restrict__ y, const double* __restrict__ M, int64_t ld,
                                                  int k, double sign, const IterState* st, const int* skip,
                                                  BatchTiles tiles) {
  __shared__ double cs[kBK];
  for (int t = blockIdx.x; t < tiles.ntiles; t += gridDim.x) {
    const int sys = tiles.sys[t];
    if (skip && skip[sys]) continue;
    if (threadIdx.x < k) cs[threadIdx.x] = sign * (XC ? st[sys].xc[threadIdx.x] : st[sys].red[threadIdx.x]);
    __syncthreads();
    const int64_t r0 = tiles.sl0[t] * kSlice;
    const int rows = tiles.nsl[t] * kSlice;
    for (int i = threadIdx.x; i < rows; i += blockDim.x) {
      const int64_t row = r0 + i;
      double acc = 0.0;
      for (int j = 0; j < k; ++j) acc = fma(M[(int64_t)j * ld + row], cs[j], acc);
      y[row] += acc;
    }
    __syncthreads();
  }
}

// Out(:, c) = sum_j X(:, j) R_sys(j, c) for every system, R_sys the system's
// k x k matrix (column-major) in R[sys * kBK * kBK].  Out must not alias X.
__global__ void __launch_bounds__(kBlock) kb_gemm_sys(double* __restrict__ out, const double* __restrict__ X,
                                                      int64_t ld, int k, const double* __restrict__ R,
                                                      BatchTiles tiles) {
  __shared__ double rs[kBK * kBK];
  for (int t = blockIdx.x; t < tiles.ntiles; t += gridDim.x) {
    const int sys = tiles.sys[t];
    for (int e = threadIdx.x; e < k * k; e += blockDim.x) rs[e] = R[(size_t)sys * kBK * kBK + e];
    __syncthreads();
    const int64_t r0 = tiles.sl0[t] * kSlice;
    const int rows = tiles.nsl[t] * kSlice;
    for (int i = threadIdx.x; i < rows; i += blockDim.x) {
      const int64_t row = r0 + i;
      double xv[kBK];
#pragma unroll
      for (int j = 0; j < kBK; ++j) xv[j] = j < k ? X[(int64_t)j * ld + row] : 0.0;
      for (int c = 0; c < k; ++c) {
        double acc = 0.0;
#pragma unroll
        for (int j = 0; j < kBK; ++j)
          if (j < k) acc = fma(xv[j], rs[j + c * k], acc);
        out[(int64_t)c * ld + row] = acc;
      }
    }
    __syncthreads();
  }
}

// Compact (sum n_i) <-> padded (sum npad_i) layouts of stacked vectors or of
// stacked column blocks (cols columns per system: compact column c of system
// i starts at cofs_i * cols + c * n_i; padded column c at c * ld).
struct SysLayout {
  const int64_t* row0;   // first padded row of each system
  const int64_t* n;      // rows of each system
  const int64_t* cofs;   // first compact row of each system
};

template <bool TO_PADDED>
__global__ void __launch_bounds__(kBlock) kb_relayout(double* __restrict__ padded, double* __restrict__ compact,
                                                      int cols, int64_t ld, SysLayout L, BatchTiles tiles) {
  for (int t = blockIdx.x; t < tiles.ntiles; t += gridDim.x) {
    const int sys = tiles.sys[t];
    const int64_t r0 = tiles.sl0[t] * kSlice;
    const int rows = tiles.nsl[t] * kSlice;
    const int64_t row0 = L.row0[sys], ni = L.n[sys], cofs = L.cofs[sys];
    for (int c = 0; c < cols; ++c)
      for (int i = threadIdx.x; i < rows; i += blockDim.x) {
        const int64_t row = r0 + i, l = row - row0;
        const int64_t ci = cofs * cols + (int64_t)c * ni + l;
        if (TO_PADDED) padded[(int64_t)c * ld + row] = l < ni ? compact[ci] : 0.0;
        else if (l < ni) compact[ci] = padded[(int64_t)c * ld + row];
      }
  }
}

// What the host reads of every system after a graph replay.
struct SysFlag {
  int32_t done, status, iter, half;
  double rnorm2, rmax2;
};

__global__ void kb_flags(const IterState* st, int nsys, SysFlag* flags) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < nsys; i += gridDim.x * blockDim.x)
    flags[i] = SysFlag{st[i].done, st[i].status, st[i].iter, st[i].half, st[i].rnorm2, st[i].rmax2};
}

// Per-system commands of the mixed mode's residual replacement.
enum SysCmd { kCmdNone = 0, kCmdFold = 1, kCmdDrop = 2 };

// cmd[sys] == kCmdFold: x += fx - U x_c (the inner increment of the FP32
// solve since the last fold, eq. (3.5)'s final correction); kCmdDrop: the
// increment is discarded (a non-finite inner iterate).  Both zero fx.
__global__ void __launch_bounds__(kBlock) kb_fold(double* __restrict__ x, float* __restrict__ fx,
                                                  const double* __restrict__ U, int64_t ld, int k,
                                                  const IterState* st, const int* cmd, BatchTiles tiles) {
  __shared__ double cs[kBK];
  for (int t = blockIdx.x; t < tiles.ntiles; t += gridDim.x) {
    const int sys = tiles.sys[t];
    const int c = cmd[sys];
    if (c == kCmdNone) continue;
    if (threadIdx.x < k) cs[threadIdx.x] = st[sys].xc[threadIdx.x];
    __syncthreads();
    const int64_t r0 = tiles.sl0[t] * kSlice;
    const int rows = tiles.nsl[t] * kSlice;
    for (int i = threadIdx.x; i < rows; i += blockDim.x) {
      const int64_t row = r0 + i;
      if (c == kCmdFold) {
        double d = (double)fx[row];
        for (int j = 0; j < k; ++j) d = fma(-U[(int64_t)j * ld + row], cs[j], d);
        x[row] += d;
      }
      fx[row] = 0.f;
    }
    __syncthreads();
  }
}

// For every system with cmd[sys] != kCmdNone (cmd may be null): x_c = 0.
// run[sys] (run may be null): 1 = iterate again (done = half = 0) with the
// residual peak restarted at rmax2[sys], 2 = stop (done = 1), 3 = carry on
// with the peak restarted at rmax2[sys].
__global__ void kb_state_cmd(IterState* st, int nsys, int k, const int* cmd, const int* run, const double* rmax2) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < nsys; i += gridDim.x * blockDim.x) {
    if (cmd && cmd[i] != kCmdNone)
      for (int j = 0; j < k; ++j) st[i].xc[j] = 0.0;
    const int c = run ? run[i] : 0;
    if (c == 1) {
      st[i].done = 0;
      st[i].half = 0;
    } else if (c == 2) {
      st[i].done = 1;
    }
    if ((c == 1 || c == 3) && rmax2) st[i].rmax2 = rmax2[i];
  }
}

// dst = src over the rows of the systems with mask[sys] != 0.
__global__ void __launch_bounds__(kBlock) kb_copy_rows(double* __restrict__ dst, const double* __restrict__ src,
                                                       const int* mask, BatchTiles tiles) {
  for (int t = blockIdx.x; t < tiles.ntiles; t += gridDim.x) {
    if (!mask[tiles.sys[t]]) continue;
    const int64_t r0 = tiles.sl0[t] * kSlice;
    const int rows = tiles.nsl[t] * kSlice;
    for (int i = threadIdx.x; i < rows; i += blockDim.x) dst[r0 + i] = src[r0 + i];
  }
}

// out = (float) in over the rows of the systems with mask[sys] != 0.
__global__ void __launch_bounds__(kBlock) kb_to_float(float* __restrict__ out, const double* __restrict__ in,
                                                      const int* mask, BatchTiles tiles) {
  for (int t = blockIdx.x; t < tiles.ntiles; t += gridDim.x) {
    if (!mask[tiles.sys[t]]) continue;
    const int64_t r0 = tiles.sl0[t] * kSlice;
    const int rows = tiles.nsl[t] * kSlice;
    for (int i = threadIdx.x; i < rows; i += blockDim.x) out[r0 + i] = (float)in[r0 + i];
  }
}

}  // namespace
}  // namespace rb

// ============================================================ host side
using rb::BatchArgs;
using rb::BatchTiles;
using rb::IterState;
using rb::SellBuf;

struct rb_batch_ctx {
  rb_opts o{};
  cudaStream_t us = nullptr, cs = nullptr;
  int nsm = 0;
  int S = 0;
  std::vector<int64_t> n, npad, row0, cofs, nnz_sys;
  int64_t NP = 0, NC = 0, nnz = 0;   // padded rows, compact rows, nonzeros
  int32_t *rp = nullptr, *ci = nullptr, *trp = nullptr, *tci = nullptr;
  int64_t* tsrc = nullptr;
  double *cv = nullptr, *tcv = nullptr;
  SellBuf<double> A, AT;
  SellBuf<float> A32;
  bool have = false;
  // work list
  int tile_slices = 0, ctas_per_sm = 0, grid = 0, ntiles = 0;
  rb::PassGrids pg64[2]{}, pg32[2]{};   // per-pass grids: [plain, recycled]
  double tune_ms = 0.0;
  int32_t *t_sys = nullptr, *t_nsl = nullptr, *s_t0 = nullptr, *s_nt = nullptr;
  int64_t* t_sl0 = nullptr;
  int64_t *d_row0 = nullptr, *d_n = nullptr, *d_cofs = nullptr;
  // recycle space (fixed), padded columns of ld = NP
  int kin = 0, k = 0;
  bool setup_owed = false;
  double *U = nullptr, *C = nullptr, *Ct = nullptr, *Chat = nullptr, *dR = nullptr;
  float *fU = nullptr, *fC = nullptr, *fChat = nullptr;
  std::vector<int> k_used;
  // vectors
  double *b = nullptr, *x = nullptr, *r = nullptr, *stage = nullptr;
  double *p = nullptr, *s = nullptr, *q = nullptr, *t = nullptr, *qraw = nullptr, *traw = nullptr, *rt0 = nullptr;
  float *fx = nullptr, *fr = nullptr, *fp = nullptr, *fs = nullptr, *fq = nullptr, *ft = nullptr,
        *fqraw = nullptr, *ftraw = nullptr, *frt0 = nullptr;
  IterState* st = nullptr;
  IterState* hst = nullptr;
  double* partials = nullptr;
  int* dflags = nullptr;     // device validation flag
  int* dskip = nullptr;      // per-system "already converged" mask of a restart
  int *dcmd = nullptr, *dres = nullptr;   // per-system fold / resume commands
  double* drm = nullptr;                  // per-system residual peaks after a replacement
  rb::SysFlag* dsf = nullptr;             // flags gathered after each graph replay
  rb::SysFlag* hsf = nullptr;
  // captured iteration graphs (FP64, FP32) and the layout they were made for
  cudaGraphExec_t g64 = nullptr, g32 = nullptr;
  int g_key64 = -1, g_key32 = -1;
};

namespace rb {
namespace {

template <typename T>
int balloc(T** p, int64_t count) {
  cudaFree(*p);
  *p = nullptr;
  if (count <= 0) count = 1;
  const cudaError_t e = cudaMalloc(p, sizeof(T) * (size_t)count);
  if (e != cudaSuccess) return e == cudaErrorMemoryAllocation ? RB_ENOMEM : RB_ECUDA;
  return cudaMemset(*p, 0, sizeof(T) * (size_t)count) == cudaSuccess ? RB_OK : RB_ECUDA;
}

BatchTiles tiles_of(rb_batch_ctx* h) {
  return BatchTiles{h->t_sys, h->t_sl0, h->t_nsl, h->s_t0, h->s_nt, h->ntiles};
}

void drop_graphs(rb_batch_ctx* h) {
  if (h->g64) cudaGraphExecDestroy(h->g64);
  if (h->g32) cudaGraphExecDestroy(h->g32);
  h->g64 = h->g32 = nullptr;
  h->g_key64 = h->g_key32 = -1;
}

// Grids of the five pass kernels of one precision: each takes
// min(ctas_per_sm, its own resident blocks per SM) blocks per SM, so that a
// grid-stride work list never starts a second wave of blocks that wait for
// the first to finish all their tiles, and a light kernel is not held to a
// heavier one's occupancy.
template <typename T>
PassGrids pass_grids(int ctas_per_sm, int nsm, int ntiles, bool recycled) {
  auto grid = [&](const void* f) {
    int b = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, f, kBlock, 0) != cudaSuccess || b < 1) b = 1;
    return std::max(1, std::min(ntiles, std::min(ctas_per_sm, b) * nsm));
  };
  PassGrids g{};
  if (recycled) {
    g.g[0] = grid((const void*)kb_spmv_proj<T, false>);
    g.g[1] = grid((const void*)kb_p2<T, kBK>);
    g.g[2] = grid((const void*)kb_spmv_proj<T, true>);
    g.g[3] = grid((const void*)kb_p4<T, kBK>);
    g.g[4] = grid((const void*)kb_p5<T, kBK>);
  } else {
    g.g[0] = grid((const void*)kb_spmv_plain<T, false>);
    g.g[1] = grid((const void*)kb_p2<T, 0>);
    g.g[2] = grid((const void*)kb_spmv_plain<T, true>);
    g.g[3] = g.g[2];
    g.g[4] = grid((const void*)kb_p5<T, 0>);
  }
  return g;
}

// Work list for tiles of `ts` slices: every system's slices split into tiles.
int build_tiles(rb_batch_ctx* h, int ts, int ctas_per_sm) {
  std::vector<int32_t> tsys, tnsl, t0(h->S), nt(h->S);
  std::vector<int64_t> tsl0;
  for (int i = 0; i < h->S; ++i) {
    const int64_t sl_first = h->row0[i] / kSlice, nsl = h->npad[i] / kSlice;
    t0[i] = (int32_t)tsys.size();
    for (int64_t q = 0; q < nsl; q += ts) {
      tsys.push_back(i);
      tsl0.push_back(sl_first + q);
      tnsl.push_back((int32_t)std::min<int64_t>(ts, nsl - q));
    }
    nt[i] = (int32_t)tsys.size() - t0[i];
  }
  h->ntiles = (int)tsys.size();
  int rc;
  if ((rc = balloc(&h->t_sys, h->ntiles)) || (rc = balloc(&h->t_nsl, h->ntiles)) ||
      (rc = balloc(&h->t_sl0, h->ntiles)) || (rc = balloc(&h->s_t0, h->S)) || (rc = balloc(&h->s_nt, h->S)) ||
      (rc = balloc(&h->partials, (int64_t)h->ntiles * kBNV)))
    return rc;
  RB_CUDA_TRY(cudaMemcpy(h->t_sys, tsys.data(), sizeof(int32_t) * h->ntiles, cudaMemcpyHostToDevice));
  RB_CUDA_TRY(cudaMemcpy(h->t_nsl, tnsl.data(), sizeof(int32_t) * h->ntiles, cudaMemcpyHostToDevice));
  RB_CUDA_TRY(cudaMemcpy(h->t_sl0, tsl0.data(), sizeof(int64_t) * h->ntiles, cudaMemcpyHostToDevice));
  RB_CUDA_TRY(cudaMemcpy(h->s_t0, t0.data(), sizeof(int32_t) * h->S, cudaMemcpyHostToDevice));
  RB_CUDA_TRY(cudaMemcpy(h->s_nt, nt.data(), sizeof(int32_t) * h->S, cudaMemcpyHostToDevice));
  h->tile_slices = ts;
  h->ctas_per_sm = ctas_per_sm;
  h->grid = std::max(1, std::min(h->ntiles, ctas_per_sm * h->nsm));
  for (int rec = 0; rec < 2; ++rec) {
    h->pg64[rec] = pass_grids<double>(ctas_per_sm, h->nsm, h->ntiles, rec != 0);
    h->pg32[rec] = pass_grids<float>(ctas_per_sm, h->nsm, h->ntiles, rec != 0);
  }
  drop_graphs(h);
  return RB_OK;
}

template <typename T>
BatchArgs<T> batch_args(rb_batch_ctx* h);

template <>
BatchArgs<double> batch_args<double>(rb_batch_ctx* h) {
  BatchArgs<double> a{};
  a.A = h->A.view();
  a.Chat = h->Chat;
  a.C = h->C;
  a.ld = h->NP;
  a.k = h->k;
  a.rt0 = h->rt0;
  a.x = h->x;   // the FP64 mode iterates on x, r directly
  a.r = h->r;
  a.p = h->p;
  a.s = h->s;
  a.qraw = h->qraw;
  a.traw = h->traw;
  a.q = h->k > 0 ? h->q : h->qraw;
  a.t = h->k > 0 ? h->t : h->traw;
  a.st = h->st;
  a.partials = h->partials;
  a.tiles = tiles_of(h);
  return a;
}

template <>
BatchArgs<float> batch_args<float>(rb_batch_ctx* h) {
  BatchArgs<float> a{};
  a.A = h->A32.view();
  a.Chat = h->fChat;
  a.C = h->fC;
  a.ld = h->NP;
  a.k = h->k;
  a.rt0 = h->frt0;
  a.x = h->fx;
  a.r = h->fr;
  a.p = h->fp;
  a.s = h->fs;
  a.qraw = h->fqraw;
  a.traw = h->ftraw;
  a.q = h->k > 0 ? h->fq : h->fqraw;
  a.t = h->k > 0 ? h->ft : h->ftraw;
  a.st = h->st;
  a.partials = h->partials;
  a.tiles = tiles_of(h);
  return a;
}

template <typename T, int KB>
cudaError_t launch_iteration_kb(const BatchArgs<T>& a, const PassGrids& g, cudaStream_t s) {
  if (KB > 0) kb_spmv_proj<T, false><<<g.g[0], kBlock, 0, s>>>(a);
  else kb_spmv_plain<T, false><<<g.g[0], kBlock, 0, s>>>(a);
  kb_p2<T, KB><<<g.g[1], kBlock, 0, s>>>(a);
  if (KB > 0) kb_spmv_proj<T, true><<<g.g[2], kBlock, 0, s>>>(a);
  else kb_spmv_plain<T, true><<<g.g[2], kBlock, 0, s>>>(a);
  if (KB > 0) kb_p4<T, KB><<<g.g[3], kBlock, 0, s>>>(a);
  kb_p5<T, KB><<<g.g[4], kBlock, 0, s>>>(a);
  return cudaGetLastError();
}

template <typename T>
const PassGrids& grids_of(rb_batch_ctx* h) {
  const int rec = h->k > 0 ? 1 : 0;
  return std::is_same<T, float>::value ? h->pg32[rec] : h->pg64[rec];
}

template <typename T>
cudaError_t launch_iteration_b(const BatchArgs<T>& a, const PassGrids& g, cudaStream_t s) {
  count_launches(a.k > 0 ? 5 : 4);
  return a.k > 0 ? launch_iteration_kb<T, kBK>(a, g, s) : launch_iteration_kb<T, 0>(a, g, s);
}

int poll_iters_b(rb_batch_ctx* h) { return h->o.poll > 0 ? h->o.poll : 8; }

// Graph of poll iterations plus the gather of the systems' flags.  After
// each replay `hook` (if given) may act on the flags (fold, replace, resume
// systems); the loop ends once every system reports done.
template <typename T>
int iterate_b(rb_batch_ctx* h, int64_t max_itn_all, const std::function<int()>& hook = nullptr) {
  cudaGraphExec_t* g = std::is_same<T, float>::value ? &h->g32 : &h->g64;
  int* key = std::is_same<T, float>::value ? &h->g_key32 : &h->g_key64;
  const int want = h->k * 100000 + h->tile_slices * 100 + h->ctas_per_sm;
  if (!*g || *key != want) {
    if (*g) cudaGraphExecDestroy(*g);
    *g = nullptr;
    const BatchArgs<T> a = batch_args<T>(h);
    RB_CUDA_TRY(cudaStreamBeginCapture(h->cs, cudaStreamCaptureModeThreadLocal));
    cudaError_t e = cudaSuccess;
    for (int it = 0; it < poll_iters_b(h) && e == cudaSuccess; ++it) e = launch_iteration_b<T>(a, grids_of<T>(h), h->cs);
    if (e == cudaSuccess) {
      kb_flags<<<(h->S + 255) / 256, 256, 0, h->cs>>>(h->st, h->S, h->dsf);
      e = cudaGetLastError();
    }
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(h->hsf, h->dsf, sizeof(SysFlag) * h->S, cudaMemcpyDeviceToHost, h->cs);
    cudaGraph_t graph = nullptr;
    const cudaError_t ec = cudaStreamEndCapture(h->cs, &graph);
    if (e != cudaSuccess || ec != cudaSuccess) {
      if (graph) cudaGraphDestroy(graph);
      return RB_ECUDA;
    }
    const cudaError_t ei = cudaGraphInstantiate(g, graph, 0);
    cudaGraphDestroy(graph);
    if (ei != cudaSuccess) return RB_ECUDA;
    *key = want;
  }
  // every system stops by its max_itn (finish_p5), so this bound only
  // guards against a state that never reports done
  for (int64_t launch = 0;; ++launch) {
    if (launch > max_itn_all / poll_iters_b(h) + 4) return RB_ETIMEOUT;
    RB_CUDA_TRY(cudaGraphLaunch(*g, h->us));
    count_launches((long long)poll_iters_b(h) * (h->k > 0 ? 5 : 4) + 1);
    RB_CUDA_TRY(cudaStreamSynchronize(h->us));
    if (hook) {
      const int rc = hook();
      if (rc) return rc;
    }
    bool all = true;
    for (int i = 0; i < h->S && all; ++i) all = h->hsf[i].done != 0;
    if (all) return RB_OK;
  }
}

int sync_b(rb_batch_ctx* h) {
  RB_CUDA_TRY(cudaStreamSynchronize(h->us));
  return RB_OK;
}

// Per-system reductions into st[i].red, copied back to hst[i].red.
int sysdots(rb_batch_ctx* h, const SysDots& d, bool read_back = true) {
  count_launches(1);
  kb_sysdots<<<h->grid, kBlock, 0, h->us>>>(d, h->NP, h->st, h->partials, tiles_of(h));
  RB_CUDA_TRY(cudaGetLastError());
  if (!read_back) return RB_OK;
  RB_CUDA_TRY(cudaMemcpyAsync(h->hst, h->st, sizeof(IterState) * h->S, cudaMemcpyDeviceToHost, h->us));
  return sync_b(h);
}

int gemv_b(rb_batch_ctx* h, double* y, const double* M, double sign, bool xc, const int* skip = nullptr) {
  if (h->k == 0) return RB_OK;
  count_launches(1);
  if (xc) kb_gemv<true><<<h->grid, kBlock, 0, h->us>>>(y, M, h->NP, h->k, sign, h->st, skip, tiles_of(h));
  else kb_gemv<false><<<h->grid, kBlock, 0, h->us>>>(y, M, h->NP, h->k, sign, h->st, skip, tiles_of(h));
  RB_CUDA_TRY(cudaGetLastError());
  return RB_OK;
}

SysLayout layout_of(rb_batch_ctx* h) { return SysLayout{h->d_row0, h->d_n, h->d_cofs}; }

}  // namespace
}  // namespace rb

namespace rb {
namespace {

// Autotuner: time the SpMV + projection pass (P1) for each candidate tile size
// and CTAs per SM on the current matrices and space, every system active,
// and keeps the fastest configuration that gives every block of P1 at least
// kTilesPerBlock tiles (the fastest overall when none does): systems converge
// at different times, and the tiles of those still iterating must stay
// spread over many blocks, which the all-active timing does not see (256
// systems of the 2D sweep: 512-slice tiles, 1.2 per block, timed 2% faster
// than 128-slice tiles, 4.6 per block, but solved 6-16% slower).  RB_TIMING
// in the environment prints every candidate.
int autotune(rb_batch_ctx* h) {
  const int cand_ts[] = {16, 32, 64, 128, 256, 512, 1024};
  const int cand_cps[] = {2, 4, 8};
  const bool print = getenv("RB_TIMING") != nullptr;
  constexpr int kTilesPerBlock = 4;
  struct Cand {
    int ts, cps;
    double ms;
    bool spread;
  };
  std::vector<Cand> cands;
  double best = 1e30;
  cudaEvent_t e0, e1;
  RB_CUDA_TRY(cudaEventCreate(&e0));
  RB_CUDA_TRY(cudaEventCreate(&e1));
  const bool f32 = h->o.precision == RB_MIXED;
  for (int ts : cand_ts) {
    for (int cps : cand_cps) {
      int rc = build_tiles(h, ts, cps);
      if (rc) return rc;
      float total = 0.f;
      for (int rep = 0; rep < 4; ++rep) {
        RB_CUDA_TRY(cudaMemsetAsync(h->st, 0, sizeof(IterState) * h->S, h->us));
        RB_CUDA_TRY(cudaEventRecord(e0, h->us));
        if (f32) {
          const BatchArgs<float> a = batch_args<float>(h);
          const int g = grids_of<float>(h).g[0];
          if (h->k > 0) kb_spmv_proj<float, false><<<g, kBlock, 0, h->us>>>(a);
          else kb_spmv_plain<float, false><<<g, kBlock, 0, h->us>>>(a);
        } else {
          const BatchArgs<double> a = batch_args<double>(h);
          const int g = grids_of<double>(h).g[0];
          if (h->k > 0) kb_spmv_proj<double, false><<<g, kBlock, 0, h->us>>>(a);
          else kb_spmv_plain<double, false><<<g, kBlock, 0, h->us>>>(a);
        }
        count_launches(1);
        RB_CUDA_TRY(cudaGetLastError());
        RB_CUDA_TRY(cudaEventRecord(e1, h->us));
        RB_CUDA_TRY(cudaEventSynchronize(e1));
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        if (rep > 0) total += ms;
      }
      const double avg = total / 3.0;
      if (print) fprintf(stderr, "rb_batch_tune tile_slices %3d ctas_per_sm %d tiles %7d  %.4f ms\n", ts, cps, h->ntiles, avg);
      const int g1 = f32 ? grids_of<float>(h).g[0] : grids_of<double>(h).g[0];
      const bool spread = h->ntiles >= kTilesPerBlock * g1;
      cands.push_back({ts, cps, avg, spread});
      if (spread) best = std::min(best, avg);
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  const bool any_spread = best < 1e30;
  int bts = cands[0].ts, bcps = cands[0].cps;
  double bms = 1e30;
  for (const Cand& c : cands)
    if ((c.spread || !any_spread) && c.ms < bms) {
      bms = c.ms;
      bts = c.ts;
      bcps = c.cps;
    }
  h->tune_ms = bms;
  RB_CUDA_TRY(cudaMemsetAsync(h->st, 0, sizeof(IterState) * h->S, h->us));
  return build_tiles(h, bts, bcps);
}

// Per-system recycle setup (Sec. 3) for the kin columns in U: C = A U,
// C~ = A^T U (U~ = U), M_i = C~_i^T C_i, SVD, C-hat_i = C~_i (M_i^+)^T with the
// pseudo-inverse of the singular values above the drop tolerance (rank
// deficiency needs no rotation: C M^+ C~^T is still the projector).
int batch_setup(rb_batch_ctx* h) {
  h->setup_owed = false;
  h->k = 0;
  drop_graphs(h);
  if (h->kin == 0) return RB_OK;
  const int kin = h->kin;
  const int64_t ld = h->NP;
  const int gs = std::max(1, 4 * h->nsm);
  for (int j = 0; j < kin; ++j) {
    RB_CUDA_TRY(spmv<double>(h->A.view(), h->U + j * ld, h->C + j * ld, 1.0, 0.0, gs, h->us));
    RB_CUDA_TRY(spmv<double>(h->AT.view(), h->U + j * ld, h->Ct + j * ld, 1.0, 0.0, gs, h->us));
  }
  h->k = kin;   // the reductions below use k columns
  std::vector<double> M((size_t)h->S * kin * kin);
  for (int j = 0; j < kin; ++j) {   // column j of every M_i: C~_i^T C_i(:, j)
    SysDots d{};
    d.M = h->Ct;
    d.km = kin;
    d.v = h->C + j * ld;
    int rc = sysdots(h, d);
    if (rc) return rc;
    for (int i = 0; i < h->S; ++i)
      for (int r = 0; r < kin; ++r) M[(size_t)i * kin * kin + r + (size_t)j * kin] = h->hst[i].red[r];
  }
  const double drop = h->o.precision == RB_MIXED ? 1e-6 : 1e-12;
  std::vector<double> R((size_t)h->S * kBK * kBK, 0.0), P((size_t)kin * kin), Q((size_t)kin * kin), sig(kin);
  h->k_used.assign(h->S, 0);
  for (int i = 0; i < h->S; ++i) {
    const double* Mi = &M[(size_t)i * kin * kin];
    for (int e = 0; e < kin * kin; ++e)
      if (!std::isfinite(Mi[e])) return RB_ENONFINITE;
    svd_small(kin, Mi, P.data(), sig.data(), Q.data());
    int kk = 0;
    if (sig[0] > 0)
      while (kk < kin && sig[kk] >= drop * sig[0]) ++kk;
    h->k_used[i] = kk;
    double* Ri = &R[(size_t)i * kBK * kBK];   // Mpt = P_kk S^-1 Q_kk^T, k x k column-major (ld k)
    for (int c = 0; c < kin; ++c)
      for (int r = 0; r < kin; ++r) {
        double acc = 0.0;
        for (int j = 0; j < kk; ++j) acc += P[r + (size_t)j * kin] * Q[c + (size_t)j * kin] / sig[j];
        Ri[r + c * kin] = acc;
      }
  }
  RB_CUDA_TRY(cudaMemcpyAsync(h->dR, R.data(), sizeof(double) * R.size(), cudaMemcpyHostToDevice, h->us));
  count_launches(1);
  kb_gemm_sys<<<h->grid, kBlock, 0, h->us>>>(h->Chat, h->Ct, ld, kin, h->dR, tiles_of(h));
  RB_CUDA_TRY(cudaGetLastError());
  if (h->o.precision == RB_MIXED) {   // the FP32 copies exist in the mixed mode only
    RB_CUDA_TRY(to_float(h->U, h->fU, ld * kin, h->us));
    RB_CUDA_TRY(to_float(h->C, h->fC, ld * kin, h->us));
    RB_CUDA_TRY(to_float(h->Chat, h->fChat, ld * kin, h->us));
  }
  return sync_b(h);
}

// Start of Alg. 2 for every system from xv (eq. (3.5)): r = rhs - A xv with the
// projections, the per-system shadow r~_0 (SplitMix64 on the system's own
// row index, the generator of the single-system path), the initial states.
// thresh[i] is the system's convergence threshold on ||r||^2; systems with
// skip[i] start done.  The vectors are FP64; the caller converts for FP32.
int batch_start(rb_batch_ctx* h, const double* rhs, double* xv, const std::vector<double>& thresh2,
                const std::vector<char>& skip, const std::vector<int>& max_itn, uint64_t seed) {
  const int64_t ld = h->NP;
  const int gs = std::max(1, 4 * h->nsm);
  RB_CUDA_TRY(cudaMemcpyAsync(h->r, rhs, sizeof(double) * ld, cudaMemcpyDeviceToDevice, h->us));
  RB_CUDA_TRY(spmv<double>(h->A.view(), xv, h->r, -1.0, 1.0, gs, h->us));
  int rc;
  if (h->k > 0) {
    // a skipped system keeps xv: the oblique projection could raise the
    // residual of a system that has already converged
    std::vector<int> sk(skip.begin(), skip.end());
    RB_CUDA_TRY(cudaMemcpyAsync(h->dskip, sk.data(), sizeof(int) * h->S, cudaMemcpyHostToDevice, h->us));
    SysDots d{};
    d.M = h->Chat; d.km = h->k; d.v = h->r;
    if ((rc = sysdots(h, d, false))) return rc;
    if ((rc = gemv_b(h, xv, h->U, 1.0, false, h->dskip))) return rc;
    RB_CUDA_TRY(cudaStreamSynchronize(h->us));   // sk is read by the copy above
    if ((rc = gemv_b(h, h->r, h->C, -1.0, false))) return rc;
  }
  for (int i = 0; i < h->S; ++i)
    RB_CUDA_TRY(shadow(h->rt0 + h->row0[i], h->n[i], h->npad[i], seed, h->us));
  if (h->k > 0) {
    SysDots d{};
    d.M = h->C; d.km = h->k; d.v = h->rt0;
    if ((rc = sysdots(h, d, false))) return rc;
    if ((rc = gemv_b(h, h->rt0, h->Chat, -1.0, false))) return rc;
  }
  SysDots d{};
  d.M = h->k > 0 ? h->C : nullptr; d.km = h->k; d.v = h->rt0;
  d.nd = 2;
  d.pa[0] = h->rt0; d.pb[0] = h->r;
  d.pa[1] = h->r; d.pb[1] = h->r;
  if ((rc = sysdots(h, d))) return rc;
  for (int i = 0; i < h->S; ++i) {
    IterState& s = h->hst[i];
    const double rho = s.red[h->k], rn2 = s.red[h->k + 1];
    double cr[kBK];
    for (int j = 0; j < h->k; ++j) cr[j] = s.red[j];
    std::memset(&s, 0, sizeof(IterState));
    s.k = h->k;
    for (int j = 0; j < h->k; ++j) s.cr[j] = cr[j];
    s.rho = rho;
    s.rnorm2 = rn2;
    s.rmax2 = rn2;
    s.thresh2 = thresh2[i];
    s.max_itn = max_itn[i];
    s.status = RB_OK;
    if (skip[i] || rn2 <= thresh2[i]) s.done = 1;
    else if (!std::isfinite(rho) || !std::isfinite(rn2)) { s.status = RB_ENONFINITE; s.done = 1; }
    else if (rho == 0.0) { s.status = RB_EBREAKDOWN_RHO; s.done = 1; }
  }
  RB_CUDA_TRY(cudaMemcpyAsync(h->st, h->hst, sizeof(IterState) * h->S, cudaMemcpyHostToDevice, h->us));
  RB_CUDA_TRY(cudaMemcpyAsync(h->p, h->r, sizeof(double) * ld, cudaMemcpyDeviceToDevice, h->us));
  return sync_b(h);
}

// ||b_i - A_i x_i||^2 and ||b_i||^2 of every system into out (FP64).
int true_residuals(rb_batch_ctx* h, std::vector<double>& rn2, std::vector<double>& bn2) {
  const int gs = std::max(1, 4 * h->nsm);
  RB_CUDA_TRY(cudaMemcpyAsync(h->r, h->b, sizeof(double) * h->NP, cudaMemcpyDeviceToDevice, h->us));
  RB_CUDA_TRY(spmv<double>(h->A.view(), h->x, h->r, -1.0, 1.0, gs, h->us));
  SysDots d{};
  d.nd = 2;
  d.pa[0] = h->r; d.pb[0] = h->r;
  d.pa[1] = h->b; d.pb[1] = h->b;
  int rc = sysdots(h, d);
  if (rc) return rc;
  rn2.resize(h->S);
  bn2.resize(h->S);
  for (int i = 0; i < h->S; ++i) {
    rn2[i] = h->hst[i].red[0];
    bn2[i] = h->hst[i].red[1];
  }
  return RB_OK;
}

}  // namespace
}  // namespace rb

// ============================================================ C ABI
using namespace rb;

extern "C" int rbicgstab_batch_create(rb_batch* out, const rb_opts* opts) {
  if (!out) return RB_EINVAL;
  *out = nullptr;
  rb_opts o = opts ? *opts : rb_opts{};
  if (o.tol == 0) o.tol = 1e-8;
  if (o.shadow_seed == 0) o.shadow_seed = 0x5EED;
  if (o.k_max < 0 || o.k_max > kBK || !(o.tol > 0) || o.max_itn < 0 || o.poll < 0 ||
      (o.precision != RB_FP64 && o.precision != RB_MIXED))
    return RB_EINVAL;
  rb_batch_ctx* h = new rb_batch_ctx();
  h->o = o;
  h->us = (cudaStream_t)o.cuda_stream;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&h->nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
      cudaStreamCreateWithFlags(&h->cs, cudaStreamNonBlocking) != cudaSuccess) {
    delete h;
    return RB_ECUDA;
  }
  *out = h;
  return RB_OK;
}

extern "C" int rbicgstab_batch_destroy(rb_batch h) {
  if (!h) return RB_OK;
  cudaStreamSynchronize(h->us);
  drop_graphs(h);
  sell_free(&h->A);
  sell_free(&h->AT);
  cudaFree(h->A32.val);
  void* ptrs[] = {h->rp, h->ci, h->trp, h->tci, h->tsrc, h->cv, h->tcv, h->t_sys, h->t_nsl, h->s_t0, h->s_nt,
                  h->t_sl0, h->d_row0, h->d_n, h->d_cofs, h->U, h->C, h->Ct, h->Chat, h->dR, h->fU, h->fC, h->fChat,
                  h->b, h->x, h->r, h->stage, h->p, h->s, h->q, h->t, h->qraw, h->traw, h->rt0, h->fx, h->fr, h->fp,
                  h->fs, h->fq, h->ft, h->fqraw, h->ftraw, h->frt0, h->st, h->partials, h->dflags, h->dskip, h->dcmd, h->dres, h->dsf, h->drm};
  for (void* p : ptrs) cudaFree(p);
  if (h->hst) cudaFreeHost(h->hst);
  if (h->hsf) cudaFreeHost(h->hsf);
  if (h->cs) cudaStreamDestroy(h->cs);
  delete h;
  return RB_OK;
}

extern "C" int rbicgstab_batch_set_matrices(rb_batch h, int32_t nsys, const int64_t* n, const int32_t* row_ptr,
                                             const int32_t* col, const double* val) {
  if (!h || nsys < 1 || !n || !row_ptr || !col || !val) return RB_EINVAL;
  // the padded block-diagonal CSR (host), every system's rows padded to 32
  h->S = nsys;
  h->n.assign(n, n + nsys);
  h->npad.resize(nsys);
  h->row0.resize(nsys);
  h->cofs.resize(nsys);
  h->nnz_sys.resize(nsys);
  int64_t NP = 0, NC = 0, nnz = 0, rpo = 0;
  for (int i = 0; i < nsys; ++i) {
    if (n[i] < 1) return RB_EINVAL;
    h->npad[i] = (n[i] + kSlice - 1) / kSlice * kSlice;
    h->row0[i] = NP;
    h->cofs[i] = NC;
    const int32_t* rpi = row_ptr + rpo;
    if (rpi[0] != 0) return RB_EBADCSR;
    for (int64_t r = 0; r < n[i]; ++r)
      if (rpi[r + 1] < rpi[r]) return RB_EBADCSR;
    h->nnz_sys[i] = rpi[n[i]];
    NP += h->npad[i];
    NC += n[i];
    nnz += rpi[n[i]];
    rpo += n[i] + 1;
  }
  if (NP >= INT32_MAX || nnz >= INT32_MAX) return RB_EINVAL;
  std::vector<int32_t> grp(NP + 1), gci(nnz);
  int64_t ebase = 0;
  rpo = 0;
  for (int i = 0; i < nsys; ++i) {
    const int32_t* rpi = row_ptr + rpo;
    for (int64_t r = 0; r < h->npad[i]; ++r) grp[h->row0[i] + r] = (int32_t)(ebase + (r < n[i] ? rpi[r] : rpi[n[i]]));
    ebase += rpi[n[i]];
    rpo += n[i] + 1;
  }
  // columns: the per-system local indices shifted to the system's first row
  int64_t e = 0;
  for (int i = 0; i < nsys; ++i)
    for (int64_t q = 0; q < h->nnz_sys[i]; ++q, ++e) {
      const int32_t c = col[e];
      if (c < 0 || c >= n[i]) return RB_EBADCSR;
      gci[e] = (int32_t)(c + h->row0[i]);
    }
  grp[NP] = (int32_t)nnz;
  h->NP = NP;
  h->NC = NC;
  h->nnz = nnz;
  int rc;
  if ((rc = balloc(&h->rp, NP + 1)) || (rc = balloc(&h->ci, nnz)) || (rc = balloc(&h->cv, nnz)) ||
      (rc = balloc(&h->trp, NP + 1)) || (rc = balloc(&h->tci, nnz)) || (rc = balloc(&h->tsrc, nnz)) ||
      (rc = balloc(&h->tcv, nnz)))
    return rc;
  RB_CUDA_TRY(cudaMemcpy(h->rp, grp.data(), sizeof(int32_t) * (NP + 1), cudaMemcpyHostToDevice));
  RB_CUDA_TRY(cudaMemcpy(h->ci, gci.data(), sizeof(int32_t) * nnz, cudaMemcpyHostToDevice));
  // no stencil slices: a stencil slice lets a row that lacks an offset gather
  // (with a zero weight) from the next system's rows, which would carry a
  // failed system's non-finite values into its neighbour
  if ((rc = sell_build(NP, nnz, h->rp, h->ci, &h->A, h->us, false))) return rc;
  if ((rc = csr_transpose(NP, nnz, h->rp, h->ci, h->trp, h->tci, h->tsrc, h->us))) return rc;
  if ((rc = sell_build(NP, nnz, h->trp, h->tci, &h->AT, h->us, false))) return rc;
  cudaFree(h->A32.val);
  h->A32 = SellBuf<float>();
  h->A32.nslices = h->A.nslices;
  h->A32.cap = h->A.cap;
  h->A32.slice_ptr = h->A.slice_ptr;
  h->A32.width = h->A.width;
  h->A32.col = h->A.col;
  h->A32.perm = h->A.perm;
  h->A32.offs = h->A.offs;
  h->A32.offs_stride = h->A.offs_stride;
  if ((rc = balloc(&h->A32.val, h->A.cap))) return rc;
  // layout, vectors, states
  if ((rc = balloc(&h->d_row0, nsys)) || (rc = balloc(&h->d_n, nsys)) || (rc = balloc(&h->d_cofs, nsys))) return rc;
  RB_CUDA_TRY(cudaMemcpy(h->d_row0, h->row0.data(), sizeof(int64_t) * nsys, cudaMemcpyHostToDevice));
  RB_CUDA_TRY(cudaMemcpy(h->d_n, h->n.data(), sizeof(int64_t) * nsys, cudaMemcpyHostToDevice));
  RB_CUDA_TRY(cudaMemcpy(h->d_cofs, h->cofs.data(), sizeof(int64_t) * nsys, cudaMemcpyHostToDevice));
  double** dv[] = {&h->b, &h->x, &h->r, &h->p, &h->s, &h->q, &h->t, &h->qraw, &h->traw, &h->rt0};
  for (double** v : dv)
    if ((rc = balloc(v, NP))) return rc;
  if ((rc = balloc(&h->stage, std::max<int64_t>(NC, NC * std::max(1, h->o.k_max))))) return rc;
  if (h->o.precision == RB_MIXED) {
    float** fv[] = {&h->fx, &h->fr, &h->fp, &h->fs, &h->fq, &h->ft, &h->fqraw, &h->ftraw, &h->frt0};
    for (float** v : fv)
      if ((rc = balloc(v, NP))) return rc;
  }
  if (h->o.k_max > 0) {
    double** bv[] = {&h->U, &h->C, &h->Ct, &h->Chat};
    for (double** v : bv)
      if ((rc = balloc(v, NP * h->o.k_max))) return rc;
    if (h->o.precision == RB_MIXED) {
      float** fb[] = {&h->fU, &h->fC, &h->fChat};
      for (float** v : fb)
        if ((rc = balloc(v, NP * h->o.k_max))) return rc;
    }
    if ((rc = balloc(&h->dR, (int64_t)nsys * kBK * kBK))) return rc;
  }
  if ((rc = balloc(&h->st, nsys)) || (rc = balloc(&h->dflags, nsys)) || (rc = balloc(&h->dskip, nsys)) ||
      (rc = balloc(&h->dcmd, nsys)) || (rc = balloc(&h->dres, nsys)) || (rc = balloc(&h->dsf, nsys)) ||
      (rc = balloc(&h->drm, nsys)))
    return rc;
  if (h->hst) cudaFreeHost(h->hst);
  if (h->hsf) cudaFreeHost(h->hsf);
  h->hst = nullptr;
  h->hsf = nullptr;
  if (cudaMallocHost(&h->hst, sizeof(IterState) * nsys) != cudaSuccess ||
      cudaMallocHost(&h->hsf, sizeof(rb::SysFlag) * nsys) != cudaSuccess)
    return RB_ENOMEM;
  h->kin = h->k = 0;
  h->have = true;
  h->ntiles = 0;
  h->tune_ms = 0.0;
  if ((rc = build_tiles(h, 8, 4))) return rc;
  return rbicgstab_batch_set_values(h, val, RB_HOST);
}

extern "C" int rbicgstab_batch_set_values(rb_batch h, const double* val, int where) {
  if (!h || !val || (where != RB_HOST && where != RB_DEVICE)) return RB_EINVAL;
  if (!h->have) return RB_EDIM;
  RB_CUDA_TRY(cudaMemcpyAsync(h->cv, val, sizeof(double) * h->nnz,
                              where == RB_HOST ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice, h->us));
  int rc;
  if ((rc = check_finite(h->cv, h->nnz, h->dflags, h->us) == cudaSuccess ? RB_OK : RB_ECUDA)) return rc;
  int bad = 0;
  RB_CUDA_TRY(cudaMemcpyAsync(&bad, h->dflags, sizeof(int), cudaMemcpyDeviceToHost, h->us));
  if ((rc = sync_b(h))) return rc;
  if (bad) return RB_ENONFINITE;
  if ((rc = sell_fill_values<double>(h->A, h->cv, h->us))) return rc;
  if ((rc = gather_values(h->nnz, h->tsrc, h->cv, h->tcv, h->us))) return rc;
  if ((rc = sell_fill_values<double>(h->AT, h->tcv, h->us))) return rc;
  if (h->o.precision == RB_MIXED && (rc = sell_fill_values<float>(h->A32, h->cv, h->us))) return rc;
  h->setup_owed = h->kin > 0;
  h->k = 0;
  drop_graphs(h);
  return sync_b(h);
}

extern "C" int rbicgstab_batch_set_recycle(rb_batch h, int32_t k, const double* U, int where) {
  if (!h || k < 0 || k > h->o.k_max || (k > 0 && !U) || (where != RB_HOST && where != RB_DEVICE)) return RB_EINVAL;
  if (!h->have) return RB_EDIM;
  h->kin = k;
  h->k = 0;
  h->setup_owed = k > 0;
  h->tune_ms = 0.0;
  drop_graphs(h);
  if (k == 0) return RB_OK;
  RB_CUDA_TRY(cudaMemcpyAsync(h->stage, U, sizeof(double) * h->NC * k,
                              where == RB_HOST ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice, h->us));
  count_launches(1);
  kb_relayout<true><<<h->grid, kBlock, 0, h->us>>>(h->U, h->stage, k, h->NP, layout_of(h), tiles_of(h));
  RB_CUDA_TRY(cudaGetLastError());
  return sync_b(h);
}

extern "C" int rbicgstab_batch_info(rb_batch h, int32_t* tile_slices, int32_t* ctas_per_sm, int32_t* ntiles,
                                    double* tune_ms) {
  if (!h) return RB_EINVAL;
  if (tile_slices) *tile_slices = h->tile_slices;
  if (ctas_per_sm) *ctas_per_sm = h->ctas_per_sm;
  if (ntiles) *ntiles = h->ntiles;
  if (tune_ms) *tune_ms = h->tune_ms;
  return RB_OK;
}

extern "C" int rbicgstab_batch_solve(rb_batch h, const double* b, double* x, int where, rb_stats* st_out) {
  if (!h || !b || !x || (where != RB_HOST && where != RB_DEVICE)) return RB_EINVAL;
  if (!h->have) return RB_EDIM;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  auto done = [&](int code) {
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    return code;
  };
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) return done(RB_ECUDA);
  cudaEventRecord(e0, h->us);
  int rc;
  if (h->setup_owed && (rc = batch_setup(h))) return done(rc);
  if (h->tune_ms == 0.0 && (rc = autotune(h))) return done(rc);
  const auto kind = where == RB_HOST ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice;
  // inputs into the padded layout
  RB_CUDA_TRY(cudaMemcpyAsync(h->stage, b, sizeof(double) * h->NC, kind, h->us));
  kb_relayout<true><<<h->grid, kBlock, 0, h->us>>>(h->b, h->stage, 1, h->NP, layout_of(h), tiles_of(h));
  RB_CUDA_TRY(cudaMemcpyAsync(h->stage, x, sizeof(double) * h->NC, kind, h->us));
  kb_relayout<true><<<h->grid, kBlock, 0, h->us>>>(h->x, h->stage, 1, h->NP, layout_of(h), tiles_of(h));
  count_launches(2);
  RB_CUDA_TRY(cudaGetLastError());
  for (double* v : {h->b, h->x}) {
    int f = 0;
    RB_CUDA_TRY(check_finite(v, h->NP, h->dflags, h->us));
    RB_CUDA_TRY(cudaMemcpyAsync(&f, h->dflags, sizeof(int), cudaMemcpyDeviceToHost, h->us));
    if ((rc = sync_b(h))) return done(rc);
    if (f) return done(RB_ENONFINITE);
  }
  const int S = h->S;
  std::vector<int> max_itn(S);
  for (int i = 0; i < S; ++i)
    max_itn[i] = h->o.max_itn > 0 ? h->o.max_itn : (int)std::min<int64_t>(h->n[i], 20000);
  std::vector<double> rn2, bn2;
  if ((rc = true_residuals(h, rn2, bn2))) return done(rc);
  const double tol2 = h->o.tol * h->o.tol;
  std::vector<int> iters(S, 0), status(S, RB_OK), outer(S, 0);
  std::vector<double> rec2(S, 0.0);
  if (h->o.precision == RB_FP64) {
    std::vector<double> th(S);
    for (int i = 0; i < S; ++i) th[i] = tol2 * bn2[i];
    if ((rc = batch_start(h, h->b, h->x, th, std::vector<char>(S, 0), max_itn, h->o.shadow_seed))) return done(rc);
    if ((rc = iterate_b<double>(h, *std::max_element(max_itn.begin(), max_itn.end())))) return done(rc);
    if ((rc = gemv_b(h, h->x, h->U, -1.0, true))) return done(rc);
    RB_CUDA_TRY(cudaMemcpyAsync(h->hst, h->st, sizeof(IterState) * S, cudaMemcpyDeviceToHost, h->us));
    if ((rc = sync_b(h))) return done(rc);
    for (int i = 0; i < S; ++i) {
      iters[i] = h->hst[i].iter;
      status[i] = h->hst[i].status;
      rec2[i] = h->hst[i].rnorm2;
      outer[i] = 1;
    }
  } else {
    // FP32 inner iteration with FP64 residual replacement per system, the
    // single-system mixed scheme (reliable updates): a system folds its FP32
    // increment into the FP64 x whenever its recursive residual has fallen
    // by kReplaceB below the larger of its last true residual and its peak
    // since then, or it reports convergence; the true residual then either
    // meets the target (a tenth of the tolerance) or, projected as in eq.
    // (3.5), replaces the FP32 residual while the search direction and the
    // scalars carry on.  A half-step exit above the target, and a fold that
    // would raise the true residual (the FP32 process diverged: an
    // ill-conditioned system at the FP32 accuracy floor; the fold is undone),
    // restart the system in the next round.  Two undone folds in a row, a
    // breakdown or a non-finite inner iterate (its increment dropped) hand
    // the system to FP64 rounds from its current x at the end.
    constexpr double kReplaceB = 1e-2;
    constexpr int kStallSwitchB = 2;   // folds undone in a row before the FP64 rounds
    constexpr int kRounds = 6;
    std::vector<double> target(S), rlast(S, 0.0), rmx(S, 0.0);
    for (int i = 0; i < S; ++i) target[i] = 0.1 * h->o.tol * std::sqrt(bn2[i]);
    std::vector<char> fin(S, 0), skip(S, 1), ended(S, 0), to64(S, 0);
    std::vector<int> cmd(S), res(S), last_status(S, RB_OK), stalls(S, 0);
    for (int round = 0; round < kRounds; ++round) {
      bool any = false;
      for (int i = 0; i < S; ++i) {
        skip[i] = 1;
        ended[i] = 0;
        if (fin[i] || to64[i]) continue;
        if (!std::isfinite(rn2[i])) {
          status[i] = RB_ENONFINITE;
          fin[i] = 1;
        } else if (std::sqrt(rn2[i]) <= target[i] || bn2[i] == 0.0) {
          status[i] = RB_OK;
          fin[i] = 1;
        } else if (iters[i] >= max_itn[i]) {
          status[i] = last_status[i] != RB_OK ? last_status[i] : RB_ENOTCONV;
          fin[i] = 1;
        } else {
          skip[i] = 0;
          any = true;
        }
      }
      if (!any) break;
      std::vector<double> th(S);
      std::vector<int> cap(S);
      for (int i = 0; i < S; ++i) {
        th[i] = target[i] * target[i];
        cap[i] = std::max(1, max_itn[i] - iters[i]);
        rlast[i] = std::sqrt(rn2[i]);
      }
      if ((rc = batch_start(h, h->b, h->x, th, skip, cap, h->o.shadow_seed))) return done(rc);
      RB_CUDA_TRY(to_float(h->r, h->fr, h->NP, h->us));
      RB_CUDA_TRY(to_float(h->r, h->fp, h->NP, h->us));
      RB_CUDA_TRY(to_float(h->rt0, h->frt0, h->NP, h->us));
      RB_CUDA_TRY(cudaMemsetAsync(h->fx, 0, sizeof(float) * h->NP, h->us));
      for (int i = 0; i < S; ++i)
        if (!skip[i]) outer[i] += 1;
      auto hook = [&]() -> int {
        bool anyc = false;
        for (int i = 0; i < S; ++i) {
          cmd[i] = kCmdNone;
          res[i] = 0;
          if (skip[i] || ended[i]) continue;
          const SysFlag& f = h->hsf[i];
          const double peak2 = std::max(f.rmax2, rlast[i] * rlast[i]);
          if (f.done) cmd[i] = f.status == RB_ENONFINITE ? kCmdDrop : kCmdFold;
          else if (f.rnorm2 <= kReplaceB * kReplaceB * peak2) cmd[i] = kCmdFold;
          anyc = anyc || cmd[i] != kCmdNone;
        }
        if (!anyc) return RB_OK;
        RB_CUDA_TRY(cudaMemcpyAsync(h->dcmd, cmd.data(), sizeof(int) * S, cudaMemcpyHostToDevice, h->us));
        count_launches(3);
        // the folded systems' previous x waits in s (idle in the FP32 rounds)
        kb_copy_rows<<<h->grid, kBlock, 0, h->us>>>(h->s, h->x, h->dcmd, tiles_of(h));
        kb_fold<<<h->grid, kBlock, 0, h->us>>>(h->x, h->fx, h->U, h->NP, h->k, h->st, h->dcmd, tiles_of(h));
        kb_state_cmd<<<(S + 255) / 256, 256, 0, h->us>>>(h->st, S, h->k, h->dcmd, nullptr, nullptr);
        RB_CUDA_TRY(cudaGetLastError());
        int rc2 = true_residuals(h, rn2, bn2);   // synchronises: cmd is free again after it
        if (rc2) return rc2;
        bool anyr = false, anyu = false;   // systems whose FP32 residual is replaced / whose fold is undone
        std::vector<int> rep(S, 0), undo(S, 0);
        for (int i = 0; i < S; ++i) {
          if (cmd[i] == kCmdNone) continue;
          const SysFlag& f = h->hsf[i];
          const double rn = std::sqrt(rn2[i]);
          const bool finite = std::isfinite(rn);
          if (!finite || rn > rlast[i]) {    // the fold made x worse: undo it, restart next round
            undo[i] = 1;
            anyu = true;
            rn2[i] = rlast[i] * rlast[i];
            if (!f.done) res[i] = 2;
            h->hsf[i].done = 1;
            ended[i] = 1;
            if (++stalls[i] >= kStallSwitchB) to64[i] = 1;
            continue;
          }
          stalls[i] = 0;
          if (rn <= target[i]) {             // converged: stop it
            if (!f.done) res[i] = 2;
            h->hsf[i].done = 1;
            ended[i] = 1;
            fin[i] = 1;
            status[i] = RB_OK;
          } else if (f.done && f.status != RB_OK && f.status != RB_ENOTCONV) {   // breakdown / overflow
            ended[i] = 1;
            to64[i] = 1;
            last_status[i] = f.status;
          } else if (f.done && f.status == RB_ENOTCONV) {
            ended[i] = 1;
            fin[i] = 1;
            status[i] = RB_ENOTCONV;
          } else if (!f.done || !f.half) {   // replace and carry on
            rep[i] = 1;
            anyr = true;
            res[i] = f.done ? 1 : 3;
            h->hsf[i].done = 0;
            rlast[i] = rn;
            rmx[i] = rn2[i];
            outer[i] += 1;
          } else {   // a half-step exit above the target: the next round restarts it
            ended[i] = 1;
          }
        }
        if (anyu) {
          RB_CUDA_TRY(cudaMemcpyAsync(h->dres, undo.data(), sizeof(int) * S, cudaMemcpyHostToDevice, h->us));
          count_launches(1);
          kb_copy_rows<<<h->grid, kBlock, 0, h->us>>>(h->x, h->s, h->dres, tiles_of(h));
          RB_CUDA_TRY(cudaGetLastError());
          RB_CUDA_TRY(cudaStreamSynchronize(h->us));   // dres is written again below
        }
        if (anyr) {
          RB_CUDA_TRY(cudaMemcpyAsync(h->dskip, rep.data(), sizeof(int) * S, cudaMemcpyHostToDevice, h->us));
          if (h->k > 0) {
            // gemv skip mask = not replaced (cmd is free after the sync above)
            for (int i = 0; i < S; ++i) cmd[i] = rep[i] ? 0 : 1;
            RB_CUDA_TRY(cudaMemcpyAsync(h->dcmd, cmd.data(), sizeof(int) * S, cudaMemcpyHostToDevice, h->us));
            SysDots d{};
            d.M = h->Chat; d.km = h->k; d.v = h->r;
            if ((rc2 = sysdots(h, d, false))) return rc2;
            if ((rc2 = gemv_b(h, h->x, h->U, 1.0, false, h->dcmd))) return rc2;
            if ((rc2 = gemv_b(h, h->r, h->C, -1.0, false, h->dcmd))) return rc2;
          }
          count_launches(1);
          kb_to_float<<<h->grid, kBlock, 0, h->us>>>(h->fr, h->r, h->dskip, tiles_of(h));
          RB_CUDA_TRY(cudaGetLastError());
        }
        bool anys = false;
        for (int i = 0; i < S; ++i) anys = anys || res[i] != 0;
        if (anys) {
          RB_CUDA_TRY(cudaMemcpyAsync(h->dres, res.data(), sizeof(int) * S, cudaMemcpyHostToDevice, h->us));
          RB_CUDA_TRY(cudaMemcpyAsync(h->drm, rmx.data(), sizeof(double) * S, cudaMemcpyHostToDevice, h->us));
          count_launches(1);
          kb_state_cmd<<<(S + 255) / 256, 256, 0, h->us>>>(h->st, S, h->k, nullptr, h->dres, h->drm);
          RB_CUDA_TRY(cudaGetLastError());
        }
        return sync_b(h);   // the host vectors above are read by the copies
      };
      if ((rc = iterate_b<float>(h, *std::max_element(cap.begin(), cap.end()), hook))) return done(rc);
      RB_CUDA_TRY(cudaMemcpyAsync(h->hst, h->st, sizeof(IterState) * S, cudaMemcpyDeviceToHost, h->us));
      if ((rc = sync_b(h))) return done(rc);
      for (int i = 0; i < S; ++i)
        if (!skip[i]) iters[i] += h->hst[i].iter;
    }
    for (int i = 0; i < S; ++i)   // FP32 rounds used up: those systems finish in FP64
      if (!fin[i] && !to64[i] && iters[i] < max_itn[i]) to64[i] = 1;
    // FP64 rounds for the systems the FP32 iteration could not finish: Alg. 2
    // in FP64 from the current x to the mixed target on the recursive
    // residual; a true residual still above the tolerance after a round (the
    // recursive residual drifts from the true one over a long run) takes
    // another round, at most three.
    for (int round64 = 0; round64 < 3; ++round64) {
      bool any64 = false;
      std::vector<char> skip64(S, 1);
      for (int i = 0; i < S; ++i)
        if (to64[i] && !fin[i]) {
          skip64[i] = 0;
          any64 = true;
        }
      if (!any64) break;
      if ((rc = true_residuals(h, rn2, bn2))) return done(rc);
      std::vector<double> th(S);
      std::vector<int> cap(S);
      for (int i = 0; i < S; ++i) {
        th[i] = target[i] * target[i];
        cap[i] = std::max(1, max_itn[i] - iters[i]);
      }
      if ((rc = batch_start(h, h->b, h->x, th, skip64, cap, h->o.shadow_seed))) return done(rc);
      if ((rc = iterate_b<double>(h, *std::max_element(cap.begin(), cap.end())))) return done(rc);
      if ((rc = gemv_b(h, h->x, h->U, -1.0, true))) return done(rc);
      RB_CUDA_TRY(cudaMemcpyAsync(h->hst, h->st, sizeof(IterState) * S, cudaMemcpyDeviceToHost, h->us));
      if ((rc = sync_b(h))) return done(rc);
      if ((rc = true_residuals(h, rn2, bn2))) return done(rc);
      for (int i = 0; i < S; ++i) {
        if (skip64[i]) continue;
        iters[i] += h->hst[i].iter;
        outer[i] += 1;
        status[i] = h->hst[i].status;
        const bool more = status[i] == RB_OK && std::sqrt(rn2[i]) > h->o.tol * std::sqrt(bn2[i]) &&
                          iters[i] < max_itn[i] && round64 < 2;
        if (!more) fin[i] = 1;
        if (status[i] == RB_OK && std::sqrt(rn2[i]) > h->o.tol * std::sqrt(bn2[i]) && !more) status[i] = RB_ENOTCONV;
      }
    }
    for (int i = 0; i < S; ++i) {
      rec2[i] = rn2[i];
      if (!fin[i] && status[i] == RB_OK) status[i] = last_status[i] != RB_OK ? last_status[i] : RB_ENOTCONV;
    }
  }
  std::vector<double> tr2;
  if ((rc = true_residuals(h, tr2, bn2))) return done(rc);
  kb_relayout<false><<<h->grid, kBlock, 0, h->us>>>(h->x, h->stage, 1, h->NP, layout_of(h), tiles_of(h));
  count_launches(1);
  RB_CUDA_TRY(cudaGetLastError());
  RB_CUDA_TRY(cudaMemcpyAsync(x, h->stage, sizeof(double) * h->NC,
                              where == RB_HOST ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice, h->us));
  cudaEventRecord(e1, h->us);
  if ((rc = sync_b(h))) return done(rc);
  float ms = 0.f;
  cudaEventElapsedTime(&ms, e0, e1);
  int first_fail = RB_OK;
  for (int i = 0; i < S; ++i) {
    if (status[i] != RB_OK && first_fail == RB_OK) first_fail = status[i];
    if (!st_out) continue;
    rb_stats& o = st_out[i];
    o = rb_stats{};
    o.iters = iters[i];
    o.status = status[i];
    o.k_used = h->k > 0 ? h->k_used[i] : 0;
    o.seeds_used = 1;
    o.matvecs = 2 * (int64_t)iters[i] + outer[i];
    o.matvecs_setup = h->k > 0 ? 2 * h->k : 0;
    o.outer = outer[i];
    o.relres_rec = bn2[i] > 0 ? std::sqrt(rec2[i] / bn2[i]) : 0.0;
    o.relres_true = bn2[i] > 0 ? std::sqrt(tr2[i] / bn2[i]) : 0.0;
    o.ms_total = ms;
  }
  return done(first_fail);
}
