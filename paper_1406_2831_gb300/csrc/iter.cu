// The fused passes of one RBiCGSTAB iteration (Alg. 2).
//
// One iteration is five kernels, each one streaming pass over HBM that ends in
// a deterministic grid reduction whose last block computes the scalars:
//
//   P1  q_raw = A p_i (SELL-32 SpMV);  zeta = C-hat^T q_raw,  (r~_0, q_raw)
//       -> (r~_0, q) = (r~_0, q_raw) - (C^T r~_0)^T zeta,  alpha = rho / (r~_0, q)
//   P2  q = q_raw - C zeta;  s = r - alpha q;  ||s||^2  (half-step test)
//   P3  t_raw = A s;  gamma = C-hat^T t_raw
//   P4  t = t_raw - C gamma;  (s,t), (t,t), (r~_0,t), (r~_0,s)
//       -> omega = (s,t)/(t,t),  rho_i = (r~_0,s) - omega (r~_0,t) = (r~_0, r_i),
//          beta = (rho_i/rho_{i-1}) (alpha/omega),  x_c += alpha zeta + omega gamma
//   P5  x += alpha p + omega s;  r = s - omega t;  ||r||^2;  p_{i+1} = r + beta (p - omega q)
//
// With k = 0 (plain BiCGSTAB) q = q_raw and t = t_raw, P3 also forms the four
// dots and P4 is not launched.  (r~_0, q) and rho_i use the algebraically
// equal forms above instead of fresh dots with q and r_i; they differ from
// the literal ones only by rounding.
//
// Blocked solves: every pass handles R right-hand sides of the same matrix
// and recycle space at once (R = 1, 2 or 4; per-RHS vectors and device
// state, one grid reduction), so A, C, C-hat and r~_0 are read once per pass
// for all R.  A right-hand side whose solve has ended is masked out.
//
// T is the storage and SpMV type (double for RB_FP64, float for the inner
// solve of RB_MIXED).  Dot products of the scalar recurrences accumulate in
// FP64 (FP64 data) or Dot2-compensated FP32 (FP32 data).  The projection
// coefficients zeta, gamma of FP32 data are summed in FP32 within each
// 32-row slice and compensated across slices: accuracy at the level of the
// FP32 vectors they project.
#include <algorithm>
#include <cstdlib>
#include <type_traits>

#include "device.cuh"
#include "kernels.h"
#include "mbar.cuh"
#include "scalars.cuh"

namespace rb {

// Scratch doubles per warp in a RedT buffer ([warp][kRedCH][33]).
constexpr int kScr = kRedCH * 33;

// Run a scalar step in the last block: warp r handles right-hand side r.
#define RB_FINISH_WARPS(R, ACT, CALL)                       \
  do {                                                      \
    const int r_ = threadIdx.x >> 5;                        \
    _Pragma("unroll") for (int rr_ = 0; rr_ < (R); ++rr_)   \
      if (rr_ == r_ && (ACT)[rr_]) { const int r = rr_; CALL; } \
  } while (0)


// ---------------------------------------------------------------- helpers
template <typename T, int KMAX, int R>
struct ColProj {   // projections column-per-lane (FP32 data, or several RHS)
  static constexpr bool value = KMAX > 0 && (std::is_same<T, float>::value || R > 1);
};

// Warp sum of one per-thread accumulator; lane 0 stores it to sm.w[warp][slot].
template <int NV>
__device__ __forceinline__ void warp_slot(const Acc<float>& a, int slot, ReduceCore<NV>& sm) {
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
  if ((threadIdx.x & 31) == 0) sm.w[threadIdx.x >> 5][slot] = (double)hi + (double)lo;
}

template <int NV>
__device__ __forceinline__ void warp_slot(const Acc<double>& a, int slot, ReduceCore<NV>& sm) {
  double x = a.v;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) x += __shfl_down_sync(0xffffffffu, x, o);
  if ((threadIdx.x & 31) == 0) sm.w[threadIdx.x >> 5][slot] = x;
}

template <int NV>
__device__ __forceinline__ void zero_slot(int slot, ReduceCore<NV>& sm) {
  if ((threadIdx.x & 31) == 0) sm.w[threadIdx.x >> 5][slot] = 0.0;
}

// 16-byte vector of T.
template <typename T>
struct Vec;
template <>
struct Vec<float> {
  using type = float4;
  static constexpr int W = 4;
};
template <>
struct Vec<double> {
  using type = double2;
  static constexpr int W = 2;
};

// Dot products of one 32-row column (shared memory) with the R slice
// vectors ys[r] (shared memory, read as broadcasts), each summed in T in row
// order: part[r] = sum_i col[i] * ys[r][i].
template <int R>
__device__ __forceinline__ void col_dot(const float* col, const float (*ys)[32], const bool (&act)[R],
                                        float (&part)[R]) {
#pragma unroll
  for (int u = 0; u < 8; ++u) {
    const float4 c = *reinterpret_cast<const float4*>(col + 4 * u);
#pragma unroll
    for (int r = 0; r < R; ++r) {
      if (!act[r]) continue;
      const float4 y = *reinterpret_cast<const float4*>(ys[r] + 4 * u);
      part[r] = __fmaf_rn(c.x, y.x, part[r]);
      part[r] = __fmaf_rn(c.y, y.y, part[r]);
      part[r] = __fmaf_rn(c.z, y.z, part[r]);
      part[r] = __fmaf_rn(c.w, y.w, part[r]);
    }
  }
}
template <int R>
__device__ __forceinline__ void col_dot(const double* col, const double (*ys)[32], const bool (&act)[R],
                                        double (&part)[R]) {
#pragma unroll
  for (int u = 0; u < 16; ++u) {
    const double2 c = *reinterpret_cast<const double2*>(col + 2 * u);
#pragma unroll
    for (int r = 0; r < R; ++r) {
      if (!act[r]) continue;
      const double2 y = *reinterpret_cast<const double2*>(ys[r] + 2 * u);
      part[r] = __fma_rn(c.x, y.x, part[r]);
      part[r] = __fma_rn(c.y, y.y, part[r]);
    }
  }
}

// Dot products of one 32-row column (shared memory) with the slice products
// of R right-hand sides stored row-major (yi[i][r], read as broadcasts), for
// pairs of right-hand sides: part[h] = sum_i col[i] * (yi[i][2h], yi[i][2h+1]),
// each lane summed in T in row order (the order of col_dot).
template <typename T, int R>
__device__ __forceinline__ void col_dot_pairs(const T* col, const T (*yi)[R], typename Pair<T>::V (&part)[R / 2]) {
  using P = Pair<T>;
  using V = typename P::V;
  using C16 = typename Vec<T>::type;
  constexpr int VC = Vec<T>::W;
#pragma unroll
  for (int u = 0; u < 32 / VC; ++u) {
    const C16 cv = *reinterpret_cast<const C16*>(col + VC * u);
    const T* c = reinterpret_cast<const T*>(&cv);
#pragma unroll
    for (int e = 0; e < VC; ++e) {
      const V* yp = reinterpret_cast<const V*>(yi[VC * u + e]);
      const V cc = P::mk(c[e], c[e]);
#pragma unroll
      for (int h = 0; h < R / 2; ++h) part[h] = P::fma(cc, yp[h], part[h]);
    }
  }
}

// ---------------------------------------------------------------- cp.async
// Asynchronous 16-byte global -> shared copies (L2 only), grouped per thread.
__device__ __forceinline__ void cp_async16(void* smem, const void* gmem) {
  const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(s), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() {
  asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory");
}
// Bring bytes [p, p + bytes) into L2 (no register or shared-memory cost);
// p 16-byte aligned, bytes a multiple of 16.
__device__ __forceinline__ void prefetch_l2(const void* p, unsigned bytes) {
  asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;\n" ::"l"(p), "r"(bytes) : "memory");
}

// ---------------------------------------------------------------- SpMV core
// Rows sl*32+lane of two slices at once (sl1 < 0: only the first), so each
// warp keeps two independent gather chains in flight (single RHS, FP64).
template <typename T>
__device__ __forceinline__ void sell_rows2(const Sell<T>& A, int64_t sl0, int64_t sl1, int lane,
                                           const T* __restrict__ v, T& y0, T& y1) {
  const int32_t* __restrict__ col = A.col;
  const T* __restrict__ val = A.val;
  const int w0 = __ldg(A.width + sl0);
  const int w1 = sl1 >= 0 ? __ldg(A.width + sl1) : 0;
  const int64_t b0 = __ldg(A.slice_ptr + sl0) + lane;
  const int64_t b1 = sl1 >= 0 ? __ldg(A.slice_ptr + sl1) + lane : 0;
  const int wm = w0 < w1 ? w0 : w1;
  T a0 = T(0), a1 = T(0);
#pragma unroll 4
  for (int j = 0; j < wm; ++j) {
    const int64_t e0 = b0 + (int64_t)j * kSlice, e1 = b1 + (int64_t)j * kSlice;
    const int c0 = __ldg(col + e0), c1 = __ldg(col + e1);
    const T v0 = __ldg(val + e0), v1 = __ldg(val + e1);
    a0 = fma_t(v0, __ldg(v + c0), a0);
    a1 = fma_t(v1, __ldg(v + c1), a1);
  }
  for (int j = wm; j < w0; ++j) {
    const int64_t e0 = b0 + (int64_t)j * kSlice;
    a0 = fma_t(__ldg(val + e0), __ldg(v + __ldg(col + e0)), a0);
  }
  for (int j = wm; j < w1; ++j) {
    const int64_t e1 = b1 + (int64_t)j * kSlice;
    a1 = fma_t(__ldg(val + e1), __ldg(v + __ldg(col + e1)), a1);
  }
  y0 = a0;
  y1 = a1;
}

// ---------------------------------------------------------------- P1 / P3
// Single RHS, FP64, row-per-lane projection: y = A v stored to `out`;
// acc[OFF + j] += Chat_j^T y (j < k); RTQ adds acc[0] += (r~0, y).
// STAGE: the C-hat rows of the warp's two slices are copied into the warp's
// shared tiles (tile[h][j][lane], h = slice, j = column) with cp.async before
// the gathers start, so those bytes are in flight during the SpMV and cost no
// registers; otherwise they are loaded from global after the products.
template <typename T, int KMAX, bool RTQ, bool STAGE>
__device__ __forceinline__ void spmv_project(const IterArgs<T>& a, const T* __restrict__ v,
                                             T* __restrict__ out, Acc<T>* acc, int k, T* tile) {
  constexpr int KT = KMAX > 0 ? KMAX : 1;
  constexpr int VC = 16 / (int)sizeof(T);   // values per 16-byte chunk
  constexpr int VPR = kSlice / VC;          // chunks per 32-row column
  const int lane = threadIdx.x & 31;
  const int64_t w0 = gtid() >> 5, nw = gstride() >> 5;
  constexpr int OFF = RTQ ? 1 : 0;
  const T* __restrict__ Chat = a.Chat;
  const T* __restrict__ rt0 = a.rt0;
  const int64_t ld = a.ld, ns = a.A.nslices;
  for (int64_t sl = w0; sl < ns; sl += 2 * nw) {
    const int64_t sl1 = (sl + nw < ns) ? sl + nw : -1;
    if constexpr (STAGE) {
      __syncwarp();   // every lane is done with the previous tiles
      for (int q = lane; q < k * VPR; q += 32) {
        const int j = q / VPR, c = q % VPR;
        cp_async16(tile + j * kSlice + c * VC, Chat + (int64_t)j * ld + sl * kSlice + c * VC);
        if (sl1 >= 0) cp_async16(tile + (KT + j) * kSlice + c * VC, Chat + (int64_t)j * ld + sl1 * kSlice + c * VC);
      }
      cp_async_commit();
    }
    T y[2];
    sell_rows2<T>(a.A, sl, sl1, lane, v, y[0], y[1]);
    if constexpr (STAGE) {
      cp_async_wait<0>();
      __syncwarp();
    }
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      if (h == 1 && sl1 < 0) break;
      const int64_t row = (h == 0 ? sl : sl1) * kSlice + lane;
      out[row] = y[h];
      const T yd = y[h];
      if (RTQ) acc[0].add(__ldg(rt0 + row), yd);
#pragma unroll
      for (int j = 0; j < KMAX; ++j)
        if (j < k) acc[OFF + j].add(STAGE ? tile[(h * KT + j) * kSlice + lane] : __ldg(Chat + j * ld + row), yd);
    }
  }
}

// Per-warp shared memory of the multi-RHS / FP32 SpMV + projection passes:
// the C-hat tile of the current slice, transposed (column j's 32 rows
// contiguous, row stride 32 elements plus 16 bytes, which keeps the 16-byte
// column reads of the projection free of bank conflicts), and the slice
// products y_r.  After the main loop the storage serves the last block's
// reduction.
template <typename T, int KMAX, int R>
struct PipeSmem {
  static constexpr int KT = KMAX > 0 ? KMAX : 1;
  static constexpr int PAD = 32 + 16 / (int)sizeof(T);
  static constexpr int NE = 8;   // matrix entries per row loaded up front
  struct Warp {
    T tile[KT][PAD];
    union {
      T y[R][32];    // slice products, one row per right-hand side (odd R)
      T yi[32][R];   // slice products, right-hand sides interleaved (even R)
    };
  };
  union {
    Warp w[kBlock / 32];
    RedT t;
  };
};

// Issue the copies of slice sl's C-hat tile (rows sl*32 .. sl*32+31 of the k
// columns) into the warp's shared tile.
template <typename T, int KMAX, int R>
__device__ __forceinline__ void stage_tile(const IterArgs<T>& a, typename PipeSmem<T, KMAX, R>::Warp& ws,
                                           int64_t sl, int k) {
  constexpr int VC = 16 / (int)sizeof(T);   // values per 16-byte chunk
  constexpr int VPR = 32 / VC;              // chunks per 32-row column
  const int lane = threadIdx.x & 31;
  const int64_t base = sl * kSlice;
  for (int q = lane; q < k * VPR; q += 32) {
    const int j = q / VPR, c = q % VPR;
    cp_async16(&ws.tile[j][c * VC], a.Chat + (int64_t)j * a.ld + base + c * VC);
  }
}

// R right-hand sides (or FP32 data), one slice per warp and step: y_r = A v_r
// stored to out_r.  Per RHS r the block values live at sm.w[.][r*nvr + ...]:
// RTQ -> slot 0 = (r~0, y_r), projections -> slots OFF + j = Chat_j^T y_r,
// DOTS (k = 0) -> slots 0..3 = (s,t), (t,t), (r~0,t), (r~0,s) with s = v_r.
// Per slice the warp issues the asynchronous copy of the C-hat tile first (it
// lands while the products are formed), loads the first NE entries of every
// row straight into registers (all in flight together) and gathers v_r; the
// next slice's width and start are loaded one step ahead.  Lane j owns
// column j of the projection (no cross-lane reduction); each slice's 32
// products are summed in T and the total is carried across slices in the
// accumulator (Dot2 for FP32).
template <typename T, int KMAX, int R, bool RTQ, bool DOTS, int NVT>
__device__ __forceinline__ void spmv_multi(const IterArgs<T>& a, const T* const* v, T* const* out,
                                           const bool (&act)[R], int k, int nvr, ReduceCore<NVT>& sm,
                                           PipeSmem<T, KMAX, R>& ps) {
  using PS = PipeSmem<T, KMAX, R>;
  using P = Pair<T>;
  using V = typename P::V;
  constexpr bool PAIRS = R % 2 == 0;   // pairs of right-hand sides on packed instructions
  constexpr int H = PAIRS ? R / 2 : 1;
  constexpr int NE = PS::NE;
  constexpr int CPL = KMAX > 0 ? (KMAX + 31) / 32 : 1;
  constexpr int OFF = RTQ ? 1 : 0;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int64_t w0 = gtid() >> 5, nw = gstride() >> 5;
  const int64_t ns = a.A.nslices;
  const int32_t* __restrict__ colp = a.A.col;
  const T* __restrict__ valp = a.A.val;
  typename PS::Warp& ws = ps.w[warp];
  // Every right-hand side is gathered and reduced unconditionally (no
  // per-slot branches between the loads); an inactive one reads an active
  // one's vector and only its stores and its block values are masked.
  const T* vg[R];
  {
    int ra = 0;
#pragma unroll
    for (int r = R - 1; r >= 0; --r)
      if (act[r]) ra = r;
#pragma unroll
    for (int r = 0; r < R; ++r) vg[r] = act[r] ? v[r] : v[ra];
  }
  Acc<T> accr1[R], accd1[R][4], accp1[R][CPL];   // R = 1
  AccP<T> accr[H], accd[H][4], accp[H][CPL];      // pairs
  // width, first entry and column offset `lane` of the warp's next slice.
  // Stencil slices take the offset path for FP32 data and for one FP64
  // right-hand side; FP64 blocks measured slower with it (more register
  // spills: 7-point 128^3, four RHS, 29.2 -> 26.8 solves/s), while one FP64
  // RHS has no spills either way and needs it on wide stencils (27-point:
  // plain FP64 sequence 2.95 s with it, 3.82 s without).
  constexpr bool kOffsets = sizeof(T) == 4 || R == 1;
  const int ostride = a.A.offs_stride;
  int wn = 0;
  int64_t en = 0;
  int32_t on = kNoStencil;
  if (w0 < ns) {
    wn = __ldg(a.A.width + w0);
    en = __ldg(a.A.slice_ptr + w0);
    if (kOffsets) on = lane < ostride ? __ldg(a.A.offs + w0 * ostride + lane) : 0;
  }
  for (int64_t sl = w0; sl < ns; sl += nw) {
    const int wc = wn;
    const int64_t b = en + lane;
    const int32_t oc = on;
    if (sl + nw < ns) {
      wn = __ldg(a.A.width + sl + nw);
      en = __ldg(a.A.slice_ptr + sl + nw);
      if (kOffsets) on = lane < ostride ? __ldg(a.A.offs + (sl + nw) * ostride + lane) : 0;
    }
    // stencil slice: entry j's column is row + offset j (no column loads)
    const bool stencil = kOffsets && __shfl_sync(0xffffffffu, oc, 0) != kNoStencil;
    if (KMAX > 0) {
      __syncwarp();   // every lane is done with the previous slice's tile
      stage_tile<T, KMAX, R>(a, ws, sl, k);
      cp_async_commit();
    }
    const int64_t row = sl * kSlice + lane;
    const T rv = (RTQ || DOTS) ? __ldg(a.rt0 + row) : T(0);
    int cu[NE];
    T au[NE];
#pragma unroll
    for (int u = 0; u < NE; ++u) {
      const int32_t ou = __shfl_sync(0xffffffffu, oc, u);
      cu[u] = u < wc ? (stencil ? (int32_t)row + ou : __ldg(colp + b + (int64_t)u * kSlice)) : 0;
      au[u] = u < wc ? __ldg(valp + b + (int64_t)u * kSlice) : T(0);
    }
    T y[R];
#pragma unroll
    for (int r = 0; r < R; ++r) y[r] = T(0);
#pragma unroll
    for (int u = 0; u < NE; ++u) {
      if (u < wc) {
#pragma unroll
        for (int r = 0; r < R; ++r) y[r] = fma_t(au[u], __ldg(vg[r] + cu[u]), y[r]);
      }
    }
    for (int j = NE; j < wc; ++j) {   // rows wider than NE entries
      const int64_t e = b + (int64_t)j * kSlice;
      const int32_t oj = __shfl_sync(0xffffffffu, oc, j & 31);
      const int cc = stencil ? (int32_t)row + oj : __ldg(colp + e);
      const T vv = __ldg(valp + e);
#pragma unroll
      for (int r = 0; r < R; ++r) y[r] = fma_t(vv, __ldg(vg[r] + cc), y[r]);
    }
#pragma unroll
    for (int r = 0; r < R; ++r)
      if (act[r]) out[r][row] = y[r];
    if constexpr (PAIRS) {
      const V rv2 = P::mk(rv, rv);
#pragma unroll
      for (int h = 0; h < H; ++h) {
        const V yy = P::mk(y[2 * h], y[2 * h + 1]);
        if (RTQ) accr[h].add(rv2, yy);
        if (DOTS) {
          const V sv = P::mk(__ldg(vg[2 * h] + row), __ldg(vg[2 * h + 1] + row));
          accd[h][0].add(sv, yy);
          accd[h][1].add(yy, yy);
          accd[h][2].add(rv2, yy);
          accd[h][3].add(rv2, sv);
        }
      }
    } else {
#pragma unroll
      for (int r = 0; r < R; ++r) {
        if (RTQ) accr1[r].add(rv, y[r]);
        if (DOTS) {
          const T sv = __ldg(vg[r] + row);
          accd1[r][0].add(sv, y[r]);
          accd1[r][1].add(y[r], y[r]);
          accd1[r][2].add(rv, y[r]);
          accd1[r][3].add(rv, sv);
        }
      }
    }
    if (KMAX > 0) {
#pragma unroll
      for (int r = 0; r < R; ++r) {
        if (PAIRS) ws.yi[lane][r] = y[r];
        else ws.y[r][lane] = y[r];
      }
      cp_async_wait<0>();   // this thread's tile copies landed
      __syncwarp();         // ... and every lane's, and y is visible
#pragma unroll
      for (int cc = 0; cc < CPL; ++cc) {
        const int j = lane + 32 * cc;
        if (j < k) {
          if constexpr (PAIRS) {
            V part[H];
#pragma unroll
            for (int h = 0; h < H; ++h) part[h] = P::mk(T(0), T(0));
            col_dot_pairs<T, R>(ws.tile[j], ws.yi, part);
#pragma unroll
            for (int h = 0; h < H; ++h) accp[h][cc].add1(part[h]);
          } else {
            T part[R];
#pragma unroll
            for (int r = 0; r < R; ++r) part[r] = T(0);
            col_dot<R>(ws.tile[j], ws.y, act, part);
#pragma unroll
            for (int r = 0; r < R; ++r) accp1[r][cc].add1(part[r]);
          }
        }
      }
    }
  }
  // warp sums into sm.w (inactive right-hand sides contribute zeros)
#pragma unroll
  for (int r = 0; r < R; ++r) {
    if (RTQ) {
      if (act[r]) warp_slot(PAIRS ? accr[r / 2].lane(r & 1) : accr1[r], r * nvr, sm);
      else zero_slot(r * nvr, sm);
    }
    if (DOTS) {
#pragma unroll
      for (int d = 0; d < 4; ++d) {
        if (act[r]) warp_slot(PAIRS ? accd[r / 2][d].lane(r & 1) : accd1[r][d], r * nvr + d, sm);
        else zero_slot(r * nvr + d, sm);
      }
    }
    if (KMAX > 0) {
#pragma unroll
      for (int cc = 0; cc < CPL; ++cc) {
        const int j = lane + 32 * cc;
        if (j < k) sm.w[warp][r * nvr + OFF + j] = act[r] ? (PAIRS ? accp[r / 2][cc].lane(r & 1) : accp1[r][cc]).get() : 0.0;
      }
    }
  }
  __syncthreads();   // the tile storage is reused by the reduction
}

// Dynamic shared memory of the FP64 single-RHS P1 / P3: per warp the C-hat
// tiles of its two current slices (k <= 24: two blocks per SM still fit),
// reused after the main loop by the block reduction.
template <typename T, int KMAX>
struct TileSmem1 {
  static constexpr bool staged = KMAX > 0 && KMAX <= 24;
  static constexpr int KT = staged ? KMAX : 1;
  union {
    T tile[kBlock / 32][2 * KT * kSlice];
    ReduceSmem<KMAX + 1> red;   // P1's reduction (k + 1 values) is the larger one
  };
};

// Dynamic shared memory of P1 / P3 (the tile storage of the multi-RHS path, or
// TileSmem1), and the resident blocks per SM the kernels are compiled for.
template <typename T, int KMAX, int R>
struct P13Smem {
  static constexpr bool multi = ColProj<T, KMAX, R>::value || R > 1 || KMAX == 0;
  static constexpr size_t bytes = multi ? sizeof(PipeSmem<T, KMAX, R>) : sizeof(TileSmem1<T, KMAX>);
  static constexpr int min_blocks = !multi ? 2 : ((sizeof(T) == 8 || KMAX == 0) && R > 1 ? 3 : 4);
};

template <typename T, int KMAX, int R>
__global__ void __launch_bounds__(kBlock, P13Smem<T, KMAX, R>::min_blocks) k_p1(IterArgs<T> a) {
  IterState* st = a.st;
  bool act[R];
  bool any = false;
#pragma unroll
  for (int r = 0; r < R; ++r) {
    act[r] = (r < a.nrhs) && !st[r].done;
    any |= act[r];
  }
  if (!any) return;
  constexpr int NVR = KMAX + 1;
  const int k = KMAX > 0 ? st[0].k : 0;
  const int nvr = 1 + k;
  bool last;
  double *res, *scr;   // grid totals; scratch of the scalar step (free after the reduction)
  if constexpr (!P13Smem<T, KMAX, R>::multi) {
    using TS = TileSmem1<T, KMAX>;
    extern __shared__ __align__(16) unsigned char dsm[];
    auto& ts = *reinterpret_cast<TS*>(dsm);
    Acc<T> acc[NVR];
    spmv_project<T, KMAX, true, TS::staged>(a, a.p_in[0], a.qraw[0], acc, k, ts.tile[threadIdx.x >> 5]);
    __syncthreads();   // the tiles are reused by the reduction
    auto& sm = *reinterpret_cast<ReduceSmem<NVR>*>(dsm);
    last = block_reduce_last<T, NVR>(acc, nvr, sm, a.partials, &st[0].ticket[P1]);
    res = sm.res;
    scr = &sm.t[0][0][0];
  } else {
    __shared__ ReduceCore<R * NVR> sm;
    extern __shared__ __align__(16) unsigned char dsm[];
    auto& ps = *reinterpret_cast<PipeSmem<T, KMAX, R>*>(dsm);
    spmv_multi<T, KMAX, R, true, false, R * NVR>(a, a.p_in, a.qraw, act, k, nvr, sm, ps);
    last = grid_finish<R * NVR>(R * nvr, sm, a.partials, &st[0].ticket[P1]);
    res = sm.res;
    scr = &ps.t[0][0][0];
  }
  if (last) RB_FINISH_WARPS(R, act, finish_p1(&st[r], res + r * nvr, k, scr + r * kScr));
}

template <typename T, int KMAX, int R>
__global__ void __launch_bounds__(kBlock, P13Smem<T, KMAX, R>::min_blocks) k_p3(IterArgs<T> a) {
  IterState* st = a.st;
  bool act[R];
  bool any = false;
#pragma unroll
  for (int r = 0; r < R; ++r) {
    act[r] = (r < a.nrhs) && !st[r].done && !st[r].half;
    any |= act[r];
  }
  if (!any) return;
  constexpr bool DOTS = (KMAX == 0);
  constexpr int NVR = DOTS ? 4 : KMAX;
  const int k = KMAX > 0 ? st[0].k : 0;
  const int nvr = DOTS ? 4 : k;
  bool last;
  double* res;
  if constexpr (!P13Smem<T, KMAX, R>::multi) {
    using TS = TileSmem1<T, KMAX>;
    extern __shared__ __align__(16) unsigned char dsm[];
    auto& ts = *reinterpret_cast<TS*>(dsm);
    Acc<T> acc[NVR];
    spmv_project<T, KMAX, false, TS::staged>(a, a.s[0], a.traw[0], acc, k, ts.tile[threadIdx.x >> 5]);
    __syncthreads();   // the tiles are reused by the reduction
    auto& sm = *reinterpret_cast<ReduceSmem<NVR>*>(dsm);
    last = block_reduce_last<T, NVR>(acc, nvr, sm, a.partials, &st[0].ticket[P3]);
    res = sm.res;
  } else {
    __shared__ ReduceCore<R * NVR> sm;
    extern __shared__ __align__(16) unsigned char dsm[];
    auto& ps = *reinterpret_cast<PipeSmem<T, KMAX, R>*>(dsm);
    spmv_multi<T, KMAX, R, false, DOTS, R * NVR>(a, a.s, a.traw, act, k, nvr, sm, ps);
    last = grid_finish<R * NVR>(R * nvr, sm, a.partials, &st[0].ticket[P3]);
    res = sm.res;
  }
  if (last) RB_FINISH_WARPS(R, act, (DOTS ? finish_p4(&st[r], res + r * nvr, 0) : finish_p3(&st[r], res + r * nvr, k)));
}

// L2 prefetch, by one warp, of rows [row0, row0 + nrows) of the first ncols
// columns of the column-major block M (leading dimension ld) and of the
// vectors vs[0..nvs): one bulk prefetch per lane and segment.
template <typename T>
__device__ __forceinline__ void prefetch_rows(const T* M, int64_t ld, int ncols, const T* const* vs, int nvs,
                                              int64_t row0, int nrows) {
  const int lane = threadIdx.x & 31;
  const unsigned bytes = (unsigned)nrows * sizeof(T);
  for (int q = lane; q < ncols + nvs; q += 32) {
    const T* p = q < ncols ? M + (int64_t)q * ld + row0 : vs[q - ncols] + row0;
    prefetch_l2(p, bytes);
  }
}

// ---------------------------------------------------------------- streaming passes
// P2, P4 and P5 stream n-vectors and the n x k block C.  With one RHS each
// thread takes VW consecutive rows per step (one 16-byte vector of each
// stream), the C columns of a step are loaded up front (predicated, no
// branches) so that they are all in flight together, and the warp's rows two
// steps ahead are prefetched into L2.  A block of several RHS already has
// R times the streams in flight per row: one row per thread.
template <typename T, int W>
struct Pack;
template <typename T>
struct Pack<T, 1> {
  using type = T;
};
template <>
struct Pack<float, 4> {
  using type = float4;
};
template <>
struct Pack<double, 2> {
  using type = double2;
};

template <typename T, int R>
struct StreamVW {
  static constexpr int value = R == 1 ? Vec<T>::W : 1;
};

template <typename T, int W>
__device__ __forceinline__ typename Pack<T, W>::type ldv(const T* p) {
  return __ldg(reinterpret_cast<const typename Pack<T, W>::type*>(p));
}
template <typename T, int W>
__device__ __forceinline__ typename Pack<T, W>::type ldv_coherent(const T* p) {
  return *reinterpret_cast<const typename Pack<T, W>::type*>(p);
}
template <typename T, int W>
__device__ __forceinline__ void stv(T* p, const T (&v)[W]) {
  typename Pack<T, W>::type x;
  T* xs = reinterpret_cast<T*>(&x);
#pragma unroll
  for (int e = 0; e < W; ++e) xs[e] = v[e];
  *reinterpret_cast<typename Pack<T, W>::type*>(p) = x;
}
template <typename T, int W>
__device__ __forceinline__ void unpack(const typename Pack<T, W>::type& x, T (&v)[W]) {
  const T* xs = reinterpret_cast<const T*>(&x);
#pragma unroll
  for (int e = 0; e < W; ++e) v[e] = xs[e];
}

// corr[r][e] = sum_{j < KMAX} C[j*ld + i + e] cs[r][j] for the VW rows at i
// (cs zero beyond k, so the predicated-off columns add nothing).  Columns go
// in chunks (24 vectors for one RHS, fewer for several, whose loaded vectors
// and accumulators need the registers), each chunk's loads issued together.
template <typename T, int KMAX, int R, int W>
__device__ __forceinline__ void correct_vec(const T* __restrict__ C, int64_t ld, int k, int64_t i,
                                            const T (*cs)[KMAX > 0 ? KMAX : 1], const bool (&act)[R],
                                            T (&corr)[R][W]) {
  constexpr int CHR = W > 1 ? 24 : (KMAX > 0 ? KMAX : 1);
  constexpr int CH = KMAX < CHR ? (KMAX > 0 ? KMAX : 1) : CHR;
  using V = typename Pack<T, W>::type;
#pragma unroll
  for (int r = 0; r < R; ++r)
#pragma unroll
    for (int e = 0; e < W; ++e) corr[r][e] = T(0);
#pragma unroll
  for (int j0 = 0; j0 < KMAX; j0 += CH) {
    V m[CH];
#pragma unroll
    for (int u = 0; u < CH; ++u) {
      const int j = j0 + u;
      if (j < KMAX && j < k) m[u] = ldv<T, W>(C + (int64_t)j * ld + i);
      else m[u] = V{};
    }
#pragma unroll
    for (int u = 0; u < CH; ++u) {
      const int j = j0 + u;
      if (j >= KMAX) break;
      T mv[W];
      unpack<T, W>(m[u], mv);
#pragma unroll
      for (int r = 0; r < R; ++r) {
        if (!act[r]) continue;
        const T z = cs[r][j];
#pragma unroll
        for (int e = 0; e < W; ++e) corr[r][e] = fma_t(mv[e], z, corr[r][e]);
      }
    }
  }
}

// ---------------------------------------------------------------- P2
template <typename T, int KMAX, int R>
__global__ void __launch_bounds__(kBlock, 2) k_p2(IterArgs<T> a) {
  IterState* st = a.st;
  bool act[R];
  bool any = false;
#pragma unroll
  for (int r = 0; r < R; ++r) {
    act[r] = (r < a.nrhs) && !st[r].done;
    any |= act[r];
  }
  if (!any) return;
  constexpr int KK = KMAX > 0 ? KMAX : 1;
  constexpr int W = StreamVW<T, R>::value;
  using V = typename Pack<T, W>::type;
  __shared__ ReduceSmem<R> sm;
  __shared__ __align__(16) T zs[R][KK];
  __shared__ const T* pvs[2 * R];
  __shared__ int npvs;
  if (threadIdx.x == 0) {
    int n = 0;
    for (int r = 0; r < R; ++r)
      if (act[r]) {
        pvs[n++] = a.qraw[r];
        pvs[n++] = a.r[r];
      }
    npvs = n;
  }
  const int k = KMAX > 0 ? st[0].k : 0;
  for (int e = threadIdx.x; e < R * KK; e += blockDim.x) {
    const int r = e / KK, j = e % KK;
    zs[r][j] = (act[r] && j < k) ? (T)st[r].zeta[j] : T(0);
  }
  T al[R];
#pragma unroll
  for (int r = 0; r < R; ++r) al[r] = (T)st[r].alpha;
  __syncthreads();
  const int npv = npvs;
  const int64_t npad = a.npad, nvec = npad / W, stride = gstride(), ld = a.ld;
  const int lane = threadIdx.x & 31;
  Acc<T> acc[R];
  for (int64_t i0 = gtid(); i0 < nvec; i0 += stride) {
    const int64_t i = i0 * W;
    if (W > 1) {   // the warp's rows two steps ahead go to L2
      const int64_t row0 = (i0 - lane + 2 * stride) * W;
      if (row0 < npad)
        prefetch_rows<T>(a.C, ld, KMAX > 0 ? k : 0, pvs, npv, row0, (int)(npad - row0 < 32 * W ? npad - row0 : 32 * W));
    }
    V qr[R], rr[R];
#pragma unroll
    for (int r = 0; r < R; ++r) {
      qr[r] = act[r] ? ldv<T, W>(a.qraw[r] + i) : V{};
      rr[r] = act[r] ? ldv<T, W>(a.r[r] + i) : V{};
    }
    T corr[R][W];
    if (KMAX > 0) correct_vec<T, KMAX, R, W>(a.C, ld, k, i, zs, act, corr);
#pragma unroll
    for (int r = 0; r < R; ++r) {
      if (!act[r]) continue;
      T q[W], rv[W], sv[W];
      unpack<T, W>(qr[r], q);
      unpack<T, W>(rr[r], rv);
#pragma unroll
      for (int e = 0; e < W; ++e) {
        if (KMAX > 0) q[e] -= corr[r][e];
        sv[e] = rv[e] - al[r] * q[e];
        acc[r].add(sv[e], sv[e]);
      }
      if (KMAX > 0) stv<T, W>(a.q[r] + i, q);
      stv<T, W>(a.s[r] + i, sv);
    }
  }
#pragma unroll
  for (int r = 0; r < R; ++r) {
    if (act[r]) warp_slot(acc[r], r, sm);
    else zero_slot(r, sm);
  }
  if (grid_finish<R>(R, sm, a.partials, &st[0].ticket[P2])) RB_FINISH_WARPS(R, act, finish_p2(&st[r], sm.res + r));
}

// ---------------------------------------------------------------- P4 (k > 0)
template <typename T, int KMAX, int R>
__global__ void __launch_bounds__(kBlock, 2) k_p4(IterArgs<T> a) {
  IterState* st = a.st;
  bool act[R];
  bool any = false;
#pragma unroll
  for (int r = 0; r < R; ++r) {
    act[r] = (r < a.nrhs) && !st[r].done && !st[r].half;
    any |= act[r];
  }
  if (!any) return;
  constexpr int W = StreamVW<T, R>::value;
  using V = typename Pack<T, W>::type;
  __shared__ ReduceSmem<4 * R> sm;
  __shared__ __align__(16) T gs[R][KMAX];
  __shared__ const T* pvs[2 * R + 1];
  __shared__ int npvs;
  if (threadIdx.x == 0) {
    int n = 0;
    pvs[n++] = a.rt0;
    for (int r = 0; r < R; ++r)
      if (act[r]) {
        pvs[n++] = a.traw[r];
        pvs[n++] = a.s[r];
      }
    npvs = n;
  }
  const int k = st[0].k;
  for (int e = threadIdx.x; e < R * KMAX; e += blockDim.x) {
    const int r = e / KMAX, j = e % KMAX;
    gs[r][j] = (act[r] && j < k) ? (T)st[r].gamma[j] : T(0);
  }
  __syncthreads();
  const int npv = npvs;
  const T* __restrict__ rt0 = a.rt0;
  const int64_t npad = a.npad, nvec = npad / W, stride = gstride(), ld = a.ld;
  const int lane = threadIdx.x & 31;
  Acc<T> acc[R][4];
  for (int64_t i0 = gtid(); i0 < nvec; i0 += stride) {
    const int64_t i = i0 * W;
    if (W > 1) {
      const int64_t row0 = (i0 - lane + 2 * stride) * W;
      if (row0 < npad) prefetch_rows<T>(a.C, ld, k, pvs, npv, row0, (int)(npad - row0 < 32 * W ? npad - row0 : 32 * W));
    }
    V tr[R], sr[R];
#pragma unroll
    for (int r = 0; r < R; ++r) {
      tr[r] = act[r] ? ldv<T, W>(a.traw[r] + i) : V{};
      sr[r] = act[r] ? ldv<T, W>(a.s[r] + i) : V{};
    }
    T rv[W];
    unpack<T, W>(ldv<T, W>(rt0 + i), rv);
    T corr[R][W];
    correct_vec<T, KMAX, R, W>(a.C, ld, k, i, gs, act, corr);
#pragma unroll
    for (int r = 0; r < R; ++r) {
      if (!act[r]) continue;
      T t[W], sv[W];
      unpack<T, W>(tr[r], t);
      unpack<T, W>(sr[r], sv);
#pragma unroll
      for (int e = 0; e < W; ++e) {
        t[e] -= corr[r][e];
        acc[r][0].add(sv[e], t[e]);
        acc[r][1].add(t[e], t[e]);
        acc[r][2].add(rv[e], t[e]);
        acc[r][3].add(rv[e], sv[e]);
      }
      stv<T, W>(a.t[r] + i, t);
    }
  }
#pragma unroll
  for (int r = 0; r < R; ++r)
#pragma unroll
    for (int d = 0; d < 4; ++d) {
      if (act[r]) warp_slot(acc[r][d], 4 * r + d, sm);
      else zero_slot(4 * r + d, sm);
    }
  if (grid_finish<4 * R>(4 * R, sm, a.partials, &st[0].ticket[P4]))
    RB_FINISH_WARPS(R, act, finish_p4(&st[r], sm.res + 4 * r, k));
}

// ---------------------------------------------------------------- P5
template <typename T, int KMAX, int R>
__global__ void __launch_bounds__(kBlock, 3) k_p5(IterArgs<T> a) {
  IterState* st = a.st;
  bool act[R], half[R];
  bool any = false;
#pragma unroll
  for (int r = 0; r < R; ++r) {
    act[r] = (r < a.nrhs) && !st[r].done;
    half[r] = act[r] && st[r].half;
    any |= act[r];
  }
  if (!any) return;
  constexpr int W = StreamVW<T, R>::value;
  using V = typename Pack<T, W>::type;
  __shared__ ReduceSmem<R> sm;
  // vectors read by this pass (x and p are also written here, so they use
  // coherent loads; s, t, q use the read-only path)
  __shared__ const T* pvs[5 * R];
  __shared__ int npvs;
  if (threadIdx.x == 0) {
    int n = 0;
    for (int r = 0; r < R; ++r)
      if (act[r]) {
        pvs[n++] = a.p_in[r];
        pvs[n++] = a.s[r];
        pvs[n++] = a.x[r];
        if (!half[r]) {
          pvs[n++] = a.t[r];
          pvs[n++] = a.q[r];
        }
      }
    npvs = n;
  }
  __syncthreads();
  const int npv = npvs;
  const int k = KMAX > 0 ? st[0].k : 0;
  T al[R], om[R], be[R];
#pragma unroll
  for (int r = 0; r < R; ++r) {
    al[r] = (T)st[r].alpha;
    om[r] = (T)st[r].omega;
    be[r] = (T)st[r].beta;
  }
  const int64_t npad = a.npad, nvec = npad / W, stride = gstride();
  const int lane = threadIdx.x & 31;
  Acc<T> acc[R];
  for (int64_t i0 = gtid(); i0 < nvec; i0 += stride) {
    const int64_t i = i0 * W;
    {
      const int64_t row0 = (i0 - lane + 2 * stride) * W;
      if (row0 < npad)
        prefetch_rows<T>(nullptr, 0, 0, pvs, npv, row0, (int)(npad - row0 < 32 * W ? npad - row0 : 32 * W));
    }
    V P[R], S[R], X[R], Tt[R], Q[R];
#pragma unroll
    for (int r = 0; r < R; ++r) {
      P[r] = act[r] ? ldv_coherent<T, W>(a.p_in[r] + i) : V{};
      S[r] = act[r] ? ldv<T, W>(a.s[r] + i) : V{};
      X[r] = act[r] ? ldv_coherent<T, W>(a.x[r] + i) : V{};
      Tt[r] = (act[r] && !half[r]) ? ldv<T, W>(a.t[r] + i) : V{};
      Q[r] = (act[r] && !half[r]) ? ldv<T, W>(a.q[r] + i) : V{};
    }
#pragma unroll
    for (int r = 0; r < R; ++r) {
      if (!act[r]) continue;
      T p[W], s_[W], x[W], t[W], q[W];
      unpack<T, W>(P[r], p);
      unpack<T, W>(S[r], s_);
      unpack<T, W>(X[r], x);
      unpack<T, W>(Tt[r], t);
      unpack<T, W>(Q[r], q);
      if (half[r]) {
#pragma unroll
        for (int e = 0; e < W; ++e) x[e] = fma_t(al[r], p[e], x[e]);
        stv<T, W>(a.x[r] + i, x);
        stv<T, W>(a.r[r] + i, s_);
        continue;
      }
      T rr[W], pn[W];
#pragma unroll
      for (int e = 0; e < W; ++e) {
        rr[e] = s_[e] - om[r] * t[e];
        x[e] = fma_t(om[r], s_[e], fma_t(al[r], p[e], x[e]));
        pn[e] = fma_t(be[r], p[e] - om[r] * q[e], rr[e]);
        acc[r].add(rr[e], rr[e]);
      }
      stv<T, W>(a.x[r] + i, x);
      stv<T, W>(a.r[r] + i, rr);
      stv<T, W>(a.p_out[r] + i, pn);
    }
  }
#pragma unroll
  for (int r = 0; r < R; ++r) {
    if (act[r]) warp_slot(acc[r], r, sm);
    else zero_slot(r, sm);
  }
  if (grid_finish<R>(R, sm, a.partials, &st[0].ticket[P5])) RB_FINISH_WARPS(R, act, finish_p5(&st[r], sm.res + r, k));
}

// ---------------------------------------------------------------- staged streaming (R > 1)
// A block of several right-hand sides streams up to k + 9 arrays per row
// (P4: k columns of C, r~_0, t_raw and s per RHS).  Register-held loads
// cannot keep enough of them in flight, so these passes stage tiles of
// kBlock rows of every stream into shared memory with cp.async (16-byte
// copies spread over the block's threads, NSTG tiles in flight) and then
// compute one row per thread from the staged tile.  Blocks take tiles
// round-robin; the arithmetic per row is the same as the register-held
// path's, in the same order.
template <typename T, int NSMAX>
struct StageCfg {
  static constexpr size_t per = (size_t)NSMAX * kBlock * sizeof(T);   // one tile of every stream
  static constexpr int nstg = 3 * per <= 112 * 1024 ? 3 : 2;
  static constexpr bool ok = 2 * per <= 200 * 1024;
  static constexpr size_t bytes = ok ? nstg * per : 0;
};

template <typename T, int KMAX, int R>
struct Staged {
  static constexpr bool value = R > 1 && StageCfg<T, (KMAX + 2 * R + 1 > 5 * R ? KMAX + 2 * R + 1 : 5 * R)>::ok;
  using P2 = StageCfg<T, KMAX + 2 * R>;
  using P4 = StageCfg<T, KMAX + 2 * R + 1>;
  using P5 = StageCfg<T, 5 * R>;
};

// Stream rows [0, npad) of kc columns of the column-major block C (leading
// dimension ld) followed by the nv vectors vsrc[0..nv) (a list in shared
// memory) through the NSTG-stage buffer `buf` ([stage][stream][kBlock]) and
// call f(row, sb) for this thread's row of each tile, with stream s's value
// at sb[s * kBlock].  Each thread always copies the same 16-byte chunk
// position of a stream's tile.  Every thread of the block must call this.
template <typename T, int NSTG, typename F>
__device__ __forceinline__ void staged_rows(const T* __restrict__ C, int64_t ld, int kc, const T* const* vsrc, int nv,
                                            int64_t npad, T* buf, F&& f) {
  constexpr int VC = 16 / (int)sizeof(T);   // values per 16-byte copy
  constexpr int CPS = kBlock / VC;          // copies per stream and tile
  constexpr int SPP = kBlock / CPS;         // streams per pass of the block
  const int ns = kc + nv;
  const int64_t ntiles = (npad + kBlock - 1) / kBlock;
  const int64_t stage = (int64_t)ns * kBlock;
  const int64_t step = gridDim.x;
  const int c = threadIdx.x % CPS, s0 = threadIdx.x / CPS;
  auto issue = [&](int64_t tile, int stg) {
    const int64_t row = tile * kBlock + (int64_t)c * VC;
    if (tile < ntiles && row < npad) {
      T* b = buf + stg * stage + c * VC;
      for (int sidx = s0; sidx < ns; sidx += SPP) {
        const T* src = sidx < kc ? C + (int64_t)sidx * ld : vsrc[sidx - kc];
        cp_async16(b + (int64_t)sidx * kBlock, src + row);
      }
    }
    cp_async_commit();
  };
  int64_t tile = blockIdx.x;
#pragma unroll
  for (int q = 0; q < NSTG - 1; ++q) issue(tile + q * step, q);
  int stg = 0;
  for (; tile < ntiles; tile += step) {
    // refill the stage read in the previous step (all threads are past it)
    issue(tile + (NSTG - 1) * step, stg == 0 ? NSTG - 1 : stg - 1);
    cp_async_wait<NSTG - 1>();   // this thread's copies of `tile` landed
    __syncthreads();             // ... and every thread's
    const int64_t row = tile * kBlock + threadIdx.x;
    if (row < npad) f(row, buf + stg * stage + threadIdx.x);
    __syncthreads();
    stg = stg == NSTG - 1 ? 0 : stg + 1;
  }
  cp_async_wait<0>();
}

// The same stream through bulk copies: one 1D cp.async.bulk per stream and
// tile (kBlock rows, 16-byte aligned as every array here is), issued by the
// lanes of warp 0 and completing as transaction bytes on the stage's
// mbarrier, so the block's threads spend no instructions on addresses and
// copies and only wait (bounded, mbar.cuh) for the stage to land.  Returns
// false when a wait expired; the copies still in flight are then waited for
// (bounded) before the CTA leaves.
template <typename T, int NSTG, typename F>
__device__ __forceinline__ bool staged_rows_bulk(const T* __restrict__ C, int64_t ld, int kc, const T* const* vsrc,
                                                 int nv, int64_t npad, T* buf, F&& f) {
  __shared__ __align__(8) uint64_t bars[NSTG];
  __shared__ int s_abort;
  const int ns = kc + nv;
  const int64_t ntiles = (npad + kBlock - 1) / kBlock;
  const int64_t stage = (int64_t)ns * kBlock;
  const int64_t step = gridDim.x;
  const int lane = threadIdx.x & 31;
  const bool producer = threadIdx.x < 32;
  if (threadIdx.x == 0) {
    for (int q = 0; q < NSTG; ++q) mbar_init(smem_u32(&bars[q]), 1);
    s_abort = 0;
    fence_barrier_init();
  }
  __syncthreads();
  uint32_t pending = 0;   // warp 0: stages issued and not yet consumed
  auto issue = [&](int64_t tile, int stg) {
    if (tile >= ntiles) return;
    const int64_t row0 = tile * kBlock;
    const uint32_t bytes = (uint32_t)(npad - row0 < kBlock ? npad - row0 : kBlock) * (uint32_t)sizeof(T);
    const uint32_t bar = smem_u32(&bars[stg]);
    if (lane == 0) {
      fence_proxy_async();   // the block's reads of this stage come first
      mbar_expect_tx(bar, bytes * (uint32_t)ns);
    }
    __syncwarp();
    T* b = buf + stg * stage;
    for (int sidx = lane; sidx < ns; sidx += 32) {
      const T* src = sidx < kc ? C + (int64_t)sidx * ld : vsrc[sidx - kc];
      bulk_load_1d(smem_u32(b + (int64_t)sidx * kBlock), src + row0, bytes, bar);
    }
    pending |= 1u << stg;
  };
  int64_t tile = blockIdx.x;
  if (producer)
#pragma unroll
    for (int q = 0; q < NSTG - 1; ++q) issue(tile + q * step, q);
  int stg = 0;
  uint32_t phase = 0;     // parity bit per stage
  bool ok = true;
  for (; tile < ntiles; tile += step) {
    if (producer) issue(tile + (NSTG - 1) * step, stg == 0 ? NSTG - 1 : stg - 1);
    const uint32_t bar = smem_u32(&bars[stg]);
    const uint32_t par = (phase >> stg) & 1u;
    const bool landed = mbar_test(bar, par) || mbar_wait(bar, par, &s_abort);
    phase ^= 1u << stg;
    pending &= ~(1u << stg);
    const int64_t row = tile * kBlock + threadIdx.x;
    if (landed && row < npad) f(row, buf + stg * stage + threadIdx.x);
    __syncthreads();
    if (s_abort) {
      ok = false;
      break;
    }
    stg = stg == NSTG - 1 ? 0 : stg + 1;
  }
  if (!ok && lane == 0 && producer) {
    for (int q = 0; q < NSTG; ++q)
      if (pending & (1u << q)) mbar_wait(smem_u32(&bars[q]), (phase >> q) & 1u, nullptr);
  }
  __syncthreads();
  return ok;
}

// Stage rows by bulk copies (bulk != 0) or by per-thread cp.async.
template <typename T, int NSTG, typename F>
__device__ __forceinline__ bool stage_rows(int bulk, const T* __restrict__ C, int64_t ld, int kc, const T* const* vsrc,
                                           int nv, int64_t npad, T* buf, F&& f) {
  if (bulk) return staged_rows_bulk<T, NSTG>(C, ld, kc, vsrc, nv, npad, buf, f);
  staged_rows<T, NSTG>(C, ld, kc, vsrc, nv, npad, buf, f);
  return true;
}

// A staged pass whose copies did not land marks its right-hand sides failed.
#define RB_STAGE_TIMEOUT(R, ACT)                                      \
  do {                                                                \
    if (threadIdx.x == 0)                                             \
      for (int r_ = 0; r_ < (R); ++r_)                                \
        if (ACT[r_]) fail(&st[r_], RB_ETIMEOUT);                      \
  } while (0)

// Warp sums of the pair accumulators acc[h][d] (right-hand sides 2h, 2h+1)
// into the slots slot(r, d); inactive right-hand sides give zeros.
template <typename T, int R, int ND, int NV, typename SlotF>
__device__ __forceinline__ void pair_slots(const AccP<T> (&acc)[R / 2][ND], const bool (&act)[R], ReduceCore<NV>& sm,
                                           SlotF slot) {
#pragma unroll
  for (int r = 0; r < R; ++r)
#pragma unroll
    for (int d = 0; d < ND; ++d) {
      if (act[r]) warp_slot(acc[r / 2][d].lane(r & 1), slot(r, d), sm);
      else zero_slot(slot(r, d), sm);
    }
}

// Stream lists of the staged passes: slot r's vectors start at vix[r] (0 for
// an inactive slot, whose values are read but never used).
// P2 for R > 1: q = q_raw - C zeta, s = r - alpha q, ||s||^2.
template <typename T, int KMAX, int R>
__global__ void __launch_bounds__(kBlock, 1) k_p2_staged(IterArgs<T> a) {
  using P = Pair<T>;
  using V = typename P::V;
  constexpr int H = R / 2;
  IterState* st = a.st;
  bool act[R];
  bool any = false;
#pragma unroll
  for (int r = 0; r < R; ++r) {
    act[r] = (r < a.nrhs) && !st[r].done;
    any |= act[r];
  }
  if (!any) return;
  constexpr int KK = KMAX > 0 ? KMAX : 1;
  using SC = typename Staged<T, KMAX, R>::P2;
  extern __shared__ __align__(16) unsigned char dsm[];
  __shared__ ReduceCore<R> sm;
  __shared__ __align__(16) T zs[KK][R];   // zeta, interleaved by right-hand side
  __shared__ const T* src[2 * R];
  __shared__ int vix[R], nsrc;
  const int k = KMAX > 0 ? st[0].k : 0;
  if (threadIdx.x == 0) {
    int n = 0;
    for (int r = 0; r < R; ++r) {
      vix[r] = act[r] ? k + n : 0;
      if (act[r]) {
        src[n++] = a.qraw[r];
        src[n++] = a.r[r];
      }
    }
    nsrc = n;
  }
  for (int e = threadIdx.x; e < R * KK; e += blockDim.x) {
    const int j = e / R, r = e % R;
    zs[j][r] = (act[r] && j < k) ? (T)st[r].zeta[j] : T(0);
  }
  V al[H];
#pragma unroll
  for (int h = 0; h < H; ++h) al[h] = P::neg(P::mk((T)st[2 * h].alpha, (T)st[2 * h + 1].alpha));
  __syncthreads();
  int vi[R];
#pragma unroll
  for (int r = 0; r < R; ++r) vi[r] = vix[r];
  AccP<T> acc[H][1];
  auto row_fn = [&](int64_t row, const T* sb) {
    V corr[H];
#pragma unroll
    for (int h = 0; h < H; ++h) corr[h] = P::mk(T(0), T(0));
#pragma unroll
    for (int j = 0; j < KMAX; ++j) {
      if (j >= k) break;
      const T c = sb[j * kBlock];
      const V* z = reinterpret_cast<const V*>(zs[j]);
#pragma unroll
      for (int h = 0; h < H; ++h) corr[h] = P::fma(P::mk(c, c), z[h], corr[h]);
    }
#pragma unroll
    for (int h = 0; h < H; ++h) {
      const int r0 = 2 * h, r1 = 2 * h + 1;
      V q = P::mk(sb[vi[r0] * kBlock], sb[vi[r1] * kBlock]);
      const V rv = P::mk(sb[(vi[r0] + 1) * kBlock], sb[(vi[r1] + 1) * kBlock]);
      if (KMAX > 0) q = P::add(q, P::neg(corr[h]));
      const V sv = P::fma(al[h], q, rv);   // r - alpha q
      acc[h][0].add(sv, sv);
      if (act[r0]) {
        if (KMAX > 0) a.q[r0][row] = q.x;
        a.s[r0][row] = sv.x;
      }
      if (act[r1]) {
        if (KMAX > 0) a.q[r1][row] = q.y;
        a.s[r1][row] = sv.y;
      }
    }
  };
  if (!stage_rows<T, SC::nstg>(a.stage_bulk & 1, a.C, a.ld, k, src, nsrc, a.npad, reinterpret_cast<T*>(dsm), row_fn))
    RB_STAGE_TIMEOUT(R, act);
  pair_slots<T, R, 1>(acc, act, sm, [](int r, int) { return r; });
  if (grid_finish<R>(R, sm, a.partials, &st[0].ticket[P2])) RB_FINISH_WARPS(R, act, finish_p2(&st[r], sm.res + r));
}

// P4 for R > 1: t = t_raw - C gamma; (s,t), (t,t), (r~0,t), (r~0,s).
template <typename T, int KMAX, int R>
__global__ void __launch_bounds__(kBlock, 1) k_p4_staged(IterArgs<T> a) {
  using P = Pair<T>;
  using V = typename P::V;
  constexpr int H = R / 2;
  IterState* st = a.st;
  bool act[R];
  bool any = false;
#pragma unroll
  for (int r = 0; r < R; ++r) {
    act[r] = (r < a.nrhs) && !st[r].done && !st[r].half;
    any |= act[r];
  }
  if (!any) return;
  using SC = typename Staged<T, KMAX, R>::P4;
  extern __shared__ __align__(16) unsigned char dsm[];
  __shared__ ReduceCore<4 * R> sm;
  __shared__ __align__(16) T gs[KMAX][R];   // gamma, interleaved by right-hand side
  __shared__ const T* src[2 * R + 1];
  __shared__ int vix[R], nsrc;
  const int k = st[0].k;
  if (threadIdx.x == 0) {
    int n = 0;
    src[n++] = a.rt0;
    for (int r = 0; r < R; ++r) {
      vix[r] = act[r] ? k + n : 0;
      if (act[r]) {
        src[n++] = a.traw[r];
        src[n++] = a.s[r];
      }
    }
    nsrc = n;
  }
  for (int e = threadIdx.x; e < R * KMAX; e += blockDim.x) {
    const int j = e / R, r = e % R;
    gs[j][r] = (act[r] && j < k) ? (T)st[r].gamma[j] : T(0);
  }
  __syncthreads();
  int vi[R];
#pragma unroll
  for (int r = 0; r < R; ++r) vi[r] = vix[r];
  AccP<T> acc[H][4];
  auto row_fn = [&](int64_t row, const T* sb) {
    V corr[H];
#pragma unroll
    for (int h = 0; h < H; ++h) corr[h] = P::mk(T(0), T(0));
#pragma unroll
    for (int j = 0; j < KMAX; ++j) {
      if (j >= k) break;
      const T c = sb[j * kBlock];
      const V* g = reinterpret_cast<const V*>(gs[j]);
#pragma unroll
      for (int h = 0; h < H; ++h) corr[h] = P::fma(P::mk(c, c), g[h], corr[h]);
    }
    const T rs = sb[k * kBlock];
    const V rv = P::mk(rs, rs);
#pragma unroll
    for (int h = 0; h < H; ++h) {
      const int r0 = 2 * h, r1 = 2 * h + 1;
      const V t = P::add(P::mk(sb[vi[r0] * kBlock], sb[vi[r1] * kBlock]), P::neg(corr[h]));
      const V sv = P::mk(sb[(vi[r0] + 1) * kBlock], sb[(vi[r1] + 1) * kBlock]);
      acc[h][0].add(sv, t);
      acc[h][1].add(t, t);
      acc[h][2].add(rv, t);
      acc[h][3].add(rv, sv);
      if (act[r0]) a.t[r0][row] = t.x;
      if (act[r1]) a.t[r1][row] = t.y;
    }
  };
  if (!stage_rows<T, SC::nstg>(a.stage_bulk & 2, a.C, a.ld, k, src, nsrc, a.npad, reinterpret_cast<T*>(dsm), row_fn))
    RB_STAGE_TIMEOUT(R, act);
  pair_slots<T, R, 4>(acc, act, sm, [](int r, int d) { return 4 * r + d; });
  if (grid_finish<4 * R>(4 * R, sm, a.partials, &st[0].ticket[P4]))
    RB_FINISH_WARPS(R, act, finish_p4(&st[r], sm.res + 4 * r, k));
}

// P5 for R > 1: x += alpha p + omega s; r = s - omega t; ||r||^2;
// p_{i+1} = r + beta (p - omega q)  (half step: x += alpha p, r = s).
template <typename T, int KMAX, int R>
__global__ void __launch_bounds__(kBlock, 1) k_p5_staged(IterArgs<T> a) {
  using P = Pair<T>;
  using V = typename P::V;
  constexpr int H = R / 2;
  IterState* st = a.st;
  bool act[R], half[R];
  bool any = false, anyhalf = false;
#pragma unroll
  for (int r = 0; r < R; ++r) {
    act[r] = (r < a.nrhs) && !st[r].done;
    half[r] = act[r] && st[r].half;
    any |= act[r];
    anyhalf |= half[r];
  }
  if (!any) return;
  using SC = typename Staged<T, KMAX, R>::P5;
  extern __shared__ __align__(16) unsigned char dsm[];
  __shared__ ReduceCore<R> sm;
  __shared__ const T* src[5 * R];
  __shared__ int vix[R], nsrc;
  if (threadIdx.x == 0) {
    int n = 0;
    for (int r = 0; r < R; ++r) {
      vix[r] = act[r] ? n : 0;
      if (act[r]) {
        src[n++] = a.p_in[r];
        src[n++] = a.s[r];
        src[n++] = a.x[r];
        if (!half[r]) {
          src[n++] = a.t[r];
          src[n++] = a.q[r];
        }
      }
    }
    nsrc = n;
  }
  const int k = KMAX > 0 ? st[0].k : 0;
  T al[R], om[R], be[R];
#pragma unroll
  for (int r = 0; r < R; ++r) {
    al[r] = (T)st[r].alpha;
    om[r] = (T)st[r].omega;
    be[r] = (T)st[r].beta;
  }
  __syncthreads();
  int vi[R];
#pragma unroll
  for (int r = 0; r < R; ++r) vi[r] = vix[r];
  AccP<T> acc[H][1];
  auto row_fn = [&](int64_t row, const T* sb) {
    if (!anyhalf) {
#pragma unroll
      for (int h = 0; h < H; ++h) {
        const int r0 = 2 * h, r1 = 2 * h + 1;
        const T* v0 = sb + vi[r0] * kBlock;
        const T* v1 = sb + vi[r1] * kBlock;
        const V p = P::mk(v0[0], v1[0]), s_ = P::mk(v0[kBlock], v1[kBlock]), x = P::mk(v0[2 * kBlock], v1[2 * kBlock]);
        const V t = P::mk(v0[3 * kBlock], v1[3 * kBlock]), q = P::mk(v0[4 * kBlock], v1[4 * kBlock]);
        const V om2 = P::mk(om[r0], om[r1]), nom = P::neg(om2);
        const V rr = P::fma(nom, t, s_);                                        // s - omega t
        const V xn = P::fma(om2, s_, P::fma(P::mk(al[r0], al[r1]), p, x));     // x + alpha p + omega s
        const V pn = P::fma(P::mk(be[r0], be[r1]), P::fma(nom, q, p), rr);      // r + beta (p - omega q)
        acc[h][0].add(rr, rr);
        if (act[r0]) {
          a.x[r0][row] = xn.x;
          a.r[r0][row] = rr.x;
          a.p_out[r0][row] = pn.x;
        }
        if (act[r1]) {
          a.x[r1][row] = xn.y;
          a.r[r1][row] = rr.y;
          a.p_out[r1][row] = pn.y;
        }
      }
      return;
    }
#pragma unroll
    for (int r = 0; r < R; ++r) {
      if (!act[r]) continue;
      const T* v = sb + vi[r] * kBlock;
      const T p = v[0], s_ = v[kBlock], x = v[2 * kBlock];
      if (half[r]) {
        a.x[r][row] = fma_t(al[r], p, x);
        a.r[r][row] = s_;
        continue;
      }
      const T t = v[3 * kBlock], q = v[4 * kBlock];
      const T rr = fma_t(-om[r], t, s_);
      const T xn = fma_t(om[r], s_, fma_t(al[r], p, x));
      const T pn = fma_t(be[r], fma_t(-om[r], q, p), rr);
      // the lane of the pair accumulator that belongs to r
      const V rr2 = (r & 1) ? P::mk(T(0), rr) : P::mk(rr, T(0));
      acc[r / 2][0].add(rr2, rr2);
      a.x[r][row] = xn;
      a.r[r][row] = rr;
      a.p_out[r][row] = pn;
    }
  };
  if (!stage_rows<T, SC::nstg>(a.stage_bulk & 4, a.C, a.ld, 0, src, nsrc, a.npad, reinterpret_cast<T*>(dsm), row_fn))
    RB_STAGE_TIMEOUT(R, act);
  pair_slots<T, R, 1>(acc, act, sm, [](int r, int) { return r; });
  if (grid_finish<R>(R, sm, a.partials, &st[0].ticket[P5])) RB_FINISH_WARPS(R, act, finish_p5(&st[r], sm.res + r, k));
}

// Kernel and dynamic shared memory of P2 / P4 / P5 for one configuration.
template <typename T, int KMAX, int R>
struct StreamKernels {
  static constexpr bool staged = Staged<T, KMAX, R>::value;
  static constexpr int K4 = KMAX > 0 ? KMAX : 1;
  static const void* p2() {
    if constexpr (staged) return (const void*)k_p2_staged<T, KMAX, R>;
    else return (const void*)k_p2<T, KMAX, R>;
  }
  static const void* p4() {
    if constexpr (staged) return (const void*)k_p4_staged<T, K4, R>;
    else return (const void*)k_p4<T, K4, R>;
  }
  static const void* p5() {
    if constexpr (staged) return (const void*)k_p5_staged<T, KMAX, R>;
    else return (const void*)k_p5<T, KMAX, R>;
  }
  static constexpr size_t d2 = staged ? Staged<T, KMAX, R>::P2::bytes : 0;
  static constexpr size_t d4 = staged ? Staged<T, K4, R>::P4::bytes : 0;
  static constexpr size_t d5 = staged ? Staged<T, KMAX, R>::P5::bytes : 0;
};

template <typename T, int KMAX, int R>
static void launch_p2(const IterArgs<T>& a, const Grids& g, cudaStream_t s) {
  using SK = StreamKernels<T, KMAX, R>;
  if constexpr (SK::staged) k_p2_staged<T, KMAX, R><<<g.pass[P2], kBlock, SK::d2, s>>>(a);
  else k_p2<T, KMAX, R><<<g.pass[P2], kBlock, 0, s>>>(a);
}
template <typename T, int KMAX, int R>
static void launch_p4(const IterArgs<T>& a, const Grids& g, cudaStream_t s) {
  using SK = StreamKernels<T, KMAX, R>;
  constexpr int K4 = SK::K4;
  if constexpr (SK::staged) k_p4_staged<T, K4, R><<<g.pass[P4], kBlock, SK::d4, s>>>(a);
  else k_p4<T, K4, R><<<g.pass[P4], kBlock, 0, s>>>(a);
}
template <typename T, int KMAX, int R>
static void launch_p5(const IterArgs<T>& a, const Grids& g, cudaStream_t s) {
  using SK = StreamKernels<T, KMAX, R>;
  if constexpr (SK::staged) k_p5_staged<T, KMAX, R><<<g.pass[P5], kBlock, SK::d5, s>>>(a);
  else k_p5<T, KMAX, R><<<g.pass[P5], kBlock, 0, s>>>(a);
}

// ---------------------------------------------------------------- launchers
template <typename T, int KMAX, int R>
static cudaError_t launch_iter_kr(const IterArgs<T>& a, const Grids& g, cudaStream_t s) {
  constexpr size_t dsm = P13Smem<T, KMAX, R>::bytes;
  k_p1<T, KMAX, R><<<g.pass[P1], kBlock, dsm, s>>>(a);
  launch_p2<T, KMAX, R>(a, g, s);
  k_p3<T, KMAX, R><<<g.pass[P3], kBlock, dsm, s>>>(a);
  if (KMAX > 0) launch_p4<T, KMAX, R>(a, g, s);
  launch_p5<T, KMAX, R>(a, g, s);
  return cudaGetLastError();
}

template <typename T, int KMAX, int R>
static cudaError_t launch_pass_kr(int pass, const IterArgs<T>& a, const Grids& g, cudaStream_t s) {
  constexpr size_t dsm = P13Smem<T, KMAX, R>::bytes;
  switch (pass) {
    case P1: k_p1<T, KMAX, R><<<g.pass[P1], kBlock, dsm, s>>>(a); break;
    case P2: launch_p2<T, KMAX, R>(a, g, s); break;
    case P3: k_p3<T, KMAX, R><<<g.pass[P3], kBlock, dsm, s>>>(a); break;
    case P4: if (KMAX > 0) launch_p4<T, KMAX, R>(a, g, s); break;
    default: launch_p5<T, KMAX, R>(a, g, s); break;
  }
  return cudaGetLastError();
}

int kmax_bucket(int k) {
  if (k <= 0) return 0;
  if (k <= 8) return 8;
  if (k <= 16) return 16;
  if (k <= 24) return 24;
  if (k <= 32) return 32;
  if (k <= 48) return 48;
  return 64;
}

int rhs_bucket(int nrhs) { return nrhs <= 1 ? 1 : (nrhs <= 2 ? 2 : 4); }

// Dispatch (k bucket, RHS bucket) to a compile-time instantiation.
#define RB_DISPATCH(KB, RB, CALL)                                   \
  switch (KB) {                                                     \
    case 0: { constexpr int KM = 0; RB_DISPATCH_R(RB, CALL) }        \
    case 8: { constexpr int KM = 8; RB_DISPATCH_R(RB, CALL) }        \
    case 16: { constexpr int KM = 16; RB_DISPATCH_R(RB, CALL) }      \
    case 24: { constexpr int KM = 24; RB_DISPATCH_R(RB, CALL) }      \
    case 32: { constexpr int KM = 32; RB_DISPATCH_R(RB, CALL) }      \
    case 48: { constexpr int KM = 48; RB_DISPATCH_R(RB, CALL) }      \
    default: { constexpr int KM = 64; RB_DISPATCH_R(RB, CALL) }      \
  }
#define RB_DISPATCH_R(RB, CALL)                                     \
  switch (RB) {                                                     \
    case 1: { constexpr int RR = 1; return CALL; }                  \
    case 2: { constexpr int RR = 2; return CALL; }                  \
    default: { constexpr int RR = 4; return CALL; }                 \
  }

template <typename T>
cudaError_t launch_iteration(const IterArgs<T>& a, int k, const Grids& g, cudaStream_t s) {
  RB_DISPATCH(kmax_bucket(k), rhs_bucket(a.nrhs), (launch_iter_kr<T, KM, RR>(a, g, s)))
}

template <typename T>
cudaError_t launch_pass(int pass, const IterArgs<T>& a, int k, const Grids& g, cudaStream_t s) {
  count_launches(1);
  RB_DISPATCH(kmax_bucket(k), rhs_bucket(a.nrhs), (launch_pass_kr<T, KM, RR>(pass, a, g, s)))
}

template cudaError_t launch_pass<double>(int, const IterArgs<double>&, int, const Grids&, cudaStream_t);
template cudaError_t launch_pass<float>(int, const IterArgs<float>&, int, const Grids&, cudaStream_t);
template cudaError_t launch_iteration<double>(const IterArgs<double>&, int, const Grids&, cudaStream_t);
template cudaError_t launch_iteration<float>(const IterArgs<float>&, int, const Grids&, cudaStream_t);

// Grid sizes: one full wave of resident blocks per kernel configuration (a
// second partial wave would leave SMs idle at the end of every pass), capped
// by the work.
static int occ(const void* f, int nsm, size_t dsm = 0) {
  if (dsm > 0) cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)dsm);
  int b = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, f, kBlock, dsm);
  return (b > 0 ? b : 1) * nsm;
}

template <typename T, int KMAX, int R>
static void grids_kr(int nsm, int64_t npad, Grids* g) {
  // P1/P3: one warp per slice; P2/P4/P5: one thread per 16-byte row vector
  const int64_t work13 = (npad + kBlock - 1) / kBlock;
  const int64_t workv = (npad / StreamVW<T, R>::value + kBlock - 1) / kBlock;
  constexpr size_t dsm = P13Smem<T, KMAX, R>::bytes;
  using SK = StreamKernels<T, KMAX, R>;
  const int o[5] = {occ((const void*)k_p1<T, KMAX, R>, nsm, dsm), occ(SK::p2(), nsm, SK::d2),
                    occ((const void*)k_p3<T, KMAX, R>, nsm, dsm), occ(SK::p4(), nsm, SK::d4),
                    occ(SK::p5(), nsm, SK::d5)};
  for (int p = 0; p < 5; ++p)
    g->pass[p] = (int)std::max<int64_t>(1, std::min<int64_t>((p == P1 || p == P3) ? work13 : workv, o[p]));
  g->spmv = std::max(g->pass[P1], g->pass[P3]);
  g->vec = std::max(g->pass[P2], g->pass[P5]);
}

template <typename T>
static void grids_dispatch(int kb, int rb, int nsm, int64_t npad, Grids* g) {
  switch (kb) {
    case 0: { constexpr int KM = 0; switch (rb) { case 1: grids_kr<T, KM, 1>(nsm, npad, g); return; case 2: grids_kr<T, KM, 2>(nsm, npad, g); return; default: grids_kr<T, KM, 4>(nsm, npad, g); return; } }
    case 8: { constexpr int KM = 8; switch (rb) { case 1: grids_kr<T, KM, 1>(nsm, npad, g); return; case 2: grids_kr<T, KM, 2>(nsm, npad, g); return; default: grids_kr<T, KM, 4>(nsm, npad, g); return; } }
    case 16: { constexpr int KM = 16; switch (rb) { case 1: grids_kr<T, KM, 1>(nsm, npad, g); return; case 2: grids_kr<T, KM, 2>(nsm, npad, g); return; default: grids_kr<T, KM, 4>(nsm, npad, g); return; } }
    case 24: { constexpr int KM = 24; switch (rb) { case 1: grids_kr<T, KM, 1>(nsm, npad, g); return; case 2: grids_kr<T, KM, 2>(nsm, npad, g); return; default: grids_kr<T, KM, 4>(nsm, npad, g); return; } }
    case 32: { constexpr int KM = 32; switch (rb) { case 1: grids_kr<T, KM, 1>(nsm, npad, g); return; case 2: grids_kr<T, KM, 2>(nsm, npad, g); return; default: grids_kr<T, KM, 4>(nsm, npad, g); return; } }
    case 48: { constexpr int KM = 48; switch (rb) { case 1: grids_kr<T, KM, 1>(nsm, npad, g); return; case 2: grids_kr<T, KM, 2>(nsm, npad, g); return; default: grids_kr<T, KM, 4>(nsm, npad, g); return; } }
    default: { constexpr int KM = 64; switch (rb) { case 1: grids_kr<T, KM, 1>(nsm, npad, g); return; case 2: grids_kr<T, KM, 2>(nsm, npad, g); return; default: grids_kr<T, KM, 4>(nsm, npad, g); return; } }
  }
}

template <typename T>
void iteration_grids(int k, int nsm, int64_t npad, Grids* g, int nrhs) {
  grids_dispatch<T>(kmax_bucket(k), rhs_bucket(nrhs), nsm, npad, g);
}

template void iteration_grids<double>(int, int, int64_t, Grids*, int);
template void iteration_grids<float>(int, int, int64_t, Grids*, int);

// ================================================================ RBiCG (Alg. 1)
// Alg. 1 for a primary system A x = b and its dual A^T x~ = b~ (FP64, real,
// so conj(alpha) = alpha).  An iteration starts with the FP64 SpMV +
// projection pass on A (with C-hat) and on A^T (with C); these kernels do
// the rest of it:
//
//   k_b2        after z = A p, z~ = A^T p~ (with C-hat^T z and C^T z~ in the
//               gamma fields of st[0], st[1]): q = z - C zeta, q~ = z~ - C~ zeta~
//               in place (zeta~ = D_c^{-1} C^T z~) and (p~, q) -> st[0].red[0]
//   k_bi_alpha  alpha = (r~, r) / (p~, q), zeta_c += alpha zeta, zeta~_c += alpha zeta~
//   k_b3        x += alpha p, x~ += alpha p~, r -= alpha q, r~ -= alpha q~;
//               ||r||^2, ||r~||^2, (r~, r) -> convergence of both,
//               beta = (r~_i, r_i) / (r~_{i-1}, r_{i-1})
//   k_b4        p = r + beta p,  p~ = r~ + beta p~   (first line of the next iteration)
//
// st[0] carries the primary system's scalars (rho = (r~, r), alpha, beta,
// zeta_c in `xc`, its threshold), st[1] the dual's (zeta~_c, threshold,
// ||r~||^2).  Each kernel returns at once when st[0].done.

__global__ void k_bi_alpha(IterState* st, const double* __restrict__ dinv) {
  if (st[0].done) return;
  const int lane = threadIdx.x & 31;
  const int k = st[0].k;
  double alpha = 0.0;
  int ok = 0;
  if (lane == 0) {
    const double ptq = st[0].red[0];
    if (ptq == 0.0 || !isfinite(ptq)) {
      fail(&st[0], ptq == 0.0 ? RB_EBREAKDOWN_RHO : RB_ENONFINITE);
    } else {
      alpha = st[0].rho / ptq;
      st[0].alpha = alpha;
      ok = 1;
    }
  }
  ok = __shfl_sync(0xffffffffu, ok, 0);
  if (!ok) return;
  alpha = __shfl_sync(0xffffffffu, alpha, 0);
  for (int j = lane; j < k; j += 32) {
    st[0].xc[j] += alpha * st[0].gamma[j];
    st[1].xc[j] += alpha * (st[1].gamma[j] * dinv[j]);
  }
}

__device__ void finish_b3(IterState* st, const double* res) {
  if ((threadIdx.x & 31) != 0) return;
  IterState* s0 = &st[0];
  s0->iter += 1;
  const double rn2 = res[0], rtn2 = res[1], rho_new = res[2];
  s0->rnorm2 = rn2;
  st[1].rnorm2 = rtn2;
  st[1].iter = s0->iter;
  if (!isfinite(rn2) || !isfinite(rtn2) || !isfinite(rho_new)) {
    fail(s0, RB_ENONFINITE);
  } else if (rn2 <= s0->thresh2 && rtn2 <= st[1].thresh2) {
    s0->done = 1;
  } else if (rho_new == 0.0) {
    fail(s0, RB_EBREAKDOWN_RHO);
  } else {
    s0->beta = rho_new / s0->rho;
    s0->rho = rho_new;
    if (s0->iter >= s0->max_itn) fail(s0, RB_ENOTCONV);
  }
}

__global__ void __launch_bounds__(kBlock) k_b2(BiArgs a, const double* __restrict__ C,
                                               const double* __restrict__ Ct, int64_t ld,
                                               const double* __restrict__ dinv) {
  IterState* st = a.st;
  if (st[0].done) return;
  __shared__ double cz[2][kMaxK];   // -zeta and -D_c^{-1} C^T z~
  __shared__ ReduceSmem<1> sm;
  const int k = st[0].k;
  if (threadIdx.x < k) {
    cz[0][threadIdx.x] = -st[0].gamma[threadIdx.x];
    cz[1][threadIdx.x] = -(st[1].gamma[threadIdx.x] * dinv[threadIdx.x]);
  }
  __syncthreads();
  Acc<double> acc[1];
  for (int64_t i = gtid(); i < a.npad; i += gstride()) {
    double u = 0.0, ut = 0.0;
    for (int j = 0; j < k; ++j) {
      u = fma(C[j * ld + i], cz[0][j], u);
      ut = fma(Ct[j * ld + i], cz[1][j], ut);
    }
    const double q = a.q[i] + u;
    a.q[i] = q;
    a.qt[i] = a.qt[i] + ut;
    acc[0].add(a.pt[i], q);
  }
  if (block_reduce_last<double, 1>(acc, 1, sm, a.partials, &st[0].ticket[P2]) && threadIdx.x == 0)
    st[0].red[0] = sm.res[0];
}

__global__ void __launch_bounds__(kBlock) k_b3(BiArgs a) {
  IterState* st = a.st;
  if (st[0].done) return;
  __shared__ ReduceSmem<3> sm;
  const double alpha = st[0].alpha;
  Acc<double> acc[3];
  for (int64_t i = gtid(); i < a.npad; i += gstride()) {
    const double r = fma_t(-alpha, a.q[i], a.r[i]);
    const double rt = fma_t(-alpha, a.qt[i], a.rt[i]);
    a.x[i] = fma_t(alpha, a.p[i], a.x[i]);
    a.xt[i] = fma_t(alpha, a.pt[i], a.xt[i]);
    a.r[i] = r;
    a.rt[i] = rt;
    acc[0].add(r, r);
    acc[1].add(rt, rt);
    acc[2].add(rt, r);
  }
  if (block_reduce_last<double, 3>(acc, 3, sm, a.partials, &st[0].ticket[P3]) && threadIdx.x < 32)
    finish_b3(st, sm.res);
}

__global__ void __launch_bounds__(kBlock) k_b4(BiArgs a) {
  IterState* st = a.st;
  if (st[0].done) return;
  const double beta = st[0].beta;
  for (int64_t i = gtid(); i < a.npad; i += gstride()) {
    a.p[i] = fma_t(beta, a.p[i], a.r[i]);
    a.pt[i] = fma_t(beta, a.pt[i], a.rt[i]);
  }
}

cudaError_t bicg_alpha(IterState* st, const double* dinv, cudaStream_t s) {
  count_launches(1);
  k_bi_alpha<<<1, 32, 0, s>>>(st, dinv);
  return cudaGetLastError();
}

cudaError_t bicg_project(const BiArgs& a, const double* C, const double* Ct, int64_t ld, const double* dinv,
                         int grid, cudaStream_t s) {
  count_launches(1);
  k_b2<<<grid, kBlock, 0, s>>>(a, C, Ct, ld, dinv);
  return cudaGetLastError();
}

cudaError_t bicg_update(const BiArgs& a, int grid, cudaStream_t s) {
  count_launches(2);
  k_b3<<<grid, kBlock, 0, s>>>(a);
  k_b4<<<grid, kBlock, 0, s>>>(a);
  return cudaGetLastError();
}

int bicg_grid(int nsm, int64_t npad) {
  const int64_t work = (npad + kBlock - 1) / kBlock;
  const int o = std::min(occ((const void*)k_b2, nsm), occ((const void*)k_b3, nsm));
  return (int)std::max<int64_t>(1, std::min<int64_t>(work, o));
}

}  // namespace rb
