// The fused passes of one RBiCGSTAB iteration (Alg. 2, step 6).
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
// T is the storage and SpMV type (double for RB_FP64, float for the inner
// solve of RB_MIXED); all dot products and projections accumulate in FP64.
#include <algorithm>
#include <cstdlib>
#include <type_traits>

#include "device.cuh"
#include "kernels.h"

namespace rb {

__device__ __forceinline__ void fail(IterState* st, int code) {
  st->status = code;
  st->done = 1;
}

// ---------------------------------------------------------------- scalar steps
__device__ void finish_p1(IterState* st, const double* res, int k) {
  double rtq = res[0];
  for (int j = 0; j < k; ++j) {
    st->zeta[j] = res[1 + j];
    rtq -= st->cr[j] * res[1 + j];
  }
  st->rtq = rtq;
  if (rtq == 0.0 || !isfinite(rtq)) {
    fail(st, rtq == 0.0 ? RB_EBREAKDOWN_RHO : RB_ENONFINITE);
    return;
  }
  st->alpha = st->rho / rtq;
}

__device__ void finish_p2(IterState* st, const double* res) {
  st->snorm2 = res[0];
  if (!isfinite(res[0])) fail(st, RB_ENONFINITE);
  else if (res[0] <= st->thresh2) st->half = 1;
}

__device__ void finish_p3(IterState* st, const double* res, int k) {
  for (int j = 0; j < k; ++j) st->gamma[j] = res[j];
}

__device__ void finish_p4(IterState* st, const double* res, int k) {
  const double s_t = res[0], t_t = res[1], rt_t = res[2], rt_s = res[3];
  st->st = s_t; st->tt = t_t; st->rtt = rt_t; st->rts = rt_s;
  if (t_t == 0.0 || !isfinite(t_t)) {
    fail(st, t_t == 0.0 ? RB_EBREAKDOWN_OMEGA : RB_ENONFINITE);
    return;
  }
  const double omega = s_t / t_t;
  if (omega == 0.0) {
    fail(st, RB_EBREAKDOWN_OMEGA);
    return;
  }
  const double rho_new = rt_s - omega * rt_t;
  st->beta = (rho_new / st->rho) * (st->alpha / omega);
  st->omega = omega;
  for (int j = 0; j < k; ++j) st->xc[j] += st->alpha * st->zeta[j] + omega * st->gamma[j];
  st->rho = rho_new;
}

__device__ void finish_p5(IterState* st, const double* res, int k) {
  st->iter += 1;
  if (st->half) {
    for (int j = 0; j < k; ++j) st->xc[j] += st->alpha * st->zeta[j];
    st->rnorm2 = st->snorm2;
    st->done = 1;
    return;
  }
  const double rn2 = res[0];
  st->rnorm2 = rn2;
  if (!isfinite(rn2)) fail(st, RB_ENONFINITE);
  else if (rn2 <= st->thresh2) st->done = 1;
  else if (st->rho == 0.0) fail(st, RB_EBREAKDOWN_RHO);
  else if (st->iter >= st->max_itn) fail(st, RB_ENOTCONV);
}

// ---------------------------------------------------------------- SpMV core
// Rows sl*32+lane of two slices at once (sl1 < 0: only the first), so each
// warp keeps two independent gather chains in flight.
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
// y = A v stored to `out`; acc[OFF + j] += Chat_j^T y (j < k); RTQ adds
// acc[0] += (r~0, y); DOTS (k = 0 only) accumulates
// [(s,t), (t,t), (r~0,t), (r~0,s)] with s = v, t = y.
template <typename T, int KMAX, bool RTQ, bool DOTS>
__device__ __forceinline__ void spmv_project(const IterArgs<T>& a, const T* __restrict__ v,
                                             T* __restrict__ out, Acc<T>* acc, int k) {
  const int lane = threadIdx.x & 31;
  const int64_t w0 = gtid() >> 5, nw = gstride() >> 5;
  constexpr int OFF = RTQ ? 1 : 0;
  const T* __restrict__ Chat = a.Chat;
  const T* __restrict__ rt0 = a.rt0;
  const int64_t ld = a.ld, ns = a.A.nslices;
  for (int64_t sl = w0; sl < ns; sl += 2 * nw) {
    const int64_t sl1 = (sl + nw < ns) ? sl + nw : -1;
    T y[2];
    sell_rows2<T>(a.A, sl, sl1, lane, v, y[0], y[1]);
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      if (h == 1 && sl1 < 0) break;
      const int64_t row = (h == 0 ? sl : sl1) * kSlice + lane;
      out[row] = y[h];
      const T yd = y[h];
      if (RTQ) acc[0].add(__ldg(rt0 + row), yd);
      if (DOTS) {
        const T sv = __ldg(v + row), rv = __ldg(rt0 + row);
        acc[0].add(sv, yd);
        acc[1].add(yd, yd);
        acc[2].add(rv, yd);
        acc[3].add(rv, sv);
      }
#pragma unroll
      for (int j = 0; j < KMAX; ++j)
        if (j < k) acc[OFF + j].add(__ldg(Chat + j * ld + row), yd);
    }
  }
}

// FP32 projection, column per lane (KMAX <= 32): after the SpMV of a slice,
// lane j accumulates sum over the slice's 32 rows of Chat[j*ld + row] * y[row]
// with Dot2: the column's 32 consecutive values arrive as eight 16-byte loads
// and y is broadcast by warp shuffles.  One accumulator per lane instead of k
// per thread keeps registers low and occupancy high.  RTQ adds (r~0, y) per
// row.  Warp sums land in sm.w[warp][*] (value 0 = (r~0, y) when RTQ).
template <int KMAX, bool RTQ>
__device__ __forceinline__ void spmv_project_f32(const IterArgs<float>& a, const float* __restrict__ v,
                                                 float* __restrict__ out, int k, ReduceSmem<KMAX + 1>& sm) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int64_t w0 = gtid() >> 5, nw = gstride() >> 5;
  const float* __restrict__ rt0 = a.rt0;
  const float* __restrict__ col = a.Chat + (int64_t)(lane < k ? lane : 0) * a.ld;
  const int64_t ns = a.A.nslices;
  Acc<float> accr, accc;
  for (int64_t sl = w0; sl < ns; sl += 2 * nw) {
    const int64_t sl1 = (sl + nw < ns) ? sl + nw : -1;
    float y[2];
    sell_rows2<float>(a.A, sl, sl1, lane, v, y[0], y[1]);
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      if (h == 1 && sl1 < 0) break;
      const int64_t base = (h == 0 ? sl : sl1) * kSlice;
      out[base + lane] = y[h];
      if (RTQ) accr.add(__ldg(rt0 + base + lane), y[h]);
      float4 cv[8];
      if (lane < k) {
        const float4* cp = reinterpret_cast<const float4*>(col + base);
#pragma unroll
        for (int u = 0; u < 8; ++u) cv[u] = __ldg(cp + u);
      }
#pragma unroll
      for (int u = 0; u < 8; ++u) {
        const float y0 = __shfl_sync(0xffffffffu, y[h], 4 * u);
        const float y1 = __shfl_sync(0xffffffffu, y[h], 4 * u + 1);
        const float y2 = __shfl_sync(0xffffffffu, y[h], 4 * u + 2);
        const float y3 = __shfl_sync(0xffffffffu, y[h], 4 * u + 3);
        if (lane < k) {
          accc.add(cv[u].x, y0);
          accc.add(cv[u].y, y1);
          accc.add(cv[u].z, y2);
          accc.add(cv[u].w, y3);
        }
      }
    }
  }
  constexpr int OFF = RTQ ? 1 : 0;
  if (RTQ) {
    Acc<float> r1[1] = {accr};
    float hi = r1[0].hi, lo = r1[0].lo;
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
    if (lane == 0) sm.w[warp][0] = (double)hi + (double)lo;
  }
  if (lane < k) sm.w[warp][OFF + lane] = accc.get();
}

template <typename T, int KMAX>
__global__ void __launch_bounds__(kBlock) k_p1(IterArgs<T> a) {
  IterState* st = a.st;
  if (st->done) return;
  constexpr int NV = KMAX + 1;
  __shared__ ReduceSmem<NV> sm;
  const int k = KMAX > 0 ? st->k : 0;
  bool last;
  if constexpr (std::is_same<T, float>::value && KMAX > 0 && KMAX <= 32) {
    spmv_project_f32<KMAX, true>(a, a.p_in, a.qraw, k, sm);
    last = grid_finish<NV>(1 + k, sm, a.partials, &st->ticket[P1]);
  } else {
    Acc<T> acc[NV];
    spmv_project<T, KMAX, true, false>(a, a.p_in, a.qraw, acc, k);
    last = block_reduce_last<T, NV>(acc, 1 + k, sm, a.partials, &st->ticket[P1]);
  }
  if (last && threadIdx.x == 0) finish_p1(st, sm.res, k);
}

template <typename T, int KMAX>
__global__ void __launch_bounds__(kBlock) k_p3(IterArgs<T> a) {
  IterState* st = a.st;
  if (st->done || st->half) return;
  constexpr bool DOTS = (KMAX == 0);
  constexpr int NV = DOTS ? 4 : KMAX;
  const int k = KMAX > 0 ? st->k : 0;
  bool last;
  if constexpr (std::is_same<T, float>::value && KMAX > 0 && KMAX <= 32) {
    __shared__ ReduceSmem<KMAX + 1> sm;
    spmv_project_f32<KMAX, false>(a, a.s, a.traw, k, sm);
    last = grid_finish<KMAX + 1>(k, sm, a.partials, &st->ticket[P3]);
    if (last && threadIdx.x == 0) finish_p3(st, sm.res, k);
  } else {
    __shared__ ReduceSmem<NV> sm;
    Acc<T> acc[NV];
    spmv_project<T, KMAX, false, DOTS>(a, a.s, a.traw, acc, k);
    last = block_reduce_last<T, NV>(acc, DOTS ? 4 : k, sm, a.partials, &st->ticket[P3]);
    if (last && threadIdx.x == 0) {
      if (DOTS) finish_p4(st, sm.res, 0);
      else finish_p3(st, sm.res, k);
    }
  }
}

// y_i - sum_j M[j*ld + i] c_j for two rows at once.  Loads are issued in
// batches of 8 columns (16 loads in flight per thread) before their FMAs.
template <typename T, int KMAX>
__device__ __forceinline__ void correct2(const T* __restrict__ M, int64_t ld, const T* c, int k,
                                         int64_t i0, int64_t i1, bool two, T& y0, T& y1) {
  constexpr int B = 8;
  T a0 = T(0), a1 = T(0);
#pragma unroll
  for (int j0 = 0; j0 < KMAX; j0 += B) {
    if (j0 < k) {
      T m0[B], m1[B];
#pragma unroll
      for (int u = 0; u < B; ++u) {
        const bool ok = (j0 + u < KMAX) && (j0 + u < k);
        m0[u] = ok ? __ldg(M + (j0 + u) * ld + i0) : T(0);
        m1[u] = (ok && two) ? __ldg(M + (j0 + u) * ld + i1) : T(0);
      }
#pragma unroll
      for (int u = 0; u < B; ++u) {
        if (j0 + u < KMAX) {
          const T cu = (j0 + u < k) ? c[j0 + u] : T(0);
          a0 = fma_t(m0[u], cu, a0);
          a1 = fma_t(m1[u], cu, a1);
        }
      }
    }
  }
  y0 -= a0;
  y1 -= a1;
}

// ---------------------------------------------------------------- P2
template <typename T, int KMAX>
__global__ void __launch_bounds__(kBlock) k_p2(IterArgs<T> a) {
  IterState* st = a.st;
  if (st->done) return;
  __shared__ ReduceSmem<1> sm;
  __shared__ T zs[KMAX > 0 ? KMAX : 1];
  const int k = KMAX > 0 ? st->k : 0;
  if (KMAX > 0 && threadIdx.x < k) zs[threadIdx.x] = (T)st->zeta[threadIdx.x];
  const T al = (T)st->alpha;
  __syncthreads();
  const T* __restrict__ qraw = a.qraw;
  const T* __restrict__ r = a.r;
  T* __restrict__ q = a.q;
  T* __restrict__ s = a.s;
  const int64_t npad = a.npad, stride = gstride();
  Acc<T> acc[1];
  for (int64_t i = gtid(); i < npad; i += 2 * stride) {
    const int64_t i1 = i + stride;
    const bool two = i1 < npad;
    T q0 = qraw[i], q1 = two ? qraw[i1] : T(0);
    const T r0 = r[i], r1 = two ? r[i1] : T(0);
    if (KMAX > 0) {
      correct2<T, KMAX>(a.C, a.ld, zs, k, i, i1, two, q0, q1);
      q[i] = q0;
      if (two) q[i1] = q1;
    }
    const T s0 = r0 - al * q0;
    s[i] = s0;
    acc[0].add(s0, s0);
    if (two) {
      const T s1 = r1 - al * q1;
      s[i1] = s1;
      acc[0].add(s1, s1);
    }
  }
  if (block_reduce_last<T, 1>(acc, 1, sm, a.partials, &st->ticket[P2]) && threadIdx.x == 0)
    finish_p2(st, sm.res);
}

// ---------------------------------------------------------------- P4 (k > 0)
template <typename T, int KMAX>
__global__ void __launch_bounds__(kBlock) k_p4(IterArgs<T> a) {
  IterState* st = a.st;
  if (st->done || st->half) return;
  __shared__ ReduceSmem<4> sm;
  __shared__ T gs[KMAX];
  const int k = st->k;
  if (threadIdx.x < k) gs[threadIdx.x] = (T)st->gamma[threadIdx.x];
  __syncthreads();
  const T* __restrict__ traw = a.traw;
  const T* __restrict__ s = a.s;
  const T* __restrict__ rt0 = a.rt0;
  T* __restrict__ t = a.t;
  const int64_t npad = a.npad, stride = gstride();
  Acc<T> acc[4];
  for (int64_t i = gtid(); i < npad; i += 2 * stride) {
    const int64_t i1 = i + stride;
    const bool two = i1 < npad;
    T t0 = traw[i], t1 = two ? traw[i1] : T(0);
    const T s0 = s[i], s1 = two ? s[i1] : T(0);
    const T r0 = __ldg(rt0 + i), r1 = two ? __ldg(rt0 + i1) : T(0);
    correct2<T, KMAX>(a.C, a.ld, gs, k, i, i1, two, t0, t1);
    t[i] = t0;
    if (two) t[i1] = t1;
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      if (h == 1 && !two) break;
      const T td = h ? t1 : t0, sv = h ? s1 : s0, rv = h ? r1 : r0;
      acc[0].add(sv, td);
      acc[1].add(td, td);
      acc[2].add(rv, td);
      acc[3].add(rv, sv);
    }
  }
  if (block_reduce_last<T, 4>(acc, 4, sm, a.partials, &st->ticket[P4]) && threadIdx.x == 0)
    finish_p4(st, sm.res, k);
}

// ---------------------------------------------------------------- P5
template <typename T, int KMAX>
__global__ void __launch_bounds__(kBlock) k_p5(IterArgs<T> a) {
  IterState* st = a.st;
  if (st->done) return;
  __shared__ ReduceSmem<1> sm;
  const int k = KMAX > 0 ? st->k : 0;
  Acc<T> acc[1];
  T* __restrict__ x = a.x;
  T* __restrict__ r = a.r;
  const T* __restrict__ p = a.p_in;
  const T* __restrict__ s = a.s;
  const int64_t npad = a.npad, stride = gstride();
  if (st->half) {
    const T al = (T)st->alpha;
    for (int64_t i = gtid(); i < npad; i += stride) {
      x[i] = fma_t(al, p[i], x[i]);
      r[i] = s[i];
    }
  } else {
    const T al = (T)st->alpha, om = (T)st->omega, be = (T)st->beta;
    const T* __restrict__ t = a.t;
    const T* __restrict__ q = a.q;
    T* __restrict__ po = a.p_out;
    for (int64_t i = gtid(); i < npad; i += 2 * stride) {
      const int64_t i1 = i + stride;
      const bool two = i1 < npad;
      const T p0 = p[i], s0 = s[i], t0 = t[i], q0 = q[i], x0 = x[i];
      T p1 = T(0), s1 = T(0), t1 = T(0), q1 = T(0), x1 = T(0);
      if (two) {
        p1 = p[i1]; s1 = s[i1]; t1 = t[i1]; q1 = q[i1]; x1 = x[i1];
      }
      const T r0 = s0 - om * t0;
      x[i] = fma_t(om, s0, fma_t(al, p0, x0));
      r[i] = r0;
      po[i] = fma_t(be, p0 - om * q0, r0);
      acc[0].add(r0, r0);
      if (two) {
        const T r1 = s1 - om * t1;
        x[i1] = fma_t(om, s1, fma_t(al, p1, x1));
        r[i1] = r1;
        po[i1] = fma_t(be, p1 - om * q1, r1);
        acc[0].add(r1, r1);
      }
    }
  }
  if (block_reduce_last<T, 1>(acc, 1, sm, a.partials, &st->ticket[P5]) && threadIdx.x == 0)
    finish_p5(st, sm.res, k);
}

// ---------------------------------------------------------------- launchers
template <typename T, int KMAX>
static cudaError_t launch_iter_k(const IterArgs<T>& a, const Grids& g, cudaStream_t s) {
  k_p1<T, KMAX><<<g.pass[P1], kBlock, 0, s>>>(a);
  k_p2<T, KMAX><<<g.pass[P2], kBlock, 0, s>>>(a);
  k_p3<T, KMAX><<<g.pass[P3], kBlock, 0, s>>>(a);
  if (KMAX > 0) k_p4<T, (KMAX > 0 ? KMAX : 1)><<<g.pass[P4], kBlock, 0, s>>>(a);
  k_p5<T, KMAX><<<g.pass[P5], kBlock, 0, s>>>(a);
  return cudaGetLastError();
}

template <typename T, int KMAX>
static cudaError_t launch_pass_k(int pass, const IterArgs<T>& a, const Grids& g, cudaStream_t s) {
  switch (pass) {
    case P1: k_p1<T, KMAX><<<g.pass[P1], kBlock, 0, s>>>(a); break;
    case P2: k_p2<T, KMAX><<<g.pass[P2], kBlock, 0, s>>>(a); break;
    case P3: k_p3<T, KMAX><<<g.pass[P3], kBlock, 0, s>>>(a); break;
    case P4: if (KMAX > 0) k_p4<T, (KMAX > 0 ? KMAX : 1)><<<g.pass[P4], kBlock, 0, s>>>(a); break;
    default: k_p5<T, KMAX><<<g.pass[P5], kBlock, 0, s>>>(a); break;
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

template <typename T>
cudaError_t launch_iteration(const IterArgs<T>& a, int k, const Grids& g, cudaStream_t s) {
  switch (kmax_bucket(k)) {
    case 0: return launch_iter_k<T, 0>(a, g, s);
    case 8: return launch_iter_k<T, 8>(a, g, s);
    case 16: return launch_iter_k<T, 16>(a, g, s);
    case 24: return launch_iter_k<T, 24>(a, g, s);
    case 32: return launch_iter_k<T, 32>(a, g, s);
    case 48: return launch_iter_k<T, 48>(a, g, s);
    default: return launch_iter_k<T, 64>(a, g, s);
  }
}

template <typename T>
cudaError_t launch_pass(int pass, const IterArgs<T>& a, int k, const Grids& g, cudaStream_t s) {
  count_launches(1);
  switch (kmax_bucket(k)) {
    case 0: return launch_pass_k<T, 0>(pass, a, g, s);
    case 8: return launch_pass_k<T, 8>(pass, a, g, s);
    case 16: return launch_pass_k<T, 16>(pass, a, g, s);
    case 24: return launch_pass_k<T, 24>(pass, a, g, s);
    case 32: return launch_pass_k<T, 32>(pass, a, g, s);
    case 48: return launch_pass_k<T, 48>(pass, a, g, s);
    default: return launch_pass_k<T, 64>(pass, a, g, s);
  }
}

template cudaError_t launch_pass<double>(int, const IterArgs<double>&, int, const Grids&, cudaStream_t);
template cudaError_t launch_pass<float>(int, const IterArgs<float>&, int, const Grids&, cudaStream_t);
template cudaError_t launch_iteration<double>(const IterArgs<double>&, int, const Grids&, cudaStream_t);
template cudaError_t launch_iteration<float>(const IterArgs<float>&, int, const Grids&, cudaStream_t);

// Grid sizes: one full wave of resident blocks per kernel configuration (a
// second partial wave would leave SMs idle at the end of every pass), capped
// by the work.
template <typename T>
static int occ(const void* f, int nsm) {
  int b = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, f, kBlock, 0);
  return (b > 0 ? b : 1) * nsm;
}

template <typename T, int KMAX>
static void grids_k(int nsm, int64_t npad, Grids* g) {
  const int64_t work = (npad + kBlock - 1) / kBlock;
  const int o[5] = {occ<T>((const void*)k_p1<T, KMAX>, nsm), occ<T>((const void*)k_p2<T, KMAX>, nsm),
                    occ<T>((const void*)k_p3<T, KMAX>, nsm),
                    occ<T>((const void*)k_p4<T, (KMAX > 0 ? KMAX : 1)>, nsm),
                    occ<T>((const void*)k_p5<T, KMAX>, nsm)};
  for (int p = 0; p < 5; ++p) g->pass[p] = (int)std::max<int64_t>(1, std::min<int64_t>(work, o[p]));
  g->spmv = std::max(g->pass[P1], g->pass[P3]);
  g->vec = std::max(g->pass[P2], g->pass[P5]);
}

template <typename T>
void iteration_grids(int k, int nsm, int64_t npad, Grids* g) {
  switch (kmax_bucket(k)) {
    case 0: grids_k<T, 0>(nsm, npad, g); break;
    case 8: grids_k<T, 8>(nsm, npad, g); break;
    case 16: grids_k<T, 16>(nsm, npad, g); break;
    case 24: grids_k<T, 24>(nsm, npad, g); break;
    case 32: grids_k<T, 32>(nsm, npad, g); break;
    case 48: grids_k<T, 48>(nsm, npad, g); break;
    default: grids_k<T, 64>(nsm, npad, g); break;
  }
}

template void iteration_grids<double>(int, int, int64_t, Grids*);
template void iteration_grids<float>(int, int, int64_t, Grids*);

}  // namespace rb
