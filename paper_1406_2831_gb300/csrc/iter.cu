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
template <typename T>
__device__ __forceinline__ T sell_row(const Sell<T>& A, int64_t sl, int lane, const T* __restrict__ v) {
  const int w = __ldg(A.width + sl);
  const int64_t base = __ldg(A.slice_ptr + sl) + lane;
  T y = T(0);
#pragma unroll 4
  for (int j = 0; j < w; ++j) {
    const int64_t e = base + (int64_t)j * kSlice;
    y = fma(__ldg(A.val + e), __ldg(v + __ldg(A.col + e)), y);
  }
  return y;
}

// ---------------------------------------------------------------- P1 / P3
// y = A v stored to `out`; acc[0..k) += Chat^T y; with DOTS (k = 0 only)
// acc = [(s,t), (t,t), (r~0,t), (r~0,s)] where s = v, t = y.
template <typename T, int KMAX, bool RTQ, bool DOTS>
__device__ __forceinline__ void spmv_project(const IterArgs<T>& a, const T* __restrict__ v,
                                             T* __restrict__ out, double* acc, int k) {
  const int lane = threadIdx.x & 31;
  const int64_t w0 = gtid() >> 5, nw = gstride() >> 5;
  constexpr int OFF = RTQ ? 1 : 0;
  for (int64_t sl = w0; sl < a.A.nslices; sl += nw) {
    const int64_t row = sl * kSlice + lane;
    const T y = sell_row<T>(a.A, sl, lane, v);
    out[row] = y;
    const double yd = (double)y;
    if (RTQ) acc[0] = fma((double)__ldg(a.rt0 + row), yd, acc[0]);
    if (DOTS) {
      const double sv = (double)__ldg(v + row), rv = (double)__ldg(a.rt0 + row);
      acc[0] = fma(sv, yd, acc[0]);
      acc[1] = fma(yd, yd, acc[1]);
      acc[2] = fma(rv, yd, acc[2]);
      acc[3] = fma(rv, sv, acc[3]);
    }
#pragma unroll
    for (int j = 0; j < KMAX; ++j)
      if (j < k) acc[OFF + j] = fma((double)__ldg(a.Chat + j * a.ld + row), yd, acc[OFF + j]);
  }
}

template <typename T, int KMAX>
__global__ void __launch_bounds__(kBlock) k_p1(IterArgs<T> a) {
  IterState* st = a.st;
  if (st->done) return;
  constexpr int NV = KMAX + 1;
  __shared__ ReduceSmem<NV> sm;
  const int k = KMAX > 0 ? st->k : 0;
  double acc[NV];
#pragma unroll
  for (int v = 0; v < NV; ++v) acc[v] = 0.0;
  spmv_project<T, KMAX, true, false>(a, a.p_in, a.qraw, acc, k);
  if (block_reduce_last<NV>(acc, 1 + k, sm, a.partials, &st->ticket[P1]) && threadIdx.x == 0)
    finish_p1(st, sm.res, k);
}

template <typename T, int KMAX>
__global__ void __launch_bounds__(kBlock) k_p3(IterArgs<T> a) {
  IterState* st = a.st;
  if (st->done || st->half) return;
  constexpr bool DOTS = (KMAX == 0);
  constexpr int NV = DOTS ? 4 : KMAX;
  __shared__ ReduceSmem<NV> sm;
  const int k = KMAX > 0 ? st->k : 0;
  double acc[NV];
#pragma unroll
  for (int v = 0; v < NV; ++v) acc[v] = 0.0;
  spmv_project<T, KMAX, false, DOTS>(a, a.s, a.traw, acc, k);
  if (block_reduce_last<NV>(acc, DOTS ? 4 : k, sm, a.partials, &st->ticket[P3]) && threadIdx.x == 0) {
    if (DOTS) finish_p4(st, sm.res, 0);
    else finish_p3(st, sm.res, k);
  }
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
  double acc[1] = {0.0};
  for (int64_t i = gtid(); i < a.npad; i += gstride()) {
    T qv = a.qraw[i];
    if (KMAX > 0) {
      T corr = T(0);
#pragma unroll
      for (int j = 0; j < KMAX; ++j)
        if (j < k) corr = fma(__ldg(a.C + j * a.ld + i), zs[j], corr);
      qv -= corr;
      a.q[i] = qv;
    }
    const T sv = a.r[i] - al * qv;
    a.s[i] = sv;
    acc[0] = fma((double)sv, (double)sv, acc[0]);
  }
  if (block_reduce_last<1>(acc, 1, sm, a.partials, &st->ticket[P2]) && threadIdx.x == 0)
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
  double acc[4] = {0.0, 0.0, 0.0, 0.0};
  for (int64_t i = gtid(); i < a.npad; i += gstride()) {
    T corr = T(0);
#pragma unroll
    for (int j = 0; j < KMAX; ++j)
      if (j < k) corr = fma(__ldg(a.C + j * a.ld + i), gs[j], corr);
    const T tv = a.traw[i] - corr;
    a.t[i] = tv;
    const double td = (double)tv, sv = (double)a.s[i], rv = (double)__ldg(a.rt0 + i);
    acc[0] = fma(sv, td, acc[0]);
    acc[1] = fma(td, td, acc[1]);
    acc[2] = fma(rv, td, acc[2]);
    acc[3] = fma(rv, sv, acc[3]);
  }
  if (block_reduce_last<4>(acc, 4, sm, a.partials, &st->ticket[P4]) && threadIdx.x == 0)
    finish_p4(st, sm.res, k);
}

// ---------------------------------------------------------------- P5
template <typename T, int KMAX>
__global__ void __launch_bounds__(kBlock) k_p5(IterArgs<T> a) {
  IterState* st = a.st;
  if (st->done) return;
  __shared__ ReduceSmem<1> sm;
  const int k = KMAX > 0 ? st->k : 0;
  double acc[1] = {0.0};
  if (st->half) {
    const T al = (T)st->alpha;
    for (int64_t i = gtid(); i < a.npad; i += gstride()) {
      a.x[i] = fma(al, a.p_in[i], a.x[i]);
      a.r[i] = a.s[i];
    }
  } else {
    const T al = (T)st->alpha, om = (T)st->omega, be = (T)st->beta;
    for (int64_t i = gtid(); i < a.npad; i += gstride()) {
      const T pv = a.p_in[i], sv = a.s[i], tv = a.t[i], qv = a.q[i];
      a.x[i] = fma(om, sv, fma(al, pv, a.x[i]));
      const T rv = sv - om * tv;
      a.r[i] = rv;
      a.p_out[i] = fma(be, pv - om * qv, rv);
      acc[0] = fma((double)rv, (double)rv, acc[0]);
    }
  }
  if (block_reduce_last<1>(acc, 1, sm, a.partials, &st->ticket[P5]) && threadIdx.x == 0)
    finish_p5(st, sm.res, k);
}

// ---------------------------------------------------------------- launchers
template <typename T, int KMAX>
static cudaError_t launch_iter_k(const IterArgs<T>& a, const Grids& g, cudaStream_t s) {
  k_p1<T, KMAX><<<g.spmv, kBlock, 0, s>>>(a);
  k_p2<T, KMAX><<<g.vec, kBlock, 0, s>>>(a);
  k_p3<T, KMAX><<<g.spmv, kBlock, 0, s>>>(a);
  if (KMAX > 0) k_p4<T, (KMAX > 0 ? KMAX : 1)><<<g.vec, kBlock, 0, s>>>(a);
  k_p5<T, KMAX><<<g.vec, kBlock, 0, s>>>(a);
  return cudaGetLastError();
}

template <typename T, int KMAX>
static cudaError_t launch_pass_k(int pass, const IterArgs<T>& a, const Grids& g, cudaStream_t s) {
  switch (pass) {
    case P1: k_p1<T, KMAX><<<g.spmv, kBlock, 0, s>>>(a); break;
    case P2: k_p2<T, KMAX><<<g.vec, kBlock, 0, s>>>(a); break;
    case P3: k_p3<T, KMAX><<<g.spmv, kBlock, 0, s>>>(a); break;
    case P4: if (KMAX > 0) k_p4<T, (KMAX > 0 ? KMAX : 1)><<<g.vec, kBlock, 0, s>>>(a); break;
    default: k_p5<T, KMAX><<<g.vec, kBlock, 0, s>>>(a); break;
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

// Occupancy-derived grid sizes (blocks resident on all SMs at once).
template <typename T>
static int occ(const void* f, int nsm) {
  int b = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, f, kBlock, 0);
  return (b > 0 ? b : 1) * nsm;
}

template <typename T>
void iteration_grids(int k, int nsm, int64_t npad, Grids* g) {
  const int kb = kmax_bucket(k);
  const void* f1;
  const void* f2;
  switch (kb) {
    case 0: f1 = (const void*)k_p1<T, 0>; f2 = (const void*)k_p5<T, 0>; break;
    case 8: f1 = (const void*)k_p1<T, 8>; f2 = (const void*)k_p2<T, 8>; break;
    case 16: f1 = (const void*)k_p1<T, 16>; f2 = (const void*)k_p2<T, 16>; break;
    case 24: f1 = (const void*)k_p1<T, 24>; f2 = (const void*)k_p2<T, 24>; break;
    case 32: f1 = (const void*)k_p1<T, 32>; f2 = (const void*)k_p2<T, 32>; break;
    case 48: f1 = (const void*)k_p1<T, 48>; f2 = (const void*)k_p2<T, 48>; break;
    default: f1 = (const void*)k_p1<T, 64>; f2 = (const void*)k_p2<T, 64>; break;
  }
  const int64_t work_blocks = (npad + kBlock - 1) / kBlock;
  int gs = occ<T>(f1, nsm), gv = occ<T>(f2, nsm);
  g->spmv = (int)(work_blocks < gs ? work_blocks : gs);
  g->vec = (int)(work_blocks < gv ? work_blocks : gv);
  if (g->spmv < 1) g->spmv = 1;
  if (g->vec < 1) g->vec = 1;
}

template void iteration_grids<double>(int, int, int64_t, Grids*);
template void iteration_grids<float>(int, int, int64_t, Grids*);

}  // namespace rb
