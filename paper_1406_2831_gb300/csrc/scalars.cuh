// Scalar steps of one RBiCGSTAB iteration (Alg. 2), shared by the fused
// passes of one system or a block (iter.cu) and the batched passes over many
// systems (batch.cu).  Each runs in one warp once a pass's reduction is
// complete; `res` holds the reduced values of the pass.
#pragma once

#include "device.cuh"

namespace rb {

__device__ __forceinline__ void fail(IterState* st, int code) {
  st->status = code;
  st->done = 1;
}

// ---------------------------------------------------------------- scalar steps
// Each step runs in one warp of the last block, one warp per right-hand side.
// The per-column loads and stores of IterState (zeta, gamma, c_r, x_c) are
// spread over the lanes so that their memory latencies overlap instead of
// adding up; recurrences over the columns stay in lane 0, in column order.
// scr is warp-private shared scratch of at least k doubles.
static __device__ void finish_p1(IterState* st, const double* res, int k, double* scr) {
  const int lane = threadIdx.x & 31;
  for (int j = lane; j < k; j += 32) {
    st->zeta[j] = res[1 + j];
    scr[j] = st->cr[j];
  }
  __syncwarp();
  if (lane != 0) return;
  double rtq = res[0];
  for (int j = 0; j < k; ++j) rtq -= scr[j] * res[1 + j];
  st->rtq = rtq;
  if (rtq == 0.0 || !isfinite(rtq)) {
    fail(st, rtq == 0.0 ? RB_EBREAKDOWN_RHO : RB_ENONFINITE);
    return;
  }
  st->alpha = st->rho / rtq;
}

static __device__ void finish_p2(IterState* st, const double* res) {
  if ((threadIdx.x & 31) != 0) return;
  st->snorm2 = res[0];
  if (!isfinite(res[0])) fail(st, RB_ENONFINITE);
  else if (res[0] <= st->thresh2) st->half = 1;
}

static __device__ void finish_p3(IterState* st, const double* res, int k) {
  for (int j = threadIdx.x & 31; j < k; j += 32) st->gamma[j] = res[j];
}

static __device__ void finish_p4(IterState* st, const double* res, int k) {
  const int lane = threadIdx.x & 31;
  double omega = 0.0, alpha = 0.0;
  int ok = 0;
  if (lane == 0) {
    const double s_t = res[0], t_t = res[1], rt_t = res[2], rt_s = res[3];
    st->st = s_t; st->tt = t_t; st->rtt = rt_t; st->rts = rt_s;
    if (t_t == 0.0 || !isfinite(t_t)) {
      fail(st, t_t == 0.0 ? RB_EBREAKDOWN_OMEGA : RB_ENONFINITE);
    } else {
      omega = s_t / t_t;
      if (omega == 0.0) {
        fail(st, RB_EBREAKDOWN_OMEGA);
      } else {
        alpha = st->alpha;
        const double rho_new = rt_s - omega * rt_t;
        st->beta = (rho_new / st->rho) * (alpha / omega);
        st->omega = omega;
        st->rho = rho_new;
        ok = 1;
      }
    }
  }
  ok = __shfl_sync(0xffffffffu, ok, 0);
  if (!ok) return;
  omega = __shfl_sync(0xffffffffu, omega, 0);
  alpha = __shfl_sync(0xffffffffu, alpha, 0);
  for (int j = lane; j < k; j += 32) st->xc[j] += alpha * st->zeta[j] + omega * st->gamma[j];
}

static __device__ void finish_p5(IterState* st, const double* res, int k) {
  const int lane = threadIdx.x & 31;
  if (st->half) {   // set by an earlier pass; the same in every lane
    const double alpha = st->alpha;
    for (int j = lane; j < k; j += 32) st->xc[j] += alpha * st->zeta[j];
    if (lane == 0) {
      st->iter += 1;
      st->rnorm2 = st->snorm2;
      st->rmax2 = fmax(st->rmax2, st->snorm2);
      st->done = 1;
    }
    return;
  }
  if (lane != 0) return;
  st->iter += 1;
  const double rn2 = res[0];
  st->rnorm2 = rn2;
  st->rmax2 = fmax(st->rmax2, rn2);   // fmax ignores a NaN: the finiteness test below catches it
  if (!isfinite(rn2)) fail(st, RB_ENONFINITE);
  else if (rn2 <= st->thresh2) st->done = 1;
  else if (st->rho == 0.0) fail(st, RB_EBREAKDOWN_RHO);
  else if (st->iter >= st->max_itn) fail(st, RB_ENOTCONV);
}

}  // namespace rb
