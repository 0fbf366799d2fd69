// Orchestrator and C ABI of librbicgstab (see include/rbicgstab.h).
//
// A solve (Alg. 2) runs as: setup of x_0, r_0, r~_0 (eq. (3.5)) with a few
// generic kernels; then the fused five-pass iteration, captured once per
// handle as a CUDA graph of `poll` iterations and replayed until the device
// convergence flag is set (every pass returns at once after it is set, so
// the overshoot of the last replay costs only empty launches); then step 8
// (x = x - U x_c) and a true-residual check.  In the recycle-update modes the
// graph spans one cycle of s iterations whose p, s, A p, A s vectors land in
// a cycle store; between cycles the Gram matrices G = Z^T Z, H = Z^T W are
// formed on the device, the small harmonic-Ritz problem is solved on the
// host, and the candidate space Y, A Y is rebuilt on the device (Sec. 6.2).
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <vector>

#include "device.cuh"
#include "hostla.h"
#include "kernels.h"

using namespace rb;

#include <atomic>
static std::atomic<long long> g_launches{0};
void rb::count_launches(long long n) { g_launches.fetch_add(n, std::memory_order_relaxed); }

namespace {

// Rank thresholds.  FP64 solves: biorthogonalisation drops sigma_j < 1e-12
// sigma_1; the harmonic-Ritz pencil keeps eigenvalues > 1e-10 max of the
// scaled Z^T Z.  The mixed path iterates with FP32 copies of C, C-hat and
// builds the update from FP32 Krylov vectors (relative accuracy ~1e-7), so
// both thresholds are raised to 1e-6: a projector whose C-hat^T C
// conditioning exceeds 1e6 is not representable in FP32, and directions of W
// below that level are rounding noise.
constexpr double kSvdDrop = 1e-12;
constexpr double kRankTol = 1e-10;
constexpr double kSvdDropF32 = 1e-6;
constexpr double kRankTolF32 = 1e-6;
constexpr int kMaxGram = 90;         // k + 2 s must not exceed this

template <typename T>
T* dalloc(int64_t count, int* err) {
  void* p = nullptr;
  if (count <= 0) count = 1;
  cudaError_t e = cudaMalloc(&p, sizeof(T) * (size_t)count);
  if (e != cudaSuccess) {
    *err = (e == cudaErrorMemoryAllocation) ? RB_ENOMEM : RB_ECUDA;
    return nullptr;
  }
  return (T*)p;
}

struct GraphSlot {
  cudaGraphExec_t exec = nullptr;
  bool valid = false;
};

}  // namespace

struct rb_ctx {
  rb_opts o{};
  cudaStream_t us = nullptr;   // caller's stream
  cudaStream_t cs = nullptr;   // private stream used for graph capture
  int dev = 0, nsm = 0;
  // matrix
  int64_t n = 0, nnz = 0, npad = 0;
  int32_t *rp = nullptr, *ci = nullptr;
  double* cv = nullptr;
  int32_t *trp = nullptr, *tci = nullptr;
  int64_t* tsrc = nullptr;
  double* tcv = nullptr;
  SellBuf<double> A, AT;
  SellBuf<float> A32;
  bool have_matrix = false;
  int matrix_epoch = 0, update_epoch = -1;
  // recycle space (column-major, leading dimension npad), k_used columns
  int k = 0, kcap = 0;
  double *U = nullptr, *Ut = nullptr, *C = nullptr, *Ct = nullptr, *Chat = nullptr;
  double *T1 = nullptr, *T2 = nullptr;   // scratch blocks (kcap columns each)
  double* Dinv = nullptr;                // 1 / D_c (device)
  // vectors
  double *b = nullptr, *x = nullptr, *r = nullptr, *p = nullptr, *s = nullptr, *q = nullptr,
         *t = nullptr, *qraw = nullptr, *traw = nullptr, *rt0 = nullptr, *tmp = nullptr,
         *rin = nullptr, *xin = nullptr;
  // mixed path (FP32 inner solve)
  float *fx = nullptr, *fr = nullptr, *fp = nullptr, *fs = nullptr, *fq = nullptr, *ft = nullptr,
        *fqraw = nullptr, *ftraw = nullptr, *frt0 = nullptr, *fU = nullptr, *fC = nullptr,
        *fChat = nullptr;
  // device state
  IterState* st = nullptr;
  IterState* hst = nullptr;     // pinned host mirror
  double* partials = nullptr;
  int64_t partials_cap = 0;
  int* dflag = nullptr;
  // cycle store for the recycle update
  int cyc = 0;
  // P: 2*cyc, S: cyc, QR: cyc, TR: cyc vectors of the inner precision
  // (double for RB_FP64, float for RB_MIXED), and the candidate Y, A Y
  void* cstore = nullptr;
  void *Yc = nullptr, *AYc = nullptr, *Yn = nullptr, *AYn = nullptr;
  int kY = 0;
  double* gwork = nullptr;
  int64_t gwork_cap = 0;
  double *dG = nullptr, *dH = nullptr, *dR = nullptr;
  const double** dptr = nullptr;   // device pointer lists (4 * 128)
  Grids grids{1, 1};
  GraphSlot g_plain, g_cycle[2];
  int g_k = -1;
};

// ============================================================ helpers
namespace {

// Optional phase timing of the recycle update (RB_TIMING=1 prints to stderr).
struct PhaseClock {
  bool on = getenv("RB_TIMING") != nullptr;
  std::chrono::steady_clock::time_point t = std::chrono::steady_clock::now();
  void lap(const char* what) {
    if (!on) return;
    const auto now = std::chrono::steady_clock::now();
    fprintf(stderr, "rb_timing %-14s %8.3f ms\n", what, std::chrono::duration<double, std::milli>(now - t).count());
    t = now;
  }
};

int sync(rb_ctx* h) {
  RB_CUDA_TRY(cudaStreamSynchronize(h->us));
  return RB_OK;
}

void reset_graphs(rb_ctx* h) {
  for (GraphSlot* g : {&h->g_plain, &h->g_cycle[0], &h->g_cycle[1]}) {
    if (g->exec) cudaGraphExecDestroy(g->exec);
    g->exec = nullptr;
    g->valid = false;
  }
  h->g_k = -1;
}

int64_t round_up(int64_t v, int64_t m) { return (v + m - 1) / m * m; }

double* colp(double* base, int64_t ld, int j) { return base + (int64_t)j * ld; }

int copy_in(void* dst, const void* src, size_t bytes, int where, cudaStream_t s) {
  if (bytes == 0) return RB_OK;
  RB_CUDA_TRY(cudaMemcpyAsync(dst, src, bytes,
                              where == RB_DEVICE ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, s));
  return RB_OK;
}

int copy_out(void* dst, const void* src, size_t bytes, int where, cudaStream_t s) {
  if (bytes == 0) return RB_OK;
  RB_CUDA_TRY(cudaMemcpyAsync(dst, src, bytes,
                              where == RB_DEVICE ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, s));
  return RB_OK;
}

int read_state(rb_ctx* h) {
  RB_CUDA_TRY(cudaMemcpyAsync(h->hst, h->st, sizeof(IterState), cudaMemcpyDeviceToHost, h->us));
  return sync(h);
}

int vec_grid(rb_ctx* h) { return h->grids.vec; }

// Deterministic dot products / projections into st->red, then read back `cnt` values.
int run_dots(rb_ctx* h, const DotArgs& d, double* out, int cnt) {
  RB_CUDA_TRY(dots(d, h->npad, h->st, h->partials, vec_grid(h), h->us));
  if (out) {
    RB_CUDA_TRY(cudaMemcpyAsync(h->hst->red, h->st->red, sizeof(double) * cnt,
                                cudaMemcpyDeviceToHost, h->us));
    int rc = sync(h);
    if (rc) return rc;
    std::memcpy(out, h->hst->red, sizeof(double) * cnt);
  }
  return RB_OK;
}

int ensure_partials(rb_ctx* h) {
  // every kernel runs at most one full wave: <= 8 blocks of 256 threads per SM
  const int64_t need = (int64_t)std::max(8 * h->nsm, std::max(h->grids.spmv, h->grids.vec)) * kMaxNV;
  if (need <= h->partials_cap) return RB_OK;
  cudaFree(h->partials);
  int err = 0;
  h->partials = dalloc<double>(need, &err);
  if (!h->partials) return err;
  h->partials_cap = need;
  return RB_OK;
}

// Column pointer lists for gram / gemm_cols.
template <typename P>
int upload_ptrs(rb_ctx* h, int slot, const std::vector<P>& v) {
  RB_CUDA_TRY(cudaMemcpy(h->dptr + slot * 128, v.data(), sizeof(double*) * v.size(),
                         cudaMemcpyHostToDevice));
  return RB_OK;
}

// Out = X R (column lists) with R (m x kc column-major) given on the host.
template <typename T>
int block_gemm(rb_ctx* h, const std::vector<T*>& out, const std::vector<const T*>& X,
               const std::vector<double>& R, int kc) {
  const int m = (int)X.size();
  if (kc == 0 || m == 0) return RB_OK;
  int rc = sync(h);   // pointer lists and R are staged synchronously
  if (rc) return rc;
  rc = upload_ptrs(h, 0, X);
  if (rc) return rc;
  rc = upload_ptrs(h, 1, out);
  if (rc) return rc;
  RB_CUDA_TRY(cudaMemcpy(h->dR, R.data(), sizeof(double) * (size_t)m * kc, cudaMemcpyHostToDevice));
  RB_CUDA_TRY(gemm_cols<T>((T* const*)(h->dptr + 128), (const T* const*)h->dptr, m, h->dR, kc,
                           h->npad, vec_grid(h), h->us));
  return RB_OK;
}

// G (mx x my, column-major) = X^T Y, returned on the host.
template <typename T>
int block_gram(rb_ctx* h, const std::vector<const T*>& X, const std::vector<const T*>& Y,
               std::vector<double>& G) {
  const int mx = (int)X.size(), my = (int)Y.size();
  G.assign((size_t)mx * my, 0.0);
  if (!mx || !my) return RB_OK;
  int rc = sync(h);
  if (rc) return rc;
  rc = upload_ptrs(h, 2, X);
  if (rc) return rc;
  rc = upload_ptrs(h, 3, Y);
  if (rc) return rc;
  const int grid = vec_grid(h);
  const int64_t need = (int64_t)grid * mx * my;
  if (need > h->gwork_cap) {
    cudaFree(h->gwork);
    int err = 0;
    h->gwork = dalloc<double>(need, &err);
    if (!h->gwork) return err;
    h->gwork_cap = need;
  }
  RB_CUDA_TRY(gram<T>((const T* const*)(h->dptr + 256), mx, (const T* const*)(h->dptr + 384), my, h->npad,
                      h->dG, h->gwork, grid, h->us));
  RB_CUDA_TRY(cudaMemcpyAsync(G.data(), h->dG, sizeof(double) * G.size(), cudaMemcpyDeviceToHost, h->us));
  return sync(h);
}

// G = Z^T Z and H = Z^T W in one pass (both m x m, column-major, on the host).
template <typename T>
int block_gram_gh(rb_ctx* h, const std::vector<const T*>& Z, const std::vector<const T*>& W,
                  std::vector<double>& G, std::vector<double>& H) {
  const int m = (int)Z.size();
  G.assign((size_t)m * m, 0.0);
  H.assign((size_t)m * m, 0.0);
  if (!m) return RB_OK;
  int rc = sync(h);
  if (rc) return rc;
  rc = upload_ptrs(h, 2, Z);
  if (rc) return rc;
  rc = upload_ptrs(h, 3, W);
  if (rc) return rc;
  const int grid = 2 * h->nsm;
  const int64_t need = (int64_t)grid * gram_gh_work(m);
  if (need > h->gwork_cap) {
    cudaFree(h->gwork);
    int err = 0;
    h->gwork = dalloc<double>(need, &err);
    if (!h->gwork) return err;
    h->gwork_cap = need;
  }
  RB_CUDA_TRY(gram_gh<T>((const T* const*)(h->dptr + 256), (const T* const*)(h->dptr + 384), m, h->npad, h->dG,
                         h->dG + (size_t)kMaxGram * kMaxGram, h->gwork, grid, h->us));
  RB_CUDA_TRY(cudaMemcpyAsync(G.data(), h->dG, sizeof(double) * G.size(), cudaMemcpyDeviceToHost, h->us));
  RB_CUDA_TRY(cudaMemcpyAsync(H.data(), h->dG + (size_t)kMaxGram * kMaxGram, sizeof(double) * H.size(),
                              cudaMemcpyDeviceToHost, h->us));
  return sync(h);
}

// Squared 2-norms of the given columns.
template <typename T>
int block_colnorm2(rb_ctx* h, const std::vector<const T*>& M, std::vector<double>& out) {
  const int k = (int)M.size();
  out.assign(k, 0.0);
  if (!k) return RB_OK;
  int rc = sync(h);
  if (rc) return rc;
  rc = upload_ptrs(h, 2, M);
  if (rc) return rc;
  RB_CUDA_TRY(colnorm2<T>((const T* const*)(h->dptr + 256), k, h->npad, h->st, h->partials, h->grids.vec, h->us));
  RB_CUDA_TRY(cudaMemcpyAsync(h->hst->red, h->st->red, sizeof(double) * k, cudaMemcpyDeviceToHost, h->us));
  rc = sync(h);
  if (rc) return rc;
  std::memcpy(out.data(), h->hst->red, sizeof(double) * k);
  return RB_OK;
}

int alloc_vectors(rb_ctx* h) {
  int err = 0;
  double** vs[] = {&h->b, &h->x, &h->r, &h->p, &h->s, &h->q, &h->t, &h->qraw, &h->traw, &h->rt0, &h->tmp,
                    &h->rin, &h->xin};
  for (double** v : vs) {
    cudaFree(*v);
    *v = dalloc<double>(h->npad, &err);
    if (!*v) return err;
    RB_CUDA_TRY(cudaMemsetAsync(*v, 0, sizeof(double) * h->npad, h->us));
  }
  const int kc = std::max(1, h->kcap);
  double** ms[] = {&h->U, &h->Ut, &h->C, &h->Ct, &h->Chat, &h->T1, &h->T2};
  for (double** m : ms) {
    cudaFree(*m);
    *m = dalloc<double>(h->npad * kc, &err);
    if (!*m) return err;
    RB_CUDA_TRY(cudaMemsetAsync(*m, 0, sizeof(double) * h->npad * kc, h->us));
  }
  if (h->o.recycle_mode >= RB_RECYCLE_UPDATE_FIRST) {
    const size_t es = h->o.precision == RB_MIXED ? sizeof(float) : sizeof(double);
    h->cyc = h->o.cycle_s;
    void** ys[] = {&h->cstore, &h->Yc, &h->AYc, &h->Yn, &h->AYn};
    for (void** y : ys) {
      cudaFree(*y);
      const int64_t cnt = (y == &h->cstore ? 5 * (int64_t)h->cyc : (int64_t)kc) * h->npad;
      *y = dalloc<unsigned char>((int64_t)es * cnt, &err);
      if (!*y) return err;
      RB_CUDA_TRY(cudaMemsetAsync(*y, 0, es * cnt, h->us));
    }
  }
  if (h->o.precision == RB_MIXED) {
    float** fs[] = {&h->fx, &h->fr, &h->fp, &h->fs, &h->fq, &h->ft, &h->fqraw, &h->ftraw, &h->frt0};
    for (float** v : fs) {
      cudaFree(*v);
      *v = dalloc<float>(h->npad, &err);
      if (!*v) return err;
      RB_CUDA_TRY(cudaMemsetAsync(*v, 0, sizeof(float) * h->npad, h->us));
    }
    float** fm[] = {&h->fU, &h->fC, &h->fChat};
    for (float** m : fm) {
      cudaFree(*m);
      *m = dalloc<float>(h->npad * kc, &err);
      if (!*m) return err;
      RB_CUDA_TRY(cudaMemsetAsync(*m, 0, sizeof(float) * h->npad * kc, h->us));
    }
  }
  iteration_grids<double>(h->kcap, h->nsm, h->npad, &h->grids);
  Grids g0;
  iteration_grids<double>(0, h->nsm, h->npad, &g0);
  h->grids.spmv = std::max(h->grids.spmv, g0.spmv);
  h->grids.vec = std::max(h->grids.vec, g0.vec);
  return ensure_partials(h);
}

// ------------------------------------------------------------ recycle setup
// Alg. 2 step 1 for the columns currently in U, Ut (kin of them):
// C = A U, C~ = A^T U~, SVD biorthogonalisation, C-hat = C~ D_c^{-1}.
int recycle_setup(rb_ctx* h, int kin, int64_t* setup_mv) {
  PhaseClock pc;
  h->k = 0;
  reset_graphs(h);
  if (kin == 0) return RB_OK;
  const int64_t ld = h->npad;
  const int gs = h->grids.spmv;
  for (int j = 0; j < kin; ++j) {
    RB_CUDA_TRY(spmv<double>(h->A.view(), colp(h->U, ld, j), colp(h->C, ld, j), 1.0, 0.0, gs, h->us));
    RB_CUDA_TRY(spmv<double>(h->AT.view(), colp(h->Ut, ld, j), colp(h->Ct, ld, j), 1.0, 0.0, gs, h->us));
  }
  if (setup_mv) *setup_mv += 2 * kin;
  std::vector<const double*> Xc, Yc;
  for (int j = 0; j < kin; ++j) {
    Xc.push_back(colp(h->Ct, ld, j));
    Yc.push_back(colp(h->C, ld, j));
  }
  std::vector<double> M;
  int rc = block_gram<double>(h, Xc, Yc, M);
  if (rc) return rc;
  pc.lap("setup_spmm+gram");
  for (double v : M)
    if (!std::isfinite(v)) return RB_ENONFINITE;
  std::vector<double> P((size_t)kin * kin), Q((size_t)kin * kin), sig(kin);
  svd_small(kin, M.data(), P.data(), sig.data(), Q.data());
  int kk = 0;
  const double drop = h->o.precision == RB_MIXED ? kSvdDropF32 : kSvdDrop;
  if (sig[0] > 0)
    while (kk < kin && sig[kk] >= drop * sig[0]) ++kk;
  if (kk == 0) return RB_OK;
  // U <- U Q, C <- C Q, U~ <- U~ P, C~ <- C~ P (first kk columns of P, Q)
  std::vector<double> Qk(Q.begin(), Q.begin() + (size_t)kin * kk), Pk(P.begin(), P.begin() + (size_t)kin * kk);
  auto cols = [&](double* base, int cnt) {
    std::vector<double*> v;
    for (int j = 0; j < cnt; ++j) v.push_back(colp(base, ld, j));
    return v;
  };
  auto ccols = [&](double* base, int cnt) {
    std::vector<const double*> v;
    for (int j = 0; j < cnt; ++j) v.push_back(colp(base, ld, j));
    return v;
  };
  struct Job { double** src; const std::vector<double>* R; };
  Job jobs[] = {{&h->U, &Qk}, {&h->C, &Qk}, {&h->Ut, &Pk}, {&h->Ct, &Pk}};
  for (Job& jb : jobs) {
    rc = block_gemm<double>(h, cols(h->T1, kk), ccols(*jb.src, kin), *jb.R, kk);
    if (rc) return rc;
    std::swap(*jb.src, h->T1);
  }
  rc = sync(h);
  pc.lap("setup_gemm");
  std::vector<double> dinv(kk);
  for (int j = 0; j < kk; ++j) dinv[j] = 1.0 / sig[j];
  RB_CUDA_TRY(cudaMemcpyAsync(h->Chat, h->Ct, sizeof(double) * ld * kk, cudaMemcpyDeviceToDevice, h->us));
  rc = sync(h);
  if (rc) return rc;
  RB_CUDA_TRY(cudaMemcpy(h->Dinv, dinv.data(), sizeof(double) * kk, cudaMemcpyHostToDevice));
  RB_CUDA_TRY(scale_cols<double>(h->Chat, ld, kk, h->Dinv, h->npad, h->us));
  h->k = kk;
  if (h->o.precision == RB_MIXED) {
    RB_CUDA_TRY(to_float(h->U, h->fU, ld * kk, h->us));
    RB_CUDA_TRY(to_float(h->C, h->fC, ld * kk, h->us));
    RB_CUDA_TRY(to_float(h->Chat, h->fChat, ld * kk, h->us));
  }
  rc = sync(h);
  if (rc) return rc;
  return kk < kin ? RB_WRECYCLE_RANK : RB_OK;
}

// ------------------------------------------------------------ iteration args
template <typename T>
IterArgs<T> base_args(rb_ctx* h);

template <>
IterArgs<double> base_args<double>(rb_ctx* h) {
  IterArgs<double> a{};
  a.A = h->A.view();
  a.Chat = h->Chat;
  a.C = h->C;
  a.ld = h->npad;
  a.rt0 = h->rt0;
  a.x = h->x;
  a.r = h->r;
  a.p_in = h->p;
  a.p_out = h->p;
  a.s = h->s;
  a.qraw = h->qraw;
  a.traw = h->traw;
  a.q = h->k > 0 ? h->q : h->qraw;
  a.t = h->k > 0 ? h->t : h->traw;
  a.st = h->st;
  a.partials = h->partials;
  a.npad = h->npad;
  return a;
}

template <>
IterArgs<float> base_args<float>(rb_ctx* h) {
  IterArgs<float> a{};
  a.A = h->A32.view();
  a.Chat = h->fChat;
  a.C = h->fC;
  a.ld = h->npad;
  a.rt0 = h->frt0;
  a.x = h->fx;
  a.r = h->fr;
  a.p_in = h->fp;
  a.p_out = h->fp;
  a.s = h->fs;
  a.qraw = h->fqraw;
  a.traw = h->ftraw;
  a.q = h->k > 0 ? h->fq : h->fqraw;
  a.t = h->k > 0 ? h->ft : h->ftraw;
  a.st = h->st;
  a.partials = h->partials;
  a.npad = h->npad;
  return a;
}

// Cycle-store slots: P bank b slot j, S/QR/TR slot j.
template <typename T>
T* slotP(rb_ctx* h, int bank, int j) { return (T*)h->cstore + (int64_t)(bank * h->cyc + j) * h->npad; }
template <typename T>
T* slotS(rb_ctx* h, int j) { return (T*)h->cstore + (int64_t)(2 * h->cyc + j) * h->npad; }
template <typename T>
T* slotQ(rb_ctx* h, int j) { return (T*)h->cstore + (int64_t)(3 * h->cyc + j) * h->npad; }
template <typename T>
T* slotT(rb_ctx* h, int j) { return (T*)h->cstore + (int64_t)(4 * h->cyc + j) * h->npad; }

template <typename T>
int capture(rb_ctx* h, GraphSlot* g, int iters, int bank, bool cycle_mode) {
  if (g->exec) cudaGraphExecDestroy(g->exec);
  g->exec = nullptr;
  g->valid = false;
  cudaGraph_t graph = nullptr;
  RB_CUDA_TRY(cudaStreamBeginCapture(h->cs, cudaStreamCaptureModeThreadLocal));
  cudaError_t err = cudaSuccess;
  for (int j = 0; j < iters && err == cudaSuccess; ++j) {
    IterArgs<T> a = base_args<T>(h);
    if (cycle_mode) {
      a.p_in = slotP<T>(h, bank, j);
      a.p_out = (j + 1 < h->cyc) ? slotP<T>(h, bank, j + 1) : slotP<T>(h, 1 - bank, 0);
      a.s = slotS<T>(h, j);
      a.qraw = slotQ<T>(h, j);
      a.traw = slotT<T>(h, j);
      if (h->k == 0) {
        a.q = a.qraw;
        a.t = a.traw;
      }
    }
    Grids g;
    iteration_grids<T>(h->k, h->nsm, h->npad, &g);
    err = launch_iteration<T>(a, h->k, g, h->cs);
  }
  cudaError_t e2 = cudaStreamEndCapture(h->cs, &graph);
  if (err != cudaSuccess || e2 != cudaSuccess) {
    if (graph) cudaGraphDestroy(graph);
    return RB_ECUDA;
  }
  cudaError_t e3 = cudaGraphInstantiate(&g->exec, graph, 0);
  cudaGraphDestroy(graph);
  if (e3 != cudaSuccess) return RB_ECUDA;
  g->valid = true;
  return RB_OK;
}

int poll_iters(rb_ctx* h) {
  if (h->o.poll > 0) return h->o.poll;
  return h->npad >= (1 << 20) ? 8 : 16;
}

// ------------------------------------------------------------ solve core
struct SolveOut {
  int status = RB_OK;
  int iters = 0;
  int seeds = 1;
  int cycles = 0;
  int outer = 1;
  double ms_update = 0;
  int64_t mv = 0, mv_setup = 0, mv_check = 0;
  double relres_rec = 0, relres_true = 0;
  double bytes = 0;
};

double iter_bytes(rb_ctx* h, int k, size_t vb, size_t ab) {
  // per iteration: 2 SpMVs (values + int32 cols + slice padding ignored)
  // + 4 n*k reads (C-hat twice, C twice) + vector streams.
  const double z = (double)h->nnz, n = (double)h->n;
  const double spmv = 2.0 * (z * (ab + 4.0) + 4.0 * (n + 1));
  const double vec_streams = (k > 0) ? 21.0 : 14.0;  // see DESIGN notes
  return spmv + n * vb * (4.0 * k + vec_streams);
}

// Setup of one FP64 solve: x_0, r_0, r~_0, rho_0 (eq. (3.5), Alg. 2 steps 2-4).
int setup_solve(rb_ctx* h, const double* rhs, double* xb, bool x_nonzero, double tol, SolveOut* so) {
  const int k = h->k;
  const int64_t ld = h->npad;
  int rc;
  const int max_itn = h->o.max_itn > 0 ? h->o.max_itn : (int)std::min<int64_t>(h->n, 20000);
  // r_{-1} = b - A x_{-1}
  if (x_nonzero) {
    RB_CUDA_TRY(residual_norm(h->A.view(), rhs, xb, h->r, h->npad, h->st, h->partials, h->grids.spmv, h->us));
    so->mv += 1;
  } else {
    RB_CUDA_TRY(cudaMemcpyAsync(h->r, rhs, sizeof(double) * h->npad, cudaMemcpyDeviceToDevice, h->us));
  }
  if (k > 0) {
    DotArgs d{};
    d.M = h->Chat; d.ld = ld; d.km = k; d.v = h->r; d.nd = 0;
    RB_CUDA_TRY(dots(d, h->npad, h->st, h->partials, vec_grid(h), h->us));
    // x_0 = x_{-1} + U (C-hat^T r_{-1});  r_0 = r_{-1} - C (C-hat^T r_{-1})
    RB_CUDA_TRY(gemv_update(xb, h->U, ld, k, h->st->red, nullptr, 1.0, h->npad, vec_grid(h), h->us));
    RB_CUDA_TRY(gemv_update(h->r, h->C, ld, k, h->st->red, nullptr, -1.0, h->npad, vec_grid(h), h->us));
  }
  for (int attempt = 0; attempt < 4; ++attempt) {
    RB_CUDA_TRY(shadow(h->rt0, h->n, h->npad, h->o.shadow_seed + (uint64_t)attempt, h->us));
    if (k > 0) {
      DotArgs d{};
      d.M = h->C; d.ld = ld; d.km = k; d.v = h->rt0; d.nd = 0;
      RB_CUDA_TRY(dots(d, h->npad, h->st, h->partials, vec_grid(h), h->us));
      // r~_0 = r~_{-1} - C~ (D_c^{-1} C^T r~_{-1})
      RB_CUDA_TRY(gemv_update(h->rt0, h->Ct, ld, k, h->st->red, h->Dinv, -1.0, h->npad, vec_grid(h), h->us));
    }
    DotArgs d{};
    d.M = k > 0 ? h->C : nullptr; d.ld = ld; d.km = k; d.v = h->rt0;
    d.nd = 2;
    d.a[0] = h->rt0; d.b[0] = h->r;
    d.a[1] = h->r; d.b[1] = h->r;
    RB_CUDA_TRY(dots(d, h->npad, h->st, h->partials, vec_grid(h), h->us));
    RB_CUDA_TRY(init_state(h->st, k, tol, max_itn, h->us));
    rc = read_state(h);
    if (rc) return rc;
    so->seeds = attempt + 1;
    if (h->hst->status != RB_EBREAKDOWN_RHO) break;
  }
  return RB_OK;
}

// Launch graphs until the device reports done.  Non-update mode.
template <typename T>
int iterate_plain(rb_ctx* h) {
  if (!h->g_plain.valid || h->g_k != h->k) {
    int rc = capture<T>(h, &h->g_plain, poll_iters(h), 0, false);
    if (rc) return rc;
    h->g_k = h->k;
  }
  for (;;) {
    RB_CUDA_TRY(cudaGraphLaunch(h->g_plain.exec, h->us));
    count_launches((long long)poll_iters(h) * (h->k > 0 ? 5 : 4));
    int rc = read_state(h);
    if (rc) return rc;
    if (h->hst->done) break;
  }
  return RB_OK;
}

// Recycle update after a cycle: W = [Y, P, S], Z = [A Y, A P, A S] (Sec. 6.2
// cycles; harmonic-Ritz reading).  T is the inner precision: the Gram
// matrices are FP64 either way (Dot2 accumulation for FP32 columns); the new
// Y = W y and A Y = Z y are formed in T.
template <typename T>
int cycle_update(rb_ctx* h, int bank, int nit, int ns) {
  PhaseClock pc;
  const int64_t ld = h->npad;
  T* Yc = (T*)h->Yc;
  T* AYc = (T*)h->AYc;
  T* Yn = (T*)h->Yn;
  T* AYn = (T*)h->AYn;
  std::vector<const T*> W, Z;
  for (int j = 0; j < h->kY; ++j) {
    W.push_back(Yc + (int64_t)j * ld);
    Z.push_back(AYc + (int64_t)j * ld);
  }
  for (int j = 0; j < nit; ++j) {
    W.push_back(slotP<T>(h, bank, j));
    Z.push_back(slotQ<T>(h, j));
  }
  for (int j = 0; j < ns; ++j) {
    W.push_back(slotS<T>(h, j));
    Z.push_back(slotT<T>(h, j));
  }
  const int m = (int)W.size();
  if (m == 0) return RB_OK;
  std::vector<double> G, H;
  int rc = block_gram_gh<T>(h, Z, W, G, H);
  if (rc) return rc;
  pc.lap("gram");
  const int kt = std::min(h->o.k_max, m);
  std::vector<double> Y((size_t)m * std::max(kt, 1));
  const double rtol = std::is_same<T, float>::value ? kRankTolF32 : kRankTol;
  const int kn = harmonic_ritz(m, G.data(), H.data(), kt, rtol, Y.data(), nullptr, nullptr);
  pc.lap("harmonic_ritz");
  if (kn <= 0) return RB_OK;   // nothing usable: keep the old candidate
  Y.resize((size_t)m * kn);
  std::vector<T*> oY, oAY;
  for (int j = 0; j < kn; ++j) {
    oY.push_back(Yn + (int64_t)j * ld);
    oAY.push_back(AYn + (int64_t)j * ld);
  }
  rc = block_gemm<T>(h, oY, W, Y, kn);
  if (rc) return rc;
  rc = block_gemm<T>(h, oAY, Z, Y, kn);
  if (rc) return rc;
  rc = sync(h);
  pc.lap("gemm");
  // unit 2-norm columns
  std::vector<const T*> yc(oY.begin(), oY.end());
  std::vector<double> N2;
  rc = block_colnorm2<T>(h, yc, N2);
  if (rc) return rc;
  std::vector<double> f(kn);
  for (int j = 0; j < kn; ++j) {
    const double nn = N2[j];
    f[j] = nn > 0 ? 1.0 / std::sqrt(nn) : 0.0;
  }
  RB_CUDA_TRY(cudaMemcpy(h->dR, f.data(), sizeof(double) * kn, cudaMemcpyHostToDevice));
  RB_CUDA_TRY(scale_cols<T>(Yn, ld, kn, h->dR, h->npad, h->us));
  RB_CUDA_TRY(scale_cols<T>(AYn, ld, kn, h->dR, h->npad, h->us));
  std::swap(h->Yc, h->Yn);
  std::swap(h->AYc, h->AYn);
  h->kY = kn;
  rc = sync(h);
  pc.lap("normalise");
  return rc;
}

// One solve's iterations in update mode: graphs of one cycle each, the
// recycle update between cycles.  Candidate Y = U, A Y = C at the start;
// p_1 = r_0 goes to bank 0, slot 0.
template <typename T>
int iterate_cycles(rb_ctx* h, SolveOut* so) {
  const int64_t ld = h->npad;
  const bool f32 = std::is_same<T, float>::value;
  h->kY = h->k;
  if (h->k > 0) {
    RB_CUDA_TRY(cudaMemcpyAsync(h->Yc, f32 ? (const void*)h->fU : (const void*)h->U, sizeof(T) * ld * h->k,
                                cudaMemcpyDeviceToDevice, h->us));
    RB_CUDA_TRY(cudaMemcpyAsync(h->AYc, f32 ? (const void*)h->fC : (const void*)h->C, sizeof(T) * ld * h->k,
                                cudaMemcpyDeviceToDevice, h->us));
  }
  RB_CUDA_TRY(cudaMemcpyAsync(slotP<T>(h, 0, 0), f32 ? (const void*)h->fr : (const void*)h->r, sizeof(T) * ld,
                              cudaMemcpyDeviceToDevice, h->us));
  if (h->g_k != h->k || !h->g_cycle[0].valid || !h->g_cycle[1].valid) {
    for (int bnk = 0; bnk < 2; ++bnk) {
      int rc = capture<T>(h, &h->g_cycle[bnk], h->cyc, bnk, true);
      if (rc) return rc;
    }
    h->g_k = h->k;
  }
  int iters_before = 0;
  for (int c = 0;; ++c) {
    const int bank = c & 1;
    RB_CUDA_TRY(cudaGraphLaunch(h->g_cycle[bank].exec, h->us));
    count_launches((long long)h->cyc * (h->k > 0 ? 5 : 4));
    int rc = read_state(h);
    if (rc) return rc;
    const IterState& hs = *h->hst;
    const int nit = hs.iter - iters_before;
    iters_before = hs.iter;
    const bool ok = (hs.status == RB_OK || hs.status == RB_ENOTCONV);
    const bool allowed = (h->o.update_cycles == 0) || (c < h->o.update_cycles);
    if (ok && allowed && nit > 0) {
      const int ns = nit - (hs.half ? 1 : 0);
      const auto t0 = std::chrono::steady_clock::now();
      rc = cycle_update<T>(h, bank, nit, ns);
      so->ms_update += std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
      if (rc) return rc;
      so->cycles += 1;
    }
    if (hs.done) break;
  }
  return RB_OK;
}

int finish_solve(rb_ctx* h, SolveOut* so, bool check) {
  const int64_t ld = h->npad;
  if (h->k > 0)   // Alg. 2 step 8: x = x - U x_c
    RB_CUDA_TRY(gemv_update(h->x, h->U, ld, h->k, h->st->xc, nullptr, -1.0, h->npad, vec_grid(h), h->us));
  if (check) {
    RB_CUDA_TRY(residual_norm(h->A.view(), h->b, h->x, h->tmp, h->npad, h->st, h->partials, h->grids.spmv, h->us));
    so->mv_check += 1;
  }
  return read_state(h);
}

}  // namespace

// ============================================================ C ABI
static void release_a32(rb_ctx* h);


extern "C" const char* rbicgstab_error_string(int status) {
  switch (status) {
    case RB_OK: return "RB_OK";
    case RB_WRECYCLE_RANK: return "RB_WRECYCLE_RANK: recycle space rank-deficient, k reduced";
    case RB_EINVAL: return "RB_EINVAL: invalid argument";
    case RB_EDIM: return "RB_EDIM: dimension mismatch or no matrix set";
    case RB_EBADCSR: return "RB_EBADCSR: malformed CSR matrix";
    case RB_ENONFINITE: return "RB_ENONFINITE: non-finite value";
    case RB_ENOMEM: return "RB_ENOMEM: device out of memory";
    case RB_ECUDA: return "RB_ECUDA: CUDA runtime error";
    case RB_ENOTCONV: return "RB_ENOTCONV: max_itn reached";
    case RB_EBREAKDOWN_RHO: return "RB_EBREAKDOWN_RHO: (r~0, r) or (r~0, q) is zero";
    case RB_EBREAKDOWN_OMEGA: return "RB_EBREAKDOWN_OMEGA: (t, t) = 0 or omega = 0";
    case RB_ETIMEOUT: return "RB_ETIMEOUT: bounded device wait expired";
    default: return "unknown status";
  }
}

extern "C" int rbicgstab_create(rb_handle* out, const rb_opts* opts) {
  if (!out || !opts) return RB_EINVAL;
  *out = nullptr;
  rb_opts o = *opts;
  if (o.cycle_s == 0) o.cycle_s = 25;
  if (o.tol == 0.0) o.tol = 1e-8;
  if (o.shadow_seed == 0) o.shadow_seed = 0x5EED;
  if (o.k_max < 0 || o.k_max > RB_KMAX || o.cycle_s < 1 || o.max_itn < 0 || !(o.tol > 0) ||
      o.precision < RB_FP64 || o.precision > RB_MIXED || o.recycle_mode < RB_RECYCLE_NONE ||
      o.recycle_mode > RB_RECYCLE_UPDATE_ALL || o.update_cycles < 0 || o.poll < 0)
    return RB_EINVAL;
  if (o.recycle_mode >= RB_RECYCLE_UPDATE_FIRST && o.k_max + 2 * o.cycle_s > kMaxGram) return RB_EINVAL;
  rb_ctx* h = new rb_ctx();
  h->o = o;
  h->us = (cudaStream_t)o.cuda_stream;
  int err = RB_OK;
  auto fail = [&](int e) {
    rbicgstab_destroy(h);
    return e;
  };
  if (cudaGetDevice(&h->dev) != cudaSuccess) return fail(RB_ECUDA);
  if (cudaDeviceGetAttribute(&h->nsm, cudaDevAttrMultiProcessorCount, h->dev) != cudaSuccess)
    return fail(RB_ECUDA);
  if (cudaStreamCreateWithFlags(&h->cs, cudaStreamNonBlocking) != cudaSuccess) return fail(RB_ECUDA);
  h->st = dalloc<IterState>(1, &err);
  if (!h->st) return fail(err);
  if (cudaMemset(h->st, 0, sizeof(IterState)) != cudaSuccess) return fail(RB_ECUDA);
  if (cudaMallocHost(&h->hst, sizeof(IterState)) != cudaSuccess) return fail(RB_ENOMEM);
  std::memset(h->hst, 0, sizeof(IterState));
  h->dflag = dalloc<int>(1, &err);
  if (!h->dflag) return fail(err);
  h->kcap = o.k_max;
  h->Dinv = dalloc<double>(std::max(1, h->kcap), &err);
  if (!h->Dinv) return fail(err);
  h->dptr = (const double**)dalloc<double*>(4 * 128, &err);
  if (!h->dptr) return fail(err);
  h->dG = dalloc<double>(2 * kMaxGram * kMaxGram, &err);
  h->dR = dalloc<double>(kMaxGram * std::max(RB_KMAX, kMaxGram), &err);
  if (!h->dG || !h->dR) return fail(err ? err : RB_ENOMEM);
  *out = h;
  return RB_OK;
}

extern "C" int rbicgstab_destroy(rb_handle h) {
  if (!h) return RB_OK;
  cudaStreamSynchronize(h->us);
  reset_graphs(h);
  release_a32(h);
  sell_free(&h->A);
  sell_free(&h->AT);
  void* ptrs[] = {h->rp, h->ci, h->cv, h->trp, h->tci, h->tsrc, h->tcv, h->U, h->Ut, h->C, h->Ct,
                  h->Chat, h->T1, h->T2, h->Dinv, h->b, h->x, h->r, h->p, h->s, h->q, h->t,
                  h->qraw, h->traw, h->rt0, h->tmp, h->rin, h->xin, h->fx, h->fr, h->fp, h->fs, h->fq, h->ft,
                  h->fqraw, h->ftraw, h->frt0, h->fU, h->fC, h->fChat, h->st, h->partials,
                  h->dflag, h->cstore, h->Yc, h->AYc, h->Yn, h->AYn, h->gwork, h->dG, h->dR,
                  (void*)h->dptr};
  for (void* p : ptrs) cudaFree(p);
  if (h->hst) cudaFreeHost(h->hst);
  if (h->cs) cudaStreamDestroy(h->cs);
  delete h;
  return RB_OK;
}

// The FP32 copy of A shares the SELL structure of the FP64 one and owns only
// its values.
static void release_a32(rb_ctx* h) {
  cudaFree(h->A32.val);
  h->A32 = SellBuf<float>();
}

static int build_matrix_values(rb_ctx* h) {
  int rc = sell_fill_values<double>(h->A, h->cv, h->us);
  if (rc) return rc;
  rc = gather_values(h->nnz, h->tsrc, h->cv, h->tcv, h->us);
  if (rc) return rc;
  rc = sell_fill_values<double>(h->AT, h->tcv, h->us);
  if (rc) return rc;
  if (h->o.precision == RB_MIXED) {
    rc = sell_fill_values<float>(h->A32, h->cv, h->us);
    if (rc) return rc;
  }
  return sync(h);
}

extern "C" int rbicgstab_set_matrix(rb_handle h, int64_t n, int64_t nnz, const int32_t* row_ptr,
                         const int32_t* col, const double* val, int where) {
  if (!h || n <= 0 || nnz < 0 || n >= (1ll << 31) || nnz >= (1ll << 31) || !row_ptr ||
      (nnz > 0 && (!col || !val)) || (where != RB_HOST && where != RB_DEVICE))
    return RB_EINVAL;
  int err = RB_OK;
  const bool resize = (n != h->n);
  int rc = sync(h);
  if (rc) return rc;
  reset_graphs(h);
  cudaFree(h->rp); cudaFree(h->ci); cudaFree(h->cv);
  cudaFree(h->trp); cudaFree(h->tci); cudaFree(h->tsrc); cudaFree(h->tcv);
  h->rp = h->ci = h->trp = h->tci = nullptr;
  h->cv = h->tcv = nullptr;
  h->tsrc = nullptr;
  h->have_matrix = false;
  h->rp = dalloc<int32_t>(n + 1, &err);
  h->ci = dalloc<int32_t>(nnz, &err);
  h->cv = dalloc<double>(nnz, &err);
  h->trp = dalloc<int32_t>(n + 1, &err);
  h->tci = dalloc<int32_t>(nnz, &err);
  h->tsrc = dalloc<int64_t>(nnz, &err);
  h->tcv = dalloc<double>(nnz, &err);
  if (err) return err;
  rc = copy_in(h->rp, row_ptr, sizeof(int32_t) * (n + 1), where, h->us);
  if (!rc) rc = copy_in(h->ci, col, sizeof(int32_t) * nnz, where, h->us);
  if (!rc) rc = copy_in(h->cv, val, sizeof(double) * nnz, where, h->us);
  if (rc) return rc;
  int bad = 0;
  rc = csr_validate(n, nnz, h->rp, h->ci, h->cv, h->dflag, &bad, h->us);
  if (rc) return rc;
  if (bad) return bad;
  h->n = n;
  h->nnz = nnz;
  h->npad = round_up(n, kSlice);
  release_a32(h);
  rc = sell_build(n, nnz, h->rp, h->ci, &h->A, h->us);
  if (rc) return rc;
  rc = csr_transpose(n, nnz, h->rp, h->ci, h->trp, h->tci, h->tsrc, h->us);
  if (rc) return rc;
  rc = sell_build(n, nnz, h->trp, h->tci, &h->AT, h->us);
  if (rc) return rc;
  if (h->o.precision == RB_MIXED) {
    release_a32(h);
    h->A32.nslices = h->A.nslices;
    h->A32.cap = h->A.cap;
    h->A32.slice_ptr = h->A.slice_ptr;   // shared structure (not owned)
    h->A32.width = h->A.width;
    h->A32.col = h->A.col;
    h->A32.perm = h->A.perm;
    h->A32.val = dalloc<float>(h->A.cap, &err);
    if (err) return err;
  }
  if (resize) {
    h->k = 0;
    rc = alloc_vectors(h);
    if (rc) return rc;
  }
  rc = build_matrix_values(h);
  if (rc) return rc;
  h->have_matrix = true;
  h->matrix_epoch += 1;
  // keep U, U~ and recompute C, C~, D_c for the new matrix
  const int kin = h->k;
  if (kin > 0) {
    int64_t mv = 0;
    rc = recycle_setup(h, kin, &mv);
    if (rc < 0) return rc;
    return rc;
  }
  return RB_OK;
}

extern "C" int rbicgstab_set_values(rb_handle h, const double* val, int where) {
  if (!h || (!val && h->nnz > 0)) return RB_EINVAL;
  if (!h->have_matrix) return RB_EDIM;
  int rc = copy_in(h->cv, val, sizeof(double) * h->nnz, where, h->us);
  if (rc) return rc;
  int bad = 0;
  rc = csr_validate(h->n, h->nnz, h->rp, h->ci, h->cv, h->dflag, &bad, h->us);
  if (rc) return rc;
  if (bad) return bad;
  rc = build_matrix_values(h);
  if (rc) return rc;
  h->matrix_epoch += 1;
  if (h->k > 0) {
    int64_t mv = 0;
    return recycle_setup(h, h->k, &mv);
  }
  return RB_OK;
}

extern "C" int rbicgstab_set_recycle(rb_handle h, int32_t k, const double* U, const double* Ut, int64_t ld,
                          int where) {
  if (!h || k < 0 || (where != RB_HOST && where != RB_DEVICE)) return RB_EINVAL;
  if (k > h->kcap) return RB_EINVAL;
  if (!h->have_matrix) return RB_EDIM;
  if (k > 0 && (!U || ld < h->n)) return RB_EINVAL;
  int rc = sync(h);
  if (rc) return rc;
  const int64_t npad = h->npad;
  for (int j = 0; j < k; ++j) {
    rc = copy_in(colp(h->U, npad, j), U + (int64_t)j * ld, sizeof(double) * h->n, where, h->us);
    if (!rc) rc = copy_in(colp(h->Ut, npad, j), (Ut ? Ut : U) + (int64_t)j * ld, sizeof(double) * h->n, where, h->us);
    if (rc) return rc;
  }
  if (k > 0) {
    RB_CUDA_TRY(check_finite(h->U, npad * k, h->dflag, h->us));
    int f1 = 0;
    RB_CUDA_TRY(cudaMemcpyAsync(&f1, h->dflag, sizeof(int), cudaMemcpyDeviceToHost, h->us));
    rc = sync(h);
    if (rc) return rc;
    RB_CUDA_TRY(check_finite(h->Ut, npad * k, h->dflag, h->us));
    int f2 = 0;
    RB_CUDA_TRY(cudaMemcpyAsync(&f2, h->dflag, sizeof(int), cudaMemcpyDeviceToHost, h->us));
    rc = sync(h);
    if (rc) return rc;
    if (f1 || f2) {
      h->k = 0;
      reset_graphs(h);
      return RB_ENONFINITE;
    }
  }
  int64_t mv = 0;
  return recycle_setup(h, k, &mv);
}

extern "C" int rbicgstab_get_recycle(rb_handle h, int32_t* k, double* U, double* Ut, int64_t ld, int where) {
  if (!h || !k || (where != RB_HOST && where != RB_DEVICE)) return RB_EINVAL;
  *k = h->k;
  if (h->k == 0) return RB_OK;
  if ((U || Ut) && ld < h->n) return RB_EINVAL;
  for (int j = 0; j < h->k; ++j) {
    int rc = RB_OK;
    if (U) rc = copy_out(U + (int64_t)j * ld, colp(h->U, h->npad, j), sizeof(double) * h->n, where, h->us);
    if (!rc && Ut) rc = copy_out(Ut + (int64_t)j * ld, colp(h->Ut, h->npad, j), sizeof(double) * h->n, where, h->us);
    if (rc) return rc;
  }
  return sync(h);
}

extern "C" int rbicgstab_apply(rb_handle h, const double* v, double* y, int transpose, int where) {
  if (!h || !v || !y || (transpose != 0 && transpose != 1) || (where != RB_HOST && where != RB_DEVICE))
    return RB_EINVAL;
  if (!h->have_matrix) return RB_EDIM;
  int rc = copy_in(h->tmp, v, sizeof(double) * h->n, where, h->us);
  if (rc) return rc;
  RB_CUDA_TRY(spmv<double>(transpose ? h->AT.view() : h->A.view(), h->tmp, h->qraw, 1.0, 0.0,
                           h->grids.spmv, h->us));
  rc = copy_out(y, h->qraw, sizeof(double) * h->n, where, h->us);
  if (rc) return rc;
  return sync(h);
}

extern "C" int rbicgstab_harmonic_ritz(int32_t m, const double* G, const double* H, int32_t k, double* Y,
                            double* theta_re, double* theta_im, int32_t* k_used) {
  if (m <= 0 || k <= 0 || k > m || !G || !H || !Y || !k_used) return RB_EINVAL;
  const int r = rb::harmonic_ritz(m, G, H, k, kRankTol, Y, theta_re, theta_im);
  if (r < 0) return RB_ENOTCONV;
  *k_used = r;
  return RB_OK;
}

static int solve_fp64(rb_ctx* h, SolveOut* so, bool x_nonzero) {
  int rc = setup_solve(h, h->b, h->x, x_nonzero, h->o.tol, so);
  if (rc) return rc;
  const bool upd = (h->o.recycle_mode == RB_RECYCLE_UPDATE_ALL) ||
                   (h->o.recycle_mode == RB_RECYCLE_UPDATE_FIRST && h->update_epoch != h->matrix_epoch);
  if (!h->hst->done) {
    if (upd) {
      rc = iterate_cycles<double>(h, so);
    } else {
      // p_1 = r_0 (Alg. 2 step 4 with beta_0 = 0)
      RB_CUDA_TRY(cudaMemcpyAsync(h->p, h->r, sizeof(double) * h->npad, cudaMemcpyDeviceToDevice, h->us));
      rc = iterate_plain<double>(h);
    }
    if (rc) return rc;
  }
  rc = finish_solve(h, so, true);
  if (rc) return rc;
  const IterState& hs = *h->hst;
  so->status = hs.status;
  so->iters = hs.iter;
  so->mv += 2 * (int64_t)hs.iter - (hs.half ? 1 : 0);
  so->relres_rec = std::sqrt(hs.rnorm2 / hs.bnorm2);
  so->relres_true = std::sqrt(hs.red[0] / hs.bnorm2);
  if (hs.bnorm2 == 0) so->relres_rec = so->relres_true = 0.0;
  so->bytes = (double)hs.iter * iter_bytes(h, h->k, 8, 8);
  if (upd && (hs.status == RB_OK || hs.status == RB_ENOTCONV) && h->kY > 0) {
    // U_next = Y (unit columns), U~_next = U_next; recompute C, C~, D_c
    const int64_t ld = h->npad;
    RB_CUDA_TRY(cudaMemcpyAsync(h->U, h->Yc, sizeof(double) * ld * h->kY, cudaMemcpyDeviceToDevice, h->us));
    RB_CUDA_TRY(cudaMemcpyAsync(h->Ut, h->Yc, sizeof(double) * ld * h->kY, cudaMemcpyDeviceToDevice, h->us));
    int64_t mv = 0;
    const auto t0 = std::chrono::steady_clock::now();
    rc = recycle_setup(h, h->kY, &mv);
    so->ms_update += std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
    if (rc < 0) return rc;
    so->mv_setup += mv;
    h->update_epoch = h->matrix_epoch;
  }
  return RB_OK;
}


// Mixed precision: FP64 iterative refinement around an FP32 inner RBiCGSTAB.
// Outer: r = b - A x in FP64; inner: A d = r with FP32 vectors, FP32 SpMV and
// FP32 recycle blocks, FP64 dot products and scalars; x += d in FP64.
static int solve_mixed(rb_ctx* h, SolveOut* so, bool x_nonzero) {
  const int64_t ld = h->npad;
  (void)x_nonzero;
  const double bn2 = h->hst->red[0];
  // refine to a tenth of the tolerance: the last FP32 correction then leaves
  // a forward error comparable to the FP64 solver's at the tolerance itself
  const double target = 0.1 * h->o.tol * std::sqrt(bn2);
  const int max_outer = 12;
  int outer = 0, total_it = 0, last_status = RB_OK;
  const bool upd = (h->o.recycle_mode == RB_RECYCLE_UPDATE_ALL) ||
                   (h->o.recycle_mode == RB_RECYCLE_UPDATE_FIRST && h->update_epoch != h->matrix_epoch);
  bool did_update = false;
  double rn = 0.0;
  for (;;) {
    RB_CUDA_TRY(residual_norm(h->A.view(), h->b, h->x, h->rin, h->npad, h->st, h->partials, h->grids.spmv, h->us));
    so->mv_check += 1;
    int rc = read_state(h);
    if (rc) return rc;
    rn = std::sqrt(h->hst->red[0]);
    if (!std::isfinite(rn)) { so->status = RB_ENONFINITE; break; }
    if (rn <= target || bn2 == 0.0) { so->status = RB_OK; break; }
    if (outer >= max_outer || total_it >= (h->o.max_itn > 0 ? h->o.max_itn : (int)std::min<int64_t>(h->n, 20000))) {
      so->status = last_status != RB_OK ? last_status : RB_ENOTCONV;
      break;
    }
    // inner system A d = r_outer, tolerance relative to ||r_outer||
    const double tol_in = std::max(target / rn, 1e-6);
    RB_CUDA_TRY(cudaMemcpyAsync(&h->st->bnorm2, &h->st->red[0], sizeof(double), cudaMemcpyDeviceToDevice, h->us));
    RB_CUDA_TRY(cudaMemsetAsync(h->xin, 0, sizeof(double) * ld, h->us));
    rc = setup_solve(h, h->rin, h->xin, false, tol_in, so);
    if (rc) return rc;
    RB_CUDA_TRY(to_float(h->r, h->fr, ld, h->us));
    RB_CUDA_TRY(to_float(h->r, h->fp, ld, h->us));
    RB_CUDA_TRY(to_float(h->rt0, h->frt0, ld, h->us));
    RB_CUDA_TRY(to_float(h->xin, h->fx, ld, h->us));
    if (!h->hst->done) {
      if (upd && !did_update) {
        // the first (longest) inner solve collects the cycles of the update
        rc = iterate_cycles<float>(h, so);
        did_update = true;
      } else {
        rc = iterate_plain<float>(h);
      }
      if (rc) return rc;
    }
    rc = read_state(h);
    if (rc) return rc;
    const IterState& hs = *h->hst;
    total_it += hs.iter;
    so->mv += 2 * (int64_t)hs.iter - (hs.half ? 1 : 0);
    last_status = hs.status;
    // x += d, d = x_inner - U x_c (Alg. 2 step 8 of the inner solve)
    RB_CUDA_TRY(add_float_to_double(h->x, h->fx, ld, h->us));
    if (h->k > 0)
      RB_CUDA_TRY(gemv_update(h->x, h->U, ld, h->k, h->st->xc, nullptr, -1.0, h->npad, vec_grid(h), h->us));
    ++outer;
    if (hs.status != RB_OK && hs.status != RB_ENOTCONV) { so->status = hs.status; break; }
  }
  so->iters = total_it;
  so->seeds = 1;
  so->relres_true = bn2 > 0 ? rn / std::sqrt(bn2) : 0.0;
  so->relres_rec = so->relres_true;
  so->bytes = (double)total_it * iter_bytes(h, h->k, 4, 4);
  so->outer = outer;
  if (did_update && h->kY > 0 && (so->status == RB_OK || so->status == RB_ENOTCONV)) {
    // U_next = Y (FP32 candidate promoted to FP64), U~_next = U_next
    for (int j = 0; j < h->kY; ++j)
      RB_CUDA_TRY(to_double((const float*)h->Yc + (int64_t)j * ld, h->U + (int64_t)j * ld, ld, h->us));
    RB_CUDA_TRY(cudaMemcpyAsync(h->Ut, h->U, sizeof(double) * ld * h->kY, cudaMemcpyDeviceToDevice, h->us));
    int64_t mv = 0;
    const auto t0 = std::chrono::steady_clock::now();
    int rc2 = recycle_setup(h, h->kY, &mv);
    so->ms_update += std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
    if (rc2 < 0) return rc2;
    so->mv_setup += mv;
    h->update_epoch = h->matrix_epoch;
  }
  return sync(h);
}

extern "C" int rbicgstab_solve(rb_handle h, const double* b, double* x, int where, rb_stats* st_out) {
  if (!h || !b || !x || (where != RB_HOST && where != RB_DEVICE)) return RB_EINVAL;
  if (!h->have_matrix) return RB_EDIM;
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  cudaEventRecord(e0, h->us);
  SolveOut so;
  int rc = copy_in(h->b, b, sizeof(double) * h->n, where, h->us);
  if (!rc) rc = copy_in(h->x, x, sizeof(double) * h->n, where, h->us);
  if (rc) return rc;
  // finiteness of b and x, ||b||^2, ||x||^2
  RB_CUDA_TRY(check_finite(h->b, h->n, h->dflag, h->us));
  int fb = 0, fx = 0;
  RB_CUDA_TRY(cudaMemcpyAsync(&fb, h->dflag, sizeof(int), cudaMemcpyDeviceToHost, h->us));
  rc = sync(h);
  if (rc) return rc;
  RB_CUDA_TRY(check_finite(h->x, h->n, h->dflag, h->us));
  RB_CUDA_TRY(cudaMemcpyAsync(&fx, h->dflag, sizeof(int), cudaMemcpyDeviceToHost, h->us));
  DotArgs d{};
  d.nd = 2;
  d.a[0] = h->b; d.b[0] = h->b;
  d.a[1] = h->x; d.b[1] = h->x;
  double nb[2];
  rc = run_dots(h, d, nb, 2);
  if (rc) return rc;
  if (fb || fx) return RB_ENONFINITE;
  RB_CUDA_TRY(cudaMemcpyAsync(&h->st->bnorm2, &h->st->red[0], sizeof(double), cudaMemcpyDeviceToDevice, h->us));
  const bool x_nonzero = nb[1] != 0.0;
  h->hst->red[0] = nb[0];
  rc = (h->o.precision == RB_MIXED) ? solve_mixed(h, &so, x_nonzero) : solve_fp64(h, &so, x_nonzero);
  if (rc < 0 && rc != RB_ENOTCONV) return rc;
  rc = copy_out(x, h->x, sizeof(double) * h->n, where, h->us);
  if (rc) return rc;
  cudaEventRecord(e1, h->us);
  rc = sync(h);
  if (rc) return rc;
  float ms = 0;
  cudaEventElapsedTime(&ms, e0, e1);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (st_out) {
    st_out->iters = so.iters;
    st_out->status = so.status;
    st_out->k_used = h->k;
    st_out->seeds_used = so.seeds;
    st_out->matvecs = so.mv;
    st_out->matvecs_setup = so.mv_setup;
    st_out->matvecs_check = so.mv_check;
    st_out->cycles = so.cycles;
    st_out->outer = so.outer;
    st_out->relres_rec = so.relres_rec;
    st_out->relres_true = so.relres_true;
    st_out->ms_total = ms;
    st_out->bytes_model = so.bytes;
    st_out->ms_update = so.ms_update;
  }
  return so.status;
}


// Benchmark helper: average duration of each pass kernel, measured with CUDA
// events on the handle's stream over `reps` iterations started from b.
template <typename T>
static int time_passes_t(rb_ctx* h, int reps, double* ms) {
  IterArgs<T> a = base_args<T>(h);
  Grids g;
  iteration_grids<T>(h->k, h->nsm, h->npad, &g);
  const int npass = 5;
  std::vector<cudaEvent_t> ev((size_t)reps * npass * 2);
  for (auto& e : ev) cudaEventCreate(&e);
  for (int it = 0; it < reps; ++it)
    for (int pz = 0; pz < npass; ++pz) {
      if (pz == P4 && h->k == 0) continue;
      RB_CUDA_TRY(cudaEventRecord(ev[(it * npass + pz) * 2], h->us));
      RB_CUDA_TRY(launch_pass<T>(pz, a, h->k, g, h->us));
      RB_CUDA_TRY(cudaEventRecord(ev[(it * npass + pz) * 2 + 1], h->us));
    }
  int rc = read_state(h);
  for (int pz = 0; pz < npass; ++pz) ms[pz] = 0.0;
  if (!rc) {
    for (int it = 0; it < reps; ++it)
      for (int pz = 0; pz < npass; ++pz) {
        if (pz == P4 && h->k == 0) continue;
        float t = 0;
        cudaEventElapsedTime(&t, ev[(it * npass + pz) * 2], ev[(it * npass + pz) * 2 + 1]);
        ms[pz] += t / reps;
      }
  }
  for (auto& e : ev) cudaEventDestroy(e);
  if (rc) return rc;
  return h->hst->done ? (h->hst->status ? h->hst->status : RB_EBREAKDOWN_OMEGA) : RB_OK;
}

extern "C" int rbicgstab_time_passes(rb_handle h, const double* b, int where, int32_t reps, double* ms) {
  if (!h || !b || !ms || reps < 1 || reps > 1000 || (where != RB_HOST && where != RB_DEVICE)) return RB_EINVAL;
  if (!h->have_matrix) return RB_EDIM;
  int rc = copy_in(h->b, b, sizeof(double) * h->n, where, h->us);
  if (rc) return rc;
  RB_CUDA_TRY(cudaMemsetAsync(h->x, 0, sizeof(double) * h->npad, h->us));
  DotArgs d{};
  d.nd = 1;
  d.a[0] = h->b; d.b[0] = h->b;
  double nb = 0;
  rc = run_dots(h, d, &nb, 1);
  if (rc) return rc;
  RB_CUDA_TRY(cudaMemcpyAsync(&h->st->bnorm2, &h->st->red[0], sizeof(double), cudaMemcpyDeviceToDevice, h->us));
  SolveOut so;
  rc = setup_solve(h, h->b, h->x, false, 1e-300, &so);
  if (rc) return rc;
  RB_CUDA_TRY(cudaMemcpyAsync(h->p, h->r, sizeof(double) * h->npad, cudaMemcpyDeviceToDevice, h->us));
  rc = read_state(h);
  if (rc) return rc;
  if (h->hst->done) return h->hst->status ? h->hst->status : RB_EINVAL;
  if (h->o.precision == RB_MIXED) {
    RB_CUDA_TRY(to_float(h->r, h->fr, h->npad, h->us));
    RB_CUDA_TRY(to_float(h->r, h->fp, h->npad, h->us));
    RB_CUDA_TRY(to_float(h->rt0, h->frt0, h->npad, h->us));
    RB_CUDA_TRY(cudaMemsetAsync(h->fx, 0, sizeof(float) * h->npad, h->us));
    return time_passes_t<float>(h, reps, ms);
  }
  return time_passes_t<double>(h, reps, ms);
}

extern "C" long long rbicgstab_kernel_launches(void) { return g_launches.load(); }
