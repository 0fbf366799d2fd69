// Orchestrator and C ABI of librbicgstab (see include/rbicgstab.h).
//
// A solve (Alg. 2) runs as: setup of x_0, r_0, r~_0 (eq. (3.5)) with a few
// generic kernels; then the fused five-pass iteration, captured once per
// handle as a CUDA graph of `poll` iterations and replayed until the device
// convergence flags are set (every pass returns at once after they are set,
// so the overshoot of the last replay costs only empty launches); then the final correction x - U x_c
// (x = x - U x_c) and a true-residual check.  In the recycle-update modes the
// graph spans one cycle of s iterations whose p, s, A p, A s vectors land in
// a cycle store; between cycles the Gram matrices G = Z^T Z, H = Z^T W are
// formed on the device, the small harmonic-Ritz problem is solved on the
// host, and the candidate space Y, A Y is rebuilt on the device (Sec. 6.2).
//
// Blocked solves: up to four right-hand sides of the same matrix iterate
// together ("slots"), each with its own vectors and device state, so every
// pass reads A, C, C-hat and r~_0 once for all of them.  In update mode the
// cycle store takes slot 0's vectors, so the recycle update is built from the
// Krylov space of the first right-hand side of the block.
#include <algorithm>
#include <atomic>
#include <chrono>
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <functional>
#include <type_traits>
#include <vector>

#include "device.cuh"
#include "hostla.h"
#include "kernels.h"

using namespace rb;

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
constexpr int kBanks = 3;            // cycle-store banks (see slotP)

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
  int k = -1, nrhs = -1;   // the recycle dimension and block size it was captured for
};

// Vectors of one right-hand side.  FP64: b, x and the iteration vectors;
// rin, xin are the inner right-hand side and correction of the mixed path,
// whose FP32 iteration vectors are the f* fields.
struct Slot {
  double *b = nullptr, *x = nullptr, *r = nullptr, *p = nullptr, *s = nullptr, *q = nullptr, *t = nullptr,
         *qraw = nullptr, *traw = nullptr, *rin = nullptr, *xin = nullptr;
  float *fx = nullptr, *fr = nullptr, *fp = nullptr, *fs = nullptr, *fq = nullptr, *ft = nullptr,
        *fqraw = nullptr, *ftraw = nullptr;
};

const int kOne = 1;    // source of the "done" flag written for masked slots
const int kZero = 0;   // ... and of the flag cleared when a solve resumes

}  // namespace

struct rb_ctx {
  rb_opts o{};
  cudaStream_t us = nullptr;   // caller's stream
  cudaStream_t cs = nullptr;   // private stream used for graph capture
  cudaStream_t ws = nullptr;   // recycle-update stream (overlaps the next cycle)
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
  // The recycle setup (Sec. 3) owed for the first setup_pending columns of U, U~ (-1:
  // none).  A new matrix or an adopted update only marks the setup; the next
  // solve runs it, so a setup that no solve would use is never computed.
  int setup_pending = -1;
  // recycle space (column-major, leading dimension npad), k_used columns
  int k = 0, kcap = 0;
  double *U = nullptr, *Ut = nullptr, *C = nullptr, *Ct = nullptr, *Chat = nullptr;
  double *T1 = nullptr, *T2 = nullptr;   // scratch blocks (kcap columns each)
  double* Dinv = nullptr;                // ones (device): coefficient scale of the dual's C^T products
  // Mpt (k x k, column-major, host): C-hat = C~ Mpt.  The pseudo-inverse
  // transpose of M = C~^T C when the columns are kept as computed, diag(1 / D_c)
  // after a rank-reducing biorthogonalisation.
  std::vector<double> Mpt;
  float *fU = nullptr, *fC = nullptr, *fChat = nullptr;
  // per right-hand-side vectors; shared r~_0 and scratch
  Slot sl[kMaxRhs];
  int nslots = 0;
  double *rt0 = nullptr, *tmp = nullptr, *tmp2 = nullptr;
  float* frt0 = nullptr;
  // device states, one per slot (contiguous), and their pinned host mirror
  IterState* st = nullptr;
  IterState* hst = nullptr;
  double* partials = nullptr;
  int64_t partials_cap = 0;
  int* dflag = nullptr;
  int* tcerr = nullptr;   // bounded-wait failures of the tensor-core Gram
  double* lvec = nullptr;   // BiCGstab(l) work vectors (lvec_cnt columns of npad)
  int lvec_cnt = 0;
  // cycle store for the recycle update, kBanks banks of cyc vectors each for
  // P, S, QR = A P and TR = A S, of the inner precision (double for RB_FP64,
  // float for RB_MIXED), and the candidate Y, A Y
  int cyc = 0;
  void* cstore = nullptr;
  void *Yc = nullptr, *AYc = nullptr, *Yn = nullptr, *AYn = nullptr;
  int kY = 0;
  double* gwork = nullptr;
  int64_t gwork_cap = 0;
  double *dG = nullptr, *dR = nullptr;
  const double** dptr = nullptr;   // device pointer lists (4 * 128)
  Grids grids{};
  GraphSlot g_plain[2], g_cycle[kBanks];   // plain iterations: [0] FP32, [1] FP64
  GraphSlot g_bicg;       // Alg. 1 iterations (primary + dual)
  int g_bicg_k = -1;
  int g_cycle_ts = 0;     // element size the cycle graphs were captured for
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
  for (GraphSlot* g : {&h->g_plain[0], &h->g_plain[1], &h->g_cycle[0], &h->g_cycle[1], &h->g_cycle[2], &h->g_bicg}) {
    if (g->exec) cudaGraphExecDestroy(g->exec);
    g->exec = nullptr;
    g->valid = false;
    g->k = g->nrhs = -1;
  }
  h->g_cycle_ts = 0;
  h->g_bicg_k = -1;
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

// Copy the device states of slots [0, nrhs) to the pinned mirror and wait.
int read_state(rb_ctx* h, int nrhs = 1) {
  RB_CUDA_TRY(cudaMemcpyAsync(h->hst, h->st, sizeof(IterState) * nrhs, cudaMemcpyDeviceToHost, h->us));
  return sync(h);
}

int vec_grid(rb_ctx* h) { return h->grids.vec; }

// Deterministic dot products / projections into st[slot].red, then read
// back `cnt` values.
int run_dots(rb_ctx* h, const DotArgs& d, double* out, int cnt, int slot = 0) {
  RB_CUDA_TRY(dots(d, h->npad, h->st + slot, h->partials, vec_grid(h), h->us));
  if (out) {
    RB_CUDA_TRY(cudaMemcpyAsync(h->hst[slot].red, h->st[slot].red, sizeof(double) * cnt,
                                cudaMemcpyDeviceToHost, h->us));
    int rc = sync(h);
    if (rc) return rc;
    std::memcpy(out, h->hst[slot].red, sizeof(double) * cnt);
  }
  return RB_OK;
}

int ensure_partials(rb_ctx* h) {
  // every kernel runs at most one full wave (<= 8 blocks of 256 threads per
  // SM) and reduces at most kMaxRhs * kMaxNV values per block; the grid
  // reduction adds one row per group of blocks
  const int gmax = std::max(8 * h->nsm, std::max(h->grids.spmv, h->grids.vec));
  const int64_t need = grid_partial_rows(gmax) * kMaxRhs * kMaxNV;
  if (need <= h->partials_cap) return RB_OK;
  cudaFree(h->partials);
  int err = 0;
  h->partials = dalloc<double>(need, &err);
  if (!h->partials) return err;
  h->partials_cap = need;
  return RB_OK;
}

// Column pointer lists for gram / gemm_cols, copied on stream s; the host
// vector must live until s has passed the copy (callers synchronise s).
template <typename P>
int upload_ptrs(rb_ctx* h, int slot, const std::vector<P>& v, cudaStream_t s) {
  RB_CUDA_TRY(cudaMemcpyAsync(h->dptr + slot * 128, v.data(), sizeof(double*) * v.size(),
                              cudaMemcpyHostToDevice, s));
  return RB_OK;
}
template <typename P>
int upload_ptrs(rb_ctx* h, int slot, const std::vector<P>& v) {
  return upload_ptrs(h, slot, v, h->us);
}

// Out = X R (column lists) with R (m x kc column-major) given on the host;
// enqueued on stream s, which is synchronised before returning.
template <typename T>
int block_gemm(rb_ctx* h, const std::vector<T*>& out, const std::vector<const T*>& X,
               const std::vector<double>& R, int kc, cudaStream_t s) {
  const int m = (int)X.size();
  if (kc == 0 || m == 0) return RB_OK;
  int rc = upload_ptrs(h, 0, X, s);
  if (rc) return rc;
  rc = upload_ptrs(h, 1, out, s);
  if (rc) return rc;
  RB_CUDA_TRY(cudaMemcpyAsync(h->dR, R.data(), sizeof(double) * (size_t)m * kc, cudaMemcpyHostToDevice, s));
  RB_CUDA_TRY(gemm_cols<T>((T* const*)(h->dptr + 128), (const T* const*)h->dptr, m, h->dR, kc,
                           h->npad, vec_grid(h), s));
  RB_CUDA_TRY(cudaStreamSynchronize(s));
  return RB_OK;
}
template <typename T>
int block_gemm(rb_ctx* h, const std::vector<T*>& out, const std::vector<const T*>& X,
               const std::vector<double>& R, int kc) {
  int rc = sync(h);
  if (rc) return rc;
  return block_gemm<T>(h, out, X, R, kc, h->us);
}

int ensure_gwork(rb_ctx* h, int64_t need) {
  if (need <= h->gwork_cap) return RB_OK;
  cudaFree(h->gwork);
  int err = 0;
  h->gwork = dalloc<double>(need, &err);
  if (!h->gwork) return err;
  h->gwork_cap = need;
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
  rc = ensure_gwork(h, (int64_t)grid * mx * my);
  if (rc) return rc;
  RB_CUDA_TRY(gram<T>((const T* const*)(h->dptr + 256), mx, (const T* const*)(h->dptr + 384), my, h->npad,
                      h->dG, h->gwork, grid, h->us));
  RB_CUDA_TRY(cudaMemcpyAsync(G.data(), h->dG, sizeof(double) * G.size(), cudaMemcpyDeviceToHost, h->us));
  return sync(h);
}

// G = Z^T Z and H = Z^T W in one pass (both m x m, column-major, on the
// host), on stream s, which is synchronised before returning.
template <typename T>
int block_gram_gh(rb_ctx* h, const std::vector<const T*>& Z, const std::vector<const T*>& W,
                  std::vector<double>& G, std::vector<double>& H, cudaStream_t s) {
  const int m = (int)Z.size();
  G.assign((size_t)m * m, 0.0);
  H.assign((size_t)m * m, 0.0);
  if (!m) return RB_OK;
  int rc = upload_ptrs(h, 2, Z, s);
  if (rc) return rc;
  rc = upload_ptrs(h, 3, W, s);
  if (rc) return rc;
  const int grid = 2 * h->nsm;
  if (h->gwork_cap < (int64_t)grid * gram_gh_work(m)) {   // reallocation: nothing may use gwork meanwhile
    RB_CUDA_TRY(cudaStreamSynchronize(s));
    rc = ensure_gwork(h, (int64_t)grid * gram_gh_work(m));
    if (rc) return rc;
  }
  RB_CUDA_TRY(gram_gh<T>((const T* const*)(h->dptr + 256), (const T* const*)(h->dptr + 384), m, h->npad, h->dG,
                         h->dG + (size_t)kMaxGram * kMaxGram, h->gwork, grid, s));
  RB_CUDA_TRY(cudaMemcpyAsync(G.data(), h->dG, sizeof(double) * G.size(), cudaMemcpyDeviceToHost, s));
  RB_CUDA_TRY(cudaMemcpyAsync(H.data(), h->dG + (size_t)kMaxGram * kMaxGram, sizeof(double) * H.size(),
                              cudaMemcpyDeviceToHost, s));
  RB_CUDA_TRY(cudaStreamSynchronize(s));
  return RB_OK;
}

// G = Z^T Z and H = Z^T W on the tensor cores for FP32 column blocks (see
// gram_tc.cu); same outputs and stream discipline as block_gram_gh.
// Returns RB_ETIMEOUT if a CTA gave up a bounded wait.
int block_gram_gh_tc(rb_ctx* h, const GramTcBlocks& blk, std::vector<double>& G, std::vector<double>& H,
                     cudaStream_t s) {
  const int m = blk.cols[0] + blk.cols[1] + blk.cols[2];
  G.assign((size_t)m * m, 0.0);
  H.assign((size_t)m * m, 0.0);
  if (!m) return RB_OK;
  const int grid = h->nsm;
  const int64_t need = (int64_t)((gram_tc_work_floats(blk.cap, grid) + 1) / 2);
  if (h->gwork_cap < need) {   // reallocation: nothing may use gwork meanwhile
    RB_CUDA_TRY(cudaStreamSynchronize(s));
    int rc = ensure_gwork(h, need);
    if (rc) return rc;
  }
  RB_CUDA_TRY(cudaMemsetAsync(h->tcerr, 0, sizeof(int), s));
  int rc = gram_tc(blk, h->n, h->npad, h->dG, h->dG + (size_t)kMaxGram * kMaxGram, (float*)h->gwork, h->tcerr,
                   grid, s);
  if (rc) return rc;
  int herr = 0;
  RB_CUDA_TRY(cudaMemcpyAsync(G.data(), h->dG, sizeof(double) * G.size(), cudaMemcpyDeviceToHost, s));
  RB_CUDA_TRY(cudaMemcpyAsync(H.data(), h->dG + (size_t)kMaxGram * kMaxGram, sizeof(double) * H.size(),
                              cudaMemcpyDeviceToHost, s));
  RB_CUDA_TRY(cudaMemcpyAsync(&herr, h->tcerr, sizeof(int), cudaMemcpyDeviceToHost, s));
  RB_CUDA_TRY(cudaStreamSynchronize(s));
  return herr ? RB_ETIMEOUT : RB_OK;
}

// Whether the cycle Gram of this handle runs on the tensor cores: FP32
// columns and a tile layout that fits (k + 2 s small enough); RB_GRAM_CUDACORE
// in the environment selects the CUDA-core kernel instead.
bool use_gram_tc(rb_ctx* h) {
  static const bool off = getenv("RB_GRAM_CUDACORE") != nullptr;
  if (off) return false;
  const int cap[6] = {h->o.k_max, h->cyc, h->cyc, h->o.k_max, h->cyc, h->cyc};
  return gram_tc_eligible(cap);
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

template <typename T>
int zero_alloc(T** p, int64_t cnt, rb_ctx* h) {
  cudaFree(*p);
  int err = 0;
  *p = dalloc<T>(cnt, &err);
  if (!*p) return err;
  RB_CUDA_TRY(cudaMemsetAsync(*p, 0, sizeof(T) * (size_t)cnt, h->us));
  return RB_OK;
}

void free_slot(Slot& s) {
  void* ptrs[] = {s.b, s.x, s.r, s.p, s.s, s.q, s.t, s.qraw, s.traw, s.rin, s.xin,
                  s.fx, s.fr, s.fp, s.fs, s.fq, s.ft, s.fqraw, s.ftraw};
  for (void* p : ptrs) cudaFree(p);
  s = Slot();
}

// Vectors of slots [0, nrhs) (npad entries; the tail beyond n stays zero).
int ensure_slots(rb_ctx* h, int nrhs) {
  for (int i = h->nslots; i < nrhs; ++i) {
    Slot& s = h->sl[i];
    double** vs[] = {&s.b, &s.x, &s.r, &s.p, &s.s, &s.q, &s.t, &s.qraw, &s.traw, &s.rin, &s.xin};
    for (double** v : vs) {
      int rc = zero_alloc(v, h->npad, h);
      if (rc) return rc;
    }
    if (h->o.precision == RB_MIXED) {
      float** fs[] = {&s.fx, &s.fr, &s.fp, &s.fs, &s.fq, &s.ft, &s.fqraw, &s.ftraw};
      for (float** v : fs) {
        int rc = zero_alloc(v, h->npad, h);
        if (rc) return rc;
      }
    }
    h->nslots = i + 1;
    reset_graphs(h);
  }
  return RB_OK;
}

int alloc_vectors(rb_ctx* h) {
  for (int i = 0; i < h->nslots; ++i) free_slot(h->sl[i]);
  h->nslots = 0;
  int rc = ensure_slots(h, 1);
  if (rc) return rc;
  double** vs[] = {&h->rt0, &h->tmp, &h->tmp2};
  for (double** v : vs)
    if ((rc = zero_alloc(v, h->npad, h))) return rc;
  const int kc = std::max(1, h->kcap);
  double** ms[] = {&h->U, &h->Ut, &h->C, &h->Ct, &h->Chat, &h->T1, &h->T2};
  for (double** m : ms)
    if ((rc = zero_alloc(m, h->npad * kc, h))) return rc;
  if (h->o.recycle_mode >= RB_RECYCLE_UPDATE_FIRST) {
    const int64_t es = h->o.precision == RB_MIXED ? sizeof(float) : sizeof(double);
    h->cyc = h->o.cycle_s;
    void** ys[] = {&h->cstore, &h->Yc, &h->AYc, &h->Yn, &h->AYn};
    for (void** y : ys) {
      const int64_t cnt = (y == &h->cstore ? 4 * kBanks * (int64_t)h->cyc : (int64_t)kc) * h->npad;
      unsigned char* p = (unsigned char*)*y;
      rc = zero_alloc(&p, es * cnt, h);
      *y = p;
      if (rc) return rc;
    }
  }
  if (h->o.precision == RB_MIXED) {
    if ((rc = zero_alloc(&h->frt0, h->npad, h))) return rc;
    float** fm[] = {&h->fU, &h->fC, &h->fChat};
    for (float** m : fm)
      if ((rc = zero_alloc(m, h->npad * kc, h))) return rc;
  }
  // generic grids: the largest over k in {0, kcap} and every block size
  h->grids = Grids{};
  for (int kk : {0, h->kcap})
    for (int nr : {1, 2, kMaxRhs}) {
      Grids g;
      iteration_grids<double>(kk, h->nsm, h->npad, &g, nr);
      h->grids.spmv = std::max(h->grids.spmv, g.spmv);
      h->grids.vec = std::max(h->grids.vec, g.vec);
    }
  return ensure_partials(h);
}

// ------------------------------------------------------------ recycle setup
// The recycle setup (Sec. 3, eq. (3.4)) for the columns currently in U, Ut
// (kin of them): C = A U, C~ = A^T U~, M = C~^T C and its SVD M = P S Q^T.
// The iteration needs only the oblique projector C C-hat^T, the coefficient
// map C-hat^T and U in the same basis.  With the biorthogonalised columns of
// Sec. 3 (U Q, C Q, U~ P, C~ P, D_c = S) the projector is C M^+ C~^T, so
// when M has full numerical rank the columns are kept as computed and
// C-hat = C~ M^+^T (one n x k x k product instead of four rotations); when
// singular values fall below the drop tolerance the rotations are applied
// and the weak directions dropped (k_used < k, RB_WRECYCLE_RANK).
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
  if (kk == kin) {
    // Mpt = M^+^T = P S^-1 Q^T;  C-hat = C~ Mpt
    h->Mpt.assign((size_t)kin * kin, 0.0);
    for (int c = 0; c < kin; ++c)
      for (int r = 0; r < kin; ++r) {
        double acc = 0.0;
        for (int j = 0; j < kin; ++j) acc += P[r + (size_t)j * kin] * Q[c + (size_t)j * kin] / sig[j];
        h->Mpt[r + (size_t)c * kin] = acc;
      }
    rc = block_gemm<double>(h, cols(h->Chat, kin), ccols(h->Ct, kin), h->Mpt, kin);
    if (rc) return rc;
  } else {
    // U <- U Q, C <- C Q, U~ <- U~ P, C~ <- C~ P (first kk columns), C-hat = C~ D_c^-1
    std::vector<double> Qk(Q.begin(), Q.begin() + (size_t)kin * kk), Pk(P.begin(), P.begin() + (size_t)kin * kk);
    struct Job {
      double** src;
      const std::vector<double>* R;
    };
    Job jobs[] = {{&h->U, &Qk}, {&h->C, &Qk}, {&h->Ut, &Pk}, {&h->Ct, &Pk}};
    for (Job& jb : jobs) {
      rc = block_gemm<double>(h, cols(h->T1, kk), ccols(*jb.src, kin), *jb.R, kk);
      if (rc) return rc;
      std::swap(*jb.src, h->T1);
    }
    h->Mpt.assign((size_t)kk * kk, 0.0);
    for (int j = 0; j < kk; ++j) h->Mpt[j + (size_t)j * kk] = 1.0 / sig[j];
    rc = block_gemm<double>(h, cols(h->Chat, kk), ccols(h->Ct, kk), h->Mpt, kk);
    if (rc) return rc;
  }
  rc = sync(h);
  if (rc) return rc;
  pc.lap("setup_gemm");
  std::vector<double> ones(kk, 1.0);
  RB_CUDA_TRY(cudaMemcpy(h->Dinv, ones.data(), sizeof(double) * kk, cudaMemcpyHostToDevice));
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

// Defer the recycle setup for kin columns of U, U~ to the next solve.
void mark_setup(rb_ctx* h, int kin) {
  h->k = 0;
  reset_graphs(h);
  h->setup_pending = kin;
}

// Run a deferred setup; its matrix-vector products are added to *setup_mv.
int ensure_setup(rb_ctx* h, int64_t* setup_mv) {
  if (h->setup_pending < 0) return RB_OK;
  const int kin = h->setup_pending;
  h->setup_pending = -1;
  const int rc = recycle_setup(h, kin, setup_mv);
  return rc == RB_WRECYCLE_RANK ? RB_OK : rc;
}

// ------------------------------------------------------------ iteration args
// Which staged passes move their tiles by bulk copies (bit 0: P2, bit 1:
// P4, bit 2: P5; the others use per-thread cp.async; same arithmetic,
// bitwise-equal results).  Measured at 128^3, k = 20, four right-hand sides
// (microseconds, bulk / cp.async): P2 63 / 67-73, P4 76 / 71-72, P5 53 /
// 50-52, so only P2 takes bulk copies.  RB_STAGE_BULK=<mask> overrides.
int stage_bulk() {
  static const int v = [] {
    const char* e = getenv("RB_STAGE_BULK");
    return e ? atoi(e) & 7 : 1;
  }();
  return v;
}

template <typename T>
IterArgs<T> base_args(rb_ctx* h, int nrhs);

template <>
IterArgs<double> base_args<double>(rb_ctx* h, int nrhs) {
  IterArgs<double> a{};
  a.A = h->A.view();
  a.Chat = h->Chat;
  a.C = h->C;
  a.ld = h->npad;
  a.rt0 = h->rt0;
  for (int i = 0; i < nrhs; ++i) {
    Slot& s = h->sl[i];
    a.x[i] = s.x;
    a.r[i] = s.r;
    a.p_in[i] = s.p;
    a.p_out[i] = s.p;
    a.s[i] = s.s;
    a.qraw[i] = s.qraw;
    a.traw[i] = s.traw;
    a.q[i] = h->k > 0 ? s.q : s.qraw;
    a.t[i] = h->k > 0 ? s.t : s.traw;
  }
  a.st = h->st;
  a.partials = h->partials;
  a.npad = h->npad;
  a.nrhs = nrhs;
  a.stage_bulk = stage_bulk();
  return a;
}

template <>
IterArgs<float> base_args<float>(rb_ctx* h, int nrhs) {
  IterArgs<float> a{};
  a.A = h->A32.view();
  a.Chat = h->fChat;
  a.C = h->fC;
  a.ld = h->npad;
  a.rt0 = h->frt0;
  for (int i = 0; i < nrhs; ++i) {
    Slot& s = h->sl[i];
    a.x[i] = s.fx;
    a.r[i] = s.fr;
    a.p_in[i] = s.fp;
    a.p_out[i] = s.fp;
    a.s[i] = s.fs;
    a.qraw[i] = s.fqraw;
    a.traw[i] = s.ftraw;
    a.q[i] = h->k > 0 ? s.fq : s.fqraw;
    a.t[i] = h->k > 0 ? s.ft : s.ftraw;
  }
  a.st = h->st;
  a.partials = h->partials;
  a.npad = h->npad;
  a.nrhs = nrhs;
  a.stage_bulk = stage_bulk();
  return a;
}

// Cycle-store slots, bank b, slot j: P, S, QR = A P, TR = A S.  Cycle c
// uses bank c mod 3 and its last iteration writes p_{i+1} into slot 0 of the
// next bank, while the update of cycle c - 1 reads bank (c - 1) mod 3.
template <typename T>
T* slotP(rb_ctx* h, int bank, int j) { return (T*)h->cstore + (int64_t)(bank * h->cyc + j) * h->npad; }
template <typename T>
T* slotS(rb_ctx* h, int bank, int j) {
  return (T*)h->cstore + (int64_t)((kBanks + bank) * h->cyc + j) * h->npad;
}
template <typename T>
T* slotQ(rb_ctx* h, int bank, int j) {
  return (T*)h->cstore + (int64_t)((2 * kBanks + bank) * h->cyc + j) * h->npad;
}
template <typename T>
T* slotT(rb_ctx* h, int bank, int j) {
  return (T*)h->cstore + (int64_t)((3 * kBanks + bank) * h->cyc + j) * h->npad;
}

template <typename T>
int capture(rb_ctx* h, GraphSlot* g, int iters, int bank, bool cycle_mode, int nrhs) {
  if (g->exec) cudaGraphExecDestroy(g->exec);
  g->exec = nullptr;
  g->valid = false;
  cudaGraph_t graph = nullptr;
  Grids gr;
  iteration_grids<T>(h->k, h->nsm, h->npad, &gr, nrhs);
  RB_CUDA_TRY(cudaStreamBeginCapture(h->cs, cudaStreamCaptureModeThreadLocal));
  cudaError_t err = cudaSuccess;
  for (int j = 0; j < iters && err == cudaSuccess; ++j) {
    IterArgs<T> a = base_args<T>(h, nrhs);
    if (cycle_mode) {   // slot 0's vectors go to the cycle store
      a.p_in[0] = slotP<T>(h, bank, j);
      a.p_out[0] = (j + 1 < h->cyc) ? slotP<T>(h, bank, j + 1) : slotP<T>(h, (bank + 1) % kBanks, 0);
      a.s[0] = slotS<T>(h, bank, j);
      a.qraw[0] = slotQ<T>(h, bank, j);
      a.traw[0] = slotT<T>(h, bank, j);
      if (h->k == 0) {
        a.q[0] = a.qraw[0];
        a.t[0] = a.traw[0];
      }
    }
    err = launch_iteration<T>(a, h->k, gr, h->cs);
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

int passes_per_iter(rb_ctx* h) { return h->k > 0 ? 5 : 4; }

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

// Modelled HBM bytes of one iteration attributed to one of nrhs slots: two
// SpMVs (values + int32 columns + row pointers) and four n x k block reads
// (C-hat twice, C twice) are shared by the block; 21 (k > 0) or 14 vector
// streams belong to each right-hand side.
double iter_bytes(rb_ctx* h, int k, size_t vb, size_t ab, int nrhs) {
  const double z = (double)h->nnz, n = (double)h->n;
  const double shared = 2.0 * (z * (ab + 4.0) + 4.0 * (n + 1)) + 4.0 * n * k * vb;
  const double vec_streams = (k > 0) ? 21.0 : 14.0;
  return shared / nrhs + n * vb * vec_streams;
}

// Setup of a blocked FP64 solve (the start of Alg. 2, eq. (3.5)) for slots
// [0, nrhs): rhs[i], xb[i] are slot i's right-hand side and iterate; tol[i]
// is relative to st[i].bnorm2 (set by the caller); skip[i] marks slots that
// take no part and are marked done.  The shadow r~_{-1} (hence r~_0) is
// shared; when (r~_0, r_0) = 0 for any slot every slot takes the next seed.
int setup_block(rb_ctx* h, int nrhs, double* const* rhs, double* const* xb, const bool* x_nonzero,
                const bool* skip, const double* tol, SolveOut* so) {
  const int k = h->k;
  const int64_t ld = h->npad;
  const int max_itn = h->o.max_itn > 0 ? h->o.max_itn : (int)std::min<int64_t>(h->n, 20000);
  for (int i = 0; i < nrhs; ++i) {
    if (skip[i]) continue;
    Slot& s = h->sl[i];
    IterState* st = h->st + i;
    // r_{-1} = b - A x_{-1}
    if (x_nonzero[i]) {
      RB_CUDA_TRY(residual_norm(h->A.view(), rhs[i], xb[i], s.r, h->npad, st, h->partials, h->grids.spmv, h->us));
      so[i].mv += 1;
    } else {
      RB_CUDA_TRY(cudaMemcpyAsync(s.r, rhs[i], sizeof(double) * h->npad, cudaMemcpyDeviceToDevice, h->us));
    }
    if (k > 0) {
      DotArgs d{};
      d.M = h->Chat; d.ld = ld; d.km = k; d.v = s.r; d.nd = 0;
      RB_CUDA_TRY(dots(d, h->npad, st, h->partials, vec_grid(h), h->us));
      // x_0 = x_{-1} + U (C-hat^T r_{-1});  r_0 = r_{-1} - C (C-hat^T r_{-1})
      RB_CUDA_TRY(gemv_update(xb[i], h->U, ld, k, st->red, nullptr, 1.0, h->npad, vec_grid(h), h->us));
      RB_CUDA_TRY(gemv_update(s.r, h->C, ld, k, st->red, nullptr, -1.0, h->npad, vec_grid(h), h->us));
    }
  }
  for (int attempt = 0; attempt < 4; ++attempt) {
    RB_CUDA_TRY(shadow(h->rt0, h->n, h->npad, h->o.shadow_seed + (uint64_t)attempt, h->us));
    if (k > 0) {
      DotArgs d{};
      d.M = h->C; d.ld = ld; d.km = k; d.v = h->rt0; d.nd = 0;
      RB_CUDA_TRY(dots(d, h->npad, h->st, h->partials, vec_grid(h), h->us));
      // r~_0 = r~_{-1} - C~ C-check^T r~_{-1} = r~_{-1} - C-hat (C^T r~_{-1})
      RB_CUDA_TRY(gemv_update(h->rt0, h->Chat, ld, k, h->st->red, nullptr, -1.0, h->npad, vec_grid(h), h->us));
    }
    for (int i = 0; i < nrhs; ++i) {
      if (skip[i]) continue;
      DotArgs d{};
      d.M = k > 0 ? h->C : nullptr; d.ld = ld; d.km = k; d.v = h->rt0;
      d.nd = 2;
      d.a[0] = h->rt0; d.b[0] = h->sl[i].r;
      d.a[1] = h->sl[i].r; d.b[1] = h->sl[i].r;
      RB_CUDA_TRY(dots(d, h->npad, h->st + i, h->partials, vec_grid(h), h->us));
      RB_CUDA_TRY(init_state(h->st + i, k, tol[i], max_itn, h->us));
    }
    int rc = read_state(h, nrhs);
    if (rc) return rc;
    bool redo = false;
    for (int i = 0; i < nrhs; ++i) {
      so[i].seeds = attempt + 1;
      if (!skip[i] && h->hst[i].status == RB_EBREAKDOWN_RHO) redo = true;
    }
    if (!redo) break;
  }
  bool any_skip = false;
  for (int i = 0; i < nrhs; ++i)
    if (skip[i]) {
      RB_CUDA_TRY(cudaMemcpyAsync(&h->st[i].done, &kOne, sizeof(int), cudaMemcpyHostToDevice, h->us));
      any_skip = true;
    }
  return any_skip ? read_state(h, nrhs) : RB_OK;
}

bool all_done(rb_ctx* h, int nrhs) {
  for (int i = 0; i < nrhs; ++i)
    if (!h->hst[i].done) return false;
  return true;
}

// p_1 = r_0 for every slot (beta_0 = 0 before the first iteration); slot 0 writes to
// the cycle store in update mode.
template <typename T>
int init_p(rb_ctx* h, int nrhs, bool cycle_slot0) {
  const bool f32 = std::is_same<T, float>::value;
  for (int i = 0; i < nrhs; ++i) {
    Slot& s = h->sl[i];
    void* dst = f32 ? (void*)s.fp : (void*)s.p;
    const void* src = f32 ? (const void*)s.fr : (const void*)s.r;
    if (i == 0 && cycle_slot0) dst = slotP<T>(h, 0, 0);
    RB_CUDA_TRY(cudaMemcpyAsync(dst, src, sizeof(T) * h->npad, cudaMemcpyDeviceToDevice, h->us));
  }
  return RB_OK;
}

// Called after every graph replay with the states read back; may change
// device state (a residual replacement) before the done flags are checked.
using PollHook = std::function<int()>;

// Launch graphs until every slot reports done.  Non-update mode.
template <typename T>
int iterate_plain(rb_ctx* h, int nrhs, const PollHook& hook = nullptr) {
  GraphSlot& g = h->g_plain[sizeof(T) == sizeof(double) ? 1 : 0];
  if (!g.valid || g.k != h->k || g.nrhs != nrhs) {   // only this graph is captured again
    int rc = capture<T>(h, &g, poll_iters(h), 0, false, nrhs);
    if (rc) return rc;
    g.k = h->k;
    g.nrhs = nrhs;
  }
  for (;;) {
    RB_CUDA_TRY(cudaGraphLaunch(g.exec, h->us));
    count_launches((long long)poll_iters(h) * passes_per_iter(h));
    int rc = read_state(h, nrhs);
    if (rc) return rc;
    if (hook && (rc = hook())) return rc;
    if (all_done(h, nrhs)) break;
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
  const cudaStream_t s = h->ws;
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
    Z.push_back(slotQ<T>(h, bank, j));
  }
  for (int j = 0; j < ns; ++j) {
    W.push_back(slotS<T>(h, bank, j));
    Z.push_back(slotT<T>(h, bank, j));
  }
  const int m = (int)W.size();
  if (m == 0) return RB_OK;
  std::vector<double> G, H;
  int rc;
  if (std::is_same<T, float>::value && use_gram_tc(h)) {
    GramTcBlocks blk;
    const float* src[6] = {(const float*)AYc, (const float*)slotQ<T>(h, bank, 0), (const float*)slotT<T>(h, bank, 0),
                           (const float*)Yc, (const float*)slotP<T>(h, bank, 0), (const float*)slotS<T>(h, bank, 0)};
    const int cols[3] = {h->kY, nit, ns};
    for (int b = 0; b < 6; ++b) {
      blk.ptr[b] = src[b];
      blk.cols[b] = cols[b % 3];
      blk.cap[b] = (b % 3 == 0) ? h->o.k_max : h->cyc;
    }
    rc = block_gram_gh_tc(h, blk, G, H, s);
  } else {
    rc = block_gram_gh<T>(h, Z, W, G, H, s);
  }
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
  rc = block_gemm<T>(h, oY, W, Y, kn, s);
  if (rc) return rc;
  rc = block_gemm<T>(h, oAY, Z, Y, kn, s);
  if (rc) return rc;
  // The candidate's columns are not rescaled here: the next cycle's
  // harmonic-Ritz problem is invariant to a column scaling of W (with Z = A W
  // scaled alike) and rescales by diag(Z^T Z) itself.  They are normalised
  // once, when adopted as U.
  std::swap(h->Yc, h->Yn);
  std::swap(h->AYc, h->AYn);
  h->kY = kn;
  pc.lap("gemm");
  return RB_OK;
}

// Iterations in update mode: graphs of one cycle each; the recycle update of
// cycle c (from slot 0's vectors) runs on the update stream and the host
// while cycle c + 1 iterates.  Candidate Y = U, A Y = C at the start; the
// caller has put p_1 of slot 0 into bank 0, slot 0.
template <typename T>
int iterate_cycles(rb_ctx* h, int nrhs, SolveOut* so, const PollHook& hook = nullptr) {
  const int64_t ld = h->npad;
  const bool f32 = std::is_same<T, float>::value;
  h->kY = h->k;
  if (h->k > 0) {
    RB_CUDA_TRY(cudaMemcpyAsync(h->Yc, f32 ? (const void*)h->fU : (const void*)h->U, sizeof(T) * ld * h->k,
                                cudaMemcpyDeviceToDevice, h->us));
    RB_CUDA_TRY(cudaMemcpyAsync(h->AYc, f32 ? (const void*)h->fC : (const void*)h->C, sizeof(T) * ld * h->k,
                                cudaMemcpyDeviceToDevice, h->us));
  }
  bool have_graphs = h->g_cycle_ts == (int)sizeof(T);
  for (int b = 0; b < kBanks; ++b)
    have_graphs = have_graphs && h->g_cycle[b].valid && h->g_cycle[b].k == h->k && h->g_cycle[b].nrhs == nrhs;
  if (!have_graphs) {   // only the cycle graphs are captured again
    for (int b = 0; b < kBanks; ++b) {
      int rc = capture<T>(h, &h->g_cycle[b], h->cyc, b, true, nrhs);
      if (rc) return rc;
      h->g_cycle[b].k = h->k;
      h->g_cycle[b].nrhs = nrhs;
    }
    h->g_cycle_ts = (int)sizeof(T);
  }
  int rc = sync(h);   // the update stream reads the candidate set up above
  if (rc) return rc;
  int iters_before = 0;
  bool slot0_open = true;
  int pend_bank = -1, pend_nit = 0, pend_ns = 0;   // update owed for the last cycle
  auto run_update = [&]() -> int {
    if (pend_bank < 0) return RB_OK;
    const auto t0 = std::chrono::steady_clock::now();
    const int r = cycle_update<T>(h, pend_bank, pend_nit, pend_ns);
    so->ms_update += std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
    so->cycles += 1;
    pend_bank = -1;
    return r;
  };
  for (int c = 0;; ++c) {
    const int bank = c % kBanks;
    RB_CUDA_TRY(cudaGraphLaunch(h->g_cycle[bank].exec, h->us));
    count_launches((long long)h->cyc * passes_per_iter(h));
    if ((rc = run_update())) return rc;   // overlaps cycle c on the GPU
    if ((rc = read_state(h, nrhs))) return rc;
    const IterState& hs = h->hst[0];
    const int nit = hs.iter - iters_before;
    iters_before = hs.iter;
    const bool ok = (hs.status == RB_OK || hs.status == RB_ENOTCONV);
    const bool allowed = (h->o.update_cycles == 0) || (c < h->o.update_cycles);
    if (slot0_open && ok && allowed && nit > 0) {
      pend_bank = bank;
      pend_nit = nit;
      pend_ns = nit - (hs.half ? 1 : 0);
    }
    if (hs.done) slot0_open = false;
    if (hook && (rc = hook())) return rc;
    if (all_done(h, nrhs)) break;
  }
  return run_update();
}

// The final correction of Alg. 2 (x = x - U x_c) and the FP64 true residual of every slot.
int finish_block(rb_ctx* h, int nrhs, SolveOut* so) {
  const int64_t ld = h->npad;
  for (int i = 0; i < nrhs; ++i) {
    if (h->k > 0)
      RB_CUDA_TRY(gemv_update(h->sl[i].x, h->U, ld, h->k, h->st[i].xc, nullptr, -1.0, h->npad, vec_grid(h), h->us));
    RB_CUDA_TRY(residual_norm(h->A.view(), h->sl[i].b, h->sl[i].x, h->tmp, h->npad, h->st + i, h->partials,
                              h->grids.spmv, h->us));
    so[i].mv_check += 1;
  }
  return read_state(h, nrhs);
}

// U_next = Y (promoted to FP64 when the candidate is FP32), U~_next = U_next,
// and the recycle setup for the new space.
template <typename T>
int adopt_candidate(rb_ctx* h, SolveOut* so) {
  const int64_t ld = h->npad;
  const auto t0 = std::chrono::steady_clock::now();
  if (std::is_same<T, float>::value) {
    for (int j = 0; j < h->kY; ++j)
      RB_CUDA_TRY(to_double((const float*)h->Yc + (int64_t)j * ld, h->U + (int64_t)j * ld, ld, h->us));
  } else {
    RB_CUDA_TRY(cudaMemcpyAsync(h->U, h->Yc, sizeof(double) * ld * h->kY, cudaMemcpyDeviceToDevice, h->us));
  }
  {   // unit 2-norm columns (the oracle's normalisation of Y, applied once)
    std::vector<const double*> uc;
    for (int j = 0; j < h->kY; ++j) uc.push_back(h->U + (int64_t)j * ld);
    std::vector<double> N2;
    int rc = block_colnorm2<double>(h, uc, N2);
    if (rc) return rc;
    std::vector<double> f(h->kY);
    for (int j = 0; j < h->kY; ++j) f[j] = N2[j] > 0 ? 1.0 / std::sqrt(N2[j]) : 0.0;
    RB_CUDA_TRY(cudaMemcpy(h->dR, f.data(), sizeof(double) * h->kY, cudaMemcpyHostToDevice));
    RB_CUDA_TRY(scale_cols<double>(h->U, ld, h->kY, h->dR, h->npad, h->us));
  }
  RB_CUDA_TRY(cudaMemcpyAsync(h->Ut, h->U, sizeof(double) * ld * h->kY, cudaMemcpyDeviceToDevice, h->us));
  mark_setup(h, h->kY);   // C, C~ and D_c for the new space: at the next solve
  so->ms_update += std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
  h->update_epoch = h->matrix_epoch;
  return RB_OK;
}

bool update_now(rb_ctx* h) {
  return (h->o.recycle_mode == RB_RECYCLE_UPDATE_ALL) ||
         (h->o.recycle_mode == RB_RECYCLE_UPDATE_FIRST && h->update_epoch != h->matrix_epoch);
}

int solve_fp64(rb_ctx* h, int nrhs, const bool* x_nonzero, SolveOut* so) {
  double* rhs[kMaxRhs];
  double* xb[kMaxRhs];
  double tol[kMaxRhs];
  bool skip[kMaxRhs] = {false, false, false, false};
  for (int i = 0; i < nrhs; ++i) {
    rhs[i] = h->sl[i].b;
    xb[i] = h->sl[i].x;
    tol[i] = h->o.tol;
  }
  int rc = setup_block(h, nrhs, rhs, xb, x_nonzero, skip, tol, so);
  if (rc) return rc;
  const bool upd = update_now(h);
  if (!all_done(h, nrhs)) {
    if ((rc = init_p<double>(h, nrhs, upd))) return rc;
    rc = upd ? iterate_cycles<double>(h, nrhs, so) : iterate_plain<double>(h, nrhs);
    if (rc) return rc;
  }
  rc = finish_block(h, nrhs, so);
  if (rc) return rc;
  for (int i = 0; i < nrhs; ++i) {
    const IterState& hs = h->hst[i];
    so[i].status = hs.status;
    so[i].iters = hs.iter;
    so[i].mv += 2 * (int64_t)hs.iter - (hs.half ? 1 : 0);
    so[i].relres_rec = hs.bnorm2 > 0 ? std::sqrt(hs.rnorm2 / hs.bnorm2) : 0.0;
    so[i].relres_true = hs.bnorm2 > 0 ? std::sqrt(hs.red[0] / hs.bnorm2) : 0.0;
    so[i].bytes = (double)hs.iter * iter_bytes(h, h->k, 8, 8, nrhs);
  }
  if (upd && (h->hst[0].status == RB_OK || h->hst[0].status == RB_ENOTCONV) && h->kY > 0) {
    rc = adopt_candidate<double>(h, so);
    if (rc) return rc;
  }
  return RB_OK;
}

// Mixed precision: an FP32 inner RBiCGSTAB (FP32 vectors, FP32 SpMV and FP32
// recycle blocks, FP64-class dot products and FP64 scalars) with FP64
// residual replacement ("reliable updates", Sleijpen and van der Vorst,
// Computing 56, 1996).  The FP64 iterate x takes the FP32 correction
// d = x_inner - U x_c (the final correction of the inner solve) whenever the
// recursive FP32 residual has fallen by kReplace below the larger of the last
// true residual and its own peak since then (the rounding of the increment
// grows with the peak), or reports convergence; the true residual b - A x is
// then formed in FP64 and, unless it meets the target, replaces the recursive
// one while the search direction and the scalars carry on.  So one Krylov
// process serves the whole solve.  A half-step exit whose true residual misses
// the target, and a fold that would raise the true residual (the FP32 process
// diverged: an ill-conditioned system at the FP32 accuracy floor), restart the
// inner solve from the current x (a refinement step; the latter fold is
// undone).  After kStallSwitch undone folds in a row, a breakdown or an FP32
// overflow the slot is finished in FP64 from x.  The target is a tenth of the
// tolerance, so the answer carries a forward error comparable to the FP64
// solver's.
constexpr double kReplace = 1e-2;
constexpr int kStallSwitch = 2;   // folds undone in a row before the FP64 finish

int solve_mixed(rb_ctx* h, int nrhs, SolveOut* so) {
  const int64_t ld = h->npad;
  const int max_rounds = 12;
  const int max_itn = h->o.max_itn > 0 ? h->o.max_itn : (int)std::min<int64_t>(h->n, 20000);
  double bn2[kMaxRhs], target[kMaxRhs], rn[kMaxRhs], rlast[kMaxRhs];
  bool stop[kMaxRhs], running[kMaxRhs], to64[kMaxRhs] = {false, false, false, false};
  int stalls[kMaxRhs] = {0, 0, 0, 0};
  int total_it[kMaxRhs], last_status[kMaxRhs];
  double rmax_reset[kMaxRhs];   // host source of the device peak's reset after a replacement
  for (int i = 0; i < nrhs; ++i) {
    bn2[i] = h->hst[i].red[0];
    target[i] = 0.1 * h->o.tol * std::sqrt(bn2[i]);
    rn[i] = rlast[i] = 0.0;
    stop[i] = running[i] = false;
    total_it[i] = 0;
    last_status[i] = RB_OK;
    so[i].outer = 0;
  }
  const bool upd = update_now(h);
  bool did_update = false;

  // x += fx - U x_c for slot i, then fx = 0 and x_c = 0.
  auto fold = [&](int i) -> int {
    RB_CUDA_TRY(add_float_to_double(h->sl[i].x, h->sl[i].fx, ld, h->us));
    if (h->k > 0) {
      RB_CUDA_TRY(gemv_update(h->sl[i].x, h->U, ld, h->k, h->st[i].xc, nullptr, -1.0, h->npad, vec_grid(h), h->us));
      RB_CUDA_TRY(cudaMemsetAsync(h->st[i].xc, 0, sizeof(double) * h->k, h->us));
    }
    RB_CUDA_TRY(cudaMemsetAsync(h->sl[i].fx, 0, sizeof(float) * ld, h->us));
    return RB_OK;
  };
  // Drop slot i's inner increment (fx = 0, x_c = 0): x keeps its last fold.
  auto drop = [&](int i) -> int {
    if (h->k > 0) RB_CUDA_TRY(cudaMemsetAsync(h->st[i].xc, 0, sizeof(double) * h->k, h->us));
    RB_CUDA_TRY(cudaMemsetAsync(h->sl[i].fx, 0, sizeof(float) * ld, h->us));
    return RB_OK;
  };
  // True residual of slot i into sl[i].rin and rn[i].
  auto true_residual = [&](int i) -> int {
    RB_CUDA_TRY(residual_norm(h->A.view(), h->sl[i].b, h->sl[i].x, h->sl[i].rin, h->npad, h->st + i, h->partials,
                              h->grids.spmv, h->us));
    RB_CUDA_TRY(cudaMemcpyAsync(&h->hst[i].red[0], &h->st[i].red[0], sizeof(double), cudaMemcpyDeviceToHost,
                                h->us));
    int rc = sync(h);
    if (rc) return rc;
    rn[i] = std::sqrt(h->hst[i].red[0]);
    so[i].mv_check += 1;
    return RB_OK;
  };
  // After each graph replay: residual replacement / convergence per slot.
  // In update mode slot 0's search direction lives in the cycle store at a
  // position fixed by the cycle graph, so a slot 0 that stopped inside a
  // cycle is not resumed there: its true residual is checked at the end of
  // the outer (refinement) step and, if needed, the next outer step restarts it.
  const bool trace = getenv("RB_TRACE") != nullptr;
  bool cycles_running = false;
  PollHook hook = [&]() -> int {
    for (int i = 0; i < nrhs; ++i) {
      if (!running[i]) continue;
      const IterState& hs = h->hst[i];
      if (trace)
        fprintf(stderr, "rb_trace slot %d iter %d rn2 %.3e rlast %.3e done %d half %d status %d\n", i, hs.iter,
                hs.rnorm2, rlast[i], hs.done, hs.half, hs.status);
      const bool conv_rec = hs.done && hs.status == RB_OK && !hs.half && !(cycles_running && i == 0);
      const double peak2 = std::max(hs.rmax2, rlast[i] * rlast[i]);
      const bool due = !hs.done && hs.rnorm2 <= kReplace * kReplace * peak2;
      if (!conv_rec && !due) continue;
      PhaseClock pr;
      // the previous x waits in xin (unused while the inner solve runs)
      // until the fold is accepted
      RB_CUDA_TRY(cudaMemcpyAsync(h->sl[i].xin, h->sl[i].x, sizeof(double) * ld, cudaMemcpyDeviceToDevice, h->us));
      int rc = fold(i);
      if (!rc) rc = true_residual(i);
      if (rc) return rc;
      so[i].outer += 1;
      if (trace) fprintf(stderr, "rb_trace slot %d replace: true residual %.6e target %.3e\n", i, rn[i], target[i]);
      // A fold that raised the true residual (or made it non-finite): the
      // FP32 process diverged after an earlier replacement, which is where
      // an ill-conditioned system meets the FP32 accuracy floor (about u_32
      // times its condition number).  The fold is undone, the slot restarts
      // from x in the next round, and after kStallSwitch such folds in a row
      // it is finished in FP64 instead.
      if (!std::isfinite(rn[i]) || rn[i] > rlast[i]) {
        RB_CUDA_TRY(cudaMemcpyAsync(h->sl[i].x, h->sl[i].xin, sizeof(double) * ld, cudaMemcpyDeviceToDevice, h->us));
        rn[i] = rlast[i];
        if (!hs.done) RB_CUDA_TRY(cudaMemcpyAsync(&h->st[i].done, &kOne, sizeof(int), cudaMemcpyHostToDevice, h->us));
        h->hst[i].done = 1;
        running[i] = false;
        if (++stalls[i] >= kStallSwitch) {
          stop[i] = true;
          to64[i] = true;
        }
        if (trace) fprintf(stderr, "rb_trace slot %d fold undone (%d in a row)\n", i, stalls[i]);
        continue;
      }
      stalls[i] = 0;
      if (rn[i] <= target[i]) {
        if (!hs.done) RB_CUDA_TRY(cudaMemcpyAsync(&h->st[i].done, &kOne, sizeof(int), cudaMemcpyHostToDevice, h->us));
        h->hst[i].done = 1;
        running[i] = false;
        stop[i] = true;
        so[i].status = RB_OK;
        continue;
      }
      // replace the recursive residual and carry on.  The true residual is
      // projected first (eq. (3.5): x += U C-hat^T r, r -= C C-hat^T r): the
      // rounding of the FP32 iterate leaves a component along range(C) that
      // the projected iteration could never reduce.
      if (h->k > 0) {
        DotArgs d{};
        d.M = h->Chat; d.ld = ld; d.km = h->k; d.v = h->sl[i].rin; d.nd = 0;
        RB_CUDA_TRY(dots(d, h->npad, h->st + i, h->partials, vec_grid(h), h->us));
        RB_CUDA_TRY(gemv_update(h->sl[i].x, h->U, ld, h->k, h->st[i].red, nullptr, 1.0, h->npad, vec_grid(h), h->us));
        RB_CUDA_TRY(gemv_update(h->sl[i].rin, h->C, ld, h->k, h->st[i].red, nullptr, -1.0, h->npad, vec_grid(h),
                                h->us));
      }
      RB_CUDA_TRY(to_float(h->sl[i].rin, h->sl[i].fr, ld, h->us));
      if (hs.done) RB_CUDA_TRY(cudaMemcpyAsync(&h->st[i].done, &kZero, sizeof(int), cudaMemcpyHostToDevice, h->us));
      h->hst[i].done = 0;
      rlast[i] = rn[i];
      rmax_reset[i] = rn[i] * rn[i];   // the peak restarts from the replaced residual
      RB_CUDA_TRY(cudaMemcpyAsync(&h->st[i].rmax2, &rmax_reset[i], sizeof(double), cudaMemcpyHostToDevice, h->us));
      pr.lap("replace");
    }
    return sync(h);
  };

  PhaseClock pcs;
  for (int round = 0;; ++round) {
    bool any = false;
    bool skip[kMaxRhs] = {true, true, true, true};
    bool xnz[kMaxRhs] = {false, false, false, false};
    double* rhs[kMaxRhs];
    double* xb[kMaxRhs];
    double tol_in[kMaxRhs];
    for (int i = 0; i < nrhs; ++i) {
      rhs[i] = h->sl[i].rin;
      xb[i] = h->sl[i].xin;
      tol_in[i] = 1.0;
      if (stop[i]) continue;
      int rc = true_residual(i);
      if (rc) return rc;
      if (!std::isfinite(rn[i])) {
        so[i].status = RB_ENONFINITE;
        stop[i] = true;
      } else if (rn[i] <= target[i] || bn2[i] == 0.0) {
        so[i].status = RB_OK;
        stop[i] = true;
      } else if (total_it[i] >= max_itn) {
        so[i].status = last_status[i] != RB_OK ? last_status[i] : RB_ENOTCONV;
        stop[i] = true;
      } else if (round >= max_rounds) {   // FP32 rounds used up: finish in FP64
        stop[i] = true;
        to64[i] = true;
      } else {
        // inner system A d = r, converged when ||r - A d|| <= target
        skip[i] = false;
        any = true;
        tol_in[i] = target[i] / rn[i];
      }
    }
    if (!any) break;
    for (int i = 0; i < nrhs; ++i) {
      running[i] = !skip[i];
      if (skip[i]) continue;
      RB_CUDA_TRY(cudaMemcpyAsync(&h->st[i].bnorm2, &h->st[i].red[0], sizeof(double), cudaMemcpyDeviceToDevice,
                                  h->us));
      RB_CUDA_TRY(cudaMemsetAsync(h->sl[i].xin, 0, sizeof(double) * ld, h->us));
      rlast[i] = rn[i];
    }
    int rc = setup_block(h, nrhs, rhs, xb, xnz, skip, tol_in, so);
    if (rc) return rc;
    RB_CUDA_TRY(to_float(h->rt0, h->frt0, ld, h->us));
    for (int i = 0; i < nrhs; ++i) {
      if (skip[i]) continue;
      // r_0 and the initial projection x_0 = U C-hat^T r of the inner solve
      RB_CUDA_TRY(to_float(h->sl[i].r, h->sl[i].fr, ld, h->us));
      RB_CUDA_TRY(to_float(h->sl[i].xin, h->sl[i].fx, ld, h->us));
    }
    const bool cyc_now = upd && !did_update && !skip[0];
    cycles_running = cyc_now;
    pcs.lap("blk_setup");
    if (!all_done(h, nrhs)) {
      if ((rc = init_p<float>(h, nrhs, cyc_now))) return rc;
      if (cyc_now) {
        // the first (longest) inner solve collects the cycles of the update
        rc = iterate_cycles<float>(h, nrhs, so, hook);
        did_update = true;
      } else {
        rc = iterate_plain<float>(h, nrhs, hook);
      }
      if (rc) return rc;
    }
    pcs.lap("blk_iterate");
    for (int i = 0; i < nrhs; ++i) {
      if (skip[i]) continue;
      const IterState& hs = h->hst[i];
      total_it[i] += hs.iter;
      so[i].mv += 2 * (int64_t)hs.iter - (hs.half ? 1 : 0);
      last_status[i] = hs.status;
      if (stop[i]) continue;   // converged at a replacement (x already folded)
      running[i] = false;
      // max_itn or a half-step exit: fold the correction and let the next
      // outer (refinement) step restart from x.  A breakdown folds too and
      // a non-finite inner iterate (an FP32 overflow) is dropped (x keeps
      // its last fold); either hands the slot to the FP64 finish.
      if (hs.status == RB_ENONFINITE) {
        if ((rc = drop(i))) return rc;
      } else {
        if ((rc = fold(i))) return rc;
      }
      if (hs.status != RB_OK && hs.status != RB_ENOTCONV) {
        to64[i] = true;
        stop[i] = true;
      }
    }
    rc = sync(h);
    if (rc) return rc;
  }
  // FP64 finish of the slots whose FP32 iteration stalled, broke down or
  // overflowed: Alg. 2 in FP64 from the current x, with the same recycle
  // space, to the mixed target on the recursive residual; a true residual
  // still above the tolerance after it (the recursive residual drifts from
  // the true one over a long run) takes another FP64 round from x.
  for (int round64 = 0; round64 < 3; ++round64) {
    bool any64 = false;
    for (int i = 0; i < nrhs; ++i) any64 = any64 || to64[i];
    if (!any64) break;
    bool skip64[kMaxRhs] = {true, true, true, true};
    bool xnz64[kMaxRhs] = {false, false, false, false};
    double* rhs64[kMaxRhs];
    double* xb64[kMaxRhs];
    double tol64[kMaxRhs];
    for (int i = 0; i < nrhs; ++i) {
      rhs64[i] = h->sl[i].b;
      xb64[i] = h->sl[i].x;
      tol64[i] = 0.1 * h->o.tol;
      if (!to64[i]) continue;
      skip64[i] = false;
      xnz64[i] = true;
      RB_CUDA_TRY(cudaMemcpyAsync(&h->st[i].bnorm2, &bn2[i], sizeof(double), cudaMemcpyHostToDevice, h->us));
    }
    int rc = sync(h);
    if (!rc) rc = setup_block(h, nrhs, rhs64, xb64, xnz64, skip64, tol64, so);
    if (rc) return rc;
    if (!all_done(h, nrhs)) {
      if ((rc = init_p<double>(h, nrhs, false))) return rc;
      if ((rc = iterate_plain<double>(h, nrhs))) return rc;
    }
    for (int i = 0; i < nrhs; ++i) {
      if (!to64[i]) continue;
      if (h->k > 0)
        RB_CUDA_TRY(gemv_update(h->sl[i].x, h->U, ld, h->k, h->st[i].xc, nullptr, -1.0, h->npad, vec_grid(h), h->us));
      RB_CUDA_TRY(residual_norm(h->A.view(), h->sl[i].b, h->sl[i].x, h->tmp, h->npad, h->st + i, h->partials,
                                h->grids.spmv, h->us));
      so[i].mv_check += 1;
    }
    if ((rc = read_state(h, nrhs))) return rc;
    for (int i = 0; i < nrhs; ++i) {
      if (!to64[i]) continue;
      const IterState& hs = h->hst[i];
      total_it[i] += hs.iter;
      so[i].mv += 2 * (int64_t)hs.iter - (hs.half ? 1 : 0);
      so[i].outer += 1;
      so[i].status = hs.status;
      rn[i] = std::sqrt(hs.red[0]);
      // done unless the true residual misses the tolerance with iterations left
      to64[i] = hs.status == RB_OK && rn[i] > h->o.tol * std::sqrt(bn2[i]) && total_it[i] < max_itn;
    }
    pcs.lap("blk_fp64_finish");
  }
  for (int i = 0; i < nrhs; ++i)
    if (to64[i]) so[i].status = RB_ENOTCONV;   // three FP64 rounds did not meet the tolerance
  for (int i = 0; i < nrhs; ++i) {
    so[i].iters = total_it[i];
    so[i].relres_true = bn2[i] > 0 ? rn[i] / std::sqrt(bn2[i]) : 0.0;
    so[i].relres_rec = so[i].relres_true;
    so[i].bytes = (double)total_it[i] * iter_bytes(h, h->k, 4, 4, nrhs);
  }
  if (did_update && h->kY > 0 && (so[0].status == RB_OK || so[0].status == RB_ENOTCONV)) {
    int rc = adopt_candidate<float>(h, so);
    if (rc) return rc;
  }
  pcs.lap("blk_adopt");
  return sync(h);
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
  if (cudaStreamCreateWithFlags(&h->ws, cudaStreamNonBlocking) != cudaSuccess) return fail(RB_ECUDA);
  h->st = dalloc<IterState>(kMaxRhs, &err);
  if (!h->st) return fail(err);
  if (cudaMemset(h->st, 0, sizeof(IterState) * kMaxRhs) != cudaSuccess) return fail(RB_ECUDA);
  if (cudaMallocHost(&h->hst, sizeof(IterState) * kMaxRhs) != cudaSuccess) return fail(RB_ENOMEM);
  std::memset(h->hst, 0, sizeof(IterState) * kMaxRhs);
  h->dflag = dalloc<int>(1, &err);
  if (!h->dflag) return fail(err);
  h->tcerr = dalloc<int>(1, &err);
  if (!h->tcerr) return fail(err);
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
  if (h->ws) cudaStreamSynchronize(h->ws);
  reset_graphs(h);
  release_a32(h);
  sell_free(&h->A);
  sell_free(&h->AT);
  for (int i = 0; i < h->nslots; ++i) free_slot(h->sl[i]);
  void* ptrs[] = {h->rp, h->ci, h->cv, h->trp, h->tci, h->tsrc, h->tcv, h->U, h->Ut, h->C, h->Ct,
                  h->Chat, h->T1, h->T2, h->Dinv, h->rt0, h->tmp, h->tmp2, h->frt0, h->fU, h->fC, h->fChat,
                  h->st, h->partials, h->dflag, h->tcerr, h->lvec, h->cstore, h->Yc, h->AYc, h->Yn, h->AYn, h->gwork, h->dG,
                  h->dR, (void*)h->dptr};
  for (void* p : ptrs) cudaFree(p);
  if (h->hst) cudaFreeHost(h->hst);
  if (h->cs) cudaStreamDestroy(h->cs);
  if (h->ws) cudaStreamDestroy(h->ws);
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
    h->A32.offs = h->A.offs;
    h->A32.offs_stride = h->A.offs_stride;
    h->A32.stencil_slices = h->A.stencil_slices;
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
  // keep U, U~; C, C~, D_c for the new matrix are recomputed by the next solve
  const int kin = h->setup_pending >= 0 ? h->setup_pending : h->k;
  if (kin > 0) mark_setup(h, kin);
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
  const int kin = h->setup_pending >= 0 ? h->setup_pending : h->k;
  if (kin > 0) mark_setup(h, kin);
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
    int f[2] = {0, 0};
    double* blocks[2] = {h->U, h->Ut};
    for (int q = 0; q < 2; ++q) {
      RB_CUDA_TRY(check_finite(blocks[q], npad * k, h->dflag, h->us));
      RB_CUDA_TRY(cudaMemcpyAsync(&f[q], h->dflag, sizeof(int), cudaMemcpyDeviceToHost, h->us));
      rc = sync(h);
      if (rc) return rc;
    }
    if (f[0] || f[1]) {
      h->k = 0;
      reset_graphs(h);
      return RB_ENONFINITE;
    }
  }
  int64_t mv = 0;
  h->setup_pending = -1;
  return recycle_setup(h, k, &mv);
}

extern "C" int rbicgstab_get_recycle(rb_handle h, int32_t* k, double* U, double* Ut, int64_t ld, int where) {
  if (!h || !k || (where != RB_HOST && where != RB_DEVICE)) return RB_EINVAL;
  const int kk = h->setup_pending >= 0 ? h->setup_pending : h->k;
  *k = kk;
  if (kk == 0) return RB_OK;
  if ((U || Ut) && ld < h->n) return RB_EINVAL;
  for (int j = 0; j < kk; ++j) {
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
  RB_CUDA_TRY(spmv<double>(transpose ? h->AT.view() : h->A.view(), h->tmp, h->tmp2, 1.0, 0.0,
                           h->grids.spmv, h->us));
  rc = copy_out(y, h->tmp2, sizeof(double) * h->n, where, h->us);
  if (rc) return rc;
  return sync(h);
}

extern "C" int rbicgstab_pattern_outer(rb_handle h, const double* u, const double* v, double scale, double* out,
                                       int where) {
  if (!h || !u || !v || !out || where != RB_DEVICE || !std::isfinite(scale)) return RB_EINVAL;
  if (!h->have_matrix) return RB_EDIM;
  RB_CUDA_TRY(pattern_outer(h->n, h->rp, h->ci, u, v, scale, out, vec_grid(h), h->us));
  return sync(h);
}

extern "C" int rbicgstab_update_gram(int64_t n, int64_t ld, int32_t ky, int32_t nit, int32_t ns, int32_t kcap,
                                     int32_t scap, const float* Y, const float* AY, const float* P,
                                     const float* AP, const float* S, const float* AS, double* G, double* H,
                                     int32_t path, void* cuda_stream, double* ms_kernel) {
  using namespace rb;
  const int m = ky + nit + ns;
  if (n <= 0 || ld < n || ld % 4 != 0 || ky < 0 || nit < 0 || ns < 0 || m <= 0 || ky > kcap || nit > scap ||
      ns > scap || !G || !H || path < RB_GRAM_AUTO || path > RB_GRAM_TENSOR)
    return RB_EINVAL;
  if (m > kMaxGram) return RB_EINVAL;
  const float* src[6] = {AY, AP, AS, Y, P, S};
  const int cols[3] = {ky, nit, ns};
  for (int b = 0; b < 6; ++b)
    if (cols[b % 3] > 0 && !src[b]) return RB_EINVAL;
  cudaStream_t s = (cudaStream_t)cuda_stream;
  const int cap[6] = {kcap, scap, scap, kcap, scap, scap};
  const bool tc = path == RB_GRAM_TENSOR || (path == RB_GRAM_AUTO && gram_tc_eligible(cap));
  if (path == RB_GRAM_TENSOR && !gram_tc_eligible(cap)) return RB_EINVAL;
  int dev = 0, nsm = 0;
  RB_CUDA_TRY(cudaGetDevice(&dev));
  RB_CUDA_TRY(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
  int err = 0;
  double* dGH = dalloc<double>(2 * (int64_t)m * m, &err);
  if (!dGH) return err;
  cudaEvent_t ev0 = nullptr, ev1 = nullptr;
  if (ms_kernel && (cudaEventCreate(&ev0) != cudaSuccess || cudaEventCreate(&ev1) != cudaSuccess)) {
    if (ev0) cudaEventDestroy(ev0);
    cudaFree(dGH);
    return RB_ECUDA;
  }
  int rc = RB_OK;
  void* work = nullptr;
  int* derr = nullptr;
  const float** dptr = nullptr;
  if (tc) {
    GramTcBlocks blk;
    for (int b = 0; b < 6; ++b) {
      blk.ptr[b] = src[b];
      blk.cols[b] = cols[b % 3];
      blk.cap[b] = cap[b];
    }
    const size_t wf = gram_tc_work_floats(cap, nsm);
    if (cudaMalloc(&work, sizeof(float) * wf) != cudaSuccess || cudaMalloc(&derr, sizeof(int)) != cudaSuccess ||
        cudaMemsetAsync(derr, 0, sizeof(int), s) != cudaSuccess) {
      rc = RB_ENOMEM;
    } else {
      if (ev0) cudaEventRecord(ev0, s);
      rc = gram_tc(blk, n, ld, dGH, dGH + (size_t)m * m, (float*)work, derr, nsm, s);
      if (ev1) cudaEventRecord(ev1, s);
      int herr = 0;
      if (rc == RB_OK && (cudaMemcpyAsync(&herr, derr, sizeof(int), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
                          cudaStreamSynchronize(s) != cudaSuccess))
        rc = RB_ECUDA;
      if (rc == RB_OK && herr) rc = RB_ETIMEOUT;
    }
  } else {
    std::vector<const float*> Z, W;
    for (int b = 0; b < 3; ++b)
      for (int j = 0; j < cols[b]; ++j) {
        Z.push_back(src[b] + (int64_t)j * ld);
        W.push_back(src[3 + b] + (int64_t)j * ld);
      }
    const int grid = 2 * nsm;
    if (cudaMalloc(&work, sizeof(double) * (size_t)grid * gram_gh_work(m)) != cudaSuccess ||
        cudaMalloc((void**)&dptr, sizeof(float*) * 2 * m) != cudaSuccess) {
      rc = RB_ENOMEM;
    } else if (cudaMemcpyAsync(dptr, Z.data(), sizeof(float*) * m, cudaMemcpyHostToDevice, s) != cudaSuccess ||
               cudaMemcpyAsync(dptr + m, W.data(), sizeof(float*) * m, cudaMemcpyHostToDevice, s) != cudaSuccess) {
      rc = RB_ECUDA;
    } else {
      if (ev0) cudaEventRecord(ev0, s);
      if (gram_gh<float>(dptr, dptr + m, m, ld, dGH, dGH + (size_t)m * m, (double*)work, grid, s) != cudaSuccess)
        rc = RB_ECUDA;
      if (ev1) cudaEventRecord(ev1, s);
    }
  }
  if (rc == RB_OK && ms_kernel) {
    float ms = 0.f;
    if (cudaEventSynchronize(ev1) != cudaSuccess || cudaEventElapsedTime(&ms, ev0, ev1) != cudaSuccess) rc = RB_ECUDA;
    *ms_kernel = ms;
  }
  if (ev0) cudaEventDestroy(ev0);
  if (ev1) cudaEventDestroy(ev1);
  if (rc == RB_OK &&
      (cudaMemcpyAsync(G, dGH, sizeof(double) * m * m, cudaMemcpyDeviceToHost, s) != cudaSuccess ||
       cudaMemcpyAsync(H, dGH + (size_t)m * m, sizeof(double) * m * m, cudaMemcpyDeviceToHost, s) != cudaSuccess ||
       cudaStreamSynchronize(s) != cudaSuccess))
    rc = RB_ECUDA;
  cudaStreamSynchronize(s);
  cudaFree(dGH);
  cudaFree(work);
  cudaFree(derr);
  cudaFree((void*)dptr);
  return rc;
}

extern "C" int rbicgstab_sell_stats(rb_handle h, int64_t* nslices, int64_t* stencil_slices) {
  if (!h || !nslices || !stencil_slices) return RB_EINVAL;
  if (!h->have_matrix) return RB_EDIM;
  *nslices = h->A.nslices;
  *stencil_slices = h->A.stencil_slices;
  return RB_OK;
}

extern "C" int rbicgstab_svd_small(int32_t k, const double* M, double* P, double* sigma, double* Q) {
  if (k < 1 || k > 256 || !M || !P || !sigma || !Q) return RB_EINVAL;
  for (int64_t i = 0; i < (int64_t)k * k; ++i)
    if (!std::isfinite(M[i])) return RB_ENONFINITE;
  rb::svd_small(k, M, P, sigma, Q);
  return RB_OK;
}

extern "C" int rbicgstab_harmonic_ritz(int32_t m, const double* G, const double* H, int32_t k, double* Y,
                                       double* theta_re, double* theta_im, int32_t* k_used) {
  if (m <= 0 || k <= 0 || k > m || !G || !H || !Y || !k_used) return RB_EINVAL;
  const int r = rb::harmonic_ritz(m, G, H, k, kRankTol, Y, theta_re, theta_im);
  if (r < 0) return RB_ENOTCONV;
  *k_used = r;
  return RB_OK;
}

extern "C" int rbicgstab_solve_block(rb_handle h, int32_t nrhs, const double* B, double* X, int64_t ld,
                                     int where, rb_stats* st_out) {
  if (!h || !B || !X || nrhs < 1 || nrhs > kMaxRhs || (where != RB_HOST && where != RB_DEVICE)) return RB_EINVAL;
  if (!h->have_matrix) return RB_EDIM;
  if (nrhs > 1 && ld < h->n) return RB_EINVAL;
  int rc = ensure_slots(h, nrhs);
  if (rc) return rc;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  auto done = [&](int code) {
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    return code;
  };
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) return done(RB_ECUDA);
  if (cudaEventRecord(e0, h->us) != cudaSuccess) return done(RB_ECUDA);
  SolveOut so[kMaxRhs];
  bool x_nonzero[kMaxRhs] = {false, false, false, false};
  for (int i = 0; i < nrhs; ++i) {
    Slot& s = h->sl[i];
    rc = copy_in(s.b, B + (int64_t)i * ld, sizeof(double) * h->n, where, h->us);
    if (!rc) rc = copy_in(s.x, X + (int64_t)i * ld, sizeof(double) * h->n, where, h->us);
    if (rc) return done(rc);
    // finiteness of b and x, ||b||^2, ||x||^2
    int fb = 0, fx = 0;
    if (check_finite(s.b, h->n, h->dflag, h->us) != cudaSuccess ||
        cudaMemcpyAsync(&fb, h->dflag, sizeof(int), cudaMemcpyDeviceToHost, h->us) != cudaSuccess)
      return done(RB_ECUDA);
    if ((rc = sync(h))) return done(rc);
    if (check_finite(s.x, h->n, h->dflag, h->us) != cudaSuccess ||
        cudaMemcpyAsync(&fx, h->dflag, sizeof(int), cudaMemcpyDeviceToHost, h->us) != cudaSuccess)
      return done(RB_ECUDA);
    DotArgs d{};
    d.nd = 2;
    d.a[0] = s.b; d.b[0] = s.b;
    d.a[1] = s.x; d.b[1] = s.x;
    double nb[2];
    if ((rc = run_dots(h, d, nb, 2, i))) return done(rc);
    if (fb || fx) return done(RB_ENONFINITE);
    if (cudaMemcpyAsync(&h->st[i].bnorm2, &h->st[i].red[0], sizeof(double), cudaMemcpyDeviceToDevice, h->us) !=
        cudaSuccess)
      return done(RB_ECUDA);
    x_nonzero[i] = nb[1] != 0.0;
    h->hst[i].red[0] = nb[0];
  }
  {
    int64_t mv = 0;
    if ((rc = ensure_setup(h, &mv)) < 0) return done(rc);
    so[0].mv_setup += mv;
  }
  rc = (h->o.precision == RB_MIXED) ? solve_mixed(h, nrhs, so) : solve_fp64(h, nrhs, x_nonzero, so);
  if (rc < 0 && rc != RB_ENOTCONV) return done(rc);
  for (int i = 0; i < nrhs; ++i) {
    rc = copy_out(X + (int64_t)i * ld, h->sl[i].x, sizeof(double) * h->n, where, h->us);
    if (rc) return done(rc);
  }
  cudaEventRecord(e1, h->us);
  if ((rc = sync(h))) return done(rc);
  float ms = 0;
  cudaEventElapsedTime(&ms, e0, e1);
  int worst = RB_OK;
  for (int i = 0; i < nrhs; ++i) {
    if (so[i].status != RB_OK && worst == RB_OK) worst = so[i].status;
    if (!st_out) continue;
    rb_stats& o = st_out[i];
    o.iters = so[i].iters;
    o.status = so[i].status;
    o.k_used = h->k;
    o.seeds_used = so[i].seeds;
    o.matvecs = so[i].mv;
    o.matvecs_setup = so[0].mv_setup;
    o.matvecs_check = so[i].mv_check;
    o.cycles = so[0].cycles;
    o.outer = so[i].outer;
    o.relres_rec = so[i].relres_rec;
    o.relres_true = so[i].relres_true;
    o.ms_total = ms;
    o.bytes_model = so[i].bytes;
    o.ms_update = so[0].ms_update;
  }
  return done(worst);
}

// ============================================================ RBiCG (Alg. 1)
namespace {

// Eq. (3.5) for the dual system: r~_{-1} = b~ - A^T x~_{-1} (x~_{-1} in s.x),
// x~_0 = x~_{-1} + U~ C-check^T r~_{-1}, r~_0 = r~_{-1} - C~ C-check^T r~_{-1}.
// In the basis the setup keeps, C~ C-check^T = C-hat C^T and U~ C-check^T =
// (U~ Mpt) C^T; T2 holds U~ Mpt.  Slot 1 holds the dual system.
int bicg_dual_start(rb_ctx* h) {
  Slot& d = h->sl[1];
  const int64_t ld = h->npad;
  RB_CUDA_TRY(residual_norm(h->AT.view(), d.b, d.x, d.r, h->npad, h->st + 1, h->partials, h->grids.spmv, h->us));
  if (h->k > 0) {
    DotArgs da{};
    da.M = h->C; da.ld = ld; da.km = h->k; da.v = d.r; da.nd = 0;
    RB_CUDA_TRY(dots(da, h->npad, h->st + 1, h->partials, vec_grid(h), h->us));
    RB_CUDA_TRY(gemv_update(d.x, h->T2, ld, h->k, h->st[1].red, nullptr, 1.0, h->npad, vec_grid(h), h->us));
    RB_CUDA_TRY(gemv_update(d.r, h->Chat, ld, h->k, h->st[1].red, nullptr, -1.0, h->npad, vec_grid(h), h->us));
  }
  return RB_OK;
}

BiArgs bicg_args(rb_ctx* h) {
  Slot &p = h->sl[0], &d = h->sl[1];
  BiArgs a{};
  a.npad = h->npad;
  a.x = p.x; a.r = p.r; a.p = p.p; a.q = p.qraw;
  a.xt = d.x; a.rt = d.r; a.pt = d.p; a.qt = d.qraw;
  a.st = h->st;
  a.partials = h->partials;
  return a;
}

// One iteration of Alg. 1 on stream s, composed of the library's kernels:
//   z = A p, zeta = C-hat^T z        (the FP64 SpMV + projection pass, state st[0])
//   z~ = A^T p~, C^T z~              (the same pass on A^T and C, state st[1])
//   q = z - C zeta, q~ = z~ - C-hat C^T z~   (in place over z, z~) and (p~, q)
//   alpha, zeta_c, zeta~_c; x, x~, r, r~, ||r||, ||r~||, beta; p, p~
cudaError_t bicg_iteration(rb_ctx* h, const Grids& g13, int grid, cudaStream_t s) {
  Slot &P = h->sl[0], &D = h->sl[1];
  const int64_t ld = h->npad;
  const int k = h->k;
  cudaError_t e;
  if (k == 0) {
    if ((e = spmv<double>(h->A.view(), P.p, P.qraw, 1.0, 0.0, h->grids.spmv, s)) != cudaSuccess) return e;
    if ((e = spmv<double>(h->AT.view(), D.p, D.qraw, 1.0, 0.0, h->grids.spmv, s)) != cudaSuccess) return e;
  } else {
    IterArgs<double> ap{};
    ap.A = h->A.view();
    ap.Chat = h->Chat;
    ap.ld = ld;
    ap.s[0] = P.p;
    ap.traw[0] = P.qraw;
    ap.st = h->st;
    ap.partials = h->partials;
    ap.npad = h->npad;
    ap.nrhs = 1;
    IterArgs<double> ad = ap;
    ad.A = h->AT.view();
    ad.Chat = h->C;
    ad.s[0] = D.p;
    ad.traw[0] = D.qraw;
    ad.st = h->st + 1;
    if ((e = launch_pass<double>(P3, ap, k, g13, s)) != cudaSuccess) return e;
    if ((e = launch_pass<double>(P3, ad, k, g13, s)) != cudaSuccess) return e;
    if ((e = bicg_project(bicg_args(h), h->C, h->Chat, ld, h->Dinv, grid, s)) != cudaSuccess) return e;
  }
  if (k == 0) {
    DotArgs d{};
    d.nd = 1;
    d.a[0] = D.p; d.b[0] = P.qraw;
    if ((e = dots(d, h->npad, h->st, h->partials, vec_grid(h), s)) != cudaSuccess) return e;
  }
  if ((e = bicg_alpha(h->st, h->Dinv, s)) != cudaSuccess) return e;
  return bicg_update(bicg_args(h), grid, s);
}

int capture_bicg(rb_ctx* h) {
  GraphSlot* g = &h->g_bicg;
  if (g->exec) cudaGraphExecDestroy(g->exec);
  g->exec = nullptr;
  g->valid = false;
  Grids g13;
  iteration_grids<double>(h->k, h->nsm, h->npad, &g13, 1);
  const int grid = bicg_grid(h->nsm, h->npad);
  cudaGraph_t graph = nullptr;
  RB_CUDA_TRY(cudaStreamBeginCapture(h->cs, cudaStreamCaptureModeThreadLocal));
  cudaError_t err = cudaSuccess;
  for (int j = 0; j < poll_iters(h) && err == cudaSuccess; ++j) err = bicg_iteration(h, g13, grid, h->cs);
  cudaError_t e2 = cudaStreamEndCapture(h->cs, &graph);
  if (err != cudaSuccess || e2 != cudaSuccess) {
    if (graph) cudaGraphDestroy(graph);
    return RB_ECUDA;
  }
  cudaError_t e3 = cudaGraphInstantiate(&g->exec, graph, 0);
  cudaGraphDestroy(graph);
  if (e3 != cudaSuccess) return RB_ECUDA;
  g->valid = true;
  h->g_bicg_k = h->k;
  return RB_OK;
}

}  // namespace

extern "C" int rbicg_solve(rb_handle h, const double* b, const double* bt, double* x, double* xt, int where,
                           rb_stats* st, rb_stats* st_dual) {
  if (!h || !b || !x || !xt || (where != RB_HOST && where != RB_DEVICE)) return RB_EINVAL;
  if (!h->have_matrix) return RB_EDIM;
  int rc = ensure_slots(h, 2);
  if (rc) return rc;
  SolveOut so{};
  {
    int64_t mv = 0;
    if ((rc = ensure_setup(h, &mv)) < 0) return rc;
    so.mv_setup = mv;
  }
  if (h->k > 0) {   // T2 = U~ Mpt: the dual solution's basis (see bicg_dual_start)
    std::vector<double*> out;
    std::vector<const double*> src;
    for (int j = 0; j < h->k; ++j) {
      out.push_back(colp(h->T2, h->npad, j));
      src.push_back(colp(h->Ut, h->npad, j));
    }
    if ((rc = block_gemm<double>(h, out, src, h->Mpt, h->k))) return rc;
    if ((rc = sync(h))) return rc;
  }
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  auto done = [&](int code) {
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    return code;
  };
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) return done(RB_ECUDA);
  if (cudaEventRecord(e0, h->us) != cudaSuccess) return done(RB_ECUDA);
  const int64_t n = h->n, ld = h->npad;
  Slot &P = h->sl[0], &D = h->sl[1];
  // b, b~ (the shadow vector when bt is NULL), x_{-1}, x~_{-1}
  if ((rc = copy_in(P.b, b, sizeof(double) * n, where, h->us))) return done(rc);
  if (bt) {
    if ((rc = copy_in(D.b, bt, sizeof(double) * n, where, h->us))) return done(rc);
  } else {
    RB_CUDA_TRY(shadow(D.b, n, h->npad, h->o.shadow_seed, h->us));
  }
  if ((rc = copy_in(P.x, x, sizeof(double) * n, where, h->us))) return done(rc);
  if ((rc = copy_in(D.x, xt, sizeof(double) * n, where, h->us))) return done(rc);
  double nb[2];
  for (int i = 0; i < 2; ++i) {
    Slot& s = h->sl[i];
    int f = 0;
    RB_CUDA_TRY(check_finite(s.b, n, h->dflag, h->us));
    RB_CUDA_TRY(cudaMemcpyAsync(&f, h->dflag, sizeof(int), cudaMemcpyDeviceToHost, h->us));
    if ((rc = sync(h))) return done(rc);
    int fx = 0;
    RB_CUDA_TRY(check_finite(s.x, n, h->dflag, h->us));
    RB_CUDA_TRY(cudaMemcpyAsync(&fx, h->dflag, sizeof(int), cudaMemcpyDeviceToHost, h->us));
    if ((rc = sync(h))) return done(rc);
    if (f || fx) return done(RB_ENONFINITE);
    DotArgs d{};
    d.nd = 1;
    d.a[0] = s.b; d.b[0] = s.b;
    if ((rc = run_dots(h, d, &nb[i], 1, i))) return done(rc);
  }
  // eq. (3.5), primary: r_{-1} = b - A x_{-1}; x_0, r_0
  RB_CUDA_TRY(residual_norm(h->A.view(), P.b, P.x, P.r, h->npad, h->st, h->partials, h->grids.spmv, h->us));
  if (h->k > 0) {
    DotArgs d{};
    d.M = h->Chat; d.ld = ld; d.km = h->k; d.v = P.r; d.nd = 0;
    RB_CUDA_TRY(dots(d, h->npad, h->st, h->partials, vec_grid(h), h->us));
    RB_CUDA_TRY(gemv_update(P.x, h->U, ld, h->k, h->st[0].red, nullptr, 1.0, h->npad, vec_grid(h), h->us));
    RB_CUDA_TRY(gemv_update(P.r, h->C, ld, h->k, h->st[0].red, nullptr, -1.0, h->npad, vec_grid(h), h->us));
  }
  // dual; a new x~_{-1} while (r_0, r~_0) = 0
  if ((rc = bicg_dual_start(h))) return done(rc);
  double red[3];
  so.seeds = 0;
  for (int attempt = 0;; ++attempt) {
    DotArgs d{};
    d.nd = 3;
    d.a[0] = D.r; d.b[0] = P.r;
    d.a[1] = P.r; d.b[1] = P.r;
    d.a[2] = D.r; d.b[2] = D.r;
    if ((rc = run_dots(h, d, red, 3, 0))) return done(rc);
    if (red[0] != 0.0 || attempt == 3) break;
    RB_CUDA_TRY(shadow(D.x, n, h->npad, h->o.shadow_seed + (uint64_t)attempt, h->us));
    so.seeds = attempt + 1;
    if ((rc = bicg_dual_start(h))) return done(rc);
  }
  // p_0 = 0, beta_0 = 0: the first iteration's p_1 = r_0
  RB_CUDA_TRY(cudaMemcpyAsync(P.p, P.r, sizeof(double) * ld, cudaMemcpyDeviceToDevice, h->us));
  RB_CUDA_TRY(cudaMemcpyAsync(D.p, D.r, sizeof(double) * ld, cudaMemcpyDeviceToDevice, h->us));
  if ((rc = read_state(h, 2))) return done(rc);
  const int max_itn = h->o.max_itn > 0 ? h->o.max_itn : (int)std::min<int64_t>(n, 20000);
  const double tol = h->o.tol;
  for (int i = 0; i < 2; ++i) {
    IterState& hs = h->hst[i];
    hs.k = h->k;
    for (int j = 0; j < h->k; ++j) hs.xc[j] = 0.0;
    hs.iter = 0;
    hs.half = 0;
    hs.done = 0;
    hs.status = RB_OK;
    hs.max_itn = max_itn;
    hs.thresh2 = tol * tol * nb[i];
    hs.bnorm2 = nb[i];
    hs.rnorm2 = i == 0 ? red[1] : red[2];
    hs.alpha = hs.beta = hs.omega = 0.0;
    hs.rho = red[0];
  }
  IterState& h0 = h->hst[0];
  if (!std::isfinite(red[0]) || !std::isfinite(red[1]) || !std::isfinite(red[2])) {
    h0.status = RB_ENONFINITE;
    h0.done = 1;
  } else if (red[1] <= h0.thresh2 && red[2] <= h->hst[1].thresh2) {
    h0.done = 1;
  } else if (red[0] == 0.0) {
    h0.status = RB_EBREAKDOWN_RHO;
    h0.done = 1;
  }
  RB_CUDA_TRY(cudaMemcpyAsync(h->st, h->hst, sizeof(IterState) * 2, cudaMemcpyHostToDevice, h->us));
  // the iteration: graphs of poll iterations until both systems converge or the solve stops
  if (!h0.done) {
    if (!h->g_bicg.valid || h->g_bicg_k != h->k) {
      if ((rc = capture_bicg(h))) return done(rc);
    }
    for (;;) {
      RB_CUDA_TRY(cudaGraphLaunch(h->g_bicg.exec, h->us));
      count_launches((long long)poll_iters(h) * (h->k > 0 ? 8 : 6));
      if ((rc = read_state(h, 2))) return done(rc);
      if (h->hst[0].done) break;
    }
  }
  // the final correction and the true residuals
  if (h->k > 0) {
    RB_CUDA_TRY(gemv_update(P.x, h->U, ld, h->k, h->st[0].xc, nullptr, -1.0, h->npad, vec_grid(h), h->us));
    RB_CUDA_TRY(gemv_update(D.x, h->T2, ld, h->k, h->st[1].xc, nullptr, -1.0, h->npad, vec_grid(h), h->us));
  }
  double tr[2];
  RB_CUDA_TRY(residual_norm(h->A.view(), P.b, P.x, h->tmp, h->npad, h->st, h->partials, h->grids.spmv, h->us));
  RB_CUDA_TRY(residual_norm(h->AT.view(), D.b, D.x, h->tmp2, h->npad, h->st + 1, h->partials, h->grids.spmv,
                            h->us));
  if ((rc = read_state(h, 2))) return done(rc);
  tr[0] = h->hst[0].red[0];
  tr[1] = h->hst[1].red[0];
  if ((rc = copy_out(x, P.x, sizeof(double) * n, where, h->us))) return done(rc);
  if ((rc = copy_out(xt, D.x, sizeof(double) * n, where, h->us))) return done(rc);
  cudaEventRecord(e1, h->us);
  if ((rc = sync(h))) return done(rc);
  float ms = 0;
  cudaEventElapsedTime(&ms, e0, e1);
  const int status = h->hst[0].status;
  const int iters = h->hst[0].iter;
  rb_stats* outs[2] = {st, st_dual};
  for (int i = 0; i < 2; ++i) {
    if (!outs[i]) continue;
    rb_stats& o = *outs[i];
    o = rb_stats{};
    o.iters = iters;
    o.status = status;
    o.k_used = h->k;
    o.seeds_used = so.seeds + 1;
    o.matvecs = 2 * (int64_t)iters;
    o.matvecs_setup = so.mv_setup;
    o.matvecs_check = 2;
    o.outer = 1;
    o.relres_rec = nb[i] > 0 ? std::sqrt(h->hst[i].rnorm2 / nb[i]) : 0.0;
    o.relres_true = nb[i] > 0 ? std::sqrt(tr[i] / nb[i]) : 0.0;
    o.ms_total = ms;
  }
  return done(status);
}

// ============================================================ adjoint (dual) solve
// The dual system A^T lam = g of Sec. 2 by Alg. 2 on A^T with the recycle
// space's roles swapped: right space U~ (A^T U~ = C~, already formed by the
// setup) and left space U ((A^T)^T U = C).  With M = C~^T C the dual's
// M' = C^T C~ = M^T, so its C-hat' = C (M^+) (C-hat = C~ (M^+)^T of the
// primary): one n x k product; no new products with A.  FP64, the space
// held fixed.  The call swaps A with A^T and the space blocks in the handle,
// runs the blocked solve of one right-hand side, and swaps them back (the
// captured graphs of either orientation are dropped).
extern "C" int rbicgstab_solve_adjoint(rb_handle h, const double* g, double* lam, int where, rb_stats* st) {
  using namespace rb;
  if (!h || !g || !lam || (where != RB_HOST && where != RB_DEVICE)) return RB_EINVAL;
  if (!h->have_matrix) return RB_EDIM;
  int rc = ensure_slots(h, 1);
  if (rc) return rc;
  int64_t mv_setup = 0;
  if ((rc = ensure_setup(h, &mv_setup)) < 0) return rc;
  const int k = h->k;
  if (k > 0) {   // T1 = C Mpt^T = C (M^+)
    std::vector<double> MptT((size_t)k * k);
    for (int r = 0; r < k; ++r)
      for (int c = 0; c < k; ++c) MptT[r + (size_t)c * k] = h->Mpt[c + (size_t)r * k];
    std::vector<double*> out;
    std::vector<const double*> src;
    for (int j = 0; j < k; ++j) {
      out.push_back(colp(h->T1, h->npad, j));
      src.push_back(colp(h->C, h->npad, j));
    }
    if ((rc = block_gemm<double>(h, out, src, MptT, k))) return rc;
  }
  const rb_opts saved = h->o;
  auto swap_all = [&]() {
    std::swap(h->A, h->AT);
    std::swap(h->U, h->Ut);
    std::swap(h->C, h->Ct);
    std::swap(h->Chat, h->T1);
    reset_graphs(h);
  };
  h->o.precision = RB_FP64;
  if (h->o.recycle_mode != RB_RECYCLE_NONE) h->o.recycle_mode = RB_RECYCLE_FIXED;
  swap_all();
  rc = rbicgstab_solve_block(h, 1, g, lam, h->n, where, st);
  swap_all();
  h->o = saved;
  if (st) st->matvecs_setup += mv_setup;
  return rc;
}

// ============================================================ BiCGstab(l)
// Recycled BiCGstab(l) (Sleijpen and Fokkema, ETNA 1, 1993) on the projected
// operator B = (I - C C-hat^T) A of Sec. 3, FP64, with the handle's recycle
// space held fixed: the breakdown-robust variant behind the omega = 0
// remark of Sec. 4 and the outlook of Sec. 7.  Each outer step takes l BiCG
// steps (two products with B each), which keep r_j = B r_{j-1} and
// u_j = B u_{j-1}, and then minimises ||r_0 - sum_j g_j r_j|| over
// g in R^l; then x += sum_j g_j r_{j-1}, r_0 -= sum_j g_j r_j,
// u_0 -= sum_j g_j u_j, omega = g_l.  The minimiser comes from the Gram
// matrix of the residual block, diagonally scaled, by a Cholesky solve
// (the same minimiser as modified Gram-Schmidt on the block, up to
// rounding).  Every product's projection coefficients C-hat^T A v are
// carried on the host alongside the vectors (x_c of Alg. 2), so the end is
// x = x_0 + y - U x_c.  Vectors and products run in the library's kernels;
// the scalars and the k-coefficients are formed on the host between them.
namespace {
constexpr int kMaxEll = 8;
}

extern "C" int rbicgstab_solve_l(rb_handle h, int32_t ell, const double* b, double* x, int where, rb_stats* st) {
  using namespace rb;
  if (!h || !b || !x || (where != RB_HOST && where != RB_DEVICE) || ell < 1 || ell > kMaxEll) return RB_EINVAL;
  if (!h->have_matrix) return RB_EDIM;
  int rc = ensure_slots(h, 1);
  if (rc) return rc;
  int64_t mv_setup = 0;
  if ((rc = ensure_setup(h, &mv_setup)) < 0) return rc;
  const int64_t n = h->n, ld = h->npad;
  const int k = h->k, vg = vec_grid(h);
  const int nvec = 2 * (ell + 1) + 1;
  if (h->lvec_cnt < nvec) {
    cudaFree(h->lvec);
    h->lvec_cnt = 0;
    int err = 0;
    h->lvec = dalloc<double>((int64_t)nvec * ld, &err);
    if (!h->lvec) return err;
    h->lvec_cnt = nvec;
  }
  auto R = [&](int j) { return h->lvec + (int64_t)j * ld; };
  auto Uv = [&](int j) { return h->lvec + (int64_t)(ell + 1 + j) * ld; };
  double* y = h->lvec + (int64_t)(2 * (ell + 1)) * ld;
  Slot& S0 = h->sl[0];
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  auto done = [&](int code) {
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    return code;
  };
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) return done(RB_ECUDA);
  cudaEventRecord(e0, h->us);
  RB_CUDA_TRY(cudaMemsetAsync(h->lvec, 0, sizeof(double) * nvec * ld, h->us));
  if ((rc = copy_in(S0.b, b, sizeof(double) * n, where, h->us))) return done(rc);
  if ((rc = copy_in(S0.x, x, sizeof(double) * n, where, h->us))) return done(rc);
  for (double* v : {S0.b, S0.x}) {
    int f = 0;
    RB_CUDA_TRY(check_finite(v, n, h->dflag, h->us));
    RB_CUDA_TRY(cudaMemcpyAsync(&f, h->dflag, sizeof(int), cudaMemcpyDeviceToHost, h->us));
    if ((rc = sync(h))) return done(rc);
    if (f) return done(RB_ENONFINITE);
  }
  int64_t mv = 0;
  auto dot = [&](const double* a, const double* c, double* out) {
    DotArgs d{};
    d.nd = 1;
    d.a[0] = a;
    d.b[0] = c;
    return run_dots(h, d, out, 1);
  };
  auto lin = [&](double* yv, double a, std::initializer_list<std::pair<const double*, double>> terms) -> int {
    LinComb lc{};
    for (auto& t : terms) {
      lc.x[lc.nx] = t.first;
      lc.c[lc.nx] = t.second;
      ++lc.nx;
    }
    RB_CUDA_TRY(lincomb(yv, a, lc, ld, vg, h->us));
    return RB_OK;
  };
  // out = B v; z = C-hat^T A v (host)
  auto Bop = [&](const double* v, double* out, std::vector<double>& z) -> int {
    RB_CUDA_TRY(spmv<double>(h->A.view(), v, out, 1.0, 0.0, h->grids.spmv, h->us));
    ++mv;
    z.assign(k, 0.0);
    if (k > 0) {
      DotArgs d{};
      d.M = h->Chat; d.ld = ld; d.km = k; d.v = out; d.nd = 0;
      int r2 = run_dots(h, d, z.data(), k);
      if (r2) return r2;
      RB_CUDA_TRY(gemv_update(out, h->C, ld, k, h->st[0].red, nullptr, -1.0, h->npad, vg, h->us));
    }
    return RB_OK;
  };
  double nb = 0.0, nx0 = 0.0;
  if ((rc = dot(S0.b, S0.b, &nb))) return done(rc);
  if ((rc = dot(S0.x, S0.x, &nx0))) return done(rc);
  // eq. (3.5): r_{-1} = b - A x_{-1}; x_0 = x_{-1} + U C-hat^T r_{-1}; r_0 = (I - C C-hat^T) r_{-1}
  RB_CUDA_TRY(residual_norm(h->A.view(), S0.b, S0.x, R(0), h->npad, h->st, h->partials, h->grids.spmv, h->us));
  if (nx0 > 0) ++mv;
  if (k > 0) {
    DotArgs d{};
    d.M = h->Chat; d.ld = ld; d.km = k; d.v = R(0); d.nd = 0;
    RB_CUDA_TRY(dots(d, h->npad, h->st, h->partials, vg, h->us));
    RB_CUDA_TRY(gemv_update(S0.x, h->U, ld, k, h->st[0].red, nullptr, 1.0, h->npad, vg, h->us));
    RB_CUDA_TRY(gemv_update(R(0), h->C, ld, k, h->st[0].red, nullptr, -1.0, h->npad, vg, h->us));
  }
  // shadow r~_0 = (I - C~ C-check^T) r~_{-1} = r~_{-1} - C-hat (C^T r~_{-1})
  RB_CUDA_TRY(shadow(h->rt0, n, h->npad, h->o.shadow_seed, h->us));
  if (k > 0) {
    DotArgs d{};
    d.M = h->C; d.ld = ld; d.km = k; d.v = h->rt0; d.nd = 0;
    RB_CUDA_TRY(dots(d, h->npad, h->st, h->partials, vg, h->us));
    RB_CUDA_TRY(gemv_update(h->rt0, h->Chat, ld, k, h->st->red, nullptr, -1.0, h->npad, vg, h->us));
  }
  const int max_itn = h->o.max_itn > 0 ? h->o.max_itn : (int)std::min<int64_t>(n, 20000);
  const double thresh2 = h->o.tol * h->o.tol * nb;
  std::vector<std::vector<double>> zr(ell + 1, std::vector<double>(k, 0.0)), zu(ell + 1, std::vector<double>(k, 0.0));
  std::vector<double> xc(k, 0.0), z;
  double rnorm2 = 0.0;
  if ((rc = dot(R(0), R(0), &rnorm2))) return done(rc);
  int status = RB_OK, iters = 0, outer = 0;
  double rho0 = 1.0, alpha = 1.0, omega = 1.0;
  bool converged = !(rnorm2 > thresh2);
  while (!converged && status == RB_OK) {
    if (iters + ell > max_itn) {
      status = RB_ENOTCONV;
      break;
    }
    rho0 = -omega * rho0;
    for (int j = 0; j < ell && status == RB_OK; ++j) {
      double rho1 = 0.0;
      if ((rc = dot(h->rt0, R(j), &rho1))) return done(rc);
      if (rho1 == 0.0 || rho0 == 0.0 || !std::isfinite(rho1)) {
        status = std::isfinite(rho1) ? RB_EBREAKDOWN_RHO : RB_ENONFINITE;
        break;
      }
      const double beta = alpha * rho1 / rho0;
      rho0 = rho1;
      for (int i = 0; i <= j; ++i) {
        if ((rc = lin(Uv(i), -beta, {{R(i), 1.0}}))) return done(rc);
        if (i >= 1)
          for (int c = 0; c < k; ++c) zu[i][c] = zr[i][c] - beta * zu[i][c];
      }
      if ((rc = Bop(Uv(j), Uv(j + 1), z))) return done(rc);
      zu[j + 1] = z;
      double gam = 0.0;
      if ((rc = dot(h->rt0, Uv(j + 1), &gam))) return done(rc);
      if (gam == 0.0 || !std::isfinite(gam)) {
        status = std::isfinite(gam) ? RB_EBREAKDOWN_RHO : RB_ENONFINITE;
        break;
      }
      alpha = rho0 / gam;
      for (int i = 0; i <= j; ++i) {
        if ((rc = lin(R(i), 1.0, {{Uv(i + 1), -alpha}}))) return done(rc);
        if (i >= 1)
          for (int c = 0; c < k; ++c) zr[i][c] -= alpha * zu[i + 1][c];
      }
      if ((rc = Bop(R(j), R(j + 1), z))) return done(rc);
      zr[j + 1] = z;
      if ((rc = lin(y, 1.0, {{Uv(0), alpha}}))) return done(rc);
      for (int c = 0; c < k; ++c) xc[c] += alpha * zu[1][c];
      ++iters;
    }
    if (status != RB_OK) break;
    // minimal residual over span{r_1..r_l}: Gram matrix G(i, j) = (r_i, r_j)
    std::vector<double> G((size_t)(ell + 1) * (ell + 1), 0.0);
    {
      std::vector<std::pair<int, int>> pairs;
      for (int i = 0; i <= ell; ++i)
        for (int j = i; j <= ell; ++j) pairs.push_back({i, j});
      for (size_t q0 = 0; q0 < pairs.size(); q0 += 4) {
        DotArgs d{};
        for (size_t q = q0; q < std::min(pairs.size(), q0 + 4); ++q) {
          d.a[d.nd] = R(pairs[q].first);
          d.b[d.nd] = R(pairs[q].second);
          ++d.nd;
        }
        double out4[4];
        if ((rc = run_dots(h, d, out4, d.nd))) return done(rc);
        for (int q = 0; q < d.nd; ++q) {
          const int i = pairs[q0 + q].first, j = pairs[q0 + q].second;
          G[i + (size_t)j * (ell + 1)] = G[j + (size_t)i * (ell + 1)] = out4[q];
        }
      }
    }
    // scaled normal equations D G_11 D (D^-1 g) = D G_10, Cholesky
    std::vector<double> sc(ell + 1, 0.0), L((size_t)ell * ell, 0.0), g(ell + 1, 0.0);
    bool ok = true;
    for (int j = 1; j <= ell; ++j) {
      const double gjj = G[j + (size_t)j * (ell + 1)];
      if (!(gjj > 0.0) || !std::isfinite(gjj)) ok = false;
      sc[j] = ok ? 1.0 / std::sqrt(gjj) : 0.0;
    }
    for (int j = 0; ok && j < ell; ++j) {
      for (int i = j; i < ell; ++i) {
        double v = G[(i + 1) + (size_t)(j + 1) * (ell + 1)] * sc[i + 1] * sc[j + 1];
        for (int q = 0; q < j; ++q) v -= L[i + (size_t)q * ell] * L[j + (size_t)q * ell];
        if (i == j) {
          if (!(v > 1e-28)) {
            ok = false;
            break;
          }
          L[j + (size_t)j * ell] = std::sqrt(v);
        } else {
          L[i + (size_t)j * ell] = v / L[j + (size_t)j * ell];
        }
      }
    }
    if (!ok) {
      status = RB_EBREAKDOWN_OMEGA;
      break;
    }
    std::vector<double> w(ell, 0.0);
    for (int i = 0; i < ell; ++i) {   // L w = D G_10
      double v = G[(i + 1) + 0] * sc[i + 1];
      for (int q = 0; q < i; ++q) v -= L[i + (size_t)q * ell] * w[q];
      w[i] = v / L[i + (size_t)i * ell];
    }
    for (int i = ell - 1; i >= 0; --i) {   // L^T (D^-1 g) = w
      double v = w[i];
      for (int q = i + 1; q < ell; ++q) v -= L[q + (size_t)i * ell] * w[q];
      w[i] = v / L[i + (size_t)i * ell];
    }
    for (int j = 1; j <= ell; ++j) g[j] = w[j - 1] * sc[j];
    omega = g[ell];
    if (omega == 0.0 || !std::isfinite(omega)) {
      status = std::isfinite(omega) ? RB_EBREAKDOWN_OMEGA : RB_ENONFINITE;
      break;
    }
    // y gains sum_j g_j r_{j-1}; its B-image sum_j g_j r_j has the projection
    // coefficients sum_j g_j zr[j]
    for (int j = 1; j <= ell; ++j) {
      if ((rc = lin(y, 1.0, {{R(j - 1), g[j]}}))) return done(rc);
      for (int c = 0; c < k; ++c) xc[c] += g[j] * zr[j][c];
    }
    for (int j = 1; j <= ell; ++j) {
      if ((rc = lin(R(0), 1.0, {{R(j), -g[j]}}))) return done(rc);
      if ((rc = lin(Uv(0), 1.0, {{Uv(j), -g[j]}}))) return done(rc);
    }
    ++outer;
    if ((rc = dot(R(0), R(0), &rnorm2))) return done(rc);
    if (!std::isfinite(rnorm2)) {
      status = RB_ENONFINITE;
      break;
    }
    converged = rnorm2 <= thresh2;
  }
  // x = x_0 + y - U x_c
  if ((rc = lin(S0.x, 1.0, {{y, 1.0}}))) return done(rc);
  if (k > 0) {
    RB_CUDA_TRY(cudaMemcpyAsync(h->st[0].red, xc.data(), sizeof(double) * k, cudaMemcpyHostToDevice, h->us));
    RB_CUDA_TRY(gemv_update(S0.x, h->U, ld, k, h->st[0].red, nullptr, -1.0, h->npad, vg, h->us));
    if ((rc = sync(h))) return done(rc);
  }
  RB_CUDA_TRY(residual_norm(h->A.view(), S0.b, S0.x, h->tmp, h->npad, h->st, h->partials, h->grids.spmv, h->us));
  if ((rc = read_state(h, 1))) return done(rc);
  const double tr = h->hst[0].red[0];
  if ((rc = copy_out(x, S0.x, sizeof(double) * n, where, h->us))) return done(rc);
  cudaEventRecord(e1, h->us);
  if ((rc = sync(h))) return done(rc);
  float ms = 0;
  cudaEventElapsedTime(&ms, e0, e1);
  if (st) {
    *st = rb_stats{};
    st->iters = iters;
    st->status = status;
    st->k_used = k;
    st->seeds_used = 1;
    st->matvecs = mv;
    st->matvecs_setup = mv_setup;
    st->matvecs_check = 1;
    st->outer = outer;
    st->relres_rec = nb > 0 ? std::sqrt(rnorm2 / nb) : 0.0;
    st->relres_true = nb > 0 ? std::sqrt(tr / nb) : 0.0;
    st->ms_total = ms;
  }
  return done(status);
}

extern "C" int rbicgstab_solve(rb_handle h, const double* b, double* x, int where, rb_stats* st) {
  return rbicgstab_solve_block(h, 1, b, x, h ? h->n : 0, where, st);
}

// Benchmark helper: average duration of each pass kernel, measured with CUDA
// events on the handle's stream over `reps` iterations started from B.
template <typename T>
static int time_passes_t(rb_ctx* h, int nrhs, int reps, double* ms) {
  IterArgs<T> a = base_args<T>(h, nrhs);
  Grids g;
  iteration_grids<T>(h->k, h->nsm, h->npad, &g, nrhs);
  const int npass = 5;
  std::vector<cudaEvent_t> ev((size_t)reps * npass * 2);
  for (auto& e : ev) cudaEventCreate(&e);
  int rc = RB_OK;
  for (int it = 0; it < reps && !rc; ++it)
    for (int pz = 0; pz < npass; ++pz) {
      if (pz == P4 && h->k == 0) continue;
      if (cudaEventRecord(ev[(it * npass + pz) * 2], h->us) != cudaSuccess ||
          launch_pass<T>(pz, a, h->k, g, h->us) != cudaSuccess ||
          cudaEventRecord(ev[(it * npass + pz) * 2 + 1], h->us) != cudaSuccess) {
        rc = RB_ECUDA;
        break;
      }
    }
  if (!rc) rc = read_state(h, nrhs);
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
  for (int i = 0; i < nrhs; ++i)
    if (h->hst[i].done) return h->hst[i].status ? h->hst[i].status : RB_EBREAKDOWN_OMEGA;
  return RB_OK;
}

extern "C" int rbicgstab_time_passes(rb_handle h, int32_t nrhs, const double* B, int64_t ld, int where,
                                     int32_t reps, double* ms) {
  if (!h || !B || !ms || reps < 1 || reps > 1000 || nrhs < 1 || nrhs > kMaxRhs ||
      (where != RB_HOST && where != RB_DEVICE))
    return RB_EINVAL;
  if (!h->have_matrix) return RB_EDIM;
  if (nrhs > 1 && ld < h->n) return RB_EINVAL;
  int rc = ensure_slots(h, nrhs);
  if (rc) return rc;
  {
    int64_t mv = 0;
    if ((rc = ensure_setup(h, &mv)) < 0) return rc;
  }
  SolveOut so[kMaxRhs];
  double* rhs[kMaxRhs];
  double* xb[kMaxRhs];
  double tol[kMaxRhs];
  bool xnz[kMaxRhs] = {false, false, false, false}, skip[kMaxRhs] = {false, false, false, false};
  for (int i = 0; i < nrhs; ++i) {
    Slot& s = h->sl[i];
    rc = copy_in(s.b, B + (int64_t)i * ld, sizeof(double) * h->n, where, h->us);
    if (rc) return rc;
    RB_CUDA_TRY(cudaMemsetAsync(s.x, 0, sizeof(double) * h->npad, h->us));
    DotArgs d{};
    d.nd = 1;
    d.a[0] = s.b; d.b[0] = s.b;
    double nb = 0;
    if ((rc = run_dots(h, d, &nb, 1, i))) return rc;
    RB_CUDA_TRY(cudaMemcpyAsync(&h->st[i].bnorm2, &h->st[i].red[0], sizeof(double), cudaMemcpyDeviceToDevice,
                                h->us));
    rhs[i] = s.b;
    xb[i] = s.x;
    tol[i] = 1e-300;
  }
  rc = setup_block(h, nrhs, rhs, xb, xnz, skip, tol, so);
  if (rc) return rc;
  rc = read_state(h, nrhs);
  if (rc) return rc;
  for (int i = 0; i < nrhs; ++i)
    if (h->hst[i].done) return h->hst[i].status ? h->hst[i].status : RB_EINVAL;
  if (h->o.precision == RB_MIXED) {
    RB_CUDA_TRY(to_float(h->rt0, h->frt0, h->npad, h->us));
    for (int i = 0; i < nrhs; ++i) {
      RB_CUDA_TRY(to_float(h->sl[i].r, h->sl[i].fr, h->npad, h->us));
      RB_CUDA_TRY(cudaMemsetAsync(h->sl[i].fx, 0, sizeof(float) * h->npad, h->us));
    }
    if ((rc = init_p<float>(h, nrhs, false))) return rc;
    return time_passes_t<float>(h, nrhs, reps, ms);
  }
  if ((rc = init_p<double>(h, nrhs, false))) return rc;
  return time_passes_t<double>(h, nrhs, reps, ms);
}

extern "C" long long rbicgstab_kernel_launches(void) { return g_launches.load(); }
