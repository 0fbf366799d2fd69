// Internal launcher declarations (host side) for librbicgstab.
#pragma once

#include "common.cuh"

namespace rb {

// Pointers of one RBiCGSTAB iteration (Alg. 2) over nrhs <= kMaxRhs
// right-hand sides of the same matrix and recycle space.  Vectors have npad
// entries (n rounded up to the slice height; the tail is kept at zero).  For
// k = 0, q aliases qraw and t aliases traw.  st points to nrhs consecutive
// states; the grid-reduction tickets of st[0] serve all of them.
template <typename T>
struct IterArgs {
  Sell<T> A;
  const T* Chat;  // C-hat = C~ D_c^{-1}, column-major n x k, leading dim ld
  const T* C;     // C = A U, column-major, leading dim ld
  int64_t ld;
  const T* rt0;   // r~_0 (shared)
  T* x[kMaxRhs];
  T* r[kMaxRhs];
  T* p_in[kMaxRhs];   // p_i
  T* p_out[kMaxRhs];  // p_{i+1} (may equal p_in)
  T* s[kMaxRhs];
  T* q[kMaxRhs];
  T* qraw[kMaxRhs];   // A p_i before projection
  T* t[kMaxRhs];
  T* traw[kMaxRhs];   // A s_i before projection
  IterState* st;
  double* partials;
  int64_t npad;
  int nrhs;
  int stage_bulk;  // staged passes taking tiles by bulk copies: bit 0 P2, bit 1 P4, bit 2 P5
};

struct Grids {
  int spmv;     // generic SpMV-shaped kernels
  int vec;      // generic streaming kernels
  int pass[5];  // fused passes P1..P5: one full wave each
};

int kmax_bucket(int k);
// Compiled right-hand-side block sizes: 1, 2 or 4 (unused slots are masked).
int rhs_bucket(int nrhs);

// Process-wide count of kernels this library has launched (graph replays add
// the kernels their graph holds).
void count_launches(long long n);

template <typename T>
cudaError_t launch_iteration(const IterArgs<T>& a, int k, const Grids& g, cudaStream_t s);

template <typename T>
void iteration_grids(int k, int nsm, int64_t npad, Grids* g, int nrhs);

// One pass (P1..P5 = 0..4) of the iteration, launched on its own.
template <typename T>
cudaError_t launch_pass(int pass, const IterArgs<T>& a, int k, const Grids& g, cudaStream_t s);

// Alg. 1 (RBiCG) for a primary system and its dual, FP64: the vector
// arrays and scalars of the closing passes (q, qt are the corrected
// products).  st[0]: primary scalars, st[1]: dual.
struct BiArgs {
  int64_t npad;
  double *x, *r, *p, *q;        // primary
  double *xt, *rt, *pt, *qt;    // dual
  IterState* st;
  double* partials;
};
// q = z - C zeta, q~ = z~ - C~ D_c^{-1} C^T z~ in place over a.q, a.qt (zeta,
// C^T z~ in the gamma fields of st[0], st[1]; k = st[0].k) and (p~, q) ->
// st[0].red[0].
cudaError_t bicg_project(const BiArgs& a, const double* C, const double* Ct, int64_t ld, const double* dinv,
                         int grid, cudaStream_t s);
// alpha = (r~, r) / (p~, q) from st[0].red[0], and the zeta_c updates.
cudaError_t bicg_alpha(IterState* st, const double* dinv, cudaStream_t s);
// x, x~, r, r~ updates with the convergence test and beta; then p, p~.
cudaError_t bicg_update(const BiArgs& a, int grid, cudaStream_t s);
int bicg_grid(int nsm, int64_t npad);

// ---------------------------------------------------------------- matrix.cu
// Sparse matrix in SELL-32 form, owned by the library.
template <typename T>
struct SellBuf {
  int64_t* slice_ptr = nullptr;
  int32_t* width = nullptr;
  int32_t* col = nullptr;
  T* val = nullptr;
  int64_t* perm = nullptr;   // SELL position -> CSR position (or -1 for padding)
  int32_t* offs = nullptr;   // per-slice column offsets of stencil slices (see Sell)
  int offs_stride = 1;
  int64_t nslices = 0;
  int64_t cap = 0;           // entries incl. padding
  int64_t stencil_slices = 0;
  Sell<T> view() const { return Sell<T>{slice_ptr, width, col, val, nslices, offs, offs_stride}; }
};

// Validate CSR on the device; *bad receives 0 (ok), RB_EBADCSR or RB_ENONFINITE.
int csr_validate(int64_t n, int64_t nnz, const int32_t* row_ptr, const int32_t* col,
                 const double* val, int* d_flag, int* bad, cudaStream_t s);
// Build SELL-32 structure from device CSR (allocates inside `out`).
int sell_build(int64_t n, int64_t nnz, const int32_t* row_ptr, const int32_t* col,
               SellBuf<double>* out, cudaStream_t s,
               bool allow_stencil = true);
// Refill SELL values from CSR values through out->perm.
template <typename T>
int sell_fill_values(const SellBuf<T>& out, const double* csr_val, cudaStream_t s);
// Build CSR of A^T on the device (rows sorted by column index).
int csr_transpose(int64_t n, int64_t nnz, const int32_t* row_ptr, const int32_t* col,
                  int32_t* t_row_ptr, int32_t* t_col, int64_t* t_src, cudaStream_t s);
// Gather values of A^T from A's values: t_val[e] = val[t_src[e]].
int gather_values(int64_t nnz, const int64_t* t_src, const double* val, double* t_val,
                  cudaStream_t s);
template <typename T>
void sell_free(SellBuf<T>* b);

// y = alpha * A v + beta * y (FP64 or FP32), npad entries.
template <typename T>
cudaError_t spmv(const Sell<T>& A, const T* v, T* y, double alpha, double beta, int grid,
                 cudaStream_t s);

// ---------------------------------------------------------------- blas.cu
// Generic deterministic reductions into st->red:
//   red[j]      = sum_i M[j*ld + i] * v[i]            for j < km   (M may be null)
//   red[km + d] = sum_i a_d[i] * b_d[i]               for d < nd  (nd <= 4)
struct DotArgs {
  const double* M;
  int64_t ld;
  int km;
  const double* v;
  const double* a[4];
  const double* b[4];
  int nd;
};
cudaError_t dots(const DotArgs& d, int64_t npad, IterState* st, double* partials, int grid,
                 cudaStream_t s);
// y = a y + sum_{t < nx} c[t] x[t] (FP64, rows < npad; a = 0 ignores y's
// old contents).  x[t] may alias y only as x[t] == y.
struct LinComb {
  const double* x[4];
  double c[4];
  int nx;
};
cudaError_t lincomb(double* y, double a, const LinComb& lc, int64_t npad, int grid, cudaStream_t s);
// out[e] = scale * u[i] * v[ci[e]] over the entries e of each row i of the
// CSR pattern (rp, ci) with n rows (device arrays; out in CSR order).
cudaError_t pattern_outer(int64_t n, const int32_t* rp, const int32_t* ci, const double* u, const double* v,
                          double scale, double* out, int grid, cudaStream_t s);
// y[i] += sign * sum_j M[j*ld+i] * c[j], c read from device memory (c_scale[j]
// multiplies c[j] when non-null).
cudaError_t gemv_update(double* y, const double* M, int64_t ld, int k, const double* c,
                        const double* c_scale, double sign, int64_t npad, int grid,
                        cudaStream_t s);
// Out(:, c) = sum_j X(:, j) R[j + c*m] for c < kc (column pointer lists;
// R is m x kc column-major FP64 on the device; accumulation in T).  Out must
// not alias X.
template <typename T>
cudaError_t gemm_cols(T* const* out, const T* const* X, int m, const double* R, int kc, int64_t npad,
                      int grid, cudaStream_t s);
// G[a + b*mx] = sum_i X_a[i] Y_b[i] for a < mx, b < my (column pointer lists),
// FP64 result (Dot2 accumulation for FP32 columns); writes mx*my doubles to
// `out` (device).  `work` holds grid*mx*my doubles.
template <typename T>
cudaError_t gram(const T* const* X, int mx, const T* const* Y, int my, int64_t npad, double* out,
                 double* work, int grid, cudaStream_t s);
// G = Z^T Z and H = Z^T W (m x m each, column-major, FP64) in one pass over
// the column pointer lists Z[0..m), W[0..m); `work` holds grid *
// gram_gh_work(m) doubles.  m <= 90.
int gram_gh_work(int m);
template <typename T>
cudaError_t gram_gh(const T* const* Z, const T* const* W, int m, int64_t npad, double* G, double* H,
                    double* work, int grid, cudaStream_t s);
// The recycle update's Gram matrices on the tensor cores (gram_tc.cu):
// G = Z^T Z and H = Z^T W (m x m each, column-major, FP64, on the device) for
// FP32 column blocks Z = [AY, AP, AS], W = [Y, P, S], each block column-major
// with leading dimension ld, cols[b] <= cap[b] columns in use (the caps fix the
// shared-memory layout; Z's and W's caps and column counts pair up).
// `work` holds gram_tc_work_floats(cap, grid) floats; `err` (device int,
// zeroed by the caller) becomes nonzero if a CTA gave up a bounded wait.
constexpr int kMaxGramTc = 128;
struct GramTcBlocks {
  const float* ptr[6];   // AY, AP, AS, Y, P, S
  int cols[6];
  int cap[6];
};
bool gram_tc_eligible(const int cap[6]);
size_t gram_tc_work_floats(const int cap[6], int grid);
int gram_tc(const GramTcBlocks& blk, int64_t n, int64_t ld, double* G, double* H, float* work, int* err,
            int grid, cudaStream_t s);
// st->red[j] = ||M_j||^2 for column pointers M[0..k) (deterministic).
template <typename T>
cudaError_t colnorm2(const T* const* M, int k, int64_t npad, IterState* st, double* partials, int grid,
                     cudaStream_t s);
// Shadow vector r~[i] = 2 * u53(SplitMix64(seed, i)) - 1 for i < n, 0 beyond.
cudaError_t shadow(double* rt, int64_t n, int64_t npad, uint64_t seed, cudaStream_t s);
// Scale column j of M (n x k, ld) by f[j] (device array); rows < npad.
template <typename T>
cudaError_t scale_cols(T* M, int64_t ld, int k, const double* f, int64_t npad, cudaStream_t s);
// Residual r = b - A x and red[0] = ||r||^2 into st->red (deterministic).
cudaError_t residual_norm(const Sell<double>& A, const double* b, const double* x, double* r,
                          int64_t npad, IterState* st, double* partials, int grid,
                          cudaStream_t s);
// Non-finite check: *flag = 1 if any of v[0..n) is NaN/Inf.
cudaError_t check_finite(const double* v, int64_t n, int* flag, cudaStream_t s);
// Precision conversions for the mixed path.
cudaError_t to_float(const double* in, float* out, int64_t n, cudaStream_t s);
cudaError_t add_float_to_double(double* x, const float* d, int64_t n, cudaStream_t s);
cudaError_t to_double(const float* in, double* out, int64_t n, cudaStream_t s);
// Device-side solve setup: thresholds, rho_0, c_r = C^T r~_0 (from st->red).
cudaError_t init_state(IterState* st, int k, double tol, int max_itn, cudaStream_t s);

}  // namespace rb
