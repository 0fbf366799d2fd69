// Small dense FP64 linear algebra on the host (m <= ~100), for the parts of
// the method that are a k x k or m x m problem:
//   * svd_small: the biorthogonalisation of C and C~ (the recycle setup of Sec. 3 requires
//     C~^T C diagonal and positive, Sec. 3): one-sided Jacobi SVD (Hestenes).
//   * harmonic_ritz: the eigenproblem of the recycle update between cycles
//     (Sec. 6.2): column scaling, restriction to the numerical range of W by
//     a symmetric eigendecomposition of the scaled G = Z^T Z (Householder
//     tridiagonalisation + implicit symmetric QR steps with the Wilkinson
//     shift, Golub & Van Loan, Matrix Computations, Sec. 8.3), reduction to
//     a standard problem, Householder-Hessenberg + Francis double-shift QR
//     for the eigenvalues (Sec. 7.4-7.5), and complex
//     inverse iteration on the Hessenberg form for the selected eigenvectors.
// These are deliberately different algorithms from the LAPACK routines the
// CPU oracle calls, so agreement between the two is evidence for both.
#include "hostla.h"

#include <algorithm>
#include <cmath>
#include <complex>
#include <numeric>
#include <vector>

namespace rb {

using cd = std::complex<double>;

// ---------------------------------------------------------------- SVD
// M (k x k, column-major) = P diag(sigma) Q^T with sigma descending.
void svd_small(int k, const double* M, double* P, double* sigma, double* Q) {
  std::vector<double> A(M, M + (size_t)k * k), V((size_t)k * k, 0.0);
  for (int i = 0; i < k; ++i) V[i + (size_t)i * k] = 1.0;
  const double eps = 2.220446049250313e-16;
  for (int sweep = 0; sweep < 60; ++sweep) {
    double off = 0.0;
    for (int a = 0; a < k - 1; ++a) {
      for (int b = a + 1; b < k; ++b) {
        double alpha = 0, beta = 0, gamma = 0;
        for (int i = 0; i < k; ++i) {
          const double x = A[i + (size_t)a * k], y = A[i + (size_t)b * k];
          alpha += x * x;
          beta += y * y;
          gamma += x * y;
        }
        if (gamma == 0.0) continue;
        const double rel = std::fabs(gamma) / std::sqrt(alpha * beta);
        off = std::max(off, rel);
        if (rel <= eps) continue;
        const double zeta = (beta - alpha) / (2.0 * gamma);
        const double t = (zeta >= 0 ? 1.0 : -1.0) / (std::fabs(zeta) + std::sqrt(1.0 + zeta * zeta));
        const double c = 1.0 / std::sqrt(1.0 + t * t), s = c * t;
        for (int i = 0; i < k; ++i) {
          const double x = A[i + (size_t)a * k], y = A[i + (size_t)b * k];
          A[i + (size_t)a * k] = c * x - s * y;
          A[i + (size_t)b * k] = s * x + c * y;
          const double vx = V[i + (size_t)a * k], vy = V[i + (size_t)b * k];
          V[i + (size_t)a * k] = c * vx - s * vy;
          V[i + (size_t)b * k] = s * vx + c * vy;
        }
      }
    }
    if (off <= eps) break;
  }
  std::vector<double> sv(k);
  for (int j = 0; j < k; ++j) {
    double s = 0;
    for (int i = 0; i < k; ++i) s += A[i + (size_t)j * k] * A[i + (size_t)j * k];
    sv[j] = std::sqrt(s);
  }
  std::vector<int> ord(k);
  std::iota(ord.begin(), ord.end(), 0);
  std::stable_sort(ord.begin(), ord.end(), [&](int a, int b) { return sv[a] > sv[b]; });
  for (int jj = 0; jj < k; ++jj) {
    const int j = ord[jj];
    sigma[jj] = sv[j];
    for (int i = 0; i < k; ++i) {
      Q[i + (size_t)jj * k] = V[i + (size_t)j * k];
      P[i + (size_t)jj * k] = sv[j] > 0 ? A[i + (size_t)j * k] / sv[j] : 0.0;
    }
  }
}

// ---------------------------------------------------------------- Hessenberg + QR
// Reduce a (n x n, row-major h[i*n+j]) to upper Hessenberg form by Householder
// reflections P_c = I - 2 v v^T / (v^T v), H = P_{n-3} .. P_0 A P_0 .. P_{n-3};
// the reflectors are returned in refl (row c holds v for column c, zero if
// the step was skipped) so eigenvectors of H can be mapped back to A.
static void hessenberg(int n, std::vector<double>& h, std::vector<double>* refl = nullptr) {
  if (refl) refl->assign((size_t)n * n, 0.0);
  for (int c = 0; c < n - 2; ++c) {
    double alpha = 0.0;
    for (int i = c + 1; i < n; ++i) alpha += h[i * n + c] * h[i * n + c];
    alpha = std::sqrt(alpha);
    if (alpha == 0.0) continue;
    const double x0 = h[(c + 1) * n + c];
    const double beta = x0 >= 0 ? -alpha : alpha;
    std::vector<double> v(n, 0.0);
    v[c + 1] = x0 - beta;
    for (int i = c + 2; i < n; ++i) v[i] = h[i * n + c];
    double vv = 0.0;
    for (int i = c + 1; i < n; ++i) vv += v[i] * v[i];
    if (vv == 0.0) continue;
    if (refl)
      for (int i = 0; i < n; ++i) (*refl)[(size_t)c * n + i] = v[i];
    // H <- (I - 2 v v^T / vv) H (I - 2 v v^T / vv)
    for (int j = 0; j < n; ++j) {
      double s = 0.0;
      for (int i = c + 1; i < n; ++i) s += v[i] * h[i * n + j];
      s *= 2.0 / vv;
      for (int i = c + 1; i < n; ++i) h[i * n + j] -= s * v[i];
    }
    for (int i = 0; i < n; ++i) {
      double s = 0.0;
      for (int j = c + 1; j < n; ++j) s += h[i * n + j] * v[j];
      s *= 2.0 / vv;
      for (int j = c + 1; j < n; ++j) h[i * n + j] -= s * v[j];
    }
    for (int i = c + 2; i < n; ++i) h[i * n + c] = 0.0;
  }
}

// Householder reflector P = I - beta v v^T (v[0] = 1) of a 2- or 3-vector u,
// chosen so that P u is a multiple of e_1.  beta = 0 for u = 0.
static double reflector(int len, const double* u, double* v) {
  double nrm2 = 0.0;
  for (int i = 0; i < len; ++i) nrm2 += u[i] * u[i];
  v[0] = 1.0;
  for (int i = 1; i < len; ++i) v[i] = 0.0;
  if (nrm2 == 0.0) return 0.0;
  const double nrm = std::sqrt(nrm2);
  const double head = u[0] + (u[0] >= 0.0 ? nrm : -nrm);   // no cancellation
  double vv = 1.0;
  for (int i = 1; i < len; ++i) {
    v[i] = u[i] / head;
    vv += v[i] * v[i];
  }
  return 2.0 / vv;
}

// One Francis double-shift step (Golub & Van Loan, Alg. 7.5.1) on the
// unreduced window H[lo..hi, lo..hi] of the row-major n x n Hessenberg
// matrix a.  The shifts are the roots of x^2 - tr x + det; only the window is
// transformed, which is all the eigenvalues need.
static void francis_step(int n, std::vector<double>& a, int lo, int hi, double tr, double det) {
  auto H = [&](int i, int j) -> double& { return a[(size_t)i * n + j]; };
  // first column of (H - mu1 I)(H - mu2 I) restricted to the window
  double u[3];
  u[0] = H(lo, lo) * H(lo, lo) + H(lo, lo + 1) * H(lo + 1, lo) - tr * H(lo, lo) + det;
  u[1] = H(lo + 1, lo) * (H(lo, lo) + H(lo + 1, lo + 1) - tr);
  u[2] = H(lo + 1, lo) * H(lo + 2, lo + 1);
  double v[3];
  for (int k = lo; k <= hi - 1; ++k) {
    const int len = (k <= hi - 2) ? 3 : 2;
    const double beta = reflector(len, u, v);
    if (beta != 0.0) {
      // rows k..k+len-1 from the bulge column on
      for (int j = std::max(lo, k - 1); j <= hi; ++j) {
        double w = 0.0;
        for (int r = 0; r < len; ++r) w += v[r] * H(k + r, j);
        w *= beta;
        for (int r = 0; r < len; ++r) H(k + r, j) -= w * v[r];
      }
      // columns k..k+len-1 down to the row that becomes the next bulge
      const int last = std::min(k + len, hi);
      for (int i = lo; i <= last; ++i) {
        double w = 0.0;
        for (int r = 0; r < len; ++r) w += H(i, k + r) * v[r];
        w *= beta;
        for (int r = 0; r < len; ++r) H(i, k + r) -= w * v[r];
      }
    }
    if (k > lo) {   // the reflector has annihilated the old bulge below H(k, k-1)
      for (int r = 1; r < len; ++r) H(k + r, k - 1) = 0.0;
    }
    if (k <= hi - 2) {   // the next bulge: column k below the subdiagonal
      u[0] = H(k + 1, k);
      u[1] = H(k + 2, k);
      u[2] = (k + 3 <= hi) ? H(k + 3, k) : 0.0;
    }
  }
}

// Eigenvalues of a real 2 x 2 block [[p, q], [r, s]].
static void eig2(double p, double q, double r, double s, double* re, double* im) {
  const double half_tr = 0.5 * (p + s), half_diff = 0.5 * (p - s);
  const double disc = half_diff * half_diff + q * r;
  if (disc >= 0.0) {
    const double root = std::sqrt(disc);
    const double big = half_tr + (half_tr >= 0.0 ? root : -root);   // larger magnitude
    re[0] = big;
    re[1] = big != 0.0 ? (p * s - q * r) / big : 0.0;
    im[0] = im[1] = 0.0;
  } else {
    const double root = std::sqrt(-disc);
    re[0] = re[1] = half_tr;
    im[0] = root;
    im[1] = -root;
  }
}

// Eigenvalues of an upper Hessenberg matrix (row-major, destroyed) by the
// Francis double-shift QR algorithm with deflation (Golub & Van Loan,
// Alg. 7.5.2): subdiagonal entries below eps * (|h_ii| + |h_{i-1,i-1}|) are
// set to zero, a trailing 1 x 1 or 2 x 2 block is read off, otherwise the
// trailing unreduced window takes a Francis step shifted by the eigenvalues
// of its last 2 x 2 block.  Every tenth step without deflation uses an ad hoc
// pair of complex shifts displaced from the corner by the size of the last
// two subdiagonals, to break cycles.  Returns false after 60 steps without
// deflation.
static bool hqr(int n, std::vector<double>& a, std::vector<double>& wr, std::vector<double>& wi) {
  auto H = [&](int i, int j) -> double& { return a[(size_t)i * n + j]; };
  const double eps = 2.220446049250313e-16;
  double hnorm = 0.0;
  for (double x : a) hnorm = std::max(hnorm, std::fabs(x));
  int hi = n - 1, steps = 0;
  while (hi >= 0) {
    int lo = hi;
    while (lo > 0) {
      double ref = std::fabs(H(lo, lo)) + std::fabs(H(lo - 1, lo - 1));
      if (ref == 0.0) ref = hnorm;
      if (std::fabs(H(lo, lo - 1)) <= eps * ref) {
        H(lo, lo - 1) = 0.0;
        break;
      }
      --lo;
    }
    if (lo == hi) {
      wr[hi] = H(hi, hi);
      wi[hi] = 0.0;
      hi -= 1;
      steps = 0;
      continue;
    }
    if (lo == hi - 1) {
      double re[2], im[2];
      eig2(H(hi - 1, hi - 1), H(hi - 1, hi), H(hi, hi - 1), H(hi, hi), re, im);
      wr[hi - 1] = re[0];
      wi[hi - 1] = im[0];
      wr[hi] = re[1];
      wi[hi] = im[1];
      hi -= 2;
      steps = 0;
      continue;
    }
    if (steps == 60) return false;
    ++steps;
    double tr, det;
    if (steps % 10 == 0) {
      const double d = std::fabs(H(hi, hi - 1)) + std::fabs(H(hi - 1, hi - 2));
      const double cre = H(hi, hi) + 0.5 * d, cim = 0.8 * d;
      tr = 2.0 * cre;
      det = cre * cre + cim * cim;
    } else {
      tr = H(hi - 1, hi - 1) + H(hi, hi);
      det = H(hi - 1, hi - 1) * H(hi, hi) - H(hi - 1, hi) * H(hi, hi - 1);
    }
    francis_step(n, a, lo, hi, tr, det);
  }
  return true;
}

// Eigenvector of M (n x n) for eigenvalue lam by inverse iteration on its
// upper Hessenberg form Hs = P^T M P (row-major): Gaussian elimination with
// partial pivoting needs only adjacent-row swaps on a Hessenberg matrix
// (O(n^2) per solve); zero pivots are replaced by eps*||Hs||.  The result is
// mapped back to M's basis with the reflectors of the reduction.
static std::vector<cd> inverse_iteration(int n, const std::vector<double>& Hs, const std::vector<double>& refl,
                                         cd lam) {
  double mnorm = 0.0;
  for (double v : Hs) mnorm = std::max(mnorm, std::fabs(v));
  mnorm = std::max(mnorm, std::abs(lam));
  const double tiny = 2.220446049250313e-16 * (mnorm > 0 ? mnorm : 1.0);
  std::vector<cd> a((size_t)n * n);
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < n; ++j) a[(size_t)i * n + j] = cd(Hs[(size_t)i * n + j], 0.0) - (i == j ? lam : cd(0));
  std::vector<cd> mult(n, cd(0));
  std::vector<char> swp(n, 0);
  for (int c = 0; c < n - 1; ++c) {
    const int lo = std::max(c - 1, 0);   // row c and c+1 are nonzero from column c-1 on
    if (std::abs(a[(size_t)(c + 1) * n + c]) > std::abs(a[(size_t)c * n + c])) {
      swp[c] = 1;
      for (int j = lo; j < n; ++j) std::swap(a[(size_t)c * n + j], a[(size_t)(c + 1) * n + j]);
    }
    if (std::abs(a[(size_t)c * n + c]) < tiny) a[(size_t)c * n + c] = tiny;
    const cd f = a[(size_t)(c + 1) * n + c] / a[(size_t)c * n + c];
    mult[c] = f;
    a[(size_t)(c + 1) * n + c] = 0.0;
    for (int j = c + 1; j < n; ++j) a[(size_t)(c + 1) * n + j] -= f * a[(size_t)c * n + j];
  }
  if (std::abs(a[(size_t)(n - 1) * n + n - 1]) < tiny) a[(size_t)(n - 1) * n + n - 1] = tiny;
  std::vector<cd> v(n);
  for (int i = 0; i < n; ++i) v[i] = cd(1.0 + 0.01 * i, 0.0);
  for (int it = 0; it < 3; ++it) {
    for (int c = 0; c < n - 1; ++c) {
      if (swp[c]) std::swap(v[c], v[c + 1]);
      v[c + 1] -= mult[c] * v[c];
    }
    for (int i = n - 1; i >= 0; --i) {
      cd s = v[i];
      for (int j = i + 1; j < n; ++j) s -= a[(size_t)i * n + j] * v[j];
      v[i] = s / a[(size_t)i * n + i];
    }
    double nrm = 0.0;
    for (auto& z : v) nrm += std::norm(z);
    nrm = std::sqrt(nrm);
    if (!(nrm > 0) || !std::isfinite(nrm)) break;
    int im = 0;
    for (int i = 1; i < n; ++i)
      if (std::abs(v[i]) > std::abs(v[im])) im = i;
    const cd ph = std::conj(v[im]) / std::abs(v[im]);
    for (auto& z : v) z = z * ph / nrm;
  }
  // z = P_0 P_1 ... P_{n-3} v
  for (int c = n - 3; c >= 0; --c) {
    const double* u = &refl[(size_t)c * n];
    double uu = 0.0;
    for (int i = c + 1; i < n; ++i) uu += u[i] * u[i];
    if (uu == 0.0) continue;
    cd s(0.0);
    for (int i = c + 1; i < n; ++i) s += u[i] * v[i];
    s *= 2.0 / uu;
    for (int i = c + 1; i < n; ++i) v[i] -= s * u[i];
  }
  return v;
}

// ---------------------------------------------------------------- symmetric eig
// Symmetric tridiagonal T (diagonal d, off-diagonal e[i] between i and i+1)
// to diagonal form by the symmetric QR algorithm (Golub & Van Loan,
// Alg. 8.3.3): negligible off-diagonals are set to zero, the trailing
// unreduced block takes one implicit QR step with the Wilkinson shift
// (Alg. 8.3.2), a Givens rotation in plane (k, k+1) chasing the bulge from
// the top of the block to its bottom.  Every rotation is applied to the
// columns of Q (row-major), so A = Q T Q^T is kept.  Returns false if the
// step count exceeds 60 per eigenvalue.
static bool tridiagonal_qr(int m, std::vector<double>& d, std::vector<double>& e, std::vector<double>& Q) {
  const double eps = 2.220446049250313e-16;
  int hi = m - 1, steps = 0;
  while (hi > 0) {
    for (int i = 0; i < hi; ++i)
      if (std::fabs(e[i]) <= eps * (std::fabs(d[i]) + std::fabs(d[i + 1]))) e[i] = 0.0;
    if (e[hi - 1] == 0.0) {
      --hi;
      continue;
    }
    int lo = hi - 1;
    while (lo > 0 && e[lo - 1] != 0.0) --lo;
    if (++steps > 60 * m) return false;
    // Wilkinson shift: the eigenvalue of the trailing 2 x 2 block nearer d[hi]
    const double delta = 0.5 * (d[hi - 1] - d[hi]);
    const double off = e[hi - 1];
    const double mu = d[hi] - off * off / (delta + std::copysign(std::hypot(delta, off), delta));
    // rotation G_k = [[c, s], [-s, c]] on rows/columns (k, k+1), T <- G T G^T
    double x = d[lo] - mu, z = e[lo];
    for (int k = lo; k < hi; ++k) {
      const double r = std::hypot(x, z);
      const double c = r > 0.0 ? x / r : 1.0, s = r > 0.0 ? z / r : 0.0;
      if (k > lo) e[k - 1] = r;   // the bulge at (k+1, k-1) is folded into e[k-1]
      const double dk = d[k], ek = e[k], dk1 = d[k + 1];
      d[k] = c * c * dk + 2.0 * c * s * ek + s * s * dk1;
      d[k + 1] = s * s * dk - 2.0 * c * s * ek + c * c * dk1;
      e[k] = c * s * (dk1 - dk) + (c * c - s * s) * ek;
      if (k + 1 < hi) {   // new bulge at (k+2, k); the next rotation removes it
        z = s * e[k + 1];
        e[k + 1] *= c;
        x = e[k];
      }
      for (int row = 0; row < m; ++row) {
        double* q = &Q[(size_t)row * m];
        const double qa = q[k], qb = q[k + 1];
        q[k] = c * qa + s * qb;
        q[k + 1] = c * qb - s * qa;
      }
    }
  }
  return true;
}

// Symmetric S (m x m, column-major) = V diag(lam) V^T: Householder reduction
// to tridiagonal form with the transformation accumulated (Golub & Van Loan,
// Sec. 8.3.1), then the symmetric QR algorithm above.
static bool sym_eig(int m, const std::vector<double>& S, std::vector<double>& lam, std::vector<double>& V) {
  // A row-major working copy; Q accumulates the reflections (A = Q T Q^T).
  std::vector<double> A(S);   // symmetric: row- and column-major coincide
  std::vector<double> Q((size_t)m * m, 0.0);
  for (int i = 0; i < m; ++i) Q[(size_t)i * m + i] = 1.0;
  auto a = [&](int i, int j) -> double& { return A[(size_t)i * m + j]; };
  std::vector<double> v(m), p(m), w(m);
  for (int k = 0; k < m - 2; ++k) {
    double alpha = 0.0;
    for (int i = k + 1; i < m; ++i) alpha += a(i, k) * a(i, k);
    alpha = std::sqrt(alpha);
    if (alpha == 0.0) continue;
    const double x0 = a(k + 1, k);
    const double beta0 = x0 >= 0 ? -alpha : alpha;
    std::fill(v.begin(), v.end(), 0.0);
    v[k + 1] = x0 - beta0;
    for (int i = k + 2; i < m; ++i) v[i] = a(i, k);
    double vv = 0.0;
    for (int i = k + 1; i < m; ++i) vv += v[i] * v[i];
    if (vv == 0.0) continue;
    const double beta = 2.0 / vv;
    // p = beta A22 v, w = p - (beta p^T v / 2) v, A22 -= v w^T + w v^T
    double pv = 0.0;
    for (int i = k + 1; i < m; ++i) {
      double s = 0.0;
      for (int j = k + 1; j < m; ++j) s += a(i, j) * v[j];
      p[i] = beta * s;
      pv += p[i] * v[i];
    }
    const double c = 0.5 * beta * pv;
    for (int i = k + 1; i < m; ++i) w[i] = p[i] - c * v[i];
    for (int i = k + 1; i < m; ++i)
      for (int j = k + 1; j < m; ++j) a(i, j) -= v[i] * w[j] + w[i] * v[j];
    a(k + 1, k) = a(k, k + 1) = beta0;
    for (int i = k + 2; i < m; ++i) a(i, k) = a(k, i) = 0.0;
    // Q <- Q (I - beta v v^T)
    for (int r = 0; r < m; ++r) {
      double s = 0.0;
      for (int j = k + 1; j < m; ++j) s += Q[(size_t)r * m + j] * v[j];
      s *= beta;
      for (int j = k + 1; j < m; ++j) Q[(size_t)r * m + j] -= s * v[j];
    }
  }
  std::vector<double> d(m), e(m, 0.0);
  for (int i = 0; i < m; ++i) d[i] = a(i, i);
  for (int i = 0; i + 1 < m; ++i) e[i] = a(i + 1, i);   // e[i] couples i and i+1
  if (!tridiagonal_qr(m, d, e, Q)) return false;
  lam = d;
  V.assign((size_t)m * m, 0.0);
  for (int i = 0; i < m; ++i)
    for (int j = 0; j < m; ++j) V[i + (size_t)j * m] = Q[(size_t)i * m + j];   // column j = eigenvector j
  return true;
}

// ---------------------------------------------------------------- harmonic Ritz
int harmonic_ritz(int m, const double* G, const double* Hm, int k, double tol_rank, double* Y,
                  double* th_re, double* th_im) {
  if (m <= 0 || k <= 0) return 0;
  // column scaling to unit ||Z e_j||
  std::vector<double> d(m, 0.0);
  for (int j = 0; j < m; ++j) {
    const double g = G[j + (size_t)j * m];
    d[j] = g > 0 ? 1.0 / std::sqrt(g) : 0.0;
  }
  std::vector<double> Gs((size_t)m * m), Hs((size_t)m * m);
  for (int j = 0; j < m; ++j)
    for (int i = 0; i < m; ++i) {
      Gs[i + (size_t)j * m] = d[i] * G[i + (size_t)j * m] * d[j];
      Hs[i + (size_t)j * m] = d[i] * Hm[i + (size_t)j * m] * d[j];
    }
  // Restrict the pencil to the dominant eigenspace of Gs: Gs = V L V^T by
  // the symmetric eigendecomposition above; keep eigenvalues > tol_rank * max (numerical
  // rank of W); with T = V_r L_r^{-1/2}, M = T^T Hs T and M z = (1/theta) z.
  std::vector<double> lam, V;
  if (!sym_eig(m, Gs, lam, V)) return -1;
  double lmax = 0.0;
  for (double v : lam) lmax = std::max(lmax, v);
  if (!(lmax > 0)) return 0;
  std::vector<int> keep;
  for (int j = 0; j < m; ++j)
    if (lam[j] > tol_rank * lmax) keep.push_back(j);
  const int r = (int)keep.size();
  if (r == 0) return 0;
  std::vector<double> T((size_t)m * r);   // column-major m x r
  for (int c = 0; c < r; ++c) {
    const double f = 1.0 / std::sqrt(lam[keep[c]]);
    for (int i = 0; i < m; ++i) T[i + (size_t)c * m] = V[i + (size_t)keep[c] * m] * f;
  }
  // HT = Hs T (m x r), then B = T^T HT (r x r, row-major)
  std::vector<double> HT((size_t)m * r, 0.0);
  for (int c = 0; c < r; ++c)
    for (int j = 0; j < m; ++j) {
      const double t = T[j + (size_t)c * m];
      if (t == 0.0) continue;
      for (int i = 0; i < m; ++i) HT[i + (size_t)c * m] += Hs[i + (size_t)j * m] * t;
    }
  std::vector<double> B((size_t)r * r, 0.0);
  for (int a = 0; a < r; ++a)
    for (int c = 0; c < r; ++c) {
      double acc = 0.0;
      for (int i = 0; i < m; ++i) acc += T[i + (size_t)a * m] * HT[i + (size_t)c * m];
      B[(size_t)a * r + c] = acc;
    }
  std::vector<double> Hh = B, wr(r), wi(r), refl;
  hessenberg(r, Hh, &refl);
  const std::vector<double> Hhess = Hh;   // hqr works in place
  if (!hqr(r, Hh, wr, wi)) return -1;
  // theta = 1 / mu; units: real values, or pairs represented by Im(theta) > 0
  struct Unit {
    double mag, re;
    int cplx;
    cd mu;
  };
  std::vector<Unit> units;
  for (int j = 0; j < r; ++j) {
    const cd mu(wr[j], wi[j]);
    if (mu == cd(0.0)) continue;
    const cd th = 1.0 / mu;
    if (wi[j] == 0.0) units.push_back({std::abs(th), th.real(), 0, mu});
    else if (th.imag() > 0.0) units.push_back({std::abs(th), th.real(), 1, mu});
  }
  std::stable_sort(units.begin(), units.end(), [](const Unit& a, const Unit& b) {
    if (a.mag != b.mag) return a.mag < b.mag;
    return a.re < b.re;
  });
  int used = 0;
  for (const Unit& u : units) {
    const int need = u.cplx ? 2 : 1;
    if (used + need > k) break;
    std::vector<cd> z = inverse_iteration(r, Hhess, refl, u.mu);
    // y = d .* (T z)
    std::vector<cd> y(m, cd(0.0));
    for (int c = 0; c < r; ++c)
      for (int i = 0; i < m; ++i) y[i] += T[i + (size_t)c * m] * z[c];
    for (int i = 0; i < m; ++i) y[i] *= d[i];
    const cd th = 1.0 / u.mu;
    for (int i = 0; i < m; ++i) Y[i + (size_t)used * m] = y[i].real();
    if (th_re) th_re[used] = th.real();
    if (th_im) th_im[used] = th.imag();
    if (u.cplx) {
      for (int i = 0; i < m; ++i) Y[i + (size_t)(used + 1) * m] = y[i].imag();
      if (th_re) th_re[used + 1] = th.real();
      if (th_im) th_im[used + 1] = -th.imag();
    }
    used += need;
    if (used == k) break;
  }
  return used;
}

}  // namespace rb
