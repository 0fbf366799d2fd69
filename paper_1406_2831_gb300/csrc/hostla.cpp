// Small dense FP64 linear algebra on the host (m <= ~100), for the parts of
// the method that are a k x k or m x m problem:
//   * svd_small: the biorthogonalisation of C and C~ (Alg. 2 step 1 requires
//     C~^T C diagonal and positive, Sec. 3): one-sided Jacobi SVD (Hestenes).
//   * harmonic_ritz: the eigenproblem of the recycle update between cycles
//     (Sec. 6.2): column scaling, restriction to the numerical range of W by
//     a symmetric eigendecomposition of the scaled G = Z^T Z (Householder
//     tridiagonalisation + implicit QL), reduction to a standard problem,
//     Householder-Hessenberg + Francis double-shift QR for the eigenvalues
//     (Golub & Van Loan, Matrix Computations, Sec. 7.4-7.5), and complex
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

// Eigenvalues of an upper Hessenberg matrix by the Francis double-shift QR
// iteration with deflation on small subdiagonal entries.  Returns false if an
// eigenvalue needed more than 60 iterations.
static bool hqr(int n, std::vector<double>& a, std::vector<double>& wr, std::vector<double>& wi) {
  auto H = [&](int i, int j) -> double& { return a[(size_t)i * n + j]; };
  const double eps = 2.220446049250313e-16;
  double anorm = 0.0;
  for (int i = 0; i < n; ++i)
    for (int j = std::max(i - 1, 0); j < n; ++j) anorm += std::fabs(H(i, j));
  int nn = n - 1;
  double t = 0.0;
  while (nn >= 0) {
    int its = 0, l;
    for (;;) {
      for (l = nn; l >= 1; --l) {
        double s = std::fabs(H(l - 1, l - 1)) + std::fabs(H(l, l));
        if (s == 0.0) s = anorm;
        if (std::fabs(H(l, l - 1)) <= eps * s) {
          H(l, l - 1) = 0.0;
          break;
        }
      }
      double x = H(nn, nn);
      if (l == nn) {
        wr[nn] = x + t;
        wi[nn] = 0.0;
        --nn;
        break;
      }
      double y = H(nn - 1, nn - 1);
      double w = H(nn, nn - 1) * H(nn - 1, nn);
      if (l == nn - 1) {
        const double p = 0.5 * (y - x);
        const double q = p * p + w;
        const double z = std::sqrt(std::fabs(q));
        x += t;
        if (q >= 0.0) {
          const double zz = p + (p >= 0 ? z : -z);
          wr[nn - 1] = wr[nn] = x + zz;
          if (zz != 0.0) wr[nn] = x - w / zz;
          wi[nn - 1] = wi[nn] = 0.0;
        } else {
          wr[nn - 1] = wr[nn] = x + p;
          wi[nn - 1] = z;
          wi[nn] = -z;
        }
        nn -= 2;
        break;
      }
      if (its == 60) return false;
      if (its == 10 || its == 20 || its == 40) {
        t += x;
        for (int i = 0; i <= nn; ++i) H(i, i) -= x;
        const double s = std::fabs(H(nn, nn - 1)) + std::fabs(H(nn - 1, nn - 2));
        x = y = 0.75 * s;
        w = -0.4375 * s * s;
      }
      ++its;
      int m;
      double p = 0, q = 0, r = 0, z;
      for (m = nn - 2; m >= l; --m) {
        z = H(m, m);
        r = x - z;
        const double s0 = y - z;
        p = (r * s0 - w) / H(m + 1, m) + H(m, m + 1);
        q = H(m + 1, m + 1) - z - r - s0;
        r = H(m + 2, m + 1);
        const double s = std::fabs(p) + std::fabs(q) + std::fabs(r);
        p /= s;
        q /= s;
        r /= s;
        if (m == l) break;
        const double u = std::fabs(H(m, m - 1)) * (std::fabs(q) + std::fabs(r));
        const double v = std::fabs(p) * (std::fabs(H(m - 1, m - 1)) + std::fabs(z) + std::fabs(H(m + 1, m + 1)));
        if (u <= eps * v) break;
      }
      for (int i = m + 2; i <= nn; ++i) {
        H(i, i - 2) = 0.0;
        if (i != m + 2) H(i, i - 3) = 0.0;
      }
      for (int kk = m; kk <= nn - 1; ++kk) {
        if (kk != m) {
          p = H(kk, kk - 1);
          q = H(kk + 1, kk - 1);
          r = (kk != nn - 1) ? H(kk + 2, kk - 1) : 0.0;
          x = std::fabs(p) + std::fabs(q) + std::fabs(r);
          if (x != 0.0) {
            p /= x;
            q /= x;
            r /= x;
          }
        }
        const double ss = std::sqrt(p * p + q * q + r * r);
        const double s = p >= 0 ? ss : -ss;
        if (s == 0.0) continue;
        if (kk == m) {
          if (l != m) H(kk, kk - 1) = -H(kk, kk - 1);
        } else {
          H(kk, kk - 1) = -s * x;
        }
        p += s;
        x = p / s;
        y = q / s;
        z = r / s;
        q /= p;
        r /= p;
        for (int j = kk; j <= nn; ++j) {
          p = H(kk, j) + q * H(kk + 1, j);
          if (kk != nn - 1) {
            p += r * H(kk + 2, j);
            H(kk + 2, j) -= p * z;
          }
          H(kk + 1, j) -= p * y;
          H(kk, j) -= p * x;
        }
        const int mmin = nn < kk + 3 ? nn : kk + 3;
        for (int i = l; i <= mmin; ++i) {
          p = x * H(i, kk) + y * H(i, kk + 1);
          if (kk != nn - 1) {
            p += z * H(i, kk + 2);
            H(i, kk + 2) -= p * r;
          }
          H(i, kk + 1) -= p * q;
          H(i, kk) -= p;
        }
      }
    }
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
// Symmetric S (m x m, column-major) = V diag(lam) V^T: Householder reduction
// to tridiagonal form with the transformation accumulated (Golub & Van Loan,
// Sec. 8.3.1), then the implicit symmetric QL iteration with Wilkinson-type
// shifts on the tridiagonal matrix, rotating V along (Sec. 8.3.3).
static void sym_eig(int m, const std::vector<double>& S, std::vector<double>& lam, std::vector<double>& V) {
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
  const double eps = 2.220446049250313e-16;
  for (int l = 0; l < m; ++l) {
    for (int iter = 0; iter < 100; ++iter) {
      int mm = l;
      for (; mm < m - 1; ++mm) {
        const double dd = std::fabs(d[mm]) + std::fabs(d[mm + 1]);
        if (std::fabs(e[mm]) <= eps * dd) break;
      }
      if (mm == l) break;
      // shift from the leading 2x2 block, chase the bulge from mm up to l
      double g = (d[l + 1] - d[l]) / (2.0 * e[l]);
      double r = std::hypot(g, 1.0);
      g = d[mm] - d[l] + e[l] / (g + (g >= 0 ? r : -r));
      double s = 1.0, c = 1.0, pp = 0.0;
      int i = mm - 1;
      bool early = false;
      for (; i >= l; --i) {
        const double f = s * e[i], b = c * e[i];
        r = std::hypot(f, g);
        e[i + 1] = r;
        if (r == 0.0) {
          d[i + 1] -= pp;
          e[mm] = 0.0;
          early = true;
          break;
        }
        s = f / r;
        c = g / r;
        g = d[i + 1] - pp;
        r = (d[i] - g) * s + 2.0 * c * b;
        pp = s * r;
        d[i + 1] = g + pp;
        g = c * r - b;
        for (int k = 0; k < m; ++k) {
          const double qf = Q[(size_t)k * m + i + 1];
          Q[(size_t)k * m + i + 1] = s * Q[(size_t)k * m + i] + c * qf;
          Q[(size_t)k * m + i] = c * Q[(size_t)k * m + i] - s * qf;
        }
      }
      if (early) continue;
      d[l] -= pp;
      e[l] = g;
      e[mm] = 0.0;
    }
  }
  lam = d;
  V.assign((size_t)m * m, 0.0);
  for (int i = 0; i < m; ++i)
    for (int j = 0; j < m; ++j) V[i + (size_t)j * m] = Q[(size_t)i * m + j];   // column j = eigenvector j
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
  // cyclic Jacobi rotations; keep eigenvalues > tol_rank * max (numerical
  // rank of W); with T = V_r L_r^{-1/2}, M = T^T Hs T and M z = (1/theta) z.
  std::vector<double> lam, V;
  sym_eig(m, Gs, lam, V);
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
