// Small dense FP64 linear algebra on the host (m <= ~100), for the parts of
// the method that are a k x k or m x m problem:
//   * svd_small: the biorthogonalisation of C and C~ (Alg. 2 step 1 requires
//     C~^T C diagonal and positive, Sec. 3): one-sided Jacobi SVD (Hestenes).
//   * harmonic_ritz: the eigenproblem of the recycle update between cycles
//     (Sec. 6.2): column scaling, restriction to the numerical range of W by
//     a cyclic Jacobi eigendecomposition of the scaled G = Z^T Z, reduction to
//     a standard problem, Householder-Hessenberg + Francis double-shift QR for
//     the eigenvalues (Golub & Van Loan, Matrix Computations, Sec. 7.4-7.5),
//     and complex inverse iteration for the selected eigenvectors.
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
// reflections (eigenvalues only, no accumulation).
static void hessenberg(int n, std::vector<double>& h) {
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

// Eigenvector of M (n x n row-major) for eigenvalue lam by inverse iteration
// with complex LU (partial pivoting); zero pivots are replaced by eps*||M||.
static std::vector<cd> inverse_iteration(int n, const std::vector<double>& M, cd lam) {
  double mnorm = 0.0;
  for (double v : M) mnorm = std::max(mnorm, std::fabs(v));
  mnorm = std::max(mnorm, std::abs(lam));
  const double tiny = 2.220446049250313e-16 * (mnorm > 0 ? mnorm : 1.0);
  std::vector<cd> a((size_t)n * n);
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < n; ++j) a[(size_t)i * n + j] = cd(M[(size_t)i * n + j], 0.0) - (i == j ? lam : cd(0));
  std::vector<int> piv(n);
  for (int c = 0; c < n; ++c) {
    int pr = c;
    double best = std::abs(a[(size_t)c * n + c]);
    for (int i = c + 1; i < n; ++i)
      if (std::abs(a[(size_t)i * n + c]) > best) {
        best = std::abs(a[(size_t)i * n + c]);
        pr = i;
      }
    piv[c] = pr;
    if (pr != c)
      for (int j = 0; j < n; ++j) std::swap(a[(size_t)c * n + j], a[(size_t)pr * n + j]);
    if (std::abs(a[(size_t)c * n + c]) < tiny) a[(size_t)c * n + c] = tiny;
    for (int i = c + 1; i < n; ++i) {
      const cd f = a[(size_t)i * n + c] / a[(size_t)c * n + c];
      a[(size_t)i * n + c] = f;
      for (int j = c + 1; j < n; ++j) a[(size_t)i * n + j] -= f * a[(size_t)c * n + j];
    }
  }
  std::vector<cd> v(n);
  for (int i = 0; i < n; ++i) v[i] = cd(1.0 + 0.01 * i, 0.0);
  for (int it = 0; it < 3; ++it) {
    for (int c = 0; c < n; ++c) std::swap(v[c], v[piv[c]]);
    for (int i = 0; i < n; ++i)
      for (int j = 0; j < i; ++j) v[i] -= a[(size_t)i * n + j] * v[j];
    for (int i = n - 1; i >= 0; --i) {
      for (int j = i + 1; j < n; ++j) v[i] -= a[(size_t)i * n + j] * v[j];
      v[i] /= a[(size_t)i * n + i];
    }
    double nrm = 0.0;
    for (auto& z : v) nrm += std::norm(z);
    nrm = std::sqrt(nrm);
    if (!(nrm > 0) || !std::isfinite(nrm)) break;
    // phase-fix: largest component real positive
    int im = 0;
    for (int i = 1; i < n; ++i)
      if (std::abs(v[i]) > std::abs(v[im])) im = i;
    const cd ph = std::conj(v[im]) / std::abs(v[im]);
    for (auto& z : v) z = z * ph / nrm;
  }
  return v;
}

// ---------------------------------------------------------------- symmetric eig
// Cyclic Jacobi eigenvalue algorithm (Golub & Van Loan, Sec. 8.5) for a
// symmetric m x m matrix (column-major): S = V diag(lam) V^T.
static void jacobi_eig(int m, const std::vector<double>& S, std::vector<double>& lam,
                       std::vector<double>& V) {
  std::vector<double> A = S;
  V.assign((size_t)m * m, 0.0);
  for (int i = 0; i < m; ++i) V[i + (size_t)i * m] = 1.0;
  auto a = [&](int i, int j) -> double& { return A[i + (size_t)j * m]; };
  const double eps = 2.220446049250313e-16;
  for (int sweep = 0; sweep < 100; ++sweep) {
    double off = 0.0, diag = 0.0;
    for (int j = 0; j < m; ++j) {
      diag += a(j, j) * a(j, j);
      for (int i = 0; i < j; ++i) off += 2.0 * a(i, j) * a(i, j);
    }
    if (off <= eps * eps * diag || off == 0.0) break;
    for (int p = 0; p < m - 1; ++p)
      for (int q = p + 1; q < m; ++q) {
        const double apq = a(p, q);
        if (std::fabs(apq) <= 1e-300) continue;
        if (std::fabs(apq) <= eps * 1e-3 * std::sqrt(std::fabs(a(p, p) * a(q, q)))) {
          a(p, q) = a(q, p) = 0.0;
          continue;
        }
        const double theta = (a(q, q) - a(p, p)) / (2.0 * apq);
        const double t = (theta >= 0 ? 1.0 : -1.0) / (std::fabs(theta) + std::sqrt(1.0 + theta * theta));
        const double c = 1.0 / std::sqrt(1.0 + t * t), s = t * c;
        for (int k = 0; k < m; ++k) {
          const double akp = a(k, p), akq = a(k, q);
          a(k, p) = c * akp - s * akq;
          a(k, q) = s * akp + c * akq;
        }
        for (int k = 0; k < m; ++k) {
          const double apk = a(p, k), aqk = a(q, k);
          a(p, k) = c * apk - s * aqk;
          a(q, k) = s * apk + c * aqk;
        }
        for (int k = 0; k < m; ++k) {
          const double vkp = V[k + (size_t)p * m], vkq = V[k + (size_t)q * m];
          V[k + (size_t)p * m] = c * vkp - s * vkq;
          V[k + (size_t)q * m] = s * vkp + c * vkq;
        }
      }
  }
  lam.resize(m);
  for (int i = 0; i < m; ++i) lam[i] = a(i, i);
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
  jacobi_eig(m, Gs, lam, V);
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
  std::vector<double> Hh = B, wr(r), wi(r);
  hessenberg(r, Hh);
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
    std::vector<cd> z = inverse_iteration(r, B, u.mu);
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
