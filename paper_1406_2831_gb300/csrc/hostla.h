// Host-side small dense FP64 linear algebra (see hostla.cpp).
#pragma once

namespace rb {

// M (k x k, column-major) = P diag(sigma) Q^T, sigma descending.
void svd_small(int k, const double* M, double* P, double* sigma, double* Q);

// Harmonic Ritz coefficients: G = Z^T Z, H = Z^T W (m x m, column-major).
// Writes up to k columns of Y (m x k, ld m) and theta (re, im); returns the
// number of columns written, or -1 if the QR iteration failed.
int harmonic_ritz(int m, const double* G, const double* H, int k, double tol_rank, double* Y,
                  double* th_re, double* th_im);

}  // namespace rb
