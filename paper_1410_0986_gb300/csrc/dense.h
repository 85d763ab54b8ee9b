// Small dense FP64 linear algebra on the host (k x k with k <= a few hundred): symmetric
// eigen-decomposition, Cholesky, triangular inverse.
#pragma once

#include <cmath>
#include <vector>

namespace hydot {

// Symmetric eigen-decomposition by Householder reduction to tridiagonal form followed by the
// implicit-shift symmetric QR iteration (Wilkinson shift, Givens bulge chasing), with the
// transformations accumulated: A (n x n, row-major) -> eigenvalues in lam, eigenvectors in the
// columns of V (row-major, V[i*n + j] = component i of eigenvector j). O(n^3) with small constants
// (n = 320: ~0.1 s; a cyclic Jacobi method takes ~16x longer). Returns false when the QR
// iteration has not deflated every coupling after max_sweeps bulge chases (default 64 n; a
// symmetric tridiagonal matrix needs about 2 n), in which case lam and V are not valid.
inline bool sym_eig(std::vector<double> A, int n, std::vector<double>& lam, std::vector<double>& V,
                    long long max_sweeps = -1) {
  lam.assign(n, 0.0);
  V.assign((size_t)n * n, 0.0);
  if (n == 0) return true;
  if (max_sweeps < 0) max_sweeps = 64LL * n;
  auto a = [&](int i, int j) -> double& { return A[(size_t)i * n + j]; };
  // Q accumulated as a row-major matrix, starting from the identity
  std::vector<double> Q((size_t)n * n, 0.0);
  for (int i = 0; i < n; ++i) Q[(size_t)i * n + i] = 1.0;
  std::vector<double> v(n), w(n);
  // 1. Householder: for column k, reflect A[k+1:, k] onto a multiple of e_(k+1)
  for (int k = 0; k + 2 < n; ++k) {
    double alpha = 0.0;
    for (int i = k + 1; i < n; ++i) alpha += a(i, k) * a(i, k);
    alpha = std::sqrt(alpha);
    if (alpha == 0.0) continue;
    if (a(k + 1, k) > 0) alpha = -alpha;
    for (int i = 0; i < n; ++i) v[i] = 0.0;
    for (int i = k + 1; i < n; ++i) v[i] = a(i, k);
    v[k + 1] -= alpha;
    double vv = 0.0;
    for (int i = k + 1; i < n; ++i) vv += v[i] * v[i];
    if (vv == 0.0) continue;
    const double beta = 2.0 / vv;
    // A <- H A H with H = I - beta v v^T: w = beta A v, K = beta/2 v^T w, q = w - K v,
    // A <- A - v q^T - q v^T (only rows/columns k.. change)
    for (int i = k; i < n; ++i) {
      double sacc = 0.0;
      for (int j = k + 1; j < n; ++j) sacc += a(i, j) * v[j];
      w[i] = beta * sacc;
    }
    double K = 0.0;
    for (int i = k + 1; i < n; ++i) K += v[i] * w[i];
    K *= 0.5 * beta;
    for (int i = k; i < n; ++i) w[i] -= K * v[i];
    for (int i = k; i < n; ++i)
      for (int j = k; j < n; ++j) a(i, j) -= v[i] * w[j] + w[i] * v[j];
    // Q <- Q H
    for (int i = 0; i < n; ++i) {
      double sacc = 0.0;
      for (int j = k + 1; j < n; ++j) sacc += Q[(size_t)i * n + j] * v[j];
      sacc *= beta;
      for (int j = k + 1; j < n; ++j) Q[(size_t)i * n + j] -= sacc * v[j];
    }
  }
  // tridiagonal: diagonal d, off-diagonal e (e[i] couples i and i+1)
  std::vector<double> d(n), e(n, 0.0);
  for (int i = 0; i < n; ++i) d[i] = a(i, i);
  for (int i = 0; i + 1 < n; ++i) e[i] = a(i + 1, i);
  // 2. implicit symmetric QR on the unreduced trailing block [lo, hi]
  int hi = n - 1;
  long long guard = 0;
  while (hi > 0 && guard < max_sweeps) {
    ++guard;
    // deflate negligible couplings from the bottom
    if (std::fabs(e[hi - 1]) <= 1e-15 * (std::fabs(d[hi - 1]) + std::fabs(d[hi]))) {
      e[hi - 1] = 0.0;
      --hi;
      continue;
    }
    int lo = hi - 1;
    while (lo > 0 && std::fabs(e[lo - 1]) > 1e-15 * (std::fabs(d[lo - 1]) + std::fabs(d[lo]))) --lo;
    // Wilkinson shift from the trailing 2 x 2 block
    const double dd = 0.5 * (d[hi - 1] - d[hi]);
    const double ee = e[hi - 1];
    const double den = dd + (dd >= 0 ? 1.0 : -1.0) * std::sqrt(dd * dd + ee * ee);
    const double mu = d[hi] - (den != 0.0 ? ee * ee / den : 0.0);
    double x = d[lo] - mu, z = e[lo];
    for (int k = lo; k < hi; ++k) {
      // Givens rotation zeroing z against x
      const double r = std::hypot(x, z);
      const double c = r == 0.0 ? 1.0 : x / r, s = r == 0.0 ? 0.0 : z / r;
      if (k > lo) e[k - 1] = r;
      // apply G^T T G to rows/columns k, k+1 of the tridiagonal matrix
      const double dk = d[k], dk1 = d[k + 1], ek = e[k];
      d[k] = c * c * dk + 2 * c * s * ek + s * s * dk1;
      d[k + 1] = s * s * dk - 2 * c * s * ek + c * c * dk1;
      e[k] = (c * c - s * s) * ek + c * s * (dk1 - dk);
      if (k + 1 < hi) {
        z = s * e[k + 1];
        e[k + 1] *= c;
        x = e[k];
      }
      // accumulate into the eigenvector columns k, k+1
      for (int i = 0; i < n; ++i) {
        const double qk = Q[(size_t)i * n + k], qk1 = Q[(size_t)i * n + k + 1];
        Q[(size_t)i * n + k] = c * qk + s * qk1;
        Q[(size_t)i * n + k + 1] = -s * qk + c * qk1;
      }
    }
  }
  lam = d;
  V = Q;
  return hi == 0;
}

inline bool cholesky_upper(const std::vector<double>& G, int k, std::vector<double>& R) {
  R.assign((size_t)k * k, 0.0);
  for (int i = 0; i < k; ++i) {
    double s = G[(size_t)i * k + i];
    for (int p = 0; p < i; ++p) s -= R[(size_t)p * k + i] * R[(size_t)p * k + i];
    if (!(s > 0.0)) return false;
    R[(size_t)i * k + i] = std::sqrt(s);
    for (int j = i + 1; j < k; ++j) {
      double t = G[(size_t)i * k + j];
      for (int p = 0; p < i; ++p) t -= R[(size_t)p * k + i] * R[(size_t)p * k + j];
      R[(size_t)i * k + j] = t / R[(size_t)i * k + i];
    }
  }
  return true;
}

// inverse of an upper-triangular matrix
inline std::vector<double> tri_inv_upper(const std::vector<double>& R, int k) {
  std::vector<double> X((size_t)k * k, 0.0);
  for (int j = 0; j < k; ++j) {
    X[(size_t)j * k + j] = 1.0 / R[(size_t)j * k + j];
    for (int i = j - 1; i >= 0; --i) {
      double s = 0.0;
      for (int p = i + 1; p <= j; ++p) s += R[(size_t)i * k + p] * X[(size_t)p * k + j];
      X[(size_t)i * k + j] = -s / R[(size_t)i * k + i];
    }
  }
  return X;
}

}  // namespace hydot
