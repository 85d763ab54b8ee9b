// Small dense FP64 linear algebra on the host (k x k with k <= a few hundred): symmetric
// eigen-decomposition, Cholesky, triangular inverse.
#pragma once

#include <cmath>
#include <vector>

namespace hydot {

// Symmetric eigen-decomposition by cyclic Jacobi rotations: A (n x n, row-major) -> eigenvalues in
// lam, eigenvectors in the columns of V.
inline void jacobi_eig(std::vector<double> A, int n, std::vector<double>& lam, std::vector<double>& V) {
  V.assign((size_t)n * n, 0.0);
  for (int i = 0; i < n; ++i) V[(size_t)i * n + i] = 1.0;
  for (int sweep = 0; sweep < 100; ++sweep) {
    double off = 0.0, tot = 0.0;
    for (int p = 0; p < n; ++p)
      for (int q = 0; q < n; ++q) {
        tot += A[(size_t)p * n + q] * A[(size_t)p * n + q];
        if (p != q) off += A[(size_t)p * n + q] * A[(size_t)p * n + q];
      }
    if (off <= 1e-30 * tot) break;
    for (int p = 0; p < n - 1; ++p)
      for (int q = p + 1; q < n; ++q) {
        const double apq = A[(size_t)p * n + q];
        if (std::fabs(apq) < 1e-300) continue;
        const double app = A[(size_t)p * n + p], aqq = A[(size_t)q * n + q];
        const double theta = (aqq - app) / (2.0 * apq);
        const double t = (theta >= 0 ? 1.0 : -1.0) / (std::fabs(theta) + std::sqrt(theta * theta + 1.0));
        const double c = 1.0 / std::sqrt(t * t + 1.0), s = t * c;
        for (int r = 0; r < n; ++r) {  // A <- J^T A J
          const double arp = A[(size_t)r * n + p], arq = A[(size_t)r * n + q];
          A[(size_t)r * n + p] = c * arp - s * arq;
          A[(size_t)r * n + q] = s * arp + c * arq;
        }
        for (int r = 0; r < n; ++r) {
          const double apr = A[(size_t)p * n + r], aqr = A[(size_t)q * n + r];
          A[(size_t)p * n + r] = c * apr - s * aqr;
          A[(size_t)q * n + r] = s * apr + c * aqr;
        }
        for (int r = 0; r < n; ++r) {
          const double vrp = V[(size_t)r * n + p], vrq = V[(size_t)r * n + q];
          V[(size_t)r * n + p] = c * vrp - s * vrq;
          V[(size_t)r * n + q] = s * vrp + c * vrq;
        }
      }
  }
  lam.resize(n);
  for (int i = 0; i < n; ++i) lam[i] = A[(size_t)i * n + i];
}

// Cholesky G = R^T R (upper R, row-major); false if not positive definite.
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
