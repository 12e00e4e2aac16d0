// host_linalg.h -- small dense FP64 linear algebra on the host for the k x k
// and m x m matrices of the sm_103a library (POD Gram matrices, Rayleigh-Ritz
// matrices of the eigensolver): cyclic Jacobi eigen-decomposition, Cholesky
// and the inverse of a triangular factor.
#pragma once
#include <algorithm>
#include <cmath>
#include <vector>

namespace hla {

// host: cyclic Jacobi eigen-decomposition of a symmetric m x m matrix
// (row-major); eigenvalues descending in w, eigenvectors as columns of V
inline void jacobi_eig(int n, std::vector<double> &A, std::vector<double> &w, std::vector<double> &V) {
  V.assign((size_t)n * n, 0.0);
  for (int i = 0; i < n; ++i) V[(size_t)i * n + i] = 1.0;
  for (int sweep = 0; sweep < 100; ++sweep) {
    double off = 0.0, tot = 0.0;
    for (int i = 0; i < n; ++i)
      for (int j = 0; j < n; ++j) {
        const double a = A[(size_t)i * n + j];
        tot += a * a;
        if (i != j) off += a * a;
      }
    if (off <= 1e-30 * tot) break;
    for (int p = 0; p < n - 1; ++p)
      for (int q = p + 1; q < n; ++q) {
        const double apq = A[(size_t)p * n + q];
        if (apq == 0.0) continue;
        const double app = A[(size_t)p * n + p], aqq = A[(size_t)q * n + q];
        const double theta = (aqq - app) / (2.0 * apq);
        const double t = (theta >= 0 ? 1.0 : -1.0) / (std::fabs(theta) + std::sqrt(theta * theta + 1.0));
        const double c = 1.0 / std::sqrt(t * t + 1.0), s = t * c;
        for (int k = 0; k < n; ++k) {
          const double akp = A[(size_t)k * n + p], akq = A[(size_t)k * n + q];
          A[(size_t)k * n + p] = c * akp - s * akq;
          A[(size_t)k * n + q] = s * akp + c * akq;
        }
        for (int k = 0; k < n; ++k) {
          const double apk = A[(size_t)p * n + k], aqk = A[(size_t)q * n + k];
          A[(size_t)p * n + k] = c * apk - s * aqk;
          A[(size_t)q * n + k] = s * apk + c * aqk;
        }
        for (int k = 0; k < n; ++k) {
          const double vkp = V[(size_t)k * n + p], vkq = V[(size_t)k * n + q];
          V[(size_t)k * n + p] = c * vkp - s * vkq;
          V[(size_t)k * n + q] = s * vkp + c * vkq;
        }
      }
  }
  std::vector<int> ord(n);
  for (int i = 0; i < n; ++i) ord[i] = i;
  std::stable_sort(ord.begin(), ord.end(), [&](int a, int b) {
    return A[(size_t)a * n + a] > A[(size_t)b * n + b];
  });
  std::vector<double> V2((size_t)n * n);
  w.resize(n);
  for (int j = 0; j < n; ++j) {
    w[j] = A[(size_t)ord[j] * n + ord[j]];
    for (int i = 0; i < n; ++i) V2[(size_t)i * n + j] = V[(size_t)i * n + ord[j]];
  }
  V.swap(V2);
}


// Cholesky A = L L^T of a symmetric positive definite n x n matrix (row-major,
// lower factor returned in L); false if a pivot is not positive.
inline bool cholesky(int n, const std::vector<double> &A, std::vector<double> &L) {
  L.assign((size_t)n * n, 0.0);
  for (int j = 0; j < n; ++j) {
    double d = A[(size_t)j * n + j];
    for (int q = 0; q < j; ++q) d -= L[(size_t)j * n + q] * L[(size_t)j * n + q];
    if (!(d > 0.0)) return false;
    const double ljj = std::sqrt(d);
    L[(size_t)j * n + j] = ljj;
    for (int i = j + 1; i < n; ++i) {
      double s = A[(size_t)i * n + j];
      for (int q = 0; q < j; ++q) s -= L[(size_t)i * n + q] * L[(size_t)j * n + q];
      L[(size_t)i * n + j] = s / ljj;
    }
  }
  return true;
}

// W = L^-T (upper triangular, row-major) for a lower-triangular L, so that
// X W has orthonormal columns when X^T X = L L^T.
inline void inv_lower_transpose(int n, const std::vector<double> &L, std::vector<double> &W) {
  std::vector<double> Li((size_t)n * n, 0.0);  // L^-1 (lower)
  for (int j = 0; j < n; ++j) {
    Li[(size_t)j * n + j] = 1.0 / L[(size_t)j * n + j];
    for (int i = j + 1; i < n; ++i) {
      double s = 0.0;
      for (int q = j; q < i; ++q) s += L[(size_t)i * n + q] * Li[(size_t)q * n + j];
      Li[(size_t)i * n + j] = -s / L[(size_t)i * n + i];
    }
  }
  W.assign((size_t)n * n, 0.0);
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < n; ++j) W[(size_t)i * n + j] = Li[(size_t)j * n + i];
}

}  // namespace hla
