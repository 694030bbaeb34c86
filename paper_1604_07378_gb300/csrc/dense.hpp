// Dense float64 kernels for the host-side supernodal Cholesky factorisation of
// A0 = M/h^2 + L (the prefactored initial Hessian of Sec. 4.2).  Row-major
// storage, leading dimensions in elements.  OpenMP-parallel over output rows.
#pragma once

namespace hqn {

// C[i][j] = beta * C[i][j] + alpha * sum_{k<K} A[i][k] * B[j][k]
// for i < m, j < n; with lower = true only j <= i is touched (m == n).
void gemm_nt(int m, int n, int K, double alpha, const double *A, int lda,
             const double *B, int ldb, double beta, double *C, int ldc, bool lower);

// In-place Cholesky A = L L^T of the lower triangle (upper part untouched).
// Returns 0, or j + 1 if the j-th pivot is not positive.
int potrf_lower(int n, double *A, int lda);

// B := B L^{-T} for B (m x n) and lower-triangular L (n x n).
void trsm_right_lower_t(int m, int n, const double *L, int ldl, double *B, int ldb);

// LinvT := (L^{-1})^T, i.e. row j of LinvT is column j of L^{-1} (upper triangular).
void trtri_lower_t(int n, const double *L, int ldl, double *LinvT, int ldi);

}  // namespace hqn
