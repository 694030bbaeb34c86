// Dense float64 building blocks of the host-side multifrontal Cholesky.
#include "dense.hpp"

#include <algorithm>
#include <cmath>
#include <vector>

namespace hqn {

namespace {

constexpr int KC = 256;  // k-chunk kept in L1 by the 4x4 register block

// 4x4 block of C += alpha * A B^T over k in [k0, k1)
inline void block4x4(const double *A, int lda, const double *B, int ldb, int k0, int k1,
                     double acc[4][4]) {
    const double *a0 = A, *a1 = A + lda, *a2 = A + 2 * lda, *a3 = A + 3 * lda;
    const double *b0 = B, *b1 = B + ldb, *b2 = B + 2 * ldb, *b3 = B + 3 * ldb;
    double c00 = 0, c01 = 0, c02 = 0, c03 = 0, c10 = 0, c11 = 0, c12 = 0, c13 = 0;
    double c20 = 0, c21 = 0, c22 = 0, c23 = 0, c30 = 0, c31 = 0, c32 = 0, c33 = 0;
    for (int k = k0; k < k1; ++k) {
        const double x0 = a0[k], x1 = a1[k], x2 = a2[k], x3 = a3[k];
        const double y0 = b0[k], y1 = b1[k], y2 = b2[k], y3 = b3[k];
        c00 += x0 * y0; c01 += x0 * y1; c02 += x0 * y2; c03 += x0 * y3;
        c10 += x1 * y0; c11 += x1 * y1; c12 += x1 * y2; c13 += x1 * y3;
        c20 += x2 * y0; c21 += x2 * y1; c22 += x2 * y2; c23 += x2 * y3;
        c30 += x3 * y0; c31 += x3 * y1; c32 += x3 * y2; c33 += x3 * y3;
    }
    acc[0][0] += c00; acc[0][1] += c01; acc[0][2] += c02; acc[0][3] += c03;
    acc[1][0] += c10; acc[1][1] += c11; acc[1][2] += c12; acc[1][3] += c13;
    acc[2][0] += c20; acc[2][1] += c21; acc[2][2] += c22; acc[2][3] += c23;
    acc[3][0] += c30; acc[3][1] += c31; acc[3][2] += c32; acc[3][3] += c33;
}

inline double dot(const double *a, const double *b, int n) {
    double s0 = 0, s1 = 0, s2 = 0, s3 = 0;
    int k = 0;
    for (; k + 4 <= n; k += 4) {
        s0 += a[k] * b[k]; s1 += a[k + 1] * b[k + 1];
        s2 += a[k + 2] * b[k + 2]; s3 += a[k + 3] * b[k + 3];
    }
    for (; k < n; ++k) s0 += a[k] * b[k];
    return (s0 + s1) + (s2 + s3);
}

}  // namespace

void gemm_nt(int m, int n, int K, double alpha, const double *A, int lda, const double *B,
             int ldb, double beta, double *C, int ldc, bool lower) {
    if (m <= 0 || n <= 0) return;
    if (beta != 1.0) {
#pragma omp parallel for schedule(static) if (m > 64)
        for (int i = 0; i < m; ++i) {
            int jn = lower ? std::min(n, i + 1) : n;
            for (int j = 0; j < jn; ++j) C[(size_t)i * ldc + j] *= beta;
        }
    }
    if (K <= 0 || alpha == 0.0) return;
    const int mb = (m + 3) / 4;
    for (int k0 = 0; k0 < K; k0 += KC) {
        const int k1 = std::min(K, k0 + KC);
#pragma omp parallel for schedule(dynamic, 4) if ((double)m * n * (k1 - k0) > 2e6)
        for (int ib = 0; ib < mb; ++ib) {
            const int i0 = ib * 4;
            const int ni = std::min(4, m - i0);
            const int jend = lower ? std::min(n, i0 + ni) : n;
            for (int j0 = 0; j0 < jend; j0 += 4) {
                const int nj = std::min(4, jend - j0);
                if (ni == 4 && nj == 4) {
                    double acc[4][4] = {};
                    block4x4(A + (size_t)i0 * lda, lda, B + (size_t)j0 * ldb, ldb, k0, k1, acc);
                    for (int a = 0; a < 4; ++a)
                        for (int b = 0; b < 4; ++b) {
                            if (lower && j0 + b > i0 + a) continue;
                            C[(size_t)(i0 + a) * ldc + j0 + b] += alpha * acc[a][b];
                        }
                } else {
                    for (int a = 0; a < ni; ++a)
                        for (int b = 0; b < nj; ++b) {
                            if (lower && j0 + b > i0 + a) continue;
                            double s = dot(A + (size_t)(i0 + a) * lda + k0,
                                           B + (size_t)(j0 + b) * ldb + k0, k1 - k0);
                            C[(size_t)(i0 + a) * ldc + j0 + b] += alpha * s;
                        }
                }
            }
        }
    }
}

int potrf_lower(int n, double *A, int lda) {
    constexpr int NB = 64;
    for (int k0 = 0; k0 < n; k0 += NB) {
        const int nb = std::min(NB, n - k0);
        // unblocked factor of the diagonal block (already updated by earlier panels)
        for (int j = k0; j < k0 + nb; ++j) {
            double *rj = A + (size_t)j * lda;
            double d = rj[j] - dot(rj + k0, rj + k0, j - k0);
            if (!(d > 0.0) || !std::isfinite(d)) return j + 1;
            d = std::sqrt(d);
            rj[j] = d;
            for (int i = j + 1; i < k0 + nb; ++i) {
                double *ri = A + (size_t)i * lda;
                ri[j] = (ri[j] - dot(ri + k0, rj + k0, j - k0)) / d;
            }
        }
        const int rest = n - k0 - nb;
        if (rest <= 0) continue;
        // panel below: P := P L_kk^{-T}
        trsm_right_lower_t(rest, nb, A + (size_t)k0 * lda + k0, lda,
                           A + (size_t)(k0 + nb) * lda + k0, lda);
        // trailing update: A22 -= P P^T (lower)
        gemm_nt(rest, rest, nb, -1.0, A + (size_t)(k0 + nb) * lda + k0, lda,
                A + (size_t)(k0 + nb) * lda + k0, lda, 1.0,
                A + (size_t)(k0 + nb) * lda + k0 + nb, lda, true);
    }
    return 0;
}

void trsm_right_lower_t(int m, int n, const double *L, int ldl, double *B, int ldb) {
    if (m <= 0 || n <= 0) return;
    constexpr int NB = 64;
    for (int j0 = 0; j0 < n; j0 += NB) {
        const int nb = std::min(NB, n - j0);
        if (j0 > 0) {
            // B[:, j0:j0+nb] -= X[:, 0:j0] L[j0:j0+nb, 0:j0]^T
            gemm_nt(m, nb, j0, -1.0, B, ldb, L + (size_t)j0 * ldl, ldl, 1.0, B + j0, ldb, false);
        }
#pragma omp parallel for schedule(static) if (m > 256)
        for (int i = 0; i < m; ++i) {
            double *bi = B + (size_t)i * ldb;
            for (int j = j0; j < j0 + nb; ++j) {
                const double *lj = L + (size_t)j * ldl;
                bi[j] = (bi[j] - dot(bi + j0, lj + j0, j - j0)) / lj[j];
            }
        }
    }
}

void trtri_lower_t(int n, const double *L, int ldl, double *LinvT, int ldi) {
    // column j of L^{-1} solves L x = e_j: x_i = 0 (i < j), x_j = 1/L_jj,
    // x_i = -(sum_{j<=k<i} L_ik x_k) / L_ii.  Stored as row j of LinvT.
#pragma omp parallel for schedule(dynamic, 8) if (n > 128)
    for (int j = 0; j < n; ++j) {
        double *x = LinvT + (size_t)j * ldi;
        for (int i = 0; i < j; ++i) x[i] = 0.0;
        x[j] = 1.0 / L[(size_t)j * ldl + j];
        for (int i = j + 1; i < n; ++i) {
            const double *li = L + (size_t)i * ldl;
            x[i] = -dot(li + j, x + j, i - j) / li[i];
        }
    }
}

}  // namespace hqn
