// Per-tetrahedron mathematics of the energy/gradient kernel: deformation
// gradient from displacements, signed 3x3 SVD, Valanis-Landel stress in
// principal stretches (Eq. valanis-landel) and the corner gradients.
//
// Precision design.  The kernels store displacements u = x - X, so
// F = I + G with G = [u1-u0, u2-u0, u3-u0] Dm^{-1} carries the strain at the
// relative precision of the arithmetic instead of being the difference of two
// nearly equal absolute positions.  The symmetric eigenproblem is solved for
// S = F^T F - I = G + G^T + G^T G, whose eigenvalues are l_i = s_i^2 - 1, so
// every material below is written in terms of l_i and s_i and no term of
// size mu is cancelled against another near the rest state.
#pragma once

#include "common.cuh"

namespace hqn {

template <typename R> __device__ __forceinline__ R rsqrt_(R v);
template <> __device__ __forceinline__ float rsqrt_<float>(float v) { return rsqrtf(v); }
template <> __device__ __forceinline__ double rsqrt_<double>(double v) { return rsqrt(v); }

template <typename R> __device__ __forceinline__ R sqrt_(R v) { return sqrt(v); }
template <typename R> __device__ __forceinline__ R log1p_(R v) { return log1p(v); }
template <typename R> __device__ __forceinline__ R abs_(R v) { return fabs(v); }

template <typename R> struct Eps;
template <> struct Eps<float> { static constexpr float v = 1.1920929e-7f; };
template <> struct Eps<double> { static constexpr double v = 2.220446049250313e-16; };

// x - log(1 + x) without cancellation: for |x| < 0.1 its Taylor series
// sum_{k>=2} (-1)^k x^k / k in Horner form, x^2 (1/2 - x (1/3 - x (1/4 - ...))),
// truncated where the next term is below the precision of R (k <= 9 in float,
// k <= 18 in double); the direct form elsewhere.
template <typename R> struct LogSeries;
template <> struct LogSeries<float> { static constexpr int K = 9; };
template <> struct LogSeries<double> { static constexpr int K = 18; };

template <typename R>
__device__ __forceinline__ R x_minus_log1p(R x) {
    if (abs_(x) < R(0.1)) {
        constexpr int K = LogSeries<R>::K;
        R p = R(1.0 / K);
#pragma unroll
        for (int k = K - 1; k >= 2; --k) p = R(1.0 / k) - x * p;
        return x * x * p;
    }
    return x - log1p_(x);
}

// One Jacobi rotation zeroing A[p][q] of the symmetric 3x3 A (Golub & Van Loan,
// "Matrix Computations", the symmetric Schur decomposition of Sec. 8.5), with
// the rotation accumulated into the columns of V when WithV.
template <typename R, int p, int q, bool WithV>
__device__ __forceinline__ void jacobi_rotate(R A[3][3], R V[3][3]) {
    const R apq = A[p][q];
    if (apq == R(0)) return;
    const R theta = (A[q][q] - A[p][p]) / (R(2) * apq);
    R t;
    if (abs_(theta) > R(1e15)) t = R(0.5) / theta;
    else t = (theta >= R(0) ? R(1) : R(-1)) / (abs_(theta) + sqrt_(theta * theta + R(1)));
    const R c = rsqrt_(t * t + R(1));
    const R s = t * c;
    constexpr int r = 3 - p - q;
    A[p][p] -= t * apq;
    A[q][q] += t * apq;
    A[p][q] = A[q][p] = R(0);
    const R arp = A[r][p], arq = A[r][q];
    A[r][p] = A[p][r] = c * arp - s * arq;
    A[r][q] = A[q][r] = s * arp + c * arq;
    if (WithV) {
#pragma unroll
        for (int i = 0; i < 3; ++i) {
            const R vp = V[i][p], vq = V[i][q];
            V[i][p] = c * vp - s * vq;
            V[i][q] = s * vp + c * vq;
        }
    }
}

// Cyclic Jacobi sweeps until the off-diagonal part is at round-off level.
template <typename R, bool WithV>
__device__ __forceinline__ void jacobi_sweeps(R A[3][3], R V[3][3]) {
    for (int sweep = 0; sweep < 8; ++sweep) {
        const R off = abs_(A[0][1]) + abs_(A[0][2]) + abs_(A[1][2]);
        const R dia = abs_(A[0][0]) + abs_(A[1][1]) + abs_(A[2][2]);
        if (!(off > R(0.25) * Eps<R>::v * dia)) break;
        jacobi_rotate<R, 0, 1, WithV>(A, V);
        jacobi_rotate<R, 0, 2, WithV>(A, V);
        jacobi_rotate<R, 1, 2, WithV>(A, V);
    }
}

// S = F^T F - I = G + G^T + G^T G for F = I + G.
template <typename R>
__device__ __forceinline__ void strain2(const R G[3][3], R A[3][3]) {
#pragma unroll
    for (int a = 0; a < 3; ++a)
#pragma unroll
        for (int b = 0; b < 3; ++b)
            A[a][b] = G[a][b] + G[b][a] + G[0][a] * G[0][b] + G[1][a] * G[1][b] + G[2][a] * G[2][b];
}

template <typename R>
__device__ __forceinline__ void swap_cols(R l[3], R V[3][3], int a, int b) {
    R t = l[a]; l[a] = l[b]; l[b] = t;
#pragma unroll
    for (int i = 0; i < 3; ++i) { R v = V[i][a]; V[i][a] = V[i][b]; V[i][b] = v; }
}

// Signed SVD of F = I + G in the invertible-element convention: F = U diag(s) V^T,
// U, V in SO(3), s1 >= s2 >= |s3|, s3 < 0 exactly when det F < 0.  Also returns
// l_i = s_i^2 - 1 at the precision of G.
//   1. Cyclic Jacobi on S = G + G^T + G^T G gives l and V (sorted, det V = +1).
//   2. U from a Gram-Schmidt QR of B = F V: u1 = b1/|b1|, u2 from b2, u3 = u1 x u2.
//   3. s_i = sqrt(1 + l_i) where l_i > -1/2 (relative precision near rest);
//      below that, s_i = u_i . b_i, the R diagonal of the QR, which keeps the
//      precision of nearly collapsed and inverted elements; l_i is then recomputed.
template <typename R>
__device__ __forceinline__ void signed_svd(const R G[3][3], R U[3][3], R s[3], R l[3], R V[3][3]) {
    R A[3][3];
    strain2(G, A);
#pragma unroll
    for (int a = 0; a < 3; ++a)
#pragma unroll
        for (int b = 0; b < 3; ++b) V[a][b] = a == b ? R(1) : R(0);
    jacobi_sweeps<R, true>(A, V);
    l[0] = A[0][0]; l[1] = A[1][1]; l[2] = A[2][2];
    if (l[0] < l[1]) swap_cols(l, V, 0, 1);
    if (l[0] < l[2]) swap_cols(l, V, 0, 2);
    if (l[1] < l[2]) swap_cols(l, V, 1, 2);
    const R detV = V[0][0] * (V[1][1] * V[2][2] - V[1][2] * V[2][1]) -
                   V[0][1] * (V[1][0] * V[2][2] - V[1][2] * V[2][0]) +
                   V[0][2] * (V[1][0] * V[2][1] - V[1][1] * V[2][0]);
    if (detV < R(0)) { V[0][2] = -V[0][2]; V[1][2] = -V[1][2]; V[2][2] = -V[2][2]; }
    // B = F V = V + G V
    R B[3][3];
#pragma unroll
    for (int a = 0; a < 3; ++a)
#pragma unroll
        for (int i = 0; i < 3; ++i) B[a][i] = V[a][i] + G[a][0] * V[0][i] + G[a][1] * V[1][i] + G[a][2] * V[2][i];
    // u1
    R n1 = sqrt_(B[0][0] * B[0][0] + B[1][0] * B[1][0] + B[2][0] * B[2][0]);
    R u1[3];
    if (n1 > R(1e-30)) {
        const R inv = R(1) / n1;
        u1[0] = B[0][0] * inv; u1[1] = B[1][0] * inv; u1[2] = B[2][0] * inv;
    } else {
        u1[0] = R(1); u1[1] = R(0); u1[2] = R(0);
        n1 = R(0);
    }
    // u2
    const R d12 = u1[0] * B[0][1] + u1[1] * B[1][1] + u1[2] * B[2][1];
    R w[3] = {B[0][1] - d12 * u1[0], B[1][1] - d12 * u1[1], B[2][1] - d12 * u1[2]};
    R n2 = sqrt_(w[0] * w[0] + w[1] * w[1] + w[2] * w[2]);
    R u2[3];
    if (n2 > R(64) * Eps<R>::v * (n1 > R(1) ? n1 : R(1))) {
        const R inv = R(1) / n2;
        u2[0] = w[0] * inv; u2[1] = w[1] * inv; u2[2] = w[2] * inv;
    } else {
        // any unit vector orthogonal to u1
        R e[3] = {R(0), R(0), R(0)};
        const int k = (abs_(u1[0]) <= abs_(u1[1]) && abs_(u1[0]) <= abs_(u1[2])) ? 0
                      : (abs_(u1[1]) <= abs_(u1[2]) ? 1 : 2);
        e[k] = R(1);
        R dd = u1[0] * e[0] + u1[1] * e[1] + u1[2] * e[2];
        R v2[3] = {e[0] - dd * u1[0], e[1] - dd * u1[1], e[2] - dd * u1[2]};
        const R inv = rsqrt_(v2[0] * v2[0] + v2[1] * v2[1] + v2[2] * v2[2]);
        u2[0] = v2[0] * inv; u2[1] = v2[1] * inv; u2[2] = v2[2] * inv;
        n2 = u2[0] * B[0][1] + u2[1] * B[1][1] + u2[2] * B[2][1];
    }
    const R u3[3] = {u1[1] * u2[2] - u1[2] * u2[1], u1[2] * u2[0] - u1[0] * u2[2],
                     u1[0] * u2[1] - u1[1] * u2[0]};
    const R n3 = u3[0] * B[0][2] + u3[1] * B[1][2] + u3[2] * B[2][2];
#pragma unroll
    for (int a = 0; a < 3; ++a) { U[a][0] = u1[a]; U[a][1] = u2[a]; U[a][2] = u3[a]; }
    const R half = R(-0.5);
    if (l[0] > half) s[0] = sqrt_(R(1) + l[0]);
    else { s[0] = n1; l[0] = n1 * n1 - R(1); }
    if (l[1] > half) s[1] = sqrt_(R(1) + l[1]);
    else { s[1] = n2; l[1] = n2 * n2 - R(1); }
    if (l[2] > half) s[2] = n3 >= R(0) ? sqrt_(R(1) + l[2]) : -sqrt_(R(1) + l[2]);
    else { s[2] = n3; l[2] = n3 * n3 - R(1); }
}

// s - 1 from (s, l = s^2 - 1) without cancellation near s = 1.
template <typename R>
__device__ __forceinline__ R stretch_minus_one(R s, R l) {
    return s > R(0.5) ? l / (s + R(1)) : s - R(1);
}

// Spline function f about its rest point, for the argument t = 1 + e (e
// given, formed without cancellation): df = f(t) - f(1) - f'(1) e and
// ddf = f'(t) - f'(1); cubic Hermite segments (knots stored as offsets
// kx = x - 1) with quadratic continuation outside the knots.  Inside segment i
// the cubic is expanded about u_r (its point nearest t = 1): with du = u - u_r,
//   f'(u) - f'(u_r) = du (2 p2 + 3 p3 (u + u_r)) / h,
//   f(u) - f(u_r) - f'(u_r) h du = du^2 (p2 + p3 (u + 2 u_r)),
// whose terms do not cancel near t = 1.
template <typename R>
__device__ __forceinline__ void spline_delta(const MatDev<R> &M, int f, R e, R &df, R &ddf) {
    const R lo = M.kx[f][0], hi = M.kx[f][7];
    const R ec = e < lo ? lo : (e > hi ? hi : e);
    int i = 0;
#pragma unroll
    for (int k = 1; k < 7; ++k) i = ec >= M.kx[f][k] ? k : i;
    const R ih = M.inv_h[f][i];
    const R u = (ec - M.kx[f][i]) * ih;
    const R *p = M.p[f][i];
    const R ur = M.ur[f][i];
    const R du = u - ur;
    const R dd1 = M.dD[f][i] + du * (R(2) * p[2] + R(3) * p[3] * (u + ur)) * ih;
    const R dv = M.dE[f][i] + M.dD[f][i] * du / ih + du * du * (p[2] + p[3] * (u + R(2) * ur));
    const R f2 = (R(2) * p[2] + R(6) * u * p[3]) * ih * ih;
    const R dt = e - ec;
    df = dv + dt * (dd1 + R(0.5) * f2 * dt);
    ddf = dd1 + f2 * dt;
}

// Energy density Psi and tau_i = dPsi/ds_i from (s, l) for the material.
template <typename R>
__device__ __forceinline__ R material_tau(const MatDev<R> &M, const R s[3], const R l[3], R tau[3]) {
    const R mu = M.mu, lam = M.lam;
    const R J = s[0] * s[1] * s[2];
    switch (M.kind) {
        case HQN_NEOHOOKEAN: {
            // a = mu/2 (x^2 - 1), c = -mu ln J + lam/2 ln^2 J (Taylor below J0)
            if (J >= M.J0) {
                const R lnJ = R(0.5) * (log1p_(l[0]) + log1p_(l[1]) + log1p_(l[2]));
                const R psi = R(0.5) * mu * (x_minus_log1p(l[0]) + x_minus_log1p(l[1]) + x_minus_log1p(l[2])) +
                              R(0.5) * lam * lnJ * lnJ;
#pragma unroll
                for (int i = 0; i < 3; ++i) tau[i] = (mu * l[i] + lam * lnJ) / s[i];
                return psi;
            }
            const R dJ = J - M.J0;
            const R dc = M.c1 + M.c2 * dJ;
            const R psi = R(0.5) * mu * (l[0] + l[1] + l[2]) + M.c0 + dJ * (M.c1 + R(0.5) * M.c2 * dJ);
            tau[0] = mu * s[0] + dc * s[1] * s[2];
            tau[1] = mu * s[1] + dc * s[0] * s[2];
            tau[2] = mu * s[2] + dc * s[0] * s[1];
            return psi;
        }
        case HQN_STVK: {
            // mu sum e_i^2 + lam/2 (sum e_i)^2, e_i = (s_i^2 - 1)/2
            const R e0 = R(0.5) * l[0], e1 = R(0.5) * l[1], e2 = R(0.5) * l[2];
            const R tr = e0 + e1 + e2;
            tau[0] = (R(2) * mu * e0 + lam * tr) * s[0];
            tau[1] = (R(2) * mu * e1 + lam * tr) * s[1];
            tau[2] = (R(2) * mu * e2 + lam * tr) * s[2];
            return mu * (e0 * e0 + e1 * e1 + e2 * e2) + R(0.5) * lam * tr * tr;
        }
        case HQN_COROTATED: {
            // a = mu (x-1)^2, c = lam/2 (J-1)^2
            const R d0 = stretch_minus_one(s[0], l[0]), d1 = stretch_minus_one(s[1], l[1]),
                    d2 = stretch_minus_one(s[2], l[2]);
            const R Jm1 = d0 + d1 + d2 + d0 * d1 + d0 * d2 + d1 * d2 + d0 * d1 * d2;
            tau[0] = R(2) * mu * d0 + lam * Jm1 * s[1] * s[2];
            tau[1] = R(2) * mu * d1 + lam * Jm1 * s[0] * s[2];
            tau[2] = R(2) * mu * d2 + lam * Jm1 * s[0] * s[1];
            return mu * (d0 * d0 + d1 * d1 + d2 * d2) + R(0.5) * lam * Jm1 * Jm1;
        }
        case HQN_POLY4: {
            // a = mu (x-1)^4
            R psi = R(0);
#pragma unroll
            for (int i = 0; i < 3; ++i) {
                const R d = stretch_minus_one(s[i], l[i]);
                const R d2 = d * d;
                psi += mu * d2 * d2;
                tau[i] = R(4) * mu * d2 * d;
            }
            return psi;
        }
        default: {  // HQN_SPLINE_VL
            // Psi = psi_rest + K0 sum d_i + (b'(1) + c'(1)) sum_{i<j} d_i d_j + c'(1) d1 d2 d3
            //       + sum da(s_i) + sum db(s_i s_j) + dc(J),  d_i = s_i - 1
            const R d0 = stretch_minus_one(s[0], l[0]), d1 = stretch_minus_one(s[1], l[1]),
                    d2 = stretch_minus_one(s[2], l[2]);
            R ea0, ga0, ea1, ga1, ea2, ga2;
            spline_delta(M, 0, d0, ea0, ga0);
            spline_delta(M, 0, d1, ea1, ga1);
            spline_delta(M, 0, d2, ea2, ga2);
            // b and c at products of stretches: their offsets from 1 without cancellation
            R eb01, gb01, eb02, gb02, eb12, gb12, ec, gc;
            spline_delta(M, 1, d0 + d1 + d0 * d1, eb01, gb01);
            spline_delta(M, 1, d0 + d2 + d0 * d2, eb02, gb02);
            spline_delta(M, 1, d1 + d2 + d1 * d2, eb12, gb12);
            spline_delta(M, 2, (d0 + d1 + d2) + (d0 * d1 + d0 * d2 + d1 * d2) + d0 * d1 * d2, ec, gc);
            tau[0] = M.K0 + M.B1C1 * (d1 + d2) + M.C1 * d1 * d2 + ga0 + gb01 * s[1] + gb02 * s[2] + gc * s[1] * s[2];
            tau[1] = M.K0 + M.B1C1 * (d0 + d2) + M.C1 * d0 * d2 + ga1 + gb01 * s[0] + gb12 * s[2] + gc * s[0] * s[2];
            tau[2] = M.K0 + M.B1C1 * (d0 + d1) + M.C1 * d0 * d1 + ga2 + gb02 * s[0] + gb12 * s[1] + gc * s[0] * s[1];
            return M.psi_rest + M.K0 * (d0 + d1 + d2) + M.B1C1 * (d0 * d1 + d0 * d2 + d1 * d2) + M.C1 * d0 * d1 * d2 +
                   (ea0 + ea1 + ea2) + (eb01 + eb02 + eb12) + ec;
        }
    }
}

// Anisotropic fibre term of Sec. 4.4, kappa/2 (|F d| - 1)^2 for F = I + G:
// with g = G d, |F d|^2 = 1 + 2 d.g + |g|^2, so |F d| - 1 =
// (2 d.g + |g|^2) / (|F d| + 1) without cancellation near rest.  Returns the
// energy density; w (if not null) gets F d and fac = kappa (|F d| - 1)/|F d|,
// so that dPsi/dF = fac (F d) d^T.
template <typename R>
__device__ __forceinline__ R fiber_psi(const MatDev<R> &M, const R G[3][3], R Fd[3], R *fac) {
    R g[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) g[a] = G[a][0] * M.fd[0] + G[a][1] * M.fd[1] + G[a][2] * M.fd[2];
    const R s2 = R(2) * (M.fd[0] * g[0] + M.fd[1] * g[1] + M.fd[2] * g[2]) + (g[0] * g[0] + g[1] * g[1] + g[2] * g[2]);
    const R nrm = sqrt_(R(1) + s2);
    const R e = s2 / (nrm + R(1));
#pragma unroll
    for (int a = 0; a < 3; ++a) Fd[a] = M.fd[a] + g[a];
    if (fac) *fac = M.kappa * e / nrm;
    return R(0.5) * M.kappa * e * e;
}

// Psi(F) alone, F = I + G, for the line-search trials (no singular vectors).
// Neo-Hookean and StVK use the invariants, written so that no first-order
// term is cancelled against another:
//   NH:   I1 - 3 - 2 ln J = |G|^2 - 2 (m2 + det G) + 2 (d - log1p d),
//         d = det F - 1 = tr G + m2 + det G, m2 = sum of principal 2x2 minors of G;
//   StVK: mu |E|^2 + lam/2 tr^2 E with E = S / 2.
// The other materials take the stretches from the eigenvalues of S (Jacobi
// without vectors); s3 carries the sign of det F.
template <typename R>
__device__ __forceinline__ R tet_psi_base(const MatDev<R> &M, const R G[3][3]) {
    if (M.kind == HQN_NEOHOOKEAN) {
        const R tr = G[0][0] + G[1][1] + G[2][2];
        R n2 = R(0);
#pragma unroll
        for (int a = 0; a < 3; ++a)
#pragma unroll
            for (int b = 0; b < 3; ++b) n2 += G[a][b] * G[a][b];
        const R m2 = (G[0][0] * G[1][1] - G[0][1] * G[1][0]) + (G[0][0] * G[2][2] - G[0][2] * G[2][0]) +
                     (G[1][1] * G[2][2] - G[1][2] * G[2][1]);
        const R dg = G[0][0] * (G[1][1] * G[2][2] - G[1][2] * G[2][1]) -
                     G[0][1] * (G[1][0] * G[2][2] - G[1][2] * G[2][0]) +
                     G[0][2] * (G[1][0] * G[2][1] - G[1][1] * G[2][0]);
        const R d = tr + m2 + dg;
        const R J = R(1) + d;
        if (J >= M.J0) {
            const R lnJ = log1p_(d);
            return R(0.5) * M.mu * (n2 - R(2) * (m2 + dg) + R(2) * x_minus_log1p(d)) + R(0.5) * M.lam * lnJ * lnJ;
        }
        const R dJ = J - M.J0;
        return R(0.5) * M.mu * (R(2) * tr + n2) + M.c0 + dJ * (M.c1 + R(0.5) * M.c2 * dJ);
    }
    R A[3][3];
    strain2(G, A);
    if (M.kind == HQN_STVK) {
        const R tr = R(0.5) * (A[0][0] + A[1][1] + A[2][2]);
        R n2 = R(0);
#pragma unroll
        for (int a = 0; a < 3; ++a)
#pragma unroll
            for (int b = 0; b < 3; ++b) n2 += A[a][b] * A[a][b];
        return R(0.25) * M.mu * n2 + R(0.5) * M.lam * tr * tr;
    }
    R Vd[3][3];
    jacobi_sweeps<R, false>(A, Vd);
    R l[3] = {A[0][0], A[1][1], A[2][2]};
    if (l[0] < l[1]) { R t = l[0]; l[0] = l[1]; l[1] = t; }
    if (l[0] < l[2]) { R t = l[0]; l[0] = l[2]; l[2] = t; }
    if (l[1] < l[2]) { R t = l[1]; l[1] = l[2]; l[2] = t; }
    const R dg = G[0][0] * (G[1][1] * G[2][2] - G[1][2] * G[2][1]) -
                 G[0][1] * (G[1][0] * G[2][2] - G[1][2] * G[2][0]) +
                 G[0][2] * (G[1][0] * G[2][1] - G[1][1] * G[2][0]);
    const R d = (G[0][0] + G[1][1] + G[2][2]) +
                (G[0][0] * G[1][1] - G[0][1] * G[1][0]) + (G[0][0] * G[2][2] - G[0][2] * G[2][0]) +
                (G[1][1] * G[2][2] - G[1][2] * G[2][1]) + dg;
    R s[3];
#pragma unroll
    for (int i = 0; i < 3; ++i) s[i] = sqrt_(R(1) + l[i] > R(0) ? R(1) + l[i] : R(0));
    if (d < R(-1)) s[2] = -s[2];
    R tau[3];
    return material_tau(M, s, l, tau);
}

// The energy density: the material's plus the fibre term, if any.
template <typename R>
__device__ __forceinline__ R tet_psi(const MatDev<R> &M, const R G[3][3]) {
    R psi = tet_psi_base(M, G);
    if (M.kappa > R(0)) {
        R Fd[3];
        psi += fiber_psi(M, G, Fd, (R *)nullptr);
    }
    return psi;
}

template <typename R> __device__ __forceinline__ R fma_(R a, R b, R c) { return fma(a, b, c); }

// Psi(I + Gk + alpha Gd) for many step lengths alpha of one line search.
// Neo-Hookean and StVK are polynomials in alpha once the tet's Gk and Gd are
// known, so their coefficients are formed once and each alpha costs a few
// fused multiply-adds plus, for Neo-Hookean, log1p and the series above:
//   NH:   with d = det F - 1 = tr G + m2(G) + det G (cubic in alpha),
//         I1 - 3 - 2 ln J = |G|^2 - 2 (m2 + det G) + 2 (d - log1p d),
//         so |G|^2 - 2 (m2 + det G) is a cubic P(alpha) and d a cubic D(alpha);
//         below J0 the quadratic continuation uses |G|^2 + 2 tr G (quadratic).
//   StVK: E = (G + G^T + G^T G) / 2 = E0 + alpha E1 + alpha^2 E2, so |E|^2 is a
//         quartic and tr E a quadratic.
// The other materials evaluate tet_psi at G = Gk + alpha Gd.
template <typename R>
struct PsiRay {
    R c[11];      // polynomial coefficients (material-specific)
    R Gk[3][3], Gd[3][3];
};

template <typename R>
__device__ __forceinline__ R det3g(const R G[3][3]) {
    return G[0][0] * (G[1][1] * G[2][2] - G[1][2] * G[2][1]) - G[0][1] * (G[1][0] * G[2][2] - G[1][2] * G[2][0]) +
           G[0][2] * (G[1][0] * G[2][1] - G[1][1] * G[2][0]);
}

// Cofactor matrix: C[a][b] = d det(G) / d G[a][b].
template <typename R>
__device__ __forceinline__ void cofactor3(const R G[3][3], R C[3][3]) {
    C[0][0] = G[1][1] * G[2][2] - G[1][2] * G[2][1];
    C[0][1] = G[1][2] * G[2][0] - G[1][0] * G[2][2];
    C[0][2] = G[1][0] * G[2][1] - G[1][1] * G[2][0];
    C[1][0] = G[0][2] * G[2][1] - G[0][1] * G[2][2];
    C[1][1] = G[0][0] * G[2][2] - G[0][2] * G[2][0];
    C[1][2] = G[0][1] * G[2][0] - G[0][0] * G[2][1];
    C[2][0] = G[0][1] * G[1][2] - G[0][2] * G[1][1];
    C[2][1] = G[0][2] * G[1][0] - G[0][0] * G[1][2];
    C[2][2] = G[0][0] * G[1][1] - G[0][1] * G[1][0];
}

template <typename R>
__device__ __forceinline__ void psi_ray_setup(const MatDev<R> &M, const R Gk[3][3], const R Gd[3][3], PsiRay<R> &r) {
    // G along the ray (the fibre term and the materials without a polynomial form)
#pragma unroll
    for (int a = 0; a < 3; ++a)
#pragma unroll
        for (int b = 0; b < 3; ++b) {
            r.Gk[a][b] = Gk[a][b];
            r.Gd[a][b] = Gd[a][b];
        }
    if (M.kind == HQN_NEOHOOKEAN) {
        // tr G, |G|^2, m2(G) (sum of principal 2x2 minors) and det G along the ray
        const R t0 = Gk[0][0] + Gk[1][1] + Gk[2][2], t1 = Gd[0][0] + Gd[1][1] + Gd[2][2];
        R n0 = R(0), n1 = R(0), n2 = R(0);
#pragma unroll
        for (int a = 0; a < 3; ++a)
#pragma unroll
            for (int b = 0; b < 3; ++b) {
                n0 += Gk[a][b] * Gk[a][b];
                n1 += Gk[a][b] * Gd[a][b];
                n2 += Gd[a][b] * Gd[a][b];
            }
        n1 *= R(2);
        // m2(A + alpha B) = m2(A) + alpha (tr A tr B - tr(AB)) + alpha^2 m2(B)
        R trAB = R(0);
#pragma unroll
        for (int a = 0; a < 3; ++a)
#pragma unroll
            for (int b = 0; b < 3; ++b) trAB += Gk[a][b] * Gd[b][a];
        const R m2k = (Gk[0][0] * Gk[1][1] - Gk[0][1] * Gk[1][0]) + (Gk[0][0] * Gk[2][2] - Gk[0][2] * Gk[2][0]) +
                      (Gk[1][1] * Gk[2][2] - Gk[1][2] * Gk[2][1]);
        const R m2d = (Gd[0][0] * Gd[1][1] - Gd[0][1] * Gd[1][0]) + (Gd[0][0] * Gd[2][2] - Gd[0][2] * Gd[2][0]) +
                      (Gd[1][1] * Gd[2][2] - Gd[1][2] * Gd[2][1]);
        const R m1 = t0 * t1 - trAB;
        // det(A + alpha B) = det A + alpha <cof A, B> + alpha^2 <A, cof B> + alpha^3 det B
        R Ck[3][3], Cd[3][3];
        cofactor3(Gk, Ck);
        cofactor3(Gd, Cd);
        R e1 = R(0), e2 = R(0);
#pragma unroll
        for (int a = 0; a < 3; ++a)
#pragma unroll
            for (int b = 0; b < 3; ++b) {
                e1 += Ck[a][b] * Gd[a][b];
                e2 += Gk[a][b] * Cd[a][b];
            }
        const R e0 = det3g(Gk), e3 = det3g(Gd);
        // D = tr + m2 + det; P = |G|^2 - 2 (m2 + det); Q = |G|^2 + 2 tr (below J0)
        r.c[0] = t0 + m2k + e0; r.c[1] = t1 + m1 + e1; r.c[2] = m2d + e2; r.c[3] = e3;
        r.c[4] = n0 - R(2) * (m2k + e0); r.c[5] = n1 - R(2) * (m1 + e1);
        r.c[6] = n2 - R(2) * (m2d + e2); r.c[7] = -R(2) * e3;
        r.c[8] = n0 + R(2) * t0; r.c[9] = n1 + R(2) * t1; r.c[10] = n2;
        return;
    }
    if (M.kind == HQN_STVK) {
        // E0 = (Gk + Gk^T + Gk^T Gk)/2, E1 = (Gd + Gd^T + Gk^T Gd + Gd^T Gk)/2, E2 = Gd^T Gd / 2
        R E0[3][3], E1[3][3], E2[3][3];
#pragma unroll
        for (int a = 0; a < 3; ++a)
#pragma unroll
            for (int b = 0; b < 3; ++b) {
                R kk = R(0), kd = R(0), dk = R(0), dd = R(0);
#pragma unroll
                for (int i = 0; i < 3; ++i) {
                    kk += Gk[i][a] * Gk[i][b];
                    kd += Gk[i][a] * Gd[i][b];
                    dk += Gd[i][a] * Gk[i][b];
                    dd += Gd[i][a] * Gd[i][b];
                }
                E0[a][b] = R(0.5) * (Gk[a][b] + Gk[b][a] + kk);
                E1[a][b] = R(0.5) * (Gd[a][b] + Gd[b][a] + kd + dk);
                E2[a][b] = R(0.5) * dd;
            }
        R p00 = R(0), p01 = R(0), p02 = R(0), p11 = R(0), p12 = R(0), p22 = R(0);
#pragma unroll
        for (int a = 0; a < 3; ++a)
#pragma unroll
            for (int b = 0; b < 3; ++b) {
                p00 += E0[a][b] * E0[a][b];
                p01 += E0[a][b] * E1[a][b];
                p02 += E0[a][b] * E2[a][b];
                p11 += E1[a][b] * E1[a][b];
                p12 += E1[a][b] * E2[a][b];
                p22 += E2[a][b] * E2[a][b];
            }
        // |E|^2 = p00 + 2 p01 a + (p11 + 2 p02) a^2 + 2 p12 a^3 + p22 a^4
        r.c[0] = p00; r.c[1] = R(2) * p01; r.c[2] = p11 + R(2) * p02; r.c[3] = R(2) * p12; r.c[4] = p22;
        r.c[5] = E0[0][0] + E0[1][1] + E0[2][2];
        r.c[6] = E1[0][0] + E1[1][1] + E1[2][2];
        r.c[7] = E2[0][0] + E2[1][1] + E2[2][2];
        return;
    }
}

// Neo-Hookean and StVK along the ray from the polynomial coefficients.
template <typename R>
__device__ __forceinline__ R psi_ray_poly(const MatDev<R> &M, const PsiRay<R> &r, R al) {
    if (M.kind == HQN_NEOHOOKEAN) {
        const R d = r.c[0] + al * (r.c[1] + al * (r.c[2] + al * r.c[3]));
        const R J = R(1) + d;
        if (J >= M.J0) {
            const R P = r.c[4] + al * (r.c[5] + al * (r.c[6] + al * r.c[7]));
            const R lnJ = log1p_(d);
            return R(0.5) * M.mu * (P + R(2) * x_minus_log1p(d)) + R(0.5) * M.lam * lnJ * lnJ;
        }
        const R Q = r.c[8] + al * (r.c[9] + al * r.c[10]);
        const R dJ = J - M.J0;
        return R(0.5) * M.mu * Q + M.c0 + dJ * (M.c1 + R(0.5) * M.c2 * dJ);
    }
    const R n2 = r.c[0] + al * (r.c[1] + al * (r.c[2] + al * (r.c[3] + al * r.c[4])));
    const R tr = r.c[5] + al * (r.c[6] + al * r.c[7]);
    return M.mu * n2 + R(0.5) * M.lam * tr * tr;
}

template <typename R>
__device__ __forceinline__ R psi_ray_fiber(const MatDev<R> &M, const PsiRay<R> &r, R al) {
    if (!(M.kappa > R(0))) return R(0);
    R G[3][3], Fd[3];
#pragma unroll
    for (int p = 0; p < 3; ++p)
#pragma unroll
        for (int q = 0; q < 3; ++q) G[p][q] = fma_(al, r.Gd[p][q], r.Gk[p][q]);
    return fiber_psi(M, G, Fd, (R *)nullptr);
}

template <typename R>
__device__ __forceinline__ R psi_ray_eval(const MatDev<R> &M, const PsiRay<R> &r, R al) {
    if (M.kind == HQN_NEOHOOKEAN || M.kind == HQN_STVK) return psi_ray_poly(M, r, al) + psi_ray_fiber(M, r, al);
    R G[3][3];
#pragma unroll
    for (int p = 0; p < 3; ++p)
#pragma unroll
        for (int q = 0; q < 3; ++q) G[p][q] = fma_(al, r.Gd[p][q], r.Gk[p][q]);
    return tet_psi(M, G);
}


// G = Du Dm^{-1}: du[j] = u_{j+1} - u_0 (rows), Di = Dm^{-1} row-major.
template <typename R>
__device__ __forceinline__ void def_grad(const R du[3][3], const R Di[9], R G[3][3]) {
#pragma unroll
    for (int a = 0; a < 3; ++a)
#pragma unroll
        for (int b = 0; b < 3; ++b)
            G[a][b] = du[0][a] * Di[0 * 3 + b] + du[1][a] * Di[1 * 3 + b] + du[2][a] * Di[2 * 3 + b];
}

// First Piola stress of the Neo-Hookean and StVK materials from the
// invariants of F = I + G (no singular vectors).  Both energies depend on the
// stretches only through I1 = |F|^2 and J = det F (NH: a = mu/2 (x^2 - 1),
// c(J) with its Taylor continuation below J0) or through E = (F^T F - I)/2
// (StVK), so P = dPsi/dF equals U diag(tau) V^T of the stretch form:
//   NH:   P = mu F + c'(J) cof F, written for J >= J0 as
//         P = (mu (J F - cof F) + lam ln J cof F) / J with
//         J F - cof F = (m2 + det G) I + J G + G^T - cof G and
//         cof F = (1 + tr G) I - G^T + cof G  (cof is quadratic: cof(I + G) =
//         I + (tr G) I - G^T + cof G), so no term of size mu cancels near rest;
//         m2 = tr cof G, J - 1 = tr G + m2 + det G;
//   StVK: P = F (mu A + lam/2 tr A I), A = F^T F - I = G + G^T + G^T G.
template <typename R>
__device__ __forceinline__ void invariant_stress(const MatDev<R> &M, const R G[3][3], R P[3][3]) {
    if (M.kind == HQN_NEOHOOKEAN) {
        R cg[3][3];
#pragma unroll
        for (int a = 0; a < 3; ++a)
#pragma unroll
            for (int b = 0; b < 3; ++b) {
                const int a1 = (a + 1) % 3, a2 = (a + 2) % 3, b1 = (b + 1) % 3, b2 = (b + 2) % 3;
                cg[a][b] = G[a1][b1] * G[a2][b2] - G[a1][b2] * G[a2][b1];
            }
        const R tr = G[0][0] + G[1][1] + G[2][2];
        const R m2 = cg[0][0] + cg[1][1] + cg[2][2];
        const R dg = G[0][0] * cg[0][0] + G[0][1] * cg[0][1] + G[0][2] * cg[0][2];
        const R d = tr + m2 + dg;
        const R J = R(1) + d;
        if (J >= M.J0) {
            const R lnJ = log1p_(d), inv = R(1) / J;
            const R base = m2 + dg;
#pragma unroll
            for (int a = 0; a < 3; ++a)
#pragma unroll
                for (int b = 0; b < 3; ++b) {
                    const R id = a == b ? R(1) : R(0);
                    const R jf_cof = id * base + J * G[a][b] + G[b][a] - cg[a][b];
                    const R cofF = id * (R(1) + tr) - G[b][a] + cg[a][b];
                    P[a][b] = inv * (M.mu * jf_cof + M.lam * lnJ * cofF);
                }
        } else {
            const R dc = M.c1 + M.c2 * (J - M.J0);
#pragma unroll
            for (int a = 0; a < 3; ++a)
#pragma unroll
                for (int b = 0; b < 3; ++b) {
                    const R id = a == b ? R(1) : R(0);
                    P[a][b] = M.mu * (id + G[a][b]) + dc * (id * (R(1) + tr) - G[b][a] + cg[a][b]);
                }
        }
        return;
    }
    // StVK
    R A[3][3];
    strain2(G, A);
    const R htr = R(0.5) * M.lam * (A[0][0] + A[1][1] + A[2][2]);
    R Sv[3][3];
#pragma unroll
    for (int a = 0; a < 3; ++a)
#pragma unroll
        for (int b = 0; b < 3; ++b) Sv[a][b] = M.mu * A[a][b] + (a == b ? htr : R(0));
#pragma unroll
    for (int a = 0; a < 3; ++a)
#pragma unroll
        for (int b = 0; b < 3; ++b) P[a][b] = Sv[a][b] + G[a][0] * Sv[0][b] + G[a][1] * Sv[1][b] + G[a][2] * Sv[2][b];
}

// P += d/dF of the fibre term: kappa (|F d| - 1) (F d / |F d|) d^T.
template <typename R>
__device__ __forceinline__ void add_fiber_stress(const MatDev<R> &M, const R G[3][3], R P[3][3]) {
    if (!(M.kappa > R(0))) return;
    R Fd[3], fac;
    fiber_psi(M, G, Fd, &fac);
#pragma unroll
    for (int a = 0; a < 3; ++a)
#pragma unroll
        for (int b = 0; b < 3; ++b) P[a][b] += fac * Fd[a] * M.fd[b];
}

// Gradients of V*Psi with respect to the four corner positions, F = I + G.
// First Piola P (invariant form for Neo-Hookean and StVK, otherwise
// U diag(tau) V^T from the signed SVD); corners 1..3 get the columns of
// V P Dm^{-T}, corner 0 minus their sum.
template <typename R>
__device__ __forceinline__ void tet_grad(const MatDev<R> &M, const R G[3][3], const R Di[9], R vol, R g[4][3]) {
    R P[3][3];
    if (M.kind == HQN_NEOHOOKEAN || M.kind == HQN_STVK) {
        invariant_stress(M, G, P);
        add_fiber_stress(M, G, P);
#pragma unroll
        for (int a = 0; a < 3; ++a)
#pragma unroll
            for (int b = 0; b < 3; ++b) P[a][b] *= vol;
    } else {
        R U[3][3], s[3], l[3], V[3][3];
        signed_svd(G, U, s, l, V);
        R tau[3];
        material_tau(M, s, l, tau);
#pragma unroll
        for (int a = 0; a < 3; ++a)
#pragma unroll
            for (int b = 0; b < 3; ++b)
                P[a][b] = U[a][0] * tau[0] * V[b][0] + U[a][1] * tau[1] * V[b][1] + U[a][2] * tau[2] * V[b][2];
        add_fiber_stress(M, G, P);
#pragma unroll
        for (int a = 0; a < 3; ++a)
#pragma unroll
            for (int b = 0; b < 3; ++b) P[a][b] *= vol;
    }
#pragma unroll
    for (int j = 0; j < 3; ++j)
#pragma unroll
        for (int a = 0; a < 3; ++a)
            g[j + 1][a] = P[a][0] * Di[j * 3 + 0] + P[a][1] * Di[j * 3 + 1] + P[a][2] * Di[j * 3 + 2];
#pragma unroll
    for (int a = 0; a < 3; ++a) g[0][a] = -(g[1][a] + g[2][a] + g[3][a]);
}

}  // namespace hqn
