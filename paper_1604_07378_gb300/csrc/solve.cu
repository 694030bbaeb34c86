// Device forward and backward sweeps of r = A0^{-1} q, A0 = M/h^2 + L
// (Eq. PDsolution; the constant initial Hessian of Alg. 2, prefactored once),
// on 3 right-hand sides (x, y, z share one n x n factor, Sec. 3).
//
// The factor L is supernodal over a nested-dissection tree.  Each supernode s
// (columns C, later coupled rows R) holds Q_s = [L_CC^{-1}; L_RC L_CC^{-1}], so
// both sweeps are independent dense row dot products:
//   forward (leaves first):  f = q_C - (child updates landing on C);
//                            z_C = L_CC^{-1} f;  u_R = L_RC z_C + (child updates on R)
//   backward (root first):   r_C = Q_s^T [z_C; -r_R]
// The forward sweep reads Q_s row-major (rows padded to 16 bytes), the
// backward sweep a transposed copy, so every output is a dot of a contiguous
// row with a vector staged in shared memory, read with 16-byte loads by a group
// of G lanes (G sized to the row length).  A tree level is one launch; within
// a level every supernode is independent, and updates pass up the tree through
// index tables (each entry receives from at most two children; no atomics).
#include "kernels.cuh"
#include "reduce.cuh"

namespace hqn {

namespace {

constexpr int SBS = 256;  // threads per block of the sweeps

template <typename R> struct Vec16;
template <> struct Vec16<float> {
    using T = float4;
    static constexpr int N = 4;
    __device__ static float at(const float4 &v, int e) { return e == 0 ? v.x : e == 1 ? v.y : e == 2 ? v.z : v.w; }
};
template <> struct Vec16<double> {
    using T = double2;
    static constexpr int N = 2;
    __device__ static double at(const double2 &v, int e) { return e == 0 ? v.x : v.y; }
};

template <typename R, int G>
__device__ __forceinline__ R group_sum(R v) {
#pragma unroll
    for (int o = G / 2; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// acc += sum_k row[k] . (fx, fy, fz)[k] over 16-byte vectors k = k0 + lane, step G.
template <typename R, int G>
__device__ __forceinline__ void row_dot(const R *__restrict__ row, const R *fx, const R *fy, const R *fz, int k0,
                                        int nv, int lane, R &ax, R &ay, R &az) {
    using VT = typename Vec16<R>::T;
    constexpr int VN = Vec16<R>::N;
    const VT *rv = reinterpret_cast<const VT *>(row);
    const VT *vx = reinterpret_cast<const VT *>(fx);
    const VT *vy = reinterpret_cast<const VT *>(fy);
    const VT *vz = reinterpret_cast<const VT *>(fz);
#pragma unroll 4
    for (int k = k0 + lane; k < nv; k += G) {
        const VT q = __ldg(rv + k);
        const VT a = vx[k], b = vy[k], c = vz[k];
#pragma unroll
        for (int e = 0; e < VN; ++e) {
            const R qe = Vec16<R>::at(q, e);
            ax += qe * Vec16<R>::at(a, e);
            ay += qe * Vec16<R>::at(b, e);
            az += qe * Vec16<R>::at(c, e);
        }
    }
}

// Forward item (s, row0, row1, G).
template <typename R, int G>
__device__ __forceinline__ void fwd_rows(const DevSolve<R> &S, int s, int r0, int r1, const R *f, int ldc,
                                         V4<R> *z) {
    const int4 sn = S.sn[s];
    const int col = sn.x, nc = sn.y;
    const R *Qs = S.QF + S.sn_qf[s];
    const int uoff = S.sn_u[s];
    constexpr int NG = SBS / G;
    const int lane = threadIdx.x % G, grp = threadIdx.x / G;
    constexpr int VN = Vec16<R>::N;
    for (int base = r0; base < r1; base += NG) {
        const int i = base + grp;
        const bool valid = i < r1;
        R ax = R(0), ay = R(0), az = R(0);
        if (valid) {
            const int len = i < nc ? i + 1 : nc;
            row_dot<R, G>(Qs + (size_t)i * ldc, f, f + ldc, f + 2 * ldc, 0, (len + VN - 1) / VN, lane, ax, ay, az);
            if (i >= nc) {
                const int2 c = S.ug2[uoff + i - nc];
                for (int k = lane; k < 2; k += G) {
                    const int e = k == 0 ? c.x : c.y;
                    if (e >= 0) {
                        const V4<R> v = S.u[e];
                        ax += v.x; ay += v.y; az += v.z;
                    }
                }
            }
        }
        ax = group_sum<R, G>(ax);
        ay = group_sum<R, G>(ay);
        az = group_sum<R, G>(az);
        if (valid && lane == 0) {
            V4<R> o;
            o.x = ax; o.y = ay; o.z = az; o.w = R(0);
            if (i < nc) z[col + i] = o;
            else S.u[uoff + i - nc] = o;
        }
    }
}

template <typename R>
__global__ void __launch_bounds__(SBS) k_fwd(DevSolve<R> S, int item0, const V4<R> *rhs, V4<R> *z) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    R *f = reinterpret_cast<R *>(smem_raw);
    const int4 it = S.fwd_items[item0 + blockIdx.x];
    const int s = it.x;
    const int4 sn = S.sn[s];
    const int col = sn.x, nc = sn.y;
    const int ldc = S.sn_ld[s].x;
    for (int j = threadIdx.x; j < ldc; j += SBS) {
        R vx = R(0), vy = R(0), vz = R(0);
        if (j < nc) {
            const V4<R> v = rhs[col + j];
            const int2 c = S.fg2[col + j];
            vx = v.x; vy = v.y; vz = v.z;
            if (c.x >= 0) { const V4<R> a = S.u[c.x]; vx -= a.x; vy -= a.y; vz -= a.z; }
            if (c.y >= 0) { const V4<R> a = S.u[c.y]; vx -= a.x; vy -= a.y; vz -= a.z; }
        }
        f[j] = vx; f[ldc + j] = vy; f[2 * ldc + j] = vz;
    }
    __syncthreads();
    const int r0 = it.y, r1 = it.z;
    switch (it.w) {
        case 1: fwd_rows<R, 1>(S, s, r0, r1, f, ldc, z); break;
        case 2: fwd_rows<R, 2>(S, s, r0, r1, f, ldc, z); break;
        case 4: fwd_rows<R, 4>(S, s, r0, r1, f, ldc, z); break;
        case 8: fwd_rows<R, 8>(S, s, r0, r1, f, ldc, z); break;
        case 16: fwd_rows<R, 16>(S, s, r0, r1, f, ldc, z); break;
        default: fwd_rows<R, 32>(S, s, r0, r1, f, ldc, z); break;
    }
}

// Backward item (s, col0, col1, G): r_j = (row j of Q_s^T) . [z_C; -r_R].
template <typename R, int G>
__device__ __forceinline__ void bwd_cols(const DevSolve<R> &S, int s, int c0, int c1, const R *w, int ldr,
                                         V4<R> *r) {
    const int col = S.sn[s].x;
    const R *Qb = S.QB + S.sn_qb[s];
    constexpr int NG = SBS / G;
    constexpr int VN = Vec16<R>::N;
    const int lane = threadIdx.x % G, grp = threadIdx.x / G;
    const int nv = ldr / VN;
    for (int base = c0; base < c1; base += NG) {
        const int j = base + grp;
        const bool valid = j < c1;
        R ax = R(0), ay = R(0), az = R(0);
        if (valid) row_dot<R, G>(Qb + (size_t)j * ldr, w, w + ldr, w + 2 * ldr, j / VN, nv, lane, ax, ay, az);
        ax = group_sum<R, G>(ax);
        ay = group_sum<R, G>(ay);
        az = group_sum<R, G>(az);
        if (valid && lane == 0) {
            V4<R> o;
            o.x = ax; o.y = ay; o.z = az; o.w = R(0);
            r[col + j] = o;
        }
    }
}

template <typename R>
__global__ void __launch_bounds__(SBS) k_bwd(DevSolve<R> S, int item0, const V4<R> *z, V4<R> *r) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    R *w = reinterpret_cast<R *>(smem_raw);
    const int4 it = S.bwd_items[item0 + blockIdx.x];
    const int s = it.x;
    const int4 sn = S.sn[s];
    const int col = sn.x, nc = sn.y, nr = sn.z, roff = sn.w;
    const int rows = nc + nr;
    const int ldr = S.sn_ld[s].y;
    constexpr int VN = Vec16<R>::N;
    const int c0 = it.y;
    const int i0 = (c0 / VN) * VN;  // entries of w below i0 meet only zeros of Q_s^T
    for (int i = i0 + threadIdx.x; i < ldr; i += SBS) {
        R vx = R(0), vy = R(0), vz = R(0);
        if (i < nc) {
            const V4<R> v = z[col + i];
            vx = v.x; vy = v.y; vz = v.z;
        } else if (i < rows) {
            const V4<R> v = r[S.rows[roff + i - nc]];
            vx = -v.x; vy = -v.y; vz = -v.z;
        }
        w[i] = vx; w[ldr + i] = vy; w[2 * ldr + i] = vz;
    }
    __syncthreads();
    switch (it.w) {
        case 1: bwd_cols<R, 1>(S, s, c0, it.z, w, ldr, r); break;
        case 2: bwd_cols<R, 2>(S, s, c0, it.z, w, ldr, r); break;
        case 4: bwd_cols<R, 4>(S, s, c0, it.z, w, ldr, r); break;
        case 8: bwd_cols<R, 8>(S, s, c0, it.z, w, ldr, r); break;
        case 16: bwd_cols<R, 16>(S, s, c0, it.z, w, ldr, r); break;
        default: bwd_cols<R, 32>(S, s, c0, it.z, w, ldr, r); break;
    }
}

}  // namespace

template <typename R> int solve_smem_limit_ok(int max_ld) {
    return (size_t)3 * max_ld * sizeof(R) <= (size_t)SOLVE_MAX_SMEM;
}

template <typename R> cudaError_t solve_prepare() {
    cudaError_t e = cudaFuncSetAttribute(k_fwd<R>, cudaFuncAttributeMaxDynamicSharedMemorySize, SOLVE_MAX_SMEM);
    if (e != cudaSuccess) return e;
    return cudaFuncSetAttribute(k_bwd<R>, cudaFuncAttributeMaxDynamicSharedMemorySize, SOLVE_MAX_SMEM);
}

template <typename R>
void launch_solve(const DevSolve<R> &s, const V4<R> *q, V4<R> *z, V4<R> *r, cudaStream_t st) {
    for (int l = 0; l < s.n_levels; ++l) {
        const int a = s.fwd_lvl_ptr[l], b = s.fwd_lvl_ptr[l + 1];
        if (b > a) k_fwd<R><<<b - a, SBS, (size_t)3 * s.fwd_lvl_ld[l] * sizeof(R), st>>>(s, a, q, z);
    }
    for (int l = s.n_levels - 1; l >= 0; --l) {
        const int a = s.bwd_lvl_ptr[l], b = s.bwd_lvl_ptr[l + 1];
        if (b > a) k_bwd<R><<<b - a, SBS, (size_t)3 * s.bwd_lvl_ld[l] * sizeof(R), st>>>(s, a, z, r);
    }
}

template void launch_solve<float>(const DevSolve<float> &, const V4<float> *, V4<float> *, V4<float> *, cudaStream_t);
template void launch_solve<double>(const DevSolve<double> &, const V4<double> *, V4<double> *, V4<double> *, cudaStream_t);
template int solve_smem_limit_ok<float>(int);
template int solve_smem_limit_ok<double>(int);
template cudaError_t solve_prepare<float>();
template cudaError_t solve_prepare<double>();

}  // namespace hqn
