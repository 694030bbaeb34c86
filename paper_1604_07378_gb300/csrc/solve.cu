// Device forward and backward sweeps of r = A0^{-1} q, A0 = M/h^2 + L
// (Eq. PDsolution; the constant initial Hessian of Alg. 2, prefactored once),
// on 3 right-hand sides (x, y, z share one n x n factor, Sec. 3).
//
// The factor L is supernodal over a nested-dissection tree.  Each supernode s
// (columns C, later coupled rows R) stores Q_s = [L_CC^{-1}; L_RC L_CC^{-1}]
// densely, so both sweeps are dense matrix-vector products per supernode:
//   forward (leaves first):  f = q_C - (child updates landing on C);
//                            z_C = L_CC^{-1} f;  u_R = L_RC z_C + (child updates on R)
//   backward (root first):   r_C = Q_s^T [z_C; -r_R]
// A level of the tree is one launch; within a level every supernode is
// independent, and updates are passed up the tree by index lists (no atomics).
#include "kernels.cuh"
#include "reduce.cuh"

namespace hqn {

namespace {

constexpr int SBS = 256;          // threads per block of the sweeps
constexpr int BWD_CHUNK = 1024;   // rows of [z_C; -r_R] staged per pass

// Forward item (s, row0, row1): rows [row0, row1) of Q_s times f.
template <typename R>
__global__ void __launch_bounds__(SBS) k_fwd(DevSolve<R> S, int item0, const V4<R> *rhs, V4<R> *z) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    R *f = reinterpret_cast<R *>(smem_raw);
    const int4 it = S.fwd_items[item0 + blockIdx.x];
    const int4 sn = S.sn[it.x];
    const int col = sn.x, nc = sn.y;
    const R *Qs = S.Q + S.sn_q[it.x];
    const int uoff = S.sn_u[it.x];
    for (int j = threadIdx.x; j < nc; j += SBS) {
        V4<R> v = rhs[col + j];
        for (int e = S.fg_ptr[col + j]; e < S.fg_ptr[col + j + 1]; ++e) {
            const V4<R> c = S.u[S.fg_idx[e]];
            v.x -= c.x; v.y -= c.y; v.z -= c.z;
        }
        f[j] = v.x; f[nc + j] = v.y; f[2 * nc + j] = v.z;
    }
    __syncthreads();
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int i = it.y + warp; i < it.z; i += SBS / 32) {
        const int jn = i < nc ? i + 1 : nc;
        const R *qr = Qs + (size_t)i * nc;
        R ax = R(0), ay = R(0), az = R(0);
        for (int j = lane; j < jn; j += 32) {
            const R qv = qr[j];
            ax += qv * f[j]; ay += qv * f[nc + j]; az += qv * f[2 * nc + j];
        }
        ax = warp_sum_r(ax); ay = warp_sum_r(ay); az = warp_sum_r(az);
        if (lane == 0) {
            V4<R> o;
            o.w = R(0);
            if (i < nc) {
                o.x = ax; o.y = ay; o.z = az;
                z[col + i] = o;
            } else {
                const int ui = uoff + i - nc;
                for (int e = S.ug_ptr[ui]; e < S.ug_ptr[ui + 1]; ++e) {
                    const V4<R> c = S.u[S.ug_idx[e]];
                    ax += c.x; ay += c.y; az += c.z;
                }
                o.x = ax; o.y = ay; o.z = az;
                S.u[ui] = o;
            }
        }
    }
}

// Backward item (s, c0): columns [c0, c0 + 32) of r_C = Q_s^T [z_C; -r_R].
// Lane = column, warps split the rows, partial sums meet in shared memory.
template <typename R>
__global__ void __launch_bounds__(SBS) k_bwd(DevSolve<R> S, int item0, const V4<R> *z, V4<R> *r) {
    __shared__ R w[3][BWD_CHUNK];
    __shared__ R red[3][SBS / 32][32];
    const int4 it = S.bwd_items[item0 + blockIdx.x];
    const int4 sn = S.sn[it.x];
    const int col = sn.x, nc = sn.y, nr = sn.z, roff = sn.w;
    const int rows = nc + nr;
    const R *Qs = S.Q + S.sn_q[it.x];
    const int c0 = it.y;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int j = c0 + lane;
    const bool active = j < nc;
    R ax = R(0), ay = R(0), az = R(0);
    for (int base = c0; base < rows; base += BWD_CHUNK) {
        const int cnt = min(BWD_CHUNK, rows - base);
        __syncthreads();
        for (int k = threadIdx.x; k < cnt; k += SBS) {
            const int i = base + k;
            V4<R> v;
            if (i < nc) {
                v = z[col + i];
            } else {
                v = r[S.rows[roff + i - nc]];
                v.x = -v.x; v.y = -v.y; v.z = -v.z;
            }
            w[0][k] = v.x; w[1][k] = v.y; w[2][k] = v.z;
        }
        __syncthreads();
        if (active)
            for (int k = warp; k < cnt; k += SBS / 32) {
                const R qv = Qs[(size_t)(base + k) * nc + j];
                ax += qv * w[0][k]; ay += qv * w[1][k]; az += qv * w[2][k];
            }
    }
    red[0][warp][lane] = ax; red[1][warp][lane] = ay; red[2][warp][lane] = az;
    __syncthreads();
    if (warp == 0 && active) {
        R sx = R(0), sy = R(0), sz = R(0);
#pragma unroll
        for (int k = 0; k < SBS / 32; ++k) { sx += red[0][k][lane]; sy += red[1][k][lane]; sz += red[2][k][lane]; }
        V4<R> o;
        o.x = sx; o.y = sy; o.z = sz; o.w = R(0);
        r[col + j] = o;
    }
}

}  // namespace

template <typename R> int solve_smem_limit_ok(int max_cols) {
    return (size_t)3 * max_cols * sizeof(R) <= 200 * 1024;
}

template <typename R> cudaError_t solve_prepare() {
    return cudaFuncSetAttribute(k_fwd<R>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
}

template <typename R>
void launch_solve(const DevSolve<R> &s, const V4<R> *q, V4<R> *z, V4<R> *r, cudaStream_t st) {
    for (int l = 0; l < s.n_levels; ++l) {
        const int a = s.fwd_lvl_ptr[l], b = s.fwd_lvl_ptr[l + 1];
        if (b > a) {
            const size_t smem = (size_t)3 * s.fwd_lvl_cols[l] * sizeof(R);
            k_fwd<R><<<b - a, SBS, smem, st>>>(s, a, q, z);
        }
    }
    for (int l = s.n_levels - 1; l >= 0; --l) {
        const int a = s.bwd_lvl_ptr[l], b = s.bwd_lvl_ptr[l + 1];
        if (b > a) k_bwd<R><<<b - a, SBS, 0, st>>>(s, a, z, r);
    }
}

template void launch_solve<float>(const DevSolve<float> &, const V4<float> *, V4<float> *, V4<float> *, cudaStream_t);
template void launch_solve<double>(const DevSolve<double> &, const V4<double> *, V4<double> *, V4<double> *, cudaStream_t);
template int solve_smem_limit_ok<float>(int);
template cudaError_t solve_prepare<float>();
template cudaError_t solve_prepare<double>();
template int solve_smem_limit_ok<double>(int);

}  // namespace hqn
