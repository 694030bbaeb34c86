// Host-callable launchers of the step kernels (explicitly instantiated for
// float and double in kernels.cu and solve.cu).  All pointers are device
// pointers owned by the simulation handle.
#pragma once

#include "common.cuh"

namespace hqn {

constexpr int VBS = 256;  // threads per block of the vertex kernels

// Device view of one simulation's buffers.
template <typename R>
struct DevSim {
    StepConst<R> c;
    MatDev<R> mat;
    int tet_bs;                 // threads per block of the tet kernel (64, 128 or 256)
    // mesh
    const int4 *tets;           // T
    const R *dminv;             // 9 x T (SoA), Dm^{-1}[j][b] at (3j + b) * T + t
    const R *vol;               // T
    const R *mh2;               // n, m_v / h^2
    const int *vt_ptr;          // n + 1
    const int *vt_slot;         // corner slots c * T + t, ascending t per vertex
    // state and work vectors (n entries each, internal vertex order)
    V4<R> *u_cur, *u_prev, *y, *xk, *xt, *gk, *d, *q, *z;
    V4<R> *S, *Tt;              // (m + 1) x n history ring
    V4<R> *corner;              // 4 x T corner gradients
    double *part_in, *part_el, *part_g, *part_v, *part_ls;
    Ctl *ctl;
};

enum TetMode { TET_INIT = 0, TET_GRAD = 1, TET_EVAL = 2 };
enum GatherMode { G_INIT = 0, G_ITER = 1, G_EVAL = 2 };

template <typename R> void launch_predict(const DevSim<R> &s, cudaStream_t st);
// Inertia partials of the caller-given point x_t.
template <typename R> void launch_inertia(const DevSim<R> &s, cudaStream_t st);
template <typename R> void launch_tet(const DevSim<R> &s, int mode, cudaStream_t st);
// One multi-trial line-search pass (K = ls_batch step lengths).
template <typename R> void launch_ls(const DevSim<R> &s, CondHandles h, cudaStream_t st);
template <typename R> void launch_gather(const DevSim<R> &s, int mode, CondHandles h, cudaStream_t st);
// Alg. 2 first loop: p = -1 starts it (q = -grad), p = 0..m-1 applies pair p.
template <typename R> void launch_first_loop(const DevSim<R> &s, int p, cudaStream_t st);
// Alg. 2 second loop: j = -1 starts it, j = 0..m-1 applies the j-th oldest pair.
template <typename R> void launch_second_loop(const DevSim<R> &s, int j, cudaStream_t st);
// gd = tr(grad^T d); flags a non-descent direction (sets h.nd when set_nd).
template <typename R> void launch_direction_final(const DevSim<R> &s, CondHandles h, int set_nd, cudaStream_t st);
template <typename R> void launch_ls_begin(const DevSim<R> &s, CondHandles h, cudaStream_t st);
template <typename R> void launch_reset_history(const DevSim<R> &s, cudaStream_t st);
template <typename R> void launch_commit(const DevSim<R> &s, cudaStream_t st);
// rho of ring slot `slot` = tr(Tt[slot]^T S[slot]) (history given by the caller).
template <typename R> void launch_pair_rho(const DevSim<R> &s, int slot, cudaStream_t st);

// ---- triangular solves (solve.cu)
constexpr int SOLVE_MAX_SMEM = 220 * 1024;  // dynamic shared memory of one sweep block

template <typename R>
struct DevSolve {
    int nf, n_levels;
    const R *QF;                // per supernode: Q_s row-major, rows padded to ldc (16 B)
    const R *QB;                // per supernode: Q_s^T row-major, rows padded to ldr (16 B)
    const int4 *sn;             // (col, ncol, nrow, roff)
    const long long *sn_qf, *sn_qb;  // offsets of the two copies
    const int2 *sn_ld;          // (ldc, ldr)
    const int *sn_u;            // offset of the supernode's update entries
    const int *rows;            // row structures
    const int2 *fg2;            // per column: the (<= 2) child update entries to subtract
    const int2 *ug2;            // per update entry: the (<= 2) child update entries to add
    const int4 *fwd_items;      // (s, row0, row1, G)
    const int4 *bwd_items;      // (s, col0, col1, G)
    const int *fwd_lvl_ptr, *bwd_lvl_ptr;  // host: items of level l in [ptr[l], ptr[l+1])
    const int *fwd_lvl_ld, *bwd_lvl_ld;    // host: max ldc / ldr of the level (shared memory)
    V4<R> *u;                   // update vectors
};

// r = A0^{-1} q on the first nf entries (q, r: V4 arrays, may not alias).
template <typename R>
void launch_solve(const DevSolve<R> &s, const V4<R> *q, V4<R> *z, V4<R> *r, cudaStream_t st);
template <typename R> int solve_smem_limit_ok(int max_cols);
// Raises the forward sweep's dynamic shared-memory limit (once per device).
template <typename R> cudaError_t solve_prepare();

}  // namespace hqn
