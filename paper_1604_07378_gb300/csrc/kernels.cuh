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

enum TetMode { TET_INIT = 0, TET_GRAD = 1, TET_EVAL = 2, TET_TRIAL1 = 3 };
enum GatherMode { G_INIT = 0, G_ITER = 1, G_EVAL = 2 };

template <typename R> void launch_predict(const DevSim<R> &s, cudaStream_t st);
// Inertia partials of the caller-given point x_t.
template <typename R> void launch_inertia(const DevSim<R> &s, cudaStream_t st);
// TET_TRIAL1 is the first line-search trial (alpha = 1) fused with the
// gradient: it runs the Armijo test and, on acceptance, leaves the corner
// gradients of the new point in place (TET_GRAD then returns at once).
template <typename R> void launch_tet(const DevSim<R> &s, int mode, CondHandles h, cudaStream_t st);
// One multi-trial line-search pass (K = ls_batch step lengths).
template <typename R> void launch_ls(const DevSim<R> &s, CondHandles h, cudaStream_t st);
template <typename R> void launch_gather(const DevSim<R> &s, int mode, CondHandles h, cudaStream_t st);
// Alg. 2 in dot-product form (the Gram matrix of the history and the
// products with grad are formed by the gather that pushes a pair):
// q = -grad - sum zeta_p t_p; after the solve, t_a^T r0 and the second loop on
// scalars; then d = r0 + sum c_p s_p with gd and the inertia coefficients
// (sets h.nd on a non-descent direction when set_nd).
template <typename R> void launch_q(const DevSim<R> &s, cudaStream_t st);
template <typename R> void launch_r0_dots(const DevSim<R> &s, cudaStream_t st);
template <typename R> void launch_direction_final(const DevSim<R> &s, CondHandles h, int set_nd, cudaStream_t st);
template <typename R> void launch_reset_history(const DevSim<R> &s, cudaStream_t st);
template <typename R> void launch_commit(const DevSim<R> &s, cudaStream_t st);
// Caller-given history: Gram row a, rho_a and s_a^T grad (run for a = 0..count-1).
template <typename R> void launch_hist_row(const DevSim<R> &s, int a, cudaStream_t st);

// ---- triangular solves (solve.cu)
constexpr int SOLVE_MAX_SMEM = 200 * 1024;  // dynamic shared memory of one sweep block

template <typename R>
struct DevSolve {
    int nf, n_levels;
    int pdl;                    // host: launch the sweeps with programmatic dependent launch
    const R *QF;                // per supernode: packed Q_s, row-major (layout.hpp)
    const R *QB;                // per supernode: packed Q_s^T, row-major (layout.hpp)
    const int *rows;            // row structures R of the supernodes
    const int2 *fg2;            // per column: the (<= 2) child update entries to subtract
    const int2 *ug2;            // per update entry: the (<= 2) child update entries to add
    // Work items, 3 int4 each:
    //   forward  {q0 lo, q0 hi, bytes, G} {col, nc, ldc, uoff} {r0, r1, ldf, off0}
    //   backward {q0 lo, q0 hi, bytes, G} {col, nc, nrow, roff} {c0, c1, ldr, off0}
    // q0 = entry offset of the item's first row in QF / QB, bytes = size of its
    // rows, off0 = offset of that row inside its supernode's block.
    const int4 *fwd_items, *bwd_items;
    const int *fwd_lvl_ptr, *bwd_lvl_ptr;  // host: items of level l in [ptr[l], ptr[l+1])
    const int *fwd_lvl_ld, *bwd_lvl_ld;    // host: max ldc / ldr of the level (shared memory)
    const int *fwd_lvl_q, *bwd_lvl_q;      // host: max factor entries of one item of the level
    V4<R> *u;                   // update vectors
    unsigned int *err;          // set nonzero if a bulk copy did not arrive in time
};

// r = A0^{-1} q on the first nf entries (q, r: V4 arrays, may not alias).
template <typename R>
void launch_solve(const DevSolve<R> &s, const V4<R> *q, V4<R> *z, V4<R> *r, cudaStream_t st);
template <typename R> int solve_smem_limit_ok(int max_cols);
// Raises the forward sweep's dynamic shared-memory limit (once per device).
template <typename R> cudaError_t solve_prepare();

}  // namespace hqn
