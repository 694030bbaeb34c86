// Host-callable launchers of the step kernels (explicitly instantiated for
// float and double in kernels.cu and solve.cu).  All pointers are device
// pointers owned by the simulation handle.
#pragma once

#include "common.cuh"

namespace hqn {

constexpr int VBS = 256;  // threads per block of the vertex kernels
constexpr int TBS = 128;  // threads per block of the tet kernels

// The scalars of Alg. 2's two loops for a window of m > kShortHist pairs
// (L = m + 1 ring slots), one array of doubles(m) per simulation: the Gram
// matrix s_a^T t_b by ring slots (row a), then rho, s_a^T grad and t_a^T r0
// by ring slot, and the coefficients zeta and c = zeta - eta by age.
struct LongHist {
    int L;
    double *gram, *rho, *sg, *tr0, *zeta, *coef;
    static __host__ __device__ size_t doubles(int m) { return (size_t)(m + 1) * (m + 1) + 5 * (size_t)(m + 1); }
    __host__ __device__ LongHist(double *base, int m) : L(m + 1) {
        gram = base;
        rho = gram + (size_t)L * L;
        sg = rho + L;
        tr0 = sg + L;
        zeta = tr0 + L;
        coef = zeta + L;
    }
};
// Slot products of a long window, per block, over chunks of LH_CHUNK slots
// (3 values per slot): LD_PUSH after a pair (s_w, t_w) is pushed:
// s_a^T t_w, s_w^T t_a, s_a^T grad; LD_R0 after the solve: t_a^T r0;
// LD_ROW for a caller-given pair a0: s_a0^T t_b and s_b^T grad.
constexpr int LH_CHUNK = 16;
enum { LD_PUSH = 0, LD_R0 = 1, LD_ROW = 2 };

// One simulation of a batch, as the kernels see it (device-resident).  Every
// block of a vertex or tet kernel belongs to exactly one simulation.
template <typename R>
struct SimDesc {
    StepConst<R> c;             // n, nf, T, history m, iterations, ... of this simulation
    MatDev<R> mat;              // material 0
    int n_mats;                 // materials of the mesh (> 1: by tet, DevSim::tmat)
    const MatDev<R> *mats;      // n_mats materials (device) when n_mats > 1
    const R *kmat;              // their stiffness k (the matrix-free A0 of the PCG solve)
    int v0, t0;                 // its first vertex / tet in the batch arrays
    int vb0, nvb;               // its vertex-kernel blocks [vb0, vb0 + nvb), nvb = ceil(n / VBS)
    int tb0, ntb;               // its tet-kernel blocks [tb0, tb0 + ntb), ntb = ceil(T / TBS)
    long long ring0;            // its history ring: S / Tt entries [ring0, ring0 + (m + 1) n)
    Ctl *ctl;                   // its control block
    double *lh;                 // m > kShortHist: the two loops' scalars, LongHist layout; else null
};

// Device view of a batch of simulations (a single simulation is a batch of
// one).  Vertex and tet arrays are the simulations' arrays back to back.
template <typename R>
struct DevSim {
    int nsims, m, ls_batch;     // history window and line-search batch (shared)
    int nvb, ntb;               // blocks of the vertex / tet kernels over the batch
    int Tn;                     // tets of the batch (stride of the SoA arrays)
    const SimDesc<R> *desc;     // nsims
    SimDesc<R> desc0;           // simulation 0, by value (read from kernel parameters when nsims == 1)
    const int *vblk_sim;        // nvb: the simulation of each vertex-kernel block
    const int *tblk_sim;        // ntb: the simulation of each tet-kernel block
    // mesh
    const int4 *tets;           // Tn, batch vertex ids
    const R *dminv;             // 9 x Tn (SoA), Dm^{-1}[j][b] at (3j + b) * Tn + t
    const R *vol;               // Tn
    const uint8_t *tmat;        // Tn material indices (null when every simulation has one material)
    const R *mh2;               // batch vertices: m_v / h^2
    const V4<R> *rest;          // batch vertices: rest positions X (collision terms)
    const int *vt_ptr;          // batch vertices + 1
    const int *corner_pos;      // position of corner c of tet t (index c * Tn + t) in `corner`,
                                // which holds every vertex's incident corners together, ascending t
    // state and work vectors (batch vertices, internal order within each simulation)
    V4<R> *u_cur, *u_prev, *y, *xk, *xt, *gk, *d, *q, *z;
    V4<R> *S, *Tt;              // history rings
    V4<R> *corner;              // 4 x Tn corner gradients in vertex order (vt_ptr ranges)
    // Jacobi-PCG in lieu of A0^{-1} (iterative solver): residual, preconditioned
    // residual, search direction, A0 p and the inverse diagonal of A0 (free vertices)
    V4<R> *pcg_r, *pcg_z, *pcg_p, *pcg_ap;
    V4<R> *xprev;               // x_{k-1} (the Chebyshev direction of Alg. 3)
    const R *pcg_dinv;
    // per-block partial sums: part_x[k * (blocks of the kernel) + block]
    double *part_in, *part_el, *part_g, *part_v, *part_ls;
    double *part_l;             // m > kShortHist: per-block partials of the slot products, 48 per chunk of 16 slots
    unsigned int *batch_ticket; // arrival counters of the simulations' last blocks (graph conditions)
};

enum TetMode { TET_INIT = 0, TET_GRAD = 1, TET_EVAL = 2, TET_TRIAL1 = 3 };
enum GatherMode { G_INIT = 0, G_ITER = 1, G_EVAL = 2 };
// Slots of batch_ticket (one per graph condition).
enum { BT_IT = 0, BT_LS = 1, BT_ND = 2 };

// Each simulation's decisions (Armijo, history, iteration count) are taken by
// that simulation's last block; the last simulation to decide sets the graph's
// conditional handles from all of them (h = 0: not inside a graph).
template <typename R> void launch_predict(const DevSim<R> &s, cudaStream_t st);
// Inertia partials of the caller-given point x_t.
template <typename R> void launch_inertia(const DevSim<R> &s, cudaStream_t st);
// TET_TRIAL1 is the first line-search trial (alpha = 1) fused with the
// gradient: it runs the Armijo test and, on acceptance, leaves the corner
// gradients of the new point in place (TET_GRAD then skips that simulation).
template <typename R> void launch_tet(const DevSim<R> &s, int mode, CondHandles h, cudaStream_t st);
// One multi-trial line-search pass (K = ls_batch step lengths).
template <typename R> void launch_ls(const DevSim<R> &s, CondHandles h, cudaStream_t st);
template <typename R> void launch_gather(const DevSim<R> &s, int mode, CondHandles h, cudaStream_t st);
// Alg. 2 in dot-product form (the Gram matrix of the history and the
// products with grad are formed by the gather that pushes a pair):
// q = -grad - sum zeta_p t_p; after the solve, t_a^T r0 and the second loop on
// scalars; then d = r0 + sum c_p s_p with gd and the inertia coefficients
// (sets h.nd if any simulation's direction is not a descent direction).
template <typename R> void launch_q(const DevSim<R> &s, cudaStream_t st);
template <typename R> void launch_r0_dots(const DevSim<R> &s, cudaStream_t st);
template <typename R> void launch_direction_final(const DevSim<R> &s, CondHandles h, int set_nd, cudaStream_t st);
// Drops the history of the simulations flagged non-descent.
template <typename R> void launch_reset_history(const DevSim<R> &s, cudaStream_t st);
// out = approximation of A0^{-1} q by `iters` Jacobi-PCG iterations from zero
// (matrix-free A0 = M/h^2 + sum_t V_t k G_t^T G_t; 1 + 3 iters launches).
template <typename R> void launch_pcg(const DevSim<R> &s, const V4<R> *q, V4<R> *out, int iters, cudaStream_t st);
template <typename R> void launch_commit(const DevSim<R> &s, cudaStream_t st);
// out[perm[i]] = X + u_cur of the n vertices from batch vertex v0 (caller order).
template <typename R> void launch_positions(const DevSim<R> &s, const int *perm, int v0, int n, V4<R> *out,
                                            cudaStream_t st);
// Caller-order float64 vectors (device, n x 3) <-> internal V4 vectors of the
// n vertices from batch vertex v0: displacements from the float64 rest
// positions X (internal order), and back with clamped rows (>= nf) zero.
template <typename R> void launch_from_caller(const double *X, const double *src, const int *perm, int v0, int n,
                                              V4<R> *dst, cudaStream_t st);
template <typename R> void launch_to_caller(const V4<R> *src, const int *perm, int v0, int n, int nf, double *dst,
                                            cudaStream_t st);
// Caller-given history of simulation 0: Gram row a, rho_a and s_a^T grad
// (run for a = 0..count-1).
template <typename R> void launch_hist_row(const DevSim<R> &s, int a, cudaStream_t st, int nblocks);
// Long windows (m > kShortHist): the slot products of `mode` (LD_*; a0 is
// the caller's pair of LD_ROW) over the vertex blocks of the batch (or of
// simulation 0's nblocks blocks for LD_ROW), then, one block per simulation,
// their sums in block order, the Gram and scalar updates and the loop's
// recursion on scalars (zeta after LD_PUSH / the last LD_ROW, c after LD_R0).
template <typename R> void launch_long_hist(const DevSim<R> &s, int mode, int a0, cudaStream_t st, int nblocks);
// Raises k_lrec's dynamic shared-memory limit for windows of m pairs.
template <typename R> cudaError_t long_hist_prepare(int m);

// ---- triangular solves (solve.cu)
constexpr int SOLVE_MAX_SMEM = 200 * 1024;  // dynamic shared memory of one sweep block

template <typename R>
struct DevSolve {
    int nf, n_levels, n_sn;
    int pdl;                    // host: launch the level sweeps with programmatic dependent launch
    int threads;                // host: threads per sweep block (128, 256 or 512)
    int leaf_threads;           // host: threads per block of the leaf level
    int prefetch;               // host: launches ahead whose factor rows a level prefetches into L2 (0: none)
    int fault_test;             // host: 1 = the first level's blocks issue no copy (tests of the bounded wait)
    long long wait_polls;       // bound on a block's wait for its bulk copy, in polls
    int n_fwd_items, n_bwd_items;
    const R *QF;                // per supernode: packed Q_s, row-major (layout.hpp)
    const R *QB;                // per supernode: packed Q_s^T, row-major (layout.hpp)
    const int *rows;            // row structures R of the supernodes
    const int4 *fg4;            // per column: the (<= 4) child update entries to subtract
    const int4 *ug4;            // per update entry: the (<= 4) child update entries to add
    // Work items, 5 int4 each:
    //   forward  {q0 lo, q0 hi, bytes, G} {col, nc, ldc, uoff} {r0, r1, ldf, off0}
    //            {child0, child1, child2, child3} {s, 0, 0, 0}
    //   backward {q0 lo, q0 hi, bytes, G} {col, nc, nrow, roff} {c0, c1, ldr, off0} {parent, s, 0, 0}
    //            {e0, e1, column block, nch << 16 | chunk}  (e0 < 0: whole rows; chunk items
    //            have q0 = their supernode's block, bytes = the sum of their rows' pieces)
    // q0 = entry offset of the item's first row in QF / QB, bytes = size of its
    // rows, off0 = offset of that row inside its supernode's block; -1 = no
    // such supernode.  Forward items are in ascending, backward items in
    // descending tree-level order.
    const int4 *fwd_items, *bwd_items;
    const int *fwd_lvl_ptr;                // host: forward items of level l in [ptr[l], ptr[l+1])
    const int *bwd_lvl_start, *bwd_lvl_cnt;  // host: backward items of level l: [start[l], start[l] + cnt[l])
    const int *fwd_lvl_ld, *bwd_lvl_ld;    // host: max ldc / ldr of the level (shared memory)
    const int *fwd_lvl_q, *bwd_lvl_q;      // host: max factor entries of one item of the level
    // L2 prefetch spans {address lo, address hi, bytes, 0}: launch k of a
    // solve (forward level k for k < L, then backward level 2L - 1 - k) asks
    // L2 to fetch spans [pf_ptr[k], pf_ptr[k + 1]) -- factor rows of a later
    // launch and shares of the dense top block's matrix.
    int pf_any;                            // host: some launch has spans
    const int4 *pf_spans;
    const int *pf_ptr;                     // host: 2 L + 1 entries
    // Dense top block (solve_dense_top; solve.cu): its tiles (3 int4 each),
    // per simulation the lower block triangle of S^{-1} as TS x TS tiles,
    // the free columns of T, and the update entries below T that reach each
    // column (CSR, n_top + 1 offsets per simulation); the partial products
    // of every band (dense_nct_max slots of TS rows: one per block column)
    // and the bands' arrival counters (re-armed by the last contribution).
    int n_dense_tiles, dense_nct_max;
    int n_sm;                   // host: SMs of the device (the dense launch's grid)
    const int4 *dense_tiles;
    const R *dense_inv;
    const int *dense_col, *dense_bptr, *dense_bidx;
    V4<R> *dense_part;
    int *dense_cnt;
    V4<R> *u;                   // update vectors
    V4<R> *part_r;              // 32 partial sums per backward item (chunk items)
    int *cb_cnt;                // chunks finished per backward column block (re-arms itself)
    unsigned int *err;          // set nonzero if a bulk copy did not arrive in time
    cudaStream_t stream;        // host: the stream of the launch in progress
};

// r = A0^{-1} q on the first nf entries (q, r: V4 arrays, may not alias).
template <typename R>
void launch_solve(const DevSolve<R> &s, const V4<R> *q, V4<R> *z, V4<R> *r, cudaStream_t st);
// Dynamic shared memory of a sweep block staging qcap factor entries and
// vectors of ld entries.
template <typename R> size_t solve_block_smem(int qcap, int ld);
// Raises the sweeps' dynamic shared-memory limits (once per device).
template <typename R> cudaError_t solve_prepare();

}  // namespace hqn
