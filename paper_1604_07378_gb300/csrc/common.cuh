// Device-side types shared by the kernels and the host orchestration of the
// quasi-Newton implicit-Euler step (Alg. 1 with the L-BFGS direction of Alg. 2).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/hqn.h"

namespace hqn {

// One vertex's 3-vector, padded to 16 B (float) or 32 B (double) so a gather
// of a vertex is one aligned vector load.  The pad lane w is kept at zero.
template <typename R>
struct alignas(4 * sizeof(R)) V4 {
    R x, y, z, w;
};

// Material as the tet kernel consumes it (Eq. valanis-landel).  For the
// spline material each of a, b, c is 7 cubic segments p0 + u(p1 + u(p2 + u p3)),
// u = (t - x_i) * inv_h, over knots x_0..x_7, continued quadratically outside.
// The spline energy is evaluated about the rest state (t = 1 for a, b, c):
// f(t) = f(1) + f'(1) (t - 1) + df(t), with df taken inside segment i about
// its point nearest 1 (u = ur[f][i]) using the constants
// dD[f][i] = f'(ref) - f'(1) and dE[f][i] = f(ref) - f(1) - f'(1) (ref - 1),
// so no first-order terms of size mu cancel in float32.
template <typename R>
struct MatDev {
    int kind;
    R mu, lam;          // Lame parameters
    R J0, c0, c1, c2;   // Neo-Hookean: c(J0), c'(J0), c''(J0) of the continuation below J0
    R kx[3][8];         // spline knots of a, b, c
    R inv_h[3][7];
    R p[3][7][4];
    R ur[3][7], dD[3][7], dE[3][7];
    R K0;               // a'(1) + 2 b'(1) + c'(1): the stress of the rest state
    R B1C1, C1;         // b'(1) + c'(1) and c'(1)
    R psi_rest;         // 3 a(1) + 3 b(1) + c(1)
    R kappa;            // anisotropic fibre term kappa/2 (|F d| - 1)^2 (0: none)
    R fd[3];            // its unit rest direction d
};

// History windows up to this many pairs keep the scalars of Alg. 2's two
// loops in the control block and the vectors' per-slot terms in registers;
// longer windows (up to HQN_MAX_HISTORY) keep them in a device array of
// their own (SimDesc::lh) and reduce over the slots in chunks.
constexpr int kShortHist = 16;

// Control block of one simulation's step, resident on the device.  Every
// scalar decision of Alg. 1 / Alg. 2 (inner products, alpha, Armijo, history
// bookkeeping) is taken here, by the last block of the kernel that produces
// its inputs, so a step runs without host round trips.
struct Ctl {
    double g_k;        // g(x_k)
    double g_trial;    // g at the current line-search trial
    double e_k;        // elastic energy E(x_k) (the Armijo test compares differences)
    double e_trial;    // E at the accepted trial
    double gd;         // tr(grad_k^T d)
    double alpha;      // current step length
    double g0;         // g(x_1), x_1 = y
    double ls_a[3];    // inertia term along d: I(alpha) = a0 + a1 alpha + a2 alpha^2
    double pcg_rz, pcg_alpha, pcg_beta;  // Jacobi-PCG scalars (iterative A0^{-1})
    double cheb_omega; // Chebyshev weight omega_k of Alg. 3
    // (windows of m <= kShortHist pairs; longer ones use SimDesc::lh)
    double zeta[kShortHist + 1];  // first-loop coefficients by age (0 = newest)
    double coef[kShortHist + 1];  // second-loop coefficients zeta - eta by age
    double rho[kShortHist + 1];   // tr(t^T s) by ring slot
    double sg[kShortHist + 1];    // s_a^T grad_k by ring slot
    double tr0[kShortHist + 1];   // t_a^T r0 by ring slot (r0 = A0^{-1} q)
    double gram[kShortHist + 1][kShortHist + 1];  // s_a^T t_b by ring slots
    double iter_g[HQN_MAX_ITERS];
    int iter_trials[HQN_MAX_ITERS];
    int k;             // 1-based iteration index of x_k
    int trials;        // trials of the current line search
    int count;         // history pairs held (<= m)
    int head;          // ring slot of the newest pair (ring has m + 1 slots)
    int hist_w;        // ring slot of the last pair pushed (long windows)
    int hist_keep;     // that pair was kept (long windows)
    int stop;          // the step's iterations have ended early
    int status;        // worst status of the step (HQN_OK or a warning)
    int accepted;      // the last trial passed the Armijo test
    int grad_ready;    // the corner gradients already belong to the accepted point
    int active;        // this simulation is still iterating in the current step
    int nondescent;    // tr(grad^T d) >= 0 with history: reset and recompute
    int trials_total;  // over the steps since the host last cleared it
    int iters_total;
    int steps;
    int worst_status;
    int passes_total;  // line-search passes (each tests up to ls_batch step lengths)
    unsigned int solve_err;  // nonzero: a sweep's bulk copy timed out (sticky)
    unsigned int ticket[8];  // arrival counters of the last-block reductions
};

// Ticket slots (one per kernel family so consecutive kernels never share one).
enum { TK_TRIAL = 0, TK_TET = 1, TK_GATHER = 2, TK_VEC = 3, TK_LS = 4, TK_DOT = 5, TK_PCG_A = 6, TK_PCG_B = 7 };

// Graph conditional handles a kernel may set (0 = not inside a graph).
struct CondHandles {
    unsigned long long it;   // while: iterations of the step
    unsigned long long ls;   // while: line-search trials
    unsigned long long nd;   // if: non-descent reset of the direction
};

// An analytic collider (Sec. 4.3): plane (point p, unit normal n) or sphere
// (centre p, radius r).
template <typename R>
struct ColDev {
    int kind;
    R px, py, pz, nx, ny, nz, r;  // point / centre, unit normal / axis, radius (tube radius)
    R ring;                       // torus ring radius
};

// Per-simulation constants passed by value.
template <typename R>
struct StepConst {
    int n, nf, T, m, iters, ls_max, ls_batch;
    R h2;              // h^2
    R gx, gy, gz;      // h^2 * gravity (the h^2 M^{-1} f_ext term of Eq. PD)
    double gamma, backtrack;
    R kstiff;          // the stiffness k of Eq. stiffness (the matrix-free L of A0)
    int cheb, cheb_S;  // the Chebyshev direction of Alg. 3 (cheb = 1) and its S
    double cheb_rho2;  // rho^2
    int ncol;          // colliders (0: no collision terms)
    R cscale;          // collision weight w_v = cscale * m_v / h^2
    ColDev<R> col[HQN_MAX_COLLIDERS];
};

}  // namespace hqn
