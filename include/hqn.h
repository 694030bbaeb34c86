/*
 * hqn.h - C ABI of the GB300 quasi-Newton implicit-Euler solver for
 * hyperelastic tetrahedral meshes.
 *
 * Method: Liu, Bouaziz & Kavan, "Towards Real-time Simulation of Hyperelastic
 * Materials" (arXiv 1604.07378).  One implicit-Euler time step is the
 * minimisation of
 *     g(x) = 1/(2h^2) tr((x - y)^T M (x - y)) + E(x),
 *     y    = 2 q_l - q_{l-1} + h^2 M^{-1} f_ext                      (Eq. PD)
 * by Alg. 1 (quasi-Newton iterations with backtracking Armijo line search),
 * whose descent direction comes from the L-BFGS two-loop recursion of Alg. 2
 * with the constant initial Hessian A0 = M/h^2 + L (Sec. 4.2, Eq. PDsolution),
 * prefactored once.  E is a Valanis-Landel energy in principal stretches
 * (Eq. valanis-landel); L is weighted by the stiffness fit of Eq. stiffness.
 *
 * Conventions common to every entry point
 *   - Positions are absolute coordinates in the caller's vertex order, host
 *     arrays of n_verts x 3 doubles, row-major (x, y, z per vertex).
 *   - Every pointer argument is owned by the caller; the library copies what it
 *     needs and keeps no reference after the call returns.
 *   - A handle owns all the device memory it allocates (on the device that is
 *     current when sim_create runs) and frees it in sim_destroy.  All device
 *     work of a handle is issued on the CUDA stream given to sim_create.
 *   - Return codes: 0 = success, > 0 = warning (the result is usable), < 0 =
 *     error (the handle's state is unchanged unless stated otherwise).
 *     sim_strerror() maps a code to a static string.  No C++ exception ever
 *     crosses this boundary.
 *   - Calls on one handle must not overlap (thread-compatible, not
 *     thread-safe); different handles are independent.
 */
#ifndef HQN_H
#define HQN_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes ------------------------------------------------------- */
#define HQN_OK                    0
#define HQN_WARN_LS_EXHAUSTED     1  /* a line search hit ls_max trials; that step's
                                        iterations ended at the last accepted x   */
#define HQN_WARN_NONDESCENT       2  /* grad^T d >= 0 (only at a stationary point);
                                        that step's iterations ended             */
#define HQN_ERR_ARG              -1  /* null pointer, bad size, index out of range */
#define HQN_ERR_DEGENERATE_TET   -2  /* a rest tet has det(Dm) <= 0              */
#define HQN_ERR_NONFINITE        -3  /* NaN/Inf in an input or in the state       */
#define HQN_ERR_NOT_SPD          -4  /* A0 is not positive definite               */
#define HQN_ERR_CUDA             -5  /* a CUDA runtime call failed                */
#define HQN_ERR_NO_MEMORY        -6  /* host or device allocation failed          */
#define HQN_ERR_UNSUPPORTED      -7  /* option or size the library does not support */
#define HQN_ERR_DEVICE_TIMEOUT   -8  /* a bounded wait on the device ran out (a sweep's
                                        copy of its factor rows did not arrive); the
                                        step was abandoned and the state is undefined */

/* ---- materials (Eq. valanis-landel: Psi = sum a(s_i) + sum b(s_i s_j) + c(J)) */
typedef enum {
    HQN_NEOHOOKEAN = 0, /* a = mu/2 (x^2-1), b = 0, c = -mu ln J + lam/2 ln^2 J;
                           for J < 0.05, c is its 2nd-order Taylor polynomial at 0.05 */
    HQN_STVK       = 1, /* mu ||E||^2 + lam/2 tr^2 E, E = (F^T F - I)/2              */
    HQN_SPLINE_VL  = 2, /* a, b, c are C1 cubic Hermite splines (Sec. 4.1,
                           "spline-based materials"); quadratic extension outside  */
    HQN_COROTATED  = 3, /* a = mu (x-1)^2, c = lam/2 (J-1)^2                           */
    HQN_POLY4      = 4  /* a = mu (x-1)^4 (the paper's polynomial material)           */
} hqn_material_kind;

typedef enum {
    HQN_FP64_PLAIN = 0, /* every kernel in float64                                  */
    HQN_FP32_MIXED = 1  /* float32 tets, two-loop vectors and triangular solves;
                           float64 energy sums, Armijo test and inner products      */
} hqn_precision;

/* An analytic collider (see hqn_params.colliders). */
#define HQN_MAX_COLLIDERS 4
typedef enum {
    HQN_COLLIDER_PLANE  = 1,  /* point[3] on the plane, normal[3] towards the free side
                                 (normalised by the library)                         */
    HQN_COLLIDER_SPHERE = 2,  /* centre point[3], radius; the body stays outside      */
    HQN_COLLIDER_TORUS  = 3   /* centre point[3], axis normal[3] (normalised by the
                                 library), ring radius major_radius, tube radius
                                 radius (0 < radius < major_radius); the body stays
                                 outside the tube.  Vertices on the axis or on the
                                 ring circle have no unique normal and get no term */
} hqn_collider_kind;
typedef struct {
    int32_t kind;             /* hqn_collider_kind */
    double  point[3];
    double  normal[3];
    double  radius;
    double  major_radius;     /* HQN_COLLIDER_TORUS only */
} hqn_collider;

typedef struct {
    int32_t        n_verts;
    int32_t        n_tets;
    const double  *rest_pos;  /* n_verts x 3 rest positions X                        */
    const int32_t *tets;      /* n_tets x 4 vertex indices; det[X1-X0,X2-X0,X3-X0] > 0 */
    const uint8_t *clamped;   /* n_verts flags, nonzero = position prescribed (held
                                 at its current state); NULL = none clamped          */
    /* Several materials in one mesh.  The energy of Eq. PD is a sum over
     * elements, so each tet may have its own material: its energy density,
     * its share of the lumped mass (that material's density) and its weight
     * V k in L (k of Eq. stiffness fitted per material) are its material's.
     * n_materials = 0 or 1: every tet has material 0 and tet_material is
     * ignored (may be NULL). */
    int32_t        n_materials;  /* 0 .. HQN_MAX_MATERIALS                          */
    const int32_t *tet_material; /* n_tets indices in [0, n_materials)              */
} hqn_mesh;
#define HQN_MAX_MATERIALS 16

typedef struct {
    int32_t       kind;       /* hqn_material_kind                                    */
    double        E, nu;      /* Young's modulus [Pa] > 0, Poisson ratio in (-1, 0.5)
                                 -> mu, lambda (HQN_ERR_ARG otherwise)               */
    double        density;    /* [kg/m^3]; lumped mass m_v = density * sum V_t / 4    */
    const double *spline;     /* HQN_SPLINE_VL only: 3 x 8 x 3 doubles, function
                                 (a, b, c) x knot x (knot, value, slope), knots
                                 strictly increasing; otherwise ignored (may be NULL) */
    double        kappa;      /* anisotropic fibre term (Sec. 4.4): adds
                                 kappa/2 (|F d| - 1)^2 per unit rest volume to any
                                 base material; 0 = none.  A0 keeps the base
                                 material's stiffness fit.                           */
    double        fiber[3];   /* rest-pose fibre direction d (normalised by the
                                 library; nonzero when kappa > 0)                   */
} hqn_material;

typedef struct {
    double  h;            /* time step [s]; paper: 1/30 (Sec. 3)                       */
    double  gamma;        /* Armijo constant; paper: 0.3 (Sec. 4.1)                    */
    double  backtrack;    /* step shrink factor; paper: 0.5 (Alg. 1)                   */
    double  x_start;      /* stiffness-fit interval; paper: [0.5, 1.5] (Sec. 5)        */
    double  x_end;
    double  gravity[3];   /* [m/s^2], f_ext = m_v * gravity                           */
    int32_t iters;        /* quasi-Newton iterations per step; paper: 10 (Table 1)    */
    int32_t history_m;    /* L-BFGS window, 0..HQN_MAX_HISTORY; paper: 5 (Sec. 4.2), up
                             to 100 in its convergence study (Sec. 5); 0 = Alg. 1
                             direction.  Windows above 16 pairs keep the two
                             loops' scalars in a device array of (m + 1)^2 +
                             5 (m + 1) doubles per simulation and form the slot
                             products in chunks of 16 slots (two more launches
                             after the gather and after the solve)          */
    int32_t ls_max;       /* line-search trials before giving up (paper is silent)    */
    int32_t precision;    /* hqn_precision                                            */
    int32_t leaf_size;    /* max vertices of a nested-dissection leaf (0 = default:
                             128 in HQN_FP32_MIXED up to 150,000 free vertices,
                             64 otherwise)                                       */
    int32_t use_graph;    /* 1 = run each step as one CUDA graph with conditional
                             (while / if) nodes for the iteration and line-search
                             loops; 0 = host-driven launches (same kernels)        */
    int32_t tet_block;    /* threads per block of the tet kernels: 0 or 128 (other
                             values are rejected with HQN_ERR_UNSUPPORTED)         */
    int32_t ls_batch;     /* line search: the first trial (alpha = 1) is one tet pass
                             fused with the gradient; after a rejection each pass
                             tests ls_batch step lengths (1, 2, 4, 8 or 16; 0 =
                             default 8; other values HQN_ERR_ARG).  The accepted
                             alpha is the one Alg. 1's sequential backtracking
                             would accept                                          */
    /* Shapes of the triangular sweeps of A0^{-1} (one launch per tree level;
     * every level's factor rows split into work items of consecutive rows,
     * one thread block each).  They change the speed, not the arithmetic of
     * a row, except that a different split of the backward rows into chunk
     * items sums some rows in another order (rounding-level differences).
     * 0 selects the default; the autotuner (paper_1604_07378_gb300/autotune.py)
     * picks them per mesh and GPU. */
    int32_t solve_threads;  /* threads per sweep block: 128, 256 or 512 (default 256) */
    int32_t solve_item_kb;  /* largest work item, KB of factor rows: 16..160
                               (default 64)                                      */
    int32_t solve_items;    /* work items a level's rows are spread over: 16..4096
                               (default 400)                                     */
    int32_t solve_leaf_kb;  /* largest work item of the leaf level (level 0, whose
                               items depend on no other level): 8..160, 0 = as
                               solve_item_kb                                     */
    int32_t solve_leaf_threads; /* threads per block of the leaf level: 128, 256 or
                               512, 0 = as solve_threads                         */
    int32_t solve_dense_top;/* the supernodes of the tree's top solve_dense_top levels
                               (1..8) are solved together, r_T = S^{-1} f_T with
                               the inverse of A0's Schur complement on their
                               columns (formed once on the host in float64):
                               one tiled dense product replaces 2 solve_dense_top
                               launches of the sweeps.  0 (default) = automatic:
                               the most levels, at most 3, whose block has at
                               most 5,000 columns (the host's cost grows as the
                               cube of the columns); -1 = none.  Set at
                               sim_create (not by sim_set_solve_shapes)        */
    int32_t solve_prefetch; /* a level's blocks ask L2 to prefetch the factor rows
                               of the level this many launches ahead: 1..8; 0 or
                               -1 = none (default; on a 40^3 lattice it left the
                               solve's time unchanged and cost the step 3% of L2
                               hits elsewhere)                                   */
    int32_t solve_dense_prefetch; /* 1 = the forward levels before the dense top
                               block stream its matrix into L2 (a faster solve,
                               a slower step on a 40^3 lattice); 0 = no (default) */
    /* Collisions (Sec. 4.3) against analytic colliders, shared by every
     * simulation of a handle.  At the start of each iteration (before the
     * gradient at x_k) every free vertex that penetrates a collider and does
     * not move away from it over the step (its displacement from the state
     * q_l has a non-positive normal component) gets the energy term
     * w_v ((x_v - t)^T n)^2, with t its projection on the collider and n the
     * surface normal there, both frozen for the iteration, and
     * w_v = contact_scale * m_v / h^2.  The terms enter the objective, its
     * gradient and the line search but not A0 (no refactorisation).
     * n_colliders = 0 (the default) disables them. */
    int32_t n_colliders;  /* 0 .. HQN_MAX_COLLIDERS                                */
    double  contact_scale;/* > 0 when n_colliders > 0 (default 100)                */
    hqn_collider colliders[HQN_MAX_COLLIDERS];
    /* The initial Hessian's solve r = A0^{-1} q of Alg. 2: 0 = the factorised
     * A0 (default); 1 = pcg_iters iterations of Jacobi-preconditioned
     * conjugate gradients from zero, A0 applied matrix-free (the paper's
     * comparison with iterative solvers; the three coordinate columns form one
     * vector).  sim_solve_A0 then returns that approximation. */
    int32_t a0_solver;
    int32_t pcg_iters;    /* >= 1 when a0_solver = 1 (default 15)                  */
    /* The descent direction: 0 = L-BFGS (Alg. 2, default); 1 = the Chebyshev
     * semi-iterative direction of Alg. 3 with cheb_S and cheb_rho (no history;
     * history_m is ignored): q = -A0^{-1} grad, d = omega (x_k + q - x_{k-1})
     * + x_{k-1} - x_k, omega = 1 for k < S, 2/(2 - rho^2) at k = S,
     * 4/(4 - rho^2 omega_k) after; x_0 is read as x_1. */
    int32_t direction;
    int32_t cheb_S;       /* default 10                                            */
    double  cheb_rho;     /* spectral radius estimate in (0, 1) (default 0.99)     */
    /* Supernode amalgamation of the factored A0: a nested-dissection node at
     * depth d (the root at 0) whose bit d is set merges with its children's
     * separators into one supernode, which removes a level from each
     * triangular sweep at the price of explicit zeros and some fill.  No two
     * adjacent bits may be set (an update entry then has at most four
     * sources); HQN_ERR_ARG otherwise.  A merge that would give a supernode
     * more than 4096 columns is skipped.  Default 0 (the plain dissection
     * tree): on a 40^3 lattice every mask tried made the solve slower, since
     * each work item of a wide supernode gathers its whole right-hand side. */
    int32_t merge_depths;
    /* Failure detection.  Every device wait of the sweeps is bounded: a block
     * polls its bulk copy's barrier at most wait_polls times (0 = default
     * 2^20), then flags the error, waits (bounded) for a copy still in
     * flight and leaves; sim_step, sim_solve_A0 and sim_direction then
     * return HQN_ERR_DEVICE_TIMEOUT.  fault_test is fault injection for
     * tests of that path and stays 0 otherwise: 1 = the blocks of the first
     * forward sweep level (the leaves) of every solve issue no copy, so
     * their waits run out with nothing in flight (a tree whose every level is
     * in the dense top block has no such level). */
    int32_t wait_polls;
    int32_t fault_test;
    /* Path of an autotuner cache (see hqn_tune_lookup), or NULL.  When set,
     * sim_create and sim_batch_create look up the mesh (hqn_mesh_key; for a
     * batch, the keys of all meshes folded in order), the precision and the
     * current device's name there, and, on a hit, replace leaf_size,
     * solve_threads, solve_item_kb, solve_items, solve_prefetch (and
     * solve_leaf_kb, solve_leaf_threads, solve_dense_top,
     * solve_dense_prefetch and ls_batch if the entry has them) by the tuned
     * values.  A missing file
     * or entry leaves the parameters as given; a malformed file is
     * HQN_ERR_ARG. */
    const char *tune_cache;
} hqn_params;

#define HQN_MAX_HISTORY 128
#define HQN_MAX_ITERS   512

/* Per-step record of the most recent step taken by sim_step. */
typedef struct {
    int32_t steps;                          /* steps taken by this sim_step call     */
    int32_t iters;                          /* iterations of the last step           */
    int32_t status;                         /* worst status over the call's steps    */
    int32_t trials_total;                   /* line-search trials, all steps         */
    int32_t iters_total;                    /* iterations, all steps                 */
    int32_t trials[HQN_MAX_ITERS];          /* trials of each iteration, last step   */
    double  g0;                             /* g(x_1), x_1 = y, last step            */
    double  g[HQN_MAX_ITERS];               /* g(x_{k+1}) after each iteration       */
    int32_t ls_passes_total;                /* line-search tet passes, all steps     */
} hqn_step_stats;

typedef struct {
    int32_t n_verts, n_tets, n_free;
    int32_t n_supernodes, n_levels;
    int64_t factor_entries;     /* stored entries of the solve operators [Linv; K]    */
    int64_t factor_nnz;         /* nonzeros of the Cholesky factor L (incl. padding)  */
    double  stiffness_k;        /* fitted k of Eq. stiffness                          */
    double  setup_seconds;      /* host time spent in sim_create                      */
    int64_t device_bytes;       /* device memory held by the handle                   */
    int32_t precision;          /* hqn_precision in use                               */
    int32_t graph_mode;         /* 1 if steps run as a CUDA graph                     */
    int64_t n_update_entries;   /* entries of the forward-sweep update vectors        */
    int32_t chained_sweeps;     /* 1 if the per-level sweeps use programmatic dependent
                                   launch (a level starts while the previous finishes) */
    int32_t solve_threads;      /* sweep shapes in use (see hqn_params.solve_*)           */
    int32_t solve_item_kb;
    int32_t solve_items;
    int32_t solve_leaf_kb;
    int32_t solve_leaf_threads;
    int32_t solve_prefetch;     /* 0 = no prefetch                                        */
    int32_t solve_dense_prefetch;
    int32_t solve_dense_top;    /* top levels solved by the dense block (0 = none), of the
                                   first simulation                                       */
    int32_t dense_top_cols;     /* columns of that block (largest simulation)              */
    int32_t n_sims;             /* simulations in the handle (1 for sim_create)        */
} hqn_info;

typedef struct sim_handle sim_handle;

/* Paper defaults: h = 1/30, gamma = 0.3, backtrack = 0.5, [0.5, 1.5], gravity
 * (0, 0, -9.81), 10 iterations, m = 5, ls_max = 30, FP32_MIXED, leaf size 0
 * (the size-dependent default), no supernode merges, graph mode on, tet
 * block 128, 8 line-search trials per pass. */
void hqn_default_params(hqn_params *p);

/* Host-only analysis: the set-up sim_create performs on the host (rest data,
 * the stiffness k of Eq. stiffness, A0's nested-dissection ordering and
 * float64 supernodal Cholesky factor, the sweeps' levels) for one mesh,
 * without a GPU and without keeping anything.  Fills the fields of *info
 * that the set-up determines: n_verts, n_tets, n_free, n_supernodes,
 * n_levels, factor_entries, factor_nnz, stiffness_k, setup_seconds,
 * n_update_entries, and precision, graph_mode and the solve_* shapes as
 * requested by *params (n_sims = 1); the device-dependent fields are 0.
 * Errors: those of sim_create other than HQN_ERR_CUDA. */
int hqn_analyse(const hqn_mesh *mesh, const hqn_material *material,
                const hqn_params *params, hqn_info *info);

/* Builds a simulation: rest data (Dm^-1, volumes, lumped mass), the stiffness k
 * of Eq. stiffness, A0 = M/h^2 + sum_t V_t k G_t^T G_t on the free vertices
 * (Eq. PDmatrixForm, PDsolution), its nested-dissection ordering and float64
 * supernodal Cholesky factor, and the device operators of the triangular
 * solves.  `material` points to max(1, mesh->n_materials) materials.  The
 * state starts at rest (q_l = q_{l-1} = X).  `stream` is a cudaStream_t
 * (NULL = legacy default stream).
 * Errors: HQN_ERR_ARG, HQN_ERR_DEGENERATE_TET, HQN_ERR_NONFINITE,
 * HQN_ERR_NOT_SPD, HQN_ERR_CUDA, HQN_ERR_NO_MEMORY.  *out is NULL on error. */
int sim_create(const hqn_mesh *mesh, const hqn_material *material,
               const hqn_params *params, void *stream, sim_handle **out);

/* ---- batches -------------------------------------------------------------
 * The paper simulates one object at a time; a batch advances `count`
 * independent simulations (each its own mesh, material, factor and state; the
 * parameters are shared) in lockstep, every kernel stage of a step launched
 * once for the whole batch and the step captured as one CUDA graph.  Each
 * simulation takes exactly the iterations and line-search trials it would
 * take alone (a finished simulation idles while others continue), so its
 * results equal those of a handle made by sim_create for it alone.
 * meshes is an array of `count`; materials holds the meshes' material arrays
 * back to back (max(1, n_materials) of them per mesh, in mesh order).
 * Errors as sim_create; a failing simulation is named in hqn_last_error().
 * For a batch handle, sim_set_state, sim_get_state, sim_energy_grad,
 * sim_solve_A0 and sim_direction act on simulation 0; sim_step advances all
 * simulations and its stats carry simulation 0's per-iteration record with
 * trials_total, iters_total and ls_passes_total summed over the batch and
 * status the worst over the batch. */
int sim_batch_create(int32_t count, const hqn_mesh *meshes, const hqn_material *materials,
                     const hqn_params *params, void *stream, sim_handle **out);

/* Simulations in the handle (0 for NULL). */
int32_t sim_batch_count(const sim_handle *sim);

/* sim_set_state / sim_get_state for simulation `index` of a batch. */
int sim_batch_set_state(sim_handle *sim, int32_t index, const double *q_cur, const double *q_prev);
int sim_batch_get_state(sim_handle *sim, int32_t index, double *q_cur, double *q_prev);

/* The step record of simulation `index` (its own totals since the last
 * sim_step call began).  Synchronises the stream. */
int sim_batch_get_stats(sim_handle *sim, int32_t index, hqn_step_stats *stats);

/* Sets the state (q_l, q_{l-1}) of Eq. PD -- the positions of the current and
 * the previous time step, from which the predictor y = 2 q_l - q_{l-1} +
 * h^2 M^{-1} f_ext of the next step is formed (Sec. 3); each n_verts x 3 host
 * doubles.  An initial velocity v enters as q_{l-1} = q_l - h v.  Clamped
 * vertices are held at their q_l.  q_prev may be NULL (= q_cur, zero
 * velocity).  The state is the whole state between steps (the L-BFGS history
 * is reset every step), so sim_get_state / sim_set_state checkpoint and
 * resume a simulation. */
int sim_set_state(sim_handle *sim, const double *q_cur, const double *q_prev);

/* Copies the state (q_l, q_{l-1}) of Eq. PD out (either pointer may be NULL).
 * Synchronises the stream. */
int sim_get_state(sim_handle *sim, double *q_cur, double *q_prev);

/* Advances nsteps time steps (Alg. 1 with Alg. 2) on the device.  stats may be
 * NULL.  Returns the worst status over the steps (a warning keeps going). */
int sim_step(sim_handle *sim, int32_t nsteps, hqn_step_stats *stats);

/* Layouts of sim_positions_device (caller's vertex order, w = 0). */
#define HQN_LAYOUT_F32X4 1  /* n_verts x {float x, y, z, w}  */
#define HQN_LAYOUT_F64X4 2  /* n_verts x {double x, y, z, w} */

/* Device copy of the current positions q_l (the state of Eq. PD) of
 * simulation 0, for consumers that stay on the device (rendering, coupling).
 * The buffer belongs to the handle (allocated on the first call) and is
 * borrowed: it is complete when the call returns and valid until the next
 * sim_positions_device, sim_step, sim_set_state or sim_destroy on the handle.
 * *layout = HQN_LAYOUT_F32X4 in HQN_FP32_MIXED (rest position plus float32
 * displacement, added in float32), HQN_LAYOUT_F64X4 in HQN_FP64_PLAIN.
 * Errors: HQN_ERR_ARG (null argument), HQN_ERR_NO_MEMORY, HQN_ERR_CUDA. */
int sim_positions_device(sim_handle *sim, void **dev_ptr, int32_t *layout);

/* Evaluates g and grad g (Eq. PD) at positions x with inertial target y (both
 * n_verts x 3 host doubles).  Clamped vertices are eliminated: the inertia
 * term sums over the free vertices only and grad is zero on clamped rows (a
 * clamped row of x still enters the elastic energy of its tets).  g_out or
 * grad_out may be NULL.  Does not change the state. */
int sim_energy_grad(sim_handle *sim, const double *x, const double *y,
                    double *g_out, double *grad_out);

/* sim_energy_grad on device arrays: x_dev and y_dev are n_verts x 3 doubles
 * in the caller's vertex order in device memory (on the handle's device;
 * read by kernels on the handle's stream, so they must be ready there), and
 * grad_dev (n_verts x 3 doubles, device; may be NULL) receives grad g in the
 * same order, zero on clamped rows.  *g_out (host; may be NULL) receives g.
 * The positions are not checked for NaN/Inf (a non-finite input gives a
 * non-finite g).  Returns after the work is done (the stream is
 * synchronised).  The first call allocates the handle's copies of its
 * float64 rest positions and vertex order on the device.
 * Errors: HQN_ERR_ARG, HQN_ERR_NO_MEMORY, HQN_ERR_CUDA. */
int sim_energy_grad_device(sim_handle *sim, const double *x_dev, const double *y_dev, double *g_out,
                           double *grad_dev);

/* r = A0^{-1} q on the free vertices by the device forward and backward
 * triangular solves (3 right-hand sides); rows of clamped vertices are ignored
 * in q and set to zero in r.  Host arrays n_verts x 3. */
int sim_solve_A0(sim_handle *sim, const double *q, double *r);

/* Alg. 2 on the device: d from grad and `npairs` history pairs (s_i, t_i),
 * oldest first, each n_verts x 3 (s and t are npairs x n_verts x 3).  Pairs are
 * used as given (no curvature filtering); npairs <= history_m. */
int sim_direction(sim_handle *sim, const double *grad, int32_t npairs,
                  const double *s, const double *t, double *d);

/* Stages that sim_time_stage can time in isolation. */
typedef enum {
    HQN_STAGE_TET      = 0, /* energy + corner gradients of every tet at the last trial x */
    HQN_STAGE_GATHER   = 1, /* vertex gather of grad g                                  */
    HQN_STAGE_SOLVE    = 2, /* forward + backward sweeps of A0^{-1} (3 right-hand sides) */
    HQN_STAGE_LS_PASS  = 3, /* one multi-trial line-search pass (ls_batch energies/tet)  */
    HQN_STAGE_TWO_LOOP = 4  /* both loops of Alg. 2 around one solve                     */
} hqn_stage;

/* Launches one stage `reps` times on the handle's stream, bracketed by CUDA
 * events recorded on that stream, and returns the mean device time of one
 * launch in *ms.  Uses the handle's current buffers (call after sim_step);
 * leaves the state (q_l, q_{l-1}) unchanged.  Synchronises the stream. */
int sim_time_stage(sim_handle *sim, int32_t stage, int32_t reps, double *ms);

/* ---- autotuning ------------------------------------------------------------
 * The paper has no counterpart: these entry points serve the project's
 * autotuner (paper_1604_07378_gb300/autotune.py), which times the sweep
 * shapes and the leaf size on the device and writes its choices to a cache
 * file that sim_create reads (hqn_params.tune_cache). */

/* New sweep shapes on an existing handle: the fields solve_threads,
 * solve_item_kb, solve_items, solve_leaf_kb, solve_leaf_threads and
 * solve_prefetch and solve_dense_prefetch of *shapes (0 = default; the other
 * fields are ignored).  The
 * work items are re-planned from the handle's own factor (no
 * refactorisation) and the step graph is rebuilt.  Results change by
 * rounding only (other row splits), or not at all (threads, prefetch).
 * solve_dense_top stays as created.  Errors: HQN_ERR_ARG (a shape out of
 * range), HQN_ERR_UNSUPPORTED (items that do not fit a block's shared
 * memory), HQN_ERR_CUDA. */
int sim_set_solve_shapes(sim_handle *sim, const hqn_params *shapes);

/* 64-bit FNV-1a hash of a mesh (sizes, rest positions, tets, clamp flags):
 * the key of its autotuner cache entries.  0 for a NULL or empty mesh.
 * Host only. */
uint64_t hqn_mesh_key(const hqn_mesh *mesh);

/* Looks up (device, key, precision) in the autotuner cache file at `path`
 * (host only; `device` is a CUDA device name).  The file holds one entry
 * per line, later lines overriding earlier ones, '#' lines ignored:
 *   hqn-tune 1 device=<name, spaces as '_'> precision=<0|1> key=<16 hex>
 *     leaf_size=<n> solve_threads=<n> solve_item_kb=<n> solve_items=<n>
 *     solve_prefetch=<n> [solve_leaf_kb=<n>] [solve_leaf_threads=<n>]
 *     [solve_dense_top=<n>] [solve_dense_prefetch=<0|1>] [ls_batch=<n>]
 *     [other key=value pairs, ignored]
 * (leaf_size=0, solve_dense_top=0 and the solve_* zeros keep the library's
 * size-dependent defaults.)
 * Returns 1 and writes the entry's values into *params on a hit, 0 when the
 * file or the entry does not exist (params unchanged), HQN_ERR_ARG for a
 * malformed file or argument. */
int hqn_tune_lookup(const char *path, const char *device, uint64_t key, int32_t precision, hqn_params *params);

int  sim_get_info(const sim_handle *sim, hqn_info *info);
void sim_destroy(sim_handle *sim);
const char *sim_strerror(int code);

/* Measures the current device's non-tensor fused multiply-add throughput in
 * the precision's floating-point type (HQN_FP32_MIXED: float, HQN_FP64_PLAIN:
 * double), in FLOP/s (an FMA counts 2): independent FMA chains on every SM,
 * timed with CUDA events over a launch of at least 20 ms.  The FLOP roofline
 * of the tet pass.  Allocates a few bytes of device memory and a stream for
 * the call.  Errors: HQN_ERR_ARG, HQN_ERR_CUDA. */
int hqn_measure_peak(int32_t precision, double *flops_per_s);

/* Message of the last error raised on the calling thread ("" if none). */
const char *hqn_last_error(void);

/* ---- allocation-free evaluation ------------------------------------------
 * The paper has no counterpart of this entry point; it exists for callers
 * that cannot allocate device memory: code running inside a memory pool or
 * budget owned by someone else, plug-ins that must not call the CUDA
 * allocator, and drivers that forbid cudaMalloc once they are running.
 *
 * hqn_energy_grad_static computes g(x) = 1/(2h^2) sum_v m_v |x_v - y_v|^2 +
 * sum_t V_t Psi(F_t) (v over the free vertices) and grad g(x) -- the
 * quantities sim_energy_grad returns -- in float64 without a handle and
 * without allocating anything.  Its
 * scratch (per-tet corner gradients, per-block partial sums) is one
 * fixed-size array of about 8.4 MB that the library places in each GPU's
 * memory when it is loaded there and keeps until the process exits.
 *
 * Arguments (device pointers unless stated; all caller-owned, caller order):
 *   n_verts, n_tets   1 <= n_tets <= HQN_STATIC_MAX_TETS,
 *                     1 <= n_verts <= HQN_STATIC_MAX_VERTS; larger meshes
 *                     are rejected with HQN_ERR_ARG before any device work
 *   rest_pos          n_verts x 3 doubles, rest positions X
 *   tets              n_tets x 4 int32 in [0, n_verts), det[X1-X0, X2-X0,
 *                     X3-X0] > 0 (a tet that breaks this makes *g_out NaN)
 *   clamped           n_verts bytes, nonzero = eliminated vertex: no inertia
 *                     term, gradient row set to zero; may be NULL
 *   vt_ptr, vt_slot   incident-corner CSR: the corners of vertex v are
 *                     vt_slot[vt_ptr[v] .. vt_ptr[v+1]), each encoded as
 *                     4 * tet + corner (vt_ptr has n_verts + 1 entries); the
 *                     gradient sums them in this order (no atomics)
 *   material          HOST pointer, checked as in sim_create (E > 0,
 *                     -1 < nu < 0.5, known kind, increasing spline knots,
 *                     fibre term) plus density > 0, which gives the lumped
 *                     mass m_v = density * sum of incident V_t / 4
 * Indices are checked on the device before use: a tet vertex outside
 * [0, n_verts), or a vt_ptr range or vt_slot entry outside [0, 4 n_tets), is
 * never dereferenced; the affected gradient rows and *g_out are then NaN.
 *   h                 time step (> 0)
 *   x, y              n_verts x 3 doubles: positions and inertial target
 *   g_out             one double (device)
 *   grad_out          n_verts x 3 doubles (device)
 *   stream            cudaStream_t (NULL = legacy default stream)
 * Work is enqueued on `stream`; the call returns without synchronising.
 *
 * The first call made with a given device current looks up the scratch's
 * device address on that device (once per device), so make that first call
 * before any stream capture.  Every call on a device shares the one scratch
 * array, which keeps the last call's contents; the call clears what must
 * start at zero itself.  Calls whose device work overlaps (different streams
 * or threads without ordering between them) race on the scratch and give
 * wrong results: order them on one stream.
 * Errors: HQN_ERR_ARG (sizes, null pointers, h, material), HQN_ERR_CUDA. */
#define HQN_STATIC_MAX_TETS  65536
#define HQN_STATIC_MAX_VERTS 262144
int hqn_energy_grad_static(int32_t n_verts, int32_t n_tets, const double *rest_pos,
                           const int32_t *tets, const uint8_t *clamped, const int32_t *vt_ptr,
                           const int32_t *vt_slot, const hqn_material *material, double h,
                           const double *x, const double *y, double *g_out, double *grad_out,
                           void *stream);

#ifdef __cplusplus
}
#endif
#endif /* HQN_H */
