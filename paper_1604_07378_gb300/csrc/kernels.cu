// Step kernels of the quasi-Newton implicit-Euler solver: predictor (Eq. PD),
// per-tet energy and corner gradients (Eq. valanis-landel), the line-search
// trials and Armijo tests (Alg. 1), the atomic-free vertex gather of grad g
// (Eq. PD), the history push and the two loops of Alg. 2.
//
// Every kernel runs over a batch of independent simulations.  Each block
// belongs to one simulation (the block tables map blocks to simulations) and
// stages that simulation's descriptor in shared memory.  Reductions are per
// simulation: each block publishes a partial, and the simulation's last block
// (an arrival ticket in its control block) sums its partials in a fixed order
// and takes its decisions.  The last simulation to decide sets the graph's
// conditional handles from every simulation's state.
#include "kernels.cuh"
#include "reduce.cuh"
#include "tetmath.cuh"

namespace hqn {

namespace {

template <typename R>
__device__ __forceinline__ void set_cond(unsigned long long h, unsigned int v) {
    if (h) cudaGraphSetConditional((cudaGraphConditionalHandle)h, v);
}

__device__ __forceinline__ int ring_slot(int head, int age, int m) {
    int s = head - age;
    return s < 0 ? s + m + 1 : s;
}

// The descriptor of the simulation that owns this block: the kernel
// parameter for a single simulation, else a copy in shared memory made by the
// block's threads (a block-uniform structure of a few hundred bytes that
// every thread reads).
template <typename R>
__device__ __forceinline__ const SimDesc<R> &stage_desc_batch(const SimDesc<R> *all, int sim) {
    __shared__ __align__(16) unsigned char raw[sizeof(SimDesc<R>)];
    static_assert(sizeof(SimDesc<R>) % 4 == 0, "descriptor size");
    const unsigned int *src = reinterpret_cast<const unsigned int *>(all + sim);
    unsigned int *dst = reinterpret_cast<unsigned int *>(raw);
    for (int k = threadIdx.x; k < (int)(sizeof(SimDesc<R>) / 4); k += blockDim.x) dst[k] = src[k];
    __syncthreads();
    return *reinterpret_cast<const SimDesc<R> *>(raw);
}

template <typename R>
__device__ __forceinline__ const SimDesc<R> &sim_desc(const DevSim<R> &s, const int *blk_sim) {
    if (s.nsims == 1) return s.desc0;
    return stage_desc_batch(s.desc, blk_sim[blockIdx.x]);
}

// Last block of a simulation, after its thread 0 wrote that simulation's
// decision: the last simulation to get here sets the graph condition `handle`
// to whether any simulation satisfies `pred` (called by every thread of the
// block).  The arrival counter re-arms itself.
template <typename R, typename Pred>
__device__ __forceinline__ void batch_condition(const DevSim<R> &s, int slot, unsigned long long handle, Pred pred) {
    if (s.nsims == 1) {  // thread 0 wrote the decision itself
        if (threadIdx.x == 0) set_cond<R>(handle, pred((const volatile Ctl *)s.desc0.ctl) ? 1u : 0u);
        return;
    }
    __shared__ int last_sim;
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        last_sim = atomicAdd(&s.batch_ticket[slot], 1u) == (unsigned)s.nsims - 1u;
        if (last_sim) __threadfence();  // acquire, ordered for the block by the barrier
    }
    __syncthreads();
    if (!last_sim) return;
    int any = 0;
    for (int k = threadIdx.x; k < s.nsims; k += blockDim.x) any |= pred((const volatile Ctl *)s.desc[k].ctl) ? 1 : 0;
    any = __syncthreads_or(any);
    if (threadIdx.x == 0) {
        s.batch_ticket[slot] = 0u;
        set_cond<R>(handle, any ? 1u : 0u);
    }
}

// Per-simulation grid reduction: the block's partials at
// part[k * stride + block]; true in every thread of the simulation's last block.
template <typename R, int NV>
__device__ __forceinline__ bool sim_arrive(const double (&v)[NV], double *part, int stride, int nblocks,
                                           unsigned int *ticket) {
    __shared__ bool last;
    if (threadIdx.x == 0) {
#pragma unroll
        for (int k = 0; k < NV; ++k) Part<R>::put(part + k * stride + blockIdx.x, v[k]);
        __threadfence();  // release: the partials before the ticket
        const unsigned int t = atomicAdd(ticket, 1u);
        last = (t == (unsigned)nblocks - 1u);
        if (last) __threadfence();  // acquire: every block's partials, ordered for the
                                    // whole block by the barrier below
    }
    __syncthreads();
    return last;
}

// ---------------------------------------------------------------- predictor

// y = 2 q_l - q_{l-1} + h^2 g on free vertices, y = q_l on clamped ones;
// x_1 = y.  The simulation's first block also clears its control block.
template <typename R>
__global__ void __launch_bounds__(VBS) k_predict(DevSim<R> s) {
    const SimDesc<R> &D = sim_desc(s, s.vblk_sim);
    const int i = (blockIdx.x - D.vb0) * VBS + threadIdx.x;
    if (i < D.c.n) {
        const int g = D.v0 + i;
        const V4<R> a = s.u_cur[g], b = s.u_prev[g];
        V4<R> yy = a;
        if (i < D.c.nf) {
            yy.x = R(2) * a.x - b.x + D.c.gx;
            yy.y = R(2) * a.y - b.y + D.c.gy;
            yy.z = R(2) * a.z - b.z + D.c.gz;
        }
        yy.w = R(0);
        s.y[g] = yy;
        s.xk[g] = yy;
        s.xt[g] = yy;
        if (D.c.cheb) s.xprev[g] = yy;  // x_0 read as x_1 (Alg. 3)
    }
    if (blockIdx.x == D.vb0 && threadIdx.x == 0) {
        Ctl *c = D.ctl;
        c->k = 0; c->trials = 0; c->count = 0; c->head = 0; c->stop = 0;
        c->status = HQN_OK; c->accepted = 0; c->nondescent = 0; c->alpha = 1.0; c->grad_ready = 0;
        c->active = 0;
        c->cheb_omega = 1.0;
    }
}

// ---------------------------------------------------------------- collision terms (Sec. 4.3)

// Calls f(gap, nx, ny, nz) for every collider that the vertex (rest position
// X, displacement u, displacement u_l at the start of the step) penetrates
// without moving away from it: gap = (x - t)^T n < 0, with t the projection of
// x = X + u on the collider and n the surface normal there.  The terms are
// w_v gap^2 (w_v = cscale m_v / h^2); with t and n frozen at the iteration's
// start, along x + alpha d the gap is gap + alpha d^T n.
template <typename R, typename F>
__device__ __forceinline__ void for_contacts(const StepConst<R> &c, const V4<R> &X, const V4<R> &u, const V4<R> &ul,
                                             F f) {
    for (int k = 0; k < c.ncol; ++k) {
        const ColDev<R> &q = c.col[k];
        const R rx = (X.x - q.px) + u.x, ry = (X.y - q.py) + u.y, rz = (X.z - q.pz) + u.z;
        R nx, ny, nz, gap;
        if (q.kind == HQN_COLLIDER_PLANE) {
            nx = q.nx; ny = q.ny; nz = q.nz;
            gap = rx * nx + ry * ny + rz * nz;
        } else if (q.kind == HQN_COLLIDER_TORUS) {
            // nearest point of the ring circle: the radial part of x - c
            // scaled to the ring radius; the surface lies `r` from it
            const R hgt = rx * q.nx + ry * q.ny + rz * q.nz;
            const R ax = rx - hgt * q.nx, ay = ry - hgt * q.ny, az = rz - hgt * q.nz;
            const R rho = sqrt_(ax * ax + ay * ay + az * az);
            if (!(rho > R(0))) continue;  // on the axis: no nearest ring point
            const R sc = q.ring / rho;
            const R vx = rx - sc * ax, vy = ry - sc * ay, vz = rz - sc * az;
            const R dist = sqrt_(vx * vx + vy * vy + vz * vz);
            if (!(dist > R(0))) continue;  // on the ring circle: no normal
            const R inv = R(1) / dist;
            nx = vx * inv; ny = vy * inv; nz = vz * inv;
            gap = dist - q.r;
        } else {
            const R dist = sqrt_(rx * rx + ry * ry + rz * rz);
            if (!(dist > R(0))) continue;  // at the centre: no normal
            const R inv = R(1) / dist;
            nx = rx * inv; ny = ry * inv; nz = rz * inv;
            gap = dist - q.r;
        }
        if (!(gap < R(0))) continue;
        const R vn = (u.x - ul.x) * nx + (u.y - ul.y) * ny + (u.z - ul.z) * nz;
        if (vn > R(0)) continue;
        f(gap, nx, ny, nz);
    }
}

// ---------------------------------------------------------------- inertia of a given x

// Block partial of the inertia term 1/(2h^2) sum m_v |x_t - y|^2 of Eq. PD at
// the caller-given point x_t (the start of a step, or an evaluation request),
// plus the collision terms active there.  The sum runs over the free
// vertices: clamped ones are eliminated (their positions are prescribed), so
// a caller's x != y on a clamped row adds nothing.
template <typename R>
__global__ void __launch_bounds__(VBS) k_inertia(DevSim<R> s) {
    using A = ExactAcc<R>;
    const SimDesc<R> &D = sim_desc(s, s.vblk_sim);
    const int i = (blockIdx.x - D.vb0) * VBS + threadIdx.x;
    typename A::T e[1] = {A::zero()};
    if (i < D.c.nf) {
        const int g = D.v0 + i;
        const V4<R> x = s.xt[g], yy = s.y[g];
        const R dx = x.x - yy.x, dy = x.y - yy.y, dz = x.z - yy.z;
        e[0] = A::add(e[0], R(0.5) * s.mh2[g] * (dx * dx + dy * dy + dz * dz));
        if (D.c.ncol > 0) {
            const R w = D.c.cscale * s.mh2[g];
            for_contacts(D.c, s.rest[g], x, s.u_cur[g], [&](R gap, R, R, R) { e[0] = A::add(e[0], w * gap * gap); });
        }
    }
    double tot[1];
    block_sum_exact<VBS, 1, R>(e, tot);
    if (threadIdx.x == 0) Part<R>::put(s.part_in + blockIdx.x, tot[0]);
}

// x_k + alpha d, rounded the same way wherever the accepted point is formed.
template <typename R>
__device__ __forceinline__ V4<R> step_point(const V4<R> &a, const V4<R> &b, R al) {
    V4<R> o;
    o.x = fma_(al, b.x, a.x);
    o.y = fma_(al, b.y, a.y);
    o.z = fma_(al, b.z, a.z);
    o.w = R(0);
    return o;
}

template <typename R>
__device__ __forceinline__ void load_dm(const DevSim<R> &s, int t, R Di[9]) {
#pragma unroll
    for (int k = 0; k < 9; ++k) Di[k] = s.dminv[(size_t)k * s.Tn + t];
}

template <typename R>
__device__ __forceinline__ void edge_diffs(const V4<R> &x0, const V4<R> &x1, const V4<R> &x2, const V4<R> &x3,
                                           R du[3][3]) {
    du[0][0] = x1.x - x0.x; du[0][1] = x1.y - x0.y; du[0][2] = x1.z - x0.z;
    du[1][0] = x2.x - x0.x; du[1][1] = x2.y - x0.y; du[1][2] = x2.z - x0.z;
    du[2][0] = x3.x - x0.x; du[2][1] = x3.y - x0.y; du[2][2] = x3.z - x0.z;
}

// Sum of the simulation's per-block partials part[b], b in [b0, b0 + nb)
// (stored by Part<R>::put), by its last block in a fixed order; result valid
// in thread 0.
template <typename R, int BS>
__device__ __forceinline__ double sum_block_range(const double *part, int b0, int nb) {
    using P = Part<R>;
    __shared__ typename P::T sh[BS / 32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    typename P::T v = part_warp_sum<R>(part_strided_sum<R>(part + b0, threadIdx.x, nb, BS));
    if (lane == 0) sh[warp] = v;
    __syncthreads();
    double out = 0.0;
    if (warp == 0) {
        typename P::T t = lane < BS / 32 ? sh[lane] : P::zero();
        out = P::to_double(part_warp_sum<R>(t));
    }
    __syncthreads();
    return out;
}

// ---------------------------------------------------------------- tet kernel

// One thread per tet: the four corner gradients of V Psi, written to their
// places in the vertex-ordered corner array.
//   TET_INIT / TET_EVAL: at the point x_t, with the energy reduced too (the
//     simulation's last block, fixed order, plus the inertia partials):
//     TET_INIT sets g(x_1), TET_EVAL reports g.
//   TET_TRIAL1: the first trial of Alg. 1's line search, alpha = 1, at
//     x_k + d; the last block adds the inertia term along the ray and runs the
//     Armijo test.  Accepted: the corners are the gradient of x_{k+1} and the
//     simulation skips the line-search loop.  Rejected: the loop continues at
//     alpha = backtrack.
//   TET_GRAD: at the accepted point x_k + alpha d, corners only; runs after
//     each line-search pass and does nothing for a simulation that has not
//     accepted yet, whose TET_TRIAL1 already left the corners, or that stopped.
template <typename R>
__global__ void __launch_bounds__(TBS, 8) k_tet(DevSim<R> s, int mode, CondHandles h) {
    using A = ExactAcc<R>;
    const SimDesc<R> &D = sim_desc(s, s.tblk_sim);
    Ctl *c = D.ctl;
    const bool grad_mode = mode == TET_GRAD;
    const bool ray_mode = mode == TET_GRAD || mode == TET_TRIAL1;
    const bool inactive = ray_mode && !c->active;
    if (grad_mode && (inactive || c->stop || c->grad_ready || !c->accepted)) return;
    const R al = grad_mode ? (R)c->alpha : R(1);
    const int tl = (blockIdx.x - D.tb0) * TBS + threadIdx.x;
    typename A::T e[1] = {A::zero()};
    if (tl < D.c.T && !inactive) {
        const int t = D.t0 + tl;
        const int4 v = s.tets[t];
        V4<R> x0, x1, x2, x3;
        if (ray_mode) {
            x0 = step_point(s.xk[v.x], s.d[v.x], al);
            x1 = step_point(s.xk[v.y], s.d[v.y], al);
            x2 = step_point(s.xk[v.z], s.d[v.z], al);
            x3 = step_point(s.xk[v.w], s.d[v.w], al);
        } else {
            x0 = s.xt[v.x]; x1 = s.xt[v.y]; x2 = s.xt[v.z]; x3 = s.xt[v.w];
        }
        R du[3][3], Di[9], G[3][3];
        edge_diffs(x0, x1, x2, x3, du);
        load_dm(s, t, Di);
        def_grad(du, Di, G);
        const R vol = s.vol[t];
        R g[4][3];
        // the tet's material: the simulation's only one, or its own from the
        // mesh's table (one branch per tet, uniform for one-material meshes)
        auto eval = [&](const MatDev<R> &M) {
            tet_grad(M, G, Di, vol, g);
            if (!grad_mode) e[0] = A::add(e[0], vol * tet_psi(M, G));
        };
        if (D.n_mats > 1) eval(D.mats[s.tmat[t]]);
        else eval(D.mat);
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            V4<R> o;
            o.x = g[k][0]; o.y = g[k][1]; o.z = g[k][2]; o.w = R(0);
            s.corner[s.corner_pos[(size_t)k * s.Tn + t]] = o;
        }
    }
    if (grad_mode) return;
    double tot[1];
    block_sum_exact<TBS, 1, R>(e, tot);
    if (!sim_arrive<R, 1>(tot, s.part_el, 0, D.ntb, &c->ticket[TK_TET])) return;
    const double el = sum_block_range<R, TBS>(s.part_el, D.tb0, D.ntb);
    if (mode == TET_TRIAL1) {
        if (threadIdx.x == 0) {
            c->ticket[TK_TET] = 0u;
            if (c->active) {
                // g(x_k + d) - g(x_k) = E(x_k + d) - E(x_k) + I(1) - I(0) with the
                // inertia term I(alpha) = a0 + a1 alpha + a2 alpha^2 along the ray
                const double dI = c->ls_a[1] + c->ls_a[2];
                c->passes_total += 1;
                c->trials = 1;
                if ((el - c->e_k) + dI <= D.c.gamma * c->gd) {
                    c->accepted = 1;
                    c->grad_ready = 1;
                    c->alpha = 1.0;
                    c->e_trial = el;
                    c->g_trial = el + c->ls_a[0] + dI;
                } else {
                    c->accepted = 0;
                    c->grad_ready = 0;
                    c->alpha = D.c.backtrack;
                    if (D.c.ls_max <= 1) {
                        c->stop = 1;
                        c->status = HQN_WARN_LS_EXHAUSTED;
                    }
                }
            }
        }
        batch_condition(s, BT_LS, h.ls,
                        [](const volatile Ctl *x) { return x->active && !x->accepted && !x->stop; });
        return;
    }
    const double in = sum_block_range<R, TBS>(s.part_in, D.vb0, D.nvb);
    if (threadIdx.x != 0) return;
    c->ticket[TK_TET] = 0u;
    const double g = el + in;
    c->g_trial = g;
    if (mode == TET_INIT) {
        c->g_k = g;
        c->e_k = el;
        c->g0 = g;
        c->accepted = 1;
    }
}

// ---------------------------------------------------------------- line search

// One pass of the backtracking line search of Alg. 1 that evaluates K trial
// step lengths at once: alpha_j = alpha * backtrack^j, j < K.  Each thread
// forms G_k = Du_k Dm^{-1} and G_d = Dd Dm^{-1} once and the energy V Psi of
// G_k + alpha_j G_d for every j (no singular vectors: PsiRay).  The last
// block adds the inertia term, a quadratic in alpha whose coefficients were
// formed with the direction, and runs the Armijo tests in the order of Alg. 1
// (written on differences, g(x_k + a d) - g(x_k) <= gamma a tr(grad^T d), so
// the inertia term's constant part never enters a comparison): the first
// alpha_j that passes is accepted (the same choice as testing them one at a
// time).  Otherwise the next pass continues from alpha_K, until ls_max
// trials in all.  Simulations that are not searching skip the pass.
template <typename R, int K>
__global__ void __launch_bounds__(TBS) k_ls(DevSim<R> s, CondHandles h) {
    using A = ExactAcc<R>;
    const SimDesc<R> &D = sim_desc(s, s.tblk_sim);
    Ctl *ctl = D.ctl;
    const bool searching = ctl->active && !ctl->accepted && !ctl->stop;
    const double a0 = ctl->alpha;
    const double bt = D.c.backtrack;
    const int tl = (blockIdx.x - D.tb0) * TBS + threadIdx.x;
    typename A::T e[K];
#pragma unroll
    for (int j = 0; j < K; ++j) e[j] = A::zero();
    if (tl < D.c.T && searching) {
        const int t = D.t0 + tl;
        const int4 v = s.tets[t];
        R Duk[3][3], Dd[3][3], Di[9], Gk[3][3], Gd[3][3];
        edge_diffs(s.xk[v.x], s.xk[v.y], s.xk[v.z], s.xk[v.w], Duk);
        edge_diffs(s.d[v.x], s.d[v.y], s.d[v.z], s.d[v.w], Dd);
        load_dm(s, t, Di);
        def_grad(Duk, Di, Gk);
        def_grad(Dd, Di, Gd);
        const R vol = s.vol[t];
        auto eval = [&](const MatDev<R> &M) {
            PsiRay<R> ray;
            psi_ray_setup(M, Gk, Gd, ray);
            double a = a0;
#pragma unroll
            for (int j = 0; j < K; ++j) {
                e[j] = A::add(e[j], vol * psi_ray_eval(M, ray, (R)a));
                a *= bt;
            }
        };
        if (D.n_mats > 1) eval(D.mats[s.tmat[t]]);
        else eval(D.mat);
    }
    double tot[K];
    block_sum_exact<TBS, K, R>(e, tot);
    if (!sim_arrive<R, K>(tot, s.part_ls, s.ntb, D.ntb, &ctl->ticket[TK_LS])) return;
    {
        // the simulation's partials, one warp per trial
        __shared__ double sh[K];
        warp_value_sums<R, K, TBS / 32>(s.part_ls + D.tb0, (size_t)s.ntb, D.ntb, sh);
        __syncthreads();
#pragma unroll
        for (int j = 0; j < K; ++j) tot[j] = sh[j];
    }
    if (threadIdx.x == 0) {
        ctl->ticket[TK_LS] = 0u;
        if (searching) {
            double a = a0;
            int tr = ctl->trials;
            ctl->passes_total += 1;
            const double ek = ctl->e_k, slope = D.c.gamma * ctl->gd;
            const double c0 = ctl->ls_a[0], c1 = ctl->ls_a[1], c2 = ctl->ls_a[2];
            bool done = false;
#pragma unroll
            for (int j = 0; j < K; ++j) {
                if (done) break;
                if (tr >= D.c.ls_max) break;
                tr += 1;
                // Armijo on differences: E(x_k + a d) - E(x_k) + I(a) - I(0) <= gamma a gd
                const double dI = a * (c1 + a * c2);
                if ((tot[j] - ek) + dI <= slope * a) {
                    ctl->accepted = 1;
                    ctl->alpha = a;
                    ctl->e_trial = tot[j];
                    ctl->g_trial = tot[j] + c0 + dI;
                    done = true;
                    break;
                }
                a *= bt;
            }
            ctl->trials = tr;
            if (!done) {
                ctl->alpha = a;
                if (tr >= D.c.ls_max) {
                    ctl->accepted = 0;
                    ctl->stop = 1;
                    ctl->status = HQN_WARN_LS_EXHAUSTED;
                }
            }
        }
    }
    batch_condition(s, BT_LS, h.ls, [](const volatile Ctl *x) { return x->active && !x->accepted && !x->stop; });
}

// ---------------------------------------------------------------- Alg. 2 in dot-product form
//
// The two loops of Alg. 2 touch the vectors only through inner products with
// the history pairs.  With q_p the value of q when pair p (age p, 0 = newest)
// is reached in the first loop, and r_p the value of r in the second loop,
//   s_p^T q_p = -s_p^T g - sum_{p' < p} zeta_p' (s_p^T t_p'),
//   t_p^T r_p =  t_p^T r0 + sum_{p' > p} c_p' (t_p^T s_p'),   c_p = zeta_p - eta_p,
// where r0 = A0^{-1} q_final, q_final = -g - sum_p zeta_p t_p and
// d = r0 + sum_p c_p s_p.  So the recursion runs on scalars once the Gram
// matrix s_a^T t_b of the ring slots and the products s_a^T g and t_a^T r0 are
// known: the gather that pushes a pair forms its row and column of the Gram
// matrix and s_a^T g for the new gradient, the vector passes are q_final, the
// t_a^T r0 products and d.  The scalars are float64.

template <typename R>
__device__ __forceinline__ double dotv(const V4<R> &a, const V4<R> &b) {
    return (double)a.x * b.x + (double)a.y * b.y + (double)a.z * b.z;
}

template <typename R>
__device__ __forceinline__ R dotr(const V4<R> &a, const V4<R> &b) {
    return a.x * b.x + a.y * b.y + a.z * b.z;
}

// The history scalars the recursions need, staged in shared memory by the
// last block of a simulation: the control block lives in global memory, and a
// recursion run on it directly would pay a memory round trip per step.
constexpr int MH = kShortHist + 1;
struct HistSmem {
    double gram[MH][MH];  // s_a^T t_b by ring slots
    double rho[MH], rinv[MH], sg[MH], tr0[MH], zeta[MH], coef[MH];  // rinv = 1 / rho
    int count, head;
};

// All threads: load the Gram matrix (rows and columns <= m), rho, zeta,
// count and head into shared memory.
__device__ __forceinline__ void hist_load(const Ctl *c, HistSmem &h, int m) {
    const int m1 = m + 1;
    for (int e = threadIdx.x; e < m1 * m1; e += blockDim.x) h.gram[e / m1][e % m1] = c->gram[e / m1][e % m1];
    for (int a = threadIdx.x; a < m1; a += blockDim.x) {
        h.rho[a] = c->rho[a];
        h.rinv[a] = 1.0 / c->rho[a];  // the recursions multiply (one division per slot, in parallel)
        h.zeta[a] = c->zeta[a];
    }
    if (threadIdx.x == 0) {
        h.count = c->count;
        h.head = c->head;
    }
    __syncthreads();
}

// First loop on scalars: zeta_p for every held pair, newest first.
__device__ __forceinline__ void zeta_recursion(HistSmem &h, int m) {
    for (int p = 0; p < h.count; ++p) {
        const int sl = ring_slot(h.head, p, m);
        double sq = -h.sg[sl];
        for (int pp = 0; pp < p; ++pp) sq -= h.zeta[pp] * h.gram[sl][ring_slot(h.head, pp, m)];
        h.zeta[p] = sq * h.rinv[sl];
    }
}

// Second loop on scalars: c_p = zeta_p - eta_p, oldest first.
__device__ __forceinline__ void coef_recursion(HistSmem &h, int m) {
    for (int p = h.count - 1; p >= 0; --p) {
        const int sl = ring_slot(h.head, p, m);
        double tr = h.tr0[sl];
        for (int pp = p + 1; pp < h.count; ++pp) tr += h.coef[pp] * h.gram[ring_slot(h.head, pp, m)][sl];
        h.coef[p] = h.zeta[p] - tr * h.rinv[sl];
    }
}

// ---------------------------------------------------------------- gather

// One thread per free vertex: grad g = m (x - y)/h^2 + sum of the vertex's
// corner gradients in a fixed (ascending tet) order -- no atomics.  In G_ITER
// mode the accepted trial becomes x_{k+1}: the pair s = x_{k+1} - x_k,
// t = grad_{k+1} - grad_k goes to the free ring slot w, and the block partials
// of rho = tr(t^T s) (float64-accurate terms) and of |s|^2, |t|^2, s_a^T t_w,
// s_w^T t_a and s_a^T grad_{k+1} for every ring slot a (R-precision terms and
// block sums, float64 beyond) are reduced.  The simulation's last block keeps
// the pair if rho > 1e-12 |s| |t|, updates the Gram matrix, runs the first
// loop of Alg. 2 on scalars and ends the simulation's iterations when its
// count is reached or its line search gave up.  The collision terms active
// at the gathered point (Sec. 4.3) add 2 w_v gap n to its gradient.
// MP1 = 0: a long window (m > kShortHist): the pair is pushed and kept or
// dropped here, its slot products and the first loop follow in
// launch_long_hist.
template <typename R, int MP1>
__global__ void __launch_bounds__(VBS) k_gather(DevSim<R> s, int mode, CondHandles h) {
    constexpr bool LONG = MP1 == 0;
    constexpr int MPA = LONG ? 1 : MP1;  // register arrays
    const SimDesc<R> &D = sim_desc(s, s.vblk_sim);
    Ctl *ctl = D.ctl;
    const int m = s.m;
    const bool iter = mode == G_ITER;
    const bool act = !iter || ctl->active;
    const bool stop = iter && ctl->stop;
    const bool push = iter && m > 0 && act && !stop;
    const int w = push ? (ctl->head + 1) % (m + 1) : 0;
    const R al = iter ? (R)ctl->alpha : R(0);
    constexpr int NG = 2 + 3 * MP1;  // |s|^2, |t|^2, then three products per slot
    constexpr int ND = 1 + NG;
    using A = ExactAcc<R>;
    typename A::T dd[1] = {A::zero()};
    R dr[NG];
#pragma unroll
    for (int k = 0; k < NG; ++k) dr[k] = R(0);
    const int i = (blockIdx.x - D.vb0) * VBS + threadIdx.x;
    if (act && !stop && i < D.c.nf) {
        const int gi = D.v0 + i;
        // every load before any store: the vertex's corner range, its vectors
        // and (history push) the ring slots; the ring slot being replaced is
        // loaded too and not used
        const int b = s.vt_ptr[gi], e = s.vt_ptr[gi + 1];
        const V4<R> xk = iter ? s.xk[gi] : s.xt[gi];
        V4<R> dv;
        dv.x = dv.y = dv.z = dv.w = R(0);
        if (iter) dv = s.d[gi];
        const V4<R> yy = s.y[gi];
        const R mh = s.mh2[gi];
        V4<R> go = dv, Xr = dv, ul = dv;
        if (D.c.ncol > 0) {
            Xr = s.rest[gi];
            ul = s.u_cur[gi];
        }
        V4<R> Sa[MPA], Ta[MPA];
        V4<R> *S = s.S + D.ring0, *Tt = s.Tt + D.ring0;
        const size_t n = (size_t)D.c.n;
        if (push) {
            go = s.gk[gi];
#pragma unroll
            for (int a = 0; a < MP1; ++a)
                if (a <= m) {
                    Sa[a] = S[(size_t)a * n + i];
                    Ta[a] = Tt[(size_t)a * n + i];
                }
        }
        R gx = R(0), gy = R(0), gz = R(0);
#pragma unroll 8
        for (int k = b; k < e; ++k) {
            const V4<R> cg = s.corner[k];
            gx += cg.x; gy += cg.y; gz += cg.z;
        }
        const V4<R> x = iter ? step_point(xk, dv, al) : xk;
        V4<R> gn;
        gn.x = gx + mh * (x.x - yy.x);
        gn.y = gy + mh * (x.y - yy.y);
        gn.z = gz + mh * (x.z - yy.z);
        gn.w = R(0);
        if (D.c.ncol > 0) {
            const R w2 = R(2) * D.c.cscale * mh;
            for_contacts(D.c, Xr, x, ul, [&](R gap, R nx, R ny, R nz) {
                gn.x += w2 * gap * nx; gn.y += w2 * gap * ny; gn.z += w2 * gap * nz;
            });
        }
        if (iter) {
            if (push) {
                V4<R> sv, tv;
                sv.x = x.x - xk.x; sv.y = x.y - xk.y; sv.z = x.z - xk.z; sv.w = R(0);
                tv.x = gn.x - go.x; tv.y = gn.y - go.y; tv.z = gn.z - go.z; tv.w = R(0);
                S[(size_t)w * n + i] = sv;
                Tt[(size_t)w * n + i] = tv;
                dd[0] = A::add_prod(A::add_prod(A::add_prod(dd[0], tv.x, sv.x), tv.y, sv.y), tv.z, sv.z);
                dr[0] = dotr(sv, sv);
                dr[1] = dotr(tv, tv);
#pragma unroll
                for (int a = 0; a < MP1; ++a) {
                    if (a > m) break;
                    const V4<R> sa = a == w ? sv : Sa[a];
                    const V4<R> ta = a == w ? tv : Ta[a];
                    dr[2 + a] = dotr(sa, tv);
                    dr[2 + MP1 + a] = dotr(sv, ta);
                    dr[2 + 2 * MP1 + a] = dotr(sa, gn);
                }
            }
            if (D.c.cheb) s.xprev[gi] = xk;  // x_{k-1} of the next direction (Alg. 3)
            s.xk[gi] = x;
        }
        s.gk[gi] = gn;
    }
    if (mode == G_EVAL) return;
    double dots[ND];
    {
        double mixed[NG], rho[1];
        block_sum_exact<VBS, 1, R>(dd, rho);
        block_sum_r<VBS, NG, R>(dr, mixed);
        dots[0] = rho[0];
#pragma unroll
        for (int k = 0; k < NG; ++k) dots[1 + k] = mixed[k];
    }
    if (!sim_arrive<R, ND>(dots, s.part_g, s.nvb, D.nvb, &ctl->ticket[TK_GATHER])) return;
    __shared__ int keep;
    if (push) {
        {
            // the simulation's partials, one warp per value
            __shared__ double sh[ND];
            warp_value_sums<R, ND, VBS / 32>(s.part_g + D.vb0, (size_t)s.nvb, D.nvb, sh);
            __syncthreads();
#pragma unroll
            for (int k = 0; k < ND; ++k) dots[k] = sh[k];
        }
        // dots: rho, |s|^2, |t|^2, s_a^T t_w, s_w^T t_a, s_a^T grad
        if constexpr (LONG) {
            if (threadIdx.x == 0) {
                keep = dots[0] > 1e-12 * sqrt(dots[1] * dots[2]);
                ctl->hist_w = w;
                ctl->hist_keep = keep;
                if (keep) {
                    LongHist(D.lh, m).rho[w] = dots[0];
                    ctl->head = w;
                    ctl->count = ctl->count < m ? ctl->count + 1 : m;
                }
            }
        } else {
        __shared__ HistSmem hs;
        hist_load(ctl, hs, m);
        if (threadIdx.x == 0) {
            keep = dots[0] > 1e-12 * sqrt(dots[1] * dots[2]);
            if (keep) {
                hs.head = w;
                hs.rho[w] = dots[0];
                hs.rinv[w] = 1.0 / dots[0];
                hs.count = hs.count < m ? hs.count + 1 : m;
#pragma unroll
                for (int a = 0; a < MP1; ++a)
                    if (a <= m) {
                        hs.gram[a][w] = dots[3 + a];
                        hs.gram[w][a] = dots[3 + MP1 + a];
                    }
            }
#pragma unroll
            for (int a = 0; a < MP1; ++a)
                if (a <= m) hs.sg[a] = dots[3 + 2 * MP1 + a];
            zeta_recursion(hs, m);
        }
        __syncthreads();
        for (int a = threadIdx.x; a <= m; a += VBS) {
            ctl->zeta[a] = hs.zeta[a];
            if (keep) {
                ctl->gram[a][w] = hs.gram[a][w];
                ctl->gram[w][a] = hs.gram[w][a];
            }
        }
        if (threadIdx.x == 0 && keep) {
            ctl->rho[w] = hs.rho[w];
            ctl->head = hs.head;
            ctl->count = hs.count;
        }
        }
    }
    if (threadIdx.x == 0) {
        ctl->ticket[TK_GATHER] = 0u;
        if (mode == G_INIT) {
            ctl->k = 1;
            ctl->count = 0;
            ctl->head = 0;
            ctl->g_k = ctl->g_trial;
            ctl->active = D.c.iters > 0 ? 1 : 0;
        } else if (act) {
            const int k = ctl->k;
            const int kk = k - 1 < HQN_MAX_ITERS ? k - 1 : HQN_MAX_ITERS - 1;
            ctl->iter_trials[kk] = ctl->trials;
            ctl->trials_total += ctl->trials;
            ctl->iters_total += 1;
            if (stop) {
                ctl->iter_g[kk] = ctl->g_k;
                ctl->active = 0;
            } else {
                ctl->g_k = ctl->g_trial;
                ctl->e_k = ctl->e_trial;
                ctl->iter_g[kk] = ctl->g_trial;
                ctl->k = k + 1;
                ctl->active = (k + 1 <= D.c.iters) ? 1 : 0;
            }
        }
    }
    batch_condition(s, BT_IT, h.it, [](const volatile Ctl *x) { return x->active != 0; });
}

// q = -grad - sum_p zeta_p t_p (the first loop's result).
template <typename R, int MP1>
__global__ void __launch_bounds__(VBS) k_q(DevSim<R> s) {
    const SimDesc<R> &D = sim_desc(s, s.vblk_sim);
    const Ctl *ctl = D.ctl;
    const int i = (blockIdx.x - D.vb0) * VBS + threadIdx.x;
    if (i >= D.c.nf || !ctl->active) return;
    const int count = ctl->count, head = ctl->head, m = s.m;
    const int gi = D.v0 + i;
    // every load first (history slots unrolled over the ring), then the sum in
    // the order p = 0, 1, ...
    const V4<R> g = s.gk[gi];
    const V4<R> *Tt = s.Tt + D.ring0;
    V4<R> q;
    q.x = -g.x; q.y = -g.y; q.z = -g.z; q.w = R(0);
    if constexpr (MP1 == 0) {  // a long window: the slots streamed one by one
        const double *zeta = LongHist(D.lh, m).zeta;
        for (int p = 0; p < count; ++p) {
            const R zp = (R)zeta[p];
            const V4<R> tp = Tt[(size_t)ring_slot(head, p, m) * D.c.n + i];
            q.x -= zp * tp.x; q.y -= zp * tp.y; q.z -= zp * tp.z;
        }
    } else {
        R z[MP1];
        V4<R> t[MP1];
#pragma unroll
        for (int p = 0; p < MP1; ++p)
            if (p < count) {
                z[p] = (R)ctl->zeta[p];
                t[p] = Tt[(size_t)ring_slot(head, p, m) * D.c.n + i];
            }
#pragma unroll
        for (int p = 0; p < MP1; ++p)
            if (p < count) {
                q.x -= z[p] * t[p].x; q.y -= z[p] * t[p].y; q.z -= z[p] * t[p].z;
            }
    }
    s.q[gi] = q;
}

// t_a^T r0 for every ring slot a (r0 = A0^{-1} q, held in d); the last block
// runs the second loop of Alg. 2 on scalars: c_p = zeta_p - eta_p, oldest first.
template <typename R, int MP1>
__global__ void __launch_bounds__(VBS) k_r0_dots(DevSim<R> s) {
    const SimDesc<R> &D = sim_desc(s, s.vblk_sim);
    Ctl *ctl = D.ctl;
    const int count = ctl->count, m = s.m;
    if (count == 0 || !ctl->active) return;  // the whole simulation skips, tickets untouched
    R dr[MP1];
#pragma unroll
    for (int a = 0; a < MP1; ++a) dr[a] = R(0);
    const int i = (blockIdx.x - D.vb0) * VBS + threadIdx.x;
    if (i < D.c.nf) {
        const V4<R> r = s.d[D.v0 + i];
        const V4<R> *Tt = s.Tt + D.ring0;
#pragma unroll
        for (int a = 0; a < MP1; ++a) {
            if (a > m) break;
            dr[a] = dotr(Tt[(size_t)a * D.c.n + i], r);
        }
    }
    double dots[MP1];
    block_sum_r<VBS, MP1, R>(dr, dots);
    if (!sim_arrive<R, MP1>(dots, s.part_v, s.nvb, D.nvb, &ctl->ticket[TK_VEC])) return;
    {
        __shared__ double sh[MP1];
        warp_value_sums<R, MP1, VBS / 32>(s.part_v + D.vb0, (size_t)s.nvb, D.nvb, sh);
        __syncthreads();
#pragma unroll
        for (int k = 0; k < MP1; ++k) dots[k] = sh[k];
    }
    __shared__ HistSmem hs;
    hist_load(ctl, hs, m);
    if (threadIdx.x == 0) {
        ctl->ticket[TK_VEC] = 0u;
#pragma unroll
        for (int a = 0; a < MP1; ++a)
            if (a <= m) hs.tr0[a] = dots[a];
        coef_recursion(hs, m);
    }
    __syncthreads();
    for (int p = threadIdx.x; p < count; p += VBS) ctl->coef[p] = hs.coef[p];
}

// omega_{k+1} of Alg. 3 from omega_k (k: the 1-based index of x_k).
template <typename R>
__device__ __forceinline__ double cheb_omega_next(const StepConst<R> &c, int k, double omega_k) {
    if (k < c.cheb_S) return 1.0;
    if (k == c.cheb_S) return 2.0 / (2.0 - c.cheb_rho2);
    return 4.0 / (4.0 - c.cheb_rho2 * omega_k);
}

// d = r0 + sum_p c_p s_p (or Alg. 3's Chebyshev direction); then gd = tr(grad_k^T d) -- with history and
// gd >= 0 the direction is not a descent direction: flag it so the history is
// dropped (h.nd: any simulation flagged) -- and the coefficients of the
// inertia term along the ray x_k + alpha d:
// 1/(2h^2) sum m |x_k + alpha d - y|^2 = a0 + a1 alpha + a2 alpha^2, with the
// iteration's collision terms sum w (gap + alpha d^T n)^2 added to them.
template <typename R, int MP1>
__global__ void __launch_bounds__(VBS) k_dir_final(DevSim<R> s, CondHandles h, int set_nd) {
    const SimDesc<R> &D = sim_desc(s, s.vblk_sim);
    Ctl *ctl = D.ctl;
    const bool act = ctl->active;
    const int i = (blockIdx.x - D.vb0) * VBS + threadIdx.x;
    R d4[4] = {R(0), R(0), R(0), R(0)};
    if (act && i < D.c.nf) {
        const int gi = D.v0 + i;
        const int count = ctl->count, head = ctl->head, m = s.m;
        const V4<R> *S = s.S + D.ring0;
        // every load before the store of d (history slots unrolled over the
        // ring); the sum runs in the order p = 0, 1, ...
        V4<R> dd = s.d[gi];
        const V4<R> g = s.gk[gi], x = s.xk[gi], yy = s.y[gi];
        const R mh = s.mh2[gi];
        if constexpr (MP1 == 0) {  // a long window: the slots streamed one by one
            const double *coef = LongHist(D.lh, m).coef;
            for (int p = 0; p < count; ++p) {
                const R cp = (R)coef[p];
                const V4<R> sp = S[(size_t)ring_slot(head, p, m) * D.c.n + i];
                dd.x += cp * sp.x; dd.y += cp * sp.y; dd.z += cp * sp.z;
            }
        } else {
            R c[MP1];
            V4<R> sv[MP1];
#pragma unroll
            for (int p = 0; p < MP1; ++p)
                if (p < count) {
                    c[p] = (R)ctl->coef[p];
                    sv[p] = S[(size_t)ring_slot(head, p, m) * D.c.n + i];
                }
#pragma unroll
            for (int p = 0; p < MP1; ++p)
                if (p < count) {
                    dd.x += c[p] * sv[p].x; dd.y += c[p] * sv[p].y; dd.z += c[p] * sv[p].z;
                }
        }
        V4<R> Xr = dd, ul = dd;
        if (D.c.ncol > 0) {
            Xr = s.rest[gi];
            ul = s.u_cur[gi];
        }
        if (D.c.cheb) {
            // Alg. 3: d = omega (x_k + q - x_{k-1}) + x_{k-1} - x_k with q = r0 (no history)
            const R om = (R)cheb_omega_next(D.c, ctl->k, ctl->cheb_omega);
            const V4<R> xp = s.xprev[gi];
            dd.x = om * ((x.x + dd.x) - xp.x) + xp.x - x.x;
            dd.y = om * ((x.y + dd.y) - xp.y) + xp.y - x.y;
            dd.z = om * ((x.z + dd.z) - xp.z) + xp.z - x.z;
        }
        if (count > 0 || D.c.cheb) s.d[gi] = dd;
        const R rx = x.x - yy.x, ry = x.y - yy.y, rz = x.z - yy.z;
        d4[0] = dotr(g, dd);
        d4[1] = R(0.5) * mh * (rx * rx + ry * ry + rz * rz);
        d4[2] = mh * (rx * dd.x + ry * dd.y + rz * dd.z);
        d4[3] = R(0.5) * mh * dotr(dd, dd);
        if (D.c.ncol > 0) {
            // the collision terms of this iteration (at x_k) along the ray
            const R w = D.c.cscale * mh;
            for_contacts(D.c, Xr, x, ul, [&](R gap, R nx, R ny, R nz) {
                const R dn = dd.x * nx + dd.y * ny + dd.z * nz;
                d4[1] += w * gap * gap;
                d4[2] += R(2) * w * gap * dn;
                d4[3] += w * dn * dn;
            });
        }
    }
    double tot[4];
    block_sum_r<VBS, 4, R>(d4, tot);
    if (!sim_arrive<R, 4>(tot, s.part_v, s.nvb, D.nvb, &ctl->ticket[TK_VEC])) return;
    {
        __shared__ double sh[4];
        warp_value_sums<R, 4, VBS / 32>(s.part_v + D.vb0, (size_t)s.nvb, D.nvb, sh);
        __syncthreads();
#pragma unroll
        for (int k = 0; k < 4; ++k) tot[k] = sh[k];
    }
    if (threadIdx.x == 0) {
        ctl->ticket[TK_VEC] = 0u;
        if (act && D.c.cheb) ctl->cheb_omega = cheb_omega_next(D.c, ctl->k, ctl->cheb_omega);
        if (act) {
            ctl->gd = tot[0];
            ctl->ls_a[0] = tot[1];
            ctl->ls_a[1] = tot[2];
            ctl->ls_a[2] = tot[3];
            ctl->nondescent = (tot[0] >= 0.0 && ctl->count > 0) ? 1 : 0;
        } else {
            ctl->nondescent = 0;
        }
    }
    if (set_nd) batch_condition(s, BT_ND, h.nd, [](const volatile Ctl *x) { return x->nondescent != 0; });
}

// ---------------------------------------------------------------- Jacobi-PCG in lieu of A0^{-1}
//
// The paper's comparison with iterative solvers (Sec. 8): a fixed number of
// Jacobi-preconditioned conjugate-gradient iterations from zero replaces the
// factorised solve.  A0 = M/h^2 + L is applied matrix-free: L p is the
// gradient of 1/2 sum_t V_t k |G_t p|^2, i.e. per tet the corner gradients of
// the linear stress P = V k G(p) (G(p) = [p1 - p0, p2 - p0, p3 - p0] Dm^{-1}),
// summed per vertex through the vertex-ordered corner array.  The three
// coordinate columns form one vector: one alpha and one beta per iteration,
// from fixed-order float64 grid sums.  Each iteration is three launches:
//   tet:    corners of L p, p = z + beta p_old formed on the fly;
//   gather: p (stored), A0 p, p^T A0 p -> alpha = r^T z / p^T A0 p;
//   update: x += alpha p, r -= alpha A0 p, z = D^{-1} r, r^T z -> beta.

template <typename R>
__device__ __forceinline__ V4<R> pcg_p(const DevSim<R> &s, int g, R beta) {
    const V4<R> z = s.pcg_z[g], p = s.pcg_p[g];
    V4<R> o;
    o.x = z.x + beta * p.x; o.y = z.y + beta * p.y; o.z = z.z + beta * p.z; o.w = R(0);
    return o;
}

// x = 0 (out), r = q, z = D^{-1} q, p_old = 0, rz = r^T z, beta = 0.
template <typename R>
__global__ void __launch_bounds__(VBS) k_pcg_init(DevSim<R> s, const V4<R> *q, V4<R> *out) {
    const SimDesc<R> &D = sim_desc(s, s.vblk_sim);
    Ctl *ctl = D.ctl;
    const int i = (blockIdx.x - D.vb0) * VBS + threadIdx.x;
    R dr[1] = {R(0)};
    if (i < D.c.n) {
        const int g = D.v0 + i;
        V4<R> r = q[g], z, zero;
        zero.x = zero.y = zero.z = zero.w = R(0);
        if (i >= D.c.nf) r = zero;
        const R di = i < D.c.nf ? s.pcg_dinv[g] : R(0);
        z.x = di * r.x; z.y = di * r.y; z.z = di * r.z; z.w = R(0);
        s.pcg_r[g] = r;
        s.pcg_z[g] = z;
        s.pcg_p[g] = zero;
        out[g] = zero;
        dr[0] = dotr(r, z);
    }
    double tot[1];
    block_sum_r<VBS, 1, R>(dr, tot);
    if (!sim_arrive<R, 1>(tot, s.part_v, s.nvb, D.nvb, &ctl->ticket[TK_PCG_B])) return;
    const double rz = sum_block_range<R, VBS>(s.part_v, D.vb0, D.nvb);
    if (threadIdx.x == 0) {
        ctl->ticket[TK_PCG_B] = 0u;
        ctl->pcg_rz = rz;
        ctl->pcg_beta = 0.0;
    }
}

// Corners of L p (one thread per tet).
template <typename R>
__global__ void __launch_bounds__(TBS, 8) k_pcg_tet(DevSim<R> s) {
    const SimDesc<R> &D = sim_desc(s, s.tblk_sim);
    const int tl = (blockIdx.x - D.tb0) * TBS + threadIdx.x;
    if (tl >= D.c.T) return;
    const R beta = (R)D.ctl->pcg_beta;
    const int t = D.t0 + tl;
    const int4 v = s.tets[t];
    const V4<R> p0 = pcg_p(s, v.x, beta), p1 = pcg_p(s, v.y, beta), p2 = pcg_p(s, v.z, beta),
                p3 = pcg_p(s, v.w, beta);
    R du[3][3], Di[9], G[3][3];
    edge_diffs(p0, p1, p2, p3, du);
    load_dm(s, t, Di);
    def_grad(du, Di, G);
    const R w = s.vol[t] * (D.n_mats > 1 ? D.kmat[s.tmat[t]] : D.c.kstiff);
    R g[4][3];
#pragma unroll
    for (int j = 0; j < 3; ++j)
#pragma unroll
        for (int a = 0; a < 3; ++a)
            g[j + 1][a] = w * (G[a][0] * Di[j * 3 + 0] + G[a][1] * Di[j * 3 + 1] + G[a][2] * Di[j * 3 + 2]);
#pragma unroll
    for (int a = 0; a < 3; ++a) g[0][a] = -(g[1][a] + g[2][a] + g[3][a]);
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        V4<R> o;
        o.x = g[k][0]; o.y = g[k][1]; o.z = g[k][2]; o.w = R(0);
        s.corner[s.corner_pos[(size_t)k * s.Tn + t]] = o;
    }
}

// p = z + beta p_old (stored), A0 p = M/h^2 p + L p, and p^T A0 p; the last
// block sets alpha = r^T z / p^T A0 p.
template <typename R>
__global__ void __launch_bounds__(VBS) k_pcg_gather(DevSim<R> s) {
    const SimDesc<R> &D = sim_desc(s, s.vblk_sim);
    Ctl *ctl = D.ctl;
    const int i = (blockIdx.x - D.vb0) * VBS + threadIdx.x;
    R dr[1] = {R(0)};
    if (i < D.c.nf) {
        const int g = D.v0 + i;
        const R beta = (R)ctl->pcg_beta;
        const int b = s.vt_ptr[g], e = s.vt_ptr[g + 1];
        const V4<R> p = pcg_p(s, g, beta);
        const R mh = s.mh2[g];
        R ax = R(0), ay = R(0), az = R(0);
#pragma unroll 8
        for (int k = b; k < e; ++k) {
            const V4<R> c = s.corner[k];
            ax += c.x; ay += c.y; az += c.z;
        }
        V4<R> ap;
        ap.x = ax + mh * p.x; ap.y = ay + mh * p.y; ap.z = az + mh * p.z; ap.w = R(0);
        s.pcg_p[g] = p;
        s.pcg_ap[g] = ap;
        dr[0] = dotr(p, ap);
    }
    double tot[1];
    block_sum_r<VBS, 1, R>(dr, tot);
    if (!sim_arrive<R, 1>(tot, s.part_v, s.nvb, D.nvb, &ctl->ticket[TK_PCG_A])) return;
    const double pap = sum_block_range<R, VBS>(s.part_v, D.vb0, D.nvb);
    if (threadIdx.x == 0) {
        ctl->ticket[TK_PCG_A] = 0u;
        ctl->pcg_alpha = pap > 0.0 ? ctl->pcg_rz / pap : 0.0;
    }
}

// x += alpha p, r -= alpha A0 p, z = D^{-1} r; the last block sets
// beta = r^T z (new) / r^T z (old).
template <typename R>
__global__ void __launch_bounds__(VBS) k_pcg_update(DevSim<R> s, V4<R> *out) {
    const SimDesc<R> &D = sim_desc(s, s.vblk_sim);
    Ctl *ctl = D.ctl;
    const int i = (blockIdx.x - D.vb0) * VBS + threadIdx.x;
    R dr[1] = {R(0)};
    if (i < D.c.nf) {
        const int g = D.v0 + i;
        const R alpha = (R)ctl->pcg_alpha;
        const V4<R> p = s.pcg_p[g], ap = s.pcg_ap[g];
        V4<R> x = out[g], r = s.pcg_r[g], z;
        const R di = s.pcg_dinv[g];
        x.x += alpha * p.x; x.y += alpha * p.y; x.z += alpha * p.z;
        r.x -= alpha * ap.x; r.y -= alpha * ap.y; r.z -= alpha * ap.z;
        z.x = di * r.x; z.y = di * r.y; z.z = di * r.z; z.w = R(0);
        out[g] = x;
        s.pcg_r[g] = r;
        s.pcg_z[g] = z;
        dr[0] = dotr(r, z);
    }
    double tot[1];
    block_sum_r<VBS, 1, R>(dr, tot);
    if (!sim_arrive<R, 1>(tot, s.part_v, s.nvb, D.nvb, &ctl->ticket[TK_PCG_B])) return;
    const double rz = sum_block_range<R, VBS>(s.part_v, D.vb0, D.nvb);
    if (threadIdx.x == 0) {
        ctl->ticket[TK_PCG_B] = 0u;
        ctl->pcg_beta = ctl->pcg_rz > 0.0 ? rz / ctl->pcg_rz : 0.0;
        ctl->pcg_rz = rz;
    }
}

// Drops the history of the simulations whose direction was not a descent
// direction (the others keep theirs and recompute the same direction).
template <typename R>
__global__ void k_reset_history(DevSim<R> s) {
    for (int k = threadIdx.x; k < s.nsims; k += blockDim.x) {
        Ctl *c = s.desc[k].ctl;
        if (c->nondescent) {
            c->count = 0;
            c->nondescent = 0;
        }
    }
}

// q_{l-1} := q_l, q_l := x (end of the time step, Eq. PD).
template <typename R>
__global__ void __launch_bounds__(VBS) k_commit(DevSim<R> s) {
    const SimDesc<R> &D = sim_desc(s, s.vblk_sim);
    const int i = (blockIdx.x - D.vb0) * VBS + threadIdx.x;
    if (i < D.c.n) {
        const int g = D.v0 + i;
        s.u_prev[g] = s.u_cur[g];
        s.u_cur[g] = s.xk[g];
    }
    if (blockIdx.x == D.vb0 && threadIdx.x == 0) {
        Ctl *c = D.ctl;
        c->steps += 1;
        if (c->status > c->worst_status) c->worst_status = c->status;
    }
}

// Absolute positions x_v = X_v + u_v of n vertices starting at batch vertex
// v0, written in the caller's vertex order (out[perm[i]], perm[i] < n).
template <typename R>
__global__ void __launch_bounds__(VBS) k_positions(const V4<R> *rest, const V4<R> *u, const int *perm, int v0, int n,
                                                   V4<R> *out) {
    const int i = blockIdx.x * VBS + threadIdx.x;
    if (i < n) {
        const V4<R> X = rest[v0 + i], d = u[v0 + i];
        V4<R> o;
        o.x = X.x + d.x; o.y = X.y + d.y; o.z = X.z + d.z; o.w = R(0);
        out[perm[i]] = o;
    }
}

// Caller-order float64 positions (n x 3, device) -> internal displacements
// u = x - X, with X the float64 rest positions in internal order (vertex i
// of the internal order is caller vertex perm[i]); subtracted in float64 and
// rounded once, as the host-side transfers do.
template <typename R>
__global__ void __launch_bounds__(VBS) k_from_caller(const double *X, const double *src, const int *perm, int v0,
                                                    int n, V4<R> *dst) {
    const int i = blockIdx.x * VBS + threadIdx.x;
    if (i < n) {
        const int v = perm[i];
        V4<R> o;
        o.x = (R)(src[3 * (size_t)v] - X[3 * (size_t)i]);
        o.y = (R)(src[3 * (size_t)v + 1] - X[3 * (size_t)i + 1]);
        o.z = (R)(src[3 * (size_t)v + 2] - X[3 * (size_t)i + 2]);
        o.w = R(0);
        dst[v0 + i] = o;
    }
}

// Internal vectors -> caller-order float64 (n x 3, device); rows of clamped
// vertices (internal index >= nf) are zero.
template <typename R>
__global__ void __launch_bounds__(VBS) k_to_caller(const V4<R> *src, const int *perm, int v0, int n, int nf,
                                                  double *dst) {
    const int i = blockIdx.x * VBS + threadIdx.x;
    if (i < n) {
        const int v = perm[i];
        const V4<R> a = src[v0 + i];
        const bool fixed = i >= nf;
        dst[3 * (size_t)v] = fixed ? 0.0 : (double)a.x;
        dst[3 * (size_t)v + 1] = fixed ? 0.0 : (double)a.y;
        dst[3 * (size_t)v + 2] = fixed ? 0.0 : (double)a.z;
    }
}

// Caller-given history of simulation 0 (sim_direction): row `a` of the Gram
// matrix, s_a^T t_b for the slots b < count, rho_a = s_a^T t_a and
// s_a^T grad.  With a == count - 1 the last block also runs the first loop
// on scalars.  Launched over simulation 0's vertex blocks.
template <typename R>
__global__ void __launch_bounds__(VBS) k_hist_row(DevSim<R> s, int a) {
    const SimDesc<R> &D = s.desc0;
    Ctl *ctl = D.ctl;
    constexpr int NB = kShortHist + 2;
    double dots[NB];
#pragma unroll
    for (int b = 0; b < NB; ++b) dots[b] = 0.0;
    const int count = ctl->count;
    const size_t n = (size_t)D.c.n;
    const int i = blockIdx.x * VBS + threadIdx.x;
    if (i < D.c.nf) {
        const V4<R> *S = s.S + D.ring0, *Tt = s.Tt + D.ring0;
        const V4<R> sa = S[(size_t)a * n + i];
#pragma unroll
        for (int b = 0; b < NB - 1; ++b)
            if (b < count) dots[b] = dotv(sa, Tt[(size_t)b * n + i]);
        dots[NB - 1] = dotv(sa, s.gk[D.v0 + i]);
    }
    block_sum<VBS, NB>(dots);
    if (!publish_and_arrive<NB>(dots, s.part_g, gridDim.x, &ctl->ticket[TK_GATHER])) return;
    sum_partials<VBS, NB>(s.part_g, gridDim.x, gridDim.x, dots, &ctl->ticket[TK_GATHER]);
    if (threadIdx.x == 0) {
#pragma unroll
        for (int b = 0; b < NB - 1; ++b) {
            if (b < count) ctl->gram[a][b] = dots[b];
            if (b == a) ctl->rho[a] = dots[b];
        }
        ctl->sg[a] = dots[NB - 1];
    }
    if (a != count - 1) return;
    // all rows are in place: the first loop on scalars
    __threadfence();
    __syncthreads();
    __shared__ HistSmem hs;
    hist_load(ctl, hs, s.m);
    if (threadIdx.x == 0) {
        for (int b = 0; b < count; ++b) hs.sg[b] = ctl->sg[b];
        zeta_recursion(hs, s.m);
    }
    __syncthreads();
    for (int p = threadIdx.x; p < count; p += VBS) ctl->zeta[p] = hs.zeta[p];
}

// ---------------------------------------------------------------- long history windows
//
// A window of m > kShortHist pairs keeps its scalars in LongHist (device
// memory of its own) and forms the slot products of Alg. 2 in two launches:
// k_ldots over (vertex blocks) x (chunks of LH_CHUNK slots), block partials
// only, then k_lrec, one block per simulation, which adds each value's
// partials in block order, updates the Gram matrix and scalars and runs a
// loop's recursion on scalars column by column (after zeta_p / c_p is known,
// every later term subtracts / adds its share in parallel; the first loop
// adds its terms in the order of the short windows' recursion, the second
// in the reverse order).

template <typename R>
__global__ void __launch_bounds__(VBS) k_ldots(DevSim<R> s, int mode, int a0) {
    const SimDesc<R> &D = mode == LD_ROW ? s.desc0 : sim_desc(s, s.vblk_sim);
    const Ctl *ctl = D.ctl;
    const int m = s.m, c0 = blockIdx.y * LH_CHUNK;
    constexpr int NV = 3 * LH_CHUNK;
    R dr[NV];
#pragma unroll
    for (int v = 0; v < NV; ++v) dr[v] = R(0);
    const int vb = mode == LD_ROW ? (int)blockIdx.x : (int)blockIdx.x - D.vb0;
    const int i = vb * VBS + threadIdx.x;
    const bool on = ctl->active && (mode != LD_R0 || ctl->count > 0);
    if (on && i < D.c.nf) {
        const size_t n = (size_t)D.c.n;
        const V4<R> *S = s.S + D.ring0, *Tt = s.Tt + D.ring0;
        const int w = mode == LD_PUSH ? ctl->hist_w : a0;
        V4<R> f0 = mode == LD_R0 ? s.d[D.v0 + i] : S[(size_t)w * n + i];  // r0, or s_w / s_a0
        V4<R> f1 = f0, g = f0;
        if (mode == LD_PUSH) f1 = Tt[(size_t)w * n + i];                     // t_w
        if (mode != LD_R0) g = s.gk[D.v0 + i];
#pragma unroll
        for (int a = 0; a < LH_CHUNK; ++a) {
            const int sl = c0 + a;
            if (sl > m) break;
            const V4<R> ta = Tt[(size_t)sl * n + i];
            if (mode == LD_R0) {
                dr[a] = dotr(ta, f0);
            } else {
                const V4<R> sa = S[(size_t)sl * n + i];
                if (mode == LD_PUSH) {
                    dr[a] = dotr(sa, f1);
                    dr[LH_CHUNK + a] = dotr(f0, ta);
                } else {
                    dr[a] = dotr(f0, ta);
                }
                dr[2 * LH_CHUNK + a] = dotr(sa, g);
            }
        }
    }
    double out[NV];
    block_sum_r<VBS, NV, R>(dr, out);
    if (threadIdx.x == 0) {
        double *part = s.part_l + (size_t)blockIdx.y * NV * gridDim.x + blockIdx.x;
#pragma unroll
        for (int v = 0; v < NV; ++v) part[(size_t)v * gridDim.x] = out[v];
    }
}

// Dynamic shared memory of k_lrec for a window of m pairs.
inline size_t lrec_smem(int m) {
    const size_t L = (size_t)m + 1, nch = (L + LH_CHUNK - 1) / LH_CHUNK;
    return sizeof(double) * (L * L + 3 * LH_CHUNK * nch + 3 * L);
}

template <typename R>
__global__ void __launch_bounds__(256) k_lrec(DevSim<R> s, int mode, int a0, int nbx) {
    const SimDesc<R> &D = (mode == LD_ROW || s.nsims == 1) ? s.desc0 : s.desc[blockIdx.x];
    Ctl *ctl = D.ctl;
    if (!ctl->active) return;
    const int m = s.m, L = m + 1, count = ctl->count, head = ctl->head;
    if (mode == LD_R0 && count == 0) return;
    constexpr int NV = 3 * LH_CHUNK;
    const int nch = (L + LH_CHUNK - 1) / LH_CHUNK;
    LongHist H(D.lh, m);
    extern __shared__ double lsm[];
    double *G = lsm;                          // L x L Gram matrix
    double *tot = G + (size_t)L * L;          // nch x NV totals
    double *acc = tot + (size_t)NV * nch;     // L running sums of the recursion
    double *rinv = acc + L;                   // 1 / rho by ring slot
    double *out = rinv + L;                   // zeta or c by age
    const int tid = threadIdx.x, nt = blockDim.x;
    // the simulation's partials, value by value, added in block order
    const int vb0 = mode == LD_ROW ? 0 : D.vb0, nb = mode == LD_ROW ? nbx : D.nvb;
    for (int v = tid; v < NV * nch; v += nt) {
        const int slot = (v / NV) * LH_CHUNK + v % LH_CHUNK;
        tot[v] = slot <= m ? strided_sum(s.part_l + (size_t)v * nbx + vb0, 0, nb, 1) : 0.0;
    }
    __syncthreads();
    auto val = [&](int q, int slot) { return tot[(slot / LH_CHUNK) * NV + q * LH_CHUNK + slot % LH_CHUNK]; };
    bool zeta_rec = false;
    if (mode == LD_PUSH) {
        const int w = ctl->hist_w;
        if (ctl->hist_keep)
            for (int a = tid; a <= m; a += nt) {
                H.gram[(size_t)a * L + w] = val(0, a);  // s_a^T t_w
                H.gram[(size_t)w * L + a] = val(1, a);  // s_w^T t_a
            }
        for (int a = tid; a <= m; a += nt) H.sg[a] = val(2, a);
        zeta_rec = true;
    } else if (mode == LD_R0) {
        for (int a = tid; a <= m; a += nt) H.tr0[a] = val(0, a);
    } else {
        for (int b = tid; b < count; b += nt) {
            H.gram[(size_t)a0 * L + b] = val(0, b);  // s_a0^T t_b
            H.sg[b] = val(2, b);
            if (b == a0) H.rho[a0] = val(0, b);
        }
        zeta_rec = a0 == count - 1;
        if (!zeta_rec) return;
    }
    __syncthreads();  // (global writes of this block, read back below)
    for (int e = tid; e < L * L; e += nt) G[e] = H.gram[e];
    for (int a = tid; a < L; a += nt) rinv[a] = 1.0 / H.rho[a];
    if (zeta_rec) {
        // zeta_p = (-s_p^T grad - sum_{p' < p} zeta_p' s_p^T t_p') / rho_p, newest first
        for (int p = tid; p < count; p += nt) acc[p] = -H.sg[ring_slot(head, p, m)];
        __syncthreads();
        for (int p = 0; p < count; ++p) {
            const int sp = ring_slot(head, p, m);
            const double z = acc[p] * rinv[sp];
            for (int q = p + 1 + tid; q < count; q += nt) acc[q] -= z * G[(size_t)ring_slot(head, q, m) * L + sp];
            if (tid == 0) out[p] = z;
            __syncthreads();
        }
        for (int p = tid; p < count; p += nt) H.zeta[p] = out[p];
    } else {
        // c_p = zeta_p - (t_p^T r0 + sum_{p' > p} c_p' s_p'^T t_p) / rho_p, oldest first
        for (int p = tid; p < count; p += nt) acc[p] = H.tr0[ring_slot(head, p, m)];
        __syncthreads();
        for (int p = count - 1; p >= 0; --p) {
            const int sp = ring_slot(head, p, m);
            const double c = H.zeta[p] - acc[p] * rinv[sp];
            for (int q = tid; q < p; q += nt) acc[q] += c * G[(size_t)sp * L + ring_slot(head, q, m)];
            if (tid == 0) out[p] = c;
            __syncthreads();
        }
        for (int p = tid; p < count; p += nt) H.coef[p] = out[p];
    }
}

}  // namespace

// ---------------------------------------------------------------- launchers

template <typename R> void launch_predict(const DevSim<R> &s, cudaStream_t st) {
    k_predict<R><<<s.nvb, VBS, 0, st>>>(s);
}
template <typename R> void launch_inertia(const DevSim<R> &s, cudaStream_t st) {
    k_inertia<R><<<s.nvb, VBS, 0, st>>>(s);
}
template <typename R> void launch_tet(const DevSim<R> &s, int mode, CondHandles h, cudaStream_t st) {
    k_tet<R><<<s.ntb, TBS, 0, st>>>(s, mode, h);
}
template <typename R> void launch_ls(const DevSim<R> &s, CondHandles h, cudaStream_t st) {
    switch (s.ls_batch) {
        case 1: k_ls<R, 1><<<s.ntb, TBS, 0, st>>>(s, h); break;
        case 2: k_ls<R, 2><<<s.ntb, TBS, 0, st>>>(s, h); break;
        case 4: k_ls<R, 4><<<s.ntb, TBS, 0, st>>>(s, h); break;
        case 16: k_ls<R, 16><<<s.ntb, TBS, 0, st>>>(s, h); break;
        default: k_ls<R, 8><<<s.ntb, TBS, 0, st>>>(s, h); break;
    }
}
template <typename R> void launch_gather(const DevSim<R> &s, int mode, CondHandles h, cudaStream_t st) {
    const int m = s.m;
    if (m <= 0) k_gather<R, 1><<<s.nvb, VBS, 0, st>>>(s, mode, h);
    else if (m <= 3) k_gather<R, 4><<<s.nvb, VBS, 0, st>>>(s, mode, h);
    else if (m <= 5) k_gather<R, 6><<<s.nvb, VBS, 0, st>>>(s, mode, h);
    else if (m <= 8) k_gather<R, 9><<<s.nvb, VBS, 0, st>>>(s, mode, h);
    else if (m <= kShortHist) k_gather<R, kShortHist + 1><<<s.nvb, VBS, 0, st>>>(s, mode, h);
    else k_gather<R, 0><<<s.nvb, VBS, 0, st>>>(s, mode, h);
}
template <typename R> void launch_q(const DevSim<R> &s, cudaStream_t st) {
    const int m = s.m;
    if (m <= 0) k_q<R, 1><<<s.nvb, VBS, 0, st>>>(s);
    else if (m <= 3) k_q<R, 4><<<s.nvb, VBS, 0, st>>>(s);
    else if (m <= 5) k_q<R, 6><<<s.nvb, VBS, 0, st>>>(s);
    else if (m <= 8) k_q<R, 9><<<s.nvb, VBS, 0, st>>>(s);
    else if (m <= kShortHist) k_q<R, kShortHist + 1><<<s.nvb, VBS, 0, st>>>(s);
    else k_q<R, 0><<<s.nvb, VBS, 0, st>>>(s);
}
template <typename R> void launch_r0_dots(const DevSim<R> &s, cudaStream_t st) {
    const int m = s.m;
    if (m <= 0) return;
    if (m <= 3) k_r0_dots<R, 4><<<s.nvb, VBS, 0, st>>>(s);
    else if (m <= 5) k_r0_dots<R, 6><<<s.nvb, VBS, 0, st>>>(s);
    else if (m <= 8) k_r0_dots<R, 9><<<s.nvb, VBS, 0, st>>>(s);
    else if (m <= kShortHist) k_r0_dots<R, kShortHist + 1><<<s.nvb, VBS, 0, st>>>(s);
    else launch_long_hist(s, LD_R0, 0, st, 0);
}
template <typename R>
void launch_direction_final(const DevSim<R> &s, CondHandles h, int set_nd, cudaStream_t st) {
    const int m = s.m;
    if (m <= 0) k_dir_final<R, 1><<<s.nvb, VBS, 0, st>>>(s, h, set_nd);
    else if (m <= 3) k_dir_final<R, 4><<<s.nvb, VBS, 0, st>>>(s, h, set_nd);
    else if (m <= 5) k_dir_final<R, 6><<<s.nvb, VBS, 0, st>>>(s, h, set_nd);
    else if (m <= 8) k_dir_final<R, 9><<<s.nvb, VBS, 0, st>>>(s, h, set_nd);
    else if (m <= kShortHist) k_dir_final<R, kShortHist + 1><<<s.nvb, VBS, 0, st>>>(s, h, set_nd);
    else k_dir_final<R, 0><<<s.nvb, VBS, 0, st>>>(s, h, set_nd);
}
template <typename R> void launch_reset_history(const DevSim<R> &s, cudaStream_t st) {
    k_reset_history<R><<<1, 256, 0, st>>>(s);
}
template <typename R> void launch_pcg(const DevSim<R> &s, const V4<R> *q, V4<R> *out, int iters, cudaStream_t st) {
    k_pcg_init<R><<<s.nvb, VBS, 0, st>>>(s, q, out);
    for (int k = 0; k < iters; ++k) {
        k_pcg_tet<R><<<s.ntb, TBS, 0, st>>>(s);
        k_pcg_gather<R><<<s.nvb, VBS, 0, st>>>(s);
        k_pcg_update<R><<<s.nvb, VBS, 0, st>>>(s, out);
    }
}
template <typename R> void launch_commit(const DevSim<R> &s, cudaStream_t st) {
    k_commit<R><<<s.nvb, VBS, 0, st>>>(s);
}
template <typename R> void launch_positions(const DevSim<R> &s, const int *perm, int v0, int n, V4<R> *out,
                                            cudaStream_t st) {
    if (n > 0) k_positions<R><<<(n + VBS - 1) / VBS, VBS, 0, st>>>(s.rest, s.u_cur, perm, v0, n, out);
}
template <typename R> void launch_from_caller(const double *X, const double *src, const int *perm, int v0, int n,
                                              V4<R> *dst, cudaStream_t st) {
    if (n > 0) k_from_caller<R><<<(n + VBS - 1) / VBS, VBS, 0, st>>>(X, src, perm, v0, n, dst);
}
template <typename R> void launch_to_caller(const V4<R> *src, const int *perm, int v0, int n, int nf, double *dst,
                                            cudaStream_t st) {
    if (n > 0) k_to_caller<R><<<(n + VBS - 1) / VBS, VBS, 0, st>>>(src, perm, v0, n, nf, dst);
}
template <typename R> void launch_hist_row(const DevSim<R> &s, int a, cudaStream_t st, int nblocks) {
    k_hist_row<R><<<nblocks, VBS, 0, st>>>(s, a);
}
template <typename R> void launch_long_hist(const DevSim<R> &s, int mode, int a0, cudaStream_t st, int nblocks) {
    const int nch = (s.m + 1 + LH_CHUNK - 1) / LH_CHUNK;
    const int gx = mode == LD_ROW ? nblocks : s.nvb;
    k_ldots<R><<<dim3((unsigned)gx, (unsigned)nch), VBS, 0, st>>>(s, mode, a0);
    k_lrec<R><<<mode == LD_ROW ? 1 : s.nsims, 256, lrec_smem(s.m), st>>>(s, mode, a0, gx);
}
template <typename R> cudaError_t long_hist_prepare(int m) {
    return cudaFuncSetAttribute(k_lrec<R>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)lrec_smem(m));
}

#define HQN_INST(R)                                                                  \
    template void launch_predict<R>(const DevSim<R> &, cudaStream_t);                \
    template void launch_inertia<R>(const DevSim<R> &, cudaStream_t);                \
    template void launch_tet<R>(const DevSim<R> &, int, CondHandles, cudaStream_t);  \
    template void launch_ls<R>(const DevSim<R> &, CondHandles, cudaStream_t);        \
    template void launch_gather<R>(const DevSim<R> &, int, CondHandles, cudaStream_t); \
    template void launch_q<R>(const DevSim<R> &, cudaStream_t);                      \
    template void launch_r0_dots<R>(const DevSim<R> &, cudaStream_t);                \
    template void launch_direction_final<R>(const DevSim<R> &, CondHandles, int, cudaStream_t); \
    template void launch_reset_history<R>(const DevSim<R> &, cudaStream_t);          \
    template void launch_commit<R>(const DevSim<R> &, cudaStream_t);                 \
    template void launch_pcg<R>(const DevSim<R> &, const V4<R> *, V4<R> *, int, cudaStream_t); \
    template void launch_hist_row<R>(const DevSim<R> &, int, cudaStream_t, int);       \
    template void launch_long_hist<R>(const DevSim<R> &, int, int, cudaStream_t, int); \
    template cudaError_t long_hist_prepare<R>(int);                                   \
    template void launch_positions<R>(const DevSim<R> &, const int *, int, int, V4<R> *, cudaStream_t); \
    template void launch_from_caller<R>(const double *, const double *, const int *, int, int, V4<R> *, cudaStream_t); \
    template void launch_to_caller<R>(const V4<R> *, const int *, int, int, int, double *, cudaStream_t);

HQN_INST(float)
HQN_INST(double)

}  // namespace hqn
