// Step kernels of the quasi-Newton implicit-Euler solver: predictor (Eq. PD),
// line-search trial update and Armijo test (Alg. 1), per-tet energy and
// corner gradients (Eq. valanis-landel), the atomic-free vertex gather of
// grad g (Eq. PD), the history push and the two loops of Alg. 2.
#include "kernels.cuh"
#include "reduce.cuh"
#include "tetmath.cuh"

namespace hqn {

namespace {

template <typename R>
__device__ __forceinline__ V4<R> ld(const V4<R> *p, int i) { return p[i]; }

template <typename R>
__device__ __forceinline__ void set_cond(unsigned long long h, unsigned int v) {
    if (h) cudaGraphSetConditional((cudaGraphConditionalHandle)h, v);
}

__device__ __forceinline__ int ring_slot(int head, int age, int m) {
    int s = head - age;
    return s < 0 ? s + m + 1 : s;
}

// ---------------------------------------------------------------- predictor

// y = 2 q_l - q_{l-1} + h^2 g on free vertices, y = q_l on clamped ones;
// x_1 = y.  Thread 0 of block 0 also clears the step's control block.
template <typename R>
__global__ void __launch_bounds__(VBS) k_predict(DevSim<R> s) {
    const int i = blockIdx.x * VBS + threadIdx.x;
    if (i < s.c.n) {
        const V4<R> a = s.u_cur[i], b = s.u_prev[i];
        V4<R> yy = a;
        if (i < s.c.nf) {
            yy.x = R(2) * a.x - b.x + s.c.gx;
            yy.y = R(2) * a.y - b.y + s.c.gy;
            yy.z = R(2) * a.z - b.z + s.c.gz;
        }
        yy.w = R(0);
        s.y[i] = yy;
        s.xk[i] = yy;
        s.xt[i] = yy;
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        Ctl *c = s.ctl;
        c->k = 0; c->trials = 0; c->count = 0; c->head = 0; c->stop = 0;
        c->status = HQN_OK; c->accepted = 0; c->nondescent = 0; c->alpha = 1.0; c->grad_ready = 0;
    }
}

// ---------------------------------------------------------------- inertia of a given x

// Block partial of the inertia term 1/(2h^2) sum m_v |x_t - y|^2 of Eq. PD at
// the caller-given point x_t (the start of a step, or an evaluation request).
template <typename R>
__global__ void __launch_bounds__(VBS) k_inertia(DevSim<R> s) {
    using A = ExactAcc<R>;
    const int i = blockIdx.x * VBS + threadIdx.x;
    typename A::T e[1] = {A::zero()};
    if (i < s.c.n) {
        const V4<R> x = s.xt[i], yy = s.y[i];
        const R dx = x.x - yy.x, dy = x.y - yy.y, dz = x.z - yy.z;
        e[0] = A::add(e[0], R(0.5) * s.mh2[i] * (dx * dx + dy * dy + dz * dz));
    }
    double tot[1];
    block_sum_exact<VBS, 1, R>(e, tot);
    if (threadIdx.x == 0) s.part_in[blockIdx.x] = tot[0];
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
    for (int k = 0; k < 9; ++k) Di[k] = s.dminv[(size_t)k * s.c.T + t];
}

template <typename R>
__device__ __forceinline__ void edge_diffs(const V4<R> &x0, const V4<R> &x1, const V4<R> &x2, const V4<R> &x3,
                                           R du[3][3]) {
    du[0][0] = x1.x - x0.x; du[0][1] = x1.y - x0.y; du[0][2] = x1.z - x0.z;
    du[1][0] = x2.x - x0.x; du[1][1] = x2.y - x0.y; du[1][2] = x2.z - x0.z;
    du[2][0] = x3.x - x0.x; du[2][1] = x3.y - x0.y; du[2][2] = x3.z - x0.z;
}

// ---------------------------------------------------------------- tet kernel

// One thread per tet: the four corner gradients of V Psi, written to
// corner[c * T + t].
//   TET_INIT / TET_EVAL: at the point x_t, with the energy reduced too (last
//     block, fixed order, float64, plus the inertia partials): TET_INIT sets
//     g(x_1), TET_EVAL reports g.
//   TET_TRIAL1: the first trial of Alg. 1's line search, alpha = 1, at
//     x_k + d; the last block adds the inertia term along the ray and runs the
//     Armijo test.  Accepted: the corners are the gradient of x_{k+1} and the
//     line-search loop is skipped.  Rejected: the loop continues at
//     alpha = backtrack.
//   TET_GRAD: at the accepted point x_k + alpha d, corners only; nothing to do
//     if TET_TRIAL1 already left them there or the iterations stopped.
template <typename R, int BS>
__global__ void __launch_bounds__(BS, 1024 / BS) k_tet(DevSim<R> s, int mode, CondHandles h) {
    const bool grad_mode = mode == TET_GRAD;
    const bool ray_mode = mode == TET_GRAD || mode == TET_TRIAL1;
    if (grad_mode && (s.ctl->stop || s.ctl->grad_ready)) return;
    const R al = grad_mode ? (R)s.ctl->alpha : R(1);
    using A = ExactAcc<R>;
    const int T = s.c.T;
    const int t = blockIdx.x * BS + threadIdx.x;
    typename A::T e[1] = {A::zero()};
    if (t < T) {
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
        tet_grad(s.mat, G, Di, vol, g);
        if (!grad_mode) e[0] = A::add(e[0], vol * tet_psi(s.mat, G));
#pragma unroll
        for (int c = 0; c < 4; ++c) {
            V4<R> o;
            o.x = g[c][0]; o.y = g[c][1]; o.z = g[c][2]; o.w = R(0);
            s.corner[(size_t)c * T + t] = o;
        }
    }
    if (grad_mode) return;
    double tot[1];
    block_sum_exact<BS, 1, R>(e, tot);
    if (!publish_and_arrive<1>(tot, s.part_el, 0, &s.ctl->ticket[TK_TET])) return;
    sum_partials<BS, 1>(s.part_el, 0, gridDim.x, tot, &s.ctl->ticket[TK_TET]);
    Ctl *c = s.ctl;
    if (mode == TET_TRIAL1) {
        if (threadIdx.x != 0) return;
        // g(x_k + d) - g(x_k) = E(x_k + d) - E(x_k) + I(1) - I(0) with the
        // inertia term I(alpha) = a0 + a1 alpha + a2 alpha^2 along the ray
        const double e = tot[0];
        const double dI = c->ls_a[1] + c->ls_a[2];
        c->passes_total += 1;
        c->trials = 1;
        if ((e - c->e_k) + dI <= s.c.gamma * c->gd) {
            c->accepted = 1;
            c->grad_ready = 1;
            c->alpha = 1.0;
            c->e_trial = e;
            c->g_trial = e + c->ls_a[0] + dI;
            set_cond<R>(h.ls, 0u);
        } else {
            c->accepted = 0;
            c->grad_ready = 0;
            c->alpha = s.c.backtrack;
            if (s.c.ls_max <= 1) {
                c->stop = 1;
                c->status = HQN_WARN_LS_EXHAUSTED;
                set_cond<R>(h.ls, 0u);
            } else {
                set_cond<R>(h.ls, 1u);
            }
        }
        return;
    }
    double in[1];
    const int nbv = (s.c.n + VBS - 1) / VBS;
    {
        double acc = 0.0;
        for (int i = threadIdx.x; i < nbv; i += BS) acc += __ldcg(s.part_in + i);
        in[0] = acc;
        block_sum<BS, 1>(in);
    }
    if (threadIdx.x != 0) return;
    const double g = tot[0] + in[0];
    c->g_trial = g;
    if (mode == TET_INIT) {
        c->g_k = g;
        c->e_k = tot[0];
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
// time).  Otherwise the next pass
// continues from alpha_K, until ls_max trials in all.
template <typename R, int BS, int K>
__global__ void __launch_bounds__(BS) k_ls(DevSim<R> s, CondHandles h) {
    Ctl *ctl = s.ctl;
    const double a0 = ctl->alpha;
    const double bt = s.c.backtrack;
    using A = ExactAcc<R>;
    const int T = s.c.T;
    const int t = blockIdx.x * BS + threadIdx.x;
    typename A::T e[K];
#pragma unroll
    for (int j = 0; j < K; ++j) e[j] = A::zero();
    if (t < T) {
        const int4 v = s.tets[t];
        R Duk[3][3], Dd[3][3], Di[9], Gk[3][3], Gd[3][3];
        edge_diffs(s.xk[v.x], s.xk[v.y], s.xk[v.z], s.xk[v.w], Duk);
        edge_diffs(s.d[v.x], s.d[v.y], s.d[v.z], s.d[v.w], Dd);
        load_dm(s, t, Di);
        def_grad(Duk, Di, Gk);
        def_grad(Dd, Di, Gd);
        const R vol = s.vol[t];
        PsiRay<R> ray;
        psi_ray_setup(s.mat, Gk, Gd, ray);
        double a = a0;
#pragma unroll
        for (int j = 0; j < K; ++j) {
            e[j] = A::add(e[j], vol * psi_ray_eval(s.mat, ray, (R)a));
            a *= bt;
        }
    }
    double tot[K];
    block_sum_exact<BS, K, R>(e, tot);
    if (!publish_and_arrive<K>(tot, s.part_ls, gridDim.x, &ctl->ticket[TK_LS])) return;
    sum_partials<BS, K>(s.part_ls, gridDim.x, gridDim.x, tot, &ctl->ticket[TK_LS]);
    if (threadIdx.x != 0) return;
    double a = a0;
    int tr = ctl->trials;
    ctl->passes_total += 1;
    const double ek = ctl->e_k, slope = s.c.gamma * ctl->gd;
    const double c0 = ctl->ls_a[0], c1 = ctl->ls_a[1], c2 = ctl->ls_a[2];
    bool done = false;
#pragma unroll
    for (int j = 0; j < K; ++j) {
        if (done) break;
        if (tr >= s.c.ls_max) {
            ctl->accepted = 0;
            ctl->stop = 1;
            ctl->status = HQN_WARN_LS_EXHAUSTED;
            done = true;
            break;
        }
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
        if (tr >= s.c.ls_max) {
            ctl->accepted = 0;
            ctl->stop = 1;
            ctl->status = HQN_WARN_LS_EXHAUSTED;
            done = true;
        }
    }
    if (done) set_cond<R>(h.ls, 0u);
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

__device__ __forceinline__ double dot3d(double ax, double ay, double az, double bx, double by, double bz) {
    return ax * bx + ay * by + az * bz;
}

template <typename R>
__device__ __forceinline__ double dotv(const V4<R> &a, const V4<R> &b) {
    return (double)a.x * b.x + (double)a.y * b.y + (double)a.z * b.z;
}

template <typename R>
__device__ __forceinline__ R dotr(const V4<R> &a, const V4<R> &b) {
    return a.x * b.x + a.y * b.y + a.z * b.z;
}

// The history scalars the recursions need, staged in shared memory by the
// last block of a kernel: the control block lives in global memory, and a
// recursion run on it directly would pay a memory round trip per step.
constexpr int MH = HQN_MAX_HISTORY + 1;
struct HistSmem {
    double gram[MH][MH];  // s_a^T t_b by ring slots
    double rho[MH], sg[MH], tr0[MH], zeta[MH], coef[MH];
    int count, head;
};

// All threads: load the Gram matrix (rows and columns <= m), rho, zeta,
// count and head into shared memory.
__device__ __forceinline__ void hist_load(const Ctl *c, HistSmem &h, int m) {
    const int m1 = m + 1;
    for (int e = threadIdx.x; e < m1 * m1; e += blockDim.x) h.gram[e / m1][e % m1] = c->gram[e / m1][e % m1];
    for (int a = threadIdx.x; a < m1; a += blockDim.x) {
        h.rho[a] = c->rho[a];
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
        h.zeta[p] = sq / h.rho[sl];
    }
}

// Second loop on scalars: c_p = zeta_p - eta_p, oldest first.
__device__ __forceinline__ void coef_recursion(HistSmem &h, int m) {
    for (int p = h.count - 1; p >= 0; --p) {
        const int sl = ring_slot(h.head, p, m);
        double tr = h.tr0[sl];
        for (int pp = p + 1; pp < h.count; ++pp) tr += h.coef[pp] * h.gram[ring_slot(h.head, pp, m)][sl];
        h.coef[p] = h.zeta[p] - tr / h.rho[sl];
    }
}

// ---------------------------------------------------------------- gather

// One thread per free vertex: grad g = m (x - y)/h^2 + sum of the vertex's
// corner gradients in a fixed (ascending tet) order -- no atomics.  In G_ITER
// mode the accepted trial becomes x_{k+1}: the pair s = x_{k+1} - x_k,
// t = grad_{k+1} - grad_k goes to the free ring slot w, and the block partials
// of rho = tr(t^T s) (float64 terms) and of |s|^2, |t|^2, s_a^T t_w, s_w^T t_a
// and s_a^T grad_{k+1} for every ring slot a (R-precision terms and warp sums,
// float64 beyond) are reduced.  The last block keeps the pair if
// rho > 1e-12 |s| |t|, updates the Gram matrix and runs the first loop of
// Alg. 2 on scalars.
template <typename R, int MP1>
__global__ void __launch_bounds__(VBS) k_gather(DevSim<R> s, int mode, CondHandles h) {
    Ctl *ctl = s.ctl;
    const int m = s.c.m;
    const bool stop = mode == G_ITER && ctl->stop;
    const bool push = mode == G_ITER && m > 0;
    const int w = push ? (ctl->head + 1) % (m + 1) : 0;
    const R al = mode == G_ITER ? (R)ctl->alpha : R(0);
    constexpr int NG = 2 + 3 * MP1;  // |s|^2, |t|^2, then three products per slot
    constexpr int ND = 1 + NG;
    using A = ExactAcc<R>;
    typename A::T dd[1] = {A::zero()};
    R dr[NG];
#pragma unroll
    for (int k = 0; k < NG; ++k) dr[k] = R(0);
    const size_t n = (size_t)s.c.n;
    const int i = blockIdx.x * VBS + threadIdx.x;
    if (!stop && i < s.c.nf) {
        const int b = s.vt_ptr[i], e = s.vt_ptr[i + 1];
        R gx = R(0), gy = R(0), gz = R(0);
        for (int k = b; k < e; ++k) {
            const V4<R> cg = s.corner[s.vt_slot[k]];
            gx += cg.x; gy += cg.y; gz += cg.z;
        }
        const V4<R> x = mode == G_ITER ? step_point(s.xk[i], s.d[i], al) : s.xt[i];
        const V4<R> yy = s.y[i];
        const R mh = s.mh2[i];
        V4<R> gn;
        gn.x = gx + mh * (x.x - yy.x);
        gn.y = gy + mh * (x.y - yy.y);
        gn.z = gz + mh * (x.z - yy.z);
        gn.w = R(0);
        if (mode == G_ITER) {
            if (push) {
                const V4<R> xo = s.xk[i], go = s.gk[i];
                V4<R> sv, tv;
                sv.x = x.x - xo.x; sv.y = x.y - xo.y; sv.z = x.z - xo.z; sv.w = R(0);
                tv.x = gn.x - go.x; tv.y = gn.y - go.y; tv.z = gn.z - go.z; tv.w = R(0);
                s.S[(size_t)w * n + i] = sv;
                s.Tt[(size_t)w * n + i] = tv;
                dd[0] = A::add_prod(A::add_prod(A::add_prod(dd[0], tv.x, sv.x), tv.y, sv.y), tv.z, sv.z);
                dr[0] = dotr(sv, sv);
                dr[1] = dotr(tv, tv);
#pragma unroll
                for (int a = 0; a < MP1; ++a) {
                    if (a > m) break;
                    const V4<R> sa = a == w ? sv : s.S[(size_t)a * n + i];
                    const V4<R> ta = a == w ? tv : s.Tt[(size_t)a * n + i];
                    dr[2 + a] = dotr(sa, tv);
                    dr[2 + MP1 + a] = dotr(sv, ta);
                    dr[2 + 2 * MP1 + a] = dotr(sa, gn);
                }
            }
            s.xk[i] = x;
        }
        s.gk[i] = gn;
    }
    if (mode == G_EVAL) return;
    double dots[ND];
    if (push) {
        double mixed[NG], rho[1];
        block_sum_exact<VBS, 1, R>(dd, rho);
        block_sum_r<VBS, NG, R>(dr, mixed);
        dots[0] = rho[0];
#pragma unroll
        for (int k = 0; k < NG; ++k) dots[1 + k] = mixed[k];
        if (!publish_and_arrive<ND>(dots, s.part_g, gridDim.x, &ctl->ticket[TK_GATHER])) return;
        sum_partials<VBS, ND>(s.part_g, gridDim.x, gridDim.x, dots, &ctl->ticket[TK_GATHER]);
    } else {
        double none[1] = {0.0};
        if (!publish_and_arrive<1>(none, s.part_g, gridDim.x, &ctl->ticket[TK_GATHER])) return;
        __threadfence();
        if (threadIdx.x == 0) ctl->ticket[TK_GATHER] = 0u;
    }
    if (mode == G_INIT) {
        if (threadIdx.x != 0) return;
        ctl->k = 1;
        ctl->count = 0;
        ctl->head = 0;
        ctl->g_k = ctl->g_trial;
        set_cond<R>(h.it, s.c.iters > 0 ? 1u : 0u);
        return;
    }
    const int k = ctl->k;
    const int kk = k - 1 < HQN_MAX_ITERS ? k - 1 : HQN_MAX_ITERS - 1;
    if (stop) {
        if (threadIdx.x != 0) return;
        ctl->iter_trials[kk] = ctl->trials;
        ctl->trials_total += ctl->trials;
        ctl->iters_total += 1;
        ctl->iter_g[kk] = ctl->g_k;
        set_cond<R>(h.it, 0u);
        return;
    }
    if (push) {
        // dots (thread 0): rho, |s|^2, |t|^2, s_a^T t_w, s_w^T t_a, s_a^T grad
        __shared__ HistSmem hs;
        __shared__ int keep;
        hist_load(ctl, hs, m);
        if (threadIdx.x == 0) {
            keep = dots[0] > 1e-12 * sqrt(dots[1] * dots[2]);
            if (keep) {
                hs.head = w;
                hs.rho[w] = dots[0];
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
    if (threadIdx.x != 0) return;
    ctl->iter_trials[kk] = ctl->trials;
    ctl->trials_total += ctl->trials;
    ctl->iters_total += 1;
    ctl->g_k = ctl->g_trial;
    ctl->e_k = ctl->e_trial;
    ctl->iter_g[kk] = ctl->g_trial;
    ctl->k = k + 1;
    set_cond<R>(h.it, (k + 1 <= s.c.iters) ? 1u : 0u);
}

// q = -grad - sum_p zeta_p t_p (the first loop's result).
template <typename R>
__global__ void __launch_bounds__(VBS) k_q(DevSim<R> s) {
    const Ctl *ctl = s.ctl;
    const int i = blockIdx.x * VBS + threadIdx.x;
    if (i >= s.c.nf) return;
    const int count = ctl->count, head = ctl->head, m = s.c.m;
    const V4<R> g = s.gk[i];
    V4<R> q;
    q.x = -g.x; q.y = -g.y; q.z = -g.z; q.w = R(0);
    for (int p = 0; p < count; ++p) {
        const R z = (R)ctl->zeta[p];
        const V4<R> t = s.Tt[(size_t)ring_slot(head, p, m) * s.c.n + i];
        q.x -= z * t.x; q.y -= z * t.y; q.z -= z * t.z;
    }
    s.q[i] = q;
}

// t_a^T r0 for every ring slot a (r0 = A0^{-1} q, held in d); the last block
// runs the second loop of Alg. 2 on scalars: c_p = zeta_p - eta_p, oldest first.
template <typename R, int MP1>
__global__ void __launch_bounds__(VBS) k_r0_dots(DevSim<R> s) {
    Ctl *ctl = s.ctl;
    const int count = ctl->count, m = s.c.m;
    if (count == 0) return;
    R dr[MP1];
#pragma unroll
    for (int a = 0; a < MP1; ++a) dr[a] = R(0);
    const size_t n = (size_t)s.c.n;
    const int i = blockIdx.x * VBS + threadIdx.x;
    if (i < s.c.nf) {
        const V4<R> r = s.d[i];
#pragma unroll
        for (int a = 0; a < MP1; ++a) {
            if (a > m) break;
            dr[a] = dotr(s.Tt[(size_t)a * n + i], r);
        }
    }
    double dots[MP1];
    block_sum_r<VBS, MP1, R>(dr, dots);
    if (!publish_and_arrive<MP1>(dots, s.part_v, gridDim.x, &ctl->ticket[TK_VEC])) return;
    sum_partials<VBS, MP1>(s.part_v, gridDim.x, gridDim.x, dots, &ctl->ticket[TK_VEC]);
    __shared__ HistSmem hs;
    hist_load(ctl, hs, m);
    if (threadIdx.x == 0) {
#pragma unroll
        for (int a = 0; a < MP1; ++a)
            if (a <= m) hs.tr0[a] = dots[a];
        coef_recursion(hs, m);
    }
    __syncthreads();
    for (int p = threadIdx.x; p < count; p += VBS) ctl->coef[p] = hs.coef[p];
}

// d = r0 + sum_p c_p s_p; then gd = tr(grad_k^T d) -- with history and
// gd >= 0 the direction is not a descent direction: flag it (and set the
// if-node) so the history is dropped -- and the coefficients of the inertia
// term along the ray x_k + alpha d:
// 1/(2h^2) sum m |x_k + alpha d - y|^2 = a0 + a1 alpha + a2 alpha^2.
template <typename R>
__global__ void __launch_bounds__(VBS) k_dir_final(DevSim<R> s, CondHandles h, int set_nd) {
    Ctl *ctl = s.ctl;
    const int i = blockIdx.x * VBS + threadIdx.x;
    R d4[4] = {R(0), R(0), R(0), R(0)};
    if (i < s.c.nf) {
        V4<R> dd = s.d[i];
        const int count = ctl->count, head = ctl->head, m = s.c.m;
        for (int p = 0; p < count; ++p) {
            const R c = (R)ctl->coef[p];
            const V4<R> sv = s.S[(size_t)ring_slot(head, p, m) * s.c.n + i];
            dd.x += c * sv.x; dd.y += c * sv.y; dd.z += c * sv.z;
        }
        if (count > 0) s.d[i] = dd;
        const V4<R> g = s.gk[i], x = s.xk[i], yy = s.y[i];
        const R mh = s.mh2[i];
        const R rx = x.x - yy.x, ry = x.y - yy.y, rz = x.z - yy.z;
        d4[0] = dotr(g, dd);
        d4[1] = R(0.5) * mh * (rx * rx + ry * ry + rz * rz);
        d4[2] = mh * (rx * dd.x + ry * dd.y + rz * dd.z);
        d4[3] = R(0.5) * mh * dotr(dd, dd);
    }
    double tot[4];
    block_sum_r<VBS, 4, R>(d4, tot);
    if (!publish_and_arrive<4>(tot, s.part_v, gridDim.x, &ctl->ticket[TK_VEC])) return;
    sum_partials<VBS, 4>(s.part_v, gridDim.x, gridDim.x, tot, &ctl->ticket[TK_VEC]);
    if (threadIdx.x != 0) return;
    ctl->gd = tot[0];
    ctl->ls_a[0] = tot[1];
    ctl->ls_a[1] = tot[2];
    ctl->ls_a[2] = tot[3];
    const int nd = (tot[0] >= 0.0 && ctl->count > 0) ? 1 : 0;
    ctl->nondescent = nd;
    if (set_nd) set_cond<R>(h.nd, (unsigned)nd);
}

template <typename R>
__global__ void k_reset_history(DevSim<R> s) {
    s.ctl->count = 0;
    s.ctl->nondescent = 0;
}

// q_{l-1} := q_l, q_l := x (end of the time step, Eq. PD).
template <typename R>
__global__ void __launch_bounds__(VBS) k_commit(DevSim<R> s) {
    const int i = blockIdx.x * VBS + threadIdx.x;
    if (i < s.c.n) {
        s.u_prev[i] = s.u_cur[i];
        s.u_cur[i] = s.xk[i];
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        Ctl *c = s.ctl;
        c->steps += 1;
        if (c->status > c->worst_status) c->worst_status = c->status;
    }
}

// Caller-given history (sim_direction): row `a` of the Gram matrix, s_a^T t_b
// for the slots b < count, rho_a = s_a^T t_a and s_a^T grad.  With
// a == count - 1 the last block also runs the first loop on scalars.
template <typename R>
__global__ void __launch_bounds__(VBS) k_hist_row(DevSim<R> s, int a) {
    Ctl *ctl = s.ctl;
    constexpr int NB = HQN_MAX_HISTORY + 2;
    double dots[NB];
#pragma unroll
    for (int b = 0; b < NB; ++b) dots[b] = 0.0;
    const int count = ctl->count;
    const size_t n = (size_t)s.c.n;
    const int i = blockIdx.x * VBS + threadIdx.x;
    if (i < s.c.nf) {
        const V4<R> sa = s.S[(size_t)a * n + i];
#pragma unroll
        for (int b = 0; b < NB - 1; ++b)
            if (b < count) dots[b] = dotv(sa, s.Tt[(size_t)b * n + i]);
        dots[NB - 1] = dotv(sa, s.gk[i]);
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
    hist_load(ctl, hs, s.c.m);
    if (threadIdx.x == 0) {
        for (int b = 0; b < count; ++b) hs.sg[b] = ctl->sg[b];
        zeta_recursion(hs, s.c.m);
    }
    __syncthreads();
    for (int p = threadIdx.x; p < count; p += VBS) ctl->zeta[p] = hs.zeta[p];
}

inline int nblk(int n) { return (n + VBS - 1) / VBS; }

}  // namespace

// ---------------------------------------------------------------- launchers

template <typename R> void launch_predict(const DevSim<R> &s, cudaStream_t st) {
    k_predict<R><<<nblk(s.c.n), VBS, 0, st>>>(s);
}
template <typename R> void launch_inertia(const DevSim<R> &s, cudaStream_t st) {
    k_inertia<R><<<nblk(s.c.n), VBS, 0, st>>>(s);
}
template <typename R> void launch_tet(const DevSim<R> &s, int mode, CondHandles h, cudaStream_t st) {
    const int T = s.c.T;
    switch (s.tet_bs) {
        case 64: k_tet<R, 64><<<(T + 63) / 64, 64, 0, st>>>(s, mode, h); break;
        case 256: k_tet<R, 256><<<(T + 255) / 256, 256, 0, st>>>(s, mode, h); break;
        default: k_tet<R, 128><<<(T + 127) / 128, 128, 0, st>>>(s, mode, h); break;
    }
}
template <typename R> void launch_ls(const DevSim<R> &s, CondHandles h, cudaStream_t st) {
    const int T = s.c.T, nb = (T + 127) / 128;
    switch (s.c.ls_batch) {
        case 1: k_ls<R, 128, 1><<<nb, 128, 0, st>>>(s, h); break;
        case 2: k_ls<R, 128, 2><<<nb, 128, 0, st>>>(s, h); break;
        case 4: k_ls<R, 128, 4><<<nb, 128, 0, st>>>(s, h); break;
        case 16: k_ls<R, 128, 16><<<nb, 128, 0, st>>>(s, h); break;
        default: k_ls<R, 128, 8><<<nb, 128, 0, st>>>(s, h); break;
    }
}
template <typename R> void launch_gather(const DevSim<R> &s, int mode, CondHandles h, cudaStream_t st) {
    const int m = s.c.m;
    const int nb = nblk(s.c.nf);
    if (m <= 0) k_gather<R, 1><<<nb, VBS, 0, st>>>(s, mode, h);
    else if (m <= 3) k_gather<R, 4><<<nb, VBS, 0, st>>>(s, mode, h);
    else if (m <= 5) k_gather<R, 6><<<nb, VBS, 0, st>>>(s, mode, h);
    else if (m <= 8) k_gather<R, 9><<<nb, VBS, 0, st>>>(s, mode, h);
    else k_gather<R, HQN_MAX_HISTORY + 1><<<nb, VBS, 0, st>>>(s, mode, h);
}
template <typename R> void launch_q(const DevSim<R> &s, cudaStream_t st) {
    k_q<R><<<nblk(s.c.nf), VBS, 0, st>>>(s);
}
template <typename R> void launch_r0_dots(const DevSim<R> &s, cudaStream_t st) {
    const int m = s.c.m;
    const int nb = nblk(s.c.nf);
    if (m <= 0) return;
    if (m <= 3) k_r0_dots<R, 4><<<nb, VBS, 0, st>>>(s);
    else if (m <= 5) k_r0_dots<R, 6><<<nb, VBS, 0, st>>>(s);
    else if (m <= 8) k_r0_dots<R, 9><<<nb, VBS, 0, st>>>(s);
    else k_r0_dots<R, HQN_MAX_HISTORY + 1><<<nb, VBS, 0, st>>>(s);
}
template <typename R>
void launch_direction_final(const DevSim<R> &s, CondHandles h, int set_nd, cudaStream_t st) {
    k_dir_final<R><<<nblk(s.c.nf), VBS, 0, st>>>(s, h, set_nd);
}
template <typename R> void launch_reset_history(const DevSim<R> &s, cudaStream_t st) {
    k_reset_history<R><<<1, 1, 0, st>>>(s);
}
template <typename R> void launch_commit(const DevSim<R> &s, cudaStream_t st) {
    k_commit<R><<<nblk(s.c.n), VBS, 0, st>>>(s);
}
template <typename R> void launch_hist_row(const DevSim<R> &s, int a, cudaStream_t st) {
    k_hist_row<R><<<nblk(s.c.nf), VBS, 0, st>>>(s, a);
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
    template void launch_hist_row<R>(const DevSim<R> &, int, cudaStream_t);

HQN_INST(float)
HQN_INST(double)

}  // namespace hqn
