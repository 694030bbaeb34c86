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
        c->status = HQN_OK; c->accepted = 0; c->nondescent = 0; c->alpha = 1.0;
    }
}

// ---------------------------------------------------------------- inertia of a given x

// Block partial of the inertia term 1/(2h^2) sum m_v |x_t - y|^2 of Eq. PD at
// the caller-given point x_t (the start of a step, or an evaluation request).
template <typename R>
__global__ void __launch_bounds__(VBS) k_inertia(DevSim<R> s) {
    const int i = blockIdx.x * VBS + threadIdx.x;
    double e[1] = {0.0};
    if (i < s.c.n) {
        const V4<R> x = s.xt[i], yy = s.y[i];
        const R dx = x.x - yy.x, dy = x.y - yy.y, dz = x.z - yy.z;
        e[0] = (double)(R(0.5) * s.mh2[i] * (dx * dx + dy * dy + dz * dz));
    }
    block_sum<VBS, 1>(e);
    if (threadIdx.x == 0) s.part_in[blockIdx.x] = e[0];
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
// corner[c * T + t].  TET_INIT / TET_EVAL: at the point x_t, and the energy
// is reduced too (last block, fixed order, float64, plus the inertia
// partials): TET_INIT sets g(x_1), TET_EVAL reports g.  TET_GRAD: at the
// accepted point x_k + alpha d of the line search, corners only.
template <typename R, int BS>
__global__ void __launch_bounds__(BS) k_tet(DevSim<R> s, int mode) {
    const bool grad_mode = mode == TET_GRAD;
    if (grad_mode && s.ctl->stop) return;
    const R al = grad_mode ? (R)s.ctl->alpha : R(0);
    const int T = s.c.T;
    const int t = blockIdx.x * BS + threadIdx.x;
    double e[1] = {0.0};
    if (t < T) {
        const int4 v = s.tets[t];
        V4<R> x0, x1, x2, x3;
        if (grad_mode) {
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
        if (!grad_mode) e[0] = (double)(vol * tet_psi(s.mat, G));
#pragma unroll
        for (int c = 0; c < 4; ++c) {
            V4<R> o;
            o.x = g[c][0]; o.y = g[c][1]; o.z = g[c][2]; o.w = R(0);
            s.corner[(size_t)c * T + t] = o;
        }
    }
    if (grad_mode) return;
    block_sum<BS, 1>(e);
    if (!publish_and_arrive<1>(e, s.part_el, 0, &s.ctl->ticket[TK_TET])) return;
    double tot[1];
    sum_partials<BS, 1>(s.part_el, 0, gridDim.x, tot, &s.ctl->ticket[TK_TET]);
    double in[1];
    const int nbv = (s.c.n + VBS - 1) / VBS;
    {
        double acc = 0.0;
        for (int i = threadIdx.x; i < nbv; i += BS) acc += __ldcg(s.part_in + i);
        in[0] = acc;
        block_sum<BS, 1>(in);
    }
    if (threadIdx.x != 0) return;
    Ctl *c = s.ctl;
    const double g = tot[0] + in[0];
    c->g_trial = g;
    if (mode == TET_INIT) {
        c->g_k = g;
        c->g0 = g;
        c->accepted = 1;
    }
}

// ---------------------------------------------------------------- line search

// One pass of the backtracking line search of Alg. 1 that evaluates K trial
// step lengths at once: alpha_j = alpha * backtrack^j, j < K.  Each thread
// forms G_k = Du_k Dm^{-1} and G_d = Dd Dm^{-1} once and the energy V Psi of
// G_k + alpha_j G_d for every j (no singular vectors: tet_psi).  The last
// block adds the inertia term, a quadratic in alpha whose coefficients were
// formed with the direction, and runs the Armijo tests in the order of Alg. 1:
// the first alpha_j with g <= g_k + gamma alpha_j tr(grad^T d) is accepted
// (the same choice as testing them one at a time).  Otherwise the next pass
// continues from alpha_K, until ls_max trials in all.
template <typename R, int BS, int K>
__global__ void __launch_bounds__(BS) k_ls(DevSim<R> s, CondHandles h) {
    Ctl *ctl = s.ctl;
    const double a0 = ctl->alpha;
    const double bt = s.c.backtrack;
    const int T = s.c.T;
    const int t = blockIdx.x * BS + threadIdx.x;
    double e[K];
#pragma unroll
    for (int j = 0; j < K; ++j) e[j] = 0.0;
    if (t < T) {
        const int4 v = s.tets[t];
        R Duk[3][3], Dd[3][3], Di[9], Gk[3][3], Gd[3][3];
        edge_diffs(s.xk[v.x], s.xk[v.y], s.xk[v.z], s.xk[v.w], Duk);
        edge_diffs(s.d[v.x], s.d[v.y], s.d[v.z], s.d[v.w], Dd);
        load_dm(s, t, Di);
        def_grad(Duk, Di, Gk);
        def_grad(Dd, Di, Gd);
        const R vol = s.vol[t];
        double a = a0;
#pragma unroll
        for (int j = 0; j < K; ++j) {
            const R al = (R)a;
            R G[3][3];
#pragma unroll
            for (int p = 0; p < 3; ++p)
#pragma unroll
                for (int q = 0; q < 3; ++q) G[p][q] = fma_(al, Gd[p][q], Gk[p][q]);
            e[j] = (double)(vol * tet_psi(s.mat, G));
            a *= bt;
        }
    }
    block_sum<BS, K>(e);
    if (!publish_and_arrive<K>(e, s.part_ls, gridDim.x, &ctl->ticket[TK_LS])) return;
    double tot[K];
    sum_partials<BS, K>(s.part_ls, gridDim.x, gridDim.x, tot, &ctl->ticket[TK_LS]);
    if (threadIdx.x != 0) return;
    double a = a0;
    int tr = ctl->trials;
    ctl->passes_total += 1;
    const double gk = ctl->g_k, slope = s.c.gamma * ctl->gd;
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
        const double g = tot[j] + (c0 + a * (c1 + a * c2));
        if (g <= gk + slope * a) {
            ctl->accepted = 1;
            ctl->alpha = a;
            ctl->g_trial = g;
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

// ---------------------------------------------------------------- gather

// One thread per free vertex: grad g = m (x - y)/h^2 + sum of the vertex's
// corner gradients in a fixed (ascending tet) order -- no atomics.  In
// G_ITER mode the accepted trial becomes x_{k+1}: the pair
// s = x_{k+1} - x_k, t = grad_{k+1} - grad_k is written to the free ring slot
// and kept (last block) if tr(t^T s) > 1e-12 |s| |t|.
template <typename R>
__global__ void __launch_bounds__(VBS) k_gather(DevSim<R> s, int mode, CondHandles h) {
    Ctl *ctl = s.ctl;
    const int m = s.c.m;
    const bool stop = mode == G_ITER && ctl->stop;
    const bool push = mode == G_ITER && m > 0;
    const int w = push ? (ctl->head + 1) % (m + 1) : 0;
    const R al = mode == G_ITER ? (R)ctl->alpha : R(0);
    const int i = blockIdx.x * VBS + threadIdx.x;
    double dots[3] = {0.0, 0.0, 0.0};
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
            const V4<R> xo = s.xk[i], go = s.gk[i];
            if (push) {
                V4<R> sv, tv;
                sv.x = x.x - xo.x; sv.y = x.y - xo.y; sv.z = x.z - xo.z; sv.w = R(0);
                tv.x = gn.x - go.x; tv.y = gn.y - go.y; tv.z = gn.z - go.z; tv.w = R(0);
                s.S[(size_t)w * s.c.n + i] = sv;
                s.Tt[(size_t)w * s.c.n + i] = tv;
                dots[0] = (double)tv.x * sv.x + (double)tv.y * sv.y + (double)tv.z * sv.z;
                dots[1] = (double)sv.x * sv.x + (double)sv.y * sv.y + (double)sv.z * sv.z;
                dots[2] = (double)tv.x * tv.x + (double)tv.y * tv.y + (double)tv.z * tv.z;
            }
            s.xk[i] = x;
        }
        s.gk[i] = gn;
    }
    if (mode == G_EVAL) return;
    block_sum<VBS, 3>(dots);
    if (!publish_and_arrive<3>(dots, s.part_g, gridDim.x, &ctl->ticket[TK_GATHER])) return;
    double tot[3];
    sum_partials<VBS, 3>(s.part_g, gridDim.x, gridDim.x, tot, &ctl->ticket[TK_GATHER]);
    if (threadIdx.x != 0) return;
    if (mode == G_INIT) {
        ctl->k = 1;
        ctl->count = 0;
        ctl->head = 0;
        ctl->g_k = ctl->g_trial;
        set_cond<R>(h.it, s.c.iters > 0 ? 1u : 0u);
        return;
    }
    const int k = ctl->k;
    const int kk = k - 1 < HQN_MAX_ITERS ? k - 1 : HQN_MAX_ITERS - 1;
    ctl->iter_trials[kk] = ctl->trials;
    ctl->trials_total += ctl->trials;
    ctl->iters_total += 1;
    if (stop) {
        ctl->iter_g[kk] = ctl->g_k;
        set_cond<R>(h.it, 0u);
        return;
    }
    if (push && tot[0] > 1e-12 * sqrt(tot[1] * tot[2])) {
        ctl->head = w;
        ctl->rho[w] = tot[0];
        ctl->count = ctl->count < m ? ctl->count + 1 : m;
    }
    ctl->g_k = ctl->g_trial;
    ctl->iter_g[kk] = ctl->g_trial;
    ctl->k = k + 1;
    set_cond<R>(h.it, (k + 1 <= s.c.iters) ? 1u : 0u);
}

// ---------------------------------------------------------------- Alg. 2

// First loop, newest pair first.  p = -1: q = -grad.  p >= 0 (if p < count):
// q -= zeta_p t_p.  Then, if pair p + 1 exists, the partial of tr(s_{p+1}^T q)
// whose final sum (last block) gives zeta_{p+1} = tr(s^T q) / rho.
template <typename R>
__global__ void __launch_bounds__(VBS) k_first(DevSim<R> s, int p) {
    Ctl *ctl = s.ctl;
    const int count = ctl->count, m = s.c.m, head = ctl->head;
    if (p >= count) return;
    const int i = blockIdx.x * VBS + threadIdx.x;
    const bool next = p + 1 < count;
    const int sn = next ? ring_slot(head, p + 1, m) : 0;
    double d1[1] = {0.0};
    if (i < s.c.nf) {
        V4<R> qq;
        if (p < 0) {
            const V4<R> g = s.gk[i];
            qq.x = -g.x; qq.y = -g.y; qq.z = -g.z; qq.w = R(0);
        } else {
            const R zeta = (R)ctl->zeta[p];
            const V4<R> tv = s.Tt[(size_t)ring_slot(head, p, m) * s.c.n + i];
            qq = s.q[i];
            qq.x -= zeta * tv.x; qq.y -= zeta * tv.y; qq.z -= zeta * tv.z;
        }
        s.q[i] = qq;
        if (next) {
            const V4<R> sv = s.S[(size_t)sn * s.c.n + i];
            d1[0] = (double)sv.x * qq.x + (double)sv.y * qq.y + (double)sv.z * qq.z;
        }
    }
    if (!next) return;
    block_sum<VBS, 1>(d1);
    if (!publish_and_arrive<1>(d1, s.part_v, 0, &ctl->ticket[TK_VEC])) return;
    double tot[1];
    sum_partials<VBS, 1>(s.part_v, 0, gridDim.x, tot, &ctl->ticket[TK_VEC]);
    if (threadIdx.x == 0) ctl->zeta[p + 1] = tot[0] / ctl->rho[sn];
}

// Second loop, oldest pair first, on r (held in d).  j = -1: the partial of
// tr(t^T r) for the oldest pair.  j >= 0: pair age p = count - 1 - j:
// r += s_p (zeta_p - eta_p), eta_p = tr(t_p^T r) / rho_p; then the partial
// of tr(t_{p-1}^T r) for the next pair.
template <typename R>
__global__ void __launch_bounds__(VBS) k_second(DevSim<R> s, int j) {
    Ctl *ctl = s.ctl;
    const int count = ctl->count, m = s.c.m, head = ctl->head;
    const int p = j < 0 ? count : count - 1 - j;  // pair applied now (count = none)
    if (p < 0 || (j < 0 && count == 0)) return;
    const int pn = p - 1;  // pair whose inner product is formed next
    const bool next = pn >= 0;
    const int sn = next ? ring_slot(head, pn, m) : 0;
    const int i = blockIdx.x * VBS + threadIdx.x;
    double d1[1] = {0.0};
    if (i < s.c.nf) {
        V4<R> r = s.d[i];
        if (j >= 0) {
            const int sp = ring_slot(head, p, m);
            const R coef = (R)(ctl->zeta[p] - ctl->dot / ctl->rho[sp]);
            const V4<R> sv = s.S[(size_t)sp * s.c.n + i];
            r.x += coef * sv.x; r.y += coef * sv.y; r.z += coef * sv.z;
            s.d[i] = r;
        }
        if (next) {
            const V4<R> tv = s.Tt[(size_t)sn * s.c.n + i];
            d1[0] = (double)tv.x * r.x + (double)tv.y * r.y + (double)tv.z * r.z;
        }
    }
    if (!next) return;
    block_sum<VBS, 1>(d1);
    if (!publish_and_arrive<1>(d1, s.part_v, 0, &ctl->ticket[TK_VEC])) return;
    double tot[1];
    sum_partials<VBS, 1>(s.part_v, 0, gridDim.x, tot, &ctl->ticket[TK_VEC]);
    if (threadIdx.x == 0) ctl->dot = tot[0];
}

// gd = tr(grad_k^T d); with history and gd >= 0 the direction is not a
// descent direction: flag it (and set the if-node) so the history is dropped.
// Also the coefficients of the inertia term along the ray x_k + alpha d:
// 1/(2h^2) sum m |x_k + alpha d - y|^2 = a0 + a1 alpha + a2 alpha^2.
template <typename R>
__global__ void __launch_bounds__(VBS) k_dir_final(DevSim<R> s, CondHandles h, int set_nd) {
    Ctl *ctl = s.ctl;
    const int i = blockIdx.x * VBS + threadIdx.x;
    double d4[4] = {0.0, 0.0, 0.0, 0.0};
    if (i < s.c.nf) {
        const V4<R> g = s.gk[i], dd = s.d[i], x = s.xk[i], yy = s.y[i];
        const double mh = (double)s.mh2[i];
        const double rx = (double)x.x - yy.x, ry = (double)x.y - yy.y, rz = (double)x.z - yy.z;
        d4[0] = (double)g.x * dd.x + (double)g.y * dd.y + (double)g.z * dd.z;
        d4[1] = 0.5 * mh * (rx * rx + ry * ry + rz * rz);
        d4[2] = mh * (rx * dd.x + ry * dd.y + rz * dd.z);
        d4[3] = 0.5 * mh * ((double)dd.x * dd.x + (double)dd.y * dd.y + (double)dd.z * dd.z);
    }
    block_sum<VBS, 4>(d4);
    if (!publish_and_arrive<4>(d4, s.part_v, gridDim.x, &ctl->ticket[TK_VEC])) return;
    double tot[4];
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
__global__ void k_ls_begin(DevSim<R> s, CondHandles h) {
    Ctl *ctl = s.ctl;
    ctl->alpha = 1.0;
    ctl->trials = 0;
    ctl->accepted = 0;
    set_cond<R>(h.ls, 1u);
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

template <typename R>
__global__ void __launch_bounds__(VBS) k_pair_rho(DevSim<R> s, int slot) {
    const int i = blockIdx.x * VBS + threadIdx.x;
    double d1[1] = {0.0};
    if (i < s.c.nf) {
        const V4<R> sv = s.S[(size_t)slot * s.c.n + i], tv = s.Tt[(size_t)slot * s.c.n + i];
        d1[0] = (double)tv.x * sv.x + (double)tv.y * sv.y + (double)tv.z * sv.z;
    }
    block_sum<VBS, 1>(d1);
    if (!publish_and_arrive<1>(d1, s.part_v, 0, &s.ctl->ticket[TK_VEC])) return;
    double tot[1];
    sum_partials<VBS, 1>(s.part_v, 0, gridDim.x, tot, &s.ctl->ticket[TK_VEC]);
    if (threadIdx.x == 0) s.ctl->rho[slot] = tot[0];
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
template <typename R> void launch_tet(const DevSim<R> &s, int mode, cudaStream_t st) {
    const int T = s.c.T;
    switch (s.tet_bs) {
        case 64: k_tet<R, 64><<<(T + 63) / 64, 64, 0, st>>>(s, mode); break;
        case 256: k_tet<R, 256><<<(T + 255) / 256, 256, 0, st>>>(s, mode); break;
        default: k_tet<R, 128><<<(T + 127) / 128, 128, 0, st>>>(s, mode); break;
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
    k_gather<R><<<nblk(s.c.nf), VBS, 0, st>>>(s, mode, h);
}
template <typename R> void launch_first_loop(const DevSim<R> &s, int p, cudaStream_t st) {
    k_first<R><<<nblk(s.c.nf), VBS, 0, st>>>(s, p);
}
template <typename R> void launch_second_loop(const DevSim<R> &s, int j, cudaStream_t st) {
    k_second<R><<<nblk(s.c.nf), VBS, 0, st>>>(s, j);
}
template <typename R>
void launch_direction_final(const DevSim<R> &s, CondHandles h, int set_nd, cudaStream_t st) {
    k_dir_final<R><<<nblk(s.c.nf), VBS, 0, st>>>(s, h, set_nd);
}
template <typename R> void launch_ls_begin(const DevSim<R> &s, CondHandles h, cudaStream_t st) {
    k_ls_begin<R><<<1, 1, 0, st>>>(s, h);
}
template <typename R> void launch_reset_history(const DevSim<R> &s, cudaStream_t st) {
    k_reset_history<R><<<1, 1, 0, st>>>(s);
}
template <typename R> void launch_commit(const DevSim<R> &s, cudaStream_t st) {
    k_commit<R><<<nblk(s.c.n), VBS, 0, st>>>(s);
}
template <typename R> void launch_pair_rho(const DevSim<R> &s, int slot, cudaStream_t st) {
    k_pair_rho<R><<<nblk(s.c.nf), VBS, 0, st>>>(s, slot);
}

#define HQN_INST(R)                                                                  \
    template void launch_predict<R>(const DevSim<R> &, cudaStream_t);                \
    template void launch_inertia<R>(const DevSim<R> &, cudaStream_t);                \
    template void launch_tet<R>(const DevSim<R> &, int, cudaStream_t);               \
    template void launch_ls<R>(const DevSim<R> &, CondHandles, cudaStream_t);        \
    template void launch_gather<R>(const DevSim<R> &, int, CondHandles, cudaStream_t); \
    template void launch_first_loop<R>(const DevSim<R> &, int, cudaStream_t);        \
    template void launch_second_loop<R>(const DevSim<R> &, int, cudaStream_t);       \
    template void launch_direction_final<R>(const DevSim<R> &, CondHandles, int, cudaStream_t); \
    template void launch_ls_begin<R>(const DevSim<R> &, CondHandles, cudaStream_t);  \
    template void launch_reset_history<R>(const DevSim<R> &, cudaStream_t);          \
    template void launch_commit<R>(const DevSim<R> &, cudaStream_t);                 \
    template void launch_pair_rho<R>(const DevSim<R> &, int, cudaStream_t);

HQN_INST(float)
HQN_INST(double)

}  // namespace hqn
