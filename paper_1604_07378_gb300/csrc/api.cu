// C ABI of the solver (include/hqn.h): handle life cycle, state transfer and
// the orchestration of one implicit-Euler step -- Alg. 1 (quasi-Newton
// iterations with backtracking Armijo line search) driving the L-BFGS
// direction of Alg. 2 with the prefactored A0 = M/h^2 + L.
//
// A step runs entirely on the device.  In graph mode it is one CUDA graph:
// a while node over the iterations whose body holds the two-loop recursion,
// the triangular sweeps, an if node for the (rare) non-descent reset and a
// while node over the line-search trials.  Every decision is taken by a
// kernel that sets the conditional handles, so the host launches one graph
// per step and never waits inside it.  Eager mode issues the same kernels
// and reads the control block between them (debugging, graph-less drivers).
#include <cmath>
#include <cstdio>
#include <cstring>
#include <memory>
#include <new>
#include <string>
#include <vector>

#include "kernels.cuh"
#include "layout.hpp"
#include "setup.hpp"

using namespace hqn;

namespace {

thread_local std::string g_last_error;

int fail(int code, const std::string &msg) {
    g_last_error = msg;
    return code;
}

#define CK(call)                                                                              \
    do {                                                                                      \
        cudaError_t e_ = (call);                                                              \
        if (e_ != cudaSuccess)                                                                \
            return fail(HQN_ERR_CUDA, std::string(#call) + ": " + cudaGetErrorString(e_));    \
    } while (0)

// Hermite segment coefficients p0 + u(p1 + u(p2 + u p3)) of one spline function.
template <typename R>
void spline_coeffs(const MaterialHost &m, int f, MatDev<R> &d) {
    for (int i = 0; i < 8; ++i) d.kx[f][i] = (R)m.sx[f][i];
    for (int i = 0; i < 7; ++i) {
        const double h = m.sx[f][i + 1] - m.sx[f][i];
        const double v0 = m.sv[f][i], v1 = m.sv[f][i + 1];
        const double m0 = m.ss[f][i] * h, m1 = m.ss[f][i + 1] * h;
        d.inv_h[f][i] = (R)(1.0 / h);
        d.p[f][i][0] = (R)v0;
        d.p[f][i][1] = (R)m0;
        d.p[f][i][2] = (R)(3.0 * (v1 - v0) - 2.0 * m0 - m1);
        d.p[f][i][3] = (R)(2.0 * (v0 - v1) + m0 + m1);
    }
}

struct SimBase {
    virtual ~SimBase() {}
    virtual int set_state(const double *qc, const double *qp) = 0;
    virtual int get_state(double *qc, double *qp) = 0;
    virtual int step(int nsteps, hqn_step_stats *stats) = 0;
    virtual int energy_grad(const double *x, const double *y, double *g, double *grad) = 0;
    virtual int solve_A0(const double *q, double *r) = 0;
    virtual int direction(const double *grad, int np, const double *s, const double *t, double *d) = 0;
    virtual void info(hqn_info *out) const = 0;
    virtual int time_stage(int stage, int reps, double *ms) = 0;
};

template <typename R>
struct Sim final : SimBase {
    Setup S;
    hqn_params prm{};
    cudaStream_t st = nullptr;
    DevSim<R> ds{};
    DevSolve<R> dsol{};
    std::vector<void *> allocs;
    int64_t dev_bytes = 0;
    Ctl *h_ctl = nullptr;  // pinned
    std::vector<V4<R>> hbuf;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t gexec = nullptr;
    bool graph_mode = false;
    std::vector<cudaStream_t> cap_streams;
    cudaStream_t own_stream = nullptr;

    ~Sim() override {
        if (st) cudaStreamSynchronize(st);
        if (gexec) cudaGraphExecDestroy(gexec);
        if (graph) cudaGraphDestroy(graph);
        for (auto s : cap_streams) cudaStreamDestroy(s);
        for (void *p : allocs) cudaFree(p);
        if (h_ctl) cudaFreeHost(h_ctl);
        if (own_stream) cudaStreamDestroy(own_stream);
    }

    template <typename X>
    int alloc(X *&p, size_t count) {
        p = nullptr;
        if (count == 0) count = 1;
        void *q = nullptr;
        cudaError_t e = cudaMalloc(&q, count * sizeof(X));
        if (e != cudaSuccess) return fail(HQN_ERR_NO_MEMORY, std::string("cudaMalloc: ") + cudaGetErrorString(e));
        allocs.push_back(q);
        dev_bytes += (int64_t)(count * sizeof(X));
        p = (X *)q;
        CK(cudaMemsetAsync(q, 0, count * sizeof(X), st));
        return HQN_OK;
    }
    template <typename X>
    int upload(const X *&p, const X *src, size_t count) {
        X *q = nullptr;
        int rc = alloc(q, count);
        if (rc) return rc;
        if (count) CK(cudaMemcpyAsync(q, src, count * sizeof(X), cudaMemcpyHostToDevice, st));
        p = q;
        return HQN_OK;
    }

    int init(const hqn_params &p, cudaStream_t stream) {
        prm = p;
        st = stream;
        const int n = S.n, T = S.T, nf = S.n_free, m = p.history_m;
        if (!solve_smem_limit_ok<R>(S.max_ld))
            return fail(HQN_ERR_UNSUPPORTED, "a separator is too large for the sweeps' shared memory");
        CK(solve_prepare<R>());
        if (st == nullptr) {  // the legacy default stream cannot be captured: use an own stream
            CK(cudaStreamCreateWithFlags(&own_stream, cudaStreamNonBlocking));
            st = own_stream;
        }
        StepConst<R> &c = ds.c;
        c.n = n; c.nf = nf; c.T = T; c.m = m; c.iters = p.iters; c.ls_max = p.ls_max;
        c.ls_batch = (p.ls_batch == 1 || p.ls_batch == 2 || p.ls_batch == 4 || p.ls_batch == 16) ? p.ls_batch : 8;
        c.h2 = (R)(p.h * p.h);
        c.gx = (R)(p.h * p.h * p.gravity[0]);
        c.gy = (R)(p.h * p.h * p.gravity[1]);
        c.gz = (R)(p.h * p.h * p.gravity[2]);
        c.gamma = p.gamma;
        c.backtrack = p.backtrack;
        ds.tet_bs = (p.tet_block == 64 || p.tet_block == 256) ? p.tet_block : 128;
        // material
        MatDev<R> &M = ds.mat;
        std::memset(&M, 0, sizeof(M));
        M.kind = S.mat.kind;
        M.mu = (R)S.mat.mu; M.lam = (R)S.mat.lam;
        M.J0 = (R)S.mat.J0; M.c0 = (R)S.mat.c0; M.c1 = (R)S.mat.c1; M.c2 = (R)S.mat.c2;
        if (S.mat.kind == HQN_SPLINE_VL)
            for (int f = 0; f < 3; ++f) spline_coeffs(S.mat, f, M);
        int rc;
        // mesh data
        std::vector<int4> tets(T);
        for (int t = 0; t < T; ++t) tets[t] = make_int4(S.tets[4 * t], S.tets[4 * t + 1], S.tets[4 * t + 2], S.tets[4 * t + 3]);
        const int4 *dt;
        if ((rc = upload(dt, tets.data(), T))) return rc;
        ds.tets = dt;
        std::vector<R> dm((size_t)9 * T);
        for (int t = 0; t < T; ++t)
            for (int e = 0; e < 9; ++e) dm[(size_t)e * T + t] = (R)S.dminv[(size_t)9 * t + e];
        const R *p_dm;
        if ((rc = upload(p_dm, dm.data(), dm.size()))) return rc;
        ds.dminv = p_dm;
        std::vector<R> vol(T), mh2(n);
        for (int t = 0; t < T; ++t) vol[t] = (R)S.vol[t];
        for (int i = 0; i < n; ++i) mh2[i] = (R)(S.mass[i] / (p.h * p.h));
        const R *p_vol, *p_mh2;
        if ((rc = upload(p_vol, vol.data(), T))) return rc;
        if ((rc = upload(p_mh2, mh2.data(), n))) return rc;
        ds.vol = p_vol; ds.mh2 = p_mh2;
        std::vector<int> slot(S.vt_slot.size());
        for (size_t k = 0; k < slot.size(); ++k) {
            const int sv = S.vt_slot[k];
            slot[k] = (sv & 3) * T + (sv >> 2);
        }
        const int *p_ptr, *p_slot;
        if ((rc = upload(p_ptr, S.vt_ptr.data(), S.vt_ptr.size()))) return rc;
        if ((rc = upload(p_slot, slot.data(), slot.size()))) return rc;
        ds.vt_ptr = p_ptr; ds.vt_slot = p_slot;
        // vectors
        V4<R> **vecs[] = {&ds.u_cur, &ds.u_prev, &ds.y, &ds.xk, &ds.xt, &ds.gk, &ds.d, &ds.q, &ds.z};
        for (auto v : vecs)
            if ((rc = alloc(*v, n))) return rc;
        const size_t ring = (size_t)(m + 1) * n;
        if ((rc = alloc(ds.S, m > 0 ? ring : 1))) return rc;
        if ((rc = alloc(ds.Tt, m > 0 ? ring : 1))) return rc;
        if ((rc = alloc(ds.corner, (size_t)4 * T))) return rc;
        const int nbv = (n + VBS - 1) / VBS, nbf = (nf + VBS - 1) / VBS, nbt = (T + 63) / 64;
        if ((rc = alloc(ds.part_in, nbv))) return rc;
        if ((rc = alloc(ds.part_el, nbt))) return rc;
        // per-block partials: up to 3 + 3 (m + 1) sums (gather with a history
        // push), m + 2 (caller-given history rows), m + 1 or 4 (direction)
        if ((rc = alloc(ds.part_g, (size_t)(3 + 3 * (HQN_MAX_HISTORY + 1)) * nbf))) return rc;
        if ((rc = alloc(ds.part_v, (size_t)(HQN_MAX_HISTORY + 1) * nbf))) return rc;
        if ((rc = alloc(ds.part_ls, (size_t)16 * ((T + 127) / 128)))) return rc;
        if ((rc = alloc(ds.ctl, 1))) return rc;
        CK(cudaMallocHost(&h_ctl, sizeof(Ctl)));
        // solve operators
        dsol.nf = nf;
        dsol.n_levels = S.n_levels;
        // the two packed copies of every Q_s (layout.hpp): forward row-major,
        // backward transposed
        std::vector<R> QF((size_t)S.qf_total, R(0)), QB((size_t)S.qb_total, R(0));
        for (const SupernodeHost &sn : S.sn) {
            const double *Qs = S.Q.data() + sn.qoff;
            const int nc = sn.ncol, rows = sn.ncol + sn.nrow;
            for (int i = 0; i < rows; ++i) {
                R *dst = QF.data() + sn.qf + fwd_row_off(i, nc, sn.ldc);
                const int len = std::min(fwd_row_len(i, nc, sn.ldc), nc);
                for (int j = 0; j < len; ++j) dst[j] = (R)Qs[(size_t)i * nc + j];
            }
            for (int j = 0; j < nc; ++j) {
                R *dst = QB.data() + sn.qb + bwd_row_off(j, sn.ldr);
                const int i0 = bwd_row_start(j);
                for (int i = i0; i < rows; ++i) dst[i - i0] = (R)Qs[(size_t)i * nc + j];
            }
        }
        const R *p_QF, *p_QB;
        if ((rc = upload(p_QF, QF.data(), QF.size()))) return rc;
        if ((rc = upload(p_QB, QB.data(), QB.size()))) return rc;
        std::vector<R>().swap(QF);
        std::vector<R>().swap(QB);
        dsol.QF = p_QF;
        dsol.QB = p_QB;
        const int *p_rows;
        const int2 *p_fg2, *p_ug2;
        if ((rc = upload(p_rows, S.rows.data(), S.rows.size()))) return rc;
        if ((rc = upload(p_fg2, reinterpret_cast<const int2 *>(S.fg2.data()), S.fg2.size() / 2))) return rc;
        if ((rc = upload(p_ug2, reinterpret_cast<const int2 *>(S.ug2.data()), S.ug2.size() / 2))) return rc;
        dsol.rows = p_rows; dsol.fg2 = p_fg2; dsol.ug2 = p_ug2;
        // work-item records (kernels.cuh): everything a block needs in one place
        std::vector<int4> fi(3 * S.fwd_items.size()), bi(3 * S.bwd_items.size());
        for (size_t k = 0; k < S.fwd_items.size(); ++k) {
            const FwdItem &f = S.fwd_items[k];
            const SupernodeHost &sn = S.sn[f.s];
            const int64_t o0 = fwd_row_off(f.row0, sn.ncol, sn.ldc), o1 = fwd_row_off(f.row1, sn.ncol, sn.ldc);
            const int64_t q0 = sn.qf + o0;
            fi[3 * k] = make_int4((int)(q0 & 0xffffffffLL), (int)(q0 >> 32), (int)((o1 - o0) * sizeof(R)), f.G);
            fi[3 * k + 1] = make_int4(sn.col, sn.ncol, sn.ldc, sn.uoff);
            fi[3 * k + 2] = make_int4(f.row0, f.row1, fwd_row_len(f.row1 - 1, sn.ncol, sn.ldc), (int)o0);
        }
        for (size_t k = 0; k < S.bwd_items.size(); ++k) {
            const BwdItem &b = S.bwd_items[k];
            const SupernodeHost &sn = S.sn[b.s];
            const int64_t o0 = bwd_row_off(b.col0, sn.ldr), o1 = bwd_row_off(b.col1, sn.ldr);
            const int64_t q0 = sn.qb + o0;
            bi[3 * k] = make_int4((int)(q0 & 0xffffffffLL), (int)(q0 >> 32), (int)((o1 - o0) * sizeof(R)), b.G);
            bi[3 * k + 1] = make_int4(sn.col, sn.ncol, sn.nrow, sn.roff);
            bi[3 * k + 2] = make_int4(b.col0, b.col1, sn.ldr, (int)o0);
        }
        const int4 *p_fi, *p_bi;
        if ((rc = upload(p_fi, fi.data(), fi.size()))) return rc;
        if ((rc = upload(p_bi, bi.data(), bi.size()))) return rc;
        dsol.fwd_items = p_fi; dsol.bwd_items = p_bi;
        dsol.fwd_lvl_ptr = S.fwd_lvl_ptr.data();
        dsol.bwd_lvl_ptr = S.bwd_lvl_ptr.data();
        dsol.fwd_lvl_ld = S.fwd_lvl_ld.data();
        dsol.bwd_lvl_ld = S.bwd_lvl_ld.data();
        dsol.fwd_lvl_q = S.fwd_lvl_q.data();
        dsol.bwd_lvl_q = S.bwd_lvl_q.data();
        dsol.err = &ds.ctl->solve_err;
        if ((rc = alloc(dsol.u, (size_t)S.n_upd))) return rc;
        hbuf.resize(n);
        CK(cudaStreamSynchronize(st));
        // graph
        // Chain the sweep levels with programmatic dependent launch when the
        // device and the runtime accept it (one probe solve on zero vectors),
        // and keep it in the graph only if the graph builds with it.
        dsol.pdl = 1;
        launch_solve(dsol, ds.q, ds.z, ds.d, st);
        if (cudaGetLastError() != cudaSuccess || cudaStreamSynchronize(st) != cudaSuccess) {
            cudaGetLastError();
            dsol.pdl = 0;
        }
        graph_mode = false;
        if (p.use_graph) {
            rc = build_graph();
            if (rc != HQN_OK && dsol.pdl) {
                abort_graph();
                dsol.pdl = 0;
                rc = build_graph();
            }
            if (rc != HQN_OK) {
                abort_graph();
                return rc;
            }
            graph_mode = true;
        }
        return HQN_OK;
    }

    // Ends any capture a failed build_graph left open and drops the graph.
    void abort_graph() {
        std::vector<cudaStream_t> ss = cap_streams;
        ss.push_back(st);
        for (cudaStream_t s : ss) {
            cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
            if (cudaStreamIsCapturing(s, &cs) == cudaSuccess && cs != cudaStreamCaptureStatusNone) {
                cudaGraph_t g = nullptr;
                cudaStreamEndCapture(s, &g);
                if (g && g != graph) cudaGraphDestroy(g);
            }
        }
        cudaGetLastError();
        if (gexec) { cudaGraphExecDestroy(gexec); gexec = nullptr; }
        if (graph) { cudaGraphDestroy(graph); graph = nullptr; }
    }

    // ---- state transfer (caller order, absolute positions <-> internal displacements)
    int put_vec(V4<R> *dst, const double *src, bool displacement, bool free_only) {
        const int n = S.n;
        for (int i = 0; i < n; ++i) {
            const int v = S.perm[i];
            V4<R> o;
            o.w = R(0);
            if (free_only && i >= S.n_free) {
                o.x = o.y = o.z = R(0);
            } else {
                double a[3];
                for (int k = 0; k < 3; ++k) {
                    a[k] = src[3 * (size_t)v + k];
                    if (!std::isfinite(a[k])) return fail(HQN_ERR_NONFINITE, "non-finite input");
                    if (displacement) a[k] -= S.X[3 * (size_t)i + k];
                }
                o.x = (R)a[0]; o.y = (R)a[1]; o.z = (R)a[2];
            }
            hbuf[i] = o;
        }
        CK(cudaMemcpyAsync(dst, hbuf.data(), (size_t)n * sizeof(V4<R>), cudaMemcpyHostToDevice, st));
        CK(cudaStreamSynchronize(st));
        return HQN_OK;
    }
    int get_vec(const V4<R> *src, double *dst, bool displacement, bool free_only) {
        const int n = S.n;
        CK(cudaMemcpyAsync(hbuf.data(), src, (size_t)n * sizeof(V4<R>), cudaMemcpyDeviceToHost, st));
        CK(cudaStreamSynchronize(st));
        for (int i = 0; i < n; ++i) {
            const int v = S.perm[i];
            const V4<R> o = hbuf[i];
            double a[3] = {(double)o.x, (double)o.y, (double)o.z};
            if (free_only && i >= S.n_free) a[0] = a[1] = a[2] = 0.0;
            for (int k = 0; k < 3; ++k)
                dst[3 * (size_t)v + k] = a[k] + (displacement ? S.X[3 * (size_t)i + k] : 0.0);
        }
        return HQN_OK;
    }

    int set_state(const double *qc, const double *qp) override {
        int rc = put_vec(ds.u_cur, qc, true, false);
        if (rc) return rc;
        return put_vec(ds.u_prev, qp ? qp : qc, true, false);
    }
    int get_state(double *qc, double *qp) override {
        int rc = HQN_OK;
        if (qc && (rc = get_vec(ds.u_cur, qc, true, false))) return rc;
        if (qp && (rc = get_vec(ds.u_prev, qp, true, false))) return rc;
        return HQN_OK;
    }

    int read_ctl() {
        CK(cudaMemcpyAsync(h_ctl, ds.ctl, sizeof(Ctl), cudaMemcpyDeviceToHost, st));
        CK(cudaStreamSynchronize(st));
        if (h_ctl->solve_err) return fail(HQN_ERR_CUDA, "a triangular sweep's bulk copy did not complete in time");
        return HQN_OK;
    }

    // ---- pieces of the step
    void enqueue_direction(CondHandles h, int set_nd, cudaStream_t s) {
        launch_q(ds, s);
        launch_solve(dsol, ds.q, ds.z, ds.d, s);
        launch_r0_dots(ds, s);
        launch_direction_final(ds, h, set_nd, s);
    }
    void enqueue_reset_direction(cudaStream_t s) {
        launch_reset_history(ds, s);
        launch_q(ds, s);
        launch_solve(dsol, ds.q, ds.z, ds.d, s);
        launch_direction_final(ds, CondHandles{0, 0, 0}, 0, s);
    }
    void enqueue_start(CondHandles h, cudaStream_t s) {
        launch_predict(ds, s);
        launch_inertia(ds, s);
        launch_tet(ds, TET_INIT, CondHandles{0, 0, 0}, s);
        launch_gather(ds, G_INIT, h, s);
    }
    // x_{k+1} = x_k + alpha d: its gradient (corners, unless the fused first
    // trial already left them, then the gather with the history push) once the
    // line search has accepted alpha.
    void enqueue_accept(CondHandles h, cudaStream_t s) {
        launch_tet(ds, TET_GRAD, CondHandles{0, 0, 0}, s);
        launch_gather(ds, G_ITER, h, s);
    }

    int step_eager() {
        const CondHandles none{0, 0, 0};
        int rc;
        enqueue_start(none, st);
        for (int it = 0; it < prm.iters; ++it) {
            enqueue_direction(none, 0, st);
            if ((rc = read_ctl())) return rc;
            if (h_ctl->nondescent) enqueue_reset_direction(st);
            launch_tet(ds, TET_TRIAL1, none, st);
            if ((rc = read_ctl())) return rc;
            for (int pass = 0; pass < prm.ls_max && !h_ctl->accepted && !h_ctl->stop; ++pass) {
                launch_ls(ds, none, st);
                if ((rc = read_ctl())) return rc;
            }
            enqueue_accept(none, st);
            if ((rc = read_ctl())) return rc;
            if (h_ctl->stop) break;
        }
        launch_commit(ds, st);
        CK(cudaGetLastError());
        return HQN_OK;
    }

    cudaStream_t cap_stream(size_t i) {
        while (cap_streams.size() <= i) {
            cudaStream_t s = nullptr;
            cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking);
            cap_streams.push_back(s);
        }
        return cap_streams[i];
    }

    // Adds a conditional node after the current capture frontier of `s` and
    // returns its body graph; the capture of `s` continues after the node.
    int add_conditional(cudaStream_t s, cudaGraphConditionalHandle hnd, cudaGraphConditionalNodeType type,
                        cudaGraph_t *body) {
        cudaStreamCaptureStatus cs;
        cudaGraph_t g = nullptr;
        const cudaGraphNode_t *deps = nullptr;
        size_t ndeps = 0;
        CK(cudaStreamGetCaptureInfo(s, &cs, nullptr, &g, &deps, nullptr, &ndeps));
        if (cs != cudaStreamCaptureStatusActive) return fail(HQN_ERR_CUDA, "stream is not capturing");
        cudaGraphNodeParams np = {cudaGraphNodeTypeConditional};
        np.conditional.handle = hnd;
        np.conditional.type = type;
        np.conditional.size = 1;
        cudaGraphNode_t node;
        CK(cudaGraphAddNode(&node, g, deps, nullptr, ndeps, &np));
        *body = np.conditional.phGraph_out[0];
        CK(cudaStreamUpdateCaptureDependencies(s, &node, nullptr, 1, cudaStreamSetCaptureDependencies));
        return HQN_OK;
    }

    int build_graph() {
        int rc;
        CK(cudaGraphCreate(&graph, 0));
        CK(cudaStreamBeginCaptureToGraph(st, graph, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal));
        cudaGraphConditionalHandle h_it, h_ls, h_nd;
        CK(cudaGraphConditionalHandleCreate(&h_it, graph, 0, 0));
        enqueue_start(CondHandles{(unsigned long long)h_it, 0, 0}, st);
        cudaGraph_t body_it;
        if ((rc = add_conditional(st, h_it, cudaGraphCondTypeWhile, &body_it))) return rc;
        {
            cudaStream_t s1 = cap_stream(0);
            CK(cudaStreamBeginCaptureToGraph(s1, body_it, nullptr, nullptr, 0, cudaStreamCaptureModeRelaxed));
            CK(cudaGraphConditionalHandleCreate(&h_ls, body_it, 0, 0));
            CK(cudaGraphConditionalHandleCreate(&h_nd, body_it, 0, 0));
            const CondHandles H{(unsigned long long)h_it, (unsigned long long)h_ls, (unsigned long long)h_nd};
            enqueue_direction(H, 1, s1);
            cudaGraph_t body_nd;
            if ((rc = add_conditional(s1, h_nd, cudaGraphCondTypeIf, &body_nd))) return rc;
            {
                cudaStream_t s2 = cap_stream(1);
                CK(cudaStreamBeginCaptureToGraph(s2, body_nd, nullptr, nullptr, 0, cudaStreamCaptureModeRelaxed));
                enqueue_reset_direction(s2);
                CK(cudaStreamEndCapture(s2, &body_nd));
            }
            launch_tet(ds, TET_TRIAL1, H, s1);
            cudaGraph_t body_ls;
            if ((rc = add_conditional(s1, h_ls, cudaGraphCondTypeWhile, &body_ls))) return rc;
            {
                cudaStream_t s2 = cap_stream(1);
                CK(cudaStreamBeginCaptureToGraph(s2, body_ls, nullptr, nullptr, 0, cudaStreamCaptureModeRelaxed));
                launch_ls(ds, H, s2);
                CK(cudaStreamEndCapture(s2, &body_ls));
            }
            enqueue_accept(H, s1);
            CK(cudaStreamEndCapture(s1, &body_it));
        }
        launch_commit(ds, st);
        cudaGraph_t out = nullptr;
        CK(cudaStreamEndCapture(st, &out));
        CK(cudaGraphInstantiate(&gexec, graph, 0));
        CK(cudaGraphUpload(gexec, st));
        CK(cudaStreamSynchronize(st));
        return HQN_OK;
    }

    int step(int nsteps, hqn_step_stats *stats) override {
        if (nsteps < 0) return fail(HQN_ERR_ARG, "negative step count");
        CK(cudaMemsetAsync(&ds.ctl->trials_total, 0, 5 * sizeof(int), st));
        for (int k = 0; k < nsteps; ++k) {
            if (graph_mode) {
                CK(cudaGraphLaunch(gexec, st));
            } else {
                int rc = step_eager();
                if (rc) return rc;
            }
        }
        int rc = read_ctl();
        if (rc) return rc;
        const Ctl &c = *h_ctl;
        if (stats) {
            std::memset(stats, 0, sizeof(*stats));
            stats->steps = c.steps;
            stats->iters = c.stop ? c.k : c.k - 1;
            stats->status = c.worst_status;
            stats->trials_total = c.trials_total;
            stats->iters_total = c.iters_total;
            for (int i = 0; i < HQN_MAX_ITERS; ++i) {
                stats->trials[i] = c.iter_trials[i];
                stats->g[i] = c.iter_g[i];
            }
            stats->g0 = c.g0;
            stats->ls_passes_total = c.passes_total;
        }
        if (nsteps > 0 && !std::isfinite(c.g_k)) return fail(HQN_ERR_NONFINITE, "objective is not finite");
        return c.worst_status;
    }

    int energy_grad(const double *x, const double *y, double *g, double *grad) override {
        int rc;
        if ((rc = put_vec(ds.xt, x, true, false))) return rc;
        if ((rc = put_vec(ds.y, y, true, false))) return rc;
        const CondHandles none{0, 0, 0};
        launch_inertia(ds, st);
        launch_tet(ds, TET_EVAL, none, st);
        launch_gather(ds, G_EVAL, none, st);
        CK(cudaGetLastError());
        if ((rc = read_ctl())) return rc;
        if (g) *g = h_ctl->g_trial;
        if (grad) {
            // clamped rows of gk are never written: they stay zero
            if ((rc = get_vec(ds.gk, grad, false, true))) return rc;
        }
        return HQN_OK;
    }

    int solve_A0(const double *q, double *r) override {
        int rc;
        if ((rc = put_vec(ds.q, q, false, true))) return rc;
        launch_solve(dsol, ds.q, ds.z, ds.d, st);
        CK(cudaGetLastError());
        if ((rc = read_ctl())) return rc;
        return get_vec(ds.d, r, false, true);
    }

    int direction(const double *grad, int np, const double *s, const double *t, double *d) override {
        const int m = prm.history_m, n = S.n;
        if (np < 0 || np > m) return fail(HQN_ERR_ARG, "npairs out of range");
        int rc;
        if ((rc = put_vec(ds.gk, grad, false, true))) return rc;
        for (int i = 0; i < np; ++i) {
            if ((rc = put_vec(ds.S + (size_t)i * n, s + (size_t)i * 3 * n, false, true))) return rc;
            if ((rc = put_vec(ds.Tt + (size_t)i * n, t + (size_t)i * 3 * n, false, true))) return rc;
        }
        int hc[2] = {np, np > 0 ? np - 1 : 0};
        CK(cudaMemcpyAsync(&ds.ctl->count, &hc[0], sizeof(int), cudaMemcpyHostToDevice, st));
        CK(cudaMemcpyAsync(&ds.ctl->head, &hc[1], sizeof(int), cudaMemcpyHostToDevice, st));
        for (int a = 0; a < np; ++a) launch_hist_row(ds, a, st);
        enqueue_direction(CondHandles{0, 0, 0}, 0, st);
        CK(cudaGetLastError());
        if ((rc = read_ctl())) return rc;
        return get_vec(ds.d, d, false, true);
    }

    int time_stage(int stage, int reps, double *ms) override {
        if (reps <= 0 || stage < HQN_STAGE_TET || stage > HQN_STAGE_TWO_LOOP)
            return fail(HQN_ERR_ARG, "bad stage or repetition count");
        const CondHandles none{0, 0, 0};
        auto launch = [&]() {
            switch (stage) {
                case HQN_STAGE_TET: launch_tet(ds, TET_EVAL, none, st); break;
                case HQN_STAGE_GATHER: launch_gather(ds, G_EVAL, none, st); break;
                case HQN_STAGE_SOLVE: launch_solve(dsol, ds.q, ds.z, ds.d, st); break;
                case HQN_STAGE_LS_PASS: launch_ls(ds, none, st); break;
                default: enqueue_direction(none, 0, st); break;
            }
        };
        launch();  // warm-up
        cudaEvent_t e0, e1;
        CK(cudaEventCreate(&e0));
        CK(cudaEventCreate(&e1));
        CK(cudaEventRecord(e0, st));
        for (int k = 0; k < reps; ++k) launch();
        CK(cudaEventRecord(e1, st));
        CK(cudaEventSynchronize(e1));
        float t = 0.f;
        CK(cudaEventElapsedTime(&t, e0, e1));
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
        CK(cudaGetLastError());
        *ms = (double)t / reps;
        return HQN_OK;
    }

    void info(hqn_info *o) const override {
        o->n_verts = S.n;
        o->n_tets = S.T;
        o->n_free = S.n_free;
        o->n_supernodes = (int)S.sn.size();
        o->n_levels = S.n_levels;
        o->factor_entries = (int64_t)S.Q.size();
        o->factor_nnz = S.factor_nnz;
        o->stiffness_k = S.k;
        o->setup_seconds = S.setup_seconds;
        o->device_bytes = dev_bytes;
        o->precision = (int)(sizeof(R) == 4 ? HQN_FP32_MIXED : HQN_FP64_PLAIN);
        o->graph_mode = graph_mode ? 1 : 0;
        o->n_update_entries = S.n_upd;
        o->chained_sweeps = dsol.pdl;
    }
};

}  // namespace

namespace hqn {
// Sets the message hqn_last_error() reports (for entry points in other files).
void set_last_error(const char *msg) { g_last_error = msg; }
}  // namespace hqn

struct sim_handle {
    std::unique_ptr<SimBase> impl;
};

extern "C" {

void hqn_default_params(hqn_params *p) {
    if (!p) return;
    std::memset(p, 0, sizeof(*p));
    p->h = 1.0 / 30.0;
    p->gamma = 0.3;
    p->backtrack = 0.5;
    p->x_start = 0.5;
    p->x_end = 1.5;
    p->gravity[0] = 0.0;
    p->gravity[1] = 0.0;
    p->gravity[2] = -9.81;
    p->iters = 10;
    p->history_m = 5;
    p->ls_max = 30;
    p->precision = HQN_FP32_MIXED;
    p->leaf_size = 64;
    p->use_graph = 1;
    p->tet_block = 128;
    p->ls_batch = 8;
}

int sim_create(const hqn_mesh *mesh, const hqn_material *material, const hqn_params *params, void *stream,
               sim_handle **out) {
    if (!out) return fail(HQN_ERR_ARG, "null output pointer");
    *out = nullptr;
    if (!mesh || !material || !params) return fail(HQN_ERR_ARG, "null argument");
    if (params->precision != HQN_FP32_MIXED && params->precision != HQN_FP64_PLAIN)
        return fail(HQN_ERR_ARG, "unknown precision");
    try {
        std::unique_ptr<SimBase> impl;
        Setup *S = nullptr;
        if (params->precision == HQN_FP32_MIXED) {
            auto *p = new Sim<float>();
            impl.reset(p);
            S = &p->S;
        } else {
            auto *p = new Sim<double>();
            impl.reset(p);
            S = &p->S;
        }
        std::string err;
        int rc = build_setup(*mesh, *material, *params, *S, err);
        if (rc != HQN_OK) return fail(rc, err);
        cudaStream_t st = (cudaStream_t)stream;
        if (params->precision == HQN_FP32_MIXED) rc = static_cast<Sim<float> *>(impl.get())->init(*params, st);
        else rc = static_cast<Sim<double> *>(impl.get())->init(*params, st);
        if (rc != HQN_OK) return rc;
        auto *h = new sim_handle;
        h->impl = std::move(impl);
        *out = h;
        return HQN_OK;
    } catch (const std::bad_alloc &) {
        return fail(HQN_ERR_NO_MEMORY, "host allocation failed");
    } catch (const std::exception &e) {
        return fail(HQN_ERR_ARG, e.what());
    }
}

int sim_set_state(sim_handle *sim, const double *q_cur, const double *q_prev) {
    if (!sim || !q_cur) return fail(HQN_ERR_ARG, "null argument");
    try { return sim->impl->set_state(q_cur, q_prev); } catch (...) { return fail(HQN_ERR_NO_MEMORY, "exception"); }
}

int sim_get_state(sim_handle *sim, double *q_cur, double *q_prev) {
    if (!sim) return fail(HQN_ERR_ARG, "null handle");
    try { return sim->impl->get_state(q_cur, q_prev); } catch (...) { return fail(HQN_ERR_NO_MEMORY, "exception"); }
}

int sim_step(sim_handle *sim, int32_t nsteps, hqn_step_stats *stats) {
    if (!sim) return fail(HQN_ERR_ARG, "null handle");
    try { return sim->impl->step(nsteps, stats); } catch (...) { return fail(HQN_ERR_NO_MEMORY, "exception"); }
}

int sim_energy_grad(sim_handle *sim, const double *x, const double *y, double *g_out, double *grad_out) {
    if (!sim || !x || !y) return fail(HQN_ERR_ARG, "null argument");
    try { return sim->impl->energy_grad(x, y, g_out, grad_out); } catch (...) { return fail(HQN_ERR_NO_MEMORY, "exception"); }
}

int sim_solve_A0(sim_handle *sim, const double *q, double *r) {
    if (!sim || !q || !r) return fail(HQN_ERR_ARG, "null argument");
    try { return sim->impl->solve_A0(q, r); } catch (...) { return fail(HQN_ERR_NO_MEMORY, "exception"); }
}

int sim_direction(sim_handle *sim, const double *grad, int32_t npairs, const double *s, const double *t,
                  double *d) {
    if (!sim || !grad || !d || (npairs > 0 && (!s || !t))) return fail(HQN_ERR_ARG, "null argument");
    try { return sim->impl->direction(grad, npairs, s, t, d); } catch (...) { return fail(HQN_ERR_NO_MEMORY, "exception"); }
}

int sim_time_stage(sim_handle *sim, int32_t stage, int32_t reps, double *ms) {
    if (!sim || !ms) return fail(HQN_ERR_ARG, "null argument");
    try { return sim->impl->time_stage(stage, reps, ms); } catch (...) { return fail(HQN_ERR_NO_MEMORY, "exception"); }
}

int sim_get_info(const sim_handle *sim, hqn_info *info) {
    if (!sim || !info) return fail(HQN_ERR_ARG, "null argument");
    std::memset(info, 0, sizeof(*info));
    sim->impl->info(info);
    return HQN_OK;
}

void sim_destroy(sim_handle *sim) { delete sim; }

const char *sim_strerror(int code) {
    switch (code) {
        case HQN_OK: return "ok";
        case HQN_WARN_LS_EXHAUSTED: return "line search exhausted";
        case HQN_WARN_NONDESCENT: return "non-descent direction";
        case HQN_ERR_ARG: return "invalid argument";
        case HQN_ERR_DEGENERATE_TET: return "degenerate or inverted rest tetrahedron";
        case HQN_ERR_NONFINITE: return "non-finite value";
        case HQN_ERR_NOT_SPD: return "A0 is not positive definite";
        case HQN_ERR_CUDA: return "CUDA error";
        case HQN_ERR_NO_MEMORY: return "out of memory";
        case HQN_ERR_UNSUPPORTED: return "unsupported option";
        default: return "unknown status";
    }
}

const char *hqn_last_error(void) { return g_last_error.c_str(); }

}  // extern "C"
