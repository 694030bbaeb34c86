// C ABI of the solver (include/hqn.h): handle life cycle, state transfer and
// the orchestration of one implicit-Euler step -- Alg. 1 (quasi-Newton
// iterations with backtracking Armijo line search) driving the L-BFGS
// direction of Alg. 2 with the prefactored A0 = M/h^2 + L.
//
// A handle holds a batch of independent simulations (sim_create makes a
// batch of one).  Their meshes, factors and states sit back to back in device
// memory, and every kernel stage runs once over the whole batch.
//
// A step runs entirely on the device.  In graph mode it is one CUDA graph:
// a while node over the iterations whose body holds the two-loop recursion,
// the triangular sweeps, an if node for the (rare) non-descent reset and a
// while node over the line-search passes.  Each simulation's decisions are
// taken by kernels on the device, and the last simulation to decide sets the
// conditional handles, so the host launches one graph per step and never
// waits inside it.  Eager mode issues the same kernels and reads the control
// blocks between them (debugging, graph-less drivers).
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <memory>
#include <new>
#include <string>
#include <vector>

#include "kernels.cuh"
#include "layout.hpp"
#include "matdev_host.hpp"
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

struct SimBase {
    virtual ~SimBase() {}
    virtual int count() const = 0;
    virtual int set_state(int idx, const double *qc, const double *qp) = 0;
    virtual int get_state(int idx, double *qc, double *qp) = 0;
    virtual int step(int nsteps, hqn_step_stats *stats) = 0;
    virtual int stats_of(int idx, hqn_step_stats *stats) = 0;
    virtual int energy_grad(const double *x, const double *y, double *g, double *grad) = 0;
    virtual int solve_A0(const double *q, double *r) = 0;
    virtual int direction(const double *grad, int np, const double *s, const double *t, double *d) = 0;
    virtual void info(hqn_info *out) const = 0;
    virtual int time_stage(int stage, int reps, double *ms) = 0;
    virtual int positions_device(void **ptr, int32_t *layout) = 0;
};

template <typename R>
struct Sim final : SimBase {
    std::vector<Setup> S;  // one set-up per simulation
    int ns = 0;            // simulations in the batch
    hqn_params prm{};
    cudaStream_t st = nullptr;
    DevSim<R> ds{};
    DevSolve<R> dsol{};
    std::vector<SimDesc<R>> hdesc;
    std::vector<void *> allocs;
    int64_t dev_bytes = 0;
    Ctl *d_ctl = nullptr;  // ns control blocks (device)
    Ctl *h_ctl = nullptr;  // ns control blocks (pinned host copy)
    std::vector<int> fwd_ptr, fwd_ld, fwd_q, bwd_start, bwd_cnt, bwd_ld, bwd_q;  // per tree level
    int pipe_nbund[2] = {0, 0};  // bundles of the pipelined forward / backward sweeps
    int pipe_ndep[2] = {0, 0};   // cross-block waits of the pipelined forward / backward sweeps
    V4<R> *hbuf = nullptr;  // pinned staging buffer of the state transfers (largest simulation)
    const int *d_perm0 = nullptr;  // simulation 0's caller ids by internal vertex (sim_positions_device)
    V4<R> *d_pos0 = nullptr;       // its positions in caller order, borrowed by the caller
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t gexec = nullptr;
    bool graph_mode = false;
    std::vector<cudaStream_t> cap_streams;
    cudaStream_t own_stream = nullptr;
    int64_t n_tot = 0, T_tot = 0, nf_tot = 0, sn_tot = 0, q_entries = 0, nnz_tot = 0, upd_tot = 0;
    int n_levels = 0;
    double setup_seconds = 0.0;

    ~Sim() override {
        if (st) cudaStreamSynchronize(st);
        if (gexec) cudaGraphExecDestroy(gexec);
        if (graph) cudaGraphDestroy(graph);
        for (auto s : cap_streams) cudaStreamDestroy(s);
        for (void *p : allocs) cudaFree(p);
        if (h_ctl) cudaFreeHost(h_ctl);
        if (hbuf) cudaFreeHost(hbuf);
        if (own_stream) cudaStreamDestroy(own_stream);
    }

    int count() const override { return ns; }

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
        if (prm.direction == 1) prm.history_m = 0;  // the Chebyshev direction keeps no history
        st = stream;
        ns = (int)S.size();
        const int m = prm.history_m;
        int max_ld = 0;
        for (const Setup &s : S) max_ld = std::max(max_ld, s.max_ld);
        if (!solve_smem_limit_ok<R>(max_ld))
            return fail(HQN_ERR_UNSUPPORTED, "a separator is too large for the sweeps' shared memory");
        CK(solve_prepare<R>());
        if (st == nullptr) {  // the legacy default stream cannot be captured: use an own stream
            CK(cudaStreamCreateWithFlags(&own_stream, cudaStreamNonBlocking));
            st = own_stream;
        }
        int rc;
        // ---- batch layout: offsets of every simulation
        std::vector<int> v0(ns), t0(ns), vb0(ns), tb0(ns), u0(ns), sn0(ns);
        std::vector<int64_t> qf0(ns), qb0(ns);
        int nvb = 0, ntb = 0;
        n_tot = T_tot = nf_tot = sn_tot = q_entries = nnz_tot = upd_tot = 0;
        int64_t qf_tot = 0, qb_tot = 0;
        n_levels = 0;
        setup_seconds = 0.0;
        for (int k = 0; k < ns; ++k) {
            const Setup &s = S[k];
            v0[k] = (int)n_tot; t0[k] = (int)T_tot; vb0[k] = nvb; tb0[k] = ntb;
            u0[k] = (int)upd_tot; sn0[k] = (int)sn_tot; qf0[k] = qf_tot; qb0[k] = qb_tot;
            n_tot += s.n; T_tot += s.T; nf_tot += s.n_free; sn_tot += (int64_t)s.sn.size();
            upd_tot += s.n_upd; qf_tot += s.qf_total; qb_tot += s.qb_total;
            q_entries += (int64_t)s.Q.size(); nnz_tot += s.factor_nnz;
            nvb += (s.n + VBS - 1) / VBS;
            ntb += (s.T + TBS - 1) / TBS;
            n_levels = std::max(n_levels, s.n_levels);
            setup_seconds += s.setup_seconds;
        }
        if (n_tot > 0x7fffffffLL / 4 || T_tot > 0x7fffffffLL / 4 || upd_tot > 0x7fffffffLL)
            return fail(HQN_ERR_UNSUPPORTED, "the batch is too large for 32-bit indices");
        const int n = (int)n_tot, T = (int)T_tot;
        ds.nsims = ns; ds.m = m; ds.nvb = nvb; ds.ntb = ntb; ds.Tn = T;
        ds.ls_batch = (p.ls_batch == 1 || p.ls_batch == 2 || p.ls_batch == 4 || p.ls_batch == 16) ? p.ls_batch : 8;
        // ---- mesh data
        {
            std::vector<int4> tets(T);
            std::vector<R> dm((size_t)9 * T), vol(T), mh2(n);
            std::vector<V4<R>> rest(n);
            std::vector<int> vptr(n + 1, 0), cpos((size_t)4 * T, -1);
            int npos = 0;
            for (int k = 0; k < ns; ++k) {
                const Setup &s = S[k];
                for (int t = 0; t < s.T; ++t) {
                    const int *tv = &s.tets[4 * (size_t)t];
                    tets[t0[k] + t] = make_int4(v0[k] + tv[0], v0[k] + tv[1], v0[k] + tv[2], v0[k] + tv[3]);
                    for (int e = 0; e < 9; ++e) dm[(size_t)e * T + t0[k] + t] = (R)s.dminv[(size_t)9 * t + e];
                    vol[t0[k] + t] = (R)s.vol[t];
                }
                for (int i = 0; i < s.n; ++i) {
                    mh2[v0[k] + i] = (R)(s.mass[i] / (p.h * p.h));
                    V4<R> &X = rest[v0[k] + i];
                    X.x = (R)s.X[3 * (size_t)i]; X.y = (R)s.X[3 * (size_t)i + 1]; X.z = (R)s.X[3 * (size_t)i + 2];
                    X.w = R(0);
                    for (int e = s.vt_ptr[i]; e < s.vt_ptr[i + 1]; ++e) {
                        const int sv = s.vt_slot[e];
                        cpos[(size_t)(sv & 3) * T + t0[k] + (sv >> 2)] = npos++;
                    }
                    vptr[v0[k] + i + 1] = npos;
                }
            }
            const int4 *p_t;
            const R *p_dm, *p_vol, *p_mh2;
            const int *p_ptr, *p_pos;
            if (npos != 4 * T || std::find(cpos.begin(), cpos.end(), -1) != cpos.end())
                return fail(HQN_ERR_ARG, "a tet corner is missing from the vertex incidence lists");
            if ((rc = upload(p_t, tets.data(), tets.size()))) return rc;
            if ((rc = upload(p_dm, dm.data(), dm.size()))) return rc;
            if ((rc = upload(p_vol, vol.data(), vol.size()))) return rc;
            if ((rc = upload(p_mh2, mh2.data(), mh2.size()))) return rc;
            if ((rc = upload(p_ptr, vptr.data(), vptr.size()))) return rc;
            if ((rc = upload(p_pos, cpos.data(), cpos.size()))) return rc;
            const V4<R> *p_rest;
            if ((rc = upload(p_rest, rest.data(), rest.size()))) return rc;
            ds.rest = p_rest;
            ds.tets = p_t; ds.dminv = p_dm; ds.vol = p_vol; ds.mh2 = p_mh2; ds.vt_ptr = p_ptr; ds.corner_pos = p_pos;
        }
        // ---- vectors, rings, partials, control blocks
        V4<R> **vecs[] = {&ds.u_cur, &ds.u_prev, &ds.y, &ds.xk, &ds.xt, &ds.gk, &ds.d, &ds.q, &ds.z};
        for (auto v : vecs)
            if ((rc = alloc(*v, n))) return rc;
        const size_t ring = m > 0 ? (size_t)(m + 1) * n : 1;
        if ((rc = alloc(ds.S, ring))) return rc;
        if ((rc = alloc(ds.Tt, ring))) return rc;
        if ((rc = alloc(ds.corner, (size_t)4 * T))) return rc;
        if (p.direction == 1 && (rc = alloc(ds.xprev, n))) return rc;
        if (p.a0_solver == 1) {
            V4<R> **pv[] = {&ds.pcg_r, &ds.pcg_z, &ds.pcg_p, &ds.pcg_ap};
            for (auto v : pv)
                if ((rc = alloc(*v, n))) return rc;
            std::vector<R> dinv(n, R(0));
            for (int k = 0; k < ns; ++k)
                for (int j = 0; j < S[k].n_free; ++j) dinv[v0[k] + j] = (R)(1.0 / S[k].a0_diag[j]);
            const R *p_dinv;
            if ((rc = upload(p_dinv, dinv.data(), dinv.size()))) return rc;
            ds.pcg_dinv = p_dinv;
        }
        if ((rc = alloc(ds.part_in, nvb))) return rc;
        if ((rc = alloc(ds.part_el, ntb))) return rc;
        // per-block partials: up to 3 + 3 (m + 1) sums (gather with a history
        // push), m + 2 (caller-given history rows), m + 1 or 4 (direction),
        // 16 (line-search pass)
        if ((rc = alloc(ds.part_g, (size_t)(3 + 3 * (HQN_MAX_HISTORY + 1)) * nvb))) return rc;
        if ((rc = alloc(ds.part_v, (size_t)(HQN_MAX_HISTORY + 1) * nvb))) return rc;
        if ((rc = alloc(ds.part_ls, (size_t)16 * ntb))) return rc;
        if ((rc = alloc(ds.batch_ticket, 4))) return rc;
        if ((rc = alloc(d_ctl, ns))) return rc;
        CK(cudaMallocHost(&h_ctl, sizeof(Ctl) * (size_t)ns));
        // ---- descriptors and block tables
        hdesc.assign(ns, SimDesc<R>{});
        std::vector<int> vblk(nvb), tblk(ntb);
        for (int k = 0; k < ns; ++k) {
            const Setup &s = S[k];
            SimDesc<R> &D = hdesc[k];
            std::memset(&D, 0, sizeof(D));
            StepConst<R> &c = D.c;
            c.n = s.n; c.nf = s.n_free; c.T = s.T; c.m = m; c.iters = p.iters; c.ls_max = p.ls_max;
            c.ls_batch = ds.ls_batch;
            c.h2 = (R)(p.h * p.h);
            c.gx = (R)(p.h * p.h * p.gravity[0]);
            c.gy = (R)(p.h * p.h * p.gravity[1]);
            c.gz = (R)(p.h * p.h * p.gravity[2]);
            c.gamma = p.gamma;
            c.backtrack = p.backtrack;
            c.kstiff = (R)s.k;
            c.cheb = p.direction == 1 ? 1 : 0;
            c.cheb_S = p.cheb_S;
            c.cheb_rho2 = p.cheb_rho * p.cheb_rho;
            c.ncol = p.n_colliders;
            c.cscale = (R)p.contact_scale;
            for (int q = 0; q < p.n_colliders; ++q) {
                const hqn_collider &hc = p.colliders[q];
                ColDev<R> &dc = c.col[q];
                dc.kind = hc.kind;
                dc.px = (R)hc.point[0]; dc.py = (R)hc.point[1]; dc.pz = (R)hc.point[2];
                const double nn = std::sqrt(hc.normal[0] * hc.normal[0] + hc.normal[1] * hc.normal[1] +
                                            hc.normal[2] * hc.normal[2]);
                dc.nx = dc.ny = dc.nz = R(0);
                if (hc.kind == HQN_COLLIDER_PLANE || hc.kind == HQN_COLLIDER_TORUS) {
                    dc.nx = (R)(hc.normal[0] / nn); dc.ny = (R)(hc.normal[1] / nn); dc.nz = (R)(hc.normal[2] / nn);
                }
                dc.r = (R)hc.radius;
                dc.ring = hc.kind == HQN_COLLIDER_TORUS ? (R)hc.major_radius : R(0);
            }
            matdev_from_host(s.mat, D.mat);
            D.v0 = v0[k]; D.t0 = t0[k];
            D.vb0 = vb0[k]; D.nvb = (s.n + VBS - 1) / VBS;
            D.tb0 = tb0[k]; D.ntb = (s.T + TBS - 1) / TBS;
            D.ring0 = (long long)(m + 1) * v0[k];
            D.ctl = d_ctl + k;
            for (int b = 0; b < D.nvb; ++b) vblk[D.vb0 + b] = k;
            for (int b = 0; b < D.ntb; ++b) tblk[D.tb0 + b] = k;
        }
        {
            const SimDesc<R> *p_desc;
            const int *p_vb, *p_tb;
            if ((rc = upload(p_desc, hdesc.data(), hdesc.size()))) return rc;
            if ((rc = upload(p_vb, vblk.data(), vblk.size()))) return rc;
            if ((rc = upload(p_tb, tblk.data(), tblk.size()))) return rc;
            ds.desc = p_desc; ds.vblk_sim = p_vb; ds.tblk_sim = p_tb;
            ds.desc0 = hdesc[0];
        }
        if ((rc = init_solve(v0, u0, sn0, qf0, qb0, qf_tot, qb_tot))) return rc;
        {
            int nmax = 1;
            for (const Setup &q : S) nmax = std::max(nmax, q.n);
            CK(cudaMallocHost(&hbuf, (size_t)nmax * sizeof(V4<R>)));
        }
        CK(cudaStreamSynchronize(st));
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

    // The solve operators of every simulation, back to back, with batch
    // offsets baked into the work-item records (kernels.cuh) and the index
    // tables.  Level l of the sweeps holds level l of every simulation's tree.
    // Backward items are stored root level first (the dependency-driven queue
    // order); bwd_start[l] is where tree level l begins.
    int init_solve(const std::vector<int> &v0, const std::vector<int> &u0, const std::vector<int> &sn0,
                   const std::vector<int64_t> &qf0, const std::vector<int64_t> &qb0, int64_t qf_tot, int64_t qb_tot) {
        int rc;
        const int L = n_levels;
        dsol.n_levels = L;
        // the two packed copies of every Q_s (layout.hpp): forward row-major,
        // backward transposed
        {
            std::vector<R> QF((size_t)qf_tot, R(0)), QB((size_t)qb_tot, R(0));
            for (int k = 0; k < ns; ++k)
                for (const SupernodeHost &sn : S[k].sn) {
                    const double *Qs = S[k].Q.data() + sn.qoff;
                    const int nc = sn.ncol, rows = sn.ncol + sn.nrow;
                    for (int i = 0; i < rows; ++i) {
                        R *dst = QF.data() + qf0[k] + sn.qf + fwd_row_off(i, nc, sn.ldc);
                        const int len = std::min(fwd_row_len(i, nc, sn.ldc), nc);
                        for (int j = 0; j < len; ++j) dst[j] = (R)Qs[(size_t)i * nc + j];
                    }
                    for (int j = 0; j < nc; ++j) {
                        R *dst = QB.data() + qb0[k] + sn.qb + bwd_row_off(j, sn.ldr);
                        const int i0 = bwd_row_start(j);
                        for (int i = i0; i < rows; ++i) dst[i - i0] = (R)Qs[(size_t)i * nc + j];
                    }
                }
            const R *p_QF, *p_QB;
            if ((rc = upload(p_QF, QF.data(), QF.size()))) return rc;
            if ((rc = upload(p_QB, QB.data(), QB.size()))) return rc;
            dsol.QF = p_QF;
            dsol.QB = p_QB;
        }
        // the double copies are no longer needed on the host
        for (Setup &s : S) std::vector<double>().swap(s.Q);
        {
            std::vector<int> rows;
            std::vector<int4> fg4, ug4;
            auto quad = [](const std::vector<int> &m, size_t e, int off) {
                auto at = [&](int k) { return m[e + k] >= 0 ? off + m[e + k] : -1; };
                return make_int4(at(0), at(1), at(2), at(3));
            };
            for (int k = 0; k < ns; ++k) {
                const Setup &s = S[k];
                for (int r : s.rows) rows.push_back(v0[k] + r);
                for (size_t e = 0; e < s.fg4.size(); e += 4) fg4.push_back(quad(s.fg4, e, u0[k]));
                for (size_t e = 0; e < s.ug4.size(); e += 4) ug4.push_back(quad(s.ug4, e, u0[k]));
            }
            // fg4 is indexed by batch vertex (free vertices of each simulation
            // come first in its range); pad each simulation to its n vertices
            std::vector<int4> fgv((size_t)n_tot, make_int4(-1, -1, -1, -1));
            size_t e = 0;
            for (int k = 0; k < ns; ++k)
                for (int j = 0; j < S[k].n_free; ++j) fgv[v0[k] + j] = fg4[e++];
            const int *p_rows;
            const int4 *p_fg4, *p_ug4;
            if ((rc = upload(p_rows, rows.data(), rows.size()))) return rc;
            if ((rc = upload(p_fg4, fgv.data(), fgv.size()))) return rc;
            if ((rc = upload(p_ug4, ug4.data(), ug4.size()))) return rc;
            dsol.rows = p_rows; dsol.fg4 = p_fg4; dsol.ug4 = p_ug4;
        }
        // work items by level, every simulation's items of a level together
        std::vector<std::vector<int4>> frec(L), brec(L);
        fwd_ld.assign(L, 0); fwd_q.assign(L, 0); bwd_ld.assign(L, 0); bwd_q.assign(L, 0);
        std::vector<int> nit_f((size_t)sn_tot, 0), nit_b((size_t)sn_tot, 0);
        int cb0 = 0;
        for (int k = 0; k < ns; ++k) {
            const Setup &s = S[k];
            int roff0 = 0;
            for (int kk = 0; kk < k; ++kk) roff0 += (int)S[kk].rows.size();
            if (k > 0) cb0 += S[k - 1].lv.n_bwd_blocks;
            for (const SupernodeHost &sn : s.sn)
                if (sn.children.size() > 4) return fail(HQN_ERR_UNSUPPORTED, "a supernode has more than four children");
            for (int l = 0; l < s.n_levels; ++l) {
                fwd_ld[l] = std::max(fwd_ld[l], s.lv.fwd_lvl_ld[l]);
                fwd_q[l] = std::max(fwd_q[l], s.lv.fwd_lvl_q[l]);
                bwd_ld[l] = std::max(bwd_ld[l], s.lv.bwd_lvl_ld[l]);
                bwd_q[l] = std::max(bwd_q[l], s.lv.bwd_lvl_q[l]);
                for (int e = s.lv.fwd_lvl_ptr[l]; e < s.lv.fwd_lvl_ptr[l + 1]; ++e) {
                    const FwdItem &f = s.lv.fwd_items[e];
                    const SupernodeHost &sn = s.sn[f.s];
                    const int64_t o0 = fwd_row_off(f.row0, sn.ncol, sn.ldc), o1 = fwd_row_off(f.row1, sn.ncol, sn.ldc);
                    const int64_t q0 = qf0[k] + sn.qf + o0;
                    auto &v = frec[l];
                    v.push_back(make_int4((int)(q0 & 0xffffffffLL), (int)(q0 >> 32), (int)((o1 - o0) * sizeof(R)), f.G));
                    v.push_back(make_int4(v0[k] + sn.col, sn.ncol, sn.ldc, u0[k] + sn.uoff));
                    v.push_back(make_int4(f.row0, f.row1, fwd_row_len(f.row1 - 1, sn.ncol, sn.ldc), (int)o0));
                    auto child = [&](size_t i) { return i < sn.children.size() ? sn0[k] + sn.children[i] : -1; };
                    v.push_back(make_int4(child(0), child(1), child(2), child(3)));
                    v.push_back(make_int4(sn0[k] + f.s, 0, 0, 0));
                    nit_f[sn0[k] + f.s]++;
                }
                for (int e = s.lv.bwd_lvl_ptr[l]; e < s.lv.bwd_lvl_ptr[l + 1]; ++e) {
                    const BwdItem &b = s.lv.bwd_items[e];
                    const SupernodeHost &sn = s.sn[b.s];
                    int64_t o0 = bwd_row_off(b.col0, sn.ldr), q0, bytes;
                    if (b.e0 < 0) {  // whole rows: one contiguous block from row col0 on
                        q0 = qb0[k] + sn.qb + o0;
                        bytes = (bwd_row_off(b.col1, sn.ldr) - o0) * (int64_t)sizeof(R);
                    } else {  // a chunk: each row's piece [max(e0, start_j), e1)
                        q0 = qb0[k] + sn.qb;
                        bytes = 0;
                        for (int j = b.col0; j < b.col1; ++j)
                            bytes += std::max(0, b.e1 - std::max(b.e0, bwd_row_start(j))) * (int64_t)sizeof(R);
                    }
                    auto &v = brec[l];
                    v.push_back(make_int4((int)(q0 & 0xffffffffLL), (int)(q0 >> 32), (int)bytes, b.G));
                    v.push_back(make_int4(v0[k] + sn.col, sn.ncol, sn.nrow, roff0 + sn.roff));
                    v.push_back(make_int4(b.col0, b.col1, sn.ldr, (int)o0));
                    v.push_back(make_int4(sn.parent >= 0 ? sn0[k] + sn.parent : -1, sn0[k] + b.s, 0, 0));
                    v.push_back(make_int4(b.e0, b.e1, b.cb >= 0 ? cb0 + b.cb : -1, (b.nch << 16) | b.k));
                    nit_b[sn0[k] + b.s]++;
                }
            }
        }
        std::vector<int4> fi, bi;
        fwd_ptr.assign(L + 1, 0);
        for (int l = 0; l < L; ++l) {
            fwd_ptr[l] = (int)(fi.size() / 5);
            fi.insert(fi.end(), frec[l].begin(), frec[l].end());
        }
        fwd_ptr[L] = (int)(fi.size() / 5);
        bwd_start.assign(L, 0);
        bwd_cnt.assign(L, 0);
        for (int l = L - 1; l >= 0; --l) {
            bwd_start[l] = (int)(bi.size() / 5);
            bwd_cnt[l] = (int)(brec[l].size() / 5);
            bi.insert(bi.end(), brec[l].begin(), brec[l].end());
        }
        int n_cb = 0;
        for (const Setup &s : S) n_cb += s.lv.n_bwd_blocks;
        const int4 *p_fi, *p_bi;
        const int *p_nf, *p_nb;
        if ((rc = upload(p_fi, fi.data(), fi.size()))) return rc;
        if ((rc = upload(p_bi, bi.data(), bi.size()))) return rc;
        if ((rc = upload(p_nf, nit_f.data(), nit_f.size()))) return rc;
        if ((rc = upload(p_nb, nit_b.data(), nit_b.size()))) return rc;
        dsol.fwd_items = p_fi; dsol.bwd_items = p_bi;
        dsol.fwd_nitems = p_nf; dsol.bwd_nitems = p_nb;
        if ((rc = alloc(dsol.fwd_done, (size_t)sn_tot))) return rc;
        if ((rc = alloc(dsol.bwd_done, (size_t)sn_tot))) return rc;
        if ((rc = alloc(dsol.queue, 2))) return rc;
        dsol.n_sn = (int)sn_tot;
        dsol.nf = (int)nf_tot;
        dsol.n_fwd_items = (int)(fi.size() / 5);
        dsol.n_bwd_items = (int)(bi.size() / 5);
        if ((rc = alloc(dsol.part_r, (size_t)std::max(1, dsol.n_bwd_items) * 32))) return rc;
        if ((rc = alloc(dsol.cb_cnt, (size_t)std::max(1, n_cb)))) return rc;
        dsol.fwd_lvl_ptr = fwd_ptr.data();
        dsol.bwd_lvl_start = bwd_start.data();
        dsol.bwd_lvl_cnt = bwd_cnt.data();
        dsol.fwd_lvl_ld = fwd_ld.data();
        dsol.bwd_lvl_ld = bwd_ld.data();
        dsol.fwd_lvl_q = fwd_q.data();
        dsol.bwd_lvl_q = bwd_q.data();
        dsol.fwd_qmax = dsol.fwd_ldmax = dsol.bwd_qmax = dsol.bwd_ldmax = 0;
        for (int l = 0; l < L; ++l) {
            dsol.fwd_qmax = std::max(dsol.fwd_qmax, fwd_q[l]);
            dsol.fwd_ldmax = std::max(dsol.fwd_ldmax, fwd_ld[l]);
            dsol.bwd_qmax = std::max(dsol.bwd_qmax, bwd_q[l]);
            dsol.bwd_ldmax = std::max(dsol.bwd_ldmax, bwd_ld[l]);
        }
        dsol.dyn = 0;
        dsol.dyn_grid = 0;
        dsol.pipe = 0;
        if (prm.dyn_sweeps == 1) {
            dsol.dyn_grid = solve_dyn_grid<R>(dsol);
            dsol.dyn = dsol.dyn_grid > 0 ? 1 : 0;
        } else if (prm.dyn_sweeps == 2) {
            if ((rc = init_pipe(v0, u0, sn0, qf0, qb0))) return rc;
        }
        dsol.err = &d_ctl[0].solve_err;
        if ((rc = alloc(dsol.u, (size_t)std::max<int64_t>(upd_tot, 1)))) return rc;
        return HQN_OK;
    }

    // ---- pipelined schedule (one persistent launch per sweep; solve.cu)
    //
    // Every tree level's items (all simulations) are split over the P blocks
    // in contiguous runs of about equal weight (bytes plus a per-item cost),
    // so a supernode's items stay together and a block's items of
    // consecutive levels tend to be parent and child.  A block's consecutive
    // items of one level form a bundle until it would hold more than half
    // the ring, overflow its vector area (fcap entries), its segments or its
    // chunk column blocks.  A supernode whose items all sit in one block
    // ("owned") needs no completion counter for consumers in that block:
    // the block's own order covers them; counters are kept only where a
    // consumer sits elsewhere.

    struct PipeSweep {  // host copy of one sweep's schedule
        std::vector<int4> items, bund, seg, cmb;
        std::vector<int2> dep, sig;
        std::vector<int> bptr, seg_sn;  // seg_sn: supernode of each segment (checks only)
    };

    // Invariants the pipelined kernels rely on for in-bounds accesses and for
    // progress, checked on the host before anything is uploaded: every item's
    // rows fit one ring slot and its vector entries lie inside its bundle's
    // area; a bundle holds at most half the ring, its items share one tree
    // level and its warp ranges tile the consumer warps; a block's bundles
    // come in sweep order; every producer a bundle reads from is either
    // owned by the same block or waited for, and everything waited for
    // publishes exactly its item count.
    static bool pipe_schedule_ok(bool bwd, const PipeSweep &W, int fcap, int ns, const std::vector<int> &lev,
                                 const std::vector<int> &nit, const std::vector<int> &owner,
                                 const std::vector<int> &gparent, const std::vector<int> &ch_ptr,
                                 const std::vector<int> &ch) {
        const int RN = bwd ? 5 : 4, SN = bwd ? 2 : 1;
        const std::vector<int4> &items = W.items, &bund = W.bund, &seg = W.seg, &cmb = W.cmb;
        const std::vector<int2> &dep = W.dep, &sig = W.sig;
        const std::vector<int> &bptr = W.bptr;
        const int nitems = (int)(items.size() / RN), nb = (int)(bund.size() / 3), nseg = (int)(seg.size() / SN);
        if ((int)W.seg_sn.size() != nseg) return false;
        std::vector<int> published(nit.size(), 0);
        std::vector<char> waited(nit.size(), 0);
        int prev_item_end = 0;
        for (size_t b = 0; b + 1 < bptr.size(); ++b) {
            if (bptr[b] > bptr[b + 1] || bptr[b + 1] > nb) return false;
            int prev_level = bwd ? INT32_MAX : -1;
            for (int q = bptr[b]; q < bptr[b + 1]; ++q) {
                const int4 B0 = bund[3 * (size_t)q], B1 = bund[3 * (size_t)q + 1], B2 = bund[3 * (size_t)q + 2];
                if (B0.x != prev_item_end || B0.y <= B0.x || B0.y > nitems || B0.y - B0.x > ns / 2) return false;
                prev_item_end = B0.y;
                if (B0.z < 0 || B0.w > nseg || B0.w - B0.z < 1 || B0.w - B0.z > PIPE_SEG_MAX) return false;
                if (B1.x < 0 || B1.y > (int)dep.size() || B1.y - B1.x > 512) return false;
                if (B1.z < 0 || B1.w > (int)sig.size() || B1.w - B1.z > 512) return false;
                if (B2.x < 0 || B2.y > (int)(cmb.size() / 2) || B2.y - B2.x > PIPE_CMB_MAX) return false;
                if (B2.z < 1 || B2.z > fcap) return false;
                // segments tile [0, ftot) and share the bundle's level
                int off = 0, level = -1;
                for (int g = B0.z; g < B0.w; ++g) {
                    const int4 sg = bwd ? seg[2 * (size_t)g + 1] : seg[g];
                    const int aoff = bwd ? sg.y : sg.z, len = bwd ? sg.z : sg.w;
                    if (aoff != off || len < 1 || (len & 3) || (aoff & 3)) return false;
                    off += len;
                    const int sn = W.seg_sn[g];
                    if (sn < 0 || sn >= (int)nit.size()) return false;
                    if (level < 0) level = lev[sn];
                    if (lev[sn] != level) return false;
                    // every producer is owned by this block or waited for
                    auto covered = [&](int p) {
                        if (nit[p] == 0 || owner[p] == (int)b) return true;
                        for (int d = B1.x; d < B1.y; ++d)
                            if (dep[d].x == p) return true;
                        return false;
                    };
                    if (bwd) {
                        if (gparent[sn] >= 0 && !covered(gparent[sn])) return false;
                    } else {
                        for (int c = ch_ptr[sn]; c < ch_ptr[sn + 1]; ++c)
                            if (!covered(ch[c])) return false;
                    }
                }
                if (off != B2.z) return false;
                if (bwd ? level > prev_level : level < prev_level) return false;
                prev_level = level;
                for (int g = B1.z; g < B1.w; ++g) {
                    const int2 sgn = sig[g];
                    if (sgn.x < 0 || sgn.x >= (int)nit.size() || sgn.y < 1 || lev[sgn.x] != level) return false;
                    published[sgn.x] += sgn.y;
                }
                for (int g = B1.x; g < B1.y; ++g) {
                    const int2 d = dep[g];
                    if (d.x < 0 || d.x >= (int)nit.size() || d.y != nit[d.x]) return false;
                    if (bwd ? lev[d.x] <= level : lev[d.x] >= level) return false;
                    waited[d.x] = 1;
                }
                int wprev = 0;
                for (int it = B0.x; it < B0.y; ++it) {
                    const int4 a = items[(size_t)RN * it], c = items[(size_t)RN * it + 2], d = items[(size_t)RN * it + 3];
                    if (a.z < 16 || a.z > 32768 || (a.z & 15)) return false;
                    const int64_t q0 = (int64_t)(unsigned)a.x | ((int64_t)a.y << 32);
                    if ((q0 * (int64_t)sizeof(R)) & 15) return false;
                    if (d.z != wprev || d.w <= d.z) return false;
                    wprev = d.w;
                    if (!bwd) {
                        if (d.x < 0 || (d.x & 3) || d.x + c.z > B2.z) return false;
                    } else {
                        const int4 e = items[(size_t)RN * it + 4];
                        const int lw = e.x >= 0 ? e.y - e.x : c.z - bwd_row_start(c.x);
                        if (d.x < 0 || (d.x & 3) || lw < 1 || d.x + lw > B2.z) return false;
                        if (e.x >= 0 && (c.y - c.x) * lw * (int)sizeof(R) > 32768) return false;
                    }
                }
                if (wprev != 16) return false;
            }
        }
        if (prev_item_end != nitems) return false;
        for (size_t q = 0; q < nit.size(); ++q)
            if (waited[q] && published[q] != nit[q]) return false;
        return true;
    }

    int init_pipe(const std::vector<int> &v0, const std::vector<int> &u0, const std::vector<int> &sn0,
                  const std::vector<int64_t> &qf0, const std::vector<int64_t> &qb0) {
        const int L = n_levels;
        int need_max = 2048;
        for (const Setup &s : S) {
            for (const FwdItem &f : s.pp.fwd_items) {
                const SupernodeHost &sn = s.sn[f.s];
                need_max = std::max(need_max, fwd_row_len(f.row1 - 1, sn.ncol, sn.ldc));
            }
            for (const BwdItem &b : s.pp.bwd_items) {
                const SupernodeHost &sn = s.sn[b.s];
                need_max = std::max(need_max, b.e0 >= 0 ? b.e1 - b.e0 : sn.ldr - bwd_row_start(b.col0));
            }
        }
        const int fcap = pad4(need_max);
        int nslots = 0;
        const int P = solve_pipe_grid<R>(fcap, &nslots);
        if (P <= 0) return HQN_OK;  // does not fit: the level schedule stays
        const int bmax = nslots / 2;
        std::vector<int> roff0(ns, 0), cb_off(ns, 0);
        for (int k = 1; k < ns; ++k) {
            roff0[k] = roff0[k - 1] + (int)S[k - 1].rows.size();
            cb_off[k] = cb_off[k - 1] + S[k - 1].pp.n_bwd_blocks;
        }
        const int n_cb = cb_off[ns - 1] + S[ns - 1].pp.n_bwd_blocks;
        // global supernodes: level, parent, children; items per sweep; column blocks
        std::vector<int> lev((size_t)sn_tot, 0), gparent((size_t)sn_tot, -1), ch_ptr((size_t)sn_tot + 1, 0), ch;
        std::vector<int> nit_f((size_t)sn_tot, 0), nit_b((size_t)sn_tot, 0), cb_nch(std::max(1, n_cb), 0),
            cb_slot(std::max(1, n_cb), 0);
        for (int k = 0; k < ns; ++k) {
            for (size_t q = 0; q < S[k].sn.size(); ++q) {
                lev[sn0[k] + q] = S[k].sn[q].level;
                gparent[sn0[k] + q] = S[k].sn[q].parent >= 0 ? sn0[k] + S[k].sn[q].parent : -1;
            }
            for (const FwdItem &f : S[k].pp.fwd_items) nit_f[sn0[k] + f.s]++;
            for (const BwdItem &b : S[k].pp.bwd_items) {
                nit_b[sn0[k] + b.s]++;
                if (b.cb >= 0) cb_nch[cb_off[k] + b.cb] = b.nch;
            }
        }
        for (int64_t q = 0; q < sn_tot; ++q)
            if (gparent[q] >= 0) ch_ptr[gparent[q] + 1]++;
        for (int64_t q = 0; q < sn_tot; ++q) ch_ptr[q + 1] += ch_ptr[q];
        ch.assign((size_t)ch_ptr[sn_tot], 0);
        {
            std::vector<int> fill(ch_ptr.begin(), ch_ptr.end() - 1);
            for (int64_t q = 0; q < sn_tot; ++q)
                if (gparent[q] >= 0) ch[fill[gparent[q]]++] = (int)q;
        }
        int n_slots_part = 0;
        for (int c = 0; c < n_cb; ++c) {
            cb_slot[c] = n_slots_part;
            n_slots_part += cb_nch[c];
        }
        struct Ref {
            int k, i;
            double w;
        };
        auto assign = [&](bool bwd) {
            std::vector<std::vector<Ref>> blk((size_t)P);
            for (int li = 0; li < L; ++li) {
                const int l = bwd ? L - 1 - li : li;
                std::vector<Ref> lv;
                double total = 0.0;
                for (int k = 0; k < ns; ++k) {
                    const ItemLists &it = S[k].pp;
                    if (l >= S[k].n_levels) continue;
                    const std::vector<int> &ptr = bwd ? it.bwd_lvl_ptr : it.fwd_lvl_ptr;
                    for (int i = ptr[l]; i < ptr[l + 1]; ++i) {
                        int64_t ent;
                        if (!bwd) {
                            const FwdItem &f = it.fwd_items[i];
                            const SupernodeHost &sn = S[k].sn[f.s];
                            ent = fwd_row_off(f.row1, sn.ncol, sn.ldc) - fwd_row_off(f.row0, sn.ncol, sn.ldc);
                        } else {
                            const BwdItem &b = it.bwd_items[i];
                            const SupernodeHost &sn = S[k].sn[b.s];
                            ent = b.e0 < 0 ? bwd_row_off(b.col1, sn.ldr) - bwd_row_off(b.col0, sn.ldr)
                                           : (int64_t)(b.col1 - b.col0) * (b.e1 - b.e0);
                        }
                        const double w = (double)ent * sizeof(R) + 2048.0;
                        lv.push_back({k, i, w});
                        total += w;
                    }
                }
                double cum = 0.0;
                for (const Ref &r : lv) {
                    int b = (int)((cum + 0.5 * r.w) / total * P);
                    b = std::min(std::max(b, 0), P - 1);
                    blk[b].push_back(r);
                    cum += r.w;
                }
            }
            return blk;
        };
        // owner[s]: the block holding every item of s (-1: split over blocks)
        auto owners = [&](bool bwd, const std::vector<std::vector<Ref>> &blk) {
            std::vector<int> own((size_t)sn_tot, -2);
            for (int b = 0; b < P; ++b)
                for (const Ref &r : blk[b]) {
                    const int s = sn0[r.k] + (bwd ? S[r.k].pp.bwd_items[r.i].s : S[r.k].pp.fwd_items[r.i].s);
                    own[s] = own[s] == -2 || own[s] == b ? b : -1;
                }
            for (int &o : own)
                if (o == -2) o = -1;
            return own;
        };
        // does s publish a completion counter (a consumer sits elsewhere)?
        auto publishes = [&](bool bwd, int s, const std::vector<int> &own, const std::vector<int> &nit) {
            if (own[s] < 0) return true;
            if (!bwd) {
                const int p = gparent[s];
                return p >= 0 && nit[p] > 0 && own[p] != own[s];
            }
            for (int c = ch_ptr[s]; c < ch_ptr[s + 1]; ++c)
                if (nit[ch[c]] > 0 && own[ch[c]] != own[s]) return true;
            return false;
        };
        auto build = [&](bool bwd, PipeSweep &W, std::vector<int> &own) {
            const std::vector<std::vector<Ref>> blk = assign(bwd);
            own = owners(bwd, blk);
            const std::vector<int> &nit = bwd ? nit_b : nit_f;
            const int RN = bwd ? 5 : 4, SN = bwd ? 2 : 1;
            W.bptr.assign((size_t)P + 1, 0);
            for (int b = 0; b < P; ++b) {
                W.bptr[b] = (int)(W.bund.size() / 3);
                int cur_level = -1, ftot = 0, seg_sn = -1, item0 = 0, seg0 = 0, dep0 = 0, sig0 = 0, cmb0 = 0;
                int last_cb = -1, sig_cur = -1;
                bool open = false;
                auto close = [&]() {
                    if (!open) return;
                    const int i1 = (int)(W.items.size() / RN), m = i1 - item0;
                    // consumer warps per item, in proportion to its bytes (at least one)
                    double tot = 0.0;
                    for (int it = item0; it < i1; ++it) tot += W.items[(size_t)RN * it].z;
                    double cum = 0.0;
                    for (int it = item0; it < i1; ++it) {
                        const int j = it - item0;
                        int4 &d = W.items[(size_t)RN * it + 3];
                        d.z = j + (int)((PIPE_CONS_WARPS - m) * cum / tot);
                        cum += W.items[(size_t)RN * it].z;
                        d.w = it + 1 < i1 ? j + 1 + (int)((PIPE_CONS_WARPS - m) * cum / tot) : PIPE_CONS_WARPS;
                    }
                    W.bund.push_back(make_int4(item0, i1, seg0, (int)(W.seg.size() / SN)));
                    W.bund.push_back(make_int4(dep0, (int)W.dep.size(), sig0, (int)W.sig.size()));
                    W.bund.push_back(make_int4(cmb0, (int)(W.cmb.size() / 2), ftot, 0));
                    open = false;
                };
                for (const Ref &r : blk[b]) {
                    const Setup &s = S[r.k];
                    int gs, start, end, level, nc;
                    const SupernodeHost *snp;
                    const BwdItem *bi = nullptr;
                    const FwdItem *fi = nullptr;
                    if (!bwd) {
                        fi = &s.pp.fwd_items[r.i];
                        snp = &s.sn[fi->s];
                        gs = sn0[r.k] + fi->s;
                        start = 0;
                        end = fwd_row_len(fi->row1 - 1, snp->ncol, snp->ldc);
                    } else {
                        bi = &s.pp.bwd_items[r.i];
                        snp = &s.sn[bi->s];
                        gs = sn0[r.k] + bi->s;
                        start = bi->e0 >= 0 ? bi->e0 : bwd_row_start(bi->col0);
                        end = bi->e0 >= 0 ? bi->e1 : snp->ldr;
                    }
                    const SupernodeHost &sn = *snp;
                    level = sn.level;
                    nc = sn.ncol;
                    const bool chunk = bwd && bi->e0 >= 0 && bi->nch > 1;
                    const int cbg = bwd && bi->cb >= 0 ? cb_off[r.k] + bi->cb : -1;
                    // segment of this supernode: [w0, w0 + len) of its vector
                    auto seg_w0 = [&]() { return bwd ? W.seg.back().x : 0; };
                    auto seg_len = [&]() { return bwd ? W.seg.back().z : W.seg.back().w; };
                    bool same = open && seg_sn == gs && start >= seg_w0();
                    int grow = same ? std::max(0, end - (seg_w0() + seg_len())) : end - start;
                    const bool new_cmb = chunk && !(open && last_cb == cbg);
                    if (!open || level != cur_level || (int)(W.items.size() / RN) - item0 == bmax ||
                        ftot + grow > fcap || (!same && (int)(W.seg.size() / SN) - seg0 == PIPE_SEG_MAX) ||
                        (new_cmb && (int)(W.cmb.size() / 2) - cmb0 == PIPE_CMB_MAX)) {
                        close();
                        open = true;
                        cur_level = level;
                        ftot = 0;
                        item0 = (int)(W.items.size() / RN);
                        seg0 = (int)(W.seg.size() / SN);
                        dep0 = (int)W.dep.size();
                        sig0 = (int)W.sig.size();
                        cmb0 = (int)(W.cmb.size() / 2);
                        last_cb = -1;
                        same = false;
                        grow = end - start;
                    }
                    if (!same) {
                        if (!bwd) {
                            W.seg.push_back(make_int4(v0[r.k] + sn.col, std::min(end, nc), ftot, end));
                        } else {
                            W.seg.push_back(make_int4(v0[r.k] + sn.col, sn.ncol, sn.nrow, roff0[r.k] + sn.roff));
                            W.seg.push_back(make_int4(start, ftot, end - start, 0));
                        }
                        W.seg_sn.push_back(gs);
                        // producers this bundle must wait for (not owned by this block)
                        auto add_dep = [&](int p) {
                            if (nit[p] == 0 || own[p] == b) return;
                            for (int d = dep0; d < (int)W.dep.size(); ++d)
                                if (W.dep[d].x == p) return;
                            W.dep.push_back(make_int2(p, nit[p]));
                        };
                        if (bwd) {
                            if (gparent[gs] >= 0) add_dep(gparent[gs]);
                        } else {
                            for (int c = ch_ptr[gs]; c < ch_ptr[gs + 1]; ++c) add_dep(ch[c]);
                        }
                        sig_cur = -1;
                        if (publishes(bwd, gs, own, nit)) {
                            W.sig.push_back(make_int2(gs, 0));
                            sig_cur = (int)W.sig.size() - 1;
                        }
                        ftot += end - start;
                        seg_sn = gs;
                    } else if (grow > 0) {
                        if (!bwd) {
                            W.seg.back().w += grow;
                            W.seg.back().y = std::min(W.seg.back().w, nc);
                        } else {
                            W.seg.back().z += grow;
                        }
                        ftot += grow;
                    }
                    if (sig_cur >= 0) W.sig[sig_cur].y++;
                    if (chunk) {
                        if (last_cb != cbg) {
                            W.cmb.push_back(make_int4(cbg, 0, cb_slot[cbg], bi->nch));
                            W.cmb.push_back(make_int4(v0[r.k] + sn.col + bi->col0, bi->col1 - bi->col0, 0, 0));
                            last_cb = cbg;
                        }
                        W.cmb[W.cmb.size() - 2].y++;
                    }
                    const int aoff = bwd ? W.seg.back().y + (start - W.seg.back().x) : W.seg.back().z;
                    if (!bwd) {
                        const int64_t o0 = fwd_row_off(fi->row0, nc, sn.ldc), o1 = fwd_row_off(fi->row1, nc, sn.ldc);
                        const int64_t q0 = qf0[r.k] + sn.qf + o0;
                        W.items.push_back(make_int4((int)(q0 & 0xffffffffLL), (int)(q0 >> 32),
                                                    (int)((o1 - o0) * sizeof(R)), fi->G));
                        W.items.push_back(make_int4(v0[r.k] + sn.col, nc, sn.ldc, u0[r.k] + sn.uoff));
                        W.items.push_back(make_int4(fi->row0, fi->row1, end, (int)o0));
                        W.items.push_back(make_int4(aoff, 0, 0, 0));
                    } else {
                        int64_t o0 = bwd_row_off(bi->col0, sn.ldr), q0, bytes;
                        if (bi->e0 < 0) {
                            q0 = qb0[r.k] + sn.qb + o0;
                            bytes = (bwd_row_off(bi->col1, sn.ldr) - o0) * (int64_t)sizeof(R);
                        } else {
                            q0 = qb0[r.k] + sn.qb;
                            bytes = 0;
                            for (int j = bi->col0; j < bi->col1; ++j)
                                bytes += std::max(0, bi->e1 - std::max(bi->e0, bwd_row_start(j))) * (int64_t)sizeof(R);
                        }
                        W.items.push_back(make_int4((int)(q0 & 0xffffffffLL), (int)(q0 >> 32), (int)bytes, bi->G));
                        W.items.push_back(make_int4(v0[r.k] + sn.col, sn.ncol, sn.nrow, roff0[r.k] + sn.roff));
                        W.items.push_back(make_int4(bi->col0, bi->col1, sn.ldr, (int)o0));
                        W.items.push_back(make_int4(aoff, cbg >= 0 ? cb_slot[cbg] : 0, 0, 0));
                        W.items.push_back(make_int4(bi->e0, bi->e1, cbg, (bi->nch << 16) | bi->k));
                    }
                }
                close();
            }
            W.bptr[P] = (int)(W.bund.size() / 3);
        };
        int rc;
        for (int dir = 0; dir < 2; ++dir) {
            const bool bwd = dir == 1;
            PipeSweep W;
            std::vector<int> own;
            build(bwd, W, own);
            if (!pipe_schedule_ok(bwd, W, fcap, nslots, lev, bwd ? nit_b : nit_f, own, gparent, ch_ptr, ch))
                return fail(HQN_ERR_UNSUPPORTED, bwd ? "pipelined backward schedule failed its consistency check"
                                                     : "pipelined forward schedule failed its consistency check");
            const int4 *p_items, *p_bund, *p_seg, *p_cmb = nullptr;
            const int2 *p_dep, *p_sig;
            const int *p_blk;
            if ((rc = upload(p_items, W.items.data(), W.items.size()))) return rc;
            if ((rc = upload(p_bund, W.bund.data(), W.bund.size()))) return rc;
            if ((rc = upload(p_seg, W.seg.data(), W.seg.size()))) return rc;
            if (bwd && (rc = upload(p_cmb, W.cmb.data(), W.cmb.size()))) return rc;
            if ((rc = upload(p_dep, W.dep.data(), W.dep.size()))) return rc;
            if ((rc = upload(p_sig, W.sig.data(), W.sig.size()))) return rc;
            if ((rc = upload(p_blk, W.bptr.data(), W.bptr.size()))) return rc;
            if (!bwd) {
                dsol.pf_items = p_items; dsol.pf_bund = p_bund; dsol.pf_seg = p_seg;
                dsol.pf_dep = p_dep; dsol.pf_sig = p_sig; dsol.pf_blk = p_blk;
            } else {
                dsol.pb_items = p_items; dsol.pb_bund = p_bund; dsol.pb_seg = p_seg; dsol.pb_cmb = p_cmb;
                dsol.pb_dep = p_dep; dsol.pb_sig = p_sig; dsol.pb_blk = p_blk;
            }
            pipe_nbund[dir] = W.bptr[P];
            pipe_ndep[dir] = (int)W.dep.size();
        }
        if ((rc = alloc(dsol.pb_part, (size_t)std::max(1, n_slots_part) * 32))) return rc;
        if ((rc = alloc(dsol.pb_cbc, (size_t)std::max(1, n_cb)))) return rc;
        dsol.pipe = 1;
        dsol.pipe_grid = P;
        dsol.pipe_ns = nslots;
        dsol.pipe_fcap = fcap;
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
    // Host <-> device state transfers through the pinned staging buffer; the
    // conversions (caller order and float64 <-> internal order and R) run on
    // the host's cores for large meshes.
    int put_vec(int idx, V4<R> *dst, const double *src, bool displacement, bool free_only) {
        const Setup &s = S[idx];
        const int n = s.n;
        int bad = 0;
#pragma omp parallel for schedule(static) reduction(| : bad) if (n > 32768)
        for (int i = 0; i < n; ++i) {
            const int v = s.perm[i];
            V4<R> o;
            o.w = R(0);
            if (free_only && i >= s.n_free) {
                o.x = o.y = o.z = R(0);
            } else {
                double a[3];
                for (int k = 0; k < 3; ++k) {
                    a[k] = src[3 * (size_t)v + k];
                    if (!std::isfinite(a[k])) bad = 1;
                    if (displacement) a[k] -= s.X[3 * (size_t)i + k];
                }
                o.x = (R)a[0]; o.y = (R)a[1]; o.z = (R)a[2];
            }
            hbuf[i] = o;
        }
        if (bad) return fail(HQN_ERR_NONFINITE, "non-finite input");
        CK(cudaMemcpyAsync(dst + hdesc[idx].v0, hbuf, (size_t)n * sizeof(V4<R>), cudaMemcpyHostToDevice, st));
        CK(cudaStreamSynchronize(st));
        return HQN_OK;
    }
    int get_vec(int idx, const V4<R> *src, double *dst, bool displacement, bool free_only) {
        const Setup &s = S[idx];
        const int n = s.n;
        CK(cudaMemcpyAsync(hbuf, src + hdesc[idx].v0, (size_t)n * sizeof(V4<R>), cudaMemcpyDeviceToHost, st));
        CK(cudaStreamSynchronize(st));
#pragma omp parallel for schedule(static) if (n > 32768)
        for (int i = 0; i < n; ++i) {
            const int v = s.perm[i];
            const V4<R> o = hbuf[i];
            double a[3] = {(double)o.x, (double)o.y, (double)o.z};
            if (free_only && i >= s.n_free) a[0] = a[1] = a[2] = 0.0;
            for (int k = 0; k < 3; ++k)
                dst[3 * (size_t)v + k] = a[k] + (displacement ? s.X[3 * (size_t)i + k] : 0.0);
        }
        return HQN_OK;
    }

    int set_state(int idx, const double *qc, const double *qp) override {
        if (idx < 0 || idx >= ns) return fail(HQN_ERR_ARG, "simulation index out of range");
        int rc = put_vec(idx, ds.u_cur, qc, true, false);
        if (rc) return rc;
        return put_vec(idx, ds.u_prev, qp ? qp : qc, true, false);
    }
    int positions_device(void **ptr, int32_t *layout) override {
        const Setup &s0 = S[0];
        int rc = HQN_OK;
        if (!d_pos0) {
            if ((rc = upload(d_perm0, s0.perm.data(), (size_t)s0.n))) return rc;
            if ((rc = alloc(d_pos0, (size_t)s0.n))) return rc;
        }
        launch_positions<R>(ds, d_perm0, hdesc[0].v0, s0.n, d_pos0, st);
        CK(cudaGetLastError());
        CK(cudaStreamSynchronize(st));
        *ptr = d_pos0;
        *layout = sizeof(R) == 4 ? HQN_LAYOUT_F32X4 : HQN_LAYOUT_F64X4;
        return HQN_OK;
    }

    int get_state(int idx, double *qc, double *qp) override {
        if (idx < 0 || idx >= ns) return fail(HQN_ERR_ARG, "simulation index out of range");
        int rc = HQN_OK;
        if (qc && (rc = get_vec(idx, ds.u_cur, qc, true, false))) return rc;
        if (qp && (rc = get_vec(idx, ds.u_prev, qp, true, false))) return rc;
        return HQN_OK;
    }

    int read_ctl() {
        CK(cudaMemcpyAsync(h_ctl, d_ctl, sizeof(Ctl) * (size_t)ns, cudaMemcpyDeviceToHost, st));
        CK(cudaStreamSynchronize(st));
        if (h_ctl[0].solve_err) return fail(HQN_ERR_CUDA, "a triangular sweep's device wait did not complete in time");
        return HQN_OK;
    }
    bool any_ctl(bool (*pred)(const Ctl &)) const {
        for (int k = 0; k < ns; ++k)
            if (pred(h_ctl[k])) return true;
        return false;
    }

    // ---- pieces of the step
    // r = A0^{-1} q into d: the factorised solve, or the Jacobi-PCG approximation.
    void enqueue_A0inv(cudaStream_t s) {
        if (prm.a0_solver == 1) launch_pcg(ds, (const V4<R> *)ds.q, ds.d, prm.pcg_iters, s);
        else launch_solve(dsol, ds.q, ds.z, ds.d, s);
    }
    void enqueue_direction(CondHandles h, int set_nd, cudaStream_t s) {
        launch_q(ds, s);
        enqueue_A0inv(s);
        launch_r0_dots(ds, s);
        launch_direction_final(ds, h, set_nd, s);
    }
    void enqueue_reset_direction(cudaStream_t s) {
        launch_reset_history(ds, s);
        launch_q(ds, s);
        enqueue_A0inv(s);
        launch_r0_dots(ds, s);
        launch_direction_final(ds, CondHandles{0, 0, 0}, 0, s);
    }
    void enqueue_start(CondHandles h, cudaStream_t s) {
        launch_predict(ds, s);
        launch_inertia(ds, s);
        launch_tet(ds, TET_INIT, CondHandles{0, 0, 0}, s);
        launch_gather(ds, G_INIT, h, s);
    }
    // x_{k+1} = x_k + alpha d once the line search has accepted alpha: the
    // gather of its gradient with the history push (the corners are left by
    // the fused first trial or by the pass that accepted).
    void enqueue_accept(CondHandles h, cudaStream_t s) { launch_gather(ds, G_ITER, h, s); }
    // One pass of the line search, then the gradient at the accepted point of
    // the simulations this pass accepted.
    void enqueue_ls_pass(CondHandles h, cudaStream_t s) {
        launch_ls(ds, h, s);
        launch_tet(ds, TET_GRAD, CondHandles{0, 0, 0}, s);
    }

    int step_eager() {
        const CondHandles none{0, 0, 0};
        int rc;
        enqueue_start(none, st);
        if ((rc = read_ctl())) return rc;
        for (int it = 0; it < prm.iters && any_ctl([](const Ctl &c) { return c.active != 0; }); ++it) {
            enqueue_direction(none, 0, st);
            if ((rc = read_ctl())) return rc;
            if (any_ctl([](const Ctl &c) { return c.nondescent != 0; })) enqueue_reset_direction(st);
            launch_tet(ds, TET_TRIAL1, none, st);
            if ((rc = read_ctl())) return rc;
            for (int pass = 0; pass < prm.ls_max &&
                               any_ctl([](const Ctl &c) { return c.active && !c.accepted && !c.stop; });
                 ++pass) {
                enqueue_ls_pass(none, st);
                if ((rc = read_ctl())) return rc;
            }
            enqueue_accept(none, st);
            if ((rc = read_ctl())) return rc;
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
                enqueue_ls_pass(H, s2);
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
        for (int k = 0; k < ns; ++k) CK(cudaMemsetAsync(&d_ctl[k].trials_total, 0, 5 * sizeof(int), st));
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
        int worst = HQN_OK;
        for (int k = 0; k < ns; ++k) worst = std::max(worst, h_ctl[k].worst_status);
        if (stats) {
            fill_stats(0, stats);
            stats->status = worst;
            stats->trials_total = stats->iters_total = stats->ls_passes_total = 0;
            for (int k = 0; k < ns; ++k) {
                stats->trials_total += h_ctl[k].trials_total;
                stats->iters_total += h_ctl[k].iters_total;
                stats->ls_passes_total += h_ctl[k].passes_total;
            }
        }
        if (nsteps > 0)
            for (int k = 0; k < ns; ++k)
                if (!std::isfinite(h_ctl[k].g_k))
                    return fail(HQN_ERR_NONFINITE, "objective of simulation " + std::to_string(k) + " is not finite");
        return worst;
    }

    void fill_stats(int idx, hqn_step_stats *stats) const {
        const Ctl &c = h_ctl[idx];
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

    int stats_of(int idx, hqn_step_stats *stats) override {
        if (idx < 0 || idx >= ns) return fail(HQN_ERR_ARG, "simulation index out of range");
        int rc = read_ctl();
        if (rc) return rc;
        fill_stats(idx, stats);
        return HQN_OK;
    }

    // The evaluation entry points act on simulation 0 (the kernels run over
    // the batch; the other simulations' results are not used).
    int energy_grad(const double *x, const double *y, double *g, double *grad) override {
        int rc;
        if ((rc = put_vec(0, ds.xt, x, true, false))) return rc;
        if ((rc = put_vec(0, ds.y, y, true, false))) return rc;
        const CondHandles none{0, 0, 0};
        launch_inertia(ds, st);
        launch_tet(ds, TET_EVAL, none, st);
        launch_gather(ds, G_EVAL, none, st);
        CK(cudaGetLastError());
        if ((rc = read_ctl())) return rc;
        if (g) *g = h_ctl[0].g_trial;
        if (grad) {
            // clamped rows of gk are never written: they stay zero
            if ((rc = get_vec(0, ds.gk, grad, false, true))) return rc;
        }
        return HQN_OK;
    }

    int solve_A0(const double *q, double *r) override {
        int rc;
        if ((rc = put_vec(0, ds.q, q, false, true))) return rc;
        enqueue_A0inv(st);
        CK(cudaGetLastError());
        if ((rc = read_ctl())) return rc;
        return get_vec(0, ds.d, r, false, true);
    }

    int direction(const double *grad, int np, const double *s, const double *t, double *d) override {
        const int m = prm.history_m, n = S[0].n;
        if (np < 0 || np > m) return fail(HQN_ERR_ARG, "npairs out of range");
        int rc;
        if ((rc = put_vec(0, ds.gk, grad, false, true))) return rc;
        V4<R> *S0 = ds.S + hdesc[0].ring0, *T0 = ds.Tt + hdesc[0].ring0;
        for (int i = 0; i < np; ++i) {
            if ((rc = put_vec(0, S0 + (size_t)i * n, s + (size_t)i * 3 * n, false, true))) return rc;
            if ((rc = put_vec(0, T0 + (size_t)i * n, t + (size_t)i * 3 * n, false, true))) return rc;
        }
        // simulation 0 alone iterates, with the caller's pairs: count, head, active
        for (int k = 0; k < ns; ++k) {
            const int v[3] = {k == 0 ? np : 0, k == 0 && np > 0 ? np - 1 : 0, k == 0 ? 1 : 0};
            CK(cudaMemcpyAsync(&d_ctl[k].count, &v[0], sizeof(int), cudaMemcpyHostToDevice, st));
            CK(cudaMemcpyAsync(&d_ctl[k].head, &v[1], sizeof(int), cudaMemcpyHostToDevice, st));
            CK(cudaMemcpyAsync(&d_ctl[k].active, &v[2], sizeof(int), cudaMemcpyHostToDevice, st));
            CK(cudaStreamSynchronize(st));
        }
        for (int a = 0; a < np; ++a) launch_hist_row(ds, a, st, hdesc[0].nvb);
        enqueue_direction(CondHandles{0, 0, 0}, 0, st);
        CK(cudaGetLastError());
        if ((rc = read_ctl())) return rc;
        return get_vec(0, ds.d, d, false, true);
    }

    int time_stage(int stage, int reps, double *ms) override {
        if (reps <= 0 || stage < HQN_STAGE_TET || stage > HQN_STAGE_TWO_LOOP)
            return fail(HQN_ERR_ARG, "bad stage or repetition count");
        const CondHandles none{0, 0, 0};
        auto launch = [&]() {
            switch (stage) {
                case HQN_STAGE_TET: launch_tet(ds, TET_EVAL, none, st); break;
                case HQN_STAGE_GATHER: launch_gather(ds, G_EVAL, none, st); break;
                case HQN_STAGE_SOLVE: enqueue_A0inv(st); break;
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
        o->n_verts = (int32_t)n_tot;
        o->n_tets = (int32_t)T_tot;
        o->n_free = (int32_t)nf_tot;
        o->n_supernodes = (int32_t)sn_tot;
        o->n_levels = n_levels;
        o->factor_entries = q_entries;
        o->factor_nnz = nnz_tot;
        o->stiffness_k = S.empty() ? 0.0 : S[0].k;
        o->setup_seconds = setup_seconds;
        o->device_bytes = dev_bytes;
        o->precision = (int)(sizeof(R) == 4 ? HQN_FP32_MIXED : HQN_FP64_PLAIN);
        o->graph_mode = graph_mode ? 1 : 0;
        o->n_update_entries = upd_tot;
        o->chained_sweeps = dsol.pdl;
        o->sweep_schedule = dsol.pipe ? 2 : dsol.dyn;
        o->n_sims = ns;
    }
};

template <typename R>
int make_batch(int count, const hqn_mesh *meshes, const hqn_material *materials, const hqn_params &prm,
               cudaStream_t st, std::unique_ptr<SimBase> &out) {
    std::unique_ptr<Sim<R>> b(new Sim<R>());
    b->S.resize(count);
    std::vector<int> rcs(count, HQN_OK);
    std::vector<std::string> errs(count);
#pragma omp parallel for schedule(dynamic, 1) if (count > 1)
    for (int k = 0; k < count; ++k) rcs[k] = build_setup(meshes[k], materials[k], prm, b->S[k], errs[k]);
    for (int k = 0; k < count; ++k)
        if (rcs[k] != HQN_OK)
            return fail(rcs[k], count > 1 ? "simulation " + std::to_string(k) + ": " + errs[k] : errs[k]);
    const int rc = b->init(prm, st);
    if (rc != HQN_OK) return rc;
    out = std::move(b);
    return HQN_OK;
}

int create_any(int count, const hqn_mesh *meshes, const hqn_material *materials, const hqn_params *params,
               void *stream, sim_handle **out);

}  // namespace

namespace hqn {
// Sets the message hqn_last_error() reports (for entry points in other files).
void set_last_error(const char *msg) { g_last_error = msg; }
}  // namespace hqn

struct sim_handle {
    std::unique_ptr<SimBase> impl;
};

namespace {

// Checks of the parameters that do not depend on a mesh (HQN_OK or a status
// set through fail()).
int validate_params(const hqn_params *params) {
    if (params->precision != HQN_FP32_MIXED && params->precision != HQN_FP64_PLAIN)
        return fail(HQN_ERR_ARG, "unknown precision");
    if (params->direction != 0 && params->direction != 1) return fail(HQN_ERR_ARG, "unknown direction");
    if (params->direction == 1 && !(params->cheb_rho > 0.0 && params->cheb_rho < 1.0 && params->cheb_S >= 0))
        return fail(HQN_ERR_ARG, "Chebyshev direction needs 0 < cheb_rho < 1 and cheb_S >= 0");
    if (params->a0_solver != 0 && params->a0_solver != 1) return fail(HQN_ERR_ARG, "unknown a0_solver");
    if (params->merge_depths < 0 || (params->merge_depths & (params->merge_depths >> 1)))
        return fail(HQN_ERR_ARG, "merge_depths must be a mask without two adjacent depths");
    if (params->a0_solver == 1 && (params->pcg_iters < 1 || params->pcg_iters > 1000))
        return fail(HQN_ERR_ARG, "pcg_iters must be in [1, 1000]");
    if (params->n_colliders < 0 || params->n_colliders > HQN_MAX_COLLIDERS)
        return fail(HQN_ERR_ARG, "n_colliders out of range");
    if (params->n_colliders > 0 && !(params->contact_scale > 0.0 && std::isfinite(params->contact_scale)))
        return fail(HQN_ERR_ARG, "contact_scale must be positive");
    for (int k = 0; k < params->n_colliders; ++k) {
        const hqn_collider &c = params->colliders[k];
        if (c.kind == HQN_COLLIDER_PLANE) {
            const double nn = c.normal[0] * c.normal[0] + c.normal[1] * c.normal[1] + c.normal[2] * c.normal[2];
            if (!(nn > 0.0) || !std::isfinite(nn)) return fail(HQN_ERR_ARG, "a plane collider needs a nonzero normal");
        } else if (c.kind == HQN_COLLIDER_SPHERE) {
            if (!(c.radius > 0.0) || !std::isfinite(c.radius)) return fail(HQN_ERR_ARG, "a sphere collider needs a positive radius");
        } else if (c.kind == HQN_COLLIDER_TORUS) {
            const double nn = c.normal[0] * c.normal[0] + c.normal[1] * c.normal[1] + c.normal[2] * c.normal[2];
            if (!(nn > 0.0) || !std::isfinite(nn)) return fail(HQN_ERR_ARG, "a torus collider needs a nonzero axis");
            if (!(c.radius > 0.0 && c.radius < c.major_radius) || !std::isfinite(c.major_radius))
                return fail(HQN_ERR_ARG, "a torus collider needs 0 < radius < major_radius");
        } else {
            return fail(HQN_ERR_ARG, "unknown collider kind");
        }
    }
    if (params->tet_block != 0 && params->tet_block != TBS)
        return fail(HQN_ERR_UNSUPPORTED, "tet_block must be 0 or 128");
    const int lb = params->ls_batch;
    if (lb != 0 && lb != 1 && lb != 2 && lb != 4 && lb != 8 && lb != 16)
        return fail(HQN_ERR_ARG, "ls_batch must be 0, 1, 2, 4, 8 or 16");
    return HQN_OK;
}

int create_any(int count, const hqn_mesh *meshes, const hqn_material *materials, const hqn_params *params,
               void *stream, sim_handle **out) {
    if (!out) return fail(HQN_ERR_ARG, "null output pointer");
    *out = nullptr;
    if (count <= 0 || !meshes || !materials || !params) return fail(HQN_ERR_ARG, "null argument or empty batch");
    if (const int rc = validate_params(params)) return rc;
    try {
        std::unique_ptr<SimBase> impl;
        const cudaStream_t st = (cudaStream_t)stream;
        const int rc = params->precision == HQN_FP32_MIXED
                           ? make_batch<float>(count, meshes, materials, *params, st, impl)
                           : make_batch<double>(count, meshes, materials, *params, st, impl);
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

}  // namespace

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
    p->leaf_size = 0;
    p->use_graph = 1;
    p->tet_block = TBS;
    p->ls_batch = 8;
    p->dyn_sweeps = 0;
    p->n_colliders = 0;
    p->contact_scale = 100.0;
    p->a0_solver = 0;
    p->pcg_iters = 15;
    p->direction = 0;
    p->cheb_S = 10;
    p->cheb_rho = 0.99;
    p->merge_depths = 0;
}

int sim_create(const hqn_mesh *mesh, const hqn_material *material, const hqn_params *params, void *stream,
               sim_handle **out) {
    return create_any(1, mesh, material, params, stream, out);
}

int sim_batch_create(int32_t count, const hqn_mesh *meshes, const hqn_material *materials,
                     const hqn_params *params, void *stream, sim_handle **out) {
    return create_any(count, meshes, materials, params, stream, out);
}

int32_t sim_batch_count(const sim_handle *sim) { return sim ? sim->impl->count() : 0; }

int sim_set_state(sim_handle *sim, const double *q_cur, const double *q_prev) {
    if (!sim || !q_cur) return fail(HQN_ERR_ARG, "null argument");
    try { return sim->impl->set_state(0, q_cur, q_prev); } catch (...) { return fail(HQN_ERR_NO_MEMORY, "exception"); }
}

int sim_get_state(sim_handle *sim, double *q_cur, double *q_prev) {
    if (!sim) return fail(HQN_ERR_ARG, "null handle");
    try { return sim->impl->get_state(0, q_cur, q_prev); } catch (...) { return fail(HQN_ERR_NO_MEMORY, "exception"); }
}

int sim_positions_device(sim_handle *sim, void **dev_ptr, int32_t *layout) {
    if (!sim || !dev_ptr || !layout) return fail(HQN_ERR_ARG, "null argument");
    *dev_ptr = nullptr;
    *layout = 0;
    try { return sim->impl->positions_device(dev_ptr, layout); } catch (...) { return fail(HQN_ERR_NO_MEMORY, "exception"); }
}

int sim_batch_set_state(sim_handle *sim, int32_t index, const double *q_cur, const double *q_prev) {
    if (!sim || !q_cur) return fail(HQN_ERR_ARG, "null argument");
    try { return sim->impl->set_state(index, q_cur, q_prev); } catch (...) { return fail(HQN_ERR_NO_MEMORY, "exception"); }
}

int sim_batch_get_state(sim_handle *sim, int32_t index, double *q_cur, double *q_prev) {
    if (!sim) return fail(HQN_ERR_ARG, "null handle");
    try { return sim->impl->get_state(index, q_cur, q_prev); } catch (...) { return fail(HQN_ERR_NO_MEMORY, "exception"); }
}

int sim_batch_get_stats(sim_handle *sim, int32_t index, hqn_step_stats *stats) {
    if (!sim || !stats) return fail(HQN_ERR_ARG, "null argument");
    try { return sim->impl->stats_of(index, stats); } catch (...) { return fail(HQN_ERR_NO_MEMORY, "exception"); }
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

int hqn_analyse(const hqn_mesh *mesh, const hqn_material *material, const hqn_params *params, hqn_info *info) {
    if (!mesh || !material || !params || !info) return fail(HQN_ERR_ARG, "null argument");
    std::memset(info, 0, sizeof(*info));
    if (const int rc = validate_params(params)) return rc;
    try {
        Setup S;
        std::string err;
        const int rc = build_setup(*mesh, *material, *params, S, err);
        if (rc != HQN_OK) return fail(rc, err);
        info->n_verts = S.n;
        info->n_tets = S.T;
        info->n_free = S.n_free;
        info->n_supernodes = (int32_t)S.sn.size();
        info->n_levels = S.n_levels;
        info->factor_entries = (int64_t)S.Q.size();
        info->factor_nnz = S.factor_nnz;
        info->stiffness_k = S.k;
        info->setup_seconds = S.setup_seconds;
        info->precision = params->precision;
        info->graph_mode = params->use_graph ? 1 : 0;
        info->n_update_entries = S.n_upd;
        info->sweep_schedule = params->dyn_sweeps;
        info->n_sims = 1;
        return HQN_OK;
    } catch (const std::bad_alloc &) {
        return fail(HQN_ERR_NO_MEMORY, "host allocation failed");
    } catch (const std::exception &e) {
        return fail(HQN_ERR_ARG, e.what());
    }
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
