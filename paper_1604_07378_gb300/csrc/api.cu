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
    virtual int energy_grad_device(const double *x, const double *y, double *g, double *grad) = 0;
    virtual int solve_A0(const double *q, double *r) = 0;
    virtual int direction(const double *grad, int np, const double *s, const double *t, double *d) = 0;
    virtual void info(hqn_info *out) const = 0;
    virtual int time_stage(int stage, int reps, double *ms) = 0;
    virtual int positions_device(void **ptr, int32_t *layout) = 0;
    virtual int set_solve_shapes(const hqn_params &shapes) = 0;
};

int check_solve_shapes(const hqn_params &p);

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
    std::vector<void *> plan_allocs;  // device memory of the current sweep plan (work items, prefetch spans)
    std::vector<void *> *alloc_to = &allocs;
    int64_t dev_bytes = 0, plan_bytes = 0;
    // batch offsets of every simulation's vertices, update entries,
    // supernodes and packed operators (kept to re-plan the sweeps)
    std::vector<int> sv0, su0, ssn0;
    std::vector<int64_t> sqf0, sqb0;
    Ctl *d_ctl = nullptr;  // ns control blocks (device)
    Ctl *h_ctl = nullptr;  // ns control blocks (pinned host copy)
    std::vector<int> fwd_ptr, fwd_ld, fwd_q, bwd_start, bwd_cnt, bwd_ld, bwd_q;  // per tree level
    std::vector<int> pf_ptr;  // L2 prefetch spans of each launch of a solve
    V4<R> *hbuf = nullptr;  // pinned staging buffer of the state transfers (largest simulation)
    const int *d_perm0 = nullptr;  // simulation 0's caller ids by internal vertex (sim_positions_device)
    const double *d_X0 = nullptr;  // simulation 0's float64 rest positions, internal order (device evaluation)
    V4<R> *d_pos0 = nullptr;       // its positions in caller order, borrowed by the caller
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t gexec = nullptr;
    bool graph_mode = false;
    std::vector<cudaStream_t> cap_streams;
    cudaStream_t own_stream = nullptr;
    int64_t n_tot = 0, T_tot = 0, nf_tot = 0, sn_tot = 0, q_entries = 0, nnz_tot = 0, upd_tot = 0;
    int n_levels = 0;
    int dense_cols = 0;   // columns of the largest dense top block
    int64_t dense_bytes = 0;  // bytes of the dense top blocks' matrices
    int spans_total = 0;  // L2 prefetch spans of one solve
    double setup_seconds = 0.0;

    ~Sim() override {
        if (st) cudaStreamSynchronize(st);
        if (gexec) cudaGraphExecDestroy(gexec);
        if (graph) cudaGraphDestroy(graph);
        for (auto s : cap_streams) cudaStreamDestroy(s);
        for (void *p : allocs) cudaFree(p);
        for (void *p : plan_allocs) cudaFree(p);
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
        alloc_to->push_back(q);
        dev_bytes += (int64_t)(count * sizeof(X));
        if (alloc_to == &plan_allocs) plan_bytes += (int64_t)(count * sizeof(X));
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
        const int item_kb = std::max(p.solve_item_kb > 0 ? p.solve_item_kb : 64, p.solve_leaf_kb);
        int max_ld = 0;
        for (const Setup &s : S) max_ld = std::max(max_ld, s.max_ld);
        if (solve_block_smem<R>(item_kb * 1024 / (int)sizeof(R), max_ld) > (size_t)SOLVE_MAX_SMEM)
            return fail(HQN_ERR_UNSUPPORTED, "a separator is too large for the sweeps' shared memory");
        CK(solve_prepare<R>());
        if (p.history_m > kShortHist) CK(long_hist_prepare<R>(p.history_m));
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
            // per-tet material indices, only when some mesh has several materials
            bool several = false;
            for (const Setup &q : S) several = several || q.mats.size() > 1;
            ds.tmat = nullptr;
            if (several) {
                std::vector<uint8_t> tm(T, 0);
                for (int k = 0; k < ns; ++k)
                    for (int t = 0; t < S[k].T; ++t) tm[t0[k] + t] = S[k].tmat[t];
                const uint8_t *p_tm;
                if ((rc = upload(p_tm, tm.data(), tm.size()))) return rc;
                ds.tmat = p_tm;
            }
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
        if ((rc = alloc(ds.part_g, (size_t)(3 + 3 * (kShortHist + 1)) * nvb))) return rc;
        if ((rc = alloc(ds.part_v, (size_t)(kShortHist + 1) * nvb))) return rc;
        // a long window: its scalars per simulation, and the partials of its
        // slot products (3 LH_CHUNK per chunk and block)
        double *lh_all = nullptr;
        if (m > kShortHist) {
            const size_t nch = (size_t)(m + 1 + LH_CHUNK - 1) / LH_CHUNK;
            if ((rc = alloc(lh_all, LongHist::doubles(m) * (size_t)ns))) return rc;
            if ((rc = alloc(ds.part_l, nch * 3 * LH_CHUNK * (size_t)nvb))) return rc;
        }
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
            D.n_mats = (int)s.mats.size();
            if (D.n_mats > 1) {
                std::vector<MatDev<R>> md(D.n_mats);
                std::vector<R> km(D.n_mats);
                for (int m = 0; m < D.n_mats; ++m) {
                    matdev_from_host(s.mats[m], md[m]);
                    km[m] = (R)s.kmat[m];
                }
                const MatDev<R> *p_md;
                const R *p_km;
                if ((rc = upload(p_md, md.data(), md.size()))) return rc;
                if ((rc = upload(p_km, km.data(), km.size()))) return rc;
                D.mats = p_md;
                D.kmat = p_km;
            }
            D.v0 = v0[k]; D.t0 = t0[k];
            D.vb0 = vb0[k]; D.nvb = (s.n + VBS - 1) / VBS;
            D.tb0 = tb0[k]; D.ntb = (s.T + TBS - 1) / TBS;
            D.ring0 = (long long)(m + 1) * v0[k];
            D.ctl = d_ctl + k;
            D.lh = lh_all ? lh_all + LongHist::doubles(m) * (size_t)k : nullptr;
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
    // Backward items are stored root level first (launch order); bwd_start[l]
    // is where tree level l begins.
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
        if ((rc = init_dense_top(v0, u0))) return rc;
        sv0 = v0; su0 = u0; ssn0 = sn0; sqf0 = qf0; sqb0 = qb0;
        dsol.err = &d_ctl[0].solve_err;
        if ((rc = alloc(dsol.u, (size_t)std::max<int64_t>(upd_tot, 1)))) return rc;
        return plan_solve();
    }

    // The dense top block of every simulation that has one (Setup::n_top > 0):
    // the lower block triangle of S^{-1} as TS x TS tiles (J <= I), each a
    // contiguous row-major block with rows LDT entries apart, zero past the
    // last row and column; the block's columns and its boundary update
    // entries in batch numbering; one tile record per tile (solve.cu, k_dense).
    int init_dense_top(const std::vector<int> &v0, const std::vector<int> &u0) {
        int rc;
        constexpr int TS = 128;                         // the tile edge of k_dense (solve.cu)
        constexpr int LDT = TS + 16 / (int)sizeof(R);  // its rows, padded by 16 bytes
        std::vector<R> inv;
        std::vector<int> col, bptr, bidx;
        std::vector<int4> tiles;
        int bands = 0, nb_max = 1;
        dense_cols = 0;
        for (int k = 0; k < ns; ++k) {
            Setup &s = S[k];
            const int n = s.n_top;
            if (n == 0) continue;
            dense_cols = std::max(dense_cols, n);
            const int nb = (n + TS - 1) / TS;
            nb_max = std::max(nb_max, nb);
            const int tc0 = (int)col.size(), bp0 = (int)bptr.size();
            for (int i = 0; i < n; ++i) col.push_back(v0[k] + s.top_col[i]);
            const int b0 = (int)bidx.size();
            for (int i = 0; i <= n; ++i) bptr.push_back(b0 + s.top_bptr[i]);
            for (int e : s.top_bidx) bidx.push_back(u0[k] + e);
            for (int I = 0; I < nb; ++I)
                for (int J = 0; J <= I; ++J) {
                    const int64_t off = (int64_t)inv.size();
                    inv.resize(inv.size() + (size_t)TS * LDT, R(0));
                    for (int i = 0; i < TS && I * TS + i < n; ++i)
                        for (int j = 0; j < TS && J * TS + j < n; ++j)
                            inv[off + (size_t)i * LDT + j] = (R)s.top_inv[(size_t)(I * TS + i) * n + J * TS + j];
                    tiles.push_back(make_int4((int)(off & 0xffffffffLL), (int)(off >> 32), I, J));
                    tiles.push_back(make_int4(n, bands, nb, tc0));
                    tiles.push_back(make_int4(bp0, 0, 0, 0));
                }
            bands += nb;
            std::vector<double>().swap(s.top_inv);  // the float64 copy is no longer needed
        }
        dsol.n_dense_tiles = (int)(tiles.size() / 3);
        dsol.dense_nct_max = nb_max;
        {
            int dev = 0;
            CK(cudaGetDevice(&dev));
            CK(cudaDeviceGetAttribute(&dsol.n_sm, cudaDevAttrMultiProcessorCount, dev));
        }
        dense_bytes = (int64_t)inv.size() * (int64_t)sizeof(R);
        if (dsol.n_dense_tiles == 0) return HQN_OK;
        const int4 *p_t;
        const R *p_inv;
        const int *p_col, *p_bptr, *p_bidx;
        if ((rc = upload(p_t, tiles.data(), tiles.size()))) return rc;
        if ((rc = upload(p_inv, inv.data(), inv.size()))) return rc;
        if ((rc = upload(p_col, col.data(), col.size()))) return rc;
        if ((rc = upload(p_bptr, bptr.data(), bptr.size()))) return rc;
        if ((rc = upload(p_bidx, bidx.data(), bidx.size()))) return rc;
        dsol.dense_tiles = p_t;
        dsol.dense_inv = p_inv;
        dsol.dense_col = p_col;
        dsol.dense_bptr = p_bptr;
        dsol.dense_bidx = p_bidx;
        if ((rc = alloc(dsol.dense_part, (size_t)bands * nb_max * TS))) return rc;
        if ((rc = alloc(dsol.dense_cnt, (size_t)bands))) return rc;
        return HQN_OK;
    }

    // The sweeps' work items and prefetch spans from every simulation's
    // plan (Setup::lv), and the shapes of hqn_params.solve_*.  Runs again
    // when the shapes change (set_solve_shapes); the factor stays.
    int plan_solve() {
        int rc;
        const int L = n_levels;
        const std::vector<int> &v0 = sv0, &u0 = su0, &sn0 = ssn0;
        const std::vector<int64_t> &qf0 = sqf0, &qb0 = sqb0;
        if (st) cudaStreamSynchronize(st);
        for (void *q : plan_allocs) cudaFree(q);
        plan_allocs.clear();
        dev_bytes -= plan_bytes;
        plan_bytes = 0;
        alloc_to = &plan_allocs;
        struct Restore {
            std::vector<void *> *&a;
            std::vector<void *> *v;
            ~Restore() { a = v; }
        } restore{alloc_to, &allocs};
        // work items by level, every simulation's items of a level together
        std::vector<std::vector<int4>> frec(L), brec(L);
        fwd_ld.assign(L, 0); fwd_q.assign(L, 0); bwd_ld.assign(L, 0); bwd_q.assign(L, 0);
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
        if ((rc = upload(p_fi, fi.data(), fi.size()))) return rc;
        if ((rc = upload(p_bi, bi.data(), bi.size()))) return rc;
        dsol.fwd_items = p_fi; dsol.bwd_items = p_bi;
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
        // L2 prefetches of every launch, in launch order.  reads[k]: the factor
        // rows launch k copies, as contiguous runs (a whole supernode's rows
        // where its items follow each other) cut into pieces of at most
        // 256 KB; a chunk item's rows are covered once, by chunk 0 of its
        // column block.  Launch k issues reads[k + prefetch] (prefetch >= 1)
        // and, when a dense top block exists (and prefetch is not -1), a share
        // of the dense matrix: the forward launches before the last one, which
        // leave HBM mostly idle, stream it into L2 for the dense launch.
        {
            std::vector<int4> spans;
            std::vector<std::vector<int4>> reads(2 * (size_t)L);
            pf_ptr.assign(2 * (size_t)L + 1, 0);
            const int esz = (int)sizeof(R);
            auto add_run = [&](const R *base, int64_t e0, int64_t e1, std::vector<std::pair<int64_t, int64_t>> &runs) {
                if (e1 <= e0) return;
                if (!runs.empty() && runs.back().second == e0) runs.back().second = e1;
                else runs.push_back({e0, e1});
                (void)base;
            };
            auto flush = [&](const R *base, std::vector<std::pair<int64_t, int64_t>> &runs) {
                constexpr int64_t kPiece = 256 * 1024;
                for (const auto &r : runs)
                    for (int64_t b0 = r.first * esz; b0 < r.second * esz; b0 += kPiece) {
                        const int64_t b1 = std::min<int64_t>(r.second * esz, b0 + kPiece);
                        const unsigned long long a = (unsigned long long)(reinterpret_cast<uintptr_t>(base) + b0);
                        spans.push_back(make_int4((int)(a & 0xffffffffULL), (int)(a >> 32), (int)(b1 - b0), 0));
                    }
                runs.clear();
            };
            std::vector<std::pair<int64_t, int64_t>> runs;
            for (int k = 0; k < 2 * L; ++k) {
                const size_t s0 = spans.size();
                if (k < L) {
                    for (int it = fwd_ptr[k]; it < fwd_ptr[k + 1]; ++it) {
                        const int4 a = fi[5 * (size_t)it];
                        const int64_t q0 = (int64_t)(unsigned)a.x | ((int64_t)a.y << 32);
                        add_run(dsol.QF, q0, q0 + a.z / esz, runs);
                    }
                    flush(dsol.QF, runs);
                } else {
                    const int l = 2 * L - 1 - k;
                    for (int it = bwd_start[l]; it < bwd_start[l] + bwd_cnt[l]; ++it) {
                        const int4 a = bi[5 * (size_t)it], c = bi[5 * (size_t)it + 2], e = bi[5 * (size_t)it + 4];
                        const int64_t q0 = (int64_t)(unsigned)a.x | ((int64_t)a.y << 32);
                        if (e.x < 0) {
                            add_run(dsol.QB, q0, q0 + a.z / esz, runs);
                        } else if ((e.w & 0xffff) == 0) {  // chunk 0: rows c0 .. c1 whole
                            add_run(dsol.QB, q0 + bwd_row_off(c.x, c.z), q0 + bwd_row_off(c.y, c.z), runs);
                        }
                    }
                    flush(dsol.QB, runs);
                }
                reads[k].assign(spans.begin() + s0, spans.end());
                spans.resize(s0);
            }
            const int dist = prm.solve_prefetch > 0 ? prm.solve_prefetch : 0;
            std::vector<std::vector<int4>> issue(2 * (size_t)L);
            for (int k = 0; k < 2 * L; ++k)
                if (dist > 0 && k + dist < 2 * L) issue[k] = reads[k + dist];
            // the dense matrix, over forward launches [1, last forward launch)
            std::vector<int> fwd_launches;
            for (int l = 0; l < L; ++l)
                if (fwd_ptr[l + 1] > fwd_ptr[l]) fwd_launches.push_back(l);
            if (dense_bytes > 0 && prm.solve_dense_prefetch > 0 && fwd_launches.size() >= 3) {
                const int first = 1, last = (int)fwd_launches.size() - 2;  // inclusive
                const int nl = last - first + 1;
                constexpr int64_t kPiece = 256 * 1024;
                const int64_t npieces = (dense_bytes + kPiece - 1) / kPiece;
                for (int64_t p = 0; p < npieces; ++p) {
                    const int64_t b0 = p * kPiece, b1 = std::min<int64_t>(dense_bytes, b0 + kPiece);
                    const unsigned long long a = (unsigned long long)(reinterpret_cast<uintptr_t>(dsol.dense_inv) + b0);
                    issue[fwd_launches[first + (int)(p * nl / npieces)]].push_back(
                        make_int4((int)(a & 0xffffffffULL), (int)(a >> 32), (int)(b1 - b0), 0));
                }
            }
            for (int k = 0; k < 2 * L; ++k) {
                pf_ptr[k] = (int)spans.size();
                spans.insert(spans.end(), issue[k].begin(), issue[k].end());
            }
            pf_ptr[2 * (size_t)L] = (int)spans.size();
            spans_total = (int)spans.size();
            const int4 *p_sp;
            if ((rc = upload(p_sp, spans.data(), spans.size()))) return rc;
            dsol.pf_spans = p_sp;
            dsol.pf_ptr = pf_ptr.data();
        }
        dsol.threads = prm.solve_threads > 0 ? prm.solve_threads : 256;
        dsol.leaf_threads = prm.solve_leaf_threads > 0 ? prm.solve_leaf_threads : dsol.threads;
        dsol.prefetch = prm.solve_prefetch <= 0 ? 0 : prm.solve_prefetch;
        dsol.pf_any = spans_total > 0 ? 1 : 0;
        dsol.wait_polls = prm.wait_polls > 0 ? prm.wait_polls : (1LL << 20);
        dsol.fault_test = prm.fault_test;
        return HQN_OK;
    }

    // New sweep shapes on an existing handle (the autotuner's entry): the
    // work items are re-planned from the kept set-up, the graph rebuilt.
    int set_solve_shapes(const hqn_params &sh) override {
        hqn_params p = prm;  // solve_dense_top stays as created (the top block is factor data)
        p.solve_threads = sh.solve_threads;
        p.solve_item_kb = sh.solve_item_kb;
        p.solve_items = sh.solve_items;
        p.solve_prefetch = sh.solve_prefetch;
        p.solve_leaf_kb = sh.solve_leaf_kb;
        p.solve_leaf_threads = sh.solve_leaf_threads;
        p.solve_dense_prefetch = sh.solve_dense_prefetch;
        if (const int rc = check_solve_shapes(p)) return rc;
        int rc;
        std::string err;
        for (Setup &s : S)
            if ((rc = plan_sweeps(s, p, err))) return fail(rc, err);
        int max_ld = 0;
        for (const Setup &s : S) max_ld = std::max(max_ld, s.max_ld);
        const int kb = std::max(p.solve_item_kb > 0 ? p.solve_item_kb : 64, p.solve_leaf_kb);
        if (solve_block_smem<R>(kb * 1024 / (int)sizeof(R), max_ld) > (size_t)SOLVE_MAX_SMEM)
            return fail(HQN_ERR_UNSUPPORTED, "the work items do not fit the sweeps' shared memory");
        prm = p;
        if (graph_mode) abort_graph();
        if ((rc = plan_solve())) return rc;
        if (graph_mode) {
            if ((rc = build_graph())) {
                abort_graph();
                graph_mode = false;
                return rc;
            }
        }
        return HQN_OK;
    }

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
        if (h_ctl[0].solve_err)
            return fail(HQN_ERR_DEVICE_TIMEOUT, "a triangular sweep's wait for its factor rows ran out (flags " +
                                                    std::to_string(h_ctl[0].solve_err) + ")");
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
    void enqueue_accept(CondHandles h, cudaStream_t s) {
        launch_gather(ds, G_ITER, h, s);
        if (prm.history_m > kShortHist) launch_long_hist(ds, LD_PUSH, 0, s, 0);
    }
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

    // g and grad g at caller-order device positions (simulation 0): the
    // conversions to and from the internal order run on the device.
    int energy_grad_device(const double *x, const double *y, double *g, double *grad) override {
        const Setup &s0 = S[0];
        int rc;
        if (!d_perm0 && (rc = upload(d_perm0, s0.perm.data(), (size_t)s0.n))) return rc;
        if (!d_X0 && (rc = upload(d_X0, s0.X.data(), s0.X.size()))) return rc;
        launch_from_caller<R>(d_X0, x, d_perm0, hdesc[0].v0, s0.n, ds.xt, st);
        launch_from_caller<R>(d_X0, y, d_perm0, hdesc[0].v0, s0.n, ds.y, st);
        const CondHandles none{0, 0, 0};
        launch_inertia(ds, st);
        launch_tet(ds, TET_EVAL, none, st);
        launch_gather(ds, G_EVAL, none, st);
        if (grad) launch_to_caller<R>(ds.gk, d_perm0, hdesc[0].v0, s0.n, s0.n_free, grad, st);
        CK(cudaGetLastError());
        if ((rc = read_ctl())) return rc;
        if (g) *g = h_ctl[0].g_trial;
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
        for (int a = 0; a < np; ++a) {
            if (m > kShortHist) launch_long_hist(ds, LD_ROW, a, st, hdesc[0].nvb);
            else launch_hist_row(ds, a, st, hdesc[0].nvb);
        }
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
        o->solve_threads = dsol.threads;
        o->solve_item_kb = prm.solve_item_kb > 0 ? prm.solve_item_kb : 64;
        o->solve_items = prm.solve_items > 0 ? prm.solve_items : 400;
        o->solve_leaf_kb = prm.solve_leaf_kb > 0 ? prm.solve_leaf_kb : o->solve_item_kb;
        o->solve_leaf_threads = dsol.leaf_threads;
        o->solve_prefetch = dsol.prefetch;
        o->solve_dense_prefetch = prm.solve_dense_prefetch;
        o->solve_dense_top = S.empty() ? 0 : S[0].top_levels;
        o->dense_top_cols = dense_cols;
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
    std::vector<int> moff(count + 1, 0);  // first material of each mesh
    for (int k = 0; k < count; ++k) moff[k + 1] = moff[k] + std::max(1, (int)meshes[k].n_materials);
#pragma omp parallel for schedule(dynamic, 1) if (count > 1)
    for (int k = 0; k < count; ++k) rcs[k] = build_setup(meshes[k], materials + moff[k], prm, b->S[k], errs[k]);
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

// Checks of the sweep shapes hqn_params.solve_*.
int check_solve_shapes(const hqn_params &p) {
    if (p.solve_threads != 0 && p.solve_threads != 128 && p.solve_threads != 256 && p.solve_threads != 512)
        return fail(HQN_ERR_ARG, "solve_threads must be 0, 128, 256 or 512");
    if (p.solve_leaf_threads != 0 && p.solve_leaf_threads != 128 && p.solve_leaf_threads != 256 &&
        p.solve_leaf_threads != 512)
        return fail(HQN_ERR_ARG, "solve_leaf_threads must be 0, 128, 256 or 512");
    if (p.solve_leaf_kb != 0 && (p.solve_leaf_kb < 8 || p.solve_leaf_kb > 160))
        return fail(HQN_ERR_ARG, "solve_leaf_kb must be 0 or in [8, 160]");
    if (p.solve_item_kb != 0 && (p.solve_item_kb < 16 || p.solve_item_kb > 160))
        return fail(HQN_ERR_ARG, "solve_item_kb must be 0 or in [16, 160]");
    if (p.solve_items != 0 && (p.solve_items < 16 || p.solve_items > 4096))
        return fail(HQN_ERR_ARG, "solve_items must be 0 or in [16, 4096]");
    if (p.solve_dense_top < -1 || p.solve_dense_top > 8)
        return fail(HQN_ERR_ARG, "solve_dense_top must be -1 (none), 0 (automatic) or in [1, 8]");
    if (p.solve_dense_prefetch != 0 && p.solve_dense_prefetch != 1)
        return fail(HQN_ERR_ARG, "solve_dense_prefetch must be 0 or 1");
    if (p.solve_prefetch < -1 || p.solve_prefetch > 8)
        return fail(HQN_ERR_ARG, "solve_prefetch must be -1 (none), 0 (default) or in [1, 8]");
    return HQN_OK;
}

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
    if (const int rc = check_solve_shapes(*params)) return rc;
    if (params->wait_polls < 0) return fail(HQN_ERR_ARG, "wait_polls must be >= 0");
    if (params->fault_test != 0 && params->fault_test != 1) return fail(HQN_ERR_ARG, "fault_test must be 0 or 1");
    return HQN_OK;
}

int create_any(int count, const hqn_mesh *meshes, const hqn_material *materials, const hqn_params *params,
               void *stream, sim_handle **out) {
    if (!out) return fail(HQN_ERR_ARG, "null output pointer");
    *out = nullptr;
    if (count <= 0 || !meshes || !materials || !params) return fail(HQN_ERR_ARG, "null argument or empty batch");
    hqn_params tuned = *params;
    if (params->tune_cache) {
        // the autotuner's choices for this mesh (or batch), precision and device
        uint64_t key = hqn_mesh_key(&meshes[0]);
        if (count > 1) {
            key = 1469598103934665603ULL;
            for (int k = 0; k < count; ++k) {
                const uint64_t mk = hqn_mesh_key(&meshes[k]);
                for (int b = 0; b < 8; ++b) {
                    key ^= (mk >> (8 * b)) & 0xffULL;
                    key *= 1099511628211ULL;
                }
            }
        }
        int dev = 0;
        cudaDeviceProp prop;
        CK(cudaGetDevice(&dev));
        CK(cudaGetDeviceProperties(&prop, dev));
        const int hit = hqn_tune_lookup(params->tune_cache, prop.name, key, params->precision, &tuned);
        if (hit < 0) return fail(hit, std::string("malformed autotuner cache ") + params->tune_cache);
    }
    params = &tuned;
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
    p->n_colliders = 0;
    p->contact_scale = 100.0;
    p->a0_solver = 0;
    p->pcg_iters = 15;
    p->direction = 0;
    p->cheb_S = 10;
    p->cheb_rho = 0.99;
    p->merge_depths = 0;
    p->solve_threads = 256;
    p->solve_item_kb = 64;
    p->solve_items = 400;
    p->solve_prefetch = 0;
    p->solve_dense_prefetch = 0;
    p->solve_dense_top = 0;
    p->wait_polls = 0;
    p->fault_test = 0;
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

int sim_energy_grad_device(sim_handle *sim, const double *x_dev, const double *y_dev, double *g_out,
                           double *grad_dev) {
    if (!sim || !x_dev || !y_dev) return fail(HQN_ERR_ARG, "null argument");
    return sim->impl->energy_grad_device(x_dev, y_dev, g_out, grad_dev);
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
        const int rc = build_setup(*mesh, material, *params, S, err);
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
        info->solve_threads = params->solve_threads > 0 ? params->solve_threads : 256;
        info->solve_item_kb = params->solve_item_kb > 0 ? params->solve_item_kb : 64;
        info->solve_leaf_kb = params->solve_leaf_kb > 0 ? params->solve_leaf_kb : info->solve_item_kb;
        info->solve_leaf_threads = params->solve_leaf_threads > 0 ? params->solve_leaf_threads : info->solve_threads;
        info->solve_items = params->solve_items > 0 ? params->solve_items : 400;
        info->solve_prefetch = params->solve_prefetch <= 0 ? 0 : params->solve_prefetch;
        info->solve_dense_prefetch = params->solve_dense_prefetch;
        info->solve_dense_top = S.top_levels;
        info->dense_top_cols = S.n_top;
        info->n_sims = 1;
        return HQN_OK;
    } catch (const std::bad_alloc &) {
        return fail(HQN_ERR_NO_MEMORY, "host allocation failed");
    } catch (const std::exception &e) {
        return fail(HQN_ERR_ARG, e.what());
    }
}

int sim_set_solve_shapes(sim_handle *sim, const hqn_params *shapes) {
    if (!sim || !shapes) return fail(HQN_ERR_ARG, "null argument");
    try {
        return sim->impl->set_solve_shapes(*shapes);
    } catch (const std::bad_alloc &) {
        return fail(HQN_ERR_NO_MEMORY, "host allocation failed");
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
        case HQN_ERR_DEVICE_TIMEOUT: return "device wait timed out";
        default: return "unknown status";
    }
}

const char *hqn_last_error(void) { return g_last_error.c_str(); }

}  // extern "C"
