// Host-side set-up: rest data, lumped mass, stiffness fit (Eq. stiffness),
// A0 = M/h^2 + L (Eq. PDmatrixForm, PDsolution), nested-dissection ordering,
// float64 multifrontal Cholesky and the per-supernode solve operators.
#include "setup.hpp"

#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstring>
#include <map>
#include <numeric>

#include "dense.hpp"
#include "layout.hpp"

namespace hqn {

namespace {

// ---------------------------------------------------------------- quadrature

// Gauss-Legendre nodes/weights on [-1, 1] by Newton's method on P_n.
void gauss_legendre(int npts, std::vector<double> &x, std::vector<double> &w) {
    x.assign(npts, 0.0);
    w.assign(npts, 0.0);
    const double pi = std::acos(-1.0);
    for (int i = 0; i < npts; ++i) {
        double t = std::cos(pi * (i + 0.75) / (npts + 0.5));
        double dp = 1.0;
        for (int it = 0; it < 100; ++it) {
            double p0 = 1.0, p1 = t;
            for (int k = 2; k <= npts; ++k) {
                double p2 = ((2.0 * k - 1.0) * t * p1 - (k - 1.0) * p0) / k;
                p0 = p1;
                p1 = p2;
            }
            dp = npts * (t * p1 - p0) / (t * t - 1.0);
            double dt = p1 / dp;
            t -= dt;
            if (std::fabs(dt) < 1e-16) break;
        }
        x[i] = t;
        w[i] = 2.0 / ((1.0 - t * t) * dp * dp);
    }
}

// cubic Hermite segment value/derivative with quadratic continuation outside
void hermite_eval(const double *kx, const double *kv, const double *ks, double t, double &val,
                  double &der) {
    const double lo = kx[0], hi = kx[7];
    const double tc = std::min(std::max(t, lo), hi);
    int i = 0;
    for (int k = 1; k < 7; ++k)
        if (tc >= kx[k]) i = k;
    const double hh = kx[i + 1] - kx[i];
    const double u = (tc - kx[i]) / hh;
    const double v0 = kv[i], v1 = kv[i + 1], m0 = ks[i] * hh, m1 = ks[i + 1] * hh;
    // p(u) = v0 + m0 u + (3(v1-v0) - 2m0 - m1) u^2 + (2(v0-v1) + m0 + m1) u^3
    const double c2 = 3.0 * (v1 - v0) - 2.0 * m0 - m1;
    const double c3 = 2.0 * (v0 - v1) + m0 + m1;
    const double p = v0 + u * (m0 + u * (c2 + u * c3));
    const double dp = (m0 + u * (2.0 * c2 + 3.0 * u * c3)) / hh;
    const double ddp = (2.0 * c2 + 6.0 * u * c3) / (hh * hh);
    const double dt = t - tc;
    val = p + dp * dt + 0.5 * ddp * dt * dt;
    der = dp + ddp * dt;
}

// a'(s) + 2 b'(s) + c'(s), the function whose best linear fit gives k
double fit_target(const MaterialHost &m, double s) {
    const double mu = m.mu, lam = m.lam;
    switch (m.kind) {
        case HQN_NEOHOOKEAN: {
            double dc = s >= m.J0 ? (-mu + lam * std::log(s)) / s : m.c1 + m.c2 * (s - m.J0);
            return mu * s + dc;
        }
        case HQN_STVK: {
            double da = (mu + 0.5 * lam) * (s * s - 1.0) * s - lam * s;
            double db = 0.5 * lam * s;
            return da + 2.0 * db;
        }
        case HQN_COROTATED: return 2.0 * mu * (s - 1.0) + lam * (s - 1.0);
        case HQN_POLY4: return 4.0 * mu * (s - 1.0) * (s - 1.0) * (s - 1.0);
        case HQN_SPLINE_VL: {
            double v, da, db, dc;
            hermite_eval(m.sx[0], m.sv[0], m.ss[0], s, v, da);
            hermite_eval(m.sx[1], m.sv[1], m.ss[1], s, v, db);
            hermite_eval(m.sx[2], m.sv[2], m.ss[2], s, v, dc);
            return da + 2.0 * db + dc;
        }
    }
    return 0.0;
}

// ---------------------------------------------------------------- small linear algebra

double det3(const double *M) {
    return M[0] * (M[4] * M[8] - M[5] * M[7]) - M[1] * (M[3] * M[8] - M[5] * M[6]) +
           M[2] * (M[3] * M[7] - M[4] * M[6]);
}

void inv3(const double *M, double *R) {
    const double d = det3(M);
    R[0] = (M[4] * M[8] - M[5] * M[7]) / d;
    R[1] = (M[2] * M[7] - M[1] * M[8]) / d;
    R[2] = (M[1] * M[5] - M[2] * M[4]) / d;
    R[3] = (M[5] * M[6] - M[3] * M[8]) / d;
    R[4] = (M[0] * M[8] - M[2] * M[6]) / d;
    R[5] = (M[2] * M[3] - M[0] * M[5]) / d;
    R[6] = (M[3] * M[7] - M[4] * M[6]) / d;
    R[7] = (M[1] * M[6] - M[0] * M[7]) / d;
    R[8] = (M[0] * M[4] - M[1] * M[3]) / d;
}

// ---------------------------------------------------------------- nested dissection

struct NDState {
    const std::vector<double> *X;      // caller-order rest positions
    const std::vector<int> *adj_ptr;   // caller-order adjacency of free vertices
    const std::vector<int> *adj;
    std::vector<char> side;            // scratch: 0 none, 1 = A, 2 = B
    std::vector<int> order;            // elimination order (caller ids)
    std::vector<SupernodeHost> nodes;
    std::vector<std::vector<int>> node_verts;
    int leaf = 64;
};

// A node of the dissection tree over vertex set V (its columns once ordered).
int nd_node(NDState &st, const std::vector<int> &V, const std::vector<int> &children) {
    SupernodeHost s;
    s.children = children;
    st.nodes.push_back(s);
    st.node_verts.push_back(V);
    const int id = (int)st.nodes.size() - 1;
    for (int c : children) st.nodes[c].parent = id;
    return id;
}

int nd_recurse(NDState &st, std::vector<int> &V) {
    const std::vector<double> &X = *st.X;
    if ((int)V.size() <= st.leaf) {
        std::sort(V.begin(), V.end());
        return nd_node(st, V, {});
    }
    double lo[3] = {1e300, 1e300, 1e300}, hi[3] = {-1e300, -1e300, -1e300};
    for (int v : V)
        for (int a = 0; a < 3; ++a) {
            lo[a] = std::min(lo[a], X[3 * v + a]);
            hi[a] = std::max(hi[a], X[3 * v + a]);
        }
    int axes[3] = {0, 1, 2};
    std::sort(axes, axes + 3, [&](int a, int b) { return hi[a] - lo[a] > hi[b] - lo[b]; });
    std::vector<int> A, B;
    for (int ai = 0; ai < 3 && A.empty(); ++ai) {
        const int ax = axes[ai];
        const double ext = hi[ax] - lo[ax];
        if (!(ext > 0)) continue;
        std::vector<int> sorted = V;
        std::sort(sorted.begin(), sorted.end(), [&](int a, int b) {
            double xa = X[3 * a + ax], xb = X[3 * b + ax];
            return xa < xb || (xa == xb && a < b);
        });
        const double c = X[3 * sorted[sorted.size() / 2] + ax];
        const double tol = 1e-9 * ext;
        A.clear();
        B.clear();
        for (int v : V) (X[3 * v + ax] < c - tol ? A : B).push_back(v);
        if (A.empty() || B.empty()) A.clear();
    }
    if (A.empty()) {  // cannot split geometrically: make it one leaf-like node
        std::sort(V.begin(), V.end());
        return nd_node(st, V, {});
    }
    for (int v : A) st.side[v] = 1;
    for (int v : B) st.side[v] = 2;
    std::vector<int> S, Bp;
    for (int v : B) {
        bool touches = false;
        for (int e = (*st.adj_ptr)[v]; e < (*st.adj_ptr)[v + 1] && !touches; ++e)
            touches = st.side[(*st.adj)[e]] == 1;
        (touches ? S : Bp).push_back(v);
    }
    if (S.empty()) {  // disconnected halves: still give the node one column
        S.push_back(Bp.back());
        Bp.pop_back();
    }
    for (int v : A) st.side[v] = 0;
    for (int v : B) st.side[v] = 0;
    std::vector<int> children;
    children.push_back(nd_recurse(st, A));
    if (!Bp.empty()) children.push_back(nd_recurse(st, Bp));
    std::sort(S.begin(), S.end());
    return nd_node(st, S, children);
}

// The supernode tree and the elimination order, from the dissection tree.
// A dissection node at depth d (the root at 0) whose bit d is set in `merge`
// takes its children's vertices into its own supernode, and theirs in turn
// when their bits are set; the supernode's children are the dissection nodes
// below the merged group.  Merging a separator with the separators under it
// gives up the zeros between them (the children's vertices are not coupled
// to each other) and some fill in the rectangle, and removes a level from
// each sweep's dependency chain.  Columns follow the tree in postorder: a
// supernode's children first, then its group, children's vertices before
// their parent's.
// A merged supernode holds at most this many columns: a forward work item
// stages its whole right-hand side in shared memory.
constexpr int kMergeMaxCols = 4096;

// Columns of the supernode that dissection node p (depth d) heads.
int nd_group_cols(const NDState &st, int p, int d, uint32_t merge) {
    int n = (int)st.node_verts[p].size();
    if (d < 32 && ((merge >> d) & 1u)) {
        int m = n;
        for (int c : st.nodes[p].children) m += nd_group_cols(st, c, d + 1, merge);
        if (m <= kMergeMaxCols) n = m;
    }
    return n;
}

void nd_collect(const NDState &st, int p, int d, uint32_t merge, std::vector<int> &group,
                std::vector<std::pair<int, int>> &kids) {
    const bool absorb = d < 32 && ((merge >> d) & 1u) &&
                        nd_group_cols(st, p, d, merge) > (int)st.node_verts[p].size();
    for (int c : st.nodes[p].children) {
        if (absorb) nd_collect(st, c, d + 1, merge, group, kids);
        else kids.push_back({c, d + 1});
    }
    group.push_back(p);
}

int nd_emit(const NDState &st, int p, int d, uint32_t merge, std::vector<SupernodeHost> &out,
            std::vector<int> &order) {
    std::vector<int> group;
    std::vector<std::pair<int, int>> kids;
    nd_collect(st, p, d, merge, group, kids);
    std::vector<int> ch;
    for (const auto &k : kids) ch.push_back(nd_emit(st, k.first, k.second, merge, out, order));
    SupernodeHost s;
    s.col = (int)order.size();
    for (int g : group)
        for (int v : st.node_verts[g]) order.push_back(v);
    s.ncol = (int)order.size() - s.col;
    s.children = ch;
    out.push_back(s);
    const int id = (int)out.size() - 1;
    for (int c : ch) out[c].parent = id;
    return id;
}

// Work items of both sweeps, level by level.  Items hold at most kMax factor
// entries (one shared-memory buffer) and aim at a level's entries / per_level.
// Forward: consecutive rows of Q_s.  Backward: consecutive rows of Q_s^T; rows longer than kLongRow
// entries are split into chunks of 32 rows x kChunk entries, so an item
// gathers a short piece of w instead of the whole vector (a few columns per
// item would otherwise each gather all of it).
int make_items(const Setup &S, int VN, int kMaxUpper, int kMaxLeaf, int64_t per_level, ItemLists &out,
               std::string &err) {
    const int L = S.n_levels, ns = (int)S.sn.size();
    // lanes per output row: enough that each lane reads a few 16-byte vectors
    auto lanes_for = [&](int len) {
        const int nv = (len + VN - 1) / VN;
        int G = 1;
        while (G < 32 && G * 4 < nv) G *= 2;
        return G;
    };
    std::vector<int64_t> lvl_entries(L, 0);
    for (auto &sn : S.sn)
        if (!sn.top) lvl_entries[sn.level] += fwd_row_off(sn.ncol + sn.nrow, sn.ncol, sn.ldc);
    out = ItemLists{};
    out.fwd_lvl_ptr.assign(L + 1, 0);
    out.bwd_lvl_ptr.assign(L + 1, 0);
    out.fwd_lvl_ld.assign(L, 0);
    out.bwd_lvl_ld.assign(L, 0);
    out.fwd_lvl_q.assign(L, 0);
    out.bwd_lvl_q.assign(L, 0);
    for (int l = 0; l < L; ++l) {
        const int kMax = l == 0 ? kMaxLeaf : kMaxUpper, kMin = kMax / 4;
        const int target = (int)std::min<int64_t>(kMax, std::max<int64_t>(kMin, lvl_entries[l] / per_level));
        out.fwd_lvl_ptr[l] = (int)out.fwd_items.size();
        for (int s = 0; s < ns; ++s) {
            const SupernodeHost &sn = S.sn[s];
            if (sn.level != l || sn.ncol == 0 || sn.top) continue;
            const int nc = sn.ncol, rows = nc + sn.nrow;
            for (int r0 = 0; r0 < rows;) {
                int r1 = r0 + 1;
                while (r1 < rows && fwd_row_off(r1 + 1, nc, sn.ldc) - fwd_row_off(r0, nc, sn.ldc) <= target) ++r1;
                // staged vectors: f (ldc entries) and the rectangle rows' child updates
                const int nrr = std::max(0, r1 - std::max(r0, nc));
                out.fwd_lvl_ld[l] = std::max(out.fwd_lvl_ld[l], sn.ldc + pad4(nrr));
                const int entries = (int)(fwd_row_off(r1, nc, sn.ldc) - fwd_row_off(r0, nc, sn.ldc));
                if (entries > kMax) {
                    err = "a factor row does not fit the sweeps' shared-memory buffer";
                    return HQN_ERR_UNSUPPORTED;
                }
                out.fwd_lvl_q[l] = std::max(out.fwd_lvl_q[l], entries);
                out.fwd_items.push_back({s, r0, r1, lanes_for(fwd_row_len(r1 - 1, nc, sn.ldc))});
                r0 = r1;
            }
        }
    }
    out.fwd_lvl_ptr[L] = (int)out.fwd_items.size();
    constexpr int kBlockCols = 32;
    const int kChunk = VN == 4 ? 256 : 128;
    const int kLongRow = 4 * kChunk;
    for (int l = 0; l < L; ++l) {
        const int kMax = l == 0 ? kMaxLeaf : kMaxUpper, kMin = kMax / 4;
        const int target = (int)std::min<int64_t>(kMax, std::max<int64_t>(kMin, lvl_entries[l] / per_level));
        out.bwd_lvl_ptr[l] = (int)out.bwd_items.size();
        for (int s = 0; s < ns; ++s) {
            const SupernodeHost &sn = S.sn[s];
            if (sn.level != l || sn.ncol == 0 || sn.top) continue;
            for (int c0 = 0; c0 < sn.ncol;) {
                const int w0 = bwd_row_start(c0);
                if (sn.ldr - w0 > kLongRow) {
                    const int c1 = std::min(sn.ncol, c0 + kBlockCols);
                    const int nch = (sn.ldr - w0 + kChunk - 1) / kChunk;
                    for (int k = 0; k < nch; ++k) {
                        BwdItem it{s, c0, c1, lanes_for(kChunk)};
                        it.e0 = w0 + k * kChunk;
                        it.e1 = std::min(sn.ldr, it.e0 + kChunk);
                        it.cb = out.n_bwd_blocks;
                        it.nch = nch;
                        it.k = k;
                        out.bwd_lvl_q[l] = std::max(out.bwd_lvl_q[l], (c1 - c0) * (it.e1 - it.e0));
                        out.bwd_lvl_ld[l] = std::max(out.bwd_lvl_ld[l], it.e1 - it.e0);
                        out.bwd_items.push_back(it);
                    }
                    ++out.n_bwd_blocks;
                    c0 = c1;
                    continue;
                }
                int c1 = c0 + 1;
                while (c1 < sn.ncol && bwd_row_off(c1 + 1, sn.ldr) - bwd_row_off(c0, sn.ldr) <= target) ++c1;
                const int entries = (int)(bwd_row_off(c1, sn.ldr) - bwd_row_off(c0, sn.ldr));
                if (entries > kMax) {
                    err = "a factor row does not fit the sweeps' shared-memory buffer";
                    return HQN_ERR_UNSUPPORTED;
                }
                out.bwd_lvl_q[l] = std::max(out.bwd_lvl_q[l], entries);
                out.bwd_lvl_ld[l] = std::max(out.bwd_lvl_ld[l], sn.ldr - w0);
                out.bwd_items.push_back({s, c0, c1, lanes_for(sn.ldr - w0)});
                c0 = c1;
            }
        }
    }
    out.bwd_lvl_ptr[L] = (int)out.bwd_items.size();
    return HQN_OK;
}

}  // namespace

// Lame parameters and the kernel form of an API material (Eq. valanis-landel),
// with its checks: E > 0 and -1 < nu < 0.5 (so that mu and lambda are finite
// and positive where the materials need them), a known kind, strictly
// increasing spline knots, and a positive fibre weight with a nonzero
// direction.  The one mapping every entry point uses.
int material_from_api(const hqn_material &in, MaterialHost &M, std::string &err) {
    M = MaterialHost{};
    if (!(in.E > 0) || !(in.nu > -1.0 && in.nu < 0.5)) {
        err = "material needs E > 0 and -1 < nu < 0.5";
        return HQN_ERR_ARG;
    }
    M.kind = in.kind;
    M.mu = in.E / (2.0 * (1.0 + in.nu));
    M.lam = in.E * in.nu / ((1.0 + in.nu) * (1.0 - 2.0 * in.nu));
    if (M.kind == HQN_NEOHOOKEAN) {
        const double J0 = M.J0, l0 = std::log(J0);
        M.c0 = -M.mu * l0 + 0.5 * M.lam * l0 * l0;
        M.c1 = (-M.mu + M.lam * l0) / J0;
        M.c2 = (M.mu + M.lam - M.lam * l0) / (J0 * J0);
    } else if (M.kind == HQN_SPLINE_VL) {
        if (!in.spline) {
            err = "spline material needs control points";
            return HQN_ERR_ARG;
        }
        for (int f = 0; f < 3; ++f)
            for (int i = 0; i < 8; ++i) {
                M.sx[f][i] = in.spline[(f * 8 + i) * 3 + 0];
                M.sv[f][i] = in.spline[(f * 8 + i) * 3 + 1];
                M.ss[f][i] = in.spline[(f * 8 + i) * 3 + 2];
                if (i > 0 && !(M.sx[f][i] > M.sx[f][i - 1])) {
                    err = "spline knots must increase";
                    return HQN_ERR_ARG;
                }
            }
    } else if (M.kind != HQN_STVK && M.kind != HQN_COROTATED && M.kind != HQN_POLY4) {
        err = "unknown material kind";
        return HQN_ERR_ARG;
    }
    // anisotropic fibre term (Sec. 4.4); not part of the stiffness fit
    if (in.kappa != 0.0) {
        const double nn = std::sqrt(in.fiber[0] * in.fiber[0] + in.fiber[1] * in.fiber[1] +
                                    in.fiber[2] * in.fiber[2]);
        if (!(in.kappa > 0.0) || !std::isfinite(in.kappa) || !(nn > 0.0) || !std::isfinite(nn)) {
            err = "the fibre term needs kappa > 0 and a nonzero direction";
            return HQN_ERR_ARG;
        }
        M.kappa = in.kappa;
        for (int a = 0; a < 3; ++a) M.fiber[a] = in.fiber[a] / nn;
    }
    return HQN_OK;
}

double fit_stiffness(const MaterialHost &m, double x_start, double x_end) {
    // k = int (s - sbar) f(s) ds / int (s - sbar)^2 ds on [x_start, x_end]
    // (continuous least-squares slope), integrated piecewise with 8-point
    // Gauss-Legendre between breakpoints (spline knots, J0) and 16 panels.
    std::vector<double> gx, gw;
    gauss_legendre(8, gx, gw);
    std::vector<double> br;
    for (int p = 0; p <= 16; ++p) br.push_back(x_start + (x_end - x_start) * p / 16.0);
    if (m.kind == HQN_SPLINE_VL)
        for (int f = 0; f < 3; ++f)
            for (int i = 0; i < 8; ++i)
                if (m.sx[f][i] > x_start && m.sx[f][i] < x_end) br.push_back(m.sx[f][i]);
    if (m.kind == HQN_NEOHOOKEAN && m.J0 > x_start && m.J0 < x_end) br.push_back(m.J0);
    std::sort(br.begin(), br.end());
    const double sbar = 0.5 * (x_start + x_end);
    double num = 0.0;
    for (size_t p = 0; p + 1 < br.size(); ++p) {
        const double a = br[p], b = br[p + 1];
        if (!(b > a)) continue;
        const double half = 0.5 * (b - a), mid = 0.5 * (a + b);
        for (int q = 0; q < 8; ++q) {
            const double s = mid + half * gx[q];
            num += half * gw[q] * (s - sbar) * fit_target(m, s);
        }
    }
    const double len = x_end - x_start;
    return num / (len * len * len / 12.0);
}

// Leaf size 0: 128 vertices in the float32 form for meshes of up to 150,000
// free vertices, 64 otherwise.  Doubling the leaf removes a level from each
// sweep's chain (~5 us per level) and adds ~20 factor entries per vertex to
// the leaf level, which streams at HBM speed: on a 40^3 lattice (67k free
// vertices) the solve gained 4%, on a 48x48x192 bar (463k) it lost 10%.  The
// float64 form's sweeps are bound by float64 arithmetic on the entries.
static int leaf_size_of(const hqn_params &prm, int n_free) {
    if (prm.leaf_size > 0) return prm.leaf_size;
    return prm.precision == HQN_FP32_MIXED && n_free <= 150000 ? 128 : 64;
}

// The dense top block of hqn_params.solve_dense_top (D < 0: none; 0: the
// automatic choice below): the subtree T of the top D levels, S^{-1} = (L_TT L_TT^T)^{-1} on its columns and the update
// entries below T that reach each of its columns.  S^{-1} = L_TT^{-T} L_TT^{-1}
// comes from the supernodal sweeps themselves, run on T alone with the
// identity as n_top right-hand sides: forward X := L_TT^{-1} X (right-looking:
// X_C := Q_ss X_C, X_R -= Q_Rs X_C), then backward X := L_TT^{-T} X
// (X_C := Q_ss^T X_C - Q_Rs^T X_R, root first), every step one GEMM.
static int build_dense_top(Setup &S, int D, std::string &err) {
    const int ns = (int)S.sn.size(), nf = S.n_free;
    S.top_levels = 0;
    S.n_top = 0;
    S.top_col.clear();
    S.top_inv.clear();
    S.top_bptr.assign(1, 0);
    S.top_bidx.clear();
    for (auto &sn : S.sn) sn.top = false;
    if (D < 0) return HQN_OK;
    if (D == 0) {
        // automatic: the most top levels (at most 3) whose block has at most
        // kAutoCols columns (the host's cost grows as the cube of the columns)
        constexpr int kAutoCols = 5000;
        for (int d = std::min(3, S.n_levels); d >= 1 && D == 0; --d) {
            int64_t cols = 0;
            for (const SupernodeHost &sn : S.sn)
                if (sn.level >= S.n_levels - d) cols += sn.ncol;
            if (cols <= kAutoCols) D = d;
        }
        if (D == 0) return HQN_OK;
    }
    D = std::min(D, S.n_levels);
    std::vector<int> pos(nf, -1);  // free column -> T-local index
    for (int s = 0; s < ns; ++s) {
        SupernodeHost &sn = S.sn[s];
        if (sn.level < S.n_levels - D || sn.ncol == 0) continue;
        sn.top = true;
    }
    // columns of T in ascending order
    for (int s = 0; s < ns; ++s)
        if (S.sn[s].top)
            for (int a = 0; a < S.sn[s].ncol; ++a) S.top_col.push_back(S.sn[s].col + a);
    std::sort(S.top_col.begin(), S.top_col.end());
    const int n = (int)S.top_col.size();
    if (n == 0) return HQN_OK;
    if (n > 16384) {
        err = "the dense top block would hold more than 16384 columns";
        return HQN_ERR_UNSUPPORTED;
    }
    for (int i = 0; i < n; ++i) pos[S.top_col[i]] = i;
    // every T supernode's columns are consecutive in T-local order and its
    // rows lie in T (an ancestor's columns)
    for (int s = 0; s < ns; ++s) {
        const SupernodeHost &sn = S.sn[s];
        if (!sn.top) continue;
        for (int a = 1; a < sn.ncol; ++a)
            if (pos[sn.col + a] != pos[sn.col] + a) {
                err = "dense top block: supernode columns not consecutive";
                return HQN_ERR_ARG;
            }
        for (int b = 0; b < sn.nrow; ++b)
            if (pos[S.rows[sn.roff + b]] < 0) {
                err = "dense top block: a row lies outside the top subtree";
                return HQN_ERR_ARG;
            }
        if (sn.parent >= 0 && !S.sn[sn.parent].top) {
            err = "dense top block: not a subtree";
            return HQN_ERR_ARG;
        }
    }
    std::vector<double> X((size_t)n * n, 0.0);
    for (int i = 0; i < n; ++i) X[(size_t)i * n + i] = 1.0;
    std::vector<double> XcT, tmp, Qt;
    // forward: X := L_TT^{-1} X (X stays lower triangular: columns >= cend of a
    // supernode's rows are still zero when it is processed)
    for (int s = 0; s < ns; ++s) {
        const SupernodeHost &sn = S.sn[s];
        if (!sn.top) continue;
        const int nc = sn.ncol, nr = sn.nrow, c0 = pos[sn.col], cend = c0 + nc;
        const double *Qs = S.Q.data() + sn.qoff;
        XcT.assign((size_t)cend * nc, 0.0);  // X_C^T (cend x nc)
        for (int a = 0; a < nc; ++a)
            for (int j = 0; j < cend; ++j) XcT[(size_t)j * nc + a] = X[(size_t)(c0 + a) * n + j];
        tmp.assign((size_t)nc * cend, 0.0);
        gemm_nt(nc, cend, nc, 1.0, Qs, nc, XcT.data(), nc, 0.0, tmp.data(), cend, false);
        for (int a = 0; a < nc; ++a)
            std::copy(tmp.begin() + (size_t)a * cend, tmp.begin() + (size_t)(a + 1) * cend, X.begin() + (size_t)(c0 + a) * n);
        if (nr > 0) {
            tmp.assign((size_t)nr * cend, 0.0);
            gemm_nt(nr, cend, nc, 1.0, Qs + (size_t)nc * nc, nc, XcT.data(), nc, 0.0, tmp.data(), cend, false);
            for (int b = 0; b < nr; ++b) {
                double *xr = X.data() + (size_t)pos[S.rows[sn.roff + b]] * n;
                const double *t = tmp.data() + (size_t)b * cend;
                for (int j = 0; j < cend; ++j) xr[j] -= t[j];
            }
        }
    }
    // backward, root first: X_C := Q_ss^T X_C - Q_Rs^T X_R (all n columns)
    for (int s = ns - 1; s >= 0; --s) {
        const SupernodeHost &sn = S.sn[s];
        if (!sn.top) continue;
        const int nc = sn.ncol, nr = sn.nrow, c0 = pos[sn.col], rows = nc + nr;
        const double *Qs = S.Q.data() + sn.qoff;
        // Qt = Q_s^T (nc x rows); W^T = [X_C; -X_R]^T (n x rows)
        Qt.assign((size_t)nc * rows, 0.0);
        for (int i = 0; i < rows; ++i)
            for (int a = 0; a < nc; ++a) Qt[(size_t)a * rows + i] = Qs[(size_t)i * nc + a];
        XcT.assign((size_t)n * rows, 0.0);
        for (int i = 0; i < rows; ++i) {
            const bool own = i < nc;
            const double *xr = X.data() + (size_t)(own ? c0 + i : pos[S.rows[sn.roff + i - nc]]) * n;
            for (int j = 0; j < n; ++j) XcT[(size_t)j * rows + i] = own ? xr[j] : -xr[j];
        }
        tmp.assign((size_t)nc * n, 0.0);
        gemm_nt(nc, n, rows, 1.0, Qt.data(), rows, XcT.data(), rows, 0.0, tmp.data(), n, false);
        std::copy(tmp.begin(), tmp.end(), X.begin() + (size_t)c0 * n);
    }
    // S^{-1} is symmetric; average the two triangles' rounding
    for (int i = 0; i < n; ++i)
        for (int j = 0; j < i; ++j) {
            const double v = 0.5 * (X[(size_t)i * n + j] + X[(size_t)j * n + i]);
            X[(size_t)i * n + j] = X[(size_t)j * n + i] = v;
        }
    S.top_inv.swap(X);
    // update entries below T that reach each T column: the column's child
    // entries, expanded through the update vectors of T's own supernodes
    std::vector<int> owner(S.n_upd, -1);
    for (int s = 0; s < ns; ++s)
        for (int b = 0; b < S.sn[s].nrow; ++b) owner[S.sn[s].uoff + b] = s;
    std::vector<int> stack;
    for (int i = 0; i < n; ++i) {
        const int j = S.top_col[i];
        stack.assign(S.fg_idx.begin() + S.fg_ptr[j], S.fg_idx.begin() + S.fg_ptr[j + 1]);
        while (!stack.empty()) {
            const int e = stack.back();
            stack.pop_back();
            if (S.sn[owner[e]].top) {
                for (int k = S.ug_ptr[e]; k < S.ug_ptr[e + 1]; ++k) stack.push_back(S.ug_idx[k]);
            } else {
                S.top_bidx.push_back(e);
            }
        }
        std::sort(S.top_bidx.begin() + S.top_bptr.back(), S.top_bidx.end());
        if ((int)S.top_bidx.size() - S.top_bptr.back() > 4) {
            err = "dense top block: a column receives more than four update entries from below";
            return HQN_ERR_UNSUPPORTED;
        }
        S.top_bptr.push_back((int)S.top_bidx.size());
    }
    S.top_levels = D;
    S.n_top = n;
    return HQN_OK;
}

int plan_sweeps(Setup &S, const hqn_params &prm, std::string &err) {
    const int VN = prm.precision == HQN_FP64_PLAIN ? 2 : 4;
    const int esize = prm.precision == HQN_FP64_PLAIN ? 8 : 4;
    // a level's entries spread over solve_items items (default 400, a few
    // blocks per SM), each within [kMax/4, kMax] entries, kMax =
    // solve_item_kb KB (default 64), solve_leaf_kb on the leaf level
    const int item_kb = prm.solve_item_kb > 0 ? prm.solve_item_kb : 64;
    const int leaf_kb = prm.solve_leaf_kb > 0 ? prm.solve_leaf_kb : item_kb;
    const int per_level = prm.solve_items > 0 ? prm.solve_items : 400;
    int rc = make_items(S, VN, item_kb * 1024 / esize, leaf_kb * 1024 / esize, per_level, S.lv, err);
    if (rc != HQN_OK) return rc;
    // the longest vector a sweep block stages (what bounds its shared memory)
    S.max_ld = 0;
    for (int l = 0; l < S.n_levels; ++l)
        S.max_ld = std::max(S.max_ld, std::max(S.lv.fwd_lvl_ld[l], S.lv.bwd_lvl_ld[l]));
    return HQN_OK;
}

int build_setup(const hqn_mesh &mesh, const hqn_material *mats_in, const hqn_params &prm,
                Setup &S, std::string &err) {
    auto t_start = std::chrono::steady_clock::now();
    const int n = mesh.n_verts, T = mesh.n_tets;
    if (n <= 0 || T <= 0 || !mesh.rest_pos || !mesh.tets) {
        err = "empty mesh or null pointer";
        return HQN_ERR_ARG;
    }
    if (!(prm.h > 0) || !(prm.x_end > prm.x_start) || prm.iters < 0 || prm.iters > HQN_MAX_ITERS ||
        prm.history_m < 0 || prm.history_m > HQN_MAX_HISTORY || prm.ls_max <= 0 ||
        !(prm.gamma > 0 && prm.gamma < 1) || !(prm.backtrack > 0 && prm.backtrack < 1)) {
        err = "parameter out of range";
        return HQN_ERR_ARG;
    }
    for (int64_t i = 0; i < 3LL * n; ++i)
        if (!std::isfinite(mesh.rest_pos[i])) {
            err = "non-finite rest position";
            return HQN_ERR_NONFINITE;
        }
    for (int64_t i = 0; i < 4LL * T; ++i)
        if (mesh.tets[i] < 0 || mesh.tets[i] >= n) {
            err = "tet vertex index out of range";
            return HQN_ERR_ARG;
        }
    // ---- materials: one, or one per index of mesh.tet_material
    const int nmat = mesh.n_materials > 0 ? mesh.n_materials : 1;
    if (!mats_in || nmat > HQN_MAX_MATERIALS || (nmat > 1 && !mesh.tet_material)) {
        err = "need 1..HQN_MAX_MATERIALS materials (and tet_material for more than one)";
        return HQN_ERR_ARG;
    }
    S.mats.assign(nmat, MaterialHost{});
    S.kmat.assign(nmat, 0.0);
    S.dens.assign(nmat, 0.0);
    for (int m = 0; m < nmat; ++m) {
        const hqn_material &matin = mats_in[m];
        if (!(matin.density > 0) || !std::isfinite(matin.E) || !std::isfinite(matin.nu)) {
            err = "material density must be positive and E, nu finite";
            return matin.density <= 0 ? HQN_ERR_NOT_SPD : HQN_ERR_NONFINITE;
        }
        if (int rc = material_from_api(matin, S.mats[m], err)) return rc;
        S.kmat[m] = fit_stiffness(S.mats[m], prm.x_start, prm.x_end);
        if (!(S.kmat[m] > 0) || !std::isfinite(S.kmat[m])) {
            err = "stiffness fit is not positive";
            return HQN_ERR_NOT_SPD;
        }
        S.dens[m] = matin.density;
    }
    std::vector<uint8_t> tmat0(T, 0);
    if (nmat > 1)
        for (int t = 0; t < T; ++t) {
            const int m = mesh.tet_material[t];
            if (m < 0 || m >= nmat) {
                err = "tet_material index out of range";
                return HQN_ERR_ARG;
            }
            tmat0[t] = (uint8_t)m;
        }
    S.mat = S.mats[0];
    S.k = S.kmat[0];
    S.h = prm.h;
    S.density = S.dens[0];

    // ---- rest data in caller order
    std::vector<double> dminv0((size_t)T * 9), vol0(T);
    for (int t = 0; t < T; ++t) {
        const int *tv = mesh.tets + 4 * t;
        double Dm[9];
        for (int j = 0; j < 3; ++j)
            for (int a = 0; a < 3; ++a)
                Dm[3 * a + j] = mesh.rest_pos[3 * tv[j + 1] + a] - mesh.rest_pos[3 * tv[0] + a];
        const double d = det3(Dm);
        if (!(d > 0)) {
            err = "degenerate or inverted rest tet " + std::to_string(t);
            return HQN_ERR_DEGENERATE_TET;
        }
        vol0[t] = d / 6.0;
        inv3(Dm, &dminv0[9 * (size_t)t]);
    }

    // ---- free vertices and their adjacency (caller ids)
    std::vector<char> clamped(n, 0);
    if (mesh.clamped)
        for (int v = 0; v < n; ++v) clamped[v] = mesh.clamped[v] != 0;
    std::vector<int> deg(n + 1, 0);
    for (int t = 0; t < T; ++t)
        for (int a = 0; a < 4; ++a)
            for (int b = 0; b < 4; ++b)
                if (a != b) deg[mesh.tets[4 * t + a]]++;
    std::vector<int> adj_ptr(n + 1, 0);
    for (int v = 0; v < n; ++v) adj_ptr[v + 1] = adj_ptr[v] + deg[v];
    std::vector<int> adj(adj_ptr[n]);
    {
        std::vector<int> fill(adj_ptr.begin(), adj_ptr.end() - 1);
        for (int t = 0; t < T; ++t)
            for (int a = 0; a < 4; ++a)
                for (int b = 0; b < 4; ++b)
                    if (a != b) adj[fill[mesh.tets[4 * t + a]]++] = mesh.tets[4 * t + b];
        // dedupe, drop clamped neighbours
        std::vector<int> nptr(n + 1, 0);
        int w = 0;
        for (int v = 0; v < n; ++v) {
            int b0 = adj_ptr[v], b1 = adj_ptr[v + 1];
            std::sort(adj.begin() + b0, adj.begin() + b1);
            nptr[v] = w;
            int last = -1;
            for (int e = b0; e < b1; ++e) {
                int u = adj[e];
                if (u == last) continue;
                last = u;
                if (!clamped[u]) adj[w++] = u;
            }
        }
        nptr[n] = w;
        adj.resize(w);
        adj_ptr.swap(nptr);
    }

    // ---- nested dissection of the free vertices
    std::vector<double> Xc(mesh.rest_pos, mesh.rest_pos + 3 * (size_t)n);
    NDState st;
    st.X = &Xc;
    st.adj_ptr = &adj_ptr;
    st.adj = &adj;
    st.side.assign(n, 0);
    std::vector<int> freev;
    for (int v = 0; v < n; ++v)
        if (!clamped[v]) freev.push_back(v);
    st.leaf = leaf_size_of(prm, (int)freev.size());
    if (freev.empty()) {
        err = "every vertex is clamped";
        return HQN_ERR_ARG;
    }
    const int root = nd_recurse(st, freev);
    S.sn.clear();
    st.order.clear();
    nd_emit(st, root, 0, (uint32_t)prm.merge_depths, S.sn, st.order);
    S.n = n;
    S.T = T;
    S.n_free = (int)st.order.size();
    S.perm = st.order;
    for (int v = 0; v < n; ++v)
        if (clamped[v]) S.perm.push_back(v);
    S.iperm.assign(n, 0);
    for (int i = 0; i < n; ++i) S.iperm[S.perm[i]] = i;
    const int nf = S.n_free;

    // ---- renumbered rest data, tets sorted by smallest vertex id
    S.X.resize(3 * (size_t)n);
    for (int i = 0; i < n; ++i)
        for (int a = 0; a < 3; ++a) S.X[3 * i + a] = Xc[3 * S.perm[i] + a];
    std::vector<int> torder(T);
    std::vector<int> tmin(T);
    for (int t = 0; t < T; ++t) {
        int m = n;
        for (int a = 0; a < 4; ++a) m = std::min(m, S.iperm[mesh.tets[4 * t + a]]);
        tmin[t] = m;
    }
    std::iota(torder.begin(), torder.end(), 0);
    std::stable_sort(torder.begin(), torder.end(), [&](int a, int b) { return tmin[a] < tmin[b]; });
    S.tets.resize(4 * (size_t)T);
    S.dminv.resize(9 * (size_t)T);
    S.vol.resize(T);
    S.tmat.assign(T, 0);
    for (int i = 0; i < T; ++i) {
        const int t = torder[i];
        S.tmat[i] = tmat0[t];
        for (int a = 0; a < 4; ++a) S.tets[4 * i + a] = S.iperm[mesh.tets[4 * t + a]];
        for (int e = 0; e < 9; ++e) S.dminv[9 * (size_t)i + e] = dminv0[9 * (size_t)t + e];
        S.vol[i] = vol0[t];
    }
    // lumped mass: a quarter of each incident tet's mass
    S.mass.assign(n, 0.0);
    for (int t = 0; t < T; ++t)
        for (int a = 0; a < 4; ++a) S.mass[S.tets[4 * t + a]] += 0.25 * S.dens[S.tmat[t]] * S.vol[t];
    // vertex -> corner slots, ascending tet
    S.vt_ptr.assign(n + 1, 0);
    for (int t = 0; t < T; ++t)
        for (int a = 0; a < 4; ++a) S.vt_ptr[S.tets[4 * t + a] + 1]++;
    for (int v = 0; v < n; ++v) S.vt_ptr[v + 1] += S.vt_ptr[v];
    S.vt_slot.assign(4 * (size_t)T, 0);
    {
        std::vector<int> fill(S.vt_ptr.begin(), S.vt_ptr.end() - 1);
        for (int t = 0; t < T; ++t)
            for (int a = 0; a < 4; ++a) S.vt_slot[fill[S.tets[4 * t + a]]++] = 4 * t + a;
    }

    // ---- A0 = M/h^2 + sum_t V_t k G_t^T G_t on free vertices, lower part by column
    // element block: K_e[a][b] = V k (B^T Dm^{-1} Dm^{-T} B)[a][b]
    std::vector<std::vector<std::pair<int, double>>> Acol(nf);
    for (int t = 0; t < T; ++t) {
        const double *Di = &S.dminv[9 * (size_t)t];
        // G = Dm^{-T} B : column a of G (a = 0..3) is the gradient of the a-th hat function
        double G[3][4];
        for (int i = 0; i < 3; ++i) {
            double s = 0;
            for (int j = 0; j < 3; ++j) {
                G[i][j + 1] = Di[3 * j + i];  // (Dm^{-T})_{i j} = Dm^{-1}_{j i}
                s += Di[3 * j + i];
            }
            G[i][0] = -s;
        }
        const double w = S.vol[t] * S.kmat[S.tmat[t]];
        for (int a = 0; a < 4; ++a)
            for (int b = 0; b < 4; ++b) {
                const int va = S.tets[4 * t + a], vb = S.tets[4 * t + b];
                if (va >= nf || vb >= nf || va < vb) continue;
                const double kab = w * (G[0][a] * G[0][b] + G[1][a] * G[1][b] + G[2][a] * G[2][b]);
                Acol[vb].push_back({va, kab});
            }
    }
    const double inv_h2 = 1.0 / (prm.h * prm.h);
    for (int j = 0; j < nf; ++j) {
        Acol[j].push_back({j, S.mass[j] * inv_h2});
        auto &c = Acol[j];
        std::sort(c.begin(), c.end(), [](auto &p, auto &q) { return p.first < q.first; });
        size_t w = 0;
        for (size_t e = 0; e < c.size(); ++e) {
            if (w > 0 && c[w - 1].first == c[e].first) c[w - 1].second += c[e].second;
            else c[w++] = c[e];
        }
        c.resize(w);
    }
    S.a0_diag.assign(nf, 0.0);
    for (int j = 0; j < nf; ++j)
        for (const auto &e : Acol[j])
            if (e.first == j) S.a0_diag[j] = e.second;

    // ---- symbolic: row structures R_s (postorder = node order)
    const int ns = (int)S.sn.size();
    std::vector<int> mark(nf, -1);
    S.rows.clear();
    for (int s = 0; s < ns; ++s) {
        SupernodeHost &sn = S.sn[s];
        const int last = sn.col + sn.ncol - 1;
        std::vector<int> R;
        for (int j = sn.col; j <= last; ++j)
            for (auto &e : Acol[j])
                if (e.first > last && mark[e.first] != s) {
                    mark[e.first] = s;
                    R.push_back(e.first);
                }
        for (int c : sn.children) {
            const SupernodeHost &cs = S.sn[c];
            for (int k = 0; k < cs.nrow; ++k) {
                const int i = S.rows[cs.roff + k];
                if (i < sn.col) {
                    err = "nested dissection produced an invalid assembly tree";
                    return HQN_ERR_ARG;
                }
                if (i > last && mark[i] != s) {
                    mark[i] = s;
                    R.push_back(i);
                }
            }
        }
        std::sort(R.begin(), R.end());
        sn.roff = (int)S.rows.size();
        sn.nrow = (int)R.size();
        S.rows.insert(S.rows.end(), R.begin(), R.end());
        sn.level = 0;
        for (int c : sn.children) sn.level = std::max(sn.level, S.sn[c].level + 1);
    }
    // check every child's rows fit in the parent's front
    for (int s = 0; s < ns; ++s) {
        const SupernodeHost &sn = S.sn[s];
        if (sn.parent < 0) continue;
        const SupernodeHost &p = S.sn[sn.parent];
        for (int k = 0; k < sn.nrow; ++k) {
            const int i = S.rows[sn.roff + k];
            if (i >= p.col && i < p.col + p.ncol) continue;
            if (!std::binary_search(S.rows.begin() + p.roff, S.rows.begin() + p.roff + p.nrow, i)) {
                err = "child row structure not contained in parent front";
                return HQN_ERR_ARG;
            }
        }
    }

    // ---- offsets
    int64_t qtot = 0;
    int utot = 0;
    S.factor_nnz = 0;
    S.max_front_cols = 0;
    for (auto &sn : S.sn) {
        sn.qoff = qtot;
        qtot += (int64_t)(sn.ncol + sn.nrow) * sn.ncol;
        sn.uoff = utot;
        utot += sn.nrow;
        S.factor_nnz += (int64_t)sn.ncol * (sn.ncol + 1) / 2 + (int64_t)sn.ncol * sn.nrow;
        S.max_front_cols = std::max(S.max_front_cols, sn.ncol);
    }
    S.n_upd = utot;
    S.Q.assign(qtot, 0.0);

    // ---- numeric multifrontal factorisation (postorder)
    std::vector<std::vector<double>> upd(ns);  // update matrices U_s (nrow x nrow, lower)
    std::vector<int> pos(nf, -1);
    for (int s = 0; s < ns; ++s) {
        SupernodeHost &sn = S.sn[s];
        const int nc = sn.ncol, nr = sn.nrow, fs = nc + nr;
        const int *R = S.rows.data() + sn.roff;
        for (int j = 0; j < nc; ++j) pos[sn.col + j] = j;
        for (int k = 0; k < nr; ++k) pos[R[k]] = nc + k;
        std::vector<double> F((size_t)fs * fs, 0.0);
        for (int j = 0; j < nc; ++j)
            for (auto &e : Acol[sn.col + j]) F[(size_t)pos[e.first] * fs + j] += e.second;
        for (int c : sn.children) {
            const SupernodeHost &cs = S.sn[c];
            const int *Rc = S.rows.data() + cs.roff;
            const std::vector<double> &U = upd[c];
            for (int a = 0; a < cs.nrow; ++a) {
                const int pa = pos[Rc[a]];
                for (int b = 0; b <= a; ++b) F[(size_t)pa * fs + pos[Rc[b]]] += U[(size_t)a * cs.nrow + b];
            }
            std::vector<double>().swap(upd[c]);
        }
        int info = potrf_lower(nc, F.data(), fs);
        if (info != 0) {
            err = "A0 not positive definite at column " + std::to_string(sn.col + info - 1);
            return HQN_ERR_NOT_SPD;
        }
        if (nr > 0) {
            trsm_right_lower_t(nr, nc, F.data(), fs, F.data() + (size_t)nc * fs, fs);
            gemm_nt(nr, nr, nc, -1.0, F.data() + (size_t)nc * fs, fs, F.data() + (size_t)nc * fs, fs,
                    1.0, F.data() + (size_t)nc * fs + nc, fs, true);
            upd[s].assign((size_t)nr * nr, 0.0);
            for (int a = 0; a < nr; ++a)
                for (int b = 0; b <= a; ++b)
                    upd[s][(size_t)a * nr + b] = F[(size_t)(nc + a) * fs + nc + b];
        }
        // Q_s = [L_ss^{-1}; L_Rs L_ss^{-1}]
        std::vector<double> LinvT((size_t)nc * nc);
        trtri_lower_t(nc, F.data(), fs, LinvT.data(), nc);
        double *Qs = S.Q.data() + sn.qoff;
        for (int i = 0; i < nc; ++i)
            for (int j = 0; j <= i; ++j) Qs[(size_t)i * nc + j] = LinvT[(size_t)j * nc + i];
        if (nr > 0)
            gemm_nt(nr, nc, nc, 1.0, F.data() + (size_t)nc * fs, fs, LinvT.data(), nc, 0.0,
                    Qs + (size_t)nc * nc, nc, false);
    }

    // ---- extend-add maps of the device solve
    S.fg_ptr.assign(nf + 1, 0);
    S.ug_ptr.assign(utot + 1, 0);
    {
        std::vector<std::vector<int>> fg(nf), ug(utot);
        for (int s = 0; s < ns; ++s) {
            const SupernodeHost &sn = S.sn[s];
            const int *R = S.rows.data() + sn.roff;
            for (int j = 0; j < sn.ncol; ++j) pos[sn.col + j] = j;
            for (int k = 0; k < sn.nrow; ++k) pos[R[k]] = sn.ncol + k;
            for (int c : sn.children) {
                const SupernodeHost &cs = S.sn[c];
                for (int a = 0; a < cs.nrow; ++a) {
                    const int p = pos[S.rows[cs.roff + a]];
                    if (p < sn.ncol) fg[sn.col + p].push_back(cs.uoff + a);
                    else ug[sn.uoff + p - sn.ncol].push_back(cs.uoff + a);
                }
            }
        }
        for (int j = 0; j < nf; ++j) S.fg_ptr[j + 1] = S.fg_ptr[j] + (int)fg[j].size();
        for (int j = 0; j < nf; ++j) S.fg_idx.insert(S.fg_idx.end(), fg[j].begin(), fg[j].end());
        for (int u = 0; u < utot; ++u) S.ug_ptr[u + 1] = S.ug_ptr[u] + (int)ug[u].size();
        for (int u = 0; u < utot; ++u) S.ug_idx.insert(S.ug_idx.end(), ug[u].begin(), ug[u].end());
    }

    // ---- quad form of the extend-add maps: each entry receives from at most
    // the two children of a dissection node, or from the four below a merged
    // pair of depths
    S.fg4.assign(4 * (size_t)nf, -1);
    S.ug4.assign(4 * (size_t)utot, -1);
    for (int j = 0; j < nf; ++j) {
        const int c = S.fg_ptr[j + 1] - S.fg_ptr[j];
        if (c > 4) {
            err = "a column receives updates from more than four children";
            return HQN_ERR_ARG;
        }
        for (int k = 0; k < c; ++k) S.fg4[4 * (size_t)j + k] = S.fg_idx[S.fg_ptr[j] + k];
    }
    for (int u = 0; u < utot; ++u) {
        const int c = S.ug_ptr[u + 1] - S.ug_ptr[u];
        if (c > 4) {
            err = "an update entry receives from more than four children";
            return HQN_ERR_ARG;
        }
        for (int k = 0; k < c; ++k) S.ug4[4 * (size_t)u + k] = S.ug_idx[S.ug_ptr[u] + k];
    }

    // ---- packed device layout (layout.hpp) and level work lists
    S.qf_total = S.qb_total = 0;
    for (auto &sn : S.sn) {
        sn.ldc = pad4(sn.ncol);
        sn.ldr = pad4(sn.ncol + sn.nrow);
        sn.qf = S.qf_total;
        sn.qb = S.qb_total;
        S.qf_total += fwd_row_off(sn.ncol + sn.nrow, sn.ncol, sn.ldc);
        S.qb_total += bwd_row_off(sn.ncol, sn.ldr);
    }
    S.n_levels = 0;
    for (auto &sn : S.sn) S.n_levels = std::max(S.n_levels, sn.level + 1);
    if (int rc = build_dense_top(S, prm.solve_dense_top, err)) return rc;
    if (int rc = plan_sweeps(S, prm, err)) return rc;

    S.setup_seconds =
        std::chrono::duration<double>(std::chrono::steady_clock::now() - t_start).count();
    return HQN_OK;
}

}  // namespace hqn
