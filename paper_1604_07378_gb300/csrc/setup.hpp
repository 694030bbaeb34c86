// Host-side set-up of one simulation: rest data, lumped mass, stiffness fit,
// A0 = M/h^2 + L on the free vertices, nested-dissection ordering, float64
// multifrontal Cholesky and the operators of the device triangular solves.
#pragma once

#include <cstdint>
#include <string>
#include <vector>

#include "../../include/hqn.h"

namespace hqn {

// Material in the form the kernels consume.  For Neo-Hookean, (c0, c1, c2) are
// c(J0), c'(J0), c''(J0) of the quadratic continuation below J0.
struct MaterialHost {
    int kind = HQN_NEOHOOKEAN;
    double mu = 0, lam = 0, J0 = 0.05, c0 = 0, c1 = 0, c2 = 0;
    double sx[3][8] = {}, sv[3][8] = {}, ss[3][8] = {};  // spline knots, values, slopes
    double kappa = 0, fiber[3] = {};  // anisotropic fibre term kappa/2 (|F d| - 1)^2, unit d
};

// One supernode = one node of the nested-dissection tree: its columns are a
// contiguous range of the free vertices in elimination order; its row structure
// R lists the later vertices coupled to it in the Cholesky factor L.
struct SupernodeHost {
    int col = 0, ncol = 0, nrow = 0;  // first column, #columns, #rows in R
    int parent = -1, level = 0;
    bool top = false;                 // solved by the dense top block instead of the sweeps
    int64_t qoff = 0;                 // offset of Q_s = [L_ss^{-1}; L_Rs L_ss^{-1}] (rows x ncol)
    int uoff = 0;                     // offset of its update vector (nrow entries)
    int roff = 0;                     // offset of R in the row-index array
    // device layout (layout.hpp): packed forward copy of Q_s and packed
    // backward copy of Q_s^T; ldc = pad4(ncol), ldr = pad4(ncol + nrow)
    int ldc = 0, ldr = 0;
    int64_t qf = 0, qb = 0;           // offsets of the two copies
    std::vector<int> children;
};

// Work items of the device sweeps.  G = lanes that share one output row.
struct FwdItem { int s, row0, row1, G; };  // rows [row0, row1) of Q_s f
// Backward item: rows [col0, col1) of Q_s^T times w.  A whole-row item
// (e0 < 0) covers each row from its diagonal to the end; a chunk item covers
// only the entries [e0, e1) of its rows and adds a partial sum, which the last
// of the column block's nch chunks to finish (chunk k of block cb) combines.
struct BwdItem { int s, col0, col1, G, e0 = -1, e1 = 0, cb = -1, nch = 1, k = 0; };

// Work items of both sweeps, grouped by tree level.
struct ItemLists {
    std::vector<int> fwd_lvl_ptr, bwd_lvl_ptr;  // items of level l: [ptr[l], ptr[l+1])
    std::vector<int> fwd_lvl_ld, bwd_lvl_ld;    // longest vectors an item of the level stages (forward:
                                                // f plus its rectangle rows' child updates)
    std::vector<int> fwd_lvl_q, bwd_lvl_q;      // max factor entries of one item of the level
    int n_bwd_blocks = 0;                       // column blocks of the backward chunk items
    std::vector<FwdItem> fwd_items;
    std::vector<BwdItem> bwd_items;
};

struct Setup {
    int n = 0, T = 0, n_free = 0;
    double h = 1.0 / 30.0, k = 0.0, density = 0.0;
    MaterialHost mat;                // material 0 (the only one unless the mesh has several)
    // several materials in one mesh (hqn_mesh.tet_material): each tet's
    // material index in the sorted tet order, the materials, their fitted k
    // and densities (one entry each when the mesh has one material)
    std::vector<uint8_t> tmat;
    std::vector<MaterialHost> mats;
    std::vector<double> kmat, dens;
    // vertex renumbering: perm[new] = caller's id; iperm[caller's id] = new.
    // Free vertices come first in elimination order, then the clamped ones.
    std::vector<int> perm, iperm;
    std::vector<double> X;           // rest positions, new order (n x 3)
    std::vector<int> tets;           // T x 4, new ids, sorted by smallest vertex id
    std::vector<double> dminv;       // T x 9, Dm^{-1} row-major
    std::vector<double> vol;         // T
    std::vector<double> mass;        // n lumped masses
    std::vector<double> a0_diag;     // n_free: diagonal of A0 (the Jacobi preconditioner)
    std::vector<int> vt_ptr, vt_slot;  // vertex -> (tet*4 + corner), ascending tet
    // factor and solve operators
    std::vector<SupernodeHost> sn;
    std::vector<int> rows;           // concatenated R of all supernodes
    std::vector<double> Q;           // concatenated Q_s, row-major
    std::vector<int> fg_ptr, fg_idx; // per free column: child update entries to subtract
    std::vector<int> ug_ptr, ug_idx; // per update entry: child update entries to add
    std::vector<int> fg4, ug4;       // the same maps as quads (-1 = none): at most two
                                     // children of a dissection node feed an entry, or
                                     // four under a merged supernode
    int n_upd = 0, n_levels = 0;
    ItemLists lv;                    // work items of the sweeps, level by level
    // Dense top block (hqn_params.solve_dense_top = D > 0): the supernodes of
    // the top D tree levels (level >= n_levels - D) form a subtree T whose
    // n_top columns are solved together: r_T = S^{-1} f_T with S = L_TT L_TT^T,
    // the Schur complement of A0 on T, and f_T = q_T minus the update entries
    // of the supernodes below T that reach T's columns (directly or passed
    // on through T's own update vectors).
    int top_levels = 0, n_top = 0;
    std::vector<int> top_col;        // n_top: free column of T-local index i (ascending)
    std::vector<double> top_inv;     // n_top x n_top: S^{-1}, row-major
    std::vector<int> top_bptr, top_bidx;  // per T-local column: update entries below T to subtract
    int64_t qf_total = 0, qb_total = 0;  // entries of the two packed copies
    int max_ld = 0;                  // longest vector a sweep block stages (bounds its shared memory)
    int max_front_cols = 0;          // max ncol
    int64_t factor_nnz = 0;
    double setup_seconds = 0.0;
};

// (Re)plans the sweeps' work items of a set-up for the shapes in prm
// (solve_item_kb, solve_items, precision); cheap, no refactorisation.
int plan_sweeps(Setup &S, const hqn_params &prm, std::string &err);

// Builds everything; returns an HQN_* status and a message on failure.
// mat points to max(1, mesh.n_materials) materials.
int build_setup(const hqn_mesh &mesh, const hqn_material *mat, const hqn_params &prm,
                Setup &S, std::string &err);

// Lame parameters and the kernel form of an API material, checked
// (HQN_ERR_ARG with a message on a bad E, nu, kind, spline or fibre term).
int material_from_api(const hqn_material &in, MaterialHost &out, std::string &err);

// Fits the stiffness k of Eq. stiffness for a material (used by build_setup).
double fit_stiffness(const MaterialHost &m, double x_start, double x_end);


}  // namespace hqn
