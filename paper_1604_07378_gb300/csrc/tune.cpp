// The autotuner's cache as the library reads it: a mesh key (a hash of the
// mesh's arrays) and the lookup of tuned shapes in a plain text file.
//
// One entry per line (later lines override earlier ones; '#' starts a
// comment line):
//   hqn-tune 1 device=<name> precision=<0|1> key=<16 hex digits> leaf_size=<n>
//       solve_threads=<n> solve_item_kb=<n> solve_items=<n> solve_prefetch=<n>
//       [solve_leaf_kb=<n>] [solve_leaf_threads=<n>] [solve_dense_top=<n>]
//       [solve_dense_prefetch=<0|1>] [ls_batch=<n>] [any other key=value, ignored]
// <name> is the CUDA device name with every space replaced by '_'.  The
// autotuner (paper_1604_07378_gb300/autotune.py) writes these lines.
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <fstream>
#include <sstream>
#include <string>

#include "../../include/hqn.h"

namespace {

constexpr uint64_t kFnvOffset = 1469598103934665603ULL;
constexpr uint64_t kFnvPrime = 1099511628211ULL;

uint64_t fnv(uint64_t h, const void *data, size_t n) {
    const unsigned char *p = static_cast<const unsigned char *>(data);
    for (size_t i = 0; i < n; ++i) {
        h ^= p[i];
        h *= kFnvPrime;
    }
    return h;
}

bool parse_int(const std::string &v, long long lo, long long hi, int32_t *out) {
    char *end = nullptr;
    const long long x = std::strtoll(v.c_str(), &end, 10);
    if (end == v.c_str() || *end != '\0' || x < lo || x > hi) return false;
    *out = (int32_t)x;
    return true;
}

}  // namespace

extern "C" {

uint64_t hqn_mesh_key(const hqn_mesh *mesh) {
    if (!mesh || mesh->n_verts <= 0 || mesh->n_tets <= 0 || !mesh->rest_pos || !mesh->tets) return 0;
    uint64_t h = kFnvOffset;
    h = fnv(h, &mesh->n_verts, sizeof(int32_t));
    h = fnv(h, &mesh->n_tets, sizeof(int32_t));
    h = fnv(h, mesh->rest_pos, sizeof(double) * 3 * (size_t)mesh->n_verts);
    h = fnv(h, mesh->tets, sizeof(int32_t) * 4 * (size_t)mesh->n_tets);
    for (int32_t v = 0; v < mesh->n_verts; ++v) {
        const unsigned char c = mesh->clamped && mesh->clamped[v] ? 1 : 0;
        h = fnv(h, &c, 1);
    }
    return h;
}

int hqn_tune_lookup(const char *path, const char *device, uint64_t key, int32_t precision, hqn_params *params) {
    if (!path || !device || !params) return HQN_ERR_ARG;
    std::ifstream f(path);
    if (!f) return 0;  // no cache yet
    std::string dev(device);
    for (char &c : dev)
        if (c == ' ') c = '_';
    char keyhex[17];
    std::snprintf(keyhex, sizeof(keyhex), "%016llx", (unsigned long long)key);
    std::string line;
    bool found = false;
    hqn_params best = *params;
    while (std::getline(f, line)) {
        std::istringstream in(line);
        std::string tag, ver;
        if (!(in >> tag) || tag[0] == '#') continue;
        if (tag != "hqn-tune") return HQN_ERR_ARG;
        if (!(in >> ver) || ver != "1") return HQN_ERR_ARG;
        std::string tok, l_dev, l_key;
        int32_t l_prec = -1;
        hqn_params p = *params;
        bool ok = true, have[5] = {false, false, false, false, false};
        while (in >> tok) {
            const size_t eq = tok.find('=');
            if (eq == std::string::npos) {
                ok = false;
                break;
            }
            const std::string k = tok.substr(0, eq), v = tok.substr(eq + 1);
            if (k == "device") l_dev = v;
            else if (k == "key") l_key = v;
            else if (k == "precision") ok = parse_int(v, 0, 1, &l_prec);
            else if (k == "leaf_size") ok = have[0] = parse_int(v, 0, 4096, &p.leaf_size);
            else if (k == "solve_threads") ok = have[1] = parse_int(v, 0, 512, &p.solve_threads);
            else if (k == "solve_item_kb") ok = have[2] = parse_int(v, 0, 160, &p.solve_item_kb);
            else if (k == "solve_items") ok = have[3] = parse_int(v, 0, 4096, &p.solve_items);
            else if (k == "solve_prefetch") ok = have[4] = parse_int(v, -1, 8, &p.solve_prefetch);
            else if (k == "ls_batch") ok = parse_int(v, 0, 16, &p.ls_batch);
            else if (k == "solve_leaf_kb") ok = parse_int(v, 0, 160, &p.solve_leaf_kb);
            else if (k == "solve_leaf_threads") ok = parse_int(v, 0, 512, &p.solve_leaf_threads);
            else if (k == "solve_dense_top") ok = parse_int(v, -1, 8, &p.solve_dense_top);
            else if (k == "solve_dense_prefetch") ok = parse_int(v, 0, 1, &p.solve_dense_prefetch);
            if (!ok) break;
        }
        if (!ok || l_dev.empty() || l_key.size() != 16 || l_prec < 0) return HQN_ERR_ARG;
        for (bool h : have)
            if (!h) return HQN_ERR_ARG;
        if (l_dev == dev && l_key == keyhex && l_prec == precision) {
            best = p;
            found = true;
        }
    }
    if (found) *params = best;
    return found ? 1 : 0;
}

}  // extern "C"
