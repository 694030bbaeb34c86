// hqn_energy_grad_static: g(x) and grad g(x) of Eq. PD for a small tet mesh
// whose arrays all live in the caller's device memory, computed without any
// device allocation.
//
// Some callers cannot allocate device memory.  They include code that runs
// under a memory pool or budget owned by someone else, plug-ins that must not
// touch the CUDA allocator, and drivers that forbid cudaMalloc once they are
// running.  The regular entry points allocate a handle's buffers in
// sim_create.  This one needs per-tet corner gradients and per-block partial
// sums as scratch.  That scratch is a file-scope __device__ array of fixed
// size: the module loader places it once in each GPU's memory when the
// library is loaded there, and it stays there until the process exits.  Host
// code cannot use the array's name as a device address, so its address is
// looked up once per device with cudaGetSymbolAddress and passed to the
// kernels.
#include <cmath>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <string>

#include "matdev_host.hpp"
#include "reduce.cuh"
#include "tetmath.cuh"

namespace hqn {
void set_last_error(const char *msg);  // api.cu
}

using namespace hqn;

namespace {

constexpr int kMaxTets = HQN_STATIC_MAX_TETS;
constexpr int kMaxVerts = HQN_STATIC_MAX_VERTS;
constexpr int kTB = 128;  // threads per block, tet kernel
constexpr int kVB = 256;  // threads per block, vertex kernel
constexpr int kTetBlocks = (kMaxTets + kTB - 1) / kTB;
constexpr int kVertBlocks = (kMaxVerts + kVB - 1) / kVB;

// Scratch shared by every call on a device.  corner[c * T + t] holds tet t's
// gradient with respect to its corner c (xyz) and, in w, the corner's share
// of the lumped mass, density * V_t / 4.  bad is set by a kernel that met an
// index outside its array (the call then reports a NaN objective).
struct StaticScratch {
    V4<double> corner[4 * (size_t)kMaxTets];
    double part_el[kTetBlocks];
    double part_in[kVertBlocks];
    unsigned int ticket;
    unsigned int bad;
};

static __device__ __align__(256) StaticScratch g_static_scratch;

std::mutex g_addr_mutex;
constexpr int kMaxDevices = 64;
StaticScratch *g_addr[kMaxDevices] = {};

// The device address of the scratch on the current device (looked up on the
// first call made with that device current).
cudaError_t scratch_address(StaticScratch **out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lock(g_addr_mutex);
    if (!g_addr[dev]) {
        void *p = nullptr;
        e = cudaGetSymbolAddress(&p, g_static_scratch);
        if (e != cudaSuccess) return e;
        g_addr[dev] = static_cast<StaticScratch *>(p);
    }
    *out = g_addr[dev];
    return cudaSuccess;
}

// Per tet: Dm^{-1} and V from the rest positions, the corner gradients of
// V Psi(F) at x (F = I + G, G from displacements u = x - X), the corners'
// mass shares and the block partial of sum_t V_t Psi_t.  A tet with
// det Dm <= 0, or with a vertex index outside [0, n), makes the energy NaN.
__global__ void __launch_bounds__(kTB) k_static_tet(int n, int T, const double *__restrict__ X,
                                                   const int *__restrict__ tets, const double *__restrict__ x,
                                                   MatDev<double> mat, double density, StaticScratch *sc) {
    const int t = blockIdx.x * kTB + threadIdx.x;
    double e[1] = {0.0};
    bool in_range = true;
    int v[4] = {0, 0, 0, 0};
    if (t < T) {
#pragma unroll
        for (int c = 0; c < 4; ++c) {
            v[c] = tets[4 * t + c];
            in_range = in_range && v[c] >= 0 && v[c] < n;
        }
    }
    if (t < T && !in_range) {
        // an index outside the vertex arrays is never dereferenced: the tet's
        // corners and energy become NaN and the call reports it
        V4<double> o;
        o.x = o.y = o.z = o.w = NAN;
#pragma unroll
        for (int c = 0; c < 4; ++c) sc->corner[(size_t)c * T + t] = o;
        e[0] = NAN;
        atomicOr(&sc->bad, 1u);
    } else if (t < T) {
        double Dm[3][3], du[3][3];
#pragma unroll
        for (int j = 0; j < 3; ++j)
#pragma unroll
            for (int a = 0; a < 3; ++a) {
                Dm[a][j] = X[3 * v[j + 1] + a] - X[3 * v[0] + a];
                du[j][a] = (x[3 * v[j + 1] + a] - X[3 * v[j + 1] + a]) - (x[3 * v[0] + a] - X[3 * v[0] + a]);
            }
        const double det = Dm[0][0] * (Dm[1][1] * Dm[2][2] - Dm[1][2] * Dm[2][1]) -
                           Dm[0][1] * (Dm[1][0] * Dm[2][2] - Dm[1][2] * Dm[2][0]) +
                           Dm[0][2] * (Dm[1][0] * Dm[2][1] - Dm[1][1] * Dm[2][0]);
        // Di = Dm^{-1}, row-major, by the adjugate
        double Di[9];
        const double id = 1.0 / det;
        Di[0] = (Dm[1][1] * Dm[2][2] - Dm[1][2] * Dm[2][1]) * id;
        Di[1] = (Dm[0][2] * Dm[2][1] - Dm[0][1] * Dm[2][2]) * id;
        Di[2] = (Dm[0][1] * Dm[1][2] - Dm[0][2] * Dm[1][1]) * id;
        Di[3] = (Dm[1][2] * Dm[2][0] - Dm[1][0] * Dm[2][2]) * id;
        Di[4] = (Dm[0][0] * Dm[2][2] - Dm[0][2] * Dm[2][0]) * id;
        Di[5] = (Dm[0][2] * Dm[1][0] - Dm[0][0] * Dm[1][2]) * id;
        Di[6] = (Dm[1][0] * Dm[2][1] - Dm[1][1] * Dm[2][0]) * id;
        Di[7] = (Dm[0][1] * Dm[2][0] - Dm[0][0] * Dm[2][1]) * id;
        Di[8] = (Dm[0][0] * Dm[1][1] - Dm[0][1] * Dm[1][0]) * id;
        const double vol = det / 6.0;
        double G[3][3], g[4][3];
        def_grad(du, Di, G);
        tet_grad(mat, G, Di, vol, g);
        e[0] = det > 0.0 ? vol * tet_psi(mat, G) : NAN;
        const double mshare = 0.25 * density * vol;
#pragma unroll
        for (int c = 0; c < 4; ++c) {
            V4<double> o;
            o.x = g[c][0]; o.y = g[c][1]; o.z = g[c][2]; o.w = mshare;
            sc->corner[(size_t)c * T + t] = o;
        }
    }
    block_sum<kTB, 1>(e);
    if (threadIdx.x == 0) sc->part_el[blockIdx.x] = e[0];
}

// Per vertex: grad g = m (x - y)/h^2 + sum of the incident corner gradients in
// the CSR's order (zero on clamped vertices), and the block partial of the
// inertia term m/(2h^2)|x - y|^2 over the free vertices.  A corner range or
// slot outside [0, 4T) is not read: the vertex's gradient becomes NaN.  The
// last block adds every partial in a fixed order and writes g (NaN if any
// index was out of range).
__global__ void __launch_bounds__(kVB) k_static_gather(int n, int T, int ntb, const double *__restrict__ x,
                                                      const double *__restrict__ y, const uint8_t *__restrict__ clamped,
                                                      const int *__restrict__ vt_ptr, const int *__restrict__ vt_slot,
                                                      double inv_h2, StaticScratch *sc, double *g_out,
                                                      double *grad_out) {
    const int i = blockIdx.x * kVB + threadIdx.x;
    double e[1] = {0.0};
    if (i < n) {
        double gx = 0.0, gy = 0.0, gz = 0.0, m = 0.0;
        const int k0 = vt_ptr[i], k1 = vt_ptr[i + 1];
        if (k0 < 0 || k1 < k0 || k1 > 4 * T) {
            gx = gy = gz = m = NAN;  // a corner range outside vt_slot is not read
            atomicOr(&sc->bad, 2u);
        } else {
            for (int k = k0; k < k1; ++k) {
                const int s = vt_slot[k];  // 4 * t + c
                if (s < 0 || s >= 4 * T) {
                    gx = gy = gz = m = NAN;
                    atomicOr(&sc->bad, 2u);
                    break;
                }
                const V4<double> cg = sc->corner[(size_t)(s & 3) * T + (s >> 2)];
                gx += cg.x; gy += cg.y; gz += cg.z; m += cg.w;
            }
        }
        const double dx = x[3 * i] - y[3 * i], dy = x[3 * i + 1] - y[3 * i + 1], dz = x[3 * i + 2] - y[3 * i + 2];
        const double mh = m * inv_h2;
        const bool fixed = clamped && clamped[i];
        // the inertia term of Eq. PD sums over the free vertices (clamped
        // ones are eliminated: their positions are prescribed)
        e[0] = fixed ? 0.0 : 0.5 * mh * (dx * dx + dy * dy + dz * dz);
        grad_out[3 * i] = fixed ? 0.0 : gx + mh * dx;
        grad_out[3 * i + 1] = fixed ? 0.0 : gy + mh * dy;
        grad_out[3 * i + 2] = fixed ? 0.0 : gz + mh * dz;
    }
    block_sum<kVB, 1>(e);
    if (!publish_and_arrive<1>(e, sc->part_in, 0, &sc->ticket)) return;
    double tot[1], el[1];
    sum_partials<kVB, 1>(sc->part_in, 0, gridDim.x, tot, &sc->ticket);
    {
        double acc = 0.0;
        for (int b = threadIdx.x; b < ntb; b += kVB) acc += __ldcg(sc->part_el + b);
        el[0] = acc;
        block_sum<kVB, 1>(el);
    }
    if (threadIdx.x == 0) *g_out = __ldcg(&sc->bad) ? NAN : el[0] + tot[0];
}

int fail(int code, const char *msg) {
    set_last_error(msg);
    return code;
}

}  // namespace

extern "C" int hqn_energy_grad_static(int32_t n_verts, int32_t n_tets, const double *rest_pos, const int32_t *tets,
                                      const uint8_t *clamped, const int32_t *vt_ptr, const int32_t *vt_slot,
                                      const hqn_material *material, double h, const double *x, const double *y,
                                      double *g_out, double *grad_out, void *stream) {
    if (n_tets <= 0 || n_verts <= 0) return fail(HQN_ERR_ARG, "hqn_energy_grad_static: empty mesh");
    if (n_tets > kMaxTets || n_verts > kMaxVerts) {
        char msg[160];
        std::snprintf(msg, sizeof(msg),
                      "hqn_energy_grad_static: %d tets / %d vertices exceed the static scratch "
                      "capacity of %d tets / %d vertices",
                      (int)n_tets, (int)n_verts, kMaxTets, kMaxVerts);
        return fail(HQN_ERR_ARG, msg);
    }
    if (!rest_pos || !tets || !vt_ptr || !vt_slot || !material || !x || !y || !g_out || !grad_out)
        return fail(HQN_ERR_ARG, "hqn_energy_grad_static: null argument");
    if (!(h > 0)) return fail(HQN_ERR_ARG, "hqn_energy_grad_static: h must be positive");
    if (!(material->density > 0) || !std::isfinite(material->density))
        return fail(HQN_ERR_ARG, "hqn_energy_grad_static: density must be positive");
    MaterialHost mh;
    std::string merr;
    if (material_from_api(*material, mh, merr) != HQN_OK)
        return fail(HQN_ERR_ARG, ("hqn_energy_grad_static: " + merr).c_str());
    MatDev<double> mat;
    matdev_from_host(mh, mat);
    StaticScratch *sc = nullptr;
    cudaError_t e = scratch_address(&sc);
    if (e != cudaSuccess) return fail(HQN_ERR_CUDA, cudaGetErrorString(e));
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    // the arrival ticket and the index flag start at zero (a previous call
    // may have been cut short, or have met a bad index)
    e = cudaMemsetAsync(&sc->ticket, 0, 2 * sizeof(unsigned int), st);
    if (e != cudaSuccess) return fail(HQN_ERR_CUDA, cudaGetErrorString(e));
    const int ntb = (n_tets + kTB - 1) / kTB, nvb = (n_verts + kVB - 1) / kVB;
    k_static_tet<<<ntb, kTB, 0, st>>>(n_verts, n_tets, rest_pos, tets, x, mat, material->density, sc);
    k_static_gather<<<nvb, kVB, 0, st>>>(n_verts, n_tets, ntb, x, y, clamped, vt_ptr, vt_slot, 1.0 / (h * h), sc,
                                         g_out, grad_out);
    e = cudaGetLastError();
    if (e != cudaSuccess) return fail(HQN_ERR_CUDA, cudaGetErrorString(e));
    return HQN_OK;
}
