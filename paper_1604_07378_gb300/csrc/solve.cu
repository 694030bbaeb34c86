// Device forward and backward sweeps of r = A0^{-1} q, A0 = M/h^2 + L
// (Eq. PDsolution; the constant initial Hessian of Alg. 2, prefactored once),
// on 3 right-hand sides (x, y, z share one n x n factor, Sec. 3).
//
// The factor L is supernodal over a nested-dissection tree.  Each supernode s
// (columns C, later coupled rows R) holds Q_s = [L_CC^{-1}; L_RC L_CC^{-1}], so
// both sweeps are independent dense row dot products:
//   forward (leaves first):  f = q_C - (child updates landing on C);
//                            z_C = L_CC^{-1} f;  u_R = L_RC z_C + (child updates on R)
//   backward (root first):   r_C = Q_s^T [z_C; -r_R]
// A tree level is one launch; within a level every supernode is independent,
// and updates pass up the tree through index tables (each entry receives from
// at most four children; no atomics).
//
// One block runs one work item: a run of consecutive rows of the packed
// forward copy of Q_s, or of the packed backward copy of Q_s^T (layout.hpp),
// which is one contiguous block of memory.  Thread 0 starts a single bulk
// copy (cp.async.bulk, completion counted on an mbarrier) of those rows into
// shared memory; meanwhile the block gathers the vector the rows multiply
// (f, or w = [z_C; -r_R]) into shared memory.  Each output is then the dot of
// a row with that vector, computed by a group of G lanes with 16-byte
// shared-memory loads, two rows per group at a time.
//
// Consecutive levels are chained by programmatic dependent launch: every
// block allows the next level to launch as soon as it starts, so a level's
// blocks may start while the previous level still runs.  Before
// griddepcontrol.wait a block touches only data that no sweep writes (its
// item record, the factor rows, the index tables); the vectors produced by
// earlier levels and by the kernels before the solve are read after it.
#include "kernels.cuh"
#include "layout.hpp"
#include "reduce.cuh"

namespace hqn {

namespace {

constexpr int SBS = 256;                  // threads per block of the sweeps
constexpr long long kWaitPolls = 1 << 20;  // bound on the bulk-copy wait (polls)

template <typename R> struct Vec16;
template <> struct Vec16<float> {
    using T = float4;
    static constexpr int N = 4;
    __device__ static float dot3(const float4 &q, const float4 &a) { return q.x * a.x + q.y * a.y + q.z * a.z + q.w * a.w; }
};
template <> struct Vec16<double> {
    using T = double2;
    static constexpr int N = 2;
    __device__ static double dot3(const double2 &q, const double2 &a) { return q.x * a.x + q.y * a.y; }
};

template <typename R, int G>
__device__ __forceinline__ R group_sum(R v) {
#pragma unroll
    for (int o = G / 2; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// ---- bulk copy global -> shared with an mbarrier (PTX ISA: cp.async.bulk, mbarrier)

__device__ __forceinline__ uint32_t smem_addr(const void *p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

// Thread 0, once per block: an mbarrier with one arrival per phase.
__device__ __forceinline__ void bulk_bar_init(uint64_t *bar) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_addr(bar)) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

// Thread 0: the phase's single arrival, with the bytes its copies will bring.
__device__ __forceinline__ void bulk_expect(uint64_t *bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)), "r"(bytes)
                 : "memory");
}

// Any thread: one copy whose bytes count against the barrier's phase.  The
// factor is streamed once per solve and does not fit in L2, so its lines are
// marked evict-first: they do not push out the vectors and mesh data the
// other kernels of an iteration reuse.
__device__ __forceinline__ void bulk_copy(uint64_t *bar, void *dst, const void *src, uint32_t bytes) {
    uint64_t pol;
    asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(pol));
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes.L2::cache_hint [%0], [%1], %2, [%3], %4;" ::"r"(
            smem_addr(dst)),
        "l"(src), "r"(bytes), "r"(smem_addr(bar)), "l"(pol)
        : "memory");
}

// Thread 0: the phase's arrival and one contiguous copy.
__device__ __forceinline__ void bulk_load_issue(uint64_t *bar, void *dst, const void *src, uint32_t bytes) {
    bulk_expect(bar, bytes);
    bulk_copy(bar, dst, src, bytes);
}

__device__ __forceinline__ bool bulk_load_wait(uint64_t *bar, uint32_t parity) {
    for (long long it = 0; it < kWaitPolls; ++it) {
        uint32_t done;
        asm volatile(
            "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
            : "=r"(done)
            : "r"(smem_addr(bar)), "r"(parity)
            : "memory");
        if (done) return true;
    }
    return false;
}

// Every thread waits for the phase `parity` of the block's bulk copy (the
// barrier's init by thread 0 and this wait are separated by a __syncthreads
// here).  Returns false (after flagging the error) if it did not complete
// within the poll bound; the block must then leave without reading the buffer.
__device__ __forceinline__ bool bulk_load_finish(uint64_t *bar, uint32_t parity, unsigned int *err) {
    __shared__ int timed_out;
    if (threadIdx.x == 0) timed_out = 0;
    __syncthreads();
    if (!bulk_load_wait(bar, parity)) timed_out = 1;
    __syncthreads();
    if (timed_out) {
        if (threadIdx.x == 0) {
            atomicOr(err, 1u);
            bulk_load_wait(bar, parity);  // give the copy in flight one more bounded chance to land
        }
        return false;
    }
    return true;
}

// ---- programmatic dependent launch (PTX ISA: griddepcontrol)

// Waits until the grids this one depends on have completed and their memory
// is visible (returns at once when the launch had no such dependency).
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
// Lets the next grid in the stream start launching its blocks.
__device__ __forceinline__ void pdl_trigger() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }

__device__ __forceinline__ const void *item_src(const void *base, int4 a, int esize) {
    const long long q0 = (long long)(unsigned)a.x | ((long long)a.y << 32);
    return static_cast<const char *>(base) + q0 * esize;
}

// Vector loads that bypass L1: the sweeps read vectors other blocks of the
// same grid have just written.
__device__ __forceinline__ V4<float> ld_cg(const V4<float> *p) {
    const float4 v = __ldcg(reinterpret_cast<const float4 *>(p));
    V4<float> o;
    o.x = v.x; o.y = v.y; o.z = v.z; o.w = v.w;
    return o;
}
__device__ __forceinline__ V4<double> ld_cg(const V4<double> *p) {
    const double2 a = __ldcg(reinterpret_cast<const double2 *>(p));
    const double2 b = __ldcg(reinterpret_cast<const double2 *>(p) + 1);
    V4<double> o;
    o.x = a.x; o.y = a.y; o.z = b.x; o.w = b.y;
    return o;
}

// ---- forward sweep

// Rows [r0, r1) of Q_s (in shared memory at qs, first row at offset off0 of
// the supernode's block) times f: z_C for rows < nc, update entries (plus the
// <= 2 child entries) for rows >= nc.
// nt threads (tid = 0..nt-1, nt a multiple of 32) share the rows; f's three
// components lie fs entries apart.
// ua (if not null): the child update entries of rows [rr0, ...) already
// summed, three components ua_s entries apart.  Each group of G lanes takes
// RPG consecutive rows at a time, so every load of f serves RPG rows.
template <typename R, int G>
__device__ __forceinline__ void fwd_rows(const DevSolve<R> &S, int col, int nc, int ldc, int uoff, int r0, int r1,
                                         int off0, const R *qs, const R *f, int fs, V4<R> *z, int tid, int nt,
                                         const R *ua, int ua_s, int rr0) {
    using VT = typename Vec16<R>::T;
    constexpr int VN = Vec16<R>::N;
    constexpr int RPG = 4;
    const int NG = nt / G;
    const int lane = tid % G, grp = tid / G;
    const VT *fx = reinterpret_cast<const VT *>(f);
    const VT *fy = reinterpret_cast<const VT *>(f + fs);
    const VT *fz = reinterpret_cast<const VT *>(f + 2 * fs);
    for (int base = r0; base < r1; base += RPG * NG) {
        int nv[RPG];
        const VT *qv[RPG];
        int nmax = 0;
#pragma unroll
        for (int h = 0; h < RPG; ++h) {
            const int i = base + RPG * grp + h;
            const bool v = i < r1;
            nv[h] = v ? fwd_row_len(i, nc, ldc) / VN : 0;
            qv[h] = reinterpret_cast<const VT *>(qs + (v ? fwd_row_off(i, nc, ldc) - off0 : 0));
            nmax = nv[h] > nmax ? nv[h] : nmax;
        }
        R acc[RPG][3];
#pragma unroll
        for (int h = 0; h < RPG; ++h) acc[h][0] = acc[h][1] = acc[h][2] = R(0);
        for (int k = lane; k < nmax; k += G) {
            const VT x = fx[k], y = fy[k], w = fz[k];
#pragma unroll
            for (int h = 0; h < RPG; ++h)
                if (k < nv[h]) {
                    const VT q = qv[h][k];
                    acc[h][0] += Vec16<R>::dot3(q, x); acc[h][1] += Vec16<R>::dot3(q, y); acc[h][2] += Vec16<R>::dot3(q, w);
                }
        }
#pragma unroll
        for (int h = 0; h < RPG; ++h) {
            acc[h][0] = group_sum<R, G>(acc[h][0]);
            acc[h][1] = group_sum<R, G>(acc[h][1]);
            acc[h][2] = group_sum<R, G>(acc[h][2]);
        }
        if (lane == 0) {
#pragma unroll
            for (int h = 0; h < RPG; ++h) {
                const int i = base + RPG * grp + h;
                if (i >= r1) continue;
                V4<R> o;
                o.x = acc[h][0]; o.y = acc[h][1]; o.z = acc[h][2]; o.w = R(0);
                if (i < nc) {
                    z[col + i] = o;
                } else {
                    if (ua) {
                        o.x += ua[i - rr0]; o.y += ua[ua_s + i - rr0]; o.z += ua[2 * ua_s + i - rr0];
                    } else {
                        const int4 c = S.ug4[uoff + i - nc];
                        if (c.x >= 0) { const V4<R> a = ld_cg(S.u + c.x); o.x += a.x; o.y += a.y; o.z += a.z; }
                        if (c.y >= 0) { const V4<R> a = ld_cg(S.u + c.y); o.x += a.x; o.y += a.y; o.z += a.z; }
                        if (c.z >= 0) { const V4<R> a = ld_cg(S.u + c.z); o.x += a.x; o.y += a.y; o.z += a.z; }
                        if (c.w >= 0) { const V4<R> a = ld_cg(S.u + c.w); o.x += a.x; o.y += a.y; o.z += a.z; }
                    }
                    S.u[uoff + i - nc] = o;
                }
            }
        }
    }
}

template <typename R>
__device__ __forceinline__ void fwd_rows_g(int G, const DevSolve<R> &S, int col, int nc, int ldc, int uoff, int r0,
                                           int r1, int off0, const R *qs, const R *f, int fs, V4<R> *z, int tid,
                                           int nt, const R *ua = nullptr, int ua_s = 0, int rr0 = 0) {
    switch (G) {
        case 1: fwd_rows<R, 1>(S, col, nc, ldc, uoff, r0, r1, off0, qs, f, fs, z, tid, nt, ua, ua_s, rr0); break;
        case 2: fwd_rows<R, 2>(S, col, nc, ldc, uoff, r0, r1, off0, qs, f, fs, z, tid, nt, ua, ua_s, rr0); break;
        case 4: fwd_rows<R, 4>(S, col, nc, ldc, uoff, r0, r1, off0, qs, f, fs, z, tid, nt, ua, ua_s, rr0); break;
        case 8: fwd_rows<R, 8>(S, col, nc, ldc, uoff, r0, r1, off0, qs, f, fs, z, tid, nt, ua, ua_s, rr0); break;
        case 16: fwd_rows<R, 16>(S, col, nc, ldc, uoff, r0, r1, off0, qs, f, fs, z, tid, nt, ua, ua_s, rr0); break;
        default: fwd_rows<R, 32>(S, col, nc, ldc, uoff, r0, r1, off0, qs, f, fs, z, tid, nt, ua, ua_s, rr0); break;
    }
}

// One forward work item (record `rec`, 5 int4).  Shared memory: qs = the
// item's factor rows (qcap entries), then f (3 x ldf entries), then the summed
// child update entries of its rectangle rows (3 x pad4(nrr) entries), then
// their source indices (ldf int4 for the columns, nrr int4 for the rows; up
// to four children feed an entry, -1 = none).  Every
// load of a vector another item produces is issued in one parallel pass
// after `wait_inputs`, so the row products read only shared memory.
template <typename R, typename Wait>
__device__ __forceinline__ void fwd_item(const DevSolve<R> &S, const int4 *rec, int qcap, R *qs, uint64_t *bar,
                                         uint32_t parity, const V4<R> *rhs, V4<R> *z, Wait wait_inputs) {
    const int4 a = rec[0];
    if (threadIdx.x == 0) bulk_load_issue(bar, qs, item_src(S.QF, a, sizeof(R)), (uint32_t)a.z);
    const int4 b = rec[1], c = rec[2];
    const int col = b.x, nc = b.y, ldc = b.z, uoff = b.w;
    const int r0 = c.x, r1 = c.y, ldf = c.z, off0 = c.w;
    const int rr0 = r0 > nc ? r0 : nc, nrr = r1 > rr0 ? r1 - rr0 : 0, nrr4 = pad4(nrr);
    R *f = qs + qcap;
    R *ua = f + 3 * ldf;
    int4 *cidx = reinterpret_cast<int4 *>(ua + 3 * nrr4);
    int4 *ridx = cidx + ldf;
    const int nf = ldf < nc ? ldf : nc;
    for (int j = threadIdx.x; j < nf; j += SBS) cidx[j] = __ldg(S.fg4 + col + j);
    for (int j = threadIdx.x; j < nrr; j += SBS) ridx[j] = __ldg(S.ug4 + uoff + rr0 - nc + j);
    if (!wait_inputs()) {
        if (threadIdx.x == 0) bulk_load_wait(bar, parity);  // let the copy in flight land first
        return;
    }
    // f = q_C - (child updates on C), entries [0, ldf), zero beyond nc; and
    // the child updates landing on the rectangle rows
    const int nj = ldf > nrr ? ldf : nrr;
#pragma unroll 2
    for (int j = threadIdx.x; j < nj; j += SBS) {
        V4<R> v, u[4], w[4];
        v.x = v.y = v.z = R(0);
#pragma unroll
        for (int k = 0; k < 4; ++k) { u[k] = v; w[k] = v; }
        if (j < nc) {
            const int4 ci = cidx[j];
            v = ld_cg(rhs + col + j);
            if (ci.x >= 0) u[0] = ld_cg(S.u + ci.x);
            if (ci.y >= 0) u[1] = ld_cg(S.u + ci.y);
            if (ci.z >= 0) u[2] = ld_cg(S.u + ci.z);
            if (ci.w >= 0) u[3] = ld_cg(S.u + ci.w);
        }
        if (j < nrr) {
            const int4 ri = ridx[j];
            if (ri.x >= 0) w[0] = ld_cg(S.u + ri.x);
            if (ri.y >= 0) w[1] = ld_cg(S.u + ri.y);
            if (ri.z >= 0) w[2] = ld_cg(S.u + ri.z);
            if (ri.w >= 0) w[3] = ld_cg(S.u + ri.w);
        }
        if (j < ldf) {
            f[j] = v.x - u[0].x - u[1].x - u[2].x - u[3].x;
            f[ldf + j] = v.y - u[0].y - u[1].y - u[2].y - u[3].y;
            f[2 * ldf + j] = v.z - u[0].z - u[1].z - u[2].z - u[3].z;
        }
        if (j < nrr) {
            ua[j] = w[0].x + w[1].x + w[2].x + w[3].x;
            ua[nrr4 + j] = w[0].y + w[1].y + w[2].y + w[3].y;
            ua[2 * nrr4 + j] = w[0].z + w[1].z + w[2].z + w[3].z;
        }
    }
    if (!bulk_load_finish(bar, parity, S.err)) return;
    fwd_rows_g<R>(a.w, S, col, nc, ldc, uoff, r0, r1, off0, qs, f, ldf, z, (int)threadIdx.x, SBS, ua, nrr4, rr0);
}

// Level-synchronous schedule: one launch per tree level, one item per block.
template <typename R>
__global__ void __launch_bounds__(SBS, 4) k_fwd(DevSolve<R> S, int item0, int qcap, const V4<R> *rhs, V4<R> *z) {
    extern __shared__ __align__(128) unsigned char smem_raw[];
    __shared__ __align__(8) uint64_t bar;
    if (threadIdx.x == 0) bulk_bar_init(&bar);
    fwd_item<R>(S, S.fwd_items + 5 * (size_t)(item0 + blockIdx.x), qcap, reinterpret_cast<R *>(smem_raw), &bar, 0u,
                rhs, z, []() {
                    pdl_trigger();
                    pdl_wait();
                    return true;
                });
}

// ---- backward sweep

// Rows [c0, c1) of Q_s^T times w, where w holds entries [w0, w0 + lw) of
// [z_C; -r_R].  Whole-row items (CHUNK false): the rows lie packed in shared
// memory at qs (first row at offset off0 of the supernode's block), row j from
// its diagonal start on.  Chunk items (CHUNK true): row j sits at
// qs + (j - c0) lw, aligned with w, holding its entries of the chunk.
// The sums go to r[col + j], or to out[j - c0] (a chunk's partial sums).
// nt threads (tid = 0..nt-1, nt a multiple of 32) share the rows; w's three
// components lie ws entries apart.  Each group of G lanes takes RPG
// consecutive rows at a time, so every load of w serves RPG rows.
template <typename R, int G, bool CHUNK>
__device__ __forceinline__ void bwd_rows(int col, int ldr, int c0, int c1, int off0, const R *qs, const R *w,
                                         int ws, int lw, int w0, V4<R> *r, V4<R> *out, int tid, int nt) {
    using VT = typename Vec16<R>::T;
    constexpr int VN = Vec16<R>::N;
    constexpr int RPG = 4;
    const int NG = nt / G;
    const int lane = tid % G, grp = tid / G;
    const VT *wx = reinterpret_cast<const VT *>(w);
    const VT *wy = reinterpret_cast<const VT *>(w + ws);
    const VT *wz = reinterpret_cast<const VT *>(w + 2 * ws);
    const int kend = lw / VN;
    for (int base = c0; base < c1; base += RPG * NG) {
        // row j covers w vectors [k_j, kend)
        int kb[RPG];
        const VT *qv[RPG];
        int kmin = kend;
#pragma unroll
        for (int h = 0; h < RPG; ++h) {
            const int j = base + RPG * grp + h;
            kb[h] = kend;
            qv[h] = nullptr;
            if (j < c1) {
                const int st = bwd_row_start(j);
                kb[h] = st > w0 ? (st - w0) / VN : 0;
                qv[h] = CHUNK ? reinterpret_cast<const VT *>(qs + (size_t)(j - c0) * lw)
                              : reinterpret_cast<const VT *>(qs + (bwd_row_off(j, ldr) - off0)) - kb[h];
            }
            kmin = kb[h] < kmin ? kb[h] : kmin;
        }
        R acc[RPG][3];
#pragma unroll
        for (int h = 0; h < RPG; ++h) acc[h][0] = acc[h][1] = acc[h][2] = R(0);
        for (int k = kmin + lane; k < kend; k += G) {
            const VT x = wx[k], y = wy[k], v = wz[k];
#pragma unroll
            for (int h = 0; h < RPG; ++h)
                if (k >= kb[h]) {
                    const VT q = qv[h][k];
                    acc[h][0] += Vec16<R>::dot3(q, x); acc[h][1] += Vec16<R>::dot3(q, y); acc[h][2] += Vec16<R>::dot3(q, v);
                }
        }
#pragma unroll
        for (int h = 0; h < RPG; ++h) {
            acc[h][0] = group_sum<R, G>(acc[h][0]);
            acc[h][1] = group_sum<R, G>(acc[h][1]);
            acc[h][2] = group_sum<R, G>(acc[h][2]);
        }
        if (lane == 0) {
#pragma unroll
            for (int h = 0; h < RPG; ++h) {
                const int j = base + RPG * grp + h;
                if (j >= c1) continue;
                V4<R> o; o.x = acc[h][0]; o.y = acc[h][1]; o.z = acc[h][2]; o.w = R(0);
                if (out) out[j - c0] = o; else r[col + j] = o;
            }
        }
    }
}

template <typename R, bool CHUNK>
__device__ __forceinline__ void bwd_rows_g(int G, int col, int ldr, int c0, int c1, int off0, const R *qs,
                                           const R *w, int ws, int lw, int w0, V4<R> *r, V4<R> *out, int tid,
                                           int nt) {
    switch (G) {
        case 1: bwd_rows<R, 1, CHUNK>(col, ldr, c0, c1, off0, qs, w, ws, lw, w0, r, out, tid, nt); break;
        case 2: bwd_rows<R, 2, CHUNK>(col, ldr, c0, c1, off0, qs, w, ws, lw, w0, r, out, tid, nt); break;
        case 4: bwd_rows<R, 4, CHUNK>(col, ldr, c0, c1, off0, qs, w, ws, lw, w0, r, out, tid, nt); break;
        case 8: bwd_rows<R, 8, CHUNK>(col, ldr, c0, c1, off0, qs, w, ws, lw, w0, r, out, tid, nt); break;
        case 16: bwd_rows<R, 16, CHUNK>(col, ldr, c0, c1, off0, qs, w, ws, lw, w0, r, out, tid, nt); break;
        default: bwd_rows<R, 32, CHUNK>(col, ldr, c0, c1, off0, qs, w, ws, lw, w0, r, out, tid, nt); break;
    }
}

// One backward work item (record `rec`, 5 int4; index `item` in the record
// array).  Shared memory: qs = the item's factor rows (qcap entries), then w
// (3 x lw entries), then the row indices of the entries of w past nc (lw int).
// A chunk item (rec[4].x >= 0) copies each of its rows' pieces separately and
// writes partial sums; the last chunk of its column block to finish adds the
// chunks' partials in chunk order and writes r.
template <typename R, typename Wait>
__device__ __forceinline__ void bwd_item(const DevSolve<R> &S, const int4 *rec, int item, int qcap, R *qs,
                                         uint64_t *bar, uint32_t parity, const V4<R> *z, V4<R> *r,
                                         Wait wait_inputs) {
    const int4 a = rec[0], b = rec[1], c = rec[2], e = rec[4];
    const int col = b.x, nc = b.y, nr = b.z, roff = b.w;
    const int c0 = c.x, c1 = c.y, ldr = c.z, off0 = c.w;
    const int rows = nc + nr;
    const bool chunk = e.x >= 0;
    // w = [z_C; -r_R] over [w0, w0 + lw): from the first row's diagonal start
    // to the end, or the chunk's entries
    const int w0 = chunk ? e.x : bwd_row_start(c0);
    const int lw = chunk ? e.y - e.x : ldr - w0;
    if (!chunk) {
        if (threadIdx.x == 0) bulk_load_issue(bar, qs, item_src(S.QB, a, sizeof(R)), (uint32_t)a.z);
    } else {
        if (threadIdx.x == 0) bulk_expect(bar, (uint32_t)a.z);
        const int j = c0 + (int)threadIdx.x;
        if (j < c1) {
            const int st = bwd_row_start(j);
            const int seg = st > w0 ? st : w0;
            const int len = w0 + lw - seg;
            if (len > 0) {
                const R *src = static_cast<const R *>(item_src(S.QB, a, sizeof(R))) + bwd_row_off(j, ldr) + (seg - st);
                bulk_copy(bar, qs + (size_t)(j - c0) * lw + (seg - w0), src, (uint32_t)(len * sizeof(R)));
            }
        }
    }
    R *w = qs + qcap;
    int *ridx = reinterpret_cast<int *>(w + 3 * lw);
    for (int k = threadIdx.x; k < lw; k += SBS) {
        const int i = w0 + k;
        ridx[k] = (i >= nc && i < rows) ? S.rows[roff + i - nc] : -1;
    }
    if (!wait_inputs()) {
        if (threadIdx.x == 0) bulk_load_wait(bar, parity);  // let the copies in flight land first
        return;
    }
#pragma unroll 4
    for (int k = threadIdx.x; k < lw; k += SBS) {
        const int i = w0 + k;
        R vx = R(0), vy = R(0), vz = R(0);
        if (i < nc) {
            const V4<R> v = ld_cg(z + col + i);
            vx = v.x; vy = v.y; vz = v.z;
        } else if (ridx[k] >= 0) {
            const V4<R> v = ld_cg(r + ridx[k]);
            vx = -v.x; vy = -v.y; vz = -v.z;
        }
        w[k] = vx; w[lw + k] = vy; w[2 * lw + k] = vz;
    }
    if (!bulk_load_finish(bar, parity, S.err)) return;
    if (!chunk) {
        bwd_rows_g<R, false>(a.w, col, ldr, c0, c1, off0, qs, w, lw, lw, w0, r, nullptr, (int)threadIdx.x, SBS);
        return;
    }
    const int nch = e.w >> 16, kch = e.w & 0xffff;
    if (nch == 1) {
        bwd_rows_g<R, true>(a.w, col, ldr, c0, c1, off0, qs, w, lw, lw, w0, r, nullptr, (int)threadIdx.x, SBS);
        return;
    }
    V4<R> *mine = S.part_r + (size_t)item * 32;
    bwd_rows_g<R, true>(a.w, col, ldr, c0, c1, off0, qs, w, lw, lw, w0, r, mine, (int)threadIdx.x, SBS);
    // the last chunk of the column block to get here combines the partials
    __shared__ int last;
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();  // release: the block's partial sums before the count
        last = atomicAdd(S.cb_cnt + e.z, 1) == nch - 1;
        if (last) __threadfence();  // acquire, ordered for the block by the barrier below
    }
    __syncthreads();
    if (!last) return;
    const V4<R> *first = S.part_r + (size_t)(item - kch) * 32;
    const int j = (int)threadIdx.x;
    if (j < c1 - c0) {
        R sx = R(0), sy = R(0), sz = R(0);
        for (int q = 0; q < nch; ++q) {
            const V4<R> p = ld_cg(first + (size_t)q * 32 + j);
            sx += p.x; sy += p.y; sz += p.z;
        }
        V4<R> o; o.x = sx; o.y = sy; o.z = sz; o.w = R(0);
        r[col + c0 + j] = o;
    }
    if (threadIdx.x == 0) S.cb_cnt[e.z] = 0;
}

template <typename R>
__global__ void __launch_bounds__(SBS, 4) k_bwd(DevSolve<R> S, int item0, int qcap, const V4<R> *z, V4<R> *r) {
    extern __shared__ __align__(128) unsigned char smem_raw[];
    __shared__ __align__(8) uint64_t bar;
    if (threadIdx.x == 0) bulk_bar_init(&bar);
    const int item = item0 + blockIdx.x;
    bwd_item<R>(S, S.bwd_items + 5 * (size_t)item, item, qcap, reinterpret_cast<R *>(smem_raw), &bar, 0u, z, r,
                []() {
                    pdl_trigger();
                    pdl_wait();
                    return true;
                });
}

// ---- dependency-driven schedule: one persistent launch per sweep
//
// Blocks take items from a queue (an atomic ticket) in topological order:
// forward items leaf level first, backward items root level first.  An item
// waits only for the items it reads from -- a forward item for every item of
// its supernode's children, a backward item for every item of its parent
// (whose own inputs were complete before it finished) -- by polling their
// supernodes' completion counters.  Because items are taken in topological
// order, every item waited on was taken earlier by a running block, so the
// waits end.  Each wait is bounded all the same: past the bound the block sets
// the error flag, and every later wait sees the flag and gives up at once.
// Each sweep resets the other sweep's counters and queue for the next solve.

constexpr long long kDepPolls = 1 << 22;

// Thread 0 waits until counter[sn] >= need (sn < 0: nothing to wait for).
__device__ __forceinline__ bool dep_wait(const int *counter, int sn, int need, unsigned int *err) {
    if (sn < 0) return true;
    const volatile int *c = counter + sn;
    for (long long it = 0; it < kDepPolls; ++it) {
        if (*c >= need) {
            __threadfence();
            return true;
        }
        if (*(volatile unsigned int *)err) return false;
        __nanosleep(32);
    }
    atomicOr(err, 2u);
    return false;
}

// Block-uniform: false once any block has flagged an error.
__device__ __forceinline__ bool still_ok(const unsigned int *err) {
    __shared__ int ok;
    __syncthreads();
    if (threadIdx.x == 0) ok = *(const volatile unsigned int *)err == 0u;
    __syncthreads();
    return ok != 0;
}

// After the block's outputs of an item are written: publish them.
__device__ __forceinline__ void dep_signal(int *counter, int sn) {
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        atomicAdd(counter + sn, 1);
    }
}

template <typename R>
__global__ void __launch_bounds__(SBS) k_fwd_dyn(DevSolve<R> S, int qcap, const V4<R> *rhs, V4<R> *z) {
    extern __shared__ __align__(128) unsigned char smem_raw[];
    __shared__ __align__(8) uint64_t bar;
    __shared__ int item_sh, ok_sh;
    R *qs = reinterpret_cast<R *>(smem_raw);
    for (int i = blockIdx.x * SBS + threadIdx.x; i < S.n_sn; i += gridDim.x * SBS) S.bwd_done[i] = 0;
    if (blockIdx.x == 0 && threadIdx.x == 0) S.queue[1] = 0;
    if (threadIdx.x == 0) bulk_bar_init(&bar);
    uint32_t parity = 0;
    for (;;) {
        if (threadIdx.x == 0) item_sh = (int)atomicAdd(&S.queue[0], 1u);
        __syncthreads();
        const int item = item_sh;
        if (item >= S.n_fwd_items) break;
        const int4 *rec = S.fwd_items + 5 * (size_t)item;
        const int4 dep = rec[3];  // children c0 .. c3 (-1: none)
        const int own = rec[4].x;
        fwd_item<R>(S, rec, qcap, qs, &bar, parity, rhs, z, [&]() {
            if (threadIdx.x == 0)
                ok_sh = dep_wait(S.fwd_done, dep.x, dep.x >= 0 ? S.fwd_nitems[dep.x] : 0, S.err) &&
                        dep_wait(S.fwd_done, dep.y, dep.y >= 0 ? S.fwd_nitems[dep.y] : 0, S.err) &&
                        dep_wait(S.fwd_done, dep.z, dep.z >= 0 ? S.fwd_nitems[dep.z] : 0, S.err) &&
                        dep_wait(S.fwd_done, dep.w, dep.w >= 0 ? S.fwd_nitems[dep.w] : 0, S.err);
            __syncthreads();
            return ok_sh != 0;
        });
        if (!still_ok(S.err)) break;
        dep_signal(S.fwd_done, own);
        parity ^= 1u;
    }
}

template <typename R>
__global__ void __launch_bounds__(SBS) k_bwd_dyn(DevSolve<R> S, int qcap, const V4<R> *z, V4<R> *r) {
    extern __shared__ __align__(128) unsigned char smem_raw[];
    __shared__ __align__(8) uint64_t bar;
    __shared__ int item_sh, ok_sh;
    R *qs = reinterpret_cast<R *>(smem_raw);
    for (int i = blockIdx.x * SBS + threadIdx.x; i < S.n_sn; i += gridDim.x * SBS) S.fwd_done[i] = 0;
    if (blockIdx.x == 0 && threadIdx.x == 0) S.queue[0] = 0;
    if (threadIdx.x == 0) bulk_bar_init(&bar);
    uint32_t parity = 0;
    for (;;) {
        if (threadIdx.x == 0) item_sh = (int)atomicAdd(&S.queue[1], 1u);
        __syncthreads();
        const int item = item_sh;
        if (item >= S.n_bwd_items) break;
        const int4 *rec = S.bwd_items + 5 * (size_t)item;
        const int4 dep = rec[3];  // parent (-1: none), own supernode
        bwd_item<R>(S, rec, item, qcap, qs, &bar, parity, z, r, [&]() {
            if (threadIdx.x == 0) ok_sh = dep_wait(S.bwd_done, dep.x, dep.x >= 0 ? S.bwd_nitems[dep.x] : 0, S.err);
            __syncthreads();
            return ok_sh != 0;
        });
        if (!still_ok(S.err)) break;
        dep_signal(S.bwd_done, dep.y);
        parity ^= 1u;
    }
}

// ---- pipelined schedule: one persistent launch per sweep, one block per SM
//
// Each block owns a fixed list of bundles (consecutive items of one tree
// level), in level order: ascending for the forward sweep, descending for the
// backward one.  Its last warp is a producer: it streams the factor rows of
// the block's items, in order, into a ring of shared-memory slots (one bulk
// copy per item, completion on the slot's `full` mbarrier) as soon as the
// consumers release a slot (its `empty` mbarrier, one arrival per consumer
// warp) -- the factor does not depend on the sweep, so the stream runs ahead
// across levels while the consumers wait for other blocks.  The other warps
// consume a bundle in four steps: wait until the items it reads from (other
// blocks' or its own) have published, gather the vector its rows multiply
// into the vector area (one segment per supernode), run its items' row dot
// products from the ring, then publish (per-supernode completion counters).
//
// Progress: every block's waits are on items of earlier levels only, and the
// grid is at most one block per SM with all blocks resident (the launch
// asks for exactly the blocks that fit), so the lowest unfinished level
// always advances.  Every wait is bounded; past the bound the block sets the
// error flag, skips its remaining work and, before it exits, waits (bounded)
// for the copies it has in flight.

constexpr int PCONS = 32 * PIPE_CONS_WARPS;  // consumer threads of a pipelined sweep block
constexpr int PTHREADS = PCONS + 32;        // plus one producer warp
constexpr int PIPE_SLOT = 32768;            // bytes per ring slot (the host's item bound)
constexpr long long kEmptyPolls = 1 << 22;  // bound on the producer's wait for a free slot

struct PipeShared {
    uint64_t full[PIPE_NS_MAX];   // slot holds its item's rows (bulk-copy bytes arrived)
    uint64_t empty[PIPE_NS_MAX];  // slot released by every consumer warp
    int abort;                    // set by a thread that gave up; ends the block's work
    int k_issued;                 // items whose copies the producer has started
    int seg_aoff[PIPE_SEG_MAX];   // vector-area offsets of the bundle's segments
    int4 seg[2 * PIPE_SEG_MAX];
    int mine[PIPE_CMB_MAX];       // this bundle completed the column block: it combines it
};

__device__ __forceinline__ void cons_sync() { asm volatile("bar.sync 1, %0;" ::"n"(PCONS) : "memory"); }
// Consumer barrier that also returns, to every consumer, whether any of them
// passed true.
__device__ __forceinline__ bool cons_any(bool v) {
    uint32_t r;
    asm volatile(
        "{\n .reg .pred p, q;\n setp.ne.u32 p, %1, 0;\n bar.red.or.pred q, 1, %2, p;\n selp.u32 %0, 1, 0, q;\n}\n"
        : "=r"(r)
        : "r"((uint32_t)v), "n"(PCONS)
        : "memory");
    return r != 0;
}

__device__ __forceinline__ void mbar_init(uint64_t *bar, unsigned count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint64_t *bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_addr(bar)) : "memory");
}
__device__ __forceinline__ bool mbar_test(uint64_t *bar, uint32_t parity) {
    uint32_t done;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(done)
        : "r"(smem_addr(bar)), "r"(parity)
        : "memory");
    return done != 0;
}

// Producer warp: items [it0, it1) of the block, slot k % ns for the k-th.
template <typename R, bool BWD>
__device__ void pipe_produce(const DevSolve<R> &S, int it0, int it1, R *ring, PipeShared &sh, int ns) {
    constexpr int SLOT_E = PIPE_SLOT / (int)sizeof(R);
    const int lane = threadIdx.x & 31;
    volatile int *abort = &sh.abort;
    for (int it = it0; it < it1; ++it) {
        const int k = it - it0, slot = k % ns, use = k / ns;
        int ok = 1;
        if (lane == 0) {
            if (use > 0) {
                ok = 0;
                for (long long p = 0; p < kEmptyPolls && !*abort; ++p)
                    if (mbar_test(&sh.empty[slot], (uint32_t)((use - 1) & 1))) {
                        ok = 1;
                        break;
                    }
                if (!ok && !*abort) {
                    atomicOr(S.err, 8u);
                    *abort = 1;
                }
            }
            if (*abort) ok = 0;
        }
        if (!__shfl_sync(0xffffffffu, ok, 0)) break;  // lane 0 decides for the warp
        R *dst = ring + (size_t)slot * SLOT_E;
        if (!BWD) {
            const int4 a = S.pf_items[4 * (size_t)it];
            if (lane == 0) bulk_load_issue(&sh.full[slot], dst, item_src(S.QF, a, sizeof(R)), (uint32_t)a.z);
        } else {
            const int4 *rec = S.pb_items + 5 * (size_t)it;
            const int4 a = rec[0], e = rec[4];
            if (e.x < 0) {
                if (lane == 0) bulk_load_issue(&sh.full[slot], dst, item_src(S.QB, a, sizeof(R)), (uint32_t)a.z);
            } else {
                // a chunk item: row j's piece [max(e0, start_j), e1) at dst + (j - c0) lw
                const int4 c = rec[2];
                const int c0 = c.x, c1 = c.y, ldr = c.z;
                const int w0 = e.x, lw = e.y - e.x;
                if (lane == 0) bulk_expect(&sh.full[slot], (uint32_t)a.z);
                const int j = c0 + lane;
                if (j < c1) {
                    const int st = bwd_row_start(j);
                    const int seg = st > w0 ? st : w0;
                    const int len = w0 + lw - seg;
                    if (len > 0) {
                        const R *src =
                            static_cast<const R *>(item_src(S.QB, a, sizeof(R))) + bwd_row_off(j, ldr) + (seg - st);
                        bulk_copy(&sh.full[slot], dst + (size_t)(j - c0) * lw + (seg - w0), src,
                                  (uint32_t)(len * sizeof(R)));
                    }
                }
            }
        }
        __syncwarp();
        if (lane == 0) sh.k_issued = k + 1;
    }
}

// Segment of vector-area entry e: the last one starting at or before it.
__device__ __forceinline__ int pipe_seg_of(const PipeShared &sh, int nseg, int e) {
    int lo = 0, hi = nseg - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (sh.seg_aoff[mid] <= e) lo = mid; else hi = mid - 1;
    }
    return lo;
}

// Gathers take PG entries per thread at a time: every load of a round is
// issued before any result is used, so a round costs two dependent trips to
// memory (index, then value) whatever PG is.
constexpr int PG = 4;

// Consumers, forward: f = q_C - (child updates on C) for every segment.
template <typename R>
__device__ __forceinline__ void pipe_gather_fwd(const DevSolve<R> &S, const PipeShared &sh, int nseg, int ftot, R *F,
                                                int fcap, const V4<R> *rhs) {
    for (int base = threadIdx.x; base < ftot; base += PG * PCONS) {
        V4<R> v[PG];
        int4 ci[PG];
#pragma unroll
        for (int g = 0; g < PG; ++g) {
            const int e = base + g * PCONS;
            v[g].x = v[g].y = v[g].z = v[g].w = R(0);
            ci[g] = make_int4(-1, -1, -1, -1);
            if (e < ftot) {
                const int4 sg = sh.seg[pipe_seg_of(sh, nseg, e)];  // {col, filled, area offset, length}
                const int j = e - sg.z;
                if (j < sg.y) {
                    v[g] = ld_cg(rhs + sg.x + j);
                    ci[g] = __ldg(S.fg4 + sg.x + j);
                }
            }
        }
        V4<R> a[PG], b[PG], c[PG], d[PG];
#pragma unroll
        for (int g = 0; g < PG; ++g) {
            a[g].x = a[g].y = a[g].z = R(0);
            b[g] = a[g]; c[g] = a[g]; d[g] = a[g];
            if (ci[g].x >= 0) a[g] = ld_cg(S.u + ci[g].x);
            if (ci[g].y >= 0) b[g] = ld_cg(S.u + ci[g].y);
            if (ci[g].z >= 0) c[g] = ld_cg(S.u + ci[g].z);
            if (ci[g].w >= 0) d[g] = ld_cg(S.u + ci[g].w);
        }
#pragma unroll
        for (int g = 0; g < PG; ++g) {
            const int e = base + g * PCONS;
            if (e < ftot) {
                F[e] = v[g].x - a[g].x - b[g].x - c[g].x - d[g].x;
                F[fcap + e] = v[g].y - a[g].y - b[g].y - c[g].y - d[g].y;
                F[2 * fcap + e] = v[g].z - a[g].z - b[g].z - c[g].z - d[g].z;
            }
        }
    }
}

// Consumers, backward: w = [z_C; -r_R] over each segment's range.
template <typename R>
__device__ __forceinline__ void pipe_gather_bwd(const DevSolve<R> &S, const PipeShared &sh, int nseg, int ftot, R *F,
                                                int fcap, const V4<R> *z, const V4<R> *r) {
    for (int base = threadIdx.x; base < ftot; base += PG * PCONS) {
        int src[PG];
        R sgn[PG];
#pragma unroll
        for (int g = 0; g < PG; ++g) {
            const int e = base + g * PCONS;
            src[g] = -1;
            sgn[g] = R(1);
            if (e < ftot) {
                const int q = pipe_seg_of(sh, nseg, e);
                const int4 sa = sh.seg[2 * q], sb = sh.seg[2 * q + 1];  // {col, nc, nrow, roff} {w0, aoff, len, 0}
                const int i = sb.x + (e - sb.y);
                if (i < sa.y) {
                    src[g] = sa.x + i;
                } else if (i < sa.y + sa.z) {
                    src[g] = __ldg(S.rows + sa.w + i - sa.y);
                    sgn[g] = R(-1);
                }
            }
        }
        V4<R> v[PG];
#pragma unroll
        for (int g = 0; g < PG; ++g) {
            v[g].x = v[g].y = v[g].z = R(0);
            if (src[g] >= 0) v[g] = ld_cg((sgn[g] > R(0) ? z : r) + src[g]);
        }
#pragma unroll
        for (int g = 0; g < PG; ++g) {
            const int e = base + g * PCONS;
            if (e < ftot) {
                F[e] = sgn[g] * v[g].x;
                F[fcap + e] = sgn[g] * v[g].y;
                F[2 * fcap + e] = sgn[g] * v[g].z;
            }
        }
    }
}

// Consumer warps: bundles [b0, b1) of the block, whose items start at it0.
// Forward: in = q, out = z.  Backward: in = z, out = r.
template <typename R, bool BWD>
__device__ void pipe_consume(const DevSolve<R> &S, int b0, int b1, int it0, const R *ring, R *F, PipeShared &sh,
                             const V4<R> *in, V4<R> *out) {
    constexpr int SLOT_E = PIPE_SLOT / (int)sizeof(R);
    const int tid = threadIdx.x;
    const int ns = S.pipe_ns, fcap = S.pipe_fcap;
    const int4 *bund = BWD ? S.pb_bund : S.pf_bund;
    const int4 *segs = BWD ? S.pb_seg : S.pf_seg;
    const int2 *dep = BWD ? S.pb_dep : S.pf_dep;
    const int2 *sig = BWD ? S.pb_sig : S.pf_sig;
    int *done = BWD ? S.bwd_done : S.fwd_done;
    volatile int *abort = &sh.abort;
    for (int b = b0; b < b1; ++b) {
        const int4 B0 = bund[3 * (size_t)b], B1 = bund[3 * (size_t)b + 1], B2 = bund[3 * (size_t)b + 2];
        // 1. the items this bundle reads from have published
        if (tid < B1.y - B1.x) {
            const int2 d = dep[B1.x + tid];
            if (!dep_wait(done, d.x, d.y, S.err)) *abort = 1;
        }
        if (tid == 0 && *(volatile unsigned int *)S.err) *abort = 1;
        const int nseg = B0.w - B0.z;
        for (int i = tid; i < nseg; i += PCONS) {
            if (BWD) {
                const int4 sa = segs[2 * (size_t)(B0.z + i)], sb = segs[2 * (size_t)(B0.z + i) + 1];
                sh.seg[2 * i] = sa;
                sh.seg[2 * i + 1] = sb;
                sh.seg_aoff[i] = sb.y;
            } else {
                const int4 sg = segs[B0.z + i];
                sh.seg[i] = sg;
                sh.seg_aoff[i] = sg.z;
            }
        }
        if (cons_any(*abort)) break;
        // 2. the vector the rows multiply
        if (BWD) pipe_gather_bwd<R>(S, sh, nseg, B2.z, F, fcap, in, out);
        else pipe_gather_fwd<R>(S, sh, nseg, B2.z, F, fcap, in);
        cons_sync();
        // 3. the items, from the ring: all of the bundle's items are resident
        // at once (the host keeps a bundle within half the ring); each runs on
        // its own range of consumer warps (item record: warps [w0, w1))
        bool ready = true;
        for (int it = B0.x; it < B0.y; ++it) {
            const int k = it - it0;
            ready = ready && bulk_load_wait(&sh.full[k % ns], (uint32_t)((k / ns) & 1));
        }
        if (!ready) *abort = 1;
        if (cons_any(!ready || *abort)) break;
        {
            const int warp = tid >> 5;
            int it = B0.x;
            int4 d = BWD ? S.pb_items[5 * (size_t)it + 3] : S.pf_items[4 * (size_t)it + 3];
            while (warp >= d.w && it + 1 < B0.y) {
                ++it;
                d = BWD ? S.pb_items[5 * (size_t)it + 3] : S.pf_items[4 * (size_t)it + 3];
            }
            const int k = it - it0;
            const R *qs = ring + (size_t)(k % ns) * SLOT_E;
            const int ltid = tid - 32 * d.z, lnt = 32 * (d.w - d.z);
            if (!BWD) {
                const int4 *rec = S.pf_items + 4 * (size_t)it;
                const int4 a = rec[0], bb = rec[1], c = rec[2];
                fwd_rows_g<R>(a.w, S, bb.x, bb.y, bb.z, bb.w, c.x, c.y, c.w, qs, F + d.x, fcap, out, ltid, lnt);
            } else {
                const int4 *rec = S.pb_items + 5 * (size_t)it;
                const int4 a = rec[0], bb = rec[1], c = rec[2], e = rec[4];
                const int c0 = c.x, c1 = c.y, ldr = c.z, off0 = c.w;
                if (e.x < 0) {
                    const int w0 = bwd_row_start(c0);
                    bwd_rows_g<R, false>(a.w, bb.x, ldr, c0, c1, off0, qs, F + d.x, fcap, ldr - w0, w0, out, nullptr,
                                         ltid, lnt);
                } else {
                    const int nch = e.w >> 16, kch = e.w & 0xffff;
                    V4<R> *part = nch > 1 ? S.pb_part + (size_t)(d.y + kch) * 32 : nullptr;
                    bwd_rows_g<R, true>(a.w, bb.x, ldr, c0, c1, off0, qs, F + d.x, fcap, e.y - e.x, e.x, out, part,
                                        ltid, lnt);
                }
            }
            __syncwarp();
            if ((tid & 31) == 0)
                for (int q = B0.x; q < B0.y; ++q) mbar_arrive(&sh.empty[(q - it0) % ns]);
        }
        if (cons_any(*abort)) break;
        // 4. (backward) column blocks whose last chunks this bundle ran: add
        // the chunks' partial sums in chunk order
        if (BWD && B2.y > B2.x) {
            const int ncmb = B2.y - B2.x;
            if (tid < ncmb) {
                const int4 c = S.pb_cmb[2 * (size_t)(B2.x + tid)];  // {column block, count, pslot0, nch}
                __threadfence();
                sh.mine[tid] = atomicAdd(S.pb_cbc + c.x, c.y) + c.y == c.w;
            }
            cons_sync();
            for (int q = 0; q < ncmb; ++q) {
                if (!sh.mine[q]) continue;
                const int4 c = S.pb_cmb[2 * (size_t)(B2.x + q)], o = S.pb_cmb[2 * (size_t)(B2.x + q) + 1];
                __threadfence();
                if (tid < o.y) {
                    R sx = R(0), sy = R(0), sz = R(0);
                    for (int kk = 0; kk < c.w; ++kk) {
                        const V4<R> p = ld_cg(S.pb_part + (size_t)(c.z + kk) * 32 + tid);
                        sx += p.x; sy += p.y; sz += p.z;
                    }
                    V4<R> v; v.x = sx; v.y = sy; v.z = sz; v.w = R(0);
                    out[o.x + tid] = v;
                }
                if (tid == 0) S.pb_cbc[c.x] = 0;
            }
            cons_sync();
        }
        // 5. publish
        if (tid < B1.w - B1.z) {
            const int2 g = sig[B1.z + tid];
            __threadfence();
            atomicAdd(done + g.x, g.y);
        }
    }
}

template <typename R, bool BWD>
__global__ void __launch_bounds__(PTHREADS, 1) k_pipe(DevSolve<R> S, const V4<R> *in, V4<R> *out) {
    extern __shared__ __align__(128) unsigned char smem_raw[];
    __shared__ PipeShared sh;
    constexpr int SLOT_E = PIPE_SLOT / (int)sizeof(R);
    const int ns = S.pipe_ns;
    R *ring = reinterpret_cast<R *>(smem_raw);
    R *F = ring + (size_t)ns * SLOT_E;
    const int tid = threadIdx.x;
    // the other sweep's counters start from zero in the next solve
    int *other = BWD ? S.fwd_done : S.bwd_done;
    for (int i = blockIdx.x * PTHREADS + tid; i < S.n_sn; i += gridDim.x * PTHREADS) other[i] = 0;
    if (tid == 0) {
        for (int q = 0; q < ns; ++q) {
            mbar_init(&sh.full[q], 1);
            mbar_init(&sh.empty[q], PCONS / 32);
        }
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        sh.abort = 0;
        sh.k_issued = 0;
    }
    __syncthreads();
    const int *blk = BWD ? S.pb_blk : S.pf_blk;
    const int4 *bund = BWD ? S.pb_bund : S.pf_bund;
    const int b0 = blk[blockIdx.x], b1 = blk[blockIdx.x + 1];
    if (b1 > b0) {
        const int it0 = bund[3 * (size_t)b0].x, it1 = bund[3 * (size_t)(b1 - 1)].y;
        if (tid >= PCONS) pipe_produce<R, BWD>(S, it0, it1, ring, sh, ns);
        else pipe_consume<R, BWD>(S, b0, b1, it0, ring, F, sh, in, out);
    }
    __syncthreads();
    // copies still in flight land before the block exits (only after an error
    // can the last use of a slot be unconsumed)
    if (tid == 0 && sh.abort) {
        const int n = sh.k_issued;
        for (int q = 0; q < ns && q < n; ++q) {
            const int last = q + ((n - 1 - q) / ns) * ns;
            if (!bulk_load_wait(&sh.full[q], (uint32_t)((last / ns) & 1))) atomicOr(S.err, 4u);
        }
    }
}

// Dynamic shared memory of a sweep block: qcap factor entries, 3 x ld vector
// entries and ld 16-byte index slots.
template <typename R>
size_t sweep_smem(int qcap, int ld) {
    return ((size_t)qcap + 3 * (size_t)ld) * sizeof(R) + 16 * (size_t)ld;
}

// Dynamic shared memory of a pipelined sweep block: ns ring slots and the
// vector area (three components of fcap entries).
template <typename R>
size_t pipe_smem(int ns, int fcap) {
    return (size_t)ns * PIPE_SLOT + 3 * (size_t)fcap * sizeof(R);
}

// One level's launch, with the programmatic-serialisation attribute when
// the handle chains levels.
template <typename R, typename... Args>
void launch_level(bool pdl, void (*kernel)(DevSolve<R>, int, int, Args...), int grid, size_t smem, cudaStream_t st,
                  const DevSolve<R> &s, int item0, int qcap, Args... args) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)grid);
    cfg.blockDim = dim3(SBS);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = pdl ? 1 : 0;
    cudaLaunchKernelEx(&cfg, kernel, s, item0, qcap, args...);
}

}  // namespace

template <typename R> int solve_smem_limit_ok(int max_ld) {
    return sweep_smem<R>(65536 / (int)sizeof(R), max_ld) <= (size_t)SOLVE_MAX_SMEM;
}

template <typename R> cudaError_t solve_prepare() {
    cudaError_t e = cudaFuncSetAttribute(k_fwd<R>, cudaFuncAttributeMaxDynamicSharedMemorySize, SOLVE_MAX_SMEM);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(k_bwd<R>, cudaFuncAttributeMaxDynamicSharedMemorySize, SOLVE_MAX_SMEM);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_fwd_dyn<R>, cudaFuncAttributeMaxDynamicSharedMemorySize, SOLVE_MAX_SMEM);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_bwd_dyn<R>, cudaFuncAttributeMaxDynamicSharedMemorySize, SOLVE_MAX_SMEM);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_pipe<R, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, PIPE_MAX_SMEM);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_pipe<R, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, PIPE_MAX_SMEM);
    return e;
}

// Ring slots for a vector area of fcap entries (as many as fit, at most
// PIPE_NS_MAX, at least 2) and the blocks of one launch: one per SM, all
// resident at once.
template <typename R> int solve_pipe_grid(int fcap, int *ns_out) {
    const size_t area = 3 * (size_t)fcap * sizeof(R);
    if (area + 2 * (size_t)PIPE_SLOT > (size_t)PIPE_MAX_SMEM) return 0;
    int ns = (int)((PIPE_MAX_SMEM - area) / PIPE_SLOT);
    if (ns > PIPE_NS_MAX) ns = PIPE_NS_MAX;
    int dev = 0, sms = 0, per_f = 0, per_b = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return 0;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return 0;
    const size_t smem = pipe_smem<R>(ns, fcap);
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_f, k_pipe<R, false>, PTHREADS, smem) != cudaSuccess)
        return 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_b, k_pipe<R, true>, PTHREADS, smem) != cudaSuccess)
        return 0;
    if (per_f < 1 || per_b < 1) return 0;
    *ns_out = ns;
    return sms;
}

template <typename R>
void launch_solve(const DevSolve<R> &s, const V4<R> *q, V4<R> *z, V4<R> *r, cudaStream_t st) {
    if (s.pipe) {
        const size_t smem = pipe_smem<R>(s.pipe_ns, s.pipe_fcap);
        k_pipe<R, false><<<s.pipe_grid, PTHREADS, smem, st>>>(s, q, z);
        k_pipe<R, true><<<s.pipe_grid, PTHREADS, smem, st>>>(s, (const V4<R> *)z, r);
        return;
    }
    if (s.dyn) {
        k_fwd_dyn<R><<<s.dyn_grid, SBS, sweep_smem<R>(s.fwd_qmax, s.fwd_ldmax), st>>>(s, s.fwd_qmax, q, z);
        k_bwd_dyn<R><<<s.dyn_grid, SBS, sweep_smem<R>(s.bwd_qmax, s.bwd_ldmax), st>>>(s, s.bwd_qmax, z, r);
        return;
    }
    for (int l = 0; l < s.n_levels; ++l) {
        const int a = s.fwd_lvl_ptr[l], b = s.fwd_lvl_ptr[l + 1];
        if (b > a)
            launch_level<R, const V4<R> *, V4<R> *>(s.pdl != 0, k_fwd<R>, b - a,
                                                     sweep_smem<R>(s.fwd_lvl_q[l], s.fwd_lvl_ld[l]), st, s, a,
                                                     s.fwd_lvl_q[l], q, z);
    }
    for (int l = s.n_levels - 1; l >= 0; --l) {
        const int a = s.bwd_lvl_start[l], cnt = s.bwd_lvl_cnt[l];
        if (cnt > 0)
            launch_level<R, const V4<R> *, V4<R> *>(s.pdl != 0, k_bwd<R>, cnt,
                                                     sweep_smem<R>(s.bwd_lvl_q[l], s.bwd_lvl_ld[l]), st, s, a,
                                                     s.bwd_lvl_q[l], (const V4<R> *)z, r);
    }
}

// Blocks of the persistent sweeps that fit on the device at once (the grid of
// the dependency-driven schedule must be co-resident only for speed, not for
// progress: items are taken in topological order).
template <typename R> int solve_dyn_grid(const DevSolve<R> &s) {
    int dev = 0, sms = 0, per_sm_f = 0, per_sm_b = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return 0;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm_f, k_fwd_dyn<R>, SBS,
                                                      sweep_smem<R>(s.fwd_qmax, s.fwd_ldmax)) != cudaSuccess)
        return 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm_b, k_bwd_dyn<R>, SBS,
                                                      sweep_smem<R>(s.bwd_qmax, s.bwd_ldmax)) != cudaSuccess)
        return 0;
    const int per_sm = per_sm_f < per_sm_b ? per_sm_f : per_sm_b;
    return per_sm > 0 ? per_sm * sms : 0;
}

template void launch_solve<float>(const DevSolve<float> &, const V4<float> *, V4<float> *, V4<float> *, cudaStream_t);
template void launch_solve<double>(const DevSolve<double> &, const V4<double> *, V4<double> *, V4<double> *, cudaStream_t);
template int solve_dyn_grid<float>(const DevSolve<float> &);
template int solve_dyn_grid<double>(const DevSolve<double> &);
template int solve_pipe_grid<float>(int, int *);
template int solve_pipe_grid<double>(int, int *);
template int solve_smem_limit_ok<float>(int);
template int solve_smem_limit_ok<double>(int);
template cudaError_t solve_prepare<float>();
template cudaError_t solve_prepare<double>();

}  // namespace hqn
