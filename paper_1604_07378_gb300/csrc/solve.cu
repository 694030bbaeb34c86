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
//
// The factor does not depend on the solve's data, only the vectors do.  So
// each level's blocks, as they start, also ask L2 to prefetch the factor rows
// of the level `prefetch` launches ahead (cp.async.bulk.prefetch.L2, spans
// listed by the host): the stream of the factor out of HBM runs ahead of the
// chain of levels, and a level's own bulk copies then read L2.
//
// When the top levels are solved by the dense block, the forward launches
// before it may also prefetch its matrix into L2 the same way
// (solve_dense_prefetch).
//
// Every wait is bounded (wait_polls polls of the copy's mbarrier); past the
// bound the block flags the error in the handle's control block and leaves
// without reading its buffer, after its copy in flight, if any, has landed
// (itself a bounded wait).  The host reports HQN_ERR_DEVICE_TIMEOUT.  For
// tests of that path, fault_test = 1 makes the first level's blocks skip
// their copies, so their waits run out with nothing in flight.
#include "kernels.cuh"
#include "layout.hpp"
#include "reduce.cuh"

namespace hqn {

namespace {

constexpr long long kDrainPolls = 1LL << 26;  // bound on waiting for a copy in flight after a timeout

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

// Polls the barrier's phase `parity` at most `polls` times.
__device__ __forceinline__ bool bulk_load_wait(uint64_t *bar, uint32_t parity, long long polls) {
    for (long long it = 0; it < polls; ++it) {
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
// within `polls` polls; the block must then leave without reading the buffer.
// A block must not exit while a bulk copy into its shared memory is in
// flight, so after a timeout thread 0 keeps waiting for an issued copy (up to
// kDrainPolls polls, flagging bit 4 if even that runs out) before it returns;
// the block ends only when thread 0 does.
__device__ __forceinline__ bool bulk_load_finish(uint64_t *bar, uint32_t parity, unsigned int *err, long long polls,
                                                 bool issued) {
    __shared__ int timed_out;
    if (threadIdx.x == 0) timed_out = 0;
    __syncthreads();
    if (!bulk_load_wait(bar, parity, polls)) timed_out = 1;
    __syncthreads();
    if (timed_out) {
        if (threadIdx.x == 0) {
            atomicOr(err, 1u);
            if (issued && !bulk_load_wait(bar, parity, kDrainPolls)) atomicOr(err, 4u);
        }
        return false;
    }
    return true;
}

// Asks L2 to fetch `bytes` (a multiple of 16) at the 16-byte aligned address p.
__device__ __forceinline__ void l2_prefetch(const void *p, uint32_t bytes) {
    asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(p), "r"(bytes) : "memory");
}

// Thread 0 of every block of a level: its share of the prefetch spans
// {address lo, address hi, bytes, 0} of the level `prefetch` launches ahead.
__device__ __forceinline__ void prefetch_ahead(const int4 *pf, int pf_n) {
    if (threadIdx.x != 0) return;
    for (int j = blockIdx.x; j < pf_n; j += gridDim.x) {
        const int4 a = pf[j];
        const unsigned long long addr = (unsigned long long)(unsigned)a.x | ((unsigned long long)(unsigned)a.y << 32);
        l2_prefetch(reinterpret_cast<const void *>(addr), (uint32_t)a.z);
    }
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
// after the wait on the previous level, so the row products read only
// shared memory.  NT threads per block.
template <typename R, int NT>
__device__ __forceinline__ void fwd_item(const DevSolve<R> &S, const int4 *rec, int qcap, R *qs, uint64_t *bar,
                                         const V4<R> *rhs, V4<R> *z, bool issue, const int4 *pf, int pf_n) {
    const int4 a = rec[0];
    if (threadIdx.x == 0 && issue) bulk_load_issue(bar, qs, item_src(S.QF, a, sizeof(R)), (uint32_t)a.z);
    prefetch_ahead(pf, pf_n);
    const int4 b = rec[1], c = rec[2];
    const int col = b.x, nc = b.y, ldc = b.z, uoff = b.w;
    const int r0 = c.x, r1 = c.y, ldf = c.z, off0 = c.w;
    const int rr0 = r0 > nc ? r0 : nc, nrr = r1 > rr0 ? r1 - rr0 : 0, nrr4 = pad4(nrr);
    R *f = qs + qcap;
    R *ua = f + 3 * ldf;
    int4 *cidx = reinterpret_cast<int4 *>(ua + 3 * nrr4);
    int4 *ridx = cidx + ldf;
    const int nf = ldf < nc ? ldf : nc;
    for (int j = threadIdx.x; j < nf; j += NT) cidx[j] = __ldg(S.fg4 + col + j);
    for (int j = threadIdx.x; j < nrr; j += NT) ridx[j] = __ldg(S.ug4 + uoff + rr0 - nc + j);
    pdl_trigger();
    pdl_wait();
    // f = q_C - (child updates on C), entries [0, ldf), zero beyond nc; and
    // the child updates landing on the rectangle rows
    const int nj = ldf > nrr ? ldf : nrr;
#pragma unroll 2
    for (int j = threadIdx.x; j < nj; j += NT) {
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
    if (!bulk_load_finish(bar, 0u, S.err, S.wait_polls, issue)) return;
    fwd_rows_g<R>(a.w, S, col, nc, ldc, uoff, r0, r1, off0, qs, f, ldf, z, (int)threadIdx.x, NT, ua, nrr4, rr0);
}

// One launch per tree level, one item per block.  skip_copy (fault tests
// only): the block issues no copy, so its wait runs out.
template <typename R, int NT>
__global__ void __launch_bounds__(NT, 1024 / NT) k_fwd(DevSolve<R> S, int item0, int qcap, const V4<R> *rhs,
                                                       V4<R> *z, const int4 *pf, int pf_n, int skip_copy) {
    extern __shared__ __align__(128) unsigned char smem_raw[];
    __shared__ __align__(8) uint64_t bar;
    if (threadIdx.x == 0) bulk_bar_init(&bar);
    fwd_item<R, NT>(S, S.fwd_items + 5 * (size_t)(item0 + blockIdx.x), qcap, reinterpret_cast<R *>(smem_raw), &bar,
                    rhs, z, skip_copy == 0, pf, pf_n);
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
template <typename R, int NT>
__device__ __forceinline__ void bwd_item(const DevSolve<R> &S, const int4 *rec, int item, int qcap, R *qs,
                                         uint64_t *bar, const V4<R> *z, V4<R> *r, const int4 *pf, int pf_n) {
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
    prefetch_ahead(pf, pf_n);
    R *w = qs + qcap;
    int *ridx = reinterpret_cast<int *>(w + 3 * lw);
    for (int k = threadIdx.x; k < lw; k += NT) {
        const int i = w0 + k;
        ridx[k] = (i >= nc && i < rows) ? S.rows[roff + i - nc] : -1;
    }
    pdl_trigger();
    pdl_wait();
#pragma unroll 4
    for (int k = threadIdx.x; k < lw; k += NT) {
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
    if (!bulk_load_finish(bar, 0u, S.err, S.wait_polls, true)) return;
    if (!chunk) {
        bwd_rows_g<R, false>(a.w, col, ldr, c0, c1, off0, qs, w, lw, lw, w0, r, nullptr, (int)threadIdx.x, NT);
        return;
    }
    const int nch = e.w >> 16, kch = e.w & 0xffff;
    if (nch == 1) {
        bwd_rows_g<R, true>(a.w, col, ldr, c0, c1, off0, qs, w, lw, lw, w0, r, nullptr, (int)threadIdx.x, NT);
        return;
    }
    V4<R> *mine = S.part_r + (size_t)item * 32;
    bwd_rows_g<R, true>(a.w, col, ldr, c0, c1, off0, qs, w, lw, lw, w0, r, mine, (int)threadIdx.x, NT);
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

template <typename R, int NT>
__global__ void __launch_bounds__(NT, 1024 / NT) k_bwd(DevSolve<R> S, int item0, int qcap, const V4<R> *z, V4<R> *r,
                                                       const int4 *pf, int pf_n) {
    extern __shared__ __align__(128) unsigned char smem_raw[];
    __shared__ __align__(8) uint64_t bar;
    if (threadIdx.x == 0) bulk_bar_init(&bar);
    const int item = item0 + blockIdx.x;
    bwd_item<R, NT>(S, S.bwd_items + 5 * (size_t)item, item, qcap, reinterpret_cast<R *>(smem_raw), &bar, z, r, pf,
                    pf_n);
}

// ---- dense top block
//
// The supernodes of the tree's top levels are solved together (solve_dense_top):
// r_T = S^{-1} f_T, with S^{-1} (the inverse of A0's Schur complement on the
// top subtree's columns T, computed on the host) and f_T = q_T minus the
// update entries of the supernodes below T that reach T.  One launch
// replaces both sweeps' top levels.
//
// S^{-1} is symmetric, so only its lower block triangle is stored: TS x TS
// tiles (I, J), J <= I, each a contiguous row-major block with rows padded
// by 16 bytes (LDT entries apart), zero past the last row and column.  Every row of a tile gives a row product
// S_IJ f_J (for band I); an off-diagonal tile also gives the column products
// S_IJ^T f_I (for band J) from the same entries.  Each product lands in its
// band's partial slot (slot J for row products, slot I for column products);
// the last of a band's nb contributions to arrive adds the slots in order and
// writes r.
//   tile record (3 int4): {tile offset lo, hi, I, J}
//                         {n_top, first band of the simulation, nb, tcol offset}
//                         {bptr offset, 0, 0, 0}
//
// The launch is persistent: block b takes the consecutive tiles
// [b T / G, (b + 1) T / G) of the T tiles (G blocks, BPS per SM, at most
// TPB tiles each) and streams them through a ring of NBUF half-tile buffers
// in shared memory.  With two blocks per SM (float), one block's arrival on
// a band (a fence and an atomic, about a microsecond) overlaps the other's
// products.  A half tile (HR padded rows) arrives by one
// bulk copy.  With the padding a thread per row reads its row in 16-byte
// pieces without bank conflicts (consecutive rows start 16 bytes apart in
// bank order), and a thread per column reads its column with the warp's 32
// columns side by side.  The first NBUF half tiles
// are requested before the wait on the previous level (the matrix does not
// depend on the solve), and each buffer is refilled as soon as the block has
// read it, so the copies run while the block computes.  f_J and f_I of all
// the block's tiles are gathered once, after the wait, into shared memory.
constexpr int TS = 128;

template <typename R> struct DenseShape {
    static constexpr bool F = sizeof(R) == 4;
    static constexpr int NT = F ? 256 : 512;          // threads per block
    static constexpr int BPS = F ? 2 : 1;             // blocks per SM
    static constexpr int TPB = F ? 4 : 8;             // most tiles per block
    static constexpr int NBUF = 2;                    // half-tile buffers per block
    static constexpr int HR = TS / 2;                 // rows per buffer
    static constexpr int CPR = 16 / (int)sizeof(R);  // entries per 16-byte piece
    static constexpr int LDT = TS + CPR;             // padded row
    static constexpr int UB = HR * LDT;               // entries per buffer
    static constexpr int RP = NT / HR;                // threads per row (row products)
    static constexpr int CP = NT / TS;                // threads per column (column products)
    // dynamic shared memory: buffers, f cache (2 TPB bands x 3 x TS), row
    // partials (2 x RP x 3 x HR), column partials (CP x 3 x TS)
    static constexpr size_t SMEM = sizeof(R) * ((size_t)NBUF * UB + 2 * TPB * 3 * TS + 2 * RP * 3 * HR + CP * 3 * TS);
};

// The grid of the dense launch for T tiles on nsm SMs.
template <typename R> int dense_grid(int tiles, int nsm) {
    using D = DenseShape<R>;
    const int g = std::max(D::BPS * nsm, (tiles + D::TPB - 1) / D::TPB);
    return std::min(g, tiles);
}

// Thread 0: requests half tile u of the block (tile t0 + u / 2, rows from
// HR (u & 1)) into buffer u % NBUF.
template <typename R>
__device__ __forceinline__ void dense_issue(const DevSolve<R> &S, int t0, int u, R *buf, uint64_t *bar) {
    using D = DenseShape<R>;
    const int4 a = S.dense_tiles[3 * (size_t)(t0 + (u >> 1))];
    const long long off = ((long long)(unsigned)a.x | ((long long)a.y << 32)) + (long long)(u & 1) * D::UB;
    static_assert(D::HR * 2 == TS, "a unit is half a tile");
    bulk_load_issue(bar + u % D::NBUF, buf + (size_t)(u % D::NBUF) * D::UB, S.dense_inv + off,
                    (uint32_t)(D::UB * sizeof(R)));
}

template <typename R>
__global__ void __launch_bounds__(DenseShape<R>::NT, DenseShape<R>::BPS)
    k_dense(DevSolve<R> S, const V4<R> *rhs, V4<R> *r) {
    using D = DenseShape<R>;
    using VT = typename Vec16<R>::T;
    constexpr int NT = D::NT, HR = D::HR, CPR = D::CPR, LDT = D::LDT, NBUF = D::NBUF;
    constexpr int RP = D::RP, CP = D::CP, TPB = D::TPB;
    constexpr int NE = (2 * TPB * TS + NT - 1) / NT;  // f entries gathered per thread
    extern __shared__ __align__(128) unsigned char smem_raw[];
    R *buf = reinterpret_cast<R *>(smem_raw);
    R *fc = buf + (size_t)NBUF * D::UB;  // [2 TPB][3][TS]: f_J, f_I of each tile
    R *rowp = fc + 2 * TPB * 3 * TS;     // [2][RP][3][HR]
    R *colp = rowp + 2 * RP * 3 * HR;       // [CP][3][TS]
    __shared__ __align__(8) uint64_t bar[NBUF];
    __shared__ int lastI, lastJ;
    const int tid = threadIdx.x;
    const int T = S.n_dense_tiles, G = gridDim.x;
    const int t0 = (int)((long long)blockIdx.x * T / G), t1 = (int)((long long)(blockIdx.x + 1) * T / G);
    const int U = 2 * (t1 - t0);  // half tiles
    if (tid == 0) {
        for (int k = 0; k < NBUF; ++k) bulk_bar_init(&bar[k]);
        for (int u = 0; u < NBUF && u < U; ++u) dense_issue<R>(S, t0, u, buf, bar);
    }
    // before the wait: the gathers' index data (nothing the solve writes).
    // Entry e: slot e / TS (2 k: f_J of tile t0 + k, 2 k + 1: its f_I), column e % TS
    int colv[NE];
    int4 bnd[NE];
#pragma unroll
    for (int q = 0; q < NE; ++q) {
        const int e = tid + q * NT;
        colv[q] = -1;
        bnd[q] = make_int4(-1, -1, -1, -1);
        if (e >= U * TS) continue;
        const int slot = e / TS, j = e % TS;
        const int4 *rec = S.dense_tiles + 3 * (size_t)(t0 + (slot >> 1));
        const int4 a = rec[0], b = rec[1], c = rec[2];
        const int B = (slot & 1) ? a.z : a.w;
        const int col = B * TS + j;
        if (col >= b.x) continue;
        const int *bptr = S.dense_bptr + c.x;
        const int k0 = bptr[col], k1 = bptr[col + 1];
        colv[q] = S.dense_col[b.w + col];
        bnd[q] = make_int4(k1 > k0 ? S.dense_bidx[k0] : -1, k1 > k0 + 1 ? S.dense_bidx[k0 + 1] : -1,
                           k1 > k0 + 2 ? S.dense_bidx[k0 + 2] : -1, k1 > k0 + 3 ? S.dense_bidx[k0 + 3] : -1);
    }
    pdl_trigger();
    pdl_wait();
    // f = q minus the (<= 4) update entries from below T, zero past n
#pragma unroll
    for (int q = 0; q < NE; ++q) {
        const int e = tid + q * NT;
        if (e >= U * TS) continue;
        R fx = R(0), fy = R(0), fz = R(0);
        if (colv[q] >= 0) {
            const int4 eb = bnd[q];
            const V4<R> v = ld_cg(rhs + colv[q]);
            V4<R> u4[4];
#pragma unroll
            for (int k = 0; k < 4; ++k) u4[k].x = u4[k].y = u4[k].z = R(0);
            if (eb.x >= 0) u4[0] = ld_cg(S.u + eb.x);
            if (eb.y >= 0) u4[1] = ld_cg(S.u + eb.y);
            if (eb.z >= 0) u4[2] = ld_cg(S.u + eb.z);
            if (eb.w >= 0) u4[3] = ld_cg(S.u + eb.w);
            fx = v.x - u4[0].x - u4[1].x - u4[2].x - u4[3].x;
            fy = v.y - u4[0].y - u4[1].y - u4[2].y - u4[3].y;
            fz = v.z - u4[0].z - u4[1].z - u4[2].z - u4[3].z;
        }
        R *f = fc + (size_t)(e / TS) * 3 * TS + e % TS;
        f[0] = fx; f[TS] = fy; f[2 * TS] = fz;
    }
    // row products: thread (row ri, part rp) takes TS / RP columns of its row;
    // column products: thread (column cj, part cq) takes HR / CP rows of the
    // half tile, summed over both halves
    const int ri = tid % HR, rp = tid / HR;
    const int cj = tid % TS, cq = tid / TS;
    constexpr int RCOLS = TS / RP, CROWS = HR / CP;
    R ca0 = R(0), ca1 = R(0), ca2 = R(0);
    for (int u = 0; u < U; ++u) {
        const int nbuf = u % NBUF;
        // (the barrier inside also orders the f gather before the first use)
        if (!bulk_load_finish(&bar[nbuf], (uint32_t)((u / NBUF) & 1), S.err, S.wait_polls, true)) {
            if (tid == 0)
                for (int v = u + 1; v < u + NBUF && v < U; ++v)
                    if (!bulk_load_wait(&bar[v % NBUF], (uint32_t)((v / NBUF) & 1), kDrainPolls)) atomicOr(S.err, 4u);
            return;
        }
        const int k = u >> 1, h = u & 1;
        const int4 *rec = S.dense_tiles + 3 * (size_t)(t0 + k);
        const int4 a = rec[0], b = rec[1];
        const int I = a.z, J = a.w;
        const int n = b.x, band0 = b.y, nb = b.z, tc0 = b.w;
        const bool diag = I == J;
        const int nI = min(TS, n - I * TS), nJ = min(TS, n - J * TS);
        const R *tile = buf + (size_t)nbuf * D::UB;
        const R *fJ = fc + (size_t)(2 * k) * 3 * TS, *fI = fc + (size_t)(2 * k + 1) * 3 * TS;
        {
            const R *row = tile + (size_t)ri * LDT + rp * RCOLS;
            R px = R(0), py = R(0), pz = R(0);
#pragma unroll
            for (int c = 0; c < RCOLS; c += CPR) {
                const VT sv = *reinterpret_cast<const VT *>(row + c);
                const R *s4 = reinterpret_cast<const R *>(&sv);
                const int j0 = rp * RCOLS + c;
                const VT fx = *reinterpret_cast<const VT *>(fJ + j0);
                const VT fy = *reinterpret_cast<const VT *>(fJ + TS + j0);
                const VT fz = *reinterpret_cast<const VT *>(fJ + 2 * TS + j0);
                const R *gx = reinterpret_cast<const R *>(&fx);
                const R *gy = reinterpret_cast<const R *>(&fy);
                const R *gz = reinterpret_cast<const R *>(&fz);
#pragma unroll
                for (int e = 0; e < CPR; ++e) {
                    px += s4[e] * gx[e];
                    py += s4[e] * gy[e];
                    pz += s4[e] * gz[e];
                }
            }
            R *rw = rowp + (size_t)(u & 1) * RP * 3 * HR + (size_t)rp * 3 * HR + ri;
            rw[0] = px; rw[HR] = py; rw[2 * HR] = pz;
        }
        if (!diag) {
            const R *col = tile + cj;
#pragma unroll 4
            for (int i0 = cq * CROWS; i0 < cq * CROWS + CROWS; i0 += CPR) {
                const int ig = h * HR + i0;
                const VT gx = *reinterpret_cast<const VT *>(fI + ig);
                const VT gy = *reinterpret_cast<const VT *>(fI + TS + ig);
                const VT gz = *reinterpret_cast<const VT *>(fI + 2 * TS + ig);
                const R *hx = reinterpret_cast<const R *>(&gx);
                const R *hy = reinterpret_cast<const R *>(&gy);
                const R *hz = reinterpret_cast<const R *>(&gz);
#pragma unroll
                for (int e = 0; e < CPR; ++e) {
                    const R sij = col[(size_t)(i0 + e) * LDT];
                    ca0 += sij * hx[e];
                    ca1 += sij * hy[e];
                    ca2 += sij * hz[e];
                }
            }
        }
        __syncthreads();  // the buffer is read; the row partials are written
        if (tid == 0 && u + NBUF < U) dense_issue<R>(S, t0, u + NBUF, buf, bar);
        V4<R> *part = S.dense_part + (size_t)band0 * S.dense_nct_max * TS;
        if (tid < HR && h * HR + tid < nI) {
            const R *rw = rowp + (size_t)(u & 1) * RP * 3 * HR + tid;
            R sx = R(0), sy = R(0), sz = R(0);
#pragma unroll
            for (int p = 0; p < RP; ++p) {
                sx += rw[(size_t)p * 3 * HR];
                sy += rw[(size_t)p * 3 * HR + HR];
                sz += rw[(size_t)p * 3 * HR + 2 * HR];
            }
            V4<R> o;
            o.x = sx; o.y = sy; o.z = sz; o.w = R(0);
            part[((size_t)I * S.dense_nct_max + J) * TS + h * HR + tid] = o;  // band I, slot J
        }
        if (h == 0) continue;
        // the tile is complete: its column products (band J, slot I), then
        // the arrivals on band I (and band J)
        if (!diag) {
            R *cw = colp + (size_t)cq * 3 * TS + cj;
            cw[0] = ca0; cw[TS] = ca1; cw[2 * TS] = ca2;
            ca0 = ca1 = ca2 = R(0);
            __syncthreads();
            if (tid < nJ) {
                R sx = R(0), sy = R(0), sz = R(0);
#pragma unroll
                for (int p = 0; p < CP; ++p) {
                    sx += colp[(size_t)p * 3 * TS + tid];
                    sy += colp[(size_t)p * 3 * TS + TS + tid];
                    sz += colp[(size_t)p * 3 * TS + 2 * TS + tid];
                }
                V4<R> o;
                o.x = sx; o.y = sy; o.z = sz; o.w = R(0);
                part[((size_t)J * S.dense_nct_max + I) * TS + tid] = o;
            }
        }
        __syncthreads();
        if (tid == 0) {
            __threadfence();  // release: this tile's partials before the counts
            lastI = atomicAdd(S.dense_cnt + band0 + I, 1) == nb - 1;
            lastJ = diag ? 0 : (atomicAdd(S.dense_cnt + band0 + J, 1) == nb - 1);
            if (lastI || lastJ) __threadfence();  // acquire, ordered for the block by the barrier below
        }
        __syncthreads();
        const int *tcol = S.dense_col + tc0;
        for (int side = 0; side < 2; ++side) {
            const bool go = side == 0 ? lastI : lastJ;
            if (!go) continue;
            const int Bd = side == 0 ? I : J, nB = side == 0 ? nI : nJ;
            const V4<R> *slots = part + (size_t)Bd * S.dense_nct_max * TS;
            for (int i = tid; i < nB; i += NT) {
                R sx = R(0), sy = R(0), sz = R(0);
                for (int t = 0; t < nb; ++t) {
                    const V4<R> p = ld_cg(slots + (size_t)t * TS + i);
                    sx += p.x; sy += p.y; sz += p.z;
                }
                V4<R> o;
                o.x = sx; o.y = sy; o.z = sz; o.w = R(0);
                r[tcol[Bd * TS + i]] = o;
            }
            if (tid == 0) S.dense_cnt[band0 + Bd] = 0;
        }
    }
}

// Dynamic shared memory of a sweep block: qcap factor entries, 3 x ld vector
// entries and ld 16-byte index slots.
template <typename R>
size_t sweep_smem(int qcap, int ld) {
    return ((size_t)qcap + 3 * (size_t)ld) * sizeof(R) + 16 * (size_t)ld;
}

template <typename R> cudaStream_t st_of(const DevSolve<R> &s) { return s.stream; }

// One level's launch, with the programmatic-serialisation attribute when
// the handle chains levels.
template <typename R, typename... KArgs, typename... Args>
void launch_level(bool pdl, void (*kernel)(DevSolve<R>, int, int, KArgs...), int grid, int threads, size_t smem,
                  cudaStream_t st, const DevSolve<R> &s, int item0, int qcap, Args... args) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)grid);
    cfg.blockDim = dim3((unsigned)threads);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = pdl ? 1 : 0;
    cudaLaunchKernelEx(&cfg, kernel, s, item0, qcap, args...);
}

template <typename R, int NT>
void launch_fwd_level(const DevSolve<R> &s, int l, const V4<R> *q, V4<R> *z, const int4 *pf, int pf_n) {
    const int a = s.fwd_lvl_ptr[l], b = s.fwd_lvl_ptr[l + 1];
    launch_level<R, const V4<R> *, V4<R> *, const int4 *, int, int>(
        s.pdl != 0, k_fwd<R, NT>, b - a, NT, sweep_smem<R>(s.fwd_lvl_q[l], s.fwd_lvl_ld[l]), st_of(s), s, a,
        s.fwd_lvl_q[l], q, z, pf, pf_n, (s.fault_test == 1 && l == 0) ? 1 : 0);
}

template <typename R, int NT>
void launch_bwd_level(const DevSolve<R> &s, int l, const V4<R> *z, V4<R> *r, const int4 *pf, int pf_n) {
    const int a = s.bwd_lvl_start[l], cnt = s.bwd_lvl_cnt[l];
    launch_level<R, const V4<R> *, V4<R> *, const int4 *, int>(
        s.pdl != 0, k_bwd<R, NT>, cnt, NT, sweep_smem<R>(s.bwd_lvl_q[l], s.bwd_lvl_ld[l]), st_of(s), s, a,
        s.bwd_lvl_q[l], z, r, pf, pf_n);
}

// One solve: the forward levels (leaves first), the dense top block if any,
// the backward levels (root first).  The leaf level may run with its own
// block size.
template <typename R>
void launch_sweeps(const DevSolve<R> &s, const V4<R> *q, V4<R> *z, V4<R> *r) {
    const int L = s.n_levels;
    // launch k of the solve: forward level k (k < L), then backward level 2L - 1 - k
    auto pf_of = [&](int k, const int4 **p, int *n) {
        *p = nullptr;
        *n = 0;
        if (!s.pf_any) return;
        *p = s.pf_spans + s.pf_ptr[k];
        *n = s.pf_ptr[k + 1] - s.pf_ptr[k];
    };
    auto nt_of = [&](int l) { return l == 0 ? s.leaf_threads : s.threads; };
    for (int l = 0; l < L; ++l) {
        if (s.fwd_lvl_ptr[l + 1] <= s.fwd_lvl_ptr[l]) continue;
        const int4 *pf;
        int pf_n;
        pf_of(l, &pf, &pf_n);
        switch (nt_of(l)) {
            case 128: launch_fwd_level<R, 128>(s, l, q, z, pf, pf_n); break;
            case 512: launch_fwd_level<R, 512>(s, l, q, z, pf, pf_n); break;
            default: launch_fwd_level<R, 256>(s, l, q, z, pf, pf_n); break;
        }
    }
    if (s.n_dense_tiles > 0) {
        cudaLaunchConfig_t cfg = {};
        cfg.gridDim = dim3((unsigned)dense_grid<R>(s.n_dense_tiles, s.n_sm));
        cfg.blockDim = dim3(DenseShape<R>::NT);
        cfg.dynamicSmemBytes = DenseShape<R>::SMEM;
        cfg.stream = st_of(s);
        cudaLaunchAttribute attr[1];
        attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
        attr[0].val.programmaticStreamSerializationAllowed = 1;
        cfg.attrs = attr;
        cfg.numAttrs = s.pdl ? 1 : 0;
        cudaLaunchKernelEx(&cfg, k_dense<R>, s, q, r);
    }
    for (int l = L - 1; l >= 0; --l) {
        if (s.bwd_lvl_cnt[l] <= 0) continue;
        const int4 *pf;
        int pf_n;
        pf_of(2 * L - 1 - l, &pf, &pf_n);
        switch (nt_of(l)) {
            case 128: launch_bwd_level<R, 128>(s, l, (const V4<R> *)z, r, pf, pf_n); break;
            case 512: launch_bwd_level<R, 512>(s, l, (const V4<R> *)z, r, pf, pf_n); break;
            default: launch_bwd_level<R, 256>(s, l, (const V4<R> *)z, r, pf, pf_n); break;
        }
    }
}

template <typename R, int NT>
cudaError_t prepare_nt() {
    cudaError_t e = cudaFuncSetAttribute(k_fwd<R, NT>, cudaFuncAttributeMaxDynamicSharedMemorySize, SOLVE_MAX_SMEM);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_bwd<R, NT>, cudaFuncAttributeMaxDynamicSharedMemorySize, SOLVE_MAX_SMEM);
    return e;
}

}  // namespace

template <typename R> size_t solve_block_smem(int qcap, int ld) { return sweep_smem<R>(qcap, ld); }

template <typename R> cudaError_t solve_prepare() {
    cudaError_t e = cudaFuncSetAttribute(k_dense<R>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)DenseShape<R>::SMEM);
    if (e == cudaSuccess) e = prepare_nt<R, 128>();
    if (e == cudaSuccess) e = prepare_nt<R, 256>();
    if (e == cudaSuccess) e = prepare_nt<R, 512>();
    return e;
}

template <typename R>
void launch_solve(const DevSolve<R> &s, const V4<R> *q, V4<R> *z, V4<R> *r, cudaStream_t st) {
    DevSolve<R> t = s;
    t.stream = st;
    launch_sweeps<R>(t, q, z, r);
}

template void launch_solve<float>(const DevSolve<float> &, const V4<float> *, V4<float> *, V4<float> *, cudaStream_t);
template void launch_solve<double>(const DevSolve<double> &, const V4<double> *, V4<double> *, V4<double> *, cudaStream_t);
template size_t solve_block_smem<float>(int, int);
template size_t solve_block_smem<double>(int, int);
template cudaError_t solve_prepare<float>();
template cudaError_t solve_prepare<double>();

}  // namespace hqn
