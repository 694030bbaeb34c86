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
// at most two children; no atomics).
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
// Consecutive levels are chained by programmatic dependent launch: a level's
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

// Any thread: one copy whose bytes count against the barrier's phase.
__device__ __forceinline__ void bulk_copy(uint64_t *bar, void *dst, const void *src, uint32_t bytes) {
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                     smem_addr(dst)),
                 "l"(src), "r"(bytes), "r"(smem_addr(bar))
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
template <typename R, int G>
__device__ __forceinline__ void fwd_rows(const DevSolve<R> &S, int col, int nc, int ldc, int uoff, int r0, int r1,
                                         int off0, const R *qs, const R *f, int ldf, V4<R> *z) {
    using VT = typename Vec16<R>::T;
    constexpr int VN = Vec16<R>::N;
    constexpr int NG = SBS / G;
    const int lane = threadIdx.x % G, grp = threadIdx.x / G;
    const VT *fx = reinterpret_cast<const VT *>(f);
    const VT *fy = reinterpret_cast<const VT *>(f + ldf);
    const VT *fz = reinterpret_cast<const VT *>(f + 2 * ldf);
    for (int base = r0; base < r1; base += 2 * NG) {
        const int i0 = base + 2 * grp, i1 = i0 + 1;
        const bool v0 = i0 < r1, v1 = i1 < r1;
        const int n0 = v0 ? fwd_row_len(i0, nc, ldc) / VN : 0;
        const int n1 = v1 ? fwd_row_len(i1, nc, ldc) / VN : 0;
        const VT *q0 = reinterpret_cast<const VT *>(qs + (v0 ? fwd_row_off(i0, nc, ldc) - off0 : 0));
        const VT *q1 = reinterpret_cast<const VT *>(qs + (v1 ? fwd_row_off(i1, nc, ldc) - off0 : 0));
        R a0x = R(0), a0y = R(0), a0z = R(0), a1x = R(0), a1y = R(0), a1z = R(0);
        const int nmax = n0 > n1 ? n0 : n1;
        for (int k = lane; k < nmax; k += G) {
            const VT x = fx[k], y = fy[k], w = fz[k];
            if (k < n0) {
                const VT q = q0[k];
                a0x += Vec16<R>::dot3(q, x); a0y += Vec16<R>::dot3(q, y); a0z += Vec16<R>::dot3(q, w);
            }
            if (k < n1) {
                const VT q = q1[k];
                a1x += Vec16<R>::dot3(q, x); a1y += Vec16<R>::dot3(q, y); a1z += Vec16<R>::dot3(q, w);
            }
        }
        a0x = group_sum<R, G>(a0x); a0y = group_sum<R, G>(a0y); a0z = group_sum<R, G>(a0z);
        a1x = group_sum<R, G>(a1x); a1y = group_sum<R, G>(a1y); a1z = group_sum<R, G>(a1z);
        if (lane == 0) {
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const int i = h ? i1 : i0;
                if (!(h ? v1 : v0)) continue;
                V4<R> o;
                o.x = h ? a1x : a0x; o.y = h ? a1y : a0y; o.z = h ? a1z : a0z; o.w = R(0);
                if (i < nc) {
                    z[col + i] = o;
                } else {
                    const int2 c = S.ug2[uoff + i - nc];
                    if (c.x >= 0) { const V4<R> a = ld_cg(S.u + c.x); o.x += a.x; o.y += a.y; o.z += a.z; }
                    if (c.y >= 0) { const V4<R> a = ld_cg(S.u + c.y); o.x += a.x; o.y += a.y; o.z += a.z; }
                    S.u[uoff + i - nc] = o;
                }
            }
        }
    }
}

// One forward work item (record `rec`, 4 int4).  Shared memory: qs = the
// item's factor rows (qcap entries), then f (3 x ldf entries), then the
// columns' child update entries (ldf int2).  `wait_inputs` runs between the
// reads of static data and the reads of vectors other items produce.
template <typename R, typename Wait>
__device__ __forceinline__ void fwd_item(const DevSolve<R> &S, const int4 *rec, int qcap, R *qs, uint64_t *bar,
                                         uint32_t parity, const V4<R> *rhs, V4<R> *z, Wait wait_inputs) {
    const int4 a = rec[0];
    if (threadIdx.x == 0) bulk_load_issue(bar, qs, item_src(S.QF, a, sizeof(R)), (uint32_t)a.z);
    const int4 b = rec[1], c = rec[2];
    const int col = b.x, nc = b.y, ldc = b.z, uoff = b.w;
    const int r0 = c.x, r1 = c.y, ldf = c.z, off0 = c.w;
    R *f = qs + qcap;
    int2 *cidx = reinterpret_cast<int2 *>(f + 3 * ldf);
    const int nf = ldf < nc ? ldf : nc;
    for (int j = threadIdx.x; j < nf; j += SBS) cidx[j] = S.fg2[col + j];
    if (!wait_inputs()) {
        if (threadIdx.x == 0) bulk_load_wait(bar, parity);  // let the copy in flight land first
        return;
    }
    // f = q_C - (child updates on C), entries [0, ldf); zero beyond nc
#pragma unroll 4
    for (int j = threadIdx.x; j < ldf; j += SBS) {
        R vx = R(0), vy = R(0), vz = R(0);
        if (j < nc) {
            const V4<R> v = ld_cg(rhs + col + j);
            const int2 ci = cidx[j];
            vx = v.x; vy = v.y; vz = v.z;
            if (ci.x >= 0) { const V4<R> u = ld_cg(S.u + ci.x); vx -= u.x; vy -= u.y; vz -= u.z; }
            if (ci.y >= 0) { const V4<R> u = ld_cg(S.u + ci.y); vx -= u.x; vy -= u.y; vz -= u.z; }
        }
        f[j] = vx; f[ldf + j] = vy; f[2 * ldf + j] = vz;
    }
    if (!bulk_load_finish(bar, parity, S.err)) return;
    switch (a.w) {
        case 1: fwd_rows<R, 1>(S, col, nc, ldc, uoff, r0, r1, off0, qs, f, ldf, z); break;
        case 2: fwd_rows<R, 2>(S, col, nc, ldc, uoff, r0, r1, off0, qs, f, ldf, z); break;
        case 4: fwd_rows<R, 4>(S, col, nc, ldc, uoff, r0, r1, off0, qs, f, ldf, z); break;
        case 8: fwd_rows<R, 8>(S, col, nc, ldc, uoff, r0, r1, off0, qs, f, ldf, z); break;
        case 16: fwd_rows<R, 16>(S, col, nc, ldc, uoff, r0, r1, off0, qs, f, ldf, z); break;
        default: fwd_rows<R, 32>(S, col, nc, ldc, uoff, r0, r1, off0, qs, f, ldf, z); break;
    }
}

// Level-synchronous schedule: one launch per tree level, one item per block.
template <typename R>
__global__ void __launch_bounds__(SBS) k_fwd(DevSolve<R> S, int item0, int qcap, const V4<R> *rhs, V4<R> *z) {
    extern __shared__ __align__(128) unsigned char smem_raw[];
    __shared__ __align__(8) uint64_t bar;
    if (threadIdx.x == 0) bulk_bar_init(&bar);
    fwd_item<R>(S, S.fwd_items + 4 * (size_t)(item0 + blockIdx.x), qcap, reinterpret_cast<R *>(smem_raw), &bar, 0u,
                rhs, z, []() {
                    pdl_wait();
                    pdl_trigger();
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
template <typename R, int G, bool CHUNK>
__device__ __forceinline__ void bwd_rows(int col, int ldr, int c0, int c1, int off0, const R *qs, const R *w,
                                         int lw, int w0, V4<R> *r, V4<R> *out) {
    using VT = typename Vec16<R>::T;
    constexpr int VN = Vec16<R>::N;
    constexpr int NG = SBS / G;
    const int lane = threadIdx.x % G, grp = threadIdx.x / G;
    const VT *wx = reinterpret_cast<const VT *>(w);
    const VT *wy = reinterpret_cast<const VT *>(w + lw);
    const VT *wz = reinterpret_cast<const VT *>(w + 2 * lw);
    const int kend = lw / VN;
    for (int base = c0; base < c1; base += 2 * NG) {
        const int j0 = base + 2 * grp, j1 = j0 + 1;
        const bool v0 = j0 < c1, v1 = j1 < c1;
        // row j covers w vectors [k_j, kend)
        int k0 = kend, k1 = kend;
        const VT *q0 = nullptr, *q1 = nullptr;
        if (v0) {
            const int st = bwd_row_start(j0);
            k0 = st > w0 ? (st - w0) / VN : 0;
            q0 = CHUNK ? reinterpret_cast<const VT *>(qs + (size_t)(j0 - c0) * lw)
                       : reinterpret_cast<const VT *>(qs + (bwd_row_off(j0, ldr) - off0)) - k0;
        }
        if (v1) {
            const int st = bwd_row_start(j1);
            k1 = st > w0 ? (st - w0) / VN : 0;
            q1 = CHUNK ? reinterpret_cast<const VT *>(qs + (size_t)(j1 - c0) * lw)
                       : reinterpret_cast<const VT *>(qs + (bwd_row_off(j1, ldr) - off0)) - k1;
        }
        R a0x = R(0), a0y = R(0), a0z = R(0), a1x = R(0), a1y = R(0), a1z = R(0);
        const int kmin = k0 < k1 ? k0 : k1;
        for (int k = kmin + lane; k < kend; k += G) {
            const VT x = wx[k], y = wy[k], v = wz[k];
            if (k >= k0) {
                const VT q = q0[k];
                a0x += Vec16<R>::dot3(q, x); a0y += Vec16<R>::dot3(q, y); a0z += Vec16<R>::dot3(q, v);
            }
            if (k >= k1) {
                const VT q = q1[k];
                a1x += Vec16<R>::dot3(q, x); a1y += Vec16<R>::dot3(q, y); a1z += Vec16<R>::dot3(q, v);
            }
        }
        a0x = group_sum<R, G>(a0x); a0y = group_sum<R, G>(a0y); a0z = group_sum<R, G>(a0z);
        a1x = group_sum<R, G>(a1x); a1y = group_sum<R, G>(a1y); a1z = group_sum<R, G>(a1z);
        if (lane == 0) {
            if (v0) {
                V4<R> o; o.x = a0x; o.y = a0y; o.z = a0z; o.w = R(0);
                if (out) out[j0 - c0] = o; else r[col + j0] = o;
            }
            if (v1) {
                V4<R> o; o.x = a1x; o.y = a1y; o.z = a1z; o.w = R(0);
                if (out) out[j1 - c0] = o; else r[col + j1] = o;
            }
        }
    }
}

template <typename R, bool CHUNK>
__device__ __forceinline__ void bwd_rows_g(int G, int col, int ldr, int c0, int c1, int off0, const R *qs,
                                           const R *w, int lw, int w0, V4<R> *r, V4<R> *out) {
    switch (G) {
        case 1: bwd_rows<R, 1, CHUNK>(col, ldr, c0, c1, off0, qs, w, lw, w0, r, out); break;
        case 2: bwd_rows<R, 2, CHUNK>(col, ldr, c0, c1, off0, qs, w, lw, w0, r, out); break;
        case 4: bwd_rows<R, 4, CHUNK>(col, ldr, c0, c1, off0, qs, w, lw, w0, r, out); break;
        case 8: bwd_rows<R, 8, CHUNK>(col, ldr, c0, c1, off0, qs, w, lw, w0, r, out); break;
        case 16: bwd_rows<R, 16, CHUNK>(col, ldr, c0, c1, off0, qs, w, lw, w0, r, out); break;
        default: bwd_rows<R, 32, CHUNK>(col, ldr, c0, c1, off0, qs, w, lw, w0, r, out); break;
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
        bwd_rows_g<R, false>(a.w, col, ldr, c0, c1, off0, qs, w, lw, w0, r, nullptr);
        return;
    }
    const int nch = e.w >> 16, kch = e.w & 0xffff;
    if (nch == 1) {
        bwd_rows_g<R, true>(a.w, col, ldr, c0, c1, off0, qs, w, lw, w0, r, nullptr);
        return;
    }
    V4<R> *mine = S.part_r + (size_t)item * 32;
    bwd_rows_g<R, true>(a.w, col, ldr, c0, c1, off0, qs, w, lw, w0, r, mine);
    // the last chunk of the column block to get here combines the partials
    __shared__ int last;
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        last = atomicAdd(S.cb_cnt + e.z, 1) == nch - 1;
    }
    __syncthreads();
    if (!last) return;
    __threadfence();
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
__global__ void __launch_bounds__(SBS) k_bwd(DevSolve<R> S, int item0, int qcap, const V4<R> *z, V4<R> *r) {
    extern __shared__ __align__(128) unsigned char smem_raw[];
    __shared__ __align__(8) uint64_t bar;
    if (threadIdx.x == 0) bulk_bar_init(&bar);
    const int item = item0 + blockIdx.x;
    bwd_item<R>(S, S.bwd_items + 5 * (size_t)item, item, qcap, reinterpret_cast<R *>(smem_raw), &bar, 0u, z, r,
                []() {
                    pdl_wait();
                    pdl_trigger();
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
        const int4 *rec = S.fwd_items + 4 * (size_t)item;
        const int4 dep = rec[3];  // children c0, c1 (-1: none), own supernode
        fwd_item<R>(S, rec, qcap, qs, &bar, parity, rhs, z, [&]() {
            if (threadIdx.x == 0)
                ok_sh = dep_wait(S.fwd_done, dep.x, dep.x >= 0 ? S.fwd_nitems[dep.x] : 0, S.err) &&
                        dep_wait(S.fwd_done, dep.y, dep.y >= 0 ? S.fwd_nitems[dep.y] : 0, S.err);
            __syncthreads();
            return ok_sh != 0;
        });
        if (!still_ok(S.err)) break;
        dep_signal(S.fwd_done, dep.z);
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

// Dynamic shared memory of a sweep block: qcap factor entries, 3 x ld vector
// entries and ld 8-byte index slots.
template <typename R>
size_t sweep_smem(int qcap, int ld) {
    return ((size_t)qcap + 3 * (size_t)ld) * sizeof(R) + 8 * (size_t)ld;
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
    return e;
}

template <typename R>
void launch_solve(const DevSolve<R> &s, const V4<R> *q, V4<R> *z, V4<R> *r, cudaStream_t st) {
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
template int solve_smem_limit_ok<float>(int);
template int solve_smem_limit_ok<double>(int);
template cudaError_t solve_prepare<float>();
template cudaError_t solve_prepare<double>();

}  // namespace hqn
