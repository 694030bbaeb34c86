// Packed layout of the per-supernode solve operators, shared by the host
// set-up (which fills them) and the device sweeps (which read them).
//
// A supernode with nc columns and nr coupled rows holds Q = [Linv; K] with
// Linv = L_CC^{-1} (nc x nc, lower triangular) and K = L_RC L_CC^{-1} (nr x nc).
//   Forward copy (row-major): row i < nc keeps entries [0, pad4(i + 1)) -- the
//   triangle without its zero upper part -- and row i >= nc all ldc = pad4(nc)
//   entries.  Rows are stored back to back.
//   Backward copy (Q^T, row-major): row j keeps entries [4 floor(j/4), ldr),
//   ldr = pad4(nc + nr), i.e. from the diagonal (rounded down to a 4-entry
//   boundary) to the end.  Rows are stored back to back.
// Every row length and offset is a multiple of 4 entries, so each row starts
// on a 16-byte boundary (float) or 32-byte boundary (double), and any run of
// consecutive rows is one contiguous block that a bulk copy can move.
#pragma once

#include <stdint.h>

#ifdef __CUDACC__
#define HQN_HD __host__ __device__ __forceinline__
#else
#define HQN_HD inline
#endif

namespace hqn {

HQN_HD int pad4(int k) { return (k + 3) & ~3; }

// Offset of forward row i (0 <= i <= nc + nr; i = nc + nr is the total size).
HQN_HD int64_t fwd_row_off(int i, int nc, int ldc) {
    const int t = i < nc ? i : nc;
    const int64_t q = t >> 2, r = t & 3;
    const int64_t tri = 4 * (q + 1) * (2 * q + r);  // sum of pad4(k + 1), k < t
    return i <= nc ? tri : tri + (int64_t)(i - nc) * ldc;
}
HQN_HD int fwd_row_len(int i, int nc, int ldc) { return i < nc ? pad4(i + 1) : ldc; }

// Offset of backward row j (0 <= j <= nc; j = nc is the total size) and the
// first column entry it stores.
HQN_HD int64_t bwd_row_off(int j, int ldr) {
    const int64_t q = j >> 2, r = j & 3;
    return (int64_t)j * ldr - 4 * (2 * q * (q - 1) + r * q);  // minus sum of 4 floor(k/4), k < j
}
HQN_HD int bwd_row_start(int j) { return j & ~3; }

}  // namespace hqn
