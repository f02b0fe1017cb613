// Building blocks of the data-aware variant (paper Sec. 5.1), shared by the
// device kernel and the host-side plan checker so that both run exactly the
// same merge and sort code.
//
// Merge: the output range of a two-list merge is cut into chunks; a chunk
// finds where it starts in each input by a binary search on the merge path
// (Odeh et al., the paper's Sec. 5.1 reference), then merges sequentially.
// Ties take A first, so the merge is stable.
// Sort: short lists (the sorted column/row segments and the corner runs)
// are sorted by one thread with a sorting network held in registers, as the
// paper recommends for many small sorts (Sec. 5.1).
#pragma once
#include <cstdint>

#include "mf_d1_plan.h"

#ifndef __CUDACC__
#define __host__
#define __device__
#define __forceinline__ inline
#endif

namespace mf {

template <class KT>
__host__ __device__ __forceinline__ KT d1_sentinel() {
    return (KT)~(KT)0;
}

// 16-byte device form of a task (one 128-bit load):
//   x = a_off | type << 17 | (a_stride == FW) << 18 | chunk << 19
//   y = b_off | a_len << 17,  z = out_off | b_len << 17,  w = lo | hi << 13
// Offsets < 2^17 list elements, lengths and ranks < 2^13, chunk < 64.
struct D1Packed {
    uint32_t x, y, z, w;
};

__host__ __device__ __forceinline__ D1Task d1_unpack(const D1Packed &p, int FW) {
    D1Task t;
    t.a_off = (int)(p.x & 0x1ffffu);
    t.type = (int)((p.x >> 17) & 1u);
    t.a_stride = ((p.x >> 18) & 1u) ? FW : 1;
    t.chunk = (int)(p.x >> 19);
    t.b_off = (int)(p.y & 0x1ffffu);
    t.a_len = (int)(p.y >> 17);
    t.out_off = (int)(p.z & 0x1ffffu);
    t.b_len = (int)(p.z >> 17);
    t.lo = (int)(p.w & 0x1fffu);
    t.hi = (int)(p.w >> 13);
    return t;
}

// Outputs lo + chunk*t.chunk ... (up to t.chunk of them, not past hi) of
// merge(A, B) into out[(p - lo)].
template <class KT>
__host__ __device__ __forceinline__ void d1_merge_chunk(KT *sm, const D1Task &t, int chunk) {
    const KT *A = sm + t.a_off;
    const KT *B = sm + t.b_off;
    const int na = t.a_len, nb = t.b_len;
    const int p0 = t.lo + chunk * t.chunk;
    int cnt = t.hi - p0 + 1;
    if (cnt > t.chunk) cnt = t.chunk;
    // i = number of A elements among the first p0 outputs
    int lo = p0 - nb > 0 ? p0 - nb : 0;
    int hi = p0 < na ? p0 : na;
    while (lo < hi) {
        const int mid = (lo + hi) >> 1;
        // A[mid] precedes B[p0-1-mid] (ties: A first) => more A elements are in front
        if (A[mid] <= B[p0 - 1 - mid]) lo = mid + 1;
        else hi = mid;
    }
    int i = lo, j = p0 - lo;
    KT *out = sm + t.out_off + (p0 - t.lo);
    // branch-free: the index of an exhausted list is clamped to its last
    // element and never chosen again (ta is forced by the length tests)
    const int ia = na - 1, jb = nb - 1;
    KT a = A[i < ia ? i : ia];
    KT b = B[j < jb ? j : jb];
#pragma unroll 4
    for (int n = 0; n < cnt; n++) {
        const bool ta = (j > jb) || (i <= ia && a <= b);
        out[n] = ta ? a : b;
        i += ta;
        j += !ta;
        a = A[i < ia ? i : ia];
        b = B[j < jb ? j : jb];
    }
}

}  // namespace mf
