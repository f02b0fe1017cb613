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
    const KT S = d1_sentinel<KT>();
    KT a = i < na ? A[i] : S;
    KT b = j < nb ? B[j] : S;
    for (int n = 0; n < cnt; n++) {
        const bool ta = (j >= nb) || (i < na && a <= b);
        out[n] = ta ? a : b;
        i += ta ? 1 : 0;
        j += ta ? 0 : 1;
        a = i < na ? A[i] : S;
        b = j < nb ? B[j] : S;
    }
}

}  // namespace mf
