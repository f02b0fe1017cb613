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
// Insert: an extra row or column extended by the 1, 2 or 4 corners of a
// split (Sec. 3.4) is a merge with a very short second list; one thread
// moves every list element up by the number of corners below it and drops
// the corners into the gaps, reading the list in order (no merge-path
// search, no data-dependent read addresses).
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

// 16-byte device form of one work item (one 128-bit load; the item carries
// everything its thread needs, so no second, dependent fetch of its task):
//   x = a_off | type << 17 | (gather stride == FW) << 19 | last << 20 | cnt << 21
//   y = b_off | a_len << 17,  z = out_off | b_len << 17,  w = start
// Offsets < 2^17 list elements, lengths and ranks < 2^13, cnt < 256.  The
// gather stride is the SORT's a_stride or the INSERT's b_stride.
struct alignas(16) D1Packed {
    uint32_t x, y, z, w;
};

// One work item, decoded.
struct D1Item {
    int type;
    int a_off, a_len, a_stride;  // SORT: gather a_len elements at a_off + i*a_stride; else list A (INSERT: L)
    int b_off, b_len, b_stride;  // MERGE: list B; INSERT: b_len corners at b_off + q*b_stride
    int out_off;                 // SORT, INSERT: the output list; MERGE: this item's first output
    int start, cnt;              // MERGE: output ranks start .. start+cnt-1 of merge(A, B);
                                 // INSERT: L elements start .. start+cnt-1
    int last;                    // the item that writes the output list's sentinel slot
};

__host__ __device__ __forceinline__ D1Item d1_unpack(const D1Packed &p, int FW) {
    D1Item t;
    t.a_off = (int)(p.x & 0x1ffffu);
    t.type = (int)((p.x >> 17) & 3u);
    t.a_stride = ((p.x >> 19) & 1u) ? FW : 1;
    t.b_stride = t.a_stride;
    t.last = (int)((p.x >> 20) & 1u);
    t.cnt = (int)(p.x >> 21);
    t.b_off = (int)(p.y & 0x1ffffu);
    t.a_len = (int)(p.y >> 17);
    t.out_off = (int)(p.z & 0x1ffffu);
    t.b_len = (int)(p.z >> 17);
    t.start = (int)p.w;
    return t;
}

// Output ranks t.start .. t.start+t.cnt-1 of merge(A, B) into
// sm[t.out_off ..].
//
// Every list is followed in shared memory by a sentinel slot holding the
// largest key (the plan allocates it, the list's producer writes it), so
// the element after a merge input is either that sentinel or, where the
// input is a leading part of a longer list, the list's next element, which
// ranks after every output of the task (it is never taken).  The loop
// therefore needs no bounds tests: B's sentinel is never taken (a <= it
// always), and A's index is held at its end, so that with A exhausted and B
// at the largest key (equal values: the same output) the merge keeps
// emitting that key without reading past A's sentinel (B's register then
// stays at that key, which is every remaining output).  The last chunk
// writes the output list's own sentinel.
template <class KT>
__host__ __device__ __forceinline__ void d1_merge_item(KT *sm, const D1Item &t) {
    const KT *A = sm + t.a_off;
    const KT *B = sm + t.b_off;
    const int na = t.a_len, nb = t.b_len;
    const int p0 = t.start, cnt = t.cnt;
    // i = number of A elements among the first p0 outputs
    int lo = p0 - nb > 0 ? p0 - nb : 0;
    int hi = p0 < na ? p0 : na;
    while (lo < hi) {
        const int mid = (lo + hi) >> 1;
        // A[mid] precedes B[p0-1-mid] (ties: A first) => more A elements are in front
        if (A[mid] <= B[p0 - 1 - mid]) lo = mid + 1;
        else hi = mid;
    }
    int i = lo;
    KT *out = sm + t.out_off;
    KT a = A[i], b = B[p0 - i];
#pragma unroll 4
    for (int n = 0; n < cnt; n++) {
        const bool ta = a <= b;
        out[n] = ta ? a : b;
        i += ta;
        i = i < na ? i : na;
        // only the list that advanced needs its next element: one
        // shared-memory read a step (the kernel is bound by shared-memory
        // wavefronts; 4096^2 u32 k = 45 12.84 -> 12.26 ms against reading both)
        const KT v = ta ? A[i] : B[p0 + n + 1 - i];
        a = ta ? v : a;
        b = ta ? b : v;
    }
    if (t.last) out[cnt] = d1_sentinel<KT>();
}

template <class KT>
__host__ __device__ __forceinline__ void d1_cx(KT &a, KT &b) {
    const KT lo = a < b ? a : b, hi = a < b ? b : a;
    a = lo;
    b = hi;
}

// out[0 .. n+C) = merge(L, sorted corners), L = sm[a_off .. a_off+n) sorted,
// corners gathered at b_off + q*b_stride.  Ties keep L first, as the merge
// does.  L element i lands at i + #(corners below it); corner q (in sorted
// order) at q + i*_q, i*_q = #(L elements not above it).  The item moves the
// L elements i0 = t.start .. i1 = i0 + t.cnt and places the corners whose
// i*_q falls in [i0, i1) (or at n, for the last item): there i*_q = i1 -
// #(elements of the item above corner q).
template <class KT, int C>
__host__ __device__ __forceinline__ void d1_insert(KT *sm, const D1Item &t) {
    KT s[C];
#pragma unroll
    for (int q = 0; q < C; q++) s[q] = sm[t.b_off + q * t.b_stride];
    if constexpr (C == 2) {
        d1_cx(s[0], s[1]);
    } else if constexpr (C == 4) {
        d1_cx(s[0], s[1]);
        d1_cx(s[2], s[3]);
        d1_cx(s[0], s[2]);
        d1_cx(s[1], s[3]);
        d1_cx(s[1], s[2]);
    }
    const KT *L = sm + t.a_off;
    KT *out = sm + t.out_off;
    const int n = t.a_len;
    const int i0 = t.start, i1 = t.start + t.cnt;
    int above[C];
#pragma unroll
    for (int q = 0; q < C; q++) above[q] = 0;
#pragma unroll 4
    for (int i = i0; i < i1; i++) {
        const KT x = L[i];
        int d = 0;
#pragma unroll
        for (int q = 0; q < C; q++) {
            const int g = s[q] < x;
            d += g;
            above[q] += g;
        }
        out[i + d] = x;
    }
    const KT before = i0 > 0 ? L[i0 - 1] : L[0], last = L[i1 - 1];
#pragma unroll
    for (int q = 0; q < C; q++)
        if ((i0 == 0 || before <= s[q]) && (i1 == n || s[q] < last)) out[q + i1 - above[q]] = s[q];
    if (i1 == n) out[n + C] = d1_sentinel<KT>();
}

template <class KT>
__host__ __device__ __forceinline__ void d1_insert_any(KT *sm, const D1Item &t) {
    if (t.b_len == 1) d1_insert<KT, 1>(sm, t);
    else if (t.b_len == 2) d1_insert<KT, 2>(sm, t);
    else d1_insert<KT, 4>(sm, t);
}

}  // namespace mf
