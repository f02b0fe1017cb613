// Data-oblivious variant (paper Sec. 4): one root tile per thread, its whole
// hierarchical selection network unrolled into register min/max code.
//
// Block: BX x BY threads, each owning `lanes` root tiles of TW x TH pixels
// (two tiles per thread for 8/16-bit data, packed in the two 16-bit halves
// of every register: the network is data-oblivious, so both run the same
// instruction stream).  The lane-0 tiles cover the left half of the block's
// region, the lane-1 tiles the right half.
//
// Stages (paper Sec. 4.3, re-planned for sm_103a):
//   1. the block footprint (clamp-to-edge) is loaded into shared memory as
//      keys, two lanes per 32-bit word;
//   2. every footprint column, restricted to the root-core rows of each
//      tile row, is sorted once (round-robin over the block's threads) and
//      written back: horizontally adjacent tiles share these sorted columns
//      (Sec. 3.3, column sort);
//   3. each thread runs the generated network for its tile: multi-way merge
//      of its sorted core columns, sorting of its extra rows, then the
//      horizontal/vertical splits down to single pixels (Sec. 3.4), reading
//      its inputs from shared memory at compile-time offsets;
//   4. the TW x TH medians of every lane are stored (or, in argmedian mode,
//      the source index recovered from the composite record).
// Networks flagged `direct` (small k) run o1_block_direct instead: each
// thread loads its own footprint into registers and sorts its own columns,
// with no shared memory and no barrier.
//
// Shared-memory words are stored column-group-transposed: word (row, gx) at
// row*RS + (gx % TW)*G + gx / TW with G odd.  Thread tx then reads
// footprint column tx*TW + fx at base + tx + const, so a warp's 32 lanes
// hit 32 consecutive words (no bank conflicts) for every network input.
#pragma once
#include <type_traits>

#include "mf_common.cuh"

namespace mf {

template <int K, int TW, int TH, int BX, int BY, bool ROWS = false>
struct O1Layout {
    static constexpr int R = (K - 1) / 2;
    static constexpr int FW = BX * TW + K - 1;  // footprint width of one lane half
    static constexpr int FH = BY * TH + K - 1;  // footprint height
    static constexpr int CH0 = K - TH + 1;      // root core height
    static constexpr int NG = (FW + TW - 1) / TW;
    static constexpr int G = NG | 1;            // odd stride between column residues
    static constexpr int RS = TW * G;           // words per shared-memory row
    static constexpr int CSB = FH * RS;         // start of the sorted column segments
    static constexpr int CSTY = CH0 * RS;       // words per tile row of segments
    // optional: each thread's root extra rows, sorted, in a slot of its own
    // (odd stride: the 32 lanes of a warp hit 32 different banks)
    static constexpr int CW0 = K - TW + 1;      // root core width
    static constexpr int NRW = 2 * (TH - 1);    // extra rows per root tile
    static constexpr int RSTRIDE = (NRW * CW0) | 1;
    static constexpr int RSB = CSB + BY * CSTY;
    static constexpr int WORDS = (RSB + (ROWS ? BX * BY * RSTRIDE : 0) + 3) & ~3;
    static __host__ __device__ constexpr int at(int fy, int gx) {
        return fy * RS + (gx % TW) * G + gx / TW;
    }
    // offsets relative to a thread's base (tx folded in): raw pixel and
    // element i of the sorted segment of footprint column fx
    static __host__ __device__ constexpr int px(int fy, int fx) {
        return fy * RS + (fx % TW) * G + fx / TW;
    }
    static __host__ __device__ constexpr int col(int fx, int i) {
        return i * RS + (fx % TW) * G + fx / TW;
    }
    // element i of the sorted extra row fy (footprint row) in the thread's slot
    static __host__ __device__ constexpr int row(int fy, int i) {
        return (fy < TH - 1 ? fy : TH - 1 + fy - K) * CW0 + i;
    }
};

// Builds the comparison word of footprint element (fy, gx) for every lane.
// Value mode: the key (two 16-bit keys per word for 8/16-bit data).
// Argmedian mode: the composite record key << IB | (fy * FW + gx), which
// orders equal keys by block-footprint row-major position -- within one
// pixel's window that is its row-major window-slot order.
template <int DT, class KO, bool ARG, int IB>
struct O1Words;

// row: the clamped source row; xl0 / xl1: the clamped columns of lanes 0 / 1.
template <int DT, int IB>
struct O1Words<DT, KoU16x2, false, IB> {
    template <class L>
    static __device__ __forceinline__ uint32_t make(const typename Dt<DT>::E *row, int xl0, int xl1, int, int) {
        const uint32_t k0 = Dt<DT>::key(__ldg(row + xl0));
        const uint32_t k1 = Dt<DT>::key(__ldg(row + xl1));
        return k0 | (k1 << 16);
    }
};

template <int DT, int IB>
struct O1Words<DT, KoU32, false, IB> {
    template <class L>
    static __device__ __forceinline__ uint32_t make(const typename Dt<DT>::E *row, int xl0, int, int, int) {
        return Dt<DT>::key(__ldg(row + xl0));
    }
};

template <int DT, int IB>
struct O1Words<DT, KoU32, true, IB> {  // 8/16-bit argmedian: key << IB | index
    template <class L>
    static __device__ __forceinline__ uint32_t make(const typename Dt<DT>::E *row, int xl0, int, int fy, int gx) {
        return (Dt<DT>::key(__ldg(row + xl0)) << IB) | (uint32_t)(fy * L::FW + gx);
    }
};

template <int DT, int IB>
struct O1Words<DT, KoU64, true, IB> {  // 32-bit argmedian: key << 32 | index
    template <class L>
    static __device__ __forceinline__ unsigned long long make(const typename Dt<DT>::E *row, int xl0, int, int fy,
                                                              int gx) {
        return ((unsigned long long)Dt<DT>::key(__ldg(row + xl0)) << 32) | (unsigned long long)(fy * L::FW + gx);
    }
};

// Writes the median of tile pixel `pix` (row-major in the TW x TH tile) of
// every lane: the value, or in argmedian mode the value and the source index
// recovered from the composite record.
template <int K, int TW, int TH, int BX, int BY, int DT, class KO, bool ARG, int IB>
struct O1Store {
    typedef O1Layout<K, TW, TH, BX, BY> L;  // FW and R do not depend on ROWS
    typedef typename KO::T T;
    typedef typename Dt<DT>::E E;
    static constexpr int OW = KO::lanes * BX * TW;  // output tile width (elements)
    const ImgArgs &a;
    char *dst;
    char *idx;
    int bx0, by0, tx, ty;
    E *otile;  // value mode: the block's output tile in shared memory
    __device__ __forceinline__ void operator()(int pix, T w) const {
        constexpr int P = KO::lanes;
        const int py = pix / TW, px = pix - py * TW;
        if (!ARG) {  // into the shared output tile; written out coalesced later
#pragma unroll
            for (int l = 0; l < P; l++) {
                const uint32_t key = P == 2 ? (uint32_t)((w >> (16 * l)) & 0xffffu) : (uint32_t)w;
                otile[(ty * TH + py) * OW + l * BX * TW + tx * TW + px] = Dt<DT>::val(key);
            }
            return;
        }
        const int y = by0 + ty * TH + py;
        if (y >= a.H) return;
#pragma unroll
        for (int l = 0; l < P; l++) {
            const int x = bx0 + l * BX * TW + tx * TW + px;
            if (x >= a.W) continue;
            {
                const uint32_t fidx = (uint32_t)(w & ((1ull << IB) - 1));
                const uint32_t key = (uint32_t)(w >> IB);
                const int fy = fidx / L::FW, gx = fidx - fy * L::FW;
                const int ys = clampi(by0 - L::R + fy, a.y_lo, a.y_hi);
                const int xs = clampi(bx0 - L::R + gx, 0, a.W - 1);
                if (dst) reinterpret_cast<E *>(dst + (size_t)y * a.pitch)[x] = Dt<DT>::val(key);
                if (idx) reinterpret_cast<int32_t *>(idx + (size_t)y * a.idx_pitch)[x] = ys * a.W + xs;
            }
        }
    }
};

// ------------------------------------------------------------ direct form
// For small k the staging, column-sort and output stages of the shared-
// memory form cost more instructions per pixel than the network itself.
// The direct form gives every thread its own (TH + K - 1) x (TW + K - 1)
// footprint in registers (clamp-to-edge loads that neighbouring threads
// share through L1), sorts its own column segments and stores its medians
// straight to global memory: no shared memory and no barriers.  Block and
// tile geometry are those of the shared-memory form (lane-0 tiles in the
// left half of the block's region, lane-1 tiles in the right half), so the
// batched paths cut work items the same way.
template <int K, int TW, int TH>
struct O1RegLayout {
    static constexpr int FW = TW + K - 1;   // footprint of one tile
    static constexpr int FH = TH + K - 1;
    static constexpr int CH0 = K - TH + 1;  // root core height
    static __host__ __device__ constexpr int px(int fy, int fx) { return fy * FW + fx; }
    static __host__ __device__ constexpr int col(int fx, int i) { return fx * CH0 + i; }
    static __host__ __device__ constexpr int row(int, int) { return 0; }  // not used: no shared rows
};

// Collects the tile's medians in registers (the flat network calls it with
// constant pixel indices).
template <class T, int N>
struct O1Collect {
    T *res;
    __device__ __forceinline__ void operator()(int pix, T w) const { res[pix] = w; }
};

template <int K, int TW, int TH, int BX, int BY, int DT, class KO, class NET, class CSORT>
__device__ __forceinline__ void o1_block_direct(const ImgArgs &a, int bxi, int byi, int z) {
    typedef O1RegLayout<K, TW, TH> RL;
    typedef typename KO::T T;
    typedef typename Dt<DT>::E E;
    constexpr int P = KO::lanes, R = (K - 1) / 2, LX = BX * TW;  // LX: lane-1 column offset
    const int tx = threadIdx.x % BX, ty = threadIdx.x / BX;
    const int x0 = bxi * (P * BX * TW) + tx * TW;
    const int y0 = byi * (BY * TH) + ty * TH;
    if (x0 >= a.W || y0 >= a.H) return;  // whole tile (both lanes) outside
    const char *src = a.src + (size_t)z * a.plane;
    T f[RL::FH * RL::FW];
    // footprint in registers.  Inside the image every row is one pointer and
    // the columns are constant offsets from it; near the border each column
    // and row is clamped.
    const bool inside = x0 - R >= 0 && x0 + (P - 1) * LX - R + RL::FW - 1 < a.W && y0 - R >= a.y_lo &&
                        y0 - R + RL::FH - 1 <= a.y_hi;
    if (inside) {
#pragma unroll
        for (int fy = 0; fy < RL::FH; fy++) {
            const E *row = reinterpret_cast<const E *>(src + (ptrdiff_t)(y0 - R + fy) * (ptrdiff_t)a.pitch) + (x0 - R);
#pragma unroll
            for (int fx = 0; fx < RL::FW; fx++)
                f[RL::px(fy, fx)] = O1Words<DT, KO, false, 0>::template make<RL>(row, fx, fx + LX, 0, 0);
        }
    } else {
        int xc0[RL::FW], xc1[RL::FW];
#pragma unroll
        for (int fx = 0; fx < RL::FW; fx++) {
            xc0[fx] = clampi(x0 - R + fx, 0, a.W - 1);
            xc1[fx] = clampi(x0 + LX - R + fx, 0, a.W - 1);
        }
#pragma unroll
        for (int fy = 0; fy < RL::FH; fy++) {
            const E *row = reinterpret_cast<const E *>(src + (ptrdiff_t)clampi(y0 - R + fy, a.y_lo, a.y_hi) * (ptrdiff_t)a.pitch);
#pragma unroll
            for (int fx = 0; fx < RL::FW; fx++)
                f[RL::px(fy, fx)] = O1Words<DT, KO, false, 0>::template make<RL>(row, xc0[fx], xc1[fx], 0, 0);
        }
    }
    // the tile's own column segments over the root core rows
    T cs[RL::FW * RL::CH0];
#pragma unroll
    for (int fx = 0; fx < RL::FW; fx++) {
        T v[RL::CH0];
#pragma unroll
        for (int i = 0; i < RL::CH0; i++) v[i] = f[RL::px(TH - 1 + i, fx)];
        CSORT::template run<KO>(v);
#pragma unroll
        for (int i = 0; i < RL::CH0; i++) cs[RL::col(fx, i)] = v[i];
    }
    T res[TW * TH];
    O1Collect<T, TW * TH> out{res};
    NET::template run<KO, RL>(cs, f, f, out);
    // medians out: constant offsets from one row pointer when the tiles of
    // both lanes lie inside the image, else element by element
    char *dst = a.dst + (size_t)z * a.plane;
    const bool full = y0 + TH - 1 < a.H && x0 + (P - 1) * LX + TW - 1 < a.W;
#pragma unroll
    for (int py = 0; py < TH; py++) {
        const int y = y0 + py;
        if (!full && y >= a.H) break;
        E *orow = reinterpret_cast<E *>(dst + (size_t)y * a.pitch) + x0;
#pragma unroll
        for (int l = 0; l < P; l++)
#pragma unroll
            for (int px = 0; px < TW; px++) {
                const T w = res[py * TW + px];
                const uint32_t key = P == 2 ? (uint32_t)((w >> (16 * l)) & 0xffffu) : (uint32_t)w;
                if (full || x0 + l * LX + px < a.W) orow[l * LX + px] = Dt<DT>::val(key);
            }
    }
}

// ------------------------------------------------------- wide direct form
// Tiles of a lane per thread (NTX) for networks emitted in the wide form
// (NET::wide), 1 otherwise.
template <class N, class = void>
struct NetWide {
    static constexpr int v = 1;
};
template <class N>
struct NetWide<N, std::void_t<decltype(N::wide)>> {
    static constexpr int v = N::wide;
};

// Footprint of a lane's run of tiles in registers: FWL columns, the sorted
// column segments CH0 long.
template <int FWL, int CH0>
struct O1RunLayout {
    static __host__ __device__ constexpr int px(int fy, int fx) { return fy * FWL + fx; }
    static __host__ __device__ constexpr int col(int fx, int i) { return fx * CH0 + i; }
    static __host__ __device__ constexpr int row(int, int) { return 0; }
};

// Row buffer of the wide form: HB + RUN*P + HB elements of one footprint
// row, starting HB elements left of the run, as 32-bit words.
template <class E, int NE>
struct O1RowBuf {
    static constexpr int WORDS = NE * (int)sizeof(E) / 4;
    uint32_t w[WORDS];
    // element i (compile-time i) as a raw value
    __device__ __forceinline__ uint32_t elem(int i) const {
        if (sizeof(E) == 1) return (w[i >> 2] >> (8 * (i & 3))) & 0xffu;
        if (sizeof(E) == 2) return (w[i >> 1] >> (16 * (i & 1))) & 0xffffu;
        return w[i];
    }
};

// Comparison word of the two lanes' elements i0 and i1 of a row buffer.
// 8-bit data: each 16-bit lane holds v * 257 (the byte in both halves of
// the lane: one byte permute builds both lanes, and v -> 257 v keeps the
// order and is one to one).  16-bit data: the two elements' halves.
// 32-bit data (one lane): the order key.
template <int DT, class KO, class BUF>
__device__ __forceinline__ typename KO::T o1_pack(const BUF &b, int i0, int i1) {
    typedef typename Dt<DT>::E E;
    if constexpr (KO::lanes == 2 && sizeof(E) == 1) {
        const int a = i0 & 3, c = i1 & 3;
        return __byte_perm(b.w[i0 >> 2], b.w[i1 >> 2], (unsigned)(a | a << 4 | (4 + c) << 8 | (4 + c) << 12));
    } else if constexpr (KO::lanes == 2) {
        const int a = 2 * (i0 & 1), c = 4 + 2 * (i1 & 1);
        return __byte_perm(b.w[i0 >> 1], b.w[i1 >> 1], (unsigned)(a | (a + 1) << 4 | c << 8 | (c + 1) << 12));
    } else {
        return (typename KO::T)Dt<DT>::key((typename Dt<DT>::E)b.elem(i0));
    }
}

// Wide direct form for small k: each thread owns NTX horizontally adjacent
// root tiles per lane, the lanes side by side (lane 1's tiles start RUN =
// NTX*TW columns after lane 0's), i.e. one contiguous run of P*RUN columns
// by TH rows.  Where the run and its halo lie inside the image, every
// footprint row is read with vector loads of up to 16 bytes;
// the two lanes' elements are packed with one byte permute per word; the
// NTX tiles of a lane share their sorted footprint columns (Sec. 3.3); the
// medians go out as vector stores.  Near the borders the same row buffers
// are filled by clamped element loads and the medians stored one by one.
template <int K, int TW, int TH, int BX, int BY, int DT, class KO, class NET, class CSORT, int NTX>
__device__ __forceinline__ void o1_block_wide(const ImgArgs &a, int bxi, int byi, int z) {
    typedef typename KO::T T;
    typedef typename Dt<DT>::E E;
    constexpr int P = KO::lanes, R = (K - 1) / 2;
    constexpr int RUN = NTX * TW, TOT = P * RUN;
    constexpr int HB = 16 / (int)sizeof(E) < 4 ? 16 / (int)sizeof(E) : 4;  // halo elements each side (>= R)
    constexpr int NE = TOT + 2 * HB;
    constexpr int FWL = RUN + K - 1, FH = TH + K - 1, CH0 = K - TH + 1;
    static_assert(R <= HB, "halo wider than the row buffer");
    static_assert(P == 1 || RUN % (sizeof(E) == 1 ? 4 : 2) == 0, "lane runs of whole output words");
    static_assert((TOT * (int)sizeof(E)) % 4 == 0 && (HB * (int)sizeof(E)) % 4 == 0, "vector geometry");
    typedef O1RunLayout<FWL, CH0> RL;
    const int tx = threadIdx.x % BX, ty = threadIdx.x / BX;
    const int x0 = bxi * (BX * TOT) + tx * TOT;
    const int y0 = byi * (BY * TH) + ty * TH;
    if (x0 >= a.W || y0 >= a.H) return;
    const char *src = a.src + (size_t)z * a.plane;
    // vector loads need the run and its halo inside the row and 16-byte
    // aligned rows (x0 * sizeof(E) is a multiple of 16 by construction)
    const bool vec = x0 - HB >= 0 && x0 + TOT + HB <= a.W && ((a.pitch | (size_t)src) & 15) == 0;
    T f[FH * FWL];
#pragma unroll
    for (int fy = 0; fy < FH; fy++) {
        const int y = clampi(y0 - R + fy, a.y_lo, a.y_hi);
        const E *row = reinterpret_cast<const E *>(src + (ptrdiff_t)y * (ptrdiff_t)a.pitch);
        O1RowBuf<E, NE> b;
        constexpr int HW = HB * (int)sizeof(E) / 4;   // halo words each side
        constexpr int MW = TOT * (int)sizeof(E) / 4;  // run words
        if (vec) {
            const uint32_t *wr = reinterpret_cast<const uint32_t *>(row + x0);
            if constexpr (HW == 1) {
                b.w[0] = __ldg(wr - 1);
                b.w[HW + MW] = __ldg(wr + MW);
            } else if constexpr (HW == 2) {
                const uint2 l = __ldg(reinterpret_cast<const uint2 *>(wr) - 1);
                const uint2 r = __ldg(reinterpret_cast<const uint2 *>(wr + MW));
                b.w[0] = l.x; b.w[1] = l.y; b.w[HW + MW] = r.x; b.w[HW + MW + 1] = r.y;
            } else {
                const uint4 l = __ldg(reinterpret_cast<const uint4 *>(wr) - 1);
                const uint4 r = __ldg(reinterpret_cast<const uint4 *>(wr + MW));
                b.w[0] = l.x; b.w[1] = l.y; b.w[2] = l.z; b.w[3] = l.w;
                b.w[HW + MW] = r.x; b.w[HW + MW + 1] = r.y; b.w[HW + MW + 2] = r.z; b.w[HW + MW + 3] = r.w;
            }
            if constexpr (MW % 4 == 0) {
#pragma unroll
                for (int m = 0; m < MW / 4; m++) {
                    const uint4 v = __ldg(reinterpret_cast<const uint4 *>(wr) + m);
                    b.w[HW + 4 * m] = v.x; b.w[HW + 4 * m + 1] = v.y; b.w[HW + 4 * m + 2] = v.z; b.w[HW + 4 * m + 3] = v.w;
                }
            } else if constexpr (MW % 2 == 0) {
#pragma unroll
                for (int m = 0; m < MW / 2; m++) {
                    const uint2 v = __ldg(reinterpret_cast<const uint2 *>(wr) + m);
                    b.w[HW + 2 * m] = v.x; b.w[HW + 2 * m + 1] = v.y;
                }
            } else {
#pragma unroll
                for (int m = 0; m < MW; m++) b.w[HW + m] = __ldg(wr + m);
            }
        } else {
#pragma unroll
            for (int m = 0; m < b.WORDS; m++) b.w[m] = 0;
#pragma unroll
            for (int i = 0; i < NE; i++) {
                if (i < HB - R || i >= HB + TOT + R) continue;  // never read
                const uint32_t v = (uint32_t)__ldg(row + clampi(x0 - HB + i, 0, a.W - 1));
                b.w[i * (int)sizeof(E) / 4] |= v << (8 * ((i * (int)sizeof(E)) & 3));
            }
        }
#pragma unroll
        for (int fx = 0; fx < FWL; fx++) f[RL::px(fy, fx)] = o1_pack<DT, KO>(b, HB - R + fx, HB - R + fx + RUN);
    }
    // the lane's footprint columns over the root core rows, shared by its NTX tiles
    T cs[FWL * CH0];
#pragma unroll
    for (int fx = 0; fx < FWL; fx++) {
        T v[CH0];
#pragma unroll
        for (int i = 0; i < CH0; i++) v[i] = f[RL::px(TH - 1 + i, fx)];
        CSORT::template run<KO>(v);
#pragma unroll
        for (int i = 0; i < CH0; i++) cs[RL::col(fx, i)] = v[i];
    }
    T res[NTX * TW * TH];
#pragma unroll
    for (int q = 0; q < NTX; q++) {
        O1Collect<T, TW * TH> out{res + q * TW * TH};
        NET::template run<KO, RL>(cs + q * TW * CH0, f + q * TW, f + q * TW, out);
    }
    // medians out: output column c of row py is lane c / RUN, tile (c % RUN) / TW
    char *dst = a.dst + (size_t)z * a.plane;
    const bool vst = x0 + TOT <= a.W && ((a.pitch | (size_t)dst) & 15) == 0;
#pragma unroll
    for (int py = 0; py < TH; py++) {
        const int y = y0 + py;
        if (y >= a.H) break;
        E *orow = reinterpret_cast<E *>(dst + (size_t)y * a.pitch) + x0;
        auto med = [&](int c) -> uint32_t {  // median key of output column c (compile-time c)
            const int l = c / RUN, cc = c % RUN;
            const T w = res[(cc / TW) * TW * TH + py * TW + cc % TW];
            return P == 2 ? (uint32_t)((w >> (16 * l)) & 0xffffu) : (uint32_t)w;
        };
        if (vst) {
            constexpr int OW = TOT * (int)sizeof(E) / 4;  // output words
            uint32_t o[OW];
            // the packed median of lane-0 column cc (both lanes in one word)
            auto rw = [&](int cc) -> uint32_t { return (uint32_t)res[(cc / TW) * TW * TH + py * TW + cc % TW]; };
            if constexpr (sizeof(E) == 1) {
                // lanes hold 257 v, so bytes 0 and 2 of a packed word are the
                // two lanes' values: two permutes gather four columns of
                // both lanes, two more make the lane-0 and lane-1 words
#pragma unroll
                for (int m = 0; m < RUN / 4; m++) {
                    const uint32_t t01 = __byte_perm(rw(4 * m), rw(4 * m + 1), 0x6240);
                    const uint32_t t23 = __byte_perm(rw(4 * m + 2), rw(4 * m + 3), 0x6240);
                    o[m] = __byte_perm(t01, t23, 0x5410);
                    o[RUN / 4 + m] = __byte_perm(t01, t23, 0x7632);
                }
            } else if constexpr (sizeof(E) == 2) {
#pragma unroll
                for (int m = 0; m < RUN / 2; m++) {
                    o[m] = __byte_perm(rw(2 * m), rw(2 * m + 1), 0x5410);
                    o[RUN / 2 + m] = __byte_perm(rw(2 * m), rw(2 * m + 1), 0x7632);
                }
            } else {
#pragma unroll
                for (int m = 0; m < OW; m++) o[m] = Dt<DT>::val(med(m));
            }
            if constexpr (OW % 4 == 0) {
#pragma unroll
                for (int m = 0; m < OW / 4; m++)
                    reinterpret_cast<uint4 *>(orow)[m] = make_uint4(o[4 * m], o[4 * m + 1], o[4 * m + 2], o[4 * m + 3]);
            } else if constexpr (OW % 2 == 0) {
#pragma unroll
                for (int m = 0; m < OW / 2; m++) reinterpret_cast<uint2 *>(orow)[m] = make_uint2(o[2 * m], o[2 * m + 1]);
            } else {
#pragma unroll
                for (int m = 0; m < OW; m++) reinterpret_cast<uint32_t *>(orow)[m] = o[m];
            }
        } else {
#pragma unroll
            for (int c = 0; c < TOT; c++) {
                if (x0 + c >= a.W) break;
                const uint32_t kv = med(c);
                orow[c] = sizeof(E) == 1 ? (E)(kv & 0xffu) : Dt<DT>::val(kv);
            }
        }
    }
}

// One block's work: the block of tiles at (bxi, byi) of plane z.
template <int K, int TW, int TH, int BX, int BY, int DT, class KO, bool ARG, int IB, class NET,
          class CSORT, class RSORT>
__device__ __forceinline__ void o1_block(const ImgArgs &a, int bxi, int byi, int z) {
    if constexpr (NET::direct) {
        static_assert(!ARG, "the direct form computes values only");
        if constexpr (NetWide<NET>::v > 1)
            o1_block_wide<K, TW, TH, BX, BY, DT, KO, NET, CSORT, NetWide<NET>::v>(a, bxi, byi, z);
        else
            o1_block_direct<K, TW, TH, BX, BY, DT, KO, NET, CSORT>(a, bxi, byi, z);
        return;
    }
    typedef O1Layout<K, TW, TH, BX, BY, NET::rows_smem> L;
    typedef typename KO::T T;
    typedef typename Dt<DT>::E E;
    constexpr int P = KO::lanes;
    constexpr int NT = BX * BY;
    extern __shared__ __align__(16) unsigned char o1_smem[];
    T *sm = reinterpret_cast<T *>(o1_smem);

    const int tid = threadIdx.x;
    const int tx = tid % BX, ty = tid / BX;
    const int bx0 = bxi * (P * BX * TW);
    const int by0 = byi * (BY * TH);
    const char *src = a.src + (size_t)z * a.plane;

    // 1. block footprint -> shared memory (clamp to edge): one work item is
    //    one footprint column over a group of 4 rows, so the column's
    //    clamps and shared-memory offset are computed once per 4 elements
    constexpr int RG = 4, NRG = (L::FH + RG - 1) / RG;
    for (int i = tid; i < L::FW * NRG; i += NT) {
        const int g = i / L::FW, gx = i - g * L::FW;
        const int x0 = clampi(bx0 - L::R + gx, 0, a.W - 1);
        const int x1 = clampi(bx0 + BX * TW - L::R + gx, 0, a.W - 1);
        const int sw = (gx % TW) * L::G + gx / TW;
#pragma unroll
        for (int j = 0; j < RG; j++) {
            const int fy = g * RG + j;
            if (RG * NRG != L::FH && fy >= L::FH) break;
            const int y = clampi(by0 - L::R + fy, a.y_lo, a.y_hi);
            const E *row = reinterpret_cast<const E *>(src + (ptrdiff_t)y * (ptrdiff_t)a.pitch);
            sm[fy * L::RS + sw] = O1Words<DT, KO, ARG, IB>::template make<L>(row, x0, x1, fy, gx);
        }
    }
    __syncthreads();

    // 2. sort every footprint column over the root-core rows of each tile row
    for (int i = tid; i < BY * L::FW; i += NT) {
        const int cty = i / L::FW, gx = i - cty * L::FW;
        T v[L::CH0];
#pragma unroll
        for (int j = 0; j < L::CH0; j++) v[j] = sm[L::at(cty * TH + TH - 1 + j, gx)];
        CSORT::template run<KO>(v);
        T *dstc = sm + L::CSB + cty * L::CSTY + (gx % TW) * L::G + gx / TW;
#pragma unroll
        for (int j = 0; j < L::CH0; j++) dstc[j * L::RS] = v[j];
    }
    __syncthreads();

    // 2b. (networks that take their extra rows sorted) each thread sorts the
    //     root extra rows of its own tile into its slot; the barrier makes the
    //     network reload them where it uses them instead of holding them in
    //     registers through the core initialisation
    if (NET::rows_smem) {
        const T *rwt = sm + ty * TH * L::RS + tx;
        T *rst = sm + L::RSB + (ty * BX + tx) * L::RSTRIDE;
#pragma unroll 1
        for (int r = 0; r < L::NRW; r++) {
            const int fy = r < TH - 1 ? r : K + r - (TH - 1);
            T v[L::CW0];
#pragma unroll
            for (int j = 0; j < L::CW0; j++) v[j] = rwt[fy * L::RS + ((TW - 1 + j) % TW) * L::G + (TW - 1 + j) / TW];
            RSORT::template run<KO>(v);
#pragma unroll
            for (int j = 0; j < L::CW0; j++) rst[r * L::CW0 + j] = v[j];
        }
        __syncthreads();
    }

    // 3. the tile's hierarchical network; each median goes straight to
    //    the store functor as the recursion reaches its leaf
    typedef O1Store<K, TW, TH, BX, BY, DT, KO, ARG, IB> Store;
    E *otile = reinterpret_cast<E *>(sm + L::WORDS);
    Store out{a, a.dst ? a.dst + (size_t)z * a.plane : nullptr,
              a.idx ? reinterpret_cast<char *>(a.idx) + (size_t)z * a.idx_plane : nullptr, bx0, by0, tx, ty, otile};
    NET::template run<KO, L>(sm + L::CSB + ty * L::CSTY + tx, sm + ty * TH * L::RS + tx,
                             sm + L::RSB + (ty * BX + tx) * L::RSTRIDE, out);

    // 4. value mode: the output tile goes out as full 16-byte rows where the
    //    block lies inside the image and the row start is aligned, else
    //    element by element
    if (!ARG && a.dst) {
        __syncthreads();
        constexpr int OW = Store::OW, OH = BY * TH;
        constexpr int VEC = 16 / (int)sizeof(E);  // elements per 16-byte store
        char *dst = a.dst + (size_t)z * a.plane;
        const bool full = bx0 + OW <= a.W && ((a.pitch | (size_t)dst | ((size_t)bx0 * sizeof(E))) & 15) == 0;
        if (full && OW % VEC == 0) {
            for (int i = tid; i < OH * (OW / VEC); i += NT) {
                const int r = i / (OW / VEC), c = i - r * (OW / VEC);
                const int y = by0 + r;
                if (y >= a.H) continue;
                const uint4 v = reinterpret_cast<const uint4 *>(otile + r * OW)[c];
                reinterpret_cast<uint4 *>(dst + (size_t)y * a.pitch + (size_t)bx0 * sizeof(E))[c] = v;
            }
        } else {
            for (int i = tid; i < OH * OW; i += NT) {
                const int r = i / OW, c = i - r * OW;
                const int y = by0 + r, x = bx0 + c;
                if (y < a.H && x < a.W) reinterpret_cast<E *>(dst + (size_t)y * a.pitch)[x] = otile[i];
            }
        }
    }
}

template <int K, int TW, int TH, int BX, int BY, int DT, class KO, bool ARG, int IB, class NET,
          class CSORT, class RSORT>
__global__ void __launch_bounds__(BX *BY) o1_kernel(ImgArgs a) {
    o1_block<K, TW, TH, BX, BY, DT, KO, ARG, IB, NET, CSORT, RSORT>(a, blockIdx.x, blockIdx.y, blockIdx.z);
}

// Persistent form for batches: each block repeatedly claims the next work
// item (image, block x, block y, plane) from a device counter until the
// list is exhausted.  Claims are atomic increments -- no block ever waits
// on another.
template <int K, int TW, int TH, int BX, int BY, int DT, class KO, bool ARG, int IB, class NET,
          class CSORT, class RSORT>
__global__ void __launch_bounds__(BX *BY) o1_persistent(const ImgArgs *imgs, const int4 *items, int n_items,
                                                        unsigned *counter) {
    __shared__ int s_item;
    for (;;) {
        if (threadIdx.x == 0) s_item = (int)atomicAdd(counter, 1u);
        __syncthreads();
        const int it = s_item;
        if (it >= n_items) break;
        const int4 w = items[it];
        o1_block<K, TW, TH, BX, BY, DT, KO, ARG, IB, NET, CSORT, RSORT>(imgs[w.x], w.y, w.z, w.w);
        __syncthreads();  // shared memory is reused by the next item
    }
}

// Shared memory of one block: the layout's words plus, in value mode, the
// output tile (16-byte aligned: the layout's word count is rounded up).
template <int K, int TW, int TH, int BX, int BY, int DT, class KO, bool ARG, class NET>
constexpr size_t o1_smem_bytes() {
    typedef O1Layout<K, TW, TH, BX, BY, NET::rows_smem> L;
    return NET::direct ? 0
                       : sizeof(typename KO::T) * (size_t)L::WORDS +
                             (ARG ? 0 : (size_t)KO::lanes * BX * TW * BY * TH * sizeof(typename Dt<DT>::E));
}

template <int K, int TW, int TH, int BX, int BY, int DT, class KO, bool ARG, int IB, class NET,
          class CSORT, class RSORT>
int persist_o1(const ImgArgs *imgs, const int4 *items, int n_items, unsigned *counter, int blocks_per_sm,
               int sms, cudaStream_t s, int *grid_out) {
    typedef O1Layout<K, TW, TH, BX, BY, NET::rows_smem> L;
    constexpr size_t smem = o1_smem_bytes<K, TW, TH, BX, BY, DT, KO, ARG, NET>();
    auto kern = o1_persistent<K, TW, TH, BX, BY, DT, KO, ARG, IB, NET, CSORT, RSORT>;
    static DevMask configured;
    int cfg_dev = 0;
    if (!dev_configured(configured, &cfg_dev)) {
        if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess)
            return MF_ERR_CUDA;
        dev_mark_configured(configured, cfg_dev);
    }
    // n_items == 0: prepare only (attributes, occupancy -> *grid_out as
    // blocks per SM); call this outside stream capture
    if (n_items == 0) {
        int occ = 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, BX * BY, smem) != cudaSuccess)
            return MF_ERR_CUDA;
        *grid_out = occ < 1 ? 1 : occ;
        return MF_OK;
    }
    const int occ = blocks_per_sm > 0 ? blocks_per_sm : 1;
    int grid = occ * sms;
    if (grid > n_items) grid = n_items;
    if (grid < 1) grid = 1;
    *grid_out = grid;
    kern<<<grid, BX * BY, smem, s>>>(imgs, items, n_items, counter);
    return cudaPeekAtLastError() == cudaSuccess ? MF_OK : MF_ERR_CUDA;
}

template <int K, int TW, int TH, int BX, int BY, int DT, class KO, bool ARG, int IB, class NET,
          class CSORT, class RSORT>
int launch_o1(const ImgArgs &a, int channels, cudaStream_t s) {
    constexpr int P = KO::lanes;
    constexpr size_t smem = o1_smem_bytes<K, TW, TH, BX, BY, DT, KO, ARG, NET>();
    auto kern = o1_kernel<K, TW, TH, BX, BY, DT, KO, ARG, IB, NET, CSORT, RSORT>;
    static DevMask configured;
    int cfg_dev = 0;
    if (!dev_configured(configured, &cfg_dev)) {
        if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) !=
            cudaSuccess)
            return MF_ERR_CUDA;
        // ask for no more shared memory than the resident blocks use: the rest
        // of the SM's 256 KB stays L1, where register spills of the large
        // networks hit
        int occ = 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, BX * BY, smem) == cudaSuccess && occ > 0) {
            const int pct = (int)((occ * (smem + 1024) * 100 + 228 * 1024 - 1) / (228 * 1024));
            cudaFuncSetAttribute(kern, cudaFuncAttributePreferredSharedMemoryCarveout, pct > 100 ? 100 : pct);
        }
        cudaGetLastError();
        dev_mark_configured(configured, cfg_dev);
    }
    constexpr int RW = P * BX * TW * NetWide<NET>::v;  // columns of a block's region
    dim3 grid((a.W + RW - 1) / RW, (a.H + BY * TH - 1) / (BY * TH), channels);
    kern<<<grid, BX * BY, smem, s>>>(a);
    count_launch();
    return cudaPeekAtLastError() == cudaSuccess ? MF_OK : MF_ERR_CUDA;
}

}  // namespace mf
