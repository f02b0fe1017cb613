// Argmedian from a computed median.
//
// Under the order (key, row-major window slot) the rank-m element of a
// window (m = (k*k-1)/2) has the median key v, and it is the j-th element
// with key v in slot order, j = m - #{window keys < v} (0-based): all
// elements below v precede it, and equal keys order by slot.  Given the
// median value (from any of the value kernels), one branch-free pass over
// the window counts the keys below v and equal to v and keeps the last
// equal slot; that slot is the answer when the median is the last of its
// ties in slot order (always, without ties), else a second pass finds the
// j-th equal key.  The window is read from a shared-memory tile of the
// block's footprint (clamp-to-edge); for 32-bit data at k <= 27 the window
// width is a compile-time constant and each window row is unrolled.
#include <cstdlib>

#include "mf_registry.h"

namespace mf {

constexpr int AM_BW = 32, AM_BH = 8;

// KC > 0: k fixed at compile time (every window loop unrolled, shared-memory
// offsets constant); KC = 0: k at run time.
template <int DT, int KC>
__global__ void __launch_bounds__(AM_BW *AM_BH) argmedian_kernel(ImgArgs a, int k_rt) {
    const int k = KC > 0 ? KC : k_rt;
    extern __shared__ __align__(16) uint32_t am_smem[];
    typedef typename Dt<DT>::E E;
    const int r = (k - 1) / 2;
    const int SW = AM_BW + k - 1, SH = AM_BH + k - 1;
    const int x0 = blockIdx.x * AM_BW, y0 = blockIdx.y * AM_BH, z = blockIdx.z;
    const char *src = a.src + (size_t)z * a.plane;
    const int tid = threadIdx.y * AM_BW + threadIdx.x;
    for (int i = tid; i < SW * SH; i += AM_BW * AM_BH) {
        const int sy = i / SW, sx = i - sy * SW;
        const int y = clampi(y0 - r + sy, a.y_lo, a.y_hi), x = clampi(x0 - r + sx, 0, a.W - 1);
        am_smem[i] = Dt<DT>::key(ldg_elem<E>(src, a.pitch, y, x));
    }
    __syncthreads();
    const int x = x0 + threadIdx.x, y = y0 + threadIdx.y;
    if (x >= a.W || y >= a.H) return;
    const char *dst = a.dst + (size_t)z * a.plane;
    const uint32_t v = Dt<DT>::key(reinterpret_cast<const E *>(dst + (size_t)y * a.pitch)[x]);
    const int m = (k * k - 1) / 2;
    // one pass: keys below v, keys equal to v and the last equal slot --
    // branch-free, so the unrolled row is straight-line code
    int below = 0, eq = 0, last = -1;
#pragma unroll 1
    for (int dy = 0; dy < k; dy++) {
        const uint32_t *row = am_smem + (threadIdx.y + dy) * SW + threadIdx.x;
#pragma unroll
        for (int dx = 0; dx < k; dx++) {
            const uint32_t e = row[dx];
            const bool same = e == v;
            below += e < v;
            eq += same;
            last = same ? dy * k + dx : last;
        }
    }
    const int j = m - below;  // 0 <= j < eq when v is the window's median
    int slot = j == eq - 1 ? last : -1;
    if (slot < 0 && j >= 0 && j < eq) {  // ties after the median's own slot: find the j-th equal key
        int seen = 0;
        for (int dy = 0; dy < k && slot < 0; dy++) {
            const uint32_t *row = am_smem + (threadIdx.y + dy) * SW + threadIdx.x;
            for (int dx = 0; dx < k; dx++) {
                if (row[dx] == v) {
                    if (seen == j) { slot = dy * k + dx; break; }
                    seen++;
                }
            }
        }
    }
    const int sy = clampi(y - r + slot / k, a.y_lo, a.y_hi);
    const int sx = clampi(x - r + slot % k, 0, a.W - 1);
    char *idx = reinterpret_cast<char *>(a.idx) + (size_t)z * a.idx_plane;
    reinterpret_cast<int32_t *>(idx + (size_t)y * a.idx_pitch)[x] = slot < 0 ? -1 : sy * a.W + sx;
}

// ------------------------------------------------------------- hash lookup
// When the median value occurs in the window at one source pixel only (every
// copy of it clamps to that pixel), that pixel is the argmedian whatever the
// tie rule.  A block of AM_BW x AM_BH pixels stages its footprint, then puts
// every footprint element into a shared-memory hash table keyed by its order
// key, holding the source pixel (ys * W + xs) -- or a mark when the key
// occurs at two different source pixels of the footprint.  A pixel then
// looks its median key up: one probe sequence instead of k^2 compares.  Keys
// that occur at several source pixels (ties, and every value of 8/16-bit
// data) take the full window pass, so the tie rule is unchanged.
constexpr int AMH_MAX_SLOTS = 16384;  // 128 KB of slots

__device__ __forceinline__ unsigned am_hash(uint32_t key, int bits) { return (key * 0x9E3779B1u) >> (32 - bits); }

template <int DT>
__global__ void __launch_bounds__(AM_BW *AM_BH) argmedian_hash_kernel(ImgArgs a, int k, int bits) {
    extern __shared__ __align__(16) unsigned long long amh_smem[];
    typedef typename Dt<DT>::E E;
    const int r = (k - 1) / 2;
    const int SW = AM_BW + k - 1, SH = AM_BH + k - 1;
    const int NS = 1 << bits;
    unsigned long long *ht = amh_smem;                                 // NS slots: (source + 1) << 32 | key, 0 = empty
    uint32_t *foot = reinterpret_cast<uint32_t *>(amh_smem + NS);      // SH x SW keys
    const int x0 = blockIdx.x * AM_BW, y0 = blockIdx.y * AM_BH, z = blockIdx.z;
    const char *src = a.src + (size_t)z * a.plane;
    const int tid = threadIdx.y * AM_BW + threadIdx.x, NT = AM_BW * AM_BH;
    for (int i = tid; i < NS; i += NT) ht[i] = 0ull;
    __syncthreads();
    // one warp a footprint row at a time: load, key, keep for the window
    // pass, and enter into the table (no index division)
    const unsigned long long DUP = 0xffffffff00000000ull;
    for (int sy = threadIdx.y; sy < SH; sy += AM_BH) {
        const int y = clampi(y0 - r + sy, a.y_lo, a.y_hi);
        const E *row = reinterpret_cast<const E *>(src + (ptrdiff_t)y * (ptrdiff_t)a.pitch);
        for (int sx = threadIdx.x; sx < SW; sx += AM_BW) {
            const int x = clampi(x0 - r + sx, 0, a.W - 1);
            const uint32_t key = Dt<DT>::key(__ldg(row + x));
            foot[sy * SW + sx] = key;
            const uint32_t srcpix = (uint32_t)(y * a.W + x);
            const unsigned long long mine = ((unsigned long long)(srcpix + 1) << 32) | key;
            unsigned h = am_hash(key, bits);
            for (int probe = 0; probe < NS; probe++) {  // the table is at most half full: ends early
                unsigned long long cur = ht[h];
                if (cur == 0ull) {
                    cur = atomicCAS(&ht[h], 0ull, mine);
                    if (cur == 0ull) break;  // inserted
                }
                if ((uint32_t)cur == key) {  // same key: same source pixel, or a duplicate
                    if ((cur >> 32) != (unsigned long long)(srcpix + 1) && (cur & DUP) != DUP) atomicOr(&ht[h], DUP);
                    break;
                }
                h = (h + 1) & (unsigned)(NS - 1);
            }
        }
    }
    __syncthreads();
    const int x = x0 + threadIdx.x, y = y0 + threadIdx.y;
    if (x >= a.W || y >= a.H) return;
    const char *dst = a.dst + (size_t)z * a.plane;
    const uint32_t v = Dt<DT>::key(reinterpret_cast<const E *>(dst + (size_t)y * a.pitch)[x]);
    int result = -1;
    bool scan = true;
    unsigned h = am_hash(v, bits);
    for (int probe = 0; probe < NS; probe++) {
        const unsigned long long cur = ht[h];
        if (cur == 0ull) break;  // not in the footprint: cannot happen for a median; scan
        if ((uint32_t)cur == v) {
            if ((cur & DUP) != DUP) {
                result = (int)((cur >> 32) - 1);
                scan = false;
            }
            break;
        }
        h = (h + 1) & (unsigned)(NS - 1);
    }
    if (scan) {  // the key occurs at several source pixels: rank it under (key, slot) order
        const int m = (k * k - 1) / 2;
        int below = 0;
        for (int dy = 0; dy < k; dy++)
            for (int dx = 0; dx < k; dx++) below += foot[(threadIdx.y + dy) * SW + threadIdx.x + dx] < v;
        const int j = m - below;
        int seen = 0, slot = -1;
        for (int dy = 0; dy < k && slot < 0; dy++)
            for (int dx = 0; dx < k; dx++)
                if (foot[(threadIdx.y + dy) * SW + threadIdx.x + dx] == v) {
                    if (seen == j) { slot = dy * k + dx; break; }
                    seen++;
                }
        if (slot >= 0)
            result = clampi(y - r + slot / k, a.y_lo, a.y_hi) * a.W + clampi(x - r + slot % k, 0, a.W - 1);
    }
    char *idx = reinterpret_cast<char *>(a.idx) + (size_t)z * a.idx_plane;
    reinterpret_cast<int32_t *>(idx + (size_t)y * a.idx_pitch)[x] = result;
}

template <int DT>
static void (*pick_k(int k))(ImgArgs, int) {
    switch (k) {  // the k of the data-oblivious range, where the value kernel is fast
        case 3: return argmedian_kernel<DT, 3>;
        case 5: return argmedian_kernel<DT, 5>;
        case 7: return argmedian_kernel<DT, 7>;
        case 9: return argmedian_kernel<DT, 9>;
        case 11: return argmedian_kernel<DT, 11>;
        case 13: return argmedian_kernel<DT, 13>;
        case 15: return argmedian_kernel<DT, 15>;
        case 17: return argmedian_kernel<DT, 17>;
        case 19: return argmedian_kernel<DT, 19>;
        case 21: return argmedian_kernel<DT, 21>;
        case 23: return argmedian_kernel<DT, 23>;
        case 25: return argmedian_kernel<DT, 25>;
        case 27: return argmedian_kernel<DT, 27>;
        default: return argmedian_kernel<DT, 0>;
    }
}

// 32-bit data takes this pass at every k; 8/16-bit data only above the
// record-carrying networks (k >= 27), where the run-time-k form serves
static void (*pick_argmedian(int dtype, int k))(ImgArgs, int) {
    return dtype == MF_U8 ? argmedian_kernel<MF_U8, 0>
           : dtype == MF_U16 ? argmedian_kernel<MF_U16, 0>
           : dtype == MF_U32 ? pick_k<MF_U32>(k)
                             : pick_k<MF_F32>(k);
}

// 32-bit data from this k on take the hash lookup (8/16-bit data repeat
// values in every window and keep the window pass).
static const int AM_HASH_FROM = getenv("MF_AM_HASH_FROM") ? atoi(getenv("MF_AM_HASH_FROM")) : 7;

static int launch_argmedian_hash(const ImgArgs &a, int channels, int k, int dtype, cudaStream_t s) {
    const int n = (AM_BW + k - 1) * (AM_BH + k - 1);
    int bits = 1;
    while ((1 << bits) < 2 * n) bits++;  // at most half full
    if ((1 << bits) > AMH_MAX_SLOTS) bits--;
    if ((1 << bits) < n + n / 4) return MF_ERR_UNSUPPORTED;  // the caller falls back to the window pass
    const size_t smem = (size_t)(1 << bits) * 8 + (size_t)n * 4;
    void (*kern)(ImgArgs, int, int) = dtype == MF_U32 ? argmedian_hash_kernel<MF_U32> : argmedian_hash_kernel<MF_F32>;
    if (smem > 48 * 1024 &&
        cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess) {
        set_error("argmedian smem: %s", cudaGetErrorString(cudaGetLastError()));
        return MF_ERR_CUDA;
    }
    dim3 grid((a.W + AM_BW - 1) / AM_BW, (a.H + AM_BH - 1) / AM_BH, channels);
    kern<<<grid, dim3(AM_BW, AM_BH), smem, s>>>(a, k, bits);
    count_launch();
    cudaError_t e = cudaPeekAtLastError();
    if (e != cudaSuccess) {
        set_error("argmedian kernel: %s", cudaGetErrorString(e));
        return MF_ERR_CUDA;
    }
    return MF_OK;
}

// a.dst must already hold the medians of a.src.
int launch_argmedian_from_values(const ImgArgs &a, int channels, int k, int dtype, cudaStream_t s) {
    if ((dtype == MF_U32 || dtype == MF_F32) && AM_HASH_FROM > 0 && k >= AM_HASH_FROM) {
        const int rc = launch_argmedian_hash(a, channels, k, dtype, s);
        if (rc != MF_ERR_UNSUPPORTED) return rc;
    }
    const size_t smem = (size_t)(AM_BW + k - 1) * (AM_BH + k - 1) * 4;
    dim3 grid((a.W + AM_BW - 1) / AM_BW, (a.H + AM_BH - 1) / AM_BH, channels);
    dim3 block(AM_BW, AM_BH);
    void (*kern)(ImgArgs, int) = pick_argmedian(dtype, k);
    if (smem > 48 * 1024 &&
        cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess) {
        set_error("argmedian smem: %s", cudaGetErrorString(cudaGetLastError()));
        return MF_ERR_CUDA;
    }
    kern<<<grid, block, smem, s>>>(a, k);
    count_launch();
    cudaError_t e = cudaPeekAtLastError();
    if (e != cudaSuccess) {
        set_error("argmedian kernel: %s", cudaGetErrorString(e));
        return MF_ERR_CUDA;
    }
    return MF_OK;
}

}  // namespace mf
