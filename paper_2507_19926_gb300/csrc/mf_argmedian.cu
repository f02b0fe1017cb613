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

// a.dst must already hold the medians of a.src.
int launch_argmedian_from_values(const ImgArgs &a, int channels, int k, int dtype, cudaStream_t s) {
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
