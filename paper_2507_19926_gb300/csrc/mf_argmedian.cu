// Argmedian from a computed median.
//
// Under the order (key, row-major window slot) the rank-m element of a
// window (m = (k*k-1)/2) has the median key v, and it is the j-th element
// with key v in slot order, j = m - #{window keys < v} (0-based): all
// elements below v precede it, and equal keys order by slot.  Given the
// median value (from any of the value kernels), one pass over the window
// finds that element: count the keys below v and remember the slots of the
// first equal keys; a second pass is only needed when more than NCAND keys
// tie with the median before the j-th one.  The window is read from a
// shared-memory tile of the block's footprint (clamp-to-edge).
#include "mf_registry.h"

namespace mf {

constexpr int AM_BW = 32, AM_BH = 8, AM_NCAND = 4;

template <int DT>
__global__ void __launch_bounds__(AM_BW *AM_BH) argmedian_kernel(ImgArgs a, int k) {
    extern __shared__ __align__(16) uint32_t am_smem[];
    typedef typename Dt<DT>::E E;
    const int r = (k - 1) / 2;
    const int SW = AM_BW + k - 1, SH = AM_BH + k - 1;
    const int x0 = blockIdx.x * AM_BW, y0 = blockIdx.y * AM_BH, z = blockIdx.z;
    const char *src = a.src + (size_t)z * a.plane;
    const int tid = threadIdx.y * AM_BW + threadIdx.x;
    for (int i = tid; i < SW * SH; i += AM_BW * AM_BH) {
        const int sy = i / SW, sx = i - sy * SW;
        const int y = clampi(y0 - r + sy, 0, a.H - 1), x = clampi(x0 - r + sx, 0, a.W - 1);
        am_smem[i] = Dt<DT>::key(ldg_elem<E>(src, a.pitch, y, x));
    }
    __syncthreads();
    const int x = x0 + threadIdx.x, y = y0 + threadIdx.y;
    if (x >= a.W || y >= a.H) return;
    const char *dst = a.dst + (size_t)z * a.plane;
    const uint32_t v = Dt<DT>::key(reinterpret_cast<const E *>(dst + (size_t)y * a.pitch)[x]);
    const int m = (k * k - 1) / 2;
    int below = 0, eq = 0;
    int cand[AM_NCAND];
#pragma unroll
    for (int c = 0; c < AM_NCAND; c++) cand[c] = 0;
    for (int dy = 0; dy < k; dy++) {
        const uint32_t *row = am_smem + (threadIdx.y + dy) * SW + threadIdx.x;
        for (int dx = 0; dx < k; dx++) {
            const uint32_t e = row[dx];
            below += e < v;
            if (e == v) {
#pragma unroll
                for (int c = 0; c < AM_NCAND; c++)
                    if (c == eq) cand[c] = dy * k + dx;
                eq++;
            }
        }
    }
    const int j = m - below;  // 0 <= j < eq when v is the window's median
    int slot = -1;
#pragma unroll
    for (int c = 0; c < AM_NCAND; c++)
        if (c == j) slot = cand[c];
    if (j >= AM_NCAND) {  // many ties: find the j-th equal key in a second pass
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
    const int sy = clampi(y - r + slot / k, 0, a.H - 1);
    const int sx = clampi(x - r + slot % k, 0, a.W - 1);
    char *idx = reinterpret_cast<char *>(a.idx) + (size_t)z * a.idx_plane;
    reinterpret_cast<int32_t *>(idx + (size_t)y * a.idx_pitch)[x] = slot < 0 ? -1 : sy * a.W + sx;
}

// a.dst must already hold the medians of a.src.
int launch_argmedian_from_values(const ImgArgs &a, int channels, int k, int dtype, cudaStream_t s) {
    const size_t smem = (size_t)(AM_BW + k - 1) * (AM_BH + k - 1) * 4;
    dim3 grid((a.W + AM_BW - 1) / AM_BW, (a.H + AM_BH - 1) / AM_BH, channels);
    dim3 block(AM_BW, AM_BH);
    void (*kern)(ImgArgs, int) = dtype == MF_U8 ? argmedian_kernel<MF_U8>
                                 : dtype == MF_U16 ? argmedian_kernel<MF_U16>
                                 : dtype == MF_U32 ? argmedian_kernel<MF_U32>
                                                   : argmedian_kernel<MF_F32>;
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
