// Backward of the median filter.  Between order changes the median is the
// identity on its selected input, so d out[q] / d in[p] = [idx[q] == p] and
// grad_in[p] = sum over q with idx[q] = p of grad_out[q].
//
// Atomic mode: zero grad_in, then one thread per output q adds grad_out[q]
// at idx[q] (float atomics; summation order unspecified).
// Deterministic mode: one thread per input p sums grad_out[q] over the
// outputs q of its clamp-aware k x k neighbourhood (the only outputs whose
// window can select p) with idx[q] = p, in increasing row-major q -- the same
// order, hence the same f32 rounding, as a sequential row-major scatter.
#include "mf_registry.h"

namespace mf {

__global__ void bwd_scatter_kernel(const float *__restrict__ g, const int32_t *__restrict__ idx,
                                   float *gi, int H, int W, size_t pitch, size_t idx_pitch) {
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int y = blockIdx.y;
    if (x >= W) return;
    const size_t pl = (size_t)H * pitch, ipl = (size_t)H * idx_pitch;
    const float *gp = reinterpret_cast<const float *>(reinterpret_cast<const char *>(g) + blockIdx.z * pl);
    const int32_t *ip = reinterpret_cast<const int32_t *>(reinterpret_cast<const char *>(idx) + blockIdx.z * ipl);
    char *gip = reinterpret_cast<char *>(gi) + blockIdx.z * pl;
    const float v = reinterpret_cast<const float *>(reinterpret_cast<const char *>(gp) + (size_t)y * pitch)[x];
    const int p = reinterpret_cast<const int32_t *>(reinterpret_cast<const char *>(ip) + (size_t)y * idx_pitch)[x];
    if ((unsigned)p >= (unsigned)(H * W)) return;  // not produced by this library; ignore
    const int py = p / W, px = p - py * W;
    atomicAdd(reinterpret_cast<float *>(gip + (size_t)py * pitch) + px, v);
}

int bwd_atomic(const float *g, const int32_t *idx, float *gi, int H, int W, size_t pitch,
               size_t idx_pitch, int C, cudaStream_t s) {
    cudaError_t e = cudaMemset2DAsync(gi, pitch, 0, (size_t)W * 4, (size_t)H * C, s);
    if (e != cudaSuccess) { set_error("memset: %s", cudaGetErrorString(e)); return MF_ERR_CUDA; }
    dim3 grid((W + 255) / 256, H, C);
    bwd_scatter_kernel<<<grid, 256, 0, s>>>(g, idx, gi, H, W, pitch, idx_pitch);
    count_launch();
    e = cudaPeekAtLastError();
    if (e != cudaSuccess) { set_error("scatter: %s", cudaGetErrorString(e)); return MF_ERR_CUDA; }
    return MF_OK;
}

// Gather: a 32 x 8 block of inputs p stages the idx and grad_out of its
// (32 + 2r) x (8 + 2r) neighbourhood in shared memory, then every thread
// walks its own (2r+1)^2 window of outputs in row-major order.
template <int BW, int BH>
__global__ void bwd_gather_kernel(const float *__restrict__ g, const int32_t *__restrict__ idx,
                                  float *__restrict__ gi, int H, int W, size_t pitch, size_t idx_pitch,
                                  int r) {
    extern __shared__ __align__(16) unsigned char bg_smem[];
    const int SW = BW + 2 * r, SH = BH + 2 * r;
    int32_t *si = reinterpret_cast<int32_t *>(bg_smem);
    float *sg = reinterpret_cast<float *>(si + SW * SH);
    const int x0 = blockIdx.x * BW, y0 = blockIdx.y * BH;
    const size_t pl = (size_t)H * pitch, ipl = (size_t)H * idx_pitch;
    const char *gp = reinterpret_cast<const char *>(g) + blockIdx.z * pl;
    const char *ip = reinterpret_cast<const char *>(idx) + blockIdx.z * ipl;
    const int tid = threadIdx.y * BW + threadIdx.x;
    for (int i = tid; i < SW * SH; i += BW * BH) {
        const int sy = i / SW, sx = i - sy * SW;
        const int y = y0 - r + sy, x = x0 - r + sx;
        int32_t iv = -1;
        float gv = 0.f;
        if (y >= 0 && y < H && x >= 0 && x < W) {
            iv = reinterpret_cast<const int32_t *>(ip + (size_t)y * idx_pitch)[x];
            gv = reinterpret_cast<const float *>(gp + (size_t)y * pitch)[x];
        }
        si[i] = iv;
        sg[i] = gv;
    }
    __syncthreads();
    const int x = x0 + threadIdx.x, y = y0 + threadIdx.y;
    if (x >= W || y >= H) return;
    const int p = y * W + x;
    float acc = 0.f;
    for (int dy = 0; dy <= 2 * r; dy++) {
        const int32_t *rowi = si + (threadIdx.y + dy) * SW + threadIdx.x;
        const float *rowg = sg + (threadIdx.y + dy) * SW + threadIdx.x;
        for (int dx = 0; dx <= 2 * r; dx++)
            if (rowi[dx] == p) acc += rowg[dx];
    }
    reinterpret_cast<float *>(reinterpret_cast<char *>(gi) + blockIdx.z * pl + (size_t)y * pitch)[x] = acc;
}

int bwd_gather(const float *g, const int32_t *idx, float *gi, int H, int W, size_t pitch,
               size_t idx_pitch, int C, int k, cudaStream_t s) {
    const int r = (k - 1) / 2;
    constexpr int BW = 32, BH = 8;
    const size_t smem = (size_t)(BW + 2 * r) * (BH + 2 * r) * 8;
    auto kern = bwd_gather_kernel<BW, BH>;
    if (smem > 48 * 1024) {
        if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess) {
            set_error("gather smem: %s", cudaGetErrorString(cudaGetLastError()));
            return MF_ERR_CUDA;
        }
    }
    dim3 grid((W + BW - 1) / BW, (H + BH - 1) / BH, C);
    kern<<<grid, dim3(BW, BH), smem, s>>>(g, idx, gi, H, W, pitch, idx_pitch, r);
    count_launch();
    cudaError_t e = cudaPeekAtLastError();
    if (e != cudaSuccess) { set_error("gather: %s", cudaGetErrorString(e)); return MF_ERR_CUDA; }
    return MF_OK;
}

}  // namespace mf
