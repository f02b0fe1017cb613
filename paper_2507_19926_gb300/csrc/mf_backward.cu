// Backward of the median filter.  Between order changes the median is the
// identity on its selected input, so d out[q] / d in[p] = [idx[q] == p] and
// grad_in[p] = sum over q with idx[q] = p of grad_out[q].
//
// Atomic mode: zero grad_in, then one thread per output q adds grad_out[q]
// at idx[q] (float atomics; summation order unspecified).
// Deterministic mode: every p receives its contributions in increasing
// row-major q -- the order, hence the f32 rounding, of a sequential
// row-major scatter -- from an ordered scatter into shared memory (below).
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

// Ordered scatter.  A block owns a 32 x 32 tile of inputs p, each of its 8
// warps 4 rows of it, with one f32 accumulator per p in shared memory.  An
// output q can select p only if p lies in q's window, so a warp visits the
// outputs q of rows (its first row - r) .. (its last row + r) and columns
// (tile start - r) .. (tile end + r), one row after another, 32 columns per
// step (lane = column), and adds grad_out[q] to p = idx[q] when p is one of
// its own.  Rows go in increasing order, columns of a step in lane order, and
// lanes of a step that hit the same p add one after the other in lane order
// (grouped by __match_any_sync), so every p sums its contributions exactly
// in increasing row-major q.  Warps own disjoint sets of p: no order between
// warps matters.  Work per p is ((4 + 2r) x (32 + 2r)) / 128 outputs visited
// instead of the (2r + 1)^2 window a gather would scan.
constexpr int BD_TX = 32, BD_WARPS = 8, BD_RPW = 4;

__global__ void __launch_bounds__(BD_WARPS * 32)
    bwd_ordered_kernel(const float *__restrict__ g, const int32_t *__restrict__ idx, float *__restrict__ gi,
                       int H, int W, size_t pitch, size_t idx_pitch, int r) {
    __shared__ float acc[BD_WARPS * BD_RPW * BD_TX];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int X0 = blockIdx.x * BD_TX;
    const int Yw = blockIdx.y * (BD_WARPS * BD_RPW) + w * BD_RPW;  // the warp's first row of p
    float *wacc = acc + w * BD_RPW * BD_TX;
#pragma unroll
    for (int j = 0; j < BD_RPW; j++) wacc[j * BD_TX + lane] = 0.f;
    __syncwarp();
    if (Yw >= H) return;  // the whole warp: nothing of its own
    const size_t pl = (size_t)H * pitch, ipl = (size_t)H * idx_pitch;
    const char *gp = reinterpret_cast<const char *>(g) + blockIdx.z * pl;
    const char *ip = reinterpret_cast<const char *>(idx) + blockIdx.z * ipl;
    const int HW = H * W;
    const int base = Yw * W + X0;               // p of the warp's first pixel
    const int cw = min(BD_TX, W - X0);          // columns of the tile inside the image
    const int qx_lo = max(0, X0 - r), qx_hi = min(W - 1, X0 + cw - 1 + r);
    const int qy_lo = max(0, Yw - r), qy_hi = min(H - 1, Yw + BD_RPW - 1 + r);
    for (int qy = qy_lo; qy <= qy_hi; qy++) {
        const int32_t *irow = reinterpret_cast<const int32_t *>(ip + (size_t)qy * idx_pitch);
        const float *grow = reinterpret_cast<const float *>(gp + (size_t)qy * pitch);
        for (int qx0 = qx_lo; qx0 <= qx_hi; qx0 += 32) {
            const int qx = qx0 + lane;
            int slot = -1;  // j * BD_TX + column of p in the warp's rows, or -1
            float gv = 0.f;
            if (qx <= qx_hi) {
                const int p = irow[qx];
                if ((unsigned)p < (unsigned)HW) {
                    const int rel = p - base;
#pragma unroll
                    for (int j = 0; j < BD_RPW; j++) {
                        const int c = rel - j * W;
                        if (c >= 0 && c < cw) slot = j * BD_TX + c;
                    }
                    if (slot >= 0) gv = grow[qx];
                }
            }
            // lanes aiming at the same p add in lane order
            const unsigned grp = __match_any_sync(0xffffffffu, slot);
            const int rank = __popc(grp & ((1u << lane) - 1u));
            const int n = __reduce_max_sync(0xffffffffu, slot >= 0 ? __popc(grp) : 0);
            for (int t = 0; t < n; t++) {
                if (slot >= 0 && rank == t) wacc[slot] += gv;
                __syncwarp();
            }
        }
    }
    __syncwarp();
    char *gip = reinterpret_cast<char *>(gi) + blockIdx.z * pl;
    if (lane < cw) {
#pragma unroll
        for (int j = 0; j < BD_RPW; j++)
            if (Yw + j < H) reinterpret_cast<float *>(gip + (size_t)(Yw + j) * pitch)[X0 + lane] = wacc[j * BD_TX + lane];
    }
}

int bwd_ordered(const float *g, const int32_t *idx, float *gi, int H, int W, size_t pitch,
               size_t idx_pitch, int C, int k, cudaStream_t s) {
    const int r = (k - 1) / 2;
    dim3 grid((W + BD_TX - 1) / BD_TX, (H + BD_WARPS * BD_RPW - 1) / (BD_WARPS * BD_RPW), C);
    bwd_ordered_kernel<<<grid, BD_WARPS * 32, 0, s>>>(g, idx, gi, H, W, pitch, idx_pitch, r);
    count_launch();
    cudaError_t e = cudaPeekAtLastError();
    if (e != cudaSuccess) { set_error("ordered scatter: %s", cudaGetErrorString(e)); return MF_ERR_CUDA; }
    return MF_OK;
}

}  // namespace mf
