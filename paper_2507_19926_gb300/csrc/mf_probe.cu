// Min/max throughput microbenchmark: the denominator of the data-oblivious
// kernels' ALU roofline.  Every thread runs 16 dependent-pair chains of the
// requested instruction form over register data (no memory traffic inside
// the loop), on 4 x SM-count blocks of 256 threads.
#include <cuda_fp16.h>

#include "mf_registry.h"

namespace mf {

template <int KIND>
__device__ __forceinline__ uint32_t pmin(uint32_t a, uint32_t b) {
    uint32_t d;
    if (KIND == 0) asm("min.u32 %0, %1, %2;" : "=r"(d) : "r"(a), "r"(b));
    if (KIND == 1) asm("min.u16x2 %0, %1, %2;" : "=r"(d) : "r"(a), "r"(b));
    if (KIND == 2) d = __float_as_uint(fminf(__uint_as_float(a), __uint_as_float(b)));
    if (KIND == 3) asm("min.f16x2 %0, %1, %2;" : "=r"(d) : "r"(a), "r"(b));
    if (KIND == 4) asm("min.u16x2 %0, %1, %2;" : "=r"(d) : "r"(a), "r"(b));
    if (KIND == 5) asm("min.u32 %0, %1, %2;" : "=r"(d) : "r"(a), "r"(b));
    if (KIND == 8) d = __vminu4(a, b);                        // four 8-bit lanes
    if (KIND == 9) d = __shfl_sync(0xffffffffu, a, b & 31u);  // register exchange across lanes
    if (KIND == 10) d = __byte_perm(a, b, 0x5140);            // byte permute (lane packing)
    return d;
}
template <int KIND>
__device__ __forceinline__ uint32_t pmax(uint32_t a, uint32_t b) {
    uint32_t d;
    if (KIND == 0) asm("max.u32 %0, %1, %2;" : "=r"(d) : "r"(a), "r"(b));
    if (KIND == 1) asm("max.u16x2 %0, %1, %2;" : "=r"(d) : "r"(a), "r"(b));
    if (KIND == 2) d = __float_as_uint(fmaxf(__uint_as_float(a), __uint_as_float(b)));
    if (KIND == 3) asm("max.f16x2 %0, %1, %2;" : "=r"(d) : "r"(a), "r"(b));
    if (KIND == 4) asm("max.f16x2 %0, %1, %2;" : "=r"(d) : "r"(a), "r"(b));
    if (KIND == 5) d = __float_as_uint(fmaxf(__uint_as_float(a), __uint_as_float(b)));
    if (KIND == 8) d = __vmaxu4(a, b);
    if (KIND == 9) d = __shfl_xor_sync(0xffffffffu, a ^ b, 1);
    if (KIND == 10) d = __byte_perm(a, b, 0x7362);
    return d;
}

// three-input forms: one instruction each where the hardware has them
template <int KIND>
__device__ __forceinline__ uint32_t pmin3(uint32_t a, uint32_t b, uint32_t c) {
    if (KIND == 6) return __vimin3_u16x2(a, b, c);
    return __vimin3_u32(a, b, c);
}
template <int KIND>
__device__ __forceinline__ uint32_t pmax3(uint32_t a, uint32_t b, uint32_t c) {
    if (KIND == 6) return __vimax3_u16x2(a, b, c);
    return __vimax3_u32(a, b, c);
}

template <int KIND>
__global__ void __launch_bounds__(256) probe3_kernel(const uint32_t *in, uint32_t *out, int iters) {
    uint32_t a[8], b[8];
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
#pragma unroll
    for (int i = 0; i < 8; i++) {
        a[i] = in[(t * 16 + i) & 1023];
        b[i] = in[(t * 16 + 8 + i) & 1023];
    }
    for (int it = 0; it < iters; it++) {
#pragma unroll
        for (int i = 0; i < 8; i++) {
            a[i] = pmin3<KIND>(a[i], b[i], a[(i + 3) & 7]);
            b[i] = pmax3<KIND>(b[i], a[(i + 1) & 7], b[(i + 5) & 7]);
        }
    }
    uint32_t acc = 0;
#pragma unroll
    for (int i = 0; i < 8; i++) acc ^= a[i] ^ b[i];
    out[t] = acc;
}

template <int KIND>
__global__ void __launch_bounds__(256) probe_kernel(const uint32_t *in, uint32_t *out, int iters) {
    uint32_t a[8], b[8];
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
#pragma unroll
    for (int i = 0; i < 8; i++) {
        a[i] = in[(t * 16 + i) & 1023];
        b[i] = in[(t * 16 + 8 + i) & 1023];
    }
    for (int it = 0; it < iters; it++) {
#pragma unroll
        for (int i = 0; i < 8; i++) {
            a[i] = pmin<KIND>(a[i], b[i]);
            b[i] = pmax<KIND>(b[i], a[(i + 1) & 7]);
        }
    }
    uint32_t acc = 0;
#pragma unroll
    for (int i = 0; i < 8; i++) acc ^= a[i] ^ b[i];
    out[t] = acc;
}

}  // namespace mf

using namespace mf;

// kind: 0 u32 min/max, 1 u16x2 min/max, 2 f32 min/max, 3 f16x2 min/max,
// 4 u16x2 min interleaved with f16x2 max, 5 u32 min interleaved with f32 max,
// 6 three-input u16x2 min/max, 7 three-input u32 min/max, 8 four-lane u8
// min/max (__vminu4/__vmaxu4), 9 warp shuffles (an index and an xor
// shuffle a pair; the xor one carries one extra logic op), 10 byte
// permutes.  Writes operations per second (per warp-lane operation: one
// call of the min/max, shuffle or permute) and the elapsed milliseconds;
// buffers are allocated and freed here.
extern "C" int mf_probe_minmax(int kind, int iters, double *instr_per_s, double *ms_out) {
    if (kind < 0 || kind > 10 || iters < 1 || !instr_per_s) { set_error("bad probe arguments"); return MF_ERR_ARG; }
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int blocks = 4 * sms, threads = 256;
    uint32_t *in = nullptr, *out = nullptr;
    if (cudaMalloc(&in, 1024 * 4) != cudaSuccess || cudaMalloc(&out, (size_t)blocks * threads * 4) != cudaSuccess) {
        cudaGetLastError();
        if (in) cudaFree(in);
        set_error("probe allocation failed");
        return MF_ERR_ALLOC;
    }
    cudaMemset(in, 0x5a, 1024 * 4);
    void (*kern)(const uint32_t *, uint32_t *, int) =
        kind == 0 ? probe_kernel<0> : kind == 1 ? probe_kernel<1> : kind == 2 ? probe_kernel<2>
        : kind == 3 ? probe_kernel<3> : kind == 4 ? probe_kernel<4> : kind == 5 ? probe_kernel<5>
        : kind == 6 ? probe3_kernel<6> : kind == 7 ? probe3_kernel<7> : kind == 8 ? probe_kernel<8>
        : kind == 9 ? probe_kernel<9> : probe_kernel<10>;
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    kern<<<blocks, threads>>>(in, out, iters);  // warm-up
    count_launch();
    float best = 1e30f;
    for (int rep = 0; rep < 3; rep++) {
        cudaEventRecord(e0);
        kern<<<blocks, threads>>>(in, out, iters);
        count_launch();
        cudaEventRecord(e1);
        cudaEventSynchronize(e1);
        float ms;
        cudaEventElapsedTime(&ms, e0, e1);
        if (ms < best) best = ms;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaFree(in);
    cudaFree(out);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) { set_error("probe: %s", cudaGetErrorString(e)); return MF_ERR_CUDA; }
    *instr_per_s = (double)blocks * threads * iters * 16.0 / (best * 1e-3);
    if (ms_out) *ms_out = best;
    return MF_OK;
}
