// Shared device-side definitions of the median-filter kernels (sm_103a).
//
// Order keys: every element is compared through an unsigned key.  u8/u16/u32
// keys are the values; f32 keys are the IEEE bits with the sign bit set for
// non-negative values and all bits inverted for negative ones, so that key
// order is -NaN < -inf < ... < -0 < +0 < ... < +inf < +NaN and equal keys
// are bit-identical values.  Min/max networks on keys therefore select the
// exact input element (paper Sec. 4: networks compile to min/max sequences).
#pragma once
#include <atomic>
#include <cstddef>
#include <cstdint>
#include <cuda_runtime.h>

#include "../../include/medianfilter.h"

namespace mf {

// ----------------------------------------------------------------- key ops
// One 32-bit register holds one u32 key, or two u16 keys (two tiles run the
// same data-oblivious network side by side, paper Sec. 4.3 packing idea:
// the network is independent of the data, so lanes never diverge).
// mn3 / mx3: three-input forms, one instruction on sm_100+ (measured at the
// two-input rate by mf_probe_minmax kinds 6 and 7).
struct KoU32 {
    typedef uint32_t T;
    static constexpr int lanes = 1;
    static __device__ __forceinline__ T mn(T a, T b) { return umin(a, b); }
    static __device__ __forceinline__ T mx(T a, T b) { return umax(a, b); }
    static __device__ __forceinline__ T mn3(T a, T b, T c) { return __vimin3_u32(a, b, c); }
    static __device__ __forceinline__ T mx3(T a, T b, T c) { return __vimax3_u32(a, b, c); }
};

struct KoU16x2 {
    typedef uint32_t T;
    static constexpr int lanes = 2;
    static __device__ __forceinline__ T mn(T a, T b) {
        T d;
        asm("min.u16x2 %0, %1, %2;" : "=r"(d) : "r"(a), "r"(b));
        return d;
    }
    static __device__ __forceinline__ T mx(T a, T b) {
        T d;
        asm("max.u16x2 %0, %1, %2;" : "=r"(d) : "r"(a), "r"(b));
        return d;
    }
    static __device__ __forceinline__ T mn3(T a, T b, T c) { return __vimin3_u16x2(a, b, c); }
    static __device__ __forceinline__ T mx3(T a, T b, T c) { return __vimax3_u16x2(a, b, c); }
};

// 64-bit composite records (key << 32 | position) for argmedian of 32-bit data.
struct KoU64 {
    typedef unsigned long long T;
    static constexpr int lanes = 1;
    static __device__ __forceinline__ T mn(T a, T b) { return a < b ? a : b; }
    static __device__ __forceinline__ T mx(T a, T b) { return a < b ? b : a; }
    static __device__ __forceinline__ T mn3(T a, T b, T c) { return mn(mn(a, b), c); }
    static __device__ __forceinline__ T mx3(T a, T b, T c) { return mx(mx(a, b), c); }
};

// a + s * d for a loop variable s in {0, 1} and d = b - a: the select
// between a and b as one multiply-add (modular arithmetic makes it exact for
// any bit patterns, packed lanes included), issued on the FMA pipe instead
// of the integer pipe the min/max networks saturate.
__device__ __forceinline__ uint32_t mad_sel(unsigned s, uint32_t d, uint32_t a) {
    uint32_t r;
    asm("mad.lo.u32 %0, %1, %2, %3;" : "=r"(r) : "r"(s), "r"(d), "r"(a));
    return r;
}

// ------------------------------------------------------------ dtype traits
__device__ __forceinline__ uint32_t f32_key(uint32_t b) {
    return (b & 0x80000000u) ? ~b : (b | 0x80000000u);
}
__device__ __forceinline__ uint32_t f32_unkey(uint32_t k) {
    return (k & 0x80000000u) ? (k & 0x7fffffffu) : ~k;
}

template <int DT> struct Dt;
template <> struct Dt<MF_U8> {
    typedef uint8_t E;
    static constexpr int bits = 8;
    static __device__ __forceinline__ uint32_t key(E v) { return v; }
    static __device__ __forceinline__ E val(uint32_t k) { return (E)k; }
};
template <> struct Dt<MF_U16> {
    typedef uint16_t E;
    static constexpr int bits = 16;
    static __device__ __forceinline__ uint32_t key(E v) { return v; }
    static __device__ __forceinline__ E val(uint32_t k) { return (E)k; }
};
template <> struct Dt<MF_U32> {
    typedef uint32_t E;
    static constexpr int bits = 32;
    static __device__ __forceinline__ uint32_t key(E v) { return v; }
    static __device__ __forceinline__ E val(uint32_t k) { return k; }
};
template <> struct Dt<MF_F32> {
    typedef uint32_t E;  // raw bits
    static constexpr int bits = 32;
    static __device__ __forceinline__ uint32_t key(E v) { return f32_key(v); }
    static __device__ __forceinline__ E val(uint32_t k) { return f32_unkey(k); }
};

__host__ __device__ __forceinline__ int clampi(int v, int lo, int hi) {
    return v < lo ? lo : (v > hi ? hi : v);
}

template <class E>
__device__ __forceinline__ E ldg_elem(const char *plane, size_t pitch, int y, int x) {
    return __ldg(reinterpret_cast<const E *>(plane + (ptrdiff_t)y * (ptrdiff_t)pitch) + x);  // y may be < 0 in a band
}

// Launch arguments common to all image kernels.  src and dst point at the
// first row to filter; H rows are filtered.  Reads clamp to rows y_lo..y_hi
// relative to src: 0..H-1 for a whole image, wider when the rows are a band
// of a larger image whose neighbouring rows are valid input.
struct ImgArgs {
    const char *src;
    char *dst;
    int32_t *idx;       // argmedian output or nullptr
    int H, W;
    int y_lo, y_hi;     // readable rows for clamp-to-edge, relative to src
    size_t pitch;       // bytes per row, src and dst
    size_t plane;       // bytes per plane = H * pitch
    size_t idx_pitch;   // bytes per row of idx
    size_t idx_plane;   // bytes per plane of idx
};

// Function attributes (cudaFuncSetAttribute) belong to the context of the
// device that is current when they are set, so every kernel instantiation is
// configured once per device: bit d of a DevMask records device d (0..63;
// devices beyond that are configured on every call).
typedef std::atomic<unsigned long long> DevMask;
inline bool dev_configured(const DevMask &m, int *dev) {
    if (cudaGetDevice(dev) != cudaSuccess) {
        cudaGetLastError();
        *dev = -1;
        return false;
    }
    return *dev >= 0 && *dev < 64 && ((m.load(std::memory_order_acquire) >> *dev) & 1ull);
}
inline void dev_mark_configured(DevMask &m, int dev) {
    if (dev >= 0 && dev < 64) m.fetch_or(1ull << dev, std::memory_order_acq_rel);
}

// Kernel launch counter (host side, see mf_kernel_launch_count).
void count_launch(unsigned n = 1);

// Every device allocation of the library goes through here.  Setting the
// environment variable MF_FAULT_INJECT=alloc makes it fail (as an
// out-of-memory device would), so the error paths can be exercised on the
// host without touching the GPU.
cudaError_t dev_alloc(void **p, size_t bytes);

}  // namespace mf
