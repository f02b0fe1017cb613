// Batched filter that allocates nothing.
//
// Some callers cannot allocate device memory at the moment they want to
// filter: code that runs while an allocator-owning framework holds the
// device (a foreign cudaMalloc would compete with its pool), latency-bound
// loops that must never stall inside the allocator, or builds whose device
// memory budget is fixed up front.  mf_batch_run_static serves them: the only
// global memory it uses beyond the caller's images is one fixed array that
// lives in this library's module for as long as the library is loaded.
//
// The array holds, in order: one queue counter per kernel class (cleared on
// every call), the image table, the per-image work records, and the
// expanded work items that the persistent kernels of the batched path
// (mf_batch.cu) consume.  A __device__ array has one instance per device;
// every call on a device reuses that device's instance, so calls whose work
// overlaps on the same device race; calls on one stream are ordered and safe.
//
// The tables are copied from the caller's stack with cudaMemcpyAsync, so a
// call made while its stream is being captured into a CUDA graph is
// rejected: the graph would keep the stack addresses and read dead memory on
// every replay.
#include <cstring>
#include <mutex>

#include "mf_registry.h"
#include "mf_tune.h"

namespace mf {

constexpr size_t kStaticScratchBytes = 2u << 20;  // 2 MiB
constexpr int kStaticMaxImages = 256;
constexpr int kStaticMaxClasses = 64;
constexpr size_t kOffImgs = 256;                   // after the counters
constexpr size_t kOffRecs = kOffImgs + (size_t)kStaticMaxImages * sizeof(ImgArgs);
constexpr size_t kOffItems = (kOffRecs + (size_t)kStaticMaxImages * sizeof(int4) * 2 + 255) & ~(size_t)255;
constexpr int kStaticMaxItems = (int)((kStaticScratchBytes - kOffItems) / sizeof(int4));
// The header documents these limits by number; keep the two in step.
static_assert(sizeof(ImgArgs) == 72, "image table layout changed: update the documented item limit");
static_assert(kStaticMaxItems == 129392, "the documented work-item limit of mf_batch_run_static is 129,392");

static __device__ __align__(256) unsigned char g_static_scratch[kStaticScratchBytes];

// Host-side device address of g_static_scratch, looked up once per device
// (the symbol name itself is only a host stand-in for the device array).
static std::mutex g_static_mu;
static unsigned char *g_static_ptr[64] = {};

static int static_scratch(unsigned char **out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) {
        set_error("no CUDA device: %s", cudaGetErrorString(e));
        return MF_ERR_CUDA;
    }
    if (dev < 0 || dev >= 64) {
        set_error("device %d out of range", dev);
        return MF_ERR_ARG;
    }
    std::lock_guard<std::mutex> lk(g_static_mu);
    if (!g_static_ptr[dev]) {
        void *p = nullptr;
        e = cudaGetSymbolAddress(&p, g_static_scratch);
        if (e != cudaSuccess || !p) {
            set_error("cannot resolve the static scratch on device %d: %s", dev, cudaGetErrorString(e));
            return MF_ERR_CUDA;
        }
        g_static_ptr[dev] = (unsigned char *)p;
    }
    *out = g_static_ptr[dev];
    return MF_OK;
}

// Per-image record: (image index, blocks across, blocks down, first item),
// and (planes, class-local item base, -, -).  One thread per work item
// finds its image by binary search over the first-item column.
__global__ void static_expand_kernel(const int4 *recs, int n_recs, int n_items, int4 *items) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n_items) return;
    int lo = 0, hi = n_recs - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (recs[2 * mid].w <= i) lo = mid;
        else hi = mid - 1;
    }
    const int4 r = recs[2 * lo];
    const int local = i - r.w;
    const int per_plane = r.y * r.z;
    const int z = local / per_plane, rem = local - z * per_plane;
    items[i] = make_int4(r.x, rem % r.y, rem / r.y, z);
}

static int esz(int dtype) {
    return dtype == MF_U8 ? 1 : dtype == MF_U16 ? 2 : (dtype == MF_U32 || dtype == MF_F32) ? 4 : 0;
}

}  // namespace mf

using namespace mf;

extern "C" int mf_batch_run_static(const mf_image_desc *descs, int n, mf_stream_t stream) {
    if (!descs || n < 1) { set_error("empty batch"); return MF_ERR_ARG; }
    if (n > kStaticMaxImages) {
        set_error("static batch holds at most %d images (got %d)", kStaticMaxImages, n);
        return MF_ERR_ARG;
    }
    // validation and class assignment (data-oblivious classes only: the
    // data-aware kernels read plan tables the library allocates)
    const O1Entry *cls[kStaticMaxClasses];
    int n_cls = 0;
    int img_cls[kStaticMaxImages];
    for (int i = 0; i < n; i++) {
        const mf_image_desc &d = descs[i];
        const int es = esz(d.dtype);
        if (!es) { set_error("image %d: unknown dtype", i); return MF_ERR_DTYPE; }
        if (d.H < 1 || d.W < 1 || d.channels < 1 || d.channels > 65535 || !d.src || !d.dst) {
            set_error("image %d: bad shape or pointer", i);
            return MF_ERR_ARG;
        }
        if (d.pitch < (size_t)d.W * es || d.pitch % es) { set_error("image %d: bad pitch", i); return MF_ERR_PITCH; }
        const size_t bytes = (size_t)d.channels * d.H * d.pitch;
        const char *a = (const char *)d.src, *b = (const char *)d.dst;
        if (a < b + bytes && b < a + bytes) { set_error("image %d: src and dst overlap", i); return MF_ERR_ALIAS; }
        img_cls[i] = -1;
        if (d.k == 1) continue;
        const O1Entry *o1 =
            (d.k >= 3 && (d.k & 1)) ? find_o1(d.k, d.dtype, false, size_bucket((long long)d.H * d.W)) : nullptr;
        if (o1) {  // wide forms need 16-byte aligned rows
            ImgArgs t{};
            t.src = (const char *)d.src;
            t.dst = (char *)d.dst;
            t.pitch = d.pitch;
            o1 = o1_for_image(o1, t);
        }
        if (!o1 || !o1->persist) {
            set_error("image %d: the static batch runs only the data-oblivious kernels, not built for k = %d "
                      "with this dtype", i, d.k);
            return MF_ERR_UNSUPPORTED;
        }
        int c = 0;
        while (c < n_cls && cls[c] != o1) c++;
        if (c == n_cls) {
            if (n_cls == kStaticMaxClasses) { set_error("too many kernel classes"); return MF_ERR_ARG; }
            cls[n_cls++] = o1;
        }
        img_cls[i] = c;
    }
    // work records, class by class
    ImgArgs args[kStaticMaxImages];
    int4 recs[2 * kStaticMaxImages];
    int n_recs = 0, n_items = 0;
    int cls_first[kStaticMaxClasses + 1];
    for (int c = 0; c < n_cls; c++) {
        cls_first[c] = n_items;
        const O1Entry *o1 = cls[c];
        for (int i = 0; i < n; i++) {
            if (img_cls[i] != c) continue;
            const mf_image_desc &d = descs[i];
            const int lanes = o1->lanes;
            const int rw = lanes * o1->bx * o1->tw * o1->run, rh = o1->by * o1->th;
            const int gx = (d.W + rw - 1) / rw, gy = (d.H + rh - 1) / rh;
            const long long cnt = (long long)gx * gy * d.channels;
            if (n_items + cnt > kStaticMaxItems) {
                set_error("static batch needs more than %d work items (%zu bytes of scratch)", kStaticMaxItems,
                          kStaticScratchBytes);
                return MF_ERR_ARG;
            }
            recs[2 * n_recs] = make_int4(i, gx, gy, n_items);
            recs[2 * n_recs + 1] = make_int4(d.channels, 0, 0, 0);
            n_recs++;
            n_items += (int)cnt;
        }
    }
    cls_first[n_cls] = n_items;
    for (int i = 0; i < n; i++) {
        const mf_image_desc &d = descs[i];
        ImgArgs &a = args[i];
        a.src = (const char *)d.src;
        a.dst = (char *)d.dst;
        a.idx = nullptr;
        a.H = d.H;
        a.y_lo = 0;
        a.y_hi = d.H - 1;
        a.W = d.W;
        a.pitch = d.pitch;
        a.plane = (size_t)d.H * d.pitch;
        a.idx_pitch = a.idx_plane = 0;
    }

    cudaStream_t s = (cudaStream_t)stream;
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    cudaError_t e = cudaStreamIsCapturing(s, &cap);
    if (e != cudaSuccess) {
        set_error("static batch: cannot query the stream: %s", cudaGetErrorString(e));
        return MF_ERR_CUDA;
    }
    if (cap != cudaStreamCaptureStatusNone) {
        set_error("static batch: the stream is being captured; this call copies its tables from the stack "
                  "and must not be captured into a graph");
        return MF_ERR_UNSUPPORTED;
    }
    unsigned char *base = nullptr;
    int rc = static_scratch(&base);
    if (rc) return rc;
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
        set_error("device attribute: %s", cudaGetErrorString(cudaGetLastError()));
        return MF_ERR_CUDA;
    }
    // tables from the stack (pageable: the copies have consumed them when
    // the calls return), counters cleared on every call
    e = cudaMemcpyAsync(base + kOffImgs, args, n * sizeof(ImgArgs), cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess && n_recs)
        e = cudaMemcpyAsync(base + kOffRecs, recs, 2 * n_recs * sizeof(int4), cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(base, 0, kOffImgs, s);
    if (e != cudaSuccess) { set_error("static batch upload: %s", cudaGetErrorString(e)); return MF_ERR_CUDA; }
    int4 *items = (int4 *)(base + kOffItems);
    if (n_items) {
        static_expand_kernel<<<(n_items + 255) / 256, 256, 0, s>>>((const int4 *)(base + kOffRecs), n_recs, n_items,
                                                                   items);
        count_launch();
    }
    for (int c = 0; c < n_cls; c++) {
        int bps = 0, grid = 0;
        rc = cls[c]->persist(nullptr, nullptr, 0, nullptr, 0, sms, nullptr, &bps);
        if (rc == MF_OK)
            rc = cls[c]->persist((const ImgArgs *)(base + kOffImgs), items + cls_first[c], cls_first[c + 1] - cls_first[c],
                                 (unsigned *)base + c, bps, sms, s, &grid);
        if (rc != MF_OK) {
            set_error("static batch, k=%d: %s", cls[c]->k, cudaGetErrorString(cudaGetLastError()));
            return rc;
        }
        count_launch();
    }
    for (int i = 0; i < n; i++) {
        const mf_image_desc &d = descs[i];
        if (d.k != 1) continue;
        e = cudaMemcpy2DAsync(d.dst, d.pitch, d.src, d.pitch, (size_t)d.W * esz(d.dtype), (size_t)d.H * d.channels,
                              cudaMemcpyDeviceToDevice, s);
        if (e != cudaSuccess) { set_error("identity copy: %s", cudaGetErrorString(e)); return MF_ERR_CUDA; }
    }
    e = cudaPeekAtLastError();
    if (e != cudaSuccess) { set_error("static batch: %s", cudaGetErrorString(e)); return MF_ERR_CUDA; }
    return MF_OK;
}
