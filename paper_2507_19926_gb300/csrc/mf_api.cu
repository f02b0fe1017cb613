// C ABI of the median filter: argument checks, variant/tile dispatch, the
// host-buffer entry point, error reporting.  The filter itself is defined in
// the paper's introduction (Sec. 1); the kernels live in mf_oblivious.cuh
// (Sec. 4) and mf_data_aware.cu (Sec. 5).
#include <atomic>
#include <cstdint>
#include <cstdarg>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <algorithm>
#include <mutex>
#include <string>
#include <vector>

#include "mf_registry.h"
#include "mf_tune.h"

namespace mf {

static thread_local char g_err[512] = "";
static std::atomic<unsigned long long> g_launches{0};

void set_error(const char *fmt, ...) {
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_err, sizeof g_err, fmt, ap);
    va_end(ap);
}

void count_launch(unsigned n) { g_launches.fetch_add(n, std::memory_order_relaxed); }

cudaError_t dev_alloc(void **p, size_t bytes) {
    const char *f = getenv("MF_FAULT_INJECT");
    if (f && strcmp(f, "alloc") == 0) {
        *p = nullptr;
        return cudaErrorMemoryAllocation;
    }
    return cudaMalloc(p, bytes);
}

// The nth (0-based) instantiated configuration for (k, dtype, arg); the
// first one is the default.
const O1Entry *find_o1_nth(int k, int dtype, bool arg, int nth) {
    for (int i = 0; i < kO1Count; i++)
        if (kO1Entries[i].k == k && kO1Entries[i].dtype == dtype && kO1Entries[i].arg == (arg ? 1 : 0))
            if (nth-- == 0) return &kO1Entries[i];
    return nullptr;
}

const O1Entry *o1_for_image(const O1Entry *e, const ImgArgs &a) {
    if (!e || e->run <= 1 || (((uintptr_t)a.src | (uintptr_t)a.dst | (uintptr_t)a.pitch) & 15) == 0) return e;
    for (int nth = 0;; nth++) {
        const O1Entry *f = find_o1_nth(e->k, e->dtype, e->arg != 0, nth);
        if (!f) return e;  // none: the wide form's own element-by-element path
        if (f->run <= 1) return f;
    }
}

// Untuned default for an image filtered on its own (`alone`) in an
// image-size bucket.  The wide forms (a run of 4 or 2 root tiles a lane)
// are the defaults at k = 3, 5 because they win on large images; a small
// image alone then has too few blocks to fill the GPU (in a batch its
// blocks run beside other images', and the default stays).
// With 16-bit keys (8/16-bit data) buckets below 10 (under 2^20 pixels)
// take the first configuration without a run and bucket 10 (up to 2^22
// pixels) the first with a run of 2, where there is one (measured from a
// CUDA graph of 200 launches: 640 x 480 u8 k = 5 3.64 -> 2.74 us, k = 3
// 2.72 -> 1.90 us; 1920 x 1080 u8 k = 5 8.08 -> 7.16 us, k = 3 4.40 ->
// 3.83 us; 32-bit keys showed no such gain).
static const O1Entry *o1_default(int k, int dtype, bool arg, int bucket, bool alone) {
    const O1Entry *d = find_o1_nth(k, dtype, arg, 0);
    if (!alone || !d || d->run <= 1 || d->lanes != 2 || bucket < 0 || bucket > 10) return d;
    const int want = bucket <= 9 ? 1 : 2;
    for (int nth = 1;; nth++) {
        const O1Entry *f = find_o1_nth(k, dtype, arg, nth);
        if (!f) return d;
        if (f->run == want && f->lanes == 2) return f;
    }
}

const O1Entry *find_o1(int k, int dtype, bool arg, int bucket, bool alone) {
    // a tuning entry (nearest size bucket) names its configuration, the
    // default one included
    const O1Entry *e = tune_lookup(k, dtype, arg, bucket) == MF_OBLIVIOUS
                           ? find_o1_nth(k, dtype, arg, tune_tile(k, dtype, arg, bucket))
                           : nullptr;
    return e ? e : o1_default(k, dtype, arg, bucket, alone);
}

static int esize(int dtype) {
    switch (dtype) {
        case MF_U8: return 1;
        case MF_U16: return 2;
        case MF_U32: return 4;
        case MF_F32: return 4;
        default: return 0;
    }
}

static int cuda_fail(cudaError_t e, const char *what) {
    set_error("%s: %s", what, cudaGetErrorString(e));
    return MF_ERR_CUDA;
}

static bool overlap(const void *a, size_t na, const void *b, size_t nb) {
    const char *pa = (const char *)a, *pb = (const char *)b;
    return pa < pb + nb && pb < pa + na;
}

// Checks shared by the forward entry points.
static int check_fwd(const void *src, const void *dst, int H, int W, size_t pitch, int C, int dtype,
                     int k, int border, const int32_t *idx, size_t idx_pitch) {
    if (esize(dtype) == 0) { set_error("unknown dtype %d", dtype); return MF_ERR_DTYPE; }
    if (k < 1 || k > 75 || (k & 1) == 0) { set_error("k must be odd in 1..75 (got %d)", k); return MF_ERR_ARG; }
    if (H < 1 || W < 1 || C < 1 || C > 65535) { set_error("bad shape H=%d W=%d C=%d", H, W, C); return MF_ERR_ARG; }
    if ((long long)H * W > (1ll << 31) - 1) { set_error("plane too large for int32 indices"); return MF_ERR_ARG; }
    if (border != MF_BORDER_CLAMP) { set_error("only clamp-to-edge borders are supported"); return MF_ERR_ARG; }
    if (!src || (!dst && !idx)) { set_error("null pointer"); return MF_ERR_ARG; }
    const int es = esize(dtype);
    if (pitch < (size_t)W * es || pitch % es) { set_error("bad pitch %zu for W=%d", pitch, W); return MF_ERR_PITCH; }
    if (idx && (idx_pitch < (size_t)W * 4 || idx_pitch % 4)) { set_error("bad idx_pitch %zu", idx_pitch); return MF_ERR_PITCH; }
    const size_t bytes = (size_t)C * H * pitch;
    if (dst && overlap(src, bytes, dst, bytes)) { set_error("src and dst overlap"); return MF_ERR_ALIAS; }
    if (idx && overlap(src, bytes, idx, (size_t)C * H * idx_pitch)) { set_error("src and argidx overlap"); return MF_ERR_ALIAS; }
    if (idx && dst && overlap(dst, bytes, idx, (size_t)C * H * idx_pitch)) { set_error("dst and argidx overlap"); return MF_ERR_ALIAS; }
    return MF_OK;
}

// ----------------------------------------------------------- k = 1 path
__global__ void identity_idx_kernel(int32_t *idx, int H, int W, size_t idx_pitch, size_t idx_plane) {
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int y = blockIdx.y;
    if (x >= W) return;
    int32_t *row = reinterpret_cast<int32_t *>(reinterpret_cast<char *>(idx) + blockIdx.z * idx_plane +
                                               (size_t)y * idx_pitch);
    row[x] = y * W + x;
}

int launch_identity_idx(const ImgArgs &a, int C, cudaStream_t s) {
    dim3 grid((a.W + 255) / 256, a.H, C);
    identity_idx_kernel<<<grid, 256, 0, s>>>(a.idx, a.H, a.W, a.idx_pitch, a.idx_plane);
    count_launch();
    cudaError_t e = cudaPeekAtLastError();
    return e == cudaSuccess ? MF_OK : cuda_fail(e, "identity index kernel");
}

// ----------------------------------------------------------- dispatch
struct Plan {
    int variant;  // MF_OBLIVIOUS or MF_DATA_AWARE (resolved)
    const O1Entry *o1;
    int tile;     // D1 root tile
};

static int resolve(int k, int dtype, bool arg, int variant, Plan *p, int bucket = -1, bool alone = false) {
    p->o1 = nullptr;
    p->tile = 0;
    const O1Entry *o1 = find_o1(k, dtype, arg, bucket, alone);
    const bool d1 = d1_supported(k, dtype, arg) != 0;
    if (variant == MF_AUTO) {
        int tuned = tune_lookup(k, dtype, arg, bucket);
        if (tuned == MF_OBLIVIOUS && o1) variant = MF_OBLIVIOUS;
        else if (tuned == MF_DATA_AWARE && d1) variant = MF_DATA_AWARE;
        else variant = o1 ? MF_OBLIVIOUS : MF_DATA_AWARE;
    }
    if (variant == MF_OBLIVIOUS) {
        if (!o1) { set_error("no data-oblivious kernel for k=%d dtype=%d%s", k, dtype, arg ? " (argmedian)" : ""); return MF_ERR_UNSUPPORTED; }
        p->variant = MF_OBLIVIOUS;
        p->o1 = o1;
        return MF_OK;
    }
    if (variant == MF_DATA_AWARE) {
        if (!d1) { set_error("no data-aware kernel for k=%d dtype=%d%s", k, dtype, arg ? " (argmedian)" : ""); return MF_ERR_UNSUPPORTED; }
        p->variant = MF_DATA_AWARE;
        p->tile = d1_default_tile(k, dtype, arg, 0, bucket);
        return MF_OK;
    }
    set_error("unknown variant %d", variant);
    return MF_ERR_ARG;
}

int resolve_variant(int k, int dtype, bool arg, int variant, const O1Entry **o1, int bucket, int *tile) {
    Plan p;
    int rc = resolve(k, dtype, arg, variant, &p, bucket);
    if (rc) return rc;
    if (o1) *o1 = p.o1;
    if (tile) *tile = p.tile;
    return p.variant;
}

// The value (or record) kernel the variant resolves to, on prepared args.
static int launch_resolved(const ImgArgs &a, int C, int k, int dtype, int variant, cudaStream_t s) {
    Plan p;
    int rc = resolve(k, dtype, a.idx != nullptr, variant, &p, size_bucket((long long)a.H * a.W), true);
    if (rc) return rc;
    if (p.variant == MF_OBLIVIOUS) {
        const O1Entry *e = o1_for_image(p.o1, a);
        rc = e->launch(a, C, s);
        if (rc == MF_ERR_CUDA) set_error("%s: %s", e->name, cudaGetErrorString(cudaGetLastError()));
        return rc;
    }
    return d1_launch(a, C, k, dtype, p.tile, s);
}

static int run_filter(const void *src, void *dst, int H, int W, size_t pitch, int C, int dtype, int k,
                      int variant, int32_t *idx, size_t idx_pitch, cudaStream_t s) {
    ImgArgs a;
    a.src = (const char *)src;
    a.dst = (char *)dst;
    a.idx = idx;
    a.H = H;
    a.y_lo = 0;
    a.y_hi = H - 1;
    a.W = W;
    a.pitch = pitch;
    a.plane = (size_t)H * pitch;
    a.idx_pitch = idx_pitch;
    a.idx_plane = (size_t)H * idx_pitch;
    if (k == 1) {
        if (dst) {
            cudaError_t e = cudaMemcpy2DAsync(dst, pitch, src, pitch, (size_t)W * esize(dtype),
                                              (size_t)H * C, cudaMemcpyDeviceToDevice, s);
            if (e != cudaSuccess) return cuda_fail(e, "identity copy");
        }
        return idx ? launch_identity_idx(a, C, s) : MF_OK;
    }
    // Argmedian where no record-carrying network is instantiated for (k,
    // dtype): compute the medians with the value kernel, then recover each
    // median's source from the window (mf_argmedian.cu).  8/16-bit windows
    // always hold repeated values, so the recovery is a full window pass;
    // from k = 27 (8-bit) and k = 29 (16-bit) the data-aware merges on
    // (key, footprint index) records are faster (16 x 1024^2, u8 k = 45
    // 25.6 -> 12.5 ms, u16 k = 45 19.8 -> 12.7 ms) and MF_AUTO takes them.
    const bool narrow_records = variant == MF_AUTO && (dtype == MF_U8 ? k >= 27 : dtype == MF_U16 ? k >= 29 : false);
    if (idx && dst && variant != MF_DATA_AWARE && !find_o1(k, dtype, true) && !narrow_records &&
        (variant == MF_AUTO || find_o1(k, dtype, false))) {
        int rc = run_filter(src, dst, H, W, pitch, C, dtype, k, variant, nullptr, 0, s);
        if (rc) return rc;
        return launch_argmedian_from_values(a, C, k, dtype, s);
    }
    return launch_resolved(a, C, k, dtype, variant, s);
}

// Rows y0 .. y0 + h - 1 of one plane of H_img rows, all of which are valid
// input (the rows around the band feed its windows): the host pipeline's
// unit of work.
static int run_filter_band(const char *src, char *dst, int H_img, int W, size_t pitch, int dtype, int k,
                           int variant, int y0, int h, cudaStream_t s) {
    if (k == 1) {
        cudaError_t e = cudaMemcpy2DAsync(dst + (size_t)y0 * pitch, pitch, src + (size_t)y0 * pitch, pitch,
                                          (size_t)W * esize(dtype), (size_t)h, cudaMemcpyDeviceToDevice, s);
        return e == cudaSuccess ? MF_OK : cuda_fail(e, "identity copy");
    }
    ImgArgs a;
    a.src = src + (size_t)y0 * pitch;
    a.dst = dst + (size_t)y0 * pitch;
    a.idx = nullptr;
    a.H = h;
    a.W = W;
    a.y_lo = -y0;
    a.y_hi = H_img - 1 - y0;
    a.pitch = pitch;
    a.plane = (size_t)H_img * pitch;
    a.idx_pitch = a.idx_plane = 0;
    return launch_resolved(a, 1, k, dtype, variant, s);
}

}  // namespace mf

using namespace mf;

extern "C" {

int mf_median_filter(const void *src, void *dst, int H, int W, size_t pitch, int channels,
                     mf_dtype dtype, int k, mf_border border, mf_stream_t stream) {
    int rc = check_fwd(src, dst, H, W, pitch, channels, dtype, k, border, nullptr, 0);
    if (rc || !dst) return rc ? rc : (set_error("null dst"), MF_ERR_ARG);
    return run_filter(src, dst, H, W, pitch, channels, dtype, k, MF_AUTO, nullptr, 0,
                      (cudaStream_t)stream);
}

int mf_median_filter_ex(const void *src, void *dst, int H, int W, size_t pitch, int channels,
                        mf_dtype dtype, int k, mf_border border, mf_variant variant,
                        int32_t *argidx, size_t idx_pitch, mf_stream_t stream) {
    int rc = check_fwd(src, dst, H, W, pitch, channels, dtype, k, border, argidx, idx_pitch);
    if (rc) return rc;
    if (variant != MF_AUTO && variant != MF_OBLIVIOUS && variant != MF_DATA_AWARE) {
        set_error("unknown variant %d", (int)variant);
        return MF_ERR_ARG;
    }
    return run_filter(src, dst, H, W, pitch, channels, dtype, k, variant, argidx, idx_pitch,
                      (cudaStream_t)stream);
}

int mf_median_filter_tile(const void *src, void *dst, int H, int W, size_t pitch, int channels,
                          mf_dtype dtype, int k, int tile, mf_stream_t stream) {
    int rc = check_fwd(src, dst, H, W, pitch, channels, dtype, k, MF_BORDER_CLAMP, nullptr, 0);
    if (rc) return rc;
    if (!dst) { set_error("null dst"); return MF_ERR_ARG; }
    if (k == 1)
        return run_filter(src, dst, H, W, pitch, channels, dtype, k, MF_AUTO, nullptr, 0, (cudaStream_t)stream);
    if (!d1_supported_tile(k, dtype, false, tile)) {
        set_error("no data-aware plan for k=%d with a %dx%d root tile", k, tile, tile);
        return MF_ERR_UNSUPPORTED;
    }
    ImgArgs a;
    a.src = (const char *)src;
    a.dst = (char *)dst;
    a.idx = nullptr;
    a.H = H;
    a.y_lo = 0;
    a.y_hi = H - 1;
    a.W = W;
    a.pitch = pitch;
    a.plane = (size_t)H * pitch;
    a.idx_pitch = a.idx_plane = 0;
    return d1_launch(a, channels, k, dtype, tile, (cudaStream_t)stream);
}

int mf_median_filter_rect(const void *src, void *dst, int H, int W, size_t pitch, int channels,
                          mf_dtype dtype, int kw, int kh, int32_t *argidx, size_t idx_pitch,
                          mf_stream_t stream) {
    int rc = check_fwd(src, dst, H, W, pitch, channels, dtype, kw, MF_BORDER_CLAMP, argidx, idx_pitch);
    if (rc) return rc;
    if (kh < 1 || kh > 75 || (kh & 1) == 0) { set_error("kh must be odd in 1..75 (got %d)", kh); return MF_ERR_ARG; }
    if (kw == kh)
        return run_filter(src, dst, H, W, pitch, channels, dtype, kw, MF_AUTO, argidx, idx_pitch,
                          (cudaStream_t)stream);
    ImgArgs a;
    a.src = (const char *)src;
    a.dst = (char *)dst;
    a.idx = argidx;
    a.H = H;
    a.W = W;
    a.y_lo = 0;
    a.y_hi = H - 1;
    a.pitch = pitch;
    a.plane = (size_t)H * pitch;
    a.idx_pitch = idx_pitch;
    a.idx_plane = (size_t)H * idx_pitch;
    return d1_launch(a, channels, kw, dtype, 0, (cudaStream_t)stream, kh);
}

int mf_median_filter_config(const void *src, void *dst, int H, int W, size_t pitch, int channels,
                            mf_dtype dtype, int k, int config, mf_stream_t stream) {
    int rc = check_fwd(src, dst, H, W, pitch, channels, dtype, k, MF_BORDER_CLAMP, nullptr, 0);
    if (rc) return rc;
    if (!dst) { set_error("null dst"); return MF_ERR_ARG; }
    const O1Entry *o1 = config >= 0 && k > 1 ? find_o1_nth(k, dtype, false, config) : nullptr;
    if (!o1) {
        set_error("no data-oblivious configuration %d for k=%d dtype=%d", config, k, (int)dtype);
        return MF_ERR_UNSUPPORTED;
    }
    ImgArgs a;
    a.src = (const char *)src;
    a.dst = (char *)dst;
    a.idx = nullptr;
    a.H = H;
    a.y_lo = 0;
    a.y_hi = H - 1;
    a.W = W;
    a.pitch = pitch;
    a.plane = (size_t)H * pitch;
    a.idx_pitch = a.idx_plane = 0;
    rc = o1->launch(a, channels, (cudaStream_t)stream);
    if (rc == MF_ERR_CUDA) set_error("%s: %s", o1->name, cudaGetErrorString(cudaGetLastError()));
    return rc;
}

// Device staging buffers and streams of the host entry point (one set per
// process, grown on demand, serialised by a mutex, released by
// mf_shutdown).  The planes are cut into bands of whole rows (about 8 MB of
// input each) that flow through four streams: uploads, two filtering
// streams taking bands in turn (so the tail of one band's kernel overlaps
// the next band's), and downloads.  A band is filtered as soon as its rows
// and the r rows below it are on the device (each row is uploaded once),
// and downloaded as soon as it is filtered, so only the first band's upload
// and the last band's download are not hidden behind the filtering.
static std::mutex g_stage_mu;
static void *g_stage_src = nullptr, *g_stage_dst = nullptr;
static size_t g_stage_bytes = 0;
static cudaStream_t g_stage_streams[4] = {nullptr, nullptr, nullptr, nullptr};  // uploads, filtering x 2, downloads
static cudaEvent_t g_stage_events[3] = {nullptr, nullptr, nullptr};    // start, uploaded, filtered

int mf_median_filter_host(const void *src_host, void *dst_host, int H, int W, size_t pitch,
                          int channels, mf_dtype dtype, int k, mf_border border,
                          mf_variant variant, mf_stream_t stream) {
    if (!src_host || !dst_host) { set_error("null pointer"); return MF_ERR_ARG; }
    const int es = esize(dtype);
    if (es == 0) { set_error("unknown dtype %d", dtype); return MF_ERR_DTYPE; }
    if (H < 1 || W < 1 || channels < 1) { set_error("bad shape"); return MF_ERR_ARG; }
    if (pitch < (size_t)W * es || pitch % es) { set_error("bad pitch"); return MF_ERR_PITCH; }
    if (variant != MF_AUTO && variant != MF_OBLIVIOUS && variant != MF_DATA_AWARE) {
        set_error("unknown variant %d", (int)variant);
        return MF_ERR_ARG;
    }
    const size_t dpitch = ((size_t)W * es + 255) & ~(size_t)255;
    const size_t plane = (size_t)H * dpitch;
    const size_t bytes = (size_t)channels * plane;
    cudaStream_t s = (cudaStream_t)stream;
    std::lock_guard<std::mutex> lk(g_stage_mu);
    if (g_stage_bytes < bytes) {
        if (g_stage_src) { cudaFree(g_stage_src); cudaFree(g_stage_dst); }
        g_stage_src = g_stage_dst = nullptr;
        g_stage_bytes = 0;
        if (dev_alloc(&g_stage_src, bytes) != cudaSuccess || dev_alloc(&g_stage_dst, bytes) != cudaSuccess) {
            cudaGetLastError();
            if (g_stage_src) cudaFree(g_stage_src);
            g_stage_src = g_stage_dst = nullptr;
            set_error("cannot allocate %zu bytes of device staging", 2 * bytes);
            return MF_ERR_ALLOC;
        }
        g_stage_bytes = bytes;
    }
    // the same checks as the device entry points (k, border, sizes)
    int rc = check_fwd(g_stage_src, g_stage_dst, H, W, dpitch, channels, dtype, k, border, nullptr, 0);
    if (rc) return rc;
    if (!g_stage_streams[0]) {
        for (int i = 0; i < 4; i++) {
            if (cudaStreamCreateWithFlags(&g_stage_streams[i], cudaStreamNonBlocking) != cudaSuccess ||
                (i < 3 && cudaEventCreateWithFlags(&g_stage_events[i], cudaEventDisableTiming) != cudaSuccess)) {
                set_error("cannot create staging streams: %s", cudaGetErrorString(cudaGetLastError()));
                return MF_ERR_CUDA;
            }
        }
    }
    cudaStream_t s_in = g_stage_streams[0], s_out = g_stage_streams[3];
    int band = 0;
    // the pipeline starts after work already queued on the caller's stream
    cudaError_t e = cudaEventRecord(g_stage_events[0], s);
    for (int i = 0; i < 4 && e == cudaSuccess; i++) e = cudaStreamWaitEvent(g_stage_streams[i], g_stage_events[0], 0);
    if (e != cudaSuccess) return cuda_fail(e, "pipeline start");
    const size_t row_bytes = (size_t)W * es;
    int bh = (int)std::min<size_t>((size_t)H, std::max<size_t>(32, ((size_t)8 << 20) / row_bytes / 32 * 32));
    const int r = (k - 1) / 2;
    const char *hs = (const char *)src_host;
    char *hd = (char *)dst_host;
    for (int c = 0; c < channels; c++) {
        char *ds = (char *)g_stage_src + c * plane, *dd = (char *)g_stage_dst + c * plane;
        const char *hsc = hs + (size_t)c * H * pitch;
        char *hdc = hd + (size_t)c * H * pitch;
        int uploaded = 0;  // rows of this plane already on the device
        for (int y0 = 0; y0 < H; y0 += bh) {
            const int h = std::min(bh, H - y0);
            const int need = std::min(H, y0 + h + r);
            if (need > uploaded) {
                e = cudaMemcpy2DAsync(ds + (size_t)uploaded * dpitch, dpitch, hsc + (size_t)uploaded * pitch, pitch,
                                      row_bytes, (size_t)(need - uploaded), cudaMemcpyHostToDevice, s_in);
                if (e != cudaSuccess) return cuda_fail(e, "host to device copy");
                uploaded = need;
            }
            cudaStream_t s_k = g_stage_streams[1 + (band++ & 1)];
            // each wait takes the event's latest record at the time it is enqueued
            e = cudaEventRecord(g_stage_events[1], s_in);
            if (e == cudaSuccess) e = cudaStreamWaitEvent(s_k, g_stage_events[1], 0);
            if (e != cudaSuccess) return cuda_fail(e, "pipeline order");
            rc = run_filter_band(ds, dd, H, W, dpitch, dtype, k, variant, y0, h, s_k);
            if (rc) return rc;
            e = cudaEventRecord(g_stage_events[2], s_k);
            if (e == cudaSuccess) e = cudaStreamWaitEvent(s_out, g_stage_events[2], 0);
            if (e != cudaSuccess) return cuda_fail(e, "pipeline order");
            e = cudaMemcpy2DAsync(hdc + (size_t)y0 * pitch, pitch, dd + (size_t)y0 * dpitch, dpitch, row_bytes,
                                  (size_t)h, cudaMemcpyDeviceToHost, s_out);
            if (e != cudaSuccess) return cuda_fail(e, "device to host copy");
        }
    }
    for (int i = 0; i < 4; i++) {
        e = cudaStreamSynchronize(g_stage_streams[i]);
        if (e != cudaSuccess) return cuda_fail(e, "stream synchronize");
    }
    return MF_OK;
}

int mf_median_filter_bwd(const float *grad_out, const int32_t *argidx, float *grad_in, int H, int W,
                         size_t pitch, size_t idx_pitch, int channels, int k, mf_grad_mode mode,
                         mf_stream_t stream) {
    if (!grad_out || !argidx || !grad_in) { set_error("null pointer"); return MF_ERR_ARG; }
    if (H < 1 || W < 1 || channels < 1 || channels > 65535) { set_error("bad shape"); return MF_ERR_ARG; }
    if ((long long)H * W > (1ll << 31) - 1) { set_error("plane too large for int32 indices"); return MF_ERR_ARG; }
    if (k < 1 || k > 75 || !(k & 1)) { set_error("k must be odd in 1..75"); return MF_ERR_ARG; }
    if (pitch < (size_t)W * 4 || pitch % 4) { set_error("bad pitch"); return MF_ERR_PITCH; }
    if (idx_pitch < (size_t)W * 4 || idx_pitch % 4) { set_error("bad idx_pitch"); return MF_ERR_PITCH; }
    const size_t gb = (size_t)channels * H * pitch, ib = (size_t)channels * H * idx_pitch;
    if (overlap(grad_in, gb, grad_out, gb) || overlap(grad_in, gb, argidx, ib)) {
        set_error("grad_in overlaps an input");
        return MF_ERR_ALIAS;
    }
    cudaStream_t s = (cudaStream_t)stream;
    if (mode == MF_GRAD_ATOMIC) return bwd_atomic(grad_out, argidx, grad_in, H, W, pitch, idx_pitch, channels, s);
    if (mode == MF_GRAD_DETERMINISTIC)
        return bwd_ordered(grad_out, argidx, grad_in, H, W, pitch, idx_pitch, channels, k, s);
    set_error("unknown gradient mode %d", (int)mode);
    return MF_ERR_ARG;
}

int mf_describe(int H, int W, int channels, mf_dtype dtype, int k, mf_variant variant, char *buf,
                size_t buflen) {
    if (!buf || buflen == 0) { set_error("null buffer"); return MF_ERR_ARG; }
    if (esize(dtype) == 0) { set_error("unknown dtype"); return MF_ERR_DTYPE; }
    if (k < 1 || k > 75 || !(k & 1) || H < 1 || W < 1 || channels < 1) { set_error("bad arguments"); return MF_ERR_ARG; }
    if (k == 1) { snprintf(buf, buflen, "identity copy"); return MF_OK; }
    Plan p;
    int rc = resolve(k, dtype, false, variant, &p, size_bucket((long long)H * W), true);
    if (rc) return rc;
    if (p.variant == MF_OBLIVIOUS)
        snprintf(buf, buflen, "oblivious k=%d tile=%dx%d block=%dx%d run=%d net_ops=%d kernel=%s", k, p.o1->tw,
                 p.o1->th, p.o1->bx, p.o1->by, p.o1->run, p.o1->net_ops, p.o1->name);
    else
        d1_describe(k, dtype, false, p.tile, buf, buflen);  // the tile of this image's size bucket
    return MF_OK;
}

uint64_t mf_kernel_launch_count(void) { return g_launches.load(); }

const char *mf_status_string(int status) {
    switch (status) {
        case MF_OK: return "ok";
        case MF_ERR_ARG: return "invalid argument";
        case MF_ERR_DTYPE: return "unsupported dtype";
        case MF_ERR_PITCH: return "invalid pitch";
        case MF_ERR_ALIAS: return "buffers overlap";
        case MF_ERR_ALLOC: return "allocation failed";
        case MF_ERR_CUDA: return "CUDA error";
        case MF_ERR_TIMEOUT: return "device wait timed out";
        case MF_ERR_INTERNAL: return "internal error";
        case MF_ERR_UNSUPPORTED: return "no kernel for this configuration";
        default: return "unknown status";
    }
}

const char *mf_last_error(void) { return g_err; }

const char *mf_version(void) { return "medianfilter-gb300 0.1 (sm_103a)"; }

int mf_shutdown(void) {
    std::lock_guard<std::mutex> lk(g_stage_mu);
    if (g_stage_src) cudaFree(g_stage_src);
    if (g_stage_dst) cudaFree(g_stage_dst);
    g_stage_src = g_stage_dst = nullptr;
    g_stage_bytes = 0;
    for (int i = 0; i < 4; i++) {
        if (g_stage_streams[i]) cudaStreamDestroy(g_stage_streams[i]);
        g_stage_streams[i] = nullptr;
    }
    for (int i = 0; i < 3; i++) {
        if (g_stage_events[i]) cudaEventDestroy(g_stage_events[i]);
        g_stage_events[i] = nullptr;
    }
    d1_release_all();
    d3_release_all();
    return MF_OK;
}

}  // extern "C"
