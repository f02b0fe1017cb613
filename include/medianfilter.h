/*
 * medianfilter.h -- C ABI of the GB300 (sm_103a) k x k median filter.
 *
 * The filter replaces every pixel by the median of the k x k neighbourhood
 * centred on it (paper: "A Fast Parallel Median Filtering Algorithm Using
 * Hierarchical Tiling", Sec. 1).  It is computed by hierarchical tiling
 * (Sec. 3) with either the data-oblivious selection network held in
 * registers (Sec. 4) or the data-aware merge variant (Sec. 5).  Both give
 * exactly the same result: selection does no arithmetic, so outputs are
 * bit-copies of input elements.
 *
 * Conventions fixed by this library where the paper is silent:
 *   - borders clamp to the edge (window reads src[clamp(y+dy)][clamp(x+dx)]);
 *   - k is odd, 1 <= k <= 75 (k = 1 is the identity); the median is the
 *     element of 0-based rank (k*k-1)/2 of the window;
 *   - f32 values are ordered by their sign-flipped bit pattern:
 *     -NaN < -inf < ... < -0 < +0 < ... < +inf < +NaN;
 *   - the argmedian of a pixel is the source pixel of the rank-(k*k-1)/2
 *     window element under (value, row-major window slot) order, stored as
 *     ys * W + xs within the channel plane.
 *
 * Memory: every image pointer below is device memory owned by the caller,
 * except where an entry point says "host".  Channels are planar: plane c of
 * an image starts at base + c * H * pitch, for src and dst alike.  pitch
 * is in bytes, a multiple of the element size and >= W * element size.
 *
 * Streams: device entry points enqueue work on `stream` (a cudaStream_t;
 * NULL = the legacy default stream) and return without synchronising.
 * Errors: every entry point returns MF_OK (0) or a negative mf_status;
 * arguments are checked before anything is launched, no error terminates
 * the process, and mf_last_error() gives a one-line description of the
 * calling thread's last failure.  For testing error paths, the environment
 * variable MF_FAULT_INJECT=alloc makes every device allocation the library
 * itself makes fail (entry points then return MF_ERR_ALLOC).
 */
#ifndef MEDIANFILTER_H
#define MEDIANFILTER_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

struct CUstream_st;
typedef struct CUstream_st *mf_stream_t; /* identical to cudaStream_t */

typedef enum { MF_U8 = 0, MF_U16 = 1, MF_U32 = 2, MF_F32 = 3 } mf_dtype;
typedef enum { MF_BORDER_CLAMP = 0 } mf_border;
typedef enum { MF_AUTO = 0, MF_OBLIVIOUS = 1, MF_DATA_AWARE = 2 } mf_variant;
typedef enum { MF_GRAD_ATOMIC = 0, MF_GRAD_DETERMINISTIC = 1 } mf_grad_mode;

typedef enum {
    MF_OK = 0,
    MF_ERR_ARG = -1,      /* bad k, H, W, channels, or a NULL pointer */
    MF_ERR_DTYPE = -2,    /* dtype not supported by this entry point */
    MF_ERR_PITCH = -3,    /* pitch too small or not a multiple of the element size */
    MF_ERR_ALIAS = -4,    /* src and dst overlap */
    MF_ERR_ALLOC = -5,    /* device or host allocation failed */
    MF_ERR_CUDA = -6,     /* a CUDA call failed; see mf_last_error() */
    MF_ERR_TIMEOUT = -7,  /* a bounded device-side wait gave up */
    MF_ERR_INTERNAL = -8, /* an internal consistency check failed */
    MF_ERR_UNSUPPORTED = -9 /* no kernel instantiated for this request */
} mf_status;

/* Median filter of `channels` planar planes of H x W elements of `dtype`
 * (paper Sec. 1 definition; computed by hierarchical tiling, Sec. 3).
 * src, dst: device pointers, caller-owned, must not overlap.  The variant
 * and tile shape are chosen automatically (autotuner cache, else the paper's
 * root-tile heuristic t(k) = 2^(floor(log2 k) - 1), Sec. 4.2). */
int mf_median_filter(const void *src, void *dst, int H, int W, size_t pitch, int channels,
                     mf_dtype dtype, int k, mf_border border, mf_stream_t stream);

/* As mf_median_filter, with an explicit variant (Sec. 4 oblivious network,
 * Sec. 5 data-aware merges) and an optional argmedian output.
 * argidx: NULL, or a caller-owned device buffer of int32 with `idx_pitch`
 * bytes per row (>= 4 * W, multiple of 4); plane c starts at
 * argidx + c * H * idx_pitch.  Entry (y, x) receives ys * W + xs of the
 * source pixel of the median (tie rule: lowest value, then lowest row-major
 * window slot).  dst may be NULL when argidx is given. */
int mf_median_filter_ex(const void *src, void *dst, int H, int W, size_t pitch, int channels,
                        mf_dtype dtype, int k, mf_border border, mf_variant variant,
                        int32_t *argidx, size_t idx_pitch, mf_stream_t stream);

/* The data-aware variant (Sec. 5) with an explicit root tile of tile x tile
 * pixels (a power of two, 2..32, at most k): every tile size is a different
 * tiling tree (Sec. 3.1) computing the same filter.  Arguments and errors
 * as mf_median_filter; MF_ERR_UNSUPPORTED if the tree's state for this tile
 * does not fit in shared memory. */
int mf_median_filter_tile(const void *src, void *dst, int H, int W, size_t pitch, int channels,
                          mf_dtype dtype, int k, int tile, mf_stream_t stream);

/* A window of kw columns by kh rows (both odd, 1..75; the paper states its
 * tile terminology for a k_w x k_h kernel, Sec. 3.2): out(y, x) is the
 * element of 0-based rank (kw*kh-1)/2 of the clamp-to-edge window rows
 * y-(kh-1)/2 .. y+(kh-1)/2 by columns x-(kw-1)/2 .. x+(kw-1)/2.  Square
 * windows take the mf_median_filter_ex path (MF_AUTO); other shapes run the
 * data-aware variant (Sec. 5) with a T x T root tile, T at most the shorter
 * side.  argidx: NULL or as for mf_median_filter_ex (tie rule: lowest
 * value, then lowest row-major window slot (dy+ry)*kw + (dx+rx)).  Errors
 * as mf_median_filter_ex. */
int mf_median_filter_rect(const void *src, void *dst, int H, int W, size_t pitch, int channels,
                          mf_dtype dtype, int kw, int kh, int32_t *argidx, size_t idx_pitch,
                          mf_stream_t stream);

/* The data-oblivious variant (Sec. 4) with the config-th instantiated
 * network configuration for (k, dtype) (0 = the default; the others are the
 * autotuner's candidates: other network forms, tiles or key widths, all
 * computing the same filter).  Arguments and errors as mf_median_filter;
 * MF_ERR_UNSUPPORTED when config is negative or past the last one, so
 * callers can enumerate them. */
int mf_median_filter_config(const void *src, void *dst, int H, int W, size_t pitch, int channels,
                            mf_dtype dtype, int k, int config, mf_stream_t stream);

/* Gradient of the filter with respect to its f32 input: grad_in[p] = sum
 * of grad_out[q] over the outputs q whose argmedian is p (the median is the
 * identity on its selected input).  All pointers are caller-owned device
 * memory; grad_out and grad_in use `pitch` (bytes, >= 4 * W), argidx uses
 * idx_pitch.  MF_GRAD_ATOMIC zeroes grad_in and scatter-adds with atomics
 * (summation order unspecified); MF_GRAD_DETERMINISTIC adds, for each p,
 * the contributions in increasing row-major q (an ordered scatter through
 * shared memory; bit-identical run to run and to a sequential scatter).
 * k bounds the distance between q and p.  grad_in must not overlap
 * grad_out or argidx. */
int mf_median_filter_bwd(const float *grad_out, const int32_t *argidx, float *grad_in,
                         int H, int W, size_t pitch, size_t idx_pitch, int channels, int k,
                         mf_grad_mode mode, mf_stream_t stream);

/* The same filter on HOST buffers: copies src (pitch bytes per row) to the
 * device, filters, copies the result back into dst (host) and waits for
 * completion.  Each plane is cut into bands of whole rows (about 8 MB of
 * input each) that flow through internal streams -- uploads, two filtering
 * streams taking bands in turn, downloads -- so that only the first band's
 * upload and the last band's download are not overlapped; a band is
 * filtered once its rows and
 * the (k-1)/2 rows below it are on the device.  The pipeline starts after
 * whatever is already queued on `stream`.  Host buffers are
 * caller-owned; page-locked memory makes the copies asynchronous DMA.
 * Device staging memory and the streams are owned by the library: one set
 * per process, grown on demand, shared by calls under a lock and released
 * by mf_shutdown(). */
int mf_median_filter_host(const void *src_host, void *dst_host, int H, int W, size_t pitch,
                          int channels, mf_dtype dtype, int k, mf_border border,
                          mf_variant variant, mf_stream_t stream);

/* ---- batched persistent launch --------------------------------------- */

typedef struct {
    const void *src;  /* device, caller-owned */
    void *dst;        /* device, caller-owned */
    int H, W;
    size_t pitch;     /* bytes, src and dst */
    int channels;
    mf_dtype dtype;
    int k;            /* odd, 1..31 */
} mf_image_desc;

typedef struct mf_batch_plan mf_batch_plan;

/* Plans many images of uneven sizes, dtypes and k (odd, 1..31) for one
 * CUDA-graph launch.  Images are grouped by the kernel the plain entry point
 * would run for them; each group gets one persistent kernel whose blocks
 * claim (image, block, plane) work items from a device-side queue, largest
 * images first; the groups run as concurrent branches of the graph.  The
 * plan owns its device memory (image table, work lists, queue counters),
 * streams and graph until destroyed.  The descriptors are copied; the image
 * buffers they point to must stay valid while the plan is run.  Must be
 * called outside any stream capture. */
int mf_batch_plan_create(const mf_image_desc *descs, int n, mf_batch_plan **out);
/* As mf_batch_plan_create; with tune != 0 every (k, dtype, image-size
 * bucket) of the batch that the tuning table has no entry for is first
 * tuned on the largest image of that group -- like mf_autotune, but each
 * candidate is timed on enough concurrent copies of the image (outputs in
 * scratch the call allocates and frees; the image's own dst is written too)
 * to fill the GPU, since the batch runs its kernel classes concurrently and
 * needs throughput, not the latency of one small launch -- and the images
 * are then grouped by the kernel each one's bucket selects (variant,
 * network configuration or data-aware root tile).  The paper picks its block
 * shape per kernel size and data type by measurement (Sec. 4.3); here the
 * choice is also per image size.  Synchronises the device when it tunes. */
int mf_batch_plan_create_ex(const mf_image_desc *descs, int n, int tune, mf_batch_plan **out);
/* Runs a plan on `stream` (one CUDA graph launch: queue reset + kernel). */
int mf_batch_run(mf_batch_plan *plan, mf_stream_t stream);
int mf_batch_plan_destroy(mf_batch_plan *plan);
/* Kernel launches per run (one per kernel class) and work items of a plan. */
int mf_batch_describe(const mf_batch_plan *plan, int *kernels, long long *items);

/* Batched filter that allocates nothing (the paper has no counterpart: this
 * serves callers that must not allocate device memory when they filter --
 * e.g. code running while another framework's caching allocator owns the
 * device, loops that must never wait inside an allocator, or deployments
 * with a device memory budget fixed in advance).  Filters each image of
 * descs (device buffers, as for mf_batch_plan_create) with the persistent
 * data-oblivious kernels, taking its work queues from one fixed array of
 * 2 MiB that the library's module holds on every device where it is used,
 * until the library is unloaded.  Limits: at most 256 images, k = 1 or a
 * k the data-oblivious kernels are built for (odd 3 to 27), and at most
 * 129,392 work items (one item is one
 * thread block's pixels -- lanes x block width x tile width x run by block
 * height x tile height, as mf_describe reports them); beyond them it returns
 * MF_ERR_ARG
 * or MF_ERR_UNSUPPORTED with a message, before touching the device.
 * Nothing is allocated (no cudaMalloc, cudaFree or allocating library
 * call): the image table and work records are copied from the stack, the
 * queue counters are cleared on every call.  The first call on a device
 * looks up the array's device address (cudaGetSymbolAddress) with that
 * device current; make that first call before any stream capture.  The
 * table copies come from pageable (stack) memory, so the call may wait
 * until earlier work on `stream` has drained before it returns; for the
 * same reason a call on a stream that is being captured is rejected with
 * MF_ERR_UNSUPPORTED.  Each device has its own copy of the array, which
 * keeps the last call's contents, so calls whose work overlaps on the GPU
 * of one device (different streams, or threads sharing a device) race;
 * calls issued in order on one stream are safe.  Work is enqueued on
 * `stream` and the call does not wait for it to finish.  An error returned
 * after the argument checks (a failed launch) can leave the kernel classes
 * enqueued before the failure in the stream: their images may be
 * filtered, the others are not. */
int mf_batch_run_static(const mf_image_desc *descs, int n, mf_stream_t stream);

/* ---- tuning and introspection ------------------------------------------ */

/* Times the instantiated candidates for one (k, dtype, H, W) on the current
 * device -- every data-oblivious configuration (network form, tile, block
 * shape, key width) and every data-aware root tile -- and records the
 * fastest in the in-memory tuning table under the image's size bucket
 * (floor(log2(H * W) / 2), clamped to 7..12), and in the JSON file named by
 * MF_TUNE_CACHE, if set.  Calls on images of other sizes use the entry of
 * the nearest bucket.  Uses caller-owned scratch: src and dst must be device
 * buffers of channels * H * pitch bytes. */
int mf_autotune(const void *src, void *dst, int H, int W, size_t pitch, int channels,
                mf_dtype dtype, int k, mf_stream_t stream);

/* Describes the plan mf_median_filter would launch: writes a one-line
 * description (variant, tile, block) into buf.  Returns MF_OK or an error. */
int mf_describe(int H, int W, int channels, mf_dtype dtype, int k, mf_variant variant,
                char *buf, size_t buflen);

/* Min/max throughput microbenchmark (the denominator of the data-oblivious
 * kernels' ALU roofline; no counterpart in the paper).  kind: 0 = u32,
 * 1 = packed u16x2, 2 = f32, 3 = packed f16x2, 4 = u16x2 min interleaved
 * with f16x2 max, 5 = u32 min interleaved with f32 max, 6 = three-input
 * u16x2 min/max, 7 = three-input u32 min/max, 8 = four-lane u8 min/max
 * (__vminu4/__vmaxu4), 9 = warp shuffles, 10 = byte permutes (the last two
 * are the exchange and packing steps the kernels could use instead of
 * shared memory).  Runs `iters`
 * iterations of 16 min/max per thread on 4 blocks of 256 threads per SM of
 * the current device (the library allocates and frees its own 8 KB-scale
 * buffers) and writes instructions per second (one per thread-instruction)
 * and the best of three elapsed times in milliseconds (ms may be NULL). */
int mf_probe_minmax(int kind, int iters, double *instr_per_s, double *ms);

/* Host-side check of the data-aware schedule (paper Sec. 5 method, as
 * planned by this library): builds the plan for a k x k kernel and a strip
 * of `strip` root tiles of tile x tile pixels side by side and, if
 * footprint and medians are non-NULL, runs it on the CPU for one footprint
 * of (tile + k - 1) rows x (strip*tile + k - 1) columns of 64-bit order keys
 * (row-major, clamped by the caller), writing the tile x strip*tile medians
 * (row-major).  stats (NULL or 7 ints): shared-memory list elements, phases,
 * tasks, work items, merged elements, sorted elements, longest sort.  No GPU
 * is used.  Returns MF_ERR_UNSUPPORTED when no plan exists. */
int mf_d1_plan_check(int k, int tile, int strip, const uint64_t *footprint, uint64_t *medians,
                     int *stats);

/* As mf_d1_plan_check for a window of kw columns by kh rows (both odd) and
 * root tiles of tile_w columns by tile_h rows (powers of two, at most the
 * window side, 1 allowed); the footprint is (tile_h + kh - 1) rows x
 * (strip*tile_w + kw - 1) columns, the medians tile_h x strip*tile_w. */
int mf_d1_plan_check_rect(int kw, int kh, int tile_w, int tile_h, int strip, const uint64_t *footprint,
                          uint64_t *medians, int *stats);

/* As mf_d1_plan_check_rect for the plan the kernels build for keys of
 * key_bytes bytes (1, 2, 4 or 8: 8-bit values, 16-bit values or 8/16-bit
 * records, 32-bit values, 32-bit records) run by blocks of `threads` threads
 * (256, 512 or 1024): the key width and the block size select the merge
 * chunks, the list padding, phase balancing and the longest sort
 * (mf_d1_plan_check_rect plans for 4-byte keys and 256 threads).  The
 * footprint still holds 64-bit keys.  MF_ERR_ARG for other key widths or
 * block sizes. */
int mf_d1_plan_check_ex(int kw, int kh, int tile_w, int tile_h, int strip, int key_bytes, int threads,
                        const uint64_t *footprint, uint64_t *medians, int *stats);

/* Number of CUDA kernels this library launched since load (all threads). */
uint64_t mf_kernel_launch_count(void);

const char *mf_status_string(int status);
const char *mf_last_error(void);
const char *mf_version(void);

/* Releases cached device memory of the calling process. */
int mf_shutdown(void);

#ifdef __cplusplus
}
#endif

#endif /* MEDIANFILTER_H */
