/*
 * CPU oracle for the 2D k x k median filter -- TEST INFRASTRUCTURE ONLY.
 *
 * This file is the plain, slow, obviously correct definition that the CUDA
 * library is checked against.  Only the test-suite, the smoke check and the
 * CPU-baseline leg of the benchmark load it.  It shares no code, header,
 * helper or table with the CUDA path (paper_2507_19926_gb300/), and the
 * CUDA path never loads it.
 *
 * What is computed (paper Sec. 1, "The problem" / introduction): every pixel
 * is replaced by the median of the k x k rectangular neighbourhood centred
 * on it.  The paper is silent on borders, on the order of f32 values and on
 * which equal element an "argmedian" refers to; the readings used here are:
 *   - borders clamp to the edge: window slot (dy, dx), dy, dx in [-r, r],
 *     r = (k-1)/2, reads src[clamp(y+dy)][clamp(x+dx)];
 *   - k is odd, so the median is the element of 0-based rank m = (k*k-1)/2;
 *   - values are ordered by an unsigned 32-bit key: u8/u16/u32 by value,
 *     f32 by the sign-flip key (negative: all bits inverted; otherwise the
 *     sign bit set), i.e. -NaN < -inf < ... < -0 < +0 < ... < +inf < +NaN;
 *   - the argmedian is the rank-m element under the lexicographic order of
 *     (key, window slot s = (dy+r)*k + (dx+r)) -- lowest value first, then
 *     lowest row-major window slot.  Its index is ys*W + xs of the source
 *     pixel (after clamping), within the channel plane.
 * The median value is copied bit-for-bit from the winning source pixel:
 * selection performs no arithmetic.
 *
 * Rectangular windows (or_median_filter_rect): the paper states its tile
 * terminology for a k_w x k_h kernel (Sec. 3.2); the same definition with
 * kw columns and kh rows (both odd) takes the element of 0-based rank
 * (kw*kh-1)/2 of window slots s = (dy+ry)*kw + (dx+rx), rx = (kw-1)/2,
 * ry = (kh-1)/2.  k x k is the case kw = kh = k.
 *
 * Backward (derivative of the filter w.r.t. its input): the median is, piece
 * by piece, the identity on the selected input, so d out[q] / d in[p] is 1
 * when p = idx[q] and 0 otherwise; grad_in[p] = sum of grad_out[q] over the
 * q with idx[q] = p, accumulated in f32 in increasing row-major q.
 *
 * Layout: planar channels, each plane H*W elements contiguous, row-major.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

enum { OR_U8 = 0, OR_U16 = 1, OR_U32 = 2, OR_F32 = 3 };

static int elem_size(int dtype)
{
    switch (dtype) {
    case OR_U8: return 1;
    case OR_U16: return 2;
    case OR_U32: return 4;
    case OR_F32: return 4;
    default: return 0;
    }
}

/* Order key of element i of a plane.  For f32 the key is the IEEE bit
 * pattern with the sign bit set for non-negative numbers and every bit
 * inverted for negative ones, which sorts as the real numbers do and puts
 * -0 directly below +0. */
static uint32_t key_at(const void *plane, long i, int dtype)
{
    uint32_t b;
    switch (dtype) {
    case OR_U8: return ((const uint8_t *)plane)[i];
    case OR_U16: return ((const uint16_t *)plane)[i];
    case OR_U32: return ((const uint32_t *)plane)[i];
    default:
        memcpy(&b, (const char *)plane + 4 * i, 4);
        return (b & 0x80000000u) ? ~b : (b | 0x80000000u);
    }
}

uint32_t or_key(int dtype, uint32_t bits)
{
    if (dtype == OR_F32)
        return (bits & 0x80000000u) ? ~bits : (bits | 0x80000000u);
    return bits;
}

static int clampi(int v, int lo, int hi) { return v < lo ? lo : (v > hi ? hi : v); }

/* Returns the element of 0-based rank m of a[0..n) (values all distinct),
 * by Hoare's selection: partition around a pivot, keep the side holding m. */
static uint64_t select_rank(uint64_t *a, int n, int m)
{
    int lo = 0, hi = n - 1;
    while (lo < hi) {
        uint64_t pivot = a[lo + (hi - lo) / 2];
        int i = lo, j = hi;
        while (i <= j) {
            while (a[i] < pivot) i++;
            while (a[j] > pivot) j--;
            if (i <= j) {
                uint64_t t = a[i]; a[i] = a[j]; a[j] = t;
                i++; j--;
            }
        }
        if (m <= j) hi = j;
        else if (m >= i) lo = i;
        else break;
    }
    return a[m];
}

/* Median (and argmedian) of one output pixel (y, x) of one plane.
 * win is scratch of k*k entries.  Each entry is the composite
 * (key << 32) | slot, so sorting entries sorts by key, then by slot. */
static void one_pixel(const void *plane, int H, int W, int dtype, int kw, int kh, int y, int x,
                      uint64_t *win, long *src_index)
{
    int rx = (kw - 1) / 2, ry = (kh - 1) / 2, s = 0;
    for (int dy = -ry; dy <= ry; dy++) {
        int ys = clampi(y + dy, 0, H - 1);
        for (int dx = -rx; dx <= rx; dx++) {
            int xs = clampi(x + dx, 0, W - 1);
            win[s] = ((uint64_t)key_at(plane, (long)ys * W + xs, dtype) << 32) | (uint64_t)s;
            s++;
        }
    }
    uint64_t best = select_rank(win, kw * kh, (kw * kh - 1) / 2);
    int slot = (int)(best & 0xffffffffu);
    int dy = slot / kw - ry, dx = slot % kw - rx;
    *src_index = (long)clampi(y + dy, 0, H - 1) * W + clampi(x + dx, 0, W - 1);
}

static int check_args(int H, int W, int C, int dtype, int k)
{
    if (H < 1 || W < 1 || C < 1 || k < 1 || (k & 1) == 0 || elem_size(dtype) == 0) return -1;
    return 0;
}

/* Median filter of C planes of H x W with a kw x kh window (both odd).
 * dst may be NULL (argmedian only); idx may be NULL (values only).
 * nthreads <= 0 means the OpenMP default.  Returns 0, or -1 on a bad
 * argument. */
int or_median_filter_rect(const void *src, void *dst, int32_t *idx, int H, int W, int C,
                          int dtype, int kw, int kh, int nthreads)
{
    if (check_args(H, W, C, dtype, kw) || kh < 1 || (kh & 1) == 0) return -1;
    int es = elem_size(dtype);
    long plane_elems = (long)H * W;
    long rows = (long)C * H;
#ifdef _OPENMP
    if (nthreads <= 0) nthreads = omp_get_max_threads();
#pragma omp parallel num_threads(nthreads)
#endif
    {
        uint64_t *win = (uint64_t *)malloc(sizeof(uint64_t) * (size_t)kw * kh);
#ifdef _OPENMP
#pragma omp for schedule(dynamic, 1)
#endif
        for (long row = 0; row < rows; row++) {
            int c = (int)(row / H), y = (int)(row % H);
            const char *plane = (const char *)src + (size_t)c * plane_elems * es;
            for (int x = 0; x < W; x++) {
                long si;
                one_pixel(plane, H, W, dtype, kw, kh, y, x, win, &si);
                long o = (long)c * plane_elems + (long)y * W + x;
                if (dst) memcpy((char *)dst + (size_t)o * es, plane + (size_t)si * es, es);
                if (idx) idx[o] = (int32_t)si;
            }
        }
        free(win);
    }
    return 0;
}

/* The k x k filter: the square case of or_median_filter_rect. */
int or_median_filter(const void *src, void *dst, int32_t *idx, int H, int W, int C,
                     int dtype, int k, int nthreads)
{
    return or_median_filter_rect(src, dst, idx, H, W, C, dtype, k, k, nthreads);
}

/* The same filter evaluated only on the listed rows of every plane.
 * Outputs are packed: dst / idx hold C * nrows * W entries, plane-major,
 * then in the order of rows[].  Used to sample very large images. */
int or_median_filter_rows(const void *src, void *dst, int32_t *idx, int H, int W, int C,
                          int dtype, int k, const int32_t *rows, int nrows, int nthreads)
{
    if (check_args(H, W, C, dtype, k) || nrows < 0) return -1;
    for (int i = 0; i < nrows; i++)
        if (rows[i] < 0 || rows[i] >= H) return -1;
    int es = elem_size(dtype);
    long plane_elems = (long)H * W;
    long jobs = (long)C * nrows;
#ifdef _OPENMP
    if (nthreads <= 0) nthreads = omp_get_max_threads();
#pragma omp parallel num_threads(nthreads)
#endif
    {
        uint64_t *win = (uint64_t *)malloc(sizeof(uint64_t) * (size_t)k * k);
#ifdef _OPENMP
#pragma omp for schedule(dynamic, 1)
#endif
        for (long j = 0; j < jobs; j++) {
            int c = (int)(j / nrows), i = (int)(j % nrows), y = rows[i];
            const char *plane = (const char *)src + (size_t)c * plane_elems * es;
            for (int x = 0; x < W; x++) {
                long si;
                one_pixel(plane, H, W, dtype, k, k, y, x, win, &si);
                long o = ((long)c * nrows + i) * W + x;
                if (dst) memcpy((char *)dst + (size_t)o * es, plane + (size_t)si * es, es);
                if (idx) idx[o] = (int32_t)si;
            }
        }
        free(win);
    }
    return 0;
}

/* Volumetric k x k x k median (the extension of hierarchical tiling to 3D
 * that the paper names as future work, Sec. 7.2, for medical volumes).
 * Definition: voxel (z, y, x) of a D x H x W volume is replaced by the
 * element of 0-based rank (k^3 - 1)/2 of the multiset of the k^3 values
 * src[clamp(z+dz)][clamp(y+dy)][clamp(x+dx)], dz, dy, dx in [-r, r],
 * under the same order keys as the 2D filter; borders clamp to the edge on
 * every axis.  Values only.  V volumes, each D*H*W elements contiguous,
 * slice-major then row-major.  Returns 0, or -1 on a bad argument. */
int or_median_filter_3d(const void *src, void *dst, int D, int H, int W, int V, int dtype, int k,
                        int nthreads)
{
    if (check_args(H, W, V, dtype, k) || D < 1) return -1;
    int es = elem_size(dtype), r = (k - 1) / 2;
    long vol = (long)D * H * W, n = (long)k * k * k;
    long rows = (long)V * D * H;
#ifdef _OPENMP
    if (nthreads <= 0) nthreads = omp_get_max_threads();
#pragma omp parallel num_threads(nthreads)
#endif
    {
        uint64_t *win = (uint64_t *)malloc(sizeof(uint64_t) * (size_t)n);
#ifdef _OPENMP
#pragma omp for schedule(dynamic, 1)
#endif
        for (long row = 0; row < rows; row++) {
            int v = (int)(row / ((long)D * H)), z = (int)((row / H) % D), y = (int)(row % H);
            const char *base = (const char *)src + (size_t)v * vol * es;
            for (int x = 0; x < W; x++) {
                int s = 0;
                for (int dz = -r; dz <= r; dz++)
                    for (int dy = -r; dy <= r; dy++)
                        for (int dx = -r; dx <= r; dx++) {
                            long si = ((long)clampi(z + dz, 0, D - 1) * H + clampi(y + dy, 0, H - 1)) * W +
                                      clampi(x + dx, 0, W - 1);
                            win[s] = ((uint64_t)key_at(base, si, dtype) << 32) | (uint64_t)s;
                            s++;
                        }
                /* entries are distinct (slot s breaks key ties); the winner's
                 * slot gives back its source voxel */
                uint64_t best = select_rank(win, (int)n, (int)((n - 1) / 2));
                int bs = (int)(best & 0xffffffffu);
                int dz = bs / (k * k) - r, dy = (bs / k) % k - r, dx = bs % k - r;
                long si = ((long)clampi(z + dz, 0, D - 1) * H + clampi(y + dy, 0, H - 1)) * W +
                          clampi(x + dx, 0, W - 1);
                long o = (long)v * vol + ((long)z * H + y) * W + x;
                memcpy((char *)dst + (size_t)o * es, base + (size_t)si * es, es);
            }
        }
        free(win);
    }
    return 0;
}

/* Gradient of the filter: grad_in = 0, then for every plane and every
 * output q in row-major order, grad_in[idx[q]] += grad_out[q] (f32). */
int or_median_backward(const float *grad_out, const int32_t *idx, float *grad_in,
                       int H, int W, int C)
{
    if (H < 1 || W < 1 || C < 1) return -1;
    long plane_elems = (long)H * W;
    for (long i = 0; i < (long)C * plane_elems; i++) grad_in[i] = 0.0f;
    for (int c = 0; c < C; c++) {
        const float *g = grad_out + (size_t)c * plane_elems;
        const int32_t *ix = idx + (size_t)c * plane_elems;
        float *gi = grad_in + (size_t)c * plane_elems;
        for (long q = 0; q < plane_elems; q++) {
            if (ix[q] < 0 || ix[q] >= plane_elems) return -1;
            gi[ix[q]] += g[q];
        }
    }
    return 0;
}

int or_max_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}
