/*
 * Volumetric k x k x k median filter by hierarchical tiling -- C ABI.
 *
 * The paper (arXiv 2507.19926) names the extension of hierarchical tiling to
 * 3D as future work (Sec. 7.2), for the volumetric medians of medical
 * imaging.  These entry points build that extension with the data-aware
 * variant (Sec. 5): every list length of a k x k x k window's tree depends
 * only on (k, root tile), so the tree of sorts and merges is planned once on
 * the host and executed by one thread block per root tile out of shared
 * memory.  Types, status codes and conventions are those of medianfilter.h.
 */
#ifndef MEDIANFILTER_VOLUME_H
#define MEDIANFILTER_VOLUME_H

#include "medianfilter.h"

#ifdef __cplusplus
extern "C" {
#endif

/* Volumetric k x k x k median (paper Sec. 7.2 names the extension of
 * hierarchical tiling to 3D as future work, for medical volumes).
 * out(z, y, x) is the element of 0-based rank (k^3 - 1)/2 of the k^3 values
 * src(clamp(z+dz), clamp(y+dy), clamp(x+dx)), dz, dy, dx in [-(k-1)/2,
 * (k-1)/2], clamped to the edge on every axis, ordered as in
 * mf_median_filter (f32 by the sign-flip key); the winner is copied bit for
 * bit.  MF_AUTO of mf_median_filter_3d_ex: the data-oblivious network
 * where one is built (k = 3, 5), else the data-aware variant (Sec. 5) on
 * T x T x T root tiles of voxels: one thread block keeps a strip of tiles'
 * footprint and its whole tree of sorted lists in shared memory.
 *   src, dst: device, caller-owned, not aliasing; `volumes` volumes of D
 *             slices of H rows of W elements; row r of slice z of volume v
 *             at base + ((v*D + z)*H + r)*pitch.
 *   pitch:    bytes between rows, a multiple of the element size, >= W*size.
 *   k:        odd, 1..19 (k = 1 copies).
 * Asynchronous on `stream`.  Errors: MF_ERR_ARG (k, sizes), MF_ERR_PITCH,
 * MF_ERR_ALIAS, MF_ERR_DTYPE, MF_ERR_UNSUPPORTED (no plan fits shared
 * memory), MF_ERR_ALLOC (plan upload), MF_ERR_CUDA; nothing is launched on
 * an error. */
int mf_median_filter_3d(const void *src, void *dst, int D, int H, int W, size_t pitch, int volumes,
                        mf_dtype dtype, int k, mf_stream_t stream);

/* As mf_median_filter_3d with a choice of variant: MF_DATA_AWARE runs the
 * data-aware plan above (every k); MF_OBLIVIOUS a generated min/max network
 * of the same tree held in registers, one thread per 2 x 2 x 2 tile (the
 * data-oblivious variant of Sec. 4 in 3D; built for k = 3 and 5, else
 * MF_ERR_UNSUPPORTED); MF_AUTO the network where one is built and the grid
 * fits, else the data-aware plan.  Bad variant: MF_ERR_ARG. */
int mf_median_filter_3d_ex(const void *src, void *dst, int D, int H, int W, size_t pitch, int volumes,
                           mf_dtype dtype, int k, mf_variant variant, mf_stream_t stream);

/* One line describing the plan mf_median_filter_3d runs for (k, dtype):
 * root tile, threads per block, shared memory, phases, tasks, merged and
 * sorted elements per voxel.  Host only; written to buf (n bytes). */
int mf_median_filter_3d_describe(int k, mf_dtype dtype, char *buf, size_t n);

/* Host-side check of the volumetric schedule: builds the plan for a
 * k x k x k window and a strip of `strip` root tiles of tile^3 voxels side
 * by side along x and, if footprint and medians are non-NULL, runs it on
 * the CPU for one footprint of F = tile + k - 1 voxels in y and z and
 * FX = strip*tile + k - 1 in x (64-bit order keys, element (fx, fy, fz) at
 * (fy*FX + fx)*F + fz, clamped by the caller), writing the strip's
 * strip*tile x tile x tile medians in (z, y, x) order.  stats: NULL or 7
 * ints as for mf_d1_plan_check.  No GPU is used.  MF_ERR_UNSUPPORTED when
 * no plan exists. */
int mf_d3_plan_check(int k, int tile, int strip, const uint64_t *footprint, uint64_t *medians, int *stats);

/* As mf_d3_plan_check for the plan the kernel builds for keys of key_bytes
 * bytes (1: 8-bit data, 2: 16-bit data, 4: 32-bit data) run by blocks of
 * `threads` threads (256, 512 or 1024), which select its merge chunks
 * (mf_d3_plan_check plans for 4-byte keys and 256 threads).  The footprint
 * still holds 64-bit keys.  MF_ERR_ARG for other key widths or block
 * sizes. */
int mf_d3_plan_check_ex(int k, int tile, int strip, int key_bytes, int threads, const uint64_t *footprint,
                        uint64_t *medians, int *stats);

#ifdef __cplusplus
}
#endif

#endif /* MEDIANFILTER_VOLUME_H */
