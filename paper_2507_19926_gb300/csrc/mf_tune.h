// Tuning table: which variant (and data-aware root tile, or data-oblivious
// configuration) runs fastest per (k, dtype, argmedian, image-size bucket)
// on the current device.
#pragma once

namespace mf {

// Size bucket of a plane of `pixels` elements: floor(log2(pixels) / 2),
// clamped to 7..12 (a quarter of a decade of pixels: up to 181^2, 256^2 ..
// 512^2, .., 2048^2 .. 4096^2, larger).  -1 stands for an unknown size.
int size_bucket(long long pixels);

// The entry for (k, dtype, arg) in `bucket`, else in the nearest bucket
// that has one (an unknown size takes the largest); MF_AUTO when nothing is
// recorded.
int tune_lookup(int k, int dtype, bool arg, int bucket = -1);
// Data-aware: the root tile; data-oblivious: the configuration index
// (0 = default).  0 when nothing is recorded.
int tune_tile(int k, int dtype, bool arg, int bucket = -1);
// True when (k, dtype, arg, bucket) itself has an entry.
bool tune_has(int k, int dtype, bool arg, int bucket);
void tune_record(int k, int dtype, bool arg, int bucket, int variant, int tile, float ms);
// Tunes (k, dtype) for the bucket of an H x W image by throughput: each
// candidate runs on enough concurrent copies of the image (scratch outputs,
// allocated here) to fill the GPU, as the classes of a batch do.  dst is
// written.  Synchronises.
int tune_for_batch(const void *src, void *dst, int H, int W, size_t pitch, int channels, int dtype, int k);

}  // namespace mf
