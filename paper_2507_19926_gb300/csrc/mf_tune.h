// Tuning table: which variant (and data-aware root tile) runs fastest per
// (k, dtype, argmedian, image-size bucket) on the current device.
#pragma once

namespace mf {

// MF_AUTO when nothing is recorded.
int tune_lookup(int k, int dtype, bool arg);
// Data-aware: the root tile; data-oblivious: the configuration index
// (0 = default).  0 when nothing is recorded.
int tune_tile(int k, int dtype, bool arg);
void tune_record(int k, int dtype, bool arg, int variant, int tile, float ms);

}  // namespace mf
