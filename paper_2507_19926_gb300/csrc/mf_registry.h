// Kernel registry shared by the C-ABI layer and the generated instantiations.
#pragma once
#include "mf_common.cuh"

namespace mf {

typedef int (*ImgLaunchFn)(const ImgArgs &a, int channels, cudaStream_t s);

// One data-oblivious kernel instantiation (generated list).
struct O1Entry {
    int k;
    int dtype;
    int arg;        // 1: argmedian (composite records)
    int tw, th;     // root tile
    int bx, by;     // threads per block (x, y)
    int net_ops;    // min/max ops of one root tile's network (excl. column sort)
    ImgLaunchFn launch;
    const char *name;
};

extern const O1Entry kO1Entries[];
extern const int kO1Count;

const O1Entry *find_o1(int k, int dtype, bool arg);

// Data-aware variant (mf_data_aware.cu).
int d1_supported(int k, int dtype, bool arg);
int d1_launch(const ImgArgs &a, int channels, int k, int dtype, int tile, cudaStream_t s);
int d1_default_tile(int k, int dtype, bool arg);
int d1_supported_tile(int k, int dtype, bool arg, int tile);
int d1_describe(int k, int dtype, bool arg, int tile, char *buf, size_t n);
void d1_release_all();

// Identity argmedian for k = 1 and small helpers (mf_api.cu).
int launch_identity_idx(const ImgArgs &a, int channels, cudaStream_t s);

// Backward (mf_backward.cu).
int bwd_atomic(const float *g, const int32_t *idx, float *gi, int H, int W, size_t pitch,
               size_t idx_pitch, int C, cudaStream_t s);
int bwd_gather(const float *g, const int32_t *idx, float *gi, int H, int W, size_t pitch,
               size_t idx_pitch, int C, int k, cudaStream_t s);

void set_error(const char *fmt, ...);

}  // namespace mf
