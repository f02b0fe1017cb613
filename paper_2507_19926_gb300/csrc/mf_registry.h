// Kernel registry shared by the C-ABI layer and the generated instantiations.
#pragma once
#include "mf_common.cuh"

namespace mf {

typedef int (*ImgLaunchFn)(const ImgArgs &a, int channels, cudaStream_t s);
// Persistent launch over a device work list (see o1_persistent).
typedef int (*PersistFn)(const ImgArgs *imgs, const int4 *items, int n_items, unsigned *counter,
                         int blocks_per_sm, int sms, cudaStream_t s, int *grid_out);

// One data-oblivious kernel instantiation (generated list).
struct O1Entry {
    int k;
    int dtype;
    int arg;        // 1: argmedian (composite records)
    int tw, th;     // root tile
    int bx, by;     // threads per block (x, y)
    int lanes;      // root tiles a thread (2: two 16-bit keys a register)
    int run;        // root tiles of a lane side by side along x (wide direct form), else 1
    int net_ops;    // min/max ops of one root tile's network (excl. column sort)
    ImgLaunchFn launch;
    PersistFn persist;
    const char *name;
};

extern const O1Entry kO1Entries[];
extern const int kO1Count;

// The configuration a call runs for (k, dtype, argmedian): the one the
// tuning table selects, else the default (for an image filtered on its
// own, `alone`, a size-aware default at k = 3, 5).  bucket: size bucket of
// the image (size_bucket in mf_tune.h), -1 unknown.
const O1Entry *find_o1(int k, int dtype, bool arg, int bucket = -1, bool alone = false);
const O1Entry *find_o1_nth(int k, int dtype, bool arg, int nth);

// Data-aware variant (mf_data_aware.cu).
int d1_supported(int k, int dtype, bool arg);
// kh: window height for a k-wide, kh-high window (0: k x k)
int d1_launch(const ImgArgs &a, int channels, int k, int dtype, int tile, cudaStream_t s, int kh = 0);
int d1_default_tile(int k, int dtype, bool arg, int kh = 0, int bucket = -1);
// The root tile of the paper's heuristic (no tuning table): 0 if none fits.
int d1_heuristic_tile(int k, int dtype, bool arg, int kh = 0);
// The configuration to run on image a: e itself, unless e is a wide form
// (vector row loads) and a's rows are not 16-byte aligned, where the first
// configuration of the same (k, dtype) that reads element by element runs.
const O1Entry *o1_for_image(const O1Entry *e, const ImgArgs &a);
int d1_supported_tile(int k, int dtype, bool arg, int tile, int kh = 0);
int d1_describe(int k, int dtype, bool arg, int tile, char *buf, size_t n);
void d1_release_all();
void d3_release_all();  // volumetric plans (mf_volume.cu)
// Persistent data-aware launch over a device work list for (k, dtype); the
// block geometry is the plan d1_geometry reports.
// tile_in: the root tile (0: the default for an image of unknown size).
int d1_geometry(int k, int dtype, bool arg, int tile_in, int *tile, int *strip, int *threads);
// n_items == 0 prepares (plan upload, attributes) and returns the blocks
// per SM in *grid_out; call that outside stream capture.
int d1_persist(const ImgArgs *imgs, const int4 *items, int n_items, unsigned *counter, int k, int dtype,
               int tile, int blocks_per_sm, int sms, cudaStream_t s, int *grid_out);

// Argmedian from medians already in a.dst (mf_argmedian.cu).
int launch_argmedian_from_values(const ImgArgs &a, int channels, int k, int dtype, cudaStream_t s);

// Identity argmedian for k = 1 and small helpers (mf_api.cu).
int launch_identity_idx(const ImgArgs &a, int channels, cudaStream_t s);

// Backward (mf_backward.cu).
int bwd_atomic(const float *g, const int32_t *idx, float *gi, int H, int W, size_t pitch,
               size_t idx_pitch, int C, cudaStream_t s);
int bwd_ordered(const float *g, const int32_t *idx, float *gi, int H, int W, size_t pitch,
               size_t idx_pitch, int C, int k, cudaStream_t s);

void set_error(const char *fmt, ...);

// Variant the plain entry point would run for (k, dtype): MF_OBLIVIOUS (and
// its entry) or MF_DATA_AWARE; negative status if neither exists.
// *tile (optional) receives the data-aware root tile.
int resolve_variant(int k, int dtype, bool arg, int variant, const O1Entry **o1, int bucket = -1,
                    int *tile = nullptr);

}  // namespace mf
