// Autotuner: times the instantiated candidates of one (k, dtype) on an
// image of the caller's on the current device with CUDA events and records
// the fastest for that image's size bucket.  The paper picks its block
// shape per kernel size and data type by measurement (Sec. 4.3); here the
// choice covers the variant (Sec. 4 vs Sec. 5), the data-oblivious
// configuration (network form, tile, block shape, key width) and the
// data-aware root tile, per image-size bucket (small images favour other
// block shapes and tiles than large ones: fewer blocks than SMs, tails).
// The table can be persisted as JSON (MF_TUNE_CACHE), keyed by GPU name and
// SM count.
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <tuple>
#include <vector>

#include "mf_registry.h"
#include "mf_tune.h"

namespace mf {

struct TuneVal {
    int variant;
    int tile;
    float ms;
};

typedef std::tuple<int, int, int, int> TuneKey;  // k, dtype, arg, size bucket
static std::mutex g_mu;
static std::map<TuneKey, TuneVal> *g_table = new std::map<TuneKey, TuneVal>();
static bool g_loaded = false;

int size_bucket(long long pixels) {
    if (pixels < 1) return -1;
    int l = 0;
    while ((2ll << l) <= pixels) l++;  // floor(log2(pixels))
    int b = l / 2;
    return b < 7 ? 7 : (b > 12 ? 12 : b);
}

static std::string device_key() {
    int dev = 0;
    cudaDeviceProp p;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaGetDeviceProperties(&p, dev) != cudaSuccess) {
        cudaGetLastError();
        return "unknown";
    }
    char buf[300];
    snprintf(buf, sizeof buf, "%s/%d", p.name, p.multiProcessorCount);
    for (char *c = buf; *c; c++)
        if (*c == '"' || *c == '\\') *c = '_';
    return buf;
}

// Cache file format: one JSON object per line,
// {"device": "...", "k": K, "dtype": D, "arg": A, "bucket": B, "variant": V, "tile": T, "ms": M}
static void load_locked() {
    if (g_loaded) return;
    g_loaded = true;
    const char *path = getenv("MF_TUNE_CACHE");
    if (!path) return;
    FILE *f = fopen(path, "r");
    if (!f) return;
    const std::string dk = device_key();
    char line[1024], dev[400];
    while (fgets(line, sizeof line, f)) {
        int k, dt, arg, bucket, var, tile;
        float ms;
        if (sscanf(line,
                   " {\"device\": \"%399[^\"]\", \"k\": %d, \"dtype\": %d, \"arg\": %d, \"bucket\": %d, \"variant\": %d, "
                   "\"tile\": %d, \"ms\": %f",
                   dev, &k, &dt, &arg, &bucket, &var, &tile, &ms) == 8 &&
            dk == dev)
            (*g_table)[std::make_tuple(k, dt, arg, bucket)] = TuneVal{var, tile, ms};
    }
    fclose(f);
}

// The entry of the bucket nearest to `bucket` (ties: the larger bucket; an
// unknown size: the largest bucket), or nullptr.
static const TuneVal *nearest_locked(int k, int dtype, bool arg, int bucket) {
    load_locked();
    const TuneVal *best = nullptr;
    int best_d = 1 << 30, best_b = -1;
    for (auto it = g_table->lower_bound(std::make_tuple(k, dtype, arg ? 1 : 0, -1000));
         it != g_table->end() && std::get<0>(it->first) == k && std::get<1>(it->first) == dtype &&
         std::get<2>(it->first) == (arg ? 1 : 0);
         ++it) {
        const int b = std::get<3>(it->first);
        const int d = bucket < 0 ? -b : (b > bucket ? b - bucket : bucket - b);
        if (d < best_d || (d == best_d && b > best_b)) {
            best = &it->second;
            best_d = d;
            best_b = b;
        }
    }
    return best;
}

int tune_lookup(int k, int dtype, bool arg, int bucket) {
    std::lock_guard<std::mutex> lk(g_mu);
    const TuneVal *v = nearest_locked(k, dtype, arg, bucket);
    return v ? v->variant : MF_AUTO;
}

int tune_tile(int k, int dtype, bool arg, int bucket) {
    std::lock_guard<std::mutex> lk(g_mu);
    const TuneVal *v = nearest_locked(k, dtype, arg, bucket);
    return v ? v->tile : 0;
}

bool tune_has(int k, int dtype, bool arg, int bucket) {
    std::lock_guard<std::mutex> lk(g_mu);
    load_locked();
    return g_table->count(std::make_tuple(k, dtype, arg ? 1 : 0, bucket)) != 0;
}

void tune_record(int k, int dtype, bool arg, int bucket, int variant, int tile, float ms) {
    std::lock_guard<std::mutex> lk(g_mu);
    load_locked();
    (*g_table)[std::make_tuple(k, dtype, arg ? 1 : 0, bucket)] = TuneVal{variant, tile, ms};
    const char *path = getenv("MF_TUNE_CACHE");
    if (!path) return;
    FILE *f = fopen(path, "a");
    if (!f) return;
    fprintf(f,
            "{\"device\": \"%s\", \"k\": %d, \"dtype\": %d, \"arg\": %d, \"bucket\": %d, \"variant\": %d, "
            "\"tile\": %d, \"ms\": %.6f}\n",
            device_key().c_str(), k, dtype, arg ? 1 : 0, bucket, variant, tile, ms);
    fclose(f);
}

// One candidate: the data-oblivious configuration o1, else the data-aware
// root tile.
struct Cand {
    const O1Entry *o1;
    int tile;
};

static int launch_cand(const Cand &c, const ImgArgs &a, int C, int k, int dtype, cudaStream_t s) {
    if (c.o1) return c.o1->launch(a, C, s);
    return d1_launch(a, C, k, dtype, c.tile, s);
}

// Best of three timings (after a warm-up) of the candidate on `copies`
// images at once: copy r reads a's input and writes dsts[r], each on its
// own stream, all forked from and joined back to s.  copies = 1 times one
// launch (latency); more copies of a small image fill the GPU the way a
// batch's concurrent classes do (throughput).  Returns ms per image.
static float time_cand(const Cand &c, const ImgArgs &a, int C, int k, int dtype, cudaStream_t s, int copies,
                       char *const *dsts, const cudaStream_t *streams, cudaEvent_t fork, cudaEvent_t *joins,
                       int *rc) {
    auto run = [&]() {
        int r0 = MF_OK;
        if (copies == 1) return launch_cand(c, a, C, k, dtype, s);
        cudaEventRecord(fork, s);
        for (int r = 0; r < copies; r++) {
            cudaStreamWaitEvent(streams[r], fork, 0);
            ImgArgs ar = a;
            ar.dst = dsts[r];
            const int rr = launch_cand(c, ar, C, k, dtype, streams[r]);
            if (rr != MF_OK) r0 = rr;
            cudaEventRecord(joins[r], streams[r]);
            cudaStreamWaitEvent(s, joins[r], 0);
        }
        return r0;
    };
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    *rc = run();  // warm-up (also sets kernel attributes, uploads plans)
    float best = 1e30f;
    for (int rep = 0; rep < 3 && *rc == MF_OK; rep++) {
        cudaEventRecord(e0, s);
        *rc = run();
        cudaEventRecord(e1, s);
        cudaEventSynchronize(e1);
        float ms = 0;
        cudaEventElapsedTime(&ms, e0, e1);
        if (ms < best) best = ms;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    return best / (float)copies;
}

// Times every candidate of (k, dtype) on the image (src, dst), `copies` at
// a time (see time_cand), and records the fastest for the image's bucket.
static int tune_image(const void *src, void *dst, int H, int W, size_t pitch, int channels, int dtype, int k,
                      cudaStream_t s, int copies) {
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
    std::vector<char *> dsts(copies, (char *)dst);
    std::vector<cudaStream_t> streams;
    std::vector<cudaEvent_t> joins;
    cudaEvent_t fork = nullptr;
    void *scratch = nullptr;
    const size_t bytes = (size_t)channels * H * pitch;
    int rc = MF_OK;
    if (copies > 1) {  // copy r > 0 writes scratch image r - 1
        if (dev_alloc(&scratch, bytes * (copies - 1)) != cudaSuccess) {
            cudaGetLastError();
            set_error("autotune: cannot allocate %zu bytes of scratch", bytes * (copies - 1));
            return MF_ERR_ALLOC;
        }
        for (int r = 1; r < copies; r++) dsts[r] = (char *)scratch + bytes * (r - 1);
        streams.resize(copies);
        joins.resize(copies);
        cudaEventCreateWithFlags(&fork, cudaEventDisableTiming);
        for (int r = 0; r < copies; r++) {
            cudaStreamCreateWithFlags(&streams[r], cudaStreamNonBlocking);
            cudaEventCreateWithFlags(&joins[r], cudaEventDisableTiming);
        }
    }
    float best = 1e30f, def_ms = 1e30f;
    int best_var = 0, best_tile = 0;
    // the choice without a table entry: the first network configuration
    // (the element-by-element one for unaligned rows), else the heuristic
    // data-aware tile; a candidate must beat it by 5% to replace it, so
    // that timing noise does not trade good defaults for equal ones
    const O1Entry *o1_def = o1_for_image(find_o1_nth(k, dtype, false, 0), a);
    const int d1_def = o1_def ? 0 : d1_heuristic_tile(k, dtype, false);
    int def_var = o1_def ? MF_OBLIVIOUS : MF_DATA_AWARE, def_tile = 0;
    const bool verbose = getenv("MF_TUNE_VERBOSE") != nullptr;
    for (int nth = 0;; nth++) {
        const O1Entry *o1 = find_o1_nth(k, dtype, false, nth);
        if (!o1) break;
        int r;
        const float ms = time_cand(Cand{o1, 0}, a, channels, k, dtype, s, copies, dsts.data(), streams.data(), fork,
                                   joins.data(), &r);
        if (verbose) fprintf(stderr, "mf_autotune k=%d dtype=%d x%d %s: %.4f ms (rc %d)\n", k, dtype, copies, o1->name, ms, r);
        if (r == MF_OK && ms < best) { best = ms; best_var = MF_OBLIVIOUS; best_tile = nth; }
        if (r == MF_OK && o1 == o1_def) { def_ms = ms; def_tile = nth; }
    }
    if (d1_supported(k, dtype, false)) {
        for (int tile = 2; tile <= 32; tile *= 2) {
            if (!d1_supported_tile(k, dtype, false, tile)) continue;
            int r;
            const float ms = time_cand(Cand{nullptr, tile}, a, channels, k, dtype, s, copies, dsts.data(),
                                       streams.data(), fork, joins.data(), &r);
            if (verbose) fprintf(stderr, "mf_autotune k=%d dtype=%d x%d data-aware tile %d: %.4f ms (rc %d)\n", k, dtype, copies, tile, ms, r);
            if (r == MF_OK && ms < best) { best = ms; best_var = MF_DATA_AWARE; best_tile = tile; }
            if (r == MF_OK && !o1_def && tile == d1_def) { def_ms = ms; def_tile = tile; }
        }
    }
    if (best_var && def_ms < 1e29f && !(best < 0.95f * def_ms)) {  // keep the default
        best = def_ms;
        best_var = def_var;
        best_tile = def_tile;
    }
    cudaError_t e = cudaStreamSynchronize(s);
    if (e == cudaSuccess) e = cudaGetLastError();
    for (cudaStream_t st : streams) cudaStreamDestroy(st);
    for (cudaEvent_t ev : joins) cudaEventDestroy(ev);
    if (fork) cudaEventDestroy(fork);
    if (scratch) cudaFree(scratch);
    if (e != cudaSuccess) { set_error("autotune: %s", cudaGetErrorString(e)); return MF_ERR_CUDA; }
    if (best_var == 0) { set_error("no candidate for k=%d dtype=%d", k, dtype); return MF_ERR_UNSUPPORTED; }
    tune_record(k, dtype, false, size_bucket((long long)H * W), best_var, best_tile, best);
    return rc;
}

int tune_for_batch(const void *src, void *dst, int H, int W, size_t pitch, int channels, int dtype, int k) {
    // enough concurrent copies for about 8 M output pixels, at most 32
    const long long px = (long long)H * W * channels;
    long long copies = (8ll << 20) / (px > 0 ? px : 1);
    if (copies < 1) copies = 1;
    if (copies > 32) copies = 32;
    return tune_image(src, dst, H, W, pitch, channels, dtype, k, nullptr, (int)copies);
}

}  // namespace mf

using namespace mf;

extern "C" int mf_autotune(const void *src, void *dst, int H, int W, size_t pitch, int channels,
                           mf_dtype dtype, int k, mf_stream_t stream) {
    if (!src || !dst || H < 1 || W < 1 || channels < 1 || k < 3 || k > 75 || !(k & 1)) {
        set_error("bad autotune arguments");
        return MF_ERR_ARG;
    }
    return tune_image(src, dst, H, W, pitch, channels, (int)dtype, k, (cudaStream_t)stream, 1);
}
