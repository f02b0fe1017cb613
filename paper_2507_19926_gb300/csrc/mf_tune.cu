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

static float time_ms(int (*fn)(void *), void *ctx, cudaStream_t s, int *rc) {
    cudaEvent_t a, b;
    cudaEventCreate(&a);
    cudaEventCreate(&b);
    *rc = fn(ctx);  // warm-up (also sets kernel attributes)
    float best = 1e30f;
    for (int rep = 0; rep < 3 && *rc == MF_OK; rep++) {
        cudaEventRecord(a, s);
        *rc = fn(ctx);
        cudaEventRecord(b, s);
        cudaEventSynchronize(b);
        float ms = 0;
        cudaEventElapsedTime(&ms, a, b);
        if (ms < best) best = ms;
    }
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    return best;
}

struct Cand {
    const ImgArgs *a;
    int C, k, dtype, tile;
    const O1Entry *o1;
    cudaStream_t s;
};

static int run_cand(void *p) {
    Cand *c = (Cand *)p;
    if (c->o1) return c->o1->launch(*c->a, c->C, c->s);
    return d1_launch(*c->a, c->C, c->k, c->dtype, c->tile, c->s);
}

}  // namespace mf

using namespace mf;

extern "C" int mf_autotune(const void *src, void *dst, int H, int W, size_t pitch, int channels,
                           mf_dtype dtype, int k, mf_stream_t stream) {
    if (!src || !dst || H < 1 || W < 1 || channels < 1 || k < 3 || k > 75 || !(k & 1)) {
        set_error("bad autotune arguments");
        return MF_ERR_ARG;
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
    cudaStream_t s = (cudaStream_t)stream;
    float best = 1e30f;
    int best_var = 0, best_tile = 0;
    const bool verbose = getenv("MF_TUNE_VERBOSE") != nullptr;
    for (int nth = 0;; nth++) {
        const O1Entry *o1 = find_o1_nth(k, dtype, false, nth);
        if (!o1) break;
        Cand c{&a, channels, k, dtype, 0, o1, s};
        int rc;
        float ms = time_ms(run_cand, &c, s, &rc);
        if (verbose) fprintf(stderr, "mf_autotune k=%d dtype=%d %s: %.4f ms (rc %d)\n", k, (int)dtype, o1->name, ms, rc);
        if (rc == MF_OK && ms < best) { best = ms; best_var = MF_OBLIVIOUS; best_tile = nth; }
    }
    if (d1_supported(k, dtype, false)) {
        for (int tile = 2; tile <= 32; tile *= 2) {
            if (!d1_supported_tile(k, dtype, false, tile)) continue;
            Cand c{&a, channels, k, dtype, tile, nullptr, s};
            int rc;
            float ms = time_ms(run_cand, &c, s, &rc);
            if (verbose) fprintf(stderr, "mf_autotune k=%d dtype=%d data-aware tile %d: %.4f ms (rc %d)\n", k, (int)dtype, tile, ms, rc);
            if (rc == MF_OK && ms < best) { best = ms; best_var = MF_DATA_AWARE; best_tile = tile; }
        }
    }
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) { set_error("autotune: %s", cudaGetErrorString(e)); return MF_ERR_CUDA; }
    if (best_var == 0) { set_error("no candidate for k=%d dtype=%d", k, (int)dtype); return MF_ERR_UNSUPPORTED; }
    tune_record(k, dtype, false, size_bucket((long long)H * W), best_var, best_tile, best);
    return MF_OK;
}
