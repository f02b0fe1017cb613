// Batched persistent launch: many images of uneven sizes, dtypes and k in
// one CUDA-graph launch with device-side work queues.
//
// Images are grouped into kernel classes -- the (variant, k, dtype) that the
// plain entry point would run.  Each class gets one persistent kernel whose
// blocks claim (image, block x, block y, plane) work items from a device
// counter (atomicAdd; no block ever waits on another) until the class's
// list is exhausted; items are ordered largest image first so the tail of
// the queue is short.  All classes are captured as independent branches of
// one CUDA graph, so a run is a single cudaGraphLaunch and the classes run
// concurrently.  One kernel per class (instead of one kernel switching over
// all classes) keeps every class at its own register count and occupancy:
// the largest networks need all 255 registers of a thread, which would
// otherwise throttle every small-k class too.
#include <algorithm>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <map>
#include <tuple>
#include <vector>

#include "mf_registry.h"
#include "mf_tune.h"

struct mf_batch_plan {
    int n = 0;
    std::vector<mf_image_desc> descs;
    void *dmem = nullptr;          // device: ImgArgs[n] | counters | items
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    std::vector<cudaStream_t> streams;
    std::vector<cudaEvent_t> events;
    int kernels = 0;               // kernel launches per run
    int copies = 0;                // k = 1 copies per run
    long long items = 0;
};

namespace mf {

static int esz(int dtype) { return dtype == MF_U8 ? 1 : dtype == MF_U16 ? 2 : (dtype == MF_U32 || dtype == MF_F32) ? 4 : 0; }

struct BatchClass {
    int variant;
    const O1Entry *o1;
    int k, dtype;
    int tile;    // data-aware root tile
    int rw, rh;  // pixels covered by one work item (block region)
    int bps;     // resident blocks per SM of its persistent kernel
    std::vector<int4> items;
};

static void destroy_plan(mf_batch_plan *p) {
    if (!p) return;
    if (p->exec) cudaGraphExecDestroy(p->exec);
    if (p->graph) cudaGraphDestroy(p->graph);
    for (cudaEvent_t e : p->events) cudaEventDestroy(e);
    for (cudaStream_t s : p->streams) cudaStreamDestroy(s);
    if (p->dmem) cudaFree(p->dmem);
    delete p;
}

}  // namespace mf

using namespace mf;

extern "C" int mf_batch_plan_create(const mf_image_desc *descs, int n, mf_batch_plan **out) {
    return mf_batch_plan_create_ex(descs, n, 0, out);
}

extern "C" int mf_batch_plan_create_ex(const mf_image_desc *descs, int n, int tune, mf_batch_plan **out) {
    if (!out) { set_error("null output"); return MF_ERR_ARG; }
    *out = nullptr;
    if (!descs || n < 1) { set_error("empty batch"); return MF_ERR_ARG; }
    // validate every descriptor first
    for (int i = 0; i < n; i++) {
        const mf_image_desc &d = descs[i];
        const int es = esz(d.dtype);
        if (!es) { set_error("image %d: unknown dtype", i); return MF_ERR_DTYPE; }
        if (d.k < 1 || d.k > 31 || !(d.k & 1)) { set_error("image %d: k must be odd in 1..31", i); return MF_ERR_ARG; }
        if (d.H < 1 || d.W < 1 || d.channels < 1 || d.channels > 65535 || !d.src || !d.dst) {
            set_error("image %d: bad shape or pointer", i);
            return MF_ERR_ARG;
        }
        if (d.pitch < (size_t)d.W * es || d.pitch % es) { set_error("image %d: bad pitch", i); return MF_ERR_PITCH; }
        const size_t bytes = (size_t)d.channels * d.H * d.pitch;
        const char *a = (const char *)d.src, *b = (const char *)d.dst;
        if (a < b + bytes && b < a + bytes) { set_error("image %d: src and dst overlap", i); return MF_ERR_ALIAS; }
    }
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
        set_error("no CUDA device: %s", cudaGetErrorString(cudaGetLastError()));
        return MF_ERR_CUDA;
    }
    // tuning: every (k, dtype, size bucket) of the batch without an entry is
    // timed on the largest image of that group, by throughput (concurrent
    // copies, as the batch's classes run concurrently); the candidates
    // write that image's dst, which every run overwrites
    if (tune) {
        std::map<std::tuple<int, int, int>, int> rep;  // (k, dtype, bucket) -> largest image
        for (int i = 0; i < n; i++) {
            const mf_image_desc &d = descs[i];
            if (d.k < 3) continue;
            const int b = size_bucket((long long)d.H * d.W);
            if (tune_has(d.k, d.dtype, false, b)) continue;
            auto key = std::make_tuple(d.k, (int)d.dtype, b);
            auto it = rep.find(key);
            if (it == rep.end() || (long long)d.H * d.W * d.channels >
                                       (long long)descs[it->second].H * descs[it->second].W * descs[it->second].channels)
                rep[key] = i;
        }
        for (auto &kv : rep) {
            const mf_image_desc &d = descs[kv.second];
            const int rc = tune_for_batch(d.src, d.dst, d.H, d.W, d.pitch, d.channels, d.dtype, d.k);
            if (rc != MF_OK) return rc;
        }
        if (cudaDeviceSynchronize() != cudaSuccess) {
            set_error("batch tuning: %s", cudaGetErrorString(cudaGetLastError()));
            return MF_ERR_CUDA;
        }
    }
    mf_batch_plan *p = new mf_batch_plan();
    p->n = n;
    p->descs.assign(descs, descs + n);

    // classes and their work items, largest images first
    std::vector<int> order(n);
    for (int i = 0; i < n; i++) order[i] = i;
    std::stable_sort(order.begin(), order.end(), [&](int x, int y) {
        return (long long)descs[x].H * descs[x].W * descs[x].channels > (long long)descs[y].H * descs[y].W * descs[y].channels;
    });
    // one class per kernel: (variant, configuration or root tile, k, dtype);
    // the tuning table picks them per image-size bucket
    std::map<std::tuple<int, long long, int, int>, BatchClass> classes;
    std::vector<int> copies;
    for (int i : order) {
        const mf_image_desc &d = descs[i];
        if (d.k == 1) { copies.push_back(i); continue; }
        const O1Entry *o1 = nullptr;
        int tile = 0;
        const int var = resolve_variant(d.k, d.dtype, false, MF_AUTO, &o1, size_bucket((long long)d.H * d.W), &tile);
        if (var < 0) { destroy_plan(p); return var; }
        if (var == MF_OBLIVIOUS) {  // wide forms need 16-byte aligned rows
            ImgArgs t{};
            t.src = (const char *)d.src;
            t.dst = (char *)d.dst;
            t.pitch = d.pitch;
            o1 = o1_for_image(o1, t);
        }
        if (var == MF_OBLIVIOUS && !o1->persist) { set_error("no persistent form for k=%d", d.k); destroy_plan(p); return MF_ERR_UNSUPPORTED; }
        const long long which = var == MF_OBLIVIOUS ? (long long)(o1 - kO1Entries) : (long long)tile;
        auto key = std::make_tuple(var, which, d.k, (int)d.dtype);
        BatchClass &c = classes[key];
        if (c.items.empty()) {
            c.variant = var;
            c.o1 = o1;
            c.k = d.k;
            c.dtype = d.dtype;
            c.tile = tile;
            if (var == MF_OBLIVIOUS) {
                const int lanes = o1->lanes;
                c.rw = lanes * o1->bx * o1->tw * o1->run;
                c.rh = o1->by * o1->th;
            } else {
                int T, B, nt;
                if (d1_geometry(d.k, d.dtype, false, tile, &T, &B, &nt)) { set_error("no data-aware plan for k=%d", d.k); destroy_plan(p); return MF_ERR_UNSUPPORTED; }
                c.tile = T;
                c.rw = B * T;
                c.rh = T;
            }
        }
        const int gx = (d.W + c.rw - 1) / c.rw, gy = (d.H + c.rh - 1) / c.rh;
        for (int z = 0; z < d.channels; z++)
            for (int by = 0; by < gy; by++)
                for (int bx = 0; bx < gx; bx++) c.items.push_back(make_int4(i, bx, by, z));
    }

    if (getenv("MF_BATCH_VERBOSE")) {  // the plan's kernel classes, one line each
        for (auto &kv : classes) {
            const BatchClass &c = kv.second;
            const long long px = (long long)c.items.size() * c.rw * c.rh;
            fprintf(stderr, "batch class k=%d dtype=%d %s items=%zu region=%dx%d px~%lld\n", c.k, c.dtype,
                    c.variant == MF_OBLIVIOUS ? c.o1->name : "data-aware", c.items.size(), c.rw, c.rh, px);
            if (c.variant != MF_OBLIVIOUS) fprintf(stderr, "  data-aware tile %d\n", c.tile);
        }
    }
    // device memory: image arguments, one counter per class, the item lists
    const size_t nclass = classes.size();
    size_t nitems = 0;
    for (auto &kv : classes) nitems += kv.second.items.size();
    const size_t off_cnt = ((size_t)n * sizeof(ImgArgs) + 255) & ~(size_t)255;
    const size_t off_items = (off_cnt + nclass * sizeof(unsigned) + 255) & ~(size_t)255;
    const size_t total = off_items + nitems * sizeof(int4) + 16;
    if (dev_alloc(&p->dmem, total) != cudaSuccess) {
        cudaGetLastError();
        set_error("cannot allocate %zu bytes for the batch plan", total);
        destroy_plan(p);
        return MF_ERR_ALLOC;
    }
    std::vector<ImgArgs> args(n);
    for (int i = 0; i < n; i++) {
        const mf_image_desc &d = descs[i];
        ImgArgs &a = args[i];
        a.src = (const char *)d.src;
        a.dst = (char *)d.dst;
        a.idx = nullptr;
        a.H = d.H;
        a.y_lo = 0;
        a.y_hi = d.H - 1;
        a.W = d.W;
        a.pitch = d.pitch;
        a.plane = (size_t)d.H * d.pitch;
        a.idx_pitch = a.idx_plane = 0;
    }
    char *dm = (char *)p->dmem;
    cudaError_t e = cudaMemcpy(dm, args.data(), n * sizeof(ImgArgs), cudaMemcpyHostToDevice);
    std::vector<int4> all;
    all.reserve(nitems);
    std::vector<size_t> first;
    for (auto &kv : classes) {
        first.push_back(all.size());
        all.insert(all.end(), kv.second.items.begin(), kv.second.items.end());
    }
    if (e == cudaSuccess && !all.empty())
        e = cudaMemcpy(dm + off_items, all.data(), all.size() * sizeof(int4), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) {
        set_error("batch upload: %s", cudaGetErrorString(e));
        destroy_plan(p);
        return MF_ERR_CUDA;
    }
    p->items = (long long)nitems;

    // prepare every class outside the capture: plan uploads, kernel
    // attributes and occupancy are not stream work
    for (auto &kv : classes) {
        BatchClass &c = kv.second;
        int bps = 0, rc0;
        if (c.variant == MF_OBLIVIOUS) rc0 = c.o1->persist(nullptr, nullptr, 0, nullptr, 0, sms, nullptr, &bps);
        else rc0 = d1_persist(nullptr, nullptr, 0, nullptr, c.k, c.dtype, c.tile, 0, sms, nullptr, &bps);
        if (rc0 != MF_OK) {
            set_error("preparing the persistent kernel for k=%d dtype=%d: %s", c.k, c.dtype,
                      cudaGetErrorString(cudaGetLastError()));
            destroy_plan(p);
            return rc0;
        }
        c.bps = bps;
    }

    // capture: one branch per class (counter reset + persistent kernel),
    // plus device-to-device copies for k = 1 images
    cudaStream_t s0;
    if (cudaStreamCreateWithFlags(&s0, cudaStreamNonBlocking) != cudaSuccess) { set_error("stream"); destroy_plan(p); return MF_ERR_CUDA; }
    p->streams.push_back(s0);
    cudaEvent_t fork;
    cudaEventCreateWithFlags(&fork, cudaEventDisableTiming);
    p->events.push_back(fork);
    int rc = MF_OK;
    e = cudaStreamBeginCapture(s0, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) { set_error("begin capture: %s", cudaGetErrorString(e)); destroy_plan(p); return MF_ERR_CUDA; }
    cudaEventRecord(fork, s0);
    size_t ci = 0;
    for (auto &kv : classes) {
        BatchClass &c = kv.second;
        cudaStream_t si;
        cudaStreamCreateWithFlags(&si, cudaStreamNonBlocking);
        p->streams.push_back(si);
        cudaEvent_t join;
        cudaEventCreateWithFlags(&join, cudaEventDisableTiming);
        p->events.push_back(join);
        cudaStreamWaitEvent(si, fork, 0);
        unsigned *cnt = (unsigned *)(dm + off_cnt) + ci;
        const int4 *items = (const int4 *)(dm + off_items) + first[ci];
        cudaMemsetAsync(cnt, 0, sizeof(unsigned), si);
        int grid = 0;
        if (rc == MF_OK) {
            if (c.variant == MF_OBLIVIOUS)
                rc = c.o1->persist((const ImgArgs *)dm, items, (int)c.items.size(), cnt, c.bps, sms, si, &grid);
            else
                rc = d1_persist((const ImgArgs *)dm, items, (int)c.items.size(), cnt, c.k, c.dtype, c.tile, c.bps, sms,
                                si, &grid);
            if (rc != MF_OK)
                set_error("persistent launch for k=%d dtype=%d: %s", c.k, c.dtype, cudaGetErrorString(cudaGetLastError()));
        }
        p->kernels++;
        cudaEventRecord(join, si);
        cudaStreamWaitEvent(s0, join, 0);
        ci++;
    }
    for (int i : copies) {
        const mf_image_desc &d = descs[i];
        cudaMemcpy2DAsync(d.dst, d.pitch, d.src, d.pitch, (size_t)d.W * esz(d.dtype), (size_t)d.H * d.channels,
                          cudaMemcpyDeviceToDevice, s0);
        p->copies++;
    }
    e = cudaStreamEndCapture(s0, &p->graph);
    if (rc != MF_OK || e != cudaSuccess) {
        if (rc == MF_OK) set_error("end capture: %s", cudaGetErrorString(e));
        cudaGetLastError();
        destroy_plan(p);
        return rc != MF_OK ? rc : MF_ERR_CUDA;
    }
    e = cudaGraphInstantiate(&p->exec, p->graph, 0);
    if (e != cudaSuccess) {
        set_error("graph instantiate: %s", cudaGetErrorString(e));
        destroy_plan(p);
        return MF_ERR_CUDA;
    }
    *out = p;
    return MF_OK;
}

extern "C" int mf_batch_run(mf_batch_plan *plan, mf_stream_t stream) {
    if (!plan || !plan->exec) { set_error("null batch plan"); return MF_ERR_ARG; }
    cudaError_t e = cudaGraphLaunch(plan->exec, (cudaStream_t)stream);
    if (e != cudaSuccess) { set_error("graph launch: %s", cudaGetErrorString(e)); return MF_ERR_CUDA; }
    count_launch((unsigned)plan->kernels);
    return MF_OK;
}

extern "C" int mf_batch_plan_destroy(mf_batch_plan *plan) {
    destroy_plan(plan);
    return MF_OK;
}

extern "C" int mf_batch_describe(const mf_batch_plan *plan, int *kernels, long long *items) {
    if (!plan) { set_error("null batch plan"); return MF_ERR_ARG; }
    if (kernels) *kernels = plan->kernels;
    if (items) *items = plan->items;
    return MF_OK;
}
