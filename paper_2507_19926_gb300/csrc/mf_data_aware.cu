// Data-aware variant (paper Sec. 5), re-planned for sm_103a.
//
// The paper runs the recursion as a multi-pass pipeline of seven kernels
// over three streams with the per-level state in global memory (up to two
// orders of magnitude above the image size, Sec. 5.3 and 7.1).  Here one
// thread block owns one T x T root tile and keeps the whole state of its
// tree -- footprint, sorted columns, rows, cores -- in shared memory; the
// statically planned phases (mf_d1_plan.cu) replace the kernel boundaries
// with block barriers, so nothing but the image and the medians touches
// HBM.  Within a phase, small sorts run as register networks (one thread
// per list), merges as merge-path chunks (one thread per chunk) and the
// corner extensions of extra rows and columns as inserts (one thread per
// list).
#include <cstdio>
#include <map>
#include <mutex>
#include <tuple>

#include "d1_sortnets.cuh"
#include "mf_d1_ops.cuh"
#include "mf_registry.h"
#include "mf_tune.h"

namespace mf {

constexpr int D1_NT_MAX = 1024;
constexpr size_t D1_SMEM_BUDGET = 200 * 1024;
// A strip whose state fits in this much shared memory runs with 256
// threads, several blocks per SM; bigger ones run alone with 1024 threads.
constexpr size_t D1_SMEM_SMALL = 56 * 1024;

struct D1Dev {
    const D1Packed *items;  // one 16-byte record per work item, in work order
    const int32_t *phase_begin;
    const int32_t *out_off;
    int nphases;
    int k, kh, T, TH, B, FW, FH;  // window k columns by kh rows; root tile T columns by TH rows
};

template <class KT, int N>
__device__ __forceinline__ void d1_sort_task(KT *sm, const D1Item &t) {
    KT v[N];
    const KT S = d1_sentinel<KT>();
#pragma unroll
    for (int i = 0; i < N; i++) v[i] = i < t.a_len ? sm[t.a_off + i * t.a_stride] : S;
    SortNet<N>::run(v);
#pragma unroll
    for (int i = 0; i < N; i++)
        if (i < t.a_len) sm[t.out_off + i] = v[i];
    sm[t.out_off + t.a_len] = S;  // the list's sentinel slot (see d1_merge_item)
}

// NMAX: the longest sort of the plan, rounded up to a power of two; the
// kernel is instantiated per NMAX so that short plans do not pay for the
// registers of a 64-element network.
template <class KT, int NMAX>
__device__ __forceinline__ void d1_sort_any(KT *sm, const D1Item &t) {
    const int n = t.a_len;
    if (n <= 2) d1_sort_task<KT, 2>(sm, t);
    else if (n <= 4) d1_sort_task<KT, 4>(sm, t);
    else if (NMAX <= 8 || n <= 8) d1_sort_task<KT, (NMAX < 8 ? NMAX : 8)>(sm, t);
    else if (NMAX <= 16 || n <= 16) d1_sort_task<KT, (NMAX < 16 ? NMAX : 16)>(sm, t);
    else d1_sort_task<KT, (NMAX < 32 ? NMAX : 32)>(sm, t);
}

// Element keys of the footprint: the order key (value mode) or the record
// key << IB | footprint index (argmedian mode: equal keys then order by
// footprint row-major position, i.e. by window slot for every pixel).
template <int DT, class KT, bool ARG>
struct D1Key {
    static constexpr int IB = sizeof(KT) == 8 ? 32 : 16;
    static __device__ __forceinline__ KT make(uint32_t key, int fidx) {
        if (ARG) return (KT)(((unsigned long long)key << IB) | (unsigned long long)fidx);
        return (KT)key;
    }
};

// One block's work: the strip at (bxi, byi) of plane z.
template <class KT, int DT, bool ARG, int NMAX>
__device__ __forceinline__ void d1_block(const ImgArgs &a, const D1Dev &p, int bxi, int byi, int z) {
    extern __shared__ __align__(16) unsigned char d1_smem[];
    KT *sm = reinterpret_cast<KT *>(d1_smem);
    typedef typename Dt<DT>::E E;
    const int tid = threadIdx.x, NT = blockDim.x;
    const int TH = p.TH, FW = p.FW, FH = p.FH, RX = (p.k - 1) / 2, RY = (p.kh - 1) / 2, SW = p.B * p.T;
    const int x0 = bxi * SW, y0 = byi * TH;
    const char *src = a.src + (size_t)z * a.plane;

    // footprint of the strip, clamped to the image: a warp a row where rows
    // are at least a warp wide and every warp gets one (coalesced loads, no
    // index division), else the block over the flattened footprint (thin
    // windows: a few narrow or short rows would leave most lanes idle)
    if (FW >= 32 && FH >= (NT >> 5)) {
        const int lane = tid & 31, nw = NT >> 5;
        for (int fy = tid >> 5; fy < FH; fy += nw) {
            const int y = clampi(y0 - RY + fy, a.y_lo, a.y_hi);
            for (int fx = lane; fx < FW; fx += 32) {
                const int x = clampi(x0 - RX + fx, 0, a.W - 1);
                const int i = fy * FW + fx;
                sm[i] = D1Key<DT, KT, ARG>::make(Dt<DT>::key(ldg_elem<E>(src, a.pitch, y, x)), i);
            }
        }
    } else {
        for (int i = tid; i < FW * FH; i += NT) {
            const int fy = i / FW, fx = i - fy * FW;
            const int y = clampi(y0 - RY + fy, a.y_lo, a.y_hi);
            const int x = clampi(x0 - RX + fx, 0, a.W - 1);
            sm[i] = D1Key<DT, KT, ARG>::make(Dt<DT>::key(ldg_elem<E>(src, a.pitch, y, x)), i);
        }
    }
    __syncthreads();

    for (int ph = 0; ph < p.nphases; ph++) {
        const int wb = p.phase_begin[ph], we = p.phase_begin[ph + 1];
        for (int w = wb + tid; w < we; w += NT) {
            const D1Item t = d1_unpack(p.items[w], FW);
            if (t.type == D1_SORT) d1_sort_any<KT, NMAX>(sm, t);
            else if (t.type == D1_INSERT) d1_insert_any<KT>(sm, t);
            else d1_merge_item<KT>(sm, t);
        }
        __syncthreads();
    }

    char *dst = a.dst ? a.dst + (size_t)z * a.plane : nullptr;
    char *idx = a.idx ? reinterpret_cast<char *>(a.idx) + (size_t)z * a.idx_plane : nullptr;
    for (int i = tid; i < TH * SW; i += NT) {
        const int py = i / SW, px = i - py * SW;
        const int y = y0 + py, x = x0 + px;
        if (y >= a.H || x >= a.W) continue;
        const KT v = sm[p.out_off[i]];
        if (!ARG) {
            reinterpret_cast<E *>(dst + (size_t)y * a.pitch)[x] = Dt<DT>::val((uint32_t)v);
        } else {
            constexpr int IB = D1Key<DT, KT, ARG>::IB;
            const int fidx = (int)((unsigned long long)v & ((1ull << IB) - 1));
            const uint32_t key = (uint32_t)((unsigned long long)v >> IB);
            const int fy = fidx / FW, fx = fidx - fy * FW;
            const int ys = clampi(y0 - RY + fy, a.y_lo, a.y_hi), xs = clampi(x0 - RX + fx, 0, a.W - 1);
            if (dst) reinterpret_cast<E *>(dst + (size_t)y * a.pitch)[x] = Dt<DT>::val(key);
            if (idx) reinterpret_cast<int32_t *>(idx + (size_t)y * a.idx_pitch)[x] = ys * a.W + xs;
        }
    }
}

template <class KT, int DT, bool ARG, int NMAX>
__global__ void __launch_bounds__(D1_NT_MAX) d1_kernel(ImgArgs a, D1Dev p) {
    d1_block<KT, DT, ARG, NMAX>(a, p, blockIdx.x, blockIdx.y, blockIdx.z);
}

// Persistent form for batches (see o1_persistent): blocks claim work items
// (image, strip x, strip y, plane) from a device counter.
template <class KT, int DT, bool ARG, int NMAX>
__global__ void __launch_bounds__(D1_NT_MAX) d1_persistent(const ImgArgs *imgs, const int4 *items, int n_items,
                                                         unsigned *counter, D1Dev p) {
    __shared__ int s_item;
    for (;;) {
        if (threadIdx.x == 0) s_item = (int)atomicAdd(counter, 1u);
        __syncthreads();
        const int it = s_item;
        if (it >= n_items) break;
        const int4 w = items[it];
        d1_block<KT, DT, ARG, NMAX>(imgs[w.x], p, w.y, w.z, w.w);
        __syncthreads();
    }
}

// ------------------------------------------------------------ host side
struct D1Cached {
    D1Plan plan;
    D1Dev dev;
    void *mem = nullptr;
};

static std::mutex g_d1_mu;
typedef std::tuple<int, int, int, int, int, int, int> PlanKey;  // k, kh, T, TH, B, nt, key bytes
static std::map<PlanKey, D1Plan *> *g_plans = new std::map<PlanKey, D1Plan *>();
static std::map<std::tuple<int, int, int, int, int, int, int, int>, D1Cached *> *g_d1 =
    new std::map<std::tuple<int, int, int, int, int, int, int, int>, D1Cached *>();

// Key width in shared memory: 8-bit values merge as 8-bit keys (half the
// state and four keys a bank word: u8 4096^2 k = 27 5.12 -> 4.37 ms, k = 45
// 9.08 -> 8.44 ms against 16-bit keys), 16-bit values as 16-bit keys,
// 32-bit values as 32-bit keys; argmedian records carry the footprint index
// in 16 (8/16-bit data) or 32 more bits.
static size_t key_bytes(int dtype, bool arg) {
    const bool wide = dtype == MF_U32 || dtype == MF_F32;
    if (arg) return wide ? 8 : 4;
    return wide ? 4 : (dtype == MF_U8 ? 1 : 2);
}

// Host plan for a window of k columns by kh rows (kh = 0: square); nullptr
// if none exists.  No device work.
static const D1Plan *host_plan(int k, int T, int B, int nt, int kb, int kh = 0, int TH = 0) {
    if (kh == 0) kh = k;
    if (TH == 0) TH = T;
    std::lock_guard<std::mutex> lk(g_d1_mu);
    const PlanKey key(k, kh, T, TH, B, nt, kb);
    auto it = g_plans->find(key);
    if (it != g_plans->end()) return it->second;
    D1Plan *pl = new D1Plan();
    if (!d1_build_plan(k, T, pl, B, nt, kb, kh, TH)) {
        delete pl;
        pl = nullptr;
    }
    (*g_plans)[key] = pl;
    return pl;
}

// Strip width and block size for a root tile: the widest strip (sharing the
// most column sorts) whose state fits the small budget runs with 256 threads
// and several blocks per SM; otherwise one tile with 512 threads.
static bool choose_config(int k, int dtype, bool arg, int T, int *B, int *nt, int kh = 0, int TH = 0) {
    if (kh == 0) kh = k;
    if (TH == 0) TH = T;
    // square windows keep root tiles of at least 2 x 2; a side of 1 only
    // where the window is that thin
    const bool square = kh == k && TH == T;
    if (k < 1 || k > 75 || !(k & 1) || kh < 1 || kh > 75 || !(kh & 1) || k * kh < 3 || T < 1 || TH < 1 ||
        (square && T < 2) || T > 32 || TH > 32 || (T & (T - 1)) || (TH & (TH - 1)) || T > k || TH > kh)
        return false;
    const int kb = (int)key_bytes(dtype, arg);
    // MF_D1_NT=256|512|1024: one root tile a block with that many threads
    // wherever its state fits (configuration sweeps)
    static const int forced_nt = getenv("MF_D1_NT") ? atoi(getenv("MF_D1_NT")) : 0;
    if (forced_nt == 256 || forced_nt == 512 || forced_nt == 1024) {
        const D1Plan *pf = host_plan(k, T, 1, forced_nt, kb, kh, TH);
        if (pf && (size_t)pf->smem_elems * kb <= D1_SMEM_BUDGET) {
            *B = 1;
            *nt = forced_nt;
            return true;
        }
    }
    // strips are as wide as 16-bit keys would allow (8-bit keys count two
    // bytes an element here: wider strips of 8-bit keys measured slower)
    const int kbs = kb < 2 ? 2 : kb;
    for (int b = 8; b >= 1; b /= 2) {
        const D1Plan *p = host_plan(k, T, b, 256, kb, kh, TH);
        if (p && (size_t)p->smem_elems * kbs <= D1_SMEM_SMALL) {
            *B = b;
            *nt = 256;
            return true;
        }
    }
    // 8-bit keys: one tile with 256 threads while three blocks fit an SM,
    // else 512 threads while two fit (u8 4096^2 against the 16-bit-key
    // shapes: k = 31 5.86 -> 4.59 ms, k = 45 8.50 -> 7.64 ms, k = 61 12.94 ->
    // 11.53 ms, k = 75 18.72 -> 15.45 ms)
    if (kb == 1) {
        const D1Plan *p2 = host_plan(k, T, 1, 256, kb, kh, TH);
        if (p2 && 3 * ((size_t)p2->smem_elems + 1024) <= 227 * 1024) {
            *B = 1;
            *nt = 256;
            return true;
        }
        const D1Plan *p4 = host_plan(k, T, 1, 512, kb, kh, TH);
        if (p4 && 2 * ((size_t)p4->smem_elems + 1024) <= 227 * 1024) {
            *B = 1;
            *nt = 512;
            return true;
        }
    }
    // one tile per block: 512 threads when two blocks share an SM, else
    // 1024 threads (32 warps) in a block of its own
    const D1Plan *p5 = host_plan(k, T, 1, 512, kb, kh, TH);
    if (p5 && 2 * ((size_t)p5->smem_elems * kbs + 1024) <= 227 * 1024) {
        *B = 1;
        *nt = 512;
        return true;
    }
    const D1Plan *p = host_plan(k, T, 1, 1024, kb, kh, TH);
    if (p && (size_t)p->smem_elems * kb <= D1_SMEM_BUDGET) {
        *B = 1;
        *nt = 1024;
        return true;
    }
    return false;
}

// Plan uploaded to the current device (once per device).
static D1Cached *get_plan(int k, int T, int B, int nt, int kb, int kh = 0, int TH = 0) {
    if (kh == 0) kh = k;
    if (TH == 0) TH = T;
    const D1Plan *hp = host_plan(k, T, B, nt, kb, kh, TH);
    if (!hp) return nullptr;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    std::lock_guard<std::mutex> lk(g_d1_mu);
    auto key = std::make_tuple(k, kh, T, TH, B, nt, kb, dev);
    auto it = g_d1->find(key);
    if (it != g_d1->end()) return it->second;
    D1Cached *c = new D1Cached();
    c->plan = *hp;
    const D1Plan &pl = c->plan;
    std::vector<D1Packed> packed;
    d1_pack_items(pl, &packed);
    const size_t bt = packed.size() * sizeof(D1Packed),
                 bp = pl.phase_begin.size() * 4, bo = pl.out_off.size() * 4;
    const size_t total = bt + bp + bo + 64;
    if (dev_alloc(&c->mem, total) != cudaSuccess) {
        cudaGetLastError();
        delete c;
        return nullptr;
    }
    char *m = (char *)c->mem;
    if (cudaMemcpy(m, packed.data(), bt, cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(m + bt, pl.phase_begin.data(), bp, cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(m + bt + bp, pl.out_off.data(), bo, cudaMemcpyHostToDevice) != cudaSuccess) {
        cudaGetLastError();
        cudaFree(c->mem);
        delete c;
        return nullptr;
    }
    c->dev.items = (const D1Packed *)m;
    c->dev.phase_begin = (const int32_t *)(m + bt);
    c->dev.out_off = (const int32_t *)(m + bt + bp);
    c->dev.nphases = (int)pl.phase_begin.size() - 1;
    c->dev.k = k;
    c->dev.kh = hp->kh;
    c->dev.T = T;
    c->dev.TH = hp->TH;
    c->dev.B = B;
    c->dev.FW = pl.FW;
    c->dev.FH = pl.FH;
    (*g_d1)[key] = c;
    return c;
}

int d1_supported_tile(int k, int dtype, bool arg, int T, int kh) {
    int B, nt;
    return choose_config(k, dtype, arg, T, &B, &nt, kh) ? 1 : 0;
}

int d1_default_tile(int k, int dtype, bool arg, int kh, int bucket) {
    const bool square = kh == 0 || kh == k;
    const int tuned =
        square && tune_lookup(k, dtype, arg, bucket) == MF_DATA_AWARE ? tune_tile(k, dtype, arg, bucket) : 0;
    if (tuned && d1_supported_tile(k, dtype, arg, tuned)) return tuned;
    return d1_heuristic_tile(k, dtype, arg, kh);
}

int d1_heuristic_tile(int k, int dtype, bool arg, int kh) {
    const bool square = kh == 0 || kh == k;
    // root-tile heuristic t(k) = 2^(floor(log2 k) - 1) (paper Sec. 4.2) on
    // the shorter window side, at least 2 (1 for a window one pixel wide or
    // high) and at most 16, lowered until the tree's state fits in shared
    // memory
    const int kmin = square ? k : (k < kh ? k : kh);
    int t = 1;
    while (t * 4 <= kmin) t *= 2;
    if (t < 2 && kmin >= 3) t = 2;
    if (t > 16) t = 16;
    // 2-byte keys: the 16 x 16 tree measured faster from k = 27 on
    // (u8 4096^2: 5.02 vs 5.61 ms at k = 27, 6.25 vs 6.40 ms at k = 31)
    if (key_bytes(dtype, arg) <= 2 && kmin >= 27) t = 16;
    for (; t >= 1; t /= 2)
        if (d1_supported_tile(k, dtype, arg, t, kh)) return t;
    return 0;
}

int d1_supported(int k, int dtype, bool arg) { return d1_default_tile(k, dtype, arg) != 0; }

// Root tile for a window of kw columns by kh rows: t(k) = 2^(floor(log2 k) - 1)
// (paper Sec. 4.2) per side, at least 1 and at most 16 (16 for 2-byte keys
// from a side of 27), the longer tile side halved until the tree's state
// fits in shared memory.
static bool rect_tiles(int kw, int kh, int dtype, bool arg, int *TW, int *TH) {
    auto t_of = [&](int k) {
        int t = 1;
        while (t * 4 <= k) t *= 2;
        if (t > 16) t = 16;
        if (key_bytes(dtype, arg) <= 2 && k >= 27) t = 16;
        return t;
    };
    int tw = t_of(kw), th = t_of(kh);
    for (;;) {
        int B, nt;
        if (choose_config(kw, dtype, arg, tw, &B, &nt, kh, th)) {
            *TW = tw;
            *TH = th;
            return true;
        }
        if (tw == 1 && th == 1) return false;
        if (tw >= th) tw /= 2;
        else th /= 2;
    }
}

template <class KT, int DT, bool ARG, int NMAX>
static int d1_launch_n(const ImgArgs &a, int C, const D1Cached *c, int nt, cudaStream_t s) {
    const size_t smem = (size_t)c->plan.smem_elems * sizeof(KT);
    auto kern = d1_kernel<KT, DT, ARG, NMAX>;
    static DevMask configured;
    int cfg_dev = 0;
    if (!dev_configured(configured, &cfg_dev)) {
        if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)D1_SMEM_BUDGET) !=
            cudaSuccess)
            return MF_ERR_CUDA;
        dev_mark_configured(configured, cfg_dev);
    }
    const int SW = c->plan.B * c->plan.T;
    dim3 grid((a.W + SW - 1) / SW, (a.H + c->plan.TH - 1) / c->plan.TH, C);
    kern<<<grid, nt, smem, s>>>(a, c->dev);
    count_launch();
    return cudaPeekAtLastError() == cudaSuccess ? MF_OK : MF_ERR_CUDA;
}

template <class KT, int DT, bool ARG>
static int d1_launch_t(const ImgArgs &a, int C, const D1Cached *c, int nt, cudaStream_t s) {
    const int ms = c->plan.max_sort;
    if (ms <= 8) return d1_launch_n<KT, DT, ARG, 8>(a, C, c, nt, s);
    if (ms <= 16) return d1_launch_n<KT, DT, ARG, 16>(a, C, c, nt, s);
    return d1_launch_n<KT, DT, ARG, 32>(a, C, c, nt, s);
}

int d1_launch(const ImgArgs &a, int C, int k, int dtype, int T, cudaStream_t s, int kh) {
    const bool arg = a.idx != nullptr;
    int TH = 0;
    if (kh != 0 && kh != k && T == 0) {  // rectangular window: rectangular root tile
        if (!rect_tiles(k, kh, dtype, arg, &T, &TH)) {
            set_error("no data-aware plan for a %dx%d window", k, kh);
            return MF_ERR_UNSUPPORTED;
        }
    }
    if (T == 0) T = d1_default_tile(k, dtype, arg, kh, size_bucket((long long)a.H * a.W));
    int B, nt;
    if (!choose_config(k, dtype, arg, T, &B, &nt, kh, TH)) {
        set_error("no data-aware plan for a %dx%d window, tile=%d", k, kh ? kh : k, T);
        return MF_ERR_UNSUPPORTED;
    }
    const D1Cached *c = get_plan(k, T, B, nt, (int)key_bytes(dtype, arg), kh, TH);
    if (!c) {
        set_error("cannot allocate or upload the data-aware plan for k=%d tile=%d", k, T);
        return MF_ERR_ALLOC;
    }
    int rc;
    switch (dtype * 2 + (arg ? 1 : 0)) {
        case MF_U8 * 2: rc = d1_launch_t<uint8_t, MF_U8, false>(a, C, c, nt, s); break;
        case MF_U16 * 2: rc = d1_launch_t<uint16_t, MF_U16, false>(a, C, c, nt, s); break;
        case MF_U32 * 2: rc = d1_launch_t<uint32_t, MF_U32, false>(a, C, c, nt, s); break;
        case MF_F32 * 2: rc = d1_launch_t<uint32_t, MF_F32, false>(a, C, c, nt, s); break;
        case MF_U8 * 2 + 1: rc = d1_launch_t<uint32_t, MF_U8, true>(a, C, c, nt, s); break;
        case MF_U16 * 2 + 1: rc = d1_launch_t<uint32_t, MF_U16, true>(a, C, c, nt, s); break;
        case MF_U32 * 2 + 1: rc = d1_launch_t<unsigned long long, MF_U32, true>(a, C, c, nt, s); break;
        case MF_F32 * 2 + 1: rc = d1_launch_t<unsigned long long, MF_F32, true>(a, C, c, nt, s); break;
        default: set_error("bad dtype"); return MF_ERR_DTYPE;
    }
    if (rc == MF_ERR_CUDA) set_error("data-aware kernel: %s", cudaGetErrorString(cudaGetLastError()));
    return rc;
}

template <class KT, int DT, int NMAX>
static int d1_persist_n(const ImgArgs *imgs, const int4 *items, int n_items, unsigned *counter,
                        const D1Cached *c, int nt, int blocks_per_sm, int sms, cudaStream_t s, int *grid_out) {
    const size_t smem = (size_t)c->plan.smem_elems * sizeof(KT);
    auto kern = d1_persistent<KT, DT, false, NMAX>;
    static DevMask configured;
    int cfg_dev = 0;
    if (!dev_configured(configured, &cfg_dev)) {
        if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)D1_SMEM_BUDGET) !=
            cudaSuccess)
            return MF_ERR_CUDA;
        dev_mark_configured(configured, cfg_dev);
    }
    if (n_items == 0) {  // prepare only (see persist_o1)
        int occ = 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, nt, smem) != cudaSuccess) return MF_ERR_CUDA;
        *grid_out = occ < 1 ? 1 : occ;
        return MF_OK;
    }
    const int occ = blocks_per_sm > 0 ? blocks_per_sm : 1;
    int grid = occ * sms;
    if (grid > n_items) grid = n_items;
    if (grid < 1) grid = 1;
    *grid_out = grid;
    kern<<<grid, nt, smem, s>>>(imgs, items, n_items, counter, c->dev);
    return cudaPeekAtLastError() == cudaSuccess ? MF_OK : MF_ERR_CUDA;
}

template <class KT, int DT>
static int d1_persist_t(const ImgArgs *imgs, const int4 *items, int n_items, unsigned *counter,
                        const D1Cached *c, int nt, int bps, int sms, cudaStream_t s, int *grid_out) {
    const int ms = c->plan.max_sort;
    if (ms <= 8) return d1_persist_n<KT, DT, 8>(imgs, items, n_items, counter, c, nt, bps, sms, s, grid_out);
    if (ms <= 16) return d1_persist_n<KT, DT, 16>(imgs, items, n_items, counter, c, nt, bps, sms, s, grid_out);
    return d1_persist_n<KT, DT, 32>(imgs, items, n_items, counter, c, nt, bps, sms, s, grid_out);
}

int d1_geometry(int k, int dtype, bool arg, int tile_in, int *tile, int *strip, int *threads) {
    const int T = tile_in > 0 ? tile_in : d1_default_tile(k, dtype, arg);
    int B, nt;
    if (!T || !choose_config(k, dtype, arg, T, &B, &nt)) return MF_ERR_UNSUPPORTED;
    *tile = T;
    *strip = B;
    *threads = nt;
    return MF_OK;
}

int d1_persist(const ImgArgs *imgs, const int4 *items, int n_items, unsigned *counter, int k, int dtype,
               int tile, int blocks_per_sm, int sms, cudaStream_t s, int *grid_out) {
    int T, B, nt;
    if (d1_geometry(k, dtype, false, tile, &T, &B, &nt)) return MF_ERR_UNSUPPORTED;
    // the plan upload (synchronous copies) happens in the prepare call,
    // before any stream capture
    const D1Cached *c = get_plan(k, T, B, nt, (int)key_bytes(dtype, false));
    if (!c) return MF_ERR_CUDA;
    const int b = blocks_per_sm;
    switch (dtype) {
        case MF_U8: return d1_persist_t<uint8_t, MF_U8>(imgs, items, n_items, counter, c, nt, b, sms, s, grid_out);
        case MF_U16: return d1_persist_t<uint16_t, MF_U16>(imgs, items, n_items, counter, c, nt, b, sms, s, grid_out);
        case MF_U32: return d1_persist_t<uint32_t, MF_U32>(imgs, items, n_items, counter, c, nt, b, sms, s, grid_out);
        case MF_F32: return d1_persist_t<uint32_t, MF_F32>(imgs, items, n_items, counter, c, nt, b, sms, s, grid_out);
        default: return MF_ERR_DTYPE;
    }
}

int d1_describe(int k, int dtype, bool arg, int T, char *buf, size_t n) {
    int B = 0, nt = 0;
    const D1Plan *p = T && choose_config(k, dtype, arg, T, &B, &nt) ? host_plan(k, T, B, nt, (int)key_bytes(dtype, arg)) : nullptr;
    if (!p) {
        snprintf(buf, n, "data-aware k=%d (no plan)", k);
        return MF_OK;
    }
    const double px = (double)B * T * T;
    snprintf(buf, n, "data-aware k=%d tile=%dx%d strip=%d block=%d smem=%zuB phases=%d tasks=%zu merged/px=%.1f sorted/px=%.1f",
             k, T, T, B, nt, (size_t)p->smem_elems * key_bytes(dtype, arg), (int)p->phase_begin.size() - 1,
             p->tasks.size(), p->merge_outputs / px, p->sort_elems / px);
    return MF_OK;
}

void d1_release_all() {
    std::lock_guard<std::mutex> lk(g_d1_mu);
    for (auto &kv : *g_d1)
        if (kv.second) {
            cudaFree(kv.second->mem);
            delete kv.second;
        }
    g_d1->clear();
}

}  // namespace mf
