// Volumetric k x k x k median by hierarchical tiling: the extension to 3D
// that the paper names as future work (Sec. 7.2), in both of its variants.
//
// Data-aware form (Sec. 5): the tree of a strip of T x T x T root tiles of
// voxels -- which z pillars and x lines of the footprint are sorted, which
// sorted planes are merged into which core, which ranks each merge keeps --
// depends only on (k, T) and is planned on the host (d3_build_plan in
// mf_d1_plan.cu).  One thread block owns one strip: it stages the footprint
// as order keys in shared memory (clamped to the volume on every axis), runs
// the planned phases with a barrier between them (register sorting networks
// for the lines, merge-path chunks for the merges, the same code as the 2D
// data-aware kernel), and writes the medians.  Nothing but the volume and
// the medians touches HBM.
//
// Data-oblivious form (Sec. 4): the same tree as a generated straight-line
// min/max network (netgen.build3d) over one thread's 2 x 2 x 2 tile, with
// the footprint in registers, for k = 3 and 5.
#include <cstdio>
#include <map>
#include <mutex>
#include <tuple>

#include "../../include/medianfilter_volume.h"
#include "d1_sortnets.cuh"
#include "d3_nets.cuh"
#include "mf_d1_ops.cuh"
#include "mf_registry.h"

namespace mf {

constexpr size_t D3_SMEM_BUDGET = 200 * 1024;
constexpr size_t D3_SMEM_SMALL = 56 * 1024;  // 256 threads, several blocks a SM

struct D3Dev {
    const D1Packed *items;  // one 16-byte record per work item, in work order
    const int32_t *phase_begin;
    const int32_t *out_off;
    int nphases;
    int k, T, F;  // window, root tile side, footprint side in y and z
    int B, FX;    // root tiles per strip (along x), footprint width B*T + k - 1
};

struct VolArgs {
    const char *src;
    char *dst;
    int D, H, W;
    size_t pitch;   // bytes per row
    size_t slice;   // bytes per slice = H * pitch
    size_t volume;  // bytes per volume = D * slice
    int tiles_x, tiles_y;  // strips along x, root tiles along y
};

template <class KT, int N>
__device__ __forceinline__ void d3_sort_task(KT *sm, const D1Item &t) {
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

template <class KT, int NMAX>
__device__ __forceinline__ void d3_sort_any(KT *sm, const D1Item &t) {
    const int n = t.a_len;
    if (n <= 2) d3_sort_task<KT, 2>(sm, t);
    else if (n <= 4) d3_sort_task<KT, 4>(sm, t);
    else if (NMAX <= 8 || n <= 8) d3_sort_task<KT, (NMAX < 8 ? NMAX : 8)>(sm, t);
    else if (NMAX <= 16 || n <= 16) d3_sort_task<KT, (NMAX < 16 ? NMAX : 16)>(sm, t);
    else d3_sort_task<KT, (NMAX < 32 ? NMAX : 32)>(sm, t);
}

// blockIdx.x: strip of B root tiles (x fastest, then y, then z);
// blockIdx.y: volume.
template <class KT, int DT, int NMAX>
__global__ void __launch_bounds__(1024) d3_kernel(VolArgs a, D3Dev p) {
    extern __shared__ __align__(16) unsigned char d3_smem[];
    KT *sm = reinterpret_cast<KT *>(d3_smem);
    typedef typename Dt<DT>::E E;
    const int tid = threadIdx.x, NT = blockDim.x;
    const int T = p.T, F = p.F, FX = p.FX, SW = p.B * p.T, R = (p.k - 1) / 2;
    int b = blockIdx.x;
    const int bx = b % a.tiles_x;
    b /= a.tiles_x;
    const int by = b % a.tiles_y, bz = b / a.tiles_y;
    const int x0 = bx * SW, y0 = by * T, z0 = bz * T;
    const char *src = a.src + (size_t)blockIdx.y * a.volume;

    // footprint (fx, fy, fz) -> (fy * FX + fx) * F + fz; consecutive threads
    // read consecutive x of one row of the volume
    const int n = FX * F * F;
    for (int i = tid; i < n; i += NT) {
        const int fx = i % FX, r = i / FX;
        const int fy = r % F, fz = r / F;
        const int x = clampi(x0 - R + fx, 0, a.W - 1);
        const int y = clampi(y0 - R + fy, 0, a.H - 1);
        const int z = clampi(z0 - R + fz, 0, a.D - 1);
        const E v = __ldg(reinterpret_cast<const E *>(src + (size_t)z * a.slice + (size_t)y * a.pitch) + x);
        sm[(fy * FX + fx) * F + fz] = (KT)Dt<DT>::key(v);
    }
    __syncthreads();

    for (int ph = 0; ph < p.nphases; ph++) {
        const int wb = p.phase_begin[ph], we = p.phase_begin[ph + 1];
        for (int w = wb + tid; w < we; w += NT) {
            const D1Item t = d1_unpack(p.items[w], F);
            if (t.type == D1_SORT) d3_sort_any<KT, NMAX>(sm, t);
            else d1_merge_item<KT>(sm, t);
        }
        __syncthreads();
    }

    char *dst = a.dst + (size_t)blockIdx.y * a.volume;
    for (int i = tid; i < SW * T * T; i += NT) {
        const int ox = i % SW, r = i / SW;
        const int oy = r % T, oz = r / T;
        const int x = x0 + ox, y = y0 + oy, z = z0 + oz;
        if (x >= a.W || y >= a.H || z >= a.D) continue;
        reinterpret_cast<E *>(dst + (size_t)z * a.slice + (size_t)y * a.pitch)[x] =
            Dt<DT>::val((uint32_t)sm[p.out_off[i]]);
    }
}

// Data-oblivious form (Sec. 4 in 3D): one thread owns one T x T x T tile and
// runs the generated min/max network of the same tree (netgen.build3d)
// straight through, loading each voxel of its (T + k - 1)^3 footprint into a
// register at its first use (clamped on every axis; neighbouring threads
// share the loads through L1): no shared memory, no barriers.  Blocks of 32 x 4 threads along x and y;
// blockIdx.z = tile slice + volume * tiles_z.
template <class NET, int DT>
__global__ void __launch_bounds__(128) d3o_kernel(VolArgs a, int tiles_z) {
    typedef typename Dt<DT>::E E;
    constexpr int T = NET::T, F = NET::F, R = (NET::k - 1) / 2;
    const int x0 = (blockIdx.x * blockDim.x + threadIdx.x) * T;
    const int y0 = (blockIdx.y * blockDim.y + threadIdx.y) * T;
    const int z0 = (blockIdx.z % tiles_z) * T;
    const int v = blockIdx.z / tiles_z;
    if (x0 >= a.W || y0 >= a.H) return;
    const char *src = a.src + (size_t)v * a.volume;
    // footprint voxel (fx, fy, fz), clamped on every axis; the network loads
    // each one just before its first use
    auto ld = [&](int fx, int fy, int fz) -> uint32_t {
        const int x = clampi(x0 - R + fx, 0, a.W - 1);
        const int y = clampi(y0 - R + fy, 0, a.H - 1);
        const int z = clampi(z0 - R + fz, 0, a.D - 1);
        return Dt<DT>::key(__ldg(reinterpret_cast<const E *>(src + (size_t)z * a.slice + (size_t)y * a.pitch) + x));
    };
    uint32_t o[T * T * T];
    NET::template run<KoU32>(ld, o);
    char *dst = a.dst + (size_t)v * a.volume;
#pragma unroll
    for (int oz = 0; oz < T; oz++)
#pragma unroll
        for (int oy = 0; oy < T; oy++)
#pragma unroll
            for (int ox = 0; ox < T; ox++) {
                const int x = x0 + ox, y = y0 + oy, z = z0 + oz;
                if (x < a.W && y < a.H && z < a.D)
                    reinterpret_cast<E *>(dst + (size_t)z * a.slice + (size_t)y * a.pitch)[x] =
                        Dt<DT>::val(o[(oz * T + oy) * T + ox]);
            }
}

// Launches the data-oblivious form if a network is built for k and the
// grid fits; returns MF_ERR_UNSUPPORTED (nothing launched) otherwise.
template <class NET>
static int d3o_launch(const VolArgs &a0, int volumes, int dtype, cudaStream_t s) {
    constexpr int T = NET::T;
    VolArgs a = a0;
    const long long tx = (a.W + T - 1) / T, ty = (a.H + T - 1) / T, tz = (a.D + T - 1) / T;
    const long long gx = (tx + 31) / 32, gy = (ty + 3) / 4, gz = tz * volumes;
    if (gx > 2147483647ll || gy > 65535 || gz > 65535) return MF_ERR_UNSUPPORTED;
    dim3 grid((unsigned)gx, (unsigned)gy, (unsigned)gz), block(32, 4, 1);
    switch (dtype) {
        case MF_U8: d3o_kernel<NET, MF_U8><<<grid, block, 0, s>>>(a, (int)tz); break;
        case MF_U16: d3o_kernel<NET, MF_U16><<<grid, block, 0, s>>>(a, (int)tz); break;
        case MF_U32: d3o_kernel<NET, MF_U32><<<grid, block, 0, s>>>(a, (int)tz); break;
        default: d3o_kernel<NET, MF_F32><<<grid, block, 0, s>>>(a, (int)tz); break;
    }
    count_launch();
    return cudaPeekAtLastError() == cudaSuccess ? MF_OK : MF_ERR_CUDA;
}

static bool d3o_built(int k) { return k == 3 || k == 5; }

// ------------------------------------------------------------ host side
struct D3Cached {
    D1Plan plan;
    D3Dev dev;
    int nt = 256;
    void *mem = nullptr;
};

static std::mutex g_d3_mu;
// (k, key bytes, device) -> uploaded plan (nullptr: none fits)
static std::map<std::tuple<int, int, int>, D3Cached *> *g_d3 = new std::map<std::tuple<int, int, int>, D3Cached *>();

// 8-bit values merge as 8-bit keys (as in the 2D data-aware kernel: half
// the state, four keys a bank word), wider values as 16/32-bit keys.
static int d3_key_bytes(int dtype) { return dtype == MF_U32 || dtype == MF_F32 ? 4 : (dtype == MF_U8 ? 1 : 2); }

// Root tile, strip and block size: the largest T (at most 4: the T = 8 trees
// need more than 200 KB from k = 9 on) whose state fits shared memory; with
// 256 threads the widest strip of 8, 4, 2 or 1 tiles whose state is small
// enough for several blocks a SM (the tiles share lines and planes, and the
// block has enough merges to spread over its threads), else one tile with
// 512 threads when two blocks fit, else 1024.
static bool d3_choose(int k, int kb, D1Plan *out, int *nt_out) {
    // 8-bit keys take the shapes of 16-bit keys: the same threads and
    // strips, half the shared memory
    const size_t kbs = kb < 2 ? 2 : (size_t)kb;
    for (int T = 4; T >= 1; T /= 2) {
        if (T > k) continue;
        for (int nb = 8; nb >= 1; nb /= 2) {
            D1Plan pl;
            if (d3_build_plan(k, T, &pl, 256, kb, nb) && (size_t)pl.smem_elems * kbs <= D3_SMEM_SMALL) {
                *out = pl;
                *nt_out = 256;
                return true;
            }
        }
        for (int nt : {512, 1024}) {
            D1Plan pl;
            if (!d3_build_plan(k, T, &pl, nt, kb, 1)) break;
            const size_t bytes = (size_t)pl.smem_elems * kbs;
            if (nt == 512 ? 2 * (bytes + 1024) <= 227 * 1024 : bytes <= D3_SMEM_BUDGET) {
                *out = pl;
                *nt_out = nt;
                return true;
            }
        }
    }
    return false;
}

static D3Cached *d3_get(int k, int dtype, int *err) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) {
        cudaGetLastError();
        *err = MF_ERR_CUDA;
        return nullptr;
    }
    const int kb = d3_key_bytes(dtype);
    std::lock_guard<std::mutex> lk(g_d3_mu);
    const auto key = std::make_tuple(k, kb, dev);
    auto it = g_d3->find(key);
    if (it != g_d3->end()) {
        if (!it->second) *err = MF_ERR_UNSUPPORTED;
        return it->second;
    }
    D3Cached *c = new D3Cached();
    if (!d3_choose(k, kb, &c->plan, &c->nt)) {
        delete c;
        (*g_d3)[key] = nullptr;
        *err = MF_ERR_UNSUPPORTED;
        return nullptr;
    }
    const D1Plan &pl = c->plan;
    std::vector<D1Packed> packed;
    d1_pack_items(pl, &packed);
    const size_t bt = packed.size() * sizeof(D1Packed), bp = pl.phase_begin.size() * 4,
                 bo = pl.out_off.size() * 4;
    if (dev_alloc(&c->mem, bt + bp + bo + 64) != cudaSuccess) {
        cudaGetLastError();
        delete c;
        *err = MF_ERR_ALLOC;
        return nullptr;
    }
    char *m = (char *)c->mem;
    if (cudaMemcpy(m, packed.data(), bt, cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(m + bt, pl.phase_begin.data(), bp, cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(m + bt + bp, pl.out_off.data(), bo, cudaMemcpyHostToDevice) != cudaSuccess) {
        cudaGetLastError();
        cudaFree(c->mem);
        delete c;
        *err = MF_ERR_CUDA;
        return nullptr;
    }
    c->dev.items = (const D1Packed *)m;
    c->dev.phase_begin = (const int32_t *)(m + bt);
    c->dev.out_off = (const int32_t *)(m + bt + bp);
    c->dev.nphases = (int)pl.phase_begin.size() - 1;
    c->dev.k = k;
    c->dev.T = pl.T;
    c->dev.F = pl.FW;
    c->dev.B = pl.B;
    c->dev.FX = pl.FD;
    (*g_d3)[key] = c;
    return c;
}

template <class KT, int DT, int NMAX>
static int d3_launch_n(const VolArgs &a, int volumes, const D3Cached *c, cudaStream_t s) {
    auto kern = d3_kernel<KT, DT, NMAX>;
    static DevMask configured;
    int cfg_dev = 0;
    if (!dev_configured(configured, &cfg_dev)) {
        if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)D3_SMEM_BUDGET) !=
            cudaSuccess)
            return MF_ERR_CUDA;
        dev_mark_configured(configured, cfg_dev);
    }
    const int T = c->plan.T;
    const long long tiles = (long long)a.tiles_x * a.tiles_y * ((a.D + T - 1) / T);
    dim3 grid((unsigned)tiles, (unsigned)volumes, 1);
    kern<<<grid, c->nt, (size_t)c->plan.smem_elems * sizeof(KT), s>>>(a, c->dev);
    count_launch();
    return cudaPeekAtLastError() == cudaSuccess ? MF_OK : MF_ERR_CUDA;
}

template <class KT, int DT>
static int d3_launch_t(const VolArgs &a, int volumes, const D3Cached *c, cudaStream_t s) {
    const int ms = c->plan.max_sort;
    if (ms <= 8) return d3_launch_n<KT, DT, 8>(a, volumes, c, s);
    if (ms <= 16) return d3_launch_n<KT, DT, 16>(a, volumes, c, s);
    return d3_launch_n<KT, DT, 32>(a, volumes, c, s);
}

void d3_release_all() {
    std::lock_guard<std::mutex> lk(g_d3_mu);
    for (auto &kv : *g_d3)
        if (kv.second) {
            cudaFree(kv.second->mem);
            delete kv.second;
        }
    g_d3->clear();
}

static int elem_bytes(int dtype) { return dtype == MF_U8 ? 1 : (dtype == MF_U16 ? 2 : 4); }

static int d3_check(const void *src, const void *dst, int D, int H, int W, size_t pitch, int volumes, int dtype,
                    int k) {
    if (dtype < MF_U8 || dtype > MF_F32) {
        set_error("bad dtype %d", dtype);
        return MF_ERR_DTYPE;
    }
    if (!src || !dst || D < 1 || H < 1 || W < 1 || volumes < 1 || volumes > 65535 || k < 1 || k > D3_MAX_K ||
        (k & 1) == 0) {
        set_error("bad volume arguments (D=%d H=%d W=%d volumes=%d k=%d; k odd 1..%d)", D, H, W, volumes, k,
                  D3_MAX_K);
        return MF_ERR_ARG;
    }
    const int es = elem_bytes(dtype);
    if (pitch < (size_t)W * es || pitch % es) {
        set_error("bad pitch %zu for W=%d", pitch, W);
        return MF_ERR_PITCH;
    }
    const size_t bytes = (size_t)volumes * D * H * pitch;
    const char *s0 = (const char *)src, *d0 = (const char *)dst;
    if (s0 < d0 + bytes && d0 < s0 + bytes) {
        set_error("src and dst overlap");
        return MF_ERR_ALIAS;
    }
    return MF_OK;
}

}  // namespace mf

using namespace mf;

extern "C" int mf_median_filter_3d_ex(const void *src, void *dst, int D, int H, int W, size_t pitch, int volumes,
                                      mf_dtype dtype, int k, mf_variant variant, mf_stream_t stream) {
    int rc = d3_check(src, dst, D, H, W, pitch, volumes, (int)dtype, k);
    if (rc) return rc;
    if (variant != MF_AUTO && variant != MF_OBLIVIOUS && variant != MF_DATA_AWARE) {
        set_error("bad variant %d", (int)variant);
        return MF_ERR_ARG;
    }
    if (variant == MF_OBLIVIOUS && k != 1 && !d3o_built(k)) {
        set_error("no volumetric data-oblivious network built for k=%d", k);
        return MF_ERR_UNSUPPORTED;
    }
    cudaStream_t s = (cudaStream_t)stream;
    if (k == 1) {
        if (cudaMemcpy2DAsync(dst, pitch, src, pitch, (size_t)W * elem_bytes(dtype), (size_t)volumes * D * H,
                              cudaMemcpyDeviceToDevice, s) != cudaSuccess) {
            set_error("copy: %s", cudaGetErrorString(cudaGetLastError()));
            return MF_ERR_CUDA;
        }
        return MF_OK;
    }
    if (variant != MF_DATA_AWARE && d3o_built(k)) {
        VolArgs a;
        a.src = (const char *)src;
        a.dst = (char *)dst;
        a.D = D;
        a.H = H;
        a.W = W;
        a.pitch = pitch;
        a.slice = (size_t)H * pitch;
        a.volume = (size_t)D * a.slice;
        a.tiles_x = a.tiles_y = 0;
        rc = k == 3 ? d3o_launch<D3Net<3>>(a, volumes, (int)dtype, s) : d3o_launch<D3Net<5>>(a, volumes, (int)dtype, s);
        if (rc == MF_OK) return MF_OK;
        if (rc == MF_ERR_CUDA) {
            set_error("volumetric network kernel: %s", cudaGetErrorString(cudaGetLastError()));
            return rc;
        }
        if (variant == MF_OBLIVIOUS) {
            set_error("volume too large for the data-oblivious grid");
            return MF_ERR_UNSUPPORTED;
        }
    }
    int err = MF_OK;
    const D3Cached *c = d3_get(k, (int)dtype, &err);
    if (!c) {
        if (err == MF_ERR_UNSUPPORTED) set_error("no volumetric plan fits shared memory for k=%d", k);
        else set_error("cannot allocate or upload the volumetric plan for k=%d", k);
        return err;
    }
    const int T = c->plan.T;
    VolArgs a;
    a.src = (const char *)src;
    a.dst = (char *)dst;
    a.D = D;
    a.H = H;
    a.W = W;
    a.pitch = pitch;
    a.slice = (size_t)H * pitch;
    a.volume = (size_t)D * a.slice;
    a.tiles_x = (W + c->plan.B * T - 1) / (c->plan.B * T);
    a.tiles_y = (H + T - 1) / T;
    if ((long long)a.tiles_x * a.tiles_y * ((D + T - 1) / T) > 2147483647ll) {
        set_error("volume too large for one launch");
        return MF_ERR_ARG;
    }
    switch (dtype) {
        case MF_U8: rc = d3_launch_t<uint8_t, MF_U8>(a, volumes, c, s); break;
        case MF_U16: rc = d3_launch_t<uint16_t, MF_U16>(a, volumes, c, s); break;
        case MF_U32: rc = d3_launch_t<uint32_t, MF_U32>(a, volumes, c, s); break;
        default: rc = d3_launch_t<uint32_t, MF_F32>(a, volumes, c, s); break;
    }
    if (rc == MF_ERR_CUDA) set_error("volumetric kernel: %s", cudaGetErrorString(cudaGetLastError()));
    return rc;
}

extern "C" int mf_median_filter_3d(const void *src, void *dst, int D, int H, int W, size_t pitch, int volumes,
                                   mf_dtype dtype, int k, mf_stream_t stream) {
    return mf_median_filter_3d_ex(src, dst, D, H, W, pitch, volumes, dtype, k, MF_AUTO, stream);
}

extern "C" int mf_median_filter_3d_describe(int k, mf_dtype dtype, char *buf, size_t n) {
    if (!buf || n == 0) return MF_ERR_ARG;
    if ((int)dtype < MF_U8 || (int)dtype > MF_F32) return MF_ERR_DTYPE;
    if (d3o_built(k)) {
        const int T = k == 3 ? D3Net<3>::T : D3Net<5>::T, ops = k == 3 ? D3Net<3>::n_ops : D3Net<5>::n_ops;
        snprintf(buf, n, "volumetric oblivious k=%d tile=%dx%dx%d block=32x4 net_ops=%d min/max per voxel=%.1f", k, T,
                 T, T, ops, (double)ops / (T * T * T));
        return MF_OK;
    }
    if (k < 3 || k > D3_MAX_K || (k & 1) == 0) {
        snprintf(buf, n, "volumetric k=%d (no plan)", k);
        return MF_OK;
    }
    D1Plan pl;
    int nt = 0;
    const int kb = d3_key_bytes((int)dtype);
    if (!d3_choose(k, kb, &pl, &nt)) {
        snprintf(buf, n, "volumetric k=%d (no plan fits)", k);
        return MF_OK;
    }
    const double vox = (double)pl.B * pl.T * pl.T * pl.T;
    snprintf(buf, n, "volumetric data-aware k=%d tile=%dx%dx%d strip=%d block=%d smem=%zuB phases=%d tasks=%zu merged/vox=%.1f sorted/vox=%.1f",
             k, pl.T, pl.T, pl.T, pl.B, nt, (size_t)pl.smem_elems * kb, (int)pl.phase_begin.size() - 1,
             pl.tasks.size(), pl.merge_outputs / vox, pl.sort_elems / vox);
    return MF_OK;
}
