// Planner of the data-aware variant: turns hierarchical tiling (paper Sec. 3)
// of one T x T root tile into a static schedule of sort and merge tasks over
// shared-memory lists (see mf_d1_plan.h).
//
// State kept per level, breadth-first over the root tile's tree (tiles of
// tw x th, NX = T/tw node columns, NY = T/th node rows):
//   - core[j][i]: the sorted core of node (i, j) minus the extrema already
//     discarded (forgetfulness, Sec. 2.2); all cores of a level have the
//     same length and the same count d of values dropped below the median;
//   - rows[i][fy]: sorted extra row fy over the core columns of node column
//     i -- shared by every node of that column (Sec. 5.3: sorted rows are
//     shared between vertically contiguous tiles);
//   - cols[j][fx]: sorted extra column fx over the core rows of node row j,
//     shared by the nodes of that row.
// Initialisation (Sec. 3.3): sort every footprint column over the root core
// rows and every extra row over the root core columns, then multi-way merge
// the core columns into the root core.  Recursion (Sec. 3.4): a horizontal
// split merges the t_w/2 new columns into one list and that into the
// parent core, keeping the ranks that can still hold the median, and
// extends every extra row with its t_w/2 sorted corners; a vertical split
// exchanges rows and columns.  Merges whose needed output ranks are known
// only read the input ranks that can reach them.
#include <algorithm>
#include <cmath>
#include <cstdlib>
#include <cstdio>
#include <functional>
#include <map>
#include <tuple>

#include "../../include/medianfilter.h"
#include "../../include/medianfilter_volume.h"
#include "mf_d1_ops.cuh"
#include "mf_d1_plan.h"

namespace mf {

// Merge chunk rule (outputs per work item; each chunk pays one binary search
// over its two input lists): the chunk between min and max that finishes
// the phase's items in the fewest rounds over the block (finish_plan).
// Measured on 4096^2 images, k = 27..75: 2-byte keys do best with min 16,
// wider keys with min 12; div only enters the clamp rule
// clamp(phase outputs / (div * threads), min, max) that MF_D1_CHUNK_FIT=0
// restores.  MF_D1_CHUNK="min:div[:max]" overrides them (tuning sweeps).
static const bool D1_ODD_CHUNKS = !getenv("MF_D1_EVEN_CHUNKS");
// Phase balancing of the tasks off the critical chain.  It shortens list
// lifetimes (less shared memory: more blocks a SM where the state limits
// them) at the price of phases that mix sorts and merges.  Measured on
// 4096^2 images it pays for 4-byte keys from k = 41 (u32 k = 75 46.9 ->
// 35.9 ms, k = 45 13.6 -> 12.8 ms) and for 2-byte keys from k = 61 (u16
// k = 61 18.6 -> 14.0 ms: two 512-thread blocks then fit an SM), and costs
// up to 12% below; 1-byte keys (whose state already fits) and volumes gain
// nothing (u8 k = 75 15.5 ms without, 16.2 with).
// MF_D1_BALANCE=0/1 forces it off/on for every plan.
static int d1_balance_env() {
    const char *e = getenv("MF_D1_BALANCE");
    return e ? (atoi(e) != 0) : -1;
}
static bool d1_balance(int n_win, int key_bytes, bool volume) {
    static const int forced = d1_balance_env();
    if (forced >= 0) return forced != 0;
    if (volume || key_bytes == 1) return false;
    return key_bytes >= 4 ? n_win >= 41 * 41 : n_win >= 61 * 61;
}
// Split cores grown from shared sorted slabs plus per-node corner blocks
// instead of extra rows and columns extended level by level
// (MF_D1_SLABS=1).  12% fewer merged elements at k = 45 but three times the
// small sorts; measured slower (u8 k = 61 14.0 -> 17.5 ms, u32 k = 31 8.6 ->
// 10.4 ms), so off by default.
static const bool D1_SLABS = getenv("MF_D1_SLABS") && atoi(getenv("MF_D1_SLABS")) != 0;

// Longest corner run extended by an INSERT task (0: every extension is a
// sort plus a merge); MF_D1_INSERT overrides it (sweeps).
static int d1_insert_max() {
    static const int v = getenv("MF_D1_INSERT") ? std::min(atoi(getenv("MF_D1_INSERT")), D1_MAX_INSERT) : D1_MAX_INSERT;
    return v;
}
// An INSERT moves chunks of this many times the phase's merge chunk; 0:
// one item per INSERT.  Swept on 4096^2 images (factors 0-3): one item for
// 1- and 2-byte keys (u8 k = 45 6.95 -> 6.63 ms, k = 75 14.73 -> 14.23 ms,
// u16 k = 45 8.75 -> 8.27 ms against factor 1), factor 1 for wider keys,
// whose smaller merge chunks keep the phases short (u32 k = 31 8.78 -> 8.38
// ms).  MF_D1_INSERT_CHUNK overrides it (sweeps).
static int d1_insert_chunk_factor(int key_bytes) {
    static const int v = getenv("MF_D1_INSERT_CHUNK") ? atoi(getenv("MF_D1_INSERT_CHUNK")) : -1;
    return v >= 0 ? v : (key_bytes <= 2 ? 0 : 1);
}

// Longest sort of one thread in the 2D plans.  A 32-element register
// network spills at the kernel's 64 registers for 1- and 2-byte keys and
// records; 16-element pieces plus a merge measured faster (4096^2: u32
// k = 61 24.9 -> 20.5 ms, u16 k = 75 18.3 -> 17.2 ms, u8 k = 45 6.69 -> 6.55
// ms) except for 2-byte keys below k = 61 (u16 k = 45 8.04 -> 8.19 ms) and
// 4-byte keys below k = 41 (u32 k = 31 8.17 -> 8.42 ms).  MF_D1_MAX_SORT
// overrides it (sweeps).
static int d1_max_sort(int n_win, int key_bytes) {
    static const int forced = getenv("MF_D1_MAX_SORT") ? atoi(getenv("MF_D1_MAX_SORT")) : 0;
    if (forced > 0) return std::min(forced, D1_MAX_SORT);
    if (key_bytes == 2 && n_win < 61 * 61) return 32;
    if (key_bytes >= 4 && n_win < 41 * 41) return 32;
    return 16;
}

static void chunk_rule(int key_bytes, int *min_chunk, int *div, int *max_chunk) {
    *min_chunk = key_bytes <= 2 ? 16 : 12;
    *div = key_bytes <= 2 ? 2 : 1;
    // 1-byte keys: phases with many outputs take chunks of up to 62 (fewer
    // merge-path searches; u8 k = 61 11.55 -> 10.88 ms, k = 75 15.46 -> 15.02
    // ms, neutral below); wider keys measured no gain from it
    *max_chunk = key_bytes == 1 ? 62 : 32;
    const char *e = getenv("MF_D1_CHUNK");  // "min:div" or "min:div:max" (max < 64: the packed field)
    int a = 0, b = 0, c = 0;
    const int n = e ? sscanf(e, "%d:%d:%d", &a, &b, &c) : 0;
    if (n >= 2 && a >= 1 && a <= 32 && b >= 1 && b <= 64) {
        *min_chunk = a;
        *div = b;
        if (n == 3 && c >= a && c <= 62) *max_chunk = c;
    }
}

namespace {

struct Ref {
    int list;   // -1: footprint; -2: empty
    int start;
    int len;
};

struct PTask {
    int type;
    Ref a;
    int a_stride;
    Ref b;
    int lo, hi;
    int out;    // output list id
    int phase;
    int b_stride;  // INSERT: gather stride of the corners
};

struct ListInfo {
    int len;
    int phase;      // phase that produces it
    int last_use;   // last phase that reads it
    bool needed;
    int off;
};

struct Builder {
    int k, T, FW;  // k: window width
    // longest corner run an INSERT takes (0: none)
    int insert_max = D1_MAX_INSERT;
    // longest run one SORT task sorts (longer runs: even pieces, merged)
    int max_sort = D1_MAX_SORT;
    std::vector<ListInfo> lists;
    std::vector<PTask> tasks;

    int phase_of(const Ref &r) const { return r.list >= 0 ? lists[r.list].phase : -1; }

    int new_list(int len, int phase) {
        lists.push_back(ListInfo{len, phase, -1, false, -1});
        return (int)lists.size() - 1;
    }

    // Sorts n footprint elements at f_off + i*stride.  Runs longer than the
    // largest register sorting network are sorted in pieces and merged.
    Ref sort_gather(int f_off, int stride, int n) {
        if (n > max_sort) {
            std::vector<Ref> parts;
            const int np = (n + max_sort - 1) / max_sort, per = (n + np - 1) / np;
            for (int s = 0; s < n; s += per)
                parts.push_back(sort_gather(f_off + s * stride, stride, std::min(per, n - s)));
            return multiway(parts, 0, n - 1);
        }
        const int id = new_list(n, 0);
        tasks.push_back(PTask{D1_SORT, Ref{-1, f_off, n}, stride, Ref{-2, 0, 0}, 0, n - 1, id, 0});
        return Ref{id, 0, n};
    }

    static Ref sub(const Ref &r, int a0, int a1) {  // elements a0..a1 (inclusive) of r
        if (a1 < a0) return Ref{-2, 0, 0};
        return Ref{r.list, r.start + a0, a1 - a0 + 1};
    }

    // Ranks lo..hi of merge(A, B).
    Ref merge_range(const Ref &A, const Ref &B, int lo, int hi) {
        const int n = A.len + B.len;
        lo = std::max(lo, 0);
        hi = std::min(hi, n - 1);
        if (lo > hi) return Ref{-2, 0, 0};
        const int a0 = std::max(0, lo - B.len), a1 = std::min(A.len - 1, hi);
        const int b0 = std::max(0, lo - A.len), b1 = std::min(B.len - 1, hi);
        const Ref As = sub(A, a0, a1), Bs = sub(B, b0, b1);
        const int off = (As.len ? a0 : 0) + (Bs.len ? b0 : 0);
        const int l2 = lo - off, h2 = hi - off;
        if (Bs.len == 0) return sub(As, l2, h2);
        if (As.len == 0) return sub(Bs, l2, h2);
        const int phase = 1 + std::max(phase_of(As), phase_of(Bs));
        const int id = new_list(h2 - l2 + 1, phase);
        tasks.push_back(PTask{D1_MERGE, As, 0, Bs, l2, h2, id, phase});
        return Ref{id, 0, h2 - l2 + 1};
    }

    Ref merge_full(const Ref &A, const Ref &B) { return merge_range(A, B, 0, A.len + B.len - 1); }

    // Sorted list `row` extended by the h footprint elements at f_off +
    // i*stride (Sec. 3.4: the corners a split adds to an extra row or
    // column).  Up to insert_max corners: one INSERT task gathering them
    // from the footprint; more: a sort and a merge.
    Ref extend(const Ref &row, int f_off, int stride, int h) {
        if (h > insert_max || row.len == 0) return merge_full(row, sort_gather(f_off, stride, h));
        const Ref corners{-1, f_off, h};
        const int phase = 1 + phase_of(row);
        const int n = row.len + h;
        const int id = new_list(n, phase);
        tasks.push_back(PTask{D1_INSERT, row, 0, corners, 0, n - 1, id, phase, stride});
        return Ref{id, 0, n};
    }

    // Ranks lo..hi of the union of sorted lists: balanced tree of two-way
    // merges, each restricted to the ranks that can reach lo..hi (a rank-j
    // element of a partial merge of p of the n elements ends at a rank in
    // [j, j + n - p]).
    Ref multiway(const std::vector<Ref> &ls, int lo, int hi) {
        std::vector<Ref> v;
        for (const Ref &r : ls)
            if (r.len > 0) v.push_back(r);
        if (v.empty()) return Ref{-2, 0, 0};
        int n = 0;
        for (const Ref &r : v) n += r.len;
        hi = std::min(hi, n - 1);
        int off;
        Ref out = rec(v, 0, (int)v.size(), lo, hi, &off);
        (void)off;
        return out;
    }

    Ref rec(const std::vector<Ref> &v, int b, int e, int lo, int hi, int *off) {
        if (e - b == 1) {
            const Ref &l = v[b];
            const int a0 = std::max(0, lo), a1 = std::min(l.len - 1, hi);
            *off = a0;
            return sub(l, a0, a1);
        }
        const int m = (b + e) / 2;
        int nl = 0, nr = 0;
        for (int i = b; i < m; i++) nl += v[i].len;
        for (int i = m; i < e; i++) nr += v[i].len;
        const int la = std::max(0, lo - nr), lb = std::min(nl - 1, hi);
        const int ra = std::max(0, lo - nl), rb = std::min(nr - 1, hi);
        int ol, orr;
        const Ref L = rec(v, b, m, la, lb, &ol);
        const Ref R = rec(v, m, e, ra, rb, &orr);
        const int o = (L.len ? ol : 0) + (R.len ? orr : 0);
        *off = std::max(lo, 0);
        return merge_range(L, R, lo - o, hi - o);
    }
};

// Forgetfulness: ranks of the held list that can still be the median of a
// window of n = kw * kh elements.
static void keep_range(int n, int c, int d, int n_held, int *lo, int *hi) {
    const int m = (n - 1) / 2, u = n - c;
    *lo = std::max(0, m - d - u);
    *hi = std::min(n_held - 1, m - d);
}

}  // namespace

static bool finish_plan(Builder &B, const std::vector<Ref> &outs, int base, int nt, int key_bytes, D1Plan *plan,
                        bool balance, bool volume = false);

bool d1_build_plan(int k, int T, D1Plan *plan, int NB, int nt, int key_bytes, int kh, int TH) {
    // k: window width (columns), kh: window height (rows); root tile T
    // columns by TH rows
    if (kh == 0) kh = k;
    if (TH == 0) TH = T;
    const int kw = k, n_win = kw * kh, TW = T;
    if (kw < 1 || kh < 1 || (kw & 1) == 0 || (kh & 1) == 0 || n_win < 3 || TW < 1 || (TW & (TW - 1)) || TW > kw ||
        TH < 1 || (TH & (TH - 1)) || TH > kh || TW > 32 || TH > 32 || NB < 1 || NB > 64)
        return false;
    Builder B;
    B.k = kw;
    B.T = TW;
    B.FW = NB * TW + kw - 1;
    // Plans with phase balancing keep extensions as sorts plus merges: an
    // INSERT keeps the footprint resident until its phase, and with corners
    // from sorted lists instead the inserts measured slower than the merges
    // (u16 k = 75 20.0 -> 20.9 ms, u32 k = 45 12.9 -> 13.3 ms at 4096^2)
    B.insert_max = d1_balance(n_win, key_bytes, false) ? 0 : d1_insert_max();
    B.max_sort = d1_max_sort(n_win, key_bytes);
    const int FW = B.FW, FH = TH + kh - 1;
    // sorted column segments over the root core rows, for every footprint
    // column of the strip: horizontally adjacent root tiles share them
    std::map<int, Ref> col_strip;
    for (int fx = 0; fx < FW; fx++) col_strip[fx] = B.sort_gather((TH - 1) * FW + fx, FW, kh - TH + 1);
    std::vector<Ref> outs(NB * TW * TH);
    for (int tb = 0; tb < NB; tb++) {
    const int bx = tb * TW;  // strip column of this root tile's footprint
    auto F = [&](int fy, int fx) { return fy * FW + bx + fx; };

    // ---------------------------------------------------------- initialisation
    int tw = TW, th = TH;
    std::map<int, Ref> col0;
    for (int fx = 0; fx < TW + kw - 1; fx++) col0[fx] = col_strip[bx + fx];
    // sorted extra rows over the root core columns
    std::map<int, Ref> row0;
    for (int fy = 0; fy < FH; fy++)
        if (fy < TH - 1 || fy > kh - 1) row0[fy] = B.sort_gather(F(fy, TW - 1), 1, kw - TW + 1);
    // root core: multi-way merge of the core columns
    std::vector<Ref> cc;
    for (int fx = TW - 1; fx <= kw - 1; fx++) cc.push_back(col0[fx]);
    int c = (kw - TW + 1) * (kh - TH + 1), lo, hi;
    keep_range(n_win, c, 0, c, &lo, &hi);
    int d = lo;
    // per level state
    std::vector<std::vector<Ref>> core(1, std::vector<Ref>(1, B.multiway(cc, lo, hi)));  // [j][i]
    if (D1_SLABS) {
        // A child's core is its parent's core plus the h new columns (rows)
        // over the parent's core rows (columns).  Those split into the part
        // over the root core's rows (columns) -- the same for every node of
        // a node column (row), sorted once from the sorted column segments
        // (root extra rows) and shared -- and a small block over the node's
        // own extra rows (columns).  Sorted rectangles are memoised, so no
        // extra row or column is ever carried and re-merged level by level.
        std::map<std::tuple<int, int, int, int>, Ref> memo;
        auto rect = [&](int y0r, int y1r, int x0r, int x1r) -> Ref {
            if (y1r < y0r || x1r < x0r) return Ref{-2, 0, 0};
            const auto key = std::make_tuple(y0r, y1r, x0r, x1r);
            auto it = memo.find(key);
            if (it != memo.end()) return it->second;
            std::vector<Ref> parts;
            if (y0r == TH - 1 && y1r == kh - 1) {
                for (int fx = x0r; fx <= x1r; fx++) parts.push_back(col0.at(fx));
            } else if (x0r == TW - 1 && x1r == kw - 1) {
                for (int fy = y0r; fy <= y1r; fy++) parts.push_back(row0.at(fy));
            } else if (x1r - x0r >= y1r - y0r) {
                for (int fy = y0r; fy <= y1r; fy++) parts.push_back(B.sort_gather(F(fy, x0r), 1, x1r - x0r + 1));
            } else {
                for (int fx = x0r; fx <= x1r; fx++) parts.push_back(B.sort_gather(F(y0r, fx), FW, y1r - y0r + 1));
            }
            const Ref r = B.multiway(parts, 0, 1 << 30);
            memo[key] = r;
            return r;
        };
        while (tw * th > 1) {
            const int NX = TW / tw, NY = TH / th;
            const bool horiz = tw >= th;
            const int h = (horiz ? tw : th) / 2;
            const int cw = kw - (horiz ? h : tw) + 1, ch = kh - (horiz ? th : h) + 1;
            c = cw * ch;
            const int K = core[0][0].len;
            const int n_held = K + h * (horiz ? kh - th + 1 : kw - tw + 1);
            keep_range(n_win, c, d, n_held, &lo, &hi);
            std::vector<std::vector<Ref>> ncore(horiz ? NY : 2 * NY, std::vector<Ref>(horiz ? 2 * NX : NX));
            for (int j = 0; j < NY; j++)
                for (int i = 0; i < NX; i++) {
                    const int x0n = i * tw, y0n = j * th;
                    for (int s2 = 0; s2 < 2; s2++) {
                        std::vector<Ref> parts;
                        if (horiz) {
                            const int q0 = s2 == 0 ? x0n + h - 1 : x0n + kw, q1 = q0 + h - 1;
                            parts.push_back(rect(TH - 1, kh - 1, q0, q1));
                            parts.push_back(rect(y0n + th - 1, TH - 2, q0, q1));
                            parts.push_back(rect(kh, y0n + kh - 1, q0, q1));
                        } else {
                            const int r0 = s2 == 0 ? y0n + h - 1 : y0n + kh, r1 = r0 + h - 1;
                            parts.push_back(rect(r0, r1, TW - 1, kw - 1));
                            parts.push_back(rect(r0, r1, x0n + tw - 1, TW - 2));
                            parts.push_back(rect(r0, r1, kw, x0n + kw - 1));
                        }
                        const Ref extra = B.multiway(parts, 0, 1 << 30);
                        const Ref nc = B.merge_range(core[j][i], extra, lo, hi);
                        if (horiz) ncore[j][2 * i + s2] = nc;
                        else ncore[2 * j + s2][i] = nc;
                    }
                }
            core.swap(ncore);
            if (horiz) tw = h;
            else th = h;
            d += lo;
        }
        for (int j = 0; j < TH; j++)
            for (int i = 0; i < TW; i++) outs[j * NB * TW + bx + i] = core[j][i];
        continue;
    }
    std::vector<std::map<int, Ref>> rows(1, row0);  // [i][fy]
    std::vector<std::map<int, Ref>> cols(1);        // [j][fx]
    for (auto &kv : col0)
        if (kv.first < TW - 1 || kv.first > kw - 1) cols[0][kv.first] = kv.second;

    // ---------------------------------------------------------- recursion
    while (tw * th > 1) {
        const int NX = TW / tw, NY = TH / th;
        if (tw >= th) {  // horizontal split: halve the width
            const int h = tw / 2;
            const int cw = kw - h + 1, ch = kh - th + 1;
            c = cw * ch;
            const int K = core[0][0].len;
            const int n_held = K + h * ch;
            keep_range(n_win, c, d, n_held, &lo, &hi);
            std::vector<std::vector<Ref>> ncore(NY, std::vector<Ref>(2 * NX));
            std::vector<std::map<int, Ref>> nrows(2 * NX);
            for (int i = 0; i < NX; i++) {
                const int x0 = i * tw;
                for (int s = 0; s < 2; s++) {
                    const int nx0 = s == 0 ? x0 + h - 1 : x0 + kw;  // first new core column
                    for (int j = 0; j < NY; j++) {
                        std::vector<Ref> nc;
                        for (int fx = nx0; fx < nx0 + h; fx++) nc.push_back(cols[j].at(fx));
                        const Ref extra = B.multiway(nc, 0, 1 << 30);
                        ncore[j][2 * i + s] = B.merge_range(core[j][i], extra, lo, hi);
                    }
                    for (auto &kv : rows[i]) nrows[2 * i + s][kv.first] = B.extend(kv.second, F(kv.first, nx0), 1, h);
                }
            }
            core.swap(ncore);
            rows.swap(nrows);
            tw = h;
        } else {  // vertical split: halve the height
            const int h = th / 2;
            const int cw = kw - tw + 1, ch = kh - h + 1;
            c = cw * ch;
            const int K = core[0][0].len;
            const int n_held = K + h * cw;
            keep_range(n_win, c, d, n_held, &lo, &hi);
            std::vector<std::vector<Ref>> ncore(2 * NY, std::vector<Ref>(NX));
            std::vector<std::map<int, Ref>> ncols(2 * NY);
            for (int j = 0; j < NY; j++) {
                const int y0 = j * th;
                for (int s = 0; s < 2; s++) {
                    const int ny0 = s == 0 ? y0 + h - 1 : y0 + kh;  // first new core row
                    for (int i = 0; i < NX; i++) {
                        std::vector<Ref> nr;
                        for (int fy = ny0; fy < ny0 + h; fy++) nr.push_back(rows[i].at(fy));
                        const Ref extra = B.multiway(nr, 0, 1 << 30);
                        ncore[2 * j + s][i] = B.merge_range(core[j][i], extra, lo, hi);
                    }
                    for (auto &kv : cols[j]) ncols[2 * j + s][kv.first] = B.extend(kv.second, F(ny0, kv.first), FW, h);
                }
            }
            core.swap(ncore);
            cols.swap(ncols);
            th = h;
        }
        d += lo;
    }

    for (int j = 0; j < TH; j++)
        for (int i = 0; i < TW; i++) outs[j * NB * TW + bx + i] = core[j][i];
    }  // root tiles of the strip

    plan->k = kw;
    plan->kh = kh;
    plan->T = TW;
    plan->TH = TH;
    plan->B = NB;
    plan->FW = FW;
    plan->FH = FH;
    plan->FD = 1;
    plan->TD = 1;
    return finish_plan(B, outs, FW * FH, nt, key_bytes, plan, d1_balance(n_win, key_bytes, false));
}

// Liveness, phases, shared-memory allocation and the emitted task list of a
// built tree (outs: the list holding each output's median, in output order;
// the footprint occupies the first `base` elements).  The geometry fields of
// `plan` are set by the caller.
static bool finish_plan(Builder &B, const std::vector<Ref> &outs, int base, int nt, int key_bytes, D1Plan *plan,
                        bool balance, bool volume) {
    // ---------------------------------------------------------- liveness
    for (const Ref &r : outs) {
        if (r.len != 1) return false;
        if (r.list >= 0) B.lists[r.list].needed = true;
    }
    std::vector<bool> keep(B.tasks.size(), false);
    for (const PTask &t : B.tasks)  // merges read lists only (each has its sentinel slot)
        if (t.type == D1_MERGE && (t.a.list < 0 || t.b.list < 0)) return false;
    for (int ti = (int)B.tasks.size() - 1; ti >= 0; ti--) {
        const PTask &t = B.tasks[ti];
        if (!B.lists[t.out].needed) continue;
        keep[ti] = true;
        if (t.a.list >= 0) B.lists[t.a.list].needed = true;
        if (t.b.list >= 0) B.lists[t.b.list].needed = true;
    }
    // recompute phases on the kept tasks (tasks are in creation = dependency order)
    std::vector<int> lphase(B.lists.size(), -1);
    int nph = 0;
    std::vector<int> task_phase(B.tasks.size(), -1);
    for (size_t ti = 0; ti < B.tasks.size(); ti++) {
        if (!keep[ti]) continue;
        const PTask &t = B.tasks[ti];
        int p = 0;
        if (t.a.list >= 0) p = std::max(p, lphase[t.a.list] + 1);
        if (t.b.list >= 0) p = std::max(p, lphase[t.b.list] + 1);
        task_phase[ti] = p;
        lphase[t.out] = p;
        nph = std::max(nph, p + 1);
    }
    // ---------------------------------------------------------- balancing
    // The phase count is the tree's dependency depth (the chain of core
    // merges).  Tasks off that chain -- extending extra rows and columns,
    // merging the new columns of a later split -- have slack: each may run
    // in any phase between its earliest (inputs ready) and its latest (all
    // readers still after it).  Placing each in the least-loaded phase of
    // that window evens out the work of the phases (the threads of a block
    // wait for the slowest one at every barrier) and produces lists closer
    // to where they are read, which shortens their lifetimes in shared
    // memory.
    if (balance && nph > 1) {
        std::vector<std::vector<int>> readers(B.lists.size());
        for (size_t ti = 0; ti < B.tasks.size(); ti++) {
            if (!keep[ti]) continue;
            const PTask &t = B.tasks[ti];
            if (t.a.list >= 0) readers[t.a.list].push_back((int)ti);
            if (t.b.list >= 0 && t.b.list != t.a.list) readers[t.b.list].push_back((int)ti);
        }
        std::vector<bool> is_out(B.lists.size(), false);
        for (const Ref &r : outs)
            if (r.list >= 0) is_out[r.list] = true;
        std::vector<int> alap(B.tasks.size(), nph - 1);
        for (int ti = (int)B.tasks.size() - 1; ti >= 0; ti--) {
            if (!keep[ti]) continue;
            int a = nph - 1;
            for (int r : readers[B.tasks[ti].out]) a = std::min(a, alap[r] - 1);
            if (is_out[B.tasks[ti].out]) a = std::min(a, nph - 1);
            alap[ti] = a;
        }
        // cost in merged-element units: a merge costs its outputs, a sort of
        // n elements about n (log2 n)^2 / 8 (a register sorting network)
        auto cost = [&](const PTask &t) -> double {
            if (t.type != D1_SORT) return t.hi - t.lo + 1;
            const double n = t.a.len, l = std::log2(std::max(2.0, n));
            return n * std::max(1.0, l * l / 8);
        };
        // windows [asap, alap]; tasks are placed least-slack first (the
        // chain has none), each in the least-loaded phase of its current
        // window; a placement narrows the windows of everything that
        // depends on it, or that it depends on, so every window stays
        // non-empty
        std::vector<int> asap(task_phase);
        std::vector<std::vector<int>> succ(B.tasks.size()), pred(B.tasks.size());
        std::vector<int> producer(B.lists.size(), -1);
        for (size_t ti = 0; ti < B.tasks.size(); ti++)
            if (keep[ti]) producer[B.tasks[ti].out] = (int)ti;
        for (size_t ti = 0; ti < B.tasks.size(); ti++) {
            if (!keep[ti]) continue;
            const PTask &t = B.tasks[ti];
            for (int l : {t.a.list, t.b.list})
                if (l >= 0 && producer[l] >= 0) {
                    succ[producer[l]].push_back((int)ti);
                    pred[ti].push_back(producer[l]);
                }
        }
        std::vector<int> order;
        for (size_t ti = 0; ti < B.tasks.size(); ti++)
            if (keep[ti]) order.push_back((int)ti);
        std::stable_sort(order.begin(), order.end(), [&](int x, int y) {
            const int sx = alap[x] - asap[x], sy = alap[y] - asap[y];
            if (sx != sy) return sx < sy;
            return cost(B.tasks[x]) > cost(B.tasks[y]);
        });
        std::vector<double> load(nph, 0.0);
        std::vector<int> stack;
        for (int ti : order) {
            const double c = cost(B.tasks[ti]);
            int p = asap[ti];
            for (int q = asap[ti] + 1; q <= alap[ti]; q++)
                if (load[q] <= load[p]) p = q;  // ties: the later phase
            load[p] += c;
            asap[ti] = alap[ti] = p;
            stack.assign(1, ti);
            while (!stack.empty()) {  // readers start after p
                const int u = stack.back();
                stack.pop_back();
                for (int v : succ[u])
                    if (asap[v] < asap[u] + 1) {
                        asap[v] = asap[u] + 1;
                        stack.push_back(v);
                    }
            }
            stack.assign(1, ti);
            while (!stack.empty()) {  // producers finish before p
                const int u = stack.back();
                stack.pop_back();
                for (int v : pred[u])
                    if (alap[v] > alap[u] - 1) {
                        alap[v] = alap[u] - 1;
                        stack.push_back(v);
                    }
            }
        }
        std::vector<int> lp(B.lists.size(), -1);
        for (size_t ti = 0; ti < B.tasks.size(); ti++)
            if (keep[ti]) {
                task_phase[ti] = asap[ti];
                lp[B.tasks[ti].out] = asap[ti];
            }
        lphase.swap(lp);
    }
    // last use of every list, and of the footprint (read by sorts only)
    std::vector<int> last(B.lists.size(), -1);
    int foot_last = -1;
    for (size_t ti = 0; ti < B.tasks.size(); ti++) {
        if (!keep[ti]) continue;
        const PTask &t = B.tasks[ti];
        if (t.a.list >= 0) last[t.a.list] = std::max(last[t.a.list], task_phase[ti]);
        if (t.b.list >= 0) last[t.b.list] = std::max(last[t.b.list], task_phase[ti]);
        if (t.a.list == -1 || t.b.list == -1) foot_last = std::max(foot_last, task_phase[ti]);
    }
    for (const Ref &r : outs) {
        if (r.list >= 0) last[r.list] = nph;  // read after the last phase
        if (r.list == -1) foot_last = nph;
    }

    // ---------------------------------------------------------- allocation
    // first fit over a free list, phase by phase; the footprint sits at 0
    std::vector<std::pair<int, int>> freel;  // (off, len), sorted by off
    // List sizes: the list, its sentinel slot (largest key) that its producer
    // writes -- merges read one element past their inputs -- and, except
    // for 2-byte keys at 41 <= k < 61 and 3D plans, padding to a whole, odd number of
    // 4-byte words (1- and 2-byte keys: lists start on a word).  Threads
    // stepping through consecutive lists in lockstep then hit distinct
    // banks: fewer bank-conflict replays (4096^2, u8 k = 31 4.40 -> 4.08 ms,
    // u16 k = 31 5.91 -> 5.55 ms, u32 k = 31 8.72 -> 8.30 ms; u16 k = 45
    // measured 8.12 -> 8.48 ms, so it keeps unpadded lists).
    const int kwin2 = B.k * B.k;  // (width squared: the rule is stated in k)
    const bool oddw = !volume && !(key_bytes == 2 && kwin2 >= 41 * 41 && kwin2 < 61 * 61);
    const int al = oddw && key_bytes < 4 ? 4 / key_bytes : 1;
    auto rnd = [&](int n) { return (n + al - 1) / al * al; };
    auto lsz = [&](int len) {
        int n = rnd(len + 1);
        if (oddw && key_bytes <= 4) {
            const int per = 4 / key_bytes;  // elements a word
            int words = (n * key_bytes + 3) / 4;
            if (!(words & 1)) words++;
            n = std::max(n, words * per);
        }
        return n;
    };
    int top = rnd(base);
    std::vector<std::vector<int>> prod(nph + 1), dies(nph + 2);
    for (size_t li = 0; li < B.lists.size(); li++) {
        if (lphase[li] < 0) continue;
        prod[lphase[li]].push_back((int)li);
        dies[std::max(last[li], lphase[li]) + 1].push_back((int)li);
    }
    auto release = [&](int off, int len) {
        freel.push_back({off, len});
        std::sort(freel.begin(), freel.end());
        std::vector<std::pair<int, int>> m;
        for (auto &f : freel) {
            if (!m.empty() && m.back().first + m.back().second == f.first) m.back().second += f.second;
            else m.push_back(f);
        }
        freel.swap(m);
    };
    auto alloc = [&](int len) {
        for (size_t i = 0; i < freel.size(); i++) {
            if (freel[i].second >= len) {
                const int off = freel[i].first;
                freel[i].first += len;
                freel[i].second -= len;
                if (freel[i].second == 0) freel.erase(freel.begin() + i);
                return off;
            }
        }
        // grow: merge with a free block ending at top
        if (!freel.empty() && freel.back().first + freel.back().second == top) {
            const int off = freel.back().first;
            top = off + len;
            freel.pop_back();
            return off;
        }
        const int off = top;
        top += len;
        return off;
    };
    // Packing of the lists as rectangles (phases x elements), largest first,
    // each at the lowest offset clear of every list live in an overlapping
    // phase.  Balanced plans free lists in every phase and first fit phase
    // by phase fragments them by up to a third (u32 k = 75, 8 x 8 tile:
    // 115.5 -> 89.5 KB, two blocks a SM again: 50.5 -> 33.6 ms at 4096^2);
    // other plans take it where it needs less shared memory (3D plans).
    auto pack = [&](std::vector<int> &offs) {
        struct Box {
            int off, end, t0, t1;
        };
        std::vector<Box> placed;
        placed.push_back(Box{0, rnd(base), 0, balance ? std::max(foot_last, 0) : nph});
        std::vector<int> order;
        for (size_t li = 0; li < B.lists.size(); li++)
            if (lphase[li] >= 0) order.push_back((int)li);
        auto t1_of = [&](int li) { return std::max(last[li], lphase[li]); };
        std::stable_sort(order.begin(), order.end(), [&](int x, int y) {
            const int sx = lsz(B.lists[x].len), sy = lsz(B.lists[y].len);
            if (sx != sy) return sx > sy;
            return t1_of(x) - lphase[x] > t1_of(y) - lphase[y];
        });
        int ptop = rnd(base);
        std::vector<std::pair<int, int>> busy;
        for (int li : order) {
            const int t0 = lphase[li], t1 = t1_of(li), sz = lsz(B.lists[li].len);
            busy.clear();
            for (const Box &b : placed)
                if (b.t0 <= t1 && t0 <= b.t1) busy.push_back({b.off, b.end});
            std::sort(busy.begin(), busy.end());
            int off = 0;
            for (auto &b : busy) {
                if (off + sz <= b.first) break;
                off = std::max(off, b.second);
            }
            offs[li] = off;
            placed.push_back(Box{off, off + sz, t0, t1});
            ptop = std::max(ptop, off + sz);
        }
        return ptop;
    };
    for (int p = 0; p <= nph; p++) {
        // the footprint is free once its last reader has run
        if (balance && p == foot_last + 1 && base > 0) release(0, rnd(base));
        for (int li : dies[p]) release(B.lists[li].off, lsz(B.lists[li].len));
        if (p < nph)
            for (int li : prod[p]) B.lists[li].off = alloc(lsz(B.lists[li].len));
    }
    if (balance || volume) {
        std::vector<int> offs(B.lists.size(), -1);
        const int ptop = pack(offs);
        if (balance || ptop < top) {
            for (size_t li = 0; li < B.lists.size(); li++)
                if (lphase[li] >= 0) B.lists[li].off = offs[li];
            top = ptop;
        }
    }

    // ---------------------------------------------------------- emit
    plan->nt = nt;
    plan->smem_elems = top;
    plan->tasks.clear();
    plan->work.clear();
    plan->phase_begin.clear();
    plan->max_sort = 0;
    plan->merge_outputs = plan->sort_elems = 0;
    auto resolve = [&](const Ref &r) { return r.list >= 0 ? B.lists[r.list].off + r.start : (r.list == -1 ? r.start : 0); };
    std::vector<std::vector<int>> by_phase(nph);
    int min_chunk = 16, div = 1, max_chunk = 32;
    chunk_rule(key_bytes, &min_chunk, &div, &max_chunk);
    for (size_t ti = 0; ti < B.tasks.size(); ti++)
        if (keep[ti]) by_phase[task_phase[ti]].push_back((int)ti);
    for (int p = 0; p < nph; p++) {
        plan->phase_begin.push_back((int)plan->work.size());
        long long outs_p = 0;
        for (int ti : by_phase[p])
            if (B.tasks[ti].type != D1_SORT) outs_p += B.tasks[ti].hi - B.tasks[ti].lo + 1;
        // about one chunk per thread: phases with few outputs (the upper tree
        // levels) get short chunks so the whole block shares them
        int chunk = (int)std::min<long long>(max_chunk, std::max<long long>(min_chunk, outs_p / ((long long)div * nt)));
        // the chunks of one merge run on consecutive threads: an odd number of
        // 4-byte words between their output runs spreads a warp's stores
        // (and its roughly proportional input reads) over all 32 banks
        // (8-bit keys: 4 mod 8 elements, 16-bit keys: 2 mod 4, wider keys:
        // odd)
        auto round_chunk = [&](int c) {
            if (!D1_ODD_CHUNKS) return c;
            return key_bytes == 1 ? (c & ~7) + 4 : key_bytes == 2 ? (c & ~3) + 2 : (c | 1);
        };
        chunk = round_chunk(chunk);
        // Of the rounded chunks from min to max, the one whose rounds of
        // work items over the block's threads finish first: rounds(c) x
        // (c + 14, an item's fixed cost in merged elements), the larger
        // chunk on ties.  A phase of 288-384 items on 256 threads otherwise
        // runs a second round for a few threads while the rest wait at the
        // barrier (4096^2: u8 k = 31 4.03 -> 3.73 ms, k = 61 10.43 -> 9.65
        // ms, u32 k = 75 33.2 -> 32.1 ms; MF_D1_CHUNK_FIT=0 keeps the clamp
        // rule above).
        static const int fit_env = getenv("MF_D1_CHUNK_FIT") ? atoi(getenv("MF_D1_CHUNK_FIT")) : 14;
        if (fit_env) {
            long best = -1;
            const int fct = d1_insert_chunk_factor(key_bytes);
            for (int c = min_chunk; c <= max_chunk; c++) {
                const int rc = round_chunk(c);
                if (rc > 62) break;
                long items = 0;
                for (int ti : by_phase[p]) {
                    const PTask &t = B.tasks[ti];
                    const int n = t.hi - t.lo + 1;
                    if (t.type == D1_SORT) items++;
                    else if (t.type == D1_INSERT) items += fct > 0 ? (t.a.len + std::min(fct * rc, 62) - 1) / std::min(fct * rc, 62) : 1;
                    else items += (n + rc - 1) / rc;
                }
                const long rounds = (items + nt - 1) / nt;
                const long cost = rounds * (fit_env + rc);
                if (best < 0 || cost <= best) {
                    best = cost;
                    chunk = rc;
                }
            }
        }
        // sorts first, grouped by size class, then merges
        std::vector<int> order = by_phase[p];
        std::stable_sort(order.begin(), order.end(), [&](int x, int y) {
            const PTask &a = B.tasks[x], &b = B.tasks[y];
            if (a.type != b.type) return a.type < b.type;
            if (a.type == D1_SORT) return a.a.len < b.a.len;
            return false;
        });
        for (int ti : order) {
            const PTask &t = B.tasks[ti];
            D1Task o;
            o.type = t.type;
            o.a_off = resolve(t.a);
            o.a_len = t.a.len;
            o.a_stride = t.a_stride;
            o.b_off = resolve(t.b);
            o.b_len = t.b.len;
            o.b_stride = t.type == D1_INSERT ? t.b_stride : 1;
            o.lo = t.lo;
            o.hi = t.hi;
            o.out_off = B.lists[t.out].off;
            const int tid = (int)plan->tasks.size();
            if (t.type == D1_SORT) {
                o.chunk = 0;
                plan->work.push_back((uint32_t)tid << 12);
                plan->max_sort = std::max(plan->max_sort, t.a.len);
                plan->sort_elems += t.a.len;
            } else if (t.type == D1_INSERT) {
                // chunks over the list elements, as long as the phase's merge chunks
                const int n = t.a.len, f = d1_insert_chunk_factor(key_bytes);
                o.chunk = f > 0 ? std::min(std::min(f * chunk, 62), n) : 0;
                const int nchunks = o.chunk ? (n + o.chunk - 1) / o.chunk : 1;
                for (int cidx = 0; cidx < nchunks; cidx++) plan->work.push_back(((uint32_t)tid << 12) | (uint32_t)cidx);
                plan->merge_outputs += t.hi - t.lo + 1;
            } else {
                const int n = t.hi - t.lo + 1;
                o.chunk = std::min(chunk, n);
                const int nchunks = (n + o.chunk - 1) / o.chunk;
                for (int cidx = 0; cidx < nchunks; cidx++) plan->work.push_back(((uint32_t)tid << 12) | (uint32_t)cidx);
                plan->merge_outputs += n;
            }
            plan->tasks.push_back(o);
        }
    }
    plan->phase_begin.push_back((int)plan->work.size());
    plan->out_off.resize(outs.size());
    for (size_t i = 0; i < outs.size(); i++) plan->out_off[i] = resolve(outs[i]);
    // limits of the packed device form (every element position, a merge
    // item's output position inside its list included, below 2^17)
    if (plan->smem_elems > (1 << 17)) return false;
    for (const D1Task &t : plan->tasks)
        if (t.a_off >= (1 << 17) || t.b_off >= (1 << 17) || t.out_off >= (1 << 17) || t.a_len >= (1 << 13) ||
            t.b_len >= (1 << 13) || t.lo >= (1 << 13) || t.hi >= (1 << 13) || t.chunk >= 64 ||
            (t.type == D1_SORT && t.a_stride != 1 && t.a_stride != plan->FW) ||
            (t.type == D1_INSERT && (t.b_len > D1_MAX_INSERT || t.a_len > 255 || (t.b_stride != 1 && t.b_stride != plan->FW))))
            return false;
    return plan->tasks.size() < (1u << 20);
}

// ---------------------------------------------------------------- volumes
// Hierarchical tiling of a k x k x k window over a T x T x T root tile of
// voxels (the extension to 3D that the paper names as future work, Sec. 7.2).
// A node is a box of tx x ty x tz outputs; its core is the box of window
// positions all of them share, (k - tx + 1) x (k - ty + 1) x (k - tz + 1),
// kept sorted and pruned to the ranks that can still hold the median
// (forgetfulness, Sec. 2.2: with n = k^3, core size c and d values dropped
// below, held ranks [max(0, m - d - (n - c)), min(held - 1, m - d)]).  A split
// halves the longest side (x, then y, then z on ties -- the 2D rule of
// Sec. 3.1 extended by one axis); each child's core grows by the h = t/2
// planes of window positions on its side, over the parent core's other two
// ranges (Sec. 3.4: the new columns or rows merged into the core).  Sorted
// planes are assembled from sorted lines of the footprint (z pillars, or x
// lines for planes one voxel deep) and memoised by box.  Every node keeps
// each of its extra planes sorted over its own core ranges, so a child
// extends its parent's copy by the strip its split added, the way sorted
// extra rows and columns are extended by their corners in 2D (12-20 % fewer
// merged elements than sorting each plane from lines where it joins a
// core).
//
// A block may own a strip of NB root tiles side by side along x, which
// share the memoised lines and planes of their overlapping footprints
// (Sec. 3.3: adjacent tiles share their column sorts).  Footprint layout:
// F = T + k - 1 in y and z, FX = NB * T + k - 1 in x, element (fx, fy, fz)
// at (fy * FX + fx) * F + fz (z innermost), so z pillars are contiguous and
// x lines have stride F (the plan's FW).  Output (ox, oy, oz) of the strip
// is entry (oz * T + oy) * NB * T + ox of out_off.
namespace {
struct Box {
    int x0, x1, y0, y1, z0, z1;  // inclusive ranges in footprint coordinates
    long long vol() const { return (long long)(x1 - x0 + 1) * (y1 - y0 + 1) * (z1 - z0 + 1); }
    bool inside(const Box &o) const {
        return x0 >= o.x0 && x1 <= o.x1 && y0 >= o.y0 && y1 <= o.y1 && z0 >= o.z0 && z1 <= o.z1;
    }
    std::tuple<int, int, int, int, int, int> key() const { return std::make_tuple(x0, x1, y0, y1, z0, z1); }
};
}  // namespace

bool d3_build_plan(int k, int T, D1Plan *plan, int nt, int key_bytes, int NB) {
    if (k < 3 || k > D3_MAX_K || (k & 1) == 0 || T < 1 || (T & (T - 1)) || T > k || T > 16 || NB < 1 || NB > 16)
        return false;
    const int F = T + k - 1, FX = NB * T + k - 1;
    const long long n_win = (long long)k * k * k;
    Builder B;
    B.k = k;
    B.T = T;
    B.FW = F;
    auto off = [&](int fx, int fy, int fz) { return (fy * FX + fx) * F + fz; };
    std::map<std::tuple<int, int, int, int, int, int>, std::pair<Box, Ref>> memo;

    // sorted list of every window position in box b (full, never pruned)
    std::function<Ref(const Box &)> get = [&](const Box &b) -> Ref {
        auto it = memo.find(b.key());
        if (it != memo.end()) return it->second.second;
        Ref r;
        if (b.x0 == b.x1 && b.y0 == b.y1) {
            r = B.sort_gather(off(b.x0, b.y0, b.z0), 1, b.z1 - b.z0 + 1);
        } else if (b.y0 == b.y1 && b.z0 == b.z1) {
            r = B.sort_gather(off(b.x0, b.y0, b.z0), F, b.x1 - b.x0 + 1);
        } else {
            // the largest box already sorted inside b, if it is more than one line
            const long long line = std::max(b.z1 - b.z0 + 1, b.x1 - b.x0 + 1);
            const Box *best = nullptr;
            Ref best_ref{-2, 0, 0};
            long long best_vol = line;
            for (const auto &kv : memo)
                if (kv.second.first.inside(b) && kv.second.first.vol() > best_vol) {
                    best = &kv.second.first;
                    best_ref = kv.second.second;
                    best_vol = best->vol();
                }
            std::vector<Ref> parts;
            if (best) {
                const Box c = *best;
                std::vector<Box> rest;
                if (b.x0 < c.x0) rest.push_back(Box{b.x0, c.x0 - 1, b.y0, b.y1, b.z0, b.z1});
                if (c.x1 < b.x1) rest.push_back(Box{c.x1 + 1, b.x1, b.y0, b.y1, b.z0, b.z1});
                if (b.y0 < c.y0) rest.push_back(Box{c.x0, c.x1, b.y0, c.y0 - 1, b.z0, b.z1});
                if (c.y1 < b.y1) rest.push_back(Box{c.x0, c.x1, c.y1 + 1, b.y1, b.z0, b.z1});
                if (b.z0 < c.z0) rest.push_back(Box{c.x0, c.x1, c.y0, c.y1, b.z0, c.z0 - 1});
                if (c.z1 < b.z1) rest.push_back(Box{c.x0, c.x1, c.y0, c.y1, c.z1 + 1, b.z1});
                for (const Box &q : rest) parts.push_back(get(q));
                const Ref small = B.multiway(parts, 0, 1 << 30);
                r = B.merge_full(best_ref, small);
            } else {
                if (b.z1 - b.z0 >= b.x1 - b.x0) {  // z pillars
                    for (int y = b.y0; y <= b.y1; y++)
                        for (int x = b.x0; x <= b.x1; x++) parts.push_back(get(Box{x, x, y, y, b.z0, b.z1}));
                } else {  // x lines
                    for (int z = b.z0; z <= b.z1; z++)
                        for (int y = b.y0; y <= b.y1; y++) parts.push_back(get(Box{b.x0, b.x1, y, y, z, z}));
                }
                r = B.multiway(parts, 0, 1 << 30);
            }
        }
        memo[b.key()] = std::make_pair(b, r);
        return r;
    };

    struct Node {
        int o[3];  // output origin (x, y, z): x in the strip, y and z in the root tile
        Ref core;
    };
    const int SW = NB * T;
    std::vector<Ref> outs(SW * T * T);
    for (int tb = 0; tb < NB; tb++) {  // root tiles of the strip share the memoised lines and planes
        const int bx = tb * T;
        // ------------------------------------------------------ initialisation
        int t[3] = {T, T, T};
        long long c = (long long)(k - T + 1) * (k - T + 1) * (k - T + 1);
        int lo, hi;
        keep_range((int)n_win, (int)c, 0, (int)c, &lo, &hi);
        int d = lo;
        std::vector<Node> nodes;
        {
            std::vector<Ref> pillars;
            for (int y = T - 1; y <= k - 1; y++)
                for (int x = bx + T - 1; x <= bx + k - 1; x++) pillars.push_back(get(Box{x, x, y, y, T - 1, k - 1}));
            nodes.push_back(Node{{bx, 0, 0}, B.multiway(pillars, lo, hi)});
        }
        // ------------------------------------------------------ recursion
        while (t[0] * t[1] * t[2] > 1) {
            // every node keeps its extra planes sorted over its own core
            // ranges (the 2D extra rows and columns of Sec. 3.3-3.4, one
            // dimension up): a child then extends its parent's copy by the
            // new strip instead of sorting the plane again from lines
            for (const Node &nd : nodes)
                for (int a = 0; a < 3; a++) {
                    if (t[a] == 1) continue;
                    int cr[3][2];
                    for (int q = 0; q < 3; q++) {
                        cr[q][0] = nd.o[q] + t[q] - 1;
                        cr[q][1] = nd.o[q] + k - 1;
                    }
                    for (int u = nd.o[a]; u < nd.o[a] + k + t[a] - 1; u++) {
                        if (u >= cr[a][0] && u <= cr[a][1]) continue;
                        int rg[3][2] = {{cr[0][0], cr[0][1]}, {cr[1][0], cr[1][1]}, {cr[2][0], cr[2][1]}};
                        rg[a][0] = rg[a][1] = u;
                        get(Box{rg[0][0], rg[0][1], rg[1][0], rg[1][1], rg[2][0], rg[2][1]});
                    }
                }
            const int ax = (t[0] >= t[1] && t[0] >= t[2]) ? 0 : (t[1] >= t[2] ? 1 : 2);
            const int h = t[ax] / 2;
            long long other = 1;
            for (int a = 0; a < 3; a++)
                if (a != ax) other *= k - t[a] + 1;
            const int held = nodes[0].core.len;
            c += (long long)h * other;
            keep_range((int)n_win, (int)c, d, held + (int)(h * other), &lo, &hi);
            std::vector<Node> next;
            for (const Node &nd : nodes) {
                int cr[3][2];  // the parent core's ranges
                for (int a = 0; a < 3; a++) {
                    cr[a][0] = nd.o[a] + t[a] - 1;
                    cr[a][1] = nd.o[a] + k - 1;
                }
                for (int s = 0; s < 2; s++) {
                    const int u0 = s == 0 ? nd.o[ax] + h - 1 : nd.o[ax] + k;  // first new plane
                    std::vector<Ref> planes;
                    for (int u = u0; u < u0 + h; u++) {
                        int rg[3][2] = {{cr[0][0], cr[0][1]}, {cr[1][0], cr[1][1]}, {cr[2][0], cr[2][1]}};
                        rg[ax][0] = rg[ax][1] = u;
                        planes.push_back(get(Box{rg[0][0], rg[0][1], rg[1][0], rg[1][1], rg[2][0], rg[2][1]}));
                    }
                    const Ref slab = B.multiway(planes, 0, 1 << 30);
                    Node ch = nd;
                    ch.o[ax] = nd.o[ax] + s * h;
                    ch.core = B.merge_range(nd.core, slab, lo, hi);
                    next.push_back(ch);
                }
            }
            nodes.swap(next);
            t[ax] = h;
            d += lo;
        }
        for (const Node &nd : nodes) outs[(nd.o[2] * T + nd.o[1]) * SW + nd.o[0]] = nd.core;
    }
    plan->k = k;
    plan->kh = k;
    plan->T = T;
    plan->TH = T;
    plan->TD = T;
    plan->B = NB;
    plan->FW = F;   // x lines are F elements apart
    plan->FH = F;
    plan->FD = FX;  // FW * FH * FD: the footprint's element count
    return finish_plan(B, outs, F * F * FX, nt, key_bytes, plan, d1_balance((int)n_win, key_bytes, true), true);
}

void d1_pack_items(const D1Plan &plan, std::vector<D1Packed> *out) {
    out->resize(plan.work.size());
    for (size_t w = 0; w < plan.work.size(); w++) {
        const D1Task &t = plan.tasks[plan.work[w] >> 12];
        const int c = (int)(plan.work[w] & 4095u);
        int out_off = t.out_off, start = 0, cnt = 0, last = 1;
        if (t.type == D1_MERGE) {
            const int p0 = t.lo + c * t.chunk;
            cnt = std::min(t.hi - p0 + 1, t.chunk);
            start = p0;
            out_off = t.out_off + (p0 - t.lo);
            last = p0 + cnt - 1 == t.hi;
        } else if (t.type == D1_INSERT) {
            const int n = t.a_len;
            start = t.chunk ? c * t.chunk : 0;
            const int i1 = t.chunk ? std::min(n, start + t.chunk) : n;
            cnt = i1 - start;
            last = i1 == n;
        }
        const bool fw = (t.type == D1_SORT && t.a_stride == plan.FW) || (t.type == D1_INSERT && t.b_stride == plan.FW);
        D1Packed &p = (*out)[w];
        p.x = (uint32_t)t.a_off | (uint32_t)t.type << 17 | (uint32_t)fw << 19 | (uint32_t)last << 20 |
              (uint32_t)cnt << 21;
        p.y = (uint32_t)t.b_off | (uint32_t)t.a_len << 17;
        p.z = (uint32_t)out_off | (uint32_t)t.b_len << 17;
        p.w = (uint32_t)start;
    }
}

void d1_run_plan_host(const D1Plan &plan, const uint64_t *footprint, uint64_t *medians) {
    std::vector<uint64_t> sm(plan.smem_elems, 0xdeadbeefdeadbeefull);
    std::copy(footprint, footprint + (size_t)plan.FW * plan.FH * plan.FD, sm.begin());
    const int nph = (int)plan.phase_begin.size() - 1;
    std::vector<D1Packed> items;
    d1_pack_items(plan, &items);
    for (int p = 0; p < nph; p++) {
        for (int w = plan.phase_begin[p]; w < plan.phase_begin[p + 1]; w++) {
            const D1Item t = d1_unpack(items[w], plan.FW);
            if (t.type == D1_SORT) {
                std::vector<uint64_t> v(t.a_len);
                for (int i = 0; i < t.a_len; i++) v[i] = sm[t.a_off + (size_t)i * t.a_stride];
                std::sort(v.begin(), v.end());
                std::copy(v.begin(), v.end(), sm.begin() + t.out_off);
                sm[t.out_off + t.a_len] = d1_sentinel<uint64_t>();
            } else if (t.type == D1_INSERT) {
                d1_insert_any<uint64_t>(sm.data(), t);
            } else {
                d1_merge_item<uint64_t>(sm.data(), t);
            }
        }
    }
    for (size_t i = 0; i < plan.out_off.size(); i++) medians[i] = sm[plan.out_off[i]];
}

}  // namespace mf

// Host check of the data-aware schedule (declared in medianfilter.h).
extern "C" int mf_d1_plan_check_ex(int kw, int kh, int tile_w, int tile_h, int strip, int key_bytes, int threads,
                                   const uint64_t *footprint, uint64_t *medians, int *stats) {
    if ((key_bytes != 1 && key_bytes != 2 && key_bytes != 4 && key_bytes != 8) ||
        (threads != 256 && threads != 512 && threads != 1024))
        return MF_ERR_ARG;
    mf::D1Plan plan;
    if (!mf::d1_build_plan(kw, tile_w, &plan, strip, threads, key_bytes, kh, tile_h)) return MF_ERR_UNSUPPORTED;
    if (stats) {
        stats[0] = plan.smem_elems;
        stats[1] = (int)plan.phase_begin.size() - 1;
        stats[2] = (int)plan.tasks.size();
        stats[3] = (int)plan.work.size();
        stats[4] = (int)std::min<long long>(plan.merge_outputs, 2147483647ll);
        stats[5] = (int)std::min<long long>(plan.sort_elems, 2147483647ll);
        stats[6] = plan.max_sort;
    }
    if (footprint && medians) mf::d1_run_plan_host(plan, footprint, medians);
    return MF_OK;
}

extern "C" int mf_d1_plan_check_rect(int kw, int kh, int tile_w, int tile_h, int strip,
                                     const uint64_t *footprint, uint64_t *medians, int *stats) {
    return mf_d1_plan_check_ex(kw, kh, tile_w, tile_h, strip, 4, 256, footprint, medians, stats);
}

extern "C" int mf_d1_plan_check(int k, int tile, int strip, const uint64_t *footprint, uint64_t *medians,
                                int *stats) {
    return mf_d1_plan_check_rect(k, k, tile, tile, strip, footprint, medians, stats);
}

// Host check of the volumetric schedule (declared in medianfilter_volume.h).
extern "C" int mf_d3_plan_check_ex(int k, int tile, int strip, int key_bytes, int threads, const uint64_t *footprint,
                                   uint64_t *medians, int *stats) {
    if ((key_bytes != 1 && key_bytes != 2 && key_bytes != 4) || (threads != 256 && threads != 512 && threads != 1024))
        return MF_ERR_ARG;
    mf::D1Plan plan;
    if (!mf::d3_build_plan(k, tile, &plan, threads, key_bytes, strip)) return MF_ERR_UNSUPPORTED;
    if (stats) {
        stats[0] = plan.smem_elems;
        stats[1] = (int)plan.phase_begin.size() - 1;
        stats[2] = (int)plan.tasks.size();
        stats[3] = (int)plan.work.size();
        stats[4] = (int)std::min<long long>(plan.merge_outputs, 2147483647ll);
        stats[5] = (int)std::min<long long>(plan.sort_elems, 2147483647ll);
        stats[6] = plan.max_sort;
    }
    if (footprint && medians) mf::d1_run_plan_host(plan, footprint, medians);
    return MF_OK;
}

extern "C" int mf_d3_plan_check(int k, int tile, int strip, const uint64_t *footprint, uint64_t *medians,
                                int *stats) {
    return mf_d3_plan_check_ex(k, tile, strip, 4, 256, footprint, medians, stats);
}
