// Static schedule of the data-aware variant (paper Sec. 5).
//
// Every list length in hierarchical tiling depends only on (k, root tile),
// never on pixel values, so the whole recursion of one root tile -- which
// lists are sorted, which are merged, which output ranks each merge keeps
// -- is planned once on the host.  The plan is a sequence of phases; the
// tasks of one phase are independent and run in parallel across a thread
// block, with a barrier between phases.  Only the merges themselves are
// data-aware (merge path + sequential merge, Sec. 5.1).
#pragma once
#include <cstdint>
#include <vector>

namespace mf {

// SORT: register network over a gathered run.  MERGE: output ranks of a
// two-list merge, cut into chunks.  INSERT: a sorted list extended by up to
// D1_MAX_INSERT gathered elements (the corners a split adds to an extra row
// or column, Sec. 3.4), one thread, no merge-path search.
enum { D1_SORT = 0, D1_MERGE = 1, D1_INSERT = 2 };

// Largest corner run an INSERT task takes (each list element is compared
// with every corner, so longer runs stay merges).
constexpr int D1_MAX_INSERT = 4;

// Longest list one thread sorts with a register network (longer runs are
// sorted in even pieces and merged): keeps the kernel within 64 registers
// so a block can run 1024 threads.  The 2D plans use 16 except for 2-byte
// keys below k = 61 (mf_d1_plan.cu, d1_max_sort).
constexpr int D1_MAX_SORT = 32;

// One task.  Offsets and lengths are in list elements of shared memory.
struct D1Task {
    int32_t type;
    int32_t a_off, a_len, a_stride;  // SORT: gathers a_len elements at a_off + i*a_stride
    int32_t b_off, b_len;            // MERGE: second input (a_stride unused); INSERT: the corners
    int32_t b_stride;                // INSERT: corners gathered at b_off + i*b_stride (a list: 1)
    int32_t lo, hi;                  // MERGE: output ranks lo..hi (inclusive) of merge(A, B)
    int32_t out_off;                 // first output element
    int32_t chunk;                   // MERGE: outputs per work item
};

struct D1Plan {
    int k = 0, T = 0;                // window k columns by kh rows (kh = k: square)
    int kh = 0;
    int TH = 0;                      // root tile T columns by TH rows (TH = T: square)
    int B = 1;                       // root tiles per strip (side by side horizontally)
    int FW = 0;                      // footprint width B*T + k - 1 (footprint at offset 0, row-major)
    int FH = 0;                      // footprint height TH + kh - 1
    int FD = 1;                      // volumes: footprint depth TD + k - 1 (2D: 1)
    int TD = 1;                      // volumes: root tile depth (2D: 1)
    int nt = 256;                    // threads per block the chunking targets
    int smem_elems = 0;              // shared-memory list elements needed (footprint included)
    std::vector<D1Task> tasks;       // host form; the device gets them packed (D1Packed)
    std::vector<uint32_t> work;      // task << 12 | chunk, grouped by phase (the device gets d1_pack_items)
    std::vector<int32_t> phase_begin;  // phases + 1 entries into work
    std::vector<int32_t> out_off;    // TH * B*T: offset of each pixel's median (row-major in the strip)
    int max_sort = 0;                // longest SORT task
    long long merge_outputs = 0;     // total merged elements (work measure)
    long long sort_elems = 0;
};

// Builds the plan for a window of k columns by kh rows (kh = 0: k x k; the
// paper states its tile terminology for a k_w x k_h kernel and t_w x t_h
// tiles, Sec. 3.2) and a strip of B root tiles of T columns by TH rows
// (TH = 0: T; powers of two, 1 <= T <= min(k, 32), 1 <= TH <= min(kh, 32);
// B >= 1), chunking merges for blocks of nt threads.  The strip's footprint
// columns are sorted once and shared by its tiles (Sec. 3.3).  Returns
// false outside that range.
bool d1_build_plan(int k, int T, D1Plan *plan, int B = 1, int nt = 256, int key_bytes = 4, int kh = 0,
                   int TH = 0);

// Largest window side of the volumetric filter: list lengths and ranks of
// the packed task form stay below 2^13 (k^3 = 6859 at k = 19).
constexpr int D3_MAX_K = 19;

// Builds the plan of a k x k x k window over a strip of NB root tiles of
// T x T x T voxels side by side along x (paper Sec. 7.2: hierarchical tiling
// extended to 3D; T a power of two, 1 <= T <= min(k, 16); 1 <= NB <= 16).
// Footprint at offset 0: F = T + k - 1 in y and z, FX = NB*T + k - 1 in x,
// element (fx, fy, fz) at (fy * FX + fx) * F + fz; the plan records FW = F
// (the x-line stride), FH = F, FD = FX.  Medians in (z, y, x) order of the
// strip (NB*T wide).  Returns false outside that range or beyond the packed
// form's limits.
bool d3_build_plan(int k, int T, D1Plan *plan, int nt = 256, int key_bytes = 4, int NB = 1);

struct D1Packed;
// The 16-byte device form of every work item, in work order (layout in
// mf_d1_ops.cuh); phase_begin indexes it.
void d1_pack_items(const D1Plan &plan, std::vector<D1Packed> *out);

// Runs a plan on the host for one footprint of keys (FH*FW, row-major),
// writing the T * B*T medians (row-major).  Used by tests to check the
// schedule itself.
void d1_run_plan_host(const D1Plan &plan, const uint64_t *footprint, uint64_t *medians);

}  // namespace mf
