"""Selection-network generator for the data-oblivious variant.

Builds, for a k x k kernel and a t_w x t_h root tile, the complete
min/max network that turns one root tile's footprint into its t_w*t_h
medians by hierarchical tiling (paper Sec. 3):

  * initialisation (Sec. 3.3): the footprint columns restricted to the core
    rows arrive already sorted (a block-wide column sort shares them between
    horizontally adjacent tiles); each extra row is sorted here; the core is
    a multi-way merge of the sorted core columns;
  * recursion (Sec. 3.4): a tile is split on its longer side, or on its
    width when square (Sec. 3.1).  A horizontal split merges t_w/2 extra
    columns into one list and that list into the parent's sorted core, and
    extends every extra row with its t_w/2 new corners; a vertical split is
    the same with rows and columns exchanged;
  * forgetfulness (Sec. 2.2, Fig. 3): a sorted core that covers c of the
    k*k window elements of every pixel of its tile keeps only the ranks
    that can still hold the median; extra rows and columns are never pruned.

The base networks (Sec. 4.1) are built here from textbook constructions:
Batcher's odd-even merge generalised to any two sizes, Batcher's
merge-sort for the small sorts, and a balanced tree of two-way merges for
the multi-way merge.  Every merge whose needed output ranks are known is
first trimmed to the input ranks that can reach them, and a final liveness
pass removes every comparator half whose result is never used, so a
compare-exchange becomes a lone min or max where only one side is needed.

The result is a straight-line SSA program over "values" that the CUDA
emitter turns into register code, and that ``evaluate`` interprets on the
host (numpy, vectorised over many tiles) for tests.
"""
from __future__ import annotations

import itertools
from dataclasses import dataclass, field

NEG, POS = -1, -2  # the -inf / +inf sentinels (never materialised)


@dataclass
class Network:
    k: int
    tw: int
    th: int
    # inputs: ("col", fx, i) = element i of the sorted column segment fx over
    # the root core rows; ("px", fy, fx) = raw footprint pixel
    inputs: list = field(default_factory=list)
    ops: list = field(default_factory=list)      # (kind, a, b) kind in {"min", "max"}
    outputs: list = field(default_factory=list)  # value id of each pixel (row-major in tile)
    _memo: dict = field(default_factory=dict)

    # ------------------------------------------------------------ values
    def inp(self, desc):
        v = self._memo.get(desc)
        if v is None:
            v = len(self.inputs) + len(self.ops)
            self.inputs.append(desc)
            self._ids_append(v, ("in", desc))
            self._memo[desc] = v
        return v

    def _ids_append(self, v, what):
        self._kind.append(what)

    def __post_init__(self):
        self.third = {}  # value id of a three-input op ("min3"/"max3") -> its third operand
        self._kind = []  # value id -> ("in", desc) | ("op", index)
        self.cur_path = ()   # tree path (child index per split) of ops being created
        self.op_path = {}    # value id -> tree path
        self.leaf_pixel = {}  # leaf tree path -> row-major pixel index in the tile

    def _op(self, kind, a, b):
        v = len(self._kind)
        self.ops.append((kind, a, b, v))
        self._kind.append(("op", len(self.ops) - 1))
        self.op_path[v] = self.cur_path
        return v

    def vmin(self, a, b):
        if a == NEG or b == NEG:
            return NEG
        if a == POS:
            return b
        if b == POS:
            return a
        if a == b:
            return a
        return self._op("min", a, b)

    def vmax(self, a, b):
        if a == POS or b == POS:
            return POS
        if a == NEG:
            return b
        if b == NEG:
            return a
        if a == b:
            return a
        return self._op("max", a, b)

    def cas(self, a, b):
        return self.vmin(a, b), self.vmax(a, b)

    # ------------------------------------------------------------ networks
    def merge(self, A, B):
        """Batcher's odd-even merge of two ascending lists of any lengths:
        merge the even-indexed and the odd-indexed subsequences separately
        (v, w), then compare w[i] with v[i+1]."""
        if not A:
            return list(B)
        if not B:
            return list(A)
        if len(A) == 1 and len(B) == 1:
            return list(self.cas(A[0], B[0]))
        v = self.merge(A[0::2], B[0::2])
        w = self.merge(A[1::2], B[1::2])
        out = [v[0]]
        for i in range(len(w)):
            if i + 1 < len(v):
                out.extend(self.cas(w[i], v[i + 1]))
            else:
                out.append(w[i])
        out.extend(v[len(w) + 1:])
        return out

    def merge_range(self, A, B, lo, hi):
        """Ranks lo..hi (inclusive) of merge(A, B).  Inputs that cannot
        reach those ranks are cut first: A[i] with i < lo - |B| lies below
        rank lo whatever B holds, A[i] with i > hi above rank hi."""
        n = len(A) + len(B)
        lo, hi = max(lo, 0), min(hi, n - 1)
        if lo > hi:
            return []
        a0, a1 = max(0, lo - len(B)), min(len(A) - 1, hi)
        b0, b1 = max(0, lo - len(A)), min(len(B) - 1, hi)
        As, Bs = A[a0:a1 + 1], B[b0:b1 + 1]
        off = a0 + b0
        if len(As) == 1 and len(Bs) == 0:
            return As
        if lo - off == 0 and hi - off == len(As) + len(Bs) - 1:
            return self.merge(As, Bs)
        if lo == hi and len(As) + len(Bs) > 2:
            return [self.select_one(As, Bs, lo - off)]
        return self.merge(As, Bs)[lo - off:hi - off + 1]

    def select_one(self, A, B, r):
        """Rank r of merge(A, B) as min over i + j = r + 1 of
        max(A[i-1], B[j-1]) (A[-1] = B[-1] = -inf): the rank-r element is
        the smallest x with at least r + 1 elements <= x."""
        best = POS
        for i in range(0, r + 2):
            j = r + 1 - i
            if i > len(A) or j > len(B):
                continue
            a = A[i - 1] if i > 0 else NEG
            b = B[j - 1] if j > 0 else NEG
            best = self.vmin(best, self.vmax(a, b))
        return best

    def sort(self, L):
        """Batcher's odd-even merge-sort: sort both halves, merge."""
        if len(L) <= 1:
            return list(L)
        h = len(L) // 2
        return self.merge(self.sort(L[:h]), self.sort(L[h:]))

    def multiway_range(self, lists, lo, hi):
        """Ranks lo..hi of the union of sorted lists: a balanced tree of
        two-way merges, each restricted to the ranks that can reach lo..hi
        (an element of rank j in a partial merge of p of the n elements ends
        at a rank in [j, j + n - p])."""
        lists = [l for l in lists if l]
        if not lists:
            return []
        n = sum(len(l) for l in lists)

        def rec(ls, lo_, hi_):
            # ranks lo_..hi_ (clipped) of the union of ls; returns (list, offset)
            if len(ls) == 1:
                l = ls[0]
                a, b = max(0, lo_), min(len(l) - 1, hi_)
                return l[a:b + 1], a
            h = len(ls) // 2
            L, R = ls[:h], ls[h:]
            nl, nr = sum(len(x) for x in L), sum(len(x) for x in R)
            # ranks of the left partial that can reach lo_..hi_ of the whole
            la, lb = max(0, lo_ - nr), min(nl - 1, hi_)
            ra, rb = max(0, lo_ - nl), min(nr - 1, hi_)
            PL, ol = rec(L, la, lb)
            PR, orr = rec(R, ra, rb)
            off = ol + orr
            out = self.merge_range(PL, PR, lo_ - off, hi_ - off)
            return out, max(lo_, 0)

        out, _ = rec(lists, lo, hi)
        return out


def keep_range(k, c, d, n_held):
    """Forgetfulness: with c of the k*k window elements covered by the
    held list of n_held values and d values already dropped below the
    median, the median sits at held ranks [max(0, m-d-u), min(n_held-1, m-d)]
    where m = (k*k-1)/2 and u = k*k - c is the number still unseen."""
    m = (k * k - 1) // 2
    u = k * k - c
    return max(0, m - d - u), min(n_held - 1, m - d)


def build(k, tw, th=None, rows_smem=False, lazy=False, pressure=False):
    """The full network for one root tile of tw x th pixels.  rows_smem:
    the root's extra rows arrive already sorted as inputs ("row", fy, i)
    (the kernel sorts them in a stage of its own) instead of being sorted
    inside the network -- same work, fewer values live in registers.

    lazy: an extra row (column) of a node is carried as a list of runs --
    the sorted parent row plus the groups of corner pixels that the splits
    added -- and the runs are merged only by the child whose core takes the
    row in (paper Sec. 3.4: each extra row or column joins the core of
    exactly one descendant on every path).  The same lists are merged, in a
    different tree; the merged copies are never held across a sibling's
    subtree, which keeps far fewer values live."""
    th = tw if th is None else th
    assert k % 2 == 1 and k >= 1
    assert tw >= 1 and th >= 1 and tw & (tw - 1) == 0 and th & (th - 1) == 0
    assert tw <= k and th <= k
    net = Network(k, tw, th)
    ch0 = k - th + 1  # root core height: footprint rows th-1 .. k-1

    def col_seg(fx):
        return [net.inp(("col", fx, i)) for i in range(ch0)]

    def px(fy, fx):
        return net.inp(("px", fy, fx))

    # Node state: core (sorted kept list), d (dropped low), and the sorted
    # extra rows/columns as dicts keyed by footprint row/column.
    # Footprint coordinates: pixel (py, px) of the root tile sees footprint
    # rows py .. py+k-1 and columns px .. px+k-1.
    def node_core_rect(x0, y0, tw_, th_):
        return (x0 + tw_ - 1, x0 + k - 1), (y0 + th_ - 1, y0 + k - 1)

    (cx0, cx1), (cy0, cy1) = node_core_rect(0, 0, tw, th)
    # root core: multi-way merge of the sorted core columns
    c0 = (cx1 - cx0 + 1) * (cy1 - cy0 + 1)
    core_cols = [col_seg(fx) for fx in range(cx0, cx1 + 1)]
    lo, hi = keep_range(k, c0, 0, c0)
    core = net.multiway_range(core_cols, lo, hi)
    d = lo
    # extra columns: footprint columns outside the core, over the core rows
    cols = {fx: col_seg(fx) for fx in range(0, k + tw - 1) if not (cx0 <= fx <= cx1)}
    # extra rows: footprint rows outside the core rows, over the core columns
    if rows_smem:
        rows = {fy: [net.inp(("row", fy, i)) for i in range(cx1 - cx0 + 1)]
                for fy in range(0, k + th - 1) if not (cy0 <= fy <= cy1)}
    else:
        rows = {fy: net.sort([px(fy, fx) for fx in range(cx0, cx1 + 1)])
                for fy in range(0, k + th - 1) if not (cy0 <= fy <= cy1)}
    if lazy:
        # runs: ("list", sorted ids) or ("px", [(fy, fx), ...]) still unsorted
        rows = {fy: [("list", r)] for fy, r in rows.items()}
        cols = {fx: [("list", c)] for fx, c in cols.items()}

    def runs_sorted(runs):
        return [r[1] if r[0] == "list" else net.sort([px(fy, fx) for fy, fx in r[1]]) for r in runs]

    def consume(lines):
        # sorted union of extra rows (or columns): eager lists or lazy runs
        if not lazy:
            return net.multiway_range(lines, 0, 10**9)
        return net.multiway_range([l for runs in lines for l in runs_sorted(runs)], 0, 10**9)

    outputs = {}

    def recurse(x0, y0, tw_, th_, core, d, cols, rows, path=()):
        if tw_ == 1 and th_ == 1:
            assert len(core) == 1
            outputs[(y0, x0)] = core[0]
            net.leaf_pixel[path] = y0 * tw + x0
            return
        (cx0, cx1), (cy0, cy1) = node_core_rect(x0, y0, tw_, th_)
        if tw_ >= th_:  # horizontal split: halve the width
            h = tw_ // 2
            for si, cx in enumerate((x0, x0 + h)):
                net.cur_path = path + (si,)
                ncx0, ncx1 = cx + h - 1, cx + k - 1
                new = [fx for fx in range(ncx0, ncx1 + 1) if not (cx0 <= fx <= cx1)]
                c = (ncx1 - ncx0 + 1) * (cy1 - cy0 + 1)
                extra = consume([cols[fx] for fx in new])
                lo, hi = keep_range(k, c, d, len(core) + len(extra))
                ncore = net.merge_range(core, extra, lo, hi)
                # extra columns of the child: its footprint columns outside its core
                ncols = {fx: cols[fx] for fx in range(cx, cx + h + k - 1)
                         if not (ncx0 <= fx <= ncx1)}
                # extra rows of the child: parent row + the new corners
                nrows = {}
                for fy, r in rows.items():
                    if y0 <= fy <= y0 + th_ + k - 2:
                        if lazy:
                            nrows[fy] = r + [("px", [(fy, fx) for fx in new])]
                        else:
                            corners = net.sort([px(fy, fx) for fx in new])
                            nrows[fy] = net.merge(r, corners)
                recurse(cx, y0, h, th_, ncore, d + lo, ncols, nrows, path + (si,))
                net.cur_path = path
        else:  # vertical split: halve the height
            h = th_ // 2
            for si, cy in enumerate((y0, y0 + h)):
                net.cur_path = path + (si,)
                ncy0, ncy1 = cy + h - 1, cy + k - 1
                new = [fy for fy in range(ncy0, ncy1 + 1) if not (cy0 <= fy <= cy1)]
                c = (cx1 - cx0 + 1) * (ncy1 - ncy0 + 1)
                extra = consume([rows[fy] for fy in new])
                lo, hi = keep_range(k, c, d, len(core) + len(extra))
                ncore = net.merge_range(core, extra, lo, hi)
                nrows = {fy: rows[fy] for fy in range(cy, cy + h + k - 1)
                         if not (ncy0 <= fy <= ncy1)}
                ncols = {}
                for fx, cl in cols.items():
                    if x0 <= fx <= x0 + tw_ + k - 2:
                        if lazy:
                            ncols[fx] = cl + [("px", [(fy, fx) for fy in new])]
                        else:
                            corners = net.sort([px(fy, fx) for fy in new])
                            ncols[fx] = net.merge(cl, corners)
                recurse(x0, cy, tw_, h, ncore, d + lo, ncols, nrows, path + (si,))
                net.cur_path = path

    recurse(0, 0, tw, th, core, d, cols, rows)
    net.outputs = [outputs[(y, x)] for y in range(th) for x in range(tw)]
    if pressure:
        return schedule_pressure(prune(net), leaf_order(tw, th))
    return schedule(prune(net), leaf_order(tw, th))


def prune(net):
    """Drop every op whose value no output depends on; renumber."""
    live = set(v for v in net.outputs if v >= 0)
    for kind, a, b, v in reversed(net.ops):
        if v in live:
            live.add(a)
            live.add(b)
    ops = [op for op in net.ops if op[3] in live]
    used_inputs = [i for i, desc in enumerate(net.inputs)
                   if net._memo[desc] in live]
    # renumber: inputs first (in first-use order), then ops
    order = {}
    for i in used_inputs:
        order[net._memo[net.inputs[i]]] = len(order)
    new_inputs = [net.inputs[i] for i in used_inputs]
    new_ops = []
    for kind, a, b, v in ops:
        order[v] = len(order)
        new_ops.append((kind, order[a], order[b], order[v]))
    out = Network(net.k, net.tw, net.th)
    out.inputs = new_inputs
    out.ops = new_ops
    out.outputs = [order[v] for v in net.outputs]
    out._memo = {d: order[net._memo[d]] for d in new_inputs}
    out.op_path = {order[v]: p for v, p in net.op_path.items() if v in order}
    out.leaf_pixel = dict(net.leaf_pixel)
    return out


def leaf_order(tw, th):
    """Pixels (row-major index in the tile) in the order the recursion
    reaches them (depth-first, first child first)."""
    out = []

    def rec(x0, y0, w, h):
        if w == 1 and h == 1:
            out.append(y0 * tw + x0)
            return
        if w >= h:
            rec(x0, y0, w // 2, h)
            rec(x0 + w // 2, y0, w // 2, h)
        else:
            rec(x0, y0, w, h // 2)
            rec(x0, y0 + h // 2, w, h // 2)

    rec(0, 0, tw, th)
    return out


def schedule(net, out_order):
    """Reorders the ops of a pruned network into demand-driven post-order
    (each output's dependencies just before it, outputs in out_order), which
    keeps values live for shorter spans: fewer registers for the same ops."""
    n_in = len(net.inputs)
    op_of = {v: i for i, (kind, a, b, v) in enumerate(net.ops)}
    done = set(range(n_in))
    order = []
    for o in out_order:
        stack = [(net.outputs[o], False)]
        while stack:
            v, expanded = stack.pop()
            if v in done:
                continue
            if expanded:
                done.add(v)
                order.append(net.ops[op_of[v]])
                continue
            stack.append((v, True))
            _, a, b, _ = net.ops[op_of[v]]
            for x in (b, a):
                if x not in done:
                    stack.append((x, False))
    assert len(order) == len(net.ops)
    out = Network(net.k, net.tw, net.th)
    out.inputs = net.inputs
    out.ops = order
    out.outputs = net.outputs
    out._memo = net._memo
    out.op_path = net.op_path
    out.leaf_pixel = net.leaf_pixel
    return out


def schedule_pressure(net, out_order):
    """Register-pressure-aware order.  Blocks follow the execution order of
    the split tree (a node's own ops, then its first child's subtree, then
    the second's -- the order a rolled kernel runs them in); inside a block
    a greedy list scheduler takes the ready op that ends the most live
    ranges (operands at their last use) and breaks ties by the
    demand-driven order of ``schedule``.  Same ops, fewer values live at
    once: the large networks then need fewer spill slots."""
    base = schedule(net, out_order)
    n_in = len(net.inputs)
    pos = {op[3]: i for i, op in enumerate(base.ops)}
    op_of = {op[3]: op for op in base.ops}
    remaining = {}
    for kind, a, b, v in base.ops:
        for x in {a, b}:
            if x >= n_in:
                remaining[x] = remaining.get(x, 0) + 1
    for v in base.outputs:
        if v >= n_in:
            remaining[v] = remaining.get(v, 0) + 1
    by_path = {}
    for kind, a, b, v in base.ops:
        by_path.setdefault(base.op_path[v], []).append(v)
    leaf_out = {}
    for P, pix in base.leaf_pixel.items():
        leaf_out.setdefault(P, []).append(base.outputs[pix])
    paths = set(by_path) | set(base.leaf_pixel)
    order = []
    done = set(range(n_in))

    def run_block(P):
        todo = set(by_path.get(P, ()))
        users = {}
        for v in todo:
            _, a, b, _ = op_of[v]
            for x in {a, b}:
                if x in todo:
                    users.setdefault(x, []).append(v)
        waiting = {v: sum(1 for x in {op_of[v][1], op_of[v][2]} if x in todo) for v in todo}
        ready = [v for v in todo if waiting[v] == 0]
        while ready:
            best, best_key = None, None
            for v in ready:
                _, a, b, _ = op_of[v]
                freed = sum(1 for x in {a, b} if x >= n_in and remaining[x] == 1)
                key = (-freed, pos[v])
                if best_key is None or key < best_key:
                    best, best_key = v, key
            ready.remove(best)
            order.append(op_of[best])
            done.add(best)
            _, a, b, _ = op_of[best]
            for x in {a, b}:
                if x >= n_in:
                    remaining[x] -= 1
            for u in users.get(best, ()):
                waiting[u] -= 1
                if waiting[u] == 0:
                    ready.append(u)
        for v in leaf_out.get(P, ()):
            if v >= n_in:
                remaining[v] -= 1
        for c in (0, 1):
            if any(q[:len(P) + 1] == P + (c,) for q in paths):
                run_block(P + (c,))

    run_block(())
    assert len(order) == len(base.ops)
    out = Network(net.k, net.tw, net.th)
    out.inputs = base.inputs
    out.ops = order
    out.outputs = base.outputs
    out._memo = base._memo
    out.op_path = base.op_path
    out.leaf_pixel = base.leaf_pixel
    return out


def fuse3(net):
    """Fuses an op into its only user when both are the same kind:
    v = min(min(a, b), c) becomes one three-input min3(a, b, c) (a single
    instruction on sm_100+, at the two-input rate).  Runs on a pruned,
    scheduled network; keeps ids, order and tree paths."""
    uses = {}
    for kind, a, b, v in net.ops:
        uses[a] = uses.get(a, 0) + 1
        uses[b] = uses.get(b, 0) + 1
    for v in net.outputs:
        uses[v] = uses.get(v, 0) + 1
    kind_of = {v: kind for kind, a, b, v in net.ops}
    src = {v: (a, b) for kind, a, b, v in net.ops}
    path = net.op_path
    absorbed, new_ops, third = set(), [], {}
    for kind, a, b, v in net.ops:
        if kind in ("min", "max"):
            for x, y in ((a, b), (b, a)):
                # same kind, used once, same tree path (keeps both children of
                # every split structurally identical for loop rolling)
                if (kind_of.get(x) == kind and uses.get(x) == 1 and x not in absorbed
                        and x not in third and path.get(x) == path.get(v)):
                    absorbed.add(x)
                    xa, xb = src[x]
                    kind, a, b = kind + "3", xa, xb
                    third[v] = y
                    break
        new_ops.append((kind, a, b, v))
    new_ops = [op for op in new_ops if op[3] not in absorbed]
    live = {v for _, _, _, v in new_ops}
    n_in = len(net.inputs)
    for kind, a, b, v in new_ops:  # nothing may refer to an absorbed op
        assert all(x < n_in or x in live for x in (a, b, third.get(v, a)))
    out = Network(net.k, net.tw, net.th)
    out.inputs = net.inputs
    out.ops = new_ops
    out.outputs = net.outputs
    out._memo = net._memo
    out.op_path = {v: p for v, p in net.op_path.items() if v in live}
    out.leaf_pixel = net.leaf_pixel
    out.third = third
    return out


def n_minmax(net):
    """Element min/max operations of a network (a three-input op counts 2)."""
    return sum(2 if kind.endswith("3") else 1 for kind, _, _, _ in net.ops)


def evaluate(net, col_fn, px_fn, row_fn=None):
    """Run the network on the host.  col_fn(fx, i), px_fn(fy, fx) and
    row_fn(fy, i) return numpy arrays (one entry per tile instance);
    returns the outputs."""
    import numpy as np
    top = max([v for _, _, _, v in net.ops], default=-1) + 1
    vals = [None] * max(top, len(net.inputs) + len(net.ops))
    for i, desc in enumerate(net.inputs):
        f = {"col": col_fn, "px": px_fn, "row": row_fn}[desc[0]]
        vals[i] = f(desc[1], desc[2])
    for kind, a, b, v in net.ops:
        f = np.minimum if kind.startswith("min") else np.maximum
        vals[v] = f(vals[a], vals[b])
        if kind.endswith("3"):
            vals[v] = f(vals[v], vals[net.third[v]])
    return [vals[v] for v in net.outputs]


def column_sort_network(n):
    """The block-wide column sort: a full sort of n values (ascending)."""
    net = Network(0, 1, 1)
    ins = [net.inp(("in", i)) for i in range(n)]
    net.outputs = net.sort(ins)
    return prune(net)


def count(net):
    return len(net.ops)


def default_tile(k):
    """Root tile heuristic t(k) = 2^(floor(log2 k) - 1) (paper Sec. 4.2)."""
    return max(1, 1 << (k.bit_length() - 2)) if k >= 2 else 1


def build3d(k, t):
    """Data-oblivious network of the k x k x k median over a t x t x t tile
    of voxels: hierarchical tiling extended to 3D (the paper's future work,
    Sec. 7.2), with the tree of the volumetric data-aware plan.  Inputs
    ("v", fx, fy, fz) are footprint voxels (F = t + k - 1 a side); outputs
    are the t^3 medians in (z, y, x) order.

    A node of tx x ty x tz outputs holds its core -- the box of window
    positions all its outputs share -- sorted and pruned by forgetfulness
    over n = k^3 (Sec. 2.2).  A split halves the longest side (x, y, z on
    ties); a child merges into the parent's core the planes of window
    positions on its side over the parent core's other two ranges.  Every
    node keeps its extra planes sorted over its own core ranges, so a
    child's plane is its parent's plane merged with the strip its split
    added (the 2D extra rows and columns of Sec. 3.3-3.4, one dimension up).
    Sorted boxes are memoised; a box is the largest sorted box inside it
    merged with the sorted remainder, or a merge of sorted z pillars / x
    lines."""
    net = Network(k, t, t)
    n = k ** 3
    m = (n - 1) // 2
    memo = {}

    def inside(a, b):
        return a[0] >= b[0] and a[1] <= b[1] and a[2] >= b[2] and a[3] <= b[3] and a[4] >= b[4] and a[5] <= b[5]

    def vol(b):
        return (b[1] - b[0] + 1) * (b[3] - b[2] + 1) * (b[5] - b[4] + 1)

    def get(b):
        if b in memo:
            return memo[b]
        x0, x1, y0, y1, z0, z1 = b
        if (x0 == x1 and y0 == y1) or (y0 == y1 and z0 == z1):  # one line
            r = net.sort([net.inp(("v", x, y, z)) for z in range(z0, z1 + 1)
                          for y in range(y0, y1 + 1) for x in range(x0, x1 + 1)])
        else:
            line = max(z1 - z0 + 1, x1 - x0 + 1)
            best = None
            for c in memo:
                if inside(c, b) and vol(c) > line and (best is None or vol(c) > vol(best)):
                    best = c
            if best is not None:
                c = best
                rest = []
                if x0 < c[0]: rest.append((x0, c[0] - 1, y0, y1, z0, z1))
                if c[1] < x1: rest.append((c[1] + 1, x1, y0, y1, z0, z1))
                if y0 < c[2]: rest.append((c[0], c[1], y0, c[2] - 1, z0, z1))
                if c[3] < y1: rest.append((c[0], c[1], c[3] + 1, y1, z0, z1))
                if z0 < c[4]: rest.append((c[0], c[1], c[2], c[3], z0, c[4] - 1))
                if c[5] < z1: rest.append((c[0], c[1], c[2], c[3], c[5] + 1, z1))
                small = net.multiway_range([get(q) for q in rest], 0, 1 << 30)
                r = net.merge(memo[c], small)
            elif z1 - z0 >= x1 - x0:
                r = net.multiway_range([get((x, x, y, y, z0, z1)) for y in range(y0, y1 + 1)
                                        for x in range(x0, x1 + 1)], 0, 1 << 30)
            else:
                r = net.multiway_range([get((x0, x1, y, y, z, z)) for z in range(z0, z1 + 1)
                                        for y in range(y0, y1 + 1)], 0, 1 << 30)
        memo[b] = r
        return r

    def keep(c, d, held):
        return max(0, m - d - (n - c)), min(held - 1, m - d)

    ts = [t, t, t]
    c = (k - t + 1) ** 3
    lo, hi = keep(c, 0, c)
    d = lo
    pillars = [get((x, x, y, y, t - 1, k - 1)) for y in range(t - 1, k) for x in range(t - 1, k)]
    nodes = [((0, 0, 0), net.multiway_range(pillars, lo, hi))]
    while ts[0] * ts[1] * ts[2] > 1:
        for o, _ in nodes:  # extra planes of every node, over its own core ranges
            cr = [(o[a] + ts[a] - 1, o[a] + k - 1) for a in range(3)]
            for a in range(3):
                if ts[a] == 1:
                    continue
                for u in range(o[a], o[a] + k + ts[a] - 1):
                    if cr[a][0] <= u <= cr[a][1]:
                        continue
                    rg = list(cr)
                    rg[a] = (u, u)
                    get((rg[0][0], rg[0][1], rg[1][0], rg[1][1], rg[2][0], rg[2][1]))
        ax = 0 if ts[0] >= ts[1] and ts[0] >= ts[2] else (1 if ts[1] >= ts[2] else 2)
        h = ts[ax] // 2
        other = 1
        for a in range(3):
            if a != ax:
                other *= k - ts[a] + 1
        held = len(nodes[0][1])
        c += h * other
        lo, hi = keep(c, d, held + h * other)
        nxt = []
        for o, core in nodes:
            cr = [(o[a] + ts[a] - 1, o[a] + k - 1) for a in range(3)]
            for s in range(2):
                u0 = o[ax] + h - 1 if s == 0 else o[ax] + k
                planes = []
                for u in range(u0, u0 + h):
                    rg = list(cr)
                    rg[ax] = (u, u)
                    planes.append(get((rg[0][0], rg[0][1], rg[1][0], rg[1][1], rg[2][0], rg[2][1])))
                slab = net.multiway_range(planes, 0, 1 << 30)
                co = list(o)
                co[ax] = o[ax] + s * h
                nxt.append((tuple(co), net.merge_range(core, slab, lo, hi)))
        nodes = nxt
        ts[ax] = h
        d += lo
    out = [None] * t ** 3
    for o, core in nodes:
        assert len(core) == 1
        out[(o[2] * t + o[1]) * t + o[0]] = core[0]
    net.outputs = out
    return prune(net)


def evaluate3d(net, vox_fn):
    """Run a build3d network on the host; vox_fn(fx, fy, fz) returns a numpy
    array (one entry per tile instance).  Returns the outputs."""
    import numpy as np
    vals = [None] * (len(net.inputs) + len(net.ops))
    for i, desc in enumerate(net.inputs):
        vals[i] = vox_fn(desc[1], desc[2], desc[3])
    for kind, a, b, v in net.ops:
        vals[v] = (np.minimum if kind == "min" else np.maximum)(vals[a], vals[b])
    return [vals[v] for v in net.outputs]
