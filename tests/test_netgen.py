"""The network generator of the data-oblivious variant (host only).

Merging networks are checked with the 0-1 principle (a comparator network
sorts every input iff it sorts every 0/1 input), exhaustively over all
sorted 0/1 inputs; the full hierarchical networks are interpreted on the
host and compared with the CPU oracle on random tie-heavy images."""
import itertools

import numpy as np
import pytest

import oracle
from paper_2507_19926_gb300 import netgen, synth


def _merge_net(p, q):
    net = netgen.Network(0, 1, 1)
    A = [net.inp(("a", i)) for i in range(p)]
    B = [net.inp(("b", i)) for i in range(q)]
    net.outputs = net.merge(A, B)
    return net


def _run(net, env):
    vals = {}
    for desc in net.inputs:
        vals[net._memo[desc]] = env[desc]
    for kind, a, b, v in net.ops:
        vals[v] = min(vals[a], vals[b]) if kind == "min" else max(vals[a], vals[b])
    return [vals[v] for v in net.outputs]


@pytest.mark.parametrize("p", range(0, 13))
@pytest.mark.parametrize("q", range(0, 13))
def test_merge_zero_one_principle(p, q):
    net = _merge_net(p, q)
    for za in range(p + 1):
        for zb in range(q + 1):
            env = {("a", i): int(i >= za) for i in range(p)}
            env.update({("b", i): int(i >= zb) for i in range(q)})
            out = _run(net, env)
            assert out == sorted(out) and len(out) == p + q


@pytest.mark.parametrize("n", list(range(1, 18)) + [24, 33])
def test_sort_zero_one_principle(n):
    net = netgen.column_sort_network(n)
    rng = np.random.default_rng(n)
    cases = itertools.product((0, 1), repeat=n) if n <= 14 else (tuple(rng.integers(0, 2, n)) for _ in range(4000))
    for bits in cases:
        env = {("in", i): bits[i] for i in range(n)}
        out = _run(net, env)
        assert out == sorted(bits)


def test_merge_range_and_select_one():
    rng = np.random.default_rng(3)
    for _ in range(300):
        p, q = rng.integers(0, 20, 2)
        A, B = np.sort(rng.integers(0, 6, p)), np.sort(rng.integers(0, 6, q))
        n = p + q
        if n == 0:
            continue
        lo = int(rng.integers(0, n))
        hi = int(rng.integers(lo, n))
        net = netgen.Network(0, 1, 1)
        ia = [net.inp(("a", i)) for i in range(p)]
        ib = [net.inp(("b", i)) for i in range(q)]
        net.outputs = net.merge_range(ia, ib, lo, hi)
        env = {("a", i): int(A[i]) for i in range(p)}
        env.update({("b", i): int(B[i]) for i in range(q)})
        assert _run(net, env) == sorted(list(A) + list(B))[lo:hi + 1]


def test_keep_range_forgetfulness():
    # all of the window seen: exactly the median rank survives
    assert netgen.keep_range(5, 25, 0, 25) == (12, 12)
    # k = 5, 2x2 root tile: core 4x4 = 16 seen, 9 unseen -> ranks 3..12
    assert netgen.keep_range(5, 16, 0, 16) == (3, 12)
    # after dropping 3 low values the median rank among the rest is 9
    assert netgen.keep_range(5, 20, 3, 14) == (4, 9)


def test_default_tile_heuristic():
    # t(k) = 2^(floor(log2 k) - 1) lies in (k/4, k/2)
    for k in range(3, 76, 2):
        t = netgen.default_tile(k)
        assert k / 4 < t < k / 2
    assert [netgen.default_tile(k) for k in (3, 5, 7, 9, 15, 17, 31, 33, 63, 65, 75)] == \
        [1, 2, 2, 4, 4, 8, 8, 16, 16, 32, 32]


def _run_hierarchy(img, k, tw, th, net, rolled_ir=None):
    H, W = img.shape
    r = k // 2
    nty, ntx = -(-H // th), -(-W // tw)
    TY, TX = np.meshgrid(np.arange(nty), np.arange(ntx), indexing="ij")
    TY, TX = TY.ravel(), TX.ravel()
    cache = {}

    def colseg(fx):
        if fx not in cache:
            xs = np.clip(TX * tw - r + fx, 0, W - 1)
            rows = [img[np.clip(TY * th - r + fy, 0, H - 1), xs] for fy in range(th - 1, k)]
            cache[fx] = np.sort(np.stack(rows), axis=0)
        return cache[fx]

    px_fn = lambda fy, fx: img[np.clip(TY * th - r + fy, 0, H - 1), np.clip(TX * tw - r + fx, 0, W - 1)]

    def row_fn(fy, i):  # sorted extra row fy over the root core columns
        seg = np.stack([px_fn(fy, fx) for fx in range(tw - 1, k)])
        return np.sort(seg, axis=0)[i]

    if rolled_ir is not None:
        from paper_2507_19926_gb300 import rolled
        outs = rolled.interpret(net, rolled_ir, lambda fx, i: colseg(fx)[i], px_fn, row_fn)
    else:
        outs = netgen.evaluate(net, lambda fx, i: colseg(fx)[i], px_fn, row_fn)
    res = np.zeros((nty * th, ntx * tw), img.dtype)
    for i, (py, px) in enumerate([(y, x) for y in range(th) for x in range(tw)]):
        res[TY * th + py, TX * tw + px] = outs[i]
    return res[:H, :W]


@pytest.mark.parametrize("k,tw,th", [(3, 1, 1), (3, 2, 2), (5, 2, 2), (5, 4, 4), (7, 4, 4), (9, 4, 4),
                                     (9, 8, 8), (11, 4, 4), (13, 4, 4), (17, 4, 4), (7, 4, 2), (9, 2, 4)])
def test_hierarchy_matches_oracle(k, tw, th):
    net = netgen.build(k, tw, th)
    for s in range(4):
        img = (synth.levels16 if s % 2 else synth.uniform)((21, 26), "u16", 50 * k + s)
        assert np.array_equal(_run_hierarchy(img, k, tw, th, net), oracle.median_filter(img, k))


def test_op_counts_grow_like_k_log_k():
    # per-pixel ops of the heuristic tile, normalised by k log2 k, stay bounded (Sec. 4.2)
    ratios = []
    for k in (5, 9, 17):
        t = netgen.default_tile(k)
        net = netgen.build(k, t)
        cs = netgen.column_sort_network(k - t + 1)
        per_px = len(net.ops) / (t * t) + len(cs.ops) / t
        ratios.append(per_px / (k * np.log2(k)))
    assert max(ratios) / min(ratios) < 3.0


@pytest.mark.parametrize("k,tw,th", [(5, 2, 2), (9, 4, 4), (13, 4, 4), (17, 4, 4), (9, 8, 2), (7, 2, 4)])
@pytest.mark.parametrize("form", [0, 1, 6, 7])
@pytest.mark.parametrize("fuse", [False, True])
def test_rolled_network_matches_oracle(k, tw, th, form, fuse):
    """The loop-rolled form (one child per split, run for both children)
    computes exactly what the straight-line network does, with and without
    three-input min/max fusion, in every network form (root rows from
    shared memory, lazy extra rows/columns, pressure-aware order)."""
    from paper_2507_19926_gb300 import rolled
    net = netgen.build(k, tw, th, rows_smem=bool(form & 1), lazy=bool(form & 2), pressure=bool(form & 4))
    if fuse:
        fused = netgen.fuse3(net)
        assert netgen.n_minmax(fused) == netgen.n_minmax(net)
        assert len(fused.ops) < len(net.ops) or len(net.ops) < 50
        net = fused
    ir, depth = rolled.build_ir(net)
    assert depth == (tw * th).bit_length() - 1
    for s in range(2):
        img = (synth.levels16 if s else synth.uniform)((19, 22), "u16", 90 * k + s)
        want = oracle.median_filter(img, k)
        assert np.array_equal(_run_hierarchy(img, k, tw, th, net, ir), want)
        assert np.array_equal(_run_hierarchy(img, k, tw, th, net), want)
    src = rolled.emit(net, ir, "T")
    assert src.count("KO::m") < len(net.ops) or len(net.ops) < 100


@pytest.mark.parametrize("k,tw,th", [(9, 4, 4), (13, 4, 4), (17, 4, 4)])
def test_pressure_order_is_a_permutation_with_lower_peak(k, tw, th):
    """The pressure-aware order runs the same ops (a topological permutation
    of them) and never holds more values live than the demand-driven order
    when both carry the extra rows lazily."""
    a = netgen.build(k, tw, th, lazy=True)
    b = netgen.build(k, tw, th, lazy=True, pressure=True)
    assert sorted(a.ops, key=lambda o: o[3]) == sorted(b.ops, key=lambda o: o[3])
    n_in = len(b.inputs)
    seen = set(range(n_in))
    for kind, x, y, v in b.ops:
        assert x in seen and y in seen
        seen.add(v)

    def peak(net):
        last = {}
        for i, (_, x, y, _) in enumerate(net.ops):
            last[x] = last[y] = i
        for v in net.outputs:
            last[v] = len(net.ops)
        live = best = 0
        for i, (_, x, y, v) in enumerate(net.ops):
            live += 1
            best = max(best, live)
            live -= sum(1 for u in {x, y} if u >= n_in and last[u] == i)
        return best
    assert peak(b) <= peak(a)



@pytest.mark.parametrize("k,t", [(3, 1), (3, 2), (5, 1), (5, 2)])
def test_volume_network_matches_oracle(k, t):
    """The 3D data-oblivious network (hierarchical tiling over a t^3 tile of
    voxels, Sec. 7.2) evaluated on the host against the volumetric oracle,
    on many footprints with heavy ties."""
    net = netgen.build3d(k, t)
    F = t + k - 1
    vols = synth.levels16((40, F, F, F), "u16", 900 + 10 * k + t).astype(np.uint32)
    outs = netgen.evaluate3d(net, lambda fx, fy, fz: vols[:, fz, fy, fx])
    r = k // 2
    for i in range(vols.shape[0]):
        want = oracle.median_filter_3d(vols[i], k)[r:r + t, r:r + t, r:r + t].ravel()
        assert np.array_equal(np.array([o[i] for o in outs]), want), (k, t, i)
    assert all(kind in ("min", "max") for kind, _, _, _ in net.ops)
    # the emitted (pressure-aware) order computes the same
    sched = netgen.schedule_pressure(net, list(range(len(net.outputs))))
    assert sorted(op[3] for op in sched.ops) == sorted(op[3] for op in net.ops)
    souts = netgen.evaluate3d(sched, lambda fx, fy, fz: vols[:, fz, fy, fx])
    assert all(np.array_equal(a, b) for a, b in zip(outs, souts))
