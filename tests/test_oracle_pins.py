"""Pins of the CPU oracle against things other than itself (no GPU).

Each check is chosen so that a plausible slip in the oracle fails one of
them: a wrong rank or border rule (hand-worked fixtures, scipy), swapped
axes (non-square fixture), a wrong f32 order (numpy's float order, the f32
fixture), a wrong tie rule for the argmedian (tie-heavy fixtures, constant
images), a dropped or misplaced gradient term (hand-worked grad, central
finite differences).
"""
import glob
import json
import os

import numpy as np
import pytest

import oracle
from paper_2507_19926_gb300 import synth

GOLD = os.path.join(os.path.dirname(__file__), "golden")
pytestmark = pytest.mark.filterwarnings("ignore::DeprecationWarning")


def _load(name):
    with open(os.path.join(GOLD, name)) as f:
        return json.load(f)


@pytest.mark.parametrize("name", ["hand_3x3_ramp_k3.json", "hand_3x3_cross_k3.json",
                                  "hand_2x4_k3.json", "hand_1x6_k3.json"])
def test_hand_worked_integer(name):
    g = _load(name)
    x = np.array(g["input"], synth.NP[g["dtype"]])
    out, idx = oracle.median_filter(x, g["k"], with_idx=True)
    np.testing.assert_array_equal(out, np.array(g["output"], x.dtype))
    np.testing.assert_array_equal(idx, np.array(g["idx"], np.int32))
    grad = oracle.median_backward(np.ones(x.shape, np.float32), idx)
    np.testing.assert_array_equal(grad, np.array(g["grad_in_ones"], np.float32))
    assert grad.sum() == x.size


def test_hand_worked_f32_order():
    g = _load("hand_f32_order_k3.json")
    for case in g["cases"]:
        bits = np.array([[int(h, 16) for h in row] for row in case["input_hex"]], np.uint32)
        x = bits.view(np.float32)
        out, idx = oracle.median_filter(x, g["k"], with_idx=True)
        want = np.array([[int(h, 16) for h in row] for row in case["output_hex"]], np.uint32)
        np.testing.assert_array_equal(out.view(np.uint32), want)
        np.testing.assert_array_equal(idx, np.array(case["idx"], np.int32))


def test_f32_key_order_matches_numpy_order():
    # numpy sorts finite values and infinities numerically; -0 and +0 compare
    # equal there, so place -0 directly below +0 as the stated order does.
    vals = synth.normal_f32((2000,), 5) * np.float32(1e3)
    extra = np.array([np.inf, -np.inf, 1e-45, -1e-45, 3.4e38, -3.4e38, 1.0, -1.0],
                     np.float32)
    v = np.unique(np.concatenate([vals, extra]))
    v = v[v != 0]
    pos = np.searchsorted(v, 0)
    v = np.concatenate([v[:pos], np.array([-0.0, 0.0], np.float32), v[pos:]])
    keys = [oracle.order_key("f32", int(b)) for b in v.view(np.uint32)]
    assert all(a < b for a, b in zip(keys, keys[1:]))
    # NaNs sit outside: negative NaNs below -inf, positive NaNs above +inf
    assert oracle.order_key("f32", 0xFFC00000) < oracle.order_key("f32", 0xFF800000)
    assert oracle.order_key("f32", 0x7FC00000) > oracle.order_key("f32", 0x7F800000)


def test_k1_is_identity():
    for dt in ("u8", "u16", "u32", "f32"):
        x = synth.uniform((3, 7, 11), dt, 1)
        out, idx = oracle.median_filter(x, 1, with_idx=True)
        np.testing.assert_array_equal(out.view(np.uint8), x.view(np.uint8))
        np.testing.assert_array_equal(idx[0], np.arange(77, dtype=np.int32).reshape(7, 11))


@pytest.mark.parametrize("k", [3, 5, 9, 15])
def test_constant_image(k):
    x = np.full((6, 13), 77, np.uint16)
    out, idx = oracle.median_filter(x, k, with_idx=True)
    assert (out == 77).all()
    # lowest-value-then-lowest-slot: of k*k equal keys the rank-m one is the
    # centre slot, so every pixel is its own argmedian
    np.testing.assert_array_equal(idx, np.arange(6 * 13, dtype=np.int32).reshape(6, 13))


@pytest.mark.parametrize("dt", ["u8", "u16", "u32", "f32"])
@pytest.mark.parametrize("k", [3, 5, 7, 11])
def test_matches_scipy_nearest(dt, k):
    scipy_nd = pytest.importorskip("scipy.ndimage")
    x = synth.uniform((23, 31), dt, 100 + k)
    if dt == "f32":  # no signed zeros: scipy compares values, not bits
        x = synth.normal_f32((23, 31), 100 + k)
    want = scipy_nd.median_filter(x, size=k, mode="nearest")
    got = oracle.median_filter(x, k)
    np.testing.assert_array_equal(got, want)
    xl = synth.levels16((17, 29), dt, 200 + k)
    np.testing.assert_array_equal(oracle.median_filter(xl, k),
                                  scipy_nd.median_filter(xl, size=k, mode="nearest"))


def _window(x, y, xx, k):
    H, W = x.shape
    r = k // 2
    ys = np.clip(np.arange(y - r, y + r + 1), 0, H - 1)
    xs = np.clip(np.arange(xx - r, xx + r + 1), 0, W - 1)
    return ys, xs


def test_counting_characterisation_tiny():
    """The rank-m element v of a multiset is the one value with
    #{< v} <= m < #{<= v}; the argmedian (v, s*) has exactly m (key, slot)
    pairs below it.  Checked on many tiny tie-heavy images of every dtype."""
    for img, k in synth.tiny_cases(7, 150):
        out, idx = oracle.median_filter(img, k, with_idx=True)
        dt = [n for n, t in synth.NP.items() if img.dtype == t][0]
        keys = np.vectorize(lambda b: oracle.order_key(dt, int(b)))(
            img.view(np.uint32) if dt == "f32" else img.astype(np.uint64))
        H, W = img.shape
        m = (k * k - 1) // 2
        for y in range(H):
            for x in range(W):
                ys, xs = _window(img, y, x, k)
                win = keys[np.ix_(ys, xs)].ravel()
                src = (ys[:, None] * W + xs[None, :]).ravel()
                v = keys.ravel()[idx[y, x]]
                assert (win < v).sum() <= m < (win <= v).sum()
                assert out.view(np.uint8).reshape(H, W, -1)[y, x].tobytes() == \
                    img.view(np.uint8).reshape(H, W, -1).reshape(H * W, -1)[idx[y, x]].tobytes()
                # slot of the argmedian: the (m - #{< v})-th slot holding key v
                slots = np.nonzero(win == v)[0]
                s_star = slots[m - (win < v).sum()]
                assert src[s_star] == idx[y, x]


def test_monotone_remap_commutes():
    """Order-preserving maps commute with the median (paper Sec. 1)."""
    g = synth.rng(11)
    lut = np.sort(g.integers(0, 65536, size=256)).astype(np.uint16)
    x = synth.uniform((2, 40, 37), "u8", 12)
    for k in (3, 7, 13):
        np.testing.assert_array_equal(oracle.median_filter(lut[x], k), lut[oracle.median_filter(x, k)])
    xf = synth.normal_f32((40, 37), 13)
    for k in (5, 9):
        f = lambda a: (np.float32(4.0) * a - np.float32(1.0)).astype(np.float32)  # non-decreasing
        np.testing.assert_array_equal(oracle.median_filter(f(xf), k), f(oracle.median_filter(xf, k)))


def test_rows_sampler_matches_full():
    x = synth.uniform((2, 50, 33), "u16", 21)
    full, fidx = oracle.median_filter(x, 9, with_idx=True)
    rows = [0, 1, 17, 48, 49]
    part, pidx = oracle.median_filter_rows(x, 9, rows, with_idx=True)
    np.testing.assert_array_equal(part, full[:, rows])
    np.testing.assert_array_equal(pidx, fidx[:, rows])


def test_rejects_even_k():
    with pytest.raises(ValueError):
        oracle.median_filter(np.zeros((4, 4), np.uint8), 4)


def test_backward_finite_differences():
    """Central differences of L(x) = sum_q g_q * med_q(x) on a tie-free 64x64
    f32 N(0,1) image, k=5: moving one input to its neighbouring float (a step
    below the minimum gap between values) must change L by exactly
    (step) * sum_{q: idx[q] = p} g_q, since the median is the identity on the
    selected input between order changes."""
    x = synth.normal_f32((64, 64), synth.SEED_BASE + 4)
    v = np.sort(x.ravel())
    assert (np.diff(v) > 0).all()
    up = np.nextafter(v, np.float32(np.inf))
    assert (up[:-1] < v[1:]).all()  # a one-ulp step never reaches another value
    g = synth.rng(synth.SEED_BASE + 5).standard_normal((64, 64)).astype(np.float32)
    med, idx = oracle.median_filter(x, 5, with_idx=True)
    grad = oracle.median_backward(g, idx).astype(np.float64)
    g64 = g.astype(np.float64)
    rel_err = []
    for p in range(0, 64 * 64, 7):
        py, px = divmod(p, 64)
        xp = x.copy()
        xm = x.copy()
        xp[py, px] = np.nextafter(x[py, px], np.float32(np.inf))
        xm[py, px] = np.nextafter(x[py, px], np.float32(-np.inf))
        dp = float(xp[py, px]) - float(x[py, px])
        dm = float(x[py, px]) - float(xm[py, px])
        diff = oracle.median_filter(xp, 5).astype(np.float64) - oracle.median_filter(xm, 5).astype(np.float64)
        fd = float((g64 * diff).sum()) / (dp + dm)
        want = float(grad[py, px])
        scale = float(np.abs(g64[idx == p]).sum()) + 1e-30
        rel_err.append(abs(fd - want) / scale)
    assert max(rel_err) <= 1e-6


@pytest.mark.parametrize("dt", ["u8", "u16", "u32", "f32"])
@pytest.mark.parametrize("kw,kh", [(1, 5), (5, 1), (3, 9), (9, 3), (7, 5), (1, 1)])
def test_rect_matches_scipy_nearest(dt, kw, kh):
    """Rectangular windows (kw columns, kh rows) against scipy's median of
    size (kh, kw): swapped axes or a wrong rank fail it."""
    scipy_nd = pytest.importorskip("scipy.ndimage")
    x = synth.uniform((21, 26), dt, 300 + 10 * kw + kh)
    if dt == "f32":
        x = synth.normal_f32((21, 26), 300 + 10 * kw + kh)
    np.testing.assert_array_equal(oracle.median_filter(x, kw, kh=kh),
                                  scipy_nd.median_filter(x, size=(kh, kw), mode="nearest"))


def test_rect_one_row_is_running_sort():
    """A 1-row window is the running median of each image row: a sort of
    the clamped k-neighbourhood written out by hand."""
    x = synth.uniform((4, 19), "u16", 77)
    k = 5
    got = oracle.median_filter(x, k, kh=1)
    for y in range(4):
        for xx in range(19):
            nb = sorted(int(x[y, min(max(xx + d, 0), 18)]) for d in range(-2, 3))
            assert got[y, xx] == nb[2]


def test_rect_transpose_symmetry_and_square_case():
    """Filtering the transpose with kw, kh swapped transposes the result,
    argmedian slots map through the transpose, and kw = kh is the square
    filter."""
    x = synth.levels16((2, 23, 17), "u8", 88)
    a, ia = oracle.median_filter(x, 7, kh=3, with_idx=True)
    xt = np.ascontiguousarray(x.transpose(0, 2, 1))
    b = oracle.median_filter(xt, 3, kh=7)
    np.testing.assert_array_equal(a, b.transpose(0, 2, 1))
    np.testing.assert_array_equal(oracle.median_filter(x, 5, kh=5), oracle.median_filter(x, 5))
    # the argmedian points at a source pixel within the window holding the median value
    H, W = 23, 17
    ys, xs = ia // W, ia % W
    yy, xx = np.meshgrid(np.arange(H), np.arange(W), indexing="ij")
    assert (np.abs(ys - yy[None]) <= 1).all() and (np.abs(xs - xx[None]) <= 3).all()
    assert (np.take_along_axis(x.reshape(2, -1), ia.reshape(2, -1), 1).reshape(a.shape) == a).all()


# ---------------------------------------------------------------- volumes
# The k x k x k median of a volume (the 3D extension of hierarchical tiling,
# Sec. 7.2).  Pins: scipy's 3D median with nearest borders, a numpy brute
# force over an edge-padded volume, one slice reducing to the 2D filter, the
# cube's symmetry under axis permutations, constants and k = 1.


@pytest.mark.parametrize("dt", ["u8", "u16", "u32", "f32"])
@pytest.mark.parametrize("k", [3, 5, 7])
def test_volume_matches_scipy_nearest(dt, k):
    scipy_nd = pytest.importorskip("scipy.ndimage")
    shape = (6, 9, 13) if k < 7 else (5, 8, 11)
    x = synth.normal_f32(shape, 300 + k) if dt == "f32" else synth.uniform(shape, dt, 300 + k)
    np.testing.assert_array_equal(oracle.median_filter_3d(x, k),
                                  scipy_nd.median_filter(x, size=k, mode="nearest"))
    xl = synth.levels16(shape, dt, 400 + k)
    np.testing.assert_array_equal(oracle.median_filter_3d(xl, k),
                                  scipy_nd.median_filter(xl, size=k, mode="nearest"))


def test_volume_hand_worked_2x2x2():
    g = _load("hand_2x2x2_k3_volume.json")
    x = np.array(g["input"], synth.NP[g["dtype"]])
    np.testing.assert_array_equal(oracle.median_filter_3d(x, g["k"]), np.array(g["output"], x.dtype))


def test_volume_brute_force_edge_padded():
    """Rank (k^3-1)/2 of the window gathered from an edge-padded volume."""
    for k, shape, seed in ((3, (4, 5, 6), 1), (5, (3, 7, 4), 2), (3, (1, 1, 9), 3)):
        x = synth.levels16(shape, "u16", 500 + seed)
        r = k // 2
        p = np.pad(x, r, mode="edge")
        want = np.empty_like(x)
        for z in range(shape[0]):
            for y in range(shape[1]):
                for xx in range(shape[2]):
                    w = np.sort(p[z:z + k, y:y + k, xx:xx + k].ravel())
                    want[z, y, xx] = w[(k ** 3 - 1) // 2]
        np.testing.assert_array_equal(oracle.median_filter_3d(x, k), want)


@pytest.mark.parametrize("k", [3, 5, 9])
def test_volume_single_slice_is_2d_filter(k):
    """With one slice, clamping repeats it k times: each value of the 2D
    window appears k times, and rank (k^3-1)/2 = k*(k^2-1)/2 + (k-1)/2 falls
    in the block of copies of the 2D median (rank (k^2-1)/2)."""
    x = synth.uniform((1, 21, 34), "u8", 600 + k)
    np.testing.assert_array_equal(oracle.median_filter_3d(x, k)[0], oracle.median_filter(x[0], k))


def test_volume_axis_permutations_commute():
    x = synth.uniform((7, 10, 12), "u32", 700)
    base = oracle.median_filter_3d(x, 5)
    for perm in ((1, 0, 2), (2, 1, 0), (0, 2, 1), (1, 2, 0)):
        got = oracle.median_filter_3d(np.ascontiguousarray(x.transpose(perm)), 5)
        np.testing.assert_array_equal(got, base.transpose(perm))


def test_volume_constant_and_identity():
    c = np.full((5, 6, 7), 77, np.uint16)
    np.testing.assert_array_equal(oracle.median_filter_3d(c, 5), c)
    x = synth.uniform((2, 4, 5, 6), "f32", 800)
    np.testing.assert_array_equal(oracle.median_filter_3d(x, 1).view(np.uint32), x.view(np.uint32))
    with pytest.raises(ValueError):
        oracle.median_filter_3d(x, 4)
