"""The data-aware schedule (host side, no GPU): for each (k, root tile) the
planned sorts and merges, run on the CPU with the same merge code the kernel
uses, must give the oracle's medians for a root tile's footprint."""
import numpy as np
import pytest

import oracle
import paper_2507_19926_gb300 as mf
from paper_2507_19926_gb300 import build, synth


@pytest.fixture(scope="module", autouse=True)
def lib():
    build.build()
    mf.load_library()


CASES = [(3, 2), (5, 2), (5, 4), (7, 4), (9, 2), (9, 8), (11, 4), (13, 8), (17, 8), (17, 16),
         (21, 8), (25, 16), (31, 16), (45, 16), (61, 16), (75, 16), (75, 8), (33, 16),
         # the default 16 x 16 root tile at every odd k from 35 to 71 not listed above
         (35, 16), (37, 16), (39, 16), (41, 16), (43, 16), (47, 16), (49, 16), (51, 16), (53, 16),
         (55, 16), (57, 16), (59, 16), (63, 16), (65, 16), (67, 16), (69, 16), (71, 16), (73, 16),
         (39, 8), (55, 8), (71, 8)]


@pytest.mark.parametrize("k,T", CASES)
def test_plan_matches_oracle(k, T):
    FW = T + k - 1
    r = k // 2
    for s in range(2):
        gen = synth.levels16 if s else synth.uniform
        img = gen((FW, FW), "u16", 7 * k + T + s)
        st, med = mf.mf_d1_plan_check(k, T, img.astype(np.uint64).ravel())
        want = oracle.median_filter(img, k)[r:r + T, r:r + T].ravel()
        assert np.array_equal(med.astype(np.uint16), want), (k, T, s)
    assert st["phases"] >= 3 and st["max_sort"] <= 32


@pytest.mark.parametrize("k,T,B", [(3, 2, 8), (9, 4, 3), (17, 8, 4), (21, 8, 2), (31, 8, 2)])
def test_strip_plan_matches_oracle(k, T, B):
    """A strip of B root tiles sharing its column sorts (Sec. 3.3)."""
    FH, FW = T + k - 1, B * T + k - 1
    r = k // 2
    img = synth.levels16((FH, FW), "u8", 11 * k + B)
    st, med = mf.mf_d1_plan_check(k, T, img.astype(np.uint64).ravel(), strip=B)
    want = oracle.median_filter(img, k)[r:r + T, r:r + B * T].ravel()
    assert np.array_equal(med.astype(np.uint8), want)
    single, _ = mf.mf_d1_plan_check(k, T)
    assert st["sorted"] < B * single["sorted"]  # column sorts are shared


def test_plan_argmedian_records():
    # 64-bit records key << 32 | footprint index: the winner's index is the
    # oracle's argmedian (lowest value, then lowest row-major window slot)
    k, T = 9, 4
    FW = T + k - 1
    r = k // 2
    img = synth.levels16((FW, FW), "u8", 3).astype(np.uint64)
    rec = (img.ravel() << np.uint64(32)) | np.arange(FW * FW, dtype=np.uint64)
    _, med = mf.mf_d1_plan_check(k, T, rec)
    _, idx = oracle.median_filter(img.astype(np.uint8), k, with_idx=True)
    want = idx[r:r + T, r:r + T].ravel()
    got = (med & np.uint64(0xFFFFFFFF)).astype(np.int64)
    assert np.array_equal(got, want)


@pytest.mark.parametrize("k,T", [(5, 4), (9, 4), (17, 8), (31, 16), (45, 16)])
def test_plan_ties_at_the_largest_key(k, T):
    """Keys equal to the largest key (the value of the sentinel slot that
    follows every list) dominate the footprint, so merges run out of one
    input while the other sits at that key; the medians must still be the
    brute-force order statistic of each window (numpy sort of the k x k
    window, rank (k*k - 1) / 2)."""
    FW = T + k - 1
    top = np.uint64(0xFFFFFFFFFFFFFFFF)
    rng = np.random.default_rng(1000 + k)
    vals = np.array([0, 1, 2, 3, top], dtype=np.uint64)
    for p_top in (0.45, 0.5, 0.55, 0.9):
        img = vals[np.where(rng.random((FW, FW)) < p_top, 4, rng.integers(0, 4, (FW, FW)))]
        _, med = mf.mf_d1_plan_check(k, T, img.ravel())
        m = (k * k - 1) // 2
        want = np.array([np.sort(img[y:y + k, x:x + k].ravel())[m] for y in range(T) for x in range(T)],
                        dtype=np.uint64)
        assert np.array_equal(med, want), (k, T, p_top)


# (k, root tile, key bytes, threads): the plans the kernels run by default
# for 8-bit values (1-byte keys), 16-bit values and 8/16-bit records (2 or 4
# bytes), 32-bit values (4) and 32-bit records (8), at the block sizes the
# kernel picks for them -- their chunking, list padding, phase balancing and
# sort lengths differ from the 4-byte, 256-thread plans above.
KB_CASES = [(27, 16, 1, 256), (31, 16, 1, 256), (45, 16, 1, 256), (61, 16, 1, 256), (75, 16, 1, 512),
            (31, 16, 2, 512), (45, 16, 2, 512), (61, 16, 2, 512), (75, 16, 2, 1024), (33, 8, 4, 256),
            (45, 16, 4, 1024), (61, 8, 4, 512), (75, 8, 4, 512), (29, 8, 8, 256), (45, 8, 8, 512)]


@pytest.mark.parametrize("k,T,kb,nt", KB_CASES)
def test_plan_by_key_width_matches_oracle(k, T, kb, nt):
    FW = T + k - 1
    r = k // 2
    m = (k * k - 1) // 2
    top = np.uint64(0xFFFFFFFFFFFFFFFF)
    for s in range(3):
        if s < 2:
            gen = synth.levels16 if s else synth.uniform
            img = gen((FW, FW), "u16", 31 * k + T + kb + s)
            _, med = mf.mf_d1_plan_check(k, T, img.astype(np.uint64).ravel(), key_bytes=kb, threads=nt)
            want = oracle.median_filter(img, k)[r:r + T, r:r + T].ravel()
            assert np.array_equal(med.astype(np.uint16), want), (k, T, kb, nt, s)
        else:  # most keys equal to the sentinel value
            rng = np.random.default_rng(k + kb)
            vals = np.array([0, 1, 2, top], dtype=np.uint64)
            img = vals[np.where(rng.random((FW, FW)) < 0.55, 3, rng.integers(0, 3, (FW, FW)))]
            _, med = mf.mf_d1_plan_check(k, T, img.ravel(), key_bytes=kb, threads=nt)
            want = np.array([np.sort(img[y:y + k, x:x + k].ravel())[m] for y in range(T) for x in range(T)],
                            dtype=np.uint64)
            assert np.array_equal(med, want), (k, T, kb, nt)


def test_plan_check_ex_rejects_bad_key_width():
    with pytest.raises(mf.MedianFilterError):
        mf.mf_d1_plan_check(9, 4, key_bytes=3)
    with pytest.raises(mf.MedianFilterError):
        mf.mf_d1_plan_check(9, 4, key_bytes=4, threads=128)


def test_plan_rejects_bad_tiles():
    with pytest.raises(mf.MedianFilterError):
        mf.mf_d1_plan_check(5, 8)
    with pytest.raises(mf.MedianFilterError):
        mf.mf_d1_plan_check(9, 3)


def test_work_per_pixel_linear_in_k():
    # data-aware recursion: merged elements per pixel grow about linearly in k (Sec. 5.2)
    per = []
    for k in (17, 33, 65):
        st, _ = mf.mf_d1_plan_check(k, 16)
        per.append(st["merged"] / 256 / k)
    assert max(per) / min(per) < 2.0


RECT = [(1, 5, 1, 1, 1), (5, 1, 1, 1, 1), (3, 9, 2, 2, 1), (9, 3, 2, 2, 2), (7, 5, 4, 4, 1), (15, 5, 4, 4, 2),
        (5, 31, 4, 4, 1), (31, 9, 8, 8, 1), (25, 13, 8, 8, 2), (3, 75, 2, 2, 1), (75, 3, 2, 2, 1),
        # rectangular root tiles (t_w x t_h, Sec. 3.2)
        (31, 7, 8, 1, 1), (31, 7, 8, 2, 2), (7, 31, 1, 8, 1), (7, 31, 2, 8, 2), (1, 25, 1, 8, 1),
        (25, 1, 8, 1, 2), (15, 3, 4, 1, 1), (45, 13, 16, 4, 1), (9, 17, 2, 4, 3)]


@pytest.mark.parametrize("kw,kh,TW,TH,B", RECT)
def test_rect_plan_matches_oracle(kw, kh, TW, TH, B):
    """Windows of kw columns by kh rows and root tiles of TW x TH (paper
    Sec. 3.2 terminology for a k_w x k_h kernel and t_w x t_h tiles): the
    planned tree's medians for a strip's footprint against the oracle's
    rectangular filter."""
    FH, FW = TH + kh - 1, B * TW + kw - 1
    rx, ry = kw // 2, kh // 2
    for s in range(2):
        gen = synth.levels16 if s else synth.uniform
        img = gen((FH, FW), "u16", 13 * kw + kh + TW + TH + s)
        st, med = mf.mf_d1_plan_check(kw, TW, img.astype(np.uint64).ravel(), strip=B, kh=kh, tile_h=TH)
        want = oracle.median_filter(img, kw, kh=kh)[ry:ry + TH, rx:rx + B * TW].ravel()
        assert np.array_equal(med.astype(np.uint16), want), (kw, kh, TW, TH, B, s)


def test_rect_plan_square_case_unchanged():
    """kh = k plans exactly the k x k schedule."""
    for k, T in [(9, 4), (17, 8), (31, 16)]:
        a, _ = mf.mf_d1_plan_check(k, T)
        b, _ = mf.mf_d1_plan_check(k, T, kh=k)
        assert a == b


def test_rect_plan_rejects_tiles_beyond_the_short_side():
    with pytest.raises(mf.MedianFilterError):
        mf.mf_d1_plan_check(9, 4, kh=3)
    with pytest.raises(mf.MedianFilterError):
        mf.mf_d1_plan_check(1, 2, kh=9)


def test_slab_form_plans_match_oracle():
    """The slab form of the split cores (environment MF_D1_SLABS=1, read when
    the library loads: new cores grow from shared sorted strips plus
    per-node corner blocks) plans the same filter; checked in a fresh
    process, with and without phase balancing."""
    import os
    import subprocess
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    code = """
import numpy as np, oracle, paper_2507_19926_gb300 as mf
from paper_2507_19926_gb300 import synth
mf.load_library()
for k, T, B in [(5, 2, 1), (9, 4, 2), (17, 8, 1), (31, 16, 1), (45, 16, 1)]:
    for s in range(2):
        gen = synth.levels16 if s else synth.uniform
        FH, FW = T + k - 1, B * T + k - 1
        img = gen((FH, FW), "u16", 5 * k + T + s)
        st, med = mf.mf_d1_plan_check(k, T, img.astype(np.uint64).ravel(), strip=B)
        r = k // 2
        want = oracle.median_filter(img, k)[r:r + T, r:r + B * T].ravel()
        assert np.array_equal(med.astype(np.uint16), want), (k, T, B, s)
print("ok")
"""
    for bal in ("0", "1"):
        env = dict(os.environ, MF_D1_SLABS="1", MF_D1_BALANCE=bal, PYTHONPATH=root)
        r = subprocess.run([sys.executable, "-c", code], env=env, capture_output=True, text=True, cwd=root)
        assert r.returncode == 0 and "ok" in r.stdout, r.stderr[-2000:]
