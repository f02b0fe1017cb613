"""The volumetric schedule (host side, no GPU): hierarchical tiling of a
k x k x k window over a T x T x T root tile of voxels (the 3D extension the
paper names as future work, Sec. 7.2), run on the CPU with the same sort and
merge code the kernel uses, must give the oracle's medians."""
import numpy as np
import pytest

import oracle
import paper_2507_19926_gb300 as mf
from paper_2507_19926_gb300 import build, synth


@pytest.fixture(scope="module", autouse=True)
def lib():
    build.build()
    mf.load_library()


def _footprint(vol):
    # vol indexed [z, y, x]; footprint element (fx, fy, fz) at (fy*F + fx)*F + fz
    return np.ascontiguousarray(vol.transpose(1, 2, 0)).astype(np.uint64).ravel()


@pytest.mark.parametrize("k,T", [(3, 1), (3, 2), (5, 2), (5, 4), (7, 4), (9, 2), (9, 4), (11, 4), (13, 2),
                                 (15, 4), (19, 1), (19, 4)])
def test_plan_matches_oracle(k, T):
    F = T + k - 1
    r = k // 2
    for s, gen in enumerate((synth.uniform, synth.levels16)):
        vol = gen((F, F, F), "u16", 31 * k + T + s)
        st, med = mf.mf_d3_plan_check(k, T, _footprint(vol))
        want = oracle.median_filter_3d(vol, k)[r:r + T, r:r + T, r:r + T].ravel()
        assert np.array_equal(med.astype(np.uint16), want), (k, T, s)
    assert st["max_sort"] <= 32 and st["phases"] >= 3


@pytest.mark.parametrize("k,T,B", [(3, 2, 8), (5, 4, 2), (5, 4, 4), (7, 2, 4), (7, 4, 2), (9, 4, 2)])
def test_strip_plan_matches_oracle(k, T, B):
    """A strip of B root tiles along x sharing their lines and planes."""
    F, FX = T + k - 1, B * T + k - 1
    r = k // 2
    vol = synth.levels16((F, F, FX), "u16", 41 * k + B)
    st, med = mf.mf_d3_plan_check(k, T, _footprint(vol), strip=B)
    want = oracle.median_filter_3d(vol, k)[r:r + T, r:r + T, r:r + B * T].ravel()
    assert np.array_equal(med.astype(np.uint16), want), (k, T, B)
    one, _ = mf.mf_d3_plan_check(k, T)
    assert st["sorted"] < B * one["sorted"]  # shared line sorts


# (k, root tile, strip, key bytes, threads): the plans the volumetric kernel
# runs by default for 8-bit (1-byte keys), 16-bit (2) and 32-bit (4) data
VOL_CASES = [(7, 4, 2, 1, 256), (9, 4, 1, 1, 256), (15, 4, 1, 1, 512), (19, 4, 1, 1, 1024), (7, 4, 2, 2, 256),
             (7, 4, 1, 4, 256), (19, 2, 1, 4, 512)]


@pytest.mark.parametrize("k,T,B,kb,nt", VOL_CASES)
def test_plan_by_key_width_matches_oracle(k, T, B, kb, nt):
    F, FX = T + k - 1, B * T + k - 1
    r = k // 2
    for s, gen in enumerate((synth.uniform, synth.levels16)):
        vol = gen((F, F, FX), "u16", 53 * k + T + kb + s)
        _, med = mf.mf_d3_plan_check(k, T, _footprint(vol), strip=B, key_bytes=kb, threads=nt)
        want = oracle.median_filter_3d(vol, k)[r:r + T, r:r + T, r:r + B * T].ravel()
        assert np.array_equal(med.astype(np.uint16), want), (k, T, B, kb, nt, s)
    # most keys equal to the sentinel value (the largest key)
    top = np.uint64(0xFFFFFFFFFFFFFFFF)
    rng = np.random.default_rng(k + kb)
    vals = np.array([0, 1, 2, top], dtype=np.uint64)
    vol = vals[np.where(rng.random((F, F, FX)) < 0.55, 3, rng.integers(0, 3, (F, F, FX)))]
    _, med = mf.mf_d3_plan_check(k, T, _footprint(vol), strip=B, key_bytes=kb, threads=nt)
    m = (k ** 3 - 1) // 2
    want = np.array([np.sort(vol[z:z + k, y:y + k, x:x + k].ravel())[m]
                     for z in range(T) for y in range(T) for x in range(B * T)], dtype=np.uint64)
    assert np.array_equal(med, want), (k, T, B, kb, nt)


def test_plan_work_grows_slower_than_the_window():
    """Sharing the sorted core among the T^3 voxels of a root tile: merged
    elements per voxel stay below the k^3 elements of one window, and their
    ratio to k^3 falls as k grows."""
    ratios = []
    for k in (9, 15, 19):
        st, _ = mf.mf_d3_plan_check(k, 4)
        ratios.append(st["merged"] / 64 / k ** 3)
    assert ratios[0] < 1 and ratios[1] < ratios[0] and ratios[2] < ratios[1], ratios


def test_plan_rejects_bad_tiles():
    for k, T in ((3, 4), (5, 3), (21, 2), (4, 2)):
        with pytest.raises(mf.MedianFilterError):
            mf.mf_d3_plan_check(k, T)
