"""Argmedian through the automatic path for every dtype and a range of k:
record-carrying networks where instantiated; for 8/16-bit data above them
the data-aware merges on (key, footprint index) records; for 32-bit data the
value kernel followed by the recovery pass (a hash lookup of the median's
source pixel, or the j-th window element equal to the median in slot
order, j = m - #below).  Tie-heavy inputs exercise the second pass."""
import numpy as np
import pytest

import oracle
from paper_2507_19926_gb300 import synth
from gpu_util import gpu_filter, same_bits

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("dt", ["u8", "u16", "u32", "f32"])
@pytest.mark.parametrize("k", [11, 17, 25, 27, 29, 31, 45, 61, 75])
def test_auto_argmedian(dt, k):
    for j, gen in enumerate((synth.levels16, synth.uniform)):
        x = gen((2, 41, 77), dt, 5000 + 10 * k + j)
        got, idx = gpu_filter(x, k, "auto", return_idx=True)
        want, widx = oracle.median_filter(x, k, with_idx=True)
        assert same_bits(got, want)
        assert np.array_equal(idx, widx), (dt, k, gen.__name__)


@pytest.mark.parametrize("k", [13, 33])
def test_constant_and_two_level_images(k):
    # constant: every window ties completely (j = m, far past the first candidates)
    x = np.full((1, 30, 50), 1234, np.uint16)
    _, idx = gpu_filter(x, k, "auto", return_idx=True)
    assert np.array_equal(idx[0], np.arange(30 * 50, dtype=np.int32).reshape(30, 50))
    g = synth.rng(k)
    y = np.where(g.random((1, 40, 60)) < 0.5, 0.25, -0.5).astype(np.float32)
    got, idx = gpu_filter(y, k, "auto", return_idx=True)
    want, widx = oracle.median_filter(y, k, with_idx=True)
    assert same_bits(got, want) and np.array_equal(idx, widx)


def test_differentiable_k25_sampled():
    """16 x 1024 x 1024 f32 at k = 25 (the differentiable workload's large
    kernel): argmedian on sampled rows of two planes."""
    x = synth.normal_f32((16, 1024, 1024), synth.SEED_BASE + 4)
    got, idx = gpu_filter(x, 25, "auto", return_idx=True)
    g = synth.rng(3)
    rows = sorted(set([0, 1, 1022, 1023] + list(g.integers(0, 1024, size=4))))
    for plane in (0, 15):
        want, widx = oracle.median_filter_rows(x[plane], 25, rows, with_idx=True)
        assert same_bits(got[plane][rows], want)
        assert np.array_equal(idx[plane][rows], widx)
