"""Data-aware variant (paper Sec. 5) against the CPU oracle, bit for bit."""
import numpy as np
import pytest

import oracle
import paper_2507_19926_gb300 as mf
from paper_2507_19926_gb300 import synth
from gpu_util import ensure_lib, gpu_filter, same_bits, f32_specials, to_dev, to_host

pytestmark = pytest.mark.gpu

DTYPES = ["u8", "u16", "u32", "f32"]
KS = list(range(3, 76, 2))  # every odd k the library accepts above 1


@pytest.mark.parametrize("dt", DTYPES)
@pytest.mark.parametrize("k", KS)
def test_value_parity(dt, k):
    for j, gen in enumerate((synth.uniform, synth.levels16)):
        x = gen((2, 67, 141), dt, 3000 + 10 * k + j)
        got = gpu_filter(x, k, "data_aware")
        assert same_bits(got, oracle.median_filter(x, k)), (dt, k, gen.__name__)


@pytest.mark.parametrize("dt", DTYPES)
@pytest.mark.parametrize("k", [3, 9, 17, 25, 35, 45, 51, 59, 67, 75])
def test_argmedian_parity(dt, k):
    for j, gen in enumerate((synth.levels16, synth.uniform)):
        x = gen((1, 53, 97), dt, 4000 + 10 * k + j)
        got, idx = gpu_filter(x, k, "data_aware", return_idx=True)
        want, widx = oracle.median_filter(x, k, with_idx=True)
        assert same_bits(got, want)
        assert np.array_equal(idx, widx), (dt, k, gen.__name__)


@pytest.mark.parametrize("dt", DTYPES)
@pytest.mark.parametrize("shape", [(1, 1), (1, 40), (33, 1), (2, 3), (9, 200), (150, 5)])
def test_small_and_thin_shapes(dt, shape):
    for k in (3, 11, 31, 75):
        x = synth.uniform(shape, dt, 17 + k)
        assert same_bits(gpu_filter(x, k, "data_aware"), oracle.median_filter(x, k)), (dt, shape, k)


@pytest.mark.parametrize("k", [5, 21, 35, 47, 63, 71])
def test_f32_special_values(k):
    x = f32_specials((60, 90), 55 + k)
    assert same_bits(gpu_filter(x, k, "data_aware"), oracle.median_filter(x, k))


@pytest.mark.parametrize("k,tiles", [(9, (2, 4, 8)), (21, (2, 4, 8, 16)), (45, (8, 16)), (33, (8, 16))])
def test_every_tile_gives_the_same_result(k, tiles):
    """Each root tile size is a different tree (Sec. 3.1) but the same filter."""
    import torch
    ensure_lib()
    x = synth.uniform((1, 70, 90), "u8", 61 + k)
    want = oracle.median_filter(x, k)
    xt = to_dev(x)
    for T in tiles:
        y = torch.zeros_like(xt)
        mf.mf_median_filter_tile(xt.data_ptr(), y.data_ptr(), 70, 90, 90, 1, mf.MF_U8, k, T, None)
        torch.cuda.synchronize()
        assert np.array_equal(to_host(y, np.uint8), want), (k, T)


def test_matches_oblivious_where_both_exist():
    for k in (5, 9, 13, 17):
        x = synth.levels16((2, 80, 130), "u16", 71 + k)
        assert same_bits(gpu_filter(x, k, "data_aware"), gpu_filter(x, k, "oblivious"))


def test_sweep_size_sampled_rows():
    """4096 x 4096 at k = 45 and 75 (the sweep's largest kernels): rows sampled."""
    g = synth.rng(5)
    for dt, k in (("u8", 45), ("f32", 75)):
        x = synth.uniform((1, 4096, 4096), dt, 91 + k)
        got = gpu_filter(x, k, "data_aware")
        rows = sorted(set([0, 1, 2, 4093, 4094, 4095] + list(g.integers(0, 4096, size=6))))
        want = oracle.median_filter_rows(x, k, rows)
        assert same_bits(got[:, rows], want), (dt, k)
