"""Rectangular windows (kw columns by kh rows; the paper states its tile
terminology for a k_w x k_h kernel, Sec. 3.2) through mf_median_filter_rect,
against the oracle's rectangular filter, bit for bit."""
import numpy as np
import pytest

import oracle
import paper_2507_19926_gb300 as mf
from paper_2507_19926_gb300 import synth
from gpu_util import ensure_lib, to_dev, to_host, same_bits

pytestmark = pytest.mark.gpu

SHAPES = [(1, 5), (5, 1), (3, 9), (9, 3), (7, 5), (15, 3), (5, 31), (31, 9), (1, 75), (45, 13)]


@pytest.mark.parametrize("dt", ["u8", "u16", "u32", "f32"])
@pytest.mark.parametrize("kw,kh", SHAPES)
def test_rect_value_and_argmedian(dt, kw, kh):
    import torch
    ensure_lib()
    for j, gen in enumerate((synth.uniform, synth.levels16)):
        x = gen((2, 61, 83), dt, 5000 + 100 * kw + kh + j)
        want, widx = oracle.median_filter(x, kw, kh=kh, with_idx=True)
        xd = to_dev(x)
        y, idx = mf.median_filter(xd, kw, kh=kh, return_idx=True)
        torch.cuda.synchronize()
        assert same_bits(to_host(y, None), want), (dt, kw, kh, gen.__name__)
        assert np.array_equal(idx.cpu().numpy(), widx), (dt, kw, kh, gen.__name__)
        y2 = mf.median_filter(xd, kw, kh=kh)
        torch.cuda.synchronize()
        assert same_bits(to_host(y2, None), want)


def test_rect_square_is_the_square_filter():
    import torch
    ensure_lib()
    x = synth.uniform((1, 50, 70), "u8", 9)
    xd = to_dev(x)
    a = mf.median_filter(xd, 9, kh=9)
    b = mf.median_filter(xd, 9)
    torch.cuda.synchronize()
    assert torch.equal(a, b)


def test_rect_rejects_even_and_large():
    ensure_lib()
    import torch
    xd = to_dev(synth.uniform((1, 8, 8), "u8", 1))
    yd = torch.empty_like(xd)
    for kh in (0, 4, 77):
        with pytest.raises(mf.MedianFilterError):
            mf.mf_median_filter_rect(xd.data_ptr(), yd.data_ptr(), 8, 8, 8, 1, mf.MF_U8, 3, kh)
