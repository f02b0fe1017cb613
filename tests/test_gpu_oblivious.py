"""Data-oblivious variant (paper Sec. 4) against the CPU oracle, bit for bit."""
import numpy as np
import pytest

import oracle
from paper_2507_19926_gb300 import build, synth
from gpu_util import gpu_filter, same_bits, f32_specials

pytestmark = pytest.mark.gpu

DTYPES = ["u8", "u16", "u32", "f32"]
KS = sorted(build.O1_VALUE)


@pytest.mark.parametrize("dt", DTYPES)
@pytest.mark.parametrize("k", KS)
def test_value_parity_ragged(dt, k):
    if not build.o1_covers(k, dt):
        pytest.skip("no data-oblivious kernel built for this k and dtype")
    # 77 x 203 spans several blocks in both directions with ragged tails
    for j, gen in enumerate((synth.uniform, synth.levels16)):
        x = gen((2, 77, 203), dt, 1000 + 10 * k + j)
        got = gpu_filter(x, k, "oblivious")
        want = oracle.median_filter(x, k)
        assert same_bits(got, want), (dt, k, gen.__name__)


@pytest.mark.parametrize("dt", DTYPES)
@pytest.mark.parametrize("shape", [(1, 1), (1, 37), (29, 1), (3, 4), (5, 300), (300, 6), (17, 17)])
def test_small_and_thin_shapes(dt, shape):
    for k in (3, 5, 9, 17):
        x = synth.uniform(shape, dt, 7 + k)
        assert same_bits(gpu_filter(x, k, "oblivious"), oracle.median_filter(x, k)), (dt, shape, k)


@pytest.mark.parametrize("k", KS)
def test_f32_special_values(k):
    x = f32_specials((64, 150), 99 + k)
    assert same_bits(gpu_filter(x, k, "oblivious"), oracle.median_filter(x, k))


def test_padded_pitch_and_channels():
    import torch
    from gpu_util import to_dev, to_host, ensure_lib
    import paper_2507_19926_gb300 as mf
    ensure_lib()
    x = synth.uniform((3, 50, 130), "u16", 5)
    big = to_dev(np.pad(x, ((0, 0), (0, 0), (0, 26))))  # pitch 156 elements
    view = big[:, :, :130]
    out = torch.zeros_like(big)
    _, H, W, pitch = mf._planes(view)
    mf.mf_median_filter_ex(view.data_ptr(), out.data_ptr(), H, W, pitch, 3, mf.MF_U16, 7,
                           mf.MF_BORDER_CLAMP, mf.MF_OBLIVIOUS, None, 0, None)
    torch.cuda.synchronize()
    got = to_host(out, np.uint16)
    assert np.array_equal(got[:, :, :130], oracle.median_filter(x, 7))
    assert (got[:, :, 130:] == 0).all()  # padding untouched


@pytest.mark.parametrize("dt", DTYPES)
def test_k1_identity(dt):
    x = synth.uniform((2, 33, 45), dt, 3)
    got, idx = gpu_filter(x, 1, return_idx=True)
    assert same_bits(got, x)
    assert np.array_equal(idx[0], np.arange(33 * 45, dtype=np.int32).reshape(33, 45))


@pytest.mark.parametrize("dt", DTYPES)
@pytest.mark.parametrize("k", KS)
def test_argmedian_parity(dt, k):
    # 32-bit data, and every dtype above k = 25: oblivious values + the
    # argmedian recovery pass
    if not build.o1_covers(k, dt):
        pytest.skip("no data-oblivious kernel built for this k and dtype")
    for j, gen in enumerate((synth.levels16, synth.uniform)):
        x = gen((2, 45, 170), dt, 2000 + 10 * k + j)
        got, idx = gpu_filter(x, k, "oblivious", return_idx=True)
        want, widx = oracle.median_filter(x, k, with_idx=True)
        assert same_bits(got, want)
        assert np.array_equal(idx, widx), (dt, k, gen.__name__)


def test_constant_image_argmedian_is_centre():
    x = np.full((40, 70), 9, np.uint8)
    for k in (3, 9, 17):
        _, idx = gpu_filter(x, k, "oblivious", return_idx=True)
        assert np.array_equal(idx, np.arange(40 * 70, dtype=np.int32).reshape(40, 70))


def test_photo_rgb_k17_sampled_rows():
    """The 30 MP RGB u8 workload at full size, k = 17: rows sampled for the oracle."""
    x = synth.photo_rgb()
    got = gpu_filter(x, 17)
    g = synth.rng(77)
    H = x.shape[1]
    rows = sorted(set([0, 1, 2, 8, 9, H - 10, H - 9, H - 3, H - 2, H - 1] +
                      list(g.integers(0, H, size=24))))
    want = oracle.median_filter_rows(x, 17, rows)
    assert np.array_equal(got[:, rows], want)


@pytest.mark.parametrize("dt", DTYPES)
@pytest.mark.parametrize("k", KS)
def test_every_configuration(dt, k):
    """Every instantiated network configuration of (k, dtype) -- the
    autotuner's candidates: network forms, key widths -- against the oracle
    through mf_median_filter_config, until the entry reports no more."""
    if not build.o1_covers(k, dt):
        pytest.skip("no data-oblivious kernel built for this k and dtype")
    import torch
    import paper_2507_19926_gb300 as mf
    from gpu_util import ensure_lib, to_dev, to_host
    ensure_lib()
    # rows of 290 elements (not 16-byte aligned: the wide forms read element
    # by element), and 500 of 512-element rows (aligned: the wide forms'
    # vector loads, with a ragged right edge)
    for shape, padw in (((2, 45, 290), 0), ((2, 37, 500), 12)):
        x = synth.levels16(shape, dt, 3000 + k + padw)
        want = oracle.median_filter(x, k)
        big = to_dev(np.pad(x, ((0, 0), (0, 0), (0, padw))))
        xd = big[:, :, :shape[2]]
        n = 0
        for config in range(16):
            yd = torch.zeros_like(big)
            _, H, W, pitch = mf._planes(xd)
            try:
                mf.mf_median_filter_config(xd.data_ptr(), yd.data_ptr(), H, W, pitch, 2, mf.DTYPE_CODES[dt], k,
                                           config, torch.cuda.current_stream().cuda_stream)
            except mf.MedianFilterError as e:
                assert e.status == mf.MF_ERR_UNSUPPORTED and config > 0, e
                break
            torch.cuda.synchronize()
            got = to_host(yd, None)
            assert same_bits(np.ascontiguousarray(got[:, :, :shape[2]]), want), (dt, k, config, shape)
            n += 1
    assert n >= 1
