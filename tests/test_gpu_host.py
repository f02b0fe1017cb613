"""The host-buffer entry point (copies inside, planes cut into row bands
pipelined over streams) against the oracle, with padded host pitches,
several planes and planes of several bands."""
import ctypes

import numpy as np
import pytest

import oracle
import paper_2507_19926_gb300 as mf
from paper_2507_19926_gb300 import synth
from gpu_util import ensure_lib

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("dt,k,C", [("u8", 17, 3), ("u16", 5, 1), ("f32", 9, 4), ("u32", 31, 2), ("u8", 1, 2)])
def test_host_entry_point(dt, k, C):
    ensure_lib()
    x = synth.uniform((C, 70, 133), dt, 900 + k)
    pad = 11
    src = np.ascontiguousarray(np.pad(x, ((0, 0), (0, 0), (0, pad))))
    dst = np.zeros_like(src)
    es = src.itemsize
    mf.mf_median_filter_host(src.ctypes.data, dst.ctypes.data, 70, 133, (133 + pad) * es, C,
                             {"u8": 0, "u16": 1, "u32": 2, "f32": 3}[dt], k)
    want = oracle.median_filter(x, k)
    assert np.array_equal(dst[:, :, :133].view(np.uint8), want.view(np.uint8))
    assert (dst[:, :, 133:].view(np.uint8) == 0).all()


@pytest.mark.parametrize("dt,k,C,H,W", [("u8", 17, 2, 4500, 4096), ("u32", 31, 1, 2300, 2048),
                                        ("f32", 3, 1, 5000, 1700), ("u16", 45, 1, 2600, 3000)])
def test_host_entry_point_bands(dt, k, C, H, W):
    """Planes larger than one band (about 8 MB of input): the rows around
    every band boundary against the oracle, every row against the device
    entry point."""
    import torch
    from gpu_util import to_dev, to_host
    ensure_lib()
    x = synth.uniform((C, H, W), dt, 950 + k)
    dst = np.zeros_like(x)
    es = x.itemsize
    code = {"u8": 0, "u16": 1, "u32": 2, "f32": 3}[dt]
    mf.mf_median_filter_host(x.ctypes.data, dst.ctypes.data, H, W, W * es, C, code, k)
    bh = max(32, (8 << 20) // (W * es) // 32 * 32)
    assert bh < H  # several bands
    r = (k - 1) // 2
    rows = sorted({y for b in range(bh, H, bh) for y in range(b - r - 1, b + r + 1) if 0 <= y < H} | {0, H - 1})
    want_rows = oracle.median_filter_rows(x, k, np.array(rows, np.int32))
    assert np.array_equal(dst[:, rows, :].view(np.uint8), want_rows.view(np.uint8))
    xd = to_dev(x)
    yd = torch.empty_like(xd)
    mf.mf_median_filter(xd.data_ptr(), yd.data_ptr(), H, W, W * es, C, code, k)
    torch.cuda.synchronize()
    assert np.array_equal(dst.view(np.uint8), np.ascontiguousarray(to_host(yd, None)).view(np.uint8))
