"""The host-buffer entry point (copies inside, planes pipelined over
streams) against the oracle, with padded host pitches and several planes."""
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
