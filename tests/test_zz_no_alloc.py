"""The batched entry point that allocates nothing (mf_batch_run_static).

It exists for callers that must not allocate device memory when they
filter; its work queues live in one fixed array inside the library.  This
file is collected last on purpose: if it fails, a run that stops at the
first failure has already run every other test.  It also passes on its own
in a fresh process (the first call sets up the array's address)."""
import numpy as np
import pytest

import oracle
import paper_2507_19926_gb300 as mf
from paper_2507_19926_gb300 import synth
from gpu_util import ensure_lib, same_bits, to_dev, to_host

pytestmark = pytest.mark.gpu

CODES = {"u8": mf.MF_U8, "u16": mf.MF_U16, "u32": mf.MF_U32, "f32": mf.MF_F32}
SPECS = [(1, 300, 200, "u8", 3), (2, 90, 130, "u16", 5), (1, 64, 256, "f32", 7), (3, 41, 77, "u8", 9),
         (1, 120, 90, "u32", 11), (1, 70, 333, "u16", 13), (1, 33, 40, "f32", 15), (1, 200, 150, "u8", 17),
         (2, 25, 60, "u8", 1), (1, 515, 700, "u8", 5), (2, 70, 290, "u8", 23), (1, 40, 150, "u16", 21),
         (1, 61, 83, "u32", 25), (1, 77, 95, "u8", 27), (1, 50, 70, "f32", 27)]

# work items the fixed array holds (the limit the header documents)
MAX_ITEMS = 129392


def _images(seed):
    import torch
    out = []
    for n, (C, H, W, dt, k) in enumerate(SPECS):
        a = synth.uniform((C, H, W), dt, seed + n)
        x = to_dev(a)
        out.append((a, x, torch.zeros_like(x), k, dt))
    return out


def _descs(imgs):
    return [mf.ImageDesc(x.data_ptr(), y.data_ptr(), x.shape[1], x.shape[2], x.shape[2] * x.element_size(),
                         x.shape[0], CODES[dt], k) for _, x, y, k, dt in imgs]


def test_static_batch_matches_plain_entry_point_twice():
    """Two calls in a row on different data: the first checked bit for bit
    against the CPU oracle, both against the plain entry point."""
    import torch
    ensure_lib()
    for call, seed in enumerate((700, 800)):
        imgs = _images(seed)
        mf.mf_batch_run_static(_descs(imgs), None)
        torch.cuda.synchronize()
        for a, x, y, k, dt in imgs:
            got = to_host(y, None)
            want = mf.median_filter(x, k)
            torch.cuda.synchronize()
            assert same_bits(got, to_host(want, None)), (call, x.shape, dt, k)
            if call == 0:
                assert same_bits(got, oracle.median_filter(a, k)), ("oracle", x.shape, dt, k)


def test_static_batch_rejects_what_it_cannot_hold():
    ensure_lib()
    import torch
    x = to_dev(synth.uniform((1, 16, 16), "u8", 1))
    y = torch.zeros_like(x)
    d = mf.ImageDesc(x.data_ptr(), y.data_ptr(), 16, 16, 16, 1, mf.MF_U8, 31)
    with pytest.raises(mf.MedianFilterError, match="data-oblivious"):
        mf.mf_batch_run_static([d])
    with pytest.raises(mf.MedianFilterError, match="at most 256"):
        mf.mf_batch_run_static([mf.ImageDesc(x.data_ptr(), y.data_ptr(), 16, 16, 16, 1, mf.MF_U8, 3)] * 257)
    # 60000 x 60000 needs ~3.5 million work items: rejected before any
    # device access, so these distant fake addresses are never dereferenced
    big = mf.ImageDesc(1 << 40, (1 << 40) + (8 << 30), 60000, 60000, 60000, 1, mf.MF_U8, 3)
    with pytest.raises(mf.MedianFilterError, match="work items"):
        mf.mf_batch_run_static([big])


def test_static_batch_item_limit_is_exact():
    """Exactly the documented number of work items runs; one more is
    rejected before the device is touched.  One item is one thread block's
    pixels (lanes x block width x tile width x tiles a lane runs, by block
    height x tile height, read from mf_describe), so a plane of 4 x 4 blocks
    is 16 items."""
    import re
    import torch
    ensure_lib()
    desc = mf.mf_describe(64, 64, 1, mf.MF_U8, 3)
    m = re.search(r"oblivious k=3 tile=(\d+)x(\d+) block=(\d+)x(\d+) run=(\d+) .*kernel=\S*_Ko(U16x2|U32)", desc)
    assert m, desc
    tw, th, bx, by, run = (int(v) for v in m.groups()[:5])
    lanes = 2 if m.group(6) == "U16x2" else 1
    rw, rh = lanes * bx * tw * run, by * th
    W, H = 4 * rw, 4 * rh
    planes = MAX_ITEMS // 16
    assert planes * 16 == MAX_ITEMS
    a = synth.uniform((planes, H, W), "u8", 31)
    x = to_dev(a)
    y = torch.zeros_like(x)
    full = mf.ImageDesc(x.data_ptr(), y.data_ptr(), H, W, W, planes, mf.MF_U8, 3)
    mf.mf_batch_run_static([full])
    torch.cuda.synchronize()
    got = to_host(y, None)
    for p in (0, planes // 2, planes - 1):
        assert same_bits(got[p], oracle.median_filter(a[p], 3)), p
    x1 = to_dev(synth.uniform((1, rh, rw), "u8", 32))
    y1 = torch.zeros_like(x1)
    one_more = mf.ImageDesc(x1.data_ptr(), y1.data_ptr(), rh, rw, rw, 1, mf.MF_U8, 3)
    with pytest.raises(mf.MedianFilterError, match="work items"):
        mf.mf_batch_run_static([full, one_more])


def test_static_batch_rejects_stream_capture():
    """The tables come from the caller's stack, so a captured call would
    leave the graph reading dead memory: it is refused, and the stream and
    the library stay usable."""
    import torch
    ensure_lib()
    a = synth.uniform((1, 40, 60), "u8", 33)
    x = to_dev(a)
    y = torch.zeros_like(x)
    d = mf.ImageDesc(x.data_ptr(), y.data_ptr(), 40, 60, 60, 1, mf.MF_U8, 5)
    mf.mf_batch_run_static([d])  # set-up call outside capture
    torch.cuda.synchronize()
    s = torch.cuda.Stream()
    g = torch.cuda.CUDAGraph()
    with pytest.raises(mf.MedianFilterError, match="captured"):
        with torch.cuda.graph(g, stream=s):
            mf.mf_batch_run_static([d], s.cuda_stream)
    y.zero_()
    mf.mf_batch_run_static([d])
    torch.cuda.synchronize()
    assert same_bits(to_host(y, None), oracle.median_filter(a, 5))
