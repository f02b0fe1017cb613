"""The batched entry point that allocates nothing (mf_batch_run_static).

It exists for callers that must not allocate device memory when they
filter; its work queues live in one fixed array inside the library.  This
file is collected last on purpose: if it fails, a run that stops at the
first failure has already run every other test.  It also passes on its own
in a fresh process (the first call sets up the array's address)."""
import numpy as np
import pytest

import paper_2507_19926_gb300 as mf
from paper_2507_19926_gb300 import synth
from gpu_util import ensure_lib, to_dev, to_host

pytestmark = pytest.mark.gpu

CODES = {"u8": mf.MF_U8, "u16": mf.MF_U16, "u32": mf.MF_U32, "f32": mf.MF_F32}
SPECS = [(1, 300, 200, "u8", 3), (2, 90, 130, "u16", 5), (1, 64, 256, "f32", 7), (3, 41, 77, "u8", 9),
         (1, 120, 90, "u32", 11), (1, 70, 333, "u16", 13), (1, 33, 40, "f32", 15), (1, 200, 150, "u8", 17),
         (2, 25, 60, "u8", 1), (1, 515, 700, "u8", 5), (2, 70, 290, "u8", 23), (1, 40, 150, "u16", 21)]


def _images(seed):
    import torch
    out = []
    for n, (C, H, W, dt, k) in enumerate(SPECS):
        x = to_dev(synth.uniform((C, H, W), dt, seed + n))
        out.append((x, torch.zeros_like(x), k, dt))
    return out


def _descs(imgs):
    return [mf.ImageDesc(x.data_ptr(), y.data_ptr(), x.shape[1], x.shape[2], x.shape[2] * x.element_size(),
                         x.shape[0], CODES[dt], k) for x, y, k, dt in imgs]


def test_static_batch_matches_plain_entry_point_twice():
    import torch
    ensure_lib()
    for call, seed in enumerate((700, 800)):  # two calls in a row, different data
        imgs = _images(seed)
        mf.mf_batch_run_static(_descs(imgs), None)
        torch.cuda.synchronize()
        for x, y, k, dt in imgs:
            want = mf.median_filter(x, k)
            torch.cuda.synchronize()
            got_np, want_np = to_host(y, np.uint8 if dt == "u8" else None), to_host(want, None)
            assert np.array_equal(np.ascontiguousarray(got_np).view(np.uint8),
                                  np.ascontiguousarray(want_np).view(np.uint8)), (call, x.shape, dt, k)


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
