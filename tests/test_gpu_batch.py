"""Batched persistent launch: every image of an uneven batch equals the
CPU oracle and the plain single-image entry point, bit for bit, on every
replay of the captured graph."""
import numpy as np
import pytest

import oracle
import paper_2507_19926_gb300 as mf
from paper_2507_19926_gb300 import synth
from gpu_util import ensure_lib, to_dev, to_host

pytestmark = pytest.mark.gpu

CODES = {"u8": mf.MF_U8, "u16": mf.MF_U16, "u32": mf.MF_U32, "f32": mf.MF_F32}


def _make_batch(specs, seed):
    import torch
    imgs = []
    for n, (C, H, W, dt, k, pad) in enumerate(specs):
        x = synth.uniform((C, H, W), dt, seed + n)
        xs = to_dev(np.pad(x, ((0, 0), (0, 0), (0, pad))))
        src = xs[:, :, :W]
        dst = torch.zeros_like(xs)
        imgs.append((x, xs, src, dst, k, dt))
    descs = []
    for x, xs, src, dst, k, dt in imgs:
        C, H, W = x.shape
        pitch = xs.stride(1) * xs.element_size()
        descs.append(mf.ImageDesc(src.data_ptr(), dst.data_ptr(), H, W, pitch, C, CODES[dt], k))
    return imgs, descs


SPECS = [(1, 40, 300, "u8", 3, 0), (2, 75, 61, "u16", 5, 7), (1, 200, 33, "f32", 9, 0),
         (3, 31, 47, "u8", 17, 16), (1, 128, 128, "u32", 13, 0), (1, 90, 140, "u16", 31, 3),
         (1, 17, 19, "f32", 21, 0), (2, 50, 80, "u8", 1, 5), (1, 260, 64, "u8", 25, 0),
         (1, 9, 300, "f32", 7, 0), (1, 64, 70, "u16", 11, 2), (1, 100, 100, "u8", 29, 0)]


def test_batch_matches_oracle_and_replays():
    import torch
    ensure_lib()
    imgs, descs = _make_batch(SPECS, 500)
    plan = mf.mf_batch_plan_create(descs)
    try:
        kernels, items = mf.mf_batch_describe(plan)
        assert kernels >= 1 and items > len(SPECS)
        for rep in range(2):
            for _, _, _, dst, _, _ in imgs:
                dst.zero_()
            mf.mf_batch_run(plan, None)
            torch.cuda.synchronize()
            for x, xs, src, dst, k, dt in imgs:
                W = x.shape[2]
                got = to_host(dst, x.dtype)
                want = oracle.median_filter(x, k)
                assert np.array_equal(got[:, :, :W].view(np.uint8), want.view(np.uint8)), (rep, x.shape, dt, k)
                assert (got[:, :, W:].view(np.uint8) == 0).all()  # padding untouched
    finally:
        mf.mf_batch_plan_destroy(plan)


def test_tuned_batch_plan_matches_oracle():
    """A plan that first autotunes its (k, dtype, size bucket) groups on its
    own images (mf_batch_plan_create_ex) still filters every image exactly:
    the tuner only chooses among kernels that compute the same filter."""
    import torch
    ensure_lib()
    imgs, descs = _make_batch(SPECS, 900)
    plan = mf.mf_batch_plan_create_ex(descs, 1)
    try:
        for _, _, _, dst, _, _ in imgs:
            dst.zero_()  # tuning ran candidates into the images' own dst
        mf.mf_batch_run(plan, None)
        torch.cuda.synchronize()
        for x, xs, src, dst, k, dt in imgs:
            W = x.shape[2]
            got = to_host(dst, x.dtype)
            want = oracle.median_filter(x, k)
            assert np.array_equal(got[:, :, :W].view(np.uint8), want.view(np.uint8)), (x.shape, dt, k)
            assert (got[:, :, W:].view(np.uint8) == 0).all()
    finally:
        mf.mf_batch_plan_destroy(plan)


def test_uneven_batch_at_full_size_matches_plain_launches():
    """The 64-image batch (sizes log-uniform 256x256 .. 4096x3072, dtypes
    u8/u16/f32, odd k 3..31): each image equals its plain launch bit for bit."""
    import torch
    ensure_lib()
    descs_spec = synth.batch_descs()
    xs, ys, descs = [], [], []
    for d in descs_spec:
        x = to_dev(synth.uniform((1, d["H"], d["W"]), d["dtype"], d["seed"]))
        y = torch.zeros_like(x)
        xs.append(x)
        ys.append(y)
        descs.append(mf.ImageDesc(x.data_ptr(), y.data_ptr(), d["H"], d["W"], d["W"] * x.element_size(), 1,
                                  CODES[d["dtype"]], d["k"]))
    plan = mf.mf_batch_plan_create(descs)
    try:
        mf.mf_batch_run(plan, None)
        torch.cuda.synchronize()
        for d, x, y in zip(descs_spec, xs, ys):
            ref = mf.median_filter(x, d["k"])
            torch.cuda.synchronize()
            assert torch.equal(ref.view(torch.uint8) if ref.dtype != torch.uint8 else ref,
                               y.view(torch.uint8) if y.dtype != torch.uint8 else y), d
    finally:
        mf.mf_batch_plan_destroy(plan)
    # and a few images against the oracle on sampled rows
    g = synth.rng(9)
    for j in (0, 7, 33):
        d = descs_spec[j]
        a = synth.uniform((1, d["H"], d["W"]), d["dtype"], d["seed"])
        rows = sorted(set([0, d["H"] - 1] + list(g.integers(0, d["H"], size=4))))
        want = oracle.median_filter_rows(a, d["k"], rows)
        got = to_host(ys[j], a.dtype)
        assert np.array_equal(got[:, rows].view(np.uint8), want.view(np.uint8)), d
