"""Helpers shared by the GPU tests: torch <-> numpy for the four dtypes, and
calls through the C ABI binding."""
import numpy as np

import paper_2507_19926_gb300 as mf

_lib_ready = False


def ensure_lib():
    global _lib_ready
    if not _lib_ready:
        from paper_2507_19926_gb300 import build
        import os
        if not os.path.exists(mf.LIB_PATH):
            build.build()
        mf.load_library()
        _lib_ready = True


def to_dev(a):
    """numpy (u8/u16/u32/f32) -> CUDA tensor of the same bits."""
    import torch
    a = np.ascontiguousarray(a)
    if a.dtype == np.uint8:
        return torch.from_numpy(a).cuda()
    if a.dtype == np.float32:
        return torch.from_numpy(a).cuda()
    if a.dtype == np.uint16:
        return torch.from_numpy(a.view(np.int16)).cuda().view(torch.uint16)
    if a.dtype == np.uint32:
        return torch.from_numpy(a.view(np.int32)).cuda().view(torch.uint32)
    raise TypeError(a.dtype)


def to_host(t, dtype):
    import torch
    t = t.contiguous()
    if t.dtype == torch.uint16:
        return t.view(torch.int16).cpu().numpy().view(np.uint16)
    if t.dtype == torch.uint32:
        return t.view(torch.int32).cpu().numpy().view(np.uint32)
    out = t.cpu().numpy()
    return out if dtype is None else out.astype(dtype, copy=False)


def gpu_filter(a, k, variant="auto", return_idx=False):
    """Runs the CUDA filter on numpy input a ((H, W) or (C, H, W))."""
    ensure_lib()
    import torch
    x = to_dev(a)
    res = mf.median_filter(x, k, variant=variant, return_idx=return_idx)
    torch.cuda.synchronize()
    if return_idx:
        y, idx = res
        return to_host(y, a.dtype), idx.cpu().numpy()
    return to_host(res, a.dtype)


def same_bits(a, b):
    return np.array_equal(np.ascontiguousarray(a).view(np.uint8), np.ascontiguousarray(b).view(np.uint8))


def f32_specials(shape, seed):
    """f32 image mixing -0, +0, +-inf, +-NaN, denormals and ordinary values."""
    from paper_2507_19926_gb300 import synth
    g = synth.rng(seed)
    bits = synth.uniform(shape, "f32", seed).view(np.uint32).copy()
    pool = np.array([0x80000000, 0x00000000, 0x7F800000, 0xFF800000, 0x7FC00000, 0xFFC00000,
                     0x7FA00001, 0x00000001, 0x80000001, 0x3F800000, 0xBF800000], np.uint32)
    m = g.random(shape) < 0.3
    bits[m] = pool[g.integers(0, len(pool), size=int(m.sum()))]
    return bits.view(np.float32)
