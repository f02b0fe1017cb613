"""GB300-native k x k median filter by hierarchical tiling (arXiv 2507.19926).

Thin Python binding of ``libmedianfilter.so`` (C ABI in
``include/medianfilter.h``).  The ``mf_*`` functions take raw pointers and
sizes exactly like their C counterparts; ``median_filter`` /
``median_filter_backward`` / ``MedianFilterFn`` marshal torch tensors into
those calls (pointers, pitch, the current CUDA stream).  All computation
runs in the library's CUDA kernels: there is no CPU or PyTorch fallback, and
every call raises if the library is missing or returns an error.
"""
from __future__ import annotations

import ctypes
import os
import threading

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libmedianfilter.so")

MF_U8, MF_U16, MF_U32, MF_F32 = 0, 1, 2, 3
DTYPE_CODES = {"u8": MF_U8, "u16": MF_U16, "u32": MF_U32, "f32": MF_F32}
MF_ERR_UNSUPPORTED = -9
MF_BORDER_CLAMP = 0
MF_AUTO, MF_OBLIVIOUS, MF_DATA_AWARE = 0, 1, 2
MF_GRAD_ATOMIC, MF_GRAD_DETERMINISTIC = 0, 1
VARIANTS = {"auto": MF_AUTO, "oblivious": MF_OBLIVIOUS, "data_aware": MF_DATA_AWARE}
GRAD_MODES = {"atomic": MF_GRAD_ATOMIC, "deterministic": MF_GRAD_DETERMINISTIC}

# C symbols declared in include/medianfilter.h and include/medianfilter_volume.h
EXPORTS = ["mf_median_filter", "mf_median_filter_ex", "mf_median_filter_tile", "mf_median_filter_config",
           "mf_median_filter_rect", "mf_d1_plan_check_rect", "mf_d1_plan_check_ex",
           "mf_median_filter_bwd",
           "mf_median_filter_host", "mf_batch_plan_create", "mf_batch_plan_create_ex", "mf_batch_run",
           "mf_batch_plan_destroy", "mf_batch_describe", "mf_batch_run_static", "mf_autotune", "mf_describe", "mf_kernel_launch_count",
           "mf_status_string", "mf_last_error", "mf_version", "mf_shutdown", "mf_probe_minmax",
           "mf_d1_plan_check",
           # include/medianfilter_volume.h
           "mf_median_filter_3d", "mf_median_filter_3d_ex", "mf_median_filter_3d_describe", "mf_d3_plan_check",
           "mf_d3_plan_check_ex"]


class MedianFilterError(RuntimeError):
    """A non-zero mf_status; .status holds the code."""
    status = 0


class ImageDesc(ctypes.Structure):
    """mf_image_desc."""
    _fields_ = [("src", ctypes.c_void_p), ("dst", ctypes.c_void_p), ("H", ctypes.c_int),
                ("W", ctypes.c_int), ("pitch", ctypes.c_size_t), ("channels", ctypes.c_int),
                ("dtype", ctypes.c_int), ("k", ctypes.c_int)]


_lock = threading.Lock()
_lib = None


def load_library(path=LIB_PATH):
    """Loads libmedianfilter.so (raises if it has not been built)."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        if not os.path.exists(path):
            raise MedianFilterError(
                "libmedianfilter.so not built (%s); run paper_2507_19926_gb300.build.build()" % path)
        lib = ctypes.CDLL(path)
        vp, i, sz, u64 = ctypes.c_void_p, ctypes.c_int, ctypes.c_size_t, ctypes.c_uint64
        lib.mf_median_filter.argtypes = [vp, vp, i, i, sz, i, i, i, i, vp]
        lib.mf_median_filter_ex.argtypes = [vp, vp, i, i, sz, i, i, i, i, i, vp, sz, vp]
        lib.mf_median_filter_tile.argtypes = [vp, vp, i, i, sz, i, i, i, i, vp]
        lib.mf_median_filter_config.argtypes = [vp, vp, i, i, sz, i, i, i, i, vp]
        lib.mf_median_filter_rect.argtypes = [vp, vp, i, i, sz, i, i, i, i, vp, sz, vp]
        lib.mf_d1_plan_check_rect.argtypes = [i, i, i, i, i, vp, vp, vp]
        lib.mf_d1_plan_check_ex.argtypes = [i, i, i, i, i, i, i, vp, vp, vp]
        lib.mf_median_filter_bwd.argtypes = [vp, vp, vp, i, i, sz, sz, i, i, i, vp]
        lib.mf_median_filter_host.argtypes = [vp, vp, i, i, sz, i, i, i, i, i, vp]
        lib.mf_batch_plan_create.argtypes = [ctypes.POINTER(ImageDesc), i, ctypes.POINTER(vp)]
        lib.mf_batch_plan_create_ex.argtypes = [ctypes.POINTER(ImageDesc), i, i, ctypes.POINTER(vp)]
        lib.mf_batch_run.argtypes = [vp, vp]
        lib.mf_batch_plan_destroy.argtypes = [vp]
        lib.mf_batch_run_static.argtypes = [ctypes.POINTER(ImageDesc), i, vp]
        lib.mf_batch_describe.argtypes = [vp, ctypes.POINTER(i), ctypes.POINTER(ctypes.c_longlong)]
        lib.mf_autotune.argtypes = [vp, vp, i, i, sz, i, i, i, vp]
        lib.mf_describe.argtypes = [i, i, i, i, i, i, ctypes.c_char_p, sz]
        lib.mf_kernel_launch_count.restype = u64
        lib.mf_probe_minmax.argtypes = [i, i, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_double)]
        lib.mf_d1_plan_check.argtypes = [i, i, i, vp, vp, vp]
        lib.mf_median_filter_3d.argtypes = [vp, vp, i, i, i, sz, i, i, i, vp]
        lib.mf_median_filter_3d_ex.argtypes = [vp, vp, i, i, i, sz, i, i, i, i, vp]
        lib.mf_median_filter_3d_describe.argtypes = [i, i, ctypes.c_char_p, sz]
        lib.mf_d3_plan_check.argtypes = [i, i, i, vp, vp, vp]
        lib.mf_d3_plan_check_ex.argtypes = [i, i, i, i, i, vp, vp, vp]
        lib.mf_status_string.argtypes = [i]
        lib.mf_status_string.restype = ctypes.c_char_p
        lib.mf_last_error.restype = ctypes.c_char_p
        lib.mf_version.restype = ctypes.c_char_p
        for name in EXPORTS:
            if not hasattr(lib, name):
                raise MedianFilterError("symbol %s missing from %s" % (name, path))
        _lib = lib
    return _lib


def _check(rc):
    if rc != 0:
        lib = load_library()
        err = MedianFilterError("%s: %s" % (lib.mf_status_string(rc).decode(),
                                            lib.mf_last_error().decode()))
        err.status = rc
        raise err
    return rc


# ------------------------------------------------------------ raw C ABI
def mf_median_filter(src, dst, H, W, pitch, channels, dtype, k, border=MF_BORDER_CLAMP, stream=None):
    return _check(load_library().mf_median_filter(src, dst, H, W, pitch, channels, dtype, k, border, stream))


def mf_median_filter_ex(src, dst, H, W, pitch, channels, dtype, k, border, variant, argidx,
                        idx_pitch, stream=None):
    return _check(load_library().mf_median_filter_ex(src, dst, H, W, pitch, channels, dtype, k, border,
                                                     variant, argidx, idx_pitch, stream))


def mf_median_filter_tile(src, dst, H, W, pitch, channels, dtype, k, tile, stream=None):
    return _check(load_library().mf_median_filter_tile(src, dst, H, W, pitch, channels, dtype, k, tile,
                                                       stream))


def mf_median_filter_rect(src, dst, H, W, pitch, channels, dtype, kw, kh, argidx=None, idx_pitch=0,
                          stream=None):
    return _check(load_library().mf_median_filter_rect(src, dst, H, W, pitch, channels, dtype, kw, kh, argidx,
                                                       idx_pitch, stream))


def mf_median_filter_config(src, dst, H, W, pitch, channels, dtype, k, config, stream=None):
    return _check(load_library().mf_median_filter_config(src, dst, H, W, pitch, channels, dtype, k, config,
                                                         stream))


def mf_median_filter_bwd(grad_out, argidx, grad_in, H, W, pitch, idx_pitch, channels, k, mode,
                         stream=None):
    return _check(load_library().mf_median_filter_bwd(grad_out, argidx, grad_in, H, W, pitch,
                                                      idx_pitch, channels, k, mode, stream))


def mf_median_filter_host(src_host, dst_host, H, W, pitch, channels, dtype, k,
                          border=MF_BORDER_CLAMP, variant=MF_AUTO, stream=None):
    return _check(load_library().mf_median_filter_host(src_host, dst_host, H, W, pitch, channels,
                                                        dtype, k, border, variant, stream))


def mf_batch_plan_create(descs):
    """descs: list of ImageDesc; returns an opaque plan handle."""
    arr = (ImageDesc * len(descs))(*descs)
    out = ctypes.c_void_p()
    _check(load_library().mf_batch_plan_create(arr, len(descs), ctypes.byref(out)))
    return out


def mf_batch_plan_create_ex(descs, tune):
    """As mf_batch_plan_create; tune != 0 autotunes the batch's missing
    (k, dtype, size bucket) entries on its own images first."""
    arr = (ImageDesc * len(descs))(*descs)
    out = ctypes.c_void_p()
    _check(load_library().mf_batch_plan_create_ex(arr, len(descs), int(tune), ctypes.byref(out)))
    return out


def mf_batch_run(plan, stream=None):
    return _check(load_library().mf_batch_run(plan, stream))


def mf_batch_plan_destroy(plan):
    return _check(load_library().mf_batch_plan_destroy(plan))


def mf_batch_run_static(descs, stream=None):
    """Filters a batch without allocating: work queues live in the library's
    fixed device array (see include/medianfilter.h for the limits)."""
    arr = (ImageDesc * len(descs))(*descs)
    return _check(load_library().mf_batch_run_static(arr, len(descs), stream))


def mf_batch_describe(plan):
    """(kernel launches per run, work items) of a batch plan."""
    k, n = ctypes.c_int(), ctypes.c_longlong()
    _check(load_library().mf_batch_describe(plan, ctypes.byref(k), ctypes.byref(n)))
    return k.value, n.value


def mf_autotune(src, dst, H, W, pitch, channels, dtype, k, stream=None):
    return _check(load_library().mf_autotune(src, dst, H, W, pitch, channels, dtype, k, stream))


def mf_describe(H, W, channels, dtype, k, variant=MF_AUTO):
    buf = ctypes.create_string_buffer(512)
    _check(load_library().mf_describe(H, W, channels, dtype, k, variant, buf, 512))
    return buf.value.decode()


def mf_kernel_launch_count():
    return int(load_library().mf_kernel_launch_count())


def mf_probe_minmax(kind, iters=4096):
    """(min/max instructions per second, ms) of one probe form (see the header)."""
    rate, ms = ctypes.c_double(), ctypes.c_double()
    _check(load_library().mf_probe_minmax(kind, iters, ctypes.byref(rate), ctypes.byref(ms)))
    return rate.value, ms.value


def mf_d1_plan_check(k, tile, footprint=None, strip=1, kh=None, tile_h=None, key_bytes=None, threads=256):
    """Builds the data-aware schedule for (k, tile, strip) -- a window of k
    columns by kh rows and root tiles of tile columns by tile_h rows when
    given, for keys of key_bytes bytes and blocks of `threads` threads when
    key_bytes is given (else 4-byte keys, 256 threads); with a uint64
    footprint of keys ((tile_h+kh-1) x (strip*tile+k-1)) also runs it on the
    CPU.  Returns (stats dict, tile_h x strip*tile medians or None)."""
    import numpy as np
    st = np.zeros(7, np.int32)
    med = None
    fp = None
    th = tile if tile_h is None else tile_h
    if footprint is not None:
        fp = np.ascontiguousarray(footprint, dtype=np.uint64)
        med = np.zeros(tile * th * strip, np.uint64)
    args = (fp.ctypes.data if fp is not None else None, med.ctypes.data if med is not None else None,
            st.ctypes.data)
    kh_ = k if kh is None else kh
    if key_bytes is None:
        _check(load_library().mf_d1_plan_check_rect(k, kh_, tile, th, strip, *args))
    else:
        _check(load_library().mf_d1_plan_check_ex(k, kh_, tile, th, strip, key_bytes, threads, *args))
    names = ["smem_elems", "phases", "tasks", "work_items", "merged", "sorted", "max_sort"]
    return dict(zip(names, [int(v) for v in st])), med


def mf_median_filter_3d(src, dst, D, H, W, pitch, volumes, dtype, k, stream=None):
    return _check(load_library().mf_median_filter_3d(src, dst, D, H, W, pitch, volumes, dtype, k, stream))


def mf_median_filter_3d_ex(src, dst, D, H, W, pitch, volumes, dtype, k, variant, stream=None):
    return _check(load_library().mf_median_filter_3d_ex(src, dst, D, H, W, pitch, volumes, dtype, k, variant,
                                                        stream))


def mf_median_filter_3d_describe(k, dtype):
    buf = ctypes.create_string_buffer(512)
    _check(load_library().mf_median_filter_3d_describe(k, dtype, buf, 512))
    return buf.value.decode()


def mf_d3_plan_check(k, tile, footprint=None, strip=1, key_bytes=None, threads=256):
    """Builds the volumetric schedule for (k, tile, strip) -- for keys of
    key_bytes bytes and blocks of `threads` threads when key_bytes is given
    (else 4-byte keys, 256 threads); with a uint64 footprint of keys
    (F = tile + k - 1 in y and z, FX = strip*tile + k - 1 in x, element
    (fx, fy, fz) at (fy*FX + fx)*F + fz) also runs it on the CPU.  Returns
    (stats dict, strip*tile^3 medians in (z, y, x) order or None)."""
    import numpy as np
    st = np.zeros(7, np.int32)
    med = fp = None
    if footprint is not None:
        fp = np.ascontiguousarray(footprint, dtype=np.uint64)
        med = np.zeros(strip * tile ** 3, np.uint64)
    args = (fp.ctypes.data if fp is not None else None, med.ctypes.data if med is not None else None,
            st.ctypes.data)
    if key_bytes is None:
        _check(load_library().mf_d3_plan_check(k, tile, strip, *args))
    else:
        _check(load_library().mf_d3_plan_check_ex(k, tile, strip, key_bytes, threads, *args))
    names = ["smem_elems", "phases", "tasks", "work_items", "merged", "sorted", "max_sort"]
    return dict(zip(names, [int(v) for v in st])), med


def mf_version():
    return load_library().mf_version().decode()


def mf_shutdown():
    return _check(load_library().mf_shutdown())


# ------------------------------------------------------------ torch helpers
def _torch():
    import torch
    return torch


def dtype_code(t):
    torch = _torch()
    m = {torch.uint8: MF_U8, torch.float32: MF_F32}
    for name, code in (("uint16", MF_U16), ("uint32", MF_U32)):
        if hasattr(torch, name):
            m[getattr(torch, name)] = code
    if t not in m:
        raise MedianFilterError("unsupported dtype %s" % t)
    return m[t]


def _planes(x):
    """(planes, H, W, pitch_bytes) of a (..., H, W) CUDA tensor whose planes
    are stacked at H * pitch bytes (row stride >= W, unit column stride)."""
    if not x.is_cuda:
        raise MedianFilterError("tensor must be on a CUDA device")
    if x.dim() < 2:
        raise MedianFilterError("need (..., H, W)")
    H, W = int(x.shape[-2]), int(x.shape[-1])
    es = x.element_size()
    if x.stride(-1) != 1 and W > 1:
        raise MedianFilterError("last dimension must be contiguous")
    rs = x.stride(-2) if H > 1 else max(W, 1)
    planes = 1
    for d in x.shape[:-2]:
        planes *= int(d)
    # every leading dim must step by whole planes of H * rs elements
    expect = H * rs
    for dim in range(x.dim() - 3, -1, -1):
        if x.shape[dim] > 1 and x.stride(dim) != expect:
            raise MedianFilterError("planes must be stacked contiguously")
        expect *= int(x.shape[dim])
    return planes, H, W, rs * es


def _stream_ptr(x):
    return _torch().cuda.current_stream(x.device).cuda_stream


def median_filter(x, k, variant="auto", return_idx=False, out=None, kh=None):
    """k x k clamp-to-edge median of every (H, W) plane of a CUDA tensor
    (u8, u16, u32 or f32); with kh, a window of k columns by kh rows
    (mf_median_filter_rect).  With return_idx also the int32 argmedian."""
    torch = _torch()
    planes, H, W, pitch = _planes(x)
    if out is None:
        out = torch.empty_like(x, memory_format=torch.contiguous_format)
    op, oH, oW, opitch = _planes(out)
    if (op, oH, oW, opitch) != (planes, H, W, pitch):
        raise MedianFilterError("out must have the layout of x")
    idx = None
    if return_idx:
        idx = torch.empty(x.shape, dtype=torch.int32, device=x.device)
    with torch.cuda.device(x.device):
        if kh is not None and int(kh) != int(k):
            mf_median_filter_rect(x.data_ptr(), out.data_ptr(), H, W, pitch, planes, dtype_code(x.dtype), int(k),
                                  int(kh), idx.data_ptr() if idx is not None else None, 4 * W, _stream_ptr(x))
        else:
            mf_median_filter_ex(x.data_ptr(), out.data_ptr(), H, W, pitch, planes, dtype_code(x.dtype), int(k),
                                MF_BORDER_CLAMP, VARIANTS[variant],
                                idx.data_ptr() if idx is not None else None, 4 * W, _stream_ptr(x))
    return (out, idx) if return_idx else out


def median_filter_3d(x, k, out=None, variant="auto"):
    """k x k x k clamp-to-edge median of every (D, H, W) volume of a CUDA
    tensor (..., D, H, W) of u8, u16, u32 or f32 (mf_median_filter_3d_ex)."""
    torch = _torch()
    if x.dim() < 3:
        raise MedianFilterError("need (..., D, H, W)")
    slices, H, W, pitch = _planes(x)
    D = int(x.shape[-3])
    if out is None:
        out = torch.empty_like(x, memory_format=torch.contiguous_format)
    if _planes(out) != (slices, H, W, pitch):
        raise MedianFilterError("out must have the layout of x")
    with torch.cuda.device(x.device):
        mf_median_filter_3d_ex(x.data_ptr(), out.data_ptr(), D, H, W, pitch, slices // D, dtype_code(x.dtype),
                               int(k), VARIANTS[variant], _stream_ptr(x))
    return out


def median_filter_backward(grad_out, idx, k, mode="atomic"):
    torch = _torch()
    grad_out = grad_out.contiguous()
    idx = idx.contiguous()
    planes, H, W, pitch = _planes(grad_out)
    gi = torch.empty_like(grad_out)
    with torch.cuda.device(grad_out.device):
        mf_median_filter_bwd(grad_out.data_ptr(), idx.data_ptr(), gi.data_ptr(), H, W, pitch, 4 * W,
                             planes, int(k), GRAD_MODES[mode], _stream_ptr(grad_out))
    return gi


class MedianFilterFn:
    """torch.autograd.Function: forward saves the int32 argmedian, backward
    scatters (atomic) or gathers (deterministic) grad_out onto it."""

    @staticmethod
    def apply(x, k, mode="atomic", variant="auto"):
        return _fn().apply(x, k, mode, variant)


_fn_cls = None


def _fn():
    global _fn_cls
    if _fn_cls is None:
        torch = _torch()

        class _MedianFilterFunction(torch.autograd.Function):
            @staticmethod
            def forward(ctx, x, k, mode, variant):
                if x.dtype != torch.float32:
                    raise MedianFilterError("gradients need f32 input")
                y, idx = median_filter(x.contiguous(), k, variant=variant, return_idx=True)
                ctx.save_for_backward(idx)
                ctx.k, ctx.mode = k, mode
                return y

            @staticmethod
            def backward(ctx, g):
                (idx,) = ctx.saved_tensors
                return median_filter_backward(g, idx, ctx.k, ctx.mode), None, None, None

        _fn_cls = _MedianFilterFunction
    return _fn_cls
