"""CPU oracle for the k x k median filter -- TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  The CUDA library never does, and this
package imports nothing from it.  The arithmetic lives in ``mf_oracle.c``
(plain brute force: gather the clamped window, select rank (k*k-1)/2); this
module only compiles it with gcc and marshals numpy arrays.

Every function follows the definition of the median filter in the paper's
introduction (each pixel replaced by the median of its k x k neighbourhood),
with the readings stated in ``mf_oracle.c``: clamp-to-edge borders, the f32
sign-flip order, and the argmedian tie rule (lowest value, then lowest
row-major window slot).

Parity status: pinned.  The value path is pinned by hand-worked fixtures,
scipy.ndimage's median filter, the counting characterisation of a rank,
k=1, constant images and monotone remaps; the argmedian tie rule by
hand-worked fixtures with ties; the backward by a hand-worked case and
central finite differences.  The volumetric k x k x k filter
(``median_filter_3d``) is pinned by a hand-worked 2x2x2 volume, scipy.ndimage's
3D median, a numpy brute force over an edge-padded volume, the one-slice reduction to the 2D filter,
axis permutations, constants and k = 1.
"""
import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "mf_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None

DTYPES = {"u8": 0, "u16": 1, "u32": 2, "f32": 3}
NP_DTYPES = {"u8": np.uint8, "u16": np.uint16, "u32": np.uint32, "f32": np.float32}


def build(force=False):
    """Compile mf_oracle.c into liboracle.so with gcc (OpenMP when available)."""
    if not force and os.path.exists(_LIB) and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC):
        return _LIB
    base = ["gcc", "-O2", "-fPIC", "-shared", "-std=c11"]
    tmp = _LIB + ".tmp%d" % os.getpid()
    try:
        subprocess.run(base + ["-fopenmp", _SRC, "-o", tmp], check=True,
                       capture_output=True)
    except subprocess.CalledProcessError:
        subprocess.run(base + [_SRC, "-o", tmp], check=True, capture_output=True)
    os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    with _lock:
        if _lib is None:
            build()
            lib = ctypes.CDLL(_LIB)
            vp, i32, u32 = ctypes.c_void_p, ctypes.c_int, ctypes.c_uint32
            lib.or_median_filter.argtypes = [vp, vp, vp, i32, i32, i32, i32, i32, i32]
            lib.or_median_filter_rect.argtypes = [vp, vp, vp, i32, i32, i32, i32, i32, i32, i32]
            lib.or_median_filter_rows.argtypes = [vp, vp, vp, i32, i32, i32, i32, i32, vp, i32, i32]
            lib.or_median_backward.argtypes = [vp, vp, vp, i32, i32, i32]
            lib.or_median_filter_3d.argtypes = [vp, vp, i32, i32, i32, i32, i32, i32, i32]
            lib.or_key.argtypes = [i32, u32]
            lib.or_key.restype = u32
            lib.or_max_threads.restype = i32
            _lib = lib
    return _lib


def _dtype_name(a):
    for name, t in NP_DTYPES.items():
        if a.dtype == t:
            return name
    raise TypeError("unsupported dtype %s" % a.dtype)


def _as_chw(x):
    x = np.ascontiguousarray(x)
    if x.ndim == 2:
        return x[None], True
    if x.ndim != 3:
        raise ValueError("expected (H, W) or (C, H, W)")
    return x, False


def median_filter(x, k, with_idx=False, threads=0, kh=None):
    """Clamp-to-edge k x k median of every plane of x ((H, W) or (C, H, W));
    with kh, a window of k columns by kh rows (paper Sec. 3.2 states the tile
    terminology for a k_w x k_h kernel).

    Returns the filtered array (same dtype, bit-copied winners), and with
    ``with_idx`` also the int32 argmedian ys*W + xs per output pixel
    (window slots row-major: (dy+ry)*k + (dx+rx)).
    """
    lib = _load()
    xc, squeeze = _as_chw(x)
    C, H, W = xc.shape
    out = np.empty_like(xc)
    idx = np.empty((C, H, W), np.int32) if with_idx else None
    kh = k if kh is None else kh
    rc = lib.or_median_filter_rect(xc.ctypes.data, out.ctypes.data,
                                   idx.ctypes.data if with_idx else None,
                                   H, W, C, DTYPES[_dtype_name(xc)], int(k), int(kh), int(threads))
    if rc != 0:
        raise ValueError("oracle rejected arguments (H=%d W=%d C=%d k=%d kh=%d)" % (H, W, C, k, kh))
    if squeeze:
        out = out[0]
        idx = idx[0] if with_idx else None
    return (out, idx) if with_idx else out


def median_filter_rows(x, k, rows, with_idx=False, threads=0):
    """The filter evaluated only on ``rows`` of every plane: (C, len(rows), W)."""
    lib = _load()
    xc, squeeze = _as_chw(x)
    C, H, W = xc.shape
    rows = np.ascontiguousarray(np.asarray(rows, np.int32))
    out = np.empty((C, len(rows), W), xc.dtype)
    idx = np.empty((C, len(rows), W), np.int32) if with_idx else None
    rc = lib.or_median_filter_rows(xc.ctypes.data, out.ctypes.data,
                                   idx.ctypes.data if with_idx else None,
                                   H, W, C, DTYPES[_dtype_name(xc)], int(k),
                                   rows.ctypes.data, len(rows), int(threads))
    if rc != 0:
        raise ValueError("oracle rejected arguments")
    if squeeze:
        out = out[0]
        idx = idx[0] if with_idx else None
    return (out, idx) if with_idx else out


def median_filter_3d(x, k, threads=0):
    """Clamp-to-edge k x k x k median of a volume (D, H, W) or of volumes
    (V, D, H, W): the 3D extension of the filter that the paper names as
    future work (Sec. 7.2).  Values only."""
    lib = _load()
    x = np.ascontiguousarray(x)
    squeeze = x.ndim == 3
    if squeeze:
        x = x[None]
    if x.ndim != 4:
        raise ValueError("expected (D, H, W) or (V, D, H, W)")
    V, D, H, W = x.shape
    out = np.empty_like(x)
    rc = lib.or_median_filter_3d(x.ctypes.data, out.ctypes.data, D, H, W, V, DTYPES[_dtype_name(x)],
                                 int(k), int(threads))
    if rc != 0:
        raise ValueError("oracle rejected arguments (D=%d H=%d W=%d k=%d)" % (D, H, W, k))
    return out[0] if squeeze else out


def median_backward(grad_out, idx):
    """grad_in of the filter: zero, then grad_in[idx[q]] += grad_out[q] in row-major q."""
    lib = _load()
    g, squeeze = _as_chw(np.asarray(grad_out, np.float32))
    ix, _ = _as_chw(np.asarray(idx, np.int32))
    C, H, W = g.shape
    if ix.shape != g.shape:
        raise ValueError("grad_out and idx shapes differ")
    out = np.empty_like(g)
    if lib.or_median_backward(g.ctypes.data, ix.ctypes.data, out.ctypes.data, H, W, C) != 0:
        raise ValueError("index out of range")
    return out[0] if squeeze else out


def order_key(dtype, bits):
    """The unsigned order key of one element given as its raw bits."""
    return int(_load().or_key(DTYPES[dtype], int(bits) & 0xFFFFFFFF))


def max_threads():
    return int(_load().or_max_threads())
