"""Seeded synthetic inputs (no median arithmetic here).

This module only draws images.  Both the CUDA path's tests/benchmark and the
CPU oracle consume these arrays, so nothing in it may compute a median, a
sort, a key order or anything else the filter does.

The paper measures on 30-megapixel photographs (Sec. 5) and a 30 MP RGB
photograph for its teaser; none ships with it, so the shapes and value
statistics below stand in for them.  All draws come from
``numpy.random.Generator(PCG64(seed))``; workload i uses seed 19926 + i.
"""
import numpy as np

SEED_BASE = 19926

NP = {"u8": np.uint8, "u16": np.uint16, "u32": np.uint32, "f32": np.float32}
MAXV = {"u8": 255, "u16": 65535, "u32": 4294967295}


def rng(seed):
    return np.random.Generator(np.random.PCG64(seed))


def uniform(shape, dtype, seed):
    """i.i.d. uniform over the whole code range.  For f32: uniform random bit
    patterns whose exponent is not all ones (finite values, including -0 and
    denormals)."""
    g = rng(seed)
    if dtype == "f32":
        bits = g.integers(0, 1 << 32, size=shape, dtype=np.uint64).astype(np.uint32)
        exp_all_ones = (bits & np.uint32(0x7F800000)) == np.uint32(0x7F800000)
        while exp_all_ones.any():
            bits[exp_all_ones] = g.integers(0, 1 << 32, size=int(exp_all_ones.sum()),
                                            dtype=np.uint64).astype(np.uint32)
            exp_all_ones = (bits & np.uint32(0x7F800000)) == np.uint32(0x7F800000)
        return bits.view(np.float32)
    hi = MAXV[dtype]
    return g.integers(0, hi + 1, size=shape, dtype=np.uint64).astype(NP[dtype])


def levels16(shape, dtype, seed):
    """Low-entropy image: 16 distinct levels chosen i.i.d. (heavy ties).
    Integers: L_i = round(i * MAX / 15); f32: 2i/15 - 1, i = 0..15."""
    g = rng(seed)
    i = g.integers(0, 16, size=shape)
    if dtype == "f32":
        return (2.0 * i / 15.0 - 1.0).astype(np.float32)
    lv = np.array([int(round(j * MAXV[dtype] / 15.0)) for j in range(16)], dtype=np.uint64)
    return lv[i].astype(NP[dtype])


def photo_rgb(H=4480, W=6720, seed=SEED_BASE + 1):
    """Photo-like 3-plane u8 image: smooth low-frequency field per channel,
    plus N(0, 12^2) noise, rounded and clamped, plus 5% salt-and-pepper."""
    g = rng(seed)
    y = (np.arange(H, dtype=np.float64) / H)[:, None]
    x = (np.arange(W, dtype=np.float64) / W)[None, :]
    out = np.empty((3, H, W), np.uint8)
    for c in range(3):
        base = (128.0 + 50.0 * np.sin(2 * np.pi * (x * 1.5 + y * 0.5) + c * 2 * np.pi / 3)
                + 40.0 * (x - 0.5) + 30.0 * (y - 0.5))
        v = base + g.normal(0.0, 12.0, size=(H, W))
        v = np.clip(np.rint(v), 0, 255)
        imp = g.random((H, W)) < 0.05
        salt = g.random((H, W)) < 0.5
        v[imp & salt] = 255
        v[imp & ~salt] = 0
        out[c] = v.astype(np.uint8)
    return out


def normal_f32(shape, seed):
    return rng(seed).standard_normal(size=shape).astype(np.float32)


def batch_descs(n=64, seed=SEED_BASE + 3):
    """The uneven batch: sizes log-uniform in 256x256 .. 4096x3072 (W, H),
    dtype from {u8, u16, f32}, odd k in 3..31, one channel each."""
    g = rng(seed)
    descs = []
    for _ in range(n):
        W = int(round(np.exp(g.uniform(np.log(256), np.log(4096)))))
        H = int(round(np.exp(g.uniform(np.log(256), np.log(3072)))))
        dt = ["u8", "u16", "f32"][int(g.integers(0, 3))]
        k = int(2 * g.integers(1, 16) + 1)
        descs.append({"H": H, "W": W, "dtype": dt, "k": k, "seed": int(g.integers(0, 2**31))})
    return descs


def tiny_cases(seed, n, max_hw=9, ks=(1, 3, 5, 7, 9), dtypes=("u8", "u16", "u32", "f32")):
    """Many tiny images (H, W in 1..max_hw) with heavy ties, for brute-force checks."""
    g = rng(seed)
    cases = []
    for _ in range(n):
        H = int(g.integers(1, max_hw + 1))
        W = int(g.integers(1, max_hw + 1))
        dt = dtypes[int(g.integers(0, len(dtypes)))]
        k = int(ks[int(g.integers(0, len(ks)))])
        s = int(g.integers(0, 2**31))
        img = levels16((H, W), dt, s) if g.random() < 0.5 else uniform((H, W), dt, s)
        cases.append((img, k))
    return cases
