"""Builds libmedianfilter.so for sm_103a.

Steps: (1) emit the data-oblivious networks and their kernel
instantiations (codegen.py) into _build/gen; (2) compile every translation
unit with nvcc in parallel; (3) link the shared library next to this file.
Outputs are git-ignored build artefacts.  Nothing here needs a GPU.
"""
from __future__ import annotations

import concurrent.futures as cf
import hashlib
import os
import shutil
import subprocess
import sys

from . import codegen, netgen

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
BUILD = os.path.join(HERE, "_build")
GEN = os.path.join(BUILD, "gen")
LIB = os.path.join(HERE, "libmedianfilter.so")
INCLUDE = os.path.join(os.path.dirname(HERE), "include")

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
NVCC_FLAGS = ["-O3", "-std=c++17", "-lineinfo", "-Xcompiler", "-fPIC", "--expt-relaxed-constexpr",
              "-I" + INCLUDE, "-I" + CSRC, "-I" + GEN]

# Data-oblivious instantiations: k -> list of (tile w, tile h, block x,
# block y, U); the first entry is the default, the autotuner may pick
# another.  U is the number of tree levels emitted unrolled: deeper levels
# are loop-rolled (rolled.py), U = -1 is the straight-line network.
# Root tiles follow t(k) = 2^(floor(log2 k) - 1) (paper Sec. 4.2) up to
# k = 7 and stay at 4x4 above: an 8x8 root tile's network no longer fits
# the 255 registers of one thread (the paper's own limit, Sec. 4.3).
# Measured on GB300 (4096^2 u8/u32): straight-line is fastest up to k = 15,
# the fully rolled tree at k = 17 (13-15% faster than straight-line there,
# where the straight-line code no longer stays in the instruction cache).
# Form 6 (lazy extra rows/columns, pressure-aware order) removes the
# register spills at k = 13 and most of them at k = 17 (1432 -> 252 spilled
# bytes a thread): k = 17 u8 0.459 -> 0.387 ms, u32 0.850 -> 0.770 ms;
# u32 k = 25 4.51 -> 2.64 ms.  The straight-line networks up to k = 15 gain
# nothing from it (within 1-5%, either way) except u8 k = 9 (0.127 -> 0.117
# ms).  At k = 23, 25 the packed two-tiles-a-thread form spills too much:
# 8/16-bit data runs one tile a thread on 32-bit keys there (u8 k = 23
# 2.53 -> 1.87 ms, k = 25 3.11 -> 2.82 ms).  With form 6 the first tree
# level unrolled (U = 1) wins at k = 17 (photo 2.147 -> 2.004 ms, u32 4096^2
# 0.770 -> 0.740) and for 32-bit keys at k = 21..25 (u32 k = 25 2.86 ->
# 2.56 ms); U = 2 loses (2.70 ms).  At k = 17 with 16-bit keys, blocks of
# 16 x 8 threads (a 128 x 32 pixel region: less halo per pixel than 256 x 16)
# run the 30 MP photo in 1.941 ms against 2.005 (32 x 4), 1.974 (16 x 4),
# 1.961 (8 x 8); u32 4096^2 0.726 against 0.738 ms.  The same shape gains
# 1-6% at k = 9..15 (u32 k = 11: 0.422 -> 0.397 ms).  The direct kernel (form 8) wins where
# staging dominates: k = 3 (u8 35.6 -> 25.0 us, u32 56.7 -> 35.4 us at
# 4096^2) and 32-bit keys up to k = 9 (u32 k = 7 180 -> 121 us, k = 9 280 ->
# 229 us); with packed 8/16-bit keys it ties at k = 5, 7 and spills at 9.
# The wide direct form (form bits 16/32: 4 or 2 tiles a lane side by side,
# vector row loads, one byte permute per packed word, vector stores) wins at
# k = 3 and 5 (4096^2, L2 flushed): u8 k = 3 27.3 -> 21.2 us, f32 k = 3
# 49.8 -> 41.6 us, u8 k = 5 58.0 -> 41.6 us, u32 k = 5 80.5 -> 68.2 us (two
# tiles a lane); u32 k = 3 ties the direct form (35.5 us).
# k = 27: 3.64 ms against 7.62 ms for the best data-aware tile (u32 4096^2),
# u8 4.03 vs 5.02 ms (one tile a thread on 32-bit keys); at k = 29 the
# data-aware kernel wins for u8 and the spilling network gains too little
# for 32-bit keys to pay its compile time.
O1_VALUE = {3: [(2, 2, 16, 8, -1, 24), (2, 2, 32, 4, -1, 8), (2, 2, 32, 4, -1, 0), (2, 2, 32, 4, -1, 24),
                (2, 2, 16, 8, -1, 40)],
            5: [(2, 2, 16, 8, -1, 24, 16), (2, 2, 16, 8, -1, 40, 32), (2, 2, 32, 4, -1, 0, 16),
                (2, 2, 32, 4, -1, 8, 32), (2, 2, 32, 4, -1, 0, 32), (2, 2, 16, 8, -1, 40, 16),
                (2, 2, 16, 8, -1, 24, 32)],
            7: [(4, 4, 32, 4, -1, 0, 16), (4, 4, 32, 4, -1, 8, 32), (4, 4, 32, 4, -1, 0, 32)],
            9: [(4, 4, 16, 8, -1, 6, 16), (4, 4, 32, 4, -1, 8, 32), (4, 4, 32, 4, -1, 0, 32)],
            11: [(4, 4, 16, 8, -1)], 13: [(4, 4, 16, 8, -1)], 15: [(4, 4, 16, 8, -1)],
            17: [(4, 4, 16, 8, 1, 6), (4, 4, 32, 4, 1, 6), (4, 4, 16, 4, 1, 6, 16), (4, 4, 32, 4, 0, 6)],
            19: [(4, 4, 32, 4, 0, 7, 16), (4, 4, 32, 4, 0, 6, 32), (4, 4, 32, 4, 1, 6)],
            21: [(4, 4, 32, 4, 0, 6, 16), (4, 4, 32, 4, 1, 6, 32)],
            23: [(4, 4, 32, 4, 1, 6, 1), (4, 4, 32, 4, 1, 6, 32), (4, 4, 32, 4, 0, 6, 1), (4, 4, 32, 4, 0, 6, 16)],
            25: [(4, 4, 32, 4, 1, 6, 1), (4, 4, 32, 4, 1, 6, 32), (4, 4, 32, 4, 0, 6, 1), (4, 4, 32, 4, 0, 0, 16)],
            27: [(4, 4, 32, 4, 1, 6, 32), (4, 4, 32, 4, 1, 6, 1)]}
# extra configurations for timing (comma list "k:tw:th:bx:by:U[:R[:keys]]"
# in MF_O1_EXTRA).  R is the network form, a bit set: 1 = the root extra
# rows are sorted into shared memory by a stage of their own (netgen.build
# rows_smem), 2 = lazy extra rows/columns, 4 = pressure-aware op order,
# 8 = the direct kernel (each thread loads its own footprint into
# registers and sorts its own columns: no shared memory, no barriers).
for _spec in filter(None, os.environ.get("MF_O1_EXTRA", "").split(",")):
    _v = [int(v) for v in _spec.split(":")]
    O1_VALUE.setdefault(_v[0], []).append(tuple((_v + [0, 0, 0])[1:8]))
# MF_O1_ONLY="k1,k2,...": build the data-oblivious kernels for these k only
# (a smaller, faster build; the data-aware variant still covers every k)
if os.environ.get("MF_O1_ONLY"):
    _only = {int(v) for v in os.environ["MF_O1_ONLY"].split(",") if v.strip()}
    O1_VALUE = {k: v for k, v in O1_VALUE.items() if k in _only}
# a 7th field restricts a configuration to 16-bit keys (u8/u16, two tiles a
# thread) or 32-bit keys (u32/f32); 0 = both; 1 = u8/u16 data with 32-bit
# keys (one tile a thread: half the values in flight of the packed form)
O1_VALUE = {k: [tuple(c) + (0,) * (7 - len(c)) for c in v] for k, v in O1_VALUE.items()}
# argmedian with 32-bit records (8/16-bit data) and 64-bit records (32-bit data);
# above k = 25 the argmedian comes from the values and the recovery pass
O1_ARG32 = {k: v[0] for k, v in O1_VALUE.items() if k <= 25}


def o1_covers(k, dtype):
    """True when a data-oblivious value kernel is built for (k, dtype name)."""
    wide = dtype in ("u32", "f32")
    return any(keys == 0 or keys == (32 if wide else 16) or (keys == 1 and not wide)
               for (_, _, _, _, _, _, keys) in O1_VALUE.get(k, []))
# 32-bit data: the argmedian comes from the value kernel plus the recovery
# pass (mf_argmedian.cu), which beats 64-bit records (1.33 vs ~0.4 ms at
# k = 9, f32 16 x 1024^2); no 64-bit-record networks are built.
O1_ARG64 = {}


DT_NAMES = {0: "MF_U8", 1: "MF_U16", 2: "MF_U32", 3: "MF_F32"}

# Loop-rolled networks (one child per split emitted, run twice): same ops,
# roughly half the code per tree level.
O1_ROLLED = os.environ.get("MF_O1_ROLLED", "1") == "1"

# Fuse min(min(a, b), c) chains into three-input min/max (one instruction).
O1_FUSE3 = os.environ.get("MF_O1_FUSE3", "1") == "1"

# Rolled networks: one-level value selects as multiply-adds (rolled.emit).
O1_MAD_SELECT = os.environ.get("MF_O1_MAD_SELECT", "0") == "1"

# Barrier spacing (min/max ops) inside long per-thread networks.
O1_SYNC_EVERY = int(os.environ.get("MF_O1_SYNC_EVERY", "0"))


def _o1_instances():
    """(k, tw, th, bx, by, dtype, ko, arg, ib) for every O1 kernel built."""
    out = []
    for k, cfgs in sorted(O1_VALUE.items()):
        for ci, (tw, th, bx, by, u, rs, keys) in enumerate(cfgs):
            if keys in (0, 16):
                for dt in (0, 1):
                    out.append((k, tw, th, bx, by, (u, rs), dt, "KoU16x2", False, 0, ci))
            if keys in (0, 32):
                for dt in (2, 3):
                    out.append((k, tw, th, bx, by, (u, rs), dt, "KoU32", False, 0, ci))
            if keys == 1:
                for dt in (0, 1):
                    out.append((k, tw, th, bx, by, (u, rs), dt, "KoU32", False, 0, ci))
    for k, (tw, th, bx, by, u, rs, keys) in sorted(O1_ARG32.items()):
        rs &= ~(8 | 16 | 32)  # argmedian records run in the shared-memory kernel
        out.append((k, tw, th, bx, by, (u, rs), 0, "KoU32", True, 24, 0))
        out.append((k, tw, th, bx, by, (u, rs), 1, "KoU32", True, 16, 0))
    for k, (tw, th, bx, by, u, rs, keys) in sorted(O1_ARG64.items()):
        for dt in (2, 3):
            out.append((k, tw, th, bx, by, (u, rs), dt, "KoU64", True, 32, 0))
    return out


def _gen_key():
    """Hash of everything the generated sources depend on: the instantiation
    tables, the generator switches and the package's Python sources."""
    h = hashlib.sha1()
    h.update(repr((sorted(O1_VALUE.items()), sorted(O1_ARG32.items()), sorted(O1_ARG64.items()), O1_ROLLED,
                   O1_FUSE3, O1_MAD_SELECT, O1_SYNC_EVERY)).encode())
    for name in sorted(os.listdir(HERE)):
        if name.endswith(".py"):
            with open(os.path.join(HERE, name), "rb") as f:
                h.update(name.encode())
                h.update(f.read())
    return h.hexdigest()


def generate():
    """Writes the generated translation units and headers into _build/gen and
    returns the translation units; skipped (the recorded list returned) when
    nothing they depend on changed since the last run."""
    import json
    stamp = os.path.join(GEN, ".stamp.json")
    key = _gen_key()
    try:
        with open(stamp) as f:
            rec = json.load(f)
        tus = [os.path.join(GEN, n) for n in rec["tus"]]
        heads = [os.path.join(GEN, n) for n in ("d1_sortnets.cuh", "d3_nets.cuh")]
        if rec["key"] == key and all(os.path.exists(t) for t in tus + heads):
            return tus
    except (OSError, ValueError, KeyError):
        pass
    tus = _generate()
    with open(stamp, "w") as f:
        json.dump({"key": key, "tus": [os.path.basename(t) for t in tus]}, f)
    return tus


def _generate():
    os.makedirs(GEN, exist_ok=True)
    for name in os.listdir(GEN):
        if name.startswith("o1_k") and name.endswith(".cu"):
            os.remove(os.path.join(GEN, name))
    codegen.write_if_changed(os.path.join(GEN, "d1_sortnets.cuh"), codegen.emit_d1_sortnets())
    codegen.write_if_changed(os.path.join(GEN, "d3_nets.cuh"), codegen.emit_d3_networks())
    insts = _o1_instances()
    by_k = {}
    for inst in insts:  # one translation unit per instantiation (parallel build)
        by_k.setdefault(inst[:6] + (inst[7], inst[8], inst[6]), []).append(inst)
    tus = []
    decls = []
    entries = []

    # each k's configurations in their listed order (default first)
    for key, lst in sorted(by_k.items(), key=lambda kv: (kv[0][0], min(i[10] for i in kv[1]))):
        k = key[0]
        parts = ['// generated by codegen/build.py -- do not edit', '#include "mf_oblivious.cuh"',
                 "namespace mf {"]
        unroll, rsm = key[5]
        nets = sorted({(i[1], i[2]) for i in lst})
        sorts = sorted({k - th + 1 for (_, th) in nets} | {k - tw + 1 for (tw, _) in nets})
        n_ops = {}
        for tw, th in nets:
            assert not (rsm & 8 and rsm & 1), "the direct kernel takes no shared-memory rows"
            assert not (rsm & 48) or rsm & 8, "the wide form is a direct form"
            net = netgen.build(k, tw, th, rows_smem=bool(rsm & 1), lazy=bool(rsm & 2), pressure=bool(rsm & 4))
            n_ops[(tw, th)] = netgen.n_minmax(net)
            if O1_FUSE3:
                net = netgen.fuse3(net)
            sync = O1_SYNC_EVERY if O1_SYNC_EVERY and len(net.ops) > 4 * O1_SYNC_EVERY else 0
            u_eff = unroll if O1_ROLLED else -1
            src, _ = codegen.emit_network_auto(net, codegen.net_name(k, tw, th, u_eff, rsm), sync, u_eff,
                                               direct=bool(rsm & 8), mad_select=O1_MAD_SELECT,
                                               wide=codegen.wide_tiles(rsm))
            parts.append(src)
        for n in sorts:
            parts.append(codegen.emit_colsort(n))
        for (k_, tw, th, bx, by, (u, rsm), dt, ko, arg, ib, _) in lst:
            fn = "o1_launch_k%d_%dx%d_b%dx%d_u%s%s_%s_%s%s" % (k, tw, th, bx, by, "m1" if u < 0 else u,
                                                            codegen.form_suffix(rsm), DT_NAMES[dt], ko,
                                                            "_arg" if arg else "")
            targs = "%d, %d, %d, %d, %d, %s, %s, %s, %d, %s, %s, %s" % (
                k, tw, th, bx, by, DT_NAMES[dt], ko, "true" if arg else "false", ib,
                codegen.net_name(k, tw, th, u if O1_ROLLED else -1, rsm), codegen.sort_name(k - th + 1),
                codegen.sort_name(k - tw + 1))
            parts.append("int %s(const ImgArgs &a, int c, cudaStream_t s) {\n"
                         "  return launch_o1<%s>(a, c, s);\n}" % (fn, targs))
            pfn = "NULL"
            if not arg:
                pfn = fn.replace("o1_launch", "o1_persist")
                parts.append("int %s(const ImgArgs *i, const int4 *w, int n, unsigned *q, int b, int sms, "
                             "cudaStream_t s, int *g) {\n  return persist_o1<%s>(i, w, n, q, b, sms, s, g);\n}"
                             % (pfn, targs))
                decls.append("int %s(const ImgArgs *i, const int4 *w, int n, unsigned *q, int b, int sms, "
                             "cudaStream_t s, int *g);" % pfn)
            decls.append("int %s(const ImgArgs &a, int c, cudaStream_t s);" % fn)
            entries.append("  {%d, %s, %d, %d, %d, %d, %d, %d, %d, %d, %s, %s, \"%s\"}," %
                           (k, DT_NAMES[dt], 1 if arg else 0, tw, th, bx, by, 2 if ko == "KoU16x2" else 1,
                            codegen.wide_tiles(rsm), n_ops[(tw, th)], fn, pfn, fn))
        parts.append("}  // namespace mf")
        path = os.path.join(GEN, "o1_k%d_%dx%d_b%dx%d_u%s%s_%s%s_%s.cu" % (
            key[:5] + ("m1" if key[5][0] < 0 else key[5][0], codegen.form_suffix(key[5][1]), key[6],
                       "_arg" if key[7] else "", DT_NAMES[key[8]])))
        codegen.write_if_changed(path, "\n".join(parts) + "\n")
        tus.append(path)
    reg = ['// generated -- do not edit', '#include "mf_registry.h"', "namespace mf {"]
    reg += decls
    reg.append("const O1Entry kO1Entries[] = {")
    reg += entries
    reg.append("};")
    reg.append("const int kO1Count = %d;" % len(entries))
    reg.append("}  // namespace mf")
    path = os.path.join(GEN, "o1_registry.cu")
    codegen.write_if_changed(path, "\n".join(reg) + "\n")
    tus.append(path)
    return tus


def _includes(path, seen):
    """path and every file it includes with #include "..." (transitively),
    resolved like the build's -I list."""
    if path in seen:
        return
    seen.append(path)
    with open(path) as f:
        for line in f:
            line = line.strip()
            if line.startswith("#include \""):
                name = line.split('"')[1]
                for d in (os.path.dirname(path), INCLUDE, CSRC, GEN):
                    cand = os.path.normpath(os.path.join(d, name))
                    if os.path.exists(cand):
                        _includes(cand, seen)
                        break


def kernel_source_hash(fn_name):
    """Hash of the sources of the registry launch function fn_name -- its
    generated translation unit, every file that includes (transitively) and
    the compiler flags -- or None: profiles record it beside ncu counters,
    so a reader can tell whether the counters still describe the kernel
    that is built."""
    if not os.path.isdir(GEN):
        return None
    needle = "int %s(" % fn_name
    root = os.path.dirname(HERE)
    for name in sorted(os.listdir(GEN)):
        if name.startswith("o1_k") and name.endswith(".cu"):
            path = os.path.join(GEN, name)
            with open(path) as f:
                if needle not in f.read():
                    continue
            files = []
            _includes(path, files)
            h = hashlib.sha1()
            # include paths name this checkout's location: hash them relative
            # to it, so that every checkout of the same sources agrees
            h.update(" ".join(f.replace(root, "<repo>") for f in NVCC_FLAGS + ARCH).encode())
            for fp in files:
                h.update(os.path.relpath(fp, root).encode())
                with open(fp, "rb") as f:
                    h.update(f.read())
            return h.hexdigest()[:16]
    return None


def _flags_hash(src, flags):
    """Hash of the flags, the translation unit and every file it includes
    (transitively): a TU is rebuilt only when something it reads changed."""
    h = hashlib.sha1()
    h.update(" ".join(flags).encode())
    files = []
    _includes(src, files)
    for fp in files:
        h.update(fp.encode())
        with open(fp, "rb") as f:
            h.update(f.read())
    return h.hexdigest()[:16]


def _compile(src, verbose=False):
    obj = os.path.join(BUILD, os.path.basename(src) + ".o")
    stamp = obj + ".hash"
    hsh = _flags_hash(src, NVCC_FLAGS + ARCH)
    if os.path.exists(obj) and os.path.exists(stamp) and open(stamp).read() == hsh:
        return obj, ""
    cmd = ["nvcc"] + ARCH + NVCC_FLAGS + (["-Xptxas", "-v"] if verbose else []) + ["-c", src, "-o", obj]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError("nvcc failed for %s:\n%s%s" % (src, r.stdout, r.stderr[-8000:]))
    with open(stamp, "w") as f:
        f.write(hsh)
    return obj, r.stderr


def build(jobs=None, verbose=False):
    """Generate, compile and link; returns the path of the shared library."""
    if shutil.which("nvcc") is None:
        raise RuntimeError("nvcc not found on PATH")
    os.makedirs(BUILD, exist_ok=True)
    tus = generate()
    tus += [os.path.join(CSRC, n) for n in sorted(os.listdir(CSRC)) if n.endswith(".cu")]
    jobs = jobs or max(1, min(len(tus), os.cpu_count() or 4))
    # biggest TUs first
    tus.sort(key=lambda p: -os.path.getsize(p))
    objs, logs = [], []
    with cf.ThreadPoolExecutor(jobs) as ex:
        for obj, log in ex.map(lambda s: _compile(s, verbose), tus):
            objs.append(obj)
            logs.append(log)
    tmp = LIB + ".tmp%d" % os.getpid()
    cmd = ["nvcc"] + ARCH + ["-shared", "-Xcompiler", "-fPIC", "-o", tmp] + sorted(objs)
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError("link failed:\n%s%s" % (r.stdout, r.stderr))
    os.replace(tmp, LIB)
    if verbose:
        sys.stderr.write("".join(logs))
    return LIB


if __name__ == "__main__":
    print(build(verbose="-v" in sys.argv))
