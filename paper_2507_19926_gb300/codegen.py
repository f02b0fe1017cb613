"""Emits CUDA source for the data-oblivious networks built by ``netgen``.

Each (k, t_w, t_h) network becomes a struct with one templated device
function: straight-line SSA code of ``KO::mn`` / ``KO::mx`` calls, each
shared-memory input loaded just before its first use at an offset that the
layout class ``L`` folds into a constant.  The kernel template in
``csrc/mf_oblivious.cuh`` supplies ``KO`` (packed u16x2 keys, u32 keys,
32/64-bit argmedian records) and ``L``.

The generated files go to a build directory; nothing here runs on the GPU.
"""
from __future__ import annotations

import os

from . import netgen


def form_suffix(form):
    """Name suffix of a network form (bit 0: root rows from shared memory,
    bit 1: lazy extra rows/columns, bit 2: pressure-aware order, bit 3: the
    direct kernel -- footprint in registers, no shared memory)."""
    return (("_rs" if form & 1 else "") + ("_lz" if form & 2 else "") + ("_pr" if form & 4 else "") +
            ("_dr" if form & 8 else "") + ("_w4" if form & 16 else "") + ("_w2" if form & 32 else ""))


def wide_tiles(form):
    """Root tiles a lane of one thread runs side by side in the wide direct
    form (form bit 16: 4, bit 32: 2), else 1."""
    return 4 if form & 16 else (2 if form & 32 else 1)


def net_name(k, tw, th, unroll=None, form=0):
    """Struct name of one generated network; distinct per emission form so
    that no two translation units define the same kernel differently."""
    base = "Net_k%d_%dx%d" % (k, tw, th)
    if unroll is None:
        return base
    return base + ("_flat" if unroll < 0 else "_u%d" % unroll) + form_suffix(form)


def sort_name(n):
    return "ColSort_%d" % n


def emit_network(net, name, sync_every=0, direct=False, wide=1):
    """sync_every > 0 inserts a block barrier after every that many ops: all
    threads of a block run this same branch-free code, so the barrier only
    keeps the block's warps within one window of the (very long) program,
    which the instruction cache can then hold."""
    lines = []
    w = lines.append
    w("struct %s {" % name)
    w("  static constexpr int n_ops = %d;" % netgen.n_minmax(net))
    w("  static constexpr bool rows_smem = %s;" % ("true" if any(d[0] == "row" for d in net.inputs) else "false"))
    w("  static constexpr bool direct = %s;" % ("true" if direct else "false"))
    if wide > 1:
        w("  static constexpr int wide = %d;" % wide)
    w("  template <class KO, class L, class OUT>")
    w("  static __device__ __forceinline__ void run(const typename KO::T *__restrict__ cs,")
    w("                                            const typename KO::T *__restrict__ rw,")
    w("                                            const typename KO::T *__restrict__ rs, OUT &out) {")
    w("    typedef typename KO::T T;")
    n_in = len(net.inputs)
    loaded = [False] * n_in

    def ref(v):
        if v < n_in and not loaded[v]:
            desc = net.inputs[v]
            if desc[0] == "col":
                w("    const T v%d = cs[L::col(%d, %d)];" % (v, desc[1], desc[2]))
            elif desc[0] == "row":
                w("    const T v%d = rs[L::row(%d, %d)];" % (v, desc[1], desc[2]))
            else:
                w("    const T v%d = rw[L::px(%d, %d)];" % (v, desc[1], desc[2]))
            loaded[v] = True
        return "v%d" % v

    third = getattr(net, "third", {})
    for n, (kind, a, b, v) in enumerate(net.ops):
        ra, rb = ref(a), ref(b)
        fn = "mn" if kind.startswith("min") else "mx"
        if kind.endswith("3"):
            w("    const T v%d = KO::%s3(%s, %s, %s);" % (v, fn, ra, rb, ref(third[v])))
        else:
            w("    const T v%d = KO::%s(%s, %s);" % (v, fn, ra, rb))
        if sync_every and n % sync_every == sync_every - 1:
            w("    __syncthreads();")
    for i, v in enumerate(net.outputs):
        w("    out(%d, %s);" % (i, ref(v)))
    w("  }")
    w("};")
    return "\n".join(lines) + "\n"


def emit_network_auto(net, name, sync_every=0, unroll_levels=0, direct=False, mad_select=False, wide=1):
    """The loop-rolled form (rolled.py) when the tree's children pair up,
    else the straight-line form.  unroll_levels < 0 forces straight-line.
    direct: the network runs in the register-footprint kernel, which needs
    the straight-line form (its inputs are constant indices of local
    arrays, kept in registers only when every index is a constant)."""
    from . import rolled
    if unroll_levels >= 0 and not direct:
        try:
            ir, _ = rolled.build_ir(net)
            return rolled.emit(net, ir, name, unroll_levels=unroll_levels, mad_select=mad_select), True
        except rolled.RollError:
            pass
    return emit_network(net, name, sync_every, direct, wide), False


def emit_colsort(n):
    net = netgen.column_sort_network(n)
    lines = []
    w = lines.append
    w("struct %s {" % sort_name(n))
    w("  static constexpr int n_ops = %d;" % len(net.ops))
    w("  template <class KO>")
    w("  static __device__ __forceinline__ void run(typename KO::T *v) {")
    w("    typedef typename KO::T T;")
    # inputs are ("in", i) in first-use order
    for j, desc in enumerate(net.inputs):
        w("    const T v%d = v[%d];" % (j, desc[1]))
    n_in = len(net.inputs)
    for kind, a, b, v in net.ops:
        w("    const T v%d = KO::%s(v%d, v%d);" % (v, "mn" if kind == "min" else "mx", a, b))
    for i, v in enumerate(net.outputs):
        w("    v[%d] = v%d;" % (i, v))
    if n_in == 0 and n == 1:
        pass
    w("  }")
    w("};")
    return "\n".join(lines) + "\n"


def write_if_changed(path, text):
    if os.path.exists(path):
        with open(path) as f:
            if f.read() == text:
                return False
    tmp = path + ".tmp%d" % os.getpid()
    with open(tmp, "w") as f:
        f.write(text)
    os.replace(tmp, path)
    return True


def emit_d1_sortnets(sizes=(2, 4, 8, 16, 32, 64)):
    """Register sorting networks (Batcher) for the data-aware variant's small
    sorts, as SortNet<N>::run(v) on a register array of N keys."""
    out = ["// generated by codegen.emit_d1_sortnets -- do not edit", "#pragma once", "namespace mf {",
           "template <int N> struct SortNet;"]
    for n in sizes:
        net = netgen.column_sort_network(n)
        out.append("template <> struct SortNet<%d> {" % n)
        out.append("  template <class KT> static __host__ __device__ __forceinline__ void run(KT *v) {")
        for j, desc in enumerate(net.inputs):
            out.append("    KT v%d = v[%d];" % (j, desc[1]))
        for kind, a, b, v in net.ops:
            if kind == "min":
                out.append("    KT v%d = v%d < v%d ? v%d : v%d;" % (v, a, b, a, b))
            else:
                out.append("    KT v%d = v%d < v%d ? v%d : v%d;" % (v, a, b, b, a))
        for i, v in enumerate(net.outputs):
            out.append("    v[%d] = v%d;" % (i, v))
        out.append("  }")
        out.append("};")
    out.append("}  // namespace mf")
    return "\n".join(out) + "\n"


# Volumetric data-oblivious networks: (k, t) with a t^3 tile of voxels per
# thread.  k = 3 with 2^3 tiles: 108 min/max per voxel over a 64-voxel
# footprint; k = 5 with 2^3 tiles: 643.5 per voxel over 216 voxels (a 1^3
# tile would need 2378), which fits 255 registers only with the footprint
# loaded at first use.
D3_NETS = ((3, 2), (5, 2))


def emit_d3_networks(cases=D3_NETS):
    """Straight-line register code of netgen.build3d networks, as
    D3Net<k>::run<KO>(ld, out): ld(fx, fy, fz) returns the key of footprint
    voxel (fx, fy, fz) (F = t + k - 1 a side), out receives the t^3 medians
    in (z, y, x) order.  Ops run in the register-pressure-aware order of
    netgen.schedule_pressure, and each footprint voxel is loaded just before
    its first use, so the F^3 inputs are never all live at once (k = 5:
    spills of 348-760 bytes a thread with the whole footprint loaded first,
    0-56 bytes this way)."""
    out = ["// generated by codegen.emit_d3_networks -- do not edit", "#pragma once", "namespace mf {",
           "template <int K> struct D3Net;"]
    for k, t in cases:
        net = netgen.build3d(k, t)
        net = netgen.schedule_pressure(net, list(range(len(net.outputs))))
        F = t + k - 1
        n_in = len(net.inputs)
        out.append("template <> struct D3Net<%d> {" % k)
        out.append("  static constexpr int k = %d, T = %d, F = %d, n_ops = %d;" % (k, t, F, len(net.ops)))
        out.append("  template <class KO, class LD> static __device__ __forceinline__ void run(const LD &ld,"
                   " typename KO::T *out) {")
        out.append("    typedef typename KO::T T;")
        loaded = set()

        def ref(v):
            if v < n_in:
                if v not in loaded:
                    loaded.add(v)
                    _, fx, fy, fz = net.inputs[v]
                    out.append("    const T i%d = ld(%d, %d, %d);" % (v, fx, fy, fz))
                return "i%d" % v
            return "v%d" % v

        for kind, a, b, v in net.ops:
            ra, rb = ref(a), ref(b)
            out.append("    const T v%d = KO::%s(%s, %s);" % (v, "mn" if kind == "min" else "mx", ra, rb))
        for i, v in enumerate(net.outputs):
            out.append("    out[%d] = %s;" % (i, ref(v)))
        out.append("  }")
        out.append("};")
    out.append("}  // namespace mf")
    return "\n".join(out) + "\n"
