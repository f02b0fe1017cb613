"""Loop-rolled form of a data-oblivious network.

At every split of hierarchical tiling (paper Sec. 3.4) the two children run
the same network on different inputs: same list sizes, same keep ranges,
same comparators.  ``build_ir`` pairs the ops of the two child subtrees
(their creation order is identical by construction), keeps the first child
as the representative and turns each split into a two-iteration loop; an
operand that differs between the children becomes a select on the loop
variable (register values) or a loop-dependent shared-memory offset
(inputs).  The op count per pixel is unchanged; the code per tile shrinks
from the whole tree to the root part plus one child per level, which keeps
the instruction stream of a GPU thread small enough to stay cached.

IR (nested lists):
  ("op", v, kind, opa, opb)    v = kind(opa, opb); kind "min" | "max"
  ("load", v, addr)            v = input addressed by ``addr``
  ("loop", level, body)        for s_level in (0, 1): body
  ("out", pix, opnd)           output pixel ``pix`` (row-major in tile) = opnd
Operands:  ("v", id) | ("sel", levels, {bits: operand})
Addresses / pixels:  ("const", x) | ("var", levels, {bits: x})
"""
from __future__ import annotations

import itertools


class RollError(Exception):
    pass


def _depth(net, v):
    return len(net.op_path[v])


def build_ir(net):
    n_in = len(net.inputs)
    third = getattr(net, "third", {})
    ops = {v: (kind, a, b, third.get(v)) for kind, a, b, v in net.ops}
    sched = [v for _, _, _, v in net.ops]
    paths = net.op_path
    leaf_paths = sorted(net.leaf_pixel)
    D = max(len(p) for p in leaf_paths)
    internal = set()
    for p in leaf_paths:
        for i in range(len(p)):
            internal.add(p[:i])
    # pair the two child subtrees of every internal node in creation order
    by_prefix = {}
    for v in sorted(ops):  # creation order
        p = paths[v]
        for i in range(len(p) + 1):
            by_prefix.setdefault(p[:i], []).append(v)
    fwd, inv = {}, {}
    for P in internal:
        A = by_prefix.get(P + (0,), [])
        B = by_prefix.get(P + (1,), [])
        if len(A) != len(B):
            raise RollError("children of %s differ in size (%d vs %d)" % (P, len(A), len(B)))
        for a, b in zip(A, B):
            if ops[a][0] != ops[b][0]:
                raise RollError("children of %s differ in op kinds" % (P,))
        fwd[P] = dict(zip(A, B))
        inv[P] = dict(zip(B, A))

    def cp(o, bits):
        """The counterpart of representative op o under loop bits."""
        for i, b in enumerate(bits):
            if b:
                p = paths[o]
                if len(p) <= i:
                    break
                o = fwd[p[:i]][o]
        return o

    def rep(t):
        """The representative (all-zero path) of an op."""
        p = paths[t]
        for i in range(len(p) - 1, -1, -1):
            if p[i] == 1:
                t = inv[p[:i]][t]
        return t

    def operand(target_fn, Dc):
        """Expression for a value that is target_fn(bits) at loop bits (len Dc)."""
        table = {}
        for bits in itertools.product((0, 1), repeat=Dc):
            t = target_fn(bits)
            if t < n_in:
                table[bits] = ("in", t)
            else:
                p = paths[t]
                if tuple(bits[:len(p)]) != p:
                    raise RollError("operand not available at its use")
                table[bits] = ("v", rep(t))
        return _compress(table, Dc)

    def _compress(table, Dc):
        vals = set(table.values())
        if len(vals) == 1:
            return next(iter(vals))
        levels = [L for L in range(Dc)
                  if any(table[b] != table[b[:L] + (1 - b[L],) + b[L + 1:]] for b in table)]
        sub = {}
        for bits, val in table.items():
            key = tuple(bits[L] for L in levels)
            if sub.setdefault(key, val) != val:
                raise RollError("select does not factor")
        return ("sel", tuple(levels), sub)

    ops_at = {}
    for v in sched:
        ops_at.setdefault(paths[v], []).append(v)

    def block(P):
        L = len(P)
        out = []
        for o in ops_at.get(P, []):
            kind = ops[o][0]
            oa = operand(lambda bits, pos=1: ops[cp(o, bits)][pos], L)
            ob = operand(lambda bits, pos=2: ops[cp(o, bits)][pos], L)
            oc = operand(lambda bits, pos=3: ops[cp(o, bits)][pos], L) if kind.endswith("3") else None
            out.append(("op", o, kind, oa, ob, oc))
        if P in net.leaf_pixel:
            pix = {bits: ("const", net.leaf_pixel[bits]) for bits in itertools.product((0, 1), repeat=L)}
            val = operand(lambda bits: net.outputs[net.leaf_pixel[bits]], L)
            out.append(("out", _compress(pix, L), val))
        elif P in internal:
            out.append(("loop", L, block(P + (0,))))
        return out

    try:
        ir = block(())
    except KeyError as e:  # an operand outside the paired subtrees
        raise RollError("unpaired operand %s" % e)
    return ir, D


def _sel_value(opnd, svals, vals, inputs_fn):
    kind = opnd[0]
    if kind == "v":
        return vals[opnd[1]]
    if kind == "in":
        return inputs_fn(opnd[1])
    levels, sub = opnd[1], opnd[2]
    key = tuple(svals[L] for L in levels)
    return _sel_value(sub[key], svals, vals, inputs_fn)


def interpret(net, ir, col_fn, px_fn, row_fn=None):
    """Runs the rolled IR on the host (numpy arrays, one entry per tile);
    returns the outputs in row-major pixel order."""
    import numpy as np
    vals = {}
    outs = {}

    def inputs_fn(i):
        desc = net.inputs[i]
        return {"col": col_fn, "px": px_fn, "row": row_fn}[desc[0]](desc[1], desc[2])

    def run(blk, svals):
        for st in blk:
            if st[0] == "op":
                _, v, kind, oa, ob, oc = st
                f = np.minimum if kind.startswith("min") else np.maximum
                vals[v] = f(_sel_value(oa, svals, vals, inputs_fn), _sel_value(ob, svals, vals, inputs_fn))
                if oc is not None:
                    vals[v] = f(vals[v], _sel_value(oc, svals, vals, inputs_fn))
            elif st[0] == "loop":
                for s in (0, 1):
                    run(st[2], svals + [s])
            else:
                pix = st[1]
                while pix[0] == "sel":
                    pix = pix[2][tuple(svals[L] for L in pix[1])]
                outs[pix[1]] = _sel_value(st[2], svals, vals, inputs_fn)

    run(ir, [])
    return [outs[i] for i in range(net.tw * net.th)]


def _value_pairs(net, blk, level):
    """(value a, value b) of every one-level value select on loop `level`
    inside blk (nested loops included) whose two values are both defined
    outside that loop, in first-use order."""
    pairs = []

    def visit(o):
        if o is None or o[0] != "sel":
            return
        leaves = list(o[2].values())
        if o[1] == (level,) and all(x[0] == "v" for x in leaves):
            pr = (o[2][(0,)][1], o[2][(1,)][1])
            if pr not in pairs and all(len(net.op_path[v]) <= level for v in pr):
                pairs.append(pr)
        else:
            for x in leaves:
                visit(x)

    def walk(b):
        for st in b:
            if st[0] == "op":
                for o in st[3:6]:
                    visit(o)
            elif st[0] == "loop":
                walk(st[2])
            else:
                visit(st[2])
    walk(blk)
    return pairs


def emit(net, ir, name, max_sel_levels=4, unroll_levels=0, mad_select=False):
    """CUDA source of the rolled network: a struct whose run() takes the
    thread's shared-memory bases and a store callback out(pixel, value).
    The loops of the first `unroll_levels` tree levels are emitted twice with
    a constant loop variable instead (selects fold away, code doubles).
    mad_select: a one-level select between two values a, b defined outside
    its loop becomes a + s * (b - a) (one multiply-add, with b - a computed
    once before the loop), which moves it off the integer min/max pipe."""
    lines = []
    w = lines.append
    n_in = len(net.inputs)
    w("struct %s {" % name)
    w("  static constexpr int n_ops = %d;" % sum(2 if op[0].endswith("3") else 1 for op in net.ops))
    w("  static constexpr bool rows_smem = %s;" % ("true" if any(d[0] == "row" for d in net.inputs) else "false"))
    w("  static constexpr bool direct = false;")
    w("  template <class KO, class L, class OUT>")
    w("  static __device__ __forceinline__ void run(const typename KO::T *__restrict__ cs,")
    w("                                            const typename KO::T *__restrict__ rw,")
    w("                                            const typename KO::T *__restrict__ rs, OUT &out) {")
    w("    typedef typename KO::T T;")
    counter = [0]

    def addr_of(i):
        desc = net.inputs[i]
        if desc[0] == "col":
            return "cs", "L::col(%d, %d)" % (desc[1], desc[2])
        if desc[0] == "row":
            return "rs", "L::row(%d, %d)" % (desc[1], desc[2])
        return "rw", "L::px(%d, %d)" % (desc[1], desc[2])

    def sel_expr(levels, sub, leaf):
        # nested conditional over loop variables, outermost level first
        def rec(li, prefix):
            if li == len(levels):
                return leaf(sub[tuple(prefix)])
            return "(s%d ? %s : %s)" % (levels[li], rec(li + 1, prefix + [1]), rec(li + 1, prefix + [0]))
        return rec(0, [])

    diffs = {}  # (level, a, b) -> name of the hoisted b - a

    def emit_block(blk, indent, scope_loads):
        pad = "  " * indent
        loads = dict(scope_loads)

        def load_expr(opnd):
            # opnd: ("in", i) or ("sel", levels, {bits: ("in", i)})
            key = repr(opnd)
            if key in loads:
                return loads[key]
            var = "l%d" % counter[0]
            counter[0] += 1
            if opnd[0] == "in":
                base, off = addr_of(opnd[1])
                w("%sconst T %s = %s[%s];" % (pad, var, base, off))
            else:
                bases = {addr_of(x[1])[0] for x in opnd[2].values()}
                if len(bases) != 1:
                    raise RollError("input select across arrays")
                base = bases.pop()
                off = sel_expr(opnd[1], opnd[2], lambda x: addr_of(x[1])[1])
                w("%sconst T %s = %s[%s];" % (pad, var, base, off))
            loads[key] = var
            return var

        def opnd_expr(opnd):
            if opnd[0] == "v":
                return "v%d" % opnd[1]
            if opnd[0] == "in":
                return load_expr(opnd)
            # select: inputs -> one load with a selected address; values -> select
            leaves = list(opnd[2].values())
            if all(x[0] == "in" for x in leaves):
                return load_expr(opnd)
            if len(opnd[1]) > max_sel_levels:
                raise RollError("select too deep")
            if len(opnd[1]) == 1 and all(x[0] == "v" for x in leaves):
                key = (opnd[1][0], opnd[2][(0,)][1], opnd[2][(1,)][1])
                if key in diffs:
                    return "mad_sel((unsigned)s%d, %s, v%d)" % (key[0], diffs[key], key[1])
            return sel_expr(opnd[1], opnd[2], lambda x: opnd_expr(x))

        for st in blk:
            if st[0] == "op":
                _, v, kind, oa, ob, oc = st
                ea, eb = opnd_expr(oa), opnd_expr(ob)
                fn = ("mn" if kind.startswith("min") else "mx") + ("3" if oc is not None else "")
                args = "%s, %s" % (ea, eb) if oc is None else "%s, %s, %s" % (ea, eb, opnd_expr(oc))
                w("%sconst T v%d = KO::%s(%s);" % (pad, v, fn, args))
            elif st[0] == "loop":
                lvl = st[1]
                if lvl < unroll_levels:
                    for sv in (0, 1):
                        w("%s{" % pad)
                        w("%s  const int s%d = %d;" % (pad, lvl, sv))
                        emit_block(st[2], indent + 1, {})
                        w("%s}" % pad)
                else:
                    if mad_select:
                        for a, b in _value_pairs(net, st[2], lvl):
                            nm = "d%d_%d_%d" % (lvl, a, b)
                            w("%sconst T %s = v%d - v%d;" % (pad, nm, b, a))
                            diffs[(lvl, a, b)] = nm
                    w("%s#pragma unroll 1" % pad)
                    w("%sfor (int s%d = 0; s%d < 2; s%d++) {" % (pad, lvl, lvl, lvl))
                    emit_block(st[2], indent + 1, loads)
                    w("%s}" % pad)
            else:
                pix = st[1]
                pe = str(pix[1]) if pix[0] == "const" else sel_expr(pix[1], pix[2], lambda x: str(x[1]))
                w("%sout(%s, %s);" % (pad, pe, opnd_expr(st[2])))

    emit_block(ir, 2, {})
    w("  }")
    w("};")
    return "\n".join(lines) + "\n"
