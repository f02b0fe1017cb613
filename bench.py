"""Benchmark of the k x k median filter on synthetic inputs (one JSON line).

Default workload: the 30-megapixel RGB photograph case of the paper's teaser
(Fig. 1): 3 planar u8 channels of 4480 x 6720, 17 x 17 median, synthetic
photo-like content (smooth field + Gaussian noise + 5% impulses).  A step is
one full filter of that image; inputs are resident in HBM; L2 is flushed
(256 MB write) between timed steps, outside the timed events.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

N > 1 (under torchrun): every rank filters its own copy (independent
replicas, no collective on the data path); value = all ranks' pixels / the
slowest rank's time.  --impl reference times the CPU oracle on a bounded
sample of the same workload (the reference arm of this tier).
"""
import argparse
import json
import os
import re
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

PAPER_MPIX_S = 6720 * 4480 * 3 / 2.2e-3 / 1e6  # teaser: 17x17, 30 MP RGB u8 in 2.2 ms (L40S)

WORKLOADS = {
    # name: (channels, H, W, dtype, k, generator)
    "photo_rgb_30mp_u8_k17": (3, 4480, 6720, "u8", 17, "photo"),
    "gray_640x480_u8_k5": (1, 480, 640, "u8", 5, "uniform"),
}
for _dt in ("u8", "u16", "u32", "f32"):
    for _k in (3, 5, 7, 9, 11, 15, 21, 31, 45, 61, 75):
        WORKLOADS["sweep_4096_%s_k%d" % (_dt, _k)] = (1, 4096, 4096, _dt, _k, "uniform")


def make_input(name):
    from paper_2507_19926_gb300 import synth
    C, H, W, dt, k, gen = WORKLOADS[name]
    if gen == "photo":
        return synth.photo_rgb(H, W)
    return synth.uniform((C, H, W), dt, synth.SEED_BASE + 2)


def to_device(a, dev):
    """numpy u8/u16/u32/f32 array -> CUDA tensor holding the same bits."""
    import numpy as np
    import torch
    a = np.ascontiguousarray(a)
    if a.dtype == np.uint16:
        return torch.from_numpy(a.view(np.int16)).to(dev).view(torch.uint16)
    if a.dtype == np.uint32:
        return torch.from_numpy(a.view(np.int32)).to(dev).view(torch.uint32)
    return torch.from_numpy(a).to(dev)


def gpu_uuid(dev):
    import torch
    try:
        u = str(torch.cuda.get_device_properties(dev).uuid)
        return u if u.startswith("GPU-") else "GPU-" + u
    except Exception:
        return str(dev.index or 0)


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), "--query-gpu=" + self.FIELDS,
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except (OSError, ValueError):
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.thread.join(timeout=2)
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            p = [s.strip() for s in ln.split(",")]
            if len(p) < 9:
                continue
            try:
                sm.append(float(p[1]))
                mx.append(float(p[2]))
            except ValueError:
                continue
            for n, v in zip(names, p[5:9]):
                if v.lower() == "active":
                    reasons.add(n)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


def algorithmic_ops_per_px(k):
    """Min/max element operations per output pixel of the cheapest
    hierarchy the network generator can emit for k (root tiles 1..16,
    with the block-wide column sort amortised over the tile width)."""
    from paper_2507_19926_gb300 import netgen
    best = None
    t = 1
    while t <= min(k, 16):
        if t * 2 <= k + 1 or t == 1:
            net = netgen.build(k, t)
            cs = netgen.column_sort_network(k - t + 1)
            v = len(net.ops) / (t * t) + len(cs.ops) / t
            best = v if best is None else min(best, v)
        t *= 2
    return best


_O1_NAME = re.compile(r"o1_launch_k(\d+)_(\d+)x(\d+)_b(\d+)x(\d+)_u(m1|\d+)((?:_[a-z][a-z0-9])*)_MF_\w+?_Ko(U16x2|U32)")


def o1_executed_per_px(plan):
    """Min/max instructions the data-oblivious kernel named in `plan` issues
    per output pixel: its generated network with three-input fusion (one
    instruction per fused op) plus the column sorts, divided by the pixels
    one instruction serves (two tiles a register for packed 16-bit keys).
    None when the plan names no such kernel."""
    from paper_2507_19926_gb300 import netgen
    m = _O1_NAME.search(plan)
    if not m:
        return None
    k, tw, th, bx, by = (int(v) for v in m.groups()[:5])
    form = m.group(7)
    lanes = 2 if m.group(8) == "U16x2" else 1
    net = netgen.build(k, tw, th, rows_smem="_rs" in form, lazy="_lz" in form, pressure="_pr" in form)
    ops = len(netgen.fuse3(net).ops)
    cs = len(netgen.column_sort_network(k - th + 1).ops)
    run = 4 if "_w4" in form else (2 if "_w2" in form else 1)
    if "_dr" in form:  # direct forms: every thread sorts its own footprint columns
        per_thread = run * ops + (run * tw + k - 1) * cs
    else:  # block-wide column sort over the block footprint, shared by its threads
        per_thread = ops + by * (bx * tw + k - 1) * cs / (bx * by)
    return per_thread / (run * tw * th * lanes)


_PROBE = {}


def probe_ipc(sms, mhz, lanes):
    """Measured min/max instructions per clock per SM (mf_probe_minmax, u32
    or packed u16x2), at the SM clock `mhz` sampled while the bench ran."""
    import paper_2507_19926_gb300 as mf
    if lanes not in _PROBE:
        rate, _ = mf.mf_probe_minmax(1 if lanes == 2 else 0)
        _PROBE[lanes] = rate / (sms * mhz * 1e6)
    return _PROBE[lanes]


def d1_key_bytes(dt, with_idx=False):
    """Bytes of one data-aware shared-memory key: 8-bit values as 8-bit keys,
    16-bit as 16, 32-bit as 32; argmedian records add 16 or 32 bits."""
    if with_idx:
        return 8 if dt in ("u32", "f32") else 4
    return {"u8": 1, "u16": 2, "u32": 4, "f32": 4}[dt]


def roofline_entry(plan, dt, k, px, ms, sms, peaks, probe_mhz=None, with_idx=False):
    """Roofline of one filter call: the floor is the slower of its HBM bytes
    (in + out) and its work at the unit that bounds the variant -- min/max
    issue for the data-oblivious networks (the cheapest hierarchy the
    generator emits), shared-memory bytes for the data-aware merges (every
    merged or sorted element read once and written once).  `frac` =
    floor / measured time for the bound that is larger."""
    import re
    max_mhz = peaks.get("sm_max_mhz", 2070.0)
    es = {"u8": 1, "u16": 2, "u32": 4, "f32": 4}[dt]
    hbm_gbs = peaks.get("hbm_gbs") or 6800.0
    t_hbm = px * (2 * es + (4 if with_idx else 0)) / (hbm_gbs * 1e9)
    out = {"hbm_frac": round(t_hbm / (ms * 1e-3), 4)}
    t_work, bound = None, None
    if "oblivious" in plan:
        lanes = 2 if dt in ("u8", "u16") else 1
        ipc = probe_ipc(sms, probe_mhz or max_mhz, lanes)
        ipc_nominal = 64.0 if ipc < 96 else 128.0
        peak = sms * ipc_nominal * max_mhz * 1e6 * lanes  # element-ops/s
        ops = algorithmic_ops_per_px(k)
        t_work, bound = ops * px / peak, "alu"
        out["alu_frac"] = round(t_work / (ms * 1e-3), 4)
        ex = o1_executed_per_px(plan)
        if ex is not None:  # instructions actually issued, against the instruction rate
            out["executed_instr_frac"] = round(ex * px / (sms * ipc_nominal * max_mhz * 1e6) / (ms * 1e-3), 4)
    elif "data-aware" in plan:
        m = re.search(r"merged/px=([\d.]+) sorted/px=([\d.]+)", plan)
        if m:
            kb = d1_key_bytes(dt, with_idx)
            elems = float(m.group(1)) + float(m.group(2))
            t_work, bound = elems * 2 * kb * px / (sms * 128 * max_mhz * 1e6), "smem"
            out["smem_frac"] = round(t_work / (ms * 1e-3), 4)
            # the same element accesses against one conflict-free 32-lane
            # wavefront a clock a SM (the access rate, whatever the key width)
            out["smem_access_frac"] = round(elems * 2 * px / (sms * 32 * max_mhz * 1e6) / (ms * 1e-3), 4)
    if t_work is None or t_hbm >= t_work:
        out["bound"], out["frac"] = "hbm", out["hbm_frac"]
    else:
        out["bound"], out["frac"] = bound, round(t_work / (ms * 1e-3), 4)
    return out


def measured_traffic(plan):
    """DRAM bytes per launch (read + write) that an ncu capture recorded for
    the kernel the plan names, from profiles/dram_traffic.md, or None when no
    row matches the kernel's current build hash (the kernel changed since)."""
    import re
    from paper_2507_19926_gb300 import build
    m = re.search(r"kernel=(\S+)", plan)
    if not m:
        return None
    h = build.kernel_source_hash(m.group(1))
    try:
        with open(os.path.join(ROOT, "profiles", "dram_traffic.md")) as f:
            for line in f:
                cells = [c.strip() for c in line.strip().strip("|").split("|")]
                if len(cells) >= 4 and cells[0] == "`%s`" % m.group(1) and h and cells[1] == "`%s`" % h:
                    return int(cells[2]) + int(cells[3])
    except (OSError, ValueError):
        return None
    return None


def read_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f)
    except (OSError, ValueError):
        return {}


def cpu_sample(x, k, seconds=8.0):
    """Times the oracle on sampled rows of x until about `seconds` have passed."""
    import numpy as np
    import oracle
    from paper_2507_19926_gb300 import synth
    C, H, W = x.shape
    g = synth.rng(12345)
    nrows, total_px, total_s = 2, 0, 0.0
    while total_s < seconds:
        rows = np.sort(g.choice(H, size=min(nrows, H), replace=False)).astype(np.int32)
        t0 = time.perf_counter()
        oracle.median_filter_rows(x, k, rows)
        dt = time.perf_counter() - t0
        total_px += C * len(rows) * W
        total_s += dt
        nrows = max(2, min(H, int(nrows * max(1.5, min(8.0, (seconds - total_s) / max(dt, 1e-3))))))
    return total_px / total_s / 1e6, total_px, total_s


# one metric for both arms: output channel-pixels filtered per second
METRIC = "median filter throughput (output channel-pixels per second)"


def run_reference(args):
    ws, rank, _ = dist_env()
    if rank != 0:
        return
    import numpy as np
    import oracle
    C, H, W, dt, k, _ = WORKLOADS[args.workload]
    x = make_input(args.workload)
    cores = oracle.max_threads()
    g = __import__("paper_2507_19926_gb300.synth", fromlist=["rng"]).rng(777)
    rows_per_step = max(1, min(H, int(args.ref_rows)))
    times, px = [], 0
    for step in range(args.warmup + args.steps):
        rows = np.sort(g.choice(H, size=rows_per_step, replace=False)).astype(np.int32)
        t0 = time.perf_counter()
        oracle.median_filter_rows(x, k, rows)
        el = time.perf_counter() - t0
        if step >= args.warmup:
            times.append(el)
            px += C * rows_per_step * W
    total = sum(times)
    value = px / total / 1e6
    sample = "%d random rows x %d channels x %d columns per step of %s" % (rows_per_step, C, W, args.workload)
    print(json.dumps({
        "impl": "reference", "metric": METRIC,
        "value": value, "unit": "Mpix/s", "n_gpus": ws, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1e3 * total / len(times), "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": dt, "data": "synthetic",
        "config": {"workload": args.workload, "channels": C, "H": H, "W": W, "k": k},
        "cpu_baseline": {"value": value, "unit": "Mpix/s", "cores": cores, "kind": "oracle", "sample": sample},
        "e2e": {"value": value, "unit": "Mpix/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }))


def aggregate(total_ms, px_per_step, steps, world_size, device=None):
    """Whole-job throughput over replicas: every rank filtered px_per_step
    pixels per step; the job took as long as the slowest rank.  Returns
    (Mpix/s, slowest rank's ms)."""
    if world_size > 1:
        import torch
        import torch.distributed as dist
        t = torch.tensor([float(total_ms)], dtype=torch.float64, device=device)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        total_ms = float(t.item())
    return world_size * px_per_step * steps / (total_ms * 1e-3) / 1e6, total_ms


def _time_ms(fn, stream, reps, flush=None):
    """Median of per-call CUDA-event times on `stream` (L2 flushed before each)."""
    import torch
    ts = []
    for i in range(reps):
        if flush is not None:
            flush.fill_(i & 0xFF)
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        fn()
        b.record(stream)
        torch.cuda.synchronize()
        ts.append(a.elapsed_time(b))
    return statistics.median(ts)


def bench_batched(dev, stream, flush, reps=5):
    """64 images of uneven sizes/dtypes/k: one graph launch vs 64 plain calls."""
    import torch
    import paper_2507_19926_gb300 as mf
    from paper_2507_19926_gb300 import synth
    codes = {"u8": mf.MF_U8, "u16": mf.MF_U16, "f32": mf.MF_F32}
    descs, bufs, px = [], [], 0
    for d in synth.batch_descs():
        x = to_device(synth.uniform((1, d["H"], d["W"]), d["dtype"], d["seed"]), dev)
        y = torch.empty_like(x)
        bufs.append((x, y, d))
        descs.append(mf.ImageDesc(x.data_ptr(), y.data_ptr(), d["H"], d["W"], d["W"] * x.element_size(), 1,
                                  codes[d["dtype"]], d["k"]))
        px += d["H"] * d["W"]
    sptr = stream.cuda_stream

    def plain():
        for x, y, d in bufs:
            mf.mf_median_filter(x.data_ptr(), y.data_ptr(), d["H"], d["W"], d["W"] * x.element_size(), 1,
                                codes[d["dtype"]], d["k"], mf.MF_BORDER_CLAMP, sptr)

    def measure(plan):
        try:
            kernels, items = mf.mf_batch_describe(plan)
            run = lambda: mf.mf_batch_run(plan, sptr)
            for _ in range(2):
                run()
            t_batch = _time_ms(run, stream, reps, flush)
        finally:
            mf.mf_batch_plan_destroy(plan)
        plain()
        t_plain = _time_ms(plain, stream, reps, flush)
        return kernels, items, t_batch, t_plain

    # default kernels (no tuning entries yet), then a plan that autotunes
    # every (k, dtype, size bucket) of the batch first; plain launches
    # after it use the same tuning table
    kernels, items, t_batch, t_plain = measure(mf.mf_batch_plan_create(descs))
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    tuned = mf.mf_batch_plan_create_ex(descs, 1)
    tune_s = time.perf_counter() - t0
    tk, ti, tt_batch, tt_plain = measure(tuned)
    return {"workload": "64 images, log-uniform 256x256..4096x3072, u8/u16/f32, odd k 3..31",
            "pixels": px, "graph_kernels": kernels, "work_items": items,
            "batched_ms": t_batch, "plain_ms": t_plain, "batched_mpix_s": px / t_batch / 1e3,
            "plain_mpix_s": px / t_plain / 1e3, "speedup": t_plain / t_batch,
            "tuned": {"tuning_s": tune_s, "graph_kernels": tk, "work_items": ti, "batched_ms": tt_batch,
                      "plain_ms": tt_plain, "batched_mpix_s": px / tt_batch / 1e3, "speedup": tt_plain / tt_batch,
                      "vs_untuned_batch": t_batch / tt_batch}}


def bench_small(dev, stream, n_graph=200, reps=20):
    """640 x 480 u8, k = 5 (a launch-latency-bound frame): the time of one
    launch, and back-to-back launches replayed from one CUDA graph."""
    import torch
    import paper_2507_19926_gb300 as mf
    from paper_2507_19926_gb300 import synth
    H, W, k = 480, 640, 5
    x = to_device(synth.uniform((1, H, W), "u8", synth.SEED_BASE + 0), dev)
    y = torch.empty_like(x)
    call = lambda s: mf.mf_median_filter(x.data_ptr(), y.data_ptr(), H, W, W, 1, mf.MF_U8, k,
                                         mf.MF_BORDER_CLAMP, s)
    with torch.cuda.stream(stream):
        for _ in range(3):
            call(stream.cuda_stream)
        ts = []
        for _ in range(reps):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            call(stream.cuda_stream)
            e1.record(stream)
            e1.synchronize()
            ts.append(e0.elapsed_time(e1))
    single = statistics.median(ts)
    # n_graph launches captured once, replayed: no per-launch CPU cost
    g = torch.cuda.CUDAGraph()
    cap = torch.cuda.Stream(device=dev)
    cap.wait_stream(torch.cuda.current_stream(dev))
    with torch.cuda.stream(cap):
        with torch.cuda.graph(g, stream=cap):
            for _ in range(n_graph):
                call(cap.cuda_stream)
    torch.cuda.current_stream(dev).wait_stream(cap)
    g.replay()
    torch.cuda.synchronize(dev)
    tg = []
    for _ in range(5):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        g.replay()
        e1.record()
        e1.synchronize()
        tg.append(e0.elapsed_time(e1))
    per = statistics.median(tg) / n_graph
    return {"workload": "1 x 480 x 640 u8, k = 5", "single_launch_ms": single,
            "graph_replayed_ms_per_frame": per, "graph_mpix_s": H * W / per / 1e3,
            "frames_per_graph": n_graph, "plan": mf.mf_describe(H, W, 1, mf.MF_U8, k)}


def bench_fwd_bwd(dev, stream, flush, reps=5):
    """f32 16x1x1024x1024, k = 9 and 25: forward, forward + argmedian, and
    forward + argmedian + backward (atomic and deterministic)."""
    import torch
    import paper_2507_19926_gb300 as mf
    from paper_2507_19926_gb300 import synth
    N, H, W = 16, 1024, 1024
    x = torch.from_numpy(synth.normal_f32((N, 1, H, W), synth.SEED_BASE + 4)).to(dev)
    g = torch.from_numpy(synth.normal_f32((N, 1, H, W), synth.SEED_BASE + 5)).to(dev)
    y = torch.empty_like(x)
    idx = torch.empty(x.shape, dtype=torch.int32, device=dev)
    gi = torch.empty_like(x)
    sptr = stream.cuda_stream
    out = {}
    for k in (9, 25):
        fwd = lambda: mf.mf_median_filter_ex(x.data_ptr(), y.data_ptr(), H, W, 4 * W, N, mf.MF_F32, k,
                                             mf.MF_BORDER_CLAMP, mf.MF_AUTO, None, 0, sptr)
        fwd_idx = lambda: mf.mf_median_filter_ex(x.data_ptr(), y.data_ptr(), H, W, 4 * W, N, mf.MF_F32, k,
                                                 mf.MF_BORDER_CLAMP, mf.MF_AUTO, idx.data_ptr(), 4 * W, sptr)
        bwd_a = lambda: mf.mf_median_filter_bwd(g.data_ptr(), idx.data_ptr(), gi.data_ptr(), H, W, 4 * W, 4 * W, N, k,
                                                mf.MF_GRAD_ATOMIC, sptr)
        bwd_d = lambda: mf.mf_median_filter_bwd(g.data_ptr(), idx.data_ptr(), gi.data_ptr(), H, W, 4 * W, 4 * W, N, k,
                                                mf.MF_GRAD_DETERMINISTIC, sptr)
        for f in (fwd, fwd_idx, bwd_a, bwd_d):
            f()
        t_f = _time_ms(fwd, stream, reps, flush)
        t_fi = _time_ms(fwd_idx, stream, reps, flush)
        t_a = _time_ms(bwd_a, stream, reps, flush)
        t_d = _time_ms(bwd_d, stream, reps, flush)
        px = N * H * W
        out["k%d" % k] = {"fwd_ms": t_f, "fwd_argmedian_ms": t_fi, "bwd_atomic_ms": t_a,
                          "bwd_deterministic_ms": t_d, "fwd_mpix_s": px / t_f / 1e3,
                          "fwd_bwd_atomic_mpix_s": px / (t_fi + t_a) / 1e3,
                          "fwd_bwd_deterministic_mpix_s": px / (t_fi + t_d) / 1e3,
                          "fwd_plan": mf.mf_describe(H, W, N, mf.MF_F32, k)}
    return out


def bench_rect(dev, stream, flush, reps=3, cases=(("u8", 31, 7), ("u8", 7, 31), ("u16", 15, 3), ("f32", 1, 25),
                                                    ("u32", 45, 13))):
    """4096 x 4096 single-plane images, windows of kw columns by kh rows
    (mf_median_filter_rect)."""
    import torch
    import paper_2507_19926_gb300 as mf
    from paper_2507_19926_gb300 import synth
    codes = {"u8": mf.MF_U8, "u16": mf.MF_U16, "u32": mf.MF_U32, "f32": mf.MF_F32}
    res = []
    sptr = stream.cuda_stream
    for dt, kw, kh in cases:
        x = to_device(synth.uniform((1, 4096, 4096), dt, synth.SEED_BASE + 2), dev)
        y = torch.empty_like(x)
        pitch = 4096 * x.element_size()
        f = lambda: mf.mf_median_filter_rect(x.data_ptr(), y.data_ptr(), 4096, 4096, pitch, 1, codes[dt], kw, kh,
                                             None, 0, sptr)
        f()
        ms = _time_ms(f, stream, reps, flush)
        res.append({"dtype": dt, "kw": kw, "kh": kh, "ms": round(ms, 4), "mpix_s": round(4096 * 4096 / ms / 1e3, 1)})
    return res


SWEEP_KS = (3, 5, 7, 9, 11, 15, 21, 31, 45, 61, 75)


def bench_sweep(dev, stream, flush, peaks, probe_mhz, reps=3, ks=SWEEP_KS, dts=("u8", "u16", "u32", "f32")):
    """4096 x 4096 single-plane images in every dtype, k over the sweep's
    set, two value distributions (uniform over the full range, and 16
    levels: heavy ties), auto variant; each cell with its roofline."""
    import torch
    import paper_2507_19926_gb300 as mf
    from paper_2507_19926_gb300 import synth
    codes = {"u8": mf.MF_U8, "u16": mf.MF_U16, "u32": mf.MF_U32, "f32": mf.MF_F32}
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    res = []
    sptr = stream.cuda_stream
    px = 4096 * 4096
    for dt in dts:
        for dist, gen in (("uniform", synth.uniform), ("levels16", synth.levels16)):
            x = to_device(gen((1, 4096, 4096), dt, synth.SEED_BASE + 2), dev)
            y = torch.empty_like(x)
            pitch = 4096 * x.element_size()
            for k in ks:
                f = lambda: mf.mf_median_filter(x.data_ptr(), y.data_ptr(), 4096, 4096, pitch, 1, codes[dt], k,
                                                mf.MF_BORDER_CLAMP, sptr)
                f()
                ms = _time_ms(f, stream, reps, flush)
                plan = mf.mf_describe(4096, 4096, 1, codes[dt], k)
                res.append({"dtype": dt, "dist": dist, "k": k, "ms": round(ms, 4),
                            "mpix_s": round(px / ms / 1e3, 1),
                            "roofline": roofline_entry(plan, dt, k, px, ms, sms, peaks, probe_mhz),
                            "plan": plan.split(" kernel=")[0]})
            del x, y
    return res


def bench_photo_data_aware(dev, stream, flush, peaks, probe_mhz, x, reps=5):
    """The 30 MP RGB u8 photo, k = 17, through the data-aware variant (the
    headline runs the auto choice, the data-oblivious network)."""
    import torch
    import paper_2507_19926_gb300 as mf
    C, H, W = x.shape
    y = torch.empty_like(x)
    sptr = stream.cuda_stream
    f = lambda: mf.mf_median_filter_ex(x.data_ptr(), y.data_ptr(), H, W, W, C, mf.MF_U8, 17, mf.MF_BORDER_CLAMP,
                                       mf.MF_DATA_AWARE, None, 0, sptr)
    f()
    ms = _time_ms(f, stream, reps, flush)
    plan = mf.mf_describe(H, W, C, mf.MF_U8, 17, mf.MF_DATA_AWARE)
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    return {"workload": "photo_rgb_30mp_u8_k17", "variant": "data_aware", "ms": round(ms, 4),
            "mpix_s": round(C * H * W / ms / 1e3, 1),
            "roofline": roofline_entry(plan, "u8", 17, C * H * W, ms, sms, peaks, probe_mhz), "plan": plan}


def bench_volume(dev, stream, flush, reps=3, cases=(("u8", 3, "auto"), ("u8", 3, "data_aware"), ("u8", 5, "auto"),
                                                      ("u8", 5, "data_aware"), ("f32", 5, "auto"),
                                                      ("u8", 7, "auto"), ("u8", 9, "auto"), ("u8", 15, "auto"),
                                                      ("u8", 19, "auto"), ("u16", 7, "auto"), ("f32", 3, "auto"),
                                                      ("f32", 7, "auto"), ("f32", 19, "auto"))):
    """256^3 single volumes, uniform values: the k x k x k median by
    hierarchical tiling in 3D (mf_median_filter_3d)."""
    import torch
    import paper_2507_19926_gb300 as mf
    from paper_2507_19926_gb300 import synth
    codes = {"u8": mf.MF_U8, "u16": mf.MF_U16, "u32": mf.MF_U32, "f32": mf.MF_F32}
    import re
    res = []
    sptr = stream.cuda_stream
    n = 256
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    smem_peak = sms * 128 * read_peaks().get("sm_max_mhz", 2070.0) * 1e6 / 1e9  # GB/s
    for dt, k, variant in cases:
        x = to_device(synth.uniform((n, n, n), dt, synth.SEED_BASE + 5), dev)
        y = torch.empty_like(x)
        pitch = n * x.element_size()
        f = lambda: mf.mf_median_filter_3d_ex(x.data_ptr(), y.data_ptr(), n, n, n, pitch, 1, codes[dt], k,
                                              mf.VARIANTS[variant], sptr)
        f()
        ms = _time_ms(f, stream, reps, flush)
        plan = mf.mf_median_filter_3d_describe(k, codes[dt]) if variant == "auto" else variant
        r = {"dtype": dt, "k": k, "variant": variant, "ms": round(ms, 4), "mvox_s": round(n ** 3 / ms / 1e3, 1),
             "plan": plan}
        m = re.search(r"min/max per voxel=([\d.]+)", plan)
        if m:  # ALU roofline: 32-bit min/max at 64 per clock per SM
            peak = sms * 64 * read_peaks().get("sm_max_mhz", 2070.0) * 1e6
            r["alu_roofline_frac"] = round(float(m.group(1)) * n ** 3 / (ms * 1e-3) / peak, 4)
        # shared-memory roofline, as for the 2D data-aware kernel: every
        # merged or sorted element read once and written once at the least
        m = re.search(r"merged/vox=([\d.]+) sorted/vox=([\d.]+)", plan)
        if m:
            kb = d1_key_bytes(dt)
            gbs = (float(m.group(1)) + float(m.group(2))) * 2 * kb * n ** 3 / (ms * 1e-3) / 1e9
            r["smem_roofline_frac"] = round(gbs / smem_peak, 4)
        res.append(r)
    return res


def run_ours(args):
    import numpy as np
    import torch
    import paper_2507_19926_gb300 as mf

    ws, rank, local = dist_env()
    if ws > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    dev = torch.device("cuda", local if ws > 1 else 0)
    torch.cuda.set_device(dev)
    mf.load_library()
    C, H, W, dt, k, _ = WORKLOADS[args.workload]
    code = {"u8": mf.MF_U8, "u16": mf.MF_U16, "u32": mf.MF_U32, "f32": mf.MF_F32}[dt]
    variant = mf.VARIANTS[args.variant]
    x_np = make_input(args.workload)
    x = to_device(x_np, dev)
    y = torch.empty_like(x)
    es = x.element_size()
    pitch = W * es
    stream = torch.cuda.current_stream(dev)
    sptr = stream.cuda_stream
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)

    def step():
        mf.mf_median_filter_ex(x.data_ptr(), y.data_ptr(), H, W, pitch, C, code, k,
                               mf.MF_BORDER_CLAMP, variant, None, 0, sptr)

    for _ in range(max(args.warmup, 0)):
        step()
    torch.cuda.synchronize(dev)
    if ws > 1:
        torch.distributed.barrier()
    sampler = ClockSampler(gpu_uuid(dev))
    sampler.start()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    launches0 = mf.mf_kernel_launch_count()
    torch.cuda.synchronize(dev)
    t_wall0 = time.perf_counter()
    for i in range(args.steps):
        flush.fill_(i & 0xFF)  # evict the image from L2 (outside the events)
        ev[i][0].record(stream)
        step()
        ev[i][1].record(stream)
    torch.cuda.synchronize(dev)
    t_wall = time.perf_counter() - t_wall0
    launches = mf.mf_kernel_launch_count() - launches0
    clocks = sampler.stop()
    step_ms = [a.elapsed_time(b) for a, b in ev]
    total_ms = sum(step_ms)
    px_per_step = C * H * W
    value, total_ms = aggregate(total_ms, px_per_step, args.steps, ws, dev)
    if ws > 1:
        torch.distributed.barrier()
    ms_per_step = total_ms / args.steps

    # end to end through the host-buffer entry point (pinned host memory)
    h_in = torch.empty(x.shape, dtype=x.dtype, pin_memory=True)
    h_in.copy_(x)
    h_out = torch.empty_like(h_in, pin_memory=True)
    mf.mf_median_filter_host(h_in.data_ptr(), h_out.data_ptr(), H, W, pitch, C, code, k,
                             mf.MF_BORDER_CLAMP, variant, sptr)
    e2e_times = []
    for i in range(max(3, min(args.steps, 10))):
        t0 = time.perf_counter()
        mf.mf_median_filter_host(h_in.data_ptr(), h_out.data_ptr(), H, W, pitch, C, code, k,
                                 mf.MF_BORDER_CLAMP, variant, sptr)
        e2e_times.append(time.perf_counter() - t0)
    e2e_s = statistics.median(e2e_times)
    e2e_val = ws * px_per_step / e2e_s / 1e6
    if not torch.equal(h_out.to(dev), y):
        raise SystemExit("host entry point disagrees with the device entry point")

    if rank != 0:
        return
    plan = mf.mf_describe(H, W, C, code, k, variant)
    peaks = read_peaks()
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    max_mhz = peaks.get("sm_max_mhz", 2070.0)
    # the probe's instructions per clock are taken at the clock sampled under load
    probe_mhz = clocks["sm_mhz"] if clocks else max_mhz
    roof = None
    extra = {}
    if "oblivious" in plan:
        lanes = 2 if dt in ("u8", "u16") else 1
        ops_px = algorithmic_ops_per_px(k)
        ipc = probe_ipc(sms, probe_mhz, lanes)
        ipc_nominal = 64.0 if ipc < 96 else 128.0
        peak = sms * ipc_nominal * max_mhz * 1e6 * lanes / 1e9  # G element-ops/s
        achieved = ops_px * px_per_step / (ms_per_step * 1e-3) / 1e9
        ex = o1_executed_per_px(plan)
        roof = {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "Gminmax/s",
                "frac": achieved / peak, "traffic": measured_traffic(plan),
                "basis": "%.1f min/max element-ops per pixel (cheapest generated hierarchy) x %d px; "
                         "peak = %d SMs x %d min/max instr/clk/SM x %.0f MHz x %d lanes "
                         "(probe: %.1f instr/clk/SM at %.0f MHz)" % (
                             ops_px, px_per_step, sms, ipc_nominal, max_mhz, lanes, ipc, probe_mhz)}
        if ex is not None:
            # what the kernel issues: its own network (lazy tree, fused
            # three-input ops) plus column sorts, one instruction each
            roof["executed_instr_per_px"] = round(ex, 2)
            roof["executed_instr_frac"] = ex * px_per_step / (sms * ipc_nominal * max_mhz * 1e6) / (ms_per_step * 1e-3)
    elif "data-aware" in plan:
        # shared-memory merging: every merged or sorted element is read once
        # and written once at the least; peak = 128 B/clk/SM of shared memory
        import re
        m = re.search(r"merged/px=([\d.]+) sorted/px=([\d.]+)", plan)
        if m:
            kb = d1_key_bytes(dt)
            elems_px = float(m.group(1)) + float(m.group(2))
            max_mhz = peaks.get("sm_max_mhz", 2070.0)
            peak = sms * 128 * max_mhz * 1e6 / 1e9  # GB/s
            achieved = elems_px * 2 * kb * px_per_step / (ms_per_step * 1e-3) / 1e9
            roof = {"bound": "smem", "achieved": achieved, "peak": peak, "unit": "GB/s",
                    "frac": achieved / peak, "traffic": None,
                    "basis": "(%.1f merged + %.1f sorted) elements per pixel x 2 accesses x %d B x %d px; "
                             "peak = %d SMs x 128 B/clk x %.0f MHz" % (
                                 float(m.group(1)), float(m.group(2)), kb, px_per_step, sms, max_mhz)}
    bytes_per_step = 2 * px_per_step * x.element_size()
    extra["hbm"] = {"achieved_gbs": bytes_per_step / (ms_per_step * 1e-3) / 1e9,
                    "peak_gbs": peaks.get("hbm_gbs"),
                    "frac": (bytes_per_step / (ms_per_step * 1e-3) / 1e9) / peaks["hbm_gbs"]
                    if peaks.get("hbm_gbs") else None}
    cpu = None
    if ws == 1 and not args.no_cpu:
        import oracle
        v, npx, secs = cpu_sample(x_np, k, args.cpu_seconds)
        cpu = {"value": v, "unit": "Mpix/s", "cores": oracle.max_threads(), "kind": "oracle",
               "sample": "%d output channel-pixels on random full rows of the same image (%.1f s)" % (npx, secs)}
    if ws == 1 and not args.no_extras:
        extra["small_frame"] = bench_small(dev, stream)
        extra["batched_vs_plain"] = bench_batched(dev, stream, flush)
        extra["fwd_bwd_vs_fwd"] = bench_fwd_bwd(dev, stream, flush)
        if args.workload == "photo_rgb_30mp_u8_k17":
            extra["photo_data_aware"] = bench_photo_data_aware(dev, stream, flush, peaks, probe_mhz, x)
        extra["sweep_4096"] = bench_sweep(dev, stream, flush, peaks, probe_mhz)
        extra["rect_4096"] = bench_rect(dev, stream, flush)
        extra["volume_256"] = bench_volume(dev, stream, flush)
    out = {
        "metric": METRIC,
        "value": value, "unit": "Mpix/s", "n_gpus": ws, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": ms_per_step, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": value / PAPER_MPIX_S if args.workload == "photo_rgb_30mp_u8_k17" else None,
        "dtype": dt, "data": "synthetic",
        "config": {"workload": args.workload, "channels": C, "H": H, "W": W, "k": k, "variant": args.variant,
                   "plan": plan, "l2": "flushed between timed steps (256 MB write)",
                   "parallelism": "replicas" if ws > 1 else "single GPU"},
        "roofline": roof,
        "cpu_baseline": cpu,
        "e2e": {"value": e2e_val, "unit": "Mpix/s", "h2d_bytes_per_step": int(x.numel() * x.element_size()),
                "d2h_bytes_per_step": int(y.numel() * y.element_size())},
        "gpu_launches": int(launches),
        "clocks": clocks,
        "wall_s_timed_region": t_wall,
        "step_ms": {"min": min(step_ms), "median": statistics.median(step_ms), "max": max(step_ms)},
        "extra": extra,
    }
    print(json.dumps(out))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="photo_rgb_30mp_u8_k17", choices=sorted(WORKLOADS))
    ap.add_argument("--variant", default="auto", choices=["auto", "oblivious", "data_aware"])
    ap.add_argument("--cpu-seconds", type=float, default=8.0)
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-extras", action="store_true", help="skip the batched, fwd+bwd and sweep extras")
    ap.add_argument("--ref-rows", type=int, default=8)
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
