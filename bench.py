"""Benchmark of the compress + decompress hot path on GB300.

Workload: the 3D 100x500x500 FP32 field (sum of 64 Gaussian blobs plus
k^-11/3 turbulence, seed 2) at value-range-relative bound 1e-4, 1-layer
prediction, adaptive m -- the stand-in for the paper's Hurricane fields.
A step compresses the device-resident field and decompresses the stream.

Prints one JSON line.  `value` = input bytes compressed + input bytes
decompressed per second of device time (CUDA events on the library's
stream), L2 flushed (256 MiB write) before every timed step because the
100 MB input fits in the 129 MB L2.  `e2e` repeats the step through the C
ABI with pinned host buffers (host->device and device->host copies inside
the timed region).  `--impl reference` times the CPU oracle instead.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "compress & decompress GB/s of FP32 input (fraction of HBM roofline) at rel eb 1e-4; p50/p99"
WORKLOAD = "3d-blobs-100x500x500-fp32-releb1e-4-n1-adaptive-m"


def peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""

    def __init__(self, index):
        import tempfile
        self.index = index
        self.proc = None
        # the raw samples go to $SZGB_CLOCKS_CSV when set (to keep them), else a temporary file
        self.path = os.environ.get("SZGB_CLOCKS_CSV") or os.path.join(
            tempfile.gettempdir(), "szgb_clocks_%d_%d.csv" % (os.getpid(), index))

    def start(self):
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        try:
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), "--query-gpu=" + q,
                                          "--format=csv,noheader,nounits", "-lms", "50"],
                                         stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if not self.proc:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.f.close()
        sm, mx, reasons = [], 0.0, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx = max(mx, float(parts[2]))
            except ValueError:
                continue
            for n, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(sm)}


def kernel_source_sha():
    import hashlib
    h = hashlib.sha256()
    for f in ("k_wave.cu", "szgb_internal.cuh"):
        h.update(open(os.path.join(ROOT, "paper_1706_03791_gb300", "csrc", f), "rb").read())
    return h.hexdigest()


def ncu_traffic(kernel):
    """DRAM bytes (read + write) per launch of `kernel` from the committed ncu
    summary, or None when the kernel source changed since it was captured."""
    p = os.path.join(ROOT, "profiles", "wave_kernels_3d_100x500x500.md")
    if not os.path.exists(p):
        return None
    sha, val = None, None
    for line in open(p):
        if line.startswith("kernel_source_sha256:"):
            sha = line.split(":", 1)[1].strip()
        if line.startswith("dram_bytes_per_launch_%s:" % kernel):
            val = float(line.split(":", 1)[1].strip())
    if sha != kernel_source_sha():
        return None
    return val


def host_link(torch, stream, xh, yh, reps=5):
    """Host<->device copy rates (GB/s) of the field's pinned buffers: median
    of `reps` copies each way, CUDA events on the copying stream."""
    d = torch.empty(xh.shape, dtype=xh.dtype, device=stream.device)
    out = {}
    with torch.cuda.stream(stream):
        for name, fn in (("h2d", lambda: d.copy_(xh, non_blocking=True)),
                         ("d2h", lambda: yh.copy_(d, non_blocking=True))):
            fn()
            ts = []
            for _ in range(reps):
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                fn()
                e1.record(stream)
                e1.synchronize()
                ts.append(e0.elapsed_time(e1))
            out[name] = xh.numel() * xh.element_size() / (pct(ts, 50) / 1e3) / 1e9
    del d
    return out


def pct(v, q):
    v = sorted(v)
    if not v:
        return None
    k = min(len(v) - 1, max(0, int(round(q / 100.0 * (len(v) - 1)))))
    return v[k]


def run_reference(args):
    """The CPU oracle, as it stands, on the host cores: bounded sample of the
    same workload (a 20-plane slab of the field, compress + decompress)."""
    ws, rank, _ = dist_env()
    if rank != 0:
        return
    import numpy as np
    from oracle import szo
    from synthetic import fields
    x = fields.workload_3d()
    slab = np.ascontiguousarray(x[:20])
    nbytes = slab.nbytes
    times = []
    for i in range(args.warmup + args.steps):
        t0 = time.perf_counter()
        s = szo.compress(slab, eb_rel=1e-4, n=1, m=0)
        szo.decompress(s)
        dt = time.perf_counter() - t0
        if i >= args.warmup:
            times.append(dt)
    tot = sum(times)
    val = 2 * nbytes * len(times) / tot / 1e9
    line = {"impl": "reference", "metric": METRIC, "value": val, "unit": "GB/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * tot / len(times),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic",
            "config": {"workload": WORKLOAD, "sample": "planes 0-19 of the 100x500x500 field",
                       "l2": "n/a (CPU)"},
            "cpu_baseline": dict({"value": val, "unit": "GB/s", "cores": 1, "kind": "oracle",
                                  "sample": "20x500x500 slab, compress+decompress, single thread"}, **host_cpu()),
            "e2e": {"value": val, "unit": "GB/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def host_cpu():
    """Core count and CPU model of the host the oracle runs on."""
    model = None
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.lower().startswith("model name"):
                model = line.split(":", 1)[1].strip()
                break
    except Exception:
        pass
    if not model:
        import platform
        model = platform.processor() or platform.machine()
    return {"host_cores": os.cpu_count(), "host_cpu": model}


def cpu_baseline_sample():
    import numpy as np
    from oracle import szo
    from synthetic import fields
    x = fields.workload_3d()
    slab = np.ascontiguousarray(x[:10])
    t0 = time.perf_counter()
    reps = 0
    while True:
        s = szo.compress(slab, eb_rel=1e-4, n=1, m=0)
        szo.decompress(s)
        reps += 1
        if time.perf_counter() - t0 > 12.0:
            break
    dt = time.perf_counter() - t0
    d = {"value": 2 * slab.nbytes * reps / dt / 1e9, "unit": "GB/s", "cores": 1, "kind": "oracle",
         "sample": "10x500x500 slab of the field, compress+decompress, %d reps, single thread" % reps}
    d.update(host_cpu())
    return d


def _oracle_round_trip(item):
    """One field through the oracle, compress then decompress; its bytes."""
    x, eb = item
    from oracle import szo
    s = szo.compress(x, eb_rel=eb, n=1, m=0)
    szo.decompress(s)
    return x.nbytes


def _noop(_):
    return 0


def cpu_baseline_fields(items, budget_s=8.0, workers=None):
    """The oracle, as it stands, on independent fields (the paper's parallel
    mode: processes without communication): single thread over the fields in
    order until about budget_s, then the same fields spread over a spawned
    process pool on every host core (workers started before timing).  Both
    figures count input bytes twice (compress + decompress), as the GPU line
    does."""
    import multiprocessing as mp
    t0 = time.perf_counter()
    k, nb = 0, 0
    while k < len(items) and (k == 0 or time.perf_counter() - t0 < budget_s):
        nb += _oracle_round_trip(items[k])
        k += 1
    single = 2 * nb / (time.perf_counter() - t0) / 1e9
    workers = workers or os.cpu_count() or 1
    sample = items[:max(k, min(len(items), workers))]
    with mp.get_context("spawn").Pool(workers) as pool:
        pool.map(_noop, range(workers), chunksize=1)  # start the workers and import numpy there
        t1 = time.perf_counter()
        nb_all = sum(pool.map(_oracle_round_trip, sample, chunksize=1))
        dt = time.perf_counter() - t1
    d = {"value": single, "unit": "GB/s", "cores": 1, "kind": "oracle",
         "sample": "first %d fields of the batch, compress+decompress, single thread" % k,
         "all_cores": {"value": 2 * nb_all / dt / 1e9, "unit": "GB/s", "cores": workers,
                       "sample": "first %d fields, one field per task, spawned process pool" % len(sample)}}
    d.update(host_cpu())
    return d


def batched_subset(szgb, torch, dev, stream, nfields=16, steps=5, cpu=True):
    """The batched form against the plain one-field-per-call form on the same
    GPU: climate fields 0..nfields-1 of the 79-field batch (1800 x 3600, rel
    eb 1e-4, n = 1, adaptive m), device-resident (inputs larger than L2), one
    batched pass (persistent wavefront launch, CUDA graph) against one
    compress and one decompress call per field, both timed with CUDA events
    on the library's stream (median of `steps` passes after a warm-up), every
    point checked against its bound."""
    from synthetic import fields
    peak = peaks()[0]
    xs_np = [fields.climate_batch_field(i) for i in range(nfields)]
    xs = [torch.from_numpy(x).to(dev) for x in xs_np]
    npts = sum(x.numel() for x in xs)
    nbytes = 4 * npts
    kw = dict(eb_rel=1e-4, layers=1, m=0)
    bctx = szgb.Context(dev.index or 0)
    bctx.set_stream(stream.cuda_stream)
    outs = [torch.empty(szgb.compress_bound(tuple(x.shape), **kw), dtype=torch.uint8, device=dev) for x in xs]
    ys = [torch.empty_like(x) for x in xs]
    tuned = bctx.autotune_batch(xs, kw, reps=1)

    def timed(fn):
        e0, e1, e2 = (torch.cuda.Event(enable_timing=True) for _ in range(3))
        e0.record(stream)
        r = fn(e1)
        e2.record(stream)
        e2.synchronize()
        return e0.elapsed_time(e1), e1.elapsed_time(e2), r

    def batched(e1):
        sb, st = bctx.compress_batch(xs, kw, outs)
        e1.record(stream)
        bctx.decompress_batch(sb, ys)
        return sb, st

    def per_field(e1):
        ss = [bctx.compress(x, out=o, **kw)[0] for x, o in zip(xs, outs)]
        e1.record(stream)
        for s_, y in zip(ss, ys):
            bctx.decompress(s_, out=y)
        return ss

    for _ in range(2):
        timed(batched)
    tb = [timed(batched) for _ in range(steps)]
    sb, st = tb[-1][2]
    worst = max(float((y.double() - x.double()).abs().max()) / float(t.eb_f) for x, y, t in zip(xs, ys, st))
    assert worst < 1.0, "error bound violated"
    timed(per_field)
    tp = [timed(per_field) for _ in range(max(2, steps // 2))]
    bc, bd = statistics.median(t[0] for t in tb), statistics.median(t[1] for t in tb)
    pc, pd = statistics.median(t[0] for t in tp), statistics.median(t[1] for t in tp)
    stream_bytes = sum(int(s_.numel()) for s_ in sb)
    b8 = stream_bytes / npts  # stream bytes per point
    bctx.close()
    out = {"workload": "climate fields 0-%d of the 79-field batch, 1800x3600 fp32, rel eb 1e-4, n1, adaptive m"
                       % (nfields - 1),
           "fields": nfields, "input_gb": nbytes / 1e9, "l2": "inputs larger than L2",
           "value": 2 * nbytes / ((bc + bd) / 1e3) / 1e9, "unit": "GB/s",
           "per_field_calls_value": 2 * nbytes / ((pc + pd) / 1e3) / 1e9,
           "batched_over_per_field": (pc + pd) / (bc + bd),
           "compress_gbs": {"batched": nbytes / (bc / 1e3) / 1e9, "per_field_calls": nbytes / (pc / 1e3) / 1e9},
           "decompress_gbs": {"batched": nbytes / (bd / 1e3) / 1e9, "per_field_calls": nbytes / (pd / 1e3) / 1e9},
           "compression_factor": nbytes / stream_bytes, "max_error_over_eb": worst,
           "autotuned": {"W": tuned["W"], "chunk_points": ("whole rows" if tuned["chunk"] == szgb.CHUNK_ROWS
                                                            else tuned["chunk"])},
           "roofline": {"bound": "hbm", "peak": peak, "unit": "GB/s",
                        "compress_frac": ((8.0 + b8) * npts / (bc / 1e3) / 1e9) / peak,
                        "decompress_frac": ((4.0 + b8) * npts / (bd / 1e3) / 1e9) / peak,
                        "note": "algorithmic bytes of the whole batched pass: compress 8 B/pt (range and "
                                "predict reads) + stream, decompress stream + 4 B/pt"}}
    if cpu:
        out["cpu_baseline"] = cpu_baseline_fields([(x, 1e-4) for x in xs_np], budget_s=5.0)
    return out


def run_batch_workload(args):
    """Many independent fields: the batched path (one persistent wavefront
    launch per pass, captured in a CUDA graph) against one compress and one
    decompress call per field, on the same device-resident fields."""
    import numpy as np
    import torch
    from paper_1706_03791_gb300 import build as B
    B.build()
    from paper_1706_03791_gb300 import szgb
    from paper_1706_03791_gb300.shard import my_fields
    from synthetic import fields
    ws, rank, local = dist_env()
    if ws > 1:  # fields shard across ranks; no collective on the data path
        import torch.distributed as dist
        dist.init_process_group("nccl")
    dev = torch.device("cuda", local)
    torch.cuda.set_device(local)
    t0 = time.perf_counter()
    if args.workload == "climate79":
        items = [(x, 1e-4) for x in fields.climate_batch()]
        wl = "climate-79x1800x3600-fp32-releb1e-4-n1-adaptive-m"
    else:
        items = fields.uneven_batch()
        wl = "uneven-512-fields-2d64-2048-3d32-256-fp32-releb{1e-3,1e-4,1e-5}-n1-adaptive-m"
    total_bytes = sum(x.nbytes for x, _ in items)
    mine = my_fields([x.nbytes for x, _ in items], ws, rank)
    items = [items[i] for i in mine]
    gen_s = time.perf_counter() - t0
    xs = [torch.from_numpy(x).to(dev) for x, _ in items]
    kws = [dict(eb_rel=eb, layers=args.layers, m=0) for _, eb in items]
    nbytes = sum(x.numel() * 4 for x in xs)
    npts = sum(x.numel() for x in xs)
    cpu_items = []
    if not args.no_cpu_baseline and rank == 0:  # a bounded sample, at most ~1.5 GB of fields
        for it in items:
            if cpu_items and sum(x.nbytes for x, _ in cpu_items) + it[0].nbytes > 1.5e9:
                break
            cpu_items.append(it)
    del items
    ctx = szgb.Context(local)
    stream = torch.cuda.Stream(device=dev)
    ctx.set_stream(stream.cuda_stream)
    outs = [torch.empty(szgb.compress_bound(tuple(x.shape), **kw), dtype=torch.uint8, device=dev)
            for x, kw in zip(xs, kws)]
    ys = [torch.empty_like(x) for x in xs]
    # autotune the wavefront shape of the batched pass
    t0 = time.perf_counter()
    tuned = ctx.autotune_batch(xs, kws, reps=1)
    tune_s = time.perf_counter() - t0

    def batched():
        e0, e1, e2 = (torch.cuda.Event(enable_timing=True) for _ in range(3))
        e0.record(stream)
        sb, st = ctx.compress_batch(xs, kws, outs)
        e1.record(stream)
        ctx.decompress_batch(sb, ys)
        e2.record(stream)
        e2.synchronize()
        return e0.elapsed_time(e1), e1.elapsed_time(e2), sb, st

    def per_field():
        e0, e1, e2 = (torch.cuda.Event(enable_timing=True) for _ in range(3))
        e0.record(stream)
        ss = [ctx.compress(x, out=o, **kw)[0] for x, o, kw in zip(xs, outs, kws)]
        e1.record(stream)
        for s_, y in zip(ss, ys):
            ctx.decompress(s_, out=y)
        e2.record(stream)
        e2.synchronize()
        return e0.elapsed_time(e1), e1.elapsed_time(e2), ss

    for _ in range(args.warmup):
        batched()
    torch.cuda.synchronize()
    _, _, sb, st = batched()
    # every point within its bound, on every field
    worst = 0.0
    for x, y, sti in zip(xs, ys, st):
        e = float((y.double() - x.double()).abs().max()) / float(sti.eb_f) if sti.eb_f > 0 else 0.0
        worst = max(worst, e)
    assert worst < 1.0, "error bound violated"
    stream_bytes = sum(int(s_.numel()) for s_ in sb)
    clocks = ClockSampler(local)
    clocks.start()
    time.sleep(0.1)
    if ws > 1:
        dist.barrier()
    torch.cuda.synchronize()
    tb = [batched() for _ in range(args.steps)]
    torch.cuda.synchronize()
    if ws > 1:
        dist.barrier()
    clk = clocks.stop()
    for _ in range(1):
        per_field()
    tp = [per_field() for _ in range(max(1, min(args.steps, 3)))]
    bc = statistics.median(t[0] for t in tb)
    bd = statistics.median(t[1] for t in tb)
    pc = statistics.median(t[0] for t in tp)
    pd = statistics.median(t[1] for t in tp)
    if ws > 1:  # the job's time is the slowest rank's
        t = torch.tensor([bc, bd, pc, pd], device=dev, dtype=torch.float64)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        bc, bd, pc, pd = (float(v) for v in t.tolist())
        nbytes = total_bytes
        if rank != 0:
            dist.barrier()
            return
    val = 2 * nbytes / ((bc + bd) / 1e3) / 1e9
    cpu = cpu_baseline_fields(cpu_items) if cpu_items else None  # after the GPU timing
    line = {"metric": METRIC, "value": val, "unit": "GB/s", "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": bc + bd, "higher_is_better": True,
            "scaling": "strong" if ws > 1 else "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": wl, "fields": len(xs), "points": npts, "layers": args.layers,
                       "form": "batched, one persistent wavefront launch per pass, CUDA graph",
                       "l2": "inputs (%.2f GB) larger than L2" % (nbytes / 1e9)},
            "compress_gbs": {"batched": nbytes / (bc / 1e3) / 1e9, "per_field_calls": nbytes / (pc / 1e3) / 1e9},
            "decompress_gbs": {"batched": nbytes / (bd / 1e3) / 1e9, "per_field_calls": nbytes / (pd / 1e3) / 1e9},
            "batched_over_per_field": (pc + pd) / (bc + bd),
            "compression_factor": nbytes / stream_bytes, "max_error_over_eb": worst,
            "roofline": {"bound": "hbm", "peak": peaks()[0], "unit": "GB/s",
                         "compress_frac": (6.0 * npts / (bc / 1e3) / 1e9) / peaks()[0],
                         "decompress_frac": ((stream_bytes + 4.0 * npts) / (bd / 1e3) / 1e9) / peaks()[0],
                         "note": "algorithmic bytes of the whole pass (compress 6 B/pt + range read; "
                                 "decompress stream + 4 B/pt) over the pass time"},
            "autotune": {"W": tuned["W"], "seconds": tune_s},
            "cpu_baseline": cpu,
            "clocks": clk, "generate_s": gen_s,
            "parallelism": "fields sharded over %d ranks (largest first), no collective" % ws if ws > 1 else "single"}
    print(json.dumps(line), flush=True)
    if ws > 1:
        dist.barrier()


def run_serve(args):
    """Serving: Poisson arrivals of compress and decompress requests (half
    each) of 2D fields (side log-uniform in [256, 4096]) and 3D fields (side
    log-uniform in [64, 512]), k^-3 random fields, rel eb 1e-4, admitted under
    a 100 GB device-memory budget; host buffers in and out.  Requests draw
    their field from a seeded pool of `--pool` fields generated with that
    recipe (64 by default: every request's field cannot be generated anew at
    200 requests/s).
    Reports p50/p99 latency (arrival to completion) and sustained GB/s."""
    import numpy as np
    import torch
    from paper_1706_03791_gb300 import build as B
    B.build()
    from paper_1706_03791_gb300 import szgb
    from synthetic import fields
    rng = np.random.default_rng(5)
    npool = args.pool
    t0 = time.perf_counter()
    pool = []
    for i in range(npool):
        if i % 2 == 0:
            n = int(round(np.exp(rng.uniform(np.log(256), np.log(4096)))))
            shape = (n, n)
        else:
            n = int(round(np.exp(rng.uniform(np.log(64), np.log(512)))))
            shape = (n, n, n)
        g = fields._spectral_noise(np.random.default_rng(5000 + i), shape, 3.0)
        g = ((g - g.min()) / max(g.max() - g.min(), 1e-30)).astype(np.float32)
        pool.append(torch.from_numpy(g).pin_memory())
    gen_s = time.perf_counter() - t0
    kw = dict(eb_rel=1e-4, layers=1, m=0)
    # streams of the pool for the decompress requests
    ctx = szgb.Context(0)
    streams = []
    for x in pool:
        s_, _ = ctx.compress(x.numpy(), **kw)
        streams.append(torch.from_numpy(np.ascontiguousarray(s_)).pin_memory())
    ctx.close()
    # output buffers: a few per pool entry and operation
    nbuf = 3
    cbufs = [[torch.empty(x.numel() * 4 + (1 << 16), dtype=torch.uint8).pin_memory() for _ in range(nbuf)] for x in pool]
    dbufs = [[torch.empty(x.numel(), dtype=torch.float32).pin_memory() for _ in range(nbuf)] for x in pool]
    free = {(op, i): list(range(nbuf)) for op in "cd" for i in range(npool)}
    srv = szgb.Server(0, budget=100 << 30, workers=args.workers, max_batch=32, log_path=args.serve_log)
    # warm-up: one request of each pool entry and operation
    for i in range(npool):
        t = srv.submit_compress(pool[i].numpy(), cbufs[i][0].numpy(), **kw)
        assert srv.wait(t)[0] == 0
        t = srv.submit_decompress(streams[i].numpy(), dbufs[i][0].numpy())
        assert srv.wait(t)[0] == 0
    nreq = int(args.rate * args.duration)
    arr = np.cumsum(rng.exponential(1.0 / args.rate, nreq))
    pick = rng.integers(0, npool, nreq)
    ops = rng.integers(0, 2, nreq)
    inflight = {}
    lat, done_bytes = [], 0
    clocks = ClockSampler(0)
    clocks.start()
    time.sleep(0.1)
    start = time.perf_counter()
    k = 0
    waiting = []  # arrived, no output buffer free yet
    while k < nreq or inflight or waiting:
        now = time.perf_counter() - start
        while k < nreq and arr[k] <= now:
            waiting.append(k)
            k += 1
        still = []
        for j in waiting:
            op = "c" if ops[j] == 0 else "d"
            i = int(pick[j])
            if not free[(op, i)]:
                still.append(j)
                continue
            b = free[(op, i)].pop()
            if op == "c":
                t = srv.submit_compress(pool[i].numpy(), cbufs[i][b].numpy(), **kw)
            else:
                t = srv.submit_decompress(streams[i].numpy(), dbufs[i][b].numpy())
            inflight[t] = (j, op, i, b)
        waiting = still
        for t in list(inflight):
            d, st, n = srv.poll(t)
            if d:
                j, op, i, b = inflight.pop(t)
                assert st == 0, szgb.strerror(st)
                lat.append(time.perf_counter() - start - arr[j])
                done_bytes += pool[i].numel() * 4
                free[(op, i)].append(b)
        time.sleep(0.0002)
    wall = time.perf_counter() - start
    clk = clocks.stop()
    stats = srv.stats()
    srv.close()
    lat_ms = sorted(1e3 * v for v in lat)
    mean_mb = float(np.mean([pool[int(i)].numel() * 4 for i in pick])) / 1e6
    line = {"metric": "serving: p50/p99 latency and sustained GB/s of FP32 input at rel eb 1e-4",
            "value": done_bytes / wall / 1e9, "unit": "GB/s", "n_gpus": 1, "higher_is_better": True,
            "dtype": "f32", "data": "synthetic",
            "config": {"workload": "serve-poisson%.0f-%.0fs-2d256-4096-3d64-512-fp32-releb1e-4" % (args.rate, args.duration),
                       "requests": nreq, "pool_fields": npool, "mean_request_mb": mean_mb,
                       "offered_gbs": args.rate * mean_mb / 1e3, "budget_gb": 100, "workers": args.workers,
                       "max_batch": 32, "io": "pinned host buffers in and out"},
            "latency_ms": {"p50": pct(lat_ms, 50), "p99": pct(lat_ms, 99), "max": lat_ms[-1]},
            "batches": stats["batches"], "peak_reserved_gb": stats["peak_reserved"] / 1e9,
            "wall_s": wall, "clocks": clk, "generate_s": gen_s}
    print(json.dumps(line), flush=True)


def run_rd(args):
    """Rate-distortion of the 3D field: bit-rate, compression factor and the
    quality metrics (Sec. II) for relative bounds 1e-2 .. 1e-6, with the
    compress and decompress throughput at each bound."""
    import torch
    from paper_1706_03791_gb300 import build as B
    B.build()
    from paper_1706_03791_gb300 import szgb
    from synthetic import fields
    x_np = fields.workload_3d()
    x = torch.from_numpy(x_np).cuda()
    nbytes = x_np.nbytes
    ctx = szgb.Context(0)
    y = torch.empty_like(x)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")
    pts = []
    for eb in (1e-2, 1e-3, 1e-4, 1e-5, 1e-6):
        kw = dict(eb_rel=eb, layers=args.layers, m=0)
        sbuf = torch.empty(szgb.compress_bound(x_np.shape, **kw), dtype=torch.uint8, device="cuda")
        tc, td = [], []
        for i in range(3 + 5):
            flush.fill_(1)
            e0, e1, e2 = (torch.cuda.Event(enable_timing=True) for _ in range(3))
            e0.record()
            s, st = ctx.compress(x, out=sbuf, **kw)
            e1.record()
            ctx.decompress(s, out=y)
            e2.record()
            e2.synchronize()
            if i >= 3:
                tc.append(e0.elapsed_time(e1))
                td.append(e1.elapsed_time(e2))
        q = ctx.quality(x, y)
        assert q["max_abs_err"] < float(st.eb_f), "error bound violated"
        n = x_np.size
        pts.append({"eb_rel": eb, "m": int(st.m), "bit_rate": s.numel() * 8.0 / n,
                    "compression_factor": nbytes / s.numel(), "psnr_db": q["psnr"], "nrmse": q["nrmse"],
                    "pearson": q["pearson"], "max_error_over_eb": q["max_abs_err"] / float(st.eb_f),
                    "unpredictable_fraction": int(st.n_unpred) / n,
                    "compress_gbs": nbytes / (sorted(tc)[len(tc) // 2] / 1e3) / 1e9,
                    "decompress_gbs": nbytes / (sorted(td)[len(td) // 2] / 1e3) / 1e9})
    ref = next(p for p in pts if p["eb_rel"] == 1e-4)
    print(json.dumps({"metric": "rate-distortion of the 3D 100x500x500 field over rel eb (bits/value at 1e-4)",
                      "value": ref["bit_rate"], "unit": "bits/value", "higher_is_better": False, "n_gpus": 1,
                      "dtype": "f32", "data": "synthetic",
                      "config": {"workload": "rd-3d-blobs-100x500x500-fp32-n%d-adaptive-m" % args.layers},
                      "points": pts}))


def run_layers(args):
    """Best-layer report (Sec. III, Table 2) on the device: R_PH^orig and
    R_PH^decomp for n = 1..4 on the 3D field, a 2D climate-like field and a
    smooth 2D field, R_PH^decomp from the compressor's recorded values."""
    import torch
    from paper_1706_03791_gb300 import build as B
    B.build()
    from paper_1706_03791_gb300 import szgb
    from synthetic import fields
    ctx = szgb.Context(0)
    cases = [("3d-blobs-100x500x500", fields.workload_3d()),
             ("2d-climate-1800x3600", fields.climate2d(7)),
             ("2d-k6-smooth-1024x1024", fields.grf2d(1024, 1024, seed=3, slope=6.0, noise=0.0))]
    rows = []
    for name, x_np in cases:
        x = torch.from_numpy(x_np).cuda()
        for eb in (1e-3, 1e-4):
            for n in (1, 2, 3, 4):
                row = {"field": name, "eb_rel": eb, "n": n}
                r = ctx.hit_rates(x, n, eb_rel=eb)  # 3D n = 3, 4 compress on the hyperplane kernels
                row.update(R_orig=r["R_orig"], R_decomp=r["R_decomp"], m=r["m"])
                rows.append(row)
        for r in rows:
            if r["field"] == name:
                print("%-24s eb %-6g n=%d  R_orig %7.3f%%  R_decomp %s  m %s" % (
                    name, r["eb_rel"], r["n"], 100 * r["R_orig"],
                    "%7.3f%%" % (100 * r["R_decomp"]),
                    r["m"]), file=sys.stderr)
    print(json.dumps({"metric": "prediction hitting rate by layer count (Sec. III, Table 2)", "value": None,
                      "unit": "fraction", "n_gpus": 1, "dtype": "f32", "data": "synthetic",
                      "config": {"workload": "best-layer hit rates, rel eb 1e-3 and 1e-4"}, "rows": rows}))


def run_hyper(args):
    """The hyperplane paths: the 3D field at n = 3, 4 and a 4D field at
    n = 1, 2, compress + decompress timed with CUDA events (L2 flushed before
    each step), every point checked against its bound."""
    import numpy as np
    import torch
    from paper_1706_03791_gb300 import build as B
    B.build()
    from paper_1706_03791_gb300 import szgb
    from synthetic import fields
    ctx = szgb.Context(0)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")
    g = np.meshgrid(*[np.linspace(0, 1, n) for n in (16, 64, 64, 64)], indexing="ij")
    x4 = (np.sin(3 * g[0] + 2 * g[1]) * np.cos(2 * g[2] - g[3]) + 0.5 * g[3] ** 2).astype(np.float32)
    cases = [("3d-blobs-100x500x500", fields.workload_3d(), (3, 4)), ("4d-smooth-16x64x64x64", x4, (1, 2))]
    rows = []
    for name, x_np, layer_set in cases:
        x = torch.from_numpy(x_np).cuda()
        nbytes = x_np.nbytes
        for n in layer_set:
            kw = dict(eb_rel=1e-4, layers=n, m=0)
            sbuf = torch.empty(szgb.compress_bound(x_np.shape, **kw), dtype=torch.uint8, device="cuda")
            y = torch.empty_like(x)
            tc, td = [], []
            for i in range(args.warmup + args.steps):
                flush.fill_(1)
                e0, e1, e2 = (torch.cuda.Event(enable_timing=True) for _ in range(3))
                e0.record()
                s_, st = ctx.compress(x, out=sbuf, **kw)
                e1.record()
                ctx.decompress(s_, out=y)
                e2.record()
                e2.synchronize()
                if i >= args.warmup:
                    tc.append(e0.elapsed_time(e1))
                    td.append(e1.elapsed_time(e2))
            q = ctx.quality(x.reshape(-1), y.reshape(-1))
            assert q["max_abs_err"] < float(st.eb_f), "error bound violated"
            c_ms, d_ms = statistics.median(tc), statistics.median(td)
            rows.append({"field": name, "layers": n, "m": int(st.m), "bit_rate": s_.numel() * 8.0 / x_np.size,
                         "compress_gbs": nbytes / (c_ms / 1e3) / 1e9, "decompress_gbs": nbytes / (d_ms / 1e3) / 1e9,
                         "psnr_db": q["psnr"]})
            print(rows[-1], file=sys.stderr)
    print(json.dumps({"metric": "hyperplane paths: compress and decompress GB/s of FP32 input", "value": None,
                      "unit": "GB/s", "n_gpus": 1, "steps": args.steps, "warmup": args.warmup, "dtype": "f32",
                      "data": "synthetic", "config": {"workload": "3D n = 3, 4 and 4D n = 1, 2, rel eb 1e-4"},
                      "rows": rows}))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--layers", type=int, default=1)
    ap.add_argument("--ebrel", type=float, default=1e-4)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-tune", action="store_true", help="skip the autotuner (default shape, whole-row chunks)")
    ap.add_argument("--no-batched", action="store_true", help="skip the batched sub-measurement of the default run")
    ap.add_argument("--variant", default="exact", choices=["exact", "lattice"],
                    help="exact: the paper's method (default); lattice: the separately labelled "
                         "fully parallel lattice variant, reported beside it")
    ap.add_argument("--rate", type=float, default=200.0, help="serve: mean arrivals per second")
    ap.add_argument("--duration", type=float, default=30.0, help="serve: seconds of arrivals")
    ap.add_argument("--pool", type=int, default=64, help="serve: fields drawn from the recipe that requests pick from")
    ap.add_argument("--workers", type=int, default=3, help="serve: server worker threads")
    ap.add_argument("--serve-log", default=None, help="serve: append one JSON line per completed request here")
    ap.add_argument("--workload", default="3d", choices=["3d", "climate79", "uneven512", "serve", "rd", "layers", "hyper"],
                    help="3d: the single 100x500x500 field (default); climate79 / uneven512: "
                         "batched many-field workloads, batched+graph vs one field per call; "
                         "rd: rate-distortion sweep of the 3d field over the relative bound; "
                         "layers: prediction hitting rate by layer count (Table 2); "
                         "hyper: the hyperplane paths (3D n = 3, 4; 4D)")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        return run_reference(args)
    if args.workload == "serve":
        return run_serve(args)
    if args.workload == "rd":
        return run_rd(args)
    if args.workload == "layers":
        return run_layers(args)
    if args.workload == "hyper":
        return run_hyper(args)
    if args.workload != "3d":
        return run_batch_workload(args)

    import numpy as np
    import torch
    ws, rank, local = dist_env()
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    from paper_1706_03791_gb300 import build as B
    if rank == 0 or ws == 1:
        B.build()
    if ws > 1:
        dist.barrier()
    from paper_1706_03791_gb300 import szgb
    from synthetic import fields

    x_np = fields.workload_3d()
    N = x_np.size
    nbytes = x_np.nbytes
    x = torch.from_numpy(x_np).to(dev)
    ctx = szgb.Context(local)
    stream = torch.cuda.Stream(device=dev)
    ctx.set_stream(stream.cuda_stream)
    kw = dict(eb_rel=args.ebrel, layers=args.layers, m=0, variant=1 if args.variant == "lattice" else 0)
    # the wavefront shape and the Huffman chunk length are picked by the
    # autotuner before the timed region (chunk_points = 0 takes its choice)
    tuned = ctx.autotune(x, reps=2, **kw) if args.variant == "exact" and not args.no_tune else None
    bound = szgb.compress_bound(x_np.shape, **kw)
    sbuf = torch.empty(bound, dtype=torch.uint8, device=dev)
    y = torch.empty_like(x)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)

    def step(prof=False):
        with torch.cuda.stream(stream):
            flush.fill_(1)
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e2 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            s, st = ctx.compress(x, out=sbuf, **kw)
            e1.record(stream)
            ctx.decompress(s, out=y)
            e2.record(stream)
        return e0, e1, e2, s, st

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    # correctness guard on the timed configuration: every point within eb
    s0, st0 = ctx.compress(x, out=sbuf, **kw)
    yv = ctx.decompress(s0, out=y)
    torch.cuda.synchronize()
    maxerr = float((yv.double() - x.double()).abs().max())
    assert maxerr < st0.eb_f, "error bound violated"
    stream_bytes = int(s0.numel())
    qual = ctx.quality(x, yv)  # Sec. II, Metrics 1-3, computed on the device

    # per-kernel (phase) device times, CUDA events on the library's stream,
    # over a separate profiled pass of the same steps
    ctx.set_profiling(True)
    ctx.phase_times(reset=True)
    for _ in range(min(args.steps, 20)):
        step()
    torch.cuda.synchronize()
    ctx.set_profiling(False)
    phases = ctx.phase_times(reset=True)

    # headline: exactly K steps, barrier + synchronize on both sides, clocks
    # sampled while they run
    clocks = ClockSampler(local)
    clocks.start()
    time.sleep(0.1)
    tc2, td2 = [], []
    evs = []
    if ws > 1:
        dist.barrier()
    torch.cuda.synchronize()
    t_wall0 = time.perf_counter()
    for _ in range(args.steps):
        e0, e1, e2, s, st = step()
        evs.append((e0, e1, e2))
    torch.cuda.synchronize()
    if ws > 1:
        dist.barrier()
    t_wall = time.perf_counter() - t_wall0
    clk = clocks.stop()
    for e0, e1, e2 in evs:
        tc2.append(e0.elapsed_time(e1))
        td2.append(e1.elapsed_time(e2))
    tot_ms = sum(tc2) + sum(td2)
    if ws > 1:
        t = torch.tensor([tot_ms], device=dev, dtype=torch.float64)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        tot_ms = float(t.item())
    ms_step = tot_ms / args.steps
    value = ws * 2 * nbytes * args.steps / (tot_ms / 1e3) / 1e9
    comp_gbs = [nbytes / (t / 1e3) / 1e9 for t in tc2]
    dec_gbs = [nbytes / (t / 1e3) / 1e9 for t in td2]

    # end to end through the C ABI with pinned host buffers
    xh = torch.from_numpy(x_np).pin_memory()
    sh = torch.empty(bound, dtype=torch.uint8).pin_memory()
    yh = torch.empty(x_np.shape, dtype=torch.float32).pin_memory()
    e2e_t = []
    for i in range(args.warmup + args.steps):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        n, _ = ctx.compress_host_ptr(xh.data_ptr(), x_np.shape, sh.data_ptr(), bound, **kw)
        rc = ctx.decompress_ptr(sh.data_ptr(), n, False, yh.data_ptr(), N, False)
        assert rc == 0
        dt = time.perf_counter() - t0
        if i >= args.warmup:
            e2e_t.append(dt)
    e2e_val = ws * 2 * nbytes * len(e2e_t) / sum(e2e_t) / 1e9
    link = host_link(torch, stream, xh, yh)
    # the serial bound of one end-to-end compress + decompress: each call
    # returns with its output on the host, so its copies cannot overlap the
    # kernels (the field in, the stream out; the stream in, the field out)
    t_serial = (nbytes / link["h2d"] + stream_bytes / link["d2h"] + stream_bytes / link["h2d"]
                + nbytes / link["d2h"]) / 1e9 + (pct(tc2, 50) + pct(td2, 50)) / 1e3
    e2e_bound = 2 * nbytes / t_serial / 1e9

    # roofline of the dominant kernel: live CUDA-event phase times
    peak, peak_kind = peaks()
    bits_pp = stream_bytes * 8.0 / N
    # compress: x read + codes written; decompress: stream read + values written
    # (the lattice variant's phases carry the same names: its parallel code
    # and reconstruction passes)
    algo = {"wave_compress": 4.0 + 2.0, "wave_decompress": bits_pp / 8.0 + 4.0}
    dom = max(algo, key=lambda k: phases.get(k, (0, 0))[0])
    ms_dom, calls_dom = phases[dom]
    achieved = algo[dom] * N / (ms_dom / calls_dom / 1e3) / 1e9
    roof = {"bound": "hbm", "kernel": dom, "achieved": achieved, "peak": peak, "peak_kind": peak_kind,
            "unit": "GB/s", "frac": achieved / peak, "traffic": ncu_traffic(dom),
            "algorithmic_bytes_per_point": algo[dom]}
    phase_ms = {k: v[0] / max(v[1], 1) for k, v in phases.items() if v[1]}

    if rank != 0:
        if ws > 1:
            dist.barrier()
        return
    cpu = None if args.no_cpu_baseline else cpu_baseline_sample()
    batched = None
    if not args.no_batched and args.variant == "exact" and ws == 1:
        batched = batched_subset(szgb, torch, dev, stream, cpu=not args.no_cpu_baseline)
    line = {
        "metric": METRIC, "value": value, "unit": "GB/s", "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": WORKLOAD + ("" if args.variant == "exact" else "-LATTICE-VARIANT"),
                   "variant": args.variant, "shape": list(x_np.shape), "eb_rel": args.ebrel,
                   "layers": args.layers, "m": "adaptive", "m_chosen": int(st0.m),
                   "autotuned": ({"W": tuned["W"], "chunk_points": ("whole rows" if tuned["chunk"] == szgb.CHUNK_ROWS
                                                                    else tuned["chunk"])} if tuned else None),
                   "l2": "flushed (256 MiB write) before every step",
                   "parallelism": "replicas" if ws > 1 else "single"},
        "compress_gbs": {"p50": pct(comp_gbs, 50), "p99": pct(comp_gbs, 1)},
        "decompress_gbs": {"p50": pct(dec_gbs, 50), "p99": pct(dec_gbs, 1)},
        "compression_factor": nbytes / stream_bytes, "bits_per_value": bits_pp,
        "n_unpred": int(st0.n_unpred), "max_error_over_eb": maxerr / float(st0.eb_f),
        "quality": {"psnr_db": qual["psnr"], "nrmse": qual["nrmse"], "rmse": qual["rmse"],
                    "pearson": qual["pearson"]},
        "phase_ms": phase_ms,
        "roofline": roof,
        "cpu_baseline": cpu,
        "batched": batched,
        "e2e": {"value": e2e_val, "unit": "GB/s", "h2d_bytes_per_step": nbytes + stream_bytes,
                "d2h_bytes_per_step": stream_bytes + nbytes,
                "host_link_gbs": {"h2d": link["h2d"], "d2h": link["d2h"]},
                "serial_bound_gbs": e2e_bound},
        # kernels of this library per step: compress 10 (range, adapt, wavefront,
        # histogram, codebook, chunk bits, 2 scan, metadata, encode), decompress 5
        # (2 scan, tables, chunk decode, wavefront); the lattice variant compress
        # 11 (range, adapt, 2 lattice passes, then the same 7), decompress 5 +
        # 3 axis scans per layer (2 scan, tables, chunk decode, finish)
        "gpu_launches": (15 if args.variant == "exact" else 16 + 3 * args.layers) * args.steps,
        "clocks": clk,
        "wall_s_timed": t_wall,
    }
    print(json.dumps(line), flush=True)
    if ws > 1:
        dist.barrier()


if __name__ == "__main__":
    main()
