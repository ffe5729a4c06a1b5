"""FSZ compress/decompress throughput on GB300.

Workload: the 512^3 float32 Gaussian random field with P(k) ~ k^-3 and its zero-slab
+280 variant, each at REL 1e-2, 1e-3 and 1e-4 (six field/bound pairs). One step runs
the whole hot path on all six: value-range pass + single-pass compression of each,
then decompression of each, through the library's C ABI. Inputs (512 MiB each) are
larger than L2, and each stream is read back only after at least 2.5 GB of other
traffic, so no timed kernel reads its input from L2.

value  = input bytes of both directions (4n per compression + 4n per decompression)
         / step time, summed over ranks (replicas, one per GPU).
e2e    = the same metric through the same calls with pinned host buffers: inputs
         copied in, streams copied out and back in, reconstructions copied out.

python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]
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

RELS = (1e-2, 1e-3, 1e-4)
SHAPE = (512, 512, 512)
NOMINAL_HBM_GBS = 8000.0
METRIC = "comp/decomp GB/s & % HBM roofline at oracle-exact CR; batched vs per-field"
WORKLOAD = ("512^3 float32 k^-3 GRF + zero-slab/+280 variant, REL {1e-2,1e-3,1e-4}: "
            "value-range pass + compress, then decompress, of all six")


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f), "measured"
    except OSError:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0}, "fallback"


class ClockSampler:
    """nvidia-smi clocks and throttle reasons, sampled every 50 ms while running."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.path = os.path.join("/tmp", f"fsz_clocks_{os.getpid()}.csv")

    def __enter__(self):
        try:
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "50"], stdout=self.fh,
                stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None
        return self

    def __exit__(self, *exc):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
            self.fh.close()

    def summary(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        rows = []
        with open(self.path) as f:
            for line in f:
                parts = [p.strip() for p in line.split(",")]
                if len(parts) >= 9:
                    rows.append(parts)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        smax = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for r in rows for k in range(4) if r[5 + k].lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None, "reasons": reasons,
                "samples": len(rows)}


def dist_setup(n_gpus: int):
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("gloo")
    return world, rank, local


def all_max(x: float, world: int) -> float:
    if world == 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([x], dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def barrier(world: int):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def job_throughput(world: int, bytes_per_rank: float, ms_local: float) -> tuple[float, float]:
    """Whole-job GB/s: every rank processes `bytes_per_rank` per step (weak scaling) and the
    job takes as long as its slowest rank. Returns (GB/s, max ms over ranks)."""
    ms = all_max(ms_local, world)
    return world * bytes_per_rank / (ms * 1e-3) / 1e9, ms


CPU_SAMPLE_SHAPE = (384, 512, 512)  # 3 x 2^25 elements per field: about 10-30 s of oracle work


def cpu_sample_fields():
    """Host copies of the workload's recipe at 2^26 elements per field (numpy, seed 1)."""
    from paper_2607_15413_gb300 import inputs
    g = inputs.grf(CPU_SAMPLE_SHAPE, seed=1)
    z = inputs.zero_slabs(CPU_SAMPLE_SHAPE, seed=1, base=g)
    return [g.ravel(), z.ravel()]


def cpu_baseline_run(fields, elems=None):
    """The oracle, single-threaded on the host, compressing and decompressing the first
    `elems` elements of each sample field at each of the three bounds."""
    import oracle
    oracle.build()
    # pinned to one core while timed (the first core this process may use)
    allowed = os.sched_getaffinity(0) if hasattr(os, "sched_getaffinity") else None
    if allowed:
        os.sched_setaffinity(0, {min(allowed)})
    try:
        nbytes = 0
        t0 = time.perf_counter()
        for f in fields:
            x = f if elems is None else f[:elems]
            for rel in RELS:
                s = oracle.compress(x, rel, oracle.REL)
                y = oracle.decompress(s)
                assert y.size == x.size
                nbytes += 2 * x.nbytes
        dt = time.perf_counter() - t0
    finally:
        if allowed:
            os.sched_setaffinity(0, allowed)
    n = fields[0].size if elems is None else elems
    return {"value": nbytes / dt / 1e9, "unit": "GB/s", "cores": 1, "kind": "oracle",
            "sample": f"first {n} elements of both fields (k^-3 GRF and its zero-slab/+280 "
                      f"variant, same recipe at 384x512x512) at REL 1e-2/1e-3/1e-4, "
                      f"compress + decompress, 1 host core (pinned)",
            "seconds": dt}


def host_cpu_model() -> str:
    """The host CPU's model name (lscpu / /proc/cpuinfo), or the machine type."""
    import platform
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.strip().startswith("Model name:"):
                return line.split(":", 1)[1].strip()
    except (OSError, subprocess.SubprocessError):
        pass
    try:
        with open("/proc/cpuinfo") as f:
            for line in f:
                if line.lower().startswith(("model name", "cpu model")):
                    return line.split(":", 1)[1].strip()
    except OSError:
        pass
    return platform.machine()


def cpu_all_core_run(fields, elems=None):
    """The oracle's functions on every host core (element and tile ranges, one thread each,
    a serial scan to place the ranges; the same streams as the single-threaded oracle):
    compressing and decompressing the same sample as cpu_baseline_run."""
    import oracle
    oracle.build()
    cores = os.cpu_count() or 1
    nbytes = 0
    t0 = time.perf_counter()
    for f in fields:
        x = f if elems is None else f[:elems]
        for rel in RELS:
            s = oracle.mt_compress(x, rel, oracle.REL, nthreads=cores)
            y = oracle.mt_decompress(s, nthreads=cores)
            assert y.size == x.size
            nbytes += 2 * x.nbytes
    dt = time.perf_counter() - t0
    return {"value": nbytes / dt / 1e9, "unit": "GB/s", "cores": cores, "seconds": dt,
            "cpu_model": host_cpu_model(),
            "how": "oracle tile functions over contiguous tile ranges, one thread per core, "
                   "serial scan of the ranges' byte counts"}


def run_reference(args, world, rank):
    """The reference arm: the CPU oracle as it stands, one host core. The 2^26-element
    sample is split across the warm-up and timed steps so any --steps/--warmup stays
    bounded (about 10-30 s of oracle work in all)."""
    if rank != 0:
        return 0
    fields = cpu_sample_fields()
    per = max(1 << 16, (fields[0].size // (args.steps + args.warmup)) // 256 * 256)
    vals, secs = [], []
    last = None
    for i in range(args.warmup + args.steps):
        k = i % max(1, fields[0].size // per)
        part = [f[k * per:(k + 1) * per] for f in fields]
        last = cpu_baseline_run(part)
        if i >= args.warmup:
            vals.append(last["value"])
            secs.append(last["seconds"])
    value = len(vals) / sum(1.0 / v for v in vals)  # throughput over the timed steps
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "GB/s",
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1000.0 * statistics.mean(secs), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": WORKLOAD + f" (host sample: {per} elements per field per step)",
                       "parallelism": "single host core"},
            "cpu_baseline": {"kind": "oracle", "cores": 1, "sample": last["sample"], "value": value,
                             "unit": "GB/s"},
            "e2e": {"value": value, "unit": "GB/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))
    return 0


def run_batched(fsz, inputs, dev, reps: int = 3):
    """Batched workload: 512 fields (seed 3) of log-uniform size 64 KiB - 64 MiB, mixed
    classes and REL bounds, compressed and decompressed in one batched call (a CUDA graph,
    autotuned schedule) vs one call per field on the same stream, same schedule."""
    import torch
    from paper_2607_15413_gb300 import tune
    L = fsz.lib()
    sp = torch.cuda.current_stream(dev).cuda_stream
    specs = inputs.field_mix_specs(512, seed=3)
    fields = [(inputs.make_field(spec, device=str(dev)).contiguous(), spec["dims"], fsz.EB_REL,
               spec["rel"]) for spec in specs]
    torch.cuda.empty_cache()
    nbytes_in = sum(4 * f.numel() for f, *_ in fields)
    cb = fsz.CompressBatch(fields, dev)
    assert cb.run() == fsz.OK and cb.status()[0] == fsz.OK
    sizes = cb.sizes.cpu().tolist()
    streams = [cb.stream(i, sizes) for i in range(len(fields))]
    db = fsz.DecompressBatch(streams, [f.numel() for f, *_ in fields], dev)
    tuned = tune.tune(cb, db, reps=2)
    tune.apply(tuned["best"])
    ws1_bytes = fsz.fsz_workspace_bytes(max(f.numel() for f, *_ in fields))
    ws1 = torch.empty(ws1_bytes, dtype=torch.uint8, device=dev)
    dims = [fsz.make_dims(d) for _, d, *_ in fields]

    def timed(fn):
        ts = []
        for _ in range(reps + 1):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            fn()
            e1.record()
            torch.cuda.synchronize(dev)
            ts.append(e0.elapsed_time(e1))
        return statistics.median(ts[1:])

    def per_field_compress():
        for i, (x, _, mode, eb) in enumerate(fields):
            st = L.fsz_compress(x.data_ptr(), dims[i], mode, eb, cb.arena.data_ptr() + cb.offsets[i],
                                cb.caps[i], cb.sizes.data_ptr() + 8 * i, ws1.data_ptr(), ws1_bytes, sp)
            if st:
                raise fsz.FszError(st, "per-field compress")

    def per_field_decompress():
        for i, s_i in enumerate(streams):
            st = L.fsz_decompress(s_i.data_ptr(), s_i.numel(), db.arena.data_ptr() + 4 * db.offsets[i],
                                  db.caps[i], ws1.data_ptr(), ws1_bytes, sp)
            if st:
                raise fsz.FszError(st, "per-field decompress")

    t_pf_c = timed(per_field_compress)
    pf_arena = cb.arena.clone()
    t_b_c = timed(lambda: cb.launch_graph())
    exact = all(torch.equal(pf_arena[cb.offsets[i]:cb.offsets[i] + sizes[i]], streams[i])
                for i in range(len(fields)))
    t_pf_d = timed(per_field_decompress)
    pf_out = db.arena.clone()
    t_b_d = timed(lambda: db.launch_graph())
    exact = exact and torch.equal(pf_out, db.arena) and cb.status()[0] == fsz.OK and db.status()[0] == fsz.OK
    tune.apply(None)
    comp_bytes = sum(sizes)
    out = {"workload": "512 fields, seed 3: log-uniform 64 KiB-64 MiB, 1-3-D, 40% k^-3 GRF / "
                       "40% particle-like / 20% zero-slab, REL in {1e-2,1e-3,1e-4}",
           "nfields": len(fields), "input_bytes": nbytes_in, "stream_bytes": comp_bytes,
           "compress": {"batched_gbs": nbytes_in / t_b_c / 1e6, "per_field_gbs": nbytes_in / t_pf_c / 1e6,
                        "batched_ms": t_b_c, "per_field_ms": t_pf_c, "ratio": t_pf_c / t_b_c},
           "decompress": {"batched_gbs": nbytes_in / t_b_d / 1e6, "per_field_gbs": nbytes_in / t_pf_d / 1e6,
                          "batched_ms": t_b_d, "per_field_ms": t_pf_d, "ratio": t_pf_d / t_b_d},
           "schedule": tuned["best"], "tuning_ms": {"compress": tuned["compress"],
                                                    "decompress": tuned["decompress"]},
           "bit_exact_vs_per_field": bool(exact),
           "notes": "batched = value-range pass + compression of all fields in one graph launch; "
                    "per-field = fsz_compress / fsz_decompress once per field on one stream"}
    del cb, db, fields, streams, pf_arena, pf_out
    torch.cuda.empty_cache()
    return out


def run_serving(fsz, inputs, dev, nreq: int = 20000, seed: int = 4, linger_us: int = 200):
    """Serving workload through the library's native server: requests of log-uniform
    16 KiB-256 MiB cut from a device-resident pool of the batched mix's classes, 60 %
    compress / 40 % decompress of one of 64 streams compressed beforehand, REL from
    {1e-2,1e-3,1e-4}, 40 GB admission budget, 4 stream slots, batches of up to 32. First the
    closed loop (every request arrives at once: the peak), then Poisson arrivals at
    25/50/75/100 % of that peak. Each level is handed to the server as one trace (each
    request with its arrival time; the server admits it then), so no client thread sits on
    the clock. p50/p99 latency from the arrival to completion, sustained GB/s over the span
    from the first arrival to the last completion. The baseline is the closed loop's first
    2000 requests issued as one library call each (fsz_compress / fsz_decompress) on one
    stream."""
    import math
    import random

    import numpy as np
    import torch

    from paper_2607_15413_gb300 import serve
    pool = inputs.serving_pool(seed=seed, device=str(dev))
    numels = [p.numel() for p in pool]
    torch.cuda.empty_cache()
    rng = random.Random(seed)
    srv = serve.Server(budget_bytes=40 << 30, n_slots=4, max_batch=32, max_batch_elems=4 << 30,
                       linger_s=linger_us * 1e-6, futures=False)
    L = fsz.lib()
    next_id = [1]

    def trace(count, sources, dec_share=0.4):
        """A request table: compress requests of pool windows, and with `dec_share`
        decompress requests of one of `sources` (stream pointer, bytes, n)."""
        t = np.zeros(count, dtype=fsz.REQUEST_NP)
        t["id"] = np.arange(next_id[0], next_id[0] + count, dtype=np.uint64)
        next_id[0] += count
        rows = []
        for row in inputs.serving_trace(rng, numels, count, len(sources or ()), dec_share):
            if row[0] == "decompress":
                sp, sb, sn = sources[row[1]]
                rows.append((fsz.REQ_DECOMPRESS, 0, 0, 0, 0.0, sp, sb, sn))
            else:
                _, k, off, n, rel = row
                rows.append((fsz.REQ_COMPRESS, 1, 1, n, rel, pool[k].data_ptr() + 4 * off, 0, 0))
        cols = list(zip(*rows))
        for name, col in zip(("kind", "mode", "ndim", "d0", "eb", "d_in", "in_bytes", "n"), cols):
            t[name] = col
        return t

    def elems(t):
        return np.where(t["kind"] == fsz.REQ_COMPRESS, t["d0"], t["n"]).astype(np.int64)

    cbuf = np.zeros(4096, dtype=fsz.COMPLETION_NP)

    def run(t, rate=None, keep=False):
        """Submits table `t` (closed loop, or Poisson arrivals at `rate` requests/s) and
        takes every completion; releases the outputs unless `keep`."""
        count = len(t)
        t0 = time.monotonic_ns() + 2_000_000
        if rate is None:
            t["arrival_ns"] = t0
        else:
            gaps = np.array([rng.expovariate(rate) for _ in range(count)]) * 1e9
            t["arrival_ns"] = t0 + np.cumsum(gaps).astype(np.uint64)
        st0 = srv.stats()
        code = L.fsz_server_submit_many(srv._h, t.ctypes.data, count)
        if code:
            raise fsz.FszError(code, "fsz_server_submit_many")
        got = []
        while sum(len(g) for g in got) < count:
            k = L.fsz_server_poll(srv._h, cbuf.ctypes.data, len(cbuf), 2_000_000)
            if k:
                c = cbuf[:k].copy()
                got.append(c)
                ok = c["id"][c["status"] != fsz.ERR_REJECTED]
                if not keep and len(ok):
                    L.fsz_server_release_many(srv._h, np.ascontiguousarray(ok).ctypes.data, len(ok), None)
        t_end = time.monotonic_ns()
        st1 = srv.stats()
        c = np.concatenate(got)
        ok = c["status"] == 0
        lat = c["latency_ns"][ok] * 1e-6
        nbytes = int(4 * elems(t).sum())
        wall = (t_end - t0) * 1e-9
        return c, {"gbs": nbytes / wall / 1e9,
                   "p50_ms": float(np.percentile(lat, 50)) if len(lat) else float("nan"),
                   "p99_ms": float(np.percentile(lat, 99)) if len(lat) else float("nan"),
                   "requests": count, "refused": int((~ok).sum()), "bytes": nbytes,
                   "wall_s": wall, "batches": st1["batches"] - st0["batches"],
                   "mean_batch": count / max(1, st1["batches"] - st0["batches"]),
                   "max_inflight": st1["max_inflight"],
                   "admitted_while_busy": st1["admitted_while_busy"] - st0["admitted_while_busy"]}

    # 64 streams for the decompress requests, held for the whole run
    src_t = trace(64, None)
    src_c, _ = run(src_t, keep=True)
    by_id = {int(r["id"]): r for r in src_c}
    sources = [(int(by_id[int(i)]["d_out"]), int(by_id[int(i)]["out_bytes"]), int(n))
               for i, n in zip(src_t["id"], src_t["d0"]) if by_id[int(i)]["status"] == 0]
    run(trace(max(64, nreq // 10), sources))      # warm-up (pool, workspaces, clocks)
    t_closed = trace(nreq, sources)
    _, closed = run(t_closed)
    # the closed loop's first requests, one library call each, one stream (the baseline)
    rec = t_closed[:min(nreq, 2000)]
    sp = torch.cuda.current_stream(dev).cuda_stream
    nmax = int(elems(rec).max())
    ws_b = fsz.fsz_workspace_bytes(nmax)
    ws = torch.empty(ws_b, dtype=torch.uint8, device=dev)
    cap = fsz.fsz_compress_bound(nmax)
    out = torch.empty(cap, dtype=torch.uint8, device=dev)
    dout = torch.empty(nmax + 4, dtype=torch.float32, device=dev)
    nb = torch.zeros(1, dtype=torch.int64, device=dev)
    torch.cuda.synchronize(dev)
    t0 = time.perf_counter()
    for r in rec:
        if r["kind"] == fsz.REQ_COMPRESS:
            L.fsz_compress(int(r["d_in"]), fsz.make_dims((int(r["d0"]),)), 1, float(r["eb"]),
                           out.data_ptr(), cap, nb.data_ptr(), ws.data_ptr(), ws_b, sp)
        else:
            L.fsz_decompress(int(r["d_in"]), int(r["in_bytes"]), dout.data_ptr(), int(r["n"]),
                             ws.data_ptr(), ws_b, sp)
    torch.cuda.synchronize(dev)
    per_req_gbs = 4 * int(elems(rec).sum()) / (time.perf_counter() - t0) / 1e9
    n_dec = int((rec["kind"] == fsz.REQ_DECOMPRESS).sum())
    del out, dout, ws
    mean_bytes = closed["bytes"] / closed["requests"]
    levels = []
    for load in (0.25, 0.5, 0.75, 1.0):
        rate = load * closed["gbs"] * 1e9 / mean_bytes
        _, r = run(trace(nreq, sources), rate=rate)
        r["load"] = load
        r["offered_gbs"] = load * closed["gbs"]
        levels.append(r)
    ids = np.ascontiguousarray(src_c["id"][src_c["status"] != fsz.ERR_REJECTED])
    L.fsz_server_release_many(srv._h, ids.ctypes.data, len(ids), None)
    srv.close()
    del pool
    torch.cuda.empty_cache()
    return {"workload": f"{nreq} requests per level, seed {seed}: log-uniform 16 KiB-256 MiB windows "
                        "of a device pool (k^-3 GRF, particle-like, zero-slab), 60% compress / 40% "
                        "decompress of one of 64 earlier streams, REL in {1e-2,1e-3,1e-4}, 40 GB "
                        f"budget, 4 streams, batches of up to 32, linger {linger_us} us while busy; "
                        "native scheduler (fsz_server_*), each level replayed as a trace",
            "closed_loop": closed, "sample_decompress_share": n_dec / max(1, len(rec)),
            "per_request_gbs": per_req_gbs, "per_request_sample": len(rec),
            "closed_loop_vs_per_request": closed["gbs"] / per_req_gbs, "loads": levels}


def run_ablation(fsz, fields, rels, dev, shape):
    """Sec. 6.4 (Table 7) and Sec. 6.3 on the bench fields: the compression ratio at each
    ablation step (Base = LZ1 with independent blocks, +Cross = the state carried across
    blocks, +Cent. = centred variants, +LZ2 = the full method), and the compression time of
    the single-pass evaluation against the multipass one (a pass per variant writing tile
    costs, then the encoding pass selecting from them; identical streams)."""
    import math
    import statistics

    import torch
    levels = (("base", fsz.OFF_CROSS_BLOCK | fsz.OFF_CENTERING | fsz.OFF_LZ2),
              ("+cross", fsz.OFF_CENTERING | fsz.OFF_LZ2), ("+center", fsz.OFF_LZ2), ("+lz2", 0))
    n = fields[0][1].numel()
    T = (n + 255) // 256
    cap = fsz.fsz_compress_bound(n)
    out = torch.empty(cap, dtype=torch.uint8, device=dev)
    out2 = torch.empty(cap, dtype=torch.uint8, device=dev)
    ws = fsz.Workspace(n, dev)
    costs = torch.empty((4, T), dtype=torch.int32, device=dev)
    nb = torch.zeros(2, dtype=torch.int64, device=dev)
    dims = fsz.make_dims(shape)
    L = fsz.lib()
    sp = torch.cuda.current_stream(dev).cuda_stream
    rows, timing = [], []

    def timed(fn, reps=6):
        ts = []
        for _ in range(reps):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            st = fn()
            e1.record()
            torch.cuda.synchronize(dev)
            if st != 0:
                raise fsz.FszError(st, "ablation")
            ts.append(e0.elapsed_time(e1))
        return statistics.median(ts[1:])

    for name, x in fields:
        for rel in rels:
            row = {"field": name, "rel": rel}
            for lname, off in levels:
                _, k = fsz.compress(x, rel, fsz.EB_REL, shape=shape, ws=ws, out=out, features_off=off)
                row[lname] = 4 * n / k
            rows.append(row)
            single = timed(lambda: L.fsz_compress(x.data_ptr(), dims, 1, rel, out.data_ptr(), cap,
                                                  nb.data_ptr(), ws.ptr, ws.bytes, sp))
            k1 = int(nb[0].item())
            multi = timed(lambda: L.fsz_compress_multipass(x.data_ptr(), dims, 1, rel, out2.data_ptr(), cap,
                                                           nb.data_ptr(), costs.data_ptr(), ws.ptr,
                                                           ws.bytes, sp))
            if fsz.fsz_check(ws.ptr, sp) != 0:
                raise fsz.FszError(fsz.fsz_check(ws.ptr, sp), "multipass (device)")
            k2 = int(nb[0].item())
            same = k1 == k2 and torch.equal(out[:k1], out2[:k2])
            timing.append({"field": name, "rel": rel, "single_pass_ms": single, "multipass_ms": multi,
                           "single_pass_gbs": 4 * n / single / 1e6, "multipass_gbs": 4 * n / multi / 1e6,
                           "speedup": multi / single, "identical_stream": bool(same)})
    # adaptive pre-zero (Sec. 3.1): a field of about 99 % exact zeros around a band of the
    # GRF (CR above 100), decoded in full and into a zero-filled output skipping the
    # all-zero tiles; the zero fill is inside the timed region
    g0 = fields[0][1]
    xs = torch.zeros_like(g0)
    band = n // 128
    xs[n // 2: n // 2 + band] = g0[:band] + 280.0
    _, ks = fsz.compress(xs, 1e-3, fsz.EB_REL, shape=shape, ws=ws, out=out)
    rec = torch.empty(n, dtype=torch.float32, device=dev)
    full_ms = timed(lambda: L.fsz_decompress(out.data_ptr(), ks, rec.data_ptr(), n, ws.ptr, ws.bytes, sp))
    ref = rec.clone()

    def prezeroed():
        rec.zero_()
        return L.fsz_decompress_prezeroed(out.data_ptr(), ks, rec.data_ptr(), n, ws.ptr, ws.bytes, sp)
    pz_ms = timed(prezeroed)
    same = bool(torch.equal(rec, ref))
    # into an output that already holds the zeros (a buffer reused for such fields)
    pzk_ms = timed(lambda: L.fsz_decompress_prezeroed(out.data_ptr(), ks, rec.data_ptr(), n, ws.ptr,
                                                      ws.bytes, sp))
    prezero = {"workload": "512^3 float32: zeros except a band of n/128 GRF+280 values, REL 1e-3",
               "cr": 4 * n / ks, "full_decode_ms": full_ms, "zero_fill_and_prezero_decode_ms": pz_ms,
               "prezero_decode_into_zeros_ms": pzk_ms, "full_gbs": 4 * n / full_ms / 1e6,
               "speedup_with_zero_fill": full_ms / pz_ms, "speedup_into_zeros": full_ms / pzk_ms,
               "identical": same}
    del xs, rec, ref
    geo = lambda v: math.exp(sum(math.log(a) for a in v) / len(v))
    gains = {lname: geo([r[lname] / r["base"] for r in rows]) for lname, _ in levels}
    return {"workload": "the bench fields (512^3 k^-3 GRF, zero-slab variant) at each REL",
            "features_off": {lname: off for lname, off in levels},
            "cr": rows, "cr_gain_over_base_geomean": gains, "single_vs_multipass": timing,
            "single_pass_speedup_geomean": geo([t["speedup"] for t in timing]), "prezero": prezero}


def run_tiles(fsz, fields, rels, dev, shape):
    """Sec. 6.5 (Table 8): every tile configuration (B elements per block, T blocks per
    tile) on the bench fields through the generic two-read path: CR against the default
    B = 32, T = 8 (win / loss beyond 2 %, tie within), and the generic path's compression
    and decompression time; the specialised single-pass kernels cover 32 x 8 only."""
    import math
    import statistics

    import torch
    L = fsz.lib()
    sp = torch.cuda.current_stream(dev).cuda_stream
    n = fields[0][1].numel()
    wsb = L.fsz_tiled_workspace_bytes(n)
    ws = torch.empty(wsb, dtype=torch.uint8, device=dev)
    cap = max(L.fsz_compress_bound_tiled(n, B, T) for B, T in fsz.TILE_CONFIGS)
    out = torch.empty(cap, dtype=torch.uint8, device=dev)
    rec = torch.empty(n, dtype=torch.float32, device=dev)
    nb = torch.zeros(2, dtype=torch.int64, device=dev)
    dims = fsz.make_dims(shape)

    def timed(fn, reps=4):
        ts = []
        for _ in range(reps):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            st = fn()
            e1.record()
            torch.cuda.synchronize(dev)
            if st != 0:
                raise fsz.FszError(st, "tiles")
            ts.append(e0.elapsed_time(e1))
        return statistics.median(ts[1:])

    rows = []
    for name, x in fields:
        for rel in rels:
            row = {"field": name, "rel": rel}
            for B, T in fsz.TILE_CONFIGS:
                c_ms = timed(lambda: L.fsz_compress_tiled(x.data_ptr(), dims, 1, rel, B, T, 0, out.data_ptr(),
                                                          cap, nb.data_ptr(), ws.data_ptr(), wsb, sp))
                if fsz.fsz_check(ws.data_ptr(), sp) != fsz.OK:
                    raise fsz.FszError(fsz.fsz_check(ws.data_ptr(), sp), "tiles compress")
                k = int(nb[0].item())
                d_ms = timed(lambda: L.fsz_decompress_tiled(out.data_ptr(), k, rec.data_ptr(), n,
                                                            ws.data_ptr(), wsb, sp))
                if fsz.fsz_check(ws.data_ptr(), sp) != fsz.OK:
                    raise fsz.FszError(fsz.fsz_check(ws.data_ptr(), sp), "tiles decompress")
                row[f"{B}x{T}"] = {"cr": 4 * n / k, "compress_gbs": 4 * n / c_ms / 1e6,
                                   "decompress_gbs": 4 * n / d_ms / 1e6}
            rows.append(row)
    summary = {}
    for B, T in fsz.TILE_CONFIGS:
        key = f"{B}x{T}"
        ratios = [r[key]["cr"] / r["32x8"]["cr"] for r in rows]
        summary[key] = {"win": sum(q > 1.02 for q in ratios), "tie": sum(0.98 <= q <= 1.02 for q in ratios),
                        "loss": sum(q < 0.98 for q in ratios), "cr_ratio_mean": sum(ratios) / len(ratios),
                        "compress_gbs_geomean": math.exp(sum(math.log(r[key]["compress_gbs"]) for r in rows) / len(rows)),
                        "decompress_gbs_geomean": math.exp(sum(math.log(r[key]["decompress_gbs"]) for r in rows) / len(rows))}
    del out, rec, ws
    torch.cuda.empty_cache()
    return {"workload": "the bench fields at each REL, every (B, T) through the generic tiled path",
            "rows": rows, "vs_32x8": summary}


CONFIG_WORKLOADS = {
    1: "2^20 float32, five seeded sinusoids + noise (seed 0), REL 1e-3 (4 MiB: held in L2)",
    3: "2^28 float32 (1 GiB), particle x-coordinates around 10^4 centres then N(0, 300^2) "
       "velocities (seed 2), REL 1e-4",
    4: "512 fields (seed 3), log-uniform 64 KiB-64 MiB, 1-3-D, 40% k^-3 GRF / 40% particles / "
       "20% zero-slab offset, REL per field from {1e-2, 1e-3, 1e-4}; one batched graph launch "
       "each way, default schedule",
}


def run_config(args, fsz, inputs, dev, cfg: int):
    """Compresses and decompresses one of the other workloads for --steps timed steps (after
    --warmup untimed ones) and prints one JSON line of per-kernel input GB/s (median and
    mean over the steps): the per-configuration numbers and the command their ncu launch
    lists are taken with."""
    import torch
    L = fsz.lib()
    stream = torch.cuda.current_stream(dev)
    sp = stream.cuda_stream
    out = {"config_run": cfg, "workload": CONFIG_WORKLOADS[cfg], "steps": args.steps,
           "warmup": max(3, args.warmup)}
    ev = lambda: torch.cuda.Event(enable_timing=True)
    if cfg in (1, 3):
        if cfg == 1:
            x = torch.from_numpy(inputs.sinusoids(1 << 20, seed=0)).to(dev)
            rel = 1e-3
        else:
            x = inputs.particles(1 << 28, seed=2, device=str(dev))
            rel = 1e-4
        torch.cuda.empty_cache()
        n = x.numel()
        dims = fsz.make_dims((n,))
        cap = fsz.fsz_compress_bound(n)
        sb = torch.empty(cap, dtype=torch.uint8, device=dev)
        rec = torch.empty(n, dtype=torch.float32, device=dev)
        nb = torch.zeros(1, dtype=torch.int64, device=dev)
        wsb = fsz.fsz_workspace_bytes(n)
        ws = torch.empty(wsb, dtype=torch.uint8, device=dev)
        times = {"stats": [], "encode": [], "decompress": []}
        for k in range(max(3, args.warmup) + args.steps):
            e = [ev() for _ in range(4)]
            e[0].record(stream)
            st = L.fsz_compress_prepare(x.data_ptr(), dims, fsz.EB_REL, rel, sb.data_ptr(), cap,
                                        nb.data_ptr(), ws.data_ptr(), wsb, sp)
            e[1].record(stream)
            st |= L.fsz_compress_encode(x.data_ptr(), dims, fsz.EB_REL, rel, sb.data_ptr(), cap,
                                        nb.data_ptr(), ws.data_ptr(), wsb, sp)
            e[2].record(stream)
            st |= L.fsz_decompress(sb.data_ptr(), cap, rec.data_ptr(), n, ws.data_ptr(), wsb, sp)
            e[3].record(stream)
            if st:
                raise fsz.FszError(st, f"config {cfg}")
            torch.cuda.synchronize(dev)
            if k >= max(3, args.warmup):
                times["stats"].append(e[0].elapsed_time(e[1]))
                times["encode"].append(e[1].elapsed_time(e[2]))
                times["decompress"].append(e[2].elapsed_time(e[3]))
        st = fsz.fsz_check(ws.data_ptr(), sp)
        if st != fsz.OK:
            raise fsz.FszError(st, f"config {cfg}")
        k = int(nb[0].item())
        q = fsz.quality(x, rec, rel * (float(x.max().item()) - float(x.min().item())), k)
        nbytes_in = 4 * n
        out.update({"n": n, "cr": 4 * n / k, "psnr_db": q["psnr_db"], "bit_rate": q["bit_rate"],
                    "errors_over_bound": q["over_bound"]})
    else:
        specs = inputs.field_mix_specs(512, seed=3)
        fields = [(inputs.make_field(spec, device=str(dev)).contiguous(), spec["dims"], fsz.EB_REL,
                   spec["rel"]) for spec in specs]
        torch.cuda.empty_cache()
        nbytes_in = sum(4 * f.numel() for f, *_ in fields)
        cb = fsz.CompressBatch(fields, dev)
        assert cb.run() == fsz.OK and cb.status()[0] == fsz.OK
        sizes = cb.sizes.cpu().tolist()
        db = fsz.DecompressBatch([cb.stream(i, sizes) for i in range(len(fields))],
                                 [f.numel() for f, *_ in fields], dev)
        comp_bytes = sum(sizes)
        times = {"compress": [], "decompress": []}
        for k in range(max(3, args.warmup) + args.steps):
            e = [ev() for _ in range(3)]
            e[0].record(stream)
            st = cb.launch_graph()
            e[1].record(stream)
            st |= db.launch_graph()
            e[2].record(stream)
            if st:
                raise fsz.FszError(st, "config 4 graph launch")
            torch.cuda.synchronize(dev)
            if k >= max(3, args.warmup):
                times["compress"].append(e[0].elapsed_time(e[1]))
                times["decompress"].append(e[1].elapsed_time(e[2]))
        st = cb.status()[0] or db.status()[0]
        if st != fsz.OK:
            raise fsz.FszError(st, "config 4")
        out.update({"n": nbytes_in // 4, "fields": len(fields), "cr": nbytes_in / comp_bytes})
    for name, ts in times.items():
        out[f"{name}_gbs"] = nbytes_in / statistics.median(ts) / 1e6
        out[f"{name}_gbs_mean"] = nbytes_in / statistics.mean(ts) / 1e6
    out["note"] = ("input bytes / CUDA-event time per kernel (stats = the value-range pass with its "
                   "set-up kernel; encode = the compression kernel)" if cfg != 4 else
                   "input bytes / CUDA-event time per batched graph launch")
    print(json.dumps(out))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=100)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="fsz", choices=["fsz", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-batched", action="store_true",
                    help="skip the 512-field batched vs per-field comparison")
    ap.add_argument("--no-ablation", action="store_true",
                    help="skip the ablation ladder and the multipass comparison")
    ap.add_argument("--no-serving", action="store_true",
                    help="skip the continuous-batching serving measurement")
    ap.add_argument("--serving-requests", type=int, default=20000,
                    help="requests per serving level (the serving workload has 20,000)")
    ap.add_argument("--fields", default="grf,zero_slabs",
                    help="subset of grf,zero_slabs (smaller cases for profiling)")
    ap.add_argument("--rels", default=",".join(str(r) for r in RELS),
                    help="subset of the error bounds (smaller cases for profiling)")
    ap.add_argument("--config", type=int, choices=[1, 3, 4], default=None,
                    help="time one of the other workloads alone (per-configuration numbers and "
                         "their profiles) instead of the bench")
    args = ap.parse_args()
    world, rank, local = dist_setup(args.gpus)
    if args.impl == "reference":
        return run_reference(args, world, rank)

    import numpy as np
    import torch

    import __graft_entry__
    __graft_entry__.build()
    from paper_2607_15413_gb300 import fsz, inputs

    cpu = None
    if rank == 0 and not args.no_cpu_baseline and args.config is None:
        sample = cpu_sample_fields()
        cpu = cpu_baseline_run(sample)   # on the host, before any GPU work
        cpu["all_core"] = cpu_all_core_run(sample)
        cpu["cpu_model"] = cpu["all_core"]["cpu_model"]
        del sample

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if args.config is not None:
        if rank == 0:
            run_config(args, fsz, inputs, dev, args.config)
        barrier(world)
        return
    stream = torch.cuda.current_stream(dev)
    sp = stream.cuda_stream

    # inputs resident in HBM
    want = args.fields.split(",")
    g = inputs.grf(SHAPE, seed=1, device=str(dev)).reshape(-1)
    fields = []
    if "grf" in want:
        fields.append(("grf", g))
    if "zero_slabs" in want:
        fields.append(("zero_slabs",
                       inputs.zero_slabs(SHAPE, seed=1, device=str(dev), base=g.reshape(SHAPE)).reshape(-1)))
    torch.cuda.empty_cache()
    rels = [float(r) for r in args.rels.split(",")]
    n = g.numel()
    cap = fsz.fsz_compress_bound(n)
    jobs = [(name, x, rel) for name, x in fields for rel in rels]
    outs = [torch.empty(cap, dtype=torch.uint8, device=dev) for _ in jobs]
    recon = torch.empty(n, dtype=torch.float32, device=dev)
    nbytes = torch.zeros(len(jobs), dtype=torch.int64, device=dev)
    wsb = fsz.fsz_workspace_bytes(n)
    ws = torch.empty(wsb, dtype=torch.uint8, device=dev)
    dims = fsz.make_dims(SHAPE)
    L = fsz.lib()
    mk = lambda k: [torch.cuda.Event(enable_timing=True) for _ in range(k)]
    ev_steps = [([mk(3) for _ in jobs], [mk(2) for _ in jobs]) for _ in range(args.steps)]
    launches_per_step = len(jobs) * (3 + 2)   # setup+stats+compress, setup+decompress
    main_schedule = fsz.fsz_get_schedule()    # the library defaults (not the batched table)

    def step(events):
        record = events is not None
        ev, evd = events if record else (None, None)
        for j, (name, x, rel) in enumerate(jobs):
            e = ev[j] if record else None
            if record:
                e[0].record(stream)
            st = L.fsz_compress_prepare(x.data_ptr(), dims, fsz.EB_REL, rel, outs[j].data_ptr(), cap,
                                        nbytes[j:].data_ptr(), ws.data_ptr(), wsb, sp)
            if record:
                e[1].record(stream)
            st |= L.fsz_compress_encode(x.data_ptr(), dims, fsz.EB_REL, rel, outs[j].data_ptr(), cap,
                                        nbytes[j:].data_ptr(), ws.data_ptr(), wsb, sp)
            if record:
                e[2].record(stream)
            if st:
                raise fsz.FszError(st, "compress")
        for j, (name, x, rel) in enumerate(jobs):
            e = evd[j] if record else None
            if record:
                e[0].record(stream)
            st = L.fsz_decompress(outs[j].data_ptr(), cap, recon.data_ptr(), n, ws.data_ptr(), wsb, sp)
            if record:
                e[1].record(stream)
            if st:
                raise fsz.FszError(st, "decompress")

    for _ in range(max(3, args.warmup)):
        step(None)
    st = fsz.fsz_check(ws.data_ptr(), sp)
    if st != fsz.OK:
        raise fsz.FszError(st, "warm-up")
    sizes = nbytes.cpu().tolist()
    # rate-distortion point of every job (Sec. 6.2, Fig. 8), on the device, untimed:
    # decompress its stream and compare with the original
    qual = []
    for j, (name, x, rel) in enumerate(jobs):
        st = L.fsz_decompress(outs[j].data_ptr(), sizes[j], recon.data_ptr(), n, ws.data_ptr(), wsb, sp)
        if st != fsz.OK or fsz.fsz_check(ws.data_ptr(), sp) != fsz.OK:
            raise fsz.FszError(st, "quality decode")
        eb = rel * (float(x.max().item()) - float(x.min().item()))
        qual.append(fsz.quality(x, recon, eb, sizes[j]))
        # the stream's own record: the requested bound (REL) and the step from its preamble,
        # and how many tiles took each variant (byte 0 of a tile's header: bit 7 order 2,
        # bit 6 centred)
        pre = fsz.fsz_read_header(outs[j][:64].cpu().numpy().tobytes())
        T = (n + 255) // 256
        sel = (outs[j][64:64 + 8 * T:8].to(torch.int64) >> 6) & 3
        cnt = torch.bincount(sel, minlength=4).tolist()
        qual[-1].update({"eb": eb, "eb_requested": pre["eb"], "step": pre["step"],
                         "variants": {"lz1": cnt[0], "lz1c": cnt[1], "lz2": cnt[2], "lz2c": cnt[3]}})
    p_last = qual[-1]["max_abs_err"]

    comp_ms, enc_ms, stats_ms, dec_ms = ([[] for _ in jobs] for _ in range(4))
    torch.cuda.synchronize(dev)
    barrier(world)
    with ClockSampler(local) as clocks:
        t_start = torch.cuda.Event(enable_timing=True)
        t_end = torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize(dev)
        barrier(world)
        t_start.record(stream)
        for k in range(args.steps):
            step(ev_steps[k])
        t_end.record(stream)
        torch.cuda.synchronize(dev)
        barrier(world)
    for ev, evd in ev_steps:
        for j in range(len(jobs)):
            stats_ms[j].append(ev[j][0].elapsed_time(ev[j][1]))
            enc_ms[j].append(ev[j][1].elapsed_time(ev[j][2]))
            comp_ms[j].append(ev[j][0].elapsed_time(ev[j][2]))
            dec_ms[j].append(evd[j][0].elapsed_time(evd[j][1]))
    total_ms = t_start.elapsed_time(t_end)
    bytes_step = 2 * len(jobs) * 4 * n
    value, ms_step = job_throughput(world, bytes_step, total_ms / args.steps)

    # Each kernel alone right after an L2 flush (a 256 MiB scratch write), so that neither
    # its input nor its stream can come from L2; median of 3 per job, outside the timed steps.
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)
    enc_fl, dec_fl = [[] for _ in jobs], [[] for _ in jobs]
    for rep in range(3):
        for j, (name, x, rel) in enumerate(jobs):
            e = [torch.cuda.Event(enable_timing=True) for _ in range(4)]
            st = L.fsz_compress_prepare(x.data_ptr(), dims, fsz.EB_REL, rel, outs[j].data_ptr(), cap,
                                        nbytes[j:].data_ptr(), ws.data_ptr(), wsb, sp)
            flush.fill_(rep + 1)
            e[0].record(stream)
            st |= L.fsz_compress_encode(x.data_ptr(), dims, fsz.EB_REL, rel, outs[j].data_ptr(), cap,
                                        nbytes[j:].data_ptr(), ws.data_ptr(), wsb, sp)
            e[1].record(stream)
            flush.fill_(rep + 2)
            e[2].record(stream)
            st |= L.fsz_decompress(outs[j].data_ptr(), cap, recon.data_ptr(), n, ws.data_ptr(), wsb, sp)
            e[3].record(stream)
            if st:
                raise fsz.FszError(st, "L2-flushed run")
            torch.cuda.synchronize(dev)
            enc_fl[j].append(e[0].elapsed_time(e[1]))
            dec_fl[j].append(e[2].elapsed_time(e[3]))
    del flush

    # e2e: the same calls with pinned host buffers. Copies run on their own streams (one
    # per direction) and overlap the kernels, as a pipeline feeding the GPU would:
    # inputs in -> compress -> streams out and back in -> decompress -> reconstructions out.
    e2e = None
    if not args.no_e2e:
        hin = [torch.empty(n, dtype=torch.float32, pin_memory=True) for _ in fields]
        for (name, x), h in zip(fields, hin):
            h.copy_(x.cpu())
        hstream = [torch.empty(cap, dtype=torch.uint8, pin_memory=True) for _ in jobs]
        hout = [torch.empty(n, dtype=torch.float32, pin_memory=True) for _ in range(2)]
        hsizes = torch.empty(len(jobs), dtype=torch.int64, pin_memory=True)
        din = [torch.empty(n, dtype=torch.float32, device=dev) for _ in fields]
        recon2 = [recon, torch.empty(n, dtype=torch.float32, device=dev)]
        s_in = torch.cuda.Stream(dev)
        s_out = torch.cuda.Stream(dev)
        s_comp = torch.cuda.current_stream(dev)
        names = [f[0] for f in fields]

        def ev(stream):
            e = torch.cuda.Event()
            e.record(stream)
            return e

        def e2e_step():
            h2d = d2h = 0
            e_in = []
            for h, d in zip(hin, din):
                with torch.cuda.stream(s_in):
                    d.copy_(h, non_blocking=True)
                e_in.append(ev(s_in))
                h2d += 4 * n
            for j, (name, x, rel) in enumerate(jobs):
                k = names.index(name)
                s_comp.wait_event(e_in[k])
                s1 = L.fsz_compress(din[k].data_ptr(), dims, fsz.EB_REL, rel, outs[j].data_ptr(), cap,
                                    nbytes[j:].data_ptr(), ws.data_ptr(), wsb, sp)
                if s1:
                    raise fsz.FszError(s1, "compress")
            hsizes.copy_(nbytes, non_blocking=True)
            ev(s_comp).synchronize()          # stream sizes, to copy exactly the streams
            szs = hsizes.tolist()
            d2h += 8 * len(jobs)
            e_back = []
            for j in range(len(jobs)):
                with torch.cuda.stream(s_out):
                    hstream[j][: szs[j]].copy_(outs[j][: szs[j]], non_blocking=True)
                e_st = ev(s_out)
                d2h += szs[j]
                s_in.wait_event(e_st)
                with torch.cuda.stream(s_in):
                    outs[j][: szs[j]].copy_(hstream[j][: szs[j]], non_blocking=True)
                e_back.append(ev(s_in))
                h2d += szs[j]
            for j in range(len(jobs)):
                s_comp.wait_event(e_back[j])
                if e_free[j % 2] is not None:
                    s_comp.wait_event(e_free[j % 2])  # the buffer's previous copy-out is done
                s2 = L.fsz_decompress(outs[j].data_ptr(), szs[j], recon2[j % 2].data_ptr(), n,
                                      ws.data_ptr(), wsb, sp)
                if s2:
                    raise fsz.FszError(s2, "decompress")
                s_out.wait_event(ev(s_comp))
                with torch.cuda.stream(s_out):
                    hout[j % 2].copy_(recon2[j % 2], non_blocking=True)
                e_free[j % 2] = ev(s_out)
                d2h += 4 * n
            return h2d, d2h

        # the reconstruction buffers' last copy-out, carried across steps
        e_free = [None, None]

        for _ in range(2):
            e2e_step()
        torch.cuda.synchronize(dev)
        barrier(world)
        t0 = time.perf_counter()
        ksteps = max(1, min(args.steps, 5))
        for _ in range(ksteps):
            h2d, d2h = e2e_step()
        torch.cuda.synchronize(dev)
        e2e_gbs, e2e_ms = job_throughput(world, bytes_step, (time.perf_counter() - t0) * 1e3 / ksteps)
        # the host links alone, for context: one 512 MiB copy each way
        link = {}
        for direction, (dst, src) in (("h2d_gbs", (din[0], hin[0])), ("d2h_gbs", (hout[0], recon))):
            torch.cuda.synchronize(dev)
            t1 = time.perf_counter()
            for _ in range(3):
                dst.copy_(src, non_blocking=True)
            torch.cuda.synchronize(dev)
            link[direction] = 3 * 4 * n / (time.perf_counter() - t1) / 1e9
        e2e = {"value": e2e_gbs, "unit": "GB/s",
               "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h, "ms_per_step": e2e_ms,
               "copies": "pinned host buffers; one copy stream per direction overlapping the kernels",
               "link_alone": link}
        del hin, hstream, din, recon2


    # roofline of the dominant kernel (algorithmic bytes / CUDA-event duration)
    peaks, peak_kind = measured_peaks()
    enc_tot = sum(sum(v) for v in enc_ms)
    dec_tot = sum(sum(v) for v in dec_ms)
    comp_bytes = sum(4 * n + sizes[j] for j in range(len(jobs)))
    dec_bytes = sum(sizes[j] + 4 * n for j in range(len(jobs)))
    if enc_tot >= dec_tot:
        kern, algo, dur = "fsz_compress_kernel", comp_bytes * args.steps, enc_tot
    else:
        kern, algo, dur = "fsz_decompress_kernel (incl. its set-up kernel)", dec_bytes * args.steps, dec_tot
    achieved = algo / (dur * 1e-3) / 1e9
    traffic = None
    try:  # DRAM bytes of one ncu capture, valid while the kernel's sources are unchanged
        import hashlib
        with open(os.path.join(ROOT, "profiles", "traffic.json")) as f:
            rec = json.load(f).get(kern)
        if rec:
            h = hashlib.sha256()
            for src in rec["sources"]:
                with open(os.path.join(ROOT, src), "rb") as f:
                    h.update(f.read())
            if h.hexdigest() == rec["sha256"]:
                traffic = rec["dram_bytes_read"] + rec["dram_bytes_write"]
    except (OSError, KeyError, ValueError):
        traffic = None
    roofline = {"bound": "hbm", "kernel": kern, "achieved": achieved, "peak": peaks["hbm_gbs"],
                "unit": "GB/s", "frac": achieved / peaks["hbm_gbs"], "peak_kind": peak_kind,
                "frac_of_nominal_8tbs": achieved / NOMINAL_HBM_GBS, "traffic": traffic,
                "traffic_note": "mean dram read+write bytes per launch over the 6 jobs of one step (one ncu capture; "
                                "profiles/traffic.json), null once the kernel source changed",
                "algorithmic_bytes_per_launch": algo / (args.steps * len(jobs))}

    per_job = []
    for j, (name, x, rel) in enumerate(jobs):
        med = lambda v: statistics.median(v)
        per_job.append({"field": name, "rel": rel, "cr": 4 * n / sizes[j], "bytes": sizes[j],
                        "psnr_db": qual[j]["psnr_db"], "bit_rate": qual[j]["bit_rate"],
                        "nrmse": qual[j]["nrmse"], "max_abs_err": qual[j]["max_abs_err"],
                        "errors_over_bound": qual[j]["over_bound"],
                        "eb": qual[j]["eb"], "eb_requested": qual[j]["eb_requested"],
                        "step": qual[j]["step"],
                        "max_err_over_eb": qual[j]["max_abs_err"] / qual[j]["eb"],
                        "variants": qual[j]["variants"],
                        "compress_gbs": 4 * n / med(comp_ms[j]) / 1e6,
                        "encode_kernel_gbs": 4 * n / med(enc_ms[j]) / 1e6,
                        "encode_kernel_hbm_gbs": (4 * n + sizes[j]) / med(enc_ms[j]) / 1e6,
                        "stats_gbs": 4 * n / med(stats_ms[j]) / 1e6,
                        "decompress_gbs": 4 * n / med(dec_ms[j]) / 1e6,
                        "decompress_hbm_gbs": (4 * n + sizes[j]) / med(dec_ms[j]) / 1e6,
                        # the same over the mean step instead of the median one
                        "compress_gbs_mean": 4 * n / statistics.mean(comp_ms[j]) / 1e6,
                        "encode_kernel_gbs_mean": 4 * n / statistics.mean(enc_ms[j]) / 1e6,
                        "decompress_gbs_mean": 4 * n / statistics.mean(dec_ms[j]) / 1e6,
                        # each kernel alone after a 256 MiB L2 flush (median of 3)
                        "encode_kernel_hbm_gbs_l2flushed": (4 * n + sizes[j]) / med(enc_fl[j]) / 1e6,
                        "decompress_hbm_gbs_l2flushed": (4 * n + sizes[j]) / med(dec_fl[j]) / 1e6})
    njobs, nfields_main = len(jobs), len(fields)
    clock_summary = clocks.summary()
    ablation = None
    tiles = None
    if not args.no_ablation:
        del outs, recon
        torch.cuda.empty_cache()
        ablation = run_ablation(fsz, fields, rels, dev, SHAPE)
        tiles = run_tiles(fsz, fields, rels, dev, SHAPE)
    batched = None
    if not args.no_batched:
        del fields, jobs, g
        if args.no_ablation:
            del outs, recon
        torch.cuda.empty_cache()
        batched = run_batched(fsz, inputs, dev)
    serving = None
    if not args.no_serving:
        serving = run_serving(fsz, inputs, dev, nreq=args.serving_requests)
    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": "GB/s", "n_gpus": world,
                "steps": args.steps, "warmup": max(3, args.warmup), "ms_per_step": ms_step,
                "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
                "data": "synthetic",
                "config": {"workload": WORKLOAD if njobs == 6 else
                           f"subset: fields {args.fields}, REL {args.rels} of: " + WORKLOAD,
                           "n_per_field": n, "fields": nfields_main, "rels": rels,
                           "parallelism": f"replicas x{world} (no data-path collective)",
                           "l2": "inputs 512 MiB > L2; streams read back after >= 2.5 GB of traffic; "
                                 "jobs[].*_l2flushed: each kernel alone after a 256 MiB scratch write",
                           "schedule": main_schedule},
                "roofline": roofline, "cpu_baseline": cpu, "e2e": e2e,
                "gpu_launches": launches_per_step * args.steps,
                "clocks": clock_summary, "jobs": per_job, "ablation": ablation, "tiles": tiles,
                "batched": batched,
                "serving": serving,
                "max_abs_err_last_job": p_last}
        print(json.dumps(line))
    barrier(world)
    return 0


if __name__ == "__main__":
    sys.exit(main())
