"""Launch-schedule autotuner for the batched path.

The tunable is the number of persistent CTAs per SM of each kernel (value-range pass,
compression, decompression), set through fsz_set_schedule; the stream format does not
depend on it. The tuner times each candidate on the caller's batch (CUDA-graph launches,
CUDA events, median of a few runs) and keeps the fastest per kernel. A table measured on
GB300 ships as schedules.json; `apply_default()` installs it.
"""
from __future__ import annotations

import json
import os
import statistics

from . import fsz

DEFAULT_TABLE = os.path.join(os.path.dirname(os.path.abspath(__file__)), "schedules.json")


def _time_graph(launch, reps: int):
    import torch
    ts = []
    for _ in range(reps):
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record()
        st = launch()
        e1.record()
        torch.cuda.synchronize()
        if st != fsz.OK:
            raise fsz.FszError(st, "tune")
        ts.append(e0.elapsed_time(e1))
    return statistics.median(ts)


def tune(cbatch: "fsz.CompressBatch", dbatch: "fsz.DecompressBatch", reps: int = 3) -> dict:
    """Times every schedule candidate on the given batches; returns the best per kernel
    and the timings. The graphs are captured once: the schedule is read at launch time
    of the host call, so each candidate is captured into its own graph."""
    lim = fsz.fsz_get_schedule_limits()
    results = {"limits": lim, "compress": {}, "decompress": {}}
    for k in range(1, lim["compress"] + 1):
        fsz.fsz_set_schedule(0, k, 0)
        g = fsz.fsz_graph_compress_batched(cbatch.table.data_ptr(), len(cbatch.fields),
                                           cbatch.n_total, cbatch.ws.data_ptr(), cbatch.ws_bytes)
        try:
            _time_graph(lambda: fsz.fsz_graph_launch(g, fsz._stream_ptr()), 1)  # warm-up
            results["compress"][k] = _time_graph(lambda: fsz.fsz_graph_launch(g, fsz._stream_ptr()), reps)
        finally:
            fsz.fsz_graph_destroy(g)
    for k in range(1, lim["decompress"] + 1):
        fsz.fsz_set_schedule(0, 0, k)
        g = fsz.fsz_graph_decompress_batched(dbatch.table.data_ptr(), len(dbatch.streams),
                                             dbatch.cap_total, dbatch.ws.data_ptr(), dbatch.ws_bytes)
        try:
            _time_graph(lambda: fsz.fsz_graph_launch(g, fsz._stream_ptr()), 1)
            results["decompress"][k] = _time_graph(lambda: fsz.fsz_graph_launch(g, fsz._stream_ptr()), reps)
        finally:
            fsz.fsz_graph_destroy(g)
    fsz.fsz_set_schedule(0, 0, 0)
    best_c = min(results["compress"], key=results["compress"].get)
    best_d = min(results["decompress"], key=results["decompress"].get)
    results["best"] = {"stats": 0, "compress": int(best_c), "decompress": int(best_d)}
    return results


def apply(best: dict) -> None:
    """Installs a schedule {stats, compress, decompress} (CTAs per SM; 0 = all that fit)."""
    st = fsz.fsz_set_schedule(int(best.get("stats", 0)), int(best.get("compress", 0)),
                              int(best.get("decompress", 0)))
    if st != fsz.OK:
        raise fsz.FszError(st, "fsz_set_schedule")


def save(results: dict, path: str) -> None:
    with open(path, "w") as f:
        json.dump(results, f, indent=1, sort_keys=True)


def apply_default(path: str = DEFAULT_TABLE) -> dict | None:
    """Installs the schedule table shipped with the package, if present."""
    try:
        with open(path) as f:
            table = json.load(f)
    except OSError:
        return None
    apply(table["best"])
    return table["best"]


def main() -> None:
    """Tunes on the 512-field batch (seed 3: log-uniform 64 KiB-64 MiB, mixed classes and
    REL bounds) on cuda:0 and writes the table that ships with the package."""
    import torch
    from . import inputs
    dev = torch.device("cuda", 0)
    specs = inputs.field_mix_specs(512, seed=3)
    fields = [(inputs.make_field(spec, device=str(dev)).contiguous(), spec["dims"], fsz.EB_REL,
               spec["rel"]) for spec in specs]
    cb = fsz.CompressBatch(fields, dev)
    if cb.run() != fsz.OK or cb.status()[0] != fsz.OK:
        raise fsz.FszError(cb.status()[0], "tune: compress")
    sizes = cb.sizes.cpu().tolist()
    db = fsz.DecompressBatch([cb.stream(i, sizes) for i in range(len(fields))],
                             [f.numel() for f, *_ in fields], dev)
    res = tune(cb, db, reps=5)
    props = torch.cuda.get_device_properties(dev)
    save({"device": f"{props.name} ({props.multi_processor_count} SMs)",
          "workload": "512 fields, seed 3: log-uniform 64 KiB-64 MiB, 1-3-D, 40% k^-3 GRF / "
                      "40% particle-like / 20% zero-slab, REL in {1e-2,1e-3,1e-4}",
          "limits": res["limits"], "best": res["best"],
          "tuning_ms": {"compress": res["compress"], "decompress": res["decompress"]},
          "note": "CTAs per SM for the value-range, compression and decompression kernels; "
                  "0 = as many as fit. Measured by paper_2607_15413_gb300.tune on the batched "
                  "workload (graph launches, median of 5)."}, DEFAULT_TABLE)
    print(json.dumps(res["best"]))


if __name__ == "__main__":
    main()
