"""Launch-schedule autotuner for the batched path.

The schedule (fsz_schedule, set through fsz_set_schedule_ex; the stream format does not
depend on it) assigns work to the persistent kernels:
  * CTAs per SM of the value-range, compression and decompression kernels;
  * the work item of compression and decompression: how many consecutive 32-tile chunks
    one ticket hands a CTA (1-4, i.e. 32-128 tiles; inside an item the chunks after the
    first take their offsets without a lookback);
  * compression: how many chunks ahead of its compute warps a CTA takes tickets (1-3);
  * decompression: how many chunks a CTA holds between ticket and decode (8, 12, 16).
The tuner times every candidate of each kernel on the caller's batch (CUDA-graph launches,
CUDA events, median of a few runs; the other kernel's settings at their defaults) and keeps
the fastest. A table measured on GB300 ships as schedules.json; `apply_default()` installs
it.
"""
from __future__ import annotations

import itertools
import json
import os
import statistics

from . import fsz

DEFAULT_TABLE = os.path.join(os.path.dirname(os.path.abspath(__file__)), "schedules.json")

TICKET_CHUNKS = (1, 2, 3, 4)
COMPRESS_LEADS = (1, 2, 3)
DECOMPRESS_RECORDS = (8, 12, 16)


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


def compress_candidates(lim: dict) -> list[dict]:
    return [{"compress_ctas_per_sm": k, "compress_ticket_chunks": g, "compress_ticket_lead": ld}
            for k, g, ld in itertools.product(range(1, lim["compress"] + 1), TICKET_CHUNKS,
                                              COMPRESS_LEADS)]


def decompress_candidates(lim: dict) -> list[dict]:
    return [{"decompress_ctas_per_sm": k, "decompress_ticket_chunks": g, "decompress_records": r}
            for k, g, r in itertools.product(range(1, lim["decompress"] + 1), TICKET_CHUNKS,
                                             DECOMPRESS_RECORDS) if r >= 2 * g]


def key(cand: dict) -> str:
    """A candidate's name in the timing tables: its settings, field=value, comma-joined."""
    return ",".join(f"{k}={v}" for k, v in sorted(cand.items()))


def tune(cbatch: "fsz.CompressBatch", dbatch: "fsz.DecompressBatch", reps: int = 3) -> dict:
    """Times every schedule candidate on the given batches; returns the best schedule (all
    fsz_schedule fields) and the timings. The schedule is read when a call is made, so each
    candidate is captured into a graph of its own."""
    lim = fsz.fsz_get_schedule_limits()
    results = {"limits": lim, "compress": {}, "decompress": {}}
    try:
        for cand in compress_candidates(lim):
            fsz.fsz_set_schedule_ex(None)
            _check(fsz.fsz_set_schedule_ex(cand))
            g = fsz.fsz_graph_compress_batched(cbatch.table.data_ptr(), len(cbatch.fields),
                                               cbatch.n_total, cbatch.ws.data_ptr(), cbatch.ws_bytes)
            try:
                _time_graph(lambda: fsz.fsz_graph_launch(g, fsz._stream_ptr()), 1)  # warm-up
                results["compress"][key(cand)] = _time_graph(
                    lambda: fsz.fsz_graph_launch(g, fsz._stream_ptr()), reps)
            finally:
                fsz.fsz_graph_destroy(g)
        for cand in decompress_candidates(lim):
            fsz.fsz_set_schedule_ex(None)
            _check(fsz.fsz_set_schedule_ex(cand))
            g = fsz.fsz_graph_decompress_batched(dbatch.table.data_ptr(), len(dbatch.streams),
                                                 dbatch.cap_total, dbatch.ws.data_ptr(), dbatch.ws_bytes)
            try:
                _time_graph(lambda: fsz.fsz_graph_launch(g, fsz._stream_ptr()), 1)
                results["decompress"][key(cand)] = _time_graph(
                    lambda: fsz.fsz_graph_launch(g, fsz._stream_ptr()), reps)
            finally:
                fsz.fsz_graph_destroy(g)
    finally:
        fsz.fsz_set_schedule_ex(None)
    best = fsz.fsz_get_schedule()  # the defaults, then each kernel's fastest candidate
    for kind, cands in (("compress", compress_candidates(lim)), ("decompress", decompress_candidates(lim))):
        best.update(min(cands, key=lambda c: results[kind][key(c)]))
    results["best"] = best
    return results


def _check(st: int) -> None:
    if st != fsz.OK:
        raise fsz.FszError(st, "fsz_set_schedule_ex")


def apply(best: dict | None) -> None:
    """Installs a schedule: a dict of fsz_schedule fields (missing ones keep their values
    in force), or the defaults for None."""
    if best is None:
        _check(fsz.fsz_set_schedule_ex(None))
        return
    _check(fsz.fsz_set_schedule_ex(best))


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
          "note": "fsz_schedule fields: CTAs per SM of the value-range, compression and "
                  "decompression kernels (0 = as many as fit); chunks per ticket; compression's "
                  "ticket lead; decompression's chunks in flight per CTA. Measured by "
                  "paper_2607_15413_gb300.tune on the batched workload (graph launches, median "
                  "of 5); timings keyed by the candidate's settings."}, DEFAULT_TABLE)
    print(json.dumps(res["best"]))


if __name__ == "__main__":
    main()
