"""The launch-schedule table shipped with the package: its shape, that its choice is the
fastest of its own timings, and that it installs through the C ABI (host-side, no GPU)."""
import json
import os

from paper_2607_15413_gb300 import tune


def test_shipped_table_is_consistent():
    with open(tune.DEFAULT_TABLE) as f:
        t = json.load(f)
    assert set(t["best"]) == {"stats", "compress", "decompress"}
    assert all(isinstance(v, int) and 0 <= v <= 64 for v in t["best"].values())
    for k in ("compress", "decompress"):
        ms = {int(c): float(v) for c, v in t["tuning_ms"][k].items()}
        assert ms and all(v > 0.0 for v in ms.values())
        assert t["best"][k] == min(ms, key=ms.get)               # the fastest candidate
        assert max(ms) <= t["limits"][k]                         # every candidate fits
    assert "GB300" in t["device"]


def test_apply_default_installs_the_table(fszlib):
    best = tune.apply_default()
    try:
        with open(tune.DEFAULT_TABLE) as f:
            assert best == json.load(f)["best"]
    finally:
        tune.apply({"stats": 0, "compress": 0, "decompress": 0})
    assert tune.apply_default(os.path.join(os.path.dirname(tune.DEFAULT_TABLE), "missing.json")) is None
