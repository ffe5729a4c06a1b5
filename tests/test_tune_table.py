"""The launch-schedule table shipped with the package: its shape, that its choice is the
fastest of its own timings, and that it installs through the C ABI; the C ABI's range
checks on a schedule (host-side, no GPU)."""
import ctypes
import json
import os

import pytest

from paper_2607_15413_gb300 import fsz, tune


def test_shipped_table_is_consistent():
    with open(tune.DEFAULT_TABLE) as f:
        t = json.load(f)
    assert set(t["best"]) == set(fsz.SCHEDULE_FIELDS)
    assert all(isinstance(v, int) and 0 <= v <= 64 for v in t["best"].values())
    lim = t["limits"]
    for kind, cands in (("compress", tune.compress_candidates(lim)),
                        ("decompress", tune.decompress_candidates(lim))):
        ms = {k: float(v) for k, v in t["tuning_ms"][kind].items()}
        assert set(ms) == {tune.key(c) for c in cands}               # the whole search space
        assert all(v > 0.0 for v in ms.values())
        fastest = min(cands, key=lambda c: ms[tune.key(c)])
        assert all(t["best"][k] == v for k, v in fastest.items())    # the fastest candidate
    assert len(t["tuning_ms"]["compress"]) >= 6
    assert "GB300" in t["device"]


def test_apply_default_installs_the_table(fszlib):
    best = tune.apply_default()
    try:
        with open(tune.DEFAULT_TABLE) as f:
            assert best == json.load(f)["best"]
        assert fsz.fsz_get_schedule() == best
    finally:
        tune.apply(None)
    assert tune.apply_default(os.path.join(os.path.dirname(tune.DEFAULT_TABLE), "missing.json")) is None


DEFAULTS = {"stats_ctas_per_sm": 0, "compress_ctas_per_sm": 0, "decompress_ctas_per_sm": 0,
            "compress_ticket_chunks": 2, "compress_ticket_lead": 2, "decompress_ticket_chunks": 4,
            "decompress_records": 16, "min_tickets_per_cta": 4}


def test_schedule_round_trip_and_defaults(fszlib):
    try:
        assert fsz.fsz_set_schedule_ex(None) == fsz.OK
        assert fsz.fsz_get_schedule() == DEFAULTS
        want = {"stats_ctas_per_sm": 3, "compress_ctas_per_sm": 1, "decompress_ctas_per_sm": 2,
                "compress_ticket_chunks": 4, "compress_ticket_lead": 3, "decompress_ticket_chunks": 1,
                "decompress_records": 2, "min_tickets_per_cta": 0}
        assert fsz.fsz_set_schedule_ex(want) == fsz.OK
        assert fsz.fsz_get_schedule() == want
        # the three-count call changes the CTA counts only
        assert fsz.fsz_set_schedule(0, 2, 1) == fsz.OK
        got = fsz.fsz_get_schedule()
        assert got == dict(want, stats_ctas_per_sm=0, compress_ctas_per_sm=2, decompress_ctas_per_sm=1)
    finally:
        fsz.fsz_set_schedule_ex(None)


@pytest.mark.parametrize("bad", [
    {"compress_ticket_chunks": 0}, {"compress_ticket_chunks": 5}, {"compress_ticket_lead": 0},
    {"compress_ticket_lead": 4}, {"decompress_ticket_chunks": 0}, {"decompress_ticket_chunks": 5},
    {"decompress_ticket_chunks": 4, "decompress_records": 7}, {"decompress_records": 17},
    {"decompress_records": 1}, {"stats_ctas_per_sm": 65}, {"compress_ctas_per_sm": 65},
    {"min_tickets_per_cta": 65}])
def test_schedule_out_of_range_is_refused(fszlib, bad):
    try:
        assert fsz.fsz_set_schedule_ex(None) == fsz.OK
        assert fsz.fsz_set_schedule_ex(bad) == fsz.ERR_INVALID_ARG
        assert fsz.fsz_get_schedule() == DEFAULTS                    # unchanged
        sc = fsz.FszSchedule(*[bad.get(k, DEFAULTS[k]) for k in fsz.SCHEDULE_FIELDS])  # the raw call
        assert fszlib.lib().fsz_set_schedule_ex(ctypes.byref(sc)) == fsz.ERR_INVALID_ARG
    finally:
        fsz.fsz_set_schedule_ex(None)
