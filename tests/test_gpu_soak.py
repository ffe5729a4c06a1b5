"""A seeded sweep of random fields through the one-field, ablation and batched entry
points, each compared with the CPU oracle byte for byte (GB300 only).

Every case draws, from one seeded generator:
- a size, log-uniform from 1 to 2^10 elements (one case in four) or from 2^10 to 2^23
  (up to 1024 chunks: lookbacks over many windows, wrapping rings), with 1-3 near-cubic
  dims (ragged ends);
- a value class: the workloads' own (sinusoids, particle coordinates, k^-3 GRF, zero
  slabs around an offset) or a degenerate one (piecewise-constant runs, one spike over
  small noise, alternating signs, a ramp on a large offset);
- a bound: REL, or ABS at the same relative magnitude, from 10^-4.5 to 10^-1.5 of the
  range (refusals, e.g. a bound too small for the float32 step, must match the oracle's);
- a launch schedule (CTAs per SM, chunks per ticket, ticket lead, chunks in flight, the
  tickets per CTA below which tickets shrink);
- a feature set (the ablation's switched-off features) for one case in three.

The bar is the parity tests' one: the stream byte for byte, the reconstruction bit for
bit, every value within the bound. The cases are then compressed and decompressed again
as batches of 8 fields in one launch each, each stream equal to the oracle's.
"""
import functools

import numpy as np
import pytest

from paper_2607_15413_gb300 import inputs

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

NCASES = 48
FEATURE_SETS = (0, 2, 4, 6, 3, 7)        # off bits: CROSS 1, CENTER 2, LZ2 4 (CROSS needs CENTER)
CLASSES = ("sin", "particles", "grf", "zero_slabs", "steps", "spike", "alternating", "ramp")


def _field(cls, dims, rng):
    n = int(np.prod(dims))
    seed = int(rng.integers(0, 1 << 30))
    if cls == "sin":
        return inputs.sinusoids(n, seed=seed)
    if cls == "particles":
        return inputs.particles(n, seed=seed, ncenters=max(4, n // 2048))
    if cls == "grf":
        return inputs.grf(dims, seed=seed).ravel()
    if cls == "zero_slabs":
        return inputs.zero_slabs(dims, seed=seed).ravel()
    r = np.random.default_rng(seed)
    if cls == "steps":              # constant runs of random lengths and levels
        lens = r.integers(1, 3000, size=n // 64 + 2)
        levels = r.normal(0.0, 50.0, size=lens.size)
        return np.repeat(levels, lens)[:n].astype(np.float32)
    if cls == "spike":              # the range is one value's: most of the field quantizes to 0
        x = r.normal(0.0, 1.0, n)
        x[int(r.integers(0, n))] = 1.0e5
        return x.astype(np.float32)
    if cls == "alternating":        # sign flips every element: large residuals everywhere
        x = (1.0 + 0.1 * r.standard_normal(n)) * np.where(np.arange(n) % 2 == 0, 1.0, -1.0)
        return (x * 7.5).astype(np.float32)
    if cls == "ramp":               # a ramp on an offset far from zero (cancellation)
        return (3.0e4 + 0.013 * np.arange(n) + r.normal(0.0, 0.2, n)).astype(np.float32)
    raise ValueError(cls)


@functools.lru_cache(maxsize=1)
def soak_cases(seed=2607):
    """The sweep's cases: dicts with x (flat float32), dims, mode, eb, features_off and a
    schedule (its fields; CTAs per SM as counts <= 2, 0 for the default)."""
    rng = np.random.default_rng(seed)
    cases = []
    for i in range(NCASES):
        lo, hi = (0.0, 10.0) if rng.uniform() < 0.25 else (10.0, 23.0)
        n = max(1, int(2.0 ** rng.uniform(lo, hi)))
        ndim = int(rng.integers(1, 4))
        cls = CLASSES[i % len(CLASSES)]
        if cls == "zero_slabs":
            ndim = 3
            n = max(n, 24 * 64)
        dims = inputs.near_cubic_dims(n, ndim)
        if cls == "zero_slabs" and dims[0] < 4:
            dims = (4,) + tuple(dims[1:])
        x = np.ascontiguousarray(_field(cls, dims, rng), dtype=np.float32)
        assert x.size == int(np.prod(dims))
        rel = float(10.0 ** rng.uniform(-4.5, -1.5))
        if rng.uniform() < 0.7:
            mode, eb = 1, rel
        else:
            span = float(x.max()) - float(x.min()) if x.size else 0.0
            mode, eb = 0, rel * (span if span > 0 else 1.0)
        off = int(rng.choice(FEATURE_SETS)) if rng.uniform() < 1 / 3 else 0
        tc = int(rng.integers(1, 5))
        dc = int(rng.integers(1, 5))
        sched = dict(stats_ctas_per_sm=int(rng.integers(0, 3)),
                     compress_ctas_per_sm=int(rng.integers(0, 3)),
                     decompress_ctas_per_sm=int(rng.integers(0, 3)),
                     compress_ticket_chunks=tc, compress_ticket_lead=int(rng.integers(1, 4)),
                     decompress_ticket_chunks=dc,
                     decompress_records=int(rng.integers(2 * dc, 17)),
                     min_tickets_per_cta=int(rng.choice([0, 1, 4])))
        cases.append(dict(index=i, cls=cls, x=x, dims=tuple(int(d) for d in dims), mode=mode,
                          eb=eb, features_off=off, sched=sched))
    return cases


def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch.device("cuda:0")


def _oracle_stream(oracle, c):
    try:
        return oracle.compress(c["x"], c["eb"], c["mode"], dims=c["dims"],
                               features_off=c["features_off"]), 0
    except oracle.OracleError as err:
        return None, err.status


def test_soak_single_field(fszlib, oracle):
    dev = _cuda()
    lim = fszlib.fsz_get_schedule_limits()
    checked = refused = 0
    try:
        for c in soak_cases():
            sched = dict(c["sched"])
            for k, cap in (("stats_ctas_per_sm", lim["stats"]), ("compress_ctas_per_sm", lim["compress"]),
                           ("decompress_ctas_per_sm", lim["decompress"])):
                sched[k] = min(sched[k], cap)
            assert fszlib.fsz_set_schedule_ex(sched) == fszlib.OK, (c["index"], sched)
            tag = (c["index"], c["cls"], c["dims"], c["mode"], c["eb"], c["features_off"])
            ref, status = _oracle_stream(oracle, c)
            xd = torch.from_numpy(c["x"]).to(dev)
            if ref is None:                      # the device must refuse it the same way
                with pytest.raises(fszlib.FszError) as e:
                    fszlib.compress(xd, c["eb"], c["mode"], shape=c["dims"],
                                    features_off=c["features_off"])
                assert e.value.status == status, tag
                refused += 1
                continue
            sb, nb = fszlib.compress(xd, c["eb"], c["mode"], shape=c["dims"],
                                     features_off=c["features_off"])
            got = sb.cpu().numpy().tobytes()
            assert len(got) == len(ref), tag
            if got != ref:
                a, b = np.frombuffer(got, np.uint8), np.frombuffer(ref, np.uint8)
                raise AssertionError(f"{tag}: stream differs first at byte {int(np.nonzero(a != b)[0][0])}")
            yref = oracle.decompress(ref)
            y = fszlib.decompress(sb, n=c["x"].size, any_stream=True).cpu().numpy()
            assert np.array_equal(y.view(np.uint32), yref.view(np.uint32)), tag
            if c["x"].size:
                p = oracle.params_for(c["x"], c["mode"], c["eb"])
                assert np.abs(c["x"].astype(np.float64) - y.astype(np.float64)).max() <= p.eb, tag
            checked += 1
    finally:
        fszlib.fsz_set_schedule_ex(None)
    assert checked >= NCASES * 3 // 4 and checked + refused == NCASES


def test_soak_batches(fszlib, oracle):
    dev = _cuda()
    cases = [c for c in soak_cases() if not (c["features_off"] & 1)]  # the batched decoder is the full method's
    refs = [_oracle_stream(oracle, c) for c in cases]
    for b0 in range(0, len(cases), 8):
        group = list(zip(cases[b0:b0 + 8], refs[b0:b0 + 8]))
        fields = [(torch.from_numpy(c["x"]).to(dev), c["dims"], c["mode"], c["eb"], c["features_off"])
                  for c, _ in group]
        cb = fszlib.CompressBatch(fields, dev)
        assert cb.run() == fszlib.OK
        st, per = cb.status()
        sizes = cb.sizes.cpu().tolist()
        ok = []
        for i, (c, (ref, status)) in enumerate(group):
            assert per[i] == status, (c["index"], per[i], status)
            if ref is None:
                continue
            s = cb.stream(i, sizes)
            assert s.cpu().numpy().tobytes() == ref, c["index"]
            ok.append((c, ref, s))
        if not ok:
            continue
        db = fszlib.DecompressBatch([s for _, _, s in ok], [c["x"].size for c, _, _ in ok], dev)
        assert db.run() == fszlib.OK
        st, per = db.status()
        assert st == fszlib.OK and all(p == 0 for p in per)
        for i, (c, ref, _) in enumerate(ok):
            yref = oracle.decompress(ref)
            assert np.array_equal(db.output(i).cpu().numpy().view(np.uint32), yref.view(np.uint32)), c["index"]
