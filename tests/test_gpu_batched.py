"""Batched compression and decompression (one persistent launch for many fields) vs
the one-field entry points and the CPU oracle, through the C ABI (GB300 only).

Each field's stream from the batch must equal, byte for byte, fsz_compress of that
field alone and the oracle's stream; decompressed floats must match bit for bit.
"""
import numpy as np
import pytest

from paper_2607_15413_gb300 import inputs

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def _dev():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch.device("cuda:0")


def _mixed_fields(seed=0):
    rng = np.random.default_rng(seed)
    out = []
    sizes = [0, 1, 3, 255, 256, 257, 4097, 8192, 8193, 40000, 70001, 300000, 1 << 20]
    for i, n in enumerate(sizes):
        kind = i % 3
        if kind == 0:
            x = inputs.sinusoids(n, seed=i) if n else np.zeros(0, np.float32)
        elif kind == 1:
            x = inputs.particles(n, seed=i, ncenters=max(4, n // 2048)) if n else np.zeros(0, np.float32)
        else:
            x = (inputs.sinusoids(n, seed=i) + np.float32(280.0)).astype(np.float32)
        mode = 0 if i % 4 == 3 else 1
        eb = float(rng.choice([1e-2, 1e-3, 1e-4])) if mode == 1 else 0.05
        out.append((x, (n,), mode, eb))
    g = inputs.grf((24, 40, 56), seed=7)
    out.append((g, g.shape, 1, 1e-3))
    z = inputs.zero_slabs((30, 20, 64), seed=8)
    out.append((z, z.shape, 1, 1e-4))
    return out


def test_batched_matches_single_and_oracle(fszlib, oracle):
    dev = _dev()
    host = _mixed_fields()
    fields = [(torch.from_numpy(np.ascontiguousarray(x).ravel()).to(dev), shape, mode, eb)
              for x, shape, mode, eb in host]
    batch = fszlib.CompressBatch(fields, dev)
    assert batch.run() == fszlib.OK
    st, per = batch.status()
    # the oracle's status per field (a tiny field with a large offset can be refused)
    refs, want = [], []
    for x, shape, mode, eb in host:
        try:
            refs.append(oracle.compress(np.ascontiguousarray(x).ravel(), eb, mode, dims=shape))
            want.append(0)
        except oracle.OracleError as err:
            refs.append(None)
            want.append(err.status)
    assert per == want
    assert want.count(0) >= len(want) - 2
    sizes = batch.sizes.cpu().tolist()
    streams, keep = [], []
    for i, ((x, shape, mode, eb), (xd, *_)) in enumerate(zip(host, fields)):
        if refs[i] is None:
            continue
        got = batch.stream(i, sizes).cpu().numpy().tobytes()
        assert got == refs[i], f"field {i}: batched stream differs from the oracle"
        one, nb = fszlib.compress(xd, eb, mode, shape=shape)
        assert one.cpu().numpy().tobytes() == refs[i], f"field {i}: single-field stream differs"
        streams.append(batch.stream(i, sizes).clone())
        keep.append(i)
    # batched decompression of every valid stream
    dbatch = fszlib.DecompressBatch(streams, [fields[i][0].numel() for i in keep], dev)
    assert dbatch.run() == fszlib.OK
    st, per = dbatch.status()
    assert st == fszlib.OK and per == [0] * len(keep)
    for j, i in enumerate(keep):
        y = dbatch.output(j).cpu().numpy()
        ref = oracle.decompress(refs[i])
        assert np.array_equal(y.view(np.uint32), ref.view(np.uint32)), f"field {i}"


def test_batched_errors_stay_per_field(fszlib, oracle):
    dev = _dev()
    good = inputs.sinusoids(50000, seed=1)
    bad = good.copy()
    bad[123] = np.nan
    off = (good + np.float32(1e4)).astype(np.float32)
    fields = [(torch.from_numpy(a).to(dev), (a.size,), 1, eb)
              for a, eb in ((good, 1e-3), (bad, 1e-3), (off, 1e-7), (good, 1e-4))]
    batch = fszlib.CompressBatch(fields, dev)
    assert batch.run() == fszlib.OK
    st, per = batch.status()
    assert per == [0, fszlib.ERR_NONFINITE, fszlib.ERR_EB_TOO_SMALL, 0]
    assert st in (fszlib.ERR_NONFINITE, fszlib.ERR_EB_TOO_SMALL)
    sizes = batch.sizes.cpu().tolist()
    for i, eb in ((0, 1e-3), (3, 1e-4)):
        assert batch.stream(i, sizes).cpu().numpy().tobytes() == oracle.compress(good, eb, 1)


def test_graph_replays_batched_calls(fszlib, oracle):
    dev = _dev()
    def accepted(f):
        try:
            oracle.compress(np.ascontiguousarray(f[0]).ravel(), f[3], f[2], dims=f[1])
            return f[0].size > 0
        except oracle.OracleError:
            return False
    host = [f for f in _mixed_fields(seed=3) if accepted(f)][:8]
    fields = [(torch.from_numpy(np.ascontiguousarray(x).ravel()).to(dev), shape, mode, eb)
              for x, shape, mode, eb in host]
    batch = fszlib.CompressBatch(fields, dev)
    for rep in range(3):  # the same graph three times; inputs change in between
        batch.arena.zero_()
        assert batch.launch_graph() == fszlib.OK
        st, per = batch.status()
        assert st == fszlib.OK
        sizes = batch.sizes.cpu().tolist()
        for i, ((x, shape, mode, eb), (xd, *_)) in enumerate(zip(host, fields)):
            xs = np.ascontiguousarray(x).ravel() * np.float32(1 + rep)
            assert batch.stream(i, sizes).cpu().numpy().tobytes() == oracle.compress(
                xs.astype(np.float32), eb, mode, dims=shape)
        for xd, *_ in fields:
            xd.mul_((rep + 2) / (rep + 1))   # next replay compresses x * (rep + 2)
    streams = [batch.stream(i, sizes).clone() for i in range(len(fields))]
    dbatch = fszlib.DecompressBatch(streams, [f[0].numel() for f in fields], dev)
    for _ in range(2):
        dbatch.arena.zero_()
        assert dbatch.launch_graph() == fszlib.OK
        assert dbatch.status()[0] == fszlib.OK
        for i in range(len(fields)):
            ref = oracle.decompress(streams[i].cpu().numpy().tobytes())
            assert np.array_equal(dbatch.output(i).cpu().numpy().view(np.uint32), ref.view(np.uint32))


# These fields are a few hundred chunks at most, so under the default min_tickets_per_cta
# every launch here takes 1-chunk tickets; the entries with min_tickets_per_cta=0 keep the
# multi-chunk tickets they name.
SCHEDULES = [
    None,                                                                  # the defaults
    dict(min_tickets_per_cta=0),                                           # default tickets held
    dict(stats_ctas_per_sm=1, compress_ctas_per_sm=1, decompress_ctas_per_sm=1),
    dict(stats_ctas_per_sm=2, compress_ctas_per_sm=2, decompress_ctas_per_sm=2),
    dict(compress_ticket_chunks=1, compress_ticket_lead=1, decompress_ticket_chunks=1,
         decompress_records=2),                                            # smallest items
    dict(compress_ticket_chunks=4, compress_ticket_lead=3, decompress_ticket_chunks=4,
         decompress_records=8, min_tickets_per_cta=0),                     # largest items
    dict(compress_ctas_per_sm=1, compress_ticket_chunks=3, compress_ticket_lead=1,
         decompress_ctas_per_sm=1, decompress_ticket_chunks=2, decompress_records=16,
         min_tickets_per_cta=0),
    dict(compress_ticket_chunks=4, decompress_ticket_chunks=4, decompress_records=8,
         min_tickets_per_cta=1),                                           # partly shrunk
]


@pytest.mark.parametrize("sched", SCHEDULES)
def test_schedules_give_identical_streams(fszlib, oracle, sched):
    """Every schedule (CTAs per SM, chunks per ticket, ticket lead, chunks in flight, the
    tickets per CTA below which tickets shrink) gives the oracle's stream and
    reconstruction, for one field (with a ragged end) and for a batch of fields of several
    sizes, some a few chunks long."""
    dev = _dev()
    lim = fszlib.fsz_get_schedule_limits()
    assert lim["compress"] >= 1 and lim["decompress"] >= 1 and lim["sms"] > 0
    x = inputs.particles(3 * (1 << 20) + 77, seed=9, ncenters=500)
    ref = oracle.compress(x, 1e-4, 1)
    rng = np.random.default_rng(21)
    fields = [(torch.from_numpy(inputs.sinusoids(int(n), seed=int(n) % 97)).to(dev), (int(n),),
               fszlib.EB_REL, rel)
              for n, rel in zip(rng.integers(1, 40 * 8192, 12), [1e-2, 1e-3, 1e-4] * 4)]
    try:
        assert fszlib.fsz_set_schedule_ex(sched) == fszlib.OK
        sb, nb = fszlib.compress(torch.from_numpy(x).to(dev), 1e-4, 1)
        assert sb.cpu().numpy().tobytes() == ref
        y = fszlib.decompress(sb, n=x.size).cpu().numpy()
        assert np.array_equal(y.view(np.uint32), oracle.decompress(ref).view(np.uint32))
        cb = fszlib.CompressBatch(fields, dev)
        assert cb.run() == fszlib.OK and cb.status()[0] == fszlib.OK
        sizes = cb.sizes.cpu().tolist()
        streams = [cb.stream(i, sizes) for i in range(len(fields))]
        for i, (f, _, _, rel) in enumerate(fields):
            assert streams[i].cpu().numpy().tobytes() == oracle.compress(f.cpu().numpy(), rel, 1), i
        db = fszlib.DecompressBatch(streams, [f.numel() for f, *_ in fields], dev)
        assert db.run() == fszlib.OK and db.status()[0] == fszlib.OK
        for i, (f, *_) in enumerate(fields):
            ref_i = oracle.decompress(streams[i].cpu().numpy().tobytes())
            assert np.array_equal(db.output(i).cpu().numpy().view(np.uint32), ref_i.view(np.uint32)), i
    finally:
        fszlib.fsz_set_schedule_ex(None)


def test_config4_all_512_fields_against_the_oracle(fszlib, oracle):
    """The batched workload itself: 512 fields (seed 3; log-uniform 64 KiB - 64 MiB, 1-3-D,
    40 % k^-3 GRF / 40 % particle-like / 20 % zero-slab, REL from {1e-2, 1e-3, 1e-4}) in one
    compression launch and one decompression launch. Every field's stream equals the oracle's
    byte for byte and every reconstruction the oracle decoder's bit for bit (host threads run
    the oracle); every stream also equals fsz_compress of that field alone."""
    import concurrent.futures as cf
    import os
    dev = _dev()
    specs = inputs.field_mix_specs(512, seed=3)
    fields = [(inputs.make_field(sp, device="cuda").contiguous(), sp["dims"], 1, sp["rel"])
              for sp in specs]
    batch = fszlib.CompressBatch(fields, dev)
    assert batch.run() == fszlib.OK
    st, per = batch.status()
    assert st == fszlib.OK, per
    sizes = batch.sizes.cpu().tolist()
    streams = [batch.stream(i, sizes).clone() for i in range(len(fields))]
    dbatch = fszlib.DecompressBatch(streams, [f[0].numel() for f in fields], dev)
    assert dbatch.run() == fszlib.OK and dbatch.status()[0] == fszlib.OK

    def check(i, x, dims, rel, got, y):
        ref = oracle.compress(x, rel, oracle.REL, dims=dims)
        if got != ref:
            return f"field {i}: stream differs from the oracle"
        if not np.array_equal(y.view(np.uint32), oracle.decompress(ref).view(np.uint32)):
            return f"field {i}: reconstruction differs from the oracle decoder"
        return None

    bad = []
    with cf.ThreadPoolExecutor(max_workers=max(2, min(16, os.cpu_count() or 2))) as ex:
        futs = []
        for i, (xd, dims, mode, rel) in enumerate(fields):
            one, nb = fszlib.compress(xd, rel, mode, shape=dims)
            assert torch.equal(one, streams[i]), f"field {i}: batched != alone"
            futs.append(ex.submit(check, i, xd.cpu().numpy(), dims, rel,
                                  streams[i].cpu().numpy().tobytes(), dbatch.output(i).cpu().numpy()))
            if len(futs) >= 48:   # bound the host copies in flight
                bad += [m for m in (f.result() for f in futs) if m]
                futs = []
        bad += [m for m in (f.result() for f in futs) if m]
    assert not bad, bad[:5]
