"""Switched-off features (the ablation of Sec. 6.4) on the CUDA path vs the CPU oracle.

Every valid feature set, byte for byte on the stream and bit for bit on the
reconstruction; one-call and batched entry points; the decoder's checks of a stream's
feature word.
"""
import numpy as np
import pytest

from paper_2607_15413_gb300 import inputs

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

VALID = [0, 2, 4, 6, 3, 7]          # off bits: CROSS 1, CENTER 2, LZ2 4 (CROSS needs CENTER)


def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch.device("cuda:0")


FIELDS = {
    "offset": lambda n, s: (10.0 * inputs.sinusoids(n, seed=s) + 280.0).astype(np.float32),
    "particles": lambda n, s: inputs.particles(n, seed=s, ncenters=max(4, n // 2048)),
    "zero_slabs": lambda n, s: inputs.zero_slabs((max(24, -(-n // 4096)), 64, 64), seed=s).ravel()[:n],
}


def _parity(fszlib, oracle, x, rel, off):
    dev = _cuda()
    ref = oracle.compress(x, rel, oracle.REL, features_off=off)
    xd = torch.from_numpy(np.ascontiguousarray(x)).to(dev)
    sb, nb = fszlib.compress(xd, rel, fszlib.EB_REL, features_off=off)
    got = sb.cpu().numpy().tobytes()
    assert len(got) == len(ref)
    if got != ref:
        a, b = np.frombuffer(got, np.uint8), np.frombuffer(ref, np.uint8)
        raise AssertionError(f"stream differs first at byte {int(np.nonzero(a != b)[0][0])}")
    yref = oracle.decompress(ref).view(np.uint32)
    y = fszlib.decompress(sb, n=x.size, any_stream=True).cpu().numpy()
    assert np.array_equal(y.view(np.uint32), yref)
    if off & oracle.OFF_CROSS:       # the full method's decoder refuses these streams
        with pytest.raises(fszlib.FszError) as e:
            fszlib.decompress(sb, n=x.size)
        assert e.value.status == fszlib.ERR_INVALID_ARG
    else:                            # and decodes the others
        y = fszlib.decompress(sb, n=x.size).cpu().numpy()
        assert np.array_equal(y.view(np.uint32), yref)
    return ref


@pytest.mark.parametrize("off", VALID)
@pytest.mark.parametrize("field", sorted(FIELDS))
def test_feature_sets_match_the_oracle(fszlib, oracle, field, off):
    x = FIELDS[field](4096 * 24, 3)
    for rel in (1e-2, 1e-3):
        ref = _parity(fszlib, oracle, x, rel, off)
        assert oracle.read_preamble(ref)["features_off"] == off


@pytest.mark.parametrize("n", [1, 33, 257, 8193, 3 * 8192 + 17])
def test_feature_sets_ragged(fszlib, oracle, n):
    x = FIELDS["offset"](n, n % 5)
    for off in (3, 7, 6):
        _parity(fszlib, oracle, x, 1e-3, off)


def test_ablation_ladder_on_a_grf(fszlib, oracle):
    """Base, +Cross, +Cent., +LZ2 on a 64^3 k^-3 GRF with an offset (the structured,
    offset-heavy case of Table 7): every step matches the oracle and raises CR."""
    x = (10.0 * inputs.grf((64, 64, 64), seed=2) + 280.0).astype(np.float32).ravel()
    sizes = [len(_parity(fszlib, oracle, x, 1e-4, off)) for _, off in oracle.ABLATION]
    assert sizes[1] < sizes[0] and sizes[2] <= sizes[1] and sizes[3] <= sizes[2]


def test_batched_fields_keep_their_own_features(fszlib, oracle):
    dev = _cuda()
    xs = [FIELDS["offset"](5000 + 997 * k, k) for k in range(6)]
    offs = [0, 7, 3, 6, 2, 4]
    fields = [(torch.from_numpy(x).to(dev), (x.size,), fszlib.EB_REL, 1e-3, off)
              for x, off in zip(xs, offs)]
    b = fszlib.CompressBatch(fields, device=dev)
    assert b.run() == fszlib.OK
    st, per = b.status()
    assert st == fszlib.OK and all(p == 0 for p in per)
    for i, (x, off) in enumerate(zip(xs, offs)):
        got = b.stream(i).cpu().numpy().tobytes()
        assert got == oracle.compress(x, 1e-3, oracle.REL, features_off=off)


def test_invalid_feature_sets_are_refused(fszlib):
    dev = _cuda()
    x = torch.zeros(1000, device=dev)
    for off in (1, 5, 8, 0x100):
        with pytest.raises(fszlib.FszError) as e:
            fszlib.compress(x, 1e-3, fszlib.EB_REL, features_off=off)
        assert e.value.status == fszlib.ERR_INVALID_ARG
    # in a batch the bad field reports INVALID_ARG, the good one compresses
    y = torch.linspace(0, 1, 3000, device=dev)
    b = fszlib.CompressBatch([(y, (3000,), fszlib.EB_REL, 1e-3, 1), (y, (3000,), fszlib.EB_REL, 1e-3, 0)],
                             device=dev)
    assert b.run() == fszlib.OK
    st, per = b.status()
    assert per[0] == fszlib.ERR_INVALID_ARG and per[1] == 0


def _decode_status(fszlib, stream: bytes, n: int) -> int:
    dev = _cuda()
    buf = torch.zeros(len(stream) + 64, dtype=torch.uint8, device=dev)
    buf[: len(stream)] = torch.from_numpy(np.frombuffer(stream, np.uint8).copy()).to(dev)
    out = torch.zeros(max(n, 16), dtype=torch.float32, device=dev)
    ws = fszlib.Workspace(out.numel(), dev)
    sp = torch.cuda.current_stream().cuda_stream
    assert fszlib.fsz_decompress(buf.data_ptr(), len(stream), out.data_ptr(), out.numel(), ws.ptr,
                                 ws.bytes, sp) == fszlib.OK
    return fszlib.fsz_check(ws.ptr, sp)


def test_decoder_checks_the_feature_word(fszlib, oracle):
    x = FIELDS["offset"](40000, 1)
    s = oracle.compress(x, 1e-4, oracle.REL)
    h0 = np.frombuffer(s[64: 64 + 8 * ((x.size + 255) // 256)], np.uint8)[::8]
    assert np.any(h0 & 0x80) and np.any(h0 & 0x40)
    assert _decode_status(fszlib, s, x.size) == fszlib.OK
    for off in (4, 2, 1, 8, 5):
        b = bytearray(s)
        b[52:56] = int(off).to_bytes(4, "little")
        assert _decode_status(fszlib, bytes(b), x.size) == fszlib.ERR_CORRUPT, off
        assert oracle.decompress_status(bytes(b)) == oracle.ERR_CORRUPT


# ---------------------------------------------------------------- multipass evaluation

@pytest.mark.parametrize("n", [1, 255, 257, 8193, 4096 * 24, 3 * 8192 + 17])
@pytest.mark.parametrize("field", sorted(FIELDS))
def test_multipass_stream_is_the_single_pass_stream(fszlib, oracle, field, n):
    """Sec. 6.3: the multipass evaluation produces identical streams; its four cost arrays
    are the oracle's four-pass costs (one residual pass per variant) tile by tile."""
    dev = _cuda()
    x = FIELDS[field](n, 7)
    xd = torch.from_numpy(np.ascontiguousarray(x)).to(dev)
    for rel in (1e-2, 1e-3):
        sb, nb, costs = fszlib.compress_multipass(xd, rel, fszlib.EB_REL)
        ref = oracle.compress(x, rel, oracle.REL)
        assert sb.cpu().numpy().tobytes() == ref
        p = oracle.params_for(x, oracle.REL, rel)
        T = (x.size + 255) // 256
        xp = np.zeros(T * 256, np.float32)
        xp[: x.size] = x
        q = oracle.quantize(xp, p.r)
        c = costs.cpu().numpy().view(np.uint32)
        for t in sorted({0, T // 2, T - 1} | set(range(0, T, max(1, T // 17)))):
            d = xp[256 * t: 256 * t + 256]
            C, _ = oracle.tile_costs(q[256 * t: 256 * t + 256], oracle.tile_mu(d, p.r), four_pass=True)
            assert list(c[:, t]) == [int(v) for v in C], t


def test_multipass_refuses_missing_or_misaligned_costs(fszlib):
    dev = _cuda()
    x = torch.linspace(0, 1, 5000, device=dev)
    ws = fszlib.Workspace(5000, dev)
    out = torch.empty(fszlib.fsz_compress_bound(5000), dtype=torch.uint8, device=dev)
    costs = torch.zeros(4 * 20 + 4, dtype=torch.int32, device=dev)
    sp = torch.cuda.current_stream().cuda_stream
    L = fszlib.lib()
    args = (x.data_ptr(), fszlib.make_dims((5000,)), 1, 1e-3, out.data_ptr(), out.numel(), None)
    assert L.fsz_compress_multipass(*args, None, ws.ptr, ws.bytes, sp) == fszlib.ERR_INVALID_ARG
    assert L.fsz_compress_multipass(*args, costs.data_ptr() + 4, ws.ptr, ws.bytes, sp) == fszlib.ERR_ALIGN


# ---------------------------------------------------------------- adaptive pre-zero (Sec. 3.1)

def _sparse(n, seed):
    """Mostly exact zeros (about 99 %), a smooth band elsewhere: a stream of CR above 100."""
    x = np.zeros(n, np.float32)
    band = inputs.sinusoids(n // 128, seed=seed) + np.float32(3.0)
    x[n // 2: n // 2 + band.size] = band
    return x


def _zero_tiles(stream: bytes, n: int) -> np.ndarray:
    T = (n + 255) // 256
    h = np.frombuffer(stream[64: 64 + 8 * T], np.uint64)
    return (h & np.uint64(0x1F1F1F1F1F1F1F5F)) == 0


@pytest.mark.parametrize("field", ["sparse", "zero_slabs", "offset"])
def test_prezeroed_decode_skips_exactly_the_zero_tiles(fszlib, oracle, field):
    dev = _cuda()
    n = 4096 * 24 + 77
    x = _sparse(n, 2) if field == "sparse" else FIELDS[field](n, 2)
    ref = oracle.compress(x, 1e-3, oracle.REL)
    sb = torch.from_numpy(np.frombuffer(ref, np.uint8).copy()).to(dev)
    yref = oracle.decompress(ref).view(np.uint32)
    # into zeros: identical to the full decode
    y = fszlib.decompress(sb, n=n, out_is_zero=True).cpu().numpy()
    assert np.array_equal(y.view(np.uint32), yref)
    # into a NaN-filled buffer: the all-zero tiles are not written, all others are
    out = torch.full((n,), float("nan"), device=dev)
    ws = fszlib.Workspace(n, dev)
    sp = torch.cuda.current_stream().cuda_stream
    assert fszlib.lib().fsz_decompress_prezeroed(sb.data_ptr(), sb.numel(), out.data_ptr(), n, ws.ptr,
                                                 ws.bytes, sp) == fszlib.OK
    assert fszlib.fsz_check(ws.ptr, sp) == fszlib.OK
    got = out.cpu().numpy()
    zt = np.repeat(_zero_tiles(ref, n), 256)[:n]
    assert np.all(np.isnan(got[zt]))
    assert np.array_equal(got[~zt].view(np.uint32), yref[~zt])
    if field == "sparse":
        assert zt.mean() > 0.9 and 4 * n / len(ref) > 100
