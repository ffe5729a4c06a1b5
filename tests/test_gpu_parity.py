"""CUDA path vs the CPU oracle, through the C ABI (GB300 only).

The bar is bit-exact: the compressed stream byte for byte, the decompressed floats
bit for bit (the tolerance is 0). Small, ragged and full-size fields (the 512^3 fields
at all three bounds, the 2^28-element particle array) are compared whole. The field past
2^32 elements is compared on sampled tiles the oracle encodes one by one, and on every
element through properties that hold at any size.
"""
import numpy as np
import pytest

from paper_2607_15413_gb300 import inputs

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch.device("cuda:0")


def gpu_roundtrip(fszlib, x: np.ndarray, eb, mode, shape=None):
    dev = _cuda()
    xd = torch.from_numpy(np.ascontiguousarray(x, np.float32).ravel()).to(dev)
    sb, nb = fszlib.compress(xd, eb, mode, shape=shape if shape is not None else (x.size,))
    y = fszlib.decompress(sb, n=x.size)
    return sb.cpu().numpy().tobytes(), y.cpu().numpy()


def assert_full_parity(fszlib, oracle, x, eb, mode=1, shape=None):
    shape = shape if shape is not None else (x.size,)
    try:
        ref = oracle.compress(x.ravel(), eb, mode, dims=shape)
    except oracle.OracleError as err:
        # The oracle refuses this field (e.g. the bound is too small for the data's
        # magnitude): the device must record the same status.
        assert _status_of_compress(fszlib, np.ascontiguousarray(x, np.float32).ravel(), eb,
                                   mode) == err.status
        return None
    got, y = gpu_roundtrip(fszlib, x, eb, mode, shape)
    assert len(got) == len(ref), (len(got), len(ref))
    if got != ref:
        a = np.frombuffer(got, np.uint8)
        b = np.frombuffer(ref, np.uint8)
        first = int(np.nonzero(a != b)[0][0])
        raise AssertionError(f"stream differs first at byte {first} of {len(ref)}")
    yref = oracle.decompress(ref)
    assert np.array_equal(y.view(np.uint32), yref.view(np.uint32))
    if x.size:
        p = oracle.params_for(x, mode, eb)
        assert np.abs(x.astype(np.float64).ravel() - y.astype(np.float64)).max() <= p.eb
    return ref


def test_config1_sinusoids_full_parity(fszlib, oracle):
    x = inputs.sinusoids(1 << 20, seed=0)
    ref = assert_full_parity(fszlib, oracle, x, 1e-3)
    assert len(ref) < x.nbytes


GENS = {
    "sin": lambda n, s: inputs.sinusoids(n, seed=s),
    "particles": lambda n, s: inputs.particles(n, seed=s, ncenters=max(4, n // 2048)),
    "offset": lambda n, s: (inputs.sinusoids(n, seed=s) + np.float32(280.0)).astype(np.float32),
}


@pytest.mark.parametrize("n", [1, 2, 3, 4, 5, 31, 32, 33, 255, 256, 257, 1000, 4097, 8191, 8192,
                               8193, 65539, 3 * 8192 + 17])
@pytest.mark.parametrize("gen", sorted(GENS))
def test_ragged_sizes(fszlib, oracle, n, gen):
    x = GENS[gen](n, n % 7)
    for rel in (1e-2, 1e-4):
        assert_full_parity(fszlib, oracle, x, rel)


@pytest.mark.parametrize("nchunks", [31, 33, 64, 70, 161])
def test_many_chunks_lookback(fszlib, oracle, nchunks):
    # More than 32 chunks: the lookback walks several windows of 32 predecessors.
    n = nchunks * 8192 - 1234
    assert_full_parity(fszlib, oracle, inputs.particles(n, seed=nchunks, ncenters=64), 1e-4)


def test_3d_shapes(fszlib, oracle):
    x = inputs.grf((40, 48, 64), seed=4)
    for rel in (1e-2, 1e-3, 1e-4):
        assert_full_parity(fszlib, oracle, x, rel, shape=x.shape)
    z = inputs.zero_slabs((30, 40, 70), seed=5)
    for rel in (1e-2, 1e-3, 1e-4):
        assert_full_parity(fszlib, oracle, z, rel, shape=z.shape)


def test_abs_mode_and_special_fields(fszlib, oracle):
    rng = np.random.default_rng(1)
    assert_full_parity(fszlib, oracle, rng.normal(0, 1, 50000).astype(np.float32), 0.01, mode=0)
    assert_full_parity(fszlib, oracle, np.full(70000, 3.25, np.float32), 1e-3)       # constant
    assert_full_parity(fszlib, oracle, np.zeros(70000, np.float32), 1e-3)            # all zero
    lin = (1000.0 + 0.37 * np.arange(90000)).astype(np.float32)                     # linear ramp
    assert_full_parity(fszlib, oracle, lin, 1e-5)
    big = (1.0e4 + rng.normal(0, 30.0, 120000)).astype(np.float32)                  # offset
    assert_full_parity(fszlib, oracle, big, 1e-3)
    tiny = (rng.normal(0, 1, 30000) * 1e-20).astype(np.float32)                     # tiny values
    assert_full_parity(fszlib, oracle, tiny, 1e-2)


def test_adversarial_midpoints(fszlib, oracle):
    A = np.float32(37.25)
    for eb in (1e-1, 7.77e-4):
        p = oracle.params(oracle.ABS, eb, -float(A), float(A))
        k = np.arange(-p.Q, p.Q + 1, max(1, p.Q // 20000), dtype=np.int64)
        mid = ((k.astype(np.float64) + 0.5) * float(np.float32(p.s))).astype(np.float32)
        x = np.concatenate([mid, np.nextafter(mid, np.float32(np.inf)),
                            np.nextafter(mid, np.float32(-np.inf)), np.array([A, -A], np.float32)])
        x = x[np.abs(x) <= A].astype(np.float32)
        assert_full_parity(fszlib, oracle, x, eb, mode=0)


def test_second_margin_tier(fszlib, oracle):
    """Fields the first margin tier (eps <= 2^-4) refuses and the second (eps <= 2^-1)
    accepts: a large offset over a small range, and bin midpoints +-1 ulp over the whole
    range of q of a second-tier bound; a bound beyond the second tier is refused on the
    device as by the oracle."""
    rng = np.random.default_rng(9)
    x = (1.0e4 + rng.normal(0, 30.0, 150000)).astype(np.float32)
    for rel in (1e-4, 3e-5):
        assert oracle.params_for(x, oracle.REL, rel).Q > 174761
        assert_full_parity(fszlib, oracle, x, rel)
    assert _status_of_compress(fszlib, x, 1e-5) == fszlib.ERR_EB_TOO_SMALL
    A = np.float32(1.0)
    eb = 1.0 / 700000.0
    p = oracle.params(oracle.ABS, eb, -float(A), float(A))
    assert p.Q > 174761
    k = np.arange(-p.Q, p.Q + 1, max(1, p.Q // 30000), dtype=np.int64)
    mid = ((k.astype(np.float64) + 0.5) * float(np.float32(p.s))).astype(np.float32)
    xm = np.concatenate([mid, np.nextafter(mid, np.float32(np.inf)),
                         np.nextafter(mid, np.float32(-np.inf)), np.array([A, -A], np.float32)])
    xm = xm[np.abs(xm) <= A].astype(np.float32)
    assert_full_parity(fszlib, oracle, xm, eb, mode=0)


def test_empty_field(fszlib, oracle):
    dev = _cuda()
    x = torch.empty(0, dtype=torch.float32, device=dev)
    sb, nb = fszlib.compress(x, 1e-3, fszlib.EB_REL, shape=(0,))
    assert nb == 64
    assert sb.cpu().numpy().tobytes() == oracle.compress(np.zeros(0, np.float32), 1e-3, oracle.REL,
                                                         dims=(0,))
    y = fszlib.decompress(sb, n=0)
    assert y.numel() == 0


@pytest.mark.parametrize("variant", [0, 1, 2, 3])
def test_decoder_on_forced_variants(fszlib, oracle, variant):
    dev = _cuda()
    x = inputs.zero_slabs((16, 30, 50), seed=6).ravel()
    ref = oracle.compress(x, 1e-4, oracle.REL, force_variant=variant)
    sb = torch.from_numpy(np.frombuffer(ref, np.uint8).copy()).to(dev)
    y = fszlib.decompress(sb, n=x.size).cpu().numpy()
    assert np.array_equal(y.view(np.uint32), oracle.decompress(ref).view(np.uint32))


def _status_of_compress(fszlib, x, eb, mode=1, cap=None):
    dev = _cuda()
    xd = torch.from_numpy(x).to(dev)
    n = x.size
    cap = fszlib.fsz_compress_bound(n) if cap is None else cap
    out = torch.zeros(cap + 16, dtype=torch.uint8, device=dev)
    ws = fszlib.Workspace(n, dev)
    nb = torch.zeros(2, dtype=torch.int64, device=dev)
    sp = torch.cuda.current_stream().cuda_stream
    st = fszlib.fsz_compress(xd.data_ptr(), fszlib.make_dims((n,)), mode, eb, out.data_ptr(), cap,
                             nb.data_ptr(), ws.ptr, ws.bytes, sp)
    assert st == fszlib.OK
    return fszlib.fsz_check(ws.ptr, sp)


def test_device_detected_errors(fszlib, oracle):
    x = inputs.sinusoids(100000, seed=3)
    bad = x.copy()
    bad[77777] = np.nan
    assert _status_of_compress(fszlib, bad, 1e-3) == fszlib.ERR_NONFINITE
    bad[77777] = -np.inf
    assert _status_of_compress(fszlib, bad, 1e-3) == fszlib.ERR_NONFINITE
    off = (x + np.float32(1e4)).astype(np.float32)
    assert _status_of_compress(fszlib, off, 1e-7) == fszlib.ERR_EB_TOO_SMALL
    need = len(oracle.compress(x, 1e-4, oracle.REL))
    assert _status_of_compress(fszlib, x, 1e-4, cap=need - 64) == fszlib.ERR_CAPACITY
    assert _status_of_compress(fszlib, x, 1e-4, cap=need) == fszlib.OK


def _status_of_decompress(fszlib, stream: bytes, n, in_bytes=None):
    dev = _cuda()
    buf = torch.zeros(len(stream) + 64, dtype=torch.uint8, device=dev)
    if stream:
        buf[: len(stream)] = torch.from_numpy(np.frombuffer(stream, np.uint8).copy()).to(dev)
    out = torch.zeros(max(n, 16), dtype=torch.float32, device=dev)
    ws = fszlib.Workspace(out.numel(), dev)
    sp = torch.cuda.current_stream().cuda_stream
    st = fszlib.fsz_decompress(buf.data_ptr(), len(stream) if in_bytes is None else in_bytes,
                               out.data_ptr(), out.numel(), ws.ptr, ws.bytes, sp)
    assert st == fszlib.OK
    return fszlib.fsz_check(ws.ptr, sp)


def test_corrupt_streams_detected(fszlib, oracle):
    x = inputs.sinusoids(300000, seed=4)
    s = bytearray(oracle.compress(x, 1e-4, oracle.REL))
    n = x.size
    T = (n + 255) // 256
    assert _status_of_decompress(fszlib, bytes(s), n) == fszlib.OK
    for cut in (0, 10, 63, 64 + 8 * T - 1, len(s) - 4):
        assert _status_of_decompress(fszlib, bytes(s[:cut]), n) == fszlib.ERR_CORRUPT
    b = bytearray(s); b[0] = ord("Y")
    assert _status_of_decompress(fszlib, bytes(b), n) == fszlib.ERR_CORRUPT
    b = bytearray(s); b[64 + 8 * 100 + 5] |= 0x40                         # reserved header bits
    assert _status_of_decompress(fszlib, bytes(b), n) == fszlib.ERR_CORRUPT
    b = bytearray(s); b[64 + 8 * (T - 1) + 2] = (b[64 + 8 * (T - 1) + 2] & 0xE0) | 31  # size mismatch
    assert _status_of_decompress(fszlib, bytes(b), n) == fszlib.ERR_CORRUPT
    assert _status_of_decompress(fszlib, bytes(s), n - 1 if n > 16 else n) in (fszlib.OK,
                                                                             fszlib.ERR_CAPACITY)
    rng = np.random.default_rng(0)
    for _ in range(20):   # random damage: any status, never a fault
        b = bytearray(s)
        for pos in rng.integers(64, len(s), size=4):
            b[int(pos)] = int(rng.integers(0, 256))
        assert _status_of_decompress(fszlib, bytes(b), n) in (fszlib.OK, fszlib.ERR_CORRUPT)


def _decode(fszlib, stream: bytes, n):
    """(device status, reconstruction) of one decode through the C ABI."""
    dev = _cuda()
    buf = torch.zeros(len(stream) + 64, dtype=torch.uint8, device=dev)
    buf[: len(stream)] = torch.from_numpy(np.frombuffer(stream, np.uint8).copy()).to(dev)
    out = torch.zeros(n, dtype=torch.float32, device=dev)
    ws = fszlib.Workspace(n, dev)
    sp = torch.cuda.current_stream().cuda_stream
    assert fszlib.fsz_decompress(buf.data_ptr(), len(stream), out.data_ptr(), n, ws.ptr, ws.bytes,
                                 sp) == fszlib.OK
    return fszlib.fsz_check(ws.ptr, sp), out.cpu().numpy()


def test_damaged_streams_decode_as_the_oracle(fszlib, oracle):
    """Damage the format still admits (payload bytes, rates traded between two blocks of a
    tile at equal size, random bytes past the preamble) decodes on the GPU to exactly the
    oracle decoder's floats (wrap-around integer arithmetic, the same conversions); what
    either decoder refuses, both refuse."""
    x = inputs.sinusoids(300000, seed=4)
    s = oracle.compress(x, 1e-4, oracle.REL)
    n = x.size
    T = (n + 255) // 256
    data0 = 64 + 8 * T
    rng = np.random.default_rng(1)
    cases = []
    for _ in range(10):  # payload bytes
        b = bytearray(s)
        for pos in rng.integers(data0, len(s), size=6):
            b[int(pos)] = int(rng.integers(0, 256))
        cases.append(b)
    hdr = np.frombuffer(s[64:data0], np.uint8).reshape(T, 8)
    for _ in range(10):  # one block's rate up by one, another's down by one: same sizes
        while True:
            t = int(rng.integers(0, T))
            r = hdr[t] & 31
            up = [k for k in range(8) if 1 <= r[k] <= 30]
            down = [k for k in range(8) if r[k] >= 2]
            pairs = [(i, j) for i in up for j in down if i != j]
            if pairs:
                break
        i, j = pairs[int(rng.integers(0, len(pairs)))]
        b = bytearray(s)
        b[64 + 8 * t + i] += 1
        b[64 + 8 * t + j] -= 1
        cases.append(b)
    for _ in range(10):  # anything past the preamble
        b = bytearray(s)
        for pos in rng.integers(64, len(s), size=3):
            b[int(pos)] = int(rng.integers(0, 256))
        cases.append(b)
    seen = set()
    for k, b in enumerate(cases):
        want = oracle.decompress_status(bytes(b))
        st, y = _decode(fszlib, bytes(b), n)
        assert st == want, (k, st, want)
        seen.add(st)
        if st == fszlib.OK:
            assert np.array_equal(y.view(np.uint32), oracle.decompress(bytes(b)).view(np.uint32)), k
    assert fszlib.OK in seen


def test_lookback_timeout_is_reported(fszlib, oracle):
    # A chunk that never publishes its flag: its successor's bounded wait runs out, the
    # kernel still finishes and the workspace status reads FSZ_ERR_TIMEOUT.
    x = inputs.sinusoids(10 * 8192, seed=5)
    try:
        fszlib.fsz_set_test_hooks(3, 20_000_000)
        assert _status_of_compress(fszlib, x, 1e-3) == fszlib.ERR_TIMEOUT
        s = oracle.compress(x, 1e-3, oracle.REL)
        assert _status_of_decompress(fszlib, s, x.size) == fszlib.ERR_TIMEOUT
    finally:
        fszlib.fsz_set_test_hooks(2 ** 64 - 1, 0)
    assert _status_of_compress(fszlib, x, 1e-3) == fszlib.OK


# --------------------------------------------------------------------------- full size

def sampled_parity(fszlib, oracle, xd, rel, shape, nsample=48, seed=0):
    """Full-size check: every element by properties; sampled tiles byte for byte."""
    n = xd.numel()
    sb, nb = fszlib.compress(xd, rel, fszlib.EB_REL, shape=shape)
    y = fszlib.decompress(sb, n=n)
    x = xd.cpu().numpy().ravel()
    lo, hi, fin = oracle.stats(x)
    p = oracle.params(oracle.REL, rel, lo, hi, fin, n)
    pre = sb[:64].cpu().numpy().tobytes()
    h = fszlib.fsz_read_header(pre)
    assert np.float32(h["step"]) == np.float32(p.s) and h["total_bytes"] == nb
    # every element: d' = fl(rint(fl(d r)) s), and |d - d'| <= eb
    r32 = torch.tensor(p.r, dtype=torch.float32, device=xd.device)
    s32 = torch.tensor(p.s, dtype=torch.float32, device=xd.device)
    q = torch.round(xd.reshape(-1) * r32) + 0.0   # q = 0 reconstructs as +0.0
    want = q * s32
    assert torch.equal(want.view(torch.int32), y.view(torch.int32))
    err = (xd.reshape(-1).double() - y.double()).abs().max().item()
    assert err <= p.eb
    # sampled tiles: header bytes and data bytes where the GPU header places them
    T = (n + 255) // 256
    stream = sb.cpu().numpy()
    hdr = stream[64:64 + 8 * T].reshape(T, 8).astype(np.int64)
    rates = hdr & 31
    sizes = np.where(rates == 0, 0, 4 + 4 * rates).sum(axis=1) + np.where(hdr[:, 0] & 0x40, 4, 0)
    offs = np.concatenate([[0], np.cumsum(sizes)])
    assert 64 + 8 * T + offs[-1] == nb
    rng = np.random.default_rng(seed)
    starts = set(int(t) for t in rng.integers(0, max(1, T - 4), size=nsample)) | {0, max(0, T - 4)}
    data0 = 64 + 8 * T
    for t0 in sorted(starts):
        t1 = min(T, t0 + 4)
        rh, rd = oracle.compress_tiles(x, p.r, t0, t1)
        assert stream[64 + 8 * t0:64 + 8 * t1].tobytes() == rh, t0
        assert stream[data0 + offs[t0]:data0 + offs[t1]].tobytes() == rd, t0
    return nb


def _first_diff(a: bytes, b: bytes) -> str:
    if len(a) != len(b):
        return f"lengths {len(a)} vs {len(b)}"
    u, v = np.frombuffer(a, np.uint8), np.frombuffer(b, np.uint8)
    k = int(np.nonzero(u != v)[0][0])
    return f"first difference at byte {k} of {len(a)}"


def _oracle_roundtrip(oracle, x, rel, shape):
    ref = oracle.compress(x, rel, oracle.REL, dims=shape)
    return ref, oracle.decompress(ref)


def whole_parity(fszlib, oracle, xd, rels, shape):
    """Full-size check: for each bound, the whole GPU stream against the oracle's stream byte
    for byte, and the whole GPU reconstruction against the oracle decoder's bit for bit (the
    oracle runs on host threads, one per bound, while the GPU works)."""
    import concurrent.futures as cf
    n = xd.numel()
    x = xd.reshape(-1).cpu().numpy()
    with cf.ThreadPoolExecutor(max_workers=len(rels)) as ex:
        futs = {rel: ex.submit(_oracle_roundtrip, oracle, x, rel, shape) for rel in rels}
        for rel in rels:
            sb, nb = fszlib.compress(xd, rel, fszlib.EB_REL, shape=shape)
            y = fszlib.decompress(sb, n=n)
            got = sb.cpu().numpy().tobytes()
            yg = y.cpu().numpy()
            del sb, y
            ref, yref = futs[rel].result()
            assert got == ref, (rel, _first_diff(got, ref))
            assert np.array_equal(yg.view(np.uint32), yref.view(np.uint32)), rel
            p = oracle.params_for(x, oracle.REL, rel)
            assert np.abs(x.astype(np.float64) - yg.astype(np.float64)).max() <= p.eb
            del yg, yref


def test_config2_grf_512cubed_whole_streams(fszlib, oracle):
    _cuda()
    shape = (512, 512, 512)
    f = inputs.grf(shape, seed=1, device="cuda")
    whole_parity(fszlib, oracle, f.reshape(-1), (1e-2, 1e-3, 1e-4), shape)
    z = inputs.zero_slabs(shape, seed=1, device="cuda", base=f)
    del f
    whole_parity(fszlib, oracle, z.reshape(-1), (1e-2, 1e-3, 1e-4), shape)


def test_config3_particles_2p28_whole_stream(fszlib, oracle):
    _cuda()
    x = inputs.particles(1 << 28, seed=2, device="cuda")
    whole_parity(fszlib, oracle, x, (1e-4,), (1 << 28,))


@pytest.mark.parametrize("rel", [1e-2, 1e-4])
def test_config2_sampled_tiles_and_properties(fszlib, oracle, rel):
    """The same fields by the checks that hold at any size: every element by the
    quantization property and the bound, sampled tile ranges against the oracle's tile
    encoder where the GPU header places them."""
    _cuda()
    f = inputs.grf((512, 512, 512), seed=1, device="cuda")
    sampled_parity(fszlib, oracle, f.reshape(-1), rel, (512, 512, 512), seed=int(rel * 1e4))


def test_field_past_2p32_elements(fszlib, oracle):
    """A 1-D field of 2^32 + 777 elements (17.2 GB) with a stream of about 4.9 GB:
    element and byte offsets pass 2^32, the last tile and the last 16 bytes are ragged. Every element by the
    quantization property and the bound, on the device in slices; the field's parameters
    from its value range; sampled tiles (the ones around element 2^32 among them) byte for
    byte against the oracle's tile encoder."""
    dev = _cuda()
    if torch.cuda.mem_get_info()[0] < (80 << 30):
        pytest.skip("needs about 80 GB of free device memory")
    n = (1 << 32) + 777
    S = 1 << 28
    xd = torch.empty(n, dtype=torch.float32, device=dev)
    g = torch.Generator(device=dev)
    g.manual_seed(5)
    for k0 in range(0, n, S):
        k1 = min(n, k0 + S)
        i = torch.arange(k0, k1, dtype=torch.float64, device=dev)
        xd[k0:k1] = (50.0 * torch.sin(i * 2.1e-4) + 20.0 * torch.sin(i * 3.7e-7)
                     + 2.0 * torch.randn(k1 - k0, generator=g, dtype=torch.float64, device=dev)
                     ).to(torch.float32)
        del i
    rel = 1e-4  # noise of ~70 steps: CR ~3.5, a stream past 2^32 bytes
    sb, nb = fszlib.compress(xd, rel, fszlib.EB_REL)
    lo, hi = float(xd.min().item()), float(xd.max().item())
    assert bool(torch.isfinite(xd).all())
    p = oracle.params(oracle.REL, rel, lo, hi, True, n)
    h = fszlib.fsz_read_header(sb[:64].cpu().numpy().tobytes())
    assert h["n"] == n and h["total_bytes"] == nb and np.float32(h["step"]) == np.float32(p.s)
    y = fszlib.decompress(sb, n=n)
    r32 = torch.tensor(p.r, dtype=torch.float32, device=dev)
    s32 = torch.tensor(p.s, dtype=torch.float32, device=dev)
    for k0 in range(0, n, S):
        xs, ys = xd[k0:k0 + S], y[k0:k0 + S]
        want = (torch.round(xs * r32) + 0.0) * s32
        assert torch.equal(want.view(torch.int32), ys.view(torch.int32)), k0
        assert (xs.double() - ys.double()).abs().max().item() <= p.eb, k0
        del want
    del y
    T = (n + 255) // 256
    hdr = sb[64:64 + 8 * T].cpu().numpy().reshape(T, 8).astype(np.int64)
    rates = hdr & 31
    sizes = np.where(rates == 0, 0, 4 + 4 * rates).sum(axis=1) + np.where(hdr[:, 0] & 0x40, 4, 0)
    offs = np.concatenate([[0], np.cumsum(sizes)])
    data0 = 64 + 8 * T
    assert data0 + int(offs[-1]) == nb and data0 + int(offs[-1]) > (1 << 32)
    rng = np.random.default_rng(11)
    starts = set(int(t) for t in rng.integers(0, T - 4, size=32))
    starts |= {0, T - 4, (1 << 24) - 2}  # tile 2^24 starts at element 2^32
    for t0 in sorted(starts):
        t1 = min(T, t0 + 4)
        xs = xd[256 * t0:min(n, 256 * t1)].cpu().numpy()
        rh, rd = oracle.compress_tiles(xs, p.r, 0, t1 - t0)
        assert sb[64 + 8 * t0:64 + 8 * t1].cpu().numpy().tobytes() == rh, t0
        assert sb[data0 + int(offs[t0]):data0 + int(offs[t1])].cpu().numpy().tobytes() == rd, t0


def test_workspace_reused_across_calls(fszlib, oracle):
    """One workspace for a run of calls of different sizes, a batched call among them: a
    single-field call clears what it uses in its set-up kernel (control words, field
    record, lookback flags), so whatever an earlier call left there does not leak into its
    stream or reconstruction."""
    dev = _cuda()
    big = 3 * (1 << 20) + 4097
    ws = fszlib.Workspace(big, dev)
    rng = np.random.default_rng(33)
    sizes = [big, 1000, 70_000, 8192 * 41 + 5, 257, big - 12345]
    for k, n in enumerate(sizes):
        x = inputs.sinusoids(n, seed=100 + k) if k % 2 else rng.normal(0, 1, n).astype(np.float32)
        ref = oracle.compress(x, 1e-3, oracle.REL)
        sb, nb = fszlib.compress(torch.from_numpy(x).to(dev), 1e-3, fszlib.EB_REL, ws=ws)
        assert sb.cpu().numpy().tobytes() == ref, (k, n)
        y = fszlib.decompress(sb, n=n, ws=ws).cpu().numpy()
        assert np.array_equal(y.view(np.uint32), oracle.decompress(ref).view(np.uint32)), (k, n)
        if k == 2:  # a batched call through the same memory in between
            bytes_needed = fszlib.fsz_batch_workspace_bytes(2 * 50_000, 2)
            assert bytes_needed <= ws.bytes
            fields = [(torch.from_numpy(inputs.sinusoids(50_000, seed=7 + j)).to(dev), (50_000,),
                       fszlib.EB_REL, 1e-2) for j in range(2)]
            cb = fszlib.CompressBatch(fields, dev)
            cb.ws, cb.ws_bytes = ws.buf, ws.bytes  # through the shared workspace
            assert cb.run() == fszlib.OK and cb.status()[0] == fszlib.OK
            sizes_b = cb.sizes.cpu().tolist()
            for j, (f, *_) in enumerate(fields):
                assert cb.stream(j, sizes_b).cpu().numpy().tobytes() == oracle.compress(
                    f.cpu().numpy(), 1e-2, oracle.REL), j
