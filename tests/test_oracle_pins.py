"""Pins of the CPU oracle against what the paper and mathematics fix (no GPU).

Each test checks the oracle against something other than itself: numbers the
paper prints for its worked examples, bytes derived by hand from the format,
brute force with numpy library routines, closed forms and invariants.
"""
import json
import math
import os
import struct

import numpy as np
import pytest

from paper_2607_15413_gb300 import inputs

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _load(name):
    with open(os.path.join(GOLDEN, name)) as f:
        return json.load(f)


def bitlen_np(a):
    """Bit length of non-negative integers (numpy, independent of the oracle)."""
    a = np.asarray(a, dtype=np.int64)
    return np.array([int(x).bit_length() for x in a.ravel()]).reshape(a.shape)


def residuals_np(qh, order):
    """Brute force: k-th order finite differences with two zero predecessors."""
    ext = np.concatenate([np.zeros(2, np.int64), np.asarray(qh, np.int64)])
    return np.diff(ext, n=order)[2 - order:]


def costs_np(q, mu):
    """Four separate passes with numpy: residuals, block maxima, rates, Eq. 3."""
    out = []
    for v in range(4):
        centred = v >= 2
        order = 2 if v in (1, 3) else 1
        qh = np.asarray(q, np.int64) - (mu if centred else 0)
        l = residuals_np(qh, order)
        m = np.abs(l).reshape(8, 32).max(axis=1)
        r = bitlen_np(m)
        cost = int(np.where(r == 0, 0, 4 + 4 * r).sum()) + (4 if centred else 0)
        out.append((cost, r))
    return out


# --------------------------------------------------------------------------- rate / cost

def test_rate_is_bit_length(oracle):
    for m in list(range(0, 5000)) + [2 ** k + d for k in range(1, 31) for d in (-1, 0, 1)]:
        assert oracle.rate(m) == int(m).bit_length()
        if m < 5000:
            assert oracle.rate(m) == math.ceil(math.log2(m + 1))


def test_block_cost_eq3(oracle):
    assert oracle.block_cost(0) == 0
    for r in range(1, 32):
        assert oracle.block_cost(r) == 4 + 4 * r


# --------------------------------------------------------------------------- worked examples

def test_worked_example_cross_block(oracle):
    g = _load("paper_worked_examples.json")["cross_block"]
    # A slowly rising tile whose blocks 0, 1 and 3 begin at 1000, 1008 and 1024.
    q = (1000 + np.arange(256) // 4).astype(np.int32)
    assert [int(q[0]), int(q[32]), int(q[96])] == g["boundaries"]
    indep = [bitlen_np(np.abs(np.diff(np.concatenate([[0], q[b * 32:(b + 1) * 32]]))).max())
             for b in range(8)]
    assert min(indep) >= g["independent_rates"][0] and max(indep) <= g["independent_rates"][1]
    assert indep[3] == 11 and indep[0] == 10
    C, rates = oracle.tile_costs(q, 0)
    assert all(int(r) == g["cross_block_rate"] for r in rates[oracle.LZ1][1:])
    assert oracle.block_cost(11) - oracle.block_cost(g["cross_block_rate"]) == g["max_saving_bytes"]


def test_worked_example_lz1_vs_lz2(oracle):
    g = _load("paper_worked_examples.json")["lz1_vs_lz2"]
    q = (7 + g["stride"] * np.arange(256)).astype(np.int32)
    l1 = oracle.tile_residuals(q, 0, oracle.LZ1)
    l2 = oracle.tile_residuals(q, 0, oracle.LZ2)
    b = g["block"]
    assert np.all(l1[32 * b:32 * b + 32] == g["lz1_residual"])
    assert np.all(l2[32 * b:32 * b + 32] == 0)
    C, rates = oracle.tile_costs(q, 0)
    assert rates[oracle.LZ1][b] == g["lz1_rate"] and oracle.block_cost(g["lz1_rate"]) == g["lz1_cost"]
    assert rates[oracle.LZ2][b] == g["lz2_rate"] and oracle.block_cost(0) == g["lz2_cost"]


def test_worked_example_centering(oracle):
    g = _load("paper_worked_examples.json")["centering"]
    # q_0 = 1000 on a tile whose values hover around 1001 with steps of at most 3.
    rng = np.random.default_rng(5)
    a = np.zeros(256, np.int64)
    a[0] = -1
    a[1] = 2            # residual 3 at i = 1
    for i in range(2, 256):
        a[i] = int(np.clip(a[i - 1] + rng.integers(-1, 2), -1, 1))
    a[255] = 0
    q = (g["mu"] + a).astype(np.int32)
    assert q[0] == g["q0"]
    # mu from the float tile mean: d_i = q_i s must quantize back to q_i.
    p = oracle.params(oracle.ABS, 0.5, -2000.0, 2000.0)
    d = (q.astype(np.float32) * np.float32(p.s)).astype(np.float32)
    assert np.array_equal(oracle.quantize(d, p.r), q)
    assert abs(a.mean()) < 0.3                       # the tile's mean quantizes to mu
    assert oracle.tile_mu(d, p.r) == g["mu"]
    C, rates = oracle.tile_costs(q, g["mu"])
    assert rates[oracle.LZ1][0] == g["plain_rate"]
    assert oracle.block_cost(g["plain_rate"]) == g["plain_cost"]
    l1c = oracle.tile_residuals(q, g["mu"], oracle.LZ1C)
    assert l1c[0] == g["centred_boundary"] and np.abs(l1c[:32]).max() == g["centred_max"]
    assert rates[oracle.LZ1C][0] == g["centred_rate"]
    assert oracle.block_cost(g["centred_rate"]) + 4 == g["centred_cost_with_mu"]
    assert g["plain_cost"] / g["centred_cost_with_mu"] == g["saving_factor"]


# --------------------------------------------------------------------------- residuals

@pytest.mark.parametrize("seed", range(6))
def test_residuals_match_numpy_diff(oracle, seed):
    rng = np.random.default_rng(seed)
    q = np.cumsum(rng.integers(-50, 51, size=256)).astype(np.int32) + int(rng.integers(-9000, 9000))
    mu = int(rng.integers(-10000, 10000))
    for v in range(4):
        centred = v >= 2
        order = 2 if v in (1, 3) else 1
        qh = q.astype(np.int64) - (mu if centred else 0)
        assert np.array_equal(oracle.tile_residuals(q, mu, v), residuals_np(qh, order))


def test_cancellation_property_eq4(oracle):
    rng = np.random.default_rng(11)
    q = np.cumsum(rng.integers(-20, 21, size=256)).astype(np.int32)
    for mu in (-777, 1, 12345):
        for plain, cent, k in ((oracle.LZ1, oracle.LZ1C, 1), (oracle.LZ2, oracle.LZ2C, 2)):
            a = oracle.tile_residuals(q, 0, plain)
            b = oracle.tile_residuals(q, mu, cent)
            assert np.array_equal(a[k:], b[k:])
            assert not np.array_equal(a[:k], b[:k])


def test_constant_tile(oracle):
    # Constant offsets cancel (Sec. 4.2.3): only the tile's first residual is non-zero
    # without centring; with mu equal to the constant every residual is zero.
    c = 4321
    q = np.full(256, c, np.int32)
    l1 = oracle.tile_residuals(q, 0, oracle.LZ1)
    assert l1[0] == c and np.all(l1[1:] == 0)
    l2 = oracle.tile_residuals(q, 0, oracle.LZ2)
    assert l2[0] == c and l2[1] == -c and np.all(l2[2:] == 0)
    for v in (oracle.LZ1C, oracle.LZ2C):
        assert np.all(oracle.tile_residuals(q, c, v) == 0)
    C, _ = oracle.tile_costs(q, c)
    assert oracle.select(C) == oracle.LZ1C and C[oracle.LZ1C] == 4


def test_linear_tile_lz2(oracle):
    q = (-300 + 17 * np.arange(256)).astype(np.int32)
    l2 = oracle.tile_residuals(q, 0, oracle.LZ2)
    assert np.all(l2[2:] == 0)
    C, rates = oracle.tile_costs(q, 0)
    assert np.all(rates[oracle.LZ2][1:] == 0)
    assert oracle.select(C) in (oracle.LZ2, oracle.LZ2C)


# --------------------------------------------------------------------------- four-way pass

def _tiles(seed):
    rng = np.random.default_rng(seed)
    yield np.cumsum(rng.integers(-3, 4, size=256)) + 100
    yield np.cumsum(np.cumsum(rng.integers(-2, 3, size=256))) - 5000
    yield rng.integers(-1000, 1000, size=256)
    yield np.full(256, int(rng.integers(-50000, 50000)))
    yield 9000 + 5 * np.arange(256) + rng.integers(-1, 2, size=256)
    t = np.zeros(256, np.int64)
    t[int(rng.integers(0, 256))] = int(rng.integers(-2 ** 18, 2 ** 18))
    yield t


@pytest.mark.parametrize("seed", range(25))
def test_single_pass_equals_four_passes(oracle, seed):
    rng = np.random.default_rng(seed + 100)
    for q in _tiles(seed):
        q = np.asarray(q, np.int32)
        for mu in (0, int(q.mean().round()), int(rng.integers(-3000, 3000))):
            C1, R1 = oracle.tile_costs(q, mu)
            C4, R4 = oracle.tile_costs(q, mu, four_pass=True)
            assert np.array_equal(C1, C4) and np.array_equal(R1, R4)
            brute = costs_np(q, mu)
            assert [c for c, _ in brute] == [int(x) for x in C1]
            for v in range(4):
                assert np.array_equal(brute[v][1], R1[v])


def test_select_first_strict_minimum(oracle):
    assert oracle.select(np.array([10, 10, 10, 10])) == 0
    assert oracle.select(np.array([12, 10, 10, 10])) == 1
    assert oracle.select(np.array([12, 11, 10, 10])) == 2
    assert oracle.select(np.array([12, 11, 10, 9])) == 3


# --------------------------------------------------------------------------- params

def test_params_rel_and_margin(oracle):
    p = oracle.params(oracle.REL, 1e-3, -2.0, 3.0)
    assert p.eb == 1e-3 * (3.0 - (-2.0))
    e = np.float32(p.e)
    assert float(e) < p.eb
    eps = (3 * p.Q + 4) * 2.0 ** -23
    target = p.eb_eff * (1 - eps)
    assert float(e) <= target < float(np.nextafter(e, np.float32(np.inf)))
    assert np.float32(p.s) == np.float32(2) * e
    assert np.float32(p.r) == np.float32(1) / np.float32(p.s)
    assert p.Q == math.ceil(3.0 / (2 * p.eb_eff * (1 - 2 ** -4))) + 1


def test_params_constant_and_errors(oracle):
    assert oracle.params(oracle.REL, 1e-2, 5.0, 5.0).eb == pytest.approx(5e-2, rel=1e-15)
    assert oracle.params(oracle.REL, 1e-2, 0.0, 0.0).eb == 1e-2
    for bad in (0.0, -1.0, float("nan"), float("inf")):
        with pytest.raises(oracle.OracleError) as ei:
            oracle.params(oracle.ABS, bad, 0.0, 1.0)
        assert ei.value.status == oracle.ERR_INVALID_ARG
    with pytest.raises(oracle.OracleError) as ei:
        oracle.params(oracle.ABS, 1e-3, 0.0, 1.0, finite=False)
    assert ei.value.status == oracle.ERR_NONFINITE
    with pytest.raises(oracle.OracleError) as ei:  # A / (2 eb) far beyond the int range
        oracle.params(oracle.REL, 1e-7, 1000.0, 1001.0)
    assert ei.value.status == oracle.ERR_EB_TOO_SMALL


# --------------------------------------------------------------------------- error bound

def _check_bound(oracle, x, eb, mode):
    s = oracle.compress(x, eb, mode)
    y = oracle.decompress(s)
    p = oracle.params_for(x, mode, eb)
    err = np.abs(x.astype(np.float64) - y.astype(np.float64))
    assert err.max() <= p.eb, (err.max(), p.eb)
    q = oracle.decompress(s, q=True)
    assert np.array_equal(q, oracle.quantize(x, p.r))       # integers survive exactly
    assert np.array_equal(y, (q.astype(np.float32) * np.float32(p.s)).astype(np.float32))
    return s, y


@pytest.mark.parametrize("rel", [1e-2, 1e-3, 1e-4, 1e-5])
def test_error_bound_rel_fields(oracle, rel):
    for x in (inputs.sinusoids(20000, seed=3), inputs.grf((24, 20, 16), seed=4).ravel(),
              inputs.zero_slabs((20, 8, 16), seed=5).ravel(), inputs.particles(12000, seed=6)):
        _check_bound(oracle, x, rel, oracle.REL)


def test_error_bound_adversarial_midpoints(oracle):
    A = np.float32(37.25)
    for eb in (1e-1, 3.3e-3, 7.77e-4):
        p = oracle.params(oracle.ABS, eb, -float(A), float(A))
        s = np.float32(p.s)
        k = np.arange(-p.Q, p.Q + 1, max(1, p.Q // 3000), dtype=np.int64)
        mid = ((k.astype(np.float64) + 0.5) * float(s)).astype(np.float32)
        cand = [mid]
        for ulps in (1, 2):
            cand.append(np.nextafter(mid, np.float32(np.inf)))
            cand.append(np.nextafter(mid, np.float32(-np.inf)))
            mid = cand[-2]
        x = np.concatenate(cand + [np.array([A, -A], np.float32)])
        x = x[np.abs(x) <= A].astype(np.float32)
        _check_bound(oracle, x, eb, oracle.ABS)


def test_error_bound_large_offset(oracle):
    rng = np.random.default_rng(9)
    x = (1.0e4 + rng.normal(0, 30.0, 50000)).astype(np.float32)  # A / range ~ 50
    _check_bound(oracle, x, 1e-3, oracle.REL)
    with pytest.raises(oracle.OracleError) as ei:
        oracle.compress(x, 1e-6, oracle.REL)
    assert ei.value.status == oracle.ERR_EB_TOO_SMALL


# --------------------------------------------------------------------------- stream format

@pytest.mark.parametrize("name", ["spike", "offset_ramp"])
def test_hand_built_golden_bytes(oracle, name):
    g = _load("hand_tiles.json")[name]
    q = np.zeros(256, np.int64)
    if name == "spike":
        q[0] = 5
    else:
        q = 5000 + 2 * np.arange(256)
    # Keep the field's max |d| fixed at 8000 s' so the params are those of the test.
    p = oracle.params(oracle.ABS, 0.5, -8000.0, 8000.0)
    s = np.float32(p.s)
    d = (q.astype(np.float32) * s).astype(np.float32)
    x = np.concatenate([d, np.zeros(256, np.float32)])
    x[256] = np.float32(8000.0)   # second tile pins A; its bytes are not checked
    x[257] = np.float32(-8000.0)
    assert np.array_equal(oracle.quantize(d, p.r), q.astype(np.int32))
    stream = oracle.compress(x, 0.5, oracle.ABS)
    T = 2
    header = stream[64:64 + 8 * T]
    assert header[:8].hex() == g["header_hex"]
    data = stream[64 + 8 * T:]
    want = bytes.fromhex(g["data_hex"])
    assert data[:len(want)] == want
    # Preamble fields (little-endian): magic, version, ndim, mode, n, dims, eb, s, 0, data_bytes.
    magic, ver, ndim, mode, n, d0, d1, d2, eb, sv, res, db = struct.unpack("<4sHBBQQQQdfIQ", stream[:64])
    assert (magic, ver, ndim, mode, n, d0, d1, d2) == (b"FSZ1", 1, 1, 0, 512, 512, 0, 0)
    assert eb == 0.5 and np.float32(sv) == s and res == 0 and db == len(data)


def test_stream_size_and_alignment(oracle):
    x = inputs.grf((16, 16, 40), seed=7).ravel()
    s = oracle.compress(x, 1e-3, oracle.REL, dims=(16, 16, 40))
    info = oracle.read_preamble(s)
    T = (x.size + 255) // 256
    assert info["dims"] == (16, 16, 40) and info["n"] == x.size
    assert len(s) == 64 + 8 * T + info["data_bytes"]
    hdr = np.frombuffer(s[64:64 + 8 * T], np.uint8).reshape(T, 8).astype(np.int64)
    sizes = [(4 if h[0] & 0x40 else 0)
             + sum(0 if (int(b) & 31) == 0 else 4 + 4 * (int(b) & 31) for b in h) for h in hdr]
    assert sum(sizes) == info["data_bytes"] and all(sz % 4 == 0 for sz in sizes)


@pytest.mark.parametrize("n", [0, 1, 31, 32, 33, 255, 256, 257, 1000, 4097])
def test_ragged_sizes_roundtrip(oracle, n):
    rng = np.random.default_rng(n)
    x = np.cumsum(rng.normal(0, 1, n)).astype(np.float32)
    s = oracle.compress(x, 1e-3, oracle.REL)
    assert len(s) == 64 + 8 * ((n + 255) // 256) + oracle.read_preamble(s)["data_bytes"]
    y = oracle.decompress(s)
    assert y.size == n
    if n:
        p = oracle.params_for(x, oracle.REL, 1e-3)
        assert np.abs(x.astype(np.float64) - y).max() <= p.eb


@pytest.mark.parametrize("variant", [0, 1, 2, 3])
def test_forced_variants_roundtrip(oracle, variant):
    x = inputs.zero_slabs((12, 10, 30), seed=8).ravel()
    s = oracle.compress(x, 1e-4, oracle.REL, force_variant=variant)
    p = oracle.params_for(x, oracle.REL, 1e-4)
    assert np.array_equal(oracle.decompress(s, q=True), oracle.quantize(x, p.r))
    T = (x.size + 255) // 256
    h0 = np.frombuffer(s[64:64 + 8 * T], np.uint8)[::8]
    assert np.all(((h0 >> 7) & 1) == (variant in (1, 3)))
    assert np.all(((h0 >> 6) & 1) == (variant >= 2))


def test_adaptive_never_worse_than_forced(oracle):
    x = inputs.particles(40000, seed=12)
    sizes = [len(oracle.compress(x, 1e-4, oracle.REL, force_variant=v)) for v in range(4)]
    assert len(oracle.compress(x, 1e-4, oracle.REL)) <= min(sizes)


def test_nonfinite_rejected(oracle):
    x = np.ones(300, np.float32)
    x[7] = np.inf
    with pytest.raises(oracle.OracleError) as ei:
        oracle.compress(x, 1e-3, oracle.REL)
    assert ei.value.status == oracle.ERR_NONFINITE


def test_corrupt_streams_are_rejected(oracle):
    x = inputs.sinusoids(5000, seed=1)
    s = bytearray(oracle.compress(x, 1e-3, oracle.REL))
    assert oracle.decompress_status(bytes(s)) == oracle.OK
    for cut in (0, 10, 63, 64, 70, len(s) - 1):
        assert oracle.decompress_status(bytes(s[:cut])) == oracle.ERR_CORRUPT
    bad = bytearray(s); bad[0] = ord("X")
    assert oracle.decompress_status(bytes(bad)) == oracle.ERR_CORRUPT
    bad = bytearray(s); bad[64 + 8 + 3] |= 0x80          # reserved bits of block 3
    assert oracle.decompress_status(bytes(bad)) == oracle.ERR_CORRUPT
    bad = bytearray(s); bad[64] = (bad[64] & 0xE0) | ((bad[64] & 31) + 1) % 32  # size mismatch
    assert oracle.decompress_status(bytes(bad)) == oracle.ERR_CORRUPT
    assert oracle.decompress_status(bytes(s), cap=10) == oracle.ERR_CAPACITY
    rng = np.random.default_rng(0)
    for _ in range(300):
        bad = bytearray(s)
        for pos in rng.integers(0, len(s), size=3):
            bad[int(pos)] = int(rng.integers(0, 256))
        assert oracle.decompress_status(bytes(bad)) in (oracle.OK, oracle.ERR_CORRUPT,
                                                        oracle.ERR_CAPACITY)


# --------------------------------------------------------------------------- value range, ties, mean order

def _stats_np(x):
    """numpy restatement of the value-range pass: min, max and the all-finite flag."""
    fin = bool(np.isfinite(x).all())
    if not fin or x.size == 0:
        return None, None, fin
    return float(x.min()), float(x.max()), fin


@pytest.mark.parametrize("n", [1, 2, 3, 255, 256, 257, 4099])
def test_stats_against_numpy(oracle, n):
    # The extremes are put at the first and at the last element (a loop that skips either
    # end fails here), and one check puts them in the middle.
    rng = np.random.default_rng(n)
    base = rng.uniform(-5.0, 5.0, n).astype(np.float32)
    for lo_at, hi_at in ((0, n - 1), (n - 1, 0), (n // 2, n // 3)):
        x = base.copy()
        x[hi_at] = np.float32(7.25)
        if lo_at != hi_at:
            x[lo_at] = np.float32(-9.5)
        lo, hi, fin = oracle.stats(x)
        want = _stats_np(x)
        assert fin and want[2]
        assert (lo, hi) == (want[0], want[1]), (lo_at, hi_at)
    for bad in (np.nan, np.inf, -np.inf):
        for at in {0, n - 1, n // 2}:
            x = base.copy()
            x[at] = bad
            assert oracle.stats(x)[2] is False and _stats_np(x)[2] is False, (bad, at)


def test_stats_empty_and_constant(oracle):
    assert oracle.stats(np.zeros(0, np.float32)) == (0.0, 0.0, True)
    assert oracle.stats(np.full(300, -3.5, np.float32)) == (-3.5, -3.5, True)


def _exact_ties(r, ks):
    """float32 inputs d with fl32(d r) exactly k + 1/2, found among the float32 neighbours
    of (k + 1/2) / r (numpy float32 multiplies round once, to nearest)."""
    r32 = np.float32(r)
    out = []
    for k in ks:
        t = np.float32(k + 0.5)
        d = np.float32(float(t) / float(r32))
        for _ in range(6):
            d = np.nextafter(d, np.float32(-np.inf))
        for _ in range(13):
            if np.float32(d * r32) == t:
                out.append(d)
                break
            d = np.nextafter(d, np.float32(np.inf))
    return np.array(out, np.float32)


@pytest.mark.parametrize("r", [0.125, 1.0, 2.0 ** -20, 1.0 / 0.0062, 1.0 / 3.3e-3, 37.9])
def test_quantize_ties_to_even(oracle, r):
    # Sec. 4.2.2 rounds d / (2 eb) to an integer; the reading fixes t = fl32(d r) and the
    # nearest integer with ties to even. Inputs that land exactly on k + 1/2 for even and
    # odd k, both signs, from 1/2 up to 2^17 + 1/2: a half-away-from-zero rounding fails.
    rng = np.random.default_rng(int(r * 1000) % 2 ** 31)
    ks = sorted(set([0, 1, 2, 3, 4, 5, 100, 101, 4096, 4097, 131070, 131071]
                    + [int(k) for k in rng.integers(0, 1 << 17, 60)]))
    ks = ks + [-k - 1 for k in ks]            # k + 1/2 for k = -1, -2, ...: -1/2, -3/2, ...
    d = _exact_ties(r, ks)
    assert d.size >= len(ks) * 3 // 4
    t = (d * np.float32(r)).astype(np.float32)
    assert np.all(t - np.floor(t) == 0.5)     # every input sits on a tie
    want = np.rint(t).astype(np.int64)        # numpy's rint: ties to even
    got = oracle.quantize(d, r).astype(np.int64)
    assert np.array_equal(got, want)
    assert np.all(got % 2 == 0)               # every tie went to the even neighbour
    # off the ties the same rule is plain rounding to nearest
    y = rng.uniform(-1e5, 1e5, 2000).astype(np.float32) / np.float32(r)
    y = y.astype(np.float32)
    assert np.array_equal(oracle.quantize(y, r), np.rint(y * np.float32(r)).astype(np.int32))


def _mu_np(d, r, order):
    """The tile mean's quantized value with the float32 sum taken in a given order."""
    d = np.asarray(d, np.float32)
    if order == "runs":        # 8-element runs left to right, then the pairwise tree
        P = d.reshape(32, 8)[:, 0].copy()
        for i in range(1, 8):
            P = (P + d.reshape(32, 8)[:, i]).astype(np.float32)
        h = 16
        while h >= 1:
            P[:h] = (P[:h] + P[h:2 * h]).astype(np.float32)
            h //= 2
        S = P[0]
    elif order == "sequential":
        S = d[0]
        for v in d[1:]:
            S = np.float32(S + v)
    elif order == "strided":   # P_j = d_j + d_{32+j} + ... + d_{224+j}, then the tree
        P = d[0:32].copy()
        for i in range(1, 8):
            P = (P + d[32 * i:32 * i + 32]).astype(np.float32)
        h = 16
        while h >= 1:
            P[:h] = (P[:h] + P[h:2 * h]).astype(np.float32)
            h //= 2
        S = P[0]
    else:
        raise ValueError(order)
    dbar = np.float32(S * np.float32(2.0 ** -8))
    return int(np.rint(np.float32(dbar * np.float32(r))))


def test_tile_mu_summation_order(oracle):
    # Sec. 4.2.2 takes the tile's floating-point mean; the reading fixes the order of the
    # float32 sum (8-element runs, then a pairwise tree). Tiles with large cancelling terms
    # make the order visible: each one used here gives a different mu under a sequential
    # sum and under the strided order, so a summation order other than the fixed one fails.
    rng = np.random.default_rng(2024)
    found = 0
    for _ in range(4000):
        mag = 2.0 ** rng.integers(0, 31, 256)
        d = (rng.choice([-1.0, 1.0], 256) * mag * rng.uniform(1.0, 2.0, 256)).astype(np.float32)
        r = 1.0
        m_runs = _mu_np(d, r, "runs")
        if m_runs in (_mu_np(d, r, "sequential"), _mu_np(d, r, "strided")):
            continue
        assert oracle.tile_mu(d, r) == m_runs
        found += 1
        if found == 25:
            break
    assert found == 25
    # and on ordinary tiles, with the step of a real field
    for seed in range(40):
        x = inputs.grf((8, 8, 4), seed=seed).ravel() * np.float32(100.0) + np.float32(seed)
        p = oracle.params_for(x, oracle.REL, 1e-4)
        assert oracle.tile_mu(x, p.r) == _mu_np(x, p.r, "runs")


# --------------------------------------------------------------------------- all-core timing driver

@pytest.mark.parametrize("nthreads", [1, 3, 8])
def test_all_core_driver_reproduces_the_oracle(oracle, nthreads):
    # The all-core CPU baseline runs the oracle's functions over element and tile ranges;
    # its streams and reconstructions must be the single-threaded oracle's, byte for byte.
    cases = [(inputs.sinusoids(70001, seed=2), 1e-3, (70001,)),
             (inputs.grf((24, 20, 30), seed=3), 1e-4, (24, 20, 30)),
             (inputs.zero_slabs((10, 16, 40), seed=4), 1e-2, (10, 16, 40)),
             (np.zeros(5, np.float32), 1e-3, (5,))]
    for x, rel, dims in cases:
        ref = oracle.compress(x.ravel(), rel, oracle.REL, dims=dims)
        got = oracle.mt_compress(x.ravel(), rel, oracle.REL, dims=dims, nthreads=nthreads)
        assert got == ref
        y = oracle.mt_decompress(ref, nthreads=nthreads)
        assert np.array_equal(y.view(np.uint32), oracle.decompress(ref).view(np.uint32))
    bad = inputs.sinusoids(3000, seed=5)
    bad[2999] = np.nan
    with pytest.raises(oracle.OracleError) as ei:
        oracle.mt_compress(bad, 1e-3, oracle.REL, nthreads=nthreads)
    assert ei.value.status == oracle.ERR_NONFINITE


# --------------------------------------------------------------------------- second margin tier

def test_params_second_tier(oracle):
    # A field the first tier (eps <= 2^-4) refuses takes the second: Q from A / (2 eb (1 -
    # 2^-1)), eps = (3Q + 4) 2^-23 <= 2^-1, e = eb (1 - eps) rounded toward zero.
    for A, eb in ((1.0, 1.0 / 600000.0), (37.25, 37.25 / 1.2e6), (1.0, 1.0 / 1398000.0)):
        K1 = A / (2 * eb * (1 - 2 ** -4))
        assert math.ceil(K1) + 1 > 174761                     # beyond the first tier
        p = oracle.params(oracle.ABS, eb, -A, A)
        assert p.Q == math.ceil(A / (2 * eb * (1 - 2 ** -1))) + 1
        eps = (3 * p.Q + 4) * 2.0 ** -23
        assert eps <= 0.5
        target = p.eb_eff * (1 - eps)
        e = np.float32(p.e)
        assert float(e) <= target < float(np.nextafter(e, np.float32(np.inf)))
        assert A / (2 * float(e)) < p.Q                       # Q bounds |q|
    with pytest.raises(oracle.OracleError) as ei:              # beyond the second tier
        oracle.params(oracle.ABS, 1.0 / 1.5e6, -1.0, 1.0)
    assert ei.value.status == oracle.ERR_EB_TOO_SMALL
    # the first tier is unchanged where it applies
    p = oracle.params(oracle.ABS, 1.0 / 300000.0, -1.0, 1.0)
    assert p.Q == math.ceil(1.0 / (2 * (1.0 / 300000.0) * (1 - 2 ** -4))) + 1 <= 174761


@pytest.mark.parametrize("eb", [1.0 / 700000.0, 37.25 / 1.3e6])
def test_error_bound_adversarial_midpoints_second_tier(oracle, eb):
    # Bin midpoints +-1, +-2 ulp over the whole range of q of a second-tier field, and the
    # extremes: every reconstruction within eb (exact in float64), the integers round trip.
    A = np.float32(37.25) if eb > 1e-5 else np.float32(1.0)
    p = oracle.params(oracle.ABS, eb, -float(A), float(A))
    assert p.Q > 174761
    s = np.float32(p.s)
    k = np.arange(-p.Q, p.Q + 1, max(1, p.Q // 4000), dtype=np.int64)
    mid = ((k.astype(np.float64) + 0.5) * float(s)).astype(np.float32)
    cand = [mid]
    for ulps in (1, 2):
        cand.append(np.nextafter(mid, np.float32(np.inf)))
        cand.append(np.nextafter(mid, np.float32(-np.inf)))
        mid = cand[-2]
    x = np.concatenate(cand + [np.array([A, -A], np.float32)])
    x = x[np.abs(x) <= A].astype(np.float32)
    st = oracle.compress(x, eb, oracle.ABS)
    y = oracle.decompress(st)
    assert np.abs(x.astype(np.float64) - y.astype(np.float64)).max() <= p.eb
    q = oracle.decompress(st, q=True)
    assert np.array_equal(q, oracle.quantize(x, p.r))
    hdr = np.frombuffer(st[64:64 + 8 * ((x.size + 255) // 256)], np.uint8)
    assert int((hdr & 31).max()) <= 23                         # the rate bound of the tier
    assert len(st) <= oracle.compress_bound(x.size)


def test_offset_field_in_the_second_tier(oracle):
    # A large offset over a small range (A / range ~ 40): REL 1e-4 and 3e-5 need the second
    # tier; REL 1e-5 is beyond it.
    rng = np.random.default_rng(9)
    x = (1.0e4 + rng.normal(0, 30.0, 50000)).astype(np.float32)
    for rel in (1e-4, 3e-5):
        _check_bound(oracle, x, rel, oracle.REL)
        assert oracle.params_for(x, oracle.REL, rel).Q > 174761
    with pytest.raises(oracle.OracleError) as ei:
        oracle.compress(x, 1e-5, oracle.REL)
    assert ei.value.status == oracle.ERR_EB_TOO_SMALL
