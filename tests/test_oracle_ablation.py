"""Pins for the oracle's switched-off features (the ablation of Sec. 6.4, Table 7).

Base = LZ1 with independent blocks (every block restarts from zero predecessors, the
prediction of the block-parallel compressors described in Sec. 2, C1); +Cross = the state
carried across block boundaries (Eq. 2); +Cent. = adaptive centring (Sec. 4.2.2, variants
3-4); +LZ2 = second order (the full method). Checked against closed forms, brute force in
numpy, and the exact invariants of a minimum over a growing candidate set.
"""
import numpy as np
import pytest

import oracle as O

pytestmark = pytest.mark.filterwarnings("ignore::RuntimeWarning")


def _bitlen(x: int) -> int:
    return int(x).bit_length()


def _cost(r: int) -> int:           # Eq. 3
    return 0 if r == 0 else 4 + 4 * r


def _independent_residuals(q: np.ndarray, second: bool) -> np.ndarray:
    """Per 32-element block, zero predecessors at the block's start."""
    out = np.zeros(256, np.int64)
    for b in range(8):
        blk = q[32 * b: 32 * b + 32].astype(np.int64)
        p1 = np.concatenate([[0], blk[:-1]])
        p2 = np.concatenate([[0, 0], blk[:-2]])
        out[32 * b: 32 * b + 32] = blk - 2 * p1 + p2 if second else blk - p1
    return out


def test_independent_block_residuals_closed_form():
    """On a ramp q_i = a + b i: LZ1 gives b everywhere except a block's first element,
    which keeps its raw value; LZ2 gives q_0, q_1 - 2 q_0 at a block's start, then 0."""
    a, b = 1000, 7
    q = (a + b * np.arange(256)).astype(np.int32)
    l1 = O.tile_residuals(q, 0, O.LZ1, O.OFF_CROSS | O.OFF_CENTER)
    exp1 = np.full(256, b)
    exp1[::32] = q[::32]
    assert np.array_equal(l1, exp1)
    l2 = O.tile_residuals(q, 0, O.LZ2, O.OFF_CROSS | O.OFF_CENTER)
    exp2 = np.zeros(256, np.int64)
    exp2[::32] = q[::32]
    exp2[1::32] = q[1::32].astype(np.int64) - 2 * q[::32]
    assert np.array_equal(l2, exp2)
    # with the carried state only the tile's first element(s) are raw
    c1 = O.tile_residuals(q, 0, O.LZ1, 0)
    assert c1[0] == a and np.all(c1[1:] == b)


@pytest.mark.parametrize("seed", range(6))
def test_independent_block_costs_match_brute_force(seed):
    rng = np.random.default_rng(seed)
    scale = [0, 1, 30, 3000, 100000, 174000][seed]
    q = rng.integers(-scale, scale + 1, 256).astype(np.int32) if scale else np.zeros(256, np.int32)
    if seed == 3:                                   # smooth: a quadratic, small curvature
        i = np.arange(256)
        q = (50 + 3 * i + (i * i) // 40).astype(np.int32)
    off = O.OFF_CROSS | O.OFF_CENTER
    for fn_four in (False, True):
        C, rates = O.tile_costs(q, 0, four_pass=fn_four, features_off=off)
        for v, second in ((O.LZ1, False), (O.LZ2, True)):
            l = _independent_residuals(q, second)
            r = [_bitlen(int(np.abs(l[32 * k: 32 * k + 32]).max())) for k in range(8)]
            assert list(rates[v]) == r
            assert int(C[v]) == sum(_cost(x) for x in r)
    C, _ = O.tile_costs(q, 0, four_pass=False, features_off=off)
    assert int(C[O.LZ1C]) == int(C[O.LZ2C]) == 0xFFFFFFFF   # not costed without the state


def test_select_takes_the_cheapest_enabled_variant_first_in_order():
    C = np.array([100, 40, 30, 20], np.uint32)
    assert O.select(C, 0) == O.LZ2C
    assert O.select(C, O.OFF_LZ2) == O.LZ1C
    assert O.select(C, O.OFF_CENTER) == O.LZ2
    assert O.select(C, O.OFF_CENTER | O.OFF_LZ2) == O.LZ1
    assert O.select(np.array([40, 40, 40, 40], np.uint32), 0) == O.LZ1   # ties keep order


def test_feature_sets():
    valid = {0, O.OFF_CENTER, O.OFF_LZ2, O.OFF_CENTER | O.OFF_LZ2, O.OFF_CROSS | O.OFF_CENTER,
             O.OFF_CROSS | O.OFF_CENTER | O.OFF_LZ2}
    for off in range(16):
        assert O.features_valid(off) == (off in valid), off
    x = np.linspace(0, 1, 1000, dtype=np.float32)
    with pytest.raises(O.OracleError):
        O.compress(x, 1e-3, features_off=O.OFF_CROSS)          # centring needs the state
    with pytest.raises(O.OracleError):
        O.compress(x, 1e-3, features_off=O.OFF_LZ2, force_variant=O.LZ2)


def _field(n=64 * 256 + 77, seed=0):
    rng = np.random.default_rng(seed)
    i = np.arange(n, dtype=np.float64)
    x = 280.0 + 30.0 * np.sin(i / 300.0) + 5.0 * np.sin(i / 17.0) + rng.normal(0, 1e-2, n)
    return x.astype(np.float32)


def _headers(stream: bytes, n: int) -> np.ndarray:
    T = (n + 255) // 256
    return np.frombuffer(stream[64: 64 + 8 * T], np.uint8).reshape(T, 8)


@pytest.mark.parametrize("rel", [1e-2, 1e-4])
@pytest.mark.parametrize("off", [o for _, o in O.ABLATION] + [O.OFF_CENTER, O.OFF_CROSS | O.OFF_CENTER])
def test_streams_round_trip_and_record_the_features(off, rel):
    x = _field()
    s = O.compress(x, rel, O.REL, features_off=off)
    info = O.read_preamble(s)
    assert info["features_off"] == off
    y = O.decompress(s)
    eb = rel * (float(x.max()) - float(x.min()))
    assert float(np.max(np.abs(y.astype(np.float64) - x))) <= eb
    h0 = _headers(s, x.size)[:, 0]
    if off & O.OFF_LZ2:
        assert not np.any(h0 & 0x80)
    if off & O.OFF_CENTER:
        assert not np.any(h0 & 0x40)


def test_data_bytes_are_the_minimum_over_the_enabled_variants():
    """The tile data sum to the four-pass (one residual pass per variant, the plain
    definition) minimum over the enabled variants, for every feature set."""
    x = _field(n=24 * 256)
    p = O.params_for(x, O.REL, 1e-3)
    q = O.quantize(x, p.r)
    for _, off in O.ABLATION:
        tot = 0
        for t in range(24):
            d = x[256 * t: 256 * t + 256]
            mu = O.tile_mu(d, p.r)
            C, _ = O.tile_costs(q[256 * t: 256 * t + 256], mu, four_pass=True, features_off=off)
            on = [True, not off & O.OFF_LZ2, not off & O.OFF_CENTER,
                  not off & O.OFF_LZ2 and not off & O.OFF_CENTER]
            tot += min(int(c) for c, e in zip(C, on) if e)
        s = O.compress(x, 1e-3, O.REL, features_off=off)
        assert O.read_preamble(s)["data_bytes"] == tot


def test_more_candidates_never_cost_more():
    """With the same prediction state, each tile takes a minimum over a superset."""
    for seed in range(3):
        x = _field(seed=seed)
        for rel in (1e-2, 1e-3, 1e-4):
            size = {off: len(O.compress(x, rel, O.REL, features_off=off))
                    for off in (0, O.OFF_LZ2, O.OFF_CENTER, O.OFF_CENTER | O.OFF_LZ2)}
            assert size[0] <= size[O.OFF_LZ2] <= size[O.OFF_CENTER | O.OFF_LZ2]
            assert size[0] <= size[O.OFF_CENTER] <= size[O.OFF_CENTER | O.OFF_LZ2]


def test_each_design_helps_where_the_paper_says():
    """Sec. 6.4: the carried state pays on structured fields, centring on fields with a
    large constant offset, the second order at tight bounds on curved data."""
    x = _field()                                      # smooth, offset 280
    cr = {name: 4 * x.size / len(O.compress(x, 1e-4, O.REL, features_off=off))
          for name, off in O.ABLATION}
    assert cr["+cross"] > 1.2 * cr["base"]
    assert cr["+center"] > cr["+cross"]
    assert cr["+lz2"] > cr["+center"]


def test_decoder_rejects_tiles_that_use_switched_off_features():
    x = _field()
    s = bytearray(O.compress(x, 1e-4, O.REL))
    h0 = _headers(bytes(s), x.size)[:, 0]
    assert np.any(h0 & 0x80) and np.any(h0 & 0x40)    # the full method uses both here
    for off in (O.OFF_LZ2, O.OFF_CENTER):
        b = bytearray(s)
        b[52:56] = int(off).to_bytes(4, "little")
        assert O.decompress_status(bytes(b)) == O.ERR_CORRUPT
    for bad in (O.OFF_CROSS, 8, O.OFF_CROSS | O.OFF_LZ2):
        b = bytearray(s)
        b[52:56] = int(bad).to_bytes(4, "little")
        assert O.decompress_status(bytes(b)) == O.ERR_CORRUPT


def test_independent_block_stream_decodes_per_block():
    """A base-mode stream decodes with each block restarted: changing one block's words
    (rate unchanged) changes only that block's reconstruction."""
    x = _field(n=4 * 256)
    off = O.OFF_CROSS | O.OFF_CENTER | O.OFF_LZ2
    s = bytearray(O.compress(x, 1e-3, O.REL, features_off=off))
    q0 = O.decompress(bytes(s), q=True)
    hdr = _headers(bytes(s), x.size)
    rates = (hdr & 0x1F).astype(np.int64)
    # tile 1, block 2: flip one magnitude bit of its first plane
    data0 = 64 + 8 * 4
    t_off = sum(int(sum(4 + 4 * r for r in rates[t] if r)) for t in range(1))
    b_off = sum(4 + 4 * int(r) for r in rates[1][:2] if r)
    assert rates[1][2] > 0
    pos = data0 + t_off + b_off + 4           # the block's plane 0 (after its sign word)
    s[pos] ^= 0x80                            # element 0 of the block
    q1 = O.decompress(bytes(s), q=True)
    diff = np.nonzero(q1 != q0)[0]
    assert diff.size > 0 and diff.min() >= 256 + 64 and diff.max() < 256 + 96


# ---------------------------------------------------------------- quality (Sec. 6.2, Fig. 8)

def test_quality_closed_forms():
    """A constant error c: sum c^2 n, max c, PSNR = 20 log10(range / c); an exact copy:
    infinite PSNR; the bound count; bits per value from the stream size."""
    n = 4096
    d = ((np.arange(n) % 129) * 0.0625 - 3.0).astype(np.float32)   # range 8, d + c exact
    c = np.float32(0.25)
    q = O.quality(d, d + c, eb=0.3, stream_bytes=n // 4)        # 2 bits per value
    assert q["n"] == n and q["over_bound"] == 0
    assert q["max_abs_err"] == 0.25 and q["sum_sq_err"] == n * 0.0625
    assert q["vmin"] == -3.0 and q["vmax"] == 5.0
    assert q["psnr_db"] == pytest.approx(20 * np.log10(8.0 / 0.25), abs=1e-12)
    assert q["nrmse"] == pytest.approx(0.25 / 8.0, abs=1e-15)
    assert q["bit_rate"] == 2.0
    assert O.quality(d, d + c, eb=0.2)["over_bound"] == n
    assert np.isinf(O.quality(d, d.copy(), eb=0.1)["psnr_db"])


def test_quality_matches_numpy_on_a_round_trip():
    x = _field()
    s = O.compress(x, 1e-3, O.REL)
    y = O.decompress(s)
    eb = 1e-3 * (float(x.max()) - float(x.min()))
    q = O.quality(x, y, eb, len(s))
    e = x.astype(np.float64) - y.astype(np.float64)
    assert q["over_bound"] == 0 and q["max_abs_err"] == float(np.abs(e).max()) <= eb
    assert q["sum_sq_err"] == pytest.approx(float(np.sum(e * e)), rel=1e-12)
    rng = float(x.max()) - float(x.min())
    assert q["psnr_db"] == pytest.approx(20 * np.log10(rng) - 10 * np.log10(np.mean(e * e)), abs=1e-9)
    assert q["bit_rate"] == pytest.approx(8 * len(s) / x.size)
    # an error-bounded quantizer with step 2 eb: MSE near (2 eb)^2 / 12 on rough data
    assert 20 * np.log10(rng / (2 * eb / np.sqrt(12))) - 1.5 < q["psnr_db"] < 20 * np.log10(rng / (2 * eb / np.sqrt(12))) + 1.5
