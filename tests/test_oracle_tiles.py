"""Pins for the oracle's tile configurations (Sec. 6.5, Table 8): B elements per block,
T blocks per tile.

The configured path costs the four variants by definition, one residual pass each; the
default path uses the single-pass evaluation. The two are separate formulations, so
equal bytes at B = 32, T = 8 cross-check both. A plain numpy decoder, written here from
the format's description, pins the word layout of every configuration.
"""
import numpy as np
import pytest

import oracle as O

pytestmark = pytest.mark.filterwarnings("ignore::RuntimeWarning")


def _field(n, seed=0, offset=280.0):
    rng = np.random.default_rng(seed)
    i = np.arange(n, dtype=np.float64)
    x = offset + 30.0 * np.sin(i / 300.0) + 5.0 * np.sin(i / 17.0) + rng.normal(0, 1e-2, n)
    return x.astype(np.float32)


def _rough(n, seed=1):
    return np.random.default_rng(seed).normal(0, 1, n).astype(np.float32)


@pytest.mark.parametrize("off", [0, O.OFF_LZ2, O.OFF_CENTER, O.OFF_CROSS | O.OFF_CENTER | O.OFF_LZ2])
@pytest.mark.parametrize("rel", [1e-2, 1e-4])
def test_default_configuration_reproduces_the_default_stream(off, rel):
    for x in (_field(37 * 256 + 91), _rough(20 * 256 + 3)):
        assert O.compress_cfg(x, rel, O.REL, 32, 8, off) == O.compress(x, rel, O.REL, features_off=off)


def _np_decode(stream: bytes) -> np.ndarray:
    """The format, decoded with numpy only: preamble, T header bytes per tile, per tile an
    optional float32 mean, per block of rate r > 0 a B-bit sign word and r B-bit planes
    (most significant byte first, element j at bit B - 1 - j); LZ1 / LZ2 inverted from zero
    predecessors at the tile start (and at every block start without the carried state);
    q + mu times the step."""
    info = O.read_preamble(stream)
    n, B, T, off = info["n"], info["B"], info["T"], info["features_off"]
    tile = B * T
    NT = -(-n // tile)
    s = np.float32(info["s"])
    hdr = np.frombuffer(stream[64: 64 + T * NT], np.uint8).reshape(NT, T)
    pos = 64 + T * NT
    out = np.zeros(NT * tile, np.float32)
    for t in range(NT):
        h = hdr[t]
        second, centred = bool(h[0] & 0x80), bool(h[0] & 0x40)
        mu = 0
        if centred:
            mu = int(np.frombuffer(stream[pos: pos + 4], "<f4")[0])
            pos += 4
        l = np.zeros(tile, np.int64)
        for b in range(T):
            r = int(h[b] & 0x1F)
            if r == 0:
                continue
            words = []
            for k in range(r + 1):
                words.append(int.from_bytes(stream[pos: pos + B // 8], "big"))
                pos += B // 8
            bits = lambda w: np.array([(w >> (B - 1 - j)) & 1 for j in range(B)], np.int64)
            mag = sum(bits(words[1 + k]) << k for k in range(r))
            l[b * B:(b + 1) * B] = np.where(bits(words[0]) == 1, -mag, mag)
        q = np.zeros(tile, np.int64)
        p1 = p2 = 0
        for i in range(tile):
            if (off & O.OFF_CROSS) and i % B == 0:
                p1 = p2 = 0
            qh = l[i] + 2 * p1 - p2 if second else l[i] + p1
            p2, p1 = p1, qh
            q[i] = qh + mu
        out[t * tile:(t + 1) * tile] = (q.astype(np.float32) * s).astype(np.float32)
    assert pos == len(stream)
    return out[:n]


@pytest.mark.parametrize("B,T", O.TILE_CONFIGS)
def test_every_configuration_round_trips_and_matches_a_numpy_decoder(B, T):
    for x, rel in ((_field(3000 + 17), 1e-3), (_rough(2000 + 5), 1e-2)):
        s = O.compress_cfg(x, rel, O.REL, B, T)
        info = O.read_preamble(s)
        assert (info["B"], info["T"]) == (B, T) and info["method_word"] == O.tile_word(B, T)
        NT = -(-x.size // (B * T))
        assert len(s) == 64 + T * NT + info["data_bytes"]
        y = O.decompress(s)
        assert np.array_equal(y.view(np.uint32), _np_decode(s).view(np.uint32))
        eb = rel * (float(x.max()) - float(x.min()))
        assert float(np.max(np.abs(y.astype(np.float64) - x))) <= eb


def test_b64_words_by_hand():
    """One 64-element LZ1 block of rate 1: q alternates 0, 1, 0, 1, ... so the residuals
    after the first are -1, +1, ...: sign word 0x5555..., plane 0 all ones but element 0."""
    x = np.tile(np.array([0.0, 1.0], np.float32), 32 * 4)[:256]   # B = 64, T = 4: one tile
    st = O.compress_cfg(x, 0.5, O.ABS, 64, 4, O.OFF_CENTER | O.OFF_LZ2)
    info = O.read_preamble(st)
    assert info["s"] <= 1.0 and (info["B"], info["T"]) == (64, 4)
    hdr = st[64:68]
    assert list(hdr) == [1, 1, 1, 1]
    data = st[68:]
    sign0 = int.from_bytes(data[0:8], "big")
    plane0 = int.from_bytes(data[8:16], "big")
    # element j: residual q_j - q_{j-1}; q = j % 2 (step 1 with eb 0.5 quantizes exactly)
    exp_sign = sum(1 << (63 - j) for j in range(64) if j % 2 == 0 and j > 0)
    exp_plane = sum(1 << (63 - j) for j in range(1, 64))
    assert sign0 == exp_sign and plane0 == exp_plane
    assert len(data) == 4 * 16


def test_longer_tiles_help_smooth_fields():
    """Sec. 6.5: longer chains only help (T = 16 never loses to T = 8 there); B = 64 costs
    CR at a tight bound on rough data."""
    for seed in range(3):
        x = _field(64 * 512, seed=seed)
        for rel in (1e-2, 1e-3, 1e-4):
            assert len(O.compress_cfg(x, rel, O.REL, 32, 16)) <= len(O.compress_cfg(x, rel, O.REL, 32, 8))
    r = _rough(64 * 512)
    assert len(O.compress_cfg(r, 1e-4, O.REL, 64, 4)) > len(O.compress_cfg(r, 1e-4, O.REL, 32, 8))


def test_corrupt_configuration_words():
    x = _field(5000)
    s = bytearray(O.compress_cfg(x, 1e-3, O.REL, 64, 16))
    assert O.decompress_status(bytes(s)) == O.OK
    for bad in (0x200, 0x3000, 0x1300):
        b = bytearray(s)
        b[52:56] = int(bad).to_bytes(4, "little")
        assert O.decompress_status(bytes(b)) == O.ERR_CORRUPT
    b = bytearray(s)                       # read as the default configuration: sizes mismatch
    b[52:56] = (0).to_bytes(4, "little")
    assert O.decompress_status(bytes(b)) == O.ERR_CORRUPT
