"""Tile configurations of Sec. 6.5 (Table 8) on the CUDA path vs the CPU oracle: every
(B, T), streams byte for byte and reconstructions bit for bit."""
import numpy as np
import pytest

from paper_2607_15413_gb300 import inputs

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

CONFIGS = [(32, 4), (32, 8), (32, 16), (64, 4), (64, 8), (64, 16)]


def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch.device("cuda:0")


FIELDS = {
    "offset": lambda n, s: (10.0 * inputs.sinusoids(n, seed=s) + 280.0).astype(np.float32),
    "particles": lambda n, s: inputs.particles(n, seed=s, ncenters=max(4, n // 2048)),
    "zero_slabs": lambda n, s: inputs.zero_slabs((max(24, -(-n // 4096)), 64, 64), seed=s).ravel()[:n],
}


def _parity(fszlib, oracle, x, rel, B, T, off=0):
    dev = _cuda()
    ref = oracle.compress_cfg(x, rel, oracle.REL, B, T, off)
    xd = torch.from_numpy(np.ascontiguousarray(x)).to(dev)
    sb, nb = fszlib.compress_tiled(xd, rel, fszlib.EB_REL, B, T, off)
    got = sb.cpu().numpy().tobytes()
    assert len(got) == len(ref), (len(got), len(ref))
    if got != ref:
        a, b = np.frombuffer(got, np.uint8), np.frombuffer(ref, np.uint8)
        raise AssertionError(f"stream differs first at byte {int(np.nonzero(a != b)[0][0])} of {len(ref)}")
    y = fszlib.decompress_tiled(sb, x.size).cpu().numpy()
    assert np.array_equal(y.view(np.uint32), oracle.decompress(ref).view(np.uint32))
    return ref


@pytest.mark.parametrize("B,T", CONFIGS)
@pytest.mark.parametrize("field", sorted(FIELDS))
def test_configurations_match_the_oracle(fszlib, oracle, field, B, T):
    x = FIELDS[field](4096 * 24, 5)
    for rel in (1e-2, 1e-3):
        _parity(fszlib, oracle, x, rel, B, T)


@pytest.mark.parametrize("B,T", CONFIGS)
@pytest.mark.parametrize("n", [1, 127, 129, 1025, 8193, 3 * 8192 + 17])
def test_configurations_ragged(fszlib, oracle, B, T, n):
    _parity(fszlib, oracle, FIELDS["offset"](n, n % 7), 1e-3, B, T)


@pytest.mark.parametrize("B,T", [(32, 16), (64, 8)])
@pytest.mark.parametrize("off", [2, 4, 6, 7])
def test_configurations_with_switched_off_features(fszlib, oracle, B, T, off):
    _parity(fszlib, oracle, FIELDS["offset"](20000, 3), 1e-3, B, T, off)


def test_default_configuration_through_the_generic_path_is_the_default_stream(fszlib, oracle):
    dev = _cuda()
    x = FIELDS["particles"](70001, 2)
    xd = torch.from_numpy(x).to(dev)
    a, _ = fszlib.compress_tiled(xd, 1e-3, fszlib.EB_REL, 32, 8)
    b, _ = fszlib.compress(xd, 1e-3, fszlib.EB_REL)
    assert torch.equal(a, b)
    y = fszlib.decompress_tiled(b, x.size)            # the generic decoder takes default streams
    assert torch.equal(y, fszlib.decompress(b, n=x.size))


def test_the_default_decoder_refuses_configured_streams(fszlib, oracle):
    dev = _cuda()
    x = FIELDS["offset"](5000, 1)
    sb, _ = fszlib.compress_tiled(torch.from_numpy(x).to(dev), 1e-3, fszlib.EB_REL, 64, 8)
    with pytest.raises(fszlib.FszError) as e:
        fszlib.decompress(sb, n=x.size)
    assert e.value.status == fszlib.ERR_INVALID_ARG
