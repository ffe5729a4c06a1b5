"""Reconstruction quality on the device (fsz_quality_stats) against the oracle's
(Sec. 6.2, Fig. 8: PSNR against bit rate)."""
import numpy as np
import pytest

from paper_2607_15413_gb300 import inputs

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch.device("cuda:0")


def test_quality_closed_form(fszlib):
    dev = _cuda()
    n = 100_003                                   # not a multiple of 8
    d = ((np.arange(n) % 129) * 0.0625 - 3.0).astype(np.float32)
    a = torch.from_numpy(d).to(dev)
    q = fszlib.quality(a, a + 0.25, eb=0.3, stream_bytes=n // 4)
    assert q["n"] == n and q["over_bound"] == 0
    assert q["max_abs_err"] == 0.25 and q["sum_sq_err"] == n * 0.0625
    assert q["min"] == -3.0 and q["max"] == 5.0
    assert q["psnr_db"] == pytest.approx(20 * np.log10(32.0), abs=1e-12)
    assert q["nrmse"] == pytest.approx(0.25 / 8.0, abs=1e-15)
    assert q["bit_rate"] == pytest.approx(8 * (n // 4) / n)
    assert fszlib.quality(a, a + 0.25, eb=0.2)["over_bound"] == n
    assert np.isinf(fszlib.quality(a, a.clone(), eb=0.1)["psnr_db"])


@pytest.mark.parametrize("n", [1, 7, 8, 9, 4097, 1 << 20, 3 * 8192 + 17])
@pytest.mark.parametrize("rel", [1e-2, 1e-4])
def test_quality_matches_the_oracle(fszlib, oracle, n, rel):
    dev = _cuda()
    x = inputs.sinusoids(n, seed=n % 11)
    xd = torch.from_numpy(x).to(dev)
    try:
        oracle.compress(x, rel, oracle.REL)
    except oracle.OracleError as err:        # a bound too small for a tiny field's values
        assert err.status == oracle.ERR_EB_TOO_SMALL
        return
    sb, nb = fszlib.compress(xd, rel, fszlib.EB_REL)
    y = fszlib.decompress(sb, n=n)
    eb = oracle.params_for(x, oracle.REL, rel).eb
    q = fszlib.quality(xd, y, eb, nb)
    r = oracle.quality(x, y.cpu().numpy(), eb, nb)
    assert q["n"] == r["n"] and q["over_bound"] == r["over_bound"] == 0
    assert q["min"] == r["vmin"] and q["max"] == r["vmax"]
    assert q["max_abs_err"] == pytest.approx(r["max_abs_err"], rel=2.0 ** -23)
    # float32 squares summed over 8 elements, then float64: relative 1e-6 of the exact sum
    assert q["sum_sq_err"] == pytest.approx(r["sum_sq_err"], rel=1e-6)
    if np.isfinite(r["psnr_db"]):
        assert q["psnr_db"] == pytest.approx(r["psnr_db"], abs=1e-5)
    assert q["nrmse"] == pytest.approx(r["nrmse"], rel=1e-6)
    assert q["bit_rate"] == r["bit_rate"]


def test_quality_is_deterministic(fszlib):
    dev = _cuda()
    x = torch.from_numpy(inputs.sinusoids(1 << 22, seed=3)).to(dev)
    y = x + torch.randn_like(x) * 1e-3
    a = fszlib.quality(x, y, 1e-2)
    for _ in range(3):
        assert fszlib.quality(x, y, 1e-2) == a
