"""bench.py's per-configuration mode on the smallest workload (2^20 sinusoids, REL 1e-3):
it runs the value-range pass, the compression and decompression kernels through the C ABI
and prints one JSON line with the stream's ratio, its quality and the per-kernel rates."""
import json
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_config_1_reports_every_kernel():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    r = subprocess.run([sys.executable, "bench.py", "--config", "1", "--steps", "2", "--warmup", "3"],
                       cwd=ROOT, capture_output=True, text=True, timeout=900)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [l for l in r.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["config_run"] == 1 and d["n"] == 1 << 20 and d["steps"] == 2 and d["warmup"] == 3
    assert d["errors_over_bound"] == 0 and d["cr"] > 1.0 and d["psnr_db"] > 0.0
    for k in ("stats", "encode", "decompress"):
        assert d[f"{k}_gbs"] > 0.0 and d[f"{k}_gbs_mean"] > 0.0
