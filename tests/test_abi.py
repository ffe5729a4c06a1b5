"""The C ABI library loads, exports every entry point include/fsz.h declares, and
rejects bad arguments on the host (no GPU needed: these paths make no CUDA call)."""
import ctypes
import os
import re
import subprocess

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    text = open(os.path.join(ROOT, "include", "fsz.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(fsz_[a-z_0-9]+)\s*\(", text)))


def test_header_and_exports_agree(fszlib):
    decl = declared_functions()
    assert decl == sorted(fszlib.EXPORTS)
    out = subprocess.run(["nm", "-D", "--defined-only", fszlib.LIB_PATH], capture_output=True,
                         text=True, check=True).stdout
    exported = set(re.findall(r"\bT (fsz_\w+)", out))
    missing = [f for f in decl if f not in exported]
    assert not missing, missing
    L = fszlib.lib()
    for f in decl:
        assert hasattr(L, f)
    assert fszlib.fsz_version().endswith("sm_103a")


def test_sizes_match_format(fszlib, oracle):
    for n in (0, 1, 255, 256, 257, 10 ** 6, 1 << 27):
        assert fszlib.fsz_compress_bound(n) == oracle.compress_bound(n)
        # control block, one field record, 12 bytes per 16-tile chunk (map + lookback flag)
        assert fszlib.fsz_workspace_bytes(n) >= 256 + 12 * ((n + 255) // 256 // 16)
    assert fszlib.fsz_batch_workspace_bytes(1 << 20, 64) > fszlib.fsz_workspace_bytes(1 << 20)


def test_read_header_on_oracle_stream(fszlib, oracle):
    from paper_2607_15413_gb300 import inputs
    x = inputs.grf((20, 30, 40), seed=3)
    s = oracle.compress(x, 1e-3, oracle.REL, dims=(20, 30, 40))
    h = fszlib.fsz_read_header(s[:64])
    assert h["n"] == x.size and h["dims"] == (20, 30, 40) and h["eb"] == 1e-3
    assert h["total_bytes"] == len(s)
    assert np.float32(h["step"]) == np.float32(oracle.params_for(x, oracle.REL, 1e-3).s)
    with pytest.raises(fszlib.FszError):
        fszlib.fsz_read_header(b"XXXX" + s[4:64])


def test_host_argument_errors(fszlib):
    L = fszlib.lib()
    D = fszlib.make_dims
    good = (0x10000, D((1000,)), 1, 1e-3, 0x20000, 1 << 20, 0, 0x30000, 1 << 24, 0)
    def call(**kw):
        args = list(good)
        names = ["d_in", "dims", "mode", "eb", "d_out", "cap", "nb", "d_ws", "ws_bytes", "stream"]
        for k, v in kw.items():
            args[names.index(k)] = v
        return L.fsz_compress(*args)
    bad_dims = fszlib.FszDims()
    bad_dims.ndim = 4
    assert call(dims=bad_dims) == fszlib.ERR_INVALID_ARG
    assert call(mode=7) == fszlib.ERR_INVALID_ARG
    for eb in (0.0, -1.0, float("nan"), float("inf")):
        assert call(eb=eb) == fszlib.ERR_INVALID_ARG
    assert call(d_in=0x10004) == fszlib.ERR_ALIGN
    assert call(d_out=0x20008) == fszlib.ERR_ALIGN
    assert call(cap=64 + 8 * 3) == fszlib.ERR_CAPACITY      # below 64 + 8T
    assert call(ws_bytes=64) == fszlib.ERR_WORKSPACE
    assert L.fsz_decompress(0x10004, 100, 0x20000, 10, 0x30000, 1 << 20, 0) == fszlib.ERR_ALIGN
    assert L.fsz_decompress(0x10000, 100, 0x20000, 1 << 30, 0x30000, 16, 0) == fszlib.ERR_WORKSPACE
    assert L.fsz_compress_batched(0, 3, 100, 0x30000, 1 << 20, 0) == fszlib.ERR_INVALID_ARG
