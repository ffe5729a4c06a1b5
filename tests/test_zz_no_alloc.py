"""fsz_compress_noalloc against fsz_compress (GB300 only).

The no-allocation entry point serves callers that cannot allocate device memory
(for example a plugin whose framework owns all device memory, or a latency-critical
path that cannot take the synchronisation an allocation may cause). It must produce the same stream as the regular
entry point, byte for byte (the tolerance of every parity test here is 0), on two
calls in a row, because the built-in scratch array keeps the previous call's
contents and each call must clear what it relies on. This file is collected last so
that a run stopping at the first failure has already run every other test.
"""
import numpy as np
import pytest

from paper_2607_15413_gb300 import inputs

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def _noalloc(fszlib, xd, shape, rel):
    n = xd.numel()
    cap = fszlib.fsz_compress_bound(n)
    out = torch.zeros(cap, dtype=torch.uint8, device=xd.device)
    nb = torch.zeros(1, dtype=torch.int64, device=xd.device)
    status = torch.full((1,), 12345, dtype=torch.int32, device=xd.device)
    sp = torch.cuda.current_stream().cuda_stream
    st = fszlib.fsz_compress_noalloc(xd.data_ptr(), fszlib.make_dims(shape), fszlib.EB_REL, rel,
                                     out.data_ptr(), cap, nb.data_ptr(), status.data_ptr(), sp)
    assert st == fszlib.OK
    torch.cuda.synchronize()
    assert int(status.item()) == fszlib.OK
    k = int(nb.item())
    return out[:k].cpu().numpy().tobytes()


def test_noalloc_matches_regular_entry_point_twice(fszlib):
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    dev = torch.device("cuda:0")
    # Two different fields back to back: stale scratch from the first call (lookback
    # flags, tickets, value range) would corrupt the second if it were not cleared.
    a = torch.from_numpy(inputs.particles(40 * 8192 + 999, seed=11, ncenters=128)).to(dev)
    b = torch.from_numpy(inputs.zero_slabs((24, 64, 96), seed=12).ravel()).to(dev)
    for x, shape, rel in ((a, (a.numel(),), 1e-4), (b, (24, 64, 96), 1e-3)):
        got = _noalloc(fszlib, x, shape, rel)
        ref, nb = fszlib.compress(x, rel, fszlib.EB_REL, shape=shape)
        assert got == ref.cpu().numpy().tobytes()
        y = fszlib.decompress(ref, n=x.numel())
        assert np.array_equal(y.cpu().numpy(), fszlib.decompress(
            torch.from_numpy(np.frombuffer(got, np.uint8).copy()).to(dev), n=x.numel()).cpu().numpy())


def test_noalloc_rejects_fields_beyond_its_scratch(fszlib):
    dims = fszlib.make_dims((1 << 14, 1 << 14, 2))   # 2^29 elements > FSZ_NOALLOC_MAX_ELEMS
    st = fszlib.fsz_compress_noalloc(0x10000, dims, fszlib.EB_REL, 1e-3, 0x20000, 1 << 40, 0, 0, 0)
    assert st == fszlib.ERR_WORKSPACE


def test_noalloc_inside_a_global_mode_capture(fszlib):
    """The entry point's use inside a stream capture in global mode: after one call outside
    any capture (the device's one-time set-up), a captured call replays to the regular
    entry point's stream, and replays again after the input changes in place."""
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    dev = torch.device("cuda:0")
    n = 24 * 8192 + 321
    x = torch.from_numpy(inputs.particles(n, seed=13, ncenters=64)).to(dev)
    x2 = torch.from_numpy(inputs.sinusoids(n, seed=14)).to(dev)
    cap = fszlib.fsz_compress_bound(n)
    out = torch.zeros(cap, dtype=torch.uint8, device=dev)
    nb = torch.zeros(1, dtype=torch.int64, device=dev)
    status = torch.full((1,), 12345, dtype=torch.int32, device=dev)
    dims = fszlib.make_dims((n,))

    def call(stream_ptr):
        return fszlib.fsz_compress_noalloc(x.data_ptr(), dims, fszlib.EB_REL, 1e-3, out.data_ptr(), cap,
                                           nb.data_ptr(), status.data_ptr(), stream_ptr)

    assert call(torch.cuda.current_stream().cuda_stream) == fszlib.OK   # outside any capture
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    side = torch.cuda.Stream(dev)
    side.wait_stream(torch.cuda.current_stream())
    with torch.cuda.graph(g, stream=side, capture_error_mode="global"):
        st = call(torch.cuda.current_stream().cuda_stream)
    assert st == fszlib.OK
    for src in (None, x2):
        if src is not None:
            x.copy_(src)                  # the graph reads the same input pointer
        ref, k = fszlib.compress(x, 1e-3, fszlib.EB_REL)
        out.zero_()
        nb.zero_()
        status.fill_(12345)
        torch.cuda.synchronize()
        g.replay()
        torch.cuda.synchronize()
        assert int(status.item()) == fszlib.OK
        assert int(nb.item()) == k
        assert out[:k].cpu().numpy().tobytes() == ref.cpu().numpy().tobytes()
