"""No writes outside the outputs (a stand-in for a memory sanitizer, which is not
available): every output and workspace sits between sentinel-filled guard regions, and
the bytes of an output past what the call produced must keep their sentinel too."""
import numpy as np
import pytest

from paper_2607_15413_gb300 import inputs

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

G = 4096            # guard bytes on each side (keeps 16-byte alignment)
SENT = 0xA5


def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch.device("cuda:0")


def _guarded(nbytes, dev):
    buf = torch.full((nbytes + 2 * G,), SENT, dtype=torch.uint8, device=dev)
    return buf, buf[G:G + nbytes]


def _intact(buf, lo, hi):
    """Sentinel everywhere outside [lo, hi) of the guarded buffer's payload."""
    b = buf.cpu().numpy()
    return bool(np.all(b[:G + lo] == SENT) and np.all(b[G + hi:] == SENT))


@pytest.mark.parametrize("n", [1, 33, 257, 8193, 65539, 3 * 8192 + 17])
def test_single_field_paths_write_only_their_outputs(fszlib, oracle, n):
    dev = _cuda()
    x = torch.from_numpy((10.0 * inputs.sinusoids(n, seed=n % 5) + 3.0).astype(np.float32)).to(dev)
    sp = torch.cuda.current_stream().cuda_stream
    L = fszlib.lib()
    cap = fszlib.fsz_compress_bound(n)
    obuf, out = _guarded(cap, dev)
    wsb = fszlib.fsz_workspace_bytes(n)
    wbuf, ws = _guarded(wsb, dev)
    nb = torch.zeros(2, dtype=torch.int64, device=dev)
    assert L.fsz_compress(x.data_ptr(), fszlib.make_dims((n,)), fszlib.EB_REL, 1e-3, out.data_ptr(), cap, nb.data_ptr(),
                          ws.data_ptr(), wsb, sp) == 0
    assert fszlib.fsz_check(ws.data_ptr(), sp) == 0
    k = int(nb[0].item())
    assert _intact(obuf, 0, k) and _intact(wbuf, 0, wsb)
    # decompress into a guarded float output with a guarded workspace
    dbuf, dout = _guarded(4 * n, dev)
    wbuf2, ws2 = _guarded(fszlib.fsz_workspace_bytes(n), dev)
    assert L.fsz_decompress(out.data_ptr(), k, dout.data_ptr(), n, ws2.data_ptr(), ws2.numel(), sp) == 0
    assert fszlib.fsz_check(ws2.data_ptr(), sp) == 0
    assert _intact(dbuf, 0, 4 * n) and _intact(wbuf2, 0, ws2.numel())
    y = dout.view(torch.float32).cpu().numpy()
    ref = oracle.decompress(oracle.compress(x.cpu().numpy(), 1e-3, oracle.REL))
    assert np.array_equal(y.view(np.uint32), ref.view(np.uint32))


@pytest.mark.parametrize("B,T", [(32, 4), (64, 16)])
def test_tiled_and_multipass_paths_write_only_their_outputs(fszlib, B, T):
    dev = _cuda()
    n = 20011
    x = torch.from_numpy((10.0 * inputs.sinusoids(n, seed=2) + 3.0).astype(np.float32)).to(dev)
    sp = torch.cuda.current_stream().cuda_stream
    L = fszlib.lib()
    cap = L.fsz_compress_bound_tiled(n, B, T)
    obuf, out = _guarded(cap, dev)
    wsb = L.fsz_tiled_workspace_bytes(n)
    wbuf, ws = _guarded(wsb, dev)
    nb = torch.zeros(2, dtype=torch.int64, device=dev)
    assert L.fsz_compress_tiled(x.data_ptr(), fszlib.make_dims((n,)), fszlib.EB_REL, 1e-3, B, T, 0, out.data_ptr(), cap,
                                nb.data_ptr(), ws.data_ptr(), wsb, sp) == 0
    assert fszlib.fsz_check(ws.data_ptr(), sp) == 0
    k = int(nb[0].item())
    assert _intact(obuf, 0, k) and _intact(wbuf, 0, wsb)
    dbuf, dout = _guarded(4 * n, dev)
    wbuf2, ws2 = _guarded(L.fsz_tiled_workspace_bytes(n), dev)
    assert L.fsz_decompress_tiled(out.data_ptr(), k, dout.data_ptr(), n, ws2.data_ptr(), ws2.numel(), sp) == 0
    assert fszlib.fsz_check(ws2.data_ptr(), sp) == 0
    assert _intact(dbuf, 0, 4 * n) and _intact(wbuf2, 0, ws2.numel())
    # multipass: its cost arrays (4 T uint32 for 256-element tiles) are guarded too
    T256 = (n + 255) // 256
    cbuf, costs = _guarded(16 * T256, dev)
    cap2 = fszlib.fsz_compress_bound(n)
    obuf2, out2 = _guarded(cap2, dev)
    wsb3 = fszlib.fsz_workspace_bytes(n)
    wbuf3, ws3 = _guarded(wsb3, dev)
    assert L.fsz_compress_multipass(x.data_ptr(), fszlib.make_dims((n,)), fszlib.EB_REL, 1e-3, out2.data_ptr(), cap2,
                                    nb.data_ptr(), costs.data_ptr(), ws3.data_ptr(), wsb3, sp) == 0
    assert fszlib.fsz_check(ws3.data_ptr(), sp) == 0
    k2 = int(nb[0].item())
    assert _intact(obuf2, 0, k2) and _intact(cbuf, 0, 16 * T256) and _intact(wbuf3, 0, wsb3)


def test_batched_paths_write_only_their_outputs(fszlib):
    dev = _cuda()
    sizes = [1, 300, 9000, 70001]
    xs = [torch.from_numpy((10.0 * inputs.sinusoids(m, seed=m % 3) + 3.0).astype(np.float32)).to(dev)
          for m in sizes]
    b = fszlib.CompressBatch([(x, (x.numel(),), fszlib.EB_REL, 1e-3) for x in xs], device=dev)
    # guard the arena's unused tail of every slot by pre-filling it
    b.arena.fill_(SENT)
    assert b.run() == 0
    st, per = b.status()
    assert st == 0
    arena = b.arena.cpu().numpy()
    ks = b.sizes.cpu().tolist()
    for i in range(len(sizes)):
        lo, hi = b.offsets[i] + ks[i], b.offsets[i + 1]
        assert np.all(arena[lo:hi] == SENT), i
