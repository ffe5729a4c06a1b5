"""The continuous-batching request loop on the GPU: every result in the mix equals the
same request run alone (fsz_compress / fsz_decompress of that field), bit for bit, while
batches overlap on the device and requests are admitted as others run."""
import random
import threading
import time

import numpy as np
import pytest

from paper_2607_15413_gb300 import inputs

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def test_results_alone_equal_results_in_the_mix(fszlib):
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2607_15413_gb300.serve import COMPRESS, DECOMPRESS, Request, Server
    dev = torch.device("cuda:0")
    pool = [torch.from_numpy(inputs.sinusoids(1 << 22, seed=1)).to(dev),
            inputs.particles(1 << 22, seed=2, device="cuda"),
            inputs.zero_slabs((64, 256, 256), seed=3, device="cuda").reshape(-1).contiguous()]
    rng = random.Random(0)
    reqs = []
    for i in range(90):
        src = pool[i % 3]
        n = int(2 ** rng.uniform(12, 21))
        off = rng.randrange(0, (src.numel() - n) // 4) * 4
        x = src[off:off + n]
        reqs.append((x, (n,), rng.choice([1e-2, 1e-3, 1e-4])))
    # alone (a window with a large offset and a small range can be refused: REL x range is
    # then below what float32 quantization can hold; the mix must report the same status)
    alone, status = [], []
    for x, shape, eb in reqs:
        try:
            sb, nb = fszlib.compress(x, eb, fszlib.EB_REL, shape=shape)
            alone.append(sb.clone())
            status.append(0)
        except fszlib.FszError as err:
            alone.append(None)
            status.append(err.status)
    assert status.count(0) >= len(reqs) * 2 // 3
    alone_dec = [fszlib.decompress(s, n=x.numel()).clone() if s is not None else None
                 for s, (x, _, _) in zip(alone, reqs)]
    # in the mix: 60 % compress, 40 % decompress of an earlier result, from 3 client threads
    srv = Server(budget_bytes=256 << 20, n_slots=4, max_batch=16,
                 max_batch_elems=sum(x.numel() for x, _, _ in reqs))
    futs = [None] * len(reqs)

    def client(k):
        r = random.Random(k)
        for i in range(k, len(reqs), 3):
            x, shape, eb = reqs[i]
            if i % 5 < 3 or alone[i] is None:
                req = Request(kind=COMPRESS, data=x, shape=shape, eb=eb, mode=1)
            else:
                req = Request(kind=DECOMPRESS, data=alone[i], n=x.numel())
            futs[i] = srv.submit(req)
            time.sleep(r.uniform(0, 0.002))

    ts = [threading.Thread(target=client, args=(k,)) for k in range(3)]
    try:
        for t in ts:
            t.start()
        for t in ts:
            t.join()
        res = [f.result(timeout=60) for f in futs]
        for i, r in enumerate(res):
            assert r.status == status[i], (i, r.status, status[i])
            if status[i]:
                r.release()
                continue
            if i % 5 < 3:
                assert r.nbytes == alone[i].numel()
                assert torch.equal(r.tensor(torch.uint8), alone[i]), f"request {i}: compressed stream differs"
            else:
                got = r.tensor(torch.float32)
                assert torch.equal(got.view(torch.int32), alone_dec[i].view(torch.int32)), f"request {i}"
            r.release()
        st = srv.stats()
    finally:
        srv.close()
    assert st["completed"] == len(reqs)
    assert st["max_inflight"] >= 2
    assert st["admitted_while_busy"] > 0
    assert st["budget_free"] == 256 << 20


def _serve_table(fszlib, srv, table, keep_ids, on_kept):
    """Submits a request table at once (a closed loop), collects every completion, hands
    each kept one to on_kept(completion) before releasing it, releases the rest at once.
    Returns {id: status}."""
    L = fszlib.lib()
    code = L.fsz_server_submit_many(srv._h, table.ctypes.data, len(table))
    assert code == 0, code
    buf = np.zeros(4096, dtype=fszlib.COMPLETION_NP)
    status = {}
    while len(status) < len(table):
        k = L.fsz_server_poll(srv._h, buf.ctypes.data, len(buf), 2_000_000)
        done = []
        for c in buf[:k].copy():
            rid = int(c["id"])
            status[rid] = int(c["status"])
            if c["status"] == fszlib.ERR_REJECTED:
                continue
            if rid in keep_ids and c["status"] == 0:
                on_kept(c)
            done.append(rid)
        if done:
            ids = np.array(done, np.uint64)
            assert L.fsz_server_release_many(srv._h, ids.ctypes.data, len(ids), None) == 0
    return status


def _to_host(fszlib, c):
    t = torch.empty(int(c["out_bytes"]), dtype=torch.uint8, device="cuda")
    st = torch.cuda.current_stream()
    assert fszlib.lib().fsz_copy_device(t.data_ptr(), int(c["d_out"]), int(c["out_bytes"]),
                                        st.cuda_stream) == 0
    return t.cpu().numpy()


def test_config5_served_trace_against_the_oracle(fszlib, oracle):
    """The serving workload through the native server (seed 4; 20,000 requests of
    log-uniform 16 KiB - 256 MiB windows of a device pool of the batched mix's classes,
    60 % compress / 40 % decompress of one of 64 earlier streams, REL from {1e-2, 1e-3,
    1e-4}, 40 GB budget, 4 streams, batches of up to 32) as one closed loop. Checked against
    the oracle (stream byte for byte, reconstruction bit for bit, refusals by status): every
    request of at most 4 MiB, and 500 requests at evenly spaced ranks of size over the whole
    range; the 64 source streams too."""
    import concurrent.futures as cf
    import os
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2607_15413_gb300.serve import Server
    pool = inputs.serving_pool(seed=4, device="cuda")
    numels = [p.numel() for p in pool]
    host_pool = [p.cpu().numpy() for p in pool]
    rng = random.Random(4)
    srv = Server(budget_bytes=40 << 30, n_slots=4, max_batch=32, max_batch_elems=4 << 30,
                 linger_s=200e-6, futures=False)
    ex = cf.ThreadPoolExecutor(max_workers=max(2, min(16, os.cpu_count() or 2)))
    try:
        # the 64 source streams, kept on the host
        src_rows = inputs.serving_windows(rng, numels, 64)
        t = np.zeros(len(src_rows), dtype=fszlib.REQUEST_NP)
        t["id"] = np.arange(1, len(src_rows) + 1)
        for j, (k, off, n, rel) in enumerate(src_rows):
            t[j]["kind"], t[j]["mode"], t[j]["ndim"], t[j]["d0"] = fszlib.REQ_COMPRESS, 1, 1, n
            t[j]["eb"], t[j]["d_in"] = rel, pool[k].data_ptr() + 4 * off
        t["arrival_ns"] = time.monotonic_ns()
        src_host = {}
        st = _serve_table(fszlib, srv, t, set(int(i) for i in t["id"]),
                          lambda c: src_host.__setitem__(int(c["id"]), _to_host(fszlib, c)))

        def ref_compress(k, off, n, rel):
            try:
                return 0, oracle.compress(host_pool[k][off:off + n], rel, oracle.REL, dims=(n,))
            except oracle.OracleError as err:
                return err.status, None

        src_refs = list(ex.map(lambda r: ref_compress(*r), src_rows))
        sources = []   # (device stream pointer, bytes, n, oracle stream) of accepted sources
        for j, (k, off, n, rel) in enumerate(src_rows):
            rid = j + 1
            assert st[rid] == src_refs[j][0], (rid, st[rid], src_refs[j][0])
            if st[rid] == 0:
                assert src_host[rid].tobytes() == src_refs[j][1], f"source {rid}"
                dev_stream = torch.from_numpy(src_host[rid].copy()).to("cuda")
                sources.append((dev_stream, n, src_refs[j][1]))
        assert len(sources) >= 48
        dec_refs = list(ex.map(lambda s: oracle.decompress(s[2]), sources))

        # the closed-loop trace
        rows = inputs.serving_trace(rng, numels, 20000, len(sources))
        t = np.zeros(len(rows), dtype=fszlib.REQUEST_NP)
        t["id"] = np.arange(1000, 1000 + len(rows))
        sizes = np.zeros(len(rows), np.int64)
        for j, row in enumerate(rows):
            if row[0] == "decompress":
                s_dev, n, _ = sources[row[1]]
                t[j]["kind"], t[j]["d_in"] = fszlib.REQ_DECOMPRESS, s_dev.data_ptr()
                t[j]["in_bytes"], t[j]["n"] = s_dev.numel(), n
            else:
                _, k, off, n, rel = row
                t[j]["kind"], t[j]["mode"], t[j]["ndim"], t[j]["d0"] = fszlib.REQ_COMPRESS, 1, 1, n
                t[j]["eb"], t[j]["d_in"] = rel, pool[k].data_ptr() + 4 * off
            sizes[j] = n
        t["arrival_ns"] = time.monotonic_ns()
        order = np.argsort(sizes, kind="stable")
        picked = set(int(order[int(round(i))]) for i in np.linspace(0, len(rows) - 1, 500))
        picked |= set(int(j) for j in np.nonzero(sizes <= (1 << 20))[0])
        assert len(picked) >= 500 + 1000
        keep = set(1000 + j for j in picked)
        served = {}
        st = _serve_table(fszlib, srv, t, keep,
                          lambda c: served.__setitem__(int(c["id"]) - 1000, _to_host(fszlib, c)))
        assert len(st) == len(rows)

        def check(j):
            row = rows[j]
            if row[0] == "decompress":
                if st[1000 + j] != 0:
                    return f"request {j}: decompress status {st[1000 + j]}"
                y = served[j].view(np.float32)
                if not np.array_equal(y.view(np.uint32), dec_refs[row[1]].view(np.uint32)):
                    return f"request {j}: reconstruction differs from the oracle decoder"
                return None
            code, ref = ref_compress(*row[1:])
            if st[1000 + j] != code:
                return f"request {j}: status {st[1000 + j]}, oracle {code}"
            if code == 0 and served[j].tobytes() != ref:
                return f"request {j}: stream differs from the oracle"
            return None

        bad = [m for m in ex.map(check, sorted(picked)) if m]
        assert not bad, bad[:5]
        assert srv.stats()["budget_free"] == 40 << 30
    finally:
        ex.shutdown(wait=True)
        srv.close()
