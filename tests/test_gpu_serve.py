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
