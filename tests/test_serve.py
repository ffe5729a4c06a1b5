"""Scheduling rules of the continuous-batching request loop, on the CPU with a fake
backend whose batches take a fixed time (no GPU)."""
import random
import threading
import time

import pytest

from paper_2607_15413_gb300.serve import COMPRESS, DECOMPRESS, Request, Server


class _Data:
    def __init__(self, n):
        self.n = n

    def numel(self):
        return self.n


class FakeBackend:
    """Batches complete `service_s` after launch; records launches for inspection."""

    def __init__(self, service_s=0.02):
        self.service_s = service_s
        self.launches = []
        self.lock = threading.Lock()

    def cost(self, req):
        return req.n * 4 if req.kind == DECOMPRESS else req.data.numel() * 4

    def launch(self, slot, kind, reqs):
        with self.lock:
            self.launches.append((time.perf_counter(), slot, kind, [r.seq for r in reqs]))
        return {"t_done": time.perf_counter() + self.service_s}

    def done(self, h):
        return time.perf_counter() >= h["t_done"]

    def results(self, h, reqs):
        return [(0, None, 0) for _ in reqs]


def creq(n, kind=COMPRESS):
    if kind == COMPRESS:
        return Request(kind=COMPRESS, data=_Data(n), shape=(n,))
    return Request(kind=DECOMPRESS, data=_Data(8), n=n)


def test_oversize_request_is_rejected_at_once():
    srv = Server(FakeBackend(), budget_bytes=1000, n_slots=2)
    try:
        r = srv.submit(creq(1000)).result(timeout=5)   # 4000 bytes > budget
        assert r.status == -1
        ok = srv.submit(creq(100)).result(timeout=5)
        assert ok.status == 0
    finally:
        srv.close()
    assert srv.stats["rejected"] == 1 and srv.stats["completed"] == 1


def test_budget_admits_in_arrival_order_without_overtaking():
    be = FakeBackend(service_s=0.05)
    srv = Server(be, budget_bytes=1000, n_slots=4, max_batch=8)
    try:
        a = srv.submit(creq(200))       # 800 bytes
        b = srv.submit(creq(150))       # 600: does not fit next to a, must wait
        c = srv.submit(creq(10))        # 40: would fit, but must not overtake b
        for f in (a, b, c):
            assert f.result(timeout=5).status == 0
    finally:
        srv.close()
    order = [seqs for _, _, _, seqs in be.launches]
    flat = [s for seqs in order for s in seqs]
    assert flat == sorted(flat)                                   # launched in arrival order
    assert order[0] == [0] and 1 in order[1]                      # b waited for a's memory


def test_continuous_batching_admits_while_batches_run():
    be = FakeBackend(service_s=0.03)
    srv = Server(be, budget_bytes=10 ** 9, n_slots=3, max_batch=4)
    futs = []
    try:
        for i in range(24):
            futs.append(srv.submit(creq(1000 + i)))
            time.sleep(0.004)            # arrivals keep coming while batches run
        for f in futs:
            assert f.result(timeout=10).status == 0
    finally:
        srv.close()
    assert srv.stats["max_inflight"] >= 2            # batches overlapped
    assert srv.stats["admitted_while_busy"] > 0      # admitted during others' execution
    assert srv.stats["max_batch_seen"] <= 4
    lat = [f.result().latency_s for f in futs]
    assert min(lat) >= 0.03 - 1e-3                   # at least one service time


def test_batches_are_homogeneous_in_kind():
    be = FakeBackend(service_s=0.02)
    srv = Server(be, budget_bytes=10 ** 9, n_slots=1, max_batch=16)
    try:
        fs = [srv.submit(creq(100 + i, COMPRESS if i % 3 else DECOMPRESS)) for i in range(30)]
        for f in fs:
            f.result(timeout=10)
    finally:
        srv.close()
    kinds = {}
    for r_i in range(30):
        kinds[r_i] = COMPRESS if r_i % 3 else DECOMPRESS
    for _, _, kind, seqs in be.launches:
        assert all(kinds[s] == kind for s in seqs)


def test_random_load_never_deadlocks():
    rng = random.Random(0)
    be = FakeBackend(service_s=0.002)
    srv = Server(be, budget_bytes=400_000, n_slots=4, max_batch=8)
    futs = []

    def client(seed):
        r = random.Random(seed)
        for _ in range(50):
            n = int(10 ** r.uniform(1, 5.2))             # some exceed the budget (rejected)
            futs.append(srv.submit(creq(n, r.choice([COMPRESS, DECOMPRESS]))))
            time.sleep(r.uniform(0, 0.002))

    ts = [threading.Thread(target=client, args=(rng.random(),)) for _ in range(4)]
    try:
        for t in ts:
            t.start()
        for t in ts:
            t.join()
        res = [f.result(timeout=30) for f in futs]
    finally:
        srv.close()
    assert len(res) == 200
    assert srv.stats["completed"] + srv.stats["rejected"] == 200
    assert srv.free_budget == srv.budget                  # every admitted byte returned


def test_batches_reach_past_the_other_kind():
    """Alternating kinds still form full batches of each kind, in arrival order per kind."""
    be = FakeBackend(service_s=0.05)
    srv = Server(be, budget_bytes=10 ** 9, n_slots=1, max_batch=8)
    try:
        first = srv.submit(creq(100))                 # occupies the only slot
        time.sleep(0.01)
        fs = [srv.submit(creq(100 + i, COMPRESS if i % 2 else DECOMPRESS)) for i in range(16)]
        for f in [first] + fs:
            assert f.result(timeout=10).status == 0
    finally:
        srv.close()
    sizes = [len(seqs) for _, _, _, seqs in be.launches]
    assert sizes[0] == 1 and sizes[1:] == [8, 8]      # two full batches, one per kind
    for _, _, _, seqs in be.launches:
        assert seqs == sorted(seqs)


def test_a_skipped_request_keeps_its_memory():
    """A batch reaches past a request of the other kind only with memory to spare for it:
    a later request that would fit only by spending the skipped request's memory waits."""
    def run(z_elems):
        be = FakeBackend(service_s=0.03)
        srv = Server(be, budget_bytes=1000, n_slots=1, max_batch=8)
        try:
            fs = [srv.submit(creq(100))]                  # a: 400 bytes, takes the only slot
            time.sleep(0.01)
            fs.append(srv.submit(creq(50)))               # X: compress, 200
            fs.append(srv.submit(creq(150, DECOMPRESS)))  # Y: decompress, 600
            fs.append(srv.submit(creq(z_elems)))          # Z: compress
            for f in fs:
                assert f.result(timeout=5).status == 0
        finally:
            srv.close()
        return [seqs for _, _, _, seqs in be.launches]
    # Z = 200 bytes: X + Z + Y's 600 fit in 1000, so Z joins X's batch ahead of Y
    assert run(50) == [[0], [1, 3], [2]]
    # Z = 300 bytes: X + Z would leave less than Y's 600, so Z waits behind Y
    assert run(75) == [[0], [1], [2], [3]]
