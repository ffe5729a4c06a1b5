"""Scheduling rules of the native continuous-batching server, on the CPU: the server's
no-GPU mode runs the same scheduler, with batches that complete a fixed time after launch
and no outputs. Budget costs come from the server itself (fsz_server_request_cost)."""
import random
import threading
import time

import pytest

from paper_2607_15413_gb300.serve import COMPRESS, DECOMPRESS, Request, Server


def creq(n, kind=COMPRESS):
    if kind == COMPRESS:
        return Request(kind=COMPRESS, shape=(n,))
    return Request(kind=DECOMPRESS, n=n, nbytes=64)


def release_on_completion(fut):
    fut.add_done_callback(lambda f: f.result().release())
    return fut


def cost(srv, n, kind=COMPRESS):
    return srv.cost(creq(n, kind))


def test_costs_follow_the_output_allocation(fszlib):
    srv = Server(budget_bytes=1 << 30, sim_service_s=0.001)
    try:
        for n in (1, 255, 256, 257, 10 ** 6):
            bound = fszlib.fsz_compress_bound(n)
            assert cost(srv, n) == (bound + 15) // 16 * 16 + 16
            assert cost(srv, n, DECOMPRESS) == (4 * max(n, 4) + 15) // 16 * 16
    finally:
        srv.close()


def test_oversize_request_is_rejected_at_once():
    probe = Server(budget_bytes=1 << 30, sim_service_s=0.001)
    budget = cost(probe, 1000) - 1
    probe.close()
    srv = Server(budget_bytes=budget, n_slots=2, sim_service_s=0.02)
    try:
        r = srv.submit(creq(1000)).result(timeout=5)          # needs more than the budget
        assert r.status == 10 and r.batch == -1               # FSZ_ERR_REJECTED
        ok = srv.submit(creq(100)).result(timeout=5)
        assert ok.status == 0 and ok.batch == 0
        ok.release()
        st = srv.stats()
    finally:
        srv.close()
    assert st["rejected"] == 1 and st["completed"] == 1 and st["budget_free"] == budget


def test_budget_admits_in_arrival_order_without_overtaking():
    probe = Server(budget_bytes=1 << 30, sim_service_s=0.001)
    ca, cb, cc = cost(probe, 2000), cost(probe, 1500), cost(probe, 10)
    probe.close()
    budget = ca + cb - 1                                       # a and b do not fit together
    assert ca + cc <= budget
    srv = Server(budget_bytes=budget, n_slots=4, max_batch=8, sim_service_s=0.05)
    try:
        a = release_on_completion(srv.submit(creq(2000)))
        b = release_on_completion(srv.submit(creq(1500)))    # waits for a's memory
        c = release_on_completion(srv.submit(creq(10)))      # would fit, must not overtake b
        ra, rb, rc = (f.result(timeout=5) for f in (a, b, c))
    finally:
        srv.close()
    assert ra.batch == 0 and rb.batch == 1 and rc.batch == 1  # b and c launched together, after a
    assert rb.latency_s >= 0.05 - 1e-3                         # b waited for a's service


def test_continuous_batching_admits_while_batches_run():
    srv = Server(budget_bytes=10 ** 9, n_slots=3, max_batch=4, sim_service_s=0.03)
    futs = []
    try:
        for i in range(24):
            futs.append(release_on_completion(srv.submit(creq(1000 + i))))
            time.sleep(0.004)                                  # arrivals keep coming
        res = [f.result(timeout=10) for f in futs]
        st = srv.stats()
    finally:
        srv.close()
    assert st["max_inflight"] >= 2                             # batches overlapped
    assert st["admitted_while_busy"] > 0                       # admitted during others' service
    assert st["max_batch_seen"] <= 4
    assert min(r.latency_s for r in res) >= 0.03 - 1e-3        # at least one service time
    assert all(r.status == 0 for r in res)


def test_batches_are_homogeneous_in_kind():
    srv = Server(budget_bytes=10 ** 9, n_slots=1, max_batch=16, sim_service_s=0.02)
    try:
        kinds = [COMPRESS if i % 3 else DECOMPRESS for i in range(30)]
        futs = [release_on_completion(srv.submit(creq(100 + i, k))) for i, k in enumerate(kinds)]
        res = [f.result(timeout=10) for f in futs]
    finally:
        srv.close()
    by_batch = {}
    for k, r in zip(kinds, res):
        by_batch.setdefault(r.batch, set()).add(k)
    assert all(len(v) == 1 for v in by_batch.values())


def test_batches_reach_past_the_other_kind():
    """Alternating kinds still form full batches of each kind, in arrival order per kind."""
    srv = Server(budget_bytes=10 ** 9, n_slots=1, max_batch=8, sim_service_s=0.05)
    try:
        first = release_on_completion(srv.submit(creq(100)))  # occupies the only slot
        time.sleep(0.01)
        kinds = [COMPRESS if i % 2 else DECOMPRESS for i in range(16)]
        futs = [release_on_completion(srv.submit(creq(100 + i, k))) for i, k in enumerate(kinds)]
        r0 = first.result(timeout=10)
        res = [f.result(timeout=10) for f in futs]
    finally:
        srv.close()
    assert r0.batch == 0
    assert sorted({r.batch for r in res}) == [1, 2]
    assert all(r.batch_size == 8 for r in res)
    assert {r.batch for k, r in zip(kinds, res) if k == DECOMPRESS} == {1}   # the head's kind first


def test_a_skipped_request_keeps_its_memory():
    """A batch reaches past a request of the other kind only with memory to spare for it:
    a later request that would fit only by spending the skipped request's memory waits."""
    probe = Server(budget_bytes=1 << 30, sim_service_s=0.001)
    ca, cx, cy = cost(probe, 2000), cost(probe, 500), cost(probe, 40000, DECOMPRESS)
    small, large = cost(probe, 400), cost(probe, 4000)
    probe.close()
    budget = ca + cy + cx + small                              # X + Y + Z(small) fit, Z(large) not

    def run(z_elems):
        srv = Server(budget_bytes=budget, n_slots=1, max_batch=8, sim_service_s=0.03)
        try:
            fs = [release_on_completion(srv.submit(creq(2000)))]   # a: takes the only slot
            time.sleep(0.01)
            fs.append(release_on_completion(srv.submit(creq(500))))                 # X
            fs.append(release_on_completion(srv.submit(creq(40000, DECOMPRESS))))   # Y
            fs.append(release_on_completion(srv.submit(creq(z_elems))))             # Z
            return [f.result(timeout=5).batch for f in fs]
        finally:
            srv.close()
    assert large > budget - ca - cy - cx
    assert run(400) == [0, 1, 2, 1]        # Z joins X's batch: Y's memory stays free
    assert run(4000) == [0, 1, 2, 3]       # Z would spend Y's memory: it waits behind Y


def test_random_load_never_deadlocks():
    rng = random.Random(0)
    srv = Server(budget_bytes=400_000, n_slots=4, max_batch=8, sim_service_s=0.002)
    futs = []
    lock = threading.Lock()

    def client(seed):
        r = random.Random(seed)
        for _ in range(50):
            n = int(10 ** r.uniform(1, 5.2))                   # some exceed the budget
            f = release_on_completion(srv.submit(creq(n, r.choice([COMPRESS, DECOMPRESS]))))
            with lock:
                futs.append(f)
            time.sleep(r.uniform(0, 0.002))

    ts = [threading.Thread(target=client, args=(rng.random(),)) for _ in range(4)]
    try:
        for t in ts:
            t.start()
        for t in ts:
            t.join()
        res = [f.result(timeout=30) for f in futs]
        deadline = time.time() + 5
        while srv.stats()["budget_free"] != 400_000 and time.time() < deadline:
            time.sleep(0.01)                                   # releases run in callbacks
        st = srv.stats()
    finally:
        srv.close()
    assert len(res) == 200
    assert st["completed"] + st["rejected"] == 200
    assert st["rejected"] == sum(1 for r in res if r.status == 10)
    assert st["budget_free"] == 400_000                        # every admitted byte returned


@pytest.mark.parametrize("kw", [dict(n_slots=0), dict(n_slots=17), dict(max_batch=0),
                                dict(max_batch=1 << 20), dict(budget_bytes=0),
                                dict(max_batch_elems=0)])
def test_bad_configurations_are_refused(kw):
    from paper_2607_15413_gb300 import fsz
    args = dict(budget_bytes=1 << 20, n_slots=2, max_batch=8, sim_service_s=0.001)
    args.update(kw)
    with pytest.raises(fsz.FszError):
        Server(**args)


def test_linger_gathers_requests_while_busy():
    """With batches running, a short batch waits up to the linger time for more requests;
    an idle server launches at once."""
    def run(linger_s):
        srv = Server(budget_bytes=10 ** 9, n_slots=2, max_batch=8, linger_s=linger_s,
                     sim_service_s=0.08)
        try:
            fs = [release_on_completion(srv.submit(creq(100)))]   # idle: launches at once
            time.sleep(0.005)
            for i in range(3):
                fs.append(release_on_completion(srv.submit(creq(200 + i))))
                time.sleep(0.002)
            return [f.result(timeout=5) for f in fs]
        finally:
            srv.close()
    eager = run(0.0)
    assert eager[0].batch == 0 and eager[1].batch == 1        # the free slot takes r1 alone
    lingered = run(0.03)
    assert lingered[0].batch == 0 and lingered[0].latency_s < 0.09
    assert {r.batch for r in lingered[1:]} == {1} and lingered[1].batch_size == 3


def _table(srv, reqs, first_id):
    import numpy as np

    from paper_2607_15413_gb300 import fsz
    t = np.zeros(len(reqs), dtype=fsz.REQUEST_NP)
    for i, r in enumerate(reqs):
        nr = srv._native(r, first_id + i)
        t[i] = np.frombuffer(bytes(nr), dtype=fsz.REQUEST_NP)[0]
    return t


def _drain(srv, count, timeout_s=5.0):
    import numpy as np

    from paper_2607_15413_gb300 import fsz
    buf = np.zeros(64, dtype=fsz.COMPLETION_NP)
    got, deadline = [], time.time() + timeout_s
    while len(got) < count and time.time() < deadline:
        k = fsz.lib().fsz_server_poll(srv._h, buf.ctypes.data, len(buf), 2_000_000)
        got.extend(buf[:k].copy())
    return got


def test_trace_replay_admits_each_request_at_its_arrival_time():
    """Requests submitted ahead of their arrival times enter the queue then: the first
    completes a service time after its arrival, and one arriving after it, while it runs,
    is admitted then (not batched with it)."""
    from paper_2607_15413_gb300 import fsz
    srv = Server(budget_bytes=10 ** 9, n_slots=4, max_batch=8, sim_service_s=0.02,
                 futures=False)
    try:
        reqs = [creq(100), creq(200), creq(300)]
        t = _table(srv, reqs, 1)
        now = time.monotonic_ns()
        t["arrival_ns"] = [now + 60_000_000, now + 70_000_000, now + 70_000_000]
        t0 = time.monotonic()
        assert fsz.lib().fsz_server_submit_many(srv._h, t.ctypes.data, len(t)) == 0
        got = _drain(srv, 3)
        wall = time.monotonic() - t0
        st = srv.stats()
        for c in got:
            srv.release_raw(int(c["id"]))
    finally:
        srv.close()
    assert len(got) == 3 and all(c["status"] == 0 for c in got)
    by_id = {int(c["id"]): c for c in got}
    assert by_id[1]["batch"] == 0 and by_id[2]["batch"] == by_id[3]["batch"] == 1
    assert by_id[2]["batch_size"] == 2
    assert wall >= 0.07 + 0.02 - 2e-3                          # nothing ran before its arrival
    for c in got:                                              # latency counts from arrival
        assert 0.02 - 1e-3 <= c["latency_ns"] * 1e-9 < 0.02 + 0.015
    assert st["submitted"] == 3 and st["batches"] == 2


def test_bulk_submit_is_all_or_nothing_and_bulk_release_reports_unknown_ids():
    import numpy as np

    from paper_2607_15413_gb300 import fsz
    srv = Server(budget_bytes=10 ** 9, n_slots=2, max_batch=8, sim_service_s=0.005,
                 futures=False)
    L = fsz.lib()
    try:
        t = _table(srv, [creq(100), creq(200), creq(300)], 1)
        t["d_in"][1] = 8                                       # not 16-byte aligned
        assert L.fsz_server_submit_many(srv._h, t.ctypes.data, len(t)) == fsz.ERR_ALIGN
        assert srv.stats()["submitted"] == 0                    # none queued
        t["d_in"][1] = 0
        assert L.fsz_server_submit_many(srv._h, t.ctypes.data, len(t)) == 0
        got = _drain(srv, 3)
        ids = np.array([int(c["id"]) for c in got] + [999], dtype=np.uint64)
        assert L.fsz_server_release_many(srv._h, ids.ctypes.data, len(ids), None) == \
            fsz.ERR_INVALID_ARG                                 # 999 was never held
        assert L.fsz_server_release_many(srv._h, ids.ctypes.data, 1, None) == \
            fsz.ERR_INVALID_ARG                                 # already released
        st = srv.stats()
    finally:
        srv.close()
    assert len(got) == 3 and st["completed"] == 3 and st["budget_free"] == 10 ** 9


def test_held_outputs_stay_charged_until_released():
    # A client that keeps its outputs holds back admission (the output memory the server
    # holds never exceeds the budget); each release returns its request's cost; closing the
    # server refuses what still waits for memory the client never gave back.
    probe = Server(budget_bytes=1 << 30, sim_service_s=0.001)
    c = cost(probe, 1000)
    probe.close()
    srv = Server(budget_bytes=2 * c, n_slots=4, max_batch=8, sim_service_s=0.005)
    try:
        first = [srv.submit(creq(1000)).result(timeout=5) for _ in range(2)]
        assert all(r.status == 0 for r in first)
        assert srv.stats()["budget_free"] == 0                 # both outputs still held
        waiting = srv.submit(creq(1000))
        time.sleep(0.05)
        assert not waiting.done()                              # no memory until a release
        first[0].release()
        r = waiting.result(timeout=5)
        assert r.status == 0
        assert srv.stats()["budget_free"] == 0
        stuck = srv.submit(creq(1000))                         # waits: nothing is released
        time.sleep(0.05)
        assert not stuck.done()
    finally:
        srv.close()
    assert stuck.result(timeout=5).status == 10                # refused at close
