"""Continuous-batching request serving: a thin binding of the library's native server.

The scheduling (admission by a device-memory budget, batches of one kind on several CUDA
streams, continuous admission while batches run, completion by CUDA events) runs in the
library's own scheduler thread (fsz_server_* in the C ABI). This module marshals requests
and completions:

* `Server.submit(req)` queues a request whose input lives on the device (a float32 field to
  compress, or a stream plus its element count to decompress) and returns a future.
* A poller thread collects completions and resolves the futures with a `Result`: status,
  latency (arrival to completion), batch size and the output (a device pointer owned by
  the server, valid until `Result.release()`; `Result.tensor()` copies it into a tensor).
* `Server(sim_service_s=...)` runs the same scheduler without a GPU: each batch completes
  that long after its launch and has no output (for testing the scheduling rules).
"""
from __future__ import annotations

import concurrent.futures as cf
import ctypes
import itertools
import threading
import time
from dataclasses import dataclass, field

from . import fsz

COMPRESS, DECOMPRESS = "compress", "decompress"
_KIND = {COMPRESS: fsz.REQ_COMPRESS, DECOMPRESS: fsz.REQ_DECOMPRESS}


@dataclass
class Request:
    kind: str                 # COMPRESS or DECOMPRESS
    data: object = None       # device tensor (float32 field or uint8 stream), or None with ptr
    shape: tuple = ()         # compress: field shape
    eb: float = 1e-3          # compress: error bound
    mode: int = 1             # FSZ_EB_REL (1) or FSZ_EB_ABS (0)
    n: int = 0                # decompress: element count
    ptr: int = 0              # device pointer of the input when `data` is None
    nbytes: int = 0           # decompress: stream bytes when `data` is None
    arrival_ns: int = 0       # time.monotonic_ns() of arrival; 0 = at submission
    future: cf.Future = field(default_factory=cf.Future)


@dataclass
class Result:
    status: int
    latency_s: float
    batch_size: int = 0
    batch: int = -1           # launch index of its batch (-1 if rejected)
    ptr: int = 0              # device output (stream or float32 values), server-owned
    nbytes: int = 0           # stream bytes, or 4 n
    server: object = None
    id: int = 0

    def tensor(self, dtype=None, device="cuda"):
        """A copy of the output in a new tensor (uint8 for a stream, float32 for values)."""
        import torch
        if dtype is None:
            dtype = torch.uint8
        itemsize = torch.empty(0, dtype=dtype).element_size()
        t = torch.empty(self.nbytes // itemsize, dtype=dtype, device=device)
        st = torch.cuda.current_stream(t.device)
        code = fsz.lib().fsz_copy_device(t.data_ptr(), self.ptr, self.nbytes, st.cuda_stream)
        if code:
            raise fsz.FszError(code, "fsz_copy_device")
        st.synchronize()
        return t

    def release(self, stream=0) -> None:
        """Gives the output back to the server (once); its memory is freed with the last
        output of its batch."""
        if self.server is not None and self.status != fsz.ERR_REJECTED:
            self.server._release(self.id, stream)
        self.server = None


class Server:
    """The native scheduler. `submit()` is thread-safe; `close()` drains and stops."""

    def __init__(self, budget_bytes: int, n_slots: int = 4, max_batch: int = 32, scan: int = 0,
                 max_batch_elems: int = 1 << 31, linger_s: float = 0.0, sim_service_s: float = 0.0,
                 futures: bool = True):
        cfg = fsz.FszServerConfig()
        cfg.budget_bytes = int(budget_bytes)
        cfg.slots = n_slots
        cfg.max_batch = max_batch
        cfg.scan = scan
        cfg.linger_us = int(linger_s * 1e6)
        cfg.max_batch_elems = int(max_batch_elems)
        cfg.sim_service_ns = int(sim_service_s * 1e9)
        self._L = fsz.lib()
        self._h = ctypes.c_void_p()
        code = self._L.fsz_server_create(ctypes.byref(cfg), ctypes.byref(self._h))
        if code:
            raise fsz.FszError(code, "fsz_server_create")
        self.budget = int(budget_bytes)
        self._ids = itertools.count(1)
        self._live = {}                 # id -> Request (keeps inputs alive until completion)
        self._lock = threading.Lock()
        self._stop = False
        self._poller = None
        if futures:   # otherwise the caller drives submit_raw / poll_raw itself
            self._poller = threading.Thread(target=self._poll, daemon=True)
            self._poller.start()

    # -------------------------------------------------------------- client side
    def cost(self, req: Request) -> int:
        """Output bytes the server charges for `req` (its allocation)."""
        return int(self._L.fsz_server_request_cost(ctypes.byref(self._native(req, 0))))

    def submit(self, req: Request) -> cf.Future:
        rid = next(self._ids)
        nreq = self._native(req, rid)
        with self._lock:
            self._live[rid] = req
        code = self._L.fsz_server_submit(self._h, ctypes.byref(nreq))
        if code:
            with self._lock:
                self._live.pop(rid, None)
            req.future.set_exception(fsz.FszError(code, "fsz_server_submit"))
        return req.future

    def stats(self) -> dict:
        st = fsz.FszServerStats()
        self._L.fsz_server_get_stats(self._h, ctypes.byref(st))
        return {k: getattr(st, k) for k, _ in fsz.FszServerStats._fields_}

    def close(self) -> None:
        """Finishes the queued work (requests still waiting for memory that only a release
        would return are refused), stops the poller and frees the server (and any output
        not yet released)."""
        if self._h:
            with self._lock:
                self._stop = True
            self._L.fsz_server_stop(self._h)
            if self._poller is not None:
                self._poller.join()
            self._L.fsz_server_destroy(self._h)
            self._h = ctypes.c_void_p()

    # -------------------------------------------------------------- without futures
    # For clients that handle many requests per second from one thread: a request struct
    # filled in place, completions in bulk, releases by id (Server(futures=False)).
    def submit_raw(self, nreq: "fsz.FszRequest") -> int:
        return self._L.fsz_server_submit(self._h, ctypes.byref(nreq))

    def poll_raw(self, buf, wait_ns: int = 0) -> int:
        return self._L.fsz_server_poll(self._h, buf, len(buf), wait_ns)

    def release_raw(self, rid: int, stream=0) -> None:
        self._L.fsz_server_release(self._h, rid, stream)

    # -------------------------------------------------------------- internals
    def _native(self, req: Request, rid: int) -> fsz.FszRequest:
        r = fsz.FszRequest()
        r.id = rid
        r.kind = _KIND[req.kind]
        r.arrival_ns = int(req.arrival_ns)
        ptr = req.data.data_ptr() if req.data is not None and req.data.numel() else int(req.ptr)
        r.d_in = ptr or None
        if req.kind == COMPRESS:
            r.mode = int(req.mode)
            r.dims = fsz.make_dims(req.shape)
            r.eb = float(req.eb)
        else:
            r.n = int(req.n)
            r.in_bytes = int(req.data.numel()) if req.data is not None else int(req.nbytes)
        return r

    def _release(self, rid: int, stream) -> None:
        if self._h:
            self._L.fsz_server_release(self._h, rid, stream)

    def _poll(self) -> None:
        buf = (fsz.FszCompletion * 256)()
        while True:
            k = self._L.fsz_server_poll(self._h, buf, 256, 2_000_000)
            for i in range(k):
                c = buf[i]
                with self._lock:
                    req = self._live.pop(c.id, None)
                if req is None:
                    continue
                req.future.set_result(Result(status=c.status, latency_s=c.latency_ns * 1e-9,
                                             batch_size=c.batch_size,
                                             batch=-1 if c.batch == (1 << 64) - 1 else c.batch,
                                             ptr=c.d_out or 0,
                                             nbytes=c.out_bytes, server=self, id=c.id))
            if k == 0:
                with self._lock:
                    if self._stop and not self._live:
                        return


def percentile(xs, q: float) -> float:
    xs = sorted(xs)
    if not xs:
        return float("nan")
    k = min(len(xs) - 1, max(0, int(round(q / 100.0 * (len(xs) - 1)))))
    return xs[k]


def monotonic_ns() -> int:
    """The clock requests' arrival times are on (the server's)."""
    return time.monotonic_ns()
