"""Continuous-batching request loop for compress / decompress requests.

Clients submit requests whose inputs already live on the device (a float32 field to
compress, or a stream plus its element count to decompress) and get a future back. One
scheduler thread owns every GPU call:

* Admission: requests are admitted in arrival order while the device-memory budget
  allows. The budget counts the buffers the server allocates for a request (the output,
  and the stream-size word); inputs belong to the client. A request larger than the
  whole budget is rejected at once. A request that does not fit yet waits at the head of
  the queue: later requests do not overtake it, so nothing starves, and since in-flight
  work always completes and returns its memory, nothing deadlocks.
* Batching: the head's kind (compress or decompress) picks the batch; it takes up to
  `max_batch` waiting requests of that kind in arrival order, reaching past requests of
  the other kind (within a scan window) while holding their memory in reserve, so a
  skipped request still fits when its own batch goes next. The batch is launched as one
  batched C-ABI call on the first free stream slot. With several slots, batches overlap
  on the device; requests that arrive while batches run are admitted and launched as soon
  as a slot and budget free up (continuous batching), instead of waiting for the queue to
  drain.
* Completion: a CUDA event per batch; each request's future receives its result
  (the stream bytes for a compression, the decoded field for a decompression), its status
  and its latency (arrival to completion observed on the host).

The backend is pluggable: GpuBackend drives the CUDA library; tests use a fake backend
on the CPU to check the scheduling rules alone.
"""
from __future__ import annotations

import collections
import concurrent.futures as cf
import ctypes
import threading
import time
from dataclasses import dataclass, field

COMPRESS, DECOMPRESS = "compress", "decompress"


@dataclass
class Request:
    kind: str                 # COMPRESS or DECOMPRESS
    data: object              # device tensor: float32 field, or uint8 stream
    shape: tuple = ()         # field shape (compress)
    eb: float = 1e-3          # error bound (compress)
    mode: int = 1             # FSZ_EB_REL (1) or FSZ_EB_ABS (0)
    n: int = 0                # element count (decompress: from the compress result)
    arrival: float = 0.0      # host time.perf_counter() at submission
    future: cf.Future = field(default_factory=cf.Future)
    cost: int = 0             # device bytes the server allocates for it
    seq: int = 0


@dataclass
class Result:
    status: int
    latency_s: float
    output: object = None     # compress: uint8 stream tensor; decompress: float32 tensor
    nbytes: int = 0           # compress: stream size
    batch_size: int = 1


def _align16(x: int) -> int:
    return (x + 15) // 16 * 16


class GpuBackend:
    """Runs batches through the CUDA library: per slot a CUDA stream, a batch workspace, and
    preallocated pinned/device buffers for the field table and the stream sizes."""

    def __init__(self, n_slots: int, max_batch: int, max_elems: int, device="cuda"):
        import torch

        from . import fsz
        self.torch, self.fsz = torch, fsz
        self.device = torch.device(device)
        self.max_batch = max_batch
        self.streams = [torch.cuda.Stream(self.device) for _ in range(n_slots)]
        self.ws_bytes = fsz.fsz_batch_workspace_bytes(max_elems, max_batch)
        self.ws = [torch.empty(self.ws_bytes, dtype=torch.uint8, device=self.device)
                   for _ in range(n_slots)]
        tb = max_batch * ctypes.sizeof(fsz.FszCField)
        self.h_table = [torch.empty(tb, dtype=torch.uint8, pin_memory=True) for _ in range(n_slots)]
        self.d_table = [torch.empty(tb, dtype=torch.uint8, device=self.device) for _ in range(n_slots)]
        self.d_sizes = [torch.zeros(max_batch, dtype=torch.int64, device=self.device)
                        for _ in range(n_slots)]
        self.h_sizes = [torch.zeros(max_batch, dtype=torch.int64, pin_memory=True)
                        for _ in range(n_slots)]

    def cost(self, req: Request) -> int:
        if req.kind == COMPRESS:
            n = 1
            for s in req.shape:
                n *= int(s)
            return _align16(self.fsz.fsz_compress_bound(n)) + 16
        return _align16(4 * max(req.n, 4))

    def launch(self, slot: int, kind: str, reqs):
        """One batched call for `reqs` on stream slot `slot`. Outputs are views of one
        arena per batch; the descriptor table is filled column-wise in pinned memory."""
        import numpy as np
        torch, fsz = self.torch, self.fsz
        st = self.streams[slot]
        k = len(reqs)
        with torch.cuda.stream(st):
            if kind == COMPRESS:
                caps = np.fromiter((r.cost - 16 for r in reqs), dtype=np.uint64, count=k)
                offs = np.zeros(k, dtype=np.uint64)
                np.cumsum(caps[:-1], out=offs[1:])
                arena = torch.empty(int(caps.sum()), dtype=torch.uint8, device=self.device)
                tab = self.h_table[slot].numpy()[: k * fsz.CFIELD_NP.itemsize].view(fsz.CFIELD_NP)
                tab["in_"] = [r.data.data_ptr() if r.data.numel() else 0 for r in reqs]
                dims = [tuple(int(x) for x in r.shape) + (0, 0, 0) for r in reqs]
                tab["ndim"] = [len(r.shape) for r in reqs]
                tab["dreserved"] = 0
                tab["d0"] = [d[0] for d in dims]
                tab["d1"] = [d[1] for d in dims]
                tab["d2"] = [d[2] for d in dims]
                tab["mode"] = [int(r.mode) for r in reqs]
                tab["reserved"] = 0
                tab["eb"] = [float(r.eb) for r in reqs]
                tab["out"] = np.uint64(arena.data_ptr()) + offs
                tab["out_capacity"] = caps
                tab["out_bytes"] = np.uint64(self.d_sizes[slot].data_ptr()) + 8 * np.arange(k, dtype=np.uint64)
                n_total = sum(r.data.numel() for r in reqs)
                nb = k * fsz.CFIELD_NP.itemsize
                self.d_table[slot][:nb].copy_(self.h_table[slot][:nb], non_blocking=True)
                code = fsz.fsz_compress_batched(self.d_table[slot].data_ptr(), k, n_total,
                                                self.ws[slot].data_ptr(), self.ws_bytes,
                                                st.cuda_stream)
                self.h_sizes[slot][:k].copy_(self.d_sizes[slot][:k], non_blocking=True)
                keep = (arena, offs.tolist())
            else:
                caps = np.fromiter((_align16(4 * max(r.n, 4)) // 4 for r in reqs), dtype=np.uint64, count=k)
                offs = np.zeros(k, dtype=np.uint64)
                np.cumsum(caps[:-1], out=offs[1:])
                arena = torch.empty(int(caps.sum()), dtype=torch.float32, device=self.device)
                srcs = [r.data if r.data.data_ptr() % 16 == 0 else r.data.clone() for r in reqs]
                tab = self.h_table[slot].numpy()[: k * fsz.DFIELD_NP.itemsize].view(fsz.DFIELD_NP)
                tab["in_"] = [x.data_ptr() for x in srcs]
                tab["in_bytes"] = [x.numel() for x in srcs]
                tab["out"] = np.uint64(arena.data_ptr()) + 4 * offs
                tab["out_capacity_elems"] = caps
                nb = k * fsz.DFIELD_NP.itemsize
                self.d_table[slot][:nb].copy_(self.h_table[slot][:nb], non_blocking=True)
                code = fsz.fsz_decompress_batched(self.d_table[slot].data_ptr(), k, int(caps.sum()),
                                                  self.ws[slot].data_ptr(), self.ws_bytes,
                                                  st.cuda_stream)
                keep = (arena, offs.tolist(), srcs)
            ev = torch.cuda.Event()
            ev.record(st)
        return {"event": ev, "code": code, "keep": keep, "kind": kind, "slot": slot}

    def done(self, h) -> bool:
        return h["event"].query()

    def results(self, h, reqs):
        fsz = self.fsz
        slot = h["slot"]
        per = (ctypes.c_uint32 * len(reqs))()
        first = fsz.fsz_check_batched(self.ws[slot].data_ptr(), len(reqs), per,
                                      self.streams[slot].cuda_stream)
        arena, offs = h["keep"][0], h["keep"][1]
        out = []
        if h["kind"] == COMPRESS:
            sizes = self.h_sizes[slot][: len(reqs)].tolist()
        for i, r in enumerate(reqs):
            status = h["code"] if h["code"] else (int(per[i]) if first != fsz.ERR_CUDA else first)
            o = int(offs[i])
            if h["kind"] == COMPRESS:
                nb = int(sizes[i])
                out.append((status, arena[o: o + nb], nb))
            else:
                out.append((status, arena[o: o + r.n], 0))
        return out


class Server:
    """The scheduler. `submit()` is thread-safe; `close()` drains and stops."""

    def __init__(self, backend, budget_bytes: int, n_slots: int = 4, max_batch: int = 64,
                 poll_s: float = 5e-5, scan: int = 0):
        self.backend = backend
        self.scan = scan or 4 * max_batch  # requests looked at per batch
        self.budget = int(budget_bytes)
        self.free_budget = int(budget_bytes)
        self.n_slots = n_slots
        self.max_batch = max_batch
        self.poll_s = poll_s
        self._arrivals = collections.deque()
        self._lock = threading.Lock()
        self._wake = threading.Event()
        self._pending = collections.deque()
        self._inflight = {}          # slot -> (handle, reqs)
        self._stop = False
        self._seq = 0
        self.stats = {"completed": 0, "rejected": 0, "batches": 0, "max_inflight": 0,
                      "admitted_while_busy": 0, "bytes_in": 0, "max_batch_seen": 0}
        self._thread = threading.Thread(target=self._run, daemon=True)
        self._thread.start()

    # -------------------------------------------------------------- client side
    def submit(self, req: Request) -> cf.Future:
        req.arrival = req.arrival or time.perf_counter()
        req.cost = self.backend.cost(req)
        with self._lock:
            req.seq = self._seq
            self._seq += 1
            self._arrivals.append(req)
        self._wake.set()
        return req.future

    def close(self, timeout: float = 60.0) -> None:
        with self._lock:
            self._stop = True
        self._wake.set()
        self._thread.join(timeout)

    # -------------------------------------------------------------- scheduler
    def _run(self) -> None:
        while True:
            with self._lock:
                while self._arrivals:
                    r = self._arrivals.popleft()
                    if r.cost > self.budget:          # can never fit: reject now
                        self.stats["rejected"] += 1
                        r.future.set_result(Result(status=-1, latency_s=time.perf_counter() - r.arrival))
                        continue
                    self._pending.append(r)
                stop = self._stop
            progressed = self._complete()
            progressed |= self._launch()
            if stop and not self._pending and not self._inflight:
                with self._lock:
                    if not self._arrivals:
                        return
            if not progressed:
                self._wake.wait(self.poll_s)
                self._wake.clear()

    def _complete(self) -> bool:
        done = [s for s, (h, _) in self._inflight.items() if self.backend.done(h)]
        for s in done:
            h, reqs = self._inflight.pop(s)
            now = time.perf_counter()
            for r, (status, output, nb) in zip(reqs, self.backend.results(h, reqs)):
                self.free_budget += r.cost
                self.stats["completed"] += 1
                r.future.set_result(Result(status=status, latency_s=now - r.arrival, output=output,
                                           nbytes=nb, batch_size=len(reqs)))
        return bool(done)

    def _launch(self) -> bool:
        launched = False
        while self._pending and len(self._inflight) < self.n_slots:
            head = self._pending[0]
            if head.cost > self.free_budget:
                break                                  # wait for in-flight work to free memory
            kind = head.kind
            batch, skipped, reserved = [], [], 0
            for _ in range(min(len(self._pending), self.scan)):
                if len(batch) == self.max_batch:
                    break
                r = self._pending.popleft()
                if r.kind != kind:
                    skipped.append(r)       # waits for the next batch, its memory held back
                    reserved += r.cost
                    continue
                if r.cost + reserved > self.free_budget:
                    skipped.append(r)       # does not fit: nothing later overtakes it
                    break
                self.free_budget -= r.cost
                batch.append(r)
            self._pending.extendleft(reversed(skipped))
            slot = next(s for s in range(self.n_slots) if s not in self._inflight)
            if self._inflight:
                self.stats["admitted_while_busy"] += len(batch)
            h = self.backend.launch(slot, kind, batch)
            self._inflight[slot] = (h, batch)
            self.stats["batches"] += 1
            self.stats["max_inflight"] = max(self.stats["max_inflight"], len(self._inflight))
            self.stats["max_batch_seen"] = max(self.stats["max_batch_seen"], len(batch))
            for r in batch:
                self.stats["bytes_in"] += 4 * (r.data.numel() if kind == COMPRESS else r.n)
            launched = True
        return launched


def percentile(xs, q: float) -> float:
    xs = sorted(xs)
    if not xs:
        return float("nan")
    k = min(len(xs) - 1, max(0, int(round(q / 100.0 * (len(xs) - 1)))))
    return xs[k]
