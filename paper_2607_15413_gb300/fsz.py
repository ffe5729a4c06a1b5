"""ctypes binding of the FSZ C ABI (include/fsz.h).

The functions named like the C entry points take raw pointers (ints) and sizes and
only marshal arguments; every step of compression and decompression runs in the
CUDA library. The helpers below them (``compress``, ``decompress``, ...) allocate
device buffers with PyTorch and call the same entry points. There is no fallback:
if the library is missing, ``lib()`` raises.
"""
from __future__ import annotations

import ctypes
import os
import threading

PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(PKG, "_lib", "libfsz.so")

OK, ERR_INVALID_ARG, ERR_ALIGN, ERR_NONFINITE, ERR_EB_TOO_SMALL = 0, 1, 2, 3, 4
ERR_CAPACITY, ERR_CORRUPT, ERR_TIMEOUT, ERR_CUDA, ERR_WORKSPACE, ERR_REJECTED = 5, 6, 7, 8, 9, 10
STATUS_NAMES = {0: "FSZ_OK", 1: "FSZ_ERR_INVALID_ARG", 2: "FSZ_ERR_ALIGN", 3: "FSZ_ERR_NONFINITE",
                4: "FSZ_ERR_EB_TOO_SMALL", 5: "FSZ_ERR_CAPACITY", 6: "FSZ_ERR_CORRUPT",
                7: "FSZ_ERR_TIMEOUT", 8: "FSZ_ERR_CUDA", 9: "FSZ_ERR_WORKSPACE",
                10: "FSZ_ERR_REJECTED"}
EB_ABS, EB_REL = 0, 1
# Features switched off (fsz_feature_off), for the ablation of Sec. 6.4; 0 is the full method.
OFF_CROSS_BLOCK, OFF_CENTERING, OFF_LZ2 = 1, 2, 4

# Every entry point include/fsz.h declares.
EXPORTS = ["fsz_compress_bound", "fsz_workspace_bytes", "fsz_batch_workspace_bytes", "fsz_compress",
           "fsz_compress_features", "fsz_compress_multipass", "fsz_decompress_any",
           "fsz_decompress_prezeroed",
           "fsz_quality_workspace_bytes", "fsz_quality_stats", "fsz_compress_bound_tiled",
           "fsz_tiled_workspace_bytes", "fsz_compress_tiled", "fsz_decompress_tiled",
           "fsz_compress_prepare", "fsz_compress_encode", "fsz_decompress", "fsz_compress_batched",
           "fsz_decompress_batched", "fsz_check", "fsz_check_batched", "fsz_read_header",
           "fsz_set_test_hooks", "fsz_version", "fsz_compress_noalloc",
           "fsz_graph_compress_batched", "fsz_graph_decompress_batched", "fsz_graph_launch",
           "fsz_graph_destroy", "fsz_set_schedule", "fsz_get_schedule_limits", "fsz_set_schedule_ex",
           "fsz_get_schedule",
           "fsz_server_request_cost", "fsz_server_create", "fsz_server_submit", "fsz_server_poll",
           "fsz_server_submit_many", "fsz_server_release_many", "fsz_server_release", "fsz_server_get_stats", "fsz_server_stop", "fsz_server_destroy", "fsz_copy_device"]
REQ_COMPRESS, REQ_DECOMPRESS = 0, 1
# fsz_schedule, in its field order
SCHEDULE_FIELDS = ("stats_ctas_per_sm", "compress_ctas_per_sm", "decompress_ctas_per_sm",
                   "compress_ticket_chunks", "compress_ticket_lead", "decompress_ticket_chunks",
                   "decompress_records", "min_tickets_per_cta")


class FszSchedule(ctypes.Structure):
    _fields_ = [(name, ctypes.c_uint32) for name in SCHEDULE_FIELDS]


class FszDims(ctypes.Structure):
    _fields_ = [("ndim", ctypes.c_uint32), ("reserved", ctypes.c_uint32),
                ("dims", ctypes.c_uint64 * 3)]


class FszCField(ctypes.Structure):
    _fields_ = [("in_", ctypes.c_void_p), ("dims", FszDims), ("mode", ctypes.c_uint32),
                ("features_off", ctypes.c_uint32), ("eb", ctypes.c_double), ("out", ctypes.c_void_p),
                ("out_capacity", ctypes.c_uint64), ("out_bytes", ctypes.c_void_p)]


class FszServerConfig(ctypes.Structure):
    _fields_ = [("budget_bytes", ctypes.c_uint64), ("slots", ctypes.c_uint32),
                ("max_batch", ctypes.c_uint32), ("scan", ctypes.c_uint32), ("linger_us", ctypes.c_uint32),
                ("max_batch_elems", ctypes.c_uint64), ("sim_service_ns", ctypes.c_uint64)]


class FszRequest(ctypes.Structure):
    _fields_ = [("id", ctypes.c_uint64), ("kind", ctypes.c_uint32), ("mode", ctypes.c_uint32),
                ("dims", FszDims), ("eb", ctypes.c_double), ("d_in", ctypes.c_void_p),
                ("in_bytes", ctypes.c_uint64), ("n", ctypes.c_uint64), ("arrival_ns", ctypes.c_uint64)]


class FszCompletion(ctypes.Structure):
    _fields_ = [("id", ctypes.c_uint64), ("status", ctypes.c_int32), ("batch_size", ctypes.c_uint32),
                ("batch", ctypes.c_uint64), ("d_out", ctypes.c_void_p), ("out_bytes", ctypes.c_uint64),
                ("latency_ns", ctypes.c_uint64)]


class FszServerStats(ctypes.Structure):
    _fields_ = [(k, ctypes.c_uint64) for k in ("submitted", "completed", "rejected", "batches",
                                               "max_inflight", "max_batch_seen", "admitted_while_busy",
                                               "budget_free", "bytes_in")]


class FszDField(ctypes.Structure):
    _fields_ = [("in_", ctypes.c_void_p), ("in_bytes", ctypes.c_uint64), ("out", ctypes.c_void_p),
                ("out_capacity_elems", ctypes.c_uint64)]


# numpy views of the same layouts, for filling many descriptors at once
def _np_dtypes():
    import numpy as np
    cf = np.dtype({"names": ["in_", "ndim", "dreserved", "d0", "d1", "d2", "mode", "features_off", "eb",
                             "out", "out_capacity", "out_bytes"],
                   "formats": ["<u8", "<u4", "<u4", "<u8", "<u8", "<u8", "<u4", "<u4", "<f8", "<u8",
                               "<u8", "<u8"],
                   "offsets": [0, 8, 12, 16, 24, 32, 40, 44, 48, 56, 64, 72], "itemsize": 80})
    df = np.dtype({"names": ["in_", "in_bytes", "out", "out_capacity_elems"],
                   "formats": ["<u8", "<u8", "<u8", "<u8"], "offsets": [0, 8, 16, 24], "itemsize": 32})
    rq = np.dtype({"names": ["id", "kind", "mode", "ndim", "dreserved", "d0", "d1", "d2", "eb",
                             "d_in", "in_bytes", "n", "arrival_ns"],
                   "formats": ["<u8", "<u4", "<u4", "<u4", "<u4", "<u8", "<u8", "<u8", "<f8", "<u8",
                               "<u8", "<u8", "<u8"],
                   "offsets": [0, 8, 12, 16, 20, 24, 32, 40, 48, 56, 64, 72, 80], "itemsize": 88})
    cp = np.dtype({"names": ["id", "status", "batch_size", "batch", "d_out", "out_bytes",
                             "latency_ns"],
                   "formats": ["<u8", "<i4", "<u4", "<u8", "<u8", "<u8", "<u8"],
                   "offsets": [0, 8, 12, 16, 24, 32, 40], "itemsize": 48})
    assert cf.itemsize == ctypes.sizeof(FszCField) and df.itemsize == ctypes.sizeof(FszDField)
    assert rq.itemsize == ctypes.sizeof(FszRequest) and cp.itemsize == ctypes.sizeof(FszCompletion)
    return cf, df, rq, cp


CFIELD_NP, DFIELD_NP, REQUEST_NP, COMPLETION_NP = _np_dtypes()


class FszError(RuntimeError):
    def __init__(self, status: int, where: str):
        super().__init__(f"{where}: {STATUS_NAMES.get(status, status)}")
        self.status = status


_lock = threading.Lock()
_lib = None


def lib():
    """The loaded CUDA library. Raises if it has not been built (no CPU fallback)."""
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(LIB_PATH):
                raise RuntimeError(f"FSZ CUDA library missing at {LIB_PATH}; build it with "
                                   "paper_2607_15413_gb300._build.build()")
            L = ctypes.CDLL(LIB_PATH)
            P, u64, u32, i32, f64 = (ctypes.c_void_p, ctypes.c_uint64, ctypes.c_uint32,
                                     ctypes.c_int, ctypes.c_double)
            L.fsz_compress_bound.argtypes = [u64]
            L.fsz_compress_bound.restype = u64
            L.fsz_workspace_bytes.argtypes = [u64]
            L.fsz_workspace_bytes.restype = u64
            L.fsz_batch_workspace_bytes.argtypes = [u64, u32]
            L.fsz_batch_workspace_bytes.restype = u64
            for name in ("fsz_compress", "fsz_compress_prepare", "fsz_compress_encode"):
                fn = getattr(L, name)
                fn.argtypes = [P, FszDims, i32, f64, P, u64, P, P, u64, P]
                fn.restype = i32
            L.fsz_compress_features.argtypes = [P, FszDims, i32, f64, u32, P, u64, P, P, u64, P]
            L.fsz_compress_features.restype = i32
            L.fsz_compress_multipass.argtypes = [P, FszDims, i32, f64, P, u64, P, P, P, u64, P]
            L.fsz_compress_multipass.restype = i32
            L.fsz_decompress_any.argtypes = [P, u64, P, u64, P, u64, P]
            L.fsz_decompress_any.restype = i32
            L.fsz_decompress_prezeroed.argtypes = [P, u64, P, u64, P, u64, P]
            L.fsz_decompress_prezeroed.restype = i32
            L.fsz_quality_workspace_bytes.argtypes = []
            L.fsz_quality_workspace_bytes.restype = u64
            L.fsz_quality_stats.argtypes = [P, P, u64, f64, u64, P, P, u64, P]
            L.fsz_quality_stats.restype = i32
            L.fsz_compress_bound_tiled.argtypes = [u64, u32, u32]
            L.fsz_compress_bound_tiled.restype = u64
            L.fsz_tiled_workspace_bytes.argtypes = [u64]
            L.fsz_tiled_workspace_bytes.restype = u64
            L.fsz_compress_tiled.argtypes = [P, FszDims, i32, f64, u32, u32, u32, P, u64, P, P, u64, P]
            L.fsz_compress_tiled.restype = i32
            L.fsz_decompress_tiled.argtypes = [P, u64, P, u64, P, u64, P]
            L.fsz_decompress_tiled.restype = i32
            L.fsz_decompress.argtypes = [P, u64, P, u64, P, u64, P]
            L.fsz_decompress.restype = i32
            L.fsz_compress_batched.argtypes = [P, u32, u64, P, u64, P]
            L.fsz_compress_batched.restype = i32
            L.fsz_decompress_batched.argtypes = [P, u32, u64, P, u64, P]
            L.fsz_decompress_batched.restype = i32
            L.fsz_check.argtypes = [P, P]
            L.fsz_check.restype = i32
            L.fsz_check_batched.argtypes = [P, u32, P, P]
            L.fsz_check_batched.restype = i32
            L.fsz_read_header.argtypes = [P, P, P, P, P, P]
            L.fsz_read_header.restype = i32
            L.fsz_set_test_hooks.argtypes = [u64, u64]
            L.fsz_set_test_hooks.restype = None
            L.fsz_compress_noalloc.argtypes = [P, FszDims, i32, f64, P, u64, P, P, P]
            L.fsz_compress_noalloc.restype = i32
            L.fsz_graph_compress_batched.argtypes = [P, u32, u64, P, u64, P]
            L.fsz_graph_compress_batched.restype = i32
            L.fsz_graph_decompress_batched.argtypes = [P, u32, u64, P, u64, P]
            L.fsz_graph_decompress_batched.restype = i32
            L.fsz_graph_launch.argtypes = [P, P]
            L.fsz_graph_launch.restype = i32
            L.fsz_graph_destroy.argtypes = [P]
            L.fsz_graph_destroy.restype = None
            L.fsz_set_schedule.argtypes = [u32, u32, u32]
            L.fsz_set_schedule.restype = i32
            L.fsz_get_schedule_limits.argtypes = [P, P, P, P]
            L.fsz_get_schedule_limits.restype = i32
            L.fsz_set_schedule_ex.argtypes = [P]
            L.fsz_set_schedule_ex.restype = i32
            L.fsz_get_schedule.argtypes = [P]
            L.fsz_get_schedule.restype = i32
            L.fsz_version.argtypes = []
            L.fsz_version.restype = ctypes.c_char_p
            L.fsz_server_request_cost.argtypes = [P]
            L.fsz_server_request_cost.restype = u64
            L.fsz_server_create.argtypes = [P, P]
            L.fsz_server_create.restype = i32
            L.fsz_server_submit.argtypes = [P, P]
            L.fsz_server_submit.restype = i32
            L.fsz_server_submit_many.argtypes = [P, P, u64]
            L.fsz_server_submit_many.restype = i32
            L.fsz_server_release_many.argtypes = [P, P, u64, P]
            L.fsz_server_release_many.restype = i32
            L.fsz_server_poll.argtypes = [P, P, u32, u64]
            L.fsz_server_poll.restype = u32
            L.fsz_server_release.argtypes = [P, u64, P]
            L.fsz_server_release.restype = i32
            L.fsz_server_get_stats.argtypes = [P, P]
            L.fsz_server_get_stats.restype = i32
            L.fsz_server_stop.argtypes = [P]
            L.fsz_server_stop.restype = i32
            L.fsz_server_destroy.argtypes = [P]
            L.fsz_server_destroy.restype = i32
            L.fsz_copy_device.argtypes = [P, P, u64, P]
            L.fsz_copy_device.restype = i32
            _lib = L
    return _lib


def make_dims(shape) -> FszDims:
    shape = tuple(int(s) for s in shape)
    if not 1 <= len(shape) <= 3:
        raise ValueError("1 to 3 dims")
    d = FszDims()
    d.ndim = len(shape)
    d.reserved = 0
    for k, s in enumerate(shape):
        d.dims[k] = s
    return d


# ------------------------------------------------------------------ C-ABI names

def fsz_compress_bound(n: int) -> int:
    return lib().fsz_compress_bound(n)


def fsz_workspace_bytes(n: int) -> int:
    return lib().fsz_workspace_bytes(n)


def fsz_batch_workspace_bytes(n_total: int, nfields: int) -> int:
    return lib().fsz_batch_workspace_bytes(n_total, nfields)


def fsz_compress(d_in, dims, mode, eb, d_out, out_capacity, d_out_bytes, d_ws, ws_bytes, stream) -> int:
    return lib().fsz_compress(d_in, dims, mode, eb, d_out, out_capacity, d_out_bytes, d_ws, ws_bytes,
                              stream)


def fsz_compress_features(d_in, dims, mode, eb, features_off, d_out, out_capacity, d_out_bytes, d_ws,
                          ws_bytes, stream) -> int:
    return lib().fsz_compress_features(d_in, dims, mode, eb, features_off, d_out, out_capacity,
                                       d_out_bytes, d_ws, ws_bytes, stream)


def fsz_compress_prepare(d_in, dims, mode, eb, d_out, out_capacity, d_out_bytes, d_ws, ws_bytes,
                         stream) -> int:
    return lib().fsz_compress_prepare(d_in, dims, mode, eb, d_out, out_capacity, d_out_bytes, d_ws,
                                      ws_bytes, stream)


def fsz_compress_encode(d_in, dims, mode, eb, d_out, out_capacity, d_out_bytes, d_ws, ws_bytes,
                        stream) -> int:
    return lib().fsz_compress_encode(d_in, dims, mode, eb, d_out, out_capacity, d_out_bytes, d_ws,
                                     ws_bytes, stream)


def fsz_decompress(d_in, in_bytes, d_out, out_capacity_elems, d_ws, ws_bytes, stream) -> int:
    return lib().fsz_decompress(d_in, in_bytes, d_out, out_capacity_elems, d_ws, ws_bytes, stream)


def fsz_compress_batched(d_fields, nfields, n_total, d_ws, ws_bytes, stream) -> int:
    return lib().fsz_compress_batched(d_fields, nfields, n_total, d_ws, ws_bytes, stream)


def fsz_decompress_batched(d_fields, nfields, n_total_capacity, d_ws, ws_bytes, stream) -> int:
    return lib().fsz_decompress_batched(d_fields, nfields, n_total_capacity, d_ws, ws_bytes, stream)


def fsz_check(d_ws, stream) -> int:
    return lib().fsz_check(d_ws, stream)


def fsz_check_batched(d_ws, nfields, h_status, stream) -> int:
    return lib().fsz_check_batched(d_ws, nfields, h_status, stream)


def fsz_read_header(h_first64: bytes):
    buf = ctypes.create_string_buffer(bytes(h_first64[:64]), 64)
    n, eb, step, total = ctypes.c_uint64(), ctypes.c_double(), ctypes.c_float(), ctypes.c_uint64()
    dims = FszDims()
    st = lib().fsz_read_header(buf, ctypes.byref(n), ctypes.byref(dims), ctypes.byref(eb),
                               ctypes.byref(step), ctypes.byref(total))
    if st != OK:
        raise FszError(st, "fsz_read_header")
    return dict(n=n.value, dims=tuple(dims.dims[k] for k in range(dims.ndim)), eb=eb.value,
                step=step.value, total_bytes=total.value)


def fsz_compress_noalloc(d_in, dims, mode, eb, d_out, out_capacity, d_out_bytes, d_status,
                         stream) -> int:
    """fsz_compress with the library's built-in scratch, for callers that cannot allocate."""
    return lib().fsz_compress_noalloc(d_in, dims, mode, eb, d_out, out_capacity, d_out_bytes,
                                      d_status, stream)


def fsz_graph_compress_batched(d_fields, nfields, n_total, d_ws, ws_bytes):
    """Captures fsz_compress_batched into a CUDA graph; returns the graph handle."""
    g = ctypes.c_void_p()
    _check(lib().fsz_graph_compress_batched(d_fields, nfields, n_total, d_ws, ws_bytes,
                                            ctypes.byref(g)), "fsz_graph_compress_batched")
    return g.value


def fsz_graph_decompress_batched(d_fields, nfields, n_total_capacity, d_ws, ws_bytes):
    g = ctypes.c_void_p()
    _check(lib().fsz_graph_decompress_batched(d_fields, nfields, n_total_capacity, d_ws, ws_bytes,
                                              ctypes.byref(g)), "fsz_graph_decompress_batched")
    return g.value


def fsz_graph_launch(g, stream) -> int:
    return lib().fsz_graph_launch(g, stream)


def fsz_graph_destroy(g) -> None:
    lib().fsz_graph_destroy(g)


def fsz_set_schedule(stats_ctas_per_sm: int, compress_ctas_per_sm: int,
                     decompress_ctas_per_sm: int) -> int:
    return lib().fsz_set_schedule(stats_ctas_per_sm, compress_ctas_per_sm, decompress_ctas_per_sm)


def fsz_set_schedule_ex(schedule: dict | None) -> int:
    """Installs a full schedule (a dict with the SCHEDULE_FIELDS keys; missing keys keep
    the schedule in force), or the defaults for None. Returns the status."""
    if schedule is None:
        return lib().fsz_set_schedule_ex(None)
    cur = fsz_get_schedule()
    cur.update({k: int(v) for k, v in schedule.items() if k in SCHEDULE_FIELDS})
    sc = FszSchedule(*[cur[k] for k in SCHEDULE_FIELDS])
    return lib().fsz_set_schedule_ex(ctypes.byref(sc))


def fsz_get_schedule() -> dict:
    sc = FszSchedule()
    _check(lib().fsz_get_schedule(ctypes.byref(sc)), "fsz_get_schedule")
    return {k: int(getattr(sc, k)) for k in SCHEDULE_FIELDS}


def fsz_get_schedule_limits():
    vals = [ctypes.c_uint32() for _ in range(4)]
    _check(lib().fsz_get_schedule_limits(*[ctypes.byref(v) for v in vals]), "fsz_get_schedule_limits")
    return dict(stats=vals[0].value, compress=vals[1].value, decompress=vals[2].value,
                sms=vals[3].value)


def fsz_set_test_hooks(skip_chunk: int, timeout_ns: int) -> None:
    lib().fsz_set_test_hooks(skip_chunk, timeout_ns)


def fsz_version() -> str:
    return lib().fsz_version().decode()


# ------------------------------------------------------------------ torch helpers

def _stream_ptr(stream=None) -> int:
    import torch
    s = stream if stream is not None else torch.cuda.current_stream()
    return s.cuda_stream


def _check(st: int, where: str) -> None:
    if st != OK:
        raise FszError(st, where)


def _dev_buffer(nbytes: int, device):
    import torch
    # 16-byte aligned by the caching allocator; at least 16 bytes.
    return torch.empty(max(16, (nbytes + 15) // 16 * 16), dtype=torch.uint8, device=device)


class Workspace:
    """A reusable device workspace sized for up to n elements (one field)."""

    def __init__(self, n: int, device="cuda"):
        self.bytes = fsz_workspace_bytes(n)
        self.buf = _dev_buffer(self.bytes, device)

    @property
    def ptr(self) -> int:
        return self.buf.data_ptr()


def compress(x, eb: float, mode: int = EB_REL, shape=None, ws: Workspace | None = None,
             out=None, stream=None, check: bool = True, features_off: int = 0):
    """Compress a contiguous float32 CUDA tensor. Returns (stream_bytes_tensor, nbytes).
    features_off switches features of the method off (OFF_* bits, for ablations)."""
    import torch
    assert x.dtype == torch.float32 and x.is_cuda and x.is_contiguous()
    shape = tuple(x.shape) if shape is None else tuple(shape)
    if len(shape) == 0:
        shape = (x.numel(),)
    n = x.numel()
    cap = fsz_compress_bound(n)
    if out is None:
        out = _dev_buffer(cap, x.device)
    ws = ws if ws is not None else Workspace(n, x.device)
    nbytes = torch.zeros(2, dtype=torch.int64, device=x.device)
    sp = _stream_ptr(stream)
    if features_off:
        st = fsz_compress_features(x.data_ptr(), make_dims(shape), mode, eb, features_off,
                                   out.data_ptr(), out.numel(), nbytes.data_ptr(), ws.ptr, ws.bytes, sp)
    else:
        st = fsz_compress(x.data_ptr(), make_dims(shape), mode, eb, out.data_ptr(), out.numel(),
                          nbytes.data_ptr(), ws.ptr, ws.bytes, sp)
    _check(st, "fsz_compress")
    if check:
        _check(fsz_check(ws.ptr, sp), "fsz_compress (device)")
    nb = int(nbytes[0].item())
    return out[:nb], nb


def compress_multipass(x, eb: float, mode: int = EB_REL, shape=None, ws: Workspace | None = None,
                       out=None, costs=None, stream=None, check: bool = True):
    """compress() through the multipass evaluation (four cost passes, then the encoding
    pass selecting from them). Returns (stream_bytes_tensor, nbytes, costs) with costs a
    uint32-valued int32 tensor of shape (4, T)."""
    import torch
    assert x.dtype == torch.float32 and x.is_cuda and x.is_contiguous()
    shape = tuple(x.shape) if shape is None else tuple(shape)
    if len(shape) == 0:
        shape = (x.numel(),)
    n = x.numel()
    T = (n + 255) // 256
    cap = fsz_compress_bound(n)
    if out is None:
        out = _dev_buffer(cap, x.device)
    if costs is None:
        costs = torch.zeros((4, max(T, 1)), dtype=torch.int32, device=x.device)
    ws = ws if ws is not None else Workspace(n, x.device)
    nbytes = torch.zeros(2, dtype=torch.int64, device=x.device)
    sp = _stream_ptr(stream)
    st = lib().fsz_compress_multipass(x.data_ptr(), make_dims(shape), mode, eb, out.data_ptr(),
                                      out.numel(), nbytes.data_ptr(), costs.data_ptr(), ws.ptr,
                                      ws.bytes, sp)
    _check(st, "fsz_compress_multipass")
    if check:
        _check(fsz_check(ws.ptr, sp), "fsz_compress_multipass (device)")
    nb = int(nbytes[0].item())
    return out[:nb], nb, costs[:, :T]


def decompress(stream_bytes, n: int | None = None, ws: Workspace | None = None, out=None,
               stream=None, check: bool = True, any_stream: bool = False, out_is_zero: bool = False):
    """Decompress a device byte tensor holding one stream. Returns a float32 tensor.
    any_stream: through fsz_decompress_any, which also takes streams compressed without
    the cross-block state (OFF_CROSS_BLOCK). out_is_zero: `out` already holds zeros (or,
    with out=None, is allocated zero-filled): the all-zero tiles are neither decoded nor
    written (fsz_decompress_prezeroed); pays off for sparse fields when the zeros are
    already there."""
    import torch
    assert stream_bytes.dtype == torch.uint8 and stream_bytes.is_cuda
    if n is None:
        n = fsz_read_header(stream_bytes[:64].cpu().numpy().tobytes())["n"]
    if out is None:
        alloc = torch.zeros if out_is_zero else torch.empty
        out = alloc(max(n, 4), dtype=torch.float32, device=stream_bytes.device)
    ws = ws if ws is not None else Workspace(out.numel(), stream_bytes.device)
    src = stream_bytes
    if src.data_ptr() % 16:
        src = src.clone()
    sp = _stream_ptr(stream)
    fn = (lib().fsz_decompress_any if any_stream
          else lib().fsz_decompress_prezeroed if out_is_zero else fsz_decompress)
    st = fn(src.data_ptr(), src.numel(), out.data_ptr(), out.numel(), ws.ptr, ws.bytes, sp)
    _check(st, "fsz_decompress")
    if check:
        _check(fsz_check(ws.ptr, sp), "fsz_decompress (device)")
    return out[:n]


# ------------------------------------------------------------------ tile configurations

TILE_CONFIGS = ((32, 4), (32, 8), (32, 16), (64, 4), (64, 8), (64, 16))


def compress_tiled(x, eb: float, mode: int = EB_REL, block: int = 32, tile_blocks: int = 8,
                   features_off: int = 0, shape=None, stream=None, check: bool = True):
    """Compress with a tile configuration of Sec. 6.5 (fsz_compress_tiled). Returns
    (stream_bytes_tensor, nbytes)."""
    import torch
    assert x.dtype == torch.float32 and x.is_cuda and x.is_contiguous()
    shape = tuple(x.shape) if shape is None else tuple(shape)
    if len(shape) == 0:
        shape = (x.numel(),)
    n = x.numel()
    cap = lib().fsz_compress_bound_tiled(n, block, tile_blocks)
    out = _dev_buffer(max(cap, 16), x.device)
    wsb = lib().fsz_tiled_workspace_bytes(n)
    ws = _dev_buffer(wsb, x.device)
    nbytes = torch.zeros(2, dtype=torch.int64, device=x.device)
    sp = _stream_ptr(stream)
    _check(lib().fsz_compress_tiled(x.data_ptr(), make_dims(shape), mode, eb, block, tile_blocks,
                                    features_off, out.data_ptr(), cap, nbytes.data_ptr(),
                                    ws.data_ptr(), wsb, sp), "fsz_compress_tiled")
    if check:
        _check(fsz_check(ws.data_ptr(), sp), "fsz_compress_tiled (device)")
    nb = int(nbytes[0].item())
    return out[:nb], nb


def decompress_tiled(stream_bytes, n: int, stream=None, check: bool = True):
    """Decode a stream of any tile configuration (fsz_decompress_tiled)."""
    import torch
    src = stream_bytes if stream_bytes.data_ptr() % 16 == 0 else stream_bytes.clone()
    out = torch.empty(max(n, 4), dtype=torch.float32, device=src.device)
    wsb = lib().fsz_tiled_workspace_bytes(out.numel())
    ws = _dev_buffer(wsb, src.device)
    sp = _stream_ptr(stream)
    _check(lib().fsz_decompress_tiled(src.data_ptr(), src.numel(), out.data_ptr(), out.numel(),
                                      ws.data_ptr(), wsb, sp), "fsz_decompress_tiled")
    if check:
        _check(fsz_check(ws.data_ptr(), sp), "fsz_decompress_tiled (device)")
    return out[:n]


# ------------------------------------------------------------------ quality

QUALITY_FIELDS = ["n", "over_bound", "max_abs_err", "sum_sq_err", "min", "max", "psnr_db", "nrmse",
                  "bit_rate"]


def quality(orig, recon, eb: float, stream_bytes: int = 0, stream=None) -> dict:
    """Reconstruction quality on the device (fsz_quality_stats): PSNR, NRMSE, max error,
    errors above eb, value range, bit rate. Waits for the result."""
    import numpy as np
    import torch
    assert orig.dtype == torch.float32 and recon.dtype == torch.float32
    assert orig.is_cuda and orig.numel() == recon.numel()
    n = orig.numel()
    out = torch.zeros(16, dtype=torch.float64, device=orig.device)
    wsb = lib().fsz_quality_workspace_bytes()
    ws = _dev_buffer(wsb, orig.device)
    a, b = orig.contiguous(), recon.contiguous()
    if a.data_ptr() % 16:
        a = a.clone()
    if b.data_ptr() % 16:
        b = b.clone()
    sp = _stream_ptr(stream)
    _check(lib().fsz_quality_stats(a.data_ptr(), b.data_ptr(), n, float(eb), int(stream_bytes),
                                   out.data_ptr(), ws.data_ptr(), wsb, sp), "fsz_quality_stats")
    raw = out[:9].cpu().numpy()
    ints = raw[:2].view(np.uint64)
    vals = {k: float(v) for k, v in zip(QUALITY_FIELDS[2:], raw[2:])}
    return {"n": int(ints[0]), "over_bound": int(ints[1]), **vals}


# ------------------------------------------------------------------ batches

def _align16(x: int) -> int:
    return (x + 15) // 16 * 16


class CompressBatch:
    """Buffers and the device field table for fsz_compress_batched over a fixed set of
    fields: one output arena (each field's slot fsz_compress_bound(n) bytes, 16-byte
    aligned), per-field stream sizes and a batch workspace. run() launches one batched
    call; graph() captures it once into a CUDA graph for repeated launches."""

    def __init__(self, fields, device="cuda"):
        import torch
        self.device = torch.device(device)
        self.fields = list(fields)  # (tensor, shape, mode, eb[, features_off])
        self.n = [int(x.numel()) for x, *_ in self.fields]
        self.n_total = sum(self.n)
        caps = [_align16(fsz_compress_bound(k)) for k in self.n]
        self.offsets = [0]
        for c in caps:
            self.offsets.append(self.offsets[-1] + c)
        self.caps = caps
        self.arena = torch.empty(max(16, self.offsets[-1]), dtype=torch.uint8, device=self.device)
        self.sizes = torch.zeros(len(self.fields), dtype=torch.int64, device=self.device)
        arr = (FszCField * len(self.fields))()
        for i, (x, shape, mode, eb, *rest) in enumerate(self.fields):
            off = rest[0] if rest else 0
            assert x.dtype == torch.float32 and x.is_cuda and x.is_contiguous()
            arr[i].in_ = x.data_ptr() if x.numel() else 0
            arr[i].dims = make_dims(shape)
            arr[i].mode = int(mode)
            arr[i].features_off = int(off)
            arr[i].eb = float(eb)
            arr[i].out = self.arena.data_ptr() + self.offsets[i]
            arr[i].out_capacity = caps[i]
            arr[i].out_bytes = self.sizes.data_ptr() + 8 * i
        raw = bytes(arr)
        self.table = torch.frombuffer(bytearray(raw), dtype=torch.uint8).to(self.device)
        self.ws_bytes = fsz_batch_workspace_bytes(self.n_total, len(self.fields))
        self.ws = _dev_buffer(self.ws_bytes, self.device)
        self._graph = None

    def run(self, stream=None) -> int:
        return fsz_compress_batched(self.table.data_ptr(), len(self.fields), self.n_total,
                                    self.ws.data_ptr(), self.ws_bytes, _stream_ptr(stream))

    def graph(self):
        if self._graph is None:
            self._graph = fsz_graph_compress_batched(self.table.data_ptr(), len(self.fields),
                                                     self.n_total, self.ws.data_ptr(), self.ws_bytes)
        return self._graph

    def launch_graph(self, stream=None) -> int:
        return fsz_graph_launch(self.graph(), _stream_ptr(stream))

    def status(self, stream=None):
        """(first device status, per-field statuses); waits for the stream."""
        per = (ctypes.c_uint32 * len(self.fields))()
        st = fsz_check_batched(self.ws.data_ptr(), len(self.fields), per, _stream_ptr(stream))
        return st, list(per)

    def stream(self, i: int, sizes=None):
        k = int(self.sizes[i].item()) if sizes is None else int(sizes[i])
        return self.arena[self.offsets[i]:self.offsets[i] + k]

    def __del__(self):
        if getattr(self, "_graph", None) is not None:
            try:
                fsz_graph_destroy(self._graph)
            except Exception:
                pass


class DecompressBatch:
    """Buffers and the device field table for fsz_decompress_batched: streams (device
    byte tensors, 16-byte aligned) and their element counts."""

    def __init__(self, streams, counts, device="cuda"):
        import torch
        self.device = torch.device(device)
        self.streams = [s if s.data_ptr() % 16 == 0 else s.clone() for s in streams]
        self.counts = [int(c) for c in counts]
        caps = [_align16(max(4 * c, 16)) // 4 for c in self.counts]
        self.offsets = [0]
        for c in caps:
            self.offsets.append(self.offsets[-1] + c)
        self.caps = caps
        self.arena = torch.empty(max(4, self.offsets[-1]), dtype=torch.float32, device=self.device)
        arr = (FszDField * len(self.streams))()
        for i, s in enumerate(self.streams):
            arr[i].in_ = s.data_ptr()
            arr[i].in_bytes = s.numel()
            arr[i].out = self.arena.data_ptr() + 4 * self.offsets[i]
            arr[i].out_capacity_elems = caps[i]
        self.table = torch.frombuffer(bytearray(bytes(arr)), dtype=torch.uint8).to(self.device)
        self.cap_total = sum(caps)
        self.ws_bytes = fsz_batch_workspace_bytes(self.cap_total, len(self.streams))
        self.ws = _dev_buffer(self.ws_bytes, self.device)
        self._graph = None

    def run(self, stream=None) -> int:
        return fsz_decompress_batched(self.table.data_ptr(), len(self.streams), self.cap_total,
                                      self.ws.data_ptr(), self.ws_bytes, _stream_ptr(stream))

    def graph(self):
        if self._graph is None:
            self._graph = fsz_graph_decompress_batched(self.table.data_ptr(), len(self.streams),
                                                       self.cap_total, self.ws.data_ptr(),
                                                       self.ws_bytes)
        return self._graph

    def launch_graph(self, stream=None) -> int:
        return fsz_graph_launch(self.graph(), _stream_ptr(stream))

    def status(self, stream=None):
        per = (ctypes.c_uint32 * len(self.streams))()
        st = fsz_check_batched(self.ws.data_ptr(), len(self.streams), per, _stream_ptr(stream))
        return st, list(per)

    def output(self, i: int):
        return self.arena[self.offsets[i]:self.offsets[i] + self.counts[i]]

    def __del__(self):
        if getattr(self, "_graph", None) is not None:
            try:
                fsz_graph_destroy(self._graph)
            except Exception:
                pass
