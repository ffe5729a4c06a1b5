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
ERR_CAPACITY, ERR_CORRUPT, ERR_TIMEOUT, ERR_CUDA, ERR_WORKSPACE = 5, 6, 7, 8, 9
STATUS_NAMES = {0: "FSZ_OK", 1: "FSZ_ERR_INVALID_ARG", 2: "FSZ_ERR_ALIGN", 3: "FSZ_ERR_NONFINITE",
                4: "FSZ_ERR_EB_TOO_SMALL", 5: "FSZ_ERR_CAPACITY", 6: "FSZ_ERR_CORRUPT",
                7: "FSZ_ERR_TIMEOUT", 8: "FSZ_ERR_CUDA", 9: "FSZ_ERR_WORKSPACE"}
EB_ABS, EB_REL = 0, 1

# Every entry point include/fsz.h declares.
EXPORTS = ["fsz_compress_bound", "fsz_workspace_bytes", "fsz_batch_workspace_bytes", "fsz_compress",
           "fsz_compress_prepare", "fsz_compress_encode", "fsz_decompress", "fsz_compress_batched",
           "fsz_decompress_batched", "fsz_check", "fsz_check_batched", "fsz_read_header",
           "fsz_set_test_hooks", "fsz_version", "fsz_compress_noalloc"]


class FszDims(ctypes.Structure):
    _fields_ = [("ndim", ctypes.c_uint32), ("reserved", ctypes.c_uint32),
                ("dims", ctypes.c_uint64 * 3)]


class FszCField(ctypes.Structure):
    _fields_ = [("in_", ctypes.c_void_p), ("dims", FszDims), ("mode", ctypes.c_uint32),
                ("reserved", ctypes.c_uint32), ("eb", ctypes.c_double), ("out", ctypes.c_void_p),
                ("out_capacity", ctypes.c_uint64), ("out_bytes", ctypes.c_void_p)]


class FszDField(ctypes.Structure):
    _fields_ = [("in_", ctypes.c_void_p), ("in_bytes", ctypes.c_uint64), ("out", ctypes.c_void_p),
                ("out_capacity_elems", ctypes.c_uint64)]


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
            L.fsz_version.argtypes = []
            L.fsz_version.restype = ctypes.c_char_p
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
             out=None, stream=None, check: bool = True):
    """Compress a contiguous float32 CUDA tensor. Returns (stream_bytes_tensor, nbytes)."""
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
    st = fsz_compress(x.data_ptr(), make_dims(shape), mode, eb, out.data_ptr(), out.numel(),
                      nbytes.data_ptr(), ws.ptr, ws.bytes, sp)
    _check(st, "fsz_compress")
    if check:
        _check(fsz_check(ws.ptr, sp), "fsz_compress (device)")
    nb = int(nbytes[0].item())
    return out[:nb], nb


def decompress(stream_bytes, n: int | None = None, ws: Workspace | None = None, out=None,
               stream=None, check: bool = True):
    """Decompress a device byte tensor holding one stream. Returns a float32 tensor."""
    import torch
    assert stream_bytes.dtype == torch.uint8 and stream_bytes.is_cuda
    if n is None:
        n = fsz_read_header(stream_bytes[:64].cpu().numpy().tobytes())["n"]
    if out is None:
        out = torch.empty(max(n, 4), dtype=torch.float32, device=stream_bytes.device)
    ws = ws if ws is not None else Workspace(out.numel(), stream_bytes.device)
    src = stream_bytes
    if src.data_ptr() % 16:
        src = src.clone()
    sp = _stream_ptr(stream)
    st = fsz_decompress(src.data_ptr(), src.numel(), out.data_ptr(), out.numel(), ws.ptr, ws.bytes, sp)
    _check(st, "fsz_decompress")
    if check:
        _check(fsz_check(ws.ptr, sp), "fsz_decompress (device)")
    return out[:n]
