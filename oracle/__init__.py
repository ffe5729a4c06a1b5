"""FSZ CPU oracle (TEST INFRASTRUCTURE ONLY).

ctypes wrapper around ``fsz_oracle.cpp``, a plain single-threaded C++
restatement of the FSZ stream (arXiv 2607.15413). Only the tests, the smoke
check and the benchmark's CPU-baseline leg may import this package; the
product path (the CUDA library and its binding) never does.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "fsz_oracle.cpp")
_HDR = os.path.join(_HERE, "fsz_oracle.h")
_LIBDIR = os.path.join(_HERE, "_lib")
_LIB = os.path.join(_LIBDIR, "libfsz_oracle.so")
# All-core timing driver (the oracle's functions over element and tile ranges, one thread
# per range; for the benchmark's CPU baseline only).
_SRC_MT = os.path.join(_HERE, "fsz_oracle_mt.cpp")
_LIB_MT = os.path.join(_LIBDIR, "libfsz_oracle_mt.so")

ABS, REL = 0, 1
LZ1, LZ2, LZ1C, LZ2C = 0, 1, 2, 3
# Features switched off (Sec. 6.4 ablation); 0 is the full method.
OFF_CROSS, OFF_CENTER, OFF_LZ2 = 1, 2, 4
# The ablation's cumulative steps: Base (LZ1, independent blocks), +Cross, +Cent., +LZ2.
ABLATION = (("base", OFF_CROSS | OFF_CENTER | OFF_LZ2), ("+cross", OFF_CENTER | OFF_LZ2),
            ("+center", OFF_LZ2), ("+lz2", 0))
OK, ERR_INVALID_ARG, ERR_NONFINITE, ERR_EB_TOO_SMALL, ERR_CAPACITY, ERR_CORRUPT = 0, 1, 3, 4, 5, 6

# -ffp-contract=off keeps every float32 multiply and add a separate IEEE
# operation (GCC contracts to FMA by default on aarch64).
CFLAGS = ["-std=c++17", "-O2", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared",
          "-Wall", "-Wextra"]

_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle (and its all-core timing driver) into oracle/_lib (idempotent)."""
    os.makedirs(_LIBDIR, exist_ok=True)
    newest = max(os.path.getmtime(_SRC), os.path.getmtime(_HDR))
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < newest:
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.run(["g++", *CFLAGS, "-o", tmp, _SRC], check=True)
        os.replace(tmp, _LIB)
    newest = max(newest, os.path.getmtime(_SRC_MT))
    if force or not os.path.exists(_LIB_MT) or os.path.getmtime(_LIB_MT) < newest:
        tmp = _LIB_MT + f".tmp{os.getpid()}"
        subprocess.run(["g++", *CFLAGS, "-pthread", "-o", tmp, _SRC_MT, _SRC], check=True)
        os.replace(tmp, _LIB_MT)
    return _LIB


_lib_mt = None


def lib_mt():
    """The all-core timing driver (loaded on first use)."""
    global _lib_mt
    with _lock:
        if _lib_mt is None:
            build()
            L = ctypes.CDLL(_LIB_MT)
            P, u64, u32, f64 = ctypes.c_void_p, ctypes.c_uint64, ctypes.c_uint32, ctypes.c_double
            L.fszo_mt_compress.argtypes = [P, u32, P, ctypes.c_int, f64, P, u64, P, ctypes.c_int]
            L.fszo_mt_decompress.argtypes = [P, u64, P, u64, P, ctypes.c_int]
            _lib_mt = L
    return _lib_mt


class Params(ctypes.Structure):
    _fields_ = [("eb", ctypes.c_double), ("eb_eff", ctypes.c_double), ("K", ctypes.c_double),
                ("Q", ctypes.c_uint32), ("e", ctypes.c_float), ("s", ctypes.c_float),
                ("r", ctypes.c_float)]


def lib():
    global _lib
    with _lock:
        if _lib is None:
            L = ctypes.CDLL(build())
            P, u64, i32, u32, f32, f64 = (ctypes.c_void_p, ctypes.c_uint64, ctypes.c_int32,
                                          ctypes.c_uint32, ctypes.c_float, ctypes.c_double)
            L.fszo_stats.argtypes = [P, u64, P, P, P]
            L.fszo_params.argtypes = [ctypes.c_int, f64, f32, f32, ctypes.c_int, u64,
                                      ctypes.POINTER(Params)]
            L.fszo_quantize.argtypes = [f32, f32]
            L.fszo_quantize.restype = i32
            L.fszo_dequantize.argtypes = [i32, f32]
            L.fszo_dequantize.restype = f32
            L.fszo_tile_mu.argtypes = [P, f32]
            L.fszo_tile_mu.restype = i32
            L.fszo_tile_residuals.argtypes = [P, i32, ctypes.c_int, P]
            L.fszo_tile_residuals.restype = None
            L.fszo_rate.argtypes = [u32]
            L.fszo_rate.restype = u32
            L.fszo_block_cost.argtypes = [u32]
            L.fszo_block_cost.restype = u32
            L.fszo_tile_costs_single_pass.argtypes = [P, i32, P, P]
            L.fszo_tile_costs_single_pass.restype = None
            L.fszo_tile_costs_four_pass.argtypes = [P, i32, P, P]
            L.fszo_tile_costs_four_pass.restype = None
            L.fszo_select.argtypes = [P]
            L.fszo_compress_bound.argtypes = [u64]
            L.fszo_compress_bound.restype = u64
            L.fszo_compress.argtypes = [P, u32, P, ctypes.c_int, f64, P, u64, P, ctypes.c_int]
            L.fszo_read_preamble.argtypes = [P, u64, P, P, P, P, P, P]
            L.fszo_compress_tiles.argtypes = [P, u64, f32, u64, u64, P, P, u64, P]
            L.fszo_decompress.argtypes = [P, u64, P, u64, P]
            L.fszo_decompress_q.argtypes = [P, u64, P, u64, P]
            L.fszo_features_valid.argtypes = [u32]
            L.fszo_tile_residuals_f.argtypes = [P, i32, ctypes.c_int, u32, P]
            L.fszo_tile_residuals_f.restype = None
            L.fszo_tile_costs_single_pass_f.argtypes = [P, i32, u32, P, P]
            L.fszo_tile_costs_single_pass_f.restype = None
            L.fszo_tile_costs_four_pass_f.argtypes = [P, i32, u32, P, P]
            L.fszo_tile_costs_four_pass_f.restype = None
            L.fszo_select_f.argtypes = [P, u32]
            L.fszo_compress_f.argtypes = [P, u32, P, ctypes.c_int, f64, u32, P, u64, P,
                                          ctypes.c_int]
            L.fszo_compress_tiles_f.argtypes = [P, u64, f32, u64, u64, u32, P, P, u64, P]
            L.fszo_read_preamble_f.argtypes = [P, u64, P, P, P, P, P, P, P]
            L.fszo_quality.argtypes = [P, P, u64, f64, u64, P]
            L.fszo_tile_word.argtypes = [ctypes.c_int, ctypes.c_int]
            L.fszo_tile_word.restype = u32
            L.fszo_compress_bound_cfg.argtypes = [u64, ctypes.c_int, ctypes.c_int]
            L.fszo_compress_bound_cfg.restype = u64
            L.fszo_compress_cfg.argtypes = [P, u32, P, ctypes.c_int, f64, u32, ctypes.c_int,
                                            ctypes.c_int, P, u64, P]
            _lib = L
    return _lib


def _ptr(a: np.ndarray) -> int:
    return a.ctypes.data


class Quality(ctypes.Structure):
    _fields_ = [("n", ctypes.c_uint64), ("over_bound", ctypes.c_uint64),
                ("max_abs_err", ctypes.c_double), ("sum_sq_err", ctypes.c_double),
                ("vmin", ctypes.c_double), ("vmax", ctypes.c_double), ("psnr_db", ctypes.c_double),
                ("nrmse", ctypes.c_double), ("bit_rate", ctypes.c_double)]


class OracleError(RuntimeError):
    def __init__(self, status: int, what: str):
        super().__init__(f"{what}: oracle status {status}")
        self.status = status


def stats(d: np.ndarray):
    d = np.ascontiguousarray(d, dtype=np.float32)
    lo, hi, fin = ctypes.c_float(), ctypes.c_float(), ctypes.c_int()
    lib().fszo_stats(_ptr(d), d.size, ctypes.byref(lo), ctypes.byref(hi), ctypes.byref(fin))
    return lo.value, hi.value, bool(fin.value)


def params(mode: int, eb: float, vmin: float, vmax: float, finite: bool = True, n: int = 1):
    p = Params()
    st = lib().fszo_params(mode, eb, vmin, vmax, int(finite), n, ctypes.byref(p))
    if st != OK:
        raise OracleError(st, "params")
    return p


def params_for(d: np.ndarray, mode: int, eb: float) -> Params:
    lo, hi, fin = stats(d)
    return params(mode, eb, lo, hi, fin, int(np.asarray(d).size))


def quantize(d: np.ndarray, r: float) -> np.ndarray:
    L = lib()
    return np.array([L.fszo_quantize(float(x), r) for x in np.asarray(d, np.float32).ravel()],
                    dtype=np.int32)


def tile_mu(d256: np.ndarray, r: float) -> int:
    d = np.ascontiguousarray(d256, dtype=np.float32)
    assert d.size == 256
    return lib().fszo_tile_mu(_ptr(d), r)


def tile_residuals(q256: np.ndarray, mu: int, variant: int, features_off: int = 0) -> np.ndarray:
    q = np.ascontiguousarray(q256, dtype=np.int32)
    assert q.size == 256
    out = np.zeros(256, np.int32)
    lib().fszo_tile_residuals_f(_ptr(q), mu, variant, features_off, _ptr(out))
    return out


def features_valid(features_off: int) -> bool:
    return bool(lib().fszo_features_valid(features_off))


def rate(maxabs: int) -> int:
    return lib().fszo_rate(maxabs)


def block_cost(r: int) -> int:
    return lib().fszo_block_cost(r)


def tile_costs(q256: np.ndarray, mu: int, four_pass: bool = False, features_off: int = 0):
    q = np.ascontiguousarray(q256, dtype=np.int32)
    assert q.size == 256
    C = np.zeros(4, np.uint32)
    rates = np.zeros(32, np.uint8)
    fn = lib().fszo_tile_costs_four_pass_f if four_pass else lib().fszo_tile_costs_single_pass_f
    fn(_ptr(q), mu, features_off, _ptr(C), _ptr(rates))
    return C, rates.reshape(4, 8)


def select(C: np.ndarray, features_off: int = 0) -> int:
    c = np.ascontiguousarray(C, dtype=np.uint32)
    return lib().fszo_select_f(_ptr(c), features_off)


def compress_bound(n: int) -> int:
    return lib().fszo_compress_bound(n)


def compress(d: np.ndarray, eb: float, mode: int = REL, dims=None, force_variant: int = -1,
             features_off: int = 0) -> bytes:
    d = np.ascontiguousarray(d, dtype=np.float32)
    if dims is None:
        dims = d.shape if d.ndim >= 1 else (d.size,)
    dims_arr = np.zeros(3, np.uint64)
    dims_arr[: len(dims)] = dims
    cap = compress_bound(d.size)
    out = np.zeros(cap, np.uint8)
    nb = ctypes.c_uint64()
    st = lib().fszo_compress_f(_ptr(d), len(dims), _ptr(dims_arr), mode, eb, features_off,
                               _ptr(out), cap, ctypes.byref(nb), force_variant)
    if st != OK:
        raise OracleError(st, "compress")
    return out[: nb.value].tobytes()


# Tile configurations of Sec. 6.5 (Table 8): (B, T) = (elements per block, blocks per tile).
TILE_CONFIGS = ((32, 4), (32, 8), (32, 16), (64, 4), (64, 8), (64, 16))


def tile_word(B: int, T: int) -> int:
    return lib().fszo_tile_word(B, T)


def compress_cfg(d: np.ndarray, eb: float, mode: int = REL, B: int = 32, T: int = 8,
                 features_off: int = 0, dims=None) -> bytes:
    """A stream with B-element blocks and T blocks per tile (the four variants costed by
    definition); B = 32, T = 8 gives the default stream."""
    d = np.ascontiguousarray(d, dtype=np.float32)
    if dims is None:
        dims = d.shape if d.ndim >= 1 else (d.size,)
    dims_arr = np.zeros(3, np.uint64)
    dims_arr[: len(dims)] = dims
    cap = lib().fszo_compress_bound_cfg(d.size, B, T)
    out = np.zeros(cap, np.uint8)
    nb = ctypes.c_uint64()
    st = lib().fszo_compress_cfg(_ptr(d), len(dims), _ptr(dims_arr), mode, eb, features_off, B, T,
                                 _ptr(out), cap, ctypes.byref(nb))
    if st != OK:
        raise OracleError(st, "compress_cfg")
    return out[: nb.value].tobytes()


def compress_tiles(d: np.ndarray, r: float, t0: int, t1: int, features_off: int = 0):
    """Headers (8 bytes per tile) and data of tiles [t0, t1) of field d, given r = 1/s."""
    d = np.ascontiguousarray(d, dtype=np.float32).ravel()
    hdr = np.zeros(8 * max(t1 - t0, 1), np.uint8)
    cap = 772 * max(t1 - t0, 1)
    data = np.zeros(cap, np.uint8)
    nb = ctypes.c_uint64()
    st = lib().fszo_compress_tiles_f(_ptr(d), d.size, r, t0, t1, features_off, _ptr(hdr),
                                     _ptr(data), cap, ctypes.byref(nb))
    if st != OK:
        raise OracleError(st, "compress_tiles")
    return hdr[: 8 * (t1 - t0)].tobytes(), data[: nb.value].tobytes()


def read_preamble(stream: bytes):
    buf = np.frombuffer(stream, np.uint8)
    n, ndim, s, db = ctypes.c_uint64(), ctypes.c_uint32(), ctypes.c_float(), ctypes.c_uint64()
    dims = np.zeros(3, np.uint64)
    eb = ctypes.c_double()
    off = ctypes.c_uint32()
    st = lib().fszo_read_preamble_f(_ptr(buf), buf.size, ctypes.byref(n), ctypes.byref(ndim),
                                    _ptr(dims), ctypes.byref(eb), ctypes.byref(s),
                                    ctypes.byref(db), ctypes.byref(off))
    if st != OK:
        raise OracleError(st, "read_preamble")
    w = off.value
    B = 64 if (w >> 8) & 0xF == 1 else 32
    T = {0: 8, 1: 4, 2: 16}.get((w >> 12) & 0xF, 0)
    return dict(n=n.value, ndim=ndim.value, dims=tuple(int(x) for x in dims[: ndim.value]),
                eb=eb.value, s=s.value, data_bytes=db.value, features_off=w & 7, method_word=w,
                B=B, T=T)


def decompress(stream: bytes, q: bool = False) -> np.ndarray:
    buf = np.frombuffer(stream, np.uint8)
    info = read_preamble(stream)
    n = info["n"]
    out = np.zeros(max(n, 1), np.int32 if q else np.float32)
    nn = ctypes.c_uint64()
    fn = lib().fszo_decompress_q if q else lib().fszo_decompress
    st = fn(_ptr(buf), buf.size, _ptr(out), n, ctypes.byref(nn))
    if st != OK:
        raise OracleError(st, "decompress")
    return out[:n]


def quality(d: np.ndarray, y: np.ndarray, eb: float, stream_bytes: int = 0) -> dict:
    """Reconstruction quality (PSNR, NRMSE, max error, bit rate) of y against d."""
    d = np.ascontiguousarray(d, dtype=np.float32).ravel()
    y = np.ascontiguousarray(y, dtype=np.float32).ravel()
    assert d.size == y.size
    q = Quality()
    st = lib().fszo_quality(_ptr(d), _ptr(y), d.size, eb, stream_bytes, ctypes.byref(q))
    if st != OK:
        raise OracleError(st, "quality")
    return {k: getattr(q, k) for k, _ in Quality._fields_}


def decompress_status(stream: bytes, cap: int | None = None) -> int:
    """Status of a decode attempt (corrupt-stream tests); never raises."""
    buf = np.frombuffer(stream, np.uint8) if len(stream) else np.zeros(1, np.uint8)
    cap = (1 << 24) if cap is None else cap
    out = np.zeros(max(cap, 1), np.float32)
    nn = ctypes.c_uint64()
    return lib().fszo_decompress(_ptr(buf), len(stream), _ptr(out), cap, ctypes.byref(nn))


def mt_compress(d: np.ndarray, eb: float, mode: int = REL, dims=None, nthreads: int = 0) -> bytes:
    """The oracle's stream computed on `nthreads` host threads (all cores by default): the
    same bytes as compress(); for timing the all-core CPU baseline."""
    d = np.ascontiguousarray(d, dtype=np.float32)
    if dims is None:
        dims = d.shape if d.ndim >= 1 else (d.size,)
    dims_arr = np.zeros(3, np.uint64)
    dims_arr[: len(dims)] = dims
    cap = compress_bound(d.size)
    out = np.zeros(cap, np.uint8)
    nb = ctypes.c_uint64()
    st = lib_mt().fszo_mt_compress(_ptr(d), len(dims), _ptr(dims_arr), mode, eb, _ptr(out), cap,
                                   ctypes.byref(nb), nthreads or (os.cpu_count() or 1))
    if st != OK:
        raise OracleError(st, "mt_compress")
    return out[: nb.value].tobytes()


def mt_decompress(stream: bytes, nthreads: int = 0) -> np.ndarray:
    """decompress() on `nthreads` host threads (all cores by default); valid streams of the
    default tile configuration."""
    buf = np.frombuffer(stream, np.uint8)
    n = read_preamble(stream)["n"]
    out = np.zeros(max(n, 1), np.float32)
    nn = ctypes.c_uint64()
    st = lib_mt().fszo_mt_decompress(_ptr(buf), buf.size, _ptr(out), n, ctypes.byref(nn),
                                     nthreads or (os.cpu_count() or 1))
    if st != OK:
        raise OracleError(st, "mt_decompress")
    return out[:n]
