"""ctypes wrapper of the CPU oracle (test infrastructure, not product code).

Only tests/, __graft_entry__.smoke() and bench.py's cpu_baseline / reference
arm may import this package.  It never imports the CUDA library, and the CUDA
library never imports it.
"""
import ctypes

import numpy as np

from . import build as _build

F32, F64 = 0, 1
OK, ERR_INVALID, ERR_TOO_SMALL, ERR_CORRUPT = 0, 1, 2, 3

_lib = None


def lib():
    global _lib
    if _lib is None:
        path = _build.build()
        L = ctypes.CDLL(path)
        L.szx_ref_compress_bound.restype = ctypes.c_size_t
        L.szx_ref_compress_bound.argtypes = [ctypes.c_size_t, ctypes.c_int, ctypes.c_uint32]
        L.szx_ref_compress.restype = ctypes.c_int
        L.szx_ref_compress.argtypes = [ctypes.c_void_p, ctypes.c_size_t, ctypes.c_int, ctypes.c_double,
                                       ctypes.c_uint32, ctypes.c_void_p, ctypes.c_size_t,
                                       ctypes.POINTER(ctypes.c_size_t)]
        L.szx_ref_decompress.restype = ctypes.c_int
        L.szx_ref_decompress.argtypes = [ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p, ctypes.c_size_t,
                                         ctypes.POINTER(ctypes.c_size_t), ctypes.POINTER(ctypes.c_int)]
        L.szx_ref_error_bound_bits.restype = ctypes.c_uint64
        L.szx_ref_error_bound_bits.argtypes = [ctypes.c_double, ctypes.c_int]
        L.szx_ref_shift_overhead_bits.restype = ctypes.c_int
        L.szx_ref_shift_overhead_bits.argtypes = [ctypes.c_void_p, ctypes.c_size_t, ctypes.c_int, ctypes.c_double,
                                                  ctypes.c_uint32, ctypes.POINTER(ctypes.c_uint64),
                                                  ctypes.POINTER(ctypes.c_uint64)]
        _lib = L
    return _lib


class OracleError(RuntimeError):
    def __init__(self, status, what):
        super().__init__(f"oracle {what} failed with status {status}")
        self.status = status


def dtype_code(arr):
    if arr.dtype == np.float32:
        return F32
    if arr.dtype == np.float64:
        return F64
    raise TypeError(f"unsupported dtype {arr.dtype}")


def compress_bound(n, dtype, block=128):
    return lib().szx_ref_compress_bound(n, dtype, block)


def compress(arr, eb, block=128):
    """Compress a 1-D float32/float64 numpy array; returns the stream as a uint8 array."""
    arr = np.ascontiguousarray(arr)
    code = dtype_code(arr)
    cap = compress_bound(arr.size, code, block)
    out = np.zeros(max(cap, 64), dtype=np.uint8)
    nbytes = ctypes.c_size_t(0)
    st = lib().szx_ref_compress(arr.ctypes.data, arr.size, code, float(eb), block,
                                out.ctypes.data, out.size, ctypes.byref(nbytes))
    if st != OK:
        raise OracleError(st, "compress")
    return out[:nbytes.value].copy()


def decompress(stream):
    """Decompress a uint8 stream; returns a float32/float64 numpy array."""
    stream = np.ascontiguousarray(stream, dtype=np.uint8)
    n = ctypes.c_size_t(0)
    dt = ctypes.c_int(-1)
    st = lib().szx_ref_decompress(stream.ctypes.data, stream.size, None, 0, ctypes.byref(n), ctypes.byref(dt))
    if st not in (OK, ERR_INVALID):
        raise OracleError(st, "decompress")
    if dt.value not in (F32, F64):
        raise OracleError(ERR_CORRUPT, "decompress")
    out = np.empty(n.value, dtype=np.float32 if dt.value == F32 else np.float64)
    st = lib().szx_ref_decompress(stream.ctypes.data, stream.size, out.ctypes.data, out.nbytes,
                                  ctypes.byref(n), ctypes.byref(dt))
    if st != OK:
        raise OracleError(st, "decompress")
    return out


def decompress_status(stream):
    """Status code of decompressing `stream` (for corruption tests)."""
    stream = np.ascontiguousarray(stream, dtype=np.uint8)
    n = ctypes.c_size_t(0)
    dt = ctypes.c_int(-1)
    st = lib().szx_ref_decompress(stream.ctypes.data, stream.size, None, 0, ctypes.byref(n), ctypes.byref(dt))
    if st != ERR_INVALID:
        return st
    out = np.empty(n.value * (4 if dt.value == F32 else 8), dtype=np.uint8)
    return lib().szx_ref_decompress(stream.ctypes.data, stream.size, out.ctypes.data, out.nbytes,
                                    ctypes.byref(n), ctypes.byref(dt))


def error_bound(eb, dtype):
    """The absolute bound the codec uses for eb (f32: rounded toward zero)."""
    bits = lib().szx_ref_error_bound_bits(float(eb), dtype)
    if dtype == F32:
        return float(np.array([bits], dtype=np.uint64).astype(np.uint32).view(np.float32)[0])
    return float(np.array([bits], dtype=np.uint64).view(np.float64)[0])


def shift_overhead_bits(arr, eb, block=128):
    """(bits with the Eq. 5 right shift, bits of an unshifted bit-granular packing)."""
    arr = np.ascontiguousarray(arr)
    c = ctypes.c_uint64(0)
    ab = ctypes.c_uint64(0)
    st = lib().szx_ref_shift_overhead_bits(arr.ctypes.data, arr.size, dtype_code(arr), float(eb), block,
                                           ctypes.byref(c), ctypes.byref(ab))
    if st != OK:
        raise OracleError(st, "shift_overhead_bits")
    return c.value, ab.value
