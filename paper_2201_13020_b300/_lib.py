"""ctypes binding of libszx.so (the C ABI in include/szx.h).

Argument marshalling only: every step of compression and decompression runs in
the library's CUDA kernels.  There is no CPU fallback; if the in-tree library
is missing or cannot be loaded, every call raises.
"""
import ctypes
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "lib", "libszx.so")

SZX_F32, SZX_F64 = 0, 1
STATUS = {0: "SZX_OK", 1: "SZX_ERR_INVALID", 2: "SZX_ERR_TOO_SMALL", 3: "SZX_ERR_CORRUPT",
          4: "SZX_ERR_NOMEM", 5: "SZX_ERR_CUDA", 6: "SZX_ERR_TIMEOUT"}


class SzxHeader(ctypes.Structure):
    _fields_ = [("block", ctypes.c_uint32), ("tile_blocks", ctypes.c_uint32), ("n", ctypes.c_uint64),
                ("dtype", ctypes.c_int), ("e_bits", ctypes.c_uint64), ("nonconst", ctypes.c_uint64),
                ("raw", ctypes.c_uint64), ("escalated", ctypes.c_uint64), ("total_bytes", ctypes.c_uint64)]


class SzxField(ctypes.Structure):
    _fields_ = [("d_in", ctypes.c_void_p), ("n", ctypes.c_size_t), ("dtype", ctypes.c_int), ("eb", ctypes.c_double),
                ("block", ctypes.c_uint32), ("d_out", ctypes.c_void_p), ("out_capacity", ctypes.c_size_t)]


class SzxBatchGroup(ctypes.Structure):
    _fields_ = [("dtype", ctypes.c_int), ("block", ctypes.c_uint32), ("auto_block", ctypes.c_int),
                ("fields", ctypes.c_uint32), ("tiles", ctypes.c_uint64), ("ctas_per_sm", ctypes.c_int),
                ("warps_per_cta", ctypes.c_int), ("threads_per_cta", ctypes.c_uint32),
                ("values_per_lane", ctypes.c_uint32), ("blocks_per_warp", ctypes.c_uint32),
                ("tuned_ms", ctypes.c_float)]


class SzxStreamField(ctypes.Structure):
    _fields_ = [("d_in", ctypes.c_void_p), ("in_bytes", ctypes.c_size_t), ("header", SzxHeader),
                ("d_out", ctypes.c_void_p), ("out_capacity", ctypes.c_size_t), ("d_status", ctypes.c_void_p)]


_lib = None


def lib():
    """Load libszx.so once; raise if it is not built."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(f"{LIB_PATH} is missing: build it with `python -m paper_2201_13020_b300.build` "
                           "(or __graft_entry__.build()); there is no CPU fallback")
    L = ctypes.CDLL(LIB_PATH)
    sz, u32, u64, dbl, vp, i = (ctypes.c_size_t, ctypes.c_uint32, ctypes.c_uint64, ctypes.c_double,
                               ctypes.c_void_p, ctypes.c_int)
    L.szx_compress_bound.restype = sz
    L.szx_compress_bound.argtypes = [sz, i, u32]
    L.szx_stream_max_bytes.restype = sz
    L.szx_stream_max_bytes.argtypes = [sz, i, u32]
    L.szx_compress.restype = i
    L.szx_compress.argtypes = [vp, sz, i, dbl, u32, vp, sz, ctypes.POINTER(sz), vp]
    L.szx_compress_async.restype = i
    L.szx_compress_async.argtypes = [vp, sz, i, dbl, u32, vp, sz, vp, vp]
    L.szx_compress_static_async.restype = i
    L.szx_compress_static_async.argtypes = [vp, sz, i, dbl, u32, vp, sz, vp, vp]
    L.szx_header_read.restype = i
    L.szx_header_read.argtypes = [vp, sz, ctypes.POINTER(SzxHeader), vp]
    L.szx_decompress.restype = i
    L.szx_decompress.argtypes = [vp, sz, vp, sz, ctypes.POINTER(sz), ctypes.POINTER(i), vp]
    L.szx_decompress_range_async.restype = i
    L.szx_decompress_range_async.argtypes = [vp, sz, ctypes.POINTER(SzxHeader), sz, sz, vp, sz, vp, vp]
    L.szx_decompress_async.restype = i
    L.szx_decompress_async.argtypes = [vp, sz, ctypes.POINTER(SzxHeader), vp, sz, vp, vp]
    pp = ctypes.POINTER(ctypes.c_void_p)
    L.szx_batch_compress_plan.restype = i
    L.szx_batch_compress_plan.argtypes = [ctypes.POINTER(SzxField), i, pp]
    L.szx_batch_decompress_plan.restype = i
    L.szx_batch_decompress_plan.argtypes = [ctypes.POINTER(SzxStreamField), i, pp]
    L.szx_batch_workspace_bytes.restype = sz
    L.szx_batch_workspace_bytes.argtypes = [vp]
    L.szx_batch_upload.restype = i
    L.szx_batch_upload.argtypes = [vp, vp, sz, vp, vp]
    L.szx_batch_run.restype = i
    L.szx_batch_run.argtypes = [vp, vp, vp]
    L.szx_batch_autotune.restype = i
    L.szx_batch_autotune.argtypes = [vp, vp, vp]
    L.szx_batch_groups.restype = i
    L.szx_batch_groups.argtypes = [vp, ctypes.POINTER(i), i]
    L.szx_batch_group_info.restype = i
    L.szx_batch_group_info.argtypes = [vp, i, ctypes.POINTER(SzxBatchGroup)]
    L.szx_batch_set_group.restype = i
    L.szx_batch_set_group.argtypes = [vp, i, i, i]
    L.szx_batch_destroy.restype = None
    L.szx_batch_destroy.argtypes = [vp]
    L.szx_status_string.restype = ctypes.c_char_p
    L.szx_status_string.argtypes = [i]
    L.szx_version.restype = ctypes.c_char_p
    L.szx_version.argtypes = []
    _lib = L
    return L


EXPORTED = ["szx_compress_bound", "szx_stream_max_bytes", "szx_compress", "szx_compress_async",
            "szx_compress_static_async", "szx_decompress_range_async", "szx_batch_compress_plan", "szx_batch_decompress_plan",
            "szx_batch_workspace_bytes", "szx_batch_upload", "szx_batch_run", "szx_batch_autotune", "szx_batch_groups",
            "szx_batch_group_info", "szx_batch_set_group",
            "szx_batch_destroy", "szx_server_create", "szx_server_pool", "szx_server_free_bytes", "szx_server_run",
            "szx_server_release", "szx_server_destroy", "szx_header_read", "szx_decompress", "szx_decompress_async", "szx_status_string", "szx_version"]
