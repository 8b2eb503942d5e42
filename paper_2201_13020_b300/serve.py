"""Serving loop (Python side of szx_server_* in include/szx.h).

The loop itself runs in the library (C++): requests are admitted, oldest first,
as soon as one of the server's CUDA streams and room in the device pool are
free, their work overlaps on the device, and the compressed streams stay
resident in the pool.  This module builds the request table, owns the pool's
device memory (a torch tensor) and reads the outcomes back.
"""
import ctypes

from . import SZX_F32, SZX_F64, SzxError, _check, _dtype_code
from ._lib import lib

COMPRESS, DECOMPRESS = 0, 1


class _SzxRequest(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int), ("arrival_s", ctypes.c_double), ("d_in", ctypes.c_void_p),
                ("n", ctypes.c_size_t), ("dtype", ctypes.c_int), ("eb", ctypes.c_double), ("block", ctypes.c_uint32),
                ("source", ctypes.c_int), ("keep_output", ctypes.c_int), ("status", ctypes.c_int),
                ("admit_s", ctypes.c_double), ("done_s", ctypes.c_double), ("offset", ctypes.c_uint64),
                ("bytes", ctypes.c_uint64)]


def _bind():
    L = lib()
    if not getattr(L, "_serve_bound", False):
        vp, i, sz = ctypes.c_void_p, ctypes.c_int, ctypes.c_size_t
        L.szx_server_create.restype = i
        L.szx_server_create.argtypes = [vp, sz, i, ctypes.POINTER(vp)]
        L.szx_server_pool.restype = vp
        L.szx_server_pool.argtypes = [vp]
        L.szx_server_free_bytes.restype = sz
        L.szx_server_free_bytes.argtypes = [vp]
        L.szx_server_run.restype = i
        L.szx_server_run.argtypes = [vp, ctypes.POINTER(_SzxRequest), i, ctypes.POINTER(i)]
        L.szx_server_release.restype = i
        L.szx_server_release.argtypes = [vp, ctypes.c_uint64, ctypes.c_uint64]
        L.szx_server_destroy.restype = None
        L.szx_server_destroy.argtypes = [vp]
        L._serve_bound = True
    return L


class Request:
    """kind 'compress': x (contiguous CUDA f32/f64 tensor), eb, block.
    kind 'decompress': source = index (in the same run) of an earlier
    compress request; keep_output leaves the decoded values in the pool.
    After Server.run: status, admit_s, done_s (seconds from the run's start),
    offset and nbytes (the resident stream, or the kept output)."""

    def __init__(self, kind, arrival, x=None, eb=None, block=128, source=-1, keep_output=False):
        self.kind, self.arrival = kind, arrival
        self.x, self.eb, self.block = x, eb, block
        self.source, self.keep_output = source, keep_output
        self.status = None
        self.admit_s = self.done_s = None
        self.offset = self.nbytes = 0
        self.out_dtype = None
        self.nbytes_in = 0


class Server:
    """pool_bytes: size of the device pool the server allocates; or pool: a
    CUDA uint8 tensor to use as the pool instead (256-byte aligned), so that
    several servers in turn can share one long-lived allocation.  Allocating
    and freeing pools of many GB between runs is slow on the host for a while
    afterwards, which would show up as slower launches."""

    def __init__(self, pool_bytes=None, slots=8, device="cuda", pool=None):
        import torch
        L = _bind()
        self._t = torch
        if pool is not None:
            if pool.dtype != torch.uint8 or not pool.is_cuda or pool.data_ptr() % 256:
                raise ValueError("pool must be a 256-byte aligned CUDA uint8 tensor")
            self.pool = pool
            pool_bytes = pool.numel()
        else:
            self.pool = torch.empty(pool_bytes + 256, dtype=torch.uint8, device=device)
            off = (-self.pool.data_ptr()) % 256
            self.pool = self.pool[off:off + pool_bytes]
        self._srv = ctypes.c_void_p(0)
        _check(L.szx_server_create(ctypes.c_void_p(self.pool.data_ptr()), pool_bytes, slots,
                                   ctypes.byref(self._srv)), "szx_server_create")
        self.max_in_flight = 0

    def run(self, requests):
        """Run the requests to completion; returns the run's wall time (s).
        Raises MemoryError if a request could never fit the pool."""
        L = _bind()
        k = len(requests)
        arr = (_SzxRequest * k)()
        for i, r in enumerate(requests):
            a = arr[i]
            a.kind = COMPRESS if r.kind == "compress" else DECOMPRESS
            a.arrival_s = r.arrival
            a.source = -1
            if r.kind == "compress":
                a.d_in = r.x.data_ptr()
                a.n = r.x.numel()
                a.dtype = _dtype_code(r.x)
                a.eb = float(r.eb)
                a.block = r.block
                r.nbytes_in = r.x.numel() * r.x.element_size()
            else:
                a.source = int(r.source)
                a.keep_output = 1 if r.keep_output else 0
                src = requests[r.source] if 0 <= r.source < k else None
                if src is not None and src.kind == "compress":  # the library checks the rest
                    r.out_dtype = _dtype_code(src.x)
                    r.nbytes_in = src.x.numel() * src.x.element_size()
        peak = ctypes.c_int(0)
        st = L.szx_server_run(self._srv, arr, k, ctypes.byref(peak))
        self.max_in_flight = peak.value
        end = 0.0
        for r, a in zip(requests, arr):
            r.status, r.admit_s, r.done_s = a.status, a.admit_s, a.done_s
            r.offset, r.nbytes = int(a.offset), int(a.bytes)
            end = max(end, a.done_s)
        if st == 4:
            raise MemoryError("a request can never fit the pool")
        if st != 0:
            raise SzxError(st, "szx_server_run")
        return end

    def view(self, offset, nbytes):
        return self.pool[offset:offset + nbytes]

    def output(self, req):
        """The kept output of a decompress request, as values."""
        dt = self._t.float32 if req.out_dtype == SZX_F32 else self._t.float64
        return self.view(req.offset, req.nbytes).view(dt)

    def release(self, offset, nbytes):
        _check(_bind().szx_server_release(self._srv, offset, nbytes), "szx_server_release")

    def free_bytes(self):
        return _bind().szx_server_free_bytes(self._srv)

    def close(self):
        if self._srv:
            _bind().szx_server_destroy(self._srv)
            self._srv = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


__all__ = ["Server", "Request", "COMPRESS", "DECOMPRESS", "SZX_F32", "SZX_F64"]
