"""B300-native SZx block compressor / decompressor (arXiv 2201.13020).

Python binding of the C ABI in include/szx.h.  PyTorch supplies device memory
and streams; the codec itself runs in the library's sm_103a CUDA kernels.

    import paper_2201_13020_b300 as szx
    stream = szx.compress(x, eb)          # x: contiguous CUDA float32/float64
    y = szx.decompress(stream)            # |x - y| <= eb element-wise
"""
import ctypes

from ._lib import SZX_F32, SZX_F64, STATUS, SzxBatchGroup, SzxField, SzxHeader, SzxStreamField, lib

__all__ = ["compress", "decompress", "compress_async", "decompress_async", "decompress_range", "compress_bound",
           "stream_max_bytes", "header", "Batch", "batch_compress", "batch_decompress", "SzxError", "SZX_F32",
           "SZX_F64"]


class SzxError(RuntimeError):
    def __init__(self, status, what):
        name = STATUS.get(status, str(status))
        super().__init__(f"{what}: {name}")
        self.status = status


def _torch():
    import torch
    return torch


def _dtype_code(t):
    torch = _torch()
    if t.dtype == torch.float32:
        return SZX_F32
    if t.dtype == torch.float64:
        return SZX_F64
    raise TypeError(f"unsupported dtype {t.dtype}: float32 or float64")


def _stream_handle(stream):
    torch = _torch()
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


def _check(status, what):
    if status != 0:
        raise SzxError(status, what)


def compress_bound(n, dtype=SZX_F32, block=128):
    """Output-buffer bytes szx_compress needs (largest stream + scratch tail)."""
    return lib().szx_compress_bound(n, dtype, block)


def stream_max_bytes(n, dtype=SZX_F32, block=128):
    return lib().szx_stream_max_bytes(n, dtype, block)


def compress(x, eb, block=128, out=None, stream=None):
    """Compress a contiguous CUDA tensor; returns a uint8 view of the stream.
    block=0 picks the block length with metrics.choose_block (a sample of x
    compressed with b = 64, 128 and 256)."""
    torch = _torch()
    if not x.is_cuda or not x.is_contiguous():
        raise ValueError("x must be a contiguous CUDA tensor")
    code = _dtype_code(x)
    if block == 0:
        from .metrics import choose_block
        block, _ = choose_block(x, eb)
    n = x.numel()
    cap = compress_bound(n, code, block)
    if cap == 0:
        raise SzxError(1, "compress_bound")
    if out is None:
        out = torch.empty(cap, dtype=torch.uint8, device=x.device)
    nbytes = ctypes.c_size_t(0)
    _check(lib().szx_compress(ctypes.c_void_p(x.data_ptr()), n, code, float(eb), block,
                              ctypes.c_void_p(out.data_ptr()), out.numel(), ctypes.byref(nbytes),
                              _stream_handle(stream)), "szx_compress")
    return out[:nbytes.value]


def compress_async(x, eb, block, out, result, stream=None):
    """Enqueue compression; result (CUDA uint64 tensor of 2) gets {bytes, status}."""
    code = _dtype_code(x)
    _check(lib().szx_compress_async(ctypes.c_void_p(x.data_ptr()), x.numel(), code, float(eb), block,
                                    ctypes.c_void_p(out.data_ptr()), out.numel(),
                                    ctypes.c_void_p(result.data_ptr() if result is not None else 0),
                                    _stream_handle(stream)), "szx_compress_async")


def header(buf, stream=None):
    """Parse the header of a compressed CUDA uint8 tensor."""
    h = SzxHeader()
    _check(lib().szx_header_read(ctypes.c_void_p(buf.data_ptr()), buf.numel(), ctypes.byref(h),
                                 _stream_handle(stream)), "szx_header_read")
    return h


def header_dict(h):
    return {f: getattr(h, f) for f, _ in SzxHeader._fields_}


def decompress(buf, out=None, stream=None):
    """Decompress a CUDA uint8 tensor holding a stream; returns the values."""
    torch = _torch()
    if not buf.is_cuda:
        raise ValueError("stream must be a CUDA tensor")
    h = header(buf, stream)
    dt = torch.float32 if h.dtype == SZX_F32 else torch.float64
    if out is None:
        out = torch.empty(h.n, dtype=dt, device=buf.device)
    n = ctypes.c_size_t(0)
    d = ctypes.c_int(0)
    _check(lib().szx_decompress(ctypes.c_void_p(buf.data_ptr()), buf.numel(), ctypes.c_void_p(out.data_ptr()),
                                out.numel() * out.element_size(), ctypes.byref(n), ctypes.byref(d),
                                _stream_handle(stream)), "szx_decompress")
    return out


def decompress_async(buf, h, out, status=None, stream=None):
    """Enqueue decompression with a known header; status: CUDA uint32/int32 tensor of 1 or None."""
    _check(lib().szx_decompress_async(ctypes.c_void_p(buf.data_ptr()), buf.numel(), ctypes.byref(h),
                                      ctypes.c_void_p(out.data_ptr()), out.numel() * out.element_size(),
                                      ctypes.c_void_p(status.data_ptr() if status is not None else 0),
                                      _stream_handle(stream)), "szx_decompress_async")


def decompress_range(buf, first_block, nblocks, h=None, out=None, status=None, stream=None):
    """Decompress blocks [first_block, first_block + nblocks) of a stream (a
    CUDA uint8 tensor); h: its header (read from the device if None).  Returns
    the values of those blocks."""
    torch = _torch()
    if h is None:
        h = header(buf, stream)
    nvals = min(h.n, (first_block + nblocks) * h.block) - first_block * h.block
    if out is None:
        dt = torch.float32 if h.dtype == SZX_F32 else torch.float64
        out = torch.empty(max(nvals, 0), dtype=dt, device=buf.device)
    _check(lib().szx_decompress_range_async(ctypes.c_void_p(buf.data_ptr()), buf.numel(), ctypes.byref(h),
                                            first_block, nblocks, ctypes.c_void_p(out.data_ptr()),
                                            out.numel() * out.element_size(),
                                            ctypes.c_void_p(status.data_ptr() if status is not None else 0),
                                            _stream_handle(stream)), "szx_decompress_range_async")
    return out


class Batch:
    """A planned batch (see szx_batch_* in include/szx.h) with its device workspace.

    run() enqueues one run (one clear kernel and one persistent launch per
    (dtype, block) group) on the stream; it can be captured in a CUDA graph.
    """

    def __init__(self, plan, ws, keep):
        self._plan = plan
        self.ws = ws
        self._keep = keep  # tensors the plan points to

    def run(self, stream=None):
        _check(lib().szx_batch_run(self._plan, ctypes.c_void_p(self.ws.data_ptr()), _stream_handle(stream)),
               "szx_batch_run")

    def autotune(self, stream=None):
        """Time every shape of every group (see szx_batch_autotune) and keep
        the fastest; returns groups()."""
        _check(lib().szx_batch_autotune(self._plan, ctypes.c_void_p(self.ws.data_ptr()), _stream_handle(stream)),
               "szx_batch_autotune")
        return self.groups()

    def groups(self):
        """Each group's shape: dtype, block, fields, ctas_per_sm, warps_per_cta,
        threads_per_cta, values_per_lane, blocks_per_warp, tuned_ms."""
        L = lib()
        n = L.szx_batch_groups(self._plan, None, 0)
        out = []
        for i in range(n):
            g = SzxBatchGroup()
            _check(L.szx_batch_group_info(self._plan, i, ctypes.byref(g)), "szx_batch_group_info")
            out.append({f: getattr(g, f) for f, _ in SzxBatchGroup._fields_})
        return out

    def set_group(self, group, ctas_per_sm, warps_per_cta):
        """Set a group's shape by hand (ctas_per_sm 0, 1 or 2; warps 8 or 4)."""
        _check(lib().szx_batch_set_group(self._plan, group, ctas_per_sm, warps_per_cta), "szx_batch_set_group")

    def close(self):
        if self._plan:
            lib().szx_batch_destroy(self._plan)
            self._plan = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def _upload(plan, device, results, stream):
    torch = _torch()
    nbytes = lib().szx_batch_workspace_bytes(plan)
    ws = torch.empty(max(nbytes, 256) + 256, dtype=torch.uint8, device=device)
    off = (-ws.data_ptr()) % 256
    ws = ws[off:off + max(nbytes, 256)]
    st = lib().szx_batch_upload(plan, ctypes.c_void_p(ws.data_ptr()), ws.numel(),
                                ctypes.c_void_p(results.data_ptr() if results is not None else 0),
                                _stream_handle(stream))
    if st != 0:
        lib().szx_batch_destroy(plan)
        raise SzxError(st, "szx_batch_upload")
    return ws


# block lengths the batch autotuner tries for fields given block 0
AUTO_BLOCKS = (64, 128, 256)


def batch_compress(xs, ebs, blocks=128, outs=None, stream=None):
    """Plan and upload the compression of CUDA tensors xs (one bound each).
    A block of 0 lets Batch.autotune() choose b among 64, 128 and 256 for the
    block-0 fields of each dtype (128 until it runs).

    Returns (batch, outs, results): outs are uint8 buffers of
    stream_max_bytes each; after batch.run() and a synchronisation, field i's
    stream is outs[i][:results[2*i]] and results[2*i+1] its status.
    """
    torch = _torch()
    k = len(xs)
    if isinstance(blocks, int):
        blocks = [blocks] * k

    def cap(x, bk):
        if bk:
            return stream_max_bytes(x.numel(), _dtype_code(x), bk)
        return max(stream_max_bytes(x.numel(), _dtype_code(x), b) for b in AUTO_BLOCKS)

    if outs is None:
        outs = [torch.empty(cap(x, bk), dtype=torch.uint8, device=x.device) for x, bk in zip(xs, blocks)]
    arr = (SzxField * k)()
    for i, (x, eb, bk, o) in enumerate(zip(xs, ebs, blocks, outs)):
        if not x.is_cuda or not x.is_contiguous():
            raise ValueError("fields must be contiguous CUDA tensors")
        arr[i] = SzxField(x.data_ptr(), x.numel(), _dtype_code(x), float(eb), bk, o.data_ptr(), o.numel())
    plan = ctypes.c_void_p(0)
    _check(lib().szx_batch_compress_plan(arr, k, ctypes.byref(plan)), "szx_batch_compress_plan")
    results = torch.zeros(2 * k, dtype=torch.int64, device=xs[0].device)
    ws = _upload(plan, xs[0].device, results, stream)
    return Batch(plan, ws, (list(xs), list(outs), results)), outs, results


def batch_decompress(bufs, headers, outs=None, statuses=None, stream=None):
    """Plan and upload the decompression of streams (CUDA uint8 tensors) whose
    headers are known.  Returns (batch, outs, statuses)."""
    torch = _torch()
    k = len(bufs)
    if outs is None:
        outs = [torch.empty(h.n, dtype=torch.float32 if h.dtype == SZX_F32 else torch.float64, device=b.device)
                for b, h in zip(bufs, headers)]
    if statuses is None:
        statuses = torch.zeros(k, dtype=torch.int32, device=bufs[0].device)
    arr = (SzxStreamField * k)()
    for i, (b, h, o) in enumerate(zip(bufs, headers, outs)):
        arr[i] = SzxStreamField(b.data_ptr(), b.numel(), h, o.data_ptr(), o.numel() * o.element_size(),
                                statuses.data_ptr() + 4 * i)
    plan = ctypes.c_void_p(0)
    _check(lib().szx_batch_decompress_plan(arr, k, ctypes.byref(plan)), "szx_batch_decompress_plan")
    ws = _upload(plan, bufs[0].device, None, stream)
    return Batch(plan, ws, (list(bufs), list(outs), statuses)), outs, statuses
