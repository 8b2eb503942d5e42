"""Compressed dump to a host file, and load back (one node).

dump() cuts a CUDA tensor into chunks and pipelines three stages so that
they overlap: the GPU compresses chunk k+1 (and k+2) on one CUDA stream while
chunk k's stream is copied to pinned host memory on another and the host writes
the previous chunk to the file.  Only each chunk's stream bytes cross PCIe: the
compressor reports the size in pinned, mapped memory, and the copy is issued
once it is known.  load() reads the chunks back, copies each to the device and
decompresses it into the output.

File layout (little endian):
  magic b"SZXDUMP1" | u32 dtype | u32 block | u64 n | f64 eb | u64 chunk values
  | u64 chunks, then per chunk: u64 stream bytes | the stream.
"""
import struct

from . import SZX_F32, SZX_F64, SzxError, SzxHeader, compress_async, compress_bound, decompress_async, \
    stream_max_bytes

_MAGIC = b"SZXDUMP1"
_HEAD = struct.Struct("<8sIIQdQQ")


def _code(t):
    import torch
    if t.dtype == torch.float32:
        return SZX_F32
    if t.dtype == torch.float64:
        return SZX_F64
    raise TypeError(f"unsupported dtype {t.dtype}")


def dump(x, eb, path, chunk_values=1 << 24, block=128):
    """Compress x (contiguous CUDA f32/f64) into the file at path.  Returns
    {"input_bytes", "file_bytes", "chunks"}."""
    import torch
    if not x.is_cuda or not x.is_contiguous():
        raise ValueError("x must be a contiguous CUDA tensor")
    flat = x.reshape(-1)
    n = flat.numel()
    code = _code(x)
    chunk_values = max(block, chunk_values // block * block)
    k_total = -(-n // chunk_values)
    cap = compress_bound(min(n, chunk_values), code, block)
    smax = stream_max_bytes(min(n, chunk_values), code, block)
    dev = [torch.empty(cap, dtype=torch.uint8, device=x.device) for _ in range(2)]
    host = [torch.empty(smax, dtype=torch.uint8, pin_memory=True) for _ in range(2)]
    res = torch.zeros((k_total, 2), dtype=torch.int64, pin_memory=True)  # device-visible result words
    sc, sd = torch.cuda.Stream(device=x.device), torch.cuda.Stream(device=x.device)
    ce = [torch.cuda.Event() for _ in range(k_total)]
    de = [torch.cuda.Event() for _ in range(k_total)]
    sc.wait_stream(torch.cuda.current_stream())

    def compress(k):
        lo = k * chunk_values
        part = flat[lo:min(n, lo + chunk_values)]
        compress_async(part, eb, block, dev[k % 2], res[k], stream=sc)
        ce[k].record(sc)

    file_bytes = 0
    with open(path, "wb") as f:
        f.write(_HEAD.pack(_MAGIC, code, block, n, float(eb), chunk_values, k_total))
        file_bytes += _HEAD.size
        for k in range(min(2, k_total)):
            compress(k)
        for k in range(k_total):
            ce[k].synchronize()
            nbytes, status = (int(v) for v in res[k].tolist())
            if status != 0:
                raise SzxError(status, f"compress of chunk {k}")
            with torch.cuda.stream(sd):
                host[k % 2][:nbytes].copy_(dev[k % 2][:nbytes], non_blocking=True)
            de[k].record(sd)
            if k + 2 < k_total:
                sc.wait_event(de[k])  # the device buffer is reused once copied
                compress(k + 2)
            de[k].synchronize()
            f.write(struct.pack("<Q", nbytes))
            f.write(memoryview(host[k % 2][:nbytes].numpy()))
            file_bytes += 8 + nbytes
    return {"input_bytes": n * x.element_size(), "file_bytes": file_bytes, "chunks": k_total}


def load(path, device="cuda", out=None):
    """Read a dump and decompress it on the device; returns the values."""
    import torch
    with open(path, "rb") as f:
        magic, code, block, n, eb, chunk_values, k_total = _HEAD.unpack(f.read(_HEAD.size))
        if magic != _MAGIC:
            raise ValueError("not an SZx dump")
        dt = torch.float32 if code == SZX_F32 else torch.float64
        if out is None:
            out = torch.empty(n, dtype=dt, device=device)
        smax = stream_max_bytes(min(n, chunk_values), code, block)
        host = [torch.empty(smax, dtype=torch.uint8, pin_memory=True) for _ in range(2)]
        dev = [torch.empty(smax, dtype=torch.uint8, device=device) for _ in range(2)]
        status = torch.zeros(k_total, dtype=torch.int32, device=device)
        s = torch.cuda.Stream(device=device)
        done = [torch.cuda.Event() for _ in range(k_total)]
        for k in range(k_total):
            if k >= 2:
                done[k - 2].synchronize()  # buffers k % 2 are free again
            nbytes = struct.unpack("<Q", f.read(8))[0]
            if nbytes > smax:
                raise ValueError("corrupt dump: chunk larger than its bound")
            f.readinto(memoryview(host[k % 2].numpy())[:nbytes])
            lo = k * chunk_values
            vals = min(n, lo + chunk_values) - lo
            with torch.cuda.stream(s):
                dev[k % 2][:nbytes].copy_(host[k % 2][:nbytes], non_blocking=True)
            h = SzxHeader()
            h.block, h.dtype, h.n, h.total_bytes = block, code, vals, nbytes
            w = 4 if code == SZX_F32 else 8
            h.tile_blocks = max(8, 32768 // (block * w))
            decompress_async(dev[k % 2][:nbytes], h, out[lo:lo + vals], status[k:k + 1], stream=s)
            done[k].record(s)
        s.synchronize()
    bad = int((status != 0).sum())
    if bad:
        raise SzxError(int(status.max()), "decompress of a dumped chunk")
    return out


__all__ = ["dump", "load"]
