"""szx_compress_static_async: compression whose scratch is a fixed array in
the library, called through the C ABI and compared with szx_compress_async.

The file is collected last on purpose: it must pass both alone and after every
other test, when the library's device array has already been used.
"""
import ctypes

import pytest

from paper_2201_13020_b300 import _lib
from paper_2201_13020_b300 import inputs

SZX_OK, SZX_ERR_INVALID, SZX_ERR_TOO_SMALL = 0, 1, 2
GUARD = 4096


def _vp(p):
    return ctypes.c_void_p(p)


def _tile_values(dtype, block):
    """Values per tile: G = max(8, 32768 / (b * w)) blocks of b values."""
    w = 4 if dtype == _lib.SZX_F32 else 8
    return max(8, 32768 // (block * w)) * block


@pytest.mark.parametrize("dtype,block", [(_lib.SZX_F32, 128), (_lib.SZX_F64, 128), (_lib.SZX_F64, 1024),
                                         (_lib.SZX_F32, 32)])
def test_static_limit_and_capacity_rejected_on_host(dtype, block):
    # Every check below returns before any CUDA call, so the fake (aligned,
    # non-null) device addresses are never dereferenced.  f64 with b = 1024 is
    # the geometry where a tile holds the minimum of 8 blocks (64 KiB).
    L = _lib.lib()
    max_tiles = ((1 << 20) - 128) // 8
    tile = _tile_values(dtype, block)
    # one tile beyond the array: rejected as too large for the fixed scratch
    n_over = (max_tiles + 1) * tile
    st = L.szx_compress_static_async(_vp(256), n_over, dtype, 1e-3, block, _vp(512), 1 << 62, None, None)
    assert st == SZX_ERR_INVALID
    # so is a ragged tile past the limit
    st = L.szx_compress_static_async(_vp(256), max_tiles * tile + 1, dtype, 1e-3, block, _vp(512), 1 << 62,
                                     None, None)
    assert st == SZX_ERR_INVALID
    # exactly the limit is accepted by the tile check: a capacity just short
    # of the stream maximum then fails on capacity, not on the tile count
    n_max = max_tiles * tile
    smax = L.szx_stream_max_bytes(n_max, dtype, block)
    assert smax > 0
    st = L.szx_compress_static_async(_vp(256), n_max, dtype, 1e-3, block, _vp(512), smax - 16, None, None)
    assert st == SZX_ERR_TOO_SMALL
    n_ok = 10_000
    smax = L.szx_stream_max_bytes(n_ok, dtype, block)
    st = L.szx_compress_static_async(_vp(256), n_ok, dtype, 1e-3, block, _vp(512), smax - 16, None, None)
    assert st == SZX_ERR_TOO_SMALL


@pytest.mark.gpu
def test_static_scratch_matches_existing_entry_point_twice_in_a_row():
    torch = pytest.importorskip("torch")
    L = _lib.lib()
    dev = torch.device("cuda:0")
    s = torch.cuda.current_stream()
    h = _vp(s.cuda_stream)
    # Calls in a row, each smaller than the one before, so that their tiles
    # reuse look-back words the earlier calls left behind.  The first (500
    # tiles) clears the words with a kernel, the others (108 and 30 tiles)
    # with a memset.
    cases = [
        (inputs.grf_3d((160, 160, 160), -5.0 / 3.0, 10, dtype=torch.float32), 1e-3, 128),
        (inputs.grf_3d((96, 96, 96), -5.0 / 3.0, 11, dtype=torch.float32), 1e-3, 128),
        (inputs.grf_3d((40, 50, 61), -11.0 / 3.0, 12, dtype=torch.float64), 1e-4, 256),
    ]
    for xc, rel, block in cases:
        x = xc.reshape(-1).to(dev)
        n = x.numel()
        code = _lib.SZX_F32 if x.dtype == torch.float32 else _lib.SZX_F64
        eb = inputs.rel_to_abs(xc, rel)
        smax = L.szx_stream_max_bytes(n, code, block)
        # Static path: a buffer of exactly the stream maximum plus a guard
        # region that must come back untouched.
        buf = torch.full((smax + GUARD,), 0xA5, dtype=torch.uint8, device=dev)
        res_s = torch.zeros(2, dtype=torch.int64, device=dev)
        st = L.szx_compress_static_async(_vp(x.data_ptr()), n, code, float(eb), block, _vp(buf.data_ptr()),
                                         smax, _vp(res_s.data_ptr()), h)
        assert st == SZX_OK
        # Existing path.
        cap = L.szx_compress_bound(n, code, block)
        ref = torch.empty(cap, dtype=torch.uint8, device=dev)
        res_r = torch.zeros(2, dtype=torch.int64, device=dev)
        st = L.szx_compress_async(_vp(x.data_ptr()), n, code, float(eb), block, _vp(ref.data_ptr()), cap,
                                  _vp(res_r.data_ptr()), h)
        assert st == SZX_OK
        torch.cuda.synchronize()
        rs, rr = res_s.cpu().tolist(), res_r.cpu().tolist()
        assert rr[1] == SZX_OK and rs == rr
        nbytes = rr[0]
        assert torch.equal(buf[:nbytes], ref[:nbytes])
        # nothing is written past the stream's own bytes: neither inside the
        # capacity nor in the guard region after it
        assert bool((buf[nbytes:smax] == 0xA5).all())
        assert bool((buf[smax:] == 0xA5).all())
