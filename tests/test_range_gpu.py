"""Random access: decompressing a block range gives exactly the bits a full
decompression puts there, for ranges inside a tile, across tile boundaries,
at the ragged end, and for the whole stream."""
import numpy as np
import pytest

import oracle

torch = pytest.importorskip("torch")
import paper_2201_13020_b300 as szx  # noqa: E402
from paper_2201_13020_b300 import inputs  # noqa: E402

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("dtype,block", [(np.float32, 128), (np.float64, 256), (np.float32, 32),
                                         (np.float64, 1024)])
def test_block_ranges_match_full_decode(dtype, block):
    w = np.dtype(dtype).itemsize
    tile_vals = max(8, 32768 // (block * w)) * block
    n = 3 * tile_vals + 777
    x = inputs.sinusoid_1d(n, seed=11).astype(dtype)
    x[tile_vals + 5] = np.nan  # a raw block in the middle
    eb = inputs.rel_to_abs(x[np.isfinite(x)], 1e-3)
    s = oracle.compress(x, eb, block)
    buf = torch.from_numpy(s).cuda()
    h = szx.header(buf)
    full = oracle.decompress(s)
    u = np.uint32 if dtype == np.float32 else np.uint64
    nb = -(-n // block)
    G = tile_vals // block
    ranges = [(0, 1), (5, 70), (G - 1, 2), (G, G), (nb - 1, 1), (0, nb), (100 % nb, nb - 100 % nb), (2, nb - 4)]
    for first, count in ranges:
        count = min(count, nb - first)
        got = szx.decompress_range(buf, first, count, h=h).cpu().numpy()
        lo, hi = first * block, min(n, (first + count) * block)
        assert np.array_equal(got.view(u), full[lo:hi].view(u)), f"range ({first}, {count})"


def test_invalid_ranges_are_rejected():
    x = inputs.sinusoid_1d(10_000, seed=1)
    buf = szx.compress(torch.from_numpy(x).cuda(), 1e-3)
    h = szx.header(buf)
    nb = -(-10_000 // 128)
    for first, count in [(0, 0), (nb, 1), (nb - 1, 2)]:
        with pytest.raises(szx.SzxError):
            szx.decompress_range(buf, first, count, h=h)


@pytest.mark.gpu
def test_long_range_with_status_matches_full_decode():
    # a range of at least 256 tiles with a status word: the status is cleared
    # by a kernel and the decoder launched as its programmatic dependent
    block = 128
    n = 300 * 64 * block + 333
    x = np.cumsum(np.random.default_rng(4).normal(size=n)).astype(np.float32)
    eb = inputs.rel_to_abs(x, 1e-3)
    s = oracle.compress(x, eb, block)
    full = oracle.decompress(s)
    buf = torch.from_numpy(s).cuda()
    h = szx.header(buf)
    nb = -(-n // block)
    first, count = 70, nb - 70 - 5
    st = torch.full((1,), 99, dtype=torch.int32, device="cuda")
    got = szx.decompress_range(buf, first, count, h=h, status=st)
    torch.cuda.synchronize()
    assert int(st.item()) == 0
    lo, hi = first * block, min(n, (first + count) * block)
    assert np.array_equal(got.cpu().numpy().view(np.uint32), full[lo:hi].view(np.uint32))
