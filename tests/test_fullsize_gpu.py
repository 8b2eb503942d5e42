"""Parity at the full 512^3 f32 size, in the launch configuration bench.py times.

The oracle cannot compress 512 MiB in test time, but every tile of the stream
is independent: tile t's record, mu values and state bits must equal what the
oracle writes for the tile's slice of the input compressed alone.  Sampled
tiles are checked that way; the whole stream is checked for its byte-count
formula, and |x - x'| <= e is checked on every value on the device.
"""
import numpy as np
import pytest

import oracle
import szx_stream as ss
from exact import exact_abs_diff_le

torch = pytest.importorskip("torch")
import paper_2201_13020_b300 as szx  # noqa: E402
from paper_2201_13020_b300 import inputs  # noqa: E402

pytestmark = pytest.mark.gpu


def tile_slice_parity(x_host, stream, tile, block, w, eb):
    n = x_host.size
    G = max(8, 32768 // (block * w))
    nb = -(-n // block)
    ntiles = -(-nb // G)
    off_state = 64
    off_mu = off_state + ss.pad16(-(-nb // 8))
    off_index = off_mu + ss.pad16(nb * w)
    off_rec = off_index + ss.pad16(8 * (ntiles + 1))
    idx = stream[off_index:off_index + 8 * (ntiles + 1)].view(np.uint64)
    v0, v1 = tile * G * block, min(n, (tile + 1) * G * block)
    ref = oracle.compress(x_host[v0:v1], eb, block)
    rst = ss.parse(ref)
    rec_ref = ref[rst.off_rec:]
    rec_gpu = stream[off_rec + int(idx[tile]):off_rec + int(idx[tile + 1])]
    assert np.array_equal(rec_ref, rec_gpu), f"tile {tile} record differs"
    k0, k1 = tile * G, min(nb, tile * G + G)
    assert np.array_equal(ref[rst.off_mu:rst.off_mu + (k1 - k0) * w], stream[off_mu + k0 * w:off_mu + k1 * w])
    assert np.array_equal(ref[rst.off_state:rst.off_state + (k1 - k0 + 7) // 8],
                          stream[off_state + k0 // 8:off_state + (k0 // 8) + (k1 - k0 + 7) // 8])
    return ref


@pytest.mark.parametrize("variant,rel", [("grf", 1e-3), ("grf", 1e-2), ("grf", 1e-4), ("lognormal", 1e-3)])
def test_512cubed_f32_sampled_tiles(variant, rel):
    torch.cuda.empty_cache()
    g = inputs.grf_3d((512, 512, 512), -5.0 / 3.0, seed=2, device="cuda")
    if variant == "lognormal":
        g = inputs.lognormal(g)
    g = inputs.zero_slabs(g, 0.25, 32, seed=2)
    x = g.reshape(-1)
    eb = inputs.rel_to_abs(x, rel)
    s = szx.compress(x, eb)
    y = szx.decompress(s)
    # every value, exactly: f32 differences are exact in f64 unless the
    # exponents differ by > 29, which keeps |x - y| far from e here
    e = oracle.error_bound(eb, oracle.F32)
    d = (x.double() - y.double()).abs()
    # f64 differences of f32 values are exact or within 2^-53 relative, so only
    # values within 2^-20 of the bound need the exact rational check
    near = torch.nonzero(d > e * (1 - 2 ** -20)).flatten()
    assert float(d.max()) <= e * (1 + 2 ** -20)
    if near.numel():
        xs, ys = x[near].cpu().numpy(), y[near].cpu().numpy()
        assert exact_abs_diff_le(xs, ys, e).all()
    stream = s.cpu().numpy()
    x_host = x.cpu().numpy()
    n = x_host.size
    ntiles = -(-(n // 128) // 64)
    rng = np.random.default_rng(0)
    tiles = sorted(set([0, 1, ntiles - 1] + rng.choice(ntiles, size=24, replace=False).tolist()))
    y_host = y.cpu().numpy()
    for t in tiles:
        ref = tile_slice_parity(x_host, stream, t, 128, 4, eb)
        yr = oracle.decompress(ref)
        v0 = t * 64 * 128
        assert np.array_equal(yr.view(np.uint32), y_host[v0:v0 + yr.size].view(np.uint32))
    # header and byte-count formula of the whole stream
    h = np.frombuffer(stream[:64].tobytes(), dtype=np.uint64)
    assert int(h[7]) == stream.size
    del g, x, y, s, d
    torch.cuda.empty_cache()


@pytest.mark.parametrize("rel,block", [(1e-4, 128), (1e-6, 128), (1e-4, 256), (1e-6, 256)])
def test_384cubed_f64_sampled_tiles(rel, block):
    """The f64 field: 384^3, spectrum |k|^-11/3 plus 1e-6 white noise."""
    torch.cuda.empty_cache()
    g = inputs.grf_3d((384, 384, 384), -11.0 / 3.0, seed=3, device="cuda", dtype=torch.float64)
    gen = torch.Generator(device="cuda")
    gen.manual_seed(33)
    x = (g + 1e-6 * torch.randn(g.shape, generator=gen, device="cuda", dtype=torch.float64)).reshape(-1)
    del g
    eb = inputs.rel_to_abs(x, rel)
    s = szx.compress(x, eb, block)
    y = szx.decompress(s)
    e = oracle.error_bound(eb, oracle.F64)
    d = (x - y).abs()
    assert float(d.max()) <= e * (1 + 2 ** -40)
    near = torch.nonzero(d > e * (1 - 2 ** -40)).flatten()
    if near.numel():
        assert exact_abs_diff_le(x[near].cpu().numpy(), y[near].cpu().numpy(), e).all()
    stream = s.cpu().numpy()
    x_host = x.cpu().numpy()
    n = x_host.size
    G = max(8, 32768 // (block * 8))
    ntiles = -(-(-(-n // block)) // G)
    rng = np.random.default_rng(1)
    tiles = sorted(set([0, ntiles - 1] + rng.choice(ntiles, size=12, replace=False).tolist()))
    y_host = y.cpu().numpy()
    for t in tiles:
        ref = tile_slice_parity(x_host, stream, t, block, 8, eb)
        yr = oracle.decompress(ref)
        v0 = t * G * block
        assert np.array_equal(yr.view(np.uint64), y_host[v0:v0 + yr.size].view(np.uint64))
    h = np.frombuffer(stream[:64].tobytes(), dtype=np.uint64)
    assert int(h[7]) == stream.size
    del x, y, s, d
    torch.cuda.empty_cache()


def test_record_sizes_change_tile_to_tile():
    """Each tile of 8192 values gets its own noise level (1e-6 to 1 against a bound of
    1e-5), so nearly constant tiles and nearly incompressible ones follow each other in
    random order: every CTA handles dozens of tiles whose records, of very different
    sizes, pass through its shared-memory record buffer and wrap around its end."""
    torch.cuda.empty_cache()
    n, per_tile = 1 << 26, 64 * 128
    ntiles = n // per_tile
    gen = torch.Generator(device="cuda")
    gen.manual_seed(41)
    level = 10.0 ** (-6.0 * torch.rand(ntiles, generator=gen, device="cuda"))
    x = torch.linspace(0.0, 1.0, n, device="cuda") + \
        level.repeat_interleave(per_tile) * torch.randn(n, generator=gen, device="cuda")
    eb = 1e-5
    s = szx.compress(x, eb)
    y = szx.decompress(s)
    e = oracle.error_bound(eb, oracle.F32)
    d = (x.double() - y.double()).abs()
    assert float(d.max()) <= e * (1 + 2 ** -20)
    near = torch.nonzero(d > e * (1 - 2 ** -20)).flatten()
    if near.numel():
        assert exact_abs_diff_le(x[near].cpu().numpy(), y[near].cpu().numpy(), e).all()
    stream = s.cpu().numpy()
    nb = n // 128
    off_index = 64 + ss.pad16(-(-nb // 8)) + ss.pad16(nb * 4)
    idx = stream[off_index:off_index + 8 * (ntiles + 1)].view(np.uint64).astype(np.int64)
    sizes = np.diff(idx)
    assert sizes.min() < 2048 and sizes.max() > 24576, (sizes.min(), sizes.max())
    x_host, y_host = x.cpu().numpy(), y.cpu().numpy()
    rng = np.random.default_rng(5)
    tiles = sorted(set([0, ntiles - 1, int(sizes.argmax()), int(sizes.argmin())] +
                       rng.choice(ntiles, size=20, replace=False).tolist()))
    for t in tiles:
        ref = tile_slice_parity(x_host, stream, t, 128, 4, eb)
        yr = oracle.decompress(ref)
        v0 = t * per_tile
        assert np.array_equal(yr.view(np.uint32), y_host[v0:v0 + yr.size].view(np.uint32))
    del x, y, s, d
    torch.cuda.empty_cache()


def test_raw_tiles_of_the_largest_record_size():
    """Half the tiles, chosen at random, hold a NaN in every block: each of their blocks is
    stored raw, so their records have the largest size a tile can have.  The decoder's
    shared-memory record ring then holds only two of them, and wraps often.  The other tiles
    are a smooth random walk.  2^24 values: every CTA handles several tiles of each kind."""
    torch.cuda.empty_cache()
    n, b, per_tile = 1 << 24, 128, 64 * 128
    ntiles = n // per_tile
    gen = torch.Generator(device="cuda")
    gen.manual_seed(43)
    x = torch.cumsum(torch.randn(n, generator=gen, device="cuda"), 0) * 1e-3
    raw_tiles = torch.rand(ntiles, generator=gen, device="cuda") < 0.5
    nan_blocks = raw_tiles[torch.arange(n // b, device="cuda") // 64]
    xv = x.view(-1, b)
    xv[nan_blocks, 5] = float("nan")
    eb = 1e-3
    s = szx.compress(x, eb)
    y = szx.decompress(s)
    yv = y.view(-1, b)
    # raw blocks come back bit for bit; the others within the bound
    assert torch.equal(xv[nan_blocks].view(torch.int32), yv[nan_blocks].view(torch.int32))
    e = oracle.error_bound(eb, oracle.F32)
    d = (xv[~nan_blocks].double() - yv[~nan_blocks].double()).abs()
    assert float(d.max()) <= e * (1 + 2 ** -20)
    stream = s.cpu().numpy()
    nb = n // b
    off_index = 64 + ss.pad16(-(-nb // 8)) + ss.pad16(nb * 4)
    idx = stream[off_index:off_index + 8 * (ntiles + 1)].view(np.uint64).astype(np.int64)
    sizes = np.diff(idx)
    largest = ss.pad16(64 * (b // 4 + 1) + 64 * b * 4)
    raw_host = raw_tiles.cpu().numpy()
    assert (sizes[raw_host] == largest).all()
    assert (sizes[~raw_host] < largest // 2).all()
    x_host, y_host = x.cpu().numpy(), y.cpu().numpy()
    rng = np.random.default_rng(6)
    tiles = sorted(set([0, ntiles - 1] + rng.choice(ntiles, size=16, replace=False).tolist()))
    for t in tiles:
        ref = tile_slice_parity(x_host, stream, t, b, 4, eb)
        yr = oracle.decompress(ref)
        v0 = t * per_tile
        assert np.array_equal(yr.view(np.uint32), y_host[v0:v0 + yr.size].view(np.uint32))
    del x, y, s, d
    torch.cuda.empty_cache()
