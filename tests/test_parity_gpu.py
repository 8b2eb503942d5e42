"""Parity of the CUDA path with the CPU oracle, through the C ABI.

Streams must be byte-identical and decoded arrays bit-identical (integer and
byte work: the bar is exact), and |x - x'| <= e must hold exactly on every
value.  Sizes span several tiles with ragged tails; the edge cases cover the
degenerate blocks of the method.  The oracle only ever sees the same seeded
inputs the GPU sees; no expected value comes from the GPU.
"""
import numpy as np
import pytest

import oracle
import szx_stream as ss
from exact import exact_abs_diff_le
from cases import VALUE_RELS, bound_for, inputs_tile, value_distribution_cases

torch = pytest.importorskip("torch")
import paper_2201_13020_b300 as szx  # noqa: E402
from paper_2201_13020_b300 import inputs  # noqa: E402

pytestmark = pytest.mark.gpu


def gpu_compress(x, eb, block=128):
    t = torch.from_numpy(np.ascontiguousarray(x)).cuda()
    return szx.compress(t, eb, block).cpu().numpy()


def gpu_decompress(stream):
    buf = torch.from_numpy(np.ascontiguousarray(stream)).cuda()
    return szx.decompress(buf).cpu().numpy()


def assert_parity(x, eb, block=128):
    ref = oracle.compress(x, eb, block)
    got = gpu_compress(x, eb, block)
    if len(ref) != len(got) or not np.array_equal(ref, got):
        diff = np.flatnonzero(ref[:min(len(ref), len(got))] != got[:min(len(ref), len(got))])
        raise AssertionError(f"stream mismatch: len ref {len(ref)} gpu {len(got)}, first diff at "
                             f"{diff[:8]} (of {diff.size})")
    y_ref = oracle.decompress(ref)
    y_gpu = gpu_decompress(got)
    uint = np.uint32 if x.dtype == np.float32 else np.uint64
    assert np.array_equal(y_ref.view(uint), y_gpu.view(uint)), "decode mismatch"
    return ref, y_gpu


def _e(eb, dtype):
    return oracle.error_bound(eb, oracle.F32 if dtype == np.float32 else oracle.F64)


# ---------------------------------------------------------------------------


def test_worked_example_fig4():
    x = np.array([0x3DFCB924, 0x3DFCED91, 0x3DF80347, 0xBDFCED91], dtype=np.uint32).view(np.float32)
    s, y = assert_parity(x, 1e-3, 128)
    assert len(s) == 160


def test_config_1d_sinusoid_2p20():
    """The 2^20-value 1-D f32 sinusoid field with 10% constant blocks, e = 1e-3 x range."""
    x = inputs.sinusoid_1d(1 << 20, seed=1)
    eb = inputs.rel_to_abs(x, 1e-3)
    s, y = assert_parity(x, eb, 128)
    h = np.frombuffer(s[:64].tobytes(), dtype=np.uint64)
    nb = (1 << 20) // 128
    assert nb - h[4] >= 0.10 * nb * 0.99  # at least the planted constant blocks
    assert exact_abs_diff_le(x, y, _e(eb, np.float32)).all()


SIZES = [1, 3, 31, 32, 33, 127, 128, 129, 1000, 8191, 8192, 8193, 8192 * 3 + 77, 70001]


@pytest.mark.parametrize("dtype", [np.float32, np.float64])
@pytest.mark.parametrize("block", [32, 64, 128, 256, 512, 1024])
def test_sizes_and_blocks(dtype, block):
    rng = np.random.default_rng(block * 7 + (dtype == np.float64))
    for n in SIZES + [3 * inputs_tile(block, dtype) + 5]:
        x = np.cumsum(rng.normal(size=n)).astype(dtype)
        if n > 300:
            x[100:300] = x[100]  # constant run
        eb = max(1e-3 * float(x.max() - x.min()), 1e-6)
        assert_parity(x, eb, block)


@pytest.mark.parametrize("dtype", [np.float32, np.float64])
def test_value_distributions(dtype):
    for name, v in value_distribution_cases(dtype).items():
        x = v.astype(dtype)
        for rel in VALUE_RELS:
            try:
                assert_parity(x, bound_for(x, rel), 128)
            except AssertionError as exc:
                raise AssertionError(f"{name} rel={rel}: {exc}") from None


def _pow2_bounds(p, dtype):
    """e = 2^p and its two neighbours in the value's format."""
    e = dtype(2.0 ** p)
    return [float(e), float(np.nextafter(e, dtype(np.inf))), float(np.nextafter(e, dtype(0)))]


@pytest.mark.parametrize("dtype", [np.float32, np.float64])
@pytest.mark.parametrize("block", [32, 128, 1024])
def test_power_of_two_bounds(dtype, block):
    """Bounds e = 2^p, the next value above and the next below, with p spanning
    the data's exponents.  This is where Eq. 4's estimate is tightest (the
    lowest kept bit weighs 2^p(e), up to e itself) and where the kernel's
    block-level proof that the per-value check passes changes its answer:
    the proof compares powers of two against e's significand, which is 1 at
    e = 2^p, 2 - ulp just below it and 1 + ulp just above.  Byte-exact against
    the oracle, at least three tiles with a ragged tail."""
    rng = np.random.default_rng(block * 3 + (dtype == np.float64))
    n = 3 * inputs_tile(block, dtype) + 77
    walk = (np.cumsum(rng.normal(size=n)) * 0.37).astype(dtype)      # |x| up to ~2^6
    offset = (1000.0 + np.cumsum(rng.normal(size=n)) * 1e-3).astype(dtype)  # p(x) = 9, small r
    cases = [("walk", walk, (-16, -8, -4, -1, 0, 3)), ("offset", offset, (-14, -13, -12, -10))]
    for name, x, ps in cases:
        for p in ps:
            for eb in _pow2_bounds(p, dtype):
                try:
                    s, y = assert_parity(x, eb, block)
                except AssertionError as exc:
                    raise AssertionError(f"{name} p={p} eb={eb!r}: {exc}") from None
                assert exact_abs_diff_le(x, y, _e(eb, dtype)).all(), (name, p, eb)


@pytest.mark.parametrize("dtype", [np.float32, np.float64])
def test_nonfinite_and_overflow_blocks_are_raw(dtype):
    rng = np.random.default_rng(8)
    n = 2 * inputs_tile(128, dtype) + 99
    x = rng.normal(size=n).astype(dtype)
    x[[5, 300, 301, 5000, n - 1]] = [np.nan, np.inf, -np.inf, np.nan, np.inf]
    big = np.finfo(dtype).max
    x[1024:1024 + 128] = np.where(np.arange(128) % 2, big, -big)  # mx - mn overflows
    s, y = assert_parity(x, 1e-2, 128)
    st = ss.parse(s) if n < 20000 else None
    if st:
        assert st.nraw >= 4


@pytest.mark.parametrize("dtype", [np.float32, np.float64])
def test_subnormal_bound_escalation(dtype):
    rng = np.random.default_rng(9)
    n = 2 * inputs_tile(128, dtype) + 17
    x = np.cumsum(rng.normal(size=n))
    if dtype == np.float32:
        x, eb = (x * 1e-36).astype(dtype), 1e-42
    else:
        x, eb = (x * 1e-305).astype(dtype), 1e-318
    s, y = assert_parity(x, eb, 128)
    h = np.frombuffer(s[:64].tobytes(), dtype=np.uint64)
    assert h[6] > 0  # escalated blocks


@pytest.mark.parametrize("dtype", [np.float32, np.float64])
def test_bound_extremes(dtype):
    rng = np.random.default_rng(10)
    n = inputs_tile(128, dtype) + 500
    x = (rng.normal(size=n) * 100).astype(dtype)
    tiny = float(np.finfo(dtype).smallest_subnormal)
    _, y = assert_parity(x, tiny, 128)
    uint = np.uint32 if dtype == np.float32 else np.uint64
    assert np.array_equal(y.view(uint), x.view(uint))  # lossless
    s, _ = assert_parity(x, 1e6, 128)  # every block constant
    assert np.frombuffer(s[:64].tobytes(), dtype=np.uint64)[4] == 0
    assert_parity(x, float(np.finfo(dtype).max), 128)


def test_grf_small_fields():
    g = inputs.grf_3d((64, 64, 64), -5.0 / 3.0, seed=3).numpy()
    g = inputs.zero_slabs(g, 0.25, 8, seed=3)
    for rel in (1e-2, 1e-3, 1e-4):
        assert_parity(g.ravel(), inputs.rel_to_abs(g, rel), 128)
    ln = inputs.lognormal(g).astype(np.float32)
    ln = inputs.zero_slabs(ln, 0.25, 8, seed=3)
    assert_parity(ln.ravel(), inputs.rel_to_abs(ln, 1e-3), 128)
    g64 = inputs.grf_3d((48, 48, 48), -11.0 / 3.0, seed=4, dtype=torch.float64).numpy()
    g64 = g64 + 1e-6 * np.random.default_rng(4).normal(size=g64.shape)
    for rel in (1e-4, 1e-6):
        for block in (128, 256):
            assert_parity(g64.ravel(), inputs.rel_to_abs(g64, rel), block)


def test_gpu_decodes_oracle_stream_and_is_deterministic():
    x = inputs.sinusoid_1d(200_000, seed=2)
    eb = inputs.rel_to_abs(x, 1e-4)
    ref = oracle.compress(x, eb)
    y = gpu_decompress(ref)
    assert np.array_equal(y.view(np.uint32), oracle.decompress(ref).view(np.uint32))
    t = torch.from_numpy(x).cuda()
    first = szx.compress(t, eb).cpu().numpy()
    for _ in range(5):
        assert np.array_equal(szx.compress(t, eb).cpu().numpy(), first)


def test_async_forms_match_sync():
    x = inputs.sinusoid_1d(300_000, seed=6)
    eb = inputs.rel_to_abs(x, 1e-3)
    t = torch.from_numpy(x).cuda()
    ref = szx.compress(t, eb).cpu().numpy()
    cap = szx.compress_bound(t.numel(), 0, 128)
    out = torch.empty(cap, dtype=torch.uint8, device="cuda")
    res = torch.zeros(2, dtype=torch.int64, device="cuda")
    szx.compress_async(t, eb, 128, out, res)
    torch.cuda.synchronize()
    nbytes, status = (int(v) for v in res.cpu())
    assert status == 0 and nbytes == len(ref)
    assert np.array_equal(out[:nbytes].cpu().numpy(), ref)
    buf = out[:nbytes]
    h = szx.header(buf)
    y = torch.empty(t.numel(), dtype=torch.float32, device="cuda")
    st = torch.full((1,), 77, dtype=torch.int32, device="cuda")
    szx.decompress_async(buf, h, y, st)
    torch.cuda.synchronize()
    assert int(st.item()) == 0
    assert np.array_equal(y.cpu().numpy().view(np.uint32), oracle.decompress(ref).view(np.uint32))


def test_corrupt_streams_are_rejected_on_device():
    x = inputs.sinusoid_1d(100_000, seed=7)
    t = torch.from_numpy(x).cuda()
    s = szx.compress(t, inputs.rel_to_abs(x, 1e-3)).clone()
    good = s.cpu().numpy()
    # truncated
    with pytest.raises(szx.SzxError) as ei:
        szx.decompress(s[:len(s) - 16].clone())
    assert ei.value.status == 3
    # bad magic
    bad = s.clone()
    bad[0] ^= 1
    with pytest.raises(szx.SzxError) as ei:
        szx.decompress(bad)
    assert ei.value.status == 3
    # corrupt tile index and record bytes: detected on the device or decoded
    st = ss.parse(good)
    rng = np.random.default_rng(0)
    for _ in range(30):
        bad = good.copy()
        pos = int(rng.integers(st.off_index, len(good)))
        bad[pos] ^= np.uint8(1 << int(rng.integers(0, 8)))
        want = oracle.decompress_status(bad)
        try:
            gpu_decompress(bad)
            got = 0
        except szx.SzxError as exc:
            got = exc.status
        assert got == want, (pos, got, want)


def test_invalid_arguments_are_rejected():
    t = torch.zeros(100, device="cuda")
    for eb in (0.0, -1.0, float("nan"), float("inf")):
        with pytest.raises(szx.SzxError) as ei:
            szx.compress(t, eb)
        assert ei.value.status == 1
    with pytest.raises(szx.SzxError):
        szx.compress(t, 1e-3, block=100)
    out = torch.empty(16, dtype=torch.uint8, device="cuda")
    with pytest.raises(szx.SzxError) as ei:
        szx.compress(t, 1e-3, out=out)
    assert ei.value.status == 2
    misaligned = t.view(torch.uint8)[4:].view(torch.float32)[:10]  # 4-byte offset
    with pytest.raises(szx.SzxError) as ei:
        szx.compress(misaligned, 1e-3)
    assert ei.value.status == 1


@pytest.mark.parametrize("dtype", [np.float32, np.float64])
@pytest.mark.parametrize("block", [32, 128, 256, 1024])
def test_mixed_block_kinds_within_a_warp(dtype, block):
    """Constant, non-constant and raw blocks interleaved block by block, so that
    the lanes of one warp take different paths (a warp holds several blocks)."""
    rng = np.random.default_rng(block)
    nb = 3 * max(8, 32768 // (block * np.dtype(dtype).itemsize)) + 3
    x = np.cumsum(rng.normal(size=nb * block)).astype(dtype)
    kinds = rng.integers(0, 4, size=nb)
    for k in range(nb):
        sl = slice(k * block, (k + 1) * block)
        if kinds[k] == 0:
            x[sl] = x[k * block]                      # constant
        elif kinds[k] == 1:
            x[k * block + 3] = np.nan                 # raw
        elif kinds[k] == 2:
            x[sl] = x[k * block] + rng.normal(size=block) * 1e-9  # constant within e
    x = x[: nb * block - block // 3]                  # ragged last block
    finite = x[np.isfinite(x)]
    assert_parity(x, 1e-3 * float(finite.max() - finite.min()), block)
