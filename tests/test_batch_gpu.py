"""Batched compression / decompression (many fields, one persistent launch per
(dtype, block) group) through the C ABI: every stream byte-identical to the
single-field call and to the oracle, every decode bit-identical."""
import ctypes

import numpy as np
import pytest

import oracle

torch = pytest.importorskip("torch")
import paper_2201_13020_b300 as szx  # noqa: E402
from paper_2201_13020_b300 import _lib, inputs  # noqa: E402


def _fields():
    """Mixed dtypes, blocks and sizes (ragged ends, single block, several tiles)."""
    rng = np.random.default_rng(21)
    out = []
    out.append((inputs.sinusoid_1d((1 << 16) + 77, seed=3), 1e-3, 128))
    g = inputs.grf_3d((40, 37, 29), -5.0 / 3.0, 4).numpy()
    out.append((g.reshape(-1), 1e-3, 128))
    g64 = inputs.grf_3d((30, 31, 33), -11.0 / 3.0, 5, dtype=torch.float64).numpy()
    out.append((g64.reshape(-1), 1e-4, 256))
    out.append((rng.normal(size=5000).astype(np.float32), 1e-2, 64))
    out.append((np.cumsum(rng.normal(size=100_003)).astype(np.float64), 1e-3, 128))
    out.append((np.array([1.5], dtype=np.float32), 1e-3, 128))
    out.append((rng.normal(size=50_000).astype(np.float32), 1e-3, 1024))
    out.append((np.cumsum(rng.normal(size=70_001)).astype(np.float64), 1e-4, 1024))
    out.append((inputs.sinusoid_1d(200_000, seed=9), 1e-4, 128))  # same group as field 0
    # a single value has no range: its bound is absolute
    return [(x, inputs.rel_to_abs(x, rel) if x.size > 1 else rel, b) for x, rel, b in out]


@pytest.mark.gpu
def test_batch_compress_and_decompress_match_single_and_oracle():
    fields = _fields()
    xs = [torch.from_numpy(np.ascontiguousarray(x)).cuda() for x, _, _ in fields]
    batch, outs, results = szx.batch_compress(xs, [eb for _, eb, _ in fields], [b for _, _, b in fields])
    assert len(batch.groups()) == 6
    batch.run()
    torch.cuda.synchronize()
    res = results.cpu().numpy().reshape(-1, 2)
    streams = []
    for i, ((x, eb, b), xt) in enumerate(zip(fields, xs)):
        assert res[i, 1] == 0, f"field {i}: status {res[i, 1]}"
        got = outs[i][:int(res[i, 0])].cpu().numpy()
        single = szx.compress(xt, eb, b).cpu().numpy()
        assert np.array_equal(got, single), f"field {i}: batch stream differs from the single-field call"
        ref = oracle.compress(x, eb, b)
        assert np.array_equal(got, ref), f"field {i}: batch stream differs from the oracle"
        streams.append(ref)
    # batched decompression of the same streams
    bufs = [torch.from_numpy(s).cuda() for s in streams]
    headers = [szx.header(bb) for bb in bufs]
    dbatch, ys, statuses = szx.batch_decompress(bufs, headers)
    dbatch.run()
    torch.cuda.synchronize()
    assert statuses.cpu().tolist() == [0] * len(fields)
    for i, (s, y) in enumerate(zip(streams, ys)):
        ref = oracle.decompress(s)
        u = np.uint32 if ref.dtype == np.float32 else np.uint64
        assert np.array_equal(y.cpu().numpy().view(u), ref.view(u)), f"field {i}: decode differs"


@pytest.mark.gpu
def test_batch_graph_capture_replays_identically():
    fields = _fields()[:5]
    xs = [torch.from_numpy(np.ascontiguousarray(x)).cuda() for x, _, _ in fields]
    batch, outs, results = szx.batch_compress(xs, [eb for _, eb, _ in fields], [b for _, _, b in fields])
    batch.run()  # warm (kernel attributes set, modules loaded)
    torch.cuda.synchronize()
    first = [o.clone() for o in outs]
    s = torch.cuda.Stream()
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph, stream=s):
        batch.run(stream=s)
    for _ in range(2):
        for o in outs:
            o.zero_()
        graph.replay()
        torch.cuda.synchronize()
        for i, (a, b_) in enumerate(zip(first, outs)):
            n = int(results[2 * i].item())
            assert torch.equal(a[:n], b_[:n]), f"field {i} differs after graph replay"
            assert int(results[2 * i + 1].item()) == 0


@pytest.mark.gpu
def test_batch_autotune_keeps_streams():
    fields = _fields()[:4]
    xs = [torch.from_numpy(np.ascontiguousarray(x)).cuda() for x, _, _ in fields]
    batch, outs, results = szx.batch_compress(xs, [eb for _, eb, _ in fields], [b for _, _, b in fields])
    choice = batch.autotune()
    assert all(g["ctas_per_sm"] in (1, 2) and g["warps_per_cta"] in (8, 4) and g["tuned_ms"] > 0 for g in choice)
    batch.run()
    torch.cuda.synchronize()
    for i, (x, eb, b) in enumerate(fields):
        n = int(results[2 * i].item())
        assert np.array_equal(outs[i][:n].cpu().numpy(), oracle.compress(x, eb, b))


@pytest.mark.gpu
def test_batch_corrupt_stream_is_flagged_alone():
    fields = _fields()[:3]
    streams = [oracle.compress(x, eb, b) for x, eb, b in fields]
    bufs = [torch.from_numpy(s).cuda() for s in streams]
    headers = [szx.header(bb) for bb in bufs]
    # stream 1: make its second tile-index entry odd (offsets are multiples of 16)
    h = headers[1]
    nb = -(-h.n // h.block)
    w = 4 if h.dtype == szx.SZX_F32 else 8
    off_mu = 64 + ((nb + 7) // 8 + 15) // 16 * 16
    off_index = off_mu + (nb * w + 15) // 16 * 16
    bad = streams[1].copy()
    bad[off_index + 8] ^= 0x01
    bufs[1] = torch.from_numpy(bad).cuda()
    dbatch, ys, statuses = szx.batch_decompress(bufs, headers)
    dbatch.run()
    torch.cuda.synchronize()
    st = statuses.cpu().tolist()
    assert st[1] == 3 and st[0] == 0 and st[2] == 0
    for i in (0, 2):
        ref = oracle.decompress(streams[i])
        u = np.uint32 if ref.dtype == np.float32 else np.uint64
        assert np.array_equal(ys[i].cpu().numpy().view(u), ref.view(u))


def test_batch_plan_argument_checks_on_host():
    # plan creation is host-only: fake aligned device addresses are never touched
    L = _lib.lib()
    F = _lib.SzxField
    ok = F(256, 1000, _lib.SZX_F32, 1e-3, 128, 512, 1 << 20)
    arr = (F * 2)(ok, F(256, 1000, _lib.SZX_F32, 1e-3, 100, 512, 1 << 20))
    plan = ctypes.c_void_p(0)
    assert L.szx_batch_compress_plan(arr, 2, ctypes.byref(plan)) == 1 and not plan.value
    arr = (F * 1)(F(256, 1000, _lib.SZX_F32, 1e-3, 128, 512, 16))
    assert L.szx_batch_compress_plan(arr, 1, ctypes.byref(plan)) == 2
    arr = (F * 1)(F(257, 1000, _lib.SZX_F32, 1e-3, 128, 512, 1 << 20))
    assert L.szx_batch_compress_plan(arr, 1, ctypes.byref(plan)) == 1
    arr = (F * 2)(ok, F(256, 70_000, _lib.SZX_F64, 1e-3, 256, 512, 1 << 22))
    assert L.szx_batch_compress_plan(arr, 2, ctypes.byref(plan)) == 0 and plan.value
    assert L.szx_batch_workspace_bytes(plan) > 0
    groups = (ctypes.c_int * 4)()
    assert L.szx_batch_groups(plan, groups, 4) == 2
    L.szx_batch_destroy(plan)


@pytest.mark.gpu
def test_block_zero_picks_a_candidate_and_round_trips():
    from paper_2201_13020_b300 import metrics
    x = torch.from_numpy(inputs.sinusoid_1d(1 << 20, seed=5)).cuda()
    eb = inputs.rel_to_abs(x, 1e-3)
    pick, ratios = metrics.choose_block(x, eb)
    assert pick in (64, 128, 256) and ratios[pick] == max(ratios.values())
    s = szx.compress(x, eb, 0)
    h = szx.header(s)
    assert h.block == pick
    assert np.array_equal(s.cpu().numpy(), oracle.compress(x.cpu().numpy(), eb, pick))


@pytest.mark.gpu
def test_batch_block_zero_is_chosen_by_the_tuner():
    # block 0: the tuner picks b among 64, 128 and 256 per dtype group; every
    # stream is then the oracle's at the chosen b
    fields = _fields()[:5]
    xs = [torch.from_numpy(np.ascontiguousarray(x)).cuda() for x, _, _ in fields]
    ebs = [eb for _, eb, _ in fields]
    batch, outs, results = szx.batch_compress(xs, ebs, 0)
    groups = batch.autotune()
    assert all(g["auto_block"] == 1 and g["block"] in szx.AUTO_BLOCKS for g in groups)
    assert sorted(g["dtype"] for g in groups) == [0, 1]
    batch.run()
    torch.cuda.synchronize()
    chosen = {g["dtype"]: g["block"] for g in groups}
    for i, (x, eb, _) in enumerate(fields):
        b = chosen[0 if x.dtype == np.float32 else 1]
        n = int(results[2 * i].item())
        assert int(results[2 * i + 1].item()) == 0
        assert np.array_equal(outs[i][:n].cpu().numpy(), oracle.compress(x, eb, b)), f"field {i} (b = {b})"


def _shape_fields(dtype, block):
    """Three fields of one (dtype, block): several tiles with a ragged end, a
    partial single tile, one partial block."""
    rng = np.random.default_rng(block + (dtype == np.float64))
    tile = max(8, 32768 // (block * np.dtype(dtype).itemsize)) * block
    xs = [np.cumsum(rng.normal(size=3 * tile + block // 2 + 3)).astype(dtype),
          (np.sin(np.linspace(0, 30, tile // 2 + 1)) + 1e-3 * rng.normal(size=tile // 2 + 1)).astype(dtype),
          rng.normal(size=max(1, block // 3)).astype(dtype)]
    xs[0][tile:tile + block] = xs[0][tile]  # a constant block
    return [(x, inputs.rel_to_abs(x, 1e-3)) for x in xs]


SHAPES = [(dt, b, nw) for dt in (np.float32, np.float64) for b in (32, 64, 128, 256, 512, 1024) for nw in (8, 4)
          if nw == 8 or (b >= 64 if dt == np.float32 else b <= 512)]


@pytest.mark.gpu
@pytest.mark.parametrize("dtype,block,nw", SHAPES)
def test_every_kernel_shape_matches_the_oracle(dtype, block, nw):
    """Each instance of the kernels (consumer / decoding warps per CTA, values
    per lane) writes the oracle's streams byte for byte and decodes them bit
    for bit, at 2 and at 1 CTA per SM."""
    fields = _shape_fields(dtype, block)
    xs = [torch.from_numpy(x).cuda() for x, _ in fields]
    refs = [oracle.compress(x, eb, block) for x, eb in fields]
    batch, outs, results = szx.batch_compress(xs, [eb for _, eb in fields], block)
    bufs = [torch.from_numpy(r).cuda() for r in refs]
    dbatch, ys, statuses = szx.batch_decompress(bufs, [szx.header(bb) for bb in bufs])
    for ctas in (2, 1):
        batch.set_group(0, ctas, nw)
        dbatch.set_group(0, ctas, nw)
        g = batch.groups()[0]
        assert (g["warps_per_cta"], g["threads_per_cta"], g["ctas_per_sm"]) == (nw, 32 * nw + 64, ctas)
        for o in outs:
            o.fill_(0xA5)
        batch.run()
        dbatch.run()
        torch.cuda.synchronize()
        res = results.cpu().numpy().reshape(-1, 2)
        assert statuses.cpu().tolist() == [0, 0, 0]
        for i, ((x, eb), ref) in enumerate(zip(fields, refs)):
            assert res[i, 1] == 0 and res[i, 0] == len(ref), (i, res[i])
            assert np.array_equal(outs[i][:len(ref)].cpu().numpy(), ref), f"field {i}: stream ({ctas} CTAs/SM)"
            u = np.uint32 if dtype == np.float32 else np.uint64
            y_ref = oracle.decompress(ref)
            assert np.array_equal(ys[i].cpu().numpy().view(u), y_ref.view(u)), f"field {i}: decode ({ctas} CTAs/SM)"


def test_batch_group_shapes_on_host():
    # plan creation and shape calls are host-only: fake aligned device
    # addresses are never touched
    L = _lib.lib()
    F = _lib.SzxField
    arr = (F * 3)(F(256, 70_000, _lib.SZX_F32, 1e-3, 128, 512, 1 << 22),
                  F(256, 70_000, _lib.SZX_F32, 1e-3, 32, 512, 1 << 22),
                  F(256, 70_000, _lib.SZX_F64, 1e-3, 1024, 512, 1 << 22))
    plan = ctypes.c_void_p(0)
    assert L.szx_batch_compress_plan(arr, 3, ctypes.byref(plan)) == 0
    assert L.szx_batch_groups(plan, None, 0) == 3
    info = {}
    for i in range(3):
        g = _lib.SzxBatchGroup()
        assert L.szx_batch_group_info(plan, i, ctypes.byref(g)) == 0
        info[(g.dtype, g.block)] = (i, g)
    i128, g128 = info[(0, 128)]
    assert (g128.warps_per_cta, g128.values_per_lane, g128.blocks_per_warp, g128.threads_per_cta) == (8, 32, 8, 320)
    assert L.szx_batch_set_group(plan, i128, 2, 4) == 0
    assert L.szx_batch_group_info(plan, i128, ctypes.byref(g128)) == 0
    assert (g128.warps_per_cta, g128.values_per_lane, g128.blocks_per_warp, g128.threads_per_cta) == (4, 64, 16, 192)
    # no 4-warp instance for f32 with b = 32, nor f64 with b = 1024; no 3 CTAs per SM
    assert L.szx_batch_set_group(plan, info[(0, 32)][0], 0, 4) == 1
    assert L.szx_batch_set_group(plan, info[(1, 1024)][0], 0, 4) == 1
    assert L.szx_batch_set_group(plan, i128, 3, 8) == 1
    assert L.szx_batch_group_info(plan, 3, ctypes.byref(g128)) == 1
    L.szx_batch_destroy(plan)
    # block 0: planned at 128, the capacity must hold the largest candidate stream
    need = max(L.szx_stream_max_bytes(10_000, _lib.SZX_F32, b) for b in (64, 128, 256))
    arr = (F * 1)(F(256, 10_000, _lib.SZX_F32, 1e-3, 0, 512, need - 16))
    assert L.szx_batch_compress_plan(arr, 1, ctypes.byref(plan)) == 2
    arr = (F * 1)(F(256, 10_000, _lib.SZX_F32, 1e-3, 0, 512, need))
    assert L.szx_batch_compress_plan(arr, 1, ctypes.byref(plan)) == 0
    g = _lib.SzxBatchGroup()
    assert L.szx_batch_group_info(plan, 0, ctypes.byref(g)) == 0 and g.auto_block == 1 and g.block == 128
    L.szx_batch_destroy(plan)
