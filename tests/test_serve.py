"""The serving loop (szx_server_*): every result is the same alone and in
the mix (streams byte-identical, decodes bit-exact) and the same as the CPU
oracle's (the complex f64 state vectors included), admission waits for pool
memory, a request that can never fit is reported, and the pool accounting
returns to empty."""
import numpy as np
import pytest

import oracle
from exact import exact_abs_diff_le

torch = pytest.importorskip("torch")
import paper_2201_13020_b300 as szx  # noqa: E402
from paper_2201_13020_b300 import inputs, serve  # noqa: E402

pytestmark = pytest.mark.gpu


def _requests(seed, count, lo, hi, p_decompress=0.4, rate=2000.0):
    rng = np.random.default_rng(seed)
    t = 0.0
    reqs, comp = [], []
    for i in range(count):
        t += rng.exponential(1.0 / rate)
        if comp and rng.random() < p_decompress:
            reqs.append(serve.Request("decompress", t, source=int(rng.choice(comp)), keep_output=True))
            continue
        nbytes = int(np.exp(rng.uniform(np.log(lo), np.log(hi))))
        if rng.random() < 0.5:
            x = inputs.state_vector(max(1, nbytes // 16), seed=i, device="cuda")
        else:
            x = inputs.sinusoid_1d_torch(max(128, nbytes // 4), seed=i, device="cuda")
        rel = float(rng.choice([1e-2, 1e-3, 1e-4]))
        reqs.append(serve.Request("compress", t, x=x, eb=inputs.rel_to_abs(x, rel), block=128))
        comp.append(len(reqs) - 1)
    return reqs


def test_mixed_requests_match_each_request_alone():
    reqs = _requests(5, 60, 64 << 10, 8 << 20, rate=20000.0)
    server = serve.Server(2 << 30, slots=6)
    server.run(reqs)
    torch.cuda.synchronize()
    assert server.max_in_flight > 1  # work overlapped on the device
    for i, r in enumerate(reqs):
        assert r.status == 0, f"request {i}: status {r.status}"
        assert r.admit_s >= r.arrival - 1e-9 and r.done_s >= r.admit_s
        if r.kind == "compress":
            alone = szx.compress(r.x, r.eb, r.block)
            served = server.view(r.offset, r.nbytes)
            assert torch.equal(served, alone), f"request {i}: stream differs"
            # the oracle on the same values: the served stream byte for byte
            ref = oracle.compress(r.x.cpu().numpy(), r.eb, r.block)
            assert np.array_equal(served.cpu().numpy(), ref), f"request {i}: stream differs from the oracle"
        else:
            src = reqs[r.source]
            alone = szx.decompress(szx.compress(src.x, src.eb, src.block))
            got = server.output(r)
            it = torch.int32 if alone.dtype == torch.float32 else torch.int64
            assert torch.equal(got.view(it), alone.view(it)), f"request {i}: decode differs"
            xs = src.x.cpu().numpy()
            ref = oracle.decompress(oracle.compress(xs, src.eb, src.block))
            ui = np.uint32 if xs.dtype == np.float32 else np.uint64
            assert np.array_equal(got.cpu().numpy().view(ui), ref.view(ui)), \
                f"request {i}: decode differs from the oracle"
            e = oracle.error_bound(src.eb, oracle.F32 if xs.dtype == np.float32 else oracle.F64)
            assert exact_abs_diff_le(xs, got.cpu().numpy(), e).all(), f"request {i}: bound"
    kinds = {reqs[r.source].x.dtype for r in reqs if r.kind == "decompress"}
    assert kinds == {torch.float32, torch.float64}  # state vectors and f32 fields were both decoded
    # give everything back: the pool is empty again
    for r in reqs:
        if r.kind == "compress" or r.keep_output:
            server.release(r.offset, r.nbytes)
    assert server.free_bytes() == server.pool.numel()


def test_small_pool_makes_admission_wait():
    # four compressions, then twenty decompressions of their streams whose
    # outputs are freed on completion: the pool holds the four compressions'
    # bounds plus room for about two outputs, so the decompressions are
    # admitted as memory frees up, not as slots do
    comp = _requests(6, 4, 1 << 20, 3 << 20, p_decompress=0.0, rate=1e6)
    reqs = list(comp)
    rng = np.random.default_rng(7)
    t = max(r.arrival for r in comp)
    for j in range(20):
        reqs.append(serve.Request("decompress", t, source=int(rng.integers(4))))
    code = [szx.SZX_F32 if r.x.dtype == torch.float32 else szx.SZX_F64 for r in comp]
    bounds = sum(-(-szx.compress_bound(r.x.numel(), c, 128) // 256) * 256 for r, c in zip(comp, code))
    out_max = max(r.x.numel() * r.x.element_size() for r in comp)
    server = serve.Server(bounds + 2 * out_max + (1 << 16), slots=8)
    server.run(reqs)
    torch.cuda.synchronize()
    assert all(r.status == 0 for r in reqs)
    assert 1 < server.max_in_flight < 8  # memory, not slots, limited admission
    for r in comp:
        assert torch.equal(server.view(r.offset, r.nbytes), szx.compress(r.x, r.eb, r.block))


def test_request_that_never_fits_is_reported():
    x_big = inputs.sinusoid_1d_torch(1 << 20, seed=1, device="cuda")
    x_small = inputs.sinusoid_1d_torch(1 << 12, seed=2, device="cuda")
    reqs = [serve.Request("compress", 0.0, x=x_small, eb=1e-3),
            serve.Request("compress", 0.0, x=x_big, eb=1e-3),
            serve.Request("decompress", 0.0, source=0, keep_output=True),
            serve.Request("decompress", 0.0, source=3)]  # names itself: rejected
    server = serve.Server(1 << 20, slots=2)
    with pytest.raises(MemoryError):
        server.run(reqs)
    assert [r.status for r in reqs] == [0, 4, 0, 1]
    alone = szx.decompress(szx.compress(x_small, 1e-3))
    assert torch.equal(server.output(reqs[2]).view(torch.int32), alone.view(torch.int32))
