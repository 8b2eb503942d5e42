"""Single-field calls on one stream, back to back and inside a CUDA graph.

A call of at least 256 tiles clears its scratch or status words with a small
kernel and launches the codec kernel as that kernel's programmatic dependent,
which waits for every earlier kernel on the stream before touching memory; a
smaller one clears with a memset and launches plainly.  These tests put other
kernels right before and after the calls, with no synchronisation in between,
and capture the calls in a graph, on both sides of that size; every stream
must stay byte-identical to the oracle's and every decode bit-identical."""
import numpy as np
import pytest

import oracle

torch = pytest.importorskip("torch")
import paper_2201_13020_b300 as szx  # noqa: E402
from paper_2201_13020_b300 import inputs  # noqa: E402


def _case(dtype, n, seed):
    rng = np.random.default_rng(seed)
    x = np.cumsum(rng.normal(size=n)).astype(dtype)
    return x, inputs.rel_to_abs(x, 1e-3)


@pytest.mark.gpu
@pytest.mark.parametrize("dtype,block,tiles", [(np.float32, 128, 3), (np.float64, 256, 3), (np.float32, 32, 3),
                                               (np.float32, 128, 300), (np.float64, 128, 260)])
def test_back_to_back_calls_see_the_kernels_before_them(dtype, block, tiles):
    # whole tiles and a ragged tail at every block length here
    n = tiles * max(8, 32768 // (block * np.dtype(dtype).itemsize)) * block + 77
    x, eb = _case(dtype, n, 5)
    ref = oracle.compress(x, eb, block)
    xd = torch.from_numpy(x).cuda()
    out = torch.empty(szx.compress_bound(n, szx.SZX_F32 if dtype == np.float32 else szx.SZX_F64, block),
                      dtype=torch.uint8, device="cuda")
    res = torch.zeros(2, dtype=torch.int64, device="cuda")
    st = torch.zeros(1, dtype=torch.int32, device="cuda")
    s0 = szx.compress(xd, eb, block, out=out)
    h = szx.header(s0)
    y = torch.empty_like(xd)
    for k in range(4):
        # a kernel writes the input, the output buffer and the decode target
        # just before the calls; nothing synchronises in between
        src = xd * 1 if k % 2 == 0 else xd.clone()
        out.fill_(0xA5)
        y.fill_(7)
        st.fill_(99)
        szx.compress_async(src, eb, block, out, res)
        szx.decompress_async(out[:len(ref)], h, y, st)
        back = y * 1  # a kernel reads the decode right after
        torch.cuda.synchronize()
        assert res.tolist() == [len(ref), 0]
        assert int(st.item()) == 0
        assert np.array_equal(out[:len(ref)].cpu().numpy(), ref), f"pass {k}: stream differs"
        u = np.uint32 if dtype == np.float32 else np.uint64
        assert np.array_equal(back.cpu().numpy().view(u), oracle.decompress(ref).view(u)), f"pass {k}: decode differs"


@pytest.mark.gpu
@pytest.mark.parametrize("tiles", [5, 300])
def test_single_calls_replay_in_a_cuda_graph(tiles):
    block = 128
    n = tiles * 64 * block + 301
    x, eb = _case(np.float32, n, 9)
    ref = oracle.compress(x, eb, block)
    dref = oracle.decompress(ref)
    xd = torch.from_numpy(x).cuda()
    out = torch.empty(szx.compress_bound(n, szx.SZX_F32, block), dtype=torch.uint8, device="cuda")
    res = torch.zeros(2, dtype=torch.int64, device="cuda")
    st = torch.zeros(1, dtype=torch.int32, device="cuda")
    y = torch.empty_like(xd)
    part = torch.empty(40 * block, dtype=torch.float32, device="cuda")
    pst = torch.zeros(1, dtype=torch.int32, device="cuda")
    h = szx.header(szx.compress(xd, eb, block, out=out))  # warm: modules loaded, attributes set
    torch.cuda.synchronize()
    s = torch.cuda.Stream()
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph, stream=s):
        szx.compress_async(xd, eb, block, out, res, stream=s)
        szx.decompress_async(out[:len(ref)], h, y, st, stream=s)
        szx.decompress_range(out[:len(ref)], 100, 40, h=h, out=part, status=pst, stream=s)
    for k in range(3):
        out.fill_(0)
        y.fill_(0)
        part.fill_(0)
        st.fill_(99)
        pst.fill_(99)
        res.fill_(-1)
        graph.replay()
        torch.cuda.synchronize()
        assert res.tolist() == [len(ref), 0], f"replay {k}"
        assert int(st.item()) == 0 and int(pst.item()) == 0, f"replay {k}"
        assert np.array_equal(out[:len(ref)].cpu().numpy(), ref), f"replay {k}: stream differs"
        assert np.array_equal(y.cpu().numpy().view(np.uint32), dref.view(np.uint32)), f"replay {k}: decode differs"
        assert np.array_equal(part.cpu().numpy().view(np.uint32),
                              dref[100 * block:140 * block].view(np.uint32)), f"replay {k}: range differs"
