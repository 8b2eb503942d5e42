"""A bounded device wait that runs out is reported, not hung: with the
look-back limit cut to 1 microsecond, compressions whose look-back has to wait
for a predecessor give up, return SZX_ERR_TIMEOUT, and leave the context
usable -- the next compression with the normal limit is byte-identical to the
oracle.  (Giving up early only shortens a prefix sum, so a record lands
earlier inside the caller's buffer: no access leaves it.)  No fault, trap or
hang is involved."""
import os

import numpy as np
import pytest

import oracle

torch = pytest.importorskip("torch")
import paper_2201_13020_b300 as szx  # noqa: E402
from paper_2201_13020_b300 import inputs  # noqa: E402

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("dtype", ["f32", "f64"])
def test_lookback_timeout_is_reported_and_the_context_survives(dtype):
    # f64 at b = 128 takes the kernel whose warp 0 computes every block's
    # statistics for the tile: its exchange waits have the copy limit, so only
    # the look-back gives up
    if dtype == "f32":
        g = inputs.grf_3d((256, 256, 256), -5.0 / 3.0, 7, device="cuda")
    else:
        g = inputs.grf_3d((192, 192, 192), -11.0 / 3.0, 7, device="cuda", dtype=torch.float64)
    x = g.reshape(-1).contiguous()
    eb = inputs.rel_to_abs(x, 1e-3)
    saw_timeout = False
    os.environ["SZX_LOOKBACK_US"] = "1"
    try:
        for _ in range(5):
            try:
                szx.compress(x, eb)
            except szx.SzxError as exc:
                assert exc.status == 6, exc  # SZX_ERR_TIMEOUT, nothing else
                saw_timeout = True
                break
    finally:
        del os.environ["SZX_LOOKBACK_US"]
    assert saw_timeout, "no look-back waited longer than 1 us in five runs"
    torch.cuda.synchronize()  # the context is intact
    xs = x[:1 << 20].contiguous()
    s = szx.compress(xs, eb)
    assert np.array_equal(s.cpu().numpy(), oracle.compress(xs.cpu().numpy(), eb, 128))
