"""CPU checks of the bench's oracle baseline: the all-core measurement splits the
field into disjoint block-aligned ranges, one spawned process each, and that
is the same work as one pass because every block is coded from its own values
alone (Algorithm 1).  No GPU."""
import numpy as np

import oracle
import szx_stream as ss


def test_disjoint_block_ranges_make_the_same_blocks_as_one_pass():
    rng = np.random.default_rng(3)
    block = 128
    x = np.cumsum(rng.normal(size=20 * block + 37)).astype(np.float32)
    eb = 1e-2 * float(x.max() - x.min())
    whole = ss.parse(oracle.compress(x, eb, block))
    cut = [0, 5 * block, 13 * block, x.size]
    parts = [ss.parse(oracle.compress(x[a:b], eb, block)) for a, b in zip(cut[:-1], cut[1:])]
    blocks = [blk for p in parts for blk in p.blocks]
    assert len(blocks) == len(whole.blocks)
    for a, b in zip(whole.blocks, blocks):
        assert (a.state, a.mu_bits, a.req, a.L[:a.length], a.t[:a.length]) == \
            (b.state, b.mu_bits, b.req, b.L[:b.length], b.t[:b.length])


def test_oracle_timer_one_thread_and_all_cores():
    import bench
    saved = list(bench.SHAPE_RUN)
    bench.SHAPE_RUN[:] = [64, 64, 64]
    try:
        x = np.cumsum(np.random.default_rng(0).normal(size=64 ** 3)).astype(np.float32)
        ot = bench.OracleTimer(x, 1e-1)
        try:
            # the slice is the first 64 planes (all of this small field), split
            # into block-aligned ranges that cover it once
            assert ot.n == x.size
            assert ot.ranges[0][0] == 0 and ot.ranges[-1][1] == ot.n
            assert all(a % bench.BLOCK == 0 for a, _ in ot.ranges)
            assert all(p[1] == q[0] for p, q in zip(ot.ranges, ot.ranges[1:]))
            one = ot.single_thread(1)
            allc = ot.all_cores(1)
            assert one["cores"] == 1 and one["value"] > 0
            assert allc["cores"] == len(ot.ranges) and allc["value"] > 0 and allc["cpu_seconds"] > 0
        finally:
            ot.close()
    finally:
        bench.SHAPE_RUN[:] = saved
