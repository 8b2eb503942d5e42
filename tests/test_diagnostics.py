"""Diagnostics of the paper on synthetic data, from the oracle (CPU) and the
metrics module: Eq. 7 PSNR obeys the bound the error control implies, the
Eq. 6 right-shift overhead is small, and the block-range CDF (Fig. 2) behaves
as a CDF.  The figures are printed with -s."""
import math

import numpy as np
import pytest

import oracle

torch = pytest.importorskip("torch")
from paper_2201_13020_b300 import inputs, metrics  # noqa: E402


def _field():
    g = inputs.grf_3d((64, 64, 64), -5.0 / 3.0, 3)
    return inputs.zero_slabs(g, 0.25, 16, seed=3).reshape(-1).numpy()


@pytest.mark.parametrize("rel", [1e-2, 1e-3, 1e-4])
def test_psnr_respects_the_error_bound(rel):
    x = _field()
    eb = inputs.rel_to_abs(x, rel)
    y = oracle.decompress(oracle.compress(x, eb, 128))
    p = metrics.psnr(torch.from_numpy(x), torch.from_numpy(y))
    # |d - d'| <= e everywhere, so sqrt(MSE) <= e and PSNR >= 20 log10(range / e)
    e = oracle.error_bound(eb, oracle.F32)
    floor = 20 * math.log10((float(x.max()) - float(x.min())) / e)
    print(f"rel {rel:g}: PSNR {p:.2f} dB (floor {floor:.2f})")
    assert p >= floor - 1e-9


def test_psnr_closed_form():
    x = torch.tensor([0.0, 1.0, 2.0, 4.0], dtype=torch.float64)
    y = x + torch.tensor([0.5, -0.5, 0.5, -0.5], dtype=torch.float64)
    assert metrics.psnr(x, y) == pytest.approx(20 * math.log10(4.0 / 0.5))
    assert metrics.psnr(x, x) == math.inf


def test_block_range_cdf_is_a_cdf():
    x = torch.from_numpy(_field())
    pts = [0.0, 1e-4, 1e-3, 1e-2, 0.1, 1.0]
    for b in (32, 128, 512):
        c = metrics.block_range_cdf(x, b, pts)
        print(f"b={b}: CDF {[round(v, 3) for v in c]}")
        assert all(0.0 <= v <= 1.0 for v in c) and c == sorted(c) and c[-1] == 1.0
        assert c[0] >= 0.24  # the zeroed slabs are a quarter of the blocks, all of range 0


def test_block_range_cdf_hand_example():
    x = torch.tensor([0.0, 0.0, 1.0, 3.0, 2.0, 2.0, 10.0], dtype=torch.float64)
    # blocks of 2: ranges 0, 2, 0 and the last value alone (0); global range 10
    assert metrics.block_range_cdf(x, 2, [0.0, 0.1, 0.2]) == [0.75, 0.75, 1.0]


def test_shift_overhead_eq6_figures():
    x = _field()
    cr_rows = []
    for rel in (1e-2, 1e-3, 1e-4):
        eb = inputs.rel_to_abs(x, rel)
        c, ab = oracle.shift_overhead_bits(x, eb, 128)
        size = len(oracle.compress(x, eb, 128))
        over = (c - ab) / 8 / size
        cr_rows.append((rel, over))
        print(f"rel {rel:g}: Eq. 6 overhead {100 * over:.1f}% of the stream")
        assert -0.5 < over < 0.5
