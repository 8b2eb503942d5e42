"""Quality metrics and the block-size choice (GPU, torch).

  psnr             -- Eq. 7: 20 log10((d_max - d_min) / sqrt(MSE)), accumulated in
                      float64.
  block_range_cdf  -- the distribution the paper plots in Fig. 2: per block of b
                      values, (max - min) / (global max - global min), as a CDF
                      at given points.
  choose_block     -- block length for `block=0`: compresses an evenly spaced
                      sample of the field with each candidate b on the GPU and
                      keeps the one with the smallest streams (highest
                      compression ratio); the paper studies the trade-off in
                      Sec. V-A.2 and settles on 128 for its data.

Nothing here is on the codec's path; the codec runs in the library's kernels.
"""
import math


def psnr(x, y):
    """Eq. 7 for CUDA (or CPU) tensors x (original) and y (decoded)."""
    xd = x.double().reshape(-1)
    yd = y.double().reshape(-1)
    rng = float(xd.max() - xd.min())
    mse = float(((xd - yd) ** 2).mean())
    if mse == 0.0:
        return math.inf
    if rng == 0.0:
        return -math.inf
    return 20.0 * math.log10(rng / math.sqrt(mse))


def block_range_cdf(x, block, points):
    """Fraction of blocks whose value range, relative to the global range, is
    at most each point (a partial last block counts with its own values)."""
    import torch
    xd = x.double().reshape(-1)
    n = xd.numel()
    nb = n // block
    g = float(xd.max() - xd.min())
    ranges = []
    if nb:
        full = xd[:nb * block].view(nb, block)
        ranges.append(full.max(dim=1).values - full.min(dim=1).values)
    if n % block:
        tail = xd[nb * block:]
        ranges.append((tail.max() - tail.min()).reshape(1))
    r = torch.cat(ranges) / (g if g > 0 else 1.0)
    return [float((r <= p).double().mean()) for p in points]


def choose_block(x, eb, candidates=(64, 128, 256), sample_values=1 << 22, pieces=16):
    """The candidate block length whose streams over a sample of x are the
    smallest.  The sample is `pieces` evenly spaced runs of x, each a multiple
    of every candidate.  Returns (block, {block: sample compression ratio})."""
    import torch

    from . import compress
    flat = x.reshape(-1)
    n = flat.numel()
    lcm = max(candidates)
    run = max(lcm, (sample_values // pieces) // lcm * lcm)
    if n <= run * pieces:
        parts = [flat]
    else:
        step = n // pieces
        parts = [flat[(i * step) // lcm * lcm:(i * step) // lcm * lcm + run] for i in range(pieces)]
    sample = torch.cat([p.contiguous() for p in parts])
    nbytes = sample.numel() * sample.element_size()
    ratios = {}
    for b in candidates:
        ratios[b] = nbytes / compress(sample, eb, b).numel()
    best = max(candidates, key=lambda b: (ratios[b], b == 128))
    return best, ratios


__all__ = ["psnr", "block_range_cdf", "choose_block"]
