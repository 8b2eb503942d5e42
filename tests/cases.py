"""Seeded input cases shared by the GPU parity tests and the CPU checks of
what those cases cover.  Nothing here computes any part of the method."""
import numpy as np


def inputs_tile(block, dtype):
    """Values per tile: G = max(8, 32768 / (b w)) blocks of b values."""
    w = np.dtype(dtype).itemsize
    return max(8, 32768 // (block * w)) * block


def value_distribution_cases(dtype):
    """Three tiles and a ragged tail of each distribution (seed 5)."""
    rng = np.random.default_rng(5)
    n = 3 * inputs_tile(128, dtype) + 333
    return {
        "smooth": np.sin(np.linspace(0, 50, n)) + 1e-3 * rng.normal(size=n),
        "noise": rng.normal(size=n),
        "cauchy": rng.standard_cauchy(size=n),
        "tiny": rng.normal(size=n) * 1e-38,
        "huge": rng.normal(size=n) * (1e37 if dtype == np.float32 else 1e300),
        "offset": 1000.0 + np.cumsum(rng.normal(size=n)) * 0.01,
        "steps": np.repeat(rng.normal(size=n // 100 + 1), 100)[:n],
        "zeros": np.where(rng.random(n) < 0.5, 0.0, -0.0),
        "signs": rng.choice([-1.0, 1.0], size=n) * rng.uniform(0.5, 1.0, size=n),
    }


def bound_for(x, rel):
    """Absolute bound rel x (value range); 1e-3 where the range is zero or not finite."""
    rngv = float(np.max(x)) - float(np.min(x))
    eb = rel * rngv if np.isfinite(rngv) and rngv > 0 else 1e-3
    if not np.isfinite(eb) or eb <= 0:
        eb = 1e-3
    return eb


VALUE_RELS = (1e-1, 1e-3, 1e-6)
