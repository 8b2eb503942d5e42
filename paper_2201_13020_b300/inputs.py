"""Seeded synthetic inputs (stand-ins for the paper's SDRBench fields, Table 2).

This module only makes data: it holds none of the codec's arithmetic, and both
the CUDA path and the oracle take their inputs from it.  Every generator is
deterministic in its seed (numpy PCG64 on the host; torch.Generator on the
given device for the large 3-D fields).

  sinusoid_1d  -- 1-D sum of 8 random sinusoids + Gaussian noise (sigma 1% of
                  the clean range), 10% of 128-value blocks set constant.
  grf_3d       -- Gaussian random field with power spectrum |k|^alpha, zero
                  mean, unit variance (alpha = -5/3 for the f32 turbulence-like
                  field, -11/3 for the smoother f64 one).
  zero_slabs   -- zero 25% of a volume as 4 non-overlapping 32-plane z-slabs.
  lognormal    -- exp(sigma * g), a heavy-tailed density-like variant.
  state_vector -- unit-norm complex Gaussian amplitudes as interleaved re/im f64.
  rel_to_abs   -- value-range relative bound REL -> absolute bound (Sec. IV
                  footnote: e = REL * (max - min)).
  sinusoid_1d_torch -- the 1-D recipe computed on a torch device (large sizes).
  mixed_fields -- the many-field batch: sizes log-uniform in [lo, hi] bytes,
                  70% f32 / 30% f64, 1-D / 2-D / 3-D generators, REL drawn
                  from {1e-2, 1e-3, 1e-4}.
"""
import hashlib
import math

import numpy as np


def sinusoid_1d(n=1 << 20, seed=1, const_frac=0.10, block=128, dtype=np.float32):
    rng = np.random.Generator(np.random.PCG64(seed))
    i = np.arange(n, dtype=np.float64)
    amp = rng.uniform(0.1, 1.0, size=8)
    freq = np.exp(rng.uniform(np.log(1.0), np.log(4096.0), size=8))
    phase = rng.uniform(0.0, 2 * np.pi, size=8)
    clean = np.zeros(n)
    for a, f, p in zip(amp, freq, phase):
        clean += a * np.sin(2 * np.pi * f * i / n + p)
    rng_clean = clean.max() - clean.min()
    x = clean + rng.normal(0.0, 0.01 * rng_clean, size=n)
    nb = n // block
    chosen = rng.choice(nb, size=int(round(const_frac * nb)), replace=False)
    for k in chosen:
        x[k * block:(k + 1) * block] = x[k * block]
    return x.astype(dtype)


def grf_3d(shape, alpha, seed, device="cpu", dtype=None):
    """Gaussian random field with power spectrum |k|^alpha (k = 0 removed)."""
    import torch
    dtype = dtype or torch.float32
    work = torch.float64 if dtype == torch.float64 else torch.float32
    gen = torch.Generator(device=device)
    gen.manual_seed(seed)
    white = torch.randn(shape, generator=gen, device=device, dtype=work)
    spec = torch.fft.rfftn(white)
    del white
    axes = []
    for d, m in enumerate(shape):
        if d == len(shape) - 1:
            k = torch.fft.rfftfreq(m, device=device, dtype=work) * m
        else:
            k = torch.fft.fftfreq(m, device=device, dtype=work) * m
        view = [1] * len(shape)
        view[d] = k.numel()
        axes.append(k.view(view))
    k2 = sum(a * a for a in axes)
    k2[(0,) * len(shape)] = 1.0
    amp = k2.pow(alpha / 4.0)  # |k|^(alpha/2) amplitude gives |k|^alpha power
    amp[(0,) * len(shape)] = 0.0
    spec.mul_(amp)
    del amp, k2
    field = torch.fft.irfftn(spec, s=shape)
    del spec
    field -= field.mean()
    field /= field.std()
    return field.to(dtype).contiguous()


def zero_slabs(field, frac=0.25, planes=32, seed=0):
    """Zero `frac` of a (z, y, x) volume as non-overlapping `planes`-thick z-slabs."""
    nz = field.shape[0]
    nslabs = max(1, int(round(frac * nz / planes)))
    rng = np.random.Generator(np.random.PCG64(seed))
    slots = nz // planes
    starts = sorted(rng.choice(slots, size=min(nslabs, slots), replace=False) * planes)
    for z0 in starts:
        field[z0:z0 + planes] = 0
    return field


def lognormal(g, sigma=1.5):
    return (g * sigma).exp() if hasattr(g, "exp") else np.exp(g * sigma)


def state_vector(n_complex, seed, device="cpu"):
    import torch
    gen = torch.Generator(device=device)
    gen.manual_seed(seed)
    z = torch.randn(2 * n_complex, generator=gen, device=device, dtype=torch.float64)
    z /= torch.linalg.vector_norm(z)
    return z


def rel_to_abs(x, rel):
    """Absolute bound for a value-range relative bound (in float64)."""
    if hasattr(x, "detach"):
        lo = float(x.min())
        hi = float(x.max())
    else:
        lo = float(np.min(x))
        hi = float(np.max(x))
    return rel * (hi - lo)


def sha256(arr):
    if hasattr(arr, "detach"):
        arr = arr.detach().cpu().numpy()
    return hashlib.sha256(np.ascontiguousarray(arr).view(np.uint8)).hexdigest()


def field_sizes_loguniform(count, lo_bytes, hi_bytes, seed):
    rng = np.random.Generator(np.random.PCG64(seed))
    return [int(math.exp(v)) for v in rng.uniform(math.log(lo_bytes), math.log(hi_bytes), size=count)]


def sinusoid_1d_torch(n, seed, device="cuda", dtype=None, const_frac=0.10, block=128):
    """sinusoid_1d's recipe on a torch device (parameters drawn on the host)."""
    import torch
    dtype = dtype or torch.float32
    rng = np.random.Generator(np.random.PCG64(seed))
    amp = rng.uniform(0.1, 1.0, size=8)
    freq = np.exp(rng.uniform(np.log(1.0), np.log(4096.0), size=8))
    phase = rng.uniform(0.0, 2 * np.pi, size=8)
    i = torch.arange(n, device=device, dtype=torch.float64)
    clean = torch.zeros(n, device=device, dtype=torch.float64)
    for a, f, ph in zip(amp, freq, phase):
        clean += float(a) * torch.sin(i * (2 * np.pi * float(f) / n) + float(ph))
    del i
    span = float(clean.max() - clean.min())
    gen = torch.Generator(device=device)
    gen.manual_seed(seed)
    x = clean + torch.randn(n, generator=gen, device=device, dtype=torch.float64) * (0.01 * span)
    del clean
    nb = n // block
    if nb:
        chosen = torch.from_numpy(rng.choice(nb, size=int(round(const_frac * nb)), replace=False)).to(device)
        starts = chosen * block
        idx = (starts[:, None] + torch.arange(block, device=device)[None, :]).reshape(-1)
        x[idx] = x[starts].repeat_interleave(block)
    return x.to(dtype)


def mixed_fields(count, lo_bytes, hi_bytes, seed, device="cuda", block=128):
    """The many-field batch: a list of (tensor, rel, kind) with sizes
    log-uniform in [lo_bytes, hi_bytes] (rounded to whole blocks), 70% f32 and
    30% f64, generators 1-D sinusoid, 2-D or 3-D GRF (spectrum exponent drawn
    from {-5/3, -11/3}), REL drawn from {1e-2, 1e-3, 1e-4}."""
    import torch
    rng = np.random.Generator(np.random.PCG64(seed))
    sizes = field_sizes_loguniform(count, lo_bytes, hi_bytes, seed)
    out = []
    for i, nbytes in enumerate(sizes):
        f64 = rng.random() < 0.30
        w = 8 if f64 else 4
        n = max(block, (nbytes // (w * block)) * block)
        dt = torch.float64 if f64 else torch.float32
        kind = ["1d", "2d", "3d"][int(rng.integers(3))]
        rel = float(rng.choice([1e-2, 1e-3, 1e-4]))
        alpha = float(rng.choice([-5.0 / 3.0, -11.0 / 3.0]))
        s = seed * 1000 + i
        if kind == "1d":
            x = sinusoid_1d_torch(n, s, device=device, dtype=dt)
        else:
            d = 2 if kind == "2d" else 3
            edge = int(math.ceil(n ** (1.0 / d)))
            while edge ** d < n:
                edge += 1
            g = grf_3d((edge,) * d, alpha, s, device=device, dtype=dt)
            x = g.reshape(-1)[:n].contiguous()
            del g
        out.append((x, rel, f"{kind}/{'f64' if f64 else 'f32'}/a{alpha:.2f}"))
    return out
