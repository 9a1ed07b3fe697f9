"""Seeded synthetic inputs shared by the tests, the benchmark and the oracle checks.

This module only draws random numbers: it holds none of the transform's
arithmetic.  Every generator uses numpy's default_rng(seed) and draws in the
order x (targets), y (sources), alpha (strengths), so that the same seed gives
bit-identical host arrays to the GPU path and to the oracle.

The shapes follow the paper's experiments (Sec. 5: points uniform on [0, 1],
identical or distinct targets and sources) and the workloads the benchmark
times (clustered mixtures, batches of uneven size and bandwidth).
"""
import numpy as np


def uniform(M, N, seed=0, alpha="normal"):
    """x ~ U[0,1)^M, y ~ U[0,1)^N, alpha ~ N(0,1) (or U(-1,1), U[0,1))."""
    rng = np.random.default_rng(seed)
    x = rng.random(M)
    y = rng.random(N)
    a = _alpha(rng, N, alpha)
    return x, y, a


def _alpha(rng, N, kind):
    if kind == "normal":
        return rng.standard_normal(N)
    if kind == "sym":
        return rng.uniform(-1.0, 1.0, N)
    if kind == "pos":
        return rng.random(N)
    raise ValueError(kind)


def mixture(M, N, seed=0, n_centres=8, sigma=1e-3, background=0.1, alpha="sym"):
    """Mixture of n_centres Gaussians (centres ~ U[0,1], width sigma) plus a
    uniform background fraction; alpha ~ U(-1,1) by default."""
    rng = np.random.default_rng(seed)
    centres = rng.random(n_centres)

    def draw(n):
        pick = rng.integers(0, n_centres, n)
        pts = centres[pick] + sigma * rng.standard_normal(n)
        bg = rng.random(n) < background
        pts[bg] = rng.random(int(bg.sum()))
        return pts

    x = draw(M)
    y = draw(N)
    a = _alpha(rng, N, alpha)
    return x, y, a


def batched_sizes(B, seed=0, lo=1e2, hi=1e6, dlo=1e-6, dhi=1e-1):
    """Per-item sizes M_b = N_b = round(10^U(log lo, log hi)) and bandwidths
    delta_b = 10^U(log dlo, log dhi)."""
    rng = np.random.default_rng(seed)
    sizes = np.round(10.0 ** rng.uniform(np.log10(lo), np.log10(hi), B)).astype(np.int64)
    deltas = 10.0 ** rng.uniform(np.log10(dlo), np.log10(dhi), B)
    return sizes, deltas


def batched(B, seed=0, lo=1e2, hi=1e6, dlo=1e-6, dhi=1e-1):
    """Concatenated batch: offsets (B+1), deltas (B), x, y, alpha."""
    sizes, deltas = batched_sizes(B, seed, lo, hi, dlo, dhi)
    off = np.concatenate([[0], np.cumsum(sizes)]).astype(np.int64)
    rng = np.random.default_rng(seed + 1)
    total = int(off[-1])
    x = rng.random(total)
    y = rng.random(total)
    a = rng.standard_normal(total)
    return off, deltas, x, y, a


def with_ties(M, N, seed=0, n_distinct=64):
    """Points drawn from a small set of distinct values (many exact ties,
    including coincident sources and targets) plus signed zeros."""
    rng = np.random.default_rng(seed)
    vals = np.concatenate([[0.0, -0.0], rng.random(n_distinct - 2)])
    x = vals[rng.integers(0, n_distinct, M)]
    y = vals[rng.integers(0, n_distinct, N)]
    a = rng.standard_normal(N)
    return x, y, a


def chebyshev(N, seed=0, alpha="normal"):
    """The paper's second point set (Sec. 5): N Chebyshev points mapped to [0, 1],
    x_i = (1 - cos(pi (2 i + 1) / (2 N))) / 2 = sin^2(pi (2 i + 1) / (4 N)) (the second
    form has no cancellation near 0), in increasing order as a grid generator produces
    them, clustered at both ends, with seeded strengths alpha ~ N(0, 1)."""
    rng = np.random.default_rng(seed)
    x = np.sin(np.pi * (2.0 * np.arange(N) + 1.0) / (4.0 * N)) ** 2
    return x, _alpha(rng, N, alpha)


def batched_device(B, device, seed=0, lo=1e2, hi=1e6, dlo=1e-6, dhi=1e-1):
    """Batched workload drawn on the device (torch generator) for large B: item sizes
    M_b = N_b and bandwidths from batched_sizes (numpy, seed), then x, y ~ U[0,1) and
    alpha ~ N(0,1) from a torch generator seeded with seed + 1.  Returns
    (x_off, y_off, delta, x, y, alpha) as device tensors and the host sizes."""
    import torch
    sizes, deltas = batched_sizes(B, seed, lo, hi, dlo, dhi)
    off = np.concatenate([[0], np.cumsum(sizes)]).astype(np.int64)
    total = int(off[-1])
    g = torch.Generator(device=device)
    g.manual_seed(seed + 1)
    x = torch.rand(total, generator=g, dtype=torch.float64, device=device)
    y = torch.rand(total, generator=g, dtype=torch.float64, device=device)
    a = torch.randn(total, generator=g, dtype=torch.float64, device=device)
    t_off = torch.from_numpy(off).to(device)
    return t_off, t_off.clone(), torch.from_numpy(deltas).to(device), x, y, a, sizes
