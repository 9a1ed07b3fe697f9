"""Bit-exact check of the GPU merged sort (steps a1-a2) against the oracle's stable
merge sort: the order is unique (coordinate, then merged index)."""
import numpy as np
import pytest
import torch

import paper_1909_09825_gb300 as fgt
from oracle import oracle
from paper_1909_09825_gb300 import inputs

pytestmark = pytest.mark.gpu


def _perm(x, y, dev):
    return fgt.sort_merged(torch.from_numpy(x).to(dev), torch.from_numpy(y).to(dev)).cpu().numpy()


@pytest.mark.parametrize("M,N", [(1, 0), (0, 1), (1, 1), (5, 3), (4095, 1), (4096, 4096), (4097, 5000),
                                 (100000, 77777), (1 << 20, 1 << 20)])
def test_perm_uniform(cuda, M, N):
    x, y, _ = inputs.uniform(M, N, seed=M + N)
    assert np.array_equal(_perm(x, y, cuda), oracle.sort_merged(x, y))


def test_perm_ties_signed_zero_negative(cuda):
    rng = np.random.default_rng(9)
    vals = np.array([0.0, -0.0, -1.5, 2.0, 1e-300, -1e-300, 5e-324, 3.0, -3.0, 1e300])
    x = vals[rng.integers(0, len(vals), 30000)]
    y = vals[rng.integers(0, len(vals), 20000)]
    assert np.array_equal(_perm(x, y, cuda), oracle.sort_merged(x, y))


def test_perm_all_equal(cuda):
    x = np.full(9000, 0.75)
    y = np.full(7000, 0.75)
    assert np.array_equal(_perm(x, y, cuda), np.arange(16000))


def test_perm_mixture(cuda):
    x, y, _ = inputs.mixture(300000, 200000, seed=4)
    assert np.array_equal(_perm(x, y, cuda), oracle.sort_merged(x, y))


def _presorted(M, N, seed, n_distinct=None):
    rng = np.random.default_rng(seed)
    if n_distinct:
        vals = np.concatenate([[0.0, -0.0, -0.25], rng.random(n_distinct - 3)])
        x, y = vals[rng.integers(0, n_distinct, M)], vals[rng.integers(0, n_distinct, N)]
    else:
        x, y = rng.random(M), rng.random(N)
    return np.sort(x, kind="stable"), np.sort(y, kind="stable")


@pytest.mark.parametrize("M,N,nd", [(1, 1, None), (0, 5000, None), (5000, 0, 7), (4096, 4096, None),
                                    (4097, 12289, 5), (30001, 20000, 64), (100000, 3, None), (1 << 20, 1 << 19, None)])
def test_perm_presorted(cuda, M, N, nd):
    """Sources and targets each presorted (ties and signed zeros included): the sort is
    one merge, bit-exact against the oracle's stable sort."""
    x, y = _presorted(M, N, M + 7 * N, nd)
    assert np.array_equal(_perm(x, y, cuda), oracle.sort_merged(x, y))


@pytest.mark.parametrize("where", ["x_lane0", "x_tile_start", "y_last", "x_only_sorted"])
def test_perm_almost_presorted(cuda, where):
    """One inversion (at a warp's first lane, at a tile start, at the last source) or one
    unsorted run: the digit passes run, still bit-exact."""
    x, y = _presorted(20000, 4096, 11)
    if where == "x_lane0":
        x[[31, 32]] = x[[32, 31]]       # merged position 4096 + 32: lane 0 of a warp
    elif where == "x_tile_start":
        x[[4095, 4096]] = x[[4096, 4095]]  # merged position 8192: first point of a tile
    elif where == "y_last":
        y[[4094, 4095]] = y[[4095, 4094]]
    else:
        y = np.random.default_rng(12).random(4096)
    assert np.array_equal(_perm(x, y, cuda), oracle.sort_merged(x, y))


def _binned(n_bins, per_bin, seed, n_free=0):
    """Points that share 32-bit prefix keys: the range is pinned to [0, 1] (a source at
    each end), so a prefix is floor(z 2^31); each of n_bins random bins gets per_bin
    distinct coordinates inside it, dealt at random to targets and sources, plus n_free
    uniform points and, for short runs, a few exact ties across the two families."""
    rng = np.random.default_rng(seed)
    bins = rng.choice(1 << 31, n_bins, replace=False).astype(np.float64)
    z = ((bins[:, None] + rng.random((n_bins, per_bin))) / 2.0 ** 31).ravel()
    z = np.concatenate([z, rng.random(n_free)])
    rng.shuffle(z)
    cut = len(z) // 2
    x, y = z[:cut].copy(), np.concatenate([[0.0, 1.0], z[cut:]])
    if per_bin < 30:  # (a tie must not make a bin of 32 one of 33)
        x[:50] = y[2:52]  # coordinates shared by a target and a source
    return x, y


@pytest.mark.parametrize("n_bins,per_bin,n_free", [(60000, 2, 0), (20000, 5, 100000), (3000, 32, 5000)])
def test_perm_runs_of_equal_prefixes(cuda, n_bins, per_bin, n_free):
    """Runs of equal prefix keys, up to the longest that the fix-up sorts (32 points),
    some across tile boundaries: bit-exact."""
    x, y = _binned(n_bins, per_bin, n_bins + per_bin, n_free)
    assert np.array_equal(_perm(x, y, cuda), oracle.sort_merged(x, y))


@pytest.mark.parametrize("case", ["run_of_33", "narrow_cluster", "far_outlier"])
def test_perm_full_sort_fallback(cuda, case):
    """Runs of equal prefixes too long for the fix-up: one bin of 33 distinct points, a
    cluster of 5000 distinct points 1e-13 wide, or every point in one bin because of a
    coordinate at 1e300.  The full 64-bit sort runs; bit-exact."""
    rng = np.random.default_rng(17)
    if case == "run_of_33":
        x, y = _binned(1, 33, 3, 50000)
    else:
        x, y, _ = inputs.uniform(70000, 60000, seed=18)
        if case == "narrow_cluster":
            x[:5000] = 0.5 + 1e-13 * rng.random(5000)
        else:
            y[7] = 1e300
    assert np.array_equal(_perm(x, y, cuda), oracle.sort_merged(x, y))


def test_perm_negative_and_subnormal_ranges(cuda):
    """Items whose coordinates are all negative, or all subnormal: bit-exact."""
    rng = np.random.default_rng(19)
    x, y = -rng.random(30000) * 7.0, -rng.random(25000) * 7.0 - 1e-3
    assert np.array_equal(_perm(x, y, cuda), oracle.sort_merged(x, y))
    x, y = rng.random(20000) * 1e-310, rng.random(20000) * 1e-310
    assert np.array_equal(_perm(x, y, cuda), oracle.sort_merged(x, y))
