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
