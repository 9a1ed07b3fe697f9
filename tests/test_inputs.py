"""The seeded input generators (shared by the oracle tests and the GPU tests; they
hold none of the method's arithmetic): shapes, determinism and the point sets of the
paper's workloads."""
import numpy as np

from paper_1909_09825_gb300 import inputs


def test_uniform_seeded_and_in_range():
    x, y, a = inputs.uniform(1000, 700, seed=3)
    x2, y2, a2 = inputs.uniform(1000, 700, seed=3)
    assert x.shape == (1000,) and y.shape == (700,) and a.shape == (700,)
    assert np.array_equal(x, x2) and np.array_equal(y, y2) and np.array_equal(a, a2)
    assert x.min() >= 0 and x.max() < 1 and y.min() >= 0 and y.max() < 1


def test_chebyshev_points_increasing_first_kind_nodes():
    """Sec. 5's second point set: first-kind Chebyshev nodes mapped to [0, 1], in
    increasing order (so a transform on them takes the sort's merge path)."""
    N = 5000
    x, a = inputs.chebyshev(N, seed=1)
    assert x.shape == (N,) and a.shape == (N,)
    assert np.all(np.diff(x) > 0)
    t = np.cos(np.pi * (2.0 * np.arange(N) + 1.0) / (2.0 * N))  # nodes on [-1, 1], decreasing
    assert np.max(np.abs(x - (1.0 - t) / 2.0)) <= 1e-15
    assert np.allclose(x + x[::-1], 1.0, rtol=0, atol=1e-15)  # symmetric about 1/2


def test_with_ties_has_ties_and_signed_zeros():
    x, y, a = inputs.with_ties(4000, 3000, seed=2, n_distinct=20)
    z = np.concatenate([x, y])
    assert len(np.unique(z)) <= 20
    assert np.any(np.signbit(z) & (z == 0)) and np.any(~np.signbit(z) & (z == 0))
