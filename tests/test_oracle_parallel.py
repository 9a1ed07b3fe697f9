"""Pins of the oracle's multi-core variant of the paper's algorithm (o3_recurrence_par,
o3_sort_merged_par): the same stable order bit for bit, and the same values as the
single-thread recurrence and the brute-force SOE sum.  The segment split is what
changes; each carry crosses a segment boundary with one directly computed span
exponential, so a dropped carry, a wrong span or a reversed direction moves the values
far beyond the tolerances below."""
import numpy as np
import pytest

from oracle import oracle, soe_cf
from paper_1909_09825_gb300 import inputs


def _ties(rng, n):
    vals = np.concatenate([[0.0, -0.0, 1e-300], rng.random(5)])
    return vals[rng.integers(0, len(vals), n)]


@pytest.mark.parametrize("nthreads", [1, 3, 8])
def test_parallel_sort_is_the_stable_order(nthreads):
    rng = np.random.default_rng(nthreads)
    for M, N in ((0, 1), (1, 0), (5, 7), (1000, 777), (40000, 30001)):
        for tied in (False, True):
            x = _ties(rng, M) if tied else rng.random(M)
            y = _ties(rng, N) if tied else rng.random(N)
            p = oracle.sort_merged_par(x, y, nthreads=nthreads)
            assert np.array_equal(p, oracle.sort_merged(x, y))
            # and numpy's stable argsort over [y, x] (the merged order), -0.0 == +0.0
            assert np.array_equal(p, np.argsort(np.concatenate([y, x]) + 0.0, kind="stable"))


def test_parallel_sort_rejects_nonfinite():
    with pytest.raises(ValueError):
        oracle.sort_merged_par(np.array([0.1, np.nan]), np.array([0.2]))


@pytest.mark.parametrize("seed", range(6))
def test_parallel_recurrence_equals_soe_direct_tiny(seed):
    """Brute force on tiny inputs with ties and signed zeros, many segments of a few
    points each (every carry path crosses several boundaries)."""
    rng = np.random.default_rng(100 + seed)
    M, N = rng.integers(1, 50, 2)
    if seed % 2:
        x, y = _ties(rng, M), _ties(rng, N)
    else:
        x, y = rng.random(M), rng.random(N)
    a = rng.standard_normal(N)
    tau, W, _ = soe_cf.cf_soe(8)
    for delta in (1e-3, 1e-1):
        ref = oracle.soe_direct(x, y, a, delta, tau, W)
        for nseg in (1, 2, 5, int(M + N), int(M + N) + 9):
            u = oracle.recurrence_par(x, y, a, delta, tau, W, nseg=nseg, nthreads=3)
            assert np.max(np.abs(u - ref)) <= 1e-14 * np.abs(a).sum(), (delta, nseg)


@pytest.mark.parametrize("exact_self", [False, True])
def test_parallel_recurrence_equals_serial(exact_self):
    """Medium size, the serial recurrence as reference, with and without ties."""
    rng = np.random.default_rng(7)
    tau, W, _ = soe_cf.cf_soe(10)
    for tied in (False, True):
        x, y, a = inputs.uniform(60000, 50000, seed=3)
        if tied:
            x, y = np.round(x * 500) / 500, np.round(y * 500) / 500
        for delta in (1e-6, 1e-3, 1.0):
            ref, pref = oracle.recurrence(x, y, a, delta, tau, W, exact_self=exact_self, return_perm=True)
            for nseg, nt in ((1, 1), (17, 4), (256, 8)):
                u, perm = oracle.recurrence_par(x, y, a, delta, tau, W, exact_self=exact_self, nseg=nseg,
                                                nthreads=nt, return_perm=True)
                assert np.array_equal(perm, pref)
                assert np.max(np.abs(u - ref)) <= 1e-13 * np.abs(a).sum(), (tied, delta, nseg)


def test_parallel_recurrence_no_sources_and_one_segment_edges():
    tau, W, _ = soe_cf.cf_soe(6)
    x = np.linspace(0, 1, 11)
    u = oracle.recurrence_par(x, np.empty(0), np.empty(0), 1e-2, tau, W, nseg=4)
    assert np.array_equal(u, np.zeros(11))
    u = oracle.recurrence_par(x, np.array([0.5]), np.array([2.0]), 1e-2, tau, W, nseg=3)
    assert np.allclose(u, 2.0 * soe_cf.soe_eval(tau, W, (x - 0.5) / 0.1), rtol=0, atol=1e-14)
