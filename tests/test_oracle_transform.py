"""Pins of the C oracle (oracle/fgt_oracle.c): closed forms, invariants, the SOE
error bound, brute force on tiny inputs, and finite differences for the gradients."""
import numpy as np
import pytest

from oracle import oracle, soe_cf
from paper_1909_09825_gb300 import inputs


def test_direct_single_source_closed_form():
    x = np.linspace(-1, 1, 33)
    for delta in (1e-3, 0.5, 7.0):
        u = oracle.direct(x, np.array([0.3]), np.array([2.5]), delta)
        assert np.allclose(u, 2.5 * np.exp(-(x - 0.3) ** 2 / (4 * delta)), rtol=1e-15, atol=0)


def test_direct_gaussian_integral():
    """Sources on a fine uniform grid with alpha_j = h approximate the integral
    int exp(-(x-y)^2/(4 delta)) dy = sqrt(4 pi delta) (trapezoid rule is spectrally
    accurate for the Gaussian): pins the 4 delta in eq. 1.2."""
    delta = 1e-3
    h = 1e-3
    y = np.arange(-1.0, 2.0 + h / 2, h)
    a = np.full(len(y), h)
    x = np.array([0.2, 0.5, 0.9])
    u = oracle.direct(x, y, a, delta)
    assert np.allclose(u, np.sqrt(4 * np.pi * delta), rtol=1e-12)


def test_soe_direct_within_En():
    """|u_SOE - u_G| <= E_n sum|alpha| (eq. 3.1 and linearity)."""
    x, y, a = inputs.uniform(400, 300, seed=1)
    for n in (4, 8, 12):
        tau, W, En = soe_cf.cf_soe(n)
        for delta in (1e-4, 1e-2, 1.0):
            u2 = oracle.soe_direct(x, y, a, delta, tau, W)
            u1 = oracle.direct(x, y, a, delta)
            assert np.max(np.abs(u2 - u1)) <= En * np.abs(a).sum() * 1.0001


def test_soe_direct_single_source():
    tau, W, _ = soe_cf.cf_soe(10)
    x = np.linspace(-0.5, 0.5, 101)
    delta = 1e-2
    u = oracle.soe_direct(x, np.array([0.1]), np.array([1.0]), delta, tau, W)
    assert np.allclose(u, soe_cf.soe_eval(tau, W, (x - 0.1) / np.sqrt(delta)), rtol=0, atol=1e-14)


@pytest.mark.parametrize("seed", range(6))
def test_recurrence_equals_soe_direct_tiny(seed):
    """Brute force on tiny inputs, including ties and signed zeros: the paper's
    sorted recurrences (eqs. 4.3-4.6) reproduce the SOE sum (eqs. 4.1-4.2)."""
    rng = np.random.default_rng(seed)
    M, N = rng.integers(1, 40, 2)
    vals = np.concatenate([[0.0, -0.0], rng.random(6)])
    if seed % 2:
        x, y = vals[rng.integers(0, 8, M)], vals[rng.integers(0, 8, N)]
    else:
        x, y = rng.random(M), rng.random(N)
    a = rng.standard_normal(N)
    tau, W, _ = soe_cf.cf_soe(8)
    for delta in (1e-3, 0.3):
        u3 = oracle.recurrence(x, y, a, delta, tau, W)
        u2 = oracle.soe_direct(x, y, a, delta, tau, W)
        assert np.max(np.abs(u3 - u2)) <= 1e-14 * np.abs(a).sum()


@pytest.mark.parametrize("seed", range(6))
def test_recurrence_self_equals_soe_direct_tiny(seed):
    """Fig. 4.1's identical-points algorithm (one sort, inclusive forward and exclusive
    backward pass) against the brute-force SOE sum with y = x, ties and signed zeros
    included: every pair, the self pair too, gets the SOE kernel value."""
    rng = np.random.default_rng(100 + seed)
    N = int(rng.integers(1, 50))
    vals = np.concatenate([[0.0, -0.0], rng.random(5)])
    x = vals[rng.integers(0, 7, N)] if seed % 2 else rng.random(N)
    a = rng.standard_normal(N)
    tau, W, _ = soe_cf.cf_soe(10)
    for delta in (1e-3, 0.3):
        u = oracle.recurrence_self(x, a, delta, tau, W)
        u2 = oracle.soe_direct(x, x, a, delta, tau, W)
        assert np.max(np.abs(u - u2)) <= 1e-14 * np.abs(a).sum()


@pytest.mark.parametrize("seed", range(6))
def test_recurrence_self_exact_brute_force_tiny(seed):
    """exact_self with identical points against brute force on tiny inputs with runs of
    equal coordinates (signed zeros included): the kernel matrix is S_n(|x_i - x_j|)
    except where x_i == x_j, where it is G(0) = 1."""
    rng = np.random.default_rng(300 + seed)
    N = int(rng.integers(1, 40))
    vals = np.concatenate([[0.0, -0.0], rng.random(4)])
    x = vals[rng.integers(0, 6, N)]
    a = rng.standard_normal(N)
    tau, W, _ = soe_cf.cf_soe(8)
    delta = 0.05
    d = np.abs(x[:, None] - x[None, :]) / np.sqrt(delta)
    K = np.real(np.exp(-d[:, :, None] * tau[None, None, :]) @ W)
    K[x[:, None] == x[None, :]] = 1.0
    u = oracle.recurrence_self(x, a, delta, tau, W, exact_self=True)
    assert np.max(np.abs(u - K @ a)) <= 1e-14 * np.abs(a).sum()


def test_recurrence_self_exact_equals_general_exact():
    """Identical-points exact_self against the general recurrence on (x, x) with
    exact_self (sources before targets on ties), with ties."""
    x, _, a = inputs.with_ties(3000, 3000, seed=31, n_distinct=200)
    tau, W, _ = soe_cf.cf_soe(10)
    u = oracle.recurrence_self(x, a[:len(x)], 1e-3, tau, W, exact_self=True)
    u2 = oracle.recurrence(x, x, a[:len(x)], 1e-3, tau, W, exact_self=True)
    assert np.max(np.abs(u - u2)) <= 1e-13 * np.abs(a[:len(x)]).sum()


def test_recurrence_self_one_point():
    """N = 1: u = alpha S_n(0) = alpha Re sum_k W_k (the self weight of Fig. 4.1)."""
    tau, W, _ = soe_cf.cf_soe(8)
    u = oracle.recurrence_self(np.array([0.37]), np.array([2.0]), 1e-2, tau, W)
    assert abs(u[0] - 2.0 * np.sum(W.real)) <= 1e-15


def test_sort_matches_numpy_stable_argsort():
    x, y, _ = inputs.with_ties(5000, 4000, seed=2)
    perm = oracle.sort_merged(x, y)
    z = np.concatenate([y, x])
    z = np.where(z == 0, 0.0, z)  # -0.0 ties with +0.0
    assert np.array_equal(perm, np.argsort(z, kind="stable"))


def test_sort_presorted_runs_is_a_merge():
    """Sources and targets each presorted (ties, signed zeros): the stable merged order
    is the merge of the two runs with sources first on equal coordinates."""
    x, y, _ = inputs.with_ties(3000, 2000, seed=5, n_distinct=30)
    x, y = np.sort(x, kind="stable"), np.sort(y, kind="stable")
    perm = oracle.sort_merged(x, y)
    N = len(y)
    i = j = 0
    merged = []
    while i < N or j < len(x):  # two-run merge, written out
        if i < N and (j == len(x) or y[i] <= x[j]):
            merged.append(i)
            i += 1
        else:
            merged.append(N + j)
            j += 1
    assert np.array_equal(perm, np.array(merged))


def test_sort_rejects_nonfinite():
    with pytest.raises(ValueError):
        oracle.sort_merged(np.array([0.1, np.nan]), np.array([0.2]))


def test_recurrence_invariants():
    """Reflection (x,y -> -x,-y swaps the two passes), exact scaling (x,y -> 2x,2y with
    delta -> 4 delta), linearity in alpha and translation."""
    x, y, a = inputs.uniform(3000, 2000, seed=3)
    tau, W, _ = soe_cf.cf_soe(10)
    d = 1e-3
    u = oracle.recurrence(x, y, a, d, tau, W)
    s = np.abs(a).sum()
    assert np.max(np.abs(oracle.recurrence(-x, -y, a, d, tau, W) - u)) <= 1e-13 * s
    assert np.max(np.abs(oracle.recurrence(2 * x, 2 * y, a, 4 * d, tau, W) - u)) <= 1e-13 * s
    b = np.random.default_rng(4).standard_normal(len(y))
    ul = oracle.recurrence(x, y, 2 * a - 3 * b, d, tau, W)
    ub = oracle.recurrence(x, y, b, d, tau, W)
    assert np.max(np.abs(ul - (2 * u - 3 * ub))) <= 1e-13 * (2 * s + 3 * np.abs(b).sum())
    assert np.max(np.abs(oracle.recurrence(x + 0.375, y + 0.375, a, d, tau, W) - u)) <= 1e-11 * s


def test_exact_self_term():
    """Coincident sources get G(0) = 1 instead of S_n(0) with exact_self."""
    rng = np.random.default_rng(5)
    x = rng.random(500)
    y = np.concatenate([x[:200], rng.random(100)])
    a = rng.standard_normal(300)
    tau, W, _ = soe_cf.cf_soe(8)
    u0 = oracle.recurrence(x, y, a, 1e-3, tau, W)
    u1 = oracle.recurrence(x, y, a, 1e-3, tau, W, exact_self=True)
    corr = np.zeros(500)
    corr[:200] = (1 - np.sum(W.real)) * a[:200]
    assert np.allclose(u1 - u0, corr, rtol=0, atol=1e-14)


def _fd(f, v, h):
    g = np.empty_like(v)
    for i in range(len(v)):
        vp, vm = v.copy(), v.copy()
        vp[i] += h
        vm[i] -= h
        g[i] = (f(vp) - f(vm)) / (2 * h)
    return g


def test_grad_direct_finite_differences():
    x, y, a = inputs.uniform(15, 12, seed=6)
    g = np.random.default_rng(7).standard_normal(15)
    d = 2e-2
    L = lambda xx, yy, aa, dd: np.dot(g, oracle.direct(xx, yy, aa, dd))
    gx, gy, ga, gd = oracle.grad_direct(x, y, a, d, g)
    assert np.allclose(gx, _fd(lambda v: L(v, y, a, d), x, 1e-6), rtol=1e-6, atol=1e-8)
    assert np.allclose(gy, _fd(lambda v: L(x, v, a, d), y, 1e-6), rtol=1e-6, atol=1e-8)
    assert np.allclose(ga, _fd(lambda v: L(x, y, v, d), a, 1e-2), rtol=1e-9, atol=1e-11)  # L is linear in alpha
    assert np.isclose(gd, (L(x, y, a, d + 1e-7) - L(x, y, a, d - 1e-7)) / 2e-7, rtol=1e-6)


def test_grad_soe_finite_differences():
    x, y, a = inputs.uniform(15, 12, seed=8)
    g = np.random.default_rng(9).standard_normal(15)
    tau, W, _ = soe_cf.cf_soe(8)
    d = 2e-2
    L = lambda xx, yy, aa, dd: np.dot(g, oracle.soe_direct(xx, yy, aa, dd, tau, W))
    gx, gy, ga, gd = oracle.grad_soe(x, y, a, d, tau, W, g)
    assert np.allclose(gx, _fd(lambda v: L(v, y, a, d), x, 1e-7), rtol=1e-5, atol=1e-7)
    assert np.allclose(gy, _fd(lambda v: L(x, v, a, d), y, 1e-7), rtol=1e-5, atol=1e-7)
    assert np.allclose(ga, _fd(lambda v: L(x, y, v, d), a, 1e-2), rtol=1e-9, atol=1e-11)  # L is linear in alpha
    assert np.isclose(gd, (L(x, y, a, d + 1e-7) - L(x, y, a, d - 1e-7)) / 2e-7, rtol=1e-5)
