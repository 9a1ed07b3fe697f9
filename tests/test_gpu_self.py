"""Identical targets and sources (Fig. 4.1): fgt1d_execute_self against the oracle's
one-sort recurrence, the brute-force SOE sum and the general merged transform."""
import numpy as np
import pytest
import torch

import paper_1909_09825_gb300 as fgt
from oracle import oracle, soe_cf
from paper_1909_09825_gb300 import _lib, inputs

from gpu_util import gpu_transform, rel_inf

pytestmark = pytest.mark.gpu

TOL_ARITH64 = 1e-12


def _self(plan, x, a, dev):
    T = lambda v: torch.from_numpy(np.ascontiguousarray(v)).to(dev)
    return fgt.transform_self(plan, T(x), T(a)).cpu().numpy()


@pytest.mark.parametrize("N", [1, 2, 100, 4095, 4096, 4097, 30001])
def test_self_vs_oracle(cuda, N):
    x, _, _ = inputs.uniform(N, 1, seed=N)
    a = np.random.default_rng(N + 1).standard_normal(N)
    n, tau, W, En = soe_cf.plan_soe(1e-10)
    for delta in (1.0, 1e-4):
        plan = fgt.Plan(delta, soe=(tau, W))
        u = _self(plan, x, a, cuda)
        assert rel_inf(u, oracle.recurrence_self(x, a, delta, tau, W), a) <= TOL_ARITH64


def test_self_ties_and_signed_zeros(cuda):
    x, _, a = inputs.with_ties(6000, 6000, seed=4, n_distinct=40)
    n, tau, W, En = soe_cf.plan_soe(1e-8)
    plan = fgt.Plan(1e-2, soe=(tau, W))
    u = _self(plan, x, a, cuda)
    assert rel_inf(u, oracle.recurrence_self(x, a, 1e-2, tau, W), a) <= TOL_ARITH64
    idx = np.arange(0, 6000, 97)
    assert rel_inf(u[idx], oracle.soe_direct(x[idx], x, a, 1e-2, tau, W), a) <= TOL_ARITH64


def test_self_equals_merged_transform(cuda):
    """The same sum through the general path with y = x (2N merged points)."""
    x, _, a = inputs.mixture(50000, 1, seed=8)
    a = np.random.default_rng(9).standard_normal(50000)
    plan = fgt.Plan(1e-4, 1e-8)
    u = _self(plan, x, a, cuda)
    assert rel_inf(u, gpu_transform(plan, x, x, a), a) <= TOL_ARITH64


@pytest.mark.parametrize("delta", [1.0, 1e-6])
def test_self_chebyshev_points(cuda, delta):
    """Sec. 5's Chebyshev points (gaps from 1.2e-8 at the ends to 7.9e-5 in the middle)."""
    x, a = inputs.chebyshev(20000, seed=3)
    n, tau, W, En = soe_cf.plan_soe(1e-10)
    plan = fgt.Plan(delta, soe=(tau, W))
    u = _self(plan, x, a, cuda)
    assert rel_inf(u, oracle.recurrence_self(x, a, delta, tau, W), a) <= TOL_ARITH64
    plan2 = fgt.Plan(delta, 1e-10)
    idx = np.arange(0, 20000, 499)
    assert rel_inf(_self(plan2, x, a, cuda)[idx], oracle.direct(x[idx], x, a, delta), a) <= 2e-10 + 1e-13


def test_self_large_vs_direct(cuda):
    """Table 5.1's workload shape (uniform points, delta = 1) at N = 2^22, sampled
    targets against the direct Gauss sum."""
    N = 1 << 22
    x, _, _ = inputs.uniform(N, 1, seed=0)
    a = np.random.default_rng(1).random(N)
    plan = fgt.Plan(1.0, 1e-8)
    u = _self(plan, x, a, cuda)
    idx = np.random.default_rng(2).choice(N, 6, replace=False)
    assert rel_inf(u[idx], oracle.direct(x[idx], x, a, 1.0, nthreads=0), a) <= 2e-8 + 1e-13


@pytest.mark.parametrize("n_distinct", [40, 3])
def test_self_exact_vs_oracle(cuda, n_distinct):
    """exact_self with identical points: runs of equal coordinates (signed zeros
    included; with 3 distinct values every run spans many tiles) get G(0) = 1."""
    x, _, a = inputs.with_ties(9000, 9000, seed=14, n_distinct=n_distinct)
    n, tau, W, En = soe_cf.plan_soe(1e-8)
    for delta in (1e-2, 1.0):
        plan = fgt.Plan(delta, soe=(tau, W), exact_self=True)
        u = _self(plan, x, a, cuda)
        assert rel_inf(u, oracle.recurrence_self(x, a, delta, tau, W, exact_self=True), a) <= TOL_ARITH64


@pytest.mark.parametrize("N", [1, 4097, 30001])
def test_self_exact_distinct_points(cuda, N):
    """Distinct points: exact_self adds (1 - S_n(0)) alpha_i, the self pair only."""
    x, _, _ = inputs.uniform(N, 1, seed=N + 5)
    a = np.random.default_rng(N).standard_normal(N)
    n, tau, W, En = soe_cf.plan_soe(1e-6)
    plan = fgt.Plan(1e-3, soe=(tau, W), exact_self=True)
    u = _self(plan, x, a, cuda)
    assert rel_inf(u, oracle.recurrence_self(x, a, 1e-3, tau, W, exact_self=True), a) <= TOL_ARITH64
    u0 = _self(fgt.Plan(1e-3, soe=(tau, W)), x, a, cuda)
    assert rel_inf(u - u0, (1 - np.sum(W.real)) * a, a) <= TOL_ARITH64


def test_self_exact_vs_direct(cuda):
    """Against the direct Gauss sum (G(0) = 1 for the self pair) on a mixture with
    duplicated points, at the 2 eps + 1e-13 bound."""
    x, _, _ = inputs.mixture(20000, 1, seed=15)
    x[10000:12000] = x[:2000]  # coincident pairs
    a = np.random.default_rng(16).standard_normal(20000)
    plan = fgt.Plan(1e-4, 1e-8, exact_self=True)
    u = _self(plan, x, a, cuda)
    idx = np.concatenate([np.arange(0, 20000, 331), np.arange(10000, 10040)])
    assert rel_inf(u[idx], oracle.direct(x[idx], x, a, 1e-4), a) <= 2e-8 + 1e-13


TOL_ARITH32 = 5e-6  # the FP32 path's arithmetic budget (eps >= 1e-6)


@pytest.mark.parametrize("N", [1, 100, 4097, 30001])
def test_self_fp32_vs_oracle(cuda, N):
    """FP32 sweeps with identical points (the value channel accumulates apart from the
    strengths, which every point keeps)."""
    x, _, _ = inputs.uniform(N, 1, seed=N + 2)
    a = np.random.default_rng(N + 3).standard_normal(N)
    n, tau, W, En = soe_cf.plan_soe(1e-6)
    for delta in (1.0, 1e-4):
        plan = fgt.Plan(delta, soe=(tau, W), precision="fp32")
        u = _self(plan, x, a, cuda)
        assert rel_inf(u, oracle.recurrence_self(x, a, delta, tau, W), a) <= TOL_ARITH32


@pytest.mark.parametrize("exact", [False, True])
def test_self_fp32_ties_and_exact(cuda, exact):
    x, _, a = inputs.with_ties(9000, 9000, seed=24, n_distinct=50)
    n, tau, W, En = soe_cf.plan_soe(1e-6)
    plan = fgt.Plan(1e-2, soe=(tau, W), precision="fp32", exact_self=exact)
    u = _self(plan, x, a, cuda)
    assert rel_inf(u, oracle.recurrence_self(x, a, 1e-2, tau, W, exact_self=exact), a) <= TOL_ARITH32


def test_self_fp32_vs_direct(cuda):
    """FP32 identical points against the direct Gauss sum at 2 eps + 5e-6 (Chebyshev
    points, presorted: the sort is one merge)."""
    x, a = inputs.chebyshev(40000, seed=5)
    plan = fgt.Plan(1e-3, 1e-6, precision="fp32")
    u = _self(plan, x, a, cuda)
    idx = np.arange(0, 40000, 997)
    assert rel_inf(u[idx], oracle.direct(x[idx], x, a, 1e-3), a) <= 2e-6 + 5e-6


def test_self_unsupported_plans(cuda):
    x = torch.rand(100, dtype=torch.float64, device=cuda)
    for plan in (fgt.Plan(1e-3, 1e-6, precision="f32x2"),):
        with pytest.raises(_lib.FGTError) as e:
            fgt.transform_self(plan, x, x)
        assert e.value.code == _lib.FGT1D_EUNSUPPORTED
