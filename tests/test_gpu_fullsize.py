"""Parity at the benchmark's full size (M = N = 2^26, the launch configuration that
bench.py times): sampled targets checked one by one against the oracle's direct sum
over all 2^26 sources."""
import numpy as np
import pytest
import torch

import paper_1909_09825_gb300 as fgt
from oracle import oracle
from paper_1909_09825_gb300 import inputs

pytestmark = pytest.mark.gpu

M = N = 1 << 26


@pytest.fixture(scope="module")
def data(cuda):
    x, y, a = inputs.uniform(M, N, seed=0)
    dev = cuda
    return x, y, a, torch.from_numpy(x).to(dev), torch.from_numpy(y).to(dev), torch.from_numpy(a).to(dev)


@pytest.mark.parametrize("delta,eps,prec", [(1e-5, 1e-6, "fp64"), (1e-5, 1e-10, "fp64"), (1e-2, 1e-6, "fp64"),
                                            (1e-5, 1e-6, "fp32"), (1e-5, 1e-10, "f32x2")])
def test_fullsize_sampled(data, delta, eps, prec):
    x, y, a, X, Y, A = data
    plan = fgt.Plan(delta, eps, precision=prec)
    u = fgt.transform(plan, X, Y, A)
    rng = np.random.default_rng(17)
    idx = np.concatenate([[0, M - 1, int(np.argmin(x)), int(np.argmax(x))], rng.choice(M, 12, replace=False)])
    ug = u[torch.from_numpy(idx).to(u.device)].cpu().numpy()
    ref = oracle.direct(x[idx], y, a, delta, nthreads=0)
    tol = 2 * eps + (5e-6 if prec == "fp32" else 1e-13)
    assert np.max(np.abs(ug - ref)) / np.abs(a).sum() <= tol
    del u
    torch.cuda.empty_cache()
