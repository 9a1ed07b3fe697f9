"""Bounded inter-block waits, tested without a GPU fault: the host makes one look-back
wait run out -- FGT1D_FAULT starts a tile counter at 1, so tile 0 never publishes -- under
a short bound (FGT1D_SPIN_LIMIT_CYCLES).  The kernels end, fgt1d_check reports
FGT1D_ETIMEOUT, and the next call on the same workspace is clean and correct.  After an
expired wait in the sort the sorted codes are not valid, so the sweeps skip their work
(every access stays in bounds); after one in a sweep only values are wrong."""
import time

import numpy as np
import pytest
import torch

import paper_1909_09825_gb300 as fgt
from oracle import oracle
from paper_1909_09825_gb300 import _lib, inputs

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("fault", ["sweep_timeout", "sort_timeout"])
def test_expired_wait_is_reported_and_the_next_call_is_clean(cuda, fault, monkeypatch):
    M, N = 20000, 17000  # 10 tiles of 4096 merged points
    delta, eps = 1e-3, 1e-6
    x, y, a = inputs.uniform(M, N, seed=71)
    X, Y, A = (torch.from_numpy(v).to(cuda) for v in (x, y, a))
    plan = fgt.Plan(delta, eps)
    ws = fgt.Workspace(cuda)
    monkeypatch.setenv("FGT1D_SPIN_LIMIT_CYCLES", "2000000")  # about 1 ms
    monkeypatch.setenv("FGT1D_FAULT", fault)
    t0 = time.perf_counter()
    with pytest.raises(_lib.FGTError) as err:
        fgt.transform(plan, X, Y, A, workspace=ws)
    assert err.value.code == _lib.FGT1D_ETIMEOUT
    assert time.perf_counter() - t0 < 30
    monkeypatch.delenv("FGT1D_FAULT")
    monkeypatch.delenv("FGT1D_SPIN_LIMIT_CYCLES")
    u = fgt.transform(plan, X, Y, A, workspace=ws).cpu().numpy()
    idx = np.random.default_rng(72).choice(M, 200, replace=False)
    ref = oracle.direct(x[idx], y, a, delta, nthreads=0)
    assert np.max(np.abs(u[idx] - ref)) / np.abs(a).sum() <= 2 * eps + 1e-13
