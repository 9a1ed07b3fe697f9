"""fgt1d_execute_noalloc, the entry point for callers that cannot allocate device memory
(its scratch is a fixed array inside the library), called through the C ABI and
checked against fgt1d_execute on two calls in a row.  Kept in a file collected last so
that a run stopping at the first failure has run every other test first."""
import ctypes

import numpy as np
import pytest
import torch

import paper_1909_09825_gb300 as fgt
from paper_1909_09825_gb300 import _lib, inputs

pytestmark = pytest.mark.gpu


def _noalloc(plan, X, Y, A, out):
    stream = torch.cuda.current_stream()
    rc = _lib.lib().fgt1d_execute_noalloc(plan.handle, ctypes.c_void_p(X.data_ptr()), X.numel(),
                                          ctypes.c_void_p(Y.data_ptr()), ctypes.c_void_p(A.data_ptr()), Y.numel(),
                                          ctypes.c_void_p(out.data_ptr()), ctypes.c_void_p(stream.cuda_stream))
    torch.cuda.synchronize()
    return rc


@pytest.mark.parametrize("precision,eps,tol", [("fp64", 1e-10, 1e-12), ("fp32", 1e-6, 5e-6)])
def test_noalloc_matches_execute_twice(cuda, precision, eps, tol):
    M, N = 40000, 25536  # M + N = 65,536, the documented maximum
    x, y, a = inputs.uniform(M, N, seed=31)
    X, Y, A = (torch.from_numpy(v).to(cuda) for v in (x, y, a))
    plan = fgt.Plan(1e-4, eps, precision=precision)
    ref = fgt.transform(plan, X, Y, A).cpu().numpy()
    s = np.abs(a).sum()
    for _ in range(2):
        out = torch.full((M,), np.nan, dtype=torch.float64, device=cuda)
        assert _noalloc(plan, X, Y, A, out) == _lib.FGT1D_OK
        u = out.cpu().numpy()
        assert np.max(np.abs(u - ref)) / s <= tol


def test_noalloc_rejects_oversize(cuda):
    plan = fgt.Plan(1e-4, 1e-10)
    X = torch.rand(50000, dtype=torch.float64, device=cuda)
    Y = torch.rand(20000, dtype=torch.float64, device=cuda)
    A = torch.ones(20000, dtype=torch.float64, device=cuda)
    out = torch.empty(50000, dtype=torch.float64, device=cuda)
    assert _noalloc(plan, X, Y, A, out) == _lib.FGT1D_ETOOLARGE
