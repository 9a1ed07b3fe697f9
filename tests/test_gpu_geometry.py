"""Fixed geometry (Sec. 5: pre-sorted points and a stored exponential table reused for
many strength vectors): fgt1d_geometry_bind / fgt1d_geometry_apply against the oracle,
against the plain transform, and the guards on a mismatched or unbound workspace."""
import ctypes

import numpy as np
import pytest
import torch

import paper_1909_09825_gb300 as fgt
from oracle import oracle, soe_cf
from paper_1909_09825_gb300 import _lib, inputs

from gpu_util import gpu_transform, rel_inf

pytestmark = pytest.mark.gpu

TOL_ARITH64 = 1e-12


def _t(v, dev):
    return torch.from_numpy(np.ascontiguousarray(v)).to(dev)


# double-float: 2^-48 instead of 2^-53; FP32: the 5e-6 arithmetic budget of the FP32 path
TOL = {"fp64": TOL_ARITH64, "f32x2": 32 * TOL_ARITH64, "fp32": 5e-6}
EPS = {"fp64": 1e-10, "f32x2": 1e-10, "fp32": 1e-6}


@pytest.mark.parametrize("prec", ["fp64", "f32x2", "fp32"])
@pytest.mark.parametrize("M,N,delta", [(1, 1, 1e-3), (33, 65, 1e-2), (4097, 3000, 1e-3), (30001, 29999, 1e-5)])
def test_apply_many_alphas_vs_recurrence(cuda, M, N, delta, prec):
    x, y, a0 = inputs.uniform(M, N, seed=M + 3 * N)
    n, tau, W, En = soe_cf.plan_soe(EPS[prec])
    plan = fgt.Plan(delta, soe=(tau, W), precision=prec)
    g = fgt.Geometry(plan, _t(x, cuda), _t(y, cuda))
    rng = np.random.default_rng(5)
    for rep in range(3):
        a = a0 if rep == 0 else rng.standard_normal(N)
        u = g.apply(_t(a, cuda)).cpu().numpy()
        ref = oracle.recurrence(x, y, a, delta, tau, W)
        assert rel_inf(u, ref, a) <= TOL[prec], rep


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_apply_equals_transform(cuda, prec):
    x, y, a = inputs.mixture(50000, 40000, seed=7)
    plan = fgt.Plan(1e-4, 1e-8 if prec == "fp64" else 1e-6, precision=prec)
    g = fgt.Geometry(plan, _t(x, cuda), _t(y, cuda))
    u = g.apply(_t(a, cuda)).cpu().numpy()
    # FP32: the same sweeps over the same sorted points; only the look-back order differs
    assert rel_inf(u, gpu_transform(plan, x, y, a), a) <= TOL[prec]


def test_apply_fp32_vs_direct(cuda):
    """The FP32 apply against the direct Gauss sum at the FP32 path's bound 2 eps + 5e-6,
    for several strength vectors on one bound mixture geometry."""
    x, y, a0 = inputs.mixture(40000, 30000, seed=21)
    plan = fgt.Plan(1e-4, 1e-6, precision="fp32")
    g = fgt.Geometry(plan, _t(x, cuda), _t(y, cuda))
    rng = np.random.default_rng(22)
    idx = rng.choice(len(x), 200, replace=False)
    for rep in range(3):
        a = a0 if rep == 0 else rng.uniform(-1, 1, len(y))
        u = g.apply(_t(a, cuda)).cpu().numpy()
        ref = oracle.direct(x[idx], y, a, 1e-4)
        assert np.max(np.abs(u[idx] - ref)) / np.abs(a).sum() <= 2 * 1e-6 + 5e-6, rep


@pytest.mark.parametrize("prec", ["fp64", "f32x2", "fp32"])
def test_apply_ties_and_exact_self(cuda, prec):
    x, y, a = inputs.with_ties(6000, 5000, seed=12, n_distinct=300)
    delta = 1e-3
    n, tau, W, En = soe_cf.plan_soe(EPS[prec] if prec == "fp32" else 1e-8)
    for exact in (False, True):
        plan = fgt.Plan(delta, soe=(tau, W), exact_self=exact, precision=prec)
        g = fgt.Geometry(plan, _t(x, cuda), _t(y, cuda))
        u = g.apply(_t(a, cuda)).cpu().numpy()
        ref = oracle.recurrence(x, y, a, delta, tau, W, exact_self=exact)
        assert rel_inf(u, ref, a) <= TOL[prec]


@pytest.mark.parametrize("tile", [128, 256])
def test_apply_tile_shapes(cuda, tile):
    """The table is laid out for the plan's tile shape; changing the shape after the
    bind is caught by the geometry tag."""
    x, y, a = inputs.uniform(20000, 15000, seed=9)
    n, tau, W, En = soe_cf.plan_soe(1e-8)
    plan = fgt.Plan(1e-4, soe=(tau, W))
    plan.tile_threads = tile
    g = fgt.Geometry(plan, _t(x, cuda), _t(y, cuda))
    u = g.apply(_t(a, cuda)).cpu().numpy()
    assert rel_inf(u, oracle.recurrence(x, y, a, 1e-4, tau, W), a) <= TOL_ARITH64
    plan.tile_threads = 384 - tile
    with pytest.raises(_lib.FGTError) as e:
        g.apply(_t(a, cuda))
    assert e.value.code == _lib.FGT1D_EINVAL


def test_apply_guards(cuda):
    x, y, a = inputs.uniform(3000, 2000, seed=1)
    plan = fgt.Plan(1e-3, 1e-6)
    g = fgt.Geometry(plan, _t(x, cuda), _t(y, cuda))
    A = _t(a, cuda)
    u_ok = g.apply(A).cpu().numpy()
    # another plan (other delta) on the bound workspace: nothing runs, EINVAL at the check
    other = fgt.Plan(2e-3, 1e-6)
    out = torch.zeros(3000, dtype=torch.float64, device=cuda)
    st = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    ws = ctypes.c_void_p(g.ws.data_ptr())
    assert _lib.lib().fgt1d_geometry_apply(other.handle, 3000, 2000, ctypes.c_void_p(A.data_ptr()),
                                           ctypes.c_void_p(out.data_ptr()), ws, g.ws.numel(), st) == 0
    assert _lib.lib().fgt1d_check(ws, g.ws.numel(), st) == _lib.FGT1D_EINVAL
    # an unbound (zeroed) workspace of the right size
    fresh = torch.zeros_like(g.ws)
    wf = ctypes.c_void_p(fresh.data_ptr())
    assert _lib.lib().fgt1d_geometry_apply(plan.handle, 3000, 2000, ctypes.c_void_p(A.data_ptr()),
                                           ctypes.c_void_p(out.data_ptr()), wf, fresh.numel(), st) == 0
    assert _lib.lib().fgt1d_check(wf, fresh.numel(), st) == _lib.FGT1D_EINVAL
    # binding again restores the geometry
    g2 = fgt.Geometry(plan, _t(x, cuda), _t(y, cuda))
    assert rel_inf(g2.apply(A).cpu().numpy(), u_ok, a) <= TOL_ARITH64
    # the precision is part of the tag: an f32x2 plan on an FP64-bound workspace
    dfp = fgt.Plan(1e-3, 1e-6, precision="f32x2")
    assert _lib.lib().fgt1d_geometry_apply(dfp.handle, 3000, 2000, ctypes.c_void_p(A.data_ptr()),
                                           ctypes.c_void_p(out.data_ptr()), ctypes.c_void_p(g2.ws.data_ptr()),
                                           g2.ws.numel(), st) == 0
    assert _lib.lib().fgt1d_check(ctypes.c_void_p(g2.ws.data_ptr()), g2.ws.numel(), st) == _lib.FGT1D_EINVAL
    # and an FP32 plan (no table) on it too
    p32 = fgt.Plan(1e-3, 1e-6, precision="fp32")
    assert _lib.lib().fgt1d_geometry_apply(p32.handle, 3000, 2000, ctypes.c_void_p(A.data_ptr()),
                                           ctypes.c_void_p(out.data_ptr()), ctypes.c_void_p(g2.ws.data_ptr()),
                                           g2.ws.numel(), st) == 0
    assert _lib.lib().fgt1d_check(ctypes.c_void_p(g2.ws.data_ptr()), g2.ws.numel(), st) == _lib.FGT1D_EINVAL
