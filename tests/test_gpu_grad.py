"""GPU gradients (fgt1d_backward through the C ABI) against the oracle's direct-sum
gradients of the SOE operator, against the Gaussian's direct-sum gradients within the
derivative error of the SOE, and against central finite differences of the GPU
transform itself."""
import numpy as np
import pytest
import torch

import paper_1909_09825_gb300 as fgt
from oracle import oracle, soe_cf
from paper_1909_09825_gb300 import inputs

pytestmark = pytest.mark.gpu


def _dev(a, d):
    return torch.from_numpy(np.ascontiguousarray(a)).to(d)


@pytest.mark.parametrize("M,N,delta", [(300, 200, 1e-2), (2000, 2000, 1e-3), (5000, 3000, 1e-4)])
@pytest.mark.parametrize("prec", ["fp64", "fp32", "f32x2"])
def test_backward_vs_oracle_soe_gradients(cuda, M, N, delta, prec):
    """The adjoint of the implemented SOE operator, term by term (same nodes)."""
    x, y, a = inputs.uniform(M, N, seed=M + N)
    g = np.random.default_rng(1).standard_normal(M)
    n, tau, W, En = soe_cf.plan_soe(1e-6 if prec == "fp32" else 1e-8)
    plan = fgt.Plan(delta, soe=(tau, W), precision=prec)
    gx, gy, ga, gd = [t.cpu().numpy() for t in fgt.backward(plan, _dev(x, cuda), _dev(y, cuda), _dev(a, cuda),
                                                            _dev(g, cuda))]
    rx, ry, ra, rd = oracle.grad_soe(x, y, a, delta, tau, W, g)
    s = 1.0 / np.sqrt(delta)
    kappa = np.abs(tau).max() * s
    tol = 2e-5 if prec == "fp32" else 1e-11
    scale = np.abs(g).sum() * np.abs(a).sum() / max(M, N)
    assert np.max(np.abs(ga - ra)) <= tol * np.abs(g).sum()
    assert np.max(np.abs(gx - rx)) <= tol * kappa * np.abs(g).max() * np.abs(a).sum()
    assert np.max(np.abs(gy - ry)) <= tol * kappa * np.abs(a).max() * np.abs(g).sum()
    # dL/ddelta is assembled from -(1/(2 delta)) (sum (x-c) dL/dx + sum (y-c) dL/dy): each
    # term carries the relative error of the x / y gradients
    mag = (np.abs(x - x[0]) @ np.abs(rx) + np.abs(y - x[0]) @ np.abs(ry)) / (2 * delta)
    assert abs(gd[0] - rd) <= tol * (1 + kappa) * mag


def test_backward_tile_shapes_agree(cuda):
    x, y, a = inputs.uniform(3000, 2500, seed=5)
    g = np.random.default_rng(2).standard_normal(3000)
    out = []
    for tile in (128, 256):
        plan = fgt.Plan(1e-3, 1e-8)
        plan.tile_threads = tile
        out.append([t.cpu().numpy() for t in fgt.backward(plan, _dev(x, cuda), _dev(y, cuda), _dev(a, cuda),
                                                          _dev(g, cuda))])
    for r0, r1 in zip(*out):
        assert np.max(np.abs(r0 - r1)) <= 1e-11 * max(1.0, np.max(np.abs(r0)))


def test_backward_vs_gaussian_direct(cuda):
    """M = N = 2000, delta = 1e-3, eps = 1e-8: dL/dalpha within eps sum|g| of the
    Gaussian's; dL/dx, dL/dy, dL/ddelta within the derivative error of the SOE
    (max |G' - S'| over the E_n grid, times the strengths), measured here."""
    x, y, a = inputs.uniform(2000, 2000, seed=3)
    g = np.sin(2 * np.pi * x)
    delta, eps = 1e-3, 1e-8
    plan = fgt.Plan(delta, eps)
    gx, gy, ga, gd = [t.cpu().numpy() for t in fgt.backward(plan, _dev(x, cuda), _dev(y, cuda), _dev(a, cuda),
                                                            _dev(g, cuda))]
    rx, ry, ra, rd = oracle.grad_direct(x, y, a, delta, g)
    t = np.linspace(1e-9, 12, 400001)
    sp = np.zeros_like(t)
    for tk, wk in zip(plan.tau, plan.W):
        sp += (wk * (-tk) * np.exp(-tk * t)).real
    dErr = np.max(np.abs(-t / 2 * np.exp(-t * t / 4) - sp)) / np.sqrt(delta)  # max |G' - S'|
    assert np.max(np.abs(ga - ra)) <= 2 * eps * np.abs(g).sum()
    assert np.max(np.abs(gx - rx)) <= 1.01 * dErr * np.abs(g).max() * np.abs(a).sum()
    assert np.max(np.abs(gy - ry)) <= 1.01 * dErr * np.abs(a).max() * np.abs(g).sum()


def test_autograd_finite_differences(cuda):
    """torch.autograd through GaussTransform vs central differences of the GPU forward."""
    x, y, a = inputs.uniform(400, 300, seed=7)
    f = np.sin(2 * np.pi * x)
    delta = 2e-3
    X = _dev(x, cuda).requires_grad_(True)
    Y = _dev(y, cuda).requires_grad_(True)
    A = _dev(a, cuda).requires_grad_(True)
    D = torch.tensor(delta, dtype=torch.float64, requires_grad=True)
    F = _dev(f, cuda)
    plan = fgt.Plan(delta, 1e-10)
    u = fgt.GaussTransform.apply(X, Y, A, D, plan)
    loss = ((u - F) ** 2).sum()
    loss.backward()

    def L(xx, yy, aa, dd):
        p = plan if dd == delta else fgt.Plan(dd, 1e-10)
        uu = fgt.transform(p, _dev(xx, cuda), _dev(yy, cuda), _dev(aa, cuda)).cpu().numpy()
        return np.sum((uu - f) ** 2)

    rng = np.random.default_rng(0)
    h = 1e-6
    for arr, grad in ((x, X.grad), (y, Y.grad), (a, A.grad)):
        for i in rng.choice(len(arr), 5, replace=False):
            ap, am = arr.copy(), arr.copy()
            ap[i] += h
            am[i] -= h
            args_p = [ap if arr is v else v for v in (x, y, a)]
            args_m = [am if arr is v else v for v in (x, y, a)]
            fd = (L(*args_p, delta) - L(*args_m, delta)) / (2 * h)
            assert abs(grad[i].item() - fd) <= 1e-5 * max(1.0, abs(fd)), (i, grad[i].item(), fd)
    hd = 1e-9
    fd = (L(x, y, a, delta + hd) - L(x, y, a, delta - hd)) / (2 * hd)
    # plans at delta +- hd share the SOE nodes, so the difference quotient sees the same operator
    assert abs(D.grad.item() - fd) <= 1e-4 * abs(fd)


def test_backward_edge_cases(cuda):
    plan = fgt.Plan(1e-3, 1e-6)
    x = torch.rand(50, dtype=torch.float64, device=cuda)
    e = torch.empty(0, dtype=torch.float64, device=cuda)
    g = torch.ones(50, dtype=torch.float64, device=cuda)
    gx, gy, ga, gd = fgt.backward(plan, x, e, e, g)
    assert torch.all(gx == 0) and gy.numel() == 0 and ga.numel() == 0 and gd.item() == 0
    # coincident points: dL/dx uses S'(0) = 0 for the coincident pair
    xs = np.array([0.3, 0.5])
    ys = np.array([0.3, 0.7])
    al = np.array([1.0, 2.0])
    gg = np.array([1.0, 1.0])
    gx, gy, ga, gd = [t.cpu().numpy() for t in fgt.backward(plan, _dev(xs, cuda), _dev(ys, cuda), _dev(al, cuda),
                                                            _dev(gg, cuda))]
    rx, ry, ra, rd = oracle.grad_soe(xs, ys, al, 1e-3, plan.tau, plan.W, gg)
    assert np.allclose(gx, rx, rtol=1e-10, atol=1e-12) and np.allclose(gy, ry, rtol=1e-10, atol=1e-12)
    assert np.allclose(ga, ra, rtol=1e-12, atol=1e-14)


@pytest.mark.parametrize("prec", ["fp64", "fp32", "f32x2"])
@pytest.mark.parametrize("want", [(True, True, True, True), (True, True, False, False), (True, False, True, False),
                                  (False, True, True, False), (False, False, True, True)])
def test_backward_coincident_points(cuda, prec, want):
    """Coordinates on a grid of 400 values: long runs of coincident targets and sources
    (the second transform of the adjoint keeps the first one's sorted order, targets
    before sources on a tie), every subset of the gradients, against the oracle's SOE
    gradients (S'(0) = 0 for a coincident pair)."""
    M, N, delta = 6000, 5000, 1e-3
    x, y, a = inputs.uniform(M, N, seed=61)
    x, y = np.round(x * 400) / 400, np.round(y * 400) / 400
    g = np.random.default_rng(62).standard_normal(M)
    n, tau, W, En = soe_cf.plan_soe(1e-6 if prec == "fp32" else 1e-8)
    plan = fgt.Plan(delta, soe=(tau, W), precision=prec)
    out = [t.cpu().numpy() if t is not None else None
           for t in fgt.backward(plan, _dev(x, cuda), _dev(y, cuda), _dev(a, cuda), _dev(g, cuda), want=want)]
    ref = oracle.grad_soe(x, y, a, delta, tau, W, g)
    kappa = np.abs(tau).max() / np.sqrt(delta)
    tol = 2e-5 if prec == "fp32" else 1e-11
    scales = [tol * kappa * np.abs(g).max() * np.abs(a).sum(), tol * kappa * np.abs(a).max() * np.abs(g).sum(),
              tol * np.abs(g).sum(), None]
    for w, o, r, sc in zip(want, out, ref, scales):
        assert (o is None) == (not w)
        if w and sc is not None:
            assert np.max(np.abs(o - r)) <= sc
    if want[3]:
        mag = (np.abs(x - x[0]) @ np.abs(ref[0]) + np.abs(y - x[0]) @ np.abs(ref[1])) / (2 * delta)
        assert abs(out[3][0] - ref[3]) <= tol * (1 + kappa) * mag
