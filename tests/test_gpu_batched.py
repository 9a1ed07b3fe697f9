"""Batched transforms (fgt1d_execute_batched): many independent items of uneven size
and bandwidth in one pass, checked item by item against the oracle, against the single
transform, under CUDA-graph replay, and with bad items."""
import numpy as np
import pytest
import torch

import paper_1909_09825_gb300 as fgt
from oracle import oracle, soe_cf
from paper_1909_09825_gb300 import _lib, inputs

pytestmark = pytest.mark.gpu

TOL_ARITH64 = 1e-12


def _batch(sizes_x, sizes_y, deltas, seed):
    rng = np.random.default_rng(seed)
    x_off = np.concatenate([[0], np.cumsum(sizes_x)]).astype(np.int64)
    y_off = np.concatenate([[0], np.cumsum(sizes_y)]).astype(np.int64)
    x = rng.random(int(x_off[-1]))
    y = rng.random(int(y_off[-1]))
    a = rng.standard_normal(int(y_off[-1]))
    return x_off, y_off, np.asarray(deltas, dtype=np.float64), x, y, a


def _run(plan, b, dev, with_delta=True):
    x_off, y_off, d, x, y, a = b
    T = lambda v: torch.from_numpy(np.ascontiguousarray(v)).to(dev)
    return fgt.transform_batched(plan, T(x_off), T(y_off), T(x), T(y), T(a), delta=T(d) if with_delta else None
                                 ).cpu().numpy()


def test_batched_items_vs_oracle(cuda):
    rng = np.random.default_rng(0)
    B = 60
    sx = rng.integers(0, 3000, B)
    sy = rng.integers(0, 3000, B)
    sx[3] = 0          # no targets
    sy[5] = 0          # no sources
    sx[7] = sy[7] = 0  # empty item
    sx[11], sy[11] = 4096, 4096 - 17
    deltas = 10.0 ** rng.uniform(-6, -1, B)
    b = _batch(sx, sy, deltas, 1)
    n, tau, W, En = soe_cf.plan_soe(1e-8)
    plan = fgt.Plan(1.0, soe=(tau, W))
    u = _run(plan, b, cuda)
    x_off, y_off, d, x, y, a = b
    for i in range(B):
        xs, ys, al = x[x_off[i]:x_off[i + 1]], y[y_off[i]:y_off[i + 1]], a[y_off[i]:y_off[i + 1]]
        ui = u[x_off[i]:x_off[i + 1]]
        if len(xs) == 0:
            continue
        if len(ys) == 0:
            assert np.all(ui == 0)
            continue
        ref = oracle.recurrence(xs, ys, al, d[i], tau, W)
        assert np.max(np.abs(ui - ref)) / np.abs(al).sum() <= TOL_ARITH64, i


def test_batched_equals_single(cuda):
    rng = np.random.default_rng(2)
    B = 24
    sx = rng.integers(1, 20000, B)
    sy = rng.integers(1, 20000, B)
    deltas = 10.0 ** rng.uniform(-5, -2, B)
    b = _batch(sx, sy, deltas, 3)
    plan = fgt.Plan(1.0, 1e-10)
    u = _run(plan, b, cuda)
    x_off, y_off, d, x, y, a = b
    for i in range(B):
        p = fgt.Plan(d[i], 1e-10)
        T = lambda v: torch.from_numpy(np.ascontiguousarray(v)).to(cuda)
        ref = fgt.transform(p, T(x[x_off[i]:x_off[i + 1]]), T(y[y_off[i]:y_off[i + 1]]),
                            T(a[y_off[i]:y_off[i + 1]])).cpu().numpy()
        ui = u[x_off[i]:x_off[i + 1]]
        assert np.max(np.abs(ui - ref)) / np.abs(a[y_off[i]:y_off[i + 1]]).sum() <= TOL_ARITH64, i


@pytest.mark.parametrize("prec,eps", [("fp64", 1e-6), ("fp32", 1e-6), ("f32x2", 1e-10)])
def test_batched_uneven_vs_direct(cuda, prec, eps):
    """Sizes log-uniform in [1e2, 1e5], bandwidths log-uniform in [1e-6, 1e-1]: sampled
    targets of every item against the direct Gauss sum."""
    sizes, deltas = inputs.batched_sizes(200, seed=4, lo=1e2, hi=1e5)
    b = _batch(sizes, sizes, deltas, 5)
    plan = fgt.Plan(1.0, eps, precision=prec)
    u = _run(plan, b, cuda)
    x_off, y_off, d, x, y, a = b
    rng = np.random.default_rng(6)
    tol = 2 * eps + (5e-6 if prec == "fp32" else 1e-13)
    for i in range(len(sizes)):
        xs, ys, al = x[x_off[i]:x_off[i + 1]], y[y_off[i]:y_off[i + 1]], a[y_off[i]:y_off[i + 1]]
        idx = rng.choice(len(xs), min(len(xs), 8), replace=False)
        ref = oracle.direct(xs[idx], ys, al, d[i])
        assert np.max(np.abs(u[x_off[i] + idx] - ref)) / np.abs(al).sum() <= tol, i


def test_batched_plan_delta_default(cuda):
    b = _batch([500, 700], [600, 400], [1e-3, 1e-3], 7)
    plan = fgt.Plan(1e-3, 1e-8)
    u1 = _run(plan, b, cuda, with_delta=True)
    u2 = _run(plan, b, cuda, with_delta=False)
    assert np.max(np.abs(u1 - u2)) <= 1e-12 * np.abs(b[5]).sum()


def test_batched_cuda_graph_replay(cuda):
    """Capture once, replay with new data and bandwidths written into the same buffers."""
    rng = np.random.default_rng(8)
    B = 40
    sx = rng.integers(100, 5000, B)
    sy = rng.integers(100, 5000, B)
    b = _batch(sx, sy, 10.0 ** rng.uniform(-5, -2, B), 9)
    x_off, y_off, d, x, y, a = b
    T = lambda v: torch.from_numpy(np.ascontiguousarray(v)).to(cuda)
    X, Y, A, D, XO, YO = T(x), T(y), T(a), T(d), T(x_off), T(y_off)
    plan = fgt.Plan(1.0, 1e-8)
    ws = fgt.Workspace(cuda)
    out = torch.empty_like(X)
    fgt.transform_batched(plan, XO, YO, X, Y, A, delta=D, out=out, workspace=ws)  # warm-up: sizes the workspace
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    g = torch.cuda.CUDAGraph()
    with torch.cuda.stream(s):
        with torch.cuda.graph(g, stream=s):
            fgt.transform_batched(plan, XO, YO, X, Y, A, delta=D, out=out, workspace=ws, stream=s, sync_check=False)
    torch.cuda.current_stream().wait_stream(s)
    for rep in range(2):
        x2 = np.random.default_rng(100 + rep).random(len(x))
        d2 = 10.0 ** np.random.default_rng(200 + rep).uniform(-5, -2, B)
        X.copy_(T(x2))
        D.copy_(T(d2))
        g.replay()
        torch.cuda.synchronize()
        ref = fgt.transform_batched(plan, XO, YO, X, Y, A, delta=D).cpu().numpy()
        assert np.max(np.abs(out.cpu().numpy() - ref)) <= 1e-12 * np.abs(a).sum()


def test_batched_autotune(cuda):
    rng = np.random.default_rng(12)
    B = 64
    sx = rng.integers(100, 20000, B)
    b = _batch(sx, sx, 10.0 ** rng.uniform(-5, -2, B), 13)
    x_off, y_off, d, x, y, a = b
    T = lambda v: torch.from_numpy(np.ascontiguousarray(v)).to(cuda)
    plan = fgt.Plan(1.0, 1e-8)
    res = plan.autotune_batched(T(x_off), T(y_off), T(x), T(y), T(a), delta=T(d), reps=2)
    assert res["chosen"] in (128, 256) and plan.tile_threads == res["chosen"]
    u = _run(plan, b, cuda)
    plan.tile_threads = 384 - res["chosen"]  # the other shape
    u2 = _run(plan, b, cuda)
    assert np.max(np.abs(u - u2)) <= TOL_ARITH64 * np.abs(a).sum()


def test_batched_bad_items(cuda):
    plan = fgt.Plan(1e-3, 1e-6)
    b = _batch([100, 200], [150, 50], [1e-3, -1.0], 10)  # second item: negative delta
    with pytest.raises(_lib.FGTError) as e:
        _run(plan, b, cuda)
    assert e.value.code == _lib.FGT1D_EINVAL
    x_off, y_off, d, x, y, a = b
    bad = (np.array([0, 250, 400]), y_off, np.array([1e-3, 1e-3]), x, y, a)  # offsets past M_total = 300
    with pytest.raises(_lib.FGTError) as e:
        _run(plan, bad, cuda)
    assert e.value.code == _lib.FGT1D_EINVAL


def test_batched_presorted_items(cuda):
    """Every item's sources and targets presorted: one merge for the whole batch."""
    rng = np.random.default_rng(20)
    B = 30
    sx = rng.integers(0, 9000, B)
    sy = rng.integers(0, 9000, B)
    x_off, y_off, d, x, y, a = _batch(sx, sy, 10.0 ** rng.uniform(-5, -2, B), 21)
    for i in range(B):
        x[x_off[i]:x_off[i + 1]] = np.sort(x[x_off[i]:x_off[i + 1]])
        y[y_off[i]:y_off[i + 1]] = np.sort(y[y_off[i]:y_off[i + 1]])
    n, tau, W, En = soe_cf.plan_soe(1e-8)
    plan = fgt.Plan(1.0, soe=(tau, W))
    u = _run(plan, (x_off, y_off, d, x, y, a), cuda)
    for i in range(B):
        xs, ys, al = x[x_off[i]:x_off[i + 1]], y[y_off[i]:y_off[i + 1]], a[y_off[i]:y_off[i + 1]]
        if len(xs) == 0 or len(ys) == 0:
            continue
        ref = oracle.recurrence(xs, ys, al, d[i], tau, W)
        assert np.max(np.abs(u[x_off[i]:x_off[i + 1]] - ref)) / np.abs(al).sum() <= TOL_ARITH64, i


@pytest.mark.parametrize("case", ["ranges", "fallback"])
def test_batched_items_with_their_own_sort_keys(cuda, case):
    """Every item sorts on 32-bit keys over its own coordinate range: items on shifted,
    scaled and negative ranges, one of subnormal coordinates, one holding ties across its
    sources and targets, and (case "fallback") one with 3000 distinct targets inside
    1e-13, which makes the whole batch take the full 64-bit sort.  Item by item against
    the oracle's recurrence."""
    rng = np.random.default_rng(31)
    items = [(rng.random(2500), rng.random(2000)),
             (5.0 + 1e-3 * rng.random(3000), 5.0 + 1e-3 * rng.random(2600)),
             (-7.0 * rng.random(1200), -7.0 * rng.random(1500) - 1e-6),
             (1e-310 * rng.random(800), 1e-310 * rng.random(900)),
             (np.round(rng.random(4000) * 300) / 300, np.round(rng.random(3500) * 300) / 300)]
    if case == "fallback":
        items.append((0.5 + 1e-13 * rng.random(3000), rng.random(2000)))
    sx = [len(p[0]) for p in items]
    sy = [len(p[1]) for p in items]
    x_off = np.concatenate([[0], np.cumsum(sx)]).astype(np.int64)
    y_off = np.concatenate([[0], np.cumsum(sy)]).astype(np.int64)
    x = np.concatenate([p[0] for p in items])
    y = np.concatenate([p[1] for p in items])
    a = rng.standard_normal(len(y))
    d = 10.0 ** rng.uniform(-6, -2, len(items))
    n, tau, W, En = soe_cf.plan_soe(1e-8)
    plan = fgt.Plan(1.0, soe=(tau, W))
    u = _run(plan, (x_off, y_off, d, x, y, a), cuda)
    for i in range(len(items)):
        xs, ys, al = x[x_off[i]:x_off[i + 1]], y[y_off[i]:y_off[i + 1]], a[y_off[i]:y_off[i + 1]]
        ref = oracle.recurrence(xs, ys, al, d[i], tau, W)
        assert np.max(np.abs(u[x_off[i]:x_off[i + 1]] - ref)) / np.abs(al).sum() <= TOL_ARITH64, i
