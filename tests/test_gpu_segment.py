"""Range-partitioned transform on the GPU: fgt1d_segment_execute / _compose / _apply
through the C ABI, one segment after another in one process, and the torch.distributed
driver with two gloo ranks sharing cuda:0 (their kernels never wait on each other: the
exchange is on the host).  Against the oracle's recurrence over all points, and each
segment's boundary record against the oracle's direct sums."""
import os
import socket

import numpy as np
import pytest
import torch
import torch.multiprocessing as mp

import paper_1909_09825_gb300 as fgt
from oracle import oracle, soe_cf
from paper_1909_09825_gb300 import inputs
from paper_1909_09825_gb300.partition import DeviceSegments

pytestmark = pytest.mark.gpu


def _segments(x, y, cuts):
    """Index sets of the segments [cuts[g], cuts[g+1]) of the line (last one closed)."""
    out = []
    for g in range(len(cuts) - 1):
        lo, hi = cuts[g], cuts[g + 1]
        last = g == len(cuts) - 2
        sx = np.nonzero((x >= lo) & ((x <= hi) if last else (x < hi)))[0]
        sy = np.nonzero((y >= lo) & ((y <= hi) if last else (y < hi)))[0]
        out.append((sx, sy))
    return out


@pytest.mark.parametrize("prec,eps,delta,ties", [("fp64", 1e-10, 1e-5, False), ("fp64", 1e-6, 1e-2, True),
                                                 ("fp32", 1e-6, 1e-3, False), ("f32x2", 1e-10, 1e-4, False)])
def test_segments_equal_whole_transform(cuda, prec, eps, delta, ties):
    M, N = 150000, 120000
    x, y, a = inputs.uniform(M, N, seed=41)
    if ties:
        x, y = np.round(x * 2000) / 2000, np.round(y * 2000) / 2000
    _, tau, W, _ = soe_cf.plan_soe(eps)
    plan = fgt.Plan(delta, soe=(tau, W), precision=prec)
    # five segments: one without points, one with sources only, cuts on tied values
    cuts = [0.0, 0.3, 0.3, 0.45, 0.455, 1.0]
    segs = _segments(x, y, cuts)
    sx3 = segs[3][0]
    segs[3] = (sx3[:0], segs[3][1])  # segment 3: its targets dropped (sources only)
    keep = np.setdiff1d(np.arange(M), sx3)
    recs, runs = [], []
    for sx, sy in segs:
        d = DeviceSegments(plan)
        X, Y, A = (torch.from_numpy(np.ascontiguousarray(v)).to(cuda) for v in (x[sx], y[sy], a[sy]))
        u, b = d.execute(X, Y, A)
        bh = b.cpu().numpy()
        ob = oracle.segment_boundary(x[sx], y[sy], a[sy], delta, tau, W)
        n = len(tau)
        if len(sx) + len(sy):
            # the record carries the precision of the plan's in-tile recurrences
            tol_b = {"fp64": 1e-12, "f32x2": 32e-12, "fp32": 5e-6}[prec]
            assert np.allclose(bh[:4 * n], ob[:4 * n], rtol=0, atol=tol_b * max(np.abs(a[sy]).sum(), 1.0))
            assert bh[4 * n] == ob[4 * n] and bh[4 * n + 1] == ob[4 * n + 1]
        else:
            assert np.all(bh[:4 * n] == 0) and np.isnan(bh[4 * n]) and np.isnan(bh[4 * n + 1])
        recs.append(bh)
        runs.append((d, u, sx))
    recs = np.stack(recs)
    ug = np.full(M, np.nan)
    for g, (d, u, sx) in enumerate(runs):
        u = d.apply(d.compose(recs, g), u)
        ug[sx] = u.cpu().numpy()
    ref = oracle.recurrence(x[keep], y, a, delta, tau, W)
    err = np.max(np.abs(ug[keep] - ref)) / np.abs(a).sum()
    assert err <= (5e-6 if prec == "fp32" else 1e-12), err


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _rank(rank, world, port, q):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        from paper_1909_09825_gb300.partition import transform_partitioned
        dev = torch.device("cuda:0")
        M, N = 200000, 160000
        x, y, a = inputs.uniform(M, N, seed=43)
        _, tau, W, _ = soe_cf.plan_soe(1e-10)
        plan = fgt.Plan(1e-4, soe=(tau, W))
        xs, ys, as_ = (torch.from_numpy(v[rank::world].copy()).to(dev) for v in (x, y, a))
        u = transform_partitioned(plan, xs, ys, as_).cpu().numpy()
        ref = oracle.recurrence(x, y, a, 1e-4, tau, W)[rank::world]
        q.put((rank, float(np.max(np.abs(u - ref)) / np.abs(a).sum())))
    except Exception as e:
        q.put((rank, repr(e)))
    finally:
        dist.destroy_process_group()


def test_partitioned_two_ranks_gloo(cuda):
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = dict(q.get(timeout=600) for _ in procs)
    for p in procs:
        p.join(timeout=120)
    for r in range(2):
        assert isinstance(res[r], float), res[r]
        assert res[r] <= 1e-12, (r, res[r])
