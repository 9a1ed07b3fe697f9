"""Range partition of one transform on CPU ranks (gloo): the library's host composition
of the segments' boundary states (fgt1d_segment_compose), the driver's routing and
exchange (paper_1909_09825_gb300.partition), and a rank that leaves before a step.

The segments' own transforms are the oracle's here (test-only stand-ins for
fgt1d_segment_execute / fgt1d_segment_apply, which need a GPU): the paper's recurrence
over the segment's points with zero entering states, its boundary states as direct
sums, and the entering states' contribution as direct exponentials.  Against the
oracle's recurrence over all points, within 1e-13 sum|alpha|."""
import os
import socket

import numpy as np
import pytest
import torch
import torch.multiprocessing as mp

from oracle import oracle, soe_cf

SEED = 5


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


class OracleSegments:
    """Test stand-in for DeviceSegments: the oracle on the segment's points; the
    composition is the library's (through DeviceSegments.compose, host only)."""

    def __init__(self, plan, tau, W):
        from paper_1909_09825_gb300.partition import DeviceSegments
        self.dev = DeviceSegments(plan)
        self.plan, self.tau, self.W = plan, tau, W

    def execute(self, x, y, a):
        x, y, a = (t.numpy() for t in (x, y, a))
        d = self.plan.delta
        if len(x) and len(y):
            u = oracle.recurrence(x, y, a, d, self.tau, self.W)
        else:
            u = np.zeros(len(x))
        self.x = x
        return torch.from_numpy(u), torch.from_numpy(oracle.segment_boundary(x, y, a, d, self.tau, self.W))

    def compose(self, boundaries, g):
        return self.dev.compose(boundaries, g)

    def apply(self, carry, u):
        return torch.from_numpy(oracle.carry_apply(self.x, u.numpy(), self.plan.delta, self.tau, self.W, carry))


def _data(M, N, ties):
    rng = np.random.default_rng(SEED)
    x, y, a = rng.random(M), rng.random(N), rng.standard_normal(N)
    if ties:  # equal coordinates across sources and targets, and across ranks' shares
        x, y = np.round(x * 300) / 300, np.round(y * 300) / 300
    return x, y, a


def _worker(rank, world, port, M, N, ties, delta, q):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        import paper_1909_09825_gb300 as fgt
        from paper_1909_09825_gb300.partition import transform_partitioned
        _, tau, W, _ = soe_cf.plan_soe(1e-10)
        plan = fgt.Plan(delta, soe=(tau, W))
        x, y, a = _data(M, N, ties)
        # this rank's share: every world-th point (so routing moves most of them)
        xs, ys, as_ = (torch.from_numpy(v[rank::world].copy()) for v in (x, y, a))
        u = transform_partitioned(plan, xs, ys, as_, segments=OracleSegments(plan, tau, W), samples=64)
        ref = oracle.recurrence(x, y, a, delta, tau, W)[rank::world]
        q.put((rank, float(np.max(np.abs(u.numpy() - ref)) / np.abs(a).sum()) if len(ref) else 0.0))
    except Exception as e:  # reported to the parent
        q.put((rank, repr(e)))
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("world,M,N,ties,delta", [(3, 2500, 3500, True, 1e-2), (4, 5, 1200, False, 1.0)])
def test_partitioned_equals_whole_transform(world, M, N, ties, delta):
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, world, port, M, N, ties, delta, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = dict(q.get(timeout=300) for _ in procs)
    for p in procs:
        p.join(timeout=60)
    for r in range(world):
        assert isinstance(res[r], float), res[r]
        assert res[r] <= 1e-13, (r, res[r])
    assert all(p.exitcode == 0 for p in procs)


def _leaver(rank, world, port, q):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    if rank == 1:  # leaves between steps: never enters the transform
        q.put((rank, "left"))
        q.close()
        q.join_thread()  # flush before the hard exit
        os._exit(0)
    try:
        import paper_1909_09825_gb300 as fgt
        from paper_1909_09825_gb300.partition import transform_partitioned
        _, tau, W, _ = soe_cf.plan_soe(1e-6)
        plan = fgt.Plan(1e-3, soe=(tau, W))
        x, y, a = _data(100, 100, False)
        try:
            transform_partitioned(plan, torch.from_numpy(x), torch.from_numpy(y), torch.from_numpy(a),
                                  segments=OracleSegments(plan, tau, W), health_timeout_s=3)
            q.put((rank, "no error"))
        except RuntimeError as e:
            q.put((rank, "detected: " + str(e)[:200]))
    finally:
        q.close()
        q.join_thread()
        os._exit(0)


def test_rank_leaving_is_detected_on_the_host():
    """A rank that leaves between steps is found by the host-side health check (a
    monitored barrier with a short limit) before any exchange or kernel of the step."""
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_leaver, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = dict(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
    assert res[1] == "left"
    assert res[0].startswith("detected"), res[0]
    assert "1" in res[0]


def test_compose_matches_direct_states():
    """fgt1d_segment_compose against the plain definition: the state entering segment g
    from the left is sum over sources left of it of alpha_j e^{-tau s (z_prev - y_j)}
    (and mirrored on the right), from boundary records the oracle sums directly.
    Includes an empty segment and unordered records (rejected)."""
    import paper_1909_09825_gb300 as fgt
    from paper_1909_09825_gb300.partition import DeviceSegments
    _, tau, W, _ = soe_cf.plan_soe(1e-8)
    delta = 1e-2
    plan = fgt.Plan(delta, soe=(tau, W))
    rng = np.random.default_rng(9)
    edges = [0.0, 0.2, 0.2, 0.55, 1.0]  # segment 1 is empty
    ys = [np.sort(rng.uniform(lo, hi, 40)) if hi > lo else np.empty(0) for lo, hi in zip(edges[:-1], edges[1:])]
    als = [rng.standard_normal(len(v)) for v in ys]
    recs = np.stack([oracle.segment_boundary(np.empty(0), v, al, delta, tau, W) for v, al in zip(ys, als)])
    seg = DeviceSegments(plan)
    s = 1 / np.sqrt(delta)
    for g in range(4):
        c = seg.compose(recs, g)
        n = len(tau)
        left = [j for j in range(g) if len(ys[j])]
        right = [j for j in range(g + 1, 4) if len(ys[j])]
        if left:
            zp = ys[left[-1]].max()
            yl, al = np.concatenate([ys[j] for j in left]), np.concatenate([als[j] for j in left])
            F = np.array([np.sum(al * np.exp(-t * s * (zp - yl))) for t in tau])
            assert c[4 * n] == zp
            assert np.allclose(c[:n] + 1j * c[n:2 * n], F, rtol=0, atol=1e-13 * np.abs(al).sum())
        else:
            assert np.isnan(c[4 * n]) and np.all(c[:2 * n] == 0)
        if right:
            zn = ys[right[0]].min()
            yr, ar = np.concatenate([ys[j] for j in right]), np.concatenate([als[j] for j in right])
            Gs = np.array([np.sum(ar * np.exp(-t * s * (yr - zn))) for t in tau])
            assert c[4 * n + 1] == zn
            assert np.allclose(c[2 * n:3 * n] + 1j * c[3 * n:4 * n], Gs, rtol=0, atol=1e-13 * np.abs(ar).sum())
        else:
            assert np.isnan(c[4 * n + 1])
    from paper_1909_09825_gb300 import _lib
    with pytest.raises(_lib.FGTError):
        seg.compose(recs[::-1].copy(), 0)  # segments out of order
