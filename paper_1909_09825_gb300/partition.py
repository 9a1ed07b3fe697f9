"""Range-partitioned transform over the ranks of a torch.distributed group.

One transform of targets x and sources y spread over G ranks (each rank holds any
share of the points) is split along the coordinate line:

1. splitters: every rank contributes an evenly spaced sample of its coordinates; the
   G - 1 splitters are quantiles of the gathered sample;
2. routing: each point goes to the rank whose range holds its coordinate (points with
   equal coordinates to one rank), by an all-to-all of coordinates and strengths;
3. each rank transforms its segment with zero entering states and writes its boundary
   record (fgt1d_segment_execute);
4. one all-gather of the G boundary records (4 n_e + 2 values each);
5. each rank composes the states entering its segment (fgt1d_segment_compose) and adds
   their contribution to its targets (fgt1d_segment_apply);
6. the values go back to the ranks that own the targets (the reverse all-to-all).

The arithmetic runs in the library; this module moves data (torch.distributed) and
marshals arguments.  The communication device is the CPU for a gloo group and the
points' device otherwise (NCCL).
"""
import ctypes
import datetime

import numpy as np
import torch
import torch.distributed as dist

from ._lib import check, lib
from .fgt1d import Workspace, _dev, _stream_ptr


def segment_doubles(n_e):
    """Length of a boundary or carry record (FGT1D_SEGMENT_DOUBLES)."""
    return 4 * n_e + 2


class DeviceSegments:
    """The library's segment entry points for one plan on one device.  It keeps its own
    workspace (the sorted points stay there from execute to apply)."""

    def __init__(self, plan, workspace=None, stream=None):
        self.plan = plan
        self.workspace = workspace
        self.stream = stream
        self._ws = None
        self._sizes = None

    def execute(self, x, y, alpha):
        """Zero-carry transform of the segment's points: (u, boundary record on the device)."""
        for t, n in ((x, "x"), (y, "y"), (alpha, "alpha")):
            _dev(t, n)
        M, N = x.numel(), y.numel()
        u = torch.zeros(M, dtype=torch.float64, device=x.device)
        b = torch.empty(segment_doubles(self.plan.n_e), dtype=torch.float64, device=x.device)
        if self.workspace is None:
            self.workspace = Workspace(x.device)
        ws = self.workspace.get(self.plan.workspace_size(M, N))
        p = lambda t: ctypes.c_void_p(t.data_ptr()) if t.numel() else None
        check(lib().fgt1d_segment_execute(self.plan.handle, p(x), M, p(y), p(alpha), N, p(u),
                                          ctypes.c_void_p(b.data_ptr()), ctypes.c_void_p(ws.data_ptr()), ws.numel(),
                                          _stream_ptr(self.stream)), "segment_execute")
        self._ws, self._sizes = ws, (M, N)
        return u, b

    def compose(self, boundaries, g):
        """Carry record of segment g from the G boundary records (host arrays)."""
        b = np.ascontiguousarray(boundaries, dtype=np.float64)
        G = b.shape[0]
        carry = np.empty(segment_doubles(self.plan.n_e))
        check(lib().fgt1d_segment_compose(self.plan.handle, G, g, b.ctypes.data_as(ctypes.c_void_p),
                                          carry.ctypes.data_as(ctypes.c_void_p)), "segment_compose")
        return carry

    def apply(self, carry, u):
        """u += the entering states' contribution (after execute, on its workspace)."""
        M, N = self._sizes
        c = torch.from_numpy(np.ascontiguousarray(carry, dtype=np.float64)).to(u.device)
        check(lib().fgt1d_segment_apply(self.plan.handle, M, N, ctypes.c_void_p(c.data_ptr()),
                                        ctypes.c_void_p(u.data_ptr()) if M else None,
                                        ctypes.c_void_p(self._ws.data_ptr()), self._ws.numel(),
                                        _stream_ptr(self.stream)), "segment_apply")
        if M + N:  # the workspace status of the segment's transform (none ran without points)
            check(lib().fgt1d_check(ctypes.c_void_p(self._ws.data_ptr()), self._ws.numel(),
                                    _stream_ptr(self.stream)), "segment (device)")
        return u


def _comm_device(group, dev):
    return torch.device("cpu") if dist.get_backend(group) == "gloo" else dev


def splitters(coords, G, group=None, samples=1024):
    """G - 1 coordinate splitters from an evenly spaced sample of every rank's points."""
    dev = _comm_device(group, coords.device)
    n = coords.numel()
    k = min(samples, n)
    idx = torch.linspace(0, max(n - 1, 0), k, device=coords.device).round().long() if k else \
        torch.empty(0, dtype=torch.long, device=coords.device)
    s = coords[idx].to(dev)
    lens = [torch.zeros(1, dtype=torch.int64, device=dev) for _ in range(G)]
    dist.all_gather(lens, torch.tensor([k], dtype=torch.int64, device=dev), group=group)
    top = int(max(int(v.item()) for v in lens))
    pad = torch.full((top,), float("nan"), dtype=torch.float64, device=dev)
    pad[:k] = s
    parts = [torch.empty(top, dtype=torch.float64, device=dev) for _ in range(G)]
    dist.all_gather(parts, pad, group=group)
    allv = torch.cat([p[:int(l.item())] for p, l in zip(parts, lens)])
    allv = torch.sort(allv[~torch.isnan(allv)]).values
    if allv.numel() == 0:
        return torch.zeros(G - 1, dtype=torch.float64, device=coords.device)
    q = [allv[min(allv.numel() - 1, (allv.numel() * j) // G)] for j in range(1, G)]
    return torch.stack(q).to(coords.device) if q else torch.empty(0, dtype=torch.float64, device=coords.device)


class _Route:
    """Points grouped by destination rank, and the counts that undo the exchange."""

    def __init__(self, dest, G, group):
        self.group = group
        self.order = torch.argsort(dest, stable=True)
        send = torch.bincount(dest, minlength=G).to(torch.int64)
        dev = _comm_device(group, dest.device)
        recv = torch.empty(G, dtype=torch.int64, device=dev)
        dist.all_to_all_single(recv, send.to(dev), group=group)
        self.send = [int(v) for v in send.tolist()]
        self.recv = [int(v) for v in recv.tolist()]
        self.dev = dev

    def forward(self, t):
        out = torch.empty(sum(self.recv), dtype=t.dtype, device=self.dev)
        dist.all_to_all_single(out, t[self.order].to(self.dev), self.recv, self.send, group=self.group)
        return out

    def backward(self, t, like):
        out = torch.empty(sum(self.send), dtype=t.dtype, device=self.dev)
        dist.all_to_all_single(out, t.to(self.dev), self.send, self.recv, group=self.group)
        res = torch.empty_like(like)
        res[self.order] = out.to(like.device)
        return res


def transform_partitioned(plan, x, y, alpha, group=None, segments=None, samples=1024, health_timeout_s=None):
    """u for this rank's targets x, with the sources y, alpha of every rank (eq. 1.1).

    x, y, alpha: this rank's share (float64 tensors, one device per rank).  segments:
    the segment implementation (DeviceSegments(plan) by default).  health_timeout_s:
    on a gloo group, a monitored barrier first checks that every rank has arrived and
    raises naming the missing ones after that many seconds."""
    G = dist.get_world_size(group)
    g = dist.get_rank(group)
    if health_timeout_s is not None and dist.get_backend(group) == "gloo":
        dist.monitored_barrier(group=group, timeout=datetime.timedelta(seconds=health_timeout_s),
                               wait_all_ranks=True)
    segs = segments if segments is not None else DeviceSegments(plan)
    spl = splitters(torch.cat([x, y]), G, group, samples)
    rx = _Route(torch.searchsorted(spl, x, right=True), G, group)
    ry = _Route(torch.searchsorted(spl, y, right=True), G, group)
    dev = x.device
    xs, ys, als = rx.forward(x).to(dev), ry.forward(y).to(dev), ry.forward(alpha).to(dev)
    u_seg, bnd = segs.execute(xs, ys, als)
    cdev = _comm_device(group, dev)
    recs = [torch.empty(bnd.numel(), dtype=torch.float64, device=cdev) for _ in range(G)]
    dist.all_gather(recs, bnd.to(cdev), group=group)
    carry = segs.compose(torch.stack(recs).cpu().numpy(), g)
    u_seg = segs.apply(carry, u_seg)
    return rx.backward(u_seg, x)
