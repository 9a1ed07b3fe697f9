"""Python binding of libfgt1d (argument marshalling only; torch provides device memory
and streams).  Every step of the transform runs in the CUDA library."""
import ctypes

import numpy as np
import torch

from . import _lib
from ._lib import check, lib


def _f64_host(a, n):
    out = np.zeros(n, dtype=np.float64)
    out[: len(a)] = a
    return out


def _ptr(a):
    return a.ctypes.data_as(ctypes.c_void_p)


def soe_cf(n):
    """SOE of the CF order-n approximation (step a0): (tau, W, E_n) with tau, W complex
    arrays of length n/2 (one node of each conjugate pair, W = 2 w)."""
    ne = ctypes.c_int()
    arr = [np.zeros(_lib.MAX_TERMS) for _ in range(4)]
    En = ctypes.c_double()
    check(lib().fgt1d_soe_cf(int(n), ctypes.byref(ne), *[_ptr(a) for a in arr], ctypes.byref(En)), "soe_cf")
    k = ne.value
    return arr[0][:k] + 1j * arr[1][:k], arr[2][:k] + 1j * arr[3][:k], En.value


class Plan:
    """A transform plan for bandwidth delta and accuracy eps (or a given SOE).

    precision: "fp64" (FP64 accuracy at every step), "fp32" (FP32-complex recurrences with
    FP64 coordinate differences and inter-tile carries; eps >= 1e-6) or "f32x2"
    (double-float recurrences, FP64-grade accuracy; gradients run in FP64).
    exact_self: coincident source/target pairs contribute G(0) = 1 instead of S_n(0).
    """

    def __init__(self, delta, eps=None, precision="fp64", soe=None, exact_self=False):
        if precision not in ("fp64", "fp32", "f32x2"):
            raise ValueError(precision)
        flags = {"fp64": _lib.FGT1D_FP64, "fp32": _lib.FGT1D_FP32, "f32x2": _lib.FGT1D_F32X2}[precision]
        if exact_self:
            flags |= _lib.FGT1D_EXACT_SELF
        h = ctypes.c_void_p()
        if soe is None:
            check(lib().fgt1d_plan_create(float(delta), float(eps), flags, ctypes.byref(h)), "plan_create")
        else:
            tau, W = (np.asarray(v, dtype=complex) for v in soe)
            k = len(tau)
            a = [np.ascontiguousarray(v, dtype=np.float64) for v in (tau.real, tau.imag, W.real, W.imag)]
            check(lib().fgt1d_plan_create_soe(float(delta), k, *[_ptr(v) for v in a], flags, ctypes.byref(h)),
                  "plan_create_soe")
        self._h = h
        self.precision = precision
        n, ne, En, d, fl = ctypes.c_int(), ctypes.c_int(), ctypes.c_double(), ctypes.c_double(), ctypes.c_uint()
        arr = [np.zeros(_lib.MAX_TERMS) for _ in range(4)]
        check(lib().fgt1d_plan_info(h, ctypes.byref(n), ctypes.byref(ne), ctypes.byref(En), ctypes.byref(d),
                                    ctypes.byref(fl), *[_ptr(v) for v in arr]), "plan_info")
        self.n, self.n_e, self.E_n, self.delta = n.value, ne.value, En.value, d.value
        k = self.n_e
        self.tau = arr[0][:k] + 1j * arr[1][:k]
        self.W = arr[2][:k] + 1j * arr[3][:k]

    @property
    def handle(self):
        return self._h

    @property
    def tile_threads(self):
        """Threads per 4096-point sweep tile in use (128: 32 points each, 256: 16)."""
        t = ctypes.c_int()
        check(lib().fgt1d_plan_get_tile(self._h, ctypes.byref(t)), "plan_get_tile")
        return t.value

    @tile_threads.setter
    def tile_threads(self, threads):
        check(lib().fgt1d_plan_set_tile(self._h, int(threads or 0)), "plan_set_tile")

    def autotune(self, x, y, alpha, reps=3, workspace=None, stream=None):
        """Times each sweep tile shape on this workload (fgt1d_autotune) and keeps the
        fastest; returns {threads: mean ms}.  Overwrites nothing of the caller's."""
        for t, n in ((x, "x"), (y, "y"), (alpha, "alpha")):
            _dev(t, n)
        M, N = x.numel(), y.numel()
        out = torch.empty(M, dtype=torch.float64, device=x.device)
        ws = _workspace(workspace, x.device, self.workspace_size(M, N))
        return self._autotune(1, None, None, None, x, M, y, alpha, N, out, ws, reps, stream)

    def autotune_batched(self, x_off, y_off, x, y, alpha, delta=None, reps=3, workspace=None, stream=None):
        """fgt1d_autotune on a batch (arguments as transform_batched)."""
        B = x_off.numel() - 1
        M, N = x.numel(), y.numel()
        b = ctypes.c_size_t()
        check(lib().fgt1d_batched_workspace_size(self._h, B, M, N, ctypes.byref(b)), "batched_workspace_size")
        ws = _workspace(workspace, x.device, b.value)
        out = torch.empty(M, dtype=torch.float64, device=x.device)
        return self._autotune(B, x_off.contiguous(), y_off.contiguous(), delta, x, M, y, alpha, N, out, ws, reps,
                              stream)

    def _autotune(self, B, x_off, y_off, delta, x, M, y, alpha, N, out, ws, reps, stream):
        p = lambda t: ctypes.c_void_p(t.data_ptr()) if t is not None else None
        chosen = ctypes.c_int()
        ms = (ctypes.c_float * 2)()
        check(lib().fgt1d_autotune(self._h, B, p(x_off), p(y_off), p(delta), p(x), M, p(y), p(alpha), N, p(out),
                                   ctypes.c_void_p(ws.data_ptr()), ws.numel(), int(reps), _stream_ptr(stream),
                                   ctypes.byref(chosen), ms), "autotune")
        return {128: ms[0], 256: ms[1], "chosen": chosen.value}

    def workspace_size(self, M, N, host=False):
        b = ctypes.c_size_t()
        f = lib().fgt1d_workspace_size_host if host else lib().fgt1d_workspace_size
        check(f(self._h, int(M), int(N), ctypes.byref(b)), "workspace_size")
        return b.value

    def __del__(self):
        h = getattr(self, "_h", None)
        if h is not None and h.value:
            try:
                lib().fgt1d_plan_destroy(h)
            except Exception:
                pass
            self._h = None


class Workspace:
    """Grow-only device workspace (a torch uint8 buffer) reused across calls."""

    def __init__(self, device="cuda"):
        self.device = torch.device(device)
        self.buf = None

    def get(self, nbytes):
        if self.buf is None or self.buf.numel() < nbytes:
            self.buf = None
            self.buf = torch.empty(max(int(nbytes), 256), dtype=torch.uint8, device=self.device)
        return self.buf


def _stream_ptr(stream):
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


def _dev(t, name):
    if not (isinstance(t, torch.Tensor) and t.is_cuda and t.dtype == torch.float64 and t.is_contiguous()):
        raise TypeError("%s must be a contiguous float64 CUDA tensor" % name)
    return t


_default_ws = {}


def _workspace(ws, device, nbytes):
    if ws is None:
        key = torch.device(device).index
        ws = _default_ws.setdefault(key, Workspace(device))
    return ws.get(nbytes)


def transform(plan, x, y, alpha, out=None, workspace=None, stream=None, sync_check=True):
    """u = sum_j exp(-(x_i - y_j)^2 / (4 delta)) alpha_j on the GPU (eq. 1.1).

    x (M,), y (N,), alpha (N,): contiguous float64 CUDA tensors.  Returns u (M,).
    With sync_check the stream is synchronised and device-side errors raise."""
    _dev(x, "x"), _dev(y, "y"), _dev(alpha, "alpha")
    M, N = x.numel(), y.numel()
    if alpha.numel() != N:
        raise ValueError("alpha and y differ in length")
    if out is None:
        out = torch.empty(M, dtype=torch.float64, device=x.device)
    _dev(out, "out")
    nbytes = plan.workspace_size(M, N)
    ws = _workspace(workspace, x.device, nbytes)
    st = _stream_ptr(stream)
    check(lib().fgt1d_execute(plan.handle, ctypes.c_void_p(x.data_ptr()), M, ctypes.c_void_p(y.data_ptr()),
                              ctypes.c_void_p(alpha.data_ptr()), N, ctypes.c_void_p(out.data_ptr()),
                              ctypes.c_void_p(ws.data_ptr()), ws.numel(), st), "execute")
    if sync_check:
        check(lib().fgt1d_check(ctypes.c_void_p(ws.data_ptr()), ws.numel(), st), "execute (device)")
    return out


def execute_host(plan, x, y, alpha, out=None, workspace=None, stream=None, sync=True):
    """End-to-end transform of HOST numpy arrays through fgt1d_execute_host (copies in,
    transform, copy out, synchronise).  With sync=False, fgt1d_execute_host_async: the
    work is only enqueued on `stream`; `out` is valid, and the arrays may be reused, after
    wait_host(workspace, stream) (or a synchronisation of the stream)."""
    x = np.ascontiguousarray(x, dtype=np.float64)
    y = np.ascontiguousarray(y, dtype=np.float64)
    alpha = np.ascontiguousarray(alpha, dtype=np.float64)
    M, N = len(x), len(y)
    if out is None:
        out = np.empty(M, dtype=np.float64)
    nbytes = plan.workspace_size(M, N, host=True)
    ws = _workspace(workspace, torch.device("cuda", torch.cuda.current_device()), nbytes)
    f = lib().fgt1d_execute_host if sync else lib().fgt1d_execute_host_async
    check(f(plan.handle, _ptr(x), M, _ptr(y), _ptr(alpha), N, _ptr(out), ctypes.c_void_p(ws.data_ptr()), ws.numel(),
            _stream_ptr(stream)), "execute_host")
    return out


def wait_host(workspace, stream=None):
    """Waits for an execute_host(..., sync=False) on `stream` and raises on a device error."""
    ws = workspace.get(0) if isinstance(workspace, Workspace) else workspace
    check(lib().fgt1d_check(ctypes.c_void_p(ws.data_ptr()), ws.numel(), _stream_ptr(stream)), "execute_host (device)")


def sort_merged(x, y, workspace=None, stream=None):
    """Stable sorted order of the merged points [y, x] (uint32 merged indices as int64)."""
    _dev(x, "x"), _dev(y, "y")
    M, N = x.numel(), y.numel()
    b = ctypes.c_size_t()
    check(lib().fgt1d_sort_workspace_size(M, N, ctypes.byref(b)), "sort_workspace_size")
    ws = _workspace(workspace, x.device, b.value)
    perm = torch.empty(M + N, dtype=torch.int32, device=x.device)
    st = _stream_ptr(stream)
    check(lib().fgt1d_sort_merged(ctypes.c_void_p(x.data_ptr()), M, ctypes.c_void_p(y.data_ptr()), N,
                                  ctypes.c_void_p(perm.data_ptr()), ctypes.c_void_p(ws.data_ptr()), ws.numel(), st),
          "sort_merged")
    check(lib().fgt1d_check(ctypes.c_void_p(ws.data_ptr()), ws.numel(), st), "sort_merged (device)")
    return perm.to(torch.int64) & 0xFFFFFFFF


def backward(plan, x, y, alpha, grad_u, want=(True, True, True, True), workspace=None, stream=None,
             sync_check=True):
    """Gradients of L = sum_i grad_u[i] u_i: returns (grad_x, grad_y, grad_alpha, grad_delta),
    each None where `want` is False (order: x, y, alpha, delta)."""
    for t, n in ((x, "x"), (y, "y"), (alpha, "alpha"), (grad_u, "grad_u")):
        _dev(t, n)
    M, N = x.numel(), y.numel()
    dev = x.device
    gx = torch.empty(M, dtype=torch.float64, device=dev) if want[0] else None
    gy = torch.empty(N, dtype=torch.float64, device=dev) if want[1] else None
    ga = torch.empty(N, dtype=torch.float64, device=dev) if want[2] else None
    gd = torch.empty(1, dtype=torch.float64, device=dev) if want[3] else None
    b = ctypes.c_size_t()
    check(lib().fgt1d_backward_workspace_size(plan.handle, M, N, ctypes.byref(b)), "backward_workspace_size")
    ws = _workspace(workspace, dev, b.value)
    p = lambda t: ctypes.c_void_p(t.data_ptr()) if t is not None else None
    st = _stream_ptr(stream)
    check(lib().fgt1d_backward(plan.handle, p(x), M, p(y), p(alpha), N, p(grad_u), p(gx), p(gy), p(ga), p(gd),
                               ctypes.c_void_p(ws.data_ptr()), ws.numel(), st), "backward")
    if sync_check:
        check(lib().fgt1d_check(ctypes.c_void_p(ws.data_ptr()), ws.numel(), st), "backward (device)")
    return gx, gy, ga, gd


class GaussTransform(torch.autograd.Function):
    """u = FGT(x, y, alpha; delta) with a hand-written adjoint (fgt1d_backward)."""

    @staticmethod
    def forward(ctx, x, y, alpha, delta, plan):
        u = transform(plan, x.contiguous(), y.contiguous(), alpha.contiguous())
        ctx.save_for_backward(x, y, alpha)
        ctx.plan = plan
        return u

    @staticmethod
    def backward(ctx, gu):
        x, y, alpha = ctx.saved_tensors
        need = ctx.needs_input_grad
        gx, gy, ga, gd = backward(ctx.plan, x.contiguous(), y.contiguous(), alpha.contiguous(), gu.contiguous(),
                                  want=(need[0], need[1], need[2], need[3]))
        if gd is not None:
            gd = gd.reshape(())
        return gx, gy, ga, gd, None


_plans = {}


def gauss_transform(x, y, alpha, delta, eps=1e-10, precision="fp64"):
    """Differentiable u_i = sum_j exp(-(x_i - y_j)^2 / (4 delta)) alpha_j.  delta may be a
    float or a 0-dim float64 tensor (on any device) that requires grad."""
    d = float(delta.detach().cpu()) if isinstance(delta, torch.Tensor) else float(delta)
    key = (d, float(eps), precision)
    plan = _plans.get(key)
    if plan is None:
        plan = _plans[key] = Plan(d, eps, precision=precision)
    dt = delta if isinstance(delta, torch.Tensor) else torch.tensor(d, dtype=torch.float64)
    return GaussTransform.apply(x, y, alpha, dt, plan)


def transform_self(plan, x, alpha, out=None, workspace=None, stream=None, sync_check=True):
    """u_i = sum_j exp(-(x_i - x_j)^2 / (4 delta)) alpha_j with the N points as both
    targets and sources (fgt1d_execute_self: one sort of N points; fp64 and fp32 plans).  The
    self pair and coincident pairs get S_n(0), or G(0) = 1 with an exact_self plan."""
    _dev(x, "x"), _dev(alpha, "alpha")
    N = x.numel()
    if alpha.numel() != N:
        raise ValueError("alpha and x differ in length")
    if out is None:
        out = torch.empty(N, dtype=torch.float64, device=x.device)
    _dev(out, "out")
    b = ctypes.c_size_t()
    check(lib().fgt1d_self_workspace_size(plan.handle, N, ctypes.byref(b)), "self_workspace_size")
    ws = _workspace(workspace, x.device, b.value)
    st = _stream_ptr(stream)
    check(lib().fgt1d_execute_self(plan.handle, ctypes.c_void_p(x.data_ptr()), N, ctypes.c_void_p(alpha.data_ptr()),
                                   ctypes.c_void_p(out.data_ptr()), ctypes.c_void_p(ws.data_ptr()), ws.numel(), st),
          "execute_self")
    if sync_check:
        check(lib().fgt1d_check(ctypes.c_void_p(ws.data_ptr()), ws.numel(), st), "execute_self (device)")
    return out


class Geometry:
    """Fixed targets x and sources y bound once (fgt1d_geometry_bind: sorted merged
    points and the FP64 multiplier table kept on the device); apply() then evaluates
    the transform for any strength vector without sorting or exponentials.  Owns its
    workspace.  fp64 and f32x2 plans store the table; fp32 plans keep the sorted points
    only (their sweeps recompute each multiplier in a few FP32 multiply-adds)."""

    def __init__(self, plan, x, y, stream=None, sync_check=True):
        _dev(x, "x"), _dev(y, "y")
        self.plan, self.M, self.N = plan, x.numel(), y.numel()
        b = ctypes.c_size_t()
        check(lib().fgt1d_geometry_workspace_size(plan.handle, self.M, self.N, ctypes.byref(b)),
              "geometry_workspace_size")
        self.ws = torch.empty(max(int(b.value), 256), dtype=torch.uint8, device=x.device)
        st = _stream_ptr(stream)
        check(lib().fgt1d_geometry_bind(plan.handle, ctypes.c_void_p(x.data_ptr()), self.M,
                                        ctypes.c_void_p(y.data_ptr()), self.N, ctypes.c_void_p(self.ws.data_ptr()),
                                        self.ws.numel(), st), "geometry_bind")
        if sync_check:
            check(lib().fgt1d_check(ctypes.c_void_p(self.ws.data_ptr()), self.ws.numel(), st), "geometry_bind (device)")

    def apply(self, alpha, out=None, stream=None, sync_check=True):
        """u = the transform of alpha (N,) at the bound points; returns u (M,)."""
        _dev(alpha, "alpha")
        if alpha.numel() != self.N:
            raise ValueError("alpha must have N entries")
        if out is None:
            out = torch.empty(self.M, dtype=torch.float64, device=alpha.device)
        _dev(out, "out")
        st = _stream_ptr(stream)
        check(lib().fgt1d_geometry_apply(self.plan.handle, self.M, self.N, ctypes.c_void_p(alpha.data_ptr()),
                                         ctypes.c_void_p(out.data_ptr()), ctypes.c_void_p(self.ws.data_ptr()),
                                         self.ws.numel(), st), "geometry_apply")
        if sync_check:
            check(lib().fgt1d_check(ctypes.c_void_p(self.ws.data_ptr()), self.ws.numel(), st),
                  "geometry_apply (device)")
        return out


def transform_batched(plan, x_off, y_off, x, y, alpha, delta=None, out=None, workspace=None, stream=None,
                      sync_check=True):
    """B independent transforms in one pass (fgt1d_execute_batched).

    x_off, y_off: int64 CUDA tensors of B+1 offsets into x / u and y / alpha;
    delta: float64 CUDA tensor of B bandwidths, or None for the plan's delta."""
    for t, n in ((x, "x"), (y, "y"), (alpha, "alpha")):
        _dev(t, n)
    if not (x_off.is_cuda and y_off.is_cuda and x_off.dtype == torch.int64 and y_off.dtype == torch.int64):
        raise TypeError("offsets must be int64 CUDA tensors")
    B = x_off.numel() - 1
    if y_off.numel() != B + 1 or B < 1:
        raise ValueError("x_off and y_off need B + 1 entries")
    if delta is not None:
        _dev(delta, "delta")
    M, N = x.numel(), y.numel()
    if out is None:
        out = torch.empty(M, dtype=torch.float64, device=x.device)
    b = ctypes.c_size_t()
    check(lib().fgt1d_batched_workspace_size(plan.handle, B, M, N, ctypes.byref(b)), "batched_workspace_size")
    ws = _workspace(workspace, x.device, b.value)
    st = _stream_ptr(stream)
    p = lambda t: ctypes.c_void_p(t.data_ptr()) if t is not None else None
    check(lib().fgt1d_execute_batched(plan.handle, B, p(x_off.contiguous()), p(y_off.contiguous()), p(delta), p(x), M,
                                      p(y), p(alpha), N, p(out), ctypes.c_void_p(ws.data_ptr()), ws.numel(), st),
          "execute_batched")
    if sync_check:
        check(lib().fgt1d_check(ctypes.c_void_p(ws.data_ptr()), ws.numel(), st), "execute_batched (device)")
    return out
