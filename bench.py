"""Benchmark of the GB300 SOE fast Gauss transform.

One step = one full transform (merged sort, forward and backward SOE sweeps,
evaluation, unpermutation) of M = N = 2^26 points uniform on [0, 1] with
alpha ~ N(0, 1), inputs already resident in HBM (3.2 GB, larger than L2).  The
headline is the FP64 path at eps = 1e-6, delta = 1e-5; the other (eps, delta,
precision) combinations of the same workload are reported under "also".

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]

Under torchrun each rank runs its own replica of the workload on its GPU (the
single transform has no partition without an exchange step), the timed region is
bracketed by barriers and rank 0 prints one JSON line with the max over ranks.
"""
import argparse
import ctypes
import json
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "(M+N) points/s at eps=1e-6 and 1e-10 on 1 GB300; % of SFU/FP64/HBM roofline"
LOG2_M = 26
HEAD = dict(delta=1e-5, eps=1e-6, precision="fp64")
ALSO = [dict(delta=1e-5, eps=1e-10, precision="fp64"), dict(delta=1e-2, eps=1e-6, precision="fp64"),
        dict(delta=1e-2, eps=1e-10, precision="fp64"), dict(delta=1e-5, eps=1e-3, precision="fp64"),
        dict(delta=1e-5, eps=1e-6, precision="fp32"), dict(delta=1e-2, eps=1e-6, precision="fp32"),
        dict(delta=1e-5, eps=1e-6, precision="f32x2"), dict(delta=1e-5, eps=1e-10, precision="f32x2")]
# FP64 pipe peak when the run's own measurement (fgt1d_measure_peaks) is unavailable:
# 152 SMs x 2 DFMA/clk/SM x 2 flop x 2070 MHz maximum SM clock.
FP64_PEAK_TFLOPS = 152 * 2 * 2 * 2.070e9 / 1e12
# Algorithmic FP64 pipe ops of the forward sweep kernel per (merged point, term): the
# multiplier exp(-tau theta) as a degree-4 Taylor polynomial (C_ce = 8), one complex
# multiply-add of the recurrence (4) and the evaluation at targets (2 per target, half
# of the points); plus 2 per point (difference and scaling of the gap).
C_CE = 8
# item table; sort: range, prefix maps, histogram, pass plan, pass chain, 4 prefix digit
# passes, merge, run detection, fix-up, and the fallback's 13 kernels (launched, they
# exit at once unless a run of equal prefixes is too long); two sweeps
KERNELS_PER_TRANSFORM = 27
WORKLOAD = ("plain FP64 at scale: M=N=2^26, x,y ~ U[0,1), alpha ~ N(0,1), delta=%g, eps=%g, unsorted "
            "inputs (sort timed), seed 0")


def measure_peaks():
    """The pipes' throughput on this GPU (fgt1d_measure_peaks), measured in this run."""
    from paper_1909_09825_gb300 import _lib
    o = (ctypes.c_double * 10)()
    _lib.check(_lib.lib().fgt1d_measure_peaks(o, None), "measure_peaks")
    v = list(o)
    return {"fp64_tflops": 2 * v[0] / 1e12, "fp64_fma_per_clk_per_sm": v[1],
            "fp32_tflops": 2 * v[2] / 1e12, "fp32_fma_per_clk_per_sm": v[3],
            "sfu_ex2_per_s": v[4], "sfu_ex2_per_clk_per_sm": v[5],
            "sfu_sin_per_s": v[6], "sfu_sin_per_clk_per_sm": v[7], "sms": int(v[8]), "sm_mhz": v[9],
            "how": "fgt1d_measure_peaks: 16 independent FMA/ex2/sin chains per thread, 8 x 256 threads per "
                   "SM, best of two CUDA-event-timed launches; SM clock from clock64 over globaltimer"}


def max_over_ranks(value, device=None):
    """Max of a per-rank float over all ranks (identity without a process group)."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(value)
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


class ClockSampler:
    """nvidia-smi clock / throttle-reason samples during the timed region."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_id):
        self.gpu_id = gpu_id
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", self.gpu_id, "--query-gpu=" + self.FIELDS,
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
        time.sleep(0.3)
        return self

    def __exit__(self, *a):
        self.lines = []
        if self.proc is not None:
            self.proc.terminate()
            try:
                out, _ = self.proc.communicate(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
                out, _ = self.proc.communicate()
            self.lines = [l for l in out.splitlines() if l.strip()]

    def summary(self):
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for l in getattr(self, "lines", []):
            f = [v.strip() for v in l.split(",")]
            if len(f) < 8:
                continue
            try:
                sm.append(float(f[0]))
                mx.append(float(f[1]))
            except ValueError:
                continue
            for n, v in zip(names, f[4:8]):
                if v.lower() == "active":
                    reasons.add(n)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons), "samples": len(sm)}


def cpu_baseline(delta, eps, log2_single=22, log2_multi=24):
    """The oracle's implementation of the paper's algorithm (stable merge sort, the
    recurrences of eqs. 4.5-4.6, evaluation) on a bounded sample of the same workload:
    on every host core (coordinate segments with span carries) and on one thread (the
    paper's mode)."""
    from oracle import oracle, soe_cf
    from paper_1909_09825_gb300 import inputs
    n, tau, W, En = soe_cf.plan_soe(eps)
    cores = oracle.max_threads()
    M = 1 << log2_multi
    x, y, a = inputs.uniform(M, M, seed=0)
    oracle.recurrence_par(x, y, a, delta, tau, W)  # untimed: page in the buffers
    t0 = time.perf_counter()
    oracle.recurrence_par(x, y, a, delta, tau, W)
    dt_multi = time.perf_counter() - t0
    M1 = 1 << log2_single
    x, y, a = x[:M1], y[:M1], a[:M1]
    t0 = time.perf_counter()
    oracle.recurrence(x, y, a, delta, tau, W)
    dt_single = time.perf_counter() - t0
    return {"value": 2 * M / dt_multi, "unit": "points/s", "cores": cores, "kind": "oracle",
            "sample": "M=N=2^%d of the same distribution, delta=%g, eps=%g (n_e=%d): stable sort + "
                      "forward/backward recurrences over %d coordinate segments with direct span carries, "
                      "%d threads, %.1f s" % (log2_multi, delta, eps, len(tau), 8 * cores, cores, dt_multi),
            "single_thread": {"value": 2 * M1 / dt_single, "unit": "points/s", "cores": 1,
                              "sample": "M=N=2^%d, the serial merge sort + recurrences (the paper's mode), %.1f s"
                                        % (log2_single, dt_single)}}


def run_reference(args):
    ws, rank, _ = dist_env()
    if rank != 0:
        return
    delta, eps = HEAD["delta"], HEAD["eps"]
    from oracle import oracle, soe_cf
    from paper_1909_09825_gb300 import inputs
    n, tau, W, En = soe_cf.plan_soe(eps)
    log2 = 22
    M = 1 << log2
    cores = oracle.max_threads()
    x, y, a = inputs.uniform(M, M, seed=0)
    for _ in range(args.warmup):
        oracle.recurrence_par(x, y, a, delta, tau, W)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        oracle.recurrence_par(x, y, a, delta, tau, W)
    dt = (time.perf_counter() - t0) / args.steps
    v = 2 * M / dt
    sample = ("each step: M=N=2^%d of the headline workload's distribution (a bounded sample of M=N=2^%d) "
              "through the oracle's sort + recurrences on %d host threads" % (log2, LOG2_M, cores))
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": "points/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt * 1e3, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": (WORKLOAD % (delta, eps)) + "; timed on a sample of M=N=2^%d per step" % log2,
                       "M": M, "N": M, "sample_of": {"M": 1 << LOG2_M, "N": 1 << LOG2_M},
                       "delta": delta, "eps": eps},
            "cpu_baseline": {"value": v, "unit": "points/s", "cores": cores, "kind": "oracle", "sample": sample},
            "e2e": {"value": v, "unit": "points/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--log2", type=int, default=LOG2_M, help="log2 of M = N (default 26)")
    ap.add_argument("--no-also", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--tile", type=int, default=0, choices=[0, 128, 256],
                    help="sweep tile threads; 0 = autotune each configuration (default)")
    ap.add_argument("--precision", default=HEAD["precision"], choices=["fp64", "fp32", "f32x2"],
                    help="precision of the headline configuration (profiling runs)")
    ap.add_argument("--section", default=None, choices=["batched", "differentiation"],
                    help="run only this extra section and print its record (profiling runs)")
    args = ap.parse_args()
    if args.impl == "reference":
        return run_reference(args)

    import torch
    import torch.distributed as dist

    import paper_1909_09825_gb300 as fgt
    from paper_1909_09825_gb300 import _lib, inputs

    world, rank, local = dist_env()
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    stream = torch.cuda.current_stream(dev)
    if args.section:
        rec = batched(dev, world, check=False) if args.section == "batched" else differentiation(dev, world)
        if rank == 0:
            print(json.dumps({"section": args.section, **rec}))
        return

    def barrier():
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize(dev)

    M = N = 1 << args.log2
    P = M + N
    x, y, a = inputs.uniform(M, N, seed=0)
    X, Y, A = (torch.from_numpy(v).to(dev) for v in (x, y, a))
    U = torch.empty(M, dtype=torch.float64, device=dev)
    ws = fgt.Workspace(dev)

    def timed(cfg, steps, warmup, profile=False):
        plan = fgt.Plan(cfg["delta"], cfg["eps"], precision=cfg["precision"])
        buf = ws.get(plan.workspace_size(M, N))
        if args.tile:
            plan.tile_threads = args.tile
            tune = {}
        else:
            tune = plan.autotune(X, Y, A, reps=2, workspace=ws)  # untimed: picks the sweep tile shape
        for _ in range(warmup):
            fgt.transform(plan, X, Y, A, out=U, workspace=ws)
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(4 * steps)]
        barrier()
        t_start = torch.cuda.Event(enable_timing=True)
        t_end = torch.cuda.Event(enable_timing=True)
        t_start.record(stream)
        for s in range(steps):
            if profile:
                e4 = ev[4 * s: 4 * s + 4]
                for e in e4:
                    e.record(stream)      # creates the event; re-recorded inside the call
                arr = (ctypes.c_void_p * 4)(*[ctypes.c_void_p(e.cuda_event) for e in e4])
                _lib.check(_lib.lib().fgt1d_execute_profiled(
                    plan.handle, ctypes.c_void_p(X.data_ptr()), M, ctypes.c_void_p(Y.data_ptr()),
                    ctypes.c_void_p(A.data_ptr()), N, ctypes.c_void_p(U.data_ptr()), ctypes.c_void_p(buf.data_ptr()),
                    buf.numel(), ctypes.c_void_p(stream.cuda_stream), arr), "execute_profiled")
            else:
                fgt.transform(plan, X, Y, A, out=U, workspace=ws, sync_check=False)
        t_end.record(stream)
        barrier()
        _lib.check(_lib.lib().fgt1d_check(ctypes.c_void_p(buf.data_ptr()), buf.numel(),
                                          ctypes.c_void_p(stream.cuda_stream)), "bench (device status)")
        ms = max_over_ranks(t_start.elapsed_time(t_end) / steps, dev)
        stages = None
        if profile:
            st = np.array([[ev[4 * s + i].elapsed_time(ev[4 * s + i + 1]) for i in range(3)] for s in range(steps)])
            stages = {"sort_ms": float(st[:, 0].mean()), "fwd_sweep_ms": float(st[:, 1].mean()),
                      "bwd_sweep_ms": float(st[:, 2].mean())}
        if stages is not None:
            stages["tile_threads"] = plan.tile_threads
            stages["autotune_ms"] = {str(k): v for k, v in tune.items() if k != "chosen"}
        return plan, ms, stages

    peaks = measure_peaks()
    fp64_peak = peaks["fp64_tflops"]
    gpu_uuid = "GPU-" + str(torch.cuda.get_device_properties(dev).uuid)
    with ClockSampler(gpu_uuid) as clk:
        plan, ms, stages = timed(dict(HEAD, precision=args.precision), args.steps, args.warmup, profile=True)
    clocks = clk.summary()
    value = world * P / (ms * 1e-3)

    # roofline of the dominant kernel (forward sweep, FP64 pipe), against the FP64 FMA
    # rate measured above in this run (burst, the sweep is timed alone per launch)
    n_e = plan.n_e
    fwd_ops = P * n_e * (C_CE + 4 + 2.0 * M / P) + 2 * P
    fwd_s = stages["fwd_sweep_ms"] * 1e-3
    achieved = 2 * fwd_ops / fwd_s / 1e12
    roofline = {"bound": "alu", "pipe": "fp64",
                "kernel": "k_sweep_fwd<double, %d, %d, %d>" % (n_e, plan.tile_threads, 4096 // plan.tile_threads),
                "achieved": achieved,
                "peak": fp64_peak, "unit": "TFLOP/s", "frac": achieved / fp64_peak,
                "peak_source": "measured in this run (fgt1d_measure_peaks, DFMA chains, %.0f MHz)" % peaks["sm_mhz"],
                "algorithmic_ops_per_unit": "unit = (merged point, SOE term); C_ce=%d + 4 + 2 M/P FP64 ops, "
                                            "+2 per point" % C_CE,
                "traffic": None}
    # the backward sweep (4 + 2 M/P per point and term) and the whole transform
    # (n_e (C_ce + 20) FP64 ops per point, C_ce fixed before tuning) against the same peak
    bwd_ops = P * n_e * (4 + 2.0 * M / P)
    bwd_ach = 2 * bwd_ops / (stages["bwd_sweep_ms"] * 1e-3) / 1e12
    whole_ach = 2 * P * n_e * (C_CE + 20) / (ms * 1e-3) / 1e12
    roofline_more = {
        "bwd_sweep": {"kernel": "k_sweep_bwd<double, %d, %d, %d, 1>" % (n_e, plan.tile_threads,
                                                                        4096 // plan.tile_threads),
                      "achieved": bwd_ach, "frac": bwd_ach / fp64_peak, "unit": "TFLOP/s",
                      "algorithmic_ops_per_unit": "4 + 2 M/P FP64 ops per (merged point, term)"},
        "whole_transform": {"achieved": whole_ach, "frac": whole_ach / fp64_peak, "unit": "TFLOP/s",
                            "algorithmic_ops_per_unit": "n_e (C_ce + 20) FP64 ops per merged point"}}
    # the sort moves memory: its algorithmic bytes against the measured copy bandwidth
    hbm, hbm_src = hbm_peak()
    passes = active_sort_passes(x, y)
    sort_gbs = P * sort_bytes_per_point(passes) / (stages["sort_ms"] * 1e-3) / 1e9
    roofline_more["sort"] = {"bound": "hbm", "achieved": sort_gbs, "peak": hbm, "unit": "GB/s",
                             "frac": sort_gbs / hbm, "peak_source": hbm_src, "digit_passes": passes,
                             "algorithmic_bytes_per_point": sort_bytes_per_point(passes)}
    traffic = _traffic_record(plan)
    if traffic is not None:
        roofline["traffic"] = traffic * P

    # end to end through the host-buffer entry point (copies inside the timed region),
    # right after the headline so that both see the same GPU state: every step uploads
    # x, y, alpha from pinned host memory and reads u back into pinned host memory.
    # Steps alternate between two streams and workspaces (fgt1d_execute_host_async), so
    # one step's copies run under the other's kernels; a step's result is waited for
    # (and its device status checked) before its stream takes the step after next.
    hx = torch.from_numpy(x).pin_memory().numpy()
    hy = torch.from_numpy(y).pin_memory().numpy()
    ha = torch.from_numpy(a).pin_memory().numpy()
    hus = [torch.empty(M, dtype=torch.float64).pin_memory().numpy() for _ in range(2)]
    hwss = [fgt.Workspace(dev) for _ in range(2)]
    hst = [torch.cuda.Stream(dev) for _ in range(2)]
    for j in range(2):
        fgt.execute_host(plan, hx, hy, ha, out=hus[j], workspace=hwss[j], stream=hst[j])
    barrier()
    e2e_steps = max(4, min(args.steps, 6))
    t0 = time.perf_counter()
    for i in range(e2e_steps):
        j = i % 2
        if i >= 2:
            fgt.wait_host(hwss[j], hst[j])
        fgt.execute_host(plan, hx, hy, ha, out=hus[j], workspace=hwss[j], stream=hst[j], sync=False)
    for j in range(2):
        fgt.wait_host(hwss[j], hst[j])
    barrier()
    e2e_s = (time.perf_counter() - t0) / e2e_steps
    del hwss

    also = []
    if not args.no_also:
        for cfg in ALSO:
            p2, ms2, st2 = timed(cfg, 3, 2, profile=True)
            err2 = None
            if rank == 0 and not args.no_cpu:
                err2 = sampled_error(p2, X, Y, A, x, y, a, cfg["delta"], dev, n=4)
            entry = {"precision": cfg["precision"], "delta": cfg["delta"], "eps": cfg["eps"], "n_e": p2.n_e,
                     "value": world * P / (ms2 * 1e-3), "ms_per_step": ms2, "stages": st2, "error": err2}
            if cfg["precision"] == "fp32":
                entry["roofline"] = hbm_roofline_fp32(st2, x, y, M, N)
            also.append(entry)

    # error of the headline result against the oracle's direct sum at sampled targets
    head_err = None
    if rank == 0 and not args.no_cpu:
        head_err = sampled_error(plan, X, Y, A, x, y, a, HEAD["delta"], dev, n=256)
        head_err["every_target_vs_recurrence"] = every_target_error(args.precision, X, Y, A, x, y, a,
                                                                     HEAD["delta"], HEAD["eps"])

    extra = {}
    if not args.no_also:
        extra["geometry_reuse"] = geometry_reuse(plan, X, Y, A, x, y, a, dev, world, rank, args, fp64_peak)
        extra["identical_points"] = identical_points(X, A, dev, world, stream)
        extra["presorted"] = presorted(plan, X, Y, A, x, y, a, dev, world, stream, rank == 0 and not args.no_cpu)
        extra["precision_split"] = precision_split(args, dev, world, P)
        extra["differentiation"] = differentiation(dev, world)
        extra["batched"] = batched(dev, world, check=rank == 0 and not args.no_cpu)

    cpu = None
    if rank == 0 and not args.no_cpu:
        cpu = cpu_baseline(HEAD["delta"], HEAD["eps"])

    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": "points/s", "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
                "vs_baseline": None, "dtype": {"fp64": "f64", "fp32": "f32", "f32x2": "f32x2"}[args.precision],
                "data": "synthetic",
                "config": {"workload": WORKLOAD % (HEAD["delta"], HEAD["eps"]), "M": M, "N": N,
                           "delta": HEAD["delta"], "eps": HEAD["eps"], "n_e": plan.n_e, "E_n": plan.E_n,
                           "precision": args.precision, "tile_threads": plan.tile_threads, "l2": "inputs (24 B/point, %.1f GB) larger than the 129 MB L2"
                                                       % (24 * P / 2 ** 30 / 1.0),
                           "parallelism": "replicas" if world > 1 else "single"},
                "stages": stages, "error": head_err, "roofline": roofline, "roofline_more": roofline_more,
                "peaks": peaks, "cpu_baseline": cpu,
                "e2e": {"value": world * P / e2e_s, "unit": "points/s", "h2d_bytes_per_step": 8 * (M + 2 * N),
                        "d2h_bytes_per_step": 8 * M, "steps": e2e_steps,
                        "how": "fgt1d_execute_host_async from pinned host memory, steps alternating between "
                               "two streams (one step's copies under the other's kernels), host clock over "
                               "all steps and their waits"},
                "gpu_launches": KERNELS_PER_TRANSFORM * args.steps, "clocks": clocks, "also": also, **extra}
        gr = line.get("geometry_reuse")
        if gr:
            gr["speedup_vs_full_transform"] = ms / gr["apply_ms"]
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


def hbm_peak():
    """Measured copy bandwidth of this GPU pool (GB/s) and where it comes from."""
    f = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(f):
        return float(json.load(open(f))["hbm_gbs"]), "measured (MEASURED_PEAKS.json hbm_gbs)"
    return 6800.0, "fallback (6.8 TB/s, one earlier GB300 measurement)"


def _fixq(b, eh):
    """sign(z) floor(|z| / 2^(eh - 1075)) from the bits b (uint64 array) of z."""
    ef = ((b >> np.uint64(52)) & np.uint64(0x7FF)).astype(np.int64)
    m = b & np.uint64((1 << 52) - 1)
    m = np.where(ef > 0, m | np.uint64(1 << 52), m)
    sh = eh - np.maximum(ef, 1)
    q = np.where(sh >= 64, np.uint64(0), m >> np.minimum(np.maximum(sh, 0), 63).astype(np.uint64)).astype(np.int64)
    return np.where((b >> np.uint64(63)) == 1, -q, q)


def active_sort_passes(x, y):
    """Digit passes the sort runs on these points (one item): the 8-bit digits of the
    32-bit prefix keys that are not the same for every point, padding included."""
    z = np.concatenate([y, x])
    b = z.view(np.uint64).copy()
    b[b == np.uint64(0x8000000000000000)] = 0  # -0.0 as +0.0
    lo, hi = b[np.argmin(z)], b[np.argmax(z)]
    eh = max(1, int((lo >> np.uint64(52)) & np.uint64(0x7FF)), int((hi >> np.uint64(52)) & np.uint64(0x7FF)))
    qlo, qhi = (int(_fixq(np.array([v], dtype=np.uint64), eh)[0]) for v in (lo, hi))
    sh = max(0, (qhi - qlo).bit_length() - 32)
    k = ((_fixq(b, eh) - qlo) >> sh).astype(np.uint64)
    if len(z) % 4096:
        k = np.append(k, np.uint64(0xFFFFFFFF))
    n = 0
    for d in range(4):
        dg = (k >> np.uint64(8 * d)) & np.uint64(255)
        n += int(np.any(dg != dg[0]))
    return max(n, 1)


def sort_bytes_per_point(passes):
    """Algorithmic bytes per merged point of the prefix sort: the range pass reads the
    coordinate (8), the histogram pass reads it again and writes the prefix key, full key
    and code (8 + 16), each digit pass reads and writes those 16 bytes, and the run
    detection reads the prefix and full keys (12)."""
    return 8 + 24 + 32 * passes + 12


def hbm_roofline_fp32(st, x, y, M, N):
    """HBM roofline of the FP32 path's two stages, which move memory rather than compute:
    the sort (sort_bytes_per_point) and the two sweeps (forward: key 8, code 4, strength
    8 N/P, partial sum 4; backward: key 8, code 4, strength 8 N/P, partial sum 4, value
    8 M/P, code 4 M/P at targets)."""
    peak, src = hbm_peak()
    P = M + N
    passes = active_sort_passes(x, y)
    sort_b = P * sort_bytes_per_point(passes)
    sweep_b = P * (8 + 4 + 8 * N / P + 4) + P * (8 + 4 + 8 * N / P + 4 + 12 * M / P)
    sort_gbs = sort_b / (st["sort_ms"] * 1e-3) / 1e9
    sweep_gbs = sweep_b / ((st["fwd_sweep_ms"] + st["bwd_sweep_ms"]) * 1e-3) / 1e9
    return {"bound": "hbm", "unit": "GB/s", "peak": peak, "peak_source": src,
            "sort": {"achieved": sort_gbs, "frac": sort_gbs / peak, "passes": passes,
                     "algorithmic_bytes_per_point": sort_bytes_per_point(passes)},
            "sweeps": {"achieved": sweep_gbs, "frac": sweep_gbs / peak,
                       "algorithmic_bytes_per_point": sweep_b / P}}


def _event_time(fn, steps, warmup, stream):
    import torch
    for _ in range(warmup):
        fn()
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(steps):
        fn()
    e1.record(stream)
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / steps


def sampled_error(plan, X, Y, A, x, y, a, delta, dev, n=8, seed=17):
    """||u - u_ref||_inf / sum|alpha| over n sampled targets against the oracle's direct sum."""
    import torch
    import paper_1909_09825_gb300 as fgt
    from oracle import oracle
    u = fgt.transform(plan, X, Y, A)
    idx = np.random.default_rng(seed).choice(len(x), n, replace=False)
    ug = u[torch.from_numpy(idx).to(dev)].cpu().numpy()
    ref = oracle.direct(x[idx], y, a, delta, nthreads=0)
    return {"max_abs_err_over_sum_abs_alpha": float(np.max(np.abs(ug - ref)) / np.abs(a).sum()),
            "sampled_targets": n, "reference": "oracle direct FP64 sum over all sources"}


def every_target_error(precision, X, Y, A, x, y, a, delta, eps):
    """||u - u_O3||_inf / sum|alpha| over EVERY target: the GPU plan and the oracle's
    recurrence (paper's algorithm, all host cores) both on the oracle's SOE nodes."""
    import paper_1909_09825_gb300 as fgt
    from oracle import oracle, soe_cf
    _, tau, W, _ = soe_cf.plan_soe(eps)
    p = fgt.Plan(delta, soe=(tau, W), precision=precision)
    u = fgt.transform(p, X, Y, A).cpu().numpy()
    t0 = time.perf_counter()
    ref = oracle.recurrence_par(x, y, a, delta, tau, W)
    dt = time.perf_counter() - t0
    return {"max_abs_err_over_sum_abs_alpha": float(np.max(np.abs(u - ref)) / np.abs(a).sum()),
            "targets": len(x), "reference": "oracle recurrence (eqs. 4.5-4.6) on the oracle's nodes, every target",
            "oracle_s": dt}


def geometry_reuse(plan, X, Y, A, x, y, a, dev, world, rank, args, fp64_peak):
    """Headline workload with fixed points (Sec. 5's pre-sorted points and stored
    exponential table): bind once (sort + FP64 multiplier table), then apply to new
    strength vectors (sweeps only), timed with CUDA events on the launching stream."""
    import torch
    import paper_1909_09825_gb300 as fgt
    stream = torch.cuda.current_stream(dev)
    M, N = X.numel(), Y.numel()
    P = M + N
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    g = fgt.Geometry(plan, X, Y, sync_check=False)
    e1.record(stream)
    torch.cuda.synchronize(dev)
    bind_ms = e0.elapsed_time(e1)
    U = torch.empty(M, dtype=torch.float64, device=dev)
    apply_ms = _event_time(lambda: g.apply(A, out=U, sync_check=False), 5, 3, stream)
    g.apply(A, out=U)  # synchronises and checks the device status
    err = None
    if rank == 0 and not args.no_cpu:
        rng = np.random.default_rng(17)
        idx = np.sort(rng.choice(M, 8, replace=False))
        ug = U[torch.from_numpy(idx).to(dev)].cpu().numpy()
        from oracle import oracle
        ref = oracle.direct(x[idx], y, a, plan.delta, nthreads=0)
        err = float(np.max(np.abs(ug - ref)) / np.abs(a).sum())
    n_e = plan.n_e
    ops = P * n_e * (8 + 4.0 * M / P)  # one complex multiply-add per point and term in each sweep + evaluation
    achieved = 2 * ops / (apply_ms * 1e-3) / 1e12
    del g
    torch.cuda.empty_cache()
    # the same points bound for the double-float sweeps (double-float table entries)
    pdf = fgt.Plan(plan.delta, soe=(plan.tau, plan.W), precision="f32x2")
    pdf.tile_threads = plan.tile_threads
    gdf = fgt.Geometry(pdf, X, Y)
    apply_df_ms = _event_time(lambda: gdf.apply(A, out=U, sync_check=False), 5, 3, stream)
    gdf.apply(A, out=U)
    del gdf
    torch.cuda.empty_cache()
    # and for the FP32 sweeps at eps 1e-6 (sorted points only: the sweeps recompute)
    p32 = fgt.Plan(plan.delta, 1e-6, precision="fp32")
    p32.tile_threads = plan.tile_threads
    g32 = fgt.Geometry(p32, X, Y)
    apply_32_ms = _event_time(lambda: g32.apply(A, out=U, sync_check=False), 5, 3, stream)
    g32.apply(A, out=U)
    del g32, U
    torch.cuda.empty_cache()
    return {"workload": "headline points bound once; apply = both sweeps with the stored FP64 table",
            "bind_ms": bind_ms, "apply_ms": apply_ms, "apply_points_per_s": world * P / (apply_ms * 1e-3),
            "apply_f32x2_ms": apply_df_ms, "apply_fp32_eps1e-6_ms": apply_32_ms,
            "speedup_vs_full_transform": None, "error_vs_direct": err,
            "apply_roofline": {"bound": "alu", "pipe": "fp64", "achieved": achieved, "peak": fp64_peak,
                               "unit": "TFLOP/s", "frac": achieved / fp64_peak,
                               "algorithmic_ops_per_unit": "unit = (merged point, term): 8 + 4 M/P FP64 ops",
                               "table_bytes_per_point": 2 * 16 * n_e}}


def presorted(plan, X, Y, A, x, y, a, dev, world, stream, check):
    """Sec. 5's pre-sorted points: the headline targets and sources, each sorted
    ascending (the strengths kept in place), through the same transform; the sort step
    detects the presorted runs and merges them instead of running the digit passes.
    Stage times from CUDA events recorded inside the call."""
    import torch
    from paper_1909_09825_gb300 import _lib
    XS, YS = torch.sort(X).values, torch.sort(Y).values
    M, N = X.numel(), Y.numel()
    U = torch.empty(M, dtype=torch.float64, device=dev)
    buf = torch.empty(plan.workspace_size(M, N), dtype=torch.uint8, device=dev)
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(4)]
    arr = None

    def run():
        nonlocal arr
        for e in ev:
            e.record(stream)
        arr = (ctypes.c_void_p * 4)(*[ctypes.c_void_p(e.cuda_event) for e in ev])
        _lib.check(_lib.lib().fgt1d_execute_profiled(
            plan.handle, ctypes.c_void_p(XS.data_ptr()), M, ctypes.c_void_p(YS.data_ptr()),
            ctypes.c_void_p(A.data_ptr()), N, ctypes.c_void_p(U.data_ptr()), ctypes.c_void_p(buf.data_ptr()),
            buf.numel(), ctypes.c_void_p(stream.cuda_stream), arr), "execute_profiled")

    ms = _event_time(run, 5, 3, stream)
    st = [ev[i].elapsed_time(ev[i + 1]) for i in range(3)]
    _lib.check(_lib.lib().fgt1d_check(ctypes.c_void_p(buf.data_ptr()), buf.numel(),
                                      ctypes.c_void_p(stream.cuda_stream)), "presorted (device status)")
    err = None
    if check:
        from oracle import oracle
        xs, ys = np.sort(x), np.sort(y)
        idx = np.random.default_rng(19).choice(M, 8, replace=False)
        ug = U[torch.from_numpy(idx).to(dev)].cpu().numpy()
        ref = oracle.direct(xs[idx], ys, a, plan.delta, nthreads=0)
        err = float(np.max(np.abs(ug - ref)) / np.abs(a).sum())
    del XS, YS, U, buf
    torch.cuda.empty_cache()
    return {"workload": "headline x and y each sorted ascending (alpha in place), delta=%g, eps=%g, FP64"
                        % (plan.delta, HEAD["eps"]),
            "points_per_s": world * (M + N) / (ms * 1e-3), "ms": ms,
            "stages_last_step": {"sort_ms": st[0], "fwd_sweep_ms": st[1], "bwd_sweep_ms": st[2]},
            "error_vs_direct": err}


def identical_points(X, A, dev, world, stream):
    """Fig. 4.1's case (targets = sources, the shape of Table 5.1: uniform points,
    delta = 1): the N = 2^26 headline targets with their strengths, one sort of N
    points (fgt1d_execute_self), against the general path on (x, x) (2N merged points)."""
    import torch
    import paper_1909_09825_gb300 as fgt
    N = X.numel()
    out = []
    U = torch.empty(N, dtype=torch.float64, device=dev)
    A_ = A[:N]
    for eps in (1e-6, 1e-10):
        plan = fgt.Plan(1.0, eps)
        ws = fgt.Workspace(dev)
        ms_self = _event_time(lambda: fgt.transform_self(plan, X, A_, out=U, workspace=ws, sync_check=False), 3, 3,
                              stream)
        fgt.transform_self(plan, X, A_, out=U, workspace=ws)  # checks the device status
        ms_gen = _event_time(lambda: fgt.transform(plan, X, X, A_, out=U, workspace=ws, sync_check=False), 3, 2,
                             stream)
        # with the exact self term (G(0) = 1 for the self pair and coincident pairs)
        pex = fgt.Plan(1.0, eps, exact_self=True)
        ms_ex = _event_time(lambda: fgt.transform_self(pex, X, A_, out=U, workspace=ws, sync_check=False), 3, 2,
                            stream)
        fgt.transform_self(pex, X, A_, out=U, workspace=ws)
        out.append({"points": "uniform", "eps": eps, "n_e": plan.n_e, "points_per_s": world * N / (ms_self * 1e-3),
                     "ms": ms_self, "general_path_on_x_x_ms": ms_gen, "speedup": ms_gen / ms_self,
                     "exact_self_ms": ms_ex})
        del ws
        torch.cuda.empty_cache()
    # the FP32 sweeps on the same points
    p32 = fgt.Plan(1.0, 1e-6, precision="fp32")
    ws = fgt.Workspace(dev)
    ms32 = _event_time(lambda: fgt.transform_self(p32, X, A_, out=U, workspace=ws, sync_check=False), 3, 3, stream)
    fgt.transform_self(p32, X, A_, out=U, workspace=ws)
    out.append({"points": "uniform", "precision": "fp32", "eps": 1e-6, "n_e": p32.n_e,
                "points_per_s": world * N / (ms32 * 1e-3), "ms": ms32})
    del ws
    torch.cuda.empty_cache()
    # Sec. 5's second point set: Chebyshev points on [0, 1]
    from paper_1909_09825_gb300 import inputs
    xc, _ = inputs.chebyshev(N, seed=0)
    XC = torch.from_numpy(xc).to(dev)
    plan = fgt.Plan(1.0, 1e-6)
    ws = fgt.Workspace(dev)
    ms_c = _event_time(lambda: fgt.transform_self(plan, XC, A_, out=U, workspace=ws, sync_check=False), 3, 3, stream)
    fgt.transform_self(plan, XC, A_, out=U, workspace=ws)
    out.append({"points": "chebyshev (generated in increasing order: the sort is one merge)", "eps": 1e-6,
                "n_e": plan.n_e, "points_per_s": world * N / (ms_c * 1e-3), "ms": ms_c})
    del ws, XC
    torch.cuda.empty_cache()
    return {"workload": "N=2^%d uniform (Table 5.1's shape) or Chebyshev points on [0,1] as targets and sources, "
                        "alpha ~ N(0,1), delta=1, FP64" % int(np.log2(N)), "unit": "N points/s", "runs": out}


def precision_split(args, dev, world, P_unused):
    """Mixture of 8 Gaussians (sigma 1e-3) + 10% uniform, alpha ~ U(-1,1), delta = 1e-4,
    M = N = 2^26: FP32 at eps 1e-6 against FP64 and double-float at eps 1e-6 and 1e-10,
    with errors."""
    import torch
    import paper_1909_09825_gb300 as fgt
    from paper_1909_09825_gb300 import inputs
    M = N = 1 << args.log2
    x, y, a = inputs.mixture(M, N, seed=0)
    X, Y, A = (torch.from_numpy(v).to(dev) for v in (x, y, a))
    out = []
    U = torch.empty(M, dtype=torch.float64, device=dev)
    ws = fgt.Workspace(dev)
    stream = torch.cuda.current_stream(dev)
    for prec, eps in (("fp32", 1e-6), ("fp64", 1e-6), ("fp64", 1e-10), ("f32x2", 1e-6), ("f32x2", 1e-10)):
        plan = fgt.Plan(1e-4, eps, precision=prec)
        ms = _event_time(lambda: fgt.transform(plan, X, Y, A, out=U, workspace=ws, sync_check=False), 3, 2, stream)
        err = sampled_error(plan, X, Y, A, x, y, a, 1e-4, dev)
        out.append({"precision": prec, "eps": eps, "n_e": plan.n_e, "value": world * (M + N) / (ms * 1e-3),
                    "ms_per_step": ms, "error": err})
    fp32, fp64 = out[0], out[1]
    del X, Y, A, U, ws
    torch.cuda.empty_cache()
    return {"workload": "mixture of 8 Gaussians (centres U[0,1], sigma 1e-3) + 10%% uniform, M=N=2^%d, "
                        "alpha ~ U(-1,1), delta=1e-4, seed 0" % args.log2,
            "runs": out, "fp32_speedup_over_fp64_at_eps_1e-6": fp64["ms_per_step"] / fp32["ms_per_step"]}


def differentiation(dev, world, log2=24):
    """M = N = 2^24, delta = 1e-3, eps = 1e-8, L = sum (u_i - sin(2 pi x_i))^2: forward +
    backward (dL/dalpha, dL/dx, dL/dy, dL/ddelta) through the adjoint sweeps."""
    import torch
    import paper_1909_09825_gb300 as fgt
    from paper_1909_09825_gb300 import inputs
    M = N = 1 << log2
    x, y, a = inputs.uniform(M, N, seed=0)
    X, Y, A = (torch.from_numpy(v).to(dev) for v in (x, y, a))
    F = torch.sin(2 * np.pi * X)
    plan = fgt.Plan(1e-3, 1e-8)
    ws = fgt.Workspace(dev)
    stream = torch.cuda.current_stream(dev)
    U = torch.empty(M, dtype=torch.float64, device=dev)

    def fwd():
        fgt.transform(plan, X, Y, A, out=U, workspace=ws, sync_check=False)

    def fwd_bwd():
        fwd()
        g = 2.0 * (U - F)
        fgt.backward(plan, X, Y, A, g, workspace=ws, sync_check=False)

    ms_f = _event_time(fwd, 3, 2, stream)
    ms_fb = _event_time(fwd_bwd, 3, 2, stream)
    del X, Y, A, F, U, ws
    torch.cuda.empty_cache()
    P = M + N
    return {"workload": "M=N=2^%d uniform, alpha ~ N(0,1), delta=1e-3, eps=1e-8 (n_e=%d), "
                        "L=sum(u-sin 2 pi x)^2, grads alpha, x, y, delta" % (log2, plan.n_e),
            "forward_points_per_s": world * P / (ms_f * 1e-3), "forward_ms": ms_f,
            "forward_backward_points_per_s": world * P / (ms_fb * 1e-3), "forward_backward_ms": ms_fb,
            "backward_ms": ms_fb - ms_f}


def batched(dev, world, B=4096, check=True):
    """B = 4096 transforms, M_b = N_b log-uniform in [1e2, 1e6], delta_b log-uniform in
    [1e-6, 1e-1], eps = 1e-6 FP64, one pass of the kernels captured in a CUDA graph.
    With check, 64 sampled items (4 sampled targets each) against the oracle's direct
    Gauss sum over the item's sources."""
    import torch
    import paper_1909_09825_gb300 as fgt
    from paper_1909_09825_gb300 import inputs
    XO, YO, D, X, Y, A, sizes = inputs.batched_device(B, dev, seed=0)
    P = int(2 * sizes.sum())
    plan = fgt.Plan(1.0, 1e-6)
    ws = fgt.Workspace(dev)
    out = torch.empty_like(X)
    tune = plan.autotune_batched(XO, YO, X, Y, A, delta=D, reps=2, workspace=ws)
    fgt.transform_batched(plan, XO, YO, X, Y, A, delta=D, out=out, workspace=ws)
    s = torch.cuda.Stream(dev)
    s.wait_stream(torch.cuda.current_stream(dev))
    g = torch.cuda.CUDAGraph()
    with torch.cuda.stream(s):
        with torch.cuda.graph(g, stream=s):
            fgt.transform_batched(plan, XO, YO, X, Y, A, delta=D, out=out, workspace=ws, stream=s, sync_check=False)
    torch.cuda.current_stream(dev).wait_stream(s)
    ms = _event_time(g.replay, 3, 2, torch.cuda.current_stream(dev))
    err = None
    if check:
        from oracle import oracle
        torch.cuda.synchronize(dev)
        rng = np.random.default_rng(23)
        off = XO.cpu().numpy()
        dl = D.cpu().numpy()
        worst = 0.0
        for b in np.sort(rng.choice(B, 64, replace=False)):
            lo, hi = int(off[b]), int(off[b + 1])
            xs, ys, al = (t[lo:hi].cpu().numpy() for t in (X, Y, A))
            idx = rng.choice(hi - lo, min(4, hi - lo), replace=False)
            ref = oracle.direct(xs[idx], ys, al, float(dl[b]), nthreads=0)
            ug = out[lo:hi].cpu().numpy()[idx]
            worst = max(worst, float(np.max(np.abs(ug - ref)) / np.abs(al).sum()))
        err = {"max_abs_err_over_sum_abs_alpha": worst, "sampled_items": 64, "targets_per_item": 4,
               "reference": "oracle direct FP64 sum over the item's sources"}
    del XO, YO, D, X, Y, A, out, ws, g
    torch.cuda.empty_cache()
    return {"workload": "B=%d items, M_b=N_b=round(10^U(2,6)), delta_b=10^U(-6,-1), uniform x,y, alpha ~ N(0,1), "
                        "eps=1e-6 FP64 (n_e=%d), CUDA graph replay" % (B, plan.n_e),
            "points": P, "value": world * P / (ms * 1e-3), "unit": "points/s", "ms_per_step": ms,
            "tile_threads": plan.tile_threads, "autotune_ms": {str(k): v for k, v in tune.items() if k != "chosen"},
            "error": err}


def _kernel_source_hash():
    """sha256 (16 hex digits) of the sweep kernels' source with comments and blank lines
    removed, so that a record survives edits to comments only."""
    import hashlib
    import re
    src = open(os.path.join(ROOT, "paper_1909_09825_gb300", "csrc", "sweep.cuh")).read()
    code = [re.sub(r"//.*$", "", l).rstrip() for l in src.splitlines()]
    return hashlib.sha256("\n".join(l for l in code if l.strip()).encode()).hexdigest()[:16]


def _traffic_record(plan):
    """DRAM bytes per merged point of the forward sweep from the committed ncu summary,
    used only while the kernel source still matches the one that was profiled."""
    import hashlib
    f = os.path.join(ROOT, "profiles", "sweep_fwd_f64_traffic.txt")
    if not os.path.exists(f):
        return None
    rec = json.load(open(f))
    h = _kernel_source_hash()
    if (rec.get("source_sha256_16") != h or rec.get("n_e") != plan.n_e or
            rec.get("tile_threads") != plan.tile_threads or plan.precision != "fp64"):
        return None
    return rec["dram_bytes_per_point"]


if __name__ == "__main__":
    main()
