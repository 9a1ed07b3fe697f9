"""GPU parity of the full transform (sort + sweeps + evaluate + unpermute) against
the CPU oracle, through the C ABI.

Tolerances
- vs O1 (direct Gauss sum): ||u - u_ref||_inf / sum|alpha| <= 2 eps + 1e-13 (FP64 path)
  and <= 2 eps + 5e-6 (FP32 path).  E_n <= eps bounds the SOE error (eq. 3.1), the
  rest is rounding.
- vs O3 (the paper's recurrence with the SAME SOE, so only rounding differs):
  ||u - u_O3||_inf / sum|alpha| <= TOL_ARITH64 = 1e-12 (FP64).  Both sides lose at most
  a few ulp per multiplier product; the GPU's products are at most R + 2 log2(P) deep,
  the oracle's sequential chain up to P deep, so at P <= 1e5 the bound is
  ~ P * 2^-53 ~ 1e-11 coherent and ~ sqrt(P) 2^-53 typical; 1e-12 leaves a margin of
  about 30 over the typical case and is checked here on every case.
"""
import numpy as np
import pytest
import torch

import paper_1909_09825_gb300 as fgt
from oracle import oracle, soe_cf
from paper_1909_09825_gb300 import inputs

from gpu_util import gpu_transform, rel_inf

pytestmark = pytest.mark.gpu

TOL_ARITH64 = 1e-12
# double-float recurrences: unit roundoff 2^-48 instead of 2^-53, so the FP64 bound
# above scales by 2^5 = 32
TOL_ARITH_DF = 32 * TOL_ARITH64


def oracle_soe_plan(delta, eps, precision="fp64"):
    n, tau, W, En = soe_cf.plan_soe(eps)
    return fgt.Plan(delta, soe=(tau, W), precision=precision), tau, W


def test_small_config_vs_direct(cuda):
    """M = N = 1000, uniform, alpha ~ N(0,1), delta = 1e-3, eps = 1e-6, seed 0."""
    x, y, a = inputs.uniform(1000, 1000, seed=0)
    plan = fgt.Plan(1e-3, 1e-6)
    assert plan.E_n <= 1e-6
    u = gpu_transform(plan, x, y, a)
    ref = oracle.direct(x, y, a, 1e-3)
    assert rel_inf(u, ref, a) <= 2e-6 + 1e-13


@pytest.mark.parametrize("M,N", [(1, 1), (1, 5), (7, 1), (33, 65), (1000, 1000), (2047, 1), (1, 2047),
                                 (2048, 2048), (2049, 2047), (4097, 3000), (12345, 6789), (30001, 29999)])
def test_ragged_vs_recurrence(cuda, M, N):
    x, y, a = inputs.uniform(M, N, seed=M * 7 + N)
    delta, eps = 1e-3, 1e-10
    plan, tau, W = oracle_soe_plan(delta, eps)
    u = gpu_transform(plan, x, y, a)
    ref = oracle.recurrence(x, y, a, delta, tau, W)
    assert rel_inf(u, ref, a) <= TOL_ARITH64


@pytest.mark.parametrize("eps", [1e-3, 1e-6, 1e-8, 1e-10])
@pytest.mark.parametrize("delta", [1e-2, 1e-5])
def test_eps_delta_vs_direct(cuda, eps, delta):
    x, y, a = inputs.uniform(3000, 2500, seed=11)
    plan = fgt.Plan(delta, eps)
    u = gpu_transform(plan, x, y, a)
    ref = oracle.direct(x, y, a, delta)
    assert rel_inf(u, ref, a) <= 2 * eps + 1e-13


def test_ties_and_signed_zeros(cuda):
    x, y, a = inputs.with_ties(5000, 4000, seed=3, n_distinct=50)
    delta = 1e-2
    plan, tau, W = oracle_soe_plan(delta, 1e-10)
    u = gpu_transform(plan, x, y, a)
    ref = oracle.recurrence(x, y, a, delta, tau, W)
    assert rel_inf(u, ref, a) <= TOL_ARITH64


def test_all_points_identical(cuda):
    x = np.full(3000, 0.25)
    y = np.full(2000, 0.25)
    a = np.random.default_rng(1).standard_normal(2000)
    plan, tau, W = oracle_soe_plan(1e-3, 1e-8)
    u = gpu_transform(plan, x, y, a)
    ref = oracle.recurrence(x, y, a, 1e-3, tau, W)
    # coincident pairs get S_n(0) = Re sum W_k (Fig. 4.2 code: weight of an identical source)
    assert np.allclose(ref, np.sum(a) * np.sum(W.real), rtol=0, atol=1e-12 * np.abs(a).sum())
    assert rel_inf(u, ref, a) <= TOL_ARITH64


def test_mixture_vs_recurrence(cuda):
    x, y, a = inputs.mixture(20000, 20000, seed=5)
    delta = 1e-4
    plan, tau, W = oracle_soe_plan(delta, 1e-10)
    u = gpu_transform(plan, x, y, a)
    ref = oracle.recurrence(x, y, a, delta, tau, W)
    assert rel_inf(u, ref, a) <= TOL_ARITH64


@pytest.mark.parametrize("delta", [1e-7, 1e-4, 1e-1, 1e2, 1e4])
def test_delta_sweep_vs_direct(cuda, delta):
    """Fig. 5.2: accuracy over delta = 1e-7..1e4 stays within E_n."""
    x, y, a = inputs.uniform(2000, 2000, seed=21, alpha="pos")
    eps = 1e-8
    plan = fgt.Plan(delta, eps)
    u = gpu_transform(plan, x, y, a)
    ref = oracle.direct(x, y, a, delta)
    assert rel_inf(u, ref, a) <= 2 * eps + 1e-13


def test_hyperbolic_soe_vs_soe_direct(cuda):
    """Any SOE runs through the same kernels: the hyperbolic-contour SOE of Sec. 3.4."""
    tau, W, En = soe_cf.hyperbolic_soe(16)
    x, y, a = inputs.uniform(3000, 3000, seed=8)
    delta = 1e-3
    plan = fgt.Plan(delta, soe=(tau, W))
    u = gpu_transform(plan, x, y, a)
    ref = oracle.soe_direct(x, y, a, delta, tau, W)
    assert rel_inf(u, ref, a) <= TOL_ARITH64


@pytest.mark.parametrize("eps", [1e-3, 1e-6])
def test_fp32_path_vs_direct(cuda, eps):
    x, y, a = inputs.uniform(20000, 20000, seed=13)
    delta = 1e-4
    plan = fgt.Plan(delta, eps, precision="fp32")
    u = gpu_transform(plan, x, y, a)
    ref = oracle.direct(x, y, a, delta, nthreads=0)
    assert rel_inf(u, ref, a) <= 2 * eps + 5e-6


def test_fp32_mixture_vs_direct(cuda):
    x, y, a = inputs.mixture(40000, 40000, seed=2)
    delta, eps = 1e-4, 1e-6
    plan = fgt.Plan(delta, eps, precision="fp32")
    u = gpu_transform(plan, x, y, a)
    idx = np.random.default_rng(0).choice(len(x), 300, replace=False)
    ref = oracle.direct(x[idx], y, a, delta)
    assert rel_inf(u[idx], ref, a) <= 2 * eps + 5e-6


@pytest.mark.parametrize("M,N", [(1, 1), (33, 65), (4097, 3000), (30001, 29999)])
def test_f32x2_ragged_vs_recurrence(cuda, M, N):
    """Double-float recurrences against the oracle's FP64 recurrence, same SOE."""
    x, y, a = inputs.uniform(M, N, seed=M * 5 + N)
    delta = 1e-3
    plan, tau, W = oracle_soe_plan(delta, 1e-10, precision="f32x2")
    u = gpu_transform(plan, x, y, a)
    ref = oracle.recurrence(x, y, a, delta, tau, W)
    assert rel_inf(u, ref, a) <= TOL_ARITH_DF


@pytest.mark.parametrize("eps", [1e-6, 1e-10])
@pytest.mark.parametrize("delta", [1e-5, 1e-1])
def test_f32x2_vs_direct(cuda, eps, delta):
    x, y, a = inputs.uniform(20000, 20000, seed=23)
    plan = fgt.Plan(delta, eps, precision="f32x2")
    u = gpu_transform(plan, x, y, a)
    idx = np.random.default_rng(2).choice(len(x), 400, replace=False)
    ref = oracle.direct(x[idx], y, a, delta)
    assert rel_inf(u[idx], ref, a) <= 2 * eps + 1e-13


@pytest.mark.parametrize("delta", [1e-2, 1e-5])
def test_f32x2_dense_vs_recurrence(cuda, delta):
    """Dense points (|tau| theta below 2^-13 almost everywhere): the double-float
    multipliers take the 1 - tau theta + FP32-tail form."""
    x, y, a = inputs.uniform(1 << 20, 1 << 20, seed=41)
    plan, tau, W = oracle_soe_plan(delta, 1e-10, precision="f32x2")
    u = gpu_transform(plan, x, y, a)
    ref = oracle.recurrence(x, y, a, delta, tau, W)
    assert rel_inf(u, ref, a) <= TOL_ARITH_DF


@pytest.mark.parametrize("delta", [100.0, 10.0, 1.0, 1e-2, 1e-4, 1e-6])
def test_f32x2_matches_fp64_path(cuda, delta):
    """Double-float against the FP64 path on the same plan nodes: every split of the
    double-float Taylor evaluation (head degree J = 1, 2, 3, ... as the gaps grow
    relative to sqrt(delta)) must keep the multipliers at double-float accuracy.  The
    bound is TOL_ARITH64 / 10 relative to sum |alpha| (double-float rounding, 2^-48 per
    step, over up to P = 4e4 steps of a recurrence whose terms cancel as delta grows)."""
    x, y, a = inputs.uniform(20000, 20000, seed=43)
    n, tau, W, En = soe_cf.plan_soe(1e-10)
    u64 = gpu_transform(fgt.Plan(delta, soe=(tau, W)), x, y, a)
    udf = gpu_transform(fgt.Plan(delta, soe=(tau, W), precision="f32x2"), x, y, a)
    err = rel_inf(udf, u64, a)
    print("delta", delta, "f32x2 vs fp64 / sum|alpha|", err, "/ max|u|", np.max(np.abs(udf - u64)) / np.max(np.abs(u64)))
    assert err <= TOL_ARITH64 / 10


@pytest.mark.parametrize("delta", [100.0, 1.0, 1e-2, 1e-4, 1e-6])
def test_fp64_multipliers_at_full_precision(cuda, delta):
    """The FP64 path against the direct SOE sum (O2, compensated, no recurrence) relative
    to max |u|.  At delta = 100 every multiplier is within 1e-5 of 1 and the recurrences
    run over all 4e4 points with cancelling terms, so rounding in the multipliers shows:
    the FP64 path stays below 5e-11 (measured 1.5e-11; the oracle's own FP64 recurrence
    3.5e-11, double-float 1.8e-10), where multipliers good to only 2^-48 would not."""
    x, y, a = inputs.uniform(20000, 20000, seed=47)
    n, tau, W, En = soe_cf.plan_soe(1e-10)
    u = gpu_transform(fgt.Plan(delta, soe=(tau, W)), x, y, a)
    idx = np.arange(0, 20000, 50)
    ref = oracle.soe_direct(x[idx], y, a, delta, tau, W)
    err = np.max(np.abs(u[idx] - ref)) / np.max(np.abs(ref))
    print("delta", delta, "fp64 vs direct SOE sum / max|u|", err)
    assert err <= 5e-11


def test_f32x2_mixture_and_ties(cuda):
    """Clustered points (gaps across many binades) and exact ties / signed zeros."""
    for x, y, a, delta in [(*inputs.mixture(30000, 30000, seed=9), 1e-6), (*inputs.with_ties(5000, 4000, seed=3), 1e-2)]:
        plan, tau, W = oracle_soe_plan(delta, 1e-10, precision="f32x2")
        u = gpu_transform(plan, x, y, a)
        ref = oracle.recurrence(x, y, a, delta, tau, W)
        assert rel_inf(u, ref, a) <= TOL_ARITH_DF


@pytest.mark.parametrize("prec", ["fp64", "fp32", "f32x2"])
@pytest.mark.parametrize("tile", [128, 256])
def test_tile_shapes_vs_recurrence(cuda, prec, tile):
    """Both sweep tile shapes (128 x 32 and 256 x 16 points) in every precision."""
    x, y, a = inputs.uniform(12345, 6789, seed=31)
    delta = 1e-3
    plan, tau, W = oracle_soe_plan(delta, 1e-6 if prec == "fp32" else 1e-10, precision=prec)
    plan.tile_threads = tile
    assert plan.tile_threads == tile
    u = gpu_transform(plan, x, y, a)
    ref = oracle.recurrence(x, y, a, delta, tau, W)
    assert rel_inf(u, ref, a) <= {"fp64": TOL_ARITH64, "f32x2": TOL_ARITH_DF, "fp32": 5e-6}[prec]


@pytest.mark.parametrize("prec", ["fp64", "fp32", "f32x2"])
@pytest.mark.parametrize("nodes", ["cf14", "hyperbolic16"])
def test_term_groups_vs_recurrence(cuda, prec, nodes):
    """Plans of n_e = 7 and 8 terms: at 256 x 16 the value sweeps split the terms into
    groups (two phases A-C per tile); both shapes against the oracle recurrence."""
    if nodes == "cf14":
        n, tau, W, En = soe_cf.plan_soe(1e-10)
    else:
        tau, W, En = soe_cf.hyperbolic_soe(16)
    x, y, a = inputs.mixture(30000, 25000, seed=17)
    delta = 1e-4
    ref = oracle.recurrence(x, y, a, delta, tau, W)
    tol = {"fp64": TOL_ARITH64, "f32x2": TOL_ARITH_DF, "fp32": 5e-6}[prec]
    for tile in (256, 128):
        plan = fgt.Plan(delta, soe=(tau, W), precision=prec)
        plan.tile_threads = tile
        assert rel_inf(gpu_transform(plan, x, y, a), ref, a) <= tol, tile


def test_autotune_picks_the_faster_shape(cuda):
    x, y, a = inputs.uniform(300000, 300000, seed=3)
    X, Y, A = (torch.from_numpy(v).to(cuda) for v in (x, y, a))
    delta = 1e-4
    plan = fgt.Plan(delta, 1e-6)
    res = plan.autotune(X, Y, A, reps=2)
    assert res[128] > 0 and res[256] > 0
    assert res["chosen"] == (128 if res[128] <= res[256] else 256) == plan.tile_threads
    u = fgt.transform(plan, X, Y, A).cpu().numpy()
    idx = np.random.default_rng(1).choice(len(x), 64, replace=False)
    assert rel_inf(u[idx], oracle.direct(x[idx], y, a, delta), a) <= 2e-6 + 1e-13


def test_autotune_cache_file_round_trip(cuda, tmp_path, monkeypatch):
    """With FGT1D_TUNE_CACHE set, the first autotune times both shapes and appends its
    choice; a second plan of the same key reads it back without timing."""
    path = tmp_path / "tune.txt"
    monkeypatch.setenv("FGT1D_TUNE_CACHE", str(path))
    x, y, a = inputs.uniform(200000, 200000, seed=5)
    X, Y, A = (torch.from_numpy(v).to(cuda) for v in (x, y, a))
    first = fgt.Plan(1e-4, 1e-6).autotune(X, Y, A, reps=2)
    assert first[128] > 0 and first[256] > 0
    lines = path.read_text().split()
    assert len(lines) == 6 and int(lines[4]) == first["chosen"]
    plan = fgt.Plan(1e-4, 1e-6)
    second = plan.autotune(X, Y, A, reps=2)
    assert second["chosen"] == first["chosen"] == plan.tile_threads
    assert second[128] < 0 and second[256] < 0  # nothing timed
    assert len(path.read_text().split()) == 6  # nothing appended


def test_empty_inputs(cuda):
    plan = fgt.Plan(1e-3, 1e-6)
    d = cuda
    x = torch.rand(10, dtype=torch.float64, device=d)
    e = torch.empty(0, dtype=torch.float64, device=d)
    u = fgt.transform(plan, x, e, e)
    assert torch.all(u == 0)
    u = fgt.transform(plan, e, x, torch.ones_like(x))
    assert u.numel() == 0


def test_nonfinite_coordinate_reported(cuda):
    plan = fgt.Plan(1e-3, 1e-6)
    x, y, a = inputs.uniform(100, 100, seed=1)
    x[17] = np.nan
    with pytest.raises(fgt._lib.FGTError) as ei:
        gpu_transform(plan, x, y, a)
    assert ei.value.code == fgt._lib.FGT1D_ENONFINITE
    y[3] = np.inf
    x[17] = 0.5
    with pytest.raises(fgt._lib.FGTError) as ei:
        gpu_transform(plan, x, y, a)
    assert ei.value.code == fgt._lib.FGT1D_ENONFINITE
    # the workspace status is cleared: a clean call succeeds afterwards
    y[3] = 0.5
    gpu_transform(plan, x, y, a)


def test_execute_host_matches_device(cuda):
    x, y, a = inputs.uniform(5000, 4000, seed=4)
    plan = fgt.Plan(1e-3, 1e-6)
    u_dev = gpu_transform(plan, x, y, a)
    u_host = fgt.execute_host(plan, x, y, a)
    assert np.array_equal(u_dev, u_host)


def test_execute_host_async_two_streams(cuda):
    """Two fgt1d_execute_host_async calls in flight on two streams with two workspaces
    (pinned host arrays), then a third on the first stream after its wait: each result
    agrees with the device-buffer transform of its inputs to rounding (the look-back's
    order of predecessors depends on timing, as in test_repeat_runs_agree)."""
    plan = fgt.Plan(1e-3, 1e-6)
    runs = [inputs.uniform(70000, 60000, seed=s) for s in (11, 12)]
    pinned = [[torch.from_numpy(v).pin_memory().numpy() for v in r] for r in runs]
    outs = [torch.empty(70000, dtype=torch.float64).pin_memory().numpy() for _ in runs]
    streams = [torch.cuda.Stream(cuda) for _ in runs]
    wss = [fgt.Workspace(cuda) for _ in runs]
    for (x, y, a), o, st, ws in zip(pinned, outs, streams, wss):
        fgt.execute_host(plan, x, y, a, out=o, workspace=ws, stream=st, sync=False)
    for o, st, ws, (x, y, a) in zip(outs, streams, wss, runs):
        fgt.wait_host(ws, st)
        assert rel_inf(o, gpu_transform(plan, x, y, a), a) <= TOL_ARITH64
    x, y, a = pinned[1]
    fgt.execute_host(plan, x, y, a, out=outs[0], workspace=wss[0], stream=streams[0], sync=False)
    fgt.wait_host(wss[0], streams[0])
    assert rel_inf(outs[0], gpu_transform(plan, *runs[1]), runs[1][2]) <= TOL_ARITH64


def test_repeat_runs_agree(cuda):
    """The decoupled look-back adds a timing-dependent set of predecessor aggregates,
    so repeated runs may differ in rounding only (never by more than TOL_ARITH64)."""
    x, y, a = inputs.uniform(50000, 50000, seed=6)
    plan = fgt.Plan(1e-4, 1e-10)
    u1 = gpu_transform(plan, x, y, a)
    u2 = gpu_transform(plan, x, y, a)
    assert rel_inf(u1, u2, a) <= TOL_ARITH64


def test_exact_self_term(cuda):
    """FGT1D_EXACT_SELF: coincident pairs get G(0) = 1 (oracle recurrence, exact_self)."""
    x, y, a = inputs.with_ties(6000, 5000, seed=12, n_distinct=300)
    delta = 1e-3
    n, tau, W, En = soe_cf.plan_soe(1e-8)
    plan = fgt.Plan(delta, soe=(tau, W), exact_self=True)
    u = gpu_transform(plan, x, y, a)
    ref = oracle.recurrence(x, y, a, delta, tau, W, exact_self=True)
    assert rel_inf(u, ref, a) <= TOL_ARITH64
    plan2 = fgt.Plan(delta, 1e-8, exact_self=True)
    u2 = gpu_transform(plan2, x, y, a)
    assert rel_inf(u2, oracle.direct(x, y, a, delta), a) <= 2e-8 + 1e-13


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_presorted_inputs_vs_recurrence(cuda, prec):
    """Presorted targets and sources (Sec. 5's pre-sorted points: the sort is one merge)."""
    x, y, a = inputs.uniform(30001, 25000, seed=41)
    x, y = np.sort(x), np.sort(y)
    delta = 1e-4
    plan, tau, W = oracle_soe_plan(delta, 1e-6 if prec == "fp32" else 1e-10, precision=prec)
    u = gpu_transform(plan, x, y, a)
    ref = oracle.recurrence(x, y, a, delta, tau, W)
    assert rel_inf(u, ref, a) <= {"fp64": TOL_ARITH64, "fp32": 5e-6}[prec]


@pytest.mark.parametrize("delta", [1e-5, 1e-2, 1.0])
def test_eps_1e12_order_16_vs_direct(cuda, delta):
    """eps = 1e-12 plans the CF order n = 16 (n_e = 8, built in double-double, Sec. 3.3):
    M = N = 2^20 uniform points against the direct Gauss sum (eq. 1.1) at 2000 sampled
    targets plus the extremes, within 2 eps + 1e-13."""
    M = N = 1 << 20
    x, y, a = inputs.uniform(M, N, seed=61)
    plan = fgt.Plan(delta, 1e-12)
    assert plan.n == 16 and plan.n_e == 8
    u = gpu_transform(plan, x, y, a)
    rng = np.random.default_rng(62)
    idx = np.unique(np.concatenate([[int(np.argmin(x)), int(np.argmax(x))], rng.choice(M, 2000, replace=False)]))
    ref = oracle.direct(x[idx], y, a, delta, nthreads=0)
    assert rel_inf(u[idx], ref, a) <= 2e-12 + 1e-13
