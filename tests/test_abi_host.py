"""CPU checks of the C ABI: the library loads, exports every declared symbol, and its
host-side parts (the SOE generator of step a0, plan selection, argument checks and
workspace sizing) behave, without touching a GPU."""
import ctypes
import os
import re

import numpy as np
import pytest

from oracle import soe_cf

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def L():
    from paper_1909_09825_gb300 import build, _lib
    build.build()
    return _lib.lib()


def declared_symbols():
    src = ""
    for f in os.listdir(os.path.join(ROOT, "include")):
        if f.endswith(".h"):
            src += open(os.path.join(ROOT, "include", f)).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(fgt1d_\w+)\s*\(", src)))


def test_exports_every_declared_symbol(L):
    names = declared_symbols()
    assert len(names) >= 14
    for n in names:
        assert hasattr(L, n), n
    from paper_1909_09825_gb300 import _lib
    assert set(_lib.SIGNATURES) == set(names)


@pytest.mark.parametrize("n", [2, 4, 6, 8, 10, 12, 14])
def test_soe_generator_matches_oracle(L, n):
    """The product's C++ CF generator and the oracle's numpy one are independent
    implementations of the same construction: same E_n, same nodes (to the problem's
    conditioning, which grows with n)."""
    import paper_1909_09825_gb300 as fgt
    tau, W, En = fgt.soe_cf(n)
    ot, oW, oE = soe_cf.cf_soe(n)
    assert abs(En / oE - 1) < (0.05 if n < 14 else 0.2)
    tol = {2: 1e-12, 4: 1e-12, 6: 1e-10, 8: 1e-9, 10: 1e-7, 12: 1e-5, 14: 2e-3}[n]
    assert np.max(np.abs(W - oW)) / np.max(np.abs(oW)) < tol
    assert np.max(np.abs(tau - ot)) / np.max(np.abs(ot)) < tol
    assert np.all(tau.real > 0) and np.all(tau.imag > 0)
    # the product's E_n claim holds on an independent grid
    x = np.concatenate([[0.0], np.linspace(0, 15, 300001)])
    assert np.max(np.abs(np.exp(-x * x / 4) - soe_cf.soe_eval(tau, W, x))) <= En * 1.01


@pytest.mark.parametrize("eps", [0.1, 1e-3, 1e-6, 1e-8, 1e-10, 5e-12])
def test_plan_picks_smallest_n(L, eps):
    import paper_1909_09825_gb300 as fgt
    p = fgt.Plan(0.37, eps)
    assert p.E_n <= eps
    assert p.n == 2 or fgt.soe_cf(p.n - 2)[2] > eps
    assert p.n_e == p.n // 2 and abs(p.delta - 0.37) == 0


def test_plan_errors(L):
    import paper_1909_09825_gb300 as fgt
    from paper_1909_09825_gb300 import _lib
    for args in [(0.0, 1e-6), (-1.0, 1e-6), (float("nan"), 1e-6), (float("inf"), 1e-6), (1.0, 0.0), (1.0, 0.7)]:
        with pytest.raises(_lib.FGTError) as e:
            fgt.Plan(*args)
        assert e.value.code == _lib.FGT1D_EINVAL
    with pytest.raises(_lib.FGTError) as e:
        fgt.Plan(1.0, 1e-14)
    assert e.value.code == _lib.FGT1D_EUNSUPPORTED
    with pytest.raises(_lib.FGTError) as e:
        fgt.Plan(1.0, 1e-8, precision="fp32")
    assert e.value.code == _lib.FGT1D_EUNSUPPORTED
    with pytest.raises(_lib.FGTError) as e:
        fgt.Plan(1.0, soe=([-1.0 + 1j], [1.0]))
    assert e.value.code == _lib.FGT1D_EINVAL
    assert L.fgt1d_plan_create(ctypes.c_double(1.0), ctypes.c_double(1e-6), 0, None) == _lib.FGT1D_EINVAL
    assert L.fgt1d_plan_create(ctypes.c_double(1.0), ctypes.c_double(1e-6), 8, ctypes.byref(ctypes.c_void_p())) == _lib.FGT1D_EINVAL
    # FP32 and double-float exclude each other
    assert L.fgt1d_plan_create(ctypes.c_double(1.0), ctypes.c_double(1e-6), _lib.FGT1D_FP32 | _lib.FGT1D_F32X2,
                               ctypes.byref(ctypes.c_void_p())) == _lib.FGT1D_EINVAL
    p = fgt.Plan(1.0, 1e-10, precision="f32x2")
    assert p.E_n <= 1e-10
    assert L.fgt1d_soe_cf(7, *([None] * 6)) == _lib.FGT1D_EINVAL


def test_tile_shape_setting(L):
    import paper_1909_09825_gb300 as fgt
    from paper_1909_09825_gb300 import _lib
    assert fgt.Plan(1.0, 1e-6).tile_threads == 256
    assert fgt.Plan(1.0, 1e-6, precision="fp32").tile_threads == 256
    p = fgt.Plan(1.0, 1e-10, precision="f32x2")
    assert p.tile_threads == 256
    p.tile_threads = 128
    assert p.tile_threads == 128
    p.tile_threads = 0
    assert p.tile_threads == 256
    for bad in (64, 512, -1):
        with pytest.raises(_lib.FGTError) as e:
            p.tile_threads = bad
        assert e.value.code == _lib.FGT1D_EINVAL
    assert L.fgt1d_plan_set_tile(None, 128) == _lib.FGT1D_EINVAL
    assert L.fgt1d_autotune(p.handle, 1, None, None, None, None, 0, None, None, 0, None, None, 0, 0, None, None,
                            None) == _lib.FGT1D_EINVAL  # reps < 1


def test_geometry_argument_errors(L):
    import paper_1909_09825_gb300 as fgt
    from paper_1909_09825_gb300 import _lib
    b = ctypes.c_size_t()
    p64 = fgt.Plan(1e-3, 1e-6)
    assert L.fgt1d_geometry_workspace_size(p64.handle, 1000, 2000, ctypes.byref(b)) == _lib.FGT1D_OK
    n = ctypes.c_size_t()
    assert L.fgt1d_workspace_size(p64.handle, 1000, 2000, ctypes.byref(n)) == _lib.FGT1D_OK
    assert b.value == n.value  # the bound state is the transform's workspace
    p32 = fgt.Plan(1e-3, 1e-6, precision="fp32")
    b32 = ctypes.c_size_t()
    assert L.fgt1d_geometry_workspace_size(p32.handle, 1000, 2000, ctypes.byref(b32)) == _lib.FGT1D_OK
    assert b32.value < b.value  # FP32: sorted points, no multiplier table
    pdf = fgt.Plan(1e-3, 1e-6, precision="f32x2")
    assert L.fgt1d_geometry_workspace_size(pdf.handle, 1000, 2000, ctypes.byref(b)) == _lib.FGT1D_OK
    assert L.fgt1d_geometry_workspace_size(p64.handle, -1, 2000, ctypes.byref(b)) == _lib.FGT1D_EINVAL
    assert L.fgt1d_geometry_bind(p64.handle, None, 10, None, 10, None, 0, None) == _lib.FGT1D_EWORKSPACE
    assert L.fgt1d_geometry_apply(None, 10, 10, None, None, None, 0, None) == _lib.FGT1D_EINVAL
    assert L.fgt1d_geometry_apply(p64.handle, 0, 10, None, None, None, 0, None) == _lib.FGT1D_OK  # M = 0: no-op


def test_self_argument_errors(L):
    import paper_1909_09825_gb300 as fgt
    from paper_1909_09825_gb300 import _lib
    b = ctypes.c_size_t()
    assert L.fgt1d_self_workspace_size(fgt.Plan(1e-3, 1e-6).handle, 5000, ctypes.byref(b)) == _lib.FGT1D_OK
    n = ctypes.c_size_t()
    assert L.fgt1d_workspace_size(fgt.Plan(1e-3, 1e-6).handle, 0, 5000, ctypes.byref(n)) == _lib.FGT1D_OK
    assert b.value == n.value  # N merged points, not 2N
    assert L.fgt1d_self_workspace_size(fgt.Plan(1e-3, 1e-6, precision="f32x2").handle, 5000,
                                       ctypes.byref(b)) == _lib.FGT1D_EUNSUPPORTED
    assert L.fgt1d_self_workspace_size(fgt.Plan(1e-3, 1e-6, precision="fp32").handle, 5000,
                                       ctypes.byref(b)) == _lib.FGT1D_OK
    assert L.fgt1d_self_workspace_size(fgt.Plan(1e-3, 1e-6, exact_self=True).handle, 5000,
                                       ctypes.byref(b)) == _lib.FGT1D_OK
    assert L.fgt1d_execute_self(None, None, 10, None, None, None, 0, None) == _lib.FGT1D_EINVAL
    assert L.fgt1d_execute_self(fgt.Plan(1e-3, 1e-6).handle, None, 0, None, None, None, 0, None) == _lib.FGT1D_OK


def test_workspace_size_and_bounds(L):
    import paper_1909_09825_gb300 as fgt
    from paper_1909_09825_gb300 import _lib
    p = fgt.Plan(1e-3, 1e-6)
    a, b = p.workspace_size(1000, 1000), p.workspace_size(1 << 20, 1 << 20)
    assert 0 < a < b
    assert p.workspace_size(1 << 20, 1 << 20, host=True) >= b + 4 * 8 * (1 << 20)
    sz = ctypes.c_size_t()
    assert L.fgt1d_workspace_size(p.handle, -1, 5, ctypes.byref(sz)) == _lib.FGT1D_EINVAL
    assert L.fgt1d_workspace_size(p.handle, 1 << 30, 1 << 30, ctypes.byref(sz)) == _lib.FGT1D_EINVAL
    assert L.fgt1d_workspace_size(p.handle, (1 << 30) - 1, 1 << 30, ctypes.byref(sz)) == _lib.FGT1D_OK
    # execute rejects a missing or short workspace before touching the device
    x = (ctypes.c_double * 4)()
    assert L.fgt1d_execute(p.handle, x, 4, x, x, 4, x, None, 0, None) == _lib.FGT1D_EWORKSPACE
    assert L.fgt1d_execute(p.handle, None, 4, x, x, 4, x, None, 0, None) == _lib.FGT1D_EINVAL
    assert L.fgt1d_strerror(3).decode().startswith("a coordinate")


def test_product_imports_no_oracle():
    """The product package never reaches into the oracle."""
    pkg = os.path.join(ROOT, "paper_1909_09825_gb300")
    for dp, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".cpp", ".h")):
                txt = open(os.path.join(dp, f)).read()
                assert not re.search(r"^\s*(from|import)\s+oracle|#include.*oracle|liboracle", txt, re.M), f


def test_noalloc_rejects_null_arrays_before_the_gpu(L):
    """The no-allocation entry point applies fgt1d_execute's pointer rules on the host:
    a NULL array with a nonzero size is FGT1D_EINVAL, returned before any CUDA call
    (this container has no GPU, so reaching the device would give FGT1D_ECUDA)."""
    import paper_1909_09825_gb300 as fgt
    from paper_1909_09825_gb300 import _lib
    p = fgt.Plan(1e-3, 1e-6)
    v = (ctypes.c_double * 8)()
    f = L.fgt1d_execute_noalloc
    assert f(p.handle, None, 8, v, v, 8, v, None) == _lib.FGT1D_EINVAL     # x
    assert f(p.handle, v, 8, v, v, 8, None, None) == _lib.FGT1D_EINVAL     # u
    assert f(p.handle, v, 8, None, v, 8, v, None) == _lib.FGT1D_EINVAL     # y
    assert f(p.handle, v, 8, v, None, 8, v, None) == _lib.FGT1D_EINVAL     # alpha
    assert f(None, v, 8, v, v, 8, v, None) == _lib.FGT1D_EINVAL            # plan
    assert f(p.handle, v, 40000, v, v, 30000, v, None) == _lib.FGT1D_ETOOLARGE
    assert f(p.handle, None, 0, None, None, 0, None, None) == _lib.FGT1D_OK  # nothing to do


def test_cf_order_16_in_double_double(L):
    """n = 16, built in double-double (Sec. 3.3 builds its largest orders in extended
    precision): the claimed E_16 bounds |G - S_16| evaluated in extended precision on an
    independent grid, the error keeps falling at the paper's geometric rate (about 7.5
    per order, so E_14 / E_16 well above 20), the nodes keep Re tau > 0 with one of each
    conjugate pair, and eps = 1e-12 now plans n = 16."""
    import paper_1909_09825_gb300 as fgt
    tau, W, E16 = fgt.soe_cf(16)
    _, _, E14 = fgt.soe_cf(14)
    assert len(tau) == 8 and E16 <= 2e-13
    assert np.all(tau.real > 0) and np.all(tau.imag > 0)
    x = np.concatenate([[0.0], np.linspace(0, 15, 150001), np.geomspace(1e-6, 1e-2, 20001)]).astype(np.longdouble)
    t, w = tau.astype(np.clongdouble), W.astype(np.clongdouble)
    S = np.real(np.sum(w[:, None] * np.exp(-t[:, None] * x[None, :]), axis=0))
    true_err = float(np.max(np.abs(np.exp(-x * x / 4) - S)))
    assert true_err <= E16
    assert E14 / true_err > 20
    assert abs(float(S[0]) - 1.0) <= E16
    p = fgt.Plan(1e-3, 1e-12)
    assert p.n == 16 and p.n_e == 8 and p.E_n == E16


def test_measure_peaks_rejects_null_output(L):
    from paper_1909_09825_gb300 import _lib
    assert L.fgt1d_measure_peaks(None, None) == _lib.FGT1D_EINVAL


def test_segment_entry_points_check_arguments_on_the_host(L):
    """The segment calls reject bad arguments before any GPU work."""
    import paper_1909_09825_gb300 as fgt
    from paper_1909_09825_gb300 import _lib
    p = fgt.Plan(1e-3, 1e-6)
    v = (ctypes.c_double * 64)()
    assert L.fgt1d_segment_execute(p.handle, v, 4, v, v, 4, v, None, v, 0, None) == _lib.FGT1D_EINVAL  # boundary
    assert L.fgt1d_segment_execute(p.handle, None, 4, v, v, 4, v, v, v, 0, None) == _lib.FGT1D_EINVAL  # x
    assert L.fgt1d_segment_execute(p.handle, v, 4, v, v, 4, v, v, None, 0, None) == _lib.FGT1D_EWORKSPACE
    assert L.fgt1d_segment_apply(p.handle, 4, 4, None, v, v, 0, None) == _lib.FGT1D_EINVAL
    assert L.fgt1d_segment_apply(p.handle, 0, 4, None, None, None, 0, None) == _lib.FGT1D_OK  # no targets
    assert L.fgt1d_segment_compose(p.handle, 2, 2, v, v) == _lib.FGT1D_EINVAL                    # g out of range
    assert L.fgt1d_segment_compose(None, 1, 0, v, v) == _lib.FGT1D_EINVAL


def test_autotune_takes_a_cached_choice_without_timing(L, tmp_path, monkeypatch):
    """With FGT1D_TUNE_CACHE naming a file that holds a choice for this workload's key
    (precision flags, n_e, floor(log2(M + N)), single/batched), fgt1d_autotune takes it
    without running anything on the device (ms_out stays -1); other keys do not match."""
    import paper_1909_09825_gb300 as fgt
    from paper_1909_09825_gb300 import _lib
    p = fgt.Plan(1e-3, 1e-6)  # FP64, n_e = 5
    cache = tmp_path / "tune.txt"
    cache.write_text("0 5 10 1 256 1.0\n1 5 10 0 256 1.0\n0 5 10 0 128 3.25\n")
    monkeypatch.setenv("FGT1D_TUNE_CACHE", str(cache))
    monkeypatch.delenv("FGT1D_TILE_THREADS", raising=False)
    v = (ctypes.c_double * 4)()  # never read on a cache hit
    chosen, ms = ctypes.c_int(), (ctypes.c_float * 2)()
    rc = L.fgt1d_autotune(p.handle, 1, None, None, None, v, 1000, v, v, 1000, v, v, 1 << 20, 2, None,
                          ctypes.byref(chosen), ms)
    assert rc == _lib.FGT1D_OK and chosen.value == 128 and p.tile_threads == 128
    assert list(ms) == [-1.0, -1.0]


def test_execute_host_async_argument_errors(L):
    """The asynchronous host-buffer entry point checks its arguments on the host, as the
    synchronous one does, before any CUDA call; M = 0 is a no-op and N = 0 writes u = 0
    at once (host memory, no GPU needed)."""
    import paper_1909_09825_gb300 as fgt
    from paper_1909_09825_gb300 import _lib
    p = fgt.Plan(1e-3, 1e-6)
    v = (ctypes.c_double * 8)(*range(8))
    f = L.fgt1d_execute_host_async
    assert f(p.handle, None, 8, v, v, 8, v, None, 0, None) == _lib.FGT1D_EINVAL     # x
    assert f(p.handle, v, 8, None, v, 8, v, None, 0, None) == _lib.FGT1D_EINVAL     # y
    assert f(p.handle, v, 8, v, None, 8, v, None, 0, None) == _lib.FGT1D_EINVAL     # alpha
    assert f(p.handle, v, 8, v, v, 8, None, None, 0, None) == _lib.FGT1D_EINVAL     # u
    assert f(None, v, 8, v, v, 8, v, None, 0, None) == _lib.FGT1D_EINVAL            # plan
    assert f(p.handle, v, -1, v, v, 8, v, None, 0, None) == _lib.FGT1D_EINVAL       # size
    assert f(p.handle, None, 0, v, v, 8, None, None, 0, None) == _lib.FGT1D_OK      # M = 0
    assert f(p.handle, v, 8, None, None, 0, v, None, 0, None) == _lib.FGT1D_OK      # N = 0
    assert list(v) == [0.0] * 8
