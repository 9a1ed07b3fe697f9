"""ctypes loader and numpy wrappers for the C oracle (test infrastructure only).

``build()`` compiles ``fgt_oracle.c`` with gcc into ``liboracle.so`` beside it.
Every wrapper takes and returns float64 numpy arrays; the SOE node set is the
halved one (tau_k, W_k) of ``oracle.soe_cf``.
"""
import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "fgt_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lib = None


def build(force=False):
    """Compile the oracle (gcc, FP64, no FMA contraction, OpenMP when available)."""
    if not force and os.path.exists(_LIB) and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC):
        return _LIB
    base = ["gcc", "-O2", "-fPIC", "-shared", "-ffp-contract=off", "-fno-fast-math", _SRC, "-o", _LIB, "-lm"]
    try:
        subprocess.run(base[:1] + ["-fopenmp"] + base[1:], check=True, capture_output=True)
    except subprocess.CalledProcessError:
        subprocess.run(base, check=True, capture_output=True)
    return _LIB


def lib():
    global _lib
    if _lib is None:
        build()
        L = ctypes.CDLL(_LIB)
        d, i64, i32, p = ctypes.c_double, ctypes.c_int64, ctypes.c_int, ctypes.c_void_p
        L.o1_direct.argtypes = [p, i64, p, p, i64, d, p, i32]
        L.o2_soe_direct.argtypes = [p, i64, p, p, i64, d, i32, p, p, p, p, p, i32]
        L.o3_recurrence.argtypes = [p, i64, p, p, i64, d, i32, p, p, p, p, i32, p, p]
        L.o3_recurrence.restype = i32
        L.o3_recurrence_self.argtypes = [p, p, i64, d, i32, p, p, p, p, i32, p]
        L.o3_recurrence_self.restype = i32
        L.o3_sort_merged.argtypes = [p, i64, p, i64, p]
        L.o3_sort_merged.restype = i32
        L.o3_sort_merged_par.argtypes = [p, i64, p, i64, p, i32]
        L.o3_sort_merged_par.restype = i32
        L.o3_recurrence_par.argtypes = [p, i64, p, p, i64, d, i32, p, p, p, p, i32, i32, i32, p, p]
        L.o3_recurrence_par.restype = i32
        L.o3_segment_boundary.argtypes = [p, i64, p, p, i64, d, i32, p, p, p]
        L.o3_carry_apply.argtypes = [p, i64, d, i32, p, p, p, p, p, p]
        L.o1_grad.argtypes = [p, i64, p, p, i64, d, p, p, p, p, p]
        L.o2_grad.argtypes = [p, i64, p, p, i64, d, i32, p, p, p, p, p, p, p, p, p]
        L.oracle_openmp_max_threads.restype = i32
        _lib = L
    return _lib


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def _ptr(a):
    return a.ctypes.data_as(ctypes.c_void_p)


def _soe(tau, W):
    tau = np.asarray(tau, dtype=complex)
    W = np.asarray(W, dtype=complex)
    return (len(tau), _f64(tau.real), _f64(tau.imag), _f64(W.real), _f64(W.imag))


def max_threads():
    return lib().oracle_openmp_max_threads()


def direct(x, y, alpha, delta, nthreads=0):
    """O1: u_i = sum_j alpha_j exp(-(x_i - y_j)^2 / (4 delta))."""
    x, y, alpha = _f64(x), _f64(y), _f64(alpha)
    u = np.empty(len(x))
    lib().o1_direct(_ptr(x), len(x), _ptr(y), _ptr(alpha), len(y), float(delta), _ptr(u), int(nthreads))
    return u


def soe_direct(x, y, alpha, delta, tau, W, nthreads=0):
    """O2: u_i = sum_j alpha_j Re sum_k W_k exp(-tau_k |x_i - y_j| / sqrt(delta))."""
    x, y, alpha = _f64(x), _f64(y), _f64(alpha)
    n, tr, ti, wr, wi = _soe(tau, W)
    u = np.empty(len(x))
    lib().o2_soe_direct(_ptr(x), len(x), _ptr(y), _ptr(alpha), len(y), float(delta), n,
                        _ptr(tr), _ptr(ti), _ptr(wr), _ptr(wi), _ptr(u), int(nthreads))
    return u


def recurrence(x, y, alpha, delta, tau, W, exact_self=False, return_perm=False):
    """O3: the paper's sort + forward/backward recurrences (single thread)."""
    x, y, alpha = _f64(x), _f64(y), _f64(alpha)
    n, tr, ti, wr, wi = _soe(tau, W)
    u = np.empty(len(x))
    perm = np.empty(len(x) + len(y), dtype=np.int64)
    rc = lib().o3_recurrence(_ptr(x), len(x), _ptr(y), _ptr(alpha), len(y), float(delta), n,
                             _ptr(tr), _ptr(ti), _ptr(wr), _ptr(wi), int(bool(exact_self)), _ptr(u), _ptr(perm))
    if rc != 0:
        raise ValueError("oracle recurrence failed: %d" % rc)
    return (u, perm) if return_perm else u


def recurrence_self(x, alpha, delta, tau, W, exact_self=False):
    """O3 for identical targets and sources (Fig. 4.1): one sort of the N points,
    inclusive forward and exclusive backward recurrences; exact_self gives the self
    pair and every coincident pair G(0) = 1 instead of S_n(0)."""
    x, alpha = _f64(x), _f64(alpha)
    n, tr, ti, wr, wi = _soe(tau, W)
    u = np.empty(len(x))
    rc = lib().o3_recurrence_self(_ptr(x), _ptr(alpha), len(x), float(delta), n, _ptr(tr), _ptr(ti), _ptr(wr),
                                  _ptr(wi), int(bool(exact_self)), _ptr(u))
    if rc != 0:
        raise ValueError("oracle self recurrence failed: %d" % rc)
    return u


def recurrence_par(x, y, alpha, delta, tau, W, exact_self=False, nseg=None, nthreads=0, return_perm=False):
    """O3 on several host cores: the same sort and recurrences over nseg coordinate
    segments (default 8 per thread), carries composed with direct span exponentials."""
    x, y, alpha = _f64(x), _f64(y), _f64(alpha)
    n, tr, ti, wr, wi = _soe(tau, W)
    threads = nthreads if nthreads > 0 else max_threads()
    if nseg is None:
        nseg = 8 * threads
    u = np.empty(len(x))
    perm = np.empty(len(x) + len(y), dtype=np.int64) if return_perm else None
    rc = lib().o3_recurrence_par(_ptr(x), len(x), _ptr(y), _ptr(alpha), len(y), float(delta), n,
                                 _ptr(tr), _ptr(ti), _ptr(wr), _ptr(wi), int(bool(exact_self)), int(nseg),
                                 int(nthreads), _ptr(u), _ptr(perm) if return_perm else None)
    if rc != 0:
        raise ValueError("oracle parallel recurrence failed: %d" % rc)
    return (u, perm) if return_perm else u


def sort_merged_par(x, y, nthreads=0):
    """sort_merged on several threads (the same stable order, bit for bit)."""
    x, y = _f64(x), _f64(y)
    perm = np.empty(len(x) + len(y), dtype=np.int64)
    rc = lib().o3_sort_merged_par(_ptr(x), len(x), _ptr(y), len(y), _ptr(perm), int(nthreads))
    if rc != 0:
        raise ValueError("oracle parallel sort failed: %d" % rc)
    return perm


def segment_boundary(x, y, alpha, delta, tau, W):
    """A segment's boundary record (4 n_e + 2 values: Re F, Im F, Re G, Im G, z_first,
    z_last) by direct sums over its sources."""
    x, y, alpha = _f64(x), _f64(y), _f64(alpha)
    n, tr, ti, _, _ = _soe(tau, W)
    out = np.empty(4 * n + 2)
    lib().o3_segment_boundary(_ptr(x), len(x), _ptr(y), _ptr(alpha), len(y), float(delta), n, _ptr(tr), _ptr(ti),
                              _ptr(out))
    return out


def carry_apply(x, u, delta, tau, W, carry):
    """u + the contribution of a carry record (F_in, G_in, z_prev, z_next) at targets x."""
    x = _f64(x)
    n, tr, ti, wr, wi = _soe(tau, W)
    u = np.array(u, dtype=np.float64, copy=True)
    carry = _f64(carry)
    lib().o3_carry_apply(_ptr(x), len(x), float(delta), n, _ptr(tr), _ptr(ti), _ptr(wr), _ptr(wi), _ptr(carry),
                         _ptr(u))
    return u


def sort_merged(x, y):
    """Stable order of the merged array [y_0..y_{N-1}, x_0..x_{M-1}] by coordinate."""
    x, y = _f64(x), _f64(y)
    perm = np.empty(len(x) + len(y), dtype=np.int64)
    rc = lib().o3_sort_merged(_ptr(x), len(x), _ptr(y), len(y), _ptr(perm))
    if rc != 0:
        raise ValueError("oracle sort failed: %d" % rc)
    return perm


def grad_direct(x, y, alpha, delta, g):
    """Direct gradients of L = sum_i g_i u_i for the Gaussian kernel."""
    x, y, alpha, g = _f64(x), _f64(y), _f64(alpha), _f64(g)
    gx, gy, ga = np.empty(len(x)), np.empty(len(y)), np.empty(len(y))
    gd = np.zeros(1)
    lib().o1_grad(_ptr(x), len(x), _ptr(y), _ptr(alpha), len(y), float(delta), _ptr(g),
                  _ptr(gx), _ptr(gy), _ptr(ga), _ptr(gd))
    return gx, gy, ga, float(gd[0])


def grad_soe(x, y, alpha, delta, tau, W, g):
    """Direct gradients of L = sum_i g_i u_i for the SOE kernel (the implemented operator)."""
    x, y, alpha, g = _f64(x), _f64(y), _f64(alpha), _f64(g)
    n, tr, ti, wr, wi = _soe(tau, W)
    gx, gy, ga = np.empty(len(x)), np.empty(len(y)), np.empty(len(y))
    gd = np.zeros(1)
    lib().o2_grad(_ptr(x), len(x), _ptr(y), _ptr(alpha), len(y), float(delta), n,
                  _ptr(tr), _ptr(ti), _ptr(wr), _ptr(wi), _ptr(g), _ptr(gx), _ptr(gy), _ptr(ga), _ptr(gd))
    return gx, gy, ga, float(gd[0])
