"""Oracle SOE construction for the Gaussian kernel (test infrastructure only).

The sum-of-exponentials (SOE) approximation of eq. 1.3,

    G(x; delta) = exp(-x^2 / (4 delta)) ~ S_n(x; delta) = sum_k w_k exp(-t_k |x| / sqrt(delta)),

is obtained (Sec. 2.3) from a sum-of-poles rational function
r(z) = sum_k c_k / (z - z_k) that approximates e^z on (-inf, 0] (eq. 2.13),
through eq. 2.11:  w_k = -c_k sqrt(pi / z_k),  t_k = sqrt(z_k).
The poles and residues are those of the Caratheodory-Fejer (CF) near-best
rational approximation of e^z on the negative real axis, which the paper takes
from the 2006 CF construction of Trefethen, Weideman and Schmelzer (Sec. 3.3).
That construction is written out below from its published description:

1. map z in (-inf, 0] to s in (-1, 1] by z = a (s - 1) / (s + 1), so that
   F(s) = exp(a (s - 1)/(s + 1)) is smooth on [-1, 1] with F(-1) = 0;
2. take the Fourier coefficients c_0..c_K of F(cos phi) (for j >= 1 these are
   half the Chebyshev coefficients) and the analytic part f(v) = sum_j c_j v^j
   on the unit circle v = e^{i phi};
3. form the K x K Hankel matrix H[i, j] = c_{i+j+1}; its (n+1)-th singular value
   sigma_n and singular vectors (u, v) give the CF extension
       rt(v) = f(v) - sigma_n v^K u(v) / vrev(v),   vrev(v) = sum_j v_j v^{K-1-j},
   whose n poles outside the unit disk are the zeros q_k of vrev with |q_k| > 1;
4. the rational part of rt is p(v) / prod_k (v - q_k), with p the polynomial
   formed by the Laurent coefficients 0..n of rt(v) prod_k (v - q_k); its
   residues in v are p(q_k) / prod_{l != k} (q_k - q_l);
5. map back: z_k = a (q_k - 1)^2 / (q_k + 1)^2 and the residue in z is the
   residue in v times dz/dv(q_k) = 4 z_k / (q_k^2 - 1).

The transform only needs one member of each conjugate pair with doubled weight
(Sec. 4: "only half of them are needed"), so ``halve`` keeps Im t_k > 0 and
returns (tau_k, W_k = 2 w_k).

Parameters a, K and the FFT length L are not given in the paper (the cited
code is not reproduced there); they are chosen by convergence: doubling K and
L or changing a in [6, 9] moves E_n by under 2 % for n <= 12 (checked in
tests/test_oracle_soe.py).
"""
import numpy as np

CF_SCALE = 8.0      # a in z = a (s - 1)/(s + 1)
CF_K = 96           # number of Fourier coefficients kept
CF_L = 2048         # samples on the unit circle
N_MAX = 14          # largest n that is reliable in FP64 (Sec. 3.3)


def _fourier_coefficients(scale, K, L):
    """Fourier coefficients c_0..c_K of F(cos phi), F(s) = exp(scale (s-1)/(s+1))."""
    phi = 2.0 * np.pi * np.arange(L) / L
    s = np.cos(phi)
    F = np.zeros(L)
    inside = s > -1.0 + 1e-14
    F[inside] = np.exp(scale * (s[inside] - 1.0) / (s[inside] + 1.0))
    c = np.real(np.fft.fft(F)) / L
    return c[: K + 1]


def cf_poles_residues(n, scale=CF_SCALE, K=CF_K, L=CF_L):
    """Poles z_k and residues c_k of the CF type (n-1, n) approximant to e^z on R^-.

    Returns (z, c, sigma_n).  Steps 1-5 of the module docstring.
    """
    if n < 1 or n >= K:
        raise ValueError("n out of range")
    c = _fourier_coefficients(scale, K, L)
    v_circ = np.exp(2j * np.pi * np.arange(L) / L)
    f = np.polyval(c[::-1], v_circ)                       # sum_{j<=K} c_j v^j
    idx = np.arange(K)[:, None] + np.arange(K)[None, :] + 1
    cpad = np.concatenate([c, np.zeros(K + 2)])
    H = cpad[idx]                                         # H[i, j] = c_{i+j+1}
    U, S, Vt = np.linalg.svd(H)
    sigma = S[n]
    u = U[:, n]
    v = Vt[n, :]
    u_on_circle = np.polyval(u[::-1], v_circ)             # sum_j u_j v^j
    vrev_on_circle = np.polyval(v, v_circ)                # sum_j v_j v^{K-1-j}
    rt = f - sigma * v_circ ** K * u_on_circle / vrev_on_circle
    zeros = np.roots(v)                                   # zeros of vrev
    q = zeros[np.abs(zeros) > 1.0]
    if len(q) != n:
        raise RuntimeError("CF: expected %d poles outside the unit disk, found %d" % (n, len(q)))
    qpoly = np.poly(q)
    laurent = np.real(np.fft.fft(rt * np.polyval(qpoly, v_circ))) / L
    p = laurent[: n + 1]                                  # coefficients of v^0..v^n
    res_v = np.empty(n, dtype=complex)
    for k in range(n):
        others = np.delete(q, k)
        res_v[k] = np.polyval(p[::-1], q[k]) / np.prod(q[k] - others)
    z = scale * (q - 1.0) ** 2 / (q + 1.0) ** 2
    cz = res_v * 4.0 * z / (q ** 2 - 1.0)
    return z, cz, sigma


def soe_from_poles(z, c):
    """Eq. 2.11: w_k = -c_k sqrt(pi / z_k), t_k = sqrt(z_k) (principal branch)."""
    t = np.sqrt(z)
    w = -c * np.sqrt(np.pi) / t
    return t, w


def halve(t, w, tol=1e-9):
    """Keep one node of each conjugate pair (Im t > 0), doubling its weight.

    Checks that the full set is closed under conjugation, so that
    Re sum_{half} 2 w_k e^{-t_k x} equals the (real) full sum.
    """
    t = np.asarray(t)
    w = np.asarray(w)
    keep = t.imag > 0
    if 2 * keep.sum() != len(t):
        raise ValueError("SOE nodes are not in conjugate pairs")
    for tk, wk in zip(t[keep], w[keep]):
        j = np.argmin(np.abs(t - np.conj(tk)))
        if abs(t[j] - np.conj(tk)) > tol * abs(tk) or abs(w[j] - np.conj(wk)) > tol * max(abs(wk), 1e-300):
            raise ValueError("SOE nodes/weights are not conjugate-symmetric")
    order = np.argsort(t[keep].real)
    return t[keep][order], 2.0 * w[keep][order]


def soe_eval(tau, W, x):
    """S_n(x; 1) = Re sum_k W_k exp(-tau_k |x|) over the halved node set."""
    x = np.abs(np.asarray(x, dtype=float))
    out = np.zeros_like(x)
    for tk, wk in zip(tau, W):
        out += (wk * np.exp(-tk * x)).real
    return out


def En_grid():
    """Sample points for E_n (eq. 3.1) at delta = 1.

    The paper samples x = 0 and 100,000 log-spaced points in [1e-5, 1e2]
    (Sec. 3); a uniform grid on [0, 12] and a fine grid on [0, 1e-3] are added
    so that no oscillation between log points is missed.
    """
    return np.concatenate([[0.0], np.logspace(-5, 2, 100000), np.linspace(0.0, 12.0, 200001),
                           np.linspace(0.0, 1e-3, 10001)])


def E_n(tau, W, grid=None):
    """Eq. 3.1: max_x |G(x; 1) - S_n(x; 1)| on the grid (independent of delta)."""
    x = En_grid() if grid is None else grid
    return float(np.max(np.abs(np.exp(-x * x / 4.0) - soe_eval(tau, W, x))))


def cf_soe(n, **kw):
    """Halved SOE (tau_k, W_k) of the CF approximant with n poles, and its E_n."""
    z, c, _ = cf_poles_residues(n, **kw)
    tau, W = halve(*soe_from_poles(z, c))
    return tau, W, E_n(tau, W)


def plan_soe(eps, n_max=N_MAX):
    """Smallest even n <= n_max whose SOE has E_n <= eps (Sec. 3.3: 'n_e = n/2')."""
    for n in range(2, n_max + 1, 2):
        tau, W, en = cf_soe(n)
        if en <= eps:
            return n, tau, W, en
    raise ValueError("eps below the smallest E_n reachable in FP64")


def hyperbolic_soe(n, theta=None):
    """SOE from the hyperbolic contour of Sec. 3.4, midpoint rule (eqs. 2.6-2.9).

    z(u) = lam (1 - sin(0.8 + i u)), a = arccosh(2 / ((1 - theta) sin 0.8)),
    lam = 0.6 pi (1 - theta) n / a, h = 2a/n, theta = 1/4 for n <= 16 else 12/n.
    Midpoints u_k = -a + (k - 1/2) h, k = 1..n.  As u increases, Im z decreases,
    so the contour orientation of Sec. 2.1 (third quadrant -> second quadrant)
    runs u from +a to -a, which flips the sign of eq. 2.9:
        w_k = -h z'(u_k) e^{z_k} / (2 sqrt(pi) i t_k),  t_k = sqrt(z_k),
    with z'(u) = -i lam cos(0.8 + i u).  Returns the halved set and E_n.
    """
    if theta is None:
        theta = 0.25 if n <= 16 else 12.0 / n
    a = np.arccosh(2.0 / ((1.0 - theta) * np.sin(0.8)))
    lam = 0.6 * np.pi * (1.0 - theta) * n / a
    h = 2.0 * a / n
    u = -a + (np.arange(1, n + 1) - 0.5) * h
    zu = lam * (1.0 - np.sin(0.8 + 1j * u))
    dz = -1j * lam * np.cos(0.8 + 1j * u)
    t = np.sqrt(zu)
    w = -h * dz * np.exp(zu) / (2.0 * np.sqrt(np.pi) * 1j * t)
    tau, W = halve(t, w)
    return tau, W, E_n(tau, W)
