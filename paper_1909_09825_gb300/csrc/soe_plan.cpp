// Host SOE generator and plan objects (step a0).
//
// The Gaussian kernel is approximated by a sum of exponentials (eq. 1.3) whose
// nodes and weights come from a sum-of-poles rational approximation
// r(z) = sum_k c_k / (z - z_k) of e^z on (-inf, 0] (eq. 2.13) through eq. 2.11:
// w_k = -c_k sqrt(pi / z_k), t_k = sqrt(z_k).  As in Sec. 3.3, the poles and
// residues are those of the Caratheodory-Fejer (CF) approximation of type
// (n-1, n).  The CF construction is done here in FP64 with self-contained
// numerics (no LAPACK):
//
//   1. z = A (s - 1)/(s + 1) maps s in (-1, 1] onto (-inf, 0];
//      F(s) = exp(A (s-1)/(s+1)); its Fourier coefficients c_0..c_K in the angle
//      phi, s = cos phi, are computed by direct cosine sums over CF_L samples;
//   2. the symmetric Hankel matrix H[i][j] = c_{i+j+1} (i, j < K) is diagonalised
//      with cyclic Jacobi rotations; the (n+1)-th largest |eigenvalue| is the CF
//      singular value sigma and its eigenvector gives the singular pair (u = sign * v);
//   3. the zeros of v(w) = sum_j v_j w^j inside the unit disk (Aberth-Ehrlich
//      iteration started from Newton-polygon radii, then Newton polishing) are
//      the reciprocals of the n CF poles q_k outside the disk;
//   4. on the circle w = e^{i phi}, rt = f - sigma w^K u(w) / vrev(w) with
//      f = sum_j c_j w^j and vrev(w) = w^{K-1} v(1/w); the rational part of rt is
//      p / prod (w - q_k), p the polynomial of the Laurent coefficients 0..n of
//      rt * prod (w - q_k); residues in w are p(q_k) / prod_{l != k} (q_k - q_l);
//   5. z_k = A (q_k - 1)^2 / (q_k + 1)^2, residue in z = residue in w * 4 z_k / (q_k^2 - 1).
//
// Orders n <= 14 run in FP64; n = 16 runs the same steps in double-double
// (soe_cf_dd.cpp), as the paper builds its largest orders in extended precision.
// One node of each conjugate pair is kept (Im t_k > 0) with weight W_k = 2 w_k
// (Sec. 4).  E_n (eq. 3.1) is measured on x = 0, 1e5 log-spaced points in
// [1e-5, 1e2] (the paper's grid) and uniform grids on [0, 12] and [0, 1e-3].
#include <algorithm>
#include <cmath>
#include <complex>
#include <cstring>
#include <mutex>
#include <new>
#include <vector>

#include "fgt1d_internal.h"

namespace fgt1d {
namespace {

using cd = std::complex<double>;

constexpr double kCfScale = 8.0;   // A
constexpr int kCfK = 96;           // Hankel size / number of coefficients
constexpr int kCfL = 2048;         // samples on the unit circle

// Step 1: Fourier coefficients of F(cos phi).
std::vector<double> fourier_coefficients() {
    std::vector<double> F(kCfL), c(kCfK + 1, 0.0);
    const double two_pi = 2.0 * M_PI;
    for (int m = 0; m < kCfL; ++m) {
        double s = std::cos(two_pi * m / kCfL);
        F[m] = (s > -1.0 + 1e-14) ? std::exp(kCfScale * (s - 1.0) / (s + 1.0)) : 0.0;
    }
    for (int j = 0; j <= kCfK; ++j) {
        double acc = 0.0;
        for (int m = 0; m < kCfL; ++m) acc += F[m] * std::cos(two_pi * (double)(((long long)j * m) % kCfL) / kCfL);
        c[j] = acc / kCfL;
    }
    return c;
}

// Step 2: cyclic Jacobi eigen-decomposition of a symmetric matrix (row-major a[n*n]).
// On return the diagonal of a holds the eigenvalues and column k of V the k-th eigenvector.
void jacobi_eigen(std::vector<double>& a, std::vector<double>& V, int n) {
    V.assign((size_t)n * n, 0.0);
    for (int i = 0; i < n; ++i) V[(size_t)i * n + i] = 1.0;
    for (int sweep = 0; sweep < 100; ++sweep) {
        double off = 0.0, tot = 0.0;
        for (int i = 0; i < n; ++i)
            for (int j = 0; j < n; ++j) {
                double v = a[(size_t)i * n + j] * a[(size_t)i * n + j];
                tot += v;
                if (i != j) off += v;
            }
        if (off <= 1e-34 * tot) break;
        for (int p = 0; p < n - 1; ++p) {
            for (int q = p + 1; q < n; ++q) {
                double apq = a[(size_t)p * n + q];
                if (apq == 0.0) continue;
                double app = a[(size_t)p * n + p], aqq = a[(size_t)q * n + q];
                double theta = (aqq - app) / (2.0 * apq);
                double t = (theta >= 0 ? 1.0 : -1.0) / (std::fabs(theta) + std::sqrt(theta * theta + 1.0));
                double c = 1.0 / std::sqrt(t * t + 1.0), s = t * c;
                for (int k = 0; k < n; ++k) {  // columns p, q
                    double akp = a[(size_t)k * n + p], akq = a[(size_t)k * n + q];
                    a[(size_t)k * n + p] = c * akp - s * akq;
                    a[(size_t)k * n + q] = s * akp + c * akq;
                }
                for (int k = 0; k < n; ++k) {  // rows p, q
                    double apk = a[(size_t)p * n + k], aqk = a[(size_t)q * n + k];
                    a[(size_t)p * n + k] = c * apk - s * aqk;
                    a[(size_t)q * n + k] = s * apk + c * aqk;
                }
                for (int k = 0; k < n; ++k) {
                    double vkp = V[(size_t)k * n + p], vkq = V[(size_t)k * n + q];
                    V[(size_t)k * n + p] = c * vkp - s * vkq;
                    V[(size_t)k * n + q] = s * vkp + c * vkq;
                }
            }
        }
    }
}

// p(z) / p'(z) for p(z) = sum_j a[j] z^j of degree D; evaluated through the reversed
// polynomial when |z| > 1 so that large roots do not overflow.
cd newton_ratio(const std::vector<double>& a, cd z) {
    const int D = (int)a.size() - 1;
    if (std::abs(z) <= 1.0) {
        cd p = a[D], dp = 0.0;
        for (int j = D - 1; j >= 0; --j) { dp = dp * z + p; p = p * z + a[j]; }
        return p / dp;
    }
    cd y = 1.0 / z, r = a[0], dr = 0.0;  // R(y) = sum_j a_j y^{D-j}
    for (int j = 1; j <= D; ++j) { dr = dr * y + r; r = r * y + a[j]; }
    return z / ((double)D - y * dr / r);
}

// Step 3: all zeros of sum_j a[j] z^j (Aberth-Ehrlich).  Initial radii from the upper
// convex hull of (j, log|a_j|) (Newton polygon), one circle per hull edge.
std::vector<cd> poly_zeros(std::vector<double> a) {
    while (a.size() > 1 && a.back() == 0.0) a.pop_back();
    int lead0 = 0;
    while (lead0 < (int)a.size() - 1 && a[lead0] == 0.0) ++lead0;  // zeros at the origin
    std::vector<double> b(a.begin() + lead0, a.end());
    const int D = (int)b.size() - 1;
    std::vector<cd> z;
    if (D <= 0) return std::vector<cd>(lead0, cd(0.0));
    std::vector<int> hull;
    for (int j = 0; j <= D; ++j) {
        if (b[j] == 0.0) continue;
        double lj = std::log(std::fabs(b[j]));
        while (hull.size() >= 2) {
            int i1 = hull[hull.size() - 2], i2 = hull.back();
            double l1 = std::log(std::fabs(b[i1])), l2 = std::log(std::fabs(b[i2]));
            if ((l2 - l1) * (j - i1) <= (lj - l1) * (i2 - i1)) hull.pop_back();
            else break;
        }
        hull.push_back(j);
    }
    const double sigma0 = 0.7;
    for (size_t h = 1; h < hull.size(); ++h) {
        int j1 = hull[h - 1], j2 = hull[h], cnt = j2 - j1;
        double r = std::pow(std::fabs(b[j1] / b[j2]), 1.0 / cnt);
        for (int i = 0; i < cnt; ++i)
            z.push_back(std::polar(r, 2.0 * M_PI * i / cnt + 2.0 * M_PI * h / D + sigma0));
    }
    std::vector<bool> done(D, false);
    for (int it = 0; it < 800; ++it) {
        bool all = true;
        for (int i = 0; i < D; ++i) {
            if (done[i]) continue;
            cd ratio = newton_ratio(b, z[i]);
            cd s = 0.0;
            for (int j = 0; j < D; ++j)
                if (j != i) s += 1.0 / (z[i] - z[j]);
            cd corr = ratio / (1.0 - ratio * s);
            z[i] -= corr;
            if (std::abs(corr) <= 4e-16 * std::abs(z[i])) done[i] = true;
            else all = false;
        }
        if (all) break;
    }
    for (int i = 0; i < lead0; ++i) z.push_back(0.0);
    return z;
}

struct Soe {
    int n = 0, n_e = 0;
    double tau_re[FGT1D_MAX_TERMS], tau_im[FGT1D_MAX_TERMS], w_re[FGT1D_MAX_TERMS], w_im[FGT1D_MAX_TERMS];
    double E_n = 0.0;
    int status = FGT1D_OK;
};

double soe_value(const Soe& s, double x) {
    double acc = 0.0;
    for (int k = 0; k < s.n_e; ++k) {
        double mag = std::exp(-s.tau_re[k] * x);
        acc += mag * (s.w_re[k] * std::cos(s.tau_im[k] * x) + s.w_im[k] * std::sin(s.tau_im[k] * x));
    }
    return acc;
}

double measure_En(const Soe& s) {
    double e = std::fabs(1.0 - soe_value(s, 0.0));
    auto upd = [&](double x) { e = std::max(e, std::fabs(std::exp(-x * x / 4.0) - soe_value(s, x))); };
    for (int i = 0; i < 100000; ++i) upd(std::pow(10.0, -5.0 + 7.0 * i / 99999.0));
    for (int i = 0; i <= 200000; ++i) upd(12.0 * i / 200000.0);
    for (int i = 0; i <= 10000; ++i) upd(1e-3 * i / 10000.0);
    return e;
}

// Steps 1-2 do not depend on n: computed once per process.
struct CfBase {
    std::vector<double> c, H, V;
    std::vector<int> order;  // eigenvalue indices by decreasing |lambda|
};

const CfBase& cf_base() {
    static std::once_flag once;
    static CfBase b;
    std::call_once(once, [] {
        const int K = kCfK;
        b.c = fourier_coefficients();
        b.H.assign((size_t)K * K, 0.0);
        for (int i = 0; i < K; ++i)
            for (int j = 0; j < K; ++j) b.H[(size_t)i * K + j] = (i + j + 1 <= K) ? b.c[i + j + 1] : 0.0;
        jacobi_eigen(b.H, b.V, K);
        b.order.resize(K);
        for (int i = 0; i < K; ++i) b.order[i] = i;
        std::sort(b.order.begin(), b.order.end(), [&](int x, int y) {
            return std::fabs(b.H[(size_t)x * K + x]) > std::fabs(b.H[(size_t)y * K + y]);
        });
    });
    return b;
}

// The zeros of sum_j a[j] z^j (poly_zeros), interleaved (re, im), for the
// double-double construction's starting values.
std::vector<double> zeros_interleaved(const std::vector<double>& a) {
    std::vector<double> out;
    for (cd z : poly_zeros(a)) {
        out.push_back(z.real());
        out.push_back(z.imag());
    }
    return out;
}

}  // namespace

// soe_cf_dd.cpp: the same construction in double-double arithmetic (n = 16).
int build_cf_soe_dd(int n, std::vector<double> (*zeros_fp64)(const std::vector<double>&), double* tau_re,
                    double* tau_im, double* w_re, double* w_im);

namespace {

// Orders above this are built in double-double (Sec. 3.3: beyond n = 14 the paper's
// CF construction runs in extended precision).
constexpr int kMaxNFp64 = 14;

Soe build_cf_soe(int n) {
    Soe out;
    if (n > kMaxNFp64) {
        out.n = n;
        out.n_e = n / 2;
        out.status = build_cf_soe_dd(n, zeros_interleaved, out.tau_re, out.tau_im, out.w_re, out.w_im);
        if (out.status == FGT1D_OK) out.E_n = measure_En(out);
        return out;
    }
    out.n = n;
    out.n_e = n / 2;
    const int K = kCfK;
    const CfBase& base = cf_base();
    const std::vector<double>& c = base.c;
    const std::vector<double>& H = base.H;
    const std::vector<double>& V = base.V;
    const int col = base.order[n];
    const double lambda = H[(size_t)col * K + col];
    const double sigma = std::fabs(lambda);
    std::vector<double> v(K), u(K);
    for (int j = 0; j < K; ++j) {
        v[j] = V[(size_t)j * K + col];
        u[j] = (lambda >= 0 ? 1.0 : -1.0) * v[j];
    }
    // step 3: zeros of v inside the unit disk -> poles q = 1/zero outside
    std::vector<cd> zeros = poly_zeros(v);
    std::vector<cd> q;
    for (cd r : zeros)
        if (std::abs(r) < 1.0 && std::abs(r) > 0.0) {
            cd qq = 1.0 / r;
            // Newton polish on vrev(w) = sum_j v_j w^{K-1-j}
            for (int it = 0; it < 3; ++it) {
                cd p = 0.0, dp = 0.0;
                for (int j = 0; j < K; ++j) { dp = dp * qq + p; p = p * qq + v[j]; }
                if (std::abs(dp) == 0.0) break;
                qq -= p / dp;
            }
            q.push_back(qq);
        }
    if ((int)q.size() != n) { out.status = FGT1D_EUNSUPPORTED; return out; }
    // step 4: Laurent coefficients 0..n of rt * prod(w - q_k)
    std::vector<cd> lc(n + 1, 0.0);
    for (int m = 0; m < kCfL; ++m) {
        cd w = std::polar(1.0, 2.0 * M_PI * m / kCfL);
        cd f = c[K], uu = u[K - 1], vr = 0.0;
        for (int j = K - 1; j >= 0; --j) f = f * w + c[j];
        for (int j = K - 2; j >= 0; --j) uu = uu * w + u[j];
        for (int j = 0; j < K; ++j) vr = vr * w + v[j];
        cd rt = f - sigma * std::pow(w, K) * uu / vr;
        cd g = rt;
        for (int k = 0; k < n; ++k) g *= (w - q[k]);
        cd winv = std::conj(w), wl = 1.0;
        for (int l = 0; l <= n; ++l) { lc[l] += g * wl; wl *= winv; }
    }
    std::vector<double> pc(n + 1);
    for (int l = 0; l <= n; ++l) pc[l] = lc[l].real() / kCfL;
    // residues, step 5 mapping, eq. 2.11
    std::vector<cd> tk(n), wk(n);
    for (int k = 0; k < n; ++k) {
        cd pv = 0.0;
        for (int l = n; l >= 0; --l) pv = pv * q[k] + pc[l];
        cd den = 1.0;
        for (int l = 0; l < n; ++l)
            if (l != k) den *= (q[k] - q[l]);
        cd res_w = pv / den;
        cd zk = kCfScale * (q[k] - 1.0) * (q[k] - 1.0) / ((q[k] + 1.0) * (q[k] + 1.0));
        cd ck = res_w * 4.0 * zk / (q[k] * q[k] - 1.0);
        tk[k] = std::sqrt(zk);
        wk[k] = -ck * std::sqrt(M_PI) / tk[k];
    }
    // keep Im t > 0, check the conjugate partner, double the weight
    std::vector<int> keep;
    for (int k = 0; k < n; ++k)
        if (tk[k].imag() > 0) keep.push_back(k);
    if ((int)keep.size() != n / 2) { out.status = FGT1D_EUNSUPPORTED; return out; }
    for (int k : keep) {
        double best = 1e300;
        int bj = -1;
        for (int j = 0; j < n; ++j) {
            double d = std::abs(tk[j] - std::conj(tk[k]));
            if (d < best) { best = d; bj = j; }
        }
        if (bj < 0 || best > 1e-8 * std::abs(tk[k]) ||
            std::abs(wk[bj] - std::conj(wk[k])) > 1e-8 * std::abs(wk[k])) {
            out.status = FGT1D_EUNSUPPORTED;
            return out;
        }
    }
    std::sort(keep.begin(), keep.end(), [&](int a, int b) { return tk[a].real() < tk[b].real(); });
    for (int i = 0; i < (int)keep.size(); ++i) {
        out.tau_re[i] = tk[keep[i]].real();
        out.tau_im[i] = tk[keep[i]].imag();
        out.w_re[i] = 2.0 * wk[keep[i]].real();
        out.w_im[i] = 2.0 * wk[keep[i]].imag();
    }
    out.E_n = measure_En(out);
    return out;
}

std::once_flag g_once[FGT1D_MAX_N / 2 + 1];
Soe g_soe[FGT1D_MAX_N / 2 + 1];

const Soe& cached_soe(int n) {
    std::call_once(g_once[n / 2], [n] { g_soe[n / 2] = build_cf_soe(n); });
    return g_soe[n / 2];
}

bool finite_all(const double* a, int n) {
    for (int i = 0; i < n; ++i)
        if (!std::isfinite(a[i])) return false;
    return true;
}

}  // namespace
}  // namespace fgt1d

using fgt1d::cached_soe;

extern "C" int fgt1d_soe_cf(int n, int* n_e, double* tau_re, double* tau_im, double* w_re, double* w_im,
                            double* E_n) {
    if (n < 2 || n > FGT1D_MAX_N || (n & 1) || !n_e || !tau_re || !tau_im || !w_re || !w_im || !E_n)
        return FGT1D_EINVAL;
    const auto& s = cached_soe(n);
    if (s.status != FGT1D_OK) return s.status;
    *n_e = s.n_e;
    for (int k = 0; k < s.n_e; ++k) {
        tau_re[k] = s.tau_re[k];
        tau_im[k] = s.tau_im[k];
        w_re[k] = s.w_re[k];
        w_im[k] = s.w_im[k];
    }
    *E_n = s.E_n;
    return FGT1D_OK;
}

extern "C" int fgt1d_plan_create(double delta, double eps, unsigned flags, fgt1d_plan* out) {
    if (!out) return FGT1D_EINVAL;
    *out = nullptr;
    if (!(delta > 0.0) || !std::isfinite(delta) || !(eps > 0.0) || !(eps < 0.5) ||
        (flags & ~(FGT1D_FP32 | FGT1D_EXACT_SELF | FGT1D_F32X2)) || ((flags & FGT1D_FP32) && (flags & FGT1D_F32X2)))
        return FGT1D_EINVAL;
    if ((flags & FGT1D_FP32) && eps < 1e-6) return FGT1D_EUNSUPPORTED;
    for (int n = 2; n <= FGT1D_MAX_N; n += 2) {
        const auto& s = cached_soe(n);
        if (s.status != FGT1D_OK) continue;
        if (s.E_n <= eps) {
            auto* p = new (std::nothrow) fgt1d_plan_s();
            if (!p) return FGT1D_ENOMEM;
            p->n = n;
            p->n_e = s.n_e;
            p->delta = delta;
            p->E_n = s.E_n;
            p->flags = flags;
            for (int k = 0; k < s.n_e; ++k) {
                p->tau_re[k] = s.tau_re[k];
                p->tau_im[k] = s.tau_im[k];
                p->w_re[k] = s.w_re[k];
                p->w_im[k] = s.w_im[k];
            }
            *out = p;
            return FGT1D_OK;
        }
    }
    return FGT1D_EUNSUPPORTED;
}

extern "C" int fgt1d_plan_create_soe(double delta, int n_e, const double* tau_re, const double* tau_im,
                                     const double* w_re, const double* w_im, unsigned flags, fgt1d_plan* out) {
    if (!out) return FGT1D_EINVAL;
    *out = nullptr;
    if (!(delta > 0.0) || !std::isfinite(delta) || n_e < 1 || n_e > FGT1D_MAX_TERMS || !tau_re || !tau_im ||
        !w_re || !w_im || (flags & ~(FGT1D_FP32 | FGT1D_EXACT_SELF | FGT1D_F32X2)) ||
        ((flags & FGT1D_FP32) && (flags & FGT1D_F32X2)))
        return FGT1D_EINVAL;
    if (!fgt1d::finite_all(tau_re, n_e) || !fgt1d::finite_all(tau_im, n_e) || !fgt1d::finite_all(w_re, n_e) ||
        !fgt1d::finite_all(w_im, n_e))
        return FGT1D_EINVAL;
    for (int k = 0; k < n_e; ++k)
        if (!(tau_re[k] > 0.0)) return FGT1D_EINVAL;
    auto* p = new (std::nothrow) fgt1d_plan_s();
    if (!p) return FGT1D_ENOMEM;
    p->n = 0;
    p->n_e = n_e;
    p->delta = delta;
    p->E_n = std::nan("");
    p->flags = flags;
    for (int k = 0; k < n_e; ++k) {
        p->tau_re[k] = tau_re[k];
        p->tau_im[k] = tau_im[k];
        p->w_re[k] = w_re[k];
        p->w_im[k] = w_im[k];
    }
    *out = p;
    return FGT1D_OK;
}

extern "C" int fgt1d_plan_info(fgt1d_plan plan, int* n, int* n_e, double* E_n, double* delta, unsigned* flags,
                               double* tau_re, double* tau_im, double* w_re, double* w_im) {
    if (!plan) return FGT1D_EINVAL;
    if (n) *n = plan->n;
    if (n_e) *n_e = plan->n_e;
    if (E_n) *E_n = plan->E_n;
    if (delta) *delta = plan->delta;
    if (flags) *flags = plan->flags;
    for (int k = 0; k < plan->n_e; ++k) {
        if (tau_re) tau_re[k] = plan->tau_re[k];
        if (tau_im) tau_im[k] = plan->tau_im[k];
        if (w_re) w_re[k] = plan->w_re[k];
        if (w_im) w_im[k] = plan->w_im[k];
    }
    return FGT1D_OK;
}

extern "C" void fgt1d_plan_destroy(fgt1d_plan plan) { delete plan; }
