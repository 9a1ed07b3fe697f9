// The Caratheodory-Fejer SOE of order n = 16 (Sec. 3.3: the orders beyond 14 are built
// in extended precision) in double-double arithmetic on the host.
//
// The construction is the one of soe_plan.cpp (transplant z = A (s-1)/(s+1), Fourier
// coefficients of e^z on the circle, the Hankel singular pair at index n, the poles from
// the zeros of the singular vector inside the unit disk, residues from the Laurent
// coefficients of the rational part, the map back to z and eq. 2.11), with every step
// carried in pairs of doubles (about 32 significant digits): at n = 16 the singular
// value is near 1e-14 of the largest, below what FP64 resolves.  The results are
// rounded to FP64 at the end.
//
// Double-double operations follow the error-free transformations of Dekker and Knuth
// (two-sum, two-product by FMA); exp, cos, sin and sqrt are Taylor series after exact
// argument reduction and Newton steps, written here.  The host is compiled without
// floating-point contraction, so x86 and Arm hosts give the same nodes.
#include <algorithm>
#include <cmath>
#include <vector>

#include "fgt1d_internal.h"

namespace fgt1d {
namespace {

struct dd {
    double hi = 0.0, lo = 0.0;
    dd() = default;
    dd(double h) : hi(h), lo(0.0) {}  // NOLINT: implicit from double
    dd(double h, double l) : hi(h), lo(l) {}
};

inline dd two_sum(double a, double b) {
    const double s = a + b, bb = s - a;
    return dd(s, (a - (s - bb)) + (b - bb));
}
inline dd quick_two_sum(double a, double b) {
    const double s = a + b;
    return dd(s, b - (s - a));
}
inline dd two_prod(double a, double b) {
    const double p = a * b;
    return dd(p, std::fma(a, b, -p));
}
inline dd operator+(dd a, dd b) {
    dd s = two_sum(a.hi, b.hi), t = two_sum(a.lo, b.lo);
    s.lo += t.hi;
    s = quick_two_sum(s.hi, s.lo);
    s.lo += t.lo;
    return quick_two_sum(s.hi, s.lo);
}
inline dd operator-(dd a) { return dd(-a.hi, -a.lo); }
inline dd operator-(dd a, dd b) { return a + (-b); }
inline dd operator*(dd a, dd b) {
    dd p = two_prod(a.hi, b.hi);
    p.lo += a.hi * b.lo + a.lo * b.hi;
    return quick_two_sum(p.hi, p.lo);
}
inline dd operator/(dd a, dd b) {
    const double q1 = a.hi / b.hi;
    dd r = a - b * dd(q1);
    const double q2 = r.hi / b.hi;
    r = r - b * dd(q2);
    const double q3 = r.hi / b.hi;
    return quick_two_sum(q1, q2) + dd(q3);
}
inline dd& operator+=(dd& a, dd b) { return a = a + b; }
inline dd& operator*=(dd& a, dd b) { return a = a * b; }
inline bool operator<(dd a, dd b) { return a.hi < b.hi || (a.hi == b.hi && a.lo < b.lo); }
inline dd dabs(dd a) { return a.hi < 0 ? -a : a; }
inline dd ldexp_dd(dd a, int e) { return dd(std::ldexp(a.hi, e), std::ldexp(a.lo, e)); }

inline dd dsqrt(dd a) {
    if (a.hi <= 0.0) return dd(0.0);
    const double x = std::sqrt(a.hi);
    const dd xx(x);
    return xx + (a - xx * xx) / dd(2.0 * x);  // one Newton step doubles the digits
}

const dd kPi(3.141592653589793116e+00, 1.224646799147353207e-16);
const dd kLn2(6.931471805599452862e-01, 2.319046813846299558e-17);

// e^x, x <= 0 here: x = k ln2 + r, |r| <= ln2/2, then Taylor to 2^-110
dd dexp(dd x) {
    if (x.hi < -745.0) return dd(0.0);
    const double k = std::nearbyint(x.hi / kLn2.hi);
    const dd r = x - kLn2 * dd(k);
    dd term(1.0), sum(1.0);
    for (int i = 1; i < 40; ++i) {
        term = term * r / dd((double)i);
        sum += term;
        if (std::fabs(term.hi) < 1e-34 * std::fabs(sum.hi)) break;
    }
    return ldexp_dd(sum, (int)k);
}

// cos and sin of |r| <= pi/4 by their Taylor series
void dsincos_small(dd r, dd& s, dd& c) {
    const dd r2 = r * r;
    dd ts = r, tc(1.0);
    s = ts;
    c = tc;
    for (int i = 1; i < 30; ++i) {
        ts = -(ts * r2) / dd((double)((2 * i) * (2 * i + 1)));
        tc = -(tc * r2) / dd((double)((2 * i - 1) * (2 * i)));
        s += ts;
        c += tc;
        if (std::fabs(tc.hi) < 1e-34 && std::fabs(ts.hi) < 1e-34) break;
    }
}

// cos and sin of 2 pi m / L for integers m, L (L a multiple of 4): the quadrant by the
// integer k = round(4 m / L), the remainder 2 pi (m - k L/4) / L exactly in double-double
void dsincos_frac(long long m, long long L, dd& s, dd& c) {
    m %= L;
    if (m < 0) m += L;
    const long long q = L / 4;
    const long long k = (m + q / 2) / q;
    const dd r = dd(2.0) * kPi * dd((double)(m - k * q)) / dd((double)L);
    dd s0, c0;
    dsincos_small(r, s0, c0);
    switch (k % 4) {
        case 0: s = s0; c = c0; break;
        case 1: s = c0; c = -s0; break;
        case 2: s = -s0; c = -c0; break;
        default: s = -c0; c = s0; break;
    }
}

struct cx {
    dd re, im;
    cx() = default;
    cx(dd r) : re(r), im(0.0) {}  // NOLINT
    cx(dd r, dd i) : re(r), im(i) {}
};
inline cx operator+(cx a, cx b) { return cx(a.re + b.re, a.im + b.im); }
inline cx operator-(cx a, cx b) { return cx(a.re - b.re, a.im - b.im); }
inline cx operator-(cx a) { return cx(-a.re, -a.im); }
inline cx operator*(cx a, cx b) { return cx(a.re * b.re - a.im * b.im, a.re * b.im + a.im * b.re); }
inline cx operator/(cx a, cx b) {
    const dd d = b.re * b.re + b.im * b.im;
    return cx((a.re * b.re + a.im * b.im) / d, (a.im * b.re - a.re * b.im) / d);
}
inline cx conj(cx a) { return cx(a.re, -a.im); }
inline double cabs(cx a) { return std::hypot(a.re.hi, a.im.hi); }
// principal square root
inline cx csqrt(cx z) {
    const dd r = dsqrt(z.re * z.re + z.im * z.im);
    if (!(z.re < dd(0.0))) {
        const dd u = dsqrt((r + z.re) / dd(2.0));
        if (u.hi == 0.0) return cx(dd(0.0));
        return cx(u, z.im / (dd(2.0) * u));
    }
    dd v = dsqrt((r - z.re) / dd(2.0));
    if (z.im < dd(0.0)) v = -v;
    return cx(z.im / (dd(2.0) * v), v);
}

constexpr double kA = 8.0;  // transplant scale, as the FP64 construction
constexpr int kK = 96;      // Fourier coefficients / Hankel size
constexpr int kL = 2048;    // samples on the unit circle

// cyclic Jacobi on the symmetric K x K matrix a (row-major); V: eigenvectors by column
void jacobi_dd(std::vector<dd>& a, std::vector<dd>& V, int n) {
    V.assign((size_t)n * n, dd(0.0));
    for (int i = 0; i < n; ++i) V[(size_t)i * n + i] = dd(1.0);
    for (int sweep = 0; sweep < 60; ++sweep) {
        double off = 0.0, tot = 0.0;
        for (int i = 0; i < n; ++i)
            for (int j = 0; j < n; ++j) {
                const double v = a[(size_t)i * n + j].hi * a[(size_t)i * n + j].hi;
                tot += v;
                if (i != j) off += v;
            }
        if (off <= 1e-66 * tot) break;
        for (int p = 0; p < n - 1; ++p) {
            for (int q = p + 1; q < n; ++q) {
                const dd apq = a[(size_t)p * n + q];
                if (apq.hi == 0.0) continue;
                const dd app = a[(size_t)p * n + p], aqq = a[(size_t)q * n + q];
                // an entry below 1e-40 of the diagonal pair moves no eigenvalue within the
                // precision: dropped (its rotation angle would overflow)
                if (std::fabs(apq.hi) <= 1e-40 * (std::fabs(app.hi) + std::fabs(aqq.hi))) {
                    a[(size_t)p * n + q] = dd(0.0);
                    a[(size_t)q * n + p] = dd(0.0);
                    continue;
                }
                const dd theta = (aqq - app) / (dd(2.0) * apq);
                // t = sign(theta) / (|theta| + sqrt(theta^2 + 1)), ~ 1 / (2 theta) for huge theta
                dd t = std::fabs(theta.hi) > 1e150 ? dd(0.5) / dabs(theta)
                                                   : dd(1.0) / (dabs(theta) + dsqrt(theta * theta + dd(1.0)));
                if (theta.hi < 0) t = -t;
                const dd c = dd(1.0) / dsqrt(t * t + dd(1.0)), s = t * c;
                for (int k = 0; k < n; ++k) {
                    const dd akp = a[(size_t)k * n + p], akq = a[(size_t)k * n + q];
                    a[(size_t)k * n + p] = c * akp - s * akq;
                    a[(size_t)k * n + q] = s * akp + c * akq;
                }
                for (int k = 0; k < n; ++k) {
                    const dd apk = a[(size_t)p * n + k], aqk = a[(size_t)q * n + k];
                    a[(size_t)p * n + k] = c * apk - s * aqk;
                    a[(size_t)q * n + k] = s * apk + c * aqk;
                }
                for (int k = 0; k < n; ++k) {
                    const dd vkp = V[(size_t)k * n + p], vkq = V[(size_t)k * n + q];
                    V[(size_t)k * n + p] = c * vkp - s * vkq;
                    V[(size_t)k * n + q] = s * vkp + c * vkq;
                }
            }
        }
    }
}

// p(z) and p'(z) for p(z) = sum_j a[j] z^j
void horner_dd(const std::vector<dd>& a, cx z, cx& p, cx& dp) {
    p = cx(a.back());
    dp = cx(dd(0.0));
    for (int j = (int)a.size() - 2; j >= 0; --j) {
        dp = dp * z + p;
        p = p * z + cx(a[j]);
    }
}

}  // namespace

int build_cf_soe_dd(int n, std::vector<double> (*zeros_fp64)(const std::vector<double>&), double* tau_re,
                    double* tau_im, double* w_re, double* w_im) {
    const int K = kK, L = kL;
    // step 1: Fourier coefficients of F(cos phi), F(s) = exp(A (s - 1)/(s + 1))
    std::vector<dd> cs(L), sn(L), F(L), c(K + 1, dd(0.0));
    for (int m = 0; m < L; ++m) dsincos_frac(m, L, sn[m], cs[m]);
    for (int m = 0; m < L; ++m) {
        const dd s = cs[m];
        F[m] = (s.hi > -1.0 + 1e-14) ? dexp(dd(kA) * (s - dd(1.0)) / (s + dd(1.0))) : dd(0.0);
    }
    for (int j = 0; j <= K; ++j) {
        dd acc(0.0);
        for (int m = 0; m < L; ++m) acc += F[m] * cs[(int)(((long long)j * m) % L)];
        c[j] = acc / dd((double)L);
    }
    // step 2: Hankel matrix c_{i+j+1}, its eigenpair of the (n+1)-th largest |eigenvalue|
    std::vector<dd> H((size_t)K * K, dd(0.0)), V;
    for (int i = 0; i < K; ++i)
        for (int j = 0; j < K; ++j) H[(size_t)i * K + j] = (i + j + 1 <= K) ? c[i + j + 1] : dd(0.0);
    jacobi_dd(H, V, K);
    std::vector<int> order(K);
    for (int i = 0; i < K; ++i) order[i] = i;
    std::sort(order.begin(), order.end(),
              [&](int x, int y) { return dabs(H[(size_t)y * K + y]) < dabs(H[(size_t)x * K + x]); });
    const int col = order[n];
    const dd lambda = H[(size_t)col * K + col];
    const dd sigma = dabs(lambda);
    std::vector<dd> v(K), u(K);
    std::vector<double> v64(K);
    for (int j = 0; j < K; ++j) {
        v[j] = V[(size_t)j * K + col];
        u[j] = lambda.hi >= 0 ? v[j] : -v[j];
        v64[j] = v[j].hi;
    }
    // step 3: zeros of v inside the unit disk, started in FP64 and polished in
    // double-double (Newton on v, then on vrev(w) = w^{K-1} v(1/w) for q = 1/zero)
    const std::vector<double> zr = zeros_fp64(v64);  // interleaved re, im
    std::vector<cx> q;
    for (size_t i = 0; i + 1 < zr.size(); i += 2) {
        cx z(dd(zr[i]), dd(zr[i + 1]));
        const double az = cabs(z);
        if (!(az < 1.0) || az == 0.0) continue;
        for (int it = 0; it < 4; ++it) {
            cx p, dp;
            horner_dd(v, z, p, dp);
            if (cabs(dp) == 0.0) break;
            z = z - p / dp;
        }
        cx qq = cx(dd(1.0)) / z;
        std::vector<dd> vrev(v.rbegin(), v.rend());  // coefficients of w^{K-1} v(1/w)
        for (int it = 0; it < 3; ++it) {
            cx p, dp;
            horner_dd(vrev, qq, p, dp);
            if (cabs(dp) == 0.0) break;
            qq = qq - p / dp;
        }
        q.push_back(qq);
    }
    if ((int)q.size() != n) return FGT1D_EUNSUPPORTED;
    // step 4: Laurent coefficients 0..n of rt * prod(w - q_k) on the circle
    std::vector<cx> lc(n + 1, cx(dd(0.0)));
    for (int m = 0; m < L; ++m) {
        const cx w(cs[m], sn[m]);
        cx f(c[K]), uu(u[K - 1]), vr(dd(0.0));
        for (int j = K - 1; j >= 0; --j) f = f * w + cx(c[j]);
        for (int j = K - 2; j >= 0; --j) uu = uu * w + cx(u[j]);
        for (int j = 0; j < K; ++j) vr = vr * w + cx(v[j]);
        const int mk = (int)(((long long)K * m) % L);
        const cx wK(cs[mk], sn[mk]);
        const cx rt = f - cx(sigma) * wK * uu / vr;
        cx g = rt;
        for (int k = 0; k < n; ++k) g = g * (w - q[k]);
        for (int l = 0; l <= n; ++l) {  // times w^{-l}
            const int ml = (int)((((long long)-l * m) % L + L) % L);
            lc[l] = lc[l] + g * cx(cs[ml], sn[ml]);
        }
    }
    std::vector<dd> pc(n + 1);
    for (int l = 0; l <= n; ++l) pc[l] = lc[l].re / dd((double)L);
    // residues, the map back to z (step 5) and eq. 2.11
    const dd sqrt_pi = dsqrt(kPi);
    std::vector<cx> tk(n), wk(n);
    for (int k = 0; k < n; ++k) {
        cx pv(dd(0.0));
        for (int l = n; l >= 0; --l) pv = pv * q[k] + cx(pc[l]);
        cx den(dd(1.0));
        for (int l = 0; l < n; ++l)
            if (l != k) den = den * (q[k] - q[l]);
        const cx res_w = pv / den;
        const cx qm = q[k] - cx(dd(1.0)), qp = q[k] + cx(dd(1.0));
        const cx zk = cx(dd(kA)) * qm * qm / (qp * qp);
        const cx ck = res_w * cx(dd(4.0)) * zk / (q[k] * q[k] - cx(dd(1.0)));
        tk[k] = csqrt(zk);
        wk[k] = -(ck * cx(sqrt_pi)) / tk[k];
    }
    // one node of each conjugate pair (Im t > 0), weight doubled, ascending Re t
    std::vector<int> keep;
    for (int k = 0; k < n; ++k)
        if (tk[k].im.hi > 0) keep.push_back(k);
    if ((int)keep.size() != n / 2) return FGT1D_EUNSUPPORTED;
    for (int k : keep) {
        double best = 1e300;
        int bj = -1;
        for (int j = 0; j < n; ++j) {
            const double d = cabs(tk[j] - conj(tk[k]));
            if (d < best) { best = d; bj = j; }
        }
        if (bj < 0 || best > 1e-20 * cabs(tk[k]) || cabs(wk[bj] - conj(wk[k])) > 1e-20 * cabs(wk[k]))
            return FGT1D_EUNSUPPORTED;
    }
    std::sort(keep.begin(), keep.end(), [&](int a, int b) { return tk[a].re < tk[b].re; });
    for (int i = 0; i < (int)keep.size(); ++i) {
        const cx t = tk[keep[i]], w = wk[keep[i]];
        tau_re[i] = t.re.hi + t.re.lo;
        tau_im[i] = t.im.hi + t.im.lo;
        w_re[i] = 2.0 * (w.re.hi + w.re.lo);
        w_im[i] = 2.0 * (w.im.hi + w.im.lo);
    }
    return FGT1D_OK;
}

}  // namespace fgt1d
