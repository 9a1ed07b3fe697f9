// Steps a3-a7: the forward and backward SOE recurrences (eqs. 4.5-4.6) over the sorted
// merged points, evaluation (eq. 4.1) and unpermutation.
//
// With z_p the sorted coordinates, s = 1/sqrt(delta) and the multiplier of point p
//     m_{k,p} = exp(-tau_k s (z_p - z_{p-1})),
// the two recurrences are
//     F_{k,p} = m_{k,p} F_{k,p-1} + alpha_p          (eq. 4.5: h+ includes y_j <= x_i)
//     B_{k,p} = m_{k,p+1} B_{k,p+1} + alpha_p        (eq. 4.6: h- over y_j > x_i)
// with alpha_p = 0 at targets, and u_i = Re sum_k W_k (F_{k,p} + B_{k,p}) at the target's
// sorted position p (eq. 4.1 with W_k = 2 w_k over one node of each conjugate pair).
// Because sources sort before equal targets, F at a target holds every y_j <= x_i and
// B every y_j > x_i (eq. 4.4).
//
// GB300 design.  Each recurrence is an associative scan of affine maps h -> m h + a.
// The 128-thread shape is persistent: as many CTAs as fit on the GPU, each taking tiles in
// sweep order from an atomic counter until none is left; the 256-thread shape runs one
// CTA per tile (both measured faster that way).  A tile is T*R consecutive points;
// each thread runs R consecutive points sequentially (work-efficient), the threads of a
// warp are joined by a serial scan of their aggregates in shared memory (FP64) or a
// shuffle scan (FP32, double-float), and one lane per term joins the warps and the tiles.  Per tile the kernel runs
//   phase A  per term: multipliers, thread aggregates, warp scans (exclusive prefixes
//            kept in shared memory);
//   phase B  per term (one warp each): combine the warp totals, publish the tile
//            aggregate with the tile's span multiplier exp(-tau s (z_anchor - z_prev))
//            computed directly from the FP64 anchor coordinates, decoupled look-back
//            over the neighbouring tiles 32 at a time (a complex multiply-add per
//            predecessor, using the published span multipliers), publish the
//            inclusive value;
//   phase C  per term: apply the carries, final pass, evaluation at targets.
// When the scan region of all terms would not fit the occupancy target, the terms run
// in equal groups, each with its own phases A-C (SweepGroup).  Per-point multipliers
// use a Taylor polynomial of warp-uniform degree chosen from the warp's largest gap
// (integer compares on the bit pattern of theta), falling back to exp/sincos for large
// gaps.
//
// FP64 path (Real = double): FP64 accuracy at every step.  The forward kernel stores
// the multipliers (16 B per point and term): on GB300 one DFMA costs as much issue time
// as 62 FFMAs, and reloading 16 B is cheaper than the 5-10 DFMAs of a multiplier.  For
// small |tau theta| the multiplier's cubic-and-up Taylor tail runs on the FP32 pipe
// (taylor_hybrid).  Inside each 4096-point tile the table is thread-interleaved: the
// multiplier of a tile's point t R + r sits at slot r T + t, so that the R loads or
// stores of a warp's 32 threads are each one contiguous 512-byte segment.
// FP32 path (Real = float): gaps, multipliers and in-tile recurrences in FP32
// complex; tile aggregates, span multipliers and carries in FP64.  Gaps come from the
// integer difference of the sorted keys and FP64<->FP32 conversions are done with
// integer bit operations, so the per-point work issues no FP64-pipe instruction.
// Double-float path (Real = dfloat): the FP32 path's structure with pairs of floats
// (about 48 significant bits) for gaps, multipliers and recurrences.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <type_traits>

#include "dfloat.cuh"
#include "fgt1d_internal.h"
#include "kernels.h"

namespace fgt1d {

__device__ __forceinline__ double key_coord(uint64_t k) {
    uint64_t b = (k >> 63) ? (k & 0x7FFFFFFFFFFFFFFFull) : ~k;
    return __longlong_as_double((long long)b);
}

__device__ __forceinline__ void st_volatile_u32(uint32_t* p, uint32_t v) {
    asm volatile("st.volatile.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}
__device__ __forceinline__ uint32_t ld_volatile_u32(const uint32_t* p) {
    uint32_t v;
    asm volatile("ld.volatile.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

// ---- FP64 <-> FP32 with integer operations (no FP64-pipe instruction) ----------------------
// Value of (d * 2^e2) rounded to float (round half up), d > 0 an integer below 2^64;
// 0 when below the float normal range.
__device__ __forceinline__ float u64_scaled_to_f32(uint64_t d, int e2) {
    if (d == 0) return 0.0f;
    const int msb = 63 - __clzll((long long)d);
    uint32_t mant;
    int E = msb + e2 + 127;
    if (msb <= 23) {
        mant = (uint32_t)(d << (23 - msb));
    } else {
        const int sh = msb - 23;
        uint64_t m = (d >> sh) + ((d >> (sh - 1)) & 1ull);
        if (m >> 24) { m >>= 1; ++E; }
        mant = (uint32_t)m;
    }
    if (E <= 0) return 0.0f;
    if (E >= 255) return __int_as_float(0x7F800000);
    return __int_as_float((E << 23) | (int)(mant & 0x7FFFFFu));
}

// b - a for b >= a as float.  Exact up to the final rounding when a and b are normal,
// of the same sign and in the same binade (the common case for sorted neighbours);
// otherwise through an FP64 subtraction.
__device__ __forceinline__ float gap_f32(double a, double b) {
    const uint64_t ba = (uint64_t)__double_as_longlong(a), bb = (uint64_t)__double_as_longlong(b);
    const uint32_t ea = (uint32_t)(ba >> 52) & 0x7FFu, eb = (uint32_t)(bb >> 52) & 0x7FFu;
    if (ea == eb && ea != 0 && ea != 0x7FF && ((ba ^ bb) >> 63) == 0) {
        const uint64_t d = bb >= ba ? bb - ba : ba - bb;
        return u64_scaled_to_f32(d, (int)ea - 1075);
    }
    return (float)(b - a);
}

// float(x) for a double with round half up; zero below the float normal range.
__device__ __forceinline__ float f64_to_f32(double x) {
    const uint64_t b = (uint64_t)__double_as_longlong(x);
    const uint32_t sign = (uint32_t)(b >> 32) & 0x80000000u;
    const int e = (int)((b >> 52) & 0x7FF);
    if (e == 0x7FF) return __int_as_float((int)(sign | 0x7F800000u | ((b & 0xFFFFFFFFFFFFFull) ? 1u : 0u)));
    float mag = u64_scaled_to_f32((b & 0xFFFFFFFFFFFFFull) | (e ? (1ull << 52) : 0ull), (e ? e : 1) - 1075);
    return __int_as_float((int)(__float_as_uint(mag) | sign));
}

// (double)f, exact; float subnormals become 0.
__device__ __forceinline__ double f32_to_f64(float f) {
    const uint32_t b = __float_as_uint(f);
    const uint32_t e = (b >> 23) & 0xFFu;
    uint64_t out = (uint64_t)(b & 0x80000000u) << 32;
    if (e == 0xFFu) out |= 0x7FF0000000000000ull | ((uint64_t)(b & 0x7FFFFFu) << 29);
    else if (e != 0) out |= ((uint64_t)(e + 896u) << 52) | ((uint64_t)(b & 0x7FFFFFu) << 29);
    return __longlong_as_double((long long)out);
}

// out = a * b + c (complex)
template <typename Real>
__device__ __forceinline__ void cfma(Real ar, Real ai, Real br, Real bi, Real cr, Real ci, Real& outr, Real& outi) {
    Real r = fma(ar, br, fma(-ai, bi, cr));
    Real i = fma(ar, bi, fma(ai, br, ci));
    outr = r;
    outi = i;
}
template <typename Real>
__device__ __forceinline__ void cmul(Real ar, Real ai, Real br, Real bi, Real& outr, Real& outi) {
    Real r = fma(ar, br, -ai * bi);
    Real i = fma(ar, bi, ai * br);
    outr = r;
    outi = i;
}
// double-float: inner products left unnormalised, the outer fma renormalises
template <>
__device__ __forceinline__ void cfma<dfloat>(dfloat ar, dfloat ai, dfloat br, dfloat bi, dfloat cr, dfloat ci,
                                             dfloat& outr, dfloat& outi) {
    const dfloat r = fma(ar, br, fma_nr(-ai, bi, cr));
    const dfloat i = fma(ar, bi, fma_nr(ai, br, ci));
    outr = r;
    outi = i;
}
template <>
__device__ __forceinline__ void cmul<dfloat>(dfloat ar, dfloat ai, dfloat br, dfloat bi, dfloat& outr, dfloat& outi) {
    const dfloat r = fma(ar, br, -mul_nr(ai, bi));
    const dfloat i = fma(ar, bi, mul_nr(ai, br));
    outr = r;
    outi = i;
}

// out = a * b + c for a real addend c (the recurrence step m F + alpha)
template <typename Real>
__device__ __forceinline__ void cfma_ra(Real ar, Real ai, Real br, Real bi, Real cr, Real& outr, Real& outi) {
    cfma<Real>(ar, ai, br, bi, cr, Real(0), outr, outi);
}
// double-float: the inner products stay unnormalised (fma_nr) and the imaginary part
// has no addend
template <>
__device__ __forceinline__ void cfma_ra<dfloat>(dfloat ar, dfloat ai, dfloat br, dfloat bi, dfloat cr, dfloat& outr,
                                                dfloat& outi) {
    const dfloat r = fma(ar, br, fma_nr(-ai, bi, cr));
    const dfloat i = fma(ar, bi, mul_nr(ai, br));
    outr = r;
    outi = i;
}

// exp(-tau theta) for any theta >= 0, the anchor / span multiplier.
__device__ __forceinline__ void cexp_neg(double tr, double ti, double th, double& mr, double& mi) {
    double mag = exp(-tr * th);
    double sn, cs;
    sincos(ti * th, &sn, &cs);
    mr = mag * cs;
    mi = -mag * sn;
}
__device__ __forceinline__ void cexp_neg(float tr, float ti, float th, float& mr, float& mi) {
    float mag = expf(-tr * th);
    float sn, cs;
    sincosf(ti * th, &sn, &cs);
    mr = mag * cs;
    mi = -mag * sn;
}


template <typename Real>
struct TermConsts;
template <>
struct TermConsts<double> {
    __device__ static __forceinline__ double tc_re(const SweepConsts& c, int k, int j) { return c.tc_re[k][j]; }
    __device__ static __forceinline__ double tc_im(const SweepConsts& c, int k, int j) { return c.tc_im[k][j]; }
    __device__ static __forceinline__ double tau_re(const SweepConsts& c, int k) { return c.tau_re[k]; }
    __device__ static __forceinline__ double tau_im(const SweepConsts& c, int k) { return c.tau_im[k]; }
    __device__ static __forceinline__ uint32_t lim(const SweepConsts& c, int k, int d) { return c.theta_hi_lim[k][d]; }
    __device__ static __forceinline__ double w_re(const SweepConsts& c, int k) { return c.w_re[k]; }
    __device__ static __forceinline__ double w_im(const SweepConsts& c, int k) { return c.w_im[k]; }
    __device__ static __forceinline__ double v_re(const SweepConsts& c, int k) { return c.v_re[k]; }
    __device__ static __forceinline__ double v_im(const SweepConsts& c, int k) { return c.v_im[k]; }
};
template <>
struct TermConsts<float> {
    __device__ static __forceinline__ float tc_re(const SweepConsts& c, int k, int j) { return c.tcf_re[k][j]; }
    __device__ static __forceinline__ float tc_im(const SweepConsts& c, int k, int j) { return c.tcf_im[k][j]; }
    __device__ static __forceinline__ float tau_re(const SweepConsts& c, int k) { return c.tauf_re[k]; }
    __device__ static __forceinline__ float tau_im(const SweepConsts& c, int k) { return c.tauf_im[k]; }
    __device__ static __forceinline__ uint32_t lim(const SweepConsts& c, int k, int d) { return c.theta_hi_lim_f[k][d]; }
    __device__ static __forceinline__ float w_re(const SweepConsts& c, int k) { return c.wd_re[k][0]; }
    __device__ static __forceinline__ float w_im(const SweepConsts& c, int k) { return c.wd_im[k][0]; }
    __device__ static __forceinline__ float v_re(const SweepConsts& c, int k) { return c.vd_re[k][0]; }
    __device__ static __forceinline__ float v_im(const SweepConsts& c, int k) { return c.vd_im[k][0]; }
};
template <>
struct TermConsts<dfloat> {
    __device__ static __forceinline__ dfloat tc_re(const SweepConsts& c, int k, int j) {
        return df_make(c.tcd_re_hi[k][j], c.tcd_re_lo[k][j]);
    }
    __device__ static __forceinline__ dfloat tc_im(const SweepConsts& c, int k, int j) {
        return df_make(c.tcd_im_hi[k][j], c.tcd_im_lo[k][j]);
    }
    __device__ static __forceinline__ uint32_t lim(const SweepConsts& c, int k, int d) { return c.theta_hi_lim_d[k][d]; }
    __device__ static __forceinline__ dfloat w_re(const SweepConsts& c, int k) { return df_make(c.wd_re[k][0], c.wd_re[k][1]); }
    __device__ static __forceinline__ dfloat w_im(const SweepConsts& c, int k) { return df_make(c.wd_im[k][0], c.wd_im[k][1]); }
    __device__ static __forceinline__ dfloat v_re(const SweepConsts& c, int k) { return df_make(c.vd_re[k][0], c.vd_re[k][1]); }
    __device__ static __forceinline__ dfloat v_im(const SweepConsts& c, int k) { return df_make(c.vd_im[k][0], c.vd_im[k][1]); }
};

template <typename Real>
__device__ __forceinline__ uint32_t theta_hw(Real th);
template <>
__device__ __forceinline__ uint32_t theta_hw<double>(double th) {
    return (uint32_t)((uint64_t)__double_as_longlong(th) >> 32);
}
template <>
__device__ __forceinline__ uint32_t theta_hw<float>(float th) { return __float_as_uint(th); }
template <>
__device__ __forceinline__ uint32_t theta_hw<dfloat>(dfloat th) { return __float_as_uint(th.hi); }

// exp(-tau_k theta) beyond the Taylor range of the largest degree (rare)
template <typename Real>
__device__ __forceinline__ void cexp_term(const SweepConsts& c, int k, Real th, Real& mr, Real& mi) {
    cexp_neg(TermConsts<Real>::tau_re(c, k), TermConsts<Real>::tau_im(c, k), th, mr, mi);
}
// double-float: in FP64 from the FP64 tau_k (defined below)
template <>
__device__ __forceinline__ void cexp_term<dfloat>(const SweepConsts& c, int k, dfloat th, dfloat& mr, dfloat& mi);

template <typename Real>
struct MaxDegree;

// The double-float degree carries the split J (see taylor_split) in its bits 8 and up.
constexpr int kSplitShift = 8;

// Taylor degree for term k that covers every theta whose bit pattern is <= hw.
template <typename Real>
__device__ __forceinline__ int taylor_degree(const SweepConsts& c, int k, uint32_t hw) {
    int deg = MaxDegree<Real>::value;
#pragma unroll
    for (int d = MaxDegree<Real>::value - 1; d >= 0; --d)
        if (hw <= TermConsts<Real>::lim(c, k, d)) deg = d;
    if constexpr (std::is_same<Real, dfloat>::value) {
        int J = kTaylorMax;
#pragma unroll
        for (int j = kTaylorMax - 1; j >= 1; --j)
            if (hw <= c.theta_split_d[k][j]) J = j;
        deg |= J << kSplitShift;
    }
    return deg;
}

template <typename Real>
struct MaxDegree;
template <>
struct MaxDegree<double> { static constexpr int value = kTaylorMax; };
template <>
struct MaxDegree<float> { static constexpr int value = 8; };
template <>
struct MaxDegree<dfloat> { static constexpr int value = kTaylorMax; };

// Double-float exp(-tau_k theta) of degree D split at J (1 <= J): the head
// 1 + sum_{j<=J} c_j theta^j in double-float, the tail theta^(J+1) sum_{j>J} c_j theta^(j-J-1)
// in FP32 Horner.  J is chosen so that |tau_k theta|^(J+1) / (J+1)! <= 2^-28, which keeps
// the tail's rounding (at most (D + 1) 2^-24 relative) below 2^-48; c_j = (-tau_k)^j / j!.
template <typename Real>
__device__ __forceinline__ void taylor_split(const SweepConsts&, int, int, int, Real, Real&, Real&) {}
template <>
__device__ __forceinline__ void taylor_split<dfloat>(const SweepConsts& c, int k, int D, int J, dfloat th, dfloat& mr,
                                                     dfloat& mi) {
    const float t = th.hi;
    float tr = 0.f, ti = 0.f;  // the tail
    if (D > J) {
        float ar = c.tcf_re[k][D], ai = c.tcf_im[k][D], tp = t;
#pragma unroll 1
        for (int j = D - 1; j > J; --j) {
            ar = __fmaf_rn(ar, t, c.tcf_re[k][j]);
            ai = __fmaf_rn(ai, t, c.tcf_im[k][j]);
        }
#pragma unroll 1
        for (int j = 0; j < J; ++j) tp = __fmul_rn(tp, t);
        tr = __fmul_rn(ar, tp);
        ti = __fmul_rn(ai, tp);
    } else {
        J = D;
    }
    if (J == 0) {
        mr = dfloat(1.f);
        mi = dfloat(0.f);
    } else if (J == 1) {
        // 1 + c_1 theta: the product of the high parts split exactly (FMA), the cross
        // terms added to its error
        const float c1r = c.tcd_re_hi[k][1], c1rl = c.tcd_re_lo[k][1];
        const float c1i = c.tcd_im_hi[k][1], c1il = c.tcd_im_lo[k][1];
        const float pr = __fmul_rn(c1r, t), pi = __fmul_rn(c1i, t);
        float er = __fmaf_rn(c1r, t, -pr), ei = __fmaf_rn(c1i, t, -pi);
        er = __fmaf_rn(c1r, th.lo, __fmaf_rn(c1rl, t, er));
        ei = __fmaf_rn(c1i, th.lo, __fmaf_rn(c1il, t, ei));
        const dfloat h = fast_two_sum(1.f, pr);  // |pr| < 1
        mr = fast_two_sum(h.hi, __fadd_rn(h.lo, __fadd_rn(er, tr)));
        mi = fast_two_sum(pi, __fadd_rn(ei, ti));
        return;
    } else {
        dfloat hr = dfloat(c.tcd_re_hi[k][J], c.tcd_re_lo[k][J]), hi = dfloat(c.tcd_im_hi[k][J], c.tcd_im_lo[k][J]);
#pragma unroll 1
        for (int j = J - 1; j >= 1; --j) {
            hr = fma(hr, th, dfloat(c.tcd_re_hi[k][j], c.tcd_re_lo[k][j]));
            hi = fma(hi, th, dfloat(c.tcd_im_hi[k][j], c.tcd_im_lo[k][j]));
        }
        mr = fma(hr, th, dfloat(1.f));
        mi = hi * th;
    }
    if (D > J) {
        mr = fast_two_sum(mr.hi, __fadd_rn(mr.lo, tr));
        mi = fast_two_sum(mi.hi, __fadd_rn(mi.lo, ti));
    }
}

// Signed fixed point with 2^-62 resolution, for sums of a few floats below 2 in size.
// f32_to_fix62 truncates toward zero below 2^-62; fix62_to_f64 rounds to nearest.
__device__ __forceinline__ int64_t f32_to_fix62(float f) {
    const uint32_t b = __float_as_uint(f);
    const int e = (int)((b >> 23) & 0xFFu);
    if (e == 0) return 0;  // zero, or below 2^-126
    const int64_t m = (int64_t)((b & 0x7FFFFFu) | 0x800000u);  // f = m 2^(e - 150)
    const int sh = e - 88;                                       // f 2^62 = m 2^sh
    const int64_t v = sh >= 0 ? (m << sh) : (sh > -25 ? (m >> -sh) : 0);
    return (b >> 31) ? -v : v;
}
__device__ __forceinline__ double fix62_to_f64(int64_t v) {
    if (v == 0) return 0.0;
    const uint64_t sign = v < 0 ? 0x8000000000000000ull : 0ull;
    const uint64_t a = v < 0 ? (uint64_t)(-v) : (uint64_t)v;
    const int msb = 63 - __clzll((long long)a);
    int e = msb - 62;
    uint64_t mant;
    if (msb > 52) {
        const int sh = msb - 52;
        mant = (a >> sh) + ((a >> (sh - 1)) & 1ull);
        if (mant >> 53) {
            mant >>= 1;
            ++e;
        }
    } else {
        mant = a << (52 - msb);
    }
    return __longlong_as_double((long long)(sign | ((uint64_t)(e + 1023) << 52) | (mant & 0xFFFFFFFFFFFFFull)));
}

// FP64 exp(-tau_k theta) of degree D >= 2 for |tau_k| theta <= 2^-10 (warp-uniform), with
// two FP64 operations: m = (1 + T) + c_1 theta and i(T') + c_1 theta by one DFMA each, where
// T = sum_{j>=2} c_j theta^j is formed off the FP64 pipe.  theta is split exactly into
// two floats (top 24 bits, rest), c_2 theta^2 is a float pair (FMA two-products with
// c_2 as a float pair), the terms of degree >= 3 are one FP32 Horner sum (below
// |tau theta|^3 / 6 <= 2^-32.6, so its FP32 rounding is below 2^-54), and 1 + T is
// summed in 62-bit fixed point and rounded once to FP64.  The result carries the
// rounding of two FP64 operations, like the full FP64 polynomial's last steps.
template <int D>
__device__ __forceinline__ void taylor_hybrid(const SweepConsts& c, int k, double th, double& mr, double& mi) {
    const uint64_t tb = (uint64_t)__double_as_longlong(th);
    const int E = (int)(tb >> 52);  // theta >= 0
    float thf = 0.f, tlf = 0.f;
    if (E > 1023 - 100) {  // below 2^-100 the theta^2 terms vanish far under 2^-53
        const uint64_t m = tb & 0xFFFFFFFFFFFFFull;
        thf = __uint_as_float(((uint32_t)(E - 896) << 23) | (uint32_t)(m >> 29));
        tlf = u64_scaled_to_f32(m & 0x1FFFFFFFull, E - 1075);
    }
    // theta^2 = p + pe
    const float p = __fmul_rn(thf, thf);
    float pe = __fmaf_rn(thf, thf, -p);
    pe = __fmaf_rn(__fmul_rn(2.f, thf), tlf, pe);
    // c_2 theta^2 = q + qe (real and imaginary parts)
    const float c2r = c.tcd_re_hi[k][2], c2rl = c.tcd_re_lo[k][2], c2i = c.tcd_im_hi[k][2], c2il = c.tcd_im_lo[k][2];
    const float qr = __fmul_rn(c2r, p), qi = __fmul_rn(c2i, p);
    float qer = __fmaf_rn(c2r, p, -qr), qei = __fmaf_rn(c2i, p, -qi);
    qer = __fmaf_rn(c2r, pe, __fmaf_rn(c2rl, p, qer));
    qei = __fmaf_rn(c2i, pe, __fmaf_rn(c2il, p, qei));
    if constexpr (D >= 3) {
        float ar = c.tcf_re[k][D], ai = c.tcf_im[k][D];
#pragma unroll
        for (int j = D - 1; j >= 3; --j) {
            ar = __fmaf_rn(ar, thf, c.tcf_re[k][j]);
            ai = __fmaf_rn(ai, thf, c.tcf_im[k][j]);
        }
        const float t3 = __fmul_rn(p, thf);
        qer = __fmaf_rn(ar, t3, qer);
        qei = __fmaf_rn(ai, t3, qei);
    }
    const double sr = fix62_to_f64((int64_t(1) << 62) + f32_to_fix62(qr) + f32_to_fix62(qer));
    const double si = fix62_to_f64(f32_to_fix62(qi) + f32_to_fix62(qei));
    mr = fma(c.tc_re[k][1], th, sr);
    mi = fma(c.tc_im[k][1], th, si);
}

// A Taylor degree known only at run time (warp-uniform): the double-float path, whose
// Horner steps are long enough that a loop costs little and one code path per degree
// would only grow the kernel.
struct RtDeg {
    static constexpr int value = -1;
    int d;  // degree
    int J;  // head degree of taylor_split
};

// exp(-tau_k theta) by a Taylor polynomial of degree Dc (Horner, complex coefficients,
// real theta).  At the largest degree, points beyond its threshold fall back to
// exp/sincos; below it the warp-uniform degree already covers every point.
template <typename Real, typename Dc>
__device__ __forceinline__ void taylor(const SweepConsts& c, int k, Dc dc, Real th, Real& mr, Real& mi,
                                       bool hybrid = false) {
    if constexpr (Dc::value >= 2 && std::is_same<Real, double>::value) {
        if (hybrid) {
            taylor_hybrid<Dc::value>(c, k, th, mr, mi);
            return;
        }
    }
    if constexpr (Dc::value >= 0) {
        constexpr int D = Dc::value;
        if constexpr (D == 0) {
            mr = Real(1);
            mi = Real(0);
        } else {
            Real ar = TermConsts<Real>::tc_re(c, k, D), ai = TermConsts<Real>::tc_im(c, k, D);
#pragma unroll
            for (int j = D - 1; j >= 1; --j) {
                ar = fma(ar, th, TermConsts<Real>::tc_re(c, k, j));
                ai = fma(ai, th, TermConsts<Real>::tc_im(c, k, j));
            }
            mr = fma(ar, th, Real(1));
            mi = ai * th;
        }
        if constexpr (D == MaxDegree<Real>::value) {
            if (theta_hw<Real>(th) > TermConsts<Real>::lim(c, k, D)) cexp_term<Real>(c, k, th, mr, mi);
        }
    } else {
        const int D = dc.d;
        taylor_split(c, k, D, dc.J, th, mr, mi);
        if (D == MaxDegree<Real>::value && theta_hw<Real>(th) > TermConsts<Real>::lim(c, k, D))
            cexp_term<Real>(c, k, th, mr, mi);
    }
}

// Runs body(Dc) for the warp-uniform degree deg: a compile-time degree
// (integral_constant) on the FP64 / FP32 paths, RtDeg for double-float.
template <typename Real, typename Body>
__device__ __forceinline__ void with_degree(int deg, Body&& body) {
    if constexpr (std::is_same<Real, dfloat>::value) {
        body(RtDeg{deg & ((1 << kSplitShift) - 1), deg >> kSplitShift});
    } else {
        switch (deg) {
            case 0: body(std::integral_constant<int, 0>{}); break;
            case 1: body(std::integral_constant<int, 1>{}); break;
            case 2: body(std::integral_constant<int, 2>{}); break;
            case 3: body(std::integral_constant<int, 3>{}); break;
            case 4: body(std::integral_constant<int, 4>{}); break;
            case 5: body(std::integral_constant<int, 5>{}); break;
            case 6: body(std::integral_constant<int, 6>{}); break;
            case 7: body(std::integral_constant<int, 7>{}); break;
            default:
                if constexpr (MaxDegree<Real>::value == 8) {
                    body(std::integral_constant<int, 8>{});
                } else {
                    switch (deg) {
                        case 8: body(std::integral_constant<int, 8>{}); break;
                        case 9: body(std::integral_constant<int, 9>{}); break;
                        case 10: body(std::integral_constant<int, 10>{}); break;
                        case 11: body(std::integral_constant<int, 11>{}); break;
                        default: body(std::integral_constant<int, MaxDegree<Real>::value>{}); break;
                    }
                }
        }
    }
}

// Single multiplier for a warp whose largest theta has bit pattern hw (thread spans):
// the degree, and the FP64 head + FP32 tail form when it applies, follow from hw.
template <typename Real>
__device__ __forceinline__ void multiplier(const SweepConsts& c, int k, uint32_t hw, Real th, Real& mr, Real& mi) {
    const bool hyb = std::is_same<Real, double>::value && hw <= c.theta_hyb_lim[k];
    with_degree<Real>(taylor_degree<Real>(c, k, hw), [&](auto Dc) { taylor<Real>(c, k, Dc, th, mr, mi, hyb); });
}

__device__ __forceinline__ void publish_agg(TileDesc* d, double ar, double ai, double Mr, double Mi) {
    d->agg_re = ar;
    d->agg_im = ai;
    d->M_re = Mr;
    d->M_im = Mi;
    __threadfence();
    st_volatile_u32(&d->flag, 1u);
}
__device__ __forceinline__ void publish_inc(TileDesc* d, double ir, double ii) {
    d->inc_re = ir;
    d->inc_im = ii;
    __threadfence();
    st_volatile_u32(&d->flag, 2u);
}

// Decoupled look-back for term k by one warp over the tiles tile+dir, tile+2 dir, ...
// (dir = -1 forward, +1 backward) of the same item ([lo, hi)), 32 tiles per round trip.  Returns (in every lane)
// the state at the anchor of the adjacent tile:
//     C = agg_{t1} + M_{t1} (agg_{t2} + M_{t2} (... + M_{tj} inc_{tj}))
// up to the nearest tile whose inclusive value is published.  Every M is one tile's
// span multiplier, computed directly from its anchor coordinates when it was published;
// within a round the products of M are formed by a lane prefix scan.
static __device__ __noinline__ void look_back_warp(const TileDesc* desc, int64_t tile, int dir, int64_t lo,
                                                   int64_t hi, int ne, int k, double& Cr, double& Ci,
                                                   uint32_t* status, long long spin_limit) {
    const int lane = threadIdx.x & 31;
    double Pr = 1.0, Pi = 0.0;  // product of the span multipliers of the tiles consumed so far
    Cr = 0.0;
    Ci = 0.0;
    int64_t jb = tile + dir;
    bool timed_out = false;
    while (true) {
        const int64_t j = jb + (int64_t)dir * lane;
        const bool valid = j >= lo && j < hi;  // the item's own tiles only
        const TileDesc* d = desc + (valid ? j : 0) * ne + k;
        uint32_t f = 2;
        if (valid) {
            f = ld_volatile_u32(&d->flag);
            if (f == 0) {
                const long long t0 = clock64();
                while ((f = ld_volatile_u32(&d->flag)) == 0) {
                    if (clock64() - t0 > spin_limit) {
                        timed_out = true;
                        f = 2;
                        break;
                    }
                }
            }
        }
        __threadfence();
        double vr = 0.0, vi = 0.0, mr = 1.0, mi = 0.0;
        if (valid && !timed_out) {
            if (f == 2) {
                vr = __ldcg(&d->inc_re);
                vi = __ldcg(&d->inc_im);
            } else {
                vr = __ldcg(&d->agg_re);
                vi = __ldcg(&d->agg_im);
            }
            mr = __ldcg(&d->M_re);
            mi = __ldcg(&d->M_im);
        }
        const unsigned incm = __ballot_sync(0xffffffffu, f == 2);
        if (incm & 1u) {
            // the nearest tile of this round has its inclusive value (the usual case: the
            // previous tile finished its own look-back first): C += P v_0, no prefix scan
            const double v0r = __shfl_sync(0xffffffffu, vr, 0), v0i = __shfl_sync(0xffffffffu, vi, 0);
            cfma<double>(Pr, Pi, v0r, v0i, Cr, Ci, Cr, Ci);
            break;
        }
        const int last = incm ? __ffs(incm) - 1 : 31;
        // inclusive prefix product of M over lanes, then exclusive
        double Er = mr, Ei = mi;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const double orr = __shfl_up_sync(0xffffffffu, Er, o), oi = __shfl_up_sync(0xffffffffu, Ei, o);
            if (lane >= o) cmul<double>(Er, Ei, orr, oi, Er, Ei);
        }
        double Xr = __shfl_up_sync(0xffffffffu, Er, 1), Xi = __shfl_up_sync(0xffffffffu, Ei, 1);
        if (lane == 0) { Xr = 1.0; Xi = 0.0; }
        double tr = 0.0, ti = 0.0;
        if (lane <= last) cmul<double>(Xr, Xi, vr, vi, tr, ti);
#pragma unroll
        for (int o = 16; o >= 1; o >>= 1) {
            tr += __shfl_xor_sync(0xffffffffu, tr, o);
            ti += __shfl_xor_sync(0xffffffffu, ti, o);
        }
        cfma<double>(Pr, Pi, tr, ti, Cr, Ci, Cr, Ci);
        if (incm) break;
        const double Lr = __shfl_sync(0xffffffffu, Er, 31), Li = __shfl_sync(0xffffffffu, Ei, 31);
        cmul<double>(Pr, Pi, Lr, Li, Pr, Pi);
        jb += 32 * (int64_t)dir;
    }
    if (__any_sync(0xffffffffu, timed_out) && lane == 0) atomicOr(status, kStatusTimeout);
}

// Shared-memory layout: coordinates (double), later overwritten by the gaps (Real) and
// finally by the output; strengths (Real); per-term exclusive thread prefixes (Real).
// Per-point arrays are padded one slot per R points so that a warp reading one point
// per thread (stride R) hits distinct banks.
// The FP64 sweeps keep the scan region transposed for the serial warp scan (ScanIndex).
template <typename Real, int NE, int T, int R>
struct SweepSmem {
    static constexpr int TILE = T * R;
    static constexpr int TP = TILE + TILE / R + 2;
    static constexpr size_t z_off = 0;
    static constexpr size_t al_off = z_off + sizeof(double) * TP;
    static constexpr size_t scan_off = (al_off + sizeof(Real) * TP + 15) / 16 * 16;
    static constexpr size_t scan_elems = std::is_same<Real, double>::value ? 4 * ((size_t)NE * T + 32)
                                                                            : 4 * (size_t)NE * T;
    static constexpr size_t bytes = scan_off + sizeof(Real) * scan_elems;
};

// FP64 scan region: component c (Re M, Im M, Re F, Im F) of thread position j (lane) in
// warp w for term kk of the group is at c * 32 * S + j * S + kk * NW + w, S = NG NW + 1.
// The threads of a warp (one term) write a column with stride S (about 2-way bank
// conflicts); the lanes of the serial scan (one sequence each) read a row, consecutive.
template <int NG, int NW>
struct ScanIndex {
    static constexpr int S = NG * NW + 1;
    __device__ static __forceinline__ int at(int c, int j, int kk, int w) { return c * 32 * S + j * S + kk * NW + w; }
};

// Serial warp scan of the FP64 sweeps: the NW x (g1 - g0) sequences (one per warp and
// term of the group) of 32 thread aggregates (M, F) each -- a thread's state map
// h -> M h + F -- are combined by one lane each, in sweep order (lane 0 to 31 forward,
// 31 to 0 backward).  Each entry is replaced by the exclusive composition of the
// threads before it in sweep order and the warp's total goes to s_w.  Eight FP64
// operations per thread and term, against forty for a shuffle scan over 32 lanes.
template <int NG, int NW, bool kFwd, int NE>
__device__ __forceinline__ void serial_warp_scan(double* s_scan, double (*s_w)[NW][4], int g0, int g1) {
    using SI = ScanIndex<NG, NW>;
    const int nseq = NW * (g1 - g0);
    for (int q = threadIdx.x; q < nseq; q += blockDim.x) {
        const int kk = q / NW, w = q % NW;
        double Pr = 1.0, Pi = 0.0, Xr = 0.0, Xi = 0.0;
#pragma unroll 4
        for (int jj = 0; jj < 32; ++jj) {
            const int j = kFwd ? jj : 31 - jj;
            double* e0 = s_scan + SI::at(0, j, kk, w);
            double* e1 = s_scan + SI::at(1, j, kk, w);
            double* e2 = s_scan + SI::at(2, j, kk, w);
            double* e3 = s_scan + SI::at(3, j, kk, w);
            const double mr = *e0, mi = *e1, fr = *e2, fi = *e3;
            *e0 = Pr;
            *e1 = Pi;
            *e2 = Xr;
            *e3 = Xi;
            double nr, ni;
            cfma<double>(mr, mi, Xr, Xi, fr, fi, nr, ni);  // X <- M X + F
            Xr = nr;
            Xi = ni;
            cmul<double>(mr, mi, Pr, Pi, Pr, Pi);          // P <- M P
        }
        s_w[g0 + kk][w][0] = Pr;
        s_w[g0 + kk][w][1] = Pi;
        s_w[g0 + kk][w][2] = Xr;
        s_w[g0 + kk][w][3] = Xi;
    }
}

// Terms per group.  The value-channel sweeps run their terms in equal groups, each
// with its own phases A-C, when the scan region of all NE terms would push the tile's
// shared memory past the occupancy target (two resident tiles per SM for 8-byte reals,
// three for FP32); the derivative channel keeps one group, since its accumulators live
// over the gaps that every phase A reads.
template <typename Real, int NE, int T, int R, int EV, bool CO>
struct SweepGroup {
    static constexpr size_t kBudget = sizeof(Real) == 8 ? 110 * 1024 : 72 * 1024;
    static constexpr int pick() {
        if (EV != 1 || CO) return NE;
        for (int G = 1; G <= NE; ++G) {
            const int n = (NE + G - 1) / G;
            const size_t scan = std::is_same<Real, double>::value ? 4 * ((size_t)n * T + 32) : 4 * (size_t)n * T;
            if (SweepSmem<Real, 1, T, R>::scan_off + sizeof(Real) * scan <= kBudget) return n;
        }
        return 1;
    }
    static constexpr int NG = pick();
};

// Resident tiles per SM that the shared-memory footprint allows (8-byte reals: two;
// FP32: three), given to the register allocator as the occupancy target.
template <typename Real>
struct SweepMinBlocks { static constexpr int value = sizeof(Real) == 8 ? 2 : 3; };

template <int R>
__device__ __forceinline__ int pad(int i) { return i + i / R; }

// Multiplier table entries (16 bytes): an FP64 complex, or a double-float complex stored
// as (re.hi, re.lo, im.hi, im.lo).
template <typename Real>
struct TableEntry;
template <>
struct TableEntry<double> {
    __device__ static __forceinline__ void store(double2* p, double mr, double mi) { *p = make_double2(mr, mi); }
    __device__ static __forceinline__ void load(const double2* p, double& mr, double& mi) {
        const double2 m = *p;
        mr = m.x;
        mi = m.y;
    }
};
template <>
struct TableEntry<dfloat> {
    __device__ static __forceinline__ void store(double2* p, dfloat mr, dfloat mi) {
        *reinterpret_cast<float4*>(p) = make_float4(mr.hi, mr.lo, mi.hi, mi.lo);
    }
    __device__ static __forceinline__ void load(const double2* p, dfloat& mr, dfloat& mi) {
        const float4 m = *reinterpret_cast<const float4*>(p);
        mr = dfloat(m.x, m.y);
        mi = dfloat(m.z, m.w);
    }
};


template <typename Real>
__device__ __forceinline__ Real to_real(double v);
template <>
__device__ __forceinline__ double to_real<double>(double v) { return v; }
template <>
__device__ __forceinline__ float to_real<float>(double v) { return f64_to_f32(v); }
template <>
__device__ __forceinline__ dfloat to_real<dfloat>(double v) {
    const float hi = f64_to_f32(v);
    return df_make(hi, f64_to_f32(v - f32_to_f64(hi)));
}

// 1/sqrt(delta) in the three precisions (the double-float split costs one DADD)
struct Scale {
    double d;
    float f;
    dfloat df;
};
template <typename Real>
__device__ __forceinline__ Scale make_scale(double s) {
    Scale sc;
    sc.d = s;
    sc.f = std::is_same<Real, double>::value ? 0.f : f64_to_f32(s);
    sc.df = std::is_same<Real, dfloat>::value ? to_real<dfloat>(s) : df_make(0.f, 0.f);
    return sc;
}

// b - a (b >= a) as a double-float: exact when a and b are normal, of one sign and in
// one binade (the integer difference of the bit patterns has at most 48 significant
// bits for neighbours); otherwise through an FP64 subtraction.
__device__ __forceinline__ dfloat gap_df(double a, double b) {
    const uint64_t ba = (uint64_t)__double_as_longlong(a), bb = (uint64_t)__double_as_longlong(b);
    const uint32_t ea = (uint32_t)(ba >> 52) & 0x7FFu, eb = (uint32_t)(bb >> 52) & 0x7FFu;
    if (ea == eb && ea != 0 && ea != 0x7FF && ((ba ^ bb) >> 63) == 0) {
        const uint64_t d = bb >= ba ? bb - ba : ba - bb;
        const int e2 = (int)ea - 1075;
        if (d == 0) return df_make(0.f, 0.f);
        const int msb = 63 - __clzll((long long)d);
        if (msb <= 23) return df_make(u64_scaled_to_f32(d, e2), 0.f);
        const int sh = msb - 23;
        const uint64_t m = (d >> sh) + ((d >> (sh - 1)) & 1ull);
        const uint64_t dh = m << sh;
        const float hi = u64_scaled_to_f32(dh, e2);
        const float lo = d >= dh ? u64_scaled_to_f32(d - dh, e2) : -u64_scaled_to_f32(dh - d, e2);
        return df_make(hi, lo);
    }
    return to_real<dfloat>(b - a);
}

// b - a (b >= a) in FP64 without an FP64 subtraction: for normal a and b of one sign in
// one binade the integer difference of the bit patterns is the exact difference in
// units of the binade's ulp (below 2^52, so exactly representable); otherwise FP64.
__device__ __forceinline__ double gap_f64(double a, double b) {
    const uint64_t ba = (uint64_t)__double_as_longlong(a), bb = (uint64_t)__double_as_longlong(b);
    const uint32_t ea = (uint32_t)(ba >> 52) & 0x7FFu, eb = (uint32_t)(bb >> 52) & 0x7FFu;
    if (ea == eb && ea > 53 && ea != 0x7FF && ((ba ^ bb) >> 63) == 0) {
        const uint64_t d = bb >= ba ? bb - ba : ba - bb;
        if (d == 0) return 0.0;
        const int msb = 63 - __clzll((long long)d);  // < 52
        // d * 2^(ea - 1075): exponent field ea - 52 + msb (>= 1 since ea > 53)
        const uint64_t bits = ((uint64_t)(ea - 52 + msb) << 52) | ((d << (52 - msb)) & 0xFFFFFFFFFFFFFull);
        return __longlong_as_double((long long)bits);
    }
    return b - a;
}

template <typename Real>
__device__ __forceinline__ Real gap_real(double a, double b, const Scale& sc);
template <>
__device__ __forceinline__ double gap_real<double>(double a, double b, const Scale& sc) { return sc.d * gap_f64(a, b); }
template <>
__device__ __forceinline__ float gap_real<float>(double a, double b, const Scale& sc) { return sc.f * gap_f32(a, b); }
template <>
__device__ __forceinline__ dfloat gap_real<dfloat>(double a, double b, const Scale& sc) { return sc.df * gap_df(a, b); }

// Stages the tile: coordinates, strengths (0 at targets) and target bits.  Points past
// the end get z = 0, alpha = 0 and are not targets.  The loads go in chunks of kChunk
// points per thread, all issued before any is used (keys and codes, then the strength
// gathers they index), so a tile waits for two memory round trips per chunk instead of
// two per point.
template <typename Real, int T, int R>
__device__ __forceinline__ void stage_tile(const SweepArgs& a, const uint64_t* __restrict__ keys,
                                           const uint32_t* __restrict__ vals, int64_t base, int nvalid,
                                           double* s_z, Real* s_al, uint32_t* s_tgt) {
    constexpr int TILE = T * R;
    constexpr int kIter = TILE / T;  // points per thread
    constexpr int kChunk = kIter < 8 ? kIter : 8;
    static_assert(kIter % kChunk == 0, "whole chunks");
    const int tid = threadIdx.x, lane = tid & 31;
#pragma unroll 1
    for (int c0 = 0; c0 < kIter; c0 += kChunk) {
        uint64_t kk[kChunk];
        uint32_t vv[kChunk];
#pragma unroll
        for (int q = 0; q < kChunk; ++q) {
            const int i = (c0 + q) * T + tid;
            kk[q] = 0;
            vv[q] = 0xFFFFFFFFu;
            if (i < nvalid) {
                kk[q] = keys[base + i];
                vv[q] = vals[base + i];
            }
        }
        double al[kChunk];
#pragma unroll
        for (int q = 0; q < kChunk; ++q) {
            const int i = (c0 + q) * T + tid;
            al[q] = (i < nvalid && (int64_t)vv[q] < a.N) ? __ldg(&a.alpha[vv[q]]) : 0.0;
        }
#pragma unroll
        for (int q = 0; q < kChunk; ++q) {
            const int i = (c0 + q) * T + tid;
            bool tg = false;
            double z = 0.0;
            if (i < nvalid) {
                z = key_coord(kk[q]);
                // a target, or any point when targets and sources are identical
                tg = (int64_t)vv[q] >= a.N || a.self != 0;
            }
            s_z[pad<R>(i)] = z;
            s_al[pad<R>(i)] = to_real<Real>(al[q]);
            const unsigned b = __ballot_sync(0xffffffffu, tg);
            if (lane == 0) s_tgt[i >> 5] = b;
        }
    }
}

// Phase B for term k by one warp: combine the warp totals s_w[k][.] in sweep order,
// publish aggregate + span multiplier, look back, publish the inclusive value, and
// leave the state entering each warp in s_win[k][.].
template <int NE, int NW>
__device__ __forceinline__ void tile_combine(const SweepArgs& a, TileDesc* desc, int64_t tile, int64_t lo, int64_t hi,
                                             int dir, bool first_in_dir, double Mr, double Mi, double (*s_w)[NW][4],
                                             double (*s_win)[NW][2], int k) {
    const int lane = threadIdx.x & 31;
    // lane q < NW takes the warp at sweep position q and the lanes scan the pairs
    // (M, F) -> h = M h + F over positions (log2 NW shuffle steps); lanes >= NW hold the
    // identity
    const int ww = dir < 0 ? lane : NW - 1 - lane;
    double Pr = 1, Pi = 0, Qr = 0, Qi = 0;
    if (lane < NW) {
        Pr = s_w[k][ww][0];
        Pi = s_w[k][ww][1];
        Qr = s_w[k][ww][2];
        Qi = s_w[k][ww][3];
    }
#pragma unroll
    for (int o = 1; o < NW; o <<= 1) {
        const double por = __shfl_up_sync(0xffffffffu, Pr, o), poi = __shfl_up_sync(0xffffffffu, Pi, o);
        const double qor = __shfl_up_sync(0xffffffffu, Qr, o), qoi = __shfl_up_sync(0xffffffffu, Qi, o);
        if (lane >= o) {
            cfma<double>(Pr, Pi, qor, qoi, Qr, Qi, Qr, Qi);
            cmul<double>(Pr, Pi, por, poi, Pr, Pi);
        }
    }
    // exclusive prefix (the state map before this lane's warp) and the tile aggregate
    double pre0 = __shfl_up_sync(0xffffffffu, Pr, 1), pre1 = __shfl_up_sync(0xffffffffu, Pi, 1);
    double pre2 = __shfl_up_sync(0xffffffffu, Qr, 1), pre3 = __shfl_up_sync(0xffffffffu, Qi, 1);
    if (lane == 0) { pre0 = 1; pre1 = 0; pre2 = 0; pre3 = 0; }
    Qr = __shfl_sync(0xffffffffu, Qr, NW - 1);
    Qi = __shfl_sync(0xffffffffu, Qi, NW - 1);
    TileDesc* dd = desc + tile * NE + k;
    double Cr = 0, Ci = 0;
    if (lane == 0) publish_agg(dd, Qr, Qi, Mr, Mi);
    __syncwarp();
    if (first_in_dir) {
        if (lane == 0) publish_inc(dd, Qr, Qi);
    } else {
        look_back_warp(desc, tile, dir, lo, hi, NE, k, Cr, Ci, a.status, a.spin_limit);
        if (lane == 0) {
            double Ir, Ii;
            cfma<double>(Mr, Mi, Cr, Ci, Qr, Qi, Ir, Ii);
            publish_inc(dd, Ir, Ii);
        }
    }
    if (lane < NW) {
        double xr, xi;
        cfma<double>(pre0, pre1, Cr, Ci, pre2, pre3, xr, xi);
        s_win[k][ww][0] = xr;
        s_win[k][ww][1] = xi;
    }
}

template <typename Real>
__device__ __forceinline__ double real_to_f64(Real v);
template <>
__device__ __forceinline__ double real_to_f64<double>(double v) { return v; }
template <>
__device__ __forceinline__ double real_to_f64<float>(float v) { return f32_to_f64(v); }
template <>
__device__ __forceinline__ double real_to_f64<dfloat>(dfloat v) { return f32_to_f64(v.hi) + f32_to_f64(v.lo); }

template <>
__device__ __forceinline__ void cexp_term<dfloat>(const SweepConsts& c, int k, dfloat th, dfloat& mr, dfloat& mi) {
    double a, b;
    cexp_neg(c.tau_re[k], c.tau_im[k], real_to_f64<dfloat>(th), a, b);
    mr = to_real<dfloat>(a);
    mi = to_real<dfloat>(b);
}

template <typename Real>
__device__ __forceinline__ Real shfl_up(Real v, int o) { return __shfl_up_sync(0xffffffffu, v, o); }
template <>
__device__ __forceinline__ dfloat shfl_up<dfloat>(dfloat v, int o) { return df_shfl_up(v, o); }
template <typename Real>
__device__ __forceinline__ Real shfl_down(Real v, int o) { return __shfl_down_sync(0xffffffffu, v, o); }
template <>
__device__ __forceinline__ dfloat shfl_down<dfloat>(dfloat v, int o) { return df_shfl_down(v, o); }

// EV: evaluation channels (bit 0 values, bit 1 derivative).  CO: coincidence mode
// (NE = 1, multiplier 1 on zero gaps and 0 otherwise, unit weight; the per-target sums
// are written straight to a.u), used by the gradients.
template <typename Real, int NE, int T, int R, int EV, bool CO>
__global__ void __launch_bounds__(T, SweepMinBlocks<Real>::value) k_sweep_fwd(const SweepArgs a, const SweepConsts c) {
    constexpr int NG = SweepGroup<Real, NE, T, R, EV, CO>::NG;
    using SM = SweepSmem<Real, NG, T, R>;
    constexpr int TILE = T * R;
    constexpr int NW = T / 32;
    constexpr bool kF64 = std::is_same<Real, double>::value;
    // multipliers stored by phase A and reloaded (FP64 and double-float); FP32 recomputes
    constexpr bool kTab = kF64 || std::is_same<Real, dfloat>::value;
    constexpr int kUnrollC = sizeof(Real) == 8 ? 4 : 8;       // phase C unroll, recomputed multipliers
    static_assert(!((EV & 2) && std::is_same<Real, dfloat>::value), "no derivative channel in double-float");
    static_assert((EV & 2) == 0 || NG == NE, "the derivative channel runs its terms as one group");
    extern __shared__ __align__(16) unsigned char smem[];
    double* s_z = reinterpret_cast<double*>(smem + SM::z_off);
    Real* s_th = reinterpret_cast<Real*>(smem + SM::z_off);  // gaps, written over s_z
    Real* s_al = reinterpret_cast<Real*>(smem + SM::al_off);
    Real* s_scan = reinterpret_cast<Real*>(smem + SM::scan_off);  // [NE][4][T]
    __shared__ double s_w[NE][NW][4];
    __shared__ double s_win[NE][NW][2];
    __shared__ double s_M[NE][2];
    __shared__ uint32_t s_tgt[TILE / 32];
    __shared__ uint32_t s_tile;
    __shared__ double s_zprev;

    static_assert(TILE == kTile, "a sweep tile is one item tile");
    __shared__ int s_item;
    const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
    // persistent: each CTA takes tiles in order from the counter until none is left
    for (;;) {
    if (tid == 0) {
        s_tile = atomicAdd(&a.tile_ctr[0], 1u);
        s_item = (int64_t)s_tile < *a.total_tiles ? item_of_tile(a.items, a.B, s_tile) : -1;
        if (ld_volatile_u32(a.status) & kStatusSortTimeout) s_item = -1;  // sorted codes not valid
        if (CO && a.ties && ld_volatile_u32(a.ties) == 0) s_item = -1;   // no equal coordinates
    }
    __syncthreads();
    if (s_item < 0) return;
    const Item itm = a.items[s_item];
    const int64_t tile = s_tile;
    const int64_t base = tile * TILE;
    const int64_t local = base - itm.start;
    const int nvalid = (int)min((int64_t)TILE, itm.nsrc + itm.ntgt - local);
    const bool first = local == 0;
    const double s = itm.s;
    // the coincidence sweep compares gaps with zero: unscaled, so that no gap between
    // distinct coordinates underflows
    const Scale sc = make_scale<Real>(CO ? 1.0 : s);
    const bool bufB = a.plan->final_buf == 1;
    const uint64_t* __restrict__ keys = bufB ? a.keysB : a.keysA;
    const uint32_t* __restrict__ vals = bufB ? a.valsB : a.valsA;
    // the previous tile's last coordinate, loaded before the staging so that both overlap
    const uint64_t kprev = (tid == 0 && !first) ? keys[base - 1] : 0ull;
    stage_tile<Real, T, R>(a, keys, vals, base, nvalid, s_z, s_al, s_tgt);
    if (tid == 0) s_zprev = !first ? key_coord(kprev) : 0.0;
    __syncthreads();

    const int i0 = tid * R;
    const double zprev = s_zprev, zend = s_z[pad<R>(nvalid - 1)];
    // multipliers read from a bound geometry's table (FP64, double-float): no gaps needed
    const bool reuse = kTab && !CO && a.reuse;
    // gaps of my R points, warp-wide largest gap
    Real thr[R];
    uint32_t hw = 0;
    bool tie = false;  // a zero gap: two merged points share a coordinate
    // (gradient sweeps only: the value channel's kernels stay free of this check)
    const bool track_ties = !CO && (EV & 2) != 0 && a.ties != nullptr;
    if (!reuse) {
#pragma unroll
        for (int r = 0; r < R; ++r) {
            const int i = i0 + r;
            Real t = 0;
            if (i < nvalid && (i > 0 || !first))
                t = gap_real<Real>(i > 0 ? s_z[pad<R>(i - 1)] : zprev, s_z[pad<R>(i)], sc);
            thr[r] = t;
            hw = max(hw, theta_hw<Real>(t));
            if (track_ties && i < nvalid && (i > 0 || !first) && t == Real(0)) tie = true;
        }
        hw = __reduce_max_sync(0xffffffffu, hw);
        if (track_ties && __any_sync(0xffffffffu, tie) && lane == 0) atomicOr(a.ties, 1u);
    }
    Real thsp = 0;
    if (i0 < nvalid && (!first || i0 > 0))
        thsp = gap_real<Real>(i0 > 0 ? s_z[pad<R>(i0 - 1)] : zprev, s_z[pad<R>(min(i0 + R - 1, nvalid - 1))], sc);
    const uint32_t hsp = __reduce_max_sync(0xffffffffu, theta_hw<Real>(thsp));
    __syncthreads();
    if (!reuse) {
#pragma unroll
        for (int r = 0; r < R; ++r) s_th[pad<R>(i0 + r)] = thr[r];
    }
    uint32_t tmask = 0;
#pragma unroll
    for (int r = 0; r < R; ++r) tmask |= ((s_tgt[(i0 + r) >> 5] >> ((i0 + r) & 31)) & 1u) << r;
    // the tile's span multipliers (lanes of the last warp, one per term)
    if (tid >= T - NE && !first) {
        const int k = tid - (T - NE);
        double mr, mi;
        if constexpr (CO) {
            mr = zend == zprev ? 1.0 : 0.0;
            mi = 0.0;
        } else {
            cexp_neg(c.tau_re[k], c.tau_im[k], s * (zend - zprev), mr, mi);
        }
        s_M[k][0] = mr;
        s_M[k][1] = mi;
    }

    // Accumulators of phase C.  The value channel accumulates in registers on the table
    // path (FP64) and in the targets' strength slots otherwise; the derivative channel in
    // shared memory (over the coordinates / gaps, which the FP64 path no longer needs and
    // the FP32 path keeps in the first half of the region).
    Real acc[R];
#pragma unroll
    for (int r = 0; r < R; ++r) acc[r] = 0;
    Real* s_acc2 = sizeof(Real) == 8 ? reinterpret_cast<Real*>(s_z) : reinterpret_cast<Real*>(s_z) + SM::TP;
    // identical points on the FP32 path: every slot keeps its strength, so the value
    // channel accumulates over the second half of the coordinate region instead (free:
    // the gaps take the first half and the derivative channel is off in this mode)
    const bool self_acc = std::is_same<Real, float>::value && a.self != 0;
    if (self_acc) {
#pragma unroll
        for (int r = 0; r < R; ++r) s_acc2[pad<R>(i0 + r)] = Real(0);
    }
    Real* s_val = self_acc ? s_acc2 : s_al;  // where the value channel accumulates
    const uint32_t zmask = self_acc ? 0u : tmask;  // slots that hold no strength
    // strength of point r in phase A: a target slot holds a running value once an earlier
    // group's phase C has passed (recomputed-multiplier paths)
    auto strength = [&](int r) {
        if constexpr (!kF64) {
            if ((zmask >> r) & 1u) return Real(0);
        }
        return s_al[pad<R>(i0 + r)];
    };
    // the terms run in groups of NG (SweepGroup); one group unless the scan region of all
    // NE terms would not fit the occupancy target
    for (int g0 = 0; g0 < NE; g0 += NG) {
        const int g1 = min(NE, g0 + NG);
        if (g0 > 0) __syncthreads();  // the previous group's phase C has read s_scan
        // phase A: per term, thread aggregates and the warp scan
#pragma unroll 1
        for (int k = g0; k < g1; ++k) {
            Real fr = 0, fi = 0;
            Real Mr, Mi;
            if constexpr (CO) {
#pragma unroll 4
                for (int r = 0; r < R; ++r)
                    fr = (s_th[pad<R>(i0 + r)] == Real(0) ? fr : Real(0)) + s_al[pad<R>(i0 + r)];
                Mr = thsp == Real(0) ? Real(1) : Real(0);
                Mi = 0;
            } else {
                // this thread's R multipliers are slots r T + tid of the tile (interleaved table)
                double2* __restrict__ mt = kTab ? a.mult + (int64_t)k * a.Ppad + base + tid : nullptr;
                bool loaded = false;
                if constexpr (kTab) {
                    if (reuse) {
#pragma unroll 4
                        for (int r = 0; r < R; ++r) {
                            Real mr = Real(1), mi = Real(0);
                            if (i0 + r < nvalid) TableEntry<Real>::load(mt + r * T, mr, mi);
                            cfma_ra<Real>(mr, mi, fr, fi, strength(r), fr, fi);
                        }
                        loaded = true;
                    }
                }
                if (!loaded) {
                    const int deg = taylor_degree<Real>(c, k, hw);
                    const bool hyb = kF64 && hw <= c.theta_hyb_lim[k];
                    with_degree<Real>(deg, [&](auto Dc) {
#pragma unroll 4
                        for (int r = 0; r < R; ++r) {
                            Real mr, mi;
                            taylor<Real>(c, k, Dc, s_th[pad<R>(i0 + r)], mr, mi, hyb);
                            if constexpr (kTab) {
                                if (i0 + r < nvalid) TableEntry<Real>::store(mt + r * T, mr, mi);
                            }
                            cfma_ra<Real>(mr, mi, fr, fi, strength(r), fr, fi);
                        }
                    });
                }
                multiplier<Real>(c, k, hsp, thsp, Mr, Mi);
            }
            if constexpr (kF64) {
                // the thread's aggregate; the serial warp scan below combines them
                using SI = ScanIndex<NG, NW>;
                s_scan[SI::at(0, lane, k - g0, w)] = Mr;
                s_scan[SI::at(1, lane, k - g0, w)] = Mi;
                s_scan[SI::at(2, lane, k - g0, w)] = fr;
                s_scan[SI::at(3, lane, k - g0, w)] = fi;
            } else {
#pragma unroll
                for (int o = 1; o < 32; o <<= 1) {
                    Real Mor = shfl_up<Real>(Mr, o), Moi = shfl_up<Real>(Mi, o);
                    Real For = shfl_up<Real>(fr, o), Foi = shfl_up<Real>(fi, o);
                    if (lane >= o) {
                        cfma<Real>(Mr, Mi, For, Foi, fr, fi, fr, fi);
                        cmul<Real>(Mr, Mi, Mor, Moi, Mr, Mi);
                    }
                }
                Real Mxr = shfl_up<Real>(Mr, 1), Mxi = shfl_up<Real>(Mi, 1);
                Real Fxr = shfl_up<Real>(fr, 1), Fxi = shfl_up<Real>(fi, 1);
                if (lane == 0) { Mxr = Real(1); Mxi = Real(0); Fxr = Real(0); Fxi = Real(0); }
                Real* sc = s_scan + (size_t)(k - g0) * 4 * T;
                sc[tid] = Mxr; sc[T + tid] = Mxi; sc[2 * T + tid] = Fxr; sc[3 * T + tid] = Fxi;
                if (lane == 31) {
                    s_w[k][w][0] = real_to_f64<Real>(Mr); s_w[k][w][1] = real_to_f64<Real>(Mi);
                    s_w[k][w][2] = real_to_f64<Real>(fr); s_w[k][w][3] = real_to_f64<Real>(fi);
                }
            }
        }
        if constexpr (kF64) {
            __syncthreads();
            serial_warp_scan<NG, NW, true, NE>(reinterpret_cast<double*>(s_scan), s_w, g0, g1);
        }
        __syncthreads();
        // phase B: one lane per term joins the warps and the tiles
        for (int k = g0 + w; k < g1; k += NW)
            tile_combine<NE, NW>(a, a.fdesc, tile, itm.tile0, itm.tile0 + itm.ntiles, -1, first, !first ? s_M[k][0] : 1.0,
                                 !first ? s_M[k][1] : 0.0, s_w, s_win, k);
        __syncthreads();
        // phase C: apply the carries, final pass, evaluation at targets.  The derivative
        // accumulators go over the gaps, which phase A has finished with (one group)
        if constexpr ((EV & 2) != 0) {
#pragma unroll
            for (int r = 0; r < R; ++r) s_acc2[pad<R>(i0 + r)] = 0;
        }
#pragma unroll 1
        for (int k = g0; k < g1; ++k) {
            const Real* sc = s_scan + (size_t)(k - g0) * 4 * T;
            Real fr, fi;
            if constexpr (kF64) {
                using SI = ScanIndex<NG, NW>;
                cfma<Real>(s_scan[SI::at(0, lane, k - g0, w)], s_scan[SI::at(1, lane, k - g0, w)], s_win[k][w][0],
                           s_win[k][w][1], s_scan[SI::at(2, lane, k - g0, w)], s_scan[SI::at(3, lane, k - g0, w)], fr,
                           fi);
            } else {
                cfma<Real>(sc[tid], sc[T + tid], to_real<Real>(s_win[k][w][0]), to_real<Real>(s_win[k][w][1]),
                           sc[2 * T + tid], sc[3 * T + tid], fr, fi);
            }
            const Real Wr = TermConsts<Real>::w_re(c, k), Wi = TermConsts<Real>::w_im(c, k);
            const Real Vr = TermConsts<Real>::v_re(c, k), Vi = TermConsts<Real>::v_im(c, k);
            auto eval = [&](int r) {
                if ((tmask >> r) & 1u) {
                    if constexpr (CO) {
                        acc[r] += fr;
                    } else {
                        if constexpr ((EV & 1) != 0) acc[r] = fma(Wr, fr, fma(-Wi, fi, acc[r]));
                        if constexpr ((EV & 2) != 0)
                            s_acc2[pad<R>(i0 + r)] = fma(Vr, fr, fma(-Vi, fi, s_acc2[pad<R>(i0 + r)]));
                    }
                }
            };
            if constexpr (CO) {
#pragma unroll
                for (int r = 0; r < R; ++r) {
                    fr = (s_th[pad<R>(i0 + r)] == Real(0) ? fr : Real(0)) + s_al[pad<R>(i0 + r)];
                    eval(r);
                }
            } else if constexpr (kF64) {
                const double2* __restrict__ mt = a.mult + (int64_t)k * a.Ppad + base + tid;
#pragma unroll
                for (int r = 0; r < R; ++r) {
                    const double2 m = i0 + r < nvalid ? mt[r * T] : make_double2(1.0, 0.0);
                    cfma_ra<Real>(m.x, m.y, fr, fi, s_al[pad<R>(i0 + r)], fr, fi);
                    eval(r);
                }
            } else if constexpr (kTab) {
                // double-float: multipliers from the table; the value channel accumulates in
                // the targets' own (zero) strength slots
                const double2* __restrict__ mt = a.mult + (int64_t)k * a.Ppad + base + tid;
#pragma unroll kUnrollC
                for (int r = 0; r < R; ++r) {
                    Real mr = Real(1), mi = Real(0);
                    if (i0 + r < nvalid) TableEntry<Real>::load(mt + r * T, mr, mi);
                    const bool tg = (tmask >> r) & 1u;
                    Real* slot = &s_al[pad<R>(i0 + r)];
                    const Real v = *slot;
                    cfma_ra<Real>(mr, mi, fr, fi, tg ? Real(0) : v, fr, fi);
                    if (tg) *slot = fma(Wr, fr, fma(-Wi, fi, v));
                }
            } else {
                // recomputed multipliers: the value channel accumulates in the targets' own
                // (zero) strength slots, so the loop needs no register array and is only
                // partly unrolled (smaller code per Taylor degree)
                // (identical points: every slot keeps its strength and the values go to
                // s_acc2; a compile-time variant, so the usual loop is unchanged)
                auto run_c = [&](auto Self) {
                    constexpr bool kSelf = decltype(Self)::value;
                    with_degree<Real>(taylor_degree<Real>(c, k, hw), [&](auto Dc) {
#pragma unroll kUnrollC
                        for (int r = 0; r < R; ++r) {
                            Real mr, mi;
                            taylor<Real>(c, k, Dc, s_th[pad<R>(i0 + r)], mr, mi);
                            const bool tg = (tmask >> r) & 1u;
                            Real* slot = &s_al[pad<R>(i0 + r)];
                            const Real v = *slot;  // strength at a source, running value at a target
                            cfma_ra<Real>(mr, mi, fr, fi, tg && !kSelf ? Real(0) : v, fr, fi);
                            if (tg) {
                                if constexpr ((EV & 1) != 0) {
                                    if constexpr (kSelf) {
                                        Real* vs = &s_acc2[pad<R>(i0 + r)];
                                        *vs = fma(Wr, fr, fma(-Wi, fi, *vs));
                                    } else {
                                        *slot = fma(Wr, fr, fma(-Wi, fi, v));
                                    }
                                }
                                if constexpr ((EV & 2) != 0)
                                    s_acc2[pad<R>(i0 + r)] = fma(Vr, fr, fma(-Vi, fi, s_acc2[pad<R>(i0 + r)]));
                            }
                        }
                    });
                };
                if constexpr (std::is_same<Real, float>::value) {
                    if (self_acc) run_c(std::true_type{});
                    else run_c(std::false_type{});
                } else {
                    run_c(std::false_type{});
                }
            }
        }
    }
    // outputs, written coalesced through shared memory (values staged over s_al)
    __syncthreads();
    if constexpr (kF64 || CO) {
#pragma unroll
        for (int r = 0; r < R; ++r) s_al[pad<R>(i0 + r)] = acc[r];
        __syncthreads();
    }
    if constexpr (CO) {
        // per target in target order; with identical points, per point in sorted order
        for (int i = tid; i < nvalid; i += T)
            if ((s_tgt[i >> 5] >> (i & 31)) & 1u)
                a.u[a.self ? base + i : (int64_t)vals[base + i] - a.N] = real_to_f64<Real>(s_al[pad<R>(i)]);
    } else {
        for (int i = tid; i < nvalid; i += T) {
            if constexpr ((EV & 1) != 0) static_cast<Real*>(a.fwd)[base + i] = s_val[pad<R>(i)];
            if constexpr ((EV & 2) != 0) static_cast<Real*>(a.fwd2)[base + i] = s_acc2[pad<R>(i)];
        }
    }
    if constexpr (T >= 256) return;  // one tile per CTA (the launch gives every tile a CTA)
    __syncthreads();  // the next tile's staging overwrites the shared arrays
    }
}

template <typename Real, int NE, int T, int R, int EV>
__global__ void __launch_bounds__(T, SweepMinBlocks<Real>::value) k_sweep_bwd(const SweepArgs a, const SweepConsts c) {
    constexpr int NG = SweepGroup<Real, NE, T, R, EV, false>::NG;
    using SM = SweepSmem<Real, NG, T, R>;
    constexpr int TILE = T * R;
    constexpr int NW = T / 32;
    constexpr bool kF64 = std::is_same<Real, double>::value;
    // multipliers reloaded from the forward sweep's table (FP64 and double-float)
    constexpr bool kTab = kF64 || std::is_same<Real, dfloat>::value;
    constexpr int kUnrollC = sizeof(Real) == 8 ? 4 : 8;       // phase C unroll, recomputed multipliers
    static_assert(!((EV & 2) && std::is_same<Real, dfloat>::value), "no derivative channel in double-float");
    static_assert((EV & 2) == 0 || NG == NE, "the derivative channel runs its terms as one group");
    extern __shared__ __align__(16) unsigned char smem[];
    double* s_z = reinterpret_cast<double*>(smem + SM::z_off);
    Real* s_th = reinterpret_cast<Real*>(smem + SM::z_off);  // gap between points i and i+1, over s_z
    Real* s_al = reinterpret_cast<Real*>(smem + SM::al_off);
    Real* s_scan = reinterpret_cast<Real*>(smem + SM::scan_off);
    __shared__ double s_w[NE][NW][4];
    __shared__ double s_win[NE][NW][2];
    __shared__ double s_M[NE][2];
    __shared__ uint32_t s_tgt[TILE / 32];

    static_assert(TILE == kTile, "a sweep tile is one item tile");
    __shared__ int s_item;
    __shared__ int64_t s_tilev;
    const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
    // persistent: each CTA takes tiles in reverse order from the counter until none is left
    for (;;) {
    if (tid == 0) {
        const int64_t T_tot = *a.total_tiles;
        const int64_t acq = atomicAdd(&a.tile_ctr[1], 1u);
        s_tilev = T_tot - 1 - acq;
        s_item = acq < T_tot ? item_of_tile(a.items, a.B, s_tilev) : -1;
        if (ld_volatile_u32(a.status) & kStatusSortTimeout) s_item = -1;  // sorted codes not valid
    }
    __syncthreads();
    if (s_item < 0) return;
    const Item itm = a.items[s_item];
    const int64_t tile = s_tilev;
    const int64_t base = tile * TILE;
    const int64_t local = base - itm.start;
    const int64_t preal = itm.nsrc + itm.ntgt;  // real points of the item
    const int nvalid = (int)min((int64_t)TILE, preal - local);
    const bool has_next = local + TILE < preal;
    const double s = itm.s;
    const Scale sc = make_scale<Real>(s);
    const bool bufB = a.plan->final_buf == 1;
    const uint64_t* __restrict__ keys = bufB ? a.keysB : a.keysA;
    const uint32_t* __restrict__ vals = bufB ? a.valsB : a.valsA;
    // the next tile's first coordinate, loaded before the staging so that both overlap
    const uint64_t knext = (tid == 0 && has_next) ? keys[base + TILE] : 0ull;
    stage_tile<Real, T, R>(a, keys, vals, base, nvalid, s_z, s_al, s_tgt);
    if (tid == 0) s_z[pad<R>(TILE)] = has_next ? key_coord(knext) : 0.0;
    __syncthreads();

    const int i0 = tid * R;
    const double znext = s_z[pad<R>(TILE)], zfirst = s_z[0];
    uint32_t hw = 0;
    Real thr[R];
    if constexpr (!kTab) {
#pragma unroll
        for (int r = 0; r < R; ++r) {
            const int i = i0 + r;
            Real t = 0;
            if (i + 1 < nvalid || (i + 1 == TILE && has_next))
                t = gap_real<Real>(s_z[pad<R>(i)], s_z[pad<R>(i + 1)], sc);
            thr[r] = t;
            hw = max(hw, theta_hw<Real>(t));
        }
        hw = __reduce_max_sync(0xffffffffu, hw);
    }
    Real thsp = 0;
    {
        const int inext = i0 + R;
        if (i0 < nvalid && (inext < nvalid || (inext == TILE && has_next)))
            thsp = gap_real<Real>(s_z[pad<R>(i0)], s_z[pad<R>(inext)], sc);
    }
    const uint32_t hsp = __reduce_max_sync(0xffffffffu, theta_hw<Real>(thsp));
    __syncthreads();
    if constexpr (!kTab) {
#pragma unroll
        for (int r = 0; r < R; ++r) s_th[pad<R>(i0 + r)] = thr[r];
    }
    uint32_t tmask = 0;
#pragma unroll
    for (int r = 0; r < R; ++r) tmask |= ((s_tgt[(i0 + r) >> 5] >> ((i0 + r) & 31)) & 1u) << r;
    if (tid >= T - NE && has_next) {
        const int k = tid - (T - NE);
        double mr, mi;
        cexp_neg(c.tau_re[k], c.tau_im[k], s * (znext - zfirst), mr, mi);
        s_M[k][0] = mr;
        s_M[k][1] = mi;
    }

    // multiplier between points i0+r and i0+r+1 (stored table, or a Taylor polynomial
    // of compile-time degree D on the FP32 path)
    // this thread's slots in the interleaved table start at base + tid; the multiplier of
    // point i0 + r + 1 is at offset (r + 1) T, or for r = R - 1 at the next thread's first
    // slot (+1), which for the last thread is the next tile's slot 0
    const int64_t next_off = tid + 1 < T ? 1 : (int64_t)TILE - tid;
    auto mult_at = [&](int k, auto Dc, int r, Real& mr, Real& mi) {
        if constexpr (kTab) {
            const double2* mt = a.mult + (int64_t)k * a.Ppad + base + tid;
            mr = Real(0);
            mi = Real(0);
            if (local + i0 + r + 1 < preal)
                TableEntry<Real>::load(mt + (r + 1 < R ? (int64_t)(r + 1) * T : next_off), mr, mi);
        } else {
            taylor<Real>(c, k, Dc, s_th[pad<R>(i0 + r)], mr, mi);
        }
    };

    Real acc[R];
#pragma unroll
    for (int r = 0; r < R; ++r) acc[r] = 0;
    Real* s_acc2 = sizeof(Real) == 8 ? reinterpret_cast<Real*>(s_z) : reinterpret_cast<Real*>(s_z) + SM::TP;
    // identical points on the FP32 path: every slot keeps its strength, so the value
    // channel accumulates over the second half of the coordinate region instead (free:
    // the gaps take the first half and the derivative channel is off in this mode)
    const bool self_acc = std::is_same<Real, float>::value && a.self != 0;
    if (self_acc) {
#pragma unroll
        for (int r = 0; r < R; ++r) s_acc2[pad<R>(i0 + r)] = Real(0);
    }
    Real* s_val = self_acc ? s_acc2 : s_al;  // where the value channel accumulates
    const uint32_t zmask = self_acc ? 0u : tmask;  // slots that hold no strength
    // strength of point r in phase A: a target slot holds a running value once an earlier
    // group's phase C has passed (recomputed-multiplier paths)
    auto strength = [&](int r) {
        if constexpr (!kF64) {
            if ((zmask >> r) & 1u) return Real(0);
        }
        return s_al[pad<R>(i0 + r)];
    };
    // the terms run in groups of NG (SweepGroup), as in the forward sweep
    for (int g0 = 0; g0 < NE; g0 += NG) {
        const int g1 = min(NE, g0 + NG);
        if (g0 > 0) __syncthreads();  // the previous group's phase C has read s_scan
#pragma unroll 1
        for (int k = g0; k < g1; ++k) {
            const int deg = kTab ? 0 : taylor_degree<Real>(c, k, hw);
            Real br = 0, bi = 0;
            with_degree<Real>(deg, [&](auto Dc) {
#pragma unroll 4
                for (int r = R - 1; r >= 0; --r) {
                    Real mr, mi;
                    mult_at(k, Dc, r, mr, mi);
                    // b_r = m_{r+1} b_{r+1} + alpha_r, with b_R (the next thread's state) = 0
                    cfma_ra<Real>(mr, mi, br, bi, strength(r), br, bi);
                }
            });
            Real Mr, Mi;
            multiplier<Real>(c, k, hsp, thsp, Mr, Mi);
            if constexpr (kF64) {
                // the thread's aggregate; the serial warp scan below combines them
                using SI = ScanIndex<NG, NW>;
                s_scan[SI::at(0, lane, k - g0, w)] = Mr;
                s_scan[SI::at(1, lane, k - g0, w)] = Mi;
                s_scan[SI::at(2, lane, k - g0, w)] = br;
                s_scan[SI::at(3, lane, k - g0, w)] = bi;
            } else {
#pragma unroll
                for (int o = 1; o < 32; o <<= 1) {
                    Real Mor = shfl_down<Real>(Mr, o), Moi = shfl_down<Real>(Mi, o);
                    Real For = shfl_down<Real>(br, o), Foi = shfl_down<Real>(bi, o);
                    if (lane + o < 32) {
                        cfma<Real>(Mr, Mi, For, Foi, br, bi, br, bi);
                        cmul<Real>(Mr, Mi, Mor, Moi, Mr, Mi);
                    }
                }
                Real Mxr = shfl_down<Real>(Mr, 1), Mxi = shfl_down<Real>(Mi, 1);
                Real Fxr = shfl_down<Real>(br, 1), Fxi = shfl_down<Real>(bi, 1);
                if (lane == 31) { Mxr = Real(1); Mxi = Real(0); Fxr = Real(0); Fxi = Real(0); }
                Real* sc = s_scan + (size_t)(k - g0) * 4 * T;
                sc[tid] = Mxr; sc[T + tid] = Mxi; sc[2 * T + tid] = Fxr; sc[3 * T + tid] = Fxi;
                if (lane == 0) {
                    s_w[k][w][0] = real_to_f64<Real>(Mr); s_w[k][w][1] = real_to_f64<Real>(Mi);
                    s_w[k][w][2] = real_to_f64<Real>(br); s_w[k][w][3] = real_to_f64<Real>(bi);
                }
            }
        }
        if constexpr (kF64) {
            __syncthreads();
            serial_warp_scan<NG, NW, false, NE>(reinterpret_cast<double*>(s_scan), s_w, g0, g1);
        }
        __syncthreads();
        for (int k = g0 + w; k < g1; k += NW)
            tile_combine<NE, NW>(a, a.bdesc, tile, itm.tile0, itm.tile0 + itm.ntiles, +1, !has_next,
                                 has_next ? s_M[k][0] : 1.0, has_next ? s_M[k][1] : 0.0, s_w, s_win, k);
        __syncthreads();
        if constexpr ((EV & 2) != 0) {  // derivative accumulators (one group)
#pragma unroll
            for (int r = 0; r < R; ++r) s_acc2[pad<R>(i0 + r)] = 0;
        }
#pragma unroll 1
        for (int k = g0; k < g1; ++k) {
            const Real* sc = s_scan + (size_t)(k - g0) * 4 * T;
            Real br, bi;  // state at the first point of the next thread
            if constexpr (kF64) {
                using SI = ScanIndex<NG, NW>;
                cfma<Real>(s_scan[SI::at(0, lane, k - g0, w)], s_scan[SI::at(1, lane, k - g0, w)], s_win[k][w][0],
                           s_win[k][w][1], s_scan[SI::at(2, lane, k - g0, w)], s_scan[SI::at(3, lane, k - g0, w)], br,
                           bi);
            } else {
                cfma<Real>(sc[tid], sc[T + tid], to_real<Real>(s_win[k][w][0]), to_real<Real>(s_win[k][w][1]),
                           sc[2 * T + tid], sc[3 * T + tid], br, bi);
            }
            const Real Wr = TermConsts<Real>::w_re(c, k), Wi = TermConsts<Real>::w_im(c, k);
            const Real Vr = TermConsts<Real>::v_re(c, k), Vi = TermConsts<Real>::v_im(c, k);
            const int deg = kTab ? 0 : taylor_degree<Real>(c, k, hw);
            with_degree<Real>(deg, [&](auto Dc) {
                if constexpr (kF64) {
#pragma unroll
                    for (int r = R - 1; r >= 0; --r) {
                        Real mr, mi;
                        mult_at(k, Dc, r, mr, mi);
                        cfma_ra<Real>(mr, mi, br, bi, s_al[pad<R>(i0 + r)], br, bi);
                        if ((tmask >> r) & 1u) {
                            if constexpr ((EV & 1) != 0) acc[r] = fma(Wr, br, fma(-Wi, bi, acc[r]));
                            if constexpr ((EV & 2) != 0)
                                s_acc2[pad<R>(i0 + r)] = fma(-Vr, br, fma(Vi, bi, s_acc2[pad<R>(i0 + r)]));
                        }
                    }
                } else {
                    // as in the forward sweep: values accumulate in the targets' strength
                    // slots, or in s_acc2 with identical points (FP32)
                    auto run_c = [&](auto Self) {
                        constexpr bool kSelf = decltype(Self)::value;
#pragma unroll kUnrollC
                        for (int r = R - 1; r >= 0; --r) {
                            Real mr, mi;
                            mult_at(k, Dc, r, mr, mi);
                            const bool tg = (tmask >> r) & 1u;
                            Real* slot = &s_al[pad<R>(i0 + r)];
                            const Real v = *slot;
                            cfma_ra<Real>(mr, mi, br, bi, tg && !kSelf ? Real(0) : v, br, bi);
                            if (tg) {
                                if constexpr ((EV & 1) != 0) {
                                    if constexpr (kSelf) {
                                        Real* vs = &s_acc2[pad<R>(i0 + r)];
                                        *vs = fma(Wr, br, fma(-Wi, bi, *vs));
                                    } else {
                                        *slot = fma(Wr, br, fma(-Wi, bi, v));
                                    }
                                }
                                if constexpr ((EV & 2) != 0)
                                    s_acc2[pad<R>(i0 + r)] = fma(-Vr, br, fma(Vi, bi, s_acc2[pad<R>(i0 + r)]));
                            }
                        }
                    };
                    if constexpr (std::is_same<Real, float>::value) {
                        if (self_acc) run_c(std::true_type{});
                        else run_c(std::false_type{});
                    } else {
                        run_c(std::false_type{});
                    }
                }
            });
        }
    }
    __syncthreads();
    if constexpr (kF64) {
#pragma unroll
        for (int r = 0; r < R; ++r) s_al[pad<R>(i0 + r)] = acc[r];
        __syncthreads();
    }
    // identical targets and sources: the backward state includes the point's own
    // strength, which the forward state already holds (eq. 4.4: the source at x_i belongs
    // to h+); it is taken out once, Re sum_k W_k alpha_i = S_n(0) alpha_i
    double s0 = 0.0;
    if (a.self) {
#pragma unroll
        for (int k = 0; k < NE; ++k) s0 += c.w_re[k];
    }
    for (int i = tid; i < nvalid; i += T) {
        if ((s_tgt[i >> 5] >> (i & 31)) & 1u) {
            const int64_t p = base + i;
            const uint32_t v = vals[p];
            const int64_t t = (int64_t)v - (a.self ? 0 : a.N);
            if constexpr ((EV & 1) != 0) {
                double ui = real_to_f64<Real>(static_cast<const Real*>(a.fwd)[p] + s_val[pad<R>(i)]);
                if (a.self) ui -= s0 * __ldg(&a.alpha[v]);
                a.u[t] = ui;
            }
            if constexpr ((EV & 2) != 0)
                a.out2[t] = s * real_to_f64<Real>(static_cast<const Real*>(a.fwd2)[p] + s_acc2[pad<R>(i)]);
        }
    }
    if constexpr (T >= 256) return;  // one tile per CTA (the launch gives every tile a CTA)
    __syncthreads();  // the next tile's staging overwrites the shared arrays
    }
}

// The multiplier table of a bound geometry (entries of Real: FP64, or double-float
// rounded from the FP64 value): exp(-tau_k s (z_p - z_{p-1})) for
// every real point p of every item (1 at an item's first point), the values the forward
// sweep would store, at the interleaved slot (i % sR) sT + i / sR of tile point i for
// the sweeps' tile shape sT x sR.  One block per
// 4096-point tile; thread t fills slots t, t + T, ... (coalesced stores).
template <int T, typename Real>
__global__ void __launch_bounds__(T) k_fill_table(const SweepArgs a, const SweepConsts c, int sT, int sR) {
    __shared__ int s_item;
    const int tid = threadIdx.x;
    const int64_t tile = blockIdx.x;
    if (tid == 0) s_item = tile < *a.total_tiles ? item_of_tile(a.items, a.B, tile) : -1;
    __syncthreads();
    if (s_item < 0) return;
    const Item itm = a.items[s_item];
    const int64_t base = tile * kTile, local = base - itm.start;
    const int nvalid = (int)min((int64_t)kTile, itm.nsrc + itm.ntgt - local);
    const uint64_t* __restrict__ keys = a.plan->final_buf == 1 ? a.keysB : a.keysA;
    const double s = itm.s;
    for (int j0 = 0; j0 < kTile; j0 += T) {
        const int j = j0 + tid;             // table slot
        const int i = (j % sT) * sR + j / sT;  // its point in the tile
        double th = 0.0;
        if (i < nvalid && (i > 0 || local > 0))
            th = s * (key_coord(keys[base + i]) - key_coord(keys[base + i - 1]));
        const uint32_t hw = __reduce_max_sync(0xffffffffu, theta_hw<double>(th));
        for (int k = 0; k < c.n_e; ++k) {
            double mr, mi;
            const bool hyb = hw <= c.theta_hyb_lim[k];
            with_degree<double>(taylor_degree<double>(c, k, hw),
                                [&](auto Dc) { taylor<double>(c, k, Dc, th, mr, mi, hyb); });
            if (i < nvalid)
                TableEntry<Real>::store(a.mult + (int64_t)k * a.Ppad + base + j, to_real<Real>(mr), to_real<Real>(mi));
        }
    }
}

}  // namespace fgt1d
