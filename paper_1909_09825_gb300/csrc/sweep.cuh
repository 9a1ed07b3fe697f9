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
// A CTA owns a tile of T*R consecutive points; each thread runs R points sequentially
// (work-efficient), a warp shuffle scan and a per-CTA combine join the threads, and a
// decoupled look-back joins the tiles: each (tile, term) publishes its aggregate and
// then its inclusive value, and a tile's carry is assembled from predecessors with
// span multipliers exp(-tau s (z_a - z_b)) computed directly from the FP64 anchor
// coordinates rather than as products, so no multiplier chain grows with the number
// of tiles.  Terms are processed one at a time so that only one term's R multipliers
// sit in registers.  Per-point multipliers use a Taylor polynomial of warp-uniform
// degree chosen from the warp's largest gap (integer compares on the high word of
// theta), falling back to exp/sincos for large gaps.
//
// FP64 path (Real = double): every step in FP64; the forward kernel stores the
// multipliers (16 B per point and term) so the backward kernel does not recompute
// them: on GB300 a DFMA costs 1/62 of an FFMA while a 32 B store+load is cheaper
// than the eight or more DFMAs it replaces.
// FP32 path (Real = float): multipliers and in-tile recurrences in FP32 complex from
// FP64 coordinate differences; tile aggregates, carries and anchor multipliers in FP64.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

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

__device__ __forceinline__ uint32_t hi_word(double v) {
    return (uint32_t)((uint64_t)__double_as_longlong(v) >> 32);
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

// exp(-tau theta) for any theta >= 0 (FP64), the anchor / span multiplier.
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
};
template <>
struct TermConsts<float> {
    __device__ static __forceinline__ float tc_re(const SweepConsts& c, int k, int j) { return c.tcf_re[k][j]; }
    __device__ static __forceinline__ float tc_im(const SweepConsts& c, int k, int j) { return c.tcf_im[k][j]; }
    __device__ static __forceinline__ float tau_re(const SweepConsts& c, int k) { return c.tauf_re[k]; }
    __device__ static __forceinline__ float tau_im(const SweepConsts& c, int k) { return c.tauf_im[k]; }
    __device__ static __forceinline__ uint32_t lim(const SweepConsts& c, int k, int d) { return c.theta_hi_lim_f[k][d]; }
};

// Taylor degree for term k that covers every theta whose high word is <= hw.
template <typename Real>
__device__ __forceinline__ int taylor_degree(const SweepConsts& c, int k, uint32_t hw) {
    int deg = kTaylorMax;
#pragma unroll
    for (int d = kTaylorMax - 1; d >= 0; --d)
        if (hw <= TermConsts<Real>::lim(c, k, d)) deg = d;
    return deg;
}

// exp(-tau_k theta) by a Taylor polynomial of (warp-uniform) degree deg, or by
// exp/sincos when theta is beyond the largest Taylor threshold.
template <typename Real>
__device__ __forceinline__ void multiplier(const SweepConsts& c, int k, int deg, Real th, uint32_t th_hw, Real& mr,
                                           Real& mi) {
    Real ar = 0, ai = 0;
#pragma unroll
    for (int j = kTaylorMax; j >= 1; --j) {
        if (j == deg) {
            ar = TermConsts<Real>::tc_re(c, k, j);
            ai = TermConsts<Real>::tc_im(c, k, j);
        } else if (j < deg) {
            ar = fma(ar, th, TermConsts<Real>::tc_re(c, k, j));
            ai = fma(ai, th, TermConsts<Real>::tc_im(c, k, j));
        }
    }
    if (deg >= 1) {
        mr = fma(ar, th, Real(1));
        mi = ai * th;
    } else {
        mr = Real(1);
        mi = Real(0);
    }
    if (th_hw > TermConsts<Real>::lim(c, k, kTaylorMax)) {
        cexp_neg(TermConsts<Real>::tau_re(c, k), TermConsts<Real>::tau_im(c, k), th, mr, mi);
    }
}

template <typename Real>
__device__ __forceinline__ uint32_t theta_hw(Real th);
template <>
__device__ __forceinline__ uint32_t theta_hw<double>(double th) { return hi_word(th); }
template <>
__device__ __forceinline__ uint32_t theta_hw<float>(float th) { return (uint32_t)__float_as_uint(th); }

__device__ __forceinline__ void publish_agg(TileDesc* d, double ar, double ai, double z) {
    d->agg_re = ar;
    d->agg_im = ai;
    d->z = z;
    __threadfence();
    st_volatile_u32(&d->flag, 1u);
}
__device__ __forceinline__ void publish_inc(TileDesc* d, double ar, double ai, double ir, double ii, double z,
                                            bool with_agg) {
    if (with_agg) {
        d->agg_re = ar;
        d->agg_im = ai;
        d->z = z;
    }
    d->inc_re = ir;
    d->inc_im = ii;
    __threadfence();
    st_volatile_u32(&d->flag, 2u);
}

// Decoupled look-back over the tiles tile+step, tile+2 step, ... (step = -1 forward,
// +1 backward) for term k: returns the carry at coordinate zref,
//     C = sum_j exp(-tau_k s |zref - z_j|) value_j,
// stopping at the first tile whose inclusive value is published.
static __device__ __noinline__ void look_back(const TileDesc* desc, int64_t tile, int step, int64_t tiles, int ne, int k,
                                       double tr, double ti, double s, double zref, double& cr, double& ci,
                                       uint32_t* status) {
    cr = 0.0;
    ci = 0.0;
    int64_t j = tile + step;
    while (j >= 0 && j < tiles) {
        const TileDesc* d = desc + j * ne + k;
        uint32_t f = ld_volatile_u32(&d->flag);
        if (f == 0) {
            long long t0 = clock64();
            while ((f = ld_volatile_u32(&d->flag)) == 0) {
                if (clock64() - t0 > kSpinLimitCycles) {
                    atomicOr(status, kStatusTimeout);
                    return;
                }
            }
        }
        __threadfence();
        double zj = __ldcg(&d->z);
        double er, ei;
        cexp_neg(tr, ti, s * fabs(zref - zj), er, ei);
        double vr = f == 2 ? __ldcg(&d->inc_re) : __ldcg(&d->agg_re);
        double vi = f == 2 ? __ldcg(&d->inc_im) : __ldcg(&d->agg_im);
        cfma(er, ei, vr, vi, cr, ci, cr, ci);
        if (f == 2) return;
        j += step;
    }
}

// Shared-memory footprint of the sweep kernels: coordinates (double), strengths (Real)
// and the per-term exclusive thread prefixes (Real), padded one slot per R points so
// that a warp reading one point per thread (stride R) hits distinct banks.
template <typename Real, int NE, int T, int R>
struct SweepSmem {
    static constexpr int TILE = T * R;
    static constexpr int TP = TILE + TILE / R + 1;
    static constexpr size_t z_off = 0;
    static constexpr size_t al_off = z_off + sizeof(double) * TP;
    static constexpr size_t scan_off = (al_off + sizeof(Real) * TP + 15) / 16 * 16;
    static constexpr size_t bytes = scan_off + sizeof(Real) * 4 * NE * T;
};

template <int R>
__device__ __forceinline__ int pad(int i) { return i + i / R; }

// Per-term combine of the warp totals, look-back and publication (one lane per term).
// dir = -1: forward (anchor = last point, carry comes from lower tiles);
// dir = +1: backward (anchor = first point, carry comes from higher tiles).
// s_w[k][w] holds each warp's total map (M, F) in the sweep direction; on return
// s_win[k][w] holds the state entering warp w (after the carry).
template <int NE, int NW>
__device__ __forceinline__ void tile_combine(const SweepArgs& a, const SweepConsts& c, TileDesc* desc, int64_t tile,
                                             int dir, bool first_in_dir, double zanchor, double zref,
                                             double (*s_w)[NW][4], double (*s_win)[NW][2], int k) {
    double pre[NW][4];
    double Pr = 1, Pi = 0, Qr = 0, Qi = 0;
#pragma unroll
    for (int q = 0; q < NW; ++q) {
        const int ww = dir < 0 ? q : NW - 1 - q;  // sweep order
        pre[ww][0] = Pr; pre[ww][1] = Pi; pre[ww][2] = Qr; pre[ww][3] = Qi;
        cfma<double>(s_w[k][ww][0], s_w[k][ww][1], Qr, Qi, s_w[k][ww][2], s_w[k][ww][3], Qr, Qi);
        cmul<double>(s_w[k][ww][0], s_w[k][ww][1], Pr, Pi, Pr, Pi);
    }
    TileDesc* dd = desc + tile * NE + k;
    double Cr = 0, Ci = 0;
    const double tr = c.tau_re[k], ti = c.tau_im[k], s = c.s;
    if (first_in_dir) {
        publish_inc(dd, Qr, Qi, Qr, Qi, zanchor, true);
    } else {
        publish_agg(dd, Qr, Qi, zanchor);
        look_back(desc, tile, dir, a.tiles, NE, k, tr, ti, s, zref, Cr, Ci, a.status);
        double Er, Ei;
        cexp_neg(tr, ti, s * fabs(zanchor - zref), Er, Ei);
        double Ir, Ii;
        cfma<double>(Er, Ei, Cr, Ci, Qr, Qi, Ir, Ii);
        publish_inc(dd, 0, 0, Ir, Ii, zanchor, false);
    }
#pragma unroll
    for (int ww = 0; ww < NW; ++ww) {
        double xr, xi;
        cfma<double>(pre[ww][0], pre[ww][1], Cr, Ci, pre[ww][2], pre[ww][3], xr, xi);
        s_win[k][ww][0] = xr;
        s_win[k][ww][1] = xi;
    }
}

// Stages the tile: coordinates, strengths (0 at targets) and target bits.  Points past
// the end get z = 0, alpha = 0 and are not targets; n_extra points after the tile
// (the next tile's first point for the backward sweep) are loaded as coordinates only.
template <typename Real, int T, int R>
__device__ __forceinline__ void stage_tile(const SweepArgs& a, const uint64_t* __restrict__ keys,
                                           const uint32_t* __restrict__ vals, int64_t base, int nvalid,
                                           double* s_z, Real* s_al, uint32_t* s_tgt) {
    constexpr int TILE = T * R;
    const int tid = threadIdx.x, lane = tid & 31;
    for (int i = tid; i < TILE; i += T) {
        double z = 0.0, al = 0.0;
        bool tg = false;
        if (i < nvalid) {
            const int64_t p = base + i;
            z = key_coord(keys[p]);
            const uint32_t v = vals[p];
            if ((int64_t)v < a.N) al = __ldg(&a.alpha[v]);
            else tg = true;
        }
        s_z[pad<R>(i)] = z;
        s_al[pad<R>(i)] = (Real)al;
        const unsigned b = __ballot_sync(0xffffffffu, tg);
        if (lane == 0) s_tgt[i >> 5] = b;
    }
}

template <typename Real, int NE, int T, int R>
__global__ void __launch_bounds__(T) k_sweep_fwd(const SweepArgs a, const SweepConsts c) {
    using SM = SweepSmem<Real, NE, T, R>;
    constexpr int TILE = T * R;
    constexpr int NW = T / 32;
    constexpr bool kF64 = sizeof(Real) == 8;
    extern __shared__ __align__(16) unsigned char smem[];
    double* s_z = reinterpret_cast<double*>(smem + SM::z_off);
    Real* s_al = reinterpret_cast<Real*>(smem + SM::al_off);
    Real* s_scan = reinterpret_cast<Real*>(smem + SM::scan_off);  // [NE][4][T]
    __shared__ double s_w[NE][NW][4];
    __shared__ double s_win[NE][NW][2];
    __shared__ uint32_t s_tgt[TILE / 32];
    __shared__ uint32_t s_tile;
    __shared__ double s_zprev;

    const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
    if (tid == 0) s_tile = atomicAdd(&a.tile_ctr[0], 1u);
    __syncthreads();
    const int64_t tile = s_tile;
    const int64_t base = tile * TILE;
    const int nvalid = (int)min((int64_t)TILE, a.P - base);
    const bool bufB = a.plan->final_buf == 1;
    const uint64_t* __restrict__ keys = bufB ? a.keysB : a.keysA;
    const uint32_t* __restrict__ vals = bufB ? a.valsB : a.valsA;
    stage_tile<Real, T, R>(a, keys, vals, base, nvalid, s_z, s_al, s_tgt);
    if (tid == 0) s_zprev = base > 0 ? key_coord(keys[base - 1]) : 0.0;
    __syncthreads();

    // my R points: gaps theta = s (z_i - z_{i-1}) (FP64 difference), target bits
    const double s = c.s;
    const int i0 = tid * R;
    const double zprev = s_zprev;
    Real th[R];
    uint32_t thw[R];
    uint32_t hw = 0;
#pragma unroll
    for (int r = 0; r < R; ++r) {
        const int i = i0 + r;
        double t = 0.0;
        if (i < nvalid && base + i > 0) t = s * (s_z[pad<R>(i)] - (i > 0 ? s_z[pad<R>(i - 1)] : zprev));
        th[r] = (Real)t;
        thw[r] = theta_hw<Real>(th[r]);
        hw = max(hw, thw[r]);
    }
    hw = __reduce_max_sync(0xffffffffu, hw);
    double th_span = 0.0;
    if (i0 < nvalid && (base > 0 || i0 > 0))
        th_span = s * (s_z[pad<R>(min(i0 + R - 1, nvalid - 1))] - (i0 > 0 ? s_z[pad<R>(i0 - 1)] : zprev));
    const Real thsp = (Real)th_span;
    const uint32_t thsp_w = theta_hw<Real>(thsp);
    const uint32_t hsp = __reduce_max_sync(0xffffffffu, thsp_w);
    uint32_t tmask = 0;
#pragma unroll
    for (int r = 0; r < R; ++r) tmask |= ((s_tgt[(i0 + r) >> 5] >> ((i0 + r) & 31)) & 1u) << r;
    const double zend = s_z[pad<R>(nvalid - 1)];

    // phase A: per term, thread aggregates and the warp scan
#pragma unroll 1
    for (int k = 0; k < NE; ++k) {
        const int deg = taylor_degree<Real>(c, k, hw);
        Real mr[R], mi[R];
#pragma unroll
        for (int r = 0; r < R; ++r) multiplier<Real>(c, k, deg, th[r], thw[r], mr[r], mi[r]);
        if constexpr (kF64) {
            double2* __restrict__ mt = a.mult + (int64_t)k * a.P + base + i0;
#pragma unroll
            for (int r = 0; r < R; ++r)
                if (i0 + r < nvalid) mt[r] = make_double2((double)mr[r], (double)mi[r]);
        }
        Real fr = s_al[pad<R>(i0)], fi = 0;
#pragma unroll
        for (int r = 1; r < R; ++r) cfma<Real>(mr[r], mi[r], fr, fi, s_al[pad<R>(i0 + r)], Real(0), fr, fi);
        Real Mr, Mi;
        multiplier<Real>(c, k, taylor_degree<Real>(c, k, hsp), thsp, thsp_w, Mr, Mi);
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            Real Mor = __shfl_up_sync(0xffffffffu, Mr, o), Moi = __shfl_up_sync(0xffffffffu, Mi, o);
            Real For = __shfl_up_sync(0xffffffffu, fr, o), Foi = __shfl_up_sync(0xffffffffu, fi, o);
            if (lane >= o) {
                cfma<Real>(Mr, Mi, For, Foi, fr, fi, fr, fi);
                cmul<Real>(Mr, Mi, Mor, Moi, Mr, Mi);
            }
        }
        Real Mxr = __shfl_up_sync(0xffffffffu, Mr, 1), Mxi = __shfl_up_sync(0xffffffffu, Mi, 1);
        Real Fxr = __shfl_up_sync(0xffffffffu, fr, 1), Fxi = __shfl_up_sync(0xffffffffu, fi, 1);
        if (lane == 0) { Mxr = 1; Mxi = 0; Fxr = 0; Fxi = 0; }
        Real* sc = s_scan + (size_t)k * 4 * T;
        sc[tid] = Mxr; sc[T + tid] = Mxi; sc[2 * T + tid] = Fxr; sc[3 * T + tid] = Fxi;
        if (lane == 31) {
            s_w[k][w][0] = (double)Mr; s_w[k][w][1] = (double)Mi;
            s_w[k][w][2] = (double)fr; s_w[k][w][3] = (double)fi;
        }
    }
    __syncthreads();
    // phase B: one lane per term joins the warps and the tiles
    if (tid < NE) tile_combine<NE, NW>(a, c, a.fdesc, tile, -1, tile == 0, zend, zprev, s_w, s_win, tid);
    __syncthreads();
    // phase C: apply the carries, final pass, evaluation at targets
    Real acc[R];
#pragma unroll
    for (int r = 0; r < R; ++r) acc[r] = 0;
#pragma unroll 1
    for (int k = 0; k < NE; ++k) {
        const Real* sc = s_scan + (size_t)k * 4 * T;
        Real fr, fi;
        cfma<Real>(sc[tid], sc[T + tid], (Real)s_win[k][w][0], (Real)s_win[k][w][1], sc[2 * T + tid],
                   sc[3 * T + tid], fr, fi);
        Real mr[R], mi[R];
        if constexpr (kF64) {
            const double2* __restrict__ mt = a.mult + (int64_t)k * a.P + base + i0;
#pragma unroll
            for (int r = 0; r < R; ++r) {
                double2 m = i0 + r < nvalid ? mt[r] : make_double2(1.0, 0.0);
                mr[r] = (Real)m.x;
                mi[r] = (Real)m.y;
            }
        } else {
            const int deg = taylor_degree<Real>(c, k, hw);
#pragma unroll
            for (int r = 0; r < R; ++r) multiplier<Real>(c, k, deg, th[r], thw[r], mr[r], mi[r]);
        }
        const Real Wr = (Real)c.w_re[k], Wi = (Real)c.w_im[k];
#pragma unroll
        for (int r = 0; r < R; ++r) {
            cfma<Real>(mr[r], mi[r], fr, fi, s_al[pad<R>(i0 + r)], Real(0), fr, fi);
            if ((tmask >> r) & 1u) acc[r] = fma(Wr, fr, fma(-Wi, fi, acc[r]));
        }
    }
    // forward partial sums, written coalesced through shared memory
    __syncthreads();
#pragma unroll
    for (int r = 0; r < R; ++r) s_z[pad<R>(i0 + r)] = (double)acc[r];
    __syncthreads();
    for (int i = tid; i < nvalid; i += T) a.fwd[base + i] = s_z[pad<R>(i)];
}

template <typename Real, int NE, int T, int R>
__global__ void __launch_bounds__(T) k_sweep_bwd(const SweepArgs a, const SweepConsts c) {
    using SM = SweepSmem<Real, NE, T, R>;
    constexpr int TILE = T * R;
    constexpr int NW = T / 32;
    constexpr bool kF64 = sizeof(Real) == 8;
    extern __shared__ __align__(16) unsigned char smem[];
    double* s_z = reinterpret_cast<double*>(smem + SM::z_off);
    Real* s_al = reinterpret_cast<Real*>(smem + SM::al_off);
    Real* s_scan = reinterpret_cast<Real*>(smem + SM::scan_off);
    __shared__ double s_w[NE][NW][4];
    __shared__ double s_win[NE][NW][2];
    __shared__ uint32_t s_tgt[TILE / 32];
    __shared__ uint32_t s_tile;

    const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
    if (tid == 0) s_tile = atomicAdd(&a.tile_ctr[1], 1u);
    __syncthreads();
    const int64_t tile = a.tiles - 1 - (int64_t)s_tile;
    const int64_t base = tile * TILE;
    const int nvalid = (int)min((int64_t)TILE, a.P - base);
    const bool has_next = base + TILE < a.P;
    const bool bufB = a.plan->final_buf == 1;
    const uint64_t* __restrict__ keys = bufB ? a.keysB : a.keysA;
    const uint32_t* __restrict__ vals = bufB ? a.valsB : a.valsA;
    stage_tile<Real, T, R>(a, keys, vals, base, nvalid, s_z, s_al, s_tgt);
    if (tid == 0) s_z[pad<R>(TILE)] = has_next ? key_coord(keys[base + TILE]) : 0.0;
    __syncthreads();

    const double s = c.s;
    const int i0 = tid * R;
    const double znext = s_z[pad<R>(TILE)], zfirst = s_z[0];
    // th[r]: gap between points i0+r and i0+r+1 (the FP64 path reads the stored multipliers)
    Real th[R];
    uint32_t thw[R];
    uint32_t hw = 0;
    if constexpr (!kF64) {
#pragma unroll
        for (int r = 0; r < R; ++r) {
            const int i = i0 + r;
            double t = 0.0;
            if (i + 1 < nvalid || (i + 1 == TILE && has_next)) t = s * (s_z[pad<R>(i + 1)] - s_z[pad<R>(i)]);
            th[r] = (Real)t;
            thw[r] = theta_hw<Real>(th[r]);
            hw = max(hw, thw[r]);
        }
        hw = __reduce_max_sync(0xffffffffu, hw);
    }
    double th_span = 0.0;
    {
        const int inext = i0 + R;
        if (i0 < nvalid && (inext < nvalid || (inext == TILE && has_next)))
            th_span = s * (s_z[pad<R>(inext)] - s_z[pad<R>(i0)]);
    }
    const Real thsp = (Real)th_span;
    const uint32_t thsp_w = theta_hw<Real>(thsp);
    const uint32_t hsp = __reduce_max_sync(0xffffffffu, thsp_w);
    uint32_t tmask = 0;
#pragma unroll
    for (int r = 0; r < R; ++r) tmask |= ((s_tgt[(i0 + r) >> 5] >> ((i0 + r) & 31)) & 1u) << r;

    auto load_mult = [&](int k, Real* mr, Real* mi) {
        if constexpr (kF64) {
            const double2* __restrict__ mt = a.mult + (int64_t)k * a.P + base + i0 + 1;
#pragma unroll
            for (int r = 0; r < R; ++r) {
                const int64_t p = base + i0 + r + 1;
                double2 m = p < a.P ? mt[r] : make_double2(0.0, 0.0);
                mr[r] = (Real)m.x;
                mi[r] = (Real)m.y;
            }
        } else {
            const int deg = taylor_degree<Real>(c, k, hw);
#pragma unroll
            for (int r = 0; r < R; ++r) multiplier<Real>(c, k, deg, th[r], thw[r], mr[r], mi[r]);
        }
    };

#pragma unroll 1
    for (int k = 0; k < NE; ++k) {
        Real mr[R], mi[R];
        load_mult(k, mr, mi);
        Real br = s_al[pad<R>(i0 + R - 1)], bi = 0;
#pragma unroll
        for (int r = R - 2; r >= 0; --r) cfma<Real>(mr[r], mi[r], br, bi, s_al[pad<R>(i0 + r)], Real(0), br, bi);
        Real Mr, Mi;
        multiplier<Real>(c, k, taylor_degree<Real>(c, k, hsp), thsp, thsp_w, Mr, Mi);
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            Real Mor = __shfl_down_sync(0xffffffffu, Mr, o), Moi = __shfl_down_sync(0xffffffffu, Mi, o);
            Real For = __shfl_down_sync(0xffffffffu, br, o), Foi = __shfl_down_sync(0xffffffffu, bi, o);
            if (lane + o < 32) {
                cfma<Real>(Mr, Mi, For, Foi, br, bi, br, bi);
                cmul<Real>(Mr, Mi, Mor, Moi, Mr, Mi);
            }
        }
        Real Mxr = __shfl_down_sync(0xffffffffu, Mr, 1), Mxi = __shfl_down_sync(0xffffffffu, Mi, 1);
        Real Fxr = __shfl_down_sync(0xffffffffu, br, 1), Fxi = __shfl_down_sync(0xffffffffu, bi, 1);
        if (lane == 31) { Mxr = 1; Mxi = 0; Fxr = 0; Fxi = 0; }
        Real* sc = s_scan + (size_t)k * 4 * T;
        sc[tid] = Mxr; sc[T + tid] = Mxi; sc[2 * T + tid] = Fxr; sc[3 * T + tid] = Fxi;
        if (lane == 0) {
            s_w[k][w][0] = (double)Mr; s_w[k][w][1] = (double)Mi;
            s_w[k][w][2] = (double)br; s_w[k][w][3] = (double)bi;
        }
    }
    __syncthreads();
    if (tid < NE) tile_combine<NE, NW>(a, c, a.bdesc, tile, +1, !has_next, zfirst, znext, s_w, s_win, tid);
    __syncthreads();
    Real acc[R];
#pragma unroll
    for (int r = 0; r < R; ++r) acc[r] = 0;
#pragma unroll 1
    for (int k = 0; k < NE; ++k) {
        const Real* sc = s_scan + (size_t)k * 4 * T;
        Real br, bi;  // state at the first point of the next thread
        cfma<Real>(sc[tid], sc[T + tid], (Real)s_win[k][w][0], (Real)s_win[k][w][1], sc[2 * T + tid],
                   sc[3 * T + tid], br, bi);
        Real mr[R], mi[R];
        load_mult(k, mr, mi);
        const Real Wr = (Real)c.w_re[k], Wi = (Real)c.w_im[k];
#pragma unroll
        for (int r = R - 1; r >= 0; --r) {
            cfma<Real>(mr[r], mi[r], br, bi, s_al[pad<R>(i0 + r)], Real(0), br, bi);
            if ((tmask >> r) & 1u) acc[r] = fma(Wr, br, fma(-Wi, bi, acc[r]));
        }
    }
    __syncthreads();
#pragma unroll
    for (int r = 0; r < R; ++r) s_z[pad<R>(i0 + r)] = (double)acc[r];
    __syncthreads();
    for (int i = tid; i < nvalid; i += T) {
        if ((s_tgt[i >> 5] >> (i & 31)) & 1u) {
            const int64_t p = base + i;
            const uint32_t v = vals[p];
            a.u[(int64_t)v - a.N] = a.fwd[p] + s_z[pad<R>(i)];
        }
    }
}

}  // namespace fgt1d
