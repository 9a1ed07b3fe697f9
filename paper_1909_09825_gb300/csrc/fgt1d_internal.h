// Internal declarations shared by the host plan code and the CUDA kernels.
#pragma once

#include <stdint.h>

#include "../../include/fgt1d.h"

struct fgt1d_plan_s {
    int n;              // CF order (0 when built from a caller SOE)
    int n_e;            // number of kept conjugate-pair terms
    double delta;
    double E_n;
    unsigned flags;
    int tile_threads;   // sweep tile shape: 0 (precision default), 128 or 256
    double tau_re[FGT1D_MAX_TERMS], tau_im[FGT1D_MAX_TERMS];
    double w_re[FGT1D_MAX_TERMS], w_im[FGT1D_MAX_TERMS];
};

namespace fgt1d {

// Device status bits recorded in the workspace header.
enum : uint32_t {
    kStatusNonFinite = 1u,
    kStatusTimeout = 2u,
    kStatusBadArg = 4u,     // a batch item with a bad delta or negative size
    kStatusSortTimeout = 8u,  // a sort wait gave up: the sorted codes are not valid, and the
                              // kernels that index outputs by them skip their work
};

// Degree limit of the per-point Taylor multiplier e^{-tau theta} and the number of
// thresholds kept per plan.
constexpr int kTaylorMax = 12;

// Per-launch constants of the sweep kernels (passed by value).
struct SweepConsts {
    int n_e;
    double s;                       // 1 / sqrt(delta)
    float s_f;                      // the same in FP32
    double tau_re[FGT1D_MAX_TERMS], tau_im[FGT1D_MAX_TERMS];
    double w_re[FGT1D_MAX_TERMS], w_im[FGT1D_MAX_TERMS];
    double v_re[FGT1D_MAX_TERMS], v_im[FGT1D_MAX_TERMS];   // V_k = -tau_k s W_k (derivative weights)
    // Taylor coefficients (-tau_k)^j / j!, j = 0..kTaylorMax, per term
    double tc_re[FGT1D_MAX_TERMS][kTaylorMax + 1], tc_im[FGT1D_MAX_TERMS][kTaylorMax + 1];
    float tcf_re[FGT1D_MAX_TERMS][kTaylorMax + 1], tcf_im[FGT1D_MAX_TERMS][kTaylorMax + 1];
    float tauf_re[FGT1D_MAX_TERMS], tauf_im[FGT1D_MAX_TERMS];
    // theta thresholds: Taylor degree d is enough (FP64) while theta <= theta_lim[d];
    // stored as the high 32 bits of the double so that warps compare them as integers.
    uint32_t theta_hi_lim[FGT1D_MAX_TERMS][kTaylorMax + 1];
    uint32_t theta_hi_lim_f[FGT1D_MAX_TERMS][kTaylorMax + 1];   // same for the FP32 path (float bits)
    // double-float path: coefficients and weights split into hi + lo floats, thresholds
    // on the bit pattern of the high float
    float tcd_re_hi[FGT1D_MAX_TERMS][kTaylorMax + 1], tcd_re_lo[FGT1D_MAX_TERMS][kTaylorMax + 1];
    float tcd_im_hi[FGT1D_MAX_TERMS][kTaylorMax + 1], tcd_im_lo[FGT1D_MAX_TERMS][kTaylorMax + 1];
    float wd_re[FGT1D_MAX_TERMS][2], wd_im[FGT1D_MAX_TERMS][2], vd_re[FGT1D_MAX_TERMS][2], vd_im[FGT1D_MAX_TERMS][2];
    uint32_t theta_hi_lim_d[FGT1D_MAX_TERMS][kTaylorMax + 1];
    // double-float: largest theta (float bits) for which the Taylor terms beyond degree J
    // can be summed in FP32, |tau_k theta|^(J+1) / (J+1)! <= 2^-28 (index J = 1..kTaylorMax)
    uint32_t theta_split_d[FGT1D_MAX_TERMS][kTaylorMax + 1];
    // FP64: largest theta (high word) with |tau_k| theta <= 2^-10, below which the Taylor
    // terms of degree >= 3 can be summed in FP32 (taylor_hybrid)
    uint32_t theta_hyb_lim[FGT1D_MAX_TERMS];
};

}  // namespace fgt1d
