// Range partition of one transform: the device kernels of the segment entry points.
//
// The recurrences of eqs. 4.5-4.6 are affine in the state, so one contiguous range of
// the sorted coordinate line (a "segment", e.g. one GPU's share of the points) can be
// swept alone with zero entering states.  Two numbers per term then summarise what the
// segment contributes to the rest of the line:
//   F_k = sum over its sources of alpha_j exp(-tau_k s (z_last - y_j))   (forward state at
//         its last point), and
//   G_k = sum over its sources of alpha_j exp(-tau_k s (y_j - z_first))  (backward state
//         at its first point, that point's own strength included),
// and the states entering it from the left and right are compositions of its
// neighbours' F and G with span exponentials (host code, fgt1d_segment_compose).  Their
// contribution to a target x of the segment is Re sum_k W_k (F_in,k exp(-tau_k s (x -
// z_prev)) + G_in,k exp(-tau_k s (z_next - x))), added by k_carry_apply with directly
// computed FP64 exponentials: terms below 2^-60 of the carry (exp(-Re tau_k s d) <
// 2^-60) are skipped, so the pass costs little once the carries have decayed.
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include "kernels.h"

namespace fgt1d {

namespace {

__device__ __forceinline__ double seg_key_coord(uint64_t k) {
    const uint64_t b = (k >> 63) ? (k & 0x7FFFFFFFFFFFFFFFull) : ~k;
    return __longlong_as_double((long long)b);
}

// One warp: the segment's boundary record from the sweeps' look-back descriptors (the
// inclusive values of the last forward tile and the first backward tile) and the sorted
// keys.  Layout: Re F, Im F, Re G, Im G (n_e each), z_first, z_last.
__global__ void k_segment_boundary(const TileDesc* __restrict__ fdesc, const TileDesc* __restrict__ bdesc,
                                   const int64_t* __restrict__ total_tiles, const SortPlan* __restrict__ plan,
                                   const uint64_t* __restrict__ keysA, const uint64_t* __restrict__ keysB, int64_t P,
                                   int n_e, double* __restrict__ out) {
    const int k = threadIdx.x;
    const int64_t nt = *total_tiles;
    if (k < n_e) {
        double fr = 0.0, fi = 0.0, gr = 0.0, gi = 0.0;
        if (nt > 0) {
            const TileDesc& f = fdesc[(nt - 1) * n_e + k];
            const TileDesc& b = bdesc[k];
            fr = f.inc_re;
            fi = f.inc_im;
            gr = b.inc_re;
            gi = b.inc_im;
        }
        out[k] = fr;
        out[n_e + k] = fi;
        out[2 * n_e + k] = gr;
        out[3 * n_e + k] = gi;
    }
    if (k == 0) {
        const uint64_t* keys = plan->final_buf == 1 ? keysB : keysA;
        const double nan = __longlong_as_double(0x7FF8000000000000ll);
        out[4 * n_e] = (P > 0 && nt > 0) ? seg_key_coord(keys[0]) : nan;
        out[4 * n_e + 1] = (P > 0 && nt > 0) ? seg_key_coord(keys[P - 1]) : nan;
    }
}

// exp(-tau s d) for d >= 0 (FP64)
__device__ __forceinline__ void seg_cexp(double tr, double ti, double sd, double& er, double& ei) {
    const double mag = exp(-tr * sd);
    double sn, cs;
    sincos(ti * sd, &sn, &cs);
    er = mag * cs;
    ei = -mag * sn;
}

// One thread per sorted position: targets gain the carries' contribution.
__global__ void __launch_bounds__(256) k_carry_apply(const SortPlan* __restrict__ plan,
                                                     const uint64_t* __restrict__ keysA,
                                                     const uint64_t* __restrict__ keysB,
                                                     const uint32_t* __restrict__ valsA,
                                                     const uint32_t* __restrict__ valsB, int64_t P, int64_t N,
                                                     SegmentConsts sc, const double* __restrict__ carry,
                                                     double* __restrict__ u, const uint32_t* status) {
    if (*(volatile const uint32_t*)status & kStatusSortTimeout) return;  // sorted codes not valid
    const uint64_t* keys = plan->final_buf == 1 ? keysB : keysA;
    const uint32_t* vals = plan->final_buf == 1 ? valsB : valsA;
    const int n = sc.n_e;
    const double zp = carry[4 * n], zn = carry[4 * n + 1];
    const bool left = !isnan(zp), right = !isnan(zn);
    // beyond this distance exp(-Re tau_k s d) < 2^-60 for every term
    const double cut = 60.0 * 0.69314718055994531 / (sc.min_re_tau * sc.s);
    for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < P; p += (int64_t)gridDim.x * blockDim.x) {
        const uint32_t v = vals[p];
        if ((int64_t)v < N) continue;  // a source
        const double z = seg_key_coord(keys[p]);
        const double dl = left ? z - zp : 0.0, dr = right ? zn - z : 0.0;
        const bool use_l = left && dl < cut, use_r = right && dr < cut;
        if (!use_l && !use_r) continue;
        double acc = 0.0;
        for (int k = 0; k < n; ++k) {
            double er, ei, hr = 0.0, hi = 0.0;
            if (use_l) {
                seg_cexp(sc.tau_re[k], sc.tau_im[k], sc.s * dl, er, ei);
                hr = er * carry[k] - ei * carry[n + k];
                hi = er * carry[n + k] + ei * carry[k];
            }
            if (use_r) {
                seg_cexp(sc.tau_re[k], sc.tau_im[k], sc.s * dr, er, ei);
                hr += er * carry[2 * n + k] - ei * carry[3 * n + k];
                hi += er * carry[3 * n + k] + ei * carry[2 * n + k];
            }
            acc += sc.w_re[k] * hr - sc.w_im[k] * hi;
        }
        u[(int64_t)v - N] += acc;
    }
}

// The boundary record of a segment without points: zero states, NaN coordinates.
__global__ void k_segment_empty(int n_e, double* __restrict__ out) {
    const int i = threadIdx.x;
    if (i < 4 * n_e) out[i] = 0.0;
    else if (i < 4 * n_e + 2) out[i] = __longlong_as_double(0x7FF8000000000000ll);
}

}  // namespace

cudaError_t launch_segment_empty(int n_e, double* out, cudaStream_t st) {
    k_segment_empty<<<1, 64, 0, st>>>(n_e, out);
    return cudaGetLastError();
}

cudaError_t launch_segment_boundary(const SweepArgs& a, int64_t P, int n_e, double* out, cudaStream_t st) {
    k_segment_boundary<<<1, 32, 0, st>>>(a.fdesc, a.bdesc, a.total_tiles, a.plan, a.keysA, a.keysB, P, n_e, out);
    return cudaGetLastError();
}

cudaError_t launch_carry_apply(const SweepArgs& a, int64_t P, const SegmentConsts& sc, const double* carry, double* u,
                               cudaStream_t st) {
    if (P <= 0) return cudaSuccess;
    const int blocks = (int)((P + 255) / 256 < 152 * 8 ? (P + 255) / 256 : 152 * 8);
    k_carry_apply<<<blocks, 256, 0, st>>>(a.plan, a.keysA, a.keysB, a.valsA, a.valsB, P, a.N, sc, carry, u, a.status);
    return cudaGetLastError();
}

}  // namespace fgt1d
