// Launch-side declarations of the CUDA kernels (internal).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "fgt1d_internal.h"

namespace fgt1d {

// ---- sort (steps a1-a2) ----
constexpr int kSortDigits = 8;      // 8-bit digits of a 64-bit key
constexpr int kSortThreads = 256;
constexpr int kSortIPT = 16;
constexpr int kSortTile = kSortThreads * kSortIPT;
// Upper bound on one inter-block spin wait, in SM clock cycles (about 2 s at 2 GHz).
constexpr long long kSpinLimitCycles = 4000000000LL;

struct SortPlan {
    uint32_t active[kSortDigits];
    int32_t src[kSortDigits];   // -1: keys generated from x/y; 0: buffer A; 1: buffer B
    int32_t dst[kSortDigits];
    int32_t final_buf;          // buffer (0 = A, 1 = B) that holds the sorted keys/indices
};

struct SortArgs {
    const double* x;
    const double* y;
    int64_t N, P;
    uint64_t* keysA;
    uint64_t* keysB;
    uint32_t* valsA;
    uint32_t* valsB;
    uint32_t* hist;       // [8][256]
    uint32_t* offs;       // [8][256]
    SortPlan* plan;
    uint64_t* desc;       // [8][desc_stride] look-back words
    size_t desc_stride;   // tiles * 256
    uint32_t* tile_ctr;   // [8]
    uint32_t* status;
};

cudaError_t launch_sort(const SortArgs& a, cudaStream_t st);

// ---- sweeps (steps a3-a7) ----
struct TileDesc {           // one (tile, term) entry of the decoupled look-back
    double agg_re, agg_im;  // tile aggregate (zero carry) at the tile's anchor point
    double inc_re, inc_im;  // inclusive value (all carries)
    double M_re, M_im;      // exp(-tau s (anchor - previous anchor)), computed directly
    uint32_t flag;          // 0 none, 1 aggregate, 2 inclusive
    uint32_t pad;
};

struct SweepArgs {
    int64_t P, N;
    const uint64_t* keysA;
    const uint64_t* keysB;
    const uint32_t* valsA;
    const uint32_t* valsB;
    const SortPlan* plan;
    const double* alpha;
    double2* mult;          // [n_e][P] multiplier table (FP64 path) or nullptr
    void* fwd;              // [P] forward partial sums Re sum_k W_k h+_k at targets (double; float on the FP32 path)
    void* fwd2;             // [P] forward partial sums Re sum_k V_k h+_k (derivative channel)
    double* u;              // [M] output: Re sum_k W_k (h+ + h-) (value channel)
    double* out2;           // [M] output: Re sum_k V_k (h+ - h-) (derivative channel)
    TileDesc* fdesc;        // [tiles][n_e]
    TileDesc* bdesc;        // [tiles][n_e]
    uint32_t* tile_ctr;     // [2]
    uint32_t* status;
    int64_t tiles;
};

int sweep_tile_f64();  // points per sweep tile
int sweep_tile_f32();
// Evaluation channels of the sweeps: bit 0 values Re sum W (h+ + h-) into u, bit 1 the
// derivative Re sum V (h+ - h-) into out2 (V_k = -tau_k s W_k).
// `mid` (may be null) is recorded on st between the forward and the backward kernel.
cudaError_t launch_sweeps_f64(const SweepArgs& a, const SweepConsts& c, cudaStream_t st, cudaEvent_t mid, int ev);
cudaError_t launch_sweeps_f32(const SweepArgs& a, const SweepConsts& c, cudaStream_t st, cudaEvent_t mid, int ev);
// Coincidence sums: u[i] = sum of alpha over the sources at exactly the coordinate of
// target i (one forward scan with multiplier 1 on zero gaps and 0 otherwise).
cudaError_t launch_coincidence(const SweepArgs& a, const SweepConsts& c, cudaStream_t st);

// copies the sorted merged indices (final sort buffer) to perm
cudaError_t launch_copy_perm(const SortArgs& a, uint32_t* perm, cudaStream_t st);

// fgt1d_execute on a caller-given workspace (checked against the layout size)
int run_transform_in(const fgt1d_plan_s& p, const double* x, int64_t M, const double* y, const double* alpha,
                     int64_t N, double* u, void* ws, size_t ws_bytes, cudaStream_t st);
size_t transform_workspace_bytes(const fgt1d_plan_s& p, int64_t M, int64_t N);

// gradient assembly: out[i] = w[i] (D[i] - A[i] sumV)
cudaError_t launch_grad_assemble(const double* w, const double* D, const double* A, double sumV, int64_t n,
                                 double* out, cudaStream_t st);
// *out = -(1/(2 delta)) (sum (x - x[0]) gx + sum (y - x[0]) gy), with nb partial sums
constexpr int kGradPartials = 608;
cudaError_t launch_grad_delta(const double* x, const double* gx, int64_t M, const double* y, const double* gy,
                              int64_t N, double delta, double* partials, int nb, double* out, cudaStream_t st);

}  // namespace fgt1d
