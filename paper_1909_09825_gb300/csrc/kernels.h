// Launch-side declarations of the CUDA kernels (internal).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "fgt1d_internal.h"

namespace fgt1d {

// Every kernel works on a batch of independent transforms ("items"; one item for
// fgt1d_execute).  Item b's merged points [y_b (sources), x_b (targets)] occupy the
// range [start_b, start_b + nsrc_b + ntgt_b) of the merged arrays, start_b a multiple of
// kTile; the rest of its padded range [start_b, start_b + ntiles_b * kTile) holds
// padding that sorts to the end.  A tile therefore never straddles two items and each
// item's decoupled look-back stays inside its own tiles.
constexpr int kTile = 4096;

struct Item {
    int64_t start;    // padded merged offset (multiple of kTile)
    int64_t nsrc;     // N_b
    int64_t ntgt;     // M_b
    int64_t y_off;    // offset of the item's sources in y / alpha
    int64_t x_off;    // offset of the item's targets in x / u
    int64_t tile0;    // start / kTile
    int64_t ntiles;   // padded size / kTile
    double s;         // 1 / sqrt(delta_b)
};

// Item b of tile t: the last item whose first tile is <= t (empty items share their
// successor's first tile and are skipped).
__device__ __forceinline__ int item_of_tile(const Item* __restrict__ items, int B, int64_t t) {
    int lo = 0, hi = B;
    while (hi - lo > 1) {
        const int mid = (lo + hi) >> 1;
        if (items[mid].tile0 <= t) lo = mid;
        else hi = mid;
    }
    while (lo + 1 < B && items[lo + 1].tile0 <= t) ++lo;
    return lo;
}

// Builds the item table from device offsets x_off/y_off (B+1 entries each) and the
// per-item bandwidths (device array, or the plan's delta when null).  Writes the total
// number of tiles to *total_tiles.  An item whose offsets leave [0, M_tot] / [0, N_tot]
// or decrease, or whose delta is not positive and finite, is left empty and flagged in
// status; if the items need more than max_tiles tiles (overlapping ranges) none runs.
cudaError_t launch_items(int B, const int64_t* x_off, const int64_t* y_off, const double* delta, double plan_delta,
                         Item* items, int64_t* total_tiles, uint32_t* status, int64_t max_tiles, int64_t M_tot,
                         int64_t N_tot, cudaStream_t st);
// One item of M targets and N sources with bandwidth delta (fgt1d_execute).
cudaError_t launch_item_single(int64_t M, int64_t N, double delta, Item* items, int64_t* total_tiles,
                               cudaStream_t st);

// ---- sort (steps a1-a2) ----
constexpr int kSortDigits = 8;      // 8-bit digits of a 64-bit key (the full sort)
constexpr int kPrefixDigits = 4;    // 8-bit digits of a 32-bit prefix key (the prefix sort)
constexpr int kSortThreads = 256;
constexpr int kSortIPT = 16;
constexpr int kSortTile = kSortThreads * kSortIPT;
static_assert(kSortTile == kTile, "sort tiles and item padding share one size");
// Longest run of equal prefix keys that the fix-up sorts (one thread per run); a longer
// run with coordinates out of order sends the sort to the full 64-bit passes.
constexpr int kRunMax = 32;
// Default upper bound on one inter-block spin wait, in SM clock cycles (about 2 s at
// 2 GHz); the launch arguments carry the bound in force (spin_limit).
constexpr long long kSpinLimitCycles = 4000000000LL;

struct SortPlan {
    uint32_t active[kSortDigits];   // full sort: digit d runs a pass
    int32_t src[kSortDigits];   // -1: keys generated from x/y; 0: buffer A; 1: buffer B
    int32_t dst[kSortDigits];
    int32_t final_buf;          // buffer (0 = A, 1 = B) that holds the sorted keys/indices
    uint32_t active_mask;       // bit d: some item has more than one populated bucket in digit d
    uint32_t unsorted;          // some item's sources or targets are not in non-decreasing order
    uint32_t merge;             // 1: every run is presorted, the sort is one merge into buffer A
};
static_assert(128 + sizeof(SortPlan) <= 256, "the sort plan sits in the workspace header");

// The prefix sort: 32-bit keys that are a non-decreasing function of the coordinate
// within each item (fixed point over the item's coordinate range), sorted by four
// digit passes that carry the full 64-bit keys and the codes.  Runs of equal prefix keys
// then hold merged-index order and are fixed up; too long a run with coordinates out
// of order sets `fallback` and the full sort runs from the start.
struct PrefixPlan {
    uint32_t active[kPrefixDigits];
    // buffers (prefix keys, full keys, codes): 0 = (pre, keysA, valsA), 1 = (pre + Ppad,
    // keysB, valsB); the histogram pass writes buffer 1
    int32_t src[kPrefixDigits];
    int32_t dst[kPrefixDigits];
    int32_t final_buf;            // buffer of the sorted points
    uint32_t mask;                // bit d: some item has more than one populated bucket in prefix digit d
    uint32_t fallback;
    uint32_t nruns;               // runs listed for the fix-up (in the other buffer's prefix words)
    uint32_t pass_ctr[kPrefixDigits];
};

// Per-item prefix map: prefix(z) = (Q(z) - qlo) >> sh, Q(z) = sign(z) floor(|z| / 2^(eh - 1075))
// (eh = the larger biased exponent of the item's extreme coordinates).  Built in place
// of the item's coordinate range (~min key, max key).
struct PrefixMap {
    int64_t qlo;
    int32_t eh;
    int32_t sh;
};

struct SortArgs {
    const double* x;
    const double* y;
    int64_t N;            // total number of sources (targets are coded N + i)
    int64_t M;            // total number of targets (codes below N + M are points)
    const Item* items;
    int B;
    const int64_t* total_tiles;  // device scalar
    int64_t max_tiles;    // grid size of the tile kernels (upper bound of *total_tiles)
    int64_t Ppad;         // max_tiles * kTile
    uint64_t* keysA;
    uint64_t* keysB;
    uint32_t* valsA;
    uint32_t* valsB;
    uint32_t* pre;        // [2][Ppad] prefix keys of the prefix sort's buffers 0 and 1 (scratch)
    uint32_t* hist;       // [B][8][256] per-item digit counts
    uint32_t* offs;       // [B][8][256] per-item bucket starts (merged positions)
    SortPlan* plan;
    PrefixPlan* pplan;
    PrefixMap* maps;      // [B], zeroed before the sort
    uint64_t* desc;       // [8][desc_stride] look-back words
    size_t desc_stride;   // max_tiles * 256
    uint32_t* tile_ctr;   // [8] (full passes)
    uint32_t* status;
    long long spin_limit = kSpinLimitCycles;  // bound of one look-back wait, SM cycles
};

cudaError_t launch_sort(const SortArgs& a, cudaStream_t st);
// copies the first P sorted merged codes (item 0) to perm
cudaError_t launch_copy_perm(const SortArgs& a, int64_t P, uint32_t* perm, cudaStream_t st);
// Exchanges the roles of a sorted single item's points in its codes: sources [0, n_src)
// become targets n_tgt + j, targets n_src + i become sources i (the order is kept).
cudaError_t launch_swap_codes(const SortArgs& a, int64_t P, int64_t n_src, int64_t n_tgt, cudaStream_t st);

// ---- sweeps (steps a3-a7) ----
struct TileDesc {           // one (tile, term) entry of the decoupled look-back
    double agg_re, agg_im;  // tile aggregate (zero carry) at the tile's anchor point
    double inc_re, inc_im;  // inclusive value (all carries)
    double M_re, M_im;      // exp(-tau s (anchor - previous anchor)), computed directly
    uint32_t flag;          // 0 none, 1 aggregate, 2 inclusive
    uint32_t pad;
};

struct SweepArgs {
    int64_t N;              // total number of sources
    const Item* items;
    int B;
    const int64_t* total_tiles;
    int64_t max_tiles;
    int64_t Ppad;           // padded merged length (multiplier table stride)
    const uint64_t* keysA;
    const uint64_t* keysB;
    const uint32_t* valsA;
    const uint32_t* valsB;
    const SortPlan* plan;
    const double* alpha;
    double2* mult;          // [n_e][Ppad] multiplier table (FP64 path) or nullptr
    void* fwd;              // [Ppad] forward partial sums Re sum_k W_k h+_k (double; float on the FP32 path)
    void* fwd2;             // [Ppad] forward partial sums of the derivative channel
    double* u;              // output, target order: Re sum_k W_k (h+ + h-) (value channel)
    double* out2;           // output, target order: s Re sum_k V'_k (h+ - h-) (derivative channel)
    TileDesc* fdesc;        // [max_tiles][n_e]
    TileDesc* bdesc;        // [max_tiles][n_e]
    uint32_t* tile_ctr;     // [2]
    uint32_t* status;
    int reuse = 0;          // 1: the multiplier table holds a bound geometry's multipliers
    int self = 0;           // 1: identical targets and sources (every point is both; FP64, FP32)
    // equal-coordinate flag (may be null; gradient sweeps only): the forward sweep of the
    // derivative channel sets it when two merged points share a coordinate; the
    // coincidence scan, whose output is then all zero, returns at once while it is clear
    uint32_t* ties = nullptr;
    long long spin_limit = kSpinLimitCycles;  // bound of one look-back wait, SM cycles
};

// Evaluation channels of the sweeps: bit 0 values Re sum W (h+ + h-) into u, bit 1 the
// derivative s Re sum V' (h+ - h-) into out2 (V'_k = -tau_k W_k).
// `mid` (may be null) is recorded on st between the forward and the backward kernel.
// shape: 0 = 128 threads x 32 points, 1 = 256 threads x 16 points.
constexpr int kNumShapes = 2;
cudaError_t launch_sweeps_f64(const SweepArgs& a, const SweepConsts& c, cudaStream_t st, cudaEvent_t mid, int ev,
                              int shape);
cudaError_t launch_sweeps_f32(const SweepArgs& a, const SweepConsts& c, cudaStream_t st, cudaEvent_t mid, int ev,
                              int shape);
// Double-float sweeps (value channel only).
cudaError_t launch_sweeps_df(const SweepArgs& a, const SweepConsts& c, cudaStream_t st, cudaEvent_t mid, int shape);
// Fills the multiplier table of a bound geometry (one block per tile) in the
// thread-interleaved layout of sweep tile shape `shape`: FP64 entries, or double-float
// entries for the double-float sweeps.
cudaError_t launch_fill_table(const SweepArgs& a, const SweepConsts& c, int shape, bool dfloat_entries,
                              cudaStream_t st);
// Geometry tag check before an apply: when *tag != expect, flags kStatusBadArg and sets
// *total_tiles = 0 so that no sweep tile runs on an unbound workspace.
cudaError_t launch_geometry_check(const uint64_t* tag, uint64_t expect, int64_t* total_tiles, uint32_t* status,
                                  cudaStream_t st);
cudaError_t launch_geometry_tag(uint64_t* tag, uint64_t value, cudaStream_t st);
// Coincidence sums: u[i] = sum of alpha over the sources at exactly the coordinate of
// target i (one forward scan with multiplier 1 on zero gaps and 0 otherwise).  With
// identical points (a.self) u[p] is, per sorted position p, the sum over the points of
// p's run of equal coordinates up to p.
cudaError_t launch_coincidence(const SweepArgs& a, const SweepConsts& c, cudaStream_t st);
// Targets before sources on equal coordinates (roles exchanged after the sort): when the
// equal-coordinate flag is set, A[i] = F[last position of target i's run of equal
// coordinates], F from launch_coincidence with a.self set (sums over sorted positions),
// i.e. the run's total source strength.
cudaError_t launch_coinc_gather(const SweepArgs& a, const double* F, int64_t n, double* A, cudaStream_t st);
// Identical points: u[point at sorted position p] += cf * F[last position of p's run of
// equal coordinates], F from launch_coincidence (the run's total strength).
cudaError_t launch_self_exact(const SweepArgs& a, const double* F, int64_t n, double cf, double* u, cudaStream_t st);

// ---- range partition (segments of one transform) ----
struct SegmentConsts {
    int n_e;
    double s;            // 1 / sqrt(delta)
    double min_re_tau;   // smallest Re tau_k (the slowest decay)
    double tau_re[FGT1D_MAX_TERMS], tau_im[FGT1D_MAX_TERMS];
    double w_re[FGT1D_MAX_TERMS], w_im[FGT1D_MAX_TERMS];
};
// The segment's boundary record (4 n_e + 2 doubles) from the sweeps' descriptors and the
// sorted keys of a single item of P points; must run before the descriptors are reused.
cudaError_t launch_segment_boundary(const SweepArgs& a, int64_t P, int n_e, double* out, cudaStream_t st);
// The record of a segment without points (zero states, NaN coordinates).
cudaError_t launch_segment_empty(int n_e, double* out, cudaStream_t st);
// u[target] += the contribution of the entering states in `carry` (device, 4 n_e + 2
// doubles: Re/Im F_in, Re/Im G_in, z_prev, z_next; NaN coordinate = no neighbour).
cudaError_t launch_carry_apply(const SweepArgs& a, int64_t P, const SegmentConsts& sc, const double* carry, double* u,
                               cudaStream_t st);

// fgt1d_execute on a caller-given workspace (checked against the layout size)
int run_transform_in(const fgt1d_plan_s& p, const double* x, int64_t M, const double* y, const double* alpha,
                     int64_t N, double* u, void* ws, size_t ws_bytes, cudaStream_t st);
size_t transform_workspace_bytes(const fgt1d_plan_s& p, int64_t M, int64_t N);

// gradient assembly: out[i] = w[i] (D[i] - A[i] sumV)
cudaError_t launch_grad_assemble(const double* w, const double* D, const double* A, double sumV, int64_t n,
                                 double* out, cudaStream_t st);
// y[i] += c a[i]
cudaError_t launch_axpy(const double* a, double c, int64_t n, double* y, cudaStream_t st);
// *out = -(1/(2 delta)) (sum (x - x[0]) gx + sum (y - x[0]) gy), with nb partial sums
constexpr int kGradPartials = 608;
cudaError_t launch_grad_delta(const double* x, const double* gx, int64_t M, const double* y, const double* gy,
                              int64_t N, double delta, double* partials, int nb, double* out, cudaStream_t st);

}  // namespace fgt1d
