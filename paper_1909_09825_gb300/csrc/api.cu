// C ABI entry points: argument checks, workspace layout, launch sequence.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstddef>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <limits>

#include "fgt1d_internal.h"
#include "kernels.h"

namespace fgt1d {
namespace {

constexpr size_t kAlign = 256;
inline size_t align_up(size_t v) { return (v + kAlign - 1) / kAlign * kAlign; }

// Workspace layout.  [0, zero_end) is cleared at the start of every pipeline.  Sizes are
// upper bounds for B items totalling M targets and N sources: each item pads its merged
// range to whole tiles, which adds at most one tile per item.
struct Layout {
    size_t header = 0;       // status (u32 at 0), full-sort tile counters (8 u32 at 32), sweep tile
                             // counters (2 u32 at 64), total tiles (i64 at 80), equal-coordinate
                             // flag (u32 at 88), geometry tag (u64 at 96), SortPlan at 128
    size_t hist = 0, offs = 0, sort_desc = 0, fdesc = 0, bdesc = 0;
    size_t sort_aux = 0;     // PrefixPlan (256 B), then the per-item prefix maps
    size_t zero_end = 0;
    size_t items = 0;
    size_t keysA = 0, keysB = 0, valsA = 0, valsB = 0, mult = 0, fwd = 0, fwd2 = 0, coinc = 0, pre = 0;
    size_t gD = 0, gA = 0, gx = 0, gy = 0, parts = 0;   // gradients
    size_t hx = 0, hy = 0, ha = 0, hu = 0;              // device copies of host arrays
    size_t total = 0;
    int64_t max_tiles = 0, Ppad = 0;
    int B = 1;
};

Layout make_layout(int64_t M, int64_t N, int B, int n_e, unsigned flags, bool sweeps, bool host, bool grad = false) {
    Layout L;
    L.B = B;
    const int64_t P = M + N;
    L.max_tiles = (P + kTile - 1) / kTile + (B - 1);
    L.Ppad = L.max_tiles * kTile;
    const size_t Pp = (size_t)L.Ppad;
    size_t off = 0;
    L.header = off; off += align_up(256);
    L.hist = off; off += align_up(sizeof(uint32_t) * kSortDigits * 256 * (size_t)B);
    L.offs = off; off += align_up(sizeof(uint32_t) * kSortDigits * 256 * (size_t)B);
    L.sort_desc = off; off += align_up(sizeof(uint64_t) * kSortDigits * (size_t)L.max_tiles * 256);
    L.sort_aux = off; off += align_up(256 + sizeof(PrefixMap) * (size_t)B);
    const int64_t st = sweeps ? L.max_tiles : 0;
    L.fdesc = off; off += align_up(sizeof(TileDesc) * (size_t)st * (size_t)n_e);
    L.bdesc = off; off += align_up(sizeof(TileDesc) * (size_t)st * (size_t)n_e);
    L.zero_end = off;
    L.items = off; off += align_up(sizeof(Item) * (size_t)B);
    L.keysA = off; off += align_up(sizeof(uint64_t) * Pp);
    L.keysB = off; off += align_up(sizeof(uint64_t) * Pp);
    L.valsA = off; off += align_up(sizeof(uint32_t) * Pp);
    L.valsB = off; off += align_up(sizeof(uint32_t) * Pp);
    if (sweeps) {
        // the multiplier table serves the FP64 and double-float sweeps (16 B per point and term)
        if (!(flags & FGT1D_FP32)) { L.mult = off; off += align_up(sizeof(double2) * (size_t)n_e * Pp); }
        L.fwd = off; off += align_up(sizeof(double) * Pp);
        if (flags & FGT1D_EXACT_SELF) { L.coinc = off; off += align_up(sizeof(double) * (size_t)M); }
    }
    // the prefix sort's scratch (two arrays of 32-bit keys): the forward partial sums,
    // which the sweeps write after the sort, or a region of its own
    if (sweeps) {
        L.pre = L.fwd;
    } else {
        L.pre = off; off += align_up(sizeof(uint32_t) * 2 * Pp);
    }
    if (grad) {
        const size_t mx = (size_t)std::max(M, N);
        L.fwd2 = off; off += align_up(sizeof(double) * Pp);
        L.gD = off; off += align_up(sizeof(double) * mx);
        L.gA = off; off += align_up(sizeof(double) * mx);
        L.gx = off; off += align_up(sizeof(double) * (size_t)M);
        L.gy = off; off += align_up(sizeof(double) * (size_t)N);
        L.parts = off; off += align_up(sizeof(double) * kGradPartials);
    }
    if (host) {
        L.hx = off; off += align_up(sizeof(double) * (size_t)M);
        L.hy = off; off += align_up(sizeof(double) * (size_t)N);
        L.ha = off; off += align_up(sizeof(double) * (size_t)N);
        L.hu = off; off += align_up(sizeof(double) * (size_t)M);
    }
    L.total = off;
    return L;
}

bool sizes_ok(int64_t M, int64_t N) {
    return M >= 0 && N >= 0 && M + N < (int64_t(1) << 31);
}

int ws_ok(const void* ws, size_t ws_bytes, const Layout& L) {
    if (!ws || (reinterpret_cast<uintptr_t>(ws) % kAlign) != 0 || ws_bytes < L.total) return FGT1D_EWORKSPACE;
    return FGT1D_OK;
}

// Bounded waits under test, without a GPU fault: FGT1D_SPIN_LIMIT_CYCLES (a positive
// integer) replaces the default bound of one inter-block wait, and FGT1D_FAULT injects
// a tile that never publishes -- "sweep_timeout" starts the forward sweep's tile counter
// at 1, "sort_timeout" every prefix digit pass's, so tile 0 is never processed and tile 1's
// look-back wait runs out.  Read at every call.
long long spin_limit_from_env() {
    const char* v = std::getenv("FGT1D_SPIN_LIMIT_CYCLES");
    if (!v) return kSpinLimitCycles;
    const long long c = std::atoll(v);
    return c > 0 ? c : kSpinLimitCycles;
}
enum Fault { kNoFault = 0, kSweepTimeout = 1, kSortTimeout = 2 };
int fault_from_env() {
    const char* v = std::getenv("FGT1D_FAULT");
    if (!v) return kNoFault;
    if (!std::strcmp(v, "sweep_timeout")) return kSweepTimeout;
    if (!std::strcmp(v, "sort_timeout")) return kSortTimeout;
    return kNoFault;
}
// Applied after the header is cleared: the tile counters that skip tile 0.
cudaError_t inject_fault(char* ws, const Layout& L, cudaStream_t st) {
    const int f = fault_from_env();
    cudaError_t e = cudaSuccess;
    if (f == kSweepTimeout) e = cudaMemsetAsync(ws + L.header + 64, 1, 1, st);  // forward sweep counter = 1
    if (f == kSortTimeout)
        for (int d = 0; d < kPrefixDigits && e == cudaSuccess; ++d)  // each prefix pass's counter = 1
            e = cudaMemsetAsync(ws + L.sort_aux + offsetof(PrefixPlan, pass_ctr) + 4 * d, 1, 1, st);
    return e;
}

SortArgs sort_args(const double* x, int64_t M, const double* y, int64_t N, char* ws, const Layout& L) {
    SortArgs a;
    a.x = x;
    a.y = y;
    a.N = N;
    a.M = M;
    a.Ppad = L.Ppad;
    a.pplan = reinterpret_cast<PrefixPlan*>(ws + L.sort_aux);
    a.maps = reinterpret_cast<PrefixMap*>(ws + L.sort_aux + 256);
    a.items = reinterpret_cast<const Item*>(ws + L.items);
    a.B = L.B;
    a.total_tiles = reinterpret_cast<const int64_t*>(ws + L.header + 80);
    a.max_tiles = L.max_tiles;
    a.keysA = reinterpret_cast<uint64_t*>(ws + L.keysA);
    a.keysB = reinterpret_cast<uint64_t*>(ws + L.keysB);
    a.valsA = reinterpret_cast<uint32_t*>(ws + L.valsA);
    a.valsB = reinterpret_cast<uint32_t*>(ws + L.valsB);
    a.pre = reinterpret_cast<uint32_t*>(ws + L.pre);
    a.hist = reinterpret_cast<uint32_t*>(ws + L.hist);
    a.offs = reinterpret_cast<uint32_t*>(ws + L.offs);
    a.plan = reinterpret_cast<SortPlan*>(ws + L.header + 128);
    a.desc = reinterpret_cast<uint64_t*>(ws + L.sort_desc);
    a.desc_stride = (size_t)L.max_tiles * 256;
    a.tile_ctr = reinterpret_cast<uint32_t*>(ws + L.header + 32);
    a.status = reinterpret_cast<uint32_t*>(ws + L.header);
    a.spin_limit = spin_limit_from_env();
    return a;
}

// Host-side constants of the sweep kernels (Taylor coefficients and thresholds).
SweepConsts make_consts(const fgt1d_plan_s& p) {
    SweepConsts c;
    std::memset(&c, 0, sizeof(c));
    c.n_e = p.n_e;
    c.s = 1.0 / std::sqrt(p.delta);
    c.s_f = (float)c.s;
    const double u64 = std::ldexp(1.0, -53), u32 = std::ldexp(1.0, -26), u48 = std::ldexp(1.0, -48);
    auto split = [](double v, float* hl) {
        hl[0] = (float)v;
        hl[1] = (float)(v - (double)hl[0]);
    };
    for (int k = 0; k < p.n_e; ++k) {
        c.tau_re[k] = p.tau_re[k];
        c.tau_im[k] = p.tau_im[k];
        c.w_re[k] = p.w_re[k];
        c.w_im[k] = p.w_im[k];
        // V'_k = -tau_k W_k (the derivative channel multiplies by s per item)
        c.v_re[k] = -(p.tau_re[k] * p.w_re[k] - p.tau_im[k] * p.w_im[k]);
        c.v_im[k] = -(p.tau_re[k] * p.w_im[k] + p.tau_im[k] * p.w_re[k]);
        split(c.w_re[k], c.wd_re[k]);
        split(c.w_im[k], c.wd_im[k]);
        split(c.v_re[k], c.vd_re[k]);
        split(c.v_im[k], c.vd_im[k]);
        c.tauf_re[k] = (float)p.tau_re[k];
        c.tauf_im[k] = (float)p.tau_im[k];
        // (-tau)^j / j!
        long double ar = 1.0L, ai = 0.0L;
        for (int j = 0; j <= kTaylorMax; ++j) {
            c.tc_re[k][j] = (double)ar;
            c.tc_im[k][j] = (double)ai;
            c.tcf_re[k][j] = (float)ar;
            c.tcf_im[k][j] = (float)ai;
            c.tcd_re_hi[k][j] = (float)(double)ar;
            c.tcd_re_lo[k][j] = (float)((double)ar - (double)c.tcd_re_hi[k][j]);
            c.tcd_im_hi[k][j] = (float)(double)ai;
            c.tcd_im_lo[k][j] = (float)((double)ai - (double)c.tcd_im_hi[k][j]);
            long double nr = (ar * -p.tau_re[k] - ai * -p.tau_im[k]) / (j + 1);
            long double ni = (ar * -p.tau_im[k] + ai * -p.tau_re[k]) / (j + 1);
            ar = nr;
            ai = ni;
        }
        // degree d is enough while (|tau| theta)^d / (d+1)! <= u (the unit roundoff): the
        // truncation error of each multiplier stays below u times its first-order term
        // |tau theta|, so along a sweep it cannot accumulate past u sum |tau theta|, i.e.
        // u (|tau| / Re tau) times the decay length, a few tens of ulps.
        const double at = std::hypot(p.tau_re[k], p.tau_im[k]);
        {
            const double th = std::ldexp(1.0, -10) / at;
            uint64_t b;
            std::memcpy(&b, &th, 8);
            c.theta_hyb_lim[k] = (uint32_t)(b >> 32) - 1u;
        }
        {
            double f = 1.0;
            c.theta_split_d[k][0] = 0;
            for (int J = 1; J <= kTaylorMax; ++J) {
                f *= (J + 1);
                const float fs = (float)(std::pow(std::ldexp(f, -28), 1.0 / (J + 1)) / at);
                std::memcpy(&c.theta_split_d[k][J], &fs, 4);
            }
        }
        double fact = 1.0;
        for (int d = 0; d <= kTaylorMax; ++d) {
            fact *= (d + 1);
            if (d == 0) {
                c.theta_hi_lim[k][0] = 0;
                c.theta_hi_lim_f[k][0] = 0;
                c.theta_hi_lim_d[k][0] = 0;
                continue;
            }
            {
                float f48 = (float)(std::pow(fact * u48, 1.0 / d) / at);
                uint32_t b48;
                std::memcpy(&b48, &f48, 4);
                c.theta_hi_lim_d[k][d] = b48 - 1u;
            }
            double th64 = std::pow(fact * u64, 1.0 / d) / at;
            double th32 = std::pow(fact * u32, 1.0 / d) / at;
            uint64_t b64;
            std::memcpy(&b64, &th64, 8);
            c.theta_hi_lim[k][d] = (uint32_t)(b64 >> 32) - 1u;
            float f32 = (float)th32;
            uint32_t b32;
            std::memcpy(&b32, &f32, 4);
            c.theta_hi_lim_f[k][d] = b32 - 1u;
        }
    }
    return c;
}

int cuda_status(cudaError_t e) { return e == cudaSuccess ? FGT1D_OK : FGT1D_ECUDA; }

// Sweep tile shape (threads per 4096-point tile): the plan's explicit choice, else
// 256 x 16 (measured faster on every value-channel workload).
int tile_threads_of(const fgt1d_plan_s& p) { return p.tile_threads ? p.tile_threads : 256; }
// Shape index (0: 128 x 32, 1: 256 x 16) for sweeps with evaluation channels ev.  By
// default the gradient sweeps (ev != 1) of plans with more than five terms run 128 x 32:
// they keep all terms in one group, and at 256 x 16 their scan region would leave one
// tile per SM.
int shape_index(const fgt1d_plan_s& p, int ev = 1) {
    if (!p.tile_threads && ev != 1 && p.n_e > 5) return 0;
    return tile_threads_of(p) == 256 ? 1 : 0;
}

// Where the items come from: one item (M targets, N sources, the plan's delta), or B
// items from device offsets and optional per-item bandwidths.
struct ItemSource {
    int B = 1;
    const int64_t* x_off = nullptr;
    const int64_t* y_off = nullptr;
    const double* delta = nullptr;
};

// Sweep arguments over the sorted keys and codes held in the workspace.
SweepArgs sweep_args(const double* alpha, int64_t N, double* u, double* out2, char* ws, const Layout& L) {
    SweepArgs w;
    w.N = N;
    w.items = reinterpret_cast<const Item*>(ws + L.items);
    w.B = L.B;
    w.total_tiles = reinterpret_cast<const int64_t*>(ws + L.header + 80);
    w.max_tiles = L.max_tiles;
    w.Ppad = L.Ppad;
    w.keysA = reinterpret_cast<const uint64_t*>(ws + L.keysA);
    w.keysB = reinterpret_cast<const uint64_t*>(ws + L.keysB);
    w.valsA = reinterpret_cast<const uint32_t*>(ws + L.valsA);
    w.valsB = reinterpret_cast<const uint32_t*>(ws + L.valsB);
    w.plan = reinterpret_cast<const SortPlan*>(ws + L.header + 128);
    w.alpha = alpha;
    w.mult = L.mult ? reinterpret_cast<double2*>(ws + L.mult) : nullptr;
    w.fwd = ws + L.fwd;
    w.fwd2 = L.fwd2 ? ws + L.fwd2 : nullptr;
    w.u = u;
    w.out2 = out2;
    w.fdesc = reinterpret_cast<TileDesc*>(ws + L.fdesc);
    w.bdesc = reinterpret_cast<TileDesc*>(ws + L.bdesc);
    w.tile_ctr = reinterpret_cast<uint32_t*>(ws + L.header + 64);
    w.status = reinterpret_cast<uint32_t*>(ws + L.header);
    w.spin_limit = spin_limit_from_env();
    return w;
}

// Sort + sweeps for targets x[M], sources y[N] with strengths alpha.  ev selects the
// evaluation channels (1: values into u, 2: derivative into out2); coinc (may be null)
// receives the per-target sums of coincident source strengths.
int run_pipeline(const fgt1d_plan_s& p, const double* x, int64_t M, const double* y, const double* alpha, int64_t N,
                 const ItemSource& src, double* u, double* out2, int ev, double* coinc, char* ws, const Layout& L,
                 cudaStream_t st, cudaEvent_t const* evs = nullptr, bool self = false,
                 cudaEvent_t alpha_ready = nullptr, double* boundary = nullptr) {
    auto rec = [&](int i) { return (evs && evs[i]) ? cudaEventRecord(evs[i], st) : cudaSuccess; };
    cudaError_t e = rec(0);
    if (e == cudaSuccess) e = cudaMemsetAsync(ws, 0, L.zero_end, st);
    if (e == cudaSuccess) e = inject_fault(ws, L, st);
    if (e != cudaSuccess) return FGT1D_ECUDA;
    Item* items = reinterpret_cast<Item*>(ws + L.items);
    int64_t* total_tiles = reinterpret_cast<int64_t*>(ws + L.header + 80);
    uint32_t* status = reinterpret_cast<uint32_t*>(ws + L.header);
    e = src.x_off ? launch_items(src.B, src.x_off, src.y_off, src.delta, p.delta, items, total_tiles, status,
                                 L.max_tiles, M, N, st)
                  : launch_item_single(M, N, p.delta, items, total_tiles, st);
    if (e != cudaSuccess) return FGT1D_ECUDA;
    SortArgs sa = sort_args(x, M, y, N, ws, L);
    e = launch_sort(sa, st);
    if (e == cudaSuccess) e = rec(1);
    // strengths copied on another stream meanwhile (the sort does not read them)
    if (e == cudaSuccess && alpha_ready) e = cudaStreamWaitEvent(st, alpha_ready, 0);
    if (e != cudaSuccess) return FGT1D_ECUDA;
    SweepArgs w = sweep_args(alpha, N, u, out2, ws, L);
    w.self = self ? 1 : 0;
    // gradient sweeps with a coincidence scan to follow: the forward sweep records whether
    // any two merged points share a coordinate (header word at 88, cleared above)
    if (coinc && !self && (ev & 2)) w.ties = reinterpret_cast<uint32_t*>(ws + L.header + 88);
    const bool f32 = (p.flags & FGT1D_FP32) != 0, df = (p.flags & FGT1D_F32X2) != 0;
    SweepConsts c = make_consts(p);
    cudaEvent_t mid = evs ? evs[2] : nullptr;
    if (f32) e = launch_sweeps_f32(w, c, st, mid, ev, shape_index(p, ev));
    else if (df && ev == 1) e = launch_sweeps_df(w, c, st, mid, shape_index(p, ev));
    else e = launch_sweeps_f64(w, c, st, mid, ev, shape_index(p, ev));
    if (e == cudaSuccess) e = rec(3);
    // a segment's boundary record, read before the coincidence scan reuses the descriptors
    if (e == cudaSuccess && boundary) e = launch_segment_boundary(w, M + N, p.n_e, boundary, st);
    if (e == cudaSuccess && coinc) {
        e = cudaMemsetAsync(ws + L.fdesc, 0, L.bdesc - L.fdesc, st);
        if (e == cudaSuccess) e = cudaMemsetAsync(w.tile_ctr, 0, sizeof(uint32_t), st);
        // all zero unless the scan runs (it returns at once when no coordinates coincide)
        if (e == cudaSuccess && w.ties) e = cudaMemsetAsync(coinc, 0, sizeof(double) * (size_t)M, st);
        w.u = coinc;
        if (e == cudaSuccess) e = launch_coincidence(w, c, st);
    }
    return cuda_status(e);
}

// The transform of the point set that the previous run_pipeline on this workspace
// sorted, with the roles of its points exchanged: targets x[M] (its sources), sources
// y[N] (its targets) with strengths alpha.  Its sorted order is kept -- on equal
// coordinates the targets now come first -- and so is its multiplier table when both
// runs use the same sweeps (table_ok: FP64 or double-float entries of the same tile
// shape, prev_ev the previous run's channels).  In the derivative channel a coincident
// source then sits in h- instead of h+; coinc receives, for each target, the total
// strength of the sources at its coordinate (the caller's correction changes sign).
int run_pipeline_swapped(const fgt1d_plan_s& p, const double* x, int64_t M, const double* y, const double* alpha,
                         int64_t N, double* u, double* out2, int ev, double* coinc, int prev_ev, char* ws,
                         const Layout& L, cudaStream_t st) {
    // sweep counters and look-back descriptors; the sort's plan, the equal-coordinate flag
    // and the status stay
    cudaError_t e = cudaMemsetAsync(ws + L.header + 64, 0, 8, st);
    if (e == cudaSuccess) e = cudaMemsetAsync(ws + L.fdesc, 0, L.zero_end - L.fdesc, st);
    Item* items = reinterpret_cast<Item*>(ws + L.items);
    int64_t* total_tiles = reinterpret_cast<int64_t*>(ws + L.header + 80);
    if (e == cudaSuccess) e = launch_item_single(M, N, p.delta, items, total_tiles, st);
    SortArgs sa = sort_args(y, N, x, M, ws, L);  // the previous run's view: targets y, sources x
    if (e == cudaSuccess) e = launch_swap_codes(sa, M + N, M, N, st);
    if (e != cudaSuccess) return FGT1D_ECUDA;
    SweepArgs w = sweep_args(alpha, N, u, out2, ws, L);
    if (coinc && (ev & 2)) w.ties = reinterpret_cast<uint32_t*>(ws + L.header + 88);  // set by the previous run
    const bool f32 = (p.flags & FGT1D_FP32) != 0, df = (p.flags & FGT1D_F32X2) != 0;
    const bool df_sweeps = df && ev == 1, prev_df = df && prev_ev == 1;
    const int shape = shape_index(p, prev_ev);
    w.reuse = (!f32 && df_sweeps == prev_df) ? 1 : 0;
    SweepConsts c = make_consts(p);
    if (f32) e = launch_sweeps_f32(w, c, st, nullptr, ev, shape);
    else if (df_sweeps) e = launch_sweeps_df(w, c, st, nullptr, shape);
    else e = launch_sweeps_f64(w, c, st, nullptr, ev, shape);
    if (e == cudaSuccess && coinc && w.ties) {
        // sums over sorted positions (every point evaluated), then each target takes its
        // run's total; the forward partial sums are free again
        double* F = reinterpret_cast<double*>(ws + L.fwd);
        e = cudaMemsetAsync(ws + L.fdesc, 0, L.bdesc - L.fdesc, st);
        if (e == cudaSuccess) e = cudaMemsetAsync(w.tile_ctr, 0, sizeof(uint32_t), st);
        if (e == cudaSuccess) e = cudaMemsetAsync(coinc, 0, sizeof(double) * (size_t)M, st);
        SweepArgs wc = w;
        wc.self = 1;
        wc.u = F;
        if (e == cudaSuccess) e = launch_coincidence(wc, c, st);
        if (e == cudaSuccess) e = launch_coinc_gather(w, F, M + N, coinc, st);
    }
    return cuda_status(e);
}

int run_transform(const fgt1d_plan_s& p, const double* x, int64_t M, const double* y, const double* alpha, int64_t N,
                  double* u, char* ws, const Layout& L, cudaStream_t st, cudaEvent_t const* evs = nullptr,
                  cudaEvent_t alpha_ready = nullptr) {
    if (M == 0) return FGT1D_OK;
    if (N == 0) return cuda_status(cudaMemsetAsync(u, 0, sizeof(double) * (size_t)M, st));
    if (!(p.flags & FGT1D_EXACT_SELF))
        return run_pipeline(p, x, M, y, alpha, N, ItemSource(), u, nullptr, 1, nullptr, ws, L, st, evs, false,
                            alpha_ready);
    // coincident pairs: add (1 - S_n(0)) times the coincident source strengths
    double* A = reinterpret_cast<double*>(ws + L.coinc);
    int r = run_pipeline(p, x, M, y, alpha, N, ItemSource(), u, nullptr, 1, A, ws, L, st, evs, false, alpha_ready);
    if (r) return r;
    double s0 = 0.0;
    for (int k = 0; k < p.n_e; ++k) s0 += p.w_re[k];
    return cuda_status(launch_axpy(A, 1.0 - s0, M, u, st));
}

// A segment of a range-partitioned transform: the transform of its own points with zero
// entering states (every size, so that a segment without targets still reports its
// sources' boundary states), plus its boundary record.
int run_segment(const fgt1d_plan_s& p, const double* x, int64_t M, const double* y, const double* alpha, int64_t N,
                double* u, double* boundary, char* ws, const Layout& L, cudaStream_t st) {
    if (!(p.flags & FGT1D_EXACT_SELF) || M == 0 || N == 0)
        return run_pipeline(p, x, M, y, alpha, N, ItemSource(), u, nullptr, 1, nullptr, ws, L, st, nullptr, false,
                            nullptr, boundary);
    double* A = reinterpret_cast<double*>(ws + L.coinc);
    int r = run_pipeline(p, x, M, y, alpha, N, ItemSource(), u, nullptr, 1, A, ws, L, st, nullptr, false, nullptr,
                         boundary);
    if (r) return r;
    double s0 = 0.0;
    for (int k = 0; k < p.n_e; ++k) s0 += p.w_re[k];
    return cuda_status(launch_axpy(A, 1.0 - s0, M, u, st));
}

}  // namespace

int run_transform_in(const fgt1d_plan_s& p, const double* x, int64_t M, const double* y, const double* alpha,
                     int64_t N, double* u, void* ws, size_t ws_bytes, cudaStream_t st) {
    if (!sizes_ok(M, N)) return FGT1D_EINVAL;
    Layout L = make_layout(M, N, 1, p.n_e, p.flags, true, false);
    if (M > 0 && N > 0) {
        int r = ws_ok(ws, ws_bytes, L);
        if (r) return r;
    }
    return run_transform(p, x, M, y, alpha, N, u, static_cast<char*>(ws), L, st);
}

size_t transform_workspace_bytes(const fgt1d_plan_s& p, int64_t M, int64_t N) {
    return make_layout(M, N, 1, p.n_e, p.flags, true, false).total;
}

}  // namespace fgt1d

using namespace fgt1d;

extern "C" int fgt1d_workspace_size(fgt1d_plan plan, int64_t M, int64_t N, size_t* bytes) {
    if (!plan || !bytes || !sizes_ok(M, N)) return FGT1D_EINVAL;
    *bytes = make_layout(M, N, 1, plan->n_e, plan->flags, true, false).total;
    return FGT1D_OK;
}

extern "C" int fgt1d_workspace_size_host(fgt1d_plan plan, int64_t M, int64_t N, size_t* bytes) {
    if (!plan || !bytes || !sizes_ok(M, N)) return FGT1D_EINVAL;
    *bytes = make_layout(M, N, 1, plan->n_e, plan->flags, true, true).total;
    return FGT1D_OK;
}

extern "C" int fgt1d_sort_workspace_size(int64_t M, int64_t N, size_t* bytes) {
    if (!bytes || !sizes_ok(M, N)) return FGT1D_EINVAL;
    *bytes = make_layout(M, N, 1, 1, FGT1D_FP64, false, false).total;
    return FGT1D_OK;
}

extern "C" int fgt1d_execute(fgt1d_plan plan, const double* x, int64_t M, const double* y, const double* alpha,
                             int64_t N, double* u, void* workspace, size_t ws_bytes, fgt1d_stream stream) {
    if (!plan || !sizes_ok(M, N)) return FGT1D_EINVAL;
    if (M > 0 && (!x || !u)) return FGT1D_EINVAL;
    if (N > 0 && M > 0 && (!y || !alpha)) return FGT1D_EINVAL;
    Layout L = make_layout(M, N, 1, plan->n_e, plan->flags, true, false);
    if (M > 0 && N > 0) {
        int r = ws_ok(workspace, ws_bytes, L);
        if (r) return r;
    }
    return run_transform(*plan, x, M, y, alpha, N, u, static_cast<char*>(workspace), L,
                         static_cast<cudaStream_t>(stream));
}

extern "C" int fgt1d_execute_profiled(fgt1d_plan plan, const double* x, int64_t M, const double* y,
                                      const double* alpha, int64_t N, double* u, void* workspace, size_t ws_bytes,
                                      fgt1d_stream stream, void* const* events) {
    if (!plan || !sizes_ok(M, N) || !events) return FGT1D_EINVAL;
    if (M > 0 && (!x || !u)) return FGT1D_EINVAL;
    if (N > 0 && M > 0 && (!y || !alpha)) return FGT1D_EINVAL;
    Layout L = make_layout(M, N, 1, plan->n_e, plan->flags, true, false);
    if (M > 0 && N > 0) {
        int r = ws_ok(workspace, ws_bytes, L);
        if (r) return r;
    }
    return run_transform(*plan, x, M, y, alpha, N, u, static_cast<char*>(workspace), L,
                         static_cast<cudaStream_t>(stream), reinterpret_cast<cudaEvent_t const*>(events));
}

extern "C" int fgt1d_batched_workspace_size(fgt1d_plan plan, int B, int64_t M_total, int64_t N_total,
                                            size_t* bytes) {
    if (!plan || !bytes || B < 1 || !sizes_ok(M_total, N_total)) return FGT1D_EINVAL;
    if ((M_total + N_total + kTile - 1) / kTile + (B - 1) > (int64_t(1) << 31) / kTile) return FGT1D_EINVAL;
    *bytes = make_layout(M_total, N_total, B, plan->n_e, plan->flags, true, false).total;
    return FGT1D_OK;
}

extern "C" int fgt1d_execute_batched(fgt1d_plan plan, int B, const int64_t* x_off, const int64_t* y_off,
                                     const double* delta, const double* x, int64_t M_total, const double* y,
                                     const double* alpha, int64_t N_total, double* u, void* workspace,
                                     size_t ws_bytes, fgt1d_stream stream) {
    if (!plan || B < 1 || !x_off || !y_off || !sizes_ok(M_total, N_total)) return FGT1D_EINVAL;
    if ((M_total > 0 && (!x || !u)) || (N_total > 0 && (!y || !alpha))) return FGT1D_EINVAL;
    if ((M_total + N_total + kTile - 1) / kTile + (B - 1) > (int64_t(1) << 31) / kTile) return FGT1D_EINVAL;
    Layout L = make_layout(M_total, N_total, B, plan->n_e, plan->flags, true, false);
    int r = ws_ok(workspace, ws_bytes, L);
    if (r) return r;
    ItemSource src;
    src.B = B;
    src.x_off = x_off;
    src.y_off = y_off;
    src.delta = delta;
    return run_pipeline(*plan, x, M_total, y, alpha, N_total, src, u, nullptr, 1, nullptr,
                        static_cast<char*>(workspace), L, static_cast<cudaStream_t>(stream));
}

extern "C" int fgt1d_backward_workspace_size(fgt1d_plan plan, int64_t M, int64_t N, size_t* bytes) {
    if (!plan || !bytes || !sizes_ok(M, N)) return FGT1D_EINVAL;
    *bytes = make_layout(M, N, 1, plan->n_e, plan->flags, true, false, true).total;
    return FGT1D_OK;
}

extern "C" int fgt1d_backward(fgt1d_plan plan, const double* x, int64_t M, const double* y, const double* alpha,
                              int64_t N, const double* grad_u, double* grad_x, double* grad_y, double* grad_alpha,
                              double* grad_delta, void* workspace, size_t ws_bytes, fgt1d_stream stream) {
    if (!plan || !sizes_ok(M, N)) return FGT1D_EINVAL;
    if ((M > 0 && (!x || !grad_u)) || (N > 0 && (!y || !alpha))) return FGT1D_EINVAL;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    if (M == 0 || N == 0) {  // no pair interacts: every gradient is zero
        cudaError_t e = cudaSuccess;
        if (grad_x && M) e = cudaMemsetAsync(grad_x, 0, sizeof(double) * (size_t)M, st);
        if (e == cudaSuccess && grad_y && N) e = cudaMemsetAsync(grad_y, 0, sizeof(double) * (size_t)N, st);
        if (e == cudaSuccess && grad_alpha && N) e = cudaMemsetAsync(grad_alpha, 0, sizeof(double) * (size_t)N, st);
        if (e == cudaSuccess && grad_delta) e = cudaMemsetAsync(grad_delta, 0, sizeof(double), st);
        return cuda_status(e);
    }
    Layout L = make_layout(M, N, 1, plan->n_e, plan->flags, true, false, true);
    int r = ws_ok(workspace, ws_bytes, L);
    if (r) return r;
    char* ws = static_cast<char*>(workspace);
    double sumV = 0.0;
    {
        SweepConsts c = make_consts(*plan);
        for (int k = 0; k < plan->n_e; ++k) sumV += c.v_re[k];
        sumV *= c.s;  // the derivative channel carries s = 1/sqrt(delta)
    }
    double* D = reinterpret_cast<double*>(ws + L.gD);
    double* A = reinterpret_cast<double*>(ws + L.gA);
    double* gx = grad_x ? grad_x : reinterpret_cast<double*>(ws + L.gx);
    double* gy = grad_y ? grad_y : reinterpret_cast<double*>(ws + L.gy);
    const bool need_x = grad_x || grad_delta, need_y = grad_y || grad_delta, need_a = grad_alpha != nullptr;
    if (need_x) {
        // targets x, sources y, strengths alpha: D_i = Re sum V (h+ - h-), A_i coincident sums
        r = run_pipeline(*plan, x, M, y, alpha, N, ItemSource(), nullptr, D, 2, A, ws, L, st);
        if (r) return r;
        if (launch_grad_assemble(grad_u, D, A, sumV, M, gx, st) != cudaSuccess) return FGT1D_ECUDA;
    }
    if (need_a || need_y) {
        // targets y, sources x, strengths grad_u: values -> dL/dalpha, derivative -> dL/dy / alpha.
        // After the first transform the same points are sorted already (and its multipliers
        // tabulated): their order is kept, with coincident sources after their targets, so
        // the coincidence correction changes sign
        const int ev = (need_a ? 1 : 0) | (need_y ? 2 : 0);
        double sign = 1.0;
        if (need_x) {
            r = run_pipeline_swapped(*plan, y, N, x, grad_u, M, grad_alpha, need_y ? D : nullptr, ev,
                                     need_y ? A : nullptr, 2, ws, L, st);
            sign = -1.0;
        } else {
            r = run_pipeline(*plan, y, N, x, grad_u, M, ItemSource(), grad_alpha, need_y ? D : nullptr, ev,
                             need_y ? A : nullptr, ws, L, st);
        }
        if (r) return r;
        if (need_y && launch_grad_assemble(alpha, D, A, sign * sumV, N, gy, st) != cudaSuccess) return FGT1D_ECUDA;
    }
    if (grad_delta) {
        if (launch_grad_delta(x, gx, M, y, gy, N, plan->delta, reinterpret_cast<double*>(ws + L.parts), kGradPartials,
                              grad_delta, st) != cudaSuccess)
            return FGT1D_ECUDA;
    }
    return FGT1D_OK;
}

namespace fgt1d {
namespace {

// fgt1d_execute_host and its asynchronous form: copies in, the transform, the copy out;
// with sync the stream is synchronised and the device status returned.
int execute_host(fgt1d_plan plan, const double* x_host, int64_t M, const double* y_host, const double* alpha_host,
                 int64_t N, double* u_host, void* workspace, size_t ws_bytes, fgt1d_stream stream, bool sync) {
    if (!plan || !sizes_ok(M, N)) return FGT1D_EINVAL;
    if (M > 0 && (!x_host || !u_host)) return FGT1D_EINVAL;
    if (N > 0 && M > 0 && (!y_host || !alpha_host)) return FGT1D_EINVAL;
    if (M == 0) return FGT1D_OK;
    if (N == 0) {
        std::memset(u_host, 0, sizeof(double) * (size_t)M);
        return FGT1D_OK;
    }
    Layout L = make_layout(M, N, 1, plan->n_e, plan->flags, true, true);
    int r = ws_ok(workspace, ws_bytes, L);
    if (r) return r;
    char* ws = static_cast<char*>(workspace);
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    double* dx = reinterpret_cast<double*>(ws + L.hx);
    double* dy = reinterpret_cast<double*>(ws + L.hy);
    double* da = reinterpret_cast<double*>(ws + L.ha);
    double* du = reinterpret_cast<double*>(ws + L.hu);
    // coordinates on the caller's stream; the strengths on a second stream, overlapping
    // the sort, which does not read them
    cudaStream_t s2 = nullptr;
    cudaEvent_t ev_in = nullptr, ev_alpha = nullptr;
    auto release = [&]() {
        if (ev_in) cudaEventDestroy(ev_in);
        if (ev_alpha) cudaEventDestroy(ev_alpha);
        if (s2) cudaStreamDestroy(s2);
    };
    if (cudaStreamCreateWithFlags(&s2, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&ev_in, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&ev_alpha, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventRecord(ev_in, st) != cudaSuccess || cudaStreamWaitEvent(s2, ev_in, 0) != cudaSuccess ||
        cudaMemcpyAsync(da, alpha_host, sizeof(double) * (size_t)N, cudaMemcpyHostToDevice, s2) != cudaSuccess ||
        cudaEventRecord(ev_alpha, s2) != cudaSuccess ||
        cudaMemcpyAsync(dx, x_host, sizeof(double) * (size_t)M, cudaMemcpyHostToDevice, st) != cudaSuccess ||
        cudaMemcpyAsync(dy, y_host, sizeof(double) * (size_t)N, cudaMemcpyHostToDevice, st) != cudaSuccess) {
        release();
        return FGT1D_ECUDA;
    }
    r = run_transform(*plan, dx, M, dy, da, N, du, ws, L, st, nullptr, ev_alpha);
    if (r) {
        cudaStreamSynchronize(s2);
        release();
        return r;
    }
    release();  // the stream and events go once their work is done
    if (cudaMemcpyAsync(u_host, du, sizeof(double) * (size_t)M, cudaMemcpyDeviceToHost, st) != cudaSuccess)
        return FGT1D_ECUDA;
    return sync ? fgt1d_check(workspace, ws_bytes, stream) : FGT1D_OK;
}

}  // namespace
}  // namespace fgt1d

extern "C" int fgt1d_execute_host(fgt1d_plan plan, const double* x_host, int64_t M, const double* y_host,
                                  const double* alpha_host, int64_t N, double* u_host, void* workspace,
                                  size_t ws_bytes, fgt1d_stream stream) {
    return execute_host(plan, x_host, M, y_host, alpha_host, N, u_host, workspace, ws_bytes, stream, true);
}

extern "C" int fgt1d_execute_host_async(fgt1d_plan plan, const double* x_host, int64_t M, const double* y_host,
                                        const double* alpha_host, int64_t N, double* u_host, void* workspace,
                                        size_t ws_bytes, fgt1d_stream stream) {
    return execute_host(plan, x_host, M, y_host, alpha_host, N, u_host, workspace, ws_bytes, stream, false);
}

extern "C" int fgt1d_sort_merged(const double* x, int64_t M, const double* y, int64_t N, uint32_t* perm,
                                 void* workspace, size_t ws_bytes, fgt1d_stream stream) {
    if (!sizes_ok(M, N)) return FGT1D_EINVAL;
    if ((M > 0 && !x) || (N > 0 && !y) || (M + N > 0 && !perm)) return FGT1D_EINVAL;
    if (M + N == 0) return FGT1D_OK;
    Layout L = make_layout(M, N, 1, 1, FGT1D_FP64, false, false);
    int r = ws_ok(workspace, ws_bytes, L);
    if (r) return r;
    char* ws = static_cast<char*>(workspace);
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    if (cudaMemsetAsync(ws, 0, L.zero_end, st) != cudaSuccess) return FGT1D_ECUDA;
    if (launch_item_single(M, N, 1.0, reinterpret_cast<Item*>(ws + L.items),
                           reinterpret_cast<int64_t*>(ws + L.header + 80), st) != cudaSuccess)
        return FGT1D_ECUDA;
    SortArgs sa = sort_args(x, M, y, N, ws, L);
    if (launch_sort(sa, st) != cudaSuccess) return FGT1D_ECUDA;
    return cuda_status(launch_copy_perm(sa, M + N, perm, st));
}

// ---- identical targets and sources --------------------------------------------------------
extern "C" int fgt1d_self_workspace_size(fgt1d_plan plan, int64_t N, size_t* bytes) {
    if (!plan || !bytes || !sizes_ok(0, N)) return FGT1D_EINVAL;
    if (plan->flags & FGT1D_F32X2) return FGT1D_EUNSUPPORTED;
    *bytes = make_layout(0, N, 1, plan->n_e, plan->flags, true, false).total;
    return FGT1D_OK;
}

extern "C" int fgt1d_execute_self(fgt1d_plan plan, const double* x, int64_t N, const double* alpha, double* u,
                                  void* workspace, size_t ws_bytes, fgt1d_stream stream) {
    if (!plan || !sizes_ok(0, N)) return FGT1D_EINVAL;
    if (plan->flags & FGT1D_F32X2) return FGT1D_EUNSUPPORTED;
    if (N == 0) return FGT1D_OK;
    if (!x || !alpha || !u) return FGT1D_EINVAL;
    Layout L = make_layout(0, N, 1, plan->n_e, plan->flags, true, false);
    int r = ws_ok(workspace, ws_bytes, L);
    if (r) return r;
    char* ws = static_cast<char*>(workspace);
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    // the N points are merged once, as sources; the sweeps treat each as a target too
    r = run_pipeline(*plan, nullptr, 0, x, alpha, N, ItemSource(), u, nullptr, 1, nullptr, ws, L, st, nullptr, true);
    if (r || !(plan->flags & FGT1D_EXACT_SELF)) return r;
    // exact self term: add (1 - S_n(0)) times the total strength of each point's run of
    // equal coordinates (the point itself included).  The coincidence sweep leaves the
    // running run sums in sorted order over the forward partial sums, which are spent.
    double* F = reinterpret_cast<double*>(ws + L.fwd);
    SweepArgs w = sweep_args(alpha, N, F, nullptr, ws, L);
    w.self = 1;
    cudaError_t e = cudaMemsetAsync(ws + L.fdesc, 0, L.bdesc - L.fdesc, st);
    if (e == cudaSuccess) e = cudaMemsetAsync(w.tile_ctr, 0, sizeof(uint32_t), st);
    if (e == cudaSuccess) e = launch_coincidence(w, make_consts(*plan), st);
    double s0 = 0.0;
    for (int k = 0; k < plan->n_e; ++k) s0 += plan->w_re[k];
    if (e == cudaSuccess) e = launch_self_exact(w, F, N, 1.0 - s0, u, st);
    return cuda_status(e);
}

// ---- fixed geometry: bind once, apply many strength vectors ------------------------------
namespace {

constexpr size_t kTagOffset = 96;  // geometry tag in the workspace header

// Identifies what a bound table depends on: sizes, delta and the nodes tau_k.
uint64_t geometry_tag(const fgt1d_plan_s& p, int64_t M, int64_t N) {
    uint64_t h = 0xcbf29ce484222325ull;  // FNV-1a over the raw bytes
    auto mix = [&](const void* v, size_t n) {
        const unsigned char* b = static_cast<const unsigned char*>(v);
        for (size_t i = 0; i < n; ++i) {
            h ^= b[i];
            h *= 0x100000001b3ull;
        }
    };
    const uint64_t magic = 0x6667743167656f6dull;
    mix(&magic, 8);
    mix(&M, 8);
    mix(&N, 8);
    mix(&p.n_e, sizeof(p.n_e));
    mix(&p.delta, 8);
    mix(p.tau_re, sizeof(double) * (size_t)p.n_e);
    mix(p.tau_im, sizeof(double) * (size_t)p.n_e);
    const int shape = shape_index(p);  // the table layout follows the tile shape
    mix(&shape, sizeof(shape));
    const unsigned prec = p.flags & (FGT1D_F32X2 | FGT1D_FP32);  // and its entries the precision
    mix(&prec, sizeof(prec));
    return h;
}

int geometry_checks(fgt1d_plan plan, int64_t M, int64_t N, void* ws, size_t ws_bytes, Layout& L) {
    if (!plan || !sizes_ok(M, N)) return FGT1D_EINVAL;
    L = make_layout(M, N, 1, plan->n_e, plan->flags, true, false);
    if (M > 0 && N > 0) return ws_ok(ws, ws_bytes, L);
    return FGT1D_OK;
}

}  // namespace

extern "C" int fgt1d_geometry_workspace_size(fgt1d_plan plan, int64_t M, int64_t N, size_t* bytes) {
    if (!bytes) return FGT1D_EINVAL;
    Layout L;
    int r = geometry_checks(plan, M, N, nullptr, 0, L);
    if (r && r != FGT1D_EWORKSPACE) return r;
    *bytes = L.total;
    return FGT1D_OK;
}

extern "C" int fgt1d_geometry_bind(fgt1d_plan plan, const double* x, int64_t M, const double* y, int64_t N,
                                   void* workspace, size_t ws_bytes, fgt1d_stream stream) {
    Layout L;
    int r = geometry_checks(plan, M, N, workspace, ws_bytes, L);
    if (r) return r;
    if (M == 0 || N == 0) return FGT1D_OK;
    if (!x || !y) return FGT1D_EINVAL;
    char* ws = static_cast<char*>(workspace);
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    cudaError_t e = cudaMemsetAsync(ws, 0, L.zero_end, st);
    int64_t* total_tiles = reinterpret_cast<int64_t*>(ws + L.header + 80);
    if (e == cudaSuccess)
        e = launch_item_single(M, N, plan->delta, reinterpret_cast<Item*>(ws + L.items), total_tiles, st);
    SortArgs sa = sort_args(x, M, y, N, ws, L);
    if (e == cudaSuccess) e = launch_sort(sa, st);
    SweepArgs w = sweep_args(nullptr, N, nullptr, nullptr, ws, L);
    SweepConsts c = make_consts(*plan);
    // FP32 plans keep the sorted points only: their sweeps recompute a multiplier with a
    // few FP32 multiply-adds, fewer cycles than reading a stored entry from HBM
    if (e == cudaSuccess && !(plan->flags & FGT1D_FP32))
        e = launch_fill_table(w, c, shape_index(*plan), (plan->flags & FGT1D_F32X2) != 0, st);
    if (e == cudaSuccess)
        e = launch_geometry_tag(reinterpret_cast<uint64_t*>(ws + L.header + kTagOffset), geometry_tag(*plan, M, N), st);
    return cuda_status(e);
}

extern "C" int fgt1d_geometry_apply(fgt1d_plan plan, int64_t M, int64_t N, const double* alpha, double* u,
                                    void* workspace, size_t ws_bytes, fgt1d_stream stream) {
    Layout L;
    int r = geometry_checks(plan, M, N, workspace, ws_bytes, L);
    if (r) return r;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    if (M == 0) return FGT1D_OK;
    if (!u) return FGT1D_EINVAL;
    if (N == 0) return cuda_status(cudaMemsetAsync(u, 0, sizeof(double) * (size_t)M, st));
    if (!alpha) return FGT1D_EINVAL;
    char* ws = static_cast<char*>(workspace);
    const fgt1d_plan_s& p = *plan;
    // per-apply state: sweep tile counters and look-back descriptors (the sorted points,
    // the item table and the multiplier table stay)
    cudaError_t e = cudaMemsetAsync(ws + L.header + 64, 0, 8, st);
    if (e == cudaSuccess) e = cudaMemsetAsync(ws + L.fdesc, 0, L.zero_end - L.fdesc, st);
    int64_t* total_tiles = reinterpret_cast<int64_t*>(ws + L.header + 80);
    uint32_t* status = reinterpret_cast<uint32_t*>(ws + L.header);
    if (e == cudaSuccess)
        e = launch_geometry_check(reinterpret_cast<const uint64_t*>(ws + L.header + kTagOffset),
                                  geometry_tag(p, M, N), total_tiles, status, st);
    SweepArgs w = sweep_args(alpha, N, u, nullptr, ws, L);
    w.reuse = (p.flags & FGT1D_FP32) ? 0 : 1;
    SweepConsts c = make_consts(p);
    if (e == cudaSuccess) {
        if (p.flags & FGT1D_FP32) e = launch_sweeps_f32(w, c, st, nullptr, 1, shape_index(p));
        else if (p.flags & FGT1D_F32X2) e = launch_sweeps_df(w, c, st, nullptr, shape_index(p));
        else e = launch_sweeps_f64(w, c, st, nullptr, 1, shape_index(p));
    }
    if (e == cudaSuccess && (p.flags & FGT1D_EXACT_SELF)) {
        double* A = reinterpret_cast<double*>(ws + L.coinc);
        e = cudaMemsetAsync(ws + L.fdesc, 0, L.bdesc - L.fdesc, st);
        if (e == cudaSuccess) e = cudaMemsetAsync(w.tile_ctr, 0, sizeof(uint32_t), st);
        w.u = A;
        w.reuse = 0;
        if (e == cudaSuccess) e = launch_coincidence(w, c, st);
        double s0 = 0.0;
        for (int k = 0; k < p.n_e; ++k) s0 += p.w_re[k];
        if (e == cudaSuccess) e = launch_axpy(A, 1.0 - s0, M, u, st);
    }
    return cuda_status(e);
}

extern "C" int fgt1d_plan_set_tile(fgt1d_plan plan, int threads) {
    if (!plan || (threads != 0 && threads != 128 && threads != 256)) return FGT1D_EINVAL;
    plan->tile_threads = threads;
    return FGT1D_OK;
}

extern "C" int fgt1d_plan_get_tile(fgt1d_plan plan, int* threads) {
    if (!plan || !threads) return FGT1D_EINVAL;
    *threads = tile_threads_of(*plan);
    return FGT1D_OK;
}

namespace fgt1d {
namespace {

// Autotuner cache (FGT1D_TUNE_CACHE names a text file, one choice per line:
// "<precision> <n_e> <log2 of M_total + N_total> <batched> <threads> <ms>").  A line
// matching the workload's key gives the tile shape without timing; a timed choice is
// appended.  The file belongs to one GPU model.
struct TuneKey {
    unsigned prec;
    int n_e, lg, batched;
};
TuneKey tune_key(const fgt1d_plan_s& p, int64_t P, bool batched) {
    int lg = 0;
    while (lg < 62 && (int64_t(1) << (lg + 1)) <= P) ++lg;
    return TuneKey{p.flags & (FGT1D_FP32 | FGT1D_F32X2), p.n_e, lg, batched ? 1 : 0};
}
int tune_cache_lookup(const TuneKey& k) {
    const char* path = std::getenv("FGT1D_TUNE_CACHE");
    if (!path || !*path) return 0;
    FILE* f = std::fopen(path, "r");
    if (!f) return 0;
    unsigned prec;
    int ne, lg, b, t;
    double ms;
    int found = 0;
    char line[256];
    while (!found && std::fgets(line, sizeof(line), f))
        if (std::sscanf(line, "%u %d %d %d %d %lf", &prec, &ne, &lg, &b, &t, &ms) == 6 && prec == k.prec &&
            ne == k.n_e && lg == k.lg && b == k.batched && (t == 128 || t == 256))
            found = t;
    std::fclose(f);
    return found;
}
void tune_cache_store(const TuneKey& k, int threads, float ms) {
    const char* path = std::getenv("FGT1D_TUNE_CACHE");
    if (!path || !*path) return;
    FILE* f = std::fopen(path, "a");
    if (!f) return;
    std::fprintf(f, "%u %d %d %d %d %.4f\n", k.prec, k.n_e, k.lg, k.batched, threads, (double)ms);
    std::fclose(f);
}

}  // namespace
}  // namespace fgt1d

extern "C" int fgt1d_autotune(fgt1d_plan plan, int B, const int64_t* x_off, const int64_t* y_off, const double* delta,
                              const double* x, int64_t M_total, const double* y, const double* alpha, int64_t N_total,
                              double* u, void* workspace, size_t ws_bytes, int reps, fgt1d_stream stream,
                              int* threads_out, float* ms_out) {
    static const int kCandidates[kNumShapes] = {128, 256};
    if (!plan || reps < 1 || B < 1 || (!x_off && B != 1) || !sizes_ok(M_total, N_total)) return FGT1D_EINVAL;
    if (ms_out)
        for (int i = 0; i < kNumShapes; ++i) ms_out[i] = -1.f;
    const int prev = plan->tile_threads;
    auto done = [&](int t) {
        plan->tile_threads = t;
        if (threads_out) *threads_out = tile_threads_of(*plan);
        return FGT1D_OK;
    };
    if (const char* env = std::getenv("FGT1D_TILE_THREADS")) {
        const int t = std::atoi(env);
        if (t == 128 || t == 256) return done(t);
    }
    if (M_total == 0 || N_total == 0) return done(prev);  // nothing runs on the device
    const TuneKey key = tune_key(*plan, M_total + N_total, x_off != nullptr);
    if (const int cached = tune_cache_lookup(key)) return done(cached);
    auto run = [&]() {
        return x_off ? fgt1d_execute_batched(plan, B, x_off, y_off, delta, x, M_total, y, alpha, N_total, u, workspace,
                                             ws_bytes, stream)
                     : fgt1d_execute(plan, x, M_total, y, alpha, N_total, u, workspace, ws_bytes, stream);
    };
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
        if (e0) cudaEventDestroy(e0);
        return FGT1D_ECUDA;
    }
    int r = FGT1D_OK, best = 0;
    float best_ms = 0.f;
    for (int i = 0; i < kNumShapes && r == FGT1D_OK; ++i) {
        plan->tile_threads = kCandidates[i];
        r = run();  // untimed: first-use costs (kernel attributes, caches)
        if (r == FGT1D_OK) r = fgt1d_check(workspace, ws_bytes, stream);
        if (r == FGT1D_OK && cudaEventRecord(e0, st) != cudaSuccess) r = FGT1D_ECUDA;
        for (int k = 0; k < reps && r == FGT1D_OK; ++k) r = run();
        if (r == FGT1D_OK && cudaEventRecord(e1, st) != cudaSuccess) r = FGT1D_ECUDA;
        if (r == FGT1D_OK) r = fgt1d_check(workspace, ws_bytes, stream);
        float ms = 0.f;
        if (r == FGT1D_OK && cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess) r = FGT1D_ECUDA;
        ms /= (float)reps;
        if (r == FGT1D_OK) {
            if (ms_out) ms_out[i] = ms;
            if (i == 0 || ms < best_ms) {
                best_ms = ms;
                best = kCandidates[i];
            }
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (r != FGT1D_OK) {
        plan->tile_threads = prev;
        return r;
    }
    tune_cache_store(key, best, best_ms);
    return done(best);
}

// ---- range partition: segments of one transform ------------------------------------------
extern "C" int fgt1d_segment_execute(fgt1d_plan plan, const double* x, int64_t M, const double* y,
                                     const double* alpha, int64_t N, double* u, double* boundary, void* workspace,
                                     size_t ws_bytes, fgt1d_stream stream) {
    if (!plan || !sizes_ok(M, N) || !boundary) return FGT1D_EINVAL;
    if (M > 0 && (!x || !u)) return FGT1D_EINVAL;
    if (N > 0 && (!y || !alpha)) return FGT1D_EINVAL;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    if (M + N == 0) {  // no points: the empty record, and a clean status for fgt1d_check
        cudaError_t e = launch_segment_empty(plan->n_e, boundary, st);
        if (e == cudaSuccess && workspace && ws_bytes >= sizeof(uint32_t))
            e = cudaMemsetAsync(workspace, 0, sizeof(uint32_t), st);
        return cuda_status(e);
    }
    Layout L = make_layout(M, N, 1, plan->n_e, plan->flags, true, false);
    int r = ws_ok(workspace, ws_bytes, L);
    if (r) return r;
    return run_segment(*plan, x, M, y, alpha, N, u, boundary, static_cast<char*>(workspace), L, st);
}

extern "C" int fgt1d_segment_compose(fgt1d_plan plan, int G, int g, const double* boundaries, double* carry) {
    if (!plan || G < 1 || g < 0 || g >= G || !boundaries || !carry) return FGT1D_EINVAL;
    const int n = plan->n_e;
    const size_t stride = 4 * (size_t)n + 2;
    const double s = 1.0 / std::sqrt(plan->delta);
    // the segments must be ordered along the line: z_first <= z_last, and each segment
    // starts at or after the previous non-empty one ends
    double last = -INFINITY;
    for (int j = 0; j < G; ++j) {
        const double* b = boundaries + (size_t)j * stride;
        const double zf = b[4 * n], zl = b[4 * n + 1];
        if (std::isnan(zf) != std::isnan(zl)) return FGT1D_EINVAL;
        if (std::isnan(zf)) continue;
        if (!(zf <= zl) || !(last <= zf)) return FGT1D_EINVAL;
        for (int i = 0; i < 4 * n; ++i)
            if (!std::isfinite(b[i])) return FGT1D_EINVAL;
        last = zl;
    }
    // span multiplier exp(-tau_k s d), d >= 0, computed directly from two coordinates
    auto decay = [&](int k, double d, double& er, double& ei) {
        const double mag = std::exp(-plan->tau_re[k] * s * d), ang = plan->tau_im[k] * s * d;
        er = mag * std::cos(ang);
        ei = -mag * std::sin(ang);
    };
    const double nan = std::numeric_limits<double>::quiet_NaN();
    for (int k = 0; k < n; ++k) {
        // forward: the state at the last point of the segments before g
        double Fr = 0.0, Fi = 0.0, zl = nan;
        for (int j = 0; j < g; ++j) {
            const double* b = boundaries + (size_t)j * stride;
            if (std::isnan(b[4 * n])) continue;
            if (!std::isnan(zl)) {
                double er, ei;
                decay(k, b[4 * n + 1] - zl, er, ei);
                const double t = er * Fr - ei * Fi;
                Fi = er * Fi + ei * Fr;
                Fr = t;
            }
            Fr += b[k];
            Fi += b[n + k];
            zl = b[4 * n + 1];
        }
        // backward: the state (inclusive) at the first point of the segments after g
        double Gr = 0.0, Gi = 0.0, zf = nan;
        for (int j = G - 1; j > g; --j) {
            const double* b = boundaries + (size_t)j * stride;
            if (std::isnan(b[4 * n])) continue;
            if (!std::isnan(zf)) {
                double er, ei;
                decay(k, zf - b[4 * n], er, ei);
                const double t = er * Gr - ei * Gi;
                Gi = er * Gi + ei * Gr;
                Gr = t;
            }
            Gr += b[2 * n + k];
            Gi += b[3 * n + k];
            zf = b[4 * n];
        }
        carry[k] = Fr;
        carry[n + k] = Fi;
        carry[2 * n + k] = Gr;
        carry[3 * n + k] = Gi;
        carry[4 * n] = zl;
        carry[4 * n + 1] = zf;
    }
    return FGT1D_OK;
}

extern "C" int fgt1d_segment_apply(fgt1d_plan plan, int64_t M, int64_t N, const double* carry, double* u,
                                   void* workspace, size_t ws_bytes, fgt1d_stream stream) {
    if (!plan || !sizes_ok(M, N)) return FGT1D_EINVAL;
    if (M == 0) return FGT1D_OK;
    if (!carry || !u) return FGT1D_EINVAL;
    Layout L = make_layout(M, N, 1, plan->n_e, plan->flags, true, false);
    int r = ws_ok(workspace, ws_bytes, L);
    if (r) return r;
    SweepArgs w = sweep_args(nullptr, N, u, nullptr, static_cast<char*>(workspace), L);
    SegmentConsts sc;
    std::memset(&sc, 0, sizeof(sc));
    sc.n_e = plan->n_e;
    sc.s = 1.0 / std::sqrt(plan->delta);
    sc.min_re_tau = INFINITY;
    for (int k = 0; k < plan->n_e; ++k) {
        sc.tau_re[k] = plan->tau_re[k];
        sc.tau_im[k] = plan->tau_im[k];
        sc.w_re[k] = plan->w_re[k];
        sc.w_im[k] = plan->w_im[k];
        sc.min_re_tau = std::min(sc.min_re_tau, plan->tau_re[k]);
    }
    return cuda_status(launch_carry_apply(w, M + N, sc, carry, u, static_cast<cudaStream_t>(stream)));
}

extern "C" int fgt1d_check(void* workspace, size_t ws_bytes, fgt1d_stream stream) {
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    if (cudaStreamSynchronize(st) != cudaSuccess) return FGT1D_ECUDA;
    if (!workspace || ws_bytes < sizeof(uint32_t)) return FGT1D_EWORKSPACE;
    uint32_t status = 0;
    if (cudaMemcpy(&status, workspace, sizeof(status), cudaMemcpyDeviceToHost) != cudaSuccess) return FGT1D_ECUDA;
    if (status && cudaMemset(workspace, 0, sizeof(status)) != cudaSuccess) return FGT1D_ECUDA;
    if (status & kStatusBadArg) return FGT1D_EINVAL;
    if (status & kStatusNonFinite) return FGT1D_ENONFINITE;
    if (status & kStatusTimeout) return FGT1D_ETIMEOUT;
    return FGT1D_OK;
}

extern "C" const char* fgt1d_strerror(int status) {
    switch (status) {
        case FGT1D_OK: return "ok";
        case FGT1D_EINVAL: return "invalid argument";
        case FGT1D_EUNSUPPORTED: return "unsupported accuracy or precision";
        case FGT1D_ENONFINITE: return "a coordinate is NaN or infinite";
        case FGT1D_ENOMEM: return "host allocation failed";
        case FGT1D_ETIMEOUT: return "a bounded inter-block wait expired";
        case FGT1D_ECUDA: return "CUDA runtime error";
        case FGT1D_EWORKSPACE: return "workspace missing, misaligned or too small";
        case FGT1D_ETOOLARGE: return "problem larger than the library's fixed scratch";
        default: return "unknown status";
    }
}

extern "C" int fgt1d_version(void) { return 100; }
