// Steps a1-a2: stable LSD radix sort of the merged points (Sec. 4 "sort both target
// and source points"; Sec. 5 uses a quicksort with an index array).
//
// The merged array is [y_0..y_{N-1}, x_0..x_{M-1}]; merged index q < N is source j = q,
// q >= N is target i = q - N.  Each coordinate is mapped to an order-preserving 64-bit
// key (-0.0 is folded onto +0.0).  A stable sort by key then puts equal coordinates in
// merged-index order: sources before targets, as eq. 4.4 needs (y_j <= x_i goes to h+).
//
// GB300 design: one histogram pass counts all eight 8-bit digits at once (per-thread
// run-length counting keeps the near-constant high digits off the shared atomics);
// a one-block kernel turns the counts into bucket offsets and a device-side pass plan
// that skips digits with a single populated bucket; then one "onesweep" kernel per
// digit ranks a 4096-key tile in shared memory (ballot-based warp ranking), finds the
// tile's global offsets by decoupled look-back over the preceding tiles, and writes
// keys and merged indices out through a shared-memory reorder so that every bucket
// run is written contiguously.  The pass plan lives on the device, so the whole sort
// is launched without a host round trip (and can be captured in a CUDA graph).
//
// Presorted inputs (Sec. 5's pre-sorted points; its Chebyshev points "sort in much less
// time"): the histogram pass also checks that every item's sources and targets are each
// in non-decreasing key order; when they are, the plan runs no digit pass and one merge
// kernel writes the stable merged order (sources first on equal keys) instead.
#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>

#include "fgt1d_internal.h"
#include "kernels.h"

namespace fgt1d {

__device__ __forceinline__ uint64_t coord_key(double c) {
    uint64_t b = (uint64_t)__double_as_longlong(c);
    if (b == 0x8000000000000000ull) b = 0;  // -0.0 -> +0.0
    return (b >> 63) ? ~b : (b | 0x8000000000000000ull);
}

__device__ __forceinline__ bool coord_nonfinite(double c) {
    return ((uint64_t)__double_as_longlong(c) & 0x7FF0000000000000ull) == 0x7FF0000000000000ull;
}

// ---- item table -----------------------------------------------------------------------
__global__ void __launch_bounds__(1024) k_items(int B, const int64_t* __restrict__ x_off,
                                                const int64_t* __restrict__ y_off, const double* __restrict__ delta,
                                                double plan_delta, int64_t max_tiles, int64_t M_tot, int64_t N_tot,
                                                Item* __restrict__ items, int64_t* __restrict__ total_tiles,
                                                uint32_t* __restrict__ status) {
    __shared__ int64_t warp_sum[32];
    __shared__ int64_t carry;
    if (threadIdx.x == 0) carry = 0;
    __syncthreads();
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    bool bad = false;
    for (int b0 = 0; b0 < B; b0 += blockDim.x) {
        const int b = b0 + threadIdx.x;
        int64_t nt = 0, nsrc = 0, ntgt = 0, xo = 0, yo = 0;
        double d = plan_delta;
        if (b < B) {
            xo = x_off[b];
            yo = y_off[b];
            const int64_t x1 = x_off[b + 1], y1 = y_off[b + 1];
            if (delta) d = delta[b];
            if (xo < 0 || x1 < xo || x1 > M_tot || yo < 0 || y1 < yo || y1 > N_tot || !(d > 0.0) || !isfinite(d)) {
                bad = true;  // the item is left empty
                xo = yo = 0;
            } else {
                nsrc = y1 - yo;
                ntgt = x1 - xo;
            }
            nt = (nsrc + ntgt + kTile - 1) / kTile;
        }
        // block-wide exclusive scan of nt
        int64_t inc = nt;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int64_t t = __shfl_up_sync(0xffffffffu, inc, o);
            if (lane >= o) inc += t;
        }
        if (lane == 31) warp_sum[w] = inc;
        __syncthreads();
        int64_t wpre = 0;
        for (int q = 0; q < w; ++q) wpre += warp_sum[q];
        const int64_t excl = carry + wpre + inc - nt;
        if (b < B) {
            Item it;
            it.start = excl * kTile;
            it.nsrc = nsrc;
            it.ntgt = ntgt;
            it.y_off = yo;
            it.x_off = xo;
            it.tile0 = excl;
            it.ntiles = nt;
            it.s = nt ? 1.0 / sqrt(d) : 0.0;
            items[b] = it;
        }
        __syncthreads();
        if (threadIdx.x == blockDim.x - 1) carry = excl + nt;
        __syncthreads();
    }
    if (__syncthreads_or(bad) && threadIdx.x == 0) atomicOr(status, kStatusBadArg);
    const int64_t total = carry;
    if (total > max_tiles) {  // overlapping items: run nothing and report
        for (int b = threadIdx.x; b < B; b += blockDim.x) items[b].ntiles = 0, items[b].nsrc = 0, items[b].ntgt = 0;
        if (threadIdx.x == 0) {
            atomicOr(status, kStatusBadArg);
            *total_tiles = 0;
        }
    } else if (threadIdx.x == 0) {
        *total_tiles = total;
    }
}

__global__ void k_item_single(int64_t M, int64_t N, double delta, Item* __restrict__ items,
                              int64_t* __restrict__ total_tiles) {
    Item it;
    it.start = 0;
    it.nsrc = N;
    it.ntgt = M;
    it.y_off = 0;
    it.x_off = 0;
    it.tile0 = 0;
    it.ntiles = (M + N + kTile - 1) / kTile;
    it.s = 1.0 / sqrt(delta);
    items[0] = it;
    *total_tiles = it.ntiles;
}

cudaError_t launch_items(int B, const int64_t* x_off, const int64_t* y_off, const double* delta, double plan_delta,
                         Item* items, int64_t* total_tiles, uint32_t* status, int64_t max_tiles, int64_t M_tot,
                         int64_t N_tot, cudaStream_t st) {
    k_items<<<1, 1024, 0, st>>>(B, x_off, y_off, delta, plan_delta, max_tiles, M_tot, N_tot, items, total_tiles,
                                status);
    return cudaGetLastError();
}

cudaError_t launch_item_single(int64_t M, int64_t N, double delta, Item* items, int64_t* total_tiles,
                               cudaStream_t st) {
    k_item_single<<<1, 1, 0, st>>>(M, N, delta, items, total_tiles);
    return cudaGetLastError();
}

// Key and merged code of padded position g of item `it`: sources first, then targets,
// then padding (all-ones key, sorted last).
__device__ __forceinline__ void merged_point(const SortArgs& a, const Item& it, int64_t g, uint64_t& key,
                                             uint32_t& val, bool& bad) {
    const int64_t l = g - it.start;
    if (l < it.nsrc) {
        const double c = a.y[it.y_off + l];
        bad |= coord_nonfinite(c);
        key = coord_key(c);
        val = (uint32_t)(it.y_off + l);
    } else if (l < it.nsrc + it.ntgt) {
        const double c = a.x[it.x_off + (l - it.nsrc)];
        bad |= coord_nonfinite(c);
        key = coord_key(c);
        val = (uint32_t)(a.N + it.x_off + (l - it.nsrc));
    } else {
        key = ~0ull;
        val = 0xFFFFFFFFu;
    }
}

// ---- per-item histograms of all digits ----------------------------------------------------
// Each block walks a contiguous range of tiles, counting in shared memory and flushing
// the non-zero counts to the current item's histogram when the item changes.
__global__ void __launch_bounds__(256) k_sort_hist(SortArgs a) {
    __shared__ uint32_t sh[kSortDigits][256];
    __shared__ int s_item;
    const int64_t T = *a.total_tiles;
    const int64_t per = (T + gridDim.x - 1) / gridDim.x;
    const int64_t t0 = (int64_t)blockIdx.x * per, t1 = min(T, t0 + per);
    for (int i = threadIdx.x; i < kSortDigits * 256; i += blockDim.x) (&sh[0][0])[i] = 0;
    int cur = -1;
    bool bad = false;
    auto flush = [&](int item) {
        __syncthreads();
        uint32_t* h = a.hist + (size_t)item * kSortDigits * 256;
        for (int i = threadIdx.x; i < kSortDigits * 256; i += blockDim.x) {
            const uint32_t v = (&sh[0][0])[i];
            if (v) {
                atomicAdd(&h[i], v);
                (&sh[0][0])[i] = 0;
            }
        }
        __syncthreads();
    };
    bool unsorted = false;
    for (int64_t t = t0; t < t1; ++t) {
        if (threadIdx.x == 0) s_item = item_of_tile(a.items, a.B, t);
        __syncthreads();
        const int item = s_item;
        if (item != cur) {
            if (cur >= 0) flush(cur);
            cur = item;
        }
        const Item it = a.items[item];
        uint32_t last[kSortDigits], run[kSortDigits];
#pragma unroll
        for (int d = 0; d < kSortDigits; ++d) { last[d] = 0; run[d] = 0; }
        for (int e = threadIdx.x; e < kTile; e += blockDim.x) {
            // presorted check: the key before this one in the same run (sources or
            // targets of this item), from the lane below or, for lane 0, from memory (that
            // load is issued next to the point's own)
            const int64_t l = t * kTile + e - it.start;
            const bool chk = l > 0 && l != it.nsrc && l < it.nsrc + it.ntgt;
            double cprev = 0.0;
            if (chk && (threadIdx.x & 31) == 0)
                cprev = l < it.nsrc ? a.y[it.y_off + l - 1] : a.x[it.x_off + (l - it.nsrc) - 1];
            uint64_t k;
            uint32_t v;
            merged_point(a, it, t * kTile + e, k, v, bad);
            uint64_t kp = __shfl_up_sync(0xffffffffu, k, 1);
            if (chk) {
                if ((threadIdx.x & 31) == 0) kp = coord_key(cprev);
                unsorted |= kp > k;
            }
#pragma unroll
            for (int d = 0; d < kSortDigits; ++d) {
                const uint32_t dg = (uint32_t)(k >> (8 * d)) & 255u;
                if (dg != last[d]) {
                    if (run[d]) atomicAdd(&sh[d][last[d]], run[d]);
                    last[d] = dg;
                    run[d] = 0;
                }
                ++run[d];
            }
        }
#pragma unroll
        for (int d = 0; d < kSortDigits; ++d)
            if (run[d]) atomicAdd(&sh[d][last[d]], run[d]);
        __syncthreads();
    }
    if (cur >= 0) flush(cur);
    if (__any_sync(0xffffffffu, bad) && (threadIdx.x & 31) == 0) atomicOr(a.status, kStatusNonFinite);
    if (__any_sync(0xffffffffu, unsorted) && (threadIdx.x & 31) == 0) atomicOr(&a.plan->unsorted, 1u);
}

// ---- per-item bucket starts and the digits that need a pass (one block per item) ----------
__global__ void __launch_bounds__(256) k_sort_plan(SortArgs a) {
    __shared__ uint32_t scan[256];
    const int b = blockIdx.x;
    const Item it = a.items[b];
    const int t = threadIdx.x;
    const int64_t Pb = it.ntiles * kTile;
    for (int d = 0; d < kSortDigits; ++d) {
        const uint32_t v = a.hist[((size_t)b * kSortDigits + d) * 256 + t];
        scan[t] = v;
        __syncthreads();
        for (int o = 1; o < 256; o <<= 1) {
            const uint32_t add = t >= o ? scan[t - o] : 0;
            __syncthreads();
            scan[t] += add;
            __syncthreads();
        }
        a.offs[((size_t)b * kSortDigits + d) * 256 + t] = (uint32_t)it.start + scan[t] - v;
        const int partial = (v != 0 && (int64_t)v != Pb);
        if (__syncthreads_or(partial) && t == 0) atomicOr(&a.plan->active_mask, 1u << d);
    }
}

// ---- the pass chain: which buffers each active digit reads and writes -------------------
__global__ void k_sort_chain(SortPlan* plan) {
    const uint32_t mask = plan->active_mask;
    int cur = -1, n_active = 0;
    for (int d = 0; d < kSortDigits; ++d) {
        plan->active[d] = 0;
        plan->src[d] = 0;
        plan->dst[d] = 0;
    }
    plan->merge = plan->unsorted ? 0u : 1u;
    if (plan->merge) {  // presorted runs: no digit pass, k_sort_merge writes buffer A
        plan->final_buf = 0;
        return;
    }
    for (int d = 0; d < kSortDigits; ++d) {
        if (!((mask >> d) & 1u)) continue;
        plan->active[d] = 1;
        plan->src[d] = cur;
        plan->dst[d] = (cur == 0) ? 1 : 0;
        cur = plan->dst[d];
        ++n_active;
    }
    if (n_active == 0) {  // every key of every item equal: one pass materialises keys/codes
        plan->active[0] = 1;
        plan->src[0] = -1;
        plan->dst[0] = 0;
        cur = 0;
    }
    plan->final_buf = cur;
}

// ---- one onesweep digit pass -------------------------------------------------------------
__device__ __forceinline__ unsigned lanemask_lt() {
    unsigned m;
    asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
    return m;
}

__device__ __forceinline__ void st_volatile_u64(uint64_t* p, uint64_t v) {
    asm volatile("st.volatile.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}
__device__ __forceinline__ uint64_t ld_volatile_u64(const uint64_t* p) {
    uint64_t v;
    asm volatile("ld.volatile.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}

constexpr uint64_t kDescAgg = 1ull << 62;
constexpr uint64_t kDescInc = 2ull << 62;

struct SortSmem {
    uint64_t keys[kSortTile];
    uint32_t vals[kSortTile];
    uint32_t wcnt[kSortThreads / 32][256];
    uint32_t tile_start[256];
    uint32_t gbase[256];
    uint32_t tile_id;
};

__global__ void __launch_bounds__(kSortThreads, 3) k_sort_pass(SortArgs a, int d) {
    const SortPlan* pl = a.plan;
    if (!pl->active[d]) return;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    SortSmem& sm = *reinterpret_cast<SortSmem*>(smem_raw);
    __shared__ int s_item;
    const int src = pl->src[d], dst = pl->dst[d];
    const uint64_t* __restrict__ kin = src == 1 ? a.keysB : a.keysA;
    const uint32_t* __restrict__ vin = src == 1 ? a.valsB : a.valsA;
    uint64_t* __restrict__ kout = dst == 1 ? a.keysB : a.keysA;
    uint32_t* __restrict__ vout = dst == 1 ? a.valsB : a.valsA;
    const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
    const int shift = 8 * d;

    if (tid == 0) {
        sm.tile_id = atomicAdd(&a.tile_ctr[d], 1u);
        s_item = (int64_t)sm.tile_id < *a.total_tiles ? item_of_tile(a.items, a.B, sm.tile_id) : -1;
    }
    for (int i = tid; i < (kSortThreads / 32) * 256; i += kSortThreads) (&sm.wcnt[0][0])[i] = 0;
    __syncthreads();
    if (s_item < 0) return;
    const uint32_t tile = sm.tile_id;
    const Item it = a.items[s_item];
    const int64_t base = (int64_t)tile * kSortTile;
    const uint32_t* __restrict__ item_offs = a.offs + ((size_t)s_item * kSortDigits + d) * 256;

    // load (warp-striped: warp w owns items [w*32*IPT, (w+1)*32*IPT), slot j covers 32 consecutive items)
    uint64_t key[kSortIPT];
    uint32_t val[kSortIPT];
    uint32_t rank[kSortIPT];
    bool bad = false;
#pragma unroll
    for (int j = 0; j < kSortIPT; ++j) {
        const int li = w * 32 * kSortIPT + j * 32 + lane;
        const int64_t g = base + li;
        if (src < 0) {
            merged_point(a, it, g, key[j], val[j], bad);
        } else {
            key[j] = kin[g];
            val[j] = vin[g];
        }
    }
    // stable warp ranking per slot: the lanes holding the same digit are found with
    // eight ballots (one per digit bit), for all slots first (independent work); then,
    // slot by slot, every lane reads the warp's running count for its digit and the
    // lowest peer adds the slot's count
    unsigned peers[kSortIPT];
#pragma unroll
    for (int j = 0; j < kSortIPT; ++j) {
        const uint32_t dg = (uint32_t)(key[j] >> shift) & 255u;
        unsigned pm = 0xffffffffu;
#pragma unroll
        for (int b = 0; b < 8; ++b) {
            const unsigned m = __ballot_sync(0xffffffffu, (dg >> b) & 1u);
            pm &= ((dg >> b) & 1u) ? m : ~m;
        }
        peers[j] = pm;
    }
    const unsigned lt = lanemask_lt();
#pragma unroll
    for (int j = 0; j < kSortIPT; ++j) {
        const uint32_t dg = (uint32_t)(key[j] >> shift) & 255u;
        const uint32_t old = sm.wcnt[w][dg];
        __syncwarp();
        rank[j] = old + __popc(peers[j] & lt);
        if ((peers[j] & lt) == 0) sm.wcnt[w][dg] = old + __popc(peers[j]);
        __syncwarp();
    }
    __syncthreads();
    // per digit: exclusive prefix over warps, tile count
    uint32_t tot = 0;
    {
        const int dg = tid;  // kSortThreads == 256 digits
#pragma unroll
        for (int ww = 0; ww < kSortThreads / 32; ++ww) {
            uint32_t c = sm.wcnt[ww][dg];
            sm.wcnt[ww][dg] = tot;
            tot += c;
        }
        sm.tile_start[dg] = tot;
    }
    __syncthreads();
    // exclusive scan of tile counts over digits -> tile_start
    {
        uint32_t v = sm.tile_start[tid];
        uint32_t inc = v;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            uint32_t t = __shfl_up_sync(0xffffffffu, inc, o);
            if (lane >= o) inc += t;
        }
        __shared__ uint32_t wsum[kSortThreads / 32];
        if (lane == 31) wsum[w] = inc;
        __syncthreads();
        uint32_t wpre = 0;
        for (int ww = 0; ww < w; ++ww) wpre += wsum[ww];
        __syncthreads();
        sm.tile_start[tid] = wpre + inc - v;
    }
    // decoupled look-back over the item's earlier tiles for this digit's global base;
    // each round issues the loads of kLookAhead predecessors at once
    {
        constexpr int kLookAhead = 8;
        const int dg = tid;
        uint64_t* desc = a.desc + (size_t)d * a.desc_stride;
        uint32_t excl = 0;
        if ((int64_t)tile == it.tile0) {
            st_volatile_u64(&desc[(size_t)tile * 256 + dg], kDescInc | (uint64_t)tot);
        } else {
            st_volatile_u64(&desc[(size_t)tile * 256 + dg], kDescAgg | (uint64_t)tot);
            int64_t j = (int64_t)tile - 1;
            bool done = false;
            while (!done) {
                uint64_t v[kLookAhead];
#pragma unroll
                for (int q = 0; q < kLookAhead; ++q)
                    v[q] = (j - q >= it.tile0) ? ld_volatile_u64(&desc[(size_t)(j - q) * 256 + dg]) : kDescInc;
#pragma unroll
                for (int q = 0; q < kLookAhead; ++q) {
                    if (done) break;
                    uint64_t x = v[q];
                    if ((x >> 62) == 0) {
                        const long long t0 = clock64();
                        while (((x = ld_volatile_u64(&desc[(size_t)(j - q) * 256 + dg])) >> 62) == 0) {
                            if (clock64() - t0 > a.spin_limit) {
                                atomicOr(a.status, kStatusTimeout | kStatusSortTimeout);
                                x = kDescInc;
                                break;
                            }
                        }
                    }
                    excl += (uint32_t)(x & 0xFFFFFFFFull);
                    if ((x >> 62) == 2) done = true;
                }
                j -= kLookAhead;
            }
            st_volatile_u64(&desc[(size_t)tile * 256 + dg], kDescInc | (uint64_t)(excl + tot));
        }
        sm.gbase[dg] = item_offs[dg] + excl;
    }
    __syncthreads();
    // reorder through shared memory
#pragma unroll
    for (int j = 0; j < kSortIPT; ++j) {
        const uint32_t dg = (uint32_t)(key[j] >> shift) & 255u;
        const uint32_t pos = sm.tile_start[dg] + sm.wcnt[w][dg] + rank[j];
        sm.keys[pos] = key[j];
        sm.vals[pos] = val[j];
    }
    __syncthreads();
    const int64_t item_end = it.start + it.ntiles * kTile;
    for (int i = tid; i < kSortTile; i += kSortThreads) {
        const uint64_t k = sm.keys[i];
        const uint32_t dg = (uint32_t)(k >> shift) & 255u;
        const int64_t o = (int64_t)sm.gbase[dg] + i - sm.tile_start[dg];
        if (o < item_end) {  // always true unless a look-back wait timed out
            kout[o] = k;
            vout[o] = sm.vals[i];
        }
    }
    if (__any_sync(0xffffffffu, bad) && lane == 0) atomicOr(a.status, kStatusNonFinite);
}

// ---- presorted runs: one merge -------------------------------------------------------
constexpr int kMergeIPT = kSortTile / kSortThreads;  // merged outputs per thread

struct MergeSmem {
    uint64_t key[kSortTile];
    uint32_t val[kSortTile];
};

// Number of sources among the first d merged points of runs ys[ns], xs[nt] (each
// non-decreasing; a source goes first on equal keys): the first i in [max(0, d - nt),
// min(d, ns)) with ys[i] > xs[d - 1 - i], or min(d, ns) if there is none.  The warp tests
// 32 evenly spaced candidates per step (the predicate is monotone: true, then false), so
// the range shrinks 32-fold per step; every lane returns the same value.
template <typename KY, typename KX>
__device__ int64_t merge_split_warp(int64_t d, int64_t ns, int64_t nt, KY ky, KX kx) {
    const int lane = threadIdx.x & 31;
    int64_t lo = max((int64_t)0, d - nt), hi = min(d, ns);
    while (lo < hi) {
        const int64_t step = (hi - lo + 31) / 32;
        const int64_t i = lo + (int64_t)lane * step;
        const bool p = i < hi && ky(i) <= kx(d - 1 - i);
        const int c = __popc(__ballot_sync(0xffffffffu, p));
        if (c == 0) break;  // the first candidate (lo) already fails
        const int64_t nhi = min(hi, lo + (int64_t)c * step);
        lo += (int64_t)(c - 1) * step + 1;
        hi = nhi;
    }
    return lo;
}

// One block per 4096-position tile of an item: two warps find where the tile starts and
// ends on the merge path, the block stages the tile's sources and targets in shared
// memory, each thread merges 16 consecutive outputs from its own split (a binary search
// in shared memory), and the tile goes out through shared memory, coalesced.  Positions
// past the item's points get the padding key and code, as in the digit passes.
__global__ void __launch_bounds__(kSortThreads) k_sort_merge(SortArgs a) {
    if (!a.plan->merge) return;
    const int64_t tile = blockIdx.x;
    if (tile >= *a.total_tiles) return;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    MergeSmem& sm = *reinterpret_cast<MergeSmem*>(smem_raw);
    __shared__ int s_item;
    __shared__ int64_t s_split[2];
    const int tid = threadIdx.x, w = tid >> 5;
    if (tid == 0) s_item = item_of_tile(a.items, a.B, tile);
    __syncthreads();
    const Item it = a.items[s_item];
    const int64_t ns = it.nsrc, nt = it.ntgt, nreal = ns + nt;
    const int64_t d0 = min(tile * kSortTile - it.start, nreal), d1 = min(d0 + kSortTile, nreal);
    const double* __restrict__ ys = ns > 0 ? a.y + it.y_off : nullptr;  // no sources: never read
    const double* __restrict__ xs = nt > 0 ? a.x + it.x_off : nullptr;  // no targets: never read
    auto ky = [&](int64_t i) { return coord_key(ys[i]); };
    auto kx = [&](int64_t j) { return coord_key(xs[j]); };
    if (w < 2) {
        const int64_t sp = merge_split_warp(w == 0 ? d0 : d1, ns, nt, ky, kx);
        if ((tid & 31) == 0) s_split[w] = sp;
    }
    __syncthreads();
    const int64_t i0 = s_split[0], j0 = d0 - s_split[0];
    const int nsl = (int)(s_split[1] - i0), nl = (int)(d1 - d0), ntl = nl - nsl;
    for (int q = tid; q < nl; q += kSortThreads) sm.key[q] = q < nsl ? ky(i0 + q) : kx(j0 + (q - nsl));
    __syncthreads();
    uint64_t ok[kMergeIPT];
    uint32_t ov[kMergeIPT];
    const int dd = tid * kMergeIPT;
    {
        int lo = max(0, dd - ntl), hi = min(dd, nsl);
        while (lo < hi) {
            const int mid = (lo + hi) >> 1;
            if (sm.key[mid] <= sm.key[nsl + dd - 1 - mid]) lo = mid + 1;
            else hi = mid;
        }
        int ia = lo, ib = dd - lo;
#pragma unroll
        for (int q = 0; q < kMergeIPT; ++q) {
            ok[q] = ~0ull;
            ov[q] = 0xFFFFFFFFu;
            if (dd + q < nl) {
                if (ia < nsl && (ib >= ntl || sm.key[ia] <= sm.key[nsl + ib])) {
                    ok[q] = sm.key[ia];
                    ov[q] = (uint32_t)(it.y_off + i0 + ia);
                    ++ia;
                } else {
                    ok[q] = sm.key[nsl + ib];
                    ov[q] = (uint32_t)(a.N + it.x_off + j0 + ib);
                    ++ib;
                }
            }
        }
    }
    __syncthreads();
#pragma unroll
    for (int q = 0; q < kMergeIPT; ++q) {
        sm.key[dd + q] = ok[q];
        sm.val[dd + q] = ov[q];
    }
    __syncthreads();
    const int64_t base = tile * kSortTile;
    for (int q = tid; q < kSortTile; q += kSortThreads) {
        a.keysA[base + q] = sm.key[q];
        a.valsA[base + q] = sm.val[q];
    }
}

size_t sort_pass_smem() { return sizeof(SortSmem); }

cudaError_t launch_sort(const SortArgs& a, cudaStream_t st) {
    if (a.max_tiles <= 0) return cudaSuccess;
    cudaError_t e = cudaFuncSetAttribute(k_sort_pass, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)sizeof(SortSmem));
    if (e != cudaSuccess) return e;
    const int hist_blocks = (int)std::min<int64_t>(a.max_tiles, 152 * 4);
    k_sort_hist<<<hist_blocks, 256, 0, st>>>(a);
    k_sort_plan<<<a.B, 256, 0, st>>>(a);
    k_sort_chain<<<1, 1, 0, st>>>(a.plan);
    for (int d = 0; d < kSortDigits; ++d)
        k_sort_pass<<<(unsigned)a.max_tiles, kSortThreads, sizeof(SortSmem), st>>>(a, d);
    e = cudaFuncSetAttribute(k_sort_merge, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sizeof(MergeSmem));
    if (e != cudaSuccess) return e;
    k_sort_merge<<<(unsigned)a.max_tiles, kSortThreads, sizeof(MergeSmem), st>>>(a);
    return cudaGetLastError();
}

__global__ void k_copy_perm(const uint32_t* __restrict__ va, const uint32_t* __restrict__ vb, const SortPlan* plan,
                            int64_t P, uint32_t* __restrict__ perm) {
    const uint32_t* v = plan->final_buf == 1 ? vb : va;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < P; i += (int64_t)gridDim.x * blockDim.x)
        perm[i] = v[i];
}

cudaError_t launch_copy_perm(const SortArgs& a, int64_t P, uint32_t* perm, cudaStream_t st) {
    if (P <= 0) return cudaSuccess;
    int blocks = (int)std::min<int64_t>((P + 255) / 256, 152 * 16);
    k_copy_perm<<<blocks, 256, 0, st>>>(a.valsA, a.valsB, a.plan, P, perm);
    return cudaGetLastError();
}

}  // namespace fgt1d
