// Steps a1-a2: stable LSD radix sort of the merged points (Sec. 4 "sort both target
// and source points"; Sec. 5 uses a quicksort with an index array).
//
// The merged array is [y_0..y_{N-1}, x_0..x_{M-1}]; merged index q < N is source j = q,
// q >= N is target i = q - N.  Each coordinate is mapped to an order-preserving 64-bit
// key (-0.0 is folded onto +0.0).  A stable sort by key then puts equal coordinates in
// merged-index order: sources before targets, as eq. 4.4 needs (y_j <= x_i goes to h+).
//
// GB300 design.  The order only needs as many key bits as separate the points, so the
// sort runs on a 32-bit prefix key: per item, the fixed-point value of the coordinate
// on the grid 2^(eh - 1075) (eh = the larger exponent of the item's extreme
// coordinates), less that of the smallest coordinate, shifted right until the item's
// range fits 32 bits.  It is integer arithmetic on the coordinate's bits and a
// non-decreasing function of the coordinate, so sorting by it leaves only runs of equal
// prefixes in merged-index order; for 2^27 uniform points in 2^32 bins about 3 % of
// the points share a prefix.  Stages:
//   range   per-item smallest and largest key (one read of x and y);
//   hist    the four prefix-digit histograms per item and the presorted check; writes
//           each point's prefix key, full key and merged code (buffer 1);
//   plan    bucket offsets and the digits with more than one populated bucket;
//   4 x     a "onesweep" digit pass on the prefix keys, with the full keys and codes as
//           payload: each 4096-key tile is ranked in shared memory (ballot-based warp
//           ranking), finds its global offsets by decoupled look-back over the
//           preceding tiles, and goes out through a shared-memory reorder so that every
//           bucket run is written contiguously (prefix keys and codes first, then the
//           full keys through the same shared words);
//   detect  the neighbour pairs with equal prefixes whose keys are out of order list
//           their runs (first position and length);
//   fix-up  one thread sorts each listed run by (key, merged index).
// Carrying the full keys costs 12 bytes per point and pass; reading them back by code
// after the passes would cost a random 8-byte read per point, about 64 bytes of DRAM
// traffic each on this part.  A run longer than kRunMax with keys out of order (a
// cluster of distinct coordinates narrower than the item's range / 2^32) sets the
// fallback flag, and the full sort -- the same pass kernel on the 64-bit key, eight
// digit passes -- runs from the start.  The plans live on the device, so the whole sort
// is launched without a host round trip (and can be captured in a CUDA graph); kernels
// of a stage that does not run exit at once.
//
// Presorted inputs (Sec. 5's pre-sorted points; its Chebyshev points "sort in much less
// time"): the histogram pass also checks that every item's sources and targets are each
// in non-decreasing key order; when they are, the plan runs no digit pass and one merge
// kernel writes the stable merged order (sources first on equal keys) instead.
#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>
#include <type_traits>

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

// ---- prefix keys ----------------------------------------------------------------------
// The bits of the coordinate of key k (inverse of coord_key; -0.0 comes back as +0.0).
__device__ __forceinline__ uint64_t key_bits(uint64_t k) {
    return (k >> 63) ? (k & 0x7FFFFFFFFFFFFFFFull) : ~k;
}

// Q(z) = sign(z) floor(|z| / 2^(eh - 1075)) from the bits of z: the 53-bit significand
// (implicit bit included, subnormals at exponent 1) shifted right by eh - e.  It is a
// non-decreasing function of z for every |z| whose exponent is at most eh.
__device__ __forceinline__ int64_t fixq(uint64_t b, int eh) {
    const int ef = (int)((b >> 52) & 0x7FF);
    uint64_t m = b & 0x000FFFFFFFFFFFFFull;
    int e = 1;
    if (ef) {
        m |= 0x0010000000000000ull;
        e = ef;
    }
    const int sh = eh - e;  // >= 0 inside the item's range
    const uint64_t q = sh >= 64 ? 0ull : (sh <= 0 ? m : (m >> sh));
    return (b >> 63) ? -(int64_t)q : (int64_t)q;
}

// The 32-bit prefix key of key k in an item with map m; padding (all-ones key) and
// anything outside the map's range go to 0xFFFFFFFF.
__device__ __forceinline__ uint32_t prefix_of_key(uint64_t k, const PrefixMap& m) {
    if (k == ~0ull) return 0xFFFFFFFFu;
    const uint64_t r = (uint64_t)(fixq(key_bits(k), m.eh) - m.qlo) >> m.sh;
    return r > 0xFFFFFFFFull ? 0xFFFFFFFFu : (uint32_t)r;
}

// The map of an item whose keys span [klo, khi] (klo > khi: no points).
__device__ __forceinline__ PrefixMap make_prefix_map(uint64_t klo, uint64_t khi) {
    PrefixMap m;
    m.qlo = 0;
    m.eh = 1;
    m.sh = 0;
    if (klo > khi) return m;
    const uint64_t blo = key_bits(klo), bhi = key_bits(khi);
    m.eh = max(1, max((int)((blo >> 52) & 0x7FF), (int)((bhi >> 52) & 0x7FF)));
    m.qlo = fixq(blo, m.eh);
    const uint64_t span = (uint64_t)(fixq(bhi, m.eh) - m.qlo);
    m.sh = span >> 32 ? 32 - __clzll((long long)span) : 0;  // (span >> sh) < 2^32
    return m;
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
    // the address is chosen by selects and the load is unconditional (padding reads the
    // item's first point), so that a thread's loads of several points are all in flight
    const int64_t l = g - it.start;
    const bool src = l < it.nsrc, tgt = !src && l < it.nsrc + it.ntgt;
    const double* p = src ? a.y + it.y_off + l
                          : (tgt ? a.x + it.x_off + (l - it.nsrc) : (it.nsrc > 0 ? a.y + it.y_off : a.x + it.x_off));
    const double c = *p;
    bad |= (src || tgt) && coord_nonfinite(c);
    key = (src || tgt) ? coord_key(c) : ~0ull;
    val = src ? (uint32_t)(it.y_off + l) : (tgt ? (uint32_t)(a.N + it.x_off + (l - it.nsrc)) : 0xFFFFFFFFu);
}

// ---- per-item coordinate range (prefix sort) ----------------------------------------------
// Each block walks a contiguous range of tiles and flushes its extremes when the item
// changes; the smallest key is kept complemented, so both ends are atomicMax on words
// that start at zero.
__global__ void __launch_bounds__(256) k_sort_range(SortArgs a) {
    __shared__ int s_item;
    __shared__ uint64_t s_lo[8], s_hi[8];
    const int64_t T = *a.total_tiles;
    const int64_t per = (T + gridDim.x - 1) / gridDim.x;
    const int64_t t0 = (int64_t)blockIdx.x * per, t1 = min(T, t0 + per);
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    unsigned long long* range = reinterpret_cast<unsigned long long*>(a.maps);
    uint64_t lo = ~0ull, hi = 0ull;
    int cur = -1;
    auto flush = [&](int item) {
#pragma unroll
        for (int o = 16; o; o >>= 1) {
            lo = min(lo, (uint64_t)__shfl_xor_sync(0xffffffffu, lo, o));
            hi = max(hi, (uint64_t)__shfl_xor_sync(0xffffffffu, hi, o));
        }
        if (lane == 0) {
            s_lo[w] = lo;
            s_hi[w] = hi;
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            uint64_t l = s_lo[0], h = s_hi[0];
            for (int q = 1; q < 8; ++q) {
                l = min(l, s_lo[q]);
                h = max(h, s_hi[q]);
            }
            if (l <= h) {
                atomicMax(&range[2 * item], (unsigned long long)~l);
                atomicMax(&range[2 * item + 1], (unsigned long long)h);
            }
        }
        __syncthreads();
        lo = ~0ull;
        hi = 0ull;
    };
    for (int64_t t = t0; t < t1; ++t) {
        if (threadIdx.x == 0) s_item = item_of_tile(a.items, a.B, t);
        __syncthreads();
        const int item = s_item;
        if (item != cur) {
            if (cur >= 0) flush(cur);
            cur = item;
        }
        const Item it = a.items[item];
        double c[kSortIPT];
        bool real[kSortIPT];
#pragma unroll
        for (int j = 0; j < kSortIPT; ++j) {  // all loads first
            const int64_t l = t * kTile + threadIdx.x + j * 256 - it.start;
            real[j] = l < it.nsrc + it.ntgt;
            c[j] = *(l < it.nsrc ? a.y + it.y_off + l
                                 : (real[j] ? a.x + it.x_off + (l - it.nsrc) : (it.nsrc > 0 ? a.y + it.y_off : a.x + it.x_off)));
        }
#pragma unroll
        for (int j = 0; j < kSortIPT; ++j)
            if (real[j]) {
                const uint64_t k = coord_key(c[j]);
                lo = min(lo, k);
                hi = max(hi, k);
            }
        __syncthreads();  // s_item is rewritten for the next tile
    }
    if (cur >= 0) flush(cur);
}

// The per-item prefix maps, in place of the ranges (one thread per item).
__global__ void k_prefix_maps(SortArgs a) {
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= a.B) return;
    const uint64_t* range = reinterpret_cast<const uint64_t*>(a.maps);
    const uint64_t klo = ~range[2 * b], khi = range[2 * b + 1];
    a.maps[b] = make_prefix_map(klo, khi);
}

// ---- per-item digit histograms ------------------------------------------------------------
// PREFIX: the four digits of the prefix keys, and the presorted check; the prefix keys
// and the merged codes are written out for the first digit pass.  Otherwise (the
// full sort, only after a fallback): the eight digits of the 64-bit keys.  Each block
// walks a contiguous range of tiles, counting in shared memory and flushing the non-zero
// counts to the current item's histogram when the item changes.
template <bool PREFIX>
__global__ void __launch_bounds__(256, 4) k_sort_hist(SortArgs a) {
    constexpr int ND = PREFIX ? kPrefixDigits : kSortDigits;
    if (!PREFIX && (!a.pplan->fallback || (*a.status & kStatusSortTimeout))) return;
    __shared__ uint32_t sh[ND][256];
    __shared__ int s_item;
    const int64_t T = *a.total_tiles;
    const int64_t per = (T + gridDim.x - 1) / gridDim.x;
    const int64_t t0 = (int64_t)blockIdx.x * per, t1 = min(T, t0 + per);
    const int lane = threadIdx.x & 31;
    for (int i = threadIdx.x; i < ND * 256; i += blockDim.x) (&sh[0][0])[i] = 0;
    int cur = -1;
    bool bad = false;
    auto flush = [&](int item) {
        __syncthreads();
        uint32_t* h = a.hist + (size_t)item * kSortDigits * 256;
        for (int i = threadIdx.x; i < ND * 256; i += blockDim.x) {
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
        PrefixMap m;
        if (PREFIX) m = a.maps[item];
        uint32_t last[ND], run[ND];
#pragma unroll
        for (int d = 0; d < ND; ++d) {
            last[d] = 0;
            run[d] = 0;
        }
#pragma unroll
        for (int j = 0; j < kSortIPT; ++j) {
            const int64_t g = t * kTile + threadIdx.x + j * 256;
            uint64_t k;
            uint32_t v;
            merged_point(a, it, g, k, v, bad);
            uint64_t dk = k;
            if (PREFIX) {
                // the first digit pass reads buffer 1: codes, full keys and prefix keys
                a.valsB[g] = v;
                a.keysB[g] = k;
                dk = prefix_of_key(k, m);
                a.pre[a.Ppad + g] = (uint32_t)dk;
                // presorted check: the key before this point in the same run (sources or
                // targets of this item), from the lane below or, for lane 0, from memory
                const int64_t l = g - it.start;
                const bool chk = l > 0 && l != it.nsrc && l < it.nsrc + it.ntgt;
                uint64_t kp = __shfl_up_sync(0xffffffffu, k, 1);
                if (lane == 0 && chk)
                    kp = coord_key(l < it.nsrc ? a.y[it.y_off + l - 1] : a.x[it.x_off + (l - it.nsrc) - 1]);
                if (chk) unsorted |= kp > k;
            }
#pragma unroll
            for (int d = 0; d < ND; ++d) {
                const uint32_t dg = (uint32_t)(dk >> (8 * d)) & 255u;
                if (dg != last[d]) {
                    if (run[d]) atomicAdd(&sh[d][last[d]], run[d]);
                    last[d] = dg;
                    run[d] = 0;
                }
                ++run[d];
            }
        }
#pragma unroll
        for (int d = 0; d < ND; ++d)
            if (run[d]) atomicAdd(&sh[d][last[d]], run[d]);
        __syncthreads();
    }
    if (cur >= 0) flush(cur);
    if (PREFIX) {
        if (__any_sync(0xffffffffu, bad) && lane == 0) atomicOr(a.status, kStatusNonFinite);
        if (__any_sync(0xffffffffu, unsorted) && lane == 0) atomicOr(&a.plan->unsorted, 1u);
    }
}

// ---- per-item bucket starts and the digits that need a pass (one block per item) ----------
template <bool PREFIX>
__global__ void __launch_bounds__(256) k_sort_plan(SortArgs a) {
    constexpr int ND = PREFIX ? kPrefixDigits : kSortDigits;
    if (!PREFIX && (!a.pplan->fallback || (*a.status & kStatusSortTimeout))) return;
    __shared__ uint32_t scan[256];
    uint32_t* mask = PREFIX ? &a.pplan->mask : &a.plan->active_mask;
    const int b = blockIdx.x;
    const Item it = a.items[b];
    const int t = threadIdx.x;
    const int64_t Pb = it.ntiles * kTile;
    for (int d = 0; d < ND; ++d) {
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
        if (__syncthreads_or(partial) && t == 0) atomicOr(mask, 1u << d);
    }
}

// ---- the pass chains: which buffers each active digit reads and writes -------------------
// Prefix sort (or the merge of presorted runs): the histogram pass left the prefix keys
// and codes in buffer 1; the active digits ping-pong from there.
__global__ void k_sort_chain(SortArgs a) {
    SortPlan* plan = a.plan;
    PrefixPlan* pp = a.pplan;
    for (int d = 0; d < kSortDigits; ++d) {
        plan->active[d] = 0;
        plan->src[d] = 0;
        plan->dst[d] = 0;
    }
    for (int d = 0; d < kPrefixDigits; ++d) {
        pp->active[d] = 0;
        pp->src[d] = 0;
        pp->dst[d] = 0;
    }
    plan->final_buf = 0;  // (the merge writes buffer A)
    plan->merge = plan->unsorted ? 0u : 1u;
    int cur = 1;
    if (!plan->merge)  // (presorted runs: no digit pass, k_sort_merge writes buffer A)
        for (int d = 0; d < kPrefixDigits; ++d) {
            if (!((pp->mask >> d) & 1u)) continue;  // one populated bucket: the order stands
            pp->active[d] = 1;
            pp->src[d] = cur;
            pp->dst[d] = 1 - cur;
            cur = 1 - cur;
        }
    pp->final_buf = cur;
    if (!plan->merge) plan->final_buf = cur;
}

// Full sort (after a fallback): digits with more than one populated bucket, ping-pong
// between buffers A and B.
__global__ void k_sort_chain_full(SortArgs a) {
    if (!a.pplan->fallback || (*a.status & kStatusSortTimeout)) return;
    SortPlan* plan = a.plan;
    const uint32_t mask = plan->active_mask;
    int cur = -1, n_active = 0;
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

template <typename K>
struct SortSmem {
    // the sorted tile: keys and codes; the prefix passes stage their full keys in the
    // same words afterwards
    union {
        struct {
            K keys[kSortTile];
            uint32_t vals[kSortTile];
        } kv;
        uint64_t full[kSortTile];
    } t;
    uint32_t wcnt[kSortThreads / 32][256];
    uint32_t tile_start[256];
    uint32_t gbase[256];
    uint32_t wsum[kSortThreads / 32];
    uint32_t tile_id;
    int item;
};


// PREFIX: a pass of the prefix sort: 32-bit prefix keys, with the codes and the full
// 64-bit keys as payload (buffers: 0 = (pre, keysA, valsA), 1 = (pre + Ppad, keysB,
// valsB)).  Otherwise a pass of the full sort (64-bit keys and codes, buffers A and B),
// which runs only after a fallback.  Every block takes tiles in order from the pass's
// counter until none is left, so a grid of any size is correct: the look-back only
// waits on tiles that running blocks hold.
template <bool PREFIX>
__global__ void __launch_bounds__(kSortThreads, 3) k_sort_pass(SortArgs a, int d) {
    using K = typename std::conditional<PREFIX, uint32_t, uint64_t>::type;
    int src, dst;
    uint32_t* ctr;
    if (PREFIX) {
        if (!a.pplan->active[d]) return;
        src = a.pplan->src[d];
        dst = a.pplan->dst[d];
        ctr = &a.pplan->pass_ctr[d];
    } else {
        if (!a.pplan->fallback || (*a.status & kStatusSortTimeout) || !a.plan->active[d]) return;
        src = a.plan->src[d];
        dst = a.plan->dst[d];
        ctr = &a.tile_ctr[d];
    }
    extern __shared__ __align__(16) unsigned char smem_raw[];
    SortSmem<K>& sm = *reinterpret_cast<SortSmem<K>*>(smem_raw);
    // sort keys
    K* kb0 = PREFIX ? reinterpret_cast<K*>(a.pre) : reinterpret_cast<K*>(a.keysA);
    K* kb1 = PREFIX ? reinterpret_cast<K*>(a.pre + a.Ppad) : reinterpret_cast<K*>(a.keysB);
    const K* __restrict__ kin = src == 1 ? kb1 : kb0;
    K* __restrict__ kout = dst == 1 ? kb1 : kb0;
    const uint32_t* __restrict__ vin = src == 1 ? a.valsB : a.valsA;
    uint32_t* __restrict__ vout = dst == 1 ? a.valsB : a.valsA;
    // full-key payload of the prefix passes
    const uint64_t* __restrict__ fin = src == 1 ? a.keysB : a.keysA;
    uint64_t* __restrict__ fout = dst == 1 ? a.keysB : a.keysA;
    const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
    const int shift = 8 * d;
    const int64_t T = *a.total_tiles;
    uint64_t* desc = a.desc + (size_t)d * a.desc_stride;

    for (;;) {
        if (tid == 0) {
            sm.tile_id = atomicAdd(ctr, 1u);
            sm.item = (int64_t)sm.tile_id < T ? item_of_tile(a.items, a.B, sm.tile_id) : -1;
        }
        for (int i = tid; i < (kSortThreads / 32) * 256; i += kSortThreads) (&sm.wcnt[0][0])[i] = 0;
        __syncthreads();
        if (sm.item < 0) return;
        const uint32_t tile = sm.tile_id;
        const int item = sm.item;
        const Item it = a.items[item];
        const int64_t base = (int64_t)tile * kSortTile;
        const uint32_t* __restrict__ item_offs = a.offs + ((size_t)item * kSortDigits + d) * 256;

        // load (warp-striped: warp w owns keys [w*32*IPT, (w+1)*32*IPT), slot j covers 32 consecutive keys)
        K key[kSortIPT];
        uint32_t val[kSortIPT];
        uint32_t rank[kSortIPT];
        bool bad = false;
        if (!PREFIX && src < 0) {  // (the prefix passes start from the histogram pass's output)
#pragma unroll
            for (int j = 0; j < kSortIPT; ++j) {
                uint64_t k;
                merged_point(a, it, base + w * 32 * kSortIPT + j * 32 + lane, k, val[j], bad);
                key[j] = (K)k;
            }
        } else {
#pragma unroll
            for (int j = 0; j < kSortIPT; ++j) {
                const int64_t g = base + w * 32 * kSortIPT + j * 32 + lane;
                key[j] = kin[g];
                if (!PREFIX) val[j] = vin[g];
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
                const unsigned mb = __ballot_sync(0xffffffffu, (dg >> b) & 1u);
                pm &= ((dg >> b) & 1u) ? mb : ~mb;
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
        // the prefix passes' codes, loaded now: their latency runs under the scans and
        // the look-back
        if (PREFIX) {
#pragma unroll
            for (int j = 0; j < kSortIPT; ++j) val[j] = vin[base + w * 32 * kSortIPT + j * 32 + lane];
        }
        __syncthreads();
        // per digit: exclusive prefix over warps, tile count
        uint32_t tot = 0;
        {
            const int dg = tid;  // kSortThreads == 256 digits
#pragma unroll
            for (int ww = 0; ww < kSortThreads / 32; ++ww) {
                const uint32_t c = sm.wcnt[ww][dg];
                sm.wcnt[ww][dg] = tot;
                tot += c;
            }
        }
        // exclusive scan of tile counts over digits -> tile_start
        {
            uint32_t inc = tot;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const uint32_t t = __shfl_up_sync(0xffffffffu, inc, o);
                if (lane >= o) inc += t;
            }
            if (lane == 31) sm.wsum[w] = inc;
            __syncthreads();
            uint32_t wpre = 0;
            for (int ww = 0; ww < w; ++ww) wpre += sm.wsum[ww];
            sm.tile_start[tid] = wpre + inc - tot;
        }
        // decoupled look-back over the item's earlier tiles for this digit's global base;
        // each round issues the loads of kLookAhead predecessors at once
        {
            constexpr int kLookAhead = 8;
            const int dg = tid;
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
        // reorder through shared memory: rank[j] becomes the position in the sorted tile
#pragma unroll
        for (int j = 0; j < kSortIPT; ++j) {
            const uint32_t dg = (uint32_t)(key[j] >> shift) & 255u;
            rank[j] += sm.tile_start[dg] + sm.wcnt[w][dg];
            sm.t.kv.keys[rank[j]] = key[j];
            sm.t.kv.vals[rank[j]] = val[j];
        }
        __syncthreads();
        const int64_t item_end = it.start + it.ntiles * kTile;
        uint32_t out[kSortIPT];  // output position of sorted-tile position tid + j * kSortThreads
#pragma unroll
        for (int j = 0; j < kSortIPT; ++j) {
            const int i = tid + j * kSortThreads;
            const K k = sm.t.kv.keys[i];
            const uint32_t dg = (uint32_t)(k >> shift) & 255u;
            out[j] = sm.gbase[dg] + (uint32_t)i - sm.tile_start[dg];
            if ((int64_t)out[j] < item_end) {  // always true unless a look-back wait timed out
                kout[out[j]] = k;
                vout[out[j]] = sm.t.kv.vals[i];
            }
        }
        if (PREFIX) {  // the full keys, through the same shared words
            uint64_t full[kSortIPT];
#pragma unroll
            for (int j = 0; j < kSortIPT; ++j) full[j] = fin[base + w * 32 * kSortIPT + j * 32 + lane];
            __syncthreads();
#pragma unroll
            for (int j = 0; j < kSortIPT; ++j) sm.t.full[rank[j]] = full[j];
            __syncthreads();
#pragma unroll
            for (int j = 0; j < kSortIPT; ++j)
                if ((int64_t)out[j] < item_end) fout[out[j]] = sm.t.full[tid + j * kSortThreads];
        }
        if (__any_sync(0xffffffffu, bad) && lane == 0) atomicOr(a.status, kStatusNonFinite);
        __syncthreads();  // the shared tile is reused by the next tile
    }
}


// ---- the full keys, and runs of equal prefix keys ------------------------------------------
// A run that starts inside a thread's window and reaches past it, its first len points
// seen up to pos (exclusive; last key kprev, descent flag d): walks on while the run
// lasts and returns its length when it is to be listed (it holds a descent), else 0.  A
// run longer than kRunMax is not listed: the length check of its descents
// (check_extent) sends the sort to the fallback.
__device__ __noinline__ int walk_run(const uint32_t* pre, const uint64_t* keys, int64_t end, int64_t pos, uint32_t pk,
                                     uint64_t kprev, int len, bool d) {
    while (pos < end && pre[pos] == pk) {
        if (len >= kRunMax) return 0;
        const uint64_t kk = keys[pos];
        d |= kprev > kk;
        kprev = kk;
        ++len;
        ++pos;
    }
    return d ? len : 0;
}

// A descent in a run of prefix pk that holds points [lo, hi) and may extend below lo
// (down) or from hi on (up): sets the fallback flag when the run is longer than kRunMax.
__device__ __noinline__ void check_extent(const SortArgs& a, const uint32_t* pre, int64_t start, int64_t end,
                                          int64_t lo, int64_t hi, uint32_t pk, bool down, bool up) {
    while (down && lo > start && pre[lo - 1] == pk && hi - lo <= kRunMax) --lo;
    while (up && hi < end && pre[hi] == pk && hi - lo <= kRunMax) ++hi;
    if (hi - lo > kRunMax) atomicOr(&a.pplan->fallback, 1u);
}

// One block per tile (grid-stride), each thread 16 consecutive positions of the sorted
// prefix keys and full keys: the window's neighbour pairs with equal prefixes (bit mask
// eqm) and, among them, keys out of order (a descent, mask dsm).  A run that starts in
// the window is listed when it holds a descent, and followed past the window by
// walk_run when it reaches beyond it; a descent in a run that reaches outside the
// window also has its run's length checked.  Neither walk happens for runs inside one
// window, which are nearly all of them.
__global__ void __launch_bounds__(256) k_sort_detect(SortArgs a) {
    if (a.plan->merge || (*a.status & kStatusSortTimeout)) return;
    __shared__ int s_item;
    const int fb = a.pplan->final_buf;
    const uint32_t* pre = a.pre + (fb ? a.Ppad : 0);
    const uint64_t* keys = fb ? a.keysB : a.keysA;
    uint64_t* runs = reinterpret_cast<uint64_t*>(a.pre + (fb ? 0 : a.Ppad));
    const int64_t T = *a.total_tiles;
    for (int64_t t = blockIdx.x; t < T; t += gridDim.x) {
        if (threadIdx.x == 0) s_item = item_of_tile(a.items, a.B, t);
        __syncthreads();
        const Item it = a.items[s_item];
        const int64_t start = it.start, end = it.start + it.nsrc + it.ntgt;
        const int64_t g0 = t * kTile + threadIdx.x * kSortIPT;  // a multiple of 16
        uint32_t p[kSortIPT];
        uint64_t k[kSortIPT];
        uint32_t lst = 0, eqm = 0;
        int xlen = 0, xq = 0;
#pragma unroll
        for (int q = 0; q < kSortIPT / 4; ++q) {
            const uint4 pp = reinterpret_cast<const uint4*>(pre + g0)[q];
            p[4 * q] = pp.x, p[4 * q + 1] = pp.y, p[4 * q + 2] = pp.z, p[4 * q + 3] = pp.w;
        }
#pragma unroll
        for (int q = 0; q < kSortIPT / 2; ++q) {
            const ulonglong2 kk = reinterpret_cast<const ulonglong2*>(keys + g0)[q];
            k[2 * q] = kk.x, k[2 * q + 1] = kk.y;
        }
        if (g0 + 1 < end) {
            const uint32_t p16 = g0 + kSortIPT < end ? pre[g0 + kSortIPT] : ~p[kSortIPT - 1];
            uint32_t dsm = 0;
#pragma unroll
            for (int q = 0; q < kSortIPT; ++q) {
                const uint32_t pn = q + 1 < kSortIPT ? p[q + 1] : p16;
                const bool e = g0 + q + 1 < end && p[q] == pn;
                eqm |= (uint32_t)e << q;
                if (q + 1 < kSortIPT && e && k[q] > k[q + 1]) dsm |= 1u << q;
            }
            if (eqm) {
                uint64_t k16 = 0;
                if ((eqm >> 15) & 1u) {
                    k16 = keys[g0 + kSortIPT];
                    if (k[kSortIPT - 1] > k16) dsm |= 1u << 15;
                }
                const bool before = g0 > start && pre[g0 - 1] == p[0];  // the first run began earlier
                // runs that start in the window: bit q of lst for a run inside it with a
                // descent; the run that reaches past the window is followed by walk_run
                uint32_t st = eqm & ~((eqm << 1) | (before ? 1u : 0u));
                while (st) {
                    const int q = __ffs(st) - 1;
                    st &= st - 1;
                    const int j = __ffs(~(eqm >> q)) - 1;  // equal pairs from q: points q .. q + j
                    const bool d = (dsm & (((1u << j) - 1u) << q)) != 0;
                    if (q + j == kSortIPT) {
                        xlen = walk_run(pre, keys, end, g0 + kSortIPT + 1, p[q], k16, j + 1, d);
                        xq = q;
                    } else if (d) {
                        lst |= 1u << q;
                    }
                }
                // descents in runs that reach outside the window
                const int j0 = __ffs(~eqm) - 1;  // equal pairs from point 0
                const uint32_t first = before ? (1u << j0) - 1u : 0u;
                if (dsm & first) check_extent(a, pre, start, end, g0, g0 + j0 + 1, p[0], true, j0 == kSortIPT);
                if ((eqm >> 15) & 1u && !(before && j0 == kSortIPT)) {
                    const int tl = __clz(~(eqm << 16));  // equal pairs that end at pair 15
                    if (dsm & (((1u << tl) - 1u) << (kSortIPT - tl)))
                        check_extent(a, pre, start, end, g0 + kSortIPT - tl, g0 + kSortIPT + 1, p[kSortIPT - 1], false,
                                     true);
                }
            }
        }
        // the listed runs go out with one counter update per warp
        const uint32_t cnt = __popc(lst) + (xlen > 0 ? 1u : 0u);
        uint32_t inc = cnt;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t t2 = __shfl_up_sync(0xffffffffu, inc, o);
            if ((threadIdx.x & 31) >= o) inc += t2;
        }
        uint32_t wbase = 0;
        if ((threadIdx.x & 31) == 31 && inc) wbase = atomicAdd(&a.pplan->nruns, inc);
        wbase = __shfl_sync(0xffffffffu, wbase, 31);
        if (cnt) {
            int64_t idx = (int64_t)wbase + inc - cnt;
            if (idx + cnt > a.Ppad / 2) {
                atomicOr(&a.pplan->fallback, 1u);
            } else {
                while (lst) {
                    const int q = __ffs(lst) - 1;
                    lst &= lst - 1;
                    const int len = __ffs(~(eqm >> q));  // points q .. q + j
                    runs[idx++] = (uint64_t)(g0 + q) | ((uint64_t)len << 40);
                }
                if (xlen > 0) runs[idx] = (uint64_t)(g0 + xq) | ((uint64_t)xlen << 40);
            }
        }
        __syncthreads();  // s_item is rewritten for the next tile
    }
}

// One thread per listed run (at most kRunMax points, nearly always two or three): an
// insertion sort by (key, code) in local arrays, written back in place (the final
// buffer of the prefix sort).
__global__ void __launch_bounds__(256) k_sort_fixup(SortArgs a) {
    if (a.plan->merge || a.pplan->fallback || (*a.status & kStatusSortTimeout)) return;
    const int fb = a.pplan->final_buf;
    uint64_t* keys = fb ? a.keysB : a.keysA;
    uint32_t* vals = fb ? a.valsB : a.valsA;
    const uint64_t* runs = reinterpret_cast<const uint64_t*>(a.pre + (fb ? 0 : a.Ppad));
    const int64_t n = min((int64_t)a.pplan->nruns, a.Ppad / 2);
    for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < n; r += (int64_t)gridDim.x * blockDim.x) {
        const uint64_t e = runs[r];
        const int64_t s = (int64_t)(e & ((1ull << 40) - 1));
        const int len = min((int)(e >> 40), kRunMax);
        uint64_t k[kRunMax];
        uint32_t v[kRunMax];
        for (int i = 0; i < len; ++i) {
            const uint64_t ki = keys[s + i];
            const uint32_t vi = vals[s + i];
            int j = i;
            while (j > 0 && (k[j - 1] > ki || (k[j - 1] == ki && v[j - 1] > vi))) {
                k[j] = k[j - 1];
                v[j] = v[j - 1];
                --j;
            }
            k[j] = ki;
            v[j] = vi;
        }
        for (int i = 0; i < len; ++i) {
            keys[s + i] = k[i];
            vals[s + i] = v[i];
        }
    }
}

// Before the full sort of a fallback: clear the look-back words of the prefix digits
// and the histograms.
__global__ void __launch_bounds__(256) k_sort_fb_prepare(SortArgs a) {
    if (!a.pplan->fallback || (*a.status & kStatusSortTimeout)) return;
    const size_t nd = (size_t)kPrefixDigits * a.desc_stride, nh = (size_t)a.B * kSortDigits * 256;
    const size_t stride = (size_t)gridDim.x * blockDim.x;
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < nd; i += stride) a.desc[i] = 0;
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < nh; i += stride) a.hist[i] = 0;
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

cudaError_t launch_sort(const SortArgs& a, cudaStream_t st) {
    if (a.max_tiles <= 0) return cudaSuccess;
    int dev = 0, sms = 0, occ = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int smem32 = (int)sizeof(SortSmem<uint32_t>), smem64 = (int)sizeof(SortSmem<uint64_t>);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_sort_pass<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem32);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_sort_pass<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem64);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_sort_merge, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sizeof(MergeSmem));
    if (e == cudaSuccess)
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_sort_pass<false>, kSortThreads, smem64);

    if (e != cudaSuccess) return e;
    const int64_t tiles = a.max_tiles;
    const int hist_blocks = (int)std::min<int64_t>(tiles, (int64_t)sms * 4);
    // prefix sort (or the merge of presorted runs)
    k_sort_range<<<hist_blocks, 256, 0, st>>>(a);
    k_prefix_maps<<<(a.B + 255) / 256, 256, 0, st>>>(a);
    k_sort_hist<true><<<hist_blocks, 256, 0, st>>>(a);
    k_sort_plan<true><<<a.B, 256, 0, st>>>(a);
    k_sort_chain<<<1, 1, 0, st>>>(a);
    for (int d = 0; d < kPrefixDigits; ++d) k_sort_pass<true><<<(unsigned)tiles, kSortThreads, smem32, st>>>(a, d);
    k_sort_merge<<<(unsigned)tiles, kSortThreads, sizeof(MergeSmem), st>>>(a);
    k_sort_detect<<<(unsigned)std::min<int64_t>(tiles, (int64_t)sms * 8), 256, 0, st>>>(a);
    k_sort_fixup<<<sms * 16, 256, 0, st>>>(a);
    // full sort after a fallback: grids of resident size, so that their blocks exit at
    // once when there is none
    k_sort_fb_prepare<<<sms * 4, 256, 0, st>>>(a);
    k_sort_hist<false><<<hist_blocks, 256, 0, st>>>(a);
    k_sort_plan<false><<<a.B, 256, 0, st>>>(a);
    k_sort_chain_full<<<1, 1, 0, st>>>(a);
    const int full_grid = (int)std::min<int64_t>(tiles, (int64_t)std::max(occ, 1) * sms);
    for (int d = 0; d < kSortDigits; ++d) k_sort_pass<false><<<full_grid, kSortThreads, smem64, st>>>(a, d);
    return cudaGetLastError();
}

__global__ void k_copy_perm(const uint32_t* __restrict__ va, const uint32_t* __restrict__ vb, const SortPlan* plan,
                            int64_t P, uint32_t* __restrict__ perm) {
    const uint32_t* v = plan->final_buf == 1 ? vb : va;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < P; i += (int64_t)gridDim.x * blockDim.x)
        perm[i] = v[i];
}

// The sorted codes of a single item with the roles of its points exchanged: old
// sources [0, n_src) become targets, old targets [n_src, n_src + n_tgt) sources (padding
// codes stay).  The order is kept, so on equal coordinates the new targets come first.
__global__ void k_swap_codes(uint32_t* __restrict__ va, uint32_t* __restrict__ vb, const SortPlan* plan, int64_t P,
                             int64_t n_src, int64_t n_tgt) {
    uint32_t* v = plan->final_buf == 1 ? vb : va;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < P; i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t q = v[i];
        if (q < n_src) v[i] = (uint32_t)(q + n_tgt);
        else if (q < n_src + n_tgt) v[i] = (uint32_t)(q - n_src);
    }
}

cudaError_t launch_swap_codes(const SortArgs& a, int64_t P, int64_t n_src, int64_t n_tgt, cudaStream_t st) {
    if (P <= 0) return cudaSuccess;
    const int blocks = (int)std::min<int64_t>((P + 255) / 256, 152 * 16);
    k_swap_codes<<<blocks, 256, 0, st>>>(a.valsA, a.valsB, a.plan, P, n_src, n_tgt);
    return cudaGetLastError();
}

cudaError_t launch_copy_perm(const SortArgs& a, int64_t P, uint32_t* perm, cudaStream_t st) {
    if (P <= 0) return cudaSuccess;
    int blocks = (int)std::min<int64_t>((P + 255) / 256, 152 * 16);
    k_copy_perm<<<blocks, 256, 0, st>>>(a.valsA, a.valsB, a.plan, P, perm);
    return cudaGetLastError();
}

}  // namespace fgt1d
