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

__device__ __forceinline__ double merged_coord(const double* x, const double* y, int64_t N, int64_t q) {
    return q < N ? y[q] : x[q - N];
}

// ---- histogram of all digits --------------------------------------------------------------
__global__ void __launch_bounds__(256) k_sort_hist(const double* __restrict__ x, const double* __restrict__ y,
                                                   int64_t N, int64_t P, uint32_t* __restrict__ hist,
                                                   uint32_t* __restrict__ status) {
    __shared__ uint32_t sh[kSortDigits][256];
    for (int i = threadIdx.x; i < kSortDigits * 256; i += blockDim.x) (&sh[0][0])[i] = 0;
    __syncthreads();
    uint32_t last[kSortDigits], run[kSortDigits];
#pragma unroll
    for (int d = 0; d < kSortDigits; ++d) { last[d] = 0; run[d] = 0; }
    bool bad = false;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < P; q += stride) {
        double c = merged_coord(x, y, N, q);
        bad |= coord_nonfinite(c);
        uint64_t k = coord_key(c);
#pragma unroll
        for (int d = 0; d < kSortDigits; ++d) {
            uint32_t dg = (uint32_t)(k >> (8 * d)) & 255u;
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
    if (__any_sync(0xffffffffu, bad) && (threadIdx.x & 31) == 0) atomicOr(status, kStatusNonFinite);
    __syncthreads();
    for (int i = threadIdx.x; i < kSortDigits * 256; i += blockDim.x) {
        uint32_t v = (&sh[0][0])[i];
        if (v) atomicAdd(&hist[i], v);
    }
}

// ---- bucket offsets and the pass plan (one block of 256 threads) ---------------------------
__global__ void __launch_bounds__(256) k_sort_plan(const uint32_t* __restrict__ hist, uint32_t* __restrict__ offs,
                                                   SortPlan* __restrict__ plan, int64_t P) {
    __shared__ uint32_t scan[256];
    __shared__ int active[kSortDigits];
    const int t = threadIdx.x;
    for (int d = 0; d < kSortDigits; ++d) {
        uint32_t v = hist[d * 256 + t];
        scan[t] = v;
        __syncthreads();
        for (int o = 1; o < 256; o <<= 1) {
            uint32_t add = t >= o ? scan[t - o] : 0;
            __syncthreads();
            scan[t] += add;
            __syncthreads();
        }
        offs[d * 256 + t] = scan[t] - v;  // exclusive
        int full = (P > 0 && (int64_t)v == P);
        int any_full = __syncthreads_or(full);
        if (t == 0) active[d] = !any_full;
        __syncthreads();
    }
    if (t == 0) {
        int cur = -1, n_active = 0;
        for (int d = 0; d < kSortDigits; ++d) {
            plan->active[d] = 0;
            plan->src[d] = 0;
            plan->dst[d] = 0;
        }
        for (int d = 0; d < kSortDigits; ++d) {
            if (!active[d]) continue;
            plan->active[d] = 1;
            plan->src[d] = cur;
            plan->dst[d] = (cur == 0) ? 1 : 0;
            cur = plan->dst[d];
            ++n_active;
        }
        if (n_active == 0) {  // every key equal (or P <= 1): one pass materialises keys/indices
            plan->active[0] = 1;
            plan->src[0] = -1;
            plan->dst[0] = 0;
            cur = 0;
        }
        plan->final_buf = cur;
    }
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
    const int src = pl->src[d], dst = pl->dst[d];
    const uint64_t* __restrict__ kin = src == 1 ? a.keysB : a.keysA;
    const uint32_t* __restrict__ vin = src == 1 ? a.valsB : a.valsA;
    uint64_t* __restrict__ kout = dst == 1 ? a.keysB : a.keysA;
    uint32_t* __restrict__ vout = dst == 1 ? a.valsB : a.valsA;
    const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
    const int shift = 8 * d;

    if (tid == 0) sm.tile_id = atomicAdd(&a.tile_ctr[d], 1u);
    for (int i = tid; i < (kSortThreads / 32) * 256; i += kSortThreads) (&sm.wcnt[0][0])[i] = 0;
    __syncthreads();
    const uint32_t tile = sm.tile_id;
    const int64_t base = (int64_t)tile * kSortTile;
    const int nvalid = (int)min((int64_t)kSortTile, a.P - base);

    // load (warp-striped: warp w owns items [w*32*IPT, (w+1)*32*IPT), slot j covers 32 consecutive items)
    uint64_t key[kSortIPT];
    uint32_t val[kSortIPT];
    uint32_t rank[kSortIPT];
#pragma unroll
    for (int j = 0; j < kSortIPT; ++j) {
        const int li = w * 32 * kSortIPT + j * 32 + lane;
        const int64_t g = base + li;
        if (li < nvalid) {
            if (src < 0) {
                double c = merged_coord(a.x, a.y, a.N, g);
                key[j] = coord_key(c);
                val[j] = (uint32_t)g;
            } else {
                key[j] = kin[g];
                val[j] = vin[g];
            }
        } else {
            key[j] = 0;
            val[j] = 0;
        }
    }
    // stable warp ranking per slot: the lanes holding the same digit are found with
    // eight ballots (one per digit bit), for all slots first (independent work); then,
    // slot by slot, every lane reads the warp's running count for its digit and the
    // lowest peer adds the slot's count
    unsigned peers[kSortIPT];
#pragma unroll
    for (int j = 0; j < kSortIPT; ++j) {
        const int li = w * 32 * kSortIPT + j * 32 + lane;
        const uint32_t dg = (uint32_t)(key[j] >> shift) & 255u;
        unsigned pm = __ballot_sync(0xffffffffu, li < nvalid);
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
        const int li = w * 32 * kSortIPT + j * 32 + lane;
        const bool valid = li < nvalid;
        const uint32_t dg = (uint32_t)(key[j] >> shift) & 255u;
        const uint32_t old = valid ? sm.wcnt[w][dg] : 0u;
        __syncwarp();
        if (valid) {
            rank[j] = old + __popc(peers[j] & lt);
            if ((peers[j] & lt) == 0) sm.wcnt[w][dg] = old + __popc(peers[j]);
        }
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
        // warp inclusive scan
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
    // decoupled look-back for this digit's global base; each round issues the loads of
    // kLookAhead predecessors at once so the walk costs one round trip per kLookAhead tiles
    {
        constexpr int kLookAhead = 8;
        const int dg = tid;
        uint64_t* desc = a.desc + (size_t)d * a.desc_stride;
        uint32_t excl = 0;
        if (tile == 0) {
            st_volatile_u64(&desc[dg], kDescInc | (uint64_t)tot);
        } else {
            st_volatile_u64(&desc[(size_t)tile * 256 + dg], kDescAgg | (uint64_t)tot);
            int64_t j = (int64_t)tile - 1;
            bool done = false;
            while (!done) {
                uint64_t v[kLookAhead];
#pragma unroll
                for (int q = 0; q < kLookAhead; ++q)
                    v[q] = (j - q >= 0) ? ld_volatile_u64(&desc[(size_t)(j - q) * 256 + dg]) : kDescInc;
#pragma unroll
                for (int q = 0; q < kLookAhead; ++q) {
                    if (done) break;
                    uint64_t x = v[q];
                    if ((x >> 62) == 0) {
                        const long long t0 = clock64();
                        while (((x = ld_volatile_u64(&desc[(size_t)(j - q) * 256 + dg])) >> 62) == 0) {
                            if (clock64() - t0 > kSpinLimitCycles) {
                                atomicOr(a.status, kStatusTimeout);
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
        sm.gbase[dg] = a.offs[d * 256 + dg] + excl;
    }
    __syncthreads();
    // reorder through shared memory
#pragma unroll
    for (int j = 0; j < kSortIPT; ++j) {
        const int li = w * 32 * kSortIPT + j * 32 + lane;
        if (li < nvalid) {
            const uint32_t dg = (uint32_t)(key[j] >> shift) & 255u;
            const uint32_t pos = sm.tile_start[dg] + sm.wcnt[w][dg] + rank[j];
            sm.keys[pos] = key[j];
            sm.vals[pos] = val[j];
        }
    }
    __syncthreads();
    for (int i = tid; i < nvalid; i += kSortThreads) {
        const uint64_t k = sm.keys[i];
        const uint32_t dg = (uint32_t)(k >> shift) & 255u;
        const uint32_t o = sm.gbase[dg] + (uint32_t)i - sm.tile_start[dg];
        if ((int64_t)o < a.P) {  // always true unless a look-back wait timed out
            kout[o] = k;
            vout[o] = sm.vals[i];
        }
    }
}

size_t sort_pass_smem() { return sizeof(SortSmem); }

cudaError_t launch_sort(const SortArgs& a, cudaStream_t st) {
    if (a.P <= 0) return cudaSuccess;
    cudaError_t e = cudaFuncSetAttribute(k_sort_pass, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)sizeof(SortSmem));
    if (e != cudaSuccess) return e;
    int hist_blocks = (int)std::min<int64_t>((a.P + 255) / 256, 152 * 8);
    k_sort_hist<<<hist_blocks, 256, 0, st>>>(a.x, a.y, a.N, a.P, a.hist, a.status);
    k_sort_plan<<<1, 256, 0, st>>>(a.hist, a.offs, a.plan, a.P);
    const int64_t tiles = (a.P + kSortTile - 1) / kSortTile;
    for (int d = 0; d < kSortDigits; ++d)
        k_sort_pass<<<(unsigned)tiles, kSortThreads, sizeof(SortSmem), st>>>(a, d);
    return cudaGetLastError();
}

}  // namespace fgt1d

namespace fgt1d {

__global__ void k_copy_perm(const uint32_t* __restrict__ va, const uint32_t* __restrict__ vb, const SortPlan* plan,
                            int64_t P, uint32_t* __restrict__ perm) {
    const uint32_t* v = plan->final_buf == 1 ? vb : va;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < P; i += (int64_t)gridDim.x * blockDim.x)
        perm[i] = v[i];
}

cudaError_t launch_copy_perm(const SortArgs& a, uint32_t* perm, cudaStream_t st) {
    if (a.P <= 0) return cudaSuccess;
    int blocks = (int)std::min<int64_t>((a.P + 255) / 256, 152 * 16);
    k_copy_perm<<<blocks, 256, 0, st>>>(a.valsA, a.valsB, a.plan, a.P, perm);
    return cudaGetLastError();
}

}  // namespace fgt1d
