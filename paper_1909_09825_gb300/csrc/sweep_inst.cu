// The sweep kernels of one precision, tile shape and term count, compiled once per
// combination (-DFGT_SW_PREC=0 FP64, 1 FP32, 2 double-float; -DFGT_SW_SHAPE=0 128 x 32,
// 1 256 x 16; -DFGT_SW_NE=1..8) so that the build runs them in parallel.  Each unit
// defines sweeps_<prec>_s<shape>_ne<NE>(..., ev), the launcher of the forward +
// backward pair for evaluation channels ev.
#include "sweep_launch.cuh"

#if !defined(FGT_SW_PREC) || !defined(FGT_SW_NE) || !defined(FGT_SW_SHAPE)
#error "sweep_inst.cu is compiled once per precision, tile shape and term count"
#endif

#define FGT_CAT_(a, b, c, d) a##b##c##d
#define FGT_CAT(a, b, c, d) FGT_CAT_(a, b, c, d)

namespace fgt1d {

namespace {
constexpr int kT = Shape<FGT_SW_SHAPE>::T, kR = Shape<FGT_SW_SHAPE>::R;
}

#if FGT_SW_PREC == 0
cudaError_t FGT_CAT(sweeps_f64_s, FGT_SW_SHAPE, _ne, FGT_SW_NE)(const SweepArgs& a, const SweepConsts& c,
                                                                cudaStream_t st, cudaEvent_t mid, int ev) {
    switch (ev) {
        case 1: return run_sweep_pair<double, kT, kR, 1, FGT_SW_NE>(a, c, st, mid);
        case 2: return run_sweep_pair<double, kT, kR, 2, FGT_SW_NE>(a, c, st, mid);
        case 3: return run_sweep_pair<double, kT, kR, 3, FGT_SW_NE>(a, c, st, mid);
        default: return cudaErrorInvalidValue;
    }
}
#if FGT_SW_NE == 1 && FGT_SW_SHAPE == 0
cudaError_t launch_coincidence(const SweepArgs& a, const SweepConsts& c, cudaStream_t st) {
    const size_t smem = SweepSmem<double, 1, kT64, kR64>::bytes;
    auto kf = k_sweep_fwd<double, 1, kT64, kR64, 1, true>;
    cudaError_t e = cudaFuncSetAttribute(kf, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    kf<<<persistent_grid(kf, kT64, smem, a.max_tiles), kT64, smem, st>>>(a, c);
    return cudaGetLastError();
}

// The last position of sorted position p's run of equal keys (of n): a galloping search
// (steps 1, 2, 4, ... while the key stays equal, then bisection of the last step), at
// most ~2 log2(n) key loads for a run of any length and one for a point without ties.
__device__ __forceinline__ int64_t run_last(const uint64_t* __restrict__ keys, int64_t p, int64_t n) {
    const uint64_t k = keys[p];
    if (p + 1 >= n || keys[p + 1] != k) return p;
    int64_t lo = p + 1, step = 1;  // keys[lo] == k
    while (lo + step < n && keys[lo + step] == k) {
        lo += step;
        step <<= 1;
    }
    int64_t hi = min(lo + step, n);  // keys[hi] != k, or hi == n
    while (hi - lo > 1) {
        const int64_t mid = lo + (hi - lo) / 2;
        if (keys[mid] == k) lo = mid;
        else hi = mid;
    }
    return lo;
}

// One thread per sorted position p of a single item of n identical points.
__global__ void __launch_bounds__(256) k_self_exact(const SweepArgs a, const double* __restrict__ F, int64_t n,
                                                    double cf, double* __restrict__ u) {
    const bool bufB = a.plan->final_buf == 1;
    const uint64_t* __restrict__ keys = bufB ? a.keysB : a.keysA;
    const uint32_t* __restrict__ vals = bufB ? a.valsB : a.valsA;
    if (*(volatile const uint32_t*)a.status & kStatusSortTimeout) return;  // sorted codes not valid
    for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < n; p += (int64_t)gridDim.x * blockDim.x)
        u[vals[p]] += cf * F[run_last(keys, p, n)];
}

// One thread per sorted position p of a single item of n points; targets only.
__global__ void __launch_bounds__(256) k_coinc_gather(const SweepArgs a, const double* __restrict__ F, int64_t n,
                                                      double* __restrict__ A) {
    if (*(volatile const uint32_t*)a.status & kStatusSortTimeout) return;  // sorted codes not valid
    if (!*(volatile const uint32_t*)a.ties) return;  // no coincident points: A stays zero
    const bool bufB = a.plan->final_buf == 1;
    const uint64_t* __restrict__ keys = bufB ? a.keysB : a.keysA;
    const uint32_t* __restrict__ vals = bufB ? a.valsB : a.valsA;
    for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < n; p += (int64_t)gridDim.x * blockDim.x) {
        const int64_t v = vals[p];
        if (v >= a.N && v < n) A[v - a.N] = F[run_last(keys, p, n)];  // (codes of points are below n)
    }
}

cudaError_t launch_coinc_gather(const SweepArgs& a, const double* F, int64_t n, double* A, cudaStream_t st) {
    if (n <= 0 || !a.ties) return cudaSuccess;
    const int blocks = (int)std::min<int64_t>((n + 255) / 256, 152 * 8);
    k_coinc_gather<<<blocks, 256, 0, st>>>(a, F, n, A);
    return cudaGetLastError();
}

cudaError_t launch_self_exact(const SweepArgs& a, const double* F, int64_t n, double cf, double* u, cudaStream_t st) {
    if (n <= 0) return cudaSuccess;
    const int blocks = (int)std::min<int64_t>((n + 255) / 256, 152 * 8);
    k_self_exact<<<blocks, 256, 0, st>>>(a, F, n, cf, u);
    return cudaGetLastError();
}

cudaError_t launch_fill_table(const SweepArgs& a, const SweepConsts& c, int shape, bool dfloat_entries,
                              cudaStream_t st) {
    const int sT = shape == 1 ? Shape<1>::T : Shape<0>::T, sR = shape == 1 ? Shape<1>::R : Shape<0>::R;
    if (dfloat_entries) k_fill_table<256, dfloat><<<(unsigned)a.max_tiles, 256, 0, st>>>(a, c, sT, sR);
    else k_fill_table<256, double><<<(unsigned)a.max_tiles, 256, 0, st>>>(a, c, sT, sR);
    return cudaGetLastError();
}

__global__ void k_geometry_check(const uint64_t* tag, uint64_t expect, int64_t* total_tiles, uint32_t* status) {
    if (*tag != expect) {
        *total_tiles = 0;
        atomicOr(status, kStatusBadArg);
    }
}
__global__ void k_geometry_tag(uint64_t* tag, uint64_t value) { *tag = value; }

cudaError_t launch_geometry_check(const uint64_t* tag, uint64_t expect, int64_t* total_tiles, uint32_t* status,
                                  cudaStream_t st) {
    k_geometry_check<<<1, 1, 0, st>>>(tag, expect, total_tiles, status);
    return cudaGetLastError();
}
cudaError_t launch_geometry_tag(uint64_t* tag, uint64_t value, cudaStream_t st) {
    k_geometry_tag<<<1, 1, 0, st>>>(tag, value);
    return cudaGetLastError();
}
#endif
#elif FGT_SW_PREC == 1
cudaError_t FGT_CAT(sweeps_f32_s, FGT_SW_SHAPE, _ne, FGT_SW_NE)(const SweepArgs& a, const SweepConsts& c,
                                                                cudaStream_t st, cudaEvent_t mid, int ev) {
    switch (ev) {
        case 1: return run_sweep_pair<float, kT, kR, 1, FGT_SW_NE>(a, c, st, mid);
        case 2: return run_sweep_pair<float, kT, kR, 2, FGT_SW_NE>(a, c, st, mid);
        case 3: return run_sweep_pair<float, kT, kR, 3, FGT_SW_NE>(a, c, st, mid);
        default: return cudaErrorInvalidValue;
    }
}
#elif FGT_SW_PREC == 2
cudaError_t FGT_CAT(sweeps_df_s, FGT_SW_SHAPE, _ne, FGT_SW_NE)(const SweepArgs& a, const SweepConsts& c,
                                                               cudaStream_t st, cudaEvent_t mid, int ev) {
    if (ev != 1) return cudaErrorInvalidValue;
    return run_sweep_pair<dfloat, kT, kR, 1, FGT_SW_NE>(a, c, st, mid);
}
#else
#error "FGT_SW_PREC must be 0, 1 or 2"
#endif

}  // namespace fgt1d
