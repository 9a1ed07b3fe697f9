// Launch helpers shared by the sweep instantiation units.
#pragma once

#include "sweep.cuh"

namespace fgt1d {

template <typename Real, int T, int R, int EV, int NE>
cudaError_t run_sweep_pair(const SweepArgs& a, const SweepConsts& c, cudaStream_t st, cudaEvent_t mid) {
    const size_t smem = SweepSmem<Real, NE, T, R>::bytes;
    auto kf = k_sweep_fwd<Real, NE, T, R, EV, false>;
    auto kb = k_sweep_bwd<Real, NE, T, R, EV>;
    cudaError_t e = cudaFuncSetAttribute(kf, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    e = cudaFuncSetAttribute(kb, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    kf<<<(unsigned)a.max_tiles, T, smem, st>>>(a, c);
    if (mid && (e = cudaEventRecord(mid, st)) != cudaSuccess) return e;
    kb<<<(unsigned)a.max_tiles, T, smem, st>>>(a, c);
    return cudaGetLastError();
}

template <typename Real, int T, int R, int EV>
cudaError_t run_sweeps_ne(const SweepArgs& a, const SweepConsts& c, cudaStream_t st, cudaEvent_t mid) {
    switch (c.n_e) {
        case 1: return run_sweep_pair<Real, T, R, EV, 1>(a, c, st, mid);
        case 2: return run_sweep_pair<Real, T, R, EV, 2>(a, c, st, mid);
        case 3: return run_sweep_pair<Real, T, R, EV, 3>(a, c, st, mid);
        case 4: return run_sweep_pair<Real, T, R, EV, 4>(a, c, st, mid);
        case 5: return run_sweep_pair<Real, T, R, EV, 5>(a, c, st, mid);
        case 6: return run_sweep_pair<Real, T, R, EV, 6>(a, c, st, mid);
        case 7: return run_sweep_pair<Real, T, R, EV, 7>(a, c, st, mid);
        case 8: return run_sweep_pair<Real, T, R, EV, 8>(a, c, st, mid);
        default: return cudaErrorInvalidValue;
    }
}

// Tile shapes: FP64 128 threads x 32 points, FP32 256 threads x 16 points.
constexpr int kT64 = 128, kR64 = 32, kT32 = 256, kR32 = 16;

cudaError_t launch_sweeps_f64_ev(const SweepArgs& a, const SweepConsts& c, cudaStream_t st, cudaEvent_t mid, int ev);
cudaError_t launch_sweeps_f32_ev(const SweepArgs& a, const SweepConsts& c, cudaStream_t st, cudaEvent_t mid, int ev);

}  // namespace fgt1d
