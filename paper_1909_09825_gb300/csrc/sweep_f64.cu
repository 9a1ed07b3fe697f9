// FP64 sweeps for the transform (value channel) and the coincidence sums.
#include "sweep_launch.cuh"

namespace fgt1d {

int sweep_tile_f64() { return kT64 * kR64; }

cudaError_t launch_sweeps_f64(const SweepArgs& a, const SweepConsts& c, cudaStream_t st, cudaEvent_t mid, int ev) {
    if (ev == 1) return run_sweeps_ne<double, kT64, kR64, 1>(a, c, st, mid);
    return launch_sweeps_f64_ev(a, c, st, mid, ev);
}

cudaError_t launch_coincidence(const SweepArgs& a, const SweepConsts& c, cudaStream_t st) {
    const size_t smem = SweepSmem<double, 1, kT64, kR64>::bytes;
    auto kf = k_sweep_fwd<double, 1, kT64, kR64, 1, true>;
    cudaError_t e = cudaFuncSetAttribute(kf, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    kf<<<(unsigned)a.max_tiles, kT64, smem, st>>>(a, c);
    return cudaGetLastError();
}

}  // namespace fgt1d
