// FP32 sweeps for the transform (value channel).
#include "sweep_launch.cuh"

namespace fgt1d {

int sweep_tile_f32() { return kT32 * kR32; }

cudaError_t launch_sweeps_f32(const SweepArgs& a, const SweepConsts& c, cudaStream_t st, cudaEvent_t mid, int ev) {
    if (ev == 1) return run_sweeps_ne<float, kT32, kR32, 1>(a, c, st, mid);
    return launch_sweeps_f32_ev(a, c, st, mid, ev);
}

}  // namespace fgt1d
