// FP32 sweeps with the derivative channel (gradients).
#include "sweep_launch.cuh"

namespace fgt1d {

cudaError_t launch_sweeps_f32_ev(const SweepArgs& a, const SweepConsts& c, cudaStream_t st, cudaEvent_t mid, int ev) {
    if (ev == 2) return run_sweeps_ne<float, kT32, kR32, 2>(a, c, st, mid);
    if (ev == 3) return run_sweeps_ne<float, kT32, kR32, 3>(a, c, st, mid);
    return cudaErrorInvalidValue;
}

}  // namespace fgt1d
