// Double-float sweeps for the transform (value channel), 128 threads x 32 points.
#include "sweep_launch.cuh"

namespace fgt1d {

cudaError_t launch_sweeps_df(const SweepArgs& a, const SweepConsts& c, cudaStream_t st, cudaEvent_t mid) {
    return run_sweeps_ne<dfloat, kT64, kR64, 1>(a, c, st, mid);
}

}  // namespace fgt1d
