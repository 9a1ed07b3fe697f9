// FP64 instantiations of the sweep kernels (tile = 128 threads x 32 points).
#include "sweep.cuh"

namespace fgt1d {

namespace {
constexpr int kT = 128, kR = 32;

template <int NE>
cudaError_t run(const SweepArgs& a, const SweepConsts& c, cudaStream_t st, cudaEvent_t mid) {
    const size_t smem = SweepSmem<double, NE, kT, kR>::bytes;
    auto kf = k_sweep_fwd<double, NE, kT, kR>;
    auto kb = k_sweep_bwd<double, NE, kT, kR>;
    cudaError_t e = cudaFuncSetAttribute(kf, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    e = cudaFuncSetAttribute(kb, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    kf<<<(unsigned)a.tiles, kT, smem, st>>>(a, c);
    if (mid && (e = cudaEventRecord(mid, st)) != cudaSuccess) return e;
    kb<<<(unsigned)a.tiles, kT, smem, st>>>(a, c);
    return cudaGetLastError();
}
}  // namespace

int sweep_tile_f64() { return kT * kR; }

cudaError_t launch_sweeps_f64(const SweepArgs& a, const SweepConsts& c, cudaStream_t st, cudaEvent_t mid) {
    switch (c.n_e) {
        case 1: return run<1>(a, c, st, mid);
        case 2: return run<2>(a, c, st, mid);
        case 3: return run<3>(a, c, st, mid);
        case 4: return run<4>(a, c, st, mid);
        case 5: return run<5>(a, c, st, mid);
        case 6: return run<6>(a, c, st, mid);
        case 7: return run<7>(a, c, st, mid);
        case 8: return run<8>(a, c, st, mid);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace fgt1d
