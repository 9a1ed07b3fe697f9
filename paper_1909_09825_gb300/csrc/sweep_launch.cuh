// Launch helpers shared by the sweep instantiation units.
#pragma once

#include "sweep.cuh"

namespace fgt1d {

template <typename Real, int T, int R, int EV, int NE>
cudaError_t run_sweep_pair(const SweepArgs& a, const SweepConsts& c, cudaStream_t st, cudaEvent_t mid) {
    const size_t smem = SweepSmem<Real, SweepGroup<Real, NE, T, R, EV, false>::NG, T, R>::bytes;
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

// Tile shapes (threads x points per thread, 4096 points): shape 0 = 128 x 32,
// shape 1 = 256 x 16.  The coincidence scan runs as 128 x 32.
constexpr int kT64 = 128, kR64 = 32;
template <int S>
struct Shape;
template <>
struct Shape<0> { static constexpr int T = 128, R = 32; };
template <>
struct Shape<1> { static constexpr int T = 256, R = 16; };

}  // namespace fgt1d
