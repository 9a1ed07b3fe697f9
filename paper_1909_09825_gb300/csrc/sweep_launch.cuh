// Launch helpers shared by the sweep instantiation units.
#pragma once

#include "sweep.cuh"

namespace fgt1d {

// Grid of a sweep kernel.  128-thread tiles run persistent (the CTAs that fit on the
// device at once: its occupancy times the SM count; each loops over tiles taken in order
// from a counter), which measured faster for them (gradient backward at M = N = 2^24,
// n_e = 6: 39.7 -> 36.8 ms); 256-thread tiles run one CTA per tile (the kernel takes a
// single tile), which measured faster for them (headline forward sweep 20.0 ms against
// 20.8 ms with the loop).
template <typename K>
unsigned persistent_grid(K kernel, int threads, size_t smem, int64_t tiles) {
    if (threads >= 256) return (unsigned)tiles;
    int dev = 0, sms = 0, per_sm = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, threads, smem) != cudaSuccess || per_sm < 1)
        return (unsigned)tiles;  // one CTA per tile, as correct (tiles are taken in order either way)
    const int64_t g = (int64_t)per_sm * sms;
    return (unsigned)(g < tiles ? g : tiles);
}

template <typename Real, int T, int R, int EV, int NE>
cudaError_t run_sweep_pair(const SweepArgs& a, const SweepConsts& c, cudaStream_t st, cudaEvent_t mid) {
    const size_t smem = SweepSmem<Real, SweepGroup<Real, NE, T, R, EV, false>::NG, T, R>::bytes;
    auto kf = k_sweep_fwd<Real, NE, T, R, EV, false>;
    auto kb = k_sweep_bwd<Real, NE, T, R, EV>;
    cudaError_t e = cudaFuncSetAttribute(kf, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    e = cudaFuncSetAttribute(kb, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    kf<<<persistent_grid(kf, T, smem, a.max_tiles), T, smem, st>>>(a, c);
    if (mid && (e = cudaEventRecord(mid, st)) != cudaSuccess) return e;
    kb<<<persistent_grid(kb, T, smem, a.max_tiles), T, smem, st>>>(a, c);
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
