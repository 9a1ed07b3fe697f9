// Throughput of the pipes that bound this library's kernels, measured on the current
// device (fgt1d_measure_peaks; no counterpart in the paper).  The sweeps are bound by
// the FP64 pipe (FP64 path) or by FP32 issue (FP32 and double-float paths); the SFU
// rates show what an exp/sincos multiplier on the special-function unit would cost.
//
// Each kernel runs kChains independent dependency chains per thread for kIters steps
// on every SM (8 blocks of 256 threads per SM), so that the pipe, not latency, limits
// it; block 0's thread 0 also reads the SM cycle counter and the global nanosecond timer
// over its run, which gives the SM clock during the measurement.  The values kept
// at the end go to memory only under a condition that never holds, so the work is not
// removed.
#include <cuda_runtime.h>
#include <stdint.h>

#include "fgt1d_internal.h"

namespace fgt1d {
namespace {

constexpr int kChains = 16;
constexpr int kIters = 2048;
constexpr int kThreads = 256;

__device__ __forceinline__ unsigned long long global_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__global__ void __launch_bounds__(kThreads) k_peak_dfma(double seed, double* sink, long long* cycles) {
    const long long t0 = clock64();
    const unsigned long long n0 = global_ns();
    double v[kChains];
#pragma unroll
    for (int c = 0; c < kChains; ++c) v[c] = seed + c + threadIdx.x;
    const double b = 1.0 - 1e-9, d = 1e-9;
#pragma unroll 8
    for (int i = 0; i < kIters; ++i)
#pragma unroll
        for (int c = 0; c < kChains; ++c) v[c] = fma(v[c], b, d);
    double s = 0.0;
#pragma unroll
    for (int c = 0; c < kChains; ++c) s += v[c];
    if (s == -1.0) sink[blockIdx.x] = s;
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        cycles[0] = clock64() - t0;
        cycles[1] = (long long)(global_ns() - n0);
    }
}

__global__ void __launch_bounds__(kThreads) k_peak_ffma(float seed, float* sink, long long* cycles) {
    const long long t0 = clock64();
    const unsigned long long n0 = global_ns();
    float v[kChains];
#pragma unroll
    for (int c = 0; c < kChains; ++c) v[c] = seed + c + threadIdx.x;
    const float b = 1.0f - 1e-6f, d = 1e-6f;
#pragma unroll 8
    for (int i = 0; i < kIters; ++i)
#pragma unroll
        for (int c = 0; c < kChains; ++c) v[c] = __fmaf_rn(v[c], b, d);
    float s = 0.f;
#pragma unroll
    for (int c = 0; c < kChains; ++c) s += v[c];
    if (s == -1.0f) sink[blockIdx.x] = s;
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        cycles[0] = clock64() - t0;
        cycles[1] = (long long)(global_ns() - n0);
    }
}

// SFU: ex2.approx (op 0) or sin.approx (op 1), one PTX instruction per step
template <int OP>
__global__ void __launch_bounds__(kThreads) k_peak_sfu(float seed, float* sink, long long* cycles) {
    const long long t0 = clock64();
    const unsigned long long n0 = global_ns();
    float v[kChains];
#pragma unroll
    for (int c = 0; c < kChains; ++c) v[c] = seed * (c + 1) * 1e-3f;
#pragma unroll 8
    for (int i = 0; i < kIters; ++i)
#pragma unroll
        for (int c = 0; c < kChains; ++c) {
            float r;
            if (OP == 0) asm volatile("ex2.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(v[c]));
            else asm volatile("sin.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(v[c]));
            v[c] = r * -0.5f;  // keeps the argument in [-1, 1]
        }
    float s = 0.f;
#pragma unroll
    for (int c = 0; c < kChains; ++c) s += v[c];
    if (s == -1e30f) sink[blockIdx.x] = s;
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        cycles[0] = clock64() - t0;
        cycles[1] = (long long)(global_ns() - n0);
    }
}

}  // namespace
}  // namespace fgt1d

using namespace fgt1d;

extern "C" int fgt1d_measure_peaks(double* out, fgt1d_stream stream) {
    if (!out) return FGT1D_EINVAL;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
        return FGT1D_ECUDA;
    const int blocks = sms * 8;
    void* sink = nullptr;
    long long* cyc = nullptr;
    if (cudaMalloc(&sink, sizeof(double) * blocks) != cudaSuccess) return FGT1D_ECUDA;
    if (cudaMalloc(&cyc, 2 * sizeof(long long)) != cudaSuccess) {
        cudaFree(sink);
        return FGT1D_ECUDA;
    }
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    int r = FGT1D_OK;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) r = FGT1D_ECUDA;
    const double lanes = (double)blocks * kThreads * kChains * kIters;  // operations per launch
    double mhz = 0.0;
    for (int kind = 0; kind < 4 && r == FGT1D_OK; ++kind) {
        float best_ms = 0.f;
        double best_mhz = 0.0;
        for (int rep = 0; rep < 3 && r == FGT1D_OK; ++rep) {  // the first launch warms up
            cudaEventRecord(e0, st);
            if (kind == 0) k_peak_dfma<<<blocks, kThreads, 0, st>>>(1.0, (double*)sink, cyc);
            if (kind == 1) k_peak_ffma<<<blocks, kThreads, 0, st>>>(1.0f, (float*)sink, cyc);
            if (kind == 2) k_peak_sfu<0><<<blocks, kThreads, 0, st>>>(1.0f, (float*)sink, cyc);
            if (kind == 3) k_peak_sfu<1><<<blocks, kThreads, 0, st>>>(1.0f, (float*)sink, cyc);
            cudaEventRecord(e1, st);
            float ms = 0.f;
            long long c[2] = {0, 0};
            if (cudaGetLastError() != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess ||
                cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess ||
                cudaMemcpy(c, cyc, sizeof(c), cudaMemcpyDeviceToHost) != cudaSuccess) {
                r = FGT1D_ECUDA;
                break;
            }
            if (rep > 0 && (best_ms == 0.f || ms < best_ms)) {
                best_ms = ms;
                best_mhz = c[1] > 0 ? 1e3 * (double)c[0] / (double)c[1] : 0.0;
            }
        }
        if (r == FGT1D_OK) {
            const double rate = lanes / (best_ms * 1e-3);  // operations per second
            out[2 * kind] = rate;
            out[2 * kind + 1] = best_mhz > 0 ? rate / (sms * best_mhz * 1e6) : 0.0;  // per SM per cycle
            if (kind == 0) mhz = best_mhz;
        }
    }
    if (r == FGT1D_OK) {
        out[8] = (double)sms;
        out[9] = mhz;
    }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    cudaFree(sink);
    cudaFree(cyc);
    return r;
}
