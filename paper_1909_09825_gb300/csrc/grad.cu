// Gradient assembly of the SOE transform (no counterpart in the paper, which has no
// gradients; the formulas follow from eqs. 1.3 and 4.1-4.6).
//
// For L = sum_i g_i u_i with u_i = sum_j alpha_j S(x_i - y_j), S(d) = Re sum_k W_k e^{-tau_k s |d|}:
//   dL/dalpha_j = sum_i g_i S(y_j - x_i)                 (the transform with roles swapped)
//   dL/dx_i     = g_i sum_j alpha_j S'(x_i - y_j)
//   dL/dy_j     = alpha_j sum_i g_i S'(y_j - x_i)
//   dL/ddelta   = -(1/(2 delta)) (sum_i (x_i - c) dL/dx_i + sum_j (y_j - c) dL/dy_j)
// with S'(d) = Re sum_k V_k sgn(d) e^{-tau_k s |d|}, V_k = -tau_k s W_k, sgn(0) = 0.  The
// sweeps give D = Re sum_k V_k (h+_k - h-_k) at each target, where h+ also holds the
// sources exactly at the target (multiplier 1); with A the sum of those coincident
// strengths, sum_j alpha_j S'(x_i - y_j) = D_i - A_i Re sum_k V_k.  The delta identity is
// the scale invariance u(c x, c y, c^2 delta) = u(x, y, delta); c is any constant (the
// first target coordinate), and translation invariance (sum dL/dx + sum dL/dy = 0)
// makes the result independent of it.
#include <cuda_runtime.h>

#include <algorithm>

#include "kernels.h"

namespace fgt1d {

__global__ void k_grad_assemble(const double* __restrict__ w, const double* __restrict__ D,
                                const double* __restrict__ A, double sumV, int64_t n, double* __restrict__ out) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        out[i] = w[i] * (D[i] - A[i] * sumV);
}

// partials[b] = sum over block b's chunk of (p - c) q for the two (p, q) pairs
__global__ void __launch_bounds__(256) k_dot_partial(const double* __restrict__ x, const double* __restrict__ gx,
                                                     int64_t M, const double* __restrict__ y,
                                                     const double* __restrict__ gy, int64_t N,
                                                     double* __restrict__ partials) {
    __shared__ double red[256];
    const double c = x[0];
    double acc = 0.0;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < M; i += stride) acc += (x[i] - c) * gx[i];
    for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < N; j += stride) acc += (y[j] - c) * gy[j];
    red[threadIdx.x] = acc;
    __syncthreads();
    for (int o = 128; o > 0; o >>= 1) {
        if (threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) partials[blockIdx.x] = red[0];
}

__global__ void __launch_bounds__(256) k_dot_final(const double* __restrict__ partials, int nb, double scale,
                                                   double* __restrict__ out) {
    __shared__ double red[256];
    double acc = 0.0;
    for (int i = threadIdx.x; i < nb; i += blockDim.x) acc += partials[i];
    red[threadIdx.x] = acc;
    __syncthreads();
    for (int o = 128; o > 0; o >>= 1) {
        if (threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) *out = scale * red[0];
}

cudaError_t launch_grad_assemble(const double* w, const double* D, const double* A, double sumV, int64_t n,
                                 double* out, cudaStream_t st) {
    if (n <= 0) return cudaSuccess;
    const int blocks = (int)std::min<int64_t>((n + 255) / 256, 152 * 16);
    k_grad_assemble<<<blocks, 256, 0, st>>>(w, D, A, sumV, n, out);
    return cudaGetLastError();
}

__global__ void k_axpy(const double* __restrict__ a, double c, int64_t n, double* __restrict__ y) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        y[i] += c * a[i];
}

cudaError_t launch_axpy(const double* a, double c, int64_t n, double* y, cudaStream_t st) {
    if (n <= 0) return cudaSuccess;
    const int blocks = (int)std::min<int64_t>((n + 255) / 256, 152 * 16);
    k_axpy<<<blocks, 256, 0, st>>>(a, c, n, y);
    return cudaGetLastError();
}

cudaError_t launch_grad_delta(const double* x, const double* gx, int64_t M, const double* y, const double* gy,
                              int64_t N, double delta, double* partials, int nb, double* out, cudaStream_t st) {
    k_dot_partial<<<nb, 256, 0, st>>>(x, gx, M, y, gy, N, partials);
    k_dot_final<<<1, 256, 0, st>>>(partials, nb, -0.5 / delta, out);
    return cudaGetLastError();
}

}  // namespace fgt1d
