// Output conventions applied after a call, on the device, when the caller
// asks for them by flag:
//   SPINGP_LOG_GRAD    the gradient with respect to log theta,
//                      d ll / d log theta_p = theta_p d ll / d theta_p
//                      (a diagonal rescaling of the raw-parameter gradient);
//   SPINGP_PREDICTIVE  predictive variances of an observation at each step,
//                      the latent variance H P^s H^T plus the noise variance
//                      s_n (the last theta entry of the step's series).
#include <cuda_runtime.h>

#include <cstdint>

#include "internal.h"

namespace spg {

// grad and theta have the same layout (count entries: one row of P per series)
__global__ void __launch_bounds__(256) k_grad_to_log(double* __restrict__ grad, const double* __restrict__ theta,
                                                     int64_t count) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i < count) grad[i] *= theta[i];
}

// one series: var[i] += theta[P - 1]
__global__ void __launch_bounds__(256) k_add_noise(double* __restrict__ var, int64_t n,
                                                   const double* __restrict__ s_n) {
    const double s2 = s_n[0];
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        var[i] += s2;
}

// a batch: one block per series, var[offsets[b] .. offsets[b+1]) += theta[b * P + P - 1]
__global__ void __launch_bounds__(256) k_add_noise_batched(double* __restrict__ var,
                                                           const int64_t* __restrict__ offsets, int64_t n_series,
                                                           const double* __restrict__ theta, int P) {
    for (int64_t b = blockIdx.x; b < n_series; b += gridDim.x) {
        const double s2 = theta[b * P + P - 1];
        const int64_t e = offsets[b + 1];
        for (int64_t i = offsets[b] + threadIdx.x; i < e; i += blockDim.x) var[i] += s2;
    }
}

int grad_to_log(double* grad, const double* theta, int64_t count, cudaStream_t st) {
    if (count < 1) return 0;
    k_grad_to_log<<<(unsigned)((count + 255) / 256), 256, 0, st>>>(grad, theta, count);
    return cudaGetLastError() == cudaSuccess ? 0 : 1;
}

int add_noise(double* var, int64_t n, const double* s_n, cudaStream_t st) {
    if (n < 1) return 0;
    const int64_t blocks = (n + 255) / 256;
    k_add_noise<<<(unsigned)(blocks < 4096 ? blocks : 4096), 256, 0, st>>>(var, n, s_n);
    return cudaGetLastError() == cudaSuccess ? 0 : 1;
}

int add_noise_batched(double* var, const int64_t* offsets, int64_t n_series, const double* theta, int P,
                      cudaStream_t st) {
    if (n_series < 1) return 0;
    k_add_noise_batched<<<(unsigned)(n_series < 65535 ? n_series : 65535), 256, 0, st>>>(var, offsets, n_series,
                                                                                         theta, P);
    return cudaGetLastError() == cudaSuccess ? 0 : 1;
}

}  // namespace spg
