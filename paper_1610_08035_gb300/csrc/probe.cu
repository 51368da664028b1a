// probe.cu -- measured FP64 throughput of the current device (the ALU roofline
// denominator for the FP64-bound chain kernels), and the chain kernels'
// table-driven e^-x applied to a caller's array (for its accuracy test).
#include <cuda_runtime.h>
#include <stdint.h>

#include "chain.cuh"
#include "internal.h"

namespace spg {

static constexpr int PROBE_THREADS = 256;
static constexpr int PROBE_BLOCKS_PER_SM = 4;
static constexpr int PROBE_ITERS = 8192;

// eight independent FMA chains per thread: issue-bound on the FP64 pipe
__global__ void __launch_bounds__(PROBE_THREADS) k_probe_fp64(double* out, int iters, double a, double b) {
    double x0 = threadIdx.x * 1e-3, x1 = x0 + 1.0, x2 = x0 + 2.0, x3 = x0 + 3.0;
    double x4 = x0 + 4.0, x5 = x0 + 5.0, x6 = x0 + 6.0, x7 = x0 + 7.0;
    for (int i = 0; i < iters; ++i) {
        x0 = fma(x0, a, b); x1 = fma(x1, a, b); x2 = fma(x2, a, b); x3 = fma(x3, a, b);
        x4 = fma(x4, a, b); x5 = fma(x5, a, b); x6 = fma(x6, a, b); x7 = fma(x7, a, b);
    }
    out[blockIdx.x * (int64_t)blockDim.x + threadIdx.x] = x0 + x1 + x2 + x3 + x4 + x5 + x6 + x7;
}

// eight independent FP64 tensor-core products per warp (mma.sync m8n8k4, the
// only FP64 matrix instruction on this architecture: tcgen05 has no FP64
// kind); 8 x 8 x 4 multiply-adds each
__global__ void __launch_bounds__(PROBE_THREADS) k_probe_fp64_mma(double* out, int iters, double a, double b) {
    double c[8][2];
#pragma unroll
    for (int k = 0; k < 8; ++k) { c[k][0] = k + threadIdx.x * 1e-3; c[k][1] = -k; }
    const double av = a + threadIdx.x * 1e-9;
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int k = 0; k < 8; ++k)
            asm volatile("mma.sync.aligned.m8n8k4.row.col.f64.f64.f64.f64 {%0, %1}, {%2}, {%3}, {%0, %1};\n"
                         : "+d"(c[k][0]), "+d"(c[k][1])
                         : "d"(av), "d"(b));
    }
    double s = 0.0;
#pragma unroll
    for (int k = 0; k < 8; ++k) s += c[k][0] + c[k][1];
    out[blockIdx.x * (int64_t)blockDim.x + threadIdx.x] = s;
}

static int sm_count() {
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return 0;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return 0;
    return sms;
}

size_t probe_fp64_bytes() { return sizeof(double) * (size_t)sm_count() * PROBE_BLOCKS_PER_SM * PROBE_THREADS; }

int probe_fp64(void* scratch, size_t bytes, double* tflops, cudaStream_t st, int tensor) {
    const int sms = sm_count();
    if (sms <= 0 || !scratch || bytes < probe_fp64_bytes()) return 1;
    const unsigned blocks = (unsigned)(sms * PROBE_BLOCKS_PER_SM);
    double* out = (double*)scratch;
    cudaEvent_t e0, e1;
    if (cudaEventCreate(&e0) != cudaSuccess) return 1;
    if (cudaEventCreate(&e1) != cudaSuccess) { cudaEventDestroy(e0); return 1; }
    const int iters = tensor ? PROBE_ITERS / 8 : PROBE_ITERS;
    if (tensor) {
        k_probe_fp64_mma<<<blocks, PROBE_THREADS, 0, st>>>(out, 8, 1.0000001, 1e-9);
        cudaEventRecord(e0, st);
        k_probe_fp64_mma<<<blocks, PROBE_THREADS, 0, st>>>(out, iters, 1.0000001, 1e-9);
    } else {
        k_probe_fp64<<<blocks, PROBE_THREADS, 0, st>>>(out, 64, 1.0000001, 1e-9);
        cudaEventRecord(e0, st);
        k_probe_fp64<<<blocks, PROBE_THREADS, 0, st>>>(out, iters, 1.0000001, 1e-9);
    }
    cudaEventRecord(e1, st);
    int rc = cudaEventSynchronize(e1) == cudaSuccess ? 0 : 1;
    float ms = 0.0f;
    if (!rc) rc = cudaEventElapsedTime(&ms, e0, e1) == cudaSuccess ? 0 : 1;
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (rc || ms <= 0.0f) return 1;
    // FMA: 8 per thread per iteration; mma: 8 per warp per iteration, 256 multiply-adds each
    const double flops = tensor ? 2.0 * 256.0 * 8.0 * iters * (double)blocks * (PROBE_THREADS / 32)
                                : 2.0 * 8.0 * iters * (double)blocks * PROBE_THREADS;
    *tflops = flops / (ms * 1e-3) / 1e12;
    return 0;
}

// y_i = e^-x_i by the chain kernels' exp_neg (chain.cuh)
__global__ void __launch_bounds__(256) k_probe_exp_neg(const double* __restrict__ x, double* __restrict__ y,
                                                       int64_t n) {
    __shared__ double tbl[EXPTAB];
    exp_neg_table(tbl, threadIdx.x, blockDim.x);
    __syncthreads();
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        y[i] = exp_neg(x[i], tbl);
}

int probe_exp_neg(const double* x, double* y, int64_t n, cudaStream_t st) {
    if (n < 0 || (n > 0 && (!x || !y))) return 1;
    if (n == 0) return 0;
    const int64_t blocks = (n + 255) / 256;
    k_probe_exp_neg<<<(unsigned)(blocks < 4096 ? blocks : 4096), 256, 0, st>>>(x, y, n);
    return cudaGetLastError() == cudaSuccess ? 0 : 1;
}

}  // namespace spg
