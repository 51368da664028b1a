// internal.h -- declarations shared by the library's translation units.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>
#include <stddef.h>

namespace spg {

// device status bits (the status word at the start of every workspace)
enum { ST_EINVAL = 1 << 1, ST_ENOTSORTED = 1 << 2, ST_ENONFINITE = 1 << 3, ST_ENUMERIC = 1 << 4 };

// what a chain run computes
enum { MODE_LOGLIK = 0, MODE_GRAD = 1, MODE_POSTERIOR = 2 };

size_t matern_ws_bytes(int b, int64_t n, int64_t L, int mode);
int matern_prepare();
// ev: NULL, or 5 events recorded around the four stages
int matern_run(int b, int mode, const double* t, const double* y, int64_t n, int64_t L, const double* theta,
               double* ll_out, double* grad_out, double* mean_out, double* var_out, void* ws, cudaStream_t st,
               cudaEvent_t* ev);
int matern_launch_count(int b, int64_t n, int64_t L, int mode);

// batches of independent series: offsets (device, nseries + 1 entries), theta
// per series (nseries x 3), per-series ll_out / grad_out
size_t matern_ws_bytes_batched(int b, int64_t nseries, int64_t n_total, int64_t L, int mode);
int matern_launch_count_batched(int b, int64_t nseries, int64_t n_total, int64_t L, int mode);
int matern_run_batched(int b, int mode, const int64_t* offsets, int64_t nseries, int64_t n_total, const double* t,
                       const double* y, int64_t L, const double* theta, double* ll_out, double* grad_out,
                       double* mean_out, double* var_out, void* ws, cudaStream_t st, cudaEvent_t* ev);

size_t probe_fp64_bytes();
int probe_fp64(void* scratch, size_t bytes, double* tflops, cudaStream_t st);

}  // namespace spg
