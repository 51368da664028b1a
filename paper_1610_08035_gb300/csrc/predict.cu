// predict.cu -- prediction at new times (Eqs. mean4-mean6): the test times
// join the chain as steps whose observation is missing (infinite noise), one
// posterior pass covers both, and the test points' mean and variance are
// read back in the caller's order.
//
//   k_pr_init     the test times as sort keys with their positions; a
//                 non-finite test time sets ENONFINITE (a NaN sorts as +inf,
//                 so the keys stay totally ordered)
//   k_pr_merge    one pass of a bottom-up merge sort: runs of w keys are
//                 merged pairwise, each key moved to its rank in the merged
//                 pair (its index in its own run plus the count of keys in
//                 the sibling run ordered before it: strictly smaller for a
//                 key of the left run, smaller or equal for the right run,
//                 so equal keys keep their order)
//   k_pr_join     the observed and the sorted test times merged by the same
//                 rank rule (an observation before a test point at equal
//                 times), with NaN as the test points' observation
//   k_pr_gather   each test point's posterior moments moved to its place in
//                 the caller's order; the posterior's status joined into the
//                 call's own status word
#include <cuda_runtime.h>

#include <cstdint>

#include "internal.h"

namespace spg {

namespace {

constexpr int PR_CTA = 256;

// count of x[0 .. n) with x[k] < v (strict) or x[k] <= v, x ascending
template <bool STRICT>
__device__ __forceinline__ int64_t rank_in(const double* __restrict__ x, int64_t n, double v) {
    int64_t lo = 0, hi = n;
    while (lo < hi) {
        const int64_t mid = (lo + hi) >> 1;
        const bool before = STRICT ? (x[mid] < v) : (x[mid] <= v);
        if (before) lo = mid + 1; else hi = mid;
    }
    return lo;
}

unsigned blocks_for(int64_t n) {
    const int64_t b = (n + PR_CTA - 1) / PR_CTA;
    return (unsigned)(b < 1 ? 1 : b);
}

}  // namespace

__global__ void __launch_bounds__(PR_CTA) k_pr_init(const double* __restrict__ ts, int64_t m,
                                                    double* __restrict__ key, int64_t* __restrict__ idx,
                                                    int* __restrict__ status) {
    const int64_t j = blockIdx.x * (int64_t)PR_CTA + threadIdx.x;
    if (j >= m) return;
    const double v = ts[j];
    if (!isfinite(v)) atomicOr(status, ST_ENONFINITE);
    // a NaN key would break the order the merge ranks rely on (and with it
    // the permutation the gather writes through): it sorts as +inf instead
    key[j] = (v == v) ? v : __longlong_as_double(0x7ff0000000000000LL);
    idx[j] = j;
}

__global__ void __launch_bounds__(PR_CTA) k_pr_merge(const double* __restrict__ kin, const int64_t* __restrict__ iin,
                                                     double* __restrict__ kout, int64_t* __restrict__ iout,
                                                     int64_t m, int64_t w) {
    const int64_t j = blockIdx.x * (int64_t)PR_CTA + threadIdx.x;
    if (j >= m) return;
    const int64_t run = j / w;
    const int64_t base = (run & ~(int64_t)1) * w;          // first key of the pair
    const bool left = (run & 1) == 0;
    const int64_t sib0 = left ? base + w : base;            // the sibling run [sib0, sib1)
    const int64_t sib1 = sib0 + w < m ? sib0 + w : m;
    const int64_t nsib = sib1 > sib0 ? sib1 - sib0 : 0;
    const double v = kin[j];
    const int64_t r = left ? rank_in<true>(kin + sib0, nsib, v) : rank_in<false>(kin + sib0, nsib, v);
    const int64_t dst = base + (j - run * w) + r;
    kout[dst] = v;
    iout[dst] = iin[j];
}

__global__ void __launch_bounds__(PR_CTA) k_pr_join(const double* __restrict__ t, const double* __restrict__ y,
                                                    int64_t n, const double* __restrict__ ts_sorted, int64_t m,
                                                    double* __restrict__ T, double* __restrict__ Y,
                                                    int* __restrict__ status) {
    const int64_t i = blockIdx.x * (int64_t)PR_CTA + threadIdx.x;
    if (i < n) {
        // the ranks below need the observed times ascending
        if (i > 0 && !(t[i] >= t[i - 1])) atomicOr(status, ST_ENOTSORTED);
        const int64_t p = i + rank_in<true>(ts_sorted, m, t[i]);
        T[p] = t[i];
        Y[p] = y[i];
    } else if (i < n + m) {
        const int64_t j = i - n;
        const int64_t p = j + rank_in<false>(t, n, ts_sorted[j]);
        T[p] = ts_sorted[j];
        Y[p] = __longlong_as_double(0x7ff8000000000000LL);   // quiet NaN: no observation
    }
}

__global__ void __launch_bounds__(PR_CTA) k_pr_gather(const double* __restrict__ t, int64_t n,
                                                      const double* __restrict__ ts_sorted,
                                                      const int64_t* __restrict__ idx, int64_t m,
                                                      const double* __restrict__ mean_all,
                                                      const double* __restrict__ var_all,
                                                      double* __restrict__ mean_out, double* __restrict__ var_out,
                                                      int* __restrict__ status, const int* __restrict__ inner) {
    const int64_t j = blockIdx.x * (int64_t)PR_CTA + threadIdx.x;
    if (j == 0) {
        const int s = *inner;
        if (s) atomicOr(status, s);
    }
    if (j >= m) return;
    const int64_t p = j + rank_in<false>(t, n, ts_sorted[j]);
    const int64_t o = idx[j];
    mean_out[o] = mean_all[p];
    var_out[o] = var_all[p];
}

PredictLayout::PredictLayout(int64_t n, int64_t m) {
    auto al = [](size_t x) { return (x + 255) & ~(size_t)255; };
    const size_t nm = (size_t)(n + m);
    size_t o = 256;   // the call's status word
    off_T = o; o = al(o + sizeof(double) * nm);
    off_Y = o; o = al(o + sizeof(double) * nm);
    off_mean = o; o = al(o + sizeof(double) * nm);
    off_var = o; o = al(o + sizeof(double) * nm);
    off_k0 = o; o = al(o + sizeof(double) * (size_t)m);
    off_k1 = o; o = al(o + sizeof(double) * (size_t)m);
    off_i0 = o; o = al(o + sizeof(int64_t) * (size_t)m);
    off_i1 = o; o = al(o + sizeof(int64_t) * (size_t)m);
    off_inner = o;
}

int predict_merge_passes(int64_t m) {
    int p = 0;
    for (int64_t w = 1; w < m; w <<= 1) ++p;
    return p;
}

int predict_prepare(const double* t, const double* y, int64_t n, const double* ts, int64_t m, void* wsv,
                    const PredictLayout& lay, cudaStream_t st) {
    char* ws = (char*)wsv;
    int* status = (int*)ws;
    double* k[2] = {(double*)(ws + lay.off_k0), (double*)(ws + lay.off_k1)};
    int64_t* ix[2] = {(int64_t*)(ws + lay.off_i0), (int64_t*)(ws + lay.off_i1)};
    if (cudaMemsetAsync(status, 0, sizeof(int), st) != cudaSuccess) return 1;
    k_pr_init<<<blocks_for(m), PR_CTA, 0, st>>>(ts, m, k[0], ix[0], status);
    int cur = 0;
    for (int64_t w = 1; w < m; w <<= 1) {
        k_pr_merge<<<blocks_for(m), PR_CTA, 0, st>>>(k[cur], ix[cur], k[cur ^ 1], ix[cur ^ 1], m, w);
        cur ^= 1;
    }
    // the sorted keys and positions end in buffer predict_merge_passes(m) & 1
    k_pr_join<<<blocks_for(n + m), PR_CTA, 0, st>>>(t, y, n, k[cur], m, (double*)(ws + lay.off_T),
                                                    (double*)(ws + lay.off_Y), status);
    return cudaGetLastError() == cudaSuccess ? 0 : 1;
}

int predict_finish(const double* t, int64_t n, int64_t m, void* wsv, const PredictLayout& lay, double* mean_out,
                   double* var_out, cudaStream_t st) {
    char* ws = (char*)wsv;
    const bool odd = (predict_merge_passes(m) & 1) != 0;
    k_pr_gather<<<blocks_for(m), PR_CTA, 0, st>>>(t, n, (const double*)(ws + (odd ? lay.off_k1 : lay.off_k0)),
                                                  (const int64_t*)(ws + (odd ? lay.off_i1 : lay.off_i0)), m,
                                                  (const double*)(ws + lay.off_mean),
                                                  (const double*)(ws + lay.off_var), mean_out, var_out, (int*)ws,
                                                  (const int*)(ws + lay.off_inner));
    return cudaGetLastError() == cudaSuccess ? 0 : 1;
}

}  // namespace spg
