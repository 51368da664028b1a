// predict.cu -- prediction at new times (Eqs. mean4-mean6): the test times
// join the chain as steps whose observation is missing (infinite noise), one
// posterior pass covers both, and the test points' mean and variance are
// read back in the caller's order.
//
//   k_pr_tile_sort  the test times as sort keys with their positions,
//                 sorted in tiles of PR_TILE keys in shared memory by the
//                 merge passes below; a non-finite test time sets ENONFINITE
//                 (a NaN sorts as +inf, so the keys stay totally ordered)
//                 (a pass moves each key to its rank in the merged pair of
//                 runs: its index in its own run plus the count of keys in
//                 the sibling run ordered before it, strictly smaller for a
//                 key of the left run, smaller or equal for the right run,
//                 so equal keys keep their order)
//   k_pr_merge    the passes over runs longer than a tile, by merge path:
//                 one diagonal search per thread, then a sequential merge
//   k_pr_join     the observed and the sorted test times merged (merge
//                 path: one diagonal search per thread, then a sequential
//                 merge of PR_MERGE_E steps; an observation before a test
//                 point at equal times), with NaN as the test points'
//                 observation and each test point's merged step recorded
//   k_pr_gather   each test point's posterior moments moved to its place in
//                 the caller's order; the posterior's status joined into the
//                 call's own status word
#include <cuda_runtime.h>

#include <cstdint>

#include "internal.h"

namespace spg {

namespace {

constexpr int PR_CTA = 256;
constexpr int PR_TILE = 1024;   // keys sorted per CTA in shared memory before the global passes
constexpr int PR_MERGE_E = 16;  // merged steps per thread in the join

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

// the first merge passes (runs up to PR_TILE keys) inside one CTA's shared
// memory: the tile's keys and positions ping-pong between two buffers, one
// block barrier per pass; the sorted tile goes to key / idx
__global__ void __launch_bounds__(PR_CTA) k_pr_tile_sort(const double* __restrict__ ts, int64_t m,
                                                         double* __restrict__ key, int64_t* __restrict__ idx,
                                                         int* __restrict__ status) {
    __shared__ double sk[2][PR_TILE];
    __shared__ int si[2][PR_TILE];
    const int64_t t0 = (int64_t)blockIdx.x * PR_TILE;
    const int len = (int)((m - t0) < PR_TILE ? (m - t0) : PR_TILE);
    bool bad = false;
    for (int e = threadIdx.x; e < len; e += PR_CTA) {
        const double v = ts[t0 + e];
        if (!isfinite(v)) bad = true;
        sk[0][e] = (v == v) ? v : __longlong_as_double(0x7ff0000000000000LL);
        si[0][e] = e;
    }
    if (bad) atomicOr(status, ST_ENONFINITE);
    __syncthreads();
    int cur = 0;
    for (int w = 1; w < PR_TILE; w <<= 1) {   // uniform over the block (len only clips the runs)
        for (int e = threadIdx.x; e < len; e += PR_CTA) {
            const int run = e / w;
            const int base = (run & ~1) * w;
            const bool left = (run & 1) == 0;
            const int sib0 = left ? base + w : base;
            const int sib1 = sib0 + w < len ? sib0 + w : len;
            const int nsib = sib1 > sib0 ? sib1 - sib0 : 0;
            const double v = sk[cur][e];
            const int r = (int)(left ? rank_in<true>(&sk[cur][sib0], nsib, v) : rank_in<false>(&sk[cur][sib0], nsib, v));
            const int dst = base + (e - run * w) + r;
            sk[cur ^ 1][dst] = v;
            si[cur ^ 1][dst] = si[cur][e];
        }
        __syncthreads();
        cur ^= 1;
    }
    for (int e = threadIdx.x; e < len; e += PR_CTA) {
        key[t0 + e] = sk[cur][e];
        idx[t0 + e] = t0 + si[cur][e];
    }
}

// one global merge pass (runs of w >= PR_TILE keys, w a power of two):
// merge path again, thread g writing sorted positions [g E, g E + E) of its
// pair of runs (E divides 2 w, so a thread's positions stay in one pair),
// the left run first at equal keys so the sort stays stable
__global__ void __launch_bounds__(PR_CTA) k_pr_merge(const double* __restrict__ kin, const int64_t* __restrict__ iin,
                                                     double* __restrict__ kout, int64_t* __restrict__ iout,
                                                     int64_t m, int64_t w) {
    const int64_t g = blockIdx.x * (int64_t)PR_CTA + threadIdx.x;
    const int64_t d0 = g * PR_MERGE_E;
    if (d0 >= m) return;
    const int64_t base = (d0 / (2 * w)) * (2 * w);
    const int64_t na = (base + w < m ? base + w : m) - base;          // left run [base, base + na)
    const int64_t nb = (base + 2 * w < m ? base + 2 * w : m) - base - na;   // right run after it
    const double* A = kin + base;
    const double* B = A + na;
    const int64_t dl = d0 - base;
    const int64_t dend = (d0 + PR_MERGE_E < base + na + nb ? d0 + PR_MERGE_E : base + na + nb) - base;
    int64_t lo = dl > nb ? dl - nb : 0, hi = dl < na ? dl : na;
    while (lo < hi) {
        const int64_t mid = (lo + hi) >> 1;
        if (A[mid] <= B[dl - mid - 1]) lo = mid + 1; else hi = mid;
    }
    int64_t i = lo, j = dl - lo;
    for (int64_t p = dl; p < dend; ++p) {
        if (i < na && (j >= nb || A[i] <= B[j])) {
            kout[base + p] = A[i];
            iout[base + p] = iin[base + i];
            ++i;
        } else {
            kout[base + p] = B[j];
            iout[base + p] = iin[base + na + j];
            ++j;
        }
    }
}

// merge path: thread g writes merged steps [g E, g E + E); a binary search on
// its first diagonal finds how many observed times precede them, then it
// merges sequentially, an observation first at equal times.  A test point's
// merged step goes to pos (in sorted test order).
__global__ void __launch_bounds__(PR_CTA) k_pr_join(const double* __restrict__ t, const double* __restrict__ y,
                                                    int64_t n, const double* __restrict__ ts_sorted, int64_t m,
                                                    double* __restrict__ T, double* __restrict__ Y,
                                                    int64_t* __restrict__ pos, int* __restrict__ status) {
    const int64_t g = blockIdx.x * (int64_t)PR_CTA + threadIdx.x;
    const int64_t d0 = g * PR_MERGE_E;
    if (d0 >= n + m) return;
    const int64_t d1 = d0 + PR_MERGE_E < n + m ? d0 + PR_MERGE_E : n + m;
    // i = the observed times among the first d0 merged steps
    int64_t lo = d0 > m ? d0 - m : 0, hi = d0 < n ? d0 : n;
    while (lo < hi) {
        const int64_t mid = (lo + hi) >> 1;
        if (t[mid] <= ts_sorted[d0 - mid - 1]) lo = mid + 1; else hi = mid;
    }
    int64_t i = lo, j = d0 - lo;
    bool unsorted = false;
    for (int64_t p = d0; p < d1; ++p) {
        const bool take_obs = i < n && (j >= m || t[i] <= ts_sorted[j]);
        if (take_obs) {
            if (i > 0 && !(t[i] >= t[i - 1])) unsorted = true;   // the ranks need the observed times ascending
            T[p] = t[i];
            Y[p] = y[i];
            ++i;
        } else {
            T[p] = ts_sorted[j];
            Y[p] = __longlong_as_double(0x7ff8000000000000LL);   // quiet NaN: no observation
            pos[j] = p;
            ++j;
        }
    }
    if (unsorted) atomicOr(status, ST_ENOTSORTED);
}

__global__ void __launch_bounds__(PR_CTA) k_pr_gather(const int64_t* __restrict__ pos,
                                                      const int64_t* __restrict__ idx, int64_t m, int64_t nm,
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
    // pos holds a merged step for every test point when the observed times
    // are sorted; otherwise (ENOTSORTED is set) it is kept in range
    int64_t p = pos[j];
    p = p < 0 ? 0 : (p >= nm ? nm - 1 : p);
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
    for (int64_t w = PR_TILE; w < m; w <<= 1) ++p;
    return p;
}

int predict_prepare(const double* t, const double* y, int64_t n, const double* ts, int64_t m, void* wsv,
                    const PredictLayout& lay, cudaStream_t st) {
    char* ws = (char*)wsv;
    int* status = (int*)ws;
    double* k[2] = {(double*)(ws + lay.off_k0), (double*)(ws + lay.off_k1)};
    int64_t* ix[2] = {(int64_t*)(ws + lay.off_i0), (int64_t*)(ws + lay.off_i1)};
    if (cudaMemsetAsync(status, 0, sizeof(int), st) != cudaSuccess) return 1;
    k_pr_tile_sort<<<(unsigned)((m + PR_TILE - 1) / PR_TILE), PR_CTA, 0, st>>>(ts, m, k[0], ix[0], status);
    int cur = 0;
    static_assert((2 * PR_TILE) % PR_MERGE_E == 0, "a merge thread's positions must stay in one pair of runs");
    for (int64_t w = PR_TILE; w < m; w <<= 1) {
        k_pr_merge<<<blocks_for((m + PR_MERGE_E - 1) / PR_MERGE_E), PR_CTA, 0, st>>>(k[cur], ix[cur], k[cur ^ 1],
                                                                                      ix[cur ^ 1], m, w);
        cur ^= 1;
    }
    // the sorted keys and positions end in buffer predict_merge_passes(m) & 1;
    // the other position buffer takes each test point's merged step
    k_pr_join<<<blocks_for((n + m + PR_MERGE_E - 1) / PR_MERGE_E), PR_CTA, 0, st>>>(
        t, y, n, k[cur], m, (double*)(ws + lay.off_T), (double*)(ws + lay.off_Y), ix[cur ^ 1], status);
    return cudaGetLastError() == cudaSuccess ? 0 : 1;
}

int predict_finish(const double* t, int64_t n, int64_t m, void* wsv, const PredictLayout& lay, double* mean_out,
                   double* var_out, cudaStream_t st) {
    (void)t;
    char* ws = (char*)wsv;
    const bool odd = (predict_merge_passes(m) & 1) != 0;
    k_pr_gather<<<blocks_for(m), PR_CTA, 0, st>>>((const int64_t*)(ws + (odd ? lay.off_i0 : lay.off_i1)),
                                                  (const int64_t*)(ws + (odd ? lay.off_i1 : lay.off_i0)), m, n + m,
                                                  (const double*)(ws + lay.off_mean),
                                                  (const double*)(ws + lay.off_var), mean_out, var_out, (int*)ws,
                                                  (const int*)(ws + lay.off_inner));
    return cudaGetLastError() == cudaSuccess ? 0 : 1;
}

}  // namespace spg
