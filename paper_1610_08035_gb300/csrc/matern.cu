// matern.cu -- the hot path for Matern chains (state dimension b = 1, 2, 3).
//
// One series of n steps is cut into chunks of L consecutive steps.
//   k_fold      one thread per chunk: discretisation (Sec. 2.1) and sequential
//               elimination of the chunk's interior nodes of K~ (Sec. 3.1,
//               subproblems 1 and 3) into one boundary element (chain.cuh).
//   k_scan_tile odd-even block cyclic reduction of the chunk elements: each
//               CTA pairs neighbouring elements level by level (eliminating
//               every other boundary node), recursing over CTA totals across
//               the grid; the back-substitution sweep returns, for every
//               chunk, the filtered state before it (prefix) and the
//               information of all observations after it (suffix).
//   k_chunk     one thread per chunk: the prediction-error decomposition of
//               the log-likelihood (Eq. ml2 via Eq. det_1) from the chunk's
//               prefix state; for the gradient and the posterior, a reverse
//               sweep seeded by the suffix information that yields the
//               selected inverse of K~ in adjoint form and the per-step
//               hyperparameter adjoints (Sec. 2.4, Eq. dd1).
//   k_finalize  fixed-order reduction of the per-chunk partial sums.
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include "chain.cuh"
#include "coop.cuh"
#include "internal.h"

namespace spg {

static constexpr double LOG_2PI = 1.8378770664093454836;
static constexpr double LN2 = 0.69314718055994530942;

struct ChainArgs {
    const double* t;
    const double* y;
    int64_t n;
    int64_t L;
    int64_t nchunks;          // chunk slots (for batches: an upper bound)
    int64_t nblocks;          // ceil(nchunks / CTA)
    const double* theta;
    int* status;
    // batches of independent series (NULL / 0 for one series)
    const int64_t* offsets;   // [nseries + 1] first step of each series
    const int64_t* cstart;    // [nseries + 1] first chunk of each series
    int64_t nseries;
    int P;                    // theta entries per series
    int missing;              // 1: a NaN observation is missing (a test point)
    // one series: the index of its first step (0), or -1 when the steps
    // continue a series split across ranks; t_prev is then the time of the
    // step before step 0
    int64_t s0;
    double t_prev;
    // posterior of one series: n - 1 entries Cov(f_{i+1}, f_i | y), or NULL
    double* lag1 = nullptr;
};

// The steps of chunk c: [s, e), inside the series that starts at step s0 and
// whose hyperparameters start at th.  In a batch the chunks of each series
// are consecutive; a series' first chunk starts from the stationary prior, and
// that element (A = 0, eta = J = 0) stops information crossing between
// series in both directions, so one reduction over all chunks serves every
// series at once.
struct ChunkRange {
    int64_t s, e, s0, series;
    const double* th;
    bool valid;
};

template <bool BATCH>
__device__ __forceinline__ ChunkRange chunk_range(const ChainArgs& a, int64_t c) {
    ChunkRange r;
    if constexpr (!BATCH) {
        r.valid = c < a.nchunks;
        r.s = c * a.L;
        r.e = min(a.n, r.s + a.L);
        r.s0 = a.s0;
        r.series = 0;
        r.th = a.theta;
    } else {
        r.valid = c < a.cstart[a.nseries];
        int64_t lo = 0, hi = a.nseries;   // largest series with cstart <= c
        if (r.valid) {
            while (hi - lo > 1) {
                const int64_t mid = (lo + hi) >> 1;
                if (a.cstart[mid] <= c) lo = mid; else hi = mid;
            }
        }
        r.series = lo;
        r.s0 = a.offsets[lo];
        r.s = r.s0 + (c - a.cstart[lo]) * a.L;
        r.e = min(a.offsets[lo + 1], r.s + a.L);
        r.th = a.theta + lo * (int64_t)a.P;
    }
    return r;
}

template <int B>
__device__ __forceinline__ bool theta_ok(double ell, double sf, double s2) {
    return ell > 0.0 && sf > 0.0 && s2 > 0.0 && isfinite(ell) && isfinite(sf) && isfinite(s2);
}

// ------------------------------------------------------------------ chunk-tree constants

// The chain kernels group CTA consecutive chunks per thread block.  Their
// elements are the leaves of a binary tree of depth CTA_LV whose nodes
// (255 per block) are the odd-even reduction levels inside the block: node
// (l, j) eliminates the interior boundary nodes of chunks [j 2^l, (j+1) 2^l).
static constexpr int CTA = 128;
static constexpr int CTA_LV = 7;
static constexpr int TREE = 2 * CTA;      // node slots per block (255 used)
static constexpr int NPH = 4;             // stored per step: x, x^2/2, e^-x, e^-2x
static_assert((1 << CTA_LV) == CTA, "CTA must be 2^CTA_LV");

__device__ __forceinline__ int tree_off(int level) { return TREE - (TREE >> level); }

// Renormalise a running product to [1, 2) and move its binary exponent into
// an integer (bit operations only), so that log det needs one log per chunk.
__device__ __forceinline__ void renorm(double& prod, int& expo) {
    const unsigned long long bits = (unsigned long long)__double_as_longlong(prod);
    expo += (int)((bits >> 52) & 0x7ffULL) - 1023;
    prod = __longlong_as_double((long long)((bits & 0x800FFFFFFFFFFFFFULL) | 0x3FF0000000000000ULL));
}

// ------------------------------------------------------------------ cooperative tree levels

// Levels of the in-block tree with at most TREE_COOP_CNT nodes run on lane
// groups (coop.cuh); wider levels keep one node per thread.
static constexpr int TREE_COOP_CNT = 16;

__device__ __forceinline__ int lv_of_cnt(int cnt) { return CTA_LV - 31 + __clz(cnt); }   // cnt = CTA >> l

// Up-sweep levels with cnt <= TREE_COOP_CNT: node j of level l combines
// nodes 2j, 2j+1 of level l-1 (in sm, compacted to the front); at most two
// rounds of NG groups, results held until every group has read its inputs.
template <int B>
__device__ __forceinline__ void tree_up_coop(double* sm, double* __restrict__ nodes, int64_t nld, int64_t blk,
                                             double* __restrict__ btot, int64_t nblocks) {
    constexpr int NE = Dims<B>::NE, W = Coop<B>::W, NG = CTA / W, NGW = Coop<B>::NG_WARP;
    static_assert(2 * NG >= TREE_COOP_CNT, "at most two rounds per level");
    const int tid = threadIdx.x, g = tid / W, wg0 = (tid >> 5) * NGW;
    const CPos<B> p;
#pragma unroll 1
    for (int cnt = TREE_COOP_CNT; cnt >= 1; cnt >>= 1) {
        const int l = lv_of_cnt(cnt);
        const bool act0 = wg0 < cnt, act1 = wg0 + NG < cnt;   // warp-uniform
        CElem r0, r1;
        if (act0) {
            const int j = min(g, cnt - 1);
            CElem x, y;
            celem_load<B>(sm + (2 * j) * NE, 1, 0, x, p);
            celem_load<B>(sm + (2 * j + 1) * NE, 1, 0, y, p);
            ccombine<B>(x, y, r0, p);
        }
        if (act1) {
            const int j = min(g + NG, cnt - 1);
            CElem x, y;
            celem_load<B>(sm + (2 * j) * NE, 1, 0, x, p);
            celem_load<B>(sm + (2 * j + 1) * NE, 1, 0, y, p);
            ccombine<B>(x, y, r1, p);
        }
        __syncthreads();
        if (act0 && g < cnt) {
            celem_store<B>(sm + g * NE, 1, 0, r0, p);
            celem_store<B>(nodes, nld, blk * TREE + tree_off(l) + g, r0, p);
            if (cnt == 1) celem_store<B>(btot, nblocks, blk, r0, p);
        }
        if (act1 && g + NG < cnt) {
            celem_store<B>(sm + (g + NG) * NE, 1, 0, r1, p);
            celem_store<B>(nodes, nld, blk * TREE + tree_off(l) + g + NG, r1, p);
        }
        __syncthreads();
    }
}

// Down-sweep levels with at most TREE_COOP_CNT children: from the parents'
// states / information (spre, ssuf at [0, cnt/2)) to the children's
// ([0, cnt)).  Odd child 2j+1: the parent's state pushed through node 2j;
// even child 2j: the parent's information pulled back through node 2j+1
// (BWD only; otherwise the parent's information is not needed).  Groups
// [0, NG/2) take the odd children and [NG/2, NG) the even ones, so the two
// kinds never share a warp.
template <int B, bool BWD>
__device__ __forceinline__ void tree_down_coop(double* spre, double* ssuf, const double* __restrict__ nodes,
                                               int64_t nld, int64_t blk) {
    constexpr int NM = Dims<B>::NM, W = Coop<B>::W, NG = CTA / W, NGW = Coop<B>::NG_WARP, H = NG / 2;
    static_assert(H % NGW == 0, "a warp's groups lie in one half");
    static_assert(2 * H >= TREE_COOP_CNT / 2, "at most two rounds per level");
    const int tid = threadIdx.x, g = tid / W, wg0 = (tid >> 5) * NGW;
    const bool odd = g < H;
    const int gi = odd ? g : g - H, wgi0 = odd ? wg0 : wg0 - H;
    const CPos<B> p;
#pragma unroll 1
    for (int cnt = 2; cnt <= TREE_COOP_CNT; cnt <<= 1) {
        const int half = cnt / 2;
        const int lc = lv_of_cnt(cnt);   // the children's level
        CVS a0, b0, a1, b1;              // (pre, suf) of the child, rounds 0 and 1
        const bool act0 = wgi0 < half, act1 = wgi0 + H < half;
        const bool need = odd || BWD;
#pragma unroll
        for (int round = 0; round < 2; ++round) {
            const bool act = round ? act1 : act0;
            if (!act) continue;
            const int j = min(gi + round * H, half - 1);
            CVS pre, suf, o;
            cvs_load<B>(spre + j * NM, 1, 0, pre, p);
            if (BWD) cvs_load<B>(ssuf + j * NM, 1, 0, suf, p);
            else { suf.v = 0.0; suf.S = 0.0; }
            if (odd) {
                CElem e;
                celem_load<B>(nodes, nld, blk * TREE + tree_off(lc) + 2 * j, e, p);
                cstate_through<B>(pre, e, o, p);
                (round ? a1 : a0) = o;
                (round ? b1 : b0) = suf;
            } else if (need) {
                CElem e;
                celem_load<B>(nodes, nld, blk * TREE + tree_off(lc) + 2 * j + 1, e, p);
                cinfo_through<B>(e, suf, o, p);
                (round ? a1 : a0) = pre;
                (round ? b1 : b0) = o;
            } else {
                (round ? a1 : a0) = pre;
            }
        }
        __syncthreads();
#pragma unroll
        for (int round = 0; round < 2; ++round) {
            const bool act = round ? act1 : act0;
            const int jj = gi + round * H;
            if (!act || jj >= half) continue;
            const int k = odd ? 2 * jj + 1 : 2 * jj;
            cvs_store<B>(spre + k * NM, 1, 0, round ? a1 : a0, p);
            if (BWD) cvs_store<B>(ssuf + k * NM, 1, 0, round ? b1 : b0, p);
        }
        __syncthreads();
    }
}

// ------------------------------------------------------------------ k_fold

// One thread per chunk: discretise every step (storing x = lam dt, x^2/2,
// e^-x and e^-2x for the later pass) and eliminate the chunk's interior nodes into its
// element; then the block's odd-even up-sweep over its CTA elements, writing
// every tree node and the block total.  Jordan coordinates (chain.cuh); the
// conditional covariance is carried as C - Pinf, so the prediction is a
// single sandwich e^-2x T (C - Pinf) T^T.
// A launch may cover steps [j0, j1) of every chunk only (a piece of the
// elimination, for inputs that arrive in pieces): the first piece starts the
// element, the others resume it from `state` (the element as carried, then
// the scale sa: Dims::NE + 1 fields of nc entries), and only the last piece
// finishes the element and runs the block's up-sweep.  One launch with
// j0 = 0, j1 >= L does the whole chunk; the pieces give the same bits.
template <int B, bool BATCH>
__global__ void __launch_bounds__(CTA, 3) k_fold(ChainArgs a, double* __restrict__ nodes, double* __restrict__ btot,
                                              double* __restrict__ phis, int64_t j0, int64_t j1,
                                              double* __restrict__ state, int first, int last) {
    constexpr int NE = Dims<B>::NE;
    __shared__ double sm[CTA * NE];
    __shared__ double etab[EXPTAB];
    const int tid = threadIdx.x;
    const int64_t blk = blockIdx.x;
    exp_neg_table(etab, tid, CTA);
    __syncthreads();
    const int64_t c = blk * CTA + tid;
    const int64_t nc = a.nchunks;
    const ChunkRange cr = chunk_range<BATCH>(a, c);
    Elem<B> el;
    elem_identity<B>(el);
    int bad = 0;
    if (cr.valid) {
        const double ell = cr.th[0], sf = cr.th[1], s2 = cr.th[2];
        if (first && !theta_ok<B>(ell, sf, s2)) bad |= ST_EINVAL;
        const double lam = sqrt(2.0 * B - 1.0) / ell;
        double sp0[B];   // first column of Pinf
#pragma unroll
        for (int r = 0; r < B; ++r) sp0[r] = sf * pj<B>(r, 0);
        const int64_t s = cr.s, e = cr.e;
        const int64_t i0 = min(e, s + j0), i1 = min(e, s + j1);
        // el.C holds C - Pinf until the end of the chunk; el.A holds A / sa:
        // the factors e^-x of the steps are collected in sa
        double sa = 1.0;
        if (!first) {
            elem_load<B>(state, nc, c, el);
            sa = state[NE * nc + c];
        } else if (s == cr.s0) {
            // the first state has the stationary prior: no dependence on an earlier node
#pragma unroll
            for (int i = 0; i < B; ++i)
#pragma unroll
                for (int j = 0; j < B; ++j) { el.A[i][j] = 0.0; el.C[i][j] = 0.0; }
        } else {
#pragma unroll
            for (int i = 0; i < B; ++i)
#pragma unroll
                for (int j = 0; j < B; ++j) el.C[i][j] = -sf * pj<B>(i, j);
        }
        double tp = (i0 > cr.s0 && i0 < i1) ? (i0 > 0 ? a.t[i0 - 1] : a.t_prev) : 0.0;
        // t and y are loaded one step ahead
        double tnx = (i0 < i1) ? a.t[i0] : 0.0, ynx = (i0 < i1) ? a.y[i0] : 0.0;
        for (int64_t i = i0; i < i1; ++i) {
            const double ti = tnx, yi = ynx;
            if (i + 1 < i1) { tnx = a.t[i + 1]; ynx = a.y[i + 1]; }
            const bool obs = !(a.missing && is_nan_b(yi));
            if (!is_finite_b(ti) || (obs && !is_finite_b(yi))) bad |= ST_ENONFINITE;
            if (i > cr.s0) {
                const double dt = ti - tp;
                if (is_negative_b(dt)) bad |= ST_ENOTSORTED;
                const double x = lam * dt, h = 0.5 * x * x, ex = exp_neg(x, etab), e2 = ex * ex;
                {
                    double* ph = phis + ((i - s) * NPH) * nc + c;
                    ph[0] = x;
                    ph[nc] = h;
                    ph[2 * nc] = ex;
                    ph[3 * nc] = e2;
                }
                // A <- e T A,  bv <- e T bv,  C - Pinf <- e^2 T (C - Pinf) T^T
                const JCoef<B> tc(x, h);
                jprop_unscaled<B, B>(tc, el.A);
                sa *= ex;
                jprop_vec<B>(tc, ex, el.bv);
                jsand<B, false>(tc, e2, el.C);
            }
            // condition on y_i: innovation of y_i given the node before the chunk
            // (a missing observation has infinite noise: no update, Eqs. mean4-mean6)
            if (obs) {
            double a0[B], c0[B];   // a0: the first row of A / sa
#pragma unroll
            for (int r = 0; r < B; ++r) {
                a0[r] = el.A[0][r];
                c0[r] = el.C[r][0] + sp0[r];
            }
            const double S = c0[0] + s2;
            const double rS = 1.0 / S;
            const double res = yi - el.bv[0];
            const double rr = res * rS;
            const double rra = rr * sa, rSa = rS * sa * sa;
#pragma unroll
            for (int r = 0; r < B; ++r) {
                el.eta[r] = fma(a0[r], rra, el.eta[r]);
                const double ar = a0[r] * rSa;
#pragma unroll
                for (int q = r; q < B; ++q) { el.J[r][q] = fma(ar, a0[q], el.J[r][q]); el.J[q][r] = el.J[r][q]; }
            }
#pragma unroll
            for (int r = 0; r < B; ++r) {
                el.bv[r] = fma(c0[r], rr, el.bv[r]);
                const double g = c0[r] * rS;
#pragma unroll
                for (int q = 0; q < B; ++q) el.A[r][q] = fma(-g, a0[q], el.A[r][q]);
#pragma unroll
                for (int q = r; q < B; ++q) { el.C[r][q] = fma(-g, c0[q], el.C[r][q]); el.C[q][r] = el.C[r][q]; }
            }
            }
            tp = ti;
        }
        if (!last) {
            elem_store<B>(state, nc, c, el);
            state[NE * nc + c] = sa;
        } else {
#pragma unroll
            for (int r = 0; r < B; ++r)
#pragma unroll
                for (int q = 0; q < B; ++q) { el.C[r][q] += sf * pj<B>(r, q); el.A[r][q] *= sa; }
        }
    }
    if (bad) atomicOr(a.status, bad);
    if (!last) return;   // uniform over the launch: the up-sweep runs after the last piece
    // odd-even up-sweep inside the block (chunks past the end are identities):
    // the wide lower levels one combine per thread, the upper levels (at most
    // TREE_COOP_CNT combines) one combine per lane group
    const int64_t nld = a.nblocks * TREE;
    elem_store<B>(nodes, nld, blk * TREE + tid, el);
    elem_store<B>(sm, 1, (int64_t)tid * NE, el);
    __syncthreads();
#pragma unroll 1
    for (int l = 1; (CTA >> l) > TREE_COOP_CNT; ++l) {
        const int cnt = CTA >> l;
        Elem<B> r;
        if (tid < cnt) {
            Elem<B> x, y;
            elem_load<B>(sm, 1, (int64_t)(2 * tid) * NE, x);
            elem_load<B>(sm, 1, (int64_t)(2 * tid + 1) * NE, y);
            combine<B>(x, y, r);
        }
        __syncthreads();
        if (tid < cnt) {
            elem_store<B>(sm, 1, (int64_t)tid * NE, r);
            elem_store<B>(nodes, nld, blk * TREE + tree_off(l) + tid, r);
        }
        __syncthreads();
    }
    tree_up_coop<B>(sm, nodes, nld, blk, btot, a.nblocks);
}

// ------------------------------------------------------------------ k_scan_tile (odd-even reduction)

// A tile is SCAN_TS consecutive elements, reduced by one CTA of SCAN_CTA
// threads whose lanes form groups of Coop<B>::W (coop.cuh): every combine,
// state_through and info_through of the tile's tree is done by one group,
// so a level costs one cooperative combine (~80 FP64 instructions per lane)
// instead of a thread's full combine.
static constexpr int SCAN_TS = 32;
static constexpr int SCAN_LV = 5;
static constexpr int SCAN_CTA = 256;
static_assert((1 << SCAN_LV) == SCAN_TS, "SCAN_TS must be 2^SCAN_LV");

template <int B>
struct ScanSmem {
    static constexpr int NE = Dims<B>::NE, NM = Dims<B>::NM;
    static constexpr size_t bytes = sizeof(double) * (size_t)(2 * SCAN_TS) * (NE + 2 * NM);
};


template <int B>
__device__ __forceinline__ double elem_identity_field(int f) {
    return (f < B * B && (f % (B + 1)) == 0) ? 1.0 : 0.0;   // A = I, everything else 0
}

// Up-sweep: the tile's elements are paired level by level (odd-even), every
// node kept in shared memory; without DOWN the tile total is written.  With
// DOWN, the back-substitution sweep writes, for every element k, the state
// before it (pre_out, NM fields) and the information after it (suf_out),
// given the tile's own prefix and suffix (pre_in / suf_in; NULL at the top
// level, where the state before the first element is irrelevant: the first
// element of a series has A = 0).
template <int B, bool DOWN>
__global__ void __launch_bounds__(SCAN_CTA, 1) k_scan_tile(const double* __restrict__ E, int64_t ne,
                                                        double* __restrict__ totals, int64_t ntiles,
                                                        const double* __restrict__ pre_in,
                                                        const double* __restrict__ suf_in,
                                                        double* __restrict__ pre_out, double* __restrict__ suf_out) {
    constexpr int NE = Dims<B>::NE, NM = Dims<B>::NM, TS = SCAN_TS;
    constexpr int W = Coop<B>::W, NG = SCAN_CTA / W, NGW = Coop<B>::NG_WARP;
    static_assert(NG >= TS / 2, "one round per up-sweep level");
    static_assert((NG / 2) % NGW == 0, "a warp's groups lie in one half");
    extern __shared__ double sm[];
    double* nodes = sm;
    double* preN = nodes + 2 * TS * NE;
    double* sufN = preN + 2 * TS * NM;
    const int tid = threadIdx.x;
    const int g = tid / W;
    const int wg0 = (tid >> 5) * NGW;   // first group of this warp
    const CPos<B> p;
    const int64_t tile = blockIdx.x;
    const int64_t k0 = tile * (int64_t)TS;
    // a launch of one tile (the top of the reduction) needs only
    // ceil(log2 ne) levels: the tile shrinks to ts = 2^lv elements
    const int lv = (gridDim.x == 1) ? ((ne <= 1) ? 0 : 32 - __clz((int)ne - 1)) : SCAN_LV;
    const int ts = 1 << lv;
    auto noff = [ts](int level) { return 2 * ts - ((2 * ts) >> level); };

    for (int idx = tid; idx < ts * NE; idx += SCAN_CTA) {
        const int f = idx / ts, j = idx % ts;
        nodes[j * NE + f] = (k0 + j < ne) ? E[(int64_t)f * ne + k0 + j] : elem_identity_field<B>(f);
    }
    __syncthreads();
#pragma unroll 1
    for (int l = 1; l <= lv; ++l) {
        const int cnt = ts >> l;
        if (wg0 < cnt) {   // warp-uniform
            const int j = min(g, cnt - 1);
            CElem x, y, r;
            celem_load<B>(nodes + (noff(l - 1) + 2 * j) * NE, 1, 0, x, p);
            celem_load<B>(nodes + (noff(l - 1) + 2 * j + 1) * NE, 1, 0, y, p);
            ccombine<B>(x, y, r, p);
            if (g < cnt) celem_store<B>(nodes + (noff(l) + g) * NE, 1, 0, r, p);
        }
        __syncthreads();
    }
    if constexpr (!DOWN) {
        if (g == 0) {
            CElem r;
            celem_load<B>(nodes + noff(lv) * NE, 1, 0, r, p);
            celem_store<B>(totals, ntiles, tile, r, p);
        }
        return;
    } else {
        if (g == 0) {
            CVS x;
            x.v = 0.0; x.S = 0.0;
            if (pre_in) cvs_load<B>(pre_in, ntiles, tile, x, p);
            cvs_store<B>(preN + noff(lv) * NM, 1, 0, x, p);
            x.v = 0.0; x.S = 0.0;
            if (suf_in) cvs_load<B>(suf_in, ntiles, tile, x, p);
            cvs_store<B>(sufN + noff(lv) * NM, 1, 0, x, p);
        }
        __syncthreads();
        // level l -> its children at level l-1: odd child 2j+1 gets the
        // parent's state pushed through child 2j; even child 2j gets the
        // parent's information pulled back through child 2j+1.  Groups
        // [0, NG/2) take the odd children, [NG/2, NG) the even ones.
        const bool odd = g < NG / 2;
        const int gi = odd ? g : g - NG / 2;
        const int wgi0 = odd ? wg0 : wg0 - NG / 2;
#pragma unroll 1
        for (int l = lv; l >= 1; --l) {
            const int half = (ts >> (l - 1)) / 2;
#pragma unroll 1
            for (int base = 0; base < half; base += NG / 2) {
                if (base + wgi0 < half) {   // warp-uniform
                    const int j = min(base + gi, half - 1);
                    const bool mine = base + gi < half;
                    CVS pre, suf, o;
                    CElem e;
                    cvs_load<B>(preN + (noff(l) + j) * NM, 1, 0, pre, p);
                    cvs_load<B>(sufN + (noff(l) + j) * NM, 1, 0, suf, p);
                    if (odd) {
                        celem_load<B>(nodes + (noff(l - 1) + 2 * j) * NE, 1, 0, e, p);
                        cstate_through<B>(pre, e, o, p);
                        if (mine) {
                            cvs_store<B>(preN + (noff(l - 1) + 2 * j + 1) * NM, 1, 0, o, p);
                            cvs_store<B>(sufN + (noff(l - 1) + 2 * j + 1) * NM, 1, 0, suf, p);
                        }
                    } else {
                        celem_load<B>(nodes + (noff(l - 1) + 2 * j + 1) * NE, 1, 0, e, p);
                        cinfo_through<B>(e, suf, o, p);
                        if (mine) {
                            cvs_store<B>(preN + (noff(l - 1) + 2 * j) * NM, 1, 0, pre, p);
                            cvs_store<B>(sufN + (noff(l - 1) + 2 * j) * NM, 1, 0, o, p);
                        }
                    }
                }
            }
            __syncthreads();
        }
        for (int idx = tid; idx < ts * NM; idx += SCAN_CTA) {
            const int f = idx / ts, j = idx % ts;
            if (k0 + j < ne) {
                pre_out[(int64_t)f * ne + k0 + j] = preN[j * NM + f];
                suf_out[(int64_t)f * ne + k0 + j] = sufN[j * NM + f];
            }
        }
    }
}

// ------------------------------------------------------------------ k_chunk (forward, then reverse sweep)

// per-block partial sums: ll, sum_i x_i d ll/dx_i, 2 d ll/d(s_n), y^T C^-1 y,
// observed steps
template <int B> struct Acc { static constexpr int N = 5; };
// per-step stored values: predicted mean (B), predicted covariance minus Pinf
// (packed), innovation, 1/S
template <int B> struct Stored { static constexpr int N = B + Dims<B>::NS + 2; };
// per-step transition: x, x^2/2, e^-x, e^-2x

// the transition of step j of chunk c (slot j of the [step][field][chunk] layout)
__device__ __forceinline__ void load_trans(const double* __restrict__ phis, int64_t j, int64_t nc, int64_t c,
                                           double (&p)[NPH]) {
    const double* ph = phis + (j * NPH) * nc + c;
#pragma unroll
    for (int f = 0; f < NPH; ++f) p[f] = ph[f * nc];
}

// One thread per chunk, CTA chunks per block.
//  1. Back-substitution of the block's odd-even tree: from the block's own
//     prefix state and suffix information (grid level) down to every chunk.
//  2. Forward: the Kalman recursion over the chunk from its prefix state,
//     prediction-error log-likelihood; for BWD modes the predicted moments
//     are stored per step.
//  3. BWD: the reverse sweep.  At the chunk's last step the suffix
//     information (eta, J) becomes the adjoint of the filtered state,
//     lh = -(I + J P)^-1 (eta - J m), Lh = (I + J P)^-1 J; then per step
//     (inversion-free; the modified Bryson-Frazier form of the smoother):
//       al = v/S + k^T lh          (C^-1 y)_i
//       cc = 1/S + k^T Lh k        (C^-1)_ii
//       lt = lh - al e1,  Lt = (I - k e1^T)^T Lh (I - k e1^T) + e1 e1^T / S
//       G  = (lt lt^T - Lt)/2      d ll / d(predicted covariance)
//       lh <- A^T lt, Lh <- A^T Lt A   (to the previous step)
//     posterior mean_i = y_i - s_n al, latent variance = s_n k_0 - s_n^2 k^T Lh k
//     (the diagonal of the selected inverse); gradient terms
//       d ll/dx_i = -lt^T F mb + 2 <G, F (Pb - Pinf)>,  x_i = lam dt_i, F = N - I
//       (A = e^-x T(x) in Jordan coordinates, dA/dx = F A; Pinf and H do
//       not depend on lam there), d ll/ds_n = sum (al^2 - cc)/2.
//     d ll/ds_f follows from the others: ll(c s_f, c s_n) has derivative
//     (y^T C^-1 y - n_obs)/2 in c at c = 1 (C scales by c), so
//     s_f d ll/ds_f = (y^T C^-1 y - n_obs)/2 - s_n d ll/ds_n.
//  4. Fixed-order block reduction of the partial sums.
template <int B, int MODE, bool BATCH>
__global__ void __launch_bounds__(CTA) k_chunk(ChainArgs a, const double* __restrict__ nodes,
                                               const double* __restrict__ bpre, const double* __restrict__ bsuf,
                                               const double* __restrict__ phis, double* __restrict__ store,
                                               double* __restrict__ part, double* __restrict__ mean_out,
                                               double* __restrict__ var_out) {
    constexpr int NE = Dims<B>::NE;
    constexpr int NM = Dims<B>::NM;
    constexpr int NF = Stored<B>::N;
    constexpr int NA = Acc<B>::N;
    constexpr bool BWD = (MODE != MODE_LOGLIK);
    constexpr bool GRAD = (MODE == MODE_GRAD || MODE == MODE_GRAD_POSTERIOR);
    constexpr bool POST = (MODE == MODE_POSTERIOR || MODE == MODE_GRAD_POSTERIOR);
    (void)NE;
    __shared__ double spre[CTA * NM];
    __shared__ double ssuf[BWD ? CTA * NM : 1];
    __shared__ double red[CTA * NA];
    const int tid = threadIdx.x;
    const int64_t blk = blockIdx.x;
    const int64_t c = blk * CTA + tid;
    const int64_t nc = a.nchunks;
    const int64_t nld = a.nblocks * TREE;
    const ChunkRange cr = chunk_range<BATCH>(a, c);
    const double sf = cr.th[1], s2 = cr.th[2];

    // ---- 1. back-substitution inside the block: the upper levels on lane
    // groups, then one child per thread with the odd children (state pushed
    // through the left sibling) on threads [0, CTA/2) and the even children
    // (information pulled back through the right sibling) on [CTA/2, CTA)
    if (tid == 0) {
        double v[B], S[B][B];
        vs_load<B>(bpre, a.nblocks, blk, v, S);
        vs_store<B>(spre, 1, 0, v, S);
        if constexpr (BWD) {
            vs_load<B>(bsuf, a.nblocks, blk, v, S);
            vs_store<B>(ssuf, 1, 0, v, S);
        }
    }
    __syncthreads();
    tree_down_coop<B, BWD>(spre, ssuf, nodes, nld, blk);
#pragma unroll 1
    for (int cnt = 2 * TREE_COOP_CNT; cnt <= CTA; cnt <<= 1) {
        const int half = cnt / 2;
        const int lc = lv_of_cnt(cnt);
        const bool odd = tid < CTA / 2;
        const int j = odd ? tid : tid - CTA / 2;
        const bool act = j < half;
        double pm[B], pP[B][B], sv[B], sJ[B][B];
        if (act) {
            vs_load<B>(spre, 1, (int64_t)j * NM, pm, pP);
            if constexpr (BWD) vs_load<B>(ssuf, 1, (int64_t)j * NM, sv, sJ);
            Elem<B> sib;
            if (odd) {
                elem_load<B>(nodes, nld, blk * TREE + tree_off(lc) + 2 * j, sib);
                double om[B], oP[B][B];
                state_through<B>(pm, pP, sib, om, oP);
#pragma unroll
                for (int i = 0; i < B; ++i) { pm[i] = om[i];
#pragma unroll
                    for (int q = 0; q < B; ++q) pP[i][q] = oP[i][q]; }
            } else if constexpr (BWD) {
                elem_load<B>(nodes, nld, blk * TREE + tree_off(lc) + 2 * j + 1, sib);
                double ov[B], oJ[B][B];
                info_through<B>(sib, sv, sJ, ov, oJ);
#pragma unroll
                for (int i = 0; i < B; ++i) { sv[i] = ov[i];
#pragma unroll
                    for (int q = 0; q < B; ++q) sJ[i][q] = oJ[i][q]; }
            }
        }
        __syncthreads();
        if (act) {
            const int k = odd ? 2 * j + 1 : 2 * j;
            vs_store<B>(spre, 1, (int64_t)k * NM, pm, pP);
            if constexpr (BWD) vs_store<B>(ssuf, 1, (int64_t)k * NM, sv, sJ);
        }
        __syncthreads();
    }

    double acc[NA];
#pragma unroll
    for (int f = 0; f < NA; ++f) acc[f] = 0.0;
    int bad = 0;
    if (cr.valid) {
        const int64_t s = cr.s, e = cr.e;
        double sp0[B];   // first column of Pinf
#pragma unroll
        for (int r = 0; r < B; ++r) sp0[r] = sf * pj<B>(r, 0);
        // ---- 2. forward: filtered mean m and D = P - Pinf
        double m[B], D[B][B];
        double pe_pre[B];   // P e1 of the filtered state before the chunk (the lag-one output)
        {
            double P[B][B];
            vs_load<B>(spre, 1, (int64_t)tid * NM, m, P);
#pragma unroll
            for (int r = 0; r < B; ++r) {
                pe_pre[r] = P[r][0];
#pragma unroll
                for (int q = 0; q < B; ++q) D[r][q] = P[r][q] - sf * pj<B>(r, q);
            }
        }
        (void)pe_pre;
        double quad = 0.0, prod = 1.0;
        int expo = 0;
        int64_t nobs = 0;
        // each step's y and transition are loaded one step ahead, so their
        // latency overlaps the previous step's arithmetic (slot 0 of a series'
        // first chunk holds no transition; it is loaded and not used)
        double ynx = a.y[s], tnx[NPH];
        load_trans(phis, 0, nc, c, tnx);
        for (int64_t i = s; i < e; ++i) {
            const int64_t j = i - s;
            const double yi = ynx;
            double tr[NPH];
#pragma unroll
            for (int f = 0; f < NPH; ++f) tr[f] = tnx[f];
            if (i + 1 < e) {
                ynx = a.y[i + 1];
                load_trans(phis, j + 1, nc, c, tnx);
            }
            const bool obs = !(a.missing && is_nan_b(yi));
            double mb[B], Db[B][B];
            if (i == cr.s0) {
#pragma unroll
                for (int r = 0; r < B; ++r) { mb[r] = 0.0;
#pragma unroll
                    for (int q = 0; q < B; ++q) Db[r][q] = 0.0; }
            } else {
                const JCoef<B> tc(tr[0], tr[1]);
#pragma unroll
                for (int r = 0; r < B; ++r) {
                    mb[r] = m[r];
#pragma unroll
                    for (int q = 0; q < B; ++q) Db[r][q] = D[r][q];
                }
                jprop_vec<B>(tc, tr[2], mb);
                jsand<B, false>(tc, tr[3], Db);
            }
            double p0[B];   // first column of the predicted covariance
#pragma unroll
            for (int r = 0; r < B; ++r) p0[r] = Db[r][0] + sp0[r];
            // a missing observation stores v = 1/S = 0: the reverse sweep then
            // passes its adjoints through unchanged
            double rS = 0.0, v = 0.0;
            if (obs) {
                const double S = p0[0] + s2;
                if (!is_positive_finite_b(S)) bad |= ST_ENUMERIC;
                rS = 1.0 / S;
                v = yi - mb[0];
                quad = fma(v * v, rS, quad);
                prod *= S;
                renorm(prod, expo);
                ++nobs;
            }
            if constexpr (BWD) {
                double* st = store + (j * NF) * nc + c;
                int f = 0;
#pragma unroll
                for (int r = 0; r < B; ++r) st[(f++) * nc] = mb[r];
#pragma unroll
                for (int r = 0; r < B; ++r)
#pragma unroll
                    for (int q = r; q < B; ++q) st[(f++) * nc] = Db[r][q];
                st[(f++) * nc] = v;
                st[(f++) * nc] = rS;
            }
            const double vr = v * rS;   // both zero for a missing observation: m = mb, D = Db
#pragma unroll
            for (int r = 0; r < B; ++r) {
                m[r] = fma(p0[r], vr, mb[r]);
                const double g = p0[r] * rS;
#pragma unroll
                for (int q = r; q < B; ++q) { D[r][q] = fma(-g, p0[q], Db[r][q]); D[q][r] = D[r][q]; }
            }
        }
        acc[0] = -0.5 * (quad + log(prod) + (double)expo * LN2 + (double)nobs * LOG_2PI);
        acc[3] = quad;
        acc[4] = (double)nobs;

        if constexpr (BWD) {
            // ---- 3. reverse sweep, seeded by the information after the chunk
            double lh[B], Lh[B][B];
            {
                double eta[B], J[B][B], P[B][B], N[B][B], W[B][B], w[B];
                vs_load<B>(ssuf, 1, (int64_t)tid * NM, eta, J);
#pragma unroll
                for (int r = 0; r < B; ++r)
#pragma unroll
                    for (int q = 0; q < B; ++q) P[r][q] = D[r][q] + sf * pj<B>(r, q);
                mat_mul<B>(J, P, N);
#pragma unroll
                for (int i = 0; i < B; ++i) N[i][i] += 1.0;
                inv_pp<B>(N, W);
                mat_vec<B>(J, m, w);
#pragma unroll
                for (int i = 0; i < B; ++i) w[i] = eta[i] - w[i];
                mat_vec<B>(W, w, lh);
#pragma unroll
                for (int i = 0; i < B; ++i) lh[i] = -lh[i];
                mat_mul<B>(W, J, Lh);
                symmetrize<B>(Lh);
            }
            double gx = 0.0, gs = 0.0;
            // the stored step and its transition are loaded one step ahead
            double snx[NF], tnx[NPH];
            {
                const double* st = store + ((e - 1 - s) * NF) * nc + c;
#pragma unroll
                for (int f = 0; f < NF; ++f) snx[f] = st[f * nc];
                load_trans(phis, e - 1 - s, nc, c, tnx);
            }
            for (int64_t i = e - 1; i >= s; --i) {
                const int64_t j = i - s;
                double sv[NF], tr[NPH];
#pragma unroll
                for (int f = 0; f < NF; ++f) sv[f] = snx[f];
#pragma unroll
                for (int f = 0; f < NPH; ++f) tr[f] = tnx[f];
                if (i > s) {
                    const double* st = store + ((j - 1) * NF) * nc + c;
#pragma unroll
                    for (int f = 0; f < NF; ++f) snx[f] = st[f * nc];
                    load_trans(phis, j - 1, nc, c, tnx);
                }
                double mb[B], Db[B][B];
                int f = 0;
#pragma unroll
                for (int r = 0; r < B; ++r) mb[r] = sv[f++];
#pragma unroll
                for (int r = 0; r < B; ++r)
#pragma unroll
                    for (int q = r; q < B; ++q) { Db[r][q] = sv[f++]; Db[q][r] = Db[r][q]; }
                const double v = sv[f++];
                const double rS = sv[f++];
                // a missing step (posterior): k is taken as Pb e1, so kl and kuk
                // below are the prediction's Pb_0^T lh and Pb_0^T Lh Pb_0; its
                // adjoint then passes through unchanged (kl, kuk, u zeroed)
                double yi = 0.0;
                bool pmiss = false;
                if constexpr (POST) {
                    yi = a.y[i];
                    pmiss = a.missing && is_nan_b(yi);
                }
                const double rk = pmiss ? 1.0 : rS;
                double p0[B], k[B];
#pragma unroll
                for (int r = 0; r < B; ++r) { p0[r] = Db[r][0] + sp0[r]; k[r] = p0[r] * rk; }
                double kl = 0.0, u[B], kuk = 0.0;
#pragma unroll
                for (int r = 0; r < B; ++r) kl = fma(k[r], lh[r], kl);
                mat_vec<B>(Lh, k, u);
#pragma unroll
                for (int r = 0; r < B; ++r) kuk = fma(k[r], u[r], kuk);
                if constexpr (POST) {
                    if (pmiss) {
                        // predicted only: mean = (mb - Pb lh)_0, variance = Pb_00 - Pb_0^T Lh Pb_0
                        mean_out[i] = mb[0] - kl;
                        var_out[i] = p0[0] - kuk;
                        kl = 0.0;
                        kuk = 0.0;
#pragma unroll
                        for (int r = 0; r < B; ++r) u[r] = 0.0;
                    }
                }
                const double al = fma(v, rS, kl);     // (C^-1 y)_i
                const double cc = rS + kuk;           // (C^-1)_ii
                if constexpr (GRAD) gs = fma(al, al, gs) - cc;
                if constexpr (POST) {
                    if (!pmiss) {
                        mean_out[i] = fma(-s2, al, yi);
                        var_out[i] = s2 * k[0] - s2 * s2 * kuk;
                    }
                }
                double lt[B], Lt[B][B];
#pragma unroll
                for (int r = 0; r < B; ++r) {
                    lt[r] = lh[r];
#pragma unroll
                    for (int q = 0; q < B; ++q) Lt[r][q] = Lh[r][q];
                }
                lt[0] -= al;
#pragma unroll
                for (int q = 1; q < B; ++q) { Lt[0][q] -= u[q]; Lt[q][0] = Lt[0][q]; }
                Lt[0][0] = Lt[0][0] - 2.0 * u[0] + cc;
                if (i > cr.s0) {
                    const double x = tr[0];
                    if constexpr (POST) {
                        if (a.lag1) {
                            // Cov(f_i, f_{i-1} | y) = e1^T w - Pb_0^T Lt w with
                            // w = A P_{i-1} e1 (Lt: the adjoint with y_i and after, the
                            // information on the predicted state i; P_{i-1}: the filtered
                            // covariance, Pb_{i-1} e1 times s_n / S_{i-1}, or Pb_{i-1} e1 at
                            // a missing step; the chunk's prefix state before its first step)
                            double w[B];
                            if (i > s) {
                                const double rsp = snx[NF - 1];
                                const double fac = (rsp == 0.0) ? 1.0 : s2 * rsp;
#pragma unroll
                                for (int r = 0; r < B; ++r)   // Db_prev[0][r]: row 0 of the stored upper triangle
                                    w[r] = (snx[B + r] + sp0[r]) * fac;
                            } else {
#pragma unroll
                                for (int r = 0; r < B; ++r) w[r] = pe_pre[r];
                            }
                            const JCoef<B> tw(x, tr[1]);
                            jprop_vec<B>(tw, tr[2], w);
                            double ltw = 0.0;
#pragma unroll
                            for (int r = 0; r < B; ++r) {
                                double t = 0.0;
#pragma unroll
                                for (int q = 0; q < B; ++q) t = fma(Lt[r][q], w[q], t);
                                ltw = fma(p0[r], t, ltw);
                            }
                            a.lag1[i - 1] = w[0] - ltw;
                        }
                    }
                    if constexpr (GRAD) {
                        // d ll/dx = <G2, F Db> - lt^T F mb with G2 = lt lt^T - Lt (= 2 G), F = N - I:
                        // <G2, N Db> - <G2, Db> - lt^T N mb + lt^T mb
                        double G2[B][B];
#pragma unroll
                        for (int r = 0; r < B; ++r)
#pragma unroll
                            for (int q = r; q < B; ++q) { G2[r][q] = fma(lt[r], lt[q], -Lt[r][q]); G2[q][r] = G2[r][q]; }
                        double gn = 0.0, go = 0.0, gd = 0.0, mn = 0.0, md = 0.0;
#pragma unroll
                        for (int r = 0; r + 1 < B; ++r)
#pragma unroll
                            for (int q = 0; q < B; ++q) gn = fma(G2[r][q], Db[r + 1][q], gn);
#pragma unroll
                        for (int r = 0; r < B; ++r)
#pragma unroll
                            for (int q = r + 1; q < B; ++q) go = fma(G2[r][q], Db[r][q], go);
#pragma unroll
                        for (int r = 0; r < B; ++r) gd = fma(G2[r][r], Db[r][r], gd);
#pragma unroll
                        for (int r = 0; r + 1 < B; ++r) mn = fma(lt[r], mb[r + 1], mn);
#pragma unroll
                        for (int r = 0; r < B; ++r) md = fma(lt[r], mb[r], md);
                        const double dx = (gn - fma(2.0, go, gd)) - (mn - md);
                        gx = fma(dx, x, gx);
                    }
                    const JCoef<B> tc(x, tr[1]);
#pragma unroll
                    for (int r = 0; r < B; ++r) {
                        lh[r] = lt[r];
#pragma unroll
                        for (int q = 0; q < B; ++q) Lh[r][q] = Lt[r][q];
                    }
                    jprop_tvec<B>(tc, tr[2], lh);
                    jsand<B, true>(tc, tr[3], Lh);
                }
            }
            if constexpr (GRAD) {
                acc[1] = gx;
                acc[2] = gs;
            }
        }
    }
    if (bad) atomicOr(a.status, bad);
    constexpr int NU = GRAD ? NA : 1;
    if constexpr (BATCH) {
        // per-chunk partial sums; the per-series reduction follows
        if (cr.valid)
#pragma unroll
            for (int f = 0; f < NU; ++f) part[f * nc + c] = acc[f];
    } else {
        // ---- 4. fixed-order reduction of the block's partial sums
#pragma unroll
        for (int f = 0; f < NU; ++f) red[f * CTA + tid] = acc[f];
        __syncthreads();
#pragma unroll 1
        for (int w = CTA / 2; w > 0; w >>= 1) {
            if (tid < w)
#pragma unroll
                for (int f = 0; f < NU; ++f) red[f * CTA + tid] += red[f * CTA + tid + w];
            __syncthreads();
        }
        if (tid == 0)
#pragma unroll
            for (int f = 0; f < NU; ++f) part[f * a.nblocks + blk] = red[f * CTA];
    }
}

// ------------------------------------------------------------------ k_finalize (fixed-order reduction)

// The gradient from the summed partials (gx = sum_i x_i d ll/dx_i,
// gs = 2 d ll/ds_n, quad = y^T C^-1 y, nobs observed steps).  x = lam dt with
// lam = sqrt(2b - 1)/l, so d ll/dl = -gx / l; s_f from the scaling identity.
__device__ __forceinline__ void chain_grad(double gx, double gs, double quad, double nobs, const double* theta,
                                           double* g) {
    const double ell = theta[0], sf = theta[1], s2 = theta[2];
    g[0] = -gx / ell;
    g[2] = 0.5 * gs;
    g[1] = (0.5 * (quad - nobs) - s2 * g[2]) / sf;
}

template <int B>
__global__ void __launch_bounds__(256) k_finalize(const double* __restrict__ part, int64_t nb, int na,
                                                  const double* __restrict__ theta, double* __restrict__ ll_out,
                                                  double* __restrict__ grad_out) {
    __shared__ double red[256 * Acc<B>::N];
    const int tid = threadIdx.x;
    for (int f = 0; f < na; ++f) {
        double s = 0.0;
        for (int64_t c = tid; c < nb; c += 256) s += part[f * nb + c];
        red[f * 256 + tid] = s;
    }
    __syncthreads();
    for (int w = 128; w > 0; w >>= 1) {
        if (tid < w)
            for (int f = 0; f < na; ++f) red[f * 256 + tid] += red[f * 256 + tid + w];
        __syncthreads();
    }
    if (tid == 0) {
        if (ll_out) ll_out[0] = red[0];
        if (grad_out && na == Acc<B>::N)
            chain_grad(red[1 * 256], red[2 * 256], red[3 * 256], red[4 * 256], theta, grad_out);
    }
}

// ------------------------------------------------------------------ batches: chunk offsets and per-series sums

// cstart[i] = sum_{k<i} ceil(len_k / L), one CTA.  Offsets must start at 0,
// never decrease and end at n_total; otherwise EINVAL is recorded and every
// series gets zero chunks, so the later kernels touch nothing.
static constexpr int CS_THREADS = 1024;

__global__ void __launch_bounds__(CS_THREADS) k_chunk_starts(const int64_t* __restrict__ offsets, int64_t nseries,
                                                            int64_t n_total, int64_t L, int64_t* __restrict__ cstart,
                                                            int* status) {
    __shared__ int64_t wsum[CS_THREADS / 32];
    __shared__ int bad_any;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    if (tid == 0) bad_any = (offsets[0] != 0 || offsets[nseries] != n_total) ? 1 : 0;
    __syncthreads();
    int bad = 0;
    for (int64_t i = tid; i < nseries; i += CS_THREADS)
        if (offsets[i + 1] < offsets[i]) bad = 1;
    if (bad) atomicOr(&bad_any, 1);
    __syncthreads();
    const bool ok = bad_any == 0;
    if (!ok && tid == 0) atomicOr(status, ST_EINVAL);
    int64_t carry = 0;
    for (int64_t base = 0; base < nseries; base += CS_THREADS) {
        const int64_t i = base + tid;
        int64_t cnt = 0;
        if (ok && i < nseries) cnt = (offsets[i + 1] - offsets[i] + L - 1) / L;
        // inclusive warp scan, then across warps
        int64_t x = cnt;
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
            const int64_t yv = __shfl_up_sync(0xffffffffu, x, d);
            if (lane >= d) x += yv;
        }
        if (lane == 31) wsum[warp] = x;
        __syncthreads();
        if (warp == 0) {
            int64_t w = (lane < CS_THREADS / 32) ? wsum[lane] : 0;
#pragma unroll
            for (int d = 1; d < 32; d <<= 1) {
                const int64_t yv = __shfl_up_sync(0xffffffffu, w, d);
                if (lane >= d) w += yv;
            }
            if (lane < CS_THREADS / 32) wsum[lane] = w;
        }
        __syncthreads();
        const int64_t before = carry + (warp > 0 ? wsum[warp - 1] : 0) + x - cnt;
        if (i < nseries) cstart[i] = before;
        carry += wsum[CS_THREADS / 32 - 1];
        __syncthreads();
    }
    if (tid == 0) cstart[nseries] = carry;
}

// One warp per series: fixed-order sum of its chunks' partials, chain rule.
template <int B>
__global__ void __launch_bounds__(256) k_finalize_batched(const double* __restrict__ part, int64_t nc, int na,
                                                          const int64_t* __restrict__ cstart, int64_t nseries,
                                                          const double* __restrict__ theta, int P,
                                                          double* __restrict__ ll_out, double* __restrict__ grad_out) {
    constexpr int NA = Acc<B>::N;
    const int64_t w = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (w >= nseries) return;
    const int64_t c0 = cstart[w], c1 = cstart[w + 1];
    double acc[NA];
#pragma unroll
    for (int f = 0; f < NA; ++f) acc[f] = 0.0;
    for (int64_t c = c0 + lane; c < c1; c += 32)
#pragma unroll
        for (int f = 0; f < NA; ++f)
            if (f < na) acc[f] += part[f * nc + c];
#pragma unroll
    for (int d = 16; d > 0; d >>= 1)
#pragma unroll
        for (int f = 0; f < NA; ++f) acc[f] += __shfl_xor_sync(0xffffffffu, acc[f], d);
    if (lane == 0) {
        if (ll_out) ll_out[w] = acc[0];
        if (grad_out && na == NA) chain_grad(acc[1], acc[2], acc[3], acc[4], theta + w * P, grad_out + w * P);
    }
}

// ------------------------------------------------------------------ host side

// grid-level reduction of the block totals: tiles of SCAN_TS elements, one
// CTA each; small tiles keep each level spread over many SMs

static size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

static bool single_tile(int64_t ne) { return ne <= (int64_t)SCAN_TS; }
static int64_t mid_tiles(int64_t ne) { return (ne + SCAN_TS - 1) / SCAN_TS; }

// Workspace: [status | tree nodes | block totals | block prefix | block suffix |
//             grid scan levels | transition per step | block partials | stored steps |
//             elimination state between pieces | the ranks' elements of a split series]
static constexpr int SEG_MAX = SEG_MAX_RANKS;   // ranks of a split series (one scan tile)
template <int B>
struct Layout {
    int64_t nc, nb;
    size_t off_nodes, off_btot, off_bpre, off_bsuf, off_phis, off_part, off_store, off_state, off_seg, total;
    int nlev;
    int64_t lev_n[8];
    size_t lev_tot[8], lev_pre[8], lev_suf[8];

    size_t off_cstart;

    // one series of n steps (nseries = 0), or a batch of nseries series with
    // n steps in total (chunk slots: an upper bound on the chunk count)
    Layout(int64_t n, int64_t L, int mode, int64_t nseries = 0) {
        constexpr int NE = Dims<B>::NE, NM = Dims<B>::NM;
        nc = (n + L - 1) / L + nseries;
        nb = (nc + CTA - 1) / CTA;
        size_t o = 256;  // status word region
        off_cstart = o;
        if (nseries > 0) o = align256(o + sizeof(int64_t) * (size_t)(nseries + 1));
        off_nodes = o; o = align256(o + sizeof(double) * NE * (size_t)nb * TREE);
        off_btot = o; o = align256(o + sizeof(double) * NE * nb);
        off_bpre = o; o = align256(o + sizeof(double) * NM * nb);
        off_bsuf = o; o = align256(o + sizeof(double) * NM * nb);
        nlev = 0;
        int64_t ne = nb;
        while (!single_tile(ne)) {
            const int64_t nt = mid_tiles(ne);
            lev_n[nlev] = nt;
            lev_tot[nlev] = o; o = align256(o + sizeof(double) * NE * nt);
            lev_pre[nlev] = o; o = align256(o + sizeof(double) * NM * nt);
            lev_suf[nlev] = o; o = align256(o + sizeof(double) * NM * nt);
            ++nlev;
            ne = nt;
        }
        off_phis = o; o = align256(o + sizeof(double) * (size_t)NPH * L * nc);
        off_part = o; o = align256(o + sizeof(double) * Acc<B>::N * (nseries > 0 ? nc : nb));
        off_store = o;
        if (mode != MODE_LOGLIK) o = align256(o + sizeof(double) * Stored<B>::N * (size_t)L * nc);
        off_state = o; o = align256(o + sizeof(double) * (NE + 1) * (size_t)nc);   // a piecewise elimination
        off_seg = o; o = align256(o + sizeof(double) * (SEG_MAX * (NE + 2 * NM) + 2 * NM));   // split series
        total = o;
    }
};

// top_pre / top_suf: the state before the first element and the information
// after the last (NM contiguous doubles each), or NULL for a whole series
// (up = false: the level totals are already in the workspace, from scan_total)
template <int B>
static void scan_level(const double* E, int64_t ne, double* pre_out, double* suf_out, const Layout<B>& lay,
                       char* ws, int lev, cudaStream_t st, const double* top_pre = nullptr,
                       const double* top_suf = nullptr, bool up = true) {
    const size_t smem = ScanSmem<B>::bytes;
    if (single_tile(ne)) {
        k_scan_tile<B, true><<<1, SCAN_CTA, smem, st>>>(E, ne, nullptr, 1, top_pre, top_suf, pre_out, suf_out);
        return;
    }
    const int64_t nt = lay.lev_n[lev];
    double* tot = (double*)(ws + lay.lev_tot[lev]);
    double* tpre = (double*)(ws + lay.lev_pre[lev]);
    double* tsuf = (double*)(ws + lay.lev_suf[lev]);
    if (up)
        k_scan_tile<B, false><<<(unsigned)nt, SCAN_CTA, smem, st>>>(E, ne, tot, nt, nullptr, nullptr, nullptr,
                                                                    nullptr);
    scan_level<B>(tot, nt, tpre, tsuf, lay, ws, lev + 1, st, top_pre, top_suf, up);
    k_scan_tile<B, true><<<(unsigned)nt, SCAN_CTA, smem, st>>>(E, ne, nullptr, nt, tpre, tsuf, pre_out, suf_out);
}

// the up-sweep only: the single element of all ne (NE contiguous doubles)
template <int B>
static void scan_total(const double* E, int64_t ne, double* total, const Layout<B>& lay, char* ws, int lev,
                       cudaStream_t st) {
    const size_t smem = ScanSmem<B>::bytes;
    if (single_tile(ne)) {
        k_scan_tile<B, false><<<1, SCAN_CTA, smem, st>>>(E, ne, total, 1, nullptr, nullptr, nullptr, nullptr);
        return;
    }
    const int64_t nt = lay.lev_n[lev];
    double* tot = (double*)(ws + lay.lev_tot[lev]);
    k_scan_tile<B, false><<<(unsigned)nt, SCAN_CTA, smem, st>>>(E, ne, tot, nt, nullptr, nullptr, nullptr, nullptr);
    scan_total<B>(tot, nt, total, lay, ws, lev + 1, st);
}

template <int B>
static int scan_launches(int64_t ne, const Layout<B>& lay, int lev) {
    if (single_tile(ne)) return 1;
    return 2 + scan_launches<B>(lay.lev_n[lev], lay, lev + 1);
}

template <int B>
size_t matern_ws_bytes_t(int64_t n, int64_t L, int mode) { return Layout<B>(n, L, mode).total; }

template <int B>
int matern_launch_count_t(int64_t n, int64_t L, int mode) {
    Layout<B> lay(n, L, mode);
    return 1 + scan_launches<B>(lay.nb, lay, 0) + 1 + 1;
}

template <int B>
int matern_run_t(int mode, const double* t, const double* y, int64_t n, int64_t L, const double* theta,
                 double* ll_out, double* grad_out, double* mean_out, double* var_out, void* wsv, cudaStream_t st,
                 cudaEvent_t* ev, int missing, const HostFeed* feed, double* lag1_out) {
    Layout<B> lay(n, L, mode);
    char* ws = (char*)wsv;
    int* status = (int*)ws;
    double* nodes = (double*)(ws + lay.off_nodes);
    double* btot = (double*)(ws + lay.off_btot);
    double* bpre = (double*)(ws + lay.off_bpre);
    double* bsuf = (double*)(ws + lay.off_bsuf);
    double* phis = (double*)(ws + lay.off_phis);
    double* part = (double*)(ws + lay.off_part);
    double* store = (double*)(ws + lay.off_store);
    double* state = (double*)(ws + lay.off_state);
    ChainArgs a{t, y, n, L, lay.nc, lay.nb, theta, status, nullptr, nullptr, 0, 3, missing, 0, 0.0,
                (mode == MODE_POSTERIOR || mode == MODE_GRAD_POSTERIOR) ? lag1_out : nullptr};
    const unsigned grid = (unsigned)lay.nb;
    if (cudaMemsetAsync(status, 0, sizeof(int), st) != cudaSuccess) return 1;
    if (ev) cudaEventRecord(ev[0], st);
    if (!feed) {
        k_fold<B, false><<<grid, CTA, 0, st>>>(a, nodes, btot, phis, 0, L, state, 1, 1);
    } else {
        // t and y arrive from host memory in pieces of steps: piece p holds
        // steps [bnd[p], bnd[p+1]) of every chunk (strided copies, chunk = row
        // of L steps), and fold launch p eliminates exactly those steps once
        // its copy is done.  The copy of piece p+1 overlaps the fold of piece
        // p, and every launch keeps all SMs busy.  The widths double from
        // L/16 (a step column copies about twice as fast as it folds), so the
        // first copy, which nothing overlaps, is short.  Piece 0 also carries
        // the step before each chunk (its first transition needs that time).
        int64_t bnd[FEED_PIECES + 1];
        int64_t np = 0;
        bnd[0] = 0;
        for (int64_t w = max((int64_t)1, (L + 15) / 16); bnd[np] < L && np < feed->npieces; w *= 2, ++np)
            bnd[np + 1] = (np + 1 == feed->npieces) ? L : min(L, bnd[np] + w);
        const int64_t nfull = n / L, tail = n - nfull * L;
        if (cudaEventRecord(feed->ev[0], st) != cudaSuccess) return 1;
        if (cudaStreamWaitEvent(feed->copy, feed->ev[0], 0) != cudaSuccess) return 1;
        if (feed->theta_h && cudaMemcpyAsync(const_cast<double*>(theta), feed->theta_h, feed->theta_bytes,
                                             cudaMemcpyHostToDevice, feed->copy) != cudaSuccess)
            return 1;
        for (int64_t p = 0; p < np; ++p) {
            const int64_t c0 = bnd[p], c1 = bnd[p + 1];
            const bool prev = (p == 0 && c1 < L);   // piece 0 also copies column L-1 of the row before
            for (int arr = 0; arr < 2; ++arr) {
                double* dst = const_cast<double*>(arr ? y : t);
                const double* src = arr ? feed->y : feed->t;
                const size_t w = sizeof(double) * (size_t)(c1 - c0), pitch = sizeof(double) * (size_t)L;
                if (!prev) {
                    if (nfull > 0 && cudaMemcpy2DAsync(dst + c0, pitch, src + c0, pitch, w, (size_t)nfull,
                                                       cudaMemcpyHostToDevice, feed->copy) != cudaSuccess)
                        return 1;
                } else {
                    // row 0, then rows 1.. from one step before their start (c1 + 1 <= L)
                    if (nfull > 0 && cudaMemcpyAsync(dst, src, w, cudaMemcpyHostToDevice, feed->copy) != cudaSuccess)
                        return 1;
                    if (nfull > 1 &&
                        cudaMemcpy2DAsync(dst + L - 1, pitch, src + L - 1, pitch, w + sizeof(double),
                                          (size_t)(nfull - 1), cudaMemcpyHostToDevice, feed->copy) != cudaSuccess)
                        return 1;
                }
                if (tail > c0) {   // the last, shorter chunk
                    const int64_t b0 = nfull * L + c0 - ((prev && nfull > 0) ? 1 : 0);
                    const int64_t b1 = nfull * L + min(c1, tail);
                    if (cudaMemcpyAsync(dst + b0, src + b0, sizeof(double) * (size_t)(b1 - b0),
                                        cudaMemcpyHostToDevice, feed->copy) != cudaSuccess)
                        return 1;
                }
            }
            if (cudaEventRecord(feed->ev[1 + p], feed->copy) != cudaSuccess) return 1;
            if (cudaStreamWaitEvent(st, feed->ev[1 + p], 0) != cudaSuccess) return 1;
            k_fold<B, false><<<grid, CTA, 0, st>>>(a, nodes, btot, phis, c0, c1, state, p == 0 ? 1 : 0,
                                                   p == np - 1 ? 1 : 0);
        }
    }
    if (ev) cudaEventRecord(ev[1], st);
    scan_level<B>(btot, lay.nb, bpre, bsuf, lay, ws, 0, st);
    if (ev) cudaEventRecord(ev[2], st);
    int na = 1;
    switch (mode) {
    case MODE_LOGLIK:
        k_chunk<B, MODE_LOGLIK, false><<<grid, CTA, 0, st>>>(a, nodes, bpre, bsuf, phis, store, part, nullptr,
                                                            nullptr);
        break;
    case MODE_GRAD:
        k_chunk<B, MODE_GRAD, false><<<grid, CTA, 0, st>>>(a, nodes, bpre, bsuf, phis, store, part, nullptr,
                                                          nullptr);
        na = Acc<B>::N;
        break;
    case MODE_GRAD_POSTERIOR:
        k_chunk<B, MODE_GRAD_POSTERIOR, false><<<grid, CTA, 0, st>>>(a, nodes, bpre, bsuf, phis, store, part,
                                                                    mean_out, var_out);
        na = Acc<B>::N;
        break;
    default:
        k_chunk<B, MODE_POSTERIOR, false><<<grid, CTA, 0, st>>>(a, nodes, bpre, bsuf, phis, store, part, mean_out,
                                                        var_out);
        break;
    }
    if (ev) cudaEventRecord(ev[3], st);
    // the final reduction always runs (it is cheap), so the launch count is fixed per kind
    k_finalize<B><<<1, 256, 0, st>>>(part, lay.nb, na, theta, ll_out, grad_out);
    if (ev) cudaEventRecord(ev[4], st);
    return cudaGetLastError() == cudaSuccess ? 0 : 1;
}

template <int B>
size_t matern_ws_bytes_batched_t(int64_t nseries, int64_t n_total, int64_t L, int mode) {
    return Layout<B>(n_total, L, mode, nseries).total;
}

template <int B>
int matern_launch_count_batched_t(int64_t nseries, int64_t n_total, int64_t L, int mode) {
    Layout<B> lay(n_total, L, mode, nseries);
    return 1 + 1 + scan_launches<B>(lay.nb, lay, 0) + 1 + 1;
}

template <int B>
int matern_run_batched_t(int mode, const int64_t* offsets, int64_t nseries, int64_t n_total, const double* t,
                         const double* y, int64_t L, const double* theta, double* ll_out, double* grad_out,
                         double* mean_out, double* var_out, void* wsv, cudaStream_t st, cudaEvent_t* ev,
                         int missing) {
    Layout<B> lay(n_total, L, mode, nseries);
    char* ws = (char*)wsv;
    int* status = (int*)ws;
    int64_t* cstart = (int64_t*)(ws + lay.off_cstart);
    double* nodes = (double*)(ws + lay.off_nodes);
    double* btot = (double*)(ws + lay.off_btot);
    double* bpre = (double*)(ws + lay.off_bpre);
    double* bsuf = (double*)(ws + lay.off_bsuf);
    double* phis = (double*)(ws + lay.off_phis);
    double* part = (double*)(ws + lay.off_part);
    double* store = (double*)(ws + lay.off_store);
    double* state = (double*)(ws + lay.off_state);
    ChainArgs a{t, y, n_total, L, lay.nc, lay.nb, theta, status, offsets, cstart, nseries, 3, missing, 0, 0.0};
    const unsigned grid = (unsigned)lay.nb;
    if (cudaMemsetAsync(status, 0, sizeof(int), st) != cudaSuccess) return 1;
    if (ev) cudaEventRecord(ev[0], st);
    k_chunk_starts<<<1, CS_THREADS, 0, st>>>(offsets, nseries, n_total, L, cstart, status);
    k_fold<B, true><<<grid, CTA, 0, st>>>(a, nodes, btot, phis, 0, L, state, 1, 1);
    if (ev) cudaEventRecord(ev[1], st);
    scan_level<B>(btot, lay.nb, bpre, bsuf, lay, ws, 0, st);
    if (ev) cudaEventRecord(ev[2], st);
    int na = 1;
    switch (mode) {
    case MODE_LOGLIK:
        k_chunk<B, MODE_LOGLIK, true><<<grid, CTA, 0, st>>>(a, nodes, bpre, bsuf, phis, store, part, nullptr,
                                                           nullptr);
        break;
    case MODE_GRAD:
        k_chunk<B, MODE_GRAD, true><<<grid, CTA, 0, st>>>(a, nodes, bpre, bsuf, phis, store, part, nullptr,
                                                         nullptr);
        na = Acc<B>::N;
        break;
    case MODE_GRAD_POSTERIOR:
        k_chunk<B, MODE_GRAD_POSTERIOR, true><<<grid, CTA, 0, st>>>(a, nodes, bpre, bsuf, phis, store, part,
                                                                   mean_out, var_out);
        na = Acc<B>::N;
        break;
    default:
        k_chunk<B, MODE_POSTERIOR, true><<<grid, CTA, 0, st>>>(a, nodes, bpre, bsuf, phis, store, part, mean_out,
                                                              var_out);
        break;
    }
    if (ev) cudaEventRecord(ev[3], st);
    const unsigned fgrid = (unsigned)((nseries * 32 + 255) / 256);
    k_finalize_batched<B><<<fgrid, 256, 0, st>>>(part, lay.nc, na, cstart, nseries, theta, 3, ll_out, grad_out);
    if (ev) cudaEventRecord(ev[4], st);
    return cudaGetLastError() == cudaSuccess ? 0 : 1;
}

// ------------------------------------------------------------------ a series split across ranks
//
// Rank r of G holds a contiguous range of the series.  Phase 0 reduces the
// range to one element: the in-chunk elimination and the up-sweep, whose
// total is the Schur complement of K~ on the state before the range and the
// range's last state (for the first range, A = 0: it starts from the prior).
// The ranks' elements are all-gathered.  Phase 1 runs the same odd-even
// reduction over the G elements (one scan tile) for the state before this
// range and the information after it, then this range's down-sweep, chunk
// pass and final reduction: its share of the log-likelihood and gradient
// (the final reduction is linear in the partial sums, so the shares add up).
// Phase 1 reuses the workspace that phase 0 filled.

// elements arrive rank-major ([G][NE]); the scan reads them field-major
__global__ void __launch_bounds__(256) k_elems_to_soa(const double* __restrict__ in, double* __restrict__ out, int G,
                                                      int ne) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < G * ne) {
        const int k = i / ne, f = i % ne;
        out[f * G + k] = in[i];
    }
}

template <int B>
int matern_segment_t(int phase, const double* t, const double* y, int64_t n, int64_t L, const double* theta,
                     double t_prev, int first, const double* elems, int G, int rank, double* elem_out,
                     double* ll_out, double* grad_out, void* wsv, cudaStream_t st, int missing, double* mean_out,
                     double* var_out) {
    constexpr int NE = Dims<B>::NE, NM = Dims<B>::NM;
    if (G < 1 || G > SEG_MAX || rank < 0 || rank >= G) return 1;
    Layout<B> lay(n, L, MODE_GRAD);
    char* ws = (char*)wsv;
    int* status = (int*)ws;
    double* nodes = (double*)(ws + lay.off_nodes);
    double* btot = (double*)(ws + lay.off_btot);
    double* bpre = (double*)(ws + lay.off_bpre);
    double* bsuf = (double*)(ws + lay.off_bsuf);
    double* phis = (double*)(ws + lay.off_phis);
    double* part = (double*)(ws + lay.off_part);
    double* store = (double*)(ws + lay.off_store);
    double* state = (double*)(ws + lay.off_state);
    ChainArgs a{t, y, n, L, lay.nc, lay.nb, theta, status, nullptr, nullptr, 0, 3, missing, first ? 0 : -1, t_prev};
    const unsigned grid = (unsigned)lay.nb;
    if (phase == 0) {
        if (cudaMemsetAsync(status, 0, sizeof(int), st) != cudaSuccess) return 1;
        k_fold<B, false><<<grid, CTA, 0, st>>>(a, nodes, btot, phis, 0, L, state, 1, 1);
        scan_total<B>(btot, lay.nb, elem_out, lay, ws, 0, st);
    } else {
        double* esoa = (double*)(ws + lay.off_seg);
        double* gpre = esoa + SEG_MAX * NE;
        double* gsuf = gpre + SEG_MAX * NM;
        double* tpre = gsuf + SEG_MAX * NM;
        double* tsuf = tpre + NM;
        k_elems_to_soa<<<(unsigned)((G * NE + 255) / 256), 256, 0, st>>>(elems, esoa, G, NE);
        k_scan_tile<B, true><<<1, SCAN_CTA, ScanSmem<B>::bytes, st>>>(esoa, G, nullptr, 1, nullptr, nullptr, gpre,
                                                                      gsuf);
        // this rank's entry (field f at f * G + rank) as NM contiguous doubles
        if (cudaMemcpy2DAsync(tpre, sizeof(double), gpre + rank, sizeof(double) * G, sizeof(double), NM,
                              cudaMemcpyDeviceToDevice, st) != cudaSuccess ||
            cudaMemcpy2DAsync(tsuf, sizeof(double), gsuf + rank, sizeof(double) * G, sizeof(double), NM,
                              cudaMemcpyDeviceToDevice, st) != cudaSuccess)
            return 1;
        scan_level<B>(btot, lay.nb, bpre, bsuf, lay, ws, 0, st, tpre, tsuf, false);
        if (mean_out)
            k_chunk<B, MODE_GRAD_POSTERIOR, false><<<grid, CTA, 0, st>>>(a, nodes, bpre, bsuf, phis, store, part,
                                                                        mean_out, var_out);
        else
            k_chunk<B, MODE_GRAD, false><<<grid, CTA, 0, st>>>(a, nodes, bpre, bsuf, phis, store, part, nullptr,
                                                              nullptr);
        k_finalize<B><<<1, 256, 0, st>>>(part, lay.nb, Acc<B>::N, theta, ll_out, grad_out);
    }
    return cudaGetLastError() == cudaSuccess ? 0 : 1;
}

template <int B>
static void set_smem_attr() {
    cudaFuncSetAttribute(k_scan_tile<B, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)ScanSmem<B>::bytes);
    cudaFuncSetAttribute(k_scan_tile<B, false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)ScanSmem<B>::bytes);
}

size_t matern_ws_bytes(int b, int64_t n, int64_t L, int mode) {
    switch (b) {
    case 1: return matern_ws_bytes_t<1>(n, L, mode);
    case 2: return matern_ws_bytes_t<2>(n, L, mode);
    default: return matern_ws_bytes_t<3>(n, L, mode);
    }
}

int matern_prepare() {
    set_smem_attr<1>();
    set_smem_attr<2>();
    set_smem_attr<3>();
    return cudaGetLastError() == cudaSuccess ? 0 : 1;
}

int matern_run(int b, int mode, const double* t, const double* y, int64_t n, int64_t L, const double* theta,
               double* ll_out, double* grad_out, double* mean_out, double* var_out, void* ws, cudaStream_t st,
               cudaEvent_t* ev, int missing, const HostFeed* feed, double* lag1_out) {
    switch (b) {
    case 1:
        return matern_run_t<1>(mode, t, y, n, L, theta, ll_out, grad_out, mean_out, var_out, ws, st, ev, missing, feed, lag1_out);
    case 2:
        return matern_run_t<2>(mode, t, y, n, L, theta, ll_out, grad_out, mean_out, var_out, ws, st, ev, missing, feed, lag1_out);
    default:
        return matern_run_t<3>(mode, t, y, n, L, theta, ll_out, grad_out, mean_out, var_out, ws, st, ev, missing, feed, lag1_out);
    }
}

size_t matern_ws_bytes_batched(int b, int64_t nseries, int64_t n_total, int64_t L, int mode) {
    switch (b) {
    case 1: return matern_ws_bytes_batched_t<1>(nseries, n_total, L, mode);
    case 2: return matern_ws_bytes_batched_t<2>(nseries, n_total, L, mode);
    default: return matern_ws_bytes_batched_t<3>(nseries, n_total, L, mode);
    }
}

int matern_launch_count_batched(int b, int64_t nseries, int64_t n_total, int64_t L, int mode) {
    switch (b) {
    case 1: return matern_launch_count_batched_t<1>(nseries, n_total, L, mode);
    case 2: return matern_launch_count_batched_t<2>(nseries, n_total, L, mode);
    default: return matern_launch_count_batched_t<3>(nseries, n_total, L, mode);
    }
}

int matern_run_batched(int b, int mode, const int64_t* offsets, int64_t nseries, int64_t n_total, const double* t,
                       const double* y, int64_t L, const double* theta, double* ll_out, double* grad_out,
                       double* mean_out, double* var_out, void* ws, cudaStream_t st, cudaEvent_t* ev, int missing) {
    switch (b) {
    case 1: return matern_run_batched_t<1>(mode, offsets, nseries, n_total, t, y, L, theta, ll_out, grad_out,
                                           mean_out, var_out, ws, st, ev, missing);
    case 2: return matern_run_batched_t<2>(mode, offsets, nseries, n_total, t, y, L, theta, ll_out, grad_out,
                                           mean_out, var_out, ws, st, ev, missing);
    default: return matern_run_batched_t<3>(mode, offsets, nseries, n_total, t, y, L, theta, ll_out, grad_out,
                                            mean_out, var_out, ws, st, ev, missing);
    }
}

int matern_segment(int b, int phase, const double* t, const double* y, int64_t n, int64_t L, const double* theta,
                   double t_prev, int first, const double* elems, int G, int rank, double* elem_out, double* ll_out,
                   double* grad_out, void* ws, cudaStream_t st, int missing, double* mean_out, double* var_out) {
    switch (b) {
    case 1: return matern_segment_t<1>(phase, t, y, n, L, theta, t_prev, first, elems, G, rank, elem_out, ll_out,
                                       grad_out, ws, st, missing, mean_out, var_out);
    case 2: return matern_segment_t<2>(phase, t, y, n, L, theta, t_prev, first, elems, G, rank, elem_out, ll_out,
                                       grad_out, ws, st, missing, mean_out, var_out);
    default: return matern_segment_t<3>(phase, t, y, n, L, theta, t_prev, first, elems, G, rank, elem_out, ll_out,
                                        grad_out, ws, st, missing, mean_out, var_out);
    }
}
int matern_elem_size(int b) { return b == 1 ? Dims<1>::NE : b == 2 ? Dims<2>::NE : Dims<3>::NE; }

// launches of both phases: fold + up-sweep; transpose, the ranks' scan tile,
// the range's down-sweep, chunk pass, final reduction
template <int B>
static int segment_launches_t(int64_t n, int64_t L) {
    Layout<B> lay(n, L, MODE_GRAD);
    return 1 + (lay.nlev + 1) + 2 + (lay.nlev + 1) + 2;
}
int matern_segment_launch_count(int b, int64_t n, int64_t L) {
    return b == 1 ? segment_launches_t<1>(n, L) : b == 2 ? segment_launches_t<2>(n, L) : segment_launches_t<3>(n, L);
}

int matern_launch_count(int b, int64_t n, int64_t L, int mode) {
    switch (b) {
    case 1: return matern_launch_count_t<1>(n, L, mode);
    case 2: return matern_launch_count_t<2>(n, L, mode);
    default: return matern_launch_count_t<3>(n, L, mode);
    }
}

}  // namespace spg
