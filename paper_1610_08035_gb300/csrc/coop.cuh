// coop.cuh -- lane-cooperative forms of the chain-element algebra (b <= 3).
//
// The upper levels of an odd-even tree have few combines each, and every
// level is a chain of dependent FP64 work.  With one combine per thread a
// warp issues the combine's ~370 FP64 instructions one after another, and on
// GB300 every FP64 warp instruction costs its SM sub-partition the same issue
// time however few lanes are active.  Here one element is spread over a group
// of W lanes (W = 1, 4, 16 for b = 1, 2, 3): lane q = B r + c holds entry
// (r, c) of A, C and J and the row entries bv[r], eta[r], so a b x b product
// is b FMAs per lane after 2b shuffles, and a combine issues ~80 FP64
// instructions.  Lanes q >= b^2 (b = 3) mirror a valid entry and never
// store.  The arithmetic follows the single-thread forms in chain.cuh term by
// term (same products, same pivoting, same symmetrisation), so the two differ
// only in the order in which products are summed where a shuffle reorders
// nothing: both sum k = 0 .. b-1 left to right.
#pragma once

#include "chain.cuh"

namespace spg {

template <int B>
struct Coop {
    static constexpr int W = (B == 1) ? 1 : (B == 2) ? 4 : 16;   // lanes per group
    static constexpr int NG_WARP = 32 / W;                       // groups per warp
};

// position of this lane inside its group: (row, col) of the entry it holds
template <int B>
struct CPos {
    int q, row, col;
    bool valid;   // q < b^2: the lane owns its entry (stores it)
    __device__ __forceinline__ CPos() {
        q = threadIdx.x & (Coop<B>::W - 1);
        valid = q < B * B;
        const int qq = valid ? q : q % (B * B);
        row = qq / B;
        col = qq % B;
    }
};

template <int B>
__device__ __forceinline__ double csh(double v, int src) {
    return __shfl_sync(0xffffffffu, v, src, Coop<B>::W);
}

// (X Y)[r][c], (X^T Y)[r][c], (X Y^T)[r][c]
template <int B>
__device__ __forceinline__ double cmm(double X, double Y, const CPos<B>& p) {
    double s = csh<B>(X, p.row * B) * csh<B>(Y, p.col);
#pragma unroll
    for (int k = 1; k < B; ++k) s = fma(csh<B>(X, p.row * B + k), csh<B>(Y, k * B + p.col), s);
    return s;
}
template <int B>
__device__ __forceinline__ double cmtm(double X, double Y, const CPos<B>& p) {
    double s = csh<B>(X, p.row) * csh<B>(Y, p.col);
#pragma unroll
    for (int k = 1; k < B; ++k) s = fma(csh<B>(X, k * B + p.row), csh<B>(Y, k * B + p.col), s);
    return s;
}
template <int B>
__device__ __forceinline__ double cmmt(double X, double Y, const CPos<B>& p) {
    double s = csh<B>(X, p.row * B) * csh<B>(Y, p.col * B);
#pragma unroll
    for (int k = 1; k < B; ++k) s = fma(csh<B>(X, p.row * B + k), csh<B>(Y, p.col * B + k), s);
    return s;
}
// (X v)[r], (X^T v)[r] for a row-replicated vector v (v[k] held by row k's lanes)
template <int B>
__device__ __forceinline__ double cmv(double X, double v, const CPos<B>& p) {
    double s = csh<B>(X, p.row * B) * csh<B>(v, 0);
#pragma unroll
    for (int k = 1; k < B; ++k) s = fma(csh<B>(X, p.row * B + k), csh<B>(v, k * B), s);
    return s;
}
template <int B>
__device__ __forceinline__ double cmtv(double X, double v, const CPos<B>& p) {
    double s = csh<B>(X, p.row) * csh<B>(v, 0);
#pragma unroll
    for (int k = 1; k < B; ++k) s = fma(csh<B>(X, k * B + p.row), csh<B>(v, k * B), s);
    return s;
}
// a product known to be symmetric: keep the upper triangle, mirror it
template <int B>
__device__ __forceinline__ double csym_upper(double v, const CPos<B>& p) {
    const double m = csh<B>(v, p.col * B + p.row);
    return (p.row <= p.col) ? v : m;
}

// Inverse by Gauss-Jordan elimination with partial pivoting (the pivot rule
// of inv_pp: the first largest |a[i][k]|, i >= k).
template <int B>
__device__ __forceinline__ double cinv(double N, const CPos<B>& p) {
    double a = N, R = (p.row == p.col) ? 1.0 : 0.0;
#pragma unroll
    for (int k = 0; k < B; ++k) {
        int piv = k;
        double best = fabs(csh<B>(a, k * B + k));
#pragma unroll
        for (int i = k + 1; i < B; ++i) {
            const double v = fabs(csh<B>(a, i * B + k));
            if (v > best) { best = v; piv = i; }
        }
        {   // row swap k <-> piv (the identity when piv == k); every lane of the
            // warp shuffles, whatever its group's pivot
            const int src = (p.row == k) ? piv : (p.row == piv) ? k : p.row;
            a = csh<B>(a, src * B + p.col);
            R = csh<B>(R, src * B + p.col);
        }
        const double inv = 1.0 / csh<B>(a, k * B + k);
        if (p.row == k) { a *= inv; R *= inv; }
        const double f = csh<B>(a, p.row * B + k);
        const double ak = csh<B>(a, k * B + p.col), Rk = csh<B>(R, k * B + p.col);
        if (p.row != k) { a = fma(-f, ak, a); R = fma(-f, Rk, R); }
    }
    return R;
}

// ------------------------------------------------------------------ distributed elements and states

struct CElem { double A, C, J, bv, eta; };
struct CVS { double v, S; };   // a state (m, P) or information (eta, J)

template <int B>
__device__ __forceinline__ void celem_identity(CElem& e, const CPos<B>& p) {
    e.A = (p.row == p.col) ? 1.0 : 0.0;
    e.C = 0.0; e.J = 0.0; e.bv = 0.0; e.eta = 0.0;
}

// field offsets of the packed element (the order of elem_store)
template <int B>
struct EF {
    static constexpr int NS = Dims<B>::NS;
    static constexpr int BV = B * B, C = B * B + B, ETA = B * B + B + NS, J = B * B + 2 * B + NS;
};

template <int B>
__device__ __forceinline__ void celem_load(const double* __restrict__ base, int64_t ld, int64_t k, CElem& e,
                                           const CPos<B>& p) {
    const int s = sidx<B>(p.row, p.col);
    e.A = base[(int64_t)(p.row * B + p.col) * ld + k];
    e.bv = base[(int64_t)(EF<B>::BV + p.row) * ld + k];
    e.C = base[(int64_t)(EF<B>::C + s) * ld + k];
    e.eta = base[(int64_t)(EF<B>::ETA + p.row) * ld + k];
    e.J = base[(int64_t)(EF<B>::J + s) * ld + k];
}
template <int B>
__device__ __forceinline__ void celem_store(double* __restrict__ base, int64_t ld, int64_t k, const CElem& e,
                                            const CPos<B>& p) {
    if (!p.valid) return;
    base[(int64_t)(p.row * B + p.col) * ld + k] = e.A;
    if (p.col == 0) {
        base[(int64_t)(EF<B>::BV + p.row) * ld + k] = e.bv;
        base[(int64_t)(EF<B>::ETA + p.row) * ld + k] = e.eta;
    }
    if (p.row <= p.col) {
        const int s = sidx<B>(p.row, p.col);
        base[(int64_t)(EF<B>::C + s) * ld + k] = e.C;
        base[(int64_t)(EF<B>::J + s) * ld + k] = e.J;
    }
}
template <int B>
__device__ __forceinline__ void cvs_load(const double* __restrict__ base, int64_t ld, int64_t k, CVS& x,
                                         const CPos<B>& p) {
    x.v = base[(int64_t)p.row * ld + k];
    x.S = base[(int64_t)(B + sidx<B>(p.row, p.col)) * ld + k];
}
template <int B>
__device__ __forceinline__ void cvs_store(double* __restrict__ base, int64_t ld, int64_t k, const CVS& x,
                                          const CPos<B>& p) {
    if (!p.valid) return;
    if (p.col == 0) base[(int64_t)p.row * ld + k] = x.v;
    if (p.row <= p.col) base[(int64_t)(B + sidx<B>(p.row, p.col)) * ld + k] = x.S;
}

// ------------------------------------------------------------------ the algebra (chain.cuh's forms)

// (ei then ej): M = (I + C_i J_j)^-1, A = A_j M A_i, bv = A_j M (bv_i + C_i eta_j) + bv_j,
// C = A_j M C_i A_j^T + C_j, eta = A_i^T M^T (eta_j - J_j bv_i) + eta_i, J = A_i^T M^T J_j A_i + J_i
template <int B>
__device__ __forceinline__ void ccombine(const CElem& ei, const CElem& ej, CElem& r, const CPos<B>& p) {
    double N = cmm<B>(ei.C, ej.J, p);
    if (p.row == p.col) N += 1.0;
    const double M = cinv<B>(N, p);
    double T = cmm<B>(M, ei.A, p);
    r.A = cmm<B>(ej.A, T, p);
    double w = cmv<B>(ei.C, ej.eta, p) + ei.bv;
    double z = cmv<B>(M, w, p);
    r.bv = cmv<B>(ej.A, z, p) + ej.bv;
    T = cmm<B>(M, ei.C, p);
    double U = cmm<B>(ej.A, T, p);
    r.C = csym_upper<B>(cmmt<B>(U, ej.A, p), p) + ej.C;
    w = ej.eta - cmv<B>(ej.J, ei.bv, p);
    z = cmtv<B>(M, w, p);
    r.eta = cmtv<B>(ei.A, z, p) + ei.eta;
    T = cmtm<B>(M, ej.J, p);
    U = cmm<B>(T, ei.A, p);
    r.J = csym_upper<B>(cmtm<B>(ei.A, U, p), p) + ei.J;
}

// N(m, P) before e pushed through e: M = (I + P J_e)^-1,
// m' = A_e M (m + P eta_e) + bv_e, P' = A_e M P A_e^T + C_e
template <int B>
__device__ __forceinline__ void cstate_through(const CVS& x, const CElem& e, CVS& o, const CPos<B>& p) {
    double N = cmm<B>(x.S, e.J, p);
    if (p.row == p.col) N += 1.0;
    const double M = cinv<B>(N, p);
    const double w = cmv<B>(x.S, e.eta, p) + x.v;
    const double z = cmv<B>(M, w, p);
    o.v = cmv<B>(e.A, z, p) + e.bv;
    const double T = cmm<B>(M, x.S, p);
    const double U = cmm<B>(e.A, T, p);
    o.S = csym_upper<B>(cmmt<B>(U, e.A, p), p) + e.C;
}

// information (eta, J) after e pulled back through e and joined with e's own:
// M = (I + C_e J)^-1, eta' = A_e^T M^T (eta - J bv_e) + eta_e, J' = A_e^T M^T J A_e + J_e
template <int B>
__device__ __forceinline__ void cinfo_through(const CElem& e, const CVS& x, CVS& o, const CPos<B>& p) {
    double N = cmm<B>(e.C, x.S, p);
    if (p.row == p.col) N += 1.0;
    const double M = cinv<B>(N, p);
    const double w = x.v - cmv<B>(x.S, e.bv, p);
    const double z = cmtv<B>(M, w, p);
    o.v = cmtv<B>(e.A, z, p) + e.eta;
    const double T = cmtm<B>(M, x.S, p);
    const double U = cmm<B>(T, e.A, p);
    o.S = csym_upper<B>(cmtm<B>(e.A, U, p), p) + e.J;
}

}  // namespace spg
