// chain.cuh -- device building blocks for Matern state-space chains (b <= 3).
//
// Coordinates.  For the Matern family of order b the companion matrix of
// (s + lam)^b satisfies F(lam) = lam D F1 D^-1 with D = diag(1, lam, .., lam^(b-1))
// and F1 the companion matrix of (s + 1)^b, and the stationary covariance is
// Pinf(lam) = s_f D P1 D with P1 lam-free (Sec. 2.1, Eq. ss_matern for b = 2).
// In the state z~ = D^-1 z the model reads
//     A_i = Phi(x_i) = expm(F1 x_i),  x_i = lam (t_{i+1} - t_i),
//     Pinf = s_f P1,  H = e_1^T,
// which is the same Gaussian process (H D = H), so the likelihood, the
// posterior of f = H z and their derivatives are unchanged, and the state
// entries stay O(1) for any lengthscale.  expm(F1 x) is exact in closed form:
// F1 + I is nilpotent, so expm(F1 x) = e^-x sum_{k<b} ((F1 + I) x)^k / k!
// (Eq. ss_matern asks for expm; this finite series is its exact value).
// dPhi/dx = F1 Phi.
//
// Elements.  A chunk of consecutive steps, conditioned on the state z_p just
// before it, is summarised by the Schur complement of the posterior precision
// K~ on its boundary (Theorem 1 makes this a b x b object), stored in
// conditional-covariance form instead of as precision blocks:
//     p(z_last | z_p, y_chunk) = N(A z_p + bv, C),
//     p(y_chunk | z_p) propto exp(-z_p^T J z_p / 2 + eta^T z_p).
// Eliminating the node between two adjacent chunks is the associative
// combine below (the element algebra of Sarkka & Garcia-Fernandez 2021, a
// published parallel-in-time Kalman formulation); it never forms Q^-1, whose
// condition number grows like (lam dt)^-(2b-2).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace spg {

// ------------------------------------------------------------------ Matern constants (scaled coordinates)

// F1 = companion matrix of (s+1)^b: ones on the superdiagonal, last row -binom(b, j).
template <int B>
__device__ __forceinline__ double fcoef(int j) {
    if constexpr (B == 1) return 1.0;
    else if constexpr (B == 2) return j == 0 ? 1.0 : 2.0;
    else return j == 0 ? 1.0 : 3.0;
}

// P1: unit-variance stationary covariance in scaled coordinates, from the
// derivatives of the covariance function at zero lag.
template <int B>
__device__ __forceinline__ double p1(int i, int j) {
    if constexpr (B <= 2) return i == j ? 1.0 : 0.0;
    else {
        if (i == j) return i == 1 ? (1.0 / 3.0) : 1.0;
        if (i + j == 2) return -1.0 / 3.0;
        return 0.0;
    }
}

// Phi(x) = expm(F1 x) given e = exp(-x).
template <int B>
__device__ __forceinline__ void phi(double x, double e, double (&P)[B][B]) {
    if constexpr (B == 1) {
        P[0][0] = e;
    } else if constexpr (B == 2) {
        const double ex = e * x;
        P[0][0] = e + ex; P[0][1] = ex;
        P[1][0] = -ex;    P[1][1] = e - ex;
    } else {
        const double ex = e * x, eh = 0.5 * ex * x;   // e x, e x^2 / 2
        P[0][0] = e + ex + eh;   P[0][1] = ex + 2.0 * eh;        P[0][2] = eh;
        P[1][0] = -eh;           P[1][1] = e + ex - 2.0 * eh;    P[1][2] = ex - eh;
        P[2][0] = eh - ex;       P[2][1] = 2.0 * eh - 3.0 * ex;  P[2][2] = e - 2.0 * ex + eh;
    }
}

// ------------------------------------------------------------------ Jordan coordinates (the chain kernels)
//
// F1 + I is nilpotent with one Jordan chain: (F1 + I) V = V N, where N has
// ones on the superdiagonal and V is unit lower triangular with columns
// v_1 = (1, -1, 1, ..) (the null vector of F1 + I) and (F1 + I) v_{k+1} = v_k
// (b = 2: V = [[1, 0], [-1, 1]]; b = 3: V = [[1, 0, 0], [-1, 1, 0], [1, -2, 1]]).
// The first row of V is e_1^T, so H V = H, and in the state w = V^-1 z~
//     A_i = e^-x T(x),  T(x) = sum_k (N x)^k / k!   (unit upper triangular Toeplitz),
//     Pinf = s_f PJ,  PJ = V^-1 P1 V^-T,  H = e_1^T,  dA/dx = (N - I) A.
// A product with T costs b(b-1)/2 multiply-adds per column where a dense A
// costs b^2, and a step's transition is carried by x and e^-x (the chain
// kernels store x, x^2/2, e^-x and e^-2x per step).

// PJ = V^-1 P1 V^-T (b = 2: [[1, 1], [1, 2]]; b = 3: [[1, 1, 2/3], [1, 4/3, 4/3], [2/3, 4/3, 8/3]]).
template <int B>
__device__ __forceinline__ double pj(int i, int j) {
    if constexpr (B == 1) return 1.0;
    else if constexpr (B == 2) return (i == 1 && j == 1) ? 2.0 : 1.0;
    else {
        const int lo = i < j ? i : j, hi = i < j ? j : i;
        if (lo == 0) return hi == 2 ? (2.0 / 3.0) : 1.0;
        if (lo == 1) return 4.0 / 3.0;
        return 8.0 / 3.0;
    }
}

// the Toeplitz coefficients of T(x): c[k] = x^k / k! (given x and x^2 / 2)
template <int B>
struct JCoef {
    double c[B];
    __device__ __forceinline__ JCoef(double x, double h) {
        c[0] = 1.0;
        if constexpr (B > 1) c[1] = x;
        if constexpr (B > 2) c[2] = h;
    }
};

// ------------------------------------------------------------------ e^-x (table-driven)
//
// e^-x for x >= 0 by the table-driven method of Tang (ACM TOMS 15, 1989):
// k = round(128 x / ln 2) = 128 m + j (0 <= j < 128), r = k ln2/128 - x
// (|r| <= ln2/256; ln2/128 is carried in two parts), and
//     e^-x = 2^-m 2^(-j/128) e^r,
// with e^r - 1 from its degree-5 Taylor polynomial (the truncation is below
// 6e-19 relative), 2^(-j/128) from a 128-entry table that the caller fills
// (exp_neg_table), and 2^-m applied to the exponent bits.  x > 708 gives 0
// (e^-x is then below the smallest normal double); NaN propagates.  Against
// a correctly rounded e^-x the error is about one unit in the last place.
static constexpr int EXPTAB = 128;

__device__ __forceinline__ void exp_neg_table(double* tbl, int tid, int nthreads) {
    for (int j = tid; j < EXPTAB; j += nthreads) tbl[j] = exp2(-(double)j / EXPTAB);
}

__device__ __forceinline__ double exp_neg(double x, const double* tbl) {
    constexpr double INV = 184.6649652337873;          // 128 / ln 2
    constexpr double L_HI = 0.0054152123481245725;     // ln 2 / 128, leading part
    constexpr double L_LO = 1.8117553233174215e-19;    // ln 2 / 128 - L_HI
    constexpr double MAGIC = 6755399441055744.0;       // 1.5 * 2^52: the sum rounds to an integer
    const double kb = fma(x, INV, MAGIC);
    const int k = __double2loint(kb);
    const double kd = kb - MAGIC;
    double r = fma(kd, L_HI, -x);
    r = fma(kd, L_LO, r);
    double q = fma(r, 1.0 / 120.0, 1.0 / 24.0);
    q = fma(r, q, 1.0 / 6.0);
    q = fma(r, q, 0.5);
    q = fma(r, q, 1.0);
    const double t = tbl[k & (EXPTAB - 1)];
    const double y = fma(t, r * q, t);
    const unsigned long long m = (unsigned long long)(long long)(k >> 7);
    const double s = __longlong_as_double((long long)((unsigned long long)__double_as_longlong(y) - (m << 52)));
    return x <= 708.0 ? s : (x > 708.0 ? 0.0 : x);
}

// X <- T X (X has NC columns; row r mixes rows k >= r, so rows go in increasing order)
template <int B, int NC>
__device__ __forceinline__ void jprop_unscaled(const JCoef<B>& t, double (&X)[B][NC]) {
#pragma unroll
    for (int r = 0; r < B; ++r)
#pragma unroll
        for (int q = 0; q < NC; ++q) {
            double s = X[r][q];
#pragma unroll
            for (int k = r + 1; k < B; ++k) s = fma(t.c[k - r], X[k][q], s);
            X[r][q] = s;
        }
}
template <int B>
__device__ __forceinline__ void jprop_vec(const JCoef<B>& t, double e, double (&v)[B]) {
#pragma unroll
    for (int r = 0; r < B; ++r) {
        double s = v[r];
#pragma unroll
        for (int k = r + 1; k < B; ++k) s = fma(t.c[k - r], v[k], s);
        v[r] = s * e;
    }
}
// v <- e T^T v (entry r mixes entries k <= r: decreasing order)
template <int B>
__device__ __forceinline__ void jprop_tvec(const JCoef<B>& t, double e, double (&v)[B]) {
#pragma unroll
    for (int r = B - 1; r >= 0; --r) {
        double s = v[r];
#pragma unroll
        for (int k = r - 1; k >= 0; --k) s = fma(t.c[r - k], v[k], s);
        v[r] = s * e;
    }
}

// Symmetric D <- e2 T D T^T (REV = false) or D <- e2 T^T D T (REV = true).
// T^T = R T R for the index reversal R (T is Toeplitz), so the second is the
// first on reversed indices.  Only the upper triangle of W = T D is needed:
// (W T^T)_ij, j >= i, reads W_il for l >= j.
template <int B, bool REV>
__device__ __forceinline__ void jsand(const JCoef<B>& t, double e2, double (&D)[B][B]) {
    double W[B][B];
#pragma unroll
    for (int i = 0; i < B; ++i)
#pragma unroll
        for (int j = i; j < B; ++j) {
            const int ii = REV ? B - 1 - i : i, jj = REV ? B - 1 - j : j;
            double s = D[ii][jj];
#pragma unroll
            for (int k = i + 1; k < B; ++k) s = fma(t.c[k - i], D[REV ? B - 1 - k : k][jj], s);
            W[i][j] = s;
        }
#pragma unroll
    for (int i = 0; i < B; ++i)
#pragma unroll
        for (int j = i; j < B; ++j) {
            double s = W[i][j];
#pragma unroll
            for (int l = j + 1; l < B; ++l) s = fma(t.c[l - j], W[i][l], s);
            const int ii = REV ? B - 1 - i : i, jj = REV ? B - 1 - j : j;
            D[ii][jj] = s * e2;
            D[jj][ii] = s * e2;
        }
}

// ------------------------------------------------------------------ classification on the bit pattern
// (integer instructions: the FP64 pipe is the chain kernels' bottleneck)

__device__ __forceinline__ unsigned long long dbits(double v) { return (unsigned long long)__double_as_longlong(v); }
// finite: the exponent field is not all ones
__device__ __forceinline__ bool is_finite_b(double v) {
    return (dbits(v) & 0x7ff0000000000000ULL) != 0x7ff0000000000000ULL;
}
__device__ __forceinline__ bool is_nan_b(double v) { return (dbits(v) & 0x7fffffffffffffffULL) > 0x7ff0000000000000ULL; }
// v < 0 (for non-NaN v; -0 is not below 0)
__device__ __forceinline__ bool is_negative_b(double v) { return dbits(v) > 0x8000000000000000ULL; }
// 0 < v < inf
__device__ __forceinline__ bool is_positive_finite_b(double v) { return dbits(v) - 1ULL < 0x7fefffffffffffffULL; }

// ------------------------------------------------------------------ small dense helpers (fully unrolled)

template <int B>
__device__ __forceinline__ void mat_mul(const double (&X)[B][B], const double (&Y)[B][B], double (&R)[B][B]) {
#pragma unroll
    for (int i = 0; i < B; ++i)
#pragma unroll
        for (int j = 0; j < B; ++j) {
            double s = X[i][0] * Y[0][j];
#pragma unroll
            for (int k = 1; k < B; ++k) s = fma(X[i][k], Y[k][j], s);
            R[i][j] = s;
        }
}
// R = X^T Y
template <int B>
__device__ __forceinline__ void mat_tmul(const double (&X)[B][B], const double (&Y)[B][B], double (&R)[B][B]) {
#pragma unroll
    for (int i = 0; i < B; ++i)
#pragma unroll
        for (int j = 0; j < B; ++j) {
            double s = X[0][i] * Y[0][j];
#pragma unroll
            for (int k = 1; k < B; ++k) s = fma(X[k][i], Y[k][j], s);
            R[i][j] = s;
        }
}
// symmetric R = X Y^T where the product is known to be symmetric: upper triangle, mirrored
template <int B>
__device__ __forceinline__ void mat_mul_t_sym(const double (&X)[B][B], const double (&Y)[B][B], double (&R)[B][B]) {
#pragma unroll
    for (int i = 0; i < B; ++i)
#pragma unroll
        for (int j = i; j < B; ++j) {
            double s = X[i][0] * Y[j][0];
#pragma unroll
            for (int k = 1; k < B; ++k) s = fma(X[i][k], Y[j][k], s);
            R[i][j] = s;
            R[j][i] = s;
        }
}
// symmetric R = X^T Y (X^T Y known symmetric)
template <int B>
__device__ __forceinline__ void mat_tmul_sym(const double (&X)[B][B], const double (&Y)[B][B], double (&R)[B][B]) {
#pragma unroll
    for (int i = 0; i < B; ++i)
#pragma unroll
        for (int j = i; j < B; ++j) {
            double s = X[0][i] * Y[0][j];
#pragma unroll
            for (int k = 1; k < B; ++k) s = fma(X[k][i], Y[k][j], s);
            R[i][j] = s;
            R[j][i] = s;
        }
}
template <int B>
__device__ __forceinline__ void mat_vec(const double (&X)[B][B], const double (&v)[B], double (&r)[B]) {
#pragma unroll
    for (int i = 0; i < B; ++i) {
        double s = X[i][0] * v[0];
#pragma unroll
        for (int k = 1; k < B; ++k) s = fma(X[i][k], v[k], s);
        r[i] = s;
    }
}
template <int B>
__device__ __forceinline__ void mat_tvec(const double (&X)[B][B], const double (&v)[B], double (&r)[B]) {
#pragma unroll
    for (int i = 0; i < B; ++i) {
        double s = X[0][i] * v[0];
#pragma unroll
        for (int k = 1; k < B; ++k) s = fma(X[k][i], v[k], s);
        r[i] = s;
    }
}
template <int B>
__device__ __forceinline__ void symmetrize(double (&X)[B][B]) {
#pragma unroll
    for (int i = 0; i < B; ++i)
#pragma unroll
        for (int j = i + 1; j < B; ++j) {
            const double s = 0.5 * (X[i][j] + X[j][i]);
            X[i][j] = s;
            X[j][i] = s;
        }
}

// Inverse by Gauss-Jordan elimination with partial pivoting.  Used only on
// matrices of the form I + (PSD)(PSD), whose eigenvalues are >= 1.
template <int B>
__device__ __forceinline__ void inv_pp(const double (&N)[B][B], double (&R)[B][B]) {
    double a[B][B];
#pragma unroll
    for (int i = 0; i < B; ++i)
#pragma unroll
        for (int j = 0; j < B; ++j) { a[i][j] = N[i][j]; R[i][j] = (i == j) ? 1.0 : 0.0; }
#pragma unroll
    for (int k = 0; k < B; ++k) {
        int p = k;
        double best = fabs(a[k][k]);
#pragma unroll
        for (int i = k + 1; i < B; ++i) {
            const double v = fabs(a[i][k]);
            if (v > best) { best = v; p = i; }
        }
#pragma unroll
        for (int i = k + 1; i < B; ++i) {
            if (p == i) {
#pragma unroll
                for (int j = 0; j < B; ++j) {
                    double u = a[k][j]; a[k][j] = a[i][j]; a[i][j] = u;
                    u = R[k][j]; R[k][j] = R[i][j]; R[i][j] = u;
                }
            }
        }
        const double inv = 1.0 / a[k][k];
#pragma unroll
        for (int j = 0; j < B; ++j) { a[k][j] *= inv; R[k][j] *= inv; }
#pragma unroll
        for (int i = 0; i < B; ++i) {
            if (i == k) continue;
            const double f = a[i][k];
#pragma unroll
            for (int j = 0; j < B; ++j) { a[i][j] = fma(-f, a[k][j], a[i][j]); R[i][j] = fma(-f, R[k][j], R[i][j]); }
        }
    }
}

// ------------------------------------------------------------------ packed storage

template <int B> struct Dims {
    static constexpr int NS = B * (B + 1) / 2;        // packed symmetric entries
    static constexpr int NE = B * B + 2 * B + 2 * NS; // element: A, bv, C, eta, J
    static constexpr int NM = B + NS;                 // a Gaussian state (m, P) or information (eta, J)
};

// packed upper-triangle index of (i, j), i <= j
template <int B>
__host__ __device__ constexpr int sidx(int i, int j) {
    return i <= j ? (i * B - (i * (i - 1)) / 2 + (j - i)) : (j * B - (j * (j - 1)) / 2 + (i - j));
}

template <int B>
struct Elem {
    double A[B][B];
    double bv[B];
    double C[B][B];
    double eta[B];
    double J[B][B];
};

template <int B>
__device__ __forceinline__ void elem_identity(Elem<B>& e) {
#pragma unroll
    for (int i = 0; i < B; ++i) {
        e.bv[i] = 0.0; e.eta[i] = 0.0;
#pragma unroll
        for (int j = 0; j < B; ++j) { e.A[i][j] = (i == j) ? 1.0 : 0.0; e.C[i][j] = 0.0; e.J[i][j] = 0.0; }
    }
}

// SoA layout: field f of item k at base[f * ld + k].
template <int B>
__device__ __forceinline__ void elem_store(double* __restrict__ base, int64_t ld, int64_t k, const Elem<B>& e) {
    int f = 0;
#pragma unroll
    for (int i = 0; i < B; ++i)
#pragma unroll
        for (int j = 0; j < B; ++j) base[(f++) * ld + k] = e.A[i][j];
#pragma unroll
    for (int i = 0; i < B; ++i) base[(f++) * ld + k] = e.bv[i];
#pragma unroll
    for (int i = 0; i < B; ++i)
#pragma unroll
        for (int j = i; j < B; ++j) base[(f++) * ld + k] = e.C[i][j];
#pragma unroll
    for (int i = 0; i < B; ++i) base[(f++) * ld + k] = e.eta[i];
#pragma unroll
    for (int i = 0; i < B; ++i)
#pragma unroll
        for (int j = i; j < B; ++j) base[(f++) * ld + k] = e.J[i][j];
}
template <int B>
__device__ __forceinline__ void elem_load(const double* __restrict__ base, int64_t ld, int64_t k, Elem<B>& e) {
    int f = 0;
#pragma unroll
    for (int i = 0; i < B; ++i)
#pragma unroll
        for (int j = 0; j < B; ++j) e.A[i][j] = base[(f++) * ld + k];
#pragma unroll
    for (int i = 0; i < B; ++i) e.bv[i] = base[(f++) * ld + k];
#pragma unroll
    for (int i = 0; i < B; ++i)
#pragma unroll
        for (int j = i; j < B; ++j) { const double v = base[(f++) * ld + k]; e.C[i][j] = v; e.C[j][i] = v; }
#pragma unroll
    for (int i = 0; i < B; ++i) e.eta[i] = base[(f++) * ld + k];
#pragma unroll
    for (int i = 0; i < B; ++i)
#pragma unroll
        for (int j = i; j < B; ++j) { const double v = base[(f++) * ld + k]; e.J[i][j] = v; e.J[j][i] = v; }
}

// a vector and a symmetric matrix: (m, P) states or (eta, J) information
template <int B>
__device__ __forceinline__ void vs_store(double* __restrict__ base, int64_t ld, int64_t k, const double (&v)[B],
                                         const double (&S)[B][B]) {
    int f = 0;
#pragma unroll
    for (int i = 0; i < B; ++i) base[(f++) * ld + k] = v[i];
#pragma unroll
    for (int i = 0; i < B; ++i)
#pragma unroll
        for (int j = i; j < B; ++j) base[(f++) * ld + k] = S[i][j];
}
template <int B>
__device__ __forceinline__ void vs_load(const double* __restrict__ base, int64_t ld, int64_t k, double (&v)[B],
                                        double (&S)[B][B]) {
    int f = 0;
#pragma unroll
    for (int i = 0; i < B; ++i) v[i] = base[(f++) * ld + k];
#pragma unroll
    for (int i = 0; i < B; ++i)
#pragma unroll
        for (int j = i; j < B; ++j) { const double x = base[(f++) * ld + k]; S[i][j] = x; S[j][i] = x; }
}

// ------------------------------------------------------------------ the combine (elimination of a shared node)

// (ei then ej): eliminate the state between the two chunks.
//   M = (I + C_i J_j)^-1
//   A = A_j M A_i,  bv = A_j M (bv_i + C_i eta_j) + bv_j,  C = A_j M C_i A_j^T + C_j
//   eta = A_i^T M^T (eta_j - J_j bv_i) + eta_i,  J = A_i^T M^T J_j A_i + J_i
template <int B>
__device__ __forceinline__ void combine(const Elem<B>& ei, const Elem<B>& ej, Elem<B>& r) {
    double N[B][B], M[B][B], T[B][B], U[B][B];
    mat_mul<B>(ei.C, ej.J, N);
#pragma unroll
    for (int i = 0; i < B; ++i) N[i][i] += 1.0;
    inv_pp<B>(N, M);
    // A
    mat_mul<B>(M, ei.A, T);
    mat_mul<B>(ej.A, T, r.A);
    // bv
    double w[B], z[B];
    mat_vec<B>(ei.C, ej.eta, w);
#pragma unroll
    for (int i = 0; i < B; ++i) w[i] += ei.bv[i];
    mat_vec<B>(M, w, z);
    mat_vec<B>(ej.A, z, w);
#pragma unroll
    for (int i = 0; i < B; ++i) r.bv[i] = w[i] + ej.bv[i];
    // C
    mat_mul<B>(M, ei.C, T);
    mat_mul<B>(ej.A, T, U);
    mat_mul_t_sym<B>(U, ej.A, T);
#pragma unroll
    for (int i = 0; i < B; ++i)
#pragma unroll
        for (int j = 0; j < B; ++j) r.C[i][j] = T[i][j] + ej.C[i][j];
    // eta
    mat_vec<B>(ej.J, ei.bv, w);
#pragma unroll
    for (int i = 0; i < B; ++i) w[i] = ej.eta[i] - w[i];
    mat_tvec<B>(M, w, z);
    mat_tvec<B>(ei.A, z, w);
#pragma unroll
    for (int i = 0; i < B; ++i) r.eta[i] = w[i] + ei.eta[i];
    // J
    mat_tmul<B>(M, ej.J, T);
    mat_mul<B>(T, ei.A, U);
    mat_tmul_sym<B>(ei.A, U, T);
#pragma unroll
    for (int i = 0; i < B; ++i)
#pragma unroll
        for (int j = 0; j < B; ++j) r.J[i][j] = T[i][j] + ei.J[i][j];
}

// A Gaussian state N(m, P) of the node before element e, pushed through e:
// the filtered state after e's chunk.  M = (I + P J_e)^-1,
// m' = A_e M (m + P eta_e) + bv_e,  P' = A_e M P A_e^T + C_e.
template <int B>
__device__ __forceinline__ void state_through(const double (&m)[B], const double (&P)[B][B], const Elem<B>& e,
                                              double (&mo)[B], double (&Po)[B][B]) {
    double N[B][B], M[B][B], T[B][B], U[B][B], w[B], z[B];
    mat_mul<B>(P, e.J, N);
#pragma unroll
    for (int i = 0; i < B; ++i) N[i][i] += 1.0;
    inv_pp<B>(N, M);
    mat_vec<B>(P, e.eta, w);
#pragma unroll
    for (int i = 0; i < B; ++i) w[i] += m[i];
    mat_vec<B>(M, w, z);
    mat_vec<B>(e.A, z, w);
#pragma unroll
    for (int i = 0; i < B; ++i) mo[i] = w[i] + e.bv[i];
    mat_mul<B>(M, P, T);
    mat_mul<B>(e.A, T, U);
    mat_mul_t_sym<B>(U, e.A, T);
#pragma unroll
    for (int i = 0; i < B; ++i)
#pragma unroll
        for (int j = 0; j < B; ++j) Po[i][j] = T[i][j] + e.C[i][j];
}

// Information (eta, J) about the node after element e, pulled back through e
// and joined with e's own information: the information about the node before e.
// M = (I + C_e J)^-1, eta' = A_e^T M^T (eta - J bv_e) + eta_e, J' = A_e^T M^T J A_e + J_e.
template <int B>
__device__ __forceinline__ void info_through(const Elem<B>& e, const double (&eta)[B], const double (&J)[B][B],
                                             double (&eo)[B], double (&Jo)[B][B]) {
    double N[B][B], M[B][B], T[B][B], U[B][B], w[B], z[B];
    mat_mul<B>(e.C, J, N);
#pragma unroll
    for (int i = 0; i < B; ++i) N[i][i] += 1.0;
    inv_pp<B>(N, M);
    mat_vec<B>(J, e.bv, w);
#pragma unroll
    for (int i = 0; i < B; ++i) w[i] = eta[i] - w[i];
    mat_tvec<B>(M, w, z);
    mat_tvec<B>(e.A, z, w);
#pragma unroll
    for (int i = 0; i < B; ++i) eo[i] = w[i] + e.eta[i];
    mat_tmul<B>(M, J, T);
    mat_mul<B>(T, e.A, U);
    mat_tmul_sym<B>(e.A, U, T);
#pragma unroll
    for (int i = 0; i < B; ++i)
#pragma unroll
        for (int j = 0; j < B; ++j) Jo[i][j] = T[i][j] + e.J[i][j];
}

}  // namespace spg
