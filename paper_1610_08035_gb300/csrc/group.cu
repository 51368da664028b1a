// group.cu -- the hot path for structured state spaces built from 2x2 blocks:
// sums of Matern-3/2, periodic (order J), quasi-periodic (order J with a
// Matern-1/2 envelope) and exponentiated-quadratic (even order N, a cascade
// of second-order sections) components, state dimension b = 2K <= 16
// (Sec. 2.1; the quasi-periodic family is Eq. co2_1's periodicity term, the
// EQ approximation the one of the paper's experiments).
//
// Structure exploited: the transition A_n is made of 2x2 blocks.  Its
// diagonal blocks are a Matern-3/2 block in scaled coordinates, a rotation by
// j w dt damped by the envelope, or an EQ section's damped rotation
// exp(a x) R(b x), x = dt / l; an EQ component (its sections first in the
// state) adds the coupling blocks of its sections below the diagonal, so that
// part of A_n is block lower triangular.  H picks the first coordinate of
// every block.  Pinf is diagonal except on the EQ sections, where it has
// dense 2x2 blocks s P_k; each CTA keeps the whole Pinf in shared memory.
// The posterior covariance is dense, so the Kalman and adjoint recursions run
// on a group of 16 lanes per chunk: lane c owns column c of every b x b
// matrix.  Left products with A_n are then local to a lane; without an EQ
// coupling a right product needs only the partner column of the same block
// (one shuffle per entry), and with one a sandwich A X A^T of a symmetric X
// is two left products around a transpose through shared memory.  H^T-column
// sums of a symmetric matrix are local as well.
//
// Kernels, in order:
//   k_gsetup     per-block constants from theta (Pinf weights, rates)
//   k_gdisc      one thread per step: the transition's blocks (stored)
//   k_gfold      one group per chunk: sequential elimination into an element
//   k_gscan_up / k_gscan_down   odd-even reduction of chunk elements, level by
//                level, with group-cooperative combines (global memory)
//   k_gchunk     one group per chunk: forward recursion, reverse sweep,
//                posterior and gradient terms
//   k_gfinal     fixed-order reduction and chain rule
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include "chain.cuh"
#include "internal.h"
#include "spingp.h"

namespace spg {

static constexpr int GL = 16;               // lanes per group = largest state dimension
static constexpr int GK = GL / 2;           // largest number of 2x2 blocks
static constexpr int GCTA = 128;            // threads per block: 8 groups
static constexpr int GGRP = GCTA / GL;
static constexpr int GNE = 3 * GL + 2;      // per-lane values of an element: A, C, J columns, bv, eta
static constexpr int GNM = GL + 1;          // per-lane values of a state / information: column + vector entry
static constexpr int GNC = 3;               // per-block constants: Pinf weight, d weight/dvar, d weight/dlen
static constexpr double G_LOG_2PI = 1.8378770664093454836;
static constexpr double G_LN2 = 0.69314718055994530942;

// block kinds
enum { GB_MATERN32 = 0, GB_PERIODIC = 1, GB_QUASI = 2, GB_EQ = 3 };

// per-chunk partial sums: ll, noise, per component (rate, envelope rate), then
// the diagonal of the Pinf adjoint for every state (lane), then the adjoint
// contracted with an EQ component's P_m (its variance derivative)
static constexpr int GPART = 2 + 2 * GMAXCOMP + GL + 1;
static constexpr int GP_EQ = 2 + 2 * GMAXCOMP + GL;

// Pinf (b x b, row-major, zero-padded to GL x GL) and, for an EQ component,
// dPinf / d(its variance) = P_m on its block: built by each CTA in shared
// memory from the per-block weights and the model constants.
__device__ __forceinline__ void g_pinf_smem(const GModel& gm, const double* __restrict__ theta,
                                            const double* __restrict__ gconst, double* s_pinf, double* s_dpe) {
    const double veq = (gm.eq_nk > 0) ? theta[gm.cpoff[gm.eq_comp] + 1] : 0.0;
    const int o = 2 * gm.eq_k0, ne = 2 * gm.eq_nk;
    for (int idx = threadIdx.x; idx < GL * GL; idx += blockDim.x) {
        const int r = idx / GL, c = idx % GL;
        double v = (r == c && r < gm.b) ? gconst[(r >> 1) * GNC] : 0.0;
        double d = 0.0;
        if (r >= o && r < o + ne && c >= o && c < o + ne) {
            d = gm.eqP[(r - o) * 16 + (c - o)];
            v += veq * d;
        }
        s_pinf[idx] = v;
        s_dpe[idx] = d;
    }
}

__device__ __forceinline__ unsigned half_mask() { return (threadIdx.x & 16) ? 0xffff0000u : 0x0000ffffu; }

__device__ __forceinline__ double gshfl(double v, int src) { return __shfl_sync(half_mask(), v, src, GL); }
__device__ __forceinline__ double gxor(double v, int m) { return __shfl_xor_sync(half_mask(), v, m, GL); }

// fixed-order sum over the 16 lanes of a group (same result in every lane)
__device__ __forceinline__ double gsum(double v) {
#pragma unroll
    for (int m = 8; m > 0; m >>= 1) v += gxor(v, m);
    return v;
}

// all 16 entries of a lane-distributed vector
template <int NR>
__device__ __forceinline__ void ggather(double mine, double (&v)[GL]) {
#pragma unroll
    for (int r = 0; r < NR; ++r) v[r] = gshfl(mine, r);
}

// ------------------------------------------------------------------ setup: per-block constants

// Pinf of block k is w_k I2 with w_k = variance (Matern) or variance * c_j e^-x I_j(x),
// x = 1/lp^2 (periodic, quasi-periodic); also dw/dvariance and dw/dlp.
__device__ double g_bessel_i(int j, double x) {
    const double h = 0.5 * x;
    double term = 1.0;
    for (int i = 1; i <= j; ++i) term *= h / i;
    double s = term;
    for (int k = 1; k < 500; ++k) {
        term *= h * h / ((double)k * (double)(k + j));
        s += term;
        if (term < 1e-18 * s) break;
    }
    return s;
}

__global__ void k_gsetup(GModel gm, const double* __restrict__ theta, double* __restrict__ gconst, int* status) {
    const int k = threadIdx.x;
    if (k == 0) {
        for (int p = 0; p < gm.P; ++p)
            if (!(theta[p] > 0.0) || !isfinite(theta[p])) atomicOr(status, ST_EINVAL);
    }
    if (k >= gm.K) return;
    const int c = gm.bcomp[k];
    const double* th = theta + gm.cpoff[c];
    double w = 0.0, dwv = 0.0, dwl = 0.0;
    if (gm.bkind[k] == GB_MATERN32) {
        w = th[1]; dwv = 1.0; dwl = 0.0;
    } else if (gm.bkind[k] == GB_EQ) {
        w = 0.0; dwv = 0.0; dwl = 0.0;   // 2 x 2 blocks of the EQ sections' Pinf: g_pinf_smem
    } else {
        const int j = gm.bj[k];
        const double var = th[0], lp = th[1];
        const double x = 1.0 / (lp * lp), ex = exp(-x), cj = (j == 0) ? 1.0 : 2.0;
        const double Ij = g_bessel_i(j, x);
        const double dIj = 0.5 * (g_bessel_i(j == 0 ? 1 : j - 1, x) + g_bessel_i(j + 1, x));
        const double u = cj * ex * Ij;
        w = var * u;
        dwv = u;
        dwl = var * cj * ex * (dIj - Ij) * (-2.0 / (lp * lp * lp));
    }
    gconst[k * GNC + 0] = w;
    gconst[k * GNC + 1] = dwv;
    gconst[k * GNC + 2] = dwl;
}

// ------------------------------------------------------------------ discretisation: Phi_n per block

// Phi for step i (transition from t_{i-1}): 4 entries per block, row-major.
// (t_prev: the time before step 0 when the steps continue a split series, s0 = -1)
// The EQ component's blocks of the transition F = expm(T x): its diagonal
// blocks at ph[4 k ..], and the coupling blocks (k, i) for sections k > i at
// ph[4 GK + 4 (k (k - 1) / 2 + i) ..], row-major.  T has the diagonal blocks T_k = a_k I + b_k J, J = [[0, 1],
// [-1, 0]], and below them T_ki = -u_k w_i^T.  F commutes with T, and with
// E = F - I block (k, i) of T F = F T reads
//   T_k E_ki - E_ki T_i = E_kk T_ki - T_ki E_ii + sum_{i<j<k} (E_kj T_ji - T_kj E_ji)
//                       = -p w_i^T + u_k q^T,
//   p = sum_{j=i+1..k} E_kj u_j,   q = sum_{j=i..k-1} E_ji^T w_j,
// Parlett's recurrence for a function of a block triangular matrix, taken in
// E so that the identity terms cancel exactly and a small x loses no digits.
// X -> T_k X - X T_i acts on the part of X that commutes with J,
// (X - J X J) / 2, as left multiplication by (a_k - a_i) + (b_k - b_i) J, and
// on the part that anticommutes, (X + J X J) / 2, as (a_k - a_i) + (b_k + b_i) J:
// each part is solved by one complex division (reciprocal moduli from the
// model).  Row k runs i = k-1 down to 0, so p accumulates along the row and q
// per column.
__device__ void g_eq_blocks(const GModel& gm, double x, double* __restrict__ ph) {
    const int nk = gm.eq_nk;
    double* __restrict__ out = ph + 4 * GK;
    double c0[GK], c1[GK], q0[GK], q1[GK];
#pragma unroll
    for (int k = 0; k < GK; ++k) {
        c0[k] = 0.0; c1[k] = 0.0; q0[k] = 0.0; q1[k] = 0.0;
        if (k < nk) {
            // with s, c = sin, cos(b x / 2): e^(a x) cos(b x) - 1 = expm1(a x)(1 - 2 s^2) - 2 s^2
            // and e^(a x) sin(b x) = e^(a x) 2 s c, free of cancellation for small x
            double sh, ch;
            sincos(0.5 * gm.eqb[k] * x, &sh, &ch);
            const double em = expm1(gm.eqa[k] * x), s2 = 2.0 * sh * sh;
            c0[k] = fma(em, 1.0 - s2, -s2);
            c1[k] = (1.0 + em) * (2.0 * sh * ch);
            // the diagonal block e^(a x) [[cos bx, sin bx], [-sin bx, cos bx]] = I + E_kk
            ph[4 * k + 0] = 1.0 + c0[k]; ph[4 * k + 1] = c1[k];
            ph[4 * k + 2] = -c1[k];      ph[4 * k + 3] = 1.0 + c0[k];
            // q_k starts at E_kk^T w_k, E_kk = [[c0, c1], [-c1, c0]]
            const double w0 = gm.eqw[2 * k], w1 = gm.eqw[2 * k + 1];
            q0[k] = fma(c0[k], w0, -c1[k] * w1);
            q1[k] = fma(c1[k], w0, c0[k] * w1);
        }
    }
#pragma unroll
    for (int k = 1; k < GK; ++k) {
        if (k >= nk) break;
        const double uk0 = gm.equ[2 * k], uk1 = gm.equ[2 * k + 1], wk0 = gm.eqw[2 * k], wk1 = gm.eqw[2 * k + 1];
        double p0 = fma(c0[k], uk0, c1[k] * uk1), p1 = fma(-c1[k], uk0, c0[k] * uk1);   // E_kk u_k
#pragma unroll
        for (int i = k - 1; i >= 0; --i) {
            const int ci = k * (k - 1) / 2 + i;
            const double wi0 = gm.eqw[2 * i], wi1 = gm.eqw[2 * i + 1];
            const double r00 = fma(-p0, wi0, uk0 * q0[i]), r01 = fma(-p0, wi1, uk0 * q1[i]);
            const double r10 = fma(-p1, wi0, uk1 * q0[i]), r11 = fma(-p1, wi1, uk1 * q1[i]);
            const double pc = 0.5 * (r00 + r11), qc = 0.5 * (r01 - r10);   // commuting part [[pc, qc], [-qc, pc]]
            const double ra = 0.5 * (r00 - r11), sa = 0.5 * (r01 + r10);   // anticommuting part [[ra, sa], [sa, -ra]]
            const double al = gm.eqa[k] - gm.eqa[i], bc = gm.eqb[k] - gm.eqb[i], ba = gm.eqb[k] + gm.eqb[i];
            const double Pc = fma(al, pc, bc * qc) * gm.eqrc[ci], Qc = fma(al, qc, -bc * pc) * gm.eqrc[ci];
            const double Ra = fma(al, ra, -ba * sa) * gm.eqra[ci], Sa = fma(al, sa, ba * ra) * gm.eqra[ci];
            const double x00 = Pc + Ra, x01 = Qc + Sa, x10 = Sa - Qc, x11 = Pc - Ra;
            double* o = out + 4 * ci;
            o[0] = x00; o[1] = x01; o[2] = x10; o[3] = x11;
            const double ui0 = gm.equ[2 * i], ui1 = gm.equ[2 * i + 1];
            p0 = fma(x00, ui0, fma(x01, ui1, p0));
            p1 = fma(x10, ui0, fma(x11, ui1, p1));
            q0[i] = fma(x00, wk0, fma(x10, wk1, q0[i]));   // += X^T w_k
            q1[i] = fma(x01, wk0, fma(x11, wk1, q1[i]));
        }
    }
}

__global__ void __launch_bounds__(256) k_gdisc(GModel gm, const double* __restrict__ t, const double* __restrict__ y,
                                                int64_t n, const double* __restrict__ theta,
                                                double* __restrict__ phis, int* status, int missing, int64_t s0,
                                                double t_prev) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    int bad = 0;
    if (!isfinite(t[i]) || (!isfinite(y[i]) && !(missing && isnan(y[i])))) bad |= ST_ENONFINITE;
    const double dt = (i > 0) ? t[i] - t[i - 1] : (s0 < 0 ? t[0] - t_prev : 0.0);
    if (dt < 0.0) bad |= ST_ENOTSORTED;
    double* ph = phis + i * gm.phs;
    // per component, once: the rotation by w dt and the envelope of a
    // (quasi-)periodic component, whose harmonic j + 1 follows from harmonic
    // j by angle addition (its blocks come in order j = 0, 1, .., J); the EQ
    // sections are written by g_eq_blocks
    int pc = -1, pj = -1;
    double wdt = 0.0, c1 = 1.0, s1 = 0.0, cj = 1.0, sj = 0.0, env = 1.0;
#pragma unroll 1
    for (int k = 0; k < GK; ++k) {
        double p00 = 0.0, p01 = 0.0, p10 = 0.0, p11 = 0.0;
        if (k < gm.K) {
            const int comp = gm.bcomp[k];
            const double* th = theta + gm.cpoff[comp];
            if (gm.bkind[k] == GB_MATERN32) {
                const double lam = sqrt(3.0) / th[0];
                double P[2][2];
                phi<2>(lam * dt, exp(-lam * dt), P);
                p00 = P[0][0]; p01 = P[0][1]; p10 = P[1][0]; p11 = P[1][1];
            } else if (gm.bkind[k] == GB_EQ) {
                pc = comp;
                continue;                 // g_eq_blocks below
            } else {
                const int j = gm.bj[k];
                if (comp != pc) {
                    wdt = (2.0 * M_PI / th[2]) * dt;
                    sincos(wdt, &s1, &c1);
                    env = (gm.bkind[k] == GB_QUASI) ? exp(-dt / th[3]) : 1.0;
                    pj = -1;
                }
                if (j == 0) {
                    cj = 1.0; sj = 0.0;
                } else if (j == 1) {
                    cj = c1; sj = s1;
                } else if (j == pj + 1) {   // cos, sin of (j - 1 + 1) w dt
                    const double cn = fma(cj, c1, -sj * s1);
                    sj = fma(sj, c1, cj * s1);
                    cj = cn;
                } else {
                    sincos(j * wdt, &sj, &cj);
                }
                pj = j;
                p00 = env * cj; p01 = -env * sj; p10 = env * sj; p11 = env * cj;
            }
            pc = comp;
        }
        ph[4 * k + 0] = p00; ph[4 * k + 1] = p01; ph[4 * k + 2] = p10; ph[4 * k + 3] = p11;
    }
    if (gm.eq_nk > 0) g_eq_blocks(gm, dt / theta[gm.cpoff[gm.eq_comp]], ph);
    if (bad) atomicOr(status, bad);
}

// ------------------------------------------------------------------ group linear algebra on columns

// X <- blockdiag(Phi) X  (column-local: rows 2k, 2k+1 mix)
template <int NR>
__device__ __forceinline__ void g_left(const double* __restrict__ ph, double (&X)[GL]) {
#pragma unroll
    for (int k = 0; k < NR / 2; ++k) {
        const double a = ph[4 * k], b = ph[4 * k + 1], c = ph[4 * k + 2], d = ph[4 * k + 3];
        const double x0 = X[2 * k], x1 = X[2 * k + 1];
        X[2 * k] = fma(a, x0, b * x1);
        X[2 * k + 1] = fma(c, x0, d * x1);
    }
}
// X <- blockdiag(Phi)^T X
template <int NR>
__device__ __forceinline__ void g_left_t(const double* __restrict__ ph, double (&X)[GL]) {
#pragma unroll
    for (int k = 0; k < NR / 2; ++k) {
        const double a = ph[4 * k], b = ph[4 * k + 1], c = ph[4 * k + 2], d = ph[4 * k + 3];
        const double x0 = X[2 * k], x1 = X[2 * k + 1];
        X[2 * k] = fma(a, x0, c * x1);
        X[2 * k + 1] = fma(b, x0, d * x1);
    }
}
// column c of X Phi^T (right product: the partner column of c's block)
template <int NR>
__device__ __forceinline__ void g_right_t(const double* __restrict__ ph, int lane, double (&X)[GL]) {
    const int k = lane >> 1, odd = lane & 1;
    // row 'odd' of Phi_k: (Phi X^T)... column c of X Phi^T = sum_q X[:, 2k+q] Phi_k[odd][q]
    const double f0 = ph[4 * k + 2 * odd], f1 = ph[4 * k + 2 * odd + 1];
#pragma unroll
    for (int r = 0; r < NR; ++r) {
        const double p = gxor(X[r], 1);
        const double x0 = odd ? p : X[r], x1 = odd ? X[r] : p;
        X[r] = fma(f0, x0, f1 * x1);
    }
}
// column c of X Phi: sum_q X[:, 2k+q] Phi_k[q][odd]
template <int NR>
__device__ __forceinline__ void g_right(const double* __restrict__ ph, int lane, double (&X)[GL]) {
    const int k = lane >> 1, odd = lane & 1;
    const double f0 = ph[4 * k + odd], f1 = ph[4 * k + 2 + odd];
#pragma unroll
    for (int r = 0; r < NR; ++r) {
        const double p = gxor(X[r], 1);
        const double x0 = odd ? p : X[r], x1 = odd ? X[r] : p;
        X[r] = fma(f0, x0, f1 * x1);
    }
}
// entry c of blockdiag(Phi) v for a lane-distributed vector
__device__ __forceinline__ double g_vleft(const double* __restrict__ ph, int lane, double v) {
    const int k = lane >> 1, odd = lane & 1;
    const double p = gxor(v, 1);
    const double v0 = odd ? p : v, v1 = odd ? v : p;
    return fma(ph[4 * k + 2 * odd], v0, ph[4 * k + 2 * odd + 1] * v1);
}
// entry c of blockdiag(Phi)^T v
__device__ __forceinline__ double g_vleft_t(const double* __restrict__ ph, int lane, double v) {
    const int k = lane >> 1, odd = lane & 1;
    const double p = gxor(v, 1);
    const double v0 = odd ? p : v, v1 = odd ? v : p;
    return fma(ph[4 * k + odd], v0, ph[4 * k + 2 + odd] * v1);
}
// h^T x for a column: sum of the even entries
template <int NR>
__device__ __forceinline__ double g_hsum(const double (&X)[GL]) {
    double s = 0.0;
#pragma unroll
    for (int k = 0; k < NR / 2; ++k) s += X[2 * k];
    return s;
}

// ------------------------------------------------------------------ the transition with EQ coupling blocks

// coupling block (k, i), k > i, of a step's transition (after the GK diagonal blocks)
__device__ __forceinline__ const double* g_cpl(const double* __restrict__ ph, int k, int i) {
    return ph + 4 * GK + 4 * (k * (k - 1) / 2 + i);
}
// X <- A X for a column: the diagonal blocks, plus sum_{i<k} A_ki X_i on the
// rows of EQ section k (nk sections, the first blocks of the state); the
// blocks run from the last down, so the rows a block reads are still the
// input's, and the coupling terms accumulate into the diagonal block's sums
template <int NR>
__device__ __forceinline__ void g_left_c(const double* __restrict__ ph, int nk, double (&X)[GL]) {
#pragma unroll
    for (int k = NR / 2 - 1; k >= 0; --k) {
        const double a = ph[4 * k], b = ph[4 * k + 1], c = ph[4 * k + 2], d = ph[4 * k + 3];
        const double x0 = X[2 * k], x1 = X[2 * k + 1];
        double s0 = b * x1, s1 = d * x1;
        if (k > 0 && k < nk) {
#pragma unroll
            for (int i = 0; i < k; ++i) {
                const double* o = g_cpl(ph, k, i);
                s0 = fma(o[0], X[2 * i], fma(o[1], X[2 * i + 1], s0));
                s1 = fma(o[2], X[2 * i], fma(o[3], X[2 * i + 1], s1));
            }
        }
        X[2 * k] = fma(a, x0, s0);
        X[2 * k + 1] = fma(c, x0, s1);
    }
}
// X <- A^T X for a column: sum_{k>i} A_ki^T X_k on the rows of section i
// (the blocks run from the first up, for the same reason)
template <int NR>
__device__ __forceinline__ void g_left_t_c(const double* __restrict__ ph, int nk, double (&X)[GL]) {
#pragma unroll
    for (int i = 0; i < NR / 2; ++i) {
        const double a = ph[4 * i], b = ph[4 * i + 1], c = ph[4 * i + 2], d = ph[4 * i + 3];
        const double x0 = X[2 * i], x1 = X[2 * i + 1];
        double s0 = c * x1, s1 = d * x1;
#pragma unroll
        for (int k = i + 1; k < NR / 2; ++k) {
            if (k < nk) {
                const double* o = g_cpl(ph, k, i);
                s0 = fma(o[0], X[2 * k], fma(o[2], X[2 * k + 1], s0));
                s1 = fma(o[1], X[2 * k], fma(o[3], X[2 * k + 1], s1));
            }
        }
        X[2 * i] = fma(a, x0, s0);
        X[2 * i + 1] = fma(b, x0, s1);
    }
}
// X <- its row 'lane', given its column 'lane' in every lane of the group:
// a transpose through the group's shared scratch tb (rows of stride GL + 1,
// so neither the column writes nor the row reads meet a bank conflict)
template <int NR>
__device__ __forceinline__ void g_transpose(double* __restrict__ tb, int lane, double (&X)[GL]) {
    const unsigned mask = half_mask();
#pragma unroll
    for (int r = 0; r < NR; ++r) tb[r * (GL + 1) + lane] = X[r];
    __syncwarp(mask);
#pragma unroll
    for (int j = 0; j < NR; ++j) X[j] = (lane < NR) ? tb[lane * (GL + 1) + j] : 0.0;
    __syncwarp(mask);
}
// X <- A X A^T for a symmetric X by columns: with Y = A X, column 'lane' of
// A Y^T is A times row 'lane' of Y
template <int NR>
__device__ __forceinline__ void g_sandwich_c(const double* __restrict__ ph, int nk, double* tb, int lane,
                                             double (&X)[GL]) {
    g_left_c<NR>(ph, nk, X);
    g_transpose<NR>(tb, lane, X);
    g_left_c<NR>(ph, nk, X);
}
// X <- A^T X A for a symmetric X by columns
template <int NR>
__device__ __forceinline__ void g_sandwich_t_c(const double* __restrict__ ph, int nk, double* tb, int lane,
                                               double (&X)[GL]) {
    g_left_t_c<NR>(ph, nk, X);
    g_transpose<NR>(tb, lane, X);
    g_left_t_c<NR>(ph, nk, X);
}
// entry 'lane' of A v for a lane-distributed vector v: the diagonal block
// through the partner lane, and for a lane of EQ section k the couplings
// A_ki, i < k, from the gathered entries of the sections before it
template <int NR>
__device__ __forceinline__ double g_vleft_c(const double* __restrict__ ph, int nk, int lane, double v) {
    double r = g_vleft(ph, lane, v);
    double vv[GL];
#pragma unroll
    for (int q = 0; q < NR; ++q)
        if (q < 2 * (nk - 1)) vv[q] = gshfl(v, q);    // uniform over the group
    const int k = lane >> 1, odd = lane & 1;
#pragma unroll
    for (int i = 0; i < NR / 2 - 1; ++i) {
        if (i < k && k < nk) {
            const double* o = g_cpl(ph, k, i) + 2 * odd;
            r = fma(o[0], vv[2 * i], fma(o[1], vv[2 * i + 1], r));
        }
    }
    return r;
}
// entry 'lane' of A^T v: for a lane of section i, the couplings A_ki^T, k > i
template <int NR>
__device__ __forceinline__ double g_vleft_t_c(const double* __restrict__ ph, int nk, int lane, double v) {
    double r = g_vleft_t(ph, lane, v);
    double vv[GL];
#pragma unroll
    for (int q = 2; q < NR; ++q)
        if (q < 2 * nk) vv[q] = gshfl(v, q);
    const int i = lane >> 1, odd = lane & 1;
#pragma unroll
    for (int k = 1; k < NR / 2; ++k) {
        if (k > i && k < nk) {
            const double* o = g_cpl(ph, k, i) + odd;
            r = fma(o[0], vv[2 * k], fma(o[2], vv[2 * k + 1], r));
        }
    }
    return r;
}

// ------------------------------------------------------------------ elements in global memory

struct GElem {
    double A[GL], C[GL], J[GL];   // column 'lane'
    double bv, eta;               // entry 'lane'
};

// element e's value f of lane l at base[(f * ne + e) * GL + l]
template <int NR>
__device__ __forceinline__ void gelem_store(double* __restrict__ base, int64_t ne, int64_t e, int lane,
                                            const GElem& x) {
    double* p = base + e * GL + lane;
    const int64_t s = ne * GL;
#pragma unroll
    for (int r = 0; r < GL; ++r) {
        const bool in = r < NR;   // rows past the state are zero
        p[r * s] = in ? x.A[r] : 0.0; p[(GL + r) * s] = in ? x.C[r] : 0.0; p[(2 * GL + r) * s] = in ? x.J[r] : 0.0;
    }
    p[3 * GL * s] = x.bv;
    p[(3 * GL + 1) * s] = x.eta;
}
// a state (m, P) or information (eta, J): column + entry
template <int NR>
__device__ __forceinline__ void gvs_load(const double* __restrict__ base, int64_t ne, int64_t e, int lane,
                                         double (&S)[GL], double& v) {
    const double* p = base + e * GL + lane;
    const int64_t s = ne * GL;
#pragma unroll
    for (int r = 0; r < GL; ++r) S[r] = (r < NR) ? p[r * s] : 0.0;
    v = p[GL * s];
}

// ------------------------------------------------------------------ group matrix products through shared memory

// Per-group shared scratch: one b x b matrix stored by columns (col c at sm[c*GL])
// and inverse workspace.
struct GSmem {
    double X[GL * (GL + 1)];   // also the transpose scratch of g_transpose
    double N[GL * GL];
    double R[GL * GL];
};

template <int NR>
__device__ __forceinline__ void g_put(double* __restrict__ sm, int lane, const double (&col)[GL]) {
#pragma unroll
    for (int r = 0; r < NR; ++r) sm[lane * GL + r] = col[r];
}
// out = M y where M's columns are in sm (column-major) and y is this lane's column
template <int NR>
__device__ __forceinline__ void g_mul(const double* __restrict__ sm, const double (&y)[GL], double (&out)[GL]) {
#pragma unroll
    for (int r = 0; r < NR; ++r) out[r] = 0.0;
#pragma unroll
    for (int k = 0; k < NR; ++k) {
        const double yk = y[k];
#pragma unroll
        for (int r = 0; r < NR; ++r) out[r] = fma(sm[k * GL + r], yk, out[r]);
    }
}
// row 'lane' of M (columns in sm) dotted with a full vector
template <int NR>
__device__ __forceinline__ double g_rowdot(const double* __restrict__ sm, int lane, const double (&v)[GL]) {
    double s = 0.0;
#pragma unroll
    for (int k = 0; k < NR; ++k) s = fma(sm[k * GL + lane], v[k], s);
    return s;
}

// M = (I + X Y)^-1 with X (symmetric) given by this lane's column Xc, Y by its
// column Yc; result: this lane's column of M in Mc.  Gauss-Jordan with partial
// pivoting on the group (columns in shared memory).  I + X Y has eigenvalues >= 1.
template <int NR>
__device__ void g_inv_ixy(GSmem& s, int lane, const double (&Xc)[GL], const double (&Yc)[GL], double (&Mc)[GL]) {
    const unsigned mask = half_mask();
    g_put<NR>(s.X, lane, Xc);
    __syncwarp(mask);
    double col[GL];
    g_mul<NR>(s.X, Yc, col);            // column 'lane' of X Y
#pragma unroll
    for (int r = 0; r < NR; ++r)
        if (r == lane) col[r] += 1.0;
    __syncwarp(mask);
    g_put<NR>(s.N, lane, col);
#pragma unroll
    for (int r = 0; r < NR; ++r) s.R[lane * GL + r] = (r == lane) ? 1.0 : 0.0;
    __syncwarp(mask);
#pragma unroll 1
    for (int k = 0; k < NR; ++k) {
        // pivot row: largest |N[r][k]| for r >= k (every lane computes the same)
        int p = k;
        double best = fabs(s.N[k * GL + k]);
        for (int r = k + 1; r < NR; ++r) {
            const double v = fabs(s.N[k * GL + r]);
            if (v > best) { best = v; p = r; }
        }
        __syncwarp(mask);
        if (p != k) {
            double u = s.N[lane * GL + k]; s.N[lane * GL + k] = s.N[lane * GL + p]; s.N[lane * GL + p] = u;
            u = s.R[lane * GL + k]; s.R[lane * GL + k] = s.R[lane * GL + p]; s.R[lane * GL + p] = u;
        }
        __syncwarp(mask);
        const double piv = s.N[k * GL + k];
        const double inv = 1.0 / piv;
        double nk = s.N[lane * GL + k] * inv, rk = s.R[lane * GL + k] * inv;
        double colk[GL];
#pragma unroll
        for (int r = 0; r < NR; ++r) colk[r] = s.N[k * GL + r];
        __syncwarp(mask);
#pragma unroll
        for (int r = 0; r < NR; ++r) {
            if (r == k) continue;
            s.N[lane * GL + r] = fma(-colk[r], nk, s.N[lane * GL + r]);
            s.R[lane * GL + r] = fma(-colk[r], rk, s.R[lane * GL + r]);
        }
        s.N[lane * GL + k] = nk;
        s.R[lane * GL + k] = rk;
        __syncwarp(mask);
    }
#pragma unroll
    for (int r = 0; r < NR; ++r) Mc[r] = s.R[lane * GL + r];
    __syncwarp(mask);
}

// symmetrise a column-distributed matrix: X <- (X + X^T)/2
template <int NR>
__device__ __forceinline__ void g_sym(GSmem& s, int lane, double (&Xc)[GL]) {
    const unsigned mask = half_mask();
    g_put<NR>(s.X, lane, Xc);
    __syncwarp(mask);
#pragma unroll
    for (int q = 0; q < NR; ++q) Xc[q] = 0.5 * (Xc[q] + s.X[q * GL + lane]);
    __syncwarp(mask);
}

// ------------------------------------------------------------------ k_gfold: in-chunk elimination

struct GArgs {
    GModel gm;
    const double* t;
    const double* y;
    int64_t n, L, nc;
    const double* theta;
    const double* gconst;
    const double* phis;
    int* status;
    int missing;          // 1: a NaN observation is missing (a test point)
    int64_t s0;           // the series' first step: 0, or -1 when the steps continue a split series
    double t_prev;        // with s0 = -1: the time of the step before step 0
    double* lag1 = nullptr;   // posterior: n - 1 entries Cov(f_{i+1}, f_i | y), or NULL
};

// EQT: the model has an EQ component of two or more sections (coupling
// blocks in the transition)
template <int NR, bool EQT>
__global__ void __launch_bounds__(GCTA) k_gfold(GArgs a, double* __restrict__ nodes) {
    __shared__ double s_pinf[GL * GL], s_dpe[GL * GL];
    __shared__ double s_tb[EQT ? GGRP * GL * (GL + 1) : 1];
    g_pinf_smem(a.gm, a.theta, a.gconst, s_pinf, s_dpe);
    __syncthreads();
    const int lane = threadIdx.x & (GL - 1);
    const int64_t c = blockIdx.x * (int64_t)GGRP + (threadIdx.x >> 4);
    if (c >= a.nc) return;   // the whole group leaves together
    const int phs = EQT ? a.gm.phs : 4 * GK, nk = a.gm.eq_nk;
    double* tb = s_tb + (EQT ? (threadIdx.x >> 4) * GL * (GL + 1) : 0);
    const bool on = lane < a.gm.b;
    const double s2 = a.theta[a.gm.P - 1];
    double ph = 0.0;         // (Pinf h)[lane]
#pragma unroll
    for (int r = 0; r < NR; r += 2) ph += s_pinf[r * GL + lane];
    const int64_t s = c * a.L, e = min(a.n, s + a.L);
    GElem el;
    double Cm[GL];   // C - Pinf, column lane
#pragma unroll
    for (int r = 0; r < NR; ++r) {
        el.A[r] = (s > a.s0 && r == lane && on) ? 1.0 : 0.0;
        el.J[r] = 0.0;
        Cm[r] = (s > a.s0) ? -s_pinf[r * GL + lane] : 0.0;
    }
    el.bv = 0.0;
    el.eta = 0.0;
    for (int64_t i = s; i < e; ++i) {
        const double yi = a.y[i];
        if (i > a.s0) {
            const double* ph = a.phis + i * phs;
            if constexpr (EQT) {
                g_left_c<NR>(ph, nk, el.A);
                el.bv = g_vleft_c<NR>(ph, nk, lane, el.bv);
                g_sandwich_c<NR>(ph, nk, tb, lane, Cm);
            } else {
                g_left<NR>(ph, el.A);
                el.bv = g_vleft(ph, lane, el.bv);
                g_left<NR>(ph, Cm);
                g_right_t<NR>(ph, lane, Cm);
            }
        }
        if (a.missing && isnan(yi)) continue;               // missing: no update (Eqs. mean4-mean6)
        const double c0 = g_hsum<NR>(Cm) + ph;                  // (C h)[lane]
        const double a0 = g_hsum<NR>(el.A);                      // (h^T A)[lane]
        const double S = s2 + gsum(((lane & 1) == 0) ? c0 : 0.0);
        const double rS = 1.0 / S;
        const double res = yi - gsum(((lane & 1) == 0) ? el.bv : 0.0);
        const double rr = res * rS;
        el.eta = fma(a0, rr, el.eta);
        double v[GL];
        ggather<NR>(a0, v);
        const double ar = a0 * rS;
#pragma unroll
        for (int r = 0; r < NR; ++r) el.J[r] = fma(v[r], ar, el.J[r]);
        el.bv = fma(c0, rr, el.bv);
        ggather<NR>(c0, v);
        const double cr = c0 * rS;
#pragma unroll
        for (int r = 0; r < NR; ++r) {
            el.A[r] = fma(-v[r], ar, el.A[r]);
            Cm[r] = fma(-v[r], cr, Cm[r]);
        }
    }
#pragma unroll
    for (int r = 0; r < NR; ++r) el.C[r] = Cm[r] + s_pinf[r * GL + lane];
    gelem_store<NR>(nodes, a.nc, c, lane, el);
}

// ------------------------------------------------------------------ odd-even reduction, level by level

// Each node of a level is one CTA of 256 threads, thread (r, c) holding entry
// (r, c) of every 16 x 16 matrix in shared memory: a product is 16 FMAs per
// thread, so a level costs about one node's dependent chain of ~10 products
// and a 16-step elimination, whatever its width (the reduction's upper
// levels have few nodes, and a lane group per node would issue 256 FMAs per
// lane per product).  The arithmetic is g_combine / g_state_through /
// g_info_through's: the same products, the same pivoting, the same
// symmetrisation.
static constexpr int GSC = GL * GL;   // threads per node
// the matrices in shared memory keep rows of GL + 1 doubles: a column read
// (X[k][c] over the threads of a row) and a row read of a transposed operand
// (Y[c][k] over c) then fall on distinct banks
static constexpr int GSX = GL + 1;
static constexpr int GSP = GL * GSX;

struct GScanSmem {
    double A[GSP], C[GSP], J[GSP];    // the element (or, down-sweep, the sibling)
    double A2[GSP], C2[GSP], J2[GSP]; // the second element (up-sweep)
    double S[GSP];                    // a state's P or an information's J (down-sweep)
    double N[GSP], M[GSP], T[GSP], U[GSP];
    double bv[GL], eta[GL], bv2[GL], eta2[GL], v[GL], w[GL], z[GL];
    int piv;
    int perm[GL];                     // the pivot row of each column (the inverse's row order)
    double inv;                       // 1 / pivot
};

__device__ __forceinline__ void gc_load_elem(const double* __restrict__ base, int64_t ne, int64_t e, double* A,
                                             double* C, double* J, double* bv, double* eta) {
    const int t = threadIdx.x, r = t >> 4, c = t & 15, q = r * GSX + c;
    const double* p = base + e * GL + c;
    const int64_t st = ne * GL;
    A[q] = p[r * st];
    C[q] = p[(GL + r) * st];
    J[q] = p[(2 * GL + r) * st];
    if (r == 0) { bv[c] = p[3 * GL * st]; eta[c] = p[(3 * GL + 1) * st]; }
}
__device__ __forceinline__ void gc_store_elem(double* __restrict__ base, int64_t ne, int64_t e, const double* A,
                                              const double* C, const double* J, const double* bv,
                                              const double* eta) {
    const int t = threadIdx.x, r = t >> 4, c = t & 15, q = r * GSX + c;
    double* p = base + e * GL + c;
    const int64_t st = ne * GL;
    p[r * st] = A[q];
    p[(GL + r) * st] = C[q];
    p[(2 * GL + r) * st] = J[q];
    if (r == 0) { p[3 * GL * st] = bv[c]; p[(3 * GL + 1) * st] = eta[c]; }
}
__device__ __forceinline__ void gc_load_vs(const double* __restrict__ base, int64_t ne, int64_t e, double* S,
                                           double* v) {
    const int t = threadIdx.x, r = t >> 4, c = t & 15, q = r * GSX + c;
    const double* p = base + e * GL + c;
    const int64_t st = ne * GL;
    S[q] = p[r * st];
    if (r == 0) v[c] = p[GL * st];
}
__device__ __forceinline__ void gc_store_vs(double* __restrict__ base, int64_t ne, int64_t e, const double* S,
                                            const double* v) {
    const int t = threadIdx.x, r = t >> 4, c = t & 15, q = r * GSX + c;
    double* p = base + e * GL + c;
    const int64_t st = ne * GL;
    p[r * st] = S[q];
    if (r == 0) p[GL * st] = v[c];
}

// out[r][c] = sum_k X[r][k] Y[k][c]  (TX: X^T, TY: Y^T); returns this thread's entry
template <bool TX, bool TY>
__device__ __forceinline__ double gc_mm(const double* X, const double* Y) {
    const int r = threadIdx.x >> 4, c = threadIdx.x & 15;
    double s = 0.0;
#pragma unroll
    for (int k = 0; k < GL; ++k) s = fma(TX ? X[k * GSX + r] : X[r * GSX + k], TY ? Y[c * GSX + k] : Y[k * GSX + c], s);
    return s;
}
// out[i] = sum_k X[i][k] x[k] (TX: X^T), threads i < 16
template <bool TX>
__device__ __forceinline__ double gc_mv(const double* X, const double* x) {
    const int i = threadIdx.x;
    double s = 0.0;
#pragma unroll
    for (int k = 0; k < GL; ++k) s = fma(TX ? X[k * GSX + i] : X[i * GSX + k], x[k], s);
    return s;
}

// M = (I + X Y)^-1 by Gauss-Jordan with partial pivoting (at step k the
// largest |N[r][k]| among the rows not yet used as pivots, the first row on
// ties); X, Y, M in shared memory.  The pivot rows stay in place: step k
// rescales the pivot row p and subtracts it from every other row, reading
// one buffer and writing the other (T and U, idle here, are the second pair),
// so a step needs two block barriers; at the end row k of the inverse is
// row perm[k] of the accumulated right-hand side.
__device__ void gc_inv_ixy(GScanSmem& s, const double* X, const double* Y) {
    const int t = threadIdx.x, r = t >> 4, c = t & 15, q = r * GSX + c;
    double *Na = s.N, *Ma = s.M, *Nb = s.T, *Mb = s.U;
    Na[q] = gc_mm<false, false>(X, Y) + ((r == c) ? 1.0 : 0.0);
    Ma[q] = (r == c) ? 1.0 : 0.0;
    bool used = false;   // threads t < 16: row t has been a pivot
    __syncthreads();
#pragma unroll 1
    for (int k = 0; k < GL; ++k) {
        // the pivot row over 16 lanes, and its reciprocal, once for the block
        if (t < GL) {
            double best = used ? -1.0 : fabs(Na[t * GSX + k]);
            int p = t;
#pragma unroll
            for (int off = 8; off > 0; off >>= 1) {
                const double ob = __shfl_down_sync(0x0000ffffu, best, off, GL);
                const int op = __shfl_down_sync(0x0000ffffu, p, off, GL);
                if (ob > best || (ob == best && op < p)) { best = ob; p = op; }
            }
            if (t == 0) {
                s.piv = p;
                s.perm[k] = p;
                s.inv = 1.0 / Na[p * GSX + k];
            }
        }
        __syncthreads();
        const int p = s.piv;
        const double inv = s.inv;
        if (t == p) used = true;
        const double pn = Na[p * GSX + c] * inv, pm = Ma[p * GSX + c] * inv;
        if (r == p) {
            Nb[q] = pn;
            Mb[q] = pm;
        } else {
            const double f = Na[r * GSX + k];
            Nb[q] = fma(-f, pn, Na[q]);
            Mb[q] = fma(-f, pm, Ma[q]);
        }
        __syncthreads();
        double* u = Na; Na = Nb; Nb = u;
        u = Ma; Ma = Mb; Mb = u;
    }
    // GL steps (even): Ma is s.M again
    const double out = Ma[s.perm[r] * GSX + c];
    __syncthreads();
    s.M[q] = out;
    __syncthreads();
}

// level l from level l-1: node j = (2j) then (2j+1), or a copy of 2j at the end
__global__ void __launch_bounds__(GSC) k_gscan_up(const double* __restrict__ lo, int64_t nlo,
                                                  double* __restrict__ hi, int64_t nhi) {
    __shared__ GScanSmem s;
    const int t = threadIdx.x, r = t >> 4, c = t & 15, q = r * GSX + c;
    const int64_t j = blockIdx.x;
    if (j >= nhi) return;
    gc_load_elem(lo, nlo, 2 * j, s.A, s.C, s.J, s.bv, s.eta);
    if (2 * j + 1 >= nlo) {
        __syncthreads();
        gc_store_elem(hi, nhi, j, s.A, s.C, s.J, s.bv, s.eta);
        return;
    }
    gc_load_elem(lo, nlo, 2 * j + 1, s.A2, s.C2, s.J2, s.bv2, s.eta2);
    __syncthreads();
    // (i = first, j = second):  M = (I + C_i J_j)^-1
    gc_inv_ixy(s, s.C, s.J2);
    // A = A_j M A_i
    s.T[q] = gc_mm<false, false>(s.M, s.A);
    // bv: w = bv_i + C_i eta_j;  eta: w2 = eta_j - J_j bv_i
    if (t < GL) {
        s.v[t] = s.bv[t] + gc_mv<false>(s.C, s.eta2);
        s.w[t] = s.eta2[t] - gc_mv<false>(s.J2, s.bv);
    }
    __syncthreads();
    const double Anew = gc_mm<false, false>(s.A2, s.T);
    double bvnew = 0.0, etanew = 0.0;
    if (t < GL) s.z[t] = gc_mv<false>(s.M, s.v);        // M w
    __syncthreads();
    if (t < GL) {
        bvnew = gc_mv<false>(s.A2, s.z) + s.bv2[t];      // A_j M w + bv_j
        s.v[t] = gc_mv<true>(s.M, s.w);                  // M^T w2
    }
    // C = sym(A_j M C_i A_j^T) + C_j
    s.T[q] = gc_mm<false, false>(s.M, s.C);
    __syncthreads();
    if (t < GL) etanew = gc_mv<true>(s.A, s.v) + s.eta[t];   // A_i^T M^T w2 + eta_i
    s.U[q] = gc_mm<false, false>(s.A2, s.T);
    __syncthreads();
    s.N[q] = gc_mm<false, true>(s.U, s.A2);
    // J = sym(A_i^T M^T J_j A_i) + J_i
    s.T[q] = gc_mm<true, false>(s.M, s.J2);
    __syncthreads();
    const double Cnew = 0.5 * ((s.N[q] + s.C2[q]) + (s.N[c * GSX + r] + s.C2[c * GSX + r]));
    s.U[q] = gc_mm<false, false>(s.T, s.A);
    __syncthreads();
    s.T[q] = gc_mm<true, false>(s.A, s.U);
    __syncthreads();
    const double Jnew = 0.5 * ((s.T[q] + s.J[q]) + (s.T[c * GSX + r] + s.J[c * GSX + r]));
    __syncthreads();
    s.A[q] = Anew;
    s.C[q] = Cnew;
    s.J[q] = Jnew;
    if (t < GL) { s.bv[t] = bvnew; s.eta[t] = etanew; }
    __syncthreads();
    gc_store_elem(hi, nhi, j, s.A, s.C, s.J, s.bv, s.eta);
}

// back-substitution from level l (parents) to level l-1 (children): the
// prefix state before each child and the information after it.  Odd child
// j: the parent's state pushed through node j-1; even child j: the parent's
// information pulled back through node j+1 (or kept, at the end).
__global__ void __launch_bounds__(GSC) k_gscan_down(const double* __restrict__ lo, int64_t nlo,
                                                    const double* __restrict__ ppre, const double* __restrict__ psuf,
                                                    int64_t nhi, double* __restrict__ cpre,
                                                    double* __restrict__ csuf) {
    __shared__ GScanSmem s;
    const int t = threadIdx.x, r = t >> 4, c = t & 15, q = r * GSX + c;
    const int64_t j = blockIdx.x;
    if (j >= nlo) return;
    const int64_t parent = j >> 1;
    // the parent's state (into S, v) and information (into C2, w)
    if (ppre) {
        gc_load_vs(ppre, nhi, parent, s.S, s.v);
        gc_load_vs(psuf, nhi, parent, s.C2, s.w);
    } else {
        s.S[q] = 0.0; s.C2[q] = 0.0;
        if (t < GL) { s.v[t] = 0.0; s.w[t] = 0.0; }
    }
    const bool odd = (j & 1) != 0;
    const bool through = odd || (j + 1 < nlo);
    if (through) gc_load_elem(lo, nlo, odd ? j - 1 : j + 1, s.A, s.C, s.J, s.bv, s.eta);
    __syncthreads();
    if (!through) {   // the last even child keeps the parent's state and information
        gc_store_vs(cpre, nlo, j, s.S, s.v);
        gc_store_vs(csuf, nlo, j, s.C2, s.w);
        return;
    }
    if (odd) {
        // N(m, P) pushed through e: M = (I + P J_e)^-1, m' = A_e M (m + P eta_e) + bv_e,
        // P' = sym(A_e M P A_e^T) + C_e
        gc_inv_ixy(s, s.S, s.J);
        if (t < GL) s.z[t] = s.v[t] + gc_mv<false>(s.S, s.eta);
        s.T[q] = gc_mm<false, false>(s.M, s.S);
        __syncthreads();
        double mnew = 0.0;
        if (t < GL) s.bv2[t] = gc_mv<false>(s.M, s.z);
        s.U[q] = gc_mm<false, false>(s.A, s.T);
        __syncthreads();
        if (t < GL) mnew = gc_mv<false>(s.A, s.bv2) + s.bv[t];
        s.N[q] = gc_mm<false, true>(s.U, s.A);
        __syncthreads();
        const double Pnew = 0.5 * ((s.N[q] + s.C[q]) + (s.N[c * GSX + r] + s.C[c * GSX + r]));
        __syncthreads();
        s.T[q] = Pnew;
        if (t < GL) s.z[t] = mnew;
        __syncthreads();
        gc_store_vs(cpre, nlo, j, s.T, s.z);
        gc_store_vs(csuf, nlo, j, s.C2, s.w);
    } else {
        // information (eta, J) pulled back through e: M = (I + C_e J)^-1,
        // eta' = A_e^T M^T (eta - J bv_e) + eta_e, J' = sym(A_e^T M^T J A_e) + J_e
        gc_inv_ixy(s, s.C, s.C2);
        if (t < GL) s.z[t] = s.w[t] - gc_mv<false>(s.C2, s.bv);
        s.T[q] = gc_mm<true, false>(s.M, s.C2);
        __syncthreads();
        double enew = 0.0;
        if (t < GL) s.bv2[t] = gc_mv<true>(s.M, s.z);
        s.U[q] = gc_mm<false, false>(s.T, s.A);
        __syncthreads();
        if (t < GL) enew = gc_mv<true>(s.A, s.bv2) + s.eta[t];
        s.N[q] = gc_mm<true, false>(s.A, s.U);
        __syncthreads();
        const double Jnew = 0.5 * ((s.N[q] + s.J[q]) + (s.N[c * GSX + r] + s.J[c * GSX + r]));
        __syncthreads();
        s.T[q] = Jnew;
        if (t < GL) s.z[t] = enew;
        __syncthreads();
        gc_store_vs(cpre, nlo, j, s.S, s.v);
        gc_store_vs(csuf, nlo, j, s.T, s.z);
    }
}

// ------------------------------------------------------------------ k_gchunk: forward, reverse sweep

static constexpr int GNF = GL + 4;   // stored per lane per step: predicted covariance column, mean entry, v, 1/S, gain entry

template <int MODE, int NR, bool EQT>
__global__ void __launch_bounds__(GCTA) k_gchunk(GArgs a, const double* __restrict__ pre,
                                                 const double* __restrict__ suf, double* __restrict__ store,
                                                 double* __restrict__ part, double* __restrict__ mean_out,
                                                 double* __restrict__ var_out) {
    constexpr bool BWD = (MODE != MODE_LOGLIK);
    constexpr bool GRAD = (MODE == MODE_GRAD || MODE == MODE_GRAD_POSTERIOR);
    constexpr bool POST = (MODE == MODE_POSTERIOR || MODE == MODE_GRAD_POSTERIOR);
    __shared__ GSmem sm[GGRP];
    __shared__ double s_pinf[GL * GL], s_dpe[GL * GL];
    g_pinf_smem(a.gm, a.theta, a.gconst, s_pinf, s_dpe);
    // the group scratch starts at zero: the column products below write only
    // rows < NR, so rows past the state stay exactly zero
    {
        double* z = reinterpret_cast<double*>(sm);
        for (int i = threadIdx.x; i < (int)(sizeof(sm) / sizeof(double)); i += blockDim.x) z[i] = 0.0;
    }
    __syncthreads();
    const int lane = threadIdx.x & (GL - 1);
    const int g = threadIdx.x >> 4;
    const int64_t c = blockIdx.x * (int64_t)GGRP + g;
    if (c >= a.nc) return;
    const int64_t nc = a.nc;
    const bool even = (lane & 1) == 0;
    const bool has_eq = a.gm.eq_nk > 0;
    const int phs = EQT ? a.gm.phs : 4 * GK, nk = a.gm.eq_nk;
    double* tb = sm[g].X;   // transpose scratch (EQT)
    const double s2 = a.theta[a.gm.P - 1];
    double ph = 0.0;   // (Pinf h)[lane]
#pragma unroll
    for (int r = 0; r < NR; r += 2) ph += s_pinf[r * GL + lane];
    const int64_t s = c * a.L, e = min(a.n, s + a.L);
    int bad = 0;

    // ---- forward from the prefix state (m, D = P - Pinf)
    double m, D[GL];
    double pe_pre;   // (P h)[lane] of the filtered state before the chunk (the lag-one output)
    {
        double P[GL];
        gvs_load<NR>(pre, nc, c, lane, P, m);
        pe_pre = g_hsum<NR>(P);
#pragma unroll
        for (int r = 0; r < NR; ++r) D[r] = P[r] - s_pinf[r * GL + lane];
    }
    (void)pe_pre;
    double quad = 0.0, prod = 1.0;
    int expo = 0;
    int64_t nobs = 0;
    for (int64_t i = s; i < e; ++i) {
        const int64_t j = i - s;
        const double yi = a.y[i];
        const bool obs = !(a.missing && isnan(yi));   // the same in every lane of the group
        double mb, Db[GL];
        if (i == a.s0) {
            mb = 0.0;
#pragma unroll
            for (int r = 0; r < NR; ++r) Db[r] = 0.0;
        } else {
            const double* ph = a.phis + i * phs;
#pragma unroll
            for (int r = 0; r < NR; ++r) Db[r] = D[r];
            if constexpr (EQT) {
                mb = g_vleft_c<NR>(ph, nk, lane, m);
                g_sandwich_c<NR>(ph, nk, tb, lane, Db);
            } else {
                mb = g_vleft(ph, lane, m);
                g_left<NR>(ph, Db);
                g_right_t<NR>(ph, lane, Db);
            }
        }
        const double p0 = g_hsum<NR>(Db) + ph;
        // a missing observation stores v = 1/S = 0, so the reverse sweep passes through it
        double rS = 0.0, v = 0.0;
        if (obs) {
            const double S = s2 + gsum(even ? p0 : 0.0);
            if (!(S > 0.0) || !isfinite(S)) bad |= ST_ENUMERIC;
            rS = 1.0 / S;
            v = yi - gsum(even ? mb : 0.0);
            quad = fma(v * v, rS, quad);
            prod *= S;
            const unsigned long long bits = (unsigned long long)__double_as_longlong(prod);
            expo += (int)((bits >> 52) & 0x7ffULL) - 1023;
            prod = __longlong_as_double((long long)((bits & 0x800FFFFFFFFFFFFFULL) | 0x3FF0000000000000ULL));
            ++nobs;
        }
        const double pr = p0 * rS;   // the gain entry k = (Pb h)[lane] / S
        if constexpr (BWD) {
            double* st = store + ((j * nc + c) * GNF) * GL + lane;
#pragma unroll
            for (int r = 0; r < NR; ++r) st[r * GL] = Db[r];
            st[GL * GL] = mb;
            st[(GL + 1) * GL] = v;
            st[(GL + 2) * GL] = rS;
            // the gradient keeps the gain entry there; the posterior keeps
            // (Pb h)[lane] (the prediction at a missing step, the lag-one term)
            st[(GL + 3) * GL] = POST ? p0 : pr;
        }
        double pv[GL];
        ggather<NR>(p0, pv);
        m = fma(p0, v * rS, mb);
#pragma unroll
        for (int r = 0; r < NR; ++r) D[r] = fma(-pv[r], pr, Db[r]);
    }
    double acc[2 + 2 * GMAXCOMP];
#pragma unroll
    for (int f = 0; f < 2 + 2 * GMAXCOMP; ++f) acc[f] = 0.0;
    if (lane == 0) acc[0] = -0.5 * (quad + log(prod) + (double)expo * G_LN2 + (double)nobs * G_LOG_2PI);

    if constexpr (BWD) {
        // ---- adjoint of the last filtered state from the information after the chunk
        double lh, Lh[GL];
        {
            double J[GL], eta, P[GL], W[GL], v[GL];
            gvs_load<NR>(suf, nc, c, lane, J, eta);
#pragma unroll
            for (int r = 0; r < NR; ++r) P[r] = D[r] + s_pinf[r * GL + lane];
            g_inv_ixy<NR>(sm[g], lane, J, P, W);            // (I + J P)^-1
            ggather<NR>(m, v);
            double w = eta;
#pragma unroll
            for (int k = 0; k < NR; ++k) w = fma(-J[k], v[k], w);   // (eta - J m)[lane]
            ggather<NR>(w, v);
            const unsigned mask = half_mask();
            g_put<NR>(sm[g].X, lane, W); __syncwarp(mask);
            // (lanes past the rows hold no column; the scratch there may hold transposes)
            lh = (lane < NR) ? -g_rowdot<NR>(sm[g].X, lane, v) : 0.0; __syncwarp(mask);
            g_mul<NR>(sm[g].X, J, Lh); __syncwarp(mask);     // W J
            g_sym<NR>(sm[g], lane, Lh);
        }
        // per-block sums of the rate terms (dt times d ll / dx), folded into
        // the component slots once per chunk
        // - brate[kb]: the column part <G_k,:, X_k Db_k,:> over this lane's
        //   column, without the harmonic number of a rotation block (applied
        //   once per chunk); benv[kb]: <G_k,:, Db_k,:> (the envelope's X = -I,
        //   sign applied once per chunk);
        // - rmine, emine: the row part lt_k^T X_k mb_k (resp. lt_k^T mb_k) of
        //   the lane's own block only, from the row of X_k that the lane holds
        //   (xm0, xm1): one term per lane instead of one per block
        double brate[NR / 2], benv[NR / 2], rmine = 0.0, emine = 0.0;
#pragma unroll
        for (int kb = 0; kb < NR / 2; ++kb) { brate[kb] = 0.0; benv[kb] = 0.0; }
        const int kbm = lane >> 1;
        double xm0 = 0.0, xm1 = 0.0;
#pragma unroll
        for (int kb = 0; kb < NR / 2; ++kb) {
            if (kb >= a.gm.K) break;
            if (kb != kbm) continue;
            const int kind = a.gm.bkind[kb];
            if (kind == GB_MATERN32) {            // X = [[0, 1], [-1, -2]]
                xm0 = even ? 0.0 : -1.0; xm1 = even ? 1.0 : -2.0;
            } else if (kind == GB_EQ) {           // X = [[a, b], [-b, a]]
                const double ea = a.gm.eqa[kb], eb = a.gm.eqb[kb];
                xm0 = even ? ea : -eb; xm1 = even ? eb : ea;
            } else {                              // X = j [[0, -1], [1, 0]], j applied per chunk
                xm0 = even ? 0.0 : 1.0; xm1 = even ? -1.0 : 0.0;
            }
        }
        // gp, geq and G below carry twice their values (the factor 1/2 of the
        // adjoint is applied once per chunk, an exact power-of-two scaling)
        double gp = 0.0;   // diagonal entry 'lane' of the Pinf adjoint
        double geq = 0.0;  // column 'lane' of the Pinf adjoint contracted with the EQ sections' P
        // dPinf / d(EQ variance) is block diagonal (a 2 x 2 block per section):
        // column 'lane' has nonzeros only in the rows of the lane's own
        // section, which are this lane's and its partner's
        const int eb = lane >> 1;
        const bool eq_lane = has_eq && eb < a.gm.eq_nk;
        const double pe0 = eq_lane ? s_dpe[(2 * eb) * GL + lane] : 0.0;
        const double pe1 = eq_lane ? s_dpe[(2 * eb + 1) * GL + lane] : 0.0;
        for (int64_t i = e - 1; i >= s; --i) {
            const int64_t j = i - s;
            const double* st = store + ((j * nc + c) * GNF) * GL + lane;
            double Db[GL];
#pragma unroll
            for (int r = 0; r < NR; ++r) Db[r] = st[r * GL];
            const double mb = st[GL * GL];
            const double v = st[(GL + 1) * GL];
            const double rS = st[(GL + 2) * GL];
            // the gain entry (Pb h)[lane] / S; (Pb h)[lane] itself at a missing
            // step of the posterior, whose kl, kuk below are then (Pb h)^T lh
            // and (Pb h)^T Lh (Pb h)
            const double ks = st[(GL + 3) * GL];
            double k = ks;
            if constexpr (POST) {
                if (!(a.missing && isnan(a.y[i]))) k = ks * rS;
            }
            double kl = gsum(k * lh);
            double kv[GL];
            ggather<NR>(k, kv);
            double u = 0.0;
#pragma unroll
            for (int r = 0; r < NR; ++r) u = fma(Lh[r], kv[r], u);
            double kuk = gsum(k * u);
            if constexpr (POST) {
                const double yi = a.y[i];
                const double hk = gsum(even ? k : 0.0);
                if (a.missing && isnan(yi)) {
                    // predicted only: mean = h^T (mb - Pb lh), variance = h^T Pb h - (Pb h)^T Lh (Pb h);
                    // the adjoint then passes through unchanged
                    const double hm = gsum(even ? mb : 0.0);
                    if (lane == 0) {
                        mean_out[i] = hm - kl;
                        var_out[i] = hk - kuk;
                    }
                    kl = 0.0;
                    kuk = 0.0;
                    u = 0.0;
                } else if (lane == 0) {
                    mean_out[i] = fma(-s2, fma(v, rS, kl), yi);
                    var_out[i] = s2 * hk - s2 * s2 * kuk;
                }
            }
            const double al = fma(v, rS, kl);
            const double cc = rS + kuk;
            if constexpr (GRAD) {
                if (lane == 0) acc[1] = fma(al, al, acc[1]) - cc;
            }
            const double lt = lh - (even ? al : 0.0);
            // Lt = Lh - h u^T - u h^T + cc h h^T = Lh - h ub^T - ub h^T with ub = u - (cc / 2) h
            const double ub = even ? fma(-0.5, cc, u) : u;
            double uv[GL], Lt[GL];
            ggather<NR>(ub, uv);
#pragma unroll
            for (int r = 0; r < NR; ++r) {
                double x = Lh[r];
                if ((r & 1) == 0) x -= ub;
                if (even) x -= uv[r];
                Lt[r] = x;
            }
            double lv[GL], G[GL];
            ggather<NR>(lt, lv);
#pragma unroll
            for (int r = 0; r < NR; ++r) G[r] = fma(lv[r], lt, -Lt[r]);   // 2 x the adjoint of Q
            if constexpr (GRAD) {
                double gsel = 0.0;   // G[lane][lane]: a select, then one add
#pragma unroll
                for (int r = 0; r < NR; ++r) gsel = (r == lane) ? G[r] : gsel;
                gp += gsel;
                if (has_eq) {
                    double g0 = 0.0, g1 = 0.0;   // rows 2 eb, 2 eb + 1 of G's column: selects
#pragma unroll
                    for (int q = 0; q < NR / 2; ++q)
                        if (q == eb) { g0 = G[2 * q]; g1 = G[2 * q + 1]; }
                    geq = fma(pe0, g0, fma(pe1, g1, geq));
                }
            }
            if (i > a.s0) {
                const double* ph = a.phis + i * phs;
                if constexpr (POST) {
                    if (a.lag1) {
                        // Cov(f_i, f_{i-1} | y) = h^T w - (Pb h)^T Lt w, w = A P_{i-1} h
                        // (Lt: the adjoint with y_i and after, on the predicted state i;
                        // P_{i-1} h = (Pb_{i-1} h) s_n / S_{i-1}, or Pb_{i-1} h at a
                        // missing step; the chunk's prefix state before its first step)
                        double w = pe_pre;
                        if (i > s) {
                            const double* sp = store + (((j - 1) * nc + c) * GNF) * GL + lane;
                            const double rsp = sp[(GL + 2) * GL];
                            w = sp[(GL + 3) * GL] * ((rsp == 0.0) ? 1.0 : s2 * rsp);
                        }
                        if constexpr (EQT) w = g_vleft_c<NR>(ph, nk, lane, w);
                        else w = g_vleft(ph, lane, w);
                        double pv[GL];
                        ggather<NR>(ks, pv);
                        double tl2 = 0.0;                       // (Pb h)^T Lt[:, lane]
#pragma unroll
                        for (int r = 0; r < NR; ++r) tl2 = fma(pv[r], Lt[r], tl2);
                        const double hw = gsum(even ? w : 0.0), q = gsum(w * tl2);
                        if (lane == 0) a.lag1[i - 1] = hw - q;
                    }
                }
                if constexpr (GRAD) {
                    const double dt = (i > 0) ? a.t[i] - a.t[i - 1] : a.t[0] - a.t_prev;
                    // per block: 2 <G_k,:, X_k Db_k,:> (column 'lane' part) - lt_k^T X_k mb_k (row 'lane' part);
                    // G holds 2 G, so the first term is <G_k,:, X_k Db_k,:>
                    const double mp = gxor(mb, 1);
                    const double mb0 = even ? mb : mp, mb1 = even ? mp : mb;
                    const double tl = dt * lt;
                    rmine = fma(tl, fma(xm0, mb0, xm1 * mb1), rmine);
                    emine = fma(tl, mb, emine);
#pragma unroll
                    for (int kb = 0; kb < NR / 2; ++kb) {
                        if (kb >= a.gm.K) break;
                        const int kind = a.gm.bkind[kb];
                        const double d0 = Db[2 * kb], d1 = Db[2 * kb + 1];
                        const double g0 = G[2 * kb], g1 = G[2 * kb + 1];
                        if (kind == GB_MATERN32) {
                            brate[kb] = fma(dt, fma(g1, fma(-2.0, d1, -d0), g0 * d1), brate[kb]);
                        } else if (kind == GB_EQ) {
                            // X = [[a, b], [-b, a]] per unit of x = dt / l (rate 1 / l)
                            const double ea = a.gm.eqa[kb], eb = a.gm.eqb[kb];
                            brate[kb] = fma(dt, g0 * fma(ea, d0, eb * d1) + g1 * fma(-eb, d0, ea * d1), brate[kb]);
                        } else {
                            // X = j [[0, -1], [1, 0]] (rotation rate w); envelope X = -I
                            brate[kb] = fma(dt, fma(g1, d0, -g0 * d1), brate[kb]);
                            if (kind == GB_QUASI) benv[kb] = fma(dt, fma(g0, d0, g1 * d1), benv[kb]);
                        }
                    }
                    if constexpr (EQT) {
                        // the EQ generator's coupling blocks -u_k w_i^T (k > i): the
                        // column part <G, T_c Db> over this lane's column, T_c Db's
                        // rows of section k being -u_k sig_k, sig_k = sum_{i<k} w_i^T Db_i
                        // (a running sum down the sections), into the EQ component's
                        // slot (block 0); the row part lt^T T_c mb of the lane's own
                        // entry, (T_c mb)[lane] = -u_k[odd] sum_{i<k} w_i^T mb_i
                        double sig = 0.0, cpt = 0.0;
#pragma unroll
                        for (int k = 0; k < NR / 2; ++k) {
                            if (k < nk) {
                                if (k > 0)
                                    cpt = fma(-sig, fma(a.gm.equ[2 * k], G[2 * k], a.gm.equ[2 * k + 1] * G[2 * k + 1]),
                                              cpt);
                                sig = fma(a.gm.eqw[2 * k], Db[2 * k], fma(a.gm.eqw[2 * k + 1], Db[2 * k + 1], sig));
                            }
                        }
                        brate[0] = fma(dt, cpt, brate[0]);
                        double mv[GL];
                        ggather<NR>(mb, mv);
                        double sm_ = 0.0;
#pragma unroll
                        for (int q = 0; q < NR / 2; ++q)
                            if (q < kbm && q < nk) sm_ = fma(a.gm.eqw[2 * q], mv[2 * q], fma(a.gm.eqw[2 * q + 1], mv[2 * q + 1], sm_));
                        if (kbm < nk) rmine = fma(tl, -a.gm.equ[lane] * sm_, rmine);
                    }
                }
                // propagate to the previous step: lh = Phi^T lt, Lh = Phi^T Lt Phi
#pragma unroll
                for (int r = 0; r < NR; ++r) Lh[r] = Lt[r];
                if constexpr (EQT) {
                    lh = g_vleft_t_c<NR>(ph, nk, lane, lt);
                    g_sandwich_t_c<NR>(ph, nk, tb, lane, Lh);
                } else {
                    lh = g_vleft_t(ph, lane, lt);
                    g_right<NR>(ph, lane, Lh);
                    g_left_t<NR>(ph, Lh);
                }
                if constexpr (GRAD) {
                    double ld = 0.0;
#pragma unroll
                    for (int r = 0; r < NR; ++r)
                        if (r == lane) ld = Lh[r];
                    gp -= fma(lh, lh, -ld);
                    if (has_eq) {   // minus column 'lane' of 2 Phi^T G Phi = lh lh^T - Lh, rows 2 eb, 2 eb + 1
                        const double lp = gxor(lh, 1);
                        const double l0 = (lane & 1) ? lp : lh, l1 = (lane & 1) ? lh : lp;
                        double h0 = 0.0, h1 = 0.0;
#pragma unroll
                        for (int q = 0; q < NR / 2; ++q)
                            if (q == eb) { h0 = Lh[2 * q]; h1 = Lh[2 * q + 1]; }
                        geq -= fma(pe0, fma(l0, lh, -h0), pe1 * fma(l1, lh, -h1));
                    }
                }
            }
        }
        if constexpr (GRAD) {
#pragma unroll
            for (int kb = 0; kb < NR / 2; ++kb) {
                if (kb >= a.gm.K) break;
                const int kind = a.gm.bkind[kb];
                double r = brate[kb], ev = -benv[kb];
                if (kb == kbm) { r -= rmine; ev += emine; }
                if (kind != GB_MATERN32 && kind != GB_EQ) r *= (double)a.gm.bj[kb];
                if (kind != GB_QUASI) ev = 0.0;
                const int cp = a.gm.bcomp[kb];
#pragma unroll
                for (int q = 0; q < GMAXCOMP; ++q)
                    if (q == cp) { acc[2 + 2 * q] += r; acc[3 + 2 * q] += ev; }
            }
            part[(2 + 2 * GMAXCOMP + lane) * nc + c] = 0.5 * gp;
            geq = 0.5 * gsum(geq);
            if (lane == 0) part[GP_EQ * nc + c] = geq;
        }
    }
    if (bad) atomicOr(a.status, bad);
    // per-chunk partials: group sums for the scalar slots, per-lane for the Pinf diagonal
#pragma unroll
    for (int f = 0; f < 2 + 2 * GMAXCOMP; ++f) acc[f] = gsum(acc[f]);
    const int nu = GRAD ? 2 + 2 * GMAXCOMP : 1;
    if (lane == 0)
        for (int f = 0; f < nu; ++f) part[f * nc + c] = acc[f];
}

// ------------------------------------------------------------------ k_gfinal: fixed-order sums, chain rule

static constexpr int GFIN = 128;

__global__ void __launch_bounds__(GFIN) k_gfinal(GModel gm, const double* __restrict__ part, int64_t nc, int na,
                                                 const double* __restrict__ theta, const double* __restrict__ gconst,
                                                 double* __restrict__ ll_out, double* __restrict__ grad_out) {
    __shared__ double red[GFIN * GPART];
    __shared__ double tot[GPART];
    const int tid = threadIdx.x;
    for (int f = 0; f < na; ++f) {
        double s = 0.0;
        for (int64_t c = tid; c < nc; c += GFIN) s += part[f * nc + c];
        red[f * GFIN + tid] = s;
    }
    __syncthreads();
    for (int w = GFIN / 2; w > 0; w >>= 1) {
        if (tid < w)
            for (int f = 0; f < na; ++f) red[f * GFIN + tid] += red[f * GFIN + tid + w];
        __syncthreads();
    }
    if (tid < na) tot[tid] = red[tid * GFIN];
    __syncthreads();
    if (tid != 0) return;
    if (ll_out) ll_out[0] = tot[0];
    if (!grad_out || na != GPART) return;
    for (int p = 0; p < gm.P; ++p) grad_out[p] = 0.0;
    grad_out[gm.P - 1] = 0.5 * tot[1];
    for (int q = 0; q < gm.ncomp; ++q) {
        const double* th = theta + gm.cpoff[q];
        double* g = grad_out + gm.cpoff[q];
        const double rate = tot[2 + 2 * q], envr = tot[3 + 2 * q];
        if (gm.ckind[q] == SPINGP_MATERN32) {
            const double lam = sqrt(3.0) / th[0];
            g[0] = rate * (-lam / th[0]);
        } else if (gm.ckind[q] == SPINGP_EQ) {
            g[0] = rate * (-1.0 / (th[0] * th[0]));           // rate 1 / l
            g[1] = tot[GP_EQ];                                 // dPinf / d variance = P_m
        } else {
            const double per = th[2];
            g[2] = rate * (-2.0 * M_PI / (per * per));            // d w / d period
            if (gm.ckind[q] == SPINGP_QUASIPERIODIC) g[3] = envr * (-1.0 / (th[3] * th[3]));   // lam_e = 1/l_e
        }
    }
    // Pinf entries: block k is w_k I2
    for (int k = 0; k < gm.K; ++k) {
        if (gm.bkind[k] == GB_EQ) continue;                   // handled with its component
        const int q = gm.bcomp[k];
        const double gk = tot[2 + 2 * GMAXCOMP + 2 * k] + tot[2 + 2 * GMAXCOMP + 2 * k + 1];
        double* g = grad_out + gm.cpoff[q];
        if (gm.ckind[q] == SPINGP_MATERN32) {
            g[1] += gk * gconst[k * GNC + 1];
        } else {
            g[0] += gk * gconst[k * GNC + 1];
            g[1] += gk * gconst[k * GNC + 2];
        }
    }
}

// ------------------------------------------------------------------ host side

static size_t galign(size_t x) { return (x + 255) & ~(size_t)255; }

struct GLayout {
    int64_t nc;
    int nlev;               // levels above the chunk elements
    int64_t lev_n[40];      // node counts, level 0 = chunks
    size_t off_gconst, off_phis, off_nodes[40], off_pre[40], off_suf[40], off_part, off_store, total;

    GLayout(int64_t n, int64_t L, int mode, int phs) {
        nc = (n + L - 1) / L;
        size_t o = 256;
        off_gconst = o; o = galign(o + sizeof(double) * GK * GNC);
        off_phis = o; o = galign(o + sizeof(double) * phs * (size_t)n);
        nlev = 0;
        lev_n[0] = nc;
        while (lev_n[nlev] > 1) { lev_n[nlev + 1] = (lev_n[nlev] + 1) / 2; ++nlev; }
        for (int l = 0; l <= nlev; ++l) {
            off_nodes[l] = o; o = galign(o + sizeof(double) * GNE * GL * (size_t)lev_n[l]);
            off_pre[l] = o; o = galign(o + sizeof(double) * GNM * GL * (size_t)lev_n[l]);
            off_suf[l] = o; o = galign(o + sizeof(double) * GNM * GL * (size_t)lev_n[l]);
        }
        off_part = o; o = galign(o + sizeof(double) * GPART * (size_t)nc);
        off_store = o;
        if (mode != MODE_LOGLIK) o = galign(o + sizeof(double) * GNF * GL * (size_t)L * nc);
        // a split series: the ranks' elements and their reduction tree, and
        // this rank's prefix / suffix as one node
        seg_nlev = 0;
        seg_n[0] = SEG_MAX_RANKS;
        while (seg_n[seg_nlev] > 1) { seg_n[seg_nlev + 1] = (seg_n[seg_nlev] + 1) / 2; ++seg_nlev; }
        for (int l = 0; l <= seg_nlev; ++l) {
            off_seg_nodes[l] = o; o = galign(o + sizeof(double) * GNE * GL * (size_t)seg_n[l]);
            off_seg_pre[l] = o; o = galign(o + sizeof(double) * GNM * GL * (size_t)seg_n[l]);
            off_seg_suf[l] = o; o = galign(o + sizeof(double) * GNM * GL * (size_t)seg_n[l]);
        }
        off_seg_top = o; o = galign(o + sizeof(double) * 2 * GNM * GL);
        total = o;
    }
    int seg_nlev;
    int64_t seg_n[8];
    size_t off_seg_nodes[8], off_seg_pre[8], off_seg_suf[8], off_seg_top;
};

// The up-sweep of the level-by-level reduction over cnt[0] elements at
// nodes[0] (cnt[l] nodes at level l, nlev levels above level 0).
static void gscan_up(char* ws, const size_t* nodes, const int64_t* cnt, int nlev, cudaStream_t st) {
    for (int l = 1; l <= nlev; ++l)
        k_gscan_up<<<(unsigned)cnt[l], GSC, 0, st>>>((const double*)(ws + nodes[l - 1]), cnt[l - 1],
                                                     (double*)(ws + nodes[l]), cnt[l]);
}
// The down-sweep: the state before and the information after every level-0
// element, from top_pre / top_suf at the single top node (NULL: zero, a
// whole series).
static int gscan_down(char* ws, const size_t* nodes, const size_t* pre, const size_t* suf, const int64_t* cnt,
                      int nlev, const double* top_pre, const double* top_suf, cudaStream_t st) {
    for (int l = nlev; l >= 1; --l) {
        const bool top = (l == nlev);
        k_gscan_down<<<(unsigned)cnt[l - 1], GSC, 0, st>>>(
            (const double*)(ws + nodes[l - 1]), cnt[l - 1], top ? top_pre : (const double*)(ws + pre[l]),
            top ? top_suf : (const double*)(ws + suf[l]), cnt[l], (double*)(ws + pre[l - 1]),
            (double*)(ws + suf[l - 1]));
    }
    if (nlev == 0) {   // one element: its prefix and suffix are the top's
        const size_t b = sizeof(double) * GNM * GL;
        if (top_pre) {
            if (cudaMemcpyAsync(ws + pre[0], top_pre, b, cudaMemcpyDeviceToDevice, st) != cudaSuccess ||
                cudaMemcpyAsync(ws + suf[0], top_suf, b, cudaMemcpyDeviceToDevice, st) != cudaSuccess)
                return 1;
        } else if (cudaMemsetAsync(ws + pre[0], 0, b, st) != cudaSuccess ||
                   cudaMemsetAsync(ws + suf[0], 0, b, st) != cudaSuccess) {
            return 1;
        }
    }
    return 0;
}

// k_gfold / k_gchunk for the state's row count (the dimension rounded up to
// 4) and whether the transition has EQ coupling blocks
static void gfold_launch(int NRr, bool eqt, unsigned grid, cudaStream_t st, const GArgs& a, double* nodes0) {
#define SPG_GFOLD(NRv) (eqt ? k_gfold<NRv, true><<<grid, GCTA, 0, st>>>(a, nodes0) \
                            : k_gfold<NRv, false><<<grid, GCTA, 0, st>>>(a, nodes0))
    switch (NRr) {
    case 4: SPG_GFOLD(4); break;
    case 8: SPG_GFOLD(8); break;
    case 12: SPG_GFOLD(12); break;
    default: SPG_GFOLD(16); break;
    }
#undef SPG_GFOLD
}
template <int M>
static void gchunk_launch(int NRr, bool eqt, unsigned grid, cudaStream_t st, const GArgs& a, const double* pre,
                          const double* suf, double* store, double* part, double* mean_out, double* var_out) {
#define SPG_GCHUNK(NRv) (eqt ? k_gchunk<M, NRv, true><<<grid, GCTA, 0, st>>>(a, pre, suf, store, part, mean_out, var_out) \
                             : k_gchunk<M, NRv, false><<<grid, GCTA, 0, st>>>(a, pre, suf, store, part, mean_out, var_out))
    switch (NRr) {
    case 4: SPG_GCHUNK(4); break;
    case 8: SPG_GCHUNK(8); break;
    case 12: SPG_GCHUNK(12); break;
    default: SPG_GCHUNK(16); break;
    }
#undef SPG_GCHUNK
}

size_t group_ws_bytes(const GModel& gm, int64_t n, int64_t L, int mode) { return GLayout(n, L, mode, gm.phs).total; }

int group_launch_count(int64_t n, int64_t L, int mode) {
    GLayout lay(n, L, mode, 4 * GK);
    return 2 + 1 + 2 * lay.nlev + 1 + 1;
}

int group_run(const GModel& gm, int mode, const double* t, const double* y, int64_t n, int64_t L,
              const double* theta, double* ll_out, double* grad_out, double* mean_out, double* var_out, void* wsv,
              cudaStream_t st, cudaEvent_t* ev, int missing, double* lag1_out) {
    GLayout lay(n, L, mode, gm.phs);
    char* ws = (char*)wsv;
    int* status = (int*)ws;
    double* gconst = (double*)(ws + lay.off_gconst);
    double* phis = (double*)(ws + lay.off_phis);
    double* part = (double*)(ws + lay.off_part);
    double* store = (double*)(ws + lay.off_store);
    GArgs a{gm, t, y, n, L, lay.nc, theta, gconst, phis, status, missing, 0, 0.0};
    a.lag1 = (mode == MODE_POSTERIOR || mode == MODE_GRAD_POSTERIOR) ? lag1_out : nullptr;
    if (cudaMemsetAsync(status, 0, sizeof(int), st) != cudaSuccess) return 1;
    if (ev) cudaEventRecord(ev[0], st);
    k_gsetup<<<1, 32, 0, st>>>(gm, theta, gconst, status);
    k_gdisc<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(gm, t, y, n, theta, phis, status, missing, 0, 0.0);
    const unsigned cgrid = (unsigned)((lay.nc + GGRP - 1) / GGRP);
    // rows of the per-lane column arithmetic: the state dimension rounded up to 4
    const int NRr = (gm.b <= 4) ? 4 : (gm.b <= 8) ? 8 : (gm.b <= 12) ? 12 : 16;
    const bool eqt = gm.eq_nk > 1;
    gfold_launch(NRr, eqt, cgrid, st, a, (double*)(ws + lay.off_nodes[0]));
    if (ev) cudaEventRecord(ev[1], st);
    gscan_up(ws, lay.off_nodes, lay.lev_n, lay.nlev, st);
    if (gscan_down(ws, lay.off_nodes, lay.off_pre, lay.off_suf, lay.lev_n, lay.nlev, nullptr, nullptr, st)) return 1;
    if (ev) cudaEventRecord(ev[2], st);
    const double* pre = (const double*)(ws + lay.off_pre[0]);
    const double* suf = (const double*)(ws + lay.off_suf[0]);
    int na = 1;
    if (mode == MODE_LOGLIK) {
        gchunk_launch<MODE_LOGLIK>(NRr, eqt, cgrid, st, a, pre, suf, store, part, nullptr, nullptr);
    } else if (mode == MODE_GRAD) {
        gchunk_launch<MODE_GRAD>(NRr, eqt, cgrid, st, a, pre, suf, store, part, nullptr, nullptr);
        na = GPART;
    } else if (mode == MODE_GRAD_POSTERIOR) {
        gchunk_launch<MODE_GRAD_POSTERIOR>(NRr, eqt, cgrid, st, a, pre, suf, store, part, mean_out, var_out);
        na = GPART;
    } else {
        gchunk_launch<MODE_POSTERIOR>(NRr, eqt, cgrid, st, a, pre, suf, store, part, mean_out, var_out);
    }
    if (ev) cudaEventRecord(ev[3], st);
    k_gfinal<<<1, GFIN, 0, st>>>(gm, part, lay.nc, na, theta, gconst, ll_out, grad_out);
    if (ev) cudaEventRecord(ev[4], st);
    return cudaGetLastError() == cudaSuccess ? 0 : 1;
}

// ------------------------------------------------------------------ a series split across ranks
//
// The same two phases as the chain path (matern.cu): phase 0 reduces this
// rank's range to its top element (GNE x GL doubles: element e's value f of
// lane l at [f * GL + l]); phase 1 takes all G elements (rank-major), runs
// the level-by-level reduction over them for the state before this range and
// the information after it, then this range's down-sweep, chunk pass and
// final reduction (its share of ll and gradient).  Phase 1 reuses the
// workspace that phase 0 filled.

// rank-major elements [G][GNE * GL] to the level layout [(f * G + e) * GL + l]
__global__ void __launch_bounds__(256) k_gelems_to_soa(const double* __restrict__ in, double* __restrict__ out, int G) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    constexpr int per = GNE * GL;
    if (i < G * per) {
        const int e = i / per, fl = i % per, f = fl / GL, l = fl % GL;
        out[((int64_t)f * G + e) * GL + l] = in[i];
    }
}

int group_segment(const GModel& gm, int phase, const double* t, const double* y, int64_t n, int64_t L,
                  const double* theta, double t_prev, int first, const double* elems, int G, int rank,
                  double* elem_out, double* ll_out, double* grad_out, void* wsv, cudaStream_t st, int missing,
                  double* mean_out, double* var_out) {
    if (G < 1 || G > SEG_MAX_RANKS || rank < 0 || rank >= G) return 1;
    GLayout lay(n, L, MODE_GRAD, gm.phs);
    char* ws = (char*)wsv;
    int* status = (int*)ws;
    double* gconst = (double*)(ws + lay.off_gconst);
    double* phis = (double*)(ws + lay.off_phis);
    double* part = (double*)(ws + lay.off_part);
    double* store = (double*)(ws + lay.off_store);
    const int64_t s0 = first ? 0 : -1;
    GArgs a{gm, t, y, n, L, lay.nc, theta, gconst, phis, status, missing, s0, t_prev};
    const unsigned cgrid = (unsigned)((lay.nc + GGRP - 1) / GGRP);
    const int NRr = (gm.b <= 4) ? 4 : (gm.b <= 8) ? 8 : (gm.b <= 12) ? 12 : 16;
    if (phase == 0) {
        if (cudaMemsetAsync(status, 0, sizeof(int), st) != cudaSuccess) return 1;
        k_gsetup<<<1, 32, 0, st>>>(gm, theta, gconst, status);
        k_gdisc<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(gm, t, y, n, theta, phis, status, missing, s0, t_prev);
        gfold_launch(NRr, gm.eq_nk > 1, cgrid, st, a, (double*)(ws + lay.off_nodes[0]));
        gscan_up(ws, lay.off_nodes, lay.lev_n, lay.nlev, st);
        if (cudaMemcpyAsync(elem_out, ws + lay.off_nodes[lay.nlev], sizeof(double) * GNE * GL,
                            cudaMemcpyDeviceToDevice, st) != cudaSuccess)
            return 1;
    } else {
        // the ranks' tree over the G elements: levels of G, ceil(G/2), .. nodes
        int64_t cnt[8];
        int gl = 0;
        cnt[0] = G;
        while (cnt[gl] > 1) { cnt[gl + 1] = (cnt[gl] + 1) / 2; ++gl; }
        k_gelems_to_soa<<<(unsigned)((G * GNE * GL + 255) / 256), 256, 0, st>>>(
            elems, (double*)(ws + lay.off_seg_nodes[0]), G);
        gscan_up(ws, lay.off_seg_nodes, cnt, gl, st);
        if (gscan_down(ws, lay.off_seg_nodes, lay.off_seg_pre, lay.off_seg_suf, cnt, gl, nullptr, nullptr, st))
            return 1;
        // this rank's entry (value f of lane l at (f * G + rank) * GL + l) as one node
        double* tpre = (double*)(ws + lay.off_seg_top);
        double* tsuf = tpre + GNM * GL;
        const double* gpre = (const double*)(ws + lay.off_seg_pre[0]);
        const double* gsuf = (const double*)(ws + lay.off_seg_suf[0]);
        if (cudaMemcpy2DAsync(tpre, sizeof(double) * GL, gpre + (int64_t)rank * GL, sizeof(double) * GL * G,
                              sizeof(double) * GL, GNM, cudaMemcpyDeviceToDevice, st) != cudaSuccess ||
            cudaMemcpy2DAsync(tsuf, sizeof(double) * GL, gsuf + (int64_t)rank * GL, sizeof(double) * GL * G,
                              sizeof(double) * GL, GNM, cudaMemcpyDeviceToDevice, st) != cudaSuccess)
            return 1;
        if (gscan_down(ws, lay.off_nodes, lay.off_pre, lay.off_suf, lay.lev_n, lay.nlev, tpre, tsuf, st)) return 1;
        const double* pre = (const double*)(ws + lay.off_pre[0]);
        const double* suf = (const double*)(ws + lay.off_suf[0]);
        if (mean_out)
            gchunk_launch<MODE_GRAD_POSTERIOR>(NRr, gm.eq_nk > 1, cgrid, st, a, pre, suf, store, part, mean_out,
                                               var_out);
        else
            gchunk_launch<MODE_GRAD>(NRr, gm.eq_nk > 1, cgrid, st, a, pre, suf, store, part, nullptr, nullptr);
        k_gfinal<<<1, GFIN, 0, st>>>(gm, part, lay.nc, GPART, theta, gconst, ll_out, grad_out);
    }
    return cudaGetLastError() == cudaSuccess ? 0 : 1;
}
int group_elem_size() { return GNE * GL; }
int group_segment_launch_count(int64_t n, int64_t L) {
    GLayout lay(n, L, MODE_GRAD, 4 * GK);
    int gl = 0;
    for (int64_t c = SEG_MAX_RANKS; c > 1; c = (c + 1) / 2) ++gl;
    // phase 0: setup, disc, fold, up levels; phase 1: transpose, the ranks' tree (at most), the range's
    // down levels, chunk, final
    return 3 + lay.nlev + 1 + 2 * gl + lay.nlev + 2;
}

}  // namespace spg
