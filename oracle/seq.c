/*
 * O-seq: the sequential FP64 oracle for state-space temporal GP inference.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing on the product path may link, load or
 * call this file: only the tests, the smoke check and the CPU-baseline leg of
 * the benchmark use it.  It shares no code with the CUDA library.
 *
 * What it computes (all in plain FP64, one series at a time, sequentially):
 *   - the continuous-time state-space model of each covariance family
 *     (Sec. 2.1, Eq. ss1 and the Matern-3/2 example Eq. ss_matern), its
 *     discretisation A_n = expm(F dt_n), Q_n = P0 - A_n P0 A_n^T (Sec. 2.1),
 *     and the exact parameter derivatives of A_n, Q_n, P0;
 *   - the log marginal likelihood (Eq. ml2) by the prediction-error
 *     decomposition of a covariance-form Kalman filter;
 *   - the posterior state moments by the Rauch-Tung-Striebel smoother: the
 *     diagonal blocks (smoothed covariances) and first off-diagonal blocks
 *     (lag-one cross-covariances) of the inverse of the posterior precision
 *     K~ = Kinv + G^T Sigma^-1 G, i.e. the selected inverse of Sec. 3.1
 *     (subproblems 2 and 4), and the posterior mean (subproblem 1);
 *   - the hyperparameter gradient (Sec. 2.4): per transition, the exact
 *     partial derivative of the log-likelihood with respect to A_n and Q_n,
 *     obtained from the filtered moments and a backward information filter
 *     (two-filter form), chained through dA_n/dtheta, dQ_n/dtheta.
 *
 * Conventions (readings of the paper):
 *   - one latent state per observation; the first observed state has the
 *     stationary prior N(0, P0) (the paper's unobserved z_0 with P0 = Pinf
 *     gives the same marginal of y);
 *   - A_n maps the state at t_n to the state at t_{n+1};
 *   - the noise parameter is the variance sigma_n^2; gradients are taken with
 *     respect to the raw parameters (lengthscales, variances, period);
 *   - the latent variance H P^s H^T is reported (no noise added);
 *   - a NaN observation is missing: infinite noise there, so the state is
 *     predicted but not updated (the augmented formulation of Eqs. mean4-mean6:
 *     test points carry Sigma' = infinity and y' = 0).
 *
 * Covariance families (parameter order in theta, noise variance last):
 *   1 Matern-1/2 (b=1), 2 Matern-3/2 (b=2), 3 Matern-5/2 (b=3):
 *       (lengthscale, variance); F is the companion matrix of (s+lam)^b with
 *       lam = sqrt(2b-1)/lengthscale, H = e_1^T, P0 from the derivatives of
 *       the covariance function at zero lag.
 *   4 periodic of order J (b = 2(J+1)): (variance, lengthscale, period); the
 *       cosine series of exp(-2 sin^2(w t/2)/l^2) truncated at harmonic J,
 *       each harmonic a noiseless rotation (Solin & Sarkka 2014).
 *   5 quasi-periodic: periodic(J) times a unit-variance Matern envelope of
 *       kind env (Kronecker product of the two state spaces):
 *       (variance, lengthscale, period, envelope lengthscale).
 *   6 exponentiated quadratic, state-space approximation of even order N
 *       (b = N): (lengthscale, variance).  The spectral density
 *       s sqrt(2 pi) l exp(-l^2 w^2/2) with exp(l^2 w^2/2) replaced by its
 *       Taylor polynomial of order N in l^2 w^2/2 is rational; its stable
 *       spectral factor gives the SDE f^(N) + a_{N-1} f^(N-1) + ... + a_0 f =
 *       white noise of spectral density q_c (Hartikainen & Sarkka 2010):
 *       F the companion matrix of s^N + a_{N-1} s^{N-1} + ... + a_0, whose
 *       roots are the left-half-plane roots of sum_n (-s^2 l^2/2)^n / n!,
 *       q_c = s sqrt(2 pi) l 2^N N! / l^(2N), H = e_1^T, Pinf from the
 *       Lyapunov equation F P + P F^T + q_c e_N e_N^T = 0.
 *   Sums of components stack block-diagonally and concatenate H.
 */
#include <complex.h>
#include <math.h>
#include <stdlib.h>
#include <string.h>
#undef I   /* complex.h's imaginary unit macro; _Complex_I is used instead */

#ifndef M_PI
#define M_PI 3.14159265358979323846
#endif

#define OMAXB 32
#define OMAXC 8
#define OMAXP 24
#define OB2 (OMAXB * OMAXB)

enum { OK = 0, E_INVAL = 1, E_NOTSORTED = 2, E_NONFINITE = 3, E_NUMERIC = 4, E_NOMEM = 7 };

typedef struct {
    int ncomp;
    int kind[OMAXC], order[OMAXC], env[OMAXC];
    int off[OMAXC], bc[OMAXC], poff[OMAXC], np[OMAXC];
    int b, P;
} om_t;

/* ---------------------------------------------------------------- small dense linear algebra (row-major) */

static void mzero(int n, double* A) { memset(A, 0, sizeof(double) * n * n); }
static void meye(int n, double* A) { mzero(n, A); for (int i = 0; i < n; ++i) A[i * n + i] = 1.0; }
static void mcopy(int n, const double* A, double* B) { memcpy(B, A, sizeof(double) * n * n); }

/* C = A B */
static void mm(int n, const double* A, const double* B, double* C) {
    double T[OB2];
    for (int i = 0; i < n; ++i)
        for (int j = 0; j < n; ++j) {
            double s = 0.0;
            for (int k = 0; k < n; ++k) s += A[i * n + k] * B[k * n + j];
            T[i * n + j] = s;
        }
    mcopy(n, T, C);
}
/* C = A B^T */
static void mmt(int n, const double* A, const double* B, double* C) {
    double T[OB2];
    for (int i = 0; i < n; ++i)
        for (int j = 0; j < n; ++j) {
            double s = 0.0;
            for (int k = 0; k < n; ++k) s += A[i * n + k] * B[j * n + k];
            T[i * n + j] = s;
        }
    mcopy(n, T, C);
}
/* C = A^T B */
static void mtm(int n, const double* A, const double* B, double* C) {
    double T[OB2];
    for (int i = 0; i < n; ++i)
        for (int j = 0; j < n; ++j) {
            double s = 0.0;
            for (int k = 0; k < n; ++k) s += A[k * n + i] * B[k * n + j];
            T[i * n + j] = s;
        }
    mcopy(n, T, C);
}
static void mv(int n, const double* A, const double* x, double* y) {
    double t[OMAXB];
    for (int i = 0; i < n; ++i) { double s = 0.0; for (int k = 0; k < n; ++k) s += A[i * n + k] * x[k]; t[i] = s; }
    memcpy(y, t, sizeof(double) * n);
}
static void mtv(int n, const double* A, const double* x, double* y) {
    double t[OMAXB];
    for (int i = 0; i < n; ++i) { double s = 0.0; for (int k = 0; k < n; ++k) s += A[k * n + i] * x[k]; t[i] = s; }
    memcpy(y, t, sizeof(double) * n);
}
static void msym(int n, double* A) {
    for (int i = 0; i < n; ++i)
        for (int j = i + 1; j < n; ++j) { double s = 0.5 * (A[i * n + j] + A[j * n + i]); A[i * n + j] = s; A[j * n + i] = s; }
}
static double mdot(int n, const double* A, const double* B) { /* <A,B> = sum A_ij B_ij */
    double s = 0.0;
    for (int i = 0; i < n * n; ++i) s += A[i] * B[i];
    return s;
}
/* Solve M X = B for X (n x m), Gaussian elimination with partial pivoting.
   Returns 0, or -1 if a pivot is exactly zero. */
static int lu_solve(int n, const double* M, const double* B, int m, double* X) {
    double a[OB2], x[OMAXB * (OMAXB + 1)];
    memcpy(a, M, sizeof(double) * n * n);
    memcpy(x, B, sizeof(double) * n * m);
    for (int k = 0; k < n; ++k) {
        int p = k; double best = fabs(a[k * n + k]);
        for (int i = k + 1; i < n; ++i) if (fabs(a[i * n + k]) > best) { best = fabs(a[i * n + k]); p = i; }
        if (best == 0.0) return -1;
        if (p != k) {
            for (int j = 0; j < n; ++j) { double t = a[k * n + j]; a[k * n + j] = a[p * n + j]; a[p * n + j] = t; }
            for (int j = 0; j < m; ++j) { double t = x[k * m + j]; x[k * m + j] = x[p * m + j]; x[p * m + j] = t; }
        }
        for (int i = k + 1; i < n; ++i) {
            double f = a[i * n + k] / a[k * n + k];
            if (f == 0.0) continue;
            for (int j = k; j < n; ++j) a[i * n + j] -= f * a[k * n + j];
            for (int j = 0; j < m; ++j) x[i * m + j] -= f * x[k * m + j];
        }
    }
    for (int k = n - 1; k >= 0; --k)
        for (int j = 0; j < m; ++j) {
            double s = x[k * m + j];
            for (int i = k + 1; i < n; ++i) s -= a[k * n + i] * x[i * m + j];
            x[k * m + j] = s / a[k * n + k];
        }
    memcpy(X, x, sizeof(double) * n * m);
    return 0;
}

/* ---------------------------------------------------------------- model set-up */

static int matern_b(int kind) { return kind; } /* kinds 1,2,3 have b = 1,2,3 */

static int om_init(om_t* om, int ncomp, const int* kind, const int* order, const int* env) {
    if (ncomp < 1 || ncomp > OMAXC) return E_INVAL;
    om->ncomp = ncomp;
    int b = 0, P = 0;
    for (int c = 0; c < ncomp; ++c) {
        om->kind[c] = kind[c];
        om->order[c] = order ? order[c] : 0;
        om->env[c] = env ? env[c] : 0;
        int bc, np;
        switch (kind[c]) {
        case 1: case 2: case 3: bc = matern_b(kind[c]); np = 2; break;
        case 4: if (om->order[c] < 0) return E_INVAL; bc = 2 * (om->order[c] + 1); np = 3; break;
        case 5:
            if (om->order[c] < 0 || om->env[c] < 1 || om->env[c] > 3) return E_INVAL;
            bc = 2 * (om->order[c] + 1) * matern_b(om->env[c]); np = 4; break;
        case 6:
            if (om->order[c] < 2 || om->order[c] % 2 || om->order[c] > 16) return E_INVAL;
            bc = om->order[c]; np = 2; break;
        default: return E_INVAL;
        }
        om->off[c] = b; om->bc[c] = bc; om->poff[c] = P; om->np[c] = np;
        b += bc; P += np;
    }
    P += 1; /* noise variance */
    if (b > OMAXB || P > OMAXP) return E_INVAL;
    om->b = b; om->P = P;
    return OK;
}

/* Matern family in the paper's coordinates (state = f and its derivatives). */
static double binom(int n, int k) { double r = 1.0; for (int i = 1; i <= k; ++i) r = r * (n - k + i) / i; return r; }

/* F = companion matrix of (s+lam)^b and Fl = dF/dlam. */
static void matern_F(int b, double lam, double* F, double* Fl) {
    mzero(b, F); mzero(b, Fl);
    for (int i = 0; i + 1 < b; ++i) F[i * b + i + 1] = 1.0;
    for (int j = 0; j < b; ++j) {
        double c = binom(b, j);
        F[(b - 1) * b + j] = -c * pow(lam, b - j);
        Fl[(b - 1) * b + j] = -c * (b - j) * pow(lam, b - j - 1);
    }
}

/* Stationary covariance with unit variance, from the covariance function's
   derivatives at zero lag: Cov(f^(i), f^(j)) = (-1)^j k^(i+j)(0). */
static void matern_Pu(int b, double lam, double* Pu, double* dPu) {
    mzero(b, Pu); mzero(b, dPu);
    if (b == 1) { Pu[0] = 1.0; }
    else if (b == 2) { Pu[0] = 1.0; Pu[3] = lam * lam; dPu[3] = 2.0 * lam; }
    else { /* b == 3: k = (1 + r + r^2/3) e^-r = 1 - lam^2 t^2/6 + lam^4 t^4/24 + ... */
        double l2 = lam * lam;
        Pu[0] = 1.0;
        Pu[2] = Pu[6] = -l2 / 3.0; dPu[2] = dPu[6] = -2.0 * lam / 3.0;
        Pu[4] = l2 / 3.0; dPu[4] = 2.0 * lam / 3.0;
        Pu[8] = l2 * l2; dPu[8] = 4.0 * l2 * lam;
    }
}

/* Spectral density constant q_c of the white noise driving the Matern SDE,
   q_c = 2 sqrt(pi) lam^(2 nu) Gamma(nu + 1/2) / Gamma(nu), unit variance. */
static double matern_qc(int b, double lam) {
    double nu = b - 0.5;
    return 2.0 * sqrt(M_PI) * pow(lam, 2.0 * nu) * tgamma(nu + 0.5) / tgamma(nu);
}

/* expm(F dt) and d expm(F dt)/dlam for the Matern companion F.  F + lam I is
   nilpotent (its characteristic polynomial is s^b), so the exponential is the
   finite series exp(-lam dt) sum_{k<b} ((F+lam I) dt)^k / k!.  The derivative is
   the upper-right block of the exponential of [[F, Fl],[0, F]] dt (Van Loan
   1978), whose shifted matrix is nilpotent of order 2b. */
static void matern_expm(int b, double lam, double dt, double* A, double* dAl) {
    double F[OB2], Fl[OB2];
    matern_F(b, lam, F, Fl);
    int m = 2 * b;
    double M[4 * OMAXB * OMAXB], T[4 * OMAXB * OMAXB], S[4 * OMAXB * OMAXB], U[4 * OMAXB * OMAXB];
    memset(M, 0, sizeof(double) * m * m);
    for (int i = 0; i < b; ++i)
        for (int j = 0; j < b; ++j) {
            M[i * m + j] = F[i * b + j] * dt;
            M[(i + b) * m + (j + b)] = F[i * b + j] * dt;
            M[i * m + (j + b)] = Fl[i * b + j] * dt;
        }
    for (int i = 0; i < m; ++i) M[i * m + i] += lam * dt;
    /* S = sum_{k<m} M^k / k!,  T = M^k / k! */
    memset(S, 0, sizeof(double) * m * m);
    memset(T, 0, sizeof(double) * m * m);
    for (int i = 0; i < m; ++i) { S[i * m + i] = 1.0; T[i * m + i] = 1.0; }
    for (int k = 1; k < m; ++k) {
        for (int i = 0; i < m; ++i)
            for (int j = 0; j < m; ++j) {
                double s = 0.0;
                for (int l = 0; l < m; ++l) s += T[i * m + l] * M[l * m + j];
                U[i * m + j] = s / k;
            }
        memcpy(T, U, sizeof(double) * m * m);
        for (int i = 0; i < m * m; ++i) S[i] += T[i];
    }
    double e = exp(-lam * dt);
    for (int i = 0; i < b; ++i)
        for (int j = 0; j < b; ++j) {
            A[i * b + j] = e * S[i * m + j];
            if (dAl) dAl[i * b + j] = e * S[i * m + (j + b)];
        }
    /* exp([[F,Fl],[0,F]] dt) has upper-right block d/dlam expm(F dt) itself; the
       factor exp(-lam dt) is exact for the whole block matrix because lam*dt*I
       commutes with it, so the shift needs no separate derivative term. */
}

/* ---------------------------------------------------------------- general matrix exponential */

static double mnorm1(int n, const double* A) {
    double best = 0.0;
    for (int j = 0; j < n; ++j) {
        double s = 0.0;
        for (int i = 0; i < n; ++i) s += fabs(A[i * n + j]);
        if (s > best) best = s;
    }
    return best;
}

/* expm(M) by scaling and squaring: M / 2^s has 1-norm <= 1/4, its Taylor
   series is summed until the terms vanish against the sum, then squared s
   times.  n <= 2 OMAXB. */
static void expm_taylor(int n, const double* M, double* E) {
    double nrm = mnorm1(n, M);
    int sq = 0;
    while (nrm > 0.25) { nrm *= 0.5; ++sq; }
    double scale = ldexp(1.0, -sq);
    static _Thread_local double T[4 * OB2], U[4 * OB2], Ms[4 * OB2];   /* per thread: callers may run in parallel */
    for (int i = 0; i < n * n; ++i) Ms[i] = M[i] * scale;
    meye(n, E);
    meye(n, T);
    for (int k = 1; k < 60; ++k) {
        mm(n, T, Ms, U);
        double tn = 0.0, en = 0.0;
        for (int i = 0; i < n * n; ++i) { T[i] = U[i] / k; E[i] += T[i]; tn += fabs(T[i]); en += fabs(E[i]); }
        if (tn <= 1e-20 * en) break;
    }
    for (int r = 0; r < sq; ++r) {
        mm(n, E, E, U);
        mcopy(n, U, E);
    }
}

/* ---------------------------------------------------------------- exponentiated quadratic (order N) */

/* Left-half-plane roots of sum_{n<=N} (-s^2/2)^n / n! (l = 1).  As a
   polynomial in w = s^2 it has degree N; its roots w_j (Durand-Kerner
   iteration, then Newton polishing) give the stable roots s_j = -sqrt(w_j). */
static void eq_roots(int N, double complex* sr) {
    double complex cf[17];                       /* monic coefficients in w, cf[N] = 1 */
    double fact = 1.0;
    for (int n = 1; n <= N; ++n) fact *= n;
    /* sum (-1/2)^n w^n / n!  divided by its leading coefficient (-1/2)^N / N! */
    double lead = pow(-0.5, N) / fact, f = 1.0;
    for (int n = 0; n <= N; ++n) {
        if (n > 0) f *= n;
        cf[n] = (pow(-0.5, n) / f) / lead;
    }
    double complex w[16];
    double rad = 1.0;
    for (int n = 0; n < N; ++n) { double a = cabs(cf[n]); if (pow(a, 1.0 / (N - n)) > rad) rad = pow(a, 1.0 / (N - n)); }
    for (int j = 0; j < N; ++j) w[j] = rad * cpow(0.4 + 0.9 * _Complex_I, j);
    for (int it = 0; it < 5000; ++it) {
        double moved = 0.0;
        for (int j = 0; j < N; ++j) {
            double complex pv = 1.0;   /* monic: evaluate by Horner */
            pv = cf[N];
            for (int n = N - 1; n >= 0; --n) pv = pv * w[j] + cf[n];
            double complex den = 1.0;
            for (int k = 0; k < N; ++k) if (k != j) den *= (w[j] - w[k]);
            double complex d = pv / den;
            w[j] -= d;
            if (cabs(d) > moved * cabs(w[j]) / (cabs(w[j]) + 1e-300)) moved = cabs(d) / (cabs(w[j]) + 1e-300);
        }
        if (moved < 1e-15) break;
    }
    for (int j = 0; j < N; ++j) {
        for (int it = 0; it < 4; ++it) {     /* Newton polishing on the monic polynomial */
            double complex pv = cf[N], dv = 0.0;
            for (int n = N - 1; n >= 0; --n) { dv = dv * w[j] + pv; pv = pv * w[j] + cf[n]; }
            if (cabs(dv) == 0.0) break;
            w[j] -= pv / dv;
        }
        sr[j] = -csqrt(w[j]);
        if (creal(sr[j]) > 0.0) sr[j] = -sr[j];
    }
}

/* Monic stable factor s^N + a_{N-1} s^{N-1} + ... + a_0 (l = 1): coefficients a[0..N-1]. */
static void eq_factor(int N, double* a) {
    double complex sr[16], c[17];
    eq_roots(N, sr);
    c[0] = 1.0;
    for (int k = 1; k <= N; ++k) c[k] = 0.0;
    for (int j = 0; j < N; ++j)            /* multiply by (s - s_j); c[k] = coefficient of s^k */
        for (int k = j + 1; k >= 0; --k) c[k] = (k > 0 ? c[k - 1] : 0.0) - sr[j] * c[k];
    for (int k = 0; k < N; ++k) a[k] = creal(c[k]);
}

/* F (companion) for lengthscale l and dF/dl: a_k(l) = a_k(1) l^(k-N). */
static void eq_F(int N, const double* a1, double ell, double* F, double* Fl) {
    mzero(N, F); if (Fl) mzero(N, Fl);
    for (int i = 0; i + 1 < N; ++i) F[i * N + i + 1] = 1.0;
    for (int k = 0; k < N; ++k) {
        F[(N - 1) * N + k] = -a1[k] * pow(ell, k - N);
        if (Fl) Fl[(N - 1) * N + k] = -a1[k] * (k - N) * pow(ell, k - N - 1);
    }
}

/* Unit-variance stationary covariance at l = 1, from the Lyapunov equation
   F1 P + P F1^T + q1 e_N e_N^T = 0, q1 = sqrt(2 pi) 2^N N!, solved as the
   linear system (I (x) F1 + F1 (x) I) vec P = -q1 vec(e_N e_N^T). */
static int eq_P1(int N, const double* a1, double* P1) {
    double F1[OB2];
    eq_F(N, a1, 1.0, F1, NULL);
    int m = N * N;
    double* K = (double*)calloc((size_t)m * m, sizeof(double));
    double* rhs = (double*)calloc((size_t)m, sizeof(double));
    double* x = (double*)calloc((size_t)m, sizeof(double));
    if (!K || !rhs || !x) { free(K); free(rhs); free(x); return E_NOMEM; }
    for (int i = 0; i < N; ++i)
        for (int j = 0; j < N; ++j) {
            int r = i * N + j;   /* equation for entry (i, j): sum_k F[i][k] P[k][j] + P[i][k] F[j][k] */
            for (int k = 0; k < N; ++k) {
                K[(size_t)r * m + k * N + j] += F1[i * N + k];
                K[(size_t)r * m + i * N + k] += F1[j * N + k];
            }
        }
    double fact = 1.0;
    for (int n = 1; n <= N; ++n) fact *= n;
    rhs[(N - 1) * N + (N - 1)] = -sqrt(2.0 * M_PI) * pow(2.0, N) * fact;
    /* Gaussian elimination with partial pivoting on the m x m system (in place) */
    int st = OK;
    for (int k = 0; k < m && st == OK; ++k) {
        int p = k;
        double best = fabs(K[(size_t)k * m + k]);
        for (int i = k + 1; i < m; ++i)
            if (fabs(K[(size_t)i * m + k]) > best) { best = fabs(K[(size_t)i * m + k]); p = i; }
        if (best == 0.0) { st = E_NUMERIC; break; }
        if (p != k) {
            for (int j = 0; j < m; ++j) { double u = K[(size_t)k * m + j]; K[(size_t)k * m + j] = K[(size_t)p * m + j]; K[(size_t)p * m + j] = u; }
            double u = rhs[k]; rhs[k] = rhs[p]; rhs[p] = u;
        }
        for (int i = k + 1; i < m; ++i) {
            double f = K[(size_t)i * m + k] / K[(size_t)k * m + k];
            if (f == 0.0) continue;
            for (int j = k; j < m; ++j) K[(size_t)i * m + j] -= f * K[(size_t)k * m + j];
            rhs[i] -= f * rhs[k];
        }
    }
    for (int k = m - 1; k >= 0 && st == OK; --k) {
        double v = rhs[k];
        for (int j = k + 1; j < m; ++j) v -= K[(size_t)k * m + j] * x[j];
        x[k] = v / K[(size_t)k * m + k];
    }
    for (int i = 0; i < m; ++i) P1[i] = x[i];
    msym(N, P1);
    free(K); free(rhs); free(x);
    return st;
}

/* Modified Bessel function of the first kind I_j(x), by its power series
   sum_k (x/2)^(2k+j) / (k! (k+j)!). */
static double bessel_i(int j, double x) {
    double h = 0.5 * x, term = 1.0;
    for (int i = 1; i <= j; ++i) term *= h / i;
    double s = term;
    for (int k = 1; k < 2000; ++k) {
        term *= h * h / ((double)k * (double)(k + j));
        s += term;
        if (term < 1e-18 * s) break;
    }
    return s;
}

/* periodic component: harmonic weights q_j^2 = var * c_j * e^-x I_j(x), x = 1/l^2,
   and their derivative with respect to l. */
static void periodic_weights(int J, double var, double lp, double* q2, double* dq2_dl, double* q2u) {
    double x = 1.0 / (lp * lp), dx = -2.0 / (lp * lp * lp), ex = exp(-x);
    for (int j = 0; j <= J; ++j) {
        double c = (j == 0) ? 1.0 : 2.0;
        double Ij = bessel_i(j, x);
        double dIj = 0.5 * (bessel_i(j == 0 ? 1 : j - 1, x) + bessel_i(j + 1, x));
        q2u[j] = c * ex * Ij;
        q2[j] = var * q2u[j];
        dq2_dl[j] = var * c * ex * (dIj - Ij) * dx;
    }
}

/* Pinf (b x b) and dPinf/dtheta_p for all parameters p (P x b x b). */
static void om_pinf(const om_t* om, const double* th, double* Pinf, double* dPinf) {
    int b = om->b;
    memset(Pinf, 0, sizeof(double) * b * b);
    if (dPinf) memset(dPinf, 0, sizeof(double) * om->P * b * b);
    for (int c = 0; c < om->ncomp; ++c) {
        int o = om->off[c], po = om->poff[c], k = om->kind[c];
        if (k <= 3) {
            int bc = matern_b(k);
            double ell = th[po], var = th[po + 1], lam = sqrt(2.0 * bc - 1.0) / ell, dlam = -lam / ell;
            double Pu[9], dPu[9];
            matern_Pu(bc, lam, Pu, dPu);
            for (int i = 0; i < bc; ++i)
                for (int j = 0; j < bc; ++j) {
                    Pinf[(o + i) * b + o + j] = var * Pu[i * bc + j];
                    if (dPinf) {
                        dPinf[(size_t)(po + 0) * b * b + (o + i) * b + o + j] = var * dPu[i * bc + j] * dlam;
                        dPinf[(size_t)(po + 1) * b * b + (o + i) * b + o + j] = Pu[i * bc + j];
                    }
                }
        } else if (k == 6) {
            int N = om->order[c];
            double a1[16], P1[OB2];
            eq_factor(N, a1);
            eq_P1(N, a1, P1);
            double ell = th[po], var = th[po + 1];
            /* Pinf = var D P1 D with D = diag(l^-i): the scaling z = D z~ of time by l */
            for (int i = 0; i < N; ++i)
                for (int j = 0; j < N; ++j) {
                    double dij = pow(ell, -(i + j));
                    Pinf[(o + i) * b + o + j] = var * dij * P1[i * N + j];
                    if (dPinf) {
                        dPinf[(size_t)(po + 0) * b * b + (o + i) * b + o + j] = var * P1[i * N + j] * (-(i + j)) * dij / ell;
                        dPinf[(size_t)(po + 1) * b * b + (o + i) * b + o + j] = dij * P1[i * N + j];
                    }
                }
        } else {
            int J = om->order[c];
            double q2[64], dq2[64], q2u[64];
            double var = th[po], lp = th[po + 1];
            periodic_weights(J, var, lp, q2, dq2, q2u);
            int be = (k == 5) ? matern_b(om->env[c]) : 1;
            double Pe[9] = {1, 0, 0, 0, 0, 0, 0, 0, 0}, dPe[9] = {0};
            if (k == 5) {
                double lam = sqrt(2.0 * be - 1.0) / th[po + 3], dlam = -lam / th[po + 3];
                matern_Pu(be, lam, Pe, dPe);
                for (int i = 0; i < be * be; ++i) dPe[i] *= dlam;
            }
            for (int j = 0; j <= J; ++j)
                for (int r = 0; r < 2; ++r)
                    for (int ei = 0; ei < be; ++ei)
                        for (int ej = 0; ej < be; ++ej) {
                            int ii = o + (2 * j + r) * be + ei, jj = o + (2 * j + r) * be + ej;
                            Pinf[ii * b + jj] = q2[j] * Pe[ei * be + ej];
                            if (dPinf) {
                                dPinf[(size_t)(po + 0) * b * b + ii * b + jj] = q2u[j] * Pe[ei * be + ej];
                                dPinf[(size_t)(po + 1) * b * b + ii * b + jj] = dq2[j] * Pe[ei * be + ej];
                                if (k == 5) dPinf[(size_t)(po + 3) * b * b + ii * b + jj] = q2[j] * dPe[ei * be + ej];
                            }
                        }
        }
    }
}

/* A = expm(F dt) and dA/dtheta_p (P x b x b). */
static void om_transition(const om_t* om, const double* th, double dt, double* A, double* dA) {
    int b = om->b;
    memset(A, 0, sizeof(double) * b * b);
    if (dA) memset(dA, 0, sizeof(double) * om->P * b * b);
    for (int c = 0; c < om->ncomp; ++c) {
        int o = om->off[c], po = om->poff[c], k = om->kind[c];
        if (k <= 3) {
            int bc = matern_b(k);
            double ell = th[po], lam = sqrt(2.0 * bc - 1.0) / ell, dlam = -lam / ell;
            double Ac[9], dAc[9];
            matern_expm(bc, lam, dt, Ac, dAc);
            for (int i = 0; i < bc; ++i)
                for (int j = 0; j < bc; ++j) {
                    A[(o + i) * b + o + j] = Ac[i * bc + j];
                    if (dA) dA[(size_t)po * b * b + (o + i) * b + o + j] = dAc[i * bc + j] * dlam;
                }
        } else if (k == 6) {
            /* expm(F dt) and its l-derivative: the upper-right block of
               expm([[F, Fl], [0, F]] dt) (Van Loan 1978) */
            int N = om->order[c], m = 2 * N;
            double a1[16], F[OB2], Fl[OB2];
            static _Thread_local double M[4 * OB2], E[4 * OB2];
            eq_factor(N, a1);
            eq_F(N, a1, th[po], F, Fl);
            memset(M, 0, sizeof(double) * m * m);
            for (int i = 0; i < N; ++i)
                for (int j = 0; j < N; ++j) {
                    M[i * m + j] = F[i * N + j] * dt;
                    M[(i + N) * m + (j + N)] = F[i * N + j] * dt;
                    M[i * m + (j + N)] = Fl[i * N + j] * dt;
                }
            expm_taylor(m, M, E);
            for (int i = 0; i < N; ++i)
                for (int j = 0; j < N; ++j) {
                    A[(o + i) * b + o + j] = E[i * m + j];
                    if (dA) dA[(size_t)po * b * b + (o + i) * b + o + j] = E[i * m + (j + N)];
                }
        } else {
            int J = om->order[c];
            double per = th[po + 2], w = 2.0 * M_PI / per, dw = -2.0 * M_PI / (per * per);
            int be = (k == 5) ? matern_b(om->env[c]) : 1;
            double Ae[9] = {1, 0, 0, 0, 0, 0, 0, 0, 0}, dAe[9] = {0};
            if (k == 5) {
                double lam = sqrt(2.0 * be - 1.0) / th[po + 3], dlam = -lam / th[po + 3];
                matern_expm(be, lam, dt, Ae, dAe);
                for (int i = 0; i < be * be; ++i) dAe[i] *= dlam;
            }
            for (int j = 0; j <= J; ++j) {
                double ang = j * w * dt, cs = cos(ang), sn = sin(ang);
                /* expm([[0,-jw],[jw,0]] dt) is the rotation by j w dt */
                double R[4] = {cs, -sn, sn, cs};
                double dR[4] = {-sn * j * dt * dw, -cs * j * dt * dw, cs * j * dt * dw, -sn * j * dt * dw};
                for (int r = 0; r < 2; ++r)
                    for (int s = 0; s < 2; ++s)
                        for (int ei = 0; ei < be; ++ei)
                            for (int ej = 0; ej < be; ++ej) {
                                int ii = o + (2 * j + r) * be + ei, jj = o + (2 * j + s) * be + ej;
                                A[ii * b + jj] = R[r * 2 + s] * Ae[ei * be + ej];
                                if (dA) {
                                    dA[(size_t)(po + 2) * b * b + ii * b + jj] = dR[r * 2 + s] * Ae[ei * be + ej];
                                    if (k == 5) dA[(size_t)(po + 3) * b * b + ii * b + jj] = R[r * 2 + s] * dAe[ei * be + ej];
                                }
                            }
            }
        }
    }
}

static void om_H(const om_t* om, double* H) {
    memset(H, 0, sizeof(double) * om->b);
    for (int c = 0; c < om->ncomp; ++c) {
        int o = om->off[c], k = om->kind[c];
        if (k <= 3 || k == 6) H[o] = 1.0;
        else {
            int be = (k == 5) ? matern_b(om->env[c]) : 1;
            for (int j = 0; j <= om->order[c]; ++j) H[o + 2 * j * be] = 1.0;
        }
    }
}

/* Q = Pinf - A Pinf A^T (Sec. 2.1), symmetrised, and its derivatives
   dQ = dPinf - dA Pinf A^T - A dPinf A^T - A Pinf dA^T. */
static void om_Q(const om_t* om, const double* A, const double* Pinf, const double* dA, const double* dPinf,
                 double* Q, double* dQ) {
    int b = om->b;
    double T[OB2], U[OB2];
    mm(b, A, Pinf, T);
    mmt(b, T, A, U);
    for (int i = 0; i < b * b; ++i) Q[i] = Pinf[i] - U[i];
    msym(b, Q);
    if (!dQ) return;
    for (int p = 0; p < om->P; ++p) {
        const double* dAp = dA + (size_t)p * b * b;
        const double* dPp = dPinf + (size_t)p * b * b;
        double* dQp = dQ + (size_t)p * b * b;
        double X[OB2], Y[OB2];
        mm(b, dAp, Pinf, X); mmt(b, X, A, Y);          /* dA Pinf A^T */
        for (int i = 0; i < b * b; ++i) dQp[i] = dPp[i] - Y[i];
        mm(b, A, dPp, X); mmt(b, X, A, Y);             /* A dPinf A^T */
        for (int i = 0; i < b * b; ++i) dQp[i] -= Y[i];
        mm(b, A, Pinf, X); mmt(b, X, dAp, Y);          /* A Pinf dA^T */
        for (int i = 0; i < b * b; ++i) dQp[i] -= Y[i];
    }
}

static int check_inputs(const double* th, int P, const double* t, const double* y, long n) {
    if (n < 1) return E_INVAL;
    for (int p = 0; p < P; ++p) if (!(th[p] > 0.0) || !isfinite(th[p])) return E_INVAL;
    for (long i = 0; i < n; ++i) {
        /* a NaN observation is a missing one (a test point); infinities are errors */
        if (!isfinite(t[i]) || (y && isinf(y[i]))) return E_NONFINITE;
        if (i > 0 && t[i] < t[i - 1]) return E_NOTSORTED;
    }
    return OK;
}

/* ---------------------------------------------------------------- exported: model pieces (for the pins) */

/* The monic stable factor of the order-N approximation at l = 1 (pins). */
int oseq_eq_factor(int N, double* a) {
    if (N < 2 || N % 2 || N > 16 || !a) return E_INVAL;
    eq_factor(N, a);
    return OK;
}

int oseq_dims(int ncomp, const int* kind, const int* order, const int* env, int* b, int* P) {
    om_t om; int st = om_init(&om, ncomp, kind, order, env);
    if (st) return st;
    *b = om.b; *P = om.P;
    return OK;
}

/* Continuous model: F (b x b), Pinf, H (b), Lq = L q_c L^T (b x b). */
int oseq_continuous(int ncomp, const int* kind, const int* order, const int* env, const double* th,
                    double* F, double* Pinf, double* H, double* Lq) {
    om_t om; int st = om_init(&om, ncomp, kind, order, env);
    if (st) return st;
    int b = om.b;
    memset(F, 0, sizeof(double) * b * b);
    memset(Lq, 0, sizeof(double) * b * b);
    om_pinf(&om, th, Pinf, NULL);
    om_H(&om, H);
    for (int c = 0; c < om.ncomp; ++c) {
        int o = om.off[c], po = om.poff[c], k = om.kind[c];
        if (k <= 3) {
            int bc = matern_b(k);
            double lam = sqrt(2.0 * bc - 1.0) / th[po], Fc[9], Fl[9];
            matern_F(bc, lam, Fc, Fl);
            for (int i = 0; i < bc; ++i) for (int j = 0; j < bc; ++j) F[(o + i) * b + o + j] = Fc[i * bc + j];
            Lq[(o + bc - 1) * b + o + bc - 1] = th[po + 1] * matern_qc(bc, lam);
        } else if (k == 6) {
            int N = om.order[c];
            double a1[16], Fc[OB2], fact = 1.0, ell = th[po];
            eq_factor(N, a1);
            eq_F(N, a1, ell, Fc, NULL);
            for (int i = 0; i < N; ++i) for (int j = 0; j < N; ++j) F[(o + i) * b + o + j] = Fc[i * N + j];
            for (int n = 1; n <= N; ++n) fact *= n;
            Lq[(o + N - 1) * b + o + N - 1] = th[po + 1] * sqrt(2.0 * M_PI) * ell * pow(2.0, N) * fact / pow(ell, 2 * N);
        } else {
            int J = om.order[c];
            double w = 2.0 * M_PI / th[po + 2];
            int be = (k == 5) ? matern_b(om.env[c]) : 1;
            double Fe[9] = {0}, Fl[9], q2[64], dq2[64], q2u[64], qce = 0.0;
            if (k == 5) { double lam = sqrt(2.0 * be - 1.0) / th[po + 3]; matern_F(be, lam, Fe, Fl); qce = matern_qc(be, lam); }
            periodic_weights(J, th[po], th[po + 1], q2, dq2, q2u);
            for (int j = 0; j <= J; ++j) {
                double R[4] = {0.0, -j * w, j * w, 0.0};
                for (int r = 0; r < 2; ++r)
                    for (int s = 0; s < 2; ++s)
                        for (int e = 0; e < be; ++e) {
                            int ii = o + (2 * j + r) * be + e, jj = o + (2 * j + s) * be + e;
                            F[ii * b + jj] += R[r * 2 + s];       /* F_per (x) I */
                        }
                for (int r = 0; r < 2; ++r) {
                    for (int ei = 0; ei < be; ++ei)
                        for (int ej = 0; ej < be; ++ej) {
                            int ii = o + (2 * j + r) * be + ei, jj = o + (2 * j + r) * be + ej;
                            F[ii * b + jj] += Fe[ei * be + ej];    /* I (x) F_env */
                        }
                    if (k == 5) {
                        int ii = o + (2 * j + r) * be + be - 1;
                        Lq[ii * b + ii] = q2[j] * qce;             /* Pinf_per (x) Lq_env */
                    }
                }
            }
        }
    }
    return OK;
}

/* A, Q for one gap dt, plus dA, dQ, Pinf, dPinf (each P x b x b, may be NULL). */
int oseq_discretize(int ncomp, const int* kind, const int* order, const int* env, const double* th, double dt,
                    double* A, double* Q, double* dA, double* dQ, double* Pinf, double* dPinf) {
    om_t om; int st = om_init(&om, ncomp, kind, order, env);
    if (st) return st;
    int b = om.b;
    double Pi[OB2];
    double* dPi = (double*)malloc(sizeof(double) * om.P * b * b);
    double* dAl = (double*)malloc(sizeof(double) * om.P * b * b);
    om_pinf(&om, th, Pi, dPi);
    om_transition(&om, th, dt, A, dAl);
    om_Q(&om, A, Pi, dAl, dPi, Q, dQ);
    if (dA) memcpy(dA, dAl, sizeof(double) * om.P * b * b);
    if (Pinf) memcpy(Pinf, Pi, sizeof(double) * b * b);
    if (dPinf) memcpy(dPinf, dPi, sizeof(double) * om.P * b * b);
    free(dPi); free(dAl);
    return OK;
}

/* ---------------------------------------------------------------- Kalman filter (log-likelihood) */

/* Forward pass.  Stores filtered m (n x b) and P (n x b x b) when the
   pointers are non-NULL.  Returns the log-likelihood in *ll. */
static int kf_forward(const om_t* om, const double* th, const double* t, const double* y, long n,
                      double* ll, double* mf, double* Pf) {
    int b = om->b;
    double s2 = th[om->P - 1];
    double Pinf[OB2], H[OMAXB], A[OB2], Q[OB2], m[OMAXB], P[OB2], mb[OMAXB], Pb[OB2], T[OB2], K[OMAXB];
    om_pinf(om, th, Pinf, NULL);
    om_H(om, H);
    double acc = 0.0;
    for (long i = 0; i < n; ++i) {
        if (i == 0) { memset(mb, 0, sizeof(double) * b); mcopy(b, Pinf, Pb); }
        else {
            om_transition(om, th, t[i] - t[i - 1], A, NULL);
            om_Q(om, A, Pinf, NULL, NULL, Q, NULL);
            mv(b, A, m, mb);
            mm(b, A, P, T); mmt(b, T, A, Pb);
            for (int k = 0; k < b * b; ++k) Pb[k] += Q[k];
            msym(b, Pb);
        }
        if (isnan(y[i])) {
            /* missing observation: infinite noise, no update (Eqs. mean4-mean6) */
            memcpy(m, mb, sizeof(double) * b);
            mcopy(b, Pb, P);
        } else {
            double PH[OMAXB];
            mv(b, Pb, H, PH);
            double S = s2, hm = 0.0;
            for (int k = 0; k < b; ++k) { S += H[k] * PH[k]; hm += H[k] * mb[k]; }
            if (!(S > 0.0)) return E_NUMERIC;
            double v = y[i] - hm;
            for (int k = 0; k < b; ++k) K[k] = PH[k] / S;
            for (int k = 0; k < b; ++k) m[k] = mb[k] + K[k] * v;
            for (int r = 0; r < b; ++r) for (int c = 0; c < b; ++c) P[r * b + c] = Pb[r * b + c] - K[r] * S * K[c];
            msym(b, P);
            acc += -0.5 * (log(2.0 * M_PI * S) + v * v / S);
        }
        if (mf) memcpy(mf + (size_t)i * b, m, sizeof(double) * b);
        if (Pf) memcpy(Pf + (size_t)i * b * b, P, sizeof(double) * b * b);
    }
    *ll = acc;
    return OK;
}

int oseq_loglik(int ncomp, const int* kind, const int* order, const int* env, const double* th,
                const double* t, const double* y, long n, double* ll) {
    om_t om; int st = om_init(&om, ncomp, kind, order, env);
    if (st) return st;
    st = check_inputs(th, om.P, t, y, n);
    if (st) return st;
    return kf_forward(&om, th, t, y, n, ll, NULL, NULL);
}

/* ---------------------------------------------------------------- RTS smoother (posterior, selected inverse) */

/* Posterior of the states given all observations.  Outputs (any may be NULL):
   mean[n] = H m^s_n, var[n] = H P^s_n H^T (latent), ms[n x b], Ps[n x b x b]
   (diagonal blocks of inv(K~)), Pc[(n-1) x b x b] with Pc[i] = Cov(z_{i+1}, z_i | y)
   (first sub-diagonal blocks of inv(K~)). */
int oseq_smoother(int ncomp, const int* kind, const int* order, const int* env, const double* th,
                  const double* t, const double* y, long n, double* ll,
                  double* mean, double* var, double* ms, double* Ps, double* Pc) {
    om_t om; int st = om_init(&om, ncomp, kind, order, env);
    if (st) return st;
    st = check_inputs(th, om.P, t, y, n);
    if (st) return st;
    int b = om.b;
    double* mf = (double*)malloc(sizeof(double) * (size_t)n * b);
    double* Pf = (double*)malloc(sizeof(double) * (size_t)n * b * b);
    if (!mf || !Pf) { free(mf); free(Pf); return E_NOMEM; }
    double llv;
    st = kf_forward(&om, th, t, y, n, &llv, mf, Pf);
    if (st) { free(mf); free(Pf); return st; }
    if (ll) *ll = llv;
    double Pinf[OB2], H[OMAXB], A[OB2], Q[OB2];
    double msn[OMAXB], Psn[OB2];  /* smoothed at i+1 */
    om_pinf(&om, th, Pinf, NULL);
    om_H(&om, H);
    memcpy(msn, mf + (size_t)(n - 1) * b, sizeof(double) * b);
    mcopy(b, Pf + (size_t)(n - 1) * b * b, Psn);
    for (long i = n - 1; i >= 0; --i) {
        if (i < n - 1) {
            const double* m = mf + (size_t)i * b;
            const double* P = Pf + (size_t)i * b * b;
            double mb[OMAXB], Pb[OB2], T[OB2], G[OB2], Gt[OB2], d[OMAXB], D[OB2];
            om_transition(&om, th, t[i + 1] - t[i], A, NULL);
            om_Q(&om, A, Pinf, NULL, NULL, Q, NULL);
            mv(b, A, m, mb);
            mm(b, A, P, T); mmt(b, T, A, Pb);
            for (int k = 0; k < b * b; ++k) Pb[k] += Q[k];
            msym(b, Pb);
            /* gain G = P A^T Pb^-1  <=>  Pb G^T = A P */
            mm(b, A, P, T);
            if (lu_solve(b, Pb, T, b, Gt)) { free(mf); free(Pf); return E_NUMERIC; }
            for (int r = 0; r < b; ++r) for (int c = 0; c < b; ++c) G[r * b + c] = Gt[c * b + r];
            if (Pc) { /* Cov(z_{i+1}, z_i) = P^s_{i+1} G^T */
                mm(b, Psn, Gt, Pc + (size_t)i * b * b);
            }
            for (int k = 0; k < b; ++k) d[k] = msn[k] - mb[k];
            double Gd[OMAXB];
            mv(b, G, d, Gd);
            for (int k = 0; k < b; ++k) msn[k] = m[k] + Gd[k];
            for (int k = 0; k < b * b; ++k) D[k] = Psn[k] - Pb[k];
            mm(b, G, D, T); mmt(b, T, G, D);
            for (int k = 0; k < b * b; ++k) Psn[k] = P[k] + D[k];
            msym(b, Psn);
        }
        double hm = 0.0, hph = 0.0;
        for (int r = 0; r < b; ++r) { hm += H[r] * msn[r]; for (int c = 0; c < b; ++c) hph += H[r] * Psn[r * b + c] * H[c]; }
        if (mean) mean[i] = hm;
        if (var) var[i] = hph;
        if (ms) memcpy(ms + (size_t)i * b, msn, sizeof(double) * b);
        if (Ps) mcopy(b, Psn, Ps + (size_t)i * b * b);
    }
    free(mf); free(Pf);
    return OK;
}

/* ---------------------------------------------------------------- gradient (two-filter form) */

/* With the predicted moments (mb, Pb) of a state and the backward information
   (J, eta) of all observations from that state on, the log-likelihood is
   const + log int N(z; mb, Pb) exp(-z^T J z / 2 + eta^T z) dz.  Its partial
   derivatives are  d/dmb = v  and  d/dPb = (v v^T - W J)/2  with
   W = (I + J Pb)^-1, v = W (eta - J mb).  The smoothed moments are
   m^s = mb + Pb v and P^s = Pb W. */
static int two_filter_adjoint(int b, const double* mb, const double* Pb, const double* J, const double* eta,
                              double* v, double* Qbar, double* msm, double* Psm) {
    double M[OB2], W[OB2], I[OB2], r[OMAXB], WJ[OB2];
    mm(b, J, Pb, M);
    for (int i = 0; i < b; ++i) M[i * b + i] += 1.0;
    meye(b, I);
    if (lu_solve(b, M, I, b, W)) return E_NUMERIC;
    mv(b, J, mb, r);
    for (int i = 0; i < b; ++i) r[i] = eta[i] - r[i];
    mv(b, W, r, v);
    mm(b, W, J, WJ);
    for (int i = 0; i < b; ++i) for (int j = 0; j < b; ++j) Qbar[i * b + j] = 0.5 * (v[i] * v[j] - WJ[i * b + j]);
    msym(b, Qbar);
    double pv[OMAXB];
    mv(b, Pb, v, pv);
    for (int i = 0; i < b; ++i) msm[i] = mb[i] + pv[i];
    mm(b, Pb, W, Psm);
    msym(b, Psm);
    return OK;
}

/* Log-likelihood and its gradient with respect to all P parameters.
   Optionally also the posterior mean / latent variance from the same pass. */
int oseq_grad(int ncomp, const int* kind, const int* order, const int* env, const double* th,
              const double* t, const double* y, long n, double* ll, double* grad, double* mean, double* var,
              double* gabs) {
    om_t om; int st = om_init(&om, ncomp, kind, order, env);
    if (st) return st;
    st = check_inputs(th, om.P, t, y, n);
    if (st) return st;
    int b = om.b, P = om.P;
    double s2 = th[P - 1];
    double* mf = (double*)malloc(sizeof(double) * (size_t)n * b);
    double* Pf = (double*)malloc(sizeof(double) * (size_t)n * b * b);
    double* dA = (double*)malloc(sizeof(double) * P * b * b);
    double* dQ = (double*)malloc(sizeof(double) * P * b * b);
    double* dPinf = (double*)malloc(sizeof(double) * P * b * b);
    if (!mf || !Pf || !dA || !dQ || !dPinf) { st = E_NOMEM; goto out; }
    st = kf_forward(&om, th, t, y, n, ll, mf, Pf);
    if (st) goto out;
    double Pinf[OB2], H[OMAXB], A[OB2], Q[OB2];
    om_pinf(&om, th, Pinf, dPinf);
    om_H(&om, H);
    for (int p = 0; p < P; ++p) { grad[p] = 0.0; if (gabs) gabs[p] = 0.0; }
    /* backward information of y_{n-1}: J = H^T H / s2, eta = H^T y / s2 */
    double J[OB2], eta[OMAXB];
    const double w_last = isnan(y[n - 1]) ? 0.0 : 1.0 / s2;   /* a missing observation carries no information */
    for (int r = 0; r < b; ++r) {
        eta[r] = (w_last != 0.0) ? H[r] * y[n - 1] * w_last : 0.0;
        for (int c = 0; c < b; ++c) J[r * b + c] = H[r] * H[c] * w_last;
    }
    double gs2 = 0.0;
    for (long i = n - 1; i >= 0; --i) {
        double mb[OMAXB], Pb[OB2], T[OB2], v[OMAXB], Qbar[OB2], msm[OMAXB], Psm[OB2];
        if (i > 0) {
            const double* m = mf + (size_t)(i - 1) * b;
            const double* Pp = Pf + (size_t)(i - 1) * b * b;
            om_transition(&om, th, t[i] - t[i - 1], A, dA);
            om_Q(&om, A, Pinf, dA, dPinf, Q, dQ);
            mv(b, A, m, mb);
            mm(b, A, Pp, T); mmt(b, T, A, Pb);
            for (int k = 0; k < b * b; ++k) Pb[k] += Q[k];
            msym(b, Pb);
            if ((st = two_filter_adjoint(b, mb, Pb, J, eta, v, Qbar, msm, Psm))) goto out;
            /* dl/dA = v m^T + 2 Qbar A P ; dl/dQ = Qbar */
            double Abar[OB2], X[OB2];
            mm(b, Qbar, A, X); mm(b, X, Pp, T);
            for (int r = 0; r < b; ++r) for (int c = 0; c < b; ++c) Abar[r * b + c] = v[r] * m[c] + 2.0 * T[r * b + c];
            for (int p = 0; p < P; ++p) {
                double term = mdot(b, Abar, dA + (size_t)p * b * b) + mdot(b, Qbar, dQ + (size_t)p * b * b);
                grad[p] += term;
                if (gabs) gabs[p] += fabs(term);
            }
        } else {
            memset(mb, 0, sizeof(double) * b);
            mcopy(b, Pinf, Pb);
            if ((st = two_filter_adjoint(b, mb, Pb, J, eta, v, Qbar, msm, Psm))) goto out;
            for (int p = 0; p < P; ++p) {
                double term = mdot(b, Qbar, dPinf + (size_t)p * b * b);
                grad[p] += term;
                if (gabs) gabs[p] += fabs(term);
            }
        }
        /* observation noise: d/ds2 sum_i log N(y_i; H z_i, s2) averaged over the posterior */
        double hm = 0.0, hph = 0.0;
        for (int r = 0; r < b; ++r) { hm += H[r] * msm[r]; for (int c = 0; c < b; ++c) hph += H[r] * Psm[r * b + c] * H[c]; }
        if (!isnan(y[i])) {
            double e = y[i] - hm;
            double gterm = (e * e + hph) / (2.0 * s2 * s2) - 0.5 / s2;
            gs2 += gterm;
            if (gabs) gabs[P - 1] += fabs(gterm);
        }
        if (mean) mean[i] = hm;
        if (var) var[i] = hph;
        if (i > 0) {
            /* propagate the information through the transition into state i-1:
               J' = A^T (I + J Q)^-1 J A,  eta' = A^T (I + J Q)^-1 eta,  then add y_{i-1} */
            double M[OB2], Rhs[OB2 + OMAXB], Sol[OB2 + OMAXB], MJ[OB2], Me[OMAXB];
            mm(b, J, Q, M);
            for (int k = 0; k < b; ++k) M[k * b + k] += 1.0;
            for (int r = 0; r < b; ++r) { for (int c = 0; c < b; ++c) Rhs[r * (b + 1) + c] = J[r * b + c]; Rhs[r * (b + 1) + b] = eta[r]; }
            if (lu_solve(b, M, Rhs, b + 1, Sol)) { st = E_NUMERIC; goto out; }
            for (int r = 0; r < b; ++r) { for (int c = 0; c < b; ++c) MJ[r * b + c] = Sol[r * (b + 1) + c]; Me[r] = Sol[r * (b + 1) + b]; }
            mm(b, MJ, A, T); mtm(b, A, T, J);
            msym(b, J);
            mtv(b, A, Me, eta);
            if (!isnan(y[i - 1]))
                for (int r = 0; r < b; ++r) { eta[r] += H[r] * y[i - 1] / s2; for (int c = 0; c < b; ++c) J[r * b + c] += H[r] * H[c] / s2; }
        }
    }
    grad[P - 1] = gs2;
out:
    free(mf); free(Pf); free(dA); free(dQ); free(dPinf);
    return st;
}

/* ---------------------------------------------------------------- sampling from the state-space model */

/* y = H z + noise with z drawn from the model; eps holds n*(b+1) standard
   normal numbers drawn by the caller.  Uses a pivot-free Cholesky factor of
   Q that treats non-positive pivots as zero, so zero gaps are allowed. */
static void psd_chol(int b, const double* Q, double* L) {
    mzero(b, L);
    for (int j = 0; j < b; ++j) {
        double d = Q[j * b + j];
        for (int k = 0; k < j; ++k) d -= L[j * b + k] * L[j * b + k];
        if (d <= 1e-300) continue;
        double s = sqrt(d);
        L[j * b + j] = s;
        for (int i = j + 1; i < b; ++i) {
            double x = Q[i * b + j];
            for (int k = 0; k < j; ++k) x -= L[i * b + k] * L[j * b + k];
            L[i * b + j] = x / s;
        }
    }
}

int oseq_sample(int ncomp, const int* kind, const int* order, const int* env, const double* th,
                const double* t, long n, const double* eps, double* y) {
    om_t om; int st = om_init(&om, ncomp, kind, order, env);
    if (st) return st;
    st = check_inputs(th, om.P, t, NULL, n);
    if (st) return st;
    int b = om.b;
    double Pinf[OB2], H[OMAXB], A[OB2], Q[OB2], L[OB2], z[OMAXB], w[OMAXB];
    om_pinf(&om, th, Pinf, NULL);
    om_H(&om, H);
    double sn = sqrt(th[om.P - 1]);
    for (long i = 0; i < n; ++i) {
        const double* e = eps + (size_t)i * (b + 1);
        if (i == 0) { psd_chol(b, Pinf, L); mv(b, L, e, z); }
        else {
            om_transition(&om, th, t[i] - t[i - 1], A, NULL);
            om_Q(&om, A, Pinf, NULL, NULL, Q, NULL);
            psd_chol(b, Q, L);
            mv(b, A, z, w);
            double lw[OMAXB];
            mv(b, L, e, lw);
            for (int k = 0; k < b; ++k) z[k] = w[k] + lw[k];
        }
        double f = 0.0;
        for (int k = 0; k < b; ++k) f += H[k] * z[k];
        y[i] = f + sn * e[b];
    }
    return OK;
}
