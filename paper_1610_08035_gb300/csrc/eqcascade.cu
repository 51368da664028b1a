// eqcascade.cu -- host-side constants of the exponentiated-quadratic (EQ)
// state-space approximation of even order N, as a cascade of N/2
// second-order sections whose states are uncorrelated at stationarity.
//
// The EQ covariance s exp(-t^2/(2 l^2)) has spectral density
// s sqrt(2 pi) l exp(-l^2 w^2/2); replacing exp(l^2 w^2/2) by its Taylor
// polynomial of order N in l^2 w^2/2 gives a rational density whose stable
// spectral factor c / d(p), d(p) = prod_k (p - rho_k)(p - conj rho_k), is a
// linear SDE of order N (Hartikainen & Sarkka 2010; the paper's experiments
// use N = 10, Sec. 4.2).  At unit lengthscale the poles rho_k = a_k + i b_k
// are the left-half-plane roots of sum_{n<=N} (-r^2/2)^n / n!, and
// c^2 = sqrt(2 pi) 2^N N!; a lengthscale l divides the poles by l (time is
// measured in units of l).
//
// Realization.  Unit white noise e drives a chain of sections: section k has
// a 2-vector state x_k with dx_k/dt = S_k x_k + g_k e_{k-1}, and passes on
// e_k = e_{k-1} - g_k^T x_k.  With S_k = [[-gam^2/2, om], [-om, 0]],
// g_k = (gam, 0), gam^2 = -4 a_k and om = |rho_k|, the whole generator S
// (S_kk on the diagonal, -g_k g_i^T below it for k > i) satisfies
// S + S^T = -g g^T: the stationary covariance of x is the identity, and each
// e_k is e filtered by the all-pass factors of sections 1..k.  The output
// f = sum_k h_k^T x_k has transfer function c / d(p) when
//   sum_k gam_k (h_k0 p - h_k1 om_k) prod_{i<k} D_i(-p) prod_{i>k} D_i(p) = c,
// D_i(p) = (p - rho_i)(p - conj rho_i); evaluated at p = rho_m (where every
// term k < m vanishes) this is a triangular system for h, solved from the last
// section back.  Nothing here inverts an ill-conditioned matrix: the modal
// (diagonalised) form of the same SDE has a stationary covariance of
// condition ~1e11 at N = 10, whose entries cancel to f's variance.
//
// Coordinates used on the GPU.  Each section is mapped by W_k = [Re v, Im v],
// v the eigenvector of S_k for rho_k scaled so that h_k^T v = 1.  Then, in
// z_k = W_k^-1 x_k:
//   - the generator's diagonal blocks are [[a_k, b_k], [-b_k, a_k]] (so the
//     transition's diagonal blocks are e^(a x) times a rotation by b x);
//   - its blocks below the diagonal are -u_k w_i^T (k > i), with
//     u_k = W_k^-1 g_k and w_i = W_i^T g_i;
//   - f is the sum of the first coordinates of the sections;
//   - the stationary covariance is block diagonal, P_k = W_k^-1 W_k^-T per
//     section (Pinf = s P at variance s).
#include <complex>
#include <cmath>

namespace spg {

using cd = std::complex<double>;

// one root of c[0] + c[1] x + ... + c[n] x^n by Laguerre's method from x
static cd laguerre(const cd* c, int n, cd x) {
    for (int it = 0; it < 200; ++it) {
        cd p = c[n], d = 0.0, e = 0.0;
        for (int k = n - 1; k >= 0; --k) {
            e = e * x + d;
            d = d * x + p;
            p = p * x + c[k];
        }
        if (std::abs(p) == 0.0) return x;
        const cd G = d / p, H = G * G - 2.0 * e / p;
        const cd sq = std::sqrt(double(n - 1) * (double(n) * H - G * G));
        const cd den = (std::abs(G + sq) >= std::abs(G - sq)) ? G + sq : G - sq;
        const cd step = (std::abs(den) > 0.0) ? double(n) / den : cd(1e-3, 1e-3);
        x -= step;
        if (std::abs(step) <= 1e-16 * std::abs(x)) break;
    }
    return x;
}

// Newton polishing of x against c (degree n)
static cd polish(const cd* c, int n, cd x) {
    for (int it = 0; it < 6; ++it) {
        cd p = c[n], d = 0.0;
        for (int k = n - 1; k >= 0; --k) { d = d * x + p; p = p * x + c[k]; }
        if (std::abs(d) == 0.0) break;
        x -= p / d;
    }
    return x;
}

// The N/2 stable poles a + i b (b > 0) at unit lengthscale, by decreasing b.
static bool eq_poles(int N, cd* up) {
    // p(w) = sum_n (-w/2)^n / n!, w = r^2
    cd c[17], work[17];
    double f = 1.0;
    for (int n = 0; n <= N; ++n) {
        if (n > 0) f *= n;
        c[n] = std::pow(-0.5, n) / f;
    }
    for (int n = 0; n <= N; ++n) work[n] = c[n];
    cd w[16];
    for (int deg = N; deg >= 1; --deg) {
        cd x = laguerre(work, deg, cd(0.1, 0.3));
        x = polish(c, N, x);
        w[N - deg] = x;
        // deflate: work <- work / (w - x)
        cd carry = work[deg];
        for (int k = deg - 1; k >= 0; --k) {
            const cd t = work[k];
            work[k] = carry;
            carry = t + carry * x;
        }
    }
    int nu = 0;
    for (int j = 0; j < N; ++j) {
        cd r = -std::sqrt(w[j]);
        if (r.real() > 0.0) r = -r;
        if (!(r.real() < 0.0)) return false;
        if (r.imag() > 0.0) {
            if (nu >= N / 2) return false;
            up[nu++] = r;
        }
    }
    if (nu != N / 2) return false;
    for (int i = 1; i < nu; ++i)   // decreasing imaginary part
        for (int j = i; j > 0 && up[j].imag() > up[j - 1].imag(); --j) std::swap(up[j], up[j - 1]);
    return true;
}

// N even, 2 <= N <= 16, K = N/2 sections.  Outputs per section k: the pole
// a[k] + i b[k], u[2k..2k+1], w[2k..2k+1] and P[4k..4k+3] (row-major 2x2).
// False if the construction fails its own checks.
bool eq_cascade(int N, double* a, double* b, double* u, double* w, double* P) {
    if (N < 2 || N > 16 || (N & 1)) return false;
    const int K = N / 2;
    cd rho[8];
    if (!eq_poles(N, rho)) return false;
    double gam[8], om[8];
    for (int k = 0; k < K; ++k) {
        a[k] = rho[k].real();
        b[k] = rho[k].imag();
        gam[k] = std::sqrt(-4.0 * a[k]);
        om[k] = std::abs(rho[k]);
    }
    double fact = 1.0;
    for (int n = 2; n <= N; ++n) fact *= n;
    const double c = std::sqrt(std::sqrt(2.0 * M_PI) * std::pow(2.0, N) * fact);
    auto D = [&](int i, cd p) { return (p - rho[i]) * (p - std::conj(rho[i])); };
    // the output weights h_k, from the last section back
    double h[8][2];
    for (int m = K - 1; m >= 0; --m) {
        const cd p = rho[m];
        cd known = 0.0;
        for (int k = m + 1; k < K; ++k) {
            cd t = gam[k] * (h[k][0] * p - h[k][1] * om[k]);
            for (int i = 0; i < k; ++i) t *= D(i, -p);
            for (int i = k + 1; i < K; ++i) t *= D(i, p);
            known += t;
        }
        cd coef = gam[m];
        for (int i = 0; i < m; ++i) coef *= D(i, -p);
        for (int i = m + 1; i < K; ++i) coef *= D(i, p);
        const cd r = (c - known) / coef;      // h_m0 p - h_m1 om_m = r
        h[m][0] = r.imag() / p.imag();
        h[m][1] = (h[m][0] * p.real() - r.real()) / om[m];
        if (!std::isfinite(h[m][0]) || !std::isfinite(h[m][1])) return false;
    }
    // per-section coordinates
    for (int k = 0; k < K; ++k) {
        cd v0 = om[k], v1 = rho[k] + 0.5 * gam[k] * gam[k];   // (S_k - rho I) v = 0
        const cd s = 1.0 / (h[k][0] * v0 + h[k][1] * v1);
        v0 *= s; v1 *= s;
        const double W[2][2] = {{v0.real(), v0.imag()}, {v1.real(), v1.imag()}};
        const double det = W[0][0] * W[1][1] - W[0][1] * W[1][0];
        if (!(std::fabs(det) > 0.0)) return false;
        const double Wi[2][2] = {{W[1][1] / det, -W[0][1] / det}, {-W[1][0] / det, W[0][0] / det}};
        u[2 * k] = Wi[0][0] * gam[k];                 // W^-1 (gam, 0)
        u[2 * k + 1] = Wi[1][0] * gam[k];
        w[2 * k] = W[0][0] * gam[k];                  // W^T (gam, 0)
        w[2 * k + 1] = W[0][1] * gam[k];
        for (int i = 0; i < 2; ++i)
            for (int j = 0; j < 2; ++j) P[4 * k + 2 * i + j] = Wi[i][0] * Wi[j][0] + Wi[i][1] * Wi[j][1];
    }
    // checks: (1) the Lyapunov equation T P + P T^T + g g^T = 0 block by
    // block (g = u, T's blocks [[a, b], [-b, a]] and -u_k w_i^T); (2) the
    // transfer function at p = 0: f's response to a unit step of the noise,
    // -sum_k (T^-1 u)_k,0, equals c / prod |rho_k|^2; (3) the variance
    // sum_k P_k,00 is the approximate kernel's k(0), near 1 (1.14 at N = 2,
    // 1.017 at N = 4, closer above).
    double res = 0.0, mag = 0.0;
    for (int k = 0; k < K; ++k)
        for (int i = 0; i <= k; ++i)
            for (int r = 0; r < 2; ++r)
                for (int q = 0; q < 2; ++q) {
                    // (T P)_{ki} = T_ki P_i (P block diagonal), (P T^T)_{ki} = P_k T_ik^T
                    double tp = 0.0, pt = 0.0;
                    for (int j = 0; j < 2; ++j) {
                        const double tkj = (i == k) ? ((r == j) ? a[k] : (r == 0 ? b[k] : -b[k]))
                                                    : -u[2 * k + r] * w[2 * i + j];
                        tp += tkj * P[4 * i + 2 * j + q];
                        const double tij = (i == k) ? ((q == j) ? a[k] : (q == 0 ? b[k] : -b[k])) : 0.0;
                        pt += P[4 * k + 2 * r + j] * tij;
                    }
                    const double s = tp + pt + u[2 * k + r] * u[2 * i + q];
                    res = std::fmax(res, std::fabs(s));
                    mag = std::fmax(mag, std::fabs(u[2 * k + r] * u[2 * i + q]));
                }
    if (!(res <= 1e-10 * mag)) return false;
    // T y = u by forward substitution: T_kk y_k = u_k + u_k sum_{i<k} w_i^T y_i
    double ysum = 0.0, acc = 0.0, den = 1.0;
    for (int k = 0; k < K; ++k) {
        const double s = 1.0 + acc;
        const double r0 = u[2 * k] * s, r1 = u[2 * k + 1] * s;
        const double d = a[k] * a[k] + b[k] * b[k];    // [[a, b], [-b, a]]^-1 = [[a, -b], [b, a]] / d
        const double y0 = (a[k] * r0 - b[k] * r1) / d, y1 = (b[k] * r0 + a[k] * r1) / d;
        acc += w[2 * k] * y0 + w[2 * k + 1] * y1;
        ysum += y0;
        den *= d;
    }
    const double tf = -ysum, want = c / den;
    if (!(std::fabs(tf - want) <= 1e-9 * std::fabs(want))) return false;
    double k0 = 0.0;
    for (int k = 0; k < K; ++k) k0 += P[4 * k];
    return std::fabs(k0 - 1.0) <= 0.25;
}

}  // namespace spg
