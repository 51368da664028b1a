// eqmodal.cu -- host-side constants of the exponentiated-quadratic (EQ)
// state-space approximation of even order N, in real modal coordinates.
//
// The EQ covariance s exp(-t^2/(2 l^2)) has spectral density
// s sqrt(2 pi) l exp(-l^2 w^2/2); replacing exp(l^2 w^2/2) by its Taylor
// polynomial of order N in l^2 w^2/2 gives a rational density whose stable
// spectral factor is a linear SDE of order N (Hartikainen & Sarkka 2010; the
// paper's experiments use N = 10, Sec. 4.2).  At unit lengthscale its poles
// are the left-half-plane roots r of sum_{n<=N} (-r^2/2)^n / n!; for even N
// they form N/2 complex-conjugate pairs rho_k = a_k + i b_k, and a lengthscale
// l divides them by l (time is measured in units of l).
//
// In the companion coordinates (f, f', ...) the eigenvectors are Vandermonde
// columns v(r) = (1, r, r^2, ..); with the complex modal state zeta (one entry
// per pole) the white noise enters through c_i = 1 / prod_{j != i}(r_i - r_j)
// (the last column of the inverse Vandermonde matrix), so the stationary
// covariance is Pi_ij = -q c_i conj(c_j) / (r_i + conj(r_j)), q = sqrt(2 pi)
// 2^N N!.  The real pair x_k = (zeta + conj zeta, i (zeta - conj zeta)) of
// each pole pair then has the block generator [[a_k, b_k], [-b_k, a_k]], the
// observation picks the first entry of every pair (v(r)_0 = 1), and the
// stationary covariance is E Pi E^H with E = blockdiag([[1, 1], [i, -i]]):
// a dense, lengthscale-free matrix P_m (Pinf = s P_m), computed here without
// inverting any ill-conditioned matrix.
#include <complex>
#include <cmath>

namespace spg {

using cd = std::complex<double>;

// one root of the monic-degree polynomial c[0] + c[1] x + ... + c[n] x^n by
// Laguerre's method from x0
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

// N even, 2 <= N <= 16.  Outputs: a[N/2], b[N/2] (pole pairs a + i b, b > 0,
// by decreasing b), Pm (N x N, row stride ld).  False if the construction
// fails its own checks.
bool eq_modal(int N, double* a, double* b, double* Pm, int ld) {
    if (N < 2 || N > 16 || (N & 1)) return false;
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
    // stable poles r = -sqrt(w); keep the upper half-plane member of each pair
    cd up[8];
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
    cd r[16];
    for (int k = 0; k < nu; ++k) { r[2 * k] = up[k]; r[2 * k + 1] = std::conj(up[k]); a[k] = up[k].real(); b[k] = up[k].imag(); }
    cd ci[16];
    for (int i = 0; i < N; ++i) {
        cd pr = 1.0;
        for (int j = 0; j < N; ++j) if (j != i) pr *= (r[i] - r[j]);
        ci[i] = 1.0 / pr;
    }
    double q = std::sqrt(2.0 * M_PI) * std::pow(2.0, N);
    for (int n = 2; n <= N; ++n) q *= n;
    cd Pi[16][16];
    for (int i = 0; i < N; ++i)
        for (int j = 0; j < N; ++j) Pi[i][j] = -q * ci[i] * std::conj(ci[j]) / (r[i] + std::conj(r[j]));
    const cd E[2][2] = {{cd(1, 0), cd(1, 0)}, {cd(0, 1), cd(0, -1)}};
    double scale = 0.0, imag = 0.0;
    for (int k = 0; k < nu; ++k)
        for (int l = 0; l < nu; ++l)
            for (int al = 0; al < 2; ++al)
                for (int be = 0; be < 2; ++be) {
                    cd s = 0.0;
                    for (int u = 0; u < 2; ++u)
                        for (int v = 0; v < 2; ++v) s += E[al][u] * Pi[2 * k + u][2 * l + v] * std::conj(E[be][v]);
                    Pm[(2 * k + al) * ld + (2 * l + be)] = s.real();
                    scale = std::fmax(scale, std::abs(s.real()));
                    imag = std::fmax(imag, std::abs(s.imag()));
                }
    if (!(imag <= 1e-9 * scale)) return false;   // E Pi E^H is real
    for (int i = 0; i < N; ++i)
        for (int j = i + 1; j < N; ++j) {
            const double m = 0.5 * (Pm[i * ld + j] + Pm[j * ld + i]);
            Pm[i * ld + j] = m; Pm[j * ld + i] = m;
        }
    // Lyapunov residual X Pm + Pm X^T + q g g^T = 0 (g = E c) as a check
    double g[16];
    for (int k = 0; k < nu; ++k) {
        g[2 * k] = (ci[2 * k] + ci[2 * k + 1]).real();
        g[2 * k + 1] = (cd(0, 1) * (ci[2 * k] - ci[2 * k + 1])).real();
    }
    double res = 0.0, mag = 0.0, gmax = 0.0, xmax = 0.0;
    for (int i = 0; i < N; ++i) { gmax = std::fmax(gmax, std::abs(g[i])); xmax = std::fmax(xmax, std::abs(a[i / 2]) + std::abs(b[i / 2])); }
    for (int i = 0; i < N; ++i)
        for (int j = 0; j < N; ++j) {
            const int ki = i / 2, kj = j / 2;
            double s = q * g[i] * g[j];
            // (X Pm)[i][j] + (Pm X^T)[i][j]: rows 2k, 2k+1 of X are (a, b), (-b, a) on block k
            s += (i % 2 == 0) ? a[ki] * Pm[i * ld + j] + b[ki] * Pm[(i + 1) * ld + j]
                              : -b[ki] * Pm[(i - 1) * ld + j] + a[ki] * Pm[i * ld + j];
            s += (j % 2 == 0) ? a[kj] * Pm[i * ld + j] + b[kj] * Pm[i * ld + j + 1]
                              : -b[kj] * Pm[i * ld + j - 1] + a[kj] * Pm[i * ld + j];
            res = std::fmax(res, std::abs(s));
        }
    mag = q * gmax * gmax + 2.0 * xmax * scale;
    return res <= 1e-9 * mag;
}

}  // namespace spg
