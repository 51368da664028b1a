// optim.cu -- hyperparameter fitting by scaled conjugate gradients (Moller
// 1993), the optimiser the paper uses for the marginal likelihood (Sec. 4.3).
//
// The objective of series i is E_i(w) = -ll_i(exp(w)) over log-parameters w.
// Every series carries its own optimiser state; one thread per series runs
// the algorithm's scalar decisions on the device, between the gradient
// evaluations of the whole batch, so an optimisation of thousands of series
// is a fixed sequence of launches with no host round trip (it can be
// captured into a CUDA graph).  One iteration:
//   k_scg_a   direction length, curvature probe point w + sigma p (sigma = sigma0/|p|)
//   (gradient of every series at its probe point)
//   k_scg_b   s = (E'(w + sigma p) - E'(w)) / sigma, delta = p.s; the lambda
//             scaling and positive-definiteness fix; mu = p.r,
//             alpha = mu / delta; trial point w + alpha p
//   (objective and gradient of every series at its trial point)
//   k_scg_c   Delta = 2 delta (E(w) - E(w + alpha p)) / mu^2; accept or reject;
//             new conjugate direction (restart along r every P iterations,
//             else beta = (|r'|^2 - r'.r) / mu); lambda update
// Where the published algorithm leaves room: sigma0 = 1e-4, lambda_1 = 1e-6,
// lambda in [1e-15, 1e100]; a trial point with a non-finite objective or
// gradient is rejected (Delta = -1); a zero p.r or delta restarts along r;
// a series stops once max |E'| <= tol or p = 0.
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include "internal.h"

namespace spg {

static constexpr double SCG_SIGMA0 = 1e-4;
static constexpr double SCG_LAMBDA1 = 1e-6;
static constexpr double SCG_LAM_MIN = 1e-15;
static constexpr double SCG_LAM_MAX = 1e100;

enum { SCG_SUCCESS = 1, SCG_DONE = 2, SCG_SKIP = 4, SCG_BAD_START = 8 };

static size_t oalign(size_t x) { return (x + 255) & ~(size_t)255; }

size_t scg_state_bytes(int64_t S, int P) {
    const size_t v = oalign(sizeof(double) * (size_t)S * P), c = oalign(sizeof(double) * (size_t)S);
    return 5 * v + 8 * c + oalign(sizeof(int) * (size_t)S) + 2 * v + c;
}

ScgState scg_bind(void* base, int64_t S, int P) {
    const size_t v = oalign(sizeof(double) * (size_t)S * P), c = oalign(sizeof(double) * (size_t)S);
    char* b = (char*)base;
    ScgState st;
    st.S = S;
    st.P = P;
    st.w = (double*)b; b += v;
    st.r = (double*)b; b += v;
    st.p = (double*)b; b += v;
    st.s = (double*)b; b += v;
    st.g = (double*)b; b += v;
    st.f = (double*)b; b += c;
    st.lam = (double*)b; b += c;
    st.lambar = (double*)b; b += c;
    st.delta = (double*)b; b += c;
    st.sigma = (double*)b; b += c;
    st.mu = (double*)b; b += c;
    st.pp = (double*)b; b += c;
    st.alpha = (double*)b; b += c;
    st.flags = (int*)b; b += oalign(sizeof(int) * (size_t)S);
    st.theta_eval = (double*)b; b += v;
    st.grad_eval = (double*)b; b += v;
    st.ll_eval = (double*)b; b += c;
    return st;
}

// log-parameters from the caller's theta; the first evaluation point is theta
__global__ void k_scg_init(ScgState st, const double* __restrict__ theta0) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= st.S) return;
    int fl = 0;
    for (int j = 0; j < st.P; ++j) {
        const double th = theta0[i * st.P + j];
        if (!(th > 0.0) || !isfinite(th)) fl = SCG_BAD_START;
        st.w[i * st.P + j] = log(th);
        st.theta_eval[i * st.P + j] = th;
    }
    st.flags[i] = fl;
}

// E'(w) = -theta * d ll / d theta at an evaluated point; false if not finite
__device__ __forceinline__ bool log_grad(const ScgState& st, int64_t i, int j, double& gj) {
    gj = -st.theta_eval[i * st.P + j] * st.grad_eval[i * st.P + j];
    return isfinite(gj);
}

__global__ void k_scg_start(ScgState st, double tol) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= st.S) return;
    const int P = st.P;
    const double f = -st.ll_eval[i];
    bool ok = isfinite(f) && !(st.flags[i] & SCG_BAD_START);
    double gmax = 0.0, pp = 0.0;
    for (int j = 0; j < P; ++j) {
        double gj;
        ok = log_grad(st, i, j, gj) && ok;
        st.g[i * P + j] = gj;
        st.r[i * P + j] = -gj;
        st.p[i * P + j] = -gj;
        st.s[i * P + j] = 0.0;
        gmax = fmax(gmax, fabs(gj));
        pp += gj * gj;
    }
    st.f[i] = f;
    st.lam[i] = SCG_LAMBDA1;
    st.lambar[i] = 0.0;
    st.delta[i] = 0.0;
    int fl = SCG_SUCCESS | (st.flags[i] & SCG_BAD_START);
    if (!ok || gmax <= tol || pp == 0.0) fl |= SCG_DONE;
    st.flags[i] = fl;
}

// probe point for the second-order information (only after a success)
__global__ void k_scg_a(ScgState st) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= st.S) return;
    const int P = st.P;
    const int fl = st.flags[i];
    double pp = 0.0;
    for (int j = 0; j < P; ++j) pp += st.p[i * P + j] * st.p[i * P + j];
    st.pp[i] = pp;
    const bool probe = !(fl & SCG_DONE) && (fl & SCG_SUCCESS);
    const double sigma = probe ? SCG_SIGMA0 / sqrt(pp) : 0.0;
    st.sigma[i] = sigma;
    for (int j = 0; j < P; ++j) st.theta_eval[i * P + j] = exp(st.w[i * P + j] + sigma * st.p[i * P + j]);
}

__global__ void k_scg_b(ScgState st) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= st.S) return;
    const int P = st.P;
    int fl = st.flags[i] & ~SCG_SKIP;
    double* w = st.w + i * P;
    double* p = st.p + i * P;
    double* s = st.s + i * P;
    double alpha = 0.0;
    if (!(fl & SCG_DONE)) {
        const double pp = st.pp[i];
        double lam = st.lam[i], lambar = st.lambar[i], delta = st.delta[i];
        if (fl & SCG_SUCCESS) {
            const double sigma = st.sigma[i];
            delta = 0.0;
            for (int j = 0; j < P; ++j) {
                double gj;
                log_grad(st, i, j, gj);
                s[j] = (gj - st.g[i * P + j]) / sigma;
                delta += p[j] * s[j];
            }
        }
        for (int j = 0; j < P; ++j) s[j] += (lam - lambar) * p[j];
        delta += (lam - lambar) * pp;
        if (delta <= 0.0) {
            for (int j = 0; j < P; ++j) s[j] += (lam - 2.0 * delta / pp) * p[j];
            lambar = 2.0 * (lam - delta / pp);
            delta = -delta + lam * pp;
            lam = lambar;
        }
        double mu = 0.0;
        for (int j = 0; j < P; ++j) mu += p[j] * st.r[i * P + j];
        if (mu == 0.0 || delta == 0.0) {
            for (int j = 0; j < P; ++j) p[j] = st.r[i * P + j];
            lambar = 0.0;
            fl |= SCG_SUCCESS | SCG_SKIP;
        } else {
            alpha = mu / delta;
        }
        st.lam[i] = lam;
        st.lambar[i] = lambar;
        st.delta[i] = delta;
        st.mu[i] = mu;
    }
    st.alpha[i] = alpha;
    st.flags[i] = fl;
    for (int j = 0; j < P; ++j) st.theta_eval[i * P + j] = exp(w[j] + alpha * p[j]);
}

// k: the 1-based iteration number (the same for every series)
__global__ void k_scg_c(ScgState st, int k, double tol) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= st.S) return;
    const int P = st.P;
    int fl = st.flags[i];
    if (fl & (SCG_DONE | SCG_SKIP)) return;
    double* w = st.w + i * P;
    double* p = st.p + i * P;
    double* r = st.r + i * P;
    double* g = st.g + i * P;
    const double pp = st.pp[i], delta = st.delta[i], mu = st.mu[i], alpha = st.alpha[i];
    double lam = st.lam[i], lambar;
    const double fn = -st.ll_eval[i];
    bool ok = isfinite(fn);
    for (int j = 0; j < P; ++j) {
        double gj;
        ok = log_grad(st, i, j, gj) && ok;
    }
    const double D = ok ? 2.0 * delta * (st.f[i] - fn) / (mu * mu) : -1.0;
    if (D >= 0.0) {
        double rr = 0.0, rr_old = 0.0;
        for (int j = 0; j < P; ++j) {
            double gj;
            log_grad(st, i, j, gj);
            const double rn = -gj;
            rr += rn * rn;
            rr_old += rn * r[j];
        }
        const bool restart = (k % P) == 0;
        const double beta = restart ? 0.0 : (rr - rr_old) / mu;
        double gmax = 0.0, pn2 = 0.0;
        for (int j = 0; j < P; ++j) {
            double gj;
            log_grad(st, i, j, gj);
            w[j] = w[j] + alpha * p[j];
            g[j] = gj;
            r[j] = -gj;
            p[j] = restart ? -gj : -gj + beta * p[j];
            gmax = fmax(gmax, fabs(gj));
            pn2 += p[j] * p[j];
        }
        st.f[i] = fn;
        lambar = 0.0;
        fl |= SCG_SUCCESS;
        if (D >= 0.75) lam = fmax(lam / 4.0, SCG_LAM_MIN);
        if (gmax <= tol || pn2 == 0.0) fl |= SCG_DONE;
    } else {
        lambar = lam;
        fl &= ~SCG_SUCCESS;
    }
    if (D < 0.25) lam = fmin(lam + delta * (1.0 - D) / pp, SCG_LAM_MAX);
    st.lam[i] = lam;
    st.lambar[i] = lambar;
    st.flags[i] = fl;
}

// the final point: theta = exp(w)
__global__ void k_scg_final_point(ScgState st) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= st.S) return;
    for (int j = 0; j < st.P; ++j) st.theta_eval[i * st.P + j] = exp(st.w[i * st.P + j]);
}

// copy the result out; a series whose start was invalid raises EINVAL
__global__ void k_scg_out(ScgState st, double* __restrict__ theta_out, double* __restrict__ ll_out,
                          double* __restrict__ grad_out, int* status) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= st.S) return;
    if (st.flags[i] & SCG_BAD_START) atomicOr(status, ST_EINVAL);
    for (int j = 0; j < st.P; ++j) {
        theta_out[i * st.P + j] = st.theta_eval[i * st.P + j];
        if (grad_out) grad_out[i * st.P + j] = st.grad_eval[i * st.P + j];
    }
    if (ll_out) ll_out[i] = st.ll_eval[i];
}

static unsigned sgrid(int64_t S) { return (unsigned)((S + 127) / 128); }

int scg_launch(int what, const ScgState& st, cudaStream_t s, int k, double tol, const double* theta0,
               double* theta_out, double* ll_out, double* grad_out, int* status) {
    const unsigned g = sgrid(st.S);
    switch (what) {
    case SCG_K_INIT: k_scg_init<<<g, 128, 0, s>>>(st, theta0); break;
    case SCG_K_START: k_scg_start<<<g, 128, 0, s>>>(st, tol); break;
    case SCG_K_A: k_scg_a<<<g, 128, 0, s>>>(st); break;
    case SCG_K_B: k_scg_b<<<g, 128, 0, s>>>(st); break;
    case SCG_K_C: k_scg_c<<<g, 128, 0, s>>>(st, k, tol); break;
    case SCG_K_FINAL: k_scg_final_point<<<g, 128, 0, s>>>(st); break;
    default: k_scg_out<<<g, 128, 0, s>>>(st, theta_out, ll_out, grad_out, status); break;
    }
    return cudaGetLastError() == cudaSuccess ? 0 : 1;
}

}  // namespace spg
