// internal.h -- declarations shared by the library's translation units.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>
#include <stddef.h>

namespace spg {

// structured models on the group path: sums of components whose transitions
// are 2x2 blocks (Matern-3/2, periodic, quasi-periodic with a Matern-1/2
// envelope); state dimension b = 2K <= 16
static constexpr int GMAXCOMP = 4;
static constexpr int GMAXBLK = 8;
struct GModel {
    int b, K, P, ncomp;
    int bkind[GMAXBLK], bcomp[GMAXBLK], bj[GMAXBLK];   // per block: kind, component, harmonic
    int ckind[GMAXCOMP], cpoff[GMAXCOMP];              // per component: spingp_kind, theta offset
    // an exponentiated-quadratic component as a cascade of second-order
    // sections (at most one, its blocks first: eq_k0 = 0): block count, the
    // diagonal generator blocks [[a, b], [-b, a]] at unit lengthscale, the
    // coupling blocks -u_k w_i^T below the diagonal (k > i), and its
    // unit-variance stationary covariance P (block diagonal, order x order,
    // row stride 16; Pinf = variance P)
    int eq_comp, eq_k0, eq_nk;
    double eqa[GMAXBLK], eqb[GMAXBLK];
    double equ[2 * GMAXBLK], eqw[2 * GMAXBLK];
    // per coupling block (k, i), k > i, at index k (k - 1) / 2 + i:
    // 1 / ((a_k - a_i)^2 + (b_k - b_i)^2) and 1 / ((a_k - a_i)^2 + (b_k + b_i)^2)
    double eqrc[GMAXBLK * (GMAXBLK - 1) / 2], eqra[GMAXBLK * (GMAXBLK - 1) / 2];
    double eqP[16 * 16];
    // doubles per step of the stored transition: 4 per diagonal block (GMAXBLK
    // of them), then 4 per EQ block below the diagonal
    int phs;
};
// host: constants of the order-N EQ cascade (eqcascade.cu); per section k:
// pole a[k] + i b[k], u[2k..], w[2k..], P[4k..4k+3]
bool eq_cascade(int N, double* a, double* b, double* u, double* w, double* P);

// the driver's unique ID of the current context, 0 if unavailable (capi.cu)
unsigned long long context_id();

// device status bits (the status word at the start of every workspace)
enum { ST_EINVAL = 1 << 1, ST_ENOTSORTED = 1 << 2, ST_ENONFINITE = 1 << 3, ST_ENUMERIC = 1 << 4 };

// what a run computes (MODE_GRAD_POSTERIOR: the gradient and the posterior
// from one forward pass and one reverse sweep)
enum { MODE_LOGLIK = 0, MODE_GRAD = 1, MODE_POSTERIOR = 2, MODE_GRAD_POSTERIOR = 3 };

size_t matern_ws_bytes(int b, int64_t n, int64_t L, int mode);
int matern_prepare();
// ev: NULL, or 5 events recorded around the four stages
// missing: 1 = a NaN observation is a missing one (predicted, not conditioned on)
// Inputs from host memory (matern_run with a feed): t and y are copied on the
// copy stream in FEED_PIECES pieces of steps -- piece p is a range of step
// columns of every chunk, the widths doubling from L/16 -- and the
// elimination runs as one launch per piece on the main stream, each after its
// piece's copy.  ev[0] orders the copies after earlier work on the main
// stream, ev[1 + p] marks piece p's copy.  theta_h (host, theta_bytes) is
// copied to the run's theta on the copy stream ahead of piece 0.
static constexpr int FEED_PIECES = 4;
struct HostFeed {
    const double* t;
    const double* y;
    const double* theta_h;
    size_t theta_bytes;
    cudaStream_t copy;
    cudaEvent_t ev[1 + FEED_PIECES];
    int npieces;
};
// lag1_out (posterior only, else ignored): n - 1 entries Cov(f_{i+1}, f_i | y), or NULL
int matern_run(int b, int mode, const double* t, const double* y, int64_t n, int64_t L, const double* theta,
               double* ll_out, double* grad_out, double* mean_out, double* var_out, void* ws, cudaStream_t st,
               cudaEvent_t* ev, int missing, const HostFeed* feed = nullptr, double* lag1_out = nullptr);
int matern_launch_count(int b, int64_t n, int64_t L, int mode);
// output conventions by flag (post.cu): the gradient in log theta (count
// entries, theta in the same layout), predictive variances (latent + s_n)
int grad_to_log(double* grad, const double* theta, int64_t count, cudaStream_t st);
int add_noise(double* var, int64_t n, const double* s_n, cudaStream_t st);

// prediction at new times: the call's workspace is [status word][merged
// times and observations, the posterior over them, sort buffers][the
// posterior call's own workspace at off_inner]
struct PredictLayout {
    size_t off_T, off_Y, off_mean, off_var, off_k0, off_k1, off_i0, off_i1, off_inner;
    PredictLayout(int64_t n, int64_t m);
};
int predict_merge_passes(int64_t m);
// sort the test times (keeping their positions) and merge them with the
// observed ones into the layout's T, Y (NaN observations at test points)
int predict_prepare(const double* t, const double* y, int64_t n, const double* ts, int64_t m, void* ws,
                    const PredictLayout& lay, cudaStream_t st);
// the test points' moments into the caller's order; the posterior's status
// joined into the call's status word
int predict_finish(const double* t, int64_t n, int64_t m, void* ws, const PredictLayout& lay, double* mean_out,
                   double* var_out, cudaStream_t st);
int add_noise_batched(double* var, const int64_t* offsets, int64_t n_series, const double* theta, int P,
                      cudaStream_t st);
// a series split across ranks (phase 0: reduce this range to its element;
// phase 1: from all G elements, this range's share of ll and gradient and,
// when mean_out and var_out are given, the posterior at this range's steps)
static constexpr int SEG_MAX_RANKS = 32;
int matern_segment(int b, int phase, const double* t, const double* y, int64_t n, int64_t L, const double* theta,
                   double t_prev, int first, const double* elems, int G, int rank, double* elem_out, double* ll_out,
                   double* grad_out, void* ws, cudaStream_t st, int missing, double* mean_out = nullptr,
                   double* var_out = nullptr);
int matern_elem_size(int b);
int matern_segment_launch_count(int b, int64_t n, int64_t L);

// batches of independent series: offsets (device, nseries + 1 entries), theta
// per series (nseries x 3), per-series ll_out / grad_out
size_t matern_ws_bytes_batched(int b, int64_t nseries, int64_t n_total, int64_t L, int mode);
int matern_launch_count_batched(int b, int64_t nseries, int64_t n_total, int64_t L, int mode);
int matern_run_batched(int b, int mode, const int64_t* offsets, int64_t nseries, int64_t n_total, const double* t,
                       const double* y, int64_t L, const double* theta, double* ll_out, double* grad_out,
                       double* mean_out, double* var_out, void* ws, cudaStream_t st, cudaEvent_t* ev, int missing);

// the paper's method as written (btd.cu): explicit K~ blocks, block cyclic
// reduction with selected inverse, subproblem 4, and the composed literal path
size_t btd_ws_bytes(int b, int64_t n);
int btd_solve(int b, int64_t n, const double* D, const double* O, const double* r, double* logdet, double* x,
              double* Sd, double* So, void* ws, cudaStream_t st);
int64_t btd_launch_count(int64_t n);
size_t diagprod_ws_bytes(int64_t n);
int btd_diagprod(int b, int64_t n, const double* Sd, const double* So, const double* Xd, const double* Xo,
                 double* diag, double* trace, void* ws, cudaStream_t st);
size_t assemble_ws_bytes(int64_t n);
int assemble(int b, const double* t, const double* y, int64_t n, const double* theta, double* D, double* O,
             double* r, double* logdet_kinv, void* ws, cudaStream_t st);
size_t literal_ws_bytes(int b, int64_t n, int mode);
int literal_run(int b, int mode, const double* t, const double* y, int64_t n, const double* theta, double* ll,
                double* grad, double* mean, double* var, void* ws, cudaStream_t st);
int64_t literal_launch_count(int64_t n);

// scaled conjugate gradients over a batch of series (optim.cu): the state of
// every series, bound to caller workspace, and its evaluation buffers
struct ScgState {
    int64_t S;
    int P;
    double *w, *r, *p, *s, *g;                                   // S x P
    double *f, *lam, *lambar, *delta, *sigma, *mu, *pp, *alpha;  // S
    int* flags;                                                  // S
    double *theta_eval, *grad_eval;                              // S x P: where the next gradient is taken
    double* ll_eval;                                             // S
};
enum { SCG_K_INIT, SCG_K_START, SCG_K_A, SCG_K_B, SCG_K_C, SCG_K_FINAL, SCG_K_OUT };
size_t scg_state_bytes(int64_t S, int P);
ScgState scg_bind(void* base, int64_t S, int P);
int scg_launch(int what, const ScgState& st, cudaStream_t s, int k, double tol, const double* theta0,
               double* theta_out, double* ll_out, double* grad_out, int* status);

size_t probe_fp64_bytes();
int probe_fp64(void* scratch, size_t bytes, double* tflops, cudaStream_t st, int tensor);
int probe_exp_neg(const double* x, double* y, int64_t n, cudaStream_t st);

}  // namespace spg

namespace spg {
size_t group_ws_bytes(const GModel& gm, int64_t n, int64_t L, int mode);
int group_launch_count(int64_t n, int64_t L, int mode);
int group_run(const GModel& gm, int mode, const double* t, const double* y, int64_t n, int64_t L,
              const double* theta, double* ll_out, double* grad_out, double* mean_out, double* var_out, void* ws,
              cudaStream_t st, cudaEvent_t* ev, int missing, double* lag1_out = nullptr);
int group_segment(const GModel& gm, int phase, const double* t, const double* y, int64_t n, int64_t L,
                  const double* theta, double t_prev, int first, const double* elems, int G, int rank,
                  double* elem_out, double* ll_out, double* grad_out, void* ws, cudaStream_t st, int missing,
                  double* mean_out = nullptr, double* var_out = nullptr);
int group_elem_size();
int group_segment_launch_count(int64_t n, int64_t L);
}  // namespace spg

struct spingp_model;
namespace spg {
// true when the model runs on the b <= 3 chain kernels (matern.cu)
bool model_on_chain_path(const spingp_model* m);
}  // namespace spg
