/*
 * spingp.h -- C ABI of the GB300 library for exact inference in state-space
 * temporal Gaussian processes through their block-tridiagonal precision
 * (SpInGP, Grigorievskiy, Lawrence & Sarkka, arXiv 1610.08035).
 *
 * Model (Sec. 2.1, Eq. ss1): z_{i+1} = A_i z_i + q_i, q_i ~ N(0, Q_i);
 * y_i = H z_i + e_i, e_i ~ N(0, sigma_n^2), for sorted times t_0 <= ... <= t_{n-1},
 * with A_i = expm(F (t_{i+1} - t_i)), Q_i = Pinf - A_i Pinf A_i^T and the first
 * state z_0 ~ N(0, Pinf).  The stacked state covariance has a block-
 * tridiagonal inverse (Theorem 1); the posterior precision is
 * K~ = Kinv + G^T Sigma^-1 G with G = I_n (x) H and Sigma = sigma_n^2 I (Sec. 2.2).
 *
 * Conventions for every entry point below:
 *   - All array arguments are DEVICE pointers to FP64 data owned by the
 *     caller, on the current CUDA device; nothing is copied to the host.
 *   - theta is a device array of spingp_num_params(model) entries: for each
 *     component its parameters in the order listed at spingp_kind, then the
 *     noise variance sigma_n^2 last.  Every entry must be finite and > 0.
 *   - ws is caller-owned device scratch of at least
 *     spingp_workspace_bytes(model, n, what) bytes, 256-byte aligned; the
 *     library allocates no device memory on these paths.  One workspace must
 *     not be used by two calls that can overlap on the GPU.
 *   - stream is a cudaStream_t (NULL = legacy default stream).  Work is
 *     enqueued asynchronously.  Argument errors that the host can see are
 *     returned at once and nothing is launched.  Errors that only the device
 *     can see (unsorted or non-finite inputs, a non-positive theta entry, a
 *     non-positive innovation variance) are recorded in a status word inside
 *     ws: pass SPINGP_SYNC in flags to have the call synchronise the stream
 *     and return that status, or call spingp_ws_status() later.  Without
 *     SPINGP_SYNC the call launches kernels only (no host synchronisation,
 *     no allocation) and may be captured into a CUDA graph.
 *   - Outputs are written on the stream; their contents are unspecified when
 *     the call reports an error.
 */
#ifndef SPINGP_H
#define SPINGP_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    SPINGP_OK = 0,
    SPINGP_EINVAL = 1,       /* bad argument: NULL pointer, n < 1, bad theta, workspace too small */
    SPINGP_ENOTSORTED = 2,   /* some t[i+1] < t[i] */
    SPINGP_ENONFINITE = 3,   /* a time or an observation is NaN or infinite */
    SPINGP_ENUMERIC = 4,     /* an innovation variance or a pivot was not positive and finite */
    SPINGP_ECUDA = 5,        /* a CUDA runtime call failed */
    SPINGP_ETIMEOUT = 6,     /* reserved for bounded device-side waits */
    SPINGP_ENOMEM = 7,       /* host memory allocation failed */
    SPINGP_EUNSUPPORTED = 8  /* model structure not implemented by this build */
} spingp_status;

/* Covariance families (Sec. 2.1).  Parameters per component, in theta order:
 *   MATERN12/32/52: (lengthscale l, variance s); state dim 1/2/3; the
 *       companion-form SDE of (d/dt + lam)^b with lam = sqrt(2b-1)/l
 *       (Eq. ss_matern gives the 3/2 case).
 *   PERIODIC (order J): (variance, lengthscale, period); state dim 2(J+1).
 *   QUASIPERIODIC (order J, Matern envelope): (variance, lengthscale, period,
 *       envelope lengthscale); state dim 2(J+1) x envelope dim (Eq. co2_1).
 *   EQ (order N, even, 2..16): (lengthscale, variance); state dim N.  The
 *       exponentiated quadratic s exp(-t^2/(2 l^2)) through its state-space
 *       approximation (Sec. 2.1; the paper's experiments use N = 10): the
 *       spectral density with exp(l^2 w^2/2) replaced by its Taylor
 *       polynomial of order N, whose stable spectral factor is an SDE of
 *       order N (Hartikainen & Sarkka 2010).  The library realizes it as a
 *       cascade of N/2 second-order sections whose states are uncorrelated
 *       at stationarity (a block-diagonal stationary covariance, a
 *       transition with damped-rotation diagonal blocks and coupling blocks
 *       below them), which keeps f's quantities free of cancellation; the
 *       modal (diagonalised) form of the same SDE has a stationary
 *       covariance of condition ~1e11 at N = 10.  The approximation error
 *       against the exact covariance falls with N (below 2e-4 s at N = 10).
 *       At most one EQ component per model. */
typedef enum {
    SPINGP_MATERN12 = 1,
    SPINGP_MATERN32 = 2,
    SPINGP_MATERN52 = 3,
    SPINGP_PERIODIC = 4,
    SPINGP_QUASIPERIODIC = 5,
    SPINGP_EQ = 6
} spingp_kind;

typedef struct {
    int n_comp;          /* number of summed components (>= 1) */
    const int* kinds;    /* n_comp spingp_kind values (host memory) */
    const int* orders;   /* harmonic order J per component, or NULL */
    const int* envs;     /* envelope kind per quasi-periodic component, or NULL */
} spingp_model_desc;

typedef struct spingp_model spingp_model;

/* What a workspace is sized for. */
typedef enum { SPINGP_WS_LOGLIK = 0, SPINGP_WS_GRAD = 1, SPINGP_WS_POSTERIOR = 2 } spingp_ws_kind;

#define SPINGP_SYNC 1u
/* Treat NaN observations as missing: the state at that time is predicted but
 * not conditioned on (infinite noise there).  This is the augmented
 * formulation of Eqs. mean4-mean6: put the test times into t with y = NaN and
 * spingp_posterior returns the predictive mean and latent variance at them;
 * log-likelihoods and gradients then cover the observed points only.  Without
 * this flag a NaN observation is an error (SPINGP_ENONFINITE). */
#define SPINGP_MISSING_NAN 2u
/* Return the gradient with respect to log theta instead of theta:
 * d ll / d log theta_p = theta_p d ll / d theta_p (a diagonal rescaling; the
 * paper's hyperparameters are positive).  Honoured by spingp_grad,
 * spingp_grad_posterior, their batched forms, spingp_grad_host and the
 * split-series calls (each rank's share is
 * rescaled; the shares still sum to the series' value); one more kernel
 * launch per call. */
#define SPINGP_LOG_GRAD 4u
/* Return predictive variances of an observation instead of latent ones: the
 * latent variance H P^s H^T plus the noise variance s_n (the series' last
 * theta entry).  Honoured by every call that returns posterior variances
 * (spingp_posterior, spingp_posterior_lag1, spingp_grad_posterior, their
 * batched and split-series forms); one more kernel launch per call. */
#define SPINGP_PREDICTIVE 8u

/* Create a model handle from a host-side description (Sec. 2.1).  The handle
 * holds host constants only; it owns no device memory.  Returns EINVAL for a
 * malformed description and EUNSUPPORTED for a structure this build does not
 * run on the GPU.  *out is set to NULL on error.  The GPU runs:
 *   - one Matern-1/2, 3/2 or 5/2 component (state dimension 1 to 3);
 *   - sums of total state dimension <= 16 whose components are Matern-3/2,
 *     periodic, quasi-periodic with a Matern-1/2 envelope, and at most one
 *     EQ (every block of their transition is 2 x 2, or an EQ section).
 * Other structures (a Matern-1/2 or 5/2 inside a sum, a Matern-3/2 or 5/2
 * envelope, more than 16 states) return EUNSUPPORTED. */
spingp_status spingp_model_create(const spingp_model_desc* desc, spingp_model** out);
void spingp_model_destroy(spingp_model* model);

/* Number of theta entries (noise variance included) and state dimension b. */
int spingp_num_params(const spingp_model* model);
int spingp_state_dim(const spingp_model* model);

/* Chunk length L: the number of consecutive steps one GPU thread eliminates
 * sequentially before the odd-even reduction across chunks.  0 selects the
 * built-in default.  Returns EINVAL outside [8, 65536]. */
spingp_status spingp_set_chunk_len(spingp_model* model, int chunk_len);
int spingp_get_chunk_len(const spingp_model* model, int64_t n);

/* Workspace bytes needed for one series of n steps (0 for n < 1).
 * The single-series calls below need n >= 1 and return SPINGP_EINVAL for
 * n < 1 before any device work; an empty series is a batch entry (the
 * batched calls give it log-likelihood 0 and a zero gradient). */
size_t spingp_workspace_bytes(const spingp_model* model, int64_t n, spingp_ws_kind what);

/* Log marginal likelihood (Eq. ml2), written to ll_out[0].  Computed through
 * the determinant lemma (Eq. det_1) and subproblems 1 and 3: a sequential
 * elimination inside chunks of L steps, an odd-even cyclic reduction of the
 * chunk Schur complements, and the prediction-error decomposition within each
 * chunk.  t: n sorted times; y: n observations. */
spingp_status spingp_loglik(const spingp_model* model, const double* t, const double* y, int64_t n,
                            const double* theta, double* ll_out,
                            void* ws, size_t ws_bytes, unsigned flags, void* stream);

/* Log-likelihood and its gradient with respect to every theta entry (Sec. 2.4,
 * the data-fit derivative and the trace term of Eq. dd1), written to ll_out[0]
 * and grad_out[0 .. num_params-1].  The trace of subproblem 4 is evaluated
 * through the selected inverse of K~ in adjoint form: a reverse sweep per
 * chunk, seeded by the reduced suffix information, chained through
 * d expm(F dt)/dtheta and dQ/dtheta. */
spingp_status spingp_grad(const spingp_model* model, const double* t, const double* y, int64_t n,
                          const double* theta, double* ll_out, double* grad_out,
                          void* ws, size_t ws_bytes, unsigned flags, void* stream);

/* Posterior of the latent function at the training times (Eq. mean6,
 * subproblem 1, and the diagonal of Eq. k3, subproblem 2): mean_out[i] = H m^s_i
 * and var_out[i] = H P^s_i H^T (latent variance, no noise added), where P^s_i
 * are the diagonal blocks of inv(K~).  ll_out may be NULL. */
spingp_status spingp_posterior(const spingp_model* model, const double* t, const double* y, int64_t n,
                               const double* theta, double* ll_out, double* mean_out, double* var_out,
                               void* ws, size_t ws_bytes, unsigned flags, void* stream);

/* spingp_posterior plus the first off-diagonal of the selected inverse
 * (Sec. 3.1: the blocks of inv(K~) next to its diagonal, subproblem 4's
 * operand) for the latent function: cov_lag1_out[i] = H P^s_{i+1,i} H^T =
 * Cov(f(t_{i+1}), f(t_i) | y) for i = 0 .. n-2 (device, n - 1 doubles; may be
 * NULL only when n = 1).  P^s_{i+1,i} is formed in the reverse sweep as
 * (I - Pb_{i+1} Lt_{i+1}) A_{i+1} P_i, with P_i the filtered covariance and
 * Lt_{i+1} the adjoint information of y_{i+1} and after on the predicted
 * state; a missing observation (SPINGP_MISSING_NAN) leaves Lt unchanged
 * there.  The same workspace and flags as spingp_posterior (SPINGP_PREDICTIVE
 * affects var_out only). */
spingp_status spingp_posterior_lag1(const spingp_model* model, const double* t, const double* y, int64_t n,
                                    const double* theta, double* ll_out, double* mean_out, double* var_out,
                                    double* cov_lag1_out, void* ws, size_t ws_bytes, unsigned flags,
                                    void* stream);

/* spingp_grad and spingp_posterior_lag1 in one call: a learning step that also
 * wants the posterior at the current hyperparameters (Sec. 2.4 and Sec. 3.1
 * share subproblems 1 to 4: the same elimination, reduction and reverse
 * sweep give the gradient's trace terms and the selected inverse's blocks).
 * One forward pass and one reverse sweep, so it costs about what spingp_grad
 * costs, not the sum of both calls.  Writes ll_out[0], grad_out[0 ..
 * num_params-1], mean_out[0 .. n-1], var_out[0 .. n-1] (all required) and,
 * when cov_lag1_out is not NULL, cov_lag1_out[0 .. n-2] as
 * spingp_posterior_lag1 does.  Each output equals the separate call's up to
 * rounding order.  Workspace: spingp_workspace_bytes(model, n, SPINGP_WS_GRAD)
 * (the SPINGP_WS_POSTERIOR size is the same).  SPINGP_LOG_GRAD affects
 * grad_out only, SPINGP_PREDICTIVE var_out only; SPINGP_MISSING_NAN and
 * SPINGP_SYNC as for the other calls.  EINVAL for a NULL required output. */
spingp_status spingp_grad_posterior(const spingp_model* model, const double* t, const double* y, int64_t n,
                                    const double* theta, double* ll_out, double* grad_out, double* mean_out,
                                    double* var_out, double* cov_lag1_out, void* ws, size_t ws_bytes,
                                    unsigned flags, void* stream);

/* Prediction at new times (Eqs. mean4-mean6): the posterior mean and latent
 * variance of f at n_star test times t_star, given n observations (t, y)
 * (t ascending; NaN observations are missing).  The test times join the
 * chain as steps with no observation (infinite noise), so one posterior pass
 * over the n + n_star merged steps gives them; a test time equal to an
 * observed one is placed after it.  t_star may be in any order (it is sorted
 * on the device, stably); mean_out[j], var_out[j] belong to t_star[j].
 * n = 0 gives the prior at t_star.  All arrays are device memory; ws is
 * device scratch of spingp_predict_workspace_bytes(model, n, n_star) bytes
 * (256-byte aligned); its status word reports ENOTSORTED for observed times
 * out of order and ENONFINITE for a non-finite time.  SPINGP_PREDICTIVE
 * adds the noise variance to var_out; SPINGP_SYNC as for the other calls.
 * EINVAL for n < 0, n_star < 1 or a NULL argument. */
size_t spingp_predict_workspace_bytes(const spingp_model* model, int64_t n, int64_t n_star);
spingp_status spingp_predict(const spingp_model* model, const double* t, const double* y, int64_t n,
                             const double* theta, const double* t_star, int64_t n_star, double* mean_out,
                             double* var_out, void* ws, size_t ws_bytes, unsigned flags, void* stream);

/* ---- batches of independent series ----------------------------------------
 * n_series series, each with its own hyperparameters, concatenated: series i
 * owns steps [offsets[i], offsets[i+1]) of t and y, with offsets[0] = 0,
 * offsets non-decreasing and offsets[n_series] = n_total (an empty series has
 * log-likelihood 0 and a zero gradient).  offsets is a DEVICE array of
 * n_series + 1 int64; n_series and n_total are host values (they size the
 * launch, so a call can be captured into a CUDA graph).  theta is a device
 * array of n_series x num_params entries (row i: series i).  Times must be
 * non-decreasing within each series.  Malformed offsets are detected on the
 * device (EINVAL through the status word) and then no series is processed.
 * One odd-even reduction runs over the chunks of all series together: the
 * first chunk of every series starts from the stationary prior, whose
 * element passes no information between neighbouring series. */
size_t spingp_workspace_bytes_batched(const spingp_model* model, int64_t n_series, int64_t n_total,
                                      spingp_ws_kind what);

/* Per-series log-likelihoods (Eq. ml2) into ll_out[0 .. n_series-1]. */
spingp_status spingp_loglik_batched(const spingp_model* model, const int64_t* offsets, int64_t n_series,
                                    int64_t n_total, const double* t, const double* y, const double* theta,
                                    double* ll_out, void* ws, size_t ws_bytes, unsigned flags, void* stream);

/* Per-series log-likelihoods and gradients (Sec. 2.4): ll_out[i] and
 * grad_out[i * num_params + p]. */
spingp_status spingp_grad_batched(const spingp_model* model, const int64_t* offsets, int64_t n_series,
                                  int64_t n_total, const double* t, const double* y, const double* theta,
                                  double* ll_out, double* grad_out, void* ws, size_t ws_bytes, unsigned flags,
                                  void* stream);

/* Per-step posterior mean and latent variance of every series (Eqs. mean6,
 * k3), indexed like t and y; per-series log-likelihoods into ll_out (may be
 * NULL). */
spingp_status spingp_posterior_batched(const spingp_model* model, const int64_t* offsets, int64_t n_series,
                                       int64_t n_total, const double* t, const double* y, const double* theta,
                                       double* ll_out, double* mean_out, double* var_out, void* ws,
                                       size_t ws_bytes, unsigned flags, void* stream);

/* spingp_grad_batched and spingp_posterior_batched from one forward pass and
 * one reverse sweep (Sec. 2.4 and Sec. 3.1 share subproblems 1 to 4; see
 * spingp_grad_posterior): per-series ll_out[n_series] and
 * grad_out[n_series x num_params], per-step mean_out and var_out indexed like
 * t and y (all required when n_total > 0).  Each output equals the separate
 * call's up to rounding order.  Workspace:
 * spingp_workspace_bytes_batched(..., SPINGP_WS_GRAD).  SPINGP_LOG_GRAD
 * affects grad_out only, SPINGP_PREDICTIVE var_out only. */
spingp_status spingp_grad_posterior_batched(const spingp_model* model, const int64_t* offsets, int64_t n_series,
                                            int64_t n_total, const double* t, const double* y, const double* theta,
                                            double* ll_out, double* grad_out, double* mean_out, double* var_out,
                                            void* ws, size_t ws_bytes, unsigned flags, void* stream);

/* Number of kernels one call of the given kind launches for n steps (the
 * discretisation/elimination pass, the reduction tiles, the per-chunk pass
 * and the final reduction). */
int spingp_launch_count(const spingp_model* model, int64_t n, spingp_ws_kind what);
int spingp_launch_count_batched(const spingp_model* model, int64_t n_series, int64_t n_total, spingp_ws_kind what);

/* Stage timing.  While enabled, every call on this model records CUDA events
 * on its stream around its four stages: 0 discretisation + in-chunk
 * elimination, 1 odd-even reduction, 2 per-chunk forward/reverse pass,
 * 3 final reduction.  spingp_profile_read synchronises on the recorded events,
 * writes the summed milliseconds per stage to ms_out[0..3] and the number of
 * calls to *calls, and clears the record.  Not for use during stream capture;
 * a model with profiling enabled must not be shared between host threads. */
spingp_status spingp_profile_enable(spingp_model* model, int on);
spingp_status spingp_profile_read(spingp_model* model, double* ms_out, int* calls);

/* Measured FP64 throughput of the current device: a kernel of independent
 * fused multiply-adds (no memory traffic) on every SM, timed with CUDA events.
 * scratch: device memory of at least spingp_probe_fp64_bytes() bytes for the
 * kernel's results.  Synchronises the stream; writes TFLOP/s to *tflops_out. */
size_t spingp_probe_fp64_bytes(void);
spingp_status spingp_probe_fp64(void* scratch, size_t scratch_bytes, double* tflops_out, void* stream);

/* The same measurement for the FP64 tensor-core instruction (mma.sync
 * m8n8k4, eight independent products per warp; 512 flop each): the rate a
 * kernel that moved the b x b block products onto tensor cores could reach.
 * Same arguments and behaviour as spingp_probe_fp64. */
spingp_status spingp_probe_fp64_tensor(void* scratch, size_t scratch_bytes, double* tflops_out, void* stream);

/* y[i] = e^-x[i] for i < n, computed on the stream by the table-driven
 * exponential that the chain kernels use for the discretisation (the
 * e^-lam dt factor of Eq. ss_matern's expm).  x, y: device arrays of n
 * doubles (x[i] >= 0; 0 for x[i] > 708; NaN propagates), owned by the
 * caller.  Its accuracy is tested against a correctly rounded exponential.
 * SPINGP_EINVAL for n < 0 or a NULL array with n > 0. */
spingp_status spingp_probe_exp_neg(const double* x, double* y, int64_t n, void* stream);

/* ---- one series split across ranks (one process per GPU) -------------------
 * The series is cut into G <= 32 contiguous ranges, range r on rank r; the
 * odd-even reduction of Sec. 3.1 then spans the ranks with one exchange:
 *   1. spingp_segment_reduce: each rank reduces its range to one element, the
 *      Schur complement of K~ on the state before the range and the range's
 *      last state, in conditional-covariance form (for a single Matern
 *      model A, b, C, eta, J: b^2, b, b(b+1)/2, b, b(b+1)/2 doubles in that
 *      order, upper triangles row by row; spingp_segment_elem_size doubles
 *      in every case), written to elem_out (device).
 *      The range of rank 0 starts the series (first = 1); every other range
 *      continues it (first = 0), and t_prev is the time of the last step of
 *      the range before it (host value, finite, <= t[0]).
 *   2. the caller all-gathers the G elements, in rank order, into one device
 *      array elems of G x elem_size doubles (rank-major);
 *   3. spingp_segment_grad: from elems, this range's share of the
 *      log-likelihood and gradient (ll_out[0], grad_out[0 .. P-1], device);
 *      the series' values are the sums of the shares over the ranks (one
 *      all-reduce).
 * Calls 1 and 3 of a rank take the same t, y, n, theta, t_prev, first, flags
 * and the same workspace (spingp_workspace_bytes(model, n, SPINGP_WS_GRAD)),
 * with no other call on that workspace in between: call 3 reuses what call 1
 * left in it.  With G = 1 the result is spingp_grad's.  Every model runs
 * this way; for the structured models (b > 3 or sums) the element is the
 * group path's (b x b blocks padded to 16 x 16: spingp_segment_elem_size
 * doubles).  SPINGP_EINVAL for n < 1, G outside
 * [1, 32], rank outside [0, G), first != (rank == 0), or a non-finite t_prev
 * when first = 0. */
int spingp_segment_elem_size(const spingp_model* model);
/* GPU launches of one rank's spingp_segment_reduce plus spingp_segment_grad
 * for a range of n steps; -1 when unsupported or n < 1. */
int spingp_segment_launch_count(const spingp_model* model, int64_t n);
spingp_status spingp_segment_reduce(const spingp_model* model, const double* t, const double* y, int64_t n,
                                    const double* theta, double t_prev, int first, double* elem_out, void* ws,
                                    size_t ws_bytes, unsigned flags, void* stream);
spingp_status spingp_segment_grad(const spingp_model* model, const double* t, const double* y, int64_t n,
                                  const double* theta, double t_prev, int first, const double* elems, int n_ranks,
                                  int rank, double* ll_out, double* grad_out, void* ws, size_t ws_bytes,
                                  unsigned flags, void* stream);
/* Step 3 with the posterior as well (spingp_grad_posterior for a split
 * series): this range's share of ll and gradient, as spingp_segment_grad
 * writes them, and the posterior mean and latent variance at this range's
 * own steps, mean_out[0 .. n-1] and var_out[0 .. n-1] (device; all four
 * outputs required).  The mean and variance at a step use every rank's
 * observations, before and after the range: the elements of all G ranks
 * carry the information that the range's reverse sweep starts from, so no
 * further exchange is needed.  The same arguments, workspace and flags as
 * spingp_segment_grad; SPINGP_PREDICTIVE adds the noise variance to var_out.
 * With G = 1 the outputs are spingp_grad_posterior's. */
spingp_status spingp_segment_grad_posterior(const spingp_model* model, const double* t, const double* y, int64_t n,
                                            const double* theta, double t_prev, int first, const double* elems,
                                            int n_ranks, int rank, double* ll_out, double* grad_out,
                                            double* mean_out, double* var_out, void* ws, size_t ws_bytes,
                                            unsigned flags, void* stream);

/* Log-likelihood and gradient from HOST buffers (Sec. 2.4; the same result
 * as spingp_grad, bit for bit): t, y (n doubles each) and theta are host
 * memory -- pinned memory lets the copies run asynchronously -- and ll_out
 * (1 double) and grad_out (P doubles) are host memory written on the stream
 * (valid after the stream synchronises; SPINGP_SYNC does that).  For the
 * single-Matern chain path t and y are copied on a copy stream the model
 * keeps, in four pieces of steps (piece p: a range of steps of every chunk,
 * as strided copies; the widths double from 1/16 of a chunk), and the
 * in-chunk elimination runs as one launch per piece as soon as that piece
 * has arrived, so the transfer overlaps the computation; structured models
 * copy first, then run.  ws is device scratch of
 * spingp_workspace_bytes_host(model, n) bytes (it also holds the device
 * copies of t, y and theta).  The model's copy stream and events are
 * created on the first call, on the current device; a model's host-buffer
 * calls must not run concurrently from several host threads, and a model
 * used this way stays on one device. */
size_t spingp_workspace_bytes_host(const spingp_model* model, int64_t n);
spingp_status spingp_grad_host(spingp_model* model, const double* t, const double* y, int64_t n,
                               const double* theta, double* ll_out, double* grad_out, void* ws, size_t ws_bytes,
                               unsigned flags, void* stream);

/* Size of the fixed device scratch used by spingp_loglik_noalloc (8 MiB). */
#define SPINGP_NOALLOC_SCRATCH_BYTES (8u << 20)

/* Log-likelihood without any device allocation, for callers that cannot
 * allocate device memory at the point of the call: code running while a
 * stream is being captured into a CUDA graph without a memory pool, real-time
 * or embedded callers whose memory is all reserved at start-up, plug-ins whose
 * host framework owns the device allocator, or callers that must not risk the
 * implicit device synchronisation an allocation or a free can cause.  (The
 * paper has no counterpart: this is a deployment variant of spingp_loglik.)
 *
 * Same arguments and result as spingp_loglik, without the workspace: the
 * scratch is a file-scope array of SPINGP_NOALLOC_SCRATCH_BYTES in the
 * library's device image, which every GPU that loads the library keeps until
 * the process exits.  A series whose spingp_workspace_bytes(model, n,
 * SPINGP_WS_LOGLIK) exceeds that size is rejected with SPINGP_EINVAL before
 * anything is launched (with the default chunk length this admits every
 * n <= 65536 for state dimension b <= 3).  The call allocates nothing and
 * frees nothing.  The first call on a device performs a one-time set-up for
 * that device (looking up the array's device address); make that first call
 * before capturing any stream.  After a device reset the next call repeats
 * the set-up for the new context.  All calls on a device share the one array
 * and it keeps the last call's contents: the call clears what must start at
 * zero itself, and two calls that can overlap on the GPU (different streams,
 * or different host threads) race on the scratch and corrupt each other; the
 * library serialises only the set-up, so the caller serialises the calls.
 * With SPINGP_SYNC the call synchronises the stream and returns the device
 * status, as spingp_loglik does. */
spingp_status spingp_loglik_noalloc(const spingp_model* model, const double* t, const double* y, int64_t n,
                                    const double* theta, double* ll_out, unsigned flags, void* stream);

/* ------------------------------------------------------------------------
 * Hyperparameter fitting (Sec. 4.3): the paper maximises the marginal
 * likelihood by scaled conjugate gradients (Moller 1993).
 *
 * Each series is optimised on its own, over log-parameters w = log(theta)
 * with objective -ll(exp(w)).  Every iteration evaluates the gradient of all
 * series twice (a curvature probe at w + sigma p, sigma = 1e-4 / |p|, and the
 * trial point w + alpha p); the algorithm's scalar decisions (the
 * Levenberg-Marquardt scale lambda, starting at 1e-6 and kept in
 * [1e-15, 1e100], the acceptance ratio, conjugate directions with a restart
 * every P iterations) run in device kernels between the evaluations, so a
 * call is a fixed sequence of launches with no host synchronisation (without
 * SPINGP_SYNC it can be captured into a CUDA graph).  A trial point with a
 * non-finite objective or gradient is rejected.  A series stops early once
 * max |d(-ll)/dw| <= tol, or when its search direction vanishes.
 *
 * theta_inout: device, P entries (n_series x P for the batched form) --
 * the starting point (every entry finite and > 0, else SPINGP_EINVAL), and on
 * return the last accepted point.  ll_out (1 or n_series doubles) and
 * grad_out (d ll / d theta at the returned point, P or n_series x P doubles)
 * may be NULL.  iterations >= 0.  The workspace holds a gradient workspace
 * plus the optimiser state; its status word reports the final evaluation.
 * The batched form supports the models spingp_grad_batched supports.
 * ------------------------------------------------------------------------ */
size_t spingp_optimize_workspace_bytes(const spingp_model* model, int64_t n);
spingp_status spingp_optimize(const spingp_model* model, const double* t, const double* y, int64_t n,
                              double* theta_inout, int iterations, double tol, double* ll_out, double* grad_out,
                              void* ws, size_t ws_bytes, unsigned flags, void* stream);
size_t spingp_optimize_workspace_bytes_batched(const spingp_model* model, int64_t n_series, int64_t n_total);
spingp_status spingp_optimize_batched(const spingp_model* model, const int64_t* offsets, int64_t n_series,
                                      int64_t n_total, const double* t, const double* y, double* theta_inout,
                                      int iterations, double tol, double* ll_out, double* grad_out, void* ws,
                                      size_t ws_bytes, unsigned flags, void* stream);

/* ------------------------------------------------------------------------
 * The method as the paper writes it (Sec. 2.2-3.1): the explicit block-
 * tridiagonal posterior precision and a general symmetric BTD solver.
 *
 * These form Q_i^-1, whose condition number grows like (lam dt)^-(2b-2); they
 * are exact algebra but lose about 2(b-1) log10(1 / (lam dt_min)) digits, so
 * they are meant for well-separated times and for callers that bring their
 * own BTD matrices.  The entry points above never form Q^-1 and stay exact
 * for any gap, ties included.
 *
 * Block layout (b x b blocks, row-major, stored one after another):
 *   D[i] = T[i][i]      for i = 0 .. n-1   (n b^2 doubles, symmetric blocks)
 *   O[i] = T[i+1][i]    for i = 0 .. n-2   ((n-1) b^2 doubles; T[i][i+1] = O[i]^T)
 *   vectors r, x: n b doubles, entry i*b + k.
 * Same pointer, workspace, stream and status conventions as above; b <= 3.
 * ------------------------------------------------------------------------ */

/* Subproblems 1-3 of Sec. 3.1 for a symmetric positive-definite block-
 * tridiagonal T (the posterior precision K~ of Eq. mean3 is one): x = T^-1 r,
 * log det T, and, when Sdiag_out is not NULL, the block-tridiagonal part of
 * T^-1 (its diagonal blocks Sdiag_out[i] = (T^-1)[i][i], n b^2 doubles, and
 * sub-diagonal blocks Soff_out[i] = (T^-1)[i+1][i], (n-1) b^2 doubles;
 * Soff_out may be NULL only when n = 1) -- the selected inverse that
 * subproblems 2 and 4 need.  Odd-even block cyclic reduction: level l
 * eliminates the odd-numbered nodes of level l-1 by Schur complement, the
 * single node left is solved, and back-substitution recovers x and the
 * selected inverse level by level (2 ceil(log2 n) + 3 kernels).  A pivot
 * block that is not positive definite gives SPINGP_ENUMERIC.  logdet_out is
 * one device double. */
size_t spingp_btd_workspace_bytes(int b, int64_t n);
spingp_status spingp_btd_solve(int b, int64_t n, const double* D, const double* O, const double* r,
                               double* logdet_out, double* x_out, double* Sdiag_out, double* Soff_out, void* ws,
                               size_t ws_bytes, unsigned flags, void* stream);
int spingp_btd_launch_count(int64_t n);

/* Subproblem 4 of Sec. 3.1 (Eq. comp_2; Eq. dd1 is its trace): the diagonal
 * of S X, where S is the selected inverse from spingp_btd_solve (Sdiag, Soff)
 * and X a symmetric block-tridiagonal matrix in the layout above (Xdiag,
 * Xoff), together with its trace.  Only the block-tridiagonal part of S
 * enters.  diag_out (n b doubles) may be NULL; trace_out is one device
 * double, summed in a fixed order. */
size_t spingp_btd_diag_product_workspace_bytes(int64_t n);
spingp_status spingp_btd_diag_product(int b, int64_t n, const double* Sdiag, const double* Soff,
                                      const double* Xdiag, const double* Xoff, double* diag_out,
                                      double* trace_out, void* ws, size_t ws_bytes, unsigned flags, void* stream);

/* Assembly of the posterior precision K~ = Kinv + G^T Sigma^-1 G for a single
 * Matern component (Theorem 1 with Sec. 2.2), in the state coordinates of
 * Eq. ss1 (z = (f, f', f'', ...)):
 *   D_i = Q_{i-1}^-1 + A_i^T Q_i^-1 A_i + H^T H / sigma_n^2   (Q_{-1} = Pinf; no
 *         A-term for the last step),
 *   O_i = -Q_i^-1 A_i,   r_i = H^T y_i / sigma_n^2,
 * and logdet_kinv_out = log det Kinv = -log det Pinf - sum_i log det Q_i, the
 * term the determinant lemma (Eq. det_1) needs.  Times must be strictly
 * increasing (a tie makes Q_i = 0 and gives SPINGP_ENUMERIC); NaN inputs give
 * SPINGP_ENONFINITE. */
size_t spingp_assemble_workspace_bytes(int64_t n);
spingp_status spingp_assemble(const spingp_model* model, const double* t, const double* y, int64_t n,
                              const double* theta, double* D_out, double* O_out, double* r_out,
                              double* logdet_kinv_out, void* ws, size_t ws_bytes, unsigned flags, void* stream);

/* The whole computation the paper's way, for a single Matern component:
 * assembly, block cyclic reduction, then
 *   ll = -1/2 (y^T y / sigma_n^2 - r^T x) - 1/2 (log det K~ - log det Kinv
 *        + n log sigma_n^2) - n/2 log 2 pi                 (Eqs. ml2, det_1, mean3)
 * with x = K~^-1 r.  what = SPINGP_WS_GRAD adds the gradient (grad_out[3],
 * theta order) from Eq. dd1: for a covariance parameter,
 *   d ll = -1/2 x^T dK~ x - 1/2 tr(K~^-1 dK~) + 1/2 d log det Kinv,
 * where dK~ is block-tridiagonal, so the trace needs only the selected
 * inverse (subproblem 4).  what = SPINGP_WS_POSTERIOR writes the latent
 * posterior mean H x_i and variance H (K~^-1)_ii H^T (Eqs. mean3, k3).  Same
 * input rules as spingp_assemble. */
size_t spingp_literal_workspace_bytes(const spingp_model* model, int64_t n, spingp_ws_kind what);
spingp_status spingp_literal(const spingp_model* model, spingp_ws_kind what, const double* t, const double* y,
                             int64_t n, const double* theta, double* ll_out, double* grad_out, double* mean_out,
                             double* var_out, void* ws, size_t ws_bytes, unsigned flags, void* stream);
int spingp_literal_launch_count(int64_t n);

/* Synchronise the stream and return the device status recorded in ws by the
 * last call that used it (SPINGP_OK if none).  spingp_sync_status is the same
 * call under the name of a status read at a synchronisation point. */
spingp_status spingp_ws_status(void* ws, void* stream);
spingp_status spingp_sync_status(void* ws, void* stream);

const char* spingp_status_str(spingp_status status);

#ifdef __cplusplus
}
#endif

#endif /* SPINGP_H */
