// capi.cu -- the extern "C" boundary declared in include/spingp.h.
#include <cuda_runtime.h>
#include <cmath>
#include <math.h>
#include <mutex>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#include "spingp.h"
#include "internal.h"

#define SPG_MAXC 8
#define SPG_MAXDEV 64

// Stage-timing record: five events per call, reused across calls.
struct spg_prof {
    int on;
    int used;                      // calls recorded since the last read
    int cap;
    cudaEvent_t (*ev)[5];
};

struct spingp_model {
    int ncomp;
    int kinds[SPG_MAXC], orders[SPG_MAXC], envs[SPG_MAXC];
    int b, P;
    int chunk_len;   // 0 = default
    spg_prof* prof;  // NULL unless profiling was enabled
    int group;       // 1: structured model on the group path (spg::GModel below)
    spg::GModel gm;
    // host-buffer calls: a copy stream and its events, created on first use
    int feed_dev;    // device they belong to, -1 = none
    cudaStream_t feed_copy;
    cudaEvent_t feed_ev[1 + spg::FEED_PIECES];
};

namespace spg {
// The driver's unique ID of the current context (cuCtxGetId, reached through
// the runtime's driver entry point, so the library does not link the driver
// library itself); 0 if the driver does not provide it or no context is
// current.  Per-device state that a device reset invalidates is tagged with it.
unsigned long long context_id() {
    typedef int (*ctx_id_fn)(void*, unsigned long long*);   // CUresult cuCtxGetId(CUcontext, unsigned long long*)
    static const ctx_id_fn fn = [] {
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q = cudaDriverEntryPointSymbolNotFound;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetId", &p, 12000, cudaEnableDefault, &q) != cudaSuccess ||
            q != cudaDriverEntryPointSuccess)
            return (ctx_id_fn) nullptr;
        return (ctx_id_fn)p;
    }();
    unsigned long long id = 0;
    if (!fn || fn(nullptr, &id) != 0) return 0;
    return id;
}
}  // namespace spg

namespace {

std::mutex g_prep_mu;
bool g_prepared[SPG_MAXDEV];
unsigned long long g_prep_ctx[SPG_MAXDEV];

// per-device set-up (shared-memory opt-in of the scan kernels), once per
// context: a device reset destroys the context and the attributes with it
spingp_status prepare_device() {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= SPG_MAXDEV) return SPINGP_ECUDA;
    std::lock_guard<std::mutex> lock(g_prep_mu);
    if (!g_prepared[dev] || spg::context_id() != g_prep_ctx[dev]) {
        if (spg::matern_prepare()) return SPINGP_ECUDA;
        g_prepared[dev] = true;
        g_prep_ctx[dev] = spg::context_id();
    }
    return SPINGP_OK;
}

int matern_dim(int kind) { return kind; }

// SMs of the current device (152 on GB300), read once per device
int device_sms() {
    static int sms[SPG_MAXDEV];
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= SPG_MAXDEV) return 152;
    if (sms[dev] <= 0) {
        int v = 0;
        if (cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || v <= 0) v = 152;
        sms[dev] = v;
    }
    return sms[dev];
}

int64_t default_chunk(int64_t n) {
    // two blocks of 128 chunks per SM (the chain kernels run 128 threads per
    // block, one chunk per thread), L in [16, 512]
    const int64_t target = 2 * 128 * (int64_t)device_sms();
    int64_t L = (n + target - 1) / target;
    return L < 16 ? 16 : (L > 512 ? 512 : L);
}

int64_t default_group_chunk(int64_t n);

int64_t chunk_len(const spingp_model* m, int64_t n) {
    if (m->chunk_len > 0) return (int64_t)m->chunk_len;
    return m->group ? default_group_chunk(n) : default_chunk(n);
}

bool single_matern(const spingp_model* m) { return m->ncomp == 1 && m->kinds[0] >= 1 && m->kinds[0] <= 3; }

// Build the 2x2-block description for the group path; false if the model has
// a component that is not made of 2x2 blocks or is too large.
//
// The state lists the EQ component's sections first (when there is one), then
// the other components' blocks in component order: f sums the first
// coordinate of every block, so the order is internal, and with the EQ blocks
// at fixed positions the kernels index their coupling blocks at compile time.
bool build_group(spingp_model* m) {
    spg::GModel g;
    memset(&g, 0, sizeof(g));
    g.eq_comp = -1;
    if (m->ncomp > spg::GMAXCOMP) return false;
    int K = 0, P = 0, neq = 0;
    for (int c = 0; c < m->ncomp; ++c) neq += (m->kinds[c] == SPINGP_EQ);
    if (neq > 1) return false;                                  // one EQ component
    for (int c = 0; c < m->ncomp; ++c) {
        g.ckind[c] = m->kinds[c];
        g.cpoff[c] = P;
        const int k = m->kinds[c];
        P += (k == SPINGP_MATERN32 || k == SPINGP_EQ) ? 2 : (k == SPINGP_PERIODIC) ? 3 : 4;
    }
    for (int pass = 0; pass < 2; ++pass)
        for (int c = 0; c < m->ncomp; ++c) {
            const int k = m->kinds[c];
            if ((k == SPINGP_EQ) != (pass == 0)) continue;
            int nb, kind;
            if (k == SPINGP_MATERN32) { nb = 1; kind = 0; }
            else if (k == SPINGP_PERIODIC) { nb = m->orders[c] + 1; kind = 1; }
            else if (k == SPINGP_QUASIPERIODIC && m->envs[c] == SPINGP_MATERN12) { nb = m->orders[c] + 1; kind = 2; }
            else if (k == SPINGP_EQ) {
                const int N = m->orders[c];
                nb = N / 2; kind = 3;
                if (K + nb > spg::GMAXBLK) return false;
                double a[8], b[8], u[16], w[16], Pb[32];
                if (!spg::eq_cascade(N, a, b, u, w, Pb)) return false;
                g.eq_comp = c; g.eq_k0 = K; g.eq_nk = nb;
                for (int j = 0; j < nb; ++j) {
                    g.eqa[K + j] = a[j]; g.eqb[K + j] = b[j];
                    for (int q = 0; q < 2; ++q) { g.equ[2 * (K + j) + q] = u[2 * j + q]; g.eqw[2 * (K + j) + q] = w[2 * j + q]; }
                    for (int r = 0; r < 2; ++r)
                        for (int q = 0; q < 2; ++q) g.eqP[(2 * j + r) * 16 + 2 * j + q] = Pb[4 * j + 2 * r + q];
                }
            }
            else return false;
            for (int j = 0; j < nb; ++j) {
                if (K >= spg::GMAXBLK) return false;
                g.bkind[K] = kind; g.bcomp[K] = c; g.bj[K] = (kind == 0) ? 0 : j;
                ++K;
            }
        }
    for (int k = 1; k < g.eq_nk; ++k)
        for (int i = 0; i < k; ++i) {
            const double al = g.eqa[k] - g.eqa[i], bc = g.eqb[k] - g.eqb[i], ba = g.eqb[k] + g.eqb[i];
            g.eqrc[k * (k - 1) / 2 + i] = 1.0 / (al * al + bc * bc);
            g.eqra[k * (k - 1) / 2 + i] = 1.0 / (al * al + ba * ba);
        }
    g.phs = 4 * spg::GMAXBLK + 2 * g.eq_nk * (g.eq_nk - 1);
    g.K = K; g.b = 2 * K; g.P = P + 1; g.ncomp = m->ncomp;
    if (g.b != m->b || g.P != m->P) return false;
    m->gm = g;
    return true;
}

int64_t default_group_chunk(int64_t n) {
    // about 2400 chunk groups (16 lanes each) keep every SM busy
    int64_t L = (n + 2431) / 2432;
    return L < 4 ? 4 : (L > 4096 ? 4096 : L);
}

// the next five stage events of a profiled model (NULL when not profiling)
spingp_status profile_slot(const spingp_model* m, cudaEvent_t** ev) {
    *ev = NULL;
    spg_prof* pr = m->prof;
    if (!pr || !pr->on) return SPINGP_OK;
    if (pr->used == pr->cap) {
        const int cap = pr->cap ? 2 * pr->cap : 16;
        cudaEvent_t(*nev)[5] = (cudaEvent_t(*)[5])realloc(pr->ev, sizeof(cudaEvent_t[5]) * cap);
        if (!nev) return SPINGP_ENOMEM;
        for (int i = pr->cap; i < cap; ++i)
            for (int k = 0; k < 5; ++k)
                if (cudaEventCreate(&nev[i][k]) != cudaSuccess) return SPINGP_ECUDA;
        pr->ev = nev;
        pr->cap = cap;
    }
    *ev = pr->ev[pr->used++];
    return SPINGP_OK;
}

spingp_status run(const spingp_model* m, int mode, const double* t, const double* y, int64_t n,
                  const double* theta, double* ll, double* grad, double* mean, double* var, void* ws,
                  size_t ws_bytes, unsigned flags, void* stream, double* lag1 = nullptr) {
    if (!m || !t || !y || !theta || !ws || n < 1) return SPINGP_EINVAL;
    if (((uintptr_t)ws & 255u) != 0) return SPINGP_EINVAL;
    if (!single_matern(m) && !m->group) return SPINGP_EUNSUPPORTED;
    const int64_t L = chunk_len(m, n);
    const size_t need = m->group ? spg::group_ws_bytes(m->gm, n, L, mode) : spg::matern_ws_bytes(m->b, n, L, mode);
    if (ws_bytes < need) return SPINGP_EINVAL;
    spingp_status st = prepare_device();
    if (st != SPINGP_OK) return st;
    cudaStream_t s = (cudaStream_t)stream;
    cudaEvent_t* ev = NULL;
    st = profile_slot(m, &ev);
    if (st != SPINGP_OK) return st;
    const int miss = (flags & SPINGP_MISSING_NAN) ? 1 : 0;
    int rc = m->group ? spg::group_run(m->gm, mode, t, y, n, L, theta, ll, grad, mean, var, ws, s, ev, miss, lag1)
                      : spg::matern_run(m->b, mode, t, y, n, L, theta, ll, grad, mean, var, ws, s, ev, miss, nullptr, lag1);
    if (!rc && grad && (flags & SPINGP_LOG_GRAD)) rc = spg::grad_to_log(grad, theta, m->P, s);
    if (!rc && var && (flags & SPINGP_PREDICTIVE)) rc = spg::add_noise(var, n, theta + m->P - 1, s);
    if (rc) return SPINGP_ECUDA;
    if (flags & SPINGP_SYNC) return spingp_ws_status(ws, stream);
    return SPINGP_OK;
}

int64_t chunk_len_batched(const spingp_model* m, int64_t n_series, int64_t n_total) {
    if (m->chunk_len > 0) return m->chunk_len;
    // the single-series default for the whole batch, at most half the mean length
    int64_t L = default_chunk(n_total);
    const int64_t mean_len = n_series > 0 ? n_total / n_series : n_total;
    while (L > 16 && 2 * L > mean_len) L /= 2;
    return L;
}

int ws_mode(spingp_ws_kind what) {
    return what == SPINGP_WS_GRAD ? spg::MODE_GRAD : what == SPINGP_WS_POSTERIOR ? spg::MODE_POSTERIOR
                                                                                   : spg::MODE_LOGLIK;
}

spingp_status run_batched(const spingp_model* m, int mode, const int64_t* offsets, int64_t n_series,
                          int64_t n_total, const double* t, const double* y, const double* theta, double* ll,
                          double* grad, double* mean, double* var, void* ws, size_t ws_bytes, unsigned flags,
                          void* stream) {
    if (!m || !offsets || !theta || !ws || n_series < 1 || n_total < 0) return SPINGP_EINVAL;
    if (n_total > 0 && (!t || !y)) return SPINGP_EINVAL;
    if (((uintptr_t)ws & 255u) != 0) return SPINGP_EINVAL;
    if (!single_matern(m)) return SPINGP_EUNSUPPORTED;
    const int64_t L = chunk_len_batched(m, n_series, n_total);
    if (ws_bytes < spg::matern_ws_bytes_batched(m->b, n_series, n_total, L, mode)) return SPINGP_EINVAL;
    spingp_status st = prepare_device();
    if (st != SPINGP_OK) return st;
    cudaStream_t s = (cudaStream_t)stream;
    cudaEvent_t* ev = NULL;
    st = profile_slot(m, &ev);
    if (st != SPINGP_OK) return st;
    if (spg::matern_run_batched(m->b, mode, offsets, n_series, n_total, t, y, L, theta, ll, grad, mean, var, ws, s,
                                ev, (flags & SPINGP_MISSING_NAN) ? 1 : 0))
        return SPINGP_ECUDA;
    if (grad && (flags & SPINGP_LOG_GRAD) && spg::grad_to_log(grad, theta, n_series * m->P, s)) return SPINGP_ECUDA;
    if (var && (flags & SPINGP_PREDICTIVE) && spg::add_noise_batched(var, offsets, n_series, theta, m->P, s))
        return SPINGP_ECUDA;
    if (flags & SPINGP_SYNC) return spingp_ws_status(ws, stream);
    return SPINGP_OK;
}

}  // namespace

namespace spg {
bool model_on_chain_path(const spingp_model* m) { return m && !m->group && single_matern(m); }
}  // namespace spg

extern "C" {

size_t spingp_workspace_bytes_batched(const spingp_model* m, int64_t n_series, int64_t n_total,
                                      spingp_ws_kind what) {
    if (!m || n_series < 1 || n_total < 0 || !single_matern(m)) return 0;
    return spg::matern_ws_bytes_batched(m->b, n_series, n_total, chunk_len_batched(m, n_series, n_total),
                                        ws_mode(what));
}

spingp_status spingp_loglik_batched(const spingp_model* m, const int64_t* offsets, int64_t n_series,
                                    int64_t n_total, const double* t, const double* y, const double* theta,
                                    double* ll_out, void* ws, size_t ws_bytes, unsigned flags, void* stream) {
    if (!ll_out) return SPINGP_EINVAL;
    return run_batched(m, spg::MODE_LOGLIK, offsets, n_series, n_total, t, y, theta, ll_out, NULL, NULL, NULL, ws,
                       ws_bytes, flags, stream);
}

spingp_status spingp_grad_batched(const spingp_model* m, const int64_t* offsets, int64_t n_series,
                                  int64_t n_total, const double* t, const double* y, const double* theta,
                                  double* ll_out, double* grad_out, void* ws, size_t ws_bytes, unsigned flags,
                                  void* stream) {
    if (!ll_out || !grad_out) return SPINGP_EINVAL;
    return run_batched(m, spg::MODE_GRAD, offsets, n_series, n_total, t, y, theta, ll_out, grad_out, NULL, NULL,
                       ws, ws_bytes, flags, stream);
}

spingp_status spingp_posterior_batched(const spingp_model* m, const int64_t* offsets, int64_t n_series,
                                       int64_t n_total, const double* t, const double* y, const double* theta,
                                       double* ll_out, double* mean_out, double* var_out, void* ws,
                                       size_t ws_bytes, unsigned flags, void* stream) {
    if (n_total > 0 && (!mean_out || !var_out)) return SPINGP_EINVAL;
    return run_batched(m, spg::MODE_POSTERIOR, offsets, n_series, n_total, t, y, theta, ll_out, NULL, mean_out,
                       var_out, ws, ws_bytes, flags, stream);
}

spingp_status spingp_grad_posterior_batched(const spingp_model* m, const int64_t* offsets, int64_t n_series,
                                            int64_t n_total, const double* t, const double* y, const double* theta,
                                            double* ll_out, double* grad_out, double* mean_out, double* var_out,
                                            void* ws, size_t ws_bytes, unsigned flags, void* stream) {
    if (!ll_out || !grad_out || (n_total > 0 && (!mean_out || !var_out))) return SPINGP_EINVAL;
    return run_batched(m, spg::MODE_GRAD_POSTERIOR, offsets, n_series, n_total, t, y, theta, ll_out, grad_out,
                       mean_out, var_out, ws, ws_bytes, flags, stream);
}


spingp_status spingp_model_create(const spingp_model_desc* d, spingp_model** out) {
    if (!out) return SPINGP_EINVAL;
    *out = NULL;
    if (!d || d->n_comp < 1 || d->n_comp > SPG_MAXC || !d->kinds) return SPINGP_EINVAL;
    spingp_model m;
    memset(&m, 0, sizeof(m));
    m.ncomp = d->n_comp;
    for (int c = 0; c < d->n_comp; ++c) {
        const int k = d->kinds[c];
        const int J = d->orders ? d->orders[c] : 0;
        const int env = d->envs ? d->envs[c] : 0;
        m.kinds[c] = k; m.orders[c] = J; m.envs[c] = env;
        if (k >= SPINGP_MATERN12 && k <= SPINGP_MATERN52) { m.b += matern_dim(k); m.P += 2; }
        else if (k == SPINGP_PERIODIC) { if (J < 0 || J > 64) return SPINGP_EINVAL; m.b += 2 * (J + 1); m.P += 3; }
        else if (k == SPINGP_QUASIPERIODIC) {
            if (J < 0 || J > 64 || env < SPINGP_MATERN12 || env > SPINGP_MATERN52) return SPINGP_EINVAL;
            m.b += 2 * (J + 1) * matern_dim(env); m.P += 4;
        } else if (k == SPINGP_EQ) {
            if (J < 2 || J > 16 || (J & 1)) return SPINGP_EINVAL;
            m.b += J; m.P += 2;
        } else return SPINGP_EINVAL;
    }
    m.P += 1;
    m.feed_dev = -1;
    if (!single_matern(&m)) {
        if (!build_group(&m)) return SPINGP_EUNSUPPORTED;
        m.group = 1;
    }
    spingp_model* h = (spingp_model*)malloc(sizeof(spingp_model));
    if (!h) return SPINGP_ENOMEM;
    *h = m;
    *out = h;
    return SPINGP_OK;
}

void spingp_model_destroy(spingp_model* m) {
    if (!m) return;
    if (m->feed_dev >= 0) {
        int cur = 0;
        cudaGetDevice(&cur);
        cudaSetDevice(m->feed_dev);
        cudaStreamDestroy(m->feed_copy);
        for (int i = 0; i <= spg::FEED_PIECES; ++i) cudaEventDestroy(m->feed_ev[i]);
        cudaSetDevice(cur);
    }
    if (m->prof) {
        for (int i = 0; i < m->prof->cap; ++i)
            for (int k = 0; k < 5; ++k) cudaEventDestroy(m->prof->ev[i][k]);
        free(m->prof->ev);
        free(m->prof);
    }
    free(m);
}

int spingp_num_params(const spingp_model* m) { return m ? m->P : -1; }
int spingp_state_dim(const spingp_model* m) { return m ? m->b : -1; }

spingp_status spingp_set_chunk_len(spingp_model* m, int L) {
    if (!m || (L != 0 && (L < 8 || L > 65536))) return SPINGP_EINVAL;
    m->chunk_len = L;
    return SPINGP_OK;
}

int spingp_get_chunk_len(const spingp_model* m, int64_t n) { return m ? (int)chunk_len(m, n) : -1; }

size_t spingp_workspace_bytes(const spingp_model* m, int64_t n, spingp_ws_kind what) {
    if (!m || n < 1) return 0;
    const int mode = what == SPINGP_WS_GRAD ? spg::MODE_GRAD
                   : what == SPINGP_WS_POSTERIOR ? spg::MODE_POSTERIOR : spg::MODE_LOGLIK;
    if (m->group) return spg::group_ws_bytes(m->gm, n, chunk_len(m, n), mode);
    if (!single_matern(m)) return 0;
    return spg::matern_ws_bytes(m->b, n, chunk_len(m, n), mode);
}

spingp_status spingp_loglik(const spingp_model* m, const double* t, const double* y, int64_t n,
                            const double* theta, double* ll_out, void* ws, size_t ws_bytes, unsigned flags,
                            void* stream) {
    if (!ll_out) return SPINGP_EINVAL;
    return run(m, spg::MODE_LOGLIK, t, y, n, theta, ll_out, NULL, NULL, NULL, ws, ws_bytes, flags, stream);
}

spingp_status spingp_grad(const spingp_model* m, const double* t, const double* y, int64_t n, const double* theta,
                          double* ll_out, double* grad_out, void* ws, size_t ws_bytes, unsigned flags,
                          void* stream) {
    if (!ll_out || !grad_out) return SPINGP_EINVAL;
    return run(m, spg::MODE_GRAD, t, y, n, theta, ll_out, grad_out, NULL, NULL, ws, ws_bytes, flags, stream);
}

spingp_status spingp_posterior(const spingp_model* m, const double* t, const double* y, int64_t n,
                               const double* theta, double* ll_out, double* mean_out, double* var_out, void* ws,
                               size_t ws_bytes, unsigned flags, void* stream) {
    if (!mean_out || !var_out) return SPINGP_EINVAL;
    return run(m, spg::MODE_POSTERIOR, t, y, n, theta, ll_out, NULL, mean_out, var_out, ws, ws_bytes, flags,
               stream);
}

spingp_status spingp_posterior_lag1(const spingp_model* m, const double* t, const double* y, int64_t n,
                                    const double* theta, double* ll_out, double* mean_out, double* var_out,
                                    double* cov_lag1_out, void* ws, size_t ws_bytes, unsigned flags, void* stream) {
    if (!mean_out || !var_out || (n > 1 && !cov_lag1_out)) return SPINGP_EINVAL;
    return run(m, spg::MODE_POSTERIOR, t, y, n, theta, ll_out, NULL, mean_out, var_out, ws, ws_bytes, flags,
               stream, n > 1 ? cov_lag1_out : nullptr);
}

spingp_status spingp_grad_posterior(const spingp_model* m, const double* t, const double* y, int64_t n,
                                    const double* theta, double* ll_out, double* grad_out, double* mean_out,
                                    double* var_out, double* cov_lag1_out, void* ws, size_t ws_bytes,
                                    unsigned flags, void* stream) {
    if (!ll_out || !grad_out || !mean_out || !var_out) return SPINGP_EINVAL;
    return run(m, spg::MODE_GRAD_POSTERIOR, t, y, n, theta, ll_out, grad_out, mean_out, var_out, ws, ws_bytes,
               flags, stream, n > 1 ? cov_lag1_out : nullptr);
}

size_t spingp_predict_workspace_bytes(const spingp_model* m, int64_t n, int64_t n_star) {
    if (!m || n < 0 || n_star < 1) return 0;
    const size_t inner = spingp_workspace_bytes(m, n + n_star, SPINGP_WS_POSTERIOR);
    if (inner == 0) return 0;
    return spg::PredictLayout(n, n_star).off_inner + inner;
}

spingp_status spingp_predict(const spingp_model* m, const double* t, const double* y, int64_t n,
                             const double* theta, const double* t_star, int64_t n_star, double* mean_out,
                             double* var_out, void* ws, size_t ws_bytes, unsigned flags, void* stream) {
    if (!m || !theta || !t_star || !mean_out || !var_out || !ws || n < 0 || n_star < 1) return SPINGP_EINVAL;
    if (n > 0 && (!t || !y)) return SPINGP_EINVAL;
    if (((uintptr_t)ws & 255u) != 0) return SPINGP_EINVAL;
    const size_t need = spingp_predict_workspace_bytes(m, n, n_star);
    if (need == 0) return SPINGP_EUNSUPPORTED;
    if (ws_bytes < need) return SPINGP_EINVAL;
    spingp_status st = prepare_device();
    if (st != SPINGP_OK) return st;
    cudaStream_t s = (cudaStream_t)stream;
    const spg::PredictLayout lay(n, n_star);
    char* w = (char*)ws;
    if (spg::predict_prepare(t, y, n, t_star, n_star, ws, lay, s)) return SPINGP_ECUDA;
    // the posterior over the merged series; a test point's NaN observation is missing
    const unsigned inner_flags = SPINGP_MISSING_NAN | (flags & SPINGP_PREDICTIVE);
    st = run(m, spg::MODE_POSTERIOR, (const double*)(w + lay.off_T), (const double*)(w + lay.off_Y), n + n_star,
             theta, NULL, NULL, (double*)(w + lay.off_mean), (double*)(w + lay.off_var), w + lay.off_inner,
             ws_bytes - lay.off_inner, inner_flags, stream);
    if (st != SPINGP_OK) return st;
    if (spg::predict_finish(t, n, n_star, ws, lay, mean_out, var_out, s)) return SPINGP_ECUDA;
    if (flags & SPINGP_SYNC) return spingp_ws_status(ws, stream);
    return SPINGP_OK;
}

int spingp_launch_count(const spingp_model* m, int64_t n, spingp_ws_kind what) {
    if (!m || n < 1) return -1;
    const int mode = what == SPINGP_WS_GRAD ? spg::MODE_GRAD
                   : what == SPINGP_WS_POSTERIOR ? spg::MODE_POSTERIOR : spg::MODE_LOGLIK;
    if (m->group) return spg::group_launch_count(n, chunk_len(m, n), mode);
    if (!single_matern(m)) return -1;
    return spg::matern_launch_count(m->b, n, chunk_len(m, n), mode);
}

int spingp_launch_count_batched(const spingp_model* m, int64_t n_series, int64_t n_total, spingp_ws_kind what) {
    if (!m || n_series < 1 || n_total < 0 || !single_matern(m)) return -1;
    return spg::matern_launch_count_batched(m->b, n_series, n_total, chunk_len_batched(m, n_series, n_total),
                                            ws_mode(what));
}

spingp_status spingp_profile_enable(spingp_model* m, int on) {
    if (!m) return SPINGP_EINVAL;
    if (!m->prof) {
        m->prof = (spg_prof*)calloc(1, sizeof(spg_prof));
        if (!m->prof) return SPINGP_ENOMEM;
    }
    m->prof->on = on ? 1 : 0;
    return SPINGP_OK;
}

spingp_status spingp_profile_read(spingp_model* m, double* ms_out, int* calls) {
    if (!m || !ms_out) return SPINGP_EINVAL;
    for (int k = 0; k < 4; ++k) ms_out[k] = 0.0;
    if (calls) *calls = 0;
    spg_prof* pr = m->prof;
    if (!pr) return SPINGP_OK;
    for (int i = 0; i < pr->used; ++i) {
        if (cudaEventSynchronize(pr->ev[i][4]) != cudaSuccess) return SPINGP_ECUDA;
        for (int k = 0; k < 4; ++k) {
            float ms = 0.0f;
            if (cudaEventElapsedTime(&ms, pr->ev[i][k], pr->ev[i][k + 1]) != cudaSuccess) return SPINGP_ECUDA;
            ms_out[k] += ms;
        }
    }
    if (calls) *calls = pr->used;
    pr->used = 0;
    return SPINGP_OK;
}

size_t spingp_probe_fp64_bytes(void) { return spg::probe_fp64_bytes(); }

spingp_status spingp_probe_fp64(void* scratch, size_t bytes, double* tflops_out, void* stream) {
    if (!scratch || !tflops_out) return SPINGP_EINVAL;
    return spg::probe_fp64(scratch, bytes, tflops_out, (cudaStream_t)stream, 0) ? SPINGP_ECUDA : SPINGP_OK;
}

spingp_status spingp_probe_fp64_tensor(void* scratch, size_t bytes, double* tflops_out, void* stream) {
    if (!scratch || !tflops_out) return SPINGP_EINVAL;
    return spg::probe_fp64(scratch, bytes, tflops_out, (cudaStream_t)stream, 1) ? SPINGP_ECUDA : SPINGP_OK;
}

spingp_status spingp_probe_exp_neg(const double* x, double* y, int64_t n, void* stream) {
    if (n < 0 || (n > 0 && (!x || !y))) return SPINGP_EINVAL;
    return spg::probe_exp_neg(x, y, n, (cudaStream_t)stream) ? SPINGP_ECUDA : SPINGP_OK;
}

// ---------------------------------------------------------------- a series split across ranks

int spingp_segment_elem_size(const spingp_model* m) {
    if (!m) return -1;
    if (single_matern(m)) return spg::matern_elem_size(m->b);
    return m->group ? spg::group_elem_size() : -1;
}

int spingp_segment_launch_count(const spingp_model* m, int64_t n) {
    if (!m || n < 1) return -1;
    if (single_matern(m)) return spg::matern_segment_launch_count(m->b, n, chunk_len(m, n));
    return m->group ? spg::group_segment_launch_count(n, chunk_len(m, n)) : -1;
}

static spingp_status segment_call(const spingp_model* m, int phase, const double* t, const double* y, int64_t n,
                                  const double* theta, double t_prev, int first, const double* elems, int n_ranks,
                                  int rank, double* elem_out, double* ll_out, double* grad_out, void* ws,
                                  size_t ws_bytes, unsigned flags, void* stream, double* mean_out = nullptr,
                                  double* var_out = nullptr) {
    if (!m || !t || !y || !theta || !ws || n < 1) return SPINGP_EINVAL;
    if (!single_matern(m) && !m->group) return SPINGP_EUNSUPPORTED;
    if (((uintptr_t)ws & 255u) != 0) return SPINGP_EINVAL;
    if (!first && !std::isfinite(t_prev)) return SPINGP_EINVAL;
    const int64_t L = chunk_len(m, n);
    const size_t need = m->group ? spg::group_ws_bytes(m->gm, n, L, spg::MODE_GRAD) : spg::matern_ws_bytes(m->b, n, L, spg::MODE_GRAD);
    if (ws_bytes < need) return SPINGP_EINVAL;
    spingp_status st = prepare_device();
    if (st != SPINGP_OK) return st;
    const int miss = (flags & SPINGP_MISSING_NAN) ? 1 : 0;
    const double tp = first ? 0.0 : t_prev;
    int rc = m->group ? spg::group_segment(m->gm, phase, t, y, n, L, theta, tp, first ? 1 : 0, elems, n_ranks,
                                           rank, elem_out, ll_out, grad_out, ws, (cudaStream_t)stream, miss,
                                           mean_out, var_out)
                      : spg::matern_segment(m->b, phase, t, y, n, L, theta, tp, first ? 1 : 0, elems, n_ranks,
                                            rank, elem_out, ll_out, grad_out, ws, (cudaStream_t)stream, miss,
                                            mean_out, var_out);
    // the shares are linear in the gradient, so each scales on its own
    if (!rc && grad_out && (flags & SPINGP_LOG_GRAD)) rc = spg::grad_to_log(grad_out, theta, m->P, (cudaStream_t)stream);
    if (!rc && var_out && (flags & SPINGP_PREDICTIVE))
        rc = spg::add_noise(var_out, n, theta + m->P - 1, (cudaStream_t)stream);
    if (rc) return SPINGP_ECUDA;
    if (flags & SPINGP_SYNC) return spingp_ws_status(ws, stream);
    return SPINGP_OK;
}

spingp_status spingp_segment_reduce(const spingp_model* m, const double* t, const double* y, int64_t n,
                                    const double* theta, double t_prev, int first, double* elem_out, void* ws,
                                    size_t ws_bytes, unsigned flags, void* stream) {
    if (!elem_out) return SPINGP_EINVAL;
    return segment_call(m, 0, t, y, n, theta, t_prev, first, NULL, 1, 0, elem_out, NULL, NULL, ws, ws_bytes, flags,
                        stream);
}

spingp_status spingp_segment_grad(const spingp_model* m, const double* t, const double* y, int64_t n,
                                  const double* theta, double t_prev, int first, const double* elems, int n_ranks,
                                  int rank, double* ll_out, double* grad_out, void* ws, size_t ws_bytes,
                                  unsigned flags, void* stream) {
    if (!elems || !ll_out || !grad_out) return SPINGP_EINVAL;
    if (n_ranks < 1 || n_ranks > spg::SEG_MAX_RANKS || rank < 0 || rank >= n_ranks) return SPINGP_EINVAL;
    if ((first != 0) != (rank == 0)) return SPINGP_EINVAL;
    return segment_call(m, 1, t, y, n, theta, t_prev, first, elems, n_ranks, rank, NULL, ll_out, grad_out, ws,
                        ws_bytes, flags, stream);
}

spingp_status spingp_segment_grad_posterior(const spingp_model* m, const double* t, const double* y, int64_t n,
                                            const double* theta, double t_prev, int first, const double* elems,
                                            int n_ranks, int rank, double* ll_out, double* grad_out,
                                            double* mean_out, double* var_out, void* ws, size_t ws_bytes,
                                            unsigned flags, void* stream) {
    if (!elems || !ll_out || !grad_out || !mean_out || !var_out) return SPINGP_EINVAL;
    if (n_ranks < 1 || n_ranks > spg::SEG_MAX_RANKS || rank < 0 || rank >= n_ranks) return SPINGP_EINVAL;
    if ((first != 0) != (rank == 0)) return SPINGP_EINVAL;
    return segment_call(m, 1, t, y, n, theta, t_prev, first, elems, n_ranks, rank, NULL, ll_out, grad_out, ws,
                        ws_bytes, flags, stream, mean_out, var_out);
}

// ---------------------------------------------------------------- host buffers in, host results out

static size_t align256c(size_t x) { return (x + 255) & ~(size_t)255; }

static size_t hostws_chain(const spingp_model* m, int64_t n) {
    return align256c(spingp_workspace_bytes(m, n, SPINGP_WS_GRAD));
}

size_t spingp_workspace_bytes_host(const spingp_model* m, int64_t n) {
    if (!m || n < 1) return 0;
    const size_t base = spingp_workspace_bytes(m, n, SPINGP_WS_GRAD);
    if (base == 0) return 0;
    return hostws_chain(m, n) + 2 * align256c(sizeof(double) * (size_t)n) + 2 * align256c(sizeof(double) * 64);
}

static spingp_status feed_ready(spingp_model* m) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return SPINGP_ECUDA;
    if (m->feed_dev == dev) return SPINGP_OK;
    if (m->feed_dev >= 0) return SPINGP_EINVAL;   // the model's copy stream lives on another device
    if (cudaStreamCreateWithFlags(&m->feed_copy, cudaStreamNonBlocking) != cudaSuccess) return SPINGP_ECUDA;
    for (int i = 0; i <= spg::FEED_PIECES; ++i)
        if (cudaEventCreateWithFlags(&m->feed_ev[i], cudaEventDisableTiming) != cudaSuccess) return SPINGP_ECUDA;
    m->feed_dev = dev;
    return SPINGP_OK;
}

spingp_status spingp_grad_host(spingp_model* m, const double* t, const double* y, int64_t n, const double* theta,
                               double* ll_out, double* grad_out, void* ws, size_t ws_bytes, unsigned flags,
                               void* stream) {
    if (!m || !t || !y || !theta || !ll_out || !grad_out || !ws || n < 1) return SPINGP_EINVAL;
    if (((uintptr_t)ws & 255u) != 0) return SPINGP_EINVAL;
    if (!single_matern(m) && !m->group) return SPINGP_EUNSUPPORTED;
    const size_t need = spingp_workspace_bytes_host(m, n);
    if (need == 0 || ws_bytes < need) return SPINGP_EINVAL;
    spingp_status st = prepare_device();
    if (st != SPINGP_OK) return st;
    if ((st = feed_ready(m)) != SPINGP_OK) return st;
    cudaStream_t s = (cudaStream_t)stream;
    char* w = (char*)ws;
    const size_t o_t = hostws_chain(m, n), o_y = o_t + align256c(sizeof(double) * (size_t)n);
    const size_t o_th = o_y + align256c(sizeof(double) * (size_t)n), o_out = o_th + align256c(sizeof(double) * 64);
    double *td = (double*)(w + o_t), *yd = (double*)(w + o_y), *thd = (double*)(w + o_th), *od = (double*)(w + o_out);
    cudaEvent_t* ev = NULL;
    if ((st = profile_slot(m, &ev)) != SPINGP_OK) return st;
    const int miss = (flags & SPINGP_MISSING_NAN) ? 1 : 0;
    const int64_t L = chunk_len(m, n);
    int rc;
    if (m->group) {
        if (cudaMemcpyAsync(thd, theta, sizeof(double) * m->P, cudaMemcpyHostToDevice, s) != cudaSuccess ||
            cudaMemcpyAsync(td, t, sizeof(double) * n, cudaMemcpyHostToDevice, s) != cudaSuccess ||
            cudaMemcpyAsync(yd, y, sizeof(double) * n, cudaMemcpyHostToDevice, s) != cudaSuccess)
            return SPINGP_ECUDA;
        rc = spg::group_run(m->gm, spg::MODE_GRAD, td, yd, n, L, thd, od, od + 1, NULL, NULL, ws, s, ev, miss);
    } else {
        spg::HostFeed f;
        f.t = t; f.y = y; f.copy = m->feed_copy; f.npieces = spg::FEED_PIECES;
        f.theta_h = theta; f.theta_bytes = sizeof(double) * m->P;   // on the copy stream, ahead of t
        for (int i = 0; i <= spg::FEED_PIECES; ++i) f.ev[i] = m->feed_ev[i];
        rc = spg::matern_run(m->b, spg::MODE_GRAD, td, yd, n, L, thd, od, od + 1, NULL, NULL, ws, s, ev, miss, &f);
    }
    if (!rc && (flags & SPINGP_LOG_GRAD)) rc = spg::grad_to_log(od + 1, thd, m->P, s);
    if (rc) return SPINGP_ECUDA;
    if (cudaMemcpyAsync(ll_out, od, sizeof(double), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaMemcpyAsync(grad_out, od + 1, sizeof(double) * m->P, cudaMemcpyDeviceToHost, s) != cudaSuccess)
        return SPINGP_ECUDA;
    if (flags & SPINGP_SYNC) return spingp_ws_status(ws, stream);
    return SPINGP_OK;
}

// ---------------------------------------------------------------- hyperparameter fitting (Sec. 4.3)

static size_t optimize_inner_bytes(const spingp_model* m, bool batched, int64_t S, int64_t n) {
    return batched ? spingp_workspace_bytes_batched(m, S, n, SPINGP_WS_GRAD)
                   : spingp_workspace_bytes(m, n, SPINGP_WS_GRAD);
}

static spingp_status optimize(const spingp_model* m, bool batched, const int64_t* offsets, int64_t S, int64_t n,
                              const double* t, const double* y, double* theta, int iters, double tol,
                              double* ll_out, double* grad_out, void* ws, size_t ws_bytes, unsigned flags,
                              void* stream) {
    if (!m || !theta || !ws || iters < 0 || !(tol >= 0.0) || S < 1) return SPINGP_EINVAL;
    if (((uintptr_t)ws & 255u) != 0) return SPINGP_EINVAL;
    const size_t inner = optimize_inner_bytes(m, batched, S, n);
    if (inner == 0) return batched ? SPINGP_EUNSUPPORTED : SPINGP_EINVAL;
    const size_t off = align256c(inner);
    if (ws_bytes < off + spg::scg_state_bytes(S, m->P)) return SPINGP_EINVAL;
    spingp_status st = prepare_device();
    if (st != SPINGP_OK) return st;
    cudaStream_t s = (cudaStream_t)stream;
    const spg::ScgState sc = spg::scg_bind((char*)ws + off, S, m->P);
    const unsigned inner_flags = flags & ~SPINGP_SYNC;
    auto eval = [&]() -> spingp_status {
        return batched ? run_batched(m, spg::MODE_GRAD, offsets, S, n, t, y, sc.theta_eval, sc.ll_eval, sc.grad_eval,
                                     NULL, NULL, ws, inner, inner_flags, stream)
                       : run(m, spg::MODE_GRAD, t, y, n, sc.theta_eval, sc.ll_eval, sc.grad_eval, NULL, NULL, ws,
                             inner, inner_flags, stream);
    };
    auto kern = [&](int what, int k) {
        return spg::scg_launch(what, sc, s, k, tol, theta, theta, ll_out, grad_out, (int*)ws) ? SPINGP_ECUDA
                                                                                              : SPINGP_OK;
    };
#define SPG_TRY(x) do { const spingp_status e_ = (x); if (e_ != SPINGP_OK) return e_; } while (0)
    SPG_TRY(kern(spg::SCG_K_INIT, 0));
    SPG_TRY(eval());
    SPG_TRY(kern(spg::SCG_K_START, 0));
    for (int k = 1; k <= iters; ++k) {
        SPG_TRY(kern(spg::SCG_K_A, k));
        SPG_TRY(eval());
        SPG_TRY(kern(spg::SCG_K_B, k));
        SPG_TRY(eval());
        SPG_TRY(kern(spg::SCG_K_C, k));
    }
    SPG_TRY(kern(spg::SCG_K_FINAL, 0));
    SPG_TRY(eval());
    SPG_TRY(kern(spg::SCG_K_OUT, 0));
#undef SPG_TRY
    if (flags & SPINGP_SYNC) return spingp_ws_status(ws, stream);
    return SPINGP_OK;
}

size_t spingp_optimize_workspace_bytes(const spingp_model* m, int64_t n) {
    if (!m || n < 1) return 0;
    const size_t inner = optimize_inner_bytes(m, false, 1, n);
    return inner ? align256c(inner) + spg::scg_state_bytes(1, m->P) : 0;
}

spingp_status spingp_optimize(const spingp_model* m, const double* t, const double* y, int64_t n,
                              double* theta_inout, int iterations, double tol, double* ll_out, double* grad_out,
                              void* ws, size_t ws_bytes, unsigned flags, void* stream) {
    if (!t || !y || n < 1) return SPINGP_EINVAL;
    return optimize(m, false, NULL, 1, n, t, y, theta_inout, iterations, tol, ll_out, grad_out, ws, ws_bytes, flags,
                    stream);
}

size_t spingp_optimize_workspace_bytes_batched(const spingp_model* m, int64_t n_series, int64_t n_total) {
    if (!m || n_series < 1 || n_total < 0) return 0;
    const size_t inner = optimize_inner_bytes(m, true, n_series, n_total);
    return inner ? align256c(inner) + spg::scg_state_bytes(n_series, m->P) : 0;
}

spingp_status spingp_optimize_batched(const spingp_model* m, const int64_t* offsets, int64_t n_series,
                                      int64_t n_total, const double* t, const double* y, double* theta_inout,
                                      int iterations, double tol, double* ll_out, double* grad_out, void* ws,
                                      size_t ws_bytes, unsigned flags, void* stream) {
    if (!offsets) return SPINGP_EINVAL;
    return optimize(m, true, offsets, n_series, n_total, t, y, theta_inout, iterations, tol, ll_out, grad_out, ws,
                    ws_bytes, flags, stream);
}

// ---------------------------------------------------------------- the method as written (Sec. 2.2, 3.1)

static bool ws_ok(const void* ws, size_t have, size_t need) {
    return ws && ((uintptr_t)ws & 255u) == 0 && have >= need;
}
static spingp_status finish(int rc, void* ws, unsigned flags, void* stream) {
    if (rc) return SPINGP_ECUDA;
    if (flags & SPINGP_SYNC) return spingp_ws_status(ws, stream);
    return SPINGP_OK;
}

size_t spingp_btd_workspace_bytes(int b, int64_t n) {
    if (b < 1 || b > 3 || n < 1) return 0;
    return spg::btd_ws_bytes(b, n);
}

spingp_status spingp_btd_solve(int b, int64_t n, const double* D, const double* O, const double* r,
                               double* logdet_out, double* x_out, double* Sdiag_out, double* Soff_out, void* ws,
                               size_t ws_bytes, unsigned flags, void* stream) {
    if (b < 1 || b > 3 || n < 1 || !D || !r || !logdet_out || !x_out) return SPINGP_EINVAL;
    if (n > 1 && !O) return SPINGP_EINVAL;
    if (!Sdiag_out && Soff_out) return SPINGP_EINVAL;          // the selected inverse is wanted whole or not at all
    if (Sdiag_out && n > 1 && !Soff_out) return SPINGP_EINVAL;
    if (!ws_ok(ws, ws_bytes, spg::btd_ws_bytes(b, n))) return SPINGP_EINVAL;
    spingp_status st = prepare_device();
    if (st != SPINGP_OK) return st;
    // at n = 1 there is no off-diagonal block: a dummy pointer keeps the
    // selected inverse switched on without being written
    double* so = (n == 1 && Sdiag_out) ? Sdiag_out : Soff_out;
    return finish(spg::btd_solve(b, n, D, O, r, logdet_out, x_out, Sdiag_out, so, ws, (cudaStream_t)stream), ws,
                  flags, stream);
}

size_t spingp_btd_diag_product_workspace_bytes(int64_t n) { return n < 1 ? 0 : spg::diagprod_ws_bytes(n); }

spingp_status spingp_btd_diag_product(int b, int64_t n, const double* Sdiag, const double* Soff,
                                      const double* Xdiag, const double* Xoff, double* diag_out,
                                      double* trace_out, void* ws, size_t ws_bytes, unsigned flags, void* stream) {
    if (b < 1 || b > 3 || n < 1 || !Sdiag || !Xdiag || !trace_out) return SPINGP_EINVAL;
    if (n > 1 && (!Soff || !Xoff)) return SPINGP_EINVAL;
    if (!ws_ok(ws, ws_bytes, spg::diagprod_ws_bytes(n))) return SPINGP_EINVAL;
    spingp_status st = prepare_device();
    if (st != SPINGP_OK) return st;
    return finish(spg::btd_diagprod(b, n, Sdiag, Soff, Xdiag, Xoff, diag_out, trace_out, ws, (cudaStream_t)stream),
                  ws, flags, stream);
}

size_t spingp_assemble_workspace_bytes(int64_t n) { return n < 1 ? 0 : spg::assemble_ws_bytes(n); }

spingp_status spingp_assemble(const spingp_model* m, const double* t, const double* y, int64_t n,
                              const double* theta, double* D_out, double* O_out, double* r_out,
                              double* logdet_kinv_out, void* ws, size_t ws_bytes, unsigned flags, void* stream) {
    if (!m || !t || !y || !theta || n < 1 || !D_out || !r_out || !logdet_kinv_out) return SPINGP_EINVAL;
    if (n > 1 && !O_out) return SPINGP_EINVAL;
    if (!single_matern(m)) return SPINGP_EUNSUPPORTED;
    if (!ws_ok(ws, ws_bytes, spg::assemble_ws_bytes(n))) return SPINGP_EINVAL;
    spingp_status st = prepare_device();
    if (st != SPINGP_OK) return st;
    return finish(spg::assemble(m->b, t, y, n, theta, D_out, O_out, r_out, logdet_kinv_out, ws, (cudaStream_t)stream),
                  ws, flags, stream);
}

size_t spingp_literal_workspace_bytes(const spingp_model* m, int64_t n, spingp_ws_kind what) {
    if (!m || n < 1 || !single_matern(m)) return 0;
    return spg::literal_ws_bytes(m->b, n, ws_mode(what));
}

spingp_status spingp_literal(const spingp_model* m, spingp_ws_kind what, const double* t, const double* y,
                             int64_t n, const double* theta, double* ll_out, double* grad_out, double* mean_out,
                             double* var_out, void* ws, size_t ws_bytes, unsigned flags, void* stream) {
    if (!m || !t || !y || !theta || n < 1 || !ll_out) return SPINGP_EINVAL;
    const int mode = ws_mode(what);
    if (mode == spg::MODE_GRAD && !grad_out) return SPINGP_EINVAL;
    if (mode == spg::MODE_POSTERIOR && (!mean_out || !var_out)) return SPINGP_EINVAL;
    if (!single_matern(m)) return SPINGP_EUNSUPPORTED;
    if (!ws_ok(ws, ws_bytes, spg::literal_ws_bytes(m->b, n, mode))) return SPINGP_EINVAL;
    spingp_status st = prepare_device();
    if (st != SPINGP_OK) return st;
    return finish(spg::literal_run(m->b, mode, t, y, n, theta, ll_out, grad_out, mean_out, var_out, ws,
                                   (cudaStream_t)stream),
                  ws, flags, stream);
}

int spingp_literal_launch_count(int64_t n) { return n < 1 ? -1 : (int)spg::literal_launch_count(n); }
int spingp_btd_launch_count(int64_t n) { return n < 1 ? -1 : (int)spg::btd_launch_count(n); }

spingp_status spingp_ws_status(void* ws, void* stream) {
    if (!ws) return SPINGP_EINVAL;
    int bits = 0;
    cudaStream_t s = (cudaStream_t)stream;
    if (cudaMemcpyAsync(&bits, ws, sizeof(int), cudaMemcpyDeviceToHost, s) != cudaSuccess) return SPINGP_ECUDA;
    if (cudaStreamSynchronize(s) != cudaSuccess) return SPINGP_ECUDA;
    if (bits & spg::ST_EINVAL) return SPINGP_EINVAL;
    if (bits & spg::ST_ENONFINITE) return SPINGP_ENONFINITE;
    if (bits & spg::ST_ENOTSORTED) return SPINGP_ENOTSORTED;
    if (bits & spg::ST_ENUMERIC) return SPINGP_ENUMERIC;
    return SPINGP_OK;
}

spingp_status spingp_sync_status(void* ws, void* stream) { return spingp_ws_status(ws, stream); }

const char* spingp_status_str(spingp_status s) {
    switch (s) {
    case SPINGP_OK: return "ok";
    case SPINGP_EINVAL: return "invalid argument";
    case SPINGP_ENOTSORTED: return "times are not sorted";
    case SPINGP_ENONFINITE: return "non-finite time or observation";
    case SPINGP_ENUMERIC: return "non-positive innovation variance or pivot";
    case SPINGP_ECUDA: return "CUDA runtime error";
    case SPINGP_ETIMEOUT: return "device wait timed out";
    case SPINGP_ENOMEM: return "out of host memory";
    case SPINGP_EUNSUPPORTED: return "model not supported by this build";
    }
    return "unknown status";
}

}  // extern "C"
