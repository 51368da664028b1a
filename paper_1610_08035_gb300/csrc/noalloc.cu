// noalloc.cu -- a log-likelihood entry point that allocates no device memory.
//
// Its scratch is a fixed array in the library's own device image.  Host code
// may not pass the array's name to a kernel (on the host that name is only a
// stand-in, not a device address), so the device address is looked up with
// cudaGetSymbolAddress once per device and context, and cached with the
// context's unique ID: after a device reset the new context gets a new ID,
// and the next call looks the address up again.  The mutex guards only that
// cache; the calls themselves share the one array, so a caller must not let
// two calls on one device overlap.
#include <cuda_runtime.h>
#include <mutex>
#include <stdint.h>

#include "spingp.h"
#include "internal.h"

#define NOALLOC_MAXDEV 64

static __device__ __align__(256) unsigned char g_noalloc_scratch[SPINGP_NOALLOC_SCRATCH_BYTES];

namespace {

std::mutex g_noalloc_mu;
void* g_noalloc_ptr[NOALLOC_MAXDEV];
unsigned long long g_noalloc_ctx[NOALLOC_MAXDEV];

// Set-up, once per device and context, with that device current: resolve the
// scratch array's device address and opt the reduction kernels into their
// shared memory size.  Neither step allocates memory.
spingp_status noalloc_scratch(void** out) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= NOALLOC_MAXDEV) return SPINGP_ECUDA;
    std::lock_guard<std::mutex> lock(g_noalloc_mu);
    if (!g_noalloc_ptr[dev] || spg::context_id() != g_noalloc_ctx[dev]) {
        void* p = nullptr;
        if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) return SPINGP_ECUDA;
        if (spg::matern_prepare()) return SPINGP_ECUDA;
        g_noalloc_ptr[dev] = p;
        g_noalloc_ctx[dev] = spg::context_id();   // read after the set-up, which makes the context current
    }
    *out = g_noalloc_ptr[dev];
    return SPINGP_OK;
}

}  // namespace

extern "C" spingp_status spingp_loglik_noalloc(const spingp_model* model, const double* t, const double* y,
                                               int64_t n, const double* theta, double* ll_out, unsigned flags,
                                               void* stream) {
    if (!model || !t || !y || !theta || !ll_out || n < 1) return SPINGP_EINVAL;
    if (!spg::model_on_chain_path(model)) return SPINGP_EUNSUPPORTED;
    const size_t need = spingp_workspace_bytes(model, n, SPINGP_WS_LOGLIK);
    if (need == 0) return SPINGP_EUNSUPPORTED;
    if (need > (size_t)SPINGP_NOALLOC_SCRATCH_BYTES) return SPINGP_EINVAL;   // series too long for the fixed scratch
    void* ws = nullptr;
    spingp_status st = noalloc_scratch(&ws);
    if (st != SPINGP_OK) return st;
    cudaStream_t s = (cudaStream_t)stream;
    if (spg::matern_run(spingp_state_dim(model), spg::MODE_LOGLIK, t, y, n, spingp_get_chunk_len(model, n), theta,
                        ll_out, nullptr, nullptr, nullptr, ws, s, nullptr, (flags & SPINGP_MISSING_NAN) ? 1 : 0))
        return SPINGP_ECUDA;
    if (flags & SPINGP_SYNC) return spingp_ws_status(ws, stream);
    return SPINGP_OK;
}
