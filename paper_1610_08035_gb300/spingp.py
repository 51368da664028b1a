"""Thin Python binding of the C ABI in include/spingp.h (argument marshalling only).

Every computation runs in the CUDA library ``_lib/libspingp.so``; there is no
CPU fallback.  Torch provides device memory and the current stream.  The
functions named ``spingp_*`` mirror the C entry points one to one; ``Model``
and ``LogLik`` are conveniences on top of them.
"""
import ctypes
import os

import torch

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_lib", "libspingp.so")

OK, EINVAL, ENOTSORTED, ENONFINITE, ENUMERIC, ECUDA, ETIMEOUT, ENOMEM, EUNSUPPORTED = range(9)
WS_LOGLIK, WS_GRAD, WS_POSTERIOR = 0, 1, 2
SYNC = 1
MISSING_NAN = 2
LOG_GRAD = 4      # gradient with respect to log theta
PREDICTIVE = 8    # posterior variances of an observation (latent + noise variance)

KINDS = {"matern12": 1, "matern32": 2, "matern52": 3, "periodic": 4, "quasiperiodic": 5, "eq": 6}

# names exported by the library, in the order of include/spingp.h
EXPORTS = ("spingp_model_create", "spingp_model_destroy", "spingp_num_params", "spingp_state_dim",
           "spingp_set_chunk_len", "spingp_get_chunk_len", "spingp_workspace_bytes", "spingp_loglik",
           "spingp_grad", "spingp_posterior", "spingp_posterior_lag1", "spingp_grad_posterior",
           "spingp_predict_workspace_bytes", "spingp_predict",
           "spingp_workspace_bytes_batched", "spingp_loglik_batched",
           "spingp_grad_batched", "spingp_posterior_batched", "spingp_grad_posterior_batched", "spingp_launch_count",
           "spingp_launch_count_batched", "spingp_profile_enable",
           "spingp_profile_read", "spingp_probe_fp64_bytes", "spingp_probe_fp64", "spingp_probe_fp64_tensor",
           "spingp_probe_exp_neg",
           "spingp_workspace_bytes_host", "spingp_segment_elem_size", "spingp_segment_launch_count",
           "spingp_segment_reduce", "spingp_segment_grad", "spingp_segment_grad_posterior",
           "spingp_grad_host", "spingp_loglik_noalloc",
           "spingp_btd_workspace_bytes", "spingp_btd_solve", "spingp_btd_launch_count",
           "spingp_btd_diag_product_workspace_bytes", "spingp_btd_diag_product",
           "spingp_assemble_workspace_bytes", "spingp_assemble", "spingp_literal_workspace_bytes",
           "spingp_literal", "spingp_literal_launch_count", "spingp_optimize_workspace_bytes", "spingp_optimize",
           "spingp_optimize_workspace_bytes_batched", "spingp_optimize_batched", "spingp_ws_status",
           "spingp_sync_status", "spingp_status_str")
STAGES = ("elimination", "reduction", "chunk_pass", "final_reduction")

_lib = None


class SpinGPError(RuntimeError):
    def __init__(self, status, what=""):
        self.status = status
        msg = _status_str(status)
        super().__init__("%s%s (status %d)" % (what + ": " if what else "", msg, status))


class _Desc(ctypes.Structure):
    _fields_ = [("n_comp", ctypes.c_int), ("kinds", ctypes.POINTER(ctypes.c_int)),
                ("orders", ctypes.POINTER(ctypes.c_int)), ("envs", ctypes.POINTER(ctypes.c_int))]


def load():
    """Load the CUDA library; raises if it has not been built."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError("CUDA library missing: %s (build it with __graft_entry__.build())" % LIB_PATH)
    lib = ctypes.CDLL(LIB_PATH)
    vp, dp, i64, sz, u32 = ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int64, ctypes.c_size_t, ctypes.c_uint
    lib.spingp_model_create.argtypes = [ctypes.POINTER(_Desc), ctypes.POINTER(vp)]
    lib.spingp_model_destroy.argtypes = [vp]
    lib.spingp_model_destroy.restype = None
    lib.spingp_num_params.argtypes = [vp]
    lib.spingp_state_dim.argtypes = [vp]
    lib.spingp_set_chunk_len.argtypes = [vp, ctypes.c_int]
    lib.spingp_get_chunk_len.argtypes = [vp, i64]
    lib.spingp_workspace_bytes.argtypes = [vp, i64, ctypes.c_int]
    lib.spingp_workspace_bytes.restype = sz
    lib.spingp_loglik.argtypes = [vp, dp, dp, i64, dp, dp, vp, sz, u32, vp]
    lib.spingp_grad.argtypes = [vp, dp, dp, i64, dp, dp, dp, vp, sz, u32, vp]
    lib.spingp_posterior.argtypes = [vp, dp, dp, i64, dp, dp, dp, dp, vp, sz, u32, vp]
    lib.spingp_posterior_lag1.argtypes = [vp, dp, dp, i64, dp, dp, dp, dp, dp, vp, sz, u32, vp]
    lib.spingp_grad_posterior.argtypes = [vp, dp, dp, i64, dp, dp, dp, dp, dp, dp, vp, sz, u32, vp]
    lib.spingp_predict_workspace_bytes.argtypes = [vp, i64, i64]
    lib.spingp_predict_workspace_bytes.restype = sz
    lib.spingp_predict.argtypes = [vp, dp, dp, i64, dp, dp, i64, dp, dp, vp, sz, u32, vp]
    lib.spingp_workspace_bytes_batched.argtypes = [vp, i64, i64, ctypes.c_int]
    lib.spingp_workspace_bytes_batched.restype = sz
    lib.spingp_loglik_batched.argtypes = [vp, dp, i64, i64, dp, dp, dp, dp, vp, sz, u32, vp]
    lib.spingp_grad_batched.argtypes = [vp, dp, i64, i64, dp, dp, dp, dp, dp, vp, sz, u32, vp]
    lib.spingp_grad_posterior_batched.argtypes = [vp, dp, i64, i64, dp, dp, dp, dp, dp, dp, dp, vp, sz, u32,
                                                  vp]
    lib.spingp_posterior_batched.argtypes = [vp, dp, i64, i64, dp, dp, dp, dp, dp, dp, vp, sz, u32, vp]
    lib.spingp_launch_count.argtypes = [vp, i64, ctypes.c_int]
    lib.spingp_launch_count_batched.argtypes = [vp, i64, i64, ctypes.c_int]
    lib.spingp_profile_enable.argtypes = [vp, ctypes.c_int]
    lib.spingp_profile_read.argtypes = [vp, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_int)]
    lib.spingp_probe_fp64_bytes.argtypes = []
    lib.spingp_probe_fp64_bytes.restype = sz
    lib.spingp_probe_fp64.argtypes = [vp, sz, ctypes.POINTER(ctypes.c_double), vp]
    lib.spingp_probe_fp64_tensor.argtypes = [vp, sz, ctypes.POINTER(ctypes.c_double), vp]
    lib.spingp_segment_elem_size.argtypes = [vp]
    lib.spingp_segment_launch_count.argtypes = [vp, i64]
    lib.spingp_segment_reduce.argtypes = [vp, dp, dp, i64, dp, ctypes.c_double, ctypes.c_int, dp, vp, sz, u32, vp]
    lib.spingp_segment_grad.argtypes = [vp, dp, dp, i64, dp, ctypes.c_double, ctypes.c_int, dp, ctypes.c_int,
                                        ctypes.c_int, dp, dp, vp, sz, u32, vp]
    lib.spingp_segment_grad_posterior.argtypes = [vp, dp, dp, i64, dp, ctypes.c_double, ctypes.c_int, dp,
                                                  ctypes.c_int, ctypes.c_int, dp, dp, dp, dp, vp, sz, u32, vp]
    lib.spingp_probe_exp_neg.argtypes = [dp, dp, i64, vp]
    lib.spingp_loglik_noalloc.argtypes = [vp, dp, dp, i64, dp, dp, u32, vp]
    lib.spingp_workspace_bytes_host.argtypes = [vp, i64]
    lib.spingp_workspace_bytes_host.restype = sz
    lib.spingp_grad_host.argtypes = [vp, dp, dp, i64, dp, dp, dp, vp, sz, u32, vp]
    lib.spingp_btd_workspace_bytes.argtypes = [ctypes.c_int, i64]
    lib.spingp_btd_workspace_bytes.restype = sz
    lib.spingp_btd_solve.argtypes = [ctypes.c_int, i64, dp, dp, dp, dp, dp, dp, dp, vp, sz, u32, vp]
    lib.spingp_btd_launch_count.argtypes = [i64]
    lib.spingp_btd_diag_product_workspace_bytes.argtypes = [i64]
    lib.spingp_btd_diag_product_workspace_bytes.restype = sz
    lib.spingp_btd_diag_product.argtypes = [ctypes.c_int, i64, dp, dp, dp, dp, dp, dp, vp, sz, u32, vp]
    lib.spingp_assemble_workspace_bytes.argtypes = [i64]
    lib.spingp_assemble_workspace_bytes.restype = sz
    lib.spingp_assemble.argtypes = [vp, dp, dp, i64, dp, dp, dp, dp, dp, vp, sz, u32, vp]
    lib.spingp_literal_workspace_bytes.argtypes = [vp, i64, ctypes.c_int]
    lib.spingp_literal_workspace_bytes.restype = sz
    lib.spingp_literal.argtypes = [vp, ctypes.c_int, dp, dp, i64, dp, dp, dp, dp, dp, vp, sz, u32, vp]
    lib.spingp_literal_launch_count.argtypes = [i64]
    dbl = ctypes.c_double
    lib.spingp_optimize_workspace_bytes.argtypes = [vp, i64]
    lib.spingp_optimize_workspace_bytes.restype = sz
    lib.spingp_optimize.argtypes = [vp, dp, dp, i64, dp, ctypes.c_int, dbl, dp, dp, vp, sz, u32, vp]
    lib.spingp_optimize_workspace_bytes_batched.argtypes = [vp, i64, i64]
    lib.spingp_optimize_workspace_bytes_batched.restype = sz
    lib.spingp_optimize_batched.argtypes = [vp, dp, i64, i64, dp, dp, dp, ctypes.c_int, dbl, dp, dp, vp, sz, u32, vp]
    lib.spingp_ws_status.argtypes = [vp, vp]
    lib.spingp_sync_status.argtypes = [vp, vp]
    lib.spingp_status_str.argtypes = [ctypes.c_int]
    lib.spingp_status_str.restype = ctypes.c_char_p
    _lib = lib
    return lib


def _status_str(st):
    try:
        return load().spingp_status_str(st).decode()
    except Exception:
        return "status"


def _check(st, what):
    if st != OK:
        raise SpinGPError(st, what)


def _ptr(x):
    if x is None:
        return None
    return ctypes.c_void_p(x.data_ptr())


def _stream():
    return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)


def _dev_f64(x, name):
    if not (isinstance(x, torch.Tensor) and x.is_cuda and x.dtype == torch.float64 and x.is_contiguous()):
        raise TypeError("%s must be a contiguous float64 CUDA tensor" % name)
    return x


# ---------------------------------------------------------------- the C entry points, one to one

def spingp_model_create(spec):
    """spec: a list of components, each "matern12" | "matern32" | "matern52" |
    ("periodic", J) | ("quasiperiodic", J, envelope) | ("eq", N) (N even)."""
    lib = load()
    if isinstance(spec, (str, tuple)):
        spec = [spec]
    kinds, orders, envs = [], [], []
    for comp in spec:
        comp = (comp,) if isinstance(comp, str) else tuple(comp)
        kinds.append(KINDS[comp[0]])
        orders.append(int(comp[1]) if len(comp) > 1 else 0)
        envs.append(KINDS[comp[2]] if len(comp) > 2 else 0)
    n = len(kinds)
    arr = ctypes.c_int * n
    desc = _Desc(n, arr(*kinds), arr(*orders), arr(*envs))
    h = ctypes.c_void_p()
    _check(lib.spingp_model_create(ctypes.byref(desc), ctypes.byref(h)), "spingp_model_create")
    return h


def spingp_model_destroy(h):
    load().spingp_model_destroy(h)


def spingp_num_params(h):
    return load().spingp_num_params(h)


def spingp_state_dim(h):
    return load().spingp_state_dim(h)


def spingp_set_chunk_len(h, L):
    _check(load().spingp_set_chunk_len(h, int(L)), "spingp_set_chunk_len")


def spingp_get_chunk_len(h, n):
    return load().spingp_get_chunk_len(h, int(n))


def spingp_workspace_bytes(h, n, what):
    return load().spingp_workspace_bytes(h, int(n), int(what))


def spingp_loglik(h, t, y, n, theta, ll_out, ws, ws_bytes, flags, stream=None):
    return load().spingp_loglik(h, _ptr(t), _ptr(y), int(n), _ptr(theta), _ptr(ll_out), _ptr(ws), ws_bytes,
                                flags, stream if stream is not None else _stream())


def spingp_grad(h, t, y, n, theta, ll_out, grad_out, ws, ws_bytes, flags, stream=None):
    return load().spingp_grad(h, _ptr(t), _ptr(y), int(n), _ptr(theta), _ptr(ll_out), _ptr(grad_out), _ptr(ws),
                              ws_bytes, flags, stream if stream is not None else _stream())


def spingp_posterior(h, t, y, n, theta, ll_out, mean_out, var_out, ws, ws_bytes, flags, stream=None):
    return load().spingp_posterior(h, _ptr(t), _ptr(y), int(n), _ptr(theta), _ptr(ll_out), _ptr(mean_out),
                                   _ptr(var_out), _ptr(ws), ws_bytes, flags,
                                   stream if stream is not None else _stream())


def spingp_posterior_lag1(h, t, y, n, theta, ll_out, mean_out, var_out, lag1_out, ws, ws_bytes, flags,
                          stream=None):
    return load().spingp_posterior_lag1(h, _ptr(t), _ptr(y), int(n), _ptr(theta), _ptr(ll_out), _ptr(mean_out),
                                        _ptr(var_out), _ptr(lag1_out), _ptr(ws), int(ws_bytes), int(flags),
                                        stream if stream is not None else _stream())



def spingp_grad_posterior(h, t, y, n, theta, ll_out, grad_out, mean_out, var_out, lag1_out, ws, ws_bytes, flags,
                          stream=None):
    return load().spingp_grad_posterior(h, _ptr(t), _ptr(y), int(n), _ptr(theta), _ptr(ll_out), _ptr(grad_out),
                                        _ptr(mean_out), _ptr(var_out), _ptr(lag1_out), _ptr(ws), int(ws_bytes),
                                        int(flags), stream if stream is not None else _stream())


def spingp_predict_workspace_bytes(h, n, n_star):
    return load().spingp_predict_workspace_bytes(h, int(n), int(n_star))


def spingp_predict(h, t, y, n, theta, t_star, n_star, mean_out, var_out, ws, ws_bytes, flags, stream=None):
    return load().spingp_predict(h, _ptr(t), _ptr(y), int(n), _ptr(theta), _ptr(t_star), int(n_star),
                                 _ptr(mean_out), _ptr(var_out), _ptr(ws), int(ws_bytes), int(flags),
                                 stream if stream is not None else _stream())


def spingp_workspace_bytes_batched(h, n_series, n_total, what):
    return load().spingp_workspace_bytes_batched(h, int(n_series), int(n_total), int(what))


def spingp_loglik_batched(h, offsets, n_series, n_total, t, y, theta, ll_out, ws, ws_bytes, flags, stream=None):
    return load().spingp_loglik_batched(h, _ptr(offsets), int(n_series), int(n_total), _ptr(t), _ptr(y),
                                        _ptr(theta), _ptr(ll_out), _ptr(ws), ws_bytes, flags,
                                        stream if stream is not None else _stream())


def spingp_grad_batched(h, offsets, n_series, n_total, t, y, theta, ll_out, grad_out, ws, ws_bytes, flags,
                        stream=None):
    return load().spingp_grad_batched(h, _ptr(offsets), int(n_series), int(n_total), _ptr(t), _ptr(y), _ptr(theta),
                                      _ptr(ll_out), _ptr(grad_out), _ptr(ws), ws_bytes, flags,
                                      stream if stream is not None else _stream())


def spingp_posterior_batched(h, offsets, n_series, n_total, t, y, theta, ll_out, mean_out, var_out, ws, ws_bytes,
                             flags, stream=None):
    return load().spingp_posterior_batched(h, _ptr(offsets), int(n_series), int(n_total), _ptr(t), _ptr(y),
                                           _ptr(theta), _ptr(ll_out), _ptr(mean_out), _ptr(var_out), _ptr(ws),
                                           ws_bytes, flags, stream if stream is not None else _stream())


def spingp_grad_posterior_batched(h, offsets, n_series, n_total, t, y, theta, ll_out, grad_out, mean_out, var_out,
                                  ws, ws_bytes, flags, stream=None):
    return load().spingp_grad_posterior_batched(h, _ptr(offsets), int(n_series), int(n_total), _ptr(t), _ptr(y),
                                                _ptr(theta), _ptr(ll_out), _ptr(grad_out), _ptr(mean_out),
                                                _ptr(var_out), _ptr(ws), ws_bytes, flags,
                                                stream if stream is not None else _stream())


def spingp_launch_count_batched(h, n_series, n_total, what):
    return load().spingp_launch_count_batched(h, int(n_series), int(n_total), int(what))


def spingp_launch_count(h, n, what):
    return load().spingp_launch_count(h, int(n), int(what))


def spingp_profile_enable(h, on):
    _check(load().spingp_profile_enable(h, 1 if on else 0), "spingp_profile_enable")


def spingp_profile_read(h):
    """Summed milliseconds per stage since the last read, and the call count."""
    ms = (ctypes.c_double * 4)()
    calls = ctypes.c_int()
    _check(load().spingp_profile_read(h, ms, ctypes.byref(calls)), "spingp_profile_read")
    return dict(zip(STAGES, list(ms))), calls.value


def spingp_probe_fp64(device=None):
    """Measured FP64 TFLOP/s of the current device (independent FMA chains)."""
    lib = load()
    scratch = torch.empty(lib.spingp_probe_fp64_bytes(), dtype=torch.uint8,
                          device=device if device is not None else "cuda")
    out = ctypes.c_double()
    _check(lib.spingp_probe_fp64(_ptr(scratch), scratch.numel(), ctypes.byref(out), _stream()),
           "spingp_probe_fp64")
    return out.value


def spingp_probe_fp64_tensor(device=None):
    """Measured FP64 tensor-core TFLOP/s (mma.sync m8n8k4) of the current device."""
    lib = load()
    scratch = torch.empty(lib.spingp_probe_fp64_bytes(), dtype=torch.uint8,
                          device=device if device is not None else "cuda")
    out = ctypes.c_double()
    _check(lib.spingp_probe_fp64_tensor(_ptr(scratch), scratch.numel(), ctypes.byref(out), _stream()),
           "spingp_probe_fp64_tensor")
    return out.value


def spingp_probe_exp_neg(x):
    """e^-x of a CUDA float64 tensor by the chain kernels' table-driven exponential."""
    _dev_f64(x, "x")
    x = x.contiguous()
    y = torch.empty_like(x)
    _check(load().spingp_probe_exp_neg(_ptr(x), _ptr(y), x.numel(), _stream()), "spingp_probe_exp_neg")
    return y


def spingp_segment_elem_size(h):
    return load().spingp_segment_elem_size(h)


def spingp_segment_launch_count(h, n):
    return load().spingp_segment_launch_count(h, int(n))


def spingp_segment_reduce(h, t, y, n, theta, t_prev, first, elem_out, ws, ws_bytes, flags, stream=None):
    return load().spingp_segment_reduce(h, _ptr(t), _ptr(y), int(n), _ptr(theta), float(t_prev), int(first),
                                        _ptr(elem_out), _ptr(ws), int(ws_bytes), flags,
                                        stream if stream is not None else _stream())


def spingp_segment_grad(h, t, y, n, theta, t_prev, first, elems, n_ranks, rank, ll_out, grad_out, ws, ws_bytes,
                        flags, stream=None):
    return load().spingp_segment_grad(h, _ptr(t), _ptr(y), int(n), _ptr(theta), float(t_prev), int(first),
                                      _ptr(elems), int(n_ranks), int(rank), _ptr(ll_out), _ptr(grad_out), _ptr(ws),
                                      int(ws_bytes), flags, stream if stream is not None else _stream())


def spingp_segment_grad_posterior(h, t, y, n, theta, t_prev, first, elems, n_ranks, rank, ll_out, grad_out,
                                  mean_out, var_out, ws, ws_bytes, flags, stream=None):
    return load().spingp_segment_grad_posterior(h, _ptr(t), _ptr(y), int(n), _ptr(theta), float(t_prev),
                                                int(first), _ptr(elems), int(n_ranks), int(rank), _ptr(ll_out),
                                                _ptr(grad_out), _ptr(mean_out), _ptr(var_out), _ptr(ws),
                                                int(ws_bytes), flags, stream if stream is not None else _stream())


def spingp_workspace_bytes_host(h, n):
    return load().spingp_workspace_bytes_host(h, int(n))


def spingp_grad_host(h, t, y, n, theta, ll_out, grad_out, ws, ws_bytes, flags, stream=None):
    """t, y, theta, ll_out, grad_out: host tensors (pinned for overlap)."""
    return load().spingp_grad_host(h, _ptr(t), _ptr(y), int(n), _ptr(theta), _ptr(ll_out), _ptr(grad_out),
                                   _ptr(ws), ws_bytes, flags, stream if stream is not None else _stream())


def spingp_loglik_noalloc(h, t, y, n, theta, ll_out, flags, stream=None):
    """spingp_loglik without a workspace: the library's fixed device scratch
    is used instead, so nothing is allocated (see include/spingp.h)."""
    return load().spingp_loglik_noalloc(h, _ptr(t), _ptr(y), int(n), _ptr(theta), _ptr(ll_out), flags,
                                        stream if stream is not None else _stream())


def spingp_btd_workspace_bytes(b, n):
    return load().spingp_btd_workspace_bytes(int(b), int(n))


def spingp_btd_solve(b, n, D, O, r, logdet_out, x_out, Sdiag_out, Soff_out, ws, ws_bytes, flags, stream=None):
    return load().spingp_btd_solve(int(b), int(n), _ptr(D), _ptr(O), _ptr(r), _ptr(logdet_out), _ptr(x_out),
                                   _ptr(Sdiag_out), _ptr(Soff_out), _ptr(ws), ws_bytes, flags,
                                   stream if stream is not None else _stream())


def spingp_btd_launch_count(n):
    return load().spingp_btd_launch_count(int(n))


def spingp_btd_diag_product_workspace_bytes(n):
    return load().spingp_btd_diag_product_workspace_bytes(int(n))


def spingp_btd_diag_product(b, n, Sdiag, Soff, Xdiag, Xoff, diag_out, trace_out, ws, ws_bytes, flags, stream=None):
    return load().spingp_btd_diag_product(int(b), int(n), _ptr(Sdiag), _ptr(Soff), _ptr(Xdiag), _ptr(Xoff),
                                          _ptr(diag_out), _ptr(trace_out), _ptr(ws), ws_bytes, flags,
                                          stream if stream is not None else _stream())


def spingp_assemble_workspace_bytes(n):
    return load().spingp_assemble_workspace_bytes(int(n))


def spingp_assemble(h, t, y, n, theta, D_out, O_out, r_out, logdet_kinv_out, ws, ws_bytes, flags, stream=None):
    return load().spingp_assemble(h, _ptr(t), _ptr(y), int(n), _ptr(theta), _ptr(D_out), _ptr(O_out), _ptr(r_out),
                                  _ptr(logdet_kinv_out), _ptr(ws), ws_bytes, flags,
                                  stream if stream is not None else _stream())


def spingp_literal_workspace_bytes(h, n, what):
    return load().spingp_literal_workspace_bytes(h, int(n), int(what))


def spingp_literal(h, what, t, y, n, theta, ll_out, grad_out, mean_out, var_out, ws, ws_bytes, flags, stream=None):
    return load().spingp_literal(h, int(what), _ptr(t), _ptr(y), int(n), _ptr(theta), _ptr(ll_out),
                                 _ptr(grad_out), _ptr(mean_out), _ptr(var_out), _ptr(ws), ws_bytes, flags,
                                 stream if stream is not None else _stream())


def spingp_literal_launch_count(n):
    return load().spingp_literal_launch_count(int(n))


def spingp_optimize_workspace_bytes(h, n):
    return load().spingp_optimize_workspace_bytes(h, int(n))


def spingp_optimize(h, t, y, n, theta_inout, iterations, tol, ll_out, grad_out, ws, ws_bytes, flags, stream=None):
    return load().spingp_optimize(h, _ptr(t), _ptr(y), int(n), _ptr(theta_inout), int(iterations), float(tol),
                                  _ptr(ll_out), _ptr(grad_out), _ptr(ws), ws_bytes, flags,
                                  stream if stream is not None else _stream())


def spingp_optimize_workspace_bytes_batched(h, n_series, n_total):
    return load().spingp_optimize_workspace_bytes_batched(h, int(n_series), int(n_total))


def spingp_optimize_batched(h, offsets, n_series, n_total, t, y, theta_inout, iterations, tol, ll_out, grad_out, ws,
                            ws_bytes, flags, stream=None):
    return load().spingp_optimize_batched(h, _ptr(offsets), int(n_series), int(n_total), _ptr(t), _ptr(y),
                                          _ptr(theta_inout), int(iterations), float(tol), _ptr(ll_out),
                                          _ptr(grad_out), _ptr(ws), ws_bytes, flags,
                                          stream if stream is not None else _stream())


def spingp_ws_status(ws, stream=None):
    return load().spingp_ws_status(_ptr(ws), stream if stream is not None else _stream())


spingp_sync_status = spingp_ws_status


def spingp_status_str(st):
    return _status_str(st)


# ---------------------------------------------------------------- conveniences

class Model:
    """A model handle with workspace management on the current device."""

    def __init__(self, spec, chunk_len=0):
        self.spec = spec
        self.h = spingp_model_create(spec)
        if chunk_len:
            spingp_set_chunk_len(self.h, chunk_len)
        self._ws = {}

    def __del__(self):
        h = getattr(self, "h", None)
        if h is not None and _lib is not None:
            _lib.spingp_model_destroy(h)
            self.h = None

    @property
    def num_params(self):
        return spingp_num_params(self.h)

    @property
    def state_dim(self):
        return spingp_state_dim(self.h)

    def set_chunk_len(self, L):
        spingp_set_chunk_len(self.h, L)
        self._ws.clear()

    def chunk_len(self, n):
        return spingp_get_chunk_len(self.h, n)

    def workspace(self, n, what, device=None, purpose=None):
        nbytes = spingp_workspace_bytes(self.h, n, what)
        if nbytes == 0:
            raise SpinGPError(EUNSUPPORTED, "spingp_workspace_bytes")
        device = torch.device(device) if device is not None else torch.device("cuda", torch.cuda.current_device())
        key = (what, device, purpose)
        ws = self._ws.get(key)
        if ws is None or ws.numel() < nbytes:
            ws = torch.empty(nbytes, dtype=torch.uint8, device=device)
            self._ws[key] = ws
        return ws

    def _args(self, t, y, theta):
        _dev_f64(t, "t"); _dev_f64(y, "y"); _dev_f64(theta, "theta")
        if t.dim() != 1 or y.shape != t.shape:
            raise ValueError("t and y must be 1-D of the same length")
        if theta.numel() != self.num_params:
            raise ValueError("theta must have %d entries" % self.num_params)
        return t.numel()

    @staticmethod
    def _flags(sync, missing, log_params=False, predictive=False):
        return ((SYNC if sync else 0) | (MISSING_NAN if missing else 0) | (LOG_GRAD if log_params else 0)
                | (PREDICTIVE if predictive else 0))

    def loglik(self, t, y, theta, sync=True, out=None, missing=False):
        n = self._args(t, y, theta)
        ws = self.workspace(n, WS_LOGLIK, t.device)
        ll = out if out is not None else torch.empty(1, dtype=torch.float64, device=t.device)
        _check(spingp_loglik(self.h, t, y, n, theta, ll, ws, ws.numel(), self._flags(sync, missing)),
               "spingp_loglik")
        return ll

    def grad(self, t, y, theta, sync=True, out=None, missing=False, log_params=False):
        """(ll, d ll / d theta); with log_params, d ll / d log theta."""
        n = self._args(t, y, theta)
        ws = self.workspace(n, WS_GRAD, t.device)
        if out is None:
            ll = torch.empty(1, dtype=torch.float64, device=t.device)
            g = torch.empty(self.num_params, dtype=torch.float64, device=t.device)
        else:
            ll, g = out
        _check(spingp_grad(self.h, t, y, n, theta, ll, g, ws, ws.numel(), self._flags(sync, missing, log_params)),
               "spingp_grad")
        return ll, g

    def grad_host(self, t, y, theta, sync=True, out=None, missing=False, device=None, log_params=False):
        """spingp_grad from host (CPU) tensors: t, y, theta float64 on the
        host (pin them for overlapped copies); returns host (ll, grad)."""
        for name, v in (("t", t), ("y", y), ("theta", theta)):
            if not (isinstance(v, torch.Tensor) and not v.is_cuda and v.dtype == torch.float64 and v.is_contiguous()):
                raise TypeError("%s must be a contiguous float64 host tensor" % name)
        n = t.numel()
        if y.numel() != n or theta.numel() != self.num_params:
            raise ValueError("shapes do not match the model")
        device = torch.device(device) if device is not None else torch.device("cuda", torch.cuda.current_device())
        key = ("host", device)
        nbytes = spingp_workspace_bytes_host(self.h, n)
        ws = self._ws.get(key)
        if ws is None or ws.numel() < nbytes:
            ws = torch.empty(nbytes, dtype=torch.uint8, device=device)
            self._ws[key] = ws
        if out is None:
            ll = torch.empty(1, dtype=torch.float64).pin_memory()
            g = torch.empty(self.num_params, dtype=torch.float64).pin_memory()
        else:
            ll, g = out
        _check(spingp_grad_host(self.h, t, y, n, theta, ll, g, ws, ws.numel(),
                                self._flags(sync, missing, log_params)), "spingp_grad_host")
        return ll, g

    def segment_reduce(self, t, y, theta, t_prev=None, ws=None, sync=True, missing=False):
        """Phase 1 of a series split across ranks: this range's element
        (device, spingp_segment_elem_size doubles).  t_prev: the time of the
        previous range's last step, None for the range that starts the
        series.  ws: this rank's workspace (kept for segment_grad)."""
        n = self._args(t, y, theta)
        # a workspace of its own: segment_grad needs what this call leaves in it
        ws = ws if ws is not None else self.workspace(n, WS_GRAD, t.device, purpose="segment")
        elem = torch.empty(spingp_segment_elem_size(self.h), dtype=torch.float64, device=t.device)
        first = t_prev is None
        _check(spingp_segment_reduce(self.h, t, y, n, theta, 0.0 if first else t_prev, first, elem, ws, ws.numel(),
                                     self._flags(sync, missing)), "spingp_segment_reduce")
        return elem

    def segment_grad(self, t, y, theta, elems, rank, t_prev=None, ws=None, sync=True, missing=False,
                     log_params=False):
        """Phase 2: this range's share of (ll, grad) from all ranks' elements
        (device, n_ranks x elem_size, rank order); the same arguments and
        workspace as segment_reduce."""
        n = self._args(t, y, theta)
        ws = ws if ws is not None else self.workspace(n, WS_GRAD, t.device, purpose="segment")
        _dev_f64(elems, "elems")
        elems = elems.contiguous()
        ll = torch.empty(1, dtype=torch.float64, device=t.device)
        g = torch.empty(self.num_params, dtype=torch.float64, device=t.device)
        first = t_prev is None
        _check(spingp_segment_grad(self.h, t, y, n, theta, 0.0 if first else t_prev, first, elems, elems.shape[0],
                                   rank, ll, g, ws, ws.numel(), self._flags(sync, missing, log_params)),
               "spingp_segment_grad")
        return ll, g

    def segment_grad_posterior(self, t, y, theta, elems, rank, t_prev=None, ws=None, sync=True, missing=False,
                               log_params=False, predictive=False):
        """Phase 2 with the posterior: this range's share of (ll, grad) and
        the posterior mean and variance at this range's steps, conditioned on
        every rank's observations; the same arguments and workspace as
        segment_reduce.  Returns (ll, grad, mean, var)."""
        n = self._args(t, y, theta)
        ws = ws if ws is not None else self.workspace(n, WS_GRAD, t.device, purpose="segment")
        _dev_f64(elems, "elems")
        elems = elems.contiguous()
        dev = t.device
        ll = torch.empty(1, dtype=torch.float64, device=dev)
        g = torch.empty(self.num_params, dtype=torch.float64, device=dev)
        mean = torch.empty(n, dtype=torch.float64, device=dev)
        var = torch.empty(n, dtype=torch.float64, device=dev)
        first = t_prev is None
        _check(spingp_segment_grad_posterior(self.h, t, y, n, theta, 0.0 if first else t_prev, first, elems,
                                             elems.shape[0], rank, ll, g, mean, var, ws, ws.numel(),
                                             self._flags(sync, missing, log_params, predictive)),
               "spingp_segment_grad_posterior")
        return ll, g, mean, var

    def posterior(self, t, y, theta, sync=True, with_loglik=True, missing=False, predictive=False, out=None):
        """(mean, var, ll): latent posterior mean and variance at t; with
        predictive, var is the variance of an observation there (+ s_n).
        out: (mean, var, ll) buffers to write instead (ll may be None)."""
        n = self._args(t, y, theta)
        ws = self.workspace(n, WS_POSTERIOR, t.device)
        if out is not None:
            mean, var, ll = out
        else:
            mean = torch.empty(n, dtype=torch.float64, device=t.device)
            var = torch.empty(n, dtype=torch.float64, device=t.device)
            ll = torch.empty(1, dtype=torch.float64, device=t.device) if with_loglik else None
        _check(spingp_posterior(self.h, t, y, n, theta, ll, mean, var, ws, ws.numel(),
                                self._flags(sync, missing, predictive=predictive)), "spingp_posterior")
        return mean, var, ll

    def posterior_lag1(self, t, y, theta, sync=True, missing=False):
        """(mean, var, cov_lag1, ll): the posterior plus Cov(f_{i+1}, f_i | y)
        for i = 0 .. n-2, the first off-diagonal of the selected inverse."""
        n = self._args(t, y, theta)
        ws = self.workspace(n, WS_POSTERIOR, t.device)
        mean = torch.empty(n, dtype=torch.float64, device=t.device)
        var = torch.empty(n, dtype=torch.float64, device=t.device)
        lag = torch.empty(max(n - 1, 1), dtype=torch.float64, device=t.device)
        ll = torch.empty(1, dtype=torch.float64, device=t.device)
        _check(spingp_posterior_lag1(self.h, t, y, n, theta, ll, mean, var, lag, ws, ws.numel(),
                                     self._flags(sync, missing)), "spingp_posterior_lag1")
        return mean, var, lag[:n - 1], ll

    def grad_posterior(self, t, y, theta, sync=True, missing=False, log_params=False, predictive=False,
                       lag1=False, out=None):
        """(ll, grad, mean, var, cov_lag1 or None) from one pass: the gradient
        of grad() and the posterior of posterior() / posterior_lag1().
        out: (ll, grad, mean, var, cov_lag1 or None) buffers to write instead."""
        n = self._args(t, y, theta)
        ws = self.workspace(n, WS_GRAD, t.device)
        dev = t.device
        if out is not None:
            ll, g, mean, var, lag = out
        else:
            ll = torch.empty(1, dtype=torch.float64, device=dev)
            g = torch.empty(self.num_params, dtype=torch.float64, device=dev)
            mean = torch.empty(n, dtype=torch.float64, device=dev)
            var = torch.empty(n, dtype=torch.float64, device=dev)
            lag = torch.empty(max(n - 1, 1), dtype=torch.float64, device=dev) if lag1 else None
        _check(spingp_grad_posterior(self.h, t, y, n, theta, ll, g, mean, var, lag, ws, ws.numel(),
                                     self._flags(sync, missing, log_params, predictive)), "spingp_grad_posterior")
        return ll, g, mean, var, (lag[:n - 1] if lag is not None else None)

    def predict(self, t, y, theta, t_star, predictive=False, sync=True):
        """Latent predictive mean and variance at new times t_star (Eqs.
        mean4-mean6), through spingp_predict: the test times join the chain
        with missing observations and one posterior pass covers both.  t
        must be sorted; t_star may be in any order (it is sorted on the
        device).  NaN observations in y are missing.  Returns (mean, var) at
        t_star; with predictive, var is that of a new observation (+ s_n)."""
        _dev_f64(t_star, "t_star")
        n = self._args(t, y, theta)
        t_star = t_star.contiguous()
        m = t_star.numel()
        dev = t_star.device
        nbytes = spingp_predict_workspace_bytes(self.h, n, m)
        if nbytes == 0:
            raise SpinGPError(EUNSUPPORTED, "spingp_predict_workspace_bytes")
        ws = self._ws.get(("predict", dev))                  # kept between calls, grown when too small
        if ws is None or ws.numel() < nbytes:
            ws = torch.empty(nbytes, dtype=torch.uint8, device=dev)
            self._ws[("predict", dev)] = ws
        mean = torch.empty(m, dtype=torch.float64, device=dev)
        var = torch.empty(m, dtype=torch.float64, device=dev)
        _check(spingp_predict(self.h, t, y, n, theta, t_star, m, mean, var, ws,
                              ws.numel(), self._flags(sync, False, predictive=predictive)), "spingp_predict")
        return mean, var

    def optimize(self, t, y, theta0, iterations=100, tol=1e-8, sync=True, missing=False):
        """Maximise the marginal likelihood from theta0 by scaled conjugate
        gradients over log-parameters (Sec. 4.3).  Returns (theta, ll, grad)
        at the last accepted point."""
        n = self._args(t, y, theta0)
        dev = t.device
        theta = theta0.clone()
        ll = torch.empty(1, dtype=torch.float64, device=dev)
        g = torch.empty(self.num_params, dtype=torch.float64, device=dev)
        ws = self._scratch(spingp_optimize_workspace_bytes(self.h, n), dev, "spingp_optimize")
        _check(spingp_optimize(self.h, t, y, n, theta, iterations, tol, ll, g, ws, ws.numel(),
                               self._flags(sync, missing)), "spingp_optimize")
        return theta, ll, g

    # ------------------------------------------------------------ the method as written (Sec. 2.2-3.1)

    def _scratch(self, nbytes, device, name):
        if nbytes == 0:
            raise SpinGPError(EUNSUPPORTED, name)
        return torch.empty(nbytes, dtype=torch.uint8, device=device)

    def assemble(self, t, y, theta, sync=True):
        """The explicit blocks of the posterior precision K~ (Theorem 1, Sec.
        2.2): D (n, b, b), O (n-1, b, b) with O[i] = K~[i+1, i], r (n, b), and
        log det Kinv.  Single Matern components only."""
        n = self._args(t, y, theta)
        b = self.state_dim
        dev = t.device
        D = torch.empty(n, b, b, dtype=torch.float64, device=dev)
        O = torch.empty(max(n - 1, 0), b, b, dtype=torch.float64, device=dev)
        r = torch.empty(n, b, dtype=torch.float64, device=dev)
        ldk = torch.empty(1, dtype=torch.float64, device=dev)
        ws = self._scratch(spingp_assemble_workspace_bytes(n), dev, "spingp_assemble")
        _check(spingp_assemble(self.h, t, y, n, theta, D, O if n > 1 else None, r, ldk, ws, ws.numel(),
                               SYNC if sync else 0), "spingp_assemble")
        return D, O, r, ldk

    def literal(self, t, y, theta, what=WS_LOGLIK, sync=True):
        """Log-likelihood (and gradient, or posterior mean and variance) by
        assembling K~ and running block cyclic reduction on it.  Returns ll,
        (ll, grad) or (mean, var, ll) as what is WS_LOGLIK, WS_GRAD or
        WS_POSTERIOR."""
        n = self._args(t, y, theta)
        dev = t.device
        ll = torch.empty(1, dtype=torch.float64, device=dev)
        g = torch.empty(self.num_params, dtype=torch.float64, device=dev) if what == WS_GRAD else None
        mean = torch.empty(n, dtype=torch.float64, device=dev) if what == WS_POSTERIOR else None
        var = torch.empty(n, dtype=torch.float64, device=dev) if what == WS_POSTERIOR else None
        ws = self._scratch(spingp_literal_workspace_bytes(self.h, n, what), dev, "spingp_literal")
        _check(spingp_literal(self.h, what, t, y, n, theta, ll, g, mean, var, ws, ws.numel(), SYNC if sync else 0),
               "spingp_literal")
        if what == WS_GRAD:
            return ll, g
        if what == WS_POSTERIOR:
            return mean, var, ll
        return ll


def btd_solve(D, O, r, selected=True, sync=True):
    """Subproblems 1-3 (Sec. 3.1) for a symmetric positive-definite block-
    tridiagonal matrix with diagonal blocks D (n, b, b) and sub-diagonal blocks
    O (n-1, b, b), O[i] = T[i+1, i]: returns (logdet, x, Sdiag, Soff) with
    x = T^-1 r and, if selected, the block-tridiagonal part of T^-1."""
    _dev_f64(D, "D"); _dev_f64(r, "r")
    n, b = D.shape[0], D.shape[1]
    if D.shape != (n, b, b) or r.shape != (n, b) or not 1 <= b <= 3:
        raise ValueError("D must be (n, b, b) and r (n, b) with b <= 3")
    if n > 1:
        _dev_f64(O, "O")
        if O.shape != (n - 1, b, b):
            raise ValueError("O must be (n-1, b, b)")
    dev = D.device
    ld = torch.empty(1, dtype=torch.float64, device=dev)
    x = torch.empty(n, b, dtype=torch.float64, device=dev)
    Sd = torch.empty(n, b, b, dtype=torch.float64, device=dev) if selected else None
    So = torch.empty(max(n - 1, 0), b, b, dtype=torch.float64, device=dev) if selected else None
    nbytes = spingp_btd_workspace_bytes(b, n)
    ws = torch.empty(nbytes, dtype=torch.uint8, device=dev)
    _check(spingp_btd_solve(b, n, D, O if n > 1 else None, r, ld, x, Sd, So if (selected and n > 1) else None, ws,
                            nbytes, SYNC if sync else 0), "spingp_btd_solve")
    return ld, x, Sd, So


def btd_diag_product(Sd, So, Xd, Xo, sync=True):
    """Subproblem 4 (Sec. 3.1): the diagonal of S X and its trace, for the
    selected inverse S (Sd, So) and a symmetric block-tridiagonal X (Xd, Xo)."""
    _dev_f64(Sd, "Sdiag"); _dev_f64(Xd, "Xdiag")
    n, b = Sd.shape[0], Sd.shape[1]
    if Xd.shape != Sd.shape:
        raise ValueError("Xdiag must match Sdiag")
    if n > 1:
        _dev_f64(So, "Soff"); _dev_f64(Xo, "Xoff")
    dev = Sd.device
    diag = torch.empty(n, b, dtype=torch.float64, device=dev)
    tr = torch.empty(1, dtype=torch.float64, device=dev)
    nbytes = spingp_btd_diag_product_workspace_bytes(n)
    ws = torch.empty(nbytes, dtype=torch.uint8, device=dev)
    _check(spingp_btd_diag_product(b, n, Sd, So if n > 1 else None, Xd, Xo if n > 1 else None, diag, tr, ws, nbytes,
                                   SYNC if sync else 0), "spingp_btd_diag_product")
    return diag, tr


class Batch:
    """A batch of independent series sharing one model structure: device
    offsets (int64, n_series + 1), concatenated t and y, and one theta row per
    series.  Methods mirror Model's and return per-series results."""

    def __init__(self, model, offsets, t, y):
        if not (isinstance(offsets, torch.Tensor) and offsets.is_cuda and offsets.dtype == torch.int64):
            raise TypeError("offsets must be an int64 CUDA tensor")
        _dev_f64(t, "t"); _dev_f64(y, "y")
        self.model, self.offsets, self.t, self.y = model, offsets.contiguous(), t, y
        self.n_series = offsets.numel() - 1
        self.n_total = t.numel()
        if self.n_series < 1 or y.numel() != self.n_total:
            raise ValueError("need at least one series and len(y) == len(t)")
        self._ws = {}

    def workspace(self, what):
        nbytes = spingp_workspace_bytes_batched(self.model.h, self.n_series, self.n_total, what)
        if nbytes == 0:
            raise SpinGPError(EUNSUPPORTED, "spingp_workspace_bytes_batched")
        ws = self._ws.get(what)
        if ws is None or ws.numel() < nbytes:
            ws = torch.empty(nbytes, dtype=torch.uint8, device=self.t.device)
            self._ws[what] = ws
        return ws

    def _theta(self, theta):
        _dev_f64(theta, "theta")
        if theta.numel() != self.n_series * self.model.num_params:
            raise ValueError("theta must have n_series x %d entries" % self.model.num_params)
        return theta

    def loglik(self, theta, sync=True, out=None, missing=False):
        ws = self.workspace(WS_LOGLIK)
        ll = out if out is not None else torch.empty(self.n_series, dtype=torch.float64, device=self.t.device)
        _check(spingp_loglik_batched(self.model.h, self.offsets, self.n_series, self.n_total, self.t, self.y,
                                     self._theta(theta), ll, ws, ws.numel(), Model._flags(sync, missing)),
               "spingp_loglik_batched")
        return ll

    def grad(self, theta, sync=True, out=None, missing=False, log_params=False):
        ws = self.workspace(WS_GRAD)
        if out is None:
            ll = torch.empty(self.n_series, dtype=torch.float64, device=self.t.device)
            g = torch.empty(self.n_series * self.model.num_params, dtype=torch.float64, device=self.t.device)
        else:
            ll, g = out
        _check(spingp_grad_batched(self.model.h, self.offsets, self.n_series, self.n_total, self.t, self.y,
                                   self._theta(theta), ll, g, ws, ws.numel(),
                                   Model._flags(sync, missing, log_params)), "spingp_grad_batched")
        return ll, g.view(self.n_series, self.model.num_params)

    def posterior(self, theta, sync=True, missing=False, predictive=False):
        ws = self.workspace(WS_POSTERIOR)
        dev = self.t.device
        mean = torch.empty(self.n_total, dtype=torch.float64, device=dev)
        var = torch.empty(self.n_total, dtype=torch.float64, device=dev)
        ll = torch.empty(self.n_series, dtype=torch.float64, device=dev)
        _check(spingp_posterior_batched(self.model.h, self.offsets, self.n_series, self.n_total, self.t, self.y,
                                        self._theta(theta), ll, mean, var, ws, ws.numel(),
                                        Model._flags(sync, missing, predictive=predictive)),
               "spingp_posterior_batched")
        return mean, var, ll

    def grad_posterior(self, theta, sync=True, missing=False, log_params=False, predictive=False):
        """(ll, grad, mean, var) from one pass: grad()'s per-series values
        and posterior()'s per-step mean and variance."""
        ws = self.workspace(WS_GRAD)
        dev = self.t.device
        P = self.model.num_params
        ll = torch.empty(self.n_series, dtype=torch.float64, device=dev)
        g = torch.empty(self.n_series * P, dtype=torch.float64, device=dev)
        mean = torch.empty(self.n_total, dtype=torch.float64, device=dev)
        var = torch.empty(self.n_total, dtype=torch.float64, device=dev)
        _check(spingp_grad_posterior_batched(self.model.h, self.offsets, self.n_series, self.n_total, self.t, self.y,
                                             self._theta(theta), ll, g, mean, var, ws, ws.numel(),
                                             Model._flags(sync, missing, log_params, predictive)),
               "spingp_grad_posterior_batched")
        return ll, g.view(self.n_series, P), mean, var

    def optimize(self, theta0, iterations=100, tol=1e-8, sync=True):
        """Fit every series' hyperparameters by scaled conjugate gradients
        (Sec. 4.3), all series in one launch sequence.  theta0: n_series x P
        starting points.  Returns (theta, ll, grad), one row per series."""
        theta0 = self._theta(theta0)
        dev = self.t.device
        P = self.model.num_params
        theta = theta0.clone().view(self.n_series, P)
        ll = torch.empty(self.n_series, dtype=torch.float64, device=dev)
        g = torch.empty(self.n_series, P, dtype=torch.float64, device=dev)
        nbytes = spingp_optimize_workspace_bytes_batched(self.model.h, self.n_series, self.n_total)
        if nbytes == 0:
            raise SpinGPError(EUNSUPPORTED, "spingp_optimize_workspace_bytes_batched")
        ws = self._ws.get("optimize")
        if ws is None or ws.numel() < nbytes:
            ws = torch.empty(nbytes, dtype=torch.uint8, device=dev)
            self._ws["optimize"] = ws
        _check(spingp_optimize_batched(self.model.h, self.offsets, self.n_series, self.n_total, self.t, self.y,
                                       theta, iterations, tol, ll, g, ws, ws.numel(), SYNC if sync else 0),
               "spingp_optimize_batched")
        return theta, ll, g


class LogLik(torch.autograd.Function):
    """log p(y | t, theta) with the hand-written adjoint as its backward.

    LogLik.apply(t, y, theta, model): forward runs spingp_grad once and keeps
    the gradient; backward returns grad_output * gradient for theta (t and y
    get no gradient)."""

    @staticmethod
    def forward(ctx, t, y, theta, model):
        ll, g = model.grad(t, y, theta.detach().contiguous())
        ctx.save_for_backward(g)
        return ll[0]

    @staticmethod
    def backward(ctx, grad_out):
        (g,) = ctx.saved_tensors
        return None, None, grad_out * g, None
