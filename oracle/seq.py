"""ctypes binding of the sequential C oracle (O-seq, ``oracle/seq.c``).

TEST INFRASTRUCTURE ONLY (see the package docstring).  The shared library is
compiled with the host C compiler on first use, or by ``build()``.
"""
import ctypes
import os
import subprocess

import numpy as np

from . import normalize_spec, n_params, state_dim

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "seq.c")
_OUT_DIR = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_OUT_DIR, "liboseq.so")
_lib = None

STATUS = {0: "ok", 1: "invalid argument", 2: "times not sorted", 3: "non-finite input",
          4: "numerical failure", 7: "out of memory"}


class OracleError(RuntimeError):
    pass


def build(force=False):
    """Compile seq.c into oracle/_build/liboseq.so (plain FP64, no fast-math,
    no FMA contraction so that results do not depend on the host ISA)."""
    os.makedirs(_OUT_DIR, exist_ok=True)
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    tmp = _LIB_PATH + ".%d.tmp" % os.getpid()
    cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-ffp-contract=off",
           "-o", tmp, _SRC, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def bind(path):
    """Load a compiled copy of seq.c and declare its exported signatures."""
    lib = ctypes.CDLL(path)
    D = ctypes.POINTER(ctypes.c_double)
    I = ctypes.POINTER(ctypes.c_int)
    L = ctypes.c_long
    lib.oseq_dims.argtypes = [ctypes.c_int, I, I, I, I, I]
    lib.oseq_continuous.argtypes = [ctypes.c_int, I, I, I, D, D, D, D, D]
    lib.oseq_discretize.argtypes = [ctypes.c_int, I, I, I, D, ctypes.c_double, D, D, D, D, D, D]
    lib.oseq_loglik.argtypes = [ctypes.c_int, I, I, I, D, D, D, L, D]
    lib.oseq_smoother.argtypes = [ctypes.c_int, I, I, I, D, D, D, L, D, D, D, D, D, D]
    lib.oseq_grad.argtypes = [ctypes.c_int, I, I, I, D, D, D, L, D, D, D, D, D]
    lib.oseq_sample.argtypes = [ctypes.c_int, I, I, I, D, D, L, D, D]
    lib.oseq_eq_factor.argtypes = [ctypes.c_int, D]
    for f in ("oseq_dims", "oseq_continuous", "oseq_discretize", "oseq_loglik",
              "oseq_smoother", "oseq_grad", "oseq_sample", "oseq_eq_factor"):
        getattr(lib, f).restype = ctypes.c_int
    return lib


def _load():
    global _lib
    if _lib is None:
        build()
        _lib = bind(_LIB_PATH)
    return _lib


def _dp(a):
    if a is None:
        return ctypes.POINTER(ctypes.c_double)()
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _spec_args(spec):
    comps = normalize_spec(spec)
    n = len(comps)
    kind = (ctypes.c_int * n)(*[c[0] for c in comps])
    order = (ctypes.c_int * n)(*[c[1] for c in comps])
    env = (ctypes.c_int * n)(*[c[2] for c in comps])
    return n, kind, order, env


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def _check(st):
    if st != 0:
        raise OracleError("oracle failed: %s (%d)" % (STATUS.get(st, "?"), st))


def _theta(spec, theta):
    th = _f64(theta)
    if th.shape != (n_params(spec),):
        raise ValueError("theta must have %d entries" % n_params(spec))
    return th


def continuous(spec, theta):
    """(F, Pinf, H, Lq) of the continuous model (Eq. ss1 before discretisation)."""
    lib = _load()
    b = state_dim(spec)
    F = np.zeros((b, b)); Pinf = np.zeros((b, b)); H = np.zeros(b); Lq = np.zeros((b, b))
    _check(lib.oseq_continuous(*_spec_args(spec), _dp(_theta(spec, theta)), _dp(F), _dp(Pinf), _dp(H), _dp(Lq)))
    return F, Pinf, H, Lq


def discretize(spec, theta, dt):
    """A = expm(F dt), Q = Pinf - A Pinf A^T and their parameter derivatives
    (dA, dQ, dPinf have shape (P, b, b)); also Pinf."""
    lib = _load()
    b, P = state_dim(spec), n_params(spec)
    A = np.zeros((b, b)); Q = np.zeros((b, b)); dA = np.zeros((P, b, b)); dQ = np.zeros((P, b, b))
    Pinf = np.zeros((b, b)); dPinf = np.zeros((P, b, b))
    _check(lib.oseq_discretize(*_spec_args(spec), _dp(_theta(spec, theta)), float(dt),
                               _dp(A), _dp(Q), _dp(dA), _dp(dQ), _dp(Pinf), _dp(dPinf)))
    return dict(A=A, Q=Q, dA=dA, dQ=dQ, Pinf=Pinf, dPinf=dPinf)


def loglik(spec, theta, t, y):
    lib = _load()
    t = _f64(t); y = _f64(y)
    ll = np.zeros(1)
    _check(lib.oseq_loglik(*_spec_args(spec), _dp(_theta(spec, theta)), _dp(t), _dp(y), len(t), _dp(ll)))
    return float(ll[0])


def smoother(spec, theta, t, y, blocks=False):
    """RTS smoother.  Returns dict(ll, mean, var) and, with blocks=True, the
    smoothed state means ms (n, b), the diagonal blocks Ps (n, b, b) and the
    first sub-diagonal blocks Pc (n-1, b, b), Pc[i] = Cov(z_{i+1}, z_i | y)."""
    lib = _load()
    t = _f64(t); y = _f64(y)
    n, b = len(t), state_dim(spec)
    ll = np.zeros(1); mean = np.zeros(n); var = np.zeros(n)
    ms = np.zeros((n, b)) if blocks else None
    Ps = np.zeros((n, b, b)) if blocks else None
    Pc = np.zeros((max(n - 1, 0), b, b)) if blocks else None
    _check(lib.oseq_smoother(*_spec_args(spec), _dp(_theta(spec, theta)), _dp(t), _dp(y), n, _dp(ll),
                             _dp(mean), _dp(var), _dp(ms), _dp(Ps), _dp(Pc)))
    out = dict(ll=float(ll[0]), mean=mean, var=var)
    if blocks:
        out.update(ms=ms, Ps=Ps, Pc=Pc)
    return out


def grad(spec, theta, t, y, posterior=False, l1=False):
    """Log-likelihood and gradient with respect to every entry of theta
    (two-filter adjoint).  With posterior=True also the mean / latent variance
    obtained from the same two filters.  With l1=True also the sum over steps
    of the absolute per-step contributions to each gradient entry (the scale
    against which cancellation in the sum is judged); it is appended last."""
    lib = _load()
    t = _f64(t); y = _f64(y)
    n = len(t)
    ll = np.zeros(1); g = np.zeros(n_params(spec))
    mean = np.zeros(n) if posterior else None
    var = np.zeros(n) if posterior else None
    gabs = np.zeros(n_params(spec)) if l1 else None
    _check(lib.oseq_grad(*_spec_args(spec), _dp(_theta(spec, theta)), _dp(t), _dp(y), n, _dp(ll), _dp(g),
                         _dp(mean), _dp(var), _dp(gabs)))
    out = (float(ll[0]), g)
    if posterior:
        out = out + (mean, var)
    if l1:
        out = out + (gabs,)
    return out


def eq_factor(N):
    """Coefficients a_0 .. a_{N-1} of the monic stable spectral factor of the
    order-N exponentiated-quadratic approximation at unit lengthscale."""
    lib = _load()
    a = np.zeros(N)
    _check(lib.oseq_eq_factor(int(N), _dp(a)))
    return a


def sample(spec, theta, t, eps):
    """Draw y from the state-space model given standard normals eps of shape
    (n, b+1) chosen by the caller."""
    lib = _load()
    t = _f64(t)
    n, b = len(t), state_dim(spec)
    eps = _f64(eps)
    if eps.shape != (n, b + 1):
        raise ValueError("eps must have shape (n, b+1)")
    y = np.zeros(n)
    _check(lib.oseq_sample(*_spec_args(spec), _dp(_theta(spec, theta)), _dp(t), n, _dp(eps), _dp(y)))
    return y
