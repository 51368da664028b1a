"""Oracle for state-space temporal GP inference (SpInGP, arXiv 1610.08035).

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and
the CPU-baseline leg of ``bench.py`` may import anything in this package.  It
shares no code with the CUDA library in ``paper_1610_08035_gb300`` and imports
nothing from it.

Two independent FP64 implementations of the same plain definition:

* :mod:`oracle.dense` (O-dense): the textbook GP for small N.  The covariance
  matrix K + sigma_n^2 I is built from closed-form covariance functions and
  factorised with a library Cholesky; log-likelihood (Eq. ml2), posterior mean
  and latent variance, and the gradient 1/2 tr((a a^T - C^-1) dC/dtheta).  It
  also assembles the explicit block matrices of Sec. 2.1 (the stacked
  transition matrix, Q, the state covariance and its block-tridiagonal inverse,
  Theorem 1) for the structural pins.
* :mod:`oracle.seq` (O-seq, plain C in ``seq.c``): sequential Kalman filter,
  RTS smoother and a two-filter adjoint for the gradient; any N.

Model specification (shared by both): a list of components, each one of
``"matern12"``, ``"matern32"``, ``"matern52"``, ``("periodic", J)`` or
``("quasiperiodic", J, envelope)`` with envelope one of the Matern names, or
``("eq", N)``: the exponentiated-quadratic covariance through its state-space
approximation of even order N (the Taylor series of the inverse spectral
density truncated at N; Hartikainen & Sarkka 2010, the approximation the
paper's experiments use with N = 10).
Parameter vector theta: per component (lengthscale, variance) for Matern;
(variance, lengthscale, period) for periodic; (variance, lengthscale, period,
envelope lengthscale) for quasi-periodic; (lengthscale, variance) for eq; the
noise variance sigma_n^2 last.
"""

KIND_CODES = {"matern12": 1, "matern32": 2, "matern52": 3, "periodic": 4, "quasiperiodic": 5, "eq": 6}


def normalize_spec(spec):
    """Return the spec as a list of (kind_code, order, envelope_code)."""
    if isinstance(spec, (str, tuple)):
        spec = [spec]
    out = []
    for comp in spec:
        if isinstance(comp, str):
            comp = (comp,)
        name = comp[0]
        code = KIND_CODES[name]
        order = int(comp[1]) if len(comp) > 1 else 0
        env = KIND_CODES[comp[2]] if len(comp) > 2 else 0
        if code == 5 and env == 0:
            raise ValueError("quasiperiodic needs an envelope kind")
        if code == 6 and (order < 2 or order % 2):
            raise ValueError("eq needs an even approximation order >= 2")
        out.append((code, order, env))
    return out


def n_params(spec):
    """Number of entries of theta (noise variance included)."""
    per_kind = {1: 2, 2: 2, 3: 2, 4: 3, 5: 4, 6: 2}
    return sum(per_kind[c] for c, _, _ in normalize_spec(spec)) + 1


def state_dim(spec):
    b = 0
    for code, order, env in normalize_spec(spec):
        if code <= 3:
            b += code
        elif code == 4:
            b += 2 * (order + 1)
        elif code == 5:
            b += 2 * (order + 1) * env
        else:
            b += order
    return b
