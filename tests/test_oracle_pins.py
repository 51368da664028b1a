"""Pins of the oracle to facts fixed by the paper and by the mathematics.

Nothing here compares the oracle with itself: every check is either a closed
form, an identity the paper states (Theorem 1, the group property, the
determinant and inversion lemmas, Q = P0 - A P0 A^T), an independent library
routine (Pade expm, Cholesky), brute force on tiny inputs, or a
finite-difference derivative.  CPU only.
"""
import numpy as np
import pytest
import scipy.linalg

from oracle import btd, dense, seq, state_dim, n_params

MATERN = [
    ("matern12", [0.7, 1.3, 0.1]),
    ("matern32", [1.0, 1.0, 0.1]),
    ("matern52", [0.5, 2.0, 0.05]),
]
PERIODIC = [
    ([("periodic", 3)], [1.2, 1.0, 0.8, 0.1]),
    (["matern32", ("quasiperiodic", 6, "matern12")], [1.0, 1.0, 1.0, 1.0, 1.0, 10.0, 0.01]),
    (["matern32", ("quasiperiodic", 2, "matern32")], [0.8, 1.1, 0.9, 1.3, 0.7, 4.0, 0.02]),
]
# exponentiated quadratic through its order-N state-space approximation; the
# generic pins use well-conditioned orders (see the EQ pins below for N = 10)
EQ = [
    ([("eq", 4)], [0.9, 1.4, 0.1]),
    (["matern32", ("eq", 4)], [1.0, 0.6, 0.5, 1.2, 0.05]),
]
ALL = MATERN + PERIODIC + EQ


def _series(n, mean_dt, seed, tie_every=0):
    rng = np.random.default_rng(seed)
    d = rng.exponential(mean_dt, n)
    d[0] = 0.0
    if tie_every:
        d[::tie_every] = 0.0
    t = np.cumsum(d) + 0.3
    y = np.sin(2.3 * t) + 0.5 * np.cos(7.1 * t + 0.4) + 0.3 * rng.standard_normal(n)
    return t, y


# ---------------------------------------------------------------- model constants and discretisation

@pytest.mark.parametrize("spec,theta", ALL)
def test_lyapunov(spec, theta):
    """Pinf is the stationary covariance: F Pinf + Pinf F^T + L q_c L^T = 0."""
    F, Pinf, H, Lq = seq.continuous(spec, theta)
    R = F @ Pinf + Pinf @ F.T + Lq
    scale = np.max(np.abs(F @ Pinf)) + np.max(np.abs(Lq)) + 1e-300
    assert np.max(np.abs(R)) <= 1e-13 * scale
    assert np.allclose(Pinf, Pinf.T)
    assert np.min(np.linalg.eigvalsh(Pinf)) >= -1e-14 * np.max(np.abs(Pinf))


def test_matern32_example_matches_paper():
    """Eq. ss_matern: F = [[0,1],[-phi^2,-2 phi]], phi = sqrt(3)/l, P0 = diag(1, 3/l^2),
    H = [1 0] (unit variance)."""
    ell = 0.7
    F, Pinf, H, _ = seq.continuous("matern32", [ell, 1.0, 0.1])
    phi = np.sqrt(3.0) / ell
    assert np.allclose(F, [[0.0, 1.0], [-phi ** 2, -2.0 * phi]], rtol=1e-15, atol=0)
    assert np.allclose(Pinf, np.diag([1.0, 3.0 / ell ** 2]), rtol=1e-15, atol=0)
    assert np.array_equal(H, [1.0, 0.0])


@pytest.mark.parametrize("spec,theta", ALL)
@pytest.mark.parametrize("dt", [0.0, 1e-9, 0.013, 0.37, 2.9])
def test_expm_against_pade(spec, theta, dt):
    """A_n = expm(F dt_n) (Sec. 2.1) against scipy's Pade scaling-and-squaring.
    The Matern and periodic families have closed forms (2e-13); the EQ
    approximation uses a general exponential of a highly non-normal companion
    matrix (|F dt| up to ~10 here), where two valid algorithms differ at the
    1e-12 level (1e-11)."""
    F, Pinf, _, _ = seq.continuous(spec, theta)
    d = seq.discretize(spec, theta, dt)
    Ap = scipy.linalg.expm(F * dt)
    tol = 1e-11 if (spec, theta) in EQ else 2e-13
    assert np.max(np.abs(d["A"] - Ap)) <= tol * max(1.0, np.max(np.abs(Ap)))
    Qlit = Pinf - Ap @ Pinf @ Ap.T
    assert np.max(np.abs(d["Q"] - Qlit)) <= 1e-12 * np.max(np.abs(Pinf))
    assert np.allclose(d["Pinf"], Pinf, rtol=1e-15, atol=0)


@pytest.mark.parametrize("spec,theta", ALL)
def test_group_property(spec, theta):
    """A[d1] A[d2] = A[d1 + d2]; A[0] = I and Q[0] = 0 (Sec. 2.1)."""
    b = state_dim(spec)
    for d1, d2 in [(0.1, 0.25), (1e-7, 0.5), (1.3, 0.02)]:
        A1 = seq.discretize(spec, theta, d1)["A"]
        A2 = seq.discretize(spec, theta, d2)["A"]
        A12 = seq.discretize(spec, theta, d1 + d2)["A"]
        # general exponential for the EQ approximation (see test_expm_against_pade)
        tol = 1e-11 if (spec, theta) in EQ else 1e-13
        assert np.max(np.abs(A1 @ A2 - A12)) <= tol * max(1.0, np.max(np.abs(A12)))
    d0 = seq.discretize(spec, theta, 0.0)
    assert np.array_equal(d0["A"], np.eye(b))
    assert np.max(np.abs(d0["Q"])) == 0.0


def _period_indices(spec):
    from oracle import normalize_spec
    idx, p = [], 0
    for code, _, _ in normalize_spec(spec):
        if code >= 4:
            idx.append(p + 2)
        p += {1: 2, 2: 2, 3: 2, 4: 3, 5: 4, 6: 2}[code]
    return idx


def _fd(f, x, h):
    """Central difference with one Richardson step: error O(h^4)."""
    d1 = (f(x + h) - f(x - h)) / (2 * h)
    d2 = (f(x + h / 2) - f(x - h / 2)) / h
    return (4 * d2 - d1) / 3


@pytest.mark.parametrize("spec,theta", ALL)
def test_discretisation_derivatives(spec, theta):
    """dA/dtheta, dQ/dtheta, dPinf/dtheta against finite differences."""
    theta = np.array(theta, dtype=float)
    dt = 0.21
    d = seq.discretize(spec, theta, dt)
    for p in range(n_params(spec)):
        def comp(x, key):
            th = theta.copy(); th[p] = x
            return seq.discretize(spec, th, dt)[key]
        h = 1e-3 * theta[p]
        for key, dkey in (("A", "dA"), ("Q", "dQ"), ("Pinf", "dPinf")):
            fd = _fd(lambda x: comp(x, key), theta[p], h)
            scale = max(1e-3, np.max(np.abs(fd)))
            assert np.max(np.abs(d[dkey][p] - fd)) <= 1e-8 * scale, (key, p)


# ---------------------------------------------------------------- closed-form covariance functions

@pytest.mark.parametrize("spec,theta", ALL)
def test_kernel_derivatives(spec, theta):
    theta = np.array(theta, dtype=float)
    tau = np.linspace(-3.0, 3.0, 41)
    _, dk = dense.kernel(spec, theta, tau)
    for p in range(n_params(spec) - 1):
        def k(x):
            th = theta.copy(); th[p] = x
            return dense.kernel(spec, th, tau)[0]
        fd = _fd(k, theta[p], 1e-3 * theta[p])
        assert np.max(np.abs(dk[p] - fd)) <= 1e-8 * max(1.0, np.max(np.abs(fd))), p


def test_periodic_series_converges_to_closed_form():
    """The cosine series behind the periodic state-space model sums to
    exp(-2 sin^2(pi tau/p)/l^2); truncation at J = 20 is exact in FP64."""
    tau = np.linspace(-2.0, 2.0, 101)
    for var, lp, per in [(1.0, 1.0, 1.0), (0.7, 0.8, 1.7), (2.0, 1.5, 0.4)]:
        k, _ = dense.kernel([("periodic", 20)], [var, lp, per, 0.1], tau)
        assert np.max(np.abs(k - dense.periodic_exact(var, lp, per, tau))) <= 1e-14 * var


def test_matern_closed_forms():
    """Spot values of the Matern family (nu = 1/2, 3/2, 5/2) at r = lam |tau| = 1."""
    for name, b, val in [("matern12", 1, np.exp(-1.0)), ("matern32", 2, 2.0 * np.exp(-1.0)),
                         ("matern52", 3, (1.0 + 1.0 + 1.0 / 3.0) * np.exp(-1.0))]:
        ell = 0.9
        tau = ell / np.sqrt(2 * b - 1)
        k, _ = dense.kernel(name, [ell, 1.7, 0.1], np.array([tau, -tau]))
        assert np.allclose(k, 1.7 * val, rtol=1e-15, atol=0)


@pytest.mark.parametrize("spec,theta", ALL)
def test_state_space_covariance_equals_kernel(spec, theta):
    """Eq. k1 and Sec. 2.2: G (bold-A bold-Q bold-A^T) G^T equals K(t, t) from
    the closed-form covariance function (exact family)."""
    t, _ = _series(24, 0.15, 1)
    M = btd.stacked(spec, theta, t)
    K, _ = dense.gram(spec, theta, t)
    GKG = M["G"] @ M["Kc"] @ M["G"].T
    assert np.max(np.abs(GKG - K)) <= 1e-12 * np.max(np.abs(K))


# ---------------------------------------------------------------- Theorem 1 and the lemmas

@pytest.mark.parametrize("spec,theta", MATERN + PERIODIC[1:2])
def test_theorem1_precision_is_block_tridiagonal(spec, theta):
    """Theorem 1: the inverse of the stacked state covariance is block
    tridiagonal; bold-A^-1 is block bidiagonal with -A_i below the diagonal.
    (The pure periodic family has Q = 0 and no precision; it is left out.)"""
    b = state_dim(spec)
    rng = np.random.default_rng(5)
    n = 16
    t = np.cumsum(rng.uniform(0.3, 0.6, n))   # well-conditioned gaps
    M = btd.stacked(spec, theta, t)
    assert np.max(np.abs(np.linalg.inv(M["bA"]) - M["bAinv"])) <= 1e-12
    Kinv = np.linalg.inv(M["Kc"])
    big = np.max(np.abs(Kinv))
    for i in range(n):
        for j in range(n):
            blk = btd.block(Kinv, b, i, j)
            if abs(i - j) > 1:
                assert np.max(np.abs(blk)) <= 1e-9 * big, (i, j)
    assert np.max(np.abs(Kinv - M["Kinv"])) <= 1e-8 * big


@pytest.mark.parametrize("spec,theta", MATERN)
def test_determinant_lemma_and_inversion_lemma(spec, theta):
    """Eq. det_1: det(G Kc G^T + Sigma) = det K~ det Kc det Sigma; and the
    posterior mean via subproblem 1 (Eq. mean3) equals the dense GP mean."""
    rng = np.random.default_rng(7)
    n = 14
    t = np.cumsum(rng.uniform(0.2, 0.5, n))
    y = rng.standard_normal(n)
    s2 = theta[-1]
    M = btd.stacked(spec, theta, t)
    C = M["G"] @ M["Kc"] @ M["G"].T + s2 * np.eye(n)
    lhs = np.linalg.slogdet(C)[1]
    rhs = np.linalg.slogdet(M["Ktilde"])[1] + np.linalg.slogdet(M["Kc"])[1] + n * np.log(s2)
    assert abs(lhs - rhs) <= 1e-9 * max(1.0, abs(lhs))
    # subproblem 1: z = K~^-1 G^T Sigma^-1 y; posterior mean of f = G z
    z = np.linalg.solve(M["Ktilde"], M["G"].T @ y / s2)
    mean, _ = dense.posterior(spec, theta, t, y)
    assert np.max(np.abs(M["G"] @ z - mean)) <= 1e-9


@pytest.mark.parametrize("spec,theta", ALL)
def test_selected_inverse_equals_rts(spec, theta):
    """The diagonal blocks of K~^-1 are the smoothed covariances and its first
    off-diagonal blocks the lag-one cross-covariances (Sec. 3.1, subproblems 2
    and 4); K~^-1 G^T Sigma^-1 y are the smoothed means (subproblem 1)."""
    b = state_dim(spec)
    rng = np.random.default_rng(11)
    n = 12
    t = np.cumsum(rng.uniform(0.3, 0.6, n))
    y = rng.standard_normal(n)
    M = btd.stacked(spec, theta, t)
    # the inverse of the posterior precision is the posterior covariance
    # Kc - Kc G^T (G Kc G^T + Sigma)^-1 G Kc, formed without inverting Q
    Kc, G, s2 = M["Kc"], M["G"], theta[-1]
    Cy = G @ Kc @ G.T + s2 * np.eye(n)
    Post = Kc - Kc @ G.T @ np.linalg.solve(Cy, G @ Kc)
    zmean = Kc @ G.T @ np.linalg.solve(Cy, y)
    sm = seq.smoother(spec, theta, t, y, blocks=True)
    scale = np.max(np.abs(Post))
    for i in range(n):
        assert np.max(np.abs(btd.block(Post, b, i, i) - sm["Ps"][i])) <= 1e-10 * scale
        if i + 1 < n:
            assert np.max(np.abs(btd.block(Post, b, i + 1, i) - sm["Pc"][i])) <= 1e-10 * scale
    assert np.max(np.abs(zmean.reshape(n, b) - sm["ms"])) <= 1e-10 * max(1.0, np.max(np.abs(zmean)))
    if M["Ktilde"] is not None and spec in [s for s, _ in MATERN]:
        # K~ itself, from explicit Q^-1, agrees when the gaps are well conditioned
        Kt_inv = np.linalg.inv(M["Ktilde"])
        assert np.max(np.abs(Kt_inv - Post)) <= 1e-8 * scale


# ---------------------------------------------------------------- dense vs sequential (the plain definition)

@pytest.mark.parametrize("spec,theta", ALL)
@pytest.mark.parametrize("tie_every", [0, 7])
def test_dense_equals_sequential(spec, theta, tie_every):
    """Log-likelihood, gradient and posterior: O(N^3) definition vs Kalman/RTS
    and the two-filter adjoint, with and without tied times (dt = 0)."""
    t, y = _series(400, 0.08, 3, tie_every)
    tol = 1e-12 if spec in [s for s, _ in MATERN] else 1e-9
    lld, gd = dense.grad(spec, theta, t, y)
    lls = seq.loglik(spec, theta, t, y)
    llg, gs, mg, vg = seq.grad(spec, theta, t, y, posterior=True)
    assert abs(lld - lls) <= tol * abs(lld)
    assert abs(lld - llg) <= tol * abs(lld)
    assert np.all(np.abs(gd - gs) <= tol * 10 * np.maximum(1.0, np.abs(gd)))
    md, vd = dense.posterior(spec, theta, t, y)
    sm = seq.smoother(spec, theta, t, y)
    assert np.max(np.abs(md - sm["mean"])) <= tol * 100
    assert np.max(np.abs(vd - sm["var"]) / vd) <= tol * 100
    assert np.max(np.abs(md - mg)) <= tol * 100
    assert np.max(np.abs(vd - vg) / vd) <= tol * 100


# ---------------------------------------------------------------- special cases with closed forms

def _lognormal(x, var):
    return -0.5 * (np.log(2 * np.pi * var) + x * x / var)


@pytest.mark.parametrize("spec,theta", ALL)
def test_single_point(spec, theta):
    """N = 1: log N(y; 0, k(0) + sigma_n^2)."""
    k0 = dense.kernel(spec, theta, np.array([0.0]))[0][0]
    ll = seq.loglik(spec, theta, [0.4], [0.73])
    assert abs(ll - _lognormal(0.73, k0 + theta[-1])) <= 1e-14 * abs(ll)


def test_tied_pair_closed_form():
    """Two observations at the same time: C = [[s+r, s], [s, s+r]]."""
    s, r, y1, y2 = 1.3, 0.2, 0.4, -0.9
    det = (s + r) ** 2 - s * s
    quad = ((s + r) * (y1 * y1 + y2 * y2) - 2 * s * y1 * y2) / det
    ref = -0.5 * quad - 0.5 * np.log(det) - np.log(2 * np.pi)
    for spec in ("matern12", "matern32", "matern52"):
        ll = seq.loglik(spec, [0.6, s, r], [1.0, 1.0], [y1, y2])
        assert abs(ll - ref) <= 1e-14 * abs(ref)


def test_ornstein_uhlenbeck_closed_form():
    """b = 1 (Matern-1/2): an AR(1) with coefficient a_i = exp(-dt_i/l) observed
    in noise; written as a scalar Kalman recursion by hand."""
    rng = np.random.default_rng(2)
    n = 200
    t = np.cumsum(rng.exponential(0.3, n))
    y = rng.standard_normal(n)
    ell, s, r = 0.8, 1.4, 0.3
    m, P, ll = 0.0, s, 0.0
    for i in range(n):
        if i:
            a = np.exp(-(t[i] - t[i - 1]) / ell)
            m, P = a * m, a * a * P + s * (1 - a * a)
        S = P + r
        ll += _lognormal(y[i] - m, S)
        k = P / S
        m, P = m + k * (y[i] - m), P - k * P
    assert abs(seq.loglik("matern12", [ell, s, r], t, y) - ll) <= 1e-13 * abs(ll)


@pytest.mark.parametrize("spec,theta", MATERN)
def test_far_apart_observations_are_independent(spec, theta):
    """dt -> infinity: the likelihood factorises over observations."""
    t = np.arange(6) * 1e4
    y = np.array([0.3, -1.2, 0.8, 0.1, 2.0, -0.4])
    k0 = theta[1]
    ref = sum(_lognormal(v, k0 + theta[-1]) for v in y)
    assert abs(seq.loglik(spec, theta, t, y) - ref) <= 1e-14 * abs(ref)


# ---------------------------------------------------------------- gradient pins at larger N

@pytest.mark.parametrize("spec,theta", ALL)
def test_gradient_finite_differences(spec, theta):
    """Two-filter gradient against Richardson-extrapolated central differences
    of the Kalman log-likelihood."""
    theta = np.array(theta, dtype=float)
    t, y = _series(3000, 0.05, 4, tie_every=53)
    _, g = seq.grad(spec, theta, t, y)
    for p in range(len(theta)):
        def f(x):
            th = theta.copy(); th[p] = x
            return seq.loglik(spec, th, t, y)
        # the period enters through a phase that grows with t (about 190
        # periods here), so the log-likelihood is strongly curved in it and
        # needs a smaller step
        rel = 1e-5 if p in _period_indices(spec) else 1e-3
        fd = _fd(f, theta[p], rel * theta[p])
        assert abs(g[p] - fd) <= 1e-6 * max(1.0, abs(fd)), (p, g[p], fd)


@pytest.mark.parametrize("spec,theta", MATERN)
def test_variance_scaling_identity(spec, theta):
    """Scaling both variances by c scales C by c, so
    s_f dl/ds_f + s_n dl/ds_n = y^T C^-1 y / 2 - N/2, with y^T C^-1 y read off
    l(2 theta_var) - l(theta_var) = y^T C^-1 y / 4 - N/2 log 2 (exact at any N)."""
    theta = np.array(theta, dtype=float)
    t, y = _series(20000, 0.02, 6, tie_every=101)
    ll, g = seq.grad(spec, theta, t, y)
    th2 = theta.copy(); th2[1] *= 2; th2[2] *= 2
    ll2 = seq.loglik(spec, th2, t, y)
    n = len(y)
    q = 4.0 * (ll2 - ll + 0.5 * n * np.log(2.0))
    lhs = theta[1] * g[1] + theta[2] * g[2]
    assert abs(lhs - (0.5 * q - 0.5 * n)) <= 1e-9 * (abs(theta[1] * g[1]) + abs(theta[2] * g[2]) + n)


def test_sample_has_model_covariance():
    """The state-space sampler draws y with covariance K + sigma_n^2 I: the
    empirical covariance of many short draws matches the closed form."""
    spec, theta = "matern32", [0.5, 1.2, 0.1]
    t = np.array([0.0, 0.1, 0.35, 0.35, 1.2])
    rng = np.random.default_rng(9)
    draws = np.array([seq.sample(spec, theta, t, rng.standard_normal((5, 3))) for _ in range(20000)])
    K, _ = dense.gram(spec, theta, t)
    C = K + theta[-1] * np.eye(5)
    emp = draws.T @ draws / len(draws)
    assert np.max(np.abs(emp - C)) <= 0.05 * np.max(C)


@pytest.mark.parametrize("spec,theta", ALL)
def test_missing_observations_are_test_points(spec, theta):
    """Eqs. mean4-mean6: a test point enters the chain with infinite noise (a
    NaN observation).  The smoother's mean and latent variance there equal the
    textbook predictive equations of the dense GP on the observed points, and
    the log-likelihood and gradient equal those of the observed points alone."""
    rng = np.random.default_rng(12)
    t_obs, y_obs = _series(300, 0.05, 13)
    t_new = np.sort(rng.uniform(t_obs[0] - 0.5, t_obs[-1] + 0.5, 60))
    t_all = np.concatenate([t_obs, t_new])
    order = np.argsort(t_all, kind="stable")
    t_all = t_all[order]
    y_all = np.concatenate([y_obs, np.full(len(t_new), np.nan)])[order]
    is_new = order >= len(t_obs)
    sm = seq.smoother(spec, theta, t_all, y_all)
    md, vd = dense.predict(spec, theta, t_obs, y_obs, t_all[is_new])
    tol = 1e-10 if spec in [s for s, _ in MATERN] else 1e-8
    assert np.max(np.abs(sm["mean"][is_new] - md)) <= tol * max(1.0, np.max(np.abs(md)))
    assert np.max(np.abs(sm["var"][is_new] - vd) / vd) <= tol * 10
    ll_obs, g_obs = seq.grad(spec, theta, t_obs, y_obs)
    ll_all, g_all = seq.grad(spec, theta, t_all, y_all)
    assert abs(ll_all - ll_obs) <= 1e-12 * abs(ll_obs)
    assert np.all(np.abs(g_all - g_obs) <= 1e-9 * np.maximum(1.0, np.abs(g_obs)))
    _, g_dense = dense.grad(spec, theta, t_obs, y_obs)
    assert np.all(np.abs(g_all - g_dense) <= 1e-8 * np.maximum(1.0, np.abs(g_dense)))


def _random_spd_btd(n, b, seed):
    """A random symmetric positive-definite block-tridiagonal matrix: a block
    bidiagonal factor B (lower) times its transpose plus a small ridge."""
    rng = np.random.default_rng(seed)
    Bm = np.zeros((n * b, n * b))
    for i in range(n):
        Bm[i * b:(i + 1) * b, i * b:(i + 1) * b] = rng.standard_normal((b, b)) + 2.0 * np.eye(b)
        if i + 1 < n:
            Bm[(i + 1) * b:(i + 2) * b, i * b:(i + 1) * b] = rng.standard_normal((b, b))
    return Bm @ Bm.T + 0.1 * np.eye(n * b)


@pytest.mark.parametrize("n,b", [(1, 2), (2, 3), (17, 1), (40, 3), (33, 4)])
def test_thomas_against_dense(n, b):
    """Sequential block LDL^T and selected inverse against dense routines:
    log det, solve, diagonal and first sub-diagonal blocks of the inverse."""
    T = _random_spd_btd(n, b, n * 10 + b)
    r = np.random.default_rng(3).standard_normal(n * b)
    D, O = btd.blocks_of(T, b)
    logdet, x, Sd, So = btd.thomas(D, O, r.reshape(n, b))
    assert abs(logdet - np.linalg.slogdet(T)[1]) <= 1e-11 * max(1.0, abs(logdet))
    assert np.max(np.abs(x.reshape(-1) - np.linalg.solve(T, r))) <= 1e-10 * max(1.0, np.max(np.abs(x)))
    Ti = np.linalg.inv(T)
    for i in range(n):
        assert np.max(np.abs(Sd[i] - btd.block(Ti, b, i, i))) <= 1e-10 * np.max(np.abs(Ti))
        if i + 1 < n:
            assert np.max(np.abs(So[i] - btd.block(Ti, b, i + 1, i))) <= 1e-10 * np.max(np.abs(Ti))


@pytest.mark.parametrize("spec,theta", MATERN)
def test_literal_method_on_the_assembled_precision(spec, theta):
    """The paper's method as written: K~ assembled from Theorem 1, factorised by
    the block algorithm; log det K~ through Eq. det_1 gives the log-likelihood,
    the solve gives the posterior state means (subproblem 1) and the selected
    inverse the smoothed covariances (subproblems 2, 4).  Well-conditioned gaps."""
    b = state_dim(spec)
    rng = np.random.default_rng(21)
    n = 30
    t = np.cumsum(rng.uniform(0.3, 0.6, n))
    y = rng.standard_normal(n)
    M = btd.stacked(spec, theta, t)
    s2 = theta[-1]
    D, O = btd.blocks_of(M["Ktilde"], b)
    r = (M["G"].T @ y / s2).reshape(n, b)
    logdet, x, Sd, So = btd.thomas(D, O, r)
    logdet_Kinv = np.linalg.slogdet(M["Kinv"])[1]
    ll = -0.5 * (y @ y / s2 - r.reshape(-1) @ x.reshape(-1)) \
        - 0.5 * (logdet - logdet_Kinv + n * np.log(s2)) - 0.5 * n * np.log(2 * np.pi)
    assert abs(ll - seq.loglik(spec, theta, t, y)) <= 1e-9 * abs(ll)
    sm = seq.smoother(spec, theta, t, y, blocks=True)
    assert np.max(np.abs(x - sm["ms"])) <= 1e-9 * max(1.0, np.max(np.abs(x)))
    assert np.max(np.abs(Sd - sm["Ps"])) <= 1e-9 * np.max(np.abs(sm["Ps"]))
    assert np.max(np.abs(So - sm["Pc"])) <= 1e-9 * np.max(np.abs(sm["Ps"]))


def test_diag_product_is_the_log_det_derivative():
    """Subproblem 4's trace is Jacobi's formula d/de log det(T + e X) =
    tr(T^-1 X) (Eq. dd1): checked by a central difference of log det on a
    random SPD BTD T and a random symmetric BTD X; X = T gives the identity."""
    rng = np.random.default_rng(5)
    for b, n in ((1, 9), (2, 7), (3, 6)):
        D, O = btd.blocks_of(_random_spd_btd(n, b, 100 + b), b)
        Xd = rng.standard_normal((n, b, b))
        Xd = Xd + np.transpose(Xd, (0, 2, 1))
        Xo = rng.standard_normal((n - 1, b, b))
        d, tr = btd.diag_product(D, O, Xd, Xo)
        h = 1e-5
        lp = np.linalg.slogdet(btd.dense_of(D + h * Xd, O + h * Xo))[1]
        lm = np.linalg.slogdet(btd.dense_of(D - h * Xd, O - h * Xo))[1]
        assert abs(tr - (lp - lm) / (2 * h)) <= 1e-7 * max(1.0, abs(tr))
        d1, tr1 = btd.diag_product(D, O, D, O)
        assert np.allclose(d1, 1.0, atol=1e-12) and abs(tr1 - n * b) <= 1e-11
        # only the block-tridiagonal part of T^-1 enters (Sec. 3.1): the same
        # diagonal from the selected inverse of the sequential algorithm
        _, _, Sd, So = btd.thomas(D, O, np.zeros((n, b)))
        d2 = np.einsum("ipq,iqp->ip", Sd, Xd)
        d2[1:] += np.einsum("ipq,ipq->ip", So, Xo)
        d2[:-1] += np.einsum("iqp,iqp->ip", So, Xo)
        assert np.allclose(d2, d, rtol=1e-11, atol=1e-12)



# ---------------------------------------------------------------- the EQ approximation of order N

def test_eq_factor_is_the_stable_spectral_factor():
    """The oracle's factor s^N + a_{N-1} s^{N-1} + ... + a_0: its roots are
    the left-half-plane roots of sum_n (-s^2/2)^n / n! found by a library
    polynomial solver, and |Q(i w)|^2 times the leading coefficient of the
    Taylor polynomial reproduces p(w) = sum_n (w^2/2)^n / n! (the spectral
    factorisation of the approximate inverse spectral density)."""
    import math
    for N in (2, 4, 6, 8, 10, 12, 14, 16):
        a = seq.eq_factor(N)
        c = np.zeros(2 * N + 1)
        for n in range(N + 1):
            c[2 * N - 2 * n] = (-0.5) ** n / math.factorial(n)
        r = np.roots(c)
        ref = np.real(np.poly(r[r.real < 0]))[::-1][:N]
        assert np.max(np.abs(a - ref) / np.abs(ref)) <= 1e-11, N
        roots = np.roots(np.concatenate([[1.0], a[::-1]]))
        assert np.all(roots.real < 0), N
        w = np.linspace(0.1, 3.0, 7)
        q = np.polyval(np.concatenate([[1.0], a[::-1]]), 1j * w)
        p = sum((w * w / 2) ** n / math.factorial(n) for n in range(N + 1))
        lead = 0.5 ** N / math.factorial(N)
        assert np.max(np.abs(lead * np.abs(q) ** 2 - p) / p) <= 1e-12, N


def test_eq_approximation_approaches_the_exponentiated_quadratic():
    """The uniform error of the order-N covariance against s exp(-tau^2/(2 l^2))
    falls with N (the controllable approximation of Sec. 2.1); at N = 10 it is
    below 2e-4 s."""
    tau = np.linspace(-6.0, 6.0, 601)
    ell, var = 0.8, 1.7
    errs = []
    for N in (2, 4, 6, 8, 10, 12):
        k, _ = dense.kernel([("eq", N)], [ell, var, 0.1], tau)
        errs.append(np.max(np.abs(k - dense.eq_exact(var, ell, tau))))
    assert all(e2 < e1 for e1, e2 in zip(errs, errs[1:])), errs
    assert errs[4] <= 2e-4 * var


@pytest.mark.parametrize("N,tol", [(6, 1e-10), (10, 1e-9)])
def test_eq_state_space_covariance_at_higher_order(N, tol):
    """G bold-K G^T of the companion-form model against the residue formula at
    orders where the companion coordinates are ill-conditioned: the
    stationary covariance of (f, f', .., f^(N-1)) has condition number about
    2e4 (N = 6) and 3e9 (N = 10), so agreement is limited to about that
    times the unit roundoff; the tolerances state it."""
    t, _ = _series(30, 0.2, 2)
    th = [0.7, 1.3, 0.1]
    M = btd.stacked([("eq", N)], th, t)
    K, _ = dense.gram([("eq", N)], th, t)
    GKG = M["G"] @ M["Kc"] @ M["G"].T
    assert np.max(np.abs(GKG - K)) <= tol * np.max(np.abs(K))


def test_eq_dense_equals_sequential_at_order_10():
    """The paper's order: log-likelihood and gradient of the sequential oracle
    against the dense GP on the residue-formula kernel, Matern-3/2 + EQ(10)
    (the b = 12 model of Sec. 4.2), within the conditioning of the order-10
    state space."""
    spec = ["matern32", ("eq", 10)]
    th = [1.0, 0.5, 0.7, 1.3, 0.1]
    t, y = _series(300, 0.1, 4)
    ll_s, g_s = seq.grad(spec, th, t, y)
    ll_d, g_d = dense.grad(spec, th, t, y)
    assert abs(ll_s - ll_d) <= 1e-9 * abs(ll_d)
    assert np.max(np.abs(g_s - g_d)) <= 1e-8 * np.max(np.abs(g_d))
