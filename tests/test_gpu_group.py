"""GPU parity for structured models on the group path (sums of Matern-3/2,
periodic and quasi-periodic components, b = 2K <= 16) against the oracle.
Tolerances as in test_gpu_parity."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import seq  # noqa: E402
from paper_1610_08035_gb300 import autotune, spingp, synth  # noqa: E402

pytestmark = pytest.mark.gpu
DEV = "cuda"

CONFIG3 = (["matern32", ("quasiperiodic", 6, "matern12")], [1.0, 1.0, 1.0, 1.0, 1.0, 10.0, 0.01])
MODELS = [
    CONFIG3,
    (["matern32", "matern32"], [0.7, 1.2, 3.0, 0.5, 0.05]),
    ([("periodic", 3)], [1.2, 1.0, 0.8, 0.1]),
    (["matern32", ("periodic", 2)], [0.5, 0.8, 1.1, 0.9, 1.7, 0.05]),
    ([("quasiperiodic", 3, "matern12")], [0.9, 1.3, 0.6, 3.0, 0.02]),
]


def _t(a):
    return torch.tensor(np.asarray(a, dtype=np.float64), device=DEV)


def series(n, mean_dt, seed, ties=0, gaps=0):
    rng = np.random.default_rng(seed)
    d = rng.exponential(mean_dt, n)
    d[0] = 0.0
    if ties:
        d[::ties] = 0.0
    if gaps:
        d[gaps::gaps * 3 + 1] = 200 * mean_dt
    t = np.cumsum(d)
    y = synth.two_sinusoids(t, 1.0, 1.0, 0.05, rng)
    return t, y


def check(spec, theta, t, y, L=0, posterior=True):
    m = spingp.Model(spec, chunk_len=L)
    T, Y, TH = _t(t), _t(y), _t(theta)
    ll, g = m.grad(T, Y, TH)
    ll, g = float(ll.cpu()[0]), g.cpu().numpy()
    ll1 = float(m.loglik(T, Y, TH).cpu()[0])
    if posterior:
        mean, var, ll2 = m.posterior(T, Y, TH)
        llo, go, mo, vo, g1 = seq.grad(spec, theta, t, y, posterior=True, l1=True)
        dm = np.abs(mean.cpu().numpy() - mo)
        assert np.all(dm <= 1e-8 * np.maximum(np.abs(mo), np.sqrt(vo))), dm.max()
        assert np.all(np.abs(var.cpu().numpy() - vo) <= 1e-8 * vo), np.max(np.abs(var.cpu().numpy() - vo) / vo)
        assert abs(float(ll2.cpu()[0]) - llo) <= 1e-9 * abs(llo)
    else:
        llo, go, g1 = seq.grad(spec, theta, t, y, l1=True)
    assert abs(ll - llo) <= 1e-9 * abs(llo), (ll, llo)
    assert abs(ll1 - llo) <= 1e-9 * abs(llo), (ll1, llo)
    assert np.all(np.abs(g - go) <= 1e-8 * np.maximum(np.abs(go), g1)), (g, go, g1)


@pytest.mark.parametrize("spec,theta", MODELS)
@pytest.mark.parametrize("n,L", [(1, 0), (5, 0), (1000, 8), (3000, 0), (4099, 64)])
def test_group_parity(spec, theta, n, L):
    t, y = series(n, 0.01, n + L)
    check(spec, theta, t, y, L)


@pytest.mark.parametrize("spec,theta", MODELS[:3])
def test_group_ties_and_gaps(spec, theta):
    t, y = series(6000, 0.01, 4, ties=7, gaps=53)
    check(spec, theta, t, y, 16)


def test_config3_against_oracle():
    """Matern-3/2 + quasi-periodic (order 6, Matern-1/2 envelope), b = 16, the
    benchmark's chunk length, 2^16 steps against the oracle."""
    s = synth.single("sum_qp_n1m", n=1 << 16)
    check(s.spec, s.theta, s.t, s.y, 0, posterior=True)


def test_config3_full_size_against_oracle():
    """The b = 16 workload (Matern-3/2 + quasi-periodic of order 6 with a
    Matern-1/2 envelope, 7 parameters) in the benchmark's launch
    configuration: the log-likelihood over the whole N = 2^20 series, and the
    log-likelihood and all 7 gradient entries over its first 2^18 steps,
    against the oracle (its gradient at b = 16 runs at ~5e3 steps/s on one
    host core, so the whole series' gradient would take minutes)."""
    s = synth.single("sum_qp_n1m")
    m = spingp.Model(s.spec)
    autotune.tune(m, _t(s.t), _t(s.y), _t(s.theta), spingp.WS_GRAD)   # the benchmark's launch configuration
    ll = float(m.loglik(_t(s.t), _t(s.y), _t(s.theta)).cpu()[0])
    llo = seq.loglik(s.spec, s.theta, s.t, s.y)
    assert abs(ll - llo) <= 1e-9 * abs(llo), (ll, llo)
    n = 1 << 18
    t, y = s.t[:n], s.y[:n]
    ll, g = m.grad(_t(t), _t(y), _t(s.theta))
    ll, g = float(ll.cpu()[0]), g.cpu().numpy()
    llo, go, g1 = seq.grad(s.spec, s.theta, t, y, l1=True)
    assert abs(ll - llo) <= 1e-9 * abs(llo), (ll, llo)
    assert np.all(np.abs(g - go) <= 1e-8 * np.maximum(np.abs(go), g1)), (g, go, g1)


def test_config3_full_size_posterior_windows():
    """The b = 16 workload's posterior (mean and the variances of the
    selected inverse) at full size, N = 2^20 in the benchmark's launch
    configuration: 6 sampled steps against the oracle's smoother on a window
    of +-20000 steps (200 time units) around each.  The slowest-decaying
    component, the quasi-periodic one, carries a Matern-1/2 envelope of
    lengthscale 10, so data beyond the window moves the posterior at its
    centre by at most about e^-20 (2e-9) of its scale; measured on the
    oracle, widening the window to +-30000 steps moves the centre's mean by
    3e-15 and its variance by 1e-13 relative."""
    s = synth.single("sum_qp_n1m")
    m = spingp.Model(s.spec)
    T, Y, TH = _t(s.t), _t(s.y), _t(s.theta)
    autotune.tune(m, T, Y, TH, spingp.WS_GRAD)
    mean, var, _ = m.posterior(T, Y, TH, with_loglik=False)
    mean, var = mean.cpu().numpy(), var.cpu().numpy()
    # the benchmark's step for this workload is the fused call: its posterior
    # equals the posterior call's up to rounding order, so the windows below
    # hold for it too
    _, _, mf, vf, _ = m.grad_posterior(T, Y, TH)
    mf, vf = mf.cpu().numpy(), vf.cpu().numpy()
    vmax = float(var.max())
    assert np.max(np.abs(mf - mean)) <= 1e-13 * max(float(np.abs(mean).max()), np.sqrt(vmax))
    assert np.max(np.abs(vf - var)) <= 1e-13 * vmax
    for i in np.random.default_rng(2).integers(20000, len(s.t) - 20000, 6):
        a, b = i - 20000, i + 20001
        sm = seq.smoother(s.spec, s.theta, s.t[a:b], s.y[a:b])
        mo, vo = sm["mean"][20000], sm["var"][20000]
        assert abs(mean[i] - mo) <= 1e-8 * max(abs(mo), np.sqrt(vo)), (i, mean[i], mo)
        assert abs(var[i] - vo) <= 1e-8 * vo, (i, var[i], vo)


def test_config3_full_size_identity():
    """b = 16 at N = 2^20: scaling every variance (s_m32, s_per, s_n) by c scales
    C by c, so sum_v s_v dl/ds_v = (y^T C^-1 y - N)/2 with y^T C^-1 y read off
    l(2 s) - l(s)."""
    s = synth.single("sum_qp_n1m")
    m = spingp.Model(s.spec)
    T, Y = _t(s.t), _t(s.y)
    th = s.theta.copy()
    ll, g = m.grad(T, Y, _t(th))
    ll, g = float(ll.cpu()[0]), g.cpu().numpy()
    var_idx = [1, 2, 6]
    th2 = th.copy(); th2[var_idx] *= 2.0
    ll2 = float(m.loglik(T, Y, _t(th2)).cpu()[0])
    n = len(s.t)
    q = 4.0 * (ll2 - ll + 0.5 * n * np.log(2.0))
    lhs = sum(th[i] * g[i] for i in var_idx)
    assert abs(lhs - (0.5 * q - 0.5 * n)) <= 1e-8 * (sum(abs(th[i] * g[i]) for i in var_idx) + n)
    # deterministic
    ll_b, g_b = m.grad(T, Y, _t(th))
    assert float(ll_b.cpu()[0]) == ll and np.array_equal(g_b.cpu().numpy(), g)
