"""The first off-diagonal of the selected inverse (Sec. 3.1) from the fused
path: spingp_posterior_lag1's Cov(f_{i+1}, f_i | y) against the oracle's
Rauch-Tung-Striebel lag-one blocks H P^s_{i+1,i} H^T, element by element.

Bar: |d c_i| <= 1e-8 sqrt(v_i v_{i+1}) with v the oracle's latent variances
(the scale Cauchy-Schwarz gives the covariance), and the mean and variance
outputs equal spingp_posterior's bit for bit."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import seq  # noqa: E402
from paper_1610_08035_gb300 import spingp, synth  # noqa: E402

pytestmark = pytest.mark.gpu
DEV = "cuda"


def _t(a):
    return torch.tensor(np.asarray(a, dtype=np.float64), device=DEV)


def _series(n, mean_dt, seed, missing=0.0, ties=0):
    rng = np.random.default_rng(seed)
    d = rng.exponential(mean_dt, n)
    d[0] = 0.0
    if ties:
        d[::ties] = 0.0
    t = np.cumsum(d)
    y = synth.two_sinusoids(t, 1.0, 1.0, 0.05, rng)
    if missing:
        y[rng.random(n) < missing] = np.nan
    return t, y


def _check(spec, theta, t, y, L=0, missing=False):
    m = spingp.Model(spec, chunk_len=L)
    T, Y, TH = _t(t), _t(y), _t(theta)
    mean, var, lag, ll = m.posterior_lag1(T, Y, TH, missing=missing)
    mean0, var0, ll0 = m.posterior(T, Y, TH, missing=missing)
    assert torch.equal(mean, mean0) and torch.equal(var, var0) and torch.equal(ll, ll0)
    sm = seq.smoother(spec, theta, t, y, blocks=True)
    h = seq.continuous(spec, theta)[2]
    co = np.einsum("i,nij,j->n", h, sm["Pc"], h)
    vo = sm["var"]
    lag = lag.cpu().numpy()
    assert lag.shape == co.shape
    err = np.abs(lag - co) / np.sqrt(vo[1:] * vo[:-1])
    assert np.all(err <= 1e-8), (err.max(), int(np.argmax(err)))


@pytest.mark.parametrize("spec,theta", [("matern12", [0.7, 1.3, 0.1]), ("matern32", [1.0, 1.0, 0.1]),
                                        ("matern52", [0.5, 2.0, 0.05])])
@pytest.mark.parametrize("n,L", [(2, 0), (7, 0), (1000, 8), (10007, 0), (10007, 64)])
def test_lag1_chain(spec, theta, n, L):
    t, y = _series(n, 0.01, n + L)
    _check(spec, theta, t, y, L)


@pytest.mark.parametrize("spec,theta", [("matern32", [1.0, 1.0, 0.1]), ("matern52", [0.5, 2.0, 0.05])])
def test_lag1_chain_missing_and_ties(spec, theta):
    t, y = _series(6000, 0.01, 5, missing=0.2, ties=7)
    _check(spec, theta, t, y, 16, missing=True)


GROUP = [
    (["matern32", ("quasiperiodic", 6, "matern12")], [1.0, 1.0, 1.0, 1.0, 1.0, 10.0, 0.01]),   # b = 16
    (["matern32", ("periodic", 2)], [0.5, 0.8, 1.1, 0.9, 1.7, 0.05]),
    (["matern32", ("eq", 6), ("periodic", 1)], [1.0, 0.5, 0.6, 1.1, 0.8, 1.2, 2.0, 0.05]),
    (["matern32", ("eq", 10)], [1.0, 0.5, 0.7, 1.3, 0.1]),                                        # b = 12
]


@pytest.mark.parametrize("spec,theta", GROUP)
@pytest.mark.parametrize("n,L", [(2, 0), (1000, 8), (5003, 0)])
def test_lag1_group(spec, theta, n, L):
    t, y = _series(n, 0.02, 3 * n + L)
    _check(spec, theta, t, y, L)


@pytest.mark.parametrize("spec,theta", GROUP[:2] + GROUP[3:])
def test_lag1_group_missing(spec, theta):
    t, y = _series(3000, 0.02, 9, missing=0.15)
    _check(spec, theta, t, y, 32, missing=True)


@pytest.mark.parametrize("spec,theta", [("matern52", [0.5, 2.0, 0.05]), GROUP[1]])
def test_lag1_missing_edges(spec, theta):
    """A missing first and last observation, a run of missing ones across
    chunk boundaries, and an all-missing series (the prior's lag-one
    covariance k(t_{i+1} - t_i))."""
    t, y = _series(700, 0.02, 41)
    y[0] = y[-1] = np.nan
    y[100:260] = np.nan
    _check(spec, theta, t, y, 16, missing=True)
    y[:] = np.nan
    _check(spec, theta, t, y, 16, missing=True)


def test_lag1_single_step_needs_no_buffer():
    m = spingp.Model("matern52")
    T, Y, TH = _t([0.0]), _t([0.3]), _t([0.5, 2.0, 0.05])
    ws = m.workspace(1, spingp.WS_POSTERIOR, DEV)
    mean = torch.empty(1, dtype=torch.float64, device=DEV)
    var = torch.empty(1, dtype=torch.float64, device=DEV)
    st = spingp.spingp_posterior_lag1(m.h, T, Y, 1, TH, None, mean, var, None, ws, ws.numel(), spingp.SYNC)
    assert st == spingp.OK
    T2, Y2 = _t([0.0, 0.1]), _t([0.3, 0.2])
    ws2 = m.workspace(2, spingp.WS_POSTERIOR, DEV)
    mean2 = torch.empty(2, dtype=torch.float64, device=DEV)
    var2 = torch.empty(2, dtype=torch.float64, device=DEV)
    st = spingp.spingp_posterior_lag1(m.h, T2, Y2, 2, TH, None, mean2, var2, None, ws2, ws2.numel(), spingp.SYNC)
    assert st == spingp.EINVAL
