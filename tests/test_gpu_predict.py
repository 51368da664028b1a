"""GPU parity for prediction at new times (Eqs. mean4-mean6) and for series
with missing observations: test points ride through the same chain with
infinite noise (NaN observations and the SPINGP_MISSING_NAN flag)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import dense, seq  # noqa: E402
from paper_1610_08035_gb300 import spingp, synth  # noqa: E402

pytestmark = pytest.mark.gpu
DEV = "cuda"

MODELS = [("matern12", [0.7, 1.3, 0.1]), ("matern32", [1.0, 1.0, 0.1]), ("matern52", [0.5, 2.0, 0.05]),
          (["matern32", ("quasiperiodic", 3, "matern12")], [0.9, 1.1, 0.8, 1.2, 0.9, 3.0, 0.02])]


def _t(a):
    return torch.tensor(np.asarray(a, dtype=np.float64), device=DEV)


def data(n, m_new, seed):
    rng = np.random.default_rng(seed)
    t = synth.exp_times(n, 0.05, rng)
    y = synth.two_sinusoids(t, 0.8, 1.0, 0.1, rng)
    t_new = rng.uniform(t[0] - 1.0, t[-1] + 1.0, m_new)
    t_new[:3] = t[[5, 5, n // 2]]          # test points tied with observed times
    return t, y, t_new


@pytest.mark.parametrize("spec,theta", MODELS)
def test_predict_matches_dense_gp(spec, theta):
    t, y, t_new = data(400, 90, 3)
    m = spingp.Model(spec, chunk_len=8)
    mean, var = m.predict(_t(t), _t(y), _t(theta), _t(t_new))
    md, vd = dense.predict(spec, theta, t, y, t_new)
    tol = 1e-8 if len(theta) == 3 else 1e-7
    assert np.max(np.abs(mean.cpu().numpy() - md)) <= tol * max(1.0, np.max(np.abs(md)))
    assert np.max(np.abs(var.cpu().numpy() - vd) / vd) <= tol


@pytest.mark.parametrize("spec,theta", MODELS)
@pytest.mark.parametrize("L", [0, 16])
def test_missing_observations_against_oracle(spec, theta, L):
    """A long series with a fifth of its observations missing (in runs and
    singly, including the first and last step): log-likelihood, gradient,
    posterior at every step against the oracle (NaN = missing there too)."""
    rng = np.random.default_rng(5)
    n = 30000
    t = synth.exp_times(n, 0.01, rng)
    y = synth.two_sinusoids(t, 0.8, 1.0, 0.1, rng)
    miss = rng.random(n) < 0.2
    miss[1000:1400] = True
    miss[0] = miss[-1] = True
    y[miss] = np.nan
    m = spingp.Model(spec, chunk_len=L)
    T, Y, TH = _t(t), _t(y), _t(theta)
    ll, g = m.grad(T, Y, TH, missing=True)
    mean, var, llp = m.posterior(T, Y, TH, missing=True)
    llo, go, mo, vo, g1 = seq.grad(spec, theta, t, y, posterior=True, l1=True)
    assert abs(float(ll.cpu()[0]) - llo) <= 1e-9 * abs(llo)
    assert abs(float(llp.cpu()[0]) - llo) <= 1e-9 * abs(llo)
    assert np.all(np.abs(g.cpu().numpy() - go) <= 1e-8 * np.maximum(np.abs(go), g1))
    dm = np.abs(mean.cpu().numpy() - mo)
    assert np.all(dm <= 1e-8 * np.maximum(np.abs(mo), np.sqrt(vo))), dm.max()
    assert np.all(np.abs(var.cpu().numpy() - vo) <= 1e-8 * vo)


def test_nan_without_flag_is_an_error():
    m = spingp.Model("matern32")
    t = np.arange(100.0) * 0.1
    y = np.sin(t); y[7] = np.nan
    with pytest.raises(spingp.SpinGPError) as e:
        m.loglik(_t(t), _t(y), _t([1.0, 1.0, 0.1]))
    assert e.value.status == spingp.ENONFINITE


def test_missing_in_batches():
    rng = np.random.default_rng(8)
    lengths = [300, 1, 2000, 57]
    offsets = np.concatenate([[0], np.cumsum(lengths)]).astype(np.int64)
    t = np.concatenate([synth.exp_times(n, 0.02, rng) for n in lengths])
    y = np.sin(3 * t) + 0.1 * rng.standard_normal(len(t))
    y[rng.random(len(t)) < 0.3] = np.nan
    y[offsets[1]] = np.nan                        # the one-step series is all missing
    th = np.tile([0.5, 1.2, 0.05], (4, 1))
    m = spingp.Model("matern52")
    bt = spingp.Batch(m, torch.tensor(offsets, device=DEV), _t(t), _t(y))
    ws = bt.workspace(spingp.WS_GRAD)
    ll = torch.empty(4, dtype=torch.float64, device=DEV)
    g = torch.empty(12, dtype=torch.float64, device=DEV)
    st = spingp.spingp_grad_batched(m.h, bt.offsets, 4, len(t), bt.t, bt.y, _t(th.reshape(-1)), ll, g, ws,
                                    ws.numel(), spingp.SYNC | spingp.MISSING_NAN)
    assert st == spingp.OK
    ll, g = ll.cpu().numpy(), g.cpu().numpy().reshape(4, 3)
    for i in range(4):
        a, b = offsets[i], offsets[i + 1]
        yi = y[a:b]
        if np.all(np.isnan(yi)):
            assert ll[i] == 0.0 and np.all(g[i] == 0.0)
            continue
        llo, go, g1 = seq.grad("matern52", th[i], t[a:b], yi, l1=True)
        assert abs(ll[i] - llo) <= 1e-9 * abs(llo)
        assert np.all(np.abs(g[i] - go) <= 1e-8 * np.maximum(np.abs(go), g1))


# ---- spingp_predict itself: the device sort of t*, the merge, the gather

def _host_merged(t, y, ts):
    """The merged series built on the host (observations first at equal
    times, the test points in stable sorted order) and where each test point
    lands: the same posterior pass, assembled without the predict kernels."""
    order = np.argsort(ts, kind="stable")
    T = np.concatenate([t, ts[order]])
    Y = np.concatenate([y, np.full(len(ts), np.nan)])
    o = np.argsort(T, kind="stable")
    where = np.empty(len(T), dtype=np.int64)
    where[o] = np.arange(len(T))
    pos = np.empty(len(ts), dtype=np.int64)
    pos[order] = where[len(t):]
    return T[o], Y[o], pos


@pytest.mark.parametrize("spec,theta", [MODELS[2], MODELS[3]])
@pytest.mark.parametrize("n,m_new", [(1000, 1), (1000, 7), (5000, 4099), (3000, 100000)])
def test_predict_equals_the_posterior_of_the_merged_series(spec, theta, n, m_new):
    """Test times in any order, ties among themselves and with observed times,
    outside the observed range: spingp_predict returns, bit for bit, the
    posterior call's moments on the host-merged series at each test point."""
    rng = np.random.default_rng(n + m_new)
    t = synth.exp_times(n, 0.05, rng)
    y = synth.two_sinusoids(t, 0.8, 1.0, 0.1, rng)
    ts = rng.uniform(t[0] - 2.0, t[-1] + 2.0, m_new)
    k = min(m_new, 5)
    ts[:k] = t[rng.integers(0, n, k)]                 # tied with observed times
    if m_new > 10:
        ts[-4:] = ts[-8:-4]                           # tied among themselves
    m = spingp.Model(spec)
    mean, var = m.predict(_t(t), _t(y), _t(theta), _t(ts))
    T, Y, pos = _host_merged(t, y, ts)
    mp, vp, _ = m.posterior(_t(T), _t(Y), _t(theta), missing=True, with_loglik=False)
    assert torch.equal(mean, mp[torch.tensor(pos, device=DEV)])
    assert torch.equal(var, vp[torch.tensor(pos, device=DEV)])


def test_predict_prior_flags_and_errors():
    """No observations gives the prior (zero mean, variance s_f); the
    predictive flag adds s_n; unsorted observed times and a NaN test time are
    reported through the status word; bad arguments are EINVAL."""
    m = spingp.Model("matern32")
    th = _t([1.0, 1.7, 0.1])
    ts = _t([3.0, -1.0, 2.5])
    empty = torch.empty(0, dtype=torch.float64, device=DEV)
    mean, var = m.predict(empty, empty, th, ts)
    assert torch.all(mean == 0.0) and torch.allclose(var, torch.full_like(var, 1.7), rtol=1e-15, atol=0.0)
    t, y = _t(np.arange(50) * 0.1), _t(np.sin(np.arange(50) * 0.1))
    mean, var = m.predict(t, y, th, ts)
    mean2, var2 = m.predict(t, y, th, ts, predictive=True)
    assert torch.equal(mean, mean2) and torch.allclose(var2, var + 0.1, rtol=1e-15, atol=0.0)
    with pytest.raises(spingp.SpinGPError) as e:
        m.predict(torch.flip(t, [0]), y, th, ts)
    assert e.value.status == spingp.ENOTSORTED
    with pytest.raises(spingp.SpinGPError) as e:
        m.predict(t, y, th, _t([0.5, float("nan"), 1.0]))
    assert e.value.status == spingp.ENONFINITE
    ws = torch.empty(spingp.spingp_predict_workspace_bytes(m.h, 50, 3), dtype=torch.uint8, device=DEV)
    out = torch.empty(3, dtype=torch.float64, device=DEV)
    assert spingp.spingp_predict(m.h, t, y, 50, th, ts, 0, out, out, ws, ws.numel(), spingp.SYNC) == spingp.EINVAL
    assert spingp.spingp_predict(m.h, t, y, 50, th, ts, 3, None, out, ws, ws.numel(), spingp.SYNC) == spingp.EINVAL
    assert spingp.spingp_predict(m.h, t, y, 50, th, ts, 3, out, out, ws, 256, spingp.SYNC) == spingp.EINVAL
