"""One series split across ranks, on one GPU: the ranks are emulated in one
process (each range with its own workspace), the all-gather is a stack of
the ranges' elements in rank order, and the all-reduce is a sum of the
shares.  The summed shares must equal the whole-series gradient call (the
same arithmetic on a different chunking: rounding only) and the oracle."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import seq  # noqa: E402
from paper_1610_08035_gb300 import shard, spingp, synth  # noqa: E402

pytestmark = pytest.mark.gpu
DEV = "cuda"

MATERN = [("matern12", [0.7, 1.3, 0.2]), ("matern32", [1.0, 1.0, 0.1]), ("matern52", [0.5, 2.0, 0.05])]


def _t(a):
    return torch.tensor(np.asarray(a, dtype=np.float64), device=DEV)


def _split_grad(m, T, Y, TH, ranges, t_host, missing=False):
    wss, elems = [], []
    for r, (a, b) in enumerate(ranges):
        ws = torch.empty(spingp.spingp_workspace_bytes(m.h, b - a, spingp.WS_GRAD), dtype=torch.uint8, device=DEV)
        t_prev = None if r == 0 else float(t_host[a - 1])
        elems.append(m.segment_reduce(T[a:b], Y[a:b], TH, t_prev=t_prev, ws=ws, missing=missing))
        wss.append(ws)
    E = torch.stack(elems)
    ll, g = 0.0, 0.0
    for r, (a, b) in enumerate(ranges):
        t_prev = None if r == 0 else float(t_host[a - 1])
        lr, gr = m.segment_grad(T[a:b], Y[a:b], TH, E, r, t_prev=t_prev, ws=wss[r], missing=missing)
        ll = ll + lr.item()
        g = g + gr.cpu().numpy()
    return ll, g


@pytest.mark.parametrize("spec,theta", MATERN)
@pytest.mark.parametrize("G", [1, 2, 3, 8])
def test_split_series_equals_whole(spec, theta, G):
    n = 40009
    rng = np.random.default_rng(G)
    t = synth.exp_times(n, 0.02, rng)
    y = synth.two_sinusoids(t, 0.5, 1.0, 0.1, rng)
    m = spingp.Model(spec)
    T, Y, TH = _t(t), _t(y), _t(theta)
    ll_w, g_w = m.grad(T, Y, TH)
    ll_w, g_w = ll_w.item(), g_w.cpu().numpy()
    ll, g = _split_grad(m, T, Y, TH, shard.range_split(n, G), t)
    assert abs(ll - ll_w) <= 1e-11 * abs(ll_w)
    assert np.max(np.abs(g - g_w) / np.abs(g_w)) <= 1e-10
    llo, go, gabs = seq.grad([spec], theta, t, y, l1=True)
    assert abs(ll - llo) <= 1e-9 * abs(llo)
    assert np.max(np.abs(g - go) / np.maximum(np.abs(go), gabs)) <= 1e-8


def test_split_series_uneven_ranges_and_missing():
    """Ranges of 1 step, shorter than a chunk, and long ones; missing
    observations, including at a range boundary."""
    n = 20011
    rng = np.random.default_rng(3)
    t = synth.exp_times(n, 0.02, rng)
    y = synth.two_sinusoids(t, 0.5, 1.0, 0.1, rng)
    y[rng.random(n) < 0.1] = np.nan
    cuts = [0, 1, 5, 1000, 1001, 15000, n]
    y[999] = np.nan
    ranges = list(zip(cuts[:-1], cuts[1:]))
    m = spingp.Model("matern52")
    T, Y, TH = _t(t), _t(y), _t([0.5, 2.0, 0.05])
    ll_w, g_w = m.grad(T, Y, TH, missing=True)
    ll, g = _split_grad(m, T, Y, TH, ranges, t, missing=True)
    assert abs(ll - ll_w.item()) <= 1e-11 * abs(ll_w.item())
    assert np.max(np.abs(g - g_w.cpu().numpy()) / np.abs(g_w.cpu().numpy())) <= 1e-10


def test_split_series_errors():
    m = spingp.Model("matern32")
    T, Y, TH = _t(np.arange(100.0)), _t(np.zeros(100)), _t([1.0, 1.0, 0.1])
    E = torch.zeros(2, spingp.spingp_segment_elem_size(m.h), dtype=torch.float64, device=DEV)
    with pytest.raises(spingp.SpinGPError):             # rank 1 must continue the series
        m.segment_grad(T, Y, TH, E, 1, t_prev=None)
    with pytest.raises(spingp.SpinGPError):             # rank 0 must start it
        m.segment_grad(T, Y, TH, E, 0, t_prev=-1.0)
    with pytest.raises(spingp.SpinGPError):
        m.segment_grad(T, Y, TH, torch.zeros(33, E.shape[1], dtype=torch.float64, device=DEV), 0)
    with pytest.raises(spingp.SpinGPError):              # t_prev after the range's first time
        m.segment_reduce(T, Y, TH, t_prev=5.0)
    g = spingp.Model([("periodic", 2)])
    assert spingp.spingp_segment_elem_size(g.h) == 16 * 50   # the group path's padded element


GROUP = [
    (["matern32", ("quasiperiodic", 6, "matern12")], [1.0, 1.0, 1.0, 1.0, 1.0, 10.0, 0.01]),   # b = 16
    (["matern32", ("eq", 6)], [1.0, 0.6, 0.7, 1.2, 0.05]),                                     # b = 8, EQ
    ([("periodic", 2)], [1.2, 1.0, 0.8, 0.1]),
]


@pytest.mark.parametrize("spec,theta", GROUP)
@pytest.mark.parametrize("G", [1, 2, 5])
def test_split_series_group_path(spec, theta, G):
    """Structured models (the group path) split the same way: the shares sum
    to the whole-series call and to the oracle."""
    n = 12007
    rng = np.random.default_rng(40 + G)
    t = synth.exp_times(n, 0.02, rng)
    y = synth.two_sinusoids(t, 0.8, 1.0, 0.1, rng)
    m = spingp.Model(spec)
    T, Y, TH = _t(t), _t(y), _t(theta)
    ll_w, g_w = m.grad(T, Y, TH)
    ll_w, g_w = ll_w.item(), g_w.cpu().numpy()
    ll, g = _split_grad(m, T, Y, TH, shard.range_split(n, G), t)
    assert abs(ll - ll_w) <= 1e-11 * abs(ll_w)
    llo, go, gabs = seq.grad(spec, theta, t, y, l1=True)
    gscale = np.maximum(np.abs(go), gabs)
    # the undamped periodic component keeps the elimination's rounding alive
    # across the whole series, so two chunkings differ by more than on the
    # chain path; the bar is still 10x inside the oracle bar below
    assert np.max(np.abs(g - g_w) / gscale) <= 1e-9
    assert abs(ll - llo) <= 1e-9 * abs(llo)
    assert np.max(np.abs(g - go) / gscale) <= 1e-8


def test_split_series_group_path_uneven_ranges_and_missing():
    """The group path with ranges of 1 step, shorter than a chunk, and long
    ones, missing observations (one at a range boundary)."""
    n = 9001
    rng = np.random.default_rng(44)
    t = synth.exp_times(n, 0.02, rng)
    y = synth.two_sinusoids(t, 0.8, 1.0, 0.1, rng)
    y[rng.random(n) < 0.1] = np.nan
    y[4000] = np.nan
    cuts = [0, 1, 2, 50, 4001, 4002, n]
    ranges = list(zip(cuts[:-1], cuts[1:]))
    spec, theta = GROUP[0]
    m = spingp.Model(spec)
    T, Y, TH = _t(t), _t(y), _t(theta)
    ll_w, g_w = m.grad(T, Y, TH, missing=True)
    ll_w, g_w = ll_w.item(), g_w.cpu().numpy()
    ll, g = _split_grad(m, T, Y, TH, ranges, t, missing=True)
    assert abs(ll - ll_w) <= 1e-11 * abs(ll_w)
    llo, go, gabs = seq.grad(spec, theta, t, y, l1=True)
    gscale = np.maximum(np.abs(go), gabs)
    assert np.max(np.abs(g - g_w) / gscale) <= 1e-9
    assert abs(ll - llo) <= 1e-9 * abs(llo)
    assert np.max(np.abs(g - go) / gscale) <= 1e-8


# ---- the posterior of a split series (spingp_segment_grad_posterior)

def _split_grad_posterior(m, T, Y, TH, ranges, t_host, missing=False, predictive=False):
    wss, elems = [], []
    for r, (a, b) in enumerate(ranges):
        ws = torch.empty(spingp.spingp_workspace_bytes(m.h, b - a, spingp.WS_GRAD), dtype=torch.uint8, device=DEV)
        t_prev = None if r == 0 else float(t_host[a - 1])
        elems.append(m.segment_reduce(T[a:b], Y[a:b], TH, t_prev=t_prev, ws=ws, missing=missing))
        wss.append(ws)
    E = torch.stack(elems)
    ll, g, means, vars_ = 0.0, 0.0, [], []
    for r, (a, b) in enumerate(ranges):
        t_prev = None if r == 0 else float(t_host[a - 1])
        lr, gr, mr, vr = m.segment_grad_posterior(T[a:b], Y[a:b], TH, E, r, t_prev=t_prev, ws=wss[r],
                                                  missing=missing, predictive=predictive)
        ll = ll + lr.item()
        g = g + gr.cpu().numpy()
        means.append(mr.cpu().numpy())
        vars_.append(vr.cpu().numpy())
    return ll, g, np.concatenate(means), np.concatenate(vars_)


def _check_split_posterior(spec, theta, t, y, ranges, missing=False):
    """The split outputs against the whole-series fused call (a different
    chunking: rounding only; 1e-10 of the posterior's scale, the gradient at
    the split-gradient bars) and against the oracle's smoother at the parity
    bars (mean 1e-8 max(|m|, sqrt v), variance 1e-8 v)."""
    m = spingp.Model(spec)
    T, Y, TH = _t(t), _t(y), _t(theta)
    ll_w, g_w, m_w, v_w, _ = m.grad_posterior(T, Y, TH, missing=missing)
    ll, g, mean, var = _split_grad_posterior(m, T, Y, TH, ranges, t, missing=missing)
    ll_w, g_w, m_w, v_w = ll_w.item(), g_w.cpu().numpy(), m_w.cpu().numpy(), v_w.cpu().numpy()
    assert abs(ll - ll_w) <= 1e-11 * abs(ll_w)
    llo, go, gabs = seq.grad(spec, theta, t, y, l1=True)
    gscale = np.maximum(np.abs(go), gabs)
    assert np.max(np.abs(g - g_w) / gscale) <= 1e-9
    scale = np.maximum(np.abs(m_w), np.sqrt(v_w))
    assert np.max(np.abs(mean - m_w) / scale) <= 1e-10
    assert np.max(np.abs(var - v_w) / v_w) <= 1e-10
    sm = seq.smoother(spec, theta, t, y)
    mo, vo = sm["mean"], sm["var"]
    assert np.max(np.abs(mean - mo) / np.maximum(np.abs(mo), np.sqrt(vo))) <= 1e-8
    assert np.max(np.abs(var - vo) / vo) <= 1e-8
    assert abs(ll - llo) <= 1e-9 * abs(llo)
    assert np.max(np.abs(g - go) / gscale) <= 1e-8


@pytest.mark.parametrize("spec,theta", MATERN)
@pytest.mark.parametrize("G", [1, 2, 3, 8])
def test_split_series_posterior(spec, theta, G):
    n = 30011
    rng = np.random.default_rng(60 + G)
    t = synth.exp_times(n, 0.02, rng)
    y = synth.two_sinusoids(t, 0.5, 1.0, 0.1, rng)
    _check_split_posterior([spec], theta, t, y, shard.range_split(n, G))


@pytest.mark.parametrize("spec,theta", GROUP)
@pytest.mark.parametrize("G", [1, 3])
def test_split_series_posterior_group_path(spec, theta, G):
    n = 6007
    rng = np.random.default_rng(70 + G)
    t = synth.exp_times(n, 0.02, rng)
    y = synth.two_sinusoids(t, 0.8, 1.0, 0.1, rng)
    _check_split_posterior(spec, theta, t, y, shard.range_split(n, G))


@pytest.mark.parametrize("spec,theta", [MATERN[2], GROUP[0]])
def test_split_series_posterior_uneven_ranges_and_missing(spec, theta):
    """Ranges of 1 and 2 steps and long ones; missing observations, among
    them a range's first and last steps and a whole short range."""
    n = 5003
    rng = np.random.default_rng(81)
    t = synth.exp_times(n, 0.02, rng)
    y = synth.two_sinusoids(t, 0.8, 1.0, 0.1, rng)
    y[rng.random(n) < 0.1] = np.nan
    cuts = [0, 1, 3, 40, 2501, 2502, n]
    y[1:3] = np.nan
    y[40] = y[2500] = np.nan
    ranges = list(zip(cuts[:-1], cuts[1:]))
    _check_split_posterior(spec if isinstance(spec, list) else [spec], theta, t, y, ranges, missing=True)


def test_split_series_posterior_predictive_flag():
    n = 3001
    rng = np.random.default_rng(90)
    t = synth.exp_times(n, 0.02, rng)
    y = synth.two_sinusoids(t, 0.8, 1.0, 0.1, rng)
    m = spingp.Model("matern32")
    T, Y, TH = _t(t), _t(y), _t([1.0, 1.0, 0.1])
    ranges = shard.range_split(n, 2)
    _, _, _, v = _split_grad_posterior(m, T, Y, TH, ranges, t)
    _, _, _, vp = _split_grad_posterior(m, T, Y, TH, ranges, t, predictive=True)
    assert np.array_equal(vp, v + 0.1)
