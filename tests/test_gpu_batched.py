"""GPU parity for batches of independent series (spingp_*_batched) against the
oracle, series by series.  Tolerances as in test_gpu_parity."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import seq  # noqa: E402
from paper_1610_08035_gb300 import autotune, spingp, synth  # noqa: E402

pytestmark = pytest.mark.gpu
DEV = "cuda"


def _t(a, dtype=torch.float64):
    return torch.tensor(np.asarray(a), dtype=dtype, device=DEV)


def small_batch(spec, seed, lengths):
    rng = np.random.default_rng(seed)
    offsets = np.zeros(len(lengths) + 1, dtype=np.int64)
    offsets[1:] = np.cumsum(lengths)
    t = np.empty(offsets[-1]); y = np.empty(offsets[-1])
    th = np.stack([synth.log_uniform(0.1, 10.0, len(lengths), rng), synth.log_uniform(0.5, 2.0, len(lengths), rng),
                   synth.log_uniform(0.01, 0.5, len(lengths), rng)], axis=1)
    for i, n in enumerate(lengths):
        a, b = offsets[i], offsets[i + 1]
        ti = synth.exp_times(n, 0.01, rng) if n else np.empty(0)
        if n > 10:
            ti[5] = ti[4]                      # a tie inside the series
        t[a:b] = ti
        y[a:b] = synth.two_sinusoids(ti, th[i, 0], th[i, 1], th[i, 2], rng) if n else np.empty(0)
    return offsets, t, y, th


def check_series(spec, offsets, t, y, th, ll, g, idx, mean=None, var=None):
    for i in idx:
        a, b = offsets[i], offsets[i + 1]
        if a == b:
            assert ll[i] == 0.0 and np.all(g[i] == 0.0)
            continue
        if mean is not None:
            llo, go, mo, vo, g1 = seq.grad(spec, th[i], t[a:b], y[a:b], posterior=True, l1=True)
            dm = np.abs(mean[a:b] - mo)
            assert np.all(dm <= 1e-8 * np.maximum(np.abs(mo), np.sqrt(vo))), (i, dm.max())
            assert np.all(np.abs(var[a:b] - vo) <= 1e-8 * vo), i
        else:
            llo, go, g1 = seq.grad(spec, th[i], t[a:b], y[a:b], l1=True)
        assert abs(ll[i] - llo) <= 1e-9 * abs(llo), (i, ll[i], llo)
        if g is not None:
            assert np.all(np.abs(g[i] - go) <= 1e-8 * np.maximum(np.abs(go), g1)), (i, g[i], go)


@pytest.mark.parametrize("spec", ["matern12", "matern32", "matern52"])
@pytest.mark.parametrize("L", [0, 8, 64])
def test_batched_small(spec, L):
    lengths = [1, 2, 0, 3000, 7, 513, 0, 129, 1000, 64, 65, 2500] + [int(v) for v in
                                                                     np.random.default_rng(1).integers(1, 3000, 52)]
    offsets, t, y, th = small_batch(spec, 7, lengths)
    m = spingp.Model(spec, chunk_len=L)
    bt = spingp.Batch(m, _t(offsets, torch.int64), _t(t), _t(y))
    ll, g = bt.grad(_t(th.reshape(-1)))
    ll, g = ll.cpu().numpy(), g.cpu().numpy()
    ll2 = bt.loglik(_t(th.reshape(-1))).cpu().numpy()
    mean, var, ll3 = bt.posterior(_t(th.reshape(-1)))
    check_series(spec, offsets, t, y, th, ll, g, range(len(lengths)), mean.cpu().numpy(), var.cpu().numpy())
    nz = np.diff(offsets) > 0
    assert np.allclose(ll2[nz], ll[nz], rtol=1e-12, atol=0)
    assert np.allclose(ll3.cpu().numpy()[nz], ll[nz], rtol=1e-12, atol=0)


@pytest.mark.parametrize("L", [0, 16])
def test_batched_missing_observations(L):
    """Missing observations (NaN, Eqs. mean4-mean6) inside a batch: runs of
    them, single ones, a series with none observed and one observed only at
    its ends -- log-likelihood, gradient and posterior of every series
    against the oracle, where NaN means missing too."""
    lengths = [40, 1, 3000, 7, 0, 513, 129, 1000, 64, 2500, 90]
    offsets, t, y, th = small_batch("matern52", 19, lengths)
    rng = np.random.default_rng(4)
    miss = rng.random(len(y)) < 0.2
    miss[offsets[2] + 100:offsets[2] + 700] = True          # a long run
    miss[offsets[3]:offsets[4]] = True                       # nothing observed
    miss[offsets[9] + 1:offsets[10] - 1] = True              # only the ends observed
    y = y.copy()
    y[miss] = np.nan
    m = spingp.Model("matern52", chunk_len=L)
    bt = spingp.Batch(m, _t(offsets, torch.int64), _t(t), _t(y))
    ll, g = bt.grad(_t(th.reshape(-1)), missing=True)
    mean, var, llp = bt.posterior(_t(th.reshape(-1)), missing=True)
    check_series("matern52", offsets, t, y, th, ll.cpu().numpy(), g.cpu().numpy(), range(len(lengths)),
                 mean.cpu().numpy(), var.cpu().numpy())
    assert np.allclose(llp.cpu().numpy(), ll.cpu().numpy(), rtol=1e-12, atol=0)


def test_batched_matches_single_series_path():
    """A batch of one equals the single-series entry point (within FP64
    reduction-order rounding)."""
    s = synth.single("matern52_n4m", n=100000, seed=9)
    m = spingp.Model(s.spec)
    bt = spingp.Batch(m, _t([0, len(s.t)], torch.int64), _t(s.t), _t(s.y))
    llb, gb = bt.grad(_t(s.theta))
    lls, gs = m.grad(_t(s.t), _t(s.y), _t(s.theta))
    assert abs(float(llb[0]) - float(lls[0])) <= 1e-12 * abs(float(lls[0]))
    assert torch.allclose(gb[0], gs, rtol=1e-10, atol=0)


def test_batched_invalid_offsets():
    m = spingp.Model("matern32")
    t = _t(np.arange(10.0)); y = _t(np.zeros(10))
    th = _t(np.tile([1.0, 1.0, 0.1], 2))
    for bad in ([0, 6, 4], [1, 5, 10], [0, 5, 9]):
        bt = spingp.Batch(m, _t(bad, torch.int64), t, y)
        with pytest.raises(spingp.SpinGPError) as e:
            bt.grad(th)
        assert e.value.status == spingp.EINVAL


def test_batched_graph_capture():
    offsets, t, y, th = small_batch("matern52", 3, [500, 1200, 33, 4000])
    m = spingp.Model("matern52")
    bt = spingp.Batch(m, _t(offsets, torch.int64), _t(t), _t(y))
    TH = _t(th.reshape(-1))
    ll_ref, g_ref = bt.grad(TH)
    ll = torch.empty(4, dtype=torch.float64, device=DEV)
    g = torch.empty(12, dtype=torch.float64, device=DEV)
    stream = torch.cuda.Stream()
    stream.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(stream):
        bt.grad(TH, sync=False, out=(ll, g))
        graph = torch.cuda.CUDAGraph()
        with torch.cuda.graph(graph, stream=stream):
            bt.grad(TH, sync=False, out=(ll, g))
    torch.cuda.current_stream().wait_stream(stream)
    ll.zero_(); g.zero_()
    graph.replay()
    torch.cuda.synchronize()
    assert torch.equal(ll, ll_ref) and torch.equal(g.view(4, 3), g_ref)


def test_batched_full_config_sampled():
    """The batched workload at full size: 4096 Matern-5/2 series, lengths
    log-uniform in [256, 65536] (about 4.8e7 steps), per-series hyperparameters;
    48 series against the oracle -- the longest, the shortest, the ones with
    the smallest and largest lengthscale and 44 drawn at random -- and every
    series by the variance-scaling identity (a property that holds for each)."""
    s = synth.batched()
    offsets, th = s.extra["offsets"], s.extra["thetas"]
    m = spingp.Model("matern52")
    bt = spingp.Batch(m, _t(offsets, torch.int64), _t(s.t), _t(s.y))
    autotune.tune_batch(bt, _t(th.reshape(-1)), spingp.WS_GRAD)   # the benchmark's launch configuration
    ll, g = bt.grad(_t(th.reshape(-1)))
    ll, g = ll.cpu().numpy(), g.cpu().numpy()
    lens = np.diff(offsets)
    ends = [int(np.argmax(lens)), int(np.argmin(lens)), int(np.argmin(th[:, 0])), int(np.argmax(th[:, 0]))]
    rest = np.setdiff1d(np.arange(len(th)), ends)
    idx = np.concatenate([ends, np.random.default_rng(0).choice(rest, 48 - len(set(ends)), replace=False)])
    idx = np.unique(idx)
    assert len(idx) == 48 and lens[idx].max() == lens.max() and lens[idx].min() == lens.min()
    check_series("matern52", offsets, s.t, s.y, th, ll, g, idx)
    th2 = th.copy(); th2[:, 1:] *= 2.0
    ll2 = bt.loglik(_t(th2.reshape(-1))).cpu().numpy()
    n = np.diff(offsets).astype(np.float64)
    q = 4.0 * (ll2 - ll + 0.5 * n * np.log(2.0))
    lhs = th[:, 1] * g[:, 1] + th[:, 2] * g[:, 2]
    scale = np.abs(th[:, 1] * g[:, 1]) + np.abs(th[:, 2] * g[:, 2]) + n
    assert np.all(np.abs(lhs - (0.5 * q - 0.5 * n)) <= 1e-8 * scale)
