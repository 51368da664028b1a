"""GPU parity: the CUDA path through the C ABI against the oracle, element by
element, on seeded inputs.

Tolerances (FP64 on both sides):
  log-likelihood   |d ll|  <= 1e-9 |ll|
  posterior mean   |d m_i| <= 1e-8 max(|m_i|, sqrt(v_i))
  latent variance  |d v_i| <= 1e-8 v_i
  gradient         |d g_p| <= 1e-8 max(|g_p|, sum_i |g_p,i|)   (the L1 norm of the
                   per-step contributions guards against cancellation in the sum)
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from golden.make_golden import load_config1  # noqa: E402
from oracle import seq  # noqa: E402
from paper_1610_08035_gb300 import autotune, spingp, synth  # noqa: E402

pytestmark = pytest.mark.gpu
DEV = "cuda"


def _t(a):
    return torch.tensor(np.asarray(a, dtype=np.float64), device=DEV)


def gpu_all(spec, theta, t, y, L=0, posterior=True):
    m = spingp.Model(spec, chunk_len=L)
    T, Y, TH = _t(t), _t(y), _t(theta)
    ll, g = m.grad(T, Y, TH)
    out = dict(ll_grad=float(ll.cpu()[0]), grad=g.cpu().numpy(), ll=float(m.loglik(T, Y, TH).cpu()[0]))
    if posterior:
        mean, var, llp = m.posterior(T, Y, TH)
        out.update(mean=mean.cpu().numpy(), var=var.cpu().numpy(), ll_post=float(llp.cpu()[0]))
    return out


def check_against_oracle(spec, theta, t, y, L=0, posterior=True):
    r = gpu_all(spec, theta, t, y, L, posterior)
    if posterior:
        llo, go, mo, vo, g1 = seq.grad(spec, theta, t, y, posterior=True, l1=True)
    else:
        llo, go, g1 = seq.grad(spec, theta, t, y, l1=True)
    for key in ("ll", "ll_grad") + (("ll_post",) if posterior else ()):
        assert abs(r[key] - llo) <= 1e-9 * abs(llo), (key, r[key], llo)
    scale = np.maximum(np.abs(go), g1)
    assert np.all(np.abs(r["grad"] - go) <= 1e-8 * scale), (r["grad"], go, g1)
    if posterior:
        dm = np.abs(r["mean"] - mo)
        assert np.all(dm <= 1e-8 * np.maximum(np.abs(mo), np.sqrt(vo))), dm.max()
        dv = np.abs(r["var"] - vo)
        assert np.all(dv <= 1e-8 * vo), (dv / vo).max()
    return r


def series(n, mean_dt, seed, ell, sf, sn, ties=0, gaps=0):
    rng = np.random.default_rng(seed)
    d = rng.exponential(mean_dt, n)
    d[0] = 0.0
    if ties:
        d[::ties] = 0.0
    if gaps:
        d[gaps::gaps * 3 + 1] = 1e4 * mean_dt
    t = np.cumsum(d)
    y = synth.two_sinusoids(t, ell, sf, sn, rng)
    return t, y


MATERN = [("matern12", [0.7, 1.3, 0.1]), ("matern32", [1.0, 1.0, 0.1]), ("matern52", [0.5, 2.0, 0.05])]


def test_config1_golden():
    """Matern-3/2, N=1000 (the plain-method workload): loglik, posterior mean
    and variance, gradient against the stored oracle values."""
    g = load_config1()
    for L in (0, 8, 37):
        r = gpu_all(g["spec"], g["theta"], g["t"], g["y"], L)
        assert abs(r["ll"] - g["ll"]) <= 1e-9 * abs(g["ll"])
        assert np.all(np.abs(r["mean"] - g["mean"]) <= 1e-8 * np.maximum(np.abs(g["mean"]), np.sqrt(g["var"])))
        assert np.all(np.abs(r["var"] - g["var"]) <= 1e-8 * g["var"])
        assert np.all(np.abs(r["grad"] - g["grad"]) <= 1e-8 * np.maximum(1.0, np.abs(g["grad"])))


@pytest.mark.parametrize("spec,theta", MATERN)
@pytest.mark.parametrize("n,L", [(1, 0), (2, 8), (7, 8), (1000, 8), (1000, 64), (10007, 8), (5000, 512)])
def test_parity_sizes(spec, theta, n, L):
    """Single chunk, several chunks, two levels of the odd-even reduction
    (10007/8 -> 1251 chunks), ragged last chunks."""
    t, y = series(n, 0.05, n + L, theta[0], theta[1], theta[2])
    check_against_oracle(spec, theta, t, y, L)


@pytest.mark.parametrize("spec,theta", MATERN)
def test_parity_ties_and_large_gaps(spec, theta):
    """dt = 0 (tied times) every 5 steps and gaps of 1e4 x the mean."""
    t, y = series(20000, 0.01, 3, theta[0], theta[1], theta[2], ties=5, gaps=97)
    check_against_oracle(spec, theta, t, y, 16)


def test_parity_three_reduction_levels():
    """2^21 + 3 steps in chunks of 8: 262145 chunks, three levels of tiles."""
    spec, theta = "matern12", [0.3, 1.1, 0.2]
    t, y = series((1 << 21) + 3, 0.01, 5, theta[0], theta[1], theta[2])
    check_against_oracle(spec, theta, t, y, 8, posterior=True)


def test_parity_headline_full_size():
    """Matern-5/2, N = 2^22, dt ~ Exp(0.01), l=0.5, s_f=2, s_n=0.05, in the
    benchmark's launch configuration (the autotuned chunk length): loglik +
    gradient."""
    s = synth.single("matern52_n4m")
    m = spingp.Model(s.spec)
    L = autotune.tune(m, _t(s.t), _t(s.y), _t(s.theta), spingp.WS_GRAD) or m.chunk_len(len(s.t))
    check_against_oracle(s.spec, s.theta, s.t, s.y, L, posterior=False)


@pytest.mark.parametrize("spec,theta", MATERN)
def test_variance_scaling_identity_on_gpu(spec, theta):
    """s_f dl/ds_f + s_n dl/ds_n = (y^T C^-1 y - N)/2, with y^T C^-1 y from
    l(2 s_f, 2 s_n) - l(s_f, s_n) = y^T C^-1 y / 4 - N/2 log 2: a property that
    holds at any size, checked on GPU outputs only."""
    t, y = series(300000, 0.01, 8, theta[0], theta[1], theta[2])
    m = spingp.Model(spec)
    T, Y = _t(t), _t(y)
    th = np.array(theta)
    ll, g = m.grad(T, Y, _t(th))
    th2 = th.copy(); th2[1] *= 2; th2[2] *= 2
    ll2 = m.loglik(T, Y, _t(th2))
    ll, ll2, g = float(ll.cpu()[0]), float(ll2.cpu()[0]), g.cpu().numpy()
    n = len(y)
    q = 4.0 * (ll2 - ll + 0.5 * n * np.log(2.0))
    lhs = th[1] * g[1] + th[2] * g[2]
    assert abs(lhs - (0.5 * q - 0.5 * n)) <= 1e-8 * (abs(th[1] * g[1]) + abs(th[2] * g[2]) + n)


def test_deterministic_and_consistent():
    """Repeated calls are bit-identical; the three entry points agree on ll."""
    s = synth.single("matern52_n4m", n=200000)
    a = gpu_all(s.spec, s.theta, s.t, s.y, 32)
    b = gpu_all(s.spec, s.theta, s.t, s.y, 32)
    assert a["ll"] == b["ll"] and np.array_equal(a["grad"], b["grad"])
    assert np.array_equal(a["mean"], b["mean"]) and np.array_equal(a["var"], b["var"])
    assert a["ll"] == a["ll_grad"] == a["ll_post"]


def test_autograd_function():
    s = synth.single("matern32_n1000")
    m = spingp.Model(s.spec)
    th = _t(s.theta).requires_grad_(True)
    ll = spingp.LogLik.apply(_t(s.t), _t(s.y), th, m)
    (2.0 * ll).backward()
    _, go = seq.grad(s.spec, s.theta, s.t, s.y)
    assert np.all(np.abs(th.grad.cpu().numpy() - 2.0 * go) <= 1e-8 * np.maximum(1.0, np.abs(2.0 * go)))


def test_graph_capture_replay():
    """The asynchronous call (no SYNC flag) launches kernels only and can be
    captured into a CUDA graph; replays reproduce the eager result."""
    s = synth.single("matern52_n4m", n=100000)
    m = spingp.Model(s.spec)
    T, Y, TH = _t(s.t), _t(s.y), _t(s.theta)
    ll_ref, g_ref = m.grad(T, Y, TH)
    ll = torch.empty(1, dtype=torch.float64, device=DEV)
    g = torch.empty(3, dtype=torch.float64, device=DEV)
    stream = torch.cuda.Stream()
    stream.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(stream):
        m.grad(T, Y, TH, sync=False, out=(ll, g))   # warm-up outside capture
        graph = torch.cuda.CUDAGraph()
        with torch.cuda.graph(graph, stream=stream):
            m.grad(T, Y, TH, sync=False, out=(ll, g))
    torch.cuda.current_stream().wait_stream(stream)
    ll.zero_(); g.zero_()
    graph.replay()
    torch.cuda.synchronize()
    assert torch.equal(ll, ll_ref) and torch.equal(g, g_ref)


def test_device_detected_errors():
    m = spingp.Model("matern32")
    t, y = series(1000, 0.05, 1, 1.0, 1.0, 0.1)
    th = np.array([1.0, 1.0, 0.1])
    bad_t = t.copy(); bad_t[500] = bad_t[499] - 1.0
    with pytest.raises(spingp.SpinGPError) as e:
        m.loglik(_t(bad_t), _t(y), _t(th))
    assert e.value.status == spingp.ENOTSORTED
    bad_y = y.copy(); bad_y[17] = np.nan
    with pytest.raises(spingp.SpinGPError) as e:
        m.grad(_t(t), _t(bad_y), _t(th))
    assert e.value.status == spingp.ENONFINITE
    with pytest.raises(spingp.SpinGPError) as e:
        m.loglik(_t(t), _t(y), _t([1.0, -1.0, 0.1]))
    assert e.value.status == spingp.EINVAL
    # the status word is cleared by the next call
    m.loglik(_t(t), _t(y), _t(th))


def test_workspace_too_small_is_rejected():
    m = spingp.Model("matern52")
    T, Y, TH = _t(np.arange(1000.0)), _t(np.zeros(1000)), _t([1.0, 1.0, 0.1])
    need = spingp.spingp_workspace_bytes(m.h, 1000, spingp.WS_GRAD)
    ws = torch.empty(need - 256, dtype=torch.uint8, device=DEV)
    ll = torch.empty(1, dtype=torch.float64, device=DEV)
    g = torch.empty(3, dtype=torch.float64, device=DEV)
    st = spingp.spingp_grad(m.h, T, Y, 1000, TH, ll, g, ws, ws.numel(), spingp.SYNC)
    assert st == spingp.EINVAL


def test_large_series_full_size():
    """Matern-3/2, N = 2^26, dt ~ Exp(0.001), l = 0.05 (the long-series
    workload) in the default launch configuration.  Checks: the log-likelihood
    and all three gradient entries against the oracle over the whole series
    (the L1-scaled gradient bar); the posterior mean and variance at 16
    sampled steps against the oracle on a window of +-20000 steps around each
    (400 lengthscales: the data outside the window changes the posterior at
    its centre by far less than FP64 resolution); and the variance-scaling
    identity for the gradient."""
    s = synth.single("matern32_n64m")
    m = spingp.Model(s.spec)
    T, Y, TH = _t(s.t), _t(s.y), _t(s.theta)
    autotune.tune(m, T, Y, TH, spingp.WS_GRAD)           # the benchmark's launch configuration
    ll, g = m.grad(T, Y, TH)
    ll, g = float(ll.cpu()[0]), g.cpu().numpy()
    llo, go, g1 = seq.grad(s.spec, s.theta, s.t, s.y, l1=True)
    assert abs(ll - llo) <= 1e-9 * abs(llo), (ll, llo)
    assert np.all(np.abs(g - go) <= 1e-8 * np.maximum(np.abs(go), g1)), (g, go, g1)
    mean, var, _ = m.posterior(T, Y, TH, with_loglik=False)
    mean, var = mean.cpu().numpy(), var.cpu().numpy()
    idx = np.random.default_rng(1).integers(20000, len(s.t) - 20000, 16)
    for i in idx:
        a, b = i - 20000, i + 20001
        sm = seq.smoother(s.spec, s.theta, s.t[a:b], s.y[a:b])
        mo, vo = sm["mean"][20000], sm["var"][20000]
        assert abs(mean[i] - mo) <= 1e-8 * max(abs(mo), np.sqrt(vo)), (i, mean[i], mo)
        assert abs(var[i] - vo) <= 1e-8 * vo, (i, var[i], vo)
    th2 = s.theta.copy(); th2[1] *= 2; th2[2] *= 2
    ll2 = float(m.loglik(T, Y, _t(th2)).cpu()[0])
    n = len(s.t)
    q = 4.0 * (ll2 - ll + 0.5 * n * np.log(2.0))
    lhs = s.theta[1] * g[1] + s.theta[2] * g[2]
    assert abs(lhs - (0.5 * q - 0.5 * n)) <= 1e-8 * (abs(s.theta[1] * g[1]) + abs(s.theta[2] * g[2]) + n)


def test_large_series_step_in_a_captured_graph():
    """The long-series workload's step (N = 2^26: log-likelihood, gradient
    and posterior mean) captured once into a CUDA graph and replayed, as two
    calls and as the fused call: each replay writes the same bits as its
    eager calls."""
    s = synth.single("matern32_n64m")
    n = len(s.t)
    m = spingp.Model(s.spec)
    T, Y, TH = _t(s.t), _t(s.y), _t(s.theta)
    autotune.tune(m, T, Y, TH, spingp.WS_GRAD)
    ll_e, g_e = m.grad(T, Y, TH)
    mean_e, var_e, _ = m.posterior(T, Y, TH, with_loglik=False)
    ll = torch.empty(1, dtype=torch.float64, device=DEV)
    g = torch.empty(3, dtype=torch.float64, device=DEV)
    mean = torch.empty(n, dtype=torch.float64, device=DEV)
    var = torch.empty(n, dtype=torch.float64, device=DEV)
    stream = torch.cuda.Stream()
    stream.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(stream):
        graph = torch.cuda.CUDAGraph()
        with torch.cuda.graph(graph, stream=stream):
            m.grad(T, Y, TH, sync=False, out=(ll, g))
            m.posterior(T, Y, TH, sync=False, with_loglik=False, out=(mean, var, None))
    torch.cuda.current_stream().wait_stream(stream)
    for _ in range(2):
        ll.fill_(float("nan")); g.fill_(float("nan")); mean.fill_(float("nan"))
        graph.replay()
        torch.cuda.synchronize()
        assert torch.equal(ll, ll_e) and torch.equal(g, g_e)
        assert torch.equal(mean, mean_e) and torch.equal(var, var_e)
    assert spingp.spingp_ws_status(m.workspace(n, spingp.WS_GRAD, DEV)) == spingp.OK
    assert spingp.spingp_ws_status(m.workspace(n, spingp.WS_POSTERIOR, DEV)) == spingp.OK
    # the same step through the fused call (the benchmark's graph): its replay
    # writes the eager fused call's bits; the log-likelihood is the gradient
    # call's, the other outputs the separate calls' up to rounding order
    fused = m.grad_posterior(T, Y, TH)
    assert torch.equal(fused[0], ll_e)
    gs = np.maximum(1.0, np.abs(g_e.cpu().numpy()))
    assert np.all(np.abs(fused[1].cpu().numpy() - g_e.cpu().numpy()) <= 1e-11 * gs)
    vmax = float(var_e.max())
    scale = max(float(mean_e.abs().max()), np.sqrt(vmax))
    assert float((fused[2] - mean_e).abs().max()) <= 1e-13 * scale
    assert float((fused[3] - var_e).abs().max()) <= 1e-13 * vmax
    out = (ll, g, mean, var, None)
    with torch.cuda.stream(stream):
        graph2 = torch.cuda.CUDAGraph()
        with torch.cuda.graph(graph2, stream=stream):
            m.grad_posterior(T, Y, TH, sync=False, out=out)
    torch.cuda.current_stream().wait_stream(stream)
    ll.fill_(float("nan")); g.fill_(float("nan")); mean.fill_(float("nan")); var.fill_(float("nan"))
    graph2.replay()
    torch.cuda.synchronize()
    for a, b in zip(fused[:4], out[:4]):
        assert torch.equal(a, b)


@pytest.mark.parametrize("spec", [["matern52"], ["matern32", ("quasiperiodic", 3, "matern12")]])
def test_log_gradient_and_predictive_variance_flags(spec):
    """SPINGP_LOG_GRAD returns theta * d ll / d theta (readings R11) and
    SPINGP_PREDICTIVE adds the noise variance to the latent variances (R8),
    for the single-series, batched, host-buffer and split calls."""
    theta = [0.5, 2.0, 0.05] if spec == ["matern52"] else [1.0, 1.0, 1.0, 1.0, 1.0, 5.0, 0.05]
    n = 3001
    rng = np.random.default_rng(17)
    t = np.cumsum(rng.exponential(0.01, n))
    y = np.sin(3 * t) + 0.2 * rng.standard_normal(n)
    m = spingp.Model(spec)
    T, Y, TH = _t(t), _t(y), _t(theta)
    ll, g = m.grad(T, Y, TH)
    ll2, g2 = m.grad(T, Y, TH, log_params=True)
    assert ll2.item() == ll.item()
    assert torch.equal(g2, g * TH)
    llh, gh = m.grad_host(torch.from_numpy(t).pin_memory(), torch.from_numpy(y).pin_memory(),
                          torch.tensor(theta, dtype=torch.float64), log_params=True)
    assert torch.equal(gh, (g * TH).cpu())
    mean, var, _ = m.posterior(T, Y, TH)
    mean2, var2, _ = m.posterior(T, Y, TH, predictive=True)
    assert torch.equal(mean2, mean)
    assert torch.equal(var2, var + TH[-1])
    # split in two ranges: the shares of the log-gradient sum to the whole
    h = n // 2
    e0 = m.segment_reduce(T[:h], Y[:h], TH)
    ws1 = torch.empty(spingp.spingp_workspace_bytes(m.h, n - h, spingp.WS_GRAD), dtype=torch.uint8, device=DEV)
    e1 = m.segment_reduce(T[h:], Y[h:], TH, t_prev=float(t[h - 1]), ws=ws1)
    E = torch.stack([e0, e1])
    _, s0 = m.segment_grad(T[:h], Y[:h], TH, E, 0, log_params=True)
    _, s1 = m.segment_grad(T[h:], Y[h:], TH, E, 1, t_prev=float(t[h - 1]), ws=ws1, log_params=True)
    assert torch.allclose(s0 + s1, g * TH, rtol=1e-10, atol=0.0)
    if spec == ["matern52"]:
        off = torch.tensor([0, 1000, 1000, n], dtype=torch.int64, device=DEV)
        b = spingp.Batch(m, off, T, Y)
        ths = torch.tensor([theta, [0.7, 1.0, 0.1], theta], dtype=torch.float64, device=DEV)
        _, gb = b.grad(ths)
        _, gb2 = b.grad(ths, log_params=True)
        assert torch.equal(gb2, gb * ths)
        _, vb, _ = b.posterior(ths)
        _, vb2, _ = b.posterior(ths, predictive=True)
        noise = torch.cat([torch.full((1000,), theta[2], dtype=torch.float64, device=DEV),
                           torch.full((n - 1000,), theta[2], dtype=torch.float64, device=DEV)])
        assert torch.equal(vb2, vb + noise)
