"""Randomised parity, seeded:
- the chain path: random series lengths, chunk lengths, hyperparameters,
  time spacings (with ties and long gaps) and missing observations, through
  every entry point that shares the chain kernels -- gradient,
  log-likelihood, posterior, the fused gradient + posterior call, the
  host-buffer call and one series split in ranges (with the split
  posterior in every other case) -- against the oracle at the parity bars
  of test_gpu_parity, and the host-buffer result against the device call
  bit for bit;
- the group path: random sums of Matern-3/2, periodic, quasi-periodic and
  order-4 to 8 EQ components (b <= 16) against the oracle, whole (also
  through the fused call) and split in ranges (with the split posterior in
  every other case);
- the general BTD solver: random SPD systems of every size against the
  oracle's block LDL^T."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import seq  # noqa: E402
from paper_1610_08035_gb300 import shard, spingp, synth  # noqa: E402

pytestmark = pytest.mark.gpu
DEV = "cuda"
SPECS = ["matern12", "matern32", "matern52"]


def _t(a):
    return torch.tensor(np.asarray(a, dtype=np.float64), device=DEV)


def _case(k):
    rng = np.random.default_rng(1000 + k)
    spec = SPECS[k % 3]
    n = int(np.exp(rng.uniform(0.0, np.log(30000))))
    L = int(rng.choice([0, 8, 9, 16, 33, 100, 257, 512]))
    ell = float(np.exp(rng.uniform(np.log(0.05), np.log(5.0))))
    theta = [ell, float(np.exp(rng.uniform(np.log(0.3), np.log(3.0)))),
             float(np.exp(rng.uniform(np.log(0.01), np.log(0.5))))]
    d = rng.exponential(float(np.exp(rng.uniform(np.log(1e-3), np.log(0.3)))) * ell, n)
    d[0] = 0.0
    d[rng.random(n) < 0.02] = 0.0                 # ties
    d[rng.random(n) < 0.002] *= 1e3               # long gaps
    t = np.cumsum(d) + float(rng.uniform(-5.0, 5.0))
    y = synth.two_sinusoids(t, ell, theta[1], theta[2], rng)
    miss = rng.random() < 0.4
    if miss:
        y[rng.random(n) < rng.uniform(0.0, 0.3)] = np.nan
        if np.all(np.isnan(y)):
            y[0] = 0.1
    return spec, theta, t, y, L, miss


def _check_posterior(mean, var, mo, vo):
    assert np.all(np.abs(mean - mo) <= 1e-8 * np.maximum(np.abs(mo), np.sqrt(vo)))
    assert np.all(np.abs(var - vo) <= 1e-8 * vo)


def _check_fused(m, T, Y, TH, miss, ll, llo, go, gscale, mo, vo):
    """spingp_grad_posterior: the gradient call's log-likelihood bit for bit,
    the gradient, mean and variance at the parity bars."""
    llf, gf, mf, vf, _ = m.grad_posterior(T, Y, TH, missing=miss)
    assert llf.item() == ll.item()
    assert np.all(np.abs(gf.cpu().numpy() - go) <= 1e-8 * gscale)
    _check_posterior(mf.cpu().numpy(), vf.cpu().numpy(), mo, vo)


def _split_phase2(m, T, Y, TH, E, ranges, t, wss, miss, posterior, mo, vo):
    """Phase 2 of the split series, rank by rank: the summed shares of
    (ll, grad); with posterior, spingp_segment_grad_posterior, whose mean and
    variance at every range's steps are checked against the oracle too."""
    ls, gs, means, vars_ = 0.0, 0.0, [], []
    for r, (a, b) in enumerate(ranges):
        tp = None if r == 0 else float(t[a - 1])
        if posterior:
            lr, gr, mr, vr = m.segment_grad_posterior(T[a:b], Y[a:b], TH, E, r, t_prev=tp, ws=wss[r], missing=miss)
            means.append(mr.cpu().numpy())
            vars_.append(vr.cpu().numpy())
        else:
            lr, gr = m.segment_grad(T[a:b], Y[a:b], TH, E, r, t_prev=tp, ws=wss[r], missing=miss)
        ls += lr.item()
        gs = gs + gr.cpu().numpy()
    if posterior:
        _check_posterior(np.concatenate(means), np.concatenate(vars_), mo, vo)
    return ls, gs


@pytest.mark.parametrize("k", range(64))
def test_fuzz_chain_against_oracle(k):
    spec, theta, t, y, L, miss = _case(k)
    m = spingp.Model(spec, chunk_len=L)
    T, Y, TH = _t(t), _t(y), _t(theta)
    ll, g = m.grad(T, Y, TH, missing=miss)
    ll_l = m.loglik(T, Y, TH, missing=miss)
    mean, var, ll_p = m.posterior(T, Y, TH, missing=miss)
    llo, go, mo, vo, g1 = seq.grad([spec], theta, t, y, posterior=True, l1=True)
    for v in (ll.item(), ll_l.item(), ll_p.item()):
        assert abs(v - llo) <= 1e-9 * abs(llo), (v, llo)
    gscale = np.maximum(np.maximum(np.abs(go), g1), 1e-12)
    assert np.all(np.abs(g.cpu().numpy() - go) <= 1e-8 * gscale)
    mg, vg = mean.cpu().numpy(), var.cpu().numpy()
    assert np.all(np.abs(mg - mo) <= 1e-8 * np.maximum(np.abs(mo), np.sqrt(vo)))
    assert np.all(np.abs(vg - vo) <= 1e-8 * vo)
    # the fused gradient + posterior call: the gradient call's log-likelihood
    # bit for bit, every output at the parity bars
    _check_fused(m, T, Y, TH, miss, ll, llo, go, gscale, mo, vo)
    # the host-buffer call: the device call's bits
    ll_h, g_h = m.grad_host(torch.from_numpy(t).pin_memory(), torch.from_numpy(y).pin_memory(),
                            torch.tensor(theta, dtype=torch.float64), missing=miss)
    assert ll_h.item() == ll.item() and torch.equal(g_h, g.cpu())
    # the series split in ranges (ranks emulated in turn on this GPU)
    G = min(len(t), 1 + k % 5)
    ranges = shard.range_split(len(t), G)
    wss, elems = [], []
    for r, (a, b) in enumerate(ranges):
        ws = torch.empty(spingp.spingp_workspace_bytes(m.h, b - a, spingp.WS_GRAD), dtype=torch.uint8, device=DEV)
        tp = None if r == 0 else float(t[a - 1])
        elems.append(m.segment_reduce(T[a:b], Y[a:b], TH, t_prev=tp, ws=ws, missing=miss))
        wss.append(ws)
    E = torch.stack(elems)
    ls, gs = _split_phase2(m, T, Y, TH, E, ranges, t, wss, miss, k % 2 == 1, mo, vo)
    assert abs(ls - llo) <= 1e-9 * abs(llo)
    assert np.all(np.abs(gs - go) <= 1e-8 * gscale)


# ---- the group path (structured b <= 16) and the general BTD solver

def _group_case(k):
    rng = np.random.default_rng(2000 + k)
    comps, theta = [], []
    b = 0
    for _ in range(int(rng.integers(1, 4))):
        kind = int(rng.integers(0, 4))
        if kind == 0 and b + 2 <= 16:
            comps.append("matern32"); theta += [float(np.exp(rng.uniform(-1.5, 1.0))), float(np.exp(rng.uniform(-1, 1)))]
            b += 2
        elif kind == 1 and b + 4 <= 16:
            J = int(rng.integers(1, 4))
            if b + 2 * (J + 1) > 16:
                continue
            comps.append(("periodic", J))
            theta += [float(np.exp(rng.uniform(-1, 1))), float(np.exp(rng.uniform(-0.5, 0.7))),
                      float(np.exp(rng.uniform(-0.5, 1.0)))]
            b += 2 * (J + 1)
        elif kind == 2:
            J = int(rng.integers(1, 4))
            if b + 2 * (J + 1) > 16:
                continue
            comps.append(("quasiperiodic", J, "matern12"))
            theta += [float(np.exp(rng.uniform(-1, 1))), float(np.exp(rng.uniform(-0.5, 0.7))),
                      float(np.exp(rng.uniform(-0.5, 1.0))), float(np.exp(rng.uniform(0.0, 2.0)))]
            b += 2 * (J + 1)
        elif kind == 3 and b + 4 <= 16 and not any(isinstance(c, tuple) and c[0] == "eq" for c in comps):
            N = int(rng.choice([4, 6, 8]))
            if b + N > 16:
                N = 4
            comps.append(("eq", N)); theta += [float(np.exp(rng.uniform(-1, 1))), float(np.exp(rng.uniform(-1, 1)))]
            b += N
    if not comps:
        comps, theta = ["matern32"], [1.0, 1.0]
    theta.append(float(np.exp(rng.uniform(np.log(0.01), np.log(0.3)))))
    n = int(np.exp(rng.uniform(0.0, np.log(6000))))
    d = rng.exponential(float(np.exp(rng.uniform(np.log(0.005), np.log(0.1)))), n)
    d[0] = 0.0
    d[rng.random(n) < 0.02] = 0.0
    t = np.cumsum(d)
    y = synth.two_sinusoids(t, 0.8, 1.0, 0.1, rng)
    if k % 3 == 1:                       # every third case with missing observations
        y[rng.random(n) < 0.1] = np.nan
    L = int(rng.choice([0, 8, 33, 200]))
    return comps, theta, t, y, L


@pytest.mark.parametrize("k", range(24))
def test_fuzz_group_against_oracle(k):
    """Random structured models (with missing observations in every third
    case) through the gradient, the posterior with its lag-one covariances,
    and the series split in ranges."""
    spec, theta, t, y, L = _group_case(k)
    miss = bool(np.isnan(y).any())
    m = spingp.Model(spec, chunk_len=L)
    assert m.num_params == len(theta)
    T, Y, TH = _t(t), _t(y), _t(theta)
    ll, g = m.grad(T, Y, TH, missing=miss)
    mean, var, lag, ll_p = m.posterior_lag1(T, Y, TH, missing=miss)
    llo, go, mo, vo, g1 = seq.grad(spec, theta, t, y, posterior=True, l1=True)
    if len(t) > 1:
        sm = seq.smoother(spec, theta, t, y, blocks=True)
        h = seq.continuous(spec, theta)[2]
        co = np.einsum("i,nij,j->n", h, sm["Pc"], h)
        assert np.all(np.abs(lag.cpu().numpy() - co) <= 1e-8 * np.sqrt(vo[1:] * vo[:-1]))
    assert abs(ll.item() - llo) <= 1e-9 * abs(llo), (spec, ll.item(), llo)
    assert abs(ll_p.item() - llo) <= 1e-9 * abs(llo)
    gscale = np.maximum(np.maximum(np.abs(go), g1), 1e-12)
    assert np.all(np.abs(g.cpu().numpy() - go) <= 1e-8 * gscale), (spec, g.cpu().numpy(), go)
    assert np.all(np.abs(mean.cpu().numpy() - mo) <= 1e-8 * np.maximum(np.abs(mo), np.sqrt(vo)))
    assert np.all(np.abs(var.cpu().numpy() - vo) <= 1e-8 * vo)
    _check_fused(m, T, Y, TH, miss, ll, llo, go, gscale, mo, vo)
    # the series split in ranges
    G = min(len(t), 1 + k % 4)
    ranges = shard.range_split(len(t), G)
    wss, elems = [], []
    for r, (a, b) in enumerate(ranges):
        ws = torch.empty(spingp.spingp_workspace_bytes(m.h, b - a, spingp.WS_GRAD), dtype=torch.uint8, device=DEV)
        tp = None if r == 0 else float(t[a - 1])
        elems.append(m.segment_reduce(T[a:b], Y[a:b], TH, t_prev=tp, ws=ws, missing=miss))
        wss.append(ws)
    E = torch.stack(elems)
    ls, gs = _split_phase2(m, T, Y, TH, E, ranges, t, wss, miss, k % 2 == 0, mo, vo)
    assert abs(ls - llo) <= 1e-9 * abs(llo)
    assert np.all(np.abs(gs - go) <= 1e-8 * gscale), (spec, G, gs, go)


@pytest.mark.parametrize("k", range(24))
def test_fuzz_btd_solver(k):
    """Random SPD block-tridiagonal systems: every level size from 1 up, on
    both the one-thread and the lane-group levels."""
    from oracle import btd
    rng = np.random.default_rng(3000 + k)
    b = int(rng.integers(1, 4))
    n = int(np.exp(rng.uniform(0.0, np.log(20000))))
    D, O, r = synth.random_spd_btd(n, b, seed=4000 + k)
    ld, x, Sd, So = spingp.btd_solve(_t(D), _t(O), _t(r))
    lo, xo, Sdo, Soo = btd.thomas(D, O, r)
    assert abs(ld.item() - lo) <= 1e-11 * abs(lo)
    xs = np.max(np.abs(xo))
    assert np.max(np.abs(x.cpu().numpy() - xo)) <= 1e-10 * xs
    assert np.max(np.abs(Sd.cpu().numpy() - Sdo)) <= 1e-10 * np.max(np.abs(Sdo))
    if n > 1:
        assert np.max(np.abs(So.cpu().numpy() - Soo)) <= 1e-10 * np.max(np.abs(Sdo))
