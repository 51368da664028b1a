"""Randomised parity of the chain path: seeded random series lengths, chunk
lengths, hyperparameters, time spacings (with ties and long gaps) and missing
observations, through every entry point that shares the chain kernels --
gradient, log-likelihood, posterior, the host-buffer call and one series split
in ranges -- against the oracle at the parity bars of test_gpu_parity, and
the host-buffer and split results against the device call."""
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
    ls, gs = 0.0, 0.0
    for r, (a, b) in enumerate(ranges):
        tp = None if r == 0 else float(t[a - 1])
        lr, gr = m.segment_grad(T[a:b], Y[a:b], TH, E, r, t_prev=tp, ws=wss[r], missing=miss)
        ls += lr.item()
        gs = gs + gr.cpu().numpy()
    assert abs(ls - llo) <= 1e-9 * abs(llo)
    assert np.all(np.abs(gs - go) <= 1e-8 * gscale)
