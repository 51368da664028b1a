"""The chunk-length autotuner (the sequential tile of the reduction, and with
it the split between in-chunk elimination and the tree levels): its
candidate lengths on the CPU, and on a GPU that tuning a single series, a
structured model and a batch picks one of them, caches it, and leaves the
results at the parity bars against the untuned call."""
import os
import types

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_1610_08035_gb300 import autotune  # noqa: E402


def test_wave_candidates_fill_whole_waves():
    n, sms = 1 << 22, 152
    c = autotune.wave_candidates(n, sms)
    assert list(c) == sorted(set(c)) and all(8 <= L <= 4096 for L in c)
    blocks = lambda L: -(-(-(-n // L)) // autotune.CHUNKS_PER_BLOCK)   # noqa: E731
    for per_sm in (1, 2, 4, 8, 16):
        # the shortest length whose blocks fit in per_sm waves is a candidate
        L = min(L for L in range(8, 4097) if blocks(L) <= per_sm * sms)
        assert L in c and blocks(L - 1) > per_sm * sms, (per_sm, L)
    g = autotune.wave_candidates(1 << 20, sms, autotune.GROUP_CHUNKS_PER_BLOCK, autotune.GROUP_CANDIDATES, lo=4)
    assert 432 in g          # two 8-group blocks per SM at N = 2^20
    assert set(autotune.GROUP_CANDIDATES) <= set(g)


def test_batch_candidates_count_every_series_chunks():
    lens = np.array([256, 70000, 1000, 0, 3])
    sms = 4
    c = autotune.batch_candidates(lens, sms, per_block=2)
    chunks = lambda L: int(np.sum(-(-lens[lens > 0] // L)))   # noqa: E731
    checked = 0
    for per_sm in (1, 2, 4, 8, 16):
        cap = per_sm * sms * 2
        fits = [L for L in range(8, 4097) if chunks(L) <= cap]
        if fits:                       # (at 1 and 2 per SM no length fits the 70000-step series)
            assert min(fits) in c
            checked += 1
    assert checked >= 3


def test_group_path_detection():
    m = lambda spec, b: types.SimpleNamespace(spec=spec, state_dim=b)   # noqa: E731
    assert not autotune._on_group_path(m("matern52", 3))
    assert not autotune._on_group_path(m(["matern32"], 2))
    assert autotune._on_group_path(m(["matern32", "matern32"], 4))
    assert autotune._on_group_path(m([("eq", 10)], 10))
    assert autotune._on_group_path(m([("periodic", 2)], 6))


@pytest.mark.gpu
@pytest.mark.parametrize("spec,theta,n", [("matern52", [0.5, 2.0, 0.05], 200000),
                                          (["matern32", ("eq", 6)], [1.0, 0.6, 0.7, 1.2, 0.05], 30000)])
def test_tune_single_series(tmp_path, monkeypatch, spec, theta, n):
    from oracle import seq
    from paper_1610_08035_gb300 import spingp, synth
    monkeypatch.setenv("SPINGP_TUNE_CACHE", str(tmp_path / "chunk.json"))
    rng = np.random.default_rng(1)
    t = synth.exp_times(n, 0.01, rng)
    y = synth.two_sinusoids(t, 0.7, 1.0, 0.05, rng)
    T, Y, TH = (torch.tensor(np.asarray(a, dtype=np.float64), device="cuda") for a in (t, y, theta))
    m = spingp.Model(spec)
    L = autotune.tune(m, T, Y, TH, spingp.WS_GRAD)
    assert L == 0 or (L in autotune._candidates(m, n) and m.chunk_len(n) == L)
    assert os.path.exists(tmp_path / "chunk.json")
    m2 = spingp.Model(spec)
    assert autotune.tune(m2, T, Y, TH, spingp.WS_GRAD) == L          # from the cache
    ll, g = m.grad(T, Y, TH)
    llo, go, g1 = seq.grad(spec, theta, t, y, l1=True)
    assert abs(ll.item() - llo) <= 1e-9 * abs(llo)
    assert np.all(np.abs(g.cpu().numpy() - go) <= 1e-8 * np.maximum(np.abs(go), g1))


@pytest.mark.gpu
def test_tune_batch(tmp_path, monkeypatch):
    from oracle import seq
    from paper_1610_08035_gb300 import spingp, synth
    monkeypatch.setenv("SPINGP_TUNE_CACHE", str(tmp_path / "chunk.json"))
    s = synth.batched(n_series=96)
    off, th = s.extra["offsets"], s.extra["thetas"]
    dev = "cuda"
    bt = spingp.Batch(spingp.Model("matern52"), torch.tensor(off, device=dev), torch.tensor(s.t, device=dev),
                      torch.tensor(s.y, device=dev))
    TH = torch.tensor(th.reshape(-1), device=dev)
    L = autotune.tune_batch(bt, TH, spingp.WS_GRAD)
    mean_len = len(s.t) // 96
    assert L == 0 or 2 * L <= mean_len
    ll, g = bt.grad(TH)
    ll, g = ll.cpu().numpy(), g.cpu().numpy()
    for i in (0, int(np.argmax(np.diff(off))), int(np.argmin(np.diff(off)))):
        a, b = off[i], off[i + 1]
        llo, go, g1 = seq.grad("matern52", th[i], s.t[a:b], s.y[a:b], l1=True)
        assert abs(ll[i] - llo) <= 1e-9 * abs(llo)
        assert np.all(np.abs(g[i] - go) <= 1e-8 * np.maximum(np.abs(go), g1))
