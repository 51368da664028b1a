"""The multi-rank path on CPU: world_size-2 gloo process groups.

A batch of independent series is sharded across ranks (no exchange on the
data path); each rank computes its series' log-likelihoods and gradients
(here with the oracle, since there is no GPU) and the per-series rows are
gathered.  The gathered table must equal the unsharded computation exactly,
and the shards must cover every series once with balanced work."""
import os
import socket

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

from paper_1610_08035_gb300 import shard, synth


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _batch():
    return synth.batched(n_series=24, lo=50, hi=2000, seed=17)


def _worker(rank, world, port, out_path):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        from oracle import seq
        s = _batch()
        offsets, thetas = s.extra["offsets"], s.extra["thetas"]
        n_series = len(thetas)
        parts = shard.lpt_shard(np.diff(offsets), world)
        mine = parts[rank]
        loc, t, y, th = shard.local_batch(offsets, s.t, s.y, thetas, mine)
        rows = []
        for i in range(len(mine)):
            ll, g = seq.grad("matern52", th[i], t[loc[i]:loc[i + 1]], y[loc[i]:loc[i + 1]])
            rows.append(np.concatenate([[ll], g]))
        vals = torch.tensor(np.array(rows).reshape(len(mine), 4), dtype=torch.float64)
        full = shard.gather_per_series(vals, mine, n_series)
        if rank == 0:
            np.save(out_path, full.numpy())
        dist.barrier()
    finally:
        dist.destroy_process_group()


def test_lpt_shard_covers_and_balances():
    lengths = np.random.default_rng(0).integers(1, 65536, 4096)
    for world in (1, 2, 3, 8):
        parts = shard.lpt_shard(lengths, world)
        allidx = np.sort(np.concatenate(parts))
        assert np.array_equal(allidx, np.arange(len(lengths)))
        loads = np.array([lengths[p].sum() for p in parts])
        assert loads.max() - loads.min() <= lengths.max()


def test_local_batch_slices():
    s = _batch()
    offsets = s.extra["offsets"]
    series = np.array([3, 0, 7])
    loc, t, y, th = shard.local_batch(offsets, s.t, s.y, s.extra["thetas"], series)
    for k, i in enumerate(series):
        assert np.array_equal(t[loc[k]:loc[k + 1]], s.t[offsets[i]:offsets[i + 1]])
        assert np.array_equal(th[k], s.extra["thetas"][i])


def test_two_ranks_reproduce_the_unsharded_batch(tmp_path):
    out = str(tmp_path / "gathered.npy")
    world = 2
    mp.start_processes(_worker, args=(world, _free_port(), out), nprocs=world, start_method="spawn", join=True)
    full = np.load(out)
    from oracle import seq
    s = _batch()
    offsets, thetas = s.extra["offsets"], s.extra["thetas"]
    for i in range(len(thetas)):
        ll, g = seq.grad("matern52", thetas[i], s.t[offsets[i]:offsets[i + 1]], s.y[offsets[i]:offsets[i + 1]])
        assert np.array_equal(full[i], np.concatenate([[ll], g]))


# ---- one series split across ranks (the exchange of shard.grad_split_series)

class _OracleRange:
    """A stand-in for spingp.Model's two phases on CPU ranks.  Its 'element'
    carries the range's raw data (count, t, y, padded to a fixed size), so after
    the all-gather each rank sees the series up to its range; its share is then
    the prediction-error terms of its own steps, ll(y_<=b) - ll(y_<a), and the
    same difference of gradients (oracle).  The shares telescope to the whole
    series' values only if the exchange delivers every rank's element in rank
    order and the all-reduce sums every share once."""
    cap = 600

    def __init__(self, spec):
        self.spec = spec

    def segment_reduce(self, t, y, theta, t_prev=None, missing=False, sync=True):
        e = torch.zeros(1 + 2 * self.cap, dtype=torch.float64)
        n = t.numel()
        e[0] = n
        e[1:1 + n] = t
        e[1 + self.cap:1 + self.cap + n] = y
        if t_prev is not None:
            assert t_prev <= float(t[0])
        return e

    def segment_grad(self, t, y, theta, elems, rank, t_prev=None, missing=False, sync=True):
        from oracle import seq
        ts, ys = [], []
        for e in elems[:rank + 1]:
            n = int(e[0])
            ts.append(e[1:1 + n].numpy())
            ys.append(e[1 + self.cap:1 + self.cap + n].numpy())
        assert np.array_equal(ts[-1], t.numpy()) and np.array_equal(ys[-1], y.numpy())
        tall, yall = np.concatenate(ts), np.concatenate(ys)
        a = len(tall) - t.numel()
        th = theta.numpy()
        ll1, g1 = seq.grad(self.spec, th, tall, yall)
        ll0, g0 = seq.grad(self.spec, th, tall[:a], yall[:a]) if a > 0 else (0.0, np.zeros_like(g1))
        return (torch.tensor([ll1 - ll0], dtype=torch.float64),
                torch.tensor(g1 - g0, dtype=torch.float64))

    def segment_grad_posterior(self, t, y, theta, elems, rank, t_prev=None, missing=False, sync=True):
        """The share above plus the posterior at this range's steps, from the
        smoother over every rank's data: right only if the exchange brings
        the later ranks' elements too."""
        from oracle import seq
        ll, g = self.segment_grad(t, y, theta, elems, rank, t_prev=t_prev, missing=missing, sync=sync)
        ts, ys = [], []
        for e in elems:
            n = int(e[0])
            ts.append(e[1:1 + n].numpy())
            ys.append(e[1 + self.cap:1 + self.cap + n].numpy())
        a = sum(len(x) for x in ts[:rank])
        sm = seq.smoother(self.spec, theta.numpy(), np.concatenate(ts), np.concatenate(ys))
        b = a + t.numel()
        return ll, g, torch.from_numpy(sm["mean"][a:b].copy()), torch.from_numpy(sm["var"][a:b].copy())


def _split_worker(rank, world, port, out_path):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        rng = np.random.default_rng(23)
        n = 1000
        t = synth.exp_times(n, 0.05, rng)
        y = synth.two_sinusoids(t, 0.7, 1.0, 0.1, rng)
        theta = torch.tensor([0.7, 1.2, 0.1], dtype=torch.float64)
        a, b = shard.range_split(n, world)[rank]
        t_prev = None if rank == 0 else float(t[a - 1])
        ll, g = shard.grad_split_series(_OracleRange("matern32"), torch.from_numpy(t[a:b].copy()),
                                        torch.from_numpy(y[a:b].copy()), theta, t_prev)
        np.save(out_path + ".%d.npy" % rank, np.concatenate([ll.numpy(), g.numpy()]))
        dist.barrier()
    finally:
        dist.destroy_process_group()


def _split_posterior_worker(rank, world, port, out_path):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        rng = np.random.default_rng(29)
        n = 900
        t = synth.exp_times(n, 0.05, rng)
        y = synth.two_sinusoids(t, 0.7, 1.0, 0.1, rng)
        theta = torch.tensor([0.7, 1.2, 0.1], dtype=torch.float64)
        a, b = shard.range_split(n, world)[rank]
        t_prev = None if rank == 0 else float(t[a - 1])
        ll, g, mean, var = shard.grad_posterior_split_series(_OracleRange("matern32"), torch.from_numpy(t[a:b].copy()),
                                                             torch.from_numpy(y[a:b].copy()), theta, t_prev)
        np.save(out_path + ".%d.npy" % rank, np.concatenate([ll.numpy(), g.numpy(), mean.numpy(), var.numpy()]))
        dist.barrier()
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("world", [2, 3])
def test_split_series_posterior_exchange_on_gloo(tmp_path, world):
    """grad_posterior_split_series: every rank gets the whole series' (ll,
    grad) and the smoother's mean and variance on its own range."""
    from oracle import seq
    out = str(tmp_path / "splitpost")
    mp.spawn(_split_posterior_worker, args=(world, _free_port(), out), nprocs=world, join=True)
    rng = np.random.default_rng(29)
    n = 900
    t = synth.exp_times(n, 0.05, rng)
    y = synth.two_sinusoids(t, 0.7, 1.0, 0.1, rng)
    llo, go = seq.grad("matern32", [0.7, 1.2, 0.1], t, y)
    sm = seq.smoother("matern32", [0.7, 1.2, 0.1], t, y)
    for r, (a, b) in enumerate(shard.range_split(n, world)):
        got = np.load(out + ".%d.npy" % r)
        assert abs(got[0] - llo) <= 1e-10 * abs(llo)
        assert np.max(np.abs(got[1:4] - go) / np.abs(go)) <= 1e-9
        k = b - a
        assert np.array_equal(got[4:4 + k], sm["mean"][a:b]) and np.array_equal(got[4 + k:], sm["var"][a:b])


@pytest.mark.parametrize("world", [2, 3, 4])
def test_split_series_exchange_on_gloo(tmp_path, world):
    from oracle import seq
    out = str(tmp_path / "split")
    mp.spawn(_split_worker, args=(world, _free_port(), out), nprocs=world, join=True)
    rng = np.random.default_rng(23)
    t = synth.exp_times(1000, 0.05, rng)
    y = synth.two_sinusoids(t, 0.7, 1.0, 0.1, rng)
    llo, go = seq.grad("matern32", [0.7, 1.2, 0.1], t, y)
    for r in range(world):
        got = np.load(out + ".%d.npy" % r)
        assert abs(got[0] - llo) <= 1e-10 * abs(llo)
        assert np.max(np.abs(got[1:] - go) / np.abs(go)) <= 1e-9


def test_range_split():
    for n, world in ((10, 3), (1000, 7), (5, 5), (2 ** 22, 8)):
        rs = shard.range_split(n, world)
        assert rs[0][0] == 0 and rs[-1][1] == n
        assert all(rs[i][1] == rs[i + 1][0] for i in range(world - 1))
        sizes = [b - a for a, b in rs]
        assert min(sizes) >= 1 and max(sizes) - min(sizes) <= 1
    with pytest.raises(ValueError):
        shard.range_split(3, 4)
