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
