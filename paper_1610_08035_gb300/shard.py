"""Sharding across ranks (one process per GPU).

A batch of series has no exchange step: each rank takes a subset of whole
series, runs the batched entry points on its own GPU, and only the per-series
results are gathered at the end.  Series are assigned by the longest-
processing-time rule (longest first, to the rank with the least work so far),
which keeps every rank within one longest series of the mean load.

One long series is cut into contiguous ranges, one per rank (Sec. 3.1's
reduction spans the ranks): every rank reduces its range to one element,
the elements are all-gathered, every rank finishes its range from them, and
the shares of the log-likelihood and gradient are all-reduced -- one
all-gather of G elements and one all-reduce of P + 1 numbers.  The element
algebra runs in the library (spingp_segment_reduce / spingp_segment_grad);
this module holds the range split and the exchange.

The exchange is host-side logic: the tests run it on CPU ranks with the gloo
backend, with a stand-in model.
"""
import heapq

import numpy as np
import torch
import torch.distributed as dist


def lpt_shard(lengths, world):
    """Assign series (given their lengths) to `world` ranks.  Returns one
    sorted int64 array of series indices per rank."""
    lengths = np.asarray(lengths, dtype=np.int64)
    heap = [(0, r) for r in range(world)]
    owner = np.empty(len(lengths), dtype=np.int64)
    for i in np.argsort(-lengths, kind="stable"):
        load, r = heapq.heappop(heap)
        owner[i] = r
        heapq.heappush(heap, (load + int(lengths[i]), r))
    return [np.flatnonzero(owner == r) for r in range(world)]


def local_batch(offsets, t, y, theta, series):
    """The concatenated inputs of the given series: (offsets, t, y, theta)
    with offsets starting at 0; theta has one row per series."""
    offsets = np.asarray(offsets, dtype=np.int64)
    lengths = offsets[series + 1] - offsets[series]
    loc = np.zeros(len(series) + 1, dtype=np.int64)
    loc[1:] = np.cumsum(lengths)
    idx = np.concatenate([np.arange(offsets[i], offsets[i + 1]) for i in series]) if len(series) else \
        np.empty(0, dtype=np.int64)
    return loc, np.asarray(t)[idx], np.asarray(y)[idx], np.asarray(theta)[series]


def gather_per_series(values, series, n_series, group=None):
    """Gather per-series rows (a 2-D float64 tensor, one row per local series)
    from every rank into the full (n_series, k) table, in series order, on
    every rank.  The only collective of the batched path."""
    world = dist.get_world_size(group)
    k = values.shape[1]
    counts = torch.tensor([len(series)], dtype=torch.int64)
    all_counts = [torch.zeros(1, dtype=torch.int64) for _ in range(world)]
    dist.all_gather(all_counts, counts, group=group)
    m = int(max(c.item() for c in all_counts))
    pad_v = torch.zeros(m, k, dtype=torch.float64, device=values.device)
    pad_v[:len(series)] = values
    pad_i = torch.full((m,), -1, dtype=torch.int64, device=values.device)
    pad_i[:len(series)] = torch.as_tensor(series, dtype=torch.int64, device=values.device)
    all_v = [torch.empty_like(pad_v) for _ in range(world)]
    all_i = [torch.empty_like(pad_i) for _ in range(world)]
    dist.all_gather(all_v, pad_v, group=group)
    dist.all_gather(all_i, pad_i, group=group)
    out = torch.zeros(n_series, k, dtype=torch.float64, device=values.device)
    for v, i in zip(all_v, all_i):
        keep = i >= 0
        out[i[keep]] = v[keep]
    return out


def range_split(n, world):
    """Contiguous ranges [a_r, b_r) of n steps for `world` ranks, as equal as
    whole steps allow (every rank gets at least one step: n >= world)."""
    if n < world:
        raise ValueError("fewer steps than ranks")
    edges = (np.arange(world + 1, dtype=np.int64) * n) // world
    return [(int(edges[r]), int(edges[r + 1])) for r in range(world)]


def grad_split_series(model, t, y, theta, t_prev, group=None, missing=False, sync=True):
    """Log-likelihood and gradient of one series split across the ranks of
    `group`: this rank holds the contiguous range t, y (device tensors) of
    the series, ranks in time order; t_prev is the time of the previous
    rank's last step (None on rank 0).  Every rank returns the whole series'
    (ll, grad).  `model` provides segment_reduce / segment_grad
    (spingp.Model does).  sync=False leaves the device status word to be
    read later (spingp_ws_status), with no host synchronisation."""
    world = dist.get_world_size(group)
    rank = dist.get_rank(group)
    if (t_prev is None) != (rank == 0):
        raise ValueError("t_prev must be None exactly on rank 0")
    elem = model.segment_reduce(t, y, theta, t_prev=t_prev, missing=missing, sync=sync)
    elems = [torch.empty_like(elem) for _ in range(world)]
    dist.all_gather(elems, elem, group=group)
    ll, g = model.segment_grad(t, y, theta, torch.stack(elems), rank, t_prev=t_prev, missing=missing, sync=sync)
    out = torch.cat([ll.reshape(1), g.reshape(-1)])
    dist.all_reduce(out, op=dist.ReduceOp.SUM, group=group)
    return out[:1], out[1:]


def grad_posterior_split_series(model, t, y, theta, t_prev, group=None, missing=False, sync=True):
    """grad_split_series plus the posterior at this rank's steps: returns
    (ll, grad) of the whole series (the same on every rank) and (mean, var)
    at this rank's range, conditioned on all ranks' observations.  The
    exchange is grad_split_series': one all-gather of the ranges' elements,
    one all-reduce of (ll, grad); the posterior needs nothing more, since
    every rank's element reaches every rank.  `model` provides
    segment_reduce / segment_grad_posterior (spingp.Model does)."""
    world = dist.get_world_size(group)
    rank = dist.get_rank(group)
    if (t_prev is None) != (rank == 0):
        raise ValueError("t_prev must be None exactly on rank 0")
    elem = model.segment_reduce(t, y, theta, t_prev=t_prev, missing=missing, sync=sync)
    elems = [torch.empty_like(elem) for _ in range(world)]
    dist.all_gather(elems, elem, group=group)
    ll, g, mean, var = model.segment_grad_posterior(t, y, theta, torch.stack(elems), rank, t_prev=t_prev,
                                                    missing=missing, sync=sync)
    out = torch.cat([ll.reshape(1), g.reshape(-1)])
    dist.all_reduce(out, op=dist.ReduceOp.SUM, group=group)
    return out[:1], out[1:], mean, var
