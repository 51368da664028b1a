"""Chunk-length autotuner.

The chunk length L sets the split between sequential elimination inside a
chunk (one thread, or one 16-lane group on the structured path, L steps) and
the odd-even reduction across chunks: the in-block levels and the grid
levels.  This module times candidate lengths on the caller's own inputs
(one series with ``tune``, a batch of independent series with
``tune_batch``) and caches the fastest per (device, state dimension, call
kind, size bucket) in a JSON file (``_tune/chunk.json`` beside this module,
or $SPINGP_TUNE_CACHE).  Set SPINGP_TUNE=0 to skip timing and use the
library's built-in default.
"""
import json
import math
import os

import torch

from . import spingp

_HERE = os.path.dirname(os.path.abspath(__file__))
CANDIDATES = (16, 32, 64, 128, 256)
CHUNKS_PER_BLOCK = 128          # threads (chunks) per block of the chain kernels
GROUP_CHUNKS_PER_BLOCK = 8      # 16-lane groups (chunks) per block of the structured kernels
GROUP_CANDIDATES = (64, 128, 256, 512, 1024)


def wave_candidates(n, sms, per_block=CHUNKS_PER_BLOCK, base=CANDIDATES, lo=8):   # the library takes L >= 8
    """For 1..16 blocks per SM, the shortest chunk length whose block count
    fits in that many waves of the SM count (the last wave as full as a
    whole chunk length allows), plus the base lengths."""
    out = set(base)
    for per_sm in (1, 2, 3, 4, 5, 6, 8, 10, 12, 16):
        blocks = per_sm * sms
        L = -(-n // (blocks * per_block))
        if lo <= L <= 4096:
            out.add(int(L))
    return sorted(out)


def batch_candidates(lengths, sms, per_block=CHUNKS_PER_BLOCK, base=CANDIDATES, lo=8):
    """wave_candidates for a batch: its chunk count is the sum over series of
    ceil(n_i / L), so for 1..16 blocks per SM the shortest L whose chunks fit
    in that many waves is found by bisection on that sum."""
    import numpy as np
    lens = np.asarray(lengths, dtype=np.int64)
    lens = lens[lens > 0]
    chunks = lambda L: int(np.sum(-(-lens // L)))   # noqa: E731
    out = set(base)
    for per_sm in (1, 2, 3, 4, 5, 6, 8, 10, 12, 16):
        cap = per_sm * sms * per_block
        a, b = lo, 4096
        if chunks(b) > cap:
            continue
        while a < b:
            mid = (a + b) // 2
            if chunks(mid) <= cap:
                b = mid
            else:
                a = mid + 1
        out.add(int(a))
    return sorted(out)


def _on_group_path(model):
    """Structured models (several components, or b > 3) run on the 16-lane
    group kernels; a single Matern on the one-thread chain kernels."""
    spec = model.spec
    single = isinstance(spec, str) or (isinstance(spec, (list, tuple)) and len(spec) == 1 and isinstance(spec[0], str))
    return not (single and model.state_dim <= 3)


def _candidates(model, n):
    sms = torch.cuda.get_device_properties(torch.cuda.current_device()).multi_processor_count
    if _on_group_path(model):
        return wave_candidates(n, sms, GROUP_CHUNKS_PER_BLOCK, GROUP_CANDIDATES)
    return wave_candidates(n, sms)


def _cache_path():
    return os.environ.get("SPINGP_TUNE_CACHE", os.path.join(_HERE, "_tune", "chunk.json"))


def _key(model, n, what):
    p = torch.cuda.get_device_properties(torch.cuda.current_device())
    bucket = int(round(math.log2(max(n, 1))))
    return "%s/%d/b%d/%d/n2^%d" % (p.name, p.multi_processor_count, model.state_dim, what, bucket)


def _load():
    try:
        with open(_cache_path()) as f:
            return json.load(f)
    except (OSError, ValueError):
        return {}


def _store(cache):
    path = _cache_path()
    os.makedirs(os.path.dirname(path), exist_ok=True)
    tmp = path + ".%d.tmp" % os.getpid()
    with open(tmp, "w") as f:
        json.dump(cache, f, indent=1, sort_keys=True)
    os.replace(tmp, path)


def tune(model, t, y, theta, what=spingp.WS_GRAD, candidates=None, reps=5):
    """Pick and set the fastest chunk length for this call kind and size,
    the library's default among the candidates.  Returns the chosen length
    (0 = library default)."""
    if os.environ.get("SPINGP_TUNE", "1") == "0":
        model.set_chunk_len(0)
        return 0
    n = t.numel()
    key = _key(model, n, what)
    cache = _load()
    if key in cache:
        model.set_chunk_len(cache[key])
        return cache[key]
    call = {spingp.WS_GRAD: model.grad, spingp.WS_LOGLIK: model.loglik,
            spingp.WS_POSTERIOR: model.posterior}[what]
    if candidates is None:
        candidates = _candidates(model, n)
    # the library's default (0) always competes, so tuning never loses to it by more than the timing noise
    candidates = [0] + [L for L in candidates if L * 4 <= n or L == candidates[0]]
    best = _time_candidates(model, candidates, lambda: call(t, y, theta, sync=True),
                            lambda: call(t, y, theta, sync=False), reps)
    cache[key] = best
    try:
        _store(cache)
    except OSError:
        pass
    return best


def _time_candidates(model, candidates, warm, step, reps):
    """Set each candidate length, warm up once (the workspace is sized
    there), then time reps calls one by one with CUDA events, each after a
    write of 256 MiB that evicts the L2 (the inputs of a real call are not
    resident there); keep the length with the smallest median."""
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=torch.cuda.current_device())
    best, best_ms = 0, float("inf")
    for L in candidates:
        model.set_chunk_len(L)
        warm()
        times = []
        for r in range(reps):
            flush.fill_(r & 0xFF)
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record()
            step()
            e1.record()
            torch.cuda.synchronize()
            times.append(e0.elapsed_time(e1))
        ms = sorted(times)[len(times) // 2]
        if ms < best_ms:
            best, best_ms = L, ms
    model.set_chunk_len(best)
    del flush
    return best


def tune_batch(batch, theta, what=spingp.WS_GRAD, candidates=None, reps=5):
    """Pick and set the fastest chunk length for a batch of independent
    series (every series' chunks share it): the wave-aligned lengths of the
    whole batch, at most half the mean series length, timed on the batch's
    own call, against the library's default.  Returns the chosen length (0 =
    library default)."""
    model = batch.model
    if os.environ.get("SPINGP_TUNE", "1") == "0":
        model.set_chunk_len(0)
        return 0
    n, S = batch.n_total, batch.n_series
    mean_len = max(1, n // max(S, 1))
    p = torch.cuda.get_device_properties(torch.cuda.current_device())
    key = "%s/%d/b%d/%d/batch/n2^%d/mean2^%d" % (p.name, p.multi_processor_count, model.state_dim, what,
                                                 int(round(math.log2(max(n, 1)))),
                                                 int(round(math.log2(mean_len))))
    cache = _load()
    if key in cache:
        model.set_chunk_len(cache[key])
        return cache[key]
    call = {spingp.WS_GRAD: batch.grad, spingp.WS_LOGLIK: batch.loglik}[what]
    if candidates is None:
        sms = torch.cuda.get_device_properties(torch.cuda.current_device()).multi_processor_count
        lengths = (batch.offsets[1:] - batch.offsets[:-1]).cpu().numpy()
        candidates = batch_candidates(lengths, sms)
    candidates = [0] + [L for L in candidates if 2 * L <= mean_len]
    best = _time_candidates(model, candidates, lambda: call(theta, sync=True), lambda: call(theta, sync=False),
                            reps)
    cache[key] = best
    try:
        _store(cache)
    except OSError:
        pass
    return best
