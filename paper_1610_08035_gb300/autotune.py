"""Chunk-length autotuner.

The chunk length L sets the split between sequential elimination inside a
chunk (one thread, L steps) and the odd-even reduction across chunks.  This
module times candidate lengths on the caller's own inputs and caches the
fastest per (device, state dimension, call kind, size bucket) in a JSON file
(``_tune/chunk.json`` beside this module, or $SPINGP_TUNE_CACHE).  Set
SPINGP_TUNE=0 to skip timing and use the library's built-in default.
"""
import json
import math
import os

import torch

from . import spingp

_HERE = os.path.dirname(os.path.abspath(__file__))
CANDIDATES = (16, 32, 64, 128, 256)
CHUNKS_PER_BLOCK = 128          # threads (chunks) per block of the chain kernels


def wave_candidates(n, sms):
    """Chunk lengths for which the chain kernels' block count is a whole
    multiple of the SM count (1..16 blocks per SM), so that no SM runs a
    partial last wave, plus the powers of two."""
    out = set(CANDIDATES)
    for per_sm in (1, 2, 3, 4, 5, 6, 8, 10, 12, 16):
        blocks = per_sm * sms
        L = -(-n // (blocks * CHUNKS_PER_BLOCK))
        if 8 <= L <= 4096:
            out.add(int(L))
    return sorted(out)


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


def tune(model, t, y, theta, what=spingp.WS_GRAD, candidates=None, reps=3):
    """Pick and set the fastest chunk length for this call kind and size.
    Returns the chosen length (0 = library default)."""
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
        sms = torch.cuda.get_device_properties(torch.cuda.current_device()).multi_processor_count
        candidates = wave_candidates(n, sms)
    best, best_ms = 0, float("inf")
    for L in candidates:
        if L * 4 > n and L != candidates[0]:
            continue
        model.set_chunk_len(L)
        call(t, y, theta, sync=True)          # allocates the workspace, warms up
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(reps):
            call(t, y, theta, sync=False)
        e1.record()
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / reps
        if ms < best_ms:
            best, best_ms = L, ms
    model.set_chunk_len(best)
    cache[key] = best
    try:
        _store(cache)
    except OSError:
        pass
    return best
