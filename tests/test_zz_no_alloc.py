"""spingp_loglik_noalloc: the log-likelihood for callers that cannot allocate
device memory when they call (for example while a CUDA graph is being
captured without a memory pool, or in real-time code whose memory is all
reserved at start-up).  It runs on a fixed scratch array inside the library
instead of a caller workspace.  Checked through the C ABI against
spingp_loglik, which takes a workspace, on two calls in a row (the second
call reuses scratch the first one left behind), against the oracle directly
(with and without missing observations), at the largest admitted length, and
for the size limit.

This file is named so that pytest collects it last."""
import ctypes

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import seq  # noqa: E402
from paper_1610_08035_gb300 import spingp, synth  # noqa: E402

pytestmark = pytest.mark.gpu

LL_RTOL = 1e-9   # the log-likelihood tolerance used by the parity tests


def _dev(a):
    return torch.tensor(np.asarray(a, dtype=np.float64), device="cuda")


def _noalloc(lib, model, T, Y, TH, out, flags=0):
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    return lib.spingp_loglik_noalloc(model.h, ctypes.c_void_p(T.data_ptr()), ctypes.c_void_p(Y.data_ptr()),
                                     ctypes.c_int64(T.numel()), ctypes.c_void_p(TH.data_ptr()),
                                     ctypes.c_void_p(out.data_ptr()), ctypes.c_uint(spingp.SYNC | flags), stream)


@pytest.mark.parametrize("spec,workload,n", [("matern52", "matern52_n4m", 60000),
                                             ("matern32", "matern32_n1000", 1000)])
def test_noalloc_matches_workspace_entry_point(spec, workload, n):
    lib = spingp.load()
    s = synth.single(workload, n=n, seed=21)
    model = spingp.Model(s.spec)
    T, Y, TH = _dev(s.t), _dev(s.y), _dev(s.theta)
    ref = float(model.loglik(T, Y, TH).cpu()[0])
    for _ in range(2):
        out = torch.full((1,), float("nan"), dtype=torch.float64, device="cuda")
        assert _noalloc(lib, model, T, Y, TH, out) == spingp.OK
        got = float(out.cpu()[0])
        assert abs(got - ref) <= LL_RTOL * abs(ref), (got, ref)


def test_noalloc_consecutive_calls_of_different_sizes():
    """A longer call followed by a shorter one on the same scratch."""
    lib = spingp.load()
    model = spingp.Model("matern52")
    for n, seed in ((65000, 3), (777, 4)):
        s = synth.single("matern52_n4m", n=n, seed=seed)
        T, Y, TH = _dev(s.t), _dev(s.y), _dev(s.theta)
        ref = float(model.loglik(T, Y, TH).cpu()[0])
        out = torch.empty(1, dtype=torch.float64, device="cuda")
        assert _noalloc(lib, model, T, Y, TH, out) == spingp.OK
        assert abs(float(out.cpu()[0]) - ref) <= LL_RTOL * abs(ref)


@pytest.mark.parametrize("missing", [False, True])
def test_noalloc_matches_the_oracle(missing):
    """Against the sequential oracle itself; with SPINGP_MISSING_NAN, 15 % of
    the observations are NaN (test points with infinite noise, Eqs.
    mean4-mean6), which the oracle skips the same way."""
    lib = spingp.load()
    s = synth.single("matern52_n4m", n=30011, seed=31)
    y = s.y.copy()
    if missing:
        y[np.random.default_rng(7).random(len(y)) < 0.15] = np.nan
    model = spingp.Model(s.spec)
    T, Y, TH = _dev(s.t), _dev(y), _dev(s.theta)
    llo = seq.loglik(s.spec, s.theta, s.t, y)
    for _ in range(2):
        out = torch.full((1,), float("nan"), dtype=torch.float64, device="cuda")
        assert _noalloc(lib, model, T, Y, TH, out, spingp.MISSING_NAN if missing else 0) == spingp.OK
        assert abs(float(out.cpu()[0]) - llo) <= LL_RTOL * abs(llo)


def test_noalloc_at_the_largest_admitted_length():
    """n = 65536 with b = 3 fits the scratch at the default chunk length."""
    lib = spingp.load()
    model = spingp.Model("matern52")
    n = 65536
    assert spingp.spingp_workspace_bytes(model.h, n, spingp.WS_LOGLIK) <= spingp_noalloc_limit()
    s = synth.single("matern52_n4m", n=n, seed=6)
    T, Y, TH = _dev(s.t), _dev(s.y), _dev(s.theta)
    ref = float(model.loglik(T, Y, TH).cpu()[0])
    out = torch.empty(1, dtype=torch.float64, device="cuda")
    assert _noalloc(lib, model, T, Y, TH, out) == spingp.OK
    assert abs(float(out.cpu()[0]) - ref) <= LL_RTOL * abs(ref)


def test_noalloc_rejects_series_beyond_the_scratch():
    lib = spingp.load()
    model = spingp.Model("matern52")
    n = 200000
    assert spingp.spingp_workspace_bytes(model.h, n, spingp.WS_LOGLIK) > spingp_noalloc_limit()
    s = synth.single("matern52_n4m", n=n, seed=5)
    T, Y, TH = _dev(s.t), _dev(s.y), _dev(s.theta)
    out = torch.empty(1, dtype=torch.float64, device="cuda")
    assert _noalloc(lib, model, T, Y, TH, out) == spingp.EINVAL


def spingp_noalloc_limit():
    return 8 << 20   # SPINGP_NOALLOC_SCRATCH_BYTES in include/spingp.h
