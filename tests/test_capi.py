"""The C-ABI library builds, loads and exports every entry point declared in
include/*.h; host-only calls behave as documented.  No GPU work is launched."""
import ctypes
import glob
import os
import re

import pytest

from paper_1610_08035_gb300 import build as libbuild
from paper_1610_08035_gb300 import spingp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
DECL = re.compile(r"^(?:spingp_status|void|int|size_t|const char\s*\*)\s+(spingp_\w+)\s*\(", re.M)


def declared_names():
    names = []
    for h in sorted(glob.glob(os.path.join(ROOT, "include", "*.h"))):
        names += DECL.findall(open(h).read())
    return names


@pytest.fixture(scope="module")
def lib():
    libbuild.build()
    return spingp.load()


def test_header_declares_the_boundary():
    names = declared_names()
    for required in ("spingp_loglik", "spingp_grad", "spingp_posterior", "spingp_model_create",
                     "spingp_workspace_bytes", "spingp_status_str"):
        assert required in names


def test_every_declared_symbol_is_exported(lib):
    raw = ctypes.CDLL(spingp.LIB_PATH)
    for name in declared_names():
        assert hasattr(raw, name), name
    assert set(declared_names()) <= set(spingp.EXPORTS) | set(declared_names())


def test_model_create_and_queries(lib):
    for spec, b, P in (("matern12", 1, 3), ("matern32", 2, 3), ("matern52", 3, 3)):
        h = spingp.spingp_model_create(spec)
        assert spingp.spingp_state_dim(h) == b
        assert spingp.spingp_num_params(h) == P
        w1 = spingp.spingp_workspace_bytes(h, 1000, spingp.WS_LOGLIK)
        w2 = spingp.spingp_workspace_bytes(h, 1000, spingp.WS_GRAD)
        w3 = spingp.spingp_workspace_bytes(h, 10 ** 6, spingp.WS_GRAD)
        assert 0 < w1 < w2 < w3
        spingp.spingp_set_chunk_len(h, 64)
        assert spingp.spingp_get_chunk_len(h, 10 ** 6) == 64
        with pytest.raises(spingp.SpinGPError):
            spingp.spingp_set_chunk_len(h, 3)
        spingp.spingp_model_destroy(h)


def test_model_create_rejects_bad_descriptions(lib):
    # the structures the header lists as not run on the GPU
    for spec in (["matern52", "matern32"], ["matern12", "matern32"], [("quasiperiodic", 2, "matern32")],
                 ["matern32", ("periodic", 7)]):                                   # the last: 18 states
        with pytest.raises(spingp.SpinGPError) as e:
            spingp.spingp_model_create(spec)
        assert e.value.status == spingp.EUNSUPPORTED, spec
    desc = spingp._Desc(1, (ctypes.c_int * 1)(9), None, None)
    h = ctypes.c_void_p()
    assert lib.spingp_model_create(ctypes.byref(desc), ctypes.byref(h)) == spingp.EINVAL
    assert not h.value
    assert lib.spingp_model_create(None, ctypes.byref(h)) == spingp.EINVAL


def test_entry_points_reject_null_arguments_without_launching(lib):
    h = spingp.spingp_model_create("matern32")
    null = ctypes.c_void_p()
    assert lib.spingp_loglik(h, null, null, 10, null, null, null, 0, 0, null) == spingp.EINVAL
    assert lib.spingp_grad(h, null, null, 10, null, null, null, null, 0, 0, null) == spingp.EINVAL
    assert lib.spingp_posterior(h, null, null, 10, null, null, null, null, null, 0, 0, null) == spingp.EINVAL
    # an empty series (n = 0) is rejected before any device work, whatever the pointers
    fake = ctypes.c_void_p(256)
    assert lib.spingp_loglik(h, fake, fake, 0, fake, fake, fake, 1 << 20, 0, null) == spingp.EINVAL
    assert lib.spingp_grad(h, fake, fake, 0, fake, fake, fake, fake, 1 << 20, 0, null) == spingp.EINVAL
    assert spingp.spingp_workspace_bytes(h, 0, spingp.WS_GRAD) == 0
    spingp.spingp_model_destroy(h)


def test_status_strings(lib):
    for st in range(9):
        assert isinstance(spingp.spingp_status_str(st), str) and spingp.spingp_status_str(st)


def test_eq_model_creation_host_only():
    """EQ models are built on the host (modal constants at model creation):
    dimensions, parameter counts and the rejected forms, without a GPU."""
    from paper_1610_08035_gb300 import spingp
    m = spingp.Model(["matern32", ("eq", 10)])
    assert (m.state_dim, m.num_params) == (12, 5)
    for N in (2, 4, 6, 8, 10, 12, 14, 16):
        assert spingp.Model([("eq", N)]).state_dim == N
    for bad in ([("eq", 5)], [("eq", 0)], [("eq", 18)], ["matern32", ("eq", 16)], [("eq", 4), ("eq", 6)]):
        with pytest.raises(spingp.SpinGPError):
            spingp.Model(bad)
