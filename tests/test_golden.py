"""The stored config-1 values agree with both oracles (CPU only)."""
import numpy as np

from golden.make_golden import load_config1
from oracle import dense, seq


def test_config1_fixture_matches_oracles():
    g = load_config1()
    ll, gr = seq.grad(g["spec"], g["theta"], g["t"], g["y"])
    assert abs(ll - g["ll"]) <= 1e-13 * abs(ll)
    assert np.all(np.abs(gr - g["grad"]) <= 1e-12 * np.maximum(1.0, np.abs(gr)))
    md, vd = dense.posterior(g["spec"], g["theta"], g["t"], g["y"])
    assert np.max(np.abs(md - g["mean"])) <= 1e-12
    assert np.max(np.abs(vd - g["var"]) / vd) <= 1e-11
    lld = dense.loglik(g["spec"], g["theta"], g["t"], g["y"])
    assert abs(lld - g["ll"]) <= 1e-12 * abs(lld)
