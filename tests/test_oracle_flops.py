"""The counted restatement of the sequential method (oracle/flops.py), which
gives the benchmark its algorithmic flops per step.  Two pins: it computes
the method (its log-likelihood and every gradient entry equal the oracle's
two-filter values on the same series), and its per-step count equals the
closed form of the operations it lists, 12 b^3 + (21 + 2 P_A) b^2 + 11 b + 11
with P_A the parameters the transition depends on."""
import numpy as np
import pytest

from oracle import flops, seq


def _series(n, seed):
    rng = np.random.default_rng(seed)
    t = np.cumsum(rng.exponential(0.02, n))
    y = np.sin(5.0 * t) + 0.3 * rng.standard_normal(n)
    return t, y


CASES = [(name, spec, th, pa) for (name, (spec, th)), pa in zip(flops.MODELS.items(), (1, 1, 2, 3))]


@pytest.mark.parametrize("name,spec,theta,pa", CASES)
def test_restatement_reproduces_the_oracle(name, spec, theta, pa):
    t, y = _series(240, 3)
    ll, g, _ = flops.grad_counted(spec, theta, t, y)
    llo, go, g1 = seq.grad(spec, theta, t, y, l1=True)
    assert abs(ll - llo) <= 1e-12 * abs(llo)
    assert np.all(np.abs(g - go) <= 1e-11 * np.maximum(np.abs(go), g1)), (g, go)


@pytest.mark.parametrize("name,spec,theta,pa", CASES)
def test_count_per_step_is_the_closed_form(name, spec, theta, pa):
    t, y = _series(200, 4)
    b = len(seq.continuous(spec, theta)[2])
    want = 12 * b ** 3 + (21 + 2 * pa) * b ** 2 + 11 * b + 11
    assert flops.flops_per_step(spec, theta, t, y, 40, 200) == want


@pytest.mark.parametrize("old,new", [
    ("gpinf += c.ew(G - 0.5 * (np.outer(lh, lh) - Lh), 5)", "gpinf += c.ew(G, 5)"),   # drop A^T G A
    ("Abar = c.ew(-np.outer(lt, m_prev)", "Abar = c.ew(np.outer(lt, m_prev)"),          # sign of the mean term
    ("gnoise += c.scalar(al * al - cc, 3)", "gnoise += c.scalar(al * al + cc, 3)"),      # sign of the trace term
])
def test_planted_mistakes_are_caught(old, new):
    """A copy of the restatement with one plausible mistake no longer
    reproduces the oracle's gradient: the pin above separates them."""
    import inspect
    src = inspect.getsource(flops)
    assert old in src
    ns = {"__name__": "flops_mutant"}
    exec(compile(src.replace("from . import n_params, seq, state_dim",
                             "from oracle import n_params, seq, state_dim").replace(old, new), "mutant", "exec"), ns)
    t, y = _series(150, 5)
    spec, th = "matern52", [0.5, 2.0, 0.05]
    _, g, _ = ns["grad_counted"](spec, th, t, y)
    _, go, g1 = seq.grad(spec, th, t, y, l1=True)
    assert not np.all(np.abs(g - go) <= 1e-11 * np.maximum(np.abs(go), g1))
