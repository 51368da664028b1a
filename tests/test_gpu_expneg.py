"""The chain kernels' table-driven e^-x (the e^{-lam dt} factor of the Matern
transition, Eq. ss_matern) against NumPy's exponential and CUDA's, which
are both within one unit in the last place of the exact value: the table
method must stay within two units of either, return exactly 1 at 0, 0 above
708 and propagate NaN."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_1610_08035_gb300 import spingp  # noqa: E402

pytestmark = pytest.mark.gpu


def _inputs():
    rng = np.random.default_rng(17)
    return np.concatenate([
        rng.exponential(0.05, 200000),            # lam dt at the benchmark's spacing
        rng.exponential(2.0, 100000),
        rng.uniform(0.0, 708.0, 100000),
        np.arange(0, 4096) * (np.log(2.0) / 256.0),   # table-interval midpoints and ends
        [0.0, 5e-324, 1e-300, 1e-17, 1e-8, 0.5, 1.0, 2.0, 700.0, 707.9, 708.0],
    ])


def test_exp_neg_within_two_ulp():
    x = _inputs()
    y = spingp.spingp_probe_exp_neg(torch.tensor(x, device="cuda")).cpu().numpy()
    ref = np.exp(-x)
    ulp = np.spacing(ref)
    err = np.abs(y - ref) / ulp
    print("\nmax error %.2f ulp, mean %.3f ulp" % (err.max(), err.mean()))
    assert err.max() <= 2.0
    cuda = torch.exp(-torch.tensor(x, device="cuda")).cpu().numpy()
    assert np.max(np.abs(y - cuda) / ulp) <= 2.0
    assert y[x == 0.0][0] == 1.0


def test_exp_neg_edges():
    x = np.array([708.5, 709.0, 745.2, 1e5, 1e300, np.inf, np.nan])
    y = spingp.spingp_probe_exp_neg(torch.tensor(x, device="cuda")).cpu().numpy()
    assert np.all(y[:-1] == 0.0)
    assert np.isnan(y[-1])
    z = spingp.spingp_probe_exp_neg(torch.empty(0, dtype=torch.float64, device="cuda"))
    assert z.numel() == 0
