"""spingp_grad_host: log-likelihood and gradient from host buffers, with the
host-to-device copies overlapping the elimination.  The result must be the
device call's, bit for bit (the same kernels on the same blocks), for pinned
and pageable host memory, repeated calls, and structured models."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_1610_08035_gb300 import spingp, synth  # noqa: E402

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("spec,theta,n", [("matern52", [0.5, 2.0, 0.05], 1 << 20),
                                          ("matern32", [1.0, 1.0, 0.1], 1001),
                                          ("matern12", [0.7, 1.3, 0.1], 1),
                                          (["matern32", ("quasiperiodic", 3, "matern12")],
                                           [1.0, 1.0, 1.0, 1.0, 1.0, 5.0, 0.01], 30011)])
@pytest.mark.parametrize("pinned", [True, False])
def test_grad_host_equals_device_call(spec, theta, n, pinned):
    rng = np.random.default_rng(n)
    t = synth.exp_times(n, 0.01, rng)
    y = synth.two_sinusoids(t, 0.5, 1.0, 0.1, rng)
    m = spingp.Model(spec)
    ll_d, g_d = m.grad(torch.tensor(t, device="cuda"), torch.tensor(y, device="cuda"),
                       torch.tensor(theta, dtype=torch.float64, device="cuda"))
    th, yh, thh = torch.from_numpy(t), torch.from_numpy(y), torch.tensor(theta, dtype=torch.float64)
    if pinned:
        th, yh, thh = th.pin_memory(), yh.pin_memory(), thh.pin_memory()
    for _ in range(3):   # repeated calls reuse the copy stream and the workspace
        ll_h, g_h = m.grad_host(th, yh, thh)
        assert ll_h.item() == ll_d.item()
        assert torch.equal(g_h, g_d.cpu())


def test_grad_host_errors():
    m = spingp.Model("matern52")
    t = torch.arange(10, dtype=torch.float64)
    with pytest.raises(TypeError):
        m.grad_host(t.cuda(), t, torch.ones(3, dtype=torch.float64))
    with pytest.raises(ValueError):
        m.grad_host(t, t[:5], torch.ones(3, dtype=torch.float64))
    tu = t.clone(); tu[4] = -1.0
    with pytest.raises(spingp.SpinGPError) as e:
        m.grad_host(tu, t, torch.ones(3, dtype=torch.float64))
    assert e.value.status == spingp.ENOTSORTED


@pytest.mark.parametrize("L", [8, 9, 17, 64, 0])
@pytest.mark.parametrize("n", [5003, 4 * 128 * 17])
def test_grad_host_step_pieces(L, n):
    """The host path eliminates each chunk in four launches over strided
    pieces of its steps, of doubling widths (the copy of the next piece
    overlapping).  Pieces of one step (L = 8, 9), widths that leave an odd
    remainder, a last chunk shorter than the first pieces, and n a multiple
    of L all give the device call's bits."""
    rng = np.random.default_rng(L + n)
    t = synth.exp_times(n, 0.02, rng)
    y = synth.two_sinusoids(t, 0.5, 1.0, 0.1, rng)
    theta = [0.4, 1.5, 0.08]
    m = spingp.Model("matern52", chunk_len=L)
    ll_d, g_d = m.grad(torch.tensor(t, device="cuda"), torch.tensor(y, device="cuda"),
                       torch.tensor(theta, dtype=torch.float64, device="cuda"))
    ll_h, g_h = m.grad_host(torch.from_numpy(t).pin_memory(), torch.from_numpy(y).pin_memory(),
                            torch.tensor(theta, dtype=torch.float64))
    assert ll_h.item() == ll_d.item()
    assert torch.equal(g_h, g_d.cpu())


def test_grad_host_missing_observations():
    n = 20011
    rng = np.random.default_rng(5)
    t = synth.exp_times(n, 0.02, rng)
    y = synth.two_sinusoids(t, 0.5, 1.0, 0.1, rng)
    y[rng.random(n) < 0.2] = np.nan
    theta = [0.4, 1.5, 0.08]
    m = spingp.Model("matern32", chunk_len=13)
    ll_d, g_d = m.grad(torch.tensor(t, device="cuda"), torch.tensor(y, device="cuda"),
                       torch.tensor(theta, dtype=torch.float64, device="cuda"), missing=True)
    ll_h, g_h = m.grad_host(torch.from_numpy(t).pin_memory(), torch.from_numpy(y).pin_memory(),
                            torch.tensor(theta, dtype=torch.float64), missing=True)
    assert np.isfinite(ll_d.item())
    assert ll_h.item() == ll_d.item()
    assert torch.equal(g_h, g_d.cpu())
