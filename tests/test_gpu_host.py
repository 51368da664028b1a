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
