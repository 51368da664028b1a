"""GPU parity for the paper's method as written (Theorem 1, Sec. 2.2-3.1):
the explicit blocks of the posterior precision K~, odd-even block cyclic
reduction with selected inverse on any symmetric positive-definite block-
tridiagonal matrix (subproblems 1-3), the diagonal of S X (subproblem 4), and
the composed log-likelihood, gradient and posterior -- against the oracle's
sequential block algorithm, its dense definitions and its Kalman recursions.
The assembled path forms Q^-1, so its inputs have well-separated times."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import btd, seq  # noqa: E402
from paper_1610_08035_gb300 import spingp, synth  # noqa: E402

pytestmark = pytest.mark.gpu
DEV = "cuda"

MATERN = [("matern12", [0.7, 1.3, 0.1]), ("matern32", [1.0, 1.0, 0.1]), ("matern52", [0.5, 2.0, 0.05])]


def _t(a):
    return torch.tensor(np.asarray(a, dtype=np.float64), device=DEV)


def _np(x):
    return x.cpu().numpy()


# ---------------------------------------------------------------- subproblems 1-3 on general BTD input

@pytest.mark.parametrize("b", [1, 2, 3])
@pytest.mark.parametrize("n", [1, 2, 3, 5, 64, 1000, 4099])
def test_btd_solve_matches_sequential_algorithm(b, n):
    """log det, x = T^-1 r and the selected inverse, several reduction levels
    with ragged (odd) level sizes, against the oracle's block LDL^T."""
    D, O, r = synth.random_spd_btd(n, b, seed=1000 * b + n)
    ld, x, Sd, So = spingp.btd_solve(_t(D), _t(O), _t(r))
    lo, xo, Sdo, Soo = btd.thomas(D, O, r)
    assert abs(ld.item() - lo) <= 1e-11 * abs(lo)
    assert np.max(np.abs(_np(x) - xo)) <= 1e-10 * max(1.0, np.max(np.abs(xo)))
    scale = np.max(np.abs(Sdo))
    assert np.max(np.abs(_np(Sd) - Sdo)) <= 1e-10 * scale
    if n > 1:
        assert np.max(np.abs(_np(So) - Soo)) <= 1e-10 * scale


def test_btd_solve_without_selected_inverse_is_the_same_solve():
    """Skipping the selected inverse changes neither x nor log det (bitwise)."""
    D, O, r = synth.random_spd_btd(777, 3, seed=4)
    ld1, x1, _, _ = spingp.btd_solve(_t(D), _t(O), _t(r), selected=True)
    ld2, x2, Sd, So = spingp.btd_solve(_t(D), _t(O), _t(r), selected=False)
    assert Sd is None and So is None
    assert ld1.item() == ld2.item()
    assert torch.equal(x1, x2)


def test_btd_solve_is_deterministic():
    D, O, r = synth.random_spd_btd(5000, 2, seed=8)
    a = spingp.btd_solve(_t(D), _t(O), _t(r))
    b = spingp.btd_solve(_t(D), _t(O), _t(r))
    for u, v in zip(a, b):
        assert torch.equal(u, v)


def test_btd_solve_large_against_residual():
    """A size the dense oracle cannot hold: the residual T x - r of the
    solve, and the selected inverse against the sequential algorithm."""
    n, b = 1 << 18, 3
    D, O, r = synth.random_spd_btd(n, b, seed=12)
    ld, x, Sd, So = spingp.btd_solve(_t(D), _t(O), _t(r))
    xg = _np(x)
    res = np.einsum("ipq,iq->ip", D, xg)
    res[1:] += np.einsum("ipq,iq->ip", O, xg[:-1])
    res[:-1] += np.einsum("iqp,iq->ip", O, xg[1:])
    assert np.max(np.abs(res - r)) <= 1e-11 * np.max(np.abs(r))
    lo, xo, Sdo, Soo = btd.thomas(D, O, r)
    assert abs(ld.item() - lo) <= 1e-11 * abs(lo)
    assert np.max(np.abs(_np(Sd) - Sdo)) <= 1e-10 * np.max(np.abs(Sdo))
    assert np.max(np.abs(_np(So) - Soo)) <= 1e-10 * np.max(np.abs(Sdo))


@pytest.mark.parametrize("b,n", [(1, 1), (2, 2), (3, 50), (2, 333)])
def test_btd_diag_product_matches_definition(b, n):
    """Subproblem 4: diag(T^-1 X) and its trace from the selected inverse,
    against the dense definition."""
    D, O, r = synth.random_spd_btd(n, b, seed=n + 7 * b)
    _, Xo_, _ = synth.random_spd_btd(n, b, seed=n + 7 * b + 1)
    rng = np.random.default_rng(n)
    Xd = rng.standard_normal((n, b, b))
    Xd = Xd + np.transpose(Xd, (0, 2, 1))
    Xo = Xo_ * rng.standard_normal()
    _, _, Sd, So = spingp.btd_solve(_t(D), _t(O), _t(r))
    diag, tr = spingp.btd_diag_product(Sd, So, _t(Xd), _t(Xo))
    do, tro = btd.diag_product(D, O, Xd, Xo)
    assert np.max(np.abs(_np(diag) - do)) <= 1e-10 * max(1.0, np.max(np.abs(do)))
    assert abs(tr.item() - tro) <= 1e-10 * max(1.0, np.sum(np.abs(do)))


# ---------------------------------------------------------------- Theorem 1 assembly

@pytest.mark.parametrize("spec,theta", MATERN)
@pytest.mark.parametrize("n", [1, 2, 40])
def test_assemble_matches_theorem1(spec, theta, n):
    """D_i, O_i, r and log det Kinv against the dense stacked precision of
    the oracle (Kinv from the dense A and Q matrices, K~ = Kinv + G^T G / s_n)."""
    rng = np.random.default_rng(n)
    t = synth.separated_times(n, theta[0], rng)
    y = rng.standard_normal(n)
    m = spingp.Model(spec)
    b = m.state_dim
    D, O, r, ldk = m.assemble(_t(t), _t(y), _t(theta))
    M = btd.stacked(spec, theta, t)
    Do, Oo = btd.blocks_of(M["Ktilde"], b)
    ro = (M["G"].T @ y / theta[-1]).reshape(n, b)
    assert np.max(np.abs(_np(D) - Do)) <= 1e-10 * np.max(np.abs(Do))
    if n > 1:
        assert np.max(np.abs(_np(O) - Oo)) <= 1e-10 * np.max(np.abs(Do))
    assert np.max(np.abs(_np(r) - ro)) <= 1e-14 * np.max(np.abs(ro))
    ldo = np.linalg.slogdet(M["Kinv"])[1]
    assert abs(ldk.item() - ldo) <= 1e-10 * max(1.0, abs(ldo))


# ---------------------------------------------------------------- the composed method

def _literal_data(spec, theta, n, seed):
    rng = np.random.default_rng(seed)
    t = synth.separated_times(n, theta[0], rng)
    y = synth.two_sinusoids(t, theta[0], theta[1], theta[-1], rng)
    return t, y


@pytest.mark.parametrize("spec,theta", MATERN)
@pytest.mark.parametrize("n", [1, 7, 4097, 100000])
def test_literal_loglik_and_grad_match_oracle(spec, theta, n):
    """Eqs. ml2/det_1 and the Eq. dd1 gradient through K~ against the oracle's
    Kalman log-likelihood and two-filter gradient."""
    t, y = _literal_data(spec, theta, n, n + 3)
    m = spingp.Model(spec)
    ll = m.literal(_t(t), _t(y), _t(theta))
    ll2, g = m.literal(_t(t), _t(y), _t(theta), what=spingp.WS_GRAD)
    llo, go, gabs = seq.grad(spec, theta, t, y, l1=True)
    assert abs(ll.item() - llo) <= 1e-9 * abs(llo)
    assert ll.item() == ll2.item()
    gg = _np(g)
    # the literal gradient is a sum of O(1) terms (coordinate-scaling and
    # log det Kinv parts) that cancel exactly where the true entry is 0, e.g.
    # d ll / d l at n = 1: hence the absolute floor
    assert np.all(np.abs(gg - go) <= 1e-8 * np.maximum(np.maximum(np.abs(go), gabs), 1e-6)), (gg, go, gabs)


@pytest.mark.parametrize("spec,theta", MATERN)
@pytest.mark.parametrize("n", [1, 5, 4097])
def test_literal_posterior_matches_oracle(spec, theta, n):
    """Subproblems 1 and 2: H x and the diagonal of H K~^-1 H^T against the
    oracle's smoother."""
    t, y = _literal_data(spec, theta, n, n + 11)
    m = spingp.Model(spec)
    mean, var, ll = m.literal(_t(t), _t(y), _t(theta), what=spingp.WS_POSTERIOR)
    sm = seq.smoother(spec, theta, t, y)
    mo, vo = sm["mean"], sm["var"]
    mg, vg = _np(mean), _np(var)
    assert np.all(np.abs(mg - mo) <= 1e-8 * np.maximum(np.abs(mo), np.sqrt(vo)))
    assert np.max(np.abs(vg - vo) / vo) <= 1e-8
    assert abs(ll.item() - sm["ll"]) <= 1e-9 * abs(sm["ll"])


def test_literal_single_point():
    """n = 1: ll = log N(y; 0, s_f + s_n) and the closed-form posterior."""
    theta = [0.5, 2.0, 0.05]
    m = spingp.Model("matern52")
    y = 0.7
    mean, var, ll = m.literal(_t([3.0]), _t([y]), _t(theta), what=spingp.WS_POSTERIOR)
    s = theta[1] + theta[2]
    assert abs(ll.item() - (-0.5 * y * y / s - 0.5 * np.log(2 * np.pi * s))) <= 1e-14
    assert abs(mean.item() - theta[1] / s * y) <= 1e-14
    assert abs(var.item() - theta[1] * theta[2] / s) <= 1e-14


# ---------------------------------------------------------------- errors

def _status(fn):
    with pytest.raises(spingp.SpinGPError) as e:
        fn()
    return e.value.status


def test_literal_error_statuses():
    m = spingp.Model("matern32")
    theta = _t([1.0, 1.0, 0.1])
    t = np.cumsum(np.full(50, 0.5))
    y = np.sin(t)
    tt = t.copy(); tt[10] = tt[9]                 # a tie: Q = 0 has no inverse
    assert _status(lambda: m.literal(_t(tt), _t(y), theta)) == spingp.ENUMERIC
    tu = t.copy(); tu[10] = tu[9] - 0.1           # unsorted
    assert _status(lambda: m.literal(_t(tu), _t(y), theta)) == spingp.ENOTSORTED
    yn = y.copy(); yn[3] = np.nan
    assert _status(lambda: m.literal(_t(t), _t(yn), theta)) == spingp.ENONFINITE
    assert _status(lambda: m.literal(_t(t), _t(y), _t([1.0, -1.0, 0.1]))) == spingp.EINVAL
    mq = spingp.Model(["matern32", ("quasiperiodic", 3, "matern12")])
    with pytest.raises(spingp.SpinGPError):
        mq.assemble(_t(t), _t(y), _t([1.0, 1.0, 1.0, 1.0, 1.0, 3.0, 0.1]))
    # the model is fine again afterwards
    ll = m.literal(_t(t), _t(y), theta)
    assert np.isfinite(ll.item())


def test_btd_error_statuses():
    D, O, r = synth.random_spd_btd(64, 2, seed=3)
    Dbad = D.copy()
    Dbad[17] = -np.eye(2)
    assert _status(lambda: spingp.btd_solve(_t(Dbad), _t(O), _t(r))) == spingp.ENUMERIC
    lib = spingp.load()
    ws = torch.empty(16, dtype=torch.uint8, device=DEV)
    x = torch.empty(64, 2, dtype=torch.float64, device=DEV)
    ld = torch.empty(1, dtype=torch.float64, device=DEV)
    Dt, Ot, rt = _t(D), _t(O), _t(r)
    st = spingp.spingp_btd_solve(2, 64, Dt, Ot, rt, ld, x, None, None, ws, ws.numel(), spingp.SYNC)
    assert st == spingp.EINVAL                          # workspace too small
    assert spingp.spingp_btd_solve(4, 64, Dt, Ot, rt, ld, x, None, None, ws, 1 << 30, 0) == spingp.EINVAL
    assert lib.spingp_btd_workspace_bytes(4, 64) == 0
    assert spingp.spingp_btd_launch_count(64) == 2 * 6 + 3
    assert spingp.spingp_literal_launch_count(64) == 3 + (2 * 6 + 3) + 4
