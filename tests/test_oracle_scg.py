"""Pins for the oracle's scaled-conjugate-gradient optimiser (Moller 1993;
the paper fits hyperparameters with it, Sec. 4.3): properties fixed by the
mathematics, not by the implementation.

* on a quadratic, conjugate directions reach the minimiser A^-1 b in about
  P iterations (the finite-termination property of conjugate gradients);
* on the Rosenbrock function it reaches the known minimiser (1, 1);
* on a GP marginal likelihood it reaches the optimum that a library
  quasi-Newton method (scipy L-BFGS-B) finds on the same objective, with a
  vanishing gradient there."""
import numpy as np
from scipy.optimize import minimize

from oracle import dense, scg, seq
from paper_1610_08035_gb300 import synth


def test_quadratic_reaches_the_minimiser():
    rng = np.random.default_rng(0)
    P = 5
    Q, _ = np.linalg.qr(rng.standard_normal((P, P)))
    A = Q @ np.diag(np.logspace(0, 2, P)) @ Q.T
    b = rng.standard_normal(P)
    w_star = np.linalg.solve(A, b)
    fg = lambda w: (0.5 * w @ A @ w - b @ w, A @ w - b)
    w, f, g, traj = scg.scg(fg, np.zeros(P), 4 * P)
    assert np.max(np.abs(w - w_star)) <= 1e-9 * np.max(np.abs(w_star))
    assert len(traj) == 4 * P + 1
    # after P + 2 iterations it is already close (conjugacy, up to the small
    # initial scale lambda_1 and the one-sided curvature estimate)
    assert np.max(np.abs(traj[P + 2] - w_star)) <= 1e-4 * np.max(np.abs(w_star))


def test_rosenbrock():
    """Conjugate directions reach (1, 1) from (-1.2, 1) in about 100
    iterations (steepest descent with the same step control needs thousands):
    a budget of 300."""
    def fg(w):
        x, y = w
        f = (1 - x) ** 2 + 100 * (y - x * x) ** 2
        return f, np.array([-2 * (1 - x) - 400 * x * (y - x * x), 200 * (y - x * x)])
    w, f, g, _ = scg.scg(fg, np.array([-1.2, 1.0]), 300, tol=1e-10)
    assert np.max(np.abs(w - 1.0)) <= 1e-6


def test_gp_optimum_matches_library_quasi_newton():
    spec = "matern32"
    rng = np.random.default_rng(3)
    t = synth.exp_times(300, 0.1, rng)
    y = synth.two_sinusoids(t, 1.0, 1.0, 0.1, rng)
    fg = scg.gp_objective(spec, t, y, dense.grad)
    w0 = np.log([0.5, 0.5, 0.5])
    w, f, g, _ = scg.scg(fg, w0, 300, tol=1e-9)
    res = minimize(fg, w0, jac=True, method="L-BFGS-B", options=dict(gtol=1e-12, ftol=1e-15, maxiter=2000))
    assert np.max(np.abs(g)) <= 1e-6
    assert f <= res.fun + 1e-8
    assert np.max(np.abs(w - res.x)) <= 1e-4
    # the sequential oracle gives the same optimiser path as the dense one
    w2, f2, _, _ = scg.scg(scg.gp_objective(spec, t, y, seq.grad), w0, 300, tol=1e-9)
    assert np.max(np.abs(w2 - w)) <= 1e-6


def test_rejected_trial_points_do_not_move():
    """An objective that is infinite beyond a wall: trial points there are
    rejected, the iterate stays feasible and still converges."""
    def fg(w):
        if w[0] > 0.5:
            return np.inf, np.zeros(2)
        return (w[0] - 0.4) ** 2 + (w[1] + 1) ** 2, np.array([2 * (w[0] - 0.4), 2 * (w[1] + 1)])
    w, f, g, traj = scg.scg(fg, np.array([-3.0, 2.0]), 200, tol=1e-12)
    assert np.all(traj[:, 0] <= 0.5)
    assert np.max(np.abs(w - [0.4, -1.0])) <= 1e-8
