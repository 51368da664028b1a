"""Scaled conjugate gradients (Moller 1993), the optimiser the paper uses to
fit kernel hyperparameters by maximising the marginal likelihood (Sec. 4.3,
citing Rasmussen & Williams 2006).

TEST INFRASTRUCTURE ONLY (see the package docstring).

Moller's algorithm minimises E(w) with gradients only: the curvature along the
search direction p is a one-sided difference of gradients,
s = (E'(w + sigma p) - E'(w)) / sigma with sigma = sigma0 / |p|, and a
Levenberg-Marquardt-style scale lambda keeps the local quadratic model
positive definite and is adapted from the ratio Delta between the actual and
the predicted reduction.  The steps below follow the published order:

  1. (success) second-order information s, delta = p.s
  2. scale: s += (lambda - lambda_bar) p, delta += (lambda - lambda_bar)|p|^2
  3. delta <= 0: make the model positive definite (lambda_bar = 2(lambda - delta/|p|^2),
     delta = -delta + lambda |p|^2, lambda = lambda_bar)
  4. mu = p.r, alpha = mu / delta
  5. Delta = 2 delta (E(w) - E(w + alpha p)) / mu^2
  6. Delta >= 0: accept; r_new = -E'(w_new); lambda_bar = 0; restart p = r_new
     every P iterations, else p = r_new + beta p with
     beta = (|r_new|^2 - r_new.r) / mu; Delta >= 0.75: lambda /= 4.
     Delta < 0: reject (lambda_bar = lambda, no new second-order information).
  7. Delta < 0.25: lambda += delta (1 - Delta) / |p|^2

Choices where the published algorithm leaves room (the device optimiser makes
the same ones): sigma0 = 1e-4, lambda_1 = 1e-6, lambda kept in
[1e-15, 1e100]; a trial point whose objective is not finite counts as
Delta = -1 (rejected); a zero p.r or delta restarts along r; |p|^2 in step 7
is that of the direction just tried; the iteration stops once
max |E'| <= tol or p = 0.
"""
import numpy as np

SIGMA0 = 1e-4
LAMBDA1 = 1e-6
LAM_MIN = 1e-15
LAM_MAX = 1e100


def scg(fg, w0, iters, tol=0.0):
    """Minimise E with fg(w) -> (E(w), E'(w)).  Runs at most `iters`
    iterations.  Returns (w, E(w), E'(w), trajectory of accepted w per
    iteration (iters + 1 rows, the start included))."""
    w = np.array(w0, dtype=np.float64)
    P = len(w)
    f, g = fg(w)
    g = np.asarray(g, dtype=np.float64)
    r = -g
    p = r.copy()
    lam, lambar, success = LAMBDA1, 0.0, True
    s = np.zeros(P)
    delta = 0.0
    done = bool(np.max(np.abs(g)) <= tol) or not np.any(p)
    traj = [w.copy()]
    for k in range(1, iters + 1):
        if done:
            traj.append(w.copy())
            continue
        pp = p @ p
        if success:
            sigma = SIGMA0 / np.sqrt(pp)
            _, gs = fg(w + sigma * p)
            s = (np.asarray(gs) - g) / sigma
            delta = p @ s
        s = s + (lam - lambar) * p
        delta = delta + (lam - lambar) * pp
        if delta <= 0.0:
            s = s + (lam - 2.0 * delta / pp) * p
            lambar = 2.0 * (lam - delta / pp)
            delta = -delta + lam * pp
            lam = lambar
        mu = p @ r
        if mu == 0.0 or delta == 0.0:
            p = r.copy()
            lambar, success = 0.0, True
            traj.append(w.copy())
            continue
        alpha = mu / delta
        wn = w + alpha * p
        fn, gn = fg(wn)
        Delta = 2.0 * delta * (f - fn) / (mu * mu) if np.isfinite(fn) else -1.0
        if Delta >= 0.0:
            w, f, g = wn, fn, np.asarray(gn, dtype=np.float64)
            rn = -g
            lambar, success = 0.0, True
            if k % P == 0:
                p_new = rn.copy()
            else:
                beta = (rn @ rn - rn @ r) / mu
                p_new = rn + beta * p
            r = rn
            if Delta >= 0.75:
                lam = max(lam / 4.0, LAM_MIN)
        else:
            lambar, success = lam, False
            p_new = p
        if Delta < 0.25:
            lam = min(lam + delta * (1.0 - Delta) / pp, LAM_MAX)
        p = p_new
        traj.append(w.copy())
        if np.max(np.abs(g)) <= tol or not np.any(p):
            done = True
    return w, f, g, np.array(traj)


def gp_objective(spec, t, y, grad_fn):
    """E(w) = -ll(exp(w)) and its gradient in log-parameters, from a function
    grad_fn(spec, theta, t, y) -> (ll, dll/dtheta).  A failed evaluation is
    an infinite objective."""
    def fg(w):
        theta = np.exp(w)
        try:
            ll, gr = grad_fn(spec, theta, t, y)
        except Exception:
            return np.inf, np.zeros_like(w)
        if not np.isfinite(ll) or not np.all(np.isfinite(gr)):
            return np.inf, np.zeros_like(w)
        return -ll, -theta * np.asarray(gr)
    return fg
