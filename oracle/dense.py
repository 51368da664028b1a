"""O-dense: the plain O(N^3) Gaussian process (Eq. ml2, Sec. 2.2-2.4).

TEST INFRASTRUCTURE ONLY (see the package docstring).

The covariance matrix is built from closed-form covariance functions written
here independently of any state-space construction:

* Matern-nu with lam = sqrt(2 nu)/l and r = lam |tau|:
  nu=1/2: s e^-r;  nu=3/2: s (1+r) e^-r;  nu=5/2: s (1+r+r^2/3) e^-r
  (Sec. 2.1 gives the 3/2 case; the variance s multiplies it).
* periodic: the cosine series of s exp(-2 sin^2(w tau / 2)/l^2), w = 2 pi/p,
  which equals s e^-x sum_j c_j I_j(x) cos(j w tau) with x = 1/l^2, c_0 = 1,
  c_j = 2, truncated at harmonic J (the family the state-space form of order J
  represents exactly).
* quasi-periodic: periodic times a unit-variance Matern envelope (Eq. co2_1's
  quasi-periodic term).
* exponentiated quadratic, state-space approximation of even order N
  (Hartikainen & Sarkka 2010): the spectral density of s exp(-tau^2/(2 l^2)),
  s sqrt(2 pi) l exp(-l^2 w^2 / 2), with exp(l^2 w^2 / 2) replaced by its
  Taylor polynomial p(l w), p(u) = sum_{n<=N} (u^2/2)^n / n!.  Its covariance
  is the inverse Fourier transform of that rational density, here by residues:
  with u_j the roots of p in the upper half plane,
      k(tau) = s sqrt(2 pi) Re( i sum_j exp(i u_j |tau| / l) / p'(u_j) )
  (the roots by a library polynomial solver).
* sums of components add.

With C = K + sigma_n^2 I (Eq. k2, Sigma = sigma_n^2 I):
  log-likelihood  -1/2 y^T C^-1 y - 1/2 log det C - N/2 log 2 pi   (Eq. ml2)
  posterior mean  K C^-1 y, latent variance diag(K - K C^-1 K)      (Eqs. mean2, k3)
  gradient        1/2 tr((a a^T - C^-1) dC/dtheta), a = C^-1 y     (Sec. 2.4; the
                  textbook form, Rasmussen & Williams 2006, Eq. 5.9)
The Cholesky factorisation and triangular solves are library routines.
"""
import numpy as np
from scipy.linalg import cho_factor, cho_solve, solve_triangular
from scipy.special import iv, ivp

from . import normalize_spec, n_params

LOG2PI = np.log(2.0 * np.pi)


def _matern(b, ell, var, tau):
    """Matern covariance with nu = b - 1/2 and its derivatives (d/dl, d/dvar)."""
    lam = np.sqrt(2.0 * b - 1.0) / ell
    r = lam * np.abs(tau)
    e = np.exp(-r)
    if b == 1:
        base = e
        dbase_dl = e * r / ell
    elif b == 2:
        base = (1.0 + r) * e
        dbase_dl = r * r * e / ell
    elif b == 3:
        base = (1.0 + r + r * r / 3.0) * e
        dbase_dl = r * r * (1.0 + r) * e / (3.0 * ell)
    else:
        raise ValueError(b)
    return var * base, var * dbase_dl, base


def _periodic(J, var, lp, per, tau):
    """Truncated periodic series and derivatives (d/dvar, d/dl, d/dp)."""
    x = 1.0 / (lp * lp)
    dx_dl = -2.0 / (lp ** 3)
    w = 2.0 * np.pi / per
    dw_dp = -2.0 * np.pi / (per * per)
    ex = np.exp(-x)
    base = np.zeros_like(tau)
    dbase_dl = np.zeros_like(tau)
    dbase_dp = np.zeros_like(tau)
    for j in range(J + 1):
        c = 1.0 if j == 0 else 2.0
        wj = c * ex * iv(j, x)
        dwj_dx = c * ex * (ivp(j, x) - iv(j, x))
        cs = np.cos(j * w * tau)
        base += wj * cs
        dbase_dl += dwj_dx * dx_dl * cs
        dbase_dp += wj * (-np.sin(j * w * tau)) * j * tau * dw_dp
    return var * base, base, var * dbase_dl, var * dbase_dp


def _eq_poly(N):
    """p(u) = sum_{n<=N} (u^2/2)^n / n!, coefficients highest degree first."""
    c = np.zeros(2 * N + 1)
    f = 1.0
    for n in range(N + 1):
        if n > 0:
            f *= n
        c[2 * N - 2 * n] = 0.5 ** n / f
    return c


def _eq(N, ell, var, tau):
    """The order-N approximate EQ covariance and its derivatives (d/dl, d/dvar)."""
    c = _eq_poly(N)
    u = np.roots(c)
    u = u[u.imag > 0]
    dp = np.polyder(c)
    s = np.abs(tau) / ell
    g = np.zeros_like(s)
    dg = np.zeros_like(s)
    for uj in u:
        w = 1.0 / np.polyval(dp, uj)
        e = np.exp(1j * uj * s)
        g = g + np.real(1j * w * e)
        dg = dg + np.real(-uj * w * e)          # d/ds of Re(i w e^{i u s})
    g = g * np.sqrt(2.0 * np.pi)
    dg = dg * np.sqrt(2.0 * np.pi)
    return var * g, var * dg * (-s / ell), g


def eq_exact(var, ell, tau):
    """The exponentiated-quadratic covariance itself, s exp(-tau^2 / (2 l^2))."""
    return var * np.exp(-0.5 * (np.asarray(tau) / ell) ** 2)


def periodic_exact(var, lp, per, tau):
    """The untruncated periodic covariance s exp(-2 sin^2(pi tau / p) / l^2)."""
    return var * np.exp(-2.0 * np.sin(np.pi * tau / per) ** 2 / (lp * lp))


def kernel(spec, theta, tau):
    """k(tau) and [dk/dtheta_p for each covariance parameter] (noise excluded)."""
    theta = np.asarray(theta, dtype=np.float64)
    if theta.shape != (n_params(spec),):
        raise ValueError("theta has the wrong length")
    tau = np.asarray(tau, dtype=np.float64)
    k = np.zeros_like(tau)
    dk = []
    p = 0
    for code, order, env in normalize_spec(spec):
        if code <= 3:
            ell, var = theta[p], theta[p + 1]
            kv, dkl, base = _matern(code, ell, var, tau)
            k += kv
            dk += [dkl, base]
            p += 2
        elif code == 6:
            ell, var = theta[p], theta[p + 1]
            kv, dkl, base = _eq(order, ell, var, tau)
            k += kv
            dk += [dkl, base]
            p += 2
        else:
            var, lp, per = theta[p], theta[p + 1], theta[p + 2]
            kv, dvar, dlp, dper = _periodic(order, var, lp, per, tau)
            if code == 4:
                k += kv
                dk += [dvar, dlp, dper]
                p += 3
            else:
                lenv = theta[p + 3]
                ke, dke, _ = _matern(env, lenv, 1.0, tau)
                k += kv * ke
                dk += [dvar * ke, dlp * ke, dper * ke, kv * dke]
                p += 4
    return k, dk


def gram(spec, theta, t):
    """K(t, t) and its derivatives, one matrix per covariance parameter."""
    t = np.asarray(t, dtype=np.float64)
    tau = t[:, None] - t[None, :]
    return kernel(spec, theta, tau)


def _factor(spec, theta, t):
    K, dK = gram(spec, theta, t)
    s2 = float(theta[-1])
    C = K + s2 * np.eye(len(t))
    cf = cho_factor(C, lower=True)
    return K, dK, C, cf


def loglik(spec, theta, t, y):
    y = np.asarray(y, dtype=np.float64)
    _, _, _, cf = _factor(spec, theta, t)
    a = cho_solve(cf, y)
    logdet = 2.0 * np.sum(np.log(np.diag(cf[0])))
    return float(-0.5 * y @ a - 0.5 * logdet - 0.5 * len(y) * LOG2PI)


def posterior(spec, theta, t, y):
    """Latent posterior mean and variance at the training times."""
    y = np.asarray(y, dtype=np.float64)
    K, _, _, cf = _factor(spec, theta, t)
    a = cho_solve(cf, y)
    V = solve_triangular(cf[0], K, lower=True)
    return K @ a, np.diag(K) - np.sum(V * V, axis=0)


def grad(spec, theta, t, y):
    """Log-likelihood and gradient with respect to every entry of theta."""
    y = np.asarray(y, dtype=np.float64)
    K, dK, C, cf = _factor(spec, theta, t)
    n = len(y)
    a = cho_solve(cf, y)
    Cinv = cho_solve(cf, np.eye(n))
    logdet = 2.0 * np.sum(np.log(np.diag(cf[0])))
    ll = float(-0.5 * y @ a - 0.5 * logdet - 0.5 * n * LOG2PI)
    g = []
    for D in dK + [np.eye(n)]:
        g.append(0.5 * (a @ D @ a) - 0.5 * np.sum(Cinv * D))
    return ll, np.array(g)


def predict(spec, theta, t, y, t_star):
    """Latent posterior mean and variance at new times (Eq. mean2 and the
    variance formula of Sec. 2.2): K(t*, t) C^-1 y and k(0) - K(t*, t) C^-1 K(t, t*)."""
    t = np.asarray(t, dtype=np.float64)
    y = np.asarray(y, dtype=np.float64)
    t_star = np.asarray(t_star, dtype=np.float64)
    _, _, _, cf = _factor(spec, theta, t)
    Ks, _ = kernel(spec, theta, t_star[:, None] - t[None, :])
    k0, _ = kernel(spec, theta, np.zeros(1))
    a = cho_solve(cf, y)
    V = solve_triangular(cf[0], Ks.T, lower=True)
    return Ks @ a, k0[0] - np.sum(V * V, axis=0)
