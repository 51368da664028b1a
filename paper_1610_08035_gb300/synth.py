"""Seeded synthetic inputs for the temporal-GP workloads.

This module draws times, observations and hyperparameters only; it holds none
of the inference arithmetic, and both the library's tests and the oracle's
tests take their inputs from it.

Recipe (the shapes and distributions of the paper's simulated workload,
Sec. 4.2, "two sinusoids immersed into Gaussian noise"):

* times: t_0 = 0, t_{i+1} = t_i + dt_i with dt_i ~ Exponential(mean_dt)
  (PCG64, ``numpy.random.default_rng(seed)``), summed in FP64;
* observations: y_i = sqrt(s_f) (0.9 sin(2 pi t_i / p_1 + phi_1)
  + 0.45 sin(2 pi t_i / p_2 + phi_2)) + sqrt(s_n) e_i with e_i ~ N(0, 1),
  periods p_1 = 7.3 l and p_2 = 2.9 l tied to the lengthscale l of the
  workload and random phases, so the signal varies on the kernel's scale;
* batches: lengths round(exp(U(log lo, log hi))), per-series lengthscale,
  signal and noise variance log-uniform on the stated ranges;
* well-separated times (for the method as written, which forms Q^-1):
  dt_i ~ Uniform(lo, hi) times the lengthscale;
* general block-tridiagonal inputs: T = B B^T + ridge I for a random lower
  block-bidiagonal B (diagonal blocks N(0, 1) + 2 I, sub-diagonal blocks
  N(0, 1)), returned as its blocks without forming T;
* a series shaped like the paper's CO2 experiment (Sec. 4.3), with no data
  from it: a regular weekly grid of 2195 points in years (t_i = i / 52.1775),
  a slowly rising smooth trend, an annual cycle with its first overtone whose
  amplitude drifts slowly, and Gaussian noise, centred and scaled to unit
  variance.
"""
from dataclasses import dataclass, field

import numpy as np


def exp_times(n, mean_dt, rng):
    d = rng.exponential(mean_dt, n)
    d[0] = 0.0
    return np.cumsum(d)


def two_sinusoids(t, ell, sf2, sn2, rng):
    ph = rng.uniform(0.0, 2.0 * np.pi, 2)
    sig = 0.9 * np.sin(2.0 * np.pi * t / (7.3 * ell) + ph[0]) + 0.45 * np.sin(2.0 * np.pi * t / (2.9 * ell) + ph[1])
    return np.sqrt(sf2) * sig + np.sqrt(sn2) * rng.standard_normal(len(t))


def log_uniform(lo, hi, size, rng):
    return np.exp(rng.uniform(np.log(lo), np.log(hi), size))


@dataclass
class Series:
    """One workload: model spec, hyperparameters, times and observations."""
    name: str
    spec: list
    theta: np.ndarray
    t: np.ndarray
    y: np.ndarray
    extra: dict = field(default_factory=dict)


# name: (spec, theta, n, mean_dt, seed); theta = per-component parameters then the noise variance
SINGLE = {
    # Matern-3/2, b=2, N=1000, dt ~ Exp(0.1), l=1, s_f=1, s_n=0.1
    "matern32_n1000": (["matern32"], [1.0, 1.0, 0.1], 1000, 0.1, 0),
    # Matern-5/2, b=3, N=2^22, dt ~ Exp(0.01), l=0.5, s_f=2, s_n=0.05
    "matern52_n4m": (["matern52"], [0.5, 2.0, 0.05], 1 << 22, 0.01, 1),
    # Matern-3/2 + quasi-periodic (order 6, Matern-1/2 envelope), b=16, N=2^20
    "sum_qp_n1m": (["matern32", ("quasiperiodic", 6, "matern12")],
                   [1.0, 1.0, 1.0, 1.0, 1.0, 10.0, 0.01], 1 << 20, 0.01, 2),
    # Matern-3/2, b=2, N=2^26, dt ~ Exp(0.001), l=0.05, s_f=1, s_n=0.1
    "matern32_n64m": (["matern32"], [0.05, 1.0, 0.1], 1 << 26, 0.001, 4),
    # the paper's timing model (Sec. 4.2): Matern-3/2 + EQ of order 10, b=12,
    # N=2^20, dt ~ Exp(0.01); Matern l=1, s=1; EQ l=0.5, s=1; s_n=0.1
    "m32_eq10_n1m": (["matern32", ("eq", 10)], [1.0, 1.0, 0.5, 1.0, 0.1], 1 << 20, 0.01, 5),
}


def single(name, n=None, seed=None):
    """A single-series workload; ``n`` and ``seed`` override the defaults."""
    spec, theta, n0, mean_dt, seed0 = SINGLE[name]
    n = n0 if n is None else int(n)
    rng = np.random.default_rng(seed0 if seed is None else seed)
    t = exp_times(n, mean_dt, rng)
    y = two_sinusoids(t, theta[0], theta[1], theta[-1], rng)
    return Series(name, spec, np.array(theta, dtype=np.float64), t, y)


def batched(n_series=4096, lo=256, hi=65536, mean_dt=0.01, seed=3, spec="matern52"):
    """Independent series of log-uniform lengths, concatenated.

    Returns a Series whose t and y are the concatenation, with
    extra = dict(offsets=int64[B+1], thetas=float64[B, 3]) and theta = thetas
    flattened row-major (per series: lengthscale, s_f, s_n)."""
    rng = np.random.default_rng(seed)
    lengths = np.rint(np.exp(rng.uniform(np.log(lo), np.log(hi), n_series))).astype(np.int64)
    ell = log_uniform(0.1, 10.0, n_series, rng)
    sf2 = log_uniform(0.5, 2.0, n_series, rng)
    sn2 = log_uniform(0.01, 0.5, n_series, rng)
    offsets = np.zeros(n_series + 1, dtype=np.int64)
    offsets[1:] = np.cumsum(lengths)
    t = np.empty(offsets[-1])
    y = np.empty(offsets[-1])
    for i in range(n_series):
        a, b = offsets[i], offsets[i + 1]
        ti = exp_times(b - a, mean_dt, rng)
        t[a:b] = ti
        y[a:b] = two_sinusoids(ti, ell[i], sf2[i], sn2[i], rng)
    thetas = np.stack([ell, sf2, sn2], axis=1)
    return Series("batched_%d" % n_series, [spec], thetas.reshape(-1).copy(), t, y,
                  extra=dict(offsets=offsets, thetas=thetas))


def separated_times(n, ell, rng, lo=0.3, hi=0.6):
    d = rng.uniform(lo * ell, hi * ell, n)
    d[0] = 0.0
    return np.cumsum(d)


def random_spd_btd(n, b, seed, ridge=0.1):
    """Blocks of a random symmetric positive-definite block-tridiagonal
    matrix T = B B^T + ridge I: D (n, b, b) with D[i] = T[i, i], O (n-1, b, b)
    with O[i] = T[i+1, i], and a right-hand side r (n, b)."""
    rng = np.random.default_rng(seed)
    Bd = rng.standard_normal((n, b, b)) + 2.0 * np.eye(b)
    Bs = rng.standard_normal((max(n - 1, 0), b, b))     # B[i+1, i]
    D = Bd @ np.transpose(Bd, (0, 2, 1)) + ridge * np.eye(b)
    D[1:] += Bs @ np.transpose(Bs, (0, 2, 1))
    O = Bs @ np.transpose(Bd[:-1], (0, 2, 1))            # B[i+1,i] B[i,i]^T
    r = rng.standard_normal((n, b))
    return D, O, r


def co2_shaped(seed=6, n=2195):
    """A weekly series of the CO2 experiment's shape (Sec. 4.3) with the
    structured model of the b = 16 workload (Matern-3/2 for the trend,
    quasi-periodic of order 6 with a Matern-1/2 envelope for the cycle) and
    a starting theta for fitting: (l_m32, s_m32, s_per, l_per, period,
    l_env, s_n)."""
    rng = np.random.default_rng(seed)
    t = np.arange(n, dtype=np.float64) / 52.1775
    u = t / t[-1]
    trend = 3.0 * u + 1.5 * u * u + 0.3 * np.sin(2.0 * np.pi * t / 9.5 + rng.uniform(0.0, 2.0 * np.pi))
    amp = 1.0 + 0.15 * np.sin(2.0 * np.pi * t / 13.0 + rng.uniform(0.0, 2.0 * np.pi))
    ph = rng.uniform(0.0, 2.0 * np.pi, 2)
    cycle = amp * (0.8 * np.sin(2.0 * np.pi * t + ph[0]) + 0.25 * np.sin(4.0 * np.pi * t + ph[1]))
    y = trend + cycle + 0.1 * rng.standard_normal(n)
    y = (y - y.mean()) / y.std()
    theta = np.array([5.0, 1.0, 0.5, 1.0, 1.0, 20.0, 0.05])
    return Series("co2_shaped", ["matern32", ("quasiperiodic", 6, "matern12")], theta, t, y)
