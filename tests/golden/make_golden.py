"""Write the stored expected values under tests/golden/ (calls only oracle/).

config1_matern32_n1000.txt: the plain-method workload -- Matern-3/2 (b=2),
N=1000 sorted times with dt ~ Exponential(mean 0.1), lengthscale 1.0,
signal variance 1.0, noise variance 0.1, y sampled from the state-space model
(seed 0).  The paper prints no numbers for any workload (its timing and
forecast figures are images), so every value here is the oracle's: columns
t, y, posterior mean, latent variance, and a header with the log-likelihood
and the gradient (lengthscale, signal variance, noise variance).

Run from the repository root:  python tests/golden/make_golden.py
"""
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

from oracle import dense, seq  # noqa: E402

SPEC = "matern32"
THETA = np.array([1.0, 1.0, 0.1])


def config1_inputs():
    rng = np.random.default_rng(0)
    d = rng.exponential(0.1, 1000)
    d[0] = 0.0
    t = np.cumsum(d)
    eps = rng.standard_normal((1000, 3))
    y = seq.sample(SPEC, THETA, t, eps)
    return t, y


def main():
    t, y = config1_inputs()
    ll, g = seq.grad(SPEC, THETA, t, y)
    lld, gd = dense.grad(SPEC, THETA, t, y)
    assert abs(ll - lld) <= 1e-12 * abs(ll) and np.all(np.abs(g - gd) <= 1e-10 * np.abs(gd))
    sm = seq.smoother(SPEC, THETA, t, y)
    path = os.path.join(HERE, "config1_matern32_n1000.txt")
    with open(path, "w") as f:
        f.write("# Matern-3/2, N=1000, dt~Exp(0.1), theta=(1.0, 1.0, 0.1), y from the SS model (seed 0)\n")
        f.write("# written by tests/golden/make_golden.py from the oracle (the paper prints no values)\n")
        f.write("# loglik %.17g\n" % ll)
        f.write("# grad %.17g %.17g %.17g\n" % tuple(g))
        f.write("# columns: t y mean var\n")
        for row in zip(t, y, sm["mean"], sm["var"]):
            f.write("%.17g %.17g %.17g %.17g\n" % row)
    print("wrote", path)


def load_config1():
    path = os.path.join(HERE, "config1_matern32_n1000.txt")
    ll = g = None
    with open(path) as f:
        for line in f:
            if line.startswith("# loglik"):
                ll = float(line.split()[2])
            elif line.startswith("# grad"):
                g = np.array([float(v) for v in line.split()[2:]])
    data = np.loadtxt(path)
    return dict(spec=SPEC, theta=THETA.copy(), t=data[:, 0], y=data[:, 1], mean=data[:, 2], var=data[:, 3],
                ll=ll, grad=g)


if __name__ == "__main__":
    main()
