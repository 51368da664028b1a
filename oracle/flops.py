"""A counted restatement of the sequential method: its FP64 operations per
time step, for the roofline's algorithmic flop count.

TEST INFRASTRUCTURE ONLY (see the package docstring): the script
``python -m oracle.flops`` prints the counts that the benchmark and the
design notes quote; nothing on the product path imports it.

What is counted.  The work of one log-likelihood + gradient evaluation by the
work-efficient sequential method, per time step, written as dense b x b
linear algebra in the paper's coordinates (no structure of A, H or Pinf is
exploited):

* forward, a covariance-form Kalman filter: the prediction m^ = A m,
  P^ = A (P - Pinf) A^T + Pinf (the same matrix as A P A^T + Q_n with
  Q_n = Pinf - A Pinf A^T, Sec. 2.1), the innovation v = y - h^T m^ with
  variance S = h^T P^ h + s_n, the gain k = P^ h / S, the update, and the
  prediction-error term -1/2 (v^2 / S + log 2 pi S) of the log-likelihood
  (Eq. ml2 through the determinant lemma, Eq. det_1);
* backward, the inversion-free adjoint (modified Bryson-Frazier) that carries
  l^ = -d ll / d m^ and L^ from step to step:
  alpha = v / S + k^T l^, c = 1/S + k^T L^ k, l~ = l^ - alpha h,
  L~ = (I - k h^T)^T L^ (I - k h^T) + h h^T / S, then
  G = (l~ l~^T - L~) / 2 = d ll / d P^, and l^ <- A^T l~, L^ <- A^T L~ A;
* the gradient (Sec. 2.4, Eq. dd1 evaluated per step): d ll / d A_n =
  -l~ m_{n-1}^T + 2 G A (P_{n-1} - Pinf) contracted with d A_n / d theta_p
  for every parameter on which A depends; the direct Pinf term
  G - A^T G A = G - (l^ l^T - L^) / 2 summed over the steps and contracted
  with d Pinf / d theta_p once at the end; and the noise term
  (alpha^2 - c) / 2.

The discretisation (A_n and d A_n / d theta from the closed forms) is not
counted: it is model-specific, and the inputs here come from the oracle's
``seq.discretize``.  Costs: a product of (m x k) and (k x n) matrices is
m n (2k - 1) flops, an element-wise operation on m x n entries is m n, an
inner product of m x n entries is 2 m n - 1; a reciprocal or a log is 1.

The restatement computes the log-likelihood and gradient itself, and the
tests pin it to the oracle's two-filter values on the same series: a count
of a computation that does not reproduce the method would fail there.
"""
import numpy as np

from . import n_params, seq, state_dim


class Count:
    """Dense operations that add their flop count to ``flops``."""

    def __init__(self):
        self.flops = 0

    def mm(self, A, B):
        A, B = np.atleast_2d(A), np.atleast_2d(B)
        m, k = A.shape
        n = B.shape[1]
        self.flops += m * n * (2 * k - 1)
        return A @ B

    def mv(self, A, x):
        m, k = A.shape
        self.flops += m * (2 * k - 1)
        return A @ x

    def dot(self, x, y):
        self.flops += 2 * x.size - 1
        return float(np.sum(x * y))

    def ew(self, z, nops=1):
        """an element-wise result of nops operations per entry"""
        self.flops += nops * np.size(z)
        return z

    def scalar(self, v, nops=1):
        self.flops += nops
        return v


def grad_counted(spec, theta, t, y):
    """Log-likelihood, gradient (every entry of theta) and the flop count of
    the recursion described in the module docstring, for one series."""
    theta = np.asarray(theta, dtype=np.float64)
    t = np.asarray(t, dtype=np.float64)
    y = np.asarray(y, dtype=np.float64)
    n, b, P = len(t), state_dim(spec), n_params(spec)
    s_n = theta[-1]
    _, _, h, _ = seq.continuous(spec, theta)
    mats = [seq.discretize(spec, theta, t[i] - t[i - 1]) if i > 0 else None for i in range(n)]
    d0 = seq.discretize(spec, theta, 0.0)
    Pinf, dPinf = d0["Pinf"], d0["dPinf"]
    c = Count()
    # ---- forward
    m, Pm = np.zeros(b), None
    st = []
    ll = 0.0
    for i in range(n):
        D = None
        if i == 0:
            mb, Pb = np.zeros(b), Pinf.copy()
        else:
            A = mats[i]["A"]
            mb = c.mv(A, m)
            D = c.ew(Pm - Pinf)              # kept for the gradient's d ll / d A
            Pb = c.ew(c.mm(c.mm(A, D), A.T) + Pinf)
        p = c.mv(Pb, h)
        S = c.scalar(c.dot(h, p) + s_n)
        v = c.scalar(y[i] - c.dot(h, mb))
        rS = c.scalar(1.0 / S)
        k = c.ew(p * rS)
        st.append((mb, v, rS, k, m, D))
        m = c.ew(mb + k * v, 2)
        Pm = c.ew(Pb - np.outer(k, p), 2)
        ll += c.scalar(-0.5 * (v * v * rS + np.log(2.0 * np.pi * S)), 5)
    # ---- backward
    depends = [p for p in range(P) if any(np.any(mats[i]["dA"][p] != 0.0) for i in range(1, n))]
    g = np.zeros(P)
    gpinf = np.zeros((b, b))
    lh, Lh = np.zeros(b), np.zeros((b, b))
    gnoise = 0.0
    for i in range(n - 1, -1, -1):
        mb, v, rS, k, m_prev, D = st[i]
        al = c.scalar(v * rS + c.dot(k, lh), 2)
        u = c.mv(Lh, k)
        cc = c.scalar(rS + c.dot(k, u))
        lt = c.ew(lh - al * h, 2)
        ub = c.ew(u - c.scalar(0.5 * cc) * h, 2)
        Lt = c.ew(Lh - np.outer(h, ub) - np.outer(ub, h), 4)
        G = c.ew(0.5 * (np.outer(lt, lt) - Lt), 3)
        gnoise += c.scalar(al * al - cc, 3)
        if i > 0:
            A = mats[i]["A"]
            Abar = c.ew(-np.outer(lt, m_prev) + 2.0 * c.mm(c.mm(G, A), D), 3)
            for p in depends:
                g[p] += c.scalar(c.dot(Abar, mats[i]["dA"][p]), 1)
            lh = c.mv(A.T, lt)
            Lh = c.mm(c.mm(A.T, Lt), A)
            gpinf += c.ew(G - 0.5 * (np.outer(lh, lh) - Lh), 5)
        else:
            gpinf += c.ew(G)
    for p in range(P - 1):
        g[p] += c.dot(gpinf, dPinf[p])
    g[P - 1] += 0.5 * gnoise
    return ll, g, c.flops


def flops_per_step(spec, theta, t, y, n1=64, n2=320):
    """Flops per step: the difference of two counted runs over the first n1
    and n2 steps, divided by n2 - n1 (the first step and the final
    contractions are counted once per series, not per step)."""
    _, _, f1 = grad_counted(spec, theta, t[:n1], y[:n1])
    _, _, f2 = grad_counted(spec, theta, t[:n2], y[:n2])
    return (f2 - f1) / float(n2 - n1)


MODELS = {
    "b=2 matern32": ("matern32", [1.0, 1.0, 0.1]),
    "b=3 matern52": ("matern52", [0.5, 2.0, 0.05]),
    "b=12 matern32 + eq(10)": (["matern32", ("eq", 10)], [1.0, 1.0, 1.0, 1.0, 0.1]),
    "b=16 matern32 + quasiperiodic(6, matern12)": (["matern32", ("quasiperiodic", 6, "matern12")],
                                                   [1.0, 1.0, 1.0, 1.0, 1.0, 10.0, 0.01]),
}


def main():
    rng = np.random.default_rng(0)
    t = np.cumsum(rng.exponential(0.01, 400))
    y = np.sin(7.0 * t) + 0.3 * rng.standard_normal(400)
    for name, (spec, theta) in MODELS.items():
        print("%-46s %9.1f flop/step" % (name, flops_per_step(spec, theta, t, y)))


if __name__ == "__main__":
    main()
