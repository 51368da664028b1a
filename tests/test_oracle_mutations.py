"""Plant plausible mistakes in copies of the oracle and check that the pins in
test_oracle_pins catch every one of them.  CPU only: a mutant of the C oracle
is a text-substituted copy of seq.c compiled into a temporary directory and
swapped in for the duration of one test; the committed oracle is untouched."""
import os
import subprocess

import numpy as np
import pytest

from oracle import dense, seq
import test_oracle_pins as pins

SEQ_SRC = os.path.join(os.path.dirname(seq.__file__), "seq.c")

# (name, original text, mutated text) -- each original must occur exactly once
C_MUTANTS = [
    ("loglik drops 1/S", "acc += -0.5 * (log(2.0 * M_PI * S) + v * v / S);",
     "acc += -0.5 * (log(2.0 * M_PI * S) + v * v);"),
    ("Pinf(5/2) sign", "Pu[2] = Pu[6] = -l2 / 3.0;", "Pu[2] = Pu[6] = l2 / 3.0;"),
    ("Van Loan block misplaced", "M[i * m + (j + b)] = Fl[i * b + j] * dt;",
     "M[(i + b) * m + j] = Fl[i * b + j] * dt;"),
    ("Q misses A^T", "for (int i = 0; i < b * b; ++i) Q[i] = Pinf[i] - U[i];",
     "for (int i = 0; i < b * b; ++i) Q[i] = Pinf[i] - T[i];"),
    ("adjoint sign", "Qbar[i * b + j] = 0.5 * (v[i] * v[j] - WJ[i * b + j]);",
     "Qbar[i * b + j] = 0.5 * (v[i] * v[j] + WJ[i * b + j]);"),
    ("cross-covariance operands swapped", "mm(b, Psn, Gt, Pc + (size_t)i * b * b);",
     "mm(b, Gt, Psn, Pc + (size_t)i * b * b);"),
    ("rotation transposed", "double R[4] = {cs, -sn, sn, cs};", "double R[4] = {cs, sn, -sn, cs};"),
    ("gradient drops dQ term",
     "double term = mdot(b, Abar, dA + (size_t)p * b * b) + mdot(b, Qbar, dQ + (size_t)p * b * b);",
     "double term = mdot(b, Abar, dA + (size_t)p * b * b);"),
    ("Bessel series index", "term *= h * h / ((double)k * (double)(k + j));",
     "term *= h * h / ((double)k * (double)(k + j + 1));"),
    ("RTS gain transposed", "for (int r = 0; r < b; ++r) for (int c = 0; c < b; ++c) G[r * b + c] = Gt[c * b + r];",
     "for (int r = 0; r < b; ++r) for (int c = 0; c < b; ++c) G[r * b + c] = Gt[r * b + c];"),
    ("EQ noise intensity drops sqrt(2 pi)", "rhs[(N - 1) * N + (N - 1)] = -sqrt(2.0 * M_PI) * pow(2.0, N) * fact;",
     "rhs[(N - 1) * N + (N - 1)] = -pow(2.0, N) * fact;"),
    ("EQ time-scaling exponent", "F[(N - 1) * N + k] = -a1[k] * pow(ell, k - N);",
     "F[(N - 1) * N + k] = -a1[k] * pow(ell, k - N + 1);"),
    ("first-step prior dropped", "memset(mb, 0, sizeof(double) * b); mcopy(b, Pinf, Pb); }",
     "memset(mb, 0, sizeof(double) * b); meye(b, Pb); }"),
]


def _quick_suite():
    """A subset of the pins, small sizes; returns the names of those that fail."""
    checks = []
    for spec, th in pins.ALL:
        checks.append(("lyapunov", lambda s=spec, t=th: pins.test_lyapunov(s, t)))
        checks.append(("pade", lambda s=spec, t=th: pins.test_expm_against_pade(s, t, 0.37)))
        checks.append(("dderiv", lambda s=spec, t=th: pins.test_discretisation_derivatives(s, t)))
        checks.append(("sscov", lambda s=spec, t=th: pins.test_state_space_covariance_equals_kernel(s, t)))
        checks.append(("selinv", lambda s=spec, t=th: pins.test_selected_inverse_equals_rts(s, t)))
        checks.append(("dense", lambda s=spec, t=th: pins.test_dense_equals_sequential(s, t, 0)))
        checks.append(("single", lambda s=spec, t=th: pins.test_single_point(s, t)))
    failed = []
    for name, fn in checks:
        try:
            fn()
        except Exception:  # an assertion or an oracle error both count as caught
            failed.append(name)
    return failed


def test_unmutated_oracle_passes_quick_suite():
    assert _quick_suite() == []


@pytest.mark.parametrize("name,old,new", C_MUTANTS, ids=[m[0] for m in C_MUTANTS])
def test_c_mutant_is_caught(name, old, new, tmp_path, monkeypatch):
    src = open(SEQ_SRC).read()
    assert src.count(old) == 1, "mutation site not unique: " + name
    path = tmp_path / "mut.c"
    path.write_text(src.replace(old, new))
    so = tmp_path / "libmut.so"
    subprocess.run(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-ffp-contract=off",
                    "-o", str(so), str(path), "-lm"], check=True)
    monkeypatch.setattr(seq, "_lib", seq.bind(str(so)))
    assert _quick_suite() != [], "no pin caught: " + name


def test_dense_mutant_is_caught(monkeypatch):
    """Matern-5/2 with r^2/2 in place of r^2/3 in the closed form."""
    orig = dense._matern

    def bad(b, ell, var, tau):
        k, dk, base = orig(b, ell, var, tau)
        if b == 3:
            r = np.sqrt(5.0) * np.abs(tau) / ell
            base = (1.0 + r + r * r / 2.0) * np.exp(-r)
            k = var * base
        return k, dk, base

    monkeypatch.setattr(dense, "_matern", bad)
    assert _quick_suite() != []


def test_dense_gradient_mutant_is_caught(monkeypatch):
    """The gradient trace term with the wrong sign."""
    orig = dense.grad

    def bad(spec, theta, t, y):
        ll, g = orig(spec, theta, t, y)
        _, _, C, cf = dense._factor(spec, theta, t)
        n = len(y)
        Cinv = np.linalg.inv(C)
        return ll, g + np.array([np.sum(Cinv * D) for D in dense.gram(spec, theta, t)[1] + [np.eye(n)]])

    monkeypatch.setattr(dense, "grad", bad)
    assert _quick_suite() != []


# Python-level mutants of the optimiser (oracle/scg.py): text-substituted
# copies loaded as a module; each must fail one of the SCG pins.
# (A wrong sign of beta's r'.r term is not in the list: no convergence
# property separates it -- on a quadratic r'.r vanishes, and on Rosenbrock it
# converges in 87 iterations against 100.)
SCG_MUTANTS = [
    ("no conjugacy (beta = 0)", "beta = (rn @ rn - rn @ r) / mu", "beta = 0.0"),
    ("no lambda scaling of delta", "delta = delta + (lam - lambar) * pp", "delta = delta"),
    ("comparison ratio sign", "Delta = 2.0 * delta * (f - fn) / (mu * mu)", "Delta = 2.0 * delta * (fn - f) / (mu * mu)"),
    ("curvature from the wrong side", "s = (np.asarray(gs) - g) / sigma", "s = (g - np.asarray(gs)) / sigma"),
]


@pytest.mark.parametrize("name,old,new", SCG_MUTANTS)
def test_scg_mutant_is_caught(name, old, new, tmp_path):
    import importlib.util
    from oracle import scg
    import test_oracle_scg as scg_pins
    src = open(scg.__file__).read()
    assert src.count(old) == 1, name
    path = tmp_path / "scg_mutant.py"
    path.write_text(src.replace(old, new))
    spec = importlib.util.spec_from_file_location("scg_mutant", path)
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    caught = False
    saved = scg_pins.scg
    scg_pins.scg = mod
    try:
        for fn in (scg_pins.test_quadratic_reaches_the_minimiser, scg_pins.test_rosenbrock,
                   scg_pins.test_rejected_trial_points_do_not_move):
            try:
                fn()
            except Exception:
                caught = True
    finally:
        scg_pins.scg = saved
    assert caught, name
