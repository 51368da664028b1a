"""Explicit block matrices of the sparse-precision formulation (Sec. 2.1-2.3).

TEST INFRASTRUCTURE ONLY (see the package docstring).

For N states of dimension b (one per observation) this assembles, densely:

* the stacked transition matrix bold-A (Sec. 2.1): identity blocks on the
  diagonal and A[t_i - t_j] = A_{i-1} ... A_j below it;
* bold-Q = blockdiag(P0, Q_0, ..., Q_{N-2})  (Eq. q_matrix);
* the state covariance  Kc = bold-A bold-Q bold-A^T  (Eq. k1);
* its inverse from the factors, bold-A^-T bold-Q^-1 bold-A^-1 (Eq. hh1), with
  bold-A^-1 block-bidiagonal (I on the diagonal, -A_i below it);
* G = I_N (x) H and the posterior precision K~ = Kc^-1 + G^T Sigma^-1 G
  (Sec. 2.2, the block-diagonal data term sigma_n^-2 (I_N (x) H^T H)).

Only for small N and well-conditioned gaps: forming Q^-1 explicitly is the
literal form whose conditioning degrades like (lam dt)^-(2b-2).
"""
import numpy as np

from . import seq, state_dim


def transitions(spec, theta, t):
    """A_i and Q_i for the gaps t[i+1]-t[i], and Pinf."""
    t = np.asarray(t, dtype=np.float64)
    As, Qs = [], []
    Pinf = None
    for i in range(len(t) - 1):
        d = seq.discretize(spec, theta, t[i + 1] - t[i])
        As.append(d["A"]); Qs.append(d["Q"]); Pinf = d["Pinf"]
    if Pinf is None:
        Pinf = seq.discretize(spec, theta, 0.0)["Pinf"]
    return As, Qs, Pinf


def stacked(spec, theta, t):
    """Return dict(bA, bQ, Kc, bAinv, Kinv, G, Ktilde) as dense arrays
    (Kinv and Ktilde are None when some Q block is singular)."""
    b = state_dim(spec)
    n = len(t)
    As, Qs, Pinf = transitions(spec, theta, t)
    _, _, H, _ = seq.continuous(spec, theta)
    s2 = float(theta[-1])
    N = n * b
    bA = np.zeros((N, N))
    for j in range(n):
        blk = np.eye(b)
        bA[j * b:(j + 1) * b, j * b:(j + 1) * b] = blk
        for i in range(j + 1, n):
            blk = As[i - 1] @ blk
            bA[i * b:(i + 1) * b, j * b:(j + 1) * b] = blk
    bQ = np.zeros((N, N))
    bQ[:b, :b] = Pinf
    for i in range(1, n):
        bQ[i * b:(i + 1) * b, i * b:(i + 1) * b] = Qs[i - 1]
    Kc = bA @ bQ @ bA.T
    bAinv = np.eye(N)
    for i in range(1, n):
        bAinv[i * b:(i + 1) * b, (i - 1) * b:i * b] = -As[i - 1]
    G = np.kron(np.eye(n), H[None, :])
    # Q^-1 exists only when every Q block is non-singular; a noiseless
    # component (the pure periodic family) has Q = 0 and no precision form.
    Qinv = np.zeros((N, N))
    Kinv = Ktilde = None
    try:
        for i in range(n):
            sl = slice(i * b, (i + 1) * b)
            if np.linalg.matrix_rank(bQ[sl, sl]) < b:
                raise np.linalg.LinAlgError("singular Q block")
            Qinv[sl, sl] = np.linalg.inv(bQ[sl, sl])
        Kinv = bAinv.T @ Qinv @ bAinv
        Ktilde = Kinv + G.T @ G / s2
    except np.linalg.LinAlgError:
        pass
    return dict(bA=bA, bQ=bQ, Kc=Kc, bAinv=bAinv, Kinv=Kinv, G=G, Ktilde=Ktilde, H=H)


def block(M, b, i, j):
    return M[i * b:(i + 1) * b, j * b:(j + 1) * b]


def blocks_of(M, b):
    """Diagonal blocks D[i] = M[i,i] and sub-diagonal blocks O[i] = M[i+1,i]
    of a dense block-tridiagonal matrix."""
    n = M.shape[0] // b
    D = np.array([block(M, b, i, i) for i in range(n)])
    O = np.array([block(M, b, i + 1, i) for i in range(n - 1)]).reshape(max(n - 1, 0), b, b)
    return D, O


def thomas(D, O, r):
    """The sequential block algorithm for a symmetric positive-definite BTD
    matrix T (diagonal blocks D[i], sub-diagonal blocks O[i] = T[i+1, i]):
    block LDL^T (Sec. 3.1's Thomas algorithm, subproblems 1 and 3) and the
    selected inverse (subproblems 2 and 4) by the backward recursion of the
    same factors.

    Returns (logdet, x = T^-1 r, S_diag[i] = (T^-1)[i,i], S_off[i] = (T^-1)[i+1,i]).
    """
    D = np.asarray(D, dtype=np.float64)
    O = np.asarray(O, dtype=np.float64)
    r = np.asarray(r, dtype=np.float64)
    n, b, _ = D.shape
    S = np.empty_like(D)          # Schur complements (the pivots)
    L = np.empty_like(O)          # L[i] = O[i] S[i]^-1
    z = np.empty_like(r)
    logdet = 0.0
    for i in range(n):
        Si = D[i].copy()
        zi = r[i].copy()
        if i > 0:
            Si -= L[i - 1] @ O[i - 1].T
            zi -= L[i - 1] @ z[i - 1]
        S[i] = Si
        z[i] = zi
        logdet += np.linalg.slogdet(Si)[1]
        if i + 1 < n:
            L[i] = np.linalg.solve(Si.T, O[i].T).T
    x = np.empty_like(r)
    Sd = np.empty_like(D)
    So = np.empty_like(O)
    for i in range(n - 1, -1, -1):
        Sinv = np.linalg.inv(S[i])
        if i == n - 1:
            x[i] = Sinv @ z[i]
            Sd[i] = Sinv
        else:
            x[i] = Sinv @ z[i] - L[i].T @ x[i + 1]
            So[i] = -Sd[i + 1] @ L[i]                      # (T^-1)[i+1, i]
            Sd[i] = Sinv + L[i].T @ Sd[i + 1] @ L[i]
        Sd[i] = 0.5 * (Sd[i] + Sd[i].T)
    return logdet, x, Sd, So


def dense_of(D, O):
    """The dense symmetric matrix with diagonal blocks D[i] and sub-diagonal
    blocks O[i] = T[i+1, i] (T[i, i+1] = O[i]^T)."""
    D = np.asarray(D, dtype=np.float64)
    O = np.asarray(O, dtype=np.float64)
    n, b, _ = D.shape
    T = np.zeros((n * b, n * b))
    for i in range(n):
        T[i * b:(i + 1) * b, i * b:(i + 1) * b] = D[i]
        if i + 1 < n:
            T[(i + 1) * b:(i + 2) * b, i * b:(i + 1) * b] = O[i]
            T[i * b:(i + 1) * b, (i + 1) * b:(i + 2) * b] = O[i].T
    return T


def diag_product(D, O, Xd, Xo):
    """Subproblem 4 (Sec. 3.1, Eq. comp_2) by its definition: the diagonal of
    T^-1 X for a symmetric BTD matrix T (D, O) and a symmetric BTD right-hand
    side X (Xd, Xo), with the dense inverse (small n only).  Returns
    (diag as (n, b), trace)."""
    T = dense_of(D, O)
    X = dense_of(Xd, Xo)
    d = np.diag(np.linalg.solve(T, X)).copy()
    n, b = np.asarray(D).shape[:2]
    return d.reshape(n, b), float(np.sum(d))
