"""Deterministic and randomized TT-rounding (oracle; test infrastructure only).

Each routine restates one algorithm of the paper step by step:
  Algorithm 1  Right-to-Left Orthogonalization            orthogonalize_rl
  Algorithm 2  TT-Rounding (TT-SVD)                        tt_round_det
  Algorithm 3  Right-to-Left Partial Contractions          partial_contractions_rl
  (its left-to-right mirror, Section 3.3)                  partial_contractions_lr
  Algorithm 4  Orthogonalize-then-Randomize                round_orthrand
  Algorithm 5  Randomize-then-Orthogonalize                round_randorth
  Algorithm 6  Two-Sided-Randomization (gen. Nystrom)      round_twosided
  Algorithm 7  TT-Rounding of a Sum, Rand-then-Orth        round_sum_randorth
  Section 3.2  truncation of the left-orthogonal output    truncate_left_orthogonal

Readings where the paper is silent or inconsistent (listed with reasons in the
design notes of the repository):
  * SVD(X, eps) is used with an absolute threshold eps (Algorithm 2 computes
    eps = ||Y|| eps0 / sqrt(N-1) and passes it on); the kept rank is the
    smallest k >= 1 whose discarded tail sqrt(sum_{i>k} s_i^2) is <= eps.
  * Algorithm 2 keeps the first core produced by Algorithm 1 (its "X_1 = Y_1"
    would undo the update of core 1 made by the orthogonalization).
  * Algorithm 4 sketches Z_n = V(X_n), the core already updated by M_{n-1}.
  * Algorithm 7's last core uses M_{N-1}^{(j)}.
  * The next-core update of Algorithm 7 concatenates the blocks
    M^{(j)} Y^{(j)}_{n+1}(:, i, :) slice by slice.
  * Truncation of the left-orthogonal Randomize-then-Orthogonalize output
    (Section 3.2) sweeps right to left (the mirror of Algorithm 2's loop),
    which is the direction in which the left-orthogonal cores already play the
    role of the orthogonalized part.
  * Sigma^dagger in Algorithm 6 drops singular values <= max(l, rho) * 2^-52 * s_1.
"""
from __future__ import annotations

import numpy as np

from .tt import H, V, from_H, from_V, block_sum, ranks_of


def clamp_ranks(dims, ells):
    """Target ranks that a thin QR can deliver: l_0 = l_N = 1 and
    l_n <= min(l_{n-1} I_n, I_{n+1} l_{n+1}) (Section 2.1 thin QR needs m >= n)."""
    N = len(dims)
    ell = [1] + [int(x) for x in ells[1:N]] + [1]
    for n in range(1, N):
        ell[n] = min(ell[n], ell[n - 1] * dims[n - 1])
    for n in range(N - 1, 0, -1):
        ell[n] = min(ell[n], ell[n + 1] * dims[n])
    return ell


def svd_truncated(R, eps=0.0, max_rank=None):
    """[U_k, S_k, V_k] = SVD(R, eps) of Section 2.1 with an absolute threshold:
    the smallest k >= 1 with sqrt(sum_{i>k} s_i^2) <= eps, capped by max_rank."""
    U, s, Vt = np.linalg.svd(R, full_matrices=False)
    tail = np.sqrt(np.concatenate([np.cumsum((s * s)[::-1])[::-1], [0.0]]))
    k = len(s)
    if eps > 0:
        k = next(i for i in range(1, len(s) + 1) if tail[i] <= eps)
    if max_rank is not None:
        k = min(k, int(max_rank))
    k = max(k, 1)
    return U[:, :k], s[:k], Vt[:k, :], s


def qr_pos(A):
    """Thin QR with a nonnegative diagonal of R: for full column rank this is
    the unique thin QR factorization (Section 2.1 leaves the signs open; fixing
    them makes the basis of the orthogonalized right part, and therefore the
    sketch of Algorithm 4, independent of the QR routine)."""
    Q, R = np.linalg.qr(A)
    d = np.sign(np.diag(R))
    d[d == 0] = 1.0
    return Q * d[None, :], d[:, None] * R


def orthogonalize_rl(Y):
    """Algorithm 1: X right-orthogonal and equal to Y. For n = N..2: thin QR
    of H(X_n)^T, H(X_n) := Q^T, V(X_{n-1}) := V(Y_{n-1}) R^T (thin QR with a
    nonnegative diagonal of R, see qr_pos)."""
    X = [np.array(c, copy=True) for c in Y]
    N = len(X)
    for n in range(N, 1, -1):
        Xn = X[n - 1]
        Q, R = qr_pos(H(Xn).T)
        X[n - 1] = from_H(Q.T, Xn.shape[1])
        X[n - 2] = from_V(V(X[n - 2]) @ R.T, X[n - 2].shape[1])
    return X


def orthogonalize_lr(Y):
    """Left-to-right mirror of Algorithm 1 (Section 2.3: 'we can similarly obtain
    a left orthogonal tensor'): thin QR of V(X_n), V(X_n) := Q, H(X_{n+1}) := R H(X_{n+1})."""
    X = [np.array(c, copy=True) for c in Y]
    N = len(X)
    for n in range(1, N):
        Xn = X[n - 1]
        Q, R = np.linalg.qr(V(Xn))
        X[n - 1] = from_V(Q, Xn.shape[1])
        X[n] = from_H(R @ H(X[n]), X[n].shape[1])
    return X


def tt_round_det(Y, eps0=0.0, max_rank=None, return_sv=False):
    """Algorithm 2 (TT-Rounding): X = OrthogonalizeRL(Y); eps = ||Y|| eps0 /
    sqrt(N-1); for n = 1..N-1: [V(X_n), R] = QR(V(X_n)); [U, S, V] = SVD(R, eps);
    V(X_n) := V(X_n) U; H(X_{n+1}) := S V^T H(X_{n+1}).
    ||Y|| is the norm of the first core of the right-orthogonal X."""
    X = orthogonalize_rl(Y)
    N = len(X)
    nrm = float(np.linalg.norm(X[0]))
    eps = nrm / np.sqrt(max(N - 1, 1)) * eps0 if eps0 > 0 else 0.0
    svs = []
    for n in range(1, N):
        Xn = X[n - 1]
        Q, R = np.linalg.qr(V(Xn))
        U, s, Vt, s_all = svd_truncated(R, eps, max_rank)
        svs.append(s_all)
        X[n - 1] = from_V(Q @ U, Xn.shape[1])
        X[n] = from_H((s[:, None] * Vt) @ H(X[n]), X[n].shape[1])
    return (X, svs) if return_sv else X


def partial_contractions_rl(X, Y):
    """Algorithm 3: W_{N-1} = H(X_N) H(Y_N)^T; for n = N-1..2:
    V(Z_n) = V(X_n) W_n, W_{n-1} = H(Z_n) H(Y_n)^T.
    Returns W with W[n] = H(X_{n+1:N}) H(Y_{n+1:N})^T for n = 1..N-1 (bond
    index, paper numbering) and W[N] = [[1]]; W[0] is unused."""
    N = len(X)
    W = [None] * (N + 1)
    W[N] = np.ones((1, 1))
    W[N - 1] = H(X[N - 1]) @ H(Y[N - 1]).T
    for n in range(N - 1, 1, -1):
        Xn, Yn = X[n - 1], Y[n - 1]
        Z = from_V(V(Xn) @ W[n], Xn.shape[1])
        W[n - 1] = H(Z) @ H(Yn).T
    return W


def partial_contractions_lr(Y, L):
    """Left-to-right mirror of Algorithm 3 (used by Algorithm 6):
    W^L_n = V(L_{1:n})^T V(Y_{1:n}), computed as W^L_1 = V(L_1)^T V(Y_1) and
    W^L_n = V(L_n)^T V(T_n) with H(T_n) = W^L_{n-1} H(Y_n).
    Returns WL with WL[n] (l_n x R_n) for n = 1..N-1 and WL[0] = [[1]]."""
    N = len(Y)
    WL = [None] * (N + 1)
    WL[0] = np.ones((1, 1))
    for n in range(1, N):
        Yn, Ln = Y[n - 1], L[n - 1]
        T = from_H(WL[n - 1] @ H(Yn), Yn.shape[1])
        WL[n] = V(Ln).T @ V(T)
    return WL


def round_randorth(Y, R):
    """Algorithm 5 (Randomize-then-Orthogonalize) with the Gaussian TT sketch R
    (Definition 3.1) given: {W_n} = PartialContractionsRL(Y, R); X_1 = Y_1; for
    n = 1..N-1: Z_n = V(X_n); Y_n = Z_n W_n; [V(X_n), ~] = QR(Y_n);
    M_n = V(X_n)^T Z_n; H(X_{n+1}) = M_n H(Y_{n+1}). The result is left-orthogonal."""
    N = len(Y)
    W = partial_contractions_rl(Y, R)
    X = [None] * N
    Xn = np.array(Y[0], copy=True)
    for n in range(1, N):
        I = Xn.shape[1]
        Z = V(Xn)
        Ysk = Z @ W[n]
        Q, _ = np.linalg.qr(Ysk)
        X[n - 1] = from_V(Q, I)
        M = Q.T @ Z
        Xn = from_H(M @ H(Y[n]), Y[n].shape[1])
    X[N - 1] = Xn
    return X


def round_sum_randorth(Ys, R, coeffs=None):
    """Algorithm 7 (TT-Rounding of a Sum, Randomize-then-Orthogonalize). The
    block cores of the sum are never formed:
      W^{(j)} = PartialContractionsRL(Y^{(j)}, R) for every summand j;
      X_1 = [Y^{(1)}_1 ... Y^{(s)}_1];
      for n = 1..N-1: Z_n = V(X_n); Y_n = Z_n [W^{(1)}_n; ...; W^{(s)}_n];
        [V(X_n), ~] = QR(Y_n); [M^{(1)}_n ... M^{(s)}_n] = V(X_n)^T Z_n;
        if n < N-1: X_{n+1}(:, i, :) = [M^{(1)}_n Y^{(1)}_{n+1}(:, i, :) ... M^{(s)}_n Y^{(s)}_{n+1}(:, i, :)]
        else:       X_N = sum_j M^{(j)}_{N-1} Y^{(j)}_N.
    coeffs (optional) scale the summands (applied to their first cores)."""
    s = len(Ys)
    N = len(Ys[0])
    if coeffs is None:
        coeffs = [1.0] * s
    Ys = [[c * Y[0]] + list(Y[1:]) for c, Y in zip(coeffs, Ys)]
    W = [partial_contractions_rl(Y, R) for Y in Ys]
    X = [None] * N
    Xn = np.concatenate([Y[0] for Y in Ys], axis=2)
    if N == 1:
        return [sum(Y[0] for Y in Ys)]
    for n in range(1, N):
        I = Xn.shape[1]
        Z = V(Xn)
        Wstack = np.concatenate([W[j][n] for j in range(s)], axis=0)
        Ysk = Z @ Wstack
        Q, _ = np.linalg.qr(Ysk)
        X[n - 1] = from_V(Q, I)
        M = Q.T @ Z
        cols = np.cumsum([0] + [Y[n - 1].shape[2] for Y in Ys])
        Mj = [M[:, cols[j]:cols[j + 1]] for j in range(s)]
        Inext = Ys[0][n].shape[1]
        if n < N - 1:
            blocks = [from_H(Mj[j] @ H(Ys[j][n]), Inext) for j in range(s)]
            Xn = np.concatenate(blocks, axis=2)
        else:
            Xn = sum(from_H(Mj[j] @ H(Ys[j][N - 1]), Inext) for j in range(s))
    X[N - 1] = Xn
    return X


def round_sum_randorth_sharded(Ys_local, R, allreduce, coeffs=None):
    """Algorithm 7 with the summands spread over ranks (the block form of
    Section 3.4 makes this direct): a rank holds Ys_local (its summands and
    their coefficients). The partial contractions W^{(j)} and the projections
    M^{(j)}_n are per summand and stay local; the sketch Y_n = Z_n [W^{(j)}_n]_j
    and the last core are sums over summands, so each rank forms its part and
    allreduce(array) -> array returns the sum over the ranks; every rank then
    takes the same QR. Returns the whole rounded tensor on every rank."""
    s = len(Ys_local)
    N = len(Ys_local[0])
    if coeffs is None:
        coeffs = [1.0] * s
    Ys = [[c * Y[0]] + list(Y[1:]) for c, Y in zip(coeffs, Ys_local)]
    W = [partial_contractions_rl(Y, R) for Y in Ys]
    X = [None] * N
    Xn = np.concatenate([Y[0] for Y in Ys], axis=2)
    if N == 1:
        return [allreduce(sum(Y[0] for Y in Ys))]
    for n in range(1, N):
        I = Xn.shape[1]
        Z = V(Xn)
        Wstack = np.concatenate([W[j][n] for j in range(s)], axis=0)
        Ysk = allreduce(Z @ Wstack)
        Q, _ = np.linalg.qr(Ysk)
        X[n - 1] = from_V(Q, I)
        M = Q.T @ Z
        cols = np.cumsum([0] + [Y[n - 1].shape[2] for Y in Ys])
        Mj = [M[:, cols[j]:cols[j + 1]] for j in range(s)]
        Inext = Ys[0][n].shape[1]
        if n < N - 1:
            blocks = [from_H(Mj[j] @ H(Ys[j][n]), Inext) for j in range(s)]
            Xn = np.concatenate(blocks, axis=2)
        else:
            Xn = allreduce(sum(from_H(Mj[j] @ H(Ys[j][N - 1]), Inext) for j in range(s)))
    X[N - 1] = Xn
    return X


def round_orthrand(Y, Omegas):
    """Algorithm 4 (Orthogonalize-then-Randomize): Y := OrthogonalizeRL(Y);
    X_1 = Y_1; for n = 1..N-1: Z_n = V(X_n); Y_n = Z_n Omega_n (Omega_n an
    R_n x l_n Gaussian matrix); [V(X_n), ~] = QR(Y_n); M_n = V(X_n)^T Z_n;
    H(X_{n+1}) = M_n H(Y_{n+1}). Omegas[n] holds Omega_n for n = 1..N-1."""
    Yo = orthogonalize_rl(Y)
    N = len(Yo)
    X = [None] * N
    Xn = np.array(Yo[0], copy=True)
    for n in range(1, N):
        I = Xn.shape[1]
        Z = V(Xn)
        Ysk = Z @ Omegas[n]
        Q, _ = np.linalg.qr(Ysk)
        X[n - 1] = from_V(Q, I)
        M = Q.T @ Z
        Xn = from_H(M @ H(Yo[n]), Yo[n].shape[1])
    X[N - 1] = Xn
    return X


def _pinv_sqrt(s, l, rho):
    tol = max(l, rho) * np.finfo(np.float64).eps * (s[0] if s.size else 0.0)
    out = np.zeros_like(s)
    keep = s > tol
    out[keep] = 1.0 / np.sqrt(s[keep])
    return out


def round_twosided(Y, Lsk, Rsk):
    """Algorithm 6 (Two-Sided-Randomization, generalized Nystrom):
    W^L = PartialContractionsLR(Y, L) (ranks l), W^R = PartialContractionsRL(Y, R)
    (ranks rho); for n = 1..N-1: [U, S, V] = SVD(W^L_n W^R_n);
    L_n = W^R_n V (S^dagger)^{1/2}; R_n = (S^dagger)^{1/2} U^T W^L_n;
    V(X_1) = V(Y_1) L_1; X_n(:, i, :) = R_{n-1} Y_n(:, i, :) L_n; H(X_N) = R_{N-1} H(Y_N)."""
    N = len(Y)
    WL = partial_contractions_lr(Y, Lsk)
    WR = partial_contractions_rl(Y, Rsk)
    Lf = [None] * (N + 1)
    Rf = [None] * (N + 1)
    for n in range(1, N):
        A = WL[n] @ WR[n]
        U, s, Vt = np.linalg.svd(A, full_matrices=False)
        sh = _pinv_sqrt(s, A.shape[0], A.shape[1])
        Lf[n] = (WR[n] @ Vt.T) * sh[None, :]
        Rf[n] = sh[:, None] * (U.T @ WL[n])
    X = [None] * N
    X[0] = from_V(V(Y[0]) @ Lf[1], Y[0].shape[1])
    for n in range(2, N):
        Yn = Y[n - 1]
        X[n - 1] = np.einsum("ab,bic,cd->aid", Rf[n - 1], Yn, Lf[n])
    X[N - 1] = from_H(Rf[N - 1] @ H(Y[N - 1]), Y[N - 1].shape[1])
    return X


def round_sum_twosided(Ys, Lsk, Rsk, coeffs=None):
    """Algorithm 6 applied to the formed TT-sum (Section 2.1 block cores)."""
    return round_twosided(block_sum(Ys, coeffs), Lsk, Rsk)


def round_sum_twosided_orth(Ys, Lsk, Rsk, coeffs=None, eps0=0.0):
    """Algorithm 6 with the orthogonalizing restructure that Section 3.3
    mentions without spelling out (reading: the Two-Sided cores are
    left-orthogonalized by the left-to-right mirror of Algorithm 1, which
    carries each thin-QR R factor into the next core), followed, when eps0 > 0,
    by the Section 3.2 truncation of the left-orthogonal result."""
    X = orthogonalize_lr(round_sum_twosided(Ys, Lsk, Rsk, coeffs))
    if eps0 > 0:
        X = truncate_left_orthogonal(X, eps0)
    return X


def truncate_left_orthogonal(X, eps0=0.0, max_rank=None, return_sv=False):
    """Truncation of a left-orthogonal TT (the Randomize-then-Orthogonalize
    output, Section 3.2) without re-orthogonalizing: ||X|| = ||X_N||;
    eps = ||X|| eps0 / sqrt(N-1); for n = N..2: [Q, R] = QR(H(X_n)^T);
    [U, S, V] = SVD(R, eps); H(X_n) := (Q U)^T; V(X_{n-1}) := V(X_{n-1}) V S."""
    X = [np.array(c, copy=True) for c in X]
    N = len(X)
    nrm = float(np.linalg.norm(X[N - 1]))
    eps = nrm / np.sqrt(max(N - 1, 1)) * eps0 if eps0 > 0 else 0.0
    svs = [None] * N
    for n in range(N, 1, -1):
        Xn = X[n - 1]
        Q, R = np.linalg.qr(H(Xn).T)
        U, s, Vt, s_all = svd_truncated(R, eps, max_rank)
        svs[n - 1] = s_all
        X[n - 1] = from_H((Q @ U).T, Xn.shape[1])
        X[n - 2] = from_V(V(X[n - 2]) @ (Vt.T * s[None, :]), X[n - 2].shape[1])
    return (X, svs) if return_sv else X


def check_ranks(Y):
    r = ranks_of(Y)
    assert r[0] == 1 and r[-1] == 1
    return r
