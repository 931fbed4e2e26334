"""Adjoint of fixed-sketch Randomize-then-Orthogonalize (oracle; test
infrastructure only).

The paper has no derivative; this is the reverse-mode derivative of Algorithm 5
with the Gaussian sketch held fixed, for the scalar loss L = <X_hat, T> where
X_hat = RandOrth(Y, Omega) and T is a fixed TT. It is pinned by central finite
differences and by the closed form that holds when every target rank is at least
the input rank (then X_hat = Y near Y and dL/dY is the inner-product gradient).

Forward quantities of Algorithm 5 (n = 1..N-1): W_n from Algorithm 3,
Z_n = V(X~_n), S_n = Z_n W_n = Q_n T_n (thin QR), X_hat_n = Q_n,
M_n = Q_n^T Z_n, H(X~_{n+1}) = M_n H(Y_{n+1}), X~_1 = Y_1, X_hat_N = X~_N.
Reverse steps, in the opposite order:
  H(X~_{n+1}) = M_n H(Y_{n+1}):  Mbar_n += H(X~bar_{n+1}) H(Y_{n+1})^T,
                                  H(Ybar_{n+1}) += M_n^T H(X~bar_{n+1})
  M_n = Q_n^T Z_n:                Qbar_n += Z_n Mbar_n^T,  Zbar_n += Q_n Mbar_n
  thin QR with Tbar = 0:          Sbar_n = (Qbar_n + Q_n sym_l(-Qbar_n^T Q_n)) T_n^{-T},
                                  sym_l(A) = tril(A) + tril(A, -1)^T
  S_n = Z_n W_n:                  Zbar_n += Sbar_n W_n^T,  Wbar_n += Z_n^T Sbar_n
  Algorithm 3 in reverse, n = 2..N-1: H(Zbar'_n) = Wbar_{n-1} H(Omega_n),
                                  V(Ybar_n) += V(Zbar'_n) W_n^T, Wbar_n += V(Y_n)^T V(Zbar'_n);
  finally H(Ybar_N) += Wbar_{N-1} H(Omega_N) and Ybar_1 += X~bar_1.
"""
from __future__ import annotations

import numpy as np

from .tt import H, V, from_H, from_V
from .rounding import partial_contractions_rl, round_randorth
from .tt import inner


def randorth_fixed_sketch_loss(Y, Om, T):
    """L(Y) = <RandOrth(Y, Omega), T> with Omega fixed (Algorithm 5)."""
    return inner(round_randorth(Y, Om), T)


def _environments(X, T):
    N = len(X)
    EL = [None] * (N + 1)
    EL[0] = np.ones((1, 1))
    for n in range(1, N + 1):
        A = from_H(EL[n - 1] @ H(T[n - 1]), T[n - 1].shape[1])   # l_{n-1} x I x R^T_n
        EL[n] = V(X[n - 1]).T @ V(A)
    ER = [None] * (N + 1)
    ER[N] = np.ones((1, 1))
    for n in range(N, 0, -1):
        B = from_V(V(X[n - 1]) @ ER[n], X[n - 1].shape[1])       # l_{n-1} x I x R^T_n
        ER[n - 1] = H(B) @ H(T[n - 1]).T
    return EL, ER


def randorth_adjoint(Y, Om, T):
    """Gradient dL/dY_n (list of arrays shaped like the cores of Y) of
    L = <RandOrth(Y, Omega), T>, by the reverse steps in the module docstring."""
    N = len(Y)
    W = partial_contractions_rl(Y, Om)
    Xt = [None] * (N + 1)     # X~_n (current core before QR), 1-based
    Q = [None] * N
    Tq = [None] * N
    M = [None] * N
    Xt[1] = np.array(Y[0], copy=True)
    Xhat = [None] * N
    for n in range(1, N):
        Z = V(Xt[n])
        S = Z @ W[n]
        Q[n], Tq[n] = np.linalg.qr(S)
        Xhat[n - 1] = from_V(Q[n], Xt[n].shape[1])
        M[n] = Q[n].T @ Z
        Xt[n + 1] = from_H(M[n] @ H(Y[n]), Y[n].shape[1])
    Xhat[N - 1] = Xt[N]

    # dL/dX_hat_n(:, i, :) = EL_{n-1} T_n(:, i, :) ER_n^T
    EL, ER = _environments(Xhat, T)
    Xhat_bar = [np.einsum("ac,cid,bd->aib", EL[n], T[n], ER[n + 1]) for n in range(N)]

    Ybar = [np.zeros_like(c) for c in Y]
    Wbar = [None] * (N + 1)
    Xt_bar = Xhat_bar[N - 1]
    for n in range(N - 1, 0, -1):
        Inext = Y[n].shape[1]
        Mbar = H(Xt_bar) @ H(Y[n]).T
        Ybar[n] += from_H(M[n].T @ H(Xt_bar), Inext)
        Z = V(Xt[n])
        Qbar = Z @ Mbar.T + V(Xhat_bar[n - 1])
        Zbar = Q[n] @ Mbar
        A = -Qbar.T @ Q[n]
        sym = np.tril(A) + np.tril(A, -1).T
        Sbar = np.linalg.solve(Tq[n], (Qbar + Q[n] @ sym).T).T
        Zbar = Zbar + Sbar @ W[n].T
        Wbar[n] = Z.T @ Sbar
        Xt_bar = from_V(Zbar, Xt[n].shape[1])
    Ybar[0] += Xt_bar

    # Algorithm 3 in reverse.
    for n in range(2, N):
        Yn = Y[n - 1]
        Zp_bar = from_H(Wbar[n - 1] @ H(Om[n - 1]), Yn.shape[1])
        Ybar[n - 1] += from_V(V(Zp_bar) @ W[n].T, Yn.shape[1])
        Wbar[n] = Wbar[n] + V(Yn).T @ V(Zp_bar)
    Ybar[N - 1] += from_H(Wbar[N - 1] @ H(Om[N - 1]), Y[N - 1].shape[1])
    return Ybar
