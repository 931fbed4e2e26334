"""TT format basics of Section 2.1 (oracle; test infrastructure only).

A TT-tensor is a list of N cores; core n (0-based here, n+1 in the paper) is an
array of shape (R_{n}, I_{n+1}, R_{n+1}) with R_0 = R_N = 1. An entry of the
tensor is the product of the slices T_1(:, i_1, :) ... T_N(:, i_N, :)
(Section 2.1, definition of the TT format).
"""
from __future__ import annotations

import itertools

import numpy as np


def dims_of(cores):
    return [c.shape[1] for c in cores]


def ranks_of(cores):
    return [cores[0].shape[0]] + [c.shape[2] for c in cores]


def H(core):
    """Horizontal unfolding (Section 2.1, Fig. 1): the slices core[:, i, :]
    placed side by side, an R0 x (I*R1) matrix whose column i*R1 + b holds
    core[:, i, b]."""
    r0, I, r1 = core.shape
    return np.ascontiguousarray(core).reshape(r0, I * r1)


def V(core):
    """Vertical unfolding (Section 2.1, Fig. 1): the slices core[:, i, :]
    stacked on top of each other, an (I*R0) x R1 matrix whose row i*R0 + a
    holds core[a, i, :]."""
    r0, I, r1 = core.shape
    return np.ascontiguousarray(core.transpose(1, 0, 2)).reshape(I * r0, r1)


def from_H(M, I):
    """Inverse of H for a core with mode size I."""
    r0 = M.shape[0]
    return np.ascontiguousarray(M).reshape(r0, I, M.shape[1] // I)


def from_V(M, I):
    """Inverse of V for a core with mode size I."""
    r1 = M.shape[1]
    return np.ascontiguousarray(np.ascontiguousarray(M).reshape(I, M.shape[0] // I, r1).transpose(1, 0, 2))


def merge_left(cores, n):
    """V(T_{1:n}): the product of the first n cores as an (I_1...I_n) x R_n
    matrix, rows in C order of (i_1, ..., i_n) (Section 2.1, interface
    unfolding X_(1:n) = V(T_{1:n}) H(T_{n+1:N}))."""
    T = cores[0].reshape(cores[0].shape[1], cores[0].shape[2])
    for c in cores[1:n]:
        T = (T @ H(c)).reshape(-1, c.shape[2])
    return T


def merge_right(cores, n):
    """H(T_{n+1:N}): the product of cores n+1..N (1-based) as an
    R_n x (I_{n+1}...I_N) matrix, columns in C order of (i_{n+1}, ..., i_N)."""
    last = cores[-1]
    T = last.reshape(last.shape[0], last.shape[1])
    for c in reversed(cores[n:-1]):
        r0, I, r1 = c.shape
        T = (c.reshape(r0 * I, r1) @ T).reshape(r0, -1)
    return T


def full(cores):
    """The full tensor (shape I_1 x ... x I_N) by multiplying the cores."""
    return merge_left(cores, len(cores)).reshape(dims_of(cores))


def full_bruteforce(cores):
    """The full tensor entry by entry from the definition: product of the
    slices T_1(:, i_1, :) ... T_N(:, i_N, :). Tiny tensors only."""
    dims = dims_of(cores)
    out = np.zeros(dims)
    for idx in itertools.product(*[range(d) for d in dims]):
        p = np.ones((1, 1))
        for c, i in zip(cores, idx):
            p = p @ c[:, i, :]
        out[idx] = p[0, 0]
    return out


def block_sum(summands, coeffs=None):
    """Formed TT-sum of Section 2.1: first cores side by side, middle cores
    block diagonal slice by slice, last cores stacked. coeffs (optional) scale
    each summand through its first core."""
    K = len(summands)
    N = len(summands[0])
    if coeffs is None:
        coeffs = [1.0] * K
    out = []
    for n in range(N):
        I = summands[0][n].shape[1]
        r0s = [s[n].shape[0] for s in summands]
        r1s = [s[n].shape[2] for s in summands]
        if N == 1:
            out.append(sum(c * s[0] for c, s in zip(coeffs, summands)))
            continue
        if n == 0:
            out.append(np.concatenate([c * s[0] for c, s in zip(coeffs, summands)], axis=2))
        elif n == N - 1:
            out.append(np.concatenate([s[n] for s in summands], axis=0))
        else:
            C = np.zeros((sum(r0s), I, sum(r1s)))
            a = b = 0
            for j, s in enumerate(summands):
                C[a:a + r0s[j], :, b:b + r1s[j]] = s[n]
                a += r0s[j]
                b += r1s[j]
            out.append(C)
    return out


def _contract_rl(X, Y):
    """Right-to-left partial contractions W_n = H(X_{n+1:N}) H(Y_{n+1:N})^T
    (Eq. of Section 2.3, computed as in Algorithm 3), extended down to n = 0
    where W_0 is the 1 x 1 inner product."""
    N = len(X)
    W = [None] * (N + 1)
    W[N] = np.ones((1, 1))
    for n in range(N, 0, -1):
        Xn, Yn = X[n - 1], Y[n - 1]
        Z = from_V(V(Xn) @ W[n], Xn.shape[1])
        W[n - 1] = H(Z) @ H(Yn).T
    return W


def inner(X, Y):
    """<X, Y> as the last partial contraction W_0 (Algorithm 3 run down to the
    first core)."""
    return float(_contract_rl(X, Y)[0][0, 0])


def _orth_first_core_norm(cores):
    # Right-to-left orthogonalization (Algorithm 1) keeps the norm in core 1.
    X = [np.array(c, copy=True) for c in cores]
    for n in range(len(X) - 1, 0, -1):
        I = X[n].shape[1]
        Q, R = np.linalg.qr(H(X[n]).T)
        X[n] = from_H(Q.T, I)
        X[n - 1] = from_V(V(X[n - 1]) @ R.T, X[n - 1].shape[1])
    return float(np.linalg.norm(X[0]))


def norm(cores):
    """||X|| via right-to-left orthogonalization: the norm of the first core of
    a right-orthogonal TT (Section 2.3)."""
    return _orth_first_core_norm(cores)


def diff_norm(A, B):
    """||A - B|| computed on the difference TT A + (-1) B (formed sum) after
    orthogonalization, accurate down to round-off of ||A|| + ||B||."""
    return _orth_first_core_norm(block_sum([A, B], [1.0, -1.0]))
