"""Brute-force helpers used only by the tests to pin the oracle (computed from
full tensors and definitions, not from the oracle's algorithms)."""
import numpy as np


def unfold(F, n):
    """X_(1:n) of a full tensor: rows (i_1..i_n), columns (i_{n+1}..i_N), C order."""
    return F.reshape(int(np.prod(F.shape[:n])), -1)


def orth(A, rtol=1e-12):
    """Orthonormal basis of range(A) from the SVD (numerical rank by rtol)."""
    U, s, _ = np.linalg.svd(A, full_matrices=False)
    k = int(np.sum(s > rtol * s[0])) if s.size and s[0] > 0 else 0
    return U[:, :k]


def tt_svd_full(F, ranks):
    """Left-to-right TT-SVD of a full tensor with fixed ranks (Oseledets 2011)."""
    dims = F.shape
    N = len(dims)
    cores = []
    M = F.reshape(dims[0], -1)
    r0 = 1
    for n in range(N - 1):
        M = M.reshape(r0 * dims[n], -1)
        U, s, Vt = np.linalg.svd(M, full_matrices=False)
        r = min(ranks[n + 1], len(s))
        cores.append(U[:, :r].reshape(r0, dims[n], r))
        M = s[:r, None] * Vt[:r]
        r0 = r
    cores.append(M.reshape(r0, dims[-1], 1))
    return cores


def rel(a, b):
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def left_part_bruteforce(cores, n):
    """V(T_{1:n}) entry by entry: row (i_1..i_n) C order, column r = the r-th
    entry of the row vector T_1(:, i_1, :) ... T_n(:, i_n, :)."""
    import itertools
    dims = [c.shape[1] for c in cores[:n]]
    rn = cores[n - 1].shape[2]
    out = np.zeros((int(np.prod(dims)), rn))
    for row, idx in enumerate(itertools.product(*[range(d) for d in dims])):
        p = np.ones((1, 1))
        for c, i in zip(cores[:n], idx):
            p = p @ c[:, i, :]
        out[row] = p[0]
    return out


def right_part_bruteforce(cores, n):
    """H(T_{n+1:N}) entry by entry: row r, column (i_{n+1}..i_N) C order."""
    import itertools
    rest = cores[n:]
    dims = [c.shape[1] for c in rest]
    rn = rest[0].shape[0]
    out = np.zeros((rn, int(np.prod(dims))))
    for col, idx in enumerate(itertools.product(*[range(d) for d in dims])):
        p = np.eye(rn)
        for c, i in zip(rest, idx):
            p = p @ c[:, i, :]
        out[:, col] = p[:, 0]
    return out


def full_from_cores_bruteforce(cores):
    return (left_part_bruteforce(cores, len(cores))[:, 0]).reshape([c.shape[1] for c in cores])
