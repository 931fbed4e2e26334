"""Algorithmic flop and byte counts used to report throughput.

Flops follow the cost analysis of Section 3.5 and Appendix A, kept per core so
that uneven summand ranks and sketch ranks are counted exactly:
  * Algorithm 3 per summand and middle core:  2 I l_n R_{n-1} R_n + 2 I R_{n-1} l_n l_{n-1}
    (V(Z) = V(Y) W, then H(Z) H(Omega)^T);
  * Algorithm 7 per middle core: core update 2 I l_{n-1} sum_j R_{n-1}^{(j)} R_n^{(j)},
    sketch 2 I l_{n-1} S_n l_n, Householder QR 4 m l_n^2 - 4 l_n^3/3 with m = l_{n-1} I,
    projection 2 I l_{n-1} S_n l_n (Section 3.5.2).
For equal ranks these reduce to the paper's I(N-2)(4sR^2 l + 6sR l^2 + 4 l^3)
(with the quadratic-in-l term read as 4 l^3, the Householder count).
Bytes: inputs read twice (one pass per sweep), sketch read once, output
written once, all as float64.
"""
from __future__ import annotations


def flops_sum_randorth(dims, ranks_per_summand, ells):
    N = len(dims)
    ell = ells
    f = 0.0
    for n in range(2, N + 1):           # Algorithm 3 for every summand, cores N..2
        I = dims[n - 1]
        for R in ranks_per_summand:
            f += 2.0 * I * R[n - 1] * R[n] * ell[n] + 2.0 * I * R[n - 1] * ell[n] * ell[n - 1]
    for n in range(1, N + 1):           # left-to-right sweep
        I = dims[n - 1]
        S = sum(R[n] for R in ranks_per_summand)
        f += sum(2.0 * I * ell[n - 1] * R[n - 1] * R[n] for R in ranks_per_summand)   # X_n
        f += 2.0 * I * ell[n - 1] * S * ell[n]                                          # sketch / last core
        if n < N:
            m, k = ell[n - 1] * I, ell[n]
            f += 4.0 * m * k * k - 4.0 * k ** 3 / 3.0                                   # thin QR
            f += 2.0 * m * S * k                                                        # projection
    return f


def bytes_sum_randorth(dims, ranks_per_summand, ells):
    N = len(dims)
    inp = sum(R[n] * dims[n] * R[n + 1] for R in ranks_per_summand for n in range(N))
    sk = sum(ells[n - 1] * dims[n - 1] * ells[n] for n in range(2, N + 1))
    out = sum(ells[n] * dims[n] * ells[n + 1] for n in range(N))
    return 8.0 * (2 * inp + sk + out)


def flops_det(dims, formed_ranks, out_ranks):
    """Algorithm 1 + Algorithm 2 on the formed sum (Appendix A): per core the
    right-to-left orthogonalization costs 4 m k^2 - 4 k^3/3 (Householder QR of
    H(X_n)^T, m = I_n R_n, k = R_{n-1}) plus R_{n-2} I_{n-1} k^2 (the triangular
    update); the left-to-right truncation costs the QR of V(X_n), the SVD of R
    (~ 12 k^3) and the two updates 2 m k r + 2 r k I R_{n+1}."""
    N = len(dims)
    R = list(formed_ranks)
    f = 0.0
    for n in range(N, 1, -1):
        m, k = dims[n - 1] * R[n], R[n - 1]
        if m >= k:
            f += 4.0 * m * k * k - 4.0 * k ** 3 / 3.0 + R[n - 2] * dims[n - 2] * k * k
    r = out_ranks
    for n in range(1, N):
        m, k = R[n - 1] * dims[n - 1], R[n]
        f += 4.0 * m * k * k - 4.0 * k ** 3 / 3.0 + 12.0 * k ** 3
        f += 2.0 * m * k * r[n] + 2.0 * r[n] * k * dims[n] * R[n + 1]
    return f
