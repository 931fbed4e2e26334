"""TT-GMRES of Section 4.2 restated for the oracle: inexact Arnoldi with
rounded Krylov vectors, where both linear combinations of an iteration are
rounded by Algorithm 7 (randomized sum rounding) followed by the Section 3.2
truncation.

TEST INFRASTRUCTURE ONLY: used by the tests (and nothing in the product path).

Per iteration k, following Section 4.2:
  * preconditioning: Y = (M^{-1} (x) I (x) ... (x) I) V_k, M = sum_i A_{i,1};
  * operator: W = sum_i (A_{i,1} (x) ... (x) A_{i,N}) Y, a sum of N TTs with
    the ranks of Y, rounded;
  * Gram-Schmidt: h_{jk} = <V_j, W> (j <= k), Z = W - sum_j h_{jk} V_j rounded,
    h_{k+1,k} = ||Z||, V_{k+1} = Z / h_{k+1,k};
  * the small least-squares problem min ||beta e_1 - H y|| by Givens rotations
    (the textbook GMRES update), whose residual stops the iteration.
The approximate solution is x = M^{-1} (sum_j y_j V_j), the sum rounded too.

Sketches: every rounding draws its Gaussian TT sketch (Definition 3.1) with the
counter-based generator from its own seed (seed0 + a running count), with sketch
ranks l_n = min(formal rank of the sum at bond n, ell_cap), clamped so that
every thin QR is tall.
"""
from __future__ import annotations

import numpy as np

from .tt import inner, norm, ranks_of, dims_of
from .rounding import round_sum_randorth, truncate_left_orthogonal, clamp_ranks
from .philox import gaussian_sketch_philox


def apply_term(Y, mats):
    """(A_1 (x) ... (x) A_N) Y for a TT Y: mode-n product of core n with A_n
    (None = identity): X_n(a, j, b) = sum_i A_n(j, i) Y_n(a, i, b)."""
    return [c.copy() if A is None else np.einsum("ji,aib->ajb", A, c) for c, A in zip(Y, mats)]


def sum_sketch_ranks(summands, ell_cap):
    dims = dims_of(summands[0])
    N = len(dims)
    S = [sum(ranks_of(Y)[n] for Y in summands) for n in range(N + 1)]
    return clamp_ranks(dims, [1] + [min(S[n], ell_cap) for n in range(1, N)] + [1])


def round_sum(summands, coeffs, ell_cap, tol, seed):
    """Algorithm 7 with the seed's sketch, then the Section 3.2 truncation."""
    ell = sum_sketch_ranks(summands, ell_cap)
    sk = gaussian_sketch_philox(seed, dims_of(summands[0]), ell)
    X = round_sum_randorth(summands, sk, coeffs)
    return truncate_left_orthogonal(X, tol) if tol > 0 else X


def gram_schmidt_round(W, basis, ell_cap, tol, seed):
    """Section 4.2's Gram-Schmidt step: h_j = <V_j, W>, Z = W - sum_j h_j V_j
    (rounded), returns (Z / ||Z||, [h_1, ..., h_k, ||Z||])."""
    h = [inner(V, W) for V in basis]
    Z = round_sum([W] + list(basis), [1.0] + [-x for x in h], ell_cap, tol, seed)
    nz = norm(Z)
    if nz > 0:
        Z = [c.copy() for c in Z]
        Z[0] = Z[0] / nz
    return Z, h + [nz]


def precondition(Minv, V):
    """(M^{-1} (x) I (x) ... (x) I) V: a mode-1 product."""
    return apply_term(V, [Minv] + [None] * (len(V) - 1))


def tt_gmres(terms, Minv, f, tol=1e-8, maxit=30, ell_cap=40, round_tol=None, seed0=1000):
    """Right-preconditioned TT-GMRES (Section 4.2) for
    (sum_i A_{i,1} (x) ... (x) A_{i,N}) x = f with x = M^{-1} u. Returns
    (x cores, residual estimates |g_{k+1}| / beta per iteration, the
    triangular factor of the rotated Hessenberg matrix)."""
    rt = 0.1 * tol if round_tol is None else round_tol
    count = [seed0]

    def seed():
        count[0] += 1
        return count[0]

    beta = norm(f)
    V = [[c.copy() for c in f]]
    V[0][0] = V[0][0] / beta
    H = np.zeros((maxit + 1, maxit))
    cs, sn = np.zeros(maxit), np.zeros(maxit)
    g = np.zeros(maxit + 1)
    g[0] = beta
    res = []
    k = 0
    for k in range(maxit):
        Y = precondition(Minv, V[k])
        W = round_sum([apply_term(Y, t) for t in terms], None, ell_cap, rt, seed())
        Vn, h = gram_schmidt_round(W, V, ell_cap, rt, seed())
        H[:k + 2, k] = h
        # Givens rotations of the previous columns, then a new one for this column
        for j in range(k):
            t = cs[j] * H[j, k] + sn[j] * H[j + 1, k]
            H[j + 1, k] = -sn[j] * H[j, k] + cs[j] * H[j + 1, k]
            H[j, k] = t
        d = np.hypot(H[k, k], H[k + 1, k])
        cs[k], sn[k] = (H[k, k] / d, H[k + 1, k] / d) if d > 0 else (1.0, 0.0)
        H[k, k] = d
        H[k + 1, k] = 0.0
        g[k + 1] = -sn[k] * g[k]
        g[k] = cs[k] * g[k]
        res.append(abs(g[k + 1]) / beta)
        V.append(Vn)
        if res[-1] <= tol:
            break
    m = k + 1
    y = np.linalg.solve(np.triu(H[:m, :m]), g[:m])
    U = round_sum(V[:m], list(y), ell_cap, rt, seed())
    return precondition(Minv, U), res, H[:m + 1, :m]
