"""TT-GMRES (Section 4.2) on the GPU: right-preconditioned GMRES whose Krylov
vectors are TTs, with both linear combinations of every iteration rounded by
the randomized sum rounding (Algorithm 7 + the Section 3.2 truncation):

  Y = (M^{-1} (x) I ... (x) I) V_k                   (tt_mode_products)
  W = round( sum_i (A_{i,1} (x) ... (x) A_{i,N}) Y )   (tt_mode_products, tt_round_sum_rand)
  h, V_{k+1} = Gram-Schmidt step                      (tt_round_gram_schmidt, one call)

The operator is given by its Kronecker factors (`terms[i][n]` a float64 CUDA
matrix, None for an identity factor); a summand of W shares the cores of Y
wherever its factor is the identity. Every rounding draws its sketch on the
device from its own seed (seed0 + a running count) with sketch ranks
min(formal rank of the sum, ell_cap) per bond. The small Hessenberg
least-squares problem (at most maxit columns) is updated with Givens rotations
on the host: it is a handful of scalars per iteration.
"""
from __future__ import annotations

import math

import torch

from . import api


def _ranks(X):
    return [int(X[0].shape[0])] + [int(c.shape[2]) for c in X]


def _sketch_ranks(summands, dims, ell_cap):
    N = len(dims)
    S = [sum(_ranks(Y)[n] for Y in summands) for n in range(N + 1)]
    return api.clamp_ranks(dims, [1] + [min(S[n], ell_cap) for n in range(1, N)] + [1])


def apply_terms(terms, Y):
    """The N summands (A_{i,1} (x) ... (x) A_{i,N}) Y of the operator applied to
    Y: all non-identity factors in one grouped launch; identity factors share Y's cores."""
    mats, cores, where = [], [], []
    for i, t in enumerate(terms):
        for n, A in enumerate(t):
            if A is not None:
                mats.append(A)
                cores.append(Y[n])
                where.append((i, n))
    prod = api.tt_mode_products(mats, cores)
    out = [list(Y) for _ in terms]
    for (i, n), c in zip(where, prod):
        out[i][n] = c
    return out


def precondition(Minv, V):
    return [api.tt_mode_products([Minv], [V[0]])[0]] + list(V[1:])


def tt_gmres(terms, Minv, f, *, tol=1e-8, maxit=30, ell_cap=40, round_tol=None, seed0=1000, precision="fp64"):
    """Solve (sum_i A_{i,1} (x) ... (x) A_{i,N}) x = f (f a TT of float64 CUDA
    cores) to relative residual tol. Returns (x cores, residual estimates per
    iteration, Krylov vector ranks per iteration)."""
    rt = 0.1 * tol if round_tol is None else round_tol
    # the Krylov combinations cancel: in mixed precision their sketches take full digits too
    sum_prec = "mixed_full" if precision == "mixed" else precision
    dims = [int(c.shape[1]) for c in f]
    count = [seed0]

    def seed():
        count[0] += 1
        return count[0]

    beta = float(api.tt_norm(f))
    V = [[f[0] / beta] + list(f[1:])]
    m_max = maxit
    R = [[0.0] * m_max for _ in range(m_max + 1)]
    cs, sn = [0.0] * m_max, [0.0] * m_max
    g = [0.0] * (m_max + 1)
    g[0] = beta
    res, ranks = [], []
    k = 0
    for k in range(maxit):
        Y = precondition(Minv, V[k])
        summands = apply_terms(terms, Y)
        W = api.tt_round_sum_rand(summands, _sketch_ranks(summands, dims, ell_cap), tol=rt, seed=seed(),
                                  precision=sum_prec)
        W = [c.contiguous() for c in W]
        Vn, h = api.tt_round_gram_schmidt(W, V, _sketch_ranks([W] + V, dims, ell_cap), tol=rt, seed=seed(),
                                          precision=precision)
        col = h + [0.0] * (m_max + 1 - len(h))
        for j in range(k):
            t = cs[j] * col[j] + sn[j] * col[j + 1]
            col[j + 1] = -sn[j] * col[j] + cs[j] * col[j + 1]
            col[j] = t
        d = math.hypot(col[k], col[k + 1])
        cs[k], sn[k] = (col[k] / d, col[k + 1] / d) if d > 0 else (1.0, 0.0)
        col[k], col[k + 1] = d, 0.0
        for j in range(k + 1):
            R[j][k] = col[j]
        g[k + 1] = -sn[k] * g[k]
        g[k] = cs[k] * g[k]
        res.append(abs(g[k + 1]) / beta)
        V.append([c.contiguous() for c in Vn])
        ranks.append(_ranks(Vn))
        if res[-1] <= tol:
            break
    m = k + 1
    y = [0.0] * m
    for i in range(m - 1, -1, -1):              # back substitution with the rotated triangle
        y[i] = (g[i] - sum(R[i][j] * y[j] for j in range(i + 1, m))) / R[i][i]
    U = api.tt_round_sum_rand(V[:m], _sketch_ranks(V[:m], dims, ell_cap), coeffs=y, tol=rt, seed=seed(),
                              precision=sum_prec)
    return precondition(Minv, [c.contiguous() for c in U]), res, ranks
