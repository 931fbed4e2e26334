"""Seeded synthetic inputs for TT-rounding: shared by the tests, the benchmark and
the oracle's own checks.

This module draws random numbers and builds input tensors in TT format. It holds
none of the rounding method's arithmetic (no contraction, QR, SVD or projection):
both the CUDA path and the CPU oracle receive the arrays made here.

Storage convention (same everywhere in the project): a TT core with ranks
(r0, r1) and mode size I is a float64 array of shape (r0, I, r1) in C order, so
element (a, i, b) sits at offset (a*I + i)*r1 + b.

Distributions follow the paper:
* Definition 3.1 (random Gaussian TT, Section 3.2): entries i.i.d. normal with
  mean 0 and variance 1/(r0*I*r1). This is used for the sketch tensors and, as
  the normalisation of Section 4.1 states, for the synthetic inputs too.
* Section 4.1: a low-rank TT perturbed by a small multiple of another TT.
* Section 3.4 / 4.2: sums of many TTs of uneven ranks (TT-GMRES combinations).
"""
from __future__ import annotations

import numpy as np

__all__ = [
    "rng_for",
    "gaussian_tt",
    "gaussian_matrix",
    "scale_tt",
    "gauge_scramble",
    "perturb_cores",
    "hilbert_tt",
    "workload_single",
    "workload_sum_literal",
    "workload_sum_structured",
    "workload_batched",
    "sketch_ranks_for",
    "cookie_operator",
]


def rng_for(seed: int, stream: int = 0) -> np.random.Generator:
    """Independent PCG64 stream for (seed, stream)."""
    return np.random.Generator(np.random.PCG64(np.random.SeedSequence([int(seed), int(stream)])))


def gaussian_tt(rng: np.random.Generator, dims, ranks, dtype=np.float64):
    """Random Gaussian TT of Definition 3.1: core n has shape (ranks[n], dims[n],
    ranks[n+1]) and entries N(0, 1/(ranks[n]*dims[n]*ranks[n+1]))."""
    dims = [int(d) for d in dims]
    ranks = [int(r) for r in ranks]
    assert len(ranks) == len(dims) + 1 and ranks[0] == 1 and ranks[-1] == 1
    cores = []
    for n, I in enumerate(dims):
        r0, r1 = ranks[n], ranks[n + 1]
        std = 1.0 / np.sqrt(r0 * I * r1)
        cores.append((rng.standard_normal((r0, I, r1)) * std).astype(dtype))
    return cores


def gaussian_matrix(rng: np.random.Generator, m: int, n: int):
    """Standard Gaussian m x n matrix (the test matrix of randomized SVD, Section 2.2)."""
    return rng.standard_normal((int(m), int(n)))


def scale_tt(cores, c: float):
    """Return a copy of the TT with its first core multiplied by c."""
    out = [np.array(x, copy=True) for x in cores]
    out[0] = out[0] * c
    return out


def gauge_scramble(rng: np.random.Generator, cores, log2_spread: float = 1.0):
    """Insert a random well-conditioned gauge A_n, A_n^{-1} on every inner bond.

    The represented tensor is unchanged (up to rounding); only its cores differ.
    A_n = Q diag(2^u) with Q Haar-orthogonal and u uniform in [-s, s], so the
    condition number of each gauge is at most 4^s.
    """
    out = [np.array(x, copy=True) for x in cores]
    for n in range(len(out) - 1):
        r = out[n].shape[2]
        q, rr = np.linalg.qr(rng.standard_normal((r, r)))
        q = q * np.sign(np.diag(rr))
        d = 2.0 ** rng.uniform(-log2_spread, log2_spread, size=r)
        A = q * d[None, :]
        Ainv = (q / d[None, :]).T.copy()
        out[n] = np.tensordot(out[n], A, axes=([2], [0]))
        out[n + 1] = np.tensordot(Ainv, out[n + 1], axes=([1], [0]))
    return out


def perturb_cores(rng: np.random.Generator, cores, delta: float):
    """Add delta * N(0, var(core)) noise to every core entry (ranks unchanged)."""
    out = []
    for x in cores:
        s = np.sqrt(np.mean(x * x)) if x.size else 0.0
        out.append(x + delta * s * rng.standard_normal(x.shape))
    return out


def hilbert_tt(dims, ranks):
    """Hilbert-type TT of Appendix C: core n entries 1/(i1+i2+i3-1), 1-based."""
    cores = []
    for n, I in enumerate(dims):
        r0, r1 = ranks[n], ranks[n + 1]
        a = np.arange(1, r0 + 1)[:, None, None]
        i = np.arange(1, I + 1)[None, :, None]
        b = np.arange(1, r1 + 1)[None, None, :]
        cores.append(1.0 / (a + i + b - 1.0))
    return cores


def _uniform_ranks(N, R):
    return [1] + [int(R)] * (N - 1) + [1]


def workload_single(seed: int, N=10, I=50, R=10, R_pert=30, eps=1e-6):
    """Section 4.1 shape: X = Y + eps*E with Y of TT-rank R and E of TT-rank R_pert,
    both Gaussian with Definition 3.1 scaling. Returned as a list of two summands
    (formal rank R + R_pert once added)."""
    dims = [int(I)] * N
    Y = gaussian_tt(rng_for(seed, 1), dims, _uniform_ranks(N, R))
    E = gaussian_tt(rng_for(seed, 2), dims, _uniform_ranks(N, R_pert))
    return [Y, scale_tt(E, eps)]


def workload_sum_literal(seed: int, K=20, N=50, I=100, R=10):
    """K i.i.d. Gaussian TTs of TT-rank R (Definition 3.1 scaling): the literal
    sum-of-TTs workload of Section 3.4 (generically full rank K*R)."""
    dims = [int(I)] * N
    return [gaussian_tt(rng_for(seed, 100 + j), dims, _uniform_ranks(N, R)) for j in range(K)]


def workload_sum_structured(seed: int, K=20, N=50, I=100, R=10, m=2, p=2, delta=1e-10):
    """Redundant sum in the style of TT-GMRES combinations (Section 4.2). The
    first K - p summands are c_j times gauge-scrambled copies of m base TTs of
    rank R (so together they have TT-rank m*R); the last p summands are
    independent Gaussian TTs of rank R scaled by delta (relative to the base
    norm), a genuine tail of relative size about delta. Every summand keeps
    TT-rank R."""
    dims = [int(I)] * N
    bases = [gaussian_tt(rng_for(seed, 200 + a), dims, _uniform_ranks(N, R)) for a in range(m)]
    crng = rng_for(seed, 300)
    out = []
    for j in range(K - p):
        g = rng_for(seed, 400 + j)
        Y = gauge_scramble(g, bases[j % m])
        out.append(scale_tt(Y, float(crng.standard_normal())))
    for j in range(p):
        E = gaussian_tt(rng_for(seed, 600 + j), dims, _uniform_ranks(N, R))
        out.append(scale_tt(E, delta))
    return out


def workload_batched(seed: int, B=256, N=20, I=64, K_range=(2, 30), R_range=(4, 16), ell_range=(8, 32)):
    """B independent sums with uneven summand counts and ranks: K ~ U[K_range],
    rank of each summand ~ U[R_range] (constant over its inner bonds), sketch
    rank ~ U[ell_range]. Returns a list of (summands, ell)."""
    shp = rng_for(seed, 500)
    probs = []
    for b in range(B):
        K = int(shp.integers(K_range[0], K_range[1] + 1))
        ell = int(shp.integers(ell_range[0], ell_range[1] + 1))
        Rs = shp.integers(R_range[0], R_range[1] + 1, size=K)
        summ = [gaussian_tt(rng_for(seed, 10_000 + 64 * b + j), [I] * N, _uniform_ranks(N, int(Rs[j])))
                for j in range(K)]
        probs.append((summ, ell))
    return probs


def sketch_ranks_for(dims, ell):
    """Target ranks (1, ell, ..., ell, 1) for a TT with the given mode sizes."""
    return [1] + [int(ell)] * (len(dims) - 1) + [1]


def cookie_operator(N=5, I1=40, I=8, rho_range=(1.0, 10.0)):
    """Synthetic stand-in for the parametric "cookie" problem of Section 4.2
    (its FEM matrices are not available): the operator
        A = sum_{i=1}^{N} A_{i,1} (x) ... (x) A_{i,N}
    on a one-dimensional domain of I1 interior nodes (linear finite elements,
    homogeneous Dirichlet ends) holding N - 1 disjoint "cookie" intervals.
    A_{1,1} is the stiffness matrix of the whole domain, A_{i,1} (i >= 2) the
    stiffness assembled over the cells of cookie i - 1 only, A_{i,i} =
    diag(rho) with I parameter samples spread linearly over rho_range, and
    every other factor the identity. Returns dict(terms, f, dims): terms[i] is
    a list of N matrices (None for an identity factor), f the right-hand side
    (ones over the domain times ones over every parameter) as TT cores."""
    h = 1.0 / (I1 + 1)
    ncell = I1 + 1

    def stiffness(cells):
        K = np.zeros((I1, I1))
        for c in cells:                      # cell c joins nodes c - 1 and c (1-based interior nodes)
            a, b = c - 1, c
            for (p, q, v) in ((a, a, 1.0), (b, b, 1.0), (a, b, -1.0), (b, a, -1.0)):
                if 1 <= p <= I1 and 1 <= q <= I1:
                    K[p - 1, q - 1] += v / h
        return K

    ncook = N - 1
    width = max(1, ncell // (2 * ncook + 1))
    cookies = [list(range(1 + (2 * c + 1) * width, 1 + (2 * c + 2) * width)) for c in range(ncook)]
    rho = np.linspace(rho_range[0], rho_range[1], I)
    terms = [[stiffness(range(1, ncell + 1))] + [None] * (N - 1)]
    for i in range(2, N + 1):
        t = [stiffness(cookies[i - 2])] + [None] * (N - 1)
        t[i - 1] = np.diag(rho)
        terms.append(t)
    dims = [I1] + [I] * (N - 1)
    f = [np.ones((1, I1, 1)) * h] + [np.ones((1, I, 1)) for _ in range(N - 1)]
    return {"terms": terms, "f": f, "dims": dims}
