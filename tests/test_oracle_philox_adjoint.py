"""Pins of the oracle's counter-based sketch generator (published Philox4x32-10
known answers, Box-Muller moments) and of the fixed-sketch adjoint (central
finite differences and the identity-map closed form)."""
import os

import numpy as np
import pytest

import oracle as O
import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _kat():
    rows = []
    for line in open(os.path.join(GOLDEN, "philox4x32_10_kat.txt")):
        if line.strip() and not line.startswith("#"):
            rows.append([int(x, 16) for x in line.split()])
    return rows


@pytest.mark.parametrize("row", _kat())
def test_philox_known_answers(row):
    out = O.philox4x32_10(*[np.array([v], dtype=np.uint64) for v in row[:6]])
    assert [int(o[0]) for o in out] == row[6:]


def test_sketch_generator_moments_and_determinism():
    dims = [40, 50, 30]
    ells = [1, 20, 25, 1]
    S1 = O.gaussian_sketch_philox(1234, dims, ells)
    S2 = O.gaussian_sketch_philox(1234, dims, ells)
    S3 = O.gaussian_sketch_philox(1235, dims, ells)
    for a, b, c, (r0, I, r1) in zip(S1, S2, S3, [(1, 40, 20), (20, 50, 25), (25, 30, 1)]):
        assert a.shape == (r0, I, r1)
        np.testing.assert_array_equal(a, b)
        assert not np.array_equal(a, c)
        z = a.ravel() * np.sqrt(r0 * I * r1)          # Definition 3.1 variance
        n = z.size
        assert abs(z.mean()) < 5 / np.sqrt(n)
        assert abs(z.var() - 1.0) < 6 * np.sqrt(2.0 / n)
        assert abs(np.mean(z ** 4) - 3.0) < 6 * np.sqrt(96.0 / n)   # Gaussian kurtosis
    # E ||T_n||_F^2 = 1 (Definition 3.1)
    assert abs(np.mean([np.sum(c * c) for c in S1]) - 1.0) < 0.1


# ----------------------------------------------------------------- adjoint

def _setup(seed, dims, R, ell, RT=2):
    Y = synth.gaussian_tt(synth.rng_for(seed, 1), dims, [1] + [R] * (len(dims) - 1) + [1])
    Om = synth.gaussian_tt(synth.rng_for(seed, 2), dims, O.clamp_ranks(dims, [1] + [ell] * (len(dims) - 1) + [1]))
    T = synth.gaussian_tt(synth.rng_for(seed, 3), dims, [1] + [RT] * (len(dims) - 1) + [1])
    return Y, Om, T


def test_adjoint_matches_central_differences_full():
    """Every entry of dL/dY by central differences (tiny case, FP64)."""
    Y, Om, T = _setup(5, [3, 3, 3, 3], 4, 2)
    G = O.randorth_adjoint(Y, Om, T)
    h = 1e-6
    scale = max(np.abs(g).max() for g in G)
    for n in range(4):
        for idx in np.ndindex(Y[n].shape):
            Yp = [c.copy() for c in Y]
            Ym = [c.copy() for c in Y]
            Yp[n][idx] += h
            Ym[n][idx] -= h
            fd = (O.randorth_fixed_sketch_loss(Yp, Om, T) - O.randorth_fixed_sketch_loss(Ym, Om, T)) / (2 * h)
            assert abs(fd - G[n][idx]) <= 1e-6 * scale + 1e-6 * abs(fd)


def test_adjoint_directional_derivatives():
    Y, Om, T = _setup(6, [4, 5, 4, 5, 4], 6, 3)
    G = O.randorth_adjoint(Y, Om, T)
    rng = synth.rng_for(7)
    h = 1e-6
    for _ in range(5):
        D = [rng.standard_normal(c.shape) * np.abs(c).mean() for c in Y]
        Lp = O.randorth_fixed_sketch_loss([c + h * d for c, d in zip(Y, D)], Om, T)
        Lm = O.randorth_fixed_sketch_loss([c - h * d for c, d in zip(Y, D)], Om, T)
        fd = (Lp - Lm) / (2 * h)
        an = sum(float(np.sum(g * d)) for g, d in zip(G, D))
        assert abs(fd - an) <= 1e-6 * max(abs(an), 1e-300) + 1e-9 * sum(float(np.abs(g).sum() * np.abs(d).mean()) for g, d in zip(G, D))


def test_adjoint_identity_closed_form():
    """Target ranks equal to the input ranks (so every sketched matrix has full
    column rank and its R factor is invertible): the rounding is the identity
    near Y, so
    dL/dY_n(:, i, :) = E^L_{n-1} T_n(:, i, :) (E^R_n)^T with the environments of
    <Y, T> (gradient of a TT inner product)."""
    dims = [4, 4, 4, 4]
    Y, Om, T = _setup(8, dims, 3, 3)
    G = O.randorth_adjoint(Y, Om, T)
    N = 4
    for n in range(N):
        # environments by brute force from full left/right parts
        from tests._tt_helpers import left_part_bruteforce, right_part_bruteforce
        EL = np.ones((1, 1)) if n == 0 else left_part_bruteforce(Y, n).T @ left_part_bruteforce(T, n)
        ER = np.ones((1, 1)) if n == N - 1 else right_part_bruteforce(Y, n + 1) @ right_part_bruteforce(T, n + 1).T
        ref = np.einsum("ac,cid,bd->aib", EL, T[n], ER)
        np.testing.assert_allclose(G[n], ref, rtol=1e-9, atol=1e-12 * np.abs(ref).max())
