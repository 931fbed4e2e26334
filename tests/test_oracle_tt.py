"""Pins of the oracle's TT basics (Section 2.1) against brute force on full tensors."""
import numpy as np
import pytest

import oracle as O
import synth
from tests._tt_helpers import unfold, rel


def _tt(seed, dims, ranks):
    return synth.gaussian_tt(synth.rng_for(seed, 7), dims, ranks)


def test_unfoldings_match_definition():
    c = synth.rng_for(1).standard_normal((3, 4, 5))
    Hm, Vm = O.H(c), O.V(c)
    assert Hm.shape == (3, 20) and Vm.shape == (12, 5)
    for a in range(3):
        for i in range(4):
            for b in range(5):
                assert Hm[a, i * 5 + b] == c[a, i, b]      # slices side by side
                assert Vm[i * 3 + a, b] == c[a, i, b]      # slices stacked
    np.testing.assert_array_equal(O.from_H(Hm, 4), c)
    np.testing.assert_array_equal(O.from_V(Vm, 4), c)


@pytest.mark.parametrize("dims,ranks", [([3, 4, 2, 3], [1, 2, 3, 2, 1]), ([2, 3, 3], [1, 3, 2, 1]), ([5], [1, 1])])
def test_full_matches_bruteforce(dims, ranks):
    X = _tt(2, dims, ranks)
    np.testing.assert_allclose(O.full(X), O.full_bruteforce(X), rtol=1e-13, atol=1e-15)


def test_interface_unfolding_factorises():
    X = _tt(3, [3, 2, 4, 3], [1, 2, 3, 2, 1])
    F = O.full_bruteforce(X)
    for n in range(1, 4):
        np.testing.assert_allclose(O.merge_left(X, n) @ O.merge_right(X, n), unfold(F, n), rtol=1e-12, atol=1e-15)


def test_inner_norm_diffnorm_against_full():
    dims = [3, 4, 2, 3]
    X = _tt(4, dims, [1, 2, 3, 2, 1])
    Y = _tt(5, dims, [1, 3, 2, 3, 1])
    FX, FY = O.full_bruteforce(X), O.full_bruteforce(Y)
    assert abs(O.inner(X, Y) - np.vdot(FX, FY)) <= 1e-13 * np.linalg.norm(FX) * np.linalg.norm(FY)
    assert abs(O.norm(X) - np.linalg.norm(FX)) <= 1e-13 * np.linalg.norm(FX)
    assert abs(O.diff_norm(X, Y) - np.linalg.norm(FX - FY)) <= 1e-12 * np.linalg.norm(FX - FY)
    # diff_norm resolves differences far below sqrt(eps) relative size
    Z = [c.copy() for c in X]
    Z[2] = Z[2] + 1e-11 * synth.rng_for(9).standard_normal(Z[2].shape)
    d_ref = np.linalg.norm(O.full_bruteforce(Z) - FX)
    assert abs(O.diff_norm(X, Z) - d_ref) <= 1e-3 * d_ref


def test_block_sum_is_sum_of_full_tensors():
    dims = [3, 2, 4, 2]
    Ys = [_tt(10 + j, dims, [1, r, r + 1, r, 1]) for j, r in enumerate([1, 2, 3])]
    S = O.block_sum(Ys, [1.0, -2.0, 0.5])
    ref = O.full_bruteforce(Ys[0]) - 2.0 * O.full_bruteforce(Ys[1]) + 0.5 * O.full_bruteforce(Ys[2])
    assert O.ranks_of(S) == [1, 6, 9, 6, 1]
    assert rel(O.full(S), ref) < 1e-13
    # block-diagonal middle cores: off-diagonal blocks are exactly zero
    assert np.all(S[1][0:1, :, 2:] == 0) and np.all(S[1][1:3, :, 0:2] == 0) and np.all(S[1][1:3, :, 5:] == 0)
