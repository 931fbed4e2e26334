"""Parity of the CUDA randomized rounding (Algorithms 5 and 7, Section 3.2
truncation, Definition 3.1 sketch) with the CPU oracle, element by element on
the same seeded inputs; outputs are compared as full tensors through the
difference TT (cores of a rounding are fixed only up to orthogonal gauges)."""
import numpy as np
import pytest
import torch

import oracle as O
import synth
from tests._gpu import to_dev, to_host, const_ranks

import paper_2110_04393_gb300 as tt

pytestmark = pytest.mark.gpu
FP64_TOL = 1e-10    # relative Frobenius difference GPU FP64 vs oracle


def rel_diff(Xg, Xo):
    return O.diff_norm(Xg, Xo) / O.norm(Xo)


def run_sum(Ys, ell, sk, coeffs=None, tol=0.0):
    out = tt.tt_round_sum_rand([to_dev(Y) for Y in Ys], ell, sketch=to_dev(sk), coeffs=coeffs, tol=tol)
    return to_host(out)


def test_sketch_generator_matches_oracle_philox():
    dims = [7, 50, 33, 5]
    ells = [1, 9, 31, 4, 1]
    g = to_host(tt.tt_sketch_gaussian(dims, ells, 987654321123))
    o = O.gaussian_sketch_philox(987654321123, dims, ells)
    for a, b in zip(g, o):
        assert a.shape == b.shape
        np.testing.assert_allclose(a, b, rtol=1e-13, atol=1e-15 * np.abs(b).max())


@pytest.mark.parametrize("case", ["tiny", "ragged", "uneven", "long"])
def test_sum_randorth_fixed_rank_parity(case):
    if case == "tiny":
        dims, rs, ell = [3, 4, 3], [2, 1], [1, 2, 3, 1]
    elif case == "ragged":       # several TSQR leaves and a ragged last leaf (m = 37*7 = 259)
        dims, rs, ell = [37, 41, 29, 33, 7], [3, 5, 2], [1, 7, 9, 8, 6, 1]
    elif case == "uneven":
        dims, rs, ell = [20, 30, 25, 40, 20, 35], [1, 7, 3, 12, 5, 9, 2], [1, 15, 20, 18, 25, 10, 1]
    else:
        dims, rs, ell = [11] * 24, [4, 6, 3], [1] + [9] * 23 + [1]
    N = len(dims)
    Ys = [synth.gaussian_tt(synth.rng_for(10, j), dims, const_ranks(N, r)) for j, r in enumerate(rs)]
    ellc = O.clamp_ranks(dims, ell)
    sk = synth.gaussian_tt(synth.rng_for(11), dims, ellc)
    coeffs = list(synth.rng_for(12).standard_normal(len(Ys)))
    Xo = O.round_sum_randorth(Ys, sk, coeffs)
    Xg = run_sum(Ys, ell, sk, coeffs)
    assert [c.shape for c in Xg] == [c.shape for c in Xo]
    assert rel_diff(Xg, Xo) <= FP64_TOL
    # left-orthogonality of the GPU output
    for c in Xg[:-1]:
        Vc = O.V(c)
        np.testing.assert_allclose(Vc.T @ Vc, np.eye(Vc.shape[1]), atol=1e-12)


def test_single_tt_is_algorithm5():
    dims = [30, 40, 35, 30]
    Y = synth.gaussian_tt(synth.rng_for(20), dims, [1, 12, 20, 12, 1])
    ell = [1, 8, 10, 8, 1]
    sk = synth.gaussian_tt(synth.rng_for(21), dims, ell)
    Xo = O.round_randorth(Y, sk)
    Xg = to_host(tt.tt_round_rand(to_dev(Y), ell, sketch=to_dev(sk)))
    assert rel_diff(Xg, Xo) <= FP64_TOL


def test_x_plus_x_recovers_rank_with_tolerance():
    """spec check: X + X rounds back to rank R (exact recovery, then the
    Section 3.2 truncation removes the oversampled directions)."""
    dims = [16] * 8
    Y = synth.gaussian_tt(synth.rng_for(30), dims, const_ranks(8, 5))
    ell = const_ranks(8, 9)
    sk = synth.gaussian_tt(synth.rng_for(31), dims, ell)
    Xg = run_sum([Y, Y], ell, sk, tol=1e-10)
    assert O.ranks_of(Xg) == const_ranks(8, 5)
    assert O.diff_norm(Xg, synth.scale_tt(Y, 2.0)) <= 1e-12 * 2 * O.norm(Y)


@pytest.mark.parametrize("tol", [1e-2, 1e-6, 1e-9])
def test_tolerance_truncation_parity(tol):
    dims = [20, 25, 20, 25, 20, 25]
    N = len(dims)
    Ys = synth.workload_sum_structured(3, K=6, N=N, I=20, R=4, m=2, delta=1e-5)
    dims = [20] * N
    ell = const_ranks(N, 12)
    sk = synth.gaussian_tt(synth.rng_for(32), dims, ell)
    Xu = O.round_sum_randorth(Ys, sk)
    Xo = O.truncate_left_orthogonal(Xu, tol)
    Xg = run_sum(Ys, ell, sk, tol=tol)
    assert O.ranks_of(Xg) == O.ranks_of(Xo)
    assert rel_diff(Xg, Xo) <= FP64_TOL
    # guarantee of the truncation: ||X_out - X_untruncated|| <= tol ||X_untruncated||
    assert O.diff_norm(Xg, Xu) <= tol * O.norm(Xu) * (1 + 1e-8)


def test_edge_cases_order_one_two_and_clamped_ranks():
    # N = 1: the rounding is the weighted sum of the cores
    Y1 = [synth.gaussian_tt(synth.rng_for(40, j), [9], [1, 1]) for j in range(3)]
    Xg = run_sum(Y1, [1, 1], [np.zeros((1, 9, 1))], coeffs=[1.0, 2.0, -1.0])
    np.testing.assert_allclose(Xg[0], Y1[0][0] + 2 * Y1[1][0] - Y1[2][0], rtol=1e-14, atol=1e-15)
    # N = 2 and a target rank larger than the mode sizes allow (clamped to 3)
    dims = [3, 5]
    Ys = [synth.gaussian_tt(synth.rng_for(41, j), dims, [1, 3, 1]) for j in range(2)]
    ellc = O.clamp_ranks(dims, [1, 10, 1])
    assert ellc == [1, 3, 1]
    sk = synth.gaussian_tt(synth.rng_for(42), dims, ellc)
    Xg = run_sum(Ys, [1, 10, 1], sk)
    Xo = O.round_sum_randorth(Ys, sk)
    assert rel_diff(Xg, Xo) <= FP64_TOL


def test_device_sketch_equals_host_sketch_of_same_seed():
    dims = [12, 15, 12, 15]
    Ys = [synth.gaussian_tt(synth.rng_for(50, j), dims, [1, 4, 5, 4, 1]) for j in range(3)]
    ell = [1, 6, 7, 6, 1]
    seed = 2024
    sk = O.gaussian_sketch_philox(seed, dims, ell)
    Xo = O.round_sum_randorth(Ys, sk)
    Xg = to_host(tt.tt_round_sum_rand([to_dev(Y) for Y in Ys], ell, seed=seed))
    assert rel_diff(Xg, Xo) <= FP64_TOL


@pytest.mark.parametrize("form", ["literal", "structured"])
def test_full_size_sum_of_20_tts_n50(form):
    """The benchmark workload itself (K = 20 summands, N = 50, I = 100, rank 10,
    sketch rank 30, tolerance 1e-8), device sketch from the seed as timed."""
    if form == "literal":
        Ys = synth.workload_sum_literal(1)
    else:
        Ys = synth.workload_sum_structured(1, delta=1e-10)
    dims = [100] * 50
    ell = const_ranks(50, 30)
    seed = 7
    Xg = to_host(tt.tt_round_sum_rand([to_dev(Y) for Y in Ys], ell, seed=seed, tol=1e-8))
    sk = O.gaussian_sketch_philox(seed, dims, ell)
    Xo = O.truncate_left_orthogonal(O.round_sum_randorth(Ys, sk), 1e-8)
    assert O.ranks_of(Xg) == O.ranks_of(Xo)
    assert rel_diff(Xg, Xo) <= FP64_TOL
