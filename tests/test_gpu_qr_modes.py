"""The thin-QR implementations behind every rounding (tt_set_qr_mode): the
one-launch cooperative shifted Cholesky QR (default), the one-launch-per-pass
chain, and the Householder TSQR fallback forced for every QR. Each mode must
give the oracle's rounding (Algorithm 7, Section 3.4; any orthonormal basis of
the sketch is a valid step), and the forced fallback must be seen to run
(device counter), including on rank-deficient sketches: X + X with a sketch
rank above the true rank, and the Appendix C Hilbert TT."""
import numpy as np
import pytest

import oracle as O
import synth
from tests._gpu import to_dev, to_host, const_ranks

import paper_2110_04393_gb300 as tt

pytestmark = pytest.mark.gpu
FP64_TOL = 1e-10


@pytest.fixture(autouse=True)
def _restore_mode():
    yield
    tt.set_qr_mode(tt.QR_AUTO)


def rel_diff(A, B):
    return O.diff_norm(A, B) / O.norm(B)


@pytest.mark.parametrize("mode", [0, 1, 2], ids=["coop", "chain", "householder"])
@pytest.mark.parametrize("tol", [0.0, 1e-8])
def test_each_qr_mode_matches_oracle(mode, tol):
    dims = [20, 24, 22, 26, 20, 24]
    N = len(dims)
    Ys = [synth.gaussian_tt(synth.rng_for(150, j), dims, const_ranks(N, r)) for j, r in enumerate([4, 6, 5])]
    ell = O.clamp_ranks(dims, const_ranks(N, 11))
    sk = synth.gaussian_tt(synth.rng_for(151), dims, ell)
    Xo = O.round_sum_randorth(Ys, sk)
    if tol > 0:
        Xo = O.truncate_left_orthogonal(Xo, tol)
    tt.set_qr_mode(mode)
    before = tt.tsqr_fallback_runs()
    Xg = to_host(tt.tt_round_sum_rand([to_dev(Y) for Y in Ys], ell, sketch=to_dev(sk), tol=tol))
    runs = tt.tsqr_fallback_runs() - before
    assert O.ranks_of(Xg) == O.ranks_of(Xo)
    assert rel_diff(Xg, Xo) <= FP64_TOL
    qrs = (N - 1) * (2 if tol > 0 else 1)      # sketch QRs (+ truncation QRs)
    assert runs == (qrs if mode == 2 else 0)


@pytest.mark.parametrize("mode", [0, 2], ids=["coop", "householder"])
def test_rank_deficient_sketch_exact_recovery(mode):
    """X + X of rank 4 with sketch rank 9: every sketch Y_n has rank 4, so the
    thin QR meets exactly rank-deficient blocks."""
    dims = [10] * 6
    Y = synth.gaussian_tt(synth.rng_for(152), dims, const_ranks(6, 4))
    ell = O.clamp_ranks(dims, const_ranks(6, 9))
    sk = synth.gaussian_tt(synth.rng_for(153), dims, ell)
    tt.set_qr_mode(mode)
    before = tt.tsqr_fallback_runs()
    Yd = to_dev(Y)
    Xg = to_host(tt.tt_round_sum_rand([Yd, Yd], ell, sketch=to_dev(sk), tol=1e-10))
    runs = tt.tsqr_fallback_runs() - before
    ref = synth.scale_tt(Y, 2.0)
    assert O.ranks_of(Xg) == const_ranks(6, 4)
    assert O.diff_norm(Xg, ref) <= 1e-11 * O.norm(ref)
    Xo = O.truncate_left_orthogonal(O.round_sum_randorth([Y, Y], sk), 1e-10)
    assert rel_diff(Xg, Xo) <= FP64_TOL
    if mode == 2:
        assert runs == 2 * 5


def test_hilbert_tt_with_forced_fallback():
    """Appendix C: the Hilbert TT has rapidly decaying unfolding spectra, so the
    sketches are numerically rank deficient; the forced Householder path still
    gives the oracle's rounding."""
    dims = [8] * 6
    Y = synth.hilbert_tt(dims, const_ranks(6, 6))
    ell = O.clamp_ranks(dims, const_ranks(6, 8))
    sk = synth.gaussian_tt(synth.rng_for(154), dims, ell)
    tt.set_qr_mode(2)
    before = tt.tsqr_fallback_runs()
    Xg = to_host(tt.tt_round_rand(to_dev(Y), ell, sketch=to_dev(sk), tol=1e-12))
    assert tt.tsqr_fallback_runs() - before == 2 * 5
    Xo = O.truncate_left_orthogonal(O.round_randorth(Y, sk), 1e-12)
    assert O.diff_norm(Xg, Y) <= 1e-11 * O.norm(Y)
    assert O.diff_norm(Xo, Y) <= 1e-11 * O.norm(Y)


def test_plan_in_each_mode_matches_eager():
    dims = [16, 18, 20, 18, 16]
    N = len(dims)
    Ys = [synth.gaussian_tt(synth.rng_for(155, j), dims, const_ranks(N, r)) for j, r in enumerate([3, 5])]
    R = [const_ranks(N, r) for r in (3, 5)]
    ell = O.clamp_ranks(dims, const_ranks(N, 9))
    Yd = [to_dev(Y) for Y in Ys]
    for mode in (0, 1, 2, 3):
        tt.set_qr_mode(mode)
        plan = tt.SumRoundingPlan(dims, R, ell, tol=1e-9, precision="fp64")
        try:
            Xp = to_host(plan(Yd, seed=5))
        finally:
            plan.close()
        Xe = to_host(tt.tt_round_sum_rand(Yd, ell, seed=5, tol=1e-9))
        assert O.ranks_of(Xp) == O.ranks_of(Xe)
        assert rel_diff(Xp, Xe) <= 1e-13


@pytest.mark.parametrize("mode", [0, 1], ids=["coop", "chain"])
@pytest.mark.parametrize("k", [1, 2, 16, 31, 32, 33, 47, 64, 65, 96])
def test_sketch_rank_sizes_match_oracle(mode, k):
    # every width class of the shared-memory Cholesky with inverse (one, two or
    # three 32-lane chunks per column) through the sketch QRs of bonds 1 and 2
    # (100 x k and 12k x k), and no Householder fallback
    dims = [100, 12, 100]
    Y = synth.gaussian_tt(synth.rng_for(160, k), dims, [1, 100, 100, 1])
    ell = O.clamp_ranks(dims, [1, k, k, 1])
    sk = synth.gaussian_tt(synth.rng_for(161, k), dims, ell)
    Xo = O.round_sum_randorth([Y], sk)
    tt.set_qr_mode(mode)
    before = tt.tsqr_fallback_runs()
    Xg = to_host(tt.tt_round_sum_rand([to_dev(Y)], ell, sketch=to_dev(sk)))
    assert tt.tsqr_fallback_runs() == before
    assert O.ranks_of(Xg) == O.ranks_of(Xo)
    assert rel_diff(Xg, Xo) <= FP64_TOL
    for n in range(len(Xg) - 1):
        Vn = O.V(Xg[n])
        assert np.abs(Vn.T @ Vn - np.eye(Vn.shape[1])).max() < 1e-13


def test_pivot_rsqrt_matches_cuda_rsqrt():
    # the QR pivots' reciprocal square root (approximation + third-order
    # correction) against CUDA's rsqrt over the normal range
    max_ulp, ndiff = tt.probe_pivot_rsqrt(1 << 22)
    assert max_ulp <= 1
    assert ndiff <= (1 << 22) // 1000


@pytest.mark.parametrize("tol", [0.0, 1e-8])
def test_fallback_after_breakdown_in_eager_calls_and_plans(tol):
    """Mode 3 marks every cooperative chain failed after its first decision, so
    the Householder fallback (its launches return at once unless the chain's
    device flag is raised) recomputes each QR as after a real breakdown, in
    eager calls and in captured plans alike. Both give the oracle's rounding,
    the plan equals the eager call, and the device run counter rises by the
    number of QRs per call; in the default mode no fallback runs at all."""
    dims = [20, 24, 22, 26, 20, 24]
    N = len(dims)
    Ys = [synth.gaussian_tt(synth.rng_for(170, j), dims, const_ranks(N, r)) for j, r in enumerate([4, 6, 5])]
    R = [const_ranks(N, r) for r in (4, 6, 5)]
    ell = O.clamp_ranks(dims, const_ranks(N, 11))
    sk = O.gaussian_sketch_philox(9, dims, ell)          # the sketch the device draws from seed 9
    Xo = O.round_sum_randorth(Ys, sk)
    if tol > 0:
        Xo = O.truncate_left_orthogonal(Xo, tol)
    Yd = [to_dev(Y) for Y in Ys]
    qrs = (N - 1) * (2 if tol > 0 else 1)
    for mode, expect in ((tt.QR_COOP_THEN_FALLBACK, qrs), (tt.QR_AUTO, 0)):
        tt.set_qr_mode(mode)
        before = tt.tsqr_fallback_runs()
        Xe = to_host(tt.tt_round_sum_rand(Yd, ell, seed=9, tol=tol))
        assert tt.tsqr_fallback_runs() - before == expect
        plan = tt.SumRoundingPlan(dims, R, ell, tol=tol, precision="fp64")
        try:
            before = tt.tsqr_fallback_runs()
            Xp = to_host(plan(Yd, seed=9))
            Xp2 = to_host(plan(Yd, seed=9))
            assert tt.tsqr_fallback_runs() - before == 2 * expect
        finally:
            plan.close()
        for X in (Xe, Xp, Xp2):
            assert O.ranks_of(X) == O.ranks_of(Xo)
            assert rel_diff(X, Xo) <= FP64_TOL
        assert rel_diff(Xp, Xe) <= 1e-13
