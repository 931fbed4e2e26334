"""Captured plans (CUDA graph replay) of the sum rounding against the eager
entry point: bit-wise equal results for the same seed, over several replays
with new data, seeds and coefficients, in both precisions and both modes."""
import pytest
import torch

import synth
from tests._gpu import to_dev, const_ranks

import paper_2110_04393_gb300 as tt

pytestmark = pytest.mark.gpu

DIMS = [40, 50, 45, 60, 40, 55]
RANKS = [6, 9, 4, 7]


def _summands(seed):
    N = len(DIMS)
    return [to_dev(synth.gaussian_tt(synth.rng_for(seed, j), DIMS, const_ranks(N, r))) for j, r in enumerate(RANKS)]


def _same(a, b):
    return len(a) == len(b) and all(x.shape == y.shape and torch.equal(x, y) for x, y in zip(a, b))


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
@pytest.mark.parametrize("tol", [0.0, 1e-8])
def test_plan_replays_match_eager_bitwise(precision, tol):
    N = len(DIMS)
    ell = const_ranks(N, 20)
    ranks = [const_ranks(N, r) for r in RANKS]
    plan = tt.SumRoundingPlan(DIMS, ranks, ell, tol=tol, precision=precision)
    assert plan.launches > 0
    for rep, (dseed, sseed) in enumerate([(300, 5), (301, 9), (300, 5)]):
        Yd = _summands(dseed)
        coeffs = None if rep != 1 else [1.0, -0.5, 2.0, 0.25]
        Xp = plan(Yd, seed=sseed, coeffs=coeffs)
        Xe = tt.tt_round_sum_rand(Yd, ell, seed=sseed, tol=tol, coeffs=coeffs, precision=precision)
        torch.cuda.synchronize()
        assert _same(Xp, Xe), (rep, [tuple(x.shape) for x in Xp], [tuple(x.shape) for x in Xe])
    plan.close()


def test_plan_rejects_mismatched_summands():
    N = len(DIMS)
    plan = tt.SumRoundingPlan(DIMS, [const_ranks(N, r) for r in RANKS], const_ranks(N, 20), tol=1e-8)
    Yd = _summands(302)
    with pytest.raises(ValueError):
        plan(Yd[:3])
    plan.close()


@pytest.mark.parametrize("precision,tol", [("mixed", 1e-8), ("fp64", 0.0)])
def test_plan_host_buffers_match_device_run(precision, tol):
    """run_host (one packed copy in, replay, one copy out) returns bit-wise the
    device replay's cores, at the slots of the packed host layout."""
    N = len(DIMS)
    ell = const_ranks(N, 20)
    plan = tt.SumRoundingPlan(DIMS, [const_ranks(N, r) for r in RANKS], ell, tol=tol, precision=precision)
    io, oo, it, ot = plan.host_layout()
    assert len(io) == len(RANKS) * N and len(oo) == N
    R = [const_ranks(N, r) for r in RANKS]
    assert it == sum(Rj[n] * DIMS[n] * Rj[n + 1] for Rj in R for n in range(N))
    assert ot == sum(plan.ell[n] * DIMS[n] * plan.ell[n + 1] for n in range(N))
    assert io[0] == 0 and oo[0] == 0
    Yd = _summands(303)
    h_in = plan.pack_host([[c.cpu() for c in Y] for Y in Yd])
    assert h_in.is_pinned()
    coeffs = [0.5, 1.0, -1.5, 2.0]
    Xh = plan.run_host(h_in, seed=11, coeffs=coeffs)
    Xd = plan(Yd, seed=11, coeffs=coeffs)
    torch.cuda.synchronize()
    assert _same(Xh, [x.cpu() for x in Xd])
    # the second replay reuses the landing buffers
    Xh2 = plan.run_host(h_in, seed=12)
    Xd2 = plan(Yd, seed=12)
    torch.cuda.synchronize()
    assert _same(Xh2, [x.cpu() for x in Xd2])
    with pytest.raises(ValueError):
        plan.run_host(h_in[:10])
    plan.close()


@pytest.mark.parametrize("precision", ["mixed", "fp64"])
def test_full_size_plan_is_the_eager_rounding(precision):
    """The configuration the benchmark times: the captured plan of the 20-TT sum
    (N = 50, I = 100, rank 10, sketch rank 30, tol 1e-8) replays bit-wise the
    eager call that the full-size oracle parity tests check, on device and on
    host buffers."""
    Ys = synth.workload_sum_literal(1)
    N = len(Ys[0])
    dims = [int(c.shape[1]) for c in Ys[0]]
    ranks = [[1] + [int(c.shape[2]) for c in Y] for Y in Ys]
    ell = const_ranks(N, 30)
    Yd = [to_dev(Y) for Y in Ys]
    plan = tt.SumRoundingPlan(dims, ranks, ell, tol=1e-8, precision=precision)
    Xp = plan(Yd, seed=21)
    Xe = tt.tt_round_sum_rand(Yd, ell, seed=21, tol=1e-8, precision=precision)
    torch.cuda.synchronize()
    assert _same(Xp, Xe)
    Xh = plan.run_host(plan.pack_host(Ys), seed=21)
    assert _same(Xh, [x.cpu() for x in Xe])
    plan.close()
