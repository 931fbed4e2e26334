"""Batched plans: uneven independent sum roundings in one graph. The
per-problem schedule is bit-wise the eager entry point with its seed; the fused
schedule (grouped launches over all problems, batched thin QRs) equals it to
rounding, with a launch count that does not grow with the number of problems."""
import numpy as np
import pytest
import torch

import synth
from tests._gpu import to_dev, const_ranks

import paper_2110_04393_gb300 as tt

pytestmark = pytest.mark.gpu


def _problems():
    rng = np.random.default_rng(12)
    probs, data = [], []
    for b in range(5):
        N = int(rng.integers(3, 7))
        dims = [int(x) for x in rng.integers(5, 20, size=N)]
        K = int(rng.integers(2, 6))
        Rs = [int(x) for x in rng.integers(2, 6, size=K)]
        ell = int(rng.integers(3, 9))
        tol = 1e-8 if b == 2 else 0.0
        summand_ranks = [const_ranks(N, r) for r in Rs]
        probs.append(dict(dims=dims, summand_ranks=summand_ranks, ells=const_ranks(N, ell), tol=tol))
        data.append([to_dev(synth.gaussian_tt(synth.rng_for(500 + b, j), dims, summand_ranks[j])) for j in range(K)])
    return probs, data


@pytest.mark.parametrize("precision", ["mixed", "fp64"])
@pytest.mark.parametrize("width", [1, 2, 5])
def test_batch_matches_eager_bitwise(precision, width):
    probs, data = _problems()
    plan = tt.BatchRoundingPlan(probs, precision=precision, width=width, fused=0)
    assert plan.launches > 0 and not plan.fused
    seeds = [11, 12, 13, 14, 15]
    for rep in range(2):
        res = plan(data, seeds=seeds)
        for b, (pr, Ys) in enumerate(zip(probs, data)):
            Xe = tt.tt_round_sum_rand(Ys, pr["ells"], seed=seeds[b], tol=pr["tol"], precision=precision)
            torch.cuda.synchronize()
            assert len(Xe) == len(res[b])
            for x, y in zip(res[b], Xe):
                assert x.shape == y.shape and torch.equal(x, y), (rep, b)
    plan.close()


def _fixed_rank(probs):
    return [dict(p, tol=0.0) for p in probs]


@pytest.mark.parametrize("precision", ["mixed", "fp64"])
@pytest.mark.parametrize("width,qr_ctas", [(1, 8), (2, 4), (5, 16)])
def test_fused_batch_matches_eager(precision, width, qr_ctas):
    probs, data = _problems()
    probs = _fixed_rank(probs)
    plan = tt.BatchRoundingPlan(probs, precision=precision, width=width, qr_ctas=qr_ctas)
    assert plan.fused
    seeds = [21, 22, 23, 24, 25]
    for rep in range(2):
        res = plan(data, seeds=seeds)
        plan.status()
        for b, (pr, Ys) in enumerate(zip(probs, data)):
            Xe = tt.tt_round_sum_rand(Ys, pr["ells"], seed=seeds[b], precision=precision)
            assert [tuple(x.shape) for x in res[b]] == [tuple(y.shape) for y in Xe]
            assert _rel_full(res[b], Xe) <= 1e-10, (rep, b)
    plan.close()


def _rel_full(X, Y):
    """Relative distance of the two TT's as tensors (orthogonalized difference TT)."""
    import oracle as O
    from tests._gpu import to_host
    a, b = to_host(X), to_host(Y)
    return O.diff_norm(a, b) / O.norm(b)


def test_fused_launch_count_does_not_grow_with_the_batch():
    probs, data = _problems()
    probs = _fixed_rank(probs)
    one = tt.BatchRoundingPlan(probs[:1], precision="mixed", width=1)
    many = tt.BatchRoundingPlan(probs * 8, precision="mixed", width=1)
    try:
        assert many.fused and one.fused
        maxN = max(len(p["dims"]) for p in probs)
        assert many.launches <= 40 * maxN + 20, many.launches
    finally:
        one.close()
        many.close()


def test_fused_schedule_refuses_a_tolerance():
    probs, data = _problems()
    with pytest.raises(tt.TTError):
        tt.BatchRoundingPlan(probs, precision="mixed", fused=1)


def test_tune_batch_schedule_returns_a_candidate(tmp_path):
    probs, data = _problems()
    probs = _fixed_rank(probs)
    cache = str(tmp_path / "tune.json")
    best, times = tt.tune_batch_schedule(probs, data, precision="mixed", widths=(1, 2), qr_ctas=(4, 8), reps=1,
                                         cache_path=cache)
    assert best in times and set(times) == {(1, 4), (1, 8), (2, 4), (2, 8)}
    import json
    assert json.load(open(cache))
    w, t = tt.tune_batch_width(probs, data, precision="mixed", candidates=(1, 5), reps=1)
    assert w in (1, 5)
