"""Batched plans: uneven independent sum roundings in one graph, every problem
bit-wise equal to the eager entry point with its seed, at several chain widths."""
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
    plan = tt.BatchRoundingPlan(probs, precision=precision, width=width)
    assert plan.launches > 0
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


def test_tune_batch_width_returns_a_candidate():
    probs, data = _problems()
    best, times = tt.tune_batch_width(probs, data, precision="mixed", candidates=(1, 5), reps=1)
    assert best in (1, 5) and set(times) == {1, 5}
