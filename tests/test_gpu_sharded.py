"""Summand-sharded Algorithm 7 on the GPU (tt_round_sum_rand_sharded): two
shards of the summands rounded by two host threads on their own streams of
one GPU, their all-reduce done by the host with CUDA events and stream
waits (no kernel waits on another); every shard ends with the rounding of the
whole sum, equal to the unsharded call, and the shards agree bit for bit."""
import threading

import numpy as np
import pytest
import torch

import oracle as O
import synth
from tests._gpu import to_dev, to_host, const_ranks

import paper_2110_04393_gb300 as tt

pytestmark = pytest.mark.gpu


class _HostAllReduce:
    """Sum over `world` shards in a fixed order (shard 0 adds the others on its
    stream after their events), then every shard copies the sum."""

    def __init__(self, world):
        self.world = world
        self.barrier = threading.Barrier(world)
        self.bufs = [None] * world
        self.events = [None] * world
        self.total = None
        self.done = None

    def for_rank(self, rank):
        def fn(t, stream):
            ev = torch.cuda.Event()
            ev.record(stream)
            self.bufs[rank], self.events[rank] = t, ev
            self.barrier.wait()
            if rank == 0:
                for r in range(1, self.world):
                    stream.wait_event(self.events[r])
                with torch.cuda.stream(stream):
                    tot = self.bufs[0].clone()
                    for r in range(1, self.world):
                        tot += self.bufs[r]
                done = torch.cuda.Event()
                done.record(stream)
                self.total, self.done = tot, done
            self.barrier.wait()
            stream.wait_event(self.done)
            with torch.cuda.stream(stream):
                self.total.record_stream(stream)
                t.copy_(self.total)
            ev2 = torch.cuda.Event()
            ev2.record(stream)
            self.events[rank] = ev2
            self.barrier.wait()                 # the sum is not reused before every copy is enqueued
            if rank == 0:
                for r in range(1, self.world):
                    stream.wait_event(self.events[r])
            self.barrier.wait()
        return fn


@pytest.mark.parametrize("precision,tol", [("fp64", 0.0), ("fp64", 1e-6), ("mixed", 1e-8)])
def test_two_shards_equal_the_unsharded_rounding(precision, tol):
    dims = [12, 14, 10, 12, 14, 12]
    N = len(dims)
    Ys = [synth.gaussian_tt(synth.rng_for(610, j), dims, const_ranks(N, r)) for j, r in enumerate([3, 4, 2, 5, 3])]
    coeffs = [1.0, -0.5, 2.0, 0.25, -1.5]
    ell = O.clamp_ranks(dims, const_ranks(N, 9))
    sk = to_dev(synth.gaussian_tt(synth.rng_for(611), dims, ell))
    Yd = [to_dev(Y) for Y in Ys]
    ref = to_host(tt.tt_round_sum_rand(Yd, ell, sketch=sk, coeffs=coeffs, tol=tol, precision=precision))
    world = 2
    ar = _HostAllReduce(world)
    res, errs = [None] * world, []

    def run(rank):
        try:
            s = torch.cuda.Stream()
            mine = [j for j in range(len(Ys)) if j % world == rank]
            with torch.cuda.stream(s):
                X = tt.tt_round_sum_rand_sharded([Yd[j] for j in mine], ell, ar.for_rank(rank), sketch=sk,
                                                 coeffs=[coeffs[j] for j in mine], tol=tol, precision=precision,
                                                 stream=s)
            s.synchronize()
            res[rank] = to_host(X)
        except Exception as e:
            errs.append(e)
            ar.barrier.abort()

    th = [threading.Thread(target=run, args=(r,)) for r in range(world)]
    for t in th:
        t.start()
    for t in th:
        t.join(timeout=120)
    assert not errs, errs
    for X in res:
        assert O.ranks_of(X) == O.ranks_of(ref)
        assert O.diff_norm(X, ref) <= 1e-11 * O.norm(ref)
    for a, b in zip(res[0], res[1]):
        assert np.array_equal(a, b)
