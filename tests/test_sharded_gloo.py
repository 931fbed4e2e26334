"""Summand-sharded Algorithm 7 (each rank holds part of the summands; the
sketch and the last core are all-reduced; every rank repeats the QR), as the
oracle's host-side restatement run on world_size-2 gloo ranks on the CPU: the
result on every rank equals the unsharded Algorithm 7 on all summands."""
import os
import socket
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _problem():
    import synth
    dims = [6, 7, 5, 6, 7]
    Ys = [synth.gaussian_tt(synth.rng_for(600, j), dims, [1, r, r + 1, r, r, 1]) for j, r in enumerate([2, 3, 4, 2, 3])]
    coeffs = [1.0, -0.5, 2.0, 0.25, -1.5]
    ell = [1, 5, 6, 6, 5, 1]
    sk = synth.gaussian_tt(synth.rng_for(601), dims, ell)
    return Ys, coeffs, sk


def _rank_main(rank, world, port, out_dir):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    sys.path.insert(0, ROOT)
    import torch
    import torch.distributed as dist
    import oracle as O
    dist.init_process_group("gloo", rank=rank, world_size=world)
    Ys, coeffs, sk = _problem()
    mine = [j for j in range(len(Ys)) if j % world == rank]        # uneven shares: 3 and 2 summands

    def allreduce(a):
        t = torch.from_numpy(np.ascontiguousarray(a))
        dist.all_reduce(t)
        return t.numpy()

    X = O.round_sum_randorth_sharded([Ys[j] for j in mine], sk, allreduce, [coeffs[j] for j in mine])
    for n, c in enumerate(X):
        np.save(os.path.join(out_dir, f"rank{rank}_core{n}.npy"), c)
    dist.barrier()
    dist.destroy_process_group()


def test_sharded_rounding_equals_unsharded_on_every_rank(tmp_path):
    import torch.multiprocessing as mp
    sys.path.insert(0, ROOT)
    import oracle as O
    world = 2
    mp.start_processes(_rank_main, args=(world, _free_port(), str(tmp_path)), nprocs=world, start_method="spawn")
    Ys, coeffs, sk = _problem()
    ref = O.round_sum_randorth(Ys, sk, coeffs)
    N = len(ref)
    outs = [[np.load(tmp_path / f"rank{r}_core{n}.npy") for n in range(N)] for r in range(world)]
    for X in outs:
        assert O.ranks_of(X) == O.ranks_of(ref)
        assert O.diff_norm(X, ref) <= 1e-12 * O.norm(ref)
    for a, b in zip(outs[0], outs[1]):
        assert np.array_equal(a, b)                     # the ranks hold the same result bit for bit


def test_single_rank_sharding_is_algorithm_7():
    sys.path.insert(0, ROOT)
    import oracle as O
    Ys, coeffs, sk = _problem()
    X = O.round_sum_randorth_sharded(Ys, sk, lambda a: a, coeffs)
    ref = O.round_sum_randorth(Ys, sk, coeffs)
    for a, b in zip(X, ref):
        assert np.array_equal(a, b)
