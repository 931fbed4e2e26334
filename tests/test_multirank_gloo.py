"""The multi-GPU path runs independent replicas (no data-path collective): each
rank rounds its own sum and the job's throughput is all ranks' work over the
slowest rank's time. The host logic of that path, run as world_size-2 gloo
ranks on the CPU (no GPU involved)."""
import os
import socket
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out_dir):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    sys.path.insert(0, ROOT)
    import numpy as np
    import torch
    import torch.distributed as dist
    import bench
    import synth
    dist.init_process_group("gloo", rank=rank, world_size=world)
    t = bench.max_over_ranks(10.0 + 5.0 * rank, world, dist, torch.device("cpu"))
    seed = bench.replica_seed(rank)
    Y = synth.workload_sum_literal(seed, K=2, N=3, I=4, R=2)
    np.save(os.path.join(out_dir, f"rank{rank}.npy"), np.concatenate([np.array([t, seed]), Y[0][1].ravel()]))
    dist.barrier()
    dist.destroy_process_group()


def test_replicas_take_the_slowest_rank_and_own_data(tmp_path):
    import numpy as np
    import torch.multiprocessing as mp
    world = 2
    mp.start_processes(_rank_main, args=(world, _free_port(), str(tmp_path)), nprocs=world, start_method="spawn")
    r0, r1 = (np.load(tmp_path / f"rank{r}.npy") for r in range(world))
    assert r0[0] == r1[0] == 15.0                      # every rank sees the max of 10 and 15 ms
    assert r0[1] != r1[1]                              # distinct seeds ...
    assert not np.allclose(r0[2:], r1[2:])             # ... so distinct summands
    sys.path.insert(0, ROOT)
    import bench
    # whole-job throughput: both replicas' work within the slowest time
    assert bench.replica_tflops(3e9, 15.0, 2) == pytest.approx(2 * 3e9 / 15e-3 / 1e12)
    assert bench.max_over_ranks(7.0, 1, None, None) == 7.0
