"""The N > 1 path of the benchmark on CPU ranks (gloo, world size 2): each
rank draws its own batch (weak scaling, no data-path collective) and the
step time is the maximum over ranks; the per-rank counters are summed."""
import os
import socket

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, ws, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(ws))
    import sys
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    import bench
    import workloads as W
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    spec = W.config_rays("c2", 1000)
    spec.seed = bench.rank_seed(spec.seed, rank)
    F, _ = W.rays(spec, W.config_mesh("c2"))
    t = bench.max_over_ranks(dist, 10.0 + rank, torch.device("cpu"))
    c = bench.sum_over_ranks(dist, [3 + rank, 10 * rank, 2 ** 40], torch.device("cpu"))
    out[rank] = (float(F[:, 0].sum()), t, c)
    dist.destroy_process_group()


def test_two_cpu_ranks_shard_and_reduce():
    ws = 2
    mgr = mp.Manager()
    out = mgr.dict()
    mp.spawn(_worker, args=(ws, _free_port(), out), nprocs=ws, join=True)
    assert out[0][1] == out[1][1] == 11.0            # max over ranks
    assert out[0][2] == out[1][2] == [7, 10, 2 ** 41]  # counters summed exactly (int64)
    assert out[0][0] != out[1][0]                    # distinct batches per rank


def test_single_rank_needs_no_collective():
    import bench
    assert bench.max_over_ranks(None, 3.5, None) == 3.5
    assert bench.sum_over_ranks(None, [4, 0], None) == [4, 0]
    assert bench.rank_seed(2, 0) == 2
