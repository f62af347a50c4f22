"""The benchmark's multi-rank logic on CPU with the gloo backend (world size 2).

Ranks run independent replica sets (distinct seeds, no collective in the data
path); the only collective is the max over ranks of the step time.
"""
import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, out):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    r, w, local = bench.dist_env()
    ms = 10.0 + 5.0 * rank
    out[rank] = (r, w, local, bench.reduce_max(ms, w), bench.rank_seed(r))
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_reduce_step_time_and_use_distinct_seeds():
    ctx = mp.get_context("spawn")
    manager = ctx.Manager()
    out = manager.dict()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, out)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    res = dict(out)
    assert sorted(res) == [0, 1]
    for rank in (0, 1):
        r, w, local, mx, seed = res[rank]
        assert (r, w, local) == (rank, 2, rank)
        assert mx == 15.0                     # both ranks see the slowest rank's time
    assert res[0][4] != res[1][4]             # independent replica sets


def test_single_rank_needs_no_process_group():
    import bench
    assert bench.reduce_max(3.5, 1) == 3.5
