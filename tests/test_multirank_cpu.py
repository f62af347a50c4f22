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


def _agg_worker(rank, world, port, out):
    import numpy as np
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    from paper_2505_22631_gb300.distributed import allreduce_schedule_grads, best_across_ranks
    # graph 0: rank 1 holds the larger cut; graph 1: both ranks tie, rank 0 must win
    score = np.array([[3.0, 7.0 + rank, 1.0], [5.0, 2.0, 5.0]])
    # spin value = 10 * rank + graph + replica, so the winner can be read off
    spins = [np.full((3, 4), 10 * rank + g, np.int8) + np.arange(3, dtype=np.int8)[:, None]
             for g in range(2)]
    best, win, sp = best_across_ranks(score, spins, q=2)
    # q >= 3 scores are conflicts: smaller is better
    best3, win3, _ = best_across_ranks(score + rank, spins, q=3)
    grads = allreduce_schedule_grads([np.full((2, 5), float(rank + 1))], replicas=1 + rank)
    out[rank] = (best.tolist(), win.tolist(), [s.tolist() for s in sp], best3.tolist(),
                 win3.tolist(), grads[0].tolist())
    dist.barrier()
    dist.destroy_process_group()


def test_best_cut_and_schedule_gradients_across_two_gloo_ranks():
    ctx = mp.get_context("spawn")
    out = ctx.Manager().dict()
    port = _free_port()
    procs = [ctx.Process(target=_agg_worker, args=(r, 2, port, out)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    assert out[0] == out[1]                   # every rank ends with the same answer
    best, win, sp, best3, win3, g = out[0]
    assert best == [8.0, 5.0] and win == [1, 0]
    assert sp[0] == [11] * 4                  # rank 1, graph 0, replica 1
    assert sp[1] == [1] * 4                   # rank 0, graph 1, replica 0 (first of the tie)
    assert best3 == [1.0, 2.0] and win3 == [0, 0]
    # replica-weighted mean of rank gradients 1 (1 replica) and 2 (2 replicas)
    assert g == [[5.0 / 3.0] * 5] * 2


def test_single_process_aggregation_is_the_local_best():
    import numpy as np
    from paper_2505_22631_gb300.distributed import best_across_ranks
    score = np.array([[1.0, 4.0, 2.0]])
    spins = [np.arange(6, dtype=np.int8).reshape(3, 2)]
    best, win, sp = best_across_ranks(score, spins, q=2)
    assert best.tolist() == [4.0] and win.tolist() == [0] and sp[0].tolist() == [2, 3]
    best, _, sp = best_across_ranks(score, spins, q=3)
    assert best.tolist() == [1.0] and sp[0].tolist() == [0, 1]
