"""Rank-level aggregation for runs sharded by replica across processes.

Replicas (and the graphs of a batch) are independent trajectories, so ranks share
nothing while they simulate: each rank runs its own replica set under its own
seed.  What crosses ranks is the result only:

* ``best_across_ranks``: the best score of every graph over all ranks' replicas
  (max cut for q = 2, fewest conflicts for q >= 3, Eq. 1-2) and the spins of the
  replica that reached it, taken from the lowest rank that holds the best score;
* ``allreduce_schedule_grads``: the sum over ranks of the per-step schedule
  gradients of the replica-mean loss (each rank's mean weighted by its replica
  count), for the adjoint of Eq. 5 run sharded.

Both are plain ``torch.distributed`` collectives on host tensors (gloo) or CUDA
tensors (NCCL); with one process they return their input unchanged.
"""
from __future__ import annotations

import numpy as np
import torch


def _dist():
    import torch.distributed as dist
    return dist if dist.is_available() and dist.is_initialized() else None


def _device_for(dist):
    return torch.device("cuda", torch.cuda.current_device()) \
        if dist.get_backend() == "nccl" else torch.device("cpu")


def best_across_ranks(score: np.ndarray, spins: list[np.ndarray], q: int):
    """Best score per graph over every rank's replicas, with the winning spins.

    score: [graphs, replicas] this rank's scores (float64); spins: one
    [replicas, n_g] int8 array per graph.  Returns (best [graphs] float64,
    rank [graphs] int64, spins list of [n_g] int8), identical on every rank.
    """
    score = np.asarray(score, np.float64)
    G = score.shape[0]
    sign = 1.0 if q == 2 else -1.0             # larger is better after the sign flip
    local_r = np.argmax(sign * score, axis=1)
    local_best = sign * score[np.arange(G), local_r]
    dist = _dist()
    if dist is None or dist.get_world_size() == 1:
        return (sign * local_best, np.zeros(G, np.int64),
                [spins[g][local_r[g]].copy() for g in range(G)])
    dev = _device_for(dist)
    rank, world = dist.get_rank(), dist.get_world_size()
    best = torch.from_numpy(local_best.copy()).to(dev)
    dist.all_reduce(best, op=dist.ReduceOp.MAX)
    # the lowest rank that holds the best score wins (ties broken deterministically)
    cand = torch.from_numpy(np.where(local_best == best.cpu().numpy(), rank, world)
                            .astype(np.int64)).to(dev)
    dist.all_reduce(cand, op=dist.ReduceOp.MIN)
    winner = cand.cpu().numpy()
    out = []
    for g in range(G):
        buf = torch.from_numpy(spins[g][local_r[g]].astype(np.int8)).to(dev) if winner[g] == rank \
            else torch.zeros(spins[g].shape[1], dtype=torch.int8, device=dev)
        dist.broadcast(buf, src=int(winner[g]))
        out.append(buf.cpu().numpy())
    return sign * best.cpu().numpy(), winner.astype(np.int64), out


def allreduce_schedule_grads(grads, replicas: int):
    """Combine per-rank gradients of replica-mean losses into the gradient of the
    mean over all ranks' replicas.  grads: arrays [graphs, steps] (float64)."""
    dist = _dist()
    if dist is None or dist.get_world_size() == 1:
        return [np.asarray(g, np.float64) for g in grads]
    dev = _device_for(dist)
    total = torch.tensor([float(replicas)], dtype=torch.float64, device=dev)
    dist.all_reduce(total)
    out = []
    for g in grads:
        t = torch.from_numpy(np.asarray(g, np.float64) * replicas).to(dev)
        dist.all_reduce(t)
        out.append((t / total).cpu().numpy())
    return out
