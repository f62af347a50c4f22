"""Learning the annealing schedules K(t), Ks(t), Kn(t) by gradient descent.

The paper fixes the schedules by hand (a constant coupling, a ramped or
triangular injection strength, Sec. III-IV).  Here they are learned: each
schedule is a piecewise-linear curve through a few knots, shared by every graph
of a batch (the coupling rescaled per graph by 1 / mean degree, so that the
same curve transfers to graphs of other sizes and degrees), and the knots
follow Adam on the relaxed energy at the end of the run (Eq. 6), averaged over
replicas and normalised per graph by its total absolute weight.  Gradients come
from the library's adjoint (``oim_backward``) through ``schedule_loss``.
"""
from __future__ import annotations

import math

import numpy as np
import torch

from .autograd import schedule_loss


def interp_matrix(steps: int, knots: int) -> torch.Tensor:
    """[steps, knots] weights of linear interpolation between equally spaced knots
    (knot 0 at step 0, the last knot at step steps - 1)."""
    if knots < 2 or steps < 1:
        raise ValueError("need at least two knots and one step")
    pos = np.arange(steps, dtype=np.float64) * (knots - 1) / max(steps - 1, 1)
    lo = np.minimum(np.floor(pos).astype(np.int64), knots - 2)
    frac = pos - lo
    m = np.zeros((steps, knots))
    m[np.arange(steps), lo] = 1.0 - frac
    m[np.arange(steps), lo + 1] = frac
    return torch.from_numpy(m)


def _inv_softplus(x: np.ndarray) -> np.ndarray:
    x = np.maximum(np.asarray(x, np.float64), 1e-4)
    return x + np.log(-np.expm1(-x))


class ScheduleModel(torch.nn.Module):
    """Positive piecewise-linear schedules: K(t) = k_g * softplus(a(t)),
    Ks(t) = softplus(b(t)), Kn(t) = softplus(c(t)), knots a, b, c learned, k_g = 1 / mean
    degree of graph g."""

    def __init__(self, steps: int, knots: int, coupling_scale, K0: float = 16.0,
                 Ks_max0: float = 2.0, Kn0: float = 0.1):
        super().__init__()
        self.steps = int(steps)
        self.register_buffer("M", interp_matrix(steps, knots))
        self.register_buffer("scale", torch.as_tensor(np.asarray(coupling_scale, np.float64)).reshape(-1, 1))
        ramp = np.linspace(0.0, Ks_max0, knots)
        self.a = torch.nn.Parameter(torch.from_numpy(_inv_softplus(np.full(knots, K0))))
        self.b = torch.nn.Parameter(torch.from_numpy(_inv_softplus(ramp)))
        self.c = torch.nn.Parameter(torch.from_numpy(_inv_softplus(np.full(knots, Kn0))))

    def forward(self, scale=None):
        """[graphs, steps] float32 schedules (K, Ks, Kn) for the training graphs, or for
        graphs with the given coupling scales (1 / mean degree each)."""
        sp = torch.nn.functional.softplus
        sc = self.scale if scale is None else \
            torch.as_tensor(np.asarray(scale, np.float64)).reshape(-1, 1)
        K = sc * (self.M @ sp(self.a)).reshape(1, -1)
        Ks = (self.M @ sp(self.b)).reshape(1, -1).expand(sc.shape[0], -1)
        Kn = (self.M @ sp(self.c)).reshape(1, -1).expand(sc.shape[0], -1)
        return K.float(), Ks.float().contiguous(), Kn.float().contiguous()

    def schedules_for(self, graphs):
        """The learned curves applied to other graphs (held-out evaluation)."""
        return self.forward([1.0 / max(g.mean_degree, 1e-9) for g in graphs])


def normalised_loss(problem, graphs, model, dt, replicas, seed, checkpoint_every=100):
    """Mean over graphs of mean_r E_g(theta_T) / sum_{i<j} |w_ij| (in [-1, 1])."""
    K, Ks, Kn = model.schedules_for(graphs)
    L = schedule_loss(problem, K, Ks, Kn, dt, replicas, seed, checkpoint_every)
    wabs = torch.tensor([float(np.abs(g.w).sum()) / 2 for g in graphs], dtype=torch.float64)
    return (L / wabs).mean()


def learn_schedules(problem, graphs, steps: int, replicas: int, dt: float = 0.01, iters: int = 20,
                    lr: float = 0.05, knots: int = 8, seed: int = 1, K0: float = 16.0,
                    Ks_max0: float = 2.0, Kn0: float = 0.1, checkpoint_every: int = 100,
                    fresh_noise: bool = True):
    """Fit the schedules on `problem` (a batch of `graphs`, CSRGraph-like objects with
    mean_degree and w).  Returns (model, history of normalised losses).  With
    fresh_noise each iteration draws a new seed (stochastic gradient over the noise)."""
    scale = [1.0 / max(g.mean_degree, 1e-9) for g in graphs]
    model = ScheduleModel(steps, knots, scale, K0, Ks_max0, Kn0)
    opt = torch.optim.Adam(model.parameters(), lr=lr)
    history = []
    for it in range(iters):
        opt.zero_grad()
        loss = normalised_loss(problem, graphs, model, dt, replicas,
                               seed + it if fresh_noise else seed, checkpoint_every)
        loss.backward()
        opt.step()
        v = float(loss.detach())
        if not math.isfinite(v):
            raise FloatingPointError("schedule loss is not finite")
        history.append(v)
    return model, history


def evaluate(problem, graphs, K, Ks, Kn, dt, replicas, seed, readout_every=50):
    """Run the given [graphs, steps] schedules on `problem` (autotuned form) and return,
    per graph, the best score over replicas at each readout ([graphs, readouts])."""
    from . import Run
    K, Ks, Kn = (np.ascontiguousarray(np.asarray(x.detach() if hasattr(x, "detach") else x,
                                                 np.float32)) for x in (K, Ks, Kn))
    steps = K.shape[1]
    run = Run(problem, K, Ks, Kn, dt, steps, replicas, seed, readout_every=readout_every)
    tr = run.readout(spins=False)["trace"]
    run.close()
    return tr.max(axis=2) if problem.q == 2 else tr.min(axis=2)


def _first_hit(best_per_readout, target, readout_every):
    hit = np.nonzero(best_per_readout >= target)[0]
    return None if hit.size == 0 else int(hit[0] + 1) * readout_every


def demo(count: int = 64, steps: int = 2000, replicas: int = 32, iters: int = 15, lr: float = 0.05,
         knots: int = 8, eval_replicas: int = 128, seed: int = 1):
    """Learn schedules on the even-indexed graphs of the 64-graph Erdos-Renyi family
    (n = 800-3000, p = 0.06-0.01, weights +-1) and compare them with the hand schedules
    (K = 16 / mean degree, Ks ramped 0 -> 2, Kn = 0.1) on the odd-indexed, held-out
    graphs with unseen noise: final best cut and steps to 99 % of the better final
    best cut of the two, per graph.  Returns a dict (printed as JSON by __main__)."""
    import time

    from . import Problem
    from workloads import make_workload
    w = make_workload("er64", steps=steps, replicas=replicas)
    graphs = w.graphs[:count]
    train = [g for k, g in enumerate(graphs) if k % 2 == 0]
    held = [g for k, g in enumerate(graphs) if k % 2 == 1]
    ptrain = Problem.batch([Problem.from_graph(g, 2) for g in train])
    pheld = Problem.batch([Problem.from_graph(g, 2) for g in held])
    t0 = time.perf_counter()
    model, hist = learn_schedules(ptrain, train, steps, replicas, w.dt, iters=iters, lr=lr, knots=knots,
                                  seed=seed)
    t_train = time.perf_counter() - t0
    init = ScheduleModel(steps, knots, [1.0], 16.0, 2.0, 0.1)
    re = 50
    with torch.no_grad():
        b0 = evaluate(pheld, held, *init.schedules_for(held), w.dt, eval_replicas, 9001, re)
        b1 = evaluate(pheld, held, *model.schedules_for(held), w.dt, eval_replicas, 9001, re)
    rows = []
    for gi in range(len(held)):
        target = 0.99 * max(b0[gi, -1], b1[gi, -1])
        rows.append({"hand": {"final_best": float(b0[gi, -1]), "steps_to_99pct": _first_hit(b0[gi], target, re)},
                     "learned": {"final_best": float(b1[gi, -1]),
                                 "steps_to_99pct": _first_hit(b1[gi], target, re)}})

    def mean_steps(key):
        v = [r[key]["steps_to_99pct"] for r in rows]
        return None if any(x is None for x in v) else float(np.mean(v))

    with torch.no_grad():
        K, Ks, Kn = model(np.ones(1))
    return {"train_graphs": len(train), "held_out_graphs": len(held), "steps": steps,
            "train_replicas": replicas, "eval_replicas": eval_replicas, "iters": iters,
            "train_seconds": t_train, "loss_history": hist,
            "held_out": {"hand_mean_final_best": float(b0[:, -1].mean()),
                         "learned_mean_final_best": float(b1[:, -1].mean()),
                         "learned_better_or_equal": int(np.sum(b1[:, -1] >= b0[:, -1])),
                         "hand_mean_steps_to_99pct": mean_steps("hand"),
                         "learned_mean_steps_to_99pct": mean_steps("learned")},
            "learned_knots": {"K_times_mean_degree": K[0, ::max(1, steps // (knots - 1))].tolist(),
                              "Ks": Ks[0, ::max(1, steps // (knots - 1))].tolist(),
                              "Kn": Kn[0, ::max(1, steps // (knots - 1))].tolist()}}


if __name__ == "__main__":
    import json
    import os
    import sys
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    print(json.dumps(demo()), flush=True)
