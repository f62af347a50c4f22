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
