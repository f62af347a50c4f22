"""Helpers shared by the GPU parity tests (CUDA path through the C ABI vs the oracle)."""
from __future__ import annotations

import numpy as np
import pytest


def circ(x):
    return x - np.round(x)


def rad_dist(a, b):
    """Circular distance between phases in [0,1), in radians."""
    return np.abs(circ(np.asarray(a, np.float64) - np.asarray(b, np.float64))) * 2 * np.pi


def coupling_bound_rad(g, K, T, dt, eps=1e-2):
    """Largest phase deviation, in radians, that T steps of a coupling within eps of the
    row norm can cause when the errors add up without amplification: each step moves a
    phase by at most dt K_t eps sum_j |w_ij| cycles more than the exact coupling would.
    A sound bound over horizons where the dynamics do not yet amplify perturbations
    (a few steps at the benchmark couplings)."""
    absw = np.bincount(np.repeat(np.arange(g.n), g.degrees()), weights=np.abs(g.w), minlength=g.n)
    Kt = np.broadcast_to(np.asarray(K, np.float64), (T,)) if np.ndim(K) == 0 else np.asarray(K, np.float64)[:T]
    return 2 * np.pi * float(np.sum(dt * Kt * eps * absw.max()))


def require_gpu():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2505_22631_gb300 import build
    build.build()


def _per_graph(x, count, T):
    xs = x if isinstance(x, list) else [x] * count
    out = []
    for v in xs:
        a = np.asarray(v, np.float32)
        out.append(np.full(T, a, np.float32) if a.ndim == 0 else a[:T])
    return np.stack(out) if T > 0 else np.zeros((count, 0), np.float32)


def gpu_run(graphs, q, K, Ks, Kn, dt, T, R, seed, form="resident", precision="fp32",
            readout_every=0, **kw):
    """Run the CUDA path; graphs is one CSRGraph or a list (a batch).  Schedules are
    scalars, [T] arrays, or lists of those (one per graph)."""
    from paper_2505_22631_gb300 import Problem, Run
    if not isinstance(graphs, (list, tuple)):
        graphs = [graphs]
    probs = [Problem.from_graph(g, q) for g in graphs]
    prob = probs[0] if len(probs) == 1 else Problem.batch(probs)
    G = len(graphs)
    return Run(prob, _per_graph(K, G, T), _per_graph(Ks, G, T), _per_graph(Kn, G, T), dt, T, R,
               seed, form=form, precision=precision, readout_every=readout_every, **kw)


def _f32(x, T):
    """The schedule values exactly as the GPU receives them (float32), widened."""
    a = np.asarray(x, np.float32).astype(np.float64)
    return float(a) if a.ndim == 0 else a[:T]


def oracle_phases(orc, g, q, K, Ks, Kn, dt, T, R, seed, graph=0, replica_offset=0, nthreads=0):
    th, _ = orc.run(g, q, _f32(K, T), _f32(Ks, T), _f32(Kn, T), float(np.float32(dt)), T, R, seed,
                    graph=graph, replica_offset=replica_offset, nthreads=nthreads)
    return th
