"""The named synthetic workloads (graphs + schedules + run shape).

Shapes follow the paper's evaluation (Sec. IV): 800-node Erdos-Renyi max-cut
graphs like G-set G1 (p = 0.06, +1 weights), 2000-node toroidal +-1 grids like
G-set G39-G42, planted 3-colourable graphs for the Potts colouring runs
(Table 2), and larger uneven mixes up to 20000 nodes (Table 1's range).

Solver parameters the paper leaves open (Sec. IV-B gives none) are fixed here:
dt = 0.01, a linear ramp of the injection strength Ks from 0 to 2 over the run,
noise amplitude Kn = 0.1 (the Algorithm 1 form Kn * sqrt(dt) * N(0,1)), and a
constant coupling K = c / mean degree with c = 16 for max-cut (q = 2) and c = 8
for 3-colouring (q = 3).  Sec. IV-B advises the largest K that stays stable; a
sweep of c on these graphs with the CPU oracle put the best final cuts at
c = 16-24 (ER-800), 8-16 (torus) and 16 (ER-2000), and the fewest colouring
conflicts at c = 8, with c = 32 already unstable on the torus.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

from .graphs import CSRGraph, erdos_renyi, gnm, planted_partition, torus

BASE_SEED = 20250528


def linear_ramp(T: int, lo: float, hi: float) -> np.ndarray:
    if T <= 1:
        return np.full(max(T, 0), hi, dtype=np.float32)
    return (lo + (hi - lo) * np.arange(T, dtype=np.float64) / (T - 1)).astype(np.float32)


def constant(T: int, v: float) -> np.ndarray:
    return np.full(T, v, dtype=np.float32)


@dataclass
class Workload:
    name: str
    graphs: list[CSRGraph]
    q: int
    replicas: int
    steps: int
    dt: float
    K: list[np.ndarray]       # per graph, float32[steps]
    Ks: list[np.ndarray]
    Kn: list[np.ndarray]
    seed: int
    notes: str = ""
    extra: dict = field(default_factory=dict)

    @property
    def nnz(self) -> int:
        return sum(g.nnz for g in self.graphs)

    @property
    def nodes(self) -> int:
        return sum(g.n for g in self.graphs)

    def edge_updates(self) -> int:
        """Directed nonzeros x replicas x steps over all graphs."""
        return self.nnz * self.replicas * self.steps


COUPLING_PER_DEGREE = {2: 16.0, 3: 8.0}


def _schedules(graphs, T, q=2, ks_max=2.0, kn=0.1):
    c = COUPLING_PER_DEGREE.get(q, 8.0)
    K = [constant(T, c / g.mean_degree) for g in graphs]
    Ks = [linear_ramp(T, 0.0, ks_max) for _ in graphs]
    Kn = [constant(T, kn) for _ in graphs]
    return K, Ks, Kn


def _c1(steps=None, replicas=None):
    g = erdos_renyi(800, 0.06, BASE_SEED + 0, "+1")
    T = steps or 1000
    K, Ks, Kn = _schedules([g], T)
    return Workload("maxcut_er800_p0.06_R8", [g], 2, replicas or 8, T, 0.01, K, Ks, Kn,
                    BASE_SEED, "G1-shaped Erdos-Renyi max-cut")


def _c2(steps=None, replicas=None):
    g0 = torus(50, 40, BASE_SEED + 1, "pm1")
    g1 = erdos_renyi(2000, 0.01, BASE_SEED + 2, "+1")
    T = steps or 5000
    K, Ks, Kn = _schedules([g0, g1], T)
    return Workload("maxcut_torus50x40_er2000_R1024", [g0, g1], 2, replicas or 1024, T, 0.01,
                    K, Ks, Kn, BASE_SEED, "toroidal +-1 grid and sparse ER, batched")


def _c3(steps=None, replicas=None):
    g = planted_partition(600, 3, 4.7, BASE_SEED + 3)
    T = steps or 10000
    K, Ks, Kn = _schedules([g], T, q=3)
    return Workload("color3_planted600_d4.7_R512", [g], 3, replicas or 512, T, 0.01, K, Ks, Kn,
                    BASE_SEED, "planted 3-colourable Potts colouring")


C4_TORI = [(100, 100), (120, 100), (125, 100), (140, 100), (150, 100), (160, 100), (180, 100),
           (200, 100)]
C4_RANDOM = [(800, 4), (1000, 5), (2000, 6), (3000, 8), (5000, 4), (7000, 6), (8000, 8),
             (10000, 5)]


def _c4(steps=None, replicas=None):
    graphs = []
    for k, (r, c) in enumerate(C4_TORI):
        graphs.append(torus(r, c, BASE_SEED + 100 + k, "pm1"))
    for k, (n, d) in enumerate(C4_RANDOM):
        graphs.append(gnm(n, n * d // 2, BASE_SEED + 200 + k, "+1"))
    T = steps or 5000
    K, Ks, Kn = _schedules(graphs, T)
    return Workload("maxcut_uneven16_R256", graphs, 2, replicas or 256, T, 0.01, K, Ks, Kn,
                    BASE_SEED, "16 uneven graphs, 800-20000 nodes")


def _c4_dense(steps=None, replicas=None):
    """The 16-graph uneven batch plus one all-to-all member, the complete graph on 2000
    nodes with +-1 weights (the shape of the fully connected max-cut instances the
    paper's all-to-all couplings address): the case for choosing the form per graph,
    the dense member on the tensor cores and the rest on the CSR form."""
    graphs = _c4(steps=1).graphs + [erdos_renyi(2000, 1.0, BASE_SEED + 5, "pm1")]
    T = steps or 5000
    K, Ks, Kn = _schedules(graphs, T)
    return Workload("maxcut_uneven16_k2000_R256", graphs, 2, replicas or 256, T, 0.01, K, Ks, Kn,
                    BASE_SEED, "16 uneven graphs and a complete +-1 graph on 2000 nodes")


def _c5(steps=None, replicas=None, count=64):
    graphs = []
    for g in range(count):
        n = int(round(800 + 2200 * g / 63))
        p = 0.06 - 0.05 * g / 63
        graphs.append(erdos_renyi(n, p, BASE_SEED + 300 + g, "pm1"))
    T = steps or 2000
    K, Ks, Kn = _schedules(graphs, T)
    return Workload("schedule_er64_R32", graphs, 2, replicas or 32, T, 0.01, K, Ks, Kn, BASE_SEED,
                    "64 Erdos-Renyi graphs for schedule learning")


def _dense(steps=None, replicas=None):
    g = erdos_renyi(2000, 0.05, BASE_SEED + 4, "+1")
    T = steps or 1000
    K, Ks, Kn = _schedules([g], T)
    return Workload("maxcut_er2000_p0.05_R1024", [g], 2, replicas or 1024, T, 0.01, K, Ks, Kn,
                    BASE_SEED, "denser max-cut graph (mean degree 100), the tensor-core form's case")


WORKLOADS = {
    "er800": _c1,
    "torus_er2000": _c2,
    "planted600": _c3,
    "uneven16": _c4,
    "uneven16_k2000": _c4_dense,
    "er64": _c5,
    "dense2000": _dense,
}


def make_workload(name: str, steps: int | None = None, replicas: int | None = None) -> Workload:
    return WORKLOADS[name](steps=steps, replicas=replicas)
