"""Seeded synthetic inputs: graphs in CSR form, schedules and the named workloads.

This module holds no arithmetic of the oscillator method.  It produces the
inputs that both the GPU library and the CPU oracle consume, so that tests and
the benchmark feed the two sides identical data.  The graphs stand in for the
G-set max-cut and SATLIB colouring instances of the paper's evaluation
(Sec. IV, Tables 1-2), which are not available here: they take those suites'
shapes (sizes, densities, +1 / +-1 weights, toroidal grids, planted
3-colourable graphs), not their items.
"""
from .graphs import (CSRGraph, csr_from_edges, erdos_renyi, gnm, planted_partition, torus,
                     cycle, complete, complete_bipartite, petersen, from_dense,
                     sherrington_kirkpatrick)
from .configs import WORKLOADS, Workload, linear_ramp, constant, make_workload

__all__ = [
    "CSRGraph", "csr_from_edges", "erdos_renyi", "gnm", "planted_partition", "torus", "cycle",
    "complete", "complete_bipartite", "petersen", "from_dense", "sherrington_kirkpatrick",
    "WORKLOADS", "Workload",
    "linear_ramp", "constant", "make_workload",
]
