"""GB300 (sm_103a) simulator of the oscillator Ising/Potts machine (arXiv 2505.22631).

The C ABI lives in ``include/oim.h`` / ``liboim.so``; ``capi`` binds every entry
point under the same name.  ``Problem`` and ``Run`` below are convenience
wrappers that own the handles and marshal numpy arrays and torch tensors.
"""
from __future__ import annotations

import numpy as np

from . import capi
from .capi import (FORMS, PRECISIONS, OimError, oim_schedule_triangular, oim_create_batch,
                   oim_create_batch_csr, oim_create_problem,
                   oim_debug_derivative, oim_default_opts, oim_destroy_problem, oim_destroy_run,
                   oim_get_phases, oim_last_error, oim_problem_info, oim_readout, oim_rerun,
                   oim_run, oim_run_info, oim_run_sync, oim_version)

__all__ = [
    "Problem", "Run", "simulate", "sweep", "oim_schedule_triangular", "OimError", "FORMS", "PRECISIONS", "oim_create_problem",
    "oim_create_batch", "oim_create_batch_csr", "oim_problem_info", "oim_destroy_problem", "oim_run", "oim_rerun",
    "oim_run_sync", "oim_readout", "oim_run_info", "oim_get_phases", "oim_debug_derivative",
    "oim_destroy_run", "oim_default_opts", "oim_version", "oim_last_error",
]


class Problem:
    """One graph (or a batch of graphs) uploaded to the GPU."""

    def __init__(self, handle, graphs: int, sizes: list[int], q: int, members=()):
        self.handle = handle
        self.graphs = graphs
        self.sizes = list(sizes)
        self.q = q
        self._members = list(members)   # keep batch members alive for their lifetime

    @classmethod
    def from_csr(cls, n, q, row_ptr, col, w=None, flags=0) -> "Problem":
        row_ptr = np.ascontiguousarray(row_ptr, dtype=np.int64) if isinstance(row_ptr, np.ndarray) else row_ptr
        col = np.ascontiguousarray(col, dtype=np.int32) if isinstance(col, np.ndarray) else col
        if isinstance(w, np.ndarray):
            w = np.ascontiguousarray(w, dtype=np.float32)
        nnz = int(col.shape[0])
        h = oim_create_problem(n, q, nnz, row_ptr, col, w, flags)
        return cls(h, 1, [int(n)], q)

    @classmethod
    def from_graph(cls, g, q: int) -> "Problem":
        return cls.from_csr(g.n, q, g.row_ptr, g.col, g.w)

    @classmethod
    def from_graphs(cls, graphs, q: int, flags=0) -> "Problem":
        """A batch of graphs (objects with n, row_ptr, col, w) in one call: the graphs are
        checked and laid out on host threads (oim_create_batch_csr)."""
        cast = [(np.ascontiguousarray(g.row_ptr, dtype=np.int64), np.ascontiguousarray(g.col, dtype=np.int32),
                 None if g.w is None else np.ascontiguousarray(g.w, dtype=np.float32)) for g in graphs]
        h = oim_create_batch_csr([g.n for g in graphs], q, [c.shape[0] for _, c, _ in cast],
                                 [rp for rp, _, _ in cast], [c for _, c, _ in cast],
                                 [w for _, _, w in cast], flags)
        return cls(h, len(graphs), [int(g.n) for g in graphs], q)

    @classmethod
    def batch(cls, problems: list["Problem"]) -> "Problem":
        h = oim_create_batch([p.handle for p in problems])
        return cls(h, len(problems), [s for p in problems for s in p.sizes], problems[0].q,
                   problems)

    @property
    def nodes(self) -> int:
        return sum(self.sizes)

    def close(self):
        if self.handle:
            oim_destroy_problem(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def _stream_ptr(stream):
    if stream is not None:
        return int(getattr(stream, "cuda_stream", stream))
    try:
        import torch
        if torch.cuda.is_available():
            return int(torch.cuda.current_stream().cuda_stream)
    except Exception:
        pass
    return 0


def _schedule(x, graphs, steps):
    """Broadcast a scalar / [steps] / [graphs, steps] schedule to float32 [graphs*steps]."""
    if hasattr(x, "data_ptr") and not isinstance(x, np.ndarray):
        return x   # torch tensor already laid out by the caller
    a = np.asarray(x, dtype=np.float32)
    return np.ascontiguousarray(np.broadcast_to(a, (graphs, steps)) if a.ndim <= 1 or a.shape[0] == 1
                                else a.reshape(graphs, steps)).reshape(-1)


class Run:
    """A simulation of R replicas of every graph of a Problem (owns device state)."""

    def __init__(self, problem: Problem, K, Ks, Kn, dt, steps, replicas, seed, form="auto",
                 precision="auto", readout_every=0, stream=None, use_graph=True,
                 replicas_per_block=0, threads_per_block=0, graph_forms=None, csr_scores=False):
        """graph_forms (form "mixed"): one of "stream" / "gemm" (or the OIM_FORM_* values)
        per graph of the batch.  csr_scores: score every graph with the CSR pass (by
        default dense-form graphs with q = 2 and small integer weights are scored on the
        tensor cores)."""
        self.problem = problem
        o = oim_default_opts()
        o.form = FORMS[form] if isinstance(form, str) else int(form)
        o.precision = PRECISIONS[precision] if isinstance(precision, str) else int(precision)
        o.readout_every = int(readout_every)
        o.stream = _stream_ptr(stream)
        o.use_graph = int(bool(use_graph))
        o.replicas_per_block = int(replicas_per_block)
        o.threads_per_block = int(threads_per_block)
        o.csr_scores = int(bool(csr_scores))
        forms = None
        if graph_forms is not None:
            forms = np.ascontiguousarray([FORMS[f] if isinstance(f, str) else int(f) for f in graph_forms],
                                         dtype=np.int32)
            o.graph_forms = forms.ctypes.data
        self.opts = o
        G = problem.graphs
        self._sched = [_schedule(s, G, steps) for s in (K, Ks, Kn)]
        self.handle = oim_run(problem.handle, *self._sched, dt, steps, replicas, seed, o)
        self.opts.graph_forms = None   # read by oim_run only
        self.replicas = int(replicas)

    def rerun(self, K, Ks, Kn, dt, steps, seed):
        G = self.problem.graphs
        self._sched = [_schedule(s, G, steps) for s in (K, Ks, Kn)]
        oim_rerun(self.handle, *self._sched, dt, steps, seed)

    def info(self) -> dict:
        steps, reps, nro, form, prec = oim_run_info(self.handle)
        return {"steps": steps, "replicas": reps, "n_readouts": nro, "form": form,
                "precision": prec}

    def sync(self):
        oim_run_sync(self.handle)

    def readout(self, spins=True, trace=True, energy=False) -> dict:
        """Host copies: spins [graphs][R][n_g] flattened, score [G, R], best [G], trace, energy."""
        G, R = self.problem.graphs, self.replicas
        nro = self.info()["n_readouts"]
        out = {"score": np.zeros((G, R)), "best_replica": np.zeros(G, dtype=np.int32)}
        if spins:
            out["spins"] = np.zeros(self.problem.nodes * R, dtype=np.int8)
        if trace and nro > 0:
            out["trace"] = np.zeros((G, nro, R))
        if energy:
            out["energy"] = np.zeros((G, R))
        oim_readout(self.handle, out.get("spins"), out["score"], out["best_replica"],
                    out.get("trace"), out.get("energy"))
        if spins:
            flat, parts, off = out["spins"], [], 0
            for n in self.problem.sizes:
                parts.append(flat[off:off + n * R].reshape(R, n))
                off += n * R
            out["spins"] = parts
        return out

    def phases(self) -> list[np.ndarray]:
        R = self.replicas
        flat = np.zeros(self.problem.nodes * R, dtype=np.float32)
        oim_get_phases(self.handle, flat)
        parts, off = [], 0
        for n in self.problem.sizes:
            parts.append(flat[off:off + n * R].reshape(R, n))
            off += n * R
        return parts

    def close(self):
        if self.handle:
            oim_destroy_run(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def simulate(problem: Problem, K, Ks, Kn, dt, steps, replicas, seed, **kw) -> Run:
    return Run(problem, K, Ks, Kn, dt, steps, replicas, seed, **kw)


def sweep(problem: Problem, K_values, Ks_max_values, Kn, dt, steps, replicas, seed, periods=0, **kw):
    """Parameter sweep (the paper's K x Ks_max study, Sec. IV-B) as one batched launch.

    Every (K, Ks_max) pair becomes one graph of a batch of copies of `problem` (one
    graph) with its own schedules: constant K, and Ks a linear ramp to Ks_max
    (periods == 0) or the triangular waveform with `periods` periods.  Returns the
    Run; graph g of the batch is pair g in row-major (K, Ks_max) order.
    """
    if problem.graphs != 1:
        raise ValueError("sweep takes a single-graph problem")
    pairs = [(k, s) for k in K_values for s in Ks_max_values]
    batch = Problem.batch([problem] * len(pairs))
    K = np.stack([np.full(steps, k, np.float32) for k, _ in pairs])
    if periods > 0:
        Ks = np.stack([oim_schedule_triangular(steps, s, periods) for _, s in pairs])
    else:
        ramp = np.arange(steps, dtype=np.float64) / max(steps - 1, 1)
        Ks = np.stack([(s * ramp).astype(np.float32) for _, s in pairs])
    Kn_ = np.broadcast_to(np.asarray(Kn, np.float32), (len(pairs), steps)).copy()
    run = Run(batch, K, Ks, Kn_, dt, steps, replicas, seed, **kw)
    run.pairs = pairs
    return run
