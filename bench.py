#!/usr/bin/env python
"""Benchmark of the oscillator Ising machine hot path on GB300.

One bench step = one full simulation of the workload: every Euler-Maruyama step
of every replica of every graph, with the periodic readout and cut scoring
(the whole hot path), from the initial Philox draw to the final scores.
Default workload: the batched max-cut case, a 50x40 toroidal +-1 grid and an
Erdos-Renyi G(2000, 0.01) graph, 1024 replicas each, 5000 steps.

Prints one JSON line (rank 0).  `value` is edge-updates/s (directed CSR nonzeros
x replicas x steps per second) over all ranks; ranks run independent replicas
(weak scaling, no collective in the data path).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from workloads import make_workload  # noqa: E402

PEAKS_FALLBACK = {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0}
L2_FLUSH_BYTES = 256 << 20


def load_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            p = json.load(f)
        p["source"] = "measured"
        return p
    except Exception:
        p = dict(PEAKS_FALLBACK)
        p["source"] = "fallback"
        return p


CSRC = "paper_2505_22631_gb300/csrc/"
KERNEL_SOURCES = {
    "resident": [CSRC + "step_resident.cu", CSRC + "oim_device.cuh"],
    "stream": [CSRC + "step_stream.cu", CSRC + "oim_device.cuh"],
    "gemm": [CSRC + "gemm_step.cu", CSRC + "tc_common.cuh", CSRC + "oim_device.cuh"],
}


def kernel_source_hash(kernel):
    """sha1 prefix of the source files that define `kernel`."""
    import hashlib
    fam = "resident" if kernel.startswith("resident") else ("gemm" if kernel.startswith("gemm") else "stream")
    h = hashlib.sha1()
    for f in KERNEL_SOURCES[fam]:
        with open(os.path.join(ROOT, f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def profiled_traffic(kernel, workload):
    """DRAM bytes per launch of `kernel` on `workload` from a committed ncu summary,
    or None when no summary matches the current kernel sources."""
    path = os.path.join(ROOT, "profiles", "dram_traffic.txt")
    if not os.path.exists(path):
        return None
    want = kernel_source_hash(kernel)
    for line in open(path):
        if line.startswith("#") or not line.strip():
            continue
        f = dict(kv.split("=", 1) for kv in line.split())
        if f.get("kernel") == kernel and f.get("workload") == workload and f.get("sources") == want:
            return float(f["dram_bytes_per_launch"])
    return None


def rank_seed(rank: int) -> int:
    """Seed of a rank's replica set: ranks simulate independent replicas (weak scaling)."""
    return 1000 * (rank + 1)


def reduce_max(value: float, world: int, device="cpu") -> float:
    """Max over ranks of a per-rank scalar (the step time), on the initialised process group."""
    if world <= 1:
        return float(value)
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", str(rank)))
    return rank, world, local


class ClockSampler:
    """nvidia-smi clocks / throttle reasons sampled every 200 ms while running."""

    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []
        self.thread = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={self.QUERY}", "--format=csv,noheader,nounits",
                 "-i", str(self.gpu), "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None
            return
        self.thread = threading.Thread(target=self._read, daemon=True)
        self.thread.start()

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        if self.thread:
            self.thread.join(timeout=2)
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [x.strip() for x in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def schedules(w):
    K = np.stack(w.K).astype(np.float32)
    Ks = np.stack(w.Ks).astype(np.float32)
    Kn = np.stack(w.Kn).astype(np.float32)
    return K, Ks, Kn


def stretched(w, factor):
    """The workload's schedules stretched over factor x steps (same shape in time)."""
    T = w.steps * factor
    idx = np.minimum(np.arange(T) // factor, w.steps - 1)
    K, Ks, Kn = schedules(w)
    return np.ascontiguousarray(K[:, idx]), np.ascontiguousarray(Ks[:, idx]), np.ascontiguousarray(Kn[:, idx]), T


def cpu_oracle_sample(w, seconds_hint=15.0):
    """Time the FP64 oracle on this host's cores on a bounded sample of the workload."""
    import oracle
    cores = len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else os.cpu_count()
    oracle.build()
    K, Ks, Kn = schedules(w)
    # calibrate with a short run, then size the sample to about seconds_hint
    R_s = max(1, cores)
    T_cal = 50
    t0 = time.perf_counter()
    for gi, g in enumerate(w.graphs):
        oracle.run(g, w.q, K[gi, :T_cal].astype(np.float64), Ks[gi, :T_cal].astype(np.float64),
                   Kn[gi, :T_cal].astype(np.float64), float(np.float32(w.dt)), T_cal, R_s, 1,
                   graph=gi, nthreads=cores)
    cal = time.perf_counter() - t0
    T_s = int(min(w.steps, max(T_cal, T_cal * seconds_hint / max(cal, 1e-6))))
    t0 = time.perf_counter()
    for gi, g in enumerate(w.graphs):
        oracle.run(g, w.q, K[gi, :T_s].astype(np.float64), Ks[gi, :T_s].astype(np.float64),
                   Kn[gi, :T_s].astype(np.float64), float(np.float32(w.dt)), T_s, R_s, 1,
                   graph=gi, nthreads=cores)
    el = time.perf_counter() - t0
    edge_updates = sum(g.nnz for g in w.graphs) * R_s * T_s
    # the same oracle on one core: one replica, a tenth of the steps
    T_1 = max(1, T_s // 10)
    t0 = time.perf_counter()
    for gi, g in enumerate(w.graphs):
        oracle.run(g, w.q, K[gi, :T_1].astype(np.float64), Ks[gi, :T_1].astype(np.float64),
                   Kn[gi, :T_1].astype(np.float64), float(np.float32(w.dt)), T_1, 1, 1,
                   graph=gi, nthreads=1)
    el_1 = time.perf_counter() - t0
    one_core = sum(g.nnz for g in w.graphs) * T_1 / el_1
    return {"value": edge_updates / el, "unit": "edge-updates/s", "cores": cores, "kind": "oracle",
            "sample": f"all {len(w.graphs)} graphs, {R_s} replicas, first {T_s} of {w.steps} steps "
                      f"(FP64 C oracle, OpenMP over replicas), {el:.1f} s",
            "single_core": {"value": one_core, "unit": "edge-updates/s",
                            "sample": f"all graphs, 1 replica, first {T_1} steps, {el_1:.1f} s"}}


def run_reference(args):
    """The reference arm: the FP64 CPU oracle, timed on this host's cores."""
    rank, world, _ = dist_env()
    if rank != 0:
        return
    import oracle
    w = make_workload(args.workload)
    cores = len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else os.cpu_count()
    oracle.build()
    K, Ks, Kn = schedules(w)
    R_s = max(1, cores)
    # size one reference step to about 8 s of host time
    T_cal = 20
    t0 = time.perf_counter()
    for gi, g in enumerate(w.graphs):
        oracle.run(g, w.q, K[gi, :T_cal].astype(np.float64), Ks[gi, :T_cal].astype(np.float64),
                   Kn[gi, :T_cal].astype(np.float64), float(np.float32(w.dt)), T_cal, R_s, 1,
                   graph=gi, nthreads=cores)
    cal = time.perf_counter() - t0
    T_s = int(min(w.steps, max(T_cal, T_cal * 8.0 / max(cal, 1e-6))))

    def step(seed):
        for gi, g in enumerate(w.graphs):
            oracle.run(g, w.q, K[gi, :T_s].astype(np.float64), Ks[gi, :T_s].astype(np.float64),
                       Kn[gi, :T_s].astype(np.float64), float(np.float32(w.dt)), T_s, R_s, seed,
                       graph=gi, nthreads=cores)

    for k in range(args.warmup):
        step(100 + k)
    times = []
    for k in range(args.steps):
        t0 = time.perf_counter()
        step(1 + k)
        times.append(time.perf_counter() - t0)
    per = float(np.mean(times))
    edge_updates = sum(g.nnz for g in w.graphs) * R_s * T_s
    value = edge_updates / per
    sample = (f"all {len(w.graphs)} graphs, {R_s} replicas, first {T_s} of {w.steps} steps "
              f"per reference step (FP64 C oracle, OpenMP over replicas)")
    line = {
        "impl": "reference", "metric": "edge-updates/s", "value": value, "unit": "edge-updates/s",
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup, "ms_per_step": per * 1e3,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic", "config": {"workload": w.name, "replicas_sampled": R_s,
                                        "euler_steps_sampled": T_s},
        "cpu_baseline": {"value": value, "unit": "edge-updates/s", "cores": cores, "kind": "oracle",
                         "sample": sample},
        "e2e": {"value": value, "unit": "edge-updates/s", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def first_hit(trace_best, target):
    """Index of the first readout whose best score reaches target (None if never)."""
    hit = np.nonzero(trace_best >= target)[0]
    return int(hit[0]) if hit.size else None


def kernels_per_run(form, steps, readout_every, dense_members=0):
    """Kernels of this library that one run enqueues (memsets and copies excluded)."""
    readouts = steps // readout_every if readout_every > 0 else 0
    # the per-step forms first store the run's seed on the device (one tiny kernel)
    if form == 2:          # resident: one launch covers every step and readout
        return 1
    if form == 3:          # dense: init, a step kernel per step, relayout + spins + score per readout,
        return 1 + 1 + steps + 3 * readouts + 1   # final relayout
    if form == 5:          # persistent: init, one launch per readout period, spins + score per readout
        return 1 + 1 + max(readouts, 1) + 2 * readouts
    if form == 4:          # mixed: inits, the CSR step and one step per dense member each step,
        nd = dense_members  # the dense relayouts + spins + score per readout, final relayouts
        return 1 + (1 + nd) + (1 + nd) * steps + (2 + nd) * readouts + nd
    return 1 + 1 + steps + 2 * readouts   # stream: init, a step kernel per step, spins + score per readout


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="torus_er2000")
    ap.add_argument("--form", default="auto")
    ap.add_argument("--graph-forms", default="",
                    help="with --form mixed: stream or gemm per graph, comma-separated")
    ap.add_argument("--precision", default="auto")
    ap.add_argument("--readout-every", type=int, default=50)
    ap.add_argument("--e2e-steps", type=int, default=3)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-quality", action="store_true")
    ap.add_argument("--quality-seeds", type=int, default=8,
                    help="seeds of the time-to-99%% comparison (mean and 95%% CI)")
    ap.add_argument("--euler-steps", type=int, default=0, help="override the workload's steps")
    ap.add_argument("--replicas", type=int, default=0, help="override the workload's replicas")
    ap.add_argument("--adjoint", action="store_true",
                    help="time the checkpointed forward run plus oim_backward (schedule gradients)")
    ap.add_argument("--checkpoint-every", type=int, default=0,
                    help="adjoint: checkpoint period (0: every step, with each step's coupling sums, "
                         "when that fits in device memory, else 100)")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3

    if args.impl == "reference":
        run_reference(args)
        return

    import torch
    from paper_2505_22631_gb300 import Problem, Run, build, capi

    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    build.build()
    capi.load()

    if args.adjoint:
        run_adjoint(args, rank, world)
        return

    w = make_workload(args.workload, steps=args.euler_steps or None,
                      replicas=args.replicas or None)
    K, Ks, Kn = schedules(w)
    dK, dKs, dKn = (torch.from_numpy(a).cuda() for a in (K, Ks, Kn))
    problems = [Problem.from_graph(g, w.q) for g in w.graphs]
    prob = Problem.batch(problems) if len(problems) > 1 else problems[0]
    stream = torch.cuda.current_stream()
    seed_base = rank_seed(rank)
    form, precision, rpb, threads = args.form, args.precision, 0, 0
    tuned = None
    if args.form == "auto":
        # the library's autotuner times candidate forms / block shapes on short probes
        policy = capi.OIM_PREC_FP32 if args.precision == "fp32" else capi.OIM_PREC_AUTO
        o, us = capi.oim_autotune(prob.handle, w.replicas, policy, 200)
        form, precision, rpb, threads = o.form, o.precision, o.replicas_per_block, o.threads_per_block
        graph_forms = capi.graph_forms_of(o, len(w.graphs))
        tuned = {"form": o.form, "precision": o.precision, "replicas_per_block": rpb,
                 "threads_per_block": threads, "probe_us_per_step": us, "graph_forms": graph_forms}
    else:
        graph_forms = [capi.FORMS[f] for f in args.graph_forms.split(",")] if args.graph_forms else None
    run = Run(prob, dK, dKs, dKn, w.dt, w.steps, w.replicas, seed_base, form=form,
              precision=precision, readout_every=args.readout_every, stream=stream,
              replicas_per_block=rpb, threads_per_block=threads, graph_forms=graph_forms)
    info = run.info()
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device="cuda")

    for k in range(args.warmup):
        run.rerun(dK, dKs, dKn, w.dt, w.steps, seed_base + 1 + k)
    run.sync()

    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    sampler = ClockSampler(local)
    sampler.start()
    starts = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    ends = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    t_wall = time.perf_counter()
    for k in range(args.steps):
        flush.fill_(float(k))                 # L2 flush between timed steps, outside the events
        starts[k].record(stream)
        run.rerun(dK, dKs, dKn, w.dt, w.steps, seed_base + 100 + k)
        ends[k].record(stream)
    torch.cuda.synchronize()
    if world > 1:
        torch.distributed.barrier()
    wall = time.perf_counter() - t_wall
    clocks = sampler.stop()
    ms = [s.elapsed_time(e) for s, e in zip(starts, ends)]
    ms_step = float(np.mean(ms))
    ms_step = reduce_max(ms_step, world, device="cuda")
    edge_updates = w.edge_updates() * world
    value = edge_updates / (ms_step / 1e3)
    node_updates_per_s = w.nodes * w.replicas * w.steps * world / (ms_step / 1e3)

    # roofline of the dominant kernel.  CSR forms: algorithmic bytes per
    # node-replica-step are the state a step must move if nothing stays on chip:
    # read and write the phase (4 + 4 B), write and read the (cos, sin) cache (8 + 8 B
    # in FP32, 4 + 4 B in 16 bits), plus the CSR structure once per graph and step.
    # Dense form: a tensor-core contraction of 2 * (2R) * n * n FLOPs per step.
    peaks = load_peaks()
    # the per-step forms run readout kernels between the step kernels; the step kernel's
    # own average launch duration comes from runs of the same steps without readouts
    # (CUDA events around each run, divided by its steps; L2 flushed between runs)
    ms_kernel_run = ms_step
    if info["form"] in (1, 3, 4, 5):
        bare = Run(prob, dK, dKs, dKn, w.dt, w.steps, w.replicas, seed_base + 50, form=form,
                   precision=precision, readout_every=0, stream=stream,
                   replicas_per_block=rpb, threads_per_block=threads, graph_forms=graph_forms)
        bare.sync()
        # one untimed re-run: the second execution of a shape captures the whole run as a
        # CUDA graph (host work that would otherwise fall between the events)
        bare.rerun(dK, dKs, dKn, w.dt, w.steps, seed_base + 59)
        bare.sync()
        kt = []
        for k in range(3):
            flush.fill_(float(k))
            b0, b1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            b0.record(stream)
            bare.rerun(dK, dKs, dKn, w.dt, w.steps, seed_base + 60 + k)
            b1.record(stream)
            torch.cuda.synchronize()
            kt.append(b0.elapsed_time(b1))
        bare.close()
        ms_kernel_run = float(np.mean(kt))
    prec_name = {1: "fp32", 2: "bf16", 3: "fp16"}.get(info["precision"])
    kname = {2: f"resident_quad_kernel<{prec_name}>",
             1: "step_stream_kernel" if info["precision"] == 1 else "step_octet_kernel",
             3: "gemm_step_kernel", 4: "step_octet_kernel + gemm_step_kernel",
             5: "step_octet_persistent_kernel"}.get(info["form"], "?")
    traffic = profiled_traffic(kname, w.name)
    if info["form"] == 3:
        n = w.graphs[0].n
        flops_per_step = 2.0 * (2 * w.replicas) * n * n
        alg_flops = flops_per_step * w.steps
        achieved = alg_flops / (ms_kernel_run / 1e3) / 1e12
        peak = peaks["bf16_tflops"]
        roofline = {"bound": "tensor", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                    "frac": achieved / peak, "traffic": traffic, "kernel": kname,
                    "peak_source": peaks["source"] + " bf16 burst",
                    "algorithmic_flops_per_launch": flops_per_step,
                    "flops_per_node_replica_step": 4.0 * n,
                    "kernel_time": "CUDA events around runs of the same steps without readouts "
                                   "(one step kernel per step plus an init kernel), divided by "
                                   "the steps",
                    "us_per_launch": ms_kernel_run * 1e3 / w.steps}
    else:
        node_replica_steps = w.nodes * w.replicas * w.steps
        dense = [gi for gi, f in enumerate(graph_forms or []) if f == capi.OIM_FORM_GEMM]
        # the CSR structure of the stream-form graphs, and for the dense members of a
        # mixed run their BF16 coupling matrix, once per step
        csr_bytes = sum(4 * g.nnz + 8 * (g.n + 1) for gi, g in enumerate(w.graphs) if gi not in dense) * w.steps
        csr_bytes += sum(2 * w.graphs[gi].n ** 2 for gi in dense) * w.steps
        bytes_per_unit = 24 if info["precision"] == 1 else 16
        alg_bytes = node_replica_steps * bytes_per_unit + csr_bytes
        achieved = alg_bytes / (ms_kernel_run / 1e3) / 1e9
        resident = info["form"] == 2
        roofline = {"bound": "hbm", "achieved": achieved, "peak": peaks["hbm_gbs"], "unit": "GB/s",
                    "frac": achieved / peaks["hbm_gbs"], "traffic": traffic, "kernel": kname,
                    "peak_source": peaks["source"],
                    "algorithmic_bytes_per_launch": alg_bytes if resident else alg_bytes / w.steps,
                    "bytes_per_node_replica_step": bytes_per_unit,
                    "kernel_time": ("CUDA events around each run (one launch of the resident "
                                    "kernel, its readouts included, plus a memset of the trace "
                                    "and schedule copies)"
                                    if resident else
                                    "CUDA events around runs of the same steps without readouts "
                                    "(one step kernel per step plus an init kernel), divided by "
                                    "the steps"),
                    "us_per_launch": ms_kernel_run * 1e3 / (1 if resident else w.steps)}

    # end to end through the C ABI with host buffers: upload graphs and schedules,
    # simulate, read spins and scores back, free everything
    from paper_2505_22631_gb300 import capi as C
    host_graphs = [(g.n, np.ascontiguousarray(g.row_ptr), np.ascontiguousarray(g.col),
                    np.ascontiguousarray(g.w)) for g in w.graphs]
    pin = {k: torch.from_numpy(a).pin_memory() for k, a in (("K", K), ("Ks", Ks), ("Kn", Kn))}
    spins_h = torch.empty(w.nodes * w.replicas, dtype=torch.int8).pin_memory()
    score_h = torch.empty(len(w.graphs) * w.replicas, dtype=torch.float64).pin_memory()
    best_h = torch.empty(len(w.graphs), dtype=torch.int32).pin_memory()
    h2d = sum(8 * (n + 1) + 4 * c.shape[0] + 4 * ww.shape[0] for n, _, c, ww in host_graphs) \
        + 3 * K.size * 4
    d2h = spins_h.numel() + score_h.numel() * 8 + best_h.numel() * 4

    forms_arr = None if graph_forms is None else np.ascontiguousarray(graph_forms, dtype=np.int32)

    def e2e_step(seed):
        # one graph: oim_create_problem; a batch: oim_create_batch_csr (the graphs checked
        # and laid out on host threads, then joined and uploaded, in one call)
        if len(host_graphs) > 1:
            hb = C.oim_create_batch_csr([n for n, _, _, _ in host_graphs], w.q,
                                        [c.shape[0] for _, _, c, _ in host_graphs],
                                        [rp for _, rp, _, _ in host_graphs], [c for _, _, c, _ in host_graphs],
                                        [ww for _, _, _, ww in host_graphs])
        else:
            n, rp, c, ww = host_graphs[0]
            hb = C.oim_create_problem(n, w.q, c.shape[0], rp, c, ww, 0)
        o = C.oim_default_opts()
        o.form = run.opts.form
        o.precision = run.opts.precision
        o.replicas_per_block = run.opts.replicas_per_block
        o.threads_per_block = run.opts.threads_per_block
        if forms_arr is not None:
            o.graph_forms = forms_arr.ctypes.data
        o.readout_every = args.readout_every
        o.stream = int(stream.cuda_stream)
        hr = C.oim_run(hb, pin["K"], pin["Ks"], pin["Kn"], w.dt, w.steps, w.replicas, seed, o)
        C.oim_readout(hr, spins_h, score_h, best_h, None, None)
        C.oim_destroy_run(hr)
        C.oim_destroy_problem(hb)

    e2e = None
    if args.e2e_steps > 0:
        e2e_step(7)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for k in range(args.e2e_steps):
            e2e_step(8 + k)
        torch.cuda.synchronize()
        e2e_s = (time.perf_counter() - t0) / args.e2e_steps
        e2e = {"value": w.edge_updates() * world / e2e_s, "unit": "edge-updates/s",
               "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": int(d2h),
               "ms_per_step": e2e_s * 1e3}

    line = {
        "metric": "edge-updates/s", "value": value, "unit": "edge-updates/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_step,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f32" if info["precision"] == 1 else "f32 (16-bit cos/sin cache)",
        "data": "synthetic",
        "config": {"workload": w.name, "graphs": [g.name for g in w.graphs],
                   "nodes": [g.n for g in w.graphs], "nnz": [g.nnz for g in w.graphs],
                   "replicas": w.replicas, "euler_steps": w.steps,
                   "readout_every": args.readout_every,
                   "form": {0: "auto", 1: "stream", 2: "resident", 3: "gemm", 4: "mixed",
                            5: "persistent"}[info["form"]],
                   "graph_forms": None if graph_forms is None else
                   [{1: "stream", 3: "gemm"}[f] for f in graph_forms],
                   "precision": {1: "fp32", 2: "bf16", 3: "fp16"}.get(info["precision"]),
                   "l2": "256 MB buffer written between timed steps (outside the events)",
                   "autotuned": tuned,
                   "parallelism": f"replicas x{world} (weak)"},
        "roofline": roofline,
        "clocks": clocks,
        "e2e": e2e,
        "node_updates_per_s": node_updates_per_s,
        "gpu_launches": args.steps * kernels_per_run(
            info["form"], w.steps, args.readout_every,
            sum(1 for f in (graph_forms or []) if f == capi.OIM_FORM_GEMM)),
        "wall_s_timed_region": wall,
        "step_ms_all": ms,
    }

    # the job's answer: best score per graph over every rank's replicas and the
    # winning spins (the only cross-rank data; taken after the timed region)
    from paper_2505_22631_gb300.distributed import best_across_ranks
    res = run.readout(spins=True, trace=False)
    best, winner, _ = best_across_ranks(res["score"], res["spins"], w.q)
    line["best_score"] = {"per_graph": best.tolist(), "winning_rank": winner.tolist(),
                          "kind": "cut" if w.q == 2 else "conflicts"}

    if rank == 0 and not args.no_quality:
        line["quality"] = quality(w, prob, problems, args, stream, ms_step,
                                  (form, precision, rpb, threads, graph_forms))
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_oracle_sample(w)
    if rank == 0:
        print(json.dumps(line), flush=True)
    run.close()
    if world > 1:
        torch.distributed.destroy_process_group()


def run_adjoint(args, rank, world):
    """Schedule-gradient pass: FP32 stream forward keeping the whole trajectory (or a
    checkpoint every C steps), then oim_backward (the reverse sweep, after recomputing each
    segment when only checkpoints were kept).  Reported as edge-updates
    of the forward trajectory per second of forward + backward."""
    import torch
    from paper_2505_22631_gb300 import Problem, build, capi  # noqa: F401
    name = args.workload if args.workload != "torus_er2000" else "er64"
    w = make_workload(name, steps=args.euler_steps or None, replicas=args.replicas or None)
    K, Ks, Kn = schedules(w)
    problems = [Problem.from_graph(g, w.q) for g in w.graphs]
    prob = Problem.batch(problems) if len(problems) > 1 else problems[0]
    stream = torch.cuda.current_stream()
    G, T = len(w.graphs), w.steps
    dK, dKs, dKn = (np.zeros((G, T)) for _ in range(3))
    loss = np.zeros(G)

    # checkpoint period: every step with its coupling sums (12 B per node-replica-step:
    # the library keeps the sums when they fit with a tenth of the device to spare), else
    # a checkpoint every 100 steps and a recomputation of each segment
    C = args.checkpoint_every
    if C <= 0:
        free_b, total_b = torch.cuda.mem_get_info()
        need = 12 * w.nodes * (w.replicas + 3) * T
        C = 1 if need + max(total_b // 10, 2 << 30) + (4 << 30) <= free_b else 100
    o = capi.oim_default_opts()
    o.form = capi.OIM_FORM_STREAM
    o.precision = capi.OIM_PREC_FP32
    o.checkpoint_every = C
    o.use_graph = 1
    o.stream = int(stream.cuda_stream)
    # the run is made once and re-run per seed (buffers kept, the whole run replayed from
    # a CUDA graph once its shape comes back)
    free0 = torch.cuda.mem_get_info()[0]
    run = capi.oim_run(prob.handle, K, Ks, Kn, w.dt, T, w.replicas, 11, o)
    # the library kept every step's coupling sums if the run holds them (8 B per
    # node-replica-step on top of the phases)
    whole = C == 1 and free0 - torch.cuda.mem_get_info()[0] >= 12 * w.nodes * w.replicas * T
    capi.oim_backward(run, dK, dKs, dKn, loss)

    def step(seed):
        e0, e1, e2 = (torch.cuda.Event(enable_timing=True) for _ in range(3))
        e0.record(stream)
        capi.oim_rerun(run, K, Ks, Kn, w.dt, T, seed)
        e1.record(stream)
        capi.oim_backward(run, dK, dKs, dKn, loss)   # synchronous
        e2.record(stream)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1), e1.elapsed_time(e2)

    for k in range(args.warmup):
        step(seed=12 + k)
    fw, bw = [], []
    for k in range(args.steps):
        a, b = step(seed=101 + k)
        fw.append(a)
        bw.append(b)
    capi.oim_destroy_run(run)
    ms = float(np.mean(fw) + np.mean(bw))
    ms = reduce_max(ms, world, device="cuda")
    edge_updates = w.edge_updates() * world
    # roofline of the backward pass: per node-replica-step the adjoint step reads theta_t,
    # theta_{t-1}, lambda_{t+1}, the coupling sums (8 B) and its lambda-weighted planes
    # (8 B), and writes lambda_t and the next planes (8 B): 40 B, plus the CSR once per
    # step.  With a recomputation the recomputed FP32 step adds 24 B (phase read and write,
    # (cos, sin) pair write and read), the stored sums 8 B and the CSR once more.
    peaks = load_peaks()
    nrs = w.nodes * w.replicas * T
    csr_bytes = sum(4 * g.nnz + 8 * (g.n + 1) for g in w.graphs) * T
    per_nrs = 40 if whole else 72
    bw_bytes = nrs * per_nrs + (1 if whole else 2) * csr_bytes
    bw_achieved = bw_bytes / (float(np.mean(bw)) / 1e3) / 1e9
    roofline = {"bound": "hbm", "achieved": bw_achieved, "peak": peaks["hbm_gbs"], "unit": "GB/s",
                "frac": bw_achieved / peaks["hbm_gbs"], "traffic": None,
                "kernel": "backward pass (adj_step_kernel" + (")" if whole else
                                                              " + step_stream_kernel recomputation)"),
                "peak_source": peaks["source"], "algorithmic_bytes_per_launch": bw_bytes / T,
                "bytes_per_node_replica_step": per_nrs,
                "kernel_time": "CUDA events around oim_backward, divided by the steps"}
    line = {"metric": "edge-updates/s (forward + schedule adjoint)", "value": edge_updates / (ms / 1e3),
            "unit": "edge-updates/s", "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": ms, "ms_forward": float(np.mean(fw)), "ms_backward": float(np.mean(bw)),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32 (f64 gradient sums)",
            "data": "synthetic",
            "config": {"workload": w.name, "graphs": len(w.graphs), "nodes": w.nodes, "replicas": w.replicas,
                       "euler_steps": T, "checkpoint_every": C,
                       "trajectory": "whole (phases and coupling sums of every step kept)" if whole
                       else "checkpoints, each segment recomputed",
                       "form": "stream", "precision": "fp32",
                       "timing": "CUDA events around the forward launch sequence and around oim_backward "
                                 "(which includes its scratch allocation and the gradient copies)"},
            "roofline": roofline, "backward_over_forward": float(np.mean(bw) / np.mean(fw)),
            "mean_loss": float(loss.mean()),
            "gradient_norms": {"dK": float(np.linalg.norm(dK)), "dKs": float(np.linalg.norm(dKs)),
                               "dKn": float(np.linalg.norm(dKn))}}
    if rank == 0:
        print(json.dumps(line), flush=True)


def _mean_ci(xs):
    """Mean and the half-width of its 95 % confidence interval (Student t)."""
    x = np.asarray([v for v in xs if v is not None], dtype=np.float64)
    if x.size == 0:
        return None, None
    if x.size == 1:
        return float(x[0]), None
    try:
        from scipy.stats import t as student_t
        q = float(student_t.ppf(0.975, x.size - 1))
    except Exception:
        q = 1.96
    return float(x.mean()), float(q * x.std(ddof=1) / np.sqrt(x.size))


def quality(w, prob, problems, args, stream, ms_step_chosen, chosen_cfg):
    """Time to 99 % of the best known cut, chosen form vs the plain FP32 CSR form, over
    several seeds, with one stopping rule for both: a graph stops at the first readout
    where its best score over the replicas reaches 99 % of the best known score.  The
    chosen form steps every graph of the batch together, so it stops when the last graph
    reaches its target; the plain form runs the graphs one after another, each stopping
    at its own hit.  Also the final best-score distributions of both forms (equal
    quality)."""
    import torch
    from paper_2505_22631_gb300 import Run
    re = args.readout_every
    q2 = w.q == 2
    G = len(w.graphs)
    seeds = [777 + 13 * k for k in range(args.quality_seeds)]
    # best known: best score of a 4x longer run of the chosen form
    form, precision, rpb, threads, graph_forms = chosen_cfg
    K4, Ks4, Kn4, T4 = stretched(w, 4)
    long = Run(prob, K4, Ks4, Kn4, w.dt, T4, w.replicas, 4242, form=form, precision=precision,
               readout_every=re * 4, stream=stream, replicas_per_block=rpb, threads_per_block=threads,
               graph_forms=graph_forms)
    tr = long.readout(spins=False)["trace"]
    long.close()
    best_known = tr.max(axis=(1, 2)) if q2 else tr.min(axis=(1, 2))
    target = [0.99 * b if q2 else b / 0.99 for b in best_known]
    K, Ks, Kn = schedules(w)
    per_step_chosen = ms_step_chosen / 1e3 / w.steps

    def hits_and_finals(out, rows):
        hs, fs = [], []
        for gi, row in rows:
            tr_g, sc_g = out["trace"][row], out["score"][row]
            tb = tr_g.max(axis=1) if q2 else -tr_g.min(axis=1)
            h = first_hit(tb, target[gi] if q2 else -target[gi])
            hs.append(None if h is None else (h + 1) * re)
            fs.append(float(sc_g.max() if q2 else sc_g.min()))
        return hs, fs

    # the plain form: one graph per launch sequence, one launch per step, FP32 CSR; its
    # time per step measured on a rerun of each graph
    plain_runs, per_step_plain = [], []
    for gi in range(G):
        pr = Run(problems[gi], K[gi], Ks[gi], Kn[gi], w.dt, w.steps, w.replicas, seeds[0],
                 form="stream", precision="fp32", readout_every=re, use_graph=False, stream=stream)
        pr.sync()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        pr.rerun(K[gi], Ks[gi], Kn[gi], w.dt, w.steps, seeds[0])
        e1.record(stream)
        torch.cuda.synchronize()
        per_step_plain.append(e0.elapsed_time(e1) / 1e3 / w.steps)
        plain_runs.append(pr)
    chosen_run = Run(prob, K, Ks, Kn, w.dt, w.steps, w.replicas, seeds[0], form=form,
                     precision=precision, readout_every=re, stream=stream, replicas_per_block=rpb,
                     threads_per_block=threads, graph_forms=graph_forms)
    per_seed = []
    for sd in seeds:
        chosen_run.rerun(K, Ks, Kn, w.dt, w.steps, sd)
        hc, fc = hits_and_finals(chosen_run.readout(spins=False), [(gi, gi) for gi in range(G)])
        hp, fp = [], []
        for gi in range(G):
            plain_runs[gi].rerun(K[gi], Ks[gi], Kn[gi], w.dt, w.steps, sd)
            h, f = hits_and_finals(plain_runs[gi].readout(spins=False), [(gi, 0)])
            hp += h
            fp += f
        t_c = None if any(h is None for h in hc) else max(hc) * per_step_chosen
        t_p = None if any(h is None for h in hp) else sum(h * p for h, p in zip(hp, per_step_plain))
        per_seed.append({"seed": sd, "steps_to_99pct": {"chosen": hc, "plain_fp32_csr": hp},
                         "time_to_99pct_s": {"chosen": t_c, "plain_fp32_csr": t_p},
                         "final_best": {"chosen": fc, "plain_fp32_csr": fp}})
    chosen_run.close()
    for pr in plain_runs:
        pr.close()

    tc = [r["time_to_99pct_s"]["chosen"] for r in per_seed]
    tp = [r["time_to_99pct_s"]["plain_fp32_csr"] for r in per_seed]
    ratio = [p / c for p, c in zip(tp, tc) if p is not None and c is not None]
    m_c, ci_c = _mean_ci(tc)
    m_p, ci_p = _mean_ci(tp)
    m_r, ci_r = _mean_ci(ratio)
    graphs = []
    for gi, g in enumerate(w.graphs):
        fc = [r["final_best"]["chosen"][gi] for r in per_seed]
        fp = [r["final_best"]["plain_fp32_csr"][gi] for r in per_seed]
        mc, cc = _mean_ci(fc)
        mp, cp = _mean_ci(fp)
        graphs.append({"graph": g.name, "best_known": float(best_known[gi]),
                       "final_best_mean": {"chosen": mc, "plain_fp32_csr": mp},
                       "final_best_ci95": {"chosen": cc, "plain_fp32_csr": cp},
                       "final_best_diff_pct": None if not mp else 100.0 * (mc - mp) / abs(mp),
                       "steps_to_99pct_mean": {
                           "chosen": _mean_ci([r["steps_to_99pct"]["chosen"][gi] for r in per_seed])[0],
                           "plain_fp32_csr": _mean_ci([r["steps_to_99pct"]["plain_fp32_csr"][gi]
                                                       for r in per_seed])[0]},
                       "s_per_euler_step": {"chosen (whole batch)": per_step_chosen,
                                            "plain_fp32_csr (this graph)": per_step_plain[gi]}})
    return {
        "rule": "each graph stops at the first readout (every %d steps) whose best score over the "
                "replicas reaches 99 %% of the best known; chosen: all graphs in one batch, time = "
                "(last graph's hit) x (batch step time); plain: graphs one after another, time = "
                "sum over graphs of (its hit) x (its step time)" % re,
        "best_known_from": "a 4x longer run of the chosen form (seed 4242)",
        "seeds": seeds,
        "time_to_99pct_best_cut_s": {"chosen": m_c, "plain_fp32_csr": m_p,
                                     "chosen_ci95": ci_c, "plain_fp32_csr_ci95": ci_p,
                                     "seeds_reaching": {"chosen": sum(v is not None for v in tc),
                                                        "plain_fp32_csr": sum(v is not None for v in tp),
                                                        "of": len(seeds)}},
        "plain_over_chosen": {"mean": m_r, "ci95": ci_r, "per_seed": ratio},
        "graphs": graphs,
        "per_seed": per_seed,
    }


if __name__ == "__main__":
    main()
