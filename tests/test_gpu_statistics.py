"""Statistical best-cut parity: the forms the benchmark ships against the FP64 oracle.

The dynamics are chaotic: after a few hundred steps a GPU trajectory and the oracle's,
started from the same phases and driven by the same Philox noise, are independent
samples of the same process.  Their solution quality is compared as such: over S seeds,
the mean of the best cut over the replicas must agree within 0.5 % of the oracle's
(the criterion of the benchmark's quality claim; a 95 % CI of the difference is
printed).  Both sides score their final spins exactly (the GPU's score is its own
readout; the oracle thresholds its FP64 phases).
"""
import numpy as np
import pytest

from gpu_common import require_gpu
from workloads import make_workload

pytestmark = pytest.mark.gpu

SEEDS = list(range(1, 11))


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    require_gpu()


def _sched(w, gi, T):
    return (w.K[gi][:T].astype(np.float32), w.Ks[gi][:T].astype(np.float32),
            w.Kn[gi][:T].astype(np.float32))


def _oracle_best(orc, w, gi, T, R, seed):
    g = w.graphs[gi]
    K, Ks, Kn = (x.astype(np.float64) for x in _sched(w, gi, T))
    th, _ = orc.run(g, w.q, K, Ks, Kn, float(np.float32(w.dt)), T, R, seed, graph=gi, nthreads=16)
    return orc.scores(g, w.q, orc.readout_f64(w.q, th)).max()


def _gpu_best(w, T, seed, form, precision, rpb=0, threads=0, keep=None):
    from paper_2505_22631_gb300 import Problem, Run
    probs = [Problem.from_graph(g, w.q) for g in w.graphs]
    prob = probs[0] if len(probs) == 1 else Problem.batch(probs)
    K = np.stack([_sched(w, gi, T)[0] for gi in range(len(w.graphs))])
    Ks = np.stack([_sched(w, gi, T)[1] for gi in range(len(w.graphs))])
    Kn = np.stack([_sched(w, gi, T)[2] for gi in range(len(w.graphs))])
    run = Run(prob, K, Ks, Kn, w.dt, T, w.replicas, seed, form=form, precision=precision,
              replicas_per_block=rpb, threads_per_block=threads)
    sc = run.readout(spins=False)["score"]
    info = run.info()
    run.close()
    keep = keep or w.replicas
    return sc[:, :keep].max(axis=1), info


def _compare(name, gpu, ref):
    gpu, ref = np.asarray(gpu, float), np.asarray(ref, float)
    diff = gpu.mean() - ref.mean()
    ci = 1.96 * np.sqrt(gpu.var(ddof=1) / len(gpu) + ref.var(ddof=1) / len(ref))
    print(f"{name}: best cut GPU {gpu.mean():.1f} oracle {ref.mean():.1f} diff {diff:+.1f} "
          f"({100 * diff / ref.mean():+.3f} %, 95% CI +-{ci:.1f})")
    assert abs(diff) <= 0.005 * ref.mean()


@pytest.fixture(scope="module")
def er800_oracle(orc):
    w = make_workload("er800")
    return w, [_oracle_best(orc, w, 0, w.steps, w.replicas, s) for s in SEEDS]


@pytest.mark.parametrize("form,precision", [("resident", "fp32"), ("stream", "fp32"),
                                            ("stream", "fp16"), ("resident", "fp16"),
                                            ("autotuned", None)])
def test_er800_best_cut_matches_oracle(er800_oracle, form, precision):
    """G(800, 0.06), 8 replicas, 1000 steps: every form, including the 16-bit stream form
    with its mixed-add gather (+1 rows of 48 entries) and the autotuner's choice."""
    from paper_2505_22631_gb300 import Problem, capi
    w, ref = er800_oracle
    rpb = threads = 0
    if form == "autotuned":
        prob = Problem.from_graph(w.graphs[0], 2)   # kept alive while the autotuner runs
        o, _ = capi.oim_autotune(prob.handle, w.replicas, capi.OIM_PREC_AUTO, 200)
        form, precision = o.form, o.precision
        rpb, threads = o.replicas_per_block, o.threads_per_block
    gpu = [_gpu_best(w, w.steps, s, form, precision, rpb, threads)[0][0] for s in SEEDS]
    _compare(f"er800 {form} {precision}", gpu, ref)


def test_batched_maxcut_autotuned_form_matches_oracle_on_a_replica_sample(orc):
    """The benchmark workload (50x40 +-1 torus and G(2000, 0.01), 1024 replicas each) in
    the form the autotuner picks for it (on the GB300: the 16-bit stream form, mixed-add
    gather, both graphs in one launch), over the first 1000 steps of its schedule; the
    oracle follows replicas 0..31 of each graph and the GPU's best over the same 32
    replicas is compared, graph by graph."""
    from paper_2505_22631_gb300 import Problem, capi
    w = make_workload("torus_er2000")
    T, R_s = 1000, 32
    prob = Problem.batch([Problem.from_graph(g, 2) for g in w.graphs])
    o, _ = capi.oim_autotune(prob.handle, w.replicas, capi.OIM_PREC_AUTO, 200)
    print(f"autotuned: form {o.form} precision {o.precision}")
    gpu = np.array([_gpu_best(w, T, s, o.form, o.precision, o.replicas_per_block,
                              o.threads_per_block, keep=R_s)[0] for s in SEEDS])
    for gi, g in enumerate(w.graphs):
        ref = [_oracle_best(orc, w, gi, T, R_s, s) for s in SEEDS]
        _compare(f"{g.name} (first {T} steps, replicas 0..{R_s - 1})", gpu[:, gi], ref)
