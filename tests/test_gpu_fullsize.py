"""Full-size checks of every workload, in the launch configuration the benchmark uses.

The oracle cannot follow thousands of replicas for thousands of steps, so these
compare what it can compute one by one: sampled replicas after a short horizon
(phases), the exact recount of every replica's score from the GPU's own spins,
and properties that hold at any size.  The statistical best-cut criterion is in
test_gpu_statistics.py.
"""
import numpy as np
import pytest

from gpu_common import circ, coupling_bound_rad, oracle_phases, rad_dist, require_gpu
from workloads import make_workload

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    require_gpu()


def run_workload(w, steps=None, form="auto", precision="auto", readout_every=0, seed=1):
    from paper_2505_22631_gb300 import Problem, Run
    probs = [Problem.from_graph(g, w.q) for g in w.graphs]
    prob = probs[0] if len(probs) == 1 else Problem.batch(probs)
    T = steps or w.steps
    K = np.stack(w.K)[:, :T].copy()
    Ks = np.stack(w.Ks)[:, :T].copy()
    Kn = np.stack(w.Kn)[:, :T].copy()
    return Run(prob, K, Ks, Kn, w.dt, T, w.replicas, seed, form=form, precision=precision,
               readout_every=readout_every)


def test_batched_maxcut_sampled_replicas_fp32(orc):
    # horizon: at these couplings (K = 4 per torus edge) the FP64 dynamics alone amplify an
    # FP32-ulp perturbation of the start to 6.9e-5 rad in 10 steps, 1.8e-4 in 20, 3.3e-2 in 50
    w = make_workload("torus_er2000")
    T = 15
    run = run_workload(w, steps=T, form="resident", precision="fp32", seed=3)
    ph = run.phases()
    for gi, g in enumerate(w.graphs):
        for r0 in (0, 517, 1020):
            ref = oracle_phases(orc, g, 2, w.K[gi], w.Ks[gi], w.Kn[gi], w.dt, T, 4, 3, graph=gi,
                                replica_offset=r0, nthreads=8)
            assert rad_dist(ph[gi][r0:r0 + 4], ref).max() <= 1e-3


def test_batched_maxcut_full_run_scores_exact(orc):
    # the benchmark's form (AUTO: resident, FP16 cache), full 5000 steps, every replica
    w = make_workload("torus_er2000")
    run = run_workload(w, readout_every=50, seed=5)
    out = run.readout()
    ph = run.phases()
    for gi, g in enumerate(w.graphs):
        spins = orc.readout_f32(2, ph[gi])
        assert np.array_equal(out["spins"][gi], spins)
        assert np.array_equal(out["score"][gi], orc.scores(g, 2, spins))
        assert np.array_equal(out["trace"][gi, -1], out["score"][gi])
        # the annealed machine ends far above random assignments
        rnd = orc.scores(g, 2, np.random.default_rng(gi).integers(0, 2, (64, g.n)).astype(np.int8))
        assert out["score"][gi].mean() > rnd.max() + 0.1 * g.num_edges


def test_batched_maxcut_in_the_autotuned_stream_form(orc):
    # the form the autotuner picks for the benchmark workload on the GB300 (16-bit stream
    # form, mixed-add gather, CUDA-graph replay on the repeat): sampled replicas against
    # the oracle over a short horizon, every phase within the linear accumulation of the
    # 1e-2 coupling bound (torus: 0.10 rad over 10 steps at K = 4; measured max 2.3e-2)
    # and the bulk within 1e-3 rad; then the full 5000-step run replayed from its graph,
    # every replica's score recounted from its own spins
    w = make_workload("torus_er2000")
    T = 10
    run = run_workload(w, steps=T, form="stream", precision="fp16", seed=3)
    ph = run.phases()
    for gi, g in enumerate(w.graphs):
        d = np.concatenate([
            rad_dist(ph[gi][r0:r0 + 16], oracle_phases(orc, g, 2, w.K[gi], w.Ks[gi], w.Kn[gi], w.dt, T,
                                                       16, 3, graph=gi, replica_offset=r0,
                                                       nthreads=8)).ravel()
            for r0 in (0, 512, 1008)])
        assert d.max() <= coupling_bound_rad(g, w.K[gi], T, w.dt)
        assert np.median(d) <= 1e-3
    run = run_workload(w, form="stream", precision="fp16", readout_every=50, seed=5)
    K, Ks, Kn = (np.stack(x).astype(np.float32) for x in (w.K, w.Ks, w.Kn))
    run.rerun(K, Ks, Kn, w.dt, w.steps, 6)          # the same shape again: graph replay
    out = run.readout()
    ph = run.phases()
    for gi, g in enumerate(w.graphs):
        spins = orc.readout_f32(2, ph[gi])
        assert np.array_equal(out["spins"][gi], spins)
        assert np.array_equal(out["score"][gi], orc.scores(g, 2, spins))
        assert np.array_equal(out["trace"][gi, -1], out["score"][gi])
        rnd = orc.scores(g, 2, np.random.default_rng(gi).integers(0, 2, (64, g.n)).astype(np.int8))
        assert out["score"][gi].mean() > rnd.max() + 0.1 * g.num_edges


def test_dense_workload_in_the_tensor_core_form(orc):
    # the dense benchmark workload at full size in the form the autotuner picks for it
    # (BF16 tensor cores): sampled replicas against the oracle over a short horizon (the
    # BF16 coupling is within 1e-2 of the row norm: every phase within the linear
    # accumulation of that bound, the bulk within 1e-3 rad), then the full
    # 1000-step run with every replica's score recounted from its own spins
    w = make_workload("dense2000")
    g = w.graphs[0]
    T = 10
    run = run_workload(w, steps=T, form="gemm", precision="bf16", seed=4)
    assert run.info()["form"] == 3
    ph = run.phases()[0]
    for r0 in (0, 640, 1020):
        ref = oracle_phases(orc, g, 2, w.K[0], w.Ks[0], w.Kn[0], w.dt, T, 4, 4, replica_offset=r0,
                            nthreads=8)
        d = rad_dist(ph[r0:r0 + 4], ref)
        assert d.max() <= coupling_bound_rad(g, w.K[0], T, w.dt)   # measured max 2.3e-3
        assert np.median(d) <= 1e-3
    run = run_workload(w, form="gemm", precision="bf16", readout_every=50, seed=6)
    out = run.readout()
    spins = orc.readout_f32(2, run.phases()[0])
    assert np.array_equal(out["spins"][0], spins)
    assert np.array_equal(out["score"][0], orc.scores(g, 2, spins))
    assert np.array_equal(out["trace"][0, -1], out["score"][0])
    rnd = orc.scores(g, 2, np.random.default_rng(9).integers(0, 2, (64, g.n)).astype(np.int8))
    assert out["score"][0].mean() > rnd.max() + 0.01 * g.num_edges


@pytest.mark.parametrize("precision", ["fp32", "fp16"])
def test_planted_colouring_conflicts_exact(orc, precision):
    w = make_workload("planted600")
    run = run_workload(w, form="resident", precision=precision, readout_every=500, seed=7)
    out = run.readout()
    th = run.phases()[0]
    spins = orc.readout_f32(3, th)
    assert np.array_equal(out["spins"][0], spins)
    conf = orc.scores(w.graphs[0], 3, spins)
    assert np.array_equal(out["score"][0], conf)
    assert conf.min() <= 0.05 * w.graphs[0].num_edges   # near-proper colourings are found


def test_uneven_batch_runs_and_scores_exact(orc):
    w = make_workload("uneven16", steps=400)
    run = run_workload(w, readout_every=100, seed=9)
    out = run.readout()
    ph = run.phases()
    for gi in (0, 7, 8, 15):
        g = w.graphs[gi]
        spins = orc.readout_f32(2, ph[gi][:16])
        assert np.array_equal(out["spins"][gi][:16], spins)
        assert np.array_equal(out["score"][gi][:16], orc.scores(g, 2, spins))


def test_schedule_batch_adjoint_consistent_with_forward_energy():
    from paper_2505_22631_gb300 import Problem, capi
    w = make_workload("er64", steps=300)
    probs = [Problem.from_graph(g, 2) for g in w.graphs]
    prob = Problem.batch(probs)
    T = w.steps
    K, Ks, Kn = (np.stack(x).astype(np.float32) for x in (w.K, w.Ks, w.Kn))
    o = capi.oim_default_opts()
    o.form = capi.OIM_FORM_STREAM
    o.precision = capi.OIM_PREC_FP32
    o.checkpoint_every = 100
    r = capi.oim_run(prob.handle, K, Ks, Kn, w.dt, T, w.replicas, 11, o)
    G = len(w.graphs)
    E = np.zeros(G * w.replicas)
    capi.oim_readout(r, None, None, None, None, E)
    dK, dKs, dKn, L = np.zeros((G, T)), np.zeros((G, T)), np.zeros((G, T)), np.zeros(G)
    capi.oim_backward(r, dK, dKs, dKn, L)
    capi.oim_destroy_run(r)
    # the adjoint's loss is the mean final energy the readout reports
    assert np.allclose(L, E.reshape(G, w.replicas).mean(1), rtol=1e-5, atol=1e-3)
    assert np.all(np.isfinite(dK)) and np.all(np.isfinite(dKs)) and np.all(np.isfinite(dKn))


def test_adjoint_at_schedule_workload_sizes_matches_oracle(orc):
    # the smallest and the largest graph of the 64-graph schedule-learning workload (n = 800
    # and 3000), its 32 replicas and production schedules, over 50 steps (the horizon over
    # which FP32 and FP64 trajectories agree at this coupling), checkpoints every 20 steps
    from paper_2505_22631_gb300 import Problem, capi
    w = make_workload("er64", steps=50)
    pick = [0, len(w.graphs) - 1]
    graphs = [w.graphs[k] for k in pick]
    prob = Problem.batch([Problem.from_graph(g, 2) for g in graphs])
    T, R = w.steps, w.replicas
    K, Ks, Kn = (np.stack([np.asarray(x[k], np.float32) for k in pick]) for x in (w.K, w.Ks, w.Kn))
    o = capi.oim_default_opts()
    o.form = capi.OIM_FORM_STREAM
    o.precision = capi.OIM_PREC_FP32
    o.checkpoint_every = 20
    r = capi.oim_run(prob.handle, K, Ks, Kn, w.dt, T, R, 21, o)
    dK, dKs, dKn, L = np.zeros((2, T)), np.zeros((2, T)), np.zeros((2, T)), np.zeros(2)
    capi.oim_backward(r, dK, dKs, dKn, L)
    capi.oim_destroy_run(r)
    for gi, g in enumerate(graphs):
        rL, rK, rKs, rKn = orc.adjoint(g, 2, K[gi].astype(np.float64), Ks[gi].astype(np.float64),
                                       Kn[gi].astype(np.float64), float(np.float32(w.dt)), T, R, 21,
                                       graph=gi, nthreads=8)
        assert abs(L[gi] - rL) <= 1e-5 * np.abs(g.w).sum()
        for got, ref in ((dK[gi], rK), (dKs[gi], rKs), (dKn[gi], rKn)):
            assert np.max(np.abs(got - ref)) <= 2e-3 * np.max(np.abs(ref)) + 1e-6


def test_uneven_batch_in_the_persistent_form(orc):
    # the form the autotuner picks for the 16-graph uneven batch on the GB300: the 16-bit
    # stream steps between readouts in one cooperative launch; a full-size 400-step run with
    # readouts, bit for bit the per-step 16-bit stream form, and every sampled replica's
    # score recounted from its own spins
    w = make_workload("uneven16", steps=400)
    a = run_workload(w, form="persistent", precision="fp16", readout_every=100, seed=9)
    b = run_workload(w, form="stream", precision="fp16", readout_every=100, seed=9)
    assert a.info()["form"] == 5
    pa, pb = a.phases(), b.phases()
    oa = a.readout()
    assert np.array_equal(oa["trace"], b.readout()["trace"])
    for gi in (0, 7, 8, 15):
        assert np.array_equal(pa[gi], pb[gi])
        g = w.graphs[gi]
        spins = orc.readout_f32(2, pa[gi][:16])
        assert np.array_equal(oa["spins"][gi][:16], spins)
        assert np.array_equal(oa["score"][gi][:16], orc.scores(g, 2, spins))


def test_uneven_batch_with_a_complete_graph_in_the_mixed_form(orc):
    # 16 uneven graphs and a complete +-1 graph on 2000 nodes, 256 replicas: the mixed form
    # (the complete graph on the tensor cores, the rest in the 16-bit stream form, on two
    # streams between readouts).  Over a short horizon the complete graph's sampled
    # replicas lie within the linear accumulation of the BF16 coupling bound of the oracle
    # and a CSR member matches the stream form of the whole batch bit for bit; then a
    # 300-step run with readouts, every sampled score recounted from its own spins
    w = make_workload("uneven16_k2000", steps=300)
    G = len(w.graphs)
    forms = ["stream"] * (G - 1) + ["gemm"]
    T = 10
    from paper_2505_22631_gb300 import Problem, Run
    probs = [Problem.from_graph(g, 2) for g in w.graphs]
    prob = Problem.batch(probs)
    K, Ks, Kn = (np.stack(x)[:, :T].copy() for x in (w.K, w.Ks, w.Kn))
    short = Run(prob, K, Ks, Kn, w.dt, T, w.replicas, 3, form="mixed", precision="fp16", graph_forms=forms)
    plain = Run(prob, K, Ks, Kn, w.dt, T, w.replicas, 3, form="stream", precision="fp16")
    ps, pp = short.phases(), plain.phases()
    assert np.array_equal(ps[8], pp[8])
    g = w.graphs[-1]
    d = np.concatenate([rad_dist(ps[-1][r0:r0 + 4], oracle_phases(orc, g, 2, w.K[-1], w.Ks[-1], w.Kn[-1], w.dt,
                                                                  T, 4, 3, graph=G - 1, replica_offset=r0,
                                                                  nthreads=16)).ravel()
                        for r0 in (0, 128, 252)])
    assert d.max() <= coupling_bound_rad(g, w.K[-1], T, w.dt)
    assert np.median(d) <= 1e-3
    full = Run(prob, *(np.stack(x).copy() for x in (w.K, w.Ks, w.Kn)), w.dt, w.steps, w.replicas, 5,
               form="mixed", precision="fp16", readout_every=100, graph_forms=forms)
    out = full.readout()
    ph = full.phases()
    for gi in (0, 15, G - 1):
        spins = orc.readout_f32(2, ph[gi][:8])
        assert np.array_equal(out["spins"][gi][:8], spins)
        assert np.array_equal(out["score"][gi][:8], orc.scores(w.graphs[gi], 2, spins))
        assert np.array_equal(out["trace"][gi, -1], out["score"][gi])
