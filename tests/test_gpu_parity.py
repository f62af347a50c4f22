"""Parity of the CUDA path (through the C ABI) with the FP64 oracle.

Tolerances:
  - initial phases: bit-exact (both sides produce odd multiples of 2^-24);
  - noise draws: |xi32 - xi64| <= 4e-6 (FP32 Box-Muller plus phase quantisation);
  - drift: |f32 - f64| <= 1e-5 (K sum_j |w_ij| + Ks + |f64|);
  - phases: within 1e-3 rad after 100 steps (K = 1/mean degree, where the FP64
    dynamics amplify an FP32-ulp perturbation of the start to ~4e-6 rad) and after
    50 steps at the production coupling K = 16/mean degree (measured ~9e-5 rad);
  - spins and cut / conflict scores from the same phases: bit-exact;
  - 16-bit (cos, sin) cache: coupling within 1e-2 of the row norm of the FP64 (A, B);
    its phases within the linear accumulation of that bound over a short horizon.
"""
import numpy as np
import pytest

from gpu_common import circ, coupling_bound_rad, gpu_run, oracle_phases, rad_dist, require_gpu
from workloads import (constant, csr_from_edges, erdos_renyi, linear_ramp, make_workload,
                       planted_partition, torus)

pytestmark = pytest.mark.gpu

FORMS = ["stream", "resident"]


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    require_gpu()


@pytest.fixture(scope="module")
def c1():
    return make_workload("er800")


@pytest.mark.parametrize("form", FORMS)
@pytest.mark.parametrize("R", [8, 6])
def test_initial_phases_bitexact(orc, c1, form, R):
    g = c1.graphs[0]
    run = gpu_run(g, 2, 0.0, 0.0, 0.0, 0.01, 0, R, seed=77, form=form)
    th = run.phases()[0]
    ref = orc.init_phases(g.n, R, 77).astype(np.float32)
    assert np.array_equal(th, ref)


@pytest.mark.parametrize("form", FORMS)
def test_noise_draws_match_oracle(orc, form):
    n, R, kick = 1000, 12, 0.05
    g = csr_from_edges(n, np.zeros(0, int), np.zeros(0, int))
    run = gpu_run(g, 2, 0.0, 0.0, kick, 1.0, 1, R, seed=5, form=form)
    th1 = run.phases()[0].astype(np.float64)
    th0 = orc.init_phases(n, R, 5)
    xi = circ(th1 - th0) / kick
    ref = orc.noise_block(n, R, 5, 0)
    assert np.max(np.abs(xi - ref)) <= 4e-6


@pytest.mark.parametrize("precision", ["fp16", "bf16"])
def test_fast_noise_draws_of_16bit_forms(orc, precision):
    # the 16-bit forms draw Box-Muller with the hardware log2 / sqrt / sin / cos
    n, R, kick = 2000, 64, 0.05
    g = csr_from_edges(n, np.zeros(0, int), np.zeros(0, int))
    run = gpu_run(g, 2, 0.0, 0.0, kick, 1.0, 1, R, seed=6, form="resident", precision=precision)
    th1 = run.phases()[0].astype(np.float64)
    th0 = orc.init_phases(n, R, 6)
    err = np.abs(circ(th1 - th0) / kick - orc.noise_block(n, R, 6, 0))
    print(f"fast Box-Muller |dxi|: max {err.max():.3e}  p99.99 {np.quantile(err, 0.9999):.3e}  "
          f"median {np.median(err):.3e}")
    assert np.quantile(err, 0.9999) <= 5e-6
    assert err.max() <= 2e-5


@pytest.mark.parametrize("precision", ["fp16", "bf16"])
def test_stream_16bit_cache_start_noise_readout(orc, c1, precision):
    # the 16-bit stream form: FP32 phases, the stored neighbour (cos, sin) pairs rounded
    # to 16 bits, hardware Box-Muller (the 16-bit forms' noise bound)
    g = c1.graphs[0]
    R = 8
    run = gpu_run(g, 2, 0.0, 0.0, 0.0, 0.01, 0, R, seed=77, form="stream", precision=precision)
    assert np.array_equal(run.phases()[0], orc.init_phases(g.n, R, 77).astype(np.float32))
    n, kick = 1000, 0.05
    e = csr_from_edges(n, np.zeros(0, int), np.zeros(0, int))
    run = gpu_run(e, 2, 0.0, 0.0, kick, 1.0, 1, 12, seed=5, form="stream", precision=precision)
    xi = circ(run.phases()[0].astype(np.float64) - orc.init_phases(n, 12, 5)) / kick
    assert np.max(np.abs(xi - orc.noise_block(n, 12, 5, 0))) <= 2e-5
    T = 100
    run = gpu_run(g, 2, c1.K[0][:T], c1.Ks[0][:T], c1.Kn[0][:T], c1.dt, T, R, 5, form="stream",
                  precision=precision, readout_every=25)
    th = run.phases()[0]
    out = run.readout()
    spins = orc.readout_f32(2, th)
    assert np.array_equal(out["spins"][0], spins)
    assert np.array_equal(out["score"][0], orc.scores(g, 2, spins))
    assert np.array_equal(out["trace"][0, -1], out["score"][0])
    # every phase within the linear accumulation of the 1e-2 coupling bound over 20 steps
    # (measured max: FP16 1.9e-3, BF16 1.8e-2 rad, against a bound of 0.25 rad), the bulk
    # within 1e-3 rad
    ref = oracle_phases(orc, g, 2, c1.K[0][:20], c1.Ks[0][:20], c1.Kn[0][:20], c1.dt, 20, R, 5)
    th20 = gpu_run(g, 2, c1.K[0][:20], c1.Ks[0][:20], c1.Kn[0][:20], c1.dt, 20, R, 5, form="stream",
                   precision=precision).phases()[0]
    d = rad_dist(th20, ref)
    assert d.max() <= coupling_bound_rad(g, c1.K[0], 20, c1.dt)
    assert np.median(d) <= 1e-3


def test_drift_matches_fp64(orc, c1):
    from paper_2505_22631_gb300 import Problem, oim_debug_derivative
    g = c1.graphs[0]
    prob = Problem.from_graph(g, 2)
    rng = np.random.default_rng(3)
    R = 3
    th = rng.random((R, g.n)).astype(np.float32)
    K, Ks = 0.33, 1.3
    f = np.zeros((R, g.n), np.float32)
    oim_debug_derivative(prob.handle, th, R, K, Ks, f)
    absw = np.bincount(np.repeat(np.arange(g.n), g.degrees()), weights=np.abs(g.w), minlength=g.n)
    for r in range(R):
        ref = orc.derivative(g, 2, th[r].astype(np.float64), np.float32(K), np.float32(Ks))
        scale = np.float32(K) * absw + np.float32(Ks) + np.abs(ref)
        assert np.max(np.abs(f[r] - ref) / scale) <= 1e-5


@pytest.mark.parametrize("form", FORMS)
def test_phases_after_100_steps(orc, c1, form):
    g = c1.graphs[0]
    T, R, seed = 100, 8, 11
    K = constant(T, 1.0 / g.mean_degree)
    Ks, Kn = c1.Ks[0][:T], c1.Kn[0][:T]
    run = gpu_run(g, 2, K, Ks, Kn, c1.dt, T, R, seed, form=form)
    ref = oracle_phases(orc, g, 2, K, Ks, Kn, c1.dt, T, R, seed, nthreads=8)
    assert rad_dist(run.phases()[0], ref).max() <= 1e-3


@pytest.mark.parametrize("form", FORMS)
def test_phases_production_coupling(orc, c1, form):
    g = c1.graphs[0]
    T, R, seed = 50, 8, 12
    run = gpu_run(g, 2, c1.K[0][:T], c1.Ks[0][:T], c1.Kn[0][:T], c1.dt, T, R, seed, form=form)
    ref = oracle_phases(orc, g, 2, c1.K[0][:T], c1.Ks[0][:T], c1.Kn[0][:T], c1.dt, T, R, seed,
                        nthreads=8)
    assert rad_dist(run.phases()[0], ref).max() <= 1e-3


@pytest.mark.parametrize("form", FORMS)
@pytest.mark.parametrize("wl", ["er800", "planted600"])
def test_readout_and_scores_bitexact(orc, form, wl):
    w = make_workload(wl)
    g = w.graphs[0]
    T, R = (1000, 8) if wl == "er800" else (600, 12)
    run = gpu_run(g, w.q, w.K[0][:T], w.Ks[0][:T], w.Kn[0][:T], w.dt, T, R, seed=21, form=form,
                  readout_every=100)
    out = run.readout(energy=True)
    th = run.phases()[0]
    spins = orc.readout_f32(w.q, th)
    assert np.array_equal(out["spins"][0], spins)
    sc = orc.scores(g, w.q, spins)
    assert np.array_equal(out["score"][0], sc)
    assert np.array_equal(out["trace"][0, -1], sc)          # last readout is the final state
    best = int(np.argmax(sc)) if w.q == 2 else int(np.argmin(sc))
    assert out["best_replica"][0] == best
    E = orc.energy(g, th.astype(np.float64))
    assert np.max(np.abs(out["energy"][0] - E)) <= 1e-5 * np.abs(g.w).sum()


def test_forms_agree(c1):
    g = c1.graphs[0]
    T, R = 100, 8
    K = constant(T, 1.0 / g.mean_degree)
    a = gpu_run(g, 2, K, c1.Ks[0][:T], c1.Kn[0][:T], c1.dt, T, R, 4, form="stream").phases()[0]
    b = gpu_run(g, 2, K, c1.Ks[0][:T], c1.Kn[0][:T], c1.dt, T, R, 4, form="resident").phases()[0]
    assert rad_dist(a, b).max() <= 1e-4


@pytest.mark.parametrize("precision", ["fp32", "fp16"])
def test_resident_block_shape_does_not_change_results(c1, precision):
    g = c1.graphs[0]
    T, R = 200, 24
    args = (g, 2, c1.K[0][:T], c1.Ks[0][:T], c1.Kn[0][:T], c1.dt, T, R, 9)
    kw = dict(form="resident", precision=precision, readout_every=50)
    a = gpu_run(*args, replicas_per_block=4, **kw)
    b = gpu_run(*args, replicas_per_block=16, threads_per_block=256, **kw)
    c = gpu_run(*args, replicas_per_block=12, **kw)
    assert np.array_equal(a.phases()[0], b.phases()[0])
    assert np.array_equal(a.phases()[0], c.phases()[0])
    assert np.array_equal(a.readout()["trace"], c.readout()["trace"])


def test_resident_pair_kernel_for_mid_size_graph(orc):
    g = torus(100, 100, 6, "pm1")   # 10000 nodes: two FP32 replicas per block, not four
    T, R = 20, 6
    K, Ks, Kn = constant(T, 4.0), linear_ramp(T, 0, 1), constant(T, 0.1)
    run = gpu_run(g, 2, K, Ks, Kn, 0.01, T, R, 2, form="resident", readout_every=10)
    ref = oracle_phases(orc, g, 2, K, Ks, Kn, 0.01, T, R, 2, nthreads=8)
    th = run.phases()[0]
    assert rad_dist(th, ref).max() <= 1e-3
    out = run.readout()
    assert np.array_equal(out["score"][0], orc.scores(g, 2, orc.readout_f32(2, th)))
    assert np.array_equal(out["trace"][0, -1], out["score"][0])


def test_stream_graph_capture_matches_direct_launches(c1):
    g = c1.graphs[0]
    T, R = 120, 8
    args = (g, 2, c1.K[0][:T], c1.Ks[0][:T], c1.Kn[0][:T], c1.dt, T, R, 9)
    a = gpu_run(*args, form="stream", use_graph=True, readout_every=40)
    b = gpu_run(*args, form="stream", use_graph=False, readout_every=40)
    # a run's first execution is launched directly; the same shape again is captured
    # into a CUDA graph and replayed
    a.rerun(c1.K[0][:T], c1.Ks[0][:T], c1.Kn[0][:T], c1.dt, T, 9)
    assert np.array_equal(a.phases()[0], b.phases()[0])
    assert np.array_equal(a.readout()["trace"], b.readout()["trace"])


@pytest.mark.parametrize("precision", ["fp32", "fp16"])
def test_stream_chunked_first_execution_matches_direct_launches(orc, precision):
    """A run's first execution replays a captured chunk of steps (step base and readout
    slot read from device memory) and launches the remaining steps directly: phases,
    trace and scores equal those of plain direct launches bit for bit, also after a
    rerun that grows the run (its buffers, and with them the chunk, are made again)."""
    g0 = erdos_renyi(400, 0.04, 5, "pm1")
    g1 = torus(12, 10, 6, "pm1")
    K = [constant(400, 4.0 / g.mean_degree) for g in (g0, g1)]
    Ks, Kn = linear_ramp(400, 0, 1), constant(400, 0.1)
    R = 64
    # readout every 25 steps: chunks of 50; 130 steps = 2 chunks and a 30-step tail
    # holding one readout, 260 steps = 5 chunks and a 10-step tail
    a = gpu_run([g0, g1], 2, [k[:130] for k in K], Ks[:130], Kn[:130], 0.01, 130, R, 3,
                form="stream", precision=precision, readout_every=25, use_graph=True)
    b = gpu_run([g0, g1], 2, [k[:130] for k in K], Ks[:130], Kn[:130], 0.01, 130, R, 3,
                form="stream", precision=precision, readout_every=25, use_graph=False)

    def same(x, y):
        px, py = x.phases(), y.phases()
        for gi in range(2):
            assert np.array_equal(px[gi], py[gi])
        ox, oy = x.readout(), y.readout()
        assert np.array_equal(ox["trace"], oy["trace"])
        assert np.array_equal(ox["score"], oy["score"])
        return ox

    out = same(a, b)
    assert out["trace"].shape[1] == 130 // 25
    for gi, g in enumerate((g0, g1)):
        th = a.phases()[gi]
        assert np.array_equal(out["score"][gi], orc.scores(g, 2, orc.readout_f32(2, th)))
    for steps, seed in ((260, 4), (260, 5)):   # the second pass replays the captured run
        a.rerun([k[:steps] for k in K], Ks[:steps], Kn[:steps], 0.01, steps, seed)
        b.rerun([k[:steps] for k in K], Ks[:steps], Kn[:steps], 0.01, steps, seed)
        same(a, b)


@pytest.mark.parametrize("form", FORMS)
def test_batch_uses_graph_index_streams(orc, form):
    g0 = erdos_renyi(300, 0.05, 1, "+1")
    g1 = torus(10, 12, 2, "pm1")
    T, R = 60, 6
    K = [constant(T, 4.0 / g.mean_degree) for g in (g0, g1)]
    Ks, Kn = linear_ramp(T, 0, 1), constant(T, 0.1)
    run = gpu_run([g0, g1], 2, K, Ks, Kn, 0.01, T, R, 31, form=form, readout_every=20)
    ph = run.phases()
    out = run.readout()
    for gi, g in enumerate((g0, g1)):
        ref = oracle_phases(orc, g, 2, K[gi], Ks, Kn, 0.01, T, R, 31, graph=gi)
        assert rad_dist(ph[gi], ref).max() <= 1e-3
        assert np.array_equal(out["score"][gi], orc.scores(g, 2, orc.readout_f32(2, ph[gi])))
    # graph 0 of the batch is the same trajectory as graph 0 run on its own
    alone = gpu_run(g0, 2, K[0], Ks, Kn, 0.01, T, R, 31, form=form).phases()[0]
    assert np.array_equal(alone, ph[0])


@pytest.mark.parametrize("form", FORMS)
@pytest.mark.parametrize("kind", ["float", "integer"])
def test_ragged_sizes_and_general_weights(orc, form, kind):
    rng = np.random.default_rng(5)
    g = erdos_renyi(37, 0.2, 8, "+1")
    i, j, _ = g.edges()
    w = rng.uniform(-2, 2, i.shape[0]) if kind == "float" else rng.choice([-2, -1, 1, 3], i.shape[0])
    g = csr_from_edges(37, i, j, w.astype(np.float32))
    T, R = 60, 5
    K, Ks, Kn = constant(T, 0.1), linear_ramp(T, 0, 1.5), constant(T, 0.1)
    run = gpu_run(g, 2, K, Ks, Kn, 0.01, T, R, 3, form=form)
    th = run.phases()[0]
    assert rad_dist(th, oracle_phases(orc, g, 2, K, Ks, Kn, 0.01, T, R, 3)).max() <= 1e-3
    sc = run.readout()["score"][0]
    ref = orc.scores(g, 2, orc.readout_f32(2, th))
    if kind == "integer":
        assert np.array_equal(sc, ref)
    else:
        assert np.allclose(sc, ref, rtol=1e-6, atol=1e-5)


@pytest.mark.parametrize("form", FORMS)
@pytest.mark.parametrize("q", [3, 5])
def test_potts_orders(orc, form, q):
    g = planted_partition(90, 3, 4.0, 6)
    T, R = 50, 4
    K, Ks, Kn = constant(T, 8.0 / g.mean_degree), linear_ramp(T, 0, 2), constant(T, 0.1)
    run = gpu_run(g, q, K, Ks, Kn, 0.01, T, R, 8, form=form)
    th = run.phases()[0]
    assert rad_dist(th, oracle_phases(orc, g, q, K, Ks, Kn, 0.01, T, R, 8)).max() <= 1e-3
    assert np.array_equal(run.readout()["score"][0], orc.scores(g, q, orc.readout_f32(q, th)))


@pytest.mark.parametrize("form", FORMS)
@pytest.mark.parametrize("precision", ["fp16", "bf16"])
@pytest.mark.parametrize("weights", ["+1", "pm1", "pm1_sparse"])
def test_half_cache_coupling_within_1e2_per_row(orc, c1, form, precision, weights):
    # +1 and +-1 weights, dense rows (the stream form's mixed-add gather, with its
    # negated -1 runs) and sparse rows (its convert-and-multiply gather)
    g = {"+1": c1.graphs[0], "pm1": erdos_renyi(600, 0.03, 19, "pm1"),
         "pm1_sparse": erdos_renyi(600, 0.008, 19, "pm1")}[weights]
    R, dt, K = 16, 1e-3, 1.0
    run = gpu_run(g, 2, K, 0.0, 0.0, dt, 1, R, 13, form=form, precision=precision)
    assert run.info()["precision"] == {"fp16": 3, "bf16": 2}[precision]
    th0 = orc.init_phases(g.n, R, 13)
    D = circ(run.phases()[0].astype(np.float64) - th0) / (np.float32(dt) * K)
    A = np.zeros((R, g.n))
    B = np.zeros((R, g.n))
    rows = np.repeat(np.arange(g.n), g.degrees())
    for r in range(R):
        np.add.at(A[r], rows, g.w * np.cos(2 * np.pi * th0[r, g.col]))
        np.add.at(B[r], rows, g.w * np.sin(2 * np.pi * th0[r, g.col]))
    D64 = np.stack([orc.coupling(g, th0[r]) for r in range(R)])
    err = np.linalg.norm(D - D64, axis=0)
    ref = np.sqrt(np.sum(A**2 + B**2, axis=0))
    live = ref > 0                       # isolated nodes have no coupling at all
    assert np.all(err[~live] == 0)
    assert np.max(err[live] / ref[live]) <= 1e-2


def test_empty_graph_zero_steps_and_single_node(orc):
    g = csr_from_edges(1, np.zeros(0, int), np.zeros(0, int))
    for form in FORMS:
        run = gpu_run(g, 2, 0.0, 1.0, 0.0, 0.01, 0, 3, 1, form=form)
        out = run.readout()
        assert out["score"].shape == (1, 3) and np.all(out["score"] == 0)
        run = gpu_run(g, 3, 0.0, 1.0, 0.1, 0.01, 40, 3, 1, form=form)
        ref = oracle_phases(orc, g, 3, 0.0, 1.0, 0.1, 0.01, 40, 3, 1)
        assert rad_dist(run.phases()[0], ref).max() <= 1e-3


def test_resident_single_replica_blocks_for_large_graph(orc):
    g = torus(160, 160, 4, "pm1")   # 25600 nodes: one FP32 replica (200 KB) per block
    T, R = 20, 3
    K, Ks, Kn = constant(T, 4.0), linear_ramp(T, 0, 1), constant(T, 0.1)
    run = gpu_run(g, 2, K, Ks, Kn, 0.01, T, R, 2, form="resident")
    assert run.info()["form"] == 2
    ref = oracle_phases(orc, g, 2, K, Ks, Kn, 0.01, T, R, 2, nthreads=8)
    assert rad_dist(run.phases()[0], ref).max() <= 1e-3


def test_invalid_form_requests():
    from paper_2505_22631_gb300 import OimError
    g = torus(300, 300, 1, "pm1")   # too large for a resident FP32 replica
    with pytest.raises(OimError) as ei:
        gpu_run(g, 2, 1.0, 1.0, 0.1, 0.01, 2, 4, 1, form="resident")
    assert ei.value.code == -5
    with pytest.raises(OimError) as ei:
        gpu_run(torus(4, 4, 1), 2, 1.0, 1.0, 0.1, 0.01, 2, 64, 1, form="gemm", precision="fp16")
    assert ei.value.code == -5
    with pytest.raises(OimError) as ei:
        gpu_run([torus(4, 4, 1), torus(4, 4, 2)], 2, 1.0, 1.0, 0.1, 0.01, 2, 64, 1, form="gemm")
    assert ei.value.code == -5


def test_autotune_picks_a_valid_cached_configuration(c1):
    import time
    from paper_2505_22631_gb300 import Problem, capi
    from workloads import torus
    p = Problem.batch([Problem.from_graph(c1.graphs[0], 2), Problem.from_graph(torus(20, 20, 3), 2)])
    o, us = capi.oim_autotune(p.handle, 64, capi.OIM_PREC_AUTO, 50)
    assert o.form in (capi.OIM_FORM_RESIDENT, capi.OIM_FORM_STREAM) and us > 0
    t0 = time.perf_counter()
    o2, us2 = capi.oim_autotune(p.handle, 64, capi.OIM_PREC_AUTO, 50)
    assert time.perf_counter() - t0 < 0.05 and us2 == us and o2.form == o.form   # cached
    o3, _ = capi.oim_autotune(p.handle, 64, capi.OIM_PREC_FP32, 50)
    assert o3.precision == capi.OIM_PREC_FP32
    # the chosen configuration runs
    T = 20
    K = np.full((2, T), 0.1, np.float32)
    r = capi.oim_run(p.handle, K, K, K, 0.01, T, 64, 1, o)
    capi.oim_run_sync(r)
    capi.oim_destroy_run(r)


@pytest.mark.parametrize("periods", [0, 2])
def test_parameter_sweep_is_one_batched_launch(orc, c1, periods):
    from paper_2505_22631_gb300 import Problem, oim_schedule_triangular, sweep
    g = c1.graphs[0]
    T, R = 40, 8
    run = sweep(Problem.from_graph(g, 2), [0.2, 0.4], [1.0, 2.0], 0.1, 0.01, T, R, 3, periods=periods,
                form="resident", precision="fp32")
    ph = run.phases()
    for gi, (k, smax) in enumerate(run.pairs):
        Ks = (oim_schedule_triangular(T, smax, periods) if periods else
              (smax * np.arange(T) / (T - 1)).astype(np.float32))
        ref = oracle_phases(orc, g, 2, np.full(T, k, np.float32), Ks, 0.1, 0.01, T, R, 3, graph=gi)
        assert rad_dist(ph[gi], ref).max() <= 1e-3


@pytest.mark.parametrize("form,precision,R", [("stream", "fp32", 8), ("stream", "fp16", 8),
                                              ("gemm", "bf16", 64)])
def test_rerun_with_a_new_seed_replays_the_captured_graph(c1, form, precision, R):
    # the per-step forms keep one captured graph per (steps, dt) and read the seed from
    # device memory: a rerun under another seed equals a fresh run under that seed
    from paper_2505_22631_gb300 import Problem, Run
    g = c1.graphs[0]
    T = 30
    sched = (c1.K[0][:T], c1.Ks[0][:T], c1.Kn[0][:T])
    prob = Problem.from_graph(g, 2)
    run = Run(prob, *sched, c1.dt, T, R, 5, form=form, precision=precision, readout_every=10)
    first = run.phases()[0]
    run.rerun(*sched, c1.dt, T, 9)
    again = run.phases()[0]
    trace = run.readout()["trace"]
    fresh = Run(prob, *sched, c1.dt, T, R, 9, form=form, precision=precision, readout_every=10)
    assert np.array_equal(again, fresh.phases()[0])
    assert np.array_equal(trace, fresh.readout()["trace"])
    assert not np.array_equal(first, again)


def test_stream_launch_shapes_agree_bitwise():
    # replicas are independent trajectories keyed by their index, so the first 16 replicas
    # of a 128-replica run (warps of 32 quads of one node) and of a 16-replica run (warps
    # spanning eight nodes) must agree bit for bit; the +-1 graph, 18 entries a row, takes
    # the mixed-add gather with its negated -1 runs in both
    g = erdos_renyi(600, 0.03, 19, "pm1")
    T = 40
    args = (g, 2, constant(T, 0.5), linear_ramp(T, 0, 1.5), constant(T, 0.1), 0.01, T)
    a = gpu_run(*args, 128, 7, form="stream", precision="fp16", readout_every=10)
    b = gpu_run(*args, 16, 7, form="stream", precision="fp16", readout_every=10)
    assert np.array_equal(a.phases()[0][:16], b.phases()[0])
    assert np.array_equal(a.readout()["trace"][:, :, :16], b.readout()["trace"])


@pytest.mark.parametrize("form,precision,R", [("resident", "fp32", 8), ("resident", "fp16", 8),
                                              ("stream", "fp32", 8), ("stream", "fp16", 8),
                                              ("gemm", "bf16", 64)])
def test_rerun_with_fewer_steps_runs_only_those(orc, c1, form, precision, R):
    # a run's schedule buffer keeps the stride of its longest run, so a shorter re-run must
    # take its step count from the call, not from that stride: it equals a fresh run of the
    # same steps (trace included), and a re-run of zero steps gives the initial phases
    from paper_2505_22631_gb300 import Problem, Run
    g = c1.graphs[0]
    prob = Problem.from_graph(g, 2)
    kw = dict(form=form, precision=precision, readout_every=10)
    T0, T1 = 40, 20
    run = Run(prob, c1.K[0][:T0], c1.Ks[0][:T0], c1.Kn[0][:T0], c1.dt, T0, R, 5, **kw)
    run.rerun(c1.K[0][:T1], c1.Ks[0][:T1], c1.Kn[0][:T1], c1.dt, T1, 9)
    short = run.phases()[0]
    trace = run.readout()["trace"]
    fresh = Run(prob, c1.K[0][:T1], c1.Ks[0][:T1], c1.Kn[0][:T1], c1.dt, T1, R, 9, **kw)
    assert np.array_equal(short, fresh.phases()[0])
    assert np.array_equal(trace, fresh.readout()["trace"])
    z = np.zeros(0, np.float32)
    run.rerun(z, z, z, c1.dt, 0, 77)
    assert np.array_equal(run.phases()[0], orc.init_phases(g.n, R, 77).astype(np.float32))


def test_overlapped_scoring_matches_inline_scoring(orc):
    # the stream form scores each readout on a second stream beside the next steps (in
    # the whole-run graph of a re-run; a first execution's chunks join it at each chunk's
    # end); the mixed form with every member in the stream form runs the same step
    # kernels and scores inline, so phases, traces and scores agree bit for bit, for the
    # first execution and for the captured re-runs
    g0 = erdos_renyi(2000, 0.01, 21, "+1")
    g1 = torus(40, 50, 22, "pm1")
    T, R = 200, 256
    K = [constant(T, 4.0 / g.mean_degree) for g in (g0, g1)]
    Ks, Kn = linear_ramp(T, 0, 1.5), constant(T, 0.1)
    a = gpu_run([g0, g1], 2, K, Ks, Kn, 0.01, T, R, 3, form="stream", precision="fp16", readout_every=25)
    b = gpu_run([g0, g1], 2, K, Ks, Kn, 0.01, T, R, 3, form="mixed", precision="fp16", readout_every=25,
                graph_forms=["stream", "stream"])
    for seed in (None, 4, 5):
        if seed is not None:
            a.rerun(K, Ks, Kn, 0.01, T, seed)
            b.rerun(K, Ks, Kn, 0.01, T, seed)
        pa, pb = a.phases(), b.phases()
        oa, ob = a.readout(), b.readout()
        for gi in range(2):
            assert np.array_equal(pa[gi], pb[gi])
        assert np.array_equal(oa["trace"], ob["trace"])
        assert np.array_equal(oa["score"], ob["score"])
    for gi, g in enumerate((g0, g1)):
        assert np.array_equal(oa["score"][gi], orc.scores(g, 2, orc.readout_f32(2, pa[gi])))


@pytest.mark.parametrize("form,precision", [("stream", "fp16"), ("stream", "fp32"), ("resident", "fp32")])
def test_batch_from_csr_arrays_runs_like_members_then_batch(form, precision):
    # oim_create_batch_csr lays the graphs out on host threads and joins them in one call;
    # its batch must be the one oim_create_problem per graph plus oim_create_batch build:
    # the same phases, scores and traces bit for bit (+-1 graphs with their sign runs, a
    # real-weight batch, a graph given as device arrays)
    import torch
    from paper_2505_22631_gb300 import Problem, Run, oim_create_batch_csr
    from workloads import sherrington_kirkpatrick
    T, R = 60, 64
    edgeless = csr_from_edges(5, np.zeros(0, np.int64), np.zeros(0, np.int64), None, "edgeless5")
    single = csr_from_edges(1, np.zeros(0, np.int64), np.zeros(0, np.int64), None, "single")
    cases = [[erdos_renyi(300, 0.05, 31, "pm1"), torus(12, 10, 32, "pm1"), erdos_renyi(200, 0.08, 33, "+1")],
             [sherrington_kirkpatrick(120, 34), erdos_renyi(250, 0.05, 35, "+1")],
             [erdos_renyi(100, 0.1, 36, "pm1"), edgeless, single]]
    for gs in cases:
        K = [constant(T, 2.0 / max(g.mean_degree, 1.0)) for g in gs]
        Ks, Kn = [linear_ramp(T, 0.0, 1.0)] * len(gs), [constant(T, 0.1)] * len(gs)
        sched = (np.stack(K), np.stack(Ks), np.stack(Kn))
        kw = dict(form=form, precision=precision, readout_every=20)
        ref_prob = Problem.batch([Problem.from_graph(g, 2) for g in gs])
        ref = Run(ref_prob, *sched, 0.01, T, R, 7, **kw)
        # the first graph's arrays on the device, the others on the host
        dev = [torch.from_numpy(np.ascontiguousarray(a)).cuda() for a in (gs[0].row_ptr, gs[0].col, gs[0].w)]
        h = oim_create_batch_csr([g.n for g in gs], 2, [g.nnz for g in gs], [dev[0]] + [g.row_ptr for g in gs[1:]],
                                 [dev[1]] + [g.col for g in gs[1:]], [dev[2]] + [g.w for g in gs[1:]])
        prob = Problem(h, len(gs), [g.n for g in gs], 2)
        run = Run(prob, *sched, 0.01, T, R, 7, **kw)
        for a, b in zip(ref.phases(), run.phases()):
            assert np.array_equal(a, b)
        ra, rb = ref.readout(energy=True), run.readout(energy=True)
        for key in ("score", "best_replica", "trace", "energy"):
            assert np.array_equal(ra[key], rb[key]), key
        # the Python form, and a batch whose upload waits for its first run
        from paper_2505_22631_gb300 import capi
        for flags in (0, capi.OIM_FLAG_DEFER_UPLOAD):
            same = Problem.from_graphs(gs, 2, flags=flags)
            again = Run(same, *sched, 0.01, T, R, 7, **kw)
            for a, b in zip(ref.phases(), again.phases()):
                assert np.array_equal(a, b)
