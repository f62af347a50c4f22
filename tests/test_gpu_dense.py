"""The dense (tcgen05 tensor-core) coupling form against the FP64 oracle.

Tolerances: the BF16 operands give the coupling sum to within 1e-2 of the row
norm of the FP64 (A, B) (the stated BF16 criterion); noise draws as the other
hardware-approximation forms (<= 2e-5); spins and scores from the form's own
phases are bit-exact.
"""
import numpy as np
import pytest

from gpu_common import circ, gpu_run, oracle_phases, rad_dist, require_gpu
from workloads import (constant, csr_from_edges, erdos_renyi, linear_ramp, make_workload,
                       sherrington_kirkpatrick)

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    require_gpu()


@pytest.mark.parametrize("n,p,R", [(800, 0.06, 64), (300, 0.2, 8), (1100, 0.03, 72), (900, 0.05, 256)])
def test_dense_coupling_within_1e2_per_row(orc, n, p, R):
    g = erdos_renyi(n, p, n, "pm1")
    dt, K = 1e-3, 1.0
    run = gpu_run(g, 2, K, 0.0, 0.0, dt, 1, R, 13, form="gemm", precision="bf16")
    assert run.info()["form"] == 3
    th0 = orc.init_phases(g.n, R, 13)
    D = circ(run.phases()[0].astype(np.float64) - th0) / (np.float32(dt) * K)
    rows = np.repeat(np.arange(g.n), g.degrees())
    A = np.zeros((R, g.n))
    B = np.zeros((R, g.n))
    for r in range(R):
        np.add.at(A[r], rows, g.w * np.cos(2 * np.pi * th0[r, g.col]))
        np.add.at(B[r], rows, g.w * np.sin(2 * np.pi * th0[r, g.col]))
    D64 = np.stack([orc.coupling(g, th0[r]) for r in range(R)])
    err = np.linalg.norm(D - D64, axis=0)
    ref = np.sqrt(np.sum(A**2 + B**2, axis=0))
    assert np.max(err / ref) <= 1e-2


def test_dense_noise_draws(orc):
    n, R, kick = 500, 64, 0.05
    g = csr_from_edges(n, np.zeros(0, int), np.zeros(0, int))
    run = gpu_run(g, 2, 0.0, 0.0, kick, 1.0, 1, R, 6, form="gemm", precision="bf16")
    th1 = run.phases()[0].astype(np.float64)
    th0 = orc.init_phases(n, R, 6)
    err = np.abs(circ(th1 - th0) / kick - orc.noise_block(n, R, 6, 0))
    assert err.max() <= 2e-5


@pytest.mark.parametrize("R", [8, 70])
def test_dense_readout_bitexact_and_short_run_parity(orc, R):
    w = make_workload("er800")
    g = w.graphs[0]
    T = 100
    run = gpu_run(g, 2, w.K[0][:T], w.Ks[0][:T], w.Kn[0][:T], w.dt, T, R, 5, form="gemm",
                  precision="bf16", readout_every=25)
    th = run.phases()[0]
    out = run.readout()
    spins = orc.readout_f32(2, th)
    assert np.array_equal(out["spins"][0], spins)
    assert np.array_equal(out["score"][0], orc.scores(g, 2, spins))
    assert np.array_equal(out["trace"][0, -1], out["score"][0])
    # BF16 coupling: short horizon phase agreement with the FP64 oracle, loose
    ref = oracle_phases(orc, g, 2, w.K[0][:20], w.Ks[0][:20], w.Kn[0][:20], w.dt, 20, R, 5)
    run20 = gpu_run(g, 2, w.K[0][:20], w.Ks[0][:20], w.Kn[0][:20], w.dt, 20, R, 5, form="gemm",
                    precision="bf16")
    assert np.median(rad_dist(run20.phases()[0], ref)) <= 1e-3


@pytest.mark.parametrize("R", [64, 128])
def test_dense_graph_capture_matches_direct(R):
    g = erdos_renyi(400, 0.1, 2, "+1")
    T = 40
    args = (g, 2, constant(T, 0.3), linear_ramp(T, 0, 1), constant(T, 0.1), 0.01, T, R, 3)
    ra = gpu_run(*args, form="gemm", precision="bf16", use_graph=True)
    ra.rerun(constant(T, 0.3), linear_ramp(T, 0, 1), constant(T, 0.1), 0.01, T, 3)   # graph replay
    a = ra.phases()[0]
    b = gpu_run(*args, form="gemm", precision="bf16", use_graph=False).phases()[0]
    assert np.array_equal(a, b)


def test_dense_chunked_first_execution_matches_direct(orc):
    """The dense form's first execution replays a captured chunk of steps (step base and
    readout slot read from device memory) and launches the remaining steps directly:
    phases, trace and scores equal those of direct launches bit for bit, also after a
    rerun that grows the run."""
    g = erdos_renyi(500, 0.08, 4, "pm1")
    R = 128
    K, Ks, Kn = constant(300, 0.2), linear_ramp(300, 0, 1), constant(300, 0.1)
    # readout every 25 steps: chunks of 50; 130 steps = 2 chunks and a 30-step tail
    a = gpu_run(g, 2, K[:130], Ks[:130], Kn[:130], 0.01, 130, R, 3, form="gemm", precision="bf16",
                readout_every=25, use_graph=True)
    b = gpu_run(g, 2, K[:130], Ks[:130], Kn[:130], 0.01, 130, R, 3, form="gemm", precision="bf16",
                readout_every=25, use_graph=False)

    def same(x, y):
        assert np.array_equal(x.phases()[0], y.phases()[0])
        ox, oy = x.readout(), y.readout()
        assert np.array_equal(ox["trace"], oy["trace"])
        assert np.array_equal(ox["score"], oy["score"])
        return ox

    out = same(a, b)
    assert np.array_equal(out["score"][0], orc.scores(g, 2, orc.readout_f32(2, a.phases()[0])))
    for steps, seed in ((300, 4), (300, 5)):   # the second pass replays the captured run
        a.rerun(K[:steps], Ks[:steps], Kn[:steps], 0.01, steps, seed)
        b.rerun(K[:steps], Ks[:steps], Kn[:steps], 0.01, steps, seed)
        same(a, b)


def test_dense_real_valued_all_to_all_coupling_within_1e2_per_row(orc):
    # Gaussian couplings on every pair: the BF16 operands still meet the per-row bound
    g = sherrington_kirkpatrick(384, 11)
    R, dt, K = 64, 1e-3, 1.0
    run = gpu_run(g, 2, K, 0.0, 0.0, dt, 1, R, 21, form="gemm", precision="bf16")
    assert run.info()["form"] == 3
    th0 = orc.init_phases(g.n, R, 21)
    D = circ(run.phases()[0].astype(np.float64) - th0) / (np.float32(dt) * K)
    rows = np.repeat(np.arange(g.n), g.degrees())
    A = np.zeros((R, g.n))
    B = np.zeros((R, g.n))
    for r in range(R):
        np.add.at(A[r], rows, g.w * np.cos(2 * np.pi * th0[r, g.col]))
        np.add.at(B[r], rows, g.w * np.sin(2 * np.pi * th0[r, g.col]))
    D64 = np.stack([orc.coupling(g, th0[r]) for r in range(R)])
    err = np.linalg.norm(D - D64, axis=0)
    ref = np.sqrt(np.sum(A**2 + B**2, axis=0))
    assert np.max(err / ref) <= 1e-2


@pytest.mark.parametrize("q", [4, 5])
def test_dense_potts_readout_and_short_run_parity(orc, q):
    g = sherrington_kirkpatrick(200, 3 + q)
    T, R = 20, 64
    K, Ks, Kn = constant(T, 0.05), linear_ramp(T, 0, 1), constant(T, 0.1)
    run = gpu_run(g, q, K, Ks, Kn, 0.01, T, R, 9, form="gemm", precision="bf16", readout_every=10)
    th = run.phases()[0]
    out = run.readout()
    spins = orc.readout_f32(q, th)
    assert np.array_equal(out["spins"][0], spins)
    # real weights: each node's agreeing weight is an FP32 sum of at most n - 1 terms
    # (then FP64 across nodes), so it is off by at most (n - 1) 2^-24 sum |w| in total
    bound = (g.n - 1) * 2.0**-24 * np.abs(g.w).sum() / 2
    assert np.max(np.abs(out["score"][0] - orc.scores(g, q, spins))) <= bound
    ref = oracle_phases(orc, g, q, K, Ks, Kn, 0.01, T, R, 9)
    assert np.median(rad_dist(th, ref)) <= 1e-3


@pytest.mark.parametrize("n,R", [(800, 64), (1000, 192), (2000, 4096)])
def test_dense_tile_widths_agree_bitwise(n, R):
    # 112-, 128- and 256-wide tiles run the same K-ordered products (zero padding adds
    # exact zeros), so the launch shapes give identical phases and scores (320 threads
    # takes 112-wide tiles for the first two shapes and 128-wide for the third)
    g = erdos_renyi(n, 0.05, 17, "pm1")
    T = 30
    args = (g, 2, constant(T, 0.3), linear_ramp(T, 0, 1), constant(T, 0.1), 0.01, T, R, 3)
    a = gpu_run(*args, form="gemm", precision="bf16", readout_every=10, threads_per_block=320)
    b = gpu_run(*args, form="gemm", precision="bf16", readout_every=10, threads_per_block=576)
    assert np.array_equal(a.phases()[0], b.phases()[0])
    assert np.array_equal(a.readout()["trace"], b.readout()["trace"])


def test_dense_rejects_unknown_tile_request():
    from paper_2505_22631_gb300 import OimError
    g = erdos_renyi(200, 0.05, 1, "+1")
    with pytest.raises(OimError) as ei:
        gpu_run(g, 2, 0.3, 0.5, 0.1, 0.01, 2, 64, 1, form="gemm", precision="bf16", threads_per_block=512)
    assert ei.value.code == -1
