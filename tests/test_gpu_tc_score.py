"""Readouts of dense-form graphs on the tensor cores.

For q = 2 the agreeing weight of a spin assignment s in {-1, +1}^n is
sum_{i<j} w_ij [s_i == s_j] = (sum_ij w_ij + s^T W s) / 4 (W symmetric, zero
diagonal), and with integer weights |w_ij| <= 256 (exact in BF16) and row sums of
|w| below 2^17 every partial sum of P^T = S^T W and of s^T P is an integer below
2^24, so the tensor-core score is exact.  The checks:

- the final scores equal the oracle's recount of the run's own spins (Eq. 1);
- every trace row equals the same run's with every graph on the CSR score pass
  (same seed and form: identical phases, the readouts differ only in how they are
  scored), through the replayed chunk of steps (slot from the device step base) and
  the directly launched remainder;
- graphs outside the exact range (non-integer weights) stay on the CSR pass and
  meet the same checks.
"""
import numpy as np
import pytest

from gpu_common import gpu_run, require_gpu
from workloads import constant, erdos_renyi, linear_ramp, torus
from workloads.graphs import csr_from_edges

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    require_gpu()


def _reweighted(g, seed, kind):
    """g's edges with integer weights in [-5, 5] \\ {0}, or those plus a half."""
    i, j, _ = g.edges()
    rng = np.random.default_rng(seed)
    w = rng.integers(1, 6, i.shape[0]) * np.where(rng.random(i.shape[0]) < 0.5, -1, 1)
    if kind == "half":
        w = w + 0.5
    return csr_from_edges(g.n, i, j, w.astype(np.float32), f"{g.name}_{kind}")


def _sched(graphs, T):
    K = [constant(T, 4.0 / max(g.mean_degree, 1.0)) for g in graphs]
    return K, linear_ramp(T, 0, 1.5), constant(T, 0.1)


def _check(orc, graphs, run, ref):
    ph = run.phases()
    out, out_ref = run.readout(), ref.readout()
    for gi, g in enumerate(graphs):
        spins = orc.readout_f32(2, ph[gi])
        assert np.array_equal(out["spins"][gi], spins)
        assert np.array_equal(out["score"][gi], orc.scores(g, 2, spins)), f"graph {gi}: final scores"
        assert np.array_equal(out["trace"][gi], out_ref["trace"][gi]), f"graph {gi}: trace"
        assert np.array_equal(out["trace"][gi, -1], out["score"][gi])
    assert np.array_equal(out["score"], out_ref["score"])


@pytest.mark.parametrize("kind", ["int", "pm1", "half"])
@pytest.mark.parametrize("tpb", [0, 576])
def test_dense_form_scores_against_csr_pass_and_oracle(orc, kind, tpb):
    base = erdos_renyi(333, 0.5, 41, "pm1")
    g = base if kind == "pm1" else _reweighted(base, 42, kind)
    T, R, seed = 60, 72, 5          # 333 nodes and 72 replicas: ragged node and replica tiles
    K, Ks, Kn = _sched([g], T)
    kw = dict(form="gemm", precision="bf16", readout_every=10, threads_per_block=tpb)
    run = gpu_run(g, 2, K[0], Ks, Kn, 0.01, T, R, seed, **kw)
    ref = gpu_run(g, 2, K[0], Ks, Kn, 0.01, T, R, seed, csr_scores=True, **kw)
    assert np.array_equal(run.phases()[0], ref.phases()[0])
    _check(orc, [g], run, ref)
    # a second, identical run replays the whole run from a CUDA graph
    run.rerun(K[0], Ks, Kn, 0.01, T, seed)
    _check(orc, [g], run, ref)


def test_mixed_batch_dense_members_scored_on_tensor_cores(orc):
    graphs = [torus(20, 10, 3, "pm1"), _reweighted(erdos_renyi(300, 0.4, 43, "pm1"), 44, "int"),
              erdos_renyi(200, 0.04, 6, "pm1"), erdos_renyi(256, 0.3, 5, "+1")]
    forms = ["stream", "gemm", "stream", "gemm"]
    T, R, seed = 80, 64, 9
    K, Ks, Kn = _sched(graphs, T)
    kw = dict(form="mixed", precision="fp16", readout_every=20, graph_forms=forms)
    run = gpu_run(graphs, 2, K, Ks, Kn, 0.01, T, R, seed, **kw)
    ref = gpu_run(graphs, 2, K, Ks, Kn, 0.01, T, R, seed, csr_scores=True, **kw)
    _check(orc, graphs, run, ref)


def test_dense_only_batch_member_and_zero_steps(orc):
    # a mixed run whose every member is dense (no CSR score pass at all), and a run of
    # zero steps (the readout scores the initial phases)
    graphs = [_reweighted(erdos_renyi(150, 0.6, 45, "pm1"), 46, "int"), erdos_renyi(190, 0.5, 47, "pm1")]
    kw = dict(form="mixed", precision="fp16", graph_forms=["gemm", "gemm"])
    for T, every in ((40, 8), (0, 0)):
        K, Ks, Kn = _sched(graphs, max(T, 1))
        K = [k[:T] for k in K]
        run = gpu_run(graphs, 2, K, Ks[:T], Kn[:T], 0.01, T, 64, 3, readout_every=every, **kw)
        ref = gpu_run(graphs, 2, K, Ks[:T], Kn[:T], 0.01, T, 64, 3, readout_every=every, csr_scores=True, **kw)
        ph = run.phases()
        out, out_ref = run.readout(), ref.readout()
        for gi, g in enumerate(graphs):
            spins = orc.readout_f32(2, ph[gi])
            assert np.array_equal(out["score"][gi], orc.scores(g, 2, spins))
        assert np.array_equal(out["score"], out_ref["score"])
        if every:
            assert np.array_equal(out["trace"], out_ref["trace"])
