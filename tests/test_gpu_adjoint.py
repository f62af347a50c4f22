"""The GPU adjoint (oim_backward) against the FP64 oracle adjoint.

Tolerance: FP32 forward and adjoint vs FP64; over T <= 120 steps the per-entry
gradient error stays below 2e-3 of the largest gradient entry (the adjoint of a
100-step trajectory amplifies FP32 rounding like the forward does), and the loss
agrees to 1e-5 of sum |w|.
"""
import numpy as np
import pytest

from gpu_common import require_gpu
from workloads import csr_from_edges, erdos_renyi, linear_ramp, planted_partition, torus

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    require_gpu()


def gpu_grads(graphs, q, K, Ks, Kn, dt, T, R, seed, C):
    from paper_2505_22631_gb300 import Problem, capi
    probs = [Problem.from_graph(g, q) for g in graphs]
    prob = probs[0] if len(probs) == 1 else Problem.batch(probs)
    o = capi.oim_default_opts()
    o.form = capi.OIM_FORM_STREAM
    o.precision = capi.OIM_PREC_FP32
    o.checkpoint_every = C
    G = len(graphs)
    r = capi.oim_run(prob.handle, K, Ks, Kn, dt, T, R, seed, o)
    out = [np.zeros((G, T)) for _ in range(3)] + [np.zeros(G)]
    capi.oim_backward(r, *out)
    capi.oim_destroy_run(r)
    return out


@pytest.mark.parametrize("q", [2, 3])
@pytest.mark.parametrize("C", [1, 16, 1000])
def test_adjoint_matches_oracle(orc, q, C):
    g0 = erdos_renyi(40, 0.15, 3, "pm1")
    g1 = planted_partition(30, 3, 3.0, 4) if q == 3 else torus(5, 6, 5, "pm1")
    graphs = [g0, g1]
    T, R, dt, seed = 90, 6, 0.01, 7
    rng = np.random.default_rng(q)
    K = (0.1 + 0.1 * rng.random((2, T))).astype(np.float32)
    Ks = np.stack([linear_ramp(T, 0, 1.5)] * 2)
    Kn = (0.05 + 0.05 * rng.random((2, T))).astype(np.float32)
    dK, dKs, dKn, loss = gpu_grads(graphs, q, K, Ks, Kn, dt, T, R, seed, C)
    for gi, g in enumerate(graphs):
        L, rK, rKs, rKn = orc.adjoint(g, q, K[gi].astype(np.float64), Ks[gi].astype(np.float64),
                                      Kn[gi].astype(np.float64), float(np.float32(dt)), T, R, seed,
                                      graph=gi, nthreads=4)
        assert abs(loss[gi] - L) <= 1e-5 * np.abs(g.w).sum()
        for got, ref in ((dK[gi], rK), (dKs[gi], rKs), (dKn[gi], rKn)):
            assert np.max(np.abs(got - ref)) <= 2e-3 * np.max(np.abs(ref)) + 1e-6


def test_adjoint_general_weights_and_autograd(orc):
    import torch
    from paper_2505_22631_gb300 import Problem
    from paper_2505_22631_gb300.autograd import schedule_loss
    rng = np.random.default_rng(1)
    g = erdos_renyi(25, 0.3, 9, "+1")
    i, j, _ = g.edges()
    g = csr_from_edges(25, i, j, rng.uniform(-1.5, 1.5, i.shape[0]).astype(np.float32))
    T, R, dt, seed = 50, 4, 0.01, 3
    K = torch.full((1, T), 0.2, dtype=torch.float32, requires_grad=True)
    Ks = torch.from_numpy(linear_ramp(T, 0, 1.0)[None].copy()).requires_grad_(True)
    Kn = torch.full((1, T), 0.08, dtype=torch.float32, requires_grad=True)
    L = schedule_loss(Problem.from_graph(g, 2), K, Ks, Kn, dt, R, seed, checkpoint_every=7)
    (3.0 * L.sum()).backward()
    Lr, rK, rKs, rKn = orc.adjoint(g, 2, K.detach().numpy()[0].astype(np.float64),
                                   Ks.detach().numpy()[0].astype(np.float64),
                                   Kn.detach().numpy()[0].astype(np.float64), float(np.float32(dt)), T,
                                   R, seed)
    assert abs(L.item() - Lr) <= 1e-5 * np.abs(g.w).sum()
    for got, ref in ((K.grad, rK), (Ks.grad, rKs), (Kn.grad, rKn)):
        got = got.numpy()[0] / 3.0
        assert np.max(np.abs(got - ref)) <= 2e-3 * np.max(np.abs(ref)) + 1e-6


def test_backward_requires_checkpoints():
    from paper_2505_22631_gb300 import OimError, Problem, Run
    g = torus(4, 4, 1, "pm1")
    run = Run(Problem.from_graph(g, 2), 1.0, 0.5, 0.1, 0.01, 10, 4, 1, form="stream")
    from paper_2505_22631_gb300 import capi
    with pytest.raises(OimError) as ei:
        capi.oim_backward(run.handle, np.zeros((1, 10)), None, None, None)
    assert ei.value.code == capi.OIM_ESTATE


def test_whole_trajectory_mode_equals_recomputation():
    # checkpoint_every = 1 keeps every step's phases and coupling sums, so the backward
    # pass recomputes nothing: the same FP32 arithmetic as the recomputing pass (only the
    # order of the FP64 gradient sums differs), and a forward pass whose phases, scores
    # and trace are those of a run without checkpoints
    from paper_2505_22631_gb300 import Problem, capi
    graphs = [erdos_renyi(300, 0.05, 11, "pm1"), torus(12, 10, 12, "pm1")]
    prob = Problem.batch([Problem.from_graph(g, 2) for g in graphs])
    T, R, dt, seed = 120, 12, 0.01, 5
    rng = np.random.default_rng(7)
    K = (0.1 + 0.1 * rng.random((2, T))).astype(np.float32)
    Ks = np.stack([linear_ramp(T, 0, 1.5)] * 2)
    Kn = (0.05 + 0.05 * rng.random((2, T))).astype(np.float32)
    out = {}
    for C in (0, 1, 16):
        o = capi.oim_default_opts()
        o.form = capi.OIM_FORM_STREAM
        o.precision = capi.OIM_PREC_FP32
        o.checkpoint_every = C
        o.readout_every = 20
        r = capi.oim_run(prob.handle, K, Ks, Kn, dt, T, R, seed, o)
        th = np.zeros(prob.nodes * R, np.float32)
        capi.oim_get_phases(r, th)
        score, trace = np.zeros((2, R)), np.zeros((2, T // 20, R))
        capi.oim_readout(r, None, score, None, trace, None)
        grads = [np.zeros((2, T)) for _ in range(3)] + [np.zeros(2)]
        if C:
            capi.oim_backward(r, *grads)
        capi.oim_destroy_run(r)
        out[C] = (th, score, trace, grads)
    for C in (1, 16):
        assert np.array_equal(out[C][0], out[0][0])
        assert np.array_equal(out[C][1], out[0][1])
        assert np.array_equal(out[C][2], out[0][2])
    for a, b in zip(out[1][3], out[16][3]):
        assert np.allclose(a, b, rtol=1e-9, atol=1e-12 * max(1.0, np.abs(b).max()))
