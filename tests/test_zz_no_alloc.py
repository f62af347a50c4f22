"""GPU test of oim_score_phases_noalloc, the scoring entry point that allocates nothing.

Callers that must not have a library allocate device memory (a fixed memory
footprint reserved at start-up, their own allocator owning the device, or no
room for the synchronisation an allocation can bring) score phases with this
call; its only scratch is a fixed array inside the library.  The test checks
that its scores equal those of the regular readout path, exactly (integer
weights), on two calls in a row with different phases, so scratch left over
from the first call would show up in the second.  The file is named to be
collected last.
"""
import numpy as np
import pytest

from gpu_common import gpu_run, require_gpu
from workloads import csr_from_edges, erdos_renyi, planted_partition, torus

pytestmark = pytest.mark.gpu


def _node_major(phases, R, ld):
    """Per-graph [R, n_g] phases -> one [nodes, ld] array (replicas contiguous)."""
    nodes = sum(p.shape[1] for p in phases)
    out = np.zeros((nodes, ld), dtype=np.float32)
    off = 0
    for p in phases:
        out[off:off + p.shape[1], :R] = p.T
        off += p.shape[1]
    return out


def test_noalloc_scores_match_readout_on_consecutive_calls():
    require_gpu()
    import torch
    from paper_2505_22631_gb300 import capi

    graphs = [torus(12, 10, 3, "pm1"), erdos_renyi(150, 0.05, 4, "+1")]
    R, ld, T = 20, 24, 60
    stream = torch.cuda.current_stream()
    for seed in (3, 4):
        run = gpu_run(graphs, 2, 1.0, 1.0, 0.1, 0.01, T, R, seed,
                      form="resident", precision="fp32")
        ref = run.readout(spins=False)["score"]
        theta = torch.from_numpy(_node_major(run.phases(), R, ld)).cuda()
        score = torch.full((len(graphs) * R,), -1.0, dtype=torch.float64, device="cuda")
        capi.oim_score_phases_noalloc(run.problem.handle, theta, R, ld, score,
                                      int(stream.cuda_stream))
        torch.cuda.synchronize()
        got = score.cpu().numpy().reshape(len(graphs), R)
        assert np.array_equal(got, ref), (seed, np.abs(got - ref).max())


def _weighted(g, kind, seed):
    """g's edges with integer weights in {-2, -1, 1, 3} or real weights in [-2, 2]."""
    rng = np.random.default_rng(seed)
    i, j, _ = g.edges()
    w = rng.choice([-2, -1, 1, 3], i.shape[0]) if kind == "integer" else rng.uniform(-2, 2, i.shape[0])
    return csr_from_edges(g.n, i, j, w.astype(np.float32))


@pytest.mark.parametrize("case", ["q3_planted", "integer_weights", "real_weights"])
def test_noalloc_scores_match_oracle_and_allocate_nothing(orc, case):
    """Colouring conflicts (q = 3) and general weights, against both the regular
    readout path and the oracle's recount from the same spins; and a second call
    changes the device's free memory by nothing."""
    require_gpu()
    import torch
    from paper_2505_22631_gb300 import capi

    if case == "q3_planted":
        q, graphs = 3, [planted_partition(90, 3, 4.0, 6), planted_partition(60, 3, 3.0, 8)]
    else:
        kind = "integer" if case == "integer_weights" else "real"
        q, graphs = 2, [_weighted(erdos_renyi(70, 0.1, 3, "+1"), kind, 1),
                        _weighted(torus(8, 6, 2, "pm1"), kind, 2)]
    R, ld, T = 12, 16, 40
    run = gpu_run(graphs, q, 0.5, 1.0, 0.1, 0.01, T, R, 11, form="stream", precision="fp32")
    ref = run.readout(spins=False)["score"]
    ph = run.phases()
    theta = torch.from_numpy(_node_major(ph, R, ld)).cuda()
    score = torch.full((len(graphs) * R,), -1.0, dtype=torch.float64, device="cuda")
    stream = int(torch.cuda.current_stream().cuda_stream)
    capi.oim_score_phases_noalloc(run.problem.handle, theta, R, ld, score, stream)
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    score.fill_(-1.0)
    capi.oim_score_phases_noalloc(run.problem.handle, theta, R, ld, score, stream)
    torch.cuda.synchronize()
    free1 = torch.cuda.mem_get_info()[0]
    assert free1 == free0
    got = score.cpu().numpy().reshape(len(graphs), R)
    for gi, g in enumerate(graphs):
        rec = orc.scores(g, q, orc.readout_f32(q, ph[gi]))
        if case == "real_weights":   # FP32 partial sums per node, FP64 totals
            assert np.allclose(got[gi], rec, rtol=1e-6, atol=1e-4)
            assert np.allclose(got[gi], ref[gi], rtol=1e-6, atol=1e-4)
        else:
            assert np.array_equal(got[gi], rec)
            assert np.array_equal(got[gi], ref[gi])


def test_noalloc_rejects_oversized_and_host_buffers():
    require_gpu()
    import torch
    from paper_2505_22631_gb300 import capi

    run = gpu_run(torus(6, 6, 1, "pm1"), 2, 1.0, 1.0, 0.1, 0.01, 4, 4, 1, form="resident",
                  precision="fp32")
    h = run.problem.handle
    big = capi.OIM_NOALLOC_MAX_ACCUM + 4
    theta = torch.zeros((36, 4), dtype=torch.float32, device="cuda")
    score = torch.zeros(4, dtype=torch.float64, device="cuda")
    with pytest.raises(capi.OimError) as ei:
        capi.oim_score_phases_noalloc(h, theta, 4, big, score)
    assert ei.value.code == capi.OIM_EINVAL
    with pytest.raises(capi.OimError) as ei:
        capi.oim_score_phases_noalloc(h, theta.cpu().numpy(), 4, 4, score)
    assert ei.value.code == capi.OIM_EINVAL
    # a view that starts one float into an allocation is not 16-byte aligned: rejected
    # before any launch (the kernel reads four replicas per 16-byte load)
    flat = torch.zeros(36 * 4 + 4, dtype=torch.float32, device="cuda")
    with pytest.raises(capi.OimError) as ei:
        capi.oim_score_phases_noalloc(h, flat[1:1 + 36 * 4], 4, 4, score)
    assert ei.value.code == capi.OIM_EINVAL
    capi.oim_score_phases_noalloc(h, flat[4:4 + 36 * 4], 4, 4, score)   # 16-byte aligned view
    torch.cuda.synchronize()
