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
from workloads import erdos_renyi, torus

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
