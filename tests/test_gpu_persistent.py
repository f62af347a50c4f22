"""The persistent form (OIM_FORM_PERSISTENT): the 16-bit stream form's steps between two
readouts in one cooperative launch with a grid barrier per step.  Every (node, replica
octet) item does the arithmetic of the per-step kernel, so phases, traces and scores
equal those of the 16-bit stream form bit for bit, also when the per-step grid has more
blocks than the GPU holds at once (each block then walks several of them per step)."""
import numpy as np
import pytest

from gpu_common import gpu_run, require_gpu
from workloads import constant, erdos_renyi, gnm, linear_ramp, torus

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    require_gpu()


def _same(a, b):
    for x, y in zip(a.phases(), b.phases()):
        assert np.array_equal(x, y)
    oa, ob = a.readout(), b.readout()
    assert np.array_equal(oa["trace"], ob["trace"])
    assert np.array_equal(oa["score"], ob["score"])


@pytest.mark.parametrize("precision", ["fp16", "bf16"])
def test_persistent_equals_stream_form(precision):
    graphs = [torus(20, 12, 3, "pm1"), erdos_renyi(400, 0.04, 4, "+1")]
    T, R = 120, 64
    K = [constant(T, 4.0 / g.mean_degree) for g in graphs]
    Ks, Kn = linear_ramp(T, 0, 1.5), constant(T, 0.1)
    a = gpu_run(graphs, 2, K, Ks, Kn, 0.01, T, R, 5, form="persistent", precision=precision, readout_every=40)
    assert a.info()["form"] == 5
    b = gpu_run(graphs, 2, K, Ks, Kn, 0.01, T, R, 5, form="stream", precision=precision, readout_every=40)
    _same(a, b)
    a.rerun(K, Ks, Kn, 0.01, T, 6)
    b.rerun(K, Ks, Kn, 0.01, T, 6)
    _same(a, b)


def test_persistent_strides_over_a_grid_larger_than_the_gpu():
    graphs = [torus(150, 100, 7, "pm1"), gnm(3000, 12000, 8, "+1")]   # 18000 nodes, 256 replicas
    T, R = 30, 256
    K = [constant(T, 4.0 / g.mean_degree) for g in graphs]
    Ks, Kn = linear_ramp(T, 0, 1.0), constant(T, 0.1)
    a = gpu_run(graphs, 2, K, Ks, Kn, 0.01, T, R, 9, form="persistent", precision="fp16", readout_every=10)
    b = gpu_run(graphs, 2, K, Ks, Kn, 0.01, T, R, 9, form="stream", precision="fp16", readout_every=10)
    _same(a, b)


def test_persistent_form_rejects_fp32_and_checkpoints():
    from paper_2505_22631_gb300 import OimError
    g = torus(6, 6, 1, "pm1")
    with pytest.raises(OimError) as ei:
        gpu_run(g, 2, 1.0, 1.0, 0.1, 0.01, 4, 8, 1, form="persistent", precision="fp32")
    assert ei.value.code == -5
