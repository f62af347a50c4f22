"""Batches whose graphs take different forms (OIM_FORM_MIXED): the CSR members step
together in the stream form, each dense member on the tensor cores, every step.

- CSR members: the same step kernel over their own slots, so their phases and scores
  equal bit for bit those of a stream-form run of the whole batch (same seed, replicas
  and cache precision).
- Dense members: BF16 coupling within 1e-2 of the row norm, so against the oracle their
  phases lie within the linear accumulation of that bound over a short horizon, the
  bulk within 1e-3 rad.
- Every member's score is the exact recount of its own spins, and the trace's last row
  is the final score.
"""
import numpy as np
import pytest

from gpu_common import coupling_bound_rad, gpu_run, oracle_phases, rad_dist, require_gpu
from workloads import constant, erdos_renyi, linear_ramp, torus

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    require_gpu()


def _batch():
    return [torus(20, 10, 3, "pm1"), erdos_renyi(300, 0.05, 4, "+1"), erdos_renyi(256, 0.3, 5, "+1"),
            erdos_renyi(200, 0.04, 6, "pm1")]


def _sched(graphs, T):
    K = [constant(T, 4.0 / g.mean_degree) for g in graphs]
    return K, linear_ramp(T, 0, 1.5), constant(T, 0.1)


@pytest.mark.parametrize("precision", ["fp16", "fp32"])
def test_mixed_batch_members_against_stream_run_and_oracle(orc, precision):
    graphs = _batch()
    forms = ["stream", "stream", "gemm", "stream"]
    T, R, seed = 60, 64, 7
    K, Ks, Kn = _sched(graphs, T)
    mixed = gpu_run(graphs, 2, K, Ks, Kn, 0.01, T, R, seed, form="mixed", precision=precision,
                    readout_every=20, graph_forms=forms)
    assert mixed.info()["form"] == 4
    plain = gpu_run(graphs, 2, K, Ks, Kn, 0.01, T, R, seed, form="stream", precision=precision,
                    readout_every=20)
    pm, pp = mixed.phases(), plain.phases()
    om, op = mixed.readout(), plain.readout()
    for gi, g in enumerate(graphs):
        spins = orc.readout_f32(2, pm[gi])
        assert np.array_equal(om["spins"][gi], spins)
        assert np.array_equal(om["score"][gi], orc.scores(g, 2, spins))
        assert np.array_equal(om["trace"][gi, -1], om["score"][gi])
        if forms[gi] == "stream":
            assert np.array_equal(pm[gi], pp[gi])
            assert np.array_equal(om["trace"][gi], op["trace"][gi])
    # the dense member over a short horizon against the oracle
    Td = 10
    short = gpu_run(graphs, 2, [k[:Td] for k in K], Ks[:Td], Kn[:Td], 0.01, Td, R, seed, form="mixed",
                    precision=precision, graph_forms=forms).phases()[2]
    ref = oracle_phases(orc, graphs[2], 2, K[2][:Td], Ks[:Td], Kn[:Td], 0.01, Td, R, seed, graph=2)
    d = rad_dist(short, ref)
    assert d.max() <= coupling_bound_rad(graphs[2], K[2], Td, 0.01)
    assert np.median(d) <= 1e-3


def test_mixed_batch_rerun_replays_its_graph(orc):
    graphs = _batch()
    forms = ["gemm", "stream", "gemm", "stream"]
    T, R = 64, 64
    K, Ks, Kn = _sched(graphs, T)
    a = gpu_run(graphs, 2, K, Ks, Kn, 0.01, T, R, 3, form="mixed", readout_every=16, graph_forms=forms)
    b = gpu_run(graphs, 2, K, Ks, Kn, 0.01, T, R, 3, form="mixed", readout_every=16, graph_forms=forms,
                use_graph=False)
    for x, y in zip(a.phases(), b.phases()):
        assert np.array_equal(x, y)          # chunked replay = direct launches
    for seed in (4, 5):                      # the second rerun replays the whole captured run
        a.rerun(K, Ks, Kn, 0.01, T, seed)
        fresh = gpu_run(graphs, 2, K, Ks, Kn, 0.01, T, R, seed, form="mixed", readout_every=16,
                        graph_forms=forms, use_graph=False)
        for x, y in zip(a.phases(), fresh.phases()):
            assert np.array_equal(x, y)
        assert np.array_equal(a.readout()["trace"], fresh.readout()["trace"])


def test_mixed_batch_all_dense_and_all_csr(orc):
    graphs = _batch()[:3]
    T, R = 30, 64
    K, Ks, Kn = _sched(graphs, T)
    allcsr = gpu_run(graphs, 2, K, Ks, Kn, 0.01, T, R, 9, form="mixed", precision="fp16",
                     graph_forms=["stream"] * 3)
    stream = gpu_run(graphs, 2, K, Ks, Kn, 0.01, T, R, 9, form="stream", precision="fp16")
    for x, y in zip(allcsr.phases(), stream.phases()):
        assert np.array_equal(x, y)
    alldense = gpu_run(graphs, 2, K, Ks, Kn, 0.01, T, R, 9, form="mixed", graph_forms=["gemm"] * 3,
                       readout_every=10)
    ph = alldense.phases()
    out = alldense.readout()
    for gi, g in enumerate(graphs):
        assert np.array_equal(out["score"][gi], orc.scores(g, 2, orc.readout_f32(2, ph[gi])))


def test_mixed_form_rejects_bad_requests():
    from paper_2505_22631_gb300 import OimError
    graphs = _batch()[:2]
    T = 4
    K, Ks, Kn = _sched(graphs, T)
    with pytest.raises(OimError) as ei:
        gpu_run(graphs, 2, K, Ks, Kn, 0.01, T, 8, 1, form="mixed")            # no graph_forms
    assert ei.value.code == -1
    with pytest.raises(OimError) as ei:
        gpu_run(graphs, 2, K, Ks, Kn, 0.01, T, 8, 1, form="mixed", graph_forms=[1, 2])   # resident
    assert ei.value.code == -1


def test_autotuner_choice_for_a_batch_with_a_dense_member_runs():
    from paper_2505_22631_gb300 import Problem, Run, capi
    graphs = [torus(30, 20, 3, "pm1"), erdos_renyi(600, 0.01, 4, "+1"), erdos_renyi(1024, 0.1, 5, "+1")]
    probs = [Problem.from_graph(g, 2) for g in graphs]
    prob = Problem.batch(probs)
    o, us = capi.oim_autotune(prob.handle, 256, capi.OIM_PREC_AUTO, 100)
    forms = capi.graph_forms_of(o, len(graphs))
    print(f"autotuned: form {o.form} precision {o.precision} graph_forms {forms} ({us:.2f} us/step)")
    assert us > 0
    if o.form == capi.OIM_FORM_MIXED:
        assert forms is not None and len(forms) == 3
        assert set(forms) <= {capi.OIM_FORM_STREAM, capi.OIM_FORM_GEMM}
        assert forms[0] == capi.OIM_FORM_STREAM and forms[1] == capi.OIM_FORM_STREAM
    T = 20
    K = np.full((3, T), 0.05, np.float32)
    run = Run(prob, K, K, K, 0.01, T, 256, 1, form=o.form, precision=o.precision,
              replicas_per_block=o.replicas_per_block, threads_per_block=o.threads_per_block,
              graph_forms=forms)
    assert run.readout(spins=False)["score"].shape == (3, 256)
