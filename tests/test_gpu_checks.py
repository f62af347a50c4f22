"""The index-checked build (-DOIM_CHECKS, liboim_checks.so).

A column index is made to point outside its row's graph (into the other graph of a
batch: still inside every buffer, so no build can read out of bounds) through
oim_debug_set_column.  The checked build's step, adjoint and readout kernels must then
skip the entry and report OIM_EINDEX at the next synchronisation, and after the column
is put back they must give the phases of a clean run again.  The regular build reads the
named node as if it were a neighbour (a wrong but in-bounds trajectory, no error).
"""
import os
import subprocess
import sys
import textwrap

import numpy as np
import pytest

from gpu_common import require_gpu

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

SETUP = textwrap.dedent("""
    import sys
    import numpy as np
    sys.path.insert(0, {root!r})
    from workloads import constant, erdos_renyi, linear_ramp, torus
    ga = erdos_renyi(200, 0.08, 5, "pm1")
    gb = torus(10, 10, 6, "pm1")
    # the fifth entry of the first row of graph A with at least six entries
    v = next(i for i in range(ga.n) if ga.row_ptr[i + 1] - ga.row_ptr[i] >= 6)
    entry = int(ga.row_ptr[v]) + 4
    outside = ga.n + 5                     # a node of graph B
    T = 20
    K = [constant(T, 0.3), constant(T, 0.3)]
    Ks, Kn = linear_ramp(T, 0, 1.0), constant(T, 0.1)
""")


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    require_gpu()


def test_checked_build_reports_and_skips_foreign_columns():
    from paper_2505_22631_gb300 import build
    lib = build.build(checks=True)
    script = SETUP.format(root=ROOT) + textwrap.dedent(f"""
        from paper_2505_22631_gb300 import capi
        capi.load({lib!r})
        from paper_2505_22631_gb300 import OimError, Problem, Run
        prob = Problem.batch([Problem.from_graph(ga, 2), Problem.from_graph(gb, 2)])
        cases = [("stream", "fp16", 16), ("stream", "fp32", 8), ("resident", "fp32", 8),
                 ("resident", "fp16", 8)]
        for form, prec, R in cases:
            kw = dict(form=form, precision=prec, readout_every=10)
            sched = ([np.asarray(k) for k in K], Ks, Kn)
            clean = Run(prob, *sched, 0.01, T, R, 3, **kw).phases()
            original = capi.oim_debug_set_column(prob.handle, entry, outside)
            try:
                Run(prob, *sched, 0.01, T, R, 3, **kw).phases()
                raise SystemExit(f"{{form}} {{prec}}: no OIM_EINDEX")
            except OimError as e:
                assert e.code == capi.OIM_EINDEX, (form, prec, e.code)
            capi.oim_debug_set_column(prob.handle, entry, original)
            again = Run(prob, *sched, 0.01, T, R, 3, **kw).phases()
            assert all(np.array_equal(a, b) for a, b in zip(clean, again)), (form, prec)
        # the adjoint: the forward's steps record the foreign column, oim_backward reports it
        o = capi.oim_default_opts()
        o.form, o.precision, o.checkpoint_every = capi.OIM_FORM_STREAM, capi.OIM_PREC_FP32, 5
        KK = np.stack(K).astype(np.float32)
        KS = np.stack([Ks, Ks]).astype(np.float32)
        KN = np.stack([Kn, Kn]).astype(np.float32)
        original = capi.oim_debug_set_column(prob.handle, entry, outside)
        r = capi.oim_run(prob.handle, KK, KS, KN, 0.01, T, 8, 3, o)
        try:
            capi.oim_backward(r, np.zeros((2, T)), np.zeros((2, T)), np.zeros((2, T)), np.zeros(2))
            raise SystemExit("adjoint: no OIM_EINDEX")
        except OimError as e:
            assert e.code == capi.OIM_EINDEX, e.code
        capi.oim_destroy_run(r)
        capi.oim_debug_set_column(prob.handle, entry, original)
        print("checked ok")
    """)
    res = subprocess.run([sys.executable, "-c", script], capture_output=True, text=True, timeout=600)
    assert res.returncode == 0 and "checked ok" in res.stdout, res.stdout + res.stderr


def test_regular_build_reads_the_named_node_without_error():
    ns = {}
    exec(SETUP.format(root=ROOT), ns)
    from paper_2505_22631_gb300 import Problem, Run, capi
    ga, gb, entry, T = ns["ga"], ns["gb"], ns["entry"], ns["T"]
    prob = Problem.batch([Problem.from_graph(ga, 2), Problem.from_graph(gb, 2)])
    sched = ([np.asarray(k) for k in ns["K"]], ns["Ks"], ns["Kn"])
    clean = Run(prob, *sched, 0.01, T, 16, 3, form="stream", precision="fp16").phases()
    original = capi.oim_debug_set_column(prob.handle, entry, ns["outside"])
    moved = Run(prob, *sched, 0.01, T, 16, 3, form="stream", precision="fp16").phases()
    assert capi.oim_debug_set_column(prob.handle, entry, original) == ns["outside"]
    again = Run(prob, *sched, 0.01, T, 16, 3, form="stream", precision="fp16").phases()
    assert all(np.array_equal(a, b) for a, b in zip(clean, again))
    assert not np.array_equal(clean[0], moved[0])
    assert np.array_equal(clean[1], moved[1])          # graph B's own rows are untouched
    # entries among the first four of a row are refused (the slot descriptors hold them)
    with pytest.raises(Exception):
        capi.oim_debug_set_column(prob.handle, int(ga.row_ptr[ns["v"]]), ns["outside"])
