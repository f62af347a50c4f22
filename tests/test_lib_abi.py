"""The C-ABI library builds, loads and exports every entry point include/oim.h declares.

These run without a GPU: no call here launches device work.  Argument
validation happens on the host before any device call, so malformed inputs are
rejected with OIM_EINVAL on any machine.
"""
import ctypes
import os
import re
import subprocess
import tempfile

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "oim.h")


@pytest.fixture(scope="module")
def capi():
    from paper_2505_22631_gb300 import build, capi
    build.build()
    capi.load()
    return capi


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"^\s*(?:int|void|const char\*)\s+(oim_\w+)\s*\(", text, flags=re.M)))


def test_every_declared_symbol_is_exported(capi):
    decl = declared_functions()
    assert len(decl) >= 15
    out = subprocess.run(["nm", "-D", "--defined-only", capi.LIB_PATH], capture_output=True,
                         text=True, check=True).stdout
    exported = set(re.findall(r" T (oim_\w+)$", out, flags=re.M))
    missing = [f for f in decl if f not in exported]
    assert not missing, missing
    # and the Python binding declares each one with the same name
    assert sorted(capi.SIGNATURES) == decl


def test_opts_struct_layout_matches_header(capi):
    src = r"""
    #include <stdio.h>
    #include <stddef.h>
    #include "oim.h"
    int main(void) {
        printf("%zu %zu %zu %zu %zu %zu %zu %zu %zu %zu\n", sizeof(oim_run_opts),
               offsetof(oim_run_opts, readout_every), offsetof(oim_run_opts, stream),
               offsetof(oim_run_opts, use_graph), offsetof(oim_run_opts, replicas_per_block),
               offsetof(oim_run_opts, threads_per_block), offsetof(oim_run_opts, checkpoint_every),
               offsetof(oim_run_opts, graph_forms), offsetof(oim_run_opts, csr_scores),
               offsetof(oim_run_opts, reserved));
        return 0;
    }
    """
    with tempfile.TemporaryDirectory() as d:
        c = os.path.join(d, "t.c")
        exe = os.path.join(d, "t")
        open(c, "w").write(src)
        subprocess.run(["gcc", "-I" + os.path.join(ROOT, "include"), c, "-o", exe], check=True)
        vals = [int(x) for x in subprocess.run([exe], capture_output=True, text=True,
                                               check=True).stdout.split()]
    S = capi.oim_run_opts
    got = [ctypes.sizeof(S), S.readout_every.offset, S.stream.offset, S.use_graph.offset,
           S.replicas_per_block.offset, S.threads_per_block.offset, S.checkpoint_every.offset,
           S.graph_forms.offset, S.csr_scores.offset, S.reserved.offset]
    assert got == vals


def test_default_opts_and_version(capi):
    o = capi.oim_default_opts()
    assert o.form == capi.OIM_FORM_AUTO and o.precision == capi.OIM_PREC_AUTO
    assert o.use_graph == 1 and o.readout_every == 0
    assert "sm_103a" in capi.oim_version()


def _csr(n, edges, w=None):
    from workloads import csr_from_edges
    e = np.array(edges)
    return csr_from_edges(n, e[:, 0], e[:, 1], w)


@pytest.mark.parametrize("case", ["diag", "range", "unsorted", "asym", "rowptr", "q", "n", "nan"])
def test_malformed_problems_rejected(capi, case):
    g = _csr(4, [(0, 1), (1, 2), (2, 3)], [1.0, 2.0, 3.0])
    n, q = 4, 2
    rp, col, w = g.row_ptr.copy(), g.col.copy(), g.w.copy()
    if case == "diag":
        col[0] = 0
    elif case == "range":
        col[-1] = 7
    elif case == "unsorted":
        rp = np.array([0, 1, 3, 5, 6], dtype=np.int64)
        col = np.array([1, 2, 0, 3, 1, 2], dtype=np.int32)   # row 1 = [2, 0]
        w = np.ones(6, dtype=np.float32)
    elif case == "asym":
        w[0] = 5.0
    elif case == "rowptr":
        rp[2] = rp[1] - 1
    elif case == "q":
        q = 1
    elif case == "n":
        n = 0
    elif case == "nan":
        w[1] = np.nan
    with pytest.raises(capi.OimError) as ei:
        capi.oim_create_problem(n, q, col.shape[0], rp, col, w)
    assert ei.value.code == capi.OIM_EINVAL
    assert capi.oim_last_error() != ""


def test_symmetry_check_agrees_with_the_dense_definition(capi):
    """The library accepts a CSR exactly when its dense matrix equals its transpose
    (W = W^T, the coupling of Eq. 1-2): random symmetric graphs, and the same graphs
    with one entry dropped, one weight changed or one entry added."""
    rng = np.random.default_rng(5)
    for trial in range(60):
        n = int(rng.integers(2, 30))
        W = np.triu(rng.integers(-2, 3, size=(n, n)).astype(np.float32) * (rng.random((n, n)) < 0.3), 1)
        W = W + W.T
        kind = trial % 4
        if kind and np.count_nonzero(W):
            nz = np.argwhere(W != 0)
            i, j = nz[rng.integers(len(nz))]
            if kind == 1:
                W[i, j] = 0.0                       # drop (i, j), keep (j, i)
            elif kind == 2:
                W[i, j] += 1.0 if W[i, j] != -1.0 else 2.0   # a different weight
        if kind == 3:
            i, j = rng.choice(n, 2, replace=False)
            W[i, j] = 7.0 if W[j, i] != 7.0 else 9.0   # an entry whose mirror differs
        rows, cols = np.nonzero(W)
        rp = np.zeros(n + 1, np.int64)
        np.add.at(rp, rows + 1, 1)
        rp = np.cumsum(rp)
        col = cols.astype(np.int32)
        w = W[rows, cols].astype(np.float32)
        symmetric = np.array_equal(W, W.T)
        try:
            h = capi.oim_create_problem(n, 2, col.shape[0], rp, col, w, capi.OIM_FLAG_DEFER_UPLOAD)
            capi.oim_destroy_problem(h)
            accepted = True
        except capi.OimError as e:
            assert e.code == capi.OIM_EINVAL
            accepted = False
        assert accepted == symmetric, (trial, kind)


def test_batch_from_csr_arrays_checks_every_graph(capi):
    """oim_create_batch_csr (graphs checked on host threads, upload deferred here): the
    batch has the graphs' sizes, a malformed graph is rejected with the checks of
    oim_create_problem and its index in the message, and empty or NULL lists are refused."""
    from workloads import erdos_renyi, torus
    gs = [erdos_renyi(60 + 10 * k, 0.1, k, "pm1" if k % 2 else "+1") for k in range(6)] + [torus(6, 5, 3, "pm1")]
    ws = [None if k % 3 == 0 else g.w for k, g in enumerate(gs)]
    h = capi.oim_create_batch_csr([g.n for g in gs], 2, [g.nnz for g in gs], [g.row_ptr for g in gs],
                                  [g.col for g in gs], ws, capi.OIM_FLAG_DEFER_UPLOAD)
    assert capi.oim_problem_info(h) == (len(gs), sum(g.n for g in gs), sum(g.nnz for g in gs), 2)
    capi.oim_destroy_problem(h)
    # graphs without edges and a single node are graphs like any other
    empty_rp, empty_col = np.zeros(6, np.int64), np.zeros(0, np.int32)
    h = capi.oim_create_batch_csr([5, 1, gs[0].n], 2, [0, 0, gs[0].nnz], [empty_rp, empty_rp[:2], gs[0].row_ptr],
                                  [empty_col, empty_col, gs[0].col], None, capi.OIM_FLAG_DEFER_UPLOAD)
    assert capi.oim_problem_info(h) == (3, 6 + gs[0].n, gs[0].nnz, 2)
    capi.oim_destroy_problem(h)
    # graph 4 gets a diagonal entry, graph 5 an asymmetric weight: the first is named
    bad_col = gs[4].col.copy()
    bad_col[gs[4].row_ptr[3]] = 3
    bad_w = gs[5].w.copy()
    bad_w[0] = 3.0
    cols = [g.col for g in gs]
    cols[4] = bad_col
    wts = [g.w for g in gs]
    wts[5] = bad_w
    with pytest.raises(capi.OimError) as ei:
        capi.oim_create_batch_csr([g.n for g in gs], 2, [g.nnz for g in gs], [g.row_ptr for g in gs], cols, wts,
                                  capi.OIM_FLAG_DEFER_UPLOAD)
    assert ei.value.code == capi.OIM_EINVAL
    assert capi.oim_last_error().startswith("graph 4: ")
    # the symmetry check is the caller's to skip, as in oim_create_problem
    wts[4] = gs[4].w
    h = capi.oim_create_batch_csr([g.n for g in gs], 2, [g.nnz for g in gs], [g.row_ptr for g in gs],
                                  [g.col for g in gs], wts,
                                  capi.OIM_FLAG_DEFER_UPLOAD | capi.OIM_FLAG_SKIP_SYMMETRY_CHECK)
    capi.oim_destroy_problem(h)
    with pytest.raises(capi.OimError) as ei:
        capi.oim_create_batch_csr([], 2, [], [], [], None)
    assert ei.value.code == capi.OIM_EINVAL
    lib = capi.load()
    out = ctypes.c_void_p()
    n = np.array([4], np.int32)
    assert lib.oim_create_batch_csr(1, n.ctypes.data, 2, None, None, None, None, 0, ctypes.byref(out)) == \
        capi.OIM_EINVAL


def test_null_handles_rejected(capi):
    with pytest.raises(capi.OimError) as ei:
        capi.oim_run_sync(None)
    assert ei.value.code == capi.OIM_EINVAL
    with pytest.raises(capi.OimError):
        capi.oim_create_batch([])


def test_library_package_does_not_touch_the_oracle():
    pkg = os.path.join(ROOT, "paper_2505_22631_gb300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h", ".cpp")):
                text = open(os.path.join(dirpath, f)).read()
                assert "import oracle" not in text and "from oracle" not in text, f
                assert "oim_oracle" not in text and "orc_" not in text, f


def test_triangular_schedule_matches_oracle(capi, orc):
    got = capi.oim_schedule_triangular(1000, 2.0, 4)
    ref = orc.triangular(1000, 2.0, 4).astype(np.float32)
    assert np.array_equal(got, ref)
    with pytest.raises(capi.OimError):
        capi.oim_schedule_triangular(10, 1.0, 0)
