"""ctypes binding of liboim's C ABI (include/oim.h), one Python function per entry point.

Argument marshalling only: arrays may be numpy arrays (host memory) or torch
tensors (host or CUDA), passed to the library as plain pointers; every step of
the simulation runs in liboim's CUDA kernels.  Loading fails loudly if the
library has not been built: there is no fallback path.
"""
from __future__ import annotations

import ctypes
import os
import threading

import numpy as np

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "liboim.so")
# the same library built with -DOIM_CHECKS (build(checks=True)): kernels test every
# column index against its row's graph and report OIM_EINDEX instead of reading it
CHECKS_LIB_PATH = os.path.join(_PKG, "liboim_checks.so")

OIM_OK = 0
OIM_EINVAL = -1
OIM_ENOMEM = -2
OIM_ECUDA = -3
OIM_ETIMEOUT = -4
OIM_EUNSUPPORTED = -5
OIM_ESTATE = -6
OIM_EINDEX = -7

OIM_FORM_AUTO = 0
OIM_FORM_STREAM = 1
OIM_FORM_RESIDENT = 2
OIM_FORM_GEMM = 3
OIM_FORM_MIXED = 4
OIM_FORM_PERSISTENT = 5

OIM_PREC_AUTO = 0
OIM_PREC_FP32 = 1
OIM_PREC_BF16 = 2
OIM_PREC_FP16 = 3

OIM_FLAG_SKIP_SYMMETRY_CHECK = 1
OIM_FLAG_DEFER_UPLOAD = 2
OIM_NOALLOC_MAX_ACCUM = 131072

FORMS = {"auto": OIM_FORM_AUTO, "stream": OIM_FORM_STREAM, "resident": OIM_FORM_RESIDENT,
         "gemm": OIM_FORM_GEMM, "mixed": OIM_FORM_MIXED, "persistent": OIM_FORM_PERSISTENT}
PRECISIONS = {"auto": OIM_PREC_AUTO, "fp32": OIM_PREC_FP32, "bf16": OIM_PREC_BF16,
              "fp16": OIM_PREC_FP16}


class OimError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"liboim error {code}: {msg}")
        self.code = code


class oim_run_opts(ctypes.Structure):
    _fields_ = [
        ("form", ctypes.c_int32),
        ("precision", ctypes.c_int32),
        ("readout_every", ctypes.c_int64),
        ("stream", ctypes.c_void_p),
        ("use_graph", ctypes.c_int32),
        ("replicas_per_block", ctypes.c_int32),
        ("threads_per_block", ctypes.c_int32),
        ("checkpoint_every", ctypes.c_int32),
        ("graph_forms", ctypes.c_void_p),
        ("csr_scores", ctypes.c_int32),
        ("reserved", ctypes.c_int32 * 5),
    ]


_i32, _i64, _u32, _u64 = ctypes.c_int32, ctypes.c_int64, ctypes.c_uint32, ctypes.c_uint64
_f32, _vp, _cp = ctypes.c_float, ctypes.c_void_p, ctypes.c_char_p
_pp = ctypes.POINTER(ctypes.c_void_p)

# name -> (restype, argtypes); every entry point declared in include/oim.h
SIGNATURES = {
    "oim_default_opts": (None, [ctypes.POINTER(oim_run_opts)]),
    "oim_version": (_cp, []),
    "oim_last_error": (_cp, []),
    "oim_create_problem": (ctypes.c_int, [_i32, _i32, _i64, _vp, _vp, _vp, _u32, _pp]),
    "oim_create_batch": (ctypes.c_int, [_i32, _vp, _pp]),
    "oim_create_batch_csr": (ctypes.c_int, [_i32, _vp, _i32, _vp, _vp, _vp, _vp, _u32, _pp]),
    "oim_problem_info": (ctypes.c_int, [_vp, _vp, _vp, _vp, _vp]),
    "oim_destroy_problem": (None, [_vp]),
    "oim_run": (ctypes.c_int, [_vp, _vp, _vp, _vp, _f32, _i64, _i32, _u64,
                               ctypes.POINTER(oim_run_opts), _pp]),
    "oim_rerun": (ctypes.c_int, [_vp, _vp, _vp, _vp, _f32, _i64, _u64]),
    "oim_run_sync": (ctypes.c_int, [_vp]),
    "oim_readout": (ctypes.c_int, [_vp, _vp, _vp, _vp, _vp, _vp]),
    "oim_run_info": (ctypes.c_int, [_vp, _vp, _vp, _vp, _vp, _vp]),
    "oim_get_phases": (ctypes.c_int, [_vp, _vp]),
    "oim_debug_derivative": (ctypes.c_int, [_vp, _vp, _i32, _f32, _f32, _vp]),
    "oim_debug_set_column": (ctypes.c_int, [_vp, _i64, _i32, _vp]),
    "oim_backward": (ctypes.c_int, [_vp, _vp, _vp, _vp, _vp]),
    "oim_autotune": (ctypes.c_int, [_vp, _i32, _i32, _i64, _vp, ctypes.POINTER(oim_run_opts),
                                    ctypes.POINTER(ctypes.c_double)]),
    "oim_debug_tc_gemm": (ctypes.c_int, [_vp, _vp, _vp, _i32, _i32, _i32]),
    "oim_debug_tc_gemm_withhold": (ctypes.c_int, [_vp, _vp, _vp, _i32, _i32, _i32, _i32, _u32]),
    "oim_schedule_triangular": (ctypes.c_int, [_vp, _i64, _f32, _i32]),
    "oim_destroy_run": (None, [_vp]),
    "oim_score_phases_noalloc": (ctypes.c_int, [_vp, _vp, _i32, _i32, _vp, _vp]),
}

_lock = threading.Lock()
_lib = None


def load(path: str | None = None):
    """Load liboim.so (built by paper_2505_22631_gb300.build); raise if it is missing."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        p = path or LIB_PATH
        if not os.path.exists(p):
            raise OimError(OIM_EUNSUPPORTED,
                           f"{p} is not built; run paper_2505_22631_gb300.build.build() "
                           "(the library has no CPU fallback)")
        lib = ctypes.CDLL(p)
        for name, (res, args) in SIGNATURES.items():
            fn = getattr(lib, name)
            fn.restype = res
            fn.argtypes = args
        _lib = lib
        return lib


def _check(rc: int):
    if rc != OIM_OK:
        msg = load().oim_last_error().decode(errors="replace")
        raise OimError(rc, msg)


def ptr(x, dtype=None):
    """Raw address of a numpy array or torch tensor (contiguous, of the given dtype)."""
    if x is None:
        return None
    if isinstance(x, np.ndarray):
        if dtype is not None and x.dtype != np.dtype(dtype):
            raise TypeError(f"expected {np.dtype(dtype)}, got {x.dtype}")
        if not x.flags["C_CONTIGUOUS"]:
            raise ValueError("array must be contiguous")
        return x.ctypes.data
    if hasattr(x, "data_ptr"):
        import torch
        if dtype is not None:
            want = {np.dtype(np.float32): torch.float32, np.dtype(np.float64): torch.float64,
                    np.dtype(np.int32): torch.int32, np.dtype(np.int64): torch.int64,
                    np.dtype(np.int8): torch.int8}[np.dtype(dtype)]
            if x.dtype != want:
                raise TypeError(f"expected {want}, got {x.dtype}")
        if not x.is_contiguous():
            raise ValueError("tensor must be contiguous")
        return x.data_ptr()
    raise TypeError(f"unsupported buffer type {type(x)}")


# ----------------------------------------------------------------- entry points
def oim_default_opts() -> oim_run_opts:
    o = oim_run_opts()
    load().oim_default_opts(ctypes.byref(o))
    return o


def oim_version() -> str:
    return load().oim_version().decode()


def oim_last_error() -> str:
    return load().oim_last_error().decode(errors="replace")


def oim_create_problem(n, q, nnz, row_ptr, col_idx, weights=None, flags=0):
    h = ctypes.c_void_p()
    _check(load().oim_create_problem(int(n), int(q), int(nnz), ptr(row_ptr, np.int64),
                                     ptr(col_idx, np.int32), ptr(weights, np.float32), int(flags),
                                     ctypes.byref(h)))
    return h.value


def oim_create_batch(problems):
    arr = (ctypes.c_void_p * len(problems))(*problems)
    h = ctypes.c_void_p()
    _check(load().oim_create_batch(len(problems), ctypes.cast(arr, ctypes.c_void_p),
                                   ctypes.byref(h)))
    return h.value


def oim_create_batch_csr(n, q, nnz, row_ptrs, col_idxs, weights=None, flags=0):
    """A batch straight from per-graph CSR arrays (numpy or torch, host or device):
    n, nnz per graph; weights None or a list with None for all-+1 graphs."""
    count = len(n)
    if not (len(nnz) == len(row_ptrs) == len(col_idxs) == count):
        raise ValueError("per-graph lists differ in length")
    if weights is not None and len(weights) != count:
        raise ValueError("weights must have one entry per graph")
    n_arr = np.ascontiguousarray(n, dtype=np.int32)
    nnz_arr = np.ascontiguousarray(nnz, dtype=np.int64)
    rp = (ctypes.c_void_p * count)(*[ptr(x, np.int64) for x in row_ptrs])
    ci = (ctypes.c_void_p * count)(*[ptr(x, np.int32) for x in col_idxs])
    wp = None if weights is None else (ctypes.c_void_p * count)(*[ptr(x, np.float32) for x in weights])
    h = ctypes.c_void_p()
    _check(load().oim_create_batch_csr(count, n_arr.ctypes.data, int(q), nnz_arr.ctypes.data,
                                       ctypes.cast(rp, ctypes.c_void_p), ctypes.cast(ci, ctypes.c_void_p),
                                       None if wp is None else ctypes.cast(wp, ctypes.c_void_p), int(flags),
                                       ctypes.byref(h)))
    return h.value


def oim_problem_info(p):
    g, q = _i32(), _i32()
    nodes, nnz = _i64(), _i64()
    _check(load().oim_problem_info(p, ctypes.byref(g), ctypes.byref(nodes), ctypes.byref(nnz),
                                   ctypes.byref(q)))
    return g.value, nodes.value, nnz.value, q.value


def oim_destroy_problem(p):
    if p:
        load().oim_destroy_problem(p)


def oim_run(p, K, Ks, Kn, dt, steps, replicas, seed, opts: oim_run_opts | None = None):
    h = ctypes.c_void_p()
    o = opts if opts is not None else oim_default_opts()
    _check(load().oim_run(p, ptr(K, np.float32), ptr(Ks, np.float32), ptr(Kn, np.float32),
                          float(dt), int(steps), int(replicas), int(seed) & (2**64 - 1),
                          ctypes.byref(o), ctypes.byref(h)))
    return h.value


def oim_rerun(r, K, Ks, Kn, dt, steps, seed):
    _check(load().oim_rerun(r, ptr(K, np.float32), ptr(Ks, np.float32), ptr(Kn, np.float32),
                            float(dt), int(steps), int(seed) & (2**64 - 1)))


def oim_run_sync(r):
    _check(load().oim_run_sync(r))


def oim_readout(r, spins=None, score=None, best_replica=None, trace=None, energy=None):
    _check(load().oim_readout(r, ptr(spins, np.int8), ptr(score, np.float64),
                              ptr(best_replica, np.int32), ptr(trace, np.float64),
                              ptr(energy, np.float64)))


def oim_run_info(r):
    steps, nro = _i64(), _i64()
    reps, form, prec = _i32(), _i32(), _i32()
    _check(load().oim_run_info(r, ctypes.byref(steps), ctypes.byref(reps), ctypes.byref(nro),
                               ctypes.byref(form), ctypes.byref(prec)))
    return steps.value, reps.value, nro.value, form.value, prec.value


def oim_get_phases(r, theta):
    _check(load().oim_get_phases(r, ptr(theta, np.float32)))


def oim_debug_derivative(p, theta, replicas, K, Ks, f_out):
    _check(load().oim_debug_derivative(p, ptr(theta, np.float32), int(replicas), float(K),
                                       float(Ks), ptr(f_out, np.float32)))


def oim_debug_set_column(p, entry, column) -> int:
    """Overwrite a device column index (index-check tests); returns the previous one."""
    prev = ctypes.c_int32(0)
    _check(load().oim_debug_set_column(p, int(entry), int(column), ctypes.byref(prev)))
    return int(prev.value)


def oim_backward(r, dK=None, dKs=None, dKn=None, loss=None):
    _check(load().oim_backward(r, ptr(dK, np.float64), ptr(dKs, np.float64), ptr(dKn, np.float64),
                               ptr(loss, np.float64)))


def oim_debug_tc_gemm(A, B, D, M, N, K):
    """D = A B^T on the tensor cores (A bf16 [M,K], B bf16 [N,K], D float32 [M,N]; device)."""
    _check(load().oim_debug_tc_gemm(A.data_ptr(), B.data_ptr(), ptr(D, np.float32), int(M), int(N), int(K)))


def oim_debug_tc_gemm_withhold(A, B, D, M, N, K, withhold_k_block, wait_polls):
    """The tensor-core self-test with K block `withhold_k_block` never loaded and every
    pipeline wait limited to `wait_polls` polls (raises OimError OIM_ETIMEOUT when a
    wait gives up)."""
    _check(load().oim_debug_tc_gemm_withhold(A.data_ptr(), B.data_ptr(), ptr(D, np.float32), int(M),
                                             int(N), int(K), int(withhold_k_block), int(wait_polls)))


def oim_autotune(p, replicas, precision_policy=OIM_PREC_AUTO, probe_steps=100, stream=None):
    """Fastest launch configuration for p (by short probe runs); returns (opts, us_per_step)."""
    o = oim_run_opts()
    us = ctypes.c_double()
    _check(load().oim_autotune(p, int(replicas), int(precision_policy), int(probe_steps), stream,
                               ctypes.byref(o), ctypes.byref(us)))
    return o, us.value


def graph_forms_of(opts, graphs):
    """The per-graph forms an oim_run_opts carries (OIM_FORM_MIXED), else None."""
    if opts.form != OIM_FORM_MIXED or not opts.graph_forms:
        return None
    arr = ctypes.cast(opts.graph_forms, ctypes.POINTER(ctypes.c_int32))
    return [int(arr[g]) for g in range(graphs)]


def oim_schedule_triangular(steps, ks_max, periods):
    out = np.zeros(max(int(steps), 1), dtype=np.float32)
    _check(load().oim_schedule_triangular(ptr(out, np.float32), int(steps), float(ks_max), int(periods)))
    return out[:int(steps)]


def oim_destroy_run(r):
    if r:
        load().oim_destroy_run(r)


def oim_score_phases_noalloc(p, theta, replicas, ld, score, stream=None):
    """Scores of caller-supplied device phases [nodes][ld]; allocates no device memory."""
    _check(load().oim_score_phases_noalloc(p, ptr(theta, np.float32), int(replicas), int(ld),
                                           ptr(score, np.float64), stream))
