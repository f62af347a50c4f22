"""FP64 CPU oracle for the simulated oscillator Ising/Potts machine (arXiv 2505.22631).

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline / reference leg of ``bench.py`` may import this package.  The
library in ``paper_2505_22631_gb300`` never imports it and shares no code with it.

The arithmetic lives in ``oim_oracle.c`` (plain C, double precision, one
function per step of Algorithm 1 / Eq. 5-6); this module only builds it with gcc
and marshals numpy arrays.  Phases are ``[R, n]`` arrays here (replica-major).

Parity status of each function (what pins it is in ``tests/test_oracle_*.py``):
  philox4x32_10        pinned: library Philox4x32-10 (triton's random module, CPU interpreter)
  init / noise draws   pinned: uniformity and normality tests, Box-Muller moments
  derivative, run      pinned: two-oscillator and injection-locking closed forms (first-order
                       convergence in dt), phase-sum conservation, noise variance, Lyapunov
                       descent, gradient of the potential V
  readout, scores      pinned: lattice identities against Eq. 6, hand-countable graphs,
                       brute force
  energy, lyapunov     pinned: closed-form lattice identities, finite differences
  brute force          pinned: cycles, complete and bipartite graphs, Petersen graph
  adjoint              pinned: FP64 central finite differences of the loss
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oim_oracle.c")
_LIB_PATH = os.path.join(_HERE, "liboim_oracle.so")
_lock = threading.Lock()
_lib = None

CFLAGS = ["-O3", "-std=c11", "-fPIC", "-shared", "-fopenmp", "-ffp-contract=off",
          "-fno-fast-math"]


def build(force: bool = False) -> str:
    """Compile ``oim_oracle.c`` into ``liboim_oracle.so`` next to it (gcc, no -march)."""
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    cmd = ["gcc", *CFLAGS, "-o", tmp, _SRC, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


_i32 = ctypes.c_int32
_i64 = ctypes.c_int64
_u32 = ctypes.c_uint32
_u64 = ctypes.c_uint64
_dbl = ctypes.c_double
_vp = ctypes.c_void_p


def _load():
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        lib = ctypes.CDLL(build())
        sig = {
            "orc_philox4x32_10": (None, [_vp, _vp, _vp]),
            "orc_u01": (_dbl, [_u32]),
            "orc_init_phase": (_dbl, [_u64, _u32, _i64, _i64]),
            "orc_noise": (_dbl, [_u64, _u32, _i64, _i64, _i64]),
            "orc_init_phases": (None, [_i32, _i32, _u64, _u32, _vp]),
            "orc_noise_block": (None, [_i32, _i32, _u64, _u32, _i64, _vp]),
            "orc_coupling": (None, [_i32, _vp, _vp, _vp, _vp, _vp]),
            "orc_derivative": (None, [_i32, _i32, _vp, _vp, _vp, _vp, _dbl, _dbl, _vp]),
            "orc_readout_f32": (None, [_i32, _i32, _i32, _vp, _vp]),
            "orc_readout_f64": (None, [_i32, _i32, _i32, _vp, _vp]),
            "orc_scores": (None, [_i32, _i32, _vp, _vp, _vp, _i32, _vp, _vp]),
            "orc_energy": (None, [_i32, _vp, _vp, _vp, _i32, _vp, _vp]),
            "orc_lyapunov": (_dbl, [_i32, _i32, _vp, _vp, _vp, _vp, _dbl, _dbl]),
            "orc_run": (_i32, [_i32, _i32, _vp, _vp, _vp, _vp, _vp, _vp, _dbl, _i64, _i32, _i64,
                               _u64, _u32, _i32, _vp, _i64, _vp, _i32]),
            "orc_bruteforce_maxcut": (_dbl, [_i32, _vp, _vp, _vp, _vp]),
            "orc_bruteforce_min_conflicts": (_dbl, [_i32, _i32, _vp, _vp, _vp, _vp]),
            "orc_triangular": (None, [_i64, _dbl, _i32, _vp]),
            "orc_adjoint": (_i32, [_i32, _i32, _vp, _vp, _vp, _vp, _vp, _vp, _dbl, _i64, _i32,
                                   _u64, _u32, _i32, _vp, _vp, _vp, _vp, _vp, _i32]),
        }
        for name, (res, args) in sig.items():
            fn = getattr(lib, name)
            fn.restype = res
            fn.argtypes = args
        _lib = lib
        return lib


def _p(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


class Graph:
    """Symmetric CSR graph as the oracle consumes it (int64 row_ptr, int32 col, f64 w)."""

    def __init__(self, n, row_ptr, col, w):
        self.n = int(n)
        self.row_ptr = np.ascontiguousarray(row_ptr, dtype=np.int64)
        self.col = np.ascontiguousarray(col, dtype=np.int32)
        if w is None:
            w = np.ones(self.col.shape[0])
        self.w = np.ascontiguousarray(w, dtype=np.float64)

    @classmethod
    def of(cls, g) -> "Graph":
        if isinstance(g, Graph):
            return g
        return cls(g.n, g.row_ptr, g.col, g.w)


# --------------------------------------------------------------------------- RNG
def philox4x32_10(ctr, key) -> np.ndarray:
    c = np.ascontiguousarray(ctr, dtype=np.uint32).reshape(4)
    k = np.ascontiguousarray(key, dtype=np.uint32).reshape(2)
    out = np.zeros(4, dtype=np.uint32)
    _load().orc_philox4x32_10(_p(c), _p(k), _p(out))
    return out


def u01(x: int) -> float:
    return _load().orc_u01(int(x) & 0xFFFFFFFF)


def init_phase(seed: int, graph: int, i: int, r: int) -> float:
    return _load().orc_init_phase(seed, graph, i, r)


def noise(seed: int, graph: int, i: int, t: int, r: int) -> float:
    return _load().orc_noise(seed, graph, i, t, r)


def init_phases(n: int, R: int, seed: int, graph: int = 0) -> np.ndarray:
    out = np.zeros((R, n), dtype=np.float64)
    _load().orc_init_phases(n, R, seed, graph, _p(out))
    return out


def noise_block(n: int, R: int, seed: int, t: int, graph: int = 0) -> np.ndarray:
    out = np.zeros((R, n), dtype=np.float64)
    _load().orc_noise_block(n, R, seed, graph, t, _p(out))
    return out


# ---------------------------------------------------------------------- dynamics
def coupling(g, theta: np.ndarray) -> np.ndarray:
    g = Graph.of(g)
    th = np.ascontiguousarray(theta, dtype=np.float64).reshape(g.n)
    out = np.zeros(g.n)
    _load().orc_coupling(g.n, _p(g.row_ptr), _p(g.col), _p(g.w), _p(th), _p(out))
    return out


def derivative(g, q: int, theta: np.ndarray, K: float, Ks: float) -> np.ndarray:
    g = Graph.of(g)
    th = np.ascontiguousarray(theta, dtype=np.float64).reshape(g.n)
    out = np.zeros(g.n)
    _load().orc_derivative(g.n, q, _p(g.row_ptr), _p(g.col), _p(g.w), _p(th), K, Ks, _p(out))
    return out


def run(g, q: int, K, Ks, Kn, dt: float, T: int, R: int, seed: int, graph: int = 0,
        theta0: np.ndarray | None = None, readout_every: int = 0, nthreads: int = 0,
        replica_offset: int = 0):
    """Simulate replicas replica_offset .. replica_offset+R-1 for T steps.

    Returns (theta[R, n], trace[R, T//readout_every])."""
    g = Graph.of(g)
    K = np.ascontiguousarray(np.broadcast_to(np.asarray(K, dtype=np.float64), (T,)))
    Ks = np.ascontiguousarray(np.broadcast_to(np.asarray(Ks, dtype=np.float64), (T,)))
    Kn = np.ascontiguousarray(np.broadcast_to(np.asarray(Kn, dtype=np.float64), (T,)))
    theta = np.zeros((R, g.n), dtype=np.float64)
    init_given = 0
    if theta0 is not None:
        theta[:] = np.asarray(theta0, dtype=np.float64).reshape(R, g.n)
        init_given = 1
    nro = T // readout_every if readout_every > 0 else 0
    trace = np.zeros((R, max(nro, 1)), dtype=np.float64)
    rc = _load().orc_run(g.n, q, _p(g.row_ptr), _p(g.col), _p(g.w), _p(K), _p(Ks), _p(Kn),
                         float(dt), int(T), int(R), int(replica_offset), int(seed), int(graph),
                         init_given, _p(theta), int(readout_every), _p(trace), int(nthreads))
    if rc != 0:
        raise RuntimeError(f"orc_run failed with {rc}")
    return theta, trace[:, :nro]


def readout_f32(q: int, theta32: np.ndarray) -> np.ndarray:
    th = np.ascontiguousarray(theta32, dtype=np.float32)
    R, n = th.reshape(-1, th.shape[-1]).shape
    out = np.zeros(th.shape, dtype=np.int8)
    _load().orc_readout_f32(n, q, R, _p(th), _p(out))
    return out


def readout_f64(q: int, theta: np.ndarray) -> np.ndarray:
    th = np.ascontiguousarray(theta, dtype=np.float64)
    R, n = th.reshape(-1, th.shape[-1]).shape
    out = np.zeros(th.shape, dtype=np.int8)
    _load().orc_readout_f64(n, q, R, _p(th), _p(out))
    return out


def scores(g, q: int, spins: np.ndarray) -> np.ndarray:
    """Cut (q == 2) or monochromatic-edge weight (q >= 3) of each row of spins[R, n]."""
    g = Graph.of(g)
    s = np.ascontiguousarray(spins, dtype=np.int8).reshape(-1, g.n)
    out = np.zeros(s.shape[0])
    _load().orc_scores(g.n, q, _p(g.row_ptr), _p(g.col), _p(g.w), s.shape[0], _p(s), _p(out))
    return out


def energy(g, theta: np.ndarray) -> np.ndarray:
    g = Graph.of(g)
    th = np.ascontiguousarray(theta, dtype=np.float64).reshape(-1, g.n)
    out = np.zeros(th.shape[0])
    _load().orc_energy(g.n, _p(g.row_ptr), _p(g.col), _p(g.w), th.shape[0], _p(th), _p(out))
    return out


def lyapunov(g, q: int, theta: np.ndarray, K: float, Ks: float) -> float:
    g = Graph.of(g)
    th = np.ascontiguousarray(theta, dtype=np.float64).reshape(g.n)
    return _load().orc_lyapunov(g.n, q, _p(g.row_ptr), _p(g.col), _p(g.w), _p(th), K, Ks)


def bruteforce_maxcut(g):
    g = Graph.of(g)
    best = np.zeros(g.n, dtype=np.int8)
    v = _load().orc_bruteforce_maxcut(g.n, _p(g.row_ptr), _p(g.col), _p(g.w), _p(best))
    return v, best


def bruteforce_min_conflicts(g, q: int):
    g = Graph.of(g)
    best = np.zeros(g.n, dtype=np.int8)
    v = _load().orc_bruteforce_min_conflicts(g.n, q, _p(g.row_ptr), _p(g.col), _p(g.w), _p(best))
    return v, best


def adjoint(g, q: int, K, Ks, Kn, dt: float, T: int, R: int, seed: int, graph: int = 0,
            theta0: np.ndarray | None = None, nthreads: int = 0):
    """Gradient of L = mean_r E(theta_T) w.r.t. the schedules.  Returns (L, dK, dKs, dKn)."""
    g = Graph.of(g)
    K = np.ascontiguousarray(np.broadcast_to(np.asarray(K, dtype=np.float64), (T,)))
    Ks = np.ascontiguousarray(np.broadcast_to(np.asarray(Ks, dtype=np.float64), (T,)))
    Kn = np.ascontiguousarray(np.broadcast_to(np.asarray(Kn, dtype=np.float64), (T,)))
    th0 = np.zeros((R, g.n))
    init_given = 0
    if theta0 is not None:
        th0[:] = np.asarray(theta0, dtype=np.float64).reshape(R, g.n)
        init_given = 1
    dK = np.zeros(max(T, 1)); dKs = np.zeros(max(T, 1)); dKn = np.zeros(max(T, 1))
    loss = np.zeros(1)
    rc = _load().orc_adjoint(g.n, q, _p(g.row_ptr), _p(g.col), _p(g.w), _p(K), _p(Ks), _p(Kn),
                             float(dt), int(T), int(R), int(seed), int(graph), init_given, _p(th0),
                             _p(dK), _p(dKs), _p(dKn), _p(loss), int(nthreads))
    if rc != 0:
        raise RuntimeError(f"orc_adjoint failed with {rc}")
    return float(loss[0]), dK[:T], dKs[:T], dKn[:T]


def triangular(steps: int, ks_max: float, periods: int) -> np.ndarray:
    out = np.zeros(max(steps, 1))
    _load().orc_triangular(int(steps), float(ks_max), int(periods), _p(out))
    return out[:steps]


def accuracy_percent(cut: float, best_known: float) -> float:
    """Solution accuracy as Table 1 reports it: 100 * cut / best-known cut."""
    return 100.0 * float(cut) / float(best_known)
