"""Seeded graph generators producing symmetric CSR (no self loops, sorted columns)."""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np


@dataclass
class CSRGraph:
    """Undirected weighted graph stored as a symmetric CSR matrix.

    ``row_ptr`` is int64[n+1], ``col`` int32[nnz] (sorted within each row), ``w``
    float32[nnz].  Every undirected edge {i, j} appears twice (i->j and j->i)
    with the same weight; nnz counts directed entries.
    """
    n: int
    row_ptr: np.ndarray
    col: np.ndarray
    w: np.ndarray
    name: str = ""

    @property
    def nnz(self) -> int:
        return int(self.col.shape[0])

    @property
    def num_edges(self) -> int:
        return self.nnz // 2

    @property
    def mean_degree(self) -> float:
        return self.nnz / max(self.n, 1)

    def degrees(self) -> np.ndarray:
        return np.diff(self.row_ptr)

    def edges(self):
        """Upper-triangle edge list (i < j) with weights."""
        rows = np.repeat(np.arange(self.n, dtype=np.int64), self.degrees())
        m = self.col > rows
        return rows[m], self.col[m].astype(np.int64), self.w[m]

    def dense(self) -> np.ndarray:
        a = np.zeros((self.n, self.n), dtype=np.float64)
        rows = np.repeat(np.arange(self.n), self.degrees())
        a[rows, self.col] = self.w
        return a

    def total_weight(self) -> float:
        return float(np.sum(self.w.astype(np.float64))) / 2.0


def csr_from_edges(n: int, i: np.ndarray, j: np.ndarray, w: np.ndarray | None = None,
                   name: str = "") -> CSRGraph:
    """Build a symmetric CSR from an undirected edge list (duplicates and loops rejected)."""
    i = np.asarray(i, dtype=np.int64)
    j = np.asarray(j, dtype=np.int64)
    if w is None:
        w = np.ones(i.shape[0], dtype=np.float32)
    w = np.asarray(w, dtype=np.float32)
    if np.any(i == j):
        raise ValueError("self loops are not allowed")
    lo, hi = np.minimum(i, j), np.maximum(i, j)
    key = lo * n + hi
    if np.unique(key).shape[0] != key.shape[0]:
        raise ValueError("duplicate edges")
    src = np.concatenate([lo, hi])
    dst = np.concatenate([hi, lo])
    ww = np.concatenate([w, w])
    order = np.lexsort((dst, src))
    src, dst, ww = src[order], dst[order], ww[order]
    counts = np.bincount(src, minlength=n)
    row_ptr = np.zeros(n + 1, dtype=np.int64)
    np.cumsum(counts, out=row_ptr[1:])
    return CSRGraph(n, row_ptr, dst.astype(np.int32), ww.astype(np.float32), name)


def _weights(rng: np.random.Generator, m: int, kind: str) -> np.ndarray:
    if kind == "+1":
        return np.ones(m, dtype=np.float32)
    if kind == "pm1":
        return np.where(rng.random(m) < 0.5, -1.0, 1.0).astype(np.float32)
    raise ValueError(kind)


def erdos_renyi(n: int, p: float, seed: int, weights: str = "+1") -> CSRGraph:
    """G(n, p): each of the n(n-1)/2 pairs is an edge independently with probability p."""
    rng = np.random.default_rng(seed)
    ii, jj = [], []
    block = 1024
    for a in range(0, n, block):
        rows = np.arange(a, min(a + block, n))
        u = rng.random((rows.shape[0], n))
        mask = (u < p) & (np.arange(n)[None, :] > rows[:, None])
        r, c = np.nonzero(mask)
        ii.append(rows[r])
        jj.append(c)
    i = np.concatenate(ii)
    j = np.concatenate(jj)
    return csr_from_edges(n, i, j, _weights(rng, i.shape[0], weights), f"er{n}_p{p}")


def gnm(n: int, m: int, seed: int, weights: str = "+1") -> CSRGraph:
    """G(n, m): m distinct pairs drawn uniformly at random."""
    rng = np.random.default_rng(seed)
    total = n * (n - 1) // 2
    if m > total:
        raise ValueError("too many edges")
    keys = np.zeros(0, dtype=np.int64)
    while keys.shape[0] < m:
        a = rng.integers(0, n, size=2 * (m - keys.shape[0]) + 16)
        b = rng.integers(0, n, size=a.shape[0])
        ok = a != b
        lo, hi = np.minimum(a[ok], b[ok]), np.maximum(a[ok], b[ok])
        keys = np.unique(np.concatenate([keys, lo * n + hi]))
    keys = rng.permutation(keys)[:m]
    i, j = keys // n, keys % n
    return csr_from_edges(n, i, j, _weights(rng, m, weights), f"gnm{n}_m{m}")


def torus(rows: int, cols: int, seed: int, weights: str = "pm1") -> CSRGraph:
    """2D toroidal grid (right and down neighbours with wrap-around), degree 4."""
    rng = np.random.default_rng(seed)
    idx = np.arange(rows * cols).reshape(rows, cols)
    right = np.roll(idx, -1, axis=1)
    down = np.roll(idx, -1, axis=0)
    i = np.concatenate([idx.ravel(), idx.ravel()])
    j = np.concatenate([right.ravel(), down.ravel()])
    return csr_from_edges(rows * cols, i, j, _weights(rng, i.shape[0], weights),
                          f"torus{rows}x{cols}")


def planted_partition(n: int, q: int, avg_degree: float, seed: int) -> CSRGraph:
    """Graph with a planted proper q-colouring: balanced random classes, and
    m = round(n * avg_degree / 2) distinct edges drawn uniformly among pairs whose
    endpoints lie in different classes.  Unit weights."""
    rng = np.random.default_rng(seed)
    perm = rng.permutation(n)
    cls = np.empty(n, dtype=np.int64)
    for c in range(q):
        cls[perm[c::q]] = c
    m = int(round(n * avg_degree / 2))
    keys = np.zeros(0, dtype=np.int64)
    while keys.shape[0] < m:
        a = rng.integers(0, n, size=4 * (m - keys.shape[0]) + 16)
        b = rng.integers(0, n, size=a.shape[0])
        ok = cls[a] != cls[b]
        lo, hi = np.minimum(a[ok], b[ok]), np.maximum(a[ok], b[ok])
        keys = np.unique(np.concatenate([keys, lo * n + hi]))
    keys = rng.permutation(keys)[:m]
    g = csr_from_edges(n, keys // n, keys % n, np.ones(m, dtype=np.float32),
                       f"planted{q}_{n}_d{avg_degree}")
    g.planted = cls  # type: ignore[attr-defined]
    return g


def cycle(n: int) -> CSRGraph:
    i = np.arange(n)
    return csr_from_edges(n, i, (i + 1) % n, None, f"cycle{n}")


def complete(n: int) -> CSRGraph:
    i, j = np.triu_indices(n, 1)
    return csr_from_edges(n, i, j, None, f"K{n}")


def sherrington_kirkpatrick(n: int, seed: int) -> CSRGraph:
    """All-to-all couplings w_ij ~ N(0, 1), i.i.d. per pair (real-valued, dense)."""
    rng = np.random.default_rng(seed)
    i, j = np.triu_indices(n, 1)
    w = rng.standard_normal(i.shape[0]).astype(np.float32)
    return csr_from_edges(n, i, j, w, f"sk{n}")


def complete_bipartite(a: int, b: int) -> CSRGraph:
    i, j = np.meshgrid(np.arange(a), a + np.arange(b), indexing="ij")
    return csr_from_edges(a + b, i.ravel(), j.ravel(), None, f"K{a},{b}")


def petersen() -> CSRGraph:
    outer = [(k, (k + 1) % 5) for k in range(5)]
    spokes = [(k, k + 5) for k in range(5)]
    inner = [(5 + k, 5 + (k + 2) % 5) for k in range(5)]
    e = np.array(outer + spokes + inner)
    return csr_from_edges(10, e[:, 0], e[:, 1], None, "petersen")


def from_dense(a: np.ndarray, name: str = "") -> CSRGraph:
    a = np.asarray(a)
    i, j = np.nonzero(np.triu(a, 1))
    return csr_from_edges(a.shape[0], i, j, a[i, j].astype(np.float32), name)
