"""Seeded synthetic graphs in CSR form (row_ptr uint64[n+1], col uint32[m]).

This module builds inputs only and holds none of the method's arithmetic: the
CUDA library and the CPU oracle both consume what it returns.  The large
recipes run in ``gen/graphgen.c`` (integer PRNG, reproducible across x86-64 and
AArch64); small closed-form families are written with numpy.

Workload recipes (the paper's SNAP/LAW/IMDB graphs are not available, so these
synthetic graphs of the same kinds stand in for them):

* ``ba(2000, 3, seed=1)``                 Barabasi-Albert, 5,994 edges, connected.
* ``chung_lu(2**20, 10.0, 2.3, seed=2)``  power-law expected-degree graph, ~5M edges.
* ``rmat(20, 16, seed=3)``                directed R-MAT (0.57, 0.19, 0.19, 0.05).
* ``grid_lcc(2048, 2048, 0.05, seed=4)``  damaged grid, largest component kept.
"""
from __future__ import annotations

import ctypes
import hashlib
from dataclasses import dataclass, field

import numpy as np

from . import _build

_u32p = ctypes.POINTER(ctypes.c_uint32)
_gen = None


def _lib():
    global _gen
    if _gen is None:
        lib = ctypes.CDLL(_build.build_gen())
        lib.gen_ba.restype = ctypes.c_int64
        lib.gen_ba.argtypes = [ctypes.c_uint32, ctypes.c_uint32, ctypes.c_uint64, _u32p, _u32p]
        lib.gen_chung_lu.restype = ctypes.c_int64
        lib.gen_chung_lu.argtypes = [ctypes.c_uint32, ctypes.c_double, ctypes.c_double,
                                     ctypes.c_uint64, ctypes.c_uint64, _u32p, _u32p]
        lib.gen_rmat.restype = ctypes.c_int64
        lib.gen_rmat.argtypes = [ctypes.c_uint32, ctypes.c_uint64, ctypes.c_uint32, ctypes.c_uint32,
                                 ctypes.c_uint32, ctypes.c_uint64, _u32p, _u32p]
        lib.gen_grid_lcc.restype = ctypes.c_int64
        lib.gen_grid_lcc.argtypes = [ctypes.c_uint32, ctypes.c_uint32, ctypes.c_uint64,
                                     ctypes.c_uint64, _u32p, _u32p, _u32p]
        lib.gen_gnp.restype = ctypes.c_int64
        lib.gen_gnp.argtypes = [ctypes.c_uint32, ctypes.c_uint32, ctypes.c_int, ctypes.c_uint64,
                                ctypes.c_uint64, _u32p, _u32p]
        lib.gen_uniform_u32.restype = None
        lib.gen_uniform_u32.argtypes = [ctypes.c_uint64, ctypes.c_uint64, ctypes.c_uint32, _u32p]
        lib.gen_csr.restype = ctypes.c_int64
        lib.gen_csr.argtypes = [ctypes.c_uint32, _u32p, _u32p, ctypes.c_uint64, ctypes.c_int, ctypes.c_int,
                                ctypes.c_int, ctypes.POINTER(ctypes.c_uint64), _u32p]
        lib.gen_exponential.restype = None
        lib.gen_exponential.argtypes = [ctypes.c_uint64, ctypes.c_uint64, ctypes.c_double,
                                        ctypes.POINTER(ctypes.c_double)]
        _gen = lib
    return _gen


def _p32(a: np.ndarray):
    return a.ctypes.data_as(_u32p)


@dataclass
class Graph:
    """A graph in CSR form.  Undirected graphs store both arcs of every edge."""
    n: int
    row_ptr: np.ndarray          # uint64[n+1]
    col: np.ndarray              # uint32[m]
    directed: bool
    name: str = ""
    meta: dict = field(default_factory=dict)

    @property
    def m(self) -> int:
        return int(self.col.shape[0])

    def degrees(self) -> np.ndarray:
        return np.diff(self.row_ptr).astype(np.int64)

    def hash64(self) -> str:
        h = hashlib.sha256()
        h.update(np.array([self.n, int(self.directed)], dtype=np.uint64).tobytes())
        h.update(np.ascontiguousarray(self.row_ptr).tobytes())
        h.update(np.ascontiguousarray(self.col).tobytes())
        return h.hexdigest()[:16]

    def reverse(self) -> "Graph":
        """The transposed graph (in-arcs become out-arcs)."""
        src = np.repeat(np.arange(self.n, dtype=np.uint32), np.diff(self.row_ptr).astype(np.int64))
        return csr_from_arcs(self.n, self.col, src, directed=True, name=self.name + "^T",
                             dedup=False, drop_self_loops=False)


def csr_from_arcs(n: int, src, dst, directed: bool, name: str = "", dedup: bool = True,
                  drop_self_loops: bool = True) -> Graph:
    """CSR from an arc list.  Undirected: each pair is stored in both directions.
    Rows come out sorted; duplicates and self-loops are dropped unless asked not to."""
    src = np.ascontiguousarray(src, dtype=np.uint32)
    dst = np.ascontiguousarray(dst, dtype=np.uint32)
    k = int(src.shape[0])
    row_ptr = np.zeros(n + 1, dtype=np.uint64)
    col = np.empty(max(k * (1 if directed else 2), 1), dtype=np.uint32)
    m = _lib().gen_csr(n, _p32(src), _p32(dst), k, int(not directed), int(drop_self_loops), int(dedup),
                       row_ptr.ctypes.data_as(ctypes.POINTER(ctypes.c_uint64)), _p32(col))
    if m < 0:
        raise ValueError("gen_csr failed: an endpoint is >= n or memory ran out")
    return Graph(n=n, row_ptr=row_ptr, col=col[:m].copy(), directed=directed, name=name)


# --------------------------------------------------------------- large recipes

def ba(n: int, m: int, seed: int) -> Graph:
    m0 = m + 1
    ne = m0 * (m0 - 1) // 2 + m * (n - m0)
    src = np.empty(ne, np.uint32)
    dst = np.empty(ne, np.uint32)
    k = _lib().gen_ba(n, m, seed, _p32(src), _p32(dst))
    if k != ne:
        raise ValueError("gen_ba failed (%d)" % k)
    return csr_from_arcs(n, src, dst, directed=False, name="ba_n%d_m%d_s%d" % (n, m, seed))


def chung_lu(n: int, mean_deg: float, gamma: float, seed: int) -> Graph:
    n_draw = int(round(n * mean_deg / 2))
    src = np.empty(n_draw, np.uint32)
    dst = np.empty(n_draw, np.uint32)
    k = _lib().gen_chung_lu(n, float(mean_deg), float(gamma), n_draw, seed, _p32(src), _p32(dst))
    if k != n_draw:
        raise ValueError("gen_chung_lu failed (%d)" % k)
    return csr_from_arcs(n, src, dst, directed=False,
                         name="chunglu_n%d_d%g_g%g_s%d" % (n, mean_deg, gamma, seed))


def rmat(scale: int, edge_factor: int, seed: int, a=0.57, b=0.19, c=0.19) -> Graph:
    n = 1 << scale
    n_arcs = edge_factor * n
    two32 = float(1 << 32)
    ta = int(round(a * two32))
    tab = ta + int(round(b * two32))
    tabc = tab + int(round(c * two32))
    src = np.empty(n_arcs, np.uint32)
    dst = np.empty(n_arcs, np.uint32)
    k = _lib().gen_rmat(scale, n_arcs, ta, tab, min(tabc, (1 << 32) - 1), seed, _p32(src), _p32(dst))
    if k != n_arcs:
        raise ValueError("gen_rmat failed (%d)" % k)
    return csr_from_arcs(n, src, dst, directed=True, name="rmat_s%d_e%d_s%d" % (scale, edge_factor, seed))


def grid_lcc(rows: int, cols: int, delete_frac: float, seed: int) -> Graph:
    ne = rows * (cols - 1) + (rows - 1) * cols
    n_del = int(round(delete_frac * ne))
    src = np.empty(max(ne - n_del, 1), np.uint32)
    dst = np.empty(max(ne - n_del, 1), np.uint32)
    nout = ctypes.c_uint32(0)
    k = _lib().gen_grid_lcc(rows, cols, n_del, seed, _p32(src), _p32(dst), ctypes.byref(nout))
    if k < 0:
        raise ValueError("gen_grid_lcc failed (%d)" % k)
    g = csr_from_arcs(nout.value, src[:k], dst[:k], directed=False,
                      name="gridlcc_%dx%d_del%g_s%d" % (rows, cols, delete_frac, seed))
    g.meta["deleted_edges"] = n_del
    return g


def gnp(n: int, p: float, seed: int, directed: bool) -> Graph:
    cap = n * n + 1
    src = np.empty(cap, np.uint32)
    dst = np.empty(cap, np.uint32)
    k = _lib().gen_gnp(n, min(int(p * 2**32), 2**32 - 1), int(directed), seed, cap, _p32(src), _p32(dst))
    if k < 0:
        raise ValueError("gen_gnp failed (%d)" % k)
    return csr_from_arcs(n, src[:k], dst[:k], directed=directed, name="gnp_n%d_p%g_s%d" % (n, p, seed))


def uniform_u32(seed: int, count: int, bound: int) -> np.ndarray:
    out = np.empty(count, np.uint32)
    if count:
        _lib().gen_uniform_u32(seed, count, bound, _p32(out))
    return out


def exponential(seed: int, count: int, mean: float) -> np.ndarray:
    out = np.empty(count, np.float64)
    if count:
        _lib().gen_exponential(seed, count, mean, out.ctypes.data_as(ctypes.POINTER(ctypes.c_double)))
    return out


# ------------------------------------------------------------- small families

def _edges(n, pairs, directed, name):
    pairs = np.asarray(pairs, dtype=np.int64).reshape(-1, 2)
    return csr_from_arcs(n, pairs[:, 0], pairs[:, 1], directed=directed, name=name)


def path(n: int) -> Graph:
    return _edges(n, [(i, i + 1) for i in range(n - 1)], False, "path%d" % n)


def star(n: int) -> Graph:
    """Centre 0 joined to leaves 1..n-1."""
    return _edges(n, [(0, i) for i in range(1, n)], False, "star%d" % n)


def cycle(n: int) -> Graph:
    return _edges(n, [(i, (i + 1) % n) for i in range(n)], False, "cycle%d" % n)


def complete(n: int) -> Graph:
    return _edges(n, [(i, j) for i in range(n) for j in range(i + 1, n)], False, "complete%d" % n)


def grid(a: int, b: int) -> Graph:
    """a x b 4-neighbour grid, vertex (i, j) has id i*b + j."""
    pairs = [(i * b + j, i * b + j + 1) for i in range(a) for j in range(b - 1)]
    pairs += [(i * b + j, (i + 1) * b + j) for i in range(a - 1) for j in range(b)]
    return _edges(a * b, pairs, False, "grid%dx%d" % (a, b))


def dpath(n: int) -> Graph:
    """Directed path 0 -> 1 -> ... -> n-1."""
    return _edges(n, [(i, i + 1) for i in range(n - 1)], True, "dpath%d" % n)


def dcycle(n: int) -> Graph:
    return _edges(n, [(i, (i + 1) % n) for i in range(n)], True, "dcycle%d" % n)


def empty(n: int, directed: bool = False) -> Graph:
    return Graph(n=n, row_ptr=np.zeros(n + 1, np.uint64), col=np.zeros(0, np.uint32),
                 directed=directed, name="empty%d" % n)


def disjoint_union(*gs: Graph) -> Graph:
    """Vertex sets placed one after the other, in argument order."""
    assert len({g.directed for g in gs}) == 1
    off = 0
    src, dst = [], []
    for g in gs:
        src.append(np.repeat(np.arange(g.n, dtype=np.int64), g.degrees()) + off)
        dst.append(g.col.astype(np.int64) + off)
        off += g.n
    out = csr_from_arcs(off, np.concatenate(src), np.concatenate(dst), directed=True,
                        name="+".join(g.name for g in gs), dedup=False, drop_self_loops=False)
    out.directed = gs[0].directed
    return out


def relabel(g: Graph, seed: int) -> Graph:
    """The same graph with vertex ids permuted by a seeded shuffle."""
    rng = np.random.default_rng(seed)
    perm = rng.permutation(g.n).astype(np.int64)
    src = perm[np.repeat(np.arange(g.n, dtype=np.int64), g.degrees())]
    dst = perm[g.col.astype(np.int64)]
    out = csr_from_arcs(g.n, src, dst, directed=True, name=g.name + "~r%d" % seed)
    out.directed = g.directed
    return out


def with_self_loops_and_repeats(g: Graph, seed: int, frac: float = 0.1) -> Graph:
    """Adds self-loops and repeated arcs (neither changes a distance).  For an
    undirected graph every repeated arc is added in both directions."""
    rng = np.random.default_rng(seed)
    src = np.repeat(np.arange(g.n, dtype=np.int64), g.degrees())
    dst = g.col.astype(np.int64)
    k = max(1, int(frac * g.n))
    loops = rng.integers(0, g.n, k)
    rep = rng.integers(0, g.m, k) if g.m else np.zeros(0, np.int64)
    s = [src, loops, src[rep]]
    d = [dst, loops, dst[rep]]
    if not g.directed:
        s.append(dst[rep])
        d.append(src[rep])
    out = csr_from_arcs(g.n, np.concatenate(s), np.concatenate(d), directed=True,
                        name=g.name + "+loops", dedup=False, drop_self_loops=False)
    out.directed = g.directed
    return out


# ----------------------------------------------------------- named workloads

def workload(name: str) -> Graph:
    """The named synthetic workloads (sizes in the module docstring)."""
    if name == "ba2000":
        return ba(2000, 3, seed=1)
    if name == "chunglu1m":
        return chung_lu(1 << 20, 10.0, 2.3, seed=2)
    if name == "chunglu256k":      # the same recipe at n = 2^18 (profiling-size case)
        return chung_lu(1 << 18, 10.0, 2.3, seed=2)
    if name == "rmat20":
        return rmat(20, 16, seed=3)
    if name == "rmat18":           # the same recipe at scale 18 (profiling-size case)
        return rmat(18, 16, seed=3)
    if name == "grid2048":
        return grid_lcc(2048, 2048, 0.05, seed=4)
    if name == "grid1024":         # the same recipe at 1024 x 1024, 512 x 512 and 256 x 256 (smaller cases)
        return grid_lcc(1024, 1024, 0.05, seed=4)
    if name == "grid512":
        return grid_lcc(512, 512, 0.05, seed=4)
    if name == "grid256":
        return grid_lcc(256, 256, 0.05, seed=4)
    raise KeyError(name)
