"""CPU oracle for exact top-k closeness -- TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py``'s CPU-baseline
leg may import this package.  It shares no code with the CUDA library
(``paper_1507_01490_gb300``): it does not import it, and the library does not
import this.  The arithmetic lives in ``oracle.c`` (plain C, built with gcc on
the machine that runs it); this module only marshals numpy arrays.

Every function follows a passage of Borassi, Crescenzi, Marino, "Fast and
Simple Computation of Top-k Closeness Centralities" (arXiv 1507.01490):

* ``farness_all``   Table 1 / Section 1 definitions, one BFS per source.
* ``topk``          the textbook top-k (Section 2.1), ties by smaller id.
* ``scc``, ``alpha_omega``  Section 1.3's SCC DAG, Section 2.3's programme;
  ``alpha_omega_refined``  the same with Section 2.3's biggest-SCC refinement.
* ``bound_trace``   Lemma 1's lower bound f~_d(v, x) along one BFS.
* ``bcm``           Algorithm 1 with BFSCut (Algorithm 2), sequential.
* ``ShardRun``      the same loop over one shard's sources, resumable, with
  an outside k-th key (Section 2: parallel threads share x_k).

All of these are pinned by tests/test_oracle_*.py against closed forms,
brute force and library routines; none is "parity unpinned".
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_DIR = os.path.dirname(os.path.abspath(__file__))
_LIB_DIR = os.path.join(_DIR, "_lib")
_SRC = os.path.join(_DIR, "oracle.c")
_lock = threading.Lock()
_lib = None

GT_TABLE1, GT_FOOTNOTE, GT_ALG2 = 0, 1, 2

_u64p = ctypes.POINTER(ctypes.c_uint64)
_u32p = ctypes.POINTER(ctypes.c_uint32)
_i64p = ctypes.POINTER(ctypes.c_int64)


class _Stats(ctypes.Structure):
    _fields_ = [("m_vis", ctypes.c_uint64), ("completed", ctypes.c_uint64),
                ("cut", ctypes.c_uint64), ("max_level", ctypes.c_uint64)]


def build(force: bool = False) -> str:
    """Compile oracle.c into oracle/_lib/liboracle.so (gcc, host only)."""
    out = os.path.join(_LIB_DIR, "liboracle.so")
    with _lock:
        os.makedirs(_LIB_DIR, exist_ok=True)
        if force or not os.path.exists(out) or os.path.getmtime(_SRC) > os.path.getmtime(out):
            tmp = out + ".tmp%d" % os.getpid()
            res = subprocess.run(["gcc", "-O2", "-std=gnu11", "-fPIC", "-shared", "-pthread",
                                  "-Wall", "-o", tmp, _SRC], stdout=subprocess.PIPE,
                                 stderr=subprocess.STDOUT, text=True)
            if res.returncode != 0:
                raise RuntimeError("oracle build failed:\n" + res.stdout)
            os.replace(tmp, out)
    return out


def _get():
    global _lib
    if _lib is None:
        lib = ctypes.CDLL(build())
        lib.oracle_farness_all.restype = ctypes.c_int
        lib.oracle_farness_all.argtypes = [ctypes.c_uint32, _u64p, _u32p, _u32p, ctypes.c_uint64,
                                           _u64p, _u32p, _u64p, ctypes.c_int]
        lib.oracle_topk.restype = ctypes.c_int
        lib.oracle_topk.argtypes = [ctypes.c_uint32, _u64p, _u32p, ctypes.c_uint32, _u32p]
        lib.oracle_scc.restype = ctypes.c_int64
        lib.oracle_scc.argtypes = [ctypes.c_uint32, _u64p, _u32p, _u32p]
        lib.oracle_alpha_omega.restype = ctypes.c_int64
        lib.oracle_alpha_omega.argtypes = [ctypes.c_uint32, _u64p, _u32p, _u32p, _u32p, _u32p]
        lib.oracle_alpha_omega_refined.restype = ctypes.c_int64
        lib.oracle_alpha_omega_refined.argtypes = [ctypes.c_uint32, _u64p, _u32p, _u32p, _u32p, _u32p]
        lib.oracle_bcm2.restype = ctypes.c_int64
        lib.oracle_bcm2.argtypes = [ctypes.c_uint32, _u64p, _u32p, ctypes.c_int, ctypes.c_uint32,
                                    ctypes.c_int, ctypes.c_int, ctypes.c_int, _u32p, _u64p, _u32p,
                                    ctypes.POINTER(_Stats)]
        lib.oracle_bound_trace.restype = ctypes.c_int64
        lib.oracle_bound_trace.argtypes = [ctypes.c_uint32, _u64p, _u32p, ctypes.c_uint32,
                                           ctypes.c_int, ctypes.c_uint64, _i64p, ctypes.c_uint64]
        lib.oracle_order.restype = None
        lib.oracle_order.argtypes = [ctypes.c_uint32, _u64p, _u32p]
        lib.oracle_bcm_sources.restype = ctypes.c_int64
        lib.oracle_bcm_sources.argtypes = [ctypes.c_uint32, _u64p, _u32p, ctypes.c_int, ctypes.c_uint32,
                                           ctypes.c_int, _u32p, _u32p, _u32p, ctypes.c_uint64, ctypes.c_uint64,
                                           ctypes.c_int, ctypes.c_uint64, ctypes.c_uint64, ctypes.c_uint32,
                                           _u32p, _u64p, _u32p, _u32p, ctypes.POINTER(_Stats)]
        lib.oracle_bcm.restype = ctypes.c_int64
        lib.oracle_bcm.argtypes = [ctypes.c_uint32, _u64p, _u32p, ctypes.c_int, ctypes.c_uint32,
                                   ctypes.c_int, ctypes.c_int, _u32p, _u64p, _u32p,
                                   ctypes.POINTER(_Stats)]
        _lib = lib
    return _lib


def _csr(g):
    rp = np.ascontiguousarray(g.row_ptr, dtype=np.uint64)
    col = np.ascontiguousarray(g.col, dtype=np.uint32)
    if col.size == 0:
        col = np.zeros(1, np.uint32)
    return rp, col


def _p(a, t):
    return a.ctypes.data_as(t)


def default_threads() -> int:
    return max(1, len(os.sched_getaffinity(0)))


def farness_all(g, sources=None, threads=None, arcs=False, info=None):
    """(farness u64, reach u32[, arcs u64]) for every source (all vertices by default).
    info (a dict, optional) receives "threads_used": how many threads took work."""
    rp, col = _csr(g)
    if sources is None:
        src = None
        cnt = g.n
    else:
        src = np.ascontiguousarray(sources, dtype=np.uint32)
        cnt = src.size
    f = np.zeros(max(cnt, 1), np.uint64)
    r = np.zeros(max(cnt, 1), np.uint32)
    a = np.zeros(max(cnt, 1), np.uint64) if arcs else None
    if cnt:
        rc = _get().oracle_farness_all(g.n, _p(rp, _u64p), _p(col, _u32p),
                                       None if src is None else _p(src, _u32p), cnt,
                                       _p(f, _u64p), _p(r, _u32p),
                                       None if a is None else _p(a, _u64p),
                                       threads or default_threads())
        if rc < 0:
            raise MemoryError("oracle_farness_all failed")
        if info is not None:
            info["threads_used"] = int(rc)
    elif info is not None:
        info["threads_used"] = 0
    out = (f[:cnt], r[:cnt])
    return out + (a[:cnt],) if arcs else out


def topk(farness, reach, k):
    """ids of the min(k, n) most central vertices, best first."""
    f = np.ascontiguousarray(farness, dtype=np.uint64)
    r = np.ascontiguousarray(reach, dtype=np.uint32)
    n = f.size
    ids = np.zeros(max(min(k, n), 1), np.uint32)
    if n == 0 or k == 0:
        return ids[:0]
    got = _get().oracle_topk(n, _p(f, _u64p), _p(r, _u32p), k, _p(ids, _u32p))
    if got < 0:
        raise MemoryError("oracle_topk failed")
    return ids[:got]


def topk_exhaustive(g, k, threads=None):
    """(ids, farness, reach) of the exhaustive (textbook) top-k."""
    f, r = farness_all(g, threads=threads)
    ids = topk(f, r, k)
    return ids, f[ids], r[ids]


def scc(g):
    """(comp u32[n], n_scc) -- Tarjan's numbering."""
    rp, col = _csr(g)
    comp = np.zeros(max(g.n, 1), np.uint32)
    nc = _get().oracle_scc(g.n, _p(rp, _u64p), _p(col, _u32p), _p(comp, _u32p))
    if nc < 0:
        raise MemoryError("oracle_scc failed")
    return comp[:g.n], int(nc)


def alpha_omega(g):
    """(comp, alpha, omega, n_scc) per Section 2.3."""
    rp, col = _csr(g)
    comp = np.zeros(max(g.n, 1), np.uint32)
    al = np.zeros(max(g.n, 1), np.uint32)
    om = np.zeros(max(g.n, 1), np.uint32)
    nc = _get().oracle_alpha_omega(g.n, _p(rp, _u64p), _p(col, _u32p), _p(comp, _u32p),
                                   _p(al, _u32p), _p(om, _u32p))
    if nc < 0:
        raise MemoryError("oracle_alpha_omega failed")
    return comp[:g.n], al[:g.n], om[:g.n], int(nc)


def alpha_omega_refined(g):
    """(comp, alpha, omega, n_scc) with Section 2.3's biggest-SCC refinement."""
    rp, col = _csr(g)
    comp = np.zeros(max(g.n, 1), np.uint32)
    al = np.zeros(max(g.n, 1), np.uint32)
    om = np.zeros(max(g.n, 1), np.uint32)
    nc = _get().oracle_alpha_omega_refined(g.n, _p(rp, _u64p), _p(col, _u32p), _p(comp, _u32p),
                                           _p(al, _u32p), _p(om, _u32p))
    if nc < 0:
        raise MemoryError("oracle_alpha_omega_refined failed")
    return comp[:g.n], al[:g.n], om[:g.n], int(nc)


def order(g):
    """Algorithm 1's processing order: degree descending, ids ascending on ties."""
    rp, _ = _csr(g)
    out = np.zeros(max(g.n, 1), np.uint32)
    _get().oracle_order(g.n, _p(rp, _u64p), _p(out, _u32p))
    return out[:g.n]


def bound_trace(g, v, x, mode=GT_TABLE1):
    """Lemma 1's f~_d(v, x) for d = 0 .. ecc(v), as int64."""
    rp, col = _csr(g)
    out = np.zeros(g.n + 2, np.int64)
    k = _get().oracle_bound_trace(g.n, _p(rp, _u64p), _p(col, _u32p), v, mode, x,
                                  _p(out, _i64p), out.size)
    if k < 0:
        raise RuntimeError("oracle_bound_trace failed (%d)" % k)
    return out[:k]


def bcm(g, k, gamma_mode=None, early_test=True, refined=False):
    """Algorithm 1 (sequential).  Returns (ids, farness, reach, stats dict).
    refined: digraph bounds from the biggest-SCC refinement (Section 2.3)."""
    if gamma_mode is None:
        gamma_mode = GT_TABLE1 if g.directed else GT_FOOTNOTE
    rp, col = _csr(g)
    kk = max(min(k, g.n), 1)
    ids = np.zeros(kk, np.uint32)
    f = np.zeros(kk, np.uint64)
    r = np.zeros(kk, np.uint32)
    st = _Stats()
    got = _get().oracle_bcm2(g.n, _p(rp, _u64p), _p(col, _u32p), int(g.directed), k, gamma_mode,
                             int(bool(early_test)), int(bool(refined)), _p(ids, _u32p), _p(f, _u64p),
                             _p(r, _u32p), ctypes.byref(st))
    if got < 0:
        raise MemoryError("oracle_bcm failed")
    stats = {"m_vis": st.m_vis, "completed": st.completed, "cut": st.cut, "max_level": st.max_level}
    return ids[:got], f[:got], r[:got], stats


class ShardRun:
    """Algorithm 1 over one shard of the sources (its part of the processing
    order), run a chunk at a time so that shards can exchange their k-th keys
    in between (Section 2's shared x_k).  bounds: (xa, xb) = (r, r) on
    undirected graphs, (alpha, omega) on digraphs."""

    def __init__(self, g, k, sources, bounds, gamma_mode=None):
        if gamma_mode is None:
            gamma_mode = GT_TABLE1 if g.directed else GT_FOOTNOTE
        self.g, self.k, self.mode = g, k, gamma_mode
        self.rp, self.col = _csr(g)
        self.src = np.ascontiguousarray(sources, dtype=np.uint32)
        if self.src.size == 0:
            self.src = np.zeros(1, np.uint32)[:0]
        self.xa = np.ascontiguousarray(bounds[0], dtype=np.uint32)
        self.xb = np.ascontiguousarray(bounds[1], dtype=np.uint32)
        kk = max(k, 1)
        self.ids = np.zeros(kk, np.uint32)
        self.f = np.zeros(kk, np.uint64)
        self.r = np.zeros(kk, np.uint32)
        self.count = np.zeros(1, np.uint32)
        self.stats = _Stats()
        self.pos = 0
        self.ext = (0, 0, 1, 0)      # (valid, N, F, id)

    @property
    def done(self):
        return self.pos >= len(self.src)

    def offer(self, key):
        """Use key (valid, N, F, id) from now on if it ranks before the one held."""
        valid, N, F, vid = key
        if not valid:
            return
        if self.ext[0]:
            _, N0, F0, i0 = self.ext
            if not (N * F0 > N0 * F or (N * F0 == N0 * F and vid < i0)):
                return
        self.ext = (1, int(N), int(F), int(vid))

    def key(self):
        """This shard's own k-th key (valid, N, F, id); valid = 0 below k entries."""
        c = int(self.count[0])
        if c < self.k:
            return (0, 0, 1, 0)
        f, r, vid = int(self.f[self.k - 1]), int(self.r[self.k - 1]), int(self.ids[self.k - 1])
        return (1, 0, 1, vid) if r <= 1 or f == 0 else (1, (r - 1) ** 2, f, vid)

    def step(self, count):
        """Run the next `count` sources; returns True once all are done."""
        to = min(self.pos + count, len(self.src))
        src = self.src if self.src.size else np.zeros(1, np.uint32)
        got = _get().oracle_bcm_sources(self.g.n, _p(self.rp, _u64p), _p(self.col, _u32p), int(self.g.directed),
                                        self.k, self.mode, _p(self.xa, _u32p), _p(self.xb, _u32p),
                                        _p(src, _u32p), self.pos, to, self.ext[0], self.ext[1], self.ext[2],
                                        self.ext[3], _p(self.ids, _u32p), _p(self.f, _u64p), _p(self.r, _u32p),
                                        _p(self.count, _u32p), ctypes.byref(self.stats))
        if got < 0:
            raise MemoryError("oracle_bcm_sources failed")
        self.pos = to
        return self.done

    def result(self):
        c = int(self.count[0])
        return self.ids[:c].copy(), self.f[:c].copy(), self.r[:c].copy(), {
            "m_vis": self.stats.m_vis, "completed": self.stats.completed, "cut": self.stats.cut}
