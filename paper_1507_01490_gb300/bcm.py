"""Python binding of the C-ABI in ``include/bcm.h`` (ctypes, argument
marshalling only: every step of the computation runs in ``libbcm.so``'s CUDA
kernels).

Functions keep the C names.  Array arguments may be numpy arrays (host
memory) or torch CUDA tensors (device memory, passed by ``data_ptr()``); plain
integers are taken as raw addresses.  A non-OK status raises ``BcmError``
carrying the status and ``bcm_last_error()``.

``BcmGraph`` is a small convenience wrapper over the same calls.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

from . import _build

BCM_OK, BCM_ERR_INVALID, BCM_ERR_NOT_SYMMETRIC, BCM_ERR_OOM, BCM_ERR_CUDA, BCM_ERR_TIMEOUT, \
    BCM_ERR_UNSUPPORTED, BCM_ERR_PENDING = range(8)
STATUS_NAMES = {0: "BCM_OK", 1: "BCM_ERR_INVALID", 2: "BCM_ERR_NOT_SYMMETRIC", 3: "BCM_ERR_OOM",
                4: "BCM_ERR_CUDA", 5: "BCM_ERR_TIMEOUT", 6: "BCM_ERR_UNSUPPORTED", 7: "BCM_ERR_PENDING"}

BCM_OUT_DEVICE = 0x1
BCM_NO_FOOTNOTE = 0x2
BCM_PLAIN = 0x4
BCM_CTA_ONLY = 0x8
BCM_CHECK_SYMMETRIC = 0x10
BCM_GRID_ONLY = 0x20
BCM_NO_PULL = 0x40
BCM_PLAIN_BOUNDS = 0x80
BCM_TRACE = 0x100
BCM_NO_DEFER = 0x200
BCM_NO_PREFILTER = 0x400
BCM_NO_CUT = 0x800
BCM_TRACE_LANES = 0x1000
BCM_ALL_PULL = 0x2000
BCM_SPARSE = 0x4000
BCM_NO_SPARSE = 0x8000

# trace record kinds (bits 60..63 of a record's second word)
TRACE_GRID_LEVEL, TRACE_GRID_WAVE, TRACE_CTA_WAVE, TRACE_LANE_LEVEL, TRACE_LANE_END = 0, 1, 2, 3, 4

# every symbol include/bcm.h declares
EXPORTS = ["bcm_graph_create", "bcm_graph_destroy", "bcm_preprocess", "bcm_scc_bounds", "bcm_topk",
           "bcm_topk_start", "bcm_topk_finish", "bcm_trace", "bcm_graph_trim",
           "bcm_farness_all", "bcm_farness_all_noalloc", "bcm_topk_merge", "bcm_batch_create", "bcm_batch_run",
           "bcm_batch_destroy", "bcm_last_error", "bcm_launch_count", "bcm_workspace_bytes",
           "bcm_topk_threshold", "bcm_topk_offer"]

# id of the padding entries of a shard list (see bcm_topk_offer)
PAD_ID = 0xFFFFFFFF


class bcm_options(ctypes.Structure):
    _fields_ = [("lanes", ctypes.c_uint32), ("grid_lanes", ctypes.c_uint32), ("flags", ctypes.c_uint32),
                ("blocks", ctypes.c_uint32), ("threads", ctypes.c_uint32), ("heavy_words", ctypes.c_uint32),
                ("pull_div", ctypes.c_uint32), ("defer_words", ctypes.c_uint32), ("wait_limit_ns", ctypes.c_uint64),
                ("shard_index", ctypes.c_uint32), ("shard_count", ctypes.c_uint32), ("cta_table", ctypes.c_uint32)]


class bcm_key(ctypes.Structure):
    _fields_ = [("N", ctypes.c_uint64), ("F", ctypes.c_uint64), ("id", ctypes.c_uint32), ("valid", ctypes.c_uint32)]

    def as_tuple(self):
        """(valid, N, F, id)"""
        return (int(self.valid), int(self.N), int(self.F), int(self.id))


class bcm_stats(ctypes.Structure):
    _fields_ = [("m_vis", ctypes.c_uint64), ("visits", ctypes.c_uint64), ("completed", ctypes.c_uint64),
                ("cut", ctypes.c_uint64), ("waves", ctypes.c_uint64), ("levels", ctypes.c_uint64),
                ("max_level", ctypes.c_uint64), ("frontier_words", ctypes.c_uint64),
                ("arc_words", ctypes.c_uint64), ("new_words", ctypes.c_uint64),
                ("cleared_words", ctypes.c_uint64), ("launches", ctypes.c_uint64),
                ("kernel_ms", ctypes.c_double), ("preprocess_ms", ctypes.c_double),
                ("total_ms", ctypes.c_double), ("seed_ms", ctypes.c_double), ("wave_ms", ctypes.c_double),
                ("wave_bytes", ctypes.c_uint64), ("grid_waves", ctypes.c_uint64),
                ("grid_levels", ctypes.c_uint64), ("grid_bytes", ctypes.c_uint64), ("deferred", ctypes.c_uint64),
                ("sparse", ctypes.c_uint64)]

    def as_dict(self) -> dict:
        return {name: getattr(self, name) for name, _ in self._fields_}


class BcmError(RuntimeError):
    def __init__(self, status: int, message: str):
        super().__init__("%s: %s" % (STATUS_NAMES.get(status, status), message))
        self.status = status


_lib = None
LIB_PATH = os.path.join(_build.LIB_DIR, "libbcm.so")


def load():
    """The loaded libbcm.so.  Raises if the CUDA library has not been built:
    there is no other implementation to fall back to."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError("libbcm.so is not built (run __graft_entry__.build() or "
                           "python -m paper_1507_01490_gb300._build)")
    lib = ctypes.CDLL(LIB_PATH)
    vp, u32, u64, i32 = ctypes.c_void_p, ctypes.c_uint32, ctypes.c_uint64, ctypes.c_int
    sig = {
        "bcm_graph_create": (i32, [vp, vp, u32, u64, i32, i32, vp, u32, ctypes.POINTER(vp)]),
        "bcm_graph_destroy": (i32, [vp]),
        "bcm_preprocess": (i32, [vp, vp, vp, vp, i32]),
        "bcm_scc_bounds": (i32, [vp, vp, vp, vp, vp, i32]),
        "bcm_topk": (i32, [vp, u32, ctypes.POINTER(bcm_options), vp, vp, vp, ctypes.POINTER(bcm_stats)]),
        "bcm_topk_start": (i32, [vp, u32, ctypes.POINTER(bcm_options), vp, vp, vp]),
        "bcm_topk_finish": (i32, [vp, i32, ctypes.POINTER(bcm_stats)]),
        "bcm_trace": (i32, [vp, vp, u32, ctypes.POINTER(u32)]),
        "bcm_graph_trim": (i32, [vp]),
        "bcm_farness_all": (i32, [vp, ctypes.POINTER(bcm_options), vp, vp, ctypes.POINTER(bcm_stats)]),
        "bcm_farness_all_noalloc": (i32, [vp, vp, u32, u64, vp, vp, vp]),
        "bcm_topk_merge": (i32, [vp, vp, vp, u32, u32, vp, vp, vp, ctypes.POINTER(u32)]),
        "bcm_batch_create": (i32, [ctypes.POINTER(vp), u32, ctypes.POINTER(u32), ctypes.POINTER(bcm_options), vp,
                                   ctypes.POINTER(vp), ctypes.POINTER(vp), ctypes.POINTER(vp), ctypes.POINTER(vp)]),
        "bcm_batch_run": (i32, [vp, i32]),
        "bcm_batch_destroy": (i32, [vp]),
        "bcm_last_error": (ctypes.c_char_p, []),
        "bcm_launch_count": (u64, []),
        "bcm_workspace_bytes": (u64, [vp, ctypes.POINTER(bcm_options)]),
        "bcm_topk_threshold": (i32, [vp, ctypes.POINTER(bcm_key)]),
        "bcm_topk_offer": (i32, [vp, ctypes.POINTER(bcm_key)]),
    }
    for name, (res, args) in sig.items():
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args
    _lib = lib
    return lib


def _ptr(a):
    if a is None:
        return None
    if isinstance(a, int):
        return a
    if isinstance(a, np.ndarray):
        if not a.flags["C_CONTIGUOUS"]:
            raise ValueError("arrays must be contiguous")
        return a.ctypes.data
    if hasattr(a, "data_ptr"):
        if not a.is_contiguous():
            raise ValueError("tensors must be contiguous")
        return a.data_ptr()
    raise TypeError("cannot pass %r" % type(a))


def _check(st):
    if st != BCM_OK:
        raise BcmError(st, bcm_last_error())


SHARD_CHUNK = 64


def shard_size(n, index, count):
    """Sources of shard `index` of `count`: the degree order's positions p
    with (p // 64) % count == index (the rule of bcm_options.shard_*)."""
    if count <= 1:
        return n
    rnd = SHARD_CHUNK * count
    rem = n % rnd
    lo = index * SHARD_CHUNK
    return (n // rnd) * SHARD_CHUNK + (min(rem - lo, SHARD_CHUNK) if rem > lo else 0)


def shard_positions(n, index, count):
    """The degree-order positions shard `index` of `count` takes, in order."""
    p = np.arange(n, dtype=np.int64)
    return p if count <= 1 else p[(p // SHARD_CHUNK) % count == index]


def bcm_last_error() -> str:
    return load().bcm_last_error().decode()


def bcm_launch_count() -> int:
    return int(load().bcm_launch_count())


def make_options(lanes=0, flags=0, blocks=0, threads=0, wait_limit_ns=0, grid_lanes=0,
                 heavy_words=0, pull_div=0, defer_words=0, shard_index=0, shard_count=0, cta_table=0) -> bcm_options:
    return bcm_options(lanes, grid_lanes, flags, blocks, threads, heavy_words, pull_div, defer_words, wait_limit_ns,
                       shard_index, shard_count, cta_table)


def bcm_graph_create(row_ptr, col, n, m, directed, ptr_on_device=False, stream=None, flags=0):
    h = ctypes.c_void_p()
    _check(load().bcm_graph_create(_ptr(row_ptr), _ptr(col), n, m, int(bool(directed)),
                                   int(bool(ptr_on_device)), _ptr(stream) if stream is not None else None,
                                   flags, ctypes.byref(h)))
    return h


def bcm_graph_destroy(h):
    _check(load().bcm_graph_destroy(h))


def bcm_preprocess(h, order=None, x_lo=None, x_hi=None, out_on_device=False):
    _check(load().bcm_preprocess(h, _ptr(order), _ptr(x_lo), _ptr(x_hi), int(bool(out_on_device))))


def bcm_scc_bounds(h, comp=None, alpha=None, omega=None, out_on_device=False):
    """Returns n_scc; fills comp/alpha/omega (n uint32 each) when given."""
    n_scc = ctypes.c_uint32(0)
    if out_on_device:   # the count goes to a host variable either way
        _check(load().bcm_scc_bounds(h, _ptr(comp), _ptr(alpha), _ptr(omega), None, 1))
        _check(load().bcm_scc_bounds(h, None, None, None, ctypes.addressof(n_scc), 0))
    else:
        _check(load().bcm_scc_bounds(h, _ptr(comp), _ptr(alpha), _ptr(omega), ctypes.addressof(n_scc), 0))
    return int(n_scc.value)


def bcm_topk(h, k, options, ids, farness, reach, stats=None):
    _check(load().bcm_topk(h, k, ctypes.byref(options) if options is not None else None, _ptr(ids),
                           _ptr(farness), _ptr(reach), ctypes.byref(stats) if stats is not None else None))


def bcm_topk_start(h, k, options, ids, farness, reach):
    _check(load().bcm_topk_start(h, k, ctypes.byref(options) if options is not None else None, _ptr(ids),
                                 _ptr(farness), _ptr(reach)))


def bcm_topk_finish(h, wait=True, stats=None) -> bool:
    """True once the run has finished (its errors raise); False while it is
    still going (only with wait=False)."""
    st = load().bcm_topk_finish(h, int(bool(wait)), ctypes.byref(stats) if stats is not None else None)
    if st == BCM_ERR_PENDING:
        return False
    _check(st)
    return True


def bcm_topk_threshold(h):
    """The pending (or last) run's published k-th key as (valid, N, F, id)."""
    k = bcm_key()
    _check(load().bcm_topk_threshold(h, ctypes.byref(k)))
    return k.as_tuple()


def bcm_topk_offer(h, key):
    """Offer the pending top-k run a key (valid, N, F, id) from another shard."""
    valid, N, F, vid = key
    k = bcm_key(N, F, vid, int(bool(valid)))
    _check(load().bcm_topk_offer(h, ctypes.byref(k)))


def bcm_trace(h, cap=1 << 16):
    """The last traced run's records as a (count, 4) uint64 array, and how
    many records the run wrote."""
    buf = np.zeros((max(cap, 1), 4), np.uint64)
    count = ctypes.c_uint32(0)
    _check(load().bcm_trace(h, _ptr(buf), cap, ctypes.byref(count)))
    return buf[:min(int(count.value), cap)], int(count.value)


def bcm_graph_trim(h):
    _check(load().bcm_graph_trim(h))


def bcm_farness_all(h, options, farness, reach, stats=None):
    _check(load().bcm_farness_all(h, ctypes.byref(options) if options is not None else None, _ptr(farness),
                                  _ptr(reach), ctypes.byref(stats) if stats is not None else None))


def bcm_farness_all_noalloc(row_ptr, col, n, m, stream, farness, reach):
    """f(v), r(v) of every vertex without any allocation by the library (all
    pointers device memory; see include/bcm.h for the limits)."""
    _check(load().bcm_farness_all_noalloc(_ptr(row_ptr), _ptr(col), n, m,
                                          _ptr(stream) if stream is not None else None, _ptr(farness),
                                          _ptr(reach)))


def bcm_topk_merge(ids, farness, reach, k):
    """The best min(k, len(ids)) entries of the given lists (host arrays), best first."""
    ids = np.ascontiguousarray(ids, dtype=np.uint32)
    far = np.ascontiguousarray(farness, dtype=np.uint64)
    rch = np.ascontiguousarray(reach, dtype=np.uint32)
    if not (len(ids) == len(far) == len(rch)):
        raise ValueError("ids, farness and reach must have the same length")
    w = max(min(k, len(ids)), 1)
    oi, of, orr = np.zeros(w, np.uint32), np.zeros(w, np.uint64), np.zeros(w, np.uint32)
    written = ctypes.c_uint32(0)
    _check(load().bcm_topk_merge(_ptr(ids) if len(ids) else None, _ptr(far) if len(ids) else None,
                                 _ptr(rch) if len(ids) else None, len(ids), k, _ptr(oi), _ptr(of), _ptr(orr),
                                 ctypes.byref(written)))
    n = int(written.value)
    return oi[:n], of[:n], orr[:n]


class BcmBatch:
    """bcm_batch_*: the top-k runs of many small graphs recorded as one CUDA
    graph.  `handles` are bcm graph handles (BcmGraph.h), `ks` their k, `outs`
    (ids, farness, reach) device tensors per graph, `stream` a torch CUDA
    stream (not the default one)."""

    def __init__(self, handles, ks, outs, stream, options=None):
        n = len(handles)
        opts = options if options is not None else make_options(flags=BCM_OUT_DEVICE)
        hv = (ctypes.c_void_p * n)(*[h.value if isinstance(h, ctypes.c_void_p) else h for h in handles])
        kv = (ctypes.c_uint32 * n)(*ks)
        iv = (ctypes.c_void_p * n)(*[_ptr(o[0]) for o in outs])
        fv = (ctypes.c_void_p * n)(*[_ptr(o[1]) for o in outs])
        rv = (ctypes.c_void_p * n)(*[_ptr(o[2]) for o in outs])
        self._keep = (outs, stream)
        self.b = ctypes.c_void_p()
        _check(load().bcm_batch_create(hv, n, kv, ctypes.byref(opts), _ptr(stream.cuda_stream), iv, fv, rv,
                                       ctypes.byref(self.b)))

    def run(self, wait=True):
        _check(load().bcm_batch_run(self.b, int(bool(wait))))

    def close(self):
        if getattr(self, "b", None) is not None and self.b.value:
            load().bcm_batch_destroy(self.b)
            self.b = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def bcm_workspace_bytes(h, options=None) -> int:
    return int(load().bcm_workspace_bytes(h, ctypes.byref(options) if options is not None else None))


class BcmGraph:
    """A graph handle: ``BcmGraph(row_ptr, col, n, directed)`` with host numpy
    arrays, or torch CUDA tensors and ``on_device=True``."""

    def __init__(self, row_ptr, col, n, directed, on_device=False, stream=None, flags=0):
        m = int(col.shape[0]) if hasattr(col, "shape") else int(len(col))
        self.n, self.m, self.directed = int(n), m, bool(directed)
        if not on_device:
            row_ptr = np.ascontiguousarray(row_ptr, dtype=np.uint64)
            col = np.ascontiguousarray(col, dtype=np.uint32)
            if col.size == 0:
                col = np.zeros(1, np.uint32)
        self.h = bcm_graph_create(row_ptr, col, self.n, m, directed, on_device, stream, flags)

    @classmethod
    def from_graph(cls, g, **kw):
        return cls(g.row_ptr, g.col, g.n, g.directed, **kw)

    def close(self):
        if getattr(self, "h", None) is not None and self.h.value:
            bcm_graph_destroy(self.h)
            self.h = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def preprocess(self):
        order = np.zeros(max(self.n, 1), np.uint32)
        lo = np.zeros(max(self.n, 1), np.uint32)
        hi = np.zeros(max(self.n, 1), np.uint32)
        bcm_preprocess(self.h, order, lo, hi)
        return order[:self.n], lo[:self.n], hi[:self.n]

    def scc_bounds(self):
        comp = np.zeros(max(self.n, 1), np.uint32)
        al = np.zeros(max(self.n, 1), np.uint32)
        om = np.zeros(max(self.n, 1), np.uint32)
        nc = bcm_scc_bounds(self.h, comp, al, om)
        return comp[:self.n], al[:self.n], om[:self.n], nc

    def topk(self, k, lanes=0, flags=0, blocks=0, threads=0, wait_limit_ns=0, grid_lanes=0, heavy_words=0,
             pull_div=0, defer_words=0, shard_index=0, shard_count=0, cta_table=0):
        kk = max(min(k, self.n), 1)
        ids = np.zeros(kk, np.uint32)
        far = np.zeros(kk, np.uint64)
        reach = np.zeros(kk, np.uint32)
        st = bcm_stats()
        bcm_topk(self.h, k, make_options(lanes, flags, blocks, threads, wait_limit_ns, grid_lanes, heavy_words,
                                         pull_div, defer_words, shard_index, shard_count, cta_table),
                 ids, far, reach, st)
        n_src = shard_size(self.n, shard_index, shard_count) if shard_count > 1 else self.n
        kk = min(k, n_src)
        return ids[:kk], far[:kk], reach[:kk], st.as_dict()

    def trace(self):
        return bcm_trace(self.h)

    def trim(self):
        bcm_graph_trim(self.h)

    def farness_all(self, lanes=0, flags=0, blocks=0, threads=0, wait_limit_ns=0, grid_lanes=0, pull_div=0):
        far = np.zeros(max(self.n, 1), np.uint64)
        reach = np.zeros(max(self.n, 1), np.uint32)
        st = bcm_stats()
        bcm_farness_all(self.h, make_options(lanes, flags, blocks, threads, wait_limit_ns, grid_lanes, 0, pull_div),
                        far, reach, st)
        return far[:self.n], reach[:self.n], st.as_dict()
