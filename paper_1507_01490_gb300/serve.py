"""Serving: top-k closeness requests over many device-resident graphs, with
continuous batching.

Graphs are uploaded and preprocessed once (CSR, components or SCC bounds,
degree order all stay in HBM).  Requests (graph, k) arrive over time.  The
scheduler keeps up to ``max_inflight`` runs on the GPU at once, one per
graph (a graph's runs share its workspace), each on its graph's own CUDA
stream, so runs on different graphs overlap on the device.  A request is
admitted as soon as a slot is free, its graph is idle and its workspace
fits in the HBM budget; finished runs free their slot at once, and the
next waiting request takes it while the others keep running.  Waiting
requests are taken in arrival order, except that one whose graph is busy
or whose workspace does not fit yet lets later ones past (so a large
request cannot hold the GPU idle behind it).

The device work per request is ``bcm_topk_start`` / ``bcm_topk_finish`` of
the C-ABI: the scheduler only decides when to start what.  Its logic runs
against a small backend interface, so it is tested on the CPU with a fake
backend.

Workspace accounting: a graph keeps its run workspace after a run (the next
request on it then needs no allocation and no clearing); when an admission
needs room, the workspaces of idle graphs are given back, least recently
used first (``bcm_graph_trim``), before the request is made to wait.
"""
from __future__ import annotations

import math
import time
from collections import OrderedDict, deque
from dataclasses import dataclass, field

import numpy as np


@dataclass
class Request:
    rid: int
    graph: int
    k: int
    arrival: float          # seconds from the start of the run


@dataclass
class Result:
    rid: int
    graph: int
    k: int
    arrival: float
    admitted: float
    done: float
    ids: np.ndarray
    farness: np.ndarray
    reach: np.ndarray
    stats: dict = field(default_factory=dict)

    @property
    def latency(self) -> float:
        return self.done - self.arrival

    @property
    def queued(self) -> float:
        return self.admitted - self.arrival


class Backend:
    """What the scheduler needs from the device side.  `held` is the ledger of
    graphs that hold a run workspace (graph -> bytes, least recently used
    first); it belongs to the backend, so it stays true across schedulers."""

    def __init__(self):
        self.held: OrderedDict[int, int] = OrderedDict()

    def footprint(self, gid: int) -> int:          # workspace bytes of a run on graph gid
        raise NotImplementedError

    def start(self, gid: int, k: int) -> None:     # enqueue a run; returns at once
        raise NotImplementedError

    def poll(self, gid: int) -> bool:              # True once the run on gid has finished
        raise NotImplementedError

    def collect(self, gid: int):                   # (ids, farness, reach, stats) of the finished run
        raise NotImplementedError

    def trim(self, gid: int) -> None:              # give back gid's workspace
        raise NotImplementedError


class Scheduler:
    def __init__(self, backend: Backend, max_inflight: int = 16, hbm_budget: int = 96 << 30,
                 clock=time.perf_counter, sleep=time.sleep, idle_sleep: float = 20e-6):
        if max_inflight < 1:
            raise ValueError("max_inflight must be >= 1")
        self.be = backend
        self.max_inflight = max_inflight
        self.budget = int(hbm_budget)
        self.clock = clock
        self.sleep = sleep
        self.idle_sleep = idle_sleep
        self.inflight: dict[int, tuple[Request, float]] = {}   # graph -> (request, admitted)
        self.held = backend.held                                # graph -> workspace bytes it holds (LRU order)
        self.peak_inflight = 0
        self.peak_held = 0
        self.trims = 0

    # bytes held by every graph that has a workspace (busy or idle)
    def held_bytes(self) -> int:
        return sum(self.held.values())

    def _make_room(self, need: int) -> bool:
        """Trims idle graphs (least recently used first) until `need` more
        bytes fit in the budget; False if they cannot."""
        if self.held_bytes() + need <= self.budget:
            return True
        busy = sum(b for g, b in self.held.items() if g in self.inflight)
        if busy + need > self.budget:
            return False
        for g in list(self.held.keys()):
            if self.held_bytes() + need <= self.budget:
                break
            if g in self.inflight:
                continue
            self.be.trim(g)
            self.held.pop(g, None)
            self.trims += 1
        return self.held_bytes() + need <= self.budget

    def _admit(self, req: Request, now: float) -> bool:
        if len(self.inflight) >= self.max_inflight or req.graph in self.inflight:
            return False
        need = 0 if req.graph in self.held else self.be.footprint(req.graph)
        if need > self.budget:
            raise ValueError("request %d: graph %d needs %d workspace bytes, above the budget of %d"
                             % (req.rid, req.graph, need, self.budget))
        if not self._make_room(need):
            return False
        self.be.start(req.graph, req.k)
        self.inflight[req.graph] = (req, now)
        self.held[req.graph] = self.held.get(req.graph, 0) + need
        self.held.move_to_end(req.graph)
        self.peak_inflight = max(self.peak_inflight, len(self.inflight))
        self.peak_held = max(self.peak_held, self.held_bytes())
        return True

    def run(self, requests: list[Request]) -> list[Result]:
        """Serves every request (arrival times relative to the call) and
        returns the results in request-id order."""
        pending = deque(sorted(requests, key=lambda r: (r.arrival, r.rid)))
        waiting: list[Request] = []
        results: dict[int, Result] = {}
        t0 = self.clock()
        total = len(requests)
        while len(results) < total:
            now = self.clock() - t0
            while pending and pending[0].arrival <= now:
                waiting.append(pending.popleft())
            progressed = False
            # completions first: they free slots and memory
            for gid in list(self.inflight.keys()):
                if self.be.poll(gid):
                    req, adm = self.inflight.pop(gid)
                    ids, far, reach, st = self.be.collect(gid)
                    results[req.rid] = Result(req.rid, req.graph, req.k, req.arrival, adm,
                                              self.clock() - t0, ids, far, reach, st)
                    progressed = True
            if waiting:
                now = self.clock() - t0
                keep = []
                for req in waiting:
                    if self._admit(req, now):
                        progressed = True
                    else:
                        keep.append(req)
                waiting = keep
            if not progressed:
                if not self.inflight and not waiting and pending:
                    # idle until the next arrival
                    delay = pending[0].arrival - (self.clock() - t0)
                    if delay > 0:
                        self.sleep(min(delay, 0.05))
                elif self.idle_sleep:
                    self.sleep(self.idle_sleep)
        return [results[r.rid] for r in sorted(requests, key=lambda r: r.rid)]


def summarize(results: list[Result], makespan: float | None = None) -> dict:
    """Latency percentiles (ms) and throughput of a served run."""
    if not results:
        return {"requests": 0}
    lat = np.array([r.latency for r in results]) * 1e3
    que = np.array([r.queued for r in results]) * 1e3
    span = makespan if makespan is not None else max(r.done for r in results) - min(r.arrival for r in results)
    return {
        "requests": len(results),
        "makespan_s": span,
        "throughput_rps": len(results) / span if span > 0 else float("inf"),
        "latency_ms": {"p50": float(np.percentile(lat, 50)), "p90": float(np.percentile(lat, 90)),
                       "p99": float(np.percentile(lat, 99)), "max": float(lat.max()), "mean": float(lat.mean())},
        "queue_ms": {"p50": float(np.percentile(que, 50)), "p99": float(np.percentile(que, 99))},
    }


# ------------------------------------------------------------ workloads
def mix_specs(n_graphs: int = 200, n_lo: float = 1e3, n_hi: float = 2e6, seed_base: int = 1000):
    """The serving mix: graph i draws (from seed seed_base + i) n log-uniform
    in [n_lo, n_hi] and a mean degree uniform in 8..16.  The first half are
    Barabasi-Albert graphs with m = deg // 2 edges per new vertex, the second
    half R-MAT digraphs of scale round(log2 n) with deg // 2 arcs per vertex
    (a, b, c = 0.57, 0.19, 0.19).  Returns (kind, size parameter, degree
    parameter, seed) per graph."""
    from . import graphgen as gen
    specs = []
    for i in range(n_graphs):
        u = gen.uniform_u32(seed_base + i, 2, 1 << 30).astype(np.float64) / float(1 << 30)
        n = int(round(10 ** (math.log10(n_lo) + u[0] * (math.log10(n_hi) - math.log10(n_lo)))))
        deg = 8 + int(u[1] * 9)
        if i < n_graphs // 2:
            specs.append(("ba", max(n, deg // 2 + 2), max(deg // 2, 1), seed_base + i))
        else:
            specs.append(("rmat", max(int(round(math.log2(n))), 4), max(deg // 2, 1), seed_base + i))
    return specs


def build_graph(spec):
    from . import graphgen as gen
    kind, a, b, seed = spec
    if kind == "ba":
        return gen.ba(a, b, seed=seed)
    if kind == "rmat":
        return gen.rmat(a, b, seed=seed)
    raise ValueError(kind)


def request_stream(n_requests: int, n_graphs: int, rate: float, seed: int = 5, ks=(1, 10, 100)):
    """n_requests requests: graph uniform over n_graphs, k uniform over ks,
    Poisson arrivals at `rate` per second (rate = inf: all at time 0)."""
    from . import graphgen as gen
    u = gen.uniform_u32(seed, 2 * n_requests, 1 << 30)
    gids = (u[0::2] % n_graphs).astype(int)
    kidx = (u[1::2] % len(ks)).astype(int)
    if math.isinf(rate):
        arr = np.zeros(n_requests)
    else:
        arr = np.cumsum(gen.exponential(seed + 0x5EED, n_requests, 1.0 / rate))
    return [Request(i, int(gids[i]), int(ks[kidx[i]]), float(arr[i])) for i in range(n_requests)]


# ---------------------------------------------------------- GPU backend
class GpuBackend(Backend):
    """Graphs resident on the device, one CUDA stream and one set of pinned
    output buffers per graph."""

    def __init__(self, graphs, options=None, kmax: int = 1024, trace: bool = False, workspace_cap: int = 0):
        import torch

        from . import bcm
        super().__init__()
        self.bcm = bcm
        bcm.load()
        self.opts = options if options is not None else bcm.make_options()
        # workspace_cap > 0: a run on a large graph uses fewer per-CTA blocks,
        # so that its workspace (one n-vertex slot per block) stays under the
        # cap; with cap = budget / max_inflight the runs in flight fit the
        # budget together instead of trimming one another's workspaces
        self.workspace_cap = int(workspace_cap)
        # with trace, every run records its kernels' time stamps and collect()
        # reports the span of device time the run's waves occupied
        self.trace = trace
        if trace:
            self.opts.flags |= bcm.BCM_TRACE
        self.streams = []
        self.handles = []
        self.bufs = []
        self.kk = {}
        self.stats = {}
        for g in graphs:
            s = torch.cuda.Stream()
            h = bcm.BcmGraph.from_graph(g, stream=s.cuda_stream)
            bcm.bcm_preprocess(h.h)            # components / SCC bounds and order, once
            self.streams.append(s)
            self.handles.append(h)
            kb = max(min(kmax, g.n), 1)
            self.bufs.append((torch.zeros(kb, dtype=torch.int32).pin_memory(),
                              torch.zeros(kb, dtype=torch.int64).pin_memory(),
                              torch.zeros(kb, dtype=torch.int32).pin_memory()))
        self._fp = {}
        self._gopts = {}

    def options(self, gid):
        """The run options of graph gid: the backend's, with the per-CTA
        block count set to the largest whose workspace fits the cap when
        there is one (the library's default, every resident CTA, may not)."""
        if gid not in self._gopts:
            o = self.opts
            h = self.handles[gid].h
            if self.workspace_cap and not o.blocks and self.bcm.bcm_workspace_bytes(h, o) > self.workspace_cap:
                kw = _opts_kw(o)
                lo, hi = 1, 1
                while self.bcm.bcm_workspace_bytes(h, self.bcm.make_options(**dict(kw, blocks=hi * 2))) <= \
                        self.workspace_cap and hi < (1 << 16):
                    hi *= 2
                hi *= 2   # blocks=hi does not fit (or the library caps blocks below it)
                while hi - lo > 1:
                    mid = (lo + hi) // 2
                    if self.bcm.bcm_workspace_bytes(h, self.bcm.make_options(**dict(kw, blocks=mid))) <= \
                            self.workspace_cap:
                        lo = mid
                    else:
                        hi = mid
                o = self.bcm.make_options(**dict(kw, blocks=lo))
            self._gopts[gid] = o
        return self._gopts[gid]

    def footprint(self, gid):
        if gid not in self._fp:
            self._fp[gid] = self.bcm.bcm_workspace_bytes(self.handles[gid].h, self.options(gid))
        return self._fp[gid]

    def start(self, gid, k):
        h = self.handles[gid]
        ids, far, reach = self.bufs[gid]
        self.kk[gid] = min(k, h.n)
        self.stats[gid] = self.bcm.bcm_stats()
        self.bcm.bcm_topk_start(h.h, k, self.options(gid), ids, far, reach)

    def poll(self, gid):
        return self.bcm.bcm_topk_finish(self.handles[gid].h, wait=False, stats=self.stats[gid])

    def collect(self, gid):
        kk = self.kk[gid]
        ids, far, reach = self.bufs[gid]
        st = self.stats[gid].as_dict()
        if self.trace:
            rec, _ = self.bcm.bcm_trace(self.handles[gid].h)
            if len(rec):
                kind = rec[:, 1] >> np.uint64(60)
                starts = np.where(kind == self.bcm.TRACE_CTA_WAVE, rec[:, 3], rec[:, 0]).astype(np.int64)
                st["device_span_ns"] = (int(starts.min()), int(rec[:, 0].astype(np.int64).max()))
        return (ids.numpy()[:kk].view(np.uint32).copy(), far.numpy()[:kk].view(np.uint64).copy(),
                reach.numpy()[:kk].view(np.uint32).copy(), st)

    def trim(self, gid):
        self.bcm.bcm_graph_trim(self.handles[gid].h)
        self.held.pop(gid, None)

    def trim_all(self):
        for gid in list(self.held.keys()):
            self.trim(gid)

    def alone(self, gid, k):
        """The same request run by itself, synchronously (no trace); its
        workspace is given back afterwards unless the graph already held one."""
        kw = _opts_kw(self.options(gid))
        kw["flags"] &= ~self.bcm.BCM_TRACE
        had = gid in self.held
        res = self.handles[gid].topk(k, **kw)
        if not had:
            self.bcm.bcm_graph_trim(self.handles[gid].h)
        return res

    def close(self):
        for h in self.handles:
            h.close()
        self.handles = []


def _opts_kw(o):
    return dict(lanes=o.lanes, flags=o.flags, blocks=o.blocks, threads=o.threads, wait_limit_ns=o.wait_limit_ns,
                grid_lanes=o.grid_lanes, heavy_words=o.heavy_words, pull_div=o.pull_div, defer_words=o.defer_words,
                shard_index=o.shard_index, shard_count=o.shard_count, cta_table=o.cta_table)
