"""The serving scheduler's host logic, on the CPU, against a fake backend
with a virtual clock: slots, one run per graph, the HBM budget with LRU
trimming, continuous admission, and the workload generators."""
import math

import numpy as np
import pytest

from paper_1507_01490_gb300 import serve


class FakeBackend(serve.Backend):
    """Runs take a fixed virtual time per (graph, k); the answer is a
    function of (graph, k) only."""

    def __init__(self, sizes, durations, sched_ref):
        super().__init__()
        self.sizes = sizes
        self.dur = durations
        self.t = 0.0
        self.end = {}
        self.k = {}
        self.alloc = set()          # graphs holding device memory, as the fake device sees them
        self.sched = sched_ref
        self.log = []

    # virtual clock
    def clock(self):
        return self.t

    def sleep(self, s):
        self.t += max(s, 1e-6)

    def footprint(self, gid):
        return self.sizes[gid]

    def start(self, gid, k):
        s = self.sched[0]
        assert gid not in self.end, "two runs on one graph"
        assert len(self.end) < s.max_inflight
        self.alloc.add(gid)
        assert sum(self.sizes[g] for g in self.alloc) <= s.budget
        self.end[gid] = self.t + self.dur(gid, k)
        self.k[gid] = k
        self.log.append(("start", gid, self.t))

    def poll(self, gid):
        return self.t >= self.end[gid]

    def collect(self, gid):
        k = self.k.pop(gid)
        del self.end[gid]
        ids = (np.arange(k, dtype=np.uint32) * 7 + gid) % 1000
        return ids, ids.astype(np.uint64) * 3, ids + 1, {"m_vis": gid * 1000 + k}

    def trim(self, gid):
        assert gid not in self.end, "trimmed a busy graph"
        self.alloc.discard(gid)
        self.held.pop(gid, None)
        self.log.append(("trim", gid, self.t))


def _run(reqs, sizes, dur, **kw):
    ref = [None]
    be = FakeBackend(sizes, dur, ref)
    s = serve.Scheduler(be, clock=be.clock, sleep=be.sleep, **kw)
    ref[0] = s
    return s, be, s.run(reqs)


def test_every_request_served_with_its_answer():
    reqs = serve.request_stream(500, 20, rate=200.0, seed=11)
    s, be, res = _run(reqs, [1 << 20] * 20, lambda g, k: 0.001 * (1 + g % 5) * (1 + k / 100), max_inflight=4)
    assert [r.rid for r in res] == list(range(500))
    for q, r in zip(reqs, res):
        assert (r.graph, r.k) == (q.graph, q.k)
        exp = (np.arange(q.k, dtype=np.uint32) * 7 + q.graph) % 1000
        assert np.array_equal(r.ids, exp) and r.stats["m_vis"] == q.graph * 1000 + q.k
        assert r.arrival <= r.admitted <= r.done
    assert s.peak_inflight <= 4


def test_runs_overlap_and_later_arrivals_join():
    # one long run on graph 0; short requests on other graphs arrive while it
    # runs and are admitted and finished before it ends
    reqs = [serve.Request(0, 0, 100, 0.0)] + [serve.Request(i, i % 5 + 1, 10, 0.01 * i) for i in range(1, 30)]
    s, be, res = _run(reqs, [1] * 6, lambda g, k: 1.0 if g == 0 else 0.025, max_inflight=3)
    long = res[0]
    short_done = [r for r in res[1:] if r.done < long.done]
    assert len(short_done) == 29
    assert all(r.admitted > long.admitted for r in short_done)
    assert s.peak_inflight == 3


def test_same_graph_requests_are_serialised_in_order():
    reqs = [serve.Request(i, 3, 10, 0.0) for i in range(6)]
    s, be, res = _run(reqs, [1] * 4, lambda g, k: 0.01, max_inflight=8)
    starts = [t for kind, g, t in be.log if kind == "start"]
    assert len(starts) == 6 and all(b >= a + 0.01 - 1e-9 for a, b in zip(starts, starts[1:]))
    assert [r.rid for r in sorted(res, key=lambda r: r.admitted)] == list(range(6))


def test_budget_trims_idle_graphs_lru():
    sizes = [40, 40, 40, 40]
    reqs = [serve.Request(i, g, 1, 0.001 * i) for i, g in enumerate([0, 1, 2, 0, 3, 1])]
    s, be, res = _run(reqs, sizes, lambda g, k: 0.0005, max_inflight=1, hbm_budget=100)
    trims = [g for kind, g, t in be.log if kind == "trim"]
    assert trims[:2] == [0, 1]            # least recently used idle graphs go first
    assert s.peak_held <= 100 and len(res) == 6


def test_request_waits_for_memory_not_for_order():
    # graph 0 needs most of the budget: while it runs, graph 1 (too big to
    # fit beside it) waits, but graph 2 (small) is admitted past it
    sizes = [70, 50, 10]
    reqs = [serve.Request(0, 0, 1, 0.0), serve.Request(1, 1, 1, 0.001), serve.Request(2, 2, 1, 0.002)]
    s, be, res = _run(reqs, sizes, lambda g, k: 0.1 if g == 0 else 0.01, max_inflight=4, hbm_budget=100)
    assert res[2].admitted < res[0].done <= res[1].admitted + 1e-9


def test_ledger_survives_across_schedulers():
    # graphs keep their workspace after a run; a second scheduler on the same
    # backend sees them and trims to stay in budget
    sizes = [40, 40, 40]
    ref = [None]
    be = FakeBackend(sizes, lambda g, k: 0.001, ref)
    for gids in ([0, 1], [2, 0]):
        s = serve.Scheduler(be, clock=be.clock, sleep=be.sleep, max_inflight=1, hbm_budget=100)
        ref[0] = s
        s.run([serve.Request(i, g, 1, 0.0) for i, g in enumerate(gids)])
        assert sum(be.held.values()) <= 100 and sum(sizes[g] for g in be.alloc) <= 100
    assert [g for kind, g, t in be.log if kind == "trim"] == [0, 1]   # LRU: 0 before 2 runs, then 1 before 0 does


def test_oversized_request_is_an_error():
    with pytest.raises(ValueError):
        _run([serve.Request(0, 0, 1, 0.0)], [200], lambda g, k: 0.01, hbm_budget=100)


def test_summary_percentiles():
    res = [serve.Result(i, 0, 1, 0.0, 0.0, (i + 1) / 1000, None, None, None) for i in range(100)]
    s = serve.summarize(res)
    assert s["requests"] == 100
    assert abs(s["latency_ms"]["p50"] - 50.5) < 1e-9 and abs(s["latency_ms"]["p99"] - 99.01) < 1e-9
    assert abs(s["throughput_rps"] - 1000.0) < 1e-9


def test_mix_and_stream_recipes():
    specs = serve.mix_specs(200)
    assert specs == serve.mix_specs(200)
    assert sum(1 for s in specs if s[0] == "ba") == 100
    for kind, a, b, seed in specs:
        if kind == "ba":
            assert 1000 <= a <= 2_000_000 and 4 <= b <= 8
        else:
            assert 10 <= a <= 21 and 4 <= b <= 8
    ns = np.array([a for kind, a, b, seed in specs if kind == "ba"], dtype=float)
    assert np.log10(ns).min() < 3.5 and np.log10(ns).max() > 5.5      # spread over the log range
    reqs = serve.request_stream(20000, 200, rate=50.0, seed=5)
    arr = np.array([r.arrival for r in reqs])
    assert (np.diff(arr) >= 0).all() and abs(arr[-1] / 20000 - 1 / 50.0) < 0.05 / 50.0 * 10
    ks = np.array([r.k for r in reqs])
    assert set(ks.tolist()) == {1, 10, 100} and all(abs((ks == k).mean() - 1 / 3) < 0.02 for k in (1, 10, 100))
    gids = np.array([r.graph for r in reqs])
    assert gids.min() == 0 and gids.max() == 199
    assert all(r.arrival == 0.0 for r in serve.request_stream(10, 3, rate=math.inf))


class _FakeBcm:
    """Workspace bytes linear in the per-CTA block count (0 = the library's
    default of 608), the shape of bcm_workspace_bytes."""

    def __init__(self, per_block, fixed, default_blocks=608, max_blocks=608):
        self.per_block, self.fixed = per_block, fixed
        self.default_blocks, self.max_blocks = default_blocks, max_blocks

    class Opt:
        def __init__(self, **kw):
            self.__dict__.update(dict(lanes=0, flags=0, blocks=0, threads=0, wait_limit_ns=0, grid_lanes=0,
                                      heavy_words=0, pull_div=0, defer_words=0, shard_index=0, shard_count=0,
                                      cta_table=0), **kw)

    def make_options(self, **kw):
        return self.Opt(**kw)

    def bcm_workspace_bytes(self, h, o):
        b = o.blocks or self.default_blocks
        return self.fixed + self.per_block * min(b, self.max_blocks)


class _Handle:
    h = None


@pytest.mark.parametrize("cap_blocks", [1, 7, 100, 607])
def test_workspace_cap_picks_the_largest_block_count_that_fits(cap_blocks):
    fb = _FakeBcm(per_block=1 << 20, fixed=5 << 20)
    be = serve.GpuBackend.__new__(serve.GpuBackend)
    be.bcm, be.opts, be.handles = fb, fb.make_options(), [_Handle()]
    be._gopts, be._fp = {}, {}
    be.workspace_cap = fb.fixed + fb.per_block * cap_blocks + (fb.per_block // 2)
    o = be.options(0)
    assert o.blocks == cap_blocks
    assert be.footprint(0) <= be.workspace_cap < fb.bcm_workspace_bytes(None, fb.make_options(blocks=cap_blocks + 1))


def test_workspace_cap_leaves_fitting_graphs_and_explicit_blocks_alone():
    fb = _FakeBcm(per_block=1 << 20, fixed=5 << 20)
    be = serve.GpuBackend.__new__(serve.GpuBackend)
    be.bcm, be.handles = fb, [_Handle(), _Handle()]
    be._gopts, be._fp = {}, {}
    be.opts = fb.make_options()
    be.workspace_cap = 1 << 40                   # everything fits: the backend's options as they are
    assert be.options(0) is be.opts
    be._gopts = {}
    be.opts = fb.make_options(blocks=3)          # a fixed block count is the caller's choice
    be.workspace_cap = 1 << 20
    assert be.options(1).blocks == 3
