"""Serving with continuous batching on the GPU: every request's result is the
oracle's exact top-k (the sequential Algorithm 1, pinned against the textbook
top-k) and the same alone and in the mix (bit-exact: ids, farness, reach),
runs on different graphs overlap on the device, and admission keeps the
workspace inside the HBM budget."""
import math

import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def _oracle_topk(args):
    g, k = args
    import oracle
    ids, far, reach, _ = oracle.bcm(g, k, refined=g.directed)
    return ids, far, reach


def _oracle_answers(graphs, keys):
    """The oracle's top-k for each (graph, k), in processes of their own (spawned:
    this process already holds a CUDA context)."""
    import multiprocessing as mp
    from concurrent.futures import ProcessPoolExecutor
    keys = sorted(keys)
    with ProcessPoolExecutor(max_workers=min(16, len(keys)), mp_context=mp.get_context("spawn")) as ex:
        res = list(ex.map(_oracle_topk, [(graphs[gi], k) for gi, k in keys]))
    return dict(zip(keys, res))


@pytest.fixture(scope="module")
def backend():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    torch.cuda.set_device(0)
    from paper_1507_01490_gb300 import _build, serve
    _build.build_cuda()
    # the serving recipe, scaled down: 16 graphs, n log-uniform in [1e3, 2e5]
    specs = serve.mix_specs(16, n_hi=2e5)
    graphs = [serve.build_graph(s) for s in specs]
    be = serve.GpuBackend(graphs, trace=True)
    be.test_graphs = graphs
    yield be
    be.close()


def test_results_identical_alone_and_in_the_mix(backend):
    from paper_1507_01490_gb300 import serve
    reqs = serve.request_stream(240, 16, rate=math.inf, seed=5)
    sched = serve.Scheduler(backend, max_inflight=8)
    res = sched.run(reqs)
    assert sched.peak_inflight > 1
    exact = _oracle_answers(backend.test_graphs, {(r.graph, r.k) for r in res})
    alone = {}
    for r in res:
        key = (r.graph, r.k)
        if key not in alone:
            alone[key] = backend.alone(r.graph, r.k)
        ids, far, reach, _ = alone[key]
        assert np.array_equal(r.ids, ids), key
        assert np.array_equal(r.farness, far), key
        assert np.array_equal(r.reach, reach), key
        oi, of, orr = exact[key]
        assert np.array_equal(r.ids, oi) and np.array_equal(r.farness, of) and np.array_equal(r.reach, orr), key
    # device time of runs on different graphs overlapped
    spans = [(r.stats["device_span_ns"], r.graph) for r in res if "device_span_ns" in r.stats]
    spans.sort()
    overlap = 0
    for (a, ga), (b, gb) in zip(spans, spans[1:]):
        if b[0] < a[1] and ga != gb:
            overlap += 1
    assert overlap > 0


def test_budget_bounds_the_held_workspace(backend):
    from paper_1507_01490_gb300 import serve
    fps = [backend.footprint(g) for g in range(16)]
    budget = max(fps) + sorted(fps)[len(fps) // 2]
    for g in range(16):
        backend.trim(g)
    reqs = serve.request_stream(120, 16, rate=2000.0, seed=9)
    sched = serve.Scheduler(backend, max_inflight=8, hbm_budget=budget)
    res = sched.run(reqs)
    assert len(res) == 120 and sched.peak_held <= budget and sched.trims > 0
    for r in res[:40]:
        ids, far, reach, _ = backend.alone(r.graph, r.k)
        assert np.array_equal(r.ids, ids) and np.array_equal(r.farness, far) and np.array_equal(r.reach, reach)


def test_workspace_cap_lowers_blocks_not_results(backend):
    """A per-run workspace cap gives the large graphs fewer per-CTA blocks (the
    largest count whose workspace fits) and leaves every result unchanged."""
    from paper_1507_01490_gb300 import bcm, serve
    fps = [backend.footprint(g) for g in range(16)]
    cap = sorted(fps)[len(fps) // 2]
    capped = serve.GpuBackend.__new__(serve.GpuBackend)
    capped.__dict__.update(backend.__dict__)
    capped._fp, capped._gopts, capped.workspace_cap = {}, {}, cap
    capped.held = backend.held
    for g in range(16):
        o = capped.options(g)
        if fps[g] <= cap:
            assert o.blocks == 0 and capped.footprint(g) == fps[g]
            continue
        assert o.blocks >= 1 and capped.footprint(g) < fps[g]
        if o.blocks > 1:
            assert capped.footprint(g) <= cap
            more = bcm.make_options(**dict(serve._opts_kw(o), blocks=o.blocks + 1))
            assert bcm.bcm_workspace_bytes(backend.handles[g].h, more) > cap
        for k in (1, 10, 100):
            a = backend.alone(g, k)
            b = capped.alone(g, k)
            assert all(np.array_equal(x, y) for x, y in zip(a[:3], b[:3])), (g, k)
