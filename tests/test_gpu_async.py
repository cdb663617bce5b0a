"""bcm_topk_start / bcm_topk_finish (runs in flight on several graphs at
once), bcm_trace and bcm_graph_trim, against the synchronous bcm_topk."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def B():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    torch.cuda.set_device(0)
    from paper_1507_01490_gb300 import _build, bcm
    _build.build_cuda()
    bcm.load()
    return bcm


def _graphs(gen):
    return [gen.ba(2000, 3, seed=1), gen.chung_lu(1 << 15, 10.0, 2.3, seed=2), gen.rmat(13, 8, seed=3),
            gen.grid_lcc(80, 80, 0.05, seed=4), gen.ba(300, 2, seed=5), gen.rmat(10, 16, seed=6)]


def test_overlapping_runs_match_sync(B, gen):
    import torch
    gs = _graphs(gen)
    streams = [torch.cuda.Stream() for _ in gs]
    hs = [B.BcmGraph.from_graph(g, stream=s.cuda_stream) for g, s in zip(gs, streams)]
    try:
        for k in (1, 10, 100):
            ref = [h.topk(k) for h in hs]
            outs = []
            for g, h in zip(gs, hs):
                kk = min(k, g.n)
                o = (torch.zeros(kk, dtype=torch.int32).pin_memory(), torch.zeros(kk, dtype=torch.int64).pin_memory(),
                     torch.zeros(kk, dtype=torch.int32).pin_memory())
                B.bcm_topk_start(h.h, k, B.make_options(), *o)
                outs.append(o)
            done = [False] * len(hs)
            stats = [B.bcm_stats() for _ in hs]
            spins = 0
            while not all(done):
                for i, h in enumerate(hs):
                    if not done[i]:
                        done[i] = B.bcm_topk_finish(h.h, wait=False, stats=stats[i])
                spins += 1
                assert spins < 10_000_000
            for (ids, far, reach, st), o, s in zip(ref, outs, stats):
                assert np.array_equal(o[0].numpy().view(np.uint32), ids)
                assert np.array_equal(o[1].numpy().view(np.uint64), far)
                assert np.array_equal(o[2].numpy().view(np.uint32), reach)
                assert s.m_vis == st["m_vis"] or s.m_vis > 0
    finally:
        for h in hs:
            h.close()


def test_one_run_per_graph(B, gen):
    g = gen.ba(2000, 3, seed=1)
    with B.BcmGraph.from_graph(g) as h:
        ids = np.zeros(10, np.uint32)
        far = np.zeros(10, np.uint64)
        reach = np.zeros(10, np.uint32)
        B.bcm_topk_start(h.h, 10, None, ids, far, reach)
        with pytest.raises(B.BcmError) as ei:
            B.bcm_topk_start(h.h, 10, None, ids, far, reach)
        assert ei.value.status == B.BCM_ERR_INVALID
        with pytest.raises(B.BcmError):
            h.trim()
        assert B.bcm_topk_finish(h.h, wait=True)
        with pytest.raises(B.BcmError):
            B.bcm_topk_finish(h.h, wait=True)      # nothing pending any more
        ref = h.topk(10)
        assert np.array_equal(ids, ref[0]) and np.array_equal(far, ref[1])


def test_trim_then_run_again(B, gen):
    g = gen.chung_lu(1 << 14, 10.0, 2.3, seed=7)
    with B.BcmGraph.from_graph(g) as h:
        a = h.topk(10)
        ws = B.bcm_workspace_bytes(h.h)
        assert ws > 0
        h.trim()
        b = h.topk(10)
        f1, r1, _ = h.farness_all()
        h.trim()
        f2, r2, _ = h.farness_all()
    assert all(np.array_equal(x, y) for x, y in zip(a[:3], b[:3]))
    assert np.array_equal(f1, f2) and np.array_equal(r1, r2)


@pytest.mark.parametrize("name", ["chung_lu", "rmat"])
def test_trace_matches_counters(B, gen, name):
    g = gen.chung_lu(1 << 16, 10.0, 2.3, seed=2) if name == "chung_lu" else gen.rmat(14, 16, seed=3)
    with B.BcmGraph.from_graph(g) as h:
        plain = h.topk(10)
        ids, far, reach, st = h.topk(10, flags=B.BCM_TRACE)
        rec, count = h.trace()
        assert all(np.array_equal(x, y) for x, y in zip(plain[:3], (ids, far, reach)))
        assert count == len(rec) and count > 0
        kind = (rec[:, 1] >> np.uint64(60)).astype(int)
        assert (kind == B.TRACE_GRID_LEVEL).sum() == st["grid_levels"]
        assert (kind == B.TRACE_GRID_WAVE).sum() == st["grid_waves"]
        assert (kind == B.TRACE_CTA_WAVE).sum() == st["waves"] - st["grid_waves"]
        cta = rec[kind == B.TRACE_CTA_WAVE]
        assert (cta[:, 0] >= cta[:, 3]).all()               # a wave ends after it starts
        lv = (cta[:, 1] & np.uint64(0xffffffff)).astype(np.int64)
        assert lv.sum() == st["levels"] - st["grid_levels"]
        assert int((cta[:, 2]).sum()) + int(rec[kind == B.TRACE_GRID_WAVE][:, 2].sum()) == st["cleared_words"]
        h.topk(10)                                          # an untraced run leaves no trace
        assert h.trace()[1] == 0
