"""The autotuner on the GPU: every trial returns the same top-k (it raises
otherwise), and the tuned setting's result is the oracle's exact top-k."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def test_tuned_setting_gives_the_oracle_topk(gen, orc, tmp_path):
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    torch.cuda.set_device(0)
    from paper_1507_01490_gb300 import _build, autotune, bcm
    _build.build_cuda()
    # a lattice (largest degree 4) also tunes the per-CTA kernel
    for g in (gen.chung_lu(1 << 15, 10.0, 2.3, seed=2), gen.rmat(13, 8, seed=3), gen.grid_lcc(100, 100, 0.05, seed=7)):
        exp = orc.topk_exhaustive(g, 10)
        with bcm.BcmGraph.from_graph(g) as h:
            cfg, spent, hit = autotune.tuned_options(h, g, 10, cache_path=str(tmp_path / "t.json"), rounds=1, reps=1)
            assert not hit and cfg["threads"] >= cfg["lanes"]
            assert ("per_cta" in cfg) == (int(g.degrees().max()) <= autotune.KERNEL_MAX_DEG)
            kw, fl = autotune.options_of(cfg)
            got = h.topk(10, flags=fl, **kw)
            assert all(np.array_equal(a, b) for a, b in zip(exp, got[:3])), g.name
            assert autotune.tuned_options(h, g, 10, cache_path=str(tmp_path / "t.json"))[2]
