"""The autotuner on the GPU: every trial returns the same top-k (it raises
otherwise), and the tuned setting reproduces the default run's result."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def test_tuned_setting_gives_the_same_topk(gen, tmp_path):
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    torch.cuda.set_device(0)
    from paper_1507_01490_gb300 import _build, autotune, bcm
    _build.build_cuda()
    for g in (gen.chung_lu(1 << 15, 10.0, 2.3, seed=2), gen.rmat(13, 8, seed=3)):
        with bcm.BcmGraph.from_graph(g) as h:
            ref = h.topk(10)
            cfg, spent, hit = autotune.tuned_options(h, g, 10, cache_path=str(tmp_path / "t.json"), rounds=1, reps=1)
            assert not hit and cfg["threads"] >= cfg["lanes"]
            got = h.topk(10, **cfg)
            assert all(np.array_equal(a, b) for a, b in zip(ref[:3], got[:3]))
            assert autotune.tuned_options(h, g, 10, cache_path=str(tmp_path / "t.json"))[2]
