"""The autotuner's search and cache on the CPU, against a fake graph handle
whose run time is a known function of the parameters."""
import numpy as np
import pytest

from paper_1507_01490_gb300 import autotune


class FakeHandle:
    def __init__(self, best, change_result_for=None):
        self.best = best
        self.calls = 0
        self.change = change_result_for

    def topk(self, k, flags=0, **cfg):
        self.calls += 1
        # time grows with the distance from `best` in each coordinate
        t = 1.0
        for name, v in cfg.items():
            vals = autotune.SPACE[name]
            t += abs(vals.index(v) - vals.index(self.best[name])) * 0.3
        if autotune.PER_CTA[self.best.get("per_cta", "auto")] != (flags & (autotune.PER_CTA["sparse"] |
                                                                            autotune.PER_CTA["bitlanes"])):
            t += 0.5
        ids = np.arange(k, dtype=np.uint32)
        if self.change and all(cfg.get(a) == b for a, b in self.change.items()):
            ids = ids[::-1].copy()
        return ids, ids.astype(np.uint64), ids, {"kernel_ms": t}


def test_descent_finds_the_separable_optimum():
    target = {"grid_lanes": 256, "pull_div": 128, "lanes": 128, "threads": 1024}
    h = FakeHandle(target)
    cfg, ms, trials = autotune.tune(h, k=10, rounds=3, reps=1)
    assert cfg == target and abs(ms - 1.0) < 1e-9
    assert len(trials) < 40


def test_invalid_shapes_are_skipped():
    # lanes 256 needs at least 256 threads: never tried with fewer
    h = FakeHandle({"grid_lanes": 128, "pull_div": 32, "lanes": 256, "threads": 256})
    cfg, ms, trials = autotune.tune(h, k=5, rounds=3, reps=1)
    assert all(c["threads"] >= c["lanes"] for c, _ in trials)
    assert cfg["lanes"] == 256 and cfg["threads"] >= 256


def test_a_changed_result_is_an_error():
    h = FakeHandle(dict(autotune.DEFAULTS), change_result_for={"grid_lanes": 64})
    with pytest.raises(RuntimeError):
        autotune.tune(h, k=10, rounds=1, reps=1)


def test_cache_roundtrip(tmp_path, gen):
    g = gen.path(10)
    target = {"grid_lanes": 64, "pull_div": 8, "lanes": 64, "threads": 256}
    h = FakeHandle(target)
    path = str(tmp_path / "sub" / "tune.json")
    cfg, spent, hit = autotune.tuned_options(h, g, k=3, cache_path=path, reps=1)
    # a path's largest degree is 2: the per-CTA kernel is tuned too
    assert cfg == dict(target, per_cta="auto") and not hit
    calls = h.calls
    cfg2, spent2, hit2 = autotune.tuned_options(h, g, k=3, cache_path=path, reps=1)
    assert cfg2 == cfg and hit2 and spent2 == 0.0 and h.calls == calls
    cfg3, _, hit3 = autotune.tuned_options(h, g, k=4, cache_path=path, reps=1)   # another k: tuned again
    assert not hit3


@pytest.mark.parametrize("kernel", ["sparse", "bitlanes"])
def test_per_cta_kernel_is_searched(kernel):
    """With kernels=True the per-CTA kernel is one more coordinate, passed as
    its flag; without, it is never tried."""
    target = dict(autotune.DEFAULTS, per_cta=kernel)
    h = FakeHandle(target)
    cfg, ms, trials = autotune.tune(h, k=10, rounds=2, reps=1, kernels=True)
    assert cfg == target and abs(ms - 1.0) < 1e-9
    cfg, ms, trials = autotune.tune(FakeHandle(target), k=10, rounds=2, reps=1)
    assert "per_cta" not in cfg and abs(ms - 1.5) < 1e-9
