"""The autotuner's host logic on CPU: the candidate list by the spread of the
starting smoothing lengths, the partition of a batch, and the choice of the
fastest candidate with its cache (the pool timing replaced by a fake)."""
import json

import numpy as np
import pytest

from paper_2305_13380_gb300 import sph, tune


def _sim(h_lo, h_hi, n=64, seed=0):
    rng = np.random.default_rng(seed)
    return {"h0": np.exp(rng.uniform(np.log(h_lo), np.log(h_hi), n)).astype(np.float32)}


def test_candidates_follow_the_spread():
    smooth = [_sim(0.01, 0.012)]
    clustered = [_sim(0.001, 0.05)]
    c_smooth = tune.candidates(smooth)
    c_clust = tune.candidates(clustered)
    tree = [c for c in c_smooth if c["flags"] & sph.SPH_FLAG_TREE]
    assert len(tree) == len(tune.MARGINS) * len(tune.LEAVES)
    assert all("n_leaf" in c and "cell_margin" in c for c in tree)
    uniform = [c for c in c_smooth if c["flags"] == 0]
    assert len(uniform) == len(tune.MARGINS) * len(tune.LANES)
    assert any(c["flags"] & sph.SPH_FLAG_SYMMETRIC for c in c_smooth)
    # strongly clustered: nested grids only
    assert all(c["flags"] & sph.SPH_FLAG_TREE for c in c_clust)
    assert len(c_clust) == len(tree)
    # one clustered simulation in the pool is enough to drop the uniform grid
    assert all(c["flags"] & sph.SPH_FLAG_TREE for c in tune.candidates(smooth + clustered))


def test_partition_splits_by_spread_and_drops_empty_parts():
    sims = [_sim(0.01, 0.012, seed=1), _sim(0.001, 0.05, seed=2), _sim(0.02, 0.03, seed=3),
            _sim(0.0005, 0.02, seed=4)]
    assert tune.partition(sims) == [[0, 2], [1, 3]]
    assert tune.partition([sims[0], sims[2]]) == [[0, 1]]
    assert tune.partition([sims[1]]) == [[0]]
    assert tune.partition([]) == []


@pytest.fixture
def fake_gpu(monkeypatch, tmp_path):
    cache = tmp_path / "tune_cache.json"
    monkeypatch.setattr(tune, "_CACHE", str(cache))
    monkeypatch.setattr(tune.torch.cuda, "get_device_name", lambda *a: "fake GPU")
    return cache


def test_tune_keeps_the_fastest_and_caches(fake_gpu, monkeypatch):
    sims = [_sim(0.01, 0.012)]
    calls = []

    def fake_time(s, over, steps, give_up_ms):
        calls.append((dict(over), give_up_ms))
        ms = 10.0 + 100.0 * over["cell_margin"] + (0.5 if over["flags"] & sph.SPH_FLAG_TREE else 0.0)
        if over["flags"] & sph.SPH_FLAG_SYMMETRIC:
            return None  # a candidate that failed
        if over["flags"] == 0:
            ms -= 0.1 * over.get("lanes_per_target", 0)
        return ms

    monkeypatch.setattr(tune, "_time", fake_time)
    rec = tune.tune(sims, key="k")
    assert rec["best"] == {"flags": 0, "cell_margin": 0.03, "lanes_per_target": 4}
    assert rec["best_ms"] == pytest.approx(10.0 + 3.0 - 0.4)
    # the default of the chosen mode: margin 0.05, automatic lanes
    assert rec["default_ms"] == pytest.approx(15.0)
    assert len(rec["times"]) == len(tune.candidates(sims))
    # each candidate gives up at four times the best so far
    assert calls[0][1] == float("inf")
    assert all(g >= 4.0 * rec["best_ms"] for _, g in calls)
    # cached per GPU name and key: a second call times nothing
    data = json.load(open(fake_gpu))
    assert "fake GPU|k" in data
    calls.clear()
    assert tune.best_params(sims, key="k") == rec["best"]
    assert calls == []


def test_tune_refuses_when_nothing_runs(fake_gpu, monkeypatch):
    monkeypatch.setattr(tune, "_time", lambda *a, **k: None)
    with pytest.raises(RuntimeError):
        tune.tune([_sim(0.01, 0.012)], key="none")


def test_best_split_tunes_each_part(fake_gpu, monkeypatch):
    seen = []

    def fake_time(s, over, steps, give_up_ms):
        seen.append(len(s))
        return 1.0 + over["cell_margin"]

    monkeypatch.setattr(tune, "_time", fake_time)
    sims = [_sim(0.01, 0.012, seed=1), _sim(0.001, 0.05, seed=2), _sim(0.02, 0.03, seed=3)]
    split = tune.best_split(sims, key="b")
    assert [idx for idx, _ in split] == [[0, 2], [1]]
    assert split[1][1]["flags"] & sph.SPH_FLAG_TREE
    assert set(seen) == {2, 1}
