"""Autotuner logic on the CPU: candidate space, search, cache keys and file."""
import json

import pytest

from paper_2210_06437_gb300 import tune


def test_candidates_cover_the_space():
    c = tune.candidates({"a": (1, 2), "b": (10, 20, 30)})
    assert len(c) == 6
    assert {"a": 2, "b": 30} in c


def test_search_picks_the_fastest_and_skips_failures():
    def measure(p):
        if p["a"] == 3:
            raise RuntimeError("invalid launch")
        return abs(p["a"] - 2) + 0.1 * p["b"]
    best, table = tune.search(measure, tune.candidates({"a": (1, 2, 3), "b": (1, 2)}))
    assert best == {"a": 2, "b": 1}
    assert any(t is None for _, t, _ in table)
    with pytest.raises(RuntimeError):
        tune.search(lambda p: 1 / 0, tune.candidates({"a": (1,)}))


def test_cache_roundtrip(tmp_path, monkeypatch):
    path = tmp_path / "cache.json"
    monkeypatch.setenv("HYDRO_TUNE_CACHE", str(path))
    k1 = tune.cache_key("NVIDIA GB300", "mixed", 65536)
    k2 = tune.cache_key("NVIDIA GB300", "mixed", 40000)
    assert k1 == k2                       # same power-of-two bucket
    assert tune.cache_key("NVIDIA GB300", "fp64", 65536) != k1
    tune.store_cache(k1, {"params": {"stage_ctas_per_sm": 2, "prefetch_pass": 1, "reflux_shape": 0}})
    assert tune.load_cache()[k1]["params"]["stage_ctas_per_sm"] == 2
    path.write_text("not json")
    assert tune.load_cache() == {}
    json.loads(json.dumps(tune.SPACE_MIXED))
    assert set(tune.space_for("fp64")) <= set(tune.PARAMS) and set(tune.space_for("mixed")) == set(tune.PARAMS)
