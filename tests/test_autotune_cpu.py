"""Host logic of the autotuner: cache keys, occupancy buckets, selection and the JSON cache."""
import json

import pytest

from paper_2403_01596_gb300 import autotune as T


def test_occupancy_bucket():
    assert T.occupancy_bucket(1 << 20, 131520) == 8
    assert T.occupancy_bucket(1 << 20, 65622) == 16
    assert T.occupancy_bucket(1 << 20, 16674) == 64
    assert T.occupancy_bucket(10, 10) == 1
    assert T.occupancy_bucket(0, 0) == 0


def test_cache_key_orders_layouts():
    a = T.cache_key("NVIDIA GB300", 152, "helmholtz", 16, 1, ("redundant", "indexed"))
    b = T.cache_key("NVIDIA GB300", 152, "helmholtz", 16, 1, ("indexed", "redundant"))
    assert a == b
    assert a != T.cache_key("NVIDIA GB300", 152, "helmholtz", 16, 8, ("indexed", "redundant"))


def test_select_prefers_fastest_then_smaller():
    t = [{"layout": "redundant", "tuning": {"chunk": 128, "warps_per_cta": 8}, "ms": 0.30},
         {"layout": "indexed", "tuning": {"chunk": 256, "warps_per_cta": 8}, "ms": 0.25},
         {"layout": "indexed", "tuning": {"chunk": 128, "warps_per_cta": 8}, "ms": 0.25}]
    best = T.select(t)
    assert best["layout"] == "indexed" and best["tuning"]["chunk"] == 128
    with pytest.raises(ValueError):
        T.select([])


def test_cache_round_trip(tmp_path, monkeypatch):
    p = tmp_path / "sub" / "tune.json"
    monkeypatch.setenv("P2P_AUTOTUNE_CACHE", str(p))
    assert T.cache_path() == str(p)
    assert T.load_cache() == {}
    T.save_cache({"k": {"layout": "indexed", "tuning": {"chunk": 64}, "ms": 1.0}})
    assert json.loads(p.read_text())["k"]["tuning"]["chunk"] == 64
    p.write_text("not json")
    assert T.load_cache() == {}


def test_candidates_are_valid_tunings():
    from paper_2403_01596_gb300 import _capi as C
    for cand in T.DEFAULT_CANDIDATES:
        # a valid tuning gives a workspace size; an invalid one raises
        assert C.p2p_plan_workspace_size(1000, 100, 500, 5000, 0, 1, cand) > 0
