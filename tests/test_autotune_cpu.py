"""Cache logic of the autotuner (no GPU): keys, round trip, candidate sets."""
import json

from paper_1008_2801_gb300 import autotune


def test_cache_round_trip(tmp_path, monkeypatch):
    path = tmp_path / "tune.json"
    monkeypatch.setenv("MG_TUNE_CACHE", str(path))
    assert autotune.lookup("GPU", [(8, 8, 8)], "fp64") is None
    autotune.record("GPU", [(8, 8, 8)], "fp64", {"smoother": "passes"}, 1.5)
    autotune.record("GPU", [(8, 8, 8)], "mixed", {"smoother": "fused"}, 1.0)
    assert autotune.lookup("GPU", [(8, 8, 8)], "fp64")["opts"] == {"smoother": "passes"}
    assert autotune.lookup("GPU", [(8, 8, 8)], "mixed")["ms"] == 1.0
    assert autotune.lookup("GPU", [(8, 8, 16)], "fp64") is None
    assert len(json.loads(path.read_text())) == 2


def test_candidates_cover_the_options():
    c64 = list(autotune.candidates("fp64"))
    cmx = list(autotune.candidates("mixed"))
    # FP64 levels always use passes: no smoother choice there
    assert len(cmx) == 3 * 3 * len(c64) and len(c64) == 4 * 3
    assert {c["smoother"] for c in c64} == {"auto"}
    assert {c["smoother"] for c in cmx} == {"auto", "passes", "fused"}
    assert {c["inner_cycles"] for c in cmx} == {0, 2, 4}   # 0: adaptive
    assert {c["persistent"] for c in c64} == {False, "small", "all"}
    for c in c64 + cmx:
        assert set(c) == set(autotune.DEFAULTS)
    assert autotune.key("G", [(2, 3, 4), (5, 6, 7)], "fp64") == "G|fp64|2x3x4;5x6x7"


def test_tile_candidates_follow_the_options():
    base = dict(autotune.DEFAULTS)
    # mixed, fused sweeps possible, per-stage launches: the sweep's tile depth
    t = list(autotune.tile_candidates(dict(base, smoother="fused"), "mixed"))
    assert {c["sweep_zc"] for c in t} == set(autotune.SWEEP_ZC)
    assert {c["level_ctas"] for c in t} == {0}
    # passes only and persistent launches: their CTAs per SM
    t = list(autotune.tile_candidates(dict(base, smoother="passes", persistent="all"), "mixed"))
    assert {c["sweep_zc"] for c in t} == {0}
    assert {c["level_ctas"] for c in t} == set(autotune.LEVEL_CTAS)
    # FP64: no fused sweep
    t = list(autotune.tile_candidates(dict(base, persistent="small"), "fp64"))
    assert {c["sweep_zc"] for c in t} == {0}
