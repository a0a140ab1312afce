"""Host logic of the autotuner (no GPU): the search over candidates with a
fake timer, and the per-shape result cache."""
import json

from paper_2006_10142_gb300 import autotune


def _fake_timer(table, default=(5.0, 5.0), rejected=()):
    """measure(cfg) from a table keyed by the knobs that matter here."""
    calls = []

    def measure(cfg):
        calls.append(dict(cfg))
        if not cfg:
            return default
        if cfg.get("chunk_x") in rejected:
            return None
        x = table["x"].get(cfg.get("chunk_x"), 9.0) + table["solver"].get(cfg.get("solver"), 0.0)
        y = table["y"].get(cfg.get("chunk_y"), 9.0) if "chunk_y" in cfg else 7.0
        return (x, y)
    return measure, calls


def test_search_picks_x_then_y_and_beats_the_default():
    shared = [dict(solver=1), dict(solver=2)]
    xs = [dict(chunk_x=k) for k in (8, 16, 32)]
    ys = [dict(chunk_y=k) for k in (8, 16, 32)]
    table = {"x": {8: 4.0, 16: 2.0, 32: 3.0}, "y": {8: 1.5, 16: 3.0, 32: 2.5},
             "solver": {1: 0.0, 2: 0.5}}
    measure, calls = _fake_timer(table)
    tot, tuning, x_ms, y_ms = autotune.search(measure, shared, xs, ys)
    assert tuning == {"solver": 1, "chunk_x": 16, "chunk_y": 8}
    assert (x_ms, y_ms, tot) == (2.0, 1.5, 3.5)
    assert calls[0] == {}                                  # the planner's choice first
    # y candidates run with the best x of their shared setting
    assert {"solver": 1, "chunk_x": 16, "chunk_y": 32} in calls


def test_search_keeps_the_default_unless_a_candidate_is_faster():
    table = {"x": {8: 4.0}, "y": {8: 4.0}, "solver": {}}
    measure, _ = _fake_timer(table, default=(3.0, 3.0))
    tot, tuning, _, _ = autotune.search(measure, [dict(solver=1)], [dict(chunk_x=8)],
                                        [dict(chunk_y=8)])
    assert tuning == {} and tot == 6.0


def test_search_skips_rejected_shapes_and_can_find_nothing():
    table = {"x": {8: 1.0, 16: 2.0}, "y": {8: 1.0}, "solver": {}}
    measure, _ = _fake_timer(table, default=(9.0, 9.0), rejected=(8,))
    best = autotune.search(measure, [dict(solver=1)], [dict(chunk_x=8), dict(chunk_x=16)],
                           [dict(chunk_y=8)])
    assert best[1]["chunk_x"] == 16

    def reject_all(cfg):
        return None
    assert autotune.search(reject_all, [dict(solver=1)], [dict(chunk_x=8)], [dict(chunk_y=8)]) is None


def test_candidates_cover_every_stage_mode():
    shared, xs, ys = autotune.candidates(4096, 4096)
    assert {c["x_stage"] for c in xs} == {2, 3, 5}
    assert {c["y_stage"] for c in ys} == {1, 2, 3, 4}
    assert all(set(c) == set(autotune.X_KNOBS) for c in xs)
    assert all(set(c) == set(autotune.Y_KNOBS) for c in ys)
    assert all(set(s) == set(autotune.SHARED_KNOBS) for s in shared)


def test_cache_roundtrip(tmp_path, monkeypatch):
    path = tmp_path / "sub" / "tuning.json"
    monkeypatch.setenv("ADIWAVE_TUNE_CACHE", str(path))
    assert autotune.cache_path() == str(path)
    assert autotune._load_cache() == {}
    key = autotune._key("GB300", 4096, 2048, "auto")
    assert key == "GB300|4096x2048|auto"
    autotune._store_cache({key: {"tuning": {"chunk_x": 32}, "x_ms": 1.0, "y_ms": 2.0}})
    assert json.loads(path.read_text())[key]["tuning"] == {"chunk_x": 32}
    assert autotune._load_cache()[key]["y_ms"] == 2.0
    path.write_text("not json")
    assert autotune._load_cache() == {}
