"""The autotuner's search on the CPU: a fake context whose build time is a
known function of the setting stands in for timed GPU builds."""
import pytest

from paper_2411_12439_gb300 import autotune


class FakeCtx:
    def __init__(self, start, invalid=()):
        self.t = dict(start)
        self.invalid = set(invalid)
        self.builds = 0

    def tuning(self):
        return dict(self.t)

    def set_tuning(self, **kw):
        if any((k, v) in self.invalid for k, v in kw.items()):
            raise ValueError("not valid on this device")
        self.t = dict(kw)

    def build(self, data, offsets):
        self.builds += 1
        return type("G", (), {"free": lambda self: None})()


def _install_cost(monkeypatch, cost):
    monkeypatch.setattr(autotune, "_time_builds", lambda ctx, d, o, reps: cost(ctx.tuning()))


START = {"parse_blocks_per_sm": 0, "table_load": 0.5, "miss_flush": 64}


def test_finds_the_best_setting(monkeypatch):
    # separable cost with its minimum at (3, 0.6, 128)
    def cost(t):
        return (1.0 + abs(t["parse_blocks_per_sm"] - 3) * 0.1 + abs(t["table_load"] - 0.6) * 0.5
                + abs(t["miss_flush"] - 128) / 1000)
    _install_cost(monkeypatch, cost)
    ctx = FakeCtx(START)
    rep = autotune.autotune(ctx, None, None, reps=1)
    assert rep["tuning"] == {"parse_blocks_per_sm": 3, "table_load": 0.6, "miss_flush": 128}
    assert ctx.tuning() == rep["tuning"]  # the context keeps the best setting
    assert rep["ms"] == pytest.approx(cost(rep["tuning"]) * 1e3)
    assert rep["trials"][0][0] == START


def test_small_gains_do_not_move_it(monkeypatch):
    # every other setting is at most 1 % faster: below the 2 % bar
    _install_cost(monkeypatch, lambda t: 1.0 if t == START else 0.99)
    ctx = FakeCtx(START)
    rep = autotune.autotune(ctx, None, None, reps=1)
    assert rep["tuning"] == START and ctx.tuning() == START


def test_invalid_settings_are_skipped(monkeypatch):
    # the fastest value is refused by the device: the next best is kept
    _install_cost(monkeypatch, lambda t: {0: 1.0, 2: 0.8, 3: 0.9, 4: 0.5}[t["parse_blocks_per_sm"]])
    ctx = FakeCtx(START, invalid={("parse_blocks_per_sm", 4)})
    rep = autotune.autotune(ctx, None, None, reps=1, candidates={"parse_blocks_per_sm": [0, 2, 3, 4]})
    assert rep["tuning"]["parse_blocks_per_sm"] == 2
    assert all(s["parse_blocks_per_sm"] != 4 for s, _ in rep["trials"])


def test_config_class():
    import numpy as np
    dna = np.frombuffer(b"ACGTN" * 100, dtype=np.uint8)
    text = np.arange(256, dtype=np.uint8)
    assert autotune.config_class(12_400_000_000, 4, dna) == "dna/2^34B/1-8 strings"
    assert autotune.config_class(320_000_000, 64, dna) == "dna/2^28B/9-256 strings"
    assert autotune.config_class(8_000_000_000, 2000, dna) == "dna/2^33B/257+ strings"
    assert autotune.config_class(1 << 20, 1, text).startswith("bytes/2^20B/")


def test_tuned_uses_the_cache_and_records_new_classes(monkeypatch, tmp_path):
    calls = []
    monkeypatch.setattr(autotune, "autotune", lambda ctx, d, o, reps, sweeps: calls.append(1) or
                        {"tuning": dict(START, table_load=0.6), "ms": 5.0, "trials": [1, 2, 3]})
    path = str(tmp_path / "cache.json")
    ctx = FakeCtx(START)
    got = autotune.tuned(ctx, None, None, "dna/2^28B/9-256 strings", path=path)
    assert got["source"] == "tuned" and got["tuning"]["table_load"] == 0.6 and calls == [1]
    ctx2 = FakeCtx(START)
    got2 = autotune.tuned(ctx2, None, None, "dna/2^28B/9-256 strings", path=path)
    assert got2["source"] == "cache" and ctx2.tuning()["table_load"] == 0.6 and calls == [1]
    got3 = autotune.tuned(FakeCtx(START), None, None, "dna/2^28B/9-256 strings", path=path, retune=True)
    assert got3["source"] == "tuned" and calls == [1, 1]


def test_candidates_and_cache_name_tuning_fields():
    """Every searched parameter, and every parameter of every cached setting,
    is a field of lcg_tuning, with values the library accepts (the ranges of
    lcg_set_tuning, restated)."""
    import json
    from paper_2411_12439_gb300 import lcg
    fields = {f for f, _ in lcg.TuningC._fields_}
    assert set(autotune.CANDIDATES) <= fields
    ok = {"table_load": lambda v: 0.3 <= v <= 0.78, "parse_blocks_per_sm": lambda v: v >= 0,
          "miss_flush": lambda v: 32 <= v <= 256, "table_slots_max": lambda v: v == 0 or v >= 1024,
          "tile_stripes": lambda v: 1 <= v <= 16, "parse_tile": lambda v: v in (1024, 2048, 4096),
          "parse_tile_min": lambda v: 0 <= v <= 1024}
    assert set(ok) == fields
    for name, values in autotune.CANDIDATES.items():
        assert all(ok[name](v) for v in values), name
    with open(autotune.CACHE) as fh:
        cache = json.load(fh)
    assert cache
    for cls, entry in cache.items():
        assert set(entry["tuning"]) <= fields, cls
        assert all(ok[k](v) for k, v in entry["tuning"].items()), cls
