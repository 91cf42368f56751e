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
