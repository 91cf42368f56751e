"""Failure detection on the GPU, in forms that fault, trap or hang nothing.

* A bounded wait that runs out: lcg_selftest_wait_timeout runs the library's
  single-pass scan with its tile counter read one ahead, so the first tile
  waits for a predecessor that never publishes.  The wait gives up after its
  iteration limit and the call must return LCG_ETIMEOUT; the same context
  must then build grammars equal to the oracle's.
* Phrase tables that overflow: with table_slots_max the first table of every
  round is too small for it, so rounds fill their table past the load limit,
  are regrown and rerun (and planned rounds are redone round by round, also
  in graph mode); every grammar must still equal the oracle's.
"""
import numpy as np
import pytest

import lcg_inputs as li
from oracle import oracle as O

pytestmark = pytest.mark.gpu

LCG_ETIMEOUT = -6


@pytest.fixture
def ctx(hf):
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2411_12439_gb300 import Context
    return Context(hf, device=0)


def _collections():
    rng = np.random.default_rng(31)
    return [li.tiny_dna_collection(base_len=120_000, k=4),
            li.from_strings([li.zipf_text(rng, 150_000), li.zipf_text(rng, 60_000, copy_frac=0.0)])]


def test_bounded_wait_times_out_and_the_context_recovers(ctx, hf):
    colls = _collections()
    want = [O.build(c, hf).export() for c in colls]
    assert ctx.selftest_wait_timeout() == LCG_ETIMEOUT
    for c, w in zip(colls, want):
        assert O.grammars_equal(ctx.build(c.data, c.offsets).export(), w)
    assert ctx.selftest_wait_timeout() == LCG_ETIMEOUT  # and again, after builds
    for c, w in zip(colls, want):  # planned rounds (no host sync) after the timeout
        assert O.grammars_equal(ctx.build(c.data, c.offsets).export(), w)


def test_forced_small_tables_regrow(ctx, hf):
    ctx.set_tuning(table_slots_max=1024)
    for c in _collections():
        want = O.build(c, hf).export()
        for _ in range(2):  # round by round, then planned (the plan's tables are capped too)
            g = ctx.build(c.data, c.offsets)
            st = ctx.last_build_stats()
            assert O.grammars_equal(g.export(), want)
            assert sum(r["retries"] for r in st["per_round"]) > 0, st
            g.free()
        assert st["redone"]  # the planned rounds overflowed and were redone round by round


def test_forced_small_tables_in_graph_mode(ctx, hf):
    import torch
    c = _collections()[0]
    want = O.build(c, hf).export()
    d = torch.from_numpy(c.data).cuda()
    ctx.build(d, c.offsets).free()  # a plan
    ctx.set_tuning(table_slots_max=1024)
    ctx.set_graph(True)
    try:
        for _ in range(3):
            g = ctx.build(d, c.offsets)
            assert O.grammars_equal(g.export(), want)
            g.free()
    finally:
        ctx.set_graph(False)
    ctx.set_tuning(table_slots_max=0)
    g = ctx.build(d, c.offsets)
    assert O.grammars_equal(g.export(), want)


def test_table_slots_max_range(ctx):
    from paper_2411_12439_gb300 import LCGError
    with pytest.raises(LCGError):
        ctx.set_tuning(table_slots_max=100)
    ctx.set_tuning(table_slots_max=0)
    assert ctx.tuning()["table_slots_max"] == 0
