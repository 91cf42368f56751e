"""lcg_import and the sharded build on one GPU, through the C ABI.

A grammar exported to host arrays and imported again must be the same
grammar; a grammar of another hash family or with malformed arrays must be
refused.  The merge tree of the sharded build is run in one process with the
CUDA backend (the ranks in sequence), and must give the oracle's BuildGram of
the whole collection."""
import numpy as np
import pytest

import lcg_inputs as li
from oracle import oracle as O

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx(hf):
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2411_12439_gb300 import Context
    return Context(hf, device=0)


def test_import_roundtrip(ctx, hf):
    coll = li.tiny_dna_collection(base_len=50_000, k=4)
    want = O.build(coll, hf).export()
    g = ctx.import_grammar(want)
    assert O.grammars_equal(g.export(), want)
    for j in range(coll.k):
        assert g.decompress(j) == coll.string(j).tobytes()
    # an imported grammar takes part in merges and resident builds like a built one
    more = li.tiny_dna_collection(base_len=50_000, k=6).subset([4, 5])
    ctx.build_into(g, more.data, more.offsets)
    both = li.from_strings([coll.string(j) for j in range(coll.k)] + [more.string(j) for j in range(more.k)])
    assert O.grammars_equal(g.export(), O.build(both, hf).export())


def test_import_rejects_other_family_and_malformed(ctx, hf):
    from paper_2411_12439_gb300 import LCGError
    coll = li.tiny_dna_collection(base_len=5_000, k=2)
    other = O.build(coll, li.hash_family(seed=12345)).export()
    with pytest.raises(LCGError) as e:
        ctx.import_grammar(other)
    assert e.value.code == -4  # LCG_EMISMATCH
    ex = O.build(coll, hf).export()
    bad = {**ex, "c_rank": ex["c_rank"].copy()}
    bad["c_rank"][0] = ex["levels"][int(ex["c_level"][0]) - 1]["g"]  # one past the last rule
    with pytest.raises(LCGError) as e:
        ctx.import_grammar(bad)
    assert e.value.code == -1  # LCG_EINVAL
    lv = [dict(L) for L in ex["levels"]]
    lv[1] = {**lv[1], "rhs": lv[1]["rhs"].copy()}
    lv[1]["rhs"][0] = ex["levels"][0]["g"]  # a symbol outside level 1
    with pytest.raises(LCGError) as e:
        ctx.import_grammar({**ex, "levels": lv})
    assert e.value.code == -1
    # the context still works after refused calls
    assert O.grammars_equal(ctx.import_grammar(ex).export(), ex)


class _LocalComm:
    def __init__(self, boxes, rank):
        self.boxes, self.rank = boxes, rank

    def send(self, buf, dst):
        self.boxes[(self.rank, dst)] = buf

    def recv(self, src):
        return self.boxes.pop((src, self.rank))


@pytest.mark.parametrize("world,form", [(2, "packed"), (3, "packed"), (4, "packed"), (3, "vbyte"), (4, "vbyte")])
def test_sharded_build_merge_tree(ctx, hf, world, form):
    from paper_2411_12439_gb300 import sharding
    coll = li.tiny_dna_collection(base_len=120_000, k=7)
    backend = sharding.CudaBackend(ctx, form=form)
    boxes, out = {}, {}
    for rank in reversed(range(world)):
        out[rank] = sharding.build_sharded(coll.data, coll.offsets, rank, world, backend, _LocalComm(boxes, rank))
    assert not boxes
    assert O.grammars_equal(out[0].export(), O.build(coll, hf).export())


def test_packed_form_matches_oracle_and_roundtrips(ctx, hf):
    from paper_2411_12439_gb300 import LCGError, sharding
    coll = li.tiny_dna_collection(base_len=60_000, k=5)
    og = O.build(coll, hf)
    g = ctx.build(coll.data, coll.offsets)
    buf = np.asarray(g.export_packed())
    assert buf.size == g.packed_size()
    assert np.array_equal(buf, sharding.pack(og.export()))  # same bytes as the layout written out in Python
    back = ctx.import_packed(buf)
    assert O.grammars_equal(back.export(), og.export())
    with pytest.raises(LCGError) as e:
        ctx.import_packed(buf[:-8].copy())
    assert e.value.code == -1
    other = sharding.pack(O.build(coll, li.hash_family(seed=777)).export())
    with pytest.raises(LCGError) as e:
        ctx.import_packed(other)
    assert e.value.code == -4
    # into a caller's (page-locked) buffer
    import torch
    pinned = torch.empty(buf.size + 64, dtype=torch.uint8).pin_memory()
    view = g.export_packed(pinned)
    assert np.array_equal(view.numpy(), buf)


def test_tuning_changes_speed_not_results(hf):
    """Builds under other launch and sizing parameters give the same grammar;
    out-of-range parameters are refused; the autotuner leaves a valid setting."""
    torch = pytest.importorskip("torch")
    from paper_2411_12439_gb300 import Context, LCGError, autotune
    ctx = Context(hf, device=0)
    coll = li.tiny_dna_collection(base_len=150_000, k=5)
    text = li.from_strings([li.zipf_text(np.random.default_rng(9), 120_000)])
    want = {id(c): O.build(c, hf).export() for c in (coll, text)}
    for tun in ({"table_load": 0.3, "parse_blocks_per_sm": 1, "miss_flush": 32, "table_slots_max": 0,
                 "tile_stripes": 4, "parse_tile": 1024, "parse_tile_min": 0},
                {"table_load": 0.78, "parse_blocks_per_sm": 2, "miss_flush": 256, "table_slots_max": 0,
                 "tile_stripes": 3, "parse_tile": 4096, "parse_tile_min": 0},
                {"table_load": 0.5, "parse_blocks_per_sm": 0, "miss_flush": 64, "table_slots_max": 4096,
                 "tile_stripes": 16, "parse_tile": 2048, "parse_tile_min": 1024},
                {"table_load": 0.35, "parse_blocks_per_sm": 0, "miss_flush": 64, "table_slots_max": 0,
                 "tile_stripes": 1, "parse_tile": 4096, "parse_tile_min": 16}):
        ctx.set_tuning(**tun)
        assert ctx.tuning() == tun
        for c in (coll, text, coll):
            assert O.grammars_equal(ctx.build(c.data, c.offsets).export(), want[id(c)])
    for bad in ({"table_load": 0.9}, {"miss_flush": 8}, {"parse_blocks_per_sm": 999}, {"tile_stripes": 0},
                {"tile_stripes": 17}, {"parse_tile": 3072}, {"parse_tile": 8192},
                {"parse_tile_min": 1025}):
        with pytest.raises(LCGError) as e:
            ctx.set_tuning(**bad)
        assert e.value.code == -1
    d = torch.from_numpy(coll.data).cuda()
    rep = autotune.autotune(ctx, d, coll.offsets, reps=2, sweeps=1)
    assert rep["tuning"] == ctx.tuning() and rep["ms"] > 0 and len(rep["trials"]) > 3
    assert O.grammars_equal(ctx.build(d, coll.offsets).export(), want[id(coll)])
