"""Writes ``config_digests.json``: digests of the oracle's grammar of the two
largest seeded collections, which are too large to store or to rebuild with
the oracle inside a GPU test.

* ``uneven``: the uneven batch, 2000 strings of 0.5-12 Mbp (about 8 GB);
* ``repetitive``: 4 strings of 3.1 Gbp over ACGTN with repeat families and
  N-runs (12.4 GB).

Each grammar is BuildGram of the whole collection by the plain oracle
(``oracle.build``, one thread), digested level by level with
``tests/digests.py``.  The script calls only ``oracle/`` and the seeded
generators (``lcg_inputs``); it needs about 45 GB of host memory and some
minutes per collection.

    python tests/golden/make_config_digests.py [--out PATH] [uneven] [repetitive]

(``--out`` writes the digests to PATH instead of this folder's file, which
the GPU test reads.)
"""
from __future__ import annotations

import json
import os
import sys
import time

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)
sys.path.insert(0, os.path.dirname(HERE))

import lcg_inputs as li  # noqa: E402
from oracle import oracle as O  # noqa: E402
from digests import grammar_digests  # noqa: E402

OUT = os.path.join(HERE, "config_digests.json")

COLLECTIONS = {
    "uneven": li.uneven_collection,
    "repetitive": li.repetitive_collection,
}


def main(names):
    hf = li.hash_family()
    out = json.load(open(OUT)) if os.path.exists(OUT) else {}
    for name in names:
        t0 = time.time()
        coll = COLLECTIONS[name]()
        t1 = time.time()
        g = O.build(coll, hf)
        t2 = time.time()
        d = grammar_digests(g.export())
        d["n"] = int(coll.n)
        d["generator"] = f"lcg_inputs.{COLLECTIONS[name].__name__}() with its default arguments"
        d["hash_family"] = "lcg_inputs.hash_family() (default seed, 64 levels, m_bits 32)"
        out[name] = d
        del g
        print(f"{name}: n={coll.n} levels={len(d['levels'])} generate {t1 - t0:.0f}s oracle {t2 - t1:.0f}s",
              flush=True)
        with open(OUT, "w") as f:
            json.dump(out, f, indent=1, sort_keys=True)
            f.write("\n")


if __name__ == "__main__":
    argv = sys.argv[1:]
    if argv[:1] == ["--out"]:
        OUT = argv[1]
        argv = argv[2:]
    main(argv or list(COLLECTIONS))
