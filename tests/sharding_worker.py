"""Child process of the sharding tests: one gloo rank on the CPU.

The rank builds its part of the collection with the CPU oracle (standing in
for a GPU's lcg_build), then takes part in the merge tree over torch.distributed
(gloo).  Rank 0 writes the packed result to ``out``.  Failure injection: a rank
listed in ``fail_ranks`` raises before the exchange (a rank that dies between
steps)."""
import os
import sys

import numpy as np


class OracleBackend:
    """The oracle's grammar operations; the exchange in the packed form, or
    (form="vbyte") in the VByte form."""

    def __init__(self, hf, form="packed"):
        from oracle import oracle as O
        self.O = O
        self.hf = hf
        self.tag = O.family_tag(hf)
        self.form = form

    def build(self, data, offsets):
        import lcg_inputs as li
        coll = li.Collection(data=np.ascontiguousarray(data, dtype=np.uint8),
                             offsets=np.ascontiguousarray(offsets, dtype=np.uint64))
        return self.O.build(coll, self.hf)

    def pack(self, g):
        if self.form == "vbyte":
            from oracle import vbyte
            return np.frombuffer(vbyte.export_vbyte(g.export()), dtype=np.uint8).copy()
        from paper_2411_12439_gb300 import sharding
        return sharding.pack(g.export())

    def unpack(self, buf):
        if self.form == "vbyte":
            from oracle import vbyte
            return self.O.from_export(vbyte.import_vbyte(np.asarray(buf, dtype=np.uint8).tobytes()), self.tag)
        from paper_2411_12439_gb300 import sharding
        return self.O.from_export(sharding.unpack(buf), self.tag)

    def merge(self, a, b):
        return a.merge(b)


def run(rank, world, port, strings, out, fail_ranks=(), timeout_s=60, form="packed"):
    import datetime

    import torch.distributed as dist

    import lcg_inputs as li
    from paper_2411_12439_gb300 import sharding

    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world, timeout=datetime.timedelta(seconds=timeout_s))
    try:
        coll = li.from_strings(strings)
        if rank in fail_ranks:
            raise RuntimeError(f"rank {rank} stops before the exchange")
        g = sharding.build_sharded(coll.data, coll.offsets, rank, world, OracleBackend(li.hash_family(), form),
                                   sharding.TorchComm())
        if rank == 0:
            np.save(out, sharding.pack(g.export()))
    finally:
        if rank not in fail_ranks:
            dist.destroy_process_group()


if __name__ == "__main__":
    sys.exit(0)
