"""lcg_decompress_static: expansion without device allocation.

Some callers cannot allocate device memory when they expand a string: code
inside an allocator's or a memory-pressure callback (it cannot call back into
the allocator) and services that reserve their device memory up front.
lcg_decompress_static serves them from a static scratch array inside the
library.  These tests call it through the C ABI and check it against
lcg_decompress, twice in a row (the scratch keeps the previous call's
contents), check that the device's memory pool (which the library allocates
from) and torch's allocator hold no more memory after a call, and check that
an over-long string is rejected.  This file is collected last on purpose.
"""
import ctypes
import ctypes.util
import glob
import os

import numpy as np
import pytest

import lcg_inputs as li

pytestmark = pytest.mark.gpu


def _cudart():
    """The CUDA runtime as a shared library (to read the memory pool's use)."""
    import torch
    cands = [ctypes.util.find_library("cudart")]
    tdir = os.path.dirname(torch.__file__)
    cands += sorted(glob.glob(os.path.join(tdir, "lib", "libcudart.so*")))
    cands += sorted(glob.glob(os.path.join(os.path.dirname(tdir), "nvidia", "*", "lib", "libcudart.so*")))
    cands += sorted(glob.glob("/usr/local/cuda/lib64/libcudart.so*"))
    for c in cands:
        if not c:
            continue
        try:
            return ctypes.CDLL(c)
        except OSError:
            continue
    pytest.fail("no CUDA runtime library found to read the memory pool")


def _pool_used(rt, device=0):
    """Bytes in use in the device's current memory pool (cudaMallocAsync's)."""
    import torch
    torch.cuda.synchronize()
    pool = ctypes.c_void_p()
    assert rt.cudaDeviceGetMemPool(ctypes.byref(pool), ctypes.c_int(device)) == 0
    used = ctypes.c_uint64()
    attr_used_mem_current = 7  # cudaMemPoolAttrUsedMemCurrent
    assert rt.cudaMemPoolGetAttribute(pool, ctypes.c_int(attr_used_mem_current), ctypes.byref(used)) == 0
    return used.value


@pytest.fixture(scope="module")
def built(hf):
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2411_12439_gb300 import Context
    ctx = Context(hf, device=0)
    rng = np.random.default_rng(33)
    strings = [li.random_dna(rng, 300_000).tobytes(), b"A", li.zipf_text(rng, 70_000).tobytes(),
               li.random_dna(rng, 1 << 20).tobytes(), li.random_dna(rng, (1 << 20) + 1).tobytes(), b"ACGT" * 5000]
    coll = li.from_strings(strings)
    return ctx, ctx.build(coll.data, coll.offsets), coll


def test_static_matches_regular_twice_in_a_row(built):
    import torch
    ctx, g, coll = built
    rt = _cudart()
    for j in (0, 2, 3, 1, 5, 0):
        n = int(coll.offsets[j + 1] - coll.offsets[j])
        want = torch.zeros(n, dtype=torch.uint8, device="cuda:0")
        assert g.decompress(j, want) == n
        for _ in range(2):
            got = torch.full((n,), 7, dtype=torch.uint8, device="cuda:0")
            pool0, torch0 = _pool_used(rt), torch.cuda.memory_allocated()
            assert g.decompress_static(j, got) == n
            assert _pool_used(rt) == pool0 and torch.cuda.memory_allocated() == torch0  # nothing allocated
            assert torch.equal(got, want)
        assert bytes(want.cpu().numpy()) == coll.string(j).tobytes()


def test_static_rejects_strings_beyond_its_scratch(built):
    import torch
    from paper_2411_12439_gb300 import LCGError
    ctx, g, coll = built
    n = int(coll.offsets[5] - coll.offsets[4])
    out = torch.zeros(n, dtype=torch.uint8, device="cuda:0")
    with pytest.raises(LCGError) as e:
        g.decompress_static(4, out)
    assert e.value.code == -5  # LCG_EOVERFLOW
    # a call after the rejection still works
    m = int(coll.offsets[1] - coll.offsets[0])
    a = torch.zeros(m, dtype=torch.uint8, device="cuda:0")
    b = torch.zeros(m, dtype=torch.uint8, device="cuda:0")
    g.decompress(0, a)
    g.decompress_static(0, b)
    assert torch.equal(a, b)
