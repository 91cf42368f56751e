"""Python wrapper of the plain C oracle (``lcg_oracle.c``).

TEST INFRASTRUCTURE ONLY: the tests, the smoke check and the benchmark's CPU
baseline use it; the product path never imports it.

The oracle computes BuildGram / MergeGrams / exp(S) of the stable locally
consistent grammar method (Sec. 3.3, Sec. 3.6, Sec. 2.2) on the CPU, in plain
C with 128-bit products reduced by '%'.  Grammars are exported level by level:
``levels[i-1] = {"g", "rhs_off" (uint64, g+1), "rhs" (uint32), "F" (uint32)}``
plus ``F0`` (256 fingerprints of bytes) and ``C = (c_level, c_rank)``.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "lcg_oracle.c")
_LIB_DIR = os.path.join(_HERE, "_build")
_LIB = os.path.join(_LIB_DIR, "liblcg_oracle.so")
_lock = threading.Lock()
_lib = None

OG_OK, OG_EINVAL, OG_ENOMEM, OG_ELEVELS, OG_EMISMATCH = 0, -1, -2, -3, -4


def build_library(force: bool = False) -> str:
    """Compile the oracle with gcc into ``oracle/_build`` (no GPU needed)."""
    os.makedirs(_LIB_DIR, exist_ok=True)
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".{os.getpid()}.tmp"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-shared", "-fPIC", "-o", tmp, _SRC])
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        lib = ctypes.CDLL(build_library())
        P, U8, U32, U64 = ctypes.c_void_p, ctypes.c_uint8, ctypes.c_uint32, ctypes.c_uint64
        lib.og_build.argtypes = [P, P, U32, P, P, P, U32, U32, ctypes.POINTER(P)]
        lib.og_build.restype = ctypes.c_int
        lib.og_merge.argtypes = [P, P]
        lib.og_merge.restype = ctypes.c_int
        lib.og_decompress.argtypes = [P, U32, P, U64, ctypes.POINTER(U64)]
        lib.og_decompress.restype = ctypes.c_int
        lib.og_breaks.argtypes = [P, U64, P]
        lib.og_breaks.restype = ctypes.c_int
        lib.og_free.argtypes = [P]
        lib.og_free.restype = None
        for name, rt in [("og_nlevels", U32), ("og_k", U32), ("og_hash_tag", U64)]:
            getattr(lib, name).argtypes = [P]
            getattr(lib, name).restype = rt
        for name in ["og_level_g", "og_level_G"]:
            getattr(lib, name).argtypes = [P, U32]
            getattr(lib, name).restype = U64
        for name in ["og_level_rhs_off", "og_level_rhs", "og_level_F"]:
            getattr(lib, name).argtypes = [P, U32]
            getattr(lib, name).restype = P
        for name in ["og_F0", "og_c_level", "og_c_rank"]:
            getattr(lib, name).argtypes = [P]
            getattr(lib, name).restype = P
        lib.og_new.argtypes = [P, U64, U32, P, P]
        lib.og_new.restype = P
        lib.og_push_level.argtypes = [P, U64, P, P, P]
        lib.og_push_level.restype = ctypes.c_int
        lib.og_family_tag_of.argtypes = [P, P, P, U32, U32]
        lib.og_family_tag_of.restype = U64
        _lib = lib
        return lib


def _ptr(a: np.ndarray):
    return ctypes.c_void_p(a.ctypes.data) if a.size else ctypes.c_void_p(0)


def _copy(ptr, n, dtype):
    if n == 0:
        return np.zeros(0, dtype=dtype)
    buf = (ctypes.c_char * (n * np.dtype(dtype).itemsize)).from_address(ptr)
    return np.frombuffer(bytes(buf), dtype=dtype).copy()


class OracleError(RuntimeError):
    def __init__(self, rc):
        super().__init__(f"oracle returned {rc}")
        self.rc = rc


class Grammar:
    """Handle on an oracle grammar (owned by the C side)."""

    def __init__(self, handle):
        self._h = ctypes.c_void_p(handle) if not isinstance(handle, ctypes.c_void_p) else handle

    def __del__(self):
        if getattr(self, "_h", None) is not None and self._h.value and _lib is not None:
            _lib.og_free(self._h)
            self._h = None

    @property
    def k(self) -> int:
        return int(_load().og_k(self._h))

    @property
    def nlevels(self) -> int:
        return int(_load().og_nlevels(self._h))

    @property
    def hash_tag(self) -> int:
        return int(_load().og_hash_tag(self._h))

    def export(self) -> dict:
        lib = _load()
        levels = []
        for i in range(1, self.nlevels + 1):
            g = int(lib.og_level_g(self._h, i))
            G = int(lib.og_level_G(self._h, i))
            levels.append({
                "g": g,
                "rhs_off": _copy(lib.og_level_rhs_off(self._h, i), g + 1, np.uint64),
                "rhs": _copy(lib.og_level_rhs(self._h, i), G, np.uint32),
                "F": _copy(lib.og_level_F(self._h, i), g, np.uint32),
            })
        k = self.k
        return {
            "F0": _copy(lib.og_F0(self._h), 256, np.uint32),
            "levels": levels,
            "c_level": _copy(lib.og_c_level(self._h), k, np.uint32),
            "c_rank": _copy(lib.og_c_rank(self._h), k, np.uint32),
        }

    def decompress(self, j: int) -> bytes:
        lib = _load()
        out_len = ctypes.c_uint64(0)
        rc = lib.og_decompress(self._h, j, None, 0, ctypes.byref(out_len))
        n = out_len.value
        buf = np.zeros(max(n, 1), dtype=np.uint8)
        rc = lib.og_decompress(self._h, j, _ptr(buf), n, ctypes.byref(out_len))
        if rc != OG_OK:
            raise OracleError(rc)
        return buf[:n].tobytes()

    def merge(self, other: "Grammar") -> "Grammar":
        """In place: self absorbs other (MergeGrams(self, other))."""
        rc = _load().og_merge(self._h, other._h)
        if rc != OG_OK:
            raise OracleError(rc)
        return self

    def copy(self) -> "Grammar":
        return from_export(self.export(), self.hash_tag)


def build(coll, hf) -> Grammar:
    """BuildGram(T, H) of a ``lcg_inputs.Collection`` with hash family ``hf``."""
    lib = _load()
    data = np.ascontiguousarray(coll.data, dtype=np.uint8)
    off = np.ascontiguousarray(coll.offsets, dtype=np.uint64)
    a = np.ascontiguousarray(hf.a, dtype=np.uint64)
    b = np.ascontiguousarray(hf.b, dtype=np.uint64)
    c = np.ascontiguousarray(hf.c, dtype=np.uint64)
    h = ctypes.c_void_p(0)
    rc = lib.og_build(_ptr(data), _ptr(off), coll.k, _ptr(a), _ptr(b), _ptr(c), hf.levels, hf.m_bits,
                      ctypes.byref(h))
    if rc != OG_OK:
        raise OracleError(rc)
    return Grammar(h)


def build_parallel(coll, hf, threads: int) -> Grammar:
    """BuildGram over ``threads`` contiguous parts of the collection, one
    grammar per host thread, then MergeGrams of neighbouring parts in a tree
    until one grammar is left: the parallel construction of the paper's
    implementation (PBuildGram, appendix "Parallel grammar construction"),
    without its memory threshold.  Stability (Def. 1) and the merge of
    Sec. 3.6 make the result equal to ``build(coll, hf)``; the C calls release
    the interpreter lock, so the parts run on separate cores."""
    return build_parts(split(coll, threads), hf)


def split(coll, parts: int) -> list:
    """``parts`` contiguous, non-empty sub-collections, in string order."""
    parts = min(max(1, int(parts)), coll.k)
    cuts = [coll.k * t // parts for t in range(parts + 1)]
    return [coll.subset(range(cuts[t], cuts[t + 1])) for t in range(parts)]


def build_parts(subs: list, hf) -> Grammar:
    """BuildGram of each sub-collection on its own thread, then the tree of
    MergeGrams in order (see ``build_parallel``)."""
    from concurrent.futures import ThreadPoolExecutor
    _load()
    with ThreadPoolExecutor(len(subs)) as ex:
        gs = list(ex.map(lambda s: build(s, hf), subs))
        while len(gs) > 1:
            pairs = [(gs[t], gs[t + 1]) for t in range(0, len(gs) - 1, 2)]
            merged = list(ex.map(lambda ab: ab[0].merge(ab[1]), pairs))
            gs = merged + ([gs[-1]] if len(gs) % 2 else [])
    return gs[0]


def breaks(f) -> np.ndarray:
    """Phrase starts of one string given its fingerprint sequence (Eq. rand_types)."""
    lib = _load()
    f = np.ascontiguousarray(f, dtype=np.uint32)
    out = np.zeros(max(f.shape[0], 1), dtype=np.uint8)
    rc = lib.og_breaks(_ptr(f), f.shape[0], _ptr(out))
    if rc != OG_OK:
        raise OracleError(rc)
    return out[:f.shape[0]]


def family_tag(hf) -> int:
    lib = _load()
    a = np.ascontiguousarray(hf.a, dtype=np.uint64)
    b = np.ascontiguousarray(hf.b, dtype=np.uint64)
    c = np.ascontiguousarray(hf.c, dtype=np.uint64)
    return int(lib.og_family_tag_of(_ptr(a), _ptr(b), _ptr(c), hf.levels, hf.m_bits))


def from_export(ex: dict, tag: int) -> Grammar:
    """Grammar handle from exported arrays (hand-built fixtures, copies)."""
    lib = _load()
    F0 = np.ascontiguousarray(ex["F0"], dtype=np.uint32)
    cl = np.ascontiguousarray(ex["c_level"], dtype=np.uint32)
    cr = np.ascontiguousarray(ex["c_rank"], dtype=np.uint32)
    h = lib.og_new(_ptr(F0), tag, cl.shape[0], _ptr(cl), _ptr(cr))
    if not h:
        raise OracleError(OG_ENOMEM)
    G = Grammar(h)
    for L in ex["levels"]:
        ro = np.ascontiguousarray(L["rhs_off"], dtype=np.uint64)
        rhs = np.ascontiguousarray(L["rhs"], dtype=np.uint32)
        F = np.ascontiguousarray(L["F"], dtype=np.uint32)
        rc = lib.og_push_level(G._h, int(L["g"]), _ptr(ro), _ptr(rhs), _ptr(F))
        if rc != OG_OK:
            raise OracleError(rc)
    return G


def grammars_equal(x: dict, y: dict) -> bool:
    """Exact equality of two exported grammars."""
    if not np.array_equal(x["F0"], y["F0"]):
        return False
    if len(x["levels"]) != len(y["levels"]):
        return False
    for a, b in zip(x["levels"], y["levels"]):
        if a["g"] != b["g"]:
            return False
        for key in ("rhs_off", "rhs", "F"):
            if not np.array_equal(np.asarray(a[key]), np.asarray(b[key])):
                return False
    return np.array_equal(x["c_level"], y["c_level"]) and np.array_equal(x["c_rank"], y["c_rank"])
