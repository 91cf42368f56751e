"""Thin Python binding of the C ABI in ``include/lcg.h`` (argument marshalling only).

Every operation runs in the CUDA library ``liblcg_gb300.so``.  There is no
fallback: if the library is missing or no CUDA device is usable, the calls
raise ``LCGError``.

Inputs are either host arrays (numpy, bytes) or CUDA tensors (torch.uint8 on
the context's device); offsets are always host uint64 arrays of k+1 entries.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

from . import build as _build

LCG_OK = 0
_ERRORS = {
    -1: "LCG_EINVAL", -2: "LCG_ENOMEM", -3: "LCG_ELEVELS", -4: "LCG_EMISMATCH",
    -5: "LCG_EOVERFLOW", -6: "LCG_ETIMEOUT", -7: "LCG_EDEVICE", -8: "LCG_ETABLE",
}
SYMBOLS = [
    "lcg_ctx_create", "lcg_ctx_destroy", "lcg_last_error", "lcg_last_build_stats", "lcg_set_kernel_timing",
    "lcg_set_tuning", "lcg_get_tuning", "lcg_set_graph",
    "lcg_last_kernel_times", "lcg_build", "lcg_build_into",
    "lcg_merge", "lcg_decompress", "lcg_decompress_static", "lcg_grammar_shape", "lcg_level_size", "lcg_export_level",
    "lcg_export_start", "lcg_string_roots", "lcg_import", "lcg_packed_size", "lcg_export_packed", "lcg_import_packed",
    "lcg_grammar_free", "lcg_postprocess", "lcg_pp_stats_of", "lcg_pp_export", "lcg_pp_free",
    "lcg_vbyte_encode", "lcg_vbyte_decode", "lcg_vbyte_size", "lcg_export_vbyte", "lcg_import_vbyte",
    "lcg_last_kernel_launches", "lcg_selftest_wait_timeout",
]


class LCGError(RuntimeError):
    def __init__(self, code, msg=""):
        super().__init__(f"{_ERRORS.get(code, code)}: {msg}")
        self.code = code


class HashFamilyC(ctypes.Structure):
    _fields_ = [("levels", ctypes.c_uint32), ("m_bits", ctypes.c_uint32), ("a", ctypes.c_void_p),
                ("b", ctypes.c_void_p), ("c", ctypes.c_void_p)]


class RoundStatsC(ctypes.Structure):
    _fields_ = [("n", ctypes.c_uint64), ("phrases", ctypes.c_uint64), ("g", ctypes.c_uint64),
                ("G", ctypes.c_uint64), ("strings", ctypes.c_uint64), ("table_cap", ctypes.c_uint64),
                ("retries", ctypes.c_uint32), ("pad", ctypes.c_uint32), ("parse_ms", ctypes.c_double),
                ("round_ms", ctypes.c_double)]


class KernelTimeC(ctypes.Structure):
    _fields_ = [("name", ctypes.c_char * 24), ("launches", ctypes.c_uint32), ("pad", ctypes.c_uint32),
                ("ms", ctypes.c_double), ("bytes", ctypes.c_double)]


class KernelLaunchC(ctypes.Structure):
    _fields_ = [("name", ctypes.c_char * 24), ("round", ctypes.c_uint32), ("pad", ctypes.c_uint32),
                ("ms", ctypes.c_double), ("bytes", ctypes.c_double)]


class TuningC(ctypes.Structure):
    _fields_ = [("table_load", ctypes.c_double), ("parse_blocks_per_sm", ctypes.c_uint32),
                ("miss_flush", ctypes.c_uint32), ("table_slots_max", ctypes.c_uint32),
                ("tile_stripes", ctypes.c_uint32), ("parse_tile", ctypes.c_uint32), ("parse_tile_min", ctypes.c_uint32)]


class PPStatsC(ctypes.Structure):
    _fields_ = [(f, ctypes.c_uint64)
                for f in ("size_before", "size_rl", "size", "rl_rules", "removed", "rules", "strings")]


class BuildStatsC(ctypes.Structure):
    _fields_ = [("rounds", ctypes.c_uint32), ("async_rounds", ctypes.c_uint32), ("kernel_launches", ctypes.c_uint64),
                ("input_bytes", ctypes.c_uint64), ("redone", ctypes.c_uint32), ("graph", ctypes.c_uint32),
                ("round", RoundStatsC * 64), ("plan_slack", ctypes.c_double)]


_lib = None


def library_path() -> str:
    return _build.LIB


def load(build_if_missing: bool = True):
    """Load liblcg_gb300.so (building it first when it is missing or stale)."""
    global _lib
    if _lib is not None:
        return _lib
    if build_if_missing and not _build.up_to_date():
        _build.build()
    if not os.path.exists(_build.LIB):
        raise LCGError(-7, f"CUDA library not built: {_build.LIB}")
    lib = ctypes.CDLL(_build.LIB)
    P, U32, U64, I = ctypes.c_void_p, ctypes.c_uint32, ctypes.c_uint64, ctypes.c_int
    PP = ctypes.POINTER(ctypes.c_void_p)
    lib.lcg_ctx_create.argtypes = [I, ctypes.POINTER(HashFamilyC), P, PP]
    lib.lcg_ctx_destroy.argtypes = [P]
    lib.lcg_ctx_destroy.restype = None
    lib.lcg_last_error.argtypes = [P]
    lib.lcg_last_error.restype = ctypes.c_char_p
    lib.lcg_last_build_stats.argtypes = [P, ctypes.POINTER(BuildStatsC)]
    lib.lcg_set_kernel_timing.argtypes = [P, I]
    lib.lcg_set_tuning.argtypes = [P, ctypes.POINTER(TuningC)]
    lib.lcg_get_tuning.argtypes = [P, ctypes.POINTER(TuningC)]
    lib.lcg_set_graph.argtypes = [P, I]
    lib.lcg_last_kernel_times.argtypes = [P, P, U32, ctypes.POINTER(U32)]
    lib.lcg_last_kernel_launches.argtypes = [P, P, U32, ctypes.POINTER(U32)]
    lib.lcg_selftest_wait_timeout.argtypes = [P]
    lib.lcg_build.argtypes = [P, P, P, U32, I, PP]
    lib.lcg_build_into.argtypes = [P, P, P, P, U32, I]
    lib.lcg_merge.argtypes = [P, P, P]
    lib.lcg_decompress.argtypes = [P, P, U32, P, U64, ctypes.POINTER(U64), I]
    lib.lcg_decompress_static.argtypes = [P, P, U32, P, U64, ctypes.POINTER(U64)]
    lib.lcg_grammar_shape.argtypes = [P, ctypes.POINTER(U32), ctypes.POINTER(U32)]
    lib.lcg_level_size.argtypes = [P, U32, ctypes.POINTER(U64), ctypes.POINTER(U64)]
    lib.lcg_export_level.argtypes = [P, P, U32, P, P, P]
    lib.lcg_export_start.argtypes = [P, P, P, P, P]
    lib.lcg_string_roots.argtypes = [P, P, U32, U32, P, P, P]
    lib.lcg_import.argtypes = [P, U32, U32, P, P, P, P, P, P, PP]
    lib.lcg_packed_size.argtypes = [P, ctypes.POINTER(U64)]
    lib.lcg_export_packed.argtypes = [P, P, P, U64]
    lib.lcg_import_packed.argtypes = [P, P, U64, PP]
    lib.lcg_grammar_free.argtypes = [P]
    lib.lcg_postprocess.argtypes = [P, P, PP]
    lib.lcg_pp_stats_of.argtypes = [P, ctypes.POINTER(PPStatsC)]
    lib.lcg_pp_export.argtypes = [P, P, P, P, P]
    lib.lcg_pp_free.argtypes = [P]
    lib.lcg_vbyte_encode.argtypes = [P, P, U64, P, U64, ctypes.POINTER(U64)]
    lib.lcg_vbyte_decode.argtypes = [P, P, U64, P, U64]
    lib.lcg_vbyte_size.argtypes = [P, P, ctypes.POINTER(U64)]
    lib.lcg_export_vbyte.argtypes = [P, P, P, U64, I, ctypes.POINTER(U64)]
    lib.lcg_import_vbyte.argtypes = [P, P, U64, I, PP]
    lib.lcg_pp_free.restype = None
    lib.lcg_grammar_free.restype = None
    for name in SYMBOLS:
        if name not in ("lcg_ctx_destroy", "lcg_last_error", "lcg_grammar_free", "lcg_pp_free"):
            getattr(lib, name).restype = I
    _lib = lib
    return lib


def _np_ptr(a: np.ndarray):
    return ctypes.c_void_p(a.ctypes.data) if a.size else ctypes.c_void_p(0)


def _data_arg(data):
    """(pointer, on_device, keepalive) of a uint8 host array or CUDA tensor."""
    try:
        import torch
        if isinstance(data, torch.Tensor):
            if data.dtype != torch.uint8 or not data.is_contiguous():
                raise LCGError(-1, "data must be a contiguous uint8 tensor")
            return ctypes.c_void_p(data.data_ptr()), int(data.is_cuda), data
    except ImportError:
        pass
    if isinstance(data, (bytes, bytearray)):
        data = np.frombuffer(data, dtype=np.uint8)
    arr = np.ascontiguousarray(data, dtype=np.uint8)
    return _np_ptr(arr), 0, arr


class Context:
    """A device, a stream and a hash family (``lcg_ctx``)."""

    def __init__(self, hash_family, device: int = 0, stream=None):
        lib = load()
        self._keep = [np.ascontiguousarray(x, dtype=np.uint64) for x in (hash_family.a, hash_family.b, hash_family.c)]
        hfc = HashFamilyC(int(hash_family.levels), int(hash_family.m_bits), *[_np_ptr(x) for x in self._keep])
        h = ctypes.c_void_p(0)
        st = ctypes.c_void_p(stream) if stream is not None else ctypes.c_void_p(0)
        rc = lib.lcg_ctx_create(int(device), ctypes.byref(hfc), st, ctypes.byref(h))
        if rc != LCG_OK:
            raise LCGError(rc, "lcg_ctx_create failed")
        self._h = h
        self.device = device

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            load().lcg_ctx_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _check(self, rc):
        if rc != LCG_OK:
            msg = load().lcg_last_error(self._h)
            raise LCGError(rc, msg.decode() if msg else "")

    def build(self, data, offsets) -> "Grammar":
        """lcg_build: BuildGram over the strings data[offsets[j]:offsets[j+1]]."""
        ptr, on_dev, keep = _data_arg(data)
        off = np.ascontiguousarray(offsets, dtype=np.uint64)
        h = ctypes.c_void_p(0)
        self._check(load().lcg_build(self._h, ptr, _np_ptr(off), off.shape[0] - 1, on_dev, ctypes.byref(h)))
        del keep
        return Grammar(self, h)

    def build_into(self, grammar: "Grammar", data, offsets) -> None:
        """lcg_build_into: parse against (and extend) a resident grammar."""
        ptr, on_dev, keep = _data_arg(data)
        off = np.ascontiguousarray(offsets, dtype=np.uint64)
        self._check(load().lcg_build_into(self._h, grammar._h, ptr, _np_ptr(off), off.shape[0] - 1, on_dev))
        del keep

    def merge(self, a: "Grammar", b: "Grammar") -> "Grammar":
        """lcg_merge: a absorbs b (in place); returns a."""
        self._check(load().lcg_merge(self._h, a._h, b._h))
        return a

    def postprocess(self, g: "Grammar") -> "PPGrammar":
        """lcg_postprocess: run-length rules, then simplification, of g (g is
        unchanged); a new device-resident grammar over global ids."""
        h = ctypes.c_void_p(0)
        self._check(load().lcg_postprocess(self._h, g._h, ctypes.byref(h)))
        return PPGrammar(h)

    def import_grammar(self, ex: dict) -> "Grammar":
        """lcg_import: a device grammar from the host arrays of ``Grammar.export()``
        (for example one received from another process)."""
        levels = ex["levels"]
        nl = len(levels)
        g = np.array([int(L["g"]) for L in levels] or [0], dtype=np.uint64)
        keep = []

        def arr(x, dt):
            a = np.ascontiguousarray(x, dtype=dt)
            if a.size == 0:
                a = np.zeros(1, dtype=dt)
            keep.append(a)
            return a.ctypes.data

        ro = (ctypes.c_void_p * max(nl, 1))(*[arr(L["rhs_off"], np.uint64) for L in levels])
        rhs = (ctypes.c_void_p * max(nl, 1))(*[arr(L["rhs"], np.uint32) for L in levels])
        F = (ctypes.c_void_p * max(nl, 1))(*[arr(L["F"], np.uint32) for L in levels])
        cl = np.ascontiguousarray(ex["c_level"], dtype=np.uint32)
        cr = np.ascontiguousarray(ex["c_rank"], dtype=np.uint32)
        k = int(cl.shape[0])
        if k == 0:
            cl = np.zeros(1, dtype=np.uint32)
            cr = np.zeros(1, dtype=np.uint32)
        h = ctypes.c_void_p(0)
        self._check(load().lcg_import(self._h, k, nl, _np_ptr(g), ctypes.cast(ro, ctypes.c_void_p),
                                      ctypes.cast(rhs, ctypes.c_void_p), ctypes.cast(F, ctypes.c_void_p),
                                      _np_ptr(cl), _np_ptr(cr), ctypes.byref(h)))
        del keep
        return Grammar(self, h)

    def import_packed(self, buf) -> "Grammar":
        """lcg_import_packed: a device grammar from its packed form (a uint8
        numpy array or a CPU uint8 tensor, 8-byte aligned)."""
        ptr, on_dev, keep = _data_arg(buf)
        if on_dev:
            raise LCGError(-1, "lcg_import_packed reads host memory")
        n = int(buf.numel() if hasattr(buf, "numel") else buf.size)
        h = ctypes.c_void_p(0)
        self._check(load().lcg_import_packed(self._h, ptr, n, ctypes.byref(h)))
        del keep
        return Grammar(self, h)

    def import_vbyte(self, buf) -> "Grammar":
        """lcg_import_vbyte: a device grammar from its VByte form (a uint8 numpy
        array, or a CPU or CUDA uint8 tensor; 8-byte aligned)."""
        ptr, on_dev, keep = _data_arg(buf)
        n = int(buf.numel() if hasattr(buf, "numel") else len(buf))
        h = ctypes.c_void_p(0)
        self._check(load().lcg_import_vbyte(self._h, ptr, n, on_dev, ctypes.byref(h)))
        del keep
        return Grammar(self, h)

    def vbyte_encode(self, values, out=None):
        """lcg_vbyte_encode: the VByte stream of a CUDA int32/uint32 tensor
        (values read as unsigned 32-bit) as a CUDA uint8 tensor (a view of
        ``out`` when given)."""
        import torch
        if not values.is_cuda or values.dtype not in (torch.int32, torch.uint32) or not values.is_contiguous():
            raise LCGError(-1, "values must be a contiguous 32-bit CUDA tensor")
        n = values.numel()
        if out is None:
            out = torch.empty(max(5 * n, 1), dtype=torch.uint8, device=values.device)
        ptr, on_dev, keep = _data_arg(out)
        if not on_dev:
            raise LCGError(-1, "lcg_vbyte_encode writes device memory")
        nb = ctypes.c_uint64(0)
        self._check(load().lcg_vbyte_encode(self._h, ctypes.c_void_p(values.data_ptr()), n, ptr, out.numel(),
                                            ctypes.byref(nb)))
        return out[:int(nb.value)]

    def vbyte_decode(self, stream, n: int, out=None):
        """lcg_vbyte_decode: ``n`` values of a VByte stream (a CUDA uint8
        tensor) as a CUDA int32 tensor holding the unsigned 32-bit values."""
        import torch
        ptr, on_dev, keep = _data_arg(stream)
        if not on_dev:
            raise LCGError(-1, "lcg_vbyte_decode reads device memory")
        if out is None:
            out = torch.empty(max(n, 1), dtype=torch.int32, device=stream.device)
        self._check(load().lcg_vbyte_decode(self._h, ptr, stream.numel(), ctypes.c_void_p(out.data_ptr()), n))
        return out[:n]

    def tuning(self) -> dict:
        """lcg_get_tuning: the launch and sizing parameters of later builds."""
        t = TuningC()
        self._check(load().lcg_get_tuning(self._h, ctypes.byref(t)))
        return {"table_load": float(t.table_load), "parse_blocks_per_sm": int(t.parse_blocks_per_sm),
                "miss_flush": int(t.miss_flush), "table_slots_max": int(t.table_slots_max),
                "tile_stripes": int(t.tile_stripes), "parse_tile": int(t.parse_tile),
                "parse_tile_min": int(t.parse_tile_min)}

    def set_tuning(self, **kw) -> None:
        """lcg_set_tuning: change some of table_load, parse_blocks_per_sm,
        miss_flush, table_slots_max, tile_stripes, parse_tile, parse_tile_min
        (the others keep their values)."""
        cur = self.tuning()
        unknown = set(kw) - set(cur)
        if unknown:
            raise LCGError(-1, f"unknown tuning parameters {sorted(unknown)}")
        cur.update(kw)
        t = TuningC(float(cur["table_load"]), int(cur["parse_blocks_per_sm"]), int(cur["miss_flush"]),
                    int(cur["table_slots_max"]), int(cur["tile_stripes"]), int(cur["parse_tile"]),
                    int(cur["parse_tile_min"]))
        self._check(load().lcg_set_tuning(self._h, ctypes.byref(t)))

    def set_graph(self, enable: bool) -> None:
        """lcg_set_graph: run later builds of a repeated shape as one captured
        CUDA graph."""
        self._check(load().lcg_set_graph(self._h, int(bool(enable))))

    def set_kernel_timing(self, mode) -> None:
        """lcg_set_kernel_timing: 0/False off, 1/True every kernel launch,
        2 only the parse launches."""
        self._check(load().lcg_set_kernel_timing(self._h, int(mode)))

    def last_kernel_times(self) -> dict:
        """lcg_last_kernel_times: {kind: {"launches", "ms", "bytes"}} of the last call."""
        cnt = ctypes.c_uint32(0)
        buf = (KernelTimeC * 32)()
        self._check(load().lcg_last_kernel_times(self._h, ctypes.cast(buf, ctypes.c_void_p), 32, ctypes.byref(cnt)))
        return {buf[i].name.decode(): {"launches": int(buf[i].launches), "ms": float(buf[i].ms),
                                       "bytes": float(buf[i].bytes)} for i in range(min(cnt.value, 32))}

    def last_kernel_launches(self) -> list:
        """lcg_last_kernel_launches: [{"name", "round", "ms", "bytes"}] of the
        last call's timed launches, in launch order."""
        lib = load()
        cnt = ctypes.c_uint32(0)
        self._check(lib.lcg_last_kernel_launches(self._h, None, 0, ctypes.byref(cnt)))
        n = cnt.value
        buf = (KernelLaunchC * max(n, 1))()
        self._check(lib.lcg_last_kernel_launches(self._h, ctypes.cast(buf, ctypes.c_void_p), n, ctypes.byref(cnt)))
        return [{"name": buf[i].name.decode(), "round": int(buf[i].round), "ms": float(buf[i].ms),
                 "bytes": float(buf[i].bytes)} for i in range(min(n, cnt.value))]

    def selftest_wait_timeout(self) -> int:
        """lcg_selftest_wait_timeout: the return code (LCG_ETIMEOUT, -6, when
        the bounded wait works)."""
        return int(load().lcg_selftest_wait_timeout(self._h))

    def last_build_stats(self) -> dict:
        st = BuildStatsC()
        self._check(load().lcg_last_build_stats(self._h, ctypes.byref(st)))
        rounds = [{**{f: int(getattr(st.round[i], f)) for f in ("n", "phrases", "g", "G", "strings", "table_cap",
                                                                "retries")}, "parse_ms": float(st.round[i].parse_ms),
                   "round_ms": float(st.round[i].round_ms)}
                  for i in range(min(st.rounds, 64))]
        return {"rounds": int(st.rounds), "async_rounds": int(st.async_rounds), "redone": bool(st.redone),
                "graph": int(st.graph),
                "plan_slack": float(st.plan_slack),
                "kernel_launches": int(st.kernel_launches),
                "input_bytes": int(st.input_bytes), "per_round": rounds}


class Grammar:
    """A device-resident grammar (``lcg_grammar``), owned by the library."""

    def __init__(self, ctx: Context, handle):
        self.ctx = ctx
        self._h = handle

    def free(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            load().lcg_grammar_free(self._h)
            self._h = None

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass

    @property
    def shape(self):
        k, nl = ctypes.c_uint32(0), ctypes.c_uint32(0)
        self.ctx._check(load().lcg_grammar_shape(self._h, ctypes.byref(k), ctypes.byref(nl)))
        return int(k.value), int(nl.value)

    def level_size(self, level: int):
        g, G = ctypes.c_uint64(0), ctypes.c_uint64(0)
        self.ctx._check(load().lcg_level_size(self._h, level, ctypes.byref(g), ctypes.byref(G)))
        return int(g.value), int(G.value)

    def export(self) -> dict:
        """Host copy in the oracle's export format."""
        lib = load()
        k, nl = self.shape
        levels = []
        for i in range(1, nl + 1):
            g, G = self.level_size(i)
            ro = np.zeros(g + 1, dtype=np.uint64)
            rhs = np.zeros(max(G, 1), dtype=np.uint32)
            F = np.zeros(max(g, 1), dtype=np.uint32)
            self.ctx._check(lib.lcg_export_level(self.ctx._h, self._h, i, _np_ptr(ro), _np_ptr(rhs), _np_ptr(F)))
            levels.append({"g": g, "rhs_off": ro, "rhs": rhs[:G], "F": F[:g]})
        F0 = np.zeros(256, dtype=np.uint32)
        cl = np.zeros(max(k, 1), dtype=np.uint32)
        cr = np.zeros(max(k, 1), dtype=np.uint32)
        self.ctx._check(lib.lcg_export_start(self.ctx._h, self._h, _np_ptr(F0), _np_ptr(cl), _np_ptr(cr)))
        return {"F0": F0, "levels": levels, "c_level": cl[:k], "c_rank": cr[:k]}

    def roots(self, j0: int = 0, count=None):
        """lcg_string_roots: (level, rank, fingerprint) arrays of strings j0 ..
        j0 + count - 1 (the fingerprint depends on the string's content only)."""
        k, _ = self.shape
        count = k - j0 if count is None else count
        lv = np.zeros(max(count, 1), dtype=np.uint32)
        rk = np.zeros(max(count, 1), dtype=np.uint32)
        fp = np.zeros(max(count, 1), dtype=np.uint32)
        self.ctx._check(load().lcg_string_roots(self.ctx._h, self._h, j0, count, _np_ptr(lv), _np_ptr(rk), _np_ptr(fp)))
        return lv[:count], rk[:count], fp[:count]

    def packed_size(self) -> int:
        n = ctypes.c_uint64(0)
        self.ctx._check(load().lcg_packed_size(self._h, ctypes.byref(n)))
        return int(n.value)

    def export_packed(self, out=None):
        """lcg_export_packed: the packed form in one host buffer.  ``out`` (a
        uint8 numpy array or CPU uint8 tensor, page-locked for speed) is
        filled and a view of its first ``packed_size()`` bytes is returned;
        without it a new numpy array is returned."""
        n = self.packed_size()
        if out is None:
            out = np.empty(n, dtype=np.uint8)
        ptr, on_dev, keep = _data_arg(out)
        if on_dev:
            raise LCGError(-1, "lcg_export_packed writes host memory")
        cap = int(out.numel() if hasattr(out, "numel") else out.size)
        self.ctx._check(load().lcg_export_packed(self.ctx._h, self._h, ptr, cap))
        del keep
        return out[:n]

    def vbyte_size(self) -> int:
        n = ctypes.c_uint64(0)
        self.ctx._check(load().lcg_vbyte_size(self.ctx._h, self._h, ctypes.byref(n)))
        return int(n.value)

    def export_vbyte(self, out=None, device: bool = False):
        """lcg_export_vbyte: the VByte form in one buffer: ``out`` (a uint8
        numpy array, CPU tensor or CUDA tensor, 8-byte aligned) or a new numpy
        array (a new CUDA tensor when ``device``); returns a view of its first
        ``vbyte_size()`` bytes."""
        if out is None:
            n = self.vbyte_size()
            if device:
                import torch
                out = torch.empty(n, dtype=torch.uint8, device=f"cuda:{self.ctx.device}")
            else:
                out = np.empty(n, dtype=np.uint8)
        ptr, on_dev, keep = _data_arg(out)
        cap = int(out.numel() if hasattr(out, "numel") else out.size)
        nb = ctypes.c_uint64(0)
        self.ctx._check(load().lcg_export_vbyte(self.ctx._h, self._h, ptr, cap, on_dev, ctypes.byref(nb)))
        del keep
        return out[:int(nb.value)]

    def decompress_static(self, j: int, out) -> int:
        """lcg_decompress_static: exp(C[j]) into the CUDA uint8 tensor ``out``
        using the library's static scratch (no device allocation)."""
        ptr, on_dev, keep = _data_arg(out)
        if not on_dev:
            raise LCGError(-1, "lcg_decompress_static writes device memory only")
        n = ctypes.c_uint64(0)
        self.ctx._check(load().lcg_decompress_static(self.ctx._h, self._h, j, ptr, out.numel(), ctypes.byref(n)))
        return int(n.value)

    def decompress(self, j: int, out=None):
        """exp(C[j]) as bytes (host), or into a CUDA uint8 tensor ``out``."""
        lib = load()
        n = ctypes.c_uint64(0)
        if out is not None:
            ptr, on_dev, keep = _data_arg(out)
            self.ctx._check(lib.lcg_decompress(self.ctx._h, self._h, j, ptr, out.numel(), ctypes.byref(n), on_dev))
            return int(n.value)
        rc = lib.lcg_decompress(self.ctx._h, self._h, j, None, 0, ctypes.byref(n), 0)
        need = int(n.value)
        if rc != LCG_OK and need == 0:
            self.ctx._check(rc)
        buf = np.zeros(max(need, 1), dtype=np.uint8)
        self.ctx._check(lib.lcg_decompress(self.ctx._h, self._h, j, _np_ptr(buf), need, ctypes.byref(n), 0))
        return buf[:need].tobytes()


class PPGrammar:
    """A post-processed grammar (lcg_postprocess) on the device."""

    def __init__(self, h):
        self._h = h

    def stats(self) -> dict:
        st = PPStatsC()
        rc = load().lcg_pp_stats_of(self._h, ctypes.byref(st))
        if rc != LCG_OK:
            raise LCGError(rc, "lcg_pp_stats_of")
        return {f: int(getattr(st, f)) for f, _ in PPStatsC._fields_}

    def export(self) -> dict:
        """Host arrays: kind (uint8, per rule), rhs_off (uint64), rhs (uint32), c (uint32)."""
        st = self.stats()
        kind = np.zeros(max(st["rules"], 1), dtype=np.uint8)
        off = np.zeros(st["rules"] + 1, dtype=np.uint64)
        rhs = np.zeros(max(st["size"], 1), dtype=np.uint32)
        c = np.zeros(max(st["strings"], 1), dtype=np.uint32)
        rc = load().lcg_pp_export(self._h, _np_ptr(kind), _np_ptr(off), _np_ptr(rhs), _np_ptr(c))
        if rc != LCG_OK:
            raise LCGError(rc, "lcg_pp_export")
        return {"kind": kind[:st["rules"]], "rhs_off": off, "rhs": rhs[:st["size"]], "c": c[:st["strings"]]}

    def free(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            load().lcg_pp_free(self._h)
            self._h = None

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass

