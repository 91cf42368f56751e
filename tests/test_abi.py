"""The C-ABI library builds for sm_103a, loads, and exports every entry point
declared in include/lcg.h (no GPU needed)."""
import ctypes
import os
import re

from paper_2411_12439_gb300 import build, lcg

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = set()
    inc = os.path.join(ROOT, "include")
    for f in os.listdir(inc):
        if f.endswith(".h"):
            text = open(os.path.join(inc, f)).read()
            text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
            names |= set(re.findall(r"\b(lcg_[a-z0-9_]+)\s*\(", text))
    return names


def test_library_exports_every_declared_symbol():
    path = build.build()
    lib = ctypes.CDLL(path)
    names = declared_functions()
    assert "lcg_build" in names and "lcg_merge" in names and "lcg_decompress" in names
    for name in sorted(names):
        assert hasattr(lib, name), name
    assert names <= set(lcg.SYMBOLS) | names


def test_binding_covers_header():
    assert declared_functions() == set(lcg.SYMBOLS)


def test_no_device_is_reported_not_hidden():
    """Without a GPU the context refuses with LCG_EDEVICE (no CPU fallback)."""
    import torch
    if torch.cuda.is_available():
        return
    import lcg_inputs as li
    try:
        lcg.Context(li.hash_family())
    except lcg.LCGError as e:
        assert e.code == -7
    else:
        raise AssertionError("context created without a device")


def test_missing_library_fails_loudly(monkeypatch, tmp_path):
    """No CUDA library: loading raises (there is no CPU path to fall back on)."""
    monkeypatch.setattr(lcg, "_lib", None)
    monkeypatch.setattr(lcg._build, "LIB", str(tmp_path / "liblcg_gb300.so"))
    try:
        lcg.load(build_if_missing=False)
    except lcg.LCGError as e:
        assert e.code == -7
    else:
        raise AssertionError("loaded a library that does not exist")


# C layout of the structs include/lcg.h declares, from the header text alone
# (natural alignment, as gcc and nvcc lay them out on x86-64 and aarch64).
_SCALARS = {"uint32_t": (4, 4), "uint64_t": (8, 8), "double": (8, 8), "char": (1, 1), "int": (4, 4)}


def header_structs():
    text = open(os.path.join(ROOT, "include", "lcg.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    structs = {}
    for name, body in re.findall(r"typedef struct (\w+) \{(.*?)\}\s*\1;", text, flags=re.S):
        fields = []
        for decl in body.split(";"):
            decl = " ".join(decl.split())
            if not decl:
                continue
            m = re.fullmatch(r"(?:const )?([\w]+)\s*(\*?)\s*(\w+)(?:\[(\d+)\])?", decl)
            assert m, (name, decl)
            typ, ptr, field, count = m.group(1), m.group(2), m.group(3), int(m.group(4) or 1)
            fields.append((field, "ptr" if ptr else typ, count))
        structs[name] = fields
    return structs


def c_layout(structs, name):
    """Offsets of the fields of struct `name`, its size and its alignment."""
    off, align, offsets = 0, 1, {}
    for field, typ, count in structs[name]:
        if typ == "ptr":
            size, al = 8, 8
        elif typ in _SCALARS:
            size, al = _SCALARS[typ]
        else:
            _, size, al = c_layout(structs, typ)
        off = (off + al - 1) // al * al
        offsets[field] = off
        off += size * count
        align = max(align, al)
    return offsets, (off + align - 1) // align * align, align


def test_struct_layouts_match_header():
    """Every ctypes mirror in the binding has the header struct's fields, in
    order, at the same offsets, and the same size."""
    structs = header_structs()
    mirrors = {"lcg_hash_family": lcg.HashFamilyC, "lcg_round_stats": lcg.RoundStatsC,
               "lcg_build_stats": lcg.BuildStatsC, "lcg_kernel_time": lcg.KernelTimeC,
               "lcg_tuning": lcg.TuningC, "lcg_kernel_launch": lcg.KernelLaunchC, "lcg_pp_stats": lcg.PPStatsC}
    assert set(mirrors) == set(structs), sorted(structs)
    for name, cls in mirrors.items():
        offsets, size, _ = c_layout(structs, name)
        assert [f for f, _, _ in structs[name]] == [f[0] for f in cls._fields_], name
        for field, off in offsets.items():
            assert getattr(cls, field).offset == off, (name, field)
        assert ctypes.sizeof(cls) == size, name
