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
