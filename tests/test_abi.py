"""CPU checks of the C ABI: the library loads without a GPU, exports every
entry point include/*.h declares (g2.h, the library; g2_diag.h, its
measurement probes), and the binding's constants and struct layouts agree
with the header."""
import ctypes
import glob
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "g2.h")
HEADERS = sorted(glob.glob(os.path.join(ROOT, "include", "*.h")))


@pytest.fixture(scope="module")
def g2mod():
    from paper_2012_07990_gb300 import build_native
    build_native.build()
    from paper_2012_07990_gb300 import g2
    return g2


def declared_functions():
    names = set()
    for h in HEADERS:
        src = re.sub(r"/\*.*?\*/", "", open(h).read(), flags=re.S)
        names |= set(re.findall(r"\b(g2_[a-z0-9_]+)\s*\(", src))
    return sorted(names)


def header_defines():
    out = {}
    for name, val in re.findall(r"#define\s+(G2_[A-Z0-9_]+)\s+(0x[0-9a-fA-F]+u?|\d+)", open(HEADER).read()):
        out[name] = int(val.rstrip("u"), 0)
    return out


def test_every_declared_symbol_is_exported(g2mod):
    lib = ctypes.CDLL(g2mod.LIB_PATH)
    names = declared_functions()
    assert len(names) >= 20
    missing = [n for n in names if not hasattr(lib, n)]
    assert not missing, f"declared but not exported: {missing}"
    assert sorted(g2mod.exported_symbols()) == names


def test_constants_match_header(g2mod):
    d = header_defines()
    assert d["G2_SYMMETRIC"] == g2mod.G2_SYMMETRIC and d["G2_DEVICE_PTRS"] == g2mod.G2_DEVICE_PTRS
    for k, v in g2mod.LB.items():
        assert d[f"G2_LB_{k}"] == v
    assert d["G2_PULL"] == g2mod.G2_PULL and d["G2_BITMAP"] == g2mod.G2_BITMAP
    assert d["G2_UNFUSED_BITMAP"] == g2mod.G2_UNFUSED_BITMAP
    assert d["G2_DEDUP_DISABLED"] == g2mod.G2_DEDUP_DISABLED
    assert d["G2_DEDUP_BOOLMAP"] == g2mod.G2_DEDUP_BOOLMAP
    assert d["G2_INPUT_VERTEXSET_SIZE"] == g2mod.G2_INPUT_VERTEXSET_SIZE
    assert d["G2_FRONTIER_BOOLMAP"] == g2mod.G2_FRONTIER_BOOLMAP


def test_struct_layouts(g2mod):
    assert ctypes.sizeof(g2mod.g2_schedule) == 10 * 4
    assert ctypes.sizeof(g2mod.g2_hybrid) == 8 + 2 * 40
    assert ctypes.sizeof(g2mod.g2_stats) == 32


def test_version_and_error_string_without_gpu(g2mod):
    assert "sm_103a" in g2mod.version()
    assert isinstance(g2mod.last_error(), str)


def test_schedule_helpers(g2mod):
    s = g2mod.schedule("ETWC", direction=g2mod.G2_PULL, dedup=False, delta=8)
    assert s.load_balance == 5 and s.direction == 1 and s.dedup == 1 and s.delta == 8
    h = g2mod.hybrid(g2mod.schedule(), s, 0.05)
    assert h.criteria == 1 and abs(h.threshold - 0.05) < 1e-7 and h.s2.load_balance == 5
