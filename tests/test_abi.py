"""The C-ABI library builds, loads and exports every entry point include/gwcp.h declares
(no compute call: this runs without a GPU)."""
import ctypes
import os
import re

from conftest import ROOT
from paper_2111_12478_gb300 import build as B
from paper_2111_12478_gb300 import gwcp


def declared_functions():
    names = []
    for h in sorted(os.listdir(os.path.join(ROOT, "include"))):
        if h.endswith(".h"):
            text = open(os.path.join(ROOT, "include", h)).read()
            text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
            names += re.findall(r"^\s*(?:const\s+)?[\w\s\*]+?\b(gwcp_\w+)\s*\(", text, flags=re.M)
    return sorted(set(names))


def test_library_exports_declared_symbols():
    B.build()
    lib = ctypes.CDLL(B.LIB)
    decl = declared_functions()
    assert len(decl) >= 10
    for name in decl:
        assert hasattr(lib, name), name
    assert set(gwcp.EXPORTS) <= set(decl)


def test_strerror_without_gpu():
    B.build()
    assert gwcp.strerror(0) == "ok"
    assert "invalid trace" in gwcp.strerror(-1)
