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


def test_binding_structs_match_the_header(tmp_path):
    """Every ctypes structure of the binding (and the trace record dtype) has the size and
    field offsets that a C compiler gives the header's struct of the same name."""
    import shutil
    import subprocess

    import numpy as np

    from paper_2111_12478_gb300 import tracegen as TG

    if shutil.which("gcc") is None:
        import pytest

        pytest.skip("no C compiler")
    pairs = [("gwcp_geometry", gwcp.Geometry), ("gwcp_options", gwcp.Options),
             ("gwcp_train_options", gwcp.TrainOptions), ("gwcp_trace_desc", gwcp.TraceDesc),
             ("gwcp_pool_options", gwcp.PoolOptions), ("gwcp_request_info", gwcp.RequestInfo),
             ("gwcp_race", gwcp.Race)]
    want = {}
    lines = ['#include <stddef.h>', '#include <stdio.h>', '#include "gwcp.h"', "int main(void) {"]
    for cname, cls in pairs:
        want[(cname, "sizeof")] = ctypes.sizeof(cls)
        lines.append(f'  printf("{cname} sizeof %zu\\n", sizeof({cname}));')
        for field, *_ in cls._fields_:
            want[(cname, field)] = getattr(cls, field).offset
            lines.append(f'  printf("{cname} {field} %zu\\n", offsetof({cname}, {field}));')
    dt = TG.EVENT_DTYPE
    want[("gwcp_event", "sizeof")] = dt.itemsize
    lines.append('  printf("gwcp_event sizeof %zu\\n", sizeof(gwcp_event));')
    for field in dt.names:
        want[("gwcp_event", field)] = dt.fields[field][1]
        lines.append(f'  printf("gwcp_event {field} %zu\\n", offsetof(gwcp_event, {field}));')
    lines += ["  return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    subprocess.check_call(["gcc", "-std=c99", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)])
    got = {}
    for line in subprocess.check_output([str(exe)], text=True).splitlines():
        cname, field, value = line.split()
        got[(cname, field)] = int(value)
    assert got == want
    assert np.dtype(dt).itemsize == 16
