import os
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
for p in (ROOT, os.path.join(ROOT, "tests")):
    if p not in sys.path:
        sys.path.insert(0, p)

from paper_2111_12478_gb300.tracegen import EVENT_DTYPE, Geometry  # noqa: E402

GOLDEN = os.path.join(ROOT, "tests", "golden")
OPS = {"RD": 0, "READ": 0, "WR": 1, "WRITE": 1, "ATOMIC": 2, "AT": 2, "ACQ": 3, "REL": 4, "BARRIER": 5, "BAR": 5,
       "FENCE": 6}


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a GB300 and the CUDA library")


def load_golden(name):
    """Reads a hand-written trace fixture: returns (events, Geometry, expected race set)."""
    rows, expect, geo = [], set(), None
    with open(os.path.join(GOLDEN, name)) as f:
        for line in f:
            line = line.split("#", 1)[0].strip()
            if not line:
                continue
            tok = line.split()
            if tok[0] == "geometry":
                geo = Geometry(int(tok[1]), int(tok[2]), int(tok[3]))
            elif tok[0] == "expect":
                expect.add((int(tok[1]), int(tok[2])))
            else:
                agent, op, scope, space, addr = tok
                rows.append((int(agent), OPS[op], int(scope), int(space), 0, int(addr, 0)))
    ev = np.zeros(len(rows), dtype=EVENT_DTYPE)
    for i, r in enumerate(rows):
        ev[i] = r
    return ev, geo, expect


GOLDEN_FILES = sorted(f for f in os.listdir(GOLDEN) if f.endswith(".trace"))
