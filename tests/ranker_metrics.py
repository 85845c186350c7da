"""Measurement helpers for the address ranker (not on the analysis path): the location
key of host trace records, and the share of racy locations that a check order visits
early. Used by bench.py's ranker section and by the CPU tests; the analysis itself keys
locations on the device."""
from __future__ import annotations

import numpy as np


def location_keys(ev, agents_per_block: int) -> np.ndarray:
    """Location key of each access record: the address, or (1 << 63) | (block << 40) |
    address for shared memory (shared memory is per block, the paper's shared-memory
    adaptation of the analysis)."""
    shared = ev["space"] == 1
    blk = (ev["agent"] // agents_per_block).astype(np.uint64)
    a = ev["addr"].astype(np.uint64)
    return np.where(shared, (np.uint64(1) << np.uint64(63)) | (blk << np.uint64(40)) | a, a)


def racy_location_recall(ev, agents_per_block: int, races: np.ndarray, keys_in_check_order: np.ndarray,
                         frac: float = 0.1) -> float:
    """Share of the racy locations (those holding some race's later access) among the first
    `frac` of the locations in check order."""
    if len(races) == 0 or len(keys_in_check_order) == 0:
        return float("nan")
    racy = np.unique(location_keys(ev[races[:, 1].astype(np.int64)], agents_per_block))
    k = max(1, int(len(keys_in_check_order) * frac))
    return float(np.isin(keys_in_check_order[:k], racy).sum()) / len(racy)
