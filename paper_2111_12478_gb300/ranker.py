"""Host helpers of the address ranker (argument handling and bookkeeping only; every
feature, score, gradient and update is computed by the CUDA library).

The ranker is not part of the paper. It scores each location from features of its
accesses so that the per-location check visits likely-racy locations first; the race
set never changes. Trained weights ship as ``data/ranker_theta.f32`` (5313 little-endian
float32 values in the library's parameter order), written by the training script next to
the tests, which labels locations with the exact analysis of generated traces.
"""
from __future__ import annotations

import os

import numpy as np

from . import gwcp

WEIGHTS = os.path.join(os.path.dirname(os.path.abspath(__file__)), "data", "ranker_theta.f32")
N_PARAMS, N_FEAT, H = gwcp.RANK_PARAMS, gwcp.RANK_FEATURES, 64


def init_theta(seed: int) -> np.ndarray:
    """He-style random initial parameters (float32), biases zero."""
    rng = np.random.default_rng(seed)
    parts = [rng.normal(0, np.sqrt(2.0 / N_FEAT), H * N_FEAT), np.zeros(H), rng.normal(0, np.sqrt(2.0 / H), H * H),
             np.zeros(H), rng.normal(0, np.sqrt(1.0 / H), H), np.zeros(1)]
    return np.concatenate(parts).astype(np.float32)


def load_weights(path: str = WEIGHTS) -> np.ndarray | None:
    """The shipped parameters, or None when the file is absent."""
    if not os.path.exists(path):
        return None
    t = np.fromfile(path, dtype="<f4")
    if t.size != N_PARAMS:
        raise ValueError(f"{path}: {t.size} values, expected {N_PARAMS}")
    return t


def save_weights(theta, path: str = WEIGHTS):
    os.makedirs(os.path.dirname(path), exist_ok=True)
    np.asarray(theta, dtype="<f4").tofile(path)


def timeline_summary(start_ns: int, chunk_end_ns: np.ndarray, chunk_races: np.ndarray) -> dict:
    """Time from the check's start until the first race, and until 50% / 90% / all of the
    races were found (chunk end times; ns -> µs), plus the share of races found in the
    first 10% of the chunks in check order."""
    total = int(chunk_races.sum())
    out = {"races": total, "chunks": int(len(chunk_races))}
    if total == 0 or len(chunk_races) == 0:
        return out
    order = np.argsort(chunk_end_ns, kind="stable")
    t = (chunk_end_ns[order].astype(np.int64) - int(start_ns)) / 1e3
    cum = np.cumsum(chunk_races[order].astype(np.int64))
    for name, frac in (("first_race_us", 1e-12), ("half_races_us", 0.5), ("p90_races_us", 0.9), ("all_races_us", 1.0)):
        k = int(np.searchsorted(cum, max(1, int(np.ceil(frac * total)))))
        out[name] = float(t[min(k, len(t) - 1)])
    out["check_us"] = float(t[-1])
    k10 = max(1, len(chunk_races) // 10)
    out["races_in_first_10pct_chunks"] = float(chunk_races[:k10].sum()) / total
    return out
