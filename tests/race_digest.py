"""Order-independent digests of race sets, for comparing the CUDA path's races with the
oracle's on traces too large to store the oracle's race set itself.

A race (earlier a, later b) is the 64-bit word b << 32 | a (event indices < 2^30). The
races of a trace are cut into buckets by their later access, [k * bucket, (k + 1) *
bucket); a bucket's digest is (count, sum mod 2^64, xor) of splitmix64 of the words. A
race (a, b) depends only on the events up to b, so the races of a prefix of n events
are the whole trace's races with b < n, and every bucket below n / bucket has the same
digest in both.

Test infrastructure: shared by tests/golden/make_oracle_digests.py (which stores the
oracle's digests) and the GPU tests and bench.py (which digest the CUDA path's races).
"""
from __future__ import annotations

import hashlib

import numpy as np

_M1 = np.uint64(0x9E3779B97F4A7C15)
_M2 = np.uint64(0xBF58476D1CE4E5B9)
_M3 = np.uint64(0x94D049BB133111EB)


def _splitmix64(x: np.ndarray) -> np.ndarray:
    """splitmix64's output function (Steele, Lea, Flood 2014) on an array of words."""
    with np.errstate(over="ignore"):
        z = x + _M1
        z = (z ^ (z >> np.uint64(30))) * _M2
        z = (z ^ (z >> np.uint64(27))) * _M3
        return z ^ (z >> np.uint64(31))


def bucket_digests(races: np.ndarray, bucket: int, n_buckets: int) -> list[list[int]]:
    """[[count, sum, xor], ...] for buckets 0 .. n_buckets - 1 of a (k, 2) array of
    (earlier, later) races; races whose later access lies past the last bucket are ignored."""
    r = np.asarray(races, dtype=np.uint64).reshape(-1, 2)
    later = r[:, 1]
    keep = later < np.uint64(bucket * n_buckets)
    r = r[keep]
    b = (r[:, 1] // np.uint64(bucket)).astype(np.int64)
    h = _splitmix64((r[:, 1] << np.uint64(32)) | r[:, 0])
    cnt = np.bincount(b, minlength=n_buckets)[:n_buckets]
    s = np.zeros(n_buckets, dtype=np.uint64)
    x = np.zeros(n_buckets, dtype=np.uint64)
    with np.errstate(over="ignore"):
        np.add.at(s, b, h)
    np.bitwise_xor.at(x, b, h)
    return [[int(c), int(a), int(y)] for c, a, y in zip(cnt, s, x)]


def whole_digest(races: np.ndarray) -> list[int]:
    """(count, sum, xor) over all races."""
    r = np.asarray(races, dtype=np.uint64).reshape(-1, 2)
    if len(r) == 0:
        return [0, 0, 0]
    h = _splitmix64((r[:, 1] << np.uint64(32)) | r[:, 0])
    with np.errstate(over="ignore"):
        s = np.add.reduce(h, dtype=np.uint64)
    return [int(len(r)), int(s), int(np.bitwise_xor.reduce(h))]


def trace_sha256(ev: np.ndarray, n: int | None = None) -> str:
    """SHA-256 of the first n events' 16-byte records (the whole trace when n is None)."""
    a = ev if n is None else ev[:n]
    return hashlib.sha256(np.ascontiguousarray(a).view(np.uint8).tobytes()).hexdigest()
