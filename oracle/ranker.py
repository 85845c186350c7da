"""Plain CPU statement of the address ranker: per-location features, the BF16 MLP
16 -> 64 -> 64 -> 1, its loss, gradients and Adam step, and the race labels it is trained on.

TEST INFRASTRUCTURE ONLY (like the GWCP oracle next to it): only tests/ and the
committed training script under tests/ may import this module. It shares no code with
the CUDA path. The ranker is not part of the paper; it only reorders the per-location
check, so nothing here changes a race set.

Features of a location (the accesses to one location key, in trace order; locations in
ascending key order; shared memory is keyed per block as in the paper's
"Tracking GWCP" section). With n accesses, of which r reads, w writes, a atomics
(c of them block-scoped, d device-scoped):
  0 log1p(n)         1 log1p(r)          2 log1p(w)          3 log1p(a)
  4 log1p(#distinct agent mod 64)         5 log1p(#distinct block mod 64)
  6 c / n            7 d / n             8 (accesses inside a critical section) / n
  9 1 if the location is in shared memory
 10 sync density: acquire, release and barrier events with trace index in
    [first access, last access], divided by (last - first + 1)
 11 log1p(last - first)
 12 share of accesses by the agent of the first access
 13 agent switches: consecutive accesses by different agents / max(n - 1, 1)
 14 conflicting switches: consecutive accesses by different agents where at least one
    of the two is a write or an atomic, / max(n - 1, 1)
 15 (writes and atomics inside a critical section) / max(w + a, 1)
An access is inside a critical section when its agent holds at least one lock (acquires
minus releases of that agent before it > 0).

Network (parameters as one float32 vector, this order): W1 [64][16], b1 [64],
W2 [64][64], b2 [64], w3 [64], b3 [1]; 5313 values. With bf() = rounding to bfloat16
(round to nearest even):
  z1 = bf(x) bf(W1)^T + b1,  h1 = bf(relu(z1)),  z2 = h1 bf(W2)^T + b2,  h2 = relu(z2),
  s = h2 . w3 + b3.
Loss over a batch of B samples with labels y in {0, 1}: mean of
  wt * (softplus(s) - y s),  wt = pos_weight if y = 1 else 1.
Gradients treat the roundings as the identity (straight-through).
"""
from __future__ import annotations

import numpy as np

N_FEAT, H1, H2 = 16, 64, 64
N_PARAMS = H1 * N_FEAT + H1 + H2 * H1 + H2 + H2 + 1  # 5313
READ, WRITE, ATOMIC, ACQ, REL, BARRIER = 0, 1, 2, 3, 4, 5
SCOPE_DEVICE = 1


def split(theta):
    """Views of the parameter vector: W1, b1, W2, b2, w3, b3."""
    t = np.asarray(theta)
    o = 0
    out = []
    for shape in ((H1, N_FEAT), (H1,), (H2, H1), (H2,), (H2,), (1,)):
        k = int(np.prod(shape))
        out.append(t[o:o + k].reshape(shape))
        o += k
    assert o == N_PARAMS
    return out


def bf16(x):
    """Rounds to bfloat16 (round to nearest, ties to even) through float32; returns float64."""
    f = np.asarray(x, dtype=np.float32)
    b = f.view(np.uint32).astype(np.uint64)
    b = (b + 0x7FFF + ((b >> 16) & 1)) & 0xFFFF0000
    return b.astype(np.uint32).view(np.float32).astype(np.float64)


def location_keys(ev, agents_per_block):
    shared = ev["space"] == 1
    blk = (ev["agent"] // agents_per_block).astype(np.uint64)
    key = ev["addr"].astype(np.uint64)
    return np.where(shared, (np.uint64(1) << np.uint64(63)) | (blk << np.uint64(40)) | key, key)


def in_section(ev):
    """Per event: does its agent hold a lock at that point (acquires minus releases > 0)."""
    out = np.zeros(len(ev), dtype=bool)
    depth = {}
    for i in range(len(ev)):
        a = int(ev["agent"][i])
        op = int(ev["op"][i])
        if op == ACQ:
            depth[a] = depth.get(a, 0) + 1
        elif op == REL:
            depth[a] = depth.get(a, 0) - 1
        else:
            out[i] = depth.get(a, 0) > 0
    return out


def features(ev, agents_per_block):
    """Returns (location keys ascending, features [n_loc][16] float64) of a trace."""
    ev = np.asarray(ev)
    acc = np.nonzero(ev["op"] <= ATOMIC)[0]
    if len(acc) == 0:
        return np.zeros(0, dtype=np.uint64), np.zeros((0, N_FEAT))
    keys = location_keys(ev[acc], agents_per_block)
    ins = in_section(ev)[acc]
    sync_idx = np.nonzero((ev["op"] == ACQ) | (ev["op"] == REL) | (ev["op"] == BARRIER))[0]
    order = np.lexsort((acc, keys))  # by key, then trace index
    acc, keys, ins = acc[order], keys[order], ins[order]
    starts = np.r_[0, np.nonzero(keys[1:] != keys[:-1])[0] + 1, len(keys)]
    F = np.zeros((len(starts) - 1, N_FEAT))
    for L in range(len(starts) - 1):
        lo, hi = starts[L], starts[L + 1]
        ix = acc[lo:hi]
        e = ev[ix]
        n = hi - lo
        op, agent = e["op"].astype(int), e["agent"].astype(int)
        r, w, a = int((op == READ).sum()), int((op == WRITE).sum()), int((op == ATOMIC).sum())
        dev = int(((op == ATOMIC) & (e["scope"] == SCOPE_DEVICE)).sum())
        wc = op != READ
        first, last = int(ix[0]), int(ix[-1])
        n_sync = int(np.searchsorted(sync_idx, last, side="right") - np.searchsorted(sync_idx, first, side="left"))
        sw = agent[1:] != agent[:-1]
        csw = sw & (wc[1:] | wc[:-1])
        F[L] = [np.log1p(n), np.log1p(r), np.log1p(w), np.log1p(a),
                np.log1p(len(set((agent % 64).tolist()))),
                np.log1p(len(set(((agent // agents_per_block) % 64).tolist()))),
                (a - dev) / n, dev / n, ins[lo:hi].sum() / n, float(e["space"][0] == 1),
                n_sync / (last - first + 1), np.log1p(last - first), (agent == agent[0]).sum() / n,
                sw.sum() / max(n - 1, 1), csw.sum() / max(n - 1, 1),
                (ins[lo:hi] & wc).sum() / max(w + a, 1)]
    return keys[starts[:-1]], F


def labels(ev, agents_per_block, races, loc_keys):
    """1 for every location that holds the later access of some race, else 0."""
    if len(races) == 0:
        return np.zeros(len(loc_keys), dtype=np.float64)
    k = location_keys(np.asarray(ev)[np.asarray(races)[:, 1].astype(np.int64)], agents_per_block)
    return np.isin(loc_keys, np.unique(k)).astype(np.float64)


def forward(theta, x, rounding=True):
    """Scores s and the intermediates (z1, h1, z2, h2, xb) for a batch x [B][16]."""
    W1, b1, W2, b2, w3, b3 = [np.asarray(p, dtype=np.float64) for p in split(theta)]
    r = bf16 if rounding else (lambda v: np.asarray(v, dtype=np.float64))
    xb = r(x)
    z1 = xb @ r(W1).T + b1
    h1 = r(np.maximum(z1, 0.0))
    z2 = h1 @ r(W2).T + b2
    h2 = np.maximum(z2, 0.0)
    s = h2 @ w3 + b3[0]
    return s, (z1, h1, z2, h2, xb)


def loss(theta, x, y, pos_weight, rounding=True):
    s, _ = forward(theta, x, rounding)
    wt = np.where(y > 0, pos_weight, 1.0)
    return float(np.mean(wt * (np.logaddexp(0.0, s) - y * s)))


def grad(theta, x, y, pos_weight, rounding=True):
    """Gradient of loss() with respect to the parameter vector (float64)."""
    W1, b1, W2, b2, w3, b3 = [np.asarray(p, dtype=np.float64) for p in split(theta)]
    r = bf16 if rounding else (lambda v: np.asarray(v, dtype=np.float64))
    s, (z1, h1, z2, h2, xb) = forward(theta, x, rounding)
    B = len(s)
    wt = np.where(y > 0, pos_weight, 1.0)
    ds = wt * (1.0 / (1.0 + np.exp(-s)) - y) / B
    dw3 = h2.T @ ds
    db3 = np.array([ds.sum()])
    dz2 = np.outer(ds, w3) * (z2 > 0)
    dW2 = dz2.T @ h1
    db2 = dz2.sum(axis=0)
    dz1 = (dz2 @ r(W2)) * (z1 > 0)
    dW1 = dz1.T @ xb
    db1 = dz1.sum(axis=0)
    return np.concatenate([dW1.ravel(), db1, dW2.ravel(), db2, dw3, db3])


def adam_step(theta, m, v, g, t, lr, b1=0.9, b2=0.999, eps=1e-8):
    """One Adam update (step t counts from 1); returns new (theta, m, v)."""
    m = b1 * m + (1 - b1) * g
    v = b2 * v + (1 - b2) * g * g
    mh = m / (1 - b1 ** t)
    vh = v / (1 - b2 ** t)
    return theta - lr * mh / (np.sqrt(vh) + eps), m, v
