"""Trains the address ranker's shipped parameters (paper_2111_12478_gb300/data/ranker_theta.f32).

Labels come from the exact CPU oracle: a location is labelled 1 when some race's later
access lies on it. Features, training (gradient and Adam kernels) and the evaluation run
on the GPU through the C ABI. Training traces: the 64-warp workload's op mix at widths
64-1024 warps (seeds 1001+), 1M events each; the held-out evaluation trace is seed 2001.

  python tests/train_ranker.py [--events 1000000] [--epochs 30]

Writes the parameters and, beside them, ranker_theta.json with the recipe and the
held-out recall (share of racy locations among the first 10% of locations checked).
"""
import argparse
import json
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

from oracle import oracle as O  # noqa: E402
from oracle import ranker as R  # noqa: E402
from paper_2111_12478_gb300 import tracegen as TG  # noqa: E402

TRAIN = [(1001, 64), (1002, 64), (1003, 64), (1004, 128), (1005, 256), (1006, 512), (1007, 1024), (1008, 64)]


def trace(seed, W, n):
    nb, apb = TG.blocks_for_width(W)
    p = dict(TG.WORKLOADS["8blk_64warp_10M"])
    p.update(n_events=n, num_blocks=nb, agents_per_block=apb, n_ranks=max(1000, n // 10))
    ev, geo, _ = TG.generate(seed, **p)
    return ev, geo


def features_and_labels(gwcp, ev, geo, ranker_theta=None):
    races = O.run(ev, *geo.astuple()).races
    with gwcp.Context(0) as c:
        c.set_ranker(ranker_theta)
        c.load_trace(ev, *geo.astuple())
        c.compute_order()
        assert np.array_equal(c.report_races(), races)
        f, k = c.location_features()
        keys = k.cpu().numpy().view(np.uint64)
    return f.cpu().numpy(), R.labels(ev, geo.agents_per_block, races, keys).astype(np.float32)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--events", type=int, default=1_000_000)
    ap.add_argument("--epochs", type=int, default=30)
    ap.add_argument("--batch", type=int, default=4096)
    ap.add_argument("--lr", type=float, default=3e-3)
    args = ap.parse_args()
    import torch

    import __graft_entry__

    __graft_entry__.build()
    from paper_2111_12478_gb300 import gwcp, ranker

    X, Y = [], []
    for seed, W in TRAIN:
        f, y = features_and_labels(gwcp, *trace(seed, W, args.events))
        X.append(f)
        Y.append(y)
        print(f"seed {seed} W {W}: {len(y)} locations, {int(y.sum())} racy", flush=True)
    X, Y = np.concatenate(X), np.concatenate(Y)
    perm = np.random.default_rng(0).permutation(len(X))
    X, Y = X[perm], Y[perm]
    pw = float(min(50.0, (len(Y) - Y.sum()) / max(Y.sum(), 1)))
    th = torch.from_numpy(ranker.init_theta(1)).cuda()
    losses = gwcp.rank_train(th, torch.from_numpy(X).cuda(), torch.from_numpy(Y).cuda(), epochs=args.epochs,
                             batch=args.batch, lr=args.lr, pos_weight=pw)
    theta = th.cpu().numpy()
    ev, geo = trace(2001, 64, args.events)
    recall = {}
    for name, t in (("location_order", None), ("ranked", theta)):
        _, y = features_and_labels(gwcp, ev, geo, t)  # labels in check order
        k = max(1, len(y) // 10)
        recall[name] = float(y[:k].sum() / max(y.sum(), 1))
    ranker.save_weights(theta)
    info = {"train": [{"seed": s, "warps": W, "events": args.events} for s, W in TRAIN],
            "samples": int(len(Y)), "positives": int(Y.sum()), "pos_weight": pw, "epochs": args.epochs,
            "batch": args.batch, "lr": args.lr, "loss_first_last": [float(losses[0]), float(losses[-1])],
            "heldout": {"seed": 2001, "warps": 64, "events": args.events,
                        "racy_location_recall_first_10pct": recall}}
    with open(os.path.splitext(ranker.WEIGHTS)[0] + ".json", "w") as fh:
        json.dump(info, fh, indent=1)
    print(json.dumps(info["heldout"]), flush=True)


if __name__ == "__main__":
    main()
