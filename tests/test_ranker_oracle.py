"""Pins of the ranker oracle (oracle/ranker.py), none of which uses the oracle to check
itself: hand-computed features of a hand-built trace, central finite differences of the
loss, a closed form of the network where every unit is active (the network is then a
product of affine maps), bfloat16 rounding against torch's conversion, Adam's first
step (a signed step of size lr) and the loss at zero parameters (log 2 per sample)."""
import math

import numpy as np
import pytest

from oracle import ranker as R
from paper_2111_12478_gb300 import tracegen as TG


def hand_trace():
    b = TG.TraceBuilder()
    b.rd(0, 0x100)                     # 0
    b.acq(1, 7)                        # 1
    b.wr(1, 0x100)                     # 2  inside agent 1's section
    b.rel(1, 7)                        # 3
    b.barrier(0, agent=0, apb=2)       # 4
    b.atomic(2, 0x100, scope=TG.DEVICE)  # 5
    b.rd(0, 0x200)                     # 6
    b.atomic(3, 0x100, scope=TG.CTA)   # 7
    b.wr(1, 0x10, shared=True)         # 8  block 0's shared 0x10
    b.wr(3, 0x10, shared=True)         # 9  block 1's shared 0x10
    return b.build()


def test_features_by_hand():
    keys, F = R.features(hand_trace(), 2)
    s = 1 << 63
    assert keys.tolist() == [0x100, 0x200, s | 0x10, s | (1 << 40) | 0x10]
    L = math.log1p
    x = [L(4), L(1), L(1), L(2), L(4), L(2), 1 / 4, 1 / 4, 1 / 4, 0.0, 3 / 8, L(7), 1 / 4, 1.0, 1.0, 1 / 3]
    y = [L(1), L(1), 0, 0, L(1), L(1), 0, 0, 0, 0, 0, 0, 1, 0, 0, 0]
    z0 = [L(1), 0, L(1), 0, L(1), L(1), 0, 0, 0, 1, 0, 0, 1, 0, 0, 0]
    np.testing.assert_allclose(F[0], x, rtol=0, atol=1e-15)
    np.testing.assert_allclose(F[1], y, rtol=0, atol=1e-15)
    np.testing.assert_allclose(F[2], z0, rtol=0, atol=1e-15)
    np.testing.assert_allclose(F[3], z0, rtol=0, atol=1e-15)


def test_labels_by_hand():
    ev = hand_trace()
    keys, _ = R.features(ev, 2)
    races = np.array([[0, 2], [2, 7]], dtype=np.uint64)  # both on 0x100
    assert R.labels(ev, 2, races, keys).tolist() == [1, 0, 0, 0]
    assert R.labels(ev, 2, np.zeros((0, 2), np.uint64), keys).tolist() == [0, 0, 0, 0]


def _theta(seed, scale=0.3):
    return np.random.default_rng(seed).normal(0, scale, R.N_PARAMS)


def test_gradient_finite_differences():
    rng = np.random.default_rng(1)
    x = rng.normal(0, 1, (24, R.N_FEAT))
    y = (rng.random(24) < 0.3).astype(float)
    th = _theta(2)
    g = R.grad(th, x, y, 5.0, rounding=False)
    h = 1e-6
    idx = rng.choice(R.N_PARAMS, 300, replace=False).tolist() + [R.N_PARAMS - 1]
    for i in idx:
        e = np.zeros(R.N_PARAMS)
        e[i] = h
        fd = (R.loss(th + e, x, y, 5.0, False) - R.loss(th - e, x, y, 5.0, False)) / (2 * h)
        assert abs(fd - g[i]) <= 1e-7 + 1e-5 * abs(fd), (i, fd, g[i])


def test_all_active_is_affine():
    rng = np.random.default_rng(3)
    th = np.abs(_theta(4, 0.2))  # positive weights and inputs keep every unit active
    x = np.abs(rng.normal(0, 1, (10, R.N_FEAT)))
    W1, b1, W2, b2, w3, b3 = R.split(th)
    M = w3 @ W2 @ W1  # collapse the affine maps first, then apply
    c = w3 @ (W2 @ b1 + b2) + b3[0]
    s, _ = R.forward(th, x, rounding=False)
    np.testing.assert_allclose(s, x @ M + c, rtol=1e-12)


def test_bf16_matches_torch():
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(5)
    v = np.concatenate([rng.normal(0, 3, 20000), [1.0, 1 + 2 ** -8, 1 + 3 * 2 ** -9, -2.5, 0.0, 1e-30]])
    v32 = v.astype(np.float32)
    want = torch.from_numpy(v32).to(torch.bfloat16).float().numpy().astype(np.float64)
    np.testing.assert_array_equal(R.bf16(v32), want)
    assert R.bf16(1 + 2 ** -8) == 1.0 and R.bf16(1 + 3 * 2 ** -9) == 1 + 2 ** -7


def test_adam_first_step_is_signed_lr():
    rng = np.random.default_rng(6)
    g = rng.normal(0, 1, 50)
    th, m, v = R.adam_step(np.zeros(50), np.zeros(50), np.zeros(50), g, 1, lr=0.01, eps=0.0)
    np.testing.assert_allclose(th, -0.01 * np.sign(g), rtol=1e-12)


def test_loss_at_zero_parameters():
    rng = np.random.default_rng(7)
    x = rng.normal(0, 1, (9, R.N_FEAT))
    y = np.array([1, 0, 0, 1, 0, 0, 0, 0, 1], float)
    pw = 4.0
    want = np.mean(np.where(y > 0, pw, 1.0)) * math.log(2)
    assert abs(R.loss(np.zeros(R.N_PARAMS), x, y, pw) - want) < 1e-15
    g = R.grad(np.zeros(R.N_PARAMS), x, y, pw)
    # only the output bias moves at zero parameters: ds = wt (1/2 - y) / B
    assert abs(g[-1] - np.sum(np.where(y > 0, pw, 1.0) * (0.5 - y)) / 9) < 1e-15
    assert np.count_nonzero(g[:-1]) == 0
