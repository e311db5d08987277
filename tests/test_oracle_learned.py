"""Pins of the oracle's learned proposal (MLP features, forward, KL loss,
backpropagation, Adam) against finite differences, closed forms and the
defining properties of the KL divergence."""
import math

import numpy as np
import pytest

import oracle
from paper_2405_06997_gb300 import inputs

LO = np.zeros(3, np.float32)


def _batch(n, seed):
    rng = np.random.default_rng(seed)
    pos = rng.uniform(0, 1, (n, 3)).astype(np.float32)
    nrm = rng.normal(size=(n, 3))
    nrm = (nrm / np.linalg.norm(nrm, axis=1, keepdims=True)).astype(np.float32)
    return pos, nrm


def test_feature_layout_and_identities():
    pos = np.array([[0.25, 0.5, 0.125]], np.float32)
    nrm = np.array([[0.0, 0.6, 0.8]], np.float32)
    f = oracle.mlp_features(pos, nrm, LO, 1.0)[0]
    assert f.shape == (80,)
    np.testing.assert_allclose(f[:3], [0.25, 0.5, 0.125])
    np.testing.assert_allclose(f[75:78], [0.0, 0.6, 0.8], atol=1e-7)
    assert f[78] == 0 and f[79] == 0
    for k in range(12):
        s = f[3 + 6 * k: 6 + 6 * k]
        c = f[6 + 6 * k: 9 + 6 * k]
        np.testing.assert_allclose(s * s + c * c, 1.0, atol=1e-12)
    # k = 0: sin(pi/4), sin(pi/2), sin(pi/8); k = 1: sin(pi/2), sin(pi), sin(pi/4)
    np.testing.assert_allclose(f[3:6], [math.sqrt(0.5), 1.0, math.sin(math.pi / 8)], atol=1e-12)
    np.testing.assert_allclose(f[9:12], [1.0, 0.0, math.sqrt(0.5)], atol=1e-12)


def test_kl_nonnegative_and_zero_at_own_distribution():
    params = inputs.mlp_init(3)
    pos, nrm = _batch(5, 1)
    q = inputs.random_distributions(2, 5)
    loss, _ = oracle.mlp_grad(params, pos, nrm, LO, 1.0, q)
    assert loss > 0
    _, p = oracle.mlp_forward(params, pos, nrm, LO, 1.0)
    loss0, g0 = oracle.mlp_grad(params, pos, nrm, LO, 1.0, p.astype(np.float32))
    assert abs(loss0) < 1e-6
    assert np.max(np.abs(g0)) < 1e-6


def test_gradient_matches_central_differences():
    params = inputs.mlp_init(7)
    rng = np.random.default_rng(0)
    params = (params + rng.normal(0, 0.02, params.shape)).astype(np.float32)  # non-zero biases too
    pos, nrm = _batch(3, 5)
    q = inputs.random_distributions(6, 3)
    loss, g = oracle.mlp_grad(params, pos, nrm, LO, 1.0, q)
    P = len(params)
    offs = {"W1": (0, 64 * 78), "b1": (5120, 64), "W2": (5184, 4096), "b2": (9280, 64),
            "W3": (9344, 4096), "b3": (13440, 64), "W4": (13504, 65536), "b4": (79040, 1024)}
    checked = 0
    for name, (o, n) in offs.items():
        for idx in rng.choice(n, 6, replace=False):
            i = o + int(idx)
            if name == "W1":
                i = o + (int(idx) // 78) * 80 + int(idx) % 78
            h = np.float32(1e-3 * max(1.0, abs(float(params[i]))))
            pp = params.copy()
            pp[i] = params[i] + h
            lp, _ = oracle.mlp_grad(pp, pos, nrm, LO, 1.0, q)
            dp = float(pp[i]) - float(params[i])
            pm = params.copy()
            pm[i] = params[i] - h
            lm, _ = oracle.mlp_grad(pm, pos, nrm, LO, 1.0, q)
            dm = float(params[i]) - float(pm[i])
            fd = (lp - lm) / (dp + dm)
            assert abs(fd - g[i]) <= 2e-4 * max(abs(fd), 1e-3) + 1e-7, (name, i, fd, g[i])
            checked += 1
    # the first layer's position and normal columns, which random picks rarely reach
    for row in (3, 40):
        for col in (0, 1, 2, 75, 76, 77):
            i = row * 80 + col
            h = np.float32(1e-3 * max(1.0, abs(float(params[i]))))
            pp, pm = params.copy(), params.copy()
            pp[i], pm[i] = params[i] + h, params[i] - h
            lp, _ = oracle.mlp_grad(pp, pos, nrm, LO, 1.0, q)
            lm, _ = oracle.mlp_grad(pm, pos, nrm, LO, 1.0, q)
            fd = (lp - lm) / ((float(pp[i]) - float(params[i])) + (float(params[i]) - float(pm[i])))
            assert abs(fd - g[i]) <= 2e-4 * max(abs(fd), 1e-3) + 1e-7, ("W1", row, col, fd, g[i])
            checked += 1
    assert checked == 60
    assert P == 80064
    assert np.all(g[np.arange(64) * 80 + 78] == 0) and np.all(g[np.arange(64) * 80 + 79] == 0)


def test_bf16_emulation_close_to_fp64():
    params = inputs.mlp_init(3)
    pos, nrm = _batch(16, 9)
    z64, _ = oracle.mlp_forward(params, pos, nrm, LO, 1.0, bf16=False)
    z16, _ = oracle.mlp_forward(params, pos, nrm, LO, 1.0, bf16=True)
    # bfloat16 keeps 8 significant bits: the logits agree to a few 1e-2
    assert np.max(np.abs(z16 - z64)) < 0.05 * max(1.0, np.max(np.abs(z64)))
    assert np.max(np.abs(z16 - z64)) > 0


def test_bf16_rounding_is_the_library_conversion():
    """The emulation's bfloat16 rounding equals torch's float32 -> bfloat16
    conversion (round to nearest, ties to even), on exact ties, on values one
    step either side of a tie, and on random values of every magnitude."""
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(4)
    base = rng.integers(0, 1 << 31, 4000, dtype=np.uint64).astype(np.uint32) & np.uint32(0xFFFF0000)
    base = base[((base >> 23) & 0xFF) < 0xFE]                      # finite, not at the top binade
    ties = base | np.uint32(0x8000)
    near = np.concatenate([ties - np.uint32(1), ties + np.uint32(1)])
    rand = rng.integers(0, 1 << 31, 20000, dtype=np.uint64).astype(np.uint32)
    rand = rand[((rand >> 23) & 0xFF) < 0xFF]
    x = np.concatenate([ties, near, rand]).view(np.float32)
    x = np.concatenate([x, -x, np.array([0.0, -0.0, 1.0, 3.0e38], np.float32)])
    want = torch.from_numpy(x.copy()).to(torch.bfloat16).to(torch.float32).numpy()
    np.testing.assert_array_equal(oracle.bf16_round(x).view(np.uint32), want.view(np.uint32))


def test_adam_first_step_is_lr_times_sign():
    p = np.array([0.5, -0.25, 1.0], np.float32)
    g = np.array([3.0, -2.0, 1e-3])
    p1, m, v = oracle.adam(p, np.zeros(3), np.zeros(3), g, t=1, lr=1e-2)
    np.testing.assert_allclose(p1, p - 1e-2 * np.sign(g), atol=2e-7)
    np.testing.assert_allclose(m, 0.1 * g)
    np.testing.assert_allclose(v, 0.001 * g * g)


def test_training_on_fixed_targets_lowers_kl():
    params = inputs.mlp_init(11)
    pos, nrm = _batch(4, 2)
    q = inputs.random_distributions(3, 4, conc=2.0)
    m = np.zeros(len(params))
    v = np.zeros(len(params))
    l0, g = oracle.mlp_grad(params, pos, nrm, LO, 1.0, q)
    for t in range(1, 31):
        _, g = oracle.mlp_grad(params, pos, nrm, LO, 1.0, q)
        params, m, v = oracle.adam(params, m, v, g, t, lr=3e-3)
    l1, _ = oracle.mlp_grad(params, pos, nrm, LO, 1.0, q)
    assert l1 < 0.7 * l0
