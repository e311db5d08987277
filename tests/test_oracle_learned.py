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


# ----------------------------------------------- pins against independent code
# The layout of the parameter vector as the ABI documents it: W1[64][80], b1[64],
# W2[64][64], b2[64], W3[64][64], b3[64], W4[1024][64], b4[1024] (row = output unit).
LAYOUT = (("W1", (64, 80)), ("b1", (64,)), ("W2", (64, 64)), ("b2", (64,)), ("W3", (64, 64)),
          ("b3", (64,)), ("W4", (1024, 64)), ("b4", (1024,)))


def _unpack_np(params):
    out, o = {}, 0
    for name, shape in LAYOUT:
        k = int(np.prod(shape))
        out[name] = np.asarray(params[o:o + k], np.float64).reshape(shape)
        o += k
    assert o == len(params)
    return out


def _features_np(pos, nrm, lo, S):
    """The 78 input features from their definition (p^ = (p - lo) / S; sin and
    cos of 2^k pi p^ for k = 0..11; the normal), padded with two zeros."""
    ph = (pos.astype(np.float64) - lo.astype(np.float64)) / float(S)
    cols = [ph]
    for k in range(12):
        cols += [np.sin(2.0 ** k * np.pi * ph), np.cos(2.0 ** k * np.pi * ph)]
    cols += [nrm.astype(np.float64), np.zeros((len(pos), 2))]
    return np.concatenate(cols, axis=1)


def _torch_forward(params, x, bf16=False):
    """z = W4 relu(W3 relu(W2 relu(W1 x + b1) + b2) + b3) + b4 with torch's float64
    linear layers; with bf16 the weights, inputs and hidden activations go
    through torch's float32 -> bfloat16 conversion where the kernels store them."""
    torch = pytest.importorskip("torch")
    F = torch.nn.functional
    P = {k: torch.from_numpy(v) for k, v in _unpack_np(params).items()}
    r = (lambda t: t.float().bfloat16().double()) if bf16 else (lambda t: t)
    h = r(torch.from_numpy(x))
    for l in (1, 2, 3):
        h = r(F.relu(F.linear(h, r(P[f"W{l}"]), P[f"b{l}"])))
    z = F.linear(h, r(P["W4"]), P["b4"])
    return z, F.softmax(z, dim=1)


def _params_with_biases(seed):
    """Initial weights plus noise large enough that every bias and weight
    block moves the logits well beyond rounding."""
    rng = np.random.default_rng(seed)
    p = inputs.mlp_init(seed).astype(np.float64)
    return (p + rng.normal(0, 0.1, p.shape)).astype(np.float32)


def test_features_match_their_definition():
    pos, nrm = _batch(64, 21)
    lo = np.array([-0.5, 0.25, 1.0], np.float32)
    S = 2.0
    pos = (lo + pos * np.float32(S)).astype(np.float32)
    np.testing.assert_allclose(oracle.mlp_features(pos, nrm, lo, S), _features_np(pos, nrm, lo, S),
                               rtol=0, atol=1e-11)


@pytest.mark.parametrize("bf16", [False, True])
def test_forward_matches_an_independent_float64_network(bf16):
    """Logits and probabilities equal torch's float64 linear/ReLU/softmax network
    built from the documented parameter layout (a transposed weight block, a
    dropped bias or a ReLU on the logits each move them by far more than the
    tolerance)."""
    torch = pytest.importorskip("torch")
    params = _params_with_biases(4)
    pos, nrm = _batch(200, 13)
    lo = np.array([-0.5, 0.25, 1.0], np.float32)
    S = 2.0
    pos = (lo + pos * np.float32(S)).astype(np.float32)
    z, p = oracle.mlp_forward(params, pos, nrm, lo, S, bf16=bf16)
    x = oracle.mlp_features(pos, nrm, lo, S) if bf16 else _features_np(pos, nrm, lo, S)
    zt, pt = _torch_forward(params, x, bf16=bf16)
    np.testing.assert_allclose(z, zt.numpy(), rtol=0, atol=1e-9)
    np.testing.assert_allclose(p, pt.numpy(), rtol=1e-9, atol=1e-15)
    assert np.min(z) < -0.5 and np.ptp(z) > 1.0  # negative logits present: a ReLU there would show
    del torch


def test_forward_of_a_hand_built_network_in_closed_form():
    """A network with a few non-zero weights: every logit is a closed-form
    function of the position and normal (dyadic values, exact in binary64 and
    in bfloat16, so both modes must give exactly these numbers)."""
    P = {name: np.zeros(shape) for name, shape in LAYOUT}
    P["W1"][0, 0] = 1.0                       # u0 = relu(px)
    P["W1"][1, 1] = 1.0                       # u1 = relu(py)
    P["W1"][2, 77] = 2.0
    P["b1"][2] = 0.5                          # u2 = relu(2 nz + 0.5)
    P["W1"][3, 0] = -1.0
    P["b1"][3] = 0.25                         # u3 = relu(0.25 - px)
    for j in range(4):
        P["W2"][j, j] = 1.0
        P["W3"][j, j] = 1.0
    P["b2"][1] = 0.125                        # second layer: u1 + 1/8
    P["W4"][5, 0] = 1.0
    P["W4"][700, 1] = -3.0
    P["W4"][1023, 2] = 0.5
    P["W4"][1023, 3] = 2.0
    P["W4"][64, 3] = 4.0                      # an entry a transposed read of W4 would misplace
    P["b4"][:] = np.where(np.arange(1024) % 3 == 0, -0.75, 0.25)
    params = np.concatenate([P[name].ravel() for name, _ in LAYOUT]).astype(np.float32)
    pos = np.array([[0.125, 0.375, 0.75], [0.5, 0.0625, 0.25], [0.25, 0.5, 0.5]], np.float32)
    nrm = np.array([[0.0, 0.0, 1.0], [0.0, 0.0, -1.0], [1.0, 0.0, 0.0]], np.float32)
    px, py, nz = pos[:, 0].astype(np.float64), pos[:, 1].astype(np.float64), nrm[:, 2].astype(np.float64)
    want = np.tile(P["b4"], (3, 1))
    want[:, 5] += px
    want[:, 700] += -3.0 * (py + 0.125)
    want[:, 1023] += 0.5 * np.maximum(2 * nz + 0.5, 0) + 2.0 * np.maximum(0.25 - px, 0)
    want[:, 64] += 4.0 * np.maximum(0.25 - px, 0)
    e = np.exp(want - want.max(axis=1, keepdims=True))
    for bf16 in (False, True):
        z, p = oracle.mlp_forward(params, pos, nrm, LO, 1.0, bf16=bf16)
        np.testing.assert_array_equal(z, want)
        np.testing.assert_allclose(p, e / e.sum(axis=1, keepdims=True), rtol=1e-13, atol=0)


def test_gradient_matches_torch_autograd_everywhere():
    """Every one of the 80,064 gradient entries (and the loss) equals torch
    autograd of mean KL(q || softmax(z)) through the independent float64
    network (the padded input columns get zero)."""
    torch = pytest.importorskip("torch")
    F = torch.nn.functional
    params = _params_with_biases(6)
    pos, nrm = _batch(24, 17)
    q = inputs.random_distributions(9, 24, conc=0.5)
    loss, g = oracle.mlp_grad(params, pos, nrm, LO, 1.0, q)
    P = {k: torch.from_numpy(v).requires_grad_(True) for k, v in _unpack_np(params).items()}
    h = torch.from_numpy(_features_np(pos, nrm, LO, 1.0))
    for l in (1, 2, 3):
        h = F.relu(F.linear(h, P[f"W{l}"], P[f"b{l}"]))
    z = F.linear(h, P["W4"], P["b4"])
    qt = torch.from_numpy(q.astype(np.float64))
    qt = qt / qt.sum(dim=1, keepdim=True)  # the loss compares the normalised target
    lt = (torch.where(qt > 0, qt * (torch.log(torch.where(qt > 0, qt, 1.0)) - F.log_softmax(z, 1)),
                      torch.zeros_like(qt))).sum(1).mean()
    lt.backward()
    want = torch.cat([P[name].grad.reshape(-1) for name, _ in LAYOUT]).numpy()
    want[np.arange(64) * 80 + 78] = 0.0
    want[np.arange(64) * 80 + 79] = 0.0
    assert abs(loss - lt.item()) <= 1e-12 * abs(lt.item())
    np.testing.assert_allclose(g, want, rtol=1e-9, atol=1e-14)


def test_target_rows_are_normalised():
    """Any non-negative field is a target: scaling a row by a power of two
    leaves loss and gradient bit for bit unchanged, by another factor (the
    traced PDF's N^2 / 4 pi) up to the float32 rounding of the scaled row."""
    params = _params_with_biases(2)
    pos, nrm = _batch(6, 8)
    q = inputs.random_distributions(5, 6)
    l0, g0 = oracle.mlp_grad(params, pos, nrm, LO, 1.0, q)
    pow2 = np.array([1.0, 2.0, 0.125, 4.0, 0.5, 1024.0], np.float32)[:, None]
    l1, g1 = oracle.mlp_grad(params, pos, nrm, LO, 1.0, (q * pow2).astype(np.float32))
    assert l1 == l0
    np.testing.assert_array_equal(g1, g0)
    l2, g2 = oracle.mlp_grad(params, pos, nrm, LO, 1.0, (q * np.float32(1024 / (4 * np.pi))).astype(np.float32))
    assert abs(l2 - l0) <= 1e-6 * abs(l0)
    np.testing.assert_allclose(g2, g0, rtol=0, atol=1e-6 * np.max(np.abs(g0)))


def test_trace_is_the_gradients_own_arithmetic():
    params = _params_with_biases(8)
    pos, nrm = _batch(16, 3)
    q = inputs.random_distributions(4, 16)
    for bf16 in (False, True):
        l0, g0 = oracle.mlp_grad(params, pos, nrm, LO, 1.0, q, bf16=bf16)
        l1, g1, tr = oracle.mlp_grad_trace(params, pos, nrm, LO, 1.0, q, bf16=bf16)
        assert l0 == l1
        np.testing.assert_array_equal(g0, g1)
        z, _ = oracle.mlp_forward(params, pos, nrm, LO, 1.0, bf16=bf16)
        np.testing.assert_array_equal(tr["z"], z)
        # the output layer's weight gradient is the batch sum of g4 (x) h3
        W4 = g1[13504:13504 + 65536].reshape(1024, 64)
        np.testing.assert_allclose(W4, tr["g4"].T @ tr["h3"], rtol=1e-10, atol=1e-18)


def test_adam_matches_torch_optim_adam_over_three_steps():
    """Three steps (bias corrections at t = 1, 2, 3) equal torch.optim.Adam on
    float64 parameters, moments included; the oracle keeps float32 weights."""
    torch = pytest.importorskip("torch")
    p0 = np.array([0.5, -0.25, 1.0, 0.0, 2.0, -1.5], np.float32)
    grads = [np.array([3.0, -2.0, 1e-3, 0.5, -7.0, 1e-5]),
             np.array([-1.0, -2.5, 2e-3, 0.0, 4.0, -3e-5]),
             np.array([0.25, 1.0, -5e-3, -0.75, 1.0, 1e-5])]
    lr, b1, b2, eps = 0.05, 0.8, 0.95, 1e-4
    tp = torch.tensor(p0.astype(np.float64), requires_grad=True)
    opt = torch.optim.Adam([tp], lr=lr, betas=(b1, b2), eps=eps)
    p, m, v = p0, np.zeros(6), np.zeros(6)
    for t, g in enumerate(grads, start=1):
        p, m, v = oracle.adam(p, m, v, g, t, lr=lr, b1=b1, b2=b2, eps=eps)
        tp.grad = torch.from_numpy(g.copy())
        opt.step()
        st = opt.state[tp]
        np.testing.assert_allclose(m, st["exp_avg"].numpy(), rtol=1e-14)
        np.testing.assert_allclose(v, st["exp_avg_sq"].numpy(), rtol=1e-14)
        # float32 weights: one rounding per step away from torch's float64 trajectory
        np.testing.assert_allclose(p, tp.detach().numpy(), rtol=0, atol=4e-7 * t)
        tp.data = torch.from_numpy(p.astype(np.float64))  # follow the float32 trajectory
