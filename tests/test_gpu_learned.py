"""Learned proposal on the GPU (tcgen05 forward/backward, Adam) against the
CPU oracle's MLP with bfloat16-rounding emulation.

Tolerances: bfloat16 keeps 8 significant bits and the kernels accumulate in
float32 where the oracle uses binary64, so a stored activation can round to
the neighbouring bfloat16 value; probabilities are compared to 8% relative
(logit error of a few 1e-2), gradients by relative L2 error per tensor."""
import numpy as np
import pytest

import oracle
from paper_2405_06997_gb300 import inputs

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA device", allow_module_level=True)

from paper_2405_06997_gb300 import wfpg as W  # noqa: E402

LO = np.zeros(3, np.float32)
SEGMENTS = {"W1": (0, 5120), "b1": (5120, 64), "W2": (5184, 4096), "b2": (9280, 64), "W3": (9344, 4096),
            "b3": (13440, 64), "W4": (13504, 65536), "b4": (79040, 1024)}


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def _batch(n, seed):
    rng = np.random.default_rng(seed)
    pos = rng.uniform(0, 1, (n, 3)).astype(np.float32)
    nrm = rng.normal(size=(n, 3))
    nrm = (nrm / np.linalg.norm(nrm, axis=1, keepdims=True)).astype(np.float32)
    return pos, nrm


@pytest.mark.parametrize("n", [1, 300, 1000])
def test_forward_matches_oracle(n):
    params = inputs.mlp_init(5)
    pos, nrm = _batch(n, 2)
    mlp = W.MLP(params, max_batch=1024)
    pdf, cr, cm = W.guide_learned_build_pdf(mlp, dev(pos), dev(nrm), eps=0.0)
    _, p = oracle.mlp_forward(params, pos, nrm, LO, 1.0, bf16=True)
    p_gpu = pdf.cpu().numpy().astype(np.float64) * (4 * np.pi / 1024)
    np.testing.assert_allclose(p_gpu.sum(axis=1), 1.0, rtol=1e-5)
    np.testing.assert_allclose(p_gpu, p, rtol=0.08, atol=1e-7)
    assert mlp.status() == 0


def test_gradient_matches_oracle():
    params = inputs.mlp_init(8)
    rng = np.random.default_rng(1)
    params = (params + rng.normal(0, 0.02, params.shape)).astype(np.float32)
    n = 300
    pos, nrm = _batch(n, 4)
    q = inputs.random_distributions(7, n, conc=0.5)
    mlp = W.MLP(params, max_batch=512)
    loss, grad = W.guide_learned_train_step(mlp, dev(pos), dev(nrm), dev(q), update=False, want_grad=True)
    gl = float(loss.item())
    g = grad.cpu().numpy().astype(np.float64)
    ol, og = oracle.mlp_grad(params, pos, nrm, LO, 1.0, q, bf16=True)
    assert abs(gl - ol) < 1e-3 * abs(ol) + 1e-5
    for name, (o, k) in SEGMENTS.items():
        a, b = g[o:o + k], og[o:o + k]
        err = np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-12)
        assert err < 0.05, (name, err)
    np.testing.assert_array_equal(mlp.params(), params)  # no update was asked for
    assert mlp.status() == 0


def test_adam_step_matches_oracle_update():
    params = inputs.mlp_init(9)
    n = 256
    pos, nrm = _batch(n, 6)
    q = inputs.random_distributions(8, n)
    mlp = W.MLP(params, max_batch=256)
    W.guide_learned_train_step(mlp, dev(pos), dev(nrm), dev(q), lr=1e-3, update=True)
    got = mlp.params()
    _, og = oracle.mlp_grad(params, pos, nrm, LO, 1.0, q, bf16=True)
    want, _, _ = oracle.adam(params, np.zeros(len(params)), np.zeros(len(params)), og, t=1, lr=1e-3)
    # first Adam step moves each weight by lr * sign(g) (|g| >> eps): compare the moves
    d_got, d_want = got - params, want - params
    assert np.max(np.abs(d_got)) <= 1e-3 * 1.001
    big = np.abs(og) > 1e-6
    assert np.mean(np.sign(d_got[big]) == np.sign(d_want[big])) > 0.97


def test_training_lowers_kl_and_pdf_samples():
    params = inputs.mlp_init(12)
    n = 4096
    pos, nrm = _batch(n, 9)
    # smooth targets: a function of position, so the network can learn them
    _, q = oracle.mlp_forward(inputs.mlp_init(99), pos, nrm, LO, 1.0)
    q = q.astype(np.float32)
    mlp = W.MLP(params, max_batch=n)
    P, Nn, Q = dev(pos), dev(nrm), dev(q)
    l0 = None
    for it in range(150):
        loss, _ = W.guide_learned_train_step(mlp, P, Nn, Q, lr=3e-3)
        if it == 0:
            l0 = float(loss.item())
    l1 = float(W.guide_learned_train_step(mlp, P, Nn, Q, update=False)[0].item())
    assert l1 < 0.5 * l0, (l0, l1)
    pdf, cr, cm = W.guide_learned_build_pdf(mlp, P[:64], Nn[:64], eps=1e-4)
    d, p, c = W.guide_sample(pdf, cr, cm, 32, torch.arange(64, dtype=torch.int32, device="cuda"),
                             dev(inputs.uniforms24(3, (64, 2))))
    assert torch.all(p > 0)
    np.testing.assert_allclose(pdf.sum(dim=1).cpu().numpy() * 4 * np.pi / 1024, 1.0, rtol=1e-5)
    assert mlp.status() == 0
