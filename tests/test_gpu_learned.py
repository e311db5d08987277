"""Learned proposal on the GPU (tcgen05 forward/backward, Adam) against the
CPU oracle's MLP with its bfloat16-rounding emulation, element by element.

Tolerance.  Both sides round the same quantities to bfloat16 (inputs,
weights, hidden activations, logit and hidden-layer gradients) and the
products of bfloat16 operands are exact; they differ in how sums are
accumulated (float32 on the tensor cores, binary64 in the oracle).  So a
stored value can land on the other side of a bfloat16 rounding boundary and
differ by one unit in the last place: at most 2^-7 of its magnitude (8
significant bits).  Every compared result is a sum (a logit over its 64
hidden inputs, a weight gradient over the batch), and a unit of error in its
terms moves it by at most 2^-7 of M, the sum of its terms' magnitudes:
M = |W4| |h3| + |b4| for a logit, sum over rows of |A| |B| for a weight
gradient dW = A^T B.  The bound is two such units, one for the terms' own
rounding and one for a disagreement further up the network that reaches
them.  The float32 accumulation error (at most ~600 roundings of 2^-24 per
sum) stays two orders below it.  A dropped bias, a transposed block or a
wrong mask moves results by about M itself.  Positions are given with
lo = 0 and size 1, so that p^ = p is exact on both sides and the features
differ only by their own rounding.
"""
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
ULP = 2.0 ** -7
SEGMENTS = {"W1": (0, (64, 80)), "b1": (5120, (64,)), "W2": (5184, (64, 64)), "b2": (9280, (64,)),
            "W3": (9344, (64, 64)), "b3": (13440, (64,)), "W4": (13504, (1024, 64)), "b4": (79040, (1024,))}


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def _batch(n, seed):
    rng = np.random.default_rng(seed)
    pos = rng.uniform(0, 1, (n, 3)).astype(np.float32)
    nrm = rng.normal(size=(n, 3))
    nrm = (nrm / np.linalg.norm(nrm, axis=1, keepdims=True)).astype(np.float32)
    return pos, nrm


def _params(seed, noise=0.05):
    """Initial weights plus noise, so that every bias moves the result."""
    rng = np.random.default_rng(seed)
    p = inputs.mlp_init(seed).astype(np.float64)
    return (p + rng.normal(0, noise, p.shape)).astype(np.float32)


def _split(vec):
    return {k: np.asarray(vec[o:o + int(np.prod(s))], np.float64).reshape(s) for k, (o, s) in SEGMENTS.items()}


def magnitudes(params, tr):
    """M of every compared result (see the module docstring), from the oracle's
    bfloat16-emulated intermediates and the bfloat16 weights both sides use."""
    Wb = _split(oracle.bf16_round(params).astype(np.float64))
    M = {"z": np.abs(tr["h3"]) @ np.abs(Wb["W4"]).T + np.abs(Wb["b4"])}
    if "g4" in tr:
        for w, (a, b) in {"W4": ("g4", "h3"), "W3": ("d3", "h2"), "W2": ("d2", "h1"), "W1": ("d1", "x")}.items():
            M[w] = np.abs(tr[a]).T @ np.abs(tr[b])
            M["b" + w[1]] = np.abs(tr[a]).sum(axis=0)
    return M


@pytest.mark.parametrize("n", [1, 300, 8200])
def test_logits_match_oracle_elementwise(n):
    params = _params(5)
    pos, nrm = _batch(n, 2)
    mlp = W.MLP(params, max_batch=n)
    z = W.guide_learned_logits(mlp, dev(pos), dev(nrm)).cpu().numpy().astype(np.float64)
    q = np.full((n, 1024), 1.0 / 1024, np.float32)
    _, _, tr = oracle.mlp_grad_trace(params, pos, nrm, LO, 1.0, q, bf16=True)
    bound = 2 * ULP * magnitudes(params, {"h3": tr["h3"]})["z"]
    err = np.abs(z - tr["z"])
    worst = np.unravel_index(np.argmax(err / bound), err.shape)
    assert np.all(err <= bound), (worst, z[worst], tr["z"][worst], bound[worst])
    assert mlp.status() == 0


@pytest.mark.parametrize("n", [1, 300, 1000])
def test_pdf_matches_oracle(n):
    """guide_learned_build_pdf (softmax, then the traced path's PDF arithmetic)
    against the oracle's probabilities, within the logits' bound carried
    through the softmax plus float32 roundings (1e-5 relative)."""
    params = _params(7)
    pos, nrm = _batch(n, 12)
    mlp = W.MLP(params, max_batch=1024)
    pdf, cr, cm = W.guide_learned_build_pdf(mlp, dev(pos), dev(nrm), eps=0.0)
    q = np.full((n, 1024), 1.0 / 1024, np.float32)
    _, _, tr = oracle.mlp_grad_trace(params, pos, nrm, LO, 1.0, q, bf16=True)
    z = tr["z"]
    p = np.exp(z - z.max(axis=1, keepdims=True))
    p /= p.sum(axis=1, keepdims=True)
    ez = 2 * ULP * magnitudes(params, {"h3": tr["h3"]})["z"]
    # softmax: dp_c = p_c (dz_c - sum_k p_k dz_k); then float32 exp, sum and PDF roundings
    bound = p * (ez + (p * ez).sum(axis=1, keepdims=True)) + 1e-5 * p
    p_gpu = pdf.cpu().numpy().astype(np.float64) * (4 * np.pi / 1024)
    np.testing.assert_allclose(p_gpu.sum(axis=1), 1.0, rtol=1e-5)
    assert np.all(np.abs(p_gpu - p) <= bound)
    assert mlp.status() == 0


@pytest.mark.parametrize("n", [300, 8200])
def test_gradient_matches_oracle_elementwise(n):
    """Loss and all 80,064 gradient entries.  At 8200 rows the weight
    gradients reduce 65 split-K partial tiles (one per 128 rows) and the rows
    end in a ragged tile."""
    params = _params(8)
    pos, nrm = _batch(n, 4)
    q = inputs.random_distributions(7, n, conc=0.5)
    mlp = W.MLP(params, max_batch=n)
    loss, grad = W.guide_learned_train_step(mlp, dev(pos), dev(nrm), dev(q), update=False, want_grad=True)
    gl = float(loss.item())
    g = _split(grad.cpu().numpy().astype(np.float64))
    ol, og, tr = oracle.mlp_grad_trace(params, pos, nrm, LO, 1.0, q, bf16=True)
    og = _split(og)
    assert abs(gl - ol) < 1e-3 * abs(ol) + 1e-5
    M = magnitudes(params, tr)
    for name in SEGMENTS:
        a, b = g[name], og[name]
        if name == "W1":  # the two padding columns carry no gradient
            assert np.all(a[:, 78:] == 0)
            a, b = a[:, :78], b[:, :78]
        bound = 2 * ULP * (M[name][:, :78] if name == "W1" else M[name])
        err = np.abs(a - b)
        worst = np.unravel_index(np.argmax(err / np.maximum(bound, 1e-30)), err.shape)
        assert np.all(err <= bound), (name, worst, a[worst], b[worst], bound[worst])
    np.testing.assert_array_equal(mlp.params(), params)  # no update was asked for
    assert mlp.status() == 0


def test_adam_steps_match_oracle_by_value():
    """Three Adam steps on a seeded gradient (bias corrections at t = 1, 2, 3):
    the float32 kernel against the oracle's binary64 update of float32
    weights, within two float32 units of each weight plus 1e-5 of the step."""
    params = _params(9)
    rng = np.random.default_rng(3)
    mlp = W.MLP(params, max_batch=128)
    p, m, v = params, np.zeros(len(params)), np.zeros(len(params))
    lr, b1, b2, eps = 1e-3, 0.9, 0.999, 1e-8
    for t in range(1, 4):
        g = (rng.normal(0, 1, len(params)) * np.exp(rng.uniform(-8, 2, len(params)))).astype(np.float32)
        W.mlp_adam_step(mlp, dev(g), lr=lr, beta1=b1, beta2=b2, eps=eps)
        p, m, v = oracle.adam(p, m, v, g.astype(np.float64), t, lr=lr, b1=b1, b2=b2, eps=eps)
        got = mlp.params()
        tol = 2 * np.spacing(np.abs(p).astype(np.float32)).astype(np.float64) + 1e-5 * lr
        assert np.all(np.abs(got.astype(np.float64) - p) <= tol), t
    assert mlp.status() == 0


def test_train_step_update_is_adam_on_its_gradient():
    """guide_learned_train_step with an update equals the same step without one
    followed by mlp_adam_step on the gradient it returned."""
    params = _params(10)
    n = 2048
    pos, nrm = _batch(n, 6)
    q = dev(inputs.random_distributions(8, n))
    a, b = W.MLP(params, max_batch=n), W.MLP(params, max_batch=n)
    W.guide_learned_train_step(a, dev(pos), dev(nrm), q, lr=1e-3, update=True)
    _, g = W.guide_learned_train_step(b, dev(pos), dev(nrm), q, update=False, want_grad=True)
    W.mlp_adam_step(b, g, lr=1e-3)
    pa, pb = a.params(), b.params()
    # the bias sums use float atomics: the two gradients may differ in the last bits
    assert np.max(np.abs(pa - pb)) <= 1e-6
    assert a.status() == 0 and b.status() == 0


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


def test_mixture_estimator_is_unbiased_at_frame_scale():
    """Every fused sample carries its exact mixture density: over the 1.6M rays
    of the 1080p frame (each from its own bin's field), E[1/p] = 4 pi and
    E[cos+/p] = pi within 4 standard errors."""
    w = inputs.frame_spheres(1)
    svo = W.svo_from_scene(w.scene, w.depth)
    W.svo_accumulate(svo, dev(w.rec_pos), dev(w.rec_wout), dev(w.rec_L))
    R = w.ray_pos.shape[0]
    pos, nrm = dev(w.ray_pos), dev(w.ray_nrm)
    r = W.bin_rays(svo, pos, nrm, mode=W.BIN_RUNS, sizes=dev(w.bin_sizes.view(np.int32)), seed=w.seed,
                   bin_cap=len(w.bin_sizes))
    u = dev(inputs.uniforms24(77, (R, 3)))
    d, p = W.guide_build_sample(svo, pos, nrm, r, u, alpha=0.5, N=32, jitter=True, blur=True, seed=w.seed)
    x = (1.0 / p.double()).cpu().numpy()
    c = (torch.clamp((d * nrm).sum(dim=1), min=0).double() / p.double()).cpu().numpy()
    for v, ref in ((x, 4 * np.pi), (c, np.pi)):
        se = v.std(ddof=1) / np.sqrt(len(v))
        assert abs(v.mean() - ref) < 4 * se, (v.mean(), ref, se)
    assert torch.all(p > 0)
