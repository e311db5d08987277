"""Pins of the oracle's product guiding (Sec. 3.6): the product density is
normalised over the sphere, the two-stage sampler draws cells with exactly
that probability (chi-square), its samples evaluate to their own density,
the estimator of a known integral is unbiased, and a uniform field reduces the
product to the blockwise BSDF weights (closed form)."""
import numpy as np

import oracle

N = 32


def _fields(seed, bins=3):
    rng = np.random.default_rng(seed)
    f = rng.gamma(0.5, 1.0, (bins, N, N)).astype(np.float64) + 1e-2
    f[0, 5:9, 20:30] += 40.0  # a bright patch
    pdf = (f / f.sum(axis=(1, 2), keepdims=True) * (N * N) / (4 * np.pi)).astype(np.float32)
    return pdf.reshape(bins, N * N)


def _centres():
    j, i = np.meshgrid(np.arange(N), np.arange(N), indexing="ij")
    uv = np.stack([(i.ravel() + 0.5) * 2 / N - 1, (j.ravel() + 0.5) * 2 / N - 1], 1).astype(np.float32)
    return oracle.octa_decode(uv)


def _unit(v):
    v = np.asarray(v, np.float64)
    return (v / np.linalg.norm(v)).astype(np.float32)


NORMALS = [_unit([0, 0, 1]), _unit([0.3, -0.5, 0.8]), _unit([-1, 0.2, -0.1])]


def test_block_sums_are_sums_of_the_blocks():
    pdf = _fields(1, 2)
    S = oracle.product_block_sums(pdf, N)
    ref = pdf.reshape(2, 8, 4, 8, 4).astype(np.float64).sum(axis=(2, 4)).reshape(2, 64)
    np.testing.assert_allclose(S, ref, rtol=1e-5)


def test_block_weights_closed_form():
    kappa = 2.0 ** -10
    d = oracle.octa_decode(np.array([[(bi + 0.5) * 0.25 - 1, (bj + 0.5) * 0.25 - 1]
                                     for bj in range(8) for bi in range(8)], np.float32))
    for n in NORMALS:
        w = np.array([oracle.product_block_weight(n, B) for B in range(64)])
        ref = np.maximum(d.astype(np.float64) @ n.astype(np.float64), 0) + kappa
        np.testing.assert_allclose(w, ref, rtol=0, atol=2e-7)
        assert np.all(w[ref == kappa] == np.float32(kappa))  # below the horizon: the floor only


def test_product_density_is_normalised():
    pdf = _fields(2)
    S = oracle.product_block_sums(pdf, N)
    dirs = _centres()
    for b in range(3):
        for n in NORMALS:
            p = oracle.product_eval(pdf, S, N, np.full(N * N, b, np.uint32), np.tile(n, (N * N, 1)), dirs)
            assert abs(p.astype(np.float64).sum() * 4 * np.pi / (N * N) - 1) < 1e-5


def test_sampler_chi_square_and_self_consistency():
    pdf = _fields(3)
    S = oracle.product_block_sums(pdf, N)
    rng = np.random.default_rng(4)
    m = 400_000
    n = NORMALS[1]
    u = rng.uniform(0, 1, (m, 2)).astype(np.float32)
    bins = np.zeros(m, np.uint32)
    d, p, c = oracle.product_sample(pdf, S, N, bins, np.tile(n, (m, 1)), u)
    # expected cell probabilities: density at the cell x its solid angle
    pc = oracle.product_eval(pdf, S, N, np.zeros(N * N, np.uint32), np.tile(n, (N * N, 1)), _centres())
    prob = pc.astype(np.float64) * 4 * np.pi / (N * N)
    h = np.bincount(c.astype(np.int64), minlength=N * N)
    keep = prob * m > 20
    chi2 = np.sum((h[keep] - m * prob[keep]) ** 2 / (m * prob[keep]))
    dof = keep.sum() - 1
    assert chi2 < dof + 5 * np.sqrt(2 * dof), (chi2, dof)
    # the returned density is the density of the returned cell, and evaluates back
    np.testing.assert_array_equal(p, pc[c])
    e = oracle.product_eval(pdf, S, N, bins, np.tile(n, (m, 1)), d)
    same_cell = np.isclose(e, p, rtol=0, atol=0)
    assert same_cell.mean() > 0.999


def test_estimator_is_unbiased():
    """E[g / p] = integral of g over the sphere for g = 1 (4 pi) and g = cos+ (pi):
    the product density is positive wherever the field is."""
    pdf = _fields(5)
    S = oracle.product_block_sums(pdf, N)
    rng = np.random.default_rng(6)
    m = 400_000
    for n in NORMALS:
        u = rng.uniform(0, 1, (m, 2)).astype(np.float32)
        d, p, _ = oracle.product_sample(pdf, S, N, np.full(m, 2, np.uint32), np.tile(n, (m, 1)), u)
        for g, ref in ((np.ones(m), 4 * np.pi), (np.maximum(d.astype(np.float64) @ n, 0), np.pi)):
            x = g / p.astype(np.float64)
            se = x.std(ddof=1) / np.sqrt(m)
            assert abs(x.mean() - ref) < 4 * se, (n, x.mean(), ref, se)


def test_uniform_field_reduces_to_the_bsdf_blocks():
    pdf = np.full((1, N * N), 1 / (4 * np.pi), np.float32)
    S = oracle.product_block_sums(pdf, N)
    n = NORMALS[0]
    w = np.array([oracle.product_block_weight(n, B) for B in range(64)], np.float64)
    dirs = _centres()
    p = oracle.product_eval(pdf, S, N, np.zeros(N * N, np.uint32), np.tile(n, (N * N, 1)), dirs)
    # each cell: beta_B / (sum_B beta_B * 4 pi / 64)
    j, i = np.divmod(np.arange(N * N), N)
    B = (j // 4) * 8 + i // 4
    np.testing.assert_allclose(p, w[B] / (w.sum() * 4 * np.pi / 64), rtol=1e-5)
