"""Pins of the oracle's per-path frame steps: cosine-weighted mixture
sampling (closed forms of Malley's method and of the orthonormal frame,
normalisation, distribution) and Eq. 5 radiance records (hand-worked paths
and the identity between the first vertex's record and the path estimate)."""
import numpy as np

from oracle import frame as OF


def test_onb_is_orthonormal_and_right_handed():
    rng = np.random.default_rng(0)
    n = rng.normal(size=(2000, 3))
    n /= np.linalg.norm(n, axis=1, keepdims=True)
    n[0] = [0, 0, 1]
    n[1] = [0, 0, -1]
    n[2] = [1, 0, 0]
    t, b = OF.onb_duff(n)
    for u, v in ((t, b), (t, n), (b, n)):
        np.testing.assert_allclose(np.einsum("ij,ij->i", u, v), 0, atol=1e-12)
    for u in (t, b):
        np.testing.assert_allclose(np.linalg.norm(u, axis=1), 1, atol=1e-12)
    np.testing.assert_allclose(np.cross(t, b), n, atol=1e-12)


def test_cosine_dirs_special_normals_by_hand():
    u = np.array([[0.25, 0.125], [0.64, 0.75]])
    # n = +z: t = (1, 0, 0), b = (0, 1, 0)
    d = OF.cosine_dirs(np.array([[0.0, 0.0, 1.0]] * 2), u)
    np.testing.assert_allclose(d[0], [0.5 * np.cos(np.pi / 4), 0.5 * np.sin(np.pi / 4), np.sqrt(0.75)], atol=1e-15)
    np.testing.assert_allclose(d[1], [0.0, -0.8, 0.6], atol=1e-15)
    # n = -z: s = -1, a = 1/2, t = (1, 0, 0), b = (0, -1, 0)
    d = OF.cosine_dirs(np.array([[0.0, 0.0, -1.0]] * 2), u)
    np.testing.assert_allclose(d[1], [0.0, 0.8, -0.6], atol=1e-15)


def test_cosine_dirs_cos_theta_closed_form_and_distribution():
    rng = np.random.default_rng(1)
    m = 200_000
    n = rng.normal(size=(m, 3))
    n /= np.linalg.norm(n, axis=1, keepdims=True)
    u = rng.uniform(size=(m, 2))
    d = OF.cosine_dirs(n, u)
    np.testing.assert_allclose(np.linalg.norm(d, axis=1), 1, atol=1e-12)
    c = np.einsum("ij,ij->i", n, d)
    np.testing.assert_allclose(c, np.sqrt(1 - u[:, 0]), atol=1e-12)
    # cos(theta) has CDF c^2 on [0, 1]: chi-square over 20 equal-probability bins
    edges = np.sqrt(np.linspace(0, 1, 21))
    h, _ = np.histogram(c, edges)
    chi2 = np.sum((h - m / 20) ** 2 / (m / 20))
    assert chi2 < 43.8  # 0.999 quantile, 19 dof
    # azimuth uniform about n
    t, b = OF.onb_duff(n)
    phi = np.arctan2(np.einsum("ij,ij->i", b, d), np.einsum("ij,ij->i", t, d)) % (2 * np.pi)
    h, _ = np.histogram(phi, np.linspace(0, 2 * np.pi, 21))
    assert np.sum((h - m / 20) ** 2 / (m / 20)) < 43.8


def test_mixture_pdf_normalised():
    # with a uniform guided density 1/(4 pi) the mixture integrates to 1
    rng = np.random.default_rng(2)
    m = 400_000
    d = rng.normal(size=(m, 3))
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    n = np.tile([[0.0, 0.6, 0.8]], (m, 1))
    p = OF.mixture_pdf(np.full(m, 1 / (4 * np.pi)), n, d, 0.3)
    est = np.mean(p) * 4 * np.pi
    assert abs(est - 1) < 4e-3
    np.testing.assert_allclose(p[np.einsum("ij,ij->i", n, d) < 0], 0.3 / (4 * np.pi), rtol=1e-15)


def test_eq5_hand_paths():
    T = np.array([[1.0, 0.5, 0.2], [1.0, 0.5, 0.25], [1.0, 0.4, 0.1], [1.0, 0.0, 0.0]])
    Le = np.array([[0.0, 0.0, 10.0], [1.0, 0.0, 3.0], [0.0, 0.0, 0.0], [2.0, 0.0, 0.0]])
    nv = np.array([3, 3, 3, 1])
    p, k, L = OF.eq5_records(T, Le, nv)
    np.testing.assert_array_equal(p, [0, 0, 0, 1, 1, 1, 2, 2, 2, 3])
    np.testing.assert_array_equal(k, [1, 2, 3, 1, 2, 3, 1, 2, 3, 1])
    np.testing.assert_allclose(L, [2.0, 4.0, 10.0, 1.75, 1.5, 3.0, 0.0, 0.0, 0.0, 2.0])


def test_eq5_records_after_last_emitter_are_zero():
    T = np.array([[1.0, 0.5, 0.2, 0.1]])
    Le = np.array([[0.0, 4.0, 0.0, 0.0]])
    p, k, L = OF.eq5_records(T, Le, [4])
    np.testing.assert_array_equal(k, [1, 2, 3, 4])
    np.testing.assert_allclose(L, [2.0, 4.0, 0.0, 0.0])


def test_eq5_first_record_is_path_estimate():
    rng = np.random.default_rng(3)
    P, Dm = 300, 5
    f = rng.uniform(0.05, 2.0, (P, Dm))
    f[:, 0] = 1.0
    T = np.cumprod(f, axis=1)
    Le = np.where(rng.uniform(size=(P, Dm)) < 0.3, rng.uniform(0.5, 20, (P, Dm)), 0.0)
    nv = rng.integers(1, Dm + 1, P)
    p, k, L = OF.eq5_records(T, Le, nv)
    est = np.array([np.sum(T[i, :nv[i]] * Le[i, :nv[i]]) for i in range(P)])
    first = k == 1
    np.testing.assert_allclose(L[first], est[p[first]], rtol=1e-12)
    assert np.array_equal(p[first], np.arange(P)) and len(p) == int(np.sum(nv))
    # a record at k and at k + 1 of the same path: L_k = Le_k + (T_{k+1} / T_k) L_{k+1}
    for j in range(len(p) - 1):
        if p[j] == p[j + 1] and k[j + 1] == k[j] + 1:
            i, kk = p[j], k[j] - 1
            np.testing.assert_allclose(L[j], Le[i, kk] + T[i, kk + 1] / T[i, kk] * L[j + 1], rtol=1e-12)


def test_eq5_with_light_sampling_hand_path():
    """With light sampling a light reached by the mixture passes on only its
    MIS-weighted share w Le to the vertices before it, and keeps its full
    emission in its own record; light samples Nee_k add at their vertex."""
    T = np.array([[1.0, 0.5, 0.25]])
    Le = np.array([[0.0, 0.0, 8.0]])
    w = 0.25
    nee = np.array([[0.5, 2.0, 0.0]])
    p, k, L = OF.eq5_records(T, Le + nee, [3], Le_seen=np.array([[0.0, 0.0, w * 8.0]]) + nee)
    # L_3 = 8; L_2 = 2 + (0.25 / 0.5) * 2 = 3; L_1 = 0.5 + 0.5 * 2 + 0.25 * 2 = 2
    np.testing.assert_allclose(L, [2.0, 3.0, 8.0])
    # without a separate seen radiance it is the plain suffix sum
    p2, k2, L2 = OF.eq5_records(T, Le + nee, [3], Le_seen=Le + nee)
    np.testing.assert_allclose(L2, OF.eq5_records(T, Le + nee, [3])[2], rtol=1e-15)
    np.testing.assert_allclose(L2, [0.5 + 1.0 + 2.0, 2.0 + 4.0, 8.0])


# Sample-combination heuristics (Sec. 3.7, Eq. 7).  The weights below are the
# cases the paper prints for frames 1..7; the pins compare the combination with
# library averages of replicated frames, which a wrong weight, index or
# normalisation would not reproduce.
PRINTED = {
    "constant": [1, 1, 1, 1, 1, 1, 1],
    "linear": [1, 2, 3, 4, 5, 5, 5],
    "quadratic": [1, 4, 9, 16, 25, 25, 25],
    "one-two": [1, 2, 2, 2, 2, 2, 2],
    "discard-first": [0, 1, 1, 1, 1, 1, 1],
    "pt-first": [1, 1, 1, 1, 1, 1, 1],
}


def test_combination_weights_are_the_printed_cases():
    assert set(PRINTED) == set(OF.HEURISTICS)
    for kind, h in PRINTED.items():
        assert [OF.combine_weight(kind, i) for i in range(1, 8)] == h, kind
    for kind in OF.HEURISTICS:  # every weight stays at its last printed value
        assert OF.combine_weight(kind, 1000) == PRINTED[kind][-1]


def test_combination_equals_the_mean_of_replicated_frames():
    """Integer weights: Eq. 7 with W = 1 is the plain mean (numpy) of the
    sequence in which frame i appears h(i) times."""
    rng = np.random.default_rng(7)
    K = 7
    S = rng.uniform(0.0, 3.0, (K, 5, 4))
    for kind, h in PRINTED.items():
        rep = np.concatenate([np.repeat(S[i:i + 1], h[i], axis=0) for i in range(K)])
        np.testing.assert_allclose(OF.combine_images(S, kind), rep.mean(axis=0), rtol=1e-13, err_msg=kind)
    # the constant heuristic is numpy's mean; discard-first ignores frame 1
    np.testing.assert_allclose(OF.combine_images(S, "constant"), S.mean(axis=0), rtol=1e-13)
    S2 = S.copy()
    S2[0] = 1e6
    np.testing.assert_array_equal(OF.combine_images(S2, "discard-first"), OF.combine_images(S, "discard-first"))


def test_combination_keeps_constant_images_and_is_unbiased():
    rng = np.random.default_rng(8)
    img = rng.uniform(0.5, 2.0, (3, 3))
    for kind in OF.HEURISTICS:
        np.testing.assert_allclose(OF.combine_images(np.repeat(img[None], 9, axis=0), kind), img, rtol=1e-14)
    # independent unbiased frames (mean 1, different variances) stay unbiased
    trials, K = 20000, 8
    noise = rng.normal(size=(trials, K)) * np.linspace(2.0, 0.5, K)
    for kind in OF.HEURISTICS:
        est = np.array([OF.combine_images(1.0 + noise[t], kind) for t in range(0, trials, 4)])
        se = est.std(ddof=1) / np.sqrt(len(est))
        assert abs(est.mean() - 1.0) < 4 * se, (kind, est.mean(), se)


def test_combination_with_sample_counts():
    """W_i = samples of frame i: the constant heuristic is the per-sample mean
    (numpy's weighted average); a zero weight sum gives a zero image."""
    rng = np.random.default_rng(9)
    S = rng.uniform(size=(5, 6))
    Wn = np.array([1, 4, 2, 8, 3], np.float64)
    np.testing.assert_allclose(OF.combine_images(S, "constant", Wn), np.average(S, axis=0, weights=Wn), rtol=1e-13)
    np.testing.assert_array_equal(OF.combine_images(S[:1], "discard-first"), np.zeros(6))
