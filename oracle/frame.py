"""CPU ORACLE -- TEST INFRASTRUCTURE ONLY.

Plain float64 definitions of the two per-path steps that a wavefront frame
adds around the guiding calls:

* the last step of GuideRays (Alg. 3), where each ray of a bin draws its
  next direction from the bin's guided density or from the BSDF (MIS): a
  one-sample mixture of the guided density with cosine-weighted hemisphere
  sampling (the Lambertian BSDF), whose density is exact for every sample so
  the estimator stays unbiased;
* radiance records by back-propagation along a path (Sec. 3.2, Eq. 5):
  the radiance leaving vertex p_k toward p_{k-1} is T(p_n) / T(p_k) times the
  emission found at p_n, summed over every emitter vertex p_n at or after p_k
  (zero when the path finds no emitter after p_k);
* the sample-combination heuristics across frames (Sec. 3.7, Eq. 7): the
  image is the h(i)-weighted average of the per-frame images.

Only the tests import this module.
"""
from __future__ import annotations

import numpy as np


def onb_duff(n):
    """Orthonormal tangent frame (t, b) of unit normals n [m, 3], by the
    branchless construction of Duff et al. 2017 ("Building an orthonormal
    basis, revisited"): s = sign(n_z) (+1 at 0), a = -1 / (s + n_z),
    c = n_x n_y a, t = (1 + s n_x^2 a, s c, -s n_x), b = (c, s + n_y^2 a, -n_y)."""
    n = np.asarray(n, np.float64)
    x, y, z = n[:, 0], n[:, 1], n[:, 2]
    s = np.where(z >= 0.0, 1.0, -1.0)
    a = -1.0 / (s + z)
    c = x * y * a
    t = np.stack([1.0 + s * x * x * a, s * c, -s * x], axis=1)
    b = np.stack([c, s + y * y * a, -y], axis=1)
    return t, b


def cosine_dirs(n, u):
    """Cosine-weighted directions about unit normals n [m, 3] from uniforms
    u [m, 2]: radius sqrt(u0) and angle 2 pi u1 on the unit disk, lifted to
    the hemisphere (Malley's method), so cos(theta) = sqrt(1 - u0) and the
    density is cos(theta) / pi."""
    u = np.asarray(u, np.float64)
    t, b = onb_duff(n)
    r = np.sqrt(u[:, 0])
    phi = 2.0 * np.pi * u[:, 1]
    z = np.sqrt(np.maximum(0.0, 1.0 - u[:, 0]))
    return (t * (r * np.cos(phi))[:, None] + b * (r * np.sin(phi))[:, None]
            + np.asarray(n, np.float64) * z[:, None])


def mixture_pdf(p_guided, n, d, alpha):
    """Density of the one-sample mixture alpha * guided + (1 - alpha) * cosine
    at direction d (the cosine part is zero below the surface)."""
    cs = np.maximum(0.0, np.einsum("ij,ij->i", np.asarray(n, np.float64), np.asarray(d, np.float64)))
    return alpha * np.asarray(p_guided, np.float64) + (1.0 - alpha) * cs / np.pi


def eq5_records(T, Le, nv, Le_seen=None):
    """Radiance records of Eq. 5 for a batch of paths.

    T, Le: [paths, depth] throughput T(p_k) and emitted radiance Le(p_k) of
    vertex k (column k - 1); nv[i]: vertices of path i.  Every vertex k gives
    one record L_k = sum over n >= k of T(p_n) / T(p_k) * Le(p_n): the emitters
    found at or after it, back-propagated; a vertex with no emitter after it
    records zero radiance (the exitance is a count-weighted average of the
    records, so zeros keep it an estimate of the mean, not of the mean over
    lit paths only).  Returns (path, k, L) arrays, ordered by path then k
    (k counted from 1).

    Le_seen (optional, same shape): the radiance of vertex n as the vertices
    before it receive it, when it differs from what the vertex itself emits --
    with light sampling, a light reached by a BSDF/guided sample passes on only
    its MIS-weighted share, while its own record keeps the full emission:
    L_k = Le(p_k) + sum over n > k of T(p_n) / T(p_k) * Le_seen(p_n)."""
    T = np.asarray(T, np.float64)
    Le = np.asarray(Le, np.float64)
    Ls = Le if Le_seen is None else np.asarray(Le_seen, np.float64)
    out_p, out_k, out_L = [], [], []
    for i in range(T.shape[0]):
        for k in range(int(nv[i])):
            out_p.append(i)
            out_k.append(k + 1)
            out_L.append(Le[i, k] + sum(T[i, m] / T[i, k] * Ls[i, m] for m in range(k + 1, int(nv[i]))))
    return np.array(out_p, np.int64), np.array(out_k, np.int64), np.array(out_L, np.float64)


HEURISTICS = ("constant", "linear", "quadratic", "one-two", "discard-first", "pt-first")


def combine_weight(kind, i):
    """h(i) of the sample-combination heuristics (Sec. 3.7) for frame i
    (1-based): constant 1; linear i below 5, else 5; quadratic i^2 below 5,
    else 25; one-two 1 for the first frame, else 2; discard-first 0 for the
    first frame, else 1; PT first weighs its frames equally (its first frame
    is traced without guiding, which the frame itself decides)."""
    i = int(i)
    if i < 1:
        raise ValueError("frames are counted from 1")
    if kind == "linear":
        return float(i) if i < 5 else 5.0
    if kind == "quadratic":
        return float(i * i) if i < 5 else 25.0
    if kind == "one-two":
        return 1.0 if i == 1 else 2.0
    if kind == "discard-first":
        return 0.0 if i == 1 else 1.0
    if kind in ("constant", "pt-first"):
        return 1.0
    raise ValueError(f"unknown heuristic {kind!r}")


def combine_images(S, kind, W=None):
    """Eq. 7: I = sum_i W_i S_i h(i) / sum_i W_i h(i) over the frames' images
    S[i - 1] (any shape after the first axis), summed in frame order in
    float64.  W_i (default 1: every frame is one sample per pixel) weighs a
    frame by its sample count.  A zero weight sum gives a zero image."""
    S = np.asarray(S, np.float64)
    K = S.shape[0]
    W = np.ones(K) if W is None else np.asarray(W, np.float64)
    num = np.zeros(S.shape[1:], np.float64)
    den = 0.0
    for i in range(1, K + 1):
        w = W[i - 1] * combine_weight(kind, i)
        num = num + w * S[i - 1]
        den = den + w
    return num / den if den > 0.0 else np.zeros_like(num)
