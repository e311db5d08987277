"""Pins of the oracle's directional stages (Sec. 3.3, 3.5 and the
implementation notes of Sec. 3): own trig against the math library, the
concentric octahedral map against its defining properties, the SVO march
against brute force, the field against the furnace / single-emitter cases,
the CDF and the sampler against closed forms and statistical tests."""
import math
import os

import numpy as np
import pytest
from scipy import stats

import oracle
from paper_2405_06997_gb300 import inputs

FOUR_PI = 4 * math.pi


# ---------------------------------------------------------------- own trig
def test_own_sin_cos_atan_against_libm():
    x = np.linspace(0, math.pi / 4, 2001, dtype=np.float32)
    s = np.array([oracle.sin(v) for v in x])
    c = np.array([oracle.cos(v) for v in x])
    assert np.max(np.abs(s - np.sin(x.astype(np.float64)))) < 2.5e-7
    assert np.max(np.abs(c - np.cos(x.astype(np.float64)))) < 2.5e-7
    q = np.linspace(0, 1, 4001, dtype=np.float32)
    a = np.array([oracle.atan01(v) for v in q])
    assert np.max(np.abs(a - np.arctan(q.astype(np.float64)))) < 3e-7


# ---------------------------------------------------------------- octahedral map
def test_octa_known_points():
    pts = {(0, 0): (0, 0, 1), (1, 0): (1, 0, 0), (-1, 0): (-1, 0, 0), (0, 1): (0, 1, 0),
           (0, -1): (0, -1, 0), (1, 1): (0, 0, -1), (-1, -1): (0, 0, -1)}
    for uv, d in pts.items():
        got = oracle.octa_decode(np.array(uv, np.float32))[0]
        np.testing.assert_allclose(got, d, atol=1e-6)
    enc = oracle.octa_encode(np.array([[0, 0, 1], [1, 0, 0], [0, 1, 0], [-1, 0, 0]], np.float32))
    np.testing.assert_allclose(enc, [[0, 0], [1, 0], [0, 1], [-1, 0]], atol=1e-6)
    e = oracle.octa_encode(np.array([0, 0, -1], np.float32))[0]
    np.testing.assert_allclose(np.abs(e).sum(), 2.0, atol=1e-6)


def test_octa_unit_and_round_trip():
    rng = np.random.default_rng(0)
    uv = rng.uniform(-1, 1, (200000, 2)).astype(np.float32)
    d = oracle.octa_decode(uv)
    assert np.max(np.abs(np.linalg.norm(d.astype(np.float64), axis=1) - 1)) < 1e-6
    back = oracle.octa_encode(d)
    # round trip is exact up to float rounding away from the poles
    far = np.abs(d[:, 2]) < 0.999
    assert np.max(np.abs(back[far] - uv[far])) < 2e-5
    v = rng.normal(size=(200000, 3))
    v = (v / np.linalg.norm(v, axis=1, keepdims=True)).astype(np.float32)
    again = oracle.octa_decode(oracle.octa_encode(v))
    assert np.max(np.abs(again - v)) < 2e-5


def test_octa_edge_mirror():
    """Across the square's edge the map continues mirrored: (1, v) and (1, -v)
    are one direction, likewise (u, 1) and (-u, 1)."""
    t = np.linspace(-1, 1, 101, dtype=np.float32)
    one = np.ones_like(t)
    a = oracle.octa_decode(np.stack([one, t], 1))
    b = oracle.octa_decode(np.stack([one, -t], 1))
    np.testing.assert_allclose(a, b, atol=1e-6)
    a = oracle.octa_decode(np.stack([t, -one], 1))
    b = oracle.octa_decode(np.stack([-t, -one], 1))
    np.testing.assert_allclose(a, b, atol=1e-6)


def test_octa_equal_area_chi_square():
    """Uniform directions fall in every cell of the N x N grid with the same
    probability 1/N^2 (each cell covers 4 pi / N^2 sr)."""
    rng = np.random.default_rng(1)
    N = 8
    v = rng.normal(size=(1_000_000, 3))
    v = (v / np.linalg.norm(v, axis=1, keepdims=True)).astype(np.float32)
    uv = oracle.octa_encode(v).astype(np.float64)
    i = np.clip(np.floor((uv[:, 0] + 1) * N / 2), 0, N - 1).astype(int)
    j = np.clip(np.floor((uv[:, 1] + 1) * N / 2), 0, N - 1).astype(int)
    h = np.bincount(j * N + i, minlength=N * N)
    chi = stats.chisquare(h)
    assert chi.pvalue > 1e-3


# ---------------------------------------------------------------- SVO march
def _slab_first_leaf(leaf_cells, h, o, d, t_skip):
    """Brute force: entry time of the ray into every occupied closed voxel box;
    the answer is the box with the smallest entry time t >= t_skip."""
    lo = leaf_cells * h
    hi = lo + h
    with np.errstate(divide="ignore", invalid="ignore"):
        t0 = (lo - o) / d
        t1 = (hi - o) / d
    tn = np.where(d == 0, np.where((o >= lo) & (o <= hi), -np.inf, np.inf), np.minimum(t0, t1))
    tf = np.where(d == 0, np.where((o >= lo) & (o <= hi), np.inf, -np.inf), np.maximum(t0, t1))
    t_in = tn.max(axis=1)
    t_out = tf.min(axis=1)
    ok = (t_in <= t_out) & (t_in >= t_skip)
    t_eff = np.where(ok, t_in, np.inf)
    k = int(np.argmin(t_eff))
    if not np.isfinite(t_eff[k]):
        return None, None, None
    order = np.sort(t_eff)
    gap = order[1] - order[0] if len(order) > 1 else np.inf
    return k, t_in[k], gap


def test_trace_matches_brute_force_slabs():
    D = 4
    rng = np.random.default_rng(3)
    sc = inputs.cornell_spheres(2, n_spheres=6)
    s = oracle.SVO(sc, D)
    ex = s.export()
    lo = s.level_off
    keys = ex["key"][lo[D]:lo[D + 1]]
    cells = np.array([[(int(k) >> (3 * i + a)) & 1 for a in range(3)] for k in keys for i in range(D)])
    cells = cells.reshape(len(keys), D, 3)
    cells = (cells * (1 << np.arange(D))[None, :, None]).sum(axis=1).astype(np.float64)
    h = 1.0 / (1 << D)
    t_skip = oracle.default_t_skip(1.0, D)
    checked = 0
    for _ in range(600):
        o = rng.uniform(0.15, 0.85, 3).astype(np.float32)
        d = rng.normal(size=3)
        d = (d / np.linalg.norm(d)).astype(np.float32)
        r = s.trace(o[None], d[None], N=16, t_skip=t_skip)
        k, t_in, gap = _slab_first_leaf(cells, h, o.astype(np.float64), d.astype(np.float64),
                                        t_skip)
        if k is None:
            assert r["hit"][0] == 0
            continue
        if gap < 1e-5 or abs(t_in - t_skip) < 1e-5:
            continue  # numerical tie between two boxes: either answer is right
        assert r["hit"][0] == 1
        assert int(r["leaf_key"][0]) == int(keys[k])
        assert abs(float(r["t_entry"][0]) - t_in) < 1e-5
        checked += 1
    assert checked > 400


def test_trace_axis_ray_hits_wall():
    D = 6
    sc = inputs.closed_box(1, D)
    s = oracle.SVO(sc, D)
    o = np.array([[0.5, 0.5, 0.5]], np.float32)
    r = s.trace(o, np.array([[1, 0, 0]], np.float32), N=16)
    assert r["hit"][0] == 1
    assert int(r["leaf_key"][0]) == oracle.morton(63, 32, 32)
    assert float(r["t_entry"][0]) == 63 / 64 - 0.5
    # a wall faces the box centre: the traced side is always side 0
    v = np.random.default_rng(0).normal(size=(2000, 3))
    v = (v / np.linalg.norm(v, axis=1, keepdims=True)).astype(np.float32)
    rr = s.trace(np.repeat(o, len(v), 0), v, N=16)
    assert rr["hit"].all()
    assert (rr["side"] == 0).all()


def test_cos_weight_scales_by_the_absolute_cosine():
    """The optional cos weight multiplies the looked-up value by |N . d| (the
    value stays non-negative on either side)."""
    D = 5
    w = inputs.tiny_box(4)
    s = oracle.SVO(w.scene, D)
    s.accumulate(w.rec_pos, w.rec_wout, w.rec_L)
    rng = np.random.default_rng(6)
    v = rng.normal(size=(500, 3))
    v = (v / np.linalg.norm(v, axis=1, keepdims=True)).astype(np.float32)
    o = np.tile(np.array([[0.4, 0.55, 0.5]], np.float32), (len(v), 1))
    a = s.trace(o, v, N=16)
    b = s.trace(o, v, N=16, cos_weight=True)
    assert a["hit"].all() and np.array_equal(a["node"], b["node"])
    nrm = s.export()["normal"][a["node"]]
    c = np.abs(np.einsum("ij,ij->i", nrm, v).astype(np.float32))
    np.testing.assert_allclose(b["value"], a["value"] * c, rtol=1e-6)
    assert np.all(b["value"] >= 0) and np.any(a["side"] == 0) and np.any(a["value"] > 0)


def test_cone_level_tie_goes_to_the_finer_level():
    """Eq. 6 with A exactly halfway between two squared sides (all values
    dyadic, so nothing rounds): the reading takes the finer level; a
    footprint a little larger or smaller decides for the nearer side."""
    D = 6
    s = oracle.SVO(inputs.closed_box(1, D), D)
    o = np.array([[47 / 64, 0.5, 0.5]], np.float32)
    d = np.array([[1, 0, 0]], np.float32)
    # entry at x = 63/64: t = 1/4, A = t^2 omega = omega / 16
    r = s.trace(o, d, omega=2.5)        # A = 5/32: |1/4 - A| = |1/16 - A| = 3/32
    assert float(r["t_entry"][0]) == 0.25
    assert int(r["level"][0]) == 2
    assert int(s.trace(o, d, omega=2.5 * (1 + 2 ** -20))["level"][0]) == 1
    assert int(s.trace(o, d, omega=2.5 * (1 - 2 ** -20))["level"][0]) == 2
    r = s.trace(o, d, omega=0.625)      # A = 5/128, halfway between 1/16 and 1/64
    assert int(r["level"][0]) == 3


def test_march_ties_step_x_before_y():
    """A ray through a cell edge (equal boundary times on x and y) steps along
    x first: it enters the x-neighbour, so a voxel there is hit, while the
    y-neighbour's side of the edge would miss it."""
    D = 6
    h = 1.0 / (1 << D)
    # a small quad (normal z) inside voxel (21, 20, 20) only
    q = np.array([[2, 20.5 * h, 21.25 * h, 21.75 * h, 20.25 * h, 20.75 * h, 1, 0]], np.float32)
    sc = inputs.Scene(quads=q, spheres=np.zeros((0, 4), np.float32), albedo=np.ones(1, np.float32),
                      emission=np.zeros(1, np.float32), lo=np.zeros(3, np.float32), size=1.0)
    s = oracle.SVO(sc, D)
    assert s.n_nodes == D + 1
    c = np.float32(1 / math.sqrt(2))
    o = np.array([[20.5 * h, 20.5 * h, 20.5 * h]], np.float32)
    r = s.trace(o, np.array([[c, c, 0]], np.float32), N=16, t_skip=0.0)
    assert r["hit"][0] == 1 and int(r["leaf_key"][0]) == oracle.morton(21, 20, 20)
    # mirrored about x = y the same edge leads into the y-neighbour first: no hit
    q2 = q.copy()
    q2[0, 2:6] = [20.25 * h, 20.75 * h, 21.25 * h, 21.75 * h]
    s2 = oracle.SVO(inputs.Scene(quads=q2, spheres=sc.spheres, albedo=sc.albedo, emission=sc.emission,
                                 lo=sc.lo, size=1.0), D)
    r2 = s2.trace(o, np.array([[c, c, 0]], np.float32), N=16, t_skip=0.0)
    assert r2["hit"][0] == 0


def test_cone_level_is_closest_side():
    """Eq. 6: the chosen level's squared side is the closest to A = t^2 omega,
    and the level only gets coarser with distance."""
    D = 6
    s = oracle.SVO(inputs.closed_box(1, D), D)
    rng = np.random.default_rng(2)
    v = rng.normal(size=(3000, 3))
    v = (v / np.linalg.norm(v, axis=1, keepdims=True)).astype(np.float32)
    o = np.tile(np.array([0.3, 0.6, 0.45], np.float32), (len(v), 1))
    N = 16
    r = s.trace(o, v, N=N)
    omega = 4 * math.pi / N ** 2
    A = r["t_entry"].astype(np.float64) ** 2 * omega
    side2 = (0.5 ** np.arange(D + 1)) ** 2
    best = np.argmin(np.abs(side2[None, :] - A[:, None]) - 1e-12 * np.arange(D + 1)[None, :], 1)
    ok = np.abs(np.abs(side2[best] - A) - np.sort(np.abs(side2[None, :] - A[:, None]), 1)[:, 1]) > 1e-6
    assert np.array_equal(r["level"][ok], best[ok])
    order = np.argsort(r["t_entry"])
    assert np.all(np.diff(r["level"][order]) <= 0)


# ---------------------------------------------------------------- field, CDF
def _furnace_svo(D):
    sc = inputs.closed_box(1, D)
    sc.quads = sc.quads[:6]
    s = oracle.SVO(sc, D)
    ex = s.export()
    lo = s.level_off
    keys = ex["key"][lo[D]:lo[D + 1]]
    cells = np.array([[sum(((int(k) >> (3 * i + a)) & 1) << i for i in range(D)) for a in range(3)]
                      for k in keys], np.float64)
    pos = ((cells + 0.5) / (1 << D)).astype(np.float32)
    s.accumulate(pos, ex["normal"][lo[D]:lo[D + 1]], np.ones(len(pos), np.float32))
    return s


@pytest.mark.parametrize("blur", [False, True])
def test_furnace_gives_uniform_pdf(blur):
    s = _furnace_svo(5)
    N = 16
    g = s.guide_build(np.array([[0.5, 0.5, 0.5]], np.float32), [0], N, blur=blur, jitter=True)
    np.testing.assert_array_equal(g["field"], np.float32(1.01))
    np.testing.assert_allclose(g["pdf"], 1 / FOUR_PI, rtol=1e-6)


def test_empty_exitance_gives_uniform_pdf():
    s = oracle.SVO(inputs.closed_box(1, 5), 5)
    s.accumulate(np.zeros((0, 3), np.float32), np.zeros((0, 3), np.float32), np.zeros(0, np.float32))
    g = s.guide_build(np.array([[0.2, 0.7, 0.4]], np.float32), [0], 32, blur=True)
    assert np.all(g["field"] == np.float32(0.01))
    np.testing.assert_allclose(g["pdf"], 1 / FOUR_PI, rtol=1e-6)


def test_single_emitter_peak_on_light():
    """Only light records: the cells looking at the light hold the peak, cells
    looking at the ceiling far from the light hold only epsilon.  (The cone
    query reads a node about t * sqrt(omega) wide, so cells near the light's
    rim may also see it.)"""
    D = 6
    w = inputs.tiny_box(1)
    s = oracle.SVO(w.scene, D)
    light = w.rec_L == 10.0
    s.accumulate(w.rec_pos[light], w.rec_wout[light], w.rec_L[light])
    N = 16
    o = np.array([0.5, 0.5, 0.5], np.float32)
    g = s.guide_build(o[None], [0], N)
    f = g["field"][0]
    ii, jj = np.meshgrid(np.arange(N), np.arange(N))
    uv = np.stack([(ii.ravel() + 0.5) * 2 / N - 1, (jj.ravel() + 0.5) * 2 / N - 1], 1)
    d = oracle.octa_decode(uv.astype(np.float32)).astype(np.float64)
    y = 1 - 0.5 / (1 << D)
    with np.errstate(divide="ignore"):
        t = (y - 0.5) / d[:, 1]
    hit = o + t[:, None] * d
    up = d[:, 1] > 0
    dist = np.maximum(np.abs(hit[:, 0] - 0.5), np.abs(hit[:, 2] - 0.5))
    on_light = up & (dist < 0.15)
    far = up & (dist > 0.15 + 0.25)
    assert on_light.any() and far.any()
    assert np.all(f[on_light] == f.max())
    assert f.max() > 5
    walls_far = ~up
    assert np.all(f[walls_far] == np.float32(0.01))
    assert np.all(f[far & (t < 1.0)] < f.max())


def test_jittered_field_draws_its_offsets_from_the_counter_generator():
    """With jitter, cell c = j N + i of bin b in frame k is queried at the
    octahedral image of ((i + x0) 2/N - 1, (j + x1) 2/N - 1), x0 and x1 the
    24-bit uniforms of counters 2c and 2c + 1 of stream (k, b) under the
    jitter purpose's seed (4 seed + 1); the field is eps plus the cone
    query there.  Rebuilt here from the published generator (SplitMix64
    finaliser, itself pinned to its reference outputs) and single cone
    queries."""
    w = inputs.tiny_box(2)
    s = oracle.SVO(w.scene, w.depth)
    s.accumulate(w.rec_pos, w.rec_wout, w.rec_L)
    N, seed, frame, b, eps = 16, 7, 3, 5, np.float32(1e-2)
    o = w.ray_pos[11:12]
    g = s.guide_build(o, np.array([b]), N, eps=float(eps), jitter=True, blur=False, seed=seed, frame=frame)
    stream = (frame << 32) | b
    x = np.array([oracle.rng_u64(4 * seed + 1, stream, k) >> 40 for k in range(2 * N * N)], np.float64)
    x = (x * 2.0 ** -24).astype(np.float32).reshape(N * N, 2)
    c = np.arange(N * N)
    tn = np.float32(2.0 / N)
    uv = np.stack([((c % N).astype(np.float32) + x[:, 0]) * tn - np.float32(1),
                   ((c // N).astype(np.float32) + x[:, 1]) * tn - np.float32(1)], axis=1).astype(np.float32)
    d = oracle.octa_decode(uv)
    val = s.trace(np.repeat(o, N * N, axis=0), d, N=N)["value"]
    np.testing.assert_array_equal(g["field"][0], eps + val)
    assert not np.array_equal(x[:, 0], x[:, 1])
    # without jitter the same cells are queried at their centres
    g0 = s.guide_build(o, np.array([b]), N, eps=float(eps), jitter=False, blur=False, seed=seed, frame=frame)
    uv0 = np.stack([((c % N) + 0.5) * 2.0 / N - 1, ((c // N) + 0.5) * 2.0 / N - 1], axis=1).astype(np.float32)
    val0 = s.trace(np.repeat(o, N * N, axis=0), oracle.octa_decode(uv0), N=N)["value"]
    np.testing.assert_array_equal(g0["field"][0], eps + val0)


def test_blur_mass_and_kernel():
    rng = np.random.default_rng(0)
    N = 16
    f = rng.uniform(0, 1, N * N).astype(np.float32)
    b = oracle.blur(f, N)
    assert abs(float(b.astype(np.float64).sum()) - float(f.astype(np.float64).sum())) < 1e-4
    const = np.full(N * N, 3.25, np.float32)
    assert np.array_equal(oracle.blur(const, N), const)
    delta = np.zeros(N * N, np.float32)
    delta[5 * N + 7] = 16.0
    got = oracle.blur(delta, N).reshape(N, N)
    k = np.outer([1, 2, 1], [1, 2, 1]).astype(np.float32)
    assert np.array_equal(got[4:7, 6:9], k)
    assert got.sum() == 16.0


def test_blur_wraps_with_octahedral_mirror():
    N = 8
    delta = np.zeros(N * N, np.float32)
    delta[0 * N + 2] = 16.0            # row 0, column 2
    got = oracle.blur(delta, N).reshape(N, N)
    # the row above row 0 is row 0 mirrored: column 2 sends weight to column N-1-2
    # (column pass: 16 / 4 lands on row 0, column 5; row pass keeps half of it there)
    assert got[0, N - 1 - 2] == 2.0 and got[0, N - 1 - 2 - 1] == 1.0 and got[0, N - 1 - 2 + 1] == 1.0
    # the same at the bottom edge, and across the left and right edges (rows mirrored)
    for (r, c), (rr, cc) in {((N - 1, 2), (N - 1, N - 3)), ((1, 0), (N - 2, 0)), ((1, N - 1), (N - 2, N - 1))}:
        delta = np.zeros(N * N, np.float32)
        delta[r * N + c] = 16.0
        got = oracle.blur(delta, N).reshape(N, N)
        assert got[rr, cc] == 2.0, (r, c)
        assert got.sum() == 16.0
    assert got.sum() == 16.0


def test_warp_scan_exact_on_integers_and_close_on_reals():
    rng = np.random.default_rng(0)
    for n in (8, 16, 32, 64, 128):
        x = rng.integers(0, 1000, n).astype(np.float32)
        assert np.array_equal(oracle.warp_scan(x), np.cumsum(x.astype(np.int64)).astype(np.float32))
        y = rng.uniform(0, 1, n).astype(np.float32)
        np.testing.assert_allclose(oracle.warp_scan(y), np.cumsum(y.astype(np.float64)), rtol=1e-6)


@pytest.mark.parametrize("N", [16, 32, 64])
def test_pdf_normalised_and_cdf_monotone(N):
    rng = np.random.default_rng(N)
    f = (rng.gamma(0.3, 1.0, N * N) + 0.01).astype(np.float32)
    pdf, cr, cm = oracle.pdf_cdf(f, N)
    assert abs(float(pdf.astype(np.float64).sum()) * FOUR_PI / N ** 2 - 1) < 1e-6
    assert np.all(np.diff(cr.reshape(N, N), axis=1) >= 0)
    assert np.all(np.diff(cm) >= 0)
    assert cm[-1] > 0
    c = np.full(N * N, 0.7, np.float32)
    pc, _, _ = oracle.pdf_cdf(c, N)
    np.testing.assert_allclose(pc, 1 / FOUR_PI, rtol=1e-6)


# ---------------------------------------------------------------- sampling
def _random_guide(N, seed, nb=1):
    rng = np.random.default_rng(seed)
    fs = (rng.gamma(0.4, 1.0, (nb, N * N)) + 0.01).astype(np.float32)
    out = [oracle.pdf_cdf(f, N) for f in fs]
    return (np.stack([o[0] for o in out]), np.stack([o[1] for o in out]),
            np.stack([o[2] for o in out]))


def test_cdf_stays_monotone_where_the_tree_scan_does_not():
    """Fields whose values span many orders of magnitude make the tree-shaped
    warp scan round an entry below its predecessor; the CDFs still never
    decrease (the running maximum), and equal the scan wherever it did not."""
    rng = np.random.default_rng(0)
    N = 32
    hit = 0
    for trial in range(40):
        f = (rng.gamma(0.3, 1.0, N * N) * 10.0 ** rng.integers(-6, 3, N * N)).astype(np.float32)
        rows = np.stack([oracle.warp_scan(f[j * N:(j + 1) * N]) for j in range(N)])
        hit += int(np.any(np.diff(rows, axis=1) < 0))
        pdf, cr, cm = oracle.pdf_cdf(f, N)
        cr = cr.reshape(N, N)
        assert np.all(np.diff(cr, axis=1) >= 0) and np.all(np.diff(cm) >= 0)
        np.testing.assert_array_equal(cr, np.maximum.accumulate(rows, axis=1))
    assert hit > 10


def test_sampler_chi_square():
    N = 16
    pdf, cr, cm = _random_guide(N, 0)
    u = inputs.uniforms24(5, (1_000_000, 2))
    d, p, cell = oracle.guide_sample(pdf, cr, cm, N, np.zeros(len(u), np.uint32), u)
    h = np.bincount(cell, minlength=N * N)
    expect = pdf[0].astype(np.float64) * FOUR_PI / N ** 2
    expect = expect / expect.sum() * len(u)
    assert stats.chisquare(h, expect).pvalue > 1e-3
    np.testing.assert_array_equal(p, pdf[0][cell])


def test_sample_eval_consistency_and_bracket():
    N = 32
    pdf, cr, cm = _random_guide(N, 1, nb=3)
    n = 200_000
    bins = (np.arange(n) % 3).astype(np.uint32)
    u = inputs.uniforms24(6, (n, 2))
    d, p, cell = oracle.guide_sample(pdf, cr, cm, N, bins, u)
    e = oracle.guide_eval_pdf(pdf, N, bins, d)
    # directions away from cell borders evaluate to the density they were drawn with
    uv = oracle.octa_encode(d).astype(np.float64)
    fr = (uv + 1) * N / 2
    interior = (np.abs(fr - np.rint(fr)) > 1e-3).all(axis=1)
    assert np.mean(e[interior] == p[interior]) == 1.0
    assert interior.mean() > 0.9
    # the chosen row and column bracket the targets
    r, c = cell.astype(np.int64) // N, cell.astype(np.int64) % N
    t0 = u[:, 0] * cm[bins, N - 1]
    assert np.all(cm[bins, r] > t0)
    assert np.all(np.where(r > 0, cm[bins, np.maximum(r - 1, 0)] <= t0, True))
    crr = cr.reshape(3, N, N)
    t1 = u[:, 1] * crr[bins, r, N - 1]
    assert np.all(crr[bins, r, c] > t1)
    assert np.all(np.where(c > 0, crr[bins, r, np.maximum(c - 1, 0)] <= t1, True))


def test_sampler_skips_empty_cells_even_at_u_zero():
    """Rows and columns without mass are never chosen, also when a uniform is
    exactly 0 (the first entry strictly greater than the target)."""
    N = 16
    rng = np.random.default_rng(3)
    f = rng.gamma(0.5, 1.0, (N, N)).astype(np.float32)
    f[:3] = 0.0          # empty first rows
    f[:, :2] = 0.0       # empty first columns
    f[7] = 0.0           # an empty row inside
    pdf, cr, cm = oracle.pdf_cdf(f.ravel(), N)
    u = inputs.uniforms24(8, (20000, 2))
    u[:50] = 0.0
    u[50:100, 0] = 0.0
    u[100:150, 1] = 0.0
    d, p, cell = oracle.guide_sample(pdf[None], cr[None], cm[None], N, np.zeros(len(u), np.uint32), u)
    assert np.all(p > 0)
    assert np.all(f.ravel()[cell] > 0)


def test_sample_offsets_inside_the_cell_are_uniform_and_independent():
    """Within its cell a sample's position on the octahedral square is uniform
    (the density is constant over the cell) and its two offsets are
    independent: Kolmogorov-Smirnov against U(0, 1) and their correlation."""
    N = 16
    pdf, cr, cm = _random_guide(N, 4)
    n = 200_000
    u = inputs.uniforms24(9, (n, 2))
    d, p, cell = oracle.guide_sample(pdf, cr, cm, N, np.zeros(n, np.uint32), u)
    uv = (oracle.octa_encode(d).astype(np.float64) + 1.0) * N / 2
    a = uv[:, 0] - (cell % N)
    b = uv[:, 1] - (cell // N)
    ok = (a > -1e-4) & (a < 1 + 1e-4) & (b > -1e-4) & (b < 1 + 1e-4)
    assert ok.mean() > 0.999
    a, b = np.clip(a[ok], 0, 1), np.clip(b[ok], 0, 1)
    assert stats.kstest(a, "uniform").pvalue > 1e-3
    assert stats.kstest(b, "uniform").pvalue > 1e-3
    assert abs(np.corrcoef(a, b)[0, 1]) < 0.02


def test_guided_estimator_unbiased():
    """E[f / p] over guided samples equals the integral of f over the sphere:
    4 pi for f = 1 and pi for f = max(0, cos theta)."""
    N = 16
    pdf, cr, cm = _random_guide(N, 2)
    n = 1_000_000
    u = inputs.uniforms24(7, (n, 2))
    d, p, _ = oracle.guide_sample(pdf, cr, cm, N, np.zeros(n, np.uint32), u)
    for f, want in ((np.ones(n), FOUR_PI), (np.maximum(d[:, 2], 0).astype(np.float64), math.pi)):
        est = f / p.astype(np.float64)
        m, se = est.mean(), est.std() / math.sqrt(n)
        assert abs(m - want) < 3.5 * se + 1e-4 * want


# ---------------------------------------------------------------- Table 2
def test_table2_pdf_cdf_memory():
    path = os.path.join(os.path.dirname(__file__), "golden", "table2_pdf_cdf_memory.txt")
    rows = [l.split() for l in open(path) if l.strip() and not l.startswith("#")]
    for scene, bins, N, mb in rows:
        bins, N = int(bins), int(N)
        pdf = np.zeros((1, N * N), np.float32)
        cdf_row = np.zeros((1, N * N), np.float32)
        per_bin = pdf.nbytes + cdf_row.nbytes
        got = bins * per_bin / 1e6
        digits = len(mb.split(".")[1])
        assert round(got, digits) == float(mb), (scene, got, mb)
