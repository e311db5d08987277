"""Pins of the CPU oracle's SVO stages against facts that do not come from
the oracle: closed forms, brute force on tiny grids, special cases and
library routines (Sec. 3.2 of the paper)."""
import numpy as np
import pytest

import oracle
from paper_2405_06997_gb300 import inputs


def _decode(key, D):
    """Morton decode by plain bit extraction (x -> bit 3i, y -> 3i+1, z -> 3i+2)."""
    x = y = z = 0
    for i in range(D):
        x |= ((key >> (3 * i)) & 1) << i
        y |= ((key >> (3 * i + 1)) & 1) << i
        z |= ((key >> (3 * i + 2)) & 1) << i
    return x, y, z


# ---------------------------------------------------------------- Morton keys
def test_morton_is_bijective_and_nested():
    D = 4
    keys = {}
    for x in range(16):
        for y in range(16):
            for z in range(16):
                k = oracle.morton(x, y, z)
                assert k < 1 << (3 * D)
                keys[k] = (x, y, z)
                # nesting: the key's prefix is the key of the parent cell
                for m in range(1, D + 1):
                    assert k >> (3 * m) == oracle.morton(x >> m, y >> m, z >> m)
    assert len(keys) == 1 << (3 * D)
    assert all(_decode(k, D) == v for k, v in keys.items())


def test_morton_axis_order():
    assert oracle.morton(1, 0, 0) == 1
    assert oracle.morton(0, 1, 0) == 2
    assert oracle.morton(0, 0, 1) == 4
    assert oracle.morton(2047, 2047, 2047) == (1 << 33) - 1


# ---------------------------------------------------------------- voxelisation
@pytest.mark.parametrize("D", [3, 4, 5, 6])
def test_closed_box_shell_count(D):
    sc = inputs.closed_box(1, D)
    sc.quads = sc.quads[:6]  # walls only
    s = oracle.SVO(sc, D)
    leaves = int(s.level_off[D + 1] - s.level_off[D])
    assert leaves == (1 << 3 * D) - ((1 << D) - 2) ** 3


def test_single_quad_leaf_count():
    D = 5
    q = np.array([[2, 0.4, 0.1, 0.55, 0.2, 0.9, 1.0, 0.0]], np.float32)
    sc = inputs.Scene(quads=q, spheres=np.zeros((0, 4), np.float32), albedo=np.ones(1, np.float32),
                      emission=np.zeros(1, np.float32), lo=np.zeros(3, np.float32), size=1.0)
    s = oracle.SVO(sc, D)
    # the closed extents [0.1, 0.55] x [0.2, 0.9] cover cells floor(32 * .) inclusive
    n1 = int(np.floor(0.55 * 32)) - int(np.floor(0.1 * 32)) + 1
    n2 = int(np.floor(0.9 * 32)) - int(np.floor(0.2 * 32)) + 1
    assert int(s.level_off[D + 1] - s.level_off[D]) == n1 * n2


def test_sphere_voxels_brute_force():
    """Sample each closed voxel box densely: if sampled distances to the centre
    straddle r the surface crosses the box (must be occupied); if all sampled
    distances are clear of r by more than the sampling gap it cannot (must be
    empty).  Voxels in between are not decided by sampling and are skipped."""
    D = 4
    c = np.array([0.47, 0.52, 0.55])
    r = 0.31
    sc = inputs.single_sphere(c, r)
    s = oracle.SVO(sc, D)
    ex = s.export()
    occ = set(int(k) for k in ex["key"][s.level_off[D]:s.level_off[D + 1]])
    h = 1.0 / 16
    g = np.linspace(0, 1, 9)
    pts = np.stack(np.meshgrid(g, g, g, indexing="ij"), -1).reshape(-1, 3) * h
    gap = h * np.sqrt(3) / 8
    decided = 0
    for x in range(16):
        for y in range(16):
            for z in range(16):
                p = pts + np.array([x, y, z]) * h
                dist = np.linalg.norm(p - c, axis=1)
                k = oracle.morton(x, y, z)
                if dist.min() <= r <= dist.max():
                    assert k in occ
                    decided += 1
                elif dist.min() > r + gap or dist.max() < r - gap:
                    assert k not in occ
                    decided += 1
    assert decided > 3800  # of 4096


# ---------------------------------------------------------------- node layout
def test_node_layout_matches_coordinate_sets():
    w = inputs.tiny_box(3)
    D = w.depth
    s = oracle.SVO(w.scene, D)
    ex = s.export()
    lo = s.level_off
    leaves = [_decode(int(k), D) for k in ex["key"][lo[D]:lo[D + 1]]]
    for l in range(D + 1):
        sh = D - l
        ref = sorted(set((x >> sh, y >> sh, z >> sh) for x, y, z in leaves),
                     key=lambda c: oracle.morton(*c))
        got = [_decode(int(k), l) for k in ex["key"][lo[l]:lo[l + 1]]]
        assert got == ref
    for l in range(D):
        m = ex["child_mask"][lo[l]:lo[l + 1]]
        assert int(np.unpackbits(m).sum()) == int(lo[l + 2] - lo[l + 1])
    # parent / first_child consistency by coordinates
    for node in range(lo[1], lo[D + 1]):
        p = int(ex["parent"][node])
        assert ex["key"][node] >> np.uint64(3) == ex["key"][p]
        fc = int(ex["first_child"][p])
        k = int(ex["key"][node]) & 7
        below = bin(int(ex["child_mask"][p]) & ((1 << k) - 1)).count("1")
        assert fc + below == node
    assert ex["leaf_count"][0] == lo[D + 1] - lo[D]


# ---------------------------------------------------------------- normals
def test_wall_normals_exact():
    D = 5
    sc = inputs.closed_box(1, D)
    sc.quads = sc.quads[:6]
    s = oracle.SVO(sc, D)
    ex = s.export()
    lo = s.level_off
    res = 1 << D
    for node in range(lo[D], lo[D + 1]):
        x, y, z = _decode(int(ex["key"][node]), D)
        inner = [0 < c < res - 1 for c in (x, y, z)]
        if sum(inner) != 2:
            continue  # edges and corners mix walls
        expect = np.zeros(3, np.float32)
        for a, c in enumerate((x, y, z)):
            if not inner[a]:
                expect[a] = 1.0 if c == 0 else -1.0
        np.testing.assert_array_equal(ex["normal"][node], expect)


def test_sphere_normals_radial():
    D = 5
    c = np.array([0.5, 0.5, 0.5])
    s = oracle.SVO(inputs.single_sphere(c, 0.3), D)
    ex = s.export()
    lo = s.level_off
    h = 1.0 / (1 << D)
    for node in range(lo[D], lo[D + 1]):
        v = (np.array(_decode(int(ex["key"][node]), D)) + 0.5) * h - c
        v /= np.linalg.norm(v)
        assert float(ex["normal"][node] @ v) > 1 - 1e-6


def test_inner_normals_are_leaf_count_weighted_means_of_one_cluster():
    """Where all of a node's children have normals within 90 degrees of one
    another, k-means keeps them in one cluster, so the node's normal is the
    normalised mean of the children's normals weighted by their leaf counts."""
    sc = inputs.cornell_spheres(3, n_spheres=20)
    D = 6
    s = oracle.SVO(sc, D)
    ex = s.export()
    lo = ex["level_off"]
    n = ex["normal"].astype(np.float64)
    checked = unequal = 0
    for node in range(int(lo[D])):
        ch = ex["first_child"][node] + np.arange(bin(int(ex["child_mask"][node])).count("1"))
        cn = n[ch]
        if len(ch) < 2 or np.any(cn @ cn.T <= 0.05):
            continue
        wts = ex["leaf_count"][ch].astype(np.float64)
        m = (wts[:, None] * cn).sum(axis=0)
        np.testing.assert_allclose(n[node], m / np.linalg.norm(m), atol=2e-6)
        checked += 1
        unequal += int(wts.min() != wts.max() and np.abs(cn - cn[0]).max() > 1e-3)
    assert checked > 200 and unequal > 50


def test_kmeans_opposite_normals_do_not_cancel():
    n = np.array([[0, 0, 1], [0, 0, -1]] * 3, np.float32)
    out = oracle.kmeans2(n, np.ones(6, np.float32))
    assert abs(abs(float(out[2])) - 1.0) < 1e-7


def test_kmeans_matches_sklearn_lloyd():
    KMeans = pytest.importorskip("sklearn.cluster").KMeans
    rng = np.random.default_rng(5)
    for trial in range(20):
        m = int(rng.integers(2, 12))
        # two groups around +a and -a (the first point in +a): both clusters stay
        # populated, so the library's empty-cluster relocation never triggers
        a = rng.normal(size=3)
        sign = np.where(rng.uniform(size=(m, 1)) < 0.6, 1.0, -1.0)
        sign[0] = 1.0
        sign[1] = -1.0
        pts = sign * a + 0.4 * np.linalg.norm(a) * rng.normal(size=(m, 3))
        pts /= np.linalg.norm(pts, axis=1, keepdims=True)
        pts = pts.astype(np.float32)
        w = rng.integers(1, 5, m).astype(np.float32)
        init = np.stack([pts[0], -pts[0]]).astype(np.float64)
        km = KMeans(n_clusters=2, init=init, n_init=1, max_iter=4, tol=0.0,
                    algorithm="lloyd").fit(pts.astype(np.float64), sample_weight=w)
        c0 = km.cluster_centers_[0]
        if np.linalg.norm(c0) == 0:
            continue
        got = oracle.kmeans2(pts, w)
        np.testing.assert_allclose(got, c0 / np.linalg.norm(c0), atol=2e-6)


def test_kmeans_runs_four_rounds():
    """Widely spread normals whose assignment still changes after the first
    round: the result is the library's after four Lloyd rounds, not one.  Cases
    where some round leaves a cluster empty are skipped (the library relocates
    an empty cluster, the reading here keeps its centroid)."""
    KMeans = pytest.importorskip("sklearn.cluster").KMeans
    import warnings
    rng = np.random.default_rng(11)
    checked = 0
    for trial in range(400):
        m = int(rng.integers(6, 30))
        a = rng.normal(size=3)
        pts = a + 1.2 * np.linalg.norm(a) * rng.normal(size=(m, 3))
        pts = (pts / np.linalg.norm(pts, axis=1, keepdims=True)).astype(np.float32)
        w = rng.integers(1, 5, m).astype(np.float32)
        init = np.stack([pts[0], -pts[0]]).astype(np.float64)
        fits = {}
        with warnings.catch_warnings():
            warnings.simplefilter("ignore")
            for it in (1, 2, 3, 4):
                fits[it] = KMeans(n_clusters=2, init=init, n_init=1, max_iter=it, tol=0.0,
                                  algorithm="lloyd").fit(pts.astype(np.float64), sample_weight=w)
        d = ((pts[:, None, :].astype(np.float64) - init[None]) ** 2).sum(axis=2)
        first = (d[:, 0] > d[:, 1]).astype(np.int64)  # the first round's assignment, from the initial centroids
        if any(np.bincount(f.labels_, minlength=2).min() == 0 for f in fits.values()) or \
                np.bincount(first, minlength=2).min() == 0:
            continue
        c1, c4 = (fits[k].cluster_centers_[0] for k in (1, 4))
        c1, c4 = c1 / np.linalg.norm(c1), c4 / np.linalg.norm(c4)
        if np.linalg.norm(c1 - c4) < 1e-3:
            continue
        np.testing.assert_allclose(oracle.kmeans2(pts, w), c4, atol=2e-6)
        checked += 1
        if checked == 6:
            break
    assert checked == 6


# ---------------------------------------------------------------- UpdateExitance
def _q(L):
    Lc = np.where(L > 0, np.minimum(L, np.float32(2 ** 24)), 0).astype(np.float32)
    return np.rint(Lc.astype(np.float64) * 2.0 ** 20).astype(np.uint64)


def test_accumulate_conserves_sums_and_counts():
    w = inputs.tiny_box(2)
    s = oracle.SVO(w.scene, w.depth)
    s.accumulate(w.rec_pos, w.rec_wout, w.rec_L)
    e = s.exitance()
    q = _q(w.rec_L)
    total = int(q.astype(object).sum())
    assert int(e["acc_sum"].astype(object).sum()) == total
    assert int(e["acc_cnt"].sum()) == len(q)
    assert int(e["tot_sum"][0].astype(object).sum()) == total  # root holds everything
    assert int(e["tot_cnt"][0].sum()) == len(q)


def test_record_quantisation_clamps_and_rounds_to_even():
    """L is clamped to [0, 2^24] (NaN -> 0) and quantised to the nearest
    multiple of 2^-20, halfway cases to even; every record counts."""
    D = 4
    q = np.array([[1, 0.5, 0.0, 1.0, 0.0, 1.0, 1.0, 0.0]], np.float32)
    sc = inputs.Scene(quads=q, spheres=np.zeros((0, 4), np.float32), albedo=np.ones(1, np.float32),
                      emission=np.zeros(1, np.float32), lo=np.zeros(3, np.float32), size=1.0)
    cases = [(1e9, 1 << 44), (2.0 ** 24, 1 << 44), (-5.0, 0), (float("nan"), 0), (0.5 * 2 ** -20, 0),
             (1.5 * 2 ** -20, 2), (2.5 * 2 ** -20, 2), (3.0, 3 << 20)]
    for L, want in cases:
        s = oracle.SVO(sc, D)
        s.accumulate(np.array([[0.3, 0.5, 0.7]], np.float32), np.array([[0, 1, 0]], np.float32),
                     np.array([L], np.float32))
        e = s.exitance()
        assert int(e["acc_sum"].sum()) == want, L
        assert int(e["acc_cnt"].sum()) == 1


def test_accumulate_brute_force_counts_and_sides():
    """Records away from voxel boundaries land in the voxel holding them; walls'
    records leave toward the inside, so all of them are on side 0."""
    w = inputs.tiny_box(4)
    D = w.depth
    s = oracle.SVO(w.scene, D)
    s.accumulate(w.rec_pos, w.rec_wout, w.rec_L)
    e = s.exitance()
    ex = s.export()
    g = w.rec_pos.astype(np.float64) * (1 << D)
    inplane = np.abs(g - np.rint(g))
    # keep records whose in-plane coordinates are clear of voxel boundaries
    on_plane = inplane < 1e-9
    clear = (np.where(on_plane, 1.0, inplane) > 1e-4).all(axis=1)
    cells = np.minimum(np.floor(g), (1 << D) - 1).astype(np.int64)
    lo = s.level_off
    key_to_node = {int(k): i for i, k in enumerate(ex["key"][lo[D]:lo[D + 1]], start=int(lo[D]))}
    want = {}
    for c, ok in zip(cells, clear):
        if ok:
            n = key_to_node[oracle.morton(*c)]
            want[n] = want.get(n, 0) + 1
    # nodes that only hold clear records must match exactly
    all_nodes = {}
    for c in cells:
        n = key_to_node.get(oracle.morton(*c))
        all_nodes[n] = all_nodes.get(n, 0) + 1
    checked = 0
    for n, k in want.items():
        if all_nodes[n] == k:
            assert int(e["acc_cnt"][n].sum()) == k
            checked += 1
    assert checked > 1000
    # leaves inside a wall (axis-aligned normal) only see side 0
    axis_aligned = np.abs(ex["normal"]).max(axis=1) == 1.0
    assert int(e["acc_cnt"][axis_aligned, 1].sum()) == 0
    assert int(e["acc_cnt"][axis_aligned, 0].sum()) > 0.9 * len(w.rec_L)


def test_bottom_up_average_single_wall():
    """All normals equal: every side-0 sum flows to the root's side 0, whose
    value is the mean of the quantised records."""
    D = 5
    q = np.array([[1, 0.0, 0.0, 1.0, 0.0, 1.0, 1.0, 0.0]], np.float32)
    sc = inputs.Scene(quads=q, spheres=np.zeros((0, 4), np.float32), albedo=np.ones(1, np.float32),
                      emission=np.zeros(1, np.float32), lo=np.zeros(3, np.float32), size=1.0)
    s = oracle.SVO(sc, D)
    rng = np.random.default_rng(0)
    n = 5000
    pos = np.stack([rng.uniform(0, 1, n), np.zeros(n), rng.uniform(0, 1, n)], 1).astype(np.float32)
    wout = np.tile(np.array([0, 1, 0], np.float32), (n, 1))
    L = rng.uniform(0, 5, n).astype(np.float32)
    s.accumulate(pos, wout, L)
    e = s.exitance()
    qq = _q(L)
    assert int(e["tot_sum"][0, 0]) == int(qq.astype(object).sum())
    assert int(e["tot_cnt"][0, 0]) == n
    mean = float(np.float32(np.float32(int(qq.astype(object).sum())) * np.float32(2 ** -20)) /
                 np.float32(n))
    assert e["value"][0, 0] == np.float32(mean)
    assert e["value"][0, 1] == e["value"][0, 0]   # empty side takes the other side


def test_furnace_values_are_one():
    D = 5
    sc = inputs.closed_box(1, D)
    sc.quads = sc.quads[:6]
    s = oracle.SVO(sc, D)
    ex = s.export()
    lo = s.level_off
    keys = ex["key"][lo[D]:lo[D + 1]]
    cells = np.array([_decode(int(k), D) for k in keys], np.float64)
    pos = ((cells + 0.5) / (1 << D)).astype(np.float32)
    nrm = ex["normal"][lo[D]:lo[D + 1]]
    s.accumulate(pos, nrm, np.ones(len(pos), np.float32))
    v = s.exitance()["value"]
    assert np.all(v == 1.0)


def _subtree_index(ex, D):
    """For every level l and every node at a level >= l: the index of its
    ancestor at level l, from the Morton keys alone (key >> 3 (l' - l))."""
    lo = ex["level_off"]
    keys = ex["key"]
    anc = {}
    for l in range(D + 1):
        lk = keys[lo[l]:lo[l + 1]]
        for m in range(l, D + 1):
            mk = keys[lo[m]:lo[m + 1]] >> np.uint64(3 * (m - l))
            pos = np.searchsorted(lk, mk)
            assert np.array_equal(lk[pos], mk)
            anc[l, m] = lo[l] + pos
    return anc


def test_subtree_totals_are_conserved():
    """Every node's totals (both sides) = the records landed anywhere in its
    subtree, with the subtree taken from the keys (brute force).  Records in
    free space stay at the deepest existing node above them, so inner nodes
    hold records of their own too."""
    w = inputs.tiny_box(3)
    D = w.depth
    s = oracle.SVO(w.scene, D)
    rng = np.random.default_rng(3)
    m = 20000
    free = rng.uniform(0.2, 0.8, (m, 3)).astype(np.float32)
    d = rng.normal(size=(m, 3))
    d = (d / np.linalg.norm(d, axis=1, keepdims=True)).astype(np.float32)
    pos = np.concatenate([w.rec_pos, free])
    s.accumulate(pos, np.concatenate([w.rec_wout, d]), np.concatenate([w.rec_L, rng.uniform(0, 3, m).astype(np.float32)]))
    e, ex = s.exitance(), s.export()
    lo = ex["level_off"]
    anc = _subtree_index(ex, D)
    acc_s = e["acc_sum"].sum(axis=1, dtype=np.uint64)
    acc_c = e["acc_cnt"].sum(axis=1, dtype=np.uint64)
    want_s = np.zeros(s.n_nodes, np.uint64)
    want_c = np.zeros(s.n_nodes, np.uint64)
    for (l, m), a in anc.items():
        np.add.at(want_s, a, acc_s[lo[m]:lo[m + 1]])
        np.add.at(want_c, a, acc_c[lo[m]:lo[m + 1]])
    np.testing.assert_array_equal(e["tot_sum"].sum(axis=1, dtype=np.uint64), want_s)
    np.testing.assert_array_equal(e["tot_cnt"].sum(axis=1, dtype=np.uint64), want_c)
    assert int(want_c[0]) == len(pos)
    inner = np.arange(s.n_nodes) < lo[D]
    assert int(acc_c[inner].sum()) > m // 2   # most free-space records sit on inner nodes


def test_sides_follow_the_direction_records_leave_in():
    """Two parallel quads facing away from each other (normals -y and +y) and
    records leaving them in uniformly random directions: at every node, the
    side whose direction is +y (the node's normal, or its negation for side 1)
    holds exactly the records of its subtree that leave with w_y > 0, whatever
    the normals of the levels in between."""
    D = 5
    h = 1.0 / (1 << D)
    q = np.array([[1, 10.5 * h, 0.1, 0.9, 0.1, 0.9, -1, 0],
                  [1, 21.5 * h, 0.1, 0.9, 0.1, 0.9, +1, 0]], np.float32)
    sc = inputs.Scene(quads=q, spheres=np.zeros((0, 4), np.float32), albedo=np.ones(2, np.float32),
                      emission=np.zeros(2, np.float32), lo=np.zeros(3, np.float32), size=1.0)
    s = oracle.SVO(sc, D)
    rng = np.random.default_rng(12)
    n = 20000
    which = rng.integers(0, 2, n)
    pos = np.stack([rng.uniform(0.1, 0.9, n), q[which, 1], rng.uniform(0.1, 0.9, n)], 1).astype(np.float32)
    wout = rng.normal(size=(n, 3))
    wout = (wout / np.linalg.norm(wout, axis=1, keepdims=True)).astype(np.float32)
    L = rng.uniform(0, 4, n).astype(np.float32)
    s.accumulate(pos, wout, L)
    e, ex = s.exitance(), s.export()
    assert np.all(np.abs(ex["normal"][:, 1]) == 1.0)   # every normal is +y or -y
    lo = ex["level_off"]
    anc = _subtree_index(ex, D)
    cells = np.floor(pos.astype(np.float64) * (1 << D)).astype(np.int64)
    leaf_keys = ex["key"][lo[D]:lo[D + 1]]
    rec_leaf = lo[D] + np.searchsorted(leaf_keys, np.array([oracle.morton(*c) for c in cells], np.uint64))
    assert np.array_equal(ex["key"][rec_leaf], np.array([oracle.morton(*c) for c in cells], np.uint64))
    up = wout[:, 1] > 0
    qL = _q(L)
    leaf_pos = rec_leaf - lo[D]
    for l in range(D + 1):
        a = anc[l, D][leaf_pos]
        cnt_up = np.bincount(a[up], minlength=s.n_nodes)
        cnt_dn = np.bincount(a[~up], minlength=s.n_nodes)
        sum_up = np.zeros(s.n_nodes, np.uint64)
        np.add.at(sum_up, a[up], qL[up])
        nodes = np.arange(lo[l], lo[l + 1])
        side_up = np.where(ex["normal"][nodes, 1] > 0, 0, 1)
        np.testing.assert_array_equal(e["tot_cnt"][nodes, side_up], cnt_up[nodes], err_msg=f"level {l}")
        np.testing.assert_array_equal(e["tot_cnt"][nodes, 1 - side_up], cnt_dn[nodes], err_msg=f"level {l}")
        np.testing.assert_array_equal(e["tot_sum"][nodes, side_up], sum_up[nodes], err_msg=f"level {l}")
