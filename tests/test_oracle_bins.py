"""Pins of the oracle's Partition-S (Alg. 2), the run-length stand-in binning
and SelectOrigin against brute force and the paper's stated properties."""
import numpy as np
import pytest

import oracle
from paper_2405_06997_gb300 import inputs


def _decode(key, D):
    x = y = z = 0
    for i in range(D):
        x |= ((key >> (3 * i)) & 1) << i
        y |= ((key >> (3 * i + 1)) & 1) << i
        z |= ((key >> (3 * i + 2)) & 1) << i
    return x, y, z


def _interior_rays(w, n):
    """Rays on the walls whose in-plane coordinates are clear of voxel edges,
    so that float64 floor and the kernels' float32 floor pick the same leaf."""
    D = w.depth
    g = w.ray_pos.astype(np.float64) * (1 << D)
    frac = np.abs(g - np.rint(g))
    on_plane = frac < 1e-9
    ok = (np.where(on_plane, 1.0, frac) > 1e-4).all(axis=1)
    idx = np.flatnonzero(ok)[:n]
    return w.ray_pos[idx], w.ray_nrm[idx]


@pytest.mark.parametrize("l_min,c_ray", [(2, 0xFFFFFFFF), (1, 200), (2, 30), (3, 8), (0, 50)])
def test_partition_s_brute_force(l_min, c_ray):
    """Rays on the walls and rays in free space (whose deepest node is an inner
    node, at level 1 in the middle of the box): brute force by coordinates."""
    w = inputs.tiny_box(7, n_rays=6000)
    D = w.depth
    pos, nrm = _interior_rays(w, 4000)
    rng = np.random.default_rng(l_min + 7)
    free = rng.uniform(0.27, 0.73, (300, 3)).astype(np.float32)
    keep = (np.abs(free * (1 << D) - np.rint(free * (1 << D))) > 1e-4).all(axis=1)
    pos = np.concatenate([pos, free[keep]])
    nrm = np.concatenate([nrm, np.tile(np.array([[0, 1, 0]], np.float32), (int(keep.sum()), 1))])
    s = oracle.SVO(w.scene, D)
    r = s.bin_rays(pos, nrm, mode=0, l_min=l_min, c_ray=c_ray, seed=3, frame=1)
    # the tree's cells, level by level, from the node keys
    ex = s.export()
    lo = ex["level_off"]
    exists = {(l, _decode(int(k), l)) for l in range(D + 1) for k in ex["key"][lo[l]:lo[l + 1]]}
    cells = np.minimum(np.floor(pos.astype(np.float64) * (1 << D)), (1 << D) - 1).astype(int)
    anc = lambda c, l: (l, tuple(int(v) >> (D - l) for v in c))
    deepest = [max(l for l in range(D + 1) if anc(c, l) in exists) for c in cells]
    assert min(deepest) == 1 and max(deepest) == D
    # ray counts of every existing ancestor cell down to l_min
    counts = {}
    for c, L in zip(cells, deepest):
        for l in range(l_min, L + 1):
            counts[anc(c, l)] = counts.get(anc(c, l), 0) + 1
    groups = {}
    for i, (c, L) in enumerate(zip(cells, deepest)):
        if L < l_min:   # above l_min: the ray keeps its own node
            groups.setdefault(anc(c, L), []).append(i)
            continue
        for l in range(L, l_min - 1, -1):
            k = anc(c, l)
            if counts[k] >= c_ray or l == l_min:
                groups.setdefault(k, []).append(i)
                break
    # bins are numbered by ascending node id: level first, then Morton order
    order = sorted(groups, key=lambda k: (k[0], oracle.morton(*k[1])))
    assert r["n_bins"] == len(order)
    for b, k in enumerate(order):
        members = np.flatnonzero(r["bin_of_ray"] == b)
        assert members.tolist() == groups[k]
        lo, hi = r["bin_offset"][b], r["bin_offset"][b + 1]
        assert r["ray_order"][lo:hi].tolist() == groups[k]   # stable partition
        assert r["origin_ray"][b] in groups[k]
        if k[0] > l_min:
            # marked for its subtree total; descendants that are marked keep
            # their own rays, so the bin itself may hold fewer
            assert counts[k] >= c_ray


def test_bin_count_non_increasing_in_c_ray():
    """Fig. 4: the bins grow (fewer of them) as the ray threshold rises."""
    w = inputs.tiny_box(2, n_rays=20000)
    s = oracle.SVO(w.scene, w.depth)
    counts = [s.bin_rays(w.ray_pos, w.ray_nrm, l_min=2, c_ray=c)["n_bins"]
              for c in (16, 32, 64, 128, 256, 512, 1024)]
    assert all(a >= b for a, b in zip(counts, counts[1:]))
    assert counts[0] > counts[-1]


def test_partition_sizes_sum_and_marking():
    w = inputs.tiny_box(5, n_rays=20000)
    s = oracle.SVO(w.scene, w.depth)
    r = s.bin_rays(w.ray_pos, w.ray_nrm, l_min=2, c_ray=128)
    off = r["bin_offset"]
    assert off[0] == 0 and off[-1] == len(w.ray_pos)
    assert np.all(np.diff(off) > 0)
    assert sorted(r["ray_order"].tolist()) == list(range(len(w.ray_pos)))


def test_origin_selection_uses_counter_rng():
    """SelectOrigin draws from stream (frame, bin): another frame gives other
    origins for most bins, the same frame the same ones."""
    w = inputs.tiny_box(1, n_rays=20000)
    s = oracle.SVO(w.scene, w.depth)
    a = s.bin_rays(w.ray_pos, w.ray_nrm, l_min=3, c_ray=64, seed=9, frame=0)["origin_ray"]
    b = s.bin_rays(w.ray_pos, w.ray_nrm, l_min=3, c_ray=64, seed=9, frame=0)["origin_ray"]
    c = s.bin_rays(w.ray_pos, w.ray_nrm, l_min=3, c_ray=64, seed=9, frame=1)["origin_ray"]
    assert np.array_equal(a, b)
    assert np.mean(a != c) > 0.8


def test_runs_mode_sizes_and_spatial_order():
    w = inputs.tiny_box(3, n_rays=5000)
    D = w.depth
    s = oracle.SVO(w.scene, D)
    sizes = inputs.zipf_bin_sizes(len(w.ray_pos), 64, 1.2, 11)
    assert int(sizes.sum()) == len(w.ray_pos)
    r = s.bin_rays(w.ray_pos, w.ray_nrm, mode=1, sizes=sizes, seed=2)
    assert r["n_bins"] == 64
    assert np.array_equal(np.diff(r["bin_offset"]), sizes.astype(np.int64))
    # keys along ray_order never decrease; equal keys keep ray order
    cells = np.minimum(np.floor(w.ray_pos.astype(np.float64) * (1 << D)), (1 << D) - 1).astype(int)
    interior = (np.abs(w.ray_pos * (1 << D) - np.rint(w.ray_pos * (1 << D))) > 1e-4) | \
               (np.abs(w.ray_pos * (1 << D) - np.rint(w.ray_pos * (1 << D))) < 1e-9)
    oct_ = (w.ray_nrm[:, 0] < 0) * 1 + (w.ray_nrm[:, 1] < 0) * 2 + (w.ray_nrm[:, 2] < 0) * 4
    key = np.array([oracle.morton(*(c >> (D - 6))) * 8 + o for c, o in zip(cells, oct_)],
                   dtype=np.int64)
    ok = interior.all(axis=1)
    seq = r["ray_order"]
    ks = key[seq][ok[seq]]
    assert np.all(np.diff(ks) >= 0)
    for b in range(64):
        lo, hi = r["bin_offset"][b], r["bin_offset"][b + 1]
        assert np.all(r["bin_of_ray"][seq[lo:hi]] == b)


def test_runs_mode_rejects_bad_sizes():
    w = inputs.tiny_box(3, n_rays=100)
    s = oracle.SVO(w.scene, w.depth)
    with pytest.raises(ValueError):
        s.bin_rays(w.ray_pos, w.ray_nrm, mode=1, sizes=np.array([50, 49], np.uint32))
    with pytest.raises(ValueError):
        s.bin_rays(w.ray_pos, w.ray_nrm, mode=1, sizes=np.array([100, 0], np.uint32))


def test_splitmix64_published_outputs():
    import os
    path = os.path.join(os.path.dirname(__file__), "golden", "splitmix64_state0.txt")
    want = [int(l, 16) for l in open(path) if l.strip() and not l.startswith("#")]
    assert [oracle.rng_u64(0, 0, k) for k in range(3)] == want
