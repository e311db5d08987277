"""Pins of the oracle's triangle voxelisation (the paper voxelises triangle
meshes, Sec. 3.2): the separating-axis test against an exact rational
clipping of the triangle by the closed voxel box, special cases with known
voxel sets, the quad box rebuilt from triangles, and the leaf normals of
planar meshes."""
from fractions import Fraction

import numpy as np
import pytest

import oracle
from paper_2405_06997_gb300 import inputs


def _tri_scene(tris):
    tris = np.asarray(tris, np.float32).reshape(-1, 9)
    n = len(tris)
    return inputs.Scene(quads=np.zeros((0, 8), np.float32), spheres=np.zeros((0, 4), np.float32),
                        albedo=np.full(n, 0.5, np.float32), emission=np.zeros(n, np.float32),
                        lo=np.zeros(3, np.float32), size=1.0, tris=tris)


def _leaves(scene, D):
    s = oracle.SVO(scene, D)
    ex = s.export()
    keys = ex["key"][s.level_off[D]:s.level_off[D + 1]]
    return set(int(k) for k in keys), s, ex


def _clip(poly, a, bound, keep_ge):
    out = []
    for i in range(len(poly)):
        P, Q = poly[i], poly[(i + 1) % len(poly)]
        inP = P[a] >= bound if keep_ge else P[a] <= bound
        inQ = Q[a] >= bound if keep_ge else Q[a] <= bound
        if inP:
            out.append(P)
        if inP != inQ:
            t = (bound - P[a]) / (Q[a] - P[a])
            out.append(tuple(P[k] + t * (Q[k] - P[k]) for k in range(3)))
    return out


def _exact_overlap(tri, lo, hi):
    """Triangle and closed box intersect iff clipping the triangle by the six
    closed half-spaces of the box leaves a point (exact rationals)."""
    poly = [tuple(Fraction(float(tri[3 * i + a])) for a in range(3)) for i in range(3)]
    for a in range(3):
        poly = _clip(poly, a, lo[a], True)
        if not poly:
            return False
        poly = _clip(poly, a, hi[a], False)
        if not poly:
            return False
    return True


def _exact_set(tri, D):
    res = 1 << D
    h = Fraction(1, res)
    v = np.asarray(tri, np.float64).reshape(3, 3)
    rng_ = [range(max(0, int(np.floor(v[:, a].min() * res)) - 2), min(res, int(np.floor(v[:, a].max() * res)) + 3))
            for a in range(3)]
    out = set()
    for x in rng_[0]:
        for y in rng_[1]:
            for z in rng_[2]:
                lo = (x * h, y * h, z * h)
                hi = ((x + 1) * h, (y + 1) * h, (z + 1) * h)
                if _exact_overlap(tri, lo, hi):
                    out.add(oracle.morton(x, y, z))
    return out


@pytest.mark.parametrize("seed", range(6))
def test_sat_equals_exact_clipping_on_random_triangles(seed):
    rng = np.random.default_rng(seed)
    D = 4
    for _ in range(4):
        c = rng.uniform(0.2, 0.8, 3)
        tri = (c + rng.uniform(-0.2, 0.2, (3, 3))).astype(np.float32).ravel()
        got, _, _ = _leaves(_tri_scene(tri), D)
        assert got == _exact_set(tri, D)


def test_sat_special_cases():
    D = 4
    h = 1.0 / 16
    # a triangle in the plane x = 4h (a voxel boundary) touches both layers 3 and 4
    tri = [4 * h, 0.3, 0.3, 4 * h, 0.6, 0.31, 4 * h, 0.32, 0.7]
    got, _, _ = _leaves(_tri_scene(tri), D)
    assert got == _exact_set(tri, D)
    xs = {inputs_decode(k, D)[0] for k in got}
    assert xs == {3, 4}
    # a tiny triangle strictly inside one voxel occupies exactly that voxel
    c = np.array([5.5, 9.5, 2.5]) * h
    tri = np.concatenate([c + [0.1 * h, 0, 0], c + [0, 0.1 * h, 0], c + [0, 0, 0.1 * h]])
    got, _, _ = _leaves(_tri_scene(tri), D)
    assert got == {oracle.morton(5, 9, 2)}
    # vertices on voxel corners and a diagonal edge through corners (dyadic: exact in binary64)
    tri = [2 * h, 2 * h, 0.5, 10 * h, 2 * h, 0.5, 2 * h, 10 * h, 0.5]
    got, _, _ = _leaves(_tri_scene(tri), D)
    assert got == _exact_set(tri, D)
    # a degenerate (zero-area) triangle is a segment: the voxels it passes
    tri = [0.1, 0.1, 0.1, 0.9, 0.5, 0.3, 0.5, 0.3, 0.2]
    got, _, _ = _leaves(_tri_scene(tri), D)
    assert got == _exact_set(tri, D)


def inputs_decode(key, D):
    x = y = z = 0
    for i in range(D):
        x |= ((key >> (3 * i)) & 1) << i
        y |= ((key >> (3 * i + 1)) & 1) << i
        z |= ((key >> (3 * i + 2)) & 1) << i
    return x, y, z


@pytest.mark.parametrize("D", [4, 6])
def test_triangle_box_equals_quad_box(D):
    """The unit box's six walls as 12 triangles occupy exactly the voxels of the
    six quads, with the same (exact, inward) normals at the leaves inside a
    wall (edge and corner leaves weigh the walls by their fragment counts,
    which differ: a wall is two triangles)."""
    q = inputs.closed_box(1, D)
    q.quads = q.quads[:6]
    q.albedo, q.emission = q.albedo[:6], q.emission[:6]
    lq, sq, eq = _leaves(q, D)
    lt, _, et = _leaves(_tri_scene(inputs._box_tris()), D)
    assert lq == lt
    np.testing.assert_array_equal(eq["key"], et["key"])
    lo, res = sq.level_off, 1 << D
    walls = 0
    for node in range(lo[D], lo[D + 1]):
        c = inputs_decode(int(eq["key"][node]), D)
        if sum(0 < x < res - 1 for x in c) == 2:
            np.testing.assert_array_equal(et["normal"][node], eq["normal"][node])
            walls += 1
    assert walls == 6 * (res - 2) ** 2


def test_planar_mesh_normals():
    """Every leaf of a planar fan of triangles has the plane's unit normal."""
    n = np.array([1.0, 2.0, 3.0]) / np.sqrt(14.0)
    u = np.cross(n, [0, 0, 1.0])
    u /= np.linalg.norm(u)
    v = np.cross(n, u)
    c = np.array([0.5, 0.5, 0.5])
    ang = np.linspace(0, 2 * np.pi, 9)
    ring = [c + 0.35 * (np.cos(a) * u + np.sin(a) * v) for a in ang]
    tris = [np.concatenate([c, ring[i], ring[i + 1]]) for i in range(8)]
    leaves, s, ex = _leaves(_tri_scene(tris), 5)
    lo = s.level_off
    nl = ex["normal"][lo[5]:lo[6]].astype(np.float64)
    wind = np.cross(tris[0][3:6] - tris[0][0:3], tris[0][6:9] - tris[0][0:3])
    sign = np.sign(wind @ n)
    assert len(leaves) > 100
    np.testing.assert_allclose(nl, np.tile(sign * n, (len(nl), 1)), atol=2e-6)


def test_mesh_room_voxels_cover_its_surface():
    """Area-uniform points on every triangle of the mesh room lie in occupied
    leaves (a point of the surface is in the closed box of its leaf)."""
    sc = inputs.mesh_room(2, 6, subdiv=2)
    D = 6
    leaves, s, _ = _leaves(sc, D)
    rng = np.random.default_rng(3)
    pos, _, _ = inputs.tri_surface_points(sc, rng, 20000)
    g = np.clip(np.floor(pos.astype(np.float64) * (1 << D)), 0, (1 << D) - 1).astype(int)
    for x, y, z in g:
        assert oracle.morton(int(x), int(y), int(z)) in leaves


def test_mesh_room_windings_and_light():
    """The generator's windings: the room's walls face inward, the meshes'
    triangles outward (away from their centres / the torus tube), the light's
    two triangles face down and cover [0.35, 0.65]^2."""
    sc = inputs.mesh_room(1, 7, subdiv=2)
    t = sc.tris.astype(np.float64).reshape(-1, 3, 3)
    n = np.cross(t[:, 1] - t[:, 0], t[:, 2] - t[:, 0])
    c = t.mean(axis=1)
    assert np.all(np.einsum("ij,ij->i", n[:12], 0.5 - c[:12]) > 0)          # walls inward
    assert np.all(n[12:14, 1] < 0) and np.all(sc.emission[12:14] == 10.0)  # light faces down
    np.testing.assert_allclose(inputs.tri_area(sc.tris[12:14]).sum(), 0.09, rtol=1e-6)
    ico = slice(14, 14 + 320)
    assert np.all(np.einsum("ij,ij->i", n[ico], c[ico] - np.array([0.3, 0.25, 0.6])) > 0)
    assert np.all(sc.albedo[:12] >= 0.3) and np.all(sc.albedo[12:14] == 0.0)
