"""The seeded input recipes have the shapes, sizes and distributions the
documentation states (the workloads stand in for the paper's scenes)."""
import numpy as np
import pytest
from scipy import stats

from paper_2405_06997_gb300 import inputs


def on_quad(q, p, tol=1e-6, plane_tol=0.0):
    """Points in the quad's plane (within plane_tol; sampled points sit on it
    exactly) and inside its extent (within tol)."""
    a = int(q[0])
    b, c = (a + 1) % 3, (a + 2) % 3
    return (np.abs(p[:, a] - q[1]) <= plane_tol) & (p[:, b] >= q[2] - tol) & (p[:, b] <= q[3] + tol) & \
           (p[:, c] >= q[4] - tol) & (p[:, c] <= q[5] + tol)


def test_uniforms_lie_on_the_24_bit_lattice():
    u = inputs.uniforms24(3, (100000, 2))
    assert u.dtype == np.float32 and u.min() >= 0.0 and u.max() < 1.0
    k = u.astype(np.float64) * 2.0 ** 24
    assert np.array_equal(k, np.floor(k))
    assert stats.kstest(u[:, 0], "uniform").pvalue > 1e-3


def test_zipf_sizes_of_the_frame_workload():
    sizes = inputs.zipf_bin_sizes(1_602_720, 2048, 1.2, 1004)
    assert int(sizes.sum()) == 1_602_720 and sizes.min() >= 1
    s = np.sort(sizes)[::-1].astype(np.float64)
    k = np.arange(1, 2049, dtype=np.float64)
    w = k ** -1.2
    # floor of the Zipf shares, the remainder one each to the largest ranks
    assert np.all(np.abs(s - 1_602_720 * w / w.sum()) <= 1.0)
    # the ranks are permuted over the runs by the seed
    assert not np.array_equal(sizes, np.sort(sizes)[::-1])
    assert np.array_equal(sizes, inputs.zipf_bin_sizes(1_602_720, 2048, 1.2, 1004))


def test_tiny_box_recipe():
    D = 6
    w = inputs.tiny_box(2)
    sc = w.scene
    assert w.depth == D and w.grid_n == 16 and w.l_min == 2 and w.c_ray == 0xFFFFFFFF
    assert sc.n_quads == 7 and sc.n_spheres == 0
    walls, light = sc.quads[:6], sc.quads[6]
    assert np.all((sc.albedo[:6] >= 0.3) & (sc.albedo[:6] <= 0.8)) and sc.albedo[6] == 0
    assert sc.emission[6] == 10.0 and np.all(sc.emission[:6] == 0)
    assert light[0] == 1 and light[1] == np.float32(1 - 0.5 / (1 << D)) and light[6] == -1
    assert np.allclose(light[2:6], [0.35, 0.65, 0.35, 0.65])
    # records: 100k on the walls and the light, leaving into the box, L by the recipe
    assert len(w.rec_L) == 100_000
    owner = np.full(len(w.rec_L), -1)
    for i, q in enumerate(sc.quads):
        owner[on_quad(q, w.rec_pos) & (owner < 0)] = i
    assert np.all(owner >= 0)
    inward = np.zeros((len(owner), 3))
    inward[np.arange(len(owner)), sc.quads[owner, 0].astype(int)] = sc.quads[owner, 6]
    assert np.all(np.einsum("ij,ij->i", inward, w.rec_wout) > 0)
    lit = owner == 6
    assert np.all(w.rec_L[lit] == 10.0)
    assert np.all(w.rec_L[~lit] <= sc.albedo[owner[~lit]] * 10.0 + 1e-5) and np.all(w.rec_L[~lit] >= 0)
    # area-uniform: each wall gets about a sixth of the wall records
    frac = np.bincount(owner[~lit], minlength=6)[:6] / (~lit).sum()
    assert np.all(np.abs(frac - frac.mean()) < 0.01)
    # rays: 4096 on the walls (never the light), inward normals
    assert len(w.ray_pos) == 4096
    ro = np.full(len(w.ray_pos), -1)
    for i, q in enumerate(walls):
        ro[on_quad(q, w.ray_pos) & (ro < 0)] = i
    assert np.all(ro >= 0)
    expect = np.zeros((len(ro), 3), np.float32)
    expect[np.arange(len(ro)), walls[ro, 0].astype(int)] = walls[ro, 6]
    assert np.array_equal(w.ray_nrm, expect)


def test_frame_workload_recipe():
    w = inputs.frame_spheres(1)
    sc = w.scene
    assert w.depth == 9 and w.grid_n == 32 and w.blur and w.jitter and w.bin_mode == 1
    assert len(w.ray_pos) == 1_602_720 and len(w.rec_L) == 1_646_633
    assert len(w.bin_sizes) == 2048 and int(w.bin_sizes.max()) == 355_888 and int(w.bin_sizes.min()) == 37
    assert sc.n_quads == 5 and sc.n_spheres == 200           # the front (z = 0) is open
    assert not np.any((sc.quads[:, 0] == 2) & (sc.quads[:, 1] == 0.0))
    c, r = sc.spheres[:, :3], sc.spheres[:, 3]
    assert c.min() >= 0.1 and c.max() <= 0.9 and r.min() >= 0.02 and r.max() <= 0.1
    e = sc.emission[5:]
    assert 10 <= np.count_nonzero(e) <= 30 and e[e > 0].min() >= 1 and e[e > 0].max() <= 20
    # every primary hit lies on its primitive, with a unit normal facing the camera side
    prim = w.extra["ray_prim"]
    sp = prim >= 5
    d = np.linalg.norm(w.ray_pos[sp] - c[prim[sp] - 5], axis=1)
    assert np.allclose(d, r[prim[sp] - 5], atol=2e-5)
    for i, q in enumerate(sc.quads):
        assert on_quad(q, w.ray_pos[prim == i], tol=2e-5, plane_tol=2e-5).all()
    assert np.allclose(np.linalg.norm(w.ray_nrm, axis=1), 1.0, atol=1e-5)
    view = w.ray_pos.astype(np.float64) - np.array([0.5, 0.5, -1.0])
    assert np.all(np.einsum("ij,ij->i", view, w.ray_nrm) < 0)
    assert np.array_equal(w.u, inputs.uniforms24(1003, (1_602_720, 2)))


def test_city_recipe():
    sc = inputs.city(1)
    assert sc.size == 500.0 and sc.n_quads == 1 + 5 * 5000 + 50
    boxes = sc.quads[1:1 + 5 * 5000].reshape(5000, 5, 8)
    height = boxes[:, 2, 1]                                   # the roof's plane
    assert height.min() >= 0.5 - 1e-4 and height.max() <= 20 + 1e-3
    assert stats.kstest(np.log(height), "uniform", args=(np.log(0.5), np.log(20) - np.log(0.5))).pvalue > 1e-3
    lights = sc.quads[-50:]
    assert np.all(sc.emission[-50:] > 0) and np.all(sc.emission[:-50] == 0)
    assert np.all((lights[:, 0] == 1) & (lights[:, 6] == -1))  # facing down


@pytest.mark.parametrize("subdiv, count", [(3, 3598), (5, 41998)])
def test_mesh_room_triangle_counts(subdiv, count):
    assert inputs.mesh_room(1, 7, subdiv=subdiv).n_tris == count
