"""Triangle meshes on the GPU (the paper voxelises triangle scenes, Sec. 3.2).

* the SVO of triangle scenes (the mesh room, a random triangle soup, a scene
  mixing quads, spheres and triangles) equals the oracle's: node keys, masks,
  parents, leaf counts, k-means normals and fragment lists, bit for bit;
* the guiding path on the mesh room (records, bins, field, PDF/CDF, sampling)
  equals the oracle;
* closest hits on triangles: brute force and the SVO walk agree, and both
  agree with a plane/barycentric solve in float64;
* frames on the mesh room (triangle lights for NEE) are unbiased.
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

RTOL = 1e-5


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def u32(t):
    return t.cpu().numpy().view(np.uint32)


def assert_svo_equal(scene, D):
    g = W.svo_from_scene(scene, D)
    o = oracle.SVO(scene, D)
    ge, oe = g.export(), o.export()
    np.testing.assert_array_equal(ge["level_off"], oe["level_off"])
    for k in ("key", "first_child", "child_mask", "parent", "leaf_count"):
        np.testing.assert_array_equal(ge[k], oe[k], err_msg=k)
    np.testing.assert_array_equal(ge["normal"], oe["normal"])
    off, prim = o.frags()
    np.testing.assert_array_equal(ge["frag_off"], off)
    np.testing.assert_array_equal(ge["frag_prim"], prim)
    assert g.status() == 0
    return g, o


def soup(seed, n):
    rng = np.random.default_rng(seed)
    c = rng.uniform(0.05, 0.95, (n, 1, 3))
    s = 10 ** rng.uniform(-2.5, -0.7, (n, 1, 1))
    tris = np.clip(c + s * rng.normal(size=(n, 3, 3)), 0.0, 1.0).reshape(n, 9).astype(np.float32)
    return inputs.Scene(quads=np.zeros((0, 8), np.float32), spheres=np.zeros((0, 4), np.float32),
                        albedo=np.full(n, 0.5, np.float32), emission=np.zeros(n, np.float32),
                        lo=np.zeros(3, np.float32), size=1.0, tris=tris)


@pytest.mark.parametrize("D", [3, 5, 7])
def test_svo_build_mesh_room(D):
    assert_svo_equal(inputs.mesh_room(1, D), D)


def test_svo_build_triangle_soup_d9():
    assert_svo_equal(soup(4, 3000), 9)


def test_svo_build_mixed_primitives():
    """Quads, spheres and triangles in one scene: primitive ids count them in
    that order, and the leaves mix their fragments."""
    box = inputs.closed_box(3, 6)
    sph = inputs.cornell_spheres(5, n_spheres=12)
    tri = inputs.mesh_room(2, 6, subdiv=1)
    sel = slice(14, None)  # the meshes, not the room's walls or light
    sc = inputs.Scene(quads=box.quads, spheres=sph.spheres, tris=tri.tris[sel],
                      albedo=np.concatenate([box.albedo, sph.albedo[5:], tri.albedo[sel]]),
                      emission=np.concatenate([box.emission, sph.emission[5:], tri.emission[sel]]),
                      lo=np.zeros(3, np.float32), size=1.0)
    g, o = assert_svo_equal(sc, 6)
    prim = g.export()["frag_prim"]
    nq, ns = sc.n_quads, sc.n_spheres
    assert (prim < nq).any() and ((prim >= nq) & (prim < nq + ns)).any() and (prim >= nq + ns).any()


def test_guiding_on_the_mesh_room_matches_oracle():
    w = inputs.mesh_box(2, n_rays=4099)
    g = W.svo_from_scene(w.scene, w.depth)
    o = oracle.SVO(w.scene, w.depth)
    W.svo_accumulate(g, dev(w.rec_pos), dev(w.rec_wout), dev(w.rec_L))
    o.accumulate(w.rec_pos, w.rec_wout, w.rec_L)
    ge, oe = g.exitance(), o.exitance()
    np.testing.assert_array_equal(ge["acc_sum"], oe["acc_sum"])
    np.testing.assert_array_equal(ge["value"], oe["value"])
    pos = dev(w.ray_pos)
    r = W.bin_rays(g, pos, l_min=2, seed=3, frame=1)
    ro = o.bin_rays(w.ray_pos, w.ray_nrm, l_min=2, seed=3, frame=1)
    nb = ro["n_bins"]
    assert int(r["n_bins"].item()) == nb
    np.testing.assert_array_equal(u32(r["bin_of_ray"]), ro["bin_of_ray"])
    N = 32
    pdf, cr, cm = W.guide_build_pdf(g, pos, r["origin_ray"], r["n_bins"], r["bin_cap"], N=N, jitter=True, blur=True,
                                    seed=3, frame=1)
    og = o.guide_build(w.ray_pos[ro["origin_ray"]], np.arange(nb), N, jitter=True, blur=True, seed=3, frame=1)
    np.testing.assert_allclose(pdf[:nb].cpu().numpy(), og["pdf"], rtol=RTOL, atol=0)
    np.testing.assert_allclose(cr[:nb].cpu().numpy(), og["cdf_row"], rtol=RTOL, atol=0)
    u = inputs.uniforms24(9, (len(w.ray_pos), 2))
    d, p, c = W.guide_sample(pdf, cr, cm, N, r["bin_of_ray"], dev(u))
    od, op, oc = oracle.guide_sample(og["pdf"], og["cdf_row"], og["cdf_marg"], N, ro["bin_of_ray"], u)
    np.testing.assert_array_equal(u32(c), oc)
    np.testing.assert_allclose(p.cpu().numpy(), op, rtol=RTOL, atol=0)


def _solve_hits(tris, o, d):
    """Closest hit by solving o + t d = v0 + b1 e1 + b2 e2 in float64 for every
    triangle (numpy), inside when b1, b2 >= 0 and b1 + b2 <= 1."""
    T = tris.astype(np.float64).reshape(-1, 3, 3)
    o, d = o.astype(np.float64), d.astype(np.float64)
    best = np.full(len(o), np.inf)
    prim = np.full(len(o), -1)
    for k, t in enumerate(T):
        e1, e2 = t[1] - t[0], t[2] - t[0]
        A = np.stack([np.broadcast_to(-d.T, (3, len(o))), np.broadcast_to(e1[:, None], (3, len(o))),
                      np.broadcast_to(e2[:, None], (3, len(o)))], axis=1).transpose(2, 0, 1)
        det = np.linalg.det(A)
        ok = np.abs(det) > 1e-14
        x = np.full((len(o), 3), -1.0)
        x[ok] = np.linalg.solve(A[ok], (o - t[0])[ok][:, :, None])[:, :, 0]
        tt, b1, b2 = x[:, 0], x[:, 1], x[:, 2]
        hit = ok & (tt > 1e-4) & (b1 >= 0) & (b2 >= 0) & (b1 + b2 <= 1) & (tt < best)
        best[hit] = tt[hit]
        prim[hit] = k
    return best, prim


def test_triangle_casting():
    sc = inputs.mesh_room(3, 7, subdiv=1)
    g = W.svo_from_scene(sc, 7)
    rng = np.random.default_rng(6)
    n = 4000
    o = rng.uniform(0.05, 0.95, (n, 3)).astype(np.float32)
    d = rng.normal(size=(n, 3))
    d = (d / np.linalg.norm(d, axis=1, keepdims=True)).astype(np.float32)
    q, sp, tr = dev(sc.quads), dev(sc.spheres), dev(sc.tris)
    t0, p0, n0 = W.cast_rays(q, sp, dev(o), dev(d), tmin=1e-4, tris=tr)
    t1, p1, _ = W.cast_rays_svo(g, q, sp, dev(o), dev(d), tmin=1e-4, tris=tr)
    t0, p0, t1, p1 = t0.cpu().numpy(), p0.cpu().numpy(), t1.cpu().numpy(), p1.cpu().numpy()
    ts, ps = _solve_hits(sc.tris, o, d)
    # a closed room: every ray hits something
    assert (p0 >= 0).mean() > 0.999 and (ps >= 0).mean() > 0.999
    same = p0 == p1
    np.testing.assert_array_equal(t0[same], t1[same])
    assert same.mean() > 0.998
    agree = (p0 == ps)
    assert agree.mean() > 0.995
    np.testing.assert_allclose(t0[agree], ts[agree], rtol=1e-4, atol=1e-6)
    # the returned normal is the unit winding normal, turned against the ray
    T = sc.tris.astype(np.float64).reshape(-1, 3, 3)[p0[agree]]
    wn = np.cross(T[:, 1] - T[:, 0], T[:, 2] - T[:, 0])
    wn /= np.linalg.norm(wn, axis=1, keepdims=True)
    wn *= -np.sign(np.einsum("ij,ij->i", wn, d[agree]))[:, None]
    np.testing.assert_allclose(n0.cpu().numpy()[agree], wn, atol=2e-5)


def test_mesh_room_frames_are_unbiased_with_triangle_lights():
    w = inputs.mesh_box(4, depth=7)
    sc = w.scene
    g = W.svo_from_scene(sc, 7)
    W.svo_accumulate(g, dev(w.rec_pos), dev(w.rec_wout), dev(w.rec_L))
    frames, res = 40, {}
    for alpha, nee in ((0.0, False), (0.5, True)):
        f = W.Frame(g, sc, eye=(0.5, 0.5, 0.05), width=96, height=54, vfov=70.0, max_depth=3, rr_depth=2,
                    alpha=alpha, l_min=2, c_ray=512, N=16, seed=51 + int(nee), nee=nee)
        f.run(frames)
        m, v = f.image()
        st = f.stats()
        assert st["status"] == 0 and st["paths"][0] > 0
        res[nee] = (float(m.double().mean()), float(np.sqrt(v.double().sum().item() / frames) / f.pixels),
                    float(v.double().mean()))
    (mu0, s0, v0), (mu1, s1, v1) = res[False], res[True]
    assert abs(mu1 - mu0) < 5 * np.hypot(s0, s1), res
    assert v1 < v0
