"""The fused GuideRays launch and the batched wavefront frame on the GPU.

* guide_build_sample equals guide_build_pdf + guide_sample + guide_eval_pdf
  bit for bit, and the oracle (field, sampler, cosine sampling, mixture
  density) to the float32 bar;
* a frame's Eq. 5 records equal the oracle's back-propagation of the frame's
  own path history, and its UpdateExitance equals svo_accumulate (and the
  oracle) on those records, bit for bit;
* the guiding inside a frame equals standalone bin_rays + guide_build_sample
  on the frame's queue;
* graph replay equals eager launches; guided frames are unbiased (their mean
  image agrees with cosine-only frames within the Monte Carlo error).
"""
import numpy as np
import pytest

import oracle
from oracle import frame as OF
from paper_2405_06997_gb300 import inputs

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA device", allow_module_level=True)

from paper_2405_06997_gb300 import wfpg as W  # noqa: E402

RTOL = 1e-5
EYE = (0.5, 0.5, 0.05)


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def u32(t):
    return t.cpu().numpy().view(np.uint32)


def box_svo(seed=1, D=6, records=True):
    w = inputs.tiny_box(seed)
    g = W.svo_from_scene(w.scene, D)
    o = oracle.SVO(w.scene, D)
    if records:
        W.svo_accumulate(g, dev(w.rec_pos), dev(w.rec_wout), dev(w.rec_L))
        o.accumulate(w.rec_pos, w.rec_wout, w.rec_L)
    return w, g, o


# ------------------------------------------------------------- fused GuideRays
@pytest.mark.parametrize("N,alpha", [(16, 0.5), (32, 0.3), (32, 1.0), (64, 0.0)])
def test_fused_equals_unfused_and_oracle(N, alpha):
    w, g, o = box_svo(4)
    n = w.ray_pos.shape[0]
    pos, nrm = dev(w.ray_pos), dev(w.ray_nrm)
    u3 = inputs.uniforms24(17, (n, 3))
    u = dev(u3)
    r = W.bin_rays(g, pos, nrm, l_min=2, c_ray=64, seed=5, frame=3)
    kw = dict(N=N, jitter=True, blur=True, seed=5, frame=3)
    d, pm = W.guide_build_sample(g, pos, nrm, r, u, alpha=alpha, **kw)
    pdf, cr, cm = W.guide_build_pdf(g, pos, r["origin_ray"], r["n_bins"], r["bin_cap"], **kw)
    dg, pg, _ = W.guide_sample(pdf, cr, cm, N, r["bin_of_ray"], dev(u3[:, :2]))
    guided = u3[:, 2] < alpha
    gm = torch.from_numpy(guided).cuda()
    # the guided branch is guide_sample bit for bit
    assert torch.equal(d[gm], dg[gm])
    # the field part of every density is guide_eval_pdf at the returned direction
    pe = W.guide_eval_pdf(pdf, N, r["bin_of_ray"], d)
    cs = torch.clamp((d * nrm).sum(dim=1), min=0)
    ref = alpha * pe + (1 - alpha) * cs / np.pi
    torch.testing.assert_close(pm, ref, rtol=1e-6, atol=1e-7)
    # oracle: field tables, sampler, cosine directions, mixture density
    ro = o.bin_rays(w.ray_pos, w.ray_nrm, l_min=2, c_ray=64, seed=5, frame=3)
    np.testing.assert_array_equal(u32(r["bin_of_ray"]), ro["bin_of_ray"])
    nb = ro["n_bins"]
    og = o.guide_build(w.ray_pos[ro["origin_ray"][:nb]], np.arange(nb), N, jitter=True, blur=True, seed=5, frame=3)
    od, _, _ = oracle.guide_sample(og["pdf"], og["cdf_row"], og["cdf_marg"], N, ro["bin_of_ray"], u3[:, :2])
    dn = d.cpu().numpy()
    np.testing.assert_allclose(dn[guided], od[guided], rtol=0, atol=1e-6)
    oc = OF.cosine_dirs(w.ray_nrm[~guided].astype(np.float64), u3[~guided, :2].astype(np.float64))
    np.testing.assert_allclose(dn[~guided], oc, rtol=0, atol=4e-6)
    pf = oracle.guide_eval_pdf(og["pdf"], N, ro["bin_of_ray"], dn)
    np.testing.assert_allclose(pm.cpu().numpy(), OF.mixture_pdf(pf, w.ray_nrm, dn, alpha), rtol=RTOL, atol=1e-7)
    assert g.status() == 0


@pytest.mark.parametrize("split", [1, 64, 700])
def test_fused_split_bins_give_identical_samples(split):
    """Bins above `split` rays are sampled by the GPU-wide second launch from
    spilled tables: the directions and densities do not change."""
    w, g, _ = box_svo(8)
    n = w.ray_pos.shape[0]
    pos, nrm = dev(w.ray_pos), dev(w.ray_nrm)
    sizes = inputs.zipf_bin_sizes(n, 24, 1.2, 5)
    r = W.bin_rays(g, pos, nrm, mode=W.BIN_RUNS, sizes=dev(sizes.astype(np.uint32).view(np.int32)), seed=2)
    assert sizes.max() > 700
    u = dev(inputs.uniforms24(23, (n, 3)))
    kw = dict(alpha=0.5, N=32, jitter=True, blur=True, seed=2, frame=1)
    d0, p0 = W.guide_build_sample(g, pos, nrm, r, u, split=0xFFFFFFFF, **kw)
    d1, p1 = W.guide_build_sample(g, pos, nrm, r, u, split=split, **kw)
    assert torch.equal(d0, d1) and torch.equal(p0, p1)
    assert g.status() == 0


def test_fused_rejects_bad_alpha():
    w, g, _ = box_svo(4, records=False)
    pos, nrm = dev(w.ray_pos[:64]), dev(w.ray_nrm[:64])
    r = W.bin_rays(g, pos, nrm)
    with pytest.raises(W.WfpgError):
        W.guide_build_sample(g, pos, nrm, r, torch.zeros((64, 3), device="cuda"), alpha=1.5)


# ---------------------------------------------------------------- the frame
def make_frame(g, scene, **kw):
    args = dict(eye=EYE, width=160, height=90, vfov=70.0, max_depth=4, rr_depth=2, alpha=0.5, l_min=2,
                c_ray=512, N=16, seed=3)
    args.update(kw)
    return W.Frame(g, scene, **args)


def test_frame_records_follow_eq5():
    w, g, o = box_svo(2)
    f = make_frame(g, w.scene)
    f.run(1, use_graph=False)
    st = f.stats()
    P, Dm = f.pixels, 4
    nv = f.export("nv").cpu().numpy()
    vT = f.export("vT").cpu().numpy().reshape(Dm + 1, P).T
    vLe = f.export("vLe").cpu().numpy().reshape(Dm + 1, P).T
    assert st["records"] == int(nv.sum()) > 0
    assert st["paths"][0] > 0 and all(a >= b for a, b in zip(st["paths"], st["paths"][1:]))
    R = st["records"]
    src = u32(f.export("rec_src"))[:R]
    L = f.export("rec_L").cpu().numpy()[:R]
    p, k, oL = OF.eq5_records(vT, vLe, nv)
    osrc = (k - 1) * P + p
    order = np.argsort(src)
    np.testing.assert_array_equal(src[order], np.sort(osrc))
    np.testing.assert_allclose(L[order], oL[np.argsort(osrc)], rtol=RTOL, atol=0)
    # records carry their vertex's position and direction bit for bit
    vpos = f.export("vpos").cpu().numpy()
    vwo = f.export("vwo").cpu().numpy()
    np.testing.assert_array_equal(f.export("rec_pos").cpu().numpy()[:R], vpos[src])
    np.testing.assert_array_equal(f.export("rec_wout").cpu().numpy()[:R], vwo[src])
    # the first vertex's throughput is 1 and emitted radiance is the light's or 0
    hit = nv > 0
    assert np.all(vT[hit, 0] == 1.0)
    assert set(np.unique(vLe[hit, 0])) <= {0.0, 10.0}


def test_frame_update_equals_accumulate_and_oracle():
    w, g, o = box_svo(2)
    w2, g2, o2 = box_svo(2)
    f = make_frame(g, w.scene)
    f.run(1, use_graph=False)
    R = f.stats()["records"]
    rp, rw, rl = (f.export(k)[:R].contiguous() for k in ("rec_pos", "rec_wout", "rec_L"))
    W.svo_accumulate(g2, rp, rw, rl)
    a, b = g.exitance(), g2.exitance()
    for k in ("acc_sum", "acc_cnt", "tot_sum", "tot_cnt", "value"):
        np.testing.assert_array_equal(a[k], b[k], err_msg=k)
    o2.accumulate(rp.cpu().numpy(), rw.cpu().numpy(), rl.cpu().numpy())
    oe = o2.exitance()
    np.testing.assert_array_equal(a["acc_sum"], oe["acc_sum"])
    np.testing.assert_array_equal(a["value"], oe["value"])


def test_frame_guiding_equals_standalone_calls():
    w, g, _ = box_svo(3)
    f = make_frame(g, w.scene, max_depth=1, update=False, N=32, c_ray=128)
    f.run(1, use_graph=False)
    n = f.stats()["paths"][0]
    assert n > 0
    qp, qn, qu = (f.export(k)[:n].contiguous() for k in ("q_pos", "q_nrm", "q_u"))
    # the first frame's random streams use frame index 0 at depth 0
    r = W.bin_rays(g, qp, qn, l_min=2, c_ray=128, seed=3, frame=0, bin_cap=min(f.pixels, g.n_nodes))
    d, pm = W.guide_build_sample(g, qp, qn, r, qu, alpha=0.5, N=32, jitter=True, blur=True, seed=3, frame=0)
    assert torch.equal(f.export("q_dir")[:n], d)
    assert torch.equal(f.export("q_pdf")[:n], pm)
    # the queue holds the camera hits in pixel order
    qpath = u32(f.export("q_path"))[:n]
    assert np.all(np.diff(qpath.astype(np.int64)) > 0)


@pytest.mark.parametrize("N,width,height,c_ray,overflow", [(32, 160, 90, 64, False), (128, 640, 360, 8, True)])
def test_both_field_paths_of_the_frame_equal_the_fused_call(N, width, height, c_ray, overflow):
    """The frame's traced proposal runs the stream field kernel into tables and the mixture
    sampler while a depth's bins fit those tables (4,096 bins at N = 128), the fused GuideRays
    launch when they do not; both give the standalone fused call's directions and densities."""
    w, g, _ = box_svo(3)
    f = make_frame(g, w.scene, max_depth=1, update=False, N=N, c_ray=c_ray, width=width, height=height)
    f.run(1, use_graph=False)
    st = f.stats()
    n, nb = st["paths"][0], st["bins"][0]
    assert n > 0
    assert (nb > 4096) == overflow, nb
    qp, qn, qu = (f.export(k)[:n].contiguous() for k in ("q_pos", "q_nrm", "q_u"))
    r = W.bin_rays(g, qp, qn, l_min=2, c_ray=c_ray, seed=3, frame=0, bin_cap=min(f.pixels, g.n_nodes))
    d, pm = W.guide_build_sample(g, qp, qn, r, qu, alpha=0.5, N=N, jitter=True, blur=True, seed=3, frame=0)
    assert torch.equal(f.export("q_dir")[:n], d)
    assert torch.equal(f.export("q_pdf")[:n], pm)
    assert st["status"] == 0


def test_graph_replay_equals_eager():
    w, g1, _ = box_svo(5)
    _, g2, _ = box_svo(5)
    f1 = make_frame(g1, w.scene)
    f2 = make_frame(g2, w.scene)
    f1.run(3, use_graph=False)
    before = W.kernel_launches()
    f2.run(3, use_graph=True)
    torch.cuda.synchronize()
    s2 = f2.stats()
    assert s2["kernels_per_frame"] > 10
    assert W.kernel_launches() - before == 3 * s2["kernels_per_frame"]
    m1, v1 = f1.image()
    m2, v2 = f2.image()
    assert torch.equal(m1, m2) and torch.equal(v1, v2)
    e1, e2 = g1.exitance(), g2.exitance()
    np.testing.assert_array_equal(e1["acc_sum"], e2["acc_sum"])
    np.testing.assert_array_equal(e1["value"], e2["value"])
    assert f1.stats()["guided_samples"] == s2["guided_samples"]


def test_guided_frames_are_unbiased():
    """Every guided sample carries its exact mixture density, so the mean
    image of guided frames (alpha = 0.5 and alpha = 1) must agree with
    cosine-only frames within the Monte Carlo error."""
    w, g, _ = box_svo(6)
    frames = 48
    res = {}
    for alpha in (0.0, 0.5, 1.0):
        f = make_frame(g, w.scene, width=96, height=54, alpha=alpha, max_depth=3, seed=11 + int(alpha * 10))
        f.run(frames)
        m, v = f.image()
        P = f.pixels
        res[alpha] = (float(m.double().mean()), float(np.sqrt(v.double().sum().item() / frames) / P))
        del f
    mu0, s0 = res[0.0]
    for alpha in (0.5, 1.0):
        mu, s = res[alpha]
        assert abs(mu - mu0) < 5 * np.hypot(s, s0), (alpha, mu, mu0, s, s0)


def test_autotune_picks_a_candidate():
    w, g, _ = box_svo(7)
    f = make_frame(g, w.scene, width=128, height=72)
    choice, ms = f.autotune((16, 32), frames=2)
    assert choice["N"] in (16, 32) and choice["block"] in (64, 128, 256) and ms > 0
    p = f.get_params()
    assert p.guide.N == choice["N"]
    f.run(2)
    assert f.stats()["frames"] == 2


def test_frame_rejects_bad_params():
    w, g, _ = box_svo(7, records=False)
    with pytest.raises(W.WfpgError):
        make_frame(g, w.scene, max_depth=9)
    with pytest.raises(W.WfpgError):
        make_frame(g, w.scene, alpha=-0.1)
    f = make_frame(g, w.scene, max_depth=2)
    with pytest.raises(W.WfpgError):
        f.set_params(max_depth=3)
    with pytest.raises(W.WfpgError):
        f.set_params(N=12)
    with pytest.raises(W.WfpgError):
        f.set_params(nee=2)
    with pytest.raises(W.WfpgError):
        f.set_params(combine=6)
    # probe mode: width must be probe_n^2, probe_n in [1, 1024]
    pts = np.full((3, 3), 0.5, np.float32)
    with pytest.raises(W.WfpgError):
        make_frame(g, w.scene, probes=pts, probe_n=2000)
    f2 = make_frame(g, w.scene, probes=pts, probe_n=4, max_depth=1)
    assert f2.pixels == 3 * 16


# ------------------------------------------------- table-based mixture sampling
def test_sample_mix_from_tables_equals_fused():
    """guide_build_pdf + guide_sample_mix give guide_build_sample's directions
    and densities bit for bit (same field, same per-ray arithmetic)."""
    w, g, _ = box_svo(9)
    n = w.ray_pos.shape[0]
    pos, nrm = dev(w.ray_pos), dev(w.ray_nrm)
    u = dev(inputs.uniforms24(31, (n, 3)))
    r = W.bin_rays(g, pos, nrm, l_min=2, c_ray=64, seed=4, frame=2)
    kw = dict(N=32, jitter=True, blur=True, seed=4, frame=2)
    d0, p0 = W.guide_build_sample(g, pos, nrm, r, u, alpha=0.4, **kw)
    tabs = W.guide_build_pdf(g, pos, r["origin_ray"], r["n_bins"], r["bin_cap"], **kw)
    d1, p1 = W.guide_sample_mix(*tabs, 32, r["bin_of_ray"], nrm, u, alpha=0.4, n_bins=r["n_bins"])
    assert torch.equal(d0, d1) and torch.equal(p0, p1)
    # a bin without a table takes the cosine branch with density cos / pi
    nb0 = torch.zeros(1, dtype=torch.int32, device="cuda")
    d2, p2 = W.guide_sample_mix(*tabs, 32, r["bin_of_ray"], nrm, u, alpha=0.4, n_bins=nb0)
    oc = OF.cosine_dirs(w.ray_nrm.astype(np.float64), inputs.uniforms24(31, (n, 3))[:, :2].astype(np.float64))
    np.testing.assert_allclose(d2.cpu().numpy(), oc, rtol=0, atol=4e-6)
    cs = np.maximum(0, np.einsum("ij,ij->i", w.ray_nrm.astype(np.float64), d2.cpu().numpy().astype(np.float64)))
    np.testing.assert_allclose(p2.cpu().numpy(), cs / np.pi, rtol=1e-5, atol=1e-7)


# ------------------------------------------------------------- SVO ray caster
def _random_rays(scene, n, seed, inside=True):
    rng = np.random.default_rng(seed)
    lo, S = np.asarray(scene.lo, np.float64), float(scene.size)
    o = lo + S * rng.uniform(0.02, 0.98, (n, 3))
    if not inside:
        o[: n // 2] = lo + S * rng.uniform(-0.5, 1.5, (n // 2, 3))
    d = rng.normal(size=(n, 3))
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    return o.astype(np.float32), d.astype(np.float32)


@pytest.mark.parametrize("name", ["spheres", "city"])
def test_svo_caster_matches_brute_force(name):
    if name == "spheres":
        sc, D = inputs.cornell_spheres(3), 8
    else:
        sc, D = inputs.city(2, n_boxes=300, n_lights=10), 9
    g = W.svo_from_scene(sc, D)
    q, sp = dev(sc.quads), dev(sc.spheres)
    o, d = _random_rays(sc, 20000, 5, inside=(name == "spheres"))
    t0, p0, n0 = W.cast_rays(q, sp, dev(o), dev(d), tmin=1e-4)
    t1, p1, n1 = W.cast_rays_svo(g, q, sp, dev(o), dev(d), tmin=1e-4)
    t0, p0, t1, p1 = t0.cpu().numpy(), p0.cpu().numpy(), t1.cpu().numpy(), p1.cpu().numpy()
    same = p0 == p1
    # where both name the same primitive the distance is the same arithmetic
    np.testing.assert_array_equal(t0[same], t1[same])
    # a different primitive only where two surfaces are hit at nearly the same distance
    diff = ~same
    assert diff.sum() <= 0.001 * len(p0), diff.sum()
    hit = diff & (p0 >= 0) & (p1 >= 0)
    np.testing.assert_allclose(t1[hit], t0[hit], rtol=2e-5)
    assert np.all(p0[diff & (p1 < 0)] < 0) or diff.sum() == 0
    assert (p0 >= 0).mean() > 0.05


# ------------------------------------------------------------- frame options
def test_frame_svo_caster_gives_the_same_image():
    w, g1, _ = box_svo(10)
    _, g2, _ = box_svo(10)
    f1 = make_frame(g1, w.scene, caster=1, width=128, height=72)
    f2 = make_frame(g2, w.scene, caster=2, width=128, height=72)
    f1.run(4)
    f2.run(4)
    m1, _ = f1.image()
    m2, _ = f2.image()
    differ = (m1 != m2).float().mean().item()
    assert differ < 0.01, differ
    assert abs(m1.mean().item() - m2.mean().item()) < 0.01 * m1.mean().item()


def test_frame_learned_proposal():
    """Learned mode: the frame's guiding equals guide_learned_build_pdf +
    guide_sample_mix on its own queue, and its frames stay unbiased."""
    w, g, _ = box_svo(11)
    mlp = W.MLP(inputs.mlp_init(5), max_batch=4096)
    f = make_frame(g, w.scene, max_depth=1, update=False, N=32, c_ray=128, proposal=1)
    with pytest.raises(W.WfpgError):
        f.run(1)  # no MLP attached yet
    f.set_mlp(mlp, w.scene.lo, w.scene.size)
    f.run(1, use_graph=False)
    n = f.stats()["paths"][0]
    qp, qn, qu = (f.export(k)[:n].contiguous() for k in ("q_pos", "q_nrm", "q_u"))
    r = W.bin_rays(g, qp, qn, l_min=2, c_ray=128, seed=3, frame=0, bin_cap=min(f.pixels, g.n_nodes))
    cap = min(r["bin_cap"], 4096)
    tabs = W.guide_learned_build_pdf(mlp, qp, qn, r["origin_ray"], r["n_bins"], cap, lo=w.scene.lo,
                                     size=w.scene.size)
    d, pm = W.guide_sample_mix(*tabs, 32, r["bin_of_ray"], qn, qu, alpha=0.5, n_bins=r["n_bins"])
    assert torch.equal(f.export("q_dir")[:n], d)
    assert torch.equal(f.export("q_pdf")[:n], pm)
    # unbiased: learned-guided frames agree with cosine-only frames
    frames, res = 40, {}
    for alpha in (0.0, 0.5):
        fr = make_frame(g, w.scene, width=96, height=54, alpha=alpha, max_depth=3, N=32, proposal=1,
                        seed=21 + int(alpha * 10))
        fr.set_mlp(mlp, w.scene.lo, w.scene.size)
        fr.run(frames)
        m, v = fr.image()
        res[alpha] = (float(m.double().mean()), float(np.sqrt(v.double().sum().item() / frames) / fr.pixels))
    (mu0, s0), (mu1, s1) = res[0.0], res[0.5]
    assert abs(mu1 - mu0) < 5 * np.hypot(s0, s1), res


def test_city_frame_runs_with_the_svo_caster():
    sc = inputs.city(3, n_boxes=400, n_lights=12)
    g = W.svo_from_scene(sc, 9)
    f = W.Frame(g, sc, eye=(250.0, 120.0, -60.0), forward=(0.0, -0.3939193, 0.9191450),
                up=(0.0, 0.9191450, 0.3939193), vfov=60.0, width=192, height=108, max_depth=3, N=32, seed=2)
    f.run(3)
    st = f.stats()
    m, _ = f.image()
    assert st["status"] == 0 and st["paths"][0] > 0.3 * f.pixels
    assert torch.isfinite(m).all() and m.mean().item() > 0


def test_frame_that_sees_nothing():
    """A camera outside the scene looking away: no hits, so every depth's queue
    is empty, Partition-S and GuideRays get zero rays, no records are
    accumulated, and the image is black -- without errors or status bits."""
    w, g, _ = box_svo(12)
    before = g.exitance()
    f = make_frame(g, w.scene, eye=(0.5, 0.5, -2.0), forward=(0.0, 0.0, -1.0), width=64, height=36)
    f.run(2, use_graph=False)
    f.run(2, use_graph=True)
    st = f.stats()
    m, v = f.image()
    assert st["paths"] == [0, 0, 0, 0] and st["records"] == 0 and st["status"] == 0
    assert float(m.abs().max()) == 0.0 and float(v.abs().max()) == 0.0
    np.testing.assert_array_equal(g.exitance()["acc_sum"], before["acc_sum"])


def test_combination_heuristics_weigh_the_frames():
    """Eq. 7: the linear heuristic's image equals the oracle's combination of the
    per-frame estimates S_i (from a constant-weight run with the same seeds), and
    PT first's first frame is the unguided frame."""
    K = 7
    w, g1, _ = box_svo(13)
    _, g2, _ = box_svo(13)
    fa = make_frame(g1, w.scene, width=64, height=36)
    fb = make_frame(g2, w.scene, width=64, height=36, combine=W.COMBINE["linear"])
    means = []
    for k in range(K):
        fa.run(1)
        means.append(fa.image()[0].double().cpu().numpy())
    S = [means[0]] + [(k + 1) * means[k] - k * means[k - 1] for k in range(1, K)]
    ref = OF.combine_images(np.stack(S), "linear")
    fb.run(K)
    np.testing.assert_allclose(fb.image()[0].double().cpu().numpy(), ref, rtol=2e-5, atol=1e-6)
    # PT first: frame 1 equals a frame with alpha = 0
    _, g3, _ = box_svo(13)
    _, g4, _ = box_svo(13)
    fc = make_frame(g3, w.scene, width=64, height=36, combine=W.COMBINE["pt-first"])
    fd = make_frame(g4, w.scene, width=64, height=36, alpha=0.0)
    fc.run(1)
    fd.run(1)
    assert torch.equal(fc.image()[0], fd.image()[0])


def test_decaying_resolution_per_depth():
    """decay: depth k traces N >> k; the frame's second depth equals standalone
    calls at N / 2 on its queue (frame index 0 * 16 + 1)."""
    w, g, _ = box_svo(14)
    f = make_frame(g, w.scene, max_depth=2, update=False, N=32, c_ray=128, decay=True)
    f.run(1, use_graph=False)
    n = f.stats()["paths"][1]
    assert n > 0
    qp, qn, qu = (f.export(k)[:n].contiguous() for k in ("q_pos", "q_nrm", "q_u"))
    r = W.bin_rays(g, qp, qn, l_min=2, c_ray=128, seed=3, frame=1, bin_cap=min(f.pixels, g.n_nodes))
    d, pm = W.guide_build_sample(g, qp, qn, r, qu, alpha=0.5, N=16, jitter=True, blur=True, seed=3, frame=1)
    assert torch.equal(f.export("q_dir")[:n], d)
    assert torch.equal(f.export("q_pdf")[:n], pm)


def test_frame_product_guiding():
    """proposal 2 (product guiding, Sec. 3.6): the frame's guiding equals
    guide_build_pdf + guide_product_sums + guide_product_sample on its queue,
    and product-guided frames stay unbiased."""
    w, g, _ = box_svo(15)
    f = make_frame(g, w.scene, max_depth=1, update=False, N=32, c_ray=128, proposal=2)
    f.run(1, use_graph=False)
    n = f.stats()["paths"][0]
    qp, qn, qu = (f.export(k)[:n].contiguous() for k in ("q_pos", "q_nrm", "q_u"))
    cap = min(f.pixels, g.n_nodes, 65536)
    r = W.bin_rays(g, qp, qn, l_min=2, c_ray=128, seed=3, frame=0, bin_cap=cap)
    tabs = W.guide_build_pdf(g, qp, r["origin_ray"], r["n_bins"], cap, N=32, jitter=True, blur=True, seed=3, frame=0)
    S = W.guide_product_sums(tabs[0], 32, n_bins=r["n_bins"])
    d, pm, _ = W.guide_product_sample(tabs[0], S, 32, r["bin_of_ray"], qn, qu, alpha=0.5, n_bins=r["n_bins"])
    assert torch.equal(f.export("q_dir")[:n], d)
    assert torch.equal(f.export("q_pdf")[:n], pm)
    frames, res = 40, {}
    for alpha in (0.0, 0.5):
        fr = make_frame(g, w.scene, width=96, height=54, alpha=alpha, max_depth=3, N=32, proposal=2,
                        seed=31 + int(alpha * 10))
        fr.run(frames)
        m, v = fr.image()
        res[alpha] = (float(m.double().mean()), float(np.sqrt(v.double().sum().item() / frames) / fr.pixels))
    (mu0, s0), (mu1, s1) = res[0.0], res[0.5]
    assert abs(mu1 - mu0) < 5 * np.hypot(s0, s1), res


# ------------------------------------------------- next-event estimation + MIS
def _frame_mean(g, scene, frames, mlp=None, **kw):
    f = make_frame(g, scene, width=96, height=54, max_depth=3, **kw)
    if mlp is not None:
        f.set_mlp(mlp, scene.lo, scene.size)
    f.run(frames)
    m, v = f.image()
    P = f.pixels
    return float(m.double().mean()), float(np.sqrt(v.double().sum().item() / frames) / P), float(v.double().mean())


def test_nee_records_follow_eq5():
    """With light sampling the suffix sums of Eq. 5 run over T_k (Le_k + Nee_k):
    the records equal the oracle's back-propagation of the exported history."""
    w, g, _ = box_svo(16)
    f = make_frame(g, w.scene, nee=True)
    f.run(1, use_graph=False)
    P, Dm = f.pixels, 4
    nv = f.export("nv").cpu().numpy()
    vT = f.export("vT").cpu().numpy().reshape(Dm + 1, P).T
    vLe = f.export("vLe").cpu().numpy().reshape(Dm + 1, P).T
    vNee = f.export("vNee").cpu().numpy().reshape(Dm + 1, P).T
    vLw = f.export("vLw").cpu().numpy().reshape(Dm + 1, P).T
    R = f.stats()["records"]
    assert R == int(nv.sum()) > 0
    idx = np.arange(Dm + 1)[None, :] < nv[:, None]
    assert np.count_nonzero(vNee[idx]) > 0.05 * R      # the light is seen from many vertices
    assert np.all(vNee[idx] >= 0)
    # a vertex that ends its path (roulette or the last depth) draws no light sample
    last = np.take_along_axis(vNee, np.maximum(nv - 1, 0)[:, None], 1)[:, 0]
    assert np.all(last[(nv == Dm + 1)] == 0)
    src = u32(f.export("rec_src"))[:R]
    L = f.export("rec_L").cpu().numpy()[:R]
    # lights reached by the mixture pass on their MIS-weighted emission, and keep the full one
    hitl = idx & (vLe > 0)
    hitl[:, 0] = False
    assert np.all(vLw[hitl] <= vLe[hitl]) and np.any(vLw[hitl] < vLe[hitl])
    p, k, oL = OF.eq5_records(vT, vLe.astype(np.float64) + vNee, nv, Le_seen=vLw.astype(np.float64) + vNee)
    osrc = (k - 1) * P + p
    order = np.argsort(src)
    np.testing.assert_array_equal(src[order], np.sort(osrc))
    np.testing.assert_allclose(L[order], oL[np.argsort(osrc)], rtol=1e-4, atol=1e-6)


def test_nee_light_sample_and_mixture_density():
    """The light sample's direction points at the light, its density is the
    area-to-solid-angle change of a uniform point on the ceiling quad, and the
    mixture density there is what guide_build_pdf + guide_eval_pdf give."""
    w, g, _ = box_svo(17)
    f = make_frame(g, w.scene, max_depth=1, update=False, N=32, c_ray=128, nee=True)
    f.run(1, use_graph=False)
    n = f.stats()["paths"][0]
    qp, qn = (f.export(k)[:n].contiguous() for k in ("q_pos", "q_nrm"))
    ed = f.export("nee_dir")[:n].contiguous()
    pl = f.export("nee_pl")[:n].cpu().numpy()
    pm = f.export("nee_pm")[:n]
    nl = f.export("nee_l")[:n].cpu().numpy()
    torch.testing.assert_close(torch.linalg.norm(ed, dim=1), torch.ones(n, device="cuda"), rtol=0, atol=2e-6)
    # the mixture density of the light direction from the same field tables
    r = W.bin_rays(g, qp, qn, l_min=2, c_ray=128, seed=3, frame=0, bin_cap=min(f.pixels, g.n_nodes))
    pdf, _, _ = W.guide_build_pdf(g, qp, r["origin_ray"], r["n_bins"], min(f.pixels, g.n_nodes), N=32, jitter=True,
                                  blur=True, seed=3, frame=0)
    pe = W.guide_eval_pdf(pdf, 32, r["bin_of_ray"], ed)
    cs = torch.clamp((ed * qn).sum(dim=1), min=0)
    torch.testing.assert_close(pm, 0.5 * pe + 0.5 * cs / np.pi, rtol=1e-6, atol=1e-7)
    # light density: the ray from the offset origin meets the light's plane at distance t, cos from its axis
    quads, em = w.scene.quads, w.scene.emission
    lights = np.flatnonzero(em[:len(quads)] > 0)
    assert len(lights) == 1
    Ql = np.asarray(quads[lights[0]], np.float64)
    a = int(Ql[0])
    area = (Ql[3] - Ql[2]) * (Ql[5] - Ql[4])
    o = qp.cpu().numpy().astype(np.float64) + 1e-4 * w.scene.size * qn.cpu().numpy()
    e = ed.cpu().numpy().astype(np.float64)
    t = (Ql[1] - o[:, a]) / e[:, a]
    ref = t * t / (area * np.abs(e[:, a]))
    ok = (pl > 0) & (np.abs(e[:, a]) > 1e-2)
    assert ok.mean() > 0.5
    np.testing.assert_allclose(pl[ok], ref[ok], rtol=2e-3)
    # an unoccluded sample above the horizon carries albedo/pi cos Le / p_light
    vis = nl > 0
    assert vis.mean() > 0.3
    alb = w.scene.albedo
    cosv = (e * qn.cpu().numpy()).sum(1)
    assert np.all(cosv[vis] > 0)
    Le = em[lights[0]]
    kval = nl[vis] * pl[vis] * np.pi / (cosv[vis] * Le)
    assert np.all((kval > 0) & (kval <= 1 + 1e-4))     # the albedo of the vertex's surface
    assert np.all(np.min(np.abs(kval[:, None] - alb[None, :]), axis=1) < 1e-3)


@pytest.mark.parametrize("proposal", [0, 1, 2])
def test_nee_frames_are_unbiased_and_less_noisy(proposal):
    """Light sampling combined with the mixture by the power heuristic leaves the
    mean image unchanged (against cosine-only frames without it) and lowers its
    variance in a box lit by a small ceiling light."""
    w, g, _ = box_svo(18)
    frames = 40
    mlp = W.MLP(inputs.mlp_init(5), max_batch=4096) if proposal == 1 else None
    mu0, s0, v0 = _frame_mean(g, w.scene, frames, alpha=0.0, seed=41)
    mu1, s1, v1 = _frame_mean(g, w.scene, frames, mlp=mlp, alpha=0.5, seed=43, nee=True, proposal=proposal, N=32)
    assert abs(mu1 - mu0) < 5 * np.hypot(s0, s1), (mu0, mu1, s0, s1)
    assert v1 < 0.8 * v0, (v0, v1)


def test_nee_without_lights_is_the_plain_frame():
    """A scene with no emissive primitive has nothing to sample: nee = 1 runs
    the same frames as nee = 0 (and both images are black)."""
    import copy
    w, g1, _ = box_svo(19)
    _, g2, _ = box_svo(19)
    sc = copy.deepcopy(w.scene)
    sc.emission = np.zeros_like(sc.emission)
    f1 = make_frame(g1, sc, width=64, height=36, nee=True)
    f2 = make_frame(g2, sc, width=64, height=36, nee=False)
    f1.run(2)
    f2.run(2)
    assert torch.equal(f1.image()[0], f2.image()[0])
    assert float(f1.image()[0].abs().max()) == 0.0
    np.testing.assert_array_equal(g1.exitance()["acc_sum"], g2.exitance()["acc_sum"])
