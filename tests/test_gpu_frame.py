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
