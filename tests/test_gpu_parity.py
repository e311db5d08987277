"""CUDA path vs the CPU oracle, element by element on the same seeded inputs.

Bar: Morton keys, node layout, fragment lists, integer exitance sums, bin ids,
ray order, origins and sampled cells are bit-exact; PDFs and CDFs match to
1e-5 relative (float32).  Inputs come from paper_2405_06997_gb300.inputs; no
expected value comes from the CUDA path.
"""
import numpy as np
import pytest

import oracle
from paper_2405_06997_gb300 import inputs

pytestmark = pytest.mark.gpu

RTOL = 1e-5

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA device", allow_module_level=True)

from paper_2405_06997_gb300 import wfpg as W  # noqa: E402


def dev(a, dtype=None):
    t = torch.from_numpy(np.ascontiguousarray(a))
    if dtype is not None:
        t = t.to(dtype)
    return t.cuda()


def u32(t):
    return t.cpu().numpy().view(np.uint32)


def build_both(scene, D):
    g = W.svo_from_scene(scene, D)
    o = oracle.SVO(scene, D)
    return g, o


def assert_svo_equal(g, o):
    ge, oe = g.export(), o.export()
    np.testing.assert_array_equal(ge["level_off"], oe["level_off"])
    for k in ("key", "first_child", "child_mask", "parent", "leaf_count"):
        np.testing.assert_array_equal(ge[k], oe[k], err_msg=k)
    np.testing.assert_array_equal(ge["normal"], oe["normal"])
    off, prim = o.frags()
    np.testing.assert_array_equal(ge["frag_off"], off)
    np.testing.assert_array_equal(ge["frag_prim"], prim)


# ------------------------------------------------------------------ SVO build
@pytest.mark.parametrize("D", [1, 3, 6])
def test_svo_build_box(D):
    g, o = build_both(inputs.closed_box(2, D), D)
    assert_svo_equal(g, o)


def test_svo_build_spheres_d7():
    g, o = build_both(inputs.cornell_spheres(3, n_spheres=40), 7)
    assert_svo_equal(g, o)


def test_svo_build_city_d8():
    sc = inputs.city(1, n_boxes=300, n_lights=10, size=500.0)
    g, o = build_both(sc, 8)
    assert_svo_equal(g, o)


# ------------------------------------------------------------------ exitance
def test_accumulate_exact():
    w = inputs.tiny_box(1, n_records=100_003)
    g, o = build_both(w.scene, w.depth)
    W.svo_accumulate(g, dev(w.rec_pos), dev(w.rec_wout), dev(w.rec_L))
    o.accumulate(w.rec_pos, w.rec_wout, w.rec_L)
    # a second batch: sums are a running total
    w2 = inputs.tiny_box(9, n_records=7_777)
    W.svo_accumulate(g, dev(w2.rec_pos), dev(w2.rec_wout), dev(w2.rec_L))
    o.accumulate(w2.rec_pos, w2.rec_wout, w2.rec_L)
    ge, oe = g.exitance(), o.exitance()
    lo = g.level_off
    inner = slice(0, int(lo[w.depth]))
    for k in ("acc_sum", "acc_cnt", "value"):
        np.testing.assert_array_equal(ge[k], oe[k], err_msg=k)
    for k in ("tot_sum", "tot_cnt"):
        np.testing.assert_array_equal(ge[k][inner], oe[k][inner], err_msg=k)


def test_accumulate_over_many_small_batches():
    """300 small batches, each landing in a different corner of the box, leave
    exactly the oracle's running sums and bottom-up averages; after a reset one
    batch gives a fresh tree's values."""
    w = inputs.tiny_box(3, n_records=30_000)
    g, o = build_both(w.scene, w.depth)
    order = np.argsort(w.rec_pos[:, 0] + 2 * w.rec_pos[:, 1] + 4 * w.rec_pos[:, 2])
    chunks = np.array_split(order, 300)
    for c in chunks:
        W.svo_accumulate(g, dev(w.rec_pos[c]), dev(w.rec_wout[c]), dev(w.rec_L[c]))
        o.accumulate(w.rec_pos[c], w.rec_wout[c], w.rec_L[c])
    ge, oe = g.exitance(), o.exitance()
    lo = g.level_off
    inner = slice(0, int(lo[w.depth]))
    for k in ("acc_sum", "acc_cnt", "value"):
        np.testing.assert_array_equal(ge[k], oe[k], err_msg=k)
    for k in ("tot_sum", "tot_cnt"):
        np.testing.assert_array_equal(ge[k][inner], oe[k][inner], err_msg=k)
    # a reset, then one batch
    g.reset_exitance()
    o2 = oracle.SVO(w.scene, w.depth)
    c = chunks[7]
    W.svo_accumulate(g, dev(w.rec_pos[c]), dev(w.rec_wout[c]), dev(w.rec_L[c]))
    o2.accumulate(w.rec_pos[c], w.rec_wout[c], w.rec_L[c])
    np.testing.assert_array_equal(g.exitance()["value"], o2.exitance()["value"])


def test_accumulate_empty_batch():
    w = inputs.tiny_box(1)
    g, o = build_both(w.scene, w.depth)
    z = torch.zeros((0, 3), dtype=torch.float32, device="cuda")
    W.svo_accumulate(g, z, z, torch.zeros(0, dtype=torch.float32, device="cuda"))
    assert np.all(g.exitance()["value"] == 0)


# ------------------------------------------------------------------ binning
@pytest.mark.parametrize("l_min,c_ray", [(2, 0xFFFFFFFF), (1, 100), (3, 16), (0, 0xFFFFFFFF), (6, 1)])
def test_partition_s_exact(l_min, c_ray):
    w = inputs.tiny_box(4, n_rays=4099)
    g, o = build_both(w.scene, w.depth)
    r = W.bin_rays(g, dev(w.ray_pos), l_min=l_min, c_ray=c_ray, seed=7, frame=3)
    ro = o.bin_rays(w.ray_pos, w.ray_nrm, l_min=l_min, c_ray=c_ray, seed=7, frame=3)
    nb = int(r["n_bins"].item())
    assert nb == ro["n_bins"]
    np.testing.assert_array_equal(u32(r["bin_of_ray"]), ro["bin_of_ray"])
    np.testing.assert_array_equal(u32(r["ray_order"]), ro["ray_order"])
    np.testing.assert_array_equal(u32(r["bin_offset"])[: nb + 1], ro["bin_offset"])
    np.testing.assert_array_equal(u32(r["origin_ray"])[:nb], ro["origin_ray"])
    assert g.status() == 0


def test_runs_mode_exact():
    w = inputs.tiny_box(5, n_rays=6001)
    g, o = build_both(w.scene, w.depth)
    sizes = inputs.zipf_bin_sizes(len(w.ray_pos), 97, 1.2, 3)
    r = W.bin_rays(g, dev(w.ray_pos), dev(w.ray_nrm), mode=W.BIN_RUNS, sizes=dev(sizes.view(np.int32)),
                   seed=2, frame=1)
    ro = o.bin_rays(w.ray_pos, w.ray_nrm, mode=1, sizes=sizes, seed=2, frame=1)
    assert int(r["n_bins"].item()) == ro["n_bins"] == 97
    np.testing.assert_array_equal(u32(r["bin_of_ray"]), ro["bin_of_ray"])
    np.testing.assert_array_equal(u32(r["ray_order"]), ro["ray_order"])
    np.testing.assert_array_equal(u32(r["bin_offset"]), ro["bin_offset"])
    np.testing.assert_array_equal(u32(r["origin_ray"]), ro["origin_ray"])
    assert g.status() == 0


def test_bin_capacity_and_bad_sizes_flagged():
    w = inputs.tiny_box(5, n_rays=3000)
    g = W.svo_from_scene(w.scene, w.depth)
    r = W.bin_rays(g, dev(w.ray_pos), l_min=3, c_ray=0xFFFFFFFF, bin_cap=4)
    assert int(r["n_bins"].item()) > 4
    assert g.status() & W.STATUS_BIN_CAPACITY
    bad = np.full(10, 7, np.int32)   # 70 != 3000
    W.bin_rays(g, dev(w.ray_pos), dev(w.ray_nrm), mode=W.BIN_RUNS, sizes=dev(bad))
    assert g.status() & W.STATUS_RUN_SIZES
    assert g.status() == 0  # cleared


def test_zero_and_one_ray():
    w = inputs.tiny_box(5, n_rays=10)
    g, o = build_both(w.scene, w.depth)
    r = W.bin_rays(g, torch.zeros((0, 3), dtype=torch.float32, device="cuda"), bin_cap=4)
    assert int(r["n_bins"].item()) == 0
    assert int(r["bin_offset"][0].item()) == 0
    r = W.bin_rays(g, dev(w.ray_pos[:1]), l_min=2)
    ro = o.bin_rays(w.ray_pos[:1], w.ray_nrm[:1], l_min=2)
    assert int(r["n_bins"].item()) == ro["n_bins"] == 1
    assert int(r["origin_ray"][0].item()) == 0


def test_invalid_arguments_raise():
    w = inputs.tiny_box(5, n_rays=10)
    g = W.svo_from_scene(w.scene, w.depth)
    with pytest.raises(W.WfpgError) as e:
        W.guide_build_pdf(g, dev(w.ray_pos), bin_cap=2, N=12)
    assert e.value.code == -1
    with pytest.raises(W.WfpgError):
        W.guide_build_pdf(g, dev(w.ray_pos), bin_cap=2, N=16, parts=3)
    with pytest.raises(W.WfpgError):
        W.svo_build(dev(w.scene.quads), dev(w.scene.spheres), w.scene.lo, 1.0, 12)
    empty_q = np.array([[0, 5.0, 5.0, 6.0, 5.0, 6.0, 1.0, 0.0]], np.float32)  # outside the box
    with pytest.raises(W.WfpgError):
        W.svo_build(dev(np.array([[3, 0.5, 0, 1, 0, 1, 1, 0]], np.float32)),
                    torch.zeros((0, 4), device="cuda"), (0, 0, 0), 1.0, 4)
    assert empty_q.shape == (1, 8)


# ------------------------------------------------------------------ guide
def _pipeline(w, N, jitter, blur, l_min=2, c_ray=0xFFFFFFFF, seed=11, frame=2):
    g, o = build_both(w.scene, w.depth)
    W.svo_accumulate(g, dev(w.rec_pos), dev(w.rec_wout), dev(w.rec_L))
    o.accumulate(w.rec_pos, w.rec_wout, w.rec_L)
    pos = dev(w.ray_pos)
    r = W.bin_rays(g, pos, l_min=l_min, c_ray=c_ray, seed=seed, frame=frame)
    ro = o.bin_rays(w.ray_pos, w.ray_nrm, l_min=l_min, c_ray=c_ray, seed=seed, frame=frame)
    nb = ro["n_bins"]
    pdf, cr, cm = W.guide_build_pdf(g, pos, r["origin_ray"], r["n_bins"], r["bin_cap"], N=N,
                                    jitter=jitter, blur=blur, seed=seed, frame=frame)
    og = o.guide_build(w.ray_pos[ro["origin_ray"]], np.arange(nb), N, jitter=jitter, blur=blur,
                       seed=seed, frame=frame)
    return g, o, r, ro, (pdf, cr, cm), og, nb


@pytest.mark.parametrize("N,jitter,blur", [(16, False, False), (16, True, True), (8, True, False),
                                           (32, False, True), (64, True, True), (128, True, True)])
def test_guide_build_matches_oracle(N, jitter, blur):
    w = inputs.tiny_box(6, n_rays=4099)
    g, o, r, ro, (pdf, cr, cm), og, nb = _pipeline(w, N, jitter, blur)
    gp = pdf[:nb].cpu().numpy()
    np.testing.assert_allclose(gp, og["pdf"], rtol=RTOL, atol=0)
    np.testing.assert_allclose(cr[:nb].cpu().numpy(), og["cdf_row"], rtol=RTOL, atol=0)
    np.testing.assert_allclose(cm[:nb].cpu().numpy(), og["cdf_marg"], rtol=RTOL, atol=0)
    # the whole chain is specified in binary32 with fixed rounding: expect identity
    assert np.array_equal(gp, og["pdf"])
    assert g.status() == 0


def test_field_from_origins_outside_the_box():
    """Cone rays from origins outside the SVO's box (Sec. 3.3): most of each
    32-cell batch misses the box and ends at its start, so the stream kernel's
    batches keep few or no live rays and its lanes refill over several rounds;
    some origins inside the box mix both kinds of batch.  Fields equal the
    oracle's bit for bit."""
    w = inputs.tiny_box(6, n_rays=64)
    g, o = build_both(w.scene, w.depth)
    W.svo_accumulate(g, dev(w.rec_pos), dev(w.rec_wout), dev(w.rec_L))
    o.accumulate(w.rec_pos, w.rec_wout, w.rec_L)
    rng = np.random.default_rng(5)
    v = rng.normal(size=(48, 3))
    outside = 0.5 + 1.2 * v / np.linalg.norm(v, axis=1, keepdims=True)  # farther than the corners (0.87)
    inside = rng.uniform(0.1, 0.9, size=(16, 3))
    org = np.concatenate([outside, inside]).astype(np.float32)
    n = len(org)
    pdf, cr, cm = W.guide_build_pdf(g, dev(org), None, None, n, N=16, jitter=True, blur=True, seed=7, frame=3)
    og = o.guide_build(org, np.arange(n), 16, jitter=True, blur=True, seed=7, frame=3)
    assert np.array_equal(pdf.cpu().numpy(), og["pdf"])
    np.testing.assert_allclose(cr.cpu().numpy(), og["cdf_row"], rtol=RTOL, atol=0)
    np.testing.assert_allclose(cm.cpu().numpy(), og["cdf_marg"], rtol=RTOL, atol=0)
    # the outside origins see the box in a minority of their cells; the rest hold eps only
    field_min = og["pdf"][:48].min(axis=1, keepdims=True)
    assert np.mean(og["pdf"][:48] == field_min) > 0.5
    assert g.status() == 0


@pytest.mark.parametrize("N", [16, 32])
def test_sample_and_eval_match_oracle(N):
    w = inputs.tiny_box(7, n_rays=4099)
    g, o, r, ro, (pdf, cr, cm), og, nb = _pipeline(w, N, True, True)
    u = dev(w.u)
    d, p, c = W.guide_sample(pdf, cr, cm, N, r["bin_of_ray"], u)
    od, op, oc = oracle.guide_sample(og["pdf"], og["cdf_row"], og["cdf_marg"], N, ro["bin_of_ray"], w.u)
    np.testing.assert_array_equal(u32(c), oc)
    np.testing.assert_allclose(p.cpu().numpy(), op, rtol=RTOL, atol=0)
    np.testing.assert_allclose(d.cpu().numpy(), od, rtol=0, atol=1e-6)
    e = W.guide_eval_pdf(pdf, N, r["bin_of_ray"], d)
    oe = oracle.guide_eval_pdf(og["pdf"], N, ro["bin_of_ray"], od)
    np.testing.assert_allclose(e.cpu().numpy(), oe, rtol=RTOL, atol=0)
    # MIS queries in arbitrary directions
    rng = np.random.default_rng(3)
    v = rng.normal(size=(5000, 3))
    v = (v / np.linalg.norm(v, axis=1, keepdims=True)).astype(np.float32)
    b = rng.integers(0, nb, 5000).astype(np.uint32)
    e2 = W.guide_eval_pdf(pdf, N, dev(b.view(np.int32)), dev(v))
    np.testing.assert_allclose(e2.cpu().numpy(), oracle.guide_eval_pdf(og["pdf"], N, b, v), rtol=RTOL, atol=0)


def test_out_of_range_bins_are_zero():
    w = inputs.tiny_box(7, n_rays=300)
    g, o, r, ro, (pdf, cr, cm), og, nb = _pipeline(w, 16, False, False)
    bins = torch.tensor([0, 10_000_000], dtype=torch.int32, device="cuda")
    d, p, c = W.guide_sample(pdf, cr, cm, 16, bins, torch.full((2, 2), 0.5, device="cuda"))
    assert int(c[1].item()) == -1 and float(p[1].item()) == 0.0
    e = W.guide_eval_pdf(pdf, 16, bins, torch.tensor([[0, 0, 1.0]] * 2, device="cuda"))
    assert float(e[1].item()) == 0.0


def test_furnace_uniform_on_gpu():
    D = 5
    sc = inputs.closed_box(1, D)
    sc.quads = sc.quads[:6]
    g, o = build_both(sc, D)
    oe = o.export()
    lo = g.level_off
    keys = oe["key"][lo[D]:lo[D + 1]]
    cells = np.array([[sum(((int(k) >> (3 * i + a)) & 1) << i for i in range(D)) for a in range(3)]
                      for k in keys], np.float64)
    pos = ((cells + 0.5) / (1 << D)).astype(np.float32)
    W.svo_accumulate(g, dev(pos), dev(oe["normal"][lo[D]:lo[D + 1]]), dev(np.ones(len(pos), np.float32)))
    origin = dev(np.array([[0.5, 0.5, 0.5]], np.float32))
    pdf, _, _ = W.guide_build_pdf(g, origin, N=32, jitter=True, blur=True)
    np.testing.assert_allclose(pdf.cpu().numpy(), 1 / (4 * np.pi), rtol=1e-6)


# ------------------------------------------------------------------ frame-scale
@pytest.fixture(scope="module")
def frame_workload():
    return inputs.frame_spheres(1)


def test_frame_scale_sampled_parity(frame_workload):
    """The 1080p workload of the benchmark (D = 9, 2048 Zipf bins, 32 x 32,
    blur + jitter): whole SVO, sums and bins compared exactly; fields, CDFs and
    samples compared on a sample of bins the oracle recomputes one by one."""
    w = frame_workload
    g, o = build_both(w.scene, w.depth)
    assert_svo_equal(g, o)
    W.svo_accumulate(g, dev(w.rec_pos), dev(w.rec_wout), dev(w.rec_L))
    o.accumulate(w.rec_pos, w.rec_wout, w.rec_L)
    ge, oe = g.exitance(), o.exitance()
    np.testing.assert_array_equal(ge["acc_sum"], oe["acc_sum"])
    np.testing.assert_array_equal(ge["value"], oe["value"])
    pos = dev(w.ray_pos)
    sizes = dev(w.bin_sizes.view(np.int32))
    r = W.bin_rays(g, pos, dev(w.ray_nrm), mode=W.BIN_RUNS, sizes=sizes, seed=w.seed, frame=0)
    ro = o.bin_rays(w.ray_pos, w.ray_nrm, mode=1, sizes=w.bin_sizes, seed=w.seed, frame=0)
    np.testing.assert_array_equal(u32(r["bin_of_ray"]), ro["bin_of_ray"])
    np.testing.assert_array_equal(u32(r["origin_ray"]), ro["origin_ray"])
    N = w.grid_n
    pdf, cr, cm = W.guide_build_pdf(g, pos, r["origin_ray"], r["n_bins"], r["bin_cap"], N=N,
                                    jitter=True, blur=True, seed=w.seed, frame=0)
    sel = np.unique(np.concatenate([np.arange(0, 2048, 97), [2047], np.argsort(w.bin_sizes)[-3:]]))
    og = o.guide_build(w.ray_pos[ro["origin_ray"][sel]], sel, N, jitter=True, blur=True, seed=w.seed,
                       frame=0)
    gp = pdf.cpu().numpy()[sel]
    np.testing.assert_allclose(gp, og["pdf"], rtol=RTOL, atol=0)
    np.testing.assert_allclose(cr.cpu().numpy()[sel], og["cdf_row"], rtol=RTOL, atol=0)
    assert np.array_equal(gp, og["pdf"])
    d, p, c = W.guide_sample(pdf, cr, cm, N, r["bin_of_ray"], dev(w.u))
    rays = np.flatnonzero(np.isin(ro["bin_of_ray"], sel))
    remap = {int(b): k for k, b in enumerate(sel)}
    local = np.array([remap[int(b)] for b in ro["bin_of_ray"][rays]], np.uint32)
    od, op, oc = oracle.guide_sample(og["pdf"], og["cdf_row"], og["cdf_marg"], N, local, w.u[rays])
    np.testing.assert_array_equal(u32(c)[rays], oc)
    np.testing.assert_allclose(p.cpu().numpy()[rays], op, rtol=RTOL, atol=0)
    np.testing.assert_allclose(d.cpu().numpy()[rays], od, rtol=0, atol=1e-6)
    assert g.status() == 0


@pytest.mark.parametrize("block", [64, 128, 256])
@pytest.mark.parametrize("stage", [1, -1])
def test_guide_build_tile_variants(block, stage):
    """Every block size / staging choice of the field kernel gives the oracle's field."""
    w = inputs.tiny_box(6, n_rays=4099)
    g, o = build_both(w.scene, w.depth)
    W.svo_accumulate(g, dev(w.rec_pos), dev(w.rec_wout), dev(w.rec_L))
    o.accumulate(w.rec_pos, w.rec_wout, w.rec_L)
    pos = dev(w.ray_pos)
    r = W.bin_rays(g, pos, l_min=2, seed=11, frame=2)
    ro = o.bin_rays(w.ray_pos, w.ray_nrm, l_min=2, seed=11, frame=2)
    nb = ro["n_bins"]
    for N in (32, 64):
        pdf, cr, cm = W.guide_build_pdf(g, pos, r["origin_ray"], r["n_bins"], r["bin_cap"], N=N, jitter=True,
                                        blur=True, seed=11, frame=2, block=block, stage=stage)
        og = o.guide_build(w.ray_pos[ro["origin_ray"]], np.arange(nb), N, jitter=True, blur=True, seed=11, frame=2)
        assert np.array_equal(pdf[:nb].cpu().numpy(), og["pdf"])
        assert np.array_equal(cm[:nb].cpu().numpy(), og["cdf_marg"])
    assert g.status() == 0


@pytest.mark.parametrize("D", [7, 8, 10])
def test_field_kernel_depth_specialisations(D):
    """The stream field kernel is compiled for each SVO depth 6 .. 11 (depths 6, 9 and 11 run in
    the tests above): at depths 7, 8 and 10 its fields equal the oracle's bit for bit."""
    sc = inputs.small_deep(1)
    g, o = build_both(sc, D)
    rng = np.random.default_rng(7)
    pos, nrm, prim = inputs.surface_points(sc, rng, 20000)
    wout = inputs.cosine_dirs(nrm, rng).astype(np.float32)
    L = np.where(prim == 3, 10.0, sc.albedo[prim] * 10.0 * rng.uniform(0, 1, len(prim))).astype(np.float32)
    W.svo_accumulate(g, dev(pos), dev(wout), dev(L))
    o.accumulate(pos, wout, L)
    rp, rn, _ = inputs.surface_points(sc, np.random.default_rng(8), 3001)
    r = W.bin_rays(g, dev(rp), dev(rn), l_min=3, c_ray=64, seed=5, frame=2)
    ro = o.bin_rays(rp, rn, l_min=3, c_ray=64, seed=5, frame=2)
    nb = ro["n_bins"]
    np.testing.assert_array_equal(u32(r["origin_ray"])[:nb], ro["origin_ray"][:nb])
    pdf, cr, cm = W.guide_build_pdf(g, dev(rp), r["origin_ray"], r["n_bins"], r["bin_cap"], N=16, jitter=True,
                                    blur=True, seed=5, frame=2)
    sel = np.arange(0, nb, max(1, nb // 16))
    og = o.guide_build(rp[ro["origin_ray"][sel]], sel, 16, jitter=True, blur=True, seed=5, frame=2)
    assert np.array_equal(pdf.cpu().numpy()[sel], og["pdf"])
    assert g.status() == 0


# ------------------------------------------------------------------ maximum depth
def test_depth_11_end_to_end_exact():
    """Depth 11 (2048^3, 33-bit Morton keys): SVO layout, exitance sums, bins,
    origins and the traced fields equal the oracle's bit for bit."""
    sc = inputs.small_deep(1)
    D = 11
    g, o = build_both(sc, D)
    assert_svo_equal(g, o)
    rng = np.random.default_rng(5)
    pos, nrm, prim = inputs.surface_points(sc, rng, 20000)
    wout = inputs.cosine_dirs(nrm, rng).astype(np.float32)
    L = np.where(prim == 3, 10.0, sc.albedo[prim] * 10.0 * rng.uniform(0, 1, len(prim))).astype(np.float32)
    W.svo_accumulate(g, dev(pos), dev(wout), dev(L))
    o.accumulate(pos, wout, L)
    ge, oe = g.exitance(), o.exitance()
    np.testing.assert_array_equal(ge["acc_sum"], oe["acc_sum"])
    np.testing.assert_array_equal(ge["value"], oe["value"])
    rp, rn, _ = inputs.surface_points(sc, np.random.default_rng(6), 3001)
    for l_min, c_ray in ((3, 0xFFFFFFFF), (8, 64)):
        r = W.bin_rays(g, dev(rp), dev(rn), l_min=l_min, c_ray=c_ray, seed=4, frame=1)
        ro = o.bin_rays(rp, rn, l_min=l_min, c_ray=c_ray, seed=4, frame=1)
        nb = ro["n_bins"]
        np.testing.assert_array_equal(u32(r["bin_of_ray"]), ro["bin_of_ray"])
        np.testing.assert_array_equal(u32(r["origin_ray"])[:nb], ro["origin_ray"][:nb])
    pdf, cr, cm = W.guide_build_pdf(g, dev(rp), r["origin_ray"], r["n_bins"], r["bin_cap"], N=16, jitter=True,
                                    blur=True, seed=4, frame=1)
    sel = np.arange(0, nb, max(1, nb // 12))
    og = o.guide_build(rp[ro["origin_ray"][sel]], sel, 16, jitter=True, blur=True, seed=4, frame=1)
    assert np.array_equal(pdf.cpu().numpy()[sel], og["pdf"])
    assert g.status() == 0


@pytest.mark.parametrize("parts", [2, 8])
def test_split_bins_give_identical_tables(parts):
    """A bin's cells traced by several CTAs (the last one finishing the bin)
    give the same tables as one CTA per bin, bit for bit."""
    w = inputs.tiny_box(8, n_rays=4099)
    g, o = build_both(w.scene, w.depth)
    W.svo_accumulate(g, dev(w.rec_pos), dev(w.rec_wout), dev(w.rec_L))
    pos = dev(w.ray_pos)
    r = W.bin_rays(g, pos, l_min=2, seed=3, frame=1)
    kw = dict(N=32, jitter=True, blur=True, seed=3, frame=1)
    one = W.guide_build_pdf(g, pos, r["origin_ray"], r["n_bins"], r["bin_cap"], parts=1, **kw)
    split = W.guide_build_pdf(g, pos, r["origin_ray"], r["n_bins"], r["bin_cap"], parts=parts, **kw)
    nb = int(r["n_bins"].item())
    for a, b in zip(one, split):
        assert torch.equal(a[:nb], b[:nb])
    assert g.status() == 0
