"""Host-side argument checks of the C ABI, without a GPU.

Every call below is rejected by the checks that run before the library
touches the device, so it returns its documented error code, leaves the
output handle NULL and sets wfpg_last_error(); no kernel is launched and no
CUDA call is made.
"""
import ctypes as C

import numpy as np
import pytest

from paper_2405_06997_gb300 import build
from paper_2405_06997_gb300 import wfpg as W

P, U32, I32, F, SZ = C.c_void_p, C.c_uint32, C.c_int, C.c_float, C.c_size_t
INVALID, CAPACITY = -1, -5


@pytest.fixture(scope="module")
def lib():
    L = C.CDLL(build.build())
    sig = {
        "svo_build": [P, I32, P, P],
        "svo_destroy": [P],
        "svo_get_info": [P, P],
        "svo_reset_exitance": [P, P],
        "svo_accumulate": [P, P, P, P, U32, P],
        "bin_rays_workspace_size": [P, U32, P, P],
        "bin_rays": [P, P, P, U32, P, P, P, P, P, P, U32, P, P, SZ, P],
        "guide_build_pdf": [P, P, P, P, U32, P, P, P, P, P],
        "guide_build_sample_workspace_size": [I32, U32, U32, P],
        "guide_sample": [P, P, P, I32, U32, P, P, U32, P, P, P, P],
        "guide_eval_pdf": [P, I32, U32, P, P, U32, P, P],
        "guide_sample_mix": [P, P, P, I32, U32, P, P, P, P, U32, P, F, P, P, P],
        "guide_product_sums": [P, I32, U32, P, P, P],
        "guide_product_sample": [P, P, I32, U32, P, P, P, P, U32, P, F, P, P, P, P],
        "guide_product_eval": [P, P, I32, U32, P, P, P, P, U32, F, P, P],
        "svo_export": [P, P, P, P, P, P, P, P, P, P],
        "svo_export_exitance": [P, P, P, P, P, P, P],
        "wfpg_svo_status": [P, P, I32, P],
        "frame_create": [P, P, P, P, P, P, P, P],
        "frame_destroy": [P],
        "mlp_create": [P, U32, P, P],
        "bin_rays_static": [P, P, P, U32, P, P, P, P, P, P, U32, P, P],
        "guide_learned_logits": [P, P, P, U32, P, P, P],
        "guide_learned_train_step": [P, P, P, U32, P, P, P, P, P, P],
        "mlp_adam_step": [P, P, P, P],
    }
    for name, args in sig.items():
        fn = getattr(L, name)
        fn.restype = I32
        fn.argtypes = args
    L.wfpg_last_error.restype = C.c_char_p
    L.wfpg_last_error.argtypes = []
    return L


def err(L):
    return L.wfpg_last_error().decode()


def host_buf(nbytes=256):
    """A host buffer whose address stands in for a device pointer the checks
    only test for NULL or alignment (never dereferenced)."""
    return (C.c_char * nbytes)()


def scene(**kw):
    q = host_buf()
    s = W.Scene()
    s.quads, s.n_quads = C.addressof(q), 1
    s.lo[:] = (0.0, 0.0, 0.0)
    s.size = 1.0
    for k, v in kw.items():
        setattr(s, k, v)
    return s, q


@pytest.mark.parametrize("case, msg", [
    (dict(depth=0), "depth"),
    (dict(depth=W.MAX_DEPTH + 1), "depth"),
    (dict(n_quads=0), "no primitive"),
    (dict(n_quads=1 << 20), "2^20"),
    (dict(quads=None), "null primitive"),
    (dict(n_spheres=3), "null primitive"),
    (dict(n_tris=2), "null primitive"),
    (dict(size=0.0), "size"),
    (dict(size=float("nan")), "size"),
    (dict(size=float("inf")), "size"),
])
def test_svo_build_rejects(lib, case, msg):
    case = dict(case)
    depth = case.pop("depth", 4)
    s, keep = scene(**case)
    out = P(12345)
    assert lib.svo_build(C.byref(s), depth, None, C.byref(out)) == INVALID
    assert out.value is None
    assert msg in err(lib)
    assert lib.svo_build(None, 4, None, C.byref(out)) == INVALID
    assert lib.svo_build(C.byref(s), 4, None, None) == INVALID


def test_null_handles_are_rejected(lib):
    info = W.SvoInfo()
    flags = U32()
    nbytes = SZ()
    bp = W.BinParams()
    gp = W.GuideParams()
    gp.N = 16
    assert lib.svo_destroy(None) == 0  # like free(NULL)
    assert lib.svo_get_info(None, C.byref(info)) == INVALID
    assert lib.svo_reset_exitance(None, None) == INVALID
    assert lib.svo_accumulate(None, None, None, None, 0, None) == INVALID
    assert lib.bin_rays_workspace_size(None, 10, C.byref(bp), C.byref(nbytes)) == INVALID
    assert lib.bin_rays(None, None, None, 0, C.byref(bp), None, None, None, None, None, 0, None, None, 0,
                        None) == INVALID
    assert lib.guide_build_pdf(None, None, None, None, 0, C.byref(gp), None, None, None, None) == INVALID
    assert lib.svo_export(None, None, None, None, None, None, None, None, None, None) == INVALID
    assert lib.svo_export_exitance(None, None, None, None, None, None, None) == INVALID
    assert lib.wfpg_svo_status(None, C.byref(flags), 0, None) == INVALID
    assert lib.frame_destroy(None) == 0


def test_bin_rays_checks_mode_sizes_and_capacity(lib):
    """The SVO handle is only tested for NULL before these checks."""
    b = C.addressof(host_buf())
    sizes = (U32 * 4)(5, 5, 5, 5)

    def call(mode, n, nrm=b, sz=sizes, n_sizes=4, bin_cap=8):
        bp = W.BinParams()
        bp.mode, bp.n_sizes = mode, n_sizes
        return lib.bin_rays(b, b, nrm, n, C.byref(bp), sz, b, b, b, b, bin_cap, b, None, 0, None)

    assert call(7, 10) == INVALID and "mode" in err(lib)
    assert call(W.BIN_PARTITION_S, 0x80000000) == INVALID and "2^31" in err(lib)
    assert call(W.BIN_RUNS, 10, nrm=None) == INVALID and "nrm" in err(lib)
    assert call(W.BIN_RUNS, 10, sz=None) == INVALID and "sizes" in err(lib)
    assert call(W.BIN_RUNS, 10, n_sizes=0) == INVALID and "sizes" in err(lib)
    assert call(W.BIN_RUNS, 10, n_sizes=4, bin_cap=3) == CAPACITY and "bin_cap" in err(lib)
    nb = SZ()
    bp = W.BinParams()
    bp.mode = 9
    assert lib.bin_rays_workspace_size(b, 10, C.byref(bp), C.byref(nb)) == INVALID and "mode" in err(lib)


def test_bin_rays_static_checks_mode_sizes_and_capacity(lib):
    """The allocation-free binning call makes bin_rays's argument checks before
    it looks at its static scratch or the device."""
    b = C.addressof(host_buf())
    sizes = (U32 * 4)(5, 5, 5, 5)

    def call(mode, n, svo=b, nrm=b, sz=sizes, n_sizes=4, bin_cap=8, params=True):
        bp = W.BinParams()
        bp.mode, bp.n_sizes = mode, n_sizes
        return lib.bin_rays_static(svo, b, nrm, n, C.byref(bp) if params else None, sz, b, b, b, b, bin_cap, b,
                                   None)

    assert call(W.BIN_PARTITION_S, 10, svo=None) == INVALID and "null svo" in err(lib)
    assert call(W.BIN_PARTITION_S, 10, params=False) == INVALID and "null svo or params" in err(lib)
    assert call(7, 10) == INVALID and "mode" in err(lib)
    assert call(W.BIN_PARTITION_S, 0x80000000) == INVALID and "2^31" in err(lib)
    assert call(W.BIN_RUNS, 10, nrm=None) == INVALID and "nrm" in err(lib)
    assert call(W.BIN_RUNS, 10, sz=None) == INVALID and "sizes" in err(lib)
    assert call(W.BIN_RUNS, 10, n_sizes=0) == INVALID and "sizes" in err(lib)
    assert call(W.BIN_RUNS, 10, n_sizes=4, bin_cap=3) == CAPACITY and "bin_cap" in err(lib)
    assert err(lib).startswith("bin_rays_static:")


def test_learned_logits_and_adam_step_check_their_arguments(lib):
    b = C.addressof(host_buf())
    lp = W.LearnedParams()
    lp.size = 1.0
    opt = W.AdamParams(lr=1e-3, beta1=0.9, beta2=0.999, eps=1e-8, update=1)
    assert lib.guide_learned_logits(None, b, b, 4, C.byref(lp), b, None) == INVALID and "null" in err(lib)
    assert lib.guide_learned_logits(b, None, b, 4, C.byref(lp), b, None) == INVALID
    assert lib.guide_learned_logits(b, b, b, 4, None, b, None) == INVALID
    assert lib.guide_learned_logits(b, b, b, 4, C.byref(lp), None, None) == INVALID
    assert lib.mlp_adam_step(None, b, C.byref(opt), None) == INVALID and "null" in err(lib)
    assert lib.mlp_adam_step(b, None, C.byref(opt), None) == INVALID
    assert lib.mlp_adam_step(b, b, None, None) == INVALID
    for bad in (dict(lr=-1.0), dict(beta1=1.0), dict(beta2=-0.5), dict(eps=-1e-8)):
        o = W.AdamParams(lr=1e-3, beta1=0.9, beta2=0.999, eps=1e-8, update=1)
        for k, v in bad.items():
            setattr(o, k, v)
        assert lib.mlp_adam_step(b, b, C.byref(o), None) == INVALID and "beta1" in err(lib)


def test_learned_train_step_checks_its_arguments(lib):
    """Null arguments, then the target's 32-byte alignment (the kernel reads
    target rows with 32-byte loads), then the batch size against the handle's
    capacity (a zeroed stand-in handle has max_batch 0)."""
    keep = host_buf(8192)
    b = C.addressof(keep)
    a32 = (b + 31) // 32 * 32
    lp = W.LearnedParams()
    lp.size = 1.0
    opt = W.AdamParams(lr=1e-3, beta1=0.9, beta2=0.999, eps=1e-8, update=1)

    def call(mlp=a32, pos=a32, nrm=a32, n=4, target=a32, p=C.byref(lp), o=C.byref(opt)):
        return lib.guide_learned_train_step(mlp, pos, nrm, n, target, p, o, None, None, None)

    assert call(mlp=None) == INVALID and "null argument" in err(lib)
    assert call(p=None) == INVALID and "null argument" in err(lib)
    assert call(o=None) == INVALID and "null argument" in err(lib)
    assert call(target=None) == INVALID and "null array" in err(lib)
    assert call(pos=None) == INVALID and "null array" in err(lib)
    for off in (4, 16):
        assert call(target=a32 + off) == INVALID and "32-byte aligned" in err(lib)
    assert call() == CAPACITY and "max_batch" in err(lib)
    assert err(lib).startswith("guide_learned_train_step:")


def test_guide_build_checks_its_parameters(lib):
    b = C.addressof(host_buf())

    def call(**kw):
        gp = W.GuideParams()
        gp.N, gp.eps = 16, 1e-2
        for k, v in kw.items():
            setattr(gp, k, v)
        return lib.guide_build_pdf(b, b, b, b, 4, C.byref(gp), b, b, b, None)

    for kw, msg in ((dict(N=20), "N must be"), (dict(parts=3), "parts"), (dict(eps=-1.0), "eps"),
                    (dict(eps=float("nan")), "eps"), (dict(block=32), "block")):
        assert call(**kw) == INVALID and msg in err(lib), kw
    gp = W.GuideParams()
    gp.N, gp.eps = 16, 1e-2
    assert lib.guide_build_pdf(b, None, b, b, 4, C.byref(gp), b, b, b, None) == INVALID and "null" in err(lib)


@pytest.mark.parametrize("N", [0, 4, 12, 48, 256])
def test_grid_side_must_be_a_supported_power_of_two(lib, N):
    b = C.addressof(host_buf())
    nbytes = SZ()
    assert lib.guide_build_sample_workspace_size(N, 100, 0, C.byref(nbytes)) == INVALID
    assert lib.guide_sample(b, b, b, N, 1, b, b, 1, b, b, b, None) == INVALID
    assert lib.guide_eval_pdf(b, N, 1, b, b, 1, b, None) == INVALID
    assert lib.guide_sample_mix(b, b, b, N, 1, None, b, b, b, 1, None, 0.5, b, b, None) == INVALID
    assert lib.guide_product_sums(b, N, 1, None, b, None) == INVALID
    assert lib.guide_product_sample(b, b, N, 1, None, b, b, b, 1, None, 0.5, b, b, None, None) == INVALID
    assert lib.guide_product_eval(b, b, N, 1, None, b, b, b, 1, 0.5, b, None) == INVALID
    assert "N must be" in err(lib)


@pytest.mark.parametrize("alpha", [-0.1, 1.5, float("nan")])
def test_mixture_weight_must_lie_in_the_unit_interval(lib, alpha):
    b = C.addressof(host_buf())
    assert lib.guide_sample_mix(b, b, b, 16, 1, None, b, b, b, 1, None, alpha, b, b, None) == INVALID
    assert lib.guide_product_sample(b, b, 16, 1, None, b, b, b, 1, None, alpha, b, b, None, None) == INVALID
    assert lib.guide_product_eval(b, b, 16, 1, None, b, b, b, 1, alpha, b, None) == INVALID
    assert "alpha" in err(lib)


def test_null_arrays_with_work_are_rejected(lib):
    b = C.addressof(host_buf())
    assert lib.guide_sample(b, b, b, 16, 1, b, b, 1, b, b, None, None) == INVALID  # cell
    assert lib.guide_eval_pdf(b, 16, 1, b, None, 1, b, None) == INVALID
    assert lib.guide_sample_mix(b, b, None, 16, 1, None, b, b, b, 1, None, 0.5, b, b, None) == INVALID
    assert lib.guide_product_sums(None, 16, 1, None, b, None) == INVALID
    assert lib.guide_product_eval(b, b, 16, 1, None, b, b, b, 1, 0.5, None, None) == INVALID
    assert "null" in err(lib)


def test_guide_sample_wants_aligned_uniform_pairs(lib):
    buf = host_buf(64)
    b = C.addressof(buf)
    base = (b + 15) // 16 * 16
    assert lib.guide_sample(b, b, b, 16, 1, b, base + 4, 1, b, b, b, None) == INVALID
    assert "aligned" in err(lib)


def test_fused_workspace_size_follows_the_split(lib):
    """Spill slots: one per `split` rays plus one, each holding a bin's pdf,
    row CDF and marginal CDF; split = 0xFFFFFFFF turns spilling off."""
    sizes = {}
    for N in (16, 32):
        for n, split in ((0, 0), (100000, 0), (100000, 2048), (100000, 0xFFFFFFFF), (100000, 4096)):
            nb = SZ()
            assert lib.guide_build_sample_workspace_size(N, n, split, C.byref(nb)) == 0
            sizes[N, n, split] = nb.value
    for N in (16, 32):
        assert sizes[N, 100000, 2048] > sizes[N, 100000, 4096] > sizes[N, 100000, 0xFFFFFFFF]
        # the default split is 2048 rays
        assert sizes[N, 100000, 0] == sizes[N, 100000, 2048]
        assert sizes[N, 0, 0] < sizes[N, 100000, 0]
        slot = 4 * (2 * N * N + N)
        grow = sizes[N, 100000, 2048] - sizes[N, 100000, 4096]
        assert grow >= (100000 // 2048 - 100000 // 4096) * slot
    assert sizes[32, 100000, 2048] > sizes[16, 100000, 2048]


def camera(**kw):
    c = W.Camera()
    c.eye[:] = (0.5, 0.5, 0.05)
    c.forward[:] = (0.0, 0.0, 1.0)
    c.up[:] = (0.0, 1.0, 0.0)
    c.vfov_deg = 60.0
    c.width, c.height = 64, 36
    for k, v in kw.items():
        setattr(c, k, v)
    return c


def frame_params(**kw):
    p = W.FrameParams()
    p.max_depth, p.rr_depth, p.alpha, p.l_min, p.c_ray = 4, 2, 0.5, 2, 512
    p.guide.N, p.guide.eps, p.guide.jitter, p.guide.blur = 16, 1e-2, 1, 1
    for k, v in kw.items():
        if k.startswith("guide_"):
            setattr(p.guide, k[6:], v)
        else:
            setattr(p, k, v)
    return p


@pytest.mark.parametrize("cam_kw, p_kw, msg", [
    (dict(width=0), {}, "image size"),
    (dict(width=1 << 16, height=1 << 14), {}, "image size"),
    (dict(vfov_deg=0.0), {}, "vfov"),
    (dict(vfov_deg=180.0), {}, "vfov"),
    (dict(probe_n=0, width=16), dict(), "probe"),
    (dict(probe_n=4, width=15), dict(), "probe"),
    ({}, dict(max_depth=0), "max_depth"),
    ({}, dict(max_depth=W.FRAME_MAX_DEPTH + 1), "max_depth"),
    ({}, dict(alpha=1.5), "alpha"),
    ({}, dict(guide_N=24), "N must be"),
    ({}, dict(guide_eps=-1.0), "eps"),
    ({}, dict(guide_block=96), "block"),
    ({}, dict(c_ray=0), "c_ray"),
    ({}, dict(guide_split=100), "split"),
    ({}, dict(caster=3), "caster"),
    ({}, dict(proposal=3), "proposal"),
    ({}, dict(proposal=1, guide_N=16), "learned"),
    ({}, dict(combine=6), "combine"),
    ({}, dict(nee=2), "nee"),
])
def test_frame_create_rejects(lib, cam_kw, p_kw, msg):
    probe = host_buf()
    if "probe_n" in cam_kw:
        cam_kw = dict(cam_kw, probe_pos=C.addressof(probe))
    cam, p = camera(**cam_kw), frame_params(**p_kw)
    s, keep = scene()
    b = C.addressof(host_buf())
    out = P(12345)
    # the SVO handle is only tested for NULL before these checks
    assert lib.frame_create(b, C.byref(s), b, b, C.byref(cam), C.byref(p), C.byref(out), None) == INVALID
    assert out.value is None
    assert msg in err(lib), err(lib)


def test_frame_create_rejects_null_arguments(lib):
    cam, p = camera(), frame_params()
    s, keep = scene()
    b = C.addressof(host_buf())
    out = P()
    assert lib.frame_create(None, C.byref(s), b, b, C.byref(cam), C.byref(p), C.byref(out), None) == INVALID
    assert lib.frame_create(b, C.byref(s), None, b, C.byref(cam), C.byref(p), C.byref(out), None) == INVALID
    assert lib.frame_create(b, C.byref(s), b, b, C.byref(cam), None, C.byref(out), None) == INVALID
    assert "null" in err(lib)


@pytest.mark.parametrize("max_batch", [0, (1 << 24) + 1])
def test_mlp_create_rejects_batch_size(lib, max_batch):
    out = P(12345)
    assert lib.mlp_create(None, max_batch, None, C.byref(out)) == INVALID
    assert out.value is None
    assert "max_batch" in err(lib)
    assert lib.mlp_create(None, 16, None, None) == INVALID


def test_last_error_is_per_thread(lib):
    import threading

    s, keep = scene(size=0.0)
    out = P()
    assert lib.svo_build(C.byref(s), 4, None, C.byref(out)) == INVALID
    main_msg = err(lib)
    seen = []

    def other():
        seen.append(err(lib))
        lib.mlp_create(None, 0, None, C.byref(P()))
        seen.append(err(lib))

    t = threading.Thread(target=other)
    t.start()
    t.join()
    assert seen[0] == "" and "max_batch" in seen[1]
    assert err(lib) == main_msg


def test_error_codes_match_the_header():
    import os
    import re

    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    text = open(os.path.join(root, "include", "wfpg.h")).read()
    codes = {m[0]: int(m[1]) for m in re.findall(r"WFPG_ERR_(\w+)\s*=\s*(-?\d+)", text)}
    assert codes, "no error codes found in the header"
    for v, name in W.ERRORS.items():
        assert codes[name] == v, name
    assert np.all(np.array(sorted(codes.values())) < 0)
