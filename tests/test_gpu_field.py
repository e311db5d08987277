"""Radiance-field validation (Fig. 3): the frame's probe mode path-traces the
incident radiance at free-space points per cell of the concentric octahedral
grid, and the SVO-traced field at those points is compared with it.

* probe rays leave their point inside their own cell (cells by the oracle's
  octahedral encoding of the exported directions);
* cells that lie wholly inside the ceiling light's solid angle see exactly its
  emitted radiance in every frame;
* the traced field's distribution moves toward the path-traced reference as
  the frame's records replace the synthetic seed records in the cache (KL of
  the reference to the traced PDF), and beats the uniform distribution.
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

EYE = (0.5, 0.5, 0.05)


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def seeded_box(seed):
    w = inputs.tiny_box(seed)
    g = W.svo_from_scene(w.scene, w.depth)
    W.svo_accumulate(g, dev(w.rec_pos), dev(w.rec_wout), dev(w.rec_L))
    return w, g


def probe_points(n, seed):
    rng = np.random.default_rng(seed)
    return rng.uniform(0.25, 0.75, (n, 3)).astype(np.float32)


def probe_frame(g, scene, pts, n, **kw):
    args = dict(eye=EYE, max_depth=4, rr_depth=2, alpha=0.0, l_min=2, c_ray=512, N=16, seed=7, update=False,
                nee=True, probes=pts, probe_n=n)
    args.update(kw)
    return W.Frame(g, scene, **args)


def cells_of(d, n):
    uv = oracle.octa_encode(np.ascontiguousarray(d, np.float32))
    i = np.clip(np.floor((uv[:, 0].astype(np.float64) + 1) * n / 2), 0, n - 1).astype(np.int64)
    j = np.clip(np.floor((uv[:, 1].astype(np.float64) + 1) * n / 2), 0, n - 1).astype(np.int64)
    return j * n + i


def traced_pdf(g, pts, N, **kw):
    n = pts.shape[0]
    pos = dev(pts)
    nb = torch.tensor([n], dtype=torch.int32, device="cuda")
    org = torch.arange(n, dtype=torch.int32, device="cuda")
    pdf, _, _ = W.guide_build_pdf(g, pos, org, nb, n, N=N, **kw)
    return pdf.double().cpu().numpy()


def kl(q, p):
    q = q / q.sum(axis=1, keepdims=True)
    p = p / p.sum(axis=1, keepdims=True)
    m = q > 0
    return float(np.sum(np.where(m, q * np.log(np.where(m, q, 1) / p), 0)) / q.shape[0])


def test_probe_rays_start_in_their_cells():
    w, g = seeded_box(1)
    pts = probe_points(6, 1)
    n = 12
    f = probe_frame(g, w.scene, pts, n, max_depth=1)
    f.run(1, use_graph=False)
    P = f.pixels
    assert P == 6 * n * n
    nv = f.export("nv").cpu().numpy()
    assert np.all(nv >= 1)  # a closed box: every direction hits a wall
    d = -f.export("vwo")[:P].cpu().numpy()
    np.testing.assert_array_equal(cells_of(d, n), np.tile(np.arange(n * n), 6))
    # the first vertex lies on the probe ray
    x = f.export("vpos")[:P].cpu().numpy().astype(np.float64)
    o = np.repeat(pts.astype(np.float64), n * n, axis=0)
    t = np.sum((x - o) * d, axis=1)
    np.testing.assert_allclose(x, o + t[:, None] * d, atol=2e-5)


def test_cells_inside_the_light_see_exactly_its_radiance():
    w, g = seeded_box(2)
    q = w.scene.quads.astype(np.float64)
    li = int(np.flatnonzero(w.scene.emission[:len(q)] > 0)[0])
    Ql = q[li]
    a = int(Ql[0])
    b, c = (a + 1) % 3, (a + 2) % 3
    pt = np.array([[0.5, 0.7, 0.5]], np.float32)
    n = 16
    # a cell lies inside the light when a dense set of its directions (edges included) hits the light
    s = np.linspace(0.0, 1.0, 9)
    inside, outside = [], []
    for cell in range(n * n):
        i, j = cell % n, cell // n
        uu, vv = np.meshgrid((i + s) * 2 / n - 1, (j + s) * 2 / n - 1)
        d = oracle.octa_decode(np.stack([uu.ravel(), vv.ravel()], 1).astype(np.float32)).astype(np.float64)
        with np.errstate(divide="ignore", invalid="ignore"):
            t = (Ql[1] - pt[0, a]) / d[:, a]
            hb = pt[0, b] + t * d[:, b]
            hc = pt[0, c] + t * d[:, c]
        m = 1e-3
        if np.all((t > 0) & (hb > Ql[2] + m) & (hb < Ql[3] - m) & (hc > Ql[4] + m) & (hc < Ql[5] - m)):
            inside.append(cell)
        if not np.any((t > 0) & (hb > Ql[2] - m) & (hb < Ql[3] + m) & (hc > Ql[4] - m) & (hc < Ql[5] + m)):
            outside.append(cell)
    assert len(inside) >= 4
    f = probe_frame(g, w.scene, pt, n)
    frames = 8
    f.run(frames)
    m, v = f.image()
    m, v = m.cpu().numpy().ravel(), v.cpu().numpy().ravel()
    Le = float(w.scene.emission[li])
    assert np.all(m[inside] == np.float32(Le))
    assert np.all(v[inside] == 0)
    assert len(outside) > n * n // 2
    assert np.all(m[outside] < Le)  # walls reflect less than the light emits


def test_traced_field_approaches_the_path_traced_reference():
    """An empty cache traces the uniform field (eps everywhere); the records of
    the frame's own paths (Eq. 5 with light samples) alone bring the traced
    field most of the way to the reference.  What remains is mostly the light
    seen at the coarser level Eq. 6 picks for distant cells (a blurred light)."""
    w = inputs.tiny_box(3)
    g = W.svo_from_scene(w.scene, w.depth)
    pts = probe_points(12, 3)
    N = 16
    ref = probe_frame(g, w.scene, pts, N)
    ref.run(96)
    Lref = ref.image()[0].double().cpu().numpy().reshape(len(pts), N * N)
    assert np.all(Lref > 0)
    kw = dict(jitter=False, blur=False, eps=1e-2)
    p_empty = traced_pdf(g, pts, N, **kw)
    f = W.Frame(g, w.scene, eye=EYE, width=160, height=90, vfov=70.0, max_depth=4, rr_depth=2, alpha=0.5,
                l_min=2, c_ray=512, N=16, seed=5, nee=True)
    f.run(60)
    p_trained = traced_pdf(g, pts, N, **kw)
    k_empty, k_trained = kl(Lref, p_empty), kl(Lref, p_trained)
    k_uniform = kl(Lref, np.ones_like(Lref))
    print(f"KL(reference || traced): empty cache {k_empty:.4f}, after 60 frames {k_trained:.4f}, "
          f"uniform {k_uniform:.4f}")
    assert abs(k_empty - k_uniform) < 1e-6
    assert k_trained < 0.2 * k_uniform
