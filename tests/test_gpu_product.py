"""Product path guiding (Sec. 3.6) on the GPU against the oracle: block sums
bit for bit, the chosen cell bit for bit and the density to float32 rounding
given the same random numbers, densities of arbitrary directions, and the
unbiasedness of the mixture with cosine sampling."""
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


def tables(N, seed=3):
    w = inputs.tiny_box(seed, n_rays=4099)
    g = W.svo_from_scene(w.scene, w.depth)
    W.svo_accumulate(g, dev(w.rec_pos), dev(w.rec_wout), dev(w.rec_L))
    pos, nrm = dev(w.ray_pos), dev(w.ray_nrm)
    r = W.bin_rays(g, pos, nrm, l_min=2, seed=2, frame=1)
    pdf, cr, cm = W.guide_build_pdf(g, pos, r["origin_ray"], r["n_bins"], r["bin_cap"], N=N, jitter=True,
                                    blur=True, seed=2, frame=1)
    nb = int(r["n_bins"].item())
    return w, r, pdf, nb


@pytest.mark.parametrize("N", [16, 32, 64, 128])
def test_product_sampling_matches_oracle(N):
    w, r, pdf, nb = tables(N)
    S = W.guide_product_sums(pdf, N, n_bins=r["n_bins"])
    pdf_h = pdf.cpu().numpy()[:nb]
    S_o = oracle.product_block_sums(pdf_h, N)
    assert np.array_equal(S.cpu().numpy()[:nb], S_o)
    n = w.ray_pos.shape[0]
    u3 = inputs.uniforms24(11, (n, 3))
    d, p, c = W.guide_product_sample(pdf, S, N, r["bin_of_ray"], dev(w.ray_nrm), dev(u3), alpha=1.0,
                                     n_bins=r["n_bins"])
    bins = u32(r["bin_of_ray"])
    od, op, oc = oracle.product_sample(pdf_h, S_o, N, bins, w.ray_nrm, u3[:, :2])
    np.testing.assert_array_equal(u32(c), oc)
    np.testing.assert_allclose(p.cpu().numpy(), op, rtol=RTOL, atol=0)
    np.testing.assert_allclose(d.cpu().numpy(), od, rtol=0, atol=1e-6)
    # densities of arbitrary directions
    rng = np.random.default_rng(5)
    v = rng.normal(size=(n, 3))
    v = (v / np.linalg.norm(v, axis=1, keepdims=True)).astype(np.float32)
    e = W.guide_product_eval(pdf, S, N, r["bin_of_ray"], dev(w.ray_nrm), dev(v), alpha=1.0, n_bins=r["n_bins"])
    np.testing.assert_allclose(e.cpu().numpy(), oracle.product_eval(pdf_h, S_o, N, bins, w.ray_nrm, v), rtol=RTOL,
                               atol=0)


def test_product_mixture_is_unbiased_and_consistent():
    N = 32
    w, r, pdf, nb = tables(N, seed=4)
    S = W.guide_product_sums(pdf, N, n_bins=r["n_bins"])
    reps = 64
    n = w.ray_pos.shape[0]
    bins = r["bin_of_ray"].repeat(reps).contiguous()
    nrm = dev(np.tile(w.ray_nrm, (reps, 1)))
    u = dev(inputs.uniforms24(21, (n * reps, 3)))
    d, p, c = W.guide_product_sample(pdf, S, N, bins, nrm, u, alpha=0.5, n_bins=r["n_bins"])
    assert torch.all(p > 0)
    x = (1.0 / p.double()).cpu().numpy()
    y = (torch.clamp((d * nrm).sum(dim=1), min=0).double() / p.double()).cpu().numpy()
    for v, ref in ((x, 4 * np.pi), (y, np.pi)):
        se = v.std(ddof=1) / np.sqrt(len(v))
        assert abs(v.mean() - ref) < 4 * se, (v.mean(), ref, se)
    # the returned density is the mixture density of the returned direction
    e = W.guide_product_eval(pdf, S, N, bins, nrm, d, alpha=0.5, n_bins=r["n_bins"])
    cells_agree = (u32(c) == np.uint32(0xFFFFFFFF)) | (u32(c) == oracle_cells(d.cpu().numpy(), N))
    np.testing.assert_array_equal(e.cpu().numpy()[cells_agree], p.cpu().numpy()[cells_agree])
    assert cells_agree.mean() > 0.999


def oracle_cells(d, N):
    uv = oracle.octa_encode(d)
    i = np.clip(((uv[:, 0] + 1) * (N / 2)).astype(np.int64), 0, N - 1)
    j = np.clip(((uv[:, 1] + 1) * (N / 2)).astype(np.int64), 0, N - 1)
    return (j * N + i).astype(np.uint32)


def test_product_rejects_bad_arguments():
    N = 16
    w, r, pdf, nb = tables(N)
    S = W.guide_product_sums(pdf, N)
    with pytest.raises(W.WfpgError):
        W.guide_product_sample(pdf, S, 12, r["bin_of_ray"], dev(w.ray_nrm), torch.zeros((4099, 3), device="cuda"))
    with pytest.raises(W.WfpgError):
        W.guide_product_sample(pdf, S, N, r["bin_of_ray"], dev(w.ray_nrm), torch.zeros((4099, 3), device="cuda"),
                               alpha=2.0)
