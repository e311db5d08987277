"""The learned proposal in use (a project addition; the paper has no
counterpart): online training on the SVO-traced fields of Alg. 3, held-out KL,
the fallback rule, and an equal-samples variance comparison of guided path
estimates.

Everything on the hot path runs in libwfpg.so (guide_build_pdf,
guide_learned_build_pdf, guide_learned_train_step, guide_sample,
guide_eval_pdf, wfpg_cast_rays); this module only schedules the calls and
accumulates the estimates.
"""
from __future__ import annotations

import math
import time

import numpy as np
import torch

from . import inputs
from . import wfpg as W


def _dev(a, device):
    return torch.from_numpy(np.ascontiguousarray(a)).to(device)


class OnlineTrainer:
    """Trains the MLP on batches of surface points whose targets are traced
    through the SVO on the fly (guide_build_pdf, N = 32, jitter + blur).

    The points come from `points` = (pos, nrm) when given -- e.g. the frame's
    own guided path vertices, the places whose traced grids the method
    generates -- else area-uniformly from the scene's surfaces.  `heldout`
    points are kept out of training: the last ones of `points`, or a separate
    area-uniform draw."""

    def __init__(self, svo, scene, *, batch=65536, pool=1 << 20, lr=1e-3, seed=1, device="cuda",
                 params=None, heldout=4096, points=None):
        self.svo = svo
        self.scene = scene
        self.batch = batch
        self.lr = lr
        self.seed = seed
        if points is not None:
            pos, nrm = (torch.as_tensor(np.asarray(x) if not isinstance(x, torch.Tensor) else x) for x in points)
            pos, nrm = pos.to(device).float(), nrm.to(device).float()
            perm = torch.from_numpy(np.random.default_rng(seed).permutation(pos.shape[0])).to(device)
            pos, nrm = pos[perm], nrm[perm]
            self.hpos, self.hnrm = pos[-heldout:].contiguous(), nrm[-heldout:].contiguous()
            self.pos, self.nrm = pos[:-heldout].contiguous(), nrm[:-heldout].contiguous()
        else:
            rng = np.random.default_rng(seed)
            ppos, pnrm, _ = inputs.surface_points(scene, rng, pool)
            self.pos = _dev(ppos, device)
            self.nrm = _dev(pnrm, device)
            hrng = np.random.default_rng(seed + 7919)
            hp, hn, _ = inputs.surface_points(scene, hrng, heldout)
            self.hpos = _dev(hp, device)
            self.hnrm = _dev(hn, device)
        heldout = self.hpos.shape[0]
        self.batch = batch = min(batch, self.pos.shape[0])
        self.mlp = W.MLP(params if params is not None else inputs.mlp_init(seed), max_batch=max(batch, heldout, 65536))
        self.tgt = (torch.empty((batch, 1024), dtype=torch.float32, device=device),
                    torch.empty((batch, 1024), dtype=torch.float32, device=device),
                    torch.empty((batch, 32), dtype=torch.float32, device=device))
        self.htgt = (torch.empty((heldout, 1024), dtype=torch.float32, device=device),
                     torch.empty((heldout, 1024), dtype=torch.float32, device=device),
                     torch.empty((heldout, 32), dtype=torch.float32, device=device))
        self.loss = torch.zeros(1, dtype=torch.float32, device=device)
        self.lo = tuple(float(v) for v in scene.lo)
        self.size = float(scene.size)
        self.steps = 0
        self._htraced = False

    def _targets(self, pos, out, frame):
        return W.guide_build_pdf(self.svo, pos, None, None, pos.shape[0], N=32, jitter=True, blur=True,
                                 seed=self.seed, frame=frame, out=out)

    def step(self):
        n = self.pos.shape[0]
        k = self.steps
        start = (k * self.batch) % n
        if start + self.batch > n:
            start = 0
        pos = self.pos[start:start + self.batch]
        nrm = self.nrm[start:start + self.batch]
        pdf = self._targets(pos, self.tgt, 1 + k)[0]
        W.guide_learned_train_step(self.mlp, pos, nrm, pdf, lo=self.lo, size=self.size, lr=self.lr,
                                   loss=self.loss)
        self.steps += 1
        return self.loss

    def train(self, steps):
        for _ in range(steps):
            self.step()
        torch.cuda.synchronize()
        return float(self.loss.item())

    def heldout_kl(self):
        """Mean KL(traced || learned) on held-out surface points (no update)."""
        if not self._htraced:
            self._targets(self.hpos, self.htgt, 0)
            self._htraced = True
        loss, _ = W.guide_learned_train_step(self.mlp, self.hpos, self.hnrm, self.htgt[0], lo=self.lo,
                                             size=self.size, update=False)
        return float(loss.item())


def use_learned(heldout_kl: float, tau: float) -> bool:
    """Fallback rule: the learned proposal replaces the traced one only while its
    held-out KL against the traced fields stays below tau."""
    return math.isfinite(heldout_kl) and heldout_kl < tau


def traced_frame_kl(trainer: "OnlineTrainer") -> float:
    """The traced method's own frame-to-frame variation on the held-out points:
    mean KL between their fields traced at two frames (different jitter).  A
    learned proposal within a small factor of this is as close to a fresh
    traced field as another traced field is; it sets the fallback threshold."""
    a = W.guide_build_pdf(trainer.svo, trainer.hpos, None, None, trainer.hpos.shape[0], N=32, jitter=True,
                          blur=True, seed=trainer.seed, frame=1 << 20)[0]
    b = W.guide_build_pdf(trainer.svo, trainer.hpos, None, None, trainer.hpos.shape[0], N=32, jitter=True,
                          blur=True, seed=trainer.seed, frame=(1 << 20) + 1)[0]
    qa = a / a.sum(dim=1, keepdim=True)
    qb = b / b.sum(dim=1, keepdim=True)
    return float((qa * (qa.log() - qb.log())).sum(dim=1).mean().item())


def _cosine_dirs(nrm, u):
    """Cosine-distributed directions about unit normals (u: [n, 2] uniforms)."""
    n = nrm
    helper = torch.where((n[:, 0].abs() > 0.9).unsqueeze(1),
                         torch.tensor([0.0, 1.0, 0.0], device=n.device).expand_as(n),
                         torch.tensor([1.0, 0.0, 0.0], device=n.device).expand_as(n))
    t = torch.linalg.cross(helper, n)
    t = t / t.norm(dim=1, keepdim=True)
    b = torch.linalg.cross(n, t)
    r = torch.sqrt(u[:, 0])
    phi = 2 * math.pi * u[:, 1]
    z = torch.sqrt(torch.clamp(1 - u[:, 0], min=0))
    return t * (r * torch.cos(phi)).unsqueeze(1) + b * (r * torch.sin(phi)).unsqueeze(1) + n * z.unsqueeze(1)


def guided_estimates(w, svo, proposal, *, frames=16, alpha=0.5, mlp=None, seed=1, device="cuda", l_min=4,
                     c_ray=512, bin_cap=16384):
    """Per-pixel estimates of the light leaving each primary hit toward the
    camera, one path per pixel per frame, two bounces deep: the first bounce
    direction w1 is drawn from alpha * guided + (1 - alpha) * cosine and
    weighted by that mixture density (so the estimator stays unbiased); the
    second bounce is cosine-sampled.
        L = (albedo1 / pi) cos1 / p(w1) * (Le(x2) + albedo2 * Le(x3))
    proposal: 'svo' (traced field), 'svo_product' (traced field times the BSDF at
    8 x 8 blocks, Sec. 3.6), 'learned' (MLP) or 'bsdf' (cosine only).
    Rays are binned with Partition-S (l_min, c_ray; the paper's Table 1 uses
    c_ray = 512 and its l_min 5, i.e. 4 here).  Returns the per-pixel mean and
    variance over frames and the guiding time per frame (binning + field/PDF +
    sampling + MIS density), in seconds.  A cheap proposal can afford finer
    bins (smaller c_ray, more bins: bin_cap) than tracing."""
    q = _dev(w.scene.quads, device)
    sp = _dev(w.scene.spheres, device)
    emission = _dev(w.scene.emission, device)
    albedo_all = _dev(w.scene.albedo, device)
    albedo = _dev(w.scene.albedo[w.extra["ray_prim"]], device)
    pos = _dev(w.ray_pos, device)
    nrm = _dev(w.ray_nrm, device)
    R = pos.shape[0]
    B = bin_cap  # Partition-S at c_ray = 512 gives a few thousand bins at 1080p
    s1 = torch.zeros(R, dtype=torch.float64, device=device)
    s2 = torch.zeros(R, dtype=torch.float64, device=device)
    guide = None
    times = []
    a = alpha if proposal != "bsdf" else 0.0
    for f in range(frames):
        u = _dev(inputs.uniforms24(seed * 7919 + f, (R, 7)), device)
        dc = _cosine_dirs(nrm, u[:, 2:4])
        t_guide = 0.0
        if a > 0:
            e = [torch.cuda.Event(enable_timing=True) for _ in range(4)]
            e[0].record()
            r = W.bin_rays(svo, pos, l_min=l_min, c_ray=c_ray, seed=seed, frame=f, bin_cap=B)
            if proposal in ("svo", "svo_product"):
                guide = W.guide_build_pdf(svo, pos, r["origin_ray"], r["n_bins"], B, N=32, jitter=True, blur=True,
                                          seed=seed, frame=f, out=guide)
            else:
                guide = W.guide_learned_build_pdf(mlp, pos, nrm, r["origin_ray"], r["n_bins"], B, lo=w.scene.lo,
                                                  size=w.scene.size, out=guide)
            if proposal == "svo_product":
                # Sec. 3.6: the field times the ray's BSDF at 8 x 8 blocks; the call
                # returns the mixture (alpha product, 1 - alpha cosine) and its density
                S = W.guide_product_sums(guide[0], 32, n_bins=r["n_bins"])
                uu = torch.stack([u[:, 0], u[:, 1], u[:, 4]], dim=1).contiguous()
                d, pmix, _ = W.guide_product_sample(guide[0], S, 32, r["bin_of_ray"], nrm, uu, alpha=a,
                                                    n_bins=r["n_bins"])
                e[1].record()
                e[2].record()
                e[3].record()
                e[3].synchronize()
                t_guide = e[0].elapsed_time(e[3]) / 1e3
            else:
                dg, _, _ = W.guide_sample(*guide, 32, r["bin_of_ray"], u[:, 0:2].contiguous())
                e[1].record()
                d = torch.where((u[:, 4] < a).unsqueeze(1), dg, dc).contiguous()
                e[2].record()
                pg = W.guide_eval_pdf(guide[0], 32, r["bin_of_ray"], d)
                e[3].record()
                e[3].synchronize()
                t_guide = (e[0].elapsed_time(e[1]) + e[2].elapsed_time(e[3])) / 1e3
        else:
            d = dc.contiguous()
        cos = torch.clamp((d * nrm).sum(dim=1), min=0.0)
        if proposal == "svo_product":
            p = pmix
        else:
            p = (1 - a) * cos / math.pi
            if a > 0:
                p = p + a * pg
        t1, prim1, n2 = W.cast_rays(q, sp, (pos + 1e-4 * nrm).contiguous(), d)
        hit1 = prim1 >= 0
        pi1 = prim1.clamp(min=0).long()
        le1 = torch.where(hit1, emission[pi1], torch.zeros_like(t1))
        x2 = pos + t1.clamp(min=0).unsqueeze(1) * d
        d2 = _cosine_dirs(n2, u[:, 5:7]).contiguous()
        _, prim2, _ = W.cast_rays(q, sp, (x2 + 1e-4 * n2).contiguous(), d2, with_normal=False)
        le2 = torch.where(prim2 >= 0, emission[prim2.clamp(min=0).long()], torch.zeros_like(t1))
        li = le1 + torch.where(hit1 & (le1 == 0), albedo_all[pi1] * le2, torch.zeros_like(le2))
        est = torch.where(p > 0, albedo / math.pi * li * cos / p, torch.zeros_like(p)).double()
        s1 += est
        s2 += est * est
        times.append(t_guide)
    mean = s1 / frames
    var = (s2 - s1 * s1 / frames) / (frames - 1)
    return mean, var, float(np.mean(times[1:] if len(times) > 1 else times))


def compare_proposals(w, svo, mlp, *, frames=16, alpha=0.5, seed=1, fine_c_ray=32, fine_bin_cap=65536):
    """Equal-samples comparison of the traced and learned proposals (and the
    cosine-only baseline): mean per-pixel variance, mean estimate, proposal
    time per frame and guided samples/s.  'learned_fine' evaluates the MLP on
    Partition-S bins of fine_c_ray rays (the MLP's cost per bin is a few
    hundred kFLOP, a traced field's is N^2 cone rays)."""
    out = {}
    runs = (("bsdf", "bsdf", {}), ("svo", "svo", {}), ("svo_product", "svo_product", {}), ("learned", "learned", {}),
            ("learned_fine", "learned", {"c_ray": fine_c_ray, "bin_cap": fine_bin_cap}))
    for name, proposal, kw in runs:
        m, v, t = guided_estimates(w, svo, proposal, frames=frames, alpha=alpha, mlp=mlp, seed=seed, **kw)
        out[name] = {"mean": float(m.mean().item()), "variance": float(v.mean().item()),
                     "guiding_seconds_per_frame": t, "guided_samples_per_s": len(w.ray_pos) / t if t > 0 else None}
    out["learned_fine"]["c_ray"] = fine_c_ray
    for name in ("svo_product", "learned", "learned_fine"):
        out[f"variance_ratio_{name}_over_svo"] = out[name]["variance"] / out["svo"]["variance"]
        # work-normalised: (variance x guiding time) of the traced over the learned proposal
        out[f"efficiency_ratio_{name}_over_svo"] = (
            (out["svo"]["variance"] * out["svo"]["guiding_seconds_per_frame"]) /
            (out[name]["variance"] * out[name]["guiding_seconds_per_frame"]))
    return out
