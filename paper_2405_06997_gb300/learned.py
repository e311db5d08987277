"""The learned proposal in use (a project addition; the paper has no
counterpart): online training on the SVO-traced fields of Alg. 3, held-out KL,
the fallback rule, and an equal-samples variance comparison of guided path
estimates.

Everything on the hot path runs in libwfpg.so (guide_build_pdf,
guide_learned_build_pdf, guide_learned_train_step, frame_run and its
sampling, mixture density and shading kernels); this module only schedules
the calls and reads back their results.
"""
from __future__ import annotations

import math

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


def run_batches(frame, batches, frames):
    """Runs `batches` groups of `frames` frames on a batched frame (update off
    for an unchanging cache) and returns, per group, the mean over pixels of
    the per-pixel variance of one frame's estimate (frame_image), with the
    guided samples and the GPU time of all groups (frame_stats, CUDA events)."""
    var, ms, guided = [], 0.0, 0
    for _ in range(batches):
        frame.reset_image()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        frame.run(frames)
        e1.record()
        e1.synchronize()
        ms += e0.elapsed_time(e1)
        guided += frame.stats()["guided_samples"]
        var.append(float(frame.image()[1].double().mean().item()))
    return {"batch_variance": var, "variance": float(np.mean(var)), "ms_per_frame": ms / (batches * frames),
            "guided_samples": guided, "guided_samples_per_s": guided / (ms / 1e3) if ms > 0 else None}


def variance_ratio(a, b):
    """Mean and standard error over batches of the ratio a / b of two runs'
    batch variances (batch i of both runs draws the same frame indices)."""
    r = np.asarray(a["batch_variance"]) / np.asarray(b["batch_variance"])
    return float(r.mean()), float(r.std(ddof=1) / np.sqrt(len(r))) if len(r) > 1 else float("inf")


def compare_proposals(svo, scene, mlp, camera, *, batches=8, frames=16, alpha=0.5, seed=1, traced_bins=None,
                      learned_bins=None, with_product=True, with_bsdf=True):
    """Equal-samples comparison of the guided proposals on the batched frame
    (libwfpg.so's frame_run: binning, guided or learned tables, the one-sample
    mixture with cosine sampling and its exact density, shading, per-pixel
    variance; nothing here but scheduling).  camera: Frame keyword arguments
    (eye, forward, up, vfov, width, height, max_depth, ...).  traced_bins /
    learned_bins: Partition-S (l_min, c_ray) of each proposal; the MLP costs a
    few hundred kFLOP per bin against N^2 cone rays for a traced field, so it
    can afford finer bins.  Returns per-proposal variance, ms per frame and
    guided samples/s, and the variance ratios over the traced field with their
    standard errors."""
    traced_bins = traced_bins or {"l_min": 4, "c_ray": 512}
    learned_bins = learned_bins or {"l_min": 4, "c_ray": 32}
    base = dict(camera, alpha=alpha, seed=seed, update=False)
    runs = [("svo", dict(base, proposal=0, N=32, **traced_bins), False),
            ("learned", dict(base, proposal=1, N=32, **learned_bins), True)]
    if with_product:
        runs.append(("svo_product", dict(base, proposal=2, N=32, **traced_bins), False))
    if with_bsdf:
        runs.append(("bsdf", dict(base, proposal=0, N=32, **dict(traced_bins, alpha=0.0)), False))
    out = {}
    for name, kw, uses_mlp in runs:
        f = W.Frame(svo, scene, **kw)
        if uses_mlp:
            f.set_mlp(mlp, scene.lo, scene.size)
        f.run(2)  # warm-up (capture of the frame's graph)
        out[name] = run_batches(f, batches, frames)
        out[name]["bins"] = {k: kw[k] for k in ("l_min", "c_ray")}
        del f
    for name in list(out):
        if name != "svo":
            m, se = variance_ratio(out[name], out["svo"])
            out[f"variance_ratio_{name}_over_svo"] = m
            out[f"variance_ratio_{name}_over_svo_se"] = se
    return out
