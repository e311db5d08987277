"""Python binding of the wfpg C ABI (include/wfpg.h).

Argument marshalling only: every step of the path runs in libwfpg.so's CUDA
kernels.  Tensors are torch CUDA tensors (float32 data; uint32 data carried
in int32 tensors, bit for bit); work is enqueued on the current torch stream.
There is no CPU fallback: if the library is not built, importing the binding
raises.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np
import torch

from . import build as _build

_lib = None

P = C.c_void_p
U32 = C.c_uint32
U64 = C.c_uint64
I32 = C.c_int
F = C.c_float
SZ = C.c_size_t

WFPG_OK = 0
ERRORS = {-1: "INVALID_ARG", -2: "OOM", -3: "CUDA", -4: "TIMEOUT", -5: "CAPACITY"}
STATUS_TRACE_CAP = 1
STATUS_BIN_CAPACITY = 2
STATUS_RUN_SIZES = 4
STATUS_WAIT_TIMEOUT = 16  # a wait inside the binning's sort ran out (results invalid)
BIN_PARTITION_S = 0
BIN_RUNS = 1
MAX_DEPTH = 11
NONE = 0xFFFFFFFF


class WfpgError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"{ERRORS.get(code, code)}: {msg}")
        self.code = code


class Scene(C.Structure):
    _fields_ = [("quads", P), ("n_quads", U32), ("spheres", P), ("n_spheres", U32),
                ("lo", F * 3), ("size", F), ("tris", P), ("n_tris", U32)]


class SvoInfo(C.Structure):
    _fields_ = [("depth", I32), ("n_nodes", U32), ("n_frags", U32),
                ("level_off", U32 * (MAX_DEPTH + 2)), ("node", P), ("parent", P), ("normal", P),
                ("value", P)]


class BinParams(C.Structure):
    _fields_ = [("mode", I32), ("l_min", I32), ("c_ray", U32), ("n_sizes", U32), ("seed", U64),
                ("frame", U32), ("n_dev", P)]


class GuideParams(C.Structure):
    _fields_ = [("N", I32), ("eps", F), ("jitter", I32), ("blur", I32), ("t_skip", F),
                ("cos_weight", I32), ("seed", U64), ("frame", U32), ("block", I32), ("stage", I32),
                ("split", U32), ("parts", U32)]


FRAME_MAX_DEPTH = 8


class Camera(C.Structure):
    _fields_ = [("eye", F * 3), ("forward", F * 3), ("up", F * 3), ("vfov_deg", F), ("width", U32),
                ("height", U32), ("probe_pos", C.c_void_p), ("probe_n", U32)]


class FrameParams(C.Structure):
    _fields_ = [("max_depth", I32), ("rr_depth", I32), ("alpha", F), ("l_min", I32), ("c_ray", U32),
                ("guide", GuideParams), ("seed", U64), ("update", I32), ("caster", I32), ("proposal", I32),
                ("decay", I32), ("combine", I32), ("nee", I32)]


class FrameStats(C.Structure):
    _fields_ = [("frames", U64), ("paths", U32 * (FRAME_MAX_DEPTH + 1)), ("bins", U32 * (FRAME_MAX_DEPTH + 1)),
                ("records", U32), ("guided_samples", U64), ("status", U32), ("kernels_per_frame", C.c_ulonglong)]


COMBINE = {"constant": 0, "linear": 1, "quadratic": 2, "one-two": 3, "discard-first": 4, "pt-first": 5}
FRAME_BUF = {"vT": 0, "vLe": 1, "vpos": 2, "vwo": 3, "nv": 4, "rec_pos": 5, "rec_wout": 6, "rec_L": 7,
             "rec_src": 8, "q_pos": 9, "q_nrm": 10, "q_u": 11, "q_dir": 12, "q_pdf": 13, "q_path": 14, "vNee": 15,
             "nee_dir": 16, "nee_pl": 17, "nee_pm": 18, "nee_l": 19, "vLw": 20}


def library_path() -> str:
    return _build.LIB


def lib():
    """Load libwfpg.so (built by __graft_entry__.build() / build.py)."""
    global _lib
    if _lib is None:
        path = library_path()
        if not os.path.exists(path):
            raise RuntimeError(f"libwfpg.so is not built ({path}); run __graft_entry__.build()")
        L = C.CDLL(path)
        sig = {
            "svo_build": [P, I32, P, P],
            "svo_destroy": [P],
            "svo_get_info": [P, P],
            "svo_reset_exitance": [P, P],
            "svo_accumulate": [P, P, P, P, U32, P],
            "bin_rays_workspace_size": [P, U32, P, P],
            "bin_rays": [P, P, P, U32, P, P, P, P, P, P, U32, P, P, SZ, P],
            "guide_build_pdf": [P, P, P, P, U32, P, P, P, P, P],
            "guide_sample": [P, P, P, I32, U32, P, P, U32, P, P, P, P],
            "guide_build_sample": [P, P, P, P, P, U32, P, P, P, U32, F, P, P, P, P, SZ, P],
            "guide_build_sample_workspace_size": [I32, U32, U32, P],
            "guide_eval_pdf": [P, I32, U32, P, P, U32, P, P],
            "svo_export": [P, P, P, P, P, P, P, P, P, P],
            "svo_export_exitance": [P, P, P, P, P, P, P],
            "wfpg_svo_status": [P, P, I32, P],
            "frame_create": [P, P, P, P, P, P, P, P],
            "frame_destroy": [P],
            "frame_run": [P, U32, I32, P],
            "frame_set_params": [P, P],
            "frame_get_params": [P, P],
            "frame_reset_image": [P, P],
            "frame_image": [P, P, P, P],
            "frame_stats": [P, P, P],
            "frame_autotune": [P, P, I32, U32, P, P, P],
            "frame_export": [P, I32, P, SZ, P],
            "frame_set_mlp": [P, P, P],
            "guide_sample_mix": [P, P, P, I32, U32, P, P, P, P, U32, P, F, P, P, P],
            "guide_product_sums": [P, I32, U32, P, P, P],
            "guide_product_sample": [P, P, I32, U32, P, P, P, P, U32, P, F, P, P, P, P],
            "guide_product_eval": [P, P, I32, U32, P, P, P, P, U32, F, P, P],
            "wfpg_cast_rays_svo": [P, P, P, P, U32, F, P, P, P, P],
            "bin_rays_static": [P, P, P, U32, P, P, P, P, P, P, U32, P, P],
            "wfpg_stream_read": [P, SZ, I32, P, I32, P],
        }
        for name, args in sig.items():
            fn = getattr(L, name)
            fn.restype = I32
            fn.argtypes = args
        L.wfpg_last_error.restype = C.c_char_p
        L.wfpg_last_error.argtypes = []
        L.wfpg_kernel_launches.restype = C.c_ulonglong
        L.wfpg_kernel_launches.argtypes = []
        _lib = L
    return _lib


def kernel_launches() -> int:
    """Kernels launched by libwfpg.so in this process so far."""
    return int(lib().wfpg_kernel_launches())


def _check(rc):
    if rc != WFPG_OK:
        raise WfpgError(rc, lib().wfpg_last_error().decode())


def _stream(stream=None):
    s = stream if stream is not None else torch.cuda.current_stream()
    return P(s.cuda_stream)


def _ptr(t, dtype=None, n=None, what="tensor"):
    if t is None:
        return None
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise TypeError(f"{what} must be a CUDA tensor")
    if dtype is not None and t.dtype != dtype:
        raise TypeError(f"{what} must be {dtype}, got {t.dtype}")
    if not t.is_contiguous():
        raise ValueError(f"{what} must be contiguous")
    if n is not None and t.numel() < n:
        raise ValueError(f"{what} holds {t.numel()} elements, needs {n}")
    return P(t.data_ptr())


def _np_ptr(a):
    return a.ctypes.data_as(C.c_void_p)


class SVO:
    """Library-owned sparse voxel octree (wfpg_svo handle)."""

    def __init__(self, handle):
        self._h = P(handle)
        info = SvoInfo()
        _check(lib().svo_get_info(self._h, C.byref(info)))
        self.depth = int(info.depth)
        self.n_nodes = int(info.n_nodes)
        self.n_frags = int(info.n_frags)
        self.level_off = np.array(info.level_off[: self.depth + 2], np.uint32)
        self.size = 1.0

    @property
    def handle(self):
        return self._h

    def close(self):
        if self._h:
            lib().svo_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def export(self, stream=None):
        n = self.n_nodes
        nl = int(self.level_off[self.depth + 1] - self.level_off[self.depth])
        out = dict(key=np.zeros(n, np.uint64), first_child=np.zeros(n, np.uint32),
                   child_mask=np.zeros(n, np.uint8), parent=np.zeros(n, np.uint32),
                   normal=np.zeros((n, 3), np.float32), leaf_count=np.zeros(n, np.uint32),
                   frag_off=np.zeros(nl + 1, np.uint32), frag_prim=np.zeros(self.n_frags, np.uint32))
        _check(lib().svo_export(self._h, *[_np_ptr(out[k]) for k in (
            "key", "first_child", "child_mask", "parent", "normal", "leaf_count", "frag_off",
            "frag_prim")], _stream(stream)))
        out["level_off"] = self.level_off.copy()
        return out

    def exitance(self, stream=None):
        n = 2 * self.n_nodes
        out = dict(acc_sum=np.zeros(n, np.uint64), acc_cnt=np.zeros(n, np.uint32),
                   tot_sum=np.zeros(n, np.uint64), tot_cnt=np.zeros(n, np.uint32),
                   value=np.zeros(n, np.float32))
        _check(lib().svo_export_exitance(self._h, *[_np_ptr(out[k]) for k in (
            "acc_sum", "acc_cnt", "tot_sum", "tot_cnt", "value")], _stream(stream)))
        return {k: v.reshape(-1, 2) for k, v in out.items()}

    def status(self, clear=True, stream=None) -> int:
        f = np.zeros(1, np.uint32)
        _check(lib().wfpg_svo_status(self._h, _np_ptr(f), int(clear), _stream(stream)))
        return int(f[0])

    def reset_exitance(self, stream=None):
        _check(lib().svo_reset_exitance(self._h, _stream(stream)))


def _scene_struct(quads, spheres, tris=None, lo=(0.0, 0.0, 0.0), size=1.0):
    sc = Scene()
    sc.quads = _ptr(quads, torch.float32, what="quads") if quads.numel() else None
    sc.n_quads = quads.shape[0] if quads.numel() else 0
    sc.spheres = _ptr(spheres, torch.float32, what="spheres") if spheres.numel() else None
    sc.n_spheres = spheres.shape[0] if spheres.numel() else 0
    if tris is not None and tris.numel():
        sc.tris = _ptr(tris, torch.float32, what="tris")
        sc.n_tris = tris.shape[0]
    for a in range(3):
        sc.lo[a] = float(lo[a])
    sc.size = float(size)
    return sc


def svo_build(quads: torch.Tensor, spheres: torch.Tensor, lo, size: float, depth: int,
              stream=None, tris: torch.Tensor = None) -> SVO:
    """SVO generation (Sec. 3.2).  quads [nq, 8], spheres [ns, 4], tris [nt, 9]
    (optional) float32 CUDA."""
    sc = _scene_struct(quads, spheres, tris, lo, size)
    h = P()
    _check(lib().svo_build(C.byref(sc), int(depth), _stream(stream), C.byref(h)))
    svo = SVO(h.value)
    svo.size = float(size)
    return svo


def svo_accumulate(svo: SVO, pos, wout, L, stream=None):
    """UpdateExitance (Eq. 5, Alg. 1) + bottom-up average."""
    n = L.numel()
    _check(lib().svo_accumulate(svo.handle, _ptr(pos, torch.float32, 3 * n, "pos"),
                                _ptr(wout, torch.float32, 3 * n, "wout"),
                                _ptr(L, torch.float32, n, "L"), n, _stream(stream)))


def bin_rays_workspace_size(svo: SVO, n: int, mode=BIN_PARTITION_S, n_sizes=0) -> int:
    p = BinParams(mode=mode, n_sizes=n_sizes)
    b = SZ()
    _check(lib().bin_rays_workspace_size(svo.handle, n, C.byref(p), C.byref(b)))
    return int(b.value)


def bin_rays(svo: SVO, pos, nrm=None, *, mode=BIN_PARTITION_S, l_min=2, c_ray=0xFFFFFFFF,
             sizes=None, seed=1, frame=0, bin_cap=None, out=None, workspace=None, stream=None):
    """Partition-S (Alg. 2) or run-length bins, plus SelectOrigin.  Returns a
    dict of int32 CUDA tensors (uint32 bit patterns) and the bin-count tensor."""
    n = pos.shape[0]
    dev = pos.device
    n_sizes = 0 if sizes is None else sizes.numel()
    if bin_cap is None:
        bin_cap = n_sizes if mode == BIN_RUNS else max(1, min(n, svo.n_nodes))
    if out is None:
        out = dict(bin_of_ray=torch.empty(n, dtype=torch.int32, device=dev),
                   ray_order=torch.empty(n, dtype=torch.int32, device=dev),
                   bin_offset=torch.empty(bin_cap + 1, dtype=torch.int32, device=dev),
                   origin_ray=torch.empty(bin_cap, dtype=torch.int32, device=dev),
                   n_bins=torch.zeros(1, dtype=torch.int32, device=dev))
    need = bin_rays_workspace_size(svo, n, mode, n_sizes)
    if workspace is None or workspace.numel() < need:
        workspace = torch.empty(need, dtype=torch.uint8, device=dev)
    p = BinParams(mode=mode, l_min=l_min, c_ray=c_ray, n_sizes=n_sizes, seed=seed, frame=frame)
    _check(lib().bin_rays(svo.handle, _ptr(pos, torch.float32, 3 * n, "pos"),
                          _ptr(nrm, torch.float32, 3 * n, "nrm") if nrm is not None else None,
                          n, C.byref(p), _ptr(sizes, torch.int32, what="sizes"),
                          _ptr(out["bin_of_ray"], torch.int32, n), _ptr(out["ray_order"], torch.int32, n),
                          _ptr(out["bin_offset"], torch.int32, bin_cap + 1),
                          _ptr(out["origin_ray"], torch.int32, bin_cap), bin_cap,
                          _ptr(out["n_bins"], torch.int32, 1), _ptr(workspace, torch.uint8),
                          workspace.numel(), _stream(stream)))
    out["bin_cap"] = bin_cap
    return out


def default_t_skip(size: float, depth: int) -> float:
    """2 * sqrt(3) * leaf side: skips the origin's own surface voxels."""
    h = np.float32(size) / np.float32(1 << depth)
    return float(np.float32(np.float32(2.0 * np.sqrt(3.0)) * h))


def guide_build_pdf(svo: SVO, pos, origin_ray=None, n_bins=None, bin_cap=None, *, N=16, eps=1e-2,
                    jitter=False, blur=False, t_skip=None, cos_weight=False, seed=1, frame=0,
                    block=0, stage=0, parts=0, out=None, stream=None):
    """GuideRays field + PDF/CDF (Alg. 3).  Returns (pdf, cdf_row, cdf_marg)."""
    if bin_cap is None:
        bin_cap = origin_ray.numel() if origin_ray is not None else pos.shape[0]
    if t_skip is None:
        t_skip = default_t_skip(svo.size, svo.depth)
    dev = pos.device
    if out is None:
        out = (torch.empty((bin_cap, N * N), dtype=torch.float32, device=dev),
               torch.empty((bin_cap, N * N), dtype=torch.float32, device=dev),
               torch.empty((bin_cap, N), dtype=torch.float32, device=dev))
    pdf, cr, cm = out
    p = GuideParams(N=N, eps=eps, jitter=int(jitter), blur=int(blur), t_skip=t_skip,
                    cos_weight=int(cos_weight), seed=seed, frame=frame, block=block, stage=stage, parts=parts)
    _check(lib().guide_build_pdf(svo.handle, _ptr(pos, torch.float32, what="pos"),
                                 _ptr(origin_ray, torch.int32, what="origin_ray"),
                                 _ptr(n_bins, torch.int32, 1, "n_bins"), bin_cap, C.byref(p),
                                 _ptr(pdf, torch.float32, bin_cap * N * N),
                                 _ptr(cr, torch.float32, bin_cap * N * N),
                                 _ptr(cm, torch.float32, bin_cap * N), _stream(stream)))
    return pdf, cr, cm


def guide_build_sample_workspace_size(N: int, n: int, split: int = 0) -> int:
    b = SZ()
    _check(lib().guide_build_sample_workspace_size(N, n, split, C.byref(b)))
    return int(b.value)


def guide_build_sample(svo: SVO, pos, nrm, bins, u, *, alpha=0.5, N=16, eps=1e-2, jitter=False, blur=False,
                       t_skip=None, cos_weight=False, seed=1, frame=0, block=0, stage=0, split=0, out=None,
                       workspace=None, stream=None):
    """guide_build_pdf + one-sample mixture sampling in one launch (plus a
    GPU-wide launch for bins above `split` rays).  bins is the dict bin_rays
    returns; u holds 3 uniforms per ray.  Returns (dir [n,3], mixture pdf [n])."""
    n = pos.shape[0]
    bin_cap = bins["origin_ray"].numel()
    if t_skip is None:
        t_skip = default_t_skip(svo.size, svo.depth)
    if out is None:
        out = (torch.empty((n, 3), dtype=torch.float32, device=pos.device),
               torch.empty(n, dtype=torch.float32, device=pos.device))
    need = guide_build_sample_workspace_size(N, n, split)
    if workspace is None or workspace.numel() < need:
        workspace = torch.empty(need, dtype=torch.uint8, device=pos.device)
    d, pm = out
    p = GuideParams(N=N, eps=eps, jitter=int(jitter), blur=int(blur), t_skip=t_skip,
                    cos_weight=int(cos_weight), seed=seed, frame=frame, block=block, stage=stage, split=split)
    _check(lib().guide_build_sample(svo.handle, _ptr(pos, torch.float32, 3 * n, "pos"),
                                    _ptr(nrm, torch.float32, 3 * n, "nrm"),
                                    _ptr(bins["origin_ray"], torch.int32, bin_cap),
                                    _ptr(bins["n_bins"], torch.int32, 1), bin_cap,
                                    _ptr(bins["ray_order"], torch.int32, n),
                                    _ptr(bins["bin_offset"], torch.int32, bin_cap + 1),
                                    _ptr(u, torch.float32, 3 * n, "u"), n, alpha, C.byref(p),
                                    _ptr(d, torch.float32, 3 * n), _ptr(pm, torch.float32, n),
                                    _ptr(workspace, torch.uint8), workspace.numel(), _stream(stream)))
    return d, pm


def guide_sample(pdf, cdf_row, cdf_marg, N, bin_of_ray, u, out=None, stream=None):
    """Inverse-CDF sampling (Alg. 3).  Returns (dir [n,3], pdf [n], cell [n] int32)."""
    n = bin_of_ray.numel()
    bin_cap = cdf_marg.numel() // N
    dev = u.device
    if out is None:
        out = (torch.empty((n, 3), dtype=torch.float32, device=dev),
               torch.empty(n, dtype=torch.float32, device=dev),
               torch.empty(n, dtype=torch.int32, device=dev))
    d, p, c = out
    _check(lib().guide_sample(_ptr(pdf, torch.float32), _ptr(cdf_row, torch.float32),
                              _ptr(cdf_marg, torch.float32), N, bin_cap,
                              _ptr(bin_of_ray, torch.int32, n), _ptr(u, torch.float32, 2 * n, "u"), n,
                              _ptr(d, torch.float32, 3 * n), _ptr(p, torch.float32, n),
                              _ptr(c, torch.int32, n), _stream(stream)))
    return d, p, c


def guide_eval_pdf(pdf, N, bins, dirs, out=None, stream=None):
    """PDF of given directions (MIS)."""
    n = bins.numel()
    bin_cap = pdf.numel() // (N * N)
    if out is None:
        out = torch.empty(n, dtype=torch.float32, device=dirs.device)
    _check(lib().guide_eval_pdf(_ptr(pdf, torch.float32), N, bin_cap, _ptr(bins, torch.int32, n),
                                _ptr(dirs, torch.float32, 3 * n), n, _ptr(out, torch.float32, n),
                                _stream(stream)))
    return out


def svo_from_scene(scene, depth: int, device="cuda", stream=None) -> SVO:
    """Upload a procedural scene (paper_2405_06997_gb300.inputs.Scene) and build its SVO."""
    q = torch.as_tensor(np.ascontiguousarray(scene.quads, np.float32).reshape(-1, 8), device=device)
    s = torch.as_tensor(np.ascontiguousarray(scene.spheres, np.float32).reshape(-1, 4), device=device)
    t = torch.as_tensor(np.ascontiguousarray(getattr(scene, "tris", np.zeros((0, 9))), np.float32).reshape(-1, 9),
                        device=device)
    return svo_build(q, s, scene.lo, scene.size, depth, stream=stream, tris=t)


def bin_rays_static(svo: SVO, pos, nrm=None, *, mode=BIN_PARTITION_S, l_min=2, c_ray=0xFFFFFFFF,
                    sizes=None, seed=1, frame=0, bin_cap=None, out=None, stream=None):
    """bin_rays for callers that cannot allocate device memory (for instance a
    host whose device memory is all owned by its own fixed pool, or a caller
    with no device allocator to give bin_rays a workspace from): the same
    outputs, with the scratch taken from the library's fixed static device
    array instead of a workspace.  Raises WfpgError (CAPACITY) when the call
    needs more scratch than that array holds.  Calls whose work overlaps on
    the GPU share the array and must be serialised."""
    fn = lib().bin_rays_static
    n = pos.shape[0]
    dev = pos.device
    n_sizes = 0 if sizes is None else sizes.numel()
    if bin_cap is None:
        bin_cap = n_sizes if mode == BIN_RUNS else max(1, min(n, svo.n_nodes))
    if out is None:
        out = dict(bin_of_ray=torch.empty(n, dtype=torch.int32, device=dev),
                   ray_order=torch.empty(n, dtype=torch.int32, device=dev),
                   bin_offset=torch.empty(bin_cap + 1, dtype=torch.int32, device=dev),
                   origin_ray=torch.empty(bin_cap, dtype=torch.int32, device=dev),
                   n_bins=torch.zeros(1, dtype=torch.int32, device=dev))
    p = BinParams(mode=mode, l_min=l_min, c_ray=c_ray, n_sizes=n_sizes, seed=seed, frame=frame)
    _check(fn(svo.handle, _ptr(pos, torch.float32, 3 * n, "pos"),
              _ptr(nrm, torch.float32, 3 * n, "nrm") if nrm is not None else None, n, C.byref(p),
              _ptr(sizes, torch.int32, what="sizes"), _ptr(out["bin_of_ray"], torch.int32, n),
              _ptr(out["ray_order"], torch.int32, n), _ptr(out["bin_offset"], torch.int32, bin_cap + 1),
              _ptr(out["origin_ray"], torch.int32, bin_cap), bin_cap, _ptr(out["n_bins"], torch.int32, 1),
              _stream(stream)))
    out["bin_cap"] = bin_cap
    return out


# ------------------------------------------------------------------ learned proposal
MLP_PARAMS = 80064
STATUS_MMA_TIMEOUT = 8


class LearnedParams(C.Structure):
    _fields_ = [("lo", F * 3), ("size", F), ("eps", F)]


class AdamParams(C.Structure):
    _fields_ = [("lr", F), ("beta1", F), ("beta2", F), ("eps", F), ("update", I32)]


def _declare_mlp():
    L = lib()
    if getattr(L, "_mlp_declared", False):
        return L
    sig = {
        "mlp_create": [P, U32, P, P],
        "mlp_destroy": [P],
        "mlp_get_params": [P, P, P],
        "mlp_status": [P, P, I32, P],
        "guide_learned_build_pdf": [P, P, P, P, P, U32, P, P, P, P, P],
        "guide_learned_train_step": [P, P, P, U32, P, P, P, P, P, P],
        "guide_learned_logits": [P, P, P, U32, P, P, P],
        "mlp_adam_step": [P, P, P, P],
    }
    for name, args in sig.items():
        fn = getattr(L, name)
        fn.restype = I32
        fn.argtypes = args
    L._mlp_declared = True
    return L


class MLP:
    """The learned proposal's network and optimiser state (wfpg_mlp handle)."""

    def __init__(self, params: np.ndarray | None, max_batch: int, stream=None):
        L = _declare_mlp()
        h = P()
        arr = None if params is None else np.ascontiguousarray(params, np.float32)
        if arr is not None and arr.size != MLP_PARAMS:
            raise ValueError(f"params must hold {MLP_PARAMS} floats")
        _check(L.mlp_create(_np_ptr(arr) if arr is not None else None, max_batch, _stream(stream),
                            C.byref(h)))
        self._h = h
        self.max_batch = max_batch

    @property
    def handle(self):
        return self._h

    def close(self):
        if self._h:
            _declare_mlp().mlp_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def params(self, stream=None) -> np.ndarray:
        out = np.zeros(MLP_PARAMS, np.float32)
        _check(_declare_mlp().mlp_get_params(self._h, _np_ptr(out), _stream(stream)))
        return out

    def status(self, clear=True, stream=None) -> int:
        f = np.zeros(1, np.uint32)
        _check(_declare_mlp().mlp_status(self._h, _np_ptr(f), int(clear), _stream(stream)))
        return int(f[0])


def _learned(lo, size, eps):
    p = LearnedParams()
    for a in range(3):
        p.lo[a] = float(lo[a])
    p.size = float(size)
    p.eps = float(eps)
    return p


def guide_learned_build_pdf(mlp: MLP, pos, nrm, origin_ray=None, n_bins=None, bin_cap=None, *, lo=(0, 0, 0),
                            size=1.0, eps=1e-4, out=None, stream=None):
    """The learned counterpart of guide_build_pdf (N = 32)."""
    if bin_cap is None:
        bin_cap = origin_ray.numel() if origin_ray is not None else pos.shape[0]
    dev = pos.device
    N = 32
    if out is None:
        out = (torch.empty((bin_cap, N * N), dtype=torch.float32, device=dev),
               torch.empty((bin_cap, N * N), dtype=torch.float32, device=dev),
               torch.empty((bin_cap, N), dtype=torch.float32, device=dev))
    pdf, cr, cm = out
    p = _learned(lo, size, eps)
    _check(_declare_mlp().guide_learned_build_pdf(
        mlp.handle, _ptr(pos, torch.float32, what="pos"), _ptr(nrm, torch.float32, what="nrm"),
        _ptr(origin_ray, torch.int32, what="origin_ray"), _ptr(n_bins, torch.int32, 1, "n_bins"), bin_cap,
        C.byref(p), _ptr(pdf, torch.float32, bin_cap * N * N), _ptr(cr, torch.float32, bin_cap * N * N),
        _ptr(cm, torch.float32, bin_cap * N), _stream(stream)))
    return pdf, cr, cm


def guide_learned_train_step(mlp: MLP, pos, nrm, target, *, lo=(0, 0, 0), size=1.0, lr=1e-3, beta1=0.9,
                             beta2=0.999, eps=1e-8, update=True, want_grad=False, loss=None, grad=None,
                             stream=None):
    """One online training step; returns (loss tensor [1], grad tensor or None)."""
    n = pos.shape[0]
    dev = pos.device
    if loss is None:
        loss = torch.zeros(1, dtype=torch.float32, device=dev)
    if want_grad and grad is None:
        grad = torch.zeros(MLP_PARAMS, dtype=torch.float32, device=dev)
    p = _learned(lo, size, 0.0)
    o = AdamParams(lr=lr, beta1=beta1, beta2=beta2, eps=eps, update=int(update))
    _check(_declare_mlp().guide_learned_train_step(
        mlp.handle, _ptr(pos, torch.float32, 3 * n, "pos"), _ptr(nrm, torch.float32, 3 * n, "nrm"), n,
        _ptr(target, torch.float32, n * 1024, "target"), C.byref(p), C.byref(o),
        _ptr(loss, torch.float32, 1), _ptr(grad, torch.float32, MLP_PARAMS) if want_grad else None,
        _stream(stream)))
    return loss, (grad if want_grad else None)


def guide_learned_logits(mlp: MLP, pos, nrm, *, lo=(0, 0, 0), size=1.0, out=None, stream=None):
    """The network's logits [n][1024] for the samples at pos / nrm (float32)."""
    n = pos.shape[0]
    if out is None:
        out = torch.empty((n, 1024), dtype=torch.float32, device=pos.device)
    p = _learned(lo, size, 0.0)
    _check(_declare_mlp().guide_learned_logits(mlp.handle, _ptr(pos, torch.float32, 3 * n, "pos"),
                                               _ptr(nrm, torch.float32, 3 * n, "nrm"), n, C.byref(p),
                                               _ptr(out, torch.float32, n * 1024, "out"), _stream(stream)))
    return out


def mlp_adam_step(mlp: MLP, grad, *, lr=1e-3, beta1=0.9, beta2=0.999, eps=1e-8, stream=None):
    """One Adam step with a caller-supplied gradient (float32 CUDA tensor of MLP_PARAMS)."""
    o = AdamParams(lr=lr, beta1=beta1, beta2=beta2, eps=eps, update=1)
    _check(_declare_mlp().mlp_adam_step(mlp.handle, _ptr(grad, torch.float32, MLP_PARAMS, "grad"), C.byref(o),
                                        _stream(stream)))


def stream_read(buf, reps, sink, blocks, stream=None):
    """Reads the CUDA tensor `buf` `reps` times through L2 only (wfpg_stream_read)."""
    _check(lib().wfpg_stream_read(_ptr(buf), buf.numel() * buf.element_size(), int(reps), _ptr(sink, torch.int32, 1),
                                  int(blocks), _stream(stream)))


def cast_rays(quads, spheres, o, d, tmin=1e-5, with_normal=True, stream=None, tris=None):
    """Closest hits of rays (o + t d) against a scene's quads / spheres /
    triangles (CUDA tensors); returns (t [-1 on miss], prim [int32, -1 on
    miss], nrm or None)."""
    L = lib()
    fn = L.wfpg_cast_rays
    fn.restype = I32
    fn.argtypes = [P, P, P, U32, F, P, P, P, P]
    n = o.shape[0]
    sc = _scene_struct(quads, spheres, tris)
    t = torch.empty(n, dtype=torch.float32, device=o.device)
    prim = torch.empty(n, dtype=torch.int32, device=o.device)
    nrm = torch.empty((n, 3), dtype=torch.float32, device=o.device) if with_normal else None
    _check(fn(C.byref(sc), _ptr(o, torch.float32, 3 * n), _ptr(d, torch.float32, 3 * n), n, float(tmin),
              _ptr(t, torch.float32), _ptr(prim, torch.int32), _ptr(nrm, torch.float32) if with_normal else None,
              _stream(stream)))
    return t, prim, nrm


def cast_rays_svo(svo: SVO, quads, spheres, o, d, tmin=1e-5, with_normal=True, stream=None, tris=None):
    """cast_rays with the scene's SVO as the acceleration structure (the SVO
    must have been built from these quads, spheres and triangles)."""
    n = o.shape[0]
    sc = _scene_struct(quads, spheres, tris)
    t = torch.empty(n, dtype=torch.float32, device=o.device)
    prim = torch.empty(n, dtype=torch.int32, device=o.device)
    nrm = torch.empty((n, 3), dtype=torch.float32, device=o.device) if with_normal else None
    _check(lib().wfpg_cast_rays_svo(svo.handle, C.byref(sc), _ptr(o, torch.float32, 3 * n),
                                    _ptr(d, torch.float32, 3 * n), n, float(tmin), _ptr(t, torch.float32),
                                    _ptr(prim, torch.int32), _ptr(nrm, torch.float32) if with_normal else None,
                                    _stream(stream)))
    return t, prim, nrm


def guide_sample_mix(pdf, cdf_row, cdf_marg, N, bins, nrm, u, *, alpha=0.5, n_bins=None, n_dev=None, out=None,
                     stream=None):
    """One-sample mixture (guided with probability alpha, else cosine) from
    stored tables.  bins: bin_of_ray (int32); u: [n, 3].  Returns (dir, pdf)."""
    n = bins.numel()
    bin_cap = cdf_marg.numel() // N
    if out is None:
        out = (torch.empty((n, 3), dtype=torch.float32, device=u.device),
               torch.empty(n, dtype=torch.float32, device=u.device))
    d, pm = out
    _check(lib().guide_sample_mix(_ptr(pdf, torch.float32), _ptr(cdf_row, torch.float32),
                                  _ptr(cdf_marg, torch.float32), N, bin_cap, _ptr(n_bins, torch.int32, 1, "n_bins"),
                                  _ptr(bins, torch.int32, n), _ptr(nrm, torch.float32, 3 * n, "nrm"),
                                  _ptr(u, torch.float32, 3 * n, "u"), n, _ptr(n_dev, torch.int32, 1, "n_dev"),
                                  alpha, _ptr(d, torch.float32, 3 * n), _ptr(pm, torch.float32, n),
                                  _stream(stream)))
    return d, pm


def guide_product_sums(pdf, N, n_bins=None, out=None, stream=None):
    """Per-bin sums of the field's cell densities over its 8 x 8 blocks (Sec. 3.6)."""
    bin_cap = pdf.numel() // (N * N)
    if out is None:
        out = torch.empty((bin_cap, 64), dtype=torch.float32, device=pdf.device)
    _check(lib().guide_product_sums(_ptr(pdf, torch.float32), N, bin_cap, _ptr(n_bins, torch.int32, 1, "n_bins"),
                                    _ptr(out, torch.float32, bin_cap * 64), _stream(stream)))
    return out


def guide_product_sample(pdf, S, N, bins, nrm, u, *, alpha=1.0, n_bins=None, n_dev=None, out=None, stream=None):
    """Product-guided sampling (Sec. 3.6) mixed with cosine sampling.  bins:
    bin_of_ray; u: [n, 3].  Returns (dir, mixture pdf, cell [-1 for cosine])."""
    n = bins.numel()
    bin_cap = pdf.numel() // (N * N)
    if out is None:
        out = (torch.empty((n, 3), dtype=torch.float32, device=u.device),
               torch.empty(n, dtype=torch.float32, device=u.device),
               torch.empty(n, dtype=torch.int32, device=u.device))
    d, p, c = out
    _check(lib().guide_product_sample(_ptr(pdf, torch.float32), _ptr(S, torch.float32), N, bin_cap,
                                      _ptr(n_bins, torch.int32, 1, "n_bins"), _ptr(bins, torch.int32, n),
                                      _ptr(nrm, torch.float32, 3 * n, "nrm"), _ptr(u, torch.float32, 3 * n, "u"), n,
                                      _ptr(n_dev, torch.int32, 1, "n_dev"), alpha, _ptr(d, torch.float32, 3 * n),
                                      _ptr(p, torch.float32, n), _ptr(c, torch.int32, n), _stream(stream)))
    return d, p, c


def guide_product_eval(pdf, S, N, bins, nrm, dirs, *, alpha=1.0, n_bins=None, out=None, stream=None):
    """Mixture density alpha * product + (1 - alpha) * cosine of given directions."""
    n = bins.numel()
    bin_cap = pdf.numel() // (N * N)
    if out is None:
        out = torch.empty(n, dtype=torch.float32, device=dirs.device)
    _check(lib().guide_product_eval(_ptr(pdf, torch.float32), _ptr(S, torch.float32), N, bin_cap,
                                    _ptr(n_bins, torch.int32, 1, "n_bins"), _ptr(bins, torch.int32, n),
                                    _ptr(nrm, torch.float32, 3 * n, "nrm"), _ptr(dirs, torch.float32, 3 * n), n, alpha,
                                    _ptr(out, torch.float32, n), _stream(stream)))
    return out


class Frame:
    """Batched wavefront frame over an SVO (frame_create .. frame_destroy).

    scene: paper_2405_06997_gb300.inputs.Scene (uploaded here); the SVO must
    outlive the frame.  Camera: eye, unit forward and up, vertical fov,
    width x height; or, with probes (float [n][3] points) and probe_n, one
    image row per probe point whose pixels are the probe_n^2 octahedral cells
    around it (a uniform direction in the cell per frame: the mean image is the
    cell-averaged incident radiance).  All work runs in libwfpg.so; run(use_graph=True)
    replays one captured CUDA graph per frame."""

    def __init__(self, svo: SVO, scene, *, eye, forward=(0.0, 0.0, 1.0), up=(0.0, 1.0, 0.0), vfov=60.0,
                 width=1920, height=1080, max_depth=4, rr_depth=2, alpha=0.5, l_min=2, c_ray=512, N=32,
                 eps=1e-2, jitter=True, blur=True, cos_weight=False, block=0, stage=0, seed=1, update=True,
                 caster=0, proposal=0, decay=False, combine=0, nee=False, probes=None, probe_n=0, device="cuda",
                 stream=None):
        self.svo = svo
        self._q = torch.as_tensor(np.ascontiguousarray(scene.quads, np.float32).reshape(-1, 8), device=device)
        self._s = torch.as_tensor(np.ascontiguousarray(scene.spheres, np.float32).reshape(-1, 4), device=device)
        self._e = torch.as_tensor(np.ascontiguousarray(scene.emission, np.float32), device=device)
        self._a = torch.as_tensor(np.ascontiguousarray(scene.albedo, np.float32), device=device)
        self._t = torch.as_tensor(np.ascontiguousarray(getattr(scene, "tris", np.zeros((0, 9))), np.float32)
                                  .reshape(-1, 9), device=device)
        self._scene = _scene_struct(self._q, self._s, self._t, scene.lo, scene.size)
        self.width, self.height = int(width), int(height)
        self._probes = None
        if probes is not None:  # probe mode: one row of probe_n^2 octahedral cells per point
            self._probes = torch.as_tensor(probes, dtype=torch.float32, device=device).reshape(-1, 3).contiguous()
            self.width, self.height = int(probe_n) ** 2, self._probes.shape[0]
        self.cam = Camera(eye=(F * 3)(*eye), forward=(F * 3)(*forward), up=(F * 3)(*up), vfov_deg=vfov,
                          width=self.width, height=self.height,
                          probe_pos=_ptr(self._probes) if self._probes is not None else None,
                          probe_n=int(probe_n) if probes is not None else 0)
        gp = GuideParams(N=N, eps=eps, jitter=int(jitter), blur=int(blur),
                         t_skip=default_t_skip(svo.size, svo.depth), cos_weight=int(cos_weight), seed=seed,
                         frame=0, block=block, stage=stage)
        self.params = FrameParams(max_depth=max_depth, rr_depth=rr_depth, alpha=alpha, l_min=l_min, c_ray=c_ray,
                                  guide=gp, seed=seed, update=int(update), caster=caster, proposal=proposal,
                                  decay=int(decay), combine=combine, nee=int(nee))
        self.device = device
        h = P()
        _check(lib().frame_create(svo.handle, C.byref(self._scene), _ptr(self._e), _ptr(self._a),
                                  C.byref(self.cam), C.byref(self.params), C.byref(h), _stream(stream)))
        self.handle = h
        self.max_depth_cap = max_depth

    def __del__(self):
        h = getattr(self, "handle", None)
        if h is not None and _lib is not None:
            _lib.frame_destroy(h)
            self.handle = None

    @property
    def pixels(self):
        return self.width * self.height

    def run(self, n_frames=1, use_graph=True, stream=None):
        _check(lib().frame_run(self.handle, n_frames, int(use_graph), _stream(stream)))

    def set_params(self, **kw):
        p = FrameParams()
        _check(lib().frame_get_params(self.handle, C.byref(p)))
        for k, v in kw.items():
            if hasattr(p.guide, k) and k not in ("seed",):
                setattr(p.guide, k, v)
            else:
                setattr(p, k, v)
        _check(lib().frame_set_params(self.handle, C.byref(p)))
        self.params = p

    def set_mlp(self, mlp, lo, size, eps=1e-4):
        """Attach the learned proposal's MLP (the frame keeps a reference)."""
        self._mlp = mlp
        lp = LearnedParams(lo=(F * 3)(*[float(v) for v in lo]), size=float(size), eps=float(eps))
        _check(lib().frame_set_mlp(self.handle, mlp.handle if mlp is not None else None,
                                   C.byref(lp) if mlp is not None else None))

    def get_params(self):
        p = FrameParams()
        _check(lib().frame_get_params(self.handle, C.byref(p)))
        return p

    def reset_image(self, stream=None):
        _check(lib().frame_reset_image(self.handle, _stream(stream)))

    def image(self, stream=None):
        """(mean, variance of one estimate) per pixel, [H, W] float32 tensors."""
        m = torch.empty(self.pixels, dtype=torch.float32, device=self.device)
        v = torch.empty(self.pixels, dtype=torch.float32, device=self.device)
        _check(lib().frame_image(self.handle, _ptr(m), _ptr(v), _stream(stream)))
        return m.view(self.height, self.width), v.view(self.height, self.width)

    def stats(self, stream=None):
        st = FrameStats()
        _check(lib().frame_stats(self.handle, C.byref(st), _stream(stream)))
        d = self.get_params().max_depth
        return {"frames": int(st.frames), "paths": [int(x) for x in st.paths[:d]],
                "bins": [int(x) for x in st.bins[:d]], "records": int(st.records),
                "guided_samples": int(st.guided_samples), "status": int(st.status),
                "kernels_per_frame": int(st.kernels_per_frame)}

    def autotune(self, N_candidates=(16, 32, 64), frames=4, stream=None):
        """Native autotuner: fastest tile per N, then the N with the least
        variance x time.  Returns (chosen params dict, ms per frame)."""
        arr = (I32 * len(N_candidates))(*N_candidates)
        p = FrameParams()
        ms = F()
        _check(lib().frame_autotune(self.handle, arr, len(N_candidates), frames, C.byref(p), C.byref(ms),
                                    _stream(stream)))
        self.params = p
        return {"N": p.guide.N, "block": p.guide.block, "stage": p.guide.stage}, float(ms.value)

    def export(self, what, stream=None):
        """Copy of an internal buffer (see WFPG_FRAME_BUF_* in include/wfpg.h)."""
        P_ = self.pixels
        V = (self.max_depth_cap + 1) * P_
        shapes = {"vT": (V,), "vLe": (V,), "vNee": (V,), "vLw": (V,), "vpos": (V, 3), "vwo": (V, 3), "nv": (P_,), "rec_pos": (V, 3),
                  "rec_wout": (V, 3), "rec_L": (V,), "rec_src": (V,), "q_pos": (P_, 3), "q_nrm": (P_, 3),
                  "q_u": (P_, 3), "q_dir": (P_, 3), "q_pdf": (P_,), "q_path": (P_,), "nee_dir": (P_, 3),
                  "nee_pl": (P_,), "nee_pm": (P_,), "nee_l": (P_,)}
        ints = ("nv", "rec_src", "q_path")
        t = torch.empty(shapes[what], dtype=torch.int32 if what in ints else torch.float32, device=self.device)
        _check(lib().frame_export(self.handle, FRAME_BUF[what], _ptr(t), t.numel() * 4, _stream(stream)))
        return t
