"""CPU ORACLE -- TEST INFRASTRUCTURE ONLY.

ctypes wrapper around the plain C++ oracle of the wavefront path-guiding hot
path (oracle/*.cpp).  Only the tests, ``__graft_entry__.smoke()`` and the
benchmark's CPU-baseline leg import this package; the CUDA library never
does.  The library is compiled on first use (g++, -O2 -ffp-contract=off) into
oracle/_build/.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRCS = ["svo.cpp", "octa_trace.cpp", "bins.cpp", "guide.cpp", "api.cpp", "learned.cpp", "product.cpp"]
_HDRS = ["oracle.h", "oracle_internal.h"]
_OUT = os.path.join(_HERE, "_build", "liboracle.so")
_lock = threading.Lock()
_lib = None

CXXFLAGS = ["-O2", "-std=c++17", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared"]


def build(force: bool = False) -> str:
    """Compile the oracle if its sources are newer than the library."""
    srcs = [os.path.join(_HERE, s) for s in _SRCS]
    deps = srcs + [os.path.join(_HERE, h) for h in _HDRS]
    if not force and os.path.exists(_OUT):
        t = os.path.getmtime(_OUT)
        if all(os.path.getmtime(d) <= t for d in deps):
            return _OUT
    os.makedirs(os.path.dirname(_OUT), exist_ok=True)
    tmp = _OUT + f".{os.getpid()}.tmp"
    cmd = ["g++", *CXXFLAGS, "-o", tmp, *srcs]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _OUT)
    return _OUT


def lib():
    global _lib
    with _lock:
        if _lib is None:
            _lib = C.CDLL(build())
            _declare(_lib)
    return _lib


P = C.c_void_p
F = C.c_float
U32 = C.c_uint32
U64 = C.c_uint64
I32 = C.c_int
SZ = C.c_size_t


def _declare(L):
    sig = {
        "orc_svo_build": (P, [P, I32, P, I32, P, I32, P, F, I32]),
        "orc_svo_free": (None, [P]),
        "orc_svo_num_nodes": (U32, [P]),
        "orc_svo_level_off": (None, [P, P]),
        "orc_svo_export": (None, [P, P, P, P, P, P, P]),
        "orc_svo_num_frags": (U32, [P]),
        "orc_svo_export_frags": (None, [P, P, P]),
        "orc_svo_deepest": (U32, [P, P]),
        "orc_svo_accumulate": (None, [P, P, P, P, SZ]),
        "orc_svo_export_exitance": (None, [P, P, P, P, P, P]),
        "orc_bin_rays": (C.c_int64, [P, P, P, SZ, I32, I32, U32, P, U32, U64, U32, P, P, P, P,
                                     U32]),
        "orc_guide_build": (None, [P, P, P, U32, I32, F, I32, I32, F, I32, U64, U32, P, P, P, P,
                                   P, P]),
        "orc_guide_sample": (None, [P, P, P, I32, P, P, SZ, P, P, P]),
        "orc_guide_eval_pdf": (None, [P, I32, P, P, SZ, P]),
        "orc_morton": (U64, [U32, U32, U32]),
        "orc_rng_u64": (U64, [U64, U64, U64]),
        "orc_sin": (F, [F]),
        "orc_cos": (F, [F]),
        "orc_atan01": (F, [F]),
        "orc_octa_decode": (None, [P, SZ, P]),
        "orc_octa_encode": (None, [P, SZ, P]),
        "orc_kmeans2": (None, [P, P, I32, P]),
        "orc_warp_scan": (None, [P, I32]),
        "orc_blur": (None, [P, I32]),
        "orc_pdf_cdf": (None, [P, I32, P, P, P]),
        "orc_trace": (None, [P, P, P, SZ, F, F, I32, P, P, P, P, P, P, P, P, P]),
        "orc_mlp_num_params": (SZ, []),
        "orc_bf16_round": (None, [P, SZ, P]),
        "orc_product_block_sums": (None, [P, I32, SZ, P]),
        "orc_product_sample": (None, [P, P, I32, P, P, P, SZ, P, P, P]),
        "orc_product_eval": (None, [P, P, I32, P, P, P, SZ, P]),
        "orc_product_block_weight": (F, [P, I32]),
        "orc_mlp_features": (None, [P, P, SZ, P, F, P]),
        "orc_mlp_forward": (None, [P, P, P, SZ, P, F, I32, P, P]),
        "orc_mlp_grad": (C.c_double, [P, P, P, SZ, P, F, P, I32, P]),
        "orc_mlp_grad_trace": (C.c_double, [P, P, P, SZ, P, F, P, I32, P] + [P] * 9),
        "orc_adam": (None, [P, P, P, P, SZ, I32, C.c_double, C.c_double, C.c_double, C.c_double]),
    }
    for name, (res, args) in sig.items():
        fn = getattr(L, name)
        fn.restype = res
        fn.argtypes = args


def _p(a):
    return None if a is None else a.ctypes.data_as(C.c_void_p)


def _c(a, dt):
    return np.ascontiguousarray(a, dtype=dt)


FOUR_PI_F32 = np.float32(12.566370614359172)


class SVO:
    """The oracle's SVO for one scene (Sec. 3.2)."""

    def __init__(self, scene, depth: int):
        self.D = int(depth)
        self._q = _c(scene.quads, np.float32).reshape(-1, 8)
        self._s = _c(scene.spheres, np.float32).reshape(-1, 4)
        tris = getattr(scene, "tris", None)
        self._t = _c(np.zeros((0, 9), np.float32) if tris is None else tris, np.float32).reshape(-1, 9)
        self.lo = _c(scene.lo, np.float32)
        self.S = float(scene.size)
        h = lib().orc_svo_build(_p(self._q), len(self._q), _p(self._s), len(self._s), _p(self._t), len(self._t),
                                _p(self.lo), self.S, self.D)
        if not h:
            raise ValueError("scene occupies no voxel")
        self._h = h
        self.n_nodes = int(lib().orc_svo_num_nodes(h))
        lo_ = np.zeros(self.D + 2, np.uint32)
        lib().orc_svo_level_off(h, _p(lo_))
        self.level_off = lo_

    def __del__(self):
        h = getattr(self, "_h", None)
        if h:
            lib().orc_svo_free(h)
            self._h = None

    @property
    def handle(self):
        return self._h

    def export(self):
        n = self.n_nodes
        key = np.zeros(n, np.uint64)
        fc = np.zeros(n, np.uint32)
        mask = np.zeros(n, np.uint8)
        par = np.zeros(n, np.uint32)
        nrm = np.zeros((n, 3), np.float32)
        lc = np.zeros(n, np.uint32)
        lib().orc_svo_export(self._h, _p(key), _p(fc), _p(mask), _p(par), _p(nrm), _p(lc))
        return dict(key=key, first_child=fc, child_mask=mask, parent=par, normal=nrm,
                    leaf_count=lc, level_off=self.level_off.copy())

    def frags(self):
        nl = int(self.level_off[self.D + 1] - self.level_off[self.D])
        nf = int(lib().orc_svo_num_frags(self._h))
        off = np.zeros(nl + 1, np.uint32)
        prim = np.zeros(nf, np.uint32)
        lib().orc_svo_export_frags(self._h, _p(off), _p(prim))
        return off, prim

    def deepest(self, p):
        p = _c(p, np.float32)
        return int(lib().orc_svo_deepest(self._h, _p(p)))

    def accumulate(self, pos, wout, L):
        pos, wout, L = _c(pos, np.float32), _c(wout, np.float32), _c(L, np.float32)
        lib().orc_svo_accumulate(self._h, _p(pos), _p(wout), _p(L), len(L))

    def exitance(self):
        n = 2 * self.n_nodes
        a_s = np.zeros(n, np.uint64)
        a_c = np.zeros(n, np.uint32)
        t_s = np.zeros(n, np.uint64)
        t_c = np.zeros(n, np.uint32)
        v = np.zeros(n, np.float32)
        lib().orc_svo_export_exitance(self._h, _p(a_s), _p(a_c), _p(t_s), _p(t_c), _p(v))
        r = lambda a: a.reshape(-1, 2)
        return dict(acc_sum=r(a_s), acc_cnt=r(a_c), tot_sum=r(t_s), tot_cnt=r(t_c), value=r(v))

    def bin_rays(self, pos, nrm, mode=0, l_min=2, c_ray=0xFFFFFFFF, sizes=None, seed=1, frame=0,
                 bin_cap=None):
        pos, nrm = _c(pos, np.float32), _c(nrm, np.float32)
        n = len(pos)
        sizes_a = _c(sizes if sizes is not None else np.zeros(0), np.uint32)
        cap = bin_cap if bin_cap is not None else max(n, len(sizes_a), 1)
        b = np.zeros(n, np.uint32)
        o = np.zeros(n, np.uint32)
        off = np.zeros(cap + 1, np.uint32)
        org = np.zeros(cap, np.uint32)
        nb = lib().orc_bin_rays(self._h, _p(pos), _p(nrm), n, mode, l_min, c_ray, _p(sizes_a),
                                len(sizes_a), seed, frame, _p(b), _p(o), _p(off), _p(org), cap)
        if nb < 0:
            raise ValueError(f"orc_bin_rays failed ({nb})")
        return dict(n_bins=int(nb), bin_of_ray=b, ray_order=o, bin_offset=off[: nb + 1],
                    origin_ray=org[:nb])

    def guide_build(self, origins, bin_ids, N, eps=1e-2, jitter=False, blur=False, t_skip=None,
                    cos_weight=False, seed=1, frame=0, count_steps=False, count_blocks=False):
        origins = _c(origins, np.float32).reshape(-1, 3)
        bin_ids = _c(bin_ids, np.uint32)
        nb = len(origins)
        if t_skip is None:
            t_skip = default_t_skip(self.S, self.D)
        NN = N * N
        field = np.zeros((nb, NN), np.float32)
        pdf = np.zeros((nb, NN), np.float32)
        cr = np.zeros((nb, NN), np.float32)
        cm = np.zeros((nb, N), np.float32)
        steps = np.zeros(1, np.uint64)
        blocks = np.zeros(1, np.uint64)
        lib().orc_guide_build(self._h, _p(origins), _p(bin_ids), nb, N, float(eps), int(jitter),
                              int(blur), float(t_skip), int(cos_weight), seed, frame, _p(field),
                              _p(pdf), _p(cr), _p(cm), _p(steps),
                              _p(blocks) if count_blocks else None)
        out = dict(field=field, pdf=pdf, cdf_row=cr, cdf_marg=cm)
        if count_steps:
            out["steps"] = int(steps[0])
        if count_blocks:
            out["blocks"] = int(blocks[0])
        return out

    def trace(self, o, d, N=None, omega=None, t_skip=None, cos_weight=False):
        o = _c(o, np.float32).reshape(-1, 3)
        d = _c(d, np.float32).reshape(-1, 3)
        n = len(o)
        if omega is None:
            omega = np.float32(FOUR_PI_F32 / np.float32(N * N))
        if t_skip is None:
            t_skip = default_t_skip(self.S, self.D)
        out = dict(hit=np.zeros(n, np.int32), leaf_key=np.zeros(n, np.uint64),
                   t_entry=np.zeros(n, np.float32), level=np.zeros(n, np.int32),
                   node=np.zeros(n, np.uint32), side=np.zeros(n, np.int32),
                   value=np.zeros(n, np.float32), steps=np.zeros(n, np.uint32),
                   blocks=np.zeros(n, np.uint32))
        lib().orc_trace(self._h, _p(o), _p(d), n, float(t_skip), float(omega), int(cos_weight),
                        *[_p(out[k]) for k in ("hit", "leaf_key", "t_entry", "level", "node",
                                               "side", "value", "steps", "blocks")])
        return out


def default_t_skip(S: float, D: int) -> float:
    """t_skip = 2 * sqrt(3) * h with h the leaf side (self-occlusion offset)."""
    h = np.float32(S) / np.float32(1 << D)
    return float(np.float32(np.float32(2.0 * np.sqrt(3.0)) * h))


def guide_sample(pdf, cdf_row, cdf_marg, N, bin_of_ray, u):
    pdf, cr, cm = _c(pdf, np.float32), _c(cdf_row, np.float32), _c(cdf_marg, np.float32)
    b, u = _c(bin_of_ray, np.uint32), _c(u, np.float32)
    n = len(b)
    d = np.zeros((n, 3), np.float32)
    p = np.zeros(n, np.float32)
    c = np.zeros(n, np.uint32)
    lib().orc_guide_sample(_p(pdf), _p(cr), _p(cm), N, _p(b), _p(u), n, _p(d), _p(p), _p(c))
    return d, p, c


def guide_eval_pdf(pdf, N, bins, dirs):
    pdf, b, d = _c(pdf, np.float32), _c(bins, np.uint32), _c(dirs, np.float32)
    out = np.zeros(len(b), np.float32)
    lib().orc_guide_eval_pdf(_p(pdf), N, _p(b), _p(d), len(b), _p(out))
    return out


def morton(x, y, z) -> int:
    return int(lib().orc_morton(int(x), int(y), int(z)))


def rng_u64(seed, stream, counter) -> int:
    return int(lib().orc_rng_u64(seed, stream, counter))


def sin(x):
    return float(lib().orc_sin(float(x)))


def cos(x):
    return float(lib().orc_cos(float(x)))


def atan01(q):
    return float(lib().orc_atan01(float(q)))


def octa_decode(uv):
    uv = _c(uv, np.float32).reshape(-1, 2)
    out = np.zeros((len(uv), 3), np.float32)
    lib().orc_octa_decode(_p(uv), len(uv), _p(out))
    return out


def octa_encode(d):
    d = _c(d, np.float32).reshape(-1, 3)
    out = np.zeros((len(d), 2), np.float32)
    lib().orc_octa_encode(_p(d), len(d), _p(out))
    return out


def kmeans2(n, w):
    n = _c(n, np.float32).reshape(-1, 3)
    w = _c(w, np.float32)
    out = np.zeros(3, np.float32)
    lib().orc_kmeans2(_p(n), _p(w), len(w), _p(out))
    return out


def warp_scan(x):
    x = _c(x, np.float32).copy()
    lib().orc_warp_scan(_p(x), len(x))
    return x


def blur(f, N):
    f = _c(f, np.float32).copy()
    lib().orc_blur(_p(f), N)
    return f


def pdf_cdf(f, N):
    f = _c(f, np.float32)
    pdf = np.zeros(N * N, np.float32)
    cr = np.zeros(N * N, np.float32)
    cm = np.zeros(N, np.float32)
    lib().orc_pdf_cdf(_p(f), N, _p(pdf), _p(cr), _p(cm))
    return pdf, cr, cm


# ----------------------------------------------------------------------------- learned proposal
MLP_IN, MLP_HID, MLP_OUT = 80, 64, 1024


def mlp_num_params() -> int:
    return int(lib().orc_mlp_num_params())


def bf16_round(x):
    """The bfloat16 rounding (to nearest, ties to even) of the emulation."""
    x = _c(x, np.float32).ravel()
    out = np.zeros_like(x)
    lib().orc_bf16_round(_p(x), len(x), _p(out))
    return out


def mlp_features(pos, nrm, lo, S):
    pos, nrm, lo = _c(pos, np.float32), _c(nrm, np.float32), _c(lo, np.float32)
    out = np.zeros((len(pos), MLP_IN), np.float64)
    lib().orc_mlp_features(_p(pos), _p(nrm), len(pos), _p(lo), float(S), _p(out))
    return out


def mlp_forward(params, pos, nrm, lo, S, bf16=False):
    params, pos, nrm, lo = (_c(params, np.float32), _c(pos, np.float32), _c(nrm, np.float32),
                            _c(lo, np.float32))
    n = len(pos)
    z = np.zeros((n, MLP_OUT), np.float64)
    p = np.zeros((n, MLP_OUT), np.float64)
    lib().orc_mlp_forward(_p(params), _p(pos), _p(nrm), n, _p(lo), float(S), int(bf16), _p(z), _p(p))
    return z, p


def mlp_grad(params, pos, nrm, lo, S, target, bf16=False):
    params, pos, nrm, lo = (_c(params, np.float32), _c(pos, np.float32), _c(nrm, np.float32),
                            _c(lo, np.float32))
    target = _c(target, np.float32)
    g = np.zeros(mlp_num_params(), np.float64)
    loss = lib().orc_mlp_grad(_p(params), _p(pos), _p(nrm), len(pos), _p(lo), float(S), _p(target),
                              int(bf16), _p(g))
    return float(loss), g


def mlp_grad_trace(params, pos, nrm, lo, S, target, bf16=False):
    """mlp_grad plus its per-sample intermediates (dict of [n][width] float64
    arrays: x, h1, h2, h3, z, g4, d3, d2, d1); the same arithmetic."""
    params, pos, nrm, lo = (_c(params, np.float32), _c(pos, np.float32), _c(nrm, np.float32),
                            _c(lo, np.float32))
    target = _c(target, np.float32)
    n = len(pos)
    g = np.zeros(mlp_num_params(), np.float64)
    widths = {"x": MLP_IN, "h1": MLP_HID, "h2": MLP_HID, "h3": MLP_HID, "z": MLP_OUT, "g4": MLP_OUT,
              "d3": MLP_HID, "d2": MLP_HID, "d1": MLP_HID}
    tr = {k: np.zeros((n, w), np.float64) for k, w in widths.items()}
    loss = lib().orc_mlp_grad_trace(_p(params), _p(pos), _p(nrm), n, _p(lo), float(S), _p(target), int(bf16),
                                    _p(g), *(_p(tr[k]) for k in widths))
    return float(loss), g, tr


def adam(params, m, v, grad, t, lr=1e-3, b1=0.9, b2=0.999, eps=1e-8):
    params = _c(params, np.float32).copy()
    m = _c(m, np.float64).copy()
    v = _c(v, np.float64).copy()
    grad = _c(grad, np.float64)
    lib().orc_adam(_p(params), _p(m), _p(v), _p(grad), len(params), int(t), lr, b1, b2, eps)
    return params, m, v


# ---------------------------------------------------------------- product guiding (Sec. 3.6)
def product_block_sums(pdf, N):
    """S[bin][64]: sums of the cell densities over the 8 x 8 blocks (row-major)."""
    pdf = _c(pdf, np.float32).reshape(-1, N * N)
    S = np.zeros((pdf.shape[0], 64), np.float32)
    lib().orc_product_block_sums(_p(pdf), N, pdf.shape[0], _p(S))
    return S


def product_sample(pdf, S, N, bins, nrm, u):
    """Two-stage product sampling (block from beta_B S_B, then cell and point in
    the block from the field).  Returns (dir [n,3], pdf [n], cell [n])."""
    pdf = _c(pdf, np.float32)
    S = _c(S, np.float32)
    bins = _c(bins, np.uint32)
    nrm = _c(nrm, np.float32).reshape(-1, 3)
    u = _c(u, np.float32).reshape(-1, 2)
    n = len(bins)
    d = np.zeros((n, 3), np.float32)
    p = np.zeros(n, np.float32)
    c = np.zeros(n, np.uint32)
    lib().orc_product_sample(_p(pdf), _p(S), N, _p(bins), _p(nrm), _p(u), n, _p(d), _p(p), _p(c))
    return d, p, c


def product_eval(pdf, S, N, bins, nrm, dirs):
    """Product density of given directions."""
    pdf = _c(pdf, np.float32)
    S = _c(S, np.float32)
    bins = _c(bins, np.uint32)
    nrm = _c(nrm, np.float32).reshape(-1, 3)
    dirs = _c(dirs, np.float32).reshape(-1, 3)
    out = np.zeros(len(bins), np.float32)
    lib().orc_product_eval(_p(pdf), _p(S), N, _p(bins), _p(nrm), _p(dirs), len(bins), _p(out))
    return out


def product_block_weight(n, B):
    return float(lib().orc_product_block_weight(_p(_c(n, np.float32)), int(B)))
