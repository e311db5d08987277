"""Seeded synthetic inputs for the wavefront path-guiding hot path.

This module only *makes inputs*: procedural scenes (axis-aligned quads and
spheres), path-vertex radiance records, ray hit points with normals, Zipf bin
sizes and uniform random numbers.  It holds none of the method's arithmetic
(no voxelisation, no octree, no binning, no radiance field, no CDF) and is
imported by both the CPU oracle tests and the CUDA tests, so that both sides
see exactly the same arrays.

The paper measures on Sponza, Veach Door, Bathroom and Cornell Box (Sec. 4,
Table 1); none of those scenes exist here, so these procedural scenes stand
in for them with the paper's workload shapes (1080p, thousands of bins,
16^2..128^2 grids, SVO 64^3..2048^3).

Array conventions (all numpy, C-contiguous):
  quads   float32 [n, 8]: axis, plane, lo1, hi1, lo2, hi2, nsign, 0
          the quad lies in the plane x_axis = plane; it spans [lo1, hi1] on
          axis (axis+1)%3 and [lo2, hi2] on axis (axis+2)%3; its normal is
          nsign * e_axis.
  spheres float32 [n, 4]: cx, cy, cz, r
  positions / directions / normals float32 [n, 3]
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

QUAD_STRIDE = 8
SPHERE_STRIDE = 4


@dataclass
class Scene:
    quads: np.ndarray                 # float32 [nq, 8]
    spheres: np.ndarray               # float32 [ns, 4]
    albedo: np.ndarray                # float32 [nq + ns]  (quads first)
    emission: np.ndarray              # float32 [nq + ns]  (quads first)
    lo: np.ndarray                    # float32 [3], lower corner of the cubic AABB
    size: float                       # side S of the cubic AABB
    name: str = ""
    extra: dict = field(default_factory=dict)
    # float32 [nt, 9]: v0, v1, v2; primitive ids count quads, then spheres, then triangles
    tris: np.ndarray = field(default_factory=lambda: np.zeros((0, 9), np.float32))

    @property
    def n_quads(self) -> int:
        return int(self.quads.shape[0])

    @property
    def n_spheres(self) -> int:
        return int(self.spheres.shape[0])

    @property
    def n_tris(self) -> int:
        return int(self.tris.shape[0])


def _quad(axis, plane, lo1, hi1, lo2, hi2, nsign):
    return [float(axis), float(plane), float(lo1), float(hi1), float(lo2), float(hi2),
            float(nsign), 0.0]


def _box_walls(open_front: bool):
    """Six inward-facing walls of the unit cube (front = the z = 0 face)."""
    q = [
        _quad(0, 0.0, 0.0, 1.0, 0.0, 1.0, +1),   # x = 0 (left),  normal +x
        _quad(0, 1.0, 0.0, 1.0, 0.0, 1.0, -1),   # x = 1 (right), normal -x
        _quad(1, 0.0, 0.0, 1.0, 0.0, 1.0, +1),   # y = 0 (floor), normal +y
        _quad(1, 1.0, 0.0, 1.0, 0.0, 1.0, -1),   # y = 1 (ceiling), normal -y
        _quad(2, 1.0, 0.0, 1.0, 0.0, 1.0, -1),   # z = 1 (back),  normal -z
    ]
    if not open_front:
        q.append(_quad(2, 0.0, 0.0, 1.0, 0.0, 1.0, +1))  # z = 0 (front), normal +z
    return q


def closed_box(seed: int, depth: int) -> Scene:
    """Unit cube, 6 inward walls with albedo U[0.3, 0.8] each, plus an emissive
    ceiling quad [0.35, 0.65]^2 (radiance 10) half a leaf below the ceiling."""
    rng = np.random.default_rng(seed)
    h = 1.0 / (1 << depth)
    walls = _box_walls(open_front=False)
    light = _quad(1, 1.0 - 0.5 * h, 0.35, 0.65, 0.35, 0.65, -1)
    # axis 1 (y): lo1/hi1 is on axis 2 (z), lo2/hi2 on axis 0 (x)
    quads = np.array(walls + [light], dtype=np.float32)
    albedo = np.concatenate([rng.uniform(0.3, 0.8, len(walls)), [0.0]]).astype(np.float32)
    emission = np.array([0.0] * len(walls) + [10.0], dtype=np.float32)
    return Scene(quads=quads, spheres=np.zeros((0, 4), np.float32), albedo=albedo,
                 emission=emission, lo=np.zeros(3, np.float32), size=1.0,
                 name=f"closed_box(seed={seed},D={depth})")


def cornell_spheres(seed: int, n_spheres: int = 200) -> Scene:
    """Unit Cornell-style box with the front (z = 0) open, red/green side walls
    and n seeded spheres (centre U[0.1, 0.9]^3, radius U[0.02, 0.1]); 10% of the
    spheres are emissive with radiance U[1, 20]."""
    rng = np.random.default_rng(seed)
    walls = _box_walls(open_front=True)
    quads = np.array(walls, dtype=np.float32)
    wall_albedo = np.array([0.63, 0.45, 0.75, 0.75, 0.75], np.float32)  # red, green, white
    c = rng.uniform(0.1, 0.9, (n_spheres, 3))
    r = rng.uniform(0.02, 0.1, n_spheres)
    spheres = np.concatenate([c, r[:, None]], axis=1).astype(np.float32)
    emissive = rng.uniform(0, 1, n_spheres) < 0.10
    s_emit = np.where(emissive, rng.uniform(1.0, 20.0, n_spheres), 0.0)
    s_alb = rng.uniform(0.2, 0.9, n_spheres)
    albedo = np.concatenate([wall_albedo, s_alb]).astype(np.float32)
    emission = np.concatenate([np.zeros(len(walls)), s_emit]).astype(np.float32)
    return Scene(quads=quads, spheres=spheres, albedo=albedo, emission=emission,
                 lo=np.zeros(3, np.float32), size=1.0,
                 name=f"cornell_spheres(seed={seed},n={n_spheres})")


def single_sphere(center, radius) -> Scene:
    """One sphere inside the unit cube (used by tests)."""
    sp = np.array([[center[0], center[1], center[2], radius]], np.float32)
    return Scene(quads=np.zeros((0, 8), np.float32), spheres=sp,
                 albedo=np.array([0.5], np.float32), emission=np.array([0.0], np.float32),
                 lo=np.zeros(3, np.float32), size=1.0, name="single_sphere")


def small_deep(seed: int) -> Scene:
    """Maximum-depth test scene: six small quads facing one another (one of
    them emissive, radiance 10) around a tiny sphere, all inside [0.45, 0.55]^3
    of the unit cube -- about 2e4 occupied leaves at depth 11 (2048^3)."""
    rng = np.random.default_rng(seed)
    c, h = 0.5, 0.03
    quads = [
        _quad(0, c - h, c - h, c + h, c - h, c + h, +1), _quad(0, c + h, c - h, c + h, c - h, c + h, -1),
        _quad(1, c - h, c - h, c + h, c - h, c + h, +1), _quad(1, c + h, c - h, c + h, c - h, c + h, -1),
        _quad(2, c - h, c - h, c + h, c - h, c + h, +1), _quad(2, c + h, c - h, c + h, c - h, c + h, -1),
    ]
    albedo = np.concatenate([rng.uniform(0.3, 0.8, 6), [0.5]]).astype(np.float32)
    albedo[3] = 0.0
    emission = np.zeros(7, np.float32)
    emission[3] = 10.0
    spheres = np.array([[c + 0.004, c - 0.003, c + 0.002, 0.008]], np.float32)
    return Scene(quads=np.array(quads, np.float32), spheres=spheres, albedo=albedo, emission=emission,
                 lo=np.zeros(3, np.float32), size=1.0, name=f"small_deep(seed={seed})")


def city(seed: int, n_boxes: int = 5000, n_lights: int = 50, size: float = 500.0) -> Scene:
    """Procedural city: ground quad, n seeded boxes (side log-uniform in
    [0.5, 20], uniform on the ground) and n emissive quads hovering above."""
    rng = np.random.default_rng(seed)
    quads = [_quad(1, 0.0, 0.0, size, 0.0, size, +1)]
    alb = [0.5]
    emi = [0.0]
    side = np.exp(rng.uniform(math.log(0.5), math.log(20.0), (n_boxes, 3)))
    px = rng.uniform(0.0, size, n_boxes)
    pz = rng.uniform(0.0, size, n_boxes)
    for k in range(n_boxes):
        sx, sy, sz = side[k]
        x0 = float(min(max(px[k] - sx / 2, 0.0), size - sx))
        z0 = float(min(max(pz[k] - sz / 2, 0.0), size - sz))
        x1, y1, z1 = x0 + sx, sy, z0 + sz
        a = float(rng.uniform(0.2, 0.8))
        quads += [
            _quad(0, x0, 0.0, y1, z0, z1, -1), _quad(0, x1, 0.0, y1, z0, z1, +1),
            _quad(1, y1, z0, z1, x0, x1, +1),
            _quad(2, z0, x0, x1, 0.0, y1, -1), _quad(2, z1, x0, x1, 0.0, y1, +1),
        ]
        alb += [a] * 5
        emi += [0.0] * 5
    for k in range(n_lights):
        cx, cz = rng.uniform(20.0, size - 20.0, 2)
        hgt = float(rng.uniform(30.0, 60.0))
        w = float(rng.uniform(2.0, 8.0))
        quads.append(_quad(1, hgt, cz - w, cz + w, cx - w, cx + w, -1))
        alb.append(0.0)
        emi.append(float(rng.uniform(5.0, 50.0)))
    return Scene(quads=np.array(quads, np.float32), spheres=np.zeros((0, 4), np.float32),
                 albedo=np.array(alb, np.float32), emission=np.array(emi, np.float32),
                 lo=np.zeros(3, np.float32), size=float(size), name=f"city(seed={seed})")


# --------------------------------------------------------------------------------------
# sampling helpers (input generation only)

def uniforms24(seed: int, shape) -> np.ndarray:
    """float32 uniforms on the 2^-24 lattice in [0, 1) (exactly representable)."""
    rng = np.random.default_rng(seed)
    return (rng.integers(0, 1 << 24, size=shape, dtype=np.int64).astype(np.float64)
            * (1.0 / (1 << 24))).astype(np.float32)


def _frame(n):
    """Orthonormal tangent frames for unit normals n [k, 3] (float64)."""
    sgn = np.where(n[:, 2] >= 0, 1.0, -1.0)
    a = -1.0 / (sgn + n[:, 2])
    b = n[:, 0] * n[:, 1] * a
    t = np.stack([1.0 + sgn * n[:, 0] ** 2 * a, sgn * b, -sgn * n[:, 0]], axis=1)
    bt = np.stack([b, sgn + n[:, 1] ** 2 * a, -n[:, 1]], axis=1)
    return t, bt


def cosine_dirs(normals: np.ndarray, rng) -> np.ndarray:
    n = normals.astype(np.float64)
    u1 = rng.uniform(0, 1, len(n))
    u2 = rng.uniform(0, 1, len(n))
    r = np.sqrt(u1)
    phi = 2 * np.pi * u2
    x, y = r * np.cos(phi), r * np.sin(phi)
    z = np.sqrt(np.maximum(0.0, 1.0 - u1))
    t, bt = _frame(n)
    d = t * x[:, None] + bt * y[:, None] + n * z[:, None]
    return d / np.linalg.norm(d, axis=1, keepdims=True)


# --------------------------------------------------------------------------------------
# triangle meshes (the paper voxelises triangle scenes; these are procedural stand-ins)

def _box_tris():
    """The six walls of the unit cube as 12 triangles, (v1 - v0) x (v2 - v0) inward."""
    out = []
    for ax in range(3):
        a1, a2 = (ax + 1) % 3, (ax + 2) % 3
        for plane, sgn in ((0.0, +1.0), (1.0, -1.0)):
            c = np.zeros((4, 3))
            c[:, ax] = plane
            c[:, a1] = [0, 1, 1, 0]
            c[:, a2] = [0, 0, 1, 1]
            for t in ((0, 1, 2), (0, 2, 3)):
                v = c[list(t)]
                n = np.cross(v[1] - v[0], v[2] - v[0])
                if n[ax] * sgn < 0:
                    v = v[[0, 2, 1]]
                out.append(v.ravel())
    return np.array(out)


def _icosphere(center, radius, subdiv, rng=None, bump=0.0):
    """Subdivided icosahedron, outward winding; bump > 0 displaces the vertices
    radially by a seeded factor U[1 - bump, 1 + bump] (a rock)."""
    t = (1.0 + 5 ** 0.5) / 2.0
    V = [[-1, t, 0], [1, t, 0], [-1, -t, 0], [1, -t, 0], [0, -1, t], [0, 1, t], [0, -1, -t], [0, 1, -t],
         [t, 0, -1], [t, 0, 1], [-t, 0, -1], [-t, 0, 1]]
    V = [list(np.array(v) / np.linalg.norm(v)) for v in V]
    F = [(0, 11, 5), (0, 5, 1), (0, 1, 7), (0, 7, 10), (0, 10, 11), (1, 5, 9), (5, 11, 4), (11, 10, 2),
         (10, 7, 6), (7, 1, 8), (3, 9, 4), (3, 4, 2), (3, 2, 6), (3, 6, 8), (3, 8, 9), (4, 9, 5), (2, 4, 11),
         (6, 2, 10), (8, 6, 7), (9, 8, 1)]
    for _ in range(subdiv):
        mid = {}

        def m(a, b):
            k = (min(a, b), max(a, b))
            if k not in mid:
                v = np.array(V[a]) + np.array(V[b])
                V.append(list(v / np.linalg.norm(v)))
                mid[k] = len(V) - 1
            return mid[k]
        F = [f for a, b, c in F for f in ((a, m(a, b), m(c, a)), (b, m(b, c), m(a, b)), (c, m(c, a), m(b, c)),
                                          (m(a, b), m(b, c), m(c, a)))]
    V = np.array(V)
    if bump > 0:
        V = V * rng.uniform(1 - bump, 1 + bump, (len(V), 1))
    V = np.asarray(center) + radius * V
    tri = V[np.array(F)]
    n = np.cross(tri[:, 1] - tri[:, 0], tri[:, 2] - tri[:, 0])
    flip = np.einsum("ij,ij->i", n, tri.mean(axis=1) - np.asarray(center)) < 0
    tri[flip] = tri[flip][:, [0, 2, 1]]
    return tri.reshape(-1, 9)


def _torus(center, R, r, nu, nv):
    """Torus about the y axis (major radius R, minor r), nu x nv quads split in two."""
    u = np.linspace(0, 2 * np.pi, nu + 1)[:-1]
    v = np.linspace(0, 2 * np.pi, nv + 1)[:-1]
    P = np.zeros((nu, nv, 3))
    for i, a in enumerate(u):
        for j, b in enumerate(v):
            P[i, j] = [(R + r * np.cos(b)) * np.cos(a), r * np.sin(b), (R + r * np.cos(b)) * np.sin(a)]
    P += np.asarray(center)
    out = []
    for i in range(nu):
        for j in range(nv):
            a, b = P[i, j], P[(i + 1) % nu, j]
            c, d = P[(i + 1) % nu, (j + 1) % nv], P[i, (j + 1) % nv]
            for t in ((a, b, c), (a, c, d)):
                # outward winding: the normal points away from the tube's centre line
                m = (t[0] + t[1] + t[2]) / 3 - np.asarray(center)
                ring = R * np.array([m[0], 0.0, m[2]]) / np.hypot(m[0], m[2])
                n = np.cross(t[1] - t[0], t[2] - t[0])
                out.append(np.concatenate(t if n @ (m - ring) > 0 else (t[0], t[2], t[1])))
    return np.array(out)


def mesh_room(seed: int = 1, depth: int = 7, subdiv: int = 3) -> Scene:
    """A closed unit box made of triangles (walls albedo U[0.3, 0.8] each), a
    ceiling light of two triangles (radiance 10) half a leaf below the
    ceiling, and three meshes: an icosphere, a seeded rock (bumped
    icosphere) and a torus -- about 3.3k triangles at subdiv 3.  No quads or
    spheres: every primitive is a triangle."""
    rng = np.random.default_rng(seed)
    h = 1.0 / (1 << depth)
    walls = _box_tris()
    y = 1.0 - 0.5 * h
    light = np.array([[0.35, y, 0.35, 0.65, y, 0.35, 0.65, y, 0.65],   # winding normal -y (down)
                      [0.35, y, 0.35, 0.65, y, 0.65, 0.35, y, 0.65]])
    ico = _icosphere((0.3, 0.25, 0.6), 0.18, subdiv)
    rock = _icosphere((0.72, 0.2, 0.35), 0.15, subdiv, rng=rng, bump=0.15)
    torus = _torus((0.55, 0.55, 0.7), 0.17, 0.06, 32, 16)
    parts = [walls, light, ico, rock, torus]
    tris = np.concatenate(parts).astype(np.float32)
    alb = np.concatenate([np.repeat(rng.uniform(0.3, 0.8, 6), 2), [0.0, 0.0],
                          np.full(len(ico), 0.7), np.full(len(rock), 0.45), np.full(len(torus), 0.6)])
    emi = np.zeros(len(tris))
    emi[len(walls):len(walls) + 2] = 10.0
    return Scene(quads=np.zeros((0, 8), np.float32), spheres=np.zeros((0, 4), np.float32),
                 albedo=alb.astype(np.float32), emission=emi.astype(np.float32), lo=np.zeros(3, np.float32),
                 size=1.0, name=f"mesh_room(seed={seed},D={depth},subdiv={subdiv})", tris=tris)


def tri_area(tris):
    t = np.asarray(tris, np.float64).reshape(-1, 9)
    return 0.5 * np.linalg.norm(np.cross(t[:, 3:6] - t[:, 0:3], t[:, 6:9] - t[:, 0:3]), axis=1)


def tri_surface_points(scene: Scene, rng, n: int, use=None):
    """Area-uniform points on the scene's triangles (or the subset `use`).
    Returns (pos, nrm, prim) with nrm the winding normal (v1 - v0) x (v2 - v0)."""
    t = scene.tris.astype(np.float64)
    sel = np.arange(len(t)) if use is None else np.asarray(use)
    a = tri_area(t[sel])
    pick = sel[rng.choice(len(sel), size=n, p=a / a.sum())]
    T = t[pick]
    s = np.sqrt(rng.uniform(0, 1, n))
    b = rng.uniform(0, 1, n)
    w0, w1 = 1 - s, b * s
    pos = w0[:, None] * T[:, 0:3] + w1[:, None] * T[:, 3:6] + (1 - w0 - w1)[:, None] * T[:, 6:9]
    nrm = np.cross(T[:, 3:6] - T[:, 0:3], T[:, 6:9] - T[:, 0:3])
    nrm /= np.linalg.norm(nrm, axis=1, keepdims=True)
    return pos.astype(np.float32), nrm.astype(np.float32), pick + scene.n_quads + scene.n_spheres


def _quad_area(q):
    return (q[:, 3] - q[:, 2]) * (q[:, 5] - q[:, 4])


def surface_points(scene: Scene, rng, n: int, use_quads=None, with_spheres=True):
    """Area-uniform points on the scene's surfaces.  Returns (pos, nrm, prim)
    with quad normals as stored and sphere normals pointing outward."""
    q = scene.quads.astype(np.float64)
    qsel = np.arange(len(q)) if use_quads is None else np.asarray(use_quads)
    areas = [_quad_area(q[qsel])]
    if with_spheres and scene.n_spheres:
        areas.append(4 * np.pi * scene.spheres[:, 3].astype(np.float64) ** 2)
    area = np.concatenate(areas)
    prims = np.concatenate([qsel, scene.n_quads + np.arange(scene.n_spheres)])[: len(area)]
    pick = rng.choice(len(area), size=n, p=area / area.sum())
    prim = prims[pick]
    pos = np.zeros((n, 3))
    nrm = np.zeros((n, 3))
    isq = prim < scene.n_quads
    if isq.any():
        qq = q[prim[isq]]
        ax = qq[:, 0].astype(int)
        a1 = (ax + 1) % 3
        a2 = (ax + 2) % 3
        s1 = rng.uniform(0, 1, len(qq))
        s2 = rng.uniform(0, 1, len(qq))
        p = np.zeros((len(qq), 3))
        rows = np.arange(len(qq))
        p[rows, ax] = qq[:, 1]
        p[rows, a1] = qq[:, 2] + s1 * (qq[:, 3] - qq[:, 2])
        p[rows, a2] = qq[:, 4] + s2 * (qq[:, 5] - qq[:, 4])
        nn = np.zeros((len(qq), 3))
        nn[rows, ax] = qq[:, 6]
        pos[isq] = p
        nrm[isq] = nn
    iss = ~isq
    if iss.any():
        sp = scene.spheres[prim[iss] - scene.n_quads].astype(np.float64)
        v = rng.normal(size=(int(iss.sum()), 3))
        v /= np.linalg.norm(v, axis=1, keepdims=True)
        pos[iss] = sp[:, :3] + sp[:, 3:4] * v
        nrm[iss] = v
    return pos.astype(np.float32), nrm.astype(np.float32), prim


def box_records(scene: Scene, seed: int, n: int):
    """Radiance records (pos, w_out, L) on the closed box: area-uniform on the
    walls and the light, w_out cosine-distributed about the inward normal,
    L = emission on the light, otherwise albedo * 10 * U[0, 1]."""
    rng = np.random.default_rng(seed)
    pos, nrm, prim = surface_points(scene, rng, n, with_spheres=False)
    wout = cosine_dirs(nrm, rng)
    emi = scene.emission[prim]
    L = np.where(emi > 0, emi, scene.albedo[prim] * 10.0 * rng.uniform(0, 1, n))
    return pos, wout.astype(np.float32), L.astype(np.float32)


def box_rays(scene: Scene, seed: int, n: int):
    """Ray hit points area-uniform on the walls (not the light), inward normals."""
    rng = np.random.default_rng(seed)
    walls = [i for i in range(scene.n_quads) if scene.emission[i] == 0]
    pos, nrm, _ = surface_points(scene, rng, n, use_quads=walls, with_spheres=False)
    return pos, nrm


# --------------------------------------------------------------------------------------
# a small analytic ray caster used to make hit points and radiance records

def _cast_quads(q, o, d, tmin):
    """Closest hit among axis-aligned quads q [nq, 8] (float64)."""
    T = np.full(len(o), np.inf)
    P = np.full(len(o), -1, np.int64)
    for k in range(len(q)):
        ax = int(q[k, 0])
        a1, a2 = (ax + 1) % 3, (ax + 2) % 3
        with np.errstate(divide="ignore", invalid="ignore"):
            t = (q[k, 1] - o[:, ax]) / d[:, ax]
        p1 = o[:, a1] + t * d[:, a1]
        p2 = o[:, a2] + t * d[:, a2]
        ok = (t > tmin) & (t < T) & (p1 >= q[k, 2]) & (p1 <= q[k, 3]) & \
             (p2 >= q[k, 4]) & (p2 <= q[k, 5])
        T[ok] = t[ok]
        P[ok] = k
    return T, P


def _sphere_t(c, r, o, d, tmin):
    """Ray parameter of the first intersection in front of tmin (inf on miss)."""
    oc = o - c
    b = np.einsum("nk,nk->n", d, oc)
    cc = np.einsum("nk,nk->n", oc, oc) - r * r
    disc = b * b - cc
    sq = np.sqrt(np.maximum(disc, 0.0))
    t = -b - sq
    t = np.where(t > tmin, t, -b + sq)
    return np.where((disc >= 0) & (t > tmin), t, np.inf)


def _shade(scene, o, d, T, P):
    hit = P >= 0
    pos = o + np.where(hit, T, 0.0)[:, None] * d
    nrm = np.zeros_like(pos)
    q = scene.quads.astype(np.float64)
    hq = hit & (P < len(q))
    if hq.any():
        ax = q[P[hq], 0].astype(int)
        nrm[np.flatnonzero(hq), ax] = q[P[hq], 6]
        pos[np.flatnonzero(hq), ax] = q[P[hq], 1]      # snap onto the quad's plane
    hs = hit & (P >= len(q))
    if hs.any():
        c = scene.spheres[P[hs] - len(q)].astype(np.float64)
        v = pos[hs] - c[:, :3]
        nrm[hs] = v / np.linalg.norm(v, axis=1, keepdims=True)
    flip = np.einsum("nk,nk->n", nrm, d) > 0
    nrm[flip] *= -1
    return pos, nrm


def cast(scene: Scene, o: np.ndarray, d: np.ndarray, tmin=1e-5, spheres=None):
    """Closest hit of rays (o, d) against the scene's quads and the given
    spheres (all by default).  Returns (t, prim, pos, nrm), nrm facing the
    incoming ray; prim = -1 on a miss."""
    o = o.astype(np.float64)
    d = d.astype(np.float64)
    T, P = _cast_quads(scene.quads.astype(np.float64), o, d, tmin)
    sp = scene.spheres.astype(np.float64)
    idx = range(len(sp)) if spheres is None else spheres
    for k in idx:
        t = _sphere_t(sp[k, :3], sp[k, 3], o, d, tmin)
        upd = t < T
        T[upd] = t[upd]
        P[upd] = scene.n_quads + k
    pos, nrm = _shade(scene, o, d, T, P)
    return T, P, pos, nrm


def pinhole_rays(eye, width: int, height: int, vfov_deg: float):
    """Camera rays through pixel centres of a pinhole looking along +z."""
    tan_half = math.tan(math.radians(vfov_deg) / 2)
    aspect = width / height
    ys, xs = np.meshgrid(np.arange(height), np.arange(width), indexing="ij")
    px = ((xs + 0.5) / width * 2 - 1) * tan_half * aspect
    py = (1 - (ys + 0.5) / height * 2) * tan_half
    d = np.stack([px, py, np.ones_like(px)], axis=-1).reshape(-1, 3)
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    o = np.broadcast_to(np.asarray(eye, np.float64), d.shape).copy()
    return o, d


def camera_hits(scene: Scene, eye=(0.5, 0.5, -1.0), width=1920, height=1080, vfov=40.0):
    """Primary hits of a pinhole camera: (pos, nrm, prim, dir) of the rays that
    hit.  Each sphere is only tested against the pixels of its conservative
    screen-space bounding box."""
    o, d = pinhole_rays(eye, width, height, vfov)
    T, P = _cast_quads(scene.quads.astype(np.float64), o, d, 1e-5)
    tan_half = math.tan(math.radians(vfov) / 2)
    aspect = width / height
    ex, ey, ez = (float(v) for v in eye)
    Tim = T.reshape(height, width)
    Pim = P.reshape(height, width)
    Dim = d.reshape(height, width, 3)
    for k, (cx, cy, cz, r) in enumerate(scene.spheres.astype(np.float64)):
        zn, zf = cz - r - ez, cz + r - ez
        if zf <= 0:
            continue
        zn = max(zn, 1e-6)
        xs = [(cx + sx * r - ex) / z for sx in (-1, 1) for z in (zn, zf)]
        ys = [(cy + sy * r - ey) / z for sy in (-1, 1) for z in (zn, zf)]
        c0 = int(math.floor((min(xs) / (tan_half * aspect) + 1) * width / 2 - 0.5)) - 2
        c1 = int(math.ceil((max(xs) / (tan_half * aspect) + 1) * width / 2 - 0.5)) + 2
        r0 = int(math.floor((1 - max(ys) / tan_half) * height / 2 - 0.5)) - 2
        r1 = int(math.ceil((1 - min(ys) / tan_half) * height / 2 - 0.5)) + 2
        c0, c1 = max(c0, 0), min(c1, width - 1)
        r0, r1 = max(r0, 0), min(r1, height - 1)
        if c0 > c1 or r0 > r1:
            continue
        dd = Dim[r0:r1 + 1, c0:c1 + 1].reshape(-1, 3)
        oo = np.broadcast_to(np.asarray(eye, np.float64), dd.shape)
        t = _sphere_t(np.array([cx, cy, cz]), r, oo, dd, 1e-5).reshape(r1 - r0 + 1, c1 - c0 + 1)
        sub_t = Tim[r0:r1 + 1, c0:c1 + 1]
        sub_p = Pim[r0:r1 + 1, c0:c1 + 1]
        upd = t < sub_t
        sub_t[upd] = t[upd]
        sub_p[upd] = scene.n_quads + k
    pos, nrm = _shade(scene, o, d, T, P)
    hit = P >= 0
    return (pos[hit].astype(np.float32), nrm[hit].astype(np.float32), P[hit],
            d[hit].astype(np.float32))


def one_bounce_records(scene: Scene, pos, nrm, prim, view_dir, seed: int):
    """Radiance records from one bounce of a Lambertian path tracer (Eq. 5 of
    the paper back-propagates an emitter's radiance to every vertex of the
    path): one record per primary hit p1, L = albedo(p1) * Le(p2) + Le(p1)
    when the cosine-sampled bounce reaches an emitter p2 (else Le(p1)),
    leaving toward the camera; plus one record at every emitter vertex p2
    that a bounce reached, L = Le(p2), leaving toward p1.  Only the emissive
    primitives are tested first; rays that reach one are then checked for
    occluders."""
    rng = np.random.default_rng(seed)
    d2 = cosine_dirs(nrm, rng)
    o2 = pos.astype(np.float64) + 1e-4 * nrm.astype(np.float64)
    nq = scene.n_quads
    emi_s = [k for k in range(scene.n_spheres) if scene.emission[nq + k] > 0]
    other_s = [k for k in range(scene.n_spheres) if scene.emission[nq + k] <= 0]
    T, P = _cast_quads(scene.quads.astype(np.float64), o2, d2, 1e-5)
    sp = scene.spheres.astype(np.float64)
    for k in emi_s:
        t = _sphere_t(sp[k, :3], sp[k, 3], o2, d2, 1e-5)
        upd = t < T
        T[upd] = t[upd]
        P[upd] = nq + k
    cand = np.flatnonzero((P >= 0) & (scene.emission[np.maximum(P, 0)] > 0))
    if len(cand):
        oc, dc, tc = o2[cand], d2[cand], T[cand]
        blocked = np.zeros(len(cand), bool)
        for k in other_s:
            blocked |= _sphere_t(sp[k, :3], sp[k, 3], oc, dc, 1e-5) < tc
        P[cand[blocked]] = -1
    le2 = np.where(P >= 0, scene.emission[np.maximum(P, 0)], 0.0)
    L = scene.albedo[prim] * le2 + scene.emission[prim]
    wout = -view_dir.astype(np.float64)
    hit_e = np.flatnonzero(le2 > 0)
    p2 = o2[hit_e] + T[hit_e, None] * d2[hit_e]
    rec_pos = np.concatenate([pos.astype(np.float64), p2]).astype(np.float32)
    rec_w = np.concatenate([wout, -d2[hit_e]]).astype(np.float32)
    rec_L = np.concatenate([L, le2[hit_e]]).astype(np.float32)
    return rec_pos, rec_w, rec_L


def zipf_bin_sizes(n_rays: int, n_bins: int, s: float, seed: int) -> np.ndarray:
    """Run lengths (uint32 [n_bins], sum = n_rays) with Zipf(s) sizes by rank,
    the ranks assigned to runs by a seeded permutation.  Sizes are
    floor(R * w_k / W) with the remainder handed out one each to the largest
    ranks; every run gets at least one ray when n_rays >= n_bins."""
    k = np.arange(1, n_bins + 1, dtype=np.float64)
    w = k ** (-s)
    raw = n_rays * w / w.sum()
    sizes = np.floor(raw).astype(np.int64)
    if n_rays >= n_bins:
        sizes = np.maximum(sizes, 1)
    rem = n_rays - int(sizes.sum())
    i = 0
    while rem != 0:
        step = 1 if rem > 0 else -1
        j = i % n_bins
        if step > 0 or sizes[j] > 1:
            sizes[j] += step
            rem -= step
        i += 1
    perm = np.random.default_rng(seed).permutation(n_bins)
    return sizes[perm].astype(np.uint32)


# --------------------------------------------------------------------------------------
# workload recipes

@dataclass
class Workload:
    scene: Scene
    depth: int
    rec_pos: np.ndarray
    rec_wout: np.ndarray
    rec_L: np.ndarray
    ray_pos: np.ndarray
    ray_nrm: np.ndarray
    u: np.ndarray                     # float32 [R, 2] sampling uniforms
    grid_n: int
    bin_mode: int                     # 0 = SVO Partition-S, 1 = Zipf runs
    l_min: int = 2
    c_ray: int = 0xFFFFFFFF
    bin_sizes: np.ndarray | None = None
    n_bins_max: int = 64
    blur: bool = False
    jitter: bool = False
    seed: int = 1
    desc: str = ""
    extra: dict = field(default_factory=dict)


def mesh_box(seed: int = 1, n_records: int = 100_000, n_rays: int = 4096, depth: int = 7) -> Workload:
    """The triangle-mesh room (mesh_room), SVO depth 7 (128^3), 100k records
    (area-uniform on every triangle, w_out cosine about the winding normal,
    L = emission on the light, else albedo * 10 * U[0, 1]), 4096 rays on the
    non-emissive triangles; otherwise as tiny_box."""
    sc = mesh_room(seed, depth)
    rng = np.random.default_rng(seed * 1000 + 1)
    rp, rn, prim = tri_surface_points(sc, rng, n_records)
    rw = cosine_dirs(rn, rng).astype(np.float32)
    emi = sc.emission[prim]
    rl = np.where(emi > 0, emi, sc.albedo[prim] * 10.0 * rng.uniform(0, 1, n_records)).astype(np.float32)
    rng2 = np.random.default_rng(seed * 1000 + 2)
    pp, pn, _ = tri_surface_points(sc, rng2, n_rays, use=np.flatnonzero(sc.emission == 0))
    u = uniforms24(seed * 1000 + 3, (n_rays, 2))
    return Workload(scene=sc, depth=depth, rec_pos=rp, rec_wout=rw, rec_L=rl, ray_pos=pp, ray_nrm=pn, u=u,
                    grid_n=16, bin_mode=0, l_min=2, c_ray=0xFFFFFFFF, n_bins_max=128, blur=False, jitter=False,
                    seed=seed, desc=f"triangle-mesh room ({sc.n_tris} triangles) D={depth}, 100k records, "
                                    "4096 rays, 16x16")


def tiny_box(seed: int = 1, n_records: int = 100_000, n_rays: int = 4096) -> Workload:
    """Closed box of 6 quads + a ceiling light, SVO depth 6 (64^3), 100k
    records, 4096 rays on the walls, Partition-S with l_min = 2 and no ray
    threshold (<= 64 bins), 16x16 grid, blur off, one sample per ray."""
    D = 6
    sc = closed_box(seed, D)
    rp, rw, rl = box_records(sc, seed * 1000 + 1, n_records)
    pp, pn = box_rays(sc, seed * 1000 + 2, n_rays)
    u = uniforms24(seed * 1000 + 3, (n_rays, 2))
    return Workload(scene=sc, depth=D, rec_pos=rp, rec_wout=rw, rec_L=rl, ray_pos=pp,
                    ray_nrm=pn, u=u, grid_n=16, bin_mode=0, l_min=2, c_ray=0xFFFFFFFF,
                    n_bins_max=64, blur=False, jitter=False, seed=seed,
                    desc="closed box D=6, 100k records, 4096 rays, 64 bins, 16x16")


def frame_spheres(seed: int = 1, width=1920, height=1080, n_bins=2048, depth=9,
                  grid_n=32) -> Workload:
    """Cornell-style box + 200 spheres, SVO depth 9 (512^3), pinhole camera
    1920x1080 primary hits, one record per hit from one bounce, bins by
    spatial cell + normal octant cut into 2048 Zipf(1.2) runs, 32x32 grid,
    blur and jitter on."""
    sc = cornell_spheres(seed)
    pos, nrm, prim, vdir = camera_hits(sc, width=width, height=height)
    rp, rw, rl = one_bounce_records(sc, pos, nrm, prim, vdir, seed * 1000 + 1)
    u = uniforms24(seed * 1000 + 3, (len(pos), 2))
    sizes = zipf_bin_sizes(len(pos), n_bins, 1.2, seed * 1000 + 4)
    return Workload(scene=sc, depth=depth, rec_pos=rp, rec_wout=rw, rec_L=rl, ray_pos=pos,
                    ray_nrm=nrm, u=u, grid_n=grid_n, bin_mode=1, bin_sizes=sizes,
                    n_bins_max=n_bins, blur=True, jitter=True, seed=seed, extra={"ray_prim": prim},
                    desc=f"cornell+200 spheres D={depth}, {width}x{height} primary hits, "
                         f"{n_bins} Zipf(1.2) bins, {grid_n}x{grid_n}")


# --------------------------------------------------------------------------------------
# learned proposal: initial weights and synthetic target distributions

MLP_IN, MLP_FEAT, MLP_HID, MLP_OUT = 80, 78, 64, 1024


def mlp_init(seed: int) -> np.ndarray:
    """Seeded initial parameters (He-uniform weights, zero biases), flat float32
    in the order W1[64][80], b1, W2[64][64], b2, W3[64][64], b3, W4[1024][64],
    b4; the two padding input columns of W1 are zero."""
    rng = np.random.default_rng(seed)
    parts = []
    for nout, nin, fan in ((MLP_HID, MLP_IN, MLP_FEAT), (MLP_HID, MLP_HID, MLP_HID),
                           (MLP_HID, MLP_HID, MLP_HID), (MLP_OUT, MLP_HID, MLP_HID)):
        lim = math.sqrt(6.0 / fan)
        W = rng.uniform(-lim, lim, (nout, nin))
        if nin == MLP_IN:
            W[:, MLP_FEAT:] = 0.0
        parts += [W.ravel(), np.zeros(nout)]
    return np.concatenate(parts).astype(np.float32)


def random_distributions(seed: int, n: int, k: int = MLP_OUT, conc: float = 0.3) -> np.ndarray:
    """n seeded probability vectors over k cells (Dirichlet(conc)), float32."""
    rng = np.random.default_rng(seed)
    g = rng.gamma(conc, 1.0, (n, k)) + 1e-6
    return (g / g.sum(axis=1, keepdims=True)).astype(np.float32)
