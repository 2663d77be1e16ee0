"""Seeded synthetic inputs for the hybrid depth-of-field frame.

This module is shared by the CUDA path's tests/bench and by the FP64 oracle's
tests.  It holds scene geometry, cameras, lens and parameter records and random
buffers only: none of the method's arithmetic (no CoC, no filtering, no
shading, no intersection) lives here.  Every array it returns is float32 /
int32 / uint8 so both sides read bit-identical inputs.

Workloads (the paper's "Modern Living Room" scene is not available; these
procedural scenes stand in for it):

* ``tiny``   128x128 checker quad at z=2 plus a 0.3x0.3 occluder at z=0.5
* ``room``   procedural room with random boxes and icospheres (1080p bench scene)
* ``room4k`` 512 boxes + 256 subdivision-5 icospheres (mixed-precision 4K scene)
"""
from __future__ import annotations

import dataclasses
import math
from dataclasses import dataclass, field

import numpy as np

F32 = np.float32

# --------------------------------------------------------------------------
# records
# --------------------------------------------------------------------------


@dataclass
class Camera:
    """Pinhole camera pose.  right/up/fwd are an orthonormal basis; the view
    looks along +fwd.  ``jitter`` is the sub-pixel offset (pixels) of every
    pixel's sample point this frame."""
    pos: tuple = (0.0, 0.0, 0.0)
    right: tuple = (1.0, 0.0, 0.0)
    up: tuple = (0.0, 1.0, 0.0)
    fwd: tuple = (0.0, 0.0, 1.0)
    tan_half_fovy: float = math.tan(math.radians(30.0))
    width: int = 128
    height: int = 128
    jitter: tuple = (0.0, 0.0)

    def f32(self) -> "Camera":
        """All float fields rounded to float32 (the precision both sides read)."""
        r = lambda v: tuple(float(F32(x)) for x in v)  # noqa: E731
        return Camera(r(self.pos), r(self.right), r(self.up), r(self.fwd),
                      float(F32(self.tan_half_fovy)), int(self.width), int(self.height),
                      r(self.jitter))


@dataclass
class Lens:
    """Thin lens: focus distance (view depth of the focus plane), aperture radius
    and focal length, all in scene units."""
    focus_dist: float = 2.0
    aperture_radius: float = 0.05
    focal_length: float = 0.05

    def f32(self) -> "Lens":
        return Lens(float(F32(self.focus_dist)), float(F32(self.aperture_radius)),
                    float(F32(self.focal_length)))


@dataclass
class Params:
    """Every tunable constant of the frame (the paper prints none)."""
    # adaptive ray mask
    gauss_sigma: float = 1.0
    edge_tau: float = 0.1
    tile: int = 16
    dilate: int = 1
    spp_max: int = 16
    variance_on: int = 0
    var_tau: float = 0.02
    var_scale: float = 0.1
    hlen_young: int = 4
    # ray trace
    seed: int = 0
    frame: int = 0
    view: int = 0
    k_ambient: float = 0.05
    light_dir: list = field(default_factory=lambda: [[0.3, 0.5, -1.0]])
    light_E: list = field(default_factory=lambda: [1.0])
    miss_dist: float = 1.0e4
    trav_cap: int = 0
    # temporal reconstruction
    ema_alpha: float = 0.2
    camera_moved: int = 0
    # spatial reconstruction
    r_s: float = 16.0
    var_ref: float = 0.05
    # post-filter
    r_max: float = 16.0
    kz_rel: float = 0.05
    # composite
    h_tau: float = 0.25
    # extensions named as future work in the paper's Discussion (0 = off)
    alpha_k: float = 0.0      # per-pixel temporal blend factor threshold (history std-devs)
    mask_coc: int = 0         # edge tiles dilate over their largest CoC radius
    blades: int = 0           # aperture polygon blades (0 = circle)
    blade_rot: float = 0.0    # polygon rotation (radians)
    aberration: float = 0.0   # radial weight of the lens samples, 1 + a (2 rho^2 / A^2 - 1)
    spec_pref: float = 0.0    # composite: post-process share per unit of its specular intensity

    def replace(self, **kw) -> "Params":
        return dataclasses.replace(self, **kw)

    def unit_lights(self):
        """Light directions normalised in float64 then rounded to float32."""
        out = []
        for d in self.light_dir:
            v = np.asarray(d, np.float64)
            out.append([float(F32(x)) for x in v / np.linalg.norm(v)])
        return out


@dataclass
class Scene:
    """Triangle soup with per-triangle material.

    verts f32 [V,3]; idx i32 [T,3]; mat f32 [T,8] = (albedo_a rgb, checker_n,
    albedo_b rgb, k_s) -- checker_n > 0 selects a checkerboard of n x n cells in
    the triangle's (u,v) parameterisation, cells with even floor(n u)+floor(n v)
    taking albedo_a; k_s > 0 adds a white Blinn-Phong highlight of that
    strength (0: Lambertian); uv f32 [T,6] = (u0,v0,u1,v1,u2,v2)."""
    verts: np.ndarray
    idx: np.ndarray
    mat: np.ndarray
    uv: np.ndarray

    @property
    def n_tris(self) -> int:
        return int(self.idx.shape[0])

    def tri_verts(self) -> np.ndarray:
        """[T,9] float32 vertex positions per triangle (v0,v1,v2)."""
        return self.verts[self.idx].reshape(-1, 9).astype(F32)


# --------------------------------------------------------------------------
# geometry builders
# --------------------------------------------------------------------------


class _Builder:
    """Accumulates triangle-soup chunks as numpy arrays."""

    def __init__(self):
        self.v, self.i, self.m, self.uv = [], [], [], []
        self.nv = 0

    def _add(self, verts, tris, mats, uvs):
        verts = np.asarray(verts, np.float64).reshape(-1, 3)
        tris = np.asarray(tris, np.int64).reshape(-1, 3) + self.nv
        self.v.append(verts)
        self.i.append(tris)
        self.m.append(np.broadcast_to(np.asarray(mats, np.float64), (len(tris), 8)))
        self.uv.append(np.broadcast_to(np.asarray(uvs, np.float64).reshape(-1, 6), (len(tris), 6)))
        self.nv += len(verts)

    def quad(self, p0, p1, p2, p3, mat, uvs=((0, 0), (1, 0), (1, 1), (0, 1))):
        """Two triangles (p0,p1,p2), (p0,p2,p3)."""
        self._add([p0, p1, p2, p3], [(0, 1, 2), (0, 2, 3)], mat,
                  [(*uvs[0], *uvs[1], *uvs[2]), (*uvs[0], *uvs[2], *uvs[3])])

    def mesh(self, verts, tris, mat):
        self._add(verts, tris, mat, (0, 0, 1, 0, 0, 1))

    def box(self, lo, hi, mat):
        x0, y0, z0 = lo
        x1, y1, z1 = hi
        c = [(x0, y0, z0), (x1, y0, z0), (x1, y1, z0), (x0, y1, z0),
             (x0, y0, z1), (x1, y0, z1), (x1, y1, z1), (x0, y1, z1)]
        for a, b, cc, d in ((0, 1, 2, 3), (5, 4, 7, 6), (4, 0, 3, 7),
                            (1, 5, 6, 2), (3, 2, 6, 7), (4, 5, 1, 0)):
            self.quad(c[a], c[b], c[cc], c[d], mat)

    def scene(self) -> Scene:
        c = lambda parts, dt: np.ascontiguousarray(np.concatenate(parts), dtype=dt)  # noqa: E731
        return Scene(c(self.v, F32), c(self.i, np.int32), c(self.m, F32), c(self.uv, F32))


def grey(a: float):
    return (a, a, a, 0.0, a, a, a, 0.0)


def icosphere(subdiv: int):
    """Unit icosphere: 20 * 4**subdiv triangles (soup, shared edges bit-identical)."""
    p = (1.0 + 5.0 ** 0.5) / 2.0
    v = np.array([(-1, p, 0), (1, p, 0), (-1, -p, 0), (1, -p, 0), (0, -1, p), (0, 1, p),
                  (0, -1, -p), (0, 1, -p), (p, 0, -1), (p, 0, 1), (-p, 0, -1), (-p, 0, 1)],
                 np.float64)
    v /= np.linalg.norm(v, axis=1, keepdims=True)
    f = np.array([(0, 11, 5), (0, 5, 1), (0, 1, 7), (0, 7, 10), (0, 10, 11), (1, 5, 9),
                  (5, 11, 4), (11, 10, 2), (10, 7, 6), (7, 1, 8), (3, 9, 4), (3, 4, 2),
                  (3, 2, 6), (3, 6, 8), (3, 8, 9), (4, 9, 5), (2, 4, 11), (6, 2, 10),
                  (8, 6, 7), (9, 8, 1)], np.int64)
    tris = v[f]  # [F,3,3]
    for _ in range(subdiv):
        a, b, c = tris[:, 0], tris[:, 1], tris[:, 2]
        ab, bc, ca = a + b, b + c, c + a  # commutative sums: shared midpoints identical
        ab /= np.linalg.norm(ab, axis=1, keepdims=True)
        bc /= np.linalg.norm(bc, axis=1, keepdims=True)
        ca /= np.linalg.norm(ca, axis=1, keepdims=True)
        tris = np.concatenate([np.stack([a, ab, ca], 1), np.stack([b, bc, ab], 1),
                               np.stack([c, ca, bc], 1), np.stack([ab, bc, ca], 1)])
    return tris  # [20*4^s, 3, 3]


def tiny_scene() -> Scene:
    """Checker background quad (4x4 at z=2, 8x8 cells, albedo 0.2/0.8) and a
    0.3x0.3 occluder at z=0.5 over the lower-right image quarter (albedo 0.6)."""
    b = _Builder()
    b.quad((-2, -2, 2), (2, -2, 2), (2, 2, 2), (-2, 2, 2),
           (0.2, 0.2, 0.2, 8.0, 0.8, 0.8, 0.8, 0.0))
    b.quad((0.0, -0.3, 0.5), (0.3, -0.3, 0.5), (0.3, 0.0, 0.5), (0.0, 0.0, 0.5), grey(0.6))
    return b.scene()


def specular_scene(ks: float = 4.0) -> Scene:
    """Glossy variant of the tiny scene: the checker background quad at z=2 and
    three flat-faceted icospheres (subdivision 3, radius 0.07) at view depths
    0.5 to 0.7, grey albedo 0.3 with Blinn-Phong strength ks: their highlights
    are bright specular bokeh in the near field of a lens focused at 2."""
    b = _Builder()
    b.quad((-2, -2, 2), (2, -2, 2), (2, 2, 2), (-2, 2, 2),
           (0.2, 0.2, 0.2, 8.0, 0.8, 0.8, 0.8, 0.0))
    sphere = icosphere(3)
    for c in ((-0.1, 0.08, 0.57), (0.12, 0.1, 0.67), (0.02, -0.12, 0.77)):
        pts = sphere * 0.07 + np.array(c)
        verts = pts.reshape(-1, 3)
        b.mesh(verts, np.arange(verts.shape[0]).reshape(-1, 3), (0.3, 0.3, 0.3, 0.0, 0.3, 0.3, 0.3, ks))
    return b.scene()


def specular_config():
    """128x128 frame of the glossy scene: focus 2.0, aperture 0.05, 16 spp,
    specular preference 0.5."""
    cam = Camera(width=128, height=128).f32()
    lens = Lens(2.0, 0.05, 0.05).f32()
    params = Params(spp_max=16, variance_on=0, r_max=16.0, seed=0, spec_pref=0.5)
    return specular_scene(), cam, lens, params


def plane_scene(z: float, half: float = 50.0, cells: float = 400.0) -> Scene:
    """Single fronto-parallel checker plane at depth z (Lambert, albedo 0.2/0.8)."""
    b = _Builder()
    b.quad((-half, -half, z), (half, -half, z), (half, half, z), (-half, half, z),
           (0.2, 0.2, 0.2, cells, 0.8, 0.8, 0.8, 0.0))
    return b.scene()


ROOM_LO = (-6.0, -3.0, -0.5)
ROOM_HI = (6.0, 3.0, 8.5)


def room_scene(seed: int = 0, n_boxes: int = 64, n_spheres: int = 32, subdiv: int = 4,
               aspect: float = 16.0 / 9.0, tan_half_fovy: float = math.tan(math.radians(30.0)),
               n_near: int = 8, zmin_range=(0.3, 8.0), near_max: float = 1.0, specular: float = 0.0) -> Scene:
    """Procedural room: 6 walls (12 triangles), axis-aligned boxes with edges in
    U[0.1,1.0] and icospheres with radius U[0.05,0.4].  Objects are shuffled;
    each gets a nearest-extent depth z_min ~ U[zmin_range] (the first ``n_near``
    forced below ``near_max``) and x, y uniform inside the view frustum (camera
    at the origin looking along +z) clipped to the room.  Per-object grey
    albedo U[0.05,0.95]; ``specular`` > 0 gives the spheres that Blinn-Phong
    strength k_s (the random draws, and so the geometry, do not change)."""
    rng = np.random.default_rng(seed)
    b = _Builder()
    (x0, y0, z0), (x1, y1, z1) = ROOM_LO, ROOM_HI
    c = [(x0, y0, z0), (x1, y0, z0), (x1, y1, z0), (x0, y1, z0),
         (x0, y0, z1), (x1, y0, z1), (x1, y1, z1), (x0, y1, z1)]
    for a, bb, cc, d in ((0, 1, 2, 3), (5, 4, 7, 6), (4, 0, 3, 7),
                         (1, 5, 6, 2), (3, 2, 6, 7), (4, 5, 1, 0)):
        b.quad(c[a], c[bb], c[cc], c[d], grey(float(rng.uniform(0.05, 0.95))))
    sphere = icosphere(subdiv)
    kinds = np.array([0] * n_boxes + [1] * n_spheres)
    rng.shuffle(kinds)
    for k, kind in enumerate(kinds):
        if kind == 0:
            size = rng.uniform(0.1, 1.0, 3)
            half = size / 2.0
        else:
            r = rng.uniform(0.05, 0.4)
            half = np.array([r, r, r])
        zmin = rng.uniform(zmin_range[0], near_max) if k < n_near else rng.uniform(*zmin_range)
        zc = zmin + half[2]
        # frustum half-extents at the object's nearest depth, clipped to the room
        hy = min(zmin * tan_half_fovy, y1 - half[1])
        hx = min(zmin * tan_half_fovy * aspect, x1 - half[0])
        cx = rng.uniform(-hx, hx) if hx > 0 else 0.0
        cy = rng.uniform(-hy, hy) if hy > 0 else 0.0
        alb = grey(float(rng.uniform(0.05, 0.95)))
        if kind == 1 and specular > 0:
            alb = alb[:7] + (float(specular),)
        if kind == 0:
            lo = (cx - half[0], cy - half[1], zc - half[2])
            hi = (cx + half[0], cy + half[1], zc + half[2])
            b.box(lo, hi, alb)
        else:
            pts = sphere * half[0] + np.array([cx, cy, zc])
            verts = pts.reshape(-1, 3)
            tris = np.arange(verts.shape[0]).reshape(-1, 3)
            b.mesh(verts, tris, alb)
    return b.scene()


def room4k_scene(seed: int = 0, aspect: float = 16.0 / 9.0) -> Scene:
    """Mixed-precision 4K workload: 512 boxes and 256 subdivision-5 icospheres
    (5,249,036 triangles)."""
    return room_scene(seed=seed, n_boxes=512, n_spheres=256, subdiv=5, aspect=aspect)


def room_scene_target(seed: int, target_tris: int, **kw) -> Scene:
    """Room with 64 boxes and as many subdivision-4 icospheres as bring the
    triangle count closest to ``target_tris`` (batched multi-view workload)."""
    per = 20 * 4 ** 4
    n_sph = max(1, int(round((target_tris - 12 - 64 * 12) / per)))
    return room_scene(seed=seed, n_boxes=64, n_spheres=n_sph, subdiv=4, **kw)


# --------------------------------------------------------------------------
# cameras and configurations
# --------------------------------------------------------------------------


def dyadic_jitter(seed: int, frame: int):
    """Per-frame sub-pixel jitter in [-0.5, 0.5), multiples of 2^-24 (exact in f32)."""
    rng = np.random.default_rng([seed, frame, 0x6a17])
    k = rng.integers(0, 1 << 24, 2)
    return (float(k[0]) / (1 << 24) - 0.5, float(k[1]) / (1 << 24) - 0.5)


def tiny_config():
    """128x128 single frame: focus 2.0, aperture 0.05, 16 spp on the mask."""
    cam = Camera(width=128, height=128).f32()
    lens = Lens(2.0, 0.05, 0.05).f32()
    params = Params(spp_max=16, variance_on=0, r_max=16.0, seed=0)
    return tiny_scene(), cam, lens, params


# f/1.4 on a 35 mm full-frame equivalent: f = 12 mm / tan(30 deg), A = f / (2 * 1.4)
ROOM_FOCAL = 0.012 / math.tan(math.radians(30.0))
ROOM_APERTURE = ROOM_FOCAL / (2.0 * 1.4)


def room_params(**kw) -> Params:
    base = dict(spp_max=8, variance_on=1, r_max=32.0, ema_alpha=0.2,
                light_dir=[[0.4, 1.0, -0.3], [-0.6, 0.5, -0.8]], light_E=[0.8, 0.4])
    base.update(kw)
    return Params(**base)


def room_camera(frame: int, width: int = 1920, height: int = 1080, seed: int = 0,
                step: float = 0.01, jitter: bool = True) -> Camera:
    """Camera of frame k: origin translated by k*step along +x, jittered."""
    j = dyadic_jitter(seed, frame) if jitter else (0.0, 0.0)
    return Camera(pos=(step * frame, 0.0, 0.0), width=width, height=height,
                  jitter=j).f32()


def room_lens() -> Lens:
    return Lens(3.0, ROOM_APERTURE, ROOM_FOCAL).f32()


def room_config(width: int = 1920, height: int = 1080, frames: int = 8, seed: int = 0):
    """Procedural room, 8 consecutive frames with 0.01/frame translation and
    +-0.5 px jitter; focus 3.0, f/1.4-equivalent aperture, 1-8 spp."""
    scene = room_scene(seed=seed, aspect=width / height)
    lens = room_lens()
    cams = [room_camera(k, width, height, seed) for k in range(frames)]
    return scene, cams, lens, room_params()


def look_at(pos, target, up=(0.0, 1.0, 0.0)):
    """Orthonormal (right, up, fwd) for a camera at pos looking at target."""
    p = np.asarray(pos, np.float64)
    f = np.asarray(target, np.float64) - p
    f /= np.linalg.norm(f)
    r = np.cross(np.asarray(up, np.float64), f)
    r /= np.linalg.norm(r)
    u = np.cross(f, r)
    return tuple(r), tuple(u), tuple(f)


# --------------------------------------------------------------------------
# random per-stage buffers (unit tests of single stages)
# --------------------------------------------------------------------------


def random_gbuffer(width: int, height: int, seed: int = 0, n_regions: int = 12,
                   zrange=(0.3, 8.0)):
    """Piecewise-smooth G-buffer: random rectangles of constant unit normal and
    slanted depth over a background, plus colour.  Returns dict of planes
    nd [H,W,4] (nx,ny,nz,z), col [H,W,4] (rgb, 0), mv [H,W,2]."""
    rng = np.random.default_rng(seed)
    H, W = height, width
    yy, xx = np.mgrid[0:H, 0:W].astype(np.float64)
    n = np.zeros((H, W, 3))
    n[..., 2] = -1.0
    z = 6.0 + 0.002 * xx + 0.001 * yy
    col = np.zeros((H, W, 4))
    col[..., :3] = rng.uniform(0.0, 1.0, (H, W, 3)) * 0.2 + 0.4
    for _ in range(n_regions):
        w = int(rng.integers(max(2, W // 10), max(3, W // 2)))
        h = int(rng.integers(max(2, H // 10), max(3, H // 2)))
        x0 = int(rng.integers(-w // 2, W))
        y0 = int(rng.integers(-h // 2, H))
        sl = (slice(max(0, y0), min(H, y0 + h)), slice(max(0, x0), min(W, x0 + w)))
        nn = rng.normal(size=3)
        nn[2] = -abs(nn[2]) - 0.3
        nn /= np.linalg.norm(nn)
        n[sl] = nn
        z0 = rng.uniform(*zrange)
        z[sl] = z0 + rng.uniform(-0.01, 0.01) * (xx[sl] - x0)
        col[sl + (slice(0, 3),)] = rng.uniform(0.0, 1.0, 3)
    nd = np.concatenate([n, z[..., None]], -1).astype(F32)
    mv = rng.uniform(-3.0, 3.0, (H, W, 2)).astype(F32)
    return dict(nd=nd, col=col.astype(F32), mv=mv)


def random_history(width: int, height: int, seed: int = 0, frac_valid: float = 0.7):
    """Random accumulated history planes: near/far (A rgb, B) float4, moments
    float2 (mu1, mu2 >= mu1^2), hlen u8 (0 marks no history)."""
    rng = np.random.default_rng(seed + 7919)
    H, W = height, width
    B = rng.uniform(0.0, 1.0, (H, W)).astype(F32)
    near = np.concatenate([rng.uniform(0, 1, (H, W, 3)) * B[..., None], B[..., None]], -1)
    Bf = (1.0 - B).astype(F32)
    far = np.concatenate([rng.uniform(0, 1, (H, W, 3)) * Bf[..., None], Bf[..., None]], -1)
    mu1 = rng.uniform(0.05, 0.9, (H, W))
    var = rng.uniform(0.0, 0.12, (H, W)) ** 2 * rng.integers(0, 2, (H, W))
    mom = np.stack([mu1, mu1 * mu1 + var], -1)
    hlen = rng.integers(1, 12, (H, W)) * (rng.uniform(size=(H, W)) < frac_valid)
    return dict(near=near.astype(F32), far=far.astype(F32), mom=mom.astype(F32),
                hlen=hlen.astype(np.uint8))


def random_rt(width: int, height: int, spp, seed: int = 0, zf: float = 3.0):
    """Random normalised per-pixel trace output: rt [H,W,12] =
    (C_near rgb, h | C_far rgb, c_near | P_far xyz, c_far), empty layers marked
    by a CoC of -1 (colour 0); untraced pixels (spp == 0) are zero."""
    rng = np.random.default_rng(seed + 104729)
    H, W = height, width
    h = rng.uniform(0, 1, (H, W))
    h[rng.uniform(size=(H, W)) < 0.25] = 0.0
    h[rng.uniform(size=(H, W)) < 0.15] = 1.0
    cn = rng.uniform(0.0, 20.0, (H, W))
    cf = rng.uniform(0.0, 3.0, (H, W))
    Cn = rng.uniform(0, 1, (H, W, 3))
    Cf = rng.uniform(0, 1, (H, W, 3))
    near_empty = h == 0.0
    far_empty = h == 1.0
    Cn[near_empty] = 0.0
    cn[near_empty] = -1.0
    Cf[far_empty] = 0.0
    cf[far_empty] = -1.0
    P = np.stack([rng.uniform(-3, 3, (H, W)), rng.uniform(-2, 2, (H, W)),
                  rng.uniform(zf, 8.0, (H, W))], -1)
    P[far_empty] = 0.0
    rt = np.concatenate([Cn, h[..., None], Cf, cn[..., None], P, cf[..., None]], -1)
    rt[np.asarray(spp) == 0] = 0.0
    return rt.astype(F32)


# --------------------------------------------------------------------------
# differentiable post-path workload
# --------------------------------------------------------------------------


def random_hist_samples(width: int, height: int, seed: int = 0, frac_valid: float = 0.7):
    """History already sampled at reprojected positions, per pixel
    [H,W,12] = (near rgb*B, B_near, far rgb*B, B_far, mu1, mu2, flags, hlen)
    with flags = valid_near + 2 valid_far."""
    rng = np.random.default_rng(seed + 31337)
    H, W = height, width
    Bn = rng.uniform(0.0, 1.0, (H, W))
    hs = np.zeros((H, W, 12))
    hs[..., 0:3] = rng.uniform(0, 1, (H, W, 3)) * Bn[..., None]
    hs[..., 3] = Bn
    hs[..., 4:7] = rng.uniform(0, 1, (H, W, 3)) * (1 - Bn)[..., None]
    hs[..., 7] = 1 - Bn
    mu1 = rng.uniform(0.05, 0.9, (H, W))
    hs[..., 8] = mu1
    hs[..., 9] = mu1 * mu1 + rng.uniform(0.0, 0.1, (H, W)) ** 2
    vn = rng.uniform(size=(H, W)) < frac_valid
    vf = rng.uniform(size=(H, W)) < frac_valid
    hs[..., 10] = vn + 2 * vf
    hs[..., 11] = rng.integers(1, 12, (H, W))
    return hs.astype(F32)


def box_filter(a: np.ndarray, k: int) -> np.ndarray:
    """k x k mean filter with edge replication (input smoothing only)."""
    r = k // 2
    p = np.pad(a, r, mode="edge")
    c = np.cumsum(np.cumsum(p, 0), 1)
    c = np.pad(c, ((1, 0), (1, 0)))
    H, W = a.shape
    return (c[k:k + H, k:k + W] - c[0:H, k:k + W] - c[k:k + H, 0:W] + c[0:H, 0:W]) / (k * k)


def diff_inputs(width: int = 1024, height: int = 1024, seed: int = 0):
    """Colour U[0,1]^3 and depth U[0.3,8] smoothed by a 9x9 box (seeded)."""
    rng = np.random.default_rng(seed)
    col = rng.uniform(0.0, 1.0, (height, width, 3)).astype(F32)
    z = box_filter(rng.uniform(0.3, 8.0, (height, width)), 9).astype(F32)
    return col, z


def diff_config(width: int = 1024, height: int = 1024, seed: int = 0):
    """Differentiable post-path workload: colour/depth of diff_inputs, and a
    100k-triangle room (seed 0) whose trace at the target lens (focus 2.5,
    aperture 0.04) provides the frozen visibility."""
    col, z = diff_inputs(width, height, seed)
    scene = room_scene_target(seed, 100_000, aspect=width / height)
    cam = Camera(width=width, height=height).f32()
    target = Lens(2.5, 0.04, 0.05).f32()
    start = Lens(1.0, 0.02, 0.05).f32()
    params = room_params(r_max=32.0, variance_on=1)
    return col, z, scene, cam, target, start, params


# --------------------------------------------------------------------------
# batched multi-view workload
# --------------------------------------------------------------------------

BATCH_RESOLUTIONS = ((256, 256), (640, 480), (1280, 720), (1920, 1080))
BATCH_TRIS = (50_000, 150_000, 300_000, 500_000)


@dataclass
class BatchView:
    """One view of the batched workload: which room, its size, pose and lens."""
    room: int
    width: int
    height: int
    pos: tuple
    target: tuple
    lens: Lens
    params: Params

    def camera(self, frame: int = 0, step: float = 0.01, seed: int = 10) -> Camera:
        """Pose translated by frame*step along its right axis, jittered per frame."""
        r, u, f = look_at(self.pos, self.target)
        p = tuple(float(a) + frame * step * float(b) for a, b in zip(self.pos, r))
        return Camera(pos=p, right=r, up=u, fwd=f, width=self.width, height=self.height,
                      jitter=dyadic_jitter(seed + 1000 * (self.params.view + 1), frame)).f32()


def batch_scenes(seeds=(10, 11, 12, 13), tris=BATCH_TRIS):
    """Four rooms of 50k-500k triangles (room generator, seeds 10-13)."""
    return [room_scene_target(s, t) for s, t in zip(seeds, tris)]


def batch_views(n_views: int = 64, seed: int = 10, resolutions=BATCH_RESOLUTIONS, n_rooms: int = 4):
    """Views drawn with one generator (seed 10): room uniform over the four,
    resolution uniform over {256^2, 640x480, 1280x720, 1920x1080}, focus
    U[0.5, 6], aperture radius U[0.01, 0.1], 1-16 spp by mask, camera at a
    random point near the room's front looking at a random point 3-6 units in."""
    rng = np.random.default_rng(seed)
    out = []
    for v in range(n_views):
        room = int(rng.integers(n_rooms))
        w, h = resolutions[int(rng.integers(len(resolutions)))]
        pos = (float(rng.uniform(-1.5, 1.5)), float(rng.uniform(-1.0, 1.0)), float(rng.uniform(-0.4, 0.0)))
        target = (float(rng.uniform(-2.0, 2.0)), float(rng.uniform(-1.0, 1.0)), float(rng.uniform(3.0, 6.0)))
        lens = Lens(float(rng.uniform(0.5, 6.0)), float(rng.uniform(0.01, 0.1)), ROOM_FOCAL).f32()
        params = room_params(spp_max=16, view=v, seed=seed)
        out.append(BatchView(room, w, h, pos, target, lens, params))
    return out
