"""ctypes front end of the FP64 CPU oracle (``liboracle.so``).

TEST INFRASTRUCTURE ONLY: the tests, ``__graft_entry__.smoke()`` and the
benchmark's CPU-baseline leg call this; the library never does.  It imports
nothing from the CUDA package.  Inputs are the float32 arrays and records of
``hdof_inputs``, widened exactly to float64.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import sys

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "hdof_oracle.c")
_LIB_PATH = os.path.join(_HERE, "liboracle.so")


def build(force: bool = False, openmp: bool = True) -> str:
    """Compile liboracle.so with the host C compiler (plain C99, FP64)."""
    if not force and os.path.exists(_LIB_PATH) and os.path.getmtime(_LIB_PATH) >= max(
            os.path.getmtime(_SRC), os.path.getmtime(os.path.join(_HERE, "hdof_oracle.h"))):
        return _LIB_PATH
    cmd = ["gcc", "-O2", "-std=c99", "-D_DEFAULT_SOURCE", "-ffp-contract=off", "-fPIC", "-shared",
           _SRC, "-o", _LIB_PATH + ".tmp", "-lm"]
    if openmp:
        cmd.insert(1, "-fopenmp")
    subprocess.check_call(cmd)
    os.replace(_LIB_PATH + ".tmp", _LIB_PATH)
    return _LIB_PATH


class Cam(C.Structure):
    _fields_ = [("pos", C.c_double * 3), ("right", C.c_double * 3), ("up", C.c_double * 3),
                ("fwd", C.c_double * 3), ("tan_half_fovy", C.c_double), ("width", C.c_int32),
                ("height", C.c_int32), ("jitter", C.c_double * 2)]


class Lens(C.Structure):
    _fields_ = [("focus_dist", C.c_double), ("aperture_radius", C.c_double),
                ("focal_length", C.c_double)]


class Params(C.Structure):
    _fields_ = [("gauss_sigma", C.c_double), ("edge_tau", C.c_double), ("tile", C.c_int32),
                ("dilate", C.c_int32), ("spp_max", C.c_int32), ("variance_on", C.c_int32),
                ("var_tau", C.c_double), ("var_scale", C.c_double), ("hlen_young", C.c_int32),
                ("seed", C.c_uint32), ("frame", C.c_int32), ("view", C.c_int32),
                ("k_ambient", C.c_double), ("n_lights", C.c_int32),
                ("light_dir", (C.c_double * 3) * 4), ("light_E", C.c_double * 4),
                ("miss_dist", C.c_double), ("ema_alpha", C.c_double), ("camera_moved", C.c_int32),
                ("r_s", C.c_double), ("var_ref", C.c_double), ("r_max", C.c_double),
                ("kz_rel", C.c_double), ("h_tau", C.c_double), ("alpha_k", C.c_double), ("mask_coc", C.c_int32),
                ("blades", C.c_int32), ("blade_rot", C.c_double), ("aberration", C.c_double),
                ("spec_pref", C.c_double)]


_lib = None


def lib():
    global _lib
    if _lib is None:
        build()
        L = C.CDLL(_LIB_PATH)
        dp, ip, up8, vp = (C.POINTER(C.c_double), C.POINTER(C.c_int32), C.POINTER(C.c_uint8),
                           C.c_void_p)
        u32p = C.POINTER(C.c_uint32)
        L.orc_philox.argtypes = [u32p, u32p, u32p]
        L.orc_philox_limb.argtypes = [u32p, u32p, u32p]
        L.orc_coc.argtypes = [C.c_double, C.POINTER(Lens), C.c_int32, C.c_double]
        L.orc_coc.restype = C.c_double
        L.orc_pinhole_dir.argtypes = [C.POINTER(Cam), C.c_double, C.c_double, dp]
        L.orc_project.argtypes = [C.POINTER(Cam), dp, dp]
        L.orc_project.restype = C.c_int
        L.orc_scene_create.argtypes = [C.c_int32, dp, dp, dp]
        L.orc_scene_create.restype = vp
        L.orc_scene_destroy.argtypes = [vp]
        L.orc_intersect_tri.argtypes = [dp, dp, dp, dp, dp]
        L.orc_intersect_tri.restype = C.c_int32
        L.orc_closest_hit.argtypes = [vp, dp, dp, C.c_int32, dp, dp]
        L.orc_closest_hit.restype = C.c_int32
        L.orc_closest_hits.argtypes = [vp, C.c_int32, dp, dp, C.c_int32, ip, dp]
        L.orc_gbuffer.argtypes = [vp, C.POINTER(Cam), C.POINTER(Cam), C.POINTER(Params), dp, dp, dp, ip]
        L.orc_gaussian_weights.argtypes = [C.c_double, dp]
        L.orc_mask.argtypes = [C.c_int32, C.c_int32, dp, dp, dp, up8, C.POINTER(Params), up8, up8, dp]
        L.orc_mask_coc.argtypes = [C.c_int32, C.c_int32, dp, dp, dp, up8, C.POINTER(Params), C.POINTER(Lens),
                                   C.c_double, up8, up8, dp]
        L.orc_trace.argtypes = [vp, C.POINTER(Cam), C.POINTER(Lens), C.POINTER(Params), up8, dp,
                                C.c_int32, ip]
        L.orc_temporal.argtypes = [C.POINTER(Cam), C.POINTER(Cam), C.POINTER(Params), dp, up8, dp, dp,
                                   dp, dp, dp, up8, dp, dp, dp, up8, dp, dp]
        L.orc_spatial.argtypes = [C.c_int32, C.c_int32, C.POINTER(Params), dp, up8, dp, up8, dp,
                                  C.c_int32, ip]
        L.orc_postfilter.argtypes = [C.c_int32, C.c_int32, C.POINTER(Lens), C.c_double,
                                     C.POINTER(Params), dp, dp, dp, C.c_int32, ip]
        L.orc_composite.argtypes = [C.c_int32, C.c_int32, C.POINTER(Lens), C.c_double,
                                    C.POINTER(Params), dp, dp, up8, dp, dp, dp, dp, dp, dp]
        L.orc_num_threads.restype = C.c_int32
        L.orc_disk_area.argtypes = [C.c_double]
        i64p = C.POINTER(C.c_int64)
        L.orc_trace_records.argtypes = [vp, C.POINTER(Cam), C.POINTER(Lens), C.POINTER(Params), up8, i64p, dp]
        L.orc_replay.argtypes = [C.c_int32, C.c_int32, C.POINTER(Lens), C.c_double, up8, i64p, dp, dp]
        L.orc_temporal_frozen.argtypes = [C.c_int32, C.c_int32, C.POINTER(Params), dp, up8, dp, dp, dp, dp, up8]
        L.orc_disk_area.restype = C.c_double
        L.orc_shaped_area.argtypes = [C.c_double, C.POINTER(Params)]
        L.orc_shaped_area.restype = C.c_double
        L.orc_reference_rt.argtypes = [vp, C.POINTER(Cam), C.POINTER(Lens), C.POINTER(Params), C.c_int32, dp]
        L.orc_lens_ray.argtypes = [C.POINTER(Cam), C.POINTER(Lens), C.POINTER(Params), C.c_int64, C.c_int32, dp, dp,
                                   dp]
        L.orc_trace_hits.argtypes = [vp, C.POINTER(Cam), C.POINTER(Lens), C.POINTER(Params), up8, i64p, ip, dp, dp]
        _lib = L
    return _lib


# --------------------------------------------------------------------------
# marshalling
# --------------------------------------------------------------------------

def _d(a):
    a = np.ascontiguousarray(a, dtype=np.float64)
    return a, a.ctypes.data_as(C.POINTER(C.c_double))


def _u8(a):
    a = np.ascontiguousarray(a, dtype=np.uint8)
    return a, a.ctypes.data_as(C.POINTER(C.c_uint8))


def _i32(a):
    a = np.ascontiguousarray(a, dtype=np.int32)
    return a, a.ctypes.data_as(C.POINTER(C.c_int32))


def cam(c) -> Cam:
    o = Cam()
    o.pos[:] = c.pos
    o.right[:] = c.right
    o.up[:] = c.up
    o.fwd[:] = c.fwd
    o.tan_half_fovy = c.tan_half_fovy
    o.width, o.height = c.width, c.height
    o.jitter[:] = c.jitter
    return o


def lens(l) -> Lens:
    return Lens(l.focus_dist, l.aperture_radius, l.focal_length)


def params(p) -> Params:
    o = Params()
    for name in ("gauss_sigma", "edge_tau", "tile", "dilate", "spp_max", "variance_on", "var_tau",
                 "var_scale", "hlen_young", "seed", "frame", "view", "k_ambient", "miss_dist",
                 "ema_alpha", "camera_moved", "r_s", "var_ref", "r_max", "kz_rel", "h_tau", "alpha_k", "mask_coc",
                 "blades", "blade_rot", "aberration", "spec_pref"):
        setattr(o, name, getattr(p, name))
    lights = p.unit_lights()
    o.n_lights = len(lights)
    for k, (d, e) in enumerate(zip(lights, p.light_E)):
        o.light_dir[k][:] = d
        o.light_E[k] = float(np.float32(e))
    return o


class OScene:
    """Oracle scene: triangle soup + its own object-median BVH."""

    def __init__(self, scene):
        self.n = scene.n_tris
        self._v, pv = _d(scene.tri_verts())
        self._m, pm = _d(scene.mat)
        self._uv, pu = _d(scene.uv)
        self.h = lib().orc_scene_create(self.n, pv, pm, pu)

    def __del__(self):
        if getattr(self, "h", None):
            lib().orc_scene_destroy(self.h)
            self.h = None

    def closest_hits(self, org, dirs, use_bvh=True):
        org, po = _d(np.asarray(org).reshape(-1, 3))
        dirs, pd = _d(np.asarray(dirs).reshape(-1, 3))
        n = org.shape[0]
        ids = np.empty(n, np.int32)
        ts = np.empty(n, np.float64)
        lib().orc_closest_hits(self.h, n, po, pd, int(use_bvh), ids.ctypes.data_as(C.POINTER(C.c_int32)),
                               ts.ctypes.data_as(C.POINTER(C.c_double)))
        return ids, ts


def philox(ctr, key, limb=False):
    c = (C.c_uint32 * 4)(*[int(x) & 0xFFFFFFFF for x in ctr])
    k = (C.c_uint32 * 2)(*[int(x) & 0xFFFFFFFF for x in key])
    o = (C.c_uint32 * 4)()
    (lib().orc_philox_limb if limb else lib().orc_philox)(c, k, o)
    return list(o)


def coc(z, lens_, height, tan_half_fovy):
    return lib().orc_coc(float(z), C.byref(lens(lens_)), int(height), float(tan_half_fovy))


def pinhole_dir(cam_, sx, sy):
    d = (C.c_double * 3)()
    lib().orc_pinhole_dir(C.byref(cam(cam_)), float(sx), float(sy), d)
    return np.array(list(d))


def project(cam_, P):
    Pv = (C.c_double * 3)(*[float(x) for x in P])
    u = (C.c_double * 2)()
    ok = lib().orc_project(C.byref(cam(cam_)), Pv, u)
    return (np.array(list(u)) if ok else None)


def gaussian_weights(sigma):
    w = (C.c_double * 5)()
    lib().orc_gaussian_weights(float(sigma), w)
    return np.array(list(w))


def gbuffer(oscene: OScene, cam_, prev_cam, params_):
    W, H = cam_.width, cam_.height
    nd = np.empty((H, W, 4))
    col = np.empty((H, W, 4))
    mv = np.empty((H, W, 2))
    tri = np.empty((H, W), np.int32)
    lib().orc_gbuffer(oscene.h, C.byref(cam(cam_)), C.byref(cam(prev_cam)), C.byref(params(params_)),
                      _d(nd)[1], _d(col)[1], _d(mv)[1], _i32(tri)[1])
    return dict(nd=nd, col=col, mv=mv, tri=tri)


def mask(nd, mv, params_, hist_mom=None, hist_hlen=None, lens_=None, tan_half_fovy=None):
    """Edge bits, spp and the edge metric; with lens_ (and tan_half_fovy) the
    CoC-scaled mask of params_.mask_coc."""
    H, W = nd.shape[:2]
    nd, pnd = _d(nd)
    mv, pmv = _d(mv)
    edge = np.empty((H, W), np.uint8)
    spp = np.empty((H, W), np.uint8)
    em = np.empty((H, W))
    if hist_mom is not None:
        hm, phm = _d(hist_mom)
        hh, phh = _u8(hist_hlen)
    else:
        phm, phh = None, None
    if lens_ is None:
        lib().orc_mask(W, H, pnd, pmv, phm, phh, C.byref(params(params_)), _u8(edge)[1], _u8(spp)[1],
                       _d(em)[1])
    else:
        lib().orc_mask_coc(W, H, pnd, pmv, phm, phh, C.byref(params(params_)), C.byref(lens(lens_)),
                           float(tan_half_fovy), _u8(edge)[1], _u8(spp)[1], _d(em)[1])
    return dict(edge=edge, spp=spp, emetric=em)


def trace(oscene: OScene, cam_, lens_, params_, spp, pix=None):
    """Per-pixel normalised trace output rt [H,W,12] (or [n_pix,12] for a pixel list)."""
    H, W = cam_.height, cam_.width
    spp, pspp = _u8(spp)
    if pix is None:
        rt = np.empty((H, W, 12))
        lib().orc_trace(oscene.h, C.byref(cam(cam_)), C.byref(lens(lens_)), C.byref(params(params_)),
                        pspp, _d(rt)[1], 0, None)
    else:
        pix, ppix = _i32(pix)
        rt = np.empty((pix.shape[0], 12))
        lib().orc_trace(oscene.h, C.byref(cam(cam_)), C.byref(lens(lens_)), C.byref(params(params_)),
                        pspp, _d(rt)[1], int(pix.shape[0]), ppix)
    return rt


def empty_history(W, H):
    return dict(near=np.zeros((H, W, 4)), far=np.zeros((H, W, 4)), mom=np.zeros((H, W, 2)),
                hlen=np.zeros((H, W), np.uint8))


def temporal(cam_, prev_cam, params_, rt, spp, nd, mv, hist):
    H, W = cam_.height, cam_.width
    out = empty_history(W, H)
    crt = np.empty((H, W, 4))
    hacc = np.empty((H, W))
    args = [_d(rt)[1], _u8(spp)[1], _d(nd)[1], _d(mv)[1]]
    hn, hf, hm, hh = (_d(hist["near"]), _d(hist["far"]), _d(hist["mom"]), _u8(hist["hlen"]))
    lib().orc_temporal(C.byref(cam(cam_)), C.byref(cam(prev_cam)), C.byref(params(params_)), *args,
                       hn[1], hf[1], hm[1], hh[1], _d(out["near"])[1], _d(out["far"])[1],
                       _d(out["mom"])[1], _u8(out["hlen"])[1], _d(crt)[1], _d(hacc)[1])
    return out, crt, hacc


def spatial(params_, crt, spp, mom, hlen, pix=None):
    H, W = spp.shape
    crt, pc = _d(crt)
    spp, ps = _u8(spp)
    mom, pm = _d(mom)
    hlen, ph = _u8(hlen)
    if pix is None:
        crec = np.empty((H, W, 4))
        lib().orc_spatial(W, H, C.byref(params(params_)), pc, ps, pm, ph, _d(crec)[1], 0, None)
    else:
        pix, ppix = _i32(pix)
        crec = np.empty((pix.shape[0], 4))
        lib().orc_spatial(W, H, C.byref(params(params_)), pc, ps, pm, ph, _d(crec)[1],
                          int(pix.shape[0]), ppix)
    return crec


def postfilter(nd, col, lens_, tan_half_fovy, params_, pix=None):
    H, W = nd.shape[:2]
    nd, pnd = _d(nd)
    col, pcol = _d(col)
    if pix is None:
        pp = np.empty((H, W, 4))
        lib().orc_postfilter(W, H, C.byref(lens(lens_)), float(tan_half_fovy), C.byref(params(params_)),
                             pnd, pcol, _d(pp)[1], 0, None)
    else:
        pix, ppix = _i32(pix)
        pp = np.empty((pix.shape[0], 4))
        lib().orc_postfilter(W, H, C.byref(lens(lens_)), float(tan_half_fovy), C.byref(params(params_)),
                             pnd, pcol, _d(pp)[1], int(pix.shape[0]), ppix)
    return pp


def spec_plane(col):
    """The G-buffer's specular part S (col[..., 3]) as the grey colour (S, S, S, S)."""
    s = np.asarray(col, np.float64)[..., 3]
    return np.ascontiguousarray(np.repeat(s[..., None], 4, axis=-1))


def postfilter_spec(nd, col, lens_, tan_half_fovy, params_, pix=None):
    """Specular part of the post-process colour: the post-filter of the
    specular plane (x of the result is S_pp)."""
    return postfilter(nd, spec_plane(col), lens_, tan_half_fovy, params_, pix=pix)


def composite(nd, col, spp, pp, crt, crec, hacc, lens_, tan_half_fovy, params_, height, pp_spec=None):
    """Per-pixel composite of planes of any leading shape (image or pixel list);
    ``height`` is the image height the CoC is measured against; ``pp_spec``
    (the specular part of pp) enables the specular preference of spec_pref."""
    shape = np.asarray(spp).shape
    n = int(np.prod(shape))
    out = np.empty(shape + (4,))
    ps = _d(pp_spec)[1] if pp_spec is not None else None
    lib().orc_composite(n, int(height), C.byref(lens(lens_)), float(tan_half_fovy), C.byref(params(params_)),
                        _d(nd)[1], _d(col)[1], _u8(spp)[1], _d(pp)[1], ps, _d(crt)[1], _d(crec)[1],
                        _d(hacc)[1], _d(out)[1])
    return out


def frame(oscene, cam_, prev_cam, lens_, params_, hist=None, pp_pix=None):
    """One full frame in the paper's order.  ``pp_pix`` restricts the
    post-filter (and therefore the composite) to a pixel list, for frames too
    large for the full O(R_max^2) gather; the composite is then returned only
    at those pixels."""
    W, H = cam_.width, cam_.height
    g = gbuffer(oscene, cam_, prev_cam, params_)
    if hist is None:
        hist = empty_history(W, H)
    m = mask(g["nd"], g["mv"], params_, hist["mom"], hist["hlen"], lens_, cam_.tan_half_fovy)
    rt = trace(oscene, cam_, lens_, params_, m["spp"])
    newh, crt, hacc = temporal(cam_, prev_cam, params_, rt, m["spp"], g["nd"], g["mv"], hist)
    crec = spatial(params_, crt, m["spp"], newh["mom"], newh["hlen"])
    t = cam_.tan_half_fovy
    spec = params_.spec_pref > 0
    if pp_pix is None:
        pp = postfilter(g["nd"], g["col"], lens_, t, params_)
        pps = postfilter_spec(g["nd"], g["col"], lens_, t, params_) if spec else None
        out = composite(g["nd"], g["col"], m["spp"], pp, crt, crec, hacc, lens_, t, params_, H, pp_spec=pps)
    else:
        pp = postfilter(g["nd"], g["col"], lens_, t, params_, pix=pp_pix)
        pps = postfilter_spec(g["nd"], g["col"], lens_, t, params_, pix=pp_pix) if spec else None
        sel = np.asarray(pp_pix)
        flat = lambda a: a.reshape(H * W, *a.shape[2:])[sel]  # noqa: E731
        out = composite(flat(g["nd"]), flat(g["col"]), flat(m["spp"]), pp, flat(crt),
                        flat(crec), flat(hacc), lens_, t, params_, H, pp_spec=pps)
    return dict(g=g, mask=m, rt=rt, hist=newh, crt=crt, hacc=hacc, crec=crec, pp=pp, pp_spec=pps, out=out)


def ray_offsets(spp):
    """Row-major prefix of spp: first ray of each pixel, and the ray count."""
    s = np.asarray(spp, np.int64).ravel()
    off = np.zeros(s.size, np.int64)
    np.cumsum(s[:-1], out=off[1:])
    return off, int(s.sum())


def trace_records(oscene: OScene, cam_, lens_, params_, spp):
    """Per-ray (L rgb, z) of the thin-lens samples (z = inf for a miss)."""
    spp = np.ascontiguousarray(spp, np.uint8)
    off, n = ray_offsets(spp)
    rec = np.zeros((max(n, 1), 4))
    lib().orc_trace_records(oscene.h, C.byref(cam(cam_)), C.byref(lens(lens_)), C.byref(params(params_)),
                            spp.ctypes.data_as(C.POINTER(C.c_uint8)), off.ctypes.data_as(C.POINTER(C.c_int64)),
                            _d(rec)[1])
    return rec, off


def reference_rt(oscene: OScene, cam_, lens_, params_, passes):
    """Full ray-traced thin-lens image [H,W,4]: mean radiance of passes x
    spp_max lens samples per pixel (pass k keyed with frame + k)."""
    out = np.empty((cam_.height, cam_.width, 4))
    lib().orc_reference_rt(oscene.h, C.byref(cam(cam_)), C.byref(lens(lens_)), C.byref(params(params_)),
                           int(passes), _d(out)[1])
    return out


def lens_ray(cam_, lens_, params_, q, smp, weight=False):
    """FP64 origin and unit direction of lens sample smp of pixel q (and its
    aperture weight when asked)."""
    O = (C.c_double * 3)()
    d = (C.c_double * 3)()
    w = C.c_double()
    lib().orc_lens_ray(C.byref(cam(cam_)), C.byref(lens(lens_)), C.byref(params(params_)), int(q), int(smp), O, d,
                       C.byref(w))
    if weight:
        return np.array(list(O)), np.array(list(d)), w.value
    return np.array(list(O)), np.array(list(d))


def trace_hits(oscene: OScene, cam_, lens_, params_, spp):
    """Per-ray closest hits of the thin-lens samples at the row-major ray
    offsets: (ids, t, edge margin, off)."""
    spp = np.ascontiguousarray(spp, np.uint8)
    off, n = ray_offsets(spp)
    ids = np.full(max(n, 1), -1, np.int32)
    ts = np.full(max(n, 1), np.inf)
    mg = np.full(max(n, 1), np.inf)
    lib().orc_trace_hits(oscene.h, C.byref(cam(cam_)), C.byref(lens(lens_)), C.byref(params(params_)),
                         spp.ctypes.data_as(C.POINTER(C.c_uint8)), off.ctypes.data_as(C.POINTER(C.c_int64)),
                         ids.ctypes.data_as(C.POINTER(C.c_int32)), _d(ts)[1], _d(mg)[1])
    return ids[:n], ts[:n], mg[:n], off


def replay(lens_, tan_half_fovy, spp, rec, off):
    H, W = np.asarray(spp).shape
    rt = np.empty((H, W, 12))
    off = np.ascontiguousarray(off, np.int64)
    lib().orc_replay(W, H, C.byref(lens(lens_)), float(tan_half_fovy), _u8(spp)[1],
                     off.ctypes.data_as(C.POINTER(C.c_int64)), _d(rec)[1], _d(rt)[1])
    return rt


def temporal_frozen(params_, rt, spp, hs):
    H, W = np.asarray(spp).shape
    crt = np.empty((H, W, 4))
    hacc = np.empty((H, W))
    mom = np.empty((H, W, 2))
    hlen = np.empty((H, W), np.uint8)
    lib().orc_temporal_frozen(W, H, C.byref(params(params_)), _d(rt)[1], _u8(spp)[1], _d(hs)[1], _d(crt)[1],
                              _d(hacc)[1], _d(mom)[1], _u8(hlen)[1])
    return crt, hacc, mom, hlen


def post_forward(col, z, spp, rec, off, hs, cam_, lens_, params_, pp_pix=None):
    """Differentiable post-path with frozen visibility: replay -> temporal
    (frozen history samples) -> spatial -> post-filter -> composite."""
    H, W = np.asarray(spp).shape
    t = cam_.tan_half_fovy
    nd = np.zeros((H, W, 4))
    nd[..., 2] = -1.0
    nd[..., 3] = z
    col4 = np.zeros((H, W, 4))
    col4[..., :3] = col
    rt = replay(lens_, t, spp, rec, off)
    crt, hacc, mom, hlen = temporal_frozen(params_, rt, spp, hs)
    crec = spatial(params_, crt, spp, mom, hlen)
    pp = postfilter(nd, col4, lens_, t, params_, pix=pp_pix)
    if pp_pix is None:
        out = composite(nd, col4, spp, pp, crt, crec, hacc, lens_, t, params_, H)
    else:
        sel = np.asarray(pp_pix)
        flat = lambda a: a.reshape(H * W, *a.shape[2:])[sel]  # noqa: E731
        out = composite(flat(nd), flat(col4), flat(spp), pp, flat(crt), flat(crec), flat(hacc), lens_, t, params_, H)
    return dict(rt=rt, crt=crt, hacc=hacc, mom=mom, hlen=hlen, crec=crec, pp=pp, out=out)


def post_colour_vjp(col, z, spp, rec, off, hs, cam_, lens_, params_, g):
    """J^T g for J = d out[..., :3] / d col of post_forward (the gradient of
    sum(out * g) in the sharp colour image), by the definition of the
    Jacobian.  For a fixed lens the map is affine in col (every weight
    depends on depth, CoC and the frozen radiance only), so the column of
    pixel q is out(col + e_q) - out(col) exactly, up to FP64 rounding; every
    weight is one scalar for the three channels, so a unit step on all three
    channels of q gives its three columns at once.  H W + 1 forward maps:
    small images only."""
    col = np.asarray(col, np.float64)
    g = np.asarray(g, np.float64)
    H, W = np.asarray(spp).shape

    def out(c):
        return post_forward(c, z, spp, rec, off, hs, cam_, lens_, params_)["out"][..., :3]

    base = out(col)
    vjp = np.zeros((H, W, 3))
    for j in range(H):
        for i in range(W):
            c = col.copy()
            c[j, i, :] += 1.0
            vjp[j, i, :] = ((out(c) - base) * g).sum(axis=(0, 1))
    return vjp


def disk_area(r: float) -> float:
    return lib().orc_disk_area(float(r))


def shaped_area(r: float, params_) -> float:
    """Lattice area of the weighted soft aperture shape of radius r."""
    return lib().orc_shaped_area(float(r), C.byref(params(params_)))


def num_threads() -> int:
    return lib().orc_num_threads()


if __name__ == "__main__":  # pragma: no cover - manual build
    print(build(force="--force" in sys.argv))
