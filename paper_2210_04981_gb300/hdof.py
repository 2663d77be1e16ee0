"""Python binding of ``libhdof.so`` (ctypes).

One function per C entry point, with the same name; each marshals torch
tensors (device memory, current stream) and parameter records into the C
structs, calls the library and raises :class:`HdofError` on a non-zero
status.  No step of the frame runs here: every computation is a kernel in
the library.  The library must be built (``paper_2210_04981_gb300.build``);
loading fails loudly when it is missing.
"""
from __future__ import annotations

import ctypes as C
import math
import os

import torch

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libhdof.so")

HDOF_F32, HDOF_F16, HDOF_BF16 = 0, 1, 2
_ERRNAMES = {-1: "EINVAL", -2: "ECUDA", -3: "ENOMEM", -4: "ETIMEOUT", -5: "EUNSUPPORTED"}


class HdofError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"{_ERRNAMES.get(code, code)}: {msg}")
        self.code = code


class hdof_camera(C.Structure):
    _fields_ = [("pos", C.c_float * 3), ("right", C.c_float * 3), ("up", C.c_float * 3),
                ("fwd", C.c_float * 3), ("tan_half_fovy", C.c_float), ("width", C.c_int32),
                ("height", C.c_int32), ("jitter", C.c_float * 2)]


class hdof_lens(C.Structure):
    _fields_ = [("focus_dist", C.c_float), ("aperture_radius", C.c_float),
                ("focal_length", C.c_float)]


class hdof_params(C.Structure):
    _fields_ = [("gauss_sigma", C.c_float), ("edge_tau", C.c_float), ("tile", C.c_int32),
                ("dilate", C.c_int32), ("spp_max", C.c_int32), ("variance_on", C.c_int32),
                ("var_tau", C.c_float), ("var_scale", C.c_float), ("hlen_young", C.c_int32),
                ("seed", C.c_uint32), ("frame", C.c_int32), ("view", C.c_int32),
                ("k_ambient", C.c_float), ("n_lights", C.c_int32),
                ("light_dir", (C.c_float * 3) * 4), ("light_E", C.c_float * 4),
                ("miss_dist", C.c_float), ("trav_cap", C.c_int32), ("ema_alpha", C.c_float),
                ("camera_moved", C.c_int32), ("r_s", C.c_float), ("var_ref", C.c_float),
                ("r_max", C.c_float), ("kz_rel", C.c_float), ("h_tau", C.c_float),
                ("alpha_k", C.c_float), ("mask_coc", C.c_int32), ("blades", C.c_int32), ("blade_rot", C.c_float),
                ("aberration", C.c_float), ("spec_pref", C.c_float)]


class hdof_gbuf(C.Structure):
    _fields_ = [("width", C.c_int32), ("height", C.c_int32), ("dtype_nd", C.c_int32),
                ("dtype_col", C.c_int32), ("nd", C.c_void_p), ("col", C.c_void_p),
                ("mv", C.c_void_p), ("tri", C.c_void_p)]


class hdof_history(C.Structure):
    _fields_ = [("near_acc", C.c_void_p), ("far_acc", C.c_void_p), ("mom", C.c_void_p),
                ("hlen", C.c_void_p)]


class hdof_view(C.Structure):
    _fields_ = [("bvh", C.c_void_p), ("cam", hdof_camera), ("prev", hdof_camera), ("lens", hdof_lens),
                ("params", hdof_params), ("g", hdof_gbuf)] + \
               [(n, C.c_void_p) for n in ("edge", "spp", "rt", "stats", "pp", "crt", "hacc", "crec", "out")] + \
               [("hist_in", hdof_history), ("hist_out", hdof_history), ("workspace", C.c_void_p),
                ("workspace_bytes", C.c_size_t)]


class hdof_tuning(C.Structure):
    _fields_ = [("trace_block", C.c_int32), ("trace_refill", C.c_int32), ("trace_chunk", C.c_int32),
                ("spatial_tile", C.c_int32)]


class hdof_post_state(C.Structure):
    _fields_ = [(n, C.c_void_p) for n in ("rt", "crt", "hacc", "mom", "hlen", "crec", "sp_aux", "pp", "pp_aux",
                                          "out")]


class hdof_kernel_time(C.Structure):
    _fields_ = [("name", C.c_char * 32), ("launches", C.c_int32), ("total_ms", C.c_float)]


class hdof_bvh_stats(C.Structure):
    _fields_ = [("n_tris", C.c_int32), ("n_nodes", C.c_int32), ("depth", C.c_int32),
                ("n_big", C.c_int32), ("device_bytes", C.c_int64)]


_lib = None


def load():
    """Load libhdof.so (raises when it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(f"libhdof.so not found at {LIB_PATH}: build it with "
                           "`python -m paper_2210_04981_gb300.build` (nvcc, sm_103a)")
    L = C.CDLL(LIB_PATH)
    P, vp, i32, sz = C.POINTER, C.c_void_p, C.c_int32, C.c_size_t
    sig = {
        "hdof_version": ([], C.c_char_p),
        "hdof_last_error": ([C.c_char_p, sz], C.c_int),
        "hdof_sync": ([vp], C.c_int),
        "hdof_default_params": ([P(hdof_params)], None),
        "hdof_build_bvh": ([vp, i32, vp, i32, vp, vp, P(vp), vp], C.c_int),
        "hdof_bvh_destroy": ([vp], C.c_int),
        "hdof_bvh_info": ([vp, P(hdof_bvh_stats)], C.c_int),
        "hdof_closest_hits": ([vp, i32, vp, vp, vp, vp, vp], C.c_int),
        "hdof_gbuffer": ([vp, P(hdof_camera), P(hdof_camera), P(hdof_params), vp, P(hdof_gbuf), vp], C.c_int),
        "hdof_workspace_bytes": ([i32, i32, P(hdof_params)], sz),
        "hdof_mask": ([P(hdof_gbuf), P(hdof_history), P(hdof_params), vp, vp, vp, sz, vp], C.c_int),
        "hdof_mask_coc": ([P(hdof_gbuf), P(hdof_history), P(hdof_camera), P(hdof_lens), P(hdof_params), vp, vp, vp,
                           sz, vp], C.c_int),
        "hdof_mask_noalloc": ([P(hdof_gbuf), P(hdof_history), P(hdof_params), vp, vp, vp], C.c_int),
        "hdof_trace": ([vp, P(hdof_camera), P(hdof_lens), P(hdof_params), vp, vp, vp, vp, vp, vp, vp, sz, P(hdof_tuning), vp],
                       C.c_int),
        "hdof_profile": ([i32], C.c_int),
        "hdof_profile_read": ([P(hdof_kernel_time), i32], C.c_int),
        "hdof_probe_fma": ([i32, i32, vp, P(C.c_double), vp], C.c_int),
        "hdof_reference_rt": ([vp, P(hdof_camera), P(hdof_lens), P(hdof_params), i32, vp, vp, vp, sz, vp],
                              C.c_int),
        "hdof_error_map": ([vp, vp, vp, i32, i32, vp, vp, vp], C.c_int),
        "hdof_trace_hits": ([vp, P(hdof_camera), P(hdof_params), vp, vp, sz, vp, vp, vp], C.c_int),
        "hdof_postfilter": ([P(hdof_gbuf), P(hdof_camera), P(hdof_lens), P(hdof_params), vp, vp, sz, vp],
                            C.c_int),
        "hdof_reconstruct": ([vp, P(hdof_gbuf), vp, P(hdof_camera), P(hdof_camera), P(hdof_lens),
                              P(hdof_params), P(hdof_history), P(hdof_history), vp, vp, vp, vp], C.c_int),
        "hdof_composite": ([P(hdof_gbuf), vp, vp, vp, vp, vp, P(hdof_camera), P(hdof_lens), P(hdof_params),
                            vp, vp], C.c_int),
        "hdof_postfilter_spec": ([P(hdof_gbuf), P(hdof_camera), P(hdof_lens), P(hdof_params), vp, vp, sz, vp],
                                 C.c_int),
        "hdof_composite_spec": ([P(hdof_gbuf), vp, vp, vp, vp, vp, vp, P(hdof_camera), P(hdof_lens),
                                 P(hdof_params), vp, vp], C.c_int),
        "hdof_batch_create": ([P(hdof_view), i32, P(hdof_tuning), P(vp), vp], C.c_int),
        "hdof_batch_update": ([vp, P(hdof_view), i32, vp], C.c_int),
        "hdof_batch_render": ([vp, vp], C.c_int),
        "hdof_batch_render_range": ([vp, i32, i32, vp], C.c_int),
        "hdof_batch_bytes": ([vp], sz),
        "hdof_batch_destroy": ([vp], C.c_int),
        "hdof_post_workspace_bytes": ([i32, i32, P(hdof_params)], sz),
        "hdof_post_forward": ([P(hdof_gbuf), vp, vp, vp, vp, P(hdof_camera), P(hdof_lens), P(hdof_params),
                               P(hdof_post_state), vp, sz, vp], C.c_int),
        "hdof_post_backward": ([P(hdof_gbuf), vp, vp, vp, vp, P(hdof_camera), P(hdof_lens), P(hdof_params),
                                P(hdof_post_state), vp, vp, vp, vp, sz, vp], C.c_int),
        "hdof_post_forward_dlens": ([P(hdof_gbuf), vp, vp, vp, vp, P(hdof_camera), vp, P(hdof_params),
                                     P(hdof_post_state), vp, sz, vp], C.c_int),
        "hdof_post_backward_dlens": ([P(hdof_gbuf), vp, vp, vp, vp, P(hdof_camera), vp, P(hdof_params),
                                      P(hdof_post_state), vp, vp, vp, vp, sz, vp], C.c_int),
    }
    for name, (args, res) in sig.items():
        f = getattr(L, name)
        f.argtypes = args
        f.restype = res
    _lib = L
    return L


def exported_symbols():
    """Names of the C entry points this binding declares."""
    return ["hdof_version", "hdof_last_error", "hdof_sync", "hdof_default_params", "hdof_build_bvh",
            "hdof_bvh_destroy", "hdof_bvh_info", "hdof_closest_hits", "hdof_gbuffer", "hdof_workspace_bytes",
            "hdof_mask", "hdof_mask_coc", "hdof_mask_noalloc", "hdof_trace", "hdof_trace_hits", "hdof_reference_rt", "hdof_error_map",
            "hdof_postfilter", "hdof_postfilter_spec", "hdof_reconstruct", "hdof_composite", "hdof_composite_spec",
            "hdof_batch_create", "hdof_batch_update", "hdof_batch_render", "hdof_batch_render_range",
            "hdof_batch_destroy", "hdof_batch_bytes",
            "hdof_post_workspace_bytes", "hdof_post_forward", "hdof_post_backward", "hdof_post_forward_dlens",
            "hdof_post_backward_dlens", "hdof_profile",
            "hdof_profile_read", "hdof_probe_fma"]


def _check(rc):
    if rc != 0:
        buf = C.create_string_buffer(1024)
        load().hdof_last_error(buf, 1024)
        raise HdofError(rc, buf.value.decode(errors="replace"))


def _ptr(t):
    if t is None:
        return None
    if not isinstance(t, torch.Tensor):
        raise TypeError("expected a torch tensor")
    if not t.is_cuda:
        raise ValueError("hdof buffers must be CUDA tensors")
    if not t.is_contiguous():
        raise ValueError("hdof buffers must be contiguous")
    return C.c_void_p(t.data_ptr())


def _stream(stream):
    if stream is None:
        stream = torch.cuda.current_stream()
    return C.c_void_p(stream.cuda_stream)


# ------------------------------------------------------------ records ----

def camera(c) -> hdof_camera:
    o = hdof_camera()
    o.pos[:] = list(c.pos)
    o.right[:] = list(c.right)
    o.up[:] = list(c.up)
    o.fwd[:] = list(c.fwd)
    o.tan_half_fovy = c.tan_half_fovy
    o.width, o.height = int(c.width), int(c.height)
    o.jitter[:] = list(c.jitter)
    return o


def lens(l) -> hdof_lens:
    return hdof_lens(l.focus_dist, l.aperture_radius, l.focal_length)


_PARAM_NAMES = ("gauss_sigma", "edge_tau", "tile", "dilate", "spp_max", "variance_on", "var_tau", "var_scale",
                "hlen_young", "seed", "frame", "view", "k_ambient", "miss_dist", "trav_cap", "ema_alpha",
                "camera_moved", "r_s", "var_ref", "r_max", "kz_rel", "h_tau", "alpha_k", "mask_coc", "blades",
                "blade_rot", "aberration", "spec_pref")


def params(p=None) -> hdof_params:
    """Marshal a parameter record (attributes named as the C fields; light
    directions are normalised here); None gives the library defaults."""
    o = hdof_params()
    load().hdof_default_params(C.byref(o))
    if p is None:
        return o
    for name in _PARAM_NAMES:
        if hasattr(p, name):
            setattr(o, name, getattr(p, name))
    dirs = list(p.light_dir)
    o.n_lights = len(dirs)
    for k, (d, e) in enumerate(zip(dirs, p.light_E)):
        n = math.sqrt(sum(float(x) ** 2 for x in d))
        o.light_dir[k][:] = [float(x) / n for x in d]
        o.light_E[k] = float(e)
    return o


# ------------------------------------------------------------- buffers ---

class GBuffer:
    """Device planes of one frame's G-buffer (torch tensors)."""

    def __init__(self, width, height, device="cuda", nd_dtype=torch.float32, col_dtype=torch.float32):
        self.width, self.height = int(width), int(height)
        self.nd = torch.empty((height, width, 4), dtype=nd_dtype, device=device)
        self.col = torch.empty((height, width, 4), dtype=col_dtype, device=device)
        self.mv = torch.empty((height, width, 2), dtype=torch.float32, device=device)
        self.tri = torch.empty((height, width), dtype=torch.int32, device=device)

    @classmethod
    def from_tensors(cls, nd, col, mv=None, tri=None):
        g = cls.__new__(cls)
        g.height, g.width = int(nd.shape[0]), int(nd.shape[1])
        g.nd, g.col, g.mv, g.tri = nd, col, mv, tri
        return g

    def struct(self) -> hdof_gbuf:
        code = {torch.float32: HDOF_F32, torch.float16: HDOF_F16, torch.bfloat16: HDOF_BF16}
        return hdof_gbuf(self.width, self.height, code[self.nd.dtype], code[self.col.dtype], _ptr(self.nd),
                         _ptr(self.col), _ptr(self.mv), _ptr(self.tri))


class History:
    """Temporal history planes (near, far, mom, hlen)."""

    def __init__(self, width, height, device="cuda"):
        self.near = torch.zeros((height, width, 4), dtype=torch.float32, device=device)
        self.far = torch.zeros((height, width, 4), dtype=torch.float32, device=device)
        self.mom = torch.zeros((height, width, 2), dtype=torch.float32, device=device)
        self.hlen = torch.zeros((height, width), dtype=torch.uint8, device=device)

    @classmethod
    def from_tensors(cls, near, far, mom, hlen):
        h = cls.__new__(cls)
        h.near, h.far, h.mom, h.hlen = near, far, mom, hlen
        return h

    def struct(self) -> hdof_history:
        return hdof_history(_ptr(self.near), _ptr(self.far), _ptr(self.mom), _ptr(self.hlen))

    def reset(self):
        self.hlen.zero_()


class Bvh:
    """Owning wrapper of an hdof_bvh handle."""

    def __init__(self, handle):
        self.handle = handle

    def stats(self) -> hdof_bvh_stats:
        s = hdof_bvh_stats()
        _check(load().hdof_bvh_info(self.handle, C.byref(s)))
        return s

    def close(self):
        if self.handle:
            load().hdof_bvh_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


# ---------------------------------------------------------- entry points --

def hdof_version() -> str:
    return load().hdof_version().decode()


def hdof_sync(stream=None):
    _check(load().hdof_sync(_stream(stream)))


def hdof_profile(on: bool):
    """Switch per-kernel event timing of the compute calls on or off."""
    _check(load().hdof_profile(int(bool(on))))


def hdof_profile_read(max_out=64) -> dict:
    """{kernel name: (launches, summed device ms)} since the previous read."""
    arr = (hdof_kernel_time * max_out)()
    n = load().hdof_profile_read(arr, max_out)
    if n < 0:
        _check(n)
    return {arr[k].name.decode(): (int(arr[k].launches), float(arr[k].total_ms)) for k in range(min(n, max_out))}


def hdof_probe_fma(blocks_per_sm, iters, sink, stream=None) -> float:
    """Enqueue the FMA-throughput probe; returns its FMA lane-instruction count."""
    ops = C.c_double()
    _check(load().hdof_probe_fma(int(blocks_per_sm), int(iters), _ptr(sink), C.byref(ops), _stream(stream)))
    return ops.value


def hdof_workspace_bytes(width, height, p=None) -> int:
    return int(load().hdof_workspace_bytes(int(width), int(height), C.byref(params(p))))


def hdof_build_bvh(verts, idx, mat, uv=None, stream=None) -> Bvh:
    h = C.c_void_p()
    _check(load().hdof_build_bvh(_ptr(verts), int(verts.shape[0]), _ptr(idx), int(idx.shape[0]), _ptr(mat),
                                 _ptr(uv), C.byref(h), _stream(stream)))
    return Bvh(h)


def hdof_closest_hits(bvh: Bvh, org, dirs, ids, ts, stream=None):
    _check(load().hdof_closest_hits(bvh.handle, int(org.shape[0]), _ptr(org), _ptr(dirs), _ptr(ids), _ptr(ts),
                                    _stream(stream)))


def hdof_gbuffer(bvh: Bvh, cam, prev, p, gbuf: GBuffer, stream=None, hint=None):
    """hint (int32 [H][W], e.g. the previous frame's tri plane, possibly
    gbuf.tri itself) optionally seeds each primary ray with a likely hit."""
    _check(load().hdof_gbuffer(bvh.handle, C.byref(camera(cam)), C.byref(camera(prev)), C.byref(params(p)),
                               _ptr(hint), C.byref(gbuf.struct()), _stream(stream)))


def hdof_mask(gbuf: GBuffer, prev_hist, p, edge, spp, workspace, stream=None):
    hs = C.byref(prev_hist.struct()) if prev_hist is not None else None
    _check(load().hdof_mask(C.byref(gbuf.struct()), hs, C.byref(params(p)), _ptr(edge), _ptr(spp),
                            _ptr(workspace), workspace.numel() * workspace.element_size(), _stream(stream)))


def hdof_mask_coc(gbuf: GBuffer, prev_hist, cam, lns, p, edge, spp, workspace, stream=None):
    """hdof_mask whose edge tiles reach their pixels' largest CoC radius when p.mask_coc = 1."""
    _check(load().hdof_mask_coc(C.byref(gbuf.struct()), C.byref(prev_hist.struct()) if prev_hist is not None else None,
                                C.byref(camera(cam)), C.byref(lens(lns)), C.byref(params(p)), _ptr(edge), _ptr(spp),
                                _ptr(workspace), workspace.numel() * workspace.element_size(), _stream(stream)))


def hdof_mask_noalloc(gbuf: GBuffer, prev_hist, p, edge, spp, stream=None):
    """hdof_mask for callers that cannot give the library device memory: the
    tile flags live in a fixed array inside the library (see include/hdof.h)."""
    hs = C.byref(prev_hist.struct()) if prev_hist is not None else None
    _check(load().hdof_mask_noalloc(C.byref(gbuf.struct()), hs, C.byref(params(p)), _ptr(edge), _ptr(spp),
                                    _stream(stream)))


def hdof_trace(bvh: Bvh, cam, lns, p, spp, rt, stats, workspace, stream=None, rec=None, ray_off=None, hint=None,
               tune=None):
    """rec (float [n_rays][4]) and ray_off (int32 [H][W]) optionally receive
    the per-ray hit records (L rgb, z) and each traced pixel's first ray;
    hint (int32 [H][W], the G-buffer's tri plane) optionally seeds each lens
    ray with its pixel's primary hit; tune (hdof_tuning) optionally fixes the
    trace's form and block size (default: chosen from the lens)."""
    _check(load().hdof_trace(bvh.handle, C.byref(camera(cam)), C.byref(lens(lns)), C.byref(params(p)),
                             _ptr(spp), _ptr(hint), _ptr(rt), _ptr(stats), _ptr(rec), _ptr(ray_off), _ptr(workspace),
                             workspace.numel() * workspace.element_size(),
                             C.byref(tune) if tune is not None else None, _stream(stream)))


def hdof_trace_hits(bvh: Bvh, cam, p, spp, workspace, ids, ts=None, stream=None):
    """Per-ray hit ids (int32, -1 = miss) and hit distances of the last
    hdof_trace on this workspace, at that call's ray_off[p] + s."""
    _check(load().hdof_trace_hits(bvh.handle, C.byref(camera(cam)), C.byref(params(p)), _ptr(spp),
                                  _ptr(workspace), workspace.numel() * workspace.element_size(), _ptr(ids),
                                  _ptr(ts), _stream(stream)))


def hdof_reference_rt(bvh: Bvh, cam, lns, p, passes, out, workspace, hint=None, stream=None):
    """Full ray-traced frame: mean radiance of passes x spp_max lens samples per pixel."""
    _check(load().hdof_reference_rt(bvh.handle, C.byref(camera(cam)), C.byref(lens(lns)), C.byref(params(p)),
                                    int(passes), _ptr(hint), _ptr(out), _ptr(workspace),
                                    workspace.numel() * workspace.element_size(), _stream(stream)))


ERR_STATS, ERR_SCRATCH = 8, 8 + 8 * 1024


def hdof_error_map(a, b, stats, region=None, err=None, stream=None):
    """Per-pixel mean |a - b| over rgb into err (optional) and, into the
    device double tensor stats [ERR_SCRATCH], the summary sums."""
    Hh, W = a.shape[:2]
    _check(load().hdof_error_map(_ptr(a), _ptr(b), _ptr(region), int(W), int(Hh), _ptr(err), _ptr(stats),
                                 _stream(stream)))


def error_summary(stats) -> dict:
    """Mean absolute error, RMSE, PSNR (peak 1) and max |d| per channel, over
    all pixels and over the region, from hdof_error_map's stats."""
    v = stats[:ERR_STATS].double().cpu().tolist()

    def one(n, s1, s2, mx):
        if n <= 0:
            return {"pixels": 0}
        mse = s2 / (3 * n)
        return {"pixels": int(n), "mae": s1 / (3 * n), "rmse": mse ** 0.5,
                "psnr_db": (10 * math.log10(1.0 / mse)) if mse > 0 else float("inf"), "max": mx}

    return {"all": one(*v[0:4]), "region": one(*v[4:8])}


def hdof_postfilter(gbuf: GBuffer, cam, lns, p, pp, workspace, stream=None):
    _check(load().hdof_postfilter(C.byref(gbuf.struct()), C.byref(camera(cam)), C.byref(lens(lns)),
                                  C.byref(params(p)), _ptr(pp), _ptr(workspace),
                                  workspace.numel() * workspace.element_size(), _stream(stream)))


def hdof_reconstruct(rt, gbuf: GBuffer, spp, cam, prev, lns, p, hist_in: History, hist_out: History, crt, hacc,
                     crec, stream=None):
    _check(load().hdof_reconstruct(_ptr(rt), C.byref(gbuf.struct()), _ptr(spp), C.byref(camera(cam)),
                                   C.byref(camera(prev)), C.byref(lens(lns)), C.byref(params(p)),
                                   C.byref(hist_in.struct()), C.byref(hist_out.struct()), _ptr(crt), _ptr(hacc),
                                   _ptr(crec), _stream(stream)))


def hdof_composite(gbuf: GBuffer, spp, pp, crt, crec, hacc, cam, lns, p, out, stream=None):
    _check(load().hdof_composite(C.byref(gbuf.struct()), _ptr(spp), _ptr(pp), _ptr(crt), _ptr(crec), _ptr(hacc),
                                 C.byref(camera(cam)), C.byref(lens(lns)), C.byref(params(p)), _ptr(out),
                                 _stream(stream)))


def hdof_postfilter_spec(gbuf: GBuffer, cam, lns, p, pp_spec, workspace, stream=None):
    """Post-filter of the specular plane col.w: pp_spec [H,W,4] = (S_pp x3, alpha)."""
    _check(load().hdof_postfilter_spec(C.byref(gbuf.struct()), C.byref(camera(cam)), C.byref(lens(lns)),
                                       C.byref(params(p)), _ptr(pp_spec), _ptr(workspace),
                                       workspace.numel() * workspace.element_size(), _stream(stream)))


def hdof_composite_spec(gbuf: GBuffer, spp, pp, pp_spec, crt, crec, hacc, cam, lns, p, out, stream=None):
    _check(load().hdof_composite_spec(C.byref(gbuf.struct()), _ptr(spp), _ptr(pp),
                                      _ptr(pp_spec) if pp_spec is not None else None, _ptr(crt), _ptr(crec),
                                      _ptr(hacc), C.byref(camera(cam)), C.byref(lens(lns)), C.byref(params(p)),
                                      _ptr(out), _stream(stream)))


# ---------------------------------------------------------- frame driver --

def frame_priorities():
    """(highest, lowest) stream priority of the device: the frame's critical
    path and its concurrent post-filter."""
    low, high = torch.cuda.Stream.priority_range()
    return high, low


class Renderer:
    """Owns the device buffers of a width x height frame and enqueues the
    paper's per-frame sequence (G-buffer, mask, trace, post-filter,
    reconstruction, composite).  The post-filter needs only the G-buffer
    and has its own workspace region, so it runs on a side stream,
    concurrently with the mask, trace and reconstruction, and the composite
    waits for it.  The frame is forked from the caller's stream onto two
    streams the Renderer owns, the critical path (G-buffer, mask, trace,
    reconstruction, composite) at the highest priority so its kernels get
    the SMs first, the post-filter at the lowest, and joined back to the
    caller's stream at its end.  History is double-buffered and swapped
    after each frame."""

    def __init__(self, bvh: Bvh, width, height, p, device="cuda", nd_dtype=torch.float32,
                 col_dtype=torch.float32):
        self.bvh, self.W, self.H = bvh, int(width), int(height)
        dev = torch.device(device)
        self.g = GBuffer(width, height, dev, nd_dtype, col_dtype)
        self.edge = torch.empty((height, width), dtype=torch.uint8, device=dev)
        self.spp = torch.empty((height, width), dtype=torch.uint8, device=dev)
        self.rt = torch.empty((height, width, 12), dtype=torch.float32, device=dev)
        self.pp = torch.empty((height, width, 4), dtype=torch.float32, device=dev)
        self.crt = torch.empty((height, width, 4), dtype=torch.float32, device=dev)
        self.hacc = torch.empty((height, width), dtype=torch.float32, device=dev)
        self.crec = torch.empty((height, width, 4), dtype=torch.float32, device=dev)
        self.out = torch.empty((height, width, 4), dtype=torch.float32, device=dev)
        self.pp_spec = None  # allocated by the first frame with spec_pref > 0
        self.stats = torch.zeros(2, dtype=torch.int32, device=dev)
        self.hist = [History(width, height, dev), History(width, height, dev)]
        self.cur = 0
        nbytes = hdof_workspace_bytes(width, height, p)
        self.ws = torch.empty(nbytes, dtype=torch.uint8, device=dev)
        high, low = frame_priorities()
        self.crit = torch.cuda.Stream(device=dev, priority=high)  # the frame's critical path
        self.side = torch.cuda.Stream(device=dev, priority=low)  # the post-filter
        self._start = torch.cuda.Event()
        self._gbuf_done = torch.cuda.Event()
        self._pf_done = torch.cuda.Event()
        self._done = torch.cuda.Event()

    @property
    def history(self) -> History:
        """History written by the last frame."""
        return self.hist[self.cur]

    def reset_history(self):
        for h in self.hist:
            h.reset()

    def frame(self, cam, prev, lns, p, stream=None, with_history=True):
        caller = stream if stream is not None else torch.cuda.current_stream(self.out.device)
        main = self.crit
        self._start.record(caller)
        main.wait_event(self._start)
        hin = self.hist[self.cur]
        hout = self.hist[1 - self.cur]
        hdof_gbuffer(self.bvh, cam, prev, p, self.g, main, hint=self.g.tri)
        # the post-filter on the side stream, after the G-buffer (it touches only
        # the workspace's post-filter region)
        self._gbuf_done.record(main)
        self.side.wait_event(self._gbuf_done)
        hdof_postfilter(self.g, cam, lns, p, self.pp, self.ws, self.side)
        self._pf_done.record(self.side)
        hdof_mask_coc(self.g, hin if with_history else None, cam, lns, p, self.edge, self.spp, self.ws, main)
        hdof_trace(self.bvh, cam, lns, p, self.spp, self.rt, self.stats, self.ws, main, hint=self.g.tri)
        hdof_reconstruct(self.rt, self.g, self.spp, cam, prev, lns, p, hin, hout, self.crt, self.hacc,
                         self.crec, main)
        main.wait_event(self._pf_done)
        if p.spec_pref > 0:
            # the specular plane's post-filter uses the whole workspace: after the trace and the post-filter
            if self.pp_spec is None:
                self.pp_spec = torch.empty_like(self.pp)
            hdof_postfilter_spec(self.g, cam, lns, p, self.pp_spec, self.ws, main)
            hdof_composite_spec(self.g, self.spp, self.pp, self.pp_spec, self.crt, self.crec, self.hacc, cam, lns,
                                p, self.out, main)
        else:
            hdof_composite(self.g, self.spp, self.pp, self.crt, self.crec, self.hacc, cam, lns, p, self.out, main)
        self._done.record(main)
        caller.wait_event(self._done)
        self.cur = 1 - self.cur
        return self.out


# ------------------------------------------------------ batched multi-view --

def tuning(trace_block=128, trace_refill=0, trace_chunk=0, spatial_tile=0) -> hdof_tuning:
    t = hdof_tuning()
    t.trace_block, t.trace_refill = int(trace_block), int(trace_refill)
    t.trace_chunk, t.spatial_tile = int(trace_chunk), int(spatial_tile)
    return t


def hdof_batch_create(views, tune=None, stream=None) -> C.c_void_p:
    arr = (hdof_view * len(views))(*views)
    h = C.c_void_p()
    _check(load().hdof_batch_create(arr, len(views), C.byref(tune) if tune is not None else None, C.byref(h),
                                    _stream(stream)))
    return h


def hdof_batch_update(handle, views, stream=None):
    arr = (hdof_view * len(views))(*views)
    _check(load().hdof_batch_update(handle, arr, len(views), _stream(stream)))


def hdof_batch_render(handle, stream=None):
    _check(load().hdof_batch_render(handle, _stream(stream)))


BATCH_STAGES = ("gbuffer", "mask", "compaction", "trace", "postfilter", "reconstruct", "composite")


def hdof_batch_render_range(handle, first, last, stream=None):
    _check(load().hdof_batch_render_range(handle, int(first), int(last), _stream(stream)))


def hdof_batch_destroy(handle):
    _check(load().hdof_batch_destroy(handle))


class Batch:
    """Many views (each its own scene, size, camera, lens and constants)
    rendered by one launch per stage.  Each view owns the buffers of a
    :class:`Renderer` (FP32 planes).  ``frame`` rewrites the device launch
    records for the given cameras/lenses/params (history ping-pong
    included) and enqueues the batched frame; ``render`` only enqueues the
    launches, so it can be captured in a CUDA graph and replayed after each
    ``update``."""

    def __init__(self, bvhs, sizes, ps, tune=None, device="cuda"):
        assert len(bvhs) == len(sizes) == len(ps) and len(bvhs) > 0
        self.bvhs = list(bvhs)
        self.params = list(ps)
        self.views = [Renderer(b, w, h, p, device) for b, (w, h), p in zip(self.bvhs, sizes, ps)]
        self.tune = tune if tune is not None else tuning(trace_refill=-1)  # each view's trace in its default form
        self.handle = None

    def __len__(self):
        return len(self.views)

    def records(self, cams, prevs, lenses, ps):
        out = []
        for r, cam, prev, ln, p in zip(self.views, cams, prevs, lenses, ps):
            hin, hout = r.hist[r.cur], r.hist[1 - r.cur]
            v = hdof_view()
            h = r.bvh.handle
            v.bvh = h.value if isinstance(h, C.c_void_p) else h
            v.cam, v.prev, v.lens, v.params = camera(cam), camera(prev), lens(ln), params(p)
            v.g = r.g.struct()
            for n in ("edge", "spp", "rt", "stats", "pp", "crt", "hacc", "crec", "out"):
                setattr(v, n, _ptr(getattr(r, n)))
            v.hist_in, v.hist_out = hin.struct(), hout.struct()
            v.workspace, v.workspace_bytes = _ptr(r.ws), r.ws.numel()
            out.append(v)
        return out

    def update(self, cams, prevs, lenses, ps, stream=None):
        """Rewrite the launch records for the next frame (creates the handle
        on first use)."""
        recs = self.records(cams, prevs, lenses, ps)
        if self.handle is None:
            self.handle = hdof_batch_create(recs, self.tune, stream)
        else:
            hdof_batch_update(self.handle, recs, stream)

    def render(self, stream=None):
        hdof_batch_render(self.handle, stream)

    def handle_bytes(self) -> int:
        """Bytes of launch records one update uploads."""
        return int(load().hdof_batch_bytes(self.handle))

    def advance(self):
        """Swap every view's history ping-pong after a rendered frame."""
        for r in self.views:
            r.cur = 1 - r.cur

    def frame(self, cams, prevs, lenses, ps, stream=None):
        self.update(cams, prevs, lenses, ps, stream)
        self.render(stream)
        self.advance()
        return [r.out for r in self.views]

    def close(self):
        if self.handle is not None:
            hdof_batch_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:  # pragma: no cover - interpreter shutdown
            pass


# ------------------------------------------------ differentiable post-path --

class PostState:
    """Buffers written by hdof_post_forward and read by hdof_post_backward."""

    def __init__(self, width, height, device="cuda"):
        f = lambda *sh: torch.empty((height, width) + sh, dtype=torch.float32, device=device)  # noqa: E731
        self.rt, self.crt, self.hacc, self.mom = f(12), f(4), f(), f(2)
        self.hlen = torch.empty((height, width), dtype=torch.uint8, device=device)
        self.crec, self.sp_aux, self.pp, self.pp_aux, self.out = f(4), f(4), f(4), f(8), f(4)

    def struct(self) -> hdof_post_state:
        return hdof_post_state(*(_ptr(getattr(self, n)) for n, _ in hdof_post_state._fields_))


def hdof_post_workspace_bytes(width, height, p=None) -> int:
    return int(load().hdof_post_workspace_bytes(int(width), int(height), C.byref(params(p))))


def hdof_post_forward(gbuf: GBuffer, spp, rec, ray_off, hist_samples, cam, lns, p, st: PostState, workspace,
                      stream=None):
    _check(load().hdof_post_forward(C.byref(gbuf.struct()), _ptr(spp), _ptr(rec), _ptr(ray_off), _ptr(hist_samples),
                                    C.byref(camera(cam)), C.byref(lens(lns)), C.byref(params(p)),
                                    C.byref(st.struct()), _ptr(workspace), workspace.numel() * workspace.element_size(),
                                    _stream(stream)))


def hdof_post_backward(gbuf: GBuffer, spp, rec, ray_off, hist_samples, cam, lns, p, st: PostState, grad_out,
                       grad_col, grad_lens, workspace, stream=None):
    _check(load().hdof_post_backward(C.byref(gbuf.struct()), _ptr(spp), _ptr(rec), _ptr(ray_off),
                                     _ptr(hist_samples), C.byref(camera(cam)), C.byref(lens(lns)), C.byref(params(p)),
                                     C.byref(st.struct()), _ptr(grad_out), _ptr(grad_col), _ptr(grad_lens),
                                     _ptr(workspace), workspace.numel() * workspace.element_size(), _stream(stream)))


def _lens_dev(lens_dev):
    if not (lens_dev.is_cuda and lens_dev.dtype == torch.float32 and lens_dev.numel() == 2 and lens_dev.is_contiguous()):
        raise ValueError("lens_dev must be a contiguous float32 CUDA tensor of 2 values (focus, aperture)")
    return _ptr(lens_dev)


def hdof_post_forward_dlens(gbuf: GBuffer, spp, rec, ray_off, hist_samples, cam, lens_dev, p, st: PostState,
                            workspace, stream=None):
    """hdof_post_forward with lens_dev = (focus, aperture) read on the device."""
    _check(load().hdof_post_forward_dlens(C.byref(gbuf.struct()), _ptr(spp), _ptr(rec), _ptr(ray_off),
                                          _ptr(hist_samples), C.byref(camera(cam)), _lens_dev(lens_dev),
                                          C.byref(params(p)), C.byref(st.struct()), _ptr(workspace),
                                          workspace.numel() * workspace.element_size(), _stream(stream)))


def hdof_post_backward_dlens(gbuf: GBuffer, spp, rec, ray_off, hist_samples, cam, lens_dev, p, st: PostState,
                             grad_out, grad_col, grad_lens, workspace, stream=None):
    """hdof_post_backward with lens_dev = (focus, aperture) read on the device."""
    _check(load().hdof_post_backward_dlens(C.byref(gbuf.struct()), _ptr(spp), _ptr(rec), _ptr(ray_off),
                                           _ptr(hist_samples), C.byref(camera(cam)), _lens_dev(lens_dev),
                                           C.byref(params(p)), C.byref(st.struct()), _ptr(grad_out),
                                           _ptr(grad_col), _ptr(grad_lens), _ptr(workspace),
                                           workspace.numel() * workspace.element_size(), _stream(stream)))


class _Lens:
    def __init__(self, zf, A, f):
        self.focus_dist, self.aperture_radius, self.focal_length = zf, A, f


class PostPath:
    """Frozen inputs of the differentiable post-path (depth, mask, hit records,
    history samples) and its buffers; ``HdofPost.apply(col, lens_params, path)``
    is the differentiable call."""

    def __init__(self, z, spp, rec, ray_off, hist_samples, cam, p, focal_length=0.05):
        self.cam, self.p, self.focal = cam, p, focal_length
        H, W = z.shape
        self.nd = torch.zeros((H, W, 4), dtype=torch.float32, device=z.device)
        self.nd[..., 2] = -1.0
        self.nd[..., 3] = z
        self.spp, self.rec, self.ray_off, self.hs = spp, rec, ray_off, hist_samples
        self.st = PostState(W, H, z.device)
        self.ws = torch.empty(hdof_post_workspace_bytes(W, H, p), dtype=torch.uint8, device=z.device)
        self.col4 = torch.zeros((H, W, 4), dtype=torch.float32, device=z.device)

    def new_state(self):
        """A state (and colour plane) of its own, e.g. one per autograd context."""
        H, W = self.spp.shape
        return PostState(W, H, self.spp.device), torch.zeros((H, W, 4), dtype=torch.float32, device=self.spp.device)

    def forward(self, col, zf, A, state=None):
        st, col4 = state if state is not None else (self.st, self.col4)
        col4[..., :3] = col
        g = GBuffer.from_tensors(self.nd, col4)
        hdof_post_forward(g, self.spp, self.rec, self.ray_off, self.hs, self.cam, _Lens(zf, A, self.focal), self.p,
                          st, self.ws)
        return st.out[..., :3]

    def forward_dev(self, col, lens_dev, state=None):
        """forward with lens_dev = device float32 [2] (focus, aperture)."""
        st, col4 = state if state is not None else (self.st, self.col4)
        col4[..., :3] = col
        g = GBuffer.from_tensors(self.nd, col4)
        hdof_post_forward_dlens(g, self.spp, self.rec, self.ray_off, self.hs, self.cam, lens_dev, self.p, st, self.ws)
        return st.out[..., :3]

    def backward_dev(self, grad_out, lens_dev, state=None):
        """backward with lens_dev = device float32 [2] (focus, aperture)."""
        st, col4 = state if state is not None else (self.st, self.col4)
        H, W = self.spp.shape
        g4 = torch.zeros((H, W, 4), dtype=torch.float32, device=grad_out.device)
        g4[..., :3] = grad_out
        gcol = torch.empty_like(g4)
        glens = torch.empty(2, dtype=torch.float32, device=grad_out.device)
        g = GBuffer.from_tensors(self.nd, col4)
        hdof_post_backward_dlens(g, self.spp, self.rec, self.ray_off, self.hs, self.cam, lens_dev, self.p, st, g4,
                                 gcol, glens, self.ws)
        return gcol[..., :3], glens

    def backward(self, grad_out, zf, A, state=None):
        st, col4 = state if state is not None else (self.st, self.col4)
        H, W = self.spp.shape
        g4 = torch.zeros((H, W, 4), dtype=torch.float32, device=grad_out.device)
        g4[..., :3] = grad_out
        gcol = torch.empty_like(g4)
        glens = torch.empty(2, dtype=torch.float32, device=grad_out.device)
        g = GBuffer.from_tensors(self.nd, col4)
        hdof_post_backward(g, self.spp, self.rec, self.ray_off, self.hs, self.cam, _Lens(zf, A, self.focal), self.p,
                           st, g4, gcol, glens, self.ws)
        return gcol[..., :3], glens


class HdofPost(torch.autograd.Function):
    """out = post-path(col [H,W,3], lens_params [2] = (focus, aperture)) with
    the hand-written adjoint of hdof_post_backward.  Each call keeps its own
    forward state for its backward (no forward is re-run).  The lens stays on
    the device (the _dlens calls read it there): no host synchronisation, so
    a forward + backward step can be captured into a CUDA graph."""

    @staticmethod
    def forward(ctx, col, lens_params, path: PostPath):
        lens_dev = lens_params.detach().to(device=col.device, dtype=torch.float32).contiguous()
        state = path.new_state()
        out = path.forward_dev(col.detach().contiguous(), lens_dev, state).clone()
        ctx.path, ctx.lens_dev, ctx.state = path, lens_dev, state
        return out

    @staticmethod
    def backward(ctx, grad_out):
        gcol, glens = ctx.path.backward_dev(grad_out.contiguous().float(), ctx.lens_dev, ctx.state)
        ctx.state = None
        return gcol, glens.to(grad_out.device), None
