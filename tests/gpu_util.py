"""Helpers shared by the GPU parity tests (device transfer, tie-aware
comparison).  Imports the CUDA binding and the oracle; used by tests only."""
import numpy as np
import torch

import paper_2210_04981_gb300.hdof as H

DEV = "cuda"


def dev(a, dtype=None):
    t = torch.from_numpy(np.ascontiguousarray(a))
    if dtype is not None:
        t = t.to(dtype)
    return t.to(DEV)


def host(t):
    return t.detach().float().cpu().numpy() if t.dtype in (torch.float16, torch.bfloat16) else t.detach().cpu().numpy()


def bvh_of(scene):
    return H.hdof_build_bvh(dev(scene.verts), dev(scene.idx), dev(scene.mat), dev(scene.uv))


def gbuf_from(nd, col, mv=None, tri=None, nd_dtype=torch.float32, col_dtype=torch.float32):
    return H.GBuffer.from_tensors(dev(nd.astype(np.float32), nd_dtype), dev(col.astype(np.float32), col_dtype),
                                  None if mv is None else dev(mv.astype(np.float32)),
                                  None if tri is None else dev(tri.astype(np.int32)))


def history_from(h):
    return H.History.from_tensors(dev(h["near"].astype(np.float32)), dev(h["far"].astype(np.float32)),
                                  dev(h["mom"].astype(np.float32)), dev(h["hlen"].astype(np.uint8)))


def workspace(W, Hh, p):
    return torch.empty(H.hdof_workspace_bytes(W, Hh, p), dtype=torch.uint8, device=DEV)


def frac_close(a, b, atol, rtol=0.0, axis=-1):
    """Fraction of pixels whose every channel satisfies |a-b| <= atol + rtol |b|."""
    ok = np.abs(a - b) <= atol + rtol * np.abs(b)
    if ok.ndim > 2 and axis is not None:
        ok = ok.all(axis=axis)
    return float(ok.mean())


def report(name, a, b):
    d = np.abs(a - b)
    return f"{name}: max |d| = {d.max():.3e}, 99.9th pct = {np.percentile(d, 99.9):.3e}"


def rt_close(rt, ref, traced):
    """Per traced pixel: colours 1e-3, hit ratio 1e-4, CoC 1e-3 rel, position 1e-4 rel."""
    a, b = rt[traced], ref[traced]
    col = np.r_[0:3, 4:7]
    ok = np.all(np.abs(a[:, col] - b[:, col]) <= 1e-3, axis=1)
    ok &= np.abs(a[:, 3] - b[:, 3]) <= 1e-4
    ok &= np.all(np.abs(a[:, [7, 11]] - b[:, [7, 11]]) <= 1e-3 * np.maximum(1, np.abs(b[:, [7, 11]])), axis=1)
    ok &= np.all(np.abs(a[:, 8:11] - b[:, 8:11]) <= 1e-4 * np.maximum(1, np.abs(b[:, 8:11])), axis=1)
    return ok
