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


# ----------------------------------------------------------- hit-id ties ----

HIT_EPS = 2.0 ** -16  # world-space tie band, relative to max(1, t)


def tri_distance(tv, o, d):
    """Ray (o, d) against the triangle tv [3, 3] (float64): the ray parameter
    where it crosses the triangle's plane, and the signed distance of that
    point from the triangle (minus the distance to the nearest edge inside,
    the distance to the triangle outside)."""
    v0, v1, v2 = tv
    n = np.cross(v1 - v0, v2 - v0)
    nn = float(n @ n)
    den = float(n @ d)
    if nn == 0.0 or abs(den) < 1e-300:
        return np.inf, np.inf
    t = float(n @ (v0 - o)) / den
    P = o + t * d
    vs = (v0, v1, v2)
    b = [float(n @ np.cross(vs[(k + 2) % 3] - vs[(k + 1) % 3], P - vs[(k + 1) % 3])) / nn for k in range(3)]
    if min(b) >= 0.0:
        return t, -min(b[k] * np.sqrt(nn) / np.linalg.norm(vs[(k + 2) % 3] - vs[(k + 1) % 3]) for k in range(3))
    best = np.inf
    for k in range(3):
        a, c = vs[k], vs[(k + 1) % 3]
        e = c - a
        s = min(1.0, max(0.0, float((P - a) @ e) / float(e @ e)))
        best = min(best, float(np.linalg.norm(P - (a + s * e))))
    return t, best


def hit_tie(tris, o, d, gid, oid):
    """Whether a float32 closest hit `gid` and the float64 one `oid` (-1 =
    miss) of the ray (o, d) differ only by an epsilon-tie: the float64 hit
    lies within HIT_EPS * max(1, t) of its triangle's edge (a slightly
    different ray misses it), or the float32 triangle lies within that band
    of the ray no farther than the float64 hit (a grazed edge or two hits at
    equal t)."""
    to = np.inf
    if oid >= 0:
        to, so = tri_distance(tris[oid], o, d)
        if -so <= HIT_EPS * max(1.0, to):
            return True
    if gid >= 0:
        tg, sg = tri_distance(tris[gid], o, d)
        band = HIT_EPS * max(1.0, tg)
        if tg > 0 and sg <= band and (oid < 0 or tg <= to + band):
            return True
    return False


def classify_hits(tris, rays, gids, oids):
    """Indices of the mismatching rays (gids != oids) that are not ties, and
    the number of ties; rays(k) gives the float64 (o, d) of ray k."""
    bad, ties = [], 0
    for k in np.nonzero(gids != oids)[0]:
        o, d = rays(k)
        if hit_tie(tris, o, d, int(gids[k]), int(oids[k])):
            ties += 1
        else:
            bad.append(int(k))
    return bad, ties


# ------------------------------------------------------------ mask ties ----

def tie_tiles(emetric, tau, tile, dilate, tol=1e-4):
    """Pixels whose edge bit may legitimately differ (metric within tol
    (relative) of the threshold), and the pixels whose spp may: inside the
    (dilated) tiles whose edge OR involves such a pixel."""
    Hh, W = emetric.shape
    tie = np.abs(emetric - tau) < tol * max(1.0, tau)
    nty, ntx = (Hh + tile - 1) // tile, (W + tile - 1) // tile
    tt = np.zeros((nty, ntx), bool)
    ys, xs = np.nonzero(tie)
    tt[ys // tile, xs // tile] = True
    dil = np.zeros_like(tt)
    for dy in range(-dilate, dilate + 1):
        for dx in range(-dilate, dilate + 1):
            sh = np.zeros_like(tt)
            sy = slice(max(0, dy), nty + min(0, dy))
            sx = slice(max(0, dx), ntx + min(0, dx))
            ty = slice(max(0, -dy), nty + min(0, -dy))
            tx = slice(max(0, -dx), ntx + min(0, -dx))
            sh[ty, tx] = tt[sy, sx]
            dil |= sh
    return tie, np.kron(dil, np.ones((tile, tile), bool))[:Hh, :W]


def reprojection_ties(mv, tol=1e-4):
    """Pixels whose motion-reprojected position lies within tol of a
    half-integer: the nearest history pixel of the mask's variance term may
    differ between float32 and float64."""
    Hh, W = mv.shape[:2]
    jj, ii = np.mgrid[0:Hh, 0:W]
    ux, uy = ii - mv[..., 0].astype(np.float64), jj - mv[..., 1].astype(np.float64)
    return (np.abs((ux + 0.5) - np.round(ux + 0.5)) < tol) | (np.abs((uy + 0.5) - np.round(uy + 0.5)) < tol)


def check_gbuffer_ids(orc, scene, cam, gtri, otri, name=""):
    """G-buffer hit ids equal the oracle's except at epsilon-ties of the
    primary ray; returns the number of ties."""
    tris = scene.tri_verts().astype(np.float64).reshape(-1, 3, 3)
    W = cam.width
    flat_g, flat_o = gtri.ravel(), otri.ravel()
    o = np.asarray(cam.pos, np.float64)

    def ray(k):
        i, j = k % W, k // W
        d = orc.pinhole_dir(cam, i + 0.5 + cam.jitter[0], j + 0.5 + cam.jitter[1])
        return o, d / np.linalg.norm(d)

    bad, ties = classify_hits(tris, ray, flat_g, flat_o)
    assert not bad, f"{name}: {len(bad)} primary-ray hit ids differ beyond ties, e.g. pixels {bad[:8]}"
    return ties


def check_mask_stage(orc, p, nd, mv, edge, spp, hist_in=None, name=""):
    """The GPU's edge bits and spp equal the oracle's mask of the same
    G-buffer and input history, except at threshold ties (and their tiles)
    and, with the variance term, at reprojection ties.  Returns the number
    of pixels excluded as ties."""
    nd64, mv64 = nd.astype(np.float64), mv.astype(np.float64)
    if hist_in is not None and p.variance_on:
        ref = orc.mask(nd64, mv64, p, hist_in["mom"].astype(np.float64), hist_in["hlen"])
    else:
        ref = orc.mask(nd64, mv64, p)
    tie, tie_px = tie_tiles(ref["emetric"], p.edge_tau, p.tile, p.dilate)
    if p.variance_on:
        tie_px = tie_px | reprojection_ties(mv)
    assert np.array_equal(edge[~tie], ref["edge"][~tie]), f"{name}: edge bits differ outside ties"
    diff = (spp != ref["spp"]) & ~tie_px
    assert not diff.any(), f"{name}: spp differs outside ties at {int(diff.sum())} pixels"
    return int(((spp != ref["spp"]) | (edge != ref["edge"])).sum())


def history_host(h):
    return dict(near=host(h.near), far=host(h.far), mom=host(h.mom), hlen=host(h.hlen))
