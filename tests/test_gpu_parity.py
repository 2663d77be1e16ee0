"""GPU parity: every C-ABI call against the FP64 oracle on the same seeded
inputs, element by element.

Tolerances: radiance |d| <= 1e-3 on >= 99.9% of pixels (the stated target);
integer outputs (mask bits, spp, hit ids, history length) identical except at
documented ties, where float32 and float64 may legitimately decide
differently: a mask metric within 1e-4 (relative) of its threshold, a ray
within 1e-5 (barycentric) of a triangle edge or two hits at equal t.
"""
import math

import numpy as np
import pytest

import hdof_inputs as hi

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("needs a CUDA device", allow_module_level=True)

import paper_2210_04981_gb300.hdof as H  # noqa: E402
from gpu_util import (bvh_of, check_gbuffer_ids, check_mask_stage, classify_hits, dev, frac_close,  # noqa: E402
                      gbuf_from, history_from, history_host, host, report, reprojection_ties, rt_close,
                      tie_tiles, workspace)

T30 = math.tan(math.radians(30.0))


@pytest.fixture(scope="module")
def orc():
    from oracle import oracle
    oracle.build()
    return oracle


# ------------------------------------------------------------------ BVH ----

def _soup(rng, n):
    c = rng.uniform(-1, 1, (n, 1, 3)) + np.array([0, 0, 4.0])
    v = (c + rng.normal(scale=0.4, size=(n, 3, 3))).astype(np.float32)
    return hi.Scene(v.reshape(-1, 3), np.arange(3 * n).reshape(n, 3).astype(np.int32),
                    np.tile(np.array(hi.grey(0.5), np.float32), (n, 1)), np.zeros((n, 6), np.float32))


def _bary_margin(tv, o, d):
    """Smallest barycentric coordinate of the ray/plane intersection (float64)."""
    v0, v1, v2 = tv[0:3], tv[3:6], tv[6:9]
    e1, e2 = v1 - v0, v2 - v0
    p = np.cross(d, e2)
    det = e1 @ p
    if abs(det) < 1e-300:
        return 0.0
    s = o - v0
    u = (s @ p) / det
    q = np.cross(s, e1)
    v = (d @ q) / det
    return min(1 - u - v, u, v)


@pytest.mark.parametrize("n", [1, 2, 4, 17, 64, 3000])
def test_closest_hits_match_brute_force(orc, n):
    rng = np.random.default_rng(100 + n)
    sc = _soup(rng, n)
    bvh = bvh_of(sc)
    st = bvh.stats()
    assert st.n_tris == n and st.depth < 64
    org = rng.uniform(-0.5, 0.5, (20000, 3)).astype(np.float32)
    d = (rng.uniform(-1.2, 1.2, (20000, 3)) + np.array([0, 0, 4.0]) - org).astype(np.float32)
    ids = torch.empty(20000, dtype=torch.int32, device="cuda")
    ts = torch.empty(20000, dtype=torch.float32, device="cuda")
    H.hdof_closest_hits(bvh, dev(org), dev(d), ids, ts)
    H.hdof_sync()
    g_id, g_t = host(ids), host(ts)
    osc = orc.OScene(sc)
    o_id, o_t = osc.closest_hits(org.astype(np.float64), d.astype(np.float64), use_bvh=(n > 64))
    tv = sc.tri_verts().astype(np.float64)
    bad = []
    for k in np.nonzero(g_id != o_id)[0]:
        o, dd = org[k].astype(np.float64), d[k].astype(np.float64)
        margins = [abs(_bary_margin(tv[t], o, dd)) for t in (g_id[k], o_id[k]) if t >= 0]
        tie_t = g_id[k] >= 0 and o_id[k] >= 0 and abs(g_t[k] - o_t[k]) <= 1e-5 * o_t[k]
        if not (tie_t or (margins and min(margins) < 1e-5)):
            bad.append(k)
    assert not bad, f"{len(bad)} non-tie hit mismatches, e.g. ray {bad[0]}"
    hit = (g_id >= 0) & (g_id == o_id)
    assert np.allclose(g_t[hit], o_t[hit], rtol=1e-5)
    assert (g_id != o_id).mean() < 1e-3


def test_watertight_fan_gpu():
    n = 12
    cen = np.array([0.1, -0.05, 3.0])
    ring = [cen + np.array([math.cos(2 * math.pi * k / n), math.sin(2 * math.pi * k / n), 0.3 * (k % 2)])
            for k in range(n)]
    v = []
    for k in range(n):
        v += [cen, ring[k], ring[(k + 1) % n]]
    v = np.array(v, np.float32)
    sc = hi.Scene(v, np.arange(3 * n).reshape(n, 3).astype(np.int32),
                  np.tile(np.array(hi.grey(0.5), np.float32), (n, 1)), np.zeros((n, 6), np.float32))
    bvh = bvh_of(sc)
    vv = v.astype(np.float64)
    tgt = [vv[0]] + [vv[0] + s * (vv[3 * k + 1] - vv[0]) for k in range(n) for s in np.linspace(0.05, 0.95, 19)]
    tgt = np.array(tgt)
    for o in (np.zeros(3), np.array([0.3, 0.2, -0.1])):
        d = (tgt - o).astype(np.float32)
        ids = torch.empty(len(d), dtype=torch.int32, device="cuda")
        ts = torch.empty(len(d), dtype=torch.float32, device="cuda")
        H.hdof_closest_hits(bvh, dev(np.tile(o, (len(d), 1)).astype(np.float32)), dev(d), ids, ts)
        H.hdof_sync()
        assert np.all(host(ids) >= 0)


# -------------------------------------------------------------- G-buffer ----

def _gbuffer(scene, cam, prev, p, nd_dtype=torch.float32, col_dtype=torch.float32):
    bvh = bvh_of(scene)
    g = H.GBuffer(cam.width, cam.height, nd_dtype=nd_dtype, col_dtype=col_dtype)
    H.hdof_gbuffer(bvh, cam, prev, p, g)
    H.hdof_sync()
    return bvh, g


def test_gbuffer_tiny(orc):
    scene, cam, lens, p = hi.tiny_config()
    _, g = _gbuffer(scene, cam, cam, p)
    ref = orc.gbuffer(orc.OScene(scene), cam, cam, p)
    tri, rtri = host(g.tri), ref["tri"]
    # the background quad's diagonal (i + j = 127) is a shared edge: either triangle is correct
    jj, ii = np.mgrid[0:128, 0:128]
    diag = (ii + jj == 127)
    assert np.array_equal(tri[~diag], rtri[~diag])
    assert set(np.unique(tri[diag])) <= {0, 1}
    assert np.allclose(host(g.nd), ref["nd"], atol=1e-5)
    assert frac_close(host(g.col), ref["col"], 1e-5) == 1.0
    assert np.abs(host(g.mv)).max() < 1e-3


def test_gbuffer_room_moving_camera(orc):
    scene = hi.room_scene(seed=0, aspect=16 / 9)
    cam0 = hi.room_camera(0, 320, 180)
    cam1 = hi.room_camera(1, 320, 180)
    p = hi.room_params()
    _, g = _gbuffer(scene, cam1, cam0, p)
    ref = orc.gbuffer(orc.OScene(scene), cam1, cam0, p)
    tri, rtri = host(g.tri), ref["tri"]
    # every differing id is an epsilon-tie of the primary ray (grazed edge, equal t)
    ties = check_gbuffer_ids(orc, scene, cam1, tri, rtri, "room 320x180")
    same = tri == rtri
    print(f"room 320x180 G-buffer: {ties} hit-id ties of {tri.size} pixels")
    z, rz = host(g.nd)[..., 3], ref["nd"][..., 3]
    assert np.allclose(z[same], rz[same], rtol=1e-5)
    assert frac_close(host(g.col)[same], ref["col"][same], 1e-4, axis=-1) == 1.0
    assert frac_close(host(g.mv)[same], ref["mv"][same], 1e-3, axis=-1) == 1.0


# ------------------------------------------------------------------ mask ----

def _mask(g, hist, p):
    W, Hh = g.width, g.height
    edge = torch.empty((Hh, W), dtype=torch.uint8, device="cuda")
    spp = torch.empty((Hh, W), dtype=torch.uint8, device="cuda")
    H.hdof_mask(g, hist, p, edge, spp, workspace(W, Hh, p))
    H.hdof_sync()
    return host(edge), host(spp)


@pytest.mark.parametrize("seed,W,Hh", [(0, 128, 128), (1, 257, 131), (2, 64, 40)])
def test_mask_random_gbuffer(orc, seed, W, Hh):
    gb = hi.random_gbuffer(W, Hh, seed=seed)
    p = hi.Params(spp_max=8)
    edge, spp = _mask(gbuf_from(gb["nd"], gb["col"], gb["mv"]), None, p)
    ref = orc.mask(gb["nd"].astype(np.float64), gb["mv"].astype(np.float64), p)
    tie, tie_px = tie_tiles(ref["emetric"], p.edge_tau, p.tile, p.dilate)
    assert np.array_equal(edge[~tie], ref["edge"][~tie])
    assert np.array_equal(spp[~tie_px], ref["spp"][~tie_px])
    assert edge.sum() > 0
    if W * Hh > 64 * 64:
        assert (spp == 0).sum() > 0


@pytest.mark.parametrize("tile,dilate,W,Hh", [(1, 0, 67, 45), (7, 2, 150, 97), (24, 1, 301, 77), (16, 0, 96, 64),
                                              (5, 8, 83, 59)])
def test_mask_tile_and_dilation_shapes(orc, tile, dilate, W, Hh):
    """Mask tiles of other sizes and dilation radii (the per-block dilated
    flags span up to 32 x 8 tiles) on ragged images."""
    gb = hi.random_gbuffer(W, Hh, seed=tile + 10 * dilate)
    p = hi.Params(spp_max=8, tile=tile, dilate=dilate)
    edge, spp = _mask(gbuf_from(gb["nd"], gb["col"], gb["mv"]), None, p)
    ref = orc.mask(gb["nd"].astype(np.float64), gb["mv"].astype(np.float64), p)
    tie, tie_px = tie_tiles(ref["emetric"], p.edge_tau, p.tile, p.dilate)
    assert np.array_equal(edge[~tie], ref["edge"][~tie])
    assert np.array_equal(spp[~tie_px], ref["spp"][~tie_px])
    assert edge.sum() > 0 and (spp > 0).sum() > 0


@pytest.mark.parametrize("tile,dilate,W,Hh", [(1, 0, 1, 1), (4, 1, 7, 1), (4, 1, 1, 9), (2, 1, 3, 2), (16, 1, 33, 1),
                                              (16, 1, 1, 40), (3, 2, 27, 5)])
def test_mask_degenerate_shapes(orc, tile, dilate, W, Hh):
    """Single pixels, single rows and columns and other slivers: the edge
    pass's clamp-to-edge at every border (the Gaussian on the input, the
    Sobel on the filtered image) against the oracle."""
    gb = hi.random_gbuffer(W, Hh, seed=W * 31 + Hh)
    p = hi.Params(spp_max=8, tile=tile, dilate=dilate)
    edge, spp = _mask(gbuf_from(gb["nd"], gb["col"], gb["mv"]), None, p)
    ref = orc.mask(gb["nd"].astype(np.float64), gb["mv"].astype(np.float64), p)
    tie, tie_px = tie_tiles(ref["emetric"], p.edge_tau, p.tile, p.dilate)
    assert np.array_equal(edge[~tie], ref["edge"][~tie])
    assert np.array_equal(spp[~tie_px], ref["spp"][~tie_px])


def _reach_ties(nd, lens, t, p, edge_ties):
    """Pixels whose spp may differ in the CoC-scaled mask: within reach + 1
    tiles of a tile whose largest CoC radius lies within 1e-4 tile of a
    multiple of the tile (ceil may round either way), plus the threshold
    ties' tiles."""
    Hh, W = nd.shape[:2]
    T = p.tile
    ntx, nty = (W + T - 1) // T, (Hh + T - 1) // T
    c = lens.aperture_radius * Hh * (lens.focus_dist - nd[..., 3].astype(np.float64)) / (
        nd[..., 3].astype(np.float64) * lens.focus_dist * t)
    r = np.minimum(np.abs(c) / 2, p.r_max)
    rp = np.pad(r, ((0, nty * T - Hh), (0, ntx * T - W)))
    rt = rp.reshape(nty, T, ntx, T).max((1, 3))
    frac = rt / T - np.round(rt / T)
    bad = np.abs(frac) < 1e-4
    tie = np.zeros((nty, ntx), bool)
    for ty, tx in zip(*np.nonzero(bad)):
        k = min(8, max(p.dilate, int(math.ceil(rt[ty, tx] / T)))) + 1
        tie[max(0, ty - k):ty + k + 1, max(0, tx - k):tx + k + 1] = True
    return np.kron(tie, np.ones((T, T), bool))[:Hh, :W] | edge_ties


@pytest.mark.parametrize("tile,dilate,A,W,Hh", [(16, 1, 0.1, 257, 131), (8, 0, 0.05, 200, 120), (5, 2, 0.08, 83, 59)])
def test_mask_coc_scaled(orc, tile, dilate, A, W, Hh):
    """The CoC-scaled mask (each edge tile reaches its pixels' largest CoC
    radius) against the oracle's, on random G-buffers: identical bits outside
    threshold ties and reach-rounding ties; and with mask_coc = 0 the call
    equals hdof_mask."""
    gb = hi.random_gbuffer(W, Hh, seed=tile * 7 + dilate)
    cam = hi.Camera(width=W, height=Hh).f32()
    lens = hi.Lens(3.0, A, 0.05).f32()
    p = hi.Params(spp_max=8, tile=tile, dilate=dilate, r_max=64.0, mask_coc=1)
    g = gbuf_from(gb["nd"], gb["col"], gb["mv"])
    edge = torch.empty((Hh, W), dtype=torch.uint8, device="cuda")
    spp = torch.empty((Hh, W), dtype=torch.uint8, device="cuda")
    H.hdof_mask_coc(g, None, cam, lens, p, edge, spp, workspace(W, Hh, p))
    H.hdof_sync()
    ref = orc.mask(gb["nd"].astype(np.float64), gb["mv"].astype(np.float64), p, lens_=lens,
                   tan_half_fovy=cam.tan_half_fovy)
    tie, tie_px = tie_tiles(ref["emetric"], p.edge_tau, p.tile, p.dilate + 8)
    ties = _reach_ties(gb["nd"], lens, cam.tan_half_fovy, p, tie_px)
    assert np.array_equal(host(edge)[~tie], ref["edge"][~tie])
    assert np.array_equal(host(spp)[~ties], ref["spp"][~ties])
    base = orc.mask(gb["nd"].astype(np.float64), gb["mv"].astype(np.float64), p.replace(mask_coc=0))
    assert (ref["spp"] > 0).sum() >= (base["spp"] > 0).sum()  # the blur can only widen the traced area
    assert not np.any((base["spp"] > 0) & (ref["spp"] == 0))
    p0 = p.replace(mask_coc=0)
    H.hdof_mask_coc(g, None, cam, lens, p0, edge, spp, workspace(W, Hh, p0))
    e2, s2 = _mask(g, None, p0)
    assert np.array_equal(host(edge), e2) and np.array_equal(host(spp), s2)
    with pytest.raises(H.HdofError):
        H.hdof_mask(g, None, p, edge, spp, workspace(W, Hh, p))


def test_mask_variance_term(orc):
    W, Hh = 200, 120
    gb = hi.random_gbuffer(W, Hh, seed=5, n_regions=2)
    hist = hi.random_history(W, Hh, seed=6)
    p = hi.room_params(spp_max=8)
    edge, spp = _mask(gbuf_from(gb["nd"], gb["col"], gb["mv"]), history_from(hist), p)
    ref = orc.mask(gb["nd"].astype(np.float64), gb["mv"].astype(np.float64), p, hist["mom"].astype(np.float64),
                   hist["hlen"])
    tie, tie_px = tie_tiles(ref["emetric"], p.edge_tau, p.tile, p.dilate)
    # nearest-pixel reprojection ties: u within 1e-4 of a half-integer
    ok = ~(tie_px | reprojection_ties(gb["mv"]))
    assert np.array_equal(spp[ok], ref["spp"][ok])
    assert len(np.unique(spp)) > 3  # variance term produced intermediate ray counts


# ----------------------------------------------------------------- trace ----

def _trace(bvh, cam, lens, p, spp_np):
    W, Hh = cam.width, cam.height
    spp = dev(spp_np.astype(np.uint8))
    rt = torch.full((Hh, W, 12), float("nan"), dtype=torch.float32, device="cuda")
    stats = torch.zeros(2, dtype=torch.int32, device="cuda")
    H.hdof_trace(bvh, cam, lens, p, spp, rt, stats, workspace(W, Hh, p))
    H.hdof_sync()
    return host(rt), host(stats)


def test_trace_tiny(orc):
    scene, cam, lens, p = hi.tiny_config()
    osc = orc.OScene(scene)
    g = orc.gbuffer(osc, cam, cam, p)
    spp = orc.mask(g["nd"], g["mv"], p)["spp"]
    bvh = bvh_of(scene)
    rt, stats = _trace(bvh, cam, lens, p, spp)
    ref = orc.trace(osc, cam, lens, p, spp)
    traced = spp > 0
    assert stats[0] == traced.sum() and stats[1] == spp.astype(np.int64).sum()
    assert np.all(np.isnan(rt[~traced]))  # untraced pixels untouched
    ok = rt_close(rt, ref, traced)
    assert ok.mean() >= 0.999, f"{(~ok).sum()} of {ok.size} traced pixels differ; " + report("rt", rt[traced], ref[traced])


def test_trace_room(orc):
    W, Hh = 320, 180
    scene = hi.room_scene(seed=0, aspect=W / Hh)
    cam = hi.room_camera(2, W, Hh)
    lens = hi.room_lens()
    p = hi.room_params(frame=2)
    rng = np.random.default_rng(3)
    spp = (rng.integers(0, 9, (Hh, W)) * (rng.uniform(size=(Hh, W)) < 0.6)).astype(np.uint8)
    bvh = bvh_of(scene)
    rt, stats = _trace(bvh, cam, lens, p, spp)
    ref = orc.trace(orc.OScene(scene), cam, lens, p, spp)
    traced = spp > 0
    ok = rt_close(rt, ref, traced)
    assert ok.mean() >= 0.999, f"{(~ok).sum()} of {ok.size}; " + report("rt", rt[traced], ref[traced])


def test_gbuffer_hint_does_not_change_results():
    """The G-buffer seeded with the previous frame's ids in place (the tri
    plane itself), with arbitrary ids, or with none: the same planes bit for
    bit."""
    W, Hh = 320, 180
    scene = hi.room_scene(seed=2, aspect=W / Hh)
    cams = [hi.room_camera(k, W, Hh) for k in range(2)]
    p = hi.room_params()
    bvh = bvh_of(scene)
    rng = np.random.default_rng(8)
    outs = []
    for mode in ("none", "inplace", "junk"):
        g = H.GBuffer(W, Hh)
        H.hdof_gbuffer(bvh, cams[0], cams[0], p, g)  # frame 0 fills tri
        hint = {"none": None, "inplace": g.tri,
                "junk": dev(rng.integers(-3, scene.n_tris + 9, (Hh, W)).astype(np.int32))}[mode]
        H.hdof_gbuffer(bvh, cams[1], cams[0], p, g, hint=hint)
        H.hdof_sync()
        outs.append([t.clone() for t in (g.nd, g.col, g.mv, g.tri)])
    for o in outs[1:]:
        for a, b in zip(outs[0], o):
            assert torch.equal(a.contiguous().view(torch.uint8), b.contiguous().view(torch.uint8))


def test_trace_hint_does_not_change_results():
    """Seeding the lens rays with the primary hit (or with arbitrary ids,
    out-of-range ones included) gives the same trace bit for bit."""
    W, Hh = 320, 180
    scene = hi.room_scene(seed=1, aspect=W / Hh)
    cam = hi.room_camera(1, W, Hh)
    lens = hi.room_lens()
    p = hi.room_params(frame=1)
    bvh = bvh_of(scene)
    g = H.GBuffer(W, Hh)
    H.hdof_gbuffer(bvh, cam, cam, p, g)
    rng = np.random.default_rng(5)
    spp = dev((rng.integers(0, 9, (Hh, W)) * (rng.uniform(size=(Hh, W)) < 0.7)).astype(np.uint8))
    junk = dev(rng.integers(-5, scene.n_tris + 50, (Hh, W)).astype(np.int32))
    outs = []
    for hint in (None, g.tri, junk):
        rt = torch.zeros((Hh, W, 12), dtype=torch.float32, device="cuda")
        stats = torch.zeros(2, dtype=torch.int32, device="cuda")
        H.hdof_trace(bvh, cam, lens, p, spp, rt, stats, workspace(W, Hh, p), hint=hint)
        H.hdof_sync()
        outs.append(rt)
    assert torch.equal(outs[0].view(torch.int32), outs[1].view(torch.int32))
    assert torch.equal(outs[0].view(torch.int32), outs[2].view(torch.int32))


@pytest.mark.parametrize("aperture", [None, 0.08])
def test_trace_forms_agree(aperture):
    """Warp packets and the ray-level trace (every block size, several refill
    thresholds and queue chunks, with and without the hint) give the same
    trace bit for bit:
    the box test never culls a box that could hold the closest hit, so the
    (t, id) minimum does not depend on the traversal order.  The small
    aperture is the room's (packets by default), 0.08 a wide one."""
    W, Hh = 333, 190
    scene = hi.room_scene(seed=2, aspect=W / Hh)
    cam = hi.room_camera(2, W, Hh)
    lens = hi.room_lens() if aperture is None else hi.Lens(1.5, aperture, 0.05).f32()
    p = hi.room_params(frame=2)
    bvh = bvh_of(scene)
    g = H.GBuffer(W, Hh)
    H.hdof_gbuffer(bvh, cam, cam, p, g)
    rng = np.random.default_rng(6)
    spp = dev((rng.integers(0, 9, (Hh, W)) * (rng.uniform(size=(Hh, W)) < 0.6)).astype(np.uint8))
    outs = []
    for tune, hint in [(None, g.tri), (H.tuning(128, 0), None), (H.tuning(64, 0), g.tri), (H.tuning(256, 0), g.tri),
                       (H.tuning(128, 4), g.tri), (H.tuning(64, 1), None), (H.tuning(256, 32), g.tri),
                       (H.tuning(128, 0, 4), g.tri), (H.tuning(64, 4, 2), g.tri), (H.tuning(256, 8, 16), None)]:
        rt = torch.zeros((Hh, W, 12), dtype=torch.float32, device="cuda")
        stats = torch.zeros(2, dtype=torch.int32, device="cuda")
        H.hdof_trace(bvh, cam, lens, p, spp, rt, stats, workspace(W, Hh, p), hint=hint, tune=tune)
        H.hdof_sync()
        outs.append(rt)
    for o in outs[1:]:
        assert torch.equal(outs[0].view(torch.int32), o.view(torch.int32))


@pytest.mark.parametrize("refill", [0, 4])
def test_trace_watchdog_reports_timeout(refill):
    """A traversal step cap of 1 stops every lens ray after one step (the
    lane or packet gives up and the kernel returns; nothing waits):
    hdof_sync reports HDOF_ETIMEOUT once and clears the status word, and a
    trace with the default cap afterwards is clean."""
    scene, cam, lens, p = hi.tiny_config()
    bvh = bvh_of(scene)
    W, Hh = cam.width, cam.height
    spp = dev(np.full((Hh, W), 4, np.uint8))
    rt = torch.empty((Hh, W, 12), dtype=torch.float32, device="cuda")
    stats = torch.zeros(2, dtype=torch.int32, device="cuda")
    ws = workspace(W, Hh, p)
    tune = H.tuning(128, refill)
    H.hdof_sync()
    H.hdof_trace(bvh, cam, lens, p.replace(trav_cap=1), spp, rt, stats, ws, tune=tune)
    with pytest.raises(H.HdofError) as e:
        H.hdof_sync()
    assert e.value.code == -4
    H.hdof_sync()  # cleared
    H.hdof_trace(bvh, cam, lens, p, spp, rt, stats, ws, tune=tune)
    H.hdof_sync()
    assert int(host(stats)[1]) == 4 * W * Hh


def test_trace_rejects_bad_tuning():
    scene, cam, lens, p = hi.tiny_config()
    bvh = bvh_of(scene)
    spp = dev(np.ones((128, 128), np.uint8))
    rt = torch.zeros((128, 128, 12), dtype=torch.float32, device="cuda")
    for t in (H.tuning(96, 0), H.tuning(128, -2), H.tuning(128, 33)):
        with pytest.raises(H.HdofError):
            H.hdof_trace(bvh, cam, lens, p, spp, rt, None, workspace(128, 128, p), tune=t)


def test_trace_empty_mask():
    scene, cam, lens, p = hi.tiny_config()
    bvh = bvh_of(scene)
    rt, stats = _trace(bvh, cam, lens, p, np.zeros((128, 128), np.uint8))
    assert stats[0] == 0 and stats[1] == 0 and np.all(np.isnan(rt))


# ----------------------------------------------------------- post-filter ----

@pytest.mark.parametrize("seed,W,Hh,rmax,A", [(0, 96, 80, 16.0, 0.05), (1, 203, 97, 32.0, 0.02),
                                              (2, 64, 64, 0.0, 0.05), (3, 150, 70, 8.0, 0.0)])
def test_postfilter(orc, seed, W, Hh, rmax, A):
    gb = hi.random_gbuffer(W, Hh, seed=seed)
    cam = hi.Camera(width=W, height=Hh).f32()
    lens = hi.Lens(3.0, A, 0.05).f32()
    p = hi.Params(r_max=rmax)
    pp = torch.empty((Hh, W, 4), dtype=torch.float32, device="cuda")
    H.hdof_postfilter(gbuf_from(gb["nd"], gb["col"]), cam, lens, p, pp, workspace(W, Hh, p))
    H.hdof_sync()
    ref = orc.postfilter(gb["nd"].astype(np.float64), gb["col"].astype(np.float64), lens, cam.tan_half_fovy, p)
    got = host(pp)
    assert frac_close(got, ref, 1e-4) == 1.0, report("pp", got, ref)


@pytest.mark.parametrize("tilt,far_block", [(0.0, False), (0.004, True)])
def test_postfilter_interior_prefix(orc, tilt, far_block):
    """A smooth near field with radii around 20 px: most of each window lies
    inside every nearby source's disk, so the gather sums those taps from row
    prefixes; the result matches the oracle's tap-by-tap sums (a far block
    adds tiles where the plain loop runs next to interior tiles)."""
    W, Hh = 160, 120
    rng = np.random.default_rng(11)
    yy, xx = np.mgrid[0:Hh, 0:W].astype(np.float64)
    nd = np.zeros((Hh, W, 4))
    nd[..., 2] = -1.0
    nd[..., 3] = 0.8 + tilt * xx
    if far_block:
        nd[40:80, 100:140, 3] = 6.0
    col = np.zeros((Hh, W, 4))
    col[..., :3] = rng.uniform(0.2, 0.9, (Hh, W, 3))
    nd, col = nd.astype(np.float32), col.astype(np.float32)
    cam = hi.Camera(width=W, height=Hh).f32()
    lens = hi.Lens(3.0, 0.2, 0.05).f32()
    p = hi.Params(r_max=32.0)
    pp = torch.empty((Hh, W, 4), dtype=torch.float32, device="cuda")
    H.hdof_postfilter(gbuf_from(nd, col), cam, lens, p, pp, workspace(W, Hh, p))
    H.hdof_sync()
    ref = orc.postfilter(nd.astype(np.float64), col.astype(np.float64), lens, cam.tan_half_fovy, p)
    got = host(pp)
    assert frac_close(got, ref, 1e-4) == 1.0, report("pp", got, ref)


# -------------------------------------------------------- reconstruction ----

def _reconstruct_inputs(W, Hh, seed):
    rng = np.random.default_rng(seed)
    spp = (rng.integers(1, 9, (Hh, W)) * (rng.uniform(size=(Hh, W)) < 0.7)).astype(np.uint8)
    cam0 = hi.Camera(pos=(0.0, 0.0, 0.0), width=W, height=Hh, jitter=hi.dyadic_jitter(seed, 0)).f32()
    cam1 = hi.Camera(pos=(0.03, -0.01, 0.02), width=W, height=Hh, jitter=hi.dyadic_jitter(seed, 1)).f32()
    rt = hi.random_rt(W, Hh, spp, seed=seed)
    gb = hi.random_gbuffer(W, Hh, seed=seed)
    hist = hi.random_history(W, Hh, seed=seed)
    return spp, cam0, cam1, rt, gb, hist


@pytest.mark.parametrize("seed,W,Hh,moved,alpha_k", [(0, 96, 64, 1, 0.0), (1, 131, 77, 0, 0.0), (2, 120, 70, 1, 1.0),
                                                     (3, 64, 48, 0, 0.5)])
def test_reconstruct(orc, seed, W, Hh, moved, alpha_k):
    """Temporal + spatial reconstruction against the oracle, with the fixed
    EMA weight and with per-pixel blend factors (alpha_k > 0)."""
    spp, cam0, cam1, rt, gb, hist = _reconstruct_inputs(W, Hh, seed)
    lens = hi.Lens(3.0, 0.02, 0.05).f32()
    p = hi.room_params(camera_moved=moved, r_s=8.0, alpha_k=alpha_k)
    hin = history_from(hist)
    hout = H.History(W, Hh)
    crt = torch.empty((Hh, W, 4), dtype=torch.float32, device="cuda")
    hacc = torch.empty((Hh, W), dtype=torch.float32, device="cuda")
    crec = torch.empty((Hh, W, 4), dtype=torch.float32, device="cuda")
    g = gbuf_from(gb["nd"], gb["col"], gb["mv"])
    H.hdof_reconstruct(dev(rt), g, dev(spp), cam1, cam0, lens, p, hin, hout, crt, hacc, crec)
    H.hdof_sync()
    f64 = {k: (v.astype(np.float64) if v.dtype != np.uint8 else v) for k, v in hist.items()}
    oh, ocrt, ohacc = orc.temporal(cam1, cam0, p, rt.astype(np.float64), spp, gb["nd"].astype(np.float64),
                                   gb["mv"].astype(np.float64), f64)
    ocrec = orc.spatial(p, ocrt, spp, oh["mom"], oh["hlen"])
    tr = spp > 0
    hl = host(hout.hlen)
    assert np.array_equal(hl[~tr], np.zeros((~tr).sum(), np.uint8))
    hl_ok = hl[tr] == oh["hlen"][tr]
    assert hl_ok.mean() >= 0.999
    sel = tr.copy()
    sel[tr] = hl_ok
    for name, a, b, tol in (("near", host(hout.near), oh["near"], 1e-4), ("far", host(hout.far), oh["far"], 1e-4),
                            ("mom", host(hout.mom), oh["mom"], 1e-4), ("crt", host(crt), ocrt, 1e-4),
                            ("crec", host(crec)[..., :3], ocrec[..., :3], 1e-4)):
        assert frac_close(a[sel], b[sel], tol, 1e-4) >= 0.999, report(name, a[sel], b[sel])
    assert frac_close(host(hacc)[sel], ohacc[sel], 1e-4, axis=None) >= 0.999
    assert np.all(host(crt)[~tr][:, 3] == -1.0)


# --------------------------------------------------------------- composite --

def test_composite(orc):
    W, Hh = 77, 53
    rng = np.random.default_rng(4)
    gb = hi.random_gbuffer(W, Hh, seed=4)
    spp = (rng.integers(1, 9, (Hh, W)) * (rng.uniform(size=(Hh, W)) < 0.5)).astype(np.uint8)
    pp = rng.uniform(0, 1, (Hh, W, 4)).astype(np.float32)
    crt = rng.uniform(0, 1, (Hh, W, 4)).astype(np.float32)
    crt[..., 3] = rng.uniform(0, 4, (Hh, W))
    crec = rng.uniform(0, 1, (Hh, W, 4)).astype(np.float32)
    hacc = rng.uniform(0, 1, (Hh, W)).astype(np.float32)
    cam = hi.Camera(width=W, height=Hh).f32()
    lens = hi.Lens(3.0, 0.03, 0.05).f32()
    p = hi.Params()
    out = torch.empty((Hh, W, 4), dtype=torch.float32, device="cuda")
    H.hdof_composite(gbuf_from(gb["nd"], gb["col"]), dev(spp), dev(pp), dev(crt), dev(crec), dev(hacc), cam, lens, p,
                     out)
    H.hdof_sync()
    ref = orc.composite(gb["nd"], gb["col"], spp, pp, crt, crec, hacc, lens, cam.tan_half_fovy, p, Hh)
    assert frac_close(host(out)[..., :3], ref[..., :3], 1e-5) == 1.0, report("out", host(out), ref)


# ------------------------------------------------------------ full frames --

def _stage_check(orc, scene, cam, p, r, ref, name):
    """The frame's integer decisions stage by stage: G-buffer hit ids against
    the oracle's up to primary-ray epsilon-ties; edge bits and spp against
    the oracle's mask of the GPU's own G-buffer and input history, identical
    outside threshold and reprojection ties.  Prints the tie counts."""
    gt = check_gbuffer_ids(orc, scene, cam, host(r.g.tri), ref["g"]["tri"], name)
    hin = history_host(r.hist[1 - r.cur])
    mt = check_mask_stage(orc, p, host(r.g.nd), host(r.g.mv), host(r.edge), host(r.spp), hin, name)
    spp_eq = float((host(r.spp) == ref["mask"]["spp"]).mean())
    print(f"{name}: {gt} G-buffer hit-id ties, {mt} mask pixels at ties; spp equal to the oracle frame's on "
          f"{spp_eq:.6f} of pixels")


def _frame_check(orc, scene, cam, p, r, ref, name):
    _stage_check(orc, scene, cam, p, r, ref, name)
    out = host(r.out)[..., :3]
    ok = frac_close(out, ref["out"][..., :3], 1e-3)
    assert ok >= 0.999, f"{name}: {ok:.5f} within 1e-3; " + report("out", out, ref["out"][..., :3])


def test_frame_tiny(orc):
    scene, cam, lens, p = hi.tiny_config()
    r = H.Renderer(bvh_of(scene), cam.width, cam.height, p)
    r.frame(cam, cam, lens, p)
    H.hdof_sync()
    ref = orc.frame(orc.OScene(scene), cam, cam, lens, p)
    assert np.array_equal(host(r.spp), ref["mask"]["spp"])
    assert np.array_equal(host(r.edge), ref["mask"]["edge"])
    _frame_check(orc, scene, cam, p, r, ref, "tiny")


def test_room_sequence_8_frames(orc):
    """Procedural room at 480x270, 8 consecutive frames with camera motion,
    jitter and temporal accumulation, against the oracle's own sequence."""
    W, Hh = 480, 270
    scene, cams, lens, p0 = hi.room_config(W, Hh, frames=8)
    osc = orc.OScene(scene)
    r = H.Renderer(bvh_of(scene), W, Hh, p0)
    hist = None
    for k in range(8):
        p = p0.replace(frame=k, camera_moved=int(k > 0))
        prev = cams[k - 1] if k else cams[0]
        r.frame(cams[k], prev, lens, p)
        H.hdof_sync()
        ref = orc.frame(osc, cams[k], prev, lens, p, hist=hist)
        hist = ref["hist"]
        _frame_check(orc, scene, cams[k], p, r, ref, f"frame {k}")


def test_room_1080p_bench_config_sampled(orc):
    """The benchmark's workload and launch configuration (1920x1080 room,
    frames 0 and 1 with history and motion): mask, trace, reconstruction
    and output against the oracle's own frames; the post-filter and the
    composite on 20000 sampled pixels (the oracle's full-window gather)."""
    W, Hh = 1920, 1080
    scene, cams, lens, p0 = hi.room_config(W, Hh, frames=2)
    osc = orc.OScene(scene)
    r = H.Renderer(bvh_of(scene), W, Hh, p0)
    hist = orc.empty_history(W, Hh)
    pix = np.random.default_rng(11).choice(W * Hh, 20000, replace=False).astype(np.int32)
    for k in range(2):
        p = p0.replace(frame=k, camera_moved=int(k > 0))
        prev = cams[k - 1] if k else cams[0]
        r.frame(cams[k], prev, lens, p)
        H.hdof_sync()
        ref = orc.frame(osc, cams[k], prev, lens, p, hist=hist, pp_pix=pix)
        hist = ref["hist"]
        _stage_check(orc, scene, cams[k], p, r, ref, f"1080p frame {k}")
        spp = host(r.spp)
        same = spp == ref["mask"]["spp"]
        tr = (spp > 0) & same
        ok = rt_close(host(r.rt), ref["rt"], tr)
        assert ok.mean() >= 0.999, f"frame {k}: rt {ok.mean():.5f}"
        assert frac_close(host(r.crt)[tr], ref["crt"][tr], 1e-3, 1e-3) >= 0.999
        pp = host(r.pp).reshape(-1, 4)[pix]
        assert frac_close(pp, ref["pp"], 1e-4) >= 0.999, report("pp", pp, ref["pp"])
        out = host(r.out).reshape(-1, 4)[pix][:, :3]
        assert frac_close(out, ref["out"][:, :3], 1e-3) >= 0.999, report("out", out, ref["out"][:, :3])


def test_lens_ray_hit_ids_room_1080p(orc):
    """Visibility ray by ray at the benchmark's workload (1920x1080 room,
    frame 0, packet trace as the benchmark launches it): the closest hit of
    every lens sample of 20000 sampled traced pixels equals the oracle's
    (same pixel, sample, lens point and aim), except at epsilon-ties of the
    float32 ray against the float64 one (a hit within 2^-16 t of an edge, or
    two hits at equal t); hit distances agree to 1e-5 relative on 99.9% of
    the rays and to 1e-3 on all (grazing hits)."""
    W, Hh = 1920, 1080
    scene, cams, lens, p0 = hi.room_config(W, Hh, frames=1)
    cam, p = cams[0], p0.replace(frame=0)
    osc = orc.OScene(scene)
    bvh = bvh_of(scene)
    r = H.Renderer(bvh, W, Hh, p)
    r.frame(cam, cam, lens, p)
    H.hdof_sync()
    n_rays = int(host(r.stats)[1])
    rec = torch.empty((n_rays, 4), dtype=torch.float32, device="cuda")
    ray_off = torch.empty((Hh, W), dtype=torch.int32, device="cuda")
    rt = torch.empty_like(r.rt)
    stats = torch.zeros(2, dtype=torch.int32, device="cuda")
    H.hdof_trace(bvh, cam, lens, p, r.spp, rt, stats, r.ws, rec=rec, ray_off=ray_off, hint=r.g.tri)
    ids = torch.empty(n_rays, dtype=torch.int32, device="cuda")
    ts = torch.empty(n_rays, dtype=torch.float32, device="cuda")
    H.hdof_trace_hits(bvh, cam, p, r.spp, r.ws, ids, ts)
    H.hdof_sync()
    spp = host(r.spp)
    # the second trace reproduces the frame's (untraced pixels are not written)
    assert np.array_equal(host(rt)[spp > 0], host(r.rt)[spp > 0]) and int(host(stats)[1]) == n_rays
    traced = np.nonzero(spp.ravel())[0]
    pick = np.sort(np.random.default_rng(5).choice(traced, min(20000, traced.size), replace=False))
    spp_s = np.zeros_like(spp)
    spp_s.ravel()[pick] = spp.ravel()[pick]
    oids, ots, _, ooff = orc.trace_hits(osc, cam, lens, p, spp_s)
    n = spp.ravel()[pick].astype(np.int64)
    qs = np.repeat(pick, n)
    ss = np.concatenate([np.arange(k) for k in n])
    gidx = host(ray_off).ravel()[qs].astype(np.int64) + ss
    oidx = ooff[qs] + ss
    gid, gt = host(ids)[gidx], host(ts)[gidx]
    oid, ot = oids[oidx], ots[oidx]
    tris = scene.tri_verts().astype(np.float64).reshape(-1, 3, 3)
    bad, ties = classify_hits(tris, lambda k: orc.lens_ray(cam, lens, p, qs[k], ss[k]), gid, oid)
    assert not bad, f"{len(bad)} of {gid.size} lens-ray hit ids differ beyond ties (first: {bad[:5]})"
    hit = (gid == oid) & (oid >= 0)
    rel = np.abs(gt[hit] - ot[hit]) / ot[hit]
    # float32 rays: grazing hits move further along the ray than head-on ones
    assert (rel <= 1e-5).mean() >= 0.999 and rel.max() <= 1e-3, (np.percentile(rel, 99.9), rel.max())
    assert np.all(np.isinf(gt[(gid == oid) & (oid < 0)]))
    assert ties <= 1e-3 * gid.size
    print(f"lens rays 1080p: {gid.size} rays compared, {ties} epsilon-ties, {int((oid < 0).sum())} misses")
