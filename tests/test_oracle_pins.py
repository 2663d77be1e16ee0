"""Pins of the FP64 oracle to facts outside itself (CPU only).

Each test checks the oracle against something the paper, the thin-lens
geometry or plain mathematics fixes: the closed-form CoC against a ray
construction, the ray-traced image of a fronto-parallel plane against an
exact disk convolution (test_oracle_pins_stages.py), BVH closest hits against brute force,
filter identities on constant and linear images, and the stage invariants.
"""
import math

import numpy as np
import pytest

import hdof_inputs as hi

SQRT2 = math.sqrt(2.0)


# ---------------------------------------------------------------- Philox ----

def test_philox_two_formulations_agree(orc):
    rng = np.random.default_rng(1)
    for _ in range(500):
        ctr = rng.integers(0, 2 ** 32, 4, dtype=np.uint64)
        key = rng.integers(0, 2 ** 32, 2, dtype=np.uint64)
        assert orc.philox(ctr, key) == orc.philox(ctr, key, limb=True)
    for ctr in ([0, 0, 0, 0], [2 ** 32 - 1] * 4):
        for key in ([0, 0], [2 ** 32 - 1] * 2):
            assert orc.philox(ctr, key) == orc.philox(ctr, key, limb=True)


def test_philox_uniform_and_avalanche(orc):
    n = 1 << 14
    u = np.array([orc.philox([i, 0, 0, 0], [0, 0])[0] >> 8 for i in range(n)], np.float64) / 2 ** 24
    hist, _ = np.histogram(u, bins=64, range=(0, 1))
    chi2 = ((hist - n / 64) ** 2 / (n / 64)).sum()
    assert chi2 < 120  # 63 dof: p(chi2 > 120) ~ 1e-5
    assert abs(u.mean() - 0.5) < 0.01
    rng = np.random.default_rng(2)
    flips = []
    for _ in range(200):
        ctr = [int(x) for x in rng.integers(0, 2 ** 32, 4)]
        key = [int(x) for x in rng.integers(0, 2 ** 32, 2)]
        a = orc.philox(ctr, key)
        w, b = rng.integers(0, 4), rng.integers(0, 32)
        ctr[w] ^= 1 << int(b)
        c = orc.philox(ctr, key)
        flips.append(sum(bin(x ^ y).count("1") for x, y in zip(a, c)))
    assert 62 < np.mean(flips) < 66  # half of 128 output bits


# ------------------------------------------------------------------- CoC ----

def test_coc_worked_value(orc):
    _, cam, lens, _ = hi.tiny_config()
    c = orc.coc(0.5, lens, 128, cam.tan_half_fovy)
    # 0.05 * 128 * 1.5 / (0.5 * 2 * tan 30deg) = 16.6277
    assert abs(c - 0.05 * 128 * 1.5 / (0.5 * 2.0 * math.tan(math.radians(30)))) < 1e-6
    assert abs(c - 16.6277) < 1e-4
    assert orc.coc(2.0, lens, 128, cam.tan_half_fovy) == 0.0


@pytest.mark.parametrize("z", [0.3, 0.7, 1.9, 2.0, 2.5, 7.0, 40.0])
def test_coc_closed_form_matches_lens_ray_construction(orc, z):
    """Fact 1: the two extreme lens rays through a point at depth z land on
    the focus plane at points whose pinhole pixels are |c(z)| apart."""
    W, H = 96, 64
    cam = hi.Camera(width=W, height=H)
    for zf, A in ((2.0, 0.05), (3.0, 0.0074), (0.8, 0.1)):
        lens = hi.Lens(zf, A, 0.05)
        Q = np.array([0.11 * z, -0.07 * z, z])
        xs = []
        for xl in (-A, A):
            O = np.array([xl, 0.0, 0.0])
            Pf = O + (Q - O) * (zf / z)  # the lens ray through Q, at depth zf
            xs.append(orc.project(cam, Pf)[0])
        spread = abs(xs[1] - xs[0])
        assert abs(spread - abs(orc.coc(z, lens, H, cam.tan_half_fovy))) < 1e-9 * max(1.0, spread)
        # sign: near (z < zf) positive
        assert (orc.coc(z, lens, H, cam.tan_half_fovy) > 0) == (z < zf) or z == zf


def test_project_inverts_pinhole_dir(orc):
    cam = hi.Camera(pos=(0.3, -0.2, 0.1), width=64, height=48, jitter=(0.25, -0.125))
    r, u, f = hi.look_at(cam.pos, (1.0, 0.5, 4.0))
    cam = hi.Camera(pos=cam.pos, right=r, up=u, fwd=f, width=64, height=48, jitter=(0.25, -0.125))
    for (i, j, z) in ((0, 0, 1.0), (13, 7, 3.3), (63, 47, 0.4)):
        d = orc.pinhole_dir(cam, i + 0.5 + 0.25, j + 0.5 - 0.125)
        P = np.array(cam.pos) + z * d
        uv = orc.project(cam, P)
        assert abs(uv[0] - i) < 1e-9 and abs(uv[1] - j) < 1e-9
        assert abs(np.dot(d, f) - 1.0) < 1e-12


# ------------------------------------------------------ closest hit / BVH ---

def _soup(rng, n):
    c = rng.uniform(-1, 1, (n, 1, 3)) + np.array([0, 0, 4.0])
    v = c + rng.normal(scale=0.4, size=(n, 3, 3))
    idx = np.arange(3 * n).reshape(n, 3)
    return hi.Scene(v.reshape(-1, 3).astype(np.float32), idx.astype(np.int32),
                    np.tile(np.array(hi.grey(0.5), np.float32), (n, 1)),
                    np.zeros((n, 6), np.float32))


@pytest.mark.parametrize("n", [1, 4, 17, 64])
def test_bvh_equals_brute_force(orc, n):
    """Fact 3: the oracle's BVH returns the brute-force closest hit."""
    rng = np.random.default_rng(n)
    osc = orc.OScene(_soup(rng, n))
    org = rng.uniform(-0.5, 0.5, (4000, 3))
    d = rng.uniform(-1.2, 1.2, (4000, 3)) + np.array([0, 0, 4.0]) - org
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    a_id, a_t = osc.closest_hits(org, d, use_bvh=True)
    b_id, b_t = osc.closest_hits(org, d, use_bvh=False)
    assert np.array_equal(a_id, b_id)
    assert np.array_equal(a_t[a_id >= 0], b_t[b_id >= 0])
    assert (a_id >= 0).mean() > (0.05 if n >= 17 else 0.0)


def test_brute_force_is_closest_hit(orc):
    """Closest hit by brute force = the per-triangle test minimised over t."""
    rng = np.random.default_rng(9)
    sc = _soup(rng, 12)
    osc = orc.OScene(sc)
    tv = sc.tri_verts().astype(np.float64)
    import ctypes as C
    for _ in range(300):
        o = rng.uniform(-0.5, 0.5, 3)
        d = rng.normal(size=3)
        d[2] = abs(d[2]) + 0.5
        d /= np.linalg.norm(d)
        best, bt = -1, np.inf
        for k in range(12):
            t = C.c_double()
            b = (C.c_double * 3)()
            hit = orc.lib().orc_intersect_tri((C.c_double * 3)(*o), (C.c_double * 3)(*d),
                                              (C.c_double * 9)(*tv[k]), C.byref(t), b)
            if hit:
                assert abs(sum(b) - 1.0) < 1e-12 and min(b) >= 0.0
                P = sum(b[m] * tv[k][3 * m:3 * m + 3] for m in range(3))
                assert np.allclose(o + t.value * d, P, atol=1e-9)
                if t.value < bt:
                    best, bt = k, t.value
        ids, ts = osc.closest_hits(o, d, use_bvh=False)
        assert ids[0] == best


def test_watertight_fan(orc):
    """Rays aimed exactly at shared edges and the shared vertex of a fan never
    fall through the mesh."""
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
    osc = orc.OScene(sc)
    vv = v.astype(np.float64)
    tgt = [vv[0]]
    for k in range(n):
        for s in np.linspace(0.05, 0.95, 19):
            tgt.append(vv[0] + s * (vv[3 * k + 1] - vv[0]))
    tgt = np.array(tgt)
    for o in (np.zeros(3), np.array([0.3, 0.2, -0.1])):
        d = tgt - o
        d /= np.linalg.norm(d, axis=1, keepdims=True)
        ids, _ = osc.closest_hits(np.tile(o, (len(d), 1)), d)
        assert np.all(ids >= 0)


# --------------------------------------------------------------- G-buffer ---

def test_tiny_gbuffer_closed_form(orc):
    scene, cam, lens, p = hi.tiny_config()
    g = orc.gbuffer(orc.OScene(scene), cam, cam, p)
    jj, ii = np.mgrid[0:128, 0:128]
    occl = (ii >= 64) & (jj >= 64)
    assert np.array_equal(g["tri"] >= 2, occl)
    z = g["nd"][..., 3]
    assert np.allclose(z[occl], 0.5, atol=1e-12, rtol=0)
    assert np.allclose(z[~occl], 2.0, atol=1e-12, rtol=0)
    assert np.allclose(g["nd"][..., :3], [0, 0, -1], atol=1e-12)
    assert np.abs(g["mv"]).max() < 1e-9  # static camera
    irr = 0.05 + 1.0 / np.linalg.norm([0.3, 0.5, -1.0])
    L = g["col"][..., 0]
    assert np.allclose(L[occl], 0.6 * irr, atol=1e-6)
    bg = np.unique(np.round(L[~occl], 9))
    assert np.allclose(sorted(bg), [np.float32(0.2) * irr, np.float32(0.8) * irr], atol=1e-6)


def test_tiny_gbuffer_brute_force_ids(orc):
    scene, cam, lens, p = hi.tiny_config()
    osc = orc.OScene(scene)
    g = orc.gbuffer(osc, cam, cam, p)
    jj, ii = np.mgrid[0:128, 0:128]
    d = np.stack([orc.pinhole_dir(cam, i + 0.5, j + 0.5) for i, j in zip(ii.ravel(), jj.ravel())])
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    ids, _ = osc.closest_hits(np.zeros_like(d), d, use_bvh=False)
    assert np.array_equal(ids.reshape(128, 128), g["tri"])


# ------------------------------------------------------------------- mask ---

def test_gaussian_weights_textbook(orc):
    w = orc.gaussian_weights(1.0)
    assert abs(w.sum() - 1.0) < 1e-15
    assert np.allclose(w, [0.054488684549642, 0.244201342003233, 0.402619946894247,
                           0.244201342003233, 0.054488684549642], atol=1e-12)


def test_sobel_zero_on_constant(orc):
    """Fact 4: Sobel of a constant (Gaussian-filtered) image is exactly 0."""
    H, W = 40, 56
    nd = np.zeros((H, W, 4))
    nd[...] = [0.36, -0.48, -0.8, 3.7]
    mv = np.zeros((H, W, 2))
    m = orc.mask(nd, mv, hi.Params())
    assert np.all(m["emetric"] == 0.0)
    assert m["edge"].sum() == 0 and m["spp"].sum() == 0


def test_sobel_ramp_gives_slope(orc):
    """The 1/8-scaled Sobel of a linear ramp returns its slope (the Gaussian
    keeps linear images unchanged away from the border)."""
    H, W = 32, 32
    jj, ii = np.mgrid[0:H, 0:W].astype(np.float64)
    nd = np.zeros((H, W, 4))
    nd[..., 2] = -1.0
    nd[..., 3] = 4.0 + 0.03 * ii - 0.04 * jj
    m = orc.mask(nd, np.zeros((H, W, 2)), hi.Params())
    inner = (slice(4, H - 4), slice(4, W - 4))
    assert np.allclose(m["emetric"][inner], 0.05 / nd[..., 3][inner], rtol=1e-12)
    nd[..., 3] = 4.0
    nd[..., 0] = 0.02 * ii
    m = orc.mask(nd, np.zeros((H, W, 2)), hi.Params())
    assert np.allclose(m["emetric"][inner], 0.02, rtol=1e-12)


def test_tiny_mask_analytic(orc):
    """Edges only where the 7x7 footprint (5x5 Gaussian + 3x3 Sobel) straddles
    the occluder boundary; e = 0 (to rounding) elsewhere; spp = 16 on dilated tiles."""
    scene, cam, lens, p = hi.tiny_config()
    g = orc.gbuffer(orc.OScene(scene), cam, cam, p)
    m = orc.mask(g["nd"], g["mv"], p)
    occl = g["tri"] >= 2
    H = W = 128
    mixed = np.zeros((H, W), bool)
    for j in range(H):
        for i in range(W):
            win = occl[max(0, j - 3):j + 4, max(0, i - 3):i + 4]
            mixed[j, i] = win.any() and not win.all()
    # e = 0 analytically there; the G-buffer depth carries FP64 rounding only
    assert np.all(m["emetric"][~mixed] < 1e-12)
    assert np.all(m["edge"][~mixed] == 0)
    assert m["edge"][100, 63] == 1 and m["edge"][100, 64] == 1
    assert m["edge"][63, 100] == 1 and m["edge"][64, 100] == 1
    # tiles 16x16 with 1-tile dilation: edge tiles x in {3,4} (lower half) -> columns 32..95
    tiles = np.zeros((8, 8), bool)
    ys, xs = np.nonzero(m["edge"])
    tiles[ys // 16, xs // 16] = True
    dil = np.zeros_like(tiles)
    for ty in range(8):
        for tx in range(8):
            dil[ty, tx] = tiles[max(0, ty - 1):ty + 2, max(0, tx - 1):tx + 2].any()
    exp = np.kron(dil, np.ones((16, 16), bool)) * 16
    assert np.array_equal(m["spp"], exp.astype(np.uint8))


# ------------------------------------------------------------------ trace ---

def test_trace_focus_plane_and_far_plane(orc):
    W = H = 16
    cam = hi.Camera(width=W, height=H).f32()
    p = hi.Params(spp_max=8)
    spp = np.full((H, W), 8, np.uint8)
    # plane exactly on the focus plane: every lens ray meets the pixel's focus point
    sc = hi.plane_scene(2.0, half=50.0, cells=40.0)
    rt = orc.trace(orc.OScene(sc), cam, hi.Lens(2.0, 0.05, 0.05), p, spp)
    assert np.allclose(rt[..., 3], 0.5, atol=1e-6)
    assert np.allclose(rt[..., 0:3], rt[..., 4:7], atol=1e-9)
    assert np.all(np.abs(rt[..., 7]) < 1e-5) and np.all(np.abs(rt[..., 11]) < 1e-5)
    # plane far behind focus: no near geometry -> hit ratio 0, near layer empty
    sc = hi.plane_scene(9.0, half=500.0, cells=40.0)
    far_lens = hi.Lens(1.0, 0.2, 0.05)
    assert orc.coc(9.0, far_lens, H, cam.tan_half_fovy) < -SQRT2
    rt = orc.trace(orc.OScene(sc), cam, far_lens, p, spp)
    assert np.all(rt[..., 3] == 0.0) and np.all(rt[..., 7] == -1.0)
    assert np.allclose(rt[..., 10], 9.0, atol=1e-9)  # P_far on the plane


# ----------------------------------------------------------- post-filter ---

def test_disk_area_is_lattice_sum_of_soft_disk(orc):
    """a(r) is the soft disk summed over the integer lattice: a(0) = 1/2
    (centre only), one full ring adds 4 at r = 1.5, and for large r it
    approaches the continuous integral pi (r^2 + 1/12)."""
    assert orc.disk_area(0.0) == 0.5
    assert orc.disk_area(0.5) == 1.0
    assert abs(orc.disk_area(1.5) - (1 + 4 + 4 * (1.5 - math.sqrt(2) + 0.5))) < 1e-12
    for r in (10.0, 20.3, 31.7):
        cont = math.pi * (r * r + 1.0 / 12.0)
        assert abs(orc.disk_area(r) - cont) < 0.01 * cont
    rs = np.linspace(0, 8, 801)
    a = np.array([orc.disk_area(r) for r in rs])
    assert np.all(np.diff(a) >= 0)


def test_postfilter_zero_aperture_is_identity(orc):
    g = hi.random_gbuffer(48, 40, seed=3)
    p = hi.Params(r_max=16.0)
    pp = orc.postfilter(g["nd"], g["col"], hi.Lens(2.0, 0.0, 0.05), math.tan(math.radians(30)), p)
    assert np.allclose(pp[..., :3], g["col"][..., :3], atol=1e-12)


def test_postfilter_constant_colour(orc):
    g = hi.random_gbuffer(48, 40, seed=4)
    col = np.zeros_like(g["col"])
    col[..., :3] = [0.3, 0.6, 0.9]
    p = hi.Params(r_max=12.0)
    pp = orc.postfilter(g["nd"], col, hi.Lens(3.0, 0.05, 0.05), math.tan(math.radians(30)), p)
    assert np.allclose(pp[..., :3], [0.3, 0.6, 0.9], atol=1e-12)


def test_postfilter_uniform_near_region_is_covered(orc):
    """A large uniform near region has coverage exactly 1 inside (each pixel
    scatters unit weight); an isolated in-focus pixel covers itself by half
    (its split weight) and keeps its colour; next to the region the near blur
    adds coverage."""
    H = W = 96
    nd = np.zeros((H, W, 4))
    nd[..., 2] = -1
    nd[..., 3] = 2.0
    nd[20:76, 20:76, 3] = 0.5
    col = np.zeros((H, W, 4))
    col[..., :3] = 0.2
    col[20:76, 20:76, :3] = 0.9
    lens = hi.Lens(2.0, 0.02, 0.05)
    pp = orc.postfilter(nd, col, lens, math.tan(math.radians(30)), hi.Params(r_max=16.0))
    assert abs(pp[48, 48, 3] - 1.0) < 1e-12 and np.allclose(pp[48, 48, :3], 0.9, atol=1e-12)
    assert abs(pp[5, 5, 3] - 0.5) < 1e-12 and np.allclose(pp[5, 5, :3], 0.2, atol=1e-12)
    # the near blur spreads over the in-focus background next to the region
    assert 0.55 < pp[48, 18, 3] < 1.0 and 0.2 < pp[48, 18, 0] < 0.9


def test_postfilter_brute_force_pixel_list_matches_full(orc):
    g = hi.random_gbuffer(40, 32, seed=5)
    p = hi.Params(r_max=10.0)
    lens = hi.Lens(3.0, 0.03, 0.05)
    t = math.tan(math.radians(30))
    full = orc.postfilter(g["nd"], g["col"], lens, t, p)
    pix = np.array([0, 5, 77, 640, 1279])
    part = orc.postfilter(g["nd"], g["col"], lens, t, p, pix=pix)
    assert np.array_equal(full.reshape(-1, 4)[pix], part)


# --------------------------------------------------- temporal / spatial ----

def _static_inputs(orc, cam, seed=0):
    """Random trace output whose far positions lie on each pixel's own
    pinhole ray (as a static scene gives)."""
    W, H = cam.width, cam.height
    spp = np.full((H, W), 4, np.uint8)
    spp[:, : W // 4] = 0
    rt = _own_ray_far(orc, cam, hi.random_rt(W, H, spp, seed=seed).astype(np.float64))
    g = hi.random_gbuffer(W, H, seed=seed)
    return spp, rt, g


def _own_ray_far(orc, cam, rt):
    for j in range(cam.height):
        for i in range(cam.width):
            if rt[j, i, 11] >= 0:
                d = orc.pinhole_dir(cam, i + 0.5 + cam.jitter[0], j + 0.5 + cam.jitter[1])
                rt[j, i, 8:11] = np.array(cam.pos) + (3.0 + 0.1 * i) * d
    return rt


def test_temporal_static_fixed_point(orc):
    """Static camera, zero motion and the same trace output every frame: the
    EMA of a constant sequence is that constant, so pixels whose layers
    reproject onto themselves reconstruct the single-frame result at every
    frame.  Pixels without far hits reproject their far history from their
    neighbours' far position; they reach a steady state of their own."""
    W, H = 24, 20
    cam = hi.Camera(width=W, height=H)
    spp, rt, g = _static_inputs(orc, cam)
    mv = np.zeros((H, W, 2))
    p = hi.Params(ema_alpha=0.2)
    hist = orc.empty_history(W, H)
    first = None
    tr = spp > 0
    own = tr & (rt[..., 11] >= 0)
    assert own.sum() > 100
    prev = None
    for fr in range(150):
        hist, crt, hacc = orc.temporal(cam, cam, p, rt, spp, g["nd"], mv, hist)
        if first is None:
            first = crt.copy()
        if fr < 6:
            assert np.allclose(crt[own], first[own], atol=1e-12)
            assert np.allclose(hacc[own], rt[..., 3][own], atol=1e-12)
            assert np.all(hist["hlen"][tr] == min(fr + 1, 255)) and np.all(hist["hlen"][~tr] == 0)
        prev, last = (crt.copy() if fr == 148 else prev), crt
    assert np.allclose(last[tr], prev[tr], atol=1e-9)


def test_temporal_ema_converges(orc):
    W, H = 16, 12
    cam = hi.Camera(width=W, height=H)
    spp = np.full((H, W), 2, np.uint8)
    g = hi.random_gbuffer(W, H, seed=1)
    mv = np.zeros((H, W, 2))
    p = hi.Params(ema_alpha=0.2)
    rt0 = _own_ray_far(orc, cam, hi.random_rt(W, H, spp, seed=1).astype(np.float64))
    rt1 = _own_ray_far(orc, cam, hi.random_rt(W, H, spp, seed=2).astype(np.float64))
    own = (rt1[..., 11] >= 0) & (rt0[..., 11] >= 0)
    hist = orc.empty_history(W, H)
    hist, _, _ = orc.temporal(cam, cam, p, rt0, spp, g["nd"], mv, hist)
    for _ in range(80):
        hist, crt, hacc = orc.temporal(cam, cam, p, rt1, spp, g["nd"], mv, hist)
    single = orc.temporal(cam, cam, p, rt1, spp, g["nd"], mv, orc.empty_history(W, H))[1]
    assert own.sum() > 60
    assert np.allclose(crt[own], single[own], atol=1e-7)


def test_temporal_integer_motion_is_a_shift(orc):
    """A whole-pixel motion vector reprojects history by exactly that shift."""
    W, H = 20, 16
    cam = hi.Camera(width=W, height=H)
    spp = np.full((H, W), 3, np.uint8)
    g = hi.random_gbuffer(W, H, seed=2)
    hist = hi.random_history(W, H, seed=3, frac_valid=1.0)
    hist = {k: v.astype(np.float64) if v.dtype != np.uint8 else v for k, v in hist.items()}
    rt = hi.random_rt(W, H, spp, seed=4).astype(np.float64)
    mv = np.zeros((H, W, 2))
    mv[..., 0] = 2.0
    mv[..., 1] = -1.0
    p = hi.Params(ema_alpha=0.25)
    out, crt, _ = orc.temporal(cam, cam, p, rt, spp, g["nd"], mv, hist)
    h = rt[..., 3]
    j, i = 5, 9
    src = hist["near"][j + 1, i - 2]
    cur = np.array([h[j, i] * rt[j, i, 0], h[j, i] * rt[j, i, 1], h[j, i] * rt[j, i, 2], h[j, i]])
    assert np.allclose(out["near"][j, i], src + 0.25 * (cur - src), atol=1e-12)
    assert out["hlen"][j, i] == hist["hlen"][j + 1, i - 2] + 1


def test_spatial_constant_and_converged(orc):
    W, H = 30, 22
    spp = np.full((H, W), 4, np.uint8)
    crt = np.zeros((H, W, 4))
    crt[..., :3] = [0.25, 0.5, 0.75]
    crt[..., 3] = 12.0
    mom = np.zeros((H, W, 2))
    mom[..., 0] = 0.4
    mom[..., 1] = 0.16 + 0.0004  # sigma 0.02
    hlen = np.full((H, W), 5, np.uint8)
    rec = orc.spatial(hi.Params(), crt, spp, mom, hlen)
    assert np.allclose(rec[..., :3], crt[..., :3], atol=1e-12)
    rng = np.random.default_rng(0)
    crt[..., :3] = rng.uniform(0, 1, (H, W, 3))
    mom[..., 1] = 0.16  # zero variance, converged history -> no spatial blur
    rec = orc.spatial(hi.Params(), crt, spp, mom, hlen)
    assert np.allclose(rec[..., :3], crt[..., :3], atol=1e-12)


# -------------------------------------------------------------- composite ---

def test_composite_focus_zone_is_sharp(orc):
    scene, cam, lens, p = hi.tiny_config()
    r = orc.frame(orc.OScene(scene), cam, cam, lens, p)
    c = np.array([[orc.coc(z, lens, 128, cam.tan_half_fovy) for z in row] for row in r["g"]["nd"][..., 3]])
    traced = r["mask"]["spp"] > 0
    ce = np.where(traced, r["crt"][..., 3], np.abs(c))
    sharp = ce < SQRT2 - 0.5
    assert sharp.sum() > 5000
    assert np.array_equal(r["out"][sharp, :3], r["g"]["col"][sharp, :3])
    # untraced background far from the occluder: no near geometry anywhere
    assert np.all(r["rt"][~traced] == 0.0)


def test_tiny_frame_partial_occlusion(orc):
    """The hybrid frame shows background through the blurred occluder edge:
    inside the occluder near its edge the output lies strictly between the
    occluder's colour and the background's, unlike the post-process alone."""
    scene, cam, lens, p = hi.tiny_config()
    r = orc.frame(orc.OScene(scene), cam, cam, lens, p)
    occ = 0.6 * (0.05 + 1.0 / np.linalg.norm([0.3, 0.5, -1.0]))
    row = r["out"][100, :, 0]
    assert abs(row[100] - occ) < 2e-3  # occluder interior
    assert abs(r["pp"][100, 65, 0] - occ) < 1e-6  # post-process: opaque edge (f32 albedo)
    assert abs(row[65] - occ) > 0.01  # hybrid: background shows through


# -------------------------------------------- differentiable post-path ----

def _post_setup(orc, W=48, Hh=32, seed=3):
    """A small room frame: the oracle's own mask and hit records, a smooth
    depth plane and frozen history samples."""
    scene = hi.room_scene_target(seed, 20_000, aspect=W / Hh)
    osc = orc.OScene(scene)
    cam = hi.Camera(width=W, height=Hh).f32()
    lens = hi.Lens(2.5, 0.04, 0.05).f32()
    p = hi.room_params(r_max=16.0, camera_moved=0)
    g = orc.gbuffer(osc, cam, cam, p)
    spp = orc.mask(g["nd"], g["mv"], p)["spp"]
    rec, off = orc.trace_records(osc, cam, lens, p, spp)
    col, z = hi.diff_inputs(W, Hh, seed)
    hs = hi.random_hist_samples(W, Hh, seed).astype(np.float64)
    return osc, cam, lens, p, spp, rec, off, col.astype(np.float64), z.astype(np.float64), hs


def test_post_replay_equals_direct_trace(orc):
    """Replaying the stored hit records at the lens they were traced with
    reproduces the direct thin-lens trace of the same pixels (two different
    computations: stored (radiance, depth) per ray against tracing again)."""
    osc, cam, lens, p, spp, rec, off, col, z, hs = _post_setup(orc)
    assert (spp > 0).sum() > 50
    direct = orc.trace(osc, cam, lens, p, spp)
    rep = orc.post_forward(col, z, spp, rec, off, hs, cam, lens, p)["rt"]
    tr = spp > 0
    # colours, hit ratio and layer CoCs (the replay does not form the far-hit
    # position: with frozen history nothing reprojects by it)
    ch = [0, 1, 2, 3, 4, 5, 6, 7, 11]
    np.testing.assert_allclose(rep[tr][:, ch], direct[tr][:, ch], rtol=1e-9, atol=1e-9)
    assert np.abs(direct[tr][:, 3] - 0.5).max() > 0.1  # both layers occur


def test_post_zero_aperture_is_the_sharp_image(orc):
    """A = 0: every CoC is 0, the focus weight is 1 everywhere, so the
    post-path returns the sharp colour exactly."""
    osc, cam, lens, p, spp, rec, off, col, z, hs = _post_setup(orc)
    out = orc.post_forward(col, z, spp, rec, off, hs, cam, hi.Lens(2.5, 0.0, 0.05), p)["out"]
    assert np.array_equal(out[..., :3], col)


def test_post_path_is_affine_in_colour(orc):
    """For a fixed lens every weight depends on depth, CoC and the frozen
    radiance only, so the output is affine in the sharp colour image:
    out(C1 + C2) + out(0) = out(C1) + out(C2)."""
    osc, cam, lens, p, spp, rec, off, col, z, hs = _post_setup(orc)
    rng = np.random.default_rng(9)
    c1, c2 = col, rng.uniform(0, 1, col.shape)
    f = lambda c: orc.post_forward(c, z, spp, rec, off, hs, cam, lens, p)["out"][..., :3]  # noqa: E731
    lhs = f(c1 + c2) + f(np.zeros_like(col))
    rhs = f(c1) + f(c2)
    np.testing.assert_allclose(lhs, rhs, atol=1e-12)
    # and not trivially: the colour does move the output
    assert np.abs(f(c1) - f(c2)).max() > 0.1


def test_post_colour_vjp_at_zero_aperture_is_g(orc):
    """A = 0: the post-path is the identity in the colour image (the pin
    above), so the oracle's VJP returns g itself."""
    osc, cam, lens, p, spp, rec, off, col, z, hs = _post_setup(orc, W=16, Hh=12)
    g = np.random.default_rng(4).normal(size=col.shape)
    v = orc.post_colour_vjp(col, z, spp, rec, off, hs, cam, hi.Lens(2.5, 0.0, 0.05), p, g)
    np.testing.assert_allclose(v, g, atol=1e-12)


def test_post_colour_vjp_is_the_adjoint_of_the_forward(orc):
    """<J x, y> = <x, J^T y>: J x from two forward maps (the map is affine),
    J^T y from the oracle's VJP; x and y random on every channel (a weight
    that mixed channels would break the identity), with traced pixels and
    blur in the frame (J is not the identity)."""
    osc, cam, lens, p, spp, rec, off, col, z, hs = _post_setup(orc, W=16, Hh=12)
    spp = spp.copy()
    spp[:, :8] = 0  # the left half untraced: both composite branches
    rec, off = orc.trace_records(osc, cam, lens, p, spp)
    assert (spp > 0).any() and (spp == 0).any()
    rng = np.random.default_rng(5)
    x, y = rng.normal(size=col.shape), rng.normal(size=col.shape)
    f = lambda c: orc.post_forward(c, z, spp, rec, off, hs, cam, lens, p)["out"][..., :3]  # noqa: E731
    jx = f(col + x) - f(col)
    v = orc.post_colour_vjp(col, z, spp, rec, off, hs, cam, lens, p, y)
    lhs, rhs = float((jx * y).sum()), float((x * v).sum())
    assert abs(lhs - rhs) <= 1e-9 * max(abs(lhs), 1.0), (lhs, rhs)
    assert np.abs(v - y).max() > 1e-2
