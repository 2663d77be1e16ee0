"""Pins of the oracle's remaining stage arithmetic (CPU only).

Each case is built so that its expected value follows from the stage's
definition by a short hand derivation (a few named taps, a closed-form
geometric shift, an exact area), independent of the oracle's own loops, and so
that a plausible slip in the oracle (a dropped factor, a flipped sign, a
radius taken as the diameter, floor for round) changes the result:

* spatial reconstruction (Reconstruction section): the product weight
  s(r_p - d) s(r_q - d) with r = c/2, the rejection of samples whose CoC
  radius is smaller than their distance, the r_s cap and the variance blend;
* the mask's variance term (Ray Trace section, temporally accumulated
  variance): nearest-pixel reprojection, young history, the sigma threshold
  and ceil(spp_max sigma / var_scale);
* the post-filter's far-layer depth test (Design section): background
  sources do not bleed over a nearer far-field pixel, nearer ones do;
* G-buffer motion vectors for a translated camera against the pinhole
  projection's closed form;
* Philox4x32-10 against an independent library implementation;
* the thin-lens image of a fronto-parallel plane against its exact disk
  convolution (Ray Trace section: lens samples over the aperture disk).
"""
import math

import numpy as np
import pytest

import hdof_inputs as hi

SQRT2 = math.sqrt(2.0)


def soft(x):
    """The soft step of the gathers, s(x) = clamp(x + 1/2, 0, 1)."""
    return min(1.0, max(0.0, x + 0.5))


# ---------------------------------------------------- spatial reconstruction

def _spatial(orc, crt, spp, hlen, mom=None, **kw):
    H, W = spp.shape
    if mom is None:
        mom = np.zeros((H, W, 2))
    return orc.spatial(hi.Params(**kw), crt, spp, mom, hlen)


def test_spatial_product_weight_on_a_colour_step(orc):
    """Every pixel traced with c = 2 (r = 1): taps at d = 0, 1, sqrt2 weigh
    1, s(0)^2 = 1/4 and s(1 - sqrt2)^2; d >= 2 weighs 0.  At the first column
    of the right half the left half contributes one side tap and two
    diagonals."""
    W, H = 12, 9
    A = np.array([0.1, 0.7, 0.3])
    B = np.array([0.9, 0.2, 0.5])
    crt = np.zeros((H, W, 4))
    crt[:, :6, :3] = A
    crt[:, 6:, :3] = B
    crt[..., 3] = 2.0
    spp = np.ones((H, W), np.uint8)
    hlen = np.ones((H, W), np.uint8)  # hlen < 2: the gather is used in full
    rec = _spatial(orc, crt, spp, hlen)
    e = soft(1.0 - SQRT2) ** 2
    side = soft(0.0) ** 2
    exp = (A * (side + 2 * e) + B * (1 + 3 * side + 2 * e)) / (1 + 4 * side + 4 * e)
    np.testing.assert_allclose(rec[4, 6, :3], exp, rtol=0, atol=1e-14)
    # mirror image at the last column of the left half
    exp_l = (B * (side + 2 * e) + A * (1 + 3 * side + 2 * e)) / (1 + 4 * side + 4 * e)
    np.testing.assert_allclose(rec[4, 5, :3], exp_l, rtol=0, atol=1e-14)
    # far from the step the image is uniform
    np.testing.assert_allclose(rec[4, 2, :3], A, atol=1e-14)


def test_spatial_rejects_samples_smaller_than_their_distance(orc):
    """p (r_p = 3) with two traced neighbours at distance 2: q1 (r = 1.5) is
    rejected, s(1.5 - 2) = 0; q2 (r = 2) weighs s(3 - 2) s(2 - 2) = 1/2.  The
    weight is symmetric: q2 sees p with the same 1/2, q1 sees nothing."""
    W, H = 13, 9
    P = np.array([0.2, 0.4, 0.6])
    X = np.array([1.0, 0.0, 0.0])
    Y = np.array([0.0, 0.0, 1.0])
    crt = np.zeros((H, W, 4))
    crt[..., 3] = -1.0
    spp = np.zeros((H, W), np.uint8)
    for (j, i), c, col in (((4, 6), 6.0, P), ((4, 8), 3.0, X), ((6, 6), 4.0, Y)):
        spp[j, i] = 2
        crt[j, i, :3] = col
        crt[j, i, 3] = c
    hlen = np.ones((H, W), np.uint8)
    rec = _spatial(orc, crt, spp, hlen)
    np.testing.assert_allclose(rec[4, 6, :3], (P + 0.5 * Y) / 1.5, atol=1e-14)
    np.testing.assert_allclose(rec[4, 8, :3], X, atol=1e-14)
    np.testing.assert_allclose(rec[6, 6, :3], (Y + 0.5 * P) / 1.5, atol=1e-14)


def test_spatial_radius_cap_and_variance_blend(orc):
    """c = 40 gives r = min(20, r_s = 16): a tap at distance 16 weighs
    s(0)^2 = 1/4, one at 17 weighs 0 (uncapped it would weigh 1).  With
    history length >= 2 the gathered colour is blended by
    beta = sigma_L / var_ref = 0.025 / 0.05 = 1/2."""
    W, H = 40, 3
    P = np.array([0.3, 0.3, 0.3])
    Y = np.array([0.9, 0.5, 0.1])
    Z = np.array([0.0, 1.0, 1.0])
    crt = np.zeros((H, W, 4))
    crt[..., 3] = -1.0
    spp = np.zeros((H, W), np.uint8)
    for i, col in ((2, P), (18, Y), (19, Z)):
        spp[1, i] = 4
        crt[1, i, :3] = col
        crt[1, i, 3] = 40.0
    hlen = np.full((H, W), 5, np.uint8)
    mom = np.zeros((H, W, 2))
    mom[..., 0] = 0.5
    mom[..., 1] = 0.25 + 0.025 ** 2
    rec = _spatial(orc, crt, spp, hlen, mom=mom)
    c_sp = (P + 0.25 * Y) / 1.25
    np.testing.assert_allclose(rec[1, 2, :3], P + 0.5 * (c_sp - P), atol=1e-12)
    # zero variance with history: the temporal colour is kept as it is
    mom[..., 1] = 0.25
    rec = _spatial(orc, crt, spp, hlen, mom=mom)
    np.testing.assert_allclose(rec[1, 2, :3], P, atol=1e-12)


# ------------------------------------------------------- mask variance term

# (history length, luminance std-dev, expected rays) with spp_max 8,
# var_tau 0.02, var_scale 0.1, hlen_young 4
_VAR_CASES = [
    (0, 0.30, 0),   # no history: nothing to add
    (1, 0.00, 8),   # young: spp_max whatever the variance
    (3, 0.50, 8),
    (4, 0.01, 0),   # converged and quiet (sigma <= var_tau)
    (4, 0.03, 3),   # ceil(8 * 0.03 / 0.1) = ceil(2.4)
    (200, 0.021, 2),  # ceil(1.68)
    (9, 0.50, 8),   # ceil(40) clamped to spp_max
    (6, 0.06, 5),   # ceil(4.8)
]


def _var_history(W, H):
    """History whose case index at pixel (x, y) is (x + 3 y) mod 8."""
    hl = np.zeros((H, W), np.uint8)
    mom = np.zeros((H, W, 2))
    case = np.zeros((H, W), np.int64)
    for y in range(H):
        for x in range(W):
            k = (x + 3 * y) % len(_VAR_CASES)
            case[y, x] = k
            hl[y, x] = _VAR_CASES[k][0]
            sig = _VAR_CASES[k][1]
            mom[y, x] = (0.5, 0.25 + sig * sig)
    return hl, mom, case


def test_mask_variance_term_cases(orc):
    """A flat G-buffer (no edges) with a history of known moments: each pixel
    reads the history at the nearest pixel of its reprojected position
    (i, j) - mv and gets the rays its case dictates.  Rows alternate motion
    vectors whose rounding differs from flooring, and one band reprojects
    vertically and partly off screen (no history there: 0 rays)."""
    W, H = 48, 32
    nd = np.zeros((H, W, 4))
    nd[..., 2] = -1.0
    nd[..., 3] = 3.0
    mv = np.zeros((H, W, 2))
    mv[0::2, :, 0] = 0.4    # nearest pixel: i      (floor would take i - 1)
    mv[1::2, :, 0] = 1.4    # nearest pixel: i - 1  (floor would take i - 2)
    mv[24:, :, 1] = -1.45   # rows 24..: read row j + 1; the last row reads off screen
    hl, mom, case = _var_history(W, H)
    p = hi.Params(variance_on=1, spp_max=8, var_tau=0.02, var_scale=0.1, hlen_young=4)
    m = orc.mask(nd, mv, p, hist_mom=mom, hist_hlen=hl)
    assert not m["edge"].any()
    exp = np.zeros((H, W), np.uint8)
    for j in range(H):
        for i in range(W):
            x = i - (0 if j % 2 == 0 else 1)
            y = j + (1 if j >= 24 else 0)
            if 0 <= x < W and 0 <= y < H:
                exp[j, i] = _VAR_CASES[case[y, x]][2]
    assert np.array_equal(m["spp"], exp)
    assert exp[:, 0][1::2].max() == 0 and (exp > 0).sum() > 500
    # the variance term is off unless asked for
    m0 = orc.mask(nd, mv, p.replace(variance_on=0), hist_mom=mom, hist_hlen=hl)
    assert not m0["spp"].any()


def test_mask_edge_tiles_override_history(orc):
    """An edge tile (dilated) gets spp_max whatever the history says."""
    W, H = 64, 32
    nd = np.zeros((H, W, 4))
    nd[..., 2] = -1.0
    nd[..., 3] = 3.0
    nd[:, 40:, 3] = 1.0  # depth step at x = 40: tile column 2 holds edges
    mv = np.zeros((H, W, 2))
    hl = np.full((H, W), 4, np.uint8)
    mom = np.zeros((H, W, 2))
    mom[..., 0] = 0.5
    mom[..., 1] = 0.25  # quiet history: 0 rays outside edge tiles
    p = hi.Params(variance_on=1, spp_max=8, tile=16, dilate=1)
    m = orc.mask(nd, mv, p, hist_mom=mom, hist_hlen=hl)
    assert m["edge"][:, 36:44].any() and not m["edge"][:, :30].any()
    # edges in tile column 2 (x 32..47), dilated to columns 1..3 (x 16..63)
    assert np.all(m["spp"][:, 16:] == 8) and np.all(m["spp"][:, :16] == 0)


# ------------------------------------------------ post-filter depth test ----

def _two_depth_frame(W, H, z1, z2, A, B, split):
    nd = np.zeros((H, W, 4))
    nd[..., 2] = -1.0
    nd[..., 3] = z1
    nd[:, split:, 3] = z2
    col = np.zeros((H, W, 4))
    col[:, :split, :3] = A
    col[:, split:, :3] = B
    return nd, col


def test_postfilter_far_depth_test_direction(orc):
    """Two far-field regions (both CoC < -sqrt2), the right one 50% farther:
    the soft depth test k_z = clamp(1 - (z_q - z_p) / (kz_rel z_p), 0, 1) is 0
    for the farther sources seen from the nearer side, so next to the step the
    nearer region keeps its own colour exactly, while the farther region
    receives the nearer region's blur (k_z = 1 for nearer sources)."""
    W, H, split = 40, 24, 20
    A = np.array([0.8, 0.1, 0.1])
    B = np.array([0.1, 0.1, 0.8])
    z1, z2 = 2.0, 3.0
    nd, col = _two_depth_frame(W, H, z1, z2, A, B, split)
    t = math.tan(math.radians(30))
    lens = hi.Lens(1.0, 0.2, 0.05)
    for z in (z1, z2):
        assert orc.coc(z, lens, H, t) < -SQRT2
    r2 = abs(orc.coc(z2, lens, H, t)) / 2
    pp = orc.postfilter(nd, col, lens, t, hi.Params(r_max=16.0))
    assert np.all(pp[..., 3] == 0.0)  # no near layer
    # nearer side, within reach of the farther sources: own colour exactly
    np.testing.assert_allclose(pp[12, split - 3:split, :3], np.broadcast_to(A, (3, 3)), atol=1e-14)
    # farther side next to the step: strictly between the two colours
    mix = pp[12, split, :3]
    assert mix[0] > B[0] + 0.05 and mix[2] < B[2] - 0.05
    # and beyond the nearer region's reach it is the farther colour again
    far_col = split + int(math.ceil(abs(orc.coc(z1, lens, H, t)) / 2 + 0.5)) + 1
    assert far_col < W and r2 > 0
    np.testing.assert_allclose(pp[12, far_col, :3], B, atol=1e-14)


def test_postfilter_far_depth_test_half_weight(orc):
    """Depths 1 and 1.025 with kz_rel 0.05: from the nearer side a farther
    source weighs k_z = 1 - 0.025 / 0.05 = 1/2 (the band is relative to the
    receiving pixel's depth).  The lens makes r = 1 and 1.1 px, so the taps
    of the pixel next to the step are: itself, three side taps and two
    diagonals of its own region, one side tap and two diagonals across."""
    W, H, split = 16, 12, 8
    A = np.array([0.8, 0.1, 0.1])
    B = np.array([0.1, 0.1, 0.8])
    t = math.tan(math.radians(30))
    K = 8.2
    lens = hi.Lens(1.0 / (1.0 + 2.0 / K), K * t / H, 0.05)
    nd, col = _two_depth_frame(W, H, 1.0, 1.025, A, B, split)
    r1 = abs(orc.coc(1.0, lens, H, t)) / 2
    r2 = abs(orc.coc(1.025, lens, H, t)) / 2
    assert abs(r1 - 1.0) < 1e-9 and abs(r2 - 1.1) < 1e-3
    pp = orc.postfilter(nd, col, lens, t, hi.Params(r_max=16.0, kz_rel=0.05))
    a1, a2 = orc.disk_area(r1), orc.disk_area(r2)
    wa = (soft(r1) + 3 * soft(r1 - 1) + 2 * soft(r1 - SQRT2)) / a1
    wb = 0.5 * (soft(r2 - 1) + 2 * soft(r2 - SQRT2)) / a2
    exp = (wa * A + wb * B) / (wa + wb)
    np.testing.assert_allclose(pp[6, split - 1, :3], exp, atol=1e-12)
    assert pp[6, split - 1, 3] == 0.0


# ------------------------------------------------------- G-buffer motion ----

@pytest.mark.parametrize("axis", [0, 1])
def test_gbuffer_motion_of_a_translated_camera(orc, axis):
    """A fronto-parallel plane at depth z and a camera translated by delta
    along +x (or +y) since the previous frame.  A surface point then moved by
    -delta (x) or +delta (y, rows grow downwards) relative to the camera, i.e.
    by delta H / (2 z t) pixels, so mv = (i, j) - previous position =
    (-delta H / (2 z t), 0) or (0, +delta H / (2 z t)), plus the difference
    of the two frames' jitters (previous - current)."""
    W, H, z = 40, 30, 2.0
    scene = hi.plane_scene(z, half=50.0, cells=40.0)
    osc = orc.OScene(scene)
    d = 0.05
    jc, jp = (0.25, -0.125), (-0.375, 0.0625)
    pos = [0.0, 0.0, 0.0]
    pos[axis] = d
    cam = hi.Camera(pos=tuple(pos), width=W, height=H, jitter=jc).f32()
    prev = hi.Camera(width=W, height=H, jitter=jp).f32()
    p = hi.Params()
    g = orc.gbuffer(osc, cam, prev, p)
    assert np.allclose(g["nd"][..., 3], z, atol=1e-12)
    shift = float(np.float32(d)) * H / (2 * z * cam.tan_half_fovy)
    exp = np.array([jp[0] - jc[0], jp[1] - jc[1]])
    exp[axis] += -shift if axis == 0 else shift
    np.testing.assert_allclose(g["mv"].reshape(-1, 2), np.broadcast_to(exp, (W * H, 2)), atol=1e-9)
    # static camera, same jitter: zero motion
    g0 = orc.gbuffer(osc, prev, prev, p)
    assert np.abs(g0["mv"]).max() < 1e-9


def test_gbuffer_motion_behind_previous_camera(orc):
    """A point the previous camera cannot see (behind it) gets the off-screen
    marker 1e6."""
    W, H = 16, 12
    osc = orc.OScene(hi.plane_scene(2.0, half=50.0, cells=40.0))
    cam = hi.Camera(width=W, height=H).f32()
    prev = hi.Camera(pos=(0.0, 0.0, 3.0), width=W, height=H).f32()
    g = orc.gbuffer(osc, cam, prev, hi.Params())
    assert np.all(g["mv"] == 1e6)


# ---------------------------------------------------------------- Philox ----

def test_philox_matches_an_independent_library_implementation(orc):
    """Philox4x32-10 of the oracle equals triton's tl.philox (10 rounds, run by
    triton's CPU interpreter, whose implementation shares nothing with the
    oracle) on the all-zero / all-one / pi-digit counters and keys and on
    random ones.  triton's 64-bit seed is (key[1] << 32) | key[0]."""
    import os
    import subprocess
    import sys
    pytest.importorskip("triton")
    rng = np.random.default_rng(11)
    ctr = rng.integers(0, 2 ** 32, (64, 4), dtype=np.uint64).astype(np.uint32)
    key = rng.integers(0, 2 ** 32, (64, 2), dtype=np.uint64).astype(np.uint32)
    ctr[0], key[0] = 0, 0
    ctr[1], key[1] = 0xFFFFFFFF, 0xFFFFFFFF
    ctr[2] = [0x243F6A88, 0x85A308D3, 0x13198A2E, 0x03707344]
    key[2] = [0xA4093822, 0x299F31D0]
    # the interpreter is switched on per process: run it in a child
    code = r"""
import os, sys, numpy as np
os.environ["TRITON_INTERPRET"] = "1"
import torch, triton, triton.language as tl
@triton.jit
def k(c0, c1, c2, c3, k0, k1, o0, o1, o2, o3, N: tl.constexpr):
    i = tl.arange(0, N)
    ka = tl.load(k0 + i).to(tl.uint32, bitcast=True).to(tl.uint64)
    kb = tl.load(k1 + i).to(tl.uint32, bitcast=True).to(tl.uint64)
    x0, x1, x2, x3 = tl.philox((kb << 32) | ka, tl.load(c0 + i), tl.load(c1 + i),
                               tl.load(c2 + i), tl.load(c3 + i), 10)
    tl.store(o0 + i, x0); tl.store(o1 + i, x1); tl.store(o2 + i, x2); tl.store(o3 + i, x3)
a = np.frombuffer(sys.stdin.buffer.read(), np.uint32).reshape(-1, 6)
t = [torch.from_numpy(a[:, c].copy().view(np.int32)) for c in range(6)]
o = [torch.empty(a.shape[0], dtype=torch.int32) for _ in range(4)]
k[(1,)](*t, *o, N=a.shape[0])
sys.stdout.buffer.write(np.stack([x.numpy().view(np.uint32) for x in o], 1).tobytes())
"""
    inp = np.concatenate([ctr, key], 1).astype(np.uint32).tobytes()
    env = dict(os.environ, CUDA_VISIBLE_DEVICES="")
    r = subprocess.run([sys.executable, "-c", code], input=inp, capture_output=True, env=env, timeout=600)
    if r.returncode != 0:
        pytest.skip("triton interpreter unavailable: " + r.stderr.decode()[-300:])
    lib = np.frombuffer(r.stdout, np.uint32).reshape(-1, 4)
    for c, k, want in zip(ctr, key, lib):
        assert orc.philox(c, k) == [int(x) for x in want]


# ------------------------------------------- fact 2: exact disk convolution

def _quadrant(a, b, R):
    """Signed area of {(x, y) in the disk of radius R at the origin} between
    the axes and the point (a, b): the integral of the disk's indicator over
    [0, a] x [0, b] (negative bounds count negatively)."""
    sa, sb = (1.0 if a >= 0 else -1.0), (1.0 if b >= 0 else -1.0)
    a, b = min(abs(a), R), abs(b)
    if b >= R:
        xs = 0.0
    else:
        xs = math.sqrt(R * R - b * b)  # where the circle's height equals b
    x1 = min(a, xs)

    def prim(x):  # antiderivative of sqrt(R^2 - x^2)
        x = min(x, R)
        return 0.5 * (x * math.sqrt(max(0.0, R * R - x * x)) + R * R * math.asin(x / R))

    area = b * x1 + (prim(a) - prim(x1) if a > x1 else 0.0)
    return sa * sb * area


def _rect_disk_area(x0, x1, y0, y1, R):
    """Exact area of [x0, x1] x [y0, y1] inside the disk of radius R at the
    origin (inclusion-exclusion of the quadrant areas)."""
    return (_quadrant(x1, y1, R) - _quadrant(x0, y1, R) - _quadrant(x1, y0, R) + _quadrant(x0, y0, R))


def _exact_disk_average_checker(cam, z, R, cells, half, albedo, irr):
    """Mean and std-dev over a disk of radius R pixels of the pinhole image
    of the checker plane, per pixel, from the exact areas of the disk's
    overlap with each checker cell (the cells are axis-aligned rectangles in
    screen space: the pinhole projection of a fronto-parallel plane is
    affine)."""
    W, H = cam.width, cam.height
    t = cam.tan_half_fovy
    a = W / H
    # screen x of world X on the plane: sx = (X / (z a t) + 1) W / 2; y flips
    cell = 2.0 * half / cells
    mean = np.zeros((H, W))
    sd = np.zeros((H, W))
    for j in range(H):
        for i in range(W):
            cx, cy = i + 0.5, j + 0.5
            # world bounds of the disk's bounding box
            Xlo = ((cx - R) * 2.0 / W - 1.0) * z * a * t
            Xhi = ((cx + R) * 2.0 / W - 1.0) * z * a * t
            Ylo = (1.0 - 2.0 * (cy + R) / H) * z * t
            Yhi = (1.0 - 2.0 * (cy - R) / H) * z * t
            ku = range(int(math.floor((Xlo + half) / cell)), int(math.floor((Xhi + half) / cell)) + 1)
            kv = range(int(math.floor((Ylo + half) / cell)), int(math.floor((Yhi + half) / cell)) + 1)
            m1 = m2 = 0.0
            for cu in ku:
                for cv in kv:
                    X0, X1 = -half + cu * cell, -half + (cu + 1) * cell
                    Y0, Y1 = -half + cv * cell, -half + (cv + 1) * cell
                    sx0 = (X0 / (z * a * t) + 1.0) * 0.5 * W - cx
                    sx1 = (X1 / (z * a * t) + 1.0) * 0.5 * W - cx
                    sy0 = (1.0 - Y1 / (z * t)) * 0.5 * H - cy
                    sy1 = (1.0 - Y0 / (z * t)) * 0.5 * H - cy
                    ar = _rect_disk_area(sx0, sx1, sy0, sy1, R)
                    L = albedo[(cu + cv) % 2] * irr
                    m1 += ar * L
                    m2 += ar * L * L
            m1 /= math.pi * R * R
            m2 /= math.pi * R * R
            mean[j, i] = m1
            sd[j, i] = math.sqrt(max(0.0, m2 - m1 * m1))
    return mean, sd


def test_rect_disk_area_against_fine_grid():
    """The exact overlap area against a midpoint grid of 1.44 million nodes
    (error of order R / 1200 per unit of boundary length)."""
    n = 1200
    for (x0, x1, y0, y1, R) in ((-0.7, 1.3, -2.0, 0.4, 2.08), (0.3, 5.0, 0.2, 5.0, 2.5),
                                (-3.0, 3.0, -3.0, 3.0, 1.0), (-1.0, -0.2, 0.5, 0.9, 1.7)):
        g = (np.arange(n) + 0.5) / n * 2 * R - R
        X, Y = np.meshgrid(g, g)
        inside = (X * X + Y * Y <= R * R) & (X >= x0) & (X <= x1) & (Y >= y0) & (Y <= y1)
        grid = inside.sum() * (2 * R / n) ** 2
        exact = _rect_disk_area(x0, x1, y0, y1, R)
        h = 2 * R / n
        assert abs(grid - exact) < (2 * math.pi * R + 2 * (x1 - x0) + 2 * (y1 - y0)) * h
    assert abs(_rect_disk_area(-5, 5, -5, 5, 1.3) - math.pi * 1.69) < 1e-12


def test_fronto_plane_matches_exact_disk_convolution(orc):
    """Fact 2 with an exact reference: the thin-lens image of a fronto-parallel
    Lambert checker plane at depth z is its pinhole image averaged over a
    disk of radius |c(z)|/2 pixels (a lens point uniform on the aperture disk
    lands uniformly on that disk of the plane).  At N = 1024 samples per pixel
    the oracle's estimate is within 4 sigma_p / sqrt(N) of the exact average
    on at least 99% of pixels (1e-12 absolute is left for floating-point
    summation where sigma_p = 0), and its error shrinks with N."""
    z, zf, A = 1.0, 2.0, 0.2
    W = H = 24
    cam = hi.Camera(width=W, height=H).f32()
    lens = hi.Lens(zf, A, 0.05).f32()
    scene = hi.plane_scene(z, half=50.0, cells=400.0)
    osc = orc.OScene(scene)
    t = cam.tan_half_fovy
    c = lens.aperture_radius * H * (lens.focus_dist - z) / (z * lens.focus_dist * t)
    assert c > SQRT2
    p = hi.Params(spp_max=128)
    ldir = p.unit_lights()[0]
    irr = p.k_ambient + max(0.0, -ldir[2])  # face normal (0, 0, -1), E = 1
    albedo = (float(np.float32(0.2)), float(np.float32(0.8)))
    exp_mean, sig = _exact_disk_average_checker(cam, z, c / 2, 400.0, 50.0, albedo, irr)
    assert (sig > 0).mean() > 0.3  # many disks straddle cell edges
    spp = np.full((H, W), 128, np.uint8)
    est = []
    for fr in range(8):  # 8 independent keys x 128 spp = 1024 samples
        rt = orc.trace(osc, cam, lens, p.replace(frame=fr), spp)
        assert np.all(rt[..., 3] == 1.0)
        est.append(rt[..., 0])
    est = np.array(est)
    e1024 = np.abs(est.mean(0) - exp_mean)
    assert (e1024 <= 4 * sig / math.sqrt(1024) + 1e-12).mean() >= 0.99
    # uniform disks (sigma_p = 0) are exact
    assert e1024[sig == 0].max(initial=0.0) < 1e-12
    e128 = np.abs(est[0] - exp_mean).mean()
    assert e1024.mean() < 0.6 * e128


# ------------------------------------------- full ray-traced reference -----

def test_reference_rt_of_a_plane_is_the_disk_convolution(orc):
    """The full ray-traced frame of a fronto-parallel checker plane converges
    to the exact disk convolution (passes x spp_max = 8 x 128 samples), within
    4 sigma_p / sqrt(N) on >= 99% of pixels, as the trace's own estimate
    does."""
    z, zf, A = 1.0, 2.0, 0.2
    W = H = 24
    cam = hi.Camera(width=W, height=H).f32()
    lens = hi.Lens(zf, A, 0.05).f32()
    osc = orc.OScene(hi.plane_scene(z, half=50.0, cells=400.0))
    t = cam.tan_half_fovy
    c = lens.aperture_radius * H * (lens.focus_dist - z) / (z * lens.focus_dist * t)
    p = hi.Params(spp_max=128)
    irr = p.k_ambient + max(0.0, -p.unit_lights()[0][2])
    exp_mean, sig = _exact_disk_average_checker(cam, z, c / 2, 400.0, 50.0,
                                                (float(np.float32(0.2)), float(np.float32(0.8))), irr)
    out = orc.reference_rt(osc, cam, lens, p, 8)
    e = np.abs(out[..., 0] - exp_mean)
    assert (e <= 4 * sig / math.sqrt(1024) + 1e-12).mean() >= 0.99
    # the same samples as eight traces keyed frame 0..7 (pass k = frame k)
    spp = np.full((H, W), 128, np.uint8)
    est = np.mean([orc.trace(osc, cam, lens, p.replace(frame=k), spp)[..., 0] for k in range(8)], 0)
    np.testing.assert_allclose(out[..., 0], est, atol=1e-12)


def test_hybrid_is_closer_to_ray_tracing_than_post_processing(orc):
    """The paper's claim (Abstract; Fig. 1) on the tiny scene: against the
    full ray-traced frame (16 passes x 16 samples), after four frames of a
    static camera, the hybrid frame's mean error on the traced pixels (the
    blurry occluder's silhouette) is below half the post-process-only frame's
    (the same composite with no traced pixels); elsewhere they are equal."""
    scene, cam, lens, p = hi.tiny_config()
    osc = orc.OScene(scene)
    hist = None
    for k in range(4):
        r = orc.frame(osc, cam, cam, lens, p.replace(frame=k), hist=hist)
        hist = r["hist"]
    spp = r["mask"]["spp"]
    pp_only = orc.composite(r["g"]["nd"], r["g"]["col"], np.zeros_like(spp), r["pp"], r["crt"], r["crec"],
                            r["hacc"], lens, cam.tan_half_fovy, p, cam.height)
    rt = orc.reference_rt(osc, cam, lens, p, 16)
    tr = spp > 0
    hyb = np.abs(r["out"][..., :3] - rt[..., :3])[tr].mean()
    pp = np.abs(pp_only[..., :3] - rt[..., :3])[tr].mean()
    assert hyb < 0.5 * pp, (hyb, pp)
    assert np.array_equal(r["out"][~tr, :3], pp_only[~tr, :3])


# --------------------------------------- per-pixel temporal blend factor ----

def _one_pixel_temporal(orc, h, grey, hist_B, hist_grey, mu1, sigma, spp_n, alpha_k):
    """A 3x3 static frame whose pixels are all traced alike: this frame's
    layers both grey `grey` with hit ratio h, the history's near layer (B,
    B hist_grey) and moments (mu1, mu1^2 + sigma^2); returns the centre
    pixel's new near history and the trace record."""
    W = H = 3
    cam = hi.Camera(width=W, height=H)
    spp = np.full((H, W), spp_n, np.uint8)
    rt = np.zeros((H, W, 12))
    rt[..., 0:3] = grey
    rt[..., 3] = h
    rt[..., 4:7] = grey
    rt[..., 7] = 4.0
    rt[..., 11] = 1.0
    for j in range(H):
        for i in range(W):
            d = orc.pinhole_dir(cam, i + 0.5, j + 0.5)
            rt[j, i, 8:11] = 3.0 * d
    hist = orc.empty_history(W, H)
    hist["near"][..., :3] = hist_B * hist_grey
    hist["near"][..., 3] = hist_B
    hist["far"][..., :3] = (1 - hist_B) * hist_grey
    hist["far"][..., 3] = 1 - hist_B
    hist["mom"][..., 0] = mu1
    hist["mom"][..., 1] = mu1 * mu1 + sigma * sigma
    hist["hlen"][:] = 6
    g = hi.random_gbuffer(W, H, seed=0)
    p = hi.Params(ema_alpha=0.2, alpha_k=alpha_k)
    out, _, _ = orc.temporal(cam, cam, p, rt, spp, g["nd"], np.zeros((H, W, 2)), hist)
    return out["near"][1, 1], rt[1, 1]


@pytest.mark.parametrize("case", ["luminance", "hit_ratio", "noise", "off"])
def test_temporal_per_pixel_blend_factor(orc, case):
    """alpha = alpha_min + (1 - alpha_min) lambda with lambda the larger of
    the luminance change beyond alpha_k history std-devs (relative to the
    larger luminance) and the hit-ratio change beyond alpha_k binomial
    standard errors; the near history moves by alpha towards this frame."""
    if case == "luminance":   # Y 0.8 against mu1 0.5, sigma 0.01: (0.3 - 0.02) / 0.8 = 0.35
        args, lam = dict(h=0.5, grey=0.8, hist_B=0.5, hist_grey=0.5, mu1=0.5, sigma=0.01, spp_n=4, alpha_k=2.0), 0.35
    elif case == "hit_ratio":  # h 0.9 against B 0.1 at 4 samples: 0.8 - 2 sqrt(0.09 / 4) = 0.5
        args, lam = dict(h=0.9, grey=0.6, hist_B=0.1, hist_grey=0.6, mu1=0.6, sigma=0.0, spp_n=4, alpha_k=2.0), 0.5
    elif case == "noise":      # both changes inside the noise bands
        args, lam = dict(h=0.5, grey=0.52, hist_B=0.45, hist_grey=0.5, mu1=0.5, sigma=0.02, spp_n=4,
                         alpha_k=2.0), 0.0
    else:                      # alpha_k = 0: the fixed weight, whatever the change
        args, lam = dict(h=0.9, grey=0.8, hist_B=0.1, hist_grey=0.5, mu1=0.5, sigma=0.0, spp_n=4, alpha_k=0.0), 0.0
    near, r = _one_pixel_temporal(orc, **args)
    al = 0.2 + 0.8 * lam
    B = args["hist_B"]
    hn = np.array([B * args["hist_grey"]] * 3 + [B])
    cur = np.array([r[3] * r[0], r[3] * r[1], r[3] * r[2], r[3]])
    np.testing.assert_allclose(near, hn + al * (cur - hn), atol=1e-12)


# ------------------------------------------------------ CoC-scaled mask ----

def test_mask_reach_scales_with_coc(orc):
    """A near square (z = 0.5) over an in-focus background (z = zf = 2):
    edges lie in tile columns 3..6 (the 7-pixel footprint of the Gaussian +
    Sobel around x = 64 and x = 96) and rows 1..4.  The tiles holding near
    pixels have r = min(|c(0.5)| / 2, r_max) with c(0.5) = A H 1.5 / (0.5 zf t)
    = 249.4 A px: A = 0.3 gives r = 37.4, a reach of ceil(37.4 / 16) = 3
    tiles, so columns 1..8 are traced instead of the fixed dilation's 2..7;
    a cap r_max = 16 brings the reach back to 1."""
    W, H, T = 224, 96, 16
    nd = np.zeros((H, W, 4))
    nd[..., 2] = -1.0
    nd[..., 3] = 2.0
    nd[32:64, 64:96, 3] = 0.5
    mv = np.zeros((H, W, 2))
    t = math.tan(math.radians(30))
    lens = hi.Lens(2.0, 0.3, 0.05)
    assert abs(orc.coc(0.5, lens, H, t) / 2 - 124.7 * 0.3) < 0.05
    cols = lambda spp: sorted({i // T for i in range(W) if spp[:, i].any()})  # noqa: E731
    base = orc.mask(nd, mv, hi.Params(spp_max=8, tile=T, dilate=1, r_max=100.0), lens_=lens, tan_half_fovy=t)
    assert sorted({i // T for i in range(W) if base["edge"][:, i].any()}) == [3, 4, 5, 6]
    assert cols(base["spp"]) == [2, 3, 4, 5, 6, 7]
    coc = orc.mask(nd, mv, hi.Params(spp_max=8, tile=T, dilate=1, r_max=100.0, mask_coc=1), lens_=lens,
                   tan_half_fovy=t)
    assert np.array_equal(coc["edge"], base["edge"])
    assert cols(coc["spp"]) == [1, 2, 3, 4, 5, 6, 7, 8]
    assert np.all(coc["spp"][:, T:9 * T] == 8) and not coc["spp"][:, :T].any() and not coc["spp"][:, 9 * T:].any()
    capped = orc.mask(nd, mv, hi.Params(spp_max=8, tile=T, dilate=1, r_max=16.0, mask_coc=1), lens_=lens,
                      tan_half_fovy=t)
    assert np.array_equal(capped["spp"], base["spp"])
    # without the lens the flag has nothing to scale by: the fixed dilation
    nolens = orc.mask(nd, mv, hi.Params(spp_max=8, tile=T, dilate=1, r_max=100.0, mask_coc=1))
    assert np.array_equal(nolens["spp"], base["spp"])


# --------------------------------------------- aperture shape and weights ----

def _clip(poly, axis, bound, keep_le):
    """Sutherland-Hodgman: the part of poly with coordinate `axis` <= bound
    (keep_le) or >= bound."""
    out = []
    inside = (lambda v: v[axis] <= bound) if keep_le else (lambda v: v[axis] >= bound)
    for k in range(len(poly)):
        a, b = poly[k - 1], poly[k]
        if inside(b):
            if not inside(a):
                t = (bound - a[axis]) / (b[axis] - a[axis])
                out.append(a + t * (b - a))
            out.append(b)
        elif inside(a):
            t = (bound - a[axis]) / (b[axis] - a[axis])
            out.append(a + t * (b - a))
    return out


def _area(poly):
    if len(poly) < 3:
        return 0.0
    x = np.array([v[0] for v in poly])
    y = np.array([v[1] for v in poly])
    return 0.5 * abs(np.dot(x, np.roll(y, -1)) - np.dot(y, np.roll(x, -1)))


def test_polygon_aperture_plane_is_the_polygon_convolution(orc):
    """A triangular aperture (3 blades, a vertex up): the thin-lens image of a
    fronto-parallel checker plane in the near field averages the pinhole image
    over the aperture scaled to radius c/2 and mirrored top-bottom in screen
    space (lens point O shows the plane point at screen offset
    (c / 2A) (O_right, -O_up)); the expected value per pixel comes from exact
    polygon/cell overlaps (Sutherland-Hodgman clipping).  1024 samples per
    pixel: within 4 sigma_p / sqrt(N) on >= 99% of pixels."""
    z, zf, A = 1.0, 2.0, 0.2
    W = H = 20
    cam = hi.Camera(width=W, height=H).f32()
    lens = hi.Lens(zf, A, 0.05).f32()
    p = hi.Params(spp_max=128, blades=3, blade_rot=math.pi / 2)
    osc = orc.OScene(hi.plane_scene(z, half=50.0, cells=400.0))
    t = cam.tan_half_fovy
    c = lens.aperture_radius * H * (lens.focus_dist - z) / (z * lens.focus_dist * t)
    th = [p.blade_rot + 2 * math.pi * k / 3 for k in range(3)]
    shape = [np.array([c / 2 * math.cos(a), -c / 2 * math.sin(a)]) for a in th]
    irr = p.k_ambient + max(0.0, -p.unit_lights()[0][2])
    alb = (float(np.float32(0.2)), float(np.float32(0.8)))
    a_ = W / H
    cell = 2 * 50.0 / 400.0
    mean = np.zeros((H, W))
    sd = np.zeros((H, W))
    for j in range(H):
        for i in range(W):
            poly = [v + np.array([i + 0.5, j + 0.5]) for v in shape]
            tot = _area(poly)
            xs = [v[0] for v in poly]
            ys = [v[1] for v in poly]
            X0 = (2 * min(xs) / W - 1) * a_ * t * z
            X1 = (2 * max(xs) / W - 1) * a_ * t * z
            Y0 = (1 - 2 * max(ys) / H) * t * z
            Y1 = (1 - 2 * min(ys) / H) * t * z
            m1 = m2 = 0.0
            for cu in range(int(math.floor((X0 + 50) / cell)), int(math.floor((X1 + 50) / cell)) + 1):
                for cv in range(int(math.floor((Y0 + 50) / cell)), int(math.floor((Y1 + 50) / cell)) + 1):
                    sx0 = ((-50 + cu * cell) / (z * a_ * t) + 1) * 0.5 * W
                    sx1 = ((-50 + (cu + 1) * cell) / (z * a_ * t) + 1) * 0.5 * W
                    sy0 = (1 - (-50 + (cv + 1) * cell) / (z * t)) * 0.5 * H
                    sy1 = (1 - (-50 + cv * cell) / (z * t)) * 0.5 * H
                    q = _clip(_clip(_clip(_clip(poly, 0, sx0, False), 0, sx1, True), 1, sy0, False), 1, sy1, True)
                    L = alb[(cu + cv) % 2] * irr
                    ar = _area(q) / tot
                    m1 += ar * L
                    m2 += ar * L * L
            mean[j, i] = m1
            sd[j, i] = math.sqrt(max(0.0, m2 - m1 * m1))
    assert (sd > 0).mean() > 0.3
    spp = np.full((H, W), 128, np.uint8)
    est = np.mean([orc.trace(osc, cam, lens, p.replace(frame=k), spp)[..., 0] for k in range(8)], 0)
    e = np.abs(est - mean)
    assert (e <= 4 * sd / math.sqrt(1024) + 1e-12).mean() >= 0.99
    # the disk's image differs: the shape matters
    disk = np.mean([orc.trace(osc, cam, lens, p.replace(frame=k, blades=0), spp)[..., 0] for k in range(8)], 0)
    assert np.abs(disk - mean).max() > 3 * (4 * sd.max() / math.sqrt(1024))


def _weighted_fraction(h, R, a):
    """Fraction of the disk of radius R at the origin with x > h, each point
    weighted by 1 + a (2 rho^2 / R^2 - 1) (total weight pi R^2): Gauss-Legendre
    in theta with x = R sin(theta), where the integrand is smooth."""
    if h >= R:
        return 0.0
    if h <= -R:
        return 1.0
    t0, t1 = math.asin(h / R), math.pi / 2
    xg, wg = np.polynomial.legendre.leggauss(64)
    th = 0.5 * (t1 - t0) * xg + 0.5 * (t1 + t0)
    x = R * np.sin(th)
    y = R * np.cos(th)  # half-chord
    # integral over y in [-y, y] of 1 + a (2 (x^2 + y^2) / R^2 - 1)
    f = 2 * y * (1 - a) + (2 * a / R ** 2) * (2 * x * x * y + 2 * y ** 3 / 3)
    return float(0.5 * (t1 - t0) * np.sum(wg * f * R * np.cos(th))) / (math.pi * R * R)


def test_aberration_weights_over_an_edge(orc):
    """A circular aperture with sample weights 1 + a (2 rho^2 / A^2 - 1)
    (a = 0.8: a bright rim): the image of a plane split by one straight albedo
    edge is the weighted fraction of the blur disk on each side; pixels whose
    disk avoids the edge are exact.  1024 weighted samples: within
    4 (1 + a) (contrast / 2) / sqrt(N), and unlike the unweighted image."""
    z, zf, A, ab = 1.0, 2.0, 0.2, 0.8
    W = H = 20
    cam = hi.Camera(width=W, height=H).f32()
    lens = hi.Lens(zf, A, 0.05).f32()
    p = hi.Params(spp_max=128, aberration=ab)
    osc = orc.OScene(hi.plane_scene(z, half=50.0, cells=2.0))  # cell edges at X = 0 and Y = 0
    t = cam.tan_half_fovy
    R = lens.aperture_radius * H * (lens.focus_dist - z) / (z * lens.focus_dist * t) / 2
    irr = p.k_ambient + max(0.0, -p.unit_lights()[0][2])
    lo, hi_ = float(np.float32(0.2)) * irr, float(np.float32(0.8)) * irr
    spp = np.full((H, W), 128, np.uint8)
    est = np.mean([orc.trace(osc, cam, lens, p.replace(frame=k), spp)[..., 0] for k in range(8)], 0)
    flat = np.mean([orc.trace(osc, cam, lens, p.replace(frame=k, aberration=0.0), spp)[..., 0] for k in range(8)], 0)
    rows = [j for j in range(H) if abs(j + 0.5 - H / 2) > R + 1]  # away from the horizontal edge at Y = 0
    tol = 4 * (1 + ab) * (hi_ - lo) / 2 / math.sqrt(1024)
    e_w, e_flat = [], []
    for j in rows:
        upper = j + 0.5 < H / 2  # screen rows above the centre see Y > 0
        for i in range(W):
            h = W / 2 - (i + 0.5)  # screen offset of the edge X = 0 from the pixel centre
            fr = _weighted_fraction(h, R, ab)  # weighted share of the disk right of the edge
            right, left = (lo, hi_) if upper else (hi_, lo)  # checker parity of the two cells
            exp = fr * right + (1 - fr) * left
            if abs(h) >= R:
                assert abs(est[j, i] - exp) < 1e-12
            else:
                assert abs(est[j, i] - exp) <= tol, (i, j, est[j, i], exp)
                e_w.append(abs(est[j, i] - exp))
                e_flat.append(abs(flat[j, i] - exp))
    # the weights change the image next to the edge: the unweighted estimate misses it
    assert np.mean(e_w) < 0.5 * np.mean(e_flat), (np.mean(e_w), np.mean(e_flat))


def test_shaped_postfilter_orientation_and_unit_scatter(orc):
    """One near source pixel (z = 0.5) on an in-focus background, triangular
    aperture with a vertex up in the lens plane: its near bokeh points down on
    the screen (mirrored left-right), so a receiver 0.8 r below it is covered
    and one 0.8 r above is not; a far source's bokeh points up.  Every source
    scatters a total near-layer weight of exactly 1."""
    W, H = 41, 41
    t = math.tan(math.radians(30))
    lens = hi.Lens(2.0, 0.12, 0.05)
    p = hi.Params(r_max=16.0, blades=3, blade_rot=math.pi / 2)
    nd = np.zeros((H, W, 4))
    nd[..., 2] = -1.0
    nd[..., 3] = 2.0
    nd[20, 20, 3] = 0.5
    col = np.zeros((H, W, 4))
    r = abs(orc.coc(0.5, lens, H, t)) / 2
    assert 5 < r < 9
    pp = orc.postfilter(nd, col, lens, t, p)
    k = int(round(0.8 * r))
    # background receivers cover themselves by 1/2 (in focus: w_near = 1/2, r = 0)
    assert pp[20 + k, 20, 3] > 0.5 and pp[20 - k, 20, 3] == 0.5
    others = np.ones((H, W), bool)
    others[20, 20] = False
    # background pixels weigh 1/2 on themselves (in focus: w_near = 1/2, r = 0)
    total = pp[..., 3].sum() - 0.5 * others.sum()
    assert abs(total - 1.0) < 1e-12
    # a far source (z = 8 with the focus at 2): its bokeh points up
    nd2 = nd.copy()
    nd2[20, 20, 3] = 2.0
    lens2 = hi.Lens(2.0, 0.3, 0.05)
    rf = abs(orc.coc(8.0, lens2, H, t)) / 2
    nd2[..., 3] = 8.0
    col2 = np.zeros((H, W, 4))
    col2[20, 20, :3] = 1.0
    pp2 = orc.postfilter(nd2, col2, lens2, t, p)
    kf = int(round(0.8 * rf))
    assert pp2[20 - kf, 20, 0] > pp2[20 + kf, 20, 0] and pp2[20 + kf, 20, 0] == 0.0


def test_shaped_area_limits(orc):
    """The weighted lattice area of the soft shape approaches its continuous
    integral: the N-gon's area (N / 2) r^2 sin(2 pi / N) without weights, and
    pi (r^2 + 1/12) for the weighted disk (mean weight 1)."""
    for N in (3, 5, 6):
        p = hi.Params(blades=N, blade_rot=0.3)
        for r in (20.0, 31.7):
            cont = 0.5 * N * r * r * math.sin(2 * math.pi / N)
            assert abs(orc.shaped_area(r, p) - cont) < 0.01 * cont
    for a in (-1.0, 0.5, 1.0):
        p = hi.Params(aberration=a)
        for r in (20.0, 31.7):
            cont = math.pi * (r * r + 1.0 / 12.0)
            assert abs(orc.shaped_area(r, p) - cont) < 0.01 * cont
    assert orc.shaped_area(12.3, hi.Params()) == orc.disk_area(12.3)


# ----------------------------------------- specular highlight and preference

def _glossy_plane(z, ks, cells=40.0):
    s = hi.plane_scene(z, half=50.0, cells=cells)
    s.mat = s.mat.copy()
    s.mat[:, 7] = ks
    return s


def test_blinn_phong_highlight_of_a_plane_lit_from_the_eye(orc):
    """A fronto-parallel plane seen from the origin and lit from the camera's
    side (w = -fwd): for the ray at angle theta to the axis the half vector of
    light and viewer bisects them, so n . h = cos(theta / 2) and the highlight
    is k_s E cos(theta/2)^32 = k_s E ((1 + cos theta) / 2)^16; the diffuse part
    is the albedo (0.2 or 0.8) times n . w = 1.  With k_s = 0 the highlight is
    0 and the colour is the diffuse part alone."""
    W, H, z, ks = 24, 16, 2.0, 3.0
    cam = hi.Camera(width=W, height=H).f32()
    p = hi.Params(k_ambient=0.0, light_dir=[[0.0, 0.0, -1.0]], light_E=[1.0])
    g = orc.gbuffer(orc.OScene(_glossy_plane(z, ks)), cam, cam, p)
    t = cam.tan_half_fovy
    sx = (2.0 * (np.arange(W) + 0.5) / W - 1.0) * t * W / H
    sy = (2.0 * (np.arange(H) + 0.5) / H - 1.0) * t
    tan2 = sx[None, :] ** 2 + sy[:, None] ** 2
    cos_t = 1.0 / np.sqrt(1.0 + tan2)
    S = ks * ((1.0 + cos_t) / 2.0) ** 16
    np.testing.assert_allclose(g["col"][..., 3], S, rtol=1e-10)
    diffuse = g["col"][..., :3] - g["col"][..., 3:4]
    assert np.all(np.isclose(diffuse, 0.2, atol=1e-10) | np.isclose(diffuse, 0.8, atol=1e-10))
    g0 = orc.gbuffer(orc.OScene(_glossy_plane(z, 0.0)), cam, cam, p)
    assert np.all(g0["col"][..., 3] == 0.0)
    np.testing.assert_allclose(g0["col"][..., :3], diffuse, atol=1e-12)


def test_no_highlight_from_a_light_behind_the_surface(orc):
    """A light behind the plane (w . n < 0 for the normal facing the camera)
    gives neither diffuse light nor a highlight: the colour is the ambient
    term alone, whatever k_s."""
    W, H = 12, 10
    cam = hi.Camera(width=W, height=H).f32()
    p = hi.Params(k_ambient=0.25, light_dir=[[0.2, 0.1, 1.0]], light_E=[2.0])
    g = orc.gbuffer(orc.OScene(_glossy_plane(2.0, 5.0)), cam, cam, p)
    assert np.all(g["col"][..., 3] == 0.0)
    rgb = g["col"][..., :3]
    assert np.all(np.isclose(rgb, 0.25 * 0.2, atol=1e-12) | np.isclose(rgb, 0.25 * 0.8, atol=1e-12))


def test_composite_specular_preference_hand_values(orc):
    """One near, traced, blurred pixel (w_near = 1, focus weight 0): the near
    branch is C_rec moved toward C_pp by clamp(spec_pref S_pp, 0, 1); without
    a specular part or with spec_pref = 0 it is C_rec; an untraced pixel takes
    C_pp whatever the preference."""
    lens = hi.Lens(2.0, 0.05, 0.05)
    t = math.tan(math.radians(30.0))
    H = 128
    z = 0.5
    c = 0.05 * H * (2.0 - z) / (z * 2.0 * t)  # ~16.6 px: w_near = 1
    nd = np.array([[0.0, 0.0, -1.0, z]])
    col = np.array([[0.9, 0.9, 0.9, 0.0]])
    crt = np.array([[0.0, 0.0, 0.0, c]])
    crec = np.array([[1.0, 0.0, 0.2, 0.0]])
    pp = np.array([[0.0, 1.0, 0.6, 1.0]])
    pps = np.array([[0.5, 0.5, 0.5, 1.0]])
    hacc = np.array([1.0])
    traced = np.array([1], np.uint8)

    def comp(spec_pref, spp=traced, pp_spec=pps):
        return orc.composite(nd, col, spp, pp, crt, crec, hacc, lens, t, hi.Params(spec_pref=spec_pref), H,
                             pp_spec=pp_spec)[0, :3]

    np.testing.assert_allclose(comp(1.0), [0.5, 0.5, 0.4], atol=1e-15)
    np.testing.assert_allclose(comp(0.5), [0.75, 0.25, 0.3], atol=1e-15)
    np.testing.assert_allclose(comp(4.0), pp[0, :3], atol=1e-15)
    np.testing.assert_allclose(comp(0.0), crec[0, :3], atol=1e-15)
    np.testing.assert_allclose(comp(1.0, pp_spec=None), crec[0, :3], atol=1e-15)
    np.testing.assert_allclose(comp(1.0, spp=np.array([0], np.uint8)), pp[0, :3], atol=1e-15)


def test_specular_part_of_the_post_process_colour_is_its_share(orc):
    """The post-filter is linear in the colour plane, so filtering the
    specular plane (S, S, S) gives exactly the part of pp that S contributes:
    pp(col) - pp(col - S) over the colour channels."""
    W, Hh = 48, 40
    gb = hi.random_gbuffer(W, Hh, seed=5)
    col = gb["col"].astype(np.float64).copy()
    rng = np.random.default_rng(5)
    S = np.where(rng.random((Hh, W)) < 0.2, rng.uniform(0.5, 3.0, (Hh, W)), 0.0)
    col[..., :3] += S[..., None]
    col[..., 3] = S
    nd = gb["nd"].astype(np.float64)
    lens = hi.Lens(3.0, 0.05, 0.05)
    t = math.tan(math.radians(30.0))
    p = hi.Params(r_max=12.0)
    diffuse = col.copy()
    diffuse[..., :3] -= S[..., None]
    share = orc.postfilter(nd, col, lens, t, p)[..., :3] - orc.postfilter(nd, diffuse, lens, t, p)[..., :3]
    spec = orc.postfilter_spec(nd, col, lens, t, p)
    np.testing.assert_allclose(spec[..., :3], share, atol=1e-12)
    assert spec[..., 0].max() > 0.1  # the highlights do spread
