"""Full ray-traced reference frames and error maps on the GPU.

* hdof_reference_rt equals the oracle's full ray-traced image (mean radiance
  over every lens sample of every pass) within 1e-3 on >= 99.9% of pixels,
  on the tiny scene and a room;
* hdof_error_map equals the plain numpy definition of its outputs;
* the paper's claim, as a check on the tiny scene: next to the blurry
  occluder's edge (the traced pixels) the hybrid frame is closer to the full
  ray-traced image than the post-process alone.
"""
import numpy as np
import pytest

import hdof_inputs as hi

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("needs a CUDA device", allow_module_level=True)

import paper_2210_04981_gb300.hdof as H  # noqa: E402
from gpu_util import bvh_of, dev, frac_close, host, report, workspace  # noqa: E402


@pytest.fixture(scope="module")
def orc():
    from oracle import oracle
    oracle.build()
    return oracle


def _reference(bvh, cam, lens, p, passes, hint=None):
    out = torch.full((cam.height, cam.width, 4), float("nan"), dtype=torch.float32, device="cuda")
    H.hdof_reference_rt(bvh, cam, lens, p, passes, out, workspace(cam.width, cam.height, p), hint=hint)
    H.hdof_sync()
    return host(out)


def test_reference_rt_tiny(orc):
    scene, cam, lens, p = hi.tiny_config()
    got = _reference(bvh_of(scene), cam, lens, p, 3)
    ref = orc.reference_rt(orc.OScene(scene), cam, lens, p, 3)
    assert frac_close(got[..., :3], ref[..., :3], 1e-3) >= 0.999, report("rt", got[..., :3], ref[..., :3])
    assert np.all(got[..., 3] == 0)


def test_reference_rt_room(orc):
    W, Hh = 240, 136
    scene, cams, lens, p0 = hi.room_config(W, Hh, frames=2)
    p = p0.replace(frame=1, spp_max=6)
    bvh = bvh_of(scene)
    g = H.GBuffer(W, Hh)
    H.hdof_gbuffer(bvh, cams[1], cams[0], p, g)
    got = _reference(bvh, cams[1], lens, p, 2, hint=g.tri)
    ref = orc.reference_rt(orc.OScene(scene), cams[1], lens, p, 2)
    assert frac_close(got[..., :3], ref[..., :3], 1e-3) >= 0.999, report("rt", got[..., :3], ref[..., :3])


def test_error_map_matches_numpy():
    rng = np.random.default_rng(0)
    W, Hh = 333, 77
    a = rng.uniform(0, 1, (Hh, W, 4)).astype(np.float32)
    b = rng.uniform(0, 1, (Hh, W, 4)).astype(np.float32)
    region = (rng.uniform(size=(Hh, W)) < 0.3).astype(np.uint8)
    err = torch.empty((Hh, W), dtype=torch.float32, device="cuda")
    stats = torch.empty(H.ERR_SCRATCH, dtype=torch.float64, device="cuda")
    H.hdof_error_map(dev(a), dev(b), stats, region=dev(region), err=err)
    H.hdof_sync()
    d = np.abs(a[..., :3].astype(np.float64) - b[..., :3])
    np.testing.assert_allclose(host(err), d.mean(-1), rtol=1e-6, atol=1e-7)
    st = host(stats)[:8]
    m = region > 0
    want = [d.shape[0] * d.shape[1], d.sum(), (d * d).sum(), d.max(), m.sum(), d[m].sum(), (d[m] ** 2).sum(), d[m].max()]
    np.testing.assert_allclose(st, want, rtol=1e-5)
    # deterministic: the same inputs give the same bits
    H.hdof_error_map(dev(a), dev(b), stats, region=dev(region))
    H.hdof_sync()
    assert np.array_equal(host(stats)[:8], st)
    s = H.error_summary(stats)
    assert abs(s["all"]["mae"] - d.mean()) < 1e-6 and s["region"]["pixels"] == int(m.sum())


def test_hybrid_beats_post_process_near_blurry_edges():
    """Against a 256-sample full ray-traced frame, the hybrid frame's error on
    the traced pixels (the occluder's blurry silhouette), after four frames
    of a static camera, is well below the post-process-only frame's (the
    same composite with no traced pixels), while away from them the two
    frames are identical."""
    scene, cam, lens, p = hi.tiny_config()
    bvh = bvh_of(scene)
    r = H.Renderer(bvh, cam.width, cam.height, p)
    for k in range(4):
        r.frame(cam, cam, lens, p.replace(frame=k))
    zero = torch.zeros_like(r.spp)
    pp_only = torch.empty_like(r.out)
    H.hdof_composite(r.g, zero, r.pp, r.crt, r.crec, r.hacc, cam, lens, p, pp_only)
    rt = torch.empty_like(r.out)
    H.hdof_reference_rt(bvh, cam, lens, p, 16, rt, r.ws, hint=r.g.tri)
    stats = torch.empty(H.ERR_SCRATCH, dtype=torch.float64, device="cuda")
    traced = (r.spp > 0).to(torch.uint8)
    H.hdof_error_map(r.out, rt, stats, region=traced)
    hyb = H.error_summary(stats)
    H.hdof_error_map(pp_only, rt, stats, region=traced)
    pp = H.error_summary(stats)
    H.hdof_sync()
    assert hyb["region"]["pixels"] > 1000
    assert hyb["region"]["mae"] < 0.5 * pp["region"]["mae"], (hyb, pp)
    untraced = host(r.spp) == 0
    assert np.array_equal(host(r.out)[untraced, :3], host(pp_only)[untraced, :3])
