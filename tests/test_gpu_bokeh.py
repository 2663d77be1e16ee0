"""Shaped bokeh on the GPU against the oracle: lens samples over aperture
polygons with radial weights in the thin-lens trace and the full ray-traced
frame, and the shaped post-filter (mirrored aperture shapes, radial weights,
their lattice area).  Tolerances as for the circular forms: trace output per
traced pixel (radiance 1e-3) on >= 99.9% of pixels, post-filter 1e-4."""
import math

import numpy as np
import pytest

import hdof_inputs as hi

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("needs a CUDA device", allow_module_level=True)

import paper_2210_04981_gb300.hdof as H  # noqa: E402
from gpu_util import bvh_of, dev, frac_close, gbuf_from, host, report, rt_close, workspace  # noqa: E402

SHAPES = [dict(blades=3, blade_rot=math.pi / 2), dict(blades=6, blade_rot=0.2, aberration=0.6),
          dict(aberration=-0.7), dict(blades=5, blade_rot=1.0, aberration=1.0)]


@pytest.fixture(scope="module")
def orc():
    from oracle import oracle
    oracle.build()
    return oracle


@pytest.mark.parametrize("shape", SHAPES)
def test_trace_shaped_tiny(orc, shape):
    scene, cam, lens, p = hi.tiny_config()
    p = p.replace(**shape)
    osc = orc.OScene(scene)
    g = orc.gbuffer(osc, cam, cam, p)
    spp = orc.mask(g["nd"], g["mv"], p)["spp"]
    rt = torch.full((cam.height, cam.width, 12), float("nan"), dtype=torch.float32, device="cuda")
    stats = torch.zeros(2, dtype=torch.int32, device="cuda")
    H.hdof_trace(bvh_of(scene), cam, lens, p, dev(spp), rt, stats, workspace(cam.width, cam.height, p))
    H.hdof_sync()
    ref = orc.trace(osc, cam, lens, p, spp)
    traced = spp > 0
    ok = rt_close(host(rt), ref, traced)
    assert ok.mean() >= 0.999, f"{(~ok).sum()} of {ok.size}; " + report("rt", host(rt)[traced], ref[traced])
    # the shape changes the image (against the uniform disk)
    ref0 = orc.trace(osc, cam, lens, hi.tiny_config()[3], spp)
    assert np.abs(ref[traced][:, :3] - ref0[traced][:, :3]).max() > 0.01


@pytest.mark.parametrize("shape", SHAPES[:2])
def test_reference_rt_shaped(orc, shape):
    scene, cam, lens, p = hi.tiny_config()
    p = p.replace(**shape)
    out = torch.empty((cam.height, cam.width, 4), dtype=torch.float32, device="cuda")
    H.hdof_reference_rt(bvh_of(scene), cam, lens, p, 2, out, workspace(cam.width, cam.height, p))
    H.hdof_sync()
    ref = orc.reference_rt(orc.OScene(scene), cam, lens, p, 2)
    assert frac_close(host(out)[..., :3], ref[..., :3], 1e-3) >= 0.999, report("rt", host(out), ref)


@pytest.mark.parametrize("shape,W,Hh,rmax,A", [(SHAPES[0], 96, 64, 16.0, 0.03), (SHAPES[1], 77, 53, 12.0, 0.05),
                                               (SHAPES[2], 64, 48, 20.0, 0.04), (SHAPES[3], 90, 70, 24.0, 0.06)])
def test_postfilter_shaped(orc, shape, W, Hh, rmax, A):
    gb = hi.random_gbuffer(W, Hh, seed=W)
    cam = hi.Camera(width=W, height=Hh).f32()
    lens = hi.Lens(3.0, A, 0.05).f32()
    p = hi.Params(r_max=rmax, **shape)
    pp = torch.empty((Hh, W, 4), dtype=torch.float32, device="cuda")
    H.hdof_postfilter(gbuf_from(gb["nd"], gb["col"]), cam, lens, p, pp, workspace(W, Hh, p))
    H.hdof_sync()
    ref = orc.postfilter(gb["nd"].astype(np.float64), gb["col"].astype(np.float64), lens, cam.tan_half_fovy, p)
    assert frac_close(host(pp), ref, 1e-4) >= 0.999, report("pp", host(pp), ref)
    circ = orc.postfilter(gb["nd"].astype(np.float64), gb["col"].astype(np.float64), lens, cam.tan_half_fovy,
                          hi.Params(r_max=rmax))
    assert np.abs(ref[..., :3] - circ[..., :3]).max() > 1e-3  # the shape changes the filter


def test_shaped_bokeh_frame_and_rejections(orc):
    """A whole frame with a hexagonal, rim-weighted aperture against the
    oracle's; batches and the differentiable path reject shaped apertures."""
    scene, cam, lens, p = hi.tiny_config()
    p = p.replace(blades=6, blade_rot=0.3, aberration=0.5)
    r = H.Renderer(bvh_of(scene), cam.width, cam.height, p)
    r.frame(cam, cam, lens, p)
    H.hdof_sync()
    ref = orc.frame(orc.OScene(scene), cam, cam, lens, p)
    assert np.array_equal(host(r.spp), ref["mask"]["spp"])
    out = host(r.out)[..., :3]
    assert frac_close(out, ref["out"][..., :3], 1e-3) >= 0.999, report("out", out, ref["out"][..., :3])
    with pytest.raises(H.HdofError) as e:
        H.Batch([r.bvh], [(cam.width, cam.height)], [p]).frame([cam], [cam], [lens], [p])
    assert e.value.code == -5
