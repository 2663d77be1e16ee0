"""Specular materials and the Composite section's specular-bokeh preference on
the GPU against the oracle: the Blinn-Phong highlight in the G-buffer (its
luminance in col.w) and in the thin-lens trace, the post-filter of the
specular plane, the composite's near branch moved toward the post-process
colour by clamp(spec_pref S_pp, 0, 1), and a whole frame of a glossy scene.
Tolerances as for the Lambertian stages: G-buffer 1e-4 (the highlight's
power 32 amplifies float rounding of n . h), trace radiance 1e-3 on >= 99.9%
of traced pixels, post-filter 1e-4, composite 1e-5."""
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
from test_gpu_parity import _frame_check  # noqa: E402


@pytest.fixture(scope="module")
def orc():
    from oracle import oracle
    oracle.build()
    return oracle


def test_gbuffer_highlights(orc):
    scene, cam, lens, p = hi.specular_config()
    bvh = bvh_of(scene)
    g = H.GBuffer(cam.width, cam.height)
    H.hdof_gbuffer(bvh, cam, cam, p, g)
    H.hdof_sync()
    ref = orc.gbuffer(orc.OScene(scene), cam, cam, p)
    same = host(g.tri) == ref["tri"]
    assert same.mean() > 0.99
    col, rcol = host(g.col)[same], ref["col"][same]
    assert frac_close(col, rcol, 1e-4, rtol=1e-4) >= 0.999, report("col", col, rcol)
    assert rcol[:, 3].max() > 1.0  # the highlights are there and bright
    # a Lambertian scene keeps col.w = 0
    s0, c0, _, p0 = hi.tiny_config()
    g0 = H.GBuffer(c0.width, c0.height)
    H.hdof_gbuffer(bvh_of(s0), c0, c0, p0, g0)
    H.hdof_sync()
    assert float(g0.col[..., 3].abs().max()) == 0.0


def test_trace_highlights(orc):
    scene, cam, lens, p = hi.specular_config()
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


@pytest.mark.parametrize("W,Hh,rmax,col_dtype", [(96, 64, 16.0, torch.float32), (77, 53, 12.0, torch.float32),
                                                  (64, 48, 20.0, torch.bfloat16)])
def test_postfilter_spec(orc, W, Hh, rmax, col_dtype):
    gb = hi.random_gbuffer(W, Hh, seed=W)
    col = gb["col"].astype(np.float32).copy()
    rng = np.random.default_rng(W)
    S = np.where(rng.random((Hh, W)) < 0.15, rng.uniform(0.5, 4.0, (Hh, W)), 0.0).astype(np.float32)
    col[..., 3] = S
    cam = hi.Camera(width=W, height=Hh).f32()
    lens = hi.Lens(3.0, 0.05, 0.05).f32()
    p = hi.Params(r_max=rmax, spec_pref=1.0)
    g = gbuf_from(gb["nd"], col, col_dtype=col_dtype)
    out = torch.empty((Hh, W, 4), dtype=torch.float32, device="cuda")
    H.hdof_postfilter_spec(g, cam, lens, p, out, workspace(W, Hh, p))
    H.hdof_sync()
    col_seen = host(g.col.float()).astype(np.float64)  # what the kernel read (bf16-rounded)
    ref = orc.postfilter_spec(gb["nd"].astype(np.float64), col_seen, lens, cam.tan_half_fovy, p)
    assert frac_close(host(out), ref, 1e-4) >= 0.999, report("pp_spec", host(out), ref)
    assert ref[..., 0].max() > 0.1


def test_composite_spec(orc):
    W, Hh = 97, 61
    gb = hi.random_gbuffer(W, Hh, seed=3)
    rng = np.random.default_rng(3)
    spp = (rng.random((Hh, W)) < 0.5).astype(np.uint8) * 4
    pp = rng.random((Hh, W, 4)).astype(np.float32)
    pps = np.repeat(rng.uniform(0.0, 3.0, (Hh, W, 1)), 4, -1).astype(np.float32)
    crt = rng.random((Hh, W, 4)).astype(np.float32)
    crt[..., 3] = rng.uniform(0.0, 20.0, (Hh, W))
    crec = rng.random((Hh, W, 4)).astype(np.float32)
    hacc = rng.random((Hh, W)).astype(np.float32)
    cam = hi.Camera(width=W, height=Hh).f32()
    lens = hi.Lens(3.0, 0.08, 0.05).f32()
    g = gbuf_from(gb["nd"], gb["col"])
    for sp in (0.0, 0.4, 2.0):
        p = hi.Params(spec_pref=sp)
        out = torch.empty((Hh, W, 4), dtype=torch.float32, device="cuda")
        H.hdof_composite_spec(g, dev(spp), dev(pp), dev(pps), dev(crt), dev(crec), dev(hacc), cam, lens, p, out)
        H.hdof_sync()
        ref = orc.composite(gb["nd"], gb["col"], spp, pp, crt, crec, hacc, lens, cam.tan_half_fovy, p, Hh,
                            pp_spec=pps)
        assert frac_close(host(out)[..., :3], ref[..., :3], 1e-5) == 1.0, report("out", host(out), ref)
        if sp == 0.0:  # equals the plain composite
            out0 = torch.empty_like(out)
            H.hdof_composite(g, dev(spp), dev(pp), dev(crt), dev(crec), dev(hacc), cam, lens, p, out0)
            H.hdof_sync()
            assert torch.equal(out0, out)


def test_frame_glossy_with_preference(orc):
    scene, cam, lens, p = hi.specular_config()
    r = H.Renderer(bvh_of(scene), cam.width, cam.height, p)
    r.frame(cam, cam, lens, p)
    H.hdof_sync()
    ref = orc.frame(orc.OScene(scene), cam, cam, lens, p)
    assert np.array_equal(host(r.spp), ref["mask"]["spp"])
    ps = host(r.pp_spec)
    assert frac_close(ps, ref["pp_spec"], 1e-4) >= 0.999, report("pp_spec", ps, ref["pp_spec"])
    _frame_check(orc, scene, cam, p, r, ref, "glossy")


def test_preference_lowers_the_noise_of_near_highlights(orc):
    """Two frames of the glossy scene with different lens-sample seeds: where
    the preference is active the output's seed-to-seed difference shrinks
    (the post-process colour does not depend on the seed)."""
    scene, cam, lens, p = hi.specular_config()
    bvh = bvh_of(scene)

    def run(sp, seed):
        q = p.replace(spec_pref=sp, seed=seed)
        r = H.Renderer(bvh, cam.width, cam.height, q)
        r.frame(cam, cam, lens, q)
        H.hdof_sync()
        return host(r.out)[..., :3], host(r.pp_spec) if sp > 0 else None

    a0, _ = run(0.0, 1)
    b0, _ = run(0.0, 2)
    a1, ps = run(4.0, 1)
    b1, _ = run(4.0, 2)
    act = ps[..., 0] * 4.0 > 0.5
    assert act.sum() > 20
    d0 = np.abs(a0 - b0)[act].mean()
    d1 = np.abs(a1 - b1)[act].mean()
    assert d1 < 0.7 * d0, (d0, d1)


def test_spec_pref_rejections(orc):
    scene, cam, lens, p = hi.specular_config()
    r = H.Renderer(bvh_of(scene), cam.width, cam.height, p)
    with pytest.raises(H.HdofError) as e:
        H.Batch([r.bvh], [(cam.width, cam.height)], [p]).frame([cam], [cam], [lens], [p])
    assert e.value.code == -5
    with pytest.raises(H.HdofError) as e:
        H.hdof_composite_spec(r.g, r.spp, r.pp, r.pp, r.crt, r.crec, r.hacc, cam, lens,
                              p.replace(spec_pref=-1.0), r.out)
    assert e.value.code == -1
    # specular materials themselves render in batches, equal to the single-view frame
    q = p.replace(spec_pref=0.0)
    b = H.Batch([r.bvh], [(cam.width, cam.height)], [q])
    b.frame([cam], [cam], [lens], [q])
    r.frame(cam, cam, lens, q)
    H.hdof_sync()
    assert torch.equal(b.views[0].out, r.out)
