"""Mixed-precision storage (FP16 normal/depth, BF16 colour and post-filter
records, FP32 accumulation, FP32 intersection and lens sampling) against the
FP64 oracle, next to the FP32 plain form on the same inputs.

The bounds follow from the storage formats: FP16 keeps 11 significant bits
(relative error <= 2^-11 ~ 4.9e-4 on normals and depth), BF16 keeps 8
(<= 2^-8 ~ 3.9e-3 on colour).  Radiance is <= 1, so the composite error is
bounded by a few BF16 steps; mask decisions move only where the FP16 metric
crosses the threshold.
"""
import numpy as np
import pytest

import hdof_inputs as hi

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("needs a CUDA device", allow_module_level=True)

import paper_2210_04981_gb300.hdof as H  # noqa: E402
from gpu_util import bvh_of, host  # noqa: E402

F16_REL = 2.0 ** -11
BF16_REL = 2.0 ** -8


@pytest.fixture(scope="module")
def orc():
    from oracle import oracle
    oracle.build()
    return oracle


def _err(a, b):
    d = np.abs(a - b)
    return float(d.max()), float(np.percentile(d, 99.9))


def test_mixed_storage_gbuffer_exact_rounding(orc):
    """The FP16/BF16 G-buffer planes are the FP32 planes rounded once."""
    W, Hh = 320, 180
    scene = hi.room_scene(seed=0, aspect=W / Hh)
    cam = hi.room_camera(0, W, Hh)
    p = hi.room_params()
    bvh = bvh_of(scene)
    g32 = H.GBuffer(W, Hh)
    gmx = H.GBuffer(W, Hh, nd_dtype=torch.float16, col_dtype=torch.bfloat16)
    H.hdof_gbuffer(bvh, cam, cam, p, g32)
    H.hdof_gbuffer(bvh, cam, cam, p, gmx)
    H.hdof_sync()
    assert torch.equal(g32.nd.half(), gmx.nd)
    assert torch.equal(g32.col.bfloat16(), gmx.col)
    assert torch.equal(g32.tri, gmx.tri)


def test_mixed_room_sequence_error_report(orc):
    """Room at 480x270, 4 frames with motion: per-output error of the mixed
    and FP32 forms against the oracle."""
    W, Hh = 480, 270
    scene, cams, lens, p0 = hi.room_config(W, Hh, frames=4)
    osc = orc.OScene(scene)
    bvh = bvh_of(scene)
    r32 = H.Renderer(bvh, W, Hh, p0)
    rmx = H.Renderer(bvh, W, Hh, p0, nd_dtype=torch.float16, col_dtype=torch.bfloat16)
    hist = None
    report = {}
    for k in range(4):
        p = p0.replace(frame=k, camera_moved=int(k > 0))
        prev = cams[k - 1] if k else cams[0]
        r32.frame(cams[k], prev, lens, p)
        rmx.frame(cams[k], prev, lens, p)
        H.hdof_sync()
        ref = orc.frame(osc, cams[k], prev, lens, p, hist=hist)
        hist = ref["hist"]
        nd = host(rmx.g.nd)
        z_rel = np.abs(nd[..., 3] - ref["g"]["nd"][..., 3]) / ref["g"]["nd"][..., 3]
        same_hit = host(rmx.g.tri) == ref["g"]["tri"]
        report[k] = {
            "z_rel": float(np.percentile(z_rel[same_hit], 99.9)),
            "col_rel": float((np.abs(host(rmx.g.col)[same_hit][:, :3] - ref["g"]["col"][same_hit][:, :3]) /
                              np.maximum(ref["g"]["col"][same_hit][:, :3], 1e-3)).max()),
            "spp_agree": float((host(rmx.spp) == ref["mask"]["spp"]).mean()),
            "out_mixed": _err(host(rmx.out)[..., :3], ref["out"][..., :3]),
            "out_f32": _err(host(r32.out)[..., :3], ref["out"][..., :3]),
        }
        assert report[k]["z_rel"] <= F16_REL * 1.01
        assert report[k]["col_rel"] <= BF16_REL * 1.001
        assert report[k]["spp_agree"] >= 0.99
        # composite: a few BF16 steps of colour on 99.9% of pixels
        assert report[k]["out_mixed"][1] <= 4 * BF16_REL, report[k]
        assert report[k]["out_f32"][1] <= 1e-3, report[k]
    print("mixed-precision error report:", report)


def test_mixed_4k_crop_error_report(orc):
    """The 4K mixed-precision workload (5.25M triangles, 3840x2160): frame 0
    in FP32 and in FP16/BF16 storage against the FP64 oracle on the central
    512x512 crop (post-filter and composite on 8192 sampled crop pixels)."""
    W, Hh = 3840, 2160
    scene = hi.room4k_scene(seed=0, aspect=W / Hh)
    cam = hi.room_camera(0, W, Hh)
    lens = hi.room_lens()
    p = hi.room_params(r_max=64.0)
    bvh = bvh_of(scene)
    r32 = H.Renderer(bvh, W, Hh, p)
    rmx = H.Renderer(bvh, W, Hh, p, nd_dtype=torch.float16, col_dtype=torch.bfloat16)
    r32.frame(cam, cam, lens, p)
    rmx.frame(cam, cam, lens, p)
    H.hdof_sync()
    y0, x0 = (Hh - 512) // 2, (W - 512) // 2
    crop = (slice(y0, y0 + 512), slice(x0, x0 + 512))
    rng = np.random.default_rng(5)
    cy, cx = rng.integers(0, 512, 8192) + y0, rng.integers(0, 512, 8192) + x0
    pix = (cy * W + cx).astype(np.int32)
    ref = orc.frame(orc.OScene(scene), cam, cam, lens, p, pp_pix=pix)
    rep = {}
    for name, r in (("f32", r32), ("mixed", rmx)):
        spp = host(r.spp)
        out = host(r.out).reshape(-1, 4)[pix][:, :3]
        pp = host(r.pp).reshape(-1, 4)[pix]
        rep[name] = {"spp_agree": float((spp[crop] == ref["mask"]["spp"][crop]).mean()),
                     "z_rel": float(np.percentile(np.abs(host(r.g.nd)[crop][..., 3] - ref["g"]["nd"][crop][..., 3]) /
                                                  ref["g"]["nd"][crop][..., 3], 99.9)),
                     "pp": _err(pp, ref["pp"]), "out": _err(out, ref["out"][:, :3])}
    print("4K crop error report:", rep)
    assert rep["f32"]["spp_agree"] >= 0.999 and rep["f32"]["out"][1] <= 1e-3
    assert rep["mixed"]["spp_agree"] >= 0.99 and rep["mixed"]["out"][1] <= 4 * BF16_REL
    assert rep["mixed"]["z_rel"] <= F16_REL * 1.01
