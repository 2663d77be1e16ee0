"""Batched multi-view frame: one launch per stage over views of different
sizes, scenes, lenses and poses.  Every output plane equals the one the
single-view calls write, bit for bit (the batched kernels run the same
per-block code), for every launch shape the autotuner may pick, over
several frames with history, and when replayed from a captured CUDA graph.
On the 64-view workload sampled views also agree with the oracle."""
import numpy as np
import pytest

import hdof_inputs as hi

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("needs a CUDA device", allow_module_level=True)

import paper_2210_04981_gb300.hdof as H  # noqa: E402
from gpu_util import (bvh_of, check_gbuffer_ids, check_mask_stage, frac_close, history_host, host, report,  # noqa: E402
                      rt_close)

SMALL_RES = ((64, 64), (160, 120), (320, 180), (200, 150), (33, 17))


@pytest.fixture(scope="module")
def small():
    scenes = hi.batch_scenes(tris=(20_000, 40_000, 60_000, 80_000))
    bvhs = [bvh_of(s) for s in scenes]
    views = hi.batch_views(12, resolutions=SMALL_RES)
    return scenes, bvhs, views


def _frame_args(views, k):
    cams = [v.camera(k) for v in views]
    prevs = [v.camera(k - 1) if k else v.camera(0) for v in views]
    lenses = [v.lens for v in views]
    ps = [v.params.replace(frame=k, camera_moved=int(k > 0)) for v in views]
    return cams, prevs, lenses, ps


def _singles(bvhs, views):
    return [H.Renderer(bvhs[v.room], v.width, v.height, v.params) for v in views]


def _run_singles(rs, views, k):
    cams, prevs, lenses, ps = _frame_args(views, k)
    for r, c, pv, ln, p in zip(rs, cams, prevs, lenses, ps):
        r.frame(c, pv, ln, p)


def _assert_same(a: H.Renderer, b: H.Renderer, tag):
    """Bitwise equality of every plane (traced-only planes on traced pixels)."""
    eq = lambda x, y: torch.equal(x.contiguous().view(torch.uint8), y.contiguous().view(torch.uint8))  # noqa
    for name in ("nd", "col", "mv", "tri"):
        assert eq(getattr(a.g, name), getattr(b.g, name)), f"{tag}: gbuffer {name}"
    for name in ("edge", "spp", "pp", "crt", "out", "stats"):
        assert eq(getattr(a, name), getattr(b, name)), f"{tag}: {name}"
    tr = a.spp > 0
    for name in ("rt", "hacc", "crec"):
        assert eq(getattr(a, name)[tr], getattr(b, name)[tr]), f"{tag}: {name}"
    ha, hb = a.history, b.history
    assert eq(ha.hlen, hb.hlen), f"{tag}: hlen"
    for name in ("near", "far", "mom"):
        assert eq(getattr(ha, name)[tr], getattr(hb, name)[tr]), f"{tag}: history {name}"


@pytest.mark.parametrize("block,refill,chunk,tile", [(128, 0, 0, 8), (64, 0, 0, 0), (256, 0, 3, 16), (128, 16, 0, 8),
                                                     (64, 32, 2, 16), (256, 1, 8, 8), (128, 4, 1, 16), (64, 0, 16, 0)])
def test_batch_equals_single_view(small, block, refill, chunk, tile):
    """Every launch shape of the batched frame (trace block and form, queue
    chunk, spatial stencil tile) renders each view bit for bit as the
    single-view calls do."""
    scenes, bvhs, views = small
    rs = _singles(bvhs, views)
    b = H.Batch([bvhs[v.room] for v in views], [(v.width, v.height) for v in views], [v.params for v in views],
                tune=H.tuning(block, refill, chunk, tile))
    for k in range(3):
        _run_singles(rs, views, k)
        b.frame(*_frame_args(views, k))
        H.hdof_sync()
        assert sum(int(r.stats[0]) for r in rs) > 0
        for i, (r, rb) in enumerate(zip(rs, b.views)):
            _assert_same(r, rb, f"frame {k} view {i} ({views[i].width}x{views[i].height})")
    b.close()


def test_batch_per_view_forms_equal_single_view(small):
    """trace_refill -1: the views whose CoC scale K = A H / (zf tan(fovy/2))
    is below 20 pixels are traced as warp packets and the others at ray
    level, in two persistent launches over two ray lists; every view equals
    its single-view calls bit for bit."""
    import dataclasses
    scenes, bvhs, views = small
    wide = hi.Lens(1.0, 0.1, hi.ROOM_FOCAL).f32()
    views = [dataclasses.replace(v, lens=wide) if k % 2 else v for k, v in enumerate(views)]
    t = views[0].camera(0).tan_half_fovy
    K = [v.lens.aperture_radius * v.height / (v.lens.focus_dist * t) for v in views]
    assert any(k < 20 for k in K) and any(k >= 20 for k in K), K
    rs = _singles(bvhs, views)
    b = H.Batch([bvhs[v.room] for v in views], [(v.width, v.height) for v in views], [v.params for v in views],
                tune=H.tuning(128, -1, 0, 8))
    for k in range(3):
        _run_singles(rs, views, k)
        b.frame(*_frame_args(views, k))
        H.hdof_sync()
        assert sum(int(r.stats[1]) for r, kk in zip(rs, K) if kk >= 20) > 0  # the ray-level list is not empty
        for i, (r, rb) in enumerate(zip(rs, b.views)):
            _assert_same(r, rb, f"frame {k} view {i} (K {K[i]:.1f})")
    b.close()


def test_batch_graph_replay(small):
    """render() captured once in a CUDA graph; each frame rewrites the launch
    records (update) and replays the graph."""
    scenes, bvhs, views = small
    rs = _singles(bvhs, views)
    b = H.Batch([bvhs[v.room] for v in views], [(v.width, v.height) for v in views], [v.params for v in views],
                tune=H.tuning(128, 24))
    # warm-up frame outside the capture (loads every kernel), then start over
    b.frame(*_frame_args(views, 0))
    H.hdof_sync()
    for r in b.views:
        r.reset_history()
        r.cur = 0
    b.update(*_frame_args(views, 0))
    g = torch.cuda.CUDAGraph()
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(s):
        with torch.cuda.graph(g, stream=s):
            b.render()
    torch.cuda.current_stream().wait_stream(s)
    for k in range(3):
        if k:
            b.update(*_frame_args(views, k))
        g.replay()
        b.advance()
        _run_singles(rs, views, k)
        H.hdof_sync()
        for i, (r, rb) in enumerate(zip(rs, b.views)):
            _assert_same(r, rb, f"graph frame {k} view {i}")
    b.close()


def test_batch_degenerate_views(small):
    """1x1 and 3x2 views, a ragged 17x16 view and a view of a fronto-parallel
    plane whose mask is empty (no rays at all) in one batch: still equal to
    the single-view calls."""
    scenes, bvhs, _ = small
    plane = bvh_of(hi.plane_scene(2.0))
    base = hi.batch_views(4, resolutions=((8, 8),))
    specs = [(bvhs[0], 1, 1), (bvhs[1], 3, 2), (bvhs[2], 17, 16), (plane, 64, 48)]
    views = []
    for (b, w, h), v in zip(specs, base):
        v.width, v.height = w, h
        views.append(v)
    views[3].pos, views[3].target = (0.0, 0.0, 0.0), (0.0, 0.0, 5.0)
    blist = [b for b, _, _ in specs]
    rs = [H.Renderer(b, v.width, v.height, v.params) for b, v in zip(blist, views)]
    b = H.Batch(blist, [(v.width, v.height) for v in views], [v.params for v in views], tune=H.tuning(64, 2))
    for k in range(2):
        _run_singles(rs, views, k)
        b.frame(*_frame_args(views, k))
        H.hdof_sync()
        for i, (r, rb) in enumerate(zip(rs, b.views)):
            _assert_same(r, rb, f"frame {k} view {i}")
    assert int(rs[3].stats[1]) == 0  # the plane view traced nothing
    b.close()


def test_batch_stage_ranges_equal_full_render(small):
    """Running the seven stages one call each (hdof_batch_render_range) gives
    the same frame as hdof_batch_render; the records upload is counted."""
    scenes, bvhs, views = small
    sub = views[:5]
    a = H.Batch([bvhs[v.room] for v in sub], [(v.width, v.height) for v in sub], [v.params for v in sub])
    b = H.Batch([bvhs[v.room] for v in sub], [(v.width, v.height) for v in sub], [v.params for v in sub])
    for k in range(2):
        a.frame(*_frame_args(sub, k))
        b.update(*_frame_args(sub, k))
        for st in range(len(H.BATCH_STAGES)):
            H.hdof_batch_render_range(b.handle, st, st)
        b.advance()
        H.hdof_sync()
        for i, (ra, rb) in enumerate(zip(a.views, b.views)):
            _assert_same(ra, rb, f"frame {k} view {i}")
    assert b.handle_bytes() > 0 and b.handle_bytes() % 256 == 0
    with pytest.raises(H.HdofError, match="stages"):
        H.hdof_batch_render_range(b.handle, 3, 7)
    a.close()
    b.close()


def test_batch_rejects_changed_sizes(small):
    scenes, bvhs, views = small
    b = H.Batch([bvhs[v.room] for v in views[:2]], [(v.width, v.height) for v in views[:2]],
                [v.params for v in views[:2]])
    b.update(*_frame_args(views[:2], 0))
    recs = b.records(*_frame_args(views[:2], 1))
    recs[1].cam.width += 1
    with pytest.raises(H.HdofError, match="size"):
        H.hdof_batch_update(b.handle, recs)
    with pytest.raises(H.HdofError, match="views"):
        H.hdof_batch_update(b.handle, recs[:1])
    b.close()


@pytest.fixture(scope="module")
def orc():
    from oracle import oracle
    oracle.build()
    return oracle


def test_batch_64_views_full_workload(orc):
    """The 64-view workload at its full sizes (4 rooms of 50k-500k
    triangles, 256^2 to 1920x1080) in the launch configuration the benchmark
    times: every view bitwise equal to the single-view calls, and one view of
    each room against the oracle (mask, trace, reconstruction in full; the
    post-filter and composite on 4000 sampled pixels)."""
    scenes = hi.batch_scenes()
    bvhs = [bvh_of(s) for s in scenes]
    views = hi.batch_views(64)
    b = H.Batch([bvhs[v.room] for v in views], [(v.width, v.height) for v in views], [v.params for v in views],
                tune=H.tuning(128, 16))
    b.frame(*_frame_args(views, 0))
    H.hdof_sync()
    # single-view calls, a few views at a time (memory)
    for lo in range(0, 64, 16):
        rs = _singles(bvhs, views[lo:lo + 16])
        _run_singles(rs, views[lo:lo + 16], 0)
        H.hdof_sync()
        for i, r in enumerate(rs):
            _assert_same(r, b.views[lo + i], f"view {lo + i}")
        del rs
    # oracle: the smallest view of each room
    picks = []
    for room in range(4):
        cand = [i for i, v in enumerate(views) if v.room == room]
        picks.append(min(cand, key=lambda i: views[i].width * views[i].height))
    cams, prevs, lenses, ps = _frame_args(views, 0)
    for i in picks:
        v, r = views[i], b.views[i]
        W, Hh = v.width, v.height
        pix = np.random.default_rng(i).choice(W * Hh, min(4000, W * Hh), replace=False).astype(np.int32)
        ref = orc.frame(orc.OScene(scenes[v.room]), cams[i], prevs[i], lenses[i], ps[i], pp_pix=pix)
        spp = host(r.spp)
        check_gbuffer_ids(orc, scenes[v.room], cams[i], host(r.g.tri), ref["g"]["tri"], f"view {i}")
        check_mask_stage(orc, ps[i], host(r.g.nd), host(r.g.mv), host(r.edge), spp, history_host(r.hist[1 - r.cur]),
                         f"view {i}")
        tr = (spp > 0) & (spp == ref["mask"]["spp"])
        assert tr.any()
        ok = rt_close(host(r.rt), ref["rt"], tr)
        assert ok.mean() >= 0.999, f"view {i}: rt {ok.mean():.5f}"
        assert frac_close(host(r.crt)[tr], ref["crt"][tr], 1e-3, 1e-3) >= 0.999
        pp = host(r.pp).reshape(-1, 4)[pix]
        assert frac_close(pp, ref["pp"], 1e-4) >= 0.999, report("pp", pp, ref["pp"])
        out = host(r.out).reshape(-1, 4)[pix][:, :3]
        assert frac_close(out, ref["out"][:, :3], 1e-3) >= 0.999, report("out", out, ref["out"][:, :3])
    b.close()
