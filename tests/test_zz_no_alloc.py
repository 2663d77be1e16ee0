"""hdof_mask_noalloc: the mask call for callers that cannot allocate device
memory for the library (e.g. a real-time render thread that must not call
cudaMalloc, or a host that owns all device memory in its own arena).  Its
output must equal hdof_mask's on consecutive calls, so the fixed tile array
it reuses is cleared between calls.  Collected last on purpose."""
import numpy as np
import pytest

import hdof_inputs as hi

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("needs a CUDA device", allow_module_level=True)

import paper_2210_04981_gb300.hdof as H  # noqa: E402


def _gbuf(gb):
    return H.GBuffer.from_tensors(torch.from_numpy(gb["nd"]).cuda(), torch.from_numpy(gb["col"]).cuda(),
                                  torch.from_numpy(gb["mv"]).cuda())


def _hist(h):
    return H.History.from_tensors(*(torch.from_numpy(h[k]).cuda() for k in ("near", "far", "mom", "hlen")))


def test_noalloc_mask_matches_mask_on_consecutive_calls():
    W, Hh = 333, 201
    p = hi.room_params(spp_max=8)
    # first call: many edges (most tiles flagged); second: few edges and the
    # variance term, so stale flags from the first call would show up
    inputs = [(hi.random_gbuffer(W, Hh, seed=21, n_regions=40), None),
              (hi.random_gbuffer(W, Hh, seed=22, n_regions=1), hi.random_history(W, Hh, seed=23))]
    for gb, hist in inputs:
        g = _gbuf(gb)
        hs = _hist(hist) if hist is not None else None
        e_ref = torch.empty((Hh, W), dtype=torch.uint8, device="cuda")
        s_ref = torch.empty_like(e_ref)
        ws = torch.empty(H.hdof_workspace_bytes(W, Hh, p), dtype=torch.uint8, device="cuda")
        H.hdof_mask(g, hs, p, e_ref, s_ref, ws)
        e = torch.full_like(e_ref, 7)
        s = torch.full_like(e_ref, 7)
        H.hdof_mask_noalloc(g, hs, p, e, s)
        H.hdof_sync()
        assert torch.equal(e, e_ref)
        assert torch.equal(s, s_ref)
    # the two inputs really differ in coverage
    assert 0 < int((s_ref > 0).sum()) < W * Hh


def test_noalloc_mask_rejects_frames_beyond_capacity():
    p = hi.Params(tile=1)
    W, Hh = 300, 300  # 90000 one-pixel tiles > 65536
    g = H.GBuffer(W, Hh)
    e = torch.empty((Hh, W), dtype=torch.uint8, device="cuda")
    with pytest.raises(H.HdofError) as ei:
        H.hdof_mask_noalloc(g, None, p, e, e.clone())
    assert ei.value.code == -1 and "capacity" in str(ei.value)


def test_noalloc_mask_at_exact_capacity():
    """A frame of exactly HDOF_MASK_NOALLOC_MAX_TILES tiles (256 x 256 at tile
    1) is accepted and equals hdof_mask bit for bit; one more column of tiles
    (257 x 256) is rejected."""
    p = hi.Params(tile=1, dilate=2, spp_max=8)
    W, Hh = 256, 256
    gb = hi.random_gbuffer(W, Hh, seed=31)
    g = _gbuf(gb)
    e_ref = torch.empty((Hh, W), dtype=torch.uint8, device="cuda")
    s_ref = torch.empty_like(e_ref)
    ws = torch.empty(H.hdof_workspace_bytes(W, Hh, p), dtype=torch.uint8, device="cuda")
    H.hdof_mask(g, None, p, e_ref, s_ref, ws)
    e = torch.full_like(e_ref, 7)
    s = torch.full_like(e_ref, 7)
    H.hdof_mask_noalloc(g, None, p, e, s)
    H.hdof_sync()
    assert torch.equal(e, e_ref) and torch.equal(s, s_ref)
    assert 0 < int((s_ref > 0).sum()) < W * Hh
    g2 = H.GBuffer(257, 256)
    e2 = torch.empty((256, 257), dtype=torch.uint8, device="cuda")
    with pytest.raises(H.HdofError) as ei:
        H.hdof_mask_noalloc(g2, None, p, e2, e2.clone())
    assert ei.value.code == -1 and "capacity" in str(ei.value)
