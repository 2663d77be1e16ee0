"""Launch-shape autotuner of the batched multi-view frame.

The batched frame has free choices that change its speed but not its
results (hdof_tuning): the persistent trace's block size (64, 128 or 256
threads) and form (warp packets, refill 0: a warp traverses for 32 coherent
rays at once; ray level with a refill threshold: a warp fetches new rays for
its idle lanes once fewer than that many lanes still trace, 4 or 8; or each
view in its default form, refill -1: packets for the views with a small CoC
scale, ray level for the others, in two launches), the
trace's queue chunk (how many packets, or rays in units of 32, a warp claims
per atomic) and the spatial reconstruction's stencil tile (8x8 or 16x16
pixels per block).  Every candidate renders bit-identical images, so the
tuner only times them: it builds one batch handle per candidate over the
caller's own buffers, times whole batched frames with CUDA events on the
current stream (warm-up first, median of ``reps``), and keeps the fastest.
The search is staged: block and form first, then the chunk at the best of
those, then the tile.  Results are cached in a JSON file keyed by the GPU and
the workload's shape (view sizes, scene sizes, sample budgets), so a workload
is timed once per machine.
"""
from __future__ import annotations

import hashlib
import json
import os

import torch

from . import hdof as H

CANDIDATES = tuple((b, c) for b in (64, 128, 256) for c in (-1, 0, 4, 8))  # (trace_block, trace_refill)
CHUNKS = (0, 2, 4)      # trace_chunk
TILES = (8, 16)         # spatial_tile


def cache_path() -> str:
    return os.environ.get("HDOF_TUNE_CACHE", os.path.join(os.path.expanduser("~"), ".cache", "hdof_tuning.json"))


def workload_shape(batch: "H.Batch"):
    """Every view's (width, height, triangles, spp_max, r_max)."""
    return [(r.W, r.H, int(r.bvh.stats().n_tris), int(p.spp_max), float(p.r_max))
            for r, p in zip(batch.views, batch.params)]


def signature(shape, device_name: str) -> str:
    """Cache key of a workload shape on a GPU model."""
    return hashlib.sha1(json.dumps([device_name] + [list(v) for v in shape]).encode()).hexdigest()[:16]


def _load() -> dict:
    try:
        with open(cache_path()) as f:
            return json.load(f)
    except (OSError, ValueError):
        return {}


def _store(d: dict):
    path = cache_path()
    os.makedirs(os.path.dirname(path), exist_ok=True)
    tmp = path + f".{os.getpid()}.tmp"
    with open(tmp, "w") as f:
        json.dump(d, f, indent=1, sort_keys=True)
    os.replace(tmp, path)


def time_shape(batch: "H.Batch", frame_args, shape, reps: int = 5, warmup: int = 2) -> float:
    """Median milliseconds of one batched frame with the given tuning
    shape (trace_block, trace_refill, trace_chunk, spatial_tile)."""
    recs = batch.records(*frame_args)
    h = H.hdof_batch_create(recs, H.tuning(*shape))
    try:
        for _ in range(warmup):
            H.hdof_batch_render(h)
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(reps)]
        torch.cuda.synchronize()
        for a, b in ev:
            a.record()
            H.hdof_batch_render(h)
            b.record()
        H.hdof_sync()
        ts = sorted(a.elapsed_time(b) for a, b in ev)
        return ts[len(ts) // 2]
    finally:
        H.hdof_batch_destroy(h)


def tune(batch: "H.Batch", frame_args, candidates=CANDIDATES, chunks=CHUNKS, tiles=TILES, reps: int = 5,
         use_cache: bool = True):
    """Pick the fastest hdof_tuning for the batch's workload.

    ``frame_args`` = (cams, prevs, lenses, params) of a representative frame.
    Returns (hdof_tuning, {shape: ms}); the timings are empty on a cache hit.
    """
    key = signature(workload_shape(batch), torch.cuda.get_device_name())
    cache = _load() if use_cache else {}
    if key in cache and len(cache[key]["best"]) == 4:
        return H.tuning(*cache[key]["best"]), {}
    times = {}
    for b, c in candidates:
        times[(b, c, 0, 8)] = time_shape(batch, frame_args, (b, c, 0, 8), reps)
    b, c, _, _ = min(times, key=times.get)
    for k in chunks:
        if (b, c, k, 8) not in times:
            times[(b, c, k, 8)] = time_shape(batch, frame_args, (b, c, k, 8), reps)
    k = min((t for t in times if t[:2] == (b, c) and t[3] == 8), key=times.get)[2]
    for tile in tiles:
        if (b, c, k, tile) not in times:
            times[(b, c, k, tile)] = time_shape(batch, frame_args, (b, c, k, tile), reps)
    best = min(times, key=times.get)
    if use_cache:
        cache = _load()
        cache[key] = {"best": list(best), "ms": {"x".join(map(str, t)): ms for t, ms in times.items()}}
        _store(cache)
    return H.tuning(*best), times
