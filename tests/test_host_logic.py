"""Host-side logic that needs no GPU: the batch autotuner's choice and cache,
the benchmark's multi-rank timing reduction (world size 2 over gloo) and its
model of the post-filter gather's executed work."""
import math
import os
import socket
import sys

import numpy as np
import pytest

torch = pytest.importorskip("torch")

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_autotune_picks_fastest_and_caches(tmp_path, monkeypatch):
    from paper_2210_04981_gb300 import autotune
    monkeypatch.setenv("HDOF_TUNE_CACHE", str(tmp_path / "tune.json"))
    monkeypatch.setattr(torch.cuda, "get_device_name", lambda *a: "test-gpu")
    shape = [(256, 256, 51980, 16, 32.0), (1920, 1080, 502540, 16, 32.0)]
    monkeypatch.setattr(autotune, "workload_shape", lambda b: shape)
    calls = []

    def fake_time(batch, frame_args, shape, reps=5, warmup=2):
        block, refill, chunk, tile = shape
        calls.append(tuple(shape))
        return 1.0 + abs(block - 128) / 64.0 + abs(refill - 4) / 8.0 + abs(chunk - 2) / 16.0 + (tile == 8) / 32.0

    monkeypatch.setattr(autotune, "time_shape", fake_time)
    t, times = autotune.tune(object(), None)
    assert (t.trace_block, t.trace_refill, t.trace_chunk, t.spatial_tile) == (128, 4, 2, 16)
    # staged: every (block, form) at chunk 0 and tile 8, then the chunks, then the tiles
    n = len(autotune.CANDIDATES) + (len(autotune.CHUNKS) - 1) + (len(autotune.TILES) - 1)
    assert len(calls) == len(set(calls)) == len(times) == n
    assert {c[:2] for c in calls} >= set(autotune.CANDIDATES)
    # second call: a cache hit, nothing timed
    t2, times2 = autotune.tune(object(), None)
    assert (t2.trace_block, t2.trace_refill, t2.trace_chunk, t2.spatial_tile) == (128, 4, 2, 16) and times2 == {}
    assert len(calls) == n
    # the key separates GPUs and workloads
    assert autotune.signature(shape, "a") != autotune.signature(shape, "b")
    assert autotune.signature(shape, "a") != autotune.signature(shape[:1], "a")
    assert autotune.signature(shape, "a") == autotune.signature([tuple(v) for v in shape], "a")


def test_autotune_takes_per_view_forms_when_fastest(tmp_path, monkeypatch):
    """Each view in its default trace form (trace_refill -1: packets for the
    narrow-lens views, ray level for the others) is a candidate of the first
    stage at every block size and wins when it times fastest."""
    from paper_2210_04981_gb300 import autotune
    monkeypatch.setenv("HDOF_TUNE_CACHE", str(tmp_path / "tune.json"))
    monkeypatch.setattr(torch.cuda, "get_device_name", lambda *a: "test-gpu")
    monkeypatch.setattr(autotune, "workload_shape", lambda b: [(640, 480, 100000, 16, 32.0)])
    assert {(b, -1) for b in (64, 128, 256)} <= set(autotune.CANDIDATES)

    def fake_time(batch, frame_args, shape, reps=5, warmup=2):
        block, refill, chunk, tile = shape
        return (0.5 if refill == -1 else 1.0) + (block != 256) / 8.0 + chunk / 64.0 + (tile == 16) / 32.0

    monkeypatch.setattr(autotune, "time_shape", fake_time)
    t, _ = autotune.tune(object(), None)
    assert (t.trace_block, t.trace_refill, t.trace_chunk, t.spatial_tile) == (256, -1, 0, 8)



def _rank(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    sys.path.insert(0, ROOT)
    import torch.distributed as dist
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    env = bench.dist_env()
    value = bench.max_over_ranks(10.0 + 5.0 * rank, "cpu")
    dist.barrier()
    dist.destroy_process_group()
    out.put((rank, env, value))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def test_max_over_ranks_gloo_world_2():
    """Two CPU ranks: each sees its own rank in the environment and both get
    the slowest rank's time."""
    ctx = torch.multiprocessing.get_context("spawn")
    out = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, out)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(out.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert [r[1] for r in res] == [(2, 0, 0), (2, 1, 1)]
    assert [r[2] for r in res] == [15.0, 15.0]


def test_max_over_ranks_single_process():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(3.5, "cpu") == 3.5


def test_gather_work_model():
    """The executed-work model of the post-filter gather (the bench's roofline
    for it): a uniform near field engages the interior prefix sums and taps far
    fewer pixel-taps than contribute; an all-far frame gathers nothing in the
    near layer; a near field whose radii jump from pixel to pixel (interior
    below half the reach) falls back to tapping every column, with no lookups."""
    import bench
    import hdof_inputs as hi

    lens = hi.Lens(3.0, 0.2, 0.05).f32()
    t = math.tan(math.radians(30.0))
    W, Hh = 96, 64
    z_uniform = np.full((Hh, W), 0.8)
    taps, pre = bench.gather_work(z_uniform, lens, Hh, t, 32.0)
    contributing = bench.contributing_taps(z_uniform, lens, Hh, t, 32.0)
    assert pre > 0 and 0 < 4 * taps < contributing / 2
    z_far = np.full((Hh, W), 20.0)
    assert bench.gather_work(z_far, lens, Hh, t, 32.0) == (0, 0)
    z_mixed = np.where((np.arange(W)[None, :] + np.arange(Hh)[:, None]) % 2 == 0, 0.8, 2.9)
    taps_m, pre_m = bench.gather_work(z_mixed, lens, Hh, t, 32.0)
    assert pre_m == 0 and 4 * taps_m >= bench.contributing_taps(z_mixed, lens, Hh, t, 32.0) * 0.5
