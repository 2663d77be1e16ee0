#!/usr/bin/env python
"""Benchmark: one hybrid depth-of-field frame per step on the procedural room
at 1920x1080 (the 1080p room workload: ~164.6k triangles, focus 3.0, f/1.4
equivalent aperture, 1-8 rays per masked pixel, EMA 0.2, camera +0.01/frame
with +-0.5 px jitter), through the C ABI on one GB300.

Prints one JSON line.  ``value`` is ms/frame (lower is better) of the whole
hot path: G-buffer, adaptive mask, compaction + thin-lens trace,
post-filter, temporal + spatial reconstruction and composite.  The BVH is
built once (static scene) and reported separately.  Each step renders the
next consecutive frame with its history; L2 is flushed (256 MiB write)
between steps, outside the timed events.

``--impl reference`` times the FP64 CPU oracle on the host cores instead, on
a bounded sample of the same frame (see ``cpu_sample``).
"""
from __future__ import annotations

import argparse
import json
import math
import os
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

import hdof_inputs as hi  # noqa: E402

METRIC = "Hybrid DoF ms/frame @1080p & masked thin-lens Mrays/s vs plain form, 1 GB300"
PEAKS_PATH = os.path.join(ROOT, "MEASURED_PEAKS.json")
FALLBACK_HBM = 6800.0
# The ALU-bound kernels are measured in FP32 lane-operations: one FP32
# instruction executed by one lane (a fused multiply-add counts once), against
# the measured FFMA lane-instruction rate of the FMA probe (hdof_probe_fma).
# Traversal: two octant box tests per visited node, 14 FP32 operations each
# (6 plane-distance FMAs, 6 min/max for entry and exit, 1 multiply widening the
# exit, 1 compare; the kernel issues them as 3 packed f32x2 FMAs, 4 min/max
# with three inputs, 1 multiply and 1 compare), and ~40 per watertight
# ray-triangle test, at the visit and test counts the counting build
# (-DHDOF_TRAV_STATS=1) measured on the 1080p room's thin-lens rays (per-ray
# traversal: the intrinsic work; warp packets execute more).
TRACE_VISITS_PER_RAY = 63.9
TRACE_TESTS_PER_RAY = 6.3
TRACE_OPS_PER_RAY = 28 * TRACE_VISITS_PER_RAY + 40 * TRACE_TESTS_PER_RAY
# Post-filter gather, per executed (pixel, tap): squared distance (FMUL +
# FFMA), soft weight (FADD.SAT), the source's layer (3 colour FFMA + 1 weight
# FFMA) and, for far sources, the depth test (~1.5 on average); the square
# root runs on the MUFU pipe and is not counted.  Per interior prefix lookup:
# a float4 difference and accumulation (8 FADD).
PF_OPS_PER_TAP = 8.5
PF_OPS_PER_LOOKUP = 8
# DRAM traffic per launch (dram__bytes_read.sum + dram__bytes_write.sum, one ncu
# launch-list capture of the 1080p room frame, caches flushed before each launch)
# of the current kernels; None where the kernel changed since the capture
MEASURED_TRAFFIC = {
    ("room", "f32", "trace_packets"): 18719232,
    ("room", "f32", "pf_gather"): 120400384,
}


def peaks():
    try:
        with open(PEAKS_PATH) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), float(d.get("clocks_under_load", {}).get("sm_mhz_median", 1500.0)), "measured"
    except Exception:
        return FALLBACK_HBM, 1500.0, "fallback"


# ------------------------------------------------------------------ clocks --

class ClockSampler:
    """nvidia-smi sampling of SM clock and throttle reasons during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index, period_ms=200):
        self.idx = gpu_index
        self.period = int(period_ms)
        self.proc = None
        self.path = None

    def __enter__(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.idx}", f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", str(self.period)],
                                         stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
            # the timed region starts once the sampler is live (its first line is out)
            t_end = time.perf_counter() + 3.0
            while time.perf_counter() < t_end and self.proc.poll() is None and os.path.getsize(self.path) == 0:
                time.sleep(0.01)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *a):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        out = {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        if not self.path or not os.path.exists(self.path):
            return out
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax.append(float(f[2]))
            except ValueError:
                continue
            for n, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(n)
        os.unlink(self.path)
        if sm:
            out.update(sm_mhz=float(np.median(sm)), sm_max_mhz=float(max(smax)), samples=len(sm))
        out["reasons"] = sorted(reasons)
        return out


# ------------------------------------------------------------- distributed --

def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def max_over_ranks(value, device):
    """Largest value over all ranks (the job's time is its slowest rank's)."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(value)
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


# ----------------------------------------------------------- our kernels ---

def algorithmic_bytes(W, Hh, n_traced, variance_px, nd_b=16, col_b=16):
    """HBM bytes each call must move at minimum, per frame (nd_b, col_b: bytes
    per pixel of the normal/depth and colour planes: 16 in FP32, 8 in FP16/BF16)."""
    px = W * Hh
    return {
        "gbuffer": (nd_b + col_b + 12) * px,                        # write nd, col, mv, tri
        "mask": (nd_b + 1 + 1) * px + (8 + 8 + 1) * variance_px,     # nd -> edge, spp; mv + history where needed
        "trace": 2 * px + (4 + 4 + 1 + 48) * n_traced,               # spp twice; queue w/r; spp; rt
        "postfilter": (nd_b + 16 + 16 + col_b + 16) * px,            # nd -> prep; prep + col -> pp
        "reconstruct": (1 + 1 + 16) * px + (48 + 8 + nd_b + 41 + 41 + 16 + 4 + 16 + 9 + 16) * n_traced,
        "composite": (nd_b + col_b + 1 + 16 + 16) * px + (16 + 16 + 4) * n_traced,
    }


SCENES = {
    # name: (width, height, scene builder, params overrides, workload text)
    "room": (1920, 1080, lambda a: hi.room_scene(seed=0, aspect=a), {},
             "procedural room 1920x1080, 164620 tris, 1-8 spp masked thin-lens, consecutive frames"),
    "room4k": (3840, 2160, lambda a: hi.room4k_scene(seed=0, aspect=a), {"r_max": 64.0},
               "procedural room 3840x2160, 5249036 tris, 1-8 spp masked thin-lens, consecutive frames"),
}


def contributing_taps(z, lens, Hh, t, r_max):
    """Number of (pixel, tap) pairs with non-zero post-filter weight:
    sum over source pixels q of the lattice points within r_q + 1/2
    (ignoring the image border)."""
    c = lens.aperture_radius * Hh * (lens.focus_dist - z) / (z * lens.focus_dist * t)
    r = np.minimum(np.abs(c) * 0.5, r_max)
    R = int(math.ceil(r_max + 0.5))
    o = np.arange(-R, R + 1)
    d = np.sort(np.sqrt(o[:, None] ** 2 + o[None, :] ** 2).ravel())
    return int(np.searchsorted(d, r.ravel() + 0.5, side="left").sum())


def gather_work(z, lens, Hh, t, r_max):
    """Work the near-layer post-filter gather executes on depth plane z, by
    the kernel's own window rules: per 16x16 tile the reach R (largest r +
    1/2 of the tiles that reach it) and the interior radius R_in (smallest
    max(r_min(T) - 1/2, gap(T)) over the tiles that feed the near layer, used
    when >= R/2); per 2x2-pixel thread and source row, the columns it taps
    (interior columns of all four pixels skipped) and its prefix lookups (two
    per pixel row with an interior).  Returns (tap iterations, each of four
    pixel-taps, prefix lookups)."""
    H, W = z.shape
    c = lens.aperture_radius * Hh * (lens.focus_dist - z) / (z * lens.focus_dist * t)
    r = np.minimum(np.abs(c) * 0.5, r_max)
    wn = np.clip((c + math.sqrt(2.0)) / (2.0 * math.sqrt(2.0)), 0.0, 1.0)
    TP = 16
    ntx, nty = (W + TP - 1) // TP, (H + TP - 1) // TP

    def tiles(a, fill, red):
        a = np.pad(a, ((0, nty * TP - H), (0, ntx * TP - W)), constant_values=fill)
        return red(a.reshape(nty, TP, ntx, TP), axis=(1, 3))

    tmax = tiles(np.where(wn > 0, r, -1.0), -1.0, np.max)
    tmin = tiles(np.where(wn > 0, r, np.inf), np.inf, np.min)
    kt = math.ceil((r_max + 0.5) / TP) + 1
    offs = np.arange(-kt, kt + 1)
    gap = np.where(offs == 0, 0.0, (np.abs(offs) - 1) * TP + 1.0)
    th = np.arange(64)
    taps = pre = 0
    for ty in range(nty):
        for tx in range(ntx):
            vy, vx = (ty + offs >= 0) & (ty + offs < nty), (tx + offs >= 0) & (tx + offs < ntx)
            sub = tmax[np.ix_(ty + offs[vy], tx + offs[vx])]
            subm = tmin[np.ix_(ty + offs[vy], tx + offs[vx])]
            g2 = gap[vy][:, None] ** 2 + gap[vx][None, :] ** 2
            reach = (sub >= 0) & (g2 < (sub + 0.5) ** 2)
            if not reach.any():
                continue
            R = float((sub + 0.5)[reach].max())
            lim = np.maximum(np.maximum(subm - 0.5, np.sqrt(g2) - 1e-3), 0.0)[sub >= 0]
            Rin = min(float(lim.min()), R) - 1e-3
            if Rin < 0.5 * R:
                Rin = -1.0
            G = math.floor(R + 1e-3)
            i, j = tx * TP + 2 * (th & 7), ty * TP + 2 * (th >> 3)
            ok = (i < W) & (j < H)
            i, j = i[ok][:, None], j[ok][:, None]
            dy = np.arange(-G, G + 2, dtype=np.float64)[None, :]
            rows = (j + dy >= 0) & (j + dy < H)
            d0, d1 = dy ** 2, (dy - 1) ** 2
            dmin = np.where((dy >= 0) & (dy <= 1), 0.0, np.minimum(d0, d1))
            w = np.floor(np.sqrt(np.maximum(R * R - dmin, 0.0)) + 1e-3).astype(np.int64)
            x0, x1 = np.maximum(i - w, 0), np.minimum(i + 1 + w, W - 1)
            span = x1 - x0 + 1
            if Rin >= 0:
                R2 = Rin * Rin
                w0 = np.where(d0 <= R2, np.floor(np.sqrt(np.maximum(R2 - d0, 0.0))), -1).astype(np.int64)
                w1 = np.where(d1 <= R2, np.floor(np.sqrt(np.maximum(R2 - d1, 0.0))), -1).astype(np.int64)
                wm = np.minimum(w0, w1)
                ls, rs = np.minimum(x1, i - wm), np.maximum(x0, i + wm + 1)
                span = np.where(wm >= 1, np.maximum(ls - x0 + 1, 0) + np.maximum(x1 - rs + 1, 0), span)
                pre += int((((w0 >= 0).astype(np.int64) + (w1 >= 0)) * 2 * rows).sum())
            taps += int((span * rows).sum())
    return taps, pre


def fp32_peak(H, dev, reps=6, iters=20000):
    """Measured FFMA lane-instruction rate (lane-ops/s) of the FMA probe at
    full occupancy: the best of `reps` - 1 timed launches (the first warms
    up), CUDA events on the launching stream."""
    import torch
    stream = torch.cuda.current_stream()
    sink = torch.zeros(256, dtype=torch.float32, device=dev)
    best = 0.0
    for k in range(reps):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        ops = H.hdof_probe_fma(8, iters, sink)
        e1.record(stream)
        e1.synchronize()
        if k:
            best = max(best, ops / (e0.elapsed_time(e1) * 1e-3))
    return best


STAGES = ["gbuffer", "mask", "trace", "postfilter", "reconstruct", "composite"]


def render_frames(H, bvh, W, Hh, cams, lens, p0, dev, nd_dt, col_dt, warmup, K, flush, profile=False,
                  static=False):
    """Warm-up frames, then K consecutive timed frames (L2 flushed between
    them, outside the events) through the six C-ABI calls, as the Renderer
    runs them: forked from the caller's stream onto the Renderer's
    high-priority critical-path stream, the post-filter on its low-priority
    side stream after the G-buffer, concurrently with the mask, trace and
    reconstruction, the composite after both, joined back at the end.  Returns the renderer, the per-frame stage times [K, 6] (ms,
    each stage between its own events on its stream), the per-kernel times
    of the library's profiler (mean ms per frame), the per-frame (traced
    pixels, rays), the wall time and the per-frame times [K] (ms, from the
    frame's first call to the end of its composite)."""
    import torch
    r = H.Renderer(bvh, W, Hh, p0, device=dev, nd_dtype=nd_dt, col_dtype=col_dt)
    stream = torch.cuda.current_stream()
    crit, side = r.crit, r.side
    start, done = torch.cuda.Event(), torch.cuda.Event()
    g_done, pf_done = torch.cuda.Event(), torch.cuda.Event()

    def params_of(k):
        return p0.replace(frame=k % 65536, camera_moved=int(k > 0 and not static))

    # event slots: frame start, after G-buffer, mask, trace, reconstruct; post-filter start and end;
    # composite start and end
    SLOTS = ("f0", "g1", "m1", "t1", "r1", "p0", "p1", "c0", "c1")

    def frame(k, ev=None, serial=False):
        cam, prev, p = cams[k], cams[max(k - 1, 0)], params_of(k)
        hin, hout = r.hist[r.cur], r.hist[1 - r.cur]
        pf_stream = crit if serial else side

        def mark(name, s):
            if ev is not None:
                ev[name].record(s)

        start.record(stream)
        crit.wait_event(start)
        mark("f0", crit)
        H.hdof_gbuffer(bvh, cam, prev, p, r.g, stream=crit, hint=r.g.tri)
        mark("g1", crit)
        g_done.record(crit)
        pf_stream.wait_event(g_done)
        mark("p0", pf_stream)
        H.hdof_postfilter(r.g, cam, lens, p, r.pp, r.ws, stream=pf_stream)
        mark("p1", pf_stream)
        pf_done.record(pf_stream)
        H.hdof_mask(r.g, hin, p, r.edge, r.spp, r.ws, stream=crit)
        mark("m1", crit)
        H.hdof_trace(bvh, cam, lens, p, r.spp, r.rt, r.stats, r.ws, stream=crit, hint=r.g.tri)
        mark("t1", crit)
        H.hdof_reconstruct(r.rt, r.g, r.spp, cam, prev, lens, p, hin, hout, r.crt, r.hacc, r.crec, stream=crit)
        mark("r1", crit)
        crit.wait_event(pf_done)
        mark("c0", crit)
        H.hdof_composite(r.g, r.spp, r.pp, r.crt, r.crec, r.hacc, cam, lens, p, r.out, stream=crit)
        mark("c1", crit)
        done.record(crit)
        stream.wait_event(done)
        r.cur = 1 - r.cur

    r.frame_fn = frame
    for k in range(warmup):
        frame(k)
    H.hdof_sync()
    evs = [{n: torch.cuda.Event(enable_timing=True) for n in SLOTS} for _ in range(K)]
    stats_all = torch.zeros((K, 2), dtype=torch.int32, device=dev)
    torch.cuda.synchronize()
    wall0 = time.perf_counter()
    for s in range(K):
        flush.zero_()  # evict L2 between steps (outside the step's events)
        frame(warmup + s, evs[s])
        stats_all[s].copy_(r.stats)  # ray counts of this frame (after its events)
    torch.cuda.synchronize()
    wall = time.perf_counter() - wall0
    kern = {}
    if profile:
        # the same K frames again (history reset, warm-up repeated) with the
        # library's per-kernel events (they add ~0.05 ms per frame, so the
        # stage times above are taken without), the post-filter serialised
        # so that each kernel's events time it alone
        r.reset_history()
        for k in range(warmup):
            frame(k)
        H.hdof_sync()
        H.hdof_profile_read()  # drop anything recorded before
        H.hdof_profile(True)
        for s in range(K):
            flush.zero_()
            frame(warmup + s, serial=True)
        torch.cuda.synchronize()
        H.hdof_profile(False)
        kern = {n: t / K for n, (_, t) in H.hdof_profile_read().items()}
    H.hdof_sync()
    spans = {"gbuffer": ("f0", "g1"), "mask": ("g1", "m1"), "trace": ("m1", "t1"), "postfilter": ("p0", "p1"),
             "reconstruct": ("t1", "r1"), "composite": ("c0", "c1")}
    stage_ms = np.array([[evs[s][spans[n][0]].elapsed_time(evs[s][spans[n][1]]) for n in STAGES] for s in range(K)])
    frame_ms = np.array([evs[s]["f0"].elapsed_time(evs[s]["c1"]) for s in range(K)])
    st = stats_all.cpu().numpy().astype(np.int64) & 0xFFFFFFFF
    return r, stage_ms, kern, st, wall, frame_ms


def e2e_frames(H, r, Hh, W, warmup, K, flush):
    """The same frames end to end, run as a renderer would: host camera, lens
    and params records into the C calls every frame, and every frame's
    RGBA32F image read back to pinned host memory on a copy stream while the
    next frame renders (two device output buffers and two host buffers; a
    buffer is reused only after its previous copy finished).  One timed
    region over the K frames, from before the first frame's first call to
    the last image on the host; no L2 flush inside it (each frame streams
    several hundred MB of planes, far more than the 129 MB L2).  Returns ms
    per frame and the bytes moved per frame."""
    import ctypes

    import torch
    stream = torch.cuda.current_stream()
    copy_stream = torch.cuda.Stream()
    outs = [r.out, torch.empty_like(r.out)]
    hosts = [torch.empty((Hh, W, 4), dtype=torch.float32, pin_memory=True) for _ in range(2)]
    rendered = [torch.cuda.Event() for _ in range(2)]
    copied = [torch.cuda.Event() for _ in range(2)]
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    r.reset_history()
    for k in range(warmup):
        r.frame_fn(k)
    torch.cuda.synchronize()
    flush.zero_()
    torch.cuda.synchronize()
    e0.record(stream)
    for s in range(K):
        b = s & 1
        if s >= 2:
            stream.wait_event(copied[b])  # frame s - 2's image has left this buffer
        r.out = outs[b]
        r.frame_fn(warmup + s)
        rendered[b].record(stream)
        copy_stream.wait_event(rendered[b])
        with torch.cuda.stream(copy_stream):
            hosts[b].copy_(outs[b], non_blocking=True)
        copied[b].record(copy_stream)
    stream.wait_event(copied[(K - 1) & 1])
    e1.record(stream)
    e1.synchronize()
    r.out = outs[0]
    e_ms = e0.elapsed_time(e1)
    rec_bytes = ctypes.sizeof(H.hdof_camera) * 2 + ctypes.sizeof(H.hdof_lens) + ctypes.sizeof(H.hdof_params)
    return e_ms / max(K, 1), int(rec_bytes), int(hosts[0].numel() * 4)


def kernel_roofline(name, kms, rays, z, lens, Hh, t, r_max, lane_peak, clock_mhz, hbm, traffic_key):
    """Roofline of one kernel from its live mean time `kms` (ms per frame)."""
    peak_t = lane_peak / 1e12
    src = (f"measured: FFMA lane-instruction rate of hdof_probe_fma (8 chains x 256 threads x 8 blocks per SM) "
           f"at {clock_mhz or 'unsampled'} MHz")
    if name in ("trace_packets", "trace_rays"):
        ops = TRACE_OPS_PER_RAY * rays
        ach = ops / (kms * 1e-3) / 1e12
        return {"bound": "alu", "achieved": round(ach, 2), "peak": round(peak_t, 2), "unit": "Tlane-op/s",
                "frac": round(ach / peak_t, 3), "kernel": f"k_{name}", "kernel_ms": round(kms, 4),
                "ops_per_launch": int(ops), "ops_per_ray": TRACE_OPS_PER_RAY,
                "op_unit": "FP32 lane-op (one FP32 instruction in one lane; an FMA counts once)",
                "traffic": MEASURED_TRAFFIC.get(traffic_key), "peak_source": src}
    if name == "pf_gather":
        tap_it, lookups = gather_work(z, lens, Hh, t, r_max)
        ops = 4 * tap_it * PF_OPS_PER_TAP + PF_OPS_PER_LOOKUP * lookups
        ach = ops / (kms * 1e-3) / 1e12
        return {"bound": "alu", "achieved": round(ach, 2), "peak": round(peak_t, 2), "unit": "Tlane-op/s",
                "frac": round(ach / peak_t, 3), "kernel": "k_pf_gather", "kernel_ms": round(kms, 4),
                "ops_per_launch": int(ops), "executed_pixel_taps": 4 * tap_it, "prefix_lookups": lookups,
                "op_unit": "FP32 lane-op (one FP32 instruction in one lane; an FMA counts once)",
                "traffic": MEASURED_TRAFFIC.get(traffic_key), "peak_source": src}
    return None


def quality(H, bvh, r, cam, lens, p, passes, block=8):
    """The paper's Fig. 1 comparison on the renderer's last frame: a full
    ray-traced frame (every pixel, passes x spp_max lens samples, timed), the
    post-process-only frame (the composite with no traced pixels), and the
    error of the hybrid and post-process frames against the ray-traced one,
    over all pixels and over the traced pixels (the blurry silhouettes); also
    on block x block means of the images, which separate a systematic error
    from the Monte-Carlo noise of the few-sample hybrid frame."""
    import torch
    import torch.nn.functional as F
    stream = torch.cuda.current_stream()
    zero = torch.zeros_like(r.spp)
    pp_only = torch.empty_like(r.out)
    H.hdof_composite(r.g, zero, r.pp, r.crt, r.crec, r.hacc, cam, lens, p, pp_only)
    rt = torch.empty_like(r.out)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    H.hdof_reference_rt(bvh, cam, lens, p, passes, rt, r.ws, hint=r.g.tri)
    e1.record(stream)
    e1.synchronize()
    rt_ms = e0.elapsed_time(e1)
    stats = torch.empty(H.ERR_SCRATCH, dtype=torch.float64, device=r.out.device)
    traced = (r.spp > 0).to(torch.uint8)

    def pool(img):  # block means (analysis only), as a [H/b, W/b, 4] image
        return F.avg_pool2d(img.permute(2, 0, 1)[None], block)[0].permute(1, 2, 0).contiguous()

    tb = (F.avg_pool2d(traced[None, None].float(), block)[0, 0] > 0.5).to(torch.uint8).contiguous()
    res = {"reference": f"full ray trace, {passes * p.spp_max} lens samples per pixel",
           "reference_ms": round(rt_ms, 3), "traced_pixels": int(traced.sum())}
    for name, a, b in (("hybrid_vs_rt", r.out, rt), ("pp_vs_rt", pp_only, rt), ("hybrid_vs_pp", r.out, pp_only)):
        H.hdof_error_map(a, b, stats, region=traced)
        sm = H.error_summary(stats)
        H.hdof_error_map(pool(a), pool(b), stats, region=tb)
        smb = H.error_summary(stats)
        res[name] = {part: {k: (round(v, 6) if isinstance(v, float) else v) for k, v in sm[part].items()}
                     for part in ("all", "region")}
        res[name][f"block{block}_region_mae"] = round(smb["region"]["mae"], 6)
    return res


def quality_variants(H, bvh, W, Hh, lens, p0, dev, flush, frames, passes):
    """Hybrid against full ray tracing after `frames` frames, in three
    settings: the workload's (moving camera, fixed EMA weight), the moving
    camera with per-pixel blend factors (alpha_k = 0.5), and a static camera
    (fixed EMA); block-mean errors on the traced pixels, hybrid and
    post-process."""
    import torch
    out = {}
    for name, alpha_k, moving in (("moving_fixed_ema", 0.0, True), ("moving_per_pixel_alpha", 0.5, True),
                                  ("static_fixed_ema", 0.0, False)):
        p = p0.replace(alpha_k=alpha_k)
        cams = [hi.room_camera(k if moving else 0, W, Hh) for k in range(frames + 1)]
        r = render_frames(H, bvh, W, Hh, cams, lens, p, dev, torch.float32, torch.float32, 0, frames,
                          flush, static=not moving)[0]
        last = frames - 1
        q = quality(H, bvh, r, cams[last], lens, p.replace(frame=last, camera_moved=int(moving)), passes)
        out[name] = {"hybrid_block8_mae": q["hybrid_vs_rt"]["block8_region_mae"],
                     "pp_block8_mae": q["pp_vs_rt"]["block8_region_mae"],
                     "hybrid_mae": q["hybrid_vs_rt"]["region"]["mae"], "pp_mae": q["pp_vs_rt"]["region"]["mae"]}
        del r
    return out


def quality_glossy(H, W, Hh, lens, p0, dev, frames, passes, ks=2.0, pref=0.5):
    """The Composite section's specular-bokeh preference on the workload's
    room with glossy spheres (Blinn-Phong k_s = ks), static camera, after
    `frames` frames: the last frame composited without and with the
    preference (spec_pref = pref) and with the post-process alone, against
    full ray tracing, over the traced pixels and over the near highlights
    (traced pixels where clamp(pref S_pp, 0, 1) > 0.05)."""
    import torch
    scene = hi.room_scene(seed=0, aspect=W / Hh, specular=ks)
    bvh = H.hdof_build_bvh(*(torch.from_numpy(a).to(dev) for a in (scene.verts, scene.idx, scene.mat, scene.uv)))
    cam = hi.room_camera(0, W, Hh)
    p = p0.replace(spec_pref=pref)
    r = H.Renderer(bvh, W, Hh, p, device=dev)
    for k in range(frames):
        r.frame(cam, cam, lens, p.replace(frame=k, camera_moved=0))
    last = p.replace(frame=frames - 1, camera_moved=0)
    rt = torch.empty_like(r.out)
    H.hdof_reference_rt(bvh, cam, lens, last, passes, rt, r.ws, hint=r.g.tri)
    traced = (r.spp > 0).to(torch.uint8).contiguous()
    hl = ((r.pp_spec[..., 0] * pref > 0.05) & (r.spp > 0)).to(torch.uint8).contiguous()
    imgs = {"with_preference": r.out.clone(), "without_preference": torch.empty_like(r.out),
            "post_process_only": torch.empty_like(r.out)}
    H.hdof_composite(r.g, r.spp, r.pp, r.crt, r.crec, r.hacc, cam, lens, last.replace(spec_pref=0.0),
                     imgs["without_preference"])
    H.hdof_composite(r.g, torch.zeros_like(r.spp), r.pp, r.crt, r.crec, r.hacc, cam, lens, last,
                     imgs["post_process_only"])
    stats = torch.empty(H.ERR_SCRATCH, dtype=torch.float64, device=r.out.device)
    out = {"k_s": ks, "spec_pref": pref, "traced_pixels": int(traced.sum()), "highlight_pixels": int(hl.sum())}
    for name, img in imgs.items():
        H.hdof_error_map(img, rt, stats, region=traced)
        tr = H.error_summary(stats)["region"]
        H.hdof_error_map(img, rt, stats, region=hl)
        h = H.error_summary(stats)["region"]
        out[name] = {"traced_mae": round(tr["mae"], 6), "highlight_mae": round(h["mae"], 6),
                     "highlight_rmse": round(h["rmse"], 6)}
    del r
    bvh.close()
    return out


def run_ours(args):
    import torch

    import paper_2210_04981_gb300.hdof as H

    ws, rank, local = dist_env()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=dev)
    W, Hh, make_scene, over, workload = SCENES[args.scene]
    if args.width:
        W, Hh = args.width, args.height
    scene = make_scene(W / Hh)
    lens = hi.room_lens()
    p0 = hi.room_params(**over)
    cams = [hi.room_camera(k, W, Hh) for k in range(args.warmup + 2 * args.steps + 1)]
    mixed = args.precision == "mixed"
    nd_dt, col_dt = (torch.float16, torch.bfloat16) if mixed else (torch.float32, torch.float32)
    t0 = time.perf_counter()
    verts, idx = torch.from_numpy(scene.verts).to(dev), torch.from_numpy(scene.idx).to(dev)
    mat, uv = torch.from_numpy(scene.mat).to(dev), torch.from_numpy(scene.uv).to(dev)
    torch.cuda.synchronize()
    t1 = time.perf_counter()
    bvh = H.hdof_build_bvh(verts, idx, mat, uv)
    torch.cuda.synchronize()
    bvh_ms = (time.perf_counter() - t1) * 1e3
    upload_ms = (t1 - t0) * 1e3
    st = bvh.stats()
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)
    K = args.steps
    if ws > 1:
        torch.distributed.barrier()
    sampler = ClockSampler(local, period_ms=20)
    with sampler:
        r, stage_ms, kern, st_all, wall, frame_ms = render_frames(H, bvh, W, Hh, cams, lens, p0, dev, nd_dt,
                                                                  col_dt, args.warmup, K, flush, profile=True)
    if ws > 1:
        torch.distributed.barrier()
    step_ms = frame_ms
    total_ms = max_over_ranks(float(step_ms.sum()), dev)
    clocks = sampler.summary()
    traced, rays = st_all[:, 0], st_all[:, 1]
    spp_h = r.spp.cpu().numpy()
    var_px = int(((spp_h > 0) & (spp_h < p0.spp_max)).sum())
    mean_stage = stage_ms.mean(0)
    trace_ms = float(mean_stage[STAGES.index("trace")])
    # the trace call's own rate: its kernels (compaction, trace, resolve) as the serialised profiled pass
    # times them over the same frames; in the timed frames the concurrent post-filter shares the SMs
    # with them, which stretches the stage's span (trace_ms)
    trace_alone = sum(kern.get(n, 0.0) for n in ("trace_compact", "trace_packets", "trace_rays", "trace_resolve"))
    mrays = float(rays.mean()) / ((trace_alone or trace_ms) * 1e-3) / 1e6
    mrays_concurrent = float(rays.mean()) / (trace_ms * 1e-3) / 1e6
    hbm, sm_med, peak_src = peaks()
    ab = algorithmic_bytes(W, Hh, float(traced.mean()), float(var_px), 8 if mixed else 16, 8 if mixed else 16)
    per_stage = {}
    for i, n in enumerate(STAGES):
        gbs = ab[n] / (mean_stage[i] * 1e-3) / 1e9
        per_stage[n] = {"ms": round(float(mean_stage[i]), 4), "alg_bytes": int(ab[n]),
                        "alg_GBps": round(gbs, 1), "hbm_frac": round(gbs / hbm, 3)}
    z = r.g.nd[..., 3].float().cpu().numpy().astype(np.float64)
    t = cams[0].tan_half_fovy
    per_stage["postfilter"]["contributing_taps"] = contributing_taps(z, lens, Hh, t, p0.r_max)

    # measured FP32 peak (FMA probe), with its own clock record
    psamp = ClockSampler(local, period_ms=20)
    with psamp:
        lane_peak = fp32_peak(H, dev)
    pclk = psamp.summary()
    storage = "mixed" if mixed else "f32"
    # roofline of the dominant kernel by live time (and of the runner-up ALU kernel)
    kernels = {k: round(v, 4) for k, v in sorted(kern.items(), key=lambda kv: -kv[1])}
    roofs = []
    for name, kms in kernels.items():
        rf = kernel_roofline(name, kms, float(rays.mean()), z, lens, Hh, t, p0.r_max, lane_peak,
                             pclk["sm_mhz"], hbm, (args.scene, storage, name))
        if rf is not None:
            rf["share_of_frame"] = round(kms / float(step_ms.mean()), 3)
            roofs.append(rf)
    dom = next(iter(kernels)) if kernels else None
    roof = roofs[0] if roofs and dom and roofs[0]["kernel"].endswith(dom) else None
    if roof is None:  # an HBM-bound kernel dominates: its stage's algorithmic bytes
        stg = next((n for n in STAGES if dom and dom.startswith(n[:4])), "composite")
        gbs = ab[stg] / (mean_stage[STAGES.index(stg)] * 1e-3) / 1e9
        roof = {"bound": "hbm", "achieved": round(gbs, 1), "peak": hbm, "unit": "GB/s", "frac": round(gbs / hbm, 3),
                "traffic": MEASURED_TRAFFIC.get((args.scene, storage, dom)), "kernel": dom, "peak_source": peak_src}
    last = args.warmup + K - 1  # the last frame the renderer drew
    qual = quality(H, bvh, r, cams[last], lens, p0.replace(frame=last % 65536, camera_moved=1), args.rt_passes)
    if not args.no_compare and ws == 1:
        qual["variants_after_8_frames"] = quality_variants(H, bvh, W, Hh, lens, p0, dev, flush, 8, args.rt_passes)
        qual["glossy_static_after_8_frames"] = quality_glossy(H, W, Hh, lens, p0, dev, 8, args.rt_passes)
    e2e = None
    if not args.no_e2e:
        e_ms, h2d, d2h = e2e_frames(H, r, Hh, W, args.warmup, K, flush)
        e2e = {"value": round(e_ms, 4), "unit": "ms/frame", "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
               "note": "h2d = camera/lens/params records passed by value to the C calls; d2h = RGBA32F image of "
                       "every frame, read back on a copy stream while the next frame renders (double-buffered); "
                       "one timed region over the frames, no L2 flush (the planes exceed L2)"}
    del r
    value = total_ms / (K * ws)
    out = {
        "metric": METRIC, "value": round(value, 4), "unit": "ms/frame", "n_gpus": ws, "steps": K,
        "warmup": args.warmup, "ms_per_step": round(total_ms / K, 4), "higher_is_better": False,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": workload, "width": W, "height": Hh, "triangles": int(st.n_tris),
                   "storage": "f16 normal/depth, bf16 colour and post-filter records, f32 elsewhere" if mixed else "f32",
                   "spp_max": p0.spp_max, "r_max": p0.r_max,
                   "parallelism": f"replicas x{ws}" if ws > 1 else "single", "l2": "flushed between steps (256 MiB write)"},
        "mrays_per_s": round(mrays, 1), "mrays_per_s_concurrent": round(mrays_concurrent, 1),
        "rays_per_frame": int(rays.mean()),
        "traced_px_per_frame": int(traced.mean()), "trace_ms": round(trace_ms, 4),
        "trace_call_alone_ms": round(trace_alone, 4),
        "stages": per_stage, "kernels_ms": kernels, "bvh_build_ms": round(bvh_ms, 3), "bvh_depth": int(st.depth),
        "scene_upload_ms": round(upload_ms, 3), "wall_s_timed": round(wall, 3),
        "roofline": roof, "roofline_alu_kernels": roofs,
        "fp32_peak": {"lane_ops_per_s": round(lane_peak / 1e12, 3), "unit": "T", "clocks": pclk,
                      "sms": torch.cuda.get_device_properties(dev).multi_processor_count},
        "quality": qual, "e2e": e2e, "gpu_launches": 14 * K, "clocks": clocks,
    }
    # "vs plain form": the same frames with mixed-precision storage, and the
    # 64-view batched frame against its single-view calls
    if not mixed and args.scene == "room" and not args.no_compare and ws == 1:
        rm, sm_m, _, stm, _, fm_m = render_frames(H, bvh, W, Hh, cams, lens, p0, dev, torch.float16, torch.bfloat16,
                                                  args.warmup, K, flush)
        mixed_ms = float(fm_m.mean())
        out["mixed"] = {"value": round(mixed_ms, 4), "unit": "ms/frame",
                        "storage": "f16 normal/depth, bf16 colour and post-filter records, f32 elsewhere",
                        "speedup_vs_fp32": round(value / mixed_ms, 3),
                        "stages_ms": {n: round(float(v), 4) for n, v in zip(STAGES, sm_m.mean(0))},
                        "mrays_per_s": round(float(stm[:, 1].mean()) / (float(sm_m[:, 2].mean()) * 1e-3) / 1e6, 1)}
        del rm
        torch.cuda.empty_cache()
        bres = batch_measure(H, dev, min(K, 5), args.warmup, args.views, flush, e2e=False, stage_times=False)
        out["batch"] = {k: bres[k] for k in ("value", "unit", "plain_ms", "speedup_vs_plain", "views", "pixels",
                                             "rays_per_frame", "mrays_per_s_frame", "tuning", "steps")}
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        out["cpu_baseline"] = cpu_baseline(args, budget_s=args.cpu_budget)
    if rank == 0:
        print(json.dumps(out), flush=True)
    if ws > 1:
        torch.distributed.destroy_process_group()


# ------------------------------------------------------- batched views ---

def _batch_frame_args(views, k):
    cams = [v.camera(k) for v in views]
    prevs = [v.camera(k - 1) if k else v.camera(0) for v in views]
    ps = [v.params.replace(frame=k % 65536, camera_moved=int(k > 0)) for v in views]
    return cams, prevs, [v.lens for v in views], ps


def batch_measure(H, dev, K, Wm, n_views, flush, e2e=True, stage_times=True):
    """64 views over 4 rooms (50k-500k triangles, 256^2 to 1920x1080): each
    step is one batched frame of all views (records update + graph replay of
    the batched launches), against the plain form (the single-view calls,
    view after view) on the same views.  Returns a dict of results."""
    import torch

    from paper_2210_04981_gb300 import autotune

    scenes = hi.batch_scenes()
    views = hi.batch_views(n_views)
    t1 = time.perf_counter()
    bvhs = [H.hdof_build_bvh(*(torch.from_numpy(a).to(dev) for a in (sc.verts, sc.idx, sc.mat, sc.uv)))
            for sc in scenes]
    torch.cuda.synchronize()
    bvh_ms = (time.perf_counter() - t1) * 1e3
    sizes = [(v.width, v.height) for v in views]
    b = H.Batch([bvhs[v.room] for v in views], sizes, [v.params for v in views], device=dev)
    tune, tune_ms = autotune.tune(b, _batch_frame_args(views, 0))
    b.tune = tune
    stream = torch.cuda.current_stream()
    for k in range(Wm):
        b.frame(*_batch_frame_args(views, k))
    H.hdof_sync()
    # graph of the whole batched frame, replayed after each records update
    g = torch.cuda.CUDAGraph()
    side = torch.cuda.Stream()
    side.wait_stream(stream)
    b.update(*_batch_frame_args(views, Wm))
    with torch.cuda.stream(side):
        with torch.cuda.graph(g, stream=side):
            b.render()
    stream.wait_stream(side)
    # the captured frame was not run: render it now so frame Wm is complete
    g.replay()
    b.advance()
    H.hdof_sync()
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(K)]
    stats = torch.zeros((K, len(views), 2), dtype=torch.int32, device=dev)
    torch.cuda.synchronize()
    sampler = ClockSampler(dev.index or 0, period_ms=20)
    with sampler:
        for s in range(K):
            flush.zero_()
            evs[s][0].record(stream)
            b.update(*_batch_frame_args(views, Wm + 1 + s))
            g.replay()
            evs[s][1].record(stream)
            b.advance()
            for i, r in enumerate(b.views):
                stats[s, i].copy_(r.stats)
        torch.cuda.synchronize()
    H.hdof_sync()
    step_ms = np.array([a.elapsed_time(c) for a, c in evs])
    clocks = sampler.summary()
    st = stats.cpu().numpy().astype(np.int64) & 0xFFFFFFFF
    rays = float(st[:, :, 1].sum(1).mean())
    traced = float(st[:, :, 0].sum(1).mean())
    batch_ms = float(step_ms.mean())

    stage_ms = None
    reps = 5
    if stage_times:  # per-stage times of the batched frame (eager, stage by stage)
        n_st = len(H.BATCH_STAGES)
        sev = [torch.cuda.Event(enable_timing=True) for _ in range(n_st + 1)]
        stage_ms = np.zeros(n_st)
        for rep in range(reps):
            b.update(*_batch_frame_args(views, Wm + 1 + K + rep))
            flush.zero_()
            for i in range(n_st):
                sev[i].record(stream)
                H.hdof_batch_render_range(b.handle, i, i)
            sev[n_st].record(stream)
            b.advance()
            torch.cuda.synchronize()
            stage_ms += np.array([sev[i].elapsed_time(sev[i + 1]) for i in range(n_st)])
        stage_ms /= reps

    e2e_res = None
    if e2e:  # host records in, every view's image out to pinned memory
        outs = [torch.empty((v.height, v.width, 4), dtype=torch.float32, pin_memory=True) for v in views]
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e_ms = 0.0
        for s in range(K):
            flush.zero_()
            e0.record(stream)
            b.update(*_batch_frame_args(views, Wm + 1 + K + reps + s))
            g.replay()
            b.advance()
            for o, r in zip(outs, b.views):
                o.copy_(r.out, non_blocking=True)
            e1.record(stream)
            e1.synchronize()
            e_ms += e0.elapsed_time(e1)
        e2e_res = {"value": round(e_ms / K, 4), "unit": "ms/frame", "h2d_bytes_per_step": int(b.handle_bytes()),
                   "d2h_bytes_per_step": int(sum(o.numel() * 4 for o in outs)),
                   "note": f"h2d = the batch launch records (one pinned upload); d2h = {len(views)} RGBA32F images"}
        del outs
    b.close()
    del b, g
    torch.cuda.empty_cache()

    # plain form: the single-view calls, view after view, one frame per step
    plain = [H.Renderer(bvhs[v.room], v.width, v.height, v.params, device=dev) for v in views]

    def plain_frame(k):
        cams, prevs, lenses, ps = _batch_frame_args(views, k)
        for r, c, pv, ln, p in zip(plain, cams, prevs, lenses, ps):
            r.frame(c, pv, ln, p)

    for k in range(Wm):
        plain_frame(k)
    torch.cuda.synchronize()
    pev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(K)]
    for s in range(K):
        flush.zero_()
        pev[s][0].record(stream)
        plain_frame(Wm + s)
        pev[s][1].record(stream)
    torch.cuda.synchronize()
    plain_ms = float(np.mean([a.elapsed_time(c) for a, c in pev]))
    del plain
    torch.cuda.empty_cache()
    px = sum(v.width * v.height for v in views)
    return {
        "value": round(batch_ms, 4), "unit": "ms/frame", "steps": K, "views": len(views), "pixels": px,
        "triangles": [int(x.stats().n_tris) for x in bvhs],
        "tuning": {"trace_block": tune.trace_block, "trace_refill": tune.trace_refill,
                   "trace_chunk": tune.trace_chunk, "spatial_tile": tune.spatial_tile},
        "tuning_ms": {"x".join(map(str, k)): round(v, 3) for k, v in tune_ms.items()},
        "plain_ms": round(plain_ms, 4), "speedup_vs_plain": round(plain_ms / batch_ms, 3),
        "mrays_per_s_frame": round(rays / (batch_ms * 1e-3) / 1e6, 1),
        "mrays_per_s_trace": round(rays / (stage_ms[3] * 1e-3) / 1e6, 1) if stage_ms is not None else None,
        "rays_per_frame": int(rays), "traced_px_per_frame": int(traced),
        "stages": {n: round(float(t), 4) for n, t in zip(H.BATCH_STAGES, stage_ms)} if stage_ms is not None else None,
        "bvh_build_ms": round(bvh_ms, 3), "e2e": e2e_res, "clocks": clocks, "step_ms": step_ms,
    }


def run_batch(args):
    """The 64-view batched workload as its own bench line (--scene batch)."""
    import torch

    import paper_2210_04981_gb300.hdof as H

    ws, rank, local = dist_env()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=dev)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)
    if ws > 1:
        torch.distributed.barrier()
    res = batch_measure(H, dev, args.steps, args.warmup, args.views, flush, e2e=not args.no_e2e)
    total_ms = max_over_ranks(float(res["step_ms"].sum()), dev)
    K = args.steps
    batch_ms = total_ms / K
    stage_ms = res["stages"]
    dom = max(stage_ms, key=stage_ms.get)
    rays = res["rays_per_frame"]
    roof = {"bound": "alu", "achieved": None, "peak": None, "unit": "Tlane-op/s", "frac": None, "traffic": None,
            "kernel": dom}
    if dom == "trace":
        lane_peak = fp32_peak(H, dev) / 1e12
        ach = TRACE_OPS_PER_RAY * rays / (stage_ms["trace"] * 1e-3) / 1e12
        roof.update(achieved=round(ach, 2), peak=round(lane_peak, 2), frac=round(ach / lane_peak, 3),
                    ops_per_ray=TRACE_OPS_PER_RAY, peak_source="measured: hdof_probe_fma",
                    kernel="trace stage (k_ray_prefix, k_trace_*_batch, k_resolve_batch)")
    out = {
        "metric": METRIC, "value": round(batch_ms, 4), "unit": "ms/frame", "n_gpus": ws, "steps": K,
        "warmup": args.warmup, "ms_per_step": round(batch_ms, 4), "higher_is_better": False, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": f"{res['views']} views over 4 procedural rooms (50k-500k tris, seeds 10-13), "
                               "256^2..1920x1080, focus U[0.5,6], aperture U[0.01,0.1], 1-16 spp; one batched frame "
                               "per step",
                   "views": res["views"], "pixels": res["pixels"], "triangles": res["triangles"],
                   "tuning": res["tuning"], "tuning_ms": res["tuning_ms"],
                   "parallelism": f"replicas x{ws}" if ws > 1 else "single",
                   "l2": "flushed between steps (256 MiB write)"},
        "plain_ms": res["plain_ms"], "speedup_vs_plain": res["speedup_vs_plain"],
        "mrays_per_s_frame": res["mrays_per_s_frame"], "mrays_per_s_trace": res["mrays_per_s_trace"],
        "rays_per_frame": rays, "traced_px_per_frame": res["traced_px_per_frame"], "stages": stage_ms,
        "bvh_build_ms": res["bvh_build_ms"], "roofline": roof, "e2e": res["e2e"],
        # 16 launches per batched frame, 18 when each view's trace takes its default form (two trace launches)
        "gpu_launches": (18 if res["tuning"]["trace_refill"] == -1 else 16) * K,
        "clocks": res["clocks"],
    }
    if rank == 0:
        print(json.dumps(out), flush=True)
    if ws > 1:
        torch.distributed.destroy_process_group()


# ------------------------------------------------- differentiable path ---

# post-filter adjoint per (source, target) pair, FP32 lane-ops: squared distance
# (2), soft weight (1), depth test (2), 2 x 3 colour FFMA into dL/dC (6), two
# layer residual dots (6), four slope sums (4), selects and scaling (3)
PF_BWD_OPS_PER_TAP = 24


def run_diff(args):
    """Differentiable post-path at 1024x1024 with the visibility frozen from a
    100k-triangle room: each step is one forward and one backward pass
    (dL/dcolour, dL/dfocus, dL/daperture) at focus 2.0, aperture 0.03."""
    import torch

    import paper_2210_04981_gb300.hdof as H

    torch.cuda.set_device(0)
    dev = torch.device("cuda", 0)
    W = Hh = 1024
    col, z, scene, cam, target, start, p = hi.diff_config(W, Hh, 0)
    p = p.replace(camera_moved=0)
    bvh = H.hdof_build_bvh(*(torch.from_numpy(a).to(dev) for a in (scene.verts, scene.idx, scene.mat, scene.uv)))
    r = H.Renderer(bvh, W, Hh, p, device=dev)
    H.hdof_gbuffer(bvh, cam, cam, p, r.g)
    H.hdof_mask(r.g, None, p, r.edge, r.spp, r.ws)
    H.hdof_sync()
    spp = r.spp.clone()
    n_rays = int(spp.to(torch.int64).sum())
    rec = torch.empty((max(n_rays, 1), 4), dtype=torch.float32, device=dev)
    ray_off = torch.empty((Hh, W), dtype=torch.int32, device=dev)
    H.hdof_trace(bvh, cam, target, p, spp, r.rt, r.stats, r.ws, rec=rec, ray_off=ray_off)
    H.hdof_sync()
    del r
    hs = torch.from_numpy(hi.random_hist_samples(W, Hh, 0)).to(dev)
    path = H.PostPath(torch.from_numpy(z).to(dev), spp, rec, ray_off, hs, cam, p)
    C = torch.from_numpy(col).to(dev)
    Y = torch.from_numpy(np.random.default_rng(3).uniform(-1, 1, (Hh, W, 3)).astype(np.float32)).to(dev)
    zf, A = 2.0, 0.03
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)
    stream = torch.cuda.current_stream()
    for _ in range(args.warmup):
        path.forward(C, zf, A)
        path.backward(Y, zf, A)
    torch.cuda.synchronize()
    K = args.steps
    ev = [[torch.cuda.Event(enable_timing=True) for _ in range(3)] for _ in range(K)]
    sampler = ClockSampler(0, period_ms=20)
    sampler.__enter__()  # sampled through the eager, graph and end-to-end loops below
    for k in range(K):
        flush.zero_()
        ev[k][0].record(stream)
        path.forward(C, zf, A)
        ev[k][1].record(stream)
        path.backward(Y, zf, A)
        ev[k][2].record(stream)
    torch.cuda.synchronize()
    H.hdof_sync()
    fwd = float(np.mean([e[0].elapsed_time(e[1]) for e in ev]))
    bwd = float(np.mean([e[1].elapsed_time(e[2]) for e in ev]))
    # the same step with the lens on the device (the _dlens calls), captured
    # once into a CUDA graph and replayed: no host work between the kernels
    lens_dev = torch.tensor([zf, A], dtype=torch.float32, device=dev)
    gst = path.new_state()
    side = torch.cuda.Stream(device=dev)
    side.wait_stream(stream)
    with torch.cuda.stream(side):
        path.forward_dev(C, lens_dev, gst)
        path.backward_dev(Y, lens_dev, gst)
    stream.wait_stream(side)
    torch.cuda.synchronize()
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph):
        path.forward_dev(C, lens_dev, gst)
        path.backward_dev(Y, lens_dev, gst)
    gev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(K)]
    for k in range(K):
        flush.zero_()
        gev[k][0].record(stream)
        graph.replay()
        gev[k][1].record(stream)
    torch.cuda.synchronize()
    H.hdof_sync()
    graph_ms = float(np.mean([a.elapsed_time(b) for a, b in gev]))
    # end to end: colour image in from pinned host memory, gradients out
    hC = torch.from_numpy(col).pin_memory()
    hg = torch.empty((Hh, W, 3), dtype=torch.float32).pin_memory()
    hl = torch.empty(2, dtype=torch.float32).pin_memory()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e_ms = 0.0
    for k in range(K):
        flush.zero_()
        e0.record(stream)
        Cd = hC.to(dev, non_blocking=True)
        path.forward(Cd, zf, A)
        gcol, glens = path.backward(Y, zf, A)
        hg.copy_(gcol, non_blocking=True)
        hl.copy_(glens, non_blocking=True)
        e1.record(stream)
        e1.synchronize()
        e_ms += e0.elapsed_time(e1)
    sampler.__exit__(None, None, None)
    clocks = sampler.summary()
    taps = contributing_taps(z.astype(np.float64), hi.Lens(zf, A, 0.05), Hh, cam.tan_half_fovy, p.r_max)
    lane_peak = fp32_peak(H, dev) / 1e12
    ach = taps * PF_BWD_OPS_PER_TAP / (bwd * 1e-3) / 1e12
    out = {
        "metric": "differentiable post-path ms per forward+backward step (1024x1024, frozen visibility)",
        "value": round(fwd + bwd, 4), "unit": "ms/step", "n_gpus": 1, "steps": K, "warmup": args.warmup,
        "ms_per_step": round(fwd + bwd, 4), "higher_is_better": False, "scaling": "weak", "vs_baseline": None,
        "dtype": "f32", "data": "synthetic",
        "config": {"workload": "1024x1024 colour U[0,1], depth U[0.3,8] 9x9-box smoothed, visibility of a "
                               "100k-triangle room traced at focus 2.5 / aperture 0.04; step at focus 2.0 / "
                               "aperture 0.03", "rays": n_rays, "l2": "flushed between steps (256 MiB write)"},
        "forward_ms": round(fwd, 4), "backward_ms": round(bwd, 4), "contributing_taps": taps,
        "graph_step_ms": round(graph_ms, 4),
        "roofline": {"bound": "alu", "achieved": round(ach, 2), "peak": round(lane_peak, 2), "unit": "Tlane-op/s",
                     "frac": round(ach / lane_peak, 3), "traffic": None,
                     "kernel": "hdof_post_backward (post-filter adjoint dominates)",
                     "ops_per_tap": PF_BWD_OPS_PER_TAP, "peak_source": "measured: hdof_probe_fma"},
        "e2e": {"value": round(e_ms / K, 4), "unit": "ms/step", "h2d_bytes_per_step": int(hC.numel() * 4),
                "d2h_bytes_per_step": int(hg.numel() * 4 + 8)},
        "gpu_launches": 14 * K, "clocks": clocks,
    }
    print(json.dumps(out), flush=True)


# ------------------------------------------------------------ the oracle ---

def oracle_frame_sample(O, osc, cams, lens, p0, k, hist, W, Hh, pf_stride):
    """One oracle frame: every stage at full resolution; with pf_stride > 1 the
    post-filter and composite on pixel samples.  Returns the history, the stage
    times and the full-frame time (measured for pf_stride 1, else extrapolated
    from the two samples)."""
    cam, prev = cams[k], cams[max(k - 1, 0)]
    p = p0.replace(frame=k, camera_moved=int(k > 0))
    t = {}
    t0 = time.perf_counter()
    g = O.gbuffer(osc, cam, prev, p)
    t["gbuffer"] = time.perf_counter() - t0
    t0 = time.perf_counter()
    m = O.mask(g["nd"], g["mv"], p, hist["mom"], hist["hlen"])
    t["mask"] = time.perf_counter() - t0
    t0 = time.perf_counter()
    rt = O.trace(osc, cam, lens, p, m["spp"])
    t["trace"] = time.perf_counter() - t0
    t0 = time.perf_counter()
    nh, crt, hacc = O.temporal(cam, prev, p, rt, m["spp"], g["nd"], g["mv"], hist)
    crec = O.spatial(p, crt, m["spp"], nh["mom"], nh["hlen"])
    t["reconstruct"] = time.perf_counter() - t0
    if pf_stride <= 1:  # the whole frame, measured
        t0 = time.perf_counter()
        pp = O.postfilter(g["nd"], g["col"], lens, cam.tan_half_fovy, p)
        O.composite(g["nd"], g["col"], m["spp"], pp, crt, crec, hacc, lens, cam.tan_half_fovy, p, Hh)
        t["postfilter_composite"] = time.perf_counter() - t0
        return nh, t, sum(t.values())
    # the post-filter and composite on seeded uniform samples of 1/pf_stride and
    # 1/(4 pf_stride) of the pixels (a regular stride would be biased: the
    # gather's cost per pixel follows its blur); the full-frame time is the
    # per-call part plus the per-pixel slope times the frame's pixel count
    def pf_sample(n, seed):
        pix = np.sort(np.random.default_rng(seed).choice(W * Hh, n, replace=False)).astype(np.int32)
        t0 = time.perf_counter()
        pp = O.postfilter(g["nd"], g["col"], lens, cam.tan_half_fovy, p, pix=pix)
        flat = lambda a: a.reshape(W * Hh, *a.shape[2:])[pix]  # noqa: E731
        O.composite(flat(g["nd"]), flat(g["col"]), flat(m["spp"]), pp, flat(crt), flat(crec), flat(hacc), lens,
                    cam.tan_half_fovy, p, Hh)
        return time.perf_counter() - t0

    n1 = (W * Hh) // pf_stride
    n2 = max(n1 // 4, 1)
    t1, t2 = pf_sample(n1, 1000 + k), pf_sample(n2, 2000 + k)
    slope = max(t1 - t2, 0.0) / max(n1 - n2, 1)
    t["postfilter_sample"] = t1
    t["postfilter_quarter_sample"] = t2
    pf_full = max(t1 - slope * n1, 0.0) + slope * W * Hh
    est = t["gbuffer"] + t["mask"] + t["trace"] + t["reconstruct"] + pf_full
    return nh, t, est


def cpu_baseline(args, budget_s=30.0):
    from oracle import oracle as O
    O.build()
    W, Hh, make_scene, over, _ = SCENES["room"]
    if args.width:
        W, Hh = args.width, args.height
    scene = make_scene(W / Hh)
    lens = hi.room_lens()
    p0 = hi.room_params()
    cams = [hi.room_camera(k, W, Hh) for k in range(2)]
    osc = O.OScene(scene)
    hist = O.empty_history(W, Hh)
    stride = 16
    _, t, est = oracle_frame_sample(O, osc, cams, lens, p0, 0, hist, W, Hh, stride)
    return {"value": round(est * 1e3, 1), "unit": "ms/frame", "cores": O.num_threads(), "kind": "oracle",
            "sample": f"frame 0 at {W}x{Hh}: all stages full-frame except post-filter+composite, timed on seeded "
                      f"uniform samples of 1/{stride} and 1/{4 * stride} of the pixels and extrapolated linearly to "
                      f"the frame; measured {sum(t.values()):.1f} s",
            "stage_s": {k: round(v, 3) for k, v in t.items()}}


def run_reference(args):
    ws, rank, _ = dist_env()
    if rank != 0:
        return
    from oracle import oracle as O
    O.build()
    W, Hh, make_scene, over, workload = SCENES["room"]
    if args.width:
        W, Hh = args.width, args.height
    scene = make_scene(W / Hh)
    lens = hi.room_lens()
    p0 = hi.room_params()
    n = args.warmup + args.steps
    cams = [hi.room_camera(k, W, Hh) for k in range(n)]
    osc = O.OScene(scene)
    hist = O.empty_history(W, Hh)
    stride = args.ref_pf_stride
    ests, meas = [], []
    for k in range(n):
        hist, t, est = oracle_frame_sample(O, osc, cams, lens, p0, k, hist, W, Hh, stride)
        if k >= args.warmup:
            ests.append(est)
            meas.append(sum(t.values()))
    value = float(np.mean(ests)) * 1e3
    step = float(np.mean(meas)) * 1e3
    if stride <= 1:
        sample = (f"each step: one consecutive {W}x{Hh} frame, every stage full-frame, measured "
                  f"({step / 1e3:.2f} s per frame)")
    else:
        sample = (f"each step: one consecutive {W}x{Hh} frame, every stage full-frame except post-filter+composite, "
                  f"which run on seeded uniform samples of 1/{stride} and 1/{4 * stride} of the pixels; value = the "
                  f"full-frame time extrapolated linearly from the two samples, ms_per_step = the measured time of "
                  f"the sampled step ({step / 1e3:.2f} s)")
    out = {"impl": "reference", "metric": METRIC, "value": round(value, 1), "unit": "ms/frame", "n_gpus": ws,
           "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(step, 1), "higher_is_better": False,
           "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
           "config": {"workload": workload, "width": W, "height": Hh, "triangles": scene.n_tris,
                      "storage": "f32", "spp_max": p0.spp_max, "r_max": p0.r_max, "parallelism": "single",
                      "l2": "n/a (host CPU)"},
           "cpu_baseline": {"value": round(value, 1), "unit": "ms/frame", "cores": O.num_threads(),
                            "kind": "oracle", "sample": sample},
           "e2e": {"value": round(value, 1), "unit": "ms/frame", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out), flush=True)


def main():
    ap = argparse.ArgumentParser(description=__doc__.split("\n")[0])
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--scene", choices=sorted(SCENES) + ["batch", "diff"], default="room")
    ap.add_argument("--precision", choices=["f32", "mixed"], default="f32")
    ap.add_argument("--width", type=int, default=0, help="override the scene's resolution")
    ap.add_argument("--height", type=int, default=0)
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-budget", type=float, default=30.0)
    ap.add_argument("--ref-pf-stride", type=int, default=1,
                    help="reference arm: 1 = whole oracle frames (measured); n > 1 = post-filter and composite on "
                         "1/n and 1/(4n) pixel samples, extrapolated")
    ap.add_argument("--views", type=int, default=64, help="views of the batched workload")
    ap.add_argument("--rt-passes", type=int, default=32,
                    help="passes of spp_max lens samples of the full ray-traced quality reference")
    ap.add_argument("--no-compare", action="store_true",
                    help="skip the mixed-precision and batched comparisons of the default line")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        run_reference(args)
    elif args.scene == "batch":
        run_batch(args)
    elif args.scene == "diff":
        run_diff(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
