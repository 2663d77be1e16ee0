"""The library's kernel timing and FP32 probe on the GPU: a profiled frame
reports each of its kernels once with a positive device time, nothing is
recorded while profiling is off, and the FMA probe's lane-instruction count
and time give a rate near the SMs x 128 lanes x clock ceiling."""
import numpy as np
import pytest

import hdof_inputs as hi

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("needs a CUDA device", allow_module_level=True)

import paper_2210_04981_gb300.hdof as H  # noqa: E402
from gpu_util import bvh_of  # noqa: E402


def test_profiled_frame_names_every_kernel():
    scene, cam, lens, p = hi.tiny_config()
    r = H.Renderer(bvh_of(scene), cam.width, cam.height, p)
    r.frame(cam, cam, lens, p)
    H.hdof_sync()
    H.hdof_profile_read()
    H.hdof_profile(True)
    for _ in range(3):
        r.frame(cam, cam, lens, p)
    H.hdof_profile(False)
    got = H.hdof_profile_read()
    r.frame(cam, cam, lens, p)  # not recorded
    H.hdof_sync()
    assert H.hdof_profile_read() == {}
    want = {"gbuffer", "mask", "trace_compact", "trace_resolve", "pf_prep", "pf_rowscan", "pf_gather", "temporal",
            "spatial", "composite"}
    assert want <= set(got), got
    assert ("trace_packets" in got) != ("trace_rays" in got)
    for name, (n, ms) in got.items():
        assert n == 3 and ms > 0.0, (name, n, ms)


def test_fma_probe_rate():
    dev = torch.device("cuda")
    sink = torch.zeros(256, dtype=torch.float32, device=dev)
    props = torch.cuda.get_device_properties(dev)
    best = 0.0
    for k in range(4):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        ops = H.hdof_probe_fma(8, 4000, sink)
        e1.record()
        e1.synchronize()
        if k:
            best = max(best, ops / (e0.elapsed_time(e1) * 1e-3))
    assert ops == props.multi_processor_count * 8 * 256 * 4000 * 128
    ceiling = props.multi_processor_count * 128 * 2.2e9  # lanes x an upper bound of the SM clock
    assert 0.3 * ceiling < best < ceiling, best
    assert not np.any(sink.cpu().numpy())
