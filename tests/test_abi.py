"""The C-ABI library builds, loads without a GPU, exports every entry point
that include/hdof.h declares, and rejects bad arguments on the host before
touching the device."""
import ctypes as C
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def H():
    from paper_2210_04981_gb300 import build as b
    b.build()
    import paper_2210_04981_gb300.hdof as H
    H.load()
    return H


def declared_functions():
    src = open(os.path.join(ROOT, "include", "hdof.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(hdof_[a-z_0-9]+)\s*\(", src)))


def test_header_declares_the_boundary():
    names = declared_functions()
    for n in ("hdof_build_bvh", "hdof_gbuffer", "hdof_mask", "hdof_trace", "hdof_postfilter", "hdof_reconstruct",
              "hdof_composite"):
        assert n in names


def test_every_declared_symbol_is_exported(H):
    lib = C.CDLL(H.LIB_PATH)
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing
    assert set(H.exported_symbols()) <= set(declared_functions())


def test_host_only_calls(H):
    assert "sm_103a" in H.hdof_version()
    p = H.params(None)
    assert p.tile == 16 and p.spp_max == 16 and abs(p.light_dir[0][2] + 0.8638684) < 1e-6
    assert H.hdof_workspace_bytes(1920, 1080) >= 1920 * 1080 * 16
    assert H.hdof_workspace_bytes(0, 10) == 0


def test_struct_layout_matches_header(H, tmp_path):
    """Sizes and field offsets of the ctypes records equal those a C compiler
    gives the header's structs."""
    import subprocess
    recs = {"hdof_camera": H.hdof_camera, "hdof_lens": H.hdof_lens, "hdof_params": H.hdof_params,
            "hdof_gbuf": H.hdof_gbuf, "hdof_history": H.hdof_history, "hdof_bvh_stats": H.hdof_bvh_stats,
            "hdof_post_state": H.hdof_post_state, "hdof_view": H.hdof_view, "hdof_tuning": H.hdof_tuning,
            "hdof_kernel_time": H.hdof_kernel_time}
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "hdof.h"', "int main(void) {"]
    for name, rec in recs.items():
        lines.append(f'printf("{name} %zu\\n", sizeof({name}));')
        for f, _ in rec._fields_:
            lines.append(f'printf("{name}.{f} %zu\\n", offsetof({name}, {f}));')
    lines.append("return 0; }")
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines))
    exe = tmp_path / "layout"
    subprocess.check_call(["gcc", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)])
    out = dict(l.rsplit(" ", 1) for l in subprocess.check_output([str(exe)], text=True).split("\n") if l)
    for name, rec in recs.items():
        assert int(out[name]) == C.sizeof(rec), name
        for f, _ in rec._fields_:
            assert int(out[f"{name}.{f}"]) == getattr(rec, f).offset, f"{name}.{f}"


def _call(H, name, *args):
    return getattr(H.load(), name)(*args)


def test_invalid_arguments_rejected_before_launch(H):
    import hdof_inputs as hi
    cam = H.camera(hi.Camera(width=64, height=48))
    bad = H.camera(hi.Camera(width=0, height=48))
    p = H.params(hi.Params())
    g = H.hdof_gbuf(64, 48, 0, 0, None, None, None, None)
    lib = H.load()
    assert lib.hdof_gbuffer(None, C.byref(cam), C.byref(cam), C.byref(p), None, C.byref(g), None) == -1
    assert lib.hdof_build_bvh(None, 0, None, 0, None, None, C.byref(C.c_void_p()), None) == -1
    assert lib.hdof_mask(C.byref(g), None, C.byref(p), None, None, None, 0, None) == -1
    assert lib.hdof_postfilter(C.byref(g), C.byref(bad), None, C.byref(p), None, None, 0, None) == -1
    buf = C.create_string_buffer(256)
    lib.hdof_last_error(buf, 256)
    assert b"image size" in buf.value
    p_bad = H.params(hi.Params(spp_max=300))
    assert lib.hdof_trace(C.c_void_p(1), C.byref(cam), C.byref(H.lens(hi.Lens())), C.byref(p_bad), None, None, None,
                          None, None, None, None, 0, None, None) == -1
    lib.hdof_last_error(buf, 256)
    assert b"spp_max" in buf.value
    # batched calls: empty batch, unsupported launch shape, NULL handle
    views = (H.hdof_view * 1)()
    h = C.c_void_p()
    assert lib.hdof_batch_create(views, 0, None, C.byref(h), None) == -1
    assert lib.hdof_batch_create(views, 1, C.byref(H.tuning(96, 1)), C.byref(h), None) == -1
    lib.hdof_last_error(buf, 256)
    assert b"trace_block" in buf.value
    assert lib.hdof_batch_create(views, 1, C.byref(H.tuning(128, -2)), C.byref(h), None) == -1
    lib.hdof_last_error(buf, 256)
    assert b"trace_refill" in buf.value
    assert lib.hdof_batch_create(views, 1, C.byref(H.tuning(128, 33)), C.byref(h), None) == -1
    assert lib.hdof_batch_render(None, None) == -1
    assert lib.hdof_batch_update(None, views, 1, None) == -1
    assert lib.hdof_batch_destroy(None) == 0
    # the post-path with the lens on the device: a NULL lens array, then the
    # other arguments, are rejected on the host
    st = H.hdof_post_state()
    assert lib.hdof_post_forward_dlens(C.byref(g), None, None, None, None, C.byref(cam), None, C.byref(p),
                                       C.byref(st), None, 0, None) == -1
    lib.hdof_last_error(buf, 256)
    assert b"lens_dev" in buf.value
    assert lib.hdof_post_backward_dlens(C.byref(g), None, None, None, None, C.byref(cam), None, C.byref(p),
                                        C.byref(st), None, None, None, None, 0, None) == -1
    assert lib.hdof_post_forward_dlens(C.byref(g), None, None, None, None, C.byref(bad), C.c_void_p(256), C.byref(p),
                                       C.byref(st), None, 0, None) == -1
    lib.hdof_last_error(buf, 256)
    assert b"image size" in buf.value


def test_python_binding_requires_cuda_tensors(H):
    torch = pytest.importorskip("torch")
    with pytest.raises((ValueError, TypeError)):
        H._ptr(torch.zeros(4))
