"""GB300-native hybrid depth of field (Tan et al., SIGGRAPH '20 Posters).

The compute path is ``libhdof.so`` (hand-written CUDA for sm_103a, C ABI in
``include/hdof.h``); :mod:`.hdof` is its ctypes binding and
:class:`.hdof.Renderer` enqueues one frame.
"""
from .hdof import (Bvh, GBuffer, HdofError, History, Renderer, hdof_build_bvh, hdof_closest_hits,  # noqa: F401
                   hdof_composite, hdof_gbuffer, hdof_mask, hdof_postfilter, hdof_reconstruct, hdof_sync,
                   hdof_trace, hdof_version, hdof_workspace_bytes, load)
