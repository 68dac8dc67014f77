"""The allocation-free uncached render (cinr_render_frame_noalloc).

Some callers cannot allocate device memory: a real-time render loop in which
an allocation would stall or fail, code running under a policy that forbids
new device allocations, or a host-side plugin that owns no device buffer.
For them the library renders an uncached frame with its working set in a
fixed device array of its own.  This file checks, through the C ABI, that two
calls in a row give the same images and counts as the regular entry point
(cinr_render_frame with no cache), and that oversized requests are refused.
It is collected last on purpose: it must pass alone in a fresh process and
after every other test.
"""
import ctypes as C

import numpy as np
import pytest

from paper_2504_18001_gb300 import synthetic as S

from _scenes import gpu_inr, scene

pytestmark = pytest.mark.gpu


def _noalloc(inr, cam, tf, opts):
    import torch
    from paper_2504_18001_gb300 import cinr
    out = torch.zeros((cam["height"], cam["width"], 4), dtype=torch.float32)
    st = cinr.cinr_frame_stats()
    rc = cinr.lib().cinr_render_frame_noalloc(
        inr.h, C.byref(cinr.make_camera(cam)), C.byref(cinr.make_tf(tf)), C.byref(opts),
        C.c_void_p(out.data_ptr()), C.byref(st), cinr._stream(None))
    return rc, out.numpy(), st.as_dict()


def test_noalloc_matches_regular_entry_point_on_two_calls():
    from paper_2504_18001_gb300 import cinr
    vol = (64, 64, 64)
    cfg = S.INR_64
    table, w = scene(cfg)
    inr = gpu_inr(cfg, table, w, vol=vol)
    W, H = 96, 80
    opts = cinr.cinr_march_opts((C.c_int * 3)(*vol), 32, 1e-3, 0, 1.0, 0, 0)
    rend = cinr.Renderer(W, H, vol, K=32, eps_T=1e-3)
    for f, tf in ((2, S.tf_ramps(2)), (9, S.tf_ramps(5))):
        cam = S.orbit_camera(f, W, H)
        rc, img, st = _noalloc(inr, cam, tf, opts)
        assert rc == 0, cinr.last_error()
        ref, rst = rend.render(inr, cam, tf)
        assert np.abs(img - ref.cpu().numpy()).max() < 2e-3
        assert st["samples"] == rst["samples"] > 0
        assert st["inr_queries_direct"] == rst["inr_queries_direct"]


def test_noalloc_refuses_oversized_images():
    from paper_2504_18001_gb300 import cinr
    vol = (64, 64, 64)
    cfg = S.INR_64
    table, w = scene(cfg)
    inr = gpu_inr(cfg, table, w)
    opts = cinr.cinr_march_opts((C.c_int * 3)(*vol), 32, 1e-3, 0, 1.0, 0, 0)
    rc, _, _ = _noalloc(inr, S.orbit_camera(0, 1024, 300), S.tf_ramps(2), opts)
    assert rc == cinr.CINR_OK - 1  # CINR_ERR_ARG
    assert "allocation-free limit" in cinr.last_error()
