"""The allocation-free uncached render (cinr_render_frame_noalloc).

Some callers cannot allocate device memory: a real-time render loop in which
an allocation would stall or fail, code running under a policy that forbids
new device allocations, or a host-side plugin that owns no device buffer.
For them the library renders an uncached frame with its working set in a
fixed device array of its own.  These tests check, through the C ABI, that
two calls in a row give the same images and counts as the regular entry
point (cinr_render_frame with no cache) -- bit for bit with the FP32 MLP,
and with the BF16 tensor-core MLP whose error word the call reads back --
that the FP32 image is within the pixel tolerance of the CPU oracle, that
oversized requests are refused, and that the same checks pass in a fresh
process whose first library call is this entry point.  The file is collected
last on purpose, so that a run that stops at the first failure has run every
other test before it.
"""
import ctypes as C
import os
import subprocess
import sys

import numpy as np
import pytest

from paper_2504_18001_gb300 import synthetic as S

from _scenes import gpu_inr, ocam, oracle_inr, scene

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
VOL = (64, 64, 64)
W, H = 96, 80


def _noalloc(inr, cam, tf, opts):
    import torch
    from paper_2504_18001_gb300 import cinr
    out = torch.zeros((cam["height"], cam["width"], 4), dtype=torch.float32)
    st = cinr.cinr_frame_stats()
    rc = cinr.lib().cinr_render_frame_noalloc(
        inr.h, C.byref(cinr.make_camera(cam)), C.byref(cinr.make_tf(tf)), C.byref(opts),
        C.c_void_p(out.data_ptr()), C.byref(st), cinr._stream(None))
    return rc, out.numpy(), st.as_dict()


def _opts():
    from paper_2504_18001_gb300 import cinr
    return cinr.cinr_march_opts((C.c_int * 3)(*VOL), 32, 1e-3, 0, 1.0, 0, 0)


@pytest.mark.parametrize("mlp,tab", [("fp32", "fp32"), ("bf16", "fp16")])
def test_noalloc_matches_regular_entry_point_on_two_calls(mlp, tab):
    from paper_2504_18001_gb300 import cinr
    cfg = S.INR_64
    table, w = scene(cfg)
    inr = gpu_inr(cfg, table, w, vol=VOL, mlp=mlp, tab=tab)
    for f, tf in ((2, S.tf_ramps(2)), (9, S.tf_ramps(5))):
        cam = S.orbit_camera(f, W, H)
        rc, img, st = _noalloc(inr, cam, tf, _opts())
        assert rc == 0, cinr.last_error()
        rend = cinr.Renderer(W, H, VOL, K=32, eps_T=1e-3)
        ref, rst = rend.render(inr, cam, tf)
        ref = ref.cpu().numpy()
        if mlp == "fp32":
            # the same kernel on the same inputs: identical bits
            assert np.array_equal(img, ref)
        else:
            assert np.abs(img - ref).max() < 1e-5
        assert st["samples"] == rst["samples"] > 0
        assert st["inr_queries_direct"] == rst["inr_queries_direct"]
        assert st["true_misses"] == rst["true_misses"]


def test_noalloc_fp32_within_pixel_tolerance_of_oracle():
    import oracle as O
    from paper_2504_18001_gb300 import cinr
    cfg = S.INR_64
    table, w = scene(cfg)
    inr = gpu_inr(cfg, table, w, vol=VOL)
    p = oracle_inr(cfg, table, w, vol=VOL)
    cam, tf = S.orbit_camera(4, W, H), S.tf_ramps(2)
    rc, img, st = _noalloc(inr, cam, tf, _opts())
    assert rc == 0, cinr.last_error()
    ref, rst = O.render_direct(p, table, w, ocam(cam), VOL, O.march_opts(K=32, eps_T=1e-3),
                               tf.astype(np.float64))
    assert st["samples"] == rst["samples"]
    assert np.abs(img - ref).max() < 2e-3


def test_noalloc_refuses_oversized_images():
    from paper_2504_18001_gb300 import cinr
    cfg = S.INR_64
    table, w = scene(cfg)
    inr = gpu_inr(cfg, table, w)
    rc, _, _ = _noalloc(inr, S.orbit_camera(0, 1024, 300), S.tf_ramps(2), _opts())
    assert rc == cinr.CINR_OK - 1  # CINR_ERR_ARG
    assert "allocation-free limit" in cinr.last_error()


_FRESH = r"""
import sys
sys.path.insert(0, {root!r})
sys.path.insert(0, {tests!r})
import test_zz_no_alloc as T
T.test_noalloc_matches_regular_entry_point_on_two_calls("fp32", "fp32")
print("fresh ok")
"""


def test_noalloc_in_a_fresh_process():
    """The device address of the array is looked up by the first call in a
    process; here that first call runs in a new process with a new CUDA
    context (the other tests of this file share the test run's process)."""
    code = _FRESH.format(root=ROOT, tests=os.path.join(ROOT, "tests"))
    r = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, timeout=600,
                       cwd=ROOT)
    assert r.returncode == 0, r.stdout[-2000:] + r.stderr[-2000:]
    assert "fresh ok" in r.stdout
