"""Edge cases of the cached renderer against the oracle: a view that misses
the volume (no samples, nothing requested), a single-pixel image, a volume
smaller than one brick, a one-LoD cache (everything preloaded: no request),
a request budget of one brick, termination at the first segment boundary,
the largest request budget the library accepts, and a bounded device-side
wait that runs out (reported, not faulted)."""
import numpy as np
import pytest

import oracle as O
from paper_2504_18001_gb300 import synthetic as S

from _scenes import gpu_inr, ocam, oracle_inr, scene
from test_gpu_cache import _run

pytestmark = pytest.mark.gpu


def test_view_missing_the_volume_renders_nothing():
    def cam_fn(f, W, H):
        c = S.orbit_camera(0, W, H, distance=3.0)
        c["target"] = tuple(2 * np.asarray(c["eye"]))  # looking away
        return c
    cache, oc, hist, worst = _run(2, cam_fn=cam_fn)
    for h in hist:
        assert h["samples"] == h["bricks_requested"] == h["bricks_decoded"] == 0


def test_single_pixel_image():
    _run(3, W=1, H=1, cam_fn=lambda f, W, H: S.orbit_camera(3 * f, W, H, distance=1.5))


def test_volume_smaller_than_a_brick():
    cache, oc, hist, worst = _run(3, vol=(5, 3, 7), W=24, H=16, levels=2, slots=8, n_req=4)
    assert hist[0]["samples"] > 0


def test_single_lod_cache_is_fully_preloaded():
    cache, oc, hist, worst = _run(2, levels=1, slots=512)
    for h in hist:
        assert h["bricks_requested"] == 0 and h["fallback_hits"] == 0
        assert h["hits"] == h["samples"] > 0


def test_request_budget_of_one_brick():
    cache, oc, hist, worst = _run(4, n_req=1, slots=40)
    assert all(h["bricks_decoded"] <= 1 for h in hist)
    assert sum(h["bricks_decoded"] for h in hist) >= 3


def test_termination_at_the_first_segment_boundary():
    # eps_T = 1: every ray stops after its first K samples
    cache, oc, hist, worst = _run(2, eps=1.0, K=32)
    assert hist[0]["samples"] > 0


def test_largest_request_budget():
    from paper_2504_18001_gb300 import cinr
    cfg = S.INR_64
    table, w = scene(cfg)
    inr = gpu_inr(cfg, table, w, vol=(64, 64, 64))
    cinr.Cache(inr, (64, 64, 64), pool_bytes=600 * 4000, brick=8, levels=3, n_req=8192)
    with pytest.raises(cinr.CinrError):
        cinr.Cache(inr, (64, 64, 64), pool_bytes=600 * 4000, brick=8, levels=3, n_req=8193)


def test_bounded_wait_runs_out_and_reports_timeout():
    # failure detection without a fault: a wait on an mbarrier phase that
    # nothing completes gives up after its poll limit, the status call
    # reports CINR_ERR_TIMEOUT once (then clears), and the context stays
    # usable for inference
    import ctypes as C
    import torch
    from paper_2504_18001_gb300 import cinr
    from _scenes import gpu_inr, scene
    cfg = S.INR_64
    table, w = scene(cfg)
    inr = gpu_inr(cfg, table, w, vol=(32, 32, 32), mlp="bf16")
    L = cinr.lib()
    s = cinr._stream(None)
    assert L.cinr_inr_status(inr.h, s) == 0
    cinr.check(L.cinr_debug_wait_timeout(inr.h, 256, s), "cinr_debug_wait_timeout")
    assert L.cinr_inr_status(inr.h, s) == cinr.ERR_TIMEOUT
    assert "wait gave up" in cinr.last_error()
    assert L.cinr_inr_status(inr.h, s) == 0
    v = inr.infer(torch.from_numpy(S.random_points(1000, 3)).cuda())
    assert torch.isfinite(v).all()
    assert L.cinr_inr_status(inr.h, s) == 0
