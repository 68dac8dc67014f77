"""GPU parity of the uncached (direct INR) render against the CPU oracle."""
import math

import numpy as np
import pytest

import oracle as O
from paper_2504_18001_gb300 import synthetic as S

from _scenes import gpu_inr, ocam, oracle_inr, scene

pytestmark = pytest.mark.gpu


def _setup(cfg=S.INR_64, vol=(64, 64, 64)):
    table, w = scene(cfg)
    return table, w, gpu_inr(cfg, table, w, vol=vol), oracle_inr(cfg, table, w, vol=vol)


@pytest.mark.parametrize("size", [(128, 128), (37, 29)], ids=["128px", "ragged"])
def test_uncached_render_matches_oracle(size):
    from paper_2504_18001_gb300 import cinr
    W, H = size
    vol = (64, 64, 64)
    table, w, inr, p = _setup()
    cam = S.orbit_camera(3, W, H)
    tf = S.tf_ramps(2)
    r = cinr.Renderer(W, H, vol, K=32, eps_T=0.0)
    img, st = r.render(inr, cam, tf)
    ref, rst = O.render_direct(p, table, w, ocam(cam), vol, O.march_opts(K=32, eps_T=0.0),
                               tf.astype(np.float64))
    assert st["samples"] == rst["samples"] == st["inr_queries_direct"] == st["true_misses"]
    assert np.abs(img.cpu().numpy() - ref).max() < 2e-3


def test_uncached_early_termination_within_tolerance():
    from paper_2504_18001_gb300 import cinr
    vol = (64, 64, 64)
    table, w, inr, p = _setup()
    cam = S.orbit_camera(10, 96, 64)
    tf = S.tf_ramps(2) * np.array([1, 1, 1, 4], np.float32)
    r = cinr.Renderer(96, 64, vol, K=64, eps_T=1e-3)
    img, st = r.render(inr, cam, tf)
    ref, rst = O.render_direct(p, table, w, ocam(cam), vol, O.march_opts(K=64, eps_T=1e-3),
                               tf.astype(np.float64))
    assert np.abs(img.cpu().numpy() - ref).max() < 2e-3
    # termination decisions may differ only for rays whose T is within rounding of eps
    assert abs(st["samples"] - rst["samples"]) <= 64 * 4


@pytest.mark.parametrize("sigma", [0.5, 8.0])
def test_constant_density_slab_exp(sigma):
    from paper_2504_18001_gb300 import cinr
    cfg = S.INR_64
    vol = (64, 48, 80)
    table = np.zeros(cfg.table_entries, np.float32)
    w = np.zeros(cfg.mlp_params, np.float32)
    inr = cinr.Inr(cinr.make_inr_params(cfg, vmin=0.5, vmax=1.5), table, w)
    cam = S.orbit_camera(0, 40, 30)
    tf = S.tf_constant((0.25, 0.5, 1.0), sigma)
    r = cinr.Renderer(40, 30, vol, K=32, eps_T=0.0)
    img = r.render(inr, cam, tf)[0].cpu().numpy()
    oc = ocam(cam)
    for py in range(30):
        for px in range(40):
            hit, o, d, tn, tf_ = O.ray(oc, vol, px, py)
            a = 1.0 - math.exp(-sigma * (tf_ - tn)) if hit else 0.0
            assert abs(img[py, px, 3] - a) < 1e-5
            assert abs(img[py, px, 2] - a) < 1e-5


def test_render_host_equals_device():
    import torch
    from paper_2504_18001_gb300 import cinr
    vol = (64, 64, 64)
    table, w, inr, p = _setup()
    cam = S.orbit_camera(1, 64, 48)
    tf = S.tf_ramps(2)
    r = cinr.Renderer(64, 48, vol, K=32, eps_T=1e-3)
    img, st = r.render(inr, cam, tf)
    host = torch.empty((48, 64, 4), dtype=torch.float32).pin_memory()
    st2 = r.render_host(inr, cam, tf, host)
    assert torch.equal(host, img.cpu())
    assert st2["samples"] == st["samples"]


def test_bad_arguments_raise():
    from paper_2504_18001_gb300 import cinr
    vol = (64, 64, 64)
    table, w, inr, p = _setup()
    r = cinr.Renderer(16, 16, vol)
    with pytest.raises(cinr.CinrError):
        r.render(inr, S.orbit_camera(0, 17, 16), S.tf_ramps(2))
    with pytest.raises(cinr.CinrError):
        cinr.Renderer(16, 16, vol, K=48)
