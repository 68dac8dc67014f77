"""Macro cells (Sec. 5.2) on the GPU: value ranges against the oracle, skip
flags bit-exact, cached / uncached / explicit-field frames with skipping
against the oracle (state bit-exact, pixels within 2e-3), and the exactness
property: with ranges that bound every sample, skipping leaves the image
bit-identical."""
import numpy as np
import pytest

import oracle as O
from paper_2504_18001_gb300 import synthetic as S

from _scenes import gpu_inr, ocam, oracle_inr, scene
from test_gpu_cache import _run

pytestmark = pytest.mark.gpu


def _gated_tf(theta, seed=2):
    # ramps above value theta, transparent below
    tf = S.tf_ramps(seed)
    tf[: int(theta * 255), 3] = 0.0
    tf[int(theta * 255):, 3] = np.maximum(tf[int(theta * 255):, 3], 8.0)
    return tf


def _scene64(vol=(64, 64, 64), mlp="fp32", tab="fp32"):
    cfg = S.INR_64
    table, w = scene(cfg)
    return cfg, table, w, gpu_inr(cfg, table, w, vol=vol, mlp=mlp, tab=tab), oracle_inr(cfg, table, w, vol=vol)


@pytest.mark.parametrize("vol,cell", [((64, 64, 64), 8), ((48, 40, 72), 16)])
def test_ranges_from_inr_match_oracle(vol, cell):
    from paper_2504_18001_gb300 import cinr
    cfg, table, w, inr, p = _scene64(vol)
    ref = O.macro_ranges_inr(p, table, w, vol, cell, 3)
    m = cinr.Macro(vol, cell, inr=inr, levels=3)
    got = m.ranges()
    assert got.shape == ref.shape
    assert np.abs(got - ref).max() < 1e-4
    # with a cache: the cache's LoD count (3) and FP32 storage give the same ranges
    cache = cinr.Cache(inr, vol, pool_bytes=100 * 1000 * 4, brick=8, levels=3, n_req=8)
    got2 = cinr.Macro(vol, cell, inr=inr, cache=cache).ranges()
    assert np.array_equal(got, got2)
    # min_level > 0 narrows the ranges
    got3 = cinr.Macro(vol, cell, inr=inr, levels=3, min_level=1).ranges()
    assert np.all(got3[:, 0] >= got[:, 0]) and np.all(got3[:, 1] <= got[:, 1])


def test_ranges_from_field_exact():
    import torch
    from paper_2504_18001_gb300 import cinr
    rng = np.random.default_rng(3)
    f = rng.normal(size=(33, 20, 47)).astype(np.float32)
    ref = O.macro_ranges_field(f, 8)
    got = cinr.Macro((47, 20, 33), 8, field=torch.from_numpy(f).cuda()).ranges()
    assert np.array_equal(got, ref)


def test_skip_flags_bit_exact():
    from paper_2504_18001_gb300 import cinr
    rng = np.random.default_rng(4)
    lo = rng.uniform(-0.1, 1.0, 20000)
    ranges = np.stack([lo, lo + rng.uniform(0, 0.2, lo.size) ** 2], 1).astype(np.float32)
    # the flags are taken per cell: any 3-d shape with 20000 cells
    m = cinr.Macro((20 * 16, 25 * 16, 40 * 16), 16, ranges=ranges)
    for tf in (S.tf_ramps(2), _gated_tf(0.5), S.tf_constant((1, 1, 1), 3.0), np.zeros((256, 4), np.float32)):
        m.apply_tf(tf)
        assert np.array_equal(m.skip_flags(), O.macro_skip(ranges, tf.astype(np.float64)))


def test_cached_frames_with_macro_cells_match_oracle():
    # the median cell maximum of the oracle's ranges gates the TF
    cfg, table, w, inr, p = _scene64()
    theta = float(np.median(O.macro_ranges_inr(p, table, w, (64, 64, 64), 8, 3)[:, 1]))
    cache, oc, hist, worst = _run(4, tf=_gated_tf(theta), macro_cell=8, slots=80)
    assert all(h["samples_skipped"] > 0 for h in hist)


@pytest.mark.parametrize("layout,graph", [(1, 0), (0, 1)])
def test_cached_macro_cells_other_layout_and_graph(layout, graph):
    cfg, table, w, inr, p = _scene64()
    theta = float(np.median(O.macro_ranges_inr(p, table, w, (64, 64, 64), 16, 3)[:, 1]))
    _run(3, tf=_gated_tf(theta), macro_cell=16, slots=80, ray_layout=layout, use_graph=graph)


@pytest.mark.parametrize("prec", ["fp32", "mixed"])
def test_skipping_leaves_first_cached_frame_identical(prec):
    # GPU-built ranges (the cache's own decode arithmetic and storage) bound
    # every cached sample: a fresh cache renders frame 1 bit-identically with
    # and without skipping
    from paper_2504_18001_gb300 import cinr
    vol = (64, 64, 64)
    mlp, tab, sto = ("fp32", "fp32", "fp32") if prec == "fp32" else ("bf16", "fp16", "fp16")
    cfg, table, w, inr, p = _scene64(vol, mlp=mlp, tab=tab)
    imgs, sts = [], []
    tf = None
    for use in (0, 1):
        cache = cinr.Cache(inr, vol, pool_bytes=100 * 1000 * 4, brick=8, levels=3, n_req=8,
                           storage=sto)
        m = cinr.Macro(vol, 8, inr=inr, cache=cache)
        if tf is None:
            tf = _gated_tf(float(np.median(m.ranges()[:, 1])))
        r = cinr.Renderer(96, 80, vol, K=32, eps_T=1e-3)
        if use:
            r.set_macro(m)
        img, st = r.render(inr, S.orbit_camera(3, 96, 80, distance=1.7), tf, cache=cache)
        imgs.append(img.cpu().numpy())
        sts.append(st)
    assert sts[1]["samples_skipped"] > 0
    assert sts[0]["samples"] == sts[1]["samples"] + sts[1]["samples_skipped"]
    assert np.array_equal(imgs[0], imgs[1])


def test_uncached_render_with_macro_cells_matches_oracle():
    from paper_2504_18001_gb300 import cinr
    vol = (64, 64, 64)
    cfg, table, w, inr, p = _scene64(vol)
    ranges = O.macro_ranges_inr(p, table, w, vol, 8, 1)
    tf = _gated_tf(float(np.median(ranges[:, 1])))
    m = cinr.Macro(vol, 8, ranges=ranges)
    r = cinr.Renderer(64, 48, vol, K=32, eps_T=0.0)
    r.set_macro(m)
    cam = S.orbit_camera(5, 64, 48)
    img, st = r.render(inr, cam, tf)
    om = O.macro(vol, 8, O.macro_skip(ranges, tf.astype(np.float64)))
    ref, rst = O.render_direct(p, table, w, ocam(cam), vol, O.march_opts(K=32, eps_T=0.0, macro=om),
                               tf.astype(np.float64))
    assert st["samples"] == rst["samples"] and st["samples_skipped"] == rst["samples_skipped"] > 0
    assert np.abs(img.cpu().numpy() - ref).max() < 2e-3


def test_field_render_with_macro_cells_identical_and_matches_oracle():
    import torch
    from paper_2504_18001_gb300 import cinr
    dims = (48, 40, 32)
    f = S.explicit_field(dims, S.field_params(seed=0))
    ft = torch.from_numpy(f).cuda()
    tf = _gated_tf(0.55)
    r = cinr.Renderer(64, 48, dims, K=32, eps_T=1e-3)
    cam = S.orbit_camera(7, 64, 48)
    img0, st0 = r.render_field(ft, cam, tf)
    img0 = img0.clone()
    m = cinr.Macro(dims, 8, field=ft)
    r.set_macro(m)
    img1, st1 = r.render_field(ft, cam, tf)
    assert st1["samples_skipped"] > 0
    assert st1["samples"] + st1["samples_skipped"] == st0["samples"]
    assert torch.equal(img0, img1)
    om = O.macro(dims, 8, O.macro_skip(O.macro_ranges_field(f, 8), tf.astype(np.float64)))
    ref, rst = O.render_field(f, ocam(cam), dims, O.march_opts(K=32, eps_T=1e-3, macro=om),
                              tf.astype(np.float64))
    assert rst["samples_skipped"] == st1["samples_skipped"]
    assert np.abs(img1.cpu().numpy() - ref).max() < 2e-3


@pytest.mark.parametrize("eps", [0.0, 1e-2])
def test_cached_macro_cells_with_lod_scaled_steps(eps):
    # the jump over a transparent cell stays inside the 32-sample segment and
    # the termination boundary: counts and state stay bit-exact
    cfg, table, w, inr, p = _scene64()
    theta = float(np.median(O.macro_ranges_inr(p, table, w, (64, 64, 64), 8, 3)[:, 1]))
    cache, oc, hist, worst = _run(3, tf=_gated_tf(theta), macro_cell=8, slots=80, step_mode=1,
                                  step_lod_max=2, lod_mode=1, lod_scale=12.0, eps=eps)
    assert all(h["samples_skipped"] > 0 for h in hist)
