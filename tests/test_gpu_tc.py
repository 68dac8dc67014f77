"""Tensor-core (tcgen05) MLP: the shared-memory operand layout through a
single-tile GEMM self-test, and FP16/BF16 INR inference against the FP64
oracle (error stated per precision)."""
import ctypes as C

import numpy as np
import pytest

import oracle as O
from paper_2504_18001_gb300 import synthetic as S

from _scenes import gpu_inr, oracle_inr, scene

pytestmark = pytest.mark.gpu


def _round(x, bf16):
    import torch
    t = torch.from_numpy(x)
    return (t.to(torch.bfloat16) if bf16 else t.to(torch.float16)).float().numpy().astype(np.float64)


@pytest.mark.parametrize("K", [16, 32, 64])
@pytest.mark.parametrize("bf16", [0, 1], ids=["fp16", "bf16"])
def test_mma_tile_matches_reference_gemm(K, bf16):
    import torch
    from paper_2504_18001_gb300 import cinr
    rng = np.random.default_rng(K + 10 * bf16)
    A = rng.normal(size=(128, K)).astype(np.float32)
    B = rng.normal(size=(64, K)).astype(np.float32)
    # distinct row/column signatures catch permuted or transposed operands
    A[:, 0] += np.arange(128, dtype=np.float32) / 16
    B[:, 1] += np.arange(64, dtype=np.float32) / 8
    a, b = torch.from_numpy(A).cuda(), torch.from_numpy(B).cuda()
    d = torch.full((128, 64), float("nan"), device="cuda")
    cinr.check(cinr.lib().cinr_debug_mma_tile(C.c_void_p(a.data_ptr()), C.c_void_p(b.data_ptr()), K,
                                              bf16, C.c_void_p(d.data_ptr()), cinr._stream(None)),
               "cinr_debug_mma_tile")
    ref = _round(A, bf16) @ _round(B, bf16).T
    got = d.cpu().numpy()
    assert np.isfinite(got).all()
    assert np.abs(got - ref).max() <= 1e-4 * np.abs(ref).max() + 1e-4


@pytest.mark.parametrize("prec", ["fp16", "bf16", "fp8"])
@pytest.mark.parametrize("cfg", [S.INR_64, S.INR_512, S.INR_TERA], ids=["L8", "L16", "L24"])
def test_tensor_core_inference_error(prec, cfg):
    import torch
    from paper_2504_18001_gb300 import cinr
    vol = (64, 64, 64)
    table, w = scene(cfg, seed=4, table_scale=0.5)
    inr32 = gpu_inr(cfg, table, w, vol=vol)
    inr = gpu_inr(cfg, table, w, vol=vol, mlp=prec)
    p = oracle_inr(cfg, table, w, vol=vol)
    pts = S.random_points(10007, 21)  # ragged: not a multiple of the 128-query tile
    x = torch.from_numpy(pts).cuda()
    v = inr.infer(x).cpu().numpy()
    v32 = inr32.infer(x).cpu().numpy()
    cinr.check(cinr.lib().cinr_inr_status(inr.h, cinr._stream(None)), "cinr_inr_status")
    ref = O.inr_eval(p, table, w, pts)
    err = np.abs(v - ref).max()
    # stated error on the [0,1]-normalised field: FP32 path 1e-4; FP16 MLP
    # 1e-2; BF16 MLP (8-bit mantissa) 5e-2; FP8 E4M3 trial (4-bit mantissa,
    # no scaling) 0.3 max, 0.05 mean
    bound = {"fp16": (1e-2, 2e-3), "bf16": (5e-2, 1e-2), "fp8": (0.3, 0.05)}[prec]
    assert np.abs(v32 - ref).max() < 1e-4
    assert err < bound[0], err
    assert np.mean(np.abs(v - ref)) < bound[1]


@pytest.mark.parametrize("prec", ["fp16", "bf16"])
def test_uncached_render_tensor_core_mlp(prec):
    from paper_2504_18001_gb300 import cinr
    from _scenes import ocam
    vol = (64, 64, 64)
    cfg = S.INR_64
    table, w = scene(cfg)
    inr = gpu_inr(cfg, table, w, vol=vol, mlp=prec)
    p = oracle_inr(cfg, table, w, vol=vol)
    cam = S.orbit_camera(5, 64, 48)
    tf = S.tf_ramps(2)
    r = cinr.Renderer(64, 48, vol, K=32, eps_T=0.0)
    img, st = r.render(inr, cam, tf)
    ref, rst = O.render_direct(p, table, w, ocam(cam), vol, O.march_opts(K=32, eps_T=0.0),
                               tf.astype(np.float64))
    assert st["samples"] == rst["samples"]
    err = np.abs(img.cpu().numpy() - ref).max()
    assert err < (2e-2 if prec == "fp16" else 6e-2), err
    assert O.psnr(img.cpu().numpy().astype(np.float64), ref) > 40.0


def test_cached_mixed_precision_state_exact_and_psnr():
    # FP16 hash table, BF16 tensor-core MLP, FP16 bricks: discrete cache state
    # stays bit-exact (it depends on geometry only); pixels within the stated
    # error, PSNR >= 40 dB against the FP64 oracle image
    from test_gpu_cache import _run
    cache, oc, hist, worst = _run(4, storage="fp16", mlp="bf16", tab="fp16", check_pixels=None)
    assert worst < 6e-2, worst
    assert min(h["psnr"] for h in hist) > 40.0, [h["psnr"] for h in hist]
