"""FP16 bricks in the texture layout (CINR_PREC_FP16_TEX): the specialised
marching kernel samples them with the texture units.

The layout changes where voxels sit and how a sample is filtered, nothing
else: the discrete cache state (page tables, stamps, owners, ranks, request
and victim lists) and the frame counts equal the oracle's frame by frame,
the pool read back in slot order equals the linear FP16 layout's pool bit
for bit, and the pixels stay within 4e-2 of the FP64 oracle (the linear
FP16 layout: 2e-2; the hardware's bilinear weights carry 8 fractional
bits) and above 40 dB against the linear layout's.  Other kernels reject such a cache.
"""
import numpy as np
import pytest

import oracle as O
from paper_2504_18001_gb300 import synthetic as S

from _scenes import gpu_inr, ocam, oracle_inr, scene

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("brick", [8, 16])
def test_texture_layout_state_pool_and_pixels(brick):
    from paper_2504_18001_gb300 import cinr
    vol, W, H, levels, n_req = (64, 64, 64), 64, 48, 3, 40
    cfg = S.INR_64
    table, w = scene(cfg)
    inr = gpu_inr(cfg, table, w, vol=vol)
    p = oracle_inr(cfg, table, w, vol=vol)
    S3 = (brick + 2) ** 3
    # two block rows of the texture layout; the linear cache and the oracle
    # take the slot count the texture layout gives
    tex = cinr.Cache(inr, vol, pool_bytes=2 << 20, brick=brick, levels=levels, n_req=n_req,
                     storage="fp16tex")
    lin = cinr.Cache(inr, vol, pool_bytes=tex.n_slots * S3 * 2, brick=brick, levels=levels,
                     n_req=n_req, storage="fp16")
    assert lin.n_slots == tex.n_slots > 40
    mo = O.march_opts(K=32, eps_T=0.0, seed=11)
    oc = O.Cache(p, table, w, vol, brick, levels, tex.n_slots, mo, n_req=n_req)
    rt = cinr.Renderer(W, H, vol, K=32, eps_T=0.0, seed=11)
    rl = cinr.Renderer(W, H, vol, K=32, eps_T=0.0, seed=11)
    tf = S.tf_ramps(2)
    for f in range(4):
        cam = S.orbit_camera(4 * f, W, H, distance=1.6 + 0.05 * f)
        img_t, st_t = rt.render(inr, cam, tf, cache=tex)
        img_l, st_l = rl.render(inr, cam, tf, cache=lin)
        ref, st_o = oc.render(ocam(cam), tf.astype(np.float64))
        for k in ("samples", "hits", "fallback_hits", "true_misses", "bricks_requested",
                  "bricks_decoded", "evictions", "inr_queries_decode"):
            assert st_t[k] == st_o[k] == st_l[k], (f, k, st_t[k], st_o[k], st_l[k])
        for g, o in ((cinr.DUMP_PAGE_TABLE, O.DUMP_PT), (cinr.DUMP_STAMPS, O.DUMP_STAMP),
                     (cinr.DUMP_OWNERS, O.DUMP_OWNER), (cinr.DUMP_RANK, O.DUMP_RANK),
                     (cinr.DUMP_REQUESTS, O.DUMP_REQ), (cinr.DUMP_VICTIMS, O.DUMP_VICT)):
            assert np.array_equal(tex.dump(g), oc.dump(o)), (f, g)
        # the slots that hold a brick (a slot never written holds whatever the
        # caller's buffer held)
        own = tex.dump(cinr.DUMP_OWNERS)
        assert np.array_equal(own, lin.dump(cinr.DUMP_OWNERS)), f
        used = np.nonzero(own != 0xFFFFFFFF)[0]
        pt_, pl_ = (c.dump(cinr.DUMP_POOL).reshape(tex.n_slots, -1) for c in (tex, lin))
        assert len(used) > 0 and np.array_equal(pt_[used], pl_[used]), f
        # the linear FP16 layout is within 2e-2 of the oracle per channel; the
        # hardware's 8-bit bilinear weights add up to 2^-9 of a neighbour
        # difference per axis (measured: 0.027 at worst with 8^3 bricks)
        a, b = img_t.cpu().numpy(), img_l.cpu().numpy()
        assert np.abs(a - ref).max() < 4e-2, (f, np.abs(a - ref).max())
        assert O.psnr(a.astype(np.float64), b.astype(np.float64)) > 40.0


def test_texture_layout_is_rejected_outside_the_specialised_kernel():
    from paper_2504_18001_gb300 import cinr
    vol = (64, 64, 64)
    cfg = S.INR_64
    table, w = scene(cfg)
    inr = gpu_inr(cfg, table, w, vol=vol)
    cache = cinr.Cache(inr, vol, pool_bytes=2 << 20, brick=8, levels=3, n_req=40, storage="fp16tex")
    cam, tf = S.orbit_camera(0, 32, 32), S.tf_ramps(2)
    for r in (cinr.Renderer(32, 32, vol, lod_mode=1, lod_scale=1.0),     # distance LoD
              cinr.Renderer(32, 32, vol, ray_layout=1)):                 # warp per ray
        with pytest.raises(cinr.CinrError) as ei:
            r.render(inr, cam, tf, cache=cache)
        assert ei.value.code == cinr.ERR_UNSUPPORTED
    # the same cache still renders with the specialised kernel
    cinr.Renderer(32, 32, vol).render(inr, cam, tf, cache=cache)
