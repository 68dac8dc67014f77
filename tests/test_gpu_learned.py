"""The learned part (Sec. 4.1): an INR trained from scratch on the GPU by the
library's own kernels, rendered through the FP16 brick cache, judged by
PSNR against an explicit-voxel render of the same field."""
import numpy as np
import pytest

import oracle as O
from paper_2504_18001_gb300 import synthetic as S

from _scenes import ocam, scene

pytestmark = pytest.mark.gpu


def _psnr(a, b):
    return O.psnr(np.asarray(a, np.float64), np.asarray(b, np.float64))


def test_field_render_matches_oracle():
    import torch
    from paper_2504_18001_gb300 import cinr
    field = S.explicit_field((24, 40, 32), S.field_params(3, n_gaussians=10, noise_octaves=2))
    vol = (48, 40, 56)
    cam = S.orbit_camera(7, 48, 40)
    tf = S.tf_ramps(2)
    r = cinr.Renderer(48, 40, vol, K=32, eps_T=0.0)
    img, st = r.render_field(torch.from_numpy(field).cuda(), cam, tf)
    ref, rst = O.render_field(field, ocam(cam), vol, O.march_opts(K=32, eps_T=0.0),
                              tf.astype(np.float64))
    assert st["samples"] == rst["samples"]
    assert np.abs(img.cpu().numpy() - ref).max() < 2e-3


def test_trained_inr_cached_fp16_render_gains_over_untrained():
    import torch
    from paper_2504_18001_gb300 import cinr
    cfg = S.INR_64
    dims = (64, 64, 64)
    field = S.explicit_field(dims, S.field_params(0, n_gaussians=32, noise_octaves=2, noise_f0=4))
    f_dev = torch.from_numpy(field).cuda()
    table, w = S.inr_init(cfg, seed=1, table_scale=1e-4)
    inr = cinr.Inr(cinr.make_inr_params(cfg), table, w)
    tr = cinr.Trainer(inr, batch=1 << 16, seed=3)
    for _ in range(400):
        tr.step(f_dev)
    t_tab, t_w = cinr.inr_export(inr)
    W = H = 96
    tf = S.tf_ramps(2)
    cam = S.orbit_camera(20, W, H)
    r = cinr.Renderer(W, H, dims, K=32, eps_T=1e-3, lod_scale=1.0)
    ref, _ = r.render_field(f_dev, cam, tf)
    ref = ref.cpu().numpy()

    def cached(tab, wts, frames=6):
        m = cinr.Inr(cinr.make_inr_params(cfg, mlp_precision="bf16", table_precision="fp16"), tab, wts)
        cache = cinr.Cache(m, dims, pool_bytes=600 * 1000 * 2, brick=8, levels=3, n_req=512,
                           storage="fp16")
        img = None
        for _ in range(frames):  # fill the cache, then judge the last frame
            img, st = r.render(m, cam, tf, cache=cache)
        return img.cpu().numpy()

    trained = _psnr(cached(t_tab, t_w), ref)
    untrained = _psnr(cached(table, w), ref)
    assert trained > 30.0, trained
    assert trained > untrained + 10.0, (trained, untrained)
