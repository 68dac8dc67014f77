"""Matched GPU / oracle scenes for the parity tests.  Both sides receive the
same seeded inputs from paper_2504_18001_gb300.synthetic; each side computes
its own normalisation range with its own code."""
import numpy as np

import oracle as O
from paper_2504_18001_gb300 import synthetic as S


def oracle_params(cfg, ymin=None, ymax=None):
    p = O.inr_params(cfg.levels, cfg.feats, cfg.log2_table, cfg.base_res, cfg.growth, cfg.hidden)
    if ymin is not None:
        p.vmin = -ymin / (ymax - ymin)
        p.vmax = (1.0 - ymin) / (ymax - ymin)
    return p


def gpu_inr(cfg, table, w, vol=None, stride=4, mlp="fp32", tab="fp32"):
    from paper_2504_18001_gb300 import cinr
    inr = cinr.Inr(cinr.make_inr_params(cfg, mlp_precision=mlp, table_precision=tab), table, w)
    if vol is not None:
        lo, hi = inr.raw_range(vol, stride=stride)
        inr.set_range(-lo / (hi - lo), (1.0 - lo) / (hi - lo))
    return inr


def oracle_inr(cfg, table, w, vol=None, stride=4):
    p = oracle_params(cfg)
    if vol is not None:
        lo, hi = O.inr_raw_range(p, table, w, vol, stride)
        p.vmin = -lo / (hi - lo)
        p.vmax = (1.0 - lo) / (hi - lo)
    return p


def scene(cfg=S.INR_64, seed=1, table_scale=0.5):
    table, w = S.inr_init(cfg, seed=seed, table_scale=table_scale)
    return table, w


def ocam(d):
    return O.camera(d["eye"], d["target"], d["up"], d["fov_y_deg"], d["width"], d["height"],
                    d["step_voxels"])


def sorted_pairs(a):
    a = np.asarray(a, np.uint32).reshape(-1, 2)
    if len(a) == 0:
        return a
    order = np.lexsort((a[:, 1], a[:, 0]))
    return a[order]
