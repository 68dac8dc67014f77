"""GPU parity of the hash-grid encoder and INR inference (through the C ABI)
against the CPU FP64 oracle."""
import numpy as np
import pytest

import oracle as O
from paper_2504_18001_gb300 import synthetic as S

from _scenes import gpu_inr, oracle_inr, oracle_params, scene

pytestmark = pytest.mark.gpu

CFGS = [S.INR_64, S.INR_512, S.INR_TERA]


def _points(cfg, n, seed):
    pts = [S.random_points(n, seed)]
    res = O.level_res(oracle_params(cfg))
    for l, N in enumerate(res[:: max(1, len(res) // 4)]):
        pts.append(S.grid_aligned_points(int(N), 500, seed + l))
    return np.concatenate(pts).astype(np.float32)


@pytest.mark.parametrize("cfg", CFGS, ids=["L8", "L16", "L24"])
def test_hash_indices_bit_exact(cfg):
    """Vertex indices of every level and corner, GPU against the oracle, bit
    for bit: 10^6 random points (a ragged count) plus, at every level, points
    on that level's grid lines (x = k / N_l exactly, where the floor and the
    upper clamp decide the cell)."""
    import torch
    table, w = scene(cfg)
    inr = gpu_inr(cfg, table, w)
    res = O.level_res(oracle_params(cfg))
    pts = [S.random_points(1_000_003, 5)]
    for l, N in enumerate(res):
        pts.append(S.grid_aligned_points(int(N), 2000, 100 + l))
    pts = np.concatenate(pts).astype(np.float32)
    x = torch.from_numpy(pts).cuda()
    feats, idx = inr.encode(x, with_indices=True)
    ref = O.encode_indices(oracle_params(cfg), pts)
    assert np.array_equal(idx.cpu().numpy().astype(np.uint32), ref)


@pytest.mark.parametrize("cfg", CFGS[:2], ids=["L8", "L16"])
def test_encode_features(cfg):
    import torch
    table, w = scene(cfg)
    inr = gpu_inr(cfg, table, w)
    pts = _points(cfg, 3001, seed=6)
    feats, _ = inr.encode(torch.from_numpy(pts).cuda())
    ref = O.encode(oracle_params(cfg), table, pts)
    assert np.abs(feats.cpu().numpy() - ref).max() < 1e-5


@pytest.mark.parametrize("cfg", CFGS, ids=["L8", "L16", "L24"])
def test_infer_normalised_field_within_1e4(cfg):
    import torch
    vol = (64, 64, 64)
    table, w = scene(cfg)
    inr = gpu_inr(cfg, table, w, vol=vol)
    p = oracle_inr(cfg, table, w, vol=vol)
    pts = _points(cfg, 4099, seed=7)  # ragged: not a multiple of the block
    v = inr.infer(torch.from_numpy(pts).cuda()).cpu().numpy()
    ref = O.inr_eval(p, table, w, pts)
    assert np.abs(v - ref).max() < 1e-4


def test_raw_range_matches_oracle():
    cfg = S.INR_64
    table, w = scene(cfg)
    inr = gpu_inr(cfg, table, w)
    lo, hi = inr.raw_range((64, 64, 64), stride=4)
    olo, ohi = O.inr_raw_range(oracle_params(cfg), table, w, (64, 64, 64), 4)
    assert abs(lo - olo) < 1e-5 * (ohi - olo) and abs(hi - ohi) < 1e-5 * (ohi - olo)


def test_infer_edge_sizes():
    import torch
    cfg = S.INR_64
    table, w = scene(cfg)
    inr = gpu_inr(cfg, table, w)
    out = torch.full((4,), -7.0, device="cuda")
    inr.infer(torch.zeros((0, 3), device="cuda"), out=out)  # n = 0: no-op
    assert (out.cpu() == -7.0).all()
    one = inr.infer(torch.tensor([[0.3, 0.6, 0.9]], device="cuda")).cpu().numpy()
    ref = O.inr_eval(oracle_params(cfg), table, w, np.array([[0.3, 0.6, 0.9]], np.float32))
    assert abs(one[0] - ref[0]) < 1e-5
    # large ragged batch, sampled check
    n = 1_000_003
    pts = S.random_points(n, 9, include_edges=False)
    v = inr.infer(torch.from_numpy(pts).cuda()).cpu().numpy()
    sel = np.random.default_rng(0).choice(n, 2000, replace=False)
    assert np.abs(v[sel] - O.inr_eval(oracle_params(cfg), table, w, pts[sel])).max() < 1e-5


def test_fp16_table_error_stated():
    import torch
    cfg = S.INR_64
    vol = (64, 64, 64)
    table, w = scene(cfg)
    inr = gpu_inr(cfg, table, w, vol=vol, tab="fp16")
    p = oracle_inr(cfg, table, w, vol=vol)
    pts = S.random_points(5000, 3)
    v = inr.infer(torch.from_numpy(pts).cuda()).cpu().numpy()
    err = np.abs(v - O.inr_eval(p, table, w, pts)).max()
    # half-precision table entries of magnitude <= 0.5: relative rounding 2^-11
    assert err < 5e-3, err
