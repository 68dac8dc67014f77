"""Seeded synthetic inputs shared by the CUDA path's tests/bench and the oracle.

This module draws random inputs only: INR parameters at initialisation,
transfer-function ramps, camera paths and the parameters of the synthetic
scalar fields that stand in for the paper's datasets (which are not
available).  It holds none of the method's arithmetic (no hash encoding, no
MLP, no marching, no cache logic).  ``field_values`` evaluates the synthetic
field itself (the data being compressed), not the renderer.

Workload recipes (sizes from the paper's regime, Sec. 6):
  * uncached 64^3 scene: 32 anisotropic Gaussians, INR L=8, F=2, T=2^14,
    N_min=4, b=1.5, MLP 16-32-32-1, 128x128, 45 deg, distance 2.0, 0.5 voxel
    step, 4 seeded TF ramps;
  * cached 512^3 orbit: Gaussians + 3-octave value noise, INR L=16, F=2,
    T=2^19, N_min=16, b=1.38, MLP 32-64-64-1, brick 8 (+1 apron), 4 LoDs,
    1 GiB FP32 pool, 1024x1024, 1 deg/frame orbit then TF edits;
  * tera-scale virtual grid 10240x7680x1536, INR L=24, T=2^22, MLP 48-64-64-1,
    brick 16, 6 LoDs, 40 GB FP16 pool, 1920x1080 fly-through;
  * learned INR on an explicit 1024^3 field (batch 2^18, Adam, lr 1e-2).
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field as dc_field

import numpy as np


# ------------------------------------------------------------------ configs
@dataclass(frozen=True)
class InrConfig:
    levels: int
    feats: int
    log2_table: int
    base_res: int
    growth: float
    hidden: int
    n_hidden_layers: int = 2

    @property
    def in_dim(self) -> int:
        return self.levels * self.feats

    @property
    def table_entries(self) -> int:
        return self.levels * (1 << self.log2_table) * self.feats

    @property
    def mlp_params(self) -> int:
        h = self.hidden
        return h * self.in_dim + (self.n_hidden_layers - 1) * h * h + h


@dataclass(frozen=True)
class SceneConfig:
    name: str
    vol: tuple
    inr: InrConfig
    width: int
    height: int
    fov_y_deg: float = 45.0
    distance: float = 2.0
    step_voxels: float = 0.5
    n_gaussians: int = 32
    noise_octaves: int = 0
    noise_f0: int = 8
    brick: int = 8
    levels: int = 4
    pool_bytes: int = 1 << 30
    n_req: int = 40
    K: int = 32
    eps_T: float = 1e-3
    lod_scale: float = 1.0
    extra: dict = dc_field(default_factory=dict)


INR_64 = InrConfig(levels=8, feats=2, log2_table=14, base_res=4, growth=1.5, hidden=32)
INR_512 = InrConfig(levels=16, feats=2, log2_table=19, base_res=16, growth=1.38, hidden=64)
INR_TERA = InrConfig(levels=24, feats=2, log2_table=22, base_res=16, growth=1.38, hidden=64)
INR_LEARNED = InrConfig(levels=16, feats=2, log2_table=20, base_res=16, growth=1.38, hidden=64)

UNCACHED_64 = SceneConfig(name="uncached_fp32_64cube_128px", vol=(64, 64, 64), inr=INR_64,
                          width=128, height=128, brick=8, levels=4, pool_bytes=64 << 20)
CACHED_512 = SceneConfig(name="cached_fp32_512cube_1024px_orbit", vol=(512, 512, 512),
                         inr=INR_512, width=1024, height=1024, noise_octaves=3, noise_f0=8,
                         brick=8, levels=4, pool_bytes=1 << 30)
TERA = SceneConfig(name="terascale_10240x7680x1536_1080p", vol=(10240, 7680, 1536),
                   inr=INR_TERA, width=1920, height=1080, n_gaussians=512, noise_octaves=4,
                   noise_f0=16, brick=16, levels=6, pool_bytes=40 << 30)


# ------------------------------------------------------------- INR weights
def inr_init(cfg: InrConfig, seed: int, table_scale: float = 1e-4, level_decay: float = 1.0):
    """Initial parameters: table U(-s d^l, s d^l) for level l (L*T*F,
    level-major, feature-minor); MLP weights He-normal N(0, 2/fan_in),
    layer-major, each [out][in].  level_decay d < 1 gives a band-limited
    field whose energy sits in the coarse levels, the spectrum a network
    trained on a smooth scientific field ends up with."""
    rng = np.random.default_rng(np.random.PCG64(seed))
    table = rng.uniform(-table_scale, table_scale, cfg.table_entries).astype(np.float32)
    if level_decay != 1.0:
        per = (1 << cfg.log2_table) * cfg.feats
        scale = np.repeat(np.float32(level_decay) ** np.arange(cfg.levels, dtype=np.float32), per)
        table = (table * scale).astype(np.float32)
    ws = []
    fan = cfg.in_dim
    for _ in range(cfg.n_hidden_layers):
        ws.append(rng.normal(0.0, math.sqrt(2.0 / fan), (cfg.hidden, fan)).astype(np.float32))
        fan = cfg.hidden
    ws.append(rng.normal(0.0, math.sqrt(2.0 / fan), (1, fan)).astype(np.float32))
    w = np.concatenate([a.ravel() for a in ws]).astype(np.float32)
    assert w.size == cfg.mlp_params
    return table, w


# --------------------------------------------------------- transfer function
def tf_ramps(seed: int, n_ramps: int = 4, shift: float = 0.0) -> np.ndarray:
    """256 x (r, g, b, sigma): tent ramps with centre U(0.1, 0.9), half-width
    U(0.02, 0.1), peak extinction U(20, 100) per world unit, colour U[0,1)^3;
    extinctions add, colours add and clamp to [0, 1].  `shift` moves every
    centre (the TF-edit frames)."""
    rng = np.random.default_rng(np.random.PCG64(seed))
    x = np.arange(256, dtype=np.float64) / 255.0
    out = np.zeros((256, 4), np.float64)
    for _ in range(n_ramps):
        c = rng.uniform(0.1, 0.9) + shift
        hw = rng.uniform(0.02, 0.1)
        peak = rng.uniform(20.0, 100.0)
        rgb = rng.uniform(0.0, 1.0, 3)
        tent = np.clip(1.0 - np.abs(x - c) / hw, 0.0, None)
        out[:, :3] += tent[:, None] * rgb[None, :]
        out[:, 3] += tent * peak
    out[:, :3] = np.clip(out[:, :3], 0.0, 1.0)
    return out.astype(np.float32)


def tf_constant(rgb, sigma) -> np.ndarray:
    out = np.zeros((256, 4), np.float32)
    out[:, :3] = np.asarray(rgb, np.float32)
    out[:, 3] = sigma
    return out


# ------------------------------------------------------------------ camera
def orbit_camera(frame: int, width: int, height: int, distance: float = 2.0,
                 deg_per_frame: float = 1.0, start_deg: float = 30.0,
                 elevation: float = 0.35, fov_y_deg: float = 45.0, step_voxels: float = 0.5):
    """Eye on a circle about +y through the volume centre, 1 deg per frame."""
    th = math.radians(start_deg + deg_per_frame * frame)
    r = math.sqrt(max(distance * distance - elevation * elevation, 0.0))
    eye = (r * math.sin(th), elevation, r * math.cos(th))
    return dict(eye=eye, target=(0.0, 0.0, 0.0), up=(0.0, 1.0, 0.0), fov_y_deg=fov_y_deg,
                width=width, height=height, step_voxels=step_voxels)


def flythrough_camera(frame: int, n_frames: int, width: int, height: int, seed: int = 0,
                      d_start: float = 2.0, d_end: float = 0.3, fov_y_deg: float = 45.0,
                      step_voxels: float = 0.5):
    """Seeded fly-through: orbit that zooms from d_start to d_end and back
    with a slowly drifting target."""
    rng = np.random.default_rng(np.random.PCG64(seed))
    tgt_amp = rng.uniform(-0.15, 0.15, 3)
    ph = frame / max(n_frames - 1, 1)
    zoom = 0.5 - 0.5 * math.cos(2.0 * math.pi * ph)
    dist = d_start + (d_end - d_start) * zoom
    th = math.radians(20.0 + 90.0 * ph)
    tgt = tuple(float(a * math.sin(math.pi * ph)) for a in tgt_amp)
    eye = (tgt[0] + dist * math.sin(th), tgt[1] + 0.25 * dist, tgt[2] + dist * math.cos(th))
    return dict(eye=eye, target=tgt, up=(0.0, 1.0, 0.0), fov_y_deg=fov_y_deg, width=width,
                height=height, step_voxels=step_voxels)


# ----------------------------------------------------------- synthetic field
def field_params(seed: int, n_gaussians: int = 32, noise_octaves: int = 0, noise_f0: int = 8,
                 min_width: float = 1.0 / 64.0):
    """Gaussian centres U[0,1)^3 and widths U(0,1)^3 clamped at min_width;
    value-noise lattices U[0,1) at frequency f0*2^o for each octave."""
    rng = np.random.default_rng(np.random.PCG64(seed))
    centres = rng.uniform(0.0, 1.0, (n_gaussians, 3))
    widths = np.maximum(rng.uniform(0.0, 1.0, (n_gaussians, 3)), min_width)
    lattices = []
    for o in range(noise_octaves):
        f = noise_f0 * (1 << o)
        lattices.append(rng.uniform(0.0, 1.0, (f + 1, f + 1, f + 1)))
    return dict(centres=centres, widths=widths, lattices=lattices)


def field_values(points, params, torch_device=None):
    """Raw synthetic field at points [n,3] in [0,1]^3: the sum of unit
    Gaussians exp(-|(x-c)/s|^2 / 2) plus value noise (trilinear lattice
    interpolation, amplitude 2^-o).  Uses torch when a device is given."""
    if torch_device is not None:
        import torch
        p = torch.as_tensor(points, dtype=torch.float64, device=torch_device)
        c = torch.as_tensor(params["centres"], dtype=torch.float64, device=torch_device)
        s = torch.as_tensor(params["widths"], dtype=torch.float64, device=torch_device)
        out = torch.zeros(p.shape[0], dtype=torch.float64, device=torch_device)
        for i in range(c.shape[0]):
            z = (p - c[i]) / s[i]
            out += torch.exp(-0.5 * (z * z).sum(dim=1))
        for o, lat in enumerate(params["lattices"]):
            lt = torch.as_tensor(lat, dtype=torch.float64, device=torch_device)
            f = lt.shape[0] - 1
            q = p * f
            i0 = torch.clamp(torch.floor(q), 0, f - 1).long()
            fr = q - i0
            acc = torch.zeros_like(out)
            for cidx in range(8):
                b = [(cidx >> a) & 1 for a in range(3)]
                wgt = torch.ones_like(out)
                for a in range(3):
                    wgt = wgt * (fr[:, a] if b[a] else 1.0 - fr[:, a])
                acc += wgt * lt[i0[:, 0] + b[0], i0[:, 1] + b[1], i0[:, 2] + b[2]]
            out += acc * (0.5 ** o)
        return out
    p = np.asarray(points, np.float64)
    out = np.zeros(p.shape[0])
    for c, s in zip(params["centres"], params["widths"]):
        z = (p - c) / s
        out += np.exp(-0.5 * (z * z).sum(axis=1))
    for o, lat in enumerate(params["lattices"]):
        f = lat.shape[0] - 1
        q = p * f
        i0 = np.clip(np.floor(q), 0, f - 1).astype(np.int64)
        fr = q - i0
        acc = np.zeros_like(out)
        for cidx in range(8):
            b = [(cidx >> a) & 1 for a in range(3)]
            wgt = np.ones_like(out)
            for a in range(3):
                wgt = wgt * (fr[:, a] if b[a] else 1.0 - fr[:, a])
            acc += wgt * lat[i0[:, 0] + b[0], i0[:, 1] + b[1], i0[:, 2] + b[2]]
        out += acc * (0.5 ** o)
    return out


def explicit_field(dims, params, torch_device=None, chunk: int = 1 << 22):
    """Field at voxel centres (i+0.5)/V, normalised to [0,1] by its min/max.
    Returns float32 [z, y, x] (numpy, or torch on torch_device)."""
    nx, ny, nz = dims
    n = nx * ny * nz
    if torch_device is not None:
        import torch
        out = torch.empty(n, dtype=torch.float32, device=torch_device)
        for s in range(0, n, chunk):
            idx = torch.arange(s, min(n, s + chunk), device=torch_device, dtype=torch.int64)
            pts = torch.stack([(idx % nx).double(), ((idx // nx) % ny).double(),
                               (idx // (nx * ny)).double()], dim=1)
            pts = (pts + 0.5) / torch.tensor([nx, ny, nz], dtype=torch.float64,
                                             device=torch_device)
            out[s:s + idx.numel()] = field_values(pts, params, torch_device).float()
        lo, hi = out.min(), out.max()
        out = (out - lo) / (hi - lo)
        return out.view(nz, ny, nx)
    zz, yy, xx = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    pts = np.stack([(xx.ravel() + 0.5) / nx, (yy.ravel() + 0.5) / ny, (zz.ravel() + 0.5) / nz], 1)
    v = field_values(pts, params)
    v = (v - v.min()) / (v.max() - v.min())
    return v.astype(np.float32).reshape(nz, ny, nx)


def random_points(n: int, seed: int, include_edges: bool = True) -> np.ndarray:
    """Uniform points in [0,1)^3 plus (optionally) the corners and faces of
    the unit cube, for encoder parity tests."""
    rng = np.random.default_rng(np.random.PCG64(seed))
    pts = rng.uniform(0.0, 1.0, (n, 3)).astype(np.float32)
    if include_edges:
        edge = np.array([[0, 0, 0], [1, 1, 1], [1, 0, 0], [0, 1, 0], [0, 0, 1], [0.5, 1, 0],
                         [1, 0.5, 1], [0.999999, 0.999999, 0.999999]], np.float32)
        pts = np.concatenate([pts, edge])
    return pts


def grid_aligned_points(res: int, n: int, seed: int) -> np.ndarray:
    """Points exactly on level-grid vertices x = k / res."""
    rng = np.random.default_rng(np.random.PCG64(seed))
    k = rng.integers(0, res + 1, (n, 3))
    return (k.astype(np.float32) / np.float32(res)).astype(np.float32)
