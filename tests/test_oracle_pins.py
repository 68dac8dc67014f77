"""Pins of the CPU FP64 oracle against facts that do not come from the oracle
itself: published generator outputs, hand computations, closed forms,
invariants, brute force on tiny inputs and the paper's worked example.
Each test names the mistake it would catch."""
import math

import numpy as np
import pytest

import oracle as O
from paper_2504_18001_gb300 import synthetic as S


# ------------------------------------------------------------ generators
def test_splitmix64_published_first_output():
    # First output of SplitMix64 started from state 0 (Steele et al. 2014;
    # the widely quoted value 0xE220A8397B1DCDAF).  Catches a wrong constant
    # or shift in the mixer.
    assert O.splitmix64(0) == 0xE220A8397B1DCDAF


def test_xorshift32_hand_computed():
    # s=1: s ^= s<<13 -> 8193; s ^= s>>17 -> 8193; s ^= s<<5 -> 8193^262176.
    assert O.xorshift32(1) == 8193 ^ 262176 == 270369
    # s=0x80000000: <<13 drops the bit; >>17 -> 0x80004000; <<5 -> 0x80084000 ^ ... by hand:
    s = 0x80000000
    s ^= (s << 13) & 0xFFFFFFFF  # 0x80000000
    s ^= s >> 17                 # 0x80004000
    s ^= (s << 5) & 0xFFFFFFFF   # 0x80004000 ^ 0x00080000 = 0x80084000
    assert s == 0x80084000
    assert O.xorshift32(0x80000000) == 0x80084000


def test_uniform_coords_grid_and_range():
    x = O.uniform_coords(seed=7, first=0, n=20000)
    assert x.min() >= 0.0 and x.max() < 1.0
    # values are multiples of 2^-24 (24-bit uniform)
    assert np.all((x.astype(np.float64) * 2**24) % 1 == 0)
    assert abs(x.mean() - 0.5) < 0.01
    # counter-based: element j of batch starting at `first` is element first+j
    y = O.uniform_coords(seed=7, first=100, n=10)
    assert np.array_equal(y, x[100:110])


# ------------------------------------------------------------ hash grid
def test_level_resolutions_hand_computed():
    # 4 * 1.5^l: 4, 6, 9, 13.5, 20.25, 30.375, 45.5625, 68.34375 -> floors
    p = O.inr_params(8, 2, 14, 4, 1.5, 32)
    assert O.level_res(p).tolist() == [4, 6, 9, 13, 20, 30, 45, 68]
    # dense iff (N+1)^3 <= 2^14: 125, 343, 1000, 2744, 9261 yes; 29791 no
    assert [O.level_is_dense(p, l) for l in range(8)] == [True] * 5 + [False] * 3


def test_dense_level_is_row_major_bijection():
    p = O.inr_params(1, 2, 10, 6, 2.0, 8)  # N=6: 343 vertices <= 1024
    n1 = 7
    seen = set()
    for iz in range(n1):
        for iy in range(n1):
            for ix in range(n1):
                idx = O.vertex_index(p, 0, ix, iy, iz)
                seen.add(idx)
    assert seen == set(range(n1 ** 3))
    assert O.vertex_index(p, 0, 1, 0, 0) == 1
    assert O.vertex_index(p, 0, 0, 1, 0) == n1
    assert O.vertex_index(p, 0, 0, 0, 1) == n1 * n1


def test_hash_level_brute_force_tiny_grid():
    # N=8 (729 vertices) in T=2^6: hashed.  Brute force with the published
    # Instant-NGP primes written out independently in Python big ints.
    p = O.inr_params(1, 2, 6, 8, 2.0, 8)
    assert not O.level_is_dense(p, 0)
    primes = (1, 2654435761, 805459861)
    counts = np.zeros(64, np.int64)
    for iz in range(9):
        for iy in range(9):
            for ix in range(9):
                h = ((ix * primes[0]) ^ (iy * primes[1]) ^ (iz * primes[2])) % (1 << 32)
                ref = h % 64
                got = O.vertex_index(p, 0, ix, iy, iz)
                assert got == ref
                counts[got] += 1
    assert counts.sum() == 729 and (counts > 0).all()
    # x prime is 1: along x the hash is the identity mod T
    assert [O.vertex_index(p, 0, ix, 0, 0) for ix in range(9)] == list(range(9))


def test_encode_at_vertices_returns_table_entries():
    # N = 4, 8, 16 (growth 2) all dense in 2^13; x = k/4 lies on a vertex at
    # every level, so each level's feature equals that vertex's entry.
    p = O.inr_params(3, 2, 13, 4, 2.0, 8)
    T = 1 << 13
    rng = np.random.default_rng(0)
    table = rng.normal(size=3 * T * 2)
    pts = np.array([[0.25, 0.5, 0.75], [0.0, 1.0, 0.5], [1.0, 1.0, 1.0]], np.float32)
    feats = O.encode(p, table, pts)
    for j, x in enumerate(pts):
        for l, N in enumerate([4, 8, 16]):
            v = np.minimum((x * N).astype(np.int64), N)
            idx = int(v[0] + (N + 1) * (v[1] + (N + 1) * v[2]))
            assert np.allclose(feats[j, 2 * l:2 * l + 2], table[(l * T + idx) * 2:(l * T + idx) * 2 + 2],
                               atol=1e-15)


def test_encode_reproduces_affine_fields():
    # Trilinear interpolation reproduces affine functions of the vertex
    # coordinates exactly: catches swapped axes, flipped weights, a wrong
    # corner offset or a wrong level scale.
    p = O.inr_params(2, 2, 12, 5, 1.5, 8)  # N = 5, 7 (dense)
    T = 1 << 12
    table = np.zeros(2 * T * 2)
    coef = [(0.3, 1.0, -2.0, 0.5), (-0.1, 0.25, 0.75, -1.5)]
    for l, N in enumerate([5, 7]):
        for iz in range(N + 1):
            for iy in range(N + 1):
                for ix in range(N + 1):
                    idx = ix + (N + 1) * (iy + (N + 1) * iz)
                    for f in range(2):
                        a, b, c, d = coef[f]
                        table[(l * T + idx) * 2 + f] = a + b * ix + c * iy + d * iz + l
    pts = S.random_points(200, seed=3)
    feats = O.encode(p, table, pts)
    for l, N in enumerate([5, 7]):
        g = pts.astype(np.float64) * N
        for f in range(2):
            a, b, c, d = coef[f]
            ref = a + b * g[:, 0] + c * g[:, 1] + d * g[:, 2] + l
            assert np.allclose(feats[:, 2 * l + f], ref, atol=1e-5)


# -------------------------------------------------------------------- MLP
def test_mlp_hand_computed_one_hidden_layer():
    p = O.inr_params(1, 2, 4, 2, 2.0, 2, n_hidden_layers=1)
    w = np.array([1.0, -2.0, 0.5, 0.25,  # W0 [2][2]
                  3.0, -1.0])            # Wout [1][2]
    # a = relu([0.2 - 0.6, 0.1 + 0.075]) = [0, 0.175]; y = 3*0 - 0.175
    y = O.mlp(p, w, np.array([[0.2, 0.3]]))
    assert y[0] == pytest.approx(-0.175, abs=1e-15)


def test_mlp_relu_inactive_is_matrix_product():
    p = O.inr_params(2, 2, 4, 2, 2.0, 3, n_hidden_layers=2)
    rng = np.random.default_rng(1)
    W1 = rng.uniform(0.1, 1.0, (3, 4))
    W2 = rng.uniform(0.1, 1.0, (3, 3))
    W3 = rng.uniform(-1.0, 1.0, (1, 3))
    x = rng.uniform(0.1, 1.0, (5, 4))
    w = np.concatenate([W1.ravel(), W2.ravel(), W3.ravel()])
    ref = (W3 @ W2 @ W1 @ x.T).ravel()
    assert np.allclose(O.mlp(p, w, x), ref, rtol=1e-13)
    # negative pre-activations are cut: flip W1 sign -> all zero
    w2 = np.concatenate([(-W1).ravel(), W2.ravel(), W3.ravel()])
    assert np.allclose(O.mlp(p, w2, x), 0.0)


def test_inr_denormalisation():
    p = O.inr_params(1, 2, 4, 2, 2.0, 2, n_hidden_layers=1, vmin=-3.0, vmax=5.0)
    table = np.zeros(16 * 2)
    w = np.zeros(2 * 2 + 2)
    v = O.inr_eval(p, table, w, np.array([[0.5, 0.5, 0.5]], np.float32))
    assert v[0] == -3.0  # y = 0 -> vmin


# ------------------------------------------------------- rays + compositing
def _zero_inr():
    cfg = S.INR_64
    p = O.inr_params(cfg.levels, cfg.feats, cfg.log2_table, cfg.base_res, cfg.growth, cfg.hidden,
                     vmin=0.5, vmax=1.5)
    return p, np.zeros(cfg.table_entries), np.zeros(cfg.mlp_params)


def test_single_pixel_axis_ray_slab_closed_form():
    cam = O.camera((0, 0, 2), (0, 0, 0), (0, 1, 0), 45.0, 1, 1, 0.5)
    hit, o, d, tn, tf = O.ray(cam, (64, 64, 64), 0, 0)
    assert hit and d.tolist() == [0.0, 0.0, -1.0]
    assert tn == 1.5 and tf == 2.5


@pytest.mark.parametrize("sigma", [0.5, 3.0, 40.0])
def test_constant_density_slab_composites_to_exp(sigma):
    # Constant field (zero MLP -> v = vmin = 0.5), constant TF: opacity of a
    # ray through the box is 1 - exp(-sigma * (tf - tn)) and its colour is
    # rgb times that opacity.  Catches a wrong segment length, a dropped
    # transmittance factor or a wrong alpha.
    p, table, w = _zero_inr()
    cam = O.camera((0.3, 0.2, 2.0), (0, 0, 0), (0, 1, 0), 45.0, 16, 16, 0.5)
    tf = S.tf_constant((0.2, 0.6, 1.0), sigma).astype(np.float64)
    mo = O.march_opts(K=8, eps_T=0.0)
    img, st = O.render_direct(p, table, w, cam, (64, 64, 64), mo, tf)
    n_hit = 0
    for py in range(16):
        for px in range(16):
            hit, o, d, tn, tf_ = O.ray(cam, (64, 64, 64), px, py)
            if not hit:
                assert np.all(img[py, px] == 0.0)
                continue
            n_hit += 1
            a = 1.0 - math.exp(-sigma * (float(tf_) - float(tn)))
            assert img[py, px, 3] == pytest.approx(a, rel=1e-12, abs=1e-14)
            assert np.allclose(img[py, px, :3], np.array([0.2, 0.6, 1.0], np.float32).astype(np.float64) * a,
                               rtol=1e-12, atol=1e-14)
    assert n_hit > 100
    assert st["samples"] == st["inr_queries_direct"] == st["true_misses"]


def test_sample_count_and_termination_at_segment_boundaries():
    p, table, w = _zero_inr()
    cam = O.camera((0.3, 0.2, 2.0), (0, 0, 0), (0, 1, 0), 45.0, 8, 8, 0.5)
    vol = (64, 64, 64)
    tf = S.tf_constant((1, 1, 1), 5.0).astype(np.float64)
    n_total = 0
    n_first_seg = 0
    K = 8
    for py in range(8):
        for px in range(8):
            hit, o, d, tn, tf_ = O.ray(cam, vol, px, py)
            if not hit:
                continue
            k = 0
            while O.sample(cam, vol, o, d, tn, tf_, k)[0]:
                k += 1
            dt = np.float32(0.5) / np.float32(64)
            assert abs(k - (tf_ - tn) / dt) <= 1.0 + 1e-3
            n_total += k
            n_first_seg += min(k, K)
    _, st = O.render_direct(p, table, w, cam, vol, O.march_opts(K=K, eps_T=0.0), tf)
    assert st["samples"] == n_total
    # eps_T = 1: every ray stops at its first segment boundary
    _, st1 = O.render_direct(p, table, w, cam, vol, O.march_opts(K=K, eps_T=1.0), tf)
    assert st1["samples"] == n_first_seg


def test_tf_lookup_endpoints_and_linearity():
    tf = np.zeros((256, 4))
    tf[:, 0] = np.arange(256) / 255.0
    tf[:, 3] = 2.0 * np.arange(256)
    assert O.tf_lookup(tf, -1.0)[0] == 0.0
    assert O.tf_lookup(tf, 2.0)[0] == 1.0
    v = 0.123456
    out = O.tf_lookup(tf, v)
    assert out[0] == pytest.approx(v, abs=1e-15)
    assert out[3] == pytest.approx(2.0 * 255.0 * v, abs=1e-12)


# ------------------------------------------------------------------- LoD
def test_stochastic_lod_mean_equals_continuous_lod_distance_mode():
    cam = O.camera((0, 0, 2), (0, 0, 0), (0, 1, 0), 45.0, 64, 64, 0.5)
    mo = O.march_opts(lod_mode=1, lod_scale=1.0)
    fs = O.frame_seed(0, 1)
    for D in (0.0, 0.3, 1.7, 2.5):
        lods = [O.sample_lod(cam, (64, 64, 64), mo, 8, 0, s, D)
                for px in range(200) for s in O.ray_states(fs, px, 50)]
        lods = np.array(lods)
        assert set(np.unique(lods)) <= {math.floor(D), math.floor(D) + 1}
        assert abs(lods.mean() - D) < 0.02


def test_stochastic_lod_footprint_mode_piecewise_linear_log2():
    # footprint x = t * (2 tan(fov/2) / H) * maxV * lod_scale; D = e + m for
    # x = 2^e (1 + m).  Choose t so that x = 2.5 -> e = 1, m = 0.25.
    cam = O.camera((0, 0, 2), (0, 0, 0), (0, 1, 0), 45.0, 64, 64, 0.5)
    mo = O.march_opts(lod_mode=0, lod_scale=1.0)
    th = np.float32(math.tan(math.radians(22.5)))
    c = np.float32(np.float32(np.float32(2.0) * th) / np.float32(64)) * np.float32(64)
    c = np.float32(c * np.float32(1.0))
    t = np.float32(2.5) / c
    x = np.float32(t * c)
    e = math.floor(math.log2(float(x)))
    m = float(x) / 2 ** e - 1.0
    fs = O.frame_seed(5, 3)
    lods = np.array([O.sample_lod(cam, (64, 64, 64), mo, 8, 0, s, float(t))
                     for px in range(300) for s in O.ray_states(fs, px, 40)])
    assert abs(lods.mean() - (e + m)) < 0.02
    # below one voxel of footprint: LoD 0
    assert O.sample_lod(cam, (64, 64, 64), mo, 8, 0, 0xFFFFFFFF, float(t) / 4) == 0
    # clamped to the coarsest level
    assert O.sample_lod(cam, (64, 64, 64), mo, 2, 0, 0, float(t) * 64) == 1


# ------------------------------------------------------------------ cache
def _golden_rows(kind):
    import os
    path = os.path.join(os.path.dirname(__file__), "golden", "paper_examples.txt")
    rows = []
    for line in open(path):
        if line.startswith("#") or not line.strip():
            continue
        k, args, want, cite = line.rstrip("\n").split("\t")
        if k == kind:
            kv = lambda t: {a.split("=")[0]: a.split("=")[1] for a in t.split()}
            rows.append((kv(args), kv(want), cite))
    assert rows, kind
    return rows


def test_paper_printed_examples():
    # the worked brick mapping of Sec. 4.3.2 and the macro-cell sizes of
    # Sec. 6.3, from the golden fixture
    ints = lambda t: tuple(int(v) for v in t.split(","))
    for a, want, cite in _golden_rows("brick_origin"):
        o = O.brick_origin(ints(a["vol"]), int(a["brick"]), int(a["level"]), ints(a["id"]))
        assert tuple(o) == tuple(float(v) for v in want["origin"].split(",")), cite
    for a, want, cite in _golden_rows("macro_cells"):
        n = int(np.prod(O.macro_dims(ints(a["vol"]), int(a["cell"]))))
        assert n == int(want["cells"]), cite
        # the ranges are two binary32 per cell (float32 [cells, 2] here too)
        assert 8 * n == int(want["range_bytes"]), cite


def test_brick_origin_worked_example():
    # Sec. 4.3.2: request id (0,1,2) at LoD 1 with brick side 40 starts at
    # (0, 79, 159) in LoD-0 voxel coordinates.  y and z must match exactly.
    # x: the apron voxel before brick 0 is clamped to voxel 0, whose LoD-1
    # centre sits at 2^(l-1) = 1 (the paper's 0 has no apron at the volume
    # start; documented reading).
    o = O.brick_origin((400, 400, 400), 40, 1, (0, 1, 2))
    assert o[1] == 79.0 and o[2] == 159.0
    assert o[0] == 1.0
    # A brick of 40 stored voxels at LoD 1 / 2 covers 80 / 160 LoD-0 voxels:
    # consecutive bricks' origins are B * 2^l apart.
    for lev, span in ((1, 80.0), (2, 160.0)):
        a0 = O.brick_origin((4000, 4000, 4000), 40, lev, (1, 1, 1))
        a1 = O.brick_origin((4000, 4000, 4000), 40, lev, (2, 3, 4))
        assert np.allclose(a1 - a0, [span, 2 * span, 3 * span])


def _small_inr(seed=0, scale=0.5):
    cfg = S.INR_64
    table, w = S.inr_init(cfg, seed, table_scale=scale)
    p = O.inr_params(cfg.levels, cfg.feats, cfg.log2_table, cfg.base_res, cfg.growth, cfg.hidden)
    return p, table.astype(np.float64), w.astype(np.float64)


@pytest.mark.parametrize("level", [0, 1, 2])
@pytest.mark.parametrize("vol", [(64, 64, 64), (40, 24, 72)])
def test_brick_sample_equals_whole_grid_trilinear(level, vol):
    # Fully resident cache == trilinear reconstruction of INR values at the
    # LoD-l voxel centres with clamp-to-edge (brute force over the grid, no
    # bricks).  Catches a wrong apron, brick index or local offset.
    p, table, w = _small_inr()
    pts = S.random_points(60, seed=11 + level)
    for x in pts:
        a = O.brick_sample(p, table, w, vol, 8, level, x)
        b = O.resident_sample(p, table, w, vol, level, x)
        assert a == pytest.approx(b, rel=1e-12, abs=1e-13)


def _cache_scene(preload=1, n_slots=200, n_req=6, ranking=1, lod_scale=1.0, lod_mode=0, lag=1,
                 page=0, n_pages=0):
    p, table, w = _small_inr(seed=2)
    vol = (32, 32, 32)
    mo = O.march_opts(K=8, eps_T=0.0, lod_mode=lod_mode, lod_scale=lod_scale, seed=9)
    c = O.Cache(p, table, w, vol, brick=8, levels=3, n_slots=n_slots, mo=mo, n_req=n_req,
                ranking=ranking, preload=preload, lag=lag, page=page, n_pages=n_pages)
    cam = O.camera((0.6, 0.5, 1.6), (0, 0, 0), (0, 1, 0), 45.0, 24, 24, 0.5)
    tf = S.tf_ramps(2).astype(np.float64)
    return c, cam, tf, p, table, w, vol


def test_cache_geometry_and_preload():
    c, cam, tf, *_ = _cache_scene()
    # 32^3, B=8: LoD0 4^3=64 bricks, LoD1 16^3 -> 2^3 = 8, LoD2 8^3 -> 1
    assert c.n_bricks == 64 + 8 + 1
    assert [c.level_offset(l) for l in range(3)] == [0, 64, 72]
    pt = c.dump(O.DUMP_PT)
    assert pt[72] == 0x80000000 and np.all(pt[:72] == 0)
    assert c.dump(O.DUMP_PINNED)[0] == 1 and c.dump(O.DUMP_PINNED)[1:].sum() == 0


def test_cache_first_frame_all_fallback_then_ranked_requests():
    c, cam, tf, *_ = _cache_scene(n_req=6)
    img, st = c.render(cam, tf)
    # Only the coarsest brick is mapped: every sample falls back or hits it.
    assert st["true_misses"] == 0
    assert st["hits"] + st["fallback_hits"] == st["samples"]
    rank = c.dump(O.DUMP_RANK).astype(np.int64)
    Tf = 1001
    cand = np.nonzero(rank > Tf)[0]
    assert len(cand) == st["bricks_requested"] > 6
    score = np.minimum(rank[cand] - Tf, 1000)
    order = sorted(zip(-score, cand))[:6]
    assert c.dump(O.DUMP_REQ).tolist() == [int(k) for _, k in order]
    # victims: never-used slots in ascending order (slot 0 is pinned)
    assert c.dump(O.DUMP_VICT).tolist() == [1, 2, 3, 4, 5, 6]
    pt = c.dump(O.DUMP_PT)
    for s, k in zip(c.dump(O.DUMP_VICT), c.dump(O.DUMP_REQ)):
        assert pt[k] == (0x80000000 | int(s))
    assert st["bricks_decoded"] == 6 and st["inr_queries_decode"] == 6 * 1000
    assert st["evictions"] == 0


def test_cache_ranking_off_takes_first_keys():
    c, cam, tf, *_ = _cache_scene(n_req=5, ranking=0)
    img, st = c.render(cam, tf)
    rank = c.dump(O.DUMP_RANK)
    cand = np.nonzero(rank > 1001)[0]
    assert c.dump(O.DUMP_REQ).tolist() == cand[:5].tolist()


def test_cache_no_preload_first_frame_is_all_true_misses():
    c, cam, tf, p, table, w, vol = _cache_scene(preload=0)
    img, st = c.render(cam, tf)
    assert st["true_misses"] == st["samples"] == st["inr_queries_direct"]
    miss = c.dump(O.DUMP_MISS).reshape(-1, 2)
    assert len(miss) == st["samples"]
    # with no brick resident the cached render is the direct render
    ref, st2 = O.render_direct(p, table, w, cam, vol, c.mo, tf)
    assert np.allclose(img, ref, atol=1e-15)
    assert st2["samples"] == st["samples"]


def test_cache_lru_victims_brute_force_over_frames():
    # Small pool: replacement kicks in.  Victims of each frame must be the
    # eligible slots (not pinned, not used this frame) in ascending
    # (stamp before the frame, slot) order.
    c, cam0, tf, *_ = _cache_scene(n_slots=12, n_req=5)
    pinned = c.dump(O.DUMP_PINNED).astype(bool)
    for f in range(1, 9):
        cam = O.camera((0.6 * math.cos(0.3 * f), 0.5, 1.6 + 0.05 * f), (0, 0, 0), (0, 1, 0),
                       45.0, 24, 24, 0.5)
        before = c.dump(O.DUMP_STAMP).astype(np.int64)
        img, st = c.render(cam, tf)
        after = c.dump(O.DUMP_STAMP).astype(np.int64)
        vict = c.dump(O.DUMP_VICT).tolist()
        used = set(np.nonzero(after == f)[0].tolist()) - set(vict)
        elig = [s for s in range(12) if not pinned[s] and s not in used]
        ref = sorted(elig, key=lambda s: (before[s], s))[:len(vict)]
        assert vict == ref
        assert len(vict) == min(st["bricks_requested"], 5, len(elig))
        # page table and owners stay consistent
        pt = c.dump(O.DUMP_PT)
        own = c.dump(O.DUMP_OWNER)
        for s in range(12):
            if own[s] != 0xFFFFFFFF:
                assert pt[own[s]] == (0x80000000 | s)
        assert np.count_nonzero(pt & 0x80000000) == np.count_nonzero(own != 0xFFFFFFFF)


def test_cache_fully_resident_frame_equals_resident_trilinear():
    # Pool large enough and n_req = all bricks: after frame 1 every requested
    # brick is resident; a second frame from the same view has no requests and
    # its image must equal a render from the resident brute-force sampler.
    c, cam, tf, p, table, w, vol = _cache_scene(n_slots=200, n_req=200, lod_mode=1, lod_scale=0.0)
    c.render(cam, tf)
    img, st = c.render(cam, tf)
    assert st["bricks_requested"] == 0 and st["fallback_hits"] == 0 and st["true_misses"] == 0
    assert st["hits"] == st["samples"]
    # recomposite a few pixels from resident_sample at LoD 0
    for (px, py) in [(12, 12), (5, 17), (20, 3)]:
        hit, o, d, tn, tf_ = O.ray(cam, vol, px, py)
        if not hit:
            continue
        Cc = np.zeros(3)
        T = 1.0
        k = 0
        while True:
            ok, x, tm, ln = O.sample(cam, vol, o, d, tn, tf_, k)
            if not ok:
                break
            v = O.resident_sample(p, table, w, vol, 0, x)
            e = O.tf_lookup(tf, v)
            a = 1.0 - math.exp(-e[3] * ln)
            Cc += T * a * e[:3]
            T *= 1.0 - a
            k += 1
        assert np.allclose(img[py, px, :3], Cc, atol=1e-12)
        assert img[py, px, 3] == pytest.approx(1.0 - T, abs=1e-12)


# --------------------------------------------------------------- training
def test_field_trilinear_voxel_centres_and_affine():
    dims = (5, 4, 3)
    rng = np.random.default_rng(0)
    f = rng.normal(size=(3, 4, 5)).astype(np.float32)
    for (i, j, k) in [(0, 0, 0), (4, 3, 2), (2, 1, 1)]:
        x = np.array([(i + 0.5) / 5, (j + 0.5) / 4, (k + 0.5) / 3], np.float32)
        assert O.field_trilinear(f, x) == pytest.approx(float(f[k, j, i]), abs=1e-6)
    zz, yy, xx = np.meshgrid(np.arange(3), np.arange(4), np.arange(5), indexing="ij")
    g = (0.5 + 0.25 * xx - 0.5 * yy + 2.0 * zz).astype(np.float32)
    x = np.array([0.37, 0.61, 0.55], np.float32)
    q = x.astype(np.float64) * np.array(dims) - 0.5
    assert O.field_trilinear(g, x) == pytest.approx(0.5 + 0.25 * q[0] - 0.5 * q[1] + 2.0 * q[2],
                                                    abs=1e-5)


def test_loss_gradient_matches_central_differences():
    p = O.inr_params(2, 2, 5, 3, 1.7, 4, n_hidden_layers=2)
    T = 1 << 5
    rng = np.random.default_rng(4)
    table = rng.uniform(-0.5, 0.5, 2 * T * 2)
    w = rng.normal(0, 0.8, 4 * 4 + 4 * 4 + 4)
    xyz = rng.uniform(0, 1, (7, 3)).astype(np.float32)
    tgt = rng.uniform(0, 1, 7)
    loss, gt, gw = O.loss_grad(p, table, w, xyz, tgt)
    h = 1e-6
    for arr, g in ((table, gt), (w, gw)):
        idx = np.nonzero(g)[0]
        idx = np.concatenate([idx[:: max(1, len(idx) // 25)], [0]])
        for i in idx:
            a = arr.copy()
            a[i] += h
            lp = O.loss_grad(p, *(a, w) if arr is table else (table, a), xyz, tgt)[0]
            a[i] -= 2 * h
            lm = O.loss_grad(p, *(a, w) if arr is table else (table, a), xyz, tgt)[0]
            fd = (lp - lm) / (2 * h)
            assert g[i] == pytest.approx(fd, rel=1e-5, abs=1e-9)


def test_adam_first_step_closed_form():
    # from zero moments, bias-corrected m/sqrt(v) = g/|g|: step = -lr*sign(g)
    g = np.array([0.5, -2.0, 1e-3])
    prm = np.zeros(3)
    m = np.zeros(3)
    v = np.zeros(3)
    O.lib().orc_adam(prm.ctypes.data_as(O._dp), g.ctypes.data_as(O._dp),
                     m.ctypes.data_as(O._dp), v.ctypes.data_as(O._dp), 3, 0.01, 0.9, 0.99,
                     1e-15, 1)
    assert np.allclose(prm, -0.01 * np.sign(g), rtol=1e-9)
    assert np.allclose(m, 0.1 * g) and np.allclose(v, 0.01 * g * g)


def test_training_reduces_loss():
    cfg = S.InrConfig(levels=4, feats=2, log2_table=10, base_res=4, growth=1.6, hidden=16)
    table, w = S.inr_init(cfg, 1)
    fld = S.explicit_field((16, 16, 16), S.field_params(0, n_gaussians=8))
    p = O.inr_params(cfg.levels, cfg.feats, cfg.log2_table, cfg.base_res, cfg.growth, cfg.hidden)
    tr = O.Trainer(p, table, w, fld, 0.0, 1.0, batch=512, seed=5)
    first = tr.step()
    for _ in range(60):
        last = tr.step()
    assert last < 0.3 * first


def test_psnr_known_mse():
    a = np.zeros((10, 10, 4))
    b = a.copy()
    b[..., :3] = 0.1  # mse 0.01 -> 20 dB
    assert O.psnr(a, b) == pytest.approx(20.0, abs=1e-12)
    assert O.psnr(a, a) == float("inf")


@pytest.mark.parametrize("lod_mode,lod_scale", [(0, 3.0), (1, 10.0)])
def test_lod_scaled_steps_cover_the_chord_and_scale_by_powers_of_two(lod_mode, lod_scale):
    # step mode 1: the segments still tile [tn, tf] exactly (constant slab
    # closed form), and with the level clamped at 2 every step is 4 dt
    p, table, w = _zero_inr()
    cam = O.camera((0.3, 0.2, 2.0), (0, 0, 0), (0, 1, 0), 45.0, 16, 12, 0.5)
    vol = (64, 64, 64)
    tf = S.tf_constant((1.0, 1.0, 1.0), 4.0).astype(np.float64)
    mo = O.march_opts(K=32, eps_T=0.0, lod_mode=lod_mode, lod_scale=lod_scale, step_mode=1,
                      step_lod_max=2)
    img, st = O.render_direct(p, table, w, cam, vol, mo, tf)
    n_ref = 0
    dt = np.float32(0.5) / np.float32(64)
    for py in range(12):
        for px in range(16):
            hit, o, d, tn, tf_ = O.ray(cam, vol, px, py)
            if not hit:
                continue
            a = 1.0 - math.exp(-4.0 * (tf_ - tn))
            assert img[py, px, 3] == pytest.approx(a, abs=1e-12)
            n_ref += math.ceil((tf_ - tn) / (4 * dt))
    if lod_mode == 1:  # D >= 15 everywhere: clamped to level 2, steps of 4 dt
        assert abs(st["samples"] - n_ref) <= 2 * 16 * 12


def test_field_render_constant_field_closed_form():
    # explicit-voxel render of a constant field: opacity 1 - exp(-sigma L)
    f = np.full((8, 6, 10), 0.25, np.float32)
    cam = O.camera((0.3, 0.2, 2.0), (0, 0, 0), (0, 1, 0), 45.0, 12, 10, 0.5)
    tf = S.tf_constant((1.0, 0.5, 0.25), 6.0).astype(np.float64)
    vol = (40, 40, 40)
    img, st = O.render_field(f, cam, vol, O.march_opts(K=32, eps_T=0.0), tf)
    for py in range(10):
        for px in range(12):
            hit, o, d, tn, tf_ = O.ray(cam, vol, px, py)
            a = 1.0 - math.exp(-6.0 * (tf_ - tn)) if hit else 0.0
            assert img[py, px, 3] == pytest.approx(a, abs=1e-12)
    assert st["samples"] > 0


# ------------------------------------------------------------ macro cells
def _step_tf(first_opaque, sigma=25.0):
    # transparent below entry `first_opaque`, constant extinction above
    tf = np.zeros((256, 4), np.float64)
    tf[:, 0], tf[:, 1], tf[:, 2] = 1.0, 0.6, 0.3
    tf[first_opaque:, 3] = sigma
    return tf


def test_macro_dims_and_cell_of_hand_computed():
    # ceil(V/N) cells per axis; cell = floor(x V) / N, far faces clamped
    assert O.macro_dims((64, 40, 17), 16) == (4, 3, 2)
    m = O.macro((64, 40, 17), 16, np.zeros(24, np.uint8))
    assert O.macro_cell_of(m, (64, 40, 17), (0.0, 0.0, 0.0)) == 0
    assert O.macro_cell_of(m, (64, 40, 17), (1.0, 1.0, 1.0)) == 3 + 4 * (2 + 3 * 1)
    # x = 0.25 -> 16 voxels: cell 1; y = 0.39 -> 15.6: cell 0; z = 0.95 -> 16.15: cell 1
    assert O.macro_cell_of(m, (64, 40, 17), (0.25, 0.39, 0.95)) == 1 + 4 * (0 + 3 * 1)


def test_macro_field_ranges_bound_samples_and_are_tight():
    # Every trilinear sample of the field lies inside its cell's range (a
    # convex blend of the voxels the range covers); the range covers at least
    # the voxels centred inside the cell and at most those within one voxel of
    # it.  Catches a box that is too small (bound fails) or too wide.
    rng = np.random.default_rng(5)
    dims, N = (20, 12, 16), 4
    z, y, x = np.meshgrid(*[np.arange(d) for d in dims[::-1]], indexing="ij")
    ramp = (x + 2 * y + 3 * z).astype(np.float32)  # extremes at the box corners
    for f in (rng.normal(size=dims[::-1]).astype(np.float32), ramp):
        _check_field_ranges(f, dims, N)


def _check_field_ranges(f, dims, N):
    r = O.macro_ranges_field(f, N)
    md = O.macro_dims(dims, N)
    m = O.macro(dims, N, np.zeros(int(np.prod(md)), np.uint8))
    for x in S.random_points(4000, seed=3):
        v = O.field_trilinear(f, x)
        c = O.macro_cell_of(m, dims, x)
        assert r[c, 0] <= v <= r[c, 1]
    centres = [np.arange(d) + 0.5 for d in dims]
    for cz in range(md[2]):
        for cy in range(md[1]):
            for cx in range(md[0]):
                c3 = (cx, cy, cz)
                inner = [(cc >= c * N) & (cc < min((c + 1) * N, d)) for cc, c, d in zip(centres, c3, dims)]
                outer = [(cc >= c * N - 1) & (cc <= min((c + 1) * N, d) + 1) for cc, c, d in zip(centres, c3, dims)]
                fi = f[np.ix_(inner[2], inner[1], inner[0])]
                fo = f[np.ix_(outer[2], outer[1], outer[0])]
                ci = cx + md[0] * (cy + md[1] * cz)
                assert fo.min() <= r[ci, 0] <= fi.min()
                assert fi.max() <= r[ci, 1] <= fo.max()


def test_macro_inr_ranges_bound_resident_samples_at_every_lod():
    # The ranges from the INR's LoD voxels bound every fully resident sample
    # (brute-force whole-grid trilinear, no cache code) at every LoD.
    p, table, w = _small_inr(seed=1)
    vol, N, levels = (32, 24, 40), 8, 3
    r = O.macro_ranges_inr(p, table, w, vol, N, levels)
    m = O.macro(vol, N, np.zeros(len(r), np.uint8))
    for x in S.random_points(300, seed=8):
        c = O.macro_cell_of(m, vol, x)
        for lev in range(levels):
            v = O.resident_sample(p, table, w, vol, lev, x)
            assert r[c, 0] <= v <= r[c, 1]
    # fewer levels give narrower (or equal) ranges
    r1 = O.macro_ranges_inr(p, table, w, vol, N, levels, min_level=1)
    assert np.all(r1[:, 0] >= r[:, 0]) and np.all(r1[:, 1] <= r[:, 1])


def test_macro_skip_rule_sound_and_near_tight():
    # Skip only when the TF has zero extinction at every value of the range
    # (dense check through the oracle's TF lookup); keep a cell only when some
    # value within one TF entry (plus the 2^-20 margin) of the range is opaque.
    tf = np.zeros((256, 4), np.float64)
    tf[100:121, 3] = 7.0
    tf[200, 3] = 3.0
    rng = np.random.default_rng(2)
    lo = rng.uniform(-0.1, 1.0, 400)
    hi = lo + rng.uniform(0.0, 0.3, 400) ** 2
    ranges = np.stack([lo, hi], 1).astype(np.float32)
    skip = O.macro_skip(ranges, tf)
    pad = 2.0 ** -20 + 1.0 / 255 + 1e-9
    for (a, b), s in zip(ranges.astype(np.float64), skip):
        vs = np.concatenate([[a, b], np.linspace(a, b, 3000)])
        sig = [O.tf_lookup(tf, v)[3] for v in vs]
        if s:
            assert max(sig) == 0.0
        else:
            wide = np.linspace(a - pad, b + pad, 6000)
            assert max(O.tf_lookup(tf, v)[3] for v in wide) > 0.0
    assert 0 < skip.sum() < len(skip)


def test_macro_majorant_bounds_every_value_and_is_zero_exactly_when_skipped():
    # The majorant of a cell bounds the extinction at every value of its
    # range (dense check through the oracle's TF lookup), is reached within
    # one TF entry (plus the 2^-20 margin) of the range, and is 0 exactly for
    # the cells the skip rule marks transparent.
    rng = np.random.default_rng(5)
    tf = np.zeros((256, 4), np.float64)
    tf[60:90, 3] = rng.uniform(1.0, 9.0, 30).astype(np.float32)
    tf[150:170, 3] = 4.0
    tf[230, 3] = 11.0
    lo = rng.uniform(-0.1, 1.0, 300)
    hi = lo + rng.uniform(0.0, 0.3, 300) ** 2
    ranges = np.stack([lo, hi], 1).astype(np.float32)
    major = O.macro_majorant(ranges, tf)
    skip = O.macro_skip(ranges, tf)
    assert np.array_equal(major == 0.0, skip == 1)
    pad = 2.0 ** -20 + 1.0 / 255 + 1e-9
    for (a, b), m in zip(ranges.astype(np.float64), major):
        vs = np.concatenate([[a, b], np.linspace(a, b, 2000)])
        assert max(O.tf_lookup(tf, v)[3] for v in vs) <= m
        ks = np.arange(256) / 255.0  # the values that read one entry exactly
        wide = np.concatenate([np.linspace(a - pad, b + pad, 2000),
                               ks[(ks >= a - pad) & (ks <= b + pad)]])
        assert max(O.tf_lookup(tf, v)[3] for v in wide) >= m
    assert 0 < skip.sum() < len(skip)


def _cell_of_point(m_dims, cell, vol, o, d, t):
    # macro cell of the point o + t d, in double precision
    e = np.asarray(vol, np.float64) / max(vol)
    x = np.clip((np.asarray(o) + t * np.asarray(d) + e / 2) / e, 0.0, 1.0)
    c = np.minimum((x * np.asarray(vol)) // cell, np.asarray(m_dims) - 1).astype(int)
    return (c[2] * m_dims[1] + c[1]) * m_dims[0] + c[0]


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_pt_walk_spends_optical_depth_cell_by_cell(seed):
    # Each free flight of optical depth tau ends where the integral of the
    # cells' majorants along the ray since the previous collision reaches
    # tau (brute-force quadrature in double); zero-majorant cells hold no
    # collision, and the depth left after the last one exceeds the integral
    # to the ray's exit.
    rng = np.random.default_rng(seed)
    vol, cell = (40, 24, 56), 8
    dims = O.macro_dims(vol, cell)
    n = int(np.prod(dims))
    major = rng.uniform(2.0, 12.0, n).astype(np.float32)
    major[rng.random(n) < 0.3] = 0.0
    mac = O.macro(vol, cell, np.zeros(n, np.uint8), major)
    cam = O.camera((1.1 - 0.3 * seed, 0.4, 1.7), (0.05, -0.02, 0.0), (0, 1, 0), 30.0, 16, 16, 0.5)
    hit, o, d, t0, t1 = O.ray(cam, vol, 7 + seed, 9)
    assert hit
    taus = rng.exponential(1.0, 64).astype(np.float32)
    ts, ms = O.pt_walk_test(mac, vol, o, d, t0, t1, taus)
    assert len(ts) >= 3

    def integral(a, b, steps=20000):
        s = np.linspace(a, b, steps + 1)
        mid = (s[:-1] + s[1:]) / 2
        vals = np.array([major[_cell_of_point(dims, cell, vol, o, d, t)] for t in mid])
        return float(vals.sum() * (b - a) / steps), vals

    prev = t0
    for i, (t, m) in enumerate(zip(ts, ms)):
        assert prev <= t < t1
        got, _ = integral(prev, float(t))
        assert abs(got - taus[i]) < 2e-3 * max(1.0, taus[i]) + 0.02, (i, got, taus[i])
        near = {major[_cell_of_point(dims, cell, vol, o, d, float(t) + dt)] for dt in (-1e-5, 0.0, 1e-5)}
        assert m > 0 and m in near, (i, m, near)
        prev = float(t)
    if len(ts) < len(taus):
        rest, _ = integral(prev, t1)
        assert rest < taus[len(ts)] + 0.02


def test_pt_local_majorants_transmittance_closed_form():
    # Constant extinction c under per-cell majorants drawn from [c, 3c]
    # (some equal to c): delta tracking stays unbiased, so the escape
    # probability of a pixel's path is exp(-c L), as with the global
    # majorant.
    p, table, w, vol, cam = _pt_scene()
    c = 2.5
    tf = S.tf_constant((0.0, 0.0, 0.0), c).astype(np.float64)
    cell = 8
    n = int(np.prod(O.macro_dims(vol, cell)))
    rng = np.random.default_rng(4)
    major = (c * rng.uniform(1.0, 3.0, n)).astype(np.float32)
    major[::3] = c
    mac = O.macro(vol, cell, np.zeros(n, np.uint8), major)
    pt = O.pt_opts(light=(0, 0, 0), ambient=(1, 1, 1), max_bounces=1)
    mo = O.march_opts(seed=5, macro=mac)
    px, py = 4, 3
    hit, o, d, tn, tf_ = O.ray(cam, vol, px, py)
    frames = 3000
    acc = np.zeros(4)
    samples = 0
    for f in range(1, frames + 1):
        img, st = O.render_pt_direct(p, table, w, cam, vol, mo, tf, pt, f, window=(px, py, 1, 1))
        acc += img[0, 0]
        samples += st["samples"]
    mean = acc / frames
    T = math.exp(-c * (tf_ - tn))
    sd = math.sqrt(T * (1 - T) / frames)
    assert abs(mean[0] - T) < 4 * sd
    assert abs(mean[3] - (1 - T)) < 4 * sd
    # more tentative collisions than real ones: the majorants exceed c
    assert samples > frames * (1 - T) * 1.2


def test_pt_cached_local_majorants_skip_empty_cells_and_stay_unbiased():
    # A TF that is transparent below a threshold: cells whose range lies
    # below it get majorant 0 and are crossed without lookups.  With the
    # cache fully resident at every LoD (every sample a trilinear of the
    # voxels the ranges bound), the frame means of local- and global-
    # majorant tracking agree within their statistical error.
    c0, cam, _, p, table, w, vol = _cache_scene(n_slots=700, n_req=700)
    c1, *_ = _cache_scene(n_slots=700, n_req=700)
    r = O.macro_ranges_inr(p, table, w, vol, 8, 3)
    theta = float(np.median(r[:, 1]))
    tf = np.zeros((256, 4), np.float64)
    i0 = int(np.clip(theta, 0, 1) * 255) + 1
    tf[i0:, :3] = 0.8
    tf[i0:, 3] = 30.0
    major = O.macro_majorant(r, tf)
    assert (major == 0).sum() > 0
    mac = O.macro(vol, 8, O.macro_skip(r, tf), major)
    pt = O.pt_opts(max_bounces=2, ambient=(0.2, 0.2, 0.2))
    win = (8, 8, 8, 8)
    for cc in (c0, c1):  # warm-up: bring every requested brick in
        for _ in range(6):
            cc.render_pt(cam, tf, pt)
    a0, a1, s0, s1 = [], [], 0, 0
    for _ in range(150):
        img0, st0 = c0.render_pt(cam, tf, pt, window=win)
        img1, st1 = c1.render_pt(cam, tf, pt, window=win, macro=mac)
        assert st0["true_misses"] == st1["true_misses"] == 0
        a0.append(img0.mean(axis=(0, 1)))
        a1.append(img1.mean(axis=(0, 1)))
        s0 += st0["samples"]
        s1 += st1["samples"]
    a0, a1 = np.array(a0), np.array(a1)
    se = np.sqrt(a0.var(axis=0) / len(a0) + a1.var(axis=0) / len(a1))
    assert np.all(np.abs(a0.mean(axis=0) - a1.mean(axis=0)) < 4 * se + 1e-3)
    assert s1 < s0


def _blob_field(dims=(48, 40, 32)):
    z, y, x = np.meshgrid(*[(np.arange(d) + 0.5) / d for d in dims[::-1]], indexing="ij")
    r2 = (x - 0.45) ** 2 + (y - 0.55) ** 2 + (z - 0.5) ** 2
    return np.exp(-r2 / 0.02).astype(np.float32)


def test_macro_skip_leaves_field_render_unchanged():
    # Skipped samples have alpha = 0 exactly: the image is identical and only
    # the sample count drops (and termination is unaffected).
    f = _blob_field()
    vol = f.shape[::-1]
    tf = _step_tf(80)
    cam = O.camera((1.2, 0.6, 1.6), (0, 0, 0), (0, 1, 0), 40.0, 24, 20, 0.5)
    for eps in (0.0, 1e-2):
        mo = O.march_opts(K=32, eps_T=eps)
        ref, st0 = O.render_field(f, cam, vol, mo, tf)
        mac = O.macro(vol, 8, O.macro_skip(O.macro_ranges_field(f, 8), tf))
        img, st1 = O.render_field(f, cam, vol, O.march_opts(K=32, eps_T=eps, macro=mac), tf)
        assert np.array_equal(img, ref)
        assert st1["samples_skipped"] > 0.3 * st0["samples"]
        assert st1["samples"] + st1["samples_skipped"] == st0["samples"]


def test_macro_skip_leaves_first_cached_frame_unchanged():
    # A fresh cache with the coarsest LoD preloaded has no true misses, so
    # every sample is a trilinear blend of LoD voxels that the INR ranges
    # bound: skipping changes neither the image nor the hit samples; it only
    # withholds the requests of transparent cells.
    c0, cam, _, p, table, w, vol = _cache_scene(n_req=6)
    c1, *_ = _cache_scene(n_req=6)
    r = O.macro_ranges_inr(p, table, w, vol, 8, 3)
    theta = float(np.median(r[:, 1]))
    tf = _step_tf(int(np.clip(theta, 0, 1) * 255) + 1)
    mac = O.macro(vol, 8, O.macro_skip(r, tf))
    ref, st0 = c0.render(cam, tf)
    img, st1 = c1.render(cam, tf, macro=mac)
    assert st1["samples_skipped"] > 0
    assert np.array_equal(img, ref)
    assert st1["samples"] + st1["samples_skipped"] == st0["samples"]
    assert st1["true_misses"] == st0["true_misses"] == 0
    assert st1["bricks_requested"] <= st0["bricks_requested"]


def test_cache_lag2_maps_a_frame_later_and_never_reselects_in_flight_bricks():
    # Lag 2: the bricks selected at the end of frame f stay unmapped through
    # frame f+1 (its samples fall back and request them again) and are mapped
    # at the end of f+1, before f+1's own selection, which must not pick them.
    # LoD 0 everywhere (distance mode, scale 0): no dither, a static camera
    # renders the same image while the state is unchanged.
    c1, cam, tf, *_ = _cache_scene(n_req=6, lod_mode=1, lod_scale=0.0, lag=1)
    c2, *_ = _cache_scene(n_req=6, lod_mode=1, lod_scale=0.0, lag=2)
    a1, s1 = c1.render(cam, tf)
    b1, t1 = c2.render(cam, tf)
    assert np.array_equal(a1, b1) and s1 == t1
    req1, vic1 = c2.dump(O.DUMP_REQ), c2.dump(O.DUMP_VICT)
    assert np.array_equal(req1, c1.dump(O.DUMP_REQ)) and np.array_equal(vic1, c1.dump(O.DUMP_VICT))
    assert len(req1) == 6
    pt1 = c2.dump(O.DUMP_PT)
    assert np.all(pt1[req1] == 0)                       # in flight: not mapped
    assert np.all(c2.dump(O.DUMP_OWNER)[vic1] == 0xFFFFFFFF)
    # frame 2 sees the frame-1 state: same image, the same bricks requested again
    b2, t2 = c2.render(cam, tf)
    assert np.array_equal(b2, b1)
    assert t2["bricks_requested"] == t1["bricks_requested"]
    pt2 = c2.dump(O.DUMP_PT)
    assert np.all(pt2[req1] == (0x80000000 | vic1))     # mapped at the end of frame 2
    assert np.all(c2.dump(O.DUMP_OWNER)[vic1] == req1)
    assert np.all(c2.dump(O.DUMP_STAMP)[vic1] == 2)
    req2 = c2.dump(O.DUMP_REQ)
    assert len(req2) == 6 and not set(req2.tolist()) & set(req1.tolist())
    assert not set(c2.dump(O.DUMP_VICT).tolist()) & set(vic1.tolist())
    # lag 1 had mapped the same bricks into the same slots one frame earlier
    pa = c1.dump(O.DUMP_PT)
    assert np.array_equal(pa[req1], pt2[req1])
    # frame 3 hits them: fewer fallback samples than frame 2
    b3, t3 = c2.render(cam, tf)
    assert t3["fallback_hits"] < t2["fallback_hits"] and t3["hits"] > t2["hits"]


# ------------------------------------------------------------ path tracing
def test_neg_log1m_close_to_log_and_exact_at_zero():
    # the binary32 series log against the library log: within 2 ulp
    assert O.neg_log1m(0.0) == 0.0
    for u in list(np.arange(1, 1 << 24, 7919) / 2.0**24) + [0.5, 1 - 2.0**-24]:
        ref = -math.log1p(-u)
        assert abs(O.neg_log1m(u) - ref) <= 2.5e-7 * ref


def test_pt_uniform_is_the_splitmix64_stream():
    # element 0 of the stream from state 0 is the top 24 bits of SplitMix64's
    # published first output 0xE220A8397B1DCDAF; element j of key k is
    # element j-1 of key k + gamma; uniform mean
    assert O.pt_uniform(0, 0) == 0xE220A8 / 2.0**24
    g = 0x9E3779B97F4A7C15
    for key in (1, 12345, 2**63 + 7):
        for j in (1, 2, 17):
            assert O.pt_uniform(key, j) == O.pt_uniform((key + g) % 2**64, j - 1)
    u = np.array([O.pt_uniform(99, j) for j in range(20000)])
    assert abs(u.mean() - 0.5) < 0.01 and u.min() >= 0.0 and u.max() < 1.0


def test_pt_sphere_directions_are_uniform_unit_vectors():
    d = []
    j = 0
    for _ in range(20000):
        v, j = O.pt_sphere(777, j)
        d.append(v)
    d = np.array(d, np.float64)
    assert np.abs(np.linalg.norm(d, axis=1) - 1).max() < 1e-6
    assert np.abs(d.mean(0)).max() < 0.02
    assert np.abs((d ** 2).mean(0) - 1 / 3).max() < 0.01
    assert abs((d[:, 0] * d[:, 1]).mean()) < 0.01
    assert j >= 2 * 20000  # two uniforms per try, rejection ~21%


def _pt_scene():
    p, table, w = _small_inr(seed=3)
    vol = (32, 32, 32)
    cam = O.camera((0.2, 0.3, 1.8), (0, 0, 0), (0, 1, 0), 30.0, 8, 8, 0.5)
    return p, table, w, vol, cam


def test_pt_delta_tracking_transmittance_closed_form():
    # constant extinction c, black albedo, ambient radiance 1, one bounce:
    # a path returns 1 exactly when it crosses the volume without a real
    # collision, so the mean over frames is exp(-c L)
    p, table, w, vol, cam = _pt_scene()
    c = 2.5
    tf = S.tf_constant((0.0, 0.0, 0.0), c).astype(np.float64)
    pt = O.pt_opts(light=(0, 0, 0), ambient=(1, 1, 1), max_bounces=1)
    mo = O.march_opts(seed=5)
    px, py = 4, 3
    hit, o, d, tn, tf_ = O.ray(cam, vol, px, py)
    assert hit
    n = 3000
    acc = np.zeros(4)
    for f in range(1, n + 1):
        img, st = O.render_pt_direct(p, table, w, cam, vol, mo, tf, pt, f, window=(px, py, 1, 1))
        acc += img[0, 0]
    mean = acc / n
    T = math.exp(-c * (tf_ - tn))
    sd = math.sqrt(T * (1 - T) / n)
    assert abs(mean[0] - T) < 4 * sd
    assert abs(mean[3] - (1 - T)) < 4 * sd


def test_pt_single_scatter_with_ratio_tracking_closed_form():
    # constant extinction c, white albedo, light along the pixel's ray (the
    # shadow ray runs back to the entry point), majorant 3c (ratio tracking
    # gives a continuous transmittance), irradiance 4 pi: the expected
    # radiance is int_0^L c exp(-c t) exp(-c t) dt = (1 - exp(-2 c L)) / 2
    p, table, w, vol, cam = _pt_scene()
    c = 1.5
    tf = S.tf_constant((1.0, 1.0, 1.0), c).astype(np.float64)
    px, py = 4, 3
    hit, o, d, tn, tf_ = O.ray(cam, vol, px, py)
    pt = O.pt_opts(light_dir=tuple(float(v) for v in d), light=(4 * math.pi,) * 3,
                   ambient=(0, 0, 0), max_bounces=1, sigma_max=3 * c)
    mo = O.march_opts(seed=6)
    n = 4000
    vals = np.array([O.render_pt_direct(p, table, w, cam, vol, mo, tf, pt, f,
                                        window=(px, py, 1, 1))[0][0, 0, 0] for f in range(1, n + 1)])
    L = tf_ - tn
    ref = (1 - math.exp(-2 * c * L)) / 2
    assert abs(vals.mean() - ref) < 4 * vals.std() / math.sqrt(n) + 1e-3


def test_pt_cached_frames_deterministic_and_preloaded():
    # two fresh caches render identical frames and states; with the coarsest
    # LoD preloaded no lookup is a true miss
    runs = []
    for _ in range(2):
        c, cam, tf, *_ = _cache_scene(n_req=8)
        pt = O.pt_opts(max_bounces=2)
        imgs = [c.render_pt(cam, tf, pt) for _ in range(2)]
        runs.append((imgs, c.dump(O.DUMP_PT), c.dump(O.DUMP_STAMP), c.dump(O.DUMP_RANK)))
    (i0, pt0, s0, r0), (i1, pt1, s1, r1) = runs
    for (a, sa), (b, sb) in zip(i0, i1):
        assert np.array_equal(a, b) and sa == sb
        assert sa["true_misses"] == 0 and sa["hits"] + sa["fallback_hits"] == sa["samples"] > 0
    assert np.array_equal(pt0, pt1) and np.array_equal(s0, s1) and np.array_equal(r0, r1)
    assert i0[0][1]["bricks_requested"] > 0


# --------------------------------------------------- virtualised page tables
def _paged_check(c):
    # page accounting: refcount = mapped entries of the page; directory and
    # slot keys agree; no resident page is empty
    P3 = c.co.page ** 3
    pd, pages = c.dump(O.DUMP_PAGE_DIR), c.dump(O.DUMP_PAGES).reshape(-1, P3)
    keys, refs = c.dump(O.DUMP_PAGE_KEY), c.dump(O.DUMP_PAGE_REF)
    for ps in range(len(keys)):
        mapped = int(np.count_nonzero(pages[ps] & 0x80000000))
        if keys[ps] == 0xFFFFFFFF:
            assert mapped == 0 and refs[ps] == 0
        else:
            assert pd[keys[ps]] == (0x80000000 | ps)
            assert refs[ps] == mapped > 0
    assert np.count_nonzero(pd & 0x80000000) == np.count_nonzero(keys != 0xFFFFFFFF)


@pytest.mark.parametrize("page", [1, 2, 4])
def test_paged_tables_equal_flat_tables_with_room(page):
    # with enough page slots the two-level tables resolve every brick as the
    # flat table does: same images, statistics, requests, victims and state
    runs = []
    for pg in (0, page):
        c, cam0, tf, *_ = _cache_scene(n_slots=14, n_req=6, page=pg, n_pages=4096 if pg else 0,
                                       lod_mode=1, lod_scale=0.0)
        out = []
        for f in range(1, 7):
            a = 1.3 * f
            cam = O.camera((1.4 * math.cos(a), 0.3, 1.4 * math.sin(a)), (0, 0, 0), (0, 1, 0),
                           14.0, 24, 24, 0.5)
            img, st = c.render(cam, tf)
            out.append((img, st, c.dump(O.DUMP_PT), c.dump(O.DUMP_OWNER), c.dump(O.DUMP_STAMP),
                        c.dump(O.DUMP_REQ), c.dump(O.DUMP_VICT)))
            if pg:
                _paged_check(c)
        runs.append(out)
    for a, b in zip(*runs):
        assert np.array_equal(a[0], b[0]) and a[1] == b[1]
        for x, y in zip(a[2:], b[2:]):
            assert np.array_equal(x, y)
    assert sum(o[1]["evictions"] for o in runs[1]) > 0


def test_paged_tables_under_page_pressure_allocate_lowest_page_keys_first():
    # two page slots beyond the coarsest LoD's: the frame's mappings need
    # more pages than are free; the ascending page keys get the free slots
    # in ascending order and the other requests are dropped (their victim
    # slots stay free); the accounting stays consistent
    c, cam, tf, *_ = _cache_scene(n_slots=60, n_req=20, page=2, n_pages=3)
    keys0 = c.dump(O.DUMP_PAGE_KEY)
    assert keys0[0] != 0xFFFFFFFF and np.all(keys0[1:] == 0xFFFFFFFF)  # coarsest LoD: one page
    img, st = c.render(cam, tf)
    _paged_check(c)
    req, vic = c.dump(O.DUMP_REQ), c.dump(O.DUMP_VICT)
    own, pt = c.dump(O.DUMP_OWNER), c.dump(O.DUMP_PT)
    P = 2
    def page_key(k):
        l = 0
        while l + 1 < 3 and k >= c.level_offset(l + 1):
            l += 1
        loc = k - c.level_offset(l)
        _, nb = c.level_dims(l)
        b = (loc % nb[0], (loc // nb[0]) % nb[1], loc // (nb[0] * nb[1]))
        pg = [(n + P - 1) // P for n in nb]
        off = sum(int(np.prod([(n + P - 1) // P for n in c.level_dims(j)[1]])) for j in range(l))
        return off + b[0] // P + pg[0] * (b[1] // P + pg[1] * (b[2] // P))
    need = sorted({page_key(int(k)) for k in req})
    assert len(need) > 2
    keys = c.dump(O.DUMP_PAGE_KEY)
    assert keys[1] == need[0] and keys[2] == need[1]
    pages = c.dump(O.DUMP_PAGES).reshape(-1, P ** 3)
    for k, s in zip(req, vic):
        if page_key(int(k)) in need[:2]:
            assert pt[k] == (0x80000000 | s) and own[s] == k
            # the entry sits at (bx%P) + P ((by%P) + P (bz%P)) of its page
            l = 0
            while l + 1 < 3 and k >= c.level_offset(l + 1):
                l += 1
            loc = int(k) - c.level_offset(l)
            _, nb = c.level_dims(l)
            b = (loc % nb[0], (loc // nb[0]) % nb[1], loc // (nb[0] * nb[1]))
            local = b[0] % P + P * (b[1] % P + P * (b[2] % P))
            ps = int(np.nonzero(keys == page_key(int(k)))[0][0])
            assert pages[ps, local] == (0x80000000 | s)
        else:
            assert pt[k] == 0 and own[s] == 0xFFFFFFFF


def test_row_parallel_oracle_equals_the_plain_oracle():
    """The all-core timing build renders the same window, row by row, to the
    same bits and counts as the single-threaded oracle."""
    from paper_2504_18001_gb300 import synthetic as S
    cfg = S.INR_64
    table, w = S.inr_init(cfg, seed=1, table_scale=0.5)
    p = O.inr_params(cfg.levels, cfg.feats, cfg.log2_table, cfg.base_res, cfg.growth, cfg.hidden)
    cam = S.orbit_camera(3, 40, 40)
    oc = O.camera(cam["eye"], cam["target"], cam["up"], cam["fov_y_deg"], 40, 40, cam["step_voxels"])
    mo = O.march_opts(K=32, eps_T=1e-3)
    tf = S.tf_ramps(2).astype(np.float64)
    win = (6, 9, 21, 17)
    a, sa = O.render_direct(p, table, w, oc, (64, 64, 64), mo, tf, window=win)
    b, sb = O.render_direct_rows(p, table, w, oc, (64, 64, 64), mo, tf, window=win)
    assert np.array_equal(a, b)
    assert sa == sb and sa["samples"] > 0
    assert O.omp_threads() >= 1
    ys, xs = np.mgrid[9:26, 6:27]
    c, sc = O.render_direct_pixels(p, table, w, oc, (64, 64, 64), mo, tf, xs.ravel(), ys.ravel())
    assert np.array_equal(c.reshape(a.shape), a)
    assert sc == sa


def test_request_ranks_equal_an_independent_count_of_unmapped_lookups():
    """Sec. 4.3 / 4.3.3: every sample whose requested-LoD brick is Unmapped
    raises one request for that brick, also when a coarser LoD then serves
    the sample, and a brick's score in a frame is its request count capped
    at 1000 above the frame's timestamp T_f = 1001 f.  The samples are
    enumerated here from the ray, sample-schedule and LoD primitives (pinned
    above), the brick key of each is computed in numpy binary32, and the
    lookups that meet an Unmapped entry of the page table as it stood at the
    frame's start are counted per brick.  No termination (eps_T = 0), so the
    sample set does not depend on the composited values.  The scene is sized
    so that some bricks take more than 1000 requests in the first frame (the
    clamp) and others fewer."""
    cfg = S.INR_64
    table, w = S.inr_init(cfg, seed=1, table_scale=0.5)
    p = O.inr_params(cfg.levels, cfg.feats, cfg.log2_table, cfg.base_res, cfg.growth, cfg.hidden)
    vol, Wd, Hd, B, L = (64, 64, 64), 36, 36, 8, 4
    mo = O.march_opts(K=32, eps_T=0.0)
    cache = O.Cache(p, table, w, vol, B, L, 600, mo, n_req=40)
    offs = [cache.level_offset(l) for l in range(L)]
    nbs = [cache.level_dims(l)[1] for l in range(L)]
    volf = np.array(vol, np.float32)
    clamped = unclamped = 0
    for f in (1, 2):
        pt = cache.dump(O.DUMP_PT)  # the page table the frame's lookups see
        cam = O.camera(**S.orbit_camera(f, Wd, Hd))
        fseed = O.frame_seed(0, f)
        counts = {}
        for py in range(Hd):
            for px in range(Wd):
                hit, o, d, tn, tf = O.ray(cam, vol, px, py)
                if not hit:
                    continue
                rs = O.ray_seed(fseed, py * Wd + px)
                k = 0
                while True:
                    ok, x, tm, _ = O.sample(cam, vol, o, d, tn, tf, k)
                    if not ok:
                        break
                    l = O.sample_lod(cam, vol, mo, L, 0, int(O.lib().orc_sample_state(rs, k)), tm)
                    s = (x.astype(np.float32) * volf) * np.float32(1.0 / (1 << l))
                    b = np.clip(np.floor(s / np.float32(B)).astype(np.int64), 0, nbs[l] - 1)
                    key = int(offs[l] + b[0] + nbs[l][0] * (b[1] + nbs[l][1] * b[2]))
                    if not pt[key] & 0x80000000:
                        counts[key] = counts.get(key, 0) + 1
                    k += 1
        cache.render(cam, S.tf_ramps(2).astype(np.float64))
        rank = cache.dump(O.DUMP_RANK).astype(np.int64)
        Tf = 1001 * f
        expect = np.zeros_like(rank)
        for key, n in counts.items():
            expect[key] = min(n, 1000)
        assert np.array_equal(np.where(rank > Tf, rank - Tf, 0), expect)
        clamped += sum(1 for n in counts.values() if n > 1000)
        unclamped += sum(1 for n in counts.values() if n < 1000)
    assert clamped > 0 and unclamped > 0
