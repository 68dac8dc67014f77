"""The autotuner on a small mixed-precision scene: every candidate of the
knob grid is timed, the chosen setting meets the PSNR floor against the
uncached FP32 frame and is the fastest of the candidates that do."""
import pytest

from paper_2504_18001_gb300 import synthetic as S

from _scenes import gpu_inr

pytestmark = pytest.mark.gpu


def test_tuner_picks_the_fastest_setting_above_the_psnr_floor():
    from paper_2504_18001_gb300 import autotune
    vol = (128, 128, 128)
    cfg = S.INR_64
    # the benchmark's INR form (amplitude halving per level), pixels of about
    # one voxel: the cached frame is served at LoD 0 and stays close to the
    # uncached FP32 frame
    table, w = S.inr_init(cfg, seed=0, table_scale=1.0, level_decay=0.5)
    inr_c = gpu_inr(cfg, table, w, vol=vol, mlp="bf16", tab="fp16")
    inr32 = gpu_inr(cfg, table, w, vol=vol)
    W = H = 256
    tf = S.tf_ramps(2)
    best, trials = autotune.tune(
        inr_c, inr32, vol, lambda f: (S.orbit_camera(f, W, H), tf), W, H, bricks=(8, 16),
        n_reqs=(64, 512), layouts=(0,), graphs=(0, 1), decode_ctas=(0, 2), decode_encoders=(1, 0),
        levels=3, pool_mib=64,
        max_warmup=60, timed=3, min_psnr=30.0)
    assert len(trials) == 2 * 2 * 2 * 2 * 2
    ok = [t for t in trials if t["psnr_db"] >= 30.0]
    assert ok, trials
    fastest = min(ok, key=lambda t: t["ms_per_frame"])
    assert best == {k: fastest[k] for k in best}
    assert fastest["psnr_db"] >= 30.0
    assert all(t["ms_per_frame"] > 0 for t in trials)
