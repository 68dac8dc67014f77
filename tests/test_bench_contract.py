"""The benchmark's output contract: one JSON line with the keys the
measurement protocol fixes, for the reference arm on CPU and for the GPU
arm on a short run."""
import json
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _run(args, timeout=600):
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), *args], cwd=ROOT,
                         capture_output=True, text=True, timeout=timeout)
    assert out.returncode == 0, out.stderr[-2000:]
    lines = [ln for ln in out.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1, out.stdout[-2000:]
    return json.loads(lines[0])


BASE_KEYS = ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step",
             "higher_is_better", "scaling", "vs_baseline", "dtype", "data", "config", "e2e")


def test_reference_arm_line():
    d = _run(["--impl", "reference", "--steps", "2", "--warmup", "3"])
    for k in BASE_KEYS + ("impl", "cpu_baseline"):
        assert k in d, k
    assert d["impl"] == "reference" and d["steps"] == 2 and d["warmup"] == 3
    assert d["higher_is_better"] is False and d["value"] > 0
    assert d["config"]["workload"] == "cached_mixed_512cube_1024px_orbit"
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["value"] == d["value"] and cb["sample"]
    e = d["e2e"]
    assert e["value"] == d["value"] and e["unit"] == d["unit"]
    assert e["h2d_bytes_per_step"] == 0 and e["d2h_bytes_per_step"] == 0


@pytest.mark.gpu
def test_gpu_arm_line():
    d = _run(["--steps", "3", "--warmup", "3", "--uncached-steps", "1", "--no-other"])
    for k in BASE_KEYS + ("roofline", "cpu_baseline", "clocks", "gpu_launches"):
        assert k in d, k
    assert d["n_gpus"] == 1 and d["steps"] == 3 and d["warmup"] == 3 and d["value"] > 0
    assert d["config"]["workload"] == "cached_mixed_512cube_1024px_orbit"
    r = d["roofline"]
    for k in ("bound", "achieved", "peak", "unit", "frac", "traffic"):
        assert k in r, k
    assert abs(r["frac"] - r["achieved"] / r["peak"]) < 1e-9 * max(1.0, r["frac"])
    e = d["e2e"]
    assert e["value"] > 0 and e["h2d_bytes_per_step"] > 0 and e["d2h_bytes_per_step"] >= 1024 * 1024 * 16
    assert d["gpu_launches"] >= 3
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["cores"] >= 1
    assert "sm_mhz" in d["clocks"] and "reasons" in d["clocks"]
    # the timed frames follow the cache-fill phase and pass the quality gate;
    # the end-to-end pass replays the same cache states
    c = d["config"]
    assert c["cache_fill_frames"] >= 1 and c["timed_frames"][0] == c["cache_fill_frames"] + 3
    g = d["quality_gate"]
    assert g["ok"] and g["worst_db"] >= 40.0 and g["min_db"] == 40.0
    assert e["same_cache_state_as_timed_frames"] is True


def test_profile_counters_only_for_the_profiled_sources(tmp_path, monkeypatch):
    # the roofline's DRAM traffic and instruction counts come from an ncu
    # summary only while the kernel sources hash to the value it records
    import hashlib
    sys.path.insert(0, ROOT)
    import bench
    for rel in bench.KERNEL_SOURCES:
        dst = tmp_path / rel
        dst.parent.mkdir(parents=True, exist_ok=True)
        dst.write_bytes(open(os.path.join(ROOT, rel), "rb").read())
    h = hashlib.sha256()
    for rel in bench.KERNEL_SOURCES:
        h.update((tmp_path / rel).read_bytes())
    (tmp_path / "profiles").mkdir()
    summary = tmp_path / "profiles" / "p.md"

    def write(digest):
        summary.write_text("# kernel\n\n- frame: 95\n- samples: 100\n- dram_bytes: 2000\n"
                           f"- warp_instructions: 700\n- thread_instructions: 22000\n"
                           f"- kernel_source_sha256_12: {digest}\n")

    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    monkeypatch.setattr(bench, "PROFILE_FILES", {"orbit": "p.md"})
    write(h.hexdigest()[:12])
    got = bench.profiled_counters("orbit")
    assert got is not None and got["dram_bytes"] == 2000.0 and got["frame"] == 95
    write("000000000000")
    assert bench.profiled_counters("orbit") is None
    # a changed source invalidates a summary that matched before
    write(h.hexdigest()[:12])
    src = tmp_path / bench.KERNEL_SOURCES[0]
    src.write_bytes(src.read_bytes() + b"\n// changed\n")
    assert bench.profiled_counters("orbit") is None
