"""Device bounds checks (a library built with -DCINR_CHECK=1).

The memory checker is not available on the GPU pool; instead a checked build
tests every page-table, page, slot, pool and hash-table index on the device
before the access it guards, skips the access and reports
CINR_ERR_DEVICE_CHECK.  These tests load the checked build in a child
process (CINR_CHECKED=1), plant page-table entries that name a slot beyond
the pool or a page slot beyond the page pool, and check that the next frame
reports the error and that the frame after the entries are restored renders
normally.  Frames of an intact cache render without a report and match the
oracle's discrete state.  The cache buffers carry slack bytes after the
cache's own, so that even an unchecked read of the planted slot would stay
inside the allocation.
"""
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

_CHILD = r"""
import sys
sys.path.insert(0, {root!r})
sys.path.insert(0, {tests!r})
import numpy as np
import oracle as O
from paper_2504_18001_gb300 import cinr, synthetic as S
from _scenes import gpu_inr, oracle_inr, ocam, scene

L = cinr.lib()
assert L.cinr_device_checks() == 1, "not the checked build"
vol = (64, 64, 64)
cfg = S.INR_64
table, w = scene(cfg)
inr = gpu_inr(cfg, table, w, vol=vol)
p = oracle_inr(cfg, table, w, vol=vol)
tf = S.tf_ramps(2)


def frame(rend, cache, f):
    cam = S.orbit_camera(f, 48, 40)
    img, st = rend.render(inr, cam, tf, cache=cache)
    return st


def expect_check(fn):
    try:
        fn()
    except cinr.CinrError as e:
        assert e.code == cinr.ERR_DEVICE_CHECK, e
        return
    raise AssertionError("the planted entry was not reported")


# intact caches: no report, the oracle's discrete state
for lod_mode in (0, 1):
    rend = cinr.Renderer(48, 40, vol, K=32, eps_T=0.0, lod_mode=lod_mode, lod_scale=1.0 if lod_mode == 0 else 2.0)
    cache = cinr.Cache(inr, vol, pool_bytes=300 * 1000 * 4, brick=8, levels=4, n_req=40, slack_bytes=4 << 20)
    oc = O.Cache(p, table, w, vol, 8, 4, cache.n_slots, O.march_opts(K=32, eps_T=0.0, lod_mode=lod_mode,
                 lod_scale=1.0 if lod_mode == 0 else 2.0), n_req=40)
    for f in range(3):
        st = frame(rend, cache, f)
        ref, rst = oc.render(ocam(S.orbit_camera(f, 48, 40)), tf.astype(np.float64))
        assert st["samples"] == rst["samples"] and st["hits"] == rst["hits"], (st, rst)
        assert np.array_equal(cache.dump(cinr.DUMP_PAGE_TABLE), oc.dump(O.DUMP_PT))
    # every mapped entry names the slot one past the pool
    pt = cache.dump(cinr.DUMP_PAGE_TABLE)
    mapped = np.nonzero(pt & 0x80000000)[0]
    assert len(mapped) > 0
    for k in mapped:
        cache.set_entry(cinr.DUMP_PAGE_TABLE, int(k), 0x80000000 | cache.n_slots)
    expect_check(lambda: frame(rend, cache, 3))
    for k in mapped:
        cache.set_entry(cinr.DUMP_PAGE_TABLE, int(k), int(pt[k]))
    frame(rend, cache, 4)
    print("flat lod_mode", lod_mode, "ok")

# virtualised page tables: a page-directory entry naming a page slot beyond
# the page pool
rend = cinr.Renderer(48, 40, vol, K=32, eps_T=0.0)
cache = cinr.Cache(inr, vol, pool_bytes=300 * 1000 * 4, brick=8, levels=4, n_req=40, page=2, n_pages=64,
                   slack_bytes=4 << 20)
frame(rend, cache, 0)
pd = cache.dump(cinr.DUMP_PAGE_DIR)
mapped = np.nonzero(pd & 0x80000000)[0]
assert len(mapped) > 0
for k in mapped:  # every resident page names the page slot one past the page pool
    cache.set_entry(cinr.DUMP_PAGE_DIR, int(k), 0x80000000 | 64)
expect_check(lambda: frame(rend, cache, 1))
# the frame's cache update may have met the planted entries too (request
# candidates and evictions read the page directory): those checks report to
# the INR's status word, which the status call reads and clears
rc = L.cinr_inr_status(inr.h, cinr._stream(None))
assert rc in (0, cinr.ERR_DEVICE_CHECK), rc
for k in mapped:
    cache.set_entry(cinr.DUMP_PAGE_DIR, int(k), int(pd[k]))
frame(rend, cache, 2)
cinr.check(L.cinr_inr_status(inr.h, cinr._stream(None)), "cinr_inr_status")
print("checked build ok")
"""


def test_checked_build_reports_planted_out_of_range_entries():
    code = _CHILD.format(root=ROOT, tests=os.path.join(ROOT, "tests"))
    env = dict(os.environ, CINR_CHECKED="1")
    r = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, timeout=1200,
                       cwd=ROOT, env=env)
    assert r.returncode == 0, r.stdout[-3000:] + r.stderr[-3000:]
    assert "checked build ok" in r.stdout
