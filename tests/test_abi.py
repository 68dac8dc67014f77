"""CPU checks of the C-ABI library: it builds, loads without a GPU, exports
every function include/cinr.h declares, and its host-only size queries and
argument checks behave (no device compute is called here)."""
import ctypes as C

import pytest

from paper_2504_18001_gb300 import cinr, synthetic as S


@pytest.fixture(scope="module")
def L():
    return cinr.lib()


def test_every_header_symbol_is_exported(L):
    names = cinr.header_symbols()
    assert len(names) >= 19
    missing = [n for n in names if not hasattr(L, n)]
    assert not missing, missing
    assert L.cinr_version() >= 100


def test_inr_bytes_and_shape_checks(L):
    p = cinr.make_inr_params(S.INR_512)
    n = C.c_size_t()
    assert L.cinr_inr_bytes(C.byref(p), C.byref(n)) == 0
    # table 16 * 2^19 * 2 floats, weights, fp16 copy, scratch
    assert n.value >= 16 * (1 << 19) * 8 + S.INR_512.mlp_params * 6
    bad = cinr.make_inr_params(S.InrConfig(levels=5, feats=2, log2_table=10, base_res=4,
                                           growth=1.5, hidden=32))
    assert L.cinr_inr_bytes(C.byref(bad), C.byref(n)) == -1
    assert "unsupported MLP shape" in cinr.last_error()


def test_cache_slot_arithmetic_matches_paper_and_config(L):
    o = cinr.cinr_cache_opts(8, 4, 40, 1, 1, 0)
    dims = (C.c_int * 3)(512, 512, 512)
    nb, ns = C.c_size_t(), C.c_long()
    assert L.cinr_cache_bytes(dims, 1 << 30, C.byref(o), C.byref(nb), C.byref(ns)) == 0
    assert ns.value == (1 << 30) // (10 ** 3 * 4) == 268435
    # Sec. 6.3: a 30^3-brick cache of 40^3 stored FP32 voxels is 1.728e9
    # voxels, just under 7 GB (interior 38 + 2 apron = 40 stored per edge)
    o2 = cinr.cinr_cache_opts(38, 6, 40, 1, 1, 0)
    dims2 = (C.c_int * 3)(4096, 4096, 4096)
    pool = 30 ** 3 * 40 ** 3 * 4
    assert pool == 6_912_000_000
    assert L.cinr_cache_bytes(dims2, pool, C.byref(o2), C.byref(nb), C.byref(ns)) == 0
    assert ns.value == 27000
    # brick loading buffer of the paper: 40 requests of 40^3 FP32 = 10.24 MB
    assert 40 * 40 ** 3 * 4 == 10_240_000


def test_renderer_option_checks(L):
    o = cinr.cinr_march_opts((C.c_int * 3)(64, 64, 64), 48, 1e-3, 0, 1.0, 0, 0)
    n = C.c_size_t()
    assert L.cinr_renderer_bytes(128, 128, C.byref(o), C.byref(n)) == -1
    assert "multiple of 32" in cinr.last_error()
    o.K = 64
    assert L.cinr_renderer_bytes(128, 128, C.byref(o), C.byref(n)) == 0
    assert n.value >= 128 * 128 * 16


def test_cache_option_checks(L):
    dims = (C.c_int * 3)(64, 64, 64)
    nb, ns = C.c_size_t(), C.c_long()
    o = cinr.cinr_cache_opts(8, 13, 40, 1, 1, 0)  # too many LoDs
    assert L.cinr_cache_bytes(dims, 1 << 20, C.byref(o), C.byref(nb), C.byref(ns)) == -1
    o = cinr.cinr_cache_opts(8, 3, 10000, 1, 1, 0)  # n_req above the limit (8192)
    assert L.cinr_cache_bytes(dims, 1 << 20, C.byref(o), C.byref(nb), C.byref(ns)) == -1


def test_macro_cell_size_query_and_checks(L):
    # Sec. 6.3: 16^3 cells over a 4096^3 volume = 256^3 = 16.8 M cells; the
    # structure holds 8 B of range + 4 B of majorant + 1 B of flag per cell
    dims = (C.c_int * 3)(4096, 4096, 4096)
    n = C.c_size_t()
    assert L.cinr_macro_bytes(dims, 16, C.byref(n)) == 0
    assert 256 ** 3 == 16_777_216
    assert 13 * 256 ** 3 <= n.value < 13 * 256 ** 3 + 1024
    # ragged: ceil(V / cell) per axis
    dims2 = (C.c_int * 3)(100, 17, 33)
    assert L.cinr_macro_bytes(dims2, 16, C.byref(n)) == 0
    assert n.value >= 13 * 7 * 2 * 3
    for bad in (1, 12, 2048):
        assert L.cinr_macro_bytes(dims2, bad, C.byref(n)) == -1
        assert "power of two" in cinr.last_error()
    d = cinr.cinr_macro_desc()
    d.dims[:] = [64, 64, 64]
    d.cell, d.source = 16, 7
    h = C.c_void_p()
    assert L.cinr_create_macro(C.byref(d), None, 0, None, C.byref(h)) == -1
    d.source = cinr.MACRO_FROM_INR  # no INR given
    assert L.cinr_create_macro(C.byref(d), None, 0, None, C.byref(h)) == -1
    assert "needs an INR" in cinr.last_error()


def test_frame_stats_layout_matches_header(L):
    # 13 counters of 8 bytes, then two float timings
    assert C.sizeof(cinr.cinr_frame_stats) == 13 * 8 + 8
    assert cinr.cinr_frame_stats.samples_skipped.offset == 12 * 8


def test_null_handles_are_rejected_without_device_work(L):
    # every entry point that takes a handle checks it before any CUDA call
    assert L.cinr_trainer_set_lr(None, C.c_float(1e-3)) == cinr.ERR_ARG
    assert L.cinr_trainer_set_tensor_cores(None, 1) == cinr.ERR_ARG
    assert L.cinr_trainer_set_stratified(None, 1) == cinr.ERR_ARG
    assert L.cinr_cache_set_decode_encoder(None, 1) == cinr.ERR_ARG
    assert L.cinr_trainer_status(None, None) == cinr.ERR_ARG
    assert L.cinr_debug_wait_timeout(None, 16, None) == cinr.ERR_ARG
    assert L.cinr_macro_majorants(None, None, 0, None) == cinr.ERR_ARG
    assert L.cinr_inr_status(None, None) == cinr.ERR_ARG
    assert L.cinr_train(None, None, None, None, 1, None, 0, None) == cinr.ERR_ARG
    assert "NULL" in cinr.last_error()


def test_error_codes_match_header():
    import os
    import re
    text = open(os.path.join(os.path.dirname(__file__), "..", "include", "cinr.h")).read()
    codes = dict((m.group(1), int(m.group(2))) for m in re.finditer(r"#define CINR_(ERR_\w+) \((-\d+)\)", text))
    for name, val in codes.items():
        assert getattr(cinr, name) == val, name
    assert "ERR_NAN" in codes and "ERR_TIMEOUT" in codes


def test_default_build_has_no_device_checks_and_entry_writes_check_arguments(L):
    # the product build compiles the device bounds checks away; the checked
    # build (-DCINR_CHECK=1) is exercised by tests/test_gpu_checks.py
    assert L.cinr_device_checks() == 0
    assert L.cinr_debug_set_entry(None, cinr.DUMP_PAGE_TABLE, 0, 0, None) == cinr.ERR_ARG
