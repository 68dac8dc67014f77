"""Thin ctypes binding of the C ABI in include/cinr.h (argument marshalling
only; every step of the renderer runs in libcinr.so's CUDA kernels).

PyTorch provides device memory and streams: each object's device buffer is a
uint8 CUDA tensor sized by the library's *_bytes() query.  Importing this
module does not need a GPU; creating objects does, and fails loudly when the
library or the device is missing (there is no CPU fallback).
"""
from __future__ import annotations

import ctypes as C
import os
import re

import numpy as np

from . import build as _build

_lib = None

CINR_OK = 0
ERR_ARG, ERR_NOMEM, ERR_CUDA, ERR_TIMEOUT, ERR_DEVICE_CHECK, ERR_UNSUPPORTED, ERR_NAN = range(-1, -8, -1)
PREC = {"fp32": 0, "fp16": 1, "bf16": 2, "fp8": 3, "fp16tex": 4}  # fp16tex: cache storage only
DUMP_PAGE_TABLE, DUMP_STAMPS, DUMP_OWNERS, DUMP_RANK, DUMP_REQUESTS, DUMP_VICTIMS, \
    DUMP_MISSES, DUMP_PINNED, DUMP_POOL, DUMP_PAGE_DIR, DUMP_PAGES, DUMP_PAGE_KEYS, \
    DUMP_PAGE_REFS = range(13)


class CinrError(RuntimeError):
    def __init__(self, msg, code=None):
        super().__init__(msg)
        self.code = code


class cinr_inr_params(C.Structure):
    _fields_ = [("levels", C.c_int), ("feats", C.c_int), ("log2_table", C.c_int),
                ("base_res", C.c_int), ("growth", C.c_double), ("hidden", C.c_int),
                ("n_hidden_layers", C.c_int), ("mlp_precision", C.c_int),
                ("table_precision", C.c_int), ("vmin", C.c_float), ("vmax", C.c_float)]


class cinr_camera(C.Structure):
    _fields_ = [("eye", C.c_float * 3), ("target", C.c_float * 3), ("up", C.c_float * 3),
                ("fov_y_deg", C.c_float), ("width", C.c_int), ("height", C.c_int),
                ("step_voxels", C.c_float)]


class cinr_tf(C.Structure):
    _fields_ = [("rgba", (C.c_float * 4) * 256)]


class cinr_march_opts(C.Structure):
    _fields_ = [("dims", C.c_int * 3), ("K", C.c_int), ("eps_T", C.c_float),
                ("lod_mode", C.c_int), ("lod_scale", C.c_float), ("seed", C.c_uint64),
                ("miss_record_cap", C.c_long), ("ray_layout", C.c_int), ("step_mode", C.c_int),
                ("step_lod_max", C.c_int), ("use_graph", C.c_int)]


class cinr_cache_opts(C.Structure):
    _fields_ = [("brick", C.c_int), ("levels", C.c_int), ("n_req", C.c_int),
                ("ranking", C.c_int), ("preload", C.c_int), ("storage_precision", C.c_int),
                ("lag", C.c_int), ("page", C.c_int), ("n_pages", C.c_long)]


class cinr_frame_stats(C.Structure):
    _fields_ = [(n, C.c_uint64) for n in (
        "samples", "inr_queries_direct", "inr_queries_decode", "true_misses", "fallback_hits",
        "hits", "bricks_requested", "bricks_decoded", "evictions", "misses_recorded",
        "slots_touched", "kernel_launches", "samples_skipped")] + [
            ("ms_frame_kernel", C.c_float), ("ms_cache_update", C.c_float)]

    def as_dict(self):
        return {n: (float(getattr(self, n)) if t is C.c_float else int(getattr(self, n)))
                for n, t in self._fields_}


class cinr_pt_opts(C.Structure):
    _fields_ = [("light_dir", C.c_float * 3), ("light", C.c_float * 3), ("ambient", C.c_float * 3),
                ("max_bounces", C.c_int), ("sigma_max", C.c_float)]


def make_pt_opts(light_dir=(0.3, -1.0, -0.4), light=(3.0, 3.0, 3.0), ambient=(0.0, 0.0, 0.0),
                 max_bounces=3, sigma_max=0.0) -> cinr_pt_opts:
    return cinr_pt_opts((C.c_float * 3)(*light_dir), (C.c_float * 3)(*light),
                        (C.c_float * 3)(*ambient), int(max_bounces), float(sigma_max))


class cinr_macro_desc(C.Structure):
    _fields_ = [("dims", C.c_int * 3), ("cell", C.c_int), ("source", C.c_int),
                ("inr", C.c_void_p), ("cache", C.c_void_p), ("levels", C.c_int),
                ("min_level", C.c_int), ("ranges_host", C.c_void_p), ("field_dev", C.c_void_p)]


MACRO_FROM_INR, MACRO_FROM_RANGES, MACRO_FROM_FIELD = 0, 1, 2

_vp = C.c_void_p
_P = C.POINTER
_SIGS = {
    "cinr_last_error": [C.c_char_p, C.c_size_t],
    "cinr_version": [],
    "cinr_inr_bytes": [_P(cinr_inr_params), _P(C.c_size_t)],
    "cinr_create_inr": [_P(cinr_inr_params), _vp, C.c_size_t, _P(C.c_float), _P(C.c_float), _vp,
                        _P(_vp)],
    "cinr_inr_set_range": [_vp, C.c_float, C.c_float],
    "cinr_inr_raw_range": [_vp, _P(C.c_int), C.c_int, _P(C.c_float), _P(C.c_float), _vp],
    "cinr_infer": [_vp, _vp, C.c_long, _vp, _vp],
    "cinr_encode": [_vp, _vp, C.c_long, _vp, _vp, _vp],
    "cinr_destroy_inr": [_vp],
    "cinr_cache_bytes": [_P(C.c_int), C.c_size_t, _P(cinr_cache_opts), _P(C.c_size_t),
                         _P(C.c_long)],
    "cinr_create_cache": [_vp, _P(C.c_int), _vp, C.c_size_t, C.c_size_t, _P(cinr_cache_opts), _vp,
                          _P(_vp)],
    "cinr_destroy_cache": [_vp],
    "cinr_renderer_bytes": [C.c_int, C.c_int, _P(cinr_march_opts), _P(C.c_size_t)],
    "cinr_create_renderer": [_vp, C.c_size_t, C.c_int, C.c_int, _P(cinr_march_opts), _P(_vp)],
    "cinr_render_frame": [_vp, _vp, _vp, _P(cinr_camera), _P(cinr_tf), _vp, _P(cinr_frame_stats),
                          _vp],
    "cinr_render_frame_host": [_vp, _vp, _vp, _P(cinr_camera), _P(cinr_tf), _vp,
                               _P(cinr_frame_stats), _vp],
    "cinr_destroy_renderer": [_vp],
    "cinr_render_field": [_vp, _vp, _P(C.c_int), _P(cinr_camera), _P(cinr_tf), _vp,
                          _P(cinr_frame_stats), _vp],
    "cinr_render_frame_noalloc": [_vp, _P(cinr_camera), _P(cinr_tf), _P(cinr_march_opts), _vp,
                                  _P(cinr_frame_stats), _vp],
    "cinr_trainer_bytes": [_vp, _vp, _P(C.c_size_t)],
    "cinr_create_trainer": [_vp, _vp, _vp, C.c_size_t, _vp, _P(_vp)],
    "cinr_train_step": [_vp, _vp, _P(C.c_int), _vp, _vp],
    "cinr_inr_loss_grad": [_vp, _vp, _vp, C.c_long, _vp, _vp, _vp, _vp],
    "cinr_destroy_trainer": [_vp],
    "cinr_trainer_status": [_vp, _vp],
    "cinr_trainer_set_lr": [_vp, C.c_float],
    "cinr_trainer_set_tensor_cores": [_vp, C.c_int],
    "cinr_trainer_set_stratified": [_vp, C.c_int],
    "cinr_train": [_vp, _vp, _P(C.c_int), _vp, C.c_long, _vp, C.c_size_t, _vp],
    "cinr_inr_export": [_vp, _vp, _vp, _vp],
    "cinr_debug_dump": [_vp, C.c_int, _vp, C.c_size_t, _P(C.c_size_t), _vp],
    "cinr_debug_set_entry": [_vp, C.c_int, C.c_size_t, C.c_uint32, _vp],
    "cinr_device_checks": [],
    "cinr_cache_set_decode_ctas": [_vp, C.c_int],
    "cinr_cache_set_decode_encoder": [_vp, C.c_int],
    "cinr_debug_mma_tile": [_vp, _vp, C.c_int, C.c_int, _vp, _vp],
    "cinr_inr_status": [_vp, _vp],
    "cinr_debug_wait_timeout": [_vp, C.c_uint, _vp],
    "cinr_cache_level_info": [_vp, C.c_int, _P(C.c_int), _P(C.c_int), _P(C.c_long)],
    "cinr_macro_bytes": [_P(C.c_int), C.c_int, _P(C.c_size_t)],
    "cinr_create_macro": [_P(cinr_macro_desc), _vp, C.c_size_t, _vp, _P(_vp)],
    "cinr_macro_ranges": [_vp, _vp, C.c_size_t, _vp],
    "cinr_macro_skip_flags": [_vp, _vp, C.c_size_t, _vp],
    "cinr_macro_majorants": [_vp, _vp, C.c_size_t, _vp],
    "cinr_macro_apply_tf": [_vp, _vp, _vp],
    "cinr_destroy_macro": [_vp],
    "cinr_renderer_set_macro": [_vp, _vp],
    "cinr_render_frame_pt": [_vp, _vp, _vp, _vp, _vp, _vp, _vp, _P(cinr_frame_stats), _vp],
}


def header_symbols():
    """Function names declared in include/cinr.h."""
    hdr = os.path.join(os.path.dirname(_build.HERE), "include", "cinr.h")
    txt = open(hdr).read()
    return sorted(set(re.findall(r"^int\s+(cinr_\w+)\s*\(", txt, flags=re.M)))


def lib(build_if_missing: bool = True):
    """Load libcinr.so (building it with nvcc when stale).  With the
    environment variable CINR_CHECKED=1 the process loads the build with
    device bounds checks instead (paper_2504_18001_gb300/_build_check/)."""
    global _lib
    if _lib is None:
        checked = os.environ.get("CINR_CHECKED", "0") == "1"
        if checked:
            path = _build.build(checked=True) if build_if_missing else _build.LIB_CHECK
        else:
            path = _build.build() if build_if_missing else _build.LIB
        if not os.path.exists(path):
            raise CinrError(f"libcinr.so not found at {path}; run __graft_entry__.build()")
        L = C.CDLL(path)
        for name, args in _SIGS.items():
            f = getattr(L, name)
            f.restype = C.c_int
            f.argtypes = args
        _lib = L
    return _lib


def last_error() -> str:
    buf = C.create_string_buffer(512)
    lib().cinr_last_error(buf, 512)
    return buf.value.decode()


def check(rc: int, what: str = ""):
    if rc != CINR_OK:
        raise CinrError(f"{what} failed ({rc}): {last_error()}", rc)


def _stream(stream):
    if stream is None:
        import torch
        stream = torch.cuda.current_stream()
    return C.c_void_p(stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream))


def _dev_buffer(nbytes: int, device):
    import torch
    if not torch.cuda.is_available():
        raise CinrError("CUDA device required: the renderer has no CPU path")
    return torch.empty(max(int(nbytes), 256), dtype=torch.uint8, device=device)


def _fptr(t):
    return C.cast(C.c_void_p(t.data_ptr()), _P(C.c_float))


# ------------------------------------------------------------ high level
def make_inr_params(cfg, mlp_precision="fp32", table_precision="fp32", vmin=0.0, vmax=1.0):
    return cinr_inr_params(cfg.levels, cfg.feats, cfg.log2_table, cfg.base_res, float(cfg.growth),
                           cfg.hidden, cfg.n_hidden_layers, PREC[mlp_precision],
                           PREC[table_precision], float(vmin), float(vmax))


def make_camera(d) -> cinr_camera:
    c = cinr_camera()
    c.eye[:] = [float(v) for v in d["eye"]]
    c.target[:] = [float(v) for v in d["target"]]
    c.up[:] = [float(v) for v in d["up"]]
    c.fov_y_deg = float(d["fov_y_deg"])
    c.width, c.height = int(d["width"]), int(d["height"])
    c.step_voxels = float(d["step_voxels"])
    return c


def make_tf(arr) -> cinr_tf:
    t = cinr_tf()
    a = np.ascontiguousarray(np.asarray(arr, np.float32).reshape(256, 4))
    C.memmove(C.addressof(t), a.ctypes.data, a.nbytes)
    return t


class Inr:
    def __init__(self, params: cinr_inr_params, table: np.ndarray, mlp: np.ndarray, device="cuda",
                 stream=None):
        L = lib()
        nbytes = C.c_size_t()
        check(L.cinr_inr_bytes(C.byref(params), C.byref(nbytes)), "cinr_inr_bytes")
        self.mem = _dev_buffer(nbytes.value, device)
        t = np.ascontiguousarray(table, np.float32)
        w = np.ascontiguousarray(mlp, np.float32)
        h = C.c_void_p()
        check(L.cinr_create_inr(C.byref(params), C.c_void_p(self.mem.data_ptr()), nbytes.value,
                                t.ctypes.data_as(_P(C.c_float)), w.ctypes.data_as(_P(C.c_float)),
                                _stream(stream), C.byref(h)), "cinr_create_inr")
        self.h = h
        self.params = params

    def set_range(self, vmin, vmax):
        check(lib().cinr_inr_set_range(self.h, float(vmin), float(vmax)), "cinr_inr_set_range")

    def raw_range(self, dims, stride=1, stream=None):
        d = (C.c_int * 3)(*dims)
        lo, hi = C.c_float(), C.c_float()
        check(lib().cinr_inr_raw_range(self.h, d, int(stride), C.byref(lo), C.byref(hi),
                                       _stream(stream)), "cinr_inr_raw_range")
        return lo.value, hi.value

    def infer(self, xyz, out=None, stream=None):
        import torch
        n = xyz.shape[0]
        if out is None:
            out = torch.empty(n, dtype=torch.float32, device=xyz.device)
        check(lib().cinr_infer(self.h, C.c_void_p(xyz.data_ptr()), n, C.c_void_p(out.data_ptr()),
                               _stream(stream)), "cinr_infer")
        return out

    def encode(self, xyz, with_indices=False, stream=None):
        import torch
        n = xyz.shape[0]
        IN = self.params.levels * self.params.feats
        feats = torch.empty((n, IN), dtype=torch.float32, device=xyz.device)
        idx = torch.empty((n, self.params.levels, 8), dtype=torch.int32, device=xyz.device) \
            if with_indices else None
        check(lib().cinr_encode(self.h, C.c_void_p(xyz.data_ptr()), n, C.c_void_p(feats.data_ptr()),
                                C.c_void_p(idx.data_ptr()) if idx is not None else None,
                                _stream(stream)), "cinr_encode")
        return feats, idx

    def __del__(self):
        try:
            if getattr(self, "h", None):
                lib().cinr_destroy_inr(self.h)
                self.h = None
        except Exception:
            pass


class Cache:
    def __init__(self, inr: Inr, dims, pool_bytes, brick=8, levels=4, n_req=40, ranking=1,
                 preload=1, storage="fp32", lag=1, page=0, n_pages=0, device="cuda", stream=None,
                 slack_bytes=0):
        L = lib()
        self.opts = cinr_cache_opts(int(brick), int(levels), int(n_req), int(ranking), int(preload),
                                    PREC[storage], int(lag), int(page), int(n_pages))
        self.dims = (C.c_int * 3)(*dims)
        nbytes, nslots = C.c_size_t(), C.c_long()
        check(L.cinr_cache_bytes(self.dims, int(pool_bytes), C.byref(self.opts), C.byref(nbytes),
                                 C.byref(nslots)), "cinr_cache_bytes")
        self.n_slots = nslots.value
        # slack_bytes: unused bytes after the cache's own (tests of the device
        # bounds checks keep even an unchecked stray read inside the buffer)
        self.mem = _dev_buffer(nbytes.value + int(slack_bytes), device)
        h = C.c_void_p()
        check(L.cinr_create_cache(inr.h, self.dims, C.c_void_p(self.mem.data_ptr()), nbytes.value,
                                  int(pool_bytes), C.byref(self.opts), _stream(stream), C.byref(h)),
              "cinr_create_cache")
        self.h = h
        self.inr = inr

    def level_info(self, level):
        d = (C.c_int * 3)()
        nb = (C.c_int * 3)()
        off = C.c_long()
        check(lib().cinr_cache_level_info(self.h, level, d, nb, C.byref(off)), "level_info")
        return tuple(d), tuple(nb), off.value

    def set_decode_ctas(self, ctas_per_sm):
        """Decode CTAs per SM (0: as many as fit)."""
        check(lib().cinr_cache_set_decode_ctas(self.h, int(ctas_per_sm)), "cinr_cache_set_decode_ctas")

    def set_decode_encoder(self, staged):
        """Brick decode encoder: 1 staged tile encoder, 0 per-voxel gathers."""
        check(lib().cinr_cache_set_decode_encoder(self.h, int(staged)), "cinr_cache_set_decode_encoder")

    def set_entry(self, what, index, value, stream=None):
        """Writes one u32 page-table entry (tests of the device checks)."""
        check(lib().cinr_debug_set_entry(self.h, what, int(index), int(value) & 0xFFFFFFFF,
                                         _stream(stream)), "cinr_debug_set_entry")

    def dump(self, what, stream=None):
        return debug_dump(self.h, what, stream, pool_half=self.opts.storage_precision in (1, 4))

    def __del__(self):
        try:
            if getattr(self, "h", None):
                lib().cinr_destroy_cache(self.h)
                self.h = None
        except Exception:
            pass


class Macro:
    """Macro cells of Sec. 5.2 (per-cell value ranges; skip flags per TF).

    source: Inr (with an optional Cache whose stored values the ranges must
    bound), a float32 array of ranges [cells, 2] (host), or a device field
    tensor [z, y, x]."""

    def __init__(self, dims, cell=16, inr: Inr | None = None, cache: Cache | None = None,
                 levels=1, min_level=0, ranges=None, field=None, device="cuda", stream=None):
        L = lib()
        d = cinr_macro_desc()
        d.dims[:] = [int(v) for v in dims]
        d.cell = int(cell)
        d.levels, d.min_level = int(levels), int(min_level)
        keep = None
        if ranges is not None:
            keep = np.ascontiguousarray(ranges, dtype=np.float32)
            d.source, d.ranges_host = MACRO_FROM_RANGES, keep.ctypes.data
        elif field is not None:
            d.source, d.field_dev = MACRO_FROM_FIELD, field.data_ptr()
        else:
            d.source = MACRO_FROM_INR
            d.inr = inr.h.value if inr is not None else None
            d.cache = cache.h.value if cache is not None else None
        nbytes = C.c_size_t()
        check(L.cinr_macro_bytes(d.dims, d.cell, C.byref(nbytes)), "cinr_macro_bytes")
        self.mem = _dev_buffer(nbytes.value, device)
        h = C.c_void_p()
        check(L.cinr_create_macro(C.byref(d), C.c_void_p(self.mem.data_ptr()), nbytes.value,
                                  _stream(stream), C.byref(h)), "cinr_create_macro")
        self.h = h
        self.dims = tuple(int(v) for v in dims)
        self.cell = int(cell)
        self.cdims = tuple((v + self.cell - 1) // self.cell for v in self.dims)
        self.n = int(np.prod(self.cdims))
        self._refs = (inr, cache, field, keep)

    def ranges(self, stream=None):
        out = np.zeros((self.n, 2), np.float32)
        check(lib().cinr_macro_ranges(self.h, C.c_void_p(out.ctypes.data), out.size,
                                      _stream(stream)), "cinr_macro_ranges")
        return out

    def apply_tf(self, tf, stream=None):
        t = tf if isinstance(tf, cinr_tf) else make_tf(tf)
        check(lib().cinr_macro_apply_tf(self.h, C.byref(t), _stream(stream)), "cinr_macro_apply_tf")

    def skip_flags(self, stream=None):
        out = np.zeros(self.n, np.uint8)
        check(lib().cinr_macro_skip_flags(self.h, C.c_void_p(out.ctypes.data), out.size,
                                          _stream(stream)), "cinr_macro_skip_flags")
        return out

    def majorants(self, stream=None):
        out = np.zeros(self.n, np.float32)
        check(lib().cinr_macro_majorants(self.h, C.c_void_p(out.ctypes.data), out.size,
                                         _stream(stream)), "cinr_macro_majorants")
        return out

    def __del__(self):
        try:
            if getattr(self, "h", None):
                lib().cinr_destroy_macro(self.h)
                self.h = None
        except Exception:
            pass


def debug_dump(handle, what, stream=None, pool_half=False):
    L = lib()
    n = C.c_size_t()
    s = _stream(stream)
    check(L.cinr_debug_dump(handle, what, None, 0, C.byref(n), s), "cinr_debug_dump")
    if what == DUMP_POOL:
        out = np.zeros(n.value, np.float16 if pool_half else np.float32)
    else:
        out = np.zeros(n.value, np.uint32)
    if n.value:
        check(L.cinr_debug_dump(handle, what, C.c_void_p(out.ctypes.data), n.value, C.byref(n), s),
              "cinr_debug_dump")
    return out


class cinr_train_opts(C.Structure):
    _fields_ = [("batch", C.c_long), ("lr", C.c_float), ("beta1", C.c_float),
                ("beta2", C.c_float), ("eps", C.c_float), ("seed", C.c_uint64)]


def inr_export(inr: Inr, stream=None):
    """(table, mlp) FP32 host copies of a trained (FP32-table) INR."""
    cfg = inr.params
    table = np.zeros(cfg.levels * (1 << cfg.log2_table) * cfg.feats, np.float32)
    IN, H = cfg.levels * cfg.feats, cfg.hidden
    mlp = np.zeros(H * IN + H * H + H, np.float32)
    check(lib().cinr_inr_export(inr.h, C.c_void_p(table.ctypes.data), C.c_void_p(mlp.ctypes.data),
                                _stream(stream)), "cinr_inr_export")
    return table, mlp


def train(inr: "Inr", field, steps, batch=1 << 18, lr=1e-2, beta1=0.9, beta2=0.99, eps=1e-15, seed=0,
          stream=None):
    """cinr_train: `steps` Adam steps on field (torch float32 [z, y, x] on the
    device) in a temporary workspace; raises CinrError(ERR_NAN) on a
    non-finite gradient."""
    L = lib()
    opts = cinr_train_opts(int(batch), float(lr), float(beta1), float(beta2), float(eps), int(seed))
    nbytes = C.c_size_t()
    check(L.cinr_trainer_bytes(inr.h, C.byref(opts), C.byref(nbytes)), "cinr_trainer_bytes")
    ws = _dev_buffer(nbytes.value, field.device)
    dims = (C.c_int * 3)(field.shape[2], field.shape[1], field.shape[0])
    check(L.cinr_train(inr.h, C.c_void_p(field.data_ptr()), dims, C.byref(opts), int(steps),
                       C.c_void_p(ws.data_ptr()), nbytes.value, _stream(stream)), "cinr_train")


class Trainer:
    """INR training on an explicit field (Sec. 4.1): Adam steps on batches of
    counter-based random coordinates; updates the INR in place."""

    def __init__(self, inr: Inr, batch=1 << 18, lr=1e-2, beta1=0.9, beta2=0.99, eps=1e-15, seed=0,
                 device="cuda", stream=None):
        import torch
        L = lib()
        self.opts = cinr_train_opts(int(batch), float(lr), float(beta1), float(beta2), float(eps),
                                    int(seed))
        nbytes = C.c_size_t()
        check(L.cinr_trainer_bytes(inr.h, C.byref(self.opts), C.byref(nbytes)), "cinr_trainer_bytes")
        self.mem = _dev_buffer(nbytes.value, device)
        h = C.c_void_p()
        check(L.cinr_create_trainer(inr.h, C.byref(self.opts), C.c_void_p(self.mem.data_ptr()),
                                    nbytes.value, _stream(stream), C.byref(h)), "cinr_create_trainer")
        self.h = h
        self.inr = inr
        self.loss = torch.zeros(1, dtype=torch.float32, device=device)

    def step(self, field, stream=None):
        """One step on field (torch float32 [z, y, x] on the device)."""
        dims = (C.c_int * 3)(field.shape[2], field.shape[1], field.shape[0])
        check(lib().cinr_train_step(self.h, C.c_void_p(field.data_ptr()), dims,
                                    C.c_void_p(self.loss.data_ptr()), _stream(stream)),
              "cinr_train_step")
        return self.loss

    def set_lr(self, lr):
        check(lib().cinr_trainer_set_lr(self.h, float(lr)), "cinr_trainer_set_lr")

    def set_stratified(self, on):
        """1: one coordinate per cell of a Morton-ordered grid per batch; 0: uniform."""
        check(lib().cinr_trainer_set_stratified(self.h, int(on)), "cinr_trainer_set_stratified")

    def set_tensor_cores(self, mode):
        """The fused tensor-core forward / backward kernel with 1 FP16 or
        2 BF16 operands; 0 the FP32 kernels."""
        check(lib().cinr_trainer_set_tensor_cores(self.h, int(mode)), "cinr_trainer_set_tensor_cores")

    def status(self, stream=None):
        """Raises CinrError (CINR_ERR_NAN) when a step since the last check
        produced a non-finite gradient (CINR_ERR_TIMEOUT: a tensor-core wait
        of the fused kernel gave up)."""
        check(lib().cinr_trainer_status(self.h, _stream(stream)), "cinr_trainer_status")

    def loss_grad(self, xyz, target, stream=None):
        import torch
        p = self.inr.params
        gt = torch.empty(p.levels * (1 << p.log2_table) * p.feats, dtype=torch.float32,
                         device=xyz.device)
        IN, H = p.levels * p.feats, p.hidden
        gw = torch.empty(H * IN + H * H + H, dtype=torch.float32, device=xyz.device)
        check(lib().cinr_inr_loss_grad(self.h, C.c_void_p(xyz.data_ptr()),
                                       C.c_void_p(target.data_ptr()), xyz.shape[0],
                                       C.c_void_p(gt.data_ptr()), C.c_void_p(gw.data_ptr()),
                                       C.c_void_p(self.loss.data_ptr()), _stream(stream)),
              "cinr_inr_loss_grad")
        return self.loss, gt, gw

    def __del__(self):
        try:
            if getattr(self, "h", None):
                lib().cinr_destroy_trainer(self.h)
                self.h = None
        except Exception:
            pass


class Renderer:
    def __init__(self, width, height, dims, K=32, eps_T=1e-3, lod_mode=0, lod_scale=1.0, seed=0,
                 miss_record_cap=0, ray_layout=0, step_mode=0, step_lod_max=0, use_graph=0,
                 device="cuda"):
        L = lib()
        self.opts = cinr_march_opts((C.c_int * 3)(*dims), int(K), float(eps_T), int(lod_mode),
                                    float(lod_scale), int(seed), int(miss_record_cap),
                                    int(ray_layout), int(step_mode), int(step_lod_max),
                                    int(use_graph))
        nbytes = C.c_size_t()
        check(L.cinr_renderer_bytes(int(width), int(height), C.byref(self.opts), C.byref(nbytes)),
              "cinr_renderer_bytes")
        self.mem = _dev_buffer(nbytes.value, device)
        h = C.c_void_p()
        check(L.cinr_create_renderer(C.c_void_p(self.mem.data_ptr()), nbytes.value, int(width),
                                     int(height), C.byref(self.opts), C.byref(h)),
              "cinr_create_renderer")
        self.h = h
        self.W, self.H = int(width), int(height)
        self.device = device

    def render(self, inr: Inr, camera, tf, cache: Cache | None = None, out=None, stream=None):
        import torch
        if out is None:
            out = torch.empty((self.H, self.W, 4), dtype=torch.float32, device=self.device)
        cam = camera if isinstance(camera, cinr_camera) else make_camera(camera)
        t = tf if isinstance(tf, cinr_tf) else make_tf(tf)
        st = cinr_frame_stats()
        check(lib().cinr_render_frame(self.h, cache.h if cache is not None else None, inr.h,
                                      C.byref(cam), C.byref(t), C.c_void_p(out.data_ptr()),
                                      C.byref(st), _stream(stream)), "cinr_render_frame")
        return out, st.as_dict()

    def render_host(self, inr: Inr, camera, tf, out_host, cache: Cache | None = None, stream=None):
        cam = camera if isinstance(camera, cinr_camera) else make_camera(camera)
        t = tf if isinstance(tf, cinr_tf) else make_tf(tf)
        st = cinr_frame_stats()
        check(lib().cinr_render_frame_host(self.h, cache.h if cache is not None else None, inr.h,
                                           C.byref(cam), C.byref(t),
                                           C.c_void_p(out_host.data_ptr()), C.byref(st),
                                           _stream(stream)), "cinr_render_frame_host")
        return st.as_dict()

    def render_field(self, field, camera, tf, out=None, stream=None):
        """Explicit-voxel render of field (torch float32 [z, y, x] on the device)."""
        import torch
        if out is None:
            out = torch.empty((self.H, self.W, 4), dtype=torch.float32, device=self.device)
        cam = camera if isinstance(camera, cinr_camera) else make_camera(camera)
        t = tf if isinstance(tf, cinr_tf) else make_tf(tf)
        dims = (C.c_int * 3)(field.shape[2], field.shape[1], field.shape[0])
        st = cinr_frame_stats()
        check(lib().cinr_render_field(self.h, C.c_void_p(field.data_ptr()), dims, C.byref(cam),
                                      C.byref(t), C.c_void_p(out.data_ptr()), C.byref(st),
                                      _stream(stream)), "cinr_render_field")
        return out, st.as_dict()

    def misses(self, stream=None):
        return debug_dump(self.h, DUMP_MISSES, stream).reshape(-1, 2)

    def render_pt(self, inr: Inr, camera, tf, pt=None, cache: Cache | None = None, out=None,
                  stream=None):
        """One path-traced frame (Woodcock delta tracking); returns (rgba, stats)."""
        import torch
        if out is None:
            out = torch.empty((self.H, self.W, 4), dtype=torch.float32, device=self.device)
        cam = camera if isinstance(camera, cinr_camera) else make_camera(camera)
        t = tf if isinstance(tf, cinr_tf) else make_tf(tf)
        o = pt if isinstance(pt, cinr_pt_opts) else make_pt_opts(**(pt or {}))
        st = cinr_frame_stats()
        check(lib().cinr_render_frame_pt(self.h, cache.h if cache is not None else None, inr.h,
                                         C.byref(cam), C.byref(t), C.byref(o),
                                         C.c_void_p(out.data_ptr()), C.byref(st), _stream(stream)),
              "cinr_render_frame_pt")
        return out, st.as_dict()

    def set_macro(self, macro: Macro | None):
        """Attach macro cells (None detaches): transparent cells are skipped."""
        check(lib().cinr_renderer_set_macro(self.h, macro.h if macro is not None else None),
              "cinr_renderer_set_macro")
        self._macro = macro

    def __del__(self):
        try:
            if getattr(self, "h", None):
                lib().cinr_destroy_renderer(self.h)
                self.h = None
        except Exception:
            pass
