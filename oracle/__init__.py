"""CPU FP64 oracle of the cache-accelerated INR volume renderer.

TEST INFRASTRUCTURE ONLY: imported by tests/, ``__graft_entry__.smoke()`` and
the ``cpu_baseline`` / ``--impl reference`` legs of ``bench.py``; never by the
product path.  The arithmetic lives in ``cinr_oracle.c`` (plain C, FP64 for
values, binary32 without FMA contraction for every discrete decision); this
module only builds that library with gcc and marshals numpy arrays.

Pins (tests/test_oracle_pins.py) tie each function to something other than
itself: closed forms (constant-density slab, linear-field interpolation),
brute force on tiny grids (dense bijection, hash range), the paper's worked
brick-origin example (Sec. 4.3.2), a hand-computed MLP, finite differences
for the training gradient, and scripted cache scenarios checked by hand.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "cinr_oracle.c")
_HDR = os.path.join(_HERE, "cinr_oracle.h")
_BUILD = os.path.join(_HERE, "_build")
_LIB = os.path.join(_BUILD, "liboracle.so")
_lock = threading.Lock()
_lib = None

CFLAGS = ["-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math", "-fPIC",
          "-shared", "-Wall"]


def build(force: bool = False) -> str:
    """Compile liboracle.so with gcc (no GPU, no CUDA)."""
    os.makedirs(_BUILD, exist_ok=True)
    stale = (not os.path.exists(_LIB) or
             os.path.getmtime(_LIB) < max(os.path.getmtime(_SRC), os.path.getmtime(_HDR)))
    if force or stale:
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", *CFLAGS, "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


_SRC_OMP = os.path.join(_HERE, "cinr_oracle_omp.c")
_LIB_OMP = os.path.join(_BUILD, "liboracle_omp.so")
_lib_omp = None


def build_omp(force: bool = False) -> str:
    """Compile liboracle_omp.so: the same oracle source plus the row-parallel
    timing driver (cinr_oracle_omp.c), with -fopenmp.  Used only to time the
    oracle on all host cores; returns "" when gcc has no OpenMP."""
    os.makedirs(_BUILD, exist_ok=True)
    newest = max(os.path.getmtime(x) for x in (_SRC, _HDR, _SRC_OMP))
    if force or not os.path.exists(_LIB_OMP) or os.path.getmtime(_LIB_OMP) < newest:
        tmp = _LIB_OMP + f".tmp{os.getpid()}"
        r = subprocess.run(["gcc", *CFLAGS, "-fopenmp", "-o", tmp, _SRC, _SRC_OMP, "-lm"],
                           capture_output=True, text=True)
        if r.returncode != 0:
            return ""
        os.replace(tmp, _LIB_OMP)
    return _LIB_OMP


class InrParams(C.Structure):
    _fields_ = [("levels", C.c_int), ("feats", C.c_int), ("log2_table", C.c_int),
                ("base_res", C.c_int), ("growth", C.c_double), ("in_dim", C.c_int),
                ("hidden", C.c_int), ("n_hidden_layers", C.c_int),
                ("vmin", C.c_double), ("vmax", C.c_double)]


class Camera(C.Structure):
    _fields_ = [("eye", C.c_float * 3), ("target", C.c_float * 3), ("up", C.c_float * 3),
                ("fov_y_deg", C.c_float), ("width", C.c_int), ("height", C.c_int),
                ("step_voxels", C.c_float)]


class MarchOpts(C.Structure):
    _fields_ = [("K", C.c_int), ("eps_T", C.c_float), ("lod_mode", C.c_int),
                ("lod_scale", C.c_float), ("seed", C.c_uint64), ("step_mode", C.c_int),
                ("step_lod_max", C.c_int), ("macro", C.c_void_p)]


class PtOpts(C.Structure):
    _fields_ = [("light_dir", C.c_float * 3), ("light", C.c_float * 3), ("ambient", C.c_float * 3),
                ("max_bounces", C.c_int), ("sigma_max", C.c_float)]


class Macro(C.Structure):
    _fields_ = [("cell", C.c_int), ("dims", C.c_int * 3), ("skip", C.POINTER(C.c_uint8)),
                ("major", C.POINTER(C.c_float))]


class Stats(C.Structure):
    _fields_ = [(n, C.c_uint64) for n in (
        "samples", "inr_queries_direct", "inr_queries_decode", "true_misses",
        "fallback_hits", "hits", "bricks_requested", "bricks_decoded", "evictions",
        "samples_skipped")]

    def as_dict(self):
        return {n: int(getattr(self, n)) for n, _ in self._fields_}


class CacheOpts(C.Structure):
    _fields_ = [("brick", C.c_int), ("levels", C.c_int), ("n_slots", C.c_long),
                ("n_req", C.c_int), ("ranking", C.c_int), ("preload", C.c_int), ("lag", C.c_int),
                ("page", C.c_int), ("n_pages", C.c_long)]


_P = C.POINTER
_dp = _P(C.c_double)
_fp = _P(C.c_float)
_up = _P(C.c_uint32)
_ip = _P(C.c_int)

_SIGS = {
    "orc_splitmix64": (C.c_uint64, [C.c_uint64]),
    "orc_xorshift32": (C.c_uint32, [C.c_uint32]),
    "orc_uniform_coords": (None, [C.c_uint64, C.c_uint64, C.c_long, _fp]),
    "orc_mlp_param_count": (C.c_long, [_P(InrParams)]),
    "orc_level_res": (None, [_P(InrParams), _ip]),
    "orc_level_is_dense": (C.c_int, [_P(InrParams), C.c_int]),
    "orc_vertex_index": (C.c_uint32, [_P(InrParams), C.c_int, C.c_uint32, C.c_uint32, C.c_uint32]),
    "orc_encode_indices": (None, [_P(InrParams), _fp, C.c_long, _up]),
    "orc_encode": (None, [_P(InrParams), _dp, _fp, C.c_long, _dp]),
    "orc_mlp": (None, [_P(InrParams), _dp, _dp, C.c_long, _dp]),
    "orc_inr_eval": (None, [_P(InrParams), _dp, _dp, _fp, C.c_long, _dp]),
    "orc_inr_raw_range": (None, [_P(InrParams), _dp, _dp, _ip, C.c_int, _dp, _dp]),
    "orc_ray": (C.c_int, [_P(Camera), _ip, C.c_int, C.c_int, _fp, _fp, _fp, _fp]),
    "orc_sample": (C.c_int, [_P(Camera), _ip, _fp, _fp, C.c_float, C.c_float, C.c_int,
                             _fp, _fp, _fp]),
    "orc_sample_lod": (C.c_int, [_P(Camera), _ip, _P(MarchOpts), C.c_int, C.c_int,
                                 C.c_uint32, C.c_float]),
    "orc_frame_seed": (C.c_uint32, [C.c_uint64, C.c_uint64]),
    "orc_ray_seed": (C.c_uint32, [C.c_uint32, C.c_uint32]),
    "orc_sample_state": (C.c_uint32, [C.c_uint32, C.c_uint32]),
    "orc_tf_lookup": (None, [_dp, C.c_double, _dp]),
    "orc_render_direct": (None, [_P(InrParams), _dp, _dp, _P(Camera), _ip, _P(MarchOpts),
                                 _dp, C.c_int, C.c_int, C.c_int, C.c_int, _dp, _P(Stats)]),
    "orc_render_field": (None, [_fp, _ip, _P(Camera), _ip, _P(MarchOpts), _dp, C.c_int, C.c_int,
                                C.c_int, C.c_int, _dp, _P(Stats)]),
    "orc_cache_create": (C.c_void_p, [_P(InrParams), _dp, _dp, _ip, _P(CacheOpts),
                                      _P(MarchOpts)]),
    "orc_cache_destroy": (None, [C.c_void_p]),
    "orc_cache_num_bricks": (C.c_long, [C.c_void_p]),
    "orc_cache_level_offset": (C.c_long, [C.c_void_p, C.c_int]),
    "orc_cache_level_dims": (None, [C.c_void_p, C.c_int, _ip, _ip]),
    "orc_render_cached": (None, [C.c_void_p, _P(Camera), _dp, C.c_int, C.c_int, C.c_int,
                                 C.c_int, _dp, _P(Stats)]),
    "orc_cache_dump": (C.c_long, [C.c_void_p, C.c_int, _up, C.c_long]),
    "orc_cache_slot_values": (None, [C.c_void_p, C.c_long, _dp]),
    "orc_brick_values": (None, [_P(InrParams), _dp, _dp, _ip, C.c_int, C.c_int, C.c_int,
                                C.c_int, C.c_int, _dp]),
    "orc_brick_origin": (None, [_ip, C.c_int, C.c_int, C.c_int, C.c_int, C.c_int, _dp]),
    "orc_resident_sample": (C.c_double, [_P(InrParams), _dp, _dp, _ip, C.c_int, _fp]),
    "orc_brick_sample": (C.c_double, [_P(InrParams), _dp, _dp, _ip, C.c_int, C.c_int, _fp]),
    "orc_psnr": (C.c_double, [_dp, _dp, C.c_long]),
    "orc_macro_dims": (None, [_ip, C.c_int, _ip]),
    "orc_macro_ranges_inr": (None, [_P(InrParams), _dp, _dp, _ip, C.c_int, C.c_int, C.c_int,
                                    _fp]),
    "orc_macro_ranges_field": (None, [_fp, _ip, C.c_int, _fp]),
    "orc_macro_skip": (None, [_fp, C.c_long, _dp, _P(C.c_uint8)]),
    "orc_macro_majorant": (None, [_fp, C.c_long, _dp, _fp]),
    "orc_pt_walk_test": (C.c_int, [C.c_void_p, _ip, _fp, _fp, C.c_float, C.c_float, _fp, C.c_int,
                                   _fp, _fp]),
    "orc_macro_cell_of": (C.c_long, [_P(Macro), _ip, _fp]),
    "orc_cache_set_macro": (None, [C.c_void_p, C.c_void_p]),
    "orc_neg_log1m": (C.c_float, [C.c_float]),
    "orc_pt_uniform": (C.c_float, [C.c_uint64, C.c_uint32]),
    "orc_pt_sphere": (None, [C.c_uint64, _up, _fp]),
    "orc_render_pt_direct": (None, [_P(InrParams), _dp, _dp, _P(Camera), _ip, _P(MarchOpts), _dp,
                                    _P(PtOpts), C.c_uint64, C.c_int, C.c_int, C.c_int, C.c_int,
                                    _dp, _P(Stats)]),
    "orc_render_pt_cached": (None, [C.c_void_p, _P(Camera), _dp, _P(PtOpts), C.c_int, C.c_int,
                                    C.c_int, C.c_int, _dp, _P(Stats)]),
    "orc_field_trilinear": (C.c_double, [_fp, _ip, _fp]),
    "orc_loss_grad": (C.c_double, [_P(InrParams), _dp, _dp, _fp, _dp, C.c_long, _dp, _dp]),
    "orc_adam": (None, [_dp, _dp, _dp, _dp, C.c_long, C.c_double, C.c_double, C.c_double,
                        C.c_double, C.c_long]),
    "orc_train_step": (C.c_double, [_P(InrParams), _dp, _dp, _dp, _dp, _dp, _dp, _fp, _ip,
                                    C.c_double, C.c_double, C.c_long, C.c_uint64, C.c_long,
                                    C.c_double, C.c_double, C.c_double, C.c_double]),
}


def lib():
    global _lib
    with _lock:
        if _lib is None:
            path = build()
            L = C.CDLL(path)
            for name, (res, args) in _SIGS.items():
                fn = getattr(L, name)
                fn.restype = res
                fn.argtypes = args
            _lib = L
    return _lib


def lib_omp():
    """The OpenMP build (None when it cannot be built)."""
    global _lib_omp
    with _lock:
        if _lib_omp is None:
            path = build_omp()
            if not path:
                return None
            L = C.CDLL(path)
            L.orc_omp_threads.restype = C.c_int
            L.orc_omp_threads.argtypes = []
            L.orc_render_direct_rows.restype = None
            L.orc_render_direct_rows.argtypes = _SIGS["orc_render_direct"][1]
            L.orc_render_direct_pixels.restype = None
            L.orc_render_direct_pixels.argtypes = [
                _P(InrParams), _dp, _dp, _P(Camera), _ip, _P(MarchOpts), _dp, _ip, _ip, C.c_long,
                _dp, _P(Stats)]
            _lib_omp = L
    return _lib_omp


def omp_threads() -> int:
    L = lib_omp()
    return int(L.orc_omp_threads()) if L is not None else 1


def render_direct_rows(p, table, w, cam, vol, mo, tf, window=None):
    """render_direct with the window's rows spread over all host cores (the
    same per-pixel arithmetic; falls back to one thread without OpenMP)."""
    L = lib_omp()
    if L is None:
        return render_direct(p, table, w, cam, vol, mo, tf, window)
    px0, py0, pw, ph = window if window is not None else (0, 0, cam.width, cam.height)
    t, tp = _d(table)
    wa, wp = _d(w)
    v, vp = _i3(vol)
    tfa, tfp = _d(tf)
    out = np.zeros((ph, pw, 4), np.float64)
    st = Stats()
    L.orc_render_direct_rows(C.byref(p), tp, wp, C.byref(cam), vp, C.byref(mo), tfp,
                             px0, py0, pw, ph, out.ctypes.data_as(_dp), C.byref(st))
    return out, st.as_dict()


def render_direct_pixels(p, table, w, cam, vol, mo, tf, px, py):
    """Cache-off render of scattered pixels (px[i], py[i]) on all host cores
    (one thread without OpenMP); returns (rgba[n, 4], stats)."""
    px = np.ascontiguousarray(px, np.int32)
    py = np.ascontiguousarray(py, np.int32)
    n = len(px)
    out = np.zeros((n, 4), np.float64)
    L = lib_omp()
    if L is None:
        st = {}
        for i in range(n):
            o, s1 = render_direct(p, table, w, cam, vol, mo, tf, (int(px[i]), int(py[i]), 1, 1))
            out[i] = o[0, 0]
            for k, v in s1.items():
                st[k] = st.get(k, 0) + v
        return out, st
    t, tp = _d(table)
    wa, wp = _d(w)
    v, vp = _i3(vol)
    tfa, tfp = _d(tf)
    st = Stats()
    L.orc_render_direct_pixels(C.byref(p), tp, wp, C.byref(cam), vp, C.byref(mo), tfp,
                               px.ctypes.data_as(_ip), py.ctypes.data_as(_ip), n,
                               out.ctypes.data_as(_dp), C.byref(st))
    return out, st.as_dict()


# ----------------------------------------------------------------- helpers
def _d(a):
    a = np.ascontiguousarray(a, dtype=np.float64)
    return a, a.ctypes.data_as(_dp)


def _f(a):
    a = np.ascontiguousarray(a, dtype=np.float32)
    return a, a.ctypes.data_as(_fp)


def _i3(v):
    a = np.ascontiguousarray(np.asarray(v, dtype=np.int32).reshape(3))
    return a, a.ctypes.data_as(_ip)


def inr_params(levels, feats, log2_table, base_res, growth, hidden,
               n_hidden_layers=2, vmin=0.0, vmax=1.0) -> InrParams:
    return InrParams(levels, feats, log2_table, base_res, float(growth), levels * feats,
                     hidden, n_hidden_layers, float(vmin), float(vmax))


def camera(eye, target, up, fov_y_deg, width, height, step_voxels) -> Camera:
    c = Camera()
    c.eye[:] = [float(v) for v in eye]
    c.target[:] = [float(v) for v in target]
    c.up[:] = [float(v) for v in up]
    c.fov_y_deg, c.width, c.height, c.step_voxels = float(fov_y_deg), int(width), int(height), float(step_voxels)
    return c


def march_opts(K=32, eps_T=1e-3, lod_mode=0, lod_scale=1.0, seed=0, step_mode=0,
               step_lod_max=0, macro=None) -> MarchOpts:
    mo = MarchOpts(int(K), float(eps_T), int(lod_mode), float(lod_scale), int(seed),
                   int(step_mode), int(step_lod_max), None)
    if macro is not None:
        mo.macro = C.cast(C.pointer(macro), C.c_void_p)
        mo._keep = macro
    return mo


# ----------------------------------------------------------- path tracing
def pt_opts(light_dir=(0.3, -1.0, -0.4), light=(3.0, 3.0, 3.0), ambient=(0.0, 0.0, 0.0),
            max_bounces=3, sigma_max=0.0) -> PtOpts:
    return PtOpts((C.c_float * 3)(*light_dir), (C.c_float * 3)(*light), (C.c_float * 3)(*ambient),
                  int(max_bounces), float(sigma_max))


def neg_log1m(u: float) -> float:
    return float(lib().orc_neg_log1m(float(u)))


def pt_uniform(key: int, j: int) -> float:
    return float(lib().orc_pt_uniform(C.c_uint64(key & (2**64 - 1)), j))


def pt_sphere(key: int, j: int):
    jj = C.c_uint32(j)
    d = np.zeros(3, np.float32)
    lib().orc_pt_sphere(C.c_uint64(key & (2**64 - 1)), C.byref(jj), d.ctypes.data_as(_fp))
    return d, int(jj.value)


def render_pt_direct(p: InrParams, table, w, cam: Camera, vol, mo: MarchOpts, tf, pt: PtOpts,
                     frame, window=None):
    """One path per pixel, every density lookup by direct INR inference."""
    px0, py0, pw, ph = window if window is not None else (0, 0, cam.width, cam.height)
    t, tp = _d(table)
    wa, wp = _d(w)
    v, vp = _i3(vol)
    tfa, tfp = _d(tf)
    out = np.zeros((ph, pw, 4), np.float64)
    st = Stats()
    lib().orc_render_pt_direct(C.byref(p), tp, wp, C.byref(cam), vp, C.byref(mo), tfp,
                               C.byref(pt), int(frame), px0, py0, pw, ph,
                               out.ctypes.data_as(_dp), C.byref(st))
    return out, st.as_dict()


# ------------------------------------------------------------- macro cells
def macro_dims(vol, cell):
    v, vp = _i3(vol)
    out = np.zeros(3, np.int32)
    lib().orc_macro_dims(vp, int(cell), out.ctypes.data_as(_ip))
    return tuple(int(a) for a in out)


def macro_ranges_inr(p: InrParams, table, w, vol, cell, levels, min_level=0):
    """Per-cell (min, max) over the cache's LoD voxels; float32 [cells, 2]."""
    t, tp = _d(table)
    wa, wp = _d(w)
    v, vp = _i3(vol)
    n = int(np.prod(macro_dims(vol, cell)))
    out = np.zeros((n, 2), np.float32)
    lib().orc_macro_ranges_inr(C.byref(p), tp, wp, vp, int(cell), int(levels), int(min_level),
                               out.ctypes.data_as(_fp))
    return out


def macro_ranges_field(field, cell):
    """Per-cell (min, max) of an explicit field [z, y, x]; float32 [cells, 2]."""
    fa, fp = _f(field)
    fd, fdp = _i3(fa.shape[::-1])
    n = int(np.prod(macro_dims(fa.shape[::-1], cell)))
    out = np.zeros((n, 2), np.float32)
    lib().orc_macro_ranges_field(fp, fdp, int(cell), out.ctypes.data_as(_fp))
    return out


def macro_skip(ranges, tf):
    r, rp = _f(ranges)
    tfa, tfp = _d(tf)
    n = r.size // 2
    out = np.zeros(n, np.uint8)
    lib().orc_macro_skip(rp, n, tfp, out.ctypes.data_as(C.POINTER(C.c_uint8)))
    return out


def macro_majorant(ranges, tf):
    """Per-cell extinction majorant under tf (0 exactly where the skip rule
    marks the cell transparent); float32 [cells]."""
    r, rp = _f(ranges)
    tfa, tfp = _d(tf)
    n = r.size // 2
    out = np.zeros(n, np.float32)
    lib().orc_macro_majorant(rp, n, tfp, out.ctypes.data_as(_fp))
    return out


def macro(vol, cell, skip, major=None) -> Macro:
    """Macro-cell structure for march_opts(macro=...) / Cache.render(macro=...)
    / Cache.render_pt(macro=...): skip flags, and per-cell majorants (or None)
    for the path tracer's local-majorant tracking."""
    sk = np.ascontiguousarray(skip, dtype=np.uint8)
    mj = None if major is None else np.ascontiguousarray(major, dtype=np.float32)
    m = Macro(int(cell), (C.c_int * 3)(*macro_dims(vol, cell)),
              sk.ctypes.data_as(C.POINTER(C.c_uint8)),
              mj.ctypes.data_as(C.POINTER(C.c_float)) if mj is not None else None)
    m.skip_flags, m.majorants = sk, mj  # the arrays the structure points to
    return m


def pt_walk_test(m: Macro, vol, o, d, t0, t1, taus):
    """Tentative collisions (t, majorant) of successive free flights of
    optical depths taus along o + t d through the cells' majorants."""
    v, vp = _i3(vol)
    oa, op = _f(np.asarray(o, np.float32).reshape(3))
    da, dp = _f(np.asarray(d, np.float32).reshape(3))
    ta, tp = _f(np.asarray(taus, np.float32).reshape(-1))
    tout = np.zeros(ta.size, np.float32)
    mout = np.zeros(ta.size, np.float32)
    n = lib().orc_pt_walk_test(C.cast(C.pointer(m), C.c_void_p), vp, op, dp, float(t0), float(t1), tp,
                               ta.size, tout.ctypes.data_as(_fp), mout.ctypes.data_as(_fp))
    return tout[:n], mout[:n]


def macro_cell_of(m: Macro, vol, x):
    v, vp = _i3(vol)
    xa, xp = _f(np.asarray(x, np.float32).reshape(3))
    return int(lib().orc_macro_cell_of(C.byref(m), vp, xp))


def splitmix64(x: int) -> int:
    return int(lib().orc_splitmix64(C.c_uint64(x & (2**64 - 1))))


def xorshift32(s: int) -> int:
    return int(lib().orc_xorshift32(C.c_uint32(s & 0xFFFFFFFF)))


def uniform_coords(seed: int, first: int, n: int) -> np.ndarray:
    out = np.zeros((n, 3), np.float32)
    lib().orc_uniform_coords(seed, first, n, out.ctypes.data_as(_fp))
    return out


def level_res(p: InrParams) -> np.ndarray:
    out = np.zeros(p.levels, np.int32)
    lib().orc_level_res(C.byref(p), out.ctypes.data_as(_ip))
    return out


def level_is_dense(p: InrParams, level: int) -> bool:
    return bool(lib().orc_level_is_dense(C.byref(p), level))


def vertex_index(p: InrParams, level: int, ix: int, iy: int, iz: int) -> int:
    return int(lib().orc_vertex_index(C.byref(p), level, ix, iy, iz))


def encode_indices(p: InrParams, xyz) -> np.ndarray:
    x, xp = _f(xyz)
    n = x.shape[0]
    out = np.zeros((n, p.levels, 8), np.uint32)
    lib().orc_encode_indices(C.byref(p), xp, n, out.ctypes.data_as(_up))
    return out


def encode(p: InrParams, table, xyz) -> np.ndarray:
    t, tp = _d(table)
    x, xp = _f(xyz)
    n = x.shape[0]
    out = np.zeros((n, p.in_dim), np.float64)
    lib().orc_encode(C.byref(p), tp, xp, n, out.ctypes.data_as(_dp))
    return out


def mlp(p: InrParams, w, feats) -> np.ndarray:
    wa, wp = _d(w)
    fa, fp = _d(feats)
    n = fa.shape[0]
    out = np.zeros(n, np.float64)
    lib().orc_mlp(C.byref(p), wp, fp, n, out.ctypes.data_as(_dp))
    return out


def inr_eval(p: InrParams, table, w, xyz) -> np.ndarray:
    t, tp = _d(table)
    wa, wp = _d(w)
    x, xp = _f(xyz)
    n = x.shape[0]
    out = np.zeros(n, np.float64)
    lib().orc_inr_eval(C.byref(p), tp, wp, xp, n, out.ctypes.data_as(_dp))
    return out


def inr_raw_range(p: InrParams, table, w, vol, stride):
    t, tp = _d(table)
    wa, wp = _d(w)
    v, vp = _i3(vol)
    lo, hi = C.c_double(), C.c_double()
    lib().orc_inr_raw_range(C.byref(p), tp, wp, vp, int(stride), C.byref(lo), C.byref(hi))
    return lo.value, hi.value


def ray(cam: Camera, vol, px, py):
    v, vp = _i3(vol)
    o = np.zeros(3, np.float32)
    d = np.zeros(3, np.float32)
    tn, tf = C.c_float(), C.c_float()
    hit = lib().orc_ray(C.byref(cam), vp, px, py, o.ctypes.data_as(_fp), d.ctypes.data_as(_fp),
                        C.byref(tn), C.byref(tf))
    return bool(hit), o, d, tn.value, tf.value


def sample(cam: Camera, vol, o, d, tn, tf, k):
    v, vp = _i3(vol)
    oa, op = _f(o)
    da, dp = _f(d)
    x = np.zeros(3, np.float32)
    tm, ln = C.c_float(), C.c_float()
    ok = lib().orc_sample(C.byref(cam), vp, op, dp, tn, tf, k, x.ctypes.data_as(_fp),
                          C.byref(tm), C.byref(ln))
    return bool(ok), x, tm.value, ln.value


def sample_lod(cam: Camera, vol, mo: MarchOpts, levels, lod_min, state, t_mid):
    v, vp = _i3(vol)
    return int(lib().orc_sample_lod(C.byref(cam), vp, C.byref(mo), levels, lod_min,
                                    state & 0xFFFFFFFF, t_mid))


def frame_seed(seed: int, frame: int) -> int:
    return int(lib().orc_frame_seed(seed, frame))


def ray_seed(fseed: int, pixel: int) -> int:
    return int(lib().orc_ray_seed(fseed & 0xFFFFFFFF, pixel & 0xFFFFFFFF))


def ray_states(fseed: int, pixel: int, n: int):
    """Dither states of samples 0..n-1 of a ray."""
    rs = ray_seed(fseed, pixel)
    return [int(lib().orc_sample_state(rs, k)) for k in range(n)]


def tf_lookup(tf, v):
    t, tp = _d(tf)
    out = np.zeros(4, np.float64)
    lib().orc_tf_lookup(tp, float(v), out.ctypes.data_as(_dp))
    return out


def render_direct(p: InrParams, table, w, cam: Camera, vol, mo: MarchOpts, tf,
                  window=None):
    """Cache-off render; returns (rgba[ph, pw, 4] float64, stats dict)."""
    px0, py0, pw, ph = window if window is not None else (0, 0, cam.width, cam.height)
    t, tp = _d(table)
    wa, wp = _d(w)
    v, vp = _i3(vol)
    tfa, tfp = _d(tf)
    out = np.zeros((ph, pw, 4), np.float64)
    st = Stats()
    lib().orc_render_direct(C.byref(p), tp, wp, C.byref(cam), vp, C.byref(mo), tfp,
                            px0, py0, pw, ph, out.ctypes.data_as(_dp), C.byref(st))
    return out, st.as_dict()


def render_field(field, cam: Camera, vol, mo: MarchOpts, tf, window=None):
    """Explicit-voxel render of field [z, y, x]; returns (rgba, stats)."""
    px0, py0, pw, ph = window if window is not None else (0, 0, cam.width, cam.height)
    fa, fp = _f(field)
    fd, fdp = _i3(fa.shape[::-1])
    v, vp = _i3(vol)
    tfa, tfp = _d(tf)
    out = np.zeros((ph, pw, 4), np.float64)
    st = Stats()
    lib().orc_render_field(fp, fdp, C.byref(cam), vp, C.byref(mo), tfp, px0, py0, pw, ph,
                           out.ctypes.data_as(_dp), C.byref(st))
    return out, st.as_dict()


DUMP_PT, DUMP_STAMP, DUMP_OWNER, DUMP_RANK, DUMP_REQ, DUMP_VICT, DUMP_MISS, DUMP_PINNED = range(8)
DUMP_PAGE_DIR, DUMP_PAGES, DUMP_PAGE_KEY, DUMP_PAGE_REF = range(8, 12)


class Cache:
    """Oracle brick cache (owns its own host memory)."""

    def __init__(self, p: InrParams, table, w, vol, brick, levels, n_slots, mo: MarchOpts,
                 n_req=40, ranking=1, preload=1, lag=1, page=0, n_pages=0):
        self._t, tp = _d(table)
        self._w, wp = _d(w)
        self._v, vp = _i3(vol)
        self.p = p
        self.mo = mo
        self.co = CacheOpts(int(brick), int(levels), int(n_slots), int(n_req), int(ranking),
                            int(preload), int(lag), int(page), int(n_pages))
        h = lib().orc_cache_create(C.byref(p), tp, wp, vp, C.byref(self.co), C.byref(mo))
        if not h:
            raise ValueError("orc_cache_create failed (levels or pool too small for preload)")
        self.h = C.c_void_p(h)

    def close(self):
        if self.h:
            lib().orc_cache_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @property
    def n_bricks(self):
        return int(lib().orc_cache_num_bricks(self.h))

    def level_offset(self, level):
        return int(lib().orc_cache_level_offset(self.h, level))

    def level_dims(self, level):
        d = np.zeros(3, np.int32)
        nb = np.zeros(3, np.int32)
        lib().orc_cache_level_dims(self.h, level, d.ctypes.data_as(_ip), nb.ctypes.data_as(_ip))
        return d, nb

    def render(self, cam: Camera, tf, window=None, macro=None):
        """One cached frame; macro = skip flags of this frame's TF (or None)."""
        px0, py0, pw, ph = window if window is not None else (0, 0, cam.width, cam.height)
        tfa, tfp = _d(tf)
        out = np.zeros((ph, pw, 4), np.float64)
        st = Stats()
        lib().orc_cache_set_macro(self.h, C.cast(C.pointer(macro), C.c_void_p) if macro else None)
        try:
            lib().orc_render_cached(self.h, C.byref(cam), tfp, px0, py0, pw, ph,
                                    out.ctypes.data_as(_dp), C.byref(st))
        finally:
            lib().orc_cache_set_macro(self.h, None)
        return out, st.as_dict()

    def render_pt(self, cam: Camera, tf, pt: PtOpts, window=None, macro=None):
        """One path-traced frame through the cache; macro with majorants
        switches delta and ratio tracking to the cells' local majorants."""
        px0, py0, pw, ph = window if window is not None else (0, 0, cam.width, cam.height)
        tfa, tfp = _d(tf)
        out = np.zeros((ph, pw, 4), np.float64)
        st = Stats()
        lib().orc_cache_set_macro(self.h, C.cast(C.pointer(macro), C.c_void_p) if macro else None)
        try:
            lib().orc_render_pt_cached(self.h, C.byref(cam), tfp, C.byref(pt), px0, py0, pw, ph,
                                       out.ctypes.data_as(_dp), C.byref(st))
        finally:
            lib().orc_cache_set_macro(self.h, None)
        return out, st.as_dict()

    def dump(self, what):
        n = int(lib().orc_cache_dump(self.h, what, None, 0))
        out = np.zeros(max(n, 0), np.uint32)
        if n > 0:
            lib().orc_cache_dump(self.h, what, out.ctypes.data_as(_up), n)
        return out

    def slot_values(self, slot):
        S = self.co.brick + 2
        out = np.zeros(S ** 3, np.float64)
        lib().orc_cache_slot_values(self.h, slot, out.ctypes.data_as(_dp))
        return out


def brick_values(p: InrParams, table, w, vol, brick, level, b):
    t, tp = _d(table)
    wa, wp = _d(w)
    v, vp = _i3(vol)
    S = brick + 2
    out = np.zeros(S ** 3, np.float64)
    lib().orc_brick_values(C.byref(p), tp, wp, vp, brick, level, int(b[0]), int(b[1]), int(b[2]),
                           out.ctypes.data_as(_dp))
    return out.reshape(S, S, S)


def brick_origin(vol, brick, level, b):
    v, vp = _i3(vol)
    out = np.zeros(3, np.float64)
    lib().orc_brick_origin(vp, brick, level, int(b[0]), int(b[1]), int(b[2]),
                           out.ctypes.data_as(_dp))
    return out


def resident_sample(p: InrParams, table, w, vol, level, x):
    t, tp = _d(table)
    wa, wp = _d(w)
    v, vp = _i3(vol)
    xa, xp = _f(x)
    return float(lib().orc_resident_sample(C.byref(p), tp, wp, vp, level, xp))


def brick_sample(p: InrParams, table, w, vol, brick, level, x):
    t, tp = _d(table)
    wa, wp = _d(w)
    v, vp = _i3(vol)
    xa, xp = _f(x)
    return float(lib().orc_brick_sample(C.byref(p), tp, wp, vp, brick, level, xp))


def psnr(a, b):
    aa, ap = _d(a)
    ba, bp = _d(b)
    n = aa.size // 4
    return float(lib().orc_psnr(ap, bp, n))


def field_trilinear(field, x):
    fa, fp = _f(field)
    dims, dp = _i3(fa.shape[::-1])
    xa, xp = _f(x)
    return float(lib().orc_field_trilinear(fp, dp, xp))


def loss_grad(p: InrParams, table, w, xyz, target):
    t, tp = _d(table)
    wa, wp = _d(w)
    x, xp = _f(xyz)
    tg, tgp = _d(target)
    gt = np.zeros_like(t)
    gw = np.zeros_like(wa)
    loss = lib().orc_loss_grad(C.byref(p), tp, wp, xp, tgp, x.shape[0],
                               gt.ctypes.data_as(_dp), gw.ctypes.data_as(_dp))
    return float(loss), gt, gw


class Trainer:
    """FP64 Adam training state (Sec. 4.1); arrays are updated in place."""

    def __init__(self, p: InrParams, table, w, field, fmin, fmax, batch, seed,
                 lr=1e-2, b1=0.9, b2=0.99, eps=1e-15):
        self.p = p
        self.table = np.array(table, dtype=np.float64)
        self.w = np.array(w, dtype=np.float64)
        self.m_t = np.zeros_like(self.table)
        self.v_t = np.zeros_like(self.table)
        self.m_w = np.zeros_like(self.w)
        self.v_w = np.zeros_like(self.w)
        self.field = np.ascontiguousarray(field, dtype=np.float32)
        self.dims = np.ascontiguousarray(np.array(self.field.shape[::-1], np.int32))
        self.fmin, self.fmax = float(fmin), float(fmax)
        self.batch, self.seed = int(batch), int(seed)
        self.lr, self.b1, self.b2, self.eps = lr, b1, b2, eps
        self.step_no = 0

    def step(self) -> float:
        self.step_no += 1
        return float(lib().orc_train_step(
            C.byref(self.p), self.table.ctypes.data_as(_dp), self.w.ctypes.data_as(_dp),
            self.m_t.ctypes.data_as(_dp), self.v_t.ctypes.data_as(_dp),
            self.m_w.ctypes.data_as(_dp), self.v_w.ctypes.data_as(_dp),
            self.field.ctypes.data_as(_fp), self.dims.ctypes.data_as(_ip), self.fmin, self.fmax,
            self.batch, self.seed, self.step_no, self.lr, self.b1, self.b2, self.eps))
