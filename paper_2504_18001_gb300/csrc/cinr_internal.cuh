// Internal definitions of the GB300 INR renderer library (not part of the
// C ABI).  Device structs are passed to kernels by value.
//
// Numeric contract of the discrete decisions: every quantity that feeds a
// floor, a comparison or a hash (ray direction, sample parameter, positions,
// grid coordinates) is computed with explicitly rounded binary32 intrinsics
// (__fmul_rn, __fadd_rn, __fdiv_rn, __fsqrt_rn), never contracted into FMAs,
// in a fixed operation order, so that LoD, brick, hash index and hit/miss
// decisions are reproducible on any IEEE binary32 implementation.
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <string>

#include "cinr.h"

namespace cinr {

constexpr int kMaxLevels = 32;    // hash-grid levels
constexpr int kMaxLod = 12;       // cache LoDs
constexpr uint32_t kMapped = 0x80000000u;
constexpr uint32_t kNoOwner = 0xFFFFFFFFu;
constexpr int kFrameThreads = 128;  // 4 warps per CTA in the frame kernel

// ------------------------------------------------ device bounds checks
// A library built with -DCINR_CHECK=1 checks every page-table, page,
// slot, pool and hash-table index before the access it guards: an index out
// of range sets kErrCheck in the kernel's error word (reported on the host
// as CINR_ERR_DEVICE_CHECK) and the access is skipped.  The default build
// compiles the checks away.
#ifndef CINR_CHECK
#define CINR_CHECK 0
#endif
constexpr int kErrTimeout = 1;  // a bounded device-side wait gave up
constexpr int kErrCheck = 2;    // a device bounds check tripped

// Whether i < n; in a checked build an index out of range sets kErrCheck
// in *err (when err is not null).
__device__ __forceinline__ bool in_range(unsigned long long i, unsigned long long n, int* err) {
#if CINR_CHECK
  if (i >= n) {
    if (err) atomicOr(err, kErrCheck);
    return false;
  }
#else
  (void)i;
  (void)n;
  (void)err;
#endif
  return true;
}

// Host side: the status code of a device error word.
inline int device_status(int word) {
  if (word & kErrCheck) return CINR_ERR_DEVICE_CHECK;
  if (word) return CINR_ERR_TIMEOUT;
  return CINR_OK;
}

// ---------------------------------------------------------------- errors
int set_error(int code, const char* fmt, ...);
int cuda_error(cudaError_t e, const char* what);
#define CINR_CK(call)                                   \
  do {                                                  \
    cudaError_t e_ = (call);                            \
    if (e_ != cudaSuccess) return cuda_error(e_, #call); \
  } while (0)

inline size_t align_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

// Bump allocator over a caller-provided device buffer (no device allocation).
struct Carver {
  char* base;
  size_t off = 0;
  explicit Carver(void* b) : base(static_cast<char*>(b)) {}
  template <typename T>
  T* take(size_t count, size_t align = 256) {
    off = align_up(off, align);
    T* p = base ? reinterpret_cast<T*>(base + off) : nullptr;
    off += sizeof(T) * count;
    return p;
  }
};

// ------------------------------------------------------------ device INR
struct InrDev {
  const void* table;   // levels * T * 2 entries, float or half
  const float* w;      // fp32 weights, layer-major [out][in]
  int L, log2T;
  int res[kMaxLevels];
  uint32_t dense_mask;
  int IN, H, NH;
  int table_prec;
  float vmin, vscale;  // v = vmin + vscale * y
  int* err;            // error word of the bounds checks (checked builds)
};

// Camera and marching constants, computed on the host in binary32.
struct CamDev {
  float o[3], fwd[3], right[3], upv[3];
  float ax, ay;        // tan(fov/2) * aspect, tan(fov/2)
  int W, H;
  float e[3], h[3];    // box extent and half extent
  float inv_e[3];      // 1 / e (binary32): normalised coordinate = (p + h) * inv_e
  float dt;            // step in world units
  float lodc;          // footprint constant: t * lodc = pixel footprint in LoD-0 voxels
  float lod_scale;
  int lod_mode;
  int vol[3];
  int step_mode;       // 0 fixed step, 1 LoD-scaled 32-sample segments
  int step_lod_max;
};

// Sample schedule state of a ray under step_mode 1.
struct Sched {
  float ts, dts;  // segment start, step
};

struct CacheDev {
  int vol[3];
  uint32_t* pt;
  uint32_t* rank;
  uint32_t* stamp;
  uint32_t* owner;
  uint32_t* pinned;
  void* pool;
  int pool_prec;
  int B, S, L;
  float invB;  // 1/B when B is a power of two (exact), else 0
  int dims[kMaxLod][3];
  int nb[kMaxLod][3];
  uint32_t off[kMaxLod + 1];
  uint32_t* touched;
  uint32_t* touched_count;
  // virtualised page tables (pd != nullptr; pt is then unused): per-LoD
  // page directory over pages of 2^page_shift bricks per axis, page pool,
  // page slot keys and refcounts
  uint32_t* pd;
  uint32_t* pages;
  uint32_t* page_key;
  uint32_t* page_ref;
  int page_shift;
  int pg[kMaxLod][3];
  uint32_t pd_off[kMaxLod + 1];
  uint32_t n_pages;
  uint32_t n_slots, n_bricks;
  int* err;  // error word of the bounds checks (checked builds)
  int dec_staged;  // brick decode: 1 staged tile encoder, 0 per-voxel gathers
  // texture layout of an FP16 pool (pool_tex != 0): slice z of slot s is
  // block b = s S + z at texels (x + S (b & (2^tex_shift - 1)),
  // y + S (b >> tex_shift)) of a 2D image with tex_pitch texels per row
  int pool_tex;
  int tex_shift;
  int tex_pitch;
  unsigned long long tex;  // cudaTextureObject_t over the pool
};

// Offset of voxel (x, y, z) of slot s in a pool in the texture layout.
__host__ __device__ __forceinline__ size_t tex_offset(int S, int shift, int pitch, uint32_t s, int x, int y,
                                                      int z) {
  const uint32_t b = s * (uint32_t)S + (uint32_t)z;
  const uint32_t bc = b & ((1u << shift) - 1u), br = b >> shift;
  return ((size_t)br * S + y) * (size_t)pitch + (size_t)bc * S + x;
}

// Page-table entry of brick (b0, b1, b2) at LoD lev (key = its flat key):
// the flat table, or the entry in its page when the page is resident.
// In a checked build an entry whose slot lies beyond the pool, or a key or
// page out of range, reads as Unmapped after setting the error word.
__device__ __forceinline__ uint32_t pt_entry(const CacheDev& c, int lev, uint32_t key, int b0, int b1,
                                             int b2) {
  if (!c.pd) {
    if (!in_range(key, c.n_bricks, c.err)) return 0u;
    const uint32_t e = __ldg(c.pt + key);
    return (!(e & kMapped) || in_range(e & ~kMapped, c.n_slots, c.err)) ? e : 0u;
  }
  const int sh = c.page_shift, m = (1 << sh) - 1;
  const uint32_t pk = c.pd_off[lev] + (uint32_t)(b0 >> sh) +
                      (uint32_t)c.pg[lev][0] * ((uint32_t)(b1 >> sh) + (uint32_t)c.pg[lev][1] * (uint32_t)(b2 >> sh));
  if (!in_range(pk, c.pd_off[c.L], c.err)) return 0u;
  const uint32_t e = __ldg(c.pd + pk);
  if (!(e & kMapped)) return 0u;
  if (!in_range(e & ~kMapped, c.n_pages, c.err)) return 0u;
  const uint32_t local = (uint32_t)(b0 & m) + ((uint32_t)(b1 & m) << sh) + ((uint32_t)(b2 & m) << (2 * sh));
  const uint32_t be = __ldg(c.pages + (((size_t)(e & ~kMapped)) << (3 * sh)) + local);
  return (!(be & kMapped) || in_range(be & ~kMapped, c.n_slots, c.err)) ? be : 0u;
}

// Appends a brick first requested this frame to the touched list.
__device__ __forceinline__ void push_touched(const CacheDev& c, uint32_t key) {
  const uint32_t i = atomicAdd(c.touched_count, 1u);
  if (in_range(i, c.n_bricks, c.err)) c.touched[i] = key;
}

// Level and brick coordinates of a flat brick key.
__device__ __forceinline__ int key_brick(const CacheDev& c, uint32_t key, int b[3]) {
  int l = 0;
  while (l + 1 < c.L && key >= c.off[l + 1]) ++l;
  const uint32_t loc = key - c.off[l];
  b[0] = (int)(loc % (uint32_t)c.nb[l][0]);
  b[1] = (int)((loc / (uint32_t)c.nb[l][0]) % (uint32_t)c.nb[l][1]);
  b[2] = (int)(loc / ((uint32_t)c.nb[l][0] * (uint32_t)c.nb[l][1]));
  return l;
}

// Page key and in-page index of a brick key (paged tables).
__device__ __forceinline__ uint32_t key_page(const CacheDev& c, uint32_t key, uint32_t& local) {
  int b[3];
  const int l = key_brick(c, key, b);
  const int sh = c.page_shift, m = (1 << sh) - 1;
  local = (uint32_t)(b[0] & m) + ((uint32_t)(b[1] & m) << sh) + ((uint32_t)(b[2] & m) << (2 * sh));
  return c.pd_off[l] + (uint32_t)(b[0] >> sh) +
         (uint32_t)c.pg[l][0] * ((uint32_t)(b[1] >> sh) + (uint32_t)c.pg[l][1] * (uint32_t)(b[2] >> sh));
}

__device__ __forceinline__ uint32_t pt_entry_key(const CacheDev& c, uint32_t key) {
  if (!in_range(key, c.n_bricks, c.err)) return 0u;
  if (!c.pd) return c.pt[key];
  uint32_t local;
  const uint32_t pk = key_page(c, key, local);
  const uint32_t e = c.pd[pk];
  if (!(e & kMapped)) return 0u;
  if (!in_range(e & ~kMapped, c.n_pages, c.err)) return 0u;
  return c.pages[(((size_t)(e & ~kMapped)) << (3 * c.page_shift)) + local];
}

// Macro-cell skip flags of the current transfer function (Sec. 5.2);
// skip == nullptr turns skipping off.  Cells are 2^shift LoD-0 voxels wide.
struct MacroDev {
  const uint8_t* skip;
  const float* major;  // per-cell extinction majorant (path tracing); nullptr: global
  int shift;
  int dims[3];
};

// ------------------------------------------------- binary32 primitives
__device__ __forceinline__ float f_mul(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ float f_add(float a, float b) { return __fadd_rn(a, b); }
__device__ __forceinline__ float f_sub(float a, float b) { return __fsub_rn(a, b); }
__device__ __forceinline__ float f_div(float a, float b) { return __fdiv_rn(a, b); }
__device__ __forceinline__ float clamp01(float x) { return fminf(fmaxf(x, 0.0f), 1.0f); }
// clamp01(f_mul(a, b)) in one instruction: the rounded product saturated to
// [0, 1] (a NaN product gives 0, as clamp01 does)
__device__ __forceinline__ float f_mul_sat(float a, float b) {
  float r;
  asm("mul.rn.sat.f32 %0, %1, %2;" : "=f"(r) : "f"(a), "f"(b));
  return r;
}

// Pairs of binary32 operations in one instruction (FADD2 / FMUL2 / FFMA2 of
// sm_100 and later): each component is rounded as the scalar operation, so
// results are bit-identical to two scalar instructions.
__device__ __forceinline__ float2 f2_fma(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
__device__ __forceinline__ float2 f2_sub(float2 a, float2 b) {
  float2 r;
  asm("{\n\t.reg .b64 pa, pb, pr;\n\tmov.b64 pa, {%2, %3};\n\tmov.b64 pb, {%4, %5};\n\t"
      "sub.rn.f32x2 pr, pa, pb;\n\tmov.b64 {%0, %1}, pr;\n\t}"
      : "=f"(r.x), "=f"(r.y)
      : "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y));
  return r;
}

// Primary ray of pixel (px, py) clipped to the volume box (slab test).
// Returns true when the ray hits; o is the camera position.
__device__ __forceinline__ bool ray_setup(const CamDev& c, int px, int py, float d[3],
                                          float& tn, float& tf) {
  float sx = f_div(f_add((float)px, 0.5f), (float)c.W);
  float sy = f_div(f_add((float)py, 0.5f), (float)c.H);
  float u = f_mul(f_sub(f_mul(sx, 2.0f), 1.0f), c.ax);
  float v = f_mul(f_sub(1.0f, f_mul(sy, 2.0f)), c.ay);
  float dr[3];
#pragma unroll
  for (int a = 0; a < 3; ++a) dr[a] = f_add(f_add(c.fwd[a], f_mul(u, c.right[a])), f_mul(v, c.upv[a]));
  float l2 = f_add(f_add(f_mul(dr[0], dr[0]), f_mul(dr[1], dr[1])), f_mul(dr[2], dr[2]));
  float l = __fsqrt_rn(l2);
#pragma unroll
  for (int a = 0; a < 3; ++a) d[a] = f_div(dr[a], l);
  float tmin[3], tmax[3];
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    float inv = f_div(1.0f, d[a]);
    float t0 = f_mul(f_sub(-c.h[a], c.o[a]), inv);
    float t1 = f_mul(f_sub(c.h[a], c.o[a]), inv);
    tmin[a] = fminf(t0, t1);
    tmax[a] = fmaxf(t0, t1);
  }
  tn = fmaxf(fmaxf(tmin[0], tmin[1]), fmaxf(tmin[2], 0.0f));
  tf = fminf(fminf(tmax[0], tmax[1]), tmax[2]);
  return tn < tf;
}

// Sample k of a ray: midpoint of [tn + k dt, min(tn + (k+1) dt, tf)] and its
// length; x = normalised coordinate in [0,1]^3.  Returns false past tf.
__device__ __forceinline__ bool sample_at(const CamDev& c, const float d[3], float tn, float tf,
                                          int k, float x[3], float& tm, float& len) {
  float a = f_add(tn, f_mul((float)k, c.dt));
  if (!(a < tf)) return false;
  float b = fminf(f_add(tn, f_mul((float)(k + 1), c.dt)), tf);
  tm = f_mul(f_add(a, b), 0.5f);
  len = f_sub(b, a);
#pragma unroll
  for (int q = 0; q < 3; ++q) {
    float p = f_add(c.o[q], f_mul(tm, d[q]));
    const float num = f_add(p, c.h[q]);
    // division by an extent of exactly 1 (the longest axis) is the identity
    x[q] = f_mul_sat(num, c.inv_e[q]);
  }
  return true;
}

// Undithered LoD at distance t (floor of D, Sec. 5.3), clamped to
// [0, step_lod_max]: the step scale of step_mode 1.
__device__ __forceinline__ int step_level(const CamDev& c, float t) {
  int l;
  if (c.lod_mode == 0) {
    const float xf = f_mul(t, c.lodc);
    l = xf >= 1.0f ? (int)((__float_as_uint(xf) >> 23) & 0xFFu) - 127 : 0;
  } else {
    const float fl = floorf(f_mul(t, c.lod_scale));
    l = fl > 1e6f ? 1000000 : (int)fl;
  }
  l = l < 0 ? 0 : l;
  return l > c.step_lod_max ? c.step_lod_max : l;
}

// Enters the segment that starts at sample k (a multiple of 32).
__device__ __forceinline__ void sched_segment(const CamDev& c, float tn, int k, Sched& s) {
  if (c.step_mode == 0) return;
  s.ts = k == 0 ? tn : f_add(s.ts, f_mul(32.0f, s.dts));
  s.dts = f_mul(c.dt, (float)(1 << step_level(c, s.ts)));
}

// Sample k under the ray's schedule (the segment of k entered before).
__device__ __forceinline__ bool sample_in(const CamDev& c, const float d[3], float tn, float tf, int k,
                                          const Sched& s, float x[3], float& tm, float& len) {
  if (c.step_mode == 0) return sample_at(c, d, tn, tf, k, x, tm, len);
  const int j = k & 31;
  const float a = f_add(s.ts, f_mul((float)j, s.dts));
  if (!(a < tf)) return false;
  const float b = fminf(f_add(s.ts, f_mul((float)(j + 1), s.dts)), tf);
  tm = f_mul(f_add(a, b), 0.5f);
  len = f_sub(b, a);
#pragma unroll
  for (int q = 0; q < 3; ++q) {
    const float p = f_add(c.o[q], f_mul(tm, d[q]));
    const float num = f_add(p, c.h[q]);
    x[q] = f_mul_sat(num, c.inv_e[q]);
  }
  return true;
}

// Whether a segment follows the one that starts at sample k0 (k0 + 32 is
// the next segment's first sample).
__device__ __forceinline__ bool next_segment_exists(const CamDev& c, float tn, float tf, int k0,
                                                    const Sched& s) {
  if (c.step_mode == 0) return f_add(tn, f_mul((float)(k0 + 32), c.dt)) < tf;
  return f_add(s.ts, f_mul(32.0f, s.dts)) < tf;
}

// Whether the sample at LoD-0 position pv (= x * dims in binary32, >= 0)
// lies in a transparent macro cell: cell = floor(pv) >> shift per axis,
// clamped to the last cell at the far faces.
__device__ __forceinline__ bool macro_skips(const MacroDev& m, float pv0, float pv1, float pv2) {
  if (!m.skip) return false;
  const int c0 = min((int)pv0 >> m.shift, m.dims[0] - 1);
  const int c1 = min((int)pv1 >> m.shift, m.dims[1] - 1);
  const int c2 = min((int)pv2 >> m.shift, m.dims[2] - 1);
  return __ldg(m.skip + ((size_t)c2 * m.dims[1] + c1) * m.dims[0] + c0) != 0;
}

// Samples after the current one (LoD-0 position pv, spacing `step` along a
// ray of direction d) that certainly lie in the same macro cell: the
// distance to the cell's exit in whole steps, less one step of margin.
// The jump it allows skips exactly the samples that would be skipped one by
// one (the margin exceeds any rounding of the sample positions by orders of
// magnitude), so that a lane in empty space moves on to useful samples.
__device__ __forceinline__ int macro_run(const MacroDev& m, const CamDev& c, const float d[3], float pv0,
                                         float pv1, float pv2, float step) {
  const float pv[3] = {pv0, pv1, pv2};
  float texit = INFINITY;
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    const float dv = d[a] * c.inv_e[a] * (float)c.vol[a];  // d(pv)/dt
    const int ci = min((int)pv[a] >> m.shift, m.dims[a] - 1);
    if (dv > 0.0f) {
      const float edge = (float)min((ci + 1) << m.shift, c.vol[a]);
      texit = fminf(texit, (edge - pv[a]) / dv);
    } else if (dv < 0.0f) {
      texit = fminf(texit, ((float)(ci << m.shift) - pv[a]) / dv);
    }
  }
  const float steps = texit / step;
  if (!(steps < 1.0e6f)) return 1000000;
  return max((int)steps - 1, 0);
}

__device__ __forceinline__ uint32_t xorshift32(uint32_t s) {
  s ^= s << 13;
  s ^= s >> 17;
  s ^= s << 5;
  return s;
}

// Per-ray seed: MurmurHash3 finaliser of frame_seed ^ pixel * 0x9E3779B9.
__device__ __forceinline__ uint32_t ray_seed(uint32_t fseed, uint32_t pixel) {
  uint32_t h = fseed ^ (pixel * 0x9E3779B9u);
  h ^= h >> 16;
  h *= 0x85EBCA6Bu;
  h ^= h >> 13;
  h *= 0xC2B2AE35u;
  h ^= h >> 16;
  return h;
}

// Stochastic LoD of one sample (Alg. 2, Sec. 5.3): floor(D) plus one with
// probability frac(D), from one xorshift32 step keyed by (ray, sample).
__device__ __forceinline__ int sample_lod(const CamDev& c, int L, int lod_min, uint32_t rseed,
                                          uint32_t k, float tm) {
  uint32_t s = rseed ^ (k * 0x9E3779B9u);
  if (s == 0u) s = 0x6D2B79F5u;
  uint32_t u24 = xorshift32(s) >> 8;
  int base, inc;
  if (c.lod_mode == 0) {
    float xf = f_mul(tm, c.lodc);
    if (!(xf >= 1.0f)) {
      base = 0;
      inc = 0;
    } else {
      uint32_t bits = __float_as_uint(xf);
      base = (int)((bits >> 23) & 0xFFu) - 127;
      inc = u24 < 2u * (bits & 0x7FFFFFu);
    }
  } else {
    float D = f_mul(tm, c.lod_scale);
    float fl = floorf(D);
    float fr = f_sub(D, fl);
    base = fl > 1e6f ? 1000000 : (int)fl;
    inc = f_mul((float)u24, 5.9604644775390625e-08f) < fr;
  }
  int lod = base + inc;
  lod = lod < lod_min ? lod_min : lod;
  return lod > L - 1 ? L - 1 : lod;
}

// Explicit field stored at voxel centres (i+0.5)/dims, x fastest: trilinear
// interpolation with clamp-to-edge (training ground truth, Sec. 4.1, and the
// explicit-voxel render).
__device__ __forceinline__ float field_trilinear(const float* __restrict__ f, int3 d, float x, float y,
                                                 float z) {
  const float p[3] = {x, y, z};
  const int dd[3] = {d.x, d.y, d.z};
  int i0[3], i1[3];
  float w[3];
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    float q = f_sub(f_mul(clamp01(p[a]), (float)dd[a]), 0.5f);
    q = fminf(fmaxf(q, 0.0f), (float)(dd[a] - 1));
    i0[a] = (int)floorf(q);
    w[a] = f_sub(q, (float)i0[a]);
    i1[a] = i0[a] + 1 > dd[a] - 1 ? dd[a] - 1 : i0[a] + 1;
  }
  float v = 0.0f;
#pragma unroll
  for (int c = 0; c < 8; ++c) {
    const int ix = (c & 1) ? i1[0] : i0[0], iy = (c & 2) ? i1[1] : i0[1], iz = (c & 4) ? i1[2] : i0[2];
    const float wc = ((c & 1) ? w[0] : 1.0f - w[0]) * ((c & 2) ? w[1] : 1.0f - w[1]) *
                     ((c & 4) ? w[2] : 1.0f - w[2]);
    v = fmaf(wc, __ldg(f + ((size_t)iz * d.y + iy) * d.x + ix), v);
  }
  return v;
}

// ----------------------------------------------------- hash-grid encoding
__device__ __forceinline__ float2 load_entry(const void* table, int prec, uint32_t i) {
  if (prec == CINR_PREC_FP16) {
    __half2 h = __ldg(reinterpret_cast<const __half2*>(table) + i);
    return __half22float2(h);
  }
  return __ldg(reinterpret_cast<const float2*>(table) + i);
}

__device__ __forceinline__ uint32_t vertex_index(bool dense, uint32_t n1, uint32_t T, uint32_t cx,
                                                 uint32_t cy, uint32_t cz) {
  if (dense) return cx + n1 * (cy + n1 * cz);
  return ((cx * 1u) ^ (cy * 2654435761u) ^ (cz * 805459861u)) & (T - 1u);
}

// Cell of x in [0,1] on an N-cell grid: binary32 x*N, floor, clamp, weight.
__device__ __forceinline__ void grid_cell(float x, int N, int& i, float& w) {
  float xl = f_mul(x, (float)N);
  int ii = (int)floorf(xl);
  ii = ii < 0 ? 0 : (ii > N - 1 ? N - 1 : ii);
  i = ii;
  w = f_sub(xl, (float)ii);
}

template <bool F16>
__device__ __forceinline__ float2 load_entry_t(const void* table, uint32_t i) {
  if (F16) return __half22float2(__ldg(reinterpret_cast<const __half2*>(table) + i));
  return __ldg(reinterpret_cast<const float2*>(table) + i);
}

// Features of one point (levels concatenated, 2 per level): trilinear blend
// of the 8 vertex entries of each level (Sec. 3, Fig. 2).  The per-axis
// parts of the vertex index are formed once per level (dense: ix, iy (N+1),
// iz (N+1)^2 summed; hashed: ix, iy p2, iz p3 xor-ed, the +1 vertex by adding
// the row stride or the prime), the x-y weight products once per pair; the
// products, the corner order and the accumulation are those of the plain
// formula, so the features are unchanged bit for bit.
template <int L, bool F16>
__device__ __forceinline__ void encode_point_t(const InrDev& q, float x, float y, float z, float* feat) {
  const uint32_t T = 1u << q.log2T, Tm = T - 1u;
#pragma unroll
  for (int l = 0; l < L; ++l) {
    const int N = q.res[l];
    int ix, iy, iz;
    float wx, wy, wz;
    grid_cell(x, N, ix, wx);
    grid_cell(y, N, iy, wy);
    grid_cell(z, N, iz, wz);
    const bool dense = (q.dense_mask >> l) & 1u;
    const uint32_t n1 = (uint32_t)N + 1u;
    const uint32_t sy = dense ? n1 : 2654435761u, sz = dense ? n1 * n1 : 805459861u;
    const uint32_t ax[2] = {(uint32_t)ix, (uint32_t)ix + 1u};
    const uint32_t ay0 = (uint32_t)iy * sy, az0 = (uint32_t)iz * sz;
    const uint32_t ay[2] = {ay0, ay0 + sy}, az[2] = {az0, az0 + sz};
    const float wxs[2] = {1.0f - wx, wx}, wys[2] = {1.0f - wy, wy}, wzs[2] = {1.0f - wz, wz};
    const void* table = reinterpret_cast<const char*>(q.table) + (size_t)l * T * (F16 ? 4 : 8);
    float f0 = 0.0f, f1 = 0.0f;
#pragma unroll
    for (int c = 0; c < 8; ++c) {
      const int bx = c & 1, by = (c >> 1) & 1, bz = (c >> 2) & 1;
      uint32_t idx = dense ? ax[bx] + ay[by] + az[bz] : ((ax[bx] ^ ay[by] ^ az[bz]) & Tm);
      if (!in_range(idx, T, q.err)) idx = 0u;
      const float w = wxs[bx] * wys[by] * wzs[bz];
      const float2 e = load_entry_t<F16>(table, idx);
      f0 = fmaf(w, e.x, f0);
      f1 = fmaf(w, e.y, f1);
    }
    feat[2 * l] = f0;
    feat[2 * l + 1] = f1;
  }
}

template <int L>
__device__ __forceinline__ void encode_point(const InrDev& q, float x, float y, float z, float* feat) {
  if (q.table_prec == CINR_PREC_FP16)
    encode_point_t<L, true>(q, x, y, z, feat);
  else
    encode_point_t<L, false>(q, x, y, z, feat);
}

// FP32 SIMT MLP (in -> H -> H -> 1, ReLU, no biases); weights in shared
// memory, W1 [H][IN] then W2 [H][H] then W3 [H].
template <int IN, int H>
__device__ __forceinline__ float mlp_fp32(const float* __restrict__ sw, const float* feat) {
  float h1[H];
#pragma unroll
  for (int o = 0; o < H; ++o) {
    float s = 0.0f;
#pragma unroll
    for (int i = 0; i < IN; i += 4) {
      const float4 w4 = *reinterpret_cast<const float4*>(sw + o * IN + i);
      s = fmaf(w4.x, feat[i], s);
      s = fmaf(w4.y, feat[i + 1], s);
      s = fmaf(w4.z, feat[i + 2], s);
      s = fmaf(w4.w, feat[i + 3], s);
    }
    h1[o] = fmaxf(s, 0.0f);
  }
  const float* w2 = sw + IN * H;
  const float* w3 = w2 + H * H;
  float y = 0.0f;
#pragma unroll 2
  for (int o = 0; o < H; ++o) {
    float s = 0.0f;
#pragma unroll
    for (int i = 0; i < H; i += 4) {
      const float4 w4 = *reinterpret_cast<const float4*>(w2 + o * H + i);
      s = fmaf(w4.x, h1[i], s);
      s = fmaf(w4.y, h1[i + 1], s);
      s = fmaf(w4.z, h1[i + 2], s);
      s = fmaf(w4.w, h1[i + 3], s);
    }
    y = fmaf(w3[o], fmaxf(s, 0.0f), y);
  }
  return y;
}

template <int IN, int H>
__device__ __forceinline__ float inr_raw_fp32(const InrDev& q, const float* sw, float x, float y,
                                              float z) {
  float feat[IN];
  encode_point<IN / 2>(q, x, y, z, feat);
  return mlp_fp32<IN, H>(sw, feat);
}

template <int IN, int H>
__host__ __device__ constexpr int mlp_floats() {
  return IN * H + H * H + H;
}

// Cooperative copy of the fp32 weights into shared memory.
__device__ __forceinline__ void load_weights(float* sw, const float* w, int n) {
  for (int i = threadIdx.x; i < n; i += blockDim.x) sw[i] = __ldg(w + i);
}

// Supported (IN, H) pairs; dispatch helper for host code.
enum class Shape { S16x32, S32x64, S48x64, Bad };
inline Shape shape_of(int IN, int H) {
  if (IN == 16 && H == 32) return Shape::S16x32;
  if (IN == 32 && H == 64) return Shape::S32x64;
  if (IN == 48 && H == 64) return Shape::S48x64;
  return Shape::Bad;
}

}  // namespace cinr

// Frame statistics slots (device u64 counters).
namespace cinr {
enum StatIdx {
  ST_SAMPLES = 0, ST_DIRECT, ST_DECODE, ST_MISSES, ST_FALLBACK, ST_HITS, ST_REQ,
  ST_DECODED, ST_EVICT, ST_RECORDED, ST_SLOTS, ST_SKIPPED, ST_COUNT
};

// Radix-select state (find the n smallest unique 64-bit keys).
struct SelState {
  unsigned long long prefix;
  unsigned int k;
  unsigned int total;
  unsigned int none;
  unsigned int count;
  unsigned int hist[2048];
};
}  // namespace cinr

// Opaque handles (host side).
struct cinr_inr_s {
  cinr::InrDev dev;
  cinr_inr_params p;
  void* mem;
  size_t bytes;
  float* scratch;  // small device scratch for reductions
  uint16_t* w16;   // half-precision (FP16 or BF16) copy of the MLP weights
  int device;
};

struct cinr_cache_s {
  cinr::CacheDev dev;
  cinr_cache_opts o;
  long n_slots, n_bricks;
  uint64_t frame;
  cinr_inr_s* inr;
  cinr::SelState* sel_req;
  cinr::SelState* sel_vic;
  unsigned long long* req_keys;
  uint32_t* req_vals;
  uint32_t* req_sorted;
  uint32_t* req_n;
  unsigned long long* vic_keys;
  uint32_t* vic_vals;
  uint32_t* vic_sorted;
  uint32_t* vic_n;
  uint32_t* decode_n;
  int slot_bits, key_bits;
  uint32_t last_launches;  // kernels of the last end-of-frame update
  int decode_ctas = 0;     // decode CTAs per SM (0: as many as fit)
  // lag 2: decode stream, "selection done" and "decode done" events, and
  // whether a decoded batch waits to be mapped
  cudaStream_t dstream = nullptr;
  cudaEvent_t e_sel = nullptr, e_dec = nullptr;
  bool pending = false;
};

struct cinr_macro_s {
  int vol[3];
  int cell, shift;
  int dims[3];
  size_t n;        // cells
  float* ranges;   // 2 per cell: min, max (x fastest)
  uint8_t* skip;   // 1 per cell
  float* major;    // 1 per cell: largest extinction the cell's range reaches
  int device;
  cinr::MacroDev dev() const {
    cinr::MacroDev m;
    m.skip = skip;
    m.major = major;
    m.shift = shift;
    for (int a = 0; a < 3; ++a) m.dims[a] = dims[a];
    return m;
  }
};

// Skip flags of `tf` for macro m, enqueued on `s` (one kernel).
int cinr_macro_apply(cinr_macro_s* m, const float (*rgba)[4], cudaStream_t s);

// Cache update at the end of a frame (request selection, victims, commit,
// decode), enqueued on `s`; stats_dev receives decoded/evicted counts.
int cinr_cache_end_frame(cinr_cache_s* c, unsigned long long* stats_dev, cudaStream_t s);

// Makes `s` wait for a lag-2 decode still running on the cache's second
// stream (before reading the pool).
int cinr_cache_wait_decode(cinr_cache_s* c, cudaStream_t s);

// Tensor-core direct inference (FP16/BF16 MLP), used by cinr_infer.
int cinr_infer_tc(const cinr_inr_s* inr, const float* xyz, long n, float* out, cudaStream_t s);
