/*
 * CPU FP64 oracle of the cache-accelerated INR volume renderer.
 * TEST INFRASTRUCTURE ONLY -- see cinr_oracle.h for the rules it follows.
 *
 * Build: gcc -O2 -std=c11 -ffp-contract=off -fno-fast-math -fPIC -shared
 * (oracle/__init__.py does this).  -ffp-contract=off is part of the numeric
 * contract: every float expression below rounds after each operation.
 *
 * Readings of the paper where it is silent or ambiguous are marked READING.
 */
#include "cinr_oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>

/* ===================================================================== */
/* Random generators                                                       */
/* ===================================================================== */

/* SplitMix64 (Steele, Lea & Flood 2014): one output for state x. */
uint64_t orc_splitmix64(uint64_t x) {
  uint64_t z = x + 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

/* Xorshift32 with the (13, 17, 5) triple (Marsaglia 2003): the "simple
 * xorshift operation" of Sec. 5.3. */
uint32_t orc_xorshift32(uint32_t s) {
  s ^= s << 13;
  s ^= s >> 17;
  s ^= s << 5;
  return s;
}

/* Counter-based uniform coordinates in [0,1)^3 for training batches (Sec.
 * 4.1: each step draws a batch of random coordinates).  Coordinate c of
 * element j is the top 24 bits of splitmix64(seed + 3*(first+j) + c),
 * times 2^-24. */
void orc_uniform_coords(uint64_t seed, uint64_t first, long n, float* xyz) {
  for (long j = 0; j < n; ++j)
    for (int c = 0; c < 3; ++c) {
      uint64_t ctr = 3ull * (first + (uint64_t)j) + (uint64_t)c;
      uint64_t z = orc_splitmix64(seed + ctr);
      xyz[3 * j + c] = (float)(z >> 40) * (1.0f / 16777216.0f);
    }
}

/* ===================================================================== */
/* INR: multiresolution hash-grid encoding + small MLP (Sec. 3, Fig. 2)    */
/* ===================================================================== */

long orc_mlp_param_count(const orc_inr_params* p) {
  long h = p->hidden;
  return h * p->in_dim + (long)(p->n_hidden_layers - 1) * h * h + h;
}

/* Level resolutions.  READING: N_l = floor(N_min * b^l), with b^l formed by
 * repeated FP64 multiplication (the paper leaves the rule to Instant-NGP). */
void orc_level_res(const orc_inr_params* p, int* res) {
  double s = (double)p->base_res;
  for (int l = 0; l < p->levels; ++l) {
    res[l] = (int)floor(s);
    s = s * p->growth;
  }
}

static int level_res(const orc_inr_params* p, int level) {
  double s = (double)p->base_res;
  for (int l = 0; l < level; ++l) s = s * p->growth;
  return (int)floor(s);
}

/* A level whose (N+1)^3 grid vertices fit in the table is stored densely. */
int orc_level_is_dense(const orc_inr_params* p, int level) {
  uint64_t n1 = (uint64_t)level_res(p, level) + 1u;
  uint64_t T = 1ull << p->log2_table;
  return n1 * n1 * n1 <= T;
}

/* Table index of grid vertex (ix,iy,iz) at a level: the dense row-major index
 * when the level fits, else the spatial hash of Instant-NGP (XOR of the
 * coordinates times the per-axis primes 1, 2654435761, 805459861, in u32
 * arithmetic) modulo T. */
uint32_t orc_vertex_index(const orc_inr_params* p, int level, uint32_t ix,
                          uint32_t iy, uint32_t iz) {
  uint64_t n1 = (uint64_t)level_res(p, level) + 1u;
  uint32_t T = 1u << p->log2_table;
  if (n1 * n1 * n1 <= (uint64_t)T)
    return (uint32_t)((uint64_t)ix + n1 * ((uint64_t)iy + n1 * (uint64_t)iz));
  uint32_t h = (ix * 1u) ^ (iy * 2654435761u) ^ (iz * 805459861u);
  return h & (T - 1u);
}

/* Cell of coordinate x (already in [0,1]) on an N-cell grid: binary32
 * x_l = x*N, i = clamp(floor(x_l), 0, N-1), w = x_l - i. */
static void grid_cell(float x, int N, int* i, float* w) {
  float xl = x * (float)N;
  int ii = (int)floorf(xl);
  if (ii < 0) ii = 0;
  if (ii > N - 1) ii = N - 1;
  *i = ii;
  *w = xl - (float)ii;
}

static float clamp01(float x) {
  if (x < 0.0f) return 0.0f;
  if (x > 1.0f) return 1.0f;
  return x;
}

void orc_encode_indices(const orc_inr_params* p, const float* xyz, long n,
                        uint32_t* idx) {
  int L = p->levels;
  for (long j = 0; j < n; ++j) {
    float x[3] = {clamp01(xyz[3 * j]), clamp01(xyz[3 * j + 1]),
                  clamp01(xyz[3 * j + 2])};
    for (int l = 0; l < L; ++l) {
      int N = level_res(p, l);
      int i[3];
      float w[3];
      for (int a = 0; a < 3; ++a) grid_cell(x[a], N, &i[a], &w[a]);
      for (int c = 0; c < 8; ++c)
        idx[(j * L + l) * 8 + c] = orc_vertex_index(
            p, l, (uint32_t)(i[0] + (c & 1)), (uint32_t)(i[1] + ((c >> 1) & 1)),
            (uint32_t)(i[2] + ((c >> 2) & 1)));
    }
  }
}

/* Feature vector of one point: per level, trilinear interpolation of the n
 * features stored at the 8 surrounding vertices; levels concatenated
 * level-major (Sec. 3, Fig. 2). */
static void encode_one(const orc_inr_params* p, const double* table,
                       const float* xin, double* out) {
  int L = p->levels, F = p->feats;
  long T = 1L << p->log2_table;
  float x[3] = {clamp01(xin[0]), clamp01(xin[1]), clamp01(xin[2])};
  for (int l = 0; l < L; ++l) {
    int N = level_res(p, l);
    int i[3];
    float w[3];
    for (int a = 0; a < 3; ++a) grid_cell(x[a], N, &i[a], &w[a]);
    for (int f = 0; f < F; ++f) out[l * F + f] = 0.0;
    for (int c = 0; c < 8; ++c) {
      double wc = 1.0;
      for (int a = 0; a < 3; ++a) {
        int bit = (c >> a) & 1;
        wc *= bit ? (double)w[a] : 1.0 - (double)w[a];
      }
      uint32_t id = orc_vertex_index(p, l, (uint32_t)(i[0] + (c & 1)),
                                     (uint32_t)(i[1] + ((c >> 1) & 1)),
                                     (uint32_t)(i[2] + ((c >> 2) & 1)));
      const double* e = table + ((long)l * T + (long)id) * F;
      for (int f = 0; f < F; ++f) out[l * F + f] += wc * e[f];
    }
  }
}

void orc_encode(const orc_inr_params* p, const double* table, const float* xyz,
                long n, double* feats) {
  for (long j = 0; j < n; ++j)
    encode_one(p, table, xyz + 3 * j, feats + j * (long)p->in_dim);
}

/* MLP: in -> hidden (ReLU) [-> hidden (ReLU)]* -> 1, linear output.
 * READING: no biases (the fully fused MLP convention of the INR line of work
 * the paper builds on).  Weights: layer-major, each row-major [out][in]. */
static double mlp_one(const orc_inr_params* p, const double* w,
                      const double* in, double* act /* scratch 2*hidden */) {
  int H = p->hidden, I = p->in_dim;
  double* a = act;
  double* b = act + H;
  for (int o = 0; o < H; ++o) {
    double s = 0.0;
    for (int i = 0; i < I; ++i) s += w[(long)o * I + i] * in[i];
    a[o] = s > 0.0 ? s : 0.0;
  }
  const double* wl = w + (long)H * I;
  for (int layer = 1; layer < p->n_hidden_layers; ++layer) {
    for (int o = 0; o < H; ++o) {
      double s = 0.0;
      for (int i = 0; i < H; ++i) s += wl[(long)o * H + i] * a[i];
      b[o] = s > 0.0 ? s : 0.0;
    }
    double* t = a;
    a = b;
    b = t;
    wl += (long)H * H;
  }
  double y = 0.0;
  for (int i = 0; i < H; ++i) y += wl[i] * a[i];
  return y;
}

void orc_mlp(const orc_inr_params* p, const double* w, const double* feats,
             long n, double* y) {
  double* act = (double*)malloc(sizeof(double) * 2 * p->hidden);
  for (long j = 0; j < n; ++j) y[j] = mlp_one(p, w, feats + j * p->in_dim, act);
  free(act);
}

static double inr_one(const orc_inr_params* p, const double* table,
                      const double* w, const float* x, double* feat,
                      double* act) {
  encode_one(p, table, x, feat);
  double y = mlp_one(p, w, feat, act);
  return p->vmin + (p->vmax - p->vmin) * y; /* Sec. 4.1 de-normalisation */
}

void orc_inr_eval(const orc_inr_params* p, const double* table,
                  const double* w, const float* xyz, long n, double* v) {
  double* feat = (double*)malloc(sizeof(double) * p->in_dim);
  double* act = (double*)malloc(sizeof(double) * 2 * p->hidden);
  for (long j = 0; j < n; ++j) v[j] = inr_one(p, table, w, xyz + 3 * j, feat, act);
  free(feat);
  free(act);
}

/* Raw network output range over LoD-0 voxel centres (every stride-th voxel
 * per axis).  Used to normalise a seed-initialised (untrained) network so
 * that its field spans [0,1] (Sec. 4.1 keeps the exact value range). */
void orc_inr_raw_range(const orc_inr_params* p, const double* table,
                       const double* w, const int vol[3], int stride,
                       double* ymin, double* ymax) {
  double* feat = (double*)malloc(sizeof(double) * p->in_dim);
  double* act = (double*)malloc(sizeof(double) * 2 * p->hidden);
  double lo = INFINITY, hi = -INFINITY;
  for (int z = 0; z < vol[2]; z += stride)
    for (int y = 0; y < vol[1]; y += stride)
      for (int x = 0; x < vol[0]; x += stride) {
        float xn[3] = {((float)x + 0.5f) / (float)vol[0],
                       ((float)y + 0.5f) / (float)vol[1],
                       ((float)z + 0.5f) / (float)vol[2]};
        encode_one(p, table, xn, feat);
        double v = mlp_one(p, w, feat, act);
        if (v < lo) lo = v;
        if (v > hi) hi = v;
      }
  *ymin = lo;
  *ymax = hi;
  free(feat);
  free(act);
}

/* ===================================================================== */
/* Rays, sample schedule and LoD (Sec. 5.1, Sec. 5.3, Alg. 2)              */
/* ===================================================================== */

static int max3i(const int v[3]) {
  int m = v[0];
  if (v[1] > m) m = v[1];
  if (v[2] > m) m = v[2];
  return m;
}

static void normalize3(const float a[3], float out[3]) {
  float l2 = a[0] * a[0] + a[1] * a[1];
  l2 = l2 + a[2] * a[2];
  float l = sqrtf(l2);
  out[0] = a[0] / l;
  out[1] = a[1] / l;
  out[2] = a[2] / l;
}

static void cross3(const float a[3], const float b[3], float out[3]) {
  out[0] = a[1] * b[2] - a[2] * b[1];
  out[1] = a[2] * b[0] - a[0] * b[2];
  out[2] = a[0] * b[1] - a[1] * b[0];
}

static float tan_half_fov(const orc_camera* cam) {
  return (float)tan((double)cam->fov_y_deg * (3.14159265358979323846 / 360.0));
}

/* Box extents: the volume occupies [-e/2, e/2] with e = V / max(V). */
static void box_extent(const int vol[3], float e[3], float h[3]) {
  float m = (float)max3i(vol);
  for (int a = 0; a < 3; ++a) {
    e[a] = (float)vol[a] / m;
    h[a] = e[a] * 0.5f;
  }
}

/* One primary ray per pixel centre through a pinhole camera, clipped to the
 * volume box by the slab test (ray-generation kernel, Sec. 5.1).
 * READING: the paper gives no camera model; this one is perspective with
 * vertical field of view fov_y.  Returns 1 when the ray hits the box. */
int orc_ray(const orc_camera* cam, const int vol[3], int px, int py, float o[3],
            float d[3], float* tn, float* tf) {
  float fwd[3], right[3], upv[3], tmp[3];
  for (int a = 0; a < 3; ++a) tmp[a] = cam->target[a] - cam->eye[a];
  normalize3(tmp, fwd);
  cross3(fwd, cam->up, tmp);
  normalize3(tmp, right);
  cross3(right, fwd, upv);
  float th = tan_half_fov(cam);
  float aspect = (float)cam->width / (float)cam->height;
  float ax = th * aspect, ay = th;
  float sx = ((float)px + 0.5f) / (float)cam->width;
  float sy = ((float)py + 0.5f) / (float)cam->height;
  float u = (sx * 2.0f - 1.0f) * ax;
  float v = (1.0f - sy * 2.0f) * ay;
  float dr[3];
  for (int a = 0; a < 3; ++a) {
    float t = fwd[a] + u * right[a];
    dr[a] = t + v * upv[a];
  }
  normalize3(dr, d);
  for (int a = 0; a < 3; ++a) o[a] = cam->eye[a];
  float e[3], h[3];
  box_extent(vol, e, h);
  float tmin[3], tmax[3];
  for (int a = 0; a < 3; ++a) {
    float inv = 1.0f / d[a];
    float lo = -h[a];
    float t0 = (lo - o[a]) * inv;
    float t1 = (h[a] - o[a]) * inv;
    tmin[a] = fminf(t0, t1);
    tmax[a] = fmaxf(t0, t1);
  }
  float n = fmaxf(fmaxf(tmin[0], tmin[1]), fmaxf(tmin[2], 0.0f));
  float f = fminf(fminf(tmax[0], tmax[1]), tmax[2]);
  *tn = n;
  *tf = f;
  return n < f;
}

/* Sample k of a ray.  READING: the paper gives no step rule.  Segment k is
 * [tn + k*dt, min(tn + (k+1)*dt, tf)], dt = step / max(V) world units; the
 * sample sits at its midpoint and carries its length, so the lengths sum to
 * tf - tn.  Returns 0 when the ray has no sample k.  x is the normalised
 * coordinate in [0,1]^3. */
int orc_sample(const orc_camera* cam, const int vol[3], const float o[3],
               const float d[3], float tn, float tf, int k, float x[3],
               float* t_mid, float* seg_len) {
  float dt = cam->step_voxels / (float)max3i(vol);
  float a = tn + (float)k * dt;
  if (!(a < tf)) return 0;
  float b = fminf(tn + (float)(k + 1) * dt, tf);
  float tm = (a + b) * 0.5f;
  *t_mid = tm;
  *seg_len = b - a;
  float e[3], h[3];
  box_extent(vol, e, h);
  for (int c = 0; c < 3; ++c) {
    float pc = o[c] + tm * d[c];
    x[c] = clamp01((pc + h[c]) * (1.0f / e[c]));
  }
  return 1;
}

/* Pixel-footprint constant: t * c = footprint of a pixel at distance t in
 * LoD-0 voxels, times lod_scale (binary32). */
static float footprint_const(const orc_camera* cam, const int vol[3],
                             const orc_march_opts* mo) {
  float th = tan_half_fov(cam);
  float c1 = (2.0f * th) / (float)cam->height;
  float c2 = c1 * (float)max3i(vol);
  return c2 * mo->lod_scale;
}

/* Undithered LoD at distance t: floor of D (Sec. 5.3), at least 0. */
static int base_level(const orc_camera* cam, const int vol[3],
                      const orc_march_opts* mo, float t) {
  if (mo->lod_mode == 0) {
    float xf = t * footprint_const(cam, vol, mo);
    if (!(xf >= 1.0f)) return 0;
    uint32_t bits;
    memcpy(&bits, &xf, 4);
    return (int)((bits >> 23) & 0xFFu) - 127;
  }
  float fl = floorf(t * mo->lod_scale);
  return fl > 1e6f ? 1000000 : (int)fl;
}

/* Sample k of a ray under the schedule of mo->step_mode (k = 0, 1, 2, ... in
 * order; `s` carries the ray's segment state).
 * step_mode 0: the fixed-step schedule of orc_sample.
 * step_mode 1 (READING; the paper steps at one rate, which at tera-scale
 * oversamples the coarse LoDs that Sec. 5.3 already picks far from the
 * camera): segments of 32 samples; segment s starts at t_s (t_0 = tn,
 * t_{s+1} = t_s + 32 dt_s) and steps dt_s = dt * 2^l, l the undithered LoD
 * of t_s clamped to [0, step_lod_max]; within a segment sample j spans
 * [t_s + j dt_s, min(t_s + (j+1) dt_s, tf)]. */
int orc_sample_sched(const orc_camera* cam, const int vol[3],
                     const orc_march_opts* mo, const float o[3],
                     const float d[3], float tn, float tf, int k,
                     orc_sched* s, float x[3], float* t_mid,
                     float* seg_len) {
  if (mo->step_mode == 0)
    return orc_sample(cam, vol, o, d, tn, tf, k, x, t_mid, seg_len);
  float dt = cam->step_voxels / (float)max3i(vol);
  int j = k & 31;
  if (j == 0) {
    if (k == 0)
      s->ts = tn;
    else
      s->ts = s->ts + 32.0f * s->dts;
    int lvl = base_level(cam, vol, mo, s->ts);
    if (lvl > mo->step_lod_max) lvl = mo->step_lod_max;
    if (lvl < 0) lvl = 0;
    s->dts = dt * (float)(1 << lvl);
  }
  float a = s->ts + (float)j * s->dts;
  if (!(a < tf)) return 0;
  float b = fminf(s->ts + (float)(j + 1) * s->dts, tf);
  float tm = (a + b) * 0.5f;
  *t_mid = tm;
  *seg_len = b - a;
  float e[3], h[3];
  box_extent(vol, e, h);
  for (int c = 0; c < 3; ++c) {
    float pc = o[c] + tm * d[c];
    x[c] = clamp01((pc + h[c]) * (1.0f / e[c]));
  }
  return 1;
}

/* Higher-quality per-frame seed of the xorshift dither (Sec. 5.3). */
uint32_t orc_frame_seed(uint64_t seed, uint64_t frame) {
  return (uint32_t)orc_splitmix64(seed ^ frame);
}

/* Seed of a ray: the MurmurHash3 32-bit finaliser (Appleby) of
 * frame seed ^ pixel*0x9E3779B9. */
uint32_t orc_ray_seed(uint32_t frame_seed, uint32_t pixel) {
  uint32_t h = frame_seed ^ (pixel * 0x9E3779B9u);
  h ^= h >> 16;
  h *= 0x85EBCA6Bu;
  h ^= h >> 13;
  h *= 0xC2B2AE35u;
  h ^= h >> 16;
  return h;
}

/* Dither state of sample k of a ray: one xorshift32 step (Sec. 5.3) applied
 * to ray_seed ^ k*0x9E3779B9 (zero replaced by a fixed non-zero constant,
 * xorshift has no zero state).  Counter-based, so every sample of a ray can
 * be drawn independently. */
uint32_t orc_sample_state(uint32_t ray_seed, uint32_t k) {
  uint32_t s = ray_seed ^ (k * 0x9E3779B9u);
  if (s == 0u) s = 0x6D2B79F5u;
  return orc_xorshift32(s);
}

/* Stochastic LoD (Alg. 2, Sec. 5.3) of one sample, given its dither state
 * (orc_sample_state).
 * Distance mode (Alg. 2): D = dist * lod_scale, dist = the ray parameter.
 * Footprint mode: D = log2*(dist * pixel_angle * max(V) * lod_scale), i.e.
 * the log2 of the pixel footprint in LoD-0 voxels, with log2* the exact
 * piecewise-linear log2 read off the binary32 exponent and mantissa.
 * LoD = floor(D), plus 1 when u < frac(D) for u = (state >> 8) * 2^-24.
 * READING: Alg. 2 increments when the random number exceeds the fraction,
 * which would jump two levels at integer D and contradict the smoothing
 * purpose of Sec. 5.3; the
 * increment is taken with probability frac(D) (stochastic rounding).
 * READING: per sample (Alg. 2), keyed by (frame, pixel, sample). */
int orc_sample_lod(const orc_camera* cam, const int vol[3],
                   const orc_march_opts* mo, int levels, int lod_min,
                   uint32_t state, float t_mid) {
  uint32_t u24 = state >> 8;
  int base, inc;
  if (mo->lod_mode == 0) {
    float th = tan_half_fov(cam);
    float c1 = (2.0f * th) / (float)cam->height;
    float c2 = c1 * (float)max3i(vol);
    float c = c2 * mo->lod_scale;
    float xf = t_mid * c;
    if (!(xf >= 1.0f)) {
      base = 0;
      inc = 0;
    } else {
      uint32_t bits;
      memcpy(&bits, &xf, 4);
      base = (int)((bits >> 23) & 0xFFu) - 127;
      uint32_t mant = bits & 0x7FFFFFu; /* fraction = mant * 2^-23 */
      inc = u24 < 2u * mant;
    }
  } else {
    float D = t_mid * mo->lod_scale;
    float fl = floorf(D);
    float fr = D - fl;
    base = fl > 1e6f ? 1000000 : (int)fl;
    inc = ((float)u24 * (1.0f / 16777216.0f)) < fr;
  }
  int lod = base + inc;
  if (lod < lod_min) lod = lod_min;
  if (lod > levels - 1) lod = levels - 1;
  return lod;
}

/* ===================================================================== */
/* Transfer function and front-to-back compositing (Sec. 3, Sec. 5.1)      */
/* ===================================================================== */

/* 256-entry piecewise-linear TF; entry = (r, g, b, sigma), sigma the
 * extinction per world unit.  x = clamp(v,0,1)*255, linear between
 * floor(x) and floor(x)+1. */
void orc_tf_lookup(const double* tf, double v, double out[4]) {
  if (v < 0.0) v = 0.0;
  if (v > 1.0) v = 1.0;
  double x = v * 255.0;
  int i = (int)floor(x);
  if (i > 255) i = 255;
  int i1 = i + 1 > 255 ? 255 : i + 1;
  double fr = x - (double)i;
  for (int c = 0; c < 4; ++c)
    out[c] = tf[i * 4 + c] * (1.0 - fr) + tf[i1 * 4 + c] * fr;
}

/* Emission-absorption compositing of one sample, front to back:
 * alpha = 1 - exp(-sigma*len); C += T*alpha*rgb; T *= 1 - alpha. */
static void composite(const double* tf, double v, double len, double C[3],
                      double* T) {
  double e[4];
  orc_tf_lookup(tf, v, e);
  double alpha = 1.0 - exp(-e[3] * len);
  for (int c = 0; c < 3; ++c) C[c] += (*T) * alpha * e[c];
  *T = (*T) * (1.0 - alpha);
}

/* ===================================================================== */
/* Macro cells (Sec. 5.2, adaptive sampling)                               */
/* ===================================================================== */

/* The volume is cut into ceil(V/N) cubes of N LoD-0 voxels per axis. */
void orc_macro_dims(const int vol[3], int cell, int out[3]) {
  for (int a = 0; a < 3; ++a) out[a] = (vol[a] + cell - 1) / cell;
}

/* Cell of a normalised position: floor(x V) / N per axis (binary32 product,
 * the same LoD-0 coordinate that addresses the bricks), clamped to the last
 * cell at the far faces. */
long orc_macro_cell_of(const orc_macro* m, const int vol[3], const float x[3]) {
  long ci[3];
  for (int a = 0; a < 3; ++a) {
    float pv = x[a] * (float)vol[a];
    long i = (long)floorf(pv) / m->cell;
    if (i > m->dims[a] - 1) i = m->dims[a] - 1;
    ci[a] = i;
  }
  return ci[0] + (long)m->dims[0] * (ci[1] + (long)m->dims[1] * ci[2]);
}

static int macro_skips(const orc_march_opts* mo, const int vol[3],
                       const float x[3]) {
  return mo->macro && mo->macro->skip[orc_macro_cell_of(mo->macro, vol, x)];
}

/* LoD-l voxels a trilinear sample at LoD-0 edge coordinate e in [e0, e1] can
 * read: the lower corner floor(clamp(e 2^-l - 1/2, 0, dims-1)) and the one
 * above it, clamped to the grid. */
static void macro_box(int e0, int e1, int l, int dim_l, int* lo, int* hi) {
  float sc = 1.0f / (float)(1 << l), dmax = (float)(dim_l - 1);
  float q0 = fminf(fmaxf((float)e0 * sc - 0.5f, 0.0f), dmax);
  float q1 = fminf(fmaxf((float)e1 * sc - 0.5f, 0.0f), dmax);
  int h = (int)floorf(q1) + 1;
  *lo = (int)floorf(q0);
  *hi = h > dim_l - 1 ? dim_l - 1 : h;
}

static float round_down_f(double d) {
  float f = (float)d;
  return (double)f > d ? nextafterf(f, -INFINITY) : f;
}

static float round_up_f(double d) {
  float f = (float)d;
  return (double)f < d ? nextafterf(f, INFINITY) : f;
}

/* Min / max of grid values g (dims, x fastest) over each cell's box at LoD l,
 * merged into mn / mx. */
static void macro_merge_level(const double* g, const int dims[3], int l,
                              const int vol[3], int cell, const int md[3],
                              double* mn, double* mx) {
  for (int cz = 0; cz < md[2]; ++cz)
    for (int cy = 0; cy < md[1]; ++cy)
      for (int cx = 0; cx < md[0]; ++cx) {
        int c3[3] = {cx, cy, cz}, lo[3], hi[3];
        for (int a = 0; a < 3; ++a) {
          int e1 = (c3[a] + 1) * cell;
          macro_box(c3[a] * cell, e1 < vol[a] ? e1 : vol[a], l, dims[a], &lo[a], &hi[a]);
        }
        long ci = cx + (long)md[0] * (cy + (long)md[1] * cz);
        for (int k = lo[2]; k <= hi[2]; ++k)
          for (int j = lo[1]; j <= hi[1]; ++j)
            for (int i = lo[0]; i <= hi[0]; ++i) {
              double v = g[((long)k * dims[1] + j) * dims[0] + i];
              if (v < mn[ci]) mn[ci] = v;
              if (v > mx[ci]) mx[ci] = v;
            }
      }
}

static void macro_store(const double* mn, const double* mx, long n,
                        float* ranges) {
  for (long i = 0; i < n; ++i) {
    ranges[2 * i] = round_down_f(mn[i]);
    ranges[2 * i + 1] = round_up_f(mx[i]);
  }
}

/* Skip rule.  A sample of value v reads transfer-function entries floor(x)
 * and floor(x)+1, x = clamp(v,0,1) 255, so over a cell whose values lie in
 * [lo, hi] it can only reach entries floor(x_lo) .. floor(x_hi)+1.  When all
 * of them have zero extinction every sample in the cell has alpha = 0 and
 * leaves colour and transmittance unchanged: the cell is skipped (mu_max = 0,
 * Sec. 5.2).  READING: the range is widened by 2^-20 on both sides (binary32)
 * so that rounding in a trilinear sample or in x never leaves it. */
void orc_macro_skip(const float* ranges, long n_cells, const double* tf,
                    uint8_t* skip) {
  const float margin = 9.5367431640625e-07f; /* 2^-20 */
  for (long c = 0; c < n_cells; ++c) {
    float lo = clamp01(ranges[2 * c] - margin);
    float hi = clamp01(ranges[2 * c + 1] + margin);
    int i0 = (int)floorf(lo * 255.0f);
    int i1 = (int)floorf(hi * 255.0f) + 1;
    if (i1 > 255) i1 = 255;
    uint8_t s = 1;
    for (int i = i0; i <= i1; ++i)
      if (tf[i * 4 + 3] != 0.0) s = 0;
    skip[c] = s;
  }
}

/* Majorant of a cell for delta tracking (Sec. 5.2: the largest opacity a
 * cell's value range reaches under the current TF sets the sampling rate of
 * rays through it; Sec. 5.1: Woodcock tracking samples tentative collisions
 * at the rate of a majorant of the extinction).  The entries a sample of
 * the cell can read are those of the skip rule, floor(X(lo - 2^-20)) ..
 * floor(X(hi + 2^-20)) + 1, so the largest of their extinctions bounds the
 * extinction of every such sample; it is 0 exactly for the cells the skip
 * rule marks transparent. */
void orc_macro_majorant(const float* ranges, long n_cells, const double* tf,
                        float* major) {
  const float margin = 9.5367431640625e-07f; /* 2^-20 */
  for (long c = 0; c < n_cells; ++c) {
    float lo = clamp01(ranges[2 * c] - margin);
    float hi = clamp01(ranges[2 * c + 1] + margin);
    int i0 = (int)floorf(lo * 255.0f);
    int i1 = (int)floorf(hi * 255.0f) + 1;
    if (i1 > 255) i1 = 255;
    float m = 0.0f;
    for (int i = i0; i <= i1; ++i) m = fmaxf(m, (float)tf[i * 4 + 3]);
    major[c] = m;
  }
}

void orc_macro_ranges_field(const float* field, const int dims[3], int cell,
                            float* ranges) {
  int md[3];
  orc_macro_dims(dims, cell, md);
  long n = (long)md[0] * md[1] * md[2], nv = (long)dims[0] * dims[1] * dims[2];
  double* mn = (double*)malloc(sizeof(double) * n);
  double* mx = (double*)malloc(sizeof(double) * n);
  double* g = (double*)malloc(sizeof(double) * nv);
  for (long i = 0; i < n; ++i) {
    mn[i] = INFINITY;
    mx[i] = -INFINITY;
  }
  for (long i = 0; i < nv; ++i) g[i] = (double)field[i];
  macro_merge_level(g, dims, 0, dims, cell, md, mn, mx);
  macro_store(mn, mx, n, ranges);
  free(mn);
  free(mx);
  free(g);
}

/* Cache-off rendering: every sample is inferred directly by the INR
 * (Alg. 1 with every sample a miss).  Termination is tested only after each
 * segment of K samples (wavefront loop of Sec. 5.1).  Renders the pixel
 * window [px0, px0+pw) x [py0, py0+ph). */
void orc_render_direct(const orc_inr_params* p, const double* table,
                       const double* w, const orc_camera* cam,
                       const int vol[3], const orc_march_opts* mo,
                       const double* tf, int px0, int py0, int pw, int ph,
                       double* rgba, orc_stats* st) {
  memset(st, 0, sizeof(*st));
  double* feat = (double*)malloc(sizeof(double) * p->in_dim);
  double* act = (double*)malloc(sizeof(double) * 2 * p->hidden);
  for (int yy = 0; yy < ph; ++yy)
    for (int xx = 0; xx < pw; ++xx) {
      double* out = rgba + ((long)yy * pw + xx) * 4;
      out[0] = out[1] = out[2] = out[3] = 0.0;
      float o[3], d[3], tn, tf_;
      if (!orc_ray(cam, vol, px0 + xx, py0 + yy, o, d, &tn, &tf_)) continue;
      double C[3] = {0, 0, 0}, T = 1.0;
      orc_sched sc = {0.0f, 0.0f};
      for (int k = 0;; ++k) {
        float x[3], tm, len;
        if (!orc_sample_sched(cam, vol, mo, o, d, tn, tf_, k, &sc, x, &tm, &len))
          break;
        if (macro_skips(mo, vol, x)) {
          st->samples_skipped++;
        } else {
          double v = inr_one(p, table, w, x, feat, act);
          st->samples++;
          st->inr_queries_direct++;
          st->true_misses++;
          composite(tf, v, (double)len, C, &T);
        }
        if ((k + 1) % mo->K == 0 && T < (double)mo->eps_T) break;
      }
      out[0] = C[0];
      out[1] = C[1];
      out[2] = C[2];
      out[3] = 1.0 - T;
    }
  free(feat);
  free(act);
}

/* Explicit-voxel render: the same marching and compositing, every sample
 * valued by trilinear interpolation of an explicit field stored at voxel
 * centres (the uncompressed data an INR is trained on, Sec. 4.1). */
double orc_field_trilinear(const float* field, const int dims[3],
                           const float x[3]);

void orc_render_field(const float* field, const int fdims[3],
                      const orc_camera* cam, const int vol[3],
                      const orc_march_opts* mo, const double* tf, int px0,
                      int py0, int pw, int ph, double* rgba, orc_stats* st) {
  memset(st, 0, sizeof(*st));
  for (int yy = 0; yy < ph; ++yy)
    for (int xx = 0; xx < pw; ++xx) {
      double* out = rgba + ((long)yy * pw + xx) * 4;
      out[0] = out[1] = out[2] = out[3] = 0.0;
      float o[3], d[3], tn, tf_;
      if (!orc_ray(cam, vol, px0 + xx, py0 + yy, o, d, &tn, &tf_)) continue;
      double C[3] = {0, 0, 0}, T = 1.0;
      orc_sched sc = {0.0f, 0.0f};
      for (int k = 0;; ++k) {
        float x[3], tm, len;
        if (!orc_sample_sched(cam, vol, mo, o, d, tn, tf_, k, &sc, x, &tm, &len))
          break;
        if (macro_skips(mo, vol, x)) {
          st->samples_skipped++;
        } else {
          double v = orc_field_trilinear(field, fdims, x);
          st->samples++;
          composite(tf, v, (double)len, C, &T);
        }
        if ((k + 1) % mo->K == 0 && T < (double)mo->eps_T) break;
      }
      out[0] = C[0];
      out[1] = C[1];
      out[2] = C[2];
      out[3] = 1.0 - T;
    }
}

/* ===================================================================== */
/* Multi-resolution brick cache (Sec. 4.3)                                 */
/* ===================================================================== */

#define PT_MAPPED 0x80000000u
#define NO_OWNER 0xFFFFFFFFu

struct orc_cache {
  orc_inr_params p;
  const double* table;
  const double* w;
  int vol[3];
  orc_cache_opts co;
  orc_march_opts mo;
  int dims[16][3], nb[16][3];
  long off[17];
  long n_bricks;
  int S; /* stored edge B + 2 */
  uint32_t* pt;
  uint32_t* rank;
  uint32_t* stamp;
  uint32_t* owner;
  uint32_t* pinned;
  double* pool;
  uint64_t frame;
  uint32_t* last_req;
  long n_last_req;
  uint32_t* last_vict;
  long n_last_vict;
  long n_pending; /* lag 2: last_req/last_vict pairs decoded, not yet mapped */
  /* virtualised page tables (co.page = P > 0) */
  int pg[16][3];       /* pages per axis and LoD */
  long pd_off[17];     /* first page key of each LoD */
  uint32_t* pd;        /* page directory: Mapped | page slot */
  uint32_t* pages;     /* page pool: n_pages * P^3 entries */
  uint32_t* page_key;  /* page key held by each page slot, NO_OWNER if free */
  uint32_t* page_ref;  /* mapped bricks in each page slot */
  uint32_t* pt_view;   /* scratch of orc_cache_dump(0) in paged mode */
  uint32_t* miss;
  long n_miss, cap_miss;
};

long orc_cache_num_bricks(const orc_cache* c) { return c->n_bricks; }
long orc_cache_level_offset(const orc_cache* c, int level) {
  return c->off[level];
}
void orc_cache_level_dims(const orc_cache* c, int level, int dims[3],
                          int nb[3]) {
  for (int a = 0; a < 3; ++a) {
    dims[a] = c->dims[level][a];
    nb[a] = c->nb[level][a];
  }
}

/* LoD-l voxel grid: dims_l = ceil(V / 2^l); bricks of B voxels per edge. */
static void level_geometry(const int vol[3], int B, int l, int dims[3],
                           int nb[3]) {
  for (int a = 0; a < 3; ++a) {
    dims[a] = (vol[a] + (1 << l) - 1) >> l;
    nb[a] = (dims[a] + B - 1) / B;
  }
}

/* Normalised coordinate of the centre of LoD-l voxel j (clamped to the grid):
 * LoD-0 voxel-edge coordinate (j + 0.5) * 2^l, divided by V (Sec. 4.3.2:
 * coordinates strided by 2^LoD, no interpolation needed). */
static float voxel_centre(int j, int l, int dim_l, int V) {
  if (j < 0) j = 0;
  if (j > dim_l - 1) j = dim_l - 1;
  float t = ((float)j + 0.5f) * (float)(1 << l);
  return clamp01(t / (float)V);
}

/* Cell ranges from the INR: every LoD-l voxel grid (l in [min_level,
 * levels)) evaluated at its voxel centres, then min / max over each cell's
 * box.  READING: the paper builds the ranges during training from the data;
 * without the data they are taken from the voxels the cache serves, which
 * bounds every cached sample (a trilinear blend of them). */
void orc_macro_ranges_inr(const orc_inr_params* p, const double* table,
                          const double* w, const int vol[3], int cell,
                          int levels, int min_level, float* ranges) {
  int md[3];
  orc_macro_dims(vol, cell, md);
  long n = (long)md[0] * md[1] * md[2];
  double* mn = (double*)malloc(sizeof(double) * n);
  double* mx = (double*)malloc(sizeof(double) * n);
  for (long i = 0; i < n; ++i) {
    mn[i] = INFINITY;
    mx[i] = -INFINITY;
  }
  double* feat = (double*)malloc(sizeof(double) * p->in_dim);
  double* act = (double*)malloc(sizeof(double) * 2 * p->hidden);
  for (int l = min_level; l < levels; ++l) {
    int dims[3], nb[3];
    level_geometry(vol, 1, l, dims, nb);
    long nv = (long)dims[0] * dims[1] * dims[2];
    double* g = (double*)malloc(sizeof(double) * nv);
    for (int k = 0; k < dims[2]; ++k)
      for (int j = 0; j < dims[1]; ++j)
        for (int i = 0; i < dims[0]; ++i) {
          float x[3] = {voxel_centre(i, l, dims[0], vol[0]),
                        voxel_centre(j, l, dims[1], vol[1]),
                        voxel_centre(k, l, dims[2], vol[2])};
          g[((long)k * dims[1] + j) * dims[0] + i] = inr_one(p, table, w, x, feat, act);
        }
    macro_merge_level(g, dims, l, vol, cell, md, mn, mx);
    free(g);
  }
  macro_store(mn, mx, n, ranges);
  free(feat);
  free(act);
  free(mn);
  free(mx);
}

/* Brick (bx,by,bz) at LoD l stores voxels [b*B - 1, b*B + B] per axis, i.e.
 * the interior plus a one-voxel apron ("covering", Sec. 4.3.2), x fastest.
 * READING: the apron is kept on both sides so that trilinear sampling of any
 * point whose brick is b = floor(s/B) stays inside the brick. */
void orc_brick_values(const orc_inr_params* p, const double* table,
                      const double* w, const int vol[3], int brick, int level,
                      int bx, int by, int bz, double* out) {
  int dims[3], nb[3];
  level_geometry(vol, brick, level, dims, nb);
  int S = brick + 2;
  int b[3] = {bx, by, bz};
  double* feat = (double*)malloc(sizeof(double) * p->in_dim);
  double* act = (double*)malloc(sizeof(double) * 2 * p->hidden);
  for (int lz = 0; lz < S; ++lz)
    for (int ly = 0; ly < S; ++ly)
      for (int lx = 0; lx < S; ++lx) {
        int l3[3] = {lx, ly, lz};
        float x[3];
        for (int a = 0; a < 3; ++a)
          x[a] = voxel_centre(b[a] * brick - 1 + l3[a], level, dims[a], vol[a]);
        out[((long)lz * S + ly) * S + lx] = inr_one(p, table, w, x, feat, act);
      }
  free(feat);
  free(act);
}

/* Origin of a brick: the centre of its first stored voxel in LoD-0
 * voxel-edge coordinates (voxel i spans [i, i+1)), i.e. b*B*2^l - 2^(l-1)
 * per axis, clamped at the grid start.  The y and z components reproduce the
 * worked example of Sec. 4.3.2 (origin 79 and 159 for brick 1 and 2 at LoD 1,
 * B = 40); along x the apron voxel -1 is clamped to voxel 0, centre 2^(l-1). */
void orc_brick_origin(const int vol[3], int brick, int level, int bx, int by,
                      int bz, double origin[3]) {
  int dims[3], nb[3];
  level_geometry(vol, brick, level, dims, nb);
  int b[3] = {bx, by, bz};
  for (int a = 0; a < 3; ++a) {
    int j = b[a] * brick - 1;
    if (j < 0) j = 0;
    if (j > dims[a] - 1) j = dims[a] - 1;
    origin[a] = ((double)j + 0.5) * (double)(1 << level);
  }
}

/* Position of a sample at LoD l in LoD-l edge units, s = x*V / 2^l. */
static void level_coord(const float x[3], const int vol[3], int l, float s[3]) {
  float sc = 1.0f / (float)(1 << l);
  for (int a = 0; a < 3; ++a) {
    float pv = x[a] * (float)vol[a];
    s[a] = pv * sc;
  }
}

static void brick_of(const float s[3], int B, const int nb[3], int b[3]) {
  for (int a = 0; a < 3; ++a) {
    int bi = (int)floorf(s[a] / (float)B);
    if (bi < 0) bi = 0;
    if (bi > nb[a] - 1) bi = nb[a] - 1;
    b[a] = bi;
  }
}

/* Trilinear reconstruction inside a stored brick (Sec. 4.3: samples read from
 * brick memory).  q = clamp(s - 0.5, 0, dims-1) in binary32. */
static double brick_trilinear(const double* data, int S, int B,
                              const int b[3], const int dims[3],
                              const float s[3]) {
  int li[3];
  float f[3];
  for (int a = 0; a < 3; ++a) {
    float q = fminf(fmaxf(s[a] - 0.5f, 0.0f), (float)(dims[a] - 1));
    int i0 = (int)floorf(q);
    f[a] = q - (float)i0;
    li[a] = i0 - (b[a] * B - 1);
  }
  double v = 0.0;
  for (int c = 0; c < 8; ++c) {
    double wc = 1.0;
    int o[3];
    for (int a = 0; a < 3; ++a) {
      int bit = (c >> a) & 1;
      wc *= bit ? (double)f[a] : 1.0 - (double)f[a];
      o[a] = li[a] + bit;
    }
    v += wc * data[((long)o[2] * S + o[1]) * S + o[0]];
  }
  return v;
}

double orc_resident_sample(const orc_inr_params* p, const double* table,
                           const double* w, const int vol[3], int level,
                           const float x[3]) {
  /* Brute force: trilinear over the whole LoD-l voxel grid of INR values at
   * the voxel centres, clamp-to-edge; no bricks involved. */
  int dims[3];
  for (int a = 0; a < 3; ++a) dims[a] = (vol[a] + (1 << level) - 1) >> level;
  float s[3];
  level_coord(x, vol, level, s);
  int i0[3];
  float f[3];
  for (int a = 0; a < 3; ++a) {
    float q = fminf(fmaxf(s[a] - 0.5f, 0.0f), (float)(dims[a] - 1));
    i0[a] = (int)floorf(q);
    f[a] = q - (float)i0[a];
  }
  double* feat = (double*)malloc(sizeof(double) * p->in_dim);
  double* act = (double*)malloc(sizeof(double) * 2 * p->hidden);
  double v = 0.0;
  for (int c = 0; c < 8; ++c) {
    double wc = 1.0;
    float xc[3];
    for (int a = 0; a < 3; ++a) {
      int bit = (c >> a) & 1;
      wc *= bit ? (double)f[a] : 1.0 - (double)f[a];
      xc[a] = voxel_centre(i0[a] + bit, level, dims[a], vol[a]);
    }
    v += wc * inr_one(p, table, w, xc, feat, act);
  }
  free(feat);
  free(act);
  return v;
}

/* One sample at LoD l served from the brick that contains it (brick address,
 * apron brick contents, in-brick trilinear), without any cache state. */
double orc_brick_sample(const orc_inr_params* p, const double* table,
                        const double* w, const int vol[3], int brick, int level,
                        const float x[3]) {
  int dims[3], nb[3], b[3];
  level_geometry(vol, brick, level, dims, nb);
  float s[3];
  level_coord(x, vol, level, s);
  brick_of(s, brick, nb, b);
  int S = brick + 2;
  double* data = (double*)malloc(sizeof(double) * (size_t)S * S * S);
  orc_brick_values(p, table, w, vol, brick, level, b[0], b[1], b[2], data);
  double v = brick_trilinear(data, S, brick, b, dims, s);
  free(data);
  return v;
}

/* ---- page-table access (Sec. 4.3.1) ----------------------------------
 * Flat: one u32 entry per brick.  Paged (co.page = P): per LoD a page
 * directory over pages of P^3 bricks; a resident page lives in one of
 * n_pages page slots and holds the bricks' entries; a brick whose page is
 * not resident reads as Unmapped.  READING: the paper gives the structure,
 * not its management.  Pages are allocated when a brick in them is mapped
 * and freed when their last mapped brick is unmapped; at the end of a frame
 * all unmaps come first, then the pages left empty are freed, then the
 * pages the frame's mappings need are allocated -- in ascending page key,
 * into the free page slots in ascending order -- and then the bricks are
 * mapped; a brick whose page finds no free slot is dropped for the frame. */
static long page_index(const orc_cache* c, uint32_t key, long* local) {
  int l = 0;
  while (l + 1 < c->co.levels && (long)key >= c->off[l + 1]) ++l;
  long loc = (long)key - c->off[l];
  long bx = loc % c->nb[l][0];
  long by = (loc / c->nb[l][0]) % c->nb[l][1];
  long bz = loc / ((long)c->nb[l][0] * c->nb[l][1]);
  long P = c->co.page;
  *local = (bx % P) + P * ((by % P) + P * (bz % P));
  return c->pd_off[l] + bx / P + (long)c->pg[l][0] * (by / P + (long)c->pg[l][1] * (bz / P));
}

static uint32_t pt_get(const orc_cache* c, uint32_t key) {
  if (!c->co.page) return c->pt[key];
  long local, pk = page_index(c, key, &local);
  uint32_t e = c->pd[pk];
  if (!(e & PT_MAPPED)) return 0u;
  long P3 = (long)c->co.page * c->co.page * c->co.page;
  return c->pages[(long)(e & ~PT_MAPPED) * P3 + local];
}

static void pt_unmap(orc_cache* c, uint32_t key) {
  if (!c->co.page) {
    c->pt[key] = 0u;
    return;
  }
  long local, pk = page_index(c, key, &local);
  uint32_t ps = c->pd[pk] & ~PT_MAPPED;
  long P3 = (long)c->co.page * c->co.page * c->co.page;
  c->pages[(long)ps * P3 + local] = 0u;
  c->page_ref[ps]--;
}

/* Maps key -> slot; returns 0 when its page is not resident (paged). */
static int pt_map(orc_cache* c, uint32_t key, uint32_t slot) {
  if (!c->co.page) {
    c->pt[key] = PT_MAPPED | slot;
    return 1;
  }
  long local, pk = page_index(c, key, &local);
  uint32_t e = c->pd[pk];
  if (!(e & PT_MAPPED)) return 0;
  uint32_t ps = e & ~PT_MAPPED;
  long P3 = (long)c->co.page * c->co.page * c->co.page;
  c->pages[(long)ps * P3 + local] = PT_MAPPED | slot;
  c->page_ref[ps]++;
  return 1;
}

static void pages_free_empty(orc_cache* c) {
  if (!c->co.page) return;
  for (long ps = 0; ps < c->co.n_pages; ++ps)
    if (c->page_key[ps] != NO_OWNER && c->page_ref[ps] == 0) {
      c->pd[c->page_key[ps]] = 0u;
      c->page_key[ps] = NO_OWNER;
    }
}

static int cmp_u32(const void* x, const void* y) {
  uint32_t a = *(const uint32_t*)x, b = *(const uint32_t*)y;
  return a < b ? -1 : (a > b ? 1 : 0);
}

/* Allocates the non-resident pages of keys[0..n): ascending page keys into
 * ascending free page slots. */
static void pages_alloc(orc_cache* c, const uint32_t* keys, long n) {
  if (!c->co.page || n == 0) return;
  uint32_t* need = (uint32_t*)malloc(sizeof(uint32_t) * (size_t)n);
  long nn = 0;
  for (long i = 0; i < n; ++i) {
    long local, pk = page_index(c, keys[i], &local);
    if (!(c->pd[pk] & PT_MAPPED)) need[nn++] = (uint32_t)pk;
  }
  qsort(need, (size_t)nn, sizeof(uint32_t), cmp_u32);
  long ps = 0;
  for (long i = 0; i < nn; ++i) {
    if (i > 0 && need[i] == need[i - 1]) continue;
    while (ps < c->co.n_pages && c->page_key[ps] != NO_OWNER) ++ps;
    if (ps == c->co.n_pages) break;
    c->pd[need[i]] = PT_MAPPED | (uint32_t)ps;
    c->page_key[ps] = need[i];
    c->page_ref[ps] = 0;
  }
  free(need);
}

static void decode_into(orc_cache* c, uint32_t key, long slot) {
  int l = 0;
  while (l + 1 <= c->co.levels - 1 && (long)key >= c->off[l + 1]) ++l;
  long local = (long)key - c->off[l];
  int bx = (int)(local % c->nb[l][0]);
  int by = (int)((local / c->nb[l][0]) % c->nb[l][1]);
  int bz = (int)(local / ((long)c->nb[l][0] * c->nb[l][1]));
  long S3 = (long)c->S * c->S * c->S;
  orc_brick_values(&c->p, c->table, c->w, c->vol, c->co.brick, l, bx, by, bz,
                   c->pool + slot * S3);
}

orc_cache* orc_cache_create(const orc_inr_params* p, const double* table,
                            const double* w, const int vol[3],
                            const orc_cache_opts* co,
                            const orc_march_opts* mo) {
  if (co->levels < 1 || co->levels > 16) return NULL;
  if (co->lag != 1 && co->lag != 2) return NULL;
  orc_cache* c = (orc_cache*)calloc(1, sizeof(orc_cache));
  c->p = *p;
  c->table = table;
  c->w = w;
  for (int a = 0; a < 3; ++a) c->vol[a] = vol[a];
  c->co = *co;
  c->mo = *mo;
  c->S = co->brick + 2;
  c->off[0] = 0;
  for (int l = 0; l < co->levels; ++l) {
    level_geometry(vol, co->brick, l, c->dims[l], c->nb[l]);
    c->off[l + 1] =
        c->off[l] + (long)c->nb[l][0] * c->nb[l][1] * c->nb[l][2];
  }
  c->n_bricks = c->off[co->levels];
  if (co->page < 0 || (co->page > 0 && co->n_pages < 1)) {
    free(c);
    return NULL;
  }
  if (co->page > 0) {
    long P = co->page;
    c->pd_off[0] = 0;
    for (int l = 0; l < co->levels; ++l) {
      for (int a = 0; a < 3; ++a) c->pg[l][a] = (int)((c->nb[l][a] + P - 1) / P);
      c->pd_off[l + 1] = c->pd_off[l] + (long)c->pg[l][0] * c->pg[l][1] * c->pg[l][2];
    }
    c->pd = (uint32_t*)calloc((size_t)c->pd_off[co->levels], 4);
    c->pages = (uint32_t*)calloc((size_t)(co->n_pages * P * P * P), 4);
    c->page_key = (uint32_t*)malloc((size_t)co->n_pages * 4);
    c->page_ref = (uint32_t*)calloc((size_t)co->n_pages, 4);
    for (long i = 0; i < co->n_pages; ++i) c->page_key[i] = NO_OWNER;
  }
  c->pt = (uint32_t*)calloc((size_t)c->n_bricks, 4);
  c->rank = (uint32_t*)calloc((size_t)c->n_bricks, 4);
  c->stamp = (uint32_t*)calloc((size_t)co->n_slots, 4);
  c->owner = (uint32_t*)malloc((size_t)co->n_slots * 4);
  c->pinned = (uint32_t*)calloc((size_t)co->n_slots, 4);
  for (long s = 0; s < co->n_slots; ++s) c->owner[s] = NO_OWNER;
  long S3 = (long)c->S * c->S * c->S;
  c->pool = (double*)calloc((size_t)(co->n_slots * S3), sizeof(double));
  c->last_req = (uint32_t*)malloc(sizeof(uint32_t) * (co->n_req + 1));
  c->last_vict = (uint32_t*)malloc(sizeof(uint32_t) * (co->n_req + 1));
  c->cap_miss = 1024;
  c->miss = (uint32_t*)malloc(sizeof(uint32_t) * 2 * c->cap_miss);
  /* Preload (Sec. 4.3.4).  READING: the coarsest LoD is decoded and pinned
   * at creation, in key order into slots 0.., so that the fallback always
   * finds a brick. */
  if (co->preload) {
    int L = co->levels - 1;
    long nc = c->off[L + 1] - c->off[L];
    if (nc > co->n_slots) {
      orc_cache_destroy(c);
      return NULL;
    }
    uint32_t* keys = (uint32_t*)calloc((size_t)nc + 1, sizeof(uint32_t));
    for (long i = 0; i < nc; ++i) keys[i] = (uint32_t)(c->off[L] + i);
    pages_alloc(c, keys, nc);
    for (long i = 0; i < nc; ++i) {
      uint32_t key = keys[i];
      decode_into(c, key, i);
      if (!pt_map(c, key, (uint32_t)i)) {
        free(keys);
        orc_cache_destroy(c);
        return NULL; /* the page pool cannot hold the coarsest LoD */
      }
      c->owner[i] = key;
      c->pinned[i] = 1;
    }
    free(keys);
  }
  return c;
}

void orc_cache_destroy(orc_cache* c) {
  if (!c) return;
  free(c->pd);
  free(c->pages);
  free(c->page_key);
  free(c->page_ref);
  free(c->pt_view);
  free(c->pt);
  free(c->rank);
  free(c->stamp);
  free(c->owner);
  free(c->pinned);
  free(c->pool);
  free(c->last_req);
  free(c->last_vict);
  free(c->miss);
  free(c);
}

static void push_miss(orc_cache* c, uint32_t pixel, uint32_t k) {
  if (c->n_miss == c->cap_miss) {
    c->cap_miss *= 2;
    c->miss = (uint32_t*)realloc(c->miss, sizeof(uint32_t) * 2 * c->cap_miss);
  }
  c->miss[2 * c->n_miss] = pixel;
  c->miss[2 * c->n_miss + 1] = k;
  c->n_miss++;
}

typedef struct {
  uint64_t a;
  uint32_t b;
} sort_pair;

static int cmp_u64_key(const void* x, const void* y) {
  const sort_pair* p = (const sort_pair*)x;
  const sort_pair* q = (const sort_pair*)y;
  if (p->a < q->a) return -1;
  if (p->a > q->a) return 1;
  return 0;
}

/* One cached sample (Alg. 2, Sec. 4.3): stochastic LoD from the distance
 * `dist` to the eye; page-table lookup at that LoD; an Unmapped brick raises
 * a ranked request (Sec. 4.3.3) and the lookup falls back to coarser LoDs;
 * the first Mapped brick is sampled trilinearly and its slot stamped with
 * the frame (LRU); no Mapped brick at any LoD = true miss, recorded as
 * (pixel, k) and inferred directly by the INR (Alg. 1). */
static double cache_lookup(orc_cache* c, const orc_camera* cam, const float x[3],
                           float dist, uint32_t state, uint32_t Tf, uint64_t f,
                           uint32_t pixel, uint32_t k, double* feat, double* act,
                           orc_stats* st) {
  int L = c->co.levels, B = c->co.brick, S = c->S;
  long S3 = (long)S * S * S;
  int l = orc_sample_lod(cam, c->vol, &c->mo, L, 0, state, dist);
  for (int lev = l; lev < L; ++lev) {
    float s[3];
    int b[3];
    level_coord(x, c->vol, lev, s);
    brick_of(s, B, c->nb[lev], b);
    long key = c->off[lev] +
               b[0] + (long)c->nb[lev][0] * (b[1] + (long)c->nb[lev][1] * b[2]);
    uint32_t e = pt_get(c, (uint32_t)key);
    if (!(e & PT_MAPPED)) {
      if (lev == l) {
        uint32_t r = c->rank[key];
        if (r < Tf) {
          r = Tf;
          st->bricks_requested++;
        }
        r = r + 1u;
        if (r > Tf + 1000u) r = Tf + 1000u;
        c->rank[key] = r;
      }
      continue;
    }
    long slot = (long)(e & ~PT_MAPPED);
    double v = brick_trilinear(c->pool + slot * S3, S, B, b, c->dims[lev], s);
    c->stamp[slot] = (uint32_t)f;
    if (lev == l)
      st->hits++;
    else
      st->fallback_hits++;
    return v;
  }
  st->true_misses++;
  st->inr_queries_direct++;
  push_miss(c, pixel, k);
  return inr_one(&c->p, c->table, c->w, x, feat, act);
}

/* End of frame f: the Cache Manager's request list, the LRU victims and the
 * Request Handler's decode + write-back (Fig. 1, Sec. 4.3.2-4.3.3). */
static void cache_end_frame(orc_cache* c, uint32_t Tf, uint64_t f, orc_stats* st) {
  long S3 = (long)c->S * c->S * c->S;
  /* ---- lag 2 (asynchronous request handling, Sec. 4.3 / Sarton's RH):
   * the bricks selected and unmapped at the end of the previous frame were
   * decoded while this frame rendered; they are mapped now, before this
   * frame's selection.  READING: a fixed lag of two frames keeps the state
   * deterministic. ---- */
  pages_alloc(c, c->last_req, c->n_pending);
  for (long i = 0; i < c->n_pending; ++i) {
    uint32_t slot = c->last_vict[i], key = c->last_req[i];
    if (!pt_map(c, key, slot)) continue; /* no page slot: dropped */
    c->owner[slot] = key;
    c->stamp[slot] = (uint32_t)f;
  }
  c->n_pending = 0;

  /* ---- Cache Manager: request list (Sec. 4.3.3; Sarton first-n when the
   * ranking is off).  Candidates are bricks requested this frame that are
   * not mapped now (with lag 2 a brick in flight during the frame was
   * requested again and has just been mapped). ---- */
  long nb = c->n_bricks;
  sort_pair* cand = (sort_pair*)malloc(sizeof(sort_pair) * (size_t)(nb + 1));
  long nc = 0;
  for (long key = 0; key < nb; ++key) {
    uint32_t r = c->rank[key];
    if (r > Tf && !(pt_get(c, (uint32_t)key) & PT_MAPPED)) {
      uint64_t score = (uint64_t)(r - Tf);
      uint64_t sk = c->co.ranking ? ((1000u - score) << 32) | (uint64_t)key
                                  : (uint64_t)key;
      cand[nc].a = sk;
      cand[nc].b = (uint32_t)key;
      nc++;
    }
  }
  qsort(cand, (size_t)nc, sizeof(sort_pair), cmp_u64_key);
  long nreq = nc < c->co.n_req ? nc : c->co.n_req;
  for (long i = 0; i < nreq; ++i) c->last_req[i] = cand[i].b;
  c->n_last_req = nreq;
  free(cand);

  /* ---- victims: LRU by (stamp, slot); never-used slots carry stamp 0;
   * slots used this frame and pinned slots are not eligible ---- */
  long ns = c->co.n_slots;
  sort_pair* vc = (sort_pair*)malloc(sizeof(sort_pair) * (size_t)(ns + 1));
  long nv = 0;
  for (long s = 0; s < ns; ++s) {
    if (c->pinned[s] || c->stamp[s] >= (uint32_t)f) continue;
    vc[nv].a = ((uint64_t)c->stamp[s] << 32) | (uint64_t)s;
    vc[nv].b = (uint32_t)s;
    nv++;
  }
  qsort(vc, (size_t)nv, sizeof(sort_pair), cmp_u64_key);
  long m = nreq < nv ? nreq : nv;
  for (long i = 0; i < m; ++i) c->last_vict[i] = vc[i].b;
  c->n_last_vict = m;
  free(vc);

  /* ---- Request Handler: decode each requested brick by INR inference
   * into its victim slot, then update page table and LRU (Sec. 4.3.2,
   * Fig. 1) ---- */
  for (long i = 0; i < m; ++i) {
    uint32_t slot = c->last_vict[i];
    if (c->owner[slot] != NO_OWNER) {
      pt_unmap(c, c->owner[slot]);
      st->evictions++;
    }
    /* lag 2: in flight, unmapped until the next frame ends */
    c->owner[slot] = NO_OWNER;
  }
  pages_free_empty(c);
  for (long i = 0; i < m; ++i) decode_into(c, c->last_req[i], (long)c->last_vict[i]);
  if (c->co.lag == 1) {
    pages_alloc(c, c->last_req, m);
    for (long i = 0; i < m; ++i) {
      uint32_t slot = c->last_vict[i], key = c->last_req[i];
      if (!pt_map(c, key, slot)) continue; /* no page slot: dropped */
      c->owner[slot] = key;
      c->stamp[slot] = (uint32_t)f;
    }
  } else {
    c->n_pending = m;
  }
  st->bricks_decoded = (uint64_t)m;
  st->inr_queries_decode = (uint64_t)m * (uint64_t)S3;
}

/* Cached rendering of frame f (Fig. 1; Alg. 1 and 2; Sec. 4.3).
 * Per sample: stochastic LoD l; page-table lookup at l; if the brick is
 * Unmapped a request is raised for it (priority rank, Sec. 4.3.3) and the
 * lookup falls back to l+1, l+2, ... (Sec. 4.3); the first Mapped brick is
 * sampled trilinearly and its slot stamped with f (LRU); no Mapped brick at
 * any level = true miss, recorded and inferred directly by the INR (Alg. 1).
 * End of frame: top-n requests, victims, decode + write-back, map (lag-1:
 * the new bricks serve frame f+1). */
void orc_render_cached(orc_cache* c, const orc_camera* cam, const double* tf,
                       int px0, int py0, int pw, int ph, double* rgba,
                       orc_stats* st) {
  memset(st, 0, sizeof(*st));
  c->frame += 1;
  uint64_t f = c->frame;
  /* READING of the ranking rule (Sec. 4.3.3): the frame timestamp advances
   * by 1001 per frame; a request sets r = max(r, T_f) + 1, clamped at
   * T_f + 1000, so the score of a brick this frame is min(#requests, 1000)
   * and stale ranks never outrank fresh requests. */
  uint32_t Tf = (uint32_t)(1001u * (uint32_t)f);
  uint32_t fseed = orc_frame_seed(c->mo.seed, f);
  c->n_miss = 0;
  double* feat = (double*)malloc(sizeof(double) * c->p.in_dim);
  double* act = (double*)malloc(sizeof(double) * 2 * c->p.hidden);
  for (int yy = 0; yy < ph; ++yy)
    for (int xx = 0; xx < pw; ++xx) {
      double* out = rgba + ((long)yy * pw + xx) * 4;
      out[0] = out[1] = out[2] = out[3] = 0.0;
      int px = px0 + xx, py = py0 + yy;
      uint32_t pixel = (uint32_t)(py * cam->width + px);
      float o[3], d[3], tn, tf_;
      if (!orc_ray(cam, c->vol, px, py, o, d, &tn, &tf_)) continue;
      double C[3] = {0, 0, 0}, T = 1.0;
      uint32_t rs = orc_ray_seed(fseed, pixel);
      orc_sched sc = {0.0f, 0.0f};
      for (int k = 0;; ++k) {
        float x[3], tm, len;
        if (!orc_sample_sched(cam, c->vol, &c->mo, o, d, tn, tf_, k, &sc, x, &tm,
                              &len))
          break;
        if (macro_skips(&c->mo, c->vol, x)) {
          /* transparent cell (Sec. 5.2): no LoD, no lookup, no request */
          st->samples_skipped++;
        } else {
          st->samples++;
          double v = cache_lookup(c, cam, x, tm, orc_sample_state(rs, (uint32_t)k), Tf, f,
                                  pixel, (uint32_t)k, feat, act, st);
          composite(tf, v, (double)len, C, &T);
        }
        if ((k + 1) % c->mo.K == 0 && T < (double)c->mo.eps_T) break;
      }
      out[0] = C[0];
      out[1] = C[1];
      out[2] = C[2];
      out[3] = 1.0 - T;
    }
  free(feat);
  free(act);

  cache_end_frame(c, Tf, f, st);
}

/* ===================================================================== */
/* Path tracing with Woodcock delta tracking (Sec. 5.1)                    */
/* ===================================================================== */
/* READING: the paper names the estimator (Woodcock delta tracking on the
 * same sampler as ray marching) but no light transport details.  This
 * reading: one path per pixel and frame; free paths -ln(1-u)/sigma_bar with
 * the TF's largest extinction as majorant sigma_bar; a tentative collision
 * at value v is real with probability sigma(v)/sigma_bar; at a real
 * collision the throughput takes the TF colour as albedo, a directional
 * light is added by next-event estimation (isotropic phase 1/4pi, shadow
 * transmittance by ratio tracking), and the path scatters into a uniform
 * direction; paths that leave the volume collect the ambient radiance.
 * Every quantity that positions a lookup is binary32 in a fixed order
 * (this log, the sphere sampler and the box exits use +,-,*,/,sqrt only),
 * so the lookups, requests and stamps are reproducible bit for bit. */

#define PT_MAX_STEPS 4096
#define ORC_PI 3.14159265358979323846

float orc_neg_log1m(float u) {
  /* y = 1 - u = m 2^e with m in [sqrt(2)/2, sqrt(2)) (no cancellation for y
   * near 1); ln y = e ln2 + 2 atanh(z), z = (m-1)/(m+1), |z| < 0.172,
   * series to z^15 (truncation < 1e-12). */
  float y = 1.0f - u;
  uint32_t bits;
  memcpy(&bits, &y, 4);
  int e = (int)((bits >> 23) & 0xFFu) - 127;
  uint32_t mb = (bits & 0x7FFFFFu) | 0x3F800000u;
  float m;
  memcpy(&m, &mb, 4);
  if (m > 1.41421356f) {
    m = m * 0.5f;
    e = e + 1;
  }
  float z = (m - 1.0f) / (m + 1.0f);
  float z2 = z * z;
  float q = 1.0f / 15.0f;
  q = q * z2 + 1.0f / 13.0f;
  q = q * z2 + 1.0f / 11.0f;
  q = q * z2 + 1.0f / 9.0f;
  q = q * z2 + 1.0f / 7.0f;
  q = q * z2 + 1.0f / 5.0f;
  q = q * z2 + 1.0f / 3.0f;
  q = q * z2 + 1.0f;
  float lm = (2.0f * z) * q;
  float ln = (float)e * 0.693147180559945309f + lm;
  return -ln;
}

/* The j-th output of a SplitMix64 generator started at state `key`
 * (Steele et al. 2014: output j = mix(key + (j+1) gamma)), top 24 bits. */
float orc_pt_uniform(uint64_t key, uint32_t j) {
  uint64_t x = orc_splitmix64(key + 0x9E3779B97F4A7C15ull * (uint64_t)j);
  return (float)(x >> 40) * (1.0f / 16777216.0f);
}

/* Uniform direction on the unit sphere (Marsaglia 1972): (x1, x2) uniform
 * in the unit disc by rejection, then (2 x1 r, 2 x2 r, 1 - 2 s) with
 * s = x1^2 + x2^2 and r = sqrt(1 - s). */
void orc_pt_sphere(uint64_t key, uint32_t* j, float dir[3]) {
  for (int tries = 0; tries < 64; ++tries) {
    float x1 = orc_pt_uniform(key, (*j)++) * 2.0f - 1.0f;
    float x2 = orc_pt_uniform(key, (*j)++) * 2.0f - 1.0f;
    float s = x1 * x1 + x2 * x2;
    if (s < 1.0f) {
      float r = 2.0f * sqrtf(1.0f - s);
      dir[0] = x1 * r;
      dir[1] = x2 * r;
      dir[2] = 1.0f - 2.0f * s;
      return;
    }
  }
  dir[0] = 0.0f;
  dir[1] = 0.0f;
  dir[2] = 1.0f;
}

/* Distance from a point inside the box [-h, h] to its boundary along d. */
static float box_exit(const float h[3], const float o[3], const float d[3]) {
  float t = INFINITY;
  for (int a = 0; a < 3; ++a) {
    if (d[a] == 0.0f) continue;
    float inv = 1.0f / d[a];
    float t0 = (-h[a] - o[a]) * inv;
    float t1 = (h[a] - o[a]) * inv;
    t = fminf(t, fmaxf(t0, t1));
  }
  return t;
}

typedef struct {
  orc_cache* c;                 /* NULL: direct inference */
  const orc_inr_params* p;
  const double* table;
  const double* w;
  uint32_t Tf;
  uint64_t f;
  double* feat;
  double* act;
} pt_ctx;

static double pt_lookup(pt_ctx* ctx, const orc_camera* cam, const float x[3],
                        float dist, uint32_t state, uint32_t pixel, uint32_t k,
                        orc_stats* st) {
  st->samples++;
  if (ctx->c)
    return cache_lookup(ctx->c, cam, x, dist, state, ctx->Tf, ctx->f, pixel, k,
                        ctx->feat, ctx->act, st);
  st->inr_queries_direct++;
  st->true_misses++;
  return inr_one(ctx->p, ctx->table, ctx->w, x, ctx->feat, ctx->act);
}

/* World point o + t d: normalised coordinate (as the ray-marching samples)
 * and binary32 distance to the eye. */
static void pt_point(const orc_camera* cam, const float e[3], const float h[3],
                     const float o[3], const float d[3], float t, float p[3],
                     float x[3], float* dist) {
  for (int q = 0; q < 3; ++q) {
    p[q] = o[q] + t * d[q];
    float num = p[q] + h[q];
    x[q] = clamp01(num * (1.0f / e[q]));
  }
  float dx = p[0] - cam->eye[0], dy = p[1] - cam->eye[1], dz = p[2] - cam->eye[2];
  float s2 = dx * dx + dy * dy;
  s2 = s2 + dz * dz;
  *dist = sqrtf(s2);
}

/* READING (local majorants): Sec. 5.2 says each macro cell's largest
 * opacity under the TF sets the sampling rate of rays through that cell;
 * for Woodcock tracking that rate is the majorant.  With a macro-cell
 * structure carrying majorants, a free flight draws its optical depth
 * tau = -ln(1-u) once and spends it along the ray cell by cell (a 3D DDA
 * over the cells): in a cell with majorant m entered at t and left at t_e,
 * the tentative collision lies at t + tau/m when tau < m (t_e - t),
 * otherwise tau -= m (t_e - t) and the flight enters the next cell.  Cells
 * with m = 0 are crossed without a lookup.  A tentative collision at value v
 * is real with probability sigma(v)/m of its cell, and ratio tracking
 * multiplies by 1 - sigma(v)/m.  All of it binary32 in this order:
 *   start at o + t d (segment end t1): per axis p = o + t d,
 *          x = clamp01((p + h) (1/e)), pv = x V, c = min(floor(pv) / N,
 *          dims - 1), dv = (d (1/e)) V, r = 1/dv;
 *          dv > 0: t_max = t + ((c+1) N - pv) r, t_delta = N r;
 *          dv < 0: t_max = t + (c N - pv) r, t_delta = N (-r);
 *          dv = 0: both infinite;
 *   enter a cell: m = its majorant, r_m = 1/m (0 when m = 0),
 *          t_e = min(t_max_x, t_max_y, t_max_z, t1);
 *   flight from t: while m > 0 and tau >= dd = m (t_e - t): tau -= dd;
 *          with tau < dd the collision is at min(t + tau r_m, t_e);
 *          else t = t_e, the axis of the smallest t_max (x before y before
 *          z on ties) moves one cell, t_max += t_delta, and the next cell
 *          is entered; leaving the grid or reaching t1 ends the flight. */
typedef struct {
  const orc_macro* m;
  int c[3], step[3], live;
  float tmax[3], tdelta[3];
  float mj, rj, te, t1;
} pt_walk;

static void walk_enter(pt_walk* w) {
  const orc_macro* m = w->m;
  long cell = ((long)w->c[2] * m->dims[1] + w->c[1]) * m->dims[0] + w->c[0];
  w->mj = m->major[cell];
  w->rj = w->mj > 0.0f ? 1.0f / w->mj : 0.0f;
  w->te = fminf(fminf(fminf(w->tmax[0], w->tmax[1]), w->tmax[2]), w->t1);
}

static void walk_init(pt_walk* w, const orc_macro* m, const int vol[3],
                      const float e[3], const float h[3], const float o[3],
                      const float d[3], float t, float t1) {
  w->m = m;
  w->live = 1;
  w->t1 = t1;
  float N = (float)m->cell;
  for (int a = 0; a < 3; ++a) {
    float inv_e = 1.0f / e[a];
    float p = o[a] + t * d[a];
    float num = p + h[a];
    float x = clamp01(num * inv_e);
    float pv = x * (float)vol[a];
    int ci = (int)floorf(pv) / m->cell;
    if (ci > m->dims[a] - 1) ci = m->dims[a] - 1;
    w->c[a] = ci;
    float dv = (d[a] * inv_e) * (float)vol[a];
    if (dv > 0.0f) {
      float r = 1.0f / dv;
      w->step[a] = 1;
      w->tmax[a] = t + ((float)((ci + 1) * m->cell) - pv) * r;
      w->tdelta[a] = N * r;
    } else if (dv < 0.0f) {
      float r = 1.0f / dv;
      w->step[a] = -1;
      w->tmax[a] = t + ((float)(ci * m->cell) - pv) * r;
      w->tdelta[a] = N * -r;
    } else {
      w->step[a] = 0;
      w->tmax[a] = INFINITY;
      w->tdelta[a] = INFINITY;
    }
  }
  walk_enter(w);
}

/* Spends optical depth tau from *t: 1 with the tentative collision in *t and
 * its cell's majorant in *maj, 0 when the segment's end (or the grid's)
 * comes first. */
static int walk_flight(pt_walk* w, float tau, float* t, float* maj) {
  const orc_macro* m = w->m;
  float tt = *t;
  int guard = 3 * (m->dims[0] + m->dims[1] + m->dims[2]) + 8;
  while (w->live && guard-- > 0) {
    if (w->mj > 0.0f) {
      float dd = w->mj * (w->te - tt); /* optical depth of the cell's stretch */
      if (tau < dd) {
        *t = fminf(tt + tau * w->rj, w->te);
        *maj = w->mj;
        return 1;
      }
      tau = tau - dd;
    }
    tt = w->te;
    if (!(tt < w->t1)) break;
    int a = w->tmax[0] <= w->tmax[1] ? (w->tmax[0] <= w->tmax[2] ? 0 : 2)
                                     : (w->tmax[1] <= w->tmax[2] ? 1 : 2);
    w->c[a] += w->step[a];
    w->tmax[a] = w->tmax[a] + w->tdelta[a];
    if (w->c[a] < 0 || w->c[a] >= m->dims[a])
      w->live = 0;
    else
      walk_enter(w);
  }
  *t = w->t1;
  return 0;
}

/* Test hook: successive flights of the given optical depths along one ray;
 * returns the number of tentative collisions (t_out, maj_out per flight). */
int orc_pt_walk_test(const orc_macro* m, const int vol[3], const float o[3],
                     const float d[3], float t0, float t1, const float* taus,
                     int n_taus, float* t_out, float* maj_out) {
  float e[3], h[3];
  box_extent(vol, e, h);
  pt_walk w;
  walk_init(&w, m, vol, e, h, o, d, t0, t1);
  float t = t0;
  int n = 0;
  for (int i = 0; i < n_taus; ++i) {
    float mj = 0.0f;
    if (!walk_flight(&w, taus[i], &t, &mj)) break;
    t_out[n] = t;
    maj_out[n] = mj;
    ++n;
  }
  return n;
}

static void pt_path(pt_ctx* ctx, const orc_camera* cam, const int vol[3],
                    const orc_march_opts* mo, const double* tf,
                    const orc_pt_opts* pt, const float ls[3], float sbar,
                    uint32_t fseed, int px, int py, double out[4],
                    orc_stats* st) {
  uint32_t pixel = (uint32_t)(py * cam->width + px);
  for (int q = 0; q < 3; ++q) out[q] = (double)pt->ambient[q];
  out[3] = 0.0;
  float o[3], d[3], t0, t1;
  if (!orc_ray(cam, vol, px, py, o, d, &t0, &t1)) return;
  const orc_macro* mac =
      (mo->macro && mo->macro->major && !(pt->sigma_max > 0.0f)) ? mo->macro : NULL;
  float e[3], h[3];
  box_extent(vol, e, h);
  pt_walk W;
  uint64_t key = ((uint64_t)fseed << 32) | (uint64_t)pixel;
  uint32_t rs = orc_ray_seed(fseed, pixel);
  float inv = sbar > 0.0f ? 1.0f / sbar : 0.0f;
  double beta[3] = {1.0, 1.0, 1.0}, L[3] = {0.0, 0.0, 0.0};
  uint32_t j = 0, k = 0;
  for (int b = 0;; ++b) {
    int hit = 0;
    float t = t0, p[3] = {0, 0, 0};
    double v = 0.0;
    if (mac) walk_init(&W, mac, vol, e, h, o, d, t0, t1);
    for (int step = 0; (mac || sbar > 0.0f) && step < PT_MAX_STEPS; ++step) {
      float u = orc_pt_uniform(key, j++);
      float maj = sbar;
      if (mac) {
        if (!walk_flight(&W, orc_neg_log1m(u), &t, &maj)) break;
      } else {
        t = t + orc_neg_log1m(u) * inv;
        if (!(t < t1)) break;
      }
      float x[3], dist;
      pt_point(cam, e, h, o, d, t, p, x, &dist);
      v = pt_lookup(ctx, cam, x, dist, orc_sample_state(rs, k), pixel, k, st);
      ++k;
      double ev[4];
      orc_tf_lookup(tf, v, ev);
      float u2 = orc_pt_uniform(key, j++);
      if ((double)u2 * (double)maj < ev[3]) {
        hit = 1;
        break;
      }
    }
    if (!hit) {
      for (int q = 0; q < 3; ++q) L[q] += beta[q] * (double)pt->ambient[q];
      break;
    }
    if (b == 0) out[3] = 1.0;
    double alb[4];
    orc_tf_lookup(tf, v, alb);
    for (int q = 0; q < 3; ++q) beta[q] *= alb[q];
    /* next-event estimation: shadow transmittance by ratio tracking */
    float ts1 = box_exit(h, p, ls), ts = 0.0f;
    double Tr = 1.0;
    if (mac) walk_init(&W, mac, vol, e, h, p, ls, 0.0f, ts1);
    for (int step = 0; (mac || sbar > 0.0f) && step < PT_MAX_STEPS; ++step) {
      float u = orc_pt_uniform(key, j++);
      float maj = sbar;
      if (mac) {
        if (!walk_flight(&W, orc_neg_log1m(u), &ts, &maj)) break;
      } else {
        ts = ts + orc_neg_log1m(u) * inv;
        if (!(ts < ts1)) break;
      }
      float pq[3], x[3], dist;
      pt_point(cam, e, h, p, ls, ts, pq, x, &dist);
      double v2 = pt_lookup(ctx, cam, x, dist, orc_sample_state(rs, k), pixel, k, st);
      ++k;
      double ev[4];
      orc_tf_lookup(tf, v2, ev);
      Tr *= 1.0 - ev[3] / (double)maj;
    }
    for (int q = 0; q < 3; ++q)
      L[q] += beta[q] * (double)pt->light[q] * Tr / (4.0 * ORC_PI);
    if (b + 1 >= pt->max_bounces) break;
    orc_pt_sphere(key, &j, d);
    for (int q = 0; q < 3; ++q) o[q] = p[q];
    t0 = 0.0f;
    t1 = box_exit(h, o, d);
  }
  for (int q = 0; q < 3; ++q) out[q] = L[q];
}

/* Majorant and direction to the light (binary32, as the GPU's host code). */
static float pt_setup(const double* tf, const orc_pt_opts* pt, float ls[3]) {
  float neg[3] = {-pt->light_dir[0], -pt->light_dir[1], -pt->light_dir[2]};
  normalize3(neg, ls);
  if (pt->sigma_max > 0.0f) return pt->sigma_max;
  float m = 0.0f;
  for (int i = 0; i < 256; ++i) m = fmaxf(m, (float)tf[i * 4 + 3]);
  return m;
}

void orc_render_pt_direct(const orc_inr_params* p, const double* table,
                          const double* w, const orc_camera* cam,
                          const int vol[3], const orc_march_opts* mo,
                          const double* tf, const orc_pt_opts* pt,
                          uint64_t frame, int px0, int py0, int pw, int ph,
                          double* rgba, orc_stats* st) {
  memset(st, 0, sizeof(*st));
  pt_ctx ctx = {NULL, p, table, w, 0u, frame, NULL, NULL};
  ctx.feat = (double*)malloc(sizeof(double) * p->in_dim);
  ctx.act = (double*)malloc(sizeof(double) * 2 * p->hidden);
  float ls[3];
  float sbar = pt_setup(tf, pt, ls);
  uint32_t fseed = orc_frame_seed(mo->seed, frame);
  for (int yy = 0; yy < ph; ++yy)
    for (int xx = 0; xx < pw; ++xx)
      pt_path(&ctx, cam, vol, mo, tf, pt, ls, sbar, fseed, px0 + xx, py0 + yy,
              rgba + ((long)yy * pw + xx) * 4, st);
  free(ctx.feat);
  free(ctx.act);
}

void orc_render_pt_cached(orc_cache* c, const orc_camera* cam, const double* tf,
                          const orc_pt_opts* pt, int px0, int py0, int pw,
                          int ph, double* rgba, orc_stats* st) {
  memset(st, 0, sizeof(*st));
  c->frame += 1;
  uint64_t f = c->frame;
  pt_ctx ctx = {c, &c->p, c->table, c->w, (uint32_t)(1001u * (uint32_t)f), f, NULL, NULL};
  ctx.feat = (double*)malloc(sizeof(double) * c->p.in_dim);
  ctx.act = (double*)malloc(sizeof(double) * 2 * c->p.hidden);
  c->n_miss = 0;
  float ls[3];
  float sbar = pt_setup(tf, pt, ls);
  uint32_t fseed = orc_frame_seed(c->mo.seed, f);
  for (int yy = 0; yy < ph; ++yy)
    for (int xx = 0; xx < pw; ++xx)
      pt_path(&ctx, cam, c->vol, &c->mo, tf, pt, ls, sbar, fseed, px0 + xx,
              py0 + yy, rgba + ((long)yy * pw + xx) * 4, st);
  free(ctx.feat);
  free(ctx.act);
  cache_end_frame(c, ctx.Tf, f, st);
}

void orc_cache_set_macro(orc_cache* c, const orc_macro* m) { c->mo.macro = m; }

long orc_cache_dump(const orc_cache* c, int what, uint32_t* out, long cap) {
  const uint32_t* src = NULL;
  long n = 0;
  long P3 = (long)c->co.page * c->co.page * c->co.page;
  switch (what) {
    case 0:
      if (c->co.page) {
        orc_cache* mc = (orc_cache*)c;
        if (!mc->pt_view) mc->pt_view = (uint32_t*)malloc(sizeof(uint32_t) * (size_t)c->n_bricks);
        for (long k = 0; k < c->n_bricks; ++k) mc->pt_view[k] = pt_get(c, (uint32_t)k);
        src = c->pt_view;
      } else {
        src = c->pt;
      }
      n = c->n_bricks;
      break;
    case 8: src = c->pd; n = c->co.page ? c->pd_off[c->co.levels] : 0; break;
    case 9: src = c->pages; n = c->co.page ? c->co.n_pages * P3 : 0; break;
    case 10: src = c->page_key; n = c->co.page ? c->co.n_pages : 0; break;
    case 11: src = c->page_ref; n = c->co.page ? c->co.n_pages : 0; break;
    case 1: src = c->stamp; n = c->co.n_slots; break;
    case 2: src = c->owner; n = c->co.n_slots; break;
    case 3: src = c->rank; n = c->n_bricks; break;
    case 4: src = c->last_req; n = c->n_last_req; break;
    case 5: src = c->last_vict; n = c->n_last_vict; break;
    case 6: src = c->miss; n = 2 * c->n_miss; break;
    case 7: src = c->pinned; n = c->co.n_slots; break;
    default: return -1;
  }
  long m = n < cap ? n : cap;
  if (out && m > 0) memcpy(out, src, sizeof(uint32_t) * (size_t)m);
  return n;
}

void orc_cache_slot_values(const orc_cache* c, long slot, double* out) {
  long S3 = (long)c->S * c->S * c->S;
  memcpy(out, c->pool + slot * S3, sizeof(double) * (size_t)S3);
}

/* PSNR over RGB of premultiplied images on black, peak 1.0. */
double orc_psnr(const double* a, const double* b, long n_pixels) {
  double se = 0.0;
  for (long i = 0; i < n_pixels; ++i)
    for (int c = 0; c < 3; ++c) {
      double d = a[i * 4 + c] - b[i * 4 + c];
      se += d * d;
    }
  double mse = se / (double)(n_pixels * 3);
  if (mse <= 0.0) return INFINITY;
  return 10.0 * log10(1.0 / mse);
}

/* ===================================================================== */
/* Training (Sec. 4.1)                                                     */
/* ===================================================================== */

/* Ground truth at a random coordinate: trilinear interpolation of the
 * explicit field stored at voxel centres (i + 0.5)/V, clamp-to-edge. */
double orc_field_trilinear(const float* field, const int dims[3],
                           const float x[3]) {
  int i0[3], i1[3];
  float f[3];
  for (int a = 0; a < 3; ++a) {
    float q = clamp01(x[a]) * (float)dims[a] - 0.5f;
    q = fminf(fmaxf(q, 0.0f), (float)(dims[a] - 1));
    i0[a] = (int)floorf(q);
    f[a] = q - (float)i0[a];
    i1[a] = i0[a] + 1 > dims[a] - 1 ? dims[a] - 1 : i0[a] + 1;
  }
  double v = 0.0;
  for (int c = 0; c < 8; ++c) {
    double wc = 1.0;
    int ix[3];
    for (int a = 0; a < 3; ++a) {
      int bit = (c >> a) & 1;
      wc *= bit ? (double)f[a] : 1.0 - (double)f[a];
      ix[a] = bit ? i1[a] : i0[a];
    }
    v += wc * (double)field[((long)ix[2] * dims[1] + ix[1]) * dims[0] + ix[0]];
  }
  return v;
}

/* Mean squared error of the raw network output y against normalised targets
 * over a batch, and its exact gradient with respect to every table entry and
 * weight (back-propagation through the MLP, then through the trilinear
 * hash-grid interpolation, accumulated per table entry). */
double orc_loss_grad(const orc_inr_params* p, const double* table,
                     const double* w, const float* xyz, const double* target,
                     long n, double* g_table, double* g_w) {
  int L = p->levels, F = p->feats, H = p->hidden, I = p->in_dim;
  int NH = p->n_hidden_layers;
  long T = 1L << p->log2_table;
  long nw = orc_mlp_param_count(p);
  memset(g_table, 0, sizeof(double) * (size_t)(L * T * F));
  memset(g_w, 0, sizeof(double) * (size_t)nw);
  double* feat = (double*)malloc(sizeof(double) * I);
  double* acts = (double*)malloc(sizeof(double) * (size_t)(NH * H));
  double* delta = (double*)malloc(sizeof(double) * H);
  double* dprev = (double*)malloc(sizeof(double) * (H > I ? H : I));
  double loss = 0.0;
  for (long j = 0; j < n; ++j) {
    const float* x = xyz + 3 * j;
    encode_one(p, table, x, feat);
    /* forward, keeping post-ReLU activations of each hidden layer */
    for (int o = 0; o < H; ++o) {
      double s = 0.0;
      for (int i = 0; i < I; ++i) s += w[(long)o * I + i] * feat[i];
      acts[o] = s > 0.0 ? s : 0.0;
    }
    const double* wl = w + (long)H * I;
    for (int layer = 1; layer < NH; ++layer) {
      for (int o = 0; o < H; ++o) {
        double s = 0.0;
        for (int i = 0; i < H; ++i) s += wl[(long)o * H + i] * acts[(layer - 1) * H + i];
        acts[layer * H + o] = s > 0.0 ? s : 0.0;
      }
      wl += (long)H * H;
    }
    const double* wout = wl;
    double y = 0.0;
    for (int i = 0; i < H; ++i) y += wout[i] * acts[(NH - 1) * H + i];
    double r = y - target[j];
    loss += r * r;
    double dy = 2.0 * r / (double)n;
    /* backward: output layer */
    double* gout = g_w + (wout - w);
    for (int i = 0; i < H; ++i) {
      gout[i] += dy * acts[(NH - 1) * H + i];
      delta[i] = acts[(NH - 1) * H + i] > 0.0 ? dy * wout[i] : 0.0;
    }
    /* hidden layers NH-1 .. 1 */
    for (int layer = NH - 1; layer >= 1; --layer) {
      const double* wh = w + (long)H * I + (long)(layer - 1) * H * H;
      double* gh = g_w + (wh - w);
      for (int o = 0; o < H; ++o)
        for (int i = 0; i < H; ++i) gh[(long)o * H + i] += delta[o] * acts[(layer - 1) * H + i];
      for (int i = 0; i < H; ++i) {
        double s = 0.0;
        for (int o = 0; o < H; ++o) s += wh[(long)o * H + i] * delta[o];
        dprev[i] = acts[(layer - 1) * H + i] > 0.0 ? s : 0.0;
      }
      memcpy(delta, dprev, sizeof(double) * H);
    }
    /* first layer */
    for (int o = 0; o < H; ++o)
      for (int i = 0; i < I; ++i) g_w[(long)o * I + i] += delta[o] * feat[i];
    for (int i = 0; i < I; ++i) {
      double s = 0.0;
      for (int o = 0; o < H; ++o) s += w[(long)o * I + i] * delta[o];
      dprev[i] = s; /* d loss / d feature i */
    }
    /* hash grid: each feature is a trilinear blend of 8 table entries */
    float xc[3] = {clamp01(x[0]), clamp01(x[1]), clamp01(x[2])};
    for (int l = 0; l < L; ++l) {
      int N = level_res(p, l);
      int i3[3];
      float w3[3];
      for (int a = 0; a < 3; ++a) grid_cell(xc[a], N, &i3[a], &w3[a]);
      for (int c = 0; c < 8; ++c) {
        double wc = 1.0;
        for (int a = 0; a < 3; ++a) {
          int bit = (c >> a) & 1;
          wc *= bit ? (double)w3[a] : 1.0 - (double)w3[a];
        }
        uint32_t id = orc_vertex_index(p, l, (uint32_t)(i3[0] + (c & 1)),
                                       (uint32_t)(i3[1] + ((c >> 1) & 1)),
                                       (uint32_t)(i3[2] + ((c >> 2) & 1)));
        double* g = g_table + ((long)l * T + (long)id) * F;
        for (int f = 0; f < F; ++f) g[f] += wc * dprev[l * F + f];
      }
    }
  }
  free(feat);
  free(acts);
  free(delta);
  free(dprev);
  return loss / (double)n;
}

/* Adam (Kingma & Ba 2015), bias-corrected, step counted from 1. */
void orc_adam(double* param, const double* grad, double* m, double* v, long n,
              double lr, double b1, double b2, double eps, long step) {
  double c1 = 1.0 - pow(b1, (double)step);
  double c2 = 1.0 - pow(b2, (double)step);
  for (long i = 0; i < n; ++i) {
    m[i] = b1 * m[i] + (1.0 - b1) * grad[i];
    v[i] = b2 * v[i] + (1.0 - b2) * grad[i] * grad[i];
    double mh = m[i] / c1;
    double vh = v[i] / c2;
    param[i] -= lr * mh / (sqrt(vh) + eps);
  }
}

/* One training step (Sec. 4.1): a batch of counter-based random coordinates
 * (elements step*batch .. step*batch+batch-1), ground truth by trilinear
 * lookup normalised to [0,1] with the field range, MSE gradient, Adam on the
 * table and on the weights.  `step` counts from 1. */
double orc_train_step(const orc_inr_params* p, double* table, double* w,
                      double* m_t, double* v_t, double* m_w, double* v_w,
                      const float* field, const int dims[3], double fmin,
                      double fmax, long batch, uint64_t seed, long step,
                      double lr, double b1, double b2, double eps) {
  long T = 1L << p->log2_table;
  long nt = (long)p->levels * T * p->feats;
  long nw = orc_mlp_param_count(p);
  float* xyz = (float*)malloc(sizeof(float) * 3 * (size_t)batch);
  double* tg = (double*)malloc(sizeof(double) * (size_t)batch);
  double* gt = (double*)malloc(sizeof(double) * (size_t)nt);
  double* gw = (double*)malloc(sizeof(double) * (size_t)nw);
  orc_uniform_coords(seed, (uint64_t)(step - 1) * (uint64_t)batch, batch, xyz);
  for (long j = 0; j < batch; ++j)
    tg[j] = (orc_field_trilinear(field, dims, xyz + 3 * j) - fmin) / (fmax - fmin);
  double loss = orc_loss_grad(p, table, w, xyz, tg, batch, gt, gw);
  orc_adam(table, gt, m_t, v_t, nt, lr, b1, b2, eps, step);
  orc_adam(w, gw, m_w, v_w, nw, lr, b1, b2, eps, step);
  free(xyz);
  free(tg);
  free(gt);
  free(gw);
  return loss;
}
