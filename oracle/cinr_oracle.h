/*
 * CPU FP64 oracle of the cache-accelerated INR volume renderer
 * ("From Cluster to Desktop", arXiv 2504.18001).
 *
 * TEST INFRASTRUCTURE ONLY.  Only tests/, __graft_entry__.smoke() and the
 * cpu_baseline / reference legs of bench.py may load this library.  It shares
 * no code, header, table or constant generator with the CUDA path; it follows
 * the paper step by step in plain C:
 *   - continuous values (hash-grid features, MLP, trilinear, transfer function,
 *     compositing) in FP64;
 *   - every quantity that feeds a floor, a comparison or a hash (ray origin and
 *     direction, sample parameter t, positions, grid coordinates) in IEEE
 *     binary32 with round-to-nearest and no FMA contraction (the library is
 *     compiled with -ffp-contract=off), so that discrete decisions (LoD, brick,
 *     hash index, miss or hit) are reproducible bit for bit.
 * Function-level comments cite the paper section / algorithm each follows.
 * Parity pins are listed in the module docstring of oracle/__init__.py.
 */
#ifndef CINR_ORACLE_H
#define CINR_ORACLE_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* INR hyper-parameters (Sec. 3, Fig. 2: m levels, n features per level,
 * fixed-size hash table per level; small MLP; value range of Sec. 4.1). */
typedef struct {
  int levels;          /* m */
  int feats;           /* n (features per level) */
  int log2_table;      /* table size T = 2^log2_table entries per level */
  int base_res;        /* coarsest grid resolution */
  double growth;       /* per-level resolution growth factor */
  int in_dim;          /* = levels * feats */
  int hidden;          /* MLP width */
  int n_hidden_layers; /* number of hidden (ReLU) layers, >= 1 */
  double vmin, vmax;   /* de-normalisation v = vmin + (vmax - vmin) * y */
} orc_inr_params;

typedef struct {
  float eye[3], target[3], up[3];
  float fov_y_deg;
  int width, height;
  float step_voxels;   /* step in LoD-0 voxels */
} orc_camera;

typedef struct {
  int K;               /* samples per wavefront segment */
  float eps_T;         /* early termination threshold on transmittance */
  int lod_mode;        /* 0 = screen footprint, 1 = distance (Alg. 2) */
  float lod_scale;
  uint64_t seed;       /* per-run seed of the per-frame dither seed */
  int step_mode;       /* 0 fixed step, 1 LoD-scaled 32-sample segments */
  int step_lod_max;    /* highest LoD that scales the step (mode 1) */
  const struct orc_macro* macro; /* macro-cell skip flags, NULL = off */
} orc_march_opts;

/* Path-tracing options (Sec. 5.1, Woodcock delta tracking). */
typedef struct {
  float light_dir[3]; /* direction the directional light travels */
  float light[3];     /* its irradiance (rgb) */
  float ambient[3];   /* radiance of paths leaving the volume (rgb) */
  int max_bounces;    /* scattering events per path, >= 1 */
  float sigma_max;    /* majorant of the extinction; <= 0: max of the TF */
} orc_pt_opts;

/* Macro cells (Sec. 5.2): ceil(V/cell) cubes per axis; skip[c] = 1 when the
 * current transfer function is transparent over cell c's value range. */
typedef struct orc_macro {
  int cell;            /* edge in LoD-0 voxels */
  int dims[3];         /* cells per axis */
  const uint8_t* skip; /* one flag per cell, x fastest */
  const float* major;  /* per-cell extinction majorant for path tracing
                          (orc_macro_majorant), NULL = the TF's maximum */
} orc_macro;

typedef struct {
  float ts, dts;       /* segment start and step (schedule state of a ray) */
} orc_sched;

typedef struct {
  uint64_t samples, inr_queries_direct, inr_queries_decode, true_misses,
      fallback_hits, hits, bricks_requested, bricks_decoded, evictions,
      samples_skipped;
} orc_stats;

/* ---- random generators (published definitions) ---- */
uint64_t orc_splitmix64(uint64_t x);
uint32_t orc_xorshift32(uint32_t s);
void orc_uniform_coords(uint64_t seed, uint64_t first, long n, float* xyz);

/* ---- INR (Sec. 3, Fig. 2) ---- */
long orc_mlp_param_count(const orc_inr_params* p);
void orc_level_res(const orc_inr_params* p, int* res);
int orc_level_is_dense(const orc_inr_params* p, int level);
uint32_t orc_vertex_index(const orc_inr_params* p, int level, uint32_t ix,
                          uint32_t iy, uint32_t iz);
void orc_encode_indices(const orc_inr_params* p, const float* xyz, long n,
                        uint32_t* idx /* n * levels * 8 */);
void orc_encode(const orc_inr_params* p, const double* table, const float* xyz,
                long n, double* feats /* n * levels * feats */);
void orc_mlp(const orc_inr_params* p, const double* w, const double* feats,
             long n, double* y);
void orc_inr_eval(const orc_inr_params* p, const double* table,
                  const double* w, const float* xyz, long n, double* v);
void orc_inr_raw_range(const orc_inr_params* p, const double* table,
                       const double* w, const int vol[3], int stride,
                       double* ymin, double* ymax);

/* ---- rays, sample schedule, LoD (Sec. 5.1, Sec. 5.3, Alg. 2) ---- */
int orc_ray(const orc_camera* cam, const int vol[3], int px, int py, float o[3],
            float d[3], float* tn, float* tf);
int orc_sample(const orc_camera* cam, const int vol[3], const float o[3],
               const float d[3], float tn, float tf, int k, float x[3],
               float* t_mid, float* seg_len);
int orc_sample_sched(const orc_camera* cam, const int vol[3],
                     const orc_march_opts* mo, const float o[3],
                     const float d[3], float tn, float tf, int k,
                     orc_sched* s, float x[3], float* t_mid,
                     float* seg_len);
int orc_sample_lod(const orc_camera* cam, const int vol[3],
                   const orc_march_opts* mo, int levels, int lod_min,
                   uint32_t state, float t_mid);
uint32_t orc_frame_seed(uint64_t seed, uint64_t frame);
uint32_t orc_ray_seed(uint32_t frame_seed, uint32_t pixel);
uint32_t orc_sample_state(uint32_t ray_seed, uint32_t k);

/* ---- transfer function and compositing (Sec. 3, Sec. 5.1) ---- */
void orc_tf_lookup(const double* tf /* 256*4 */, double v, double out[4]);

/* ---- cache-off render = direct INR rendering (Alg. 1 with every sample a
 *      miss; the uncached baseline of Sec. 6) ---- */
void orc_render_direct(const orc_inr_params* p, const double* table,
                       const double* w, const orc_camera* cam,
                       const int vol[3], const orc_march_opts* mo,
                       const double* tf, int px0, int py0, int pw, int ph,
                       double* rgba /* pw*ph*4 */, orc_stats* st);

/* Explicit-voxel render (values by trilinear interpolation of the field). */
void orc_render_field(const float* field, const int fdims[3],
                      const orc_camera* cam, const int vol[3],
                      const orc_march_opts* mo, const double* tf, int px0,
                      int py0, int pw, int ph, double* rgba, orc_stats* st);

/* ---- macro cells for adaptive sampling (Sec. 5.2) ---- */
void orc_macro_dims(const int vol[3], int cell, int out[3]);
/* Value range of each cell: min and max over every LoD-l voxel (l in
 * [min_level, levels)) that a trilinear sample inside the cell can read,
 * INR values at the voxel centres; float pairs rounded outwards. */
void orc_macro_ranges_inr(const orc_inr_params* p, const double* table,
                          const double* w, const int vol[3], int cell,
                          int levels, int min_level, float* ranges);
/* The same over the voxels of an explicit field (LoD 0). */
void orc_macro_ranges_field(const float* field, const int dims[3], int cell,
                            float* ranges);
/* Skip flags of a transfer function (256 x rgba, a = extinction). */
void orc_macro_skip(const float* ranges, long n_cells, const double* tf,
                    uint8_t* skip);
long orc_macro_cell_of(const orc_macro* m, const int vol[3], const float x[3]);
void orc_macro_majorant(const float* ranges, long n_cells, const double* tf,
                        float* major);
int orc_pt_walk_test(const orc_macro* m, const int vol[3], const float o[3],
                     const float d[3], float t0, float t1, const float* taus,
                     int n_taus, float* t_out, float* maj_out);

/* ---- multi-resolution brick cache (Sec. 4.3) ---- */
typedef struct orc_cache orc_cache;
typedef struct {
  int brick;         /* B, interior edge; stored (B+2)^3 with a 1-voxel apron */
  int levels;        /* number of LoDs */
  long n_slots;      /* bricks the pool holds */
  int n_req;         /* maxNumRequests per frame */
  int ranking;       /* 1 = priority ranking (Sec. 4.3.3), 0 = first-n */
  int preload;       /* 1 = decode + pin every coarsest brick at creation */
  int lag;           /* frames from request to use: 1 (default) or 2 */
  int page;          /* 0: flat page tables; P > 0: virtualised 2-level
                        tables, pages of P^3 bricks (Sec. 4.3.1) */
  long n_pages;      /* PT pages the page pool holds (page > 0) */
} orc_cache_opts;

orc_cache* orc_cache_create(const orc_inr_params* p, const double* table,
                            const double* w, const int vol[3],
                            const orc_cache_opts* co, const orc_march_opts* mo);
void orc_cache_destroy(orc_cache* c);
long orc_cache_num_bricks(const orc_cache* c);
long orc_cache_level_offset(const orc_cache* c, int level);
void orc_cache_level_dims(const orc_cache* c, int level, int dims[3],
                          int nb[3]);
/* Macro-cell skip flags used by the following renders (NULL = off). */
void orc_cache_set_macro(orc_cache* c, const orc_macro* m);
void orc_render_cached(orc_cache* c, const orc_camera* cam, const double* tf,
                       int px0, int py0, int pw, int ph, double* rgba,
                       orc_stats* st);
/* Path-traced frame through the cache (requests, stamps, end-of-frame
 * update as for orc_render_cached). */
void orc_render_pt_cached(orc_cache* c, const orc_camera* cam, const double* tf,
                          const orc_pt_opts* pt, int px0, int py0, int pw,
                          int ph, double* rgba, orc_stats* st);
/* what: 0 page table (u32 per brick; paged: the entries the two levels
 *       resolve to), 1 slot stamps (u32 per slot),
 *       2 slot owners (u32 per slot), 3 rank (u32 per brick),
 *       4 last requests (u32 keys), 5 last victims (u32 slots),
 *       6 last true-miss list (u32 pairs pixel,k), 7 pinned (u32 per slot),
 *       8 page directory (u32 per page: Mapped | page slot),
 *       9 page pool (u32 per entry, n_pages * P^3),
 *       10 page slot keys (u32 per page slot), 11 page refcounts.
 * Returns the element count; copies min(count, cap) elements. */
long orc_cache_dump(const orc_cache* c, int what, uint32_t* out, long cap);
void orc_cache_slot_values(const orc_cache* c, long slot, double* out);

/* Brick contents for (level, brick id): (B+2)^3 INR values at the LoD-l voxel
 * centres with clamp-to-edge (Sec. 4.3.2). */
void orc_brick_values(const orc_inr_params* p, const double* table,
                      const double* w, const int vol[3], int brick, int level,
                      int bx, int by, int bz, double* out);
/* Brick origin: first stored voxel centre, LoD-0 voxel-edge coordinates. */
void orc_brick_origin(const int vol[3], int brick, int level, int bx, int by,
                      int bz, double origin[3]);
/* One LoD-l sample served from the brick that holds it (no cache state). */
double orc_brick_sample(const orc_inr_params* p, const double* table,
                        const double* w, const int vol[3], int brick, int level,
                        const float x[3]);
/* Fully resident reference: trilinear reconstruction of INR values at the
 * LoD-l voxel centres (clamp-to-edge) at normalised position x. */
double orc_resident_sample(const orc_inr_params* p, const double* table,
                           const double* w, const int vol[3], int level,
                           const float x[3]);

/* ---- path tracing with Woodcock delta tracking (Sec. 5.1) ---- */

/* -ln(1 - u) in binary32 (fixed operation order, +,-,*,/ only). */
float orc_neg_log1m(float u);
/* j-th uniform of the SplitMix64 stream seeded with key: top 24 bits. */
float orc_pt_uniform(uint64_t key, uint32_t j);
/* Uniform direction on the sphere (Marsaglia 1972) from the stream. */
void orc_pt_sphere(uint64_t key, uint32_t* j, float dir[3]);
/* One path per pixel of frame `frame`; lookups by direct INR inference. */
void orc_render_pt_direct(const orc_inr_params* p, const double* table,
                          const double* w, const orc_camera* cam,
                          const int vol[3], const orc_march_opts* mo,
                          const double* tf, const orc_pt_opts* pt,
                          uint64_t frame, int px0, int py0, int pw, int ph,
                          double* rgba, orc_stats* st);

double orc_psnr(const double* a, const double* b, long n_pixels);

/* ---- training (Sec. 4.1) ---- */
double orc_field_trilinear(const float* field, const int dims[3],
                           const float x[3]);
double orc_loss_grad(const orc_inr_params* p, const double* table,
                     const double* w, const float* xyz, const double* target,
                     long n, double* g_table, double* g_w);
void orc_adam(double* param, const double* grad, double* m, double* v, long n,
              double lr, double b1, double b2, double eps, long step);
double orc_train_step(const orc_inr_params* p, double* table, double* w,
                      double* m_t, double* v_t, double* m_w, double* v_w,
                      const float* field, const int dims[3], double fmin,
                      double fmax, long batch, uint64_t seed, long step,
                      double lr, double b1, double b2, double eps);

#ifdef __cplusplus
}
#endif
#endif
