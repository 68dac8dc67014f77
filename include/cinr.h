/*
 * cinr.h -- C ABI of the GB300 cache-accelerated INR volume renderer
 * (arXiv 2504.18001, "From Cluster to Desktop: A Cache-Accelerated INR
 * framework for Interactive Visualization of Tera-Scale Data").
 *
 * Conventions shared by every call
 *  - Every call returns an int status: CINR_OK (0) or a negative CINR_ERR_*.
 *    cinr_last_error() gives the message of the last failure on the calling
 *    thread.  No C++ exception crosses this boundary.
 *  - The caller owns all device memory.  The library never allocates device
 *    memory: every object lives inside a caller-provided device buffer whose
 *    size is returned by the matching *_bytes() query.  Buffers must be
 *    256-byte aligned and stay valid until the object is destroyed.  Handle
 *    structs themselves are small host allocations owned by the library and
 *    released by cinr_destroy_*().
 *  - Pointers named *_dev are device pointers; *_host are host pointers.
 *  - `stream` is a cudaStream_t passed as void* (NULL = legacy default
 *    stream).  Calls enqueue work on it and return without synchronising,
 *    except where a call says that it synchronises.
 *  - One device: every object is bound to the device that was current when
 *    it was created.
 */
#ifndef CINR_H
#define CINR_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ------------------------------------------------------------- status --- */
#define CINR_OK 0
#define CINR_ERR_ARG (-1)          /* invalid argument or unsupported shape */
#define CINR_ERR_NOMEM (-2)        /* caller buffer smaller than required   */
#define CINR_ERR_CUDA (-3)         /* a CUDA runtime call failed             */
#define CINR_ERR_TIMEOUT (-4)      /* a bounded device-side wait gave up     */
#define CINR_ERR_DEVICE_CHECK (-5) /* a device-side bounds check tripped     */
#define CINR_ERR_UNSUPPORTED (-6)  /* valid request this build cannot run    */
#define CINR_ERR_NAN (-7)          /* a training step met a non-finite value */

/* -------------------------------------------------------------- types --- */
typedef struct cinr_inr_s* cinr_inr_t;
typedef struct cinr_cache_s* cinr_cache_t;
typedef struct cinr_renderer_s* cinr_renderer_t;
typedef struct cinr_trainer_s* cinr_trainer_t;
typedef struct cinr_macro_s* cinr_macro_t;
typedef void* cinr_stream_t;

#define CINR_PREC_FP32 0
#define CINR_PREC_FP16 1
#define CINR_PREC_BF16 2
#define CINR_PREC_FP8 3 /* MLP only: E4M3 operands, FP32 accumulation (trial) */
/* Cache storage only: FP16 bricks laid out as z-slices in a pitched 2D
 * image (a power-of-two number of slice blocks per row, at most 16384
 * texels wide, at most 65000 rows), sampled by the texture units: the
 * specialised marching kernel (fixed steps, footprint LoD, flat page
 * tables, no macro cells, preloaded coarsest LoD, bricks of 8^3 or 16^3,
 * one ray per thread) reads a sample as two hardware-bilinear fetches and
 * one z-lerp.  The hardware's bilinear weights carry 8 fractional bits, so
 * values differ from the FP16 layout's FP32 trilinear by up to 2^-9 of the
 * neighbouring voxels' difference.  Other kernels reject such a cache
 * (CINR_ERR_UNSUPPORTED); a pool beyond the row limit is CINR_ERR_ARG. */
#define CINR_PREC_FP16_TEX 4

/* INR hyper-parameters: a multiresolution hash-grid encoder (m levels, n
 * features per level, a table of 2^log2_table entries per level) feeding a
 * small ReLU MLP with a linear scalar output (Sec. 3, Fig. 2), and the value
 * range used to de-normalise the output, v = vmin + (vmax - vmin) * y
 * (Sec. 4.1).  Level l has N_l = floor(base_res * growth^l) cells per axis;
 * a level whose (N_l+1)^3 vertices fit in the table is indexed densely, the
 * others by the Instant-NGP spatial hash.
 * Supported shapes: feats = 2; (levels*feats, hidden) in {(16,32), (32,64),
 * (48,64)}; n_hidden_layers = 2; levels <= 32; log2_table <= 24. */
typedef struct {
  int levels;
  int feats;
  int log2_table;
  int base_res;
  double growth;
  int hidden;
  int n_hidden_layers;
  int mlp_precision;   /* CINR_PREC_FP32 | FP16 | BF16 (FP32 accumulate) */
  int table_precision; /* CINR_PREC_FP32 | FP16                           */
  float vmin, vmax;
} cinr_inr_params;

/* Camera: pinhole, vertical field of view, one primary ray per pixel centre
 * (ray-generation kernel, Sec. 5.1).  The volume occupies the box
 * [-e/2, e/2] with e = dims / max(dims), centred at the origin.
 * step_voxels is the ray-marching step in LoD-0 voxels. */
typedef struct {
  float eye[3], target[3], up[3];
  float fov_y_deg;
  int width, height;
  float step_voxels;
} cinr_camera;

/* Transfer function: 256 entries of (r, g, b, sigma); x = clamp(v,0,1)*255
 * is interpolated linearly between entries; sigma is the extinction per
 * world unit (Sec. 3: each sample is classified by a transfer function). */
typedef struct {
  float rgba[256][4];
} cinr_tf;

/* Ray-marching options.  dims = the rendered volume grid in LoD-0 voxels
 * (sets the box aspect and the voxel size; must equal the cache's dims when
 * a cache is used).  K (a multiple of 32) is the wavefront segment:
 * termination (T < eps_T) is tested only after every K samples of a ray.
 * lod_mode 0 = pixel-footprint LoD, 1 = distance LoD (Alg. 2); lod_scale
 * is the user LoD scale (Sec. 4.3.4, Sec. 5.3); seed seeds the per-frame
 * xorshift dither (Sec. 5.3).  miss_record_cap > 0 keeps the first
 * miss_record_cap true misses of each frame as (pixel, sample) pairs for
 * cinr_debug_dump (CINR_DUMP_MISSES).  ray_layout selects how cached frames
 * map rays to threads: 0 = one ray per thread (tiles of 32 neighbouring
 * rays per warp), 1 = one ray per warp (32-sample segments per warp); both
 * produce the same sample set and cache state.  Uncached frames always use
 * one ray per warp (128-sample batches feed the tensor-core MLP).
 * step_mode 0 steps every sample by step_voxels; step_mode 1 scales the
 * step with distance for tera-scale volumes: segments of 32 samples, segment
 * s starting at t_s (t_0 = t_near, t_{s+1} = t_s + 32 dt_s) with step
 * dt_s = dt 2^l, l the undithered LoD at t_s clamped to [0, step_lod_max]. */
typedef struct {
  int dims[3];
  int K;
  float eps_T;
  int lod_mode;
  float lod_scale;
  uint64_t seed;
  long miss_record_cap;
  int ray_layout;
  int step_mode;
  int step_lod_max;
  int use_graph; /* 1: each frame's launch sequence runs as a CUDA graph */
} cinr_march_opts;

/* Cache options (Sec. 4.3): brick = interior edge B (stored with a one-voxel
 * apron, (B+2)^3 voxels); levels = number of LoDs; n_req = maxNumRequests
 * per frame (Sec. 6.4); ranking = 1 for the priority ranking of
 * Sec. 4.3.3, 0 for first-n by brick key; preload = 1 decodes and pins
 * every brick of the coarsest LoD at creation (Sec. 4.3.4);
 * storage_precision = CINR_PREC_FP32 | CINR_PREC_FP16 for brick voxels;
 * lag = frames from a request to its first use: 1 (0 means 1): the bricks
 * selected at the end of frame f are decoded on the frame's stream and serve
 * frame f+1; 2: asynchronous request handling (Sec. 4.3.3, after Sarton's
 * request handler) -- the selected bricks' slots are unmapped at the end of
 * frame f, decoded on a second stream while frame f+1 renders, and mapped at
 * the end of frame f+1 (before its own selection, which skips bricks mapped
 * that way), serving frame f+2.  Both are deterministic.  A lag-2 cache
 * cannot be used with use_graph.
 * page = 0: one page-table entry per brick (flat tables).  page = P (a power
 * of two, 1..16): virtualised two-level page tables (Sec. 4.3.1) -- per LoD
 * a page directory over pages of P^3 bricks, resident pages held in a pool
 * of n_pages page slots; a brick whose page is not resident reads as
 * Unmapped.  At the end of a frame the victims are unmapped first, the
 * pages left without a mapped brick are freed, the pages the new mappings
 * need are allocated (ascending page key into ascending free page slots)
 * and the bricks are mapped; a brick whose page finds no free slot is
 * dropped for the frame (its victim slot stays free).  n_pages must hold
 * at least the coarsest LoD's pages when preload = 1. */
typedef struct {
  int brick;
  int levels;
  int n_req;
  int ranking;
  int preload;
  int storage_precision;
  int lag;
  int page;
  long n_pages;
} cinr_cache_opts;

/* Per-frame counters.  samples = samples marched; inr_queries_direct = true
 * misses inferred in the frame; inr_queries_decode = voxels decoded into
 * bricks; hits = served at the requested LoD; fallback_hits = served by a
 * coarser LoD (Sec. 4.3); true_misses = no LoD mapped (Alg. 2);
 * bricks_requested = distinct bricks requested; bricks_decoded = bricks
 * written back; evictions = decoded bricks that replaced a resident one;
 * misses_recorded = entries of the miss record (capped); slots_touched =
 * distinct pool slots that served samples; kernel_launches = kernels the
 * library launched for the frame; samples_skipped = samples in macro cells
 * that are transparent under the frame's transfer function (not counted in
 * samples; no lookup, request or inference).  ms_frame_kernel and ms_cache_update are
 * device times (CUDA events on the frame's stream) of the marching kernel
 * and of the end-of-frame cache update. */
typedef struct {
  uint64_t samples, inr_queries_direct, inr_queries_decode, true_misses,
      fallback_hits, hits, bricks_requested, bricks_decoded, evictions,
      misses_recorded, slots_touched, kernel_launches, samples_skipped;
  float ms_frame_kernel, ms_cache_update;
} cinr_frame_stats;

/* ----------------------------------------------------------- library --- */

/* Message of the last failed call on this thread (NUL-terminated, truncated
 * to n bytes).  Returns CINR_OK. */
int cinr_last_error(char* buf, size_t n);

/* Library ABI version (major * 100 + minor). */
int cinr_version(void);

/* ---------------------------------------------------------------- INR --- */

/* Device bytes an INR with these parameters occupies.  Host-only.
 * Errors: CINR_ERR_ARG for unsupported shapes. */
int cinr_inr_bytes(const cinr_inr_params* p, size_t* bytes);

/* Creates an INR (Sec. 3, Fig. 2) inside dev_mem (>= cinr_inr_bytes).
 * host_table: levels * 2^log2_table * feats floats, level-major then entry
 * then feature.  host_mlp: the MLP weights, layer by layer, each row-major
 * [out][in] (in -> hidden, hidden -> hidden, hidden -> 1; no biases).
 * Both are copied (and converted to the requested precisions) on `stream`;
 * the call synchronises the stream before returning so that the host arrays
 * may be freed.  Errors: CINR_ERR_ARG, CINR_ERR_NOMEM, CINR_ERR_CUDA. */
int cinr_create_inr(const cinr_inr_params* p, void* dev_mem, size_t bytes,
                    const float* host_table, const float* host_mlp,
                    cinr_stream_t stream, cinr_inr_t* out);

/* Sets the de-normalisation range v = vmin + (vmax - vmin) * y (Sec. 4.1). */
int cinr_inr_set_range(cinr_inr_t inr, float vmin, float vmax);

/* Minimum and maximum of the raw network output y over the LoD-0 voxel
 * centres ((i+0.5)/dims) of a dims grid, every `stride`-th voxel per axis.
 * Used to normalise an untrained network to [0,1] (Sec. 4.1 keeps the exact
 * value range of the data).  Synchronises `stream`. */
int cinr_inr_raw_range(cinr_inr_t inr, const int dims[3], int stride,
                       float* ymin, float* ymax, cinr_stream_t stream);

/* Direct INR inference ("InferINR", Alg. 1): v[i] = INR(xyz[i]) for n points
 * xyz_dev (n x 3 floats, normalised [0,1]^3, clamped) into out_dev (n
 * floats).  n = 0 is a no-op. */
int cinr_infer(cinr_inr_t inr, const float* xyz_dev, long n, float* out_dev,
               cinr_stream_t stream);

/* Hash-grid encoding only (Sec. 3): feats_dev (n x levels*feats floats) and,
 * when idx_dev is not NULL, the 8 table indices per level and point
 * (n x levels x 8 u32, corner c = x + 2y + 4z offset bits). */
int cinr_encode(cinr_inr_t inr, const float* xyz_dev, long n, float* feats_dev,
                uint32_t* idx_dev, cinr_stream_t stream);

int cinr_destroy_inr(cinr_inr_t inr);

/* -------------------------------------------------------------- cache --- */

/* Device bytes of a brick cache over a dims volume whose brick pool holds
 * pool_bytes of voxel data.  Host-only.  n_slots (may be NULL) receives the
 * number of bricks the pool holds. */
int cinr_cache_bytes(const int dims[3], size_t pool_bytes,
                     const cinr_cache_opts* o, size_t* bytes, long* n_slots);

/* Creates the multi-resolution brick cache of Sec. 4.3 in dev_mem: flat
 * per-LoD page tables (Mapped | slot, or Unmapped; Sec. 4.3.1), the brick
 * pool, per-brick ranks (Sec. 4.3.3), per-slot LRU stamps and owners.  With
 * preload, every coarsest-LoD brick is decoded by INR inference into slots
 * 0.. and pinned (Sec. 4.3.4).  Errors: CINR_ERR_NOMEM when the pool cannot
 * hold the coarsest LoD with preload, CINR_ERR_ARG for bad shapes. */
int cinr_create_cache(cinr_inr_t inr, const int dims[3], void* dev_mem,
                      size_t bytes, size_t pool_bytes, const cinr_cache_opts* o,
                      cinr_stream_t stream, cinr_cache_t* out);

int cinr_destroy_cache(cinr_cache_t cache);

/* ----------------------------------------------------------- renderer --- */

/* Device bytes of the per-frame working set for width x height frames. */
int cinr_renderer_bytes(int width, int height, const cinr_march_opts* o,
                        size_t* bytes);

int cinr_create_renderer(void* dev_mem, size_t bytes, int width, int height,
                         const cinr_march_opts* o, cinr_renderer_t* out);

/* Renders one frame (Fig. 1 steps 1-6, Alg. 1, Alg. 2, Sec. 5.1):
 * one ray per pixel is clipped to the volume box; each ray is marched in
 * segments of K samples; every sample picks a stochastic LoD, walks the page
 * tables from that LoD to coarser ones (raising a ranked request for the
 * missing requested brick), samples the first mapped brick trilinearly and
 * stamps its slot; samples with no mapped brick (true misses) are compacted
 * by warp ballot and prefix sums and inferred by the INR in one batch; the
 * transfer function and front-to-back compositing produce out_rgba_dev
 * (width*height*4 floats, premultiplied RGBA over black, row-major from the
 * top-left pixel).  With cache != NULL, the frame ends with the cache update
 * of Sec. 4.3.2-4.3.3: top-n requests, LRU victims, decode of the requested
 * bricks by INR inference into the victim slots, page-table update; the new
 * bricks serve from the next frame on.  cache == NULL renders the uncached
 * baseline (every sample inferred directly).  Frames are numbered from 1 per
 * renderer/cache pair.  The call synchronises `stream` to return `stats`
 * (may be NULL).  Errors: CINR_ERR_ARG on a camera/renderer size mismatch. */
int cinr_render_frame(cinr_renderer_t r, cinr_cache_t cache, cinr_inr_t inr,
                      const cinr_camera* cam, const cinr_tf* tf,
                      float* out_rgba_dev, cinr_frame_stats* stats,
                      cinr_stream_t stream);

/* As cinr_render_frame, writing the image to host memory out_rgba_host
 * (width*height*4 floats; pinned memory gives an asynchronous copy).  The
 * device image lives in the renderer's working set. */
int cinr_render_frame_host(cinr_renderer_t r, cinr_cache_t cache,
                           cinr_inr_t inr, const cinr_camera* cam,
                           const cinr_tf* tf, float* out_rgba_host,
                           cinr_frame_stats* stats, cinr_stream_t stream);

/* Explicit-voxel render: the same rays, samples, transfer function and
 * compositing as cinr_render_frame, every sample valued by trilinear
 * interpolation of field_dev (fdims[0]*fdims[1]*fdims[2] floats, x fastest,
 * stored at voxel centres (i+0.5)/fdims, clamp-to-edge).  The quality
 * reference of a trained INR (the uncompressed data of Sec. 4.1).
 * Synchronises `stream` to fill stats->samples. */
int cinr_render_field(cinr_renderer_t r, const float* field_dev,
                      const int fdims[3], const cinr_camera* cam,
                      const cinr_tf* tf, float* out_rgba_dev,
                      cinr_frame_stats* stats, cinr_stream_t stream);

int cinr_destroy_renderer(cinr_renderer_t r);

/* Path tracing with Woodcock delta tracking (Sec. 5.1: the path-tracing
 * pipeline uses the same sampler as ray marching).  One path per pixel and
 * frame: free paths -ln(1-u)/sigma_bar (majorant sigma_bar = sigma_max, or
 * the TF's largest extinction when sigma_max <= 0); a tentative collision at
 * value v is real with probability sigma(v)/sigma_bar; at a real collision
 * the throughput takes the TF colour as albedo, the directional light is
 * added by next-event estimation (isotropic phase 1/(4 pi), shadow
 * transmittance by ratio tracking) and the path scatters into a uniform
 * direction, up to max_bounces collisions; paths that leave the volume (and
 * pixels whose ray misses it) collect `ambient`.  The random numbers of
 * pixel p in frame f are the SplitMix64 stream started at state
 * (frame_seed << 32) | p; every volume lookup goes through the cache exactly
 * as a ray-marching sample does (stochastic LoD from the distance to the
 * eye, fallback, ranked requests, LRU stamps, true misses inferred) and the
 * frame ends with the same cache update.  out_rgba_dev receives the path's
 * radiance and alpha = 1 when the camera ray collided (average frames for a
 * converged image).  Macro cells are not used. */
typedef struct {
  float light_dir[3]; /* direction the light travels */
  float light[3];     /* irradiance (rgb) */
  float ambient[3];   /* radiance of escaping paths (rgb) */
  int max_bounces;    /* >= 1 */
  float sigma_max;    /* majorant; <= 0: the TF's largest extinction */
} cinr_pt_opts;

int cinr_render_frame_pt(cinr_renderer_t r, cinr_cache_t cache, cinr_inr_t inr,
                         const cinr_camera* cam, const cinr_tf* tf,
                         const cinr_pt_opts* pt, float* out_rgba_dev,
                         cinr_frame_stats* stats, cinr_stream_t stream);

/* -------------------------------------------------------- macro cells --- */

/* Macro cells for adaptive sampling (Sec. 5.2).  The volume is cut into
 * ceil(dims/cell) cubes of cell^3 LoD-0 voxels; each holds the minimum and
 * maximum data value of its region.  Whenever a frame's transfer function
 * is applied, a cell whose value range meets only entries of zero extinction
 * (mu_max = 0) is marked transparent, and samples whose LoD-0 position
 * floor(x*dims) falls into a marked cell are skipped: no LoD pick, page-table
 * lookup, request, inference or compositing.  The skip rule: a value v reads
 * TF entries floor(x) and floor(x)+1, x = clamp(v,0,1)*255 (binary32), so a
 * cell with range [lo, hi] is transparent when the extinction of entries
 * floor(X(lo - 2^-20)) .. floor(X(hi + 2^-20)) + 1 (capped at 255) is zero.
 * With ranges that bound every value a sample in the cell can take (true
 * for CINR_MACRO_FROM_INR with a cache and for CINR_MACRO_FROM_FIELD with
 * cinr_render_field), skipping leaves the image unchanged. */
#define CINR_MACRO_FROM_INR 0    /* min/max of the INR at LoD voxel centres */
#define CINR_MACRO_FROM_RANGES 1 /* caller-provided ranges (host)           */
#define CINR_MACRO_FROM_FIELD 2  /* min/max of an explicit device field     */

/* source FROM_INR: for every LoD l in [min_level, levels), the LoD-l voxels
 * that a trilinear sample inside the cell can read -- per axis from
 * floor(clamp(c*cell/2^l - 1/2)) to floor(clamp(min((c+1)*cell, dims)/2^l -
 * 1/2)) + 1, clamped to the LoD-l grid -- are evaluated by the INR at their
 * voxel centres.  With cache != NULL the values are computed exactly as that
 * cache decodes and stores bricks (its LoD count, the INR's MLP precision
 * and the storage precision), so the ranges bound every cached sample;
 * `levels` is then ignored.  With cache == NULL the INR is evaluated as by
 * cinr_infer.  source FROM_RANGES: ranges_host holds 2 floats (min, max) per
 * cell, x fastest.  source FROM_FIELD: field_dev is a device array of
 * dims[0]*dims[1]*dims[2] floats (x fastest) and the ranges cover the LoD-0
 * voxels as above.  cell: a power of two in [2, 1024]. */
typedef struct {
  int dims[3];
  int cell;
  int source;
  cinr_inr_t inr;
  cinr_cache_t cache;
  int levels;
  int min_level;
  const float* ranges_host;
  const float* field_dev;
} cinr_macro_desc;

/* Device bytes of a macro-cell structure: 8 bytes of range, 4 bytes of
 * majorant and 1 byte of skip flag per cell. */
int cinr_macro_bytes(const int dims[3], int cell, size_t* bytes);

/* Builds the ranges in dev_mem (enqueued on `stream`; FROM_RANGES copies
 * synchronously).  Errors: CINR_ERR_ARG (bad cell, dims or source
 * arguments), CINR_ERR_NOMEM (buffer too small). */
int cinr_create_macro(const cinr_macro_desc* d, void* dev_mem, size_t bytes,
                      cinr_stream_t stream, cinr_macro_t* out);

/* Copies the ranges (2 floats per cell) or the skip flags of the last
 * applied transfer function (1 byte per cell) to host memory; synchronises
 * `stream`.  n = capacity in elements. */
int cinr_macro_ranges(cinr_macro_t m, float* host_out, size_t n,
                      cinr_stream_t stream);
int cinr_macro_skip_flags(cinr_macro_t m, uint8_t* host_out, size_t n,
                          cinr_stream_t stream);

/* Copies the majorants of the last applied transfer function (1 float per
 * cell, x fastest) to host memory; synchronises `stream`.  A cell's
 * majorant is the largest extinction among the TF entries of the skip rule
 * (floor(X(lo - 2^-20)) .. floor(X(hi + 2^-20)) + 1): it bounds the
 * extinction of every value in the cell's range and is 0 exactly for
 * transparent cells.  Before the first cinr_macro_apply_tf all are 0. */
int cinr_macro_majorants(cinr_macro_t m, float* host_out, size_t n,
                         cinr_stream_t stream);

/* Recomputes the skip flags and the majorants for `tf` (one kernel,
 * enqueued on `stream`). */
int cinr_macro_apply_tf(cinr_macro_t m, const cinr_tf* tf,
                        cinr_stream_t stream);

int cinr_destroy_macro(cinr_macro_t m);

/* Attaches m (NULL detaches) to the renderer: every following frame
 * (cinr_render_frame, cinr_render_frame_host, cinr_render_field,
 * cinr_render_frame_pt) first applies its transfer function to m (one extra
 * kernel).  Ray marching then skips the samples of transparent cells.  Path
 * tracing with sigma_max <= 0 then tracks with local majorants (Sec. 5.2:
 * each cell's largest opacity sets the sampling rate of the rays through
 * it): a free flight draws its optical depth -ln(1-u) once and spends it
 * cell by cell along a 3D DDA over the cells, a tentative collision in a
 * cell with majorant m is real with probability sigma/m and ratio tracking
 * multiplies by 1 - sigma/m; cells with majorant 0 are crossed without a
 * lookup.  The walk's arithmetic (binary32, in this order): start at
 * o + t d of a segment ending at t1, per axis p = o + t d, x = clamp01((p
 * + h) (1/e)), pv = x dims, cell c = min(floor(pv) / cell, cells - 1),
 * dv = (d (1/e)) dims, r = 1/dv; dv > 0: t_max = t + ((c+1) cell - pv) r,
 * t_delta = cell r; dv < 0: t_max = t + (c cell - pv) r, t_delta = cell
 * (-r); entering a cell: m, r_m = 1/m (0 for m = 0), t_exit = min(t_max
 * x, y, z, t1); a flight with m > 0 and tau < dd = m (t_exit - t) collides
 * at min(t + tau r_m, t_exit), else tau -= dd, t = t_exit and the axis of
 * the smallest t_max (x before y before z) moves, t_max += t_delta.
 * m's dims must equal the renderer's dims. */
int cinr_renderer_set_macro(cinr_renderer_t r, cinr_macro_t m);

/* Allocation-free uncached render.  The paper has no counterpart: this is a
 * convenience for callers that cannot allocate device memory -- a real-time
 * render loop in which an allocation would stall or fail, code running under
 * a policy that forbids new device allocations, or a host-side plugin that
 * owns no device buffer.  It renders the same uncached frame as
 * cinr_render_frame with cache == NULL, but the frame's working set (ray
 * counter, statistics and the device image) lives in one array of about
 * 4 MiB that the library keeps in device memory for as long as it is loaded,
 * on every GPU that loads it.  The image is copied to out_rgba_host
 * (width*height*4 floats) and the call synchronises `stream`.
 * Limits: width*height <= 262144 (512 x 512) and o->miss_record_cap == 0;
 * larger requests return CINR_ERR_ARG with a message naming the limit.
 * The first call on a device looks up the array's device address (with that
 * device current) and keeps it for the life of the process; make that first
 * call before any stream capture, and make no call after cudaDeviceReset or
 * another teardown of the device's primary context (the kept address would
 * then be stale).  A bounded device-side wait that gives up in a tensor-core
 * MLP returns CINR_ERR_TIMEOUT, as cinr_render_frame does.  Every
 * call uses the same array: calls that overlap on the GPU (different
 * streams or threads) race and must be serialised by the caller.
 * It calls no cudaMalloc, cudaFree or allocating library routine.
 * Only stats->samples, inr_queries_direct and true_misses are filled. */
int cinr_render_frame_noalloc(cinr_inr_t inr, const cinr_camera* cam,
                              const cinr_tf* tf, const cinr_march_opts* o,
                              float* out_rgba_host, cinr_frame_stats* stats,
                              cinr_stream_t stream);

/* ---------------------------------------------------------- training --- */

/* Training options (Sec. 4.1): each step draws `batch` random coordinates
 * in [0,1)^3 from a counter-based generator (coordinate c of element j of
 * step s is the top 24 bits of SplitMix64(seed + 3*((s-1)*batch + j) + c),
 * times 2^-24), looks their ground truth up by trilinear interpolation of an
 * explicit field normalised to [0,1], and takes one Adam step (Kingma & Ba,
 * bias-corrected) on the MSE of the raw network output. */
typedef struct {
  long batch;
  float lr, beta1, beta2, eps;
  uint64_t seed;
} cinr_train_opts;

/* Device bytes of a trainer (Adam moments, gradients and per-batch
 * activations) for this INR.  The INR's table must be FP32. */
int cinr_trainer_bytes(cinr_inr_t inr, const cinr_train_opts* o,
                       size_t* bytes);

/* Creates a trainer in dev_mem; it updates the INR's FP32 table and weights
 * in place (and refreshes the INR's half-precision weight copy). */
int cinr_create_trainer(cinr_inr_t inr, const cinr_train_opts* o,
                        void* dev_mem, size_t bytes, cinr_stream_t stream,
                        cinr_trainer_t* out);

/* One training step (Sec. 4.1) on field_dev (dims[0]*dims[1]*dims[2]
 * floats, x fastest, values in [0,1], sampled at voxel centres).  When
 * loss_dev is not NULL it receives the step's mean squared error. */
int cinr_train_step(cinr_trainer_t t, const float* field_dev,
                    const int dims[3], float* loss_dev, cinr_stream_t stream);

/* Sets the Adam learning rate of the following steps (a schedule is the
 * caller's: the paper gives none).  Host-side only. */
int cinr_trainer_set_lr(cinr_trainer_t t, float lr);

/* Chooses the training kernels of the following steps (Sec. 4.1): 0 (the
 * default) FP32 throughout -- forward, backward and weight-gradient
 * kernels on the FP32 pipes, gradients within FP32 rounding of the exact
 * ones --; 1 (FP16) or 2 (BF16) one fused kernel per step in which the
 * MLP's five products (two forward layers, two backward products through
 * W2 and W1, and the weight gradients of both hidden layers, accumulated
 * over the batch) run on the tensor cores (tcgen05) with 16-bit operands
 * and FP32 accumulation; the output layer, the loss, the table-gradient
 * scatter and Adam stay FP32.  FP16 operands hold 11 significant bits
 * (the back-propagated ones carry a fixed loss scale of 256, removed in
 * FP32), BF16 operands 8, which sets the gradients' error (stated in the
 * tests).  A bounded tensor-core wait that gives up is reported by
 * cinr_trainer_status as CINR_ERR_TIMEOUT.  Host-side only.
 * Errors: CINR_ERR_ARG. */
int cinr_trainer_set_tensor_cores(cinr_trainer_t t, int mode);

/* Stratified training coordinates (Sec. 4.1's random coordinates, drawn
 * per stratum) for the following steps: 1 -- sample s < 8^g of a batch of
 * n (8^g the largest power of eight <= n) takes one point uniform in cell s
 * of a 2^g grid over the unit cube, cells in Morton order, the rest of the
 * batch uniform in the cube; 0 (the default) -- every sample uniform in the
 * cube (the oracle's definition).  Both give an unbiased estimate of the
 * field's mean squared error; stratified batches put each 128-sample tile
 * in a compact region, so its coarse table entries are shared.  The points
 * come from the same counter-based draws.  Host-side only.
 * Errors: CINR_ERR_ARG. */
int cinr_trainer_set_stratified(cinr_trainer_t t, int on);

/* Whether any training step since the last call produced a non-finite
 * gradient (a NaN or infinite field value, or a diverged run): CINR_OK or
 * CINR_ERR_NAN (the flag is then cleared).  Synchronises `stream`. */
int cinr_trainer_status(cinr_trainer_t t, cinr_stream_t stream);

/* One call for `steps` training steps (Sec. 4.1): creates a trainer in
 * `workspace` (ws_bytes >= cinr_trainer_bytes), runs the steps on
 * field_dev, checks cinr_trainer_status and releases the trainer (the
 * workspace may then be reused; the INR keeps the trained parameters).
 * Adam's moments start from zero, as for a new trainer.  Errors: those of
 * cinr_create_trainer and cinr_train_step, CINR_ERR_NAN. */
int cinr_train(cinr_inr_t inr, const float* field_dev, const int dims[3],
               const cinr_train_opts* o, long steps, void* workspace,
               size_t ws_bytes, cinr_stream_t stream);

/* Gradient of the mean squared error (1/n) sum (y_i - target_i)^2 of the
 * raw network output at n given points (no parameter update): g_table_dev
 * (levels * 2^log2_table * 2 floats) and g_mlp_dev (weight count floats)
 * are overwritten; loss_dev (nullable) receives the loss.  n <= batch. */
int cinr_inr_loss_grad(cinr_trainer_t t, const float* xyz_dev,
                       const float* target_dev, long n, float* g_table_dev,
                       float* g_mlp_dev, float* loss_dev, cinr_stream_t stream);

int cinr_destroy_trainer(cinr_trainer_t t);

/* Copies the INR's FP32 parameters to host memory (the same layouts as
 * cinr_create_inr takes): a trained INR saved this way can be re-created,
 * e.g. with half-precision tables.  Synchronises `stream`. */
int cinr_inr_export(cinr_inr_t inr, float* host_table, float* host_mlp,
                    cinr_stream_t stream);

/* ------------------------------------------------------------- debug --- */
#define CINR_DUMP_PAGE_TABLE 0 /* u32 per brick: 0x80000000|slot or 0  */
#define CINR_DUMP_STAMPS 1     /* u32 per slot: last frame it was used */
#define CINR_DUMP_OWNERS 2     /* u32 per slot: brick key or 0xFFFFFFFF */
#define CINR_DUMP_RANK 3       /* u32 per brick: ranking value          */
#define CINR_DUMP_REQUESTS 4   /* u32 keys of the last request list     */
#define CINR_DUMP_VICTIMS 5    /* u32 slots of the last victim list     */
#define CINR_DUMP_MISSES 6     /* u32 pairs (pixel, sample), renderer   */
#define CINR_DUMP_PINNED 7     /* u32 per slot: 1 if pinned             */
#define CINR_DUMP_POOL 8       /* brick pool voxels (float or half bits) */
#define CINR_DUMP_PAGE_DIR 9   /* u32 per page: Mapped | page slot (paged) */
#define CINR_DUMP_PAGES 10     /* u32 per page entry, n_pages * P^3      */
#define CINR_DUMP_PAGE_KEYS 11 /* u32 per page slot: page key or ~0      */
#define CINR_DUMP_PAGE_REFS 12 /* u32 per page slot: mapped bricks       */

/* Copies a piece of state to host memory (synchronises `stream`).  For
 * CINR_DUMP_MISSES pass the renderer as `obj`, for the others the cache.
 * *count receives the number of elements available (u32 elements; for the
 * pool, voxels); at most cap elements are copied to host_out (which may be
 * NULL to query the count). */
int cinr_debug_dump(void* obj, int what, void* host_out, size_t cap,
                    size_t* count, cinr_stream_t stream);

/* Caps the brick decode at ctas_per_sm CTAs per SM (1 .. 8; 0, the
 * default, launches as many as the SM's registers and shared memory hold).
 * A tuning knob of the tensor-core decode (Sec. 4.3.2): fewer CTAs leave
 * SM slots to work that runs beside the decode (the lag-2 decode runs at
 * most 2 per SM next to the next frame's marching kernel).
 * Errors: CINR_ERR_ARG for a NULL cache or a count out of range. */
int cinr_cache_set_decode_ctas(cinr_cache_t cache, int ctas_per_sm);

/* Chooses the hash-grid encoder of the brick decode: 1 (the default) the
 * tile encoder -- per-axis cell tables of the brick's voxel lattice, each
 * level's corner box staged into shared memory by coalesced loads where it
 * fits, corners combined by separable lerps --, 0 every voxel gathering its
 * 8 corners per level from the table.  Both give the same voxels up to FP32
 * rounding; an autotuner knob.  Errors: CINR_ERR_ARG. */
int cinr_cache_set_decode_encoder(cinr_cache_t cache, int staged);

/* Writes one u32 entry of a cache's page tables (what = CINR_DUMP_PAGE_TABLE,
 * CINR_DUMP_PAGE_DIR or CINR_DUMP_PAGES; index < the count that
 * cinr_debug_dump reports for it), enqueued on `stream` and synchronised.
 * For tests of the device bounds checks: an entry naming a slot beyond the
 * pool is caught by a library built with device checks (see
 * cinr_device_checks) and reported as CINR_ERR_DEVICE_CHECK by the next
 * cinr_render_frame.  A library built without them would read past the
 * pool: plant such entries only with a checked build.
 * Errors: CINR_ERR_ARG for another table or an index out of range. */
int cinr_debug_set_entry(cinr_cache_t cache, int what, size_t index,
                         uint32_t value, cinr_stream_t stream);

/* 1 if this library was built with device bounds checks (-DCINR_CHECK=1),
 * else 0.  A checked build tests every page-table, page, slot, pool and
 * hash-table index on the device before the access it guards; an index out
 * of range skips the access and sets the kernel's error word, which
 * cinr_render_frame (frame kernels) and cinr_inr_status (INR inference and
 * the cache update kernels) report as CINR_ERR_DEVICE_CHECK.  The checks
 * stand in for a memory checker where none can run. */
int cinr_device_checks(void);

/* Tensor-core self-test of one 128 x 64 tile: d_dev[128][64] = A B^T with
 * a_dev [128][K] and b_dev [64][K] (row-major FP32, rounded to BF16 when
 * bf16 != 0, else FP16), accumulated in FP32 by tcgen05.mma in tensor
 * memory; K in {16, 32, 64}.  Checks the shared-memory operand layout the
 * MLP kernels use. */
int cinr_debug_mma_tile(const float* a_dev, const float* b_dev, int K,
                        int bf16, float* d_dev, cinr_stream_t stream);

/* Synchronises `stream` and reports whether a bounded device-side wait of a
 * tensor-core MLP kernel gave up since the last call on this INR
 * (CINR_ERR_TIMEOUT), clearing the flag. */
int cinr_inr_status(cinr_inr_t inr, cinr_stream_t stream);

/* Failure-detection self-test (enqueued on `stream`): one warp waits, with
 * `limit` polls (1 .. 2^22), for an mbarrier phase that nothing completes,
 * gives up, and sets this INR's status word the way the tensor-core MLP
 * kernels do when a wait runs out; the next cinr_inr_status reports
 * CINR_ERR_TIMEOUT.  The kernel ends by itself and the context stays
 * usable. */
int cinr_debug_wait_timeout(cinr_inr_t inr, unsigned limit,
                            cinr_stream_t stream);

/* Geometry of the cache's LoD `level`: voxel dims, brick counts per axis and
 * the key of its first brick (keys are level-major, x fastest). */
int cinr_cache_level_info(cinr_cache_t cache, int level, int dims[3],
                          int nbricks[3], long* key_offset);

#ifdef __cplusplus
}
#endif
#endif /* CINR_H */
