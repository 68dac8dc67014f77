// Multi-resolution brick cache (Sec. 4.3): flat per-LoD page tables
// (Sec. 4.3.1), ranked request list (Sec. 4.3.3), LRU victims by frame
// stamps, brick decode by INR inference with write-back into the pool
// (Sec. 4.3.2), coarsest-LoD preload (Sec. 4.3.4).
#include <cmath>
#include <cstring>

#include "cinr_internal.cuh"
#include "tc_mlp.cuh"

using namespace cinr;

namespace {

constexpr int kSelThreads = 256;
constexpr int kMaxReq = 8192;  // max requests (and victims) per frame

int bits_for(unsigned long long v) {
  int b = 0;
  while (b < 64 && (v >> b) != 0ull) ++b;
  return b;
}

struct CacheLayout {
  uint32_t *pt, *rank, *touched, *counters, *stamp, *owner, *pinned;
  uint32_t *pd, *pages, *page_key, *page_ref;
  void* pool;
  SelState *sel_req, *sel_vic;
  unsigned long long *req_keys, *vic_keys;
  uint32_t *req_vals, *req_sorted, *vic_vals, *vic_sorted;
  size_t bytes;
};

struct Geometry {
  int L, B, S;
  int dims[kMaxLod][3], nb[kMaxLod][3];
  unsigned long long off[kMaxLod + 1];
  int page_shift;  // -1: flat page tables
  int pg[kMaxLod][3];
  unsigned long long pd_off[kMaxLod + 1];
  long n_pages;
};

int geometry(const int vol[3], const cinr_cache_opts* o, Geometry* g) {
  if (!o || !vol) return set_error(CINR_ERR_ARG, "NULL argument");
  if (o->levels < 1 || o->levels > kMaxLod)
    return set_error(CINR_ERR_ARG, "levels must be in [1, %d]", kMaxLod);
  if (o->brick < 2 || o->brick > 64) return set_error(CINR_ERR_ARG, "brick must be in [2, 64]");
  if (vol[0] < 1 || vol[1] < 1 || vol[2] < 1) return set_error(CINR_ERR_ARG, "bad volume dims");
  if (o->n_req < 1 || o->n_req > kMaxReq)
    return set_error(CINR_ERR_ARG, "n_req must be in [1, %d]", kMaxReq);
  if (o->storage_precision != CINR_PREC_FP32 && o->storage_precision != CINR_PREC_FP16 &&
      o->storage_precision != CINR_PREC_FP16_TEX)
    return set_error(CINR_ERR_ARG, "storage_precision must be FP32, FP16 or FP16_TEX");
  if (o->lag < 0 || o->lag > 2) return set_error(CINR_ERR_ARG, "lag must be 1 or 2 (0 means 1)");
  g->page_shift = -1;
  g->n_pages = 0;
  if (o->page != 0) {
    int sh = 0;
    while (sh <= 4 && (1 << sh) != o->page) ++sh;
    if (sh > 4) return set_error(CINR_ERR_ARG, "page must be 0 or a power of two in [1, 16]");
    if (o->n_pages < 1 || o->n_pages >= (1l << 31) - 1)
      return set_error(CINR_ERR_ARG, "n_pages must be in [1, 2^31 - 1) with paged tables");
    g->page_shift = sh;
    g->n_pages = o->n_pages;
  }
  g->L = o->levels;
  g->B = o->brick;
  g->S = o->brick + 2;
  g->off[0] = 0;
  for (int l = 0; l < g->L; ++l) {
    for (int a = 0; a < 3; ++a) {
      g->dims[l][a] = (vol[a] + (1 << l) - 1) >> l;  // ceil(V / 2^l)
      g->nb[l][a] = (g->dims[l][a] + g->B - 1) / g->B;
    }
    g->off[l + 1] = g->off[l] + (unsigned long long)g->nb[l][0] * g->nb[l][1] * g->nb[l][2];
  }
  if (g->off[g->L] >= (1ull << 31)) return set_error(CINR_ERR_ARG, "too many bricks (>= 2^31)");
  g->pd_off[0] = 0;
  for (int l = 0; l < g->L; ++l) {
    for (int a = 0; a < 3; ++a)
      g->pg[l][a] = g->page_shift < 0 ? 0 : (g->nb[l][a] + (1 << g->page_shift) - 1) >> g->page_shift;
    g->pd_off[l + 1] = g->pd_off[l] + (unsigned long long)g->pg[l][0] * g->pg[l][1] * g->pg[l][2];
  }
  if (g->page_shift >= 0 && (unsigned long long)g->n_pages << (3 * g->page_shift) >= (1ull << 40))
    return set_error(CINR_ERR_ARG, "page pool too large");
  return CINR_OK;
}

// Texture layout of an FP16 pool (CINR_PREC_FP16_TEX): 2^shift slice blocks
// of S x S texels per row (the widest power of two with 2^shift S <= 16384
// texels: coordinates below 2^14 keep 10 fractional bits in binary32),
// rows of `pitch` texels (a multiple of 64: 128-byte rows), at most 65000
// texel rows (the limit of a pitched 2D texture).
constexpr int kTexMaxWidth = 16384, kTexMaxRows = 65000;
struct TexGeo {
  int shift, pitch;
};
TexGeo tex_geo(int S) {
  TexGeo t{0, 0};
  while ((2 << t.shift) * S <= kTexMaxWidth) ++t.shift;
  t.pitch = (int)align_up((size_t)((1 << t.shift) * S), 64);
  return t;
}
int elem_bytes(int prec) { return prec == CINR_PREC_FP32 ? 4 : 2; }

size_t pool_bytes_for(const Geometry& g, long n_slots, int prec) {
  const size_t S3 = (size_t)g.S * g.S * g.S;
  if (prec != CINR_PREC_FP16_TEX) return (size_t)n_slots * S3 * elem_bytes(prec);
  const TexGeo t = tex_geo(g.S);
  const size_t blocks = (size_t)n_slots * g.S, per_row = (size_t)1 << t.shift;
  const size_t block_rows = (blocks + per_row - 1) / per_row;
  return block_rows * g.S * (size_t)t.pitch * 2;
}

CacheLayout layout(const Geometry& g, long n_slots, int prec, void* base) {
  Carver c(base);
  CacheLayout L;
  size_t nb = (size_t)g.off[g.L];
  const bool paged = g.page_shift >= 0;
  L.pt = c.take<uint32_t>(paged ? 0 : nb);
  L.pd = c.take<uint32_t>(paged ? (size_t)g.pd_off[g.L] : 0);
  L.pages = c.take<uint32_t>(paged ? (size_t)g.n_pages << (3 * g.page_shift) : 0);
  L.page_key = c.take<uint32_t>(paged ? (size_t)g.n_pages : 0);
  L.page_ref = c.take<uint32_t>(paged ? (size_t)g.n_pages : 0);
  L.rank = c.take<uint32_t>(nb);
  L.touched = c.take<uint32_t>(nb);
  L.counters = c.take<uint32_t>(64);
  L.stamp = c.take<uint32_t>(n_slots);
  L.owner = c.take<uint32_t>(n_slots);
  L.pinned = c.take<uint32_t>(n_slots);
  L.sel_req = c.take<SelState>(1);
  L.sel_vic = c.take<SelState>(1);
  L.req_keys = c.take<unsigned long long>(kMaxReq);
  L.vic_keys = c.take<unsigned long long>(kMaxReq);
  L.req_vals = c.take<uint32_t>(kMaxReq);
  L.req_sorted = c.take<uint32_t>(kMaxReq);
  L.vic_vals = c.take<uint32_t>(kMaxReq);
  L.vic_sorted = c.take<uint32_t>(kMaxReq);
  size_t S3 = (size_t)g.S * g.S * g.S;
  (void)S3;
  // 1024-byte aligned (a texture's base must be 512-byte aligned)
  L.pool = c.take<char>(pool_bytes_for(g, n_slots, prec), 1024);
  L.bytes = align_up(c.off, 256);
  return L;
}

long slots_for(const Geometry& g, size_t pool_bytes, int prec) {
  size_t S3 = (size_t)g.S * g.S * g.S;
  if (prec != CINR_PREC_FP16_TEX) return (long)(pool_bytes / (S3 * elem_bytes(prec)));
  const TexGeo t = tex_geo(g.S);
  size_t block_rows = pool_bytes / ((size_t)t.pitch * 2 * g.S);
  if (block_rows > (size_t)(kTexMaxRows / g.S)) block_rows = (size_t)(kTexMaxRows / g.S);
  return (long)(block_rows * ((size_t)1 << t.shift) / g.S);
}

// ------------------------------------------------------------ kernels
__global__ void fill_u32(uint32_t* p, size_t n, uint32_t v) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
    p[i] = v;
}

// Key of a brick from its linear id: level, then (bx, by, bz).
__device__ __forceinline__ int key_level(const CacheDev& c, uint32_t key) {
  int l = 0;
  while (l + 1 < c.L && key >= c.off[l + 1]) ++l;
  return l;
}

// ------------------------------------------------ brick-tile hash encoder
// The voxels of a brick lie on a lattice, so along each axis a voxel's
// grid cell and weight at every hash-grid level depend on that axis's
// voxel coordinate alone: a tile computes them once per (level, axis,
// coordinate) into shared memory (binary32, as grid_cell).  At each level
// the corner vertices the tile can touch form a box; where the boxes fit,
// their table entries are staged into shared memory by coalesced loads
// (consecutive threads, consecutive vertices along x, dense rows
// contiguous in the table) and every voxel reads its 8 corners from there;
// finer levels, whose boxes outgrow the buffer, are gathered from the
// table directly.  Each voxel combines its corners by lerps along x, then
// y, then z (the trilinear weights of Sec. 3 in separable form).
constexpr int kDecMaxS = 18;  // the staged encoder serves bricks up to 16^3 + apron
constexpr int kDecMaxL = 24;  // and up to 24 levels

struct AxisCell {
  int i;    // cell index along the axis
  float w;  // weight of the upper vertex
};
struct LevelBox {
  int lo0, lo1, lo2;  // lowest vertex of the box
  int n0, n1, n2;     // box extent (vertices)
  int base;           // first entry in the stage buffer; -1: not staged
};

// Shared-memory bytes of the encoder's tables for L levels and bricks of S
// voxels per edge.
__host__ __device__ constexpr int dec_tables_bytes(int L, int S) {
  return L * 3 * S * (int)sizeof(AxisCell) + L * (int)sizeof(LevelBox);
}

// e / n for 0 <= e < 2^22 and n >= 1, with inv = 1/n rounded: (e + 1/2) / n
// lies at least 1/(2n) from an integer, and the two roundings move it by
// less than (e + 1/2) 2^-23 / n < 1/(2n), so the truncation is exact.
__device__ __forceinline__ int div_small(int e, float inv) {
  return (int)(((float)e + 0.5f) * inv);
}

// Voxel-centre coordinate of LoD-l voxel j (clamped to the grid) along an
// axis of V LoD-0 voxels: ((j + 0.5) 2^l) / V in binary32.
__device__ __forceinline__ float voxel_coord(int j, int dim_l, int l, int V) {
  j = j < 0 ? 0 : (j > dim_l - 1 ? dim_l - 1 : j);
  const float t = f_mul(f_add((float)j, 0.5f), (float)(1 << l));
  return clamp01(f_div(t, (float)V));
}

template <bool F16>
__device__ __forceinline__ float2 lerp_corners(const float2 e[8], float wx, float wy, float wz) {
  const float2 X = make_float2(wx, wx), Y = make_float2(wy, wy), Z = make_float2(wz, wz);
  const float2 x00 = f2_fma(X, f2_sub(e[1], e[0]), e[0]);
  const float2 x10 = f2_fma(X, f2_sub(e[3], e[2]), e[2]);
  const float2 x01 = f2_fma(X, f2_sub(e[5], e[4]), e[4]);
  const float2 x11 = f2_fma(X, f2_sub(e[7], e[6]), e[6]);
  const float2 y0 = f2_fma(Y, f2_sub(x10, x00), x00);
  const float2 y1 = f2_fma(Y, f2_sub(x11, x01), x01);
  return f2_fma(Z, f2_sub(y1, y0), y0);
}

// Stages the tile's boxes and fills the axis tables; all 128 threads.
// b: brick coordinates, l: its LoD, v0 / v1: the tile's voxel range.
// TC_BARRIERS: the tensor-core MLP's barriers already separate one tile's
// reads of the tables from the next tile's writes.
template <bool F16, bool TC_BARRIERS>
__device__ __forceinline__ void stage_tile(const InrDev& q, const CacheDev& c, int l, const int b[3], int v0,
                                           int v1, AxisCell* tab, LevelBox* box, float2* stage, int cap) {
  const int S = c.S, SS = S * S, L = q.L;
  const int t = threadIdx.x;
  if (!TC_BARRIERS) __syncthreads();  // the previous tile's voxels have read the tables
  const float inv_s = 1.0f / (float)S;
  for (int e = t; e < L * 3 * S; e += blockDim.x) {
    const int ja = div_small(e, inv_s), lv = e - ja * S;
    const int j = div_small(ja, 1.0f / 3.0f), a = ja - 3 * j;
    const float x = voxel_coord(b[a] * c.B - 1 + lv, c.dims[l][a], l, c.vol[a]);
    int ii;
    float w;
    grid_cell(x, q.res[j], ii, w);
    tab[e] = AxisCell{ii, w};
  }
  __syncthreads();
  if (t < 32) {
    // level t's box: full x rows; the y and z coordinates the tile covers
    int size = 0;
    LevelBox bx{0, 0, 0, 0, 0, 0, -1};
    if (t < L) {
      const int z0 = v0 / SS, z1 = (v1 - 1) / SS;
      const int y0 = z0 == z1 ? (v0 / S) % S : 0, y1 = z0 == z1 ? ((v1 - 1) / S) % S : S - 1;
      const AxisCell* ta = tab + t * 3 * S;
      bx.lo0 = ta[0].i;
      bx.lo1 = ta[S + y0].i;
      bx.lo2 = ta[2 * S + z0].i;
      bx.n0 = ta[S - 1].i + 2 - bx.lo0;
      bx.n1 = ta[S + y1].i + 2 - bx.lo1;
      bx.n2 = ta[2 * S + z1].i + 2 - bx.lo2;
      // a fine level's box at a coarse LoD can hold ~10^10 vertices: the
      // product in 64 bits, and anything beyond the buffer counts as cap + 1
      // (never staged; the scan of 32 such sizes stays far inside an int)
      const long long n = (long long)bx.n0 * (long long)bx.n1 * (long long)bx.n2;
      size = n > (long long)cap ? cap + 1 : (int)n;
    }
    // coarse levels first, while the stage buffer has room
    int scan = size;
    for (int o = 1; o < 32; o <<= 1) {
      const int u = __shfl_up_sync(0xffffffffu, scan, o);
      if (t >= o) scan += u;
    }
    const bool staged = t < L && scan <= cap;
    bx.base = staged ? scan - size : -1;
    if (t < L) box[t] = bx;
  }
  __syncthreads();
  const uint32_t T = 1u << q.log2T;
  const int warp = t >> 5, lane = t & 31, n_warps = blockDim.x >> 5;
  for (int j = warp; j < L; j += n_warps) {  // a level per warp; its lanes along the box
    const LevelBox bx = box[j];
    if (bx.base < 0) continue;
    const int nb01 = bx.n0 * bx.n1;
    const int size = nb01 * bx.n2;
    const float inv0 = 1.0f / (float)bx.n0, inv1 = 1.0f / (float)bx.n1;
    const bool dense = (q.dense_mask >> j) & 1u;
    const uint32_t n1 = (uint32_t)q.res[j] + 1u;
    const char* table = reinterpret_cast<const char*>(q.table) + (size_t)j * T * (F16 ? 4 : 8);
    for (int e = lane; e < size; e += 32) {
      const int yz = div_small(e, inv0), z = div_small(yz, inv1);
      const uint32_t cx = (uint32_t)(bx.lo0 + e - yz * bx.n0);
      const uint32_t cy = (uint32_t)(bx.lo1 + yz - z * bx.n1);
      const uint32_t cz = (uint32_t)(bx.lo2 + z);
      uint32_t idx = vertex_index(dense, n1, T, cx, cy, cz);
      if (!in_range(idx, T, q.err)) idx = 0u;
      stage[bx.base + e] = load_entry_t<F16>(table, idx);
    }
  }
  __syncthreads();
}

// Features of voxel (lx, ly, lz) of the tile (levels concatenated, 2 per
// level) from the axis tables, the staged boxes and the table.
template <int LV, bool F16>
__device__ __forceinline__ void encode_voxel(const InrDev& q, int S, int lx, int ly, int lz, const AxisCell* tab,
                                             const LevelBox* box, const float2* stage, float* feat) {
  const uint32_t T = 1u << q.log2T, Tm = T - 1u;
#pragma unroll
  for (int j = 0; j < LV; ++j) {
    const AxisCell ax = tab[(j * 3 + 0) * S + lx], ay = tab[(j * 3 + 1) * S + ly], az = tab[(j * 3 + 2) * S + lz];
    const LevelBox bx = box[j];
    float2 e[8];
    if (bx.base >= 0) {
      const int n01 = bx.n0 * bx.n1;
      const float2* p = stage + bx.base + (ax.i - bx.lo0) + bx.n0 * ((ay.i - bx.lo1) + bx.n1 * (az.i - bx.lo2));
      e[0] = p[0];
      e[1] = p[1];
      e[2] = p[bx.n0];
      e[3] = p[bx.n0 + 1];
      e[4] = p[n01];
      e[5] = p[n01 + 1];
      e[6] = p[n01 + bx.n0];
      e[7] = p[n01 + bx.n0 + 1];
    } else {
      const bool dense = (q.dense_mask >> j) & 1u;
      const uint32_t n1 = (uint32_t)q.res[j] + 1u;
      const uint32_t sy = dense ? n1 : 2654435761u, sz = dense ? n1 * n1 : 805459861u;
      const uint32_t x0 = (uint32_t)ax.i, x1 = x0 + 1u;
      const uint32_t y0 = (uint32_t)ay.i * sy, y1 = y0 + sy;
      const uint32_t z0 = (uint32_t)az.i * sz, z1 = z0 + sz;
      const void* table = reinterpret_cast<const char*>(q.table) + (size_t)j * T * (F16 ? 4 : 8);
#pragma unroll
      for (int cc = 0; cc < 8; ++cc) {
        const uint32_t xx = (cc & 1) ? x1 : x0, yy = (cc & 2) ? y1 : y0, zz = (cc & 4) ? z1 : z0;
        uint32_t idx = dense ? xx + yy + zz : ((xx ^ yy ^ zz) & Tm);
        if (!in_range(idx, T, q.err)) idx = 0u;
        e[cc] = load_entry_t<F16>(table, idx);
      }
    }
    const float2 r = lerp_corners<F16>(e, ax.w, ay.w, az.w);
    feat[2 * j] = r.x;
    feat[2 * j + 1] = r.y;
  }
}

// Decode (persistent): every stored voxel of a requested brick is inferred
// by the INR at its LoD-l voxel centre (clamp-to-edge) and written into the
// victim slot.  Work items are (request, 128-voxel tile) pairs, taken by the
// resident CTAs in a grid-stride loop, so one launch absorbs the uneven
// per-frame request count read from the device.
// Mode list: request i of *n_dev uses keys[i] and slots[i].  Mode preload
// (keys == nullptr): request i is brick off[L-1] + i into slot i.
// MLPP: 0 = FP32 SIMT MLP, 1 / 2 / 3 = FP16 / BF16 / FP8 tensor cores.
// Dynamic shared memory of the decode kernel: the MLP's (tensor-core tile
// state or FP32 weights), then the staged encoder's axis tables and level
// boxes, then (FP32 MLP only) its stage buffer; the tensor-core path stages
// into the hidden-layer operand buffer, which is free while a tile encodes.
constexpr int kDecStageFp32 = 1024;  // float2 entries
template <int IN, int H, int MLPP>
__host__ __device__ constexpr int dec_mlp_bytes() {
  return (int)(((MLPP ? sizeof(tc::TcSmem<IN, H>) : (size_t)mlp_floats<IN, H>() * 4) + 127) / 128 * 128);
}
template <int IN, int H, int MLPP>
__host__ __device__ constexpr int dec_smem_bytes(int L, int S, bool staged) {
  return dec_mlp_bytes<IN, H, MLPP>() +
         ((!MLPP && staged && S <= kDecMaxS && L <= kDecMaxL) ? dec_tables_bytes(L, S) + kDecStageFp32 * 8 : 0);
}

template <int IN, int H, int MLPP>
__global__ void __launch_bounds__(128) decode_kernel(InrDev q, CacheDev c, const uint16_t* w16,
                                                     const uint32_t* keys, const uint32_t* slots,
                                                     const uint32_t* n_dev, uint32_t n_fixed, int* err) {
  extern __shared__ __align__(1024) float4 smem4[];
  float* sw = reinterpret_cast<float*>(smem4);
  tc::TcSmem<IN, H>& tcs = *reinterpret_cast<tc::TcSmem<IN, H>*>(smem4);
  const uint32_t n = keys ? *n_dev : n_fixed;
  const int S = c.S, S3 = S * S * S;
  const uint32_t tiles_per = (uint32_t)((S3 + 127) / 128);
  const uint32_t work = n * tiles_per;
  if (blockIdx.x >= work) return;  // block-uniform, before any barrier
  // the staged encoder's shared memory (bricks up to 16^3 + apron, up to
  // 24 levels; otherwise every voxel encodes its own point).  The
  // tensor-core path keeps the tables and the stage buffer in the
  // hidden-layer operand buffer, free while a tile encodes; the FP32 path
  // after its weights.
  const int tb = (dec_tables_bytes(q.L, S) + 15) / 16 * 16;
  const bool staged = c.dec_staged && S <= kDecMaxS && q.L <= kDecMaxL &&
                      (!MLPP || tb + 64 * (int)sizeof(float2) <= (int)sizeof(tcs.a2));
  char* extra = MLPP ? reinterpret_cast<char*>(tcs.a2) : reinterpret_cast<char*>(smem4) + dec_mlp_bytes<IN, H, MLPP>();
  AxisCell* tab = reinterpret_cast<AxisCell*>(extra);
  LevelBox* box = reinterpret_cast<LevelBox*>(extra + q.L * 3 * S * (int)sizeof(AxisCell));
  float2* stage = reinterpret_cast<float2*>(extra + tb);
  const int cap = MLPP ? ((int)sizeof(tcs.a2) - tb) / (int)sizeof(float2) : kDecStageFp32;
  uint32_t phase = 0;
  if (MLPP) {
    tc::load_tc_weights<IN, H, (MLPP > 0 ? MLPP - 1 : 0)>(tcs, w16, q.w);
    tc::tc_setup(tcs);
  } else {
    load_weights(sw, q.w, mlp_floats<IN, H>());
    __syncthreads();
  }
  for (uint32_t wi = blockIdx.x; wi < work; wi += gridDim.x) {
    const uint32_t r = wi / tiles_per;
    const int v0 = (int)(wi % tiles_per) * 128;
    const int v = v0 + (int)threadIdx.x;
    const bool valid = v < S3;
    uint32_t key = keys ? keys[r] : c.off[c.L - 1] + r;
    const uint32_t slot = keys ? slots[r] : r;
    const bool in_pool = in_range(slot, c.n_slots, c.err);  // checked builds: skip the write
    if (!in_range(key, c.n_bricks, c.err)) key = 0u;
    const int l = key_level(c, key);
    const uint32_t local = key - c.off[l];
    const int b[3] = {(int)(local % c.nb[l][0]), (int)((local / c.nb[l][0]) % c.nb[l][1]),
                      (int)(local / ((uint32_t)c.nb[l][0] * c.nb[l][1]))};
    const int vv = valid ? v : v0;  // past the brick's end: any voxel of the tile
    const int lv[3] = {vv % S, (vv / S) % S, vv / (S * S)};
    float feat[IN];
    if (staged) {
      const int v1 = v0 + 128 < S3 ? v0 + 128 : S3;
      if (q.table_prec == CINR_PREC_FP16) {
        stage_tile<true, (MLPP > 0)>(q, c, l, b, v0, v1, tab, box, stage, cap);
        encode_voxel<IN / 2, true>(q, S, lv[0], lv[1], lv[2], tab, box, stage, feat);
      } else {
        stage_tile<false, (MLPP > 0)>(q, c, l, b, v0, v1, tab, box, stage, cap);
        encode_voxel<IN / 2, false>(q, S, lv[0], lv[1], lv[2], tab, box, stage, feat);
      }
    } else {
      float x[3];
#pragma unroll
      for (int a = 0; a < 3; ++a) x[a] = voxel_coord(b[a] * c.B - 1 + lv[a], c.dims[l][a], l, c.vol[a]);
      encode_point<IN / 2>(q, x[0], x[1], x[2], feat);
    }
    float y;
    if (MLPP == 0)
      y = valid ? mlp_fp32<IN, H>(sw, feat) : 0.0f;
    else
      y = tc::mlp_tile<IN, H, (MLPP > 0 ? MLPP - 1 : 0)>(tcs, feat, valid, phase, err);
    if (valid && in_pool) {
      const float val = fmaf(q.vscale, y, q.vmin);
      const size_t o = c.pool_tex ? tex_offset(S, c.tex_shift, c.tex_pitch, slot, lv[0], lv[1], lv[2])
                                  : (size_t)slot * S3 + v;
      if (c.pool_prec == CINR_PREC_FP16)
        reinterpret_cast<__half*>(c.pool)[o] = __float2half_rn(val);
      else
        reinterpret_cast<float*>(c.pool)[o] = val;
    }
  }
  if (MLPP) tc::tc_teardown(tcs);
}

// Preload map: brick i of the coarsest LoD into slot i.  Paged tables: the
// coarsest LoD's pages take page slots 0.. in ascending page key.
__global__ void preload_map(CacheDev c, uint32_t n) {
  uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  uint32_t key = c.off[c.L - 1] + i;
  if (c.pd) {
    uint32_t local;
    const uint32_t pk = key_page(c, key, local);
    const uint32_t ps = pk - c.pd_off[c.L - 1];
    c.pd[pk] = kMapped | ps;
    c.page_key[ps] = pk;
    c.pages[((size_t)ps << (3 * c.page_shift)) + local] = kMapped | i;
    atomicAdd(c.page_ref + ps, 1u);
  } else {
    c.pt[key] = kMapped | i;
  }
  c.owner[i] = key;
  c.pinned[i] = 1u;
}

// ------------------------------------------------------ radix select
// Candidate keys of the request list: bricks first requested this frame
// (touched list); key = (1000 - score) << key_bits | brick with ranking
// (score desc, brick asc), or the brick alone without ranking.
struct ReqKeys {
  const uint32_t* touched;
  const uint32_t* count;
  const uint32_t* rank;
  CacheDev c;
  uint32_t Tf;
  int key_bits;
  int ranking;
  __device__ bool operator()(uint32_t i, unsigned long long& key, uint32_t& val) const {
    if (i >= *count) return false;
    uint32_t b = touched[i];
    if (pt_entry_key(c, b) & kMapped) return false;  // mapped since its request (lag 2)
    uint32_t score = rank[b] - Tf;
    score = score > 1000u ? 1000u : score;
    key = ranking ? ((unsigned long long)(1000u - score) << key_bits) | b : (unsigned long long)b;
    val = b;
    return true;
  }
};

// Candidate keys of the victim list: slots neither pinned nor used this
// frame; key = stamp << slot_bits | slot (least recently used first, never
// used slots carry stamp 0).
struct VicKeys {
  const uint32_t* stamp;
  const uint32_t* pinned;
  uint32_t n_slots;
  uint32_t frame;
  int slot_bits;
  __device__ bool operator()(uint32_t i, unsigned long long& key, uint32_t& val) const {
    if (i >= n_slots) return false;
    uint32_t st = stamp[i];
    if (pinned[i] || st >= frame) return false;
    key = ((unsigned long long)st << slot_bits) | i;
    val = i;
    return true;
  }
};

template <class KF>
__global__ void __launch_bounds__(kSelThreads) sel_hist(KF kf, uint32_t n, SelState* st, int shift,
                                                        int pass) {
  __shared__ unsigned int h[2048];
  for (int i = threadIdx.x; i < 2048; i += blockDim.x) h[i] = 0;
  __syncthreads();
  if (pass > 0 && st->none) return;
  const unsigned long long prefix = st->prefix;
  unsigned int tot = 0;
  for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    unsigned long long key;
    uint32_t val;
    if (!kf(i, key, val)) continue;
    if (pass > 0 && (key >> (shift + 11)) != (prefix >> (shift + 11))) continue;
    ++tot;
    atomicAdd(&h[(key >> shift) & 2047u], 1u);
  }
  __syncthreads();
  for (int i = threadIdx.x; i < 2048; i += blockDim.x)
    if (h[i]) atomicAdd(&st->hist[i], h[i]);
  if (pass == 0) {
    for (int o = 16; o > 0; o >>= 1) tot += __shfl_xor_sync(0xffffffffu, tot, o);
    if ((threadIdx.x & 31) == 0 && tot) atomicAdd(&st->total, tot);
  }
}

// Picks the digit holding the k-th smallest key; one block of 1024 threads.
// cap (device, may be null): a further bound on the selected count, read on
// the device (the victim selection selects no more slots than requests).
__global__ void __launch_bounds__(1024) sel_pick(SelState* st, int shift, int pass, uint32_t want,
                                                 const uint32_t* cap) {
  __shared__ unsigned int warp_sum[32];
  __shared__ unsigned int s_k;
  const int t = threadIdx.x;
  if (pass == 0 && t == 0) {
    uint32_t k = st->total < want ? st->total : want;
    if (cap && *cap < k) k = *cap;
    st->none = (k == 0u);
    st->k = k;
    st->prefix = 0ull;
  }
  __syncthreads();
  if (t == 0) s_k = st->k;
  const unsigned int h0 = st->hist[2 * t], h1 = st->hist[2 * t + 1];
  __syncthreads();
  if (st->none) {
    st->hist[2 * t] = 0;
    st->hist[2 * t + 1] = 0;
    return;
  }
  // inclusive scan of per-thread pair sums
  unsigned int v = h0 + h1, x = v;
  const int lane = t & 31, w = t >> 5;
  for (int o = 1; o < 32; o <<= 1) {
    unsigned int y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) warp_sum[w] = x;
  __syncthreads();
  if (w == 0) {
    unsigned int s = warp_sum[lane], z = s;
    for (int o = 1; o < 32; o <<= 1) {
      unsigned int y = __shfl_up_sync(0xffffffffu, z, o);
      if (lane >= o) z += y;
    }
    warp_sum[lane] = z - s;  // exclusive
  }
  __syncthreads();
  const unsigned int before = warp_sum[w] + x - v;  // keys in digits < 2t
  const unsigned int k = s_k;
  if (before < k && k <= before + v) {
    unsigned int d, rem;
    if (k <= before + h0) {
      d = 2 * t;
      rem = k - before;
    } else {
      d = 2 * t + 1;
      rem = k - before - h0;
    }
    st->prefix |= (unsigned long long)d << shift;
    st->k = rem;
  }
  st->hist[2 * t] = 0;
  st->hist[2 * t + 1] = 0;
}

template <class KF>
__global__ void __launch_bounds__(kSelThreads) sel_gather(KF kf, uint32_t n, SelState* st,
                                                          unsigned long long* keys, uint32_t* vals) {
  if (st->none) return;
  const unsigned long long thr = st->prefix;
  for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    unsigned long long key;
    uint32_t val;
    if (!kf(i, key, val) || key > thr) continue;
    uint32_t pos = atomicAdd(&st->count, 1u);
    if (pos < kMaxReq) {
      keys[pos] = key;
      vals[pos] = val;
    }
  }
}

// Orders the gathered (at most kMaxReq, unique) keys: each entry's rank is
// the number of smaller keys; writes the count.
__global__ void __launch_bounds__(256) sel_sort(SelState* st, const unsigned long long* keys,
                                                const uint32_t* vals, uint32_t* sorted,
                                                uint32_t* n_out) {
  const uint32_t n = st->none ? 0u : (st->count < (uint32_t)kMaxReq ? st->count : (uint32_t)kMaxReq);
  const uint32_t t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t < n) {
    const unsigned long long k = keys[t];
    uint32_t r = 0;
    for (uint32_t j = 0; j < n; ++j) r += keys[j] < k;
    sorted[r] = vals[t];
  }
  if (t == 0) *n_out = n;
}

__global__ void sel_reset(SelState* st) {
  if (threadIdx.x == 0) {
    st->prefix = 0;
    st->k = 0;
    st->total = 0;
    st->none = 0;
    st->count = 0;
  }
}

// Commit (Fig. 1 step 5): request i gets victim i; the victim's previous
// brick is unmapped, the requested brick mapped, the slot stamped.
// With map == false (lag 2) the victims are only unmapped: the requested
// bricks are mapped by map_pending_kernel once decoded.
__global__ void commit_kernel(CacheDev c, const uint32_t* req, const uint32_t* req_n,
                              const uint32_t* vic, const uint32_t* vic_n, uint32_t frame,
                              uint32_t* decode_n, unsigned long long* stats, uint32_t S3, bool map) {
  const uint32_t m = *req_n < *vic_n ? *req_n : *vic_n;
  uint32_t ev = 0;
  for (uint32_t i = threadIdx.x; i < m; i += blockDim.x) {
    const uint32_t slot = vic[i], key = req[i];
    if (!in_range(slot, c.n_slots, c.err) || !in_range(key, c.n_bricks, c.err)) continue;
    const uint32_t old = c.owner[slot];
    if (old != kNoOwner && !in_range(old, c.n_bricks, c.err)) continue;
    if (old != kNoOwner) {
      if (c.pd) {
        uint32_t local;
        const uint32_t ps = c.pd[key_page(c, old, local)] & ~kMapped;
        if (!in_range(ps, c.n_pages, c.err)) continue;
        c.pages[((size_t)ps << (3 * c.page_shift)) + local] = 0u;
        atomicSub(c.page_ref + ps, 1u);
      } else {
        c.pt[old] = 0u;
      }
      ++ev;
    }
    if (map) {
      c.pt[key] = kMapped | slot;
      c.owner[slot] = key;
      c.stamp[slot] = frame;
    } else {
      c.owner[slot] = kNoOwner;  // in flight until the next frame's end
    }
  }
  for (int o = 16; o > 0; o >>= 1) ev += __shfl_xor_sync(0xffffffffu, ev, o);
  if ((threadIdx.x & 31) == 0 && ev) atomicAdd(&stats[ST_EVICT], (unsigned long long)ev);
  if (threadIdx.x == 0) {
    *decode_n = m;
    stats[ST_DECODED] += m;
    stats[ST_DECODE] += (unsigned long long)m * S3;
  }
}

// Lag 2: maps the bricks decoded during this frame (the previous frame's
// selection) and stamps their slots with this frame.
// With paged tables a brick whose page found no page slot is dropped (its
// slot stays free).  Used for lag 2, and for lag 1 with paged tables.
__global__ void map_pending_kernel(CacheDev c, const uint32_t* req, const uint32_t* vic,
                                   const uint32_t* decode_n, uint32_t frame) {
  const uint32_t m = *decode_n;
  for (uint32_t i = threadIdx.x; i < m; i += blockDim.x) {
    const uint32_t slot = vic[i], key = req[i];
    if (!in_range(slot, c.n_slots, c.err) || !in_range(key, c.n_bricks, c.err)) continue;
    if (c.pd) {
      uint32_t local;
      const uint32_t e = c.pd[key_page(c, key, local)];
      if (!(e & kMapped)) continue;  // no page slot: dropped
      const uint32_t ps = e & ~kMapped;
      if (!in_range(ps, c.n_pages, c.err)) continue;
      c.pages[((size_t)ps << (3 * c.page_shift)) + local] = kMapped | slot;
      atomicAdd(c.page_ref + ps, 1u);
    } else {
      c.pt[key] = kMapped | slot;
    }
    c.owner[slot] = key;
    c.stamp[slot] = frame;
  }
}

// Paged tables: frees the page slots left without a mapped brick.
__global__ void free_pages_kernel(CacheDev c) {
  for (uint32_t ps = blockIdx.x * blockDim.x + threadIdx.x; ps < c.n_pages; ps += gridDim.x * blockDim.x) {
    const uint32_t k = c.page_key[ps];
    if (k != kNoOwner && c.page_ref[ps] == 0u) {
      c.pd[k] = 0u;
      c.page_key[ps] = kNoOwner;
    }
  }
}

constexpr int kAllocThreads = 1024;
constexpr int kAllocCap = 8192;  // >= kMaxReq

// Paged tables: allocates the pages that requests 0..m-1 need and do not
// have: the distinct page keys in ascending order get the free page slots
// in ascending order (one CTA: bitonic sort in shared memory, then a
// block-wide running count of free slots).
__global__ void __launch_bounds__(kAllocThreads) alloc_pages_kernel(CacheDev c, const uint32_t* req,
                                                                     const uint32_t* n_dev) {
  __shared__ uint32_t keys[kAllocCap];
  __shared__ uint32_t n_need, n_uniq, base;
  __shared__ uint32_t wsum[kAllocThreads / 32];
  const uint32_t m = *n_dev;
  const int t = threadIdx.x;
  if (t == 0) n_need = 0;
  __syncthreads();
  for (uint32_t i = t; i < m; i += kAllocThreads) {
    uint32_t local;
    const uint32_t pk = key_page(c, req[i], local);
    if (!(c.pd[pk] & kMapped)) keys[atomicAdd(&n_need, 1u)] = pk;
  }
  __syncthreads();
  const uint32_t n = n_need;
  if (n == 0) return;  // block-uniform
  uint32_t np2 = 1;
  while (np2 < n) np2 <<= 1;
  for (uint32_t i = n + t; i < np2; i += kAllocThreads) keys[i] = 0xFFFFFFFFu;
  __syncthreads();
  for (uint32_t k = 2; k <= np2; k <<= 1)
    for (uint32_t j = k >> 1; j > 0; j >>= 1) {
      for (uint32_t i = t; i < np2; i += kAllocThreads) {
        const uint32_t p = i ^ j;
        if (p > i) {
          const bool up = (i & k) == 0;
          const uint32_t a = keys[i], b = keys[p];
          if ((a > b) == up) {
            keys[i] = b;
            keys[p] = a;
          }
        }
      }
      __syncthreads();
    }
  // unique, in place, by one thread (n <= 8192)
  if (t == 0) {
    uint32_t u = 0;
    for (uint32_t i = 0; i < n; ++i)
      if (i == 0 || keys[i] != keys[i - 1]) keys[u++] = keys[i];
    n_uniq = u;
    base = 0;
  }
  __syncthreads();
  const uint32_t u = n_uniq;
  // free page slots in ascending order: chunk of kAllocThreads slots per
  // pass, a block prefix count of the free ones
  for (uint32_t start = 0; start < c.n_pages; start += kAllocThreads) {
    if (base >= u) break;  // block-uniform (read after the barrier)
    const uint32_t ps = start + t;
    const bool is_free = ps < c.n_pages && c.page_key[ps] == kNoOwner;
    const unsigned bal = __ballot_sync(0xffffffffu, is_free);
    if ((t & 31) == 0) wsum[t >> 5] = __popc(bal);
    __syncthreads();
    uint32_t before = 0, total = 0;
    for (int w = 0; w < kAllocThreads / 32; ++w) {
      before += w < (t >> 5) ? wsum[w] : 0u;
      total += wsum[w];
    }
    const uint32_t r = base + before + __popc(bal & ((1u << (t & 31)) - 1u));
    if (is_free && r < u) {
      c.pd[keys[r]] = kMapped | ps;
      c.page_key[ps] = keys[r];
      c.page_ref[ps] = 0u;
    }
    __syncthreads();
    if (t == 0) base += total;
    __syncthreads();
  }
}

int num_sms();

int num_sms() {
  static int n = 0;
  if (!n) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
    if (n <= 0) n = 1;
  }
  return n;
}

template <class KF>
int radix_select(const KF& kf, uint32_t n, int key_bits, uint32_t want, SelState* st,
                 unsigned long long* keys, uint32_t* vals, uint32_t* sorted, uint32_t* n_out,
                 cudaStream_t s, const uint32_t* k_cap = nullptr) {
  const int passes = key_bits <= 11 ? 1 : (key_bits + 10) / 11;
  unsigned blocks = (unsigned)((n + kSelThreads - 1) / kSelThreads);
  unsigned cap = (unsigned)num_sms() * 4;
  if (blocks > cap) blocks = cap;
  if (blocks == 0) blocks = 1;
  sel_reset<<<1, 32, 0, s>>>(st);
  for (int p = 0; p < passes; ++p) {
    const int shift = 11 * (passes - 1 - p);
    sel_hist<KF><<<blocks, kSelThreads, 0, s>>>(kf, n, st, shift, p);
    sel_pick<<<1, 1024, 0, s>>>(st, shift, p, want, k_cap);
  }
  sel_gather<KF><<<blocks, kSelThreads, 0, s>>>(kf, n, st, keys, vals);
  sel_sort<<<(want + 255) / 256, 256, 0, s>>>(st, keys, vals, sorted, n_out);
  CINR_CK(cudaGetLastError());
  return CINR_OK;
}

// n_grid = the largest request count the launch may see (the device count
// n_dev decides at run time); the grid is the resident CTAs, at most one
// per work item.
template <int IN, int H, int MLPP>
int launch_decode(const cinr_inr_s* inr, const CacheDev& c, const uint32_t* keys, const uint32_t* slots,
                  const uint32_t* n_dev, uint32_t n_grid, int cap_per_sm, cudaStream_t s) {
  if (n_grid == 0) return CINR_OK;
  auto k = decode_kernel<IN, H, MLPP>;
  int smem = dec_smem_bytes<IN, H, MLPP>(inr->dev.L, c.S, c.dec_staged != 0);
  if (MLPP && smem < tc::kMinSmemPerCta) smem = tc::kMinSmemPerCta;  // <= 8 TMEM users per SM
  // residency depends on the shared memory, which depends on the INR's
  // levels and the brick size: recomputed when they change
  static int per_sm = 0, per_sm_smem = -1;
  if (per_sm_smem != smem) {
    per_sm = 0;
    per_sm_smem = smem;
    CINR_CK(cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
    // tensor-core path: the largest shared-memory carveout, so that the
    // occupancy query (and the launch) see every CTA that fits
    if (MLPP)
      CINR_CK(cudaFuncSetAttribute(k, cudaFuncAttributePreferredSharedMemoryCarveout,
                                   (int)cudaSharedmemCarveoutMaxShared));
    CINR_CK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k, 128, smem));
    if (per_sm < 1) return set_error(CINR_ERR_CUDA, "decode kernel cannot be resident");
    if (MLPP) {
      const int fit = tc::resident_ctas(k, smem);
      per_sm = fit > per_sm ? fit : per_sm;
    }
  }
  const int S3 = c.S * c.S * c.S;
  const long work = (long)n_grid * ((S3 + 127) / 128);
  long grid = (long)(cap_per_sm > 0 && cap_per_sm < per_sm ? cap_per_sm : per_sm) * num_sms();
  if (grid > work) grid = work;
  k<<<(unsigned)grid, 128, smem, s>>>(inr->dev, c, inr->w16, keys, slots, n_dev, n_grid,
                                      reinterpret_cast<int*>(inr->scratch + 16));
  CINR_CK(cudaGetLastError());
  return CINR_OK;
}

template <int MLPP>
int decode_prec(const cinr_inr_s* inr, const CacheDev& c, const uint32_t* keys, const uint32_t* slots,
                const uint32_t* n_dev, uint32_t n_grid, int cap, cudaStream_t s) {
  switch (shape_of(inr->dev.IN, inr->dev.H)) {
    case Shape::S16x32: return launch_decode<16, 32, MLPP>(inr, c, keys, slots, n_dev, n_grid, cap, s);
    case Shape::S32x64: return launch_decode<32, 64, MLPP>(inr, c, keys, slots, n_dev, n_grid, cap, s);
    case Shape::S48x64: return launch_decode<48, 64, MLPP>(inr, c, keys, slots, n_dev, n_grid, cap, s);
    default: return set_error(CINR_ERR_ARG, "unsupported shape");
  }
}

// cap > 0 limits the decode to cap CTAs per SM (lag 2: the decode shares
// the SMs with the next frame's marching kernel).
int decode(const cinr_inr_s* inr, const CacheDev& c, const uint32_t* keys, const uint32_t* slots,
           const uint32_t* n_dev, uint32_t n_grid, cudaStream_t s, int cap = 0) {
  if (inr->p.mlp_precision == CINR_PREC_FP16) return decode_prec<1>(inr, c, keys, slots, n_dev, n_grid, cap, s);
  if (inr->p.mlp_precision == CINR_PREC_BF16) return decode_prec<2>(inr, c, keys, slots, n_dev, n_grid, cap, s);
  if (inr->p.mlp_precision == CINR_PREC_FP8) return decode_prec<3>(inr, c, keys, slots, n_dev, n_grid, cap, s);
  return decode_prec<0>(inr, c, keys, slots, n_dev, n_grid, cap, s);
}

}  // namespace

extern "C" int cinr_cache_bytes(const int dims[3], size_t pool_bytes, const cinr_cache_opts* o,
                                size_t* bytes, long* n_slots) {
  Geometry g;
  int e = geometry(dims, o, &g);
  if (e) return e;
  if (!bytes) return set_error(CINR_ERR_ARG, "bytes is NULL");
  long ns = slots_for(g, pool_bytes, o->storage_precision);
  if (ns < 1) return set_error(CINR_ERR_ARG, "pool holds no brick");
  if (ns >= (1l << 31) - 1) return set_error(CINR_ERR_ARG, "too many slots");
  *bytes = layout(g, ns, o->storage_precision, nullptr).bytes;
  if (n_slots) *n_slots = ns;
  return CINR_OK;
}

extern "C" int cinr_create_cache(cinr_inr_t inr, const int dims[3], void* dev_mem, size_t bytes,
                                 size_t pool_bytes, const cinr_cache_opts* o, cinr_stream_t stream,
                                 cinr_cache_t* out) {
  if (!inr || !out) return set_error(CINR_ERR_ARG, "NULL argument");
  Geometry g;
  int e = geometry(dims, o, &g);
  if (e) return e;
  long ns = slots_for(g, pool_bytes, o->storage_precision);
  if (ns < 1) return set_error(CINR_ERR_ARG, "pool holds no brick");
  if (!dev_mem || (reinterpret_cast<uintptr_t>(dev_mem) & 255))
    return set_error(CINR_ERR_ARG, "dev_mem must be non-NULL and 256-byte aligned");
  CacheLayout L = layout(g, ns, o->storage_precision, dev_mem);
  if (bytes < L.bytes)
    return set_error(CINR_ERR_NOMEM, "cache needs %zu bytes, got %zu", L.bytes, bytes);
  const unsigned long long n_coarse = g.off[g.L] - g.off[g.L - 1];
  if (o->preload && (long)n_coarse > ns)
    return set_error(CINR_ERR_NOMEM, "pool of %ld bricks cannot hold the %llu coarsest bricks", ns,
                     n_coarse);
  if (o->preload && g.page_shift >= 0 && (long)(g.pd_off[g.L] - g.pd_off[g.L - 1]) > g.n_pages)
    return set_error(CINR_ERR_ARG, "n_pages (%ld) cannot hold the coarsest LoD's %llu pages", g.n_pages,
                     g.pd_off[g.L] - g.pd_off[g.L - 1]);
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  cinr_cache_s* c = new cinr_cache_s();
  c->o = *o;
  c->n_slots = ns;
  c->n_bricks = (long)g.off[g.L];
  c->frame = 0;
  c->inr = inr;
  CacheDev& d = c->dev;
  for (int a = 0; a < 3; ++a) d.vol[a] = dims[a];
  d.pt = L.pt;
  d.rank = L.rank;
  d.stamp = L.stamp;
  d.owner = L.owner;
  d.pinned = L.pinned;
  d.pool = L.pool;
  d.pool_prec = o->storage_precision == CINR_PREC_FP32 ? CINR_PREC_FP32 : CINR_PREC_FP16;
  d.pool_tex = o->storage_precision == CINR_PREC_FP16_TEX;
  d.tex_shift = 0;
  d.tex_pitch = 0;
  d.tex = 0;
  d.B = g.B;
  d.invB = (g.B & (g.B - 1)) == 0 ? 1.0f / (float)g.B : 0.0f;
  d.S = g.S;
  d.L = g.L;
  for (int l = 0; l < kMaxLod; ++l)
    for (int a = 0; a < 3; ++a) {
      d.dims[l][a] = l < g.L ? g.dims[l][a] : 1;
      d.nb[l][a] = l < g.L ? g.nb[l][a] : 1;
    }
  for (int l = 0; l <= kMaxLod; ++l) d.off[l] = (uint32_t)(l <= g.L ? g.off[l] : g.off[g.L]);
  d.touched = L.touched;
  d.touched_count = L.counters;
  d.pd = g.page_shift >= 0 ? L.pd : nullptr;
  d.pages = L.pages;
  d.page_key = L.page_key;
  d.page_ref = L.page_ref;
  d.page_shift = g.page_shift < 0 ? 0 : g.page_shift;
  d.n_pages = (uint32_t)g.n_pages;
  d.dec_staged = 1;  // the staged brick encoder (cinr_cache_set_decode_encoder)
  d.n_slots = (uint32_t)ns;
  d.n_bricks = (uint32_t)g.off[g.L];
  d.err = reinterpret_cast<int*>(inr->scratch + 16);  // update kernels report to the INR's status word
  for (int l = 0; l < kMaxLod; ++l)
    for (int a = 0; a < 3; ++a) d.pg[l][a] = l < g.L ? g.pg[l][a] : 1;
  for (int l = 0; l <= kMaxLod; ++l) d.pd_off[l] = (uint32_t)(l <= g.L ? g.pd_off[l] : g.pd_off[g.L]);
  c->sel_req = L.sel_req;
  c->sel_vic = L.sel_vic;
  c->req_keys = L.req_keys;
  c->req_vals = L.req_vals;
  c->req_sorted = L.req_sorted;
  c->req_n = L.counters + 1;
  c->vic_keys = L.vic_keys;
  c->vic_vals = L.vic_vals;
  c->vic_sorted = L.vic_sorted;
  c->vic_n = L.counters + 2;
  c->decode_n = L.counters + 3;
  c->key_bits = bits_for((unsigned long long)c->n_bricks);
  c->slot_bits = bits_for((unsigned long long)ns);

  // device initialisation; on any failure the handle is released
  auto init = [&]() -> int {
    if (d.pool_tex) {
      // the pool as a pitched 2D FP16 texture, bilinear filtering,
      // unnormalised coordinates (a descriptor over the caller's memory)
      if (reinterpret_cast<uintptr_t>(L.pool) & 511)
        return set_error(CINR_ERR_ARG, "the texture layout needs dev_mem 512-byte aligned");
      const TexGeo t = tex_geo(g.S);
      d.tex_shift = t.shift;
      d.tex_pitch = t.pitch;
      cudaResourceDesc rd;
      memset(&rd, 0, sizeof(rd));
      rd.resType = cudaResourceTypePitch2D;
      rd.res.pitch2D.devPtr = L.pool;
      rd.res.pitch2D.desc = cudaCreateChannelDescHalf();
      rd.res.pitch2D.width = (size_t)t.pitch;
      rd.res.pitch2D.height = pool_bytes_for(g, ns, CINR_PREC_FP16_TEX) / ((size_t)t.pitch * 2);
      rd.res.pitch2D.pitchInBytes = (size_t)t.pitch * 2;
      cudaTextureDesc td;
      memset(&td, 0, sizeof(td));
      td.addressMode[0] = cudaAddressModeClamp;
      td.addressMode[1] = cudaAddressModeClamp;
      td.filterMode = cudaFilterModeLinear;
      td.readMode = cudaReadModeElementType;
      td.normalizedCoords = 0;
      cudaTextureObject_t to = 0;
      CINR_CK(cudaCreateTextureObject(&to, &rd, &td, nullptr));
      d.tex = (unsigned long long)to;
    }
    size_t nb = (size_t)c->n_bricks;
    if (g.page_shift >= 0) {
      CINR_CK(cudaMemsetAsync(L.pd, 0, (size_t)g.pd_off[g.L] * 4, s));
      CINR_CK(cudaMemsetAsync(L.pages, 0, ((size_t)g.n_pages << (3 * g.page_shift)) * 4, s));
      CINR_CK(cudaMemsetAsync(L.page_key, 0xFF, (size_t)g.n_pages * 4, s));
      CINR_CK(cudaMemsetAsync(L.page_ref, 0, (size_t)g.n_pages * 4, s));
    } else {
      CINR_CK(cudaMemsetAsync(L.pt, 0, nb * 4, s));
    }
    CINR_CK(cudaMemsetAsync(L.rank, 0, nb * 4, s));
    CINR_CK(cudaMemsetAsync(L.counters, 0, 64 * 4, s));
    CINR_CK(cudaMemsetAsync(L.stamp, 0, (size_t)ns * 4, s));
    CINR_CK(cudaMemsetAsync(L.pinned, 0, (size_t)ns * 4, s));
    CINR_CK(cudaMemsetAsync(L.sel_req, 0, sizeof(SelState), s));
    CINR_CK(cudaMemsetAsync(L.sel_vic, 0, sizeof(SelState), s));
    fill_u32<<<256, 256, 0, s>>>(L.owner, (size_t)ns, kNoOwner);
    CINR_CK(cudaGetLastError());
    if (o->preload) {
      const int ed = decode(inr, d, nullptr, nullptr, nullptr, (uint32_t)n_coarse, s);
      if (ed) return ed;
      preload_map<<<(unsigned)((n_coarse + 255) / 256), 256, 0, s>>>(d, (uint32_t)n_coarse);
      CINR_CK(cudaGetLastError());
    }
    return CINR_OK;
  };
  e = init();
  if (e) {
    cinr_destroy_cache(c);
    return e;
  }
  if (o->lag == 2) {
    cudaError_t ce = cudaStreamCreateWithFlags(&c->dstream, cudaStreamNonBlocking);
    if (ce == cudaSuccess) ce = cudaEventCreateWithFlags(&c->e_sel, cudaEventDisableTiming);
    if (ce == cudaSuccess) ce = cudaEventCreateWithFlags(&c->e_dec, cudaEventDisableTiming);
    if (ce != cudaSuccess) {
      cinr_destroy_cache(c);
      return cuda_error(ce, "lag-2 stream or events");
    }
  }
  *out = c;
  return CINR_OK;
}

extern "C" int cinr_destroy_cache(cinr_cache_t cache) {
  if (cache && cache->dev.tex) cudaDestroyTextureObject((cudaTextureObject_t)cache->dev.tex);
  if (cache && cache->dstream) {
    cudaStreamSynchronize(cache->dstream);
    if (cache->e_sel) cudaEventDestroy(cache->e_sel);
    if (cache->e_dec) cudaEventDestroy(cache->e_dec);
    cudaStreamDestroy(cache->dstream);
  }
  delete cache;
  return CINR_OK;
}

int cinr_cache_wait_decode(cinr_cache_s* c, cudaStream_t s) {
  if (c->pending) CINR_CK(cudaStreamWaitEvent(s, c->e_dec, 0));
  return CINR_OK;
}

int cinr_cache_end_frame(cinr_cache_s* c, unsigned long long* stats_dev, cudaStream_t s) {
  const uint32_t frame = (uint32_t)c->frame;
  const uint32_t Tf = (uint32_t)(1001ull * c->frame);
  const uint32_t want = (uint32_t)c->o.n_req;
  const bool lag2 = c->o.lag == 2;
  const bool paged = c->dev.pd != nullptr;
  uint32_t extra = 0;
  // paged tables: the pages the mappings need, then the mappings
  auto map_selected = [&](uint32_t f) -> int {
    if (paged) {
      alloc_pages_kernel<<<1, kAllocThreads, 0, s>>>(c->dev, c->req_sorted, c->decode_n);
      CINR_CK(cudaGetLastError());
      ++extra;
    }
    map_pending_kernel<<<1, 1024, 0, s>>>(c->dev, c->req_sorted, c->vic_sorted, c->decode_n, f);
    CINR_CK(cudaGetLastError());
    ++extra;
    return CINR_OK;
  };
  if (lag2 && c->pending) {
    // the bricks decoded on the second stream during this frame are mapped
    // first: they serve the next frame and are no request candidates
    CINR_CK(cudaStreamWaitEvent(s, c->e_dec, 0));
    const int em = map_selected(frame);
    if (em) return em;
    c->pending = false;
  }
  ReqKeys rk{c->dev.touched, c->dev.touched_count, c->dev.rank, c->dev, Tf, c->key_bits, c->o.ranking};
  const int rbits = c->o.ranking ? c->key_bits + 10 : c->key_bits;
  int e = radix_select(rk, (uint32_t)c->n_bricks, rbits, want, c->sel_req, c->req_keys,
                       c->req_vals, c->req_sorted, c->req_n, s);
  if (e) return e;
  VicKeys vk{c->dev.stamp, c->dev.pinned, (uint32_t)c->n_slots, frame, c->slot_bits};
  const int vbits = c->slot_bits + bits_for((unsigned long long)frame);
  e = radix_select(vk, (uint32_t)c->n_slots, vbits, want, c->sel_vic, c->vic_keys, c->vic_vals,
                   c->vic_sorted, c->vic_n, s, c->req_n);
  if (e) return e;
  // commit: unmap the victims (and, flat lag 1, map the requests at once)
  commit_kernel<<<1, 1024, 0, s>>>(c->dev, c->req_sorted, c->req_n, c->vic_sorted, c->vic_n, frame,
                                   c->decode_n, stats_dev, (uint32_t)(c->dev.S * c->dev.S * c->dev.S),
                                   !lag2 && !paged);
  CINR_CK(cudaGetLastError());
  if (paged) {
    const int grid = (int)((c->dev.n_pages + 255) / 256 < 1024 ? (c->dev.n_pages + 255) / 256 : 1024);
    free_pages_kernel<<<grid, 256, 0, s>>>(c->dev);
    CINR_CK(cudaGetLastError());
    ++extra;
  }
  // kernels of this update: per radix select reset + (hist, pick) per pass +
  // gather + sort; commit; decode (+ page and map kernels)
  auto sel = [](int bits) { return 3 + 2 * (bits <= 11 ? 1 : (bits + 10) / 11); };
  if (!lag2) {
    int ed = decode(c->inr, c->dev, c->req_sorted, c->vic_sorted, c->decode_n, want, s, c->decode_ctas);
    if (ed) return ed;
    if (paged) {
      ed = map_selected(frame);
      if (ed) return ed;
    }
    c->last_launches = (uint32_t)(sel(rbits) + sel(vbits) + 2) + extra;
    return CINR_OK;
  }
  c->last_launches = (uint32_t)(sel(rbits) + sel(vbits) + 2) + extra;
  CINR_CK(cudaEventRecord(c->e_sel, s));
  CINR_CK(cudaStreamWaitEvent(c->dstream, c->e_sel, 0));
  int e2 = decode(c->inr, c->dev, c->req_sorted, c->vic_sorted, c->decode_n, want, c->dstream,
                  c->decode_ctas > 0 && c->decode_ctas < 2 ? c->decode_ctas : 2);
  if (e2) return e2;
  CINR_CK(cudaEventRecord(c->e_dec, c->dstream));
  c->pending = true;
  return CINR_OK;
}

extern "C" int cinr_cache_level_info(cinr_cache_t cache, int level, int dims[3], int nbricks[3],
                                     long* key_offset) {
  if (!cache) return set_error(CINR_ERR_ARG, "cache is NULL");
  if (level < 0 || level >= cache->dev.L) return set_error(CINR_ERR_ARG, "bad level");
  for (int a = 0; a < 3; ++a) {
    if (dims) dims[a] = cache->dev.dims[level][a];
    if (nbricks) nbricks[a] = cache->dev.nb[level][a];
  }
  if (key_offset) *key_offset = (long)cache->dev.off[level];
  return CINR_OK;
}

extern "C" int cinr_debug_set_entry(cinr_cache_t c, int what, size_t index, uint32_t value,
                                    cinr_stream_t stream) {
  if (!c) return set_error(CINR_ERR_ARG, "cache is NULL");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  uint32_t* dst = nullptr;
  size_t n = 0;
  switch (what) {
    case CINR_DUMP_PAGE_TABLE:
      dst = c->dev.pd ? nullptr : c->dev.pt;
      n = c->dev.pd ? 0 : (size_t)c->n_bricks;
      break;
    case CINR_DUMP_PAGE_DIR:
      dst = c->dev.pd;
      n = c->dev.pd ? (size_t)c->dev.pd_off[c->dev.L] : 0;
      break;
    case CINR_DUMP_PAGES:
      dst = c->dev.pages;
      n = c->dev.pd ? (size_t)c->dev.n_pages << (3 * c->dev.page_shift) : 0;
      break;
    default: return set_error(CINR_ERR_ARG, "entry writes go to the page tables only (what = %d)", what);
  }
  if (!dst || index >= n) return set_error(CINR_ERR_ARG, "index %zu out of range (%zu entries)", index, n);
  const int ew = cinr_cache_wait_decode(c, s);
  if (ew) return ew;
  CINR_CK(cudaMemcpyAsync(dst + index, &value, 4, cudaMemcpyHostToDevice, s));
  CINR_CK(cudaStreamSynchronize(s));
  return CINR_OK;
}

extern "C" int cinr_cache_set_decode_ctas(cinr_cache_t c, int ctas_per_sm) {
  if (!c) return set_error(CINR_ERR_ARG, "cache is NULL");
  if (ctas_per_sm < 0 || ctas_per_sm > 8) return set_error(CINR_ERR_ARG, "ctas_per_sm must be in [0, 8]");
  c->decode_ctas = ctas_per_sm;
  return CINR_OK;
}

extern "C" int cinr_cache_set_decode_encoder(cinr_cache_t c, int staged) {
  if (!c) return set_error(CINR_ERR_ARG, "cache is NULL");
  if (staged != 0 && staged != 1) return set_error(CINR_ERR_ARG, "staged must be 0 or 1");
  c->dev.dec_staged = staged;
  return CINR_OK;
}
