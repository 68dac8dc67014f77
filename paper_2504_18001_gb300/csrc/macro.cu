// Macro cells for adaptive sampling (Sec. 5.2): per-cell value ranges, the
// transparent-cell flags of a transfer function (mu_max = 0), and the
// structure's C ABI.  The renderer reads the flags per sample.
//
// Ranges from the INR cover, for every LoD of the cache, the LoD voxels that
// a trilinear sample inside the cell can read, evaluated with the arithmetic
// of the brick decode (same encoder, same MLP path per precision, same
// storage rounding), so they bound every cached sample.  Work items are
// (cell, LoD, 128-voxel tile) triples taken by resident CTAs in a grid-stride
// loop; each tile is reduced in the CTA and merged with one atomicMin and one
// atomicMax on order-preserving integer images of the floats.
#include <cmath>
#include <cstring>

#include "cinr_internal.cuh"
#include "tc_mlp.cuh"

using namespace cinr;

namespace {

constexpr int kMaxCell = 1024;

struct MacroBuild {
  int vol[3];
  int cell;
  int mdims[3];
  int l0, nl;                      // first LoD and number of LoDs
  int E[kMaxLod];                  // box edge per LoD (voxels)
  int ldims[kMaxLod][3];           // LoD-l grid dims
  uint32_t tile_off[kMaxLod + 1];  // first tile of each LoD within a cell
  int round_half;                  // values stored as FP16 by the cache
  uint32_t* enc;                   // 2 per cell: ordered images of min, max
  unsigned long long n_cells;
};

// Order-preserving map of floats onto unsigned integers (and back).
__device__ __forceinline__ uint32_t ord_enc(float f) {
  const uint32_t b = __float_as_uint(f);
  return (b & 0x80000000u) ? ~b : (b | 0x80000000u);
}
__device__ __forceinline__ float ord_dec(uint32_t u) {
  return __uint_as_float((u & 0x80000000u) ? (u & 0x7FFFFFFFu) : ~u);
}

// LoD-l voxel range [lo, hi] along one axis that a trilinear sample at an
// LoD-0 edge coordinate in [c*cell, min((c+1)*cell, V)] can read.
__device__ __forceinline__ void box_axis(int c, int cell, int V, int l, int dl, int& lo, int& hi) {
  const float sc = __int_as_float((127 - l) << 23);  // 2^-l
  const float dmax = (float)(dl - 1);
  const int e1 = min((c + 1) * cell, V);
  const float q0 = fminf(fmaxf(f_sub(f_mul((float)(c * cell), sc), 0.5f), 0.0f), dmax);
  const float q1 = fminf(fmaxf(f_sub(f_mul((float)e1, sc), 0.5f), 0.0f), dmax);
  lo = (int)floorf(q0);
  hi = min((int)floorf(q1) + 1, dl - 1);
}

// Work item wi, thread t: the cell, and the normalised voxel-centre
// coordinate of the thread's voxel (valid = inside the LoD box).
__device__ __forceinline__ unsigned long long macro_point(const MacroBuild& mb, unsigned long long wi,
                                                          float x[3], bool& valid) {
  const uint32_t tpc = mb.tile_off[mb.nl];
  const unsigned long long cell = wi / tpc;
  const uint32_t t = (uint32_t)(wi % tpc);
  int li = 0;
  while (li + 1 < mb.nl && t >= mb.tile_off[li + 1]) ++li;
  const int l = mb.l0 + li, E = mb.E[li];
  const int v = (int)(t - mb.tile_off[li]) * 128 + (int)threadIdx.x;
  valid = v < E * E * E;
  const int vv = valid ? v : 0;
  const int tl[3] = {vv % E, (vv / E) % E, vv / (E * E)};
  const unsigned long long cxy = (unsigned long long)mb.mdims[0] * mb.mdims[1];
  const int cc[3] = {(int)(cell % mb.mdims[0]), (int)((cell / mb.mdims[0]) % mb.mdims[1]), (int)(cell / cxy)};
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    int lo, hi;
    box_axis(cc[a], mb.cell, mb.vol[a], l, mb.ldims[li][a], lo, hi);
    const int j = min(lo + tl[a], hi);
    const float tt = f_mul(f_add((float)j, 0.5f), (float)(1 << l));
    x[a] = clamp01(f_div(tt, (float)mb.vol[a]));
  }
  return cell;
}

// CTA min / max of (valid) values, merged into the cell's range.
__device__ __forceinline__ void merge_range(const MacroBuild& mb, unsigned long long cell, float val,
                                            bool valid, float* s_red) {
  float mn = valid ? val : INFINITY, mx = valid ? val : -INFINITY;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    mn = fminf(mn, __shfl_xor_sync(0xffffffffu, mn, o));
    mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
  }
  const int warp = threadIdx.x >> 5;
  if ((threadIdx.x & 31) == 0) {
    s_red[warp] = mn;
    s_red[4 + warp] = mx;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    mn = fminf(fminf(s_red[0], s_red[1]), fminf(s_red[2], s_red[3]));
    mx = fmaxf(fmaxf(s_red[4], s_red[5]), fmaxf(s_red[6], s_red[7]));
    atomicMin(mb.enc + 2 * cell, ord_enc(mn));
    atomicMax(mb.enc + 2 * cell + 1, ord_enc(mx));
  }
  __syncthreads();
}

// MLPP: 0 = FP32 SIMT MLP, 1 / 2 / 3 = FP16 / BF16 / FP8 tensor cores (the
// decode kernel's arithmetic, value by value).
template <int IN, int H, int MLPP>
__global__ void __launch_bounds__(128) macro_inr_kernel(InrDev q, const uint16_t* w16,
                                                        const __grid_constant__ MacroBuild mb, int* err) {
  extern __shared__ __align__(1024) float4 smem4[];
  __shared__ float s_red[8];
  float* sw = reinterpret_cast<float*>(smem4);
  tc::TcSmem<IN, H>& tcs = *reinterpret_cast<tc::TcSmem<IN, H>*>(smem4);
  const unsigned long long work = mb.n_cells * mb.tile_off[mb.nl];
  if (blockIdx.x >= work) return;  // block-uniform, before any barrier
  uint32_t phase = 0;
  if (MLPP) {
    tc::load_tc_weights<IN, H, (MLPP > 0 ? MLPP - 1 : 0)>(tcs, w16, q.w);
    tc::tc_setup(tcs);
  } else {
    load_weights(sw, q.w, mlp_floats<IN, H>());
    __syncthreads();
  }
  for (unsigned long long wi = blockIdx.x; wi < work; wi += gridDim.x) {
    float x[3];
    bool valid;
    const unsigned long long cell = macro_point(mb, wi, x, valid);
    float y;
    if (MLPP == 0) {
      y = valid ? inr_raw_fp32<IN, H>(q, sw, x[0], x[1], x[2]) : 0.0f;
    } else {
      float feat[IN];
      encode_point<IN / 2>(q, x[0], x[1], x[2], feat);
      y = tc::mlp_tile<IN, H, (MLPP > 0 ? MLPP - 1 : 0)>(tcs, feat, valid, phase, err);
    }
    float val = fmaf(q.vscale, y, q.vmin);
    if (mb.round_half) val = __half2float(__float2half_rn(val));
    merge_range(mb, cell, val, valid, s_red);
  }
  if (MLPP) tc::tc_teardown(tcs);
}

// Explicit field (LoD 0): the voxel values themselves.
__global__ void __launch_bounds__(128) macro_field_kernel(const float* __restrict__ field,
                                                          const __grid_constant__ MacroBuild mb) {
  __shared__ float s_red[8];
  const unsigned long long work = mb.n_cells * mb.tile_off[mb.nl];
  for (unsigned long long wi = blockIdx.x; wi < work; wi += gridDim.x) {
    const uint32_t tpc = mb.tile_off[mb.nl];
    const unsigned long long cell = wi / tpc;
    const int E = mb.E[0];
    const int v = (int)(wi % tpc) * 128 + (int)threadIdx.x;
    const bool valid = v < E * E * E;
    const int vv = valid ? v : 0;
    const int tl[3] = {vv % E, (vv / E) % E, vv / (E * E)};
    const unsigned long long cxy = (unsigned long long)mb.mdims[0] * mb.mdims[1];
    const int cc[3] = {(int)(cell % mb.mdims[0]), (int)((cell / mb.mdims[0]) % mb.mdims[1]),
                       (int)(cell / cxy)};
    int j[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      int lo, hi;
      box_axis(cc[a], mb.cell, mb.vol[a], 0, mb.vol[a], lo, hi);
      j[a] = min(lo + tl[a], hi);
    }
    const float val = __ldg(field + ((size_t)j[2] * mb.vol[1] + j[1]) * mb.vol[0] + j[0]);
    merge_range(mb, cell, val, valid, s_red);
  }
}

__global__ void macro_init(uint32_t* enc, unsigned long long n) {
  for (unsigned long long i = blockIdx.x * (unsigned long long)blockDim.x + threadIdx.x; i < n;
       i += (unsigned long long)gridDim.x * blockDim.x) {
    enc[2 * i] = 0xFFFFFFFFu;  // image of +inf or above: any value lowers it
    enc[2 * i + 1] = 0u;
  }
}

__global__ void macro_decode(uint32_t* enc, unsigned long long n) {
  for (unsigned long long i = blockIdx.x * (unsigned long long)blockDim.x + threadIdx.x; i < 2 * n;
       i += (unsigned long long)gridDim.x * blockDim.x)
    enc[i] = __float_as_uint(ord_dec(enc[i]));
}

// Skip rule: entries floor(X(lo - 2^-20)) .. floor(X(hi + 2^-20)) + 1 of
// the TF (X(v) = clamp(v,0,1)*255 in binary32) all have zero extinction;
// nz[i] = number of entries below i with non-zero extinction.  The cell's
// majorant (Sec. 5.2's largest opacity of the cell, the tracking rate of
// the path tracer) is the largest extinction over the same entries: a
// range maximum from a sparse table of the 256 extinctions in shared
// memory (level k holds the maxima of 2^k consecutive entries).
struct SkipParams {
  const float* ranges;
  uint8_t* skip;
  float* major;
  unsigned long long n;
  uint32_t nz[257];
  float ext[256];
};

constexpr int kSkipThreads = 256;

__global__ void __launch_bounds__(kSkipThreads) macro_skip_kernel(const __grid_constant__ SkipParams p) {
  __shared__ float st[9][256];
  const int t = threadIdx.x;
  st[0][t] = p.ext[t];
  __syncthreads();
#pragma unroll 1
  for (int k = 1; k < 9; ++k) {
    const int j = t + (1 << (k - 1));
    st[k][t] = fmaxf(st[k - 1][t], st[k - 1][j < 256 ? j : 255]);
    __syncthreads();
  }
  const float margin = 9.5367431640625e-07f;  // 2^-20
  for (unsigned long long i = blockIdx.x * (unsigned long long)blockDim.x + t; i < p.n;
       i += (unsigned long long)gridDim.x * blockDim.x) {
    const float lo = clamp01(f_sub(p.ranges[2 * i], margin));
    const float hi = clamp01(f_add(p.ranges[2 * i + 1], margin));
    const int i0 = (int)floorf(f_mul(lo, 255.0f));
    const int i1 = min((int)floorf(f_mul(hi, 255.0f)) + 1, 255);
    p.skip[i] = p.nz[i1 + 1] == p.nz[i0] ? 1 : 0;
    const int k = 31 - __clz(i1 - i0 + 1);
    p.major[i] = fmaxf(st[k][i0], st[k][i1 - (1 << k) + 1]);
  }
}

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

int grid_for(unsigned long long n, int threads) {
  unsigned long long g = (n + threads - 1) / threads;
  const unsigned long long cap = 8ull * (unsigned long long)num_sms();
  return (int)(g < 1 ? 1 : (g > cap ? cap : g));
}

int check_geom(const int dims[3], int cell, int* shift, int mdims[3], size_t* n) {
  if (!dims) return set_error(CINR_ERR_ARG, "dims is NULL");
  if (cell < 2 || cell > kMaxCell || (cell & (cell - 1)))
    return set_error(CINR_ERR_ARG, "cell must be a power of two in [2, %d]", kMaxCell);
  int s = 0;
  while ((1 << s) < cell) ++s;
  *shift = s;
  size_t cnt = 1;
  for (int a = 0; a < 3; ++a) {
    if (dims[a] < 1) return set_error(CINR_ERR_ARG, "bad volume dims");
    mdims[a] = (dims[a] + cell - 1) / cell;
    cnt *= (size_t)mdims[a];
  }
  if (cnt >= (1ull << 31)) return set_error(CINR_ERR_ARG, "too many macro cells (>= 2^31)");
  *n = cnt;
  return CINR_OK;
}

struct MacroLayout {
  float* ranges;
  float* major;
  uint8_t* skip;
  size_t bytes;
};

MacroLayout mlayout(size_t n, void* base) {
  Carver c(base);
  MacroLayout L;
  L.ranges = c.take<float>(2 * n);
  L.major = c.take<float>(n);
  L.skip = c.take<uint8_t>(n);
  L.bytes = align_up(c.off, 256);
  return L;
}

MacroBuild make_build(const cinr_macro_s* m, int l0, int l1, int round_half) {
  MacroBuild mb;
  memset(&mb, 0, sizeof(mb));
  for (int a = 0; a < 3; ++a) {
    mb.vol[a] = m->vol[a];
    mb.mdims[a] = m->dims[a];
  }
  mb.cell = m->cell;
  mb.l0 = l0;
  mb.nl = l1 - l0;
  mb.tile_off[0] = 0;
  for (int i = 0; i < mb.nl; ++i) {
    const int l = l0 + i;
    const int w = m->cell >> l;
    mb.E[i] = (w > 0 ? w : 1) + 2;
    for (int a = 0; a < 3; ++a) mb.ldims[i][a] = (m->vol[a] + (1 << l) - 1) >> l;
    const uint32_t e3 = (uint32_t)(mb.E[i] * mb.E[i] * mb.E[i]);
    mb.tile_off[i + 1] = mb.tile_off[i] + (e3 + 127) / 128;
  }
  mb.round_half = round_half;
  mb.enc = reinterpret_cast<uint32_t*>(m->ranges);
  mb.n_cells = m->n;
  return mb;
}

template <int IN, int H, int MLPP>
int launch_inr(const cinr_inr_s* inr, const MacroBuild& mb, cudaStream_t s) {
  auto k = macro_inr_kernel<IN, H, MLPP>;
  int smem = MLPP ? (int)sizeof(tc::TcSmem<IN, H>) : mlp_floats<IN, H>() * 4;
  if (MLPP && smem < tc::kMinSmemPerCta) smem = tc::kMinSmemPerCta;  // <= 8 TMEM users per SM
  static int per_sm = 0;
  if (!per_sm) {
    CINR_CK(cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
    // tensor-core path: the largest shared-memory carveout, so that the
    // occupancy query (and the launch) see every CTA that fits
    if (MLPP)
      CINR_CK(cudaFuncSetAttribute(k, cudaFuncAttributePreferredSharedMemoryCarveout,
                                   (int)cudaSharedmemCarveoutMaxShared));
    CINR_CK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k, 128, smem));
    if (per_sm < 1) return set_error(CINR_ERR_CUDA, "macro-cell kernel cannot be resident");
    if (MLPP) {
      const int fit = tc::resident_ctas(k, smem);
      per_sm = fit > per_sm ? fit : per_sm;
    }
  }
  const unsigned long long work = mb.n_cells * mb.tile_off[mb.nl];
  unsigned long long grid = (unsigned long long)per_sm * num_sms();
  if (grid > work) grid = work;
  k<<<(unsigned)grid, 128, smem, s>>>(inr->dev, inr->w16, mb, reinterpret_cast<int*>(inr->scratch + 16));
  CINR_CK(cudaGetLastError());
  return CINR_OK;
}

template <int MLPP>
int inr_prec(const cinr_inr_s* inr, const MacroBuild& mb, cudaStream_t s) {
  switch (shape_of(inr->dev.IN, inr->dev.H)) {
    case Shape::S16x32: return launch_inr<16, 32, MLPP>(inr, mb, s);
    case Shape::S32x64: return launch_inr<32, 64, MLPP>(inr, mb, s);
    case Shape::S48x64: return launch_inr<48, 64, MLPP>(inr, mb, s);
    default: return set_error(CINR_ERR_ARG, "unsupported shape");
  }
}

int build_inr(const cinr_inr_s* inr, const MacroBuild& mb, cudaStream_t s) {
  switch (inr->p.mlp_precision) {
    case CINR_PREC_FP16: return inr_prec<1>(inr, mb, s);
    case CINR_PREC_BF16: return inr_prec<2>(inr, mb, s);
    case CINR_PREC_FP8: return inr_prec<3>(inr, mb, s);
    default: return inr_prec<0>(inr, mb, s);
  }
}

}  // namespace

int cinr_macro_apply(cinr_macro_s* m, const float (*rgba)[4], cudaStream_t s) {
  SkipParams p;
  p.ranges = m->ranges;
  p.skip = m->skip;
  p.major = m->major;
  p.n = m->n;
  p.nz[0] = 0;
  for (int i = 0; i < 256; ++i) {
    p.nz[i + 1] = p.nz[i] + (rgba[i][3] != 0.0f ? 1u : 0u);
    p.ext[i] = rgba[i][3];
  }
  macro_skip_kernel<<<grid_for(m->n, kSkipThreads), kSkipThreads, 0, s>>>(p);
  CINR_CK(cudaGetLastError());
  return CINR_OK;
}

extern "C" int cinr_macro_bytes(const int dims[3], int cell, size_t* bytes) {
  int shift, md[3];
  size_t n;
  int e = check_geom(dims, cell, &shift, md, &n);
  if (e) return e;
  if (!bytes) return set_error(CINR_ERR_ARG, "bytes is NULL");
  *bytes = mlayout(n, nullptr).bytes;
  return CINR_OK;
}

extern "C" int cinr_create_macro(const cinr_macro_desc* d, void* dev_mem, size_t bytes,
                                 cinr_stream_t stream, cinr_macro_t* out) {
  if (!d || !out) return set_error(CINR_ERR_ARG, "NULL argument");
  int shift, md[3];
  size_t n;
  int e = check_geom(d->dims, d->cell, &shift, md, &n);
  if (e) return e;
  // argument checks of the source before anything is enqueued
  int l0 = 0, l1 = 1, round_half = 0;
  const cinr_inr_s* inr = d->inr;
  if (d->source == CINR_MACRO_FROM_INR) {
    if (!inr) return set_error(CINR_ERR_ARG, "FROM_INR needs an INR");
    if (d->cache) {
      const cinr_cache_s* c = d->cache;
      if (c->inr != inr) return set_error(CINR_ERR_ARG, "cache was built for another INR");
      for (int a = 0; a < 3; ++a)
        if (c->dev.vol[a] != d->dims[a]) return set_error(CINR_ERR_ARG, "cache dims differ from dims");
      l1 = c->dev.L;
      round_half = c->dev.pool_prec == CINR_PREC_FP16;
    } else {
      if (d->levels < 1 || d->levels > kMaxLod) return set_error(CINR_ERR_ARG, "levels must be in [1, %d]", kMaxLod);
      l1 = d->levels;
    }
    if (d->min_level < 0 || d->min_level >= l1) return set_error(CINR_ERR_ARG, "min_level must be in [0, levels)");
    l0 = d->min_level;
  } else if (d->source == CINR_MACRO_FROM_RANGES) {
    if (!d->ranges_host) return set_error(CINR_ERR_ARG, "FROM_RANGES needs ranges_host");
  } else if (d->source == CINR_MACRO_FROM_FIELD) {
    if (!d->field_dev) return set_error(CINR_ERR_ARG, "FROM_FIELD needs field_dev");
  } else {
    return set_error(CINR_ERR_ARG, "unknown source %d", d->source);
  }
  if (!dev_mem || (reinterpret_cast<uintptr_t>(dev_mem) & 255))
    return set_error(CINR_ERR_ARG, "dev_mem must be non-NULL and 256-byte aligned");
  const MacroLayout L = mlayout(n, dev_mem);
  if (bytes < L.bytes) return set_error(CINR_ERR_NOMEM, "macro cells need %zu bytes, got %zu", L.bytes, bytes);
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  cinr_macro_s* m = new cinr_macro_s();
  for (int a = 0; a < 3; ++a) {
    m->vol[a] = d->dims[a];
    m->dims[a] = md[a];
  }
  m->cell = d->cell;
  m->shift = shift;
  m->n = n;
  m->ranges = L.ranges;
  m->skip = L.skip;
  m->major = L.major;
  cudaGetDevice(&m->device);
  auto fail = [&](int code) {
    delete m;
    return code;
  };
  cudaError_t ce = cudaMemsetAsync(m->skip, 0, n, s);
  if (ce == cudaSuccess) ce = cudaMemsetAsync(m->major, 0, n * sizeof(float), s);
  if (ce != cudaSuccess) return fail(cuda_error(ce, "cudaMemsetAsync"));
  if (d->source == CINR_MACRO_FROM_RANGES) {
    ce = cudaMemcpyAsync(m->ranges, d->ranges_host, 2 * n * sizeof(float), cudaMemcpyHostToDevice, s);
    if (ce == cudaSuccess) ce = cudaStreamSynchronize(s);
    if (ce != cudaSuccess) return fail(cuda_error(ce, "ranges upload"));
  } else {
    const MacroBuild mb = make_build(m, l0, l1, round_half);
    macro_init<<<grid_for(n, 256), 256, 0, s>>>(mb.enc, n);
    ce = cudaGetLastError();
    if (ce != cudaSuccess) return fail(cuda_error(ce, "macro_init"));
    if (d->source == CINR_MACRO_FROM_FIELD) {
      const unsigned long long work = mb.n_cells * mb.tile_off[mb.nl];
      macro_field_kernel<<<grid_for(work * 128, 128), 128, 0, s>>>(d->field_dev, mb);
      ce = cudaGetLastError();
      if (ce != cudaSuccess) return fail(cuda_error(ce, "macro_field_kernel"));
    } else {
      e = build_inr(inr, mb, s);
      if (e) return fail(e);
    }
    macro_decode<<<grid_for(2 * n, 256), 256, 0, s>>>(mb.enc, n);
    ce = cudaGetLastError();
    if (ce != cudaSuccess) return fail(cuda_error(ce, "macro_decode"));
  }
  *out = m;
  return CINR_OK;
}

extern "C" int cinr_macro_ranges(cinr_macro_t m, float* host_out, size_t n, cinr_stream_t stream) {
  if (!m || !host_out) return set_error(CINR_ERR_ARG, "NULL argument");
  if (n < 2 * m->n) return set_error(CINR_ERR_NOMEM, "need %zu floats", 2 * m->n);
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  CINR_CK(cudaMemcpyAsync(host_out, m->ranges, 2 * m->n * sizeof(float), cudaMemcpyDeviceToHost, s));
  CINR_CK(cudaStreamSynchronize(s));
  return CINR_OK;
}

extern "C" int cinr_macro_skip_flags(cinr_macro_t m, uint8_t* host_out, size_t n, cinr_stream_t stream) {
  if (!m || !host_out) return set_error(CINR_ERR_ARG, "NULL argument");
  if (n < m->n) return set_error(CINR_ERR_NOMEM, "need %zu bytes", m->n);
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  CINR_CK(cudaMemcpyAsync(host_out, m->skip, m->n, cudaMemcpyDeviceToHost, s));
  CINR_CK(cudaStreamSynchronize(s));
  return CINR_OK;
}

extern "C" int cinr_macro_majorants(cinr_macro_t m, float* host_out, size_t n, cinr_stream_t stream) {
  if (!m || !host_out) return set_error(CINR_ERR_ARG, "NULL argument");
  if (n < m->n) return set_error(CINR_ERR_NOMEM, "need %zu floats", m->n);
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  CINR_CK(cudaMemcpyAsync(host_out, m->major, m->n * sizeof(float), cudaMemcpyDeviceToHost, s));
  CINR_CK(cudaStreamSynchronize(s));
  return CINR_OK;
}

extern "C" int cinr_macro_apply_tf(cinr_macro_t m, const cinr_tf* tf, cinr_stream_t stream) {
  if (!m || !tf) return set_error(CINR_ERR_ARG, "NULL argument");
  return cinr_macro_apply(m, tf->rgba, static_cast<cudaStream_t>(stream));
}

extern "C" int cinr_destroy_macro(cinr_macro_t m) {
  delete m;
  return CINR_OK;
}
