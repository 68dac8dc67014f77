// INR object and direct inference: multiresolution hash-grid encoding + small
// MLP (Sec. 3, Fig. 2), value de-normalisation (Sec. 4.1), InferINR of Alg. 1.
#include <cmath>
#include <cstring>
#include <vector>

#include "cinr_internal.cuh"

using namespace cinr;

namespace {

int validate(const cinr_inr_params* p) {
  if (!p) return set_error(CINR_ERR_ARG, "params is NULL");
  if (p->feats != 2) return set_error(CINR_ERR_ARG, "feats must be 2 (got %d)", p->feats);
  if (p->levels < 1 || p->levels > kMaxLevels)
    return set_error(CINR_ERR_ARG, "levels must be in [1, %d]", kMaxLevels);
  if (p->log2_table < 4 || p->log2_table > 24)
    return set_error(CINR_ERR_ARG, "log2_table must be in [4, 24]");
  if (p->n_hidden_layers != 2) return set_error(CINR_ERR_ARG, "n_hidden_layers must be 2");
  if (shape_of(p->levels * p->feats, p->hidden) == Shape::Bad)
    return set_error(CINR_ERR_ARG, "unsupported MLP shape %dx%d", p->levels * p->feats, p->hidden);
  if (p->base_res < 1 || !(p->growth >= 1.0)) return set_error(CINR_ERR_ARG, "bad level scale");
  if (p->table_precision != CINR_PREC_FP32 && p->table_precision != CINR_PREC_FP16)
    return set_error(CINR_ERR_ARG, "table_precision must be FP32 or FP16");
  if (p->mlp_precision < CINR_PREC_FP32 || p->mlp_precision > CINR_PREC_FP8)
    return set_error(CINR_ERR_ARG, "mlp_precision must be FP32, FP16, BF16 or FP8");
  return CINR_OK;
}

size_t table_entries(const cinr_inr_params* p) {
  return (size_t)p->levels * ((size_t)1 << p->log2_table);
}
size_t mlp_count(const cinr_inr_params* p) {
  size_t in = (size_t)p->levels * p->feats, h = p->hidden;
  return h * in + (size_t)(p->n_hidden_layers - 1) * h * h + h;
}

struct InrLayout {
  void* table;
  float* w;
  uint16_t* w16;
  float* scratch;
  size_t bytes;
};

InrLayout layout(const cinr_inr_params* p, void* base) {
  Carver c(base);
  InrLayout L;
  size_t esz = p->table_precision == CINR_PREC_FP16 ? 4 : 8;  // one 2-feature entry
  L.table = c.take<char>(table_entries(p) * esz);
  L.w = c.take<float>(mlp_count(p));
  L.w16 = c.take<uint16_t>(mlp_count(p));
  L.scratch = c.take<float>(1024);
  L.bytes = align_up(c.off, 256);
  return L;
}

}  // namespace

extern "C" int cinr_inr_bytes(const cinr_inr_params* p, size_t* bytes) {
  int e = validate(p);
  if (e) return e;
  if (!bytes) return set_error(CINR_ERR_ARG, "bytes is NULL");
  *bytes = layout(p, nullptr).bytes;
  return CINR_OK;
}

extern "C" int cinr_create_inr(const cinr_inr_params* p, void* dev_mem, size_t bytes,
                               const float* host_table, const float* host_mlp,
                               cinr_stream_t stream, cinr_inr_t* out) {
  int e = validate(p);
  if (e) return e;
  if (!out || !host_table || !host_mlp) return set_error(CINR_ERR_ARG, "NULL argument");
  if (!dev_mem || (reinterpret_cast<uintptr_t>(dev_mem) & 255))
    return set_error(CINR_ERR_ARG, "dev_mem must be non-NULL and 256-byte aligned");
  InrLayout L = layout(p, dev_mem);
  if (bytes < L.bytes)
    return set_error(CINR_ERR_NOMEM, "INR needs %zu bytes, got %zu", L.bytes, bytes);
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  size_t ne = table_entries(p) * 2;
  if (p->table_precision == CINR_PREC_FP16) {
    std::vector<__half> h(ne);
    for (size_t i = 0; i < ne; ++i) h[i] = __float2half_rn(host_table[i]);
    CINR_CK(cudaMemcpyAsync(L.table, h.data(), ne * 2, cudaMemcpyHostToDevice, s));
    CINR_CK(cudaStreamSynchronize(s));
  } else {
    CINR_CK(cudaMemcpyAsync(L.table, host_table, ne * 4, cudaMemcpyHostToDevice, s));
  }
  size_t nw = mlp_count(p);
  CINR_CK(cudaMemcpyAsync(L.w, host_mlp, nw * 4, cudaMemcpyHostToDevice, s));
  std::vector<uint16_t> w16(nw);
  for (size_t i = 0; i < nw; ++i) {
    if (p->mlp_precision == CINR_PREC_BF16) {
      __nv_bfloat16 b = __float2bfloat16_rn(host_mlp[i]);
      memcpy(&w16[i], &b, 2);
    } else {
      __half h = __float2half_rn(host_mlp[i]);
      memcpy(&w16[i], &h, 2);
    }
  }
  CINR_CK(cudaMemcpyAsync(L.w16, w16.data(), nw * 2, cudaMemcpyHostToDevice, s));
  CINR_CK(cudaMemsetAsync(L.scratch, 0, 1024 * sizeof(float), s));
  CINR_CK(cudaStreamSynchronize(s));

  int device = 0;
  CINR_CK(cudaGetDevice(&device));
  cinr_inr_s* h = new cinr_inr_s();
  h->p = *p;
  h->mem = dev_mem;
  h->bytes = bytes;
  h->scratch = L.scratch;
  h->w16 = L.w16;
  h->device = device;
  InrDev& d = h->dev;
  d.err = reinterpret_cast<int*>(L.scratch + 16);  // the INR's status word
  d.table = L.table;
  d.w = L.w;
  d.L = p->levels;
  d.log2T = p->log2_table;
  d.dense_mask = 0;
  double sc = (double)p->base_res;
  for (int l = 0; l < p->levels; ++l) {
    d.res[l] = (int)floor(sc);  // N_l = floor(base * growth^l), repeated FP64 product
    sc = sc * p->growth;
    uint64_t n1 = (uint64_t)d.res[l] + 1;
    if (n1 * n1 * n1 <= (1ull << p->log2_table)) d.dense_mask |= 1u << l;
  }
  d.IN = p->levels * p->feats;
  d.H = p->hidden;
  d.NH = p->n_hidden_layers;
  d.table_prec = p->table_precision;
  d.vmin = p->vmin;
  d.vscale = p->vmax - p->vmin;
  *out = h;
  return CINR_OK;
}

extern "C" int cinr_inr_set_range(cinr_inr_t inr, float vmin, float vmax) {
  if (!inr) return set_error(CINR_ERR_ARG, "inr is NULL");
  inr->p.vmin = vmin;
  inr->p.vmax = vmax;
  inr->dev.vmin = vmin;
  inr->dev.vscale = vmax - vmin;
  return CINR_OK;
}

extern "C" int cinr_destroy_inr(cinr_inr_t inr) {
  delete inr;
  return CINR_OK;
}

// ------------------------------------------------------------- kernels
namespace {

template <int IN, int H>
__global__ void __launch_bounds__(128) infer_kernel(InrDev q, const float* __restrict__ xyz,
                                                    long n, float* __restrict__ out) {
  extern __shared__ float4 smem4[];
  float* sw = reinterpret_cast<float*>(smem4);
  load_weights(sw, q.w, mlp_floats<IN, H>());
  __syncthreads();
  for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x) {
    float x = clamp01(__ldg(xyz + 3 * i)), y = clamp01(__ldg(xyz + 3 * i + 1)),
          z = clamp01(__ldg(xyz + 3 * i + 2));
    float r = inr_raw_fp32<IN, H>(q, sw, x, y, z);
    out[i] = fmaf(q.vscale, r, q.vmin);
  }
}

template <int IN>
__global__ void encode_kernel(InrDev q, const float* __restrict__ xyz, long n,
                              float* __restrict__ feats, uint32_t* __restrict__ idx) {
  long i = blockIdx.x * (long)blockDim.x + threadIdx.x;
  if (i >= n) return;
  float x = clamp01(xyz[3 * i]), y = clamp01(xyz[3 * i + 1]), z = clamp01(xyz[3 * i + 2]);
  float f[IN];
  encode_point<IN / 2>(q, x, y, z, f);
  for (int j = 0; j < IN; ++j) feats[i * IN + j] = f[j];
  if (idx) {
    const uint32_t T = 1u << q.log2T;
    for (int l = 0; l < IN / 2; ++l) {
      int N = q.res[l];
      int ix, iy, iz;
      float wx, wy, wz;
      grid_cell(x, N, ix, wx);
      grid_cell(y, N, iy, wy);
      grid_cell(z, N, iz, wz);
      bool dense = (q.dense_mask >> l) & 1u;
      for (int c = 0; c < 8; ++c)
        idx[(i * (IN / 2) + l) * 8 + c] = vertex_index(dense, (uint32_t)N + 1u, T, ix + (c & 1),
                                                       iy + ((c >> 1) & 1), iz + ((c >> 2) & 1));
    }
  }
}

__device__ __forceinline__ void atomic_min_f(float* a, float v) {
  if (v >= 0.0f)
    atomicMin(reinterpret_cast<int*>(a), __float_as_int(v));
  else
    atomicMax(reinterpret_cast<unsigned int*>(a), __float_as_uint(v));
}
__device__ __forceinline__ void atomic_max_f(float* a, float v) {
  if (v >= 0.0f)
    atomicMax(reinterpret_cast<int*>(a), __float_as_int(v));
  else
    atomicMin(reinterpret_cast<unsigned int*>(a), __float_as_uint(v));
}

template <int IN, int H>
__global__ void __launch_bounds__(128) range_kernel(InrDev q, int3 dims, int stride, int3 cnt,
                                                    float* mm) {
  extern __shared__ float4 smem4[];
  float* sw = reinterpret_cast<float*>(smem4);
  load_weights(sw, q.w, mlp_floats<IN, H>());
  __syncthreads();
  long total = (long)cnt.x * cnt.y * cnt.z;
  float lo = INFINITY, hi = -INFINITY;
  for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < total; i += (long)gridDim.x * blockDim.x) {
    int gx = (int)(i % cnt.x) * stride, gy = (int)((i / cnt.x) % cnt.y) * stride,
        gz = (int)(i / ((long)cnt.x * cnt.y)) * stride;
    float x = f_div(f_add((float)gx, 0.5f), (float)dims.x);
    float y = f_div(f_add((float)gy, 0.5f), (float)dims.y);
    float z = f_div(f_add((float)gz, 0.5f), (float)dims.z);
    float r = inr_raw_fp32<IN, H>(q, sw, x, y, z);
    lo = fminf(lo, r);
    hi = fmaxf(hi, r);
  }
  for (int o = 16; o > 0; o >>= 1) {
    lo = fminf(lo, __shfl_xor_sync(0xffffffffu, lo, o));
    hi = fmaxf(hi, __shfl_xor_sync(0xffffffffu, hi, o));
  }
  if ((threadIdx.x & 31) == 0) {
    atomic_min_f(mm, lo);
    atomic_max_f(mm + 1, hi);
  }
}

__global__ void range_init(float* mm) {
  mm[0] = INFINITY;
  mm[1] = -INFINITY;
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

template <int IN, int H>
int launch_infer(const InrDev& q, const float* xyz, long n, float* out, cudaStream_t s) {
  int smem = mlp_floats<IN, H>() * 4;
  auto k = infer_kernel<IN, H>;
  CINR_CK(cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
  long blocks = (n + 127) / 128;
  long cap = (long)num_sms() * 16;
  if (blocks > cap) blocks = cap;
  k<<<(unsigned)blocks, 128, smem, s>>>(q, xyz, n, out);
  CINR_CK(cudaGetLastError());
  return CINR_OK;
}

template <int IN, int H>
int launch_range(const InrDev& q, int3 dims, int stride, float* mm, cudaStream_t s) {
  int smem = mlp_floats<IN, H>() * 4;
  auto k = range_kernel<IN, H>;
  CINR_CK(cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
  int3 cnt = make_int3((dims.x + stride - 1) / stride, (dims.y + stride - 1) / stride,
                       (dims.z + stride - 1) / stride);
  long total = (long)cnt.x * cnt.y * cnt.z;
  long blocks = (total + 127) / 128;
  long cap = (long)num_sms() * 16;
  if (blocks > cap) blocks = cap;
  range_init<<<1, 1, 0, s>>>(mm);
  k<<<(unsigned)blocks, 128, smem, s>>>(q, dims, stride, cnt, mm);
  CINR_CK(cudaGetLastError());
  return CINR_OK;
}

}  // namespace

extern "C" int cinr_infer(cinr_inr_t inr, const float* xyz_dev, long n, float* out_dev,
                          cinr_stream_t stream) {
  if (!inr) return set_error(CINR_ERR_ARG, "inr is NULL");
  if (n < 0) return set_error(CINR_ERR_ARG, "n < 0");
  if (n == 0) return CINR_OK;
  if (!xyz_dev || !out_dev) return set_error(CINR_ERR_ARG, "NULL buffer");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  if (inr->p.mlp_precision != CINR_PREC_FP32) return cinr_infer_tc(inr, xyz_dev, n, out_dev, s);
  switch (shape_of(inr->dev.IN, inr->dev.H)) {
    case Shape::S16x32: return launch_infer<16, 32>(inr->dev, xyz_dev, n, out_dev, s);
    case Shape::S32x64: return launch_infer<32, 64>(inr->dev, xyz_dev, n, out_dev, s);
    case Shape::S48x64: return launch_infer<48, 64>(inr->dev, xyz_dev, n, out_dev, s);
    default: return set_error(CINR_ERR_ARG, "unsupported shape");
  }
}

extern "C" int cinr_encode(cinr_inr_t inr, const float* xyz_dev, long n, float* feats_dev,
                           uint32_t* idx_dev, cinr_stream_t stream) {
  if (!inr) return set_error(CINR_ERR_ARG, "inr is NULL");
  if (n < 0) return set_error(CINR_ERR_ARG, "n < 0");
  if (n == 0) return CINR_OK;
  if (!xyz_dev || !feats_dev) return set_error(CINR_ERR_ARG, "NULL buffer");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  unsigned blocks = (unsigned)((n + 127) / 128);
  switch (inr->dev.IN) {
    case 16: encode_kernel<16><<<blocks, 128, 0, s>>>(inr->dev, xyz_dev, n, feats_dev, idx_dev); break;
    case 32: encode_kernel<32><<<blocks, 128, 0, s>>>(inr->dev, xyz_dev, n, feats_dev, idx_dev); break;
    case 48: encode_kernel<48><<<blocks, 128, 0, s>>>(inr->dev, xyz_dev, n, feats_dev, idx_dev); break;
    default: return set_error(CINR_ERR_ARG, "unsupported encoding width");
  }
  CINR_CK(cudaGetLastError());
  return CINR_OK;
}

extern "C" int cinr_inr_raw_range(cinr_inr_t inr, const int dims[3], int stride, float* ymin,
                                  float* ymax, cinr_stream_t stream) {
  if (!inr || !dims || !ymin || !ymax) return set_error(CINR_ERR_ARG, "NULL argument");
  if (stride < 1 || dims[0] < 1 || dims[1] < 1 || dims[2] < 1)
    return set_error(CINR_ERR_ARG, "bad dims or stride");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  int3 d = make_int3(dims[0], dims[1], dims[2]);
  int e;
  switch (shape_of(inr->dev.IN, inr->dev.H)) {
    case Shape::S16x32: e = launch_range<16, 32>(inr->dev, d, stride, inr->scratch, s); break;
    case Shape::S32x64: e = launch_range<32, 64>(inr->dev, d, stride, inr->scratch, s); break;
    case Shape::S48x64: e = launch_range<48, 64>(inr->dev, d, stride, inr->scratch, s); break;
    default: return set_error(CINR_ERR_ARG, "unsupported shape");
  }
  if (e) return e;
  float mm[2];
  CINR_CK(cudaMemcpyAsync(mm, inr->scratch, 8, cudaMemcpyDeviceToHost, s));
  CINR_CK(cudaStreamSynchronize(s));
  *ymin = mm[0];
  *ymax = mm[1];
  return CINR_OK;
}
