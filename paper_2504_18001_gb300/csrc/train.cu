// INR training (Sec. 4.1): random-coordinate batches with ground truth from
// an explicit field, MSE on the normalised value, back-propagation through
// the MLP and the hash-grid interpolation (scatter-add of table gradients),
// and Adam on the FP32 master parameters.
//
// Per step:
//   fwd_bwd_kernel   one thread per sample: coordinates (counter-based
//                    SplitMix64), trilinear ground truth, encode, MLP
//                    forward, loss, MLP backward to the feature gradient,
//                    atomic scatter-add into the table gradient; the
//                    activations the weight gradients need are stored
//                    structure-of-arrays (feature-major) for the next kernel;
//   outer_kernel     weight gradients dW = sum_s a_s b_s^T over the batch,
//                    split over blocks (partials), then reduce_kernel;
//   adam_kernel      bias-corrected Adam over table and weights, and the
//                    half-precision weight copy refreshed.
#include <cmath>
#include <cstring>
#include <vector>

#include "cinr_internal.cuh"

using namespace cinr;

struct cinr_trainer_s {
  cinr_inr_s* inr;
  cinr_train_opts o;
  long n_table, n_w;  // parameter counts
  float *m_t, *v_t, *g_t, *m_w, *v_w, *g_w;
  float* act;         // (IN + 4H + 1) x batch, feature-major
  float* partial;     // per-block weight-gradient partials
  float* loss;        // device scalar
  long step;
  int n_part;         // blocks of the outer-product reduction
};

namespace {

constexpr int kChunk = 512;      // samples per block in the weight-gradient reduction
// bit of the trainer's status word
constexpr int kTrainNan = 1;  // a non-finite gradient (Adam)
constexpr int kFwdThreads = 128;

__device__ __forceinline__ uint64_t splitmix64_dev(uint64_t x) {
  uint64_t z = x + 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

// Coordinates of sample s: given, or the counter-based uniform of the step.
__device__ __forceinline__ void train_point(const float* xyz_in, uint64_t seed, uint64_t first, long s,
                                            float& x, float& y, float& z) {
  if (xyz_in) {
    x = xyz_in[3 * s];
    y = xyz_in[3 * s + 1];
    z = xyz_in[3 * s + 2];
  } else {
    const uint64_t c0 = 3ull * (first + (uint64_t)s);
    x = (float)(splitmix64_dev(seed + c0) >> 40) * (1.0f / 16777216.0f);
    y = (float)(splitmix64_dev(seed + c0 + 1) >> 40) * (1.0f / 16777216.0f);
    z = (float)(splitmix64_dev(seed + c0 + 2) >> 40) * (1.0f / 16777216.0f);
  }
  x = clamp01(x);
  y = clamp01(y);
  z = clamp01(z);
}

// Forward pass of a batch (Sec. 4.1): encode, two ReLU layers, linear
// output, squared error against the target; the activations (features,
// h1, h2, dL/dy) go to the feature-major buffers of the weight gradients.
template <int IN, int H>
__global__ void __launch_bounds__(kFwdThreads, IN <= 32 ? 4 : 2) fwd_kernel(InrDev q, long n, const float* __restrict__ xyz_in,
                                                          const float* __restrict__ tgt_in,
                                                          const float* __restrict__ field, int3 dims,
                                                          uint64_t seed, uint64_t first, float* __restrict__ act,
                                                          float* __restrict__ loss) {
  extern __shared__ float4 smem4[];
  float* sw = reinterpret_cast<float*>(smem4);
  load_weights(sw, q.w, mlp_floats<IN, H>());
  __syncthreads();
  const float* W1 = sw;
  const float* W2 = sw + IN * H;
  const float* W3 = W2 + H * H;
  const long s = blockIdx.x * (long)blockDim.x + threadIdx.x;
  float r2 = 0.0f;
  if (s < n) {
    float x, y, z;
    train_point(xyz_in, seed, first, s, x, y, z);
    const float t = tgt_in ? tgt_in[s] : field_trilinear(field, dims, x, y, z);
    float* a_feat = act;
    float* a_h1 = act + (size_t)IN * n;
    float* a_h2 = a_h1 + (size_t)H * n;
    float* a_dy = a_h2 + (size_t)3 * H * n;
    float h1[H];
    {
      float feat[IN];
      encode_point<IN / 2>(q, x, y, z, feat);
#pragma unroll
      for (int k = 0; k < IN; ++k) a_feat[(size_t)k * n + s] = feat[k];
#pragma unroll
      for (int o = 0; o < H; ++o) {
        float acc = 0.0f;
#pragma unroll
        for (int k = 0; k < IN; ++k) acc = fmaf(W1[o * IN + k], feat[k], acc);
        h1[o] = fmaxf(acc, 0.0f);
        a_h1[(size_t)o * n + s] = h1[o];
      }
    }
    float yv = 0.0f;
#pragma unroll 4
    for (int o = 0; o < H; ++o) {
      float acc = 0.0f;
#pragma unroll
      for (int k = 0; k < H; ++k) acc = fmaf(W2[o * H + k], h1[k], acc);
      const float h2 = fmaxf(acc, 0.0f);
      a_h2[(size_t)o * n + s] = h2;
      yv = fmaf(W3[o], h2, yv);
    }
    const float r = yv - t;
    r2 = r * r;
    a_dy[s] = 2.0f * r / (float)n;
  }
  if (loss) {
    for (int o = 16; o > 0; o >>= 1) r2 += __shfl_xor_sync(0xffffffffu, r2, o);
    if ((threadIdx.x & 31) == 0 && r2 != 0.0f) atomicAdd(loss, r2 / (float)n);
  }
}

// Backward pass: through the output and second layer (dh2 = dy W3 on the
// active units, dh1 = W2^T dh2 on the active units of h1), the first layer
// (dfeat = W1^T dh1), then through the trilinear hash-grid interpolation:
// each vertex entry receives weight * dfeat by atomicAdd.  h1 > 0 and
// h2 > 0 are the ReLU masks (a unit is active exactly when its output is
// positive).
template <int IN, int H>
__global__ void __launch_bounds__(kFwdThreads, IN <= 32 ? 4 : 2) bwd_kernel(InrDev q, long n, const float* __restrict__ xyz_in,
                                                          uint64_t seed, uint64_t first, float* __restrict__ act,
                                                          float* __restrict__ g_table) {
  extern __shared__ float4 smem4[];
  float* sw = reinterpret_cast<float*>(smem4);
  load_weights(sw, q.w, mlp_floats<IN, H>());
  __syncthreads();
  const float* W1 = sw;
  const float* W2 = sw + IN * H;
  const float* W3 = W2 + H * H;
  const long s = blockIdx.x * (long)blockDim.x + threadIdx.x;
  if (s >= n) return;
  const float* a_h1 = act + (size_t)IN * n;
  const float* a_h2 = a_h1 + (size_t)H * n;
  float* a_dh1 = const_cast<float*>(a_h2) + (size_t)H * n;
  float* a_dh2 = a_dh1 + (size_t)H * n;
  const float dy = act[(size_t)IN * n + (size_t)4 * H * n + s];
  float dh1[H];
#pragma unroll
  for (int k = 0; k < H; ++k) dh1[k] = 0.0f;
#pragma unroll 4
  for (int o = 0; o < H; ++o) {
    const float dh2 = a_h2[(size_t)o * n + s] > 0.0f ? dy * W3[o] : 0.0f;
    a_dh2[(size_t)o * n + s] = dh2;
#pragma unroll
    for (int k = 0; k < H; ++k) dh1[k] = fmaf(W2[o * H + k], dh2, dh1[k]);
  }
#pragma unroll
  for (int k = 0; k < H; ++k) {
    dh1[k] = a_h1[(size_t)k * n + s] > 0.0f ? dh1[k] : 0.0f;
    a_dh1[(size_t)k * n + s] = dh1[k];
  }
  float dfeat[IN];
#pragma unroll
  for (int k = 0; k < IN; ++k) {
    float acc = 0.0f;
#pragma unroll
    for (int o = 0; o < H; ++o) acc = fmaf(W1[o * IN + k], dh1[o], acc);
    dfeat[k] = acc;
  }
  float x, y, z;
  train_point(xyz_in, seed, first, s, x, y, z);
  const uint32_t T = 1u << q.log2T;
#pragma unroll
  for (int l = 0; l < IN / 2; ++l) {
    const int N = q.res[l];
    int ix, iy, iz;
    float wx, wy, wz;
    grid_cell(x, N, ix, wx);
    grid_cell(y, N, iy, wy);
    grid_cell(z, N, iz, wz);
    const bool dense = (q.dense_mask >> l) & 1u;
    const uint32_t n1 = (uint32_t)N + 1u;
#pragma unroll
    for (int c = 0; c < 8; ++c) {
      const float w = ((c & 1) ? wx : 1.0f - wx) * ((c & 2) ? wy : 1.0f - wy) *
                      ((c & 4) ? wz : 1.0f - wz);
      const uint32_t idx = (uint32_t)l * T + vertex_index(dense, n1, T, ix + (c & 1),
                                                          iy + ((c >> 1) & 1), iz + ((c >> 2) & 1));
      // both features of the entry in one 8-byte vector atomic
      atomicAdd(reinterpret_cast<float2*>(g_table) + idx, make_float2(w * dfeat[2 * l], w * dfeat[2 * l + 1]));
    }
  }
}

// partial[blk][i][j] = sum over the block's samples of A[i][s] * B[j][s]
// (A: M x n, B: N x n, feature-major).  Thread tile 4 x 4; the staged
// tiles are sample-major in shared memory so that a thread reads its four
// rows of A and four columns of B as one 16-byte load each (the loads, not
// the FMAs, bounded the scalar-load version).
template <int M, int N>
__global__ void __launch_bounds__((M / 4) * (N / 4)) outer_kernel(const float* __restrict__ A,
                                                                  const float* __restrict__ B, long n,
                                                                  float* __restrict__ partial) {
  constexpr int TPB = (M / 4) * (N / 4);
  constexpr int SUB = 32;
  __shared__ __align__(16) float sa[SUB][M + 4];
  __shared__ __align__(16) float sb[SUB][N + 4];
  const int tid = threadIdx.x;
  const int ti = (tid / (N / 4)) * 4, tj = (tid % (N / 4)) * 4;
  float acc[4][4] = {};
  const long s0 = (long)blockIdx.x * kChunk;
  const long s1 = s0 + kChunk < n ? s0 + kChunk : n;
  // the next tile is fetched into registers while the current one is used
  constexpr int PA = (M * SUB + TPB - 1) / TPB, PB = (N * SUB + TPB - 1) / TPB;
  float ra[PA], rb[PB];
  auto fetch = [&](long base) {
#pragma unroll
    for (int q = 0; q < PA; ++q) {
      const int e = tid + q * TPB, i = e / SUB, k = e % SUB;
      ra[q] = e < M * SUB && base + k < s1 ? A[(size_t)i * n + base + k] : 0.0f;
    }
#pragma unroll
    for (int q = 0; q < PB; ++q) {
      const int e = tid + q * TPB, j = e / SUB, k = e % SUB;
      rb[q] = e < N * SUB && base + k < s1 ? B[(size_t)j * n + base + k] : 0.0f;
    }
  };
  fetch(s0);
  for (long base = s0; base < s1; base += SUB) {
#pragma unroll
    for (int q = 0; q < PA; ++q) {
      const int e = tid + q * TPB;
      if (e < M * SUB) sa[e % SUB][e / SUB] = ra[q];
    }
#pragma unroll
    for (int q = 0; q < PB; ++q) {
      const int e = tid + q * TPB;
      if (e < N * SUB) sb[e % SUB][e / SUB] = rb[q];
    }
    __syncthreads();
    if (base + SUB < s1) fetch(base + SUB);
#pragma unroll 8
    for (int k = 0; k < SUB; ++k) {
      const float4 a4 = *reinterpret_cast<const float4*>(&sa[k][ti]);
      const float4 b4 = *reinterpret_cast<const float4*>(&sb[k][tj]);
      const float a[4] = {a4.x, a4.y, a4.z, a4.w}, b[4] = {b4.x, b4.y, b4.z, b4.w};
#pragma unroll
      for (int u = 0; u < 4; ++u)
#pragma unroll
        for (int v = 0; v < 4; ++v) acc[u][v] = fmaf(a[u], b[v], acc[u][v]);
    }
    __syncthreads();
  }
  float* out = partial + (size_t)blockIdx.x * M * N;
#pragma unroll
  for (int u = 0; u < 4; ++u)
#pragma unroll
    for (int v = 0; v < 4; ++v) out[(ti + u) * N + tj + v] = acc[u][v];
}

// partial[blk][j] = sum over the block's samples of a[s] * B[j][s]: each
// warp takes N/8 of the outputs, its lanes stride over the block's samples
// (a[s] read once per lane for all of the warp's outputs), then a warp sum.
template <int N>
__global__ void __launch_bounds__(256) vec_kernel(const float* __restrict__ a, const float* __restrict__ B,
                                                  long n, float* __restrict__ partial) {
  static_assert(N % 8 == 0, "8 warps share the outputs");
  constexpr int J = N / 8;
  const long s0 = (long)blockIdx.x * kChunk;
  const long s1 = s0 + kChunk < n ? s0 + kChunk : n;
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  float acc[J] = {};
  for (long s = s0 + lane; s < s1; s += 32) {
    const float as = a[s];
#pragma unroll
    for (int q = 0; q < J; ++q) acc[q] = fmaf(as, B[(size_t)(w * J + q) * n + s], acc[q]);
  }
#pragma unroll
  for (int q = 0; q < J; ++q) {
    float t = acc[q];
    for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
    if (lane == 0) partial[(size_t)blockIdx.x * N + w * J + q] = t;
  }
}

// out[i] = sum over b of partial[b][i]: a CTA takes 32 outputs (one per
// lane), its 8 warps sum interleaved eighths of the partials, then the
// warps' sums are added in a fixed order.
__global__ void __launch_bounds__(256) reduce_kernel(const float* __restrict__ partial, int blocks, int count,
                                                     float* __restrict__ out) {
  __shared__ float red[8][32];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int i = blockIdx.x * 32 + lane;
  float t = 0.0f;
  if (i < count)
    for (int b = w; b < blocks; b += 8) t += partial[(size_t)b * count + i];
  red[w][lane] = t;
  __syncthreads();
  if (w == 0 && i < count) {
    float u = 0.0f;
#pragma unroll
    for (int q = 0; q < 8; ++q) u += red[q][lane];
    out[i] = u;
  }
}

// Bias-corrected Adam (Kingma & Ba): c1 = 1 - b1^t, c2 = 1 - b2^t.  A
// non-finite gradient sets *bad (read by cinr_trainer_status).
__device__ __forceinline__ void adam_one(float& p, float g, float& m, float& v, float lr, float b1, float b2,
                                         float eps, float c1, float c2, bool& nonfinite) {
  nonfinite |= !isfinite(g);
  m = b1 * m + (1.0f - b1) * g;
  v = b2 * v + (1.0f - b2) * g * g;
  p -= lr * (m / c1) / (sqrtf(v / c2) + eps);
}

// Four parameters per thread and iteration with 16-byte loads and stores
// (the update is elementwise: the same arithmetic as one at a time), the
// n % 4 tail one at a time.
__global__ void adam_kernel(float* __restrict__ p, const float* __restrict__ g, float* __restrict__ m,
                            float* __restrict__ v, long n, float lr, float b1, float b2, float eps,
                            float c1, float c2, int* __restrict__ bad) {
  bool nonfinite = false;
  const long n4 = n >> 2;
  const long stride = (long)gridDim.x * blockDim.x;
  float4* p4 = reinterpret_cast<float4*>(p);
  float4* m4 = reinterpret_cast<float4*>(m);
  float4* v4 = reinterpret_cast<float4*>(v);
  const float4* g4 = reinterpret_cast<const float4*>(g);
  for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < n4; i += stride) {
    float4 pp = p4[i], mm = m4[i], vv = v4[i];
    const float4 gg = g4[i];
    adam_one(pp.x, gg.x, mm.x, vv.x, lr, b1, b2, eps, c1, c2, nonfinite);
    adam_one(pp.y, gg.y, mm.y, vv.y, lr, b1, b2, eps, c1, c2, nonfinite);
    adam_one(pp.z, gg.z, mm.z, vv.z, lr, b1, b2, eps, c1, c2, nonfinite);
    adam_one(pp.w, gg.w, mm.w, vv.w, lr, b1, b2, eps, c1, c2, nonfinite);
    p4[i] = pp;
    m4[i] = mm;
    v4[i] = vv;
  }
  for (long i = (n4 << 2) + blockIdx.x * (long)blockDim.x + threadIdx.x; i < n; i += stride) {
    float pp = p[i], mm = m[i], vv = v[i];
    adam_one(pp, g[i], mm, vv, lr, b1, b2, eps, c1, c2, nonfinite);
    p[i] = pp;
    m[i] = mm;
    v[i] = vv;
  }
  if (nonfinite) atomicOr(bad, kTrainNan);
}

__global__ void half_copy_kernel(const float* __restrict__ w, uint16_t* __restrict__ w16, int n, int bf16) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  if (bf16) {
    __nv_bfloat16 b = __float2bfloat16_rn(w[i]);
    w16[i] = *reinterpret_cast<uint16_t*>(&b);
  } else {
    __half h = __float2half_rn(w[i]);
    w16[i] = *reinterpret_cast<uint16_t*>(&h);
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

struct TrainLayout {
  float *m_t, *v_t, *g_t, *m_w, *v_w, *g_w, *act, *partial, *loss;
  size_t bytes;
};

TrainLayout tlayout(const cinr_inr_s* inr, long batch, void* base) {
  const long nt = (long)inr->p.levels * (1l << inr->p.log2_table) * 2;
  const int IN = inr->dev.IN, H = inr->dev.H;
  const long nw = (long)H * IN + (long)H * H + H;
  const long blocks = (batch + kChunk - 1) / kChunk;
  Carver c(base);
  TrainLayout L;
  L.m_t = c.take<float>(nt);
  L.v_t = c.take<float>(nt);
  L.g_t = c.take<float>(nt);
  L.m_w = c.take<float>(nw);
  L.v_w = c.take<float>(nw);
  L.g_w = c.take<float>(nw);
  L.act = c.take<float>((size_t)(IN + 4 * H + 1) * batch);
  L.partial = c.take<float>((size_t)blocks * nw);
  L.loss = c.take<float>(64);
  L.bytes = align_up(c.off, 256);
  return L;
}

int check(const cinr_inr_s* inr, const cinr_train_opts* o) {
  if (!inr || !o) return set_error(CINR_ERR_ARG, "NULL argument");
  if (inr->p.table_precision != CINR_PREC_FP32) return set_error(CINR_ERR_ARG, "training needs an FP32 table");
  if (o->batch < 1 || o->batch > (1l << 26)) return set_error(CINR_ERR_ARG, "batch must be in [1, 2^26]");
  if (!(o->lr > 0.0f) || !(o->beta1 >= 0.0f && o->beta1 < 1.0f) || !(o->beta2 >= 0.0f && o->beta2 < 1.0f))
    return set_error(CINR_ERR_ARG, "bad Adam hyper-parameters");
  return CINR_OK;
}

template <int IN, int H>
int grads(cinr_trainer_s* t, const float* xyz, const float* tgt, long n, const float* field, int3 dims,
          uint64_t first, float* g_table, float* g_w, cudaStream_t s) {
  const InrDev& q = t->inr->dev;
  CINR_CK(cudaMemsetAsync(g_table, 0, sizeof(float) * t->n_table, s));
  const int smem = mlp_floats<IN, H>() * 4;
  auto kf = fwd_kernel<IN, H>;
  auto kb = bwd_kernel<IN, H>;
  CINR_CK(cudaFuncSetAttribute(kf, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
  CINR_CK(cudaFuncSetAttribute(kb, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
  const unsigned grid = (unsigned)((n + kFwdThreads - 1) / kFwdThreads);
  kf<<<grid, kFwdThreads, smem, s>>>(q, n, xyz, tgt, field, dims, t->o.seed, first, t->act, t->loss);
  kb<<<grid, kFwdThreads, smem, s>>>(q, n, xyz, t->o.seed, first, t->act, g_table);
  CINR_CK(cudaGetLastError());
  const int blocks = (int)((n + kChunk - 1) / kChunk);
  const float* a_feat = t->act;
  const float* a_h1 = a_feat + (size_t)IN * n;
  const float* a_h2 = a_h1 + (size_t)H * n;
  const float* a_dh1 = a_h2 + (size_t)H * n;
  const float* a_dh2 = a_dh1 + (size_t)H * n;
  const float* a_dy = a_dh2 + (size_t)H * n;
  float* p1 = t->partial;
  float* p2 = p1 + (size_t)blocks * H * IN;
  float* p3 = p2 + (size_t)blocks * H * H;
  outer_kernel<H, IN><<<blocks, (H / 4) * (IN / 4), 0, s>>>(a_dh1, a_feat, n, p1);
  outer_kernel<H, H><<<blocks, (H / 4) * (H / 4), 0, s>>>(a_dh2, a_h1, n, p2);
  vec_kernel<H><<<blocks, 256, 0, s>>>(a_dy, a_h2, n, p3);
  reduce_kernel<<<(H * IN + 31) / 32, 256, 0, s>>>(p1, blocks, H * IN, g_w);
  reduce_kernel<<<(H * H + 31) / 32, 256, 0, s>>>(p2, blocks, H * H, g_w + H * IN);
  reduce_kernel<<<(H + 31) / 32, 256, 0, s>>>(p3, blocks, H, g_w + H * IN + H * H);
  CINR_CK(cudaGetLastError());
  return CINR_OK;
}

int grads_dispatch(cinr_trainer_s* t, const float* xyz, const float* tgt, long n, const float* field,
                   int3 dims, uint64_t first, float* g_table, float* g_w, cudaStream_t s) {
  switch (shape_of(t->inr->dev.IN, t->inr->dev.H)) {
    case Shape::S16x32: return grads<16, 32>(t, xyz, tgt, n, field, dims, first, g_table, g_w, s);
    case Shape::S32x64: return grads<32, 64>(t, xyz, tgt, n, field, dims, first, g_table, g_w, s);
    case Shape::S48x64: return grads<48, 64>(t, xyz, tgt, n, field, dims, first, g_table, g_w, s);
    default: return set_error(CINR_ERR_ARG, "unsupported shape");
  }
}

}  // namespace

extern "C" int cinr_trainer_bytes(cinr_inr_t inr, const cinr_train_opts* o, size_t* bytes) {
  int e = check(inr, o);
  if (e) return e;
  if (!bytes) return set_error(CINR_ERR_ARG, "bytes is NULL");
  *bytes = tlayout(inr, o->batch, nullptr).bytes;
  return CINR_OK;
}

extern "C" int cinr_create_trainer(cinr_inr_t inr, const cinr_train_opts* o, void* dev_mem, size_t bytes,
                                   cinr_stream_t stream, cinr_trainer_t* out) {
  int e = check(inr, o);
  if (e) return e;
  if (!out) return set_error(CINR_ERR_ARG, "out is NULL");
  if (!dev_mem || (reinterpret_cast<uintptr_t>(dev_mem) & 255))
    return set_error(CINR_ERR_ARG, "dev_mem must be non-NULL and 256-byte aligned");
  TrainLayout L = tlayout(inr, o->batch, dev_mem);
  if (bytes < L.bytes) return set_error(CINR_ERR_NOMEM, "trainer needs %zu bytes, got %zu", L.bytes, bytes);
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  CINR_CK(cudaMemsetAsync(L.m_t, 0, sizeof(float) * (size_t)inr->p.levels * ((size_t)1 << inr->p.log2_table) * 2, s));
  CINR_CK(cudaMemsetAsync(L.v_t, 0, sizeof(float) * (size_t)inr->p.levels * ((size_t)1 << inr->p.log2_table) * 2, s));
  cinr_trainer_s* t = new cinr_trainer_s();
  t->inr = inr;
  t->o = *o;
  t->n_table = (long)inr->p.levels * (1l << inr->p.log2_table) * 2;
  t->n_w = (long)inr->dev.H * inr->dev.IN + (long)inr->dev.H * inr->dev.H + inr->dev.H;
  t->m_t = L.m_t;
  t->v_t = L.v_t;
  t->g_t = L.g_t;
  t->m_w = L.m_w;
  t->v_w = L.v_w;
  t->g_w = L.g_w;
  t->act = L.act;
  t->partial = L.partial;
  t->loss = L.loss;
  t->step = 0;
  t->n_part = (int)((o->batch + kChunk - 1) / kChunk);
  cudaError_t ce = cudaMemsetAsync(L.m_w, 0, sizeof(float) * t->n_w, s);
  if (ce == cudaSuccess) ce = cudaMemsetAsync(L.v_w, 0, sizeof(float) * t->n_w, s);
  if (ce == cudaSuccess) ce = cudaMemsetAsync(L.loss, 0, 64 * sizeof(float), s);
  if (ce != cudaSuccess) {
    delete t;
    return cuda_error(ce, "cudaMemsetAsync");
  }
  *out = t;
  return CINR_OK;
}

extern "C" int cinr_destroy_trainer(cinr_trainer_t t) {
  delete t;
  return CINR_OK;
}

extern "C" int cinr_trainer_set_lr(cinr_trainer_t t, float lr) {
  if (!t) return set_error(CINR_ERR_ARG, "NULL argument");
  if (!(lr > 0.0f)) return set_error(CINR_ERR_ARG, "lr must be positive");
  t->o.lr = lr;
  return CINR_OK;
}

extern "C" int cinr_trainer_status(cinr_trainer_t t, cinr_stream_t stream) {
  if (!t) return set_error(CINR_ERR_ARG, "NULL argument");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  int* bad = reinterpret_cast<int*>(t->loss + 1);
  int h = 0;
  CINR_CK(cudaMemcpyAsync(&h, bad, sizeof(int), cudaMemcpyDeviceToHost, s));
  CINR_CK(cudaStreamSynchronize(s));
  if (!h) return CINR_OK;
  CINR_CK(cudaMemsetAsync(bad, 0, sizeof(int), s));
  return set_error(CINR_ERR_NAN, "a training step produced a non-finite gradient");
}

extern "C" int cinr_train(cinr_inr_t inr, const float* field_dev, const int dims[3], const cinr_train_opts* o,
                          long steps, void* workspace, size_t ws_bytes, cinr_stream_t stream) {
  if (steps < 0) return set_error(CINR_ERR_ARG, "steps must be >= 0");
  cinr_trainer_t t = nullptr;
  int e = cinr_create_trainer(inr, o, workspace, ws_bytes, stream, &t);
  if (e) return e;
  for (long i = 0; i < steps && !e; ++i) e = cinr_train_step(t, field_dev, dims, nullptr, stream);
  if (!e) e = cinr_trainer_status(t, stream);
  cinr_destroy_trainer(t);
  return e;
}

extern "C" int cinr_train_step(cinr_trainer_t t, const float* field_dev, const int dims[3], float* loss_dev,
                               cinr_stream_t stream) {
  if (!t || !field_dev || !dims) return set_error(CINR_ERR_ARG, "NULL argument");
  if (dims[0] < 1 || dims[1] < 1 || dims[2] < 1) return set_error(CINR_ERR_ARG, "bad field dims");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const long n = t->o.batch;
  t->step += 1;
  CINR_CK(cudaMemsetAsync(t->loss, 0, 4, s));
  int e = grads_dispatch(t, nullptr, nullptr, n, field_dev, make_int3(dims[0], dims[1], dims[2]),
                         (uint64_t)(t->step - 1) * (uint64_t)n, t->g_t, t->g_w, s);
  if (e) return e;
  const double c1 = 1.0 - pow((double)t->o.beta1, (double)t->step);
  const double c2 = 1.0 - pow((double)t->o.beta2, (double)t->step);
  float* table = const_cast<float*>(static_cast<const float*>(t->inr->dev.table));
  float* w = const_cast<float*>(t->inr->dev.w);
  const unsigned gb = (unsigned)num_sms() * 8;
  int* bad = reinterpret_cast<int*>(t->loss + 1);
  adam_kernel<<<gb, 256, 0, s>>>(table, t->g_t, t->m_t, t->v_t, t->n_table, t->o.lr, t->o.beta1, t->o.beta2,
                                 t->o.eps, (float)c1, (float)c2, bad);
  adam_kernel<<<(unsigned)((t->n_w + 255) / 256), 256, 0, s>>>(w, t->g_w, t->m_w, t->v_w, t->n_w, t->o.lr,
                                                              t->o.beta1, t->o.beta2, t->o.eps, (float)c1,
                                                              (float)c2, bad);
  half_copy_kernel<<<(unsigned)((t->n_w + 255) / 256), 256, 0, s>>>(
      w, t->inr->w16, (int)t->n_w, t->inr->p.mlp_precision == CINR_PREC_BF16);
  CINR_CK(cudaGetLastError());
  if (loss_dev) CINR_CK(cudaMemcpyAsync(loss_dev, t->loss, 4, cudaMemcpyDeviceToDevice, s));
  return CINR_OK;
}

extern "C" int cinr_inr_loss_grad(cinr_trainer_t t, const float* xyz_dev, const float* target_dev, long n,
                                  float* g_table_dev, float* g_mlp_dev, float* loss_dev, cinr_stream_t stream) {
  if (!t || !xyz_dev || !target_dev || !g_table_dev || !g_mlp_dev) return set_error(CINR_ERR_ARG, "NULL argument");
  if (n < 1 || n > t->o.batch) return set_error(CINR_ERR_ARG, "n must be in [1, batch]");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  CINR_CK(cudaMemsetAsync(t->loss, 0, 4, s));
  int e = grads_dispatch(t, xyz_dev, target_dev, n, nullptr, make_int3(1, 1, 1), 0, g_table_dev, g_mlp_dev, s);
  if (e) return e;
  if (loss_dev) CINR_CK(cudaMemcpyAsync(loss_dev, t->loss, 4, cudaMemcpyDeviceToDevice, s));
  return CINR_OK;
}

extern "C" int cinr_inr_export(cinr_inr_t inr, float* host_table, float* host_mlp, cinr_stream_t stream) {
  if (!inr || !host_table || !host_mlp) return set_error(CINR_ERR_ARG, "NULL argument");
  if (inr->p.table_precision != CINR_PREC_FP32) return set_error(CINR_ERR_ARG, "export needs an FP32 table");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const size_t nt = (size_t)inr->p.levels * ((size_t)1 << inr->p.log2_table) * 2;
  const size_t nw = (size_t)inr->dev.H * inr->dev.IN + (size_t)inr->dev.H * inr->dev.H + inr->dev.H;
  CINR_CK(cudaMemcpyAsync(host_table, inr->dev.table, nt * 4, cudaMemcpyDeviceToHost, s));
  CINR_CK(cudaMemcpyAsync(host_mlp, inr->dev.w, nw * 4, cudaMemcpyDeviceToHost, s));
  CINR_CK(cudaStreamSynchronize(s));
  return CINR_OK;
}
