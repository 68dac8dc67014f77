// INR training (Sec. 4.1): random-coordinate batches with ground truth from
// an explicit field, MSE on the normalised value, back-propagation through
// the MLP and the hash-grid interpolation (scatter-add of table gradients),
// and Adam on the FP32 master parameters.
//
// Per step, either
//   train_tc_kernel  one fused kernel over 128-sample tiles: coordinates
//                    (counter-based SplitMix64), trilinear ground truth,
//                    encode, the MLP's forward, backward and weight-gradient
//                    products on the tensor cores (FP16 or BF16 operands,
//                    FP32 accumulation), loss, dW3, scatter-add into the
//                    table gradient; the CTAs' weight-gradient partials go
//                    to reduce_kernel;
// or the FP32 kernels
//   fwd_kernel       one thread per sample: coordinates, ground truth,
//                    encode, MLP forward, loss; activations stored
//                    feature-major for the weight gradients;
//   bwd_kernel       MLP backward to the feature gradient, scatter-add into
//                    the table gradient;
//   outer_kernel /   weight gradients dW = sum_s a_s b_s^T over the batch,
//   vec_kernel       split over blocks (partials), then reduce_kernel;
// then
//   adam_kernel      bias-corrected Adam over table and weights, and the
//                    half-precision weight copy refreshed.
#include <cmath>
#include <cstring>
#include <vector>

#include "cinr_internal.cuh"
#include "tc_mlp.cuh"

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
  int tc;             // fused tensor-core forward / backward (train_tc_kernel): 1 FP16, 2 BF16; 0 FP32 kernels
  int strat;          // 1: stratified coordinates (train_point)
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
// strat = g >= 0 (stratified sampling): samples s < 8^g take one point
// each in cell s of a 2^g grid over the unit cube, cells in Morton order
// (consecutive samples are spatially close), the point uniform in its cell
// from the same counter-based draws; the others (and strat < 0) are
// uniform in the cube.  Either way every sample is uniform over its stratum
// and the batch is an unbiased estimate of the field's mean squared error.
__device__ __forceinline__ uint32_t morton_compact3(uint32_t v) {
  v &= 0x09249249u;
  v = (v ^ (v >> 2)) & 0x030C30C3u;
  v = (v ^ (v >> 4)) & 0x0300F00Fu;
  v = (v ^ (v >> 8)) & 0x030000FFu;
  v = (v ^ (v >> 16)) & 0x000003FFu;
  return v;
}

__device__ __forceinline__ void train_point(const float* xyz_in, uint64_t seed, uint64_t first, long s,
                                            float& x, float& y, float& z, int strat = -1) {
  if (xyz_in) {
    x = xyz_in[3 * s];
    y = xyz_in[3 * s + 1];
    z = xyz_in[3 * s + 2];
  } else {
    const uint64_t c0 = 3ull * (first + (uint64_t)s);
    x = (float)(splitmix64_dev(seed + c0) >> 40) * (1.0f / 16777216.0f);
    y = (float)(splitmix64_dev(seed + c0 + 1) >> 40) * (1.0f / 16777216.0f);
    z = (float)(splitmix64_dev(seed + c0 + 2) >> 40) * (1.0f / 16777216.0f);
    if (strat >= 0 && s < (1l << (3 * strat))) {
      const uint32_t m = (uint32_t)s;
      const float inv = __int_as_float((127 - strat) << 23);  // 2^-g, exact
      x = ((float)morton_compact3(m) + x) * inv;
      y = ((float)morton_compact3(m >> 1) + y) * inv;
      z = ((float)morton_compact3(m >> 2) + z) * inv;
    }
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
                                                          float* __restrict__ loss, int strat) {
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
    train_point(xyz_in, seed, first, s, x, y, z, strat);
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
                                                          float* __restrict__ g_table, int strat) {
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
  train_point(xyz_in, seed, first, s, x, y, z, strat);
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

// ------------------------------------------------ fused tensor-core step
// Forward and backward of a 128-sample tile in one kernel, the MLP's five
// products on the tensor cores (tcgen05.mma kind::f16, FP16 or BF16
// operands, FP32 accumulation in tensor memory):
//   h1 = relu(feat W1^T)          A = features (K-major), B = W1 (K-major)
//   h2 = relu(h1 W2^T)            A = h1, B = W2
//   dh1 = (dh2 W2) on h1 > 0      A = dh2 (K-major), B = W2 read MN-major
//   dfeat = dh1 W1                A = dh1, B = W1 read MN-major
//   [dW2; dW1] += [dh2; dh1]^T [h1, feat]   A and B read MN-major, K = samples
// The activations of a tile stay in shared memory, in two buffers of
// core matrices (8 samples x 16 bytes): HF holds [h1 | feat] and DD holds
// [dh2 | dh1] (dh2 in columns 0 .. H-1, dh1 in 64 .. 64+H-1, the rest
// zero), each read as a K-major operand (rows = samples) by the per-sample
// products and as an MN-major operand (K = samples) by the weight-gradient
// product, which accumulates over all of the CTA's tiles in tensor memory
// (its off-diagonal blocks, dh2 feat^T and dh1 h1^T, are not used).  The
// output layer (H -> 1), the loss and dW3 stay in FP32 per thread; the
// table gradient is scattered as in bwd_kernel.  The back-propagated
// operands carry dL/dy as 2 r S (not 2 r / n), S = 256 for FP16 (a fixed
// power-of-two loss scale that keeps them in FP16's normal range while the
// residuals shrink; FP16 holds 11 significant bits against BF16's 8) and 1
// for BF16; 1/(n S) is applied in FP32 to the scattered and the written
// gradients.
constexpr int kTcTrainCols = 256;  // TMEM: h / dfeat in 0 .. 63, dW from 128
constexpr int kTrainTimeout = 2;   // a bounded tensor-core wait gave up

template <int IN, int H>
struct TrainTcSmem {
  static constexpr int NG = (H + IN) / 8;            // core-matrix columns of HF
  alignas(1024) unsigned char hf[128 * (H + IN) * 2];  // [h1 | feat], 128 samples
  alignas(128) unsigned char dd[128 * 128 * 2];        // [dh2 | 0 | dh1 | 0]
  alignas(128) unsigned char w1[H * IN * 2];           // W1 [H][IN], K-major
  alignas(128) unsigned char w2[H * H * 2];            // W2 [H][H], K-major
  float w3[H];
  float g3[H];  // dW3 of the CTA
  uint64_t bar;
  uint32_t tmem;
};

// Byte offset of element (r, c) of a K-major BF16 operand whose rows hold
// `groups` core-matrix columns of 8 elements.
__device__ __forceinline__ uint32_t cm_off(int r, int c, int groups) {
  return (uint32_t)((((r >> 3) * groups + (c >> 3)) << 7) + ((r & 7) << 4) + ((c & 7) << 1));
}

// Two values as an FP16 (FMT 0) or BF16 (FMT 1) pair, lo in the low half;
// the _relu form clamps negative values to zero.
template <int FMT>
__device__ __forceinline__ uint32_t pack2_relu(float lo, float hi) {
  uint32_t w;
  if (FMT == 1)
    asm("cvt.rn.relu.bf16x2.f32 %0, %1, %2;" : "=r"(w) : "f"(hi), "f"(lo));
  else
    asm("cvt.rn.relu.f16x2.f32 %0, %1, %2;" : "=r"(w) : "f"(hi), "f"(lo));
  return w;
}
template <int FMT>
__device__ __forceinline__ uint32_t pack2(float lo, float hi) {
  if (FMT == 1) {
    __nv_bfloat162 b = __floats2bfloat162_rn(lo, hi);
    return *reinterpret_cast<uint32_t*>(&b);
  }
  __half2 h = __floats2half2_rn(lo, hi);
  return *reinterpret_cast<uint32_t*>(&h);
}

// Eight values of row r, columns c0 .. c0+7, as one 16-byte store.
__device__ __forceinline__ void st8(unsigned char* buf, int r, int c0, int groups, uint32_t a, uint32_t b,
                                    uint32_t c, uint32_t d) {
  *reinterpret_cast<uint4*>(buf + cm_off(r, c0, groups)) = make_uint4(a, b, c, d);
}

template <int IN, int H, int FMT>
__global__ void __launch_bounds__(128, 2) train_tc_kernel(InrDev q, long n, const float* __restrict__ xyz_in,
                                                          const float* __restrict__ tgt_in,
                                                          const float* __restrict__ field, int3 dims, uint64_t seed,
                                                          uint64_t first, float* __restrict__ g_table,
                                                          float* __restrict__ p1, float* __restrict__ p2,
                                                          float* __restrict__ p3, float* __restrict__ loss,
                                                          int* __restrict__ status, int strat) {
  using SM = TrainTcSmem<IN, H>;
  constexpr int NG = SM::NG;
  static_assert(IN % 16 == 0 && H % 16 == 0 && H <= 64 && (H + IN) % 16 == 0, "fused training shape");
  extern __shared__ __align__(1024) unsigned char smraw[];
  SM& sm = *reinterpret_cast<SM*>(smraw);
  const int t = threadIdx.x, warp = t >> 5;
  constexpr float kScale = FMT == 0 ? 256.0f : 1.0f;  // loss scale of the back-propagated operands
  const float inv_n = 1.0f / (float)n;
  const float inv_ns = inv_n * (1.0f / kScale);
  // weights as 16-bit operands, W3 in FP32; DD's unused columns zero
  for (int e = t; e < H * IN; e += 128)
    *reinterpret_cast<uint16_t*>(sm.w1 + cm_off(e / IN, e % IN, IN / 8)) = tc::to16<FMT == 1>(q.w[e]);
  for (int e = t; e < H * H; e += 128)
    *reinterpret_cast<uint16_t*>(sm.w2 + cm_off(e / H, e % H, H / 8)) = tc::to16<FMT == 1>(q.w[H * IN + e]);
  for (int e = t; e < H; e += 128) {
    sm.w3[e] = q.w[H * IN + H * H + e];
    sm.g3[e] = 0.0f;
  }
  for (int e = t; e < 128 * 16; e += 128)  // 16-byte units of DD
    reinterpret_cast<uint4*>(sm.dd)[e] = make_uint4(0u, 0u, 0u, 0u);
  if (t == 0) tc::mbar_init(&sm.bar, 1);
  if (t < 32) tc::tmem_alloc(&sm.tmem, kTcTrainCols);
  tc::fence_proxy_async();
  tc::fence_before();
  __syncthreads();
  tc::fence_after();
  const uint32_t dh = sm.tmem, dw = sm.tmem + 128u;
  const uint32_t lane = (uint32_t)(warp * 32) << 16;
  const uint32_t a_hf = tc::smem_u32(sm.hf), a_dd = tc::smem_u32(sm.dd);
  const uint32_t a_w1 = tc::smem_u32(sm.w1), a_w2 = tc::smem_u32(sm.w2);
  constexpr uint32_t fc = tc::Fmt<FMT>::code;
  constexpr uint32_t id_h = tc::idesc_f16(128, H, fc);
  constexpr uint32_t id_hT = id_h | (1u << 16);                           // B MN-major
  constexpr uint32_t id_fT = tc::idesc_f16(128, IN, fc) | (1u << 16);     // B MN-major
  constexpr uint32_t id_w = tc::idesc_f16(128, H + IN, fc) | (1u << 15) | (1u << 16);  // A, B MN-major
  uint32_t phase = 0;
  bool ok = true;
  float g3[H];
#pragma unroll
  for (int o = 0; o < H; ++o) g3[o] = 0.0f;
  float r2 = 0.0f;
  auto wait_mma = [&]() {
    ok = tc::mbar_wait(&sm.bar, phase) && ok;
    phase ^= 1u;
    tc::fence_after();
  };
  auto sync_for_mma = [&]() {
    tc::fence_before();
    tc::fence_proxy_async();
    __syncthreads();
  };
  const long tiles = (n + 127) / 128;
  uint32_t acc_w = 0;
  for (long tile = blockIdx.x; tile < tiles; tile += gridDim.x) {
    const long s = tile * 128 + t;
    const bool valid = s < n;
    float x = 0.f, y = 0.f, z = 0.f, target = 0.f;
    {
      float feat[IN];
#pragma unroll
      for (int k = 0; k < IN; ++k) feat[k] = 0.0f;
      if (valid) {
        train_point(xyz_in, seed, first, s, x, y, z, strat);
        target = tgt_in ? tgt_in[s] : field_trilinear(field, dims, x, y, z);
        encode_point<IN / 2>(q, x, y, z, feat);
      }
#pragma unroll
      for (int k = 0; k < IN; k += 8)
        st8(sm.hf, t, H + k, NG, pack2<FMT>(feat[k], feat[k + 1]), pack2<FMT>(feat[k + 2], feat[k + 3]),
            pack2<FMT>(feat[k + 4], feat[k + 5]), pack2<FMT>(feat[k + 6], feat[k + 7]));
    }
    sync_for_mma();
    if (t == 0) {  // h1 = feat W1^T
      tc::fence_after();
#pragma unroll
      for (int kk = 0; kk < IN / 16; ++kk)
        tc::mma<FMT>(dh, tc::sdesc(a_hf + (H / 8) * 128 + kk * 256, 128, NG * 128),
                   tc::sdesc(a_w1 + kk * 256, 128, (IN / 8) * 128), id_h, kk > 0);
      tc::commit(&sm.bar);
    }
    wait_mma();
    uint64_t m1 = 0;  // h1 > 0
#pragma unroll
    for (int c0 = 0; c0 < H; c0 += 16) {
      float v[16];
      tc::ld16(dh + lane + c0, v);
      tc::wait_ld();
#pragma unroll
      for (int i = 0; i < 16; ++i) m1 |= (uint64_t)(v[i] > 0.0f) << (c0 + i);
#pragma unroll
      for (int h = 0; h < 16; h += 8)
        st8(sm.hf, t, c0 + h, NG, pack2_relu<FMT>(v[h], v[h + 1]), pack2_relu<FMT>(v[h + 2], v[h + 3]),
            pack2_relu<FMT>(v[h + 4], v[h + 5]), pack2_relu<FMT>(v[h + 6], v[h + 7]));
    }
    sync_for_mma();
    if (t == 0) {  // h2 = h1 W2^T
      tc::fence_after();
#pragma unroll
      for (int kk = 0; kk < H / 16; ++kk)
        tc::mma<FMT>(dh, tc::sdesc(a_hf + kk * 256, 128, NG * 128), tc::sdesc(a_w2 + kk * 256, 128, (H / 8) * 128),
                   id_h, kk > 0);
      tc::commit(&sm.bar);
    }
    wait_mma();
    {
      // output layer, loss, dL/dy = 2 r, dW3, dh2 = dy W3 on h2 > 0
      float h2[H];
#pragma unroll
      for (int c0 = 0; c0 < H; c0 += 16) {
        tc::ld16(dh + lane + c0, h2 + c0);
        tc::wait_ld();
      }
      float yv = 0.0f;
#pragma unroll
      for (int o = 0; o < H; ++o) yv = fmaf(sm.w3[o], fmaxf(h2[o], 0.0f), yv);
      const float r = valid ? yv - target : 0.0f;
      r2 += r * r;
      const float dy = 2.0f * r, dys = dy * kScale;
#pragma unroll
      for (int o = 0; o < H; ++o) {
        g3[o] = fmaf(dy, fmaxf(h2[o], 0.0f), g3[o]);
        h2[o] = h2[o] > 0.0f ? dys * sm.w3[o] : 0.0f;
      }
#pragma unroll
      for (int c0 = 0; c0 < H; c0 += 8)
        st8(sm.dd, t, c0, 16, pack2<FMT>(h2[c0], h2[c0 + 1]), pack2<FMT>(h2[c0 + 2], h2[c0 + 3]),
            pack2<FMT>(h2[c0 + 4], h2[c0 + 5]), pack2<FMT>(h2[c0 + 6], h2[c0 + 7]));
    }
    sync_for_mma();
    if (t == 0) {  // dh1 (before the mask) = dh2 W2
      tc::fence_after();
#pragma unroll
      for (int kk = 0; kk < H / 16; ++kk)
        tc::mma<FMT>(dh, tc::sdesc(a_dd + kk * 256, 128, 16 * 128),
                   tc::sdesc(a_w2 + kk * 2 * (H / 8) * 128, (H / 8) * 128, 128), id_hT, kk > 0);
      tc::commit(&sm.bar);
    }
    wait_mma();
#pragma unroll
    for (int c0 = 0; c0 < H; c0 += 16) {
      float v[16];
      tc::ld16(dh + lane + c0, v);
      tc::wait_ld();
#pragma unroll
      for (int i = 0; i < 16; ++i) v[i] = ((m1 >> (c0 + i)) & 1ull) ? v[i] : 0.0f;
#pragma unroll
      for (int h = 0; h < 16; h += 8)
        st8(sm.dd, t, 64 + c0 + h, 16, pack2<FMT>(v[h], v[h + 1]), pack2<FMT>(v[h + 2], v[h + 3]),
            pack2<FMT>(v[h + 4], v[h + 5]), pack2<FMT>(v[h + 6], v[h + 7]));
    }
    sync_for_mma();
    if (t == 0) {
      tc::fence_after();
      // dfeat = dh1 W1
#pragma unroll
      for (int kk = 0; kk < H / 16; ++kk)
        tc::mma<FMT>(dh, tc::sdesc(a_dd + 8 * 128 + kk * 256, 128, 16 * 128),
                   tc::sdesc(a_w1 + kk * 2 * (IN / 8) * 128, (IN / 8) * 128, 128), id_fT, kk > 0);
      // [dW2; dW1] += [dh2; dh1]^T [h1, feat] over the tile's samples
#pragma unroll
      for (int kk = 0; kk < 8; ++kk) {
        tc::mma<FMT>(dw, tc::sdesc(a_dd + kk * 2 * 2048, 2048, 128), tc::sdesc(a_hf + kk * 2 * NG * 128, NG * 128, 128),
                   id_w, acc_w);
        acc_w = 1u;
      }
      tc::commit(&sm.bar);
    }
    acc_w = 1u;
    wait_mma();
    // tcgen05.ld is warp-collective: every lane loads, valid or not
    float df[IN];
#pragma unroll
    for (int c0 = 0; c0 < IN; c0 += 16) {
      tc::ld16(dh + lane + c0, df + c0);
      tc::wait_ld();
    }
    if (valid) {
#pragma unroll
      for (int k = 0; k < IN; ++k) df[k] *= inv_ns;
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
          const float w = ((c & 1) ? wx : 1.0f - wx) * ((c & 2) ? wy : 1.0f - wy) * ((c & 4) ? wz : 1.0f - wz);
          const uint32_t idx = (uint32_t)l * T + vertex_index(dense, n1, T, ix + (c & 1), iy + ((c >> 1) & 1),
                                                              iz + ((c >> 2) & 1));
          atomicAdd(reinterpret_cast<float2*>(g_table) + idx, make_float2(w * df[2 * l], w * df[2 * l + 1]));
        }
      }
    }
    tc::fence_before();
  }
  // the CTA's weight gradients: row t of the accumulator (dW2 rows 0 .. H-1,
  // dW1 rows 64 .. 64+H-1), dW3 summed in shared memory
#pragma unroll
  for (int o = 0; o < H; ++o) atomicAdd(&sm.g3[o], g3[o]);
  tc::fence_before();
  __syncthreads();
  tc::fence_after();
  {
#pragma unroll 1
    for (int c0 = 0; c0 < H + IN; c0 += 16) {
      float v[16];
      tc::ld16(dw + lane + c0, v);
      tc::wait_ld();
      if (!acc_w)  // no tile (not reached: the grid is at most the tile count)
#pragma unroll
        for (int i = 0; i < 16; ++i) v[i] = 0.0f;
#pragma unroll
      for (int i = 0; i < 16; ++i) {
        const int c = c0 + i;
        if (t < H && c < H) p2[(size_t)blockIdx.x * H * H + t * H + c] = v[i] * inv_ns;
        if (t >= 64 && t < 64 + H && c >= H) p1[(size_t)blockIdx.x * H * IN + (t - 64) * IN + (c - H)] = v[i] * inv_ns;
      }
    }
  }
  for (int e = t; e < H; e += 128) p3[(size_t)blockIdx.x * H + e] = sm.g3[e] * inv_n;
  if (loss) {
    for (int o = 16; o > 0; o >>= 1) r2 += __shfl_xor_sync(0xffffffffu, r2, o);
    if ((t & 31) == 0 && r2 != 0.0f) atomicAdd(loss, r2 * inv_n);
  }
  if (!ok && status && t == 0) atomicOr(status, kTrainTimeout);
  tc::fence_before();
  __syncthreads();
  tc::fence_after();
  if (t < 32) tc::tmem_dealloc(sm.tmem, kTcTrainCols);
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

// log2 of the stratified sampling grid's edge for a batch of n (the
// largest g with 8^g <= n), or -1 when the trainer samples uniformly.
int strat_of(const cinr_trainer_s* t, long n) {
  if (!t->strat) return -1;
  int g = 0;
  while (g < 10 && (1l << (3 * (g + 1))) <= n) ++g;
  return g;
}

// Fused tensor-core step: one persistent launch (at most 2 CTAs per SM:
// 256 TMEM columns each; at most n_part CTAs, the partial buffers' rows),
// then the reductions of the CTAs' weight-gradient partials.
template <int IN, int H, int FMT>
int grads_tc(cinr_trainer_s* t, const float* xyz, const float* tgt, long n, const float* field, int3 dims,
             uint64_t first, float* g_table, float* g_w, cudaStream_t s) {
  const InrDev& q = t->inr->dev;
  auto k = train_tc_kernel<IN, H, FMT>;
  // shared memory above a third of the SM's, so that at most 2 CTAs (512
  // TMEM columns) share an SM
  int smem = (int)sizeof(TrainTcSmem<IN, H>) + 1024;
  if (smem < 80 * 1024) smem = 80 * 1024;
  CINR_CK(cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
  const long tiles = (n + 127) / 128;
  long grid = 2l * num_sms();
  if (grid > t->n_part) grid = t->n_part;
  if (grid > tiles) grid = tiles;
  if (grid < 1) grid = 1;
  float* p1 = t->partial;
  float* p2 = p1 + (size_t)grid * H * IN;
  float* p3 = p2 + (size_t)grid * H * H;
  k<<<(unsigned)grid, 128, smem, s>>>(q, n, xyz, tgt, field, dims, t->o.seed, first, g_table, p1, p2, p3, t->loss,
                                      reinterpret_cast<int*>(t->loss + 1), strat_of(t, n));
  reduce_kernel<<<(H * IN + 31) / 32, 256, 0, s>>>(p1, (int)grid, H * IN, g_w);
  reduce_kernel<<<(H * H + 31) / 32, 256, 0, s>>>(p2, (int)grid, H * H, g_w + H * IN);
  reduce_kernel<<<(H + 31) / 32, 256, 0, s>>>(p3, (int)grid, H, g_w + H * IN + H * H);
  CINR_CK(cudaGetLastError());
  return CINR_OK;
}

template <int IN, int H>
int grads(cinr_trainer_s* t, const float* xyz, const float* tgt, long n, const float* field, int3 dims,
          uint64_t first, float* g_table, float* g_w, cudaStream_t s) {
  const InrDev& q = t->inr->dev;
  CINR_CK(cudaMemsetAsync(g_table, 0, sizeof(float) * t->n_table, s));
  if (t->tc == 1) return grads_tc<IN, H, 0>(t, xyz, tgt, n, field, dims, first, g_table, g_w, s);
  if (t->tc == 2) return grads_tc<IN, H, 1>(t, xyz, tgt, n, field, dims, first, g_table, g_w, s);
  const int smem = mlp_floats<IN, H>() * 4;
  auto kf = fwd_kernel<IN, H>;
  auto kb = bwd_kernel<IN, H>;
  CINR_CK(cudaFuncSetAttribute(kf, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
  CINR_CK(cudaFuncSetAttribute(kb, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
  const unsigned grid = (unsigned)((n + kFwdThreads - 1) / kFwdThreads);
  kf<<<grid, kFwdThreads, smem, s>>>(q, n, xyz, tgt, field, dims, t->o.seed, first, t->act, t->loss, strat_of(t, n));
  kb<<<grid, kFwdThreads, smem, s>>>(q, n, xyz, t->o.seed, first, t->act, g_table, strat_of(t, n));
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
  t->tc = 0;
  t->strat = 0;
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

extern "C" int cinr_trainer_set_tensor_cores(cinr_trainer_t t, int mode) {
  if (!t) return set_error(CINR_ERR_ARG, "NULL argument");
  if (mode < 0 || mode > 2) return set_error(CINR_ERR_ARG, "mode must be 0, 1 or 2");
  t->tc = mode;
  return CINR_OK;
}

extern "C" int cinr_trainer_set_stratified(cinr_trainer_t t, int on) {
  if (!t) return set_error(CINR_ERR_ARG, "NULL argument");
  if (on != 0 && on != 1) return set_error(CINR_ERR_ARG, "on must be 0 or 1");
  t->strat = on;
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
  if (h & kTrainTimeout)
    return set_error(CINR_ERR_TIMEOUT, "a bounded tensor-core wait of the fused training kernel gave up");
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
