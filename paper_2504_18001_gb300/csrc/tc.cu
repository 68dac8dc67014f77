// Tensor-core (tcgen05) INR inference: direct inference of point batches
// with an FP16/BF16 MLP on 128-query tiles, and a single-tile GEMM self-test
// of the shared-memory operand layout.
#include "cinr_internal.cuh"
#include "tc_mlp.cuh"

using namespace cinr;

namespace {

// D[128 x 64] = A[128 x K] B[64 x K]^T through one tensor-core accumulation
// (A, B row-major FP32 in global memory, rounded to FP16/BF16).
template <int K>
struct DebugSmem {
  alignas(128) unsigned char a[128 * K * 2];
  alignas(128) unsigned char w1[64 * K * 2];
  uint64_t bar;
  uint32_t tmem;
};

template <int K>
__device__ __forceinline__ void debug_setup(DebugSmem<K>& s) {
  if (threadIdx.x == 0) tc::mbar_init(&s.bar, 1);
  if (threadIdx.x < 32) tc::tmem_alloc(&s.tmem, tc::kTmemCols);
  tc::fence_proxy_async();
  tc::fence_before();
  __syncthreads();
  tc::fence_after();
}

template <int K, bool BF16>
__global__ void __launch_bounds__(128) debug_mma_kernel(const float* __restrict__ A, const float* __restrict__ B,
                                                        float* __restrict__ D, int* err) {
  __shared__ DebugSmem<K> s;
  const int t = threadIdx.x;
  for (int k0 = 0; k0 < K; k0 += 8) tc::store8<BF16>(s.a, t, k0, K, A + t * K + k0);
  if (t < 64)
    for (int k0 = 0; k0 < K; k0 += 8) tc::store8<BF16>(s.w1, t, k0, K, B + t * K + k0);
  debug_setup(s);
  constexpr uint32_t idesc = tc::idesc_f16(128, 64, BF16 ? 1 : 0);
  if (t == 0) {
    tc::fence_after();
    const uint32_t a0 = tc::smem_u32(s.a), b0 = tc::smem_u32(s.w1);
    for (int kk = 0; kk < K / 16; ++kk)
      tc::mma_f16(s.tmem, tc::sdesc(a0 + kk * 256, 128, (K / 8) * 128), tc::sdesc(b0 + kk * 256, 128, (K / 8) * 128),
                  idesc, kk > 0 ? 1u : 0u);
    tc::commit(&s.bar);
  }
  const bool ok = tc::mbar_wait(&s.bar, 0);
  tc::fence_after();
  const uint32_t la = s.tmem + ((uint32_t)((t >> 5) * 32) << 16);
  for (int c0 = 0; c0 < 64; c0 += 16) {
    float v[16];
    tc::ld16(la + c0, v);
    tc::wait_ld();
    for (int i = 0; i < 16; ++i) D[t * 64 + c0 + i] = v[i];
  }
  if (!ok && err) atomicOr(err, kErrTimeout);
  tc::fence_before();
  __syncthreads();
  tc::fence_after();
  if (threadIdx.x < 32) tc::tmem_dealloc(s.tmem, tc::kTmemCols);
}

template <int IN, int H, int FMT>
__global__ void __launch_bounds__(128) infer_tc_kernel(InrDev q, const uint16_t* __restrict__ w16,
                                                       const float* __restrict__ xyz, long n,
                                                       float* __restrict__ out, int* err) {
  extern __shared__ __align__(128) unsigned char smem_raw[];
  tc::TcSmem<IN, H>& s = *reinterpret_cast<tc::TcSmem<IN, H>*>(smem_raw);
  tc::load_tc_weights<IN, H, FMT>(s, w16, q.w);
  tc::tc_setup(s);
  uint32_t phase = 0;
  const long tiles = (n + 127) / 128;
  for (long tile = blockIdx.x; tile < tiles; tile += gridDim.x) {
    const long i = tile * 128 + threadIdx.x;
    const bool valid = i < n;
    float feat[IN];
    if (valid) {
      encode_point<IN / 2>(q, clamp01(__ldg(xyz + 3 * i)), clamp01(__ldg(xyz + 3 * i + 1)),
                           clamp01(__ldg(xyz + 3 * i + 2)), feat);
    }
    const float y = tc::mlp_tile<IN, H, FMT>(s, feat, valid, phase, err);
    if (valid) out[i] = fmaf(q.vscale, y, q.vmin);
  }
  tc::tc_teardown(s);
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

template <int IN, int H, int FMT>
int launch_infer_tc(const cinr_inr_s* inr, const float* xyz, long n, float* out, cudaStream_t s) {
  auto k = infer_tc_kernel<IN, H, FMT>;
  // Each resident CTA holds 64 of the SM's 512 TMEM columns: asking for at
  // least 1/8 of the SM's shared memory keeps at most 8 CTAs resident.
  int smem = (int)sizeof(tc::TcSmem<IN, H>);
  if (smem < tc::kMinSmemPerCta) smem = tc::kMinSmemPerCta;
  CINR_CK(cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
  int per_sm = 0;
  // the largest shared-memory carveout: the occupancy query (and the
  // launch) then see every CTA that fits, not the default split
  CINR_CK(cudaFuncSetAttribute(k, cudaFuncAttributePreferredSharedMemoryCarveout,
                               (int)cudaSharedmemCarveoutMaxShared));
  CINR_CK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k, 128, smem));
  if (per_sm < 1) return set_error(CINR_ERR_CUDA, "tensor-core inference kernel cannot be resident");
  const int fit = tc::resident_ctas(k, smem);
  if (fit > per_sm) per_sm = fit;
  // each resident CTA holds 64 of the SM's 512 TMEM columns
  if (per_sm > 8) per_sm = 8;
  long tiles = (n + 127) / 128;
  long grid = (long)per_sm * num_sms();
  if (grid > tiles) grid = tiles;
  k<<<(unsigned)grid, 128, smem, s>>>(inr->dev, inr->w16, xyz, n, out, reinterpret_cast<int*>(inr->scratch + 16));
  CINR_CK(cudaGetLastError());
  return CINR_OK;
}

}  // namespace

template <int FMT>
int infer_tc_fmt(const cinr_inr_s* inr, const float* xyz, long n, float* out, cudaStream_t s) {
  switch (shape_of(inr->dev.IN, inr->dev.H)) {
    case Shape::S16x32: return launch_infer_tc<16, 32, FMT>(inr, xyz, n, out, s);
    case Shape::S32x64: return launch_infer_tc<32, 64, FMT>(inr, xyz, n, out, s);
    case Shape::S48x64: return launch_infer_tc<48, 64, FMT>(inr, xyz, n, out, s);
    default: return set_error(CINR_ERR_ARG, "unsupported shape");
  }
}

// Used by cinr_infer for FP16 / BF16 / FP8 MLPs.
int cinr_infer_tc(const cinr_inr_s* inr, const float* xyz, long n, float* out, cudaStream_t s) {
  if (inr->p.mlp_precision == CINR_PREC_BF16) return infer_tc_fmt<1>(inr, xyz, n, out, s);
  if (inr->p.mlp_precision == CINR_PREC_FP8) return infer_tc_fmt<2>(inr, xyz, n, out, s);
  return infer_tc_fmt<0>(inr, xyz, n, out, s);
}

extern "C" int cinr_debug_mma_tile(const float* a_dev, const float* b_dev, int K, int bf16, float* d_dev,
                                   cinr_stream_t stream) {
  if (!a_dev || !b_dev || !d_dev) return set_error(CINR_ERR_ARG, "NULL argument");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  int* err = nullptr;  // the self-test reports a timeout through D (left unwritten)
  switch (K) {
    case 16:
      if (bf16) debug_mma_kernel<16, true><<<1, 128, 0, s>>>(a_dev, b_dev, d_dev, err);
      else debug_mma_kernel<16, false><<<1, 128, 0, s>>>(a_dev, b_dev, d_dev, err);
      break;
    case 32:
      if (bf16) debug_mma_kernel<32, true><<<1, 128, 0, s>>>(a_dev, b_dev, d_dev, err);
      else debug_mma_kernel<32, false><<<1, 128, 0, s>>>(a_dev, b_dev, d_dev, err);
      break;
    case 64:
      if (bf16) debug_mma_kernel<64, true><<<1, 128, 0, s>>>(a_dev, b_dev, d_dev, err);
      else debug_mma_kernel<64, false><<<1, 128, 0, s>>>(a_dev, b_dev, d_dev, err);
      break;
    default: return set_error(CINR_ERR_ARG, "K must be 16, 32 or 64");
  }
  CINR_CK(cudaGetLastError());
  return CINR_OK;
}

// Failure-detection self-test: one warp waits, with `limit` polls, for a
// phase of an mbarrier that nothing arrives at, and records the timeout in
// the status word the MLP kernels use.  No tensor memory is allocated.
__global__ void debug_wait_kernel(int* err, uint32_t limit) {
  __shared__ uint64_t bar;
  if (threadIdx.x == 0) tc::mbar_init(&bar, 1);
  __syncthreads();
  const bool ok = tc::mbar_wait(&bar, 0, limit);
  if (!ok && threadIdx.x == 0) atomicOr(err, kErrTimeout);
}

extern "C" int cinr_debug_wait_timeout(cinr_inr_t inr, unsigned limit, cinr_stream_t stream) {
  if (!inr) return set_error(CINR_ERR_ARG, "inr is NULL");
  if (limit < 1 || limit > (1u << 22)) return set_error(CINR_ERR_ARG, "limit must be in [1, 2^22]");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  debug_wait_kernel<<<1, 32, 0, s>>>(reinterpret_cast<int*>(inr->scratch + 16), limit);
  CINR_CK(cudaGetLastError());
  return CINR_OK;
}

extern "C" int cinr_inr_status(cinr_inr_t inr, cinr_stream_t stream) {
  if (!inr) return set_error(CINR_ERR_ARG, "inr is NULL");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  int flag = 0;
  int* dev = reinterpret_cast<int*>(inr->scratch + 16);
  CINR_CK(cudaMemcpyAsync(&flag, dev, 4, cudaMemcpyDeviceToHost, s));
  CINR_CK(cudaMemsetAsync(dev, 0, 4, s));
  CINR_CK(cudaStreamSynchronize(s));
  if (device_status(flag) == CINR_ERR_DEVICE_CHECK)
    return set_error(CINR_ERR_DEVICE_CHECK, "a device bounds check tripped (INR or cache update kernel)");
  if (flag) return set_error(CINR_ERR_TIMEOUT, "a device-side wait gave up (tensor-core MLP)");
  return CINR_OK;
}
