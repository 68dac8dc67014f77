// Tensor-core MLP for tiles of 128 queries on sm_103a: tcgen05.mma with
// operands in shared memory and the FP32 accumulator in tensor memory
// (TMEM), read back with tcgen05.ld.  The MLP is in -> H (ReLU) -> H (ReLU)
// -> 1 with FP16, BF16 or FP8 (E4M3) operands and FP32 accumulation; the
// last layer (H -> 1) is a per-thread FP32 dot product.
//
// Shared-memory operand layout (no swizzle, K-major): 8-row x 16-byte core
// matrices, stored 128 contiguous bytes each; the core matrix of rows
// r..r+7 and bytes kb..kb+15 of a rows x Kb-byte matrix sits at
// ((r/8) * (Kb/16) + kb/16) * 128 bytes, so the core matrices adjacent
// along K are 128 B apart (leading-dimension byte offset) and the 8-row
// groups are (Kb/16) * 128 B apart (stride-dimension byte offset).  One MMA
// consumes 32 bytes of K (16 FP16/BF16 or 32 FP8 elements); FP8 operands
// are zero-padded to a multiple of 32 elements.
//
// Every wait on an mbarrier is bounded; on a timeout the routine records an
// error word and carries on, so that the kernel always frees its TMEM and
// returns.
#pragma once

#include <cuda_runtime.h>
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_fp8.h>
#include <stdint.h>

#include "cinr_internal.cuh"

namespace cinr {
namespace tc {

constexpr int kM = 128;               // queries per tile (one per thread)
constexpr int kTmemCols = 64;         // accumulator columns per CTA
constexpr uint32_t kWaitLimit = 1u << 22;
// Dynamic shared memory per CTA (bytes) that keeps at most 8 CTAs (8 x 64
// TMEM columns = 512) resident on an SM of 228 KB shared memory.
constexpr int kMinSmemPerCta = 29 * 1024;

// Resident CTAs per SM of a tensor-core kernel of 128 threads with `smem`
// bytes of dynamic shared memory: the SM's shared memory and registers
// decide, at most 8 (8 x 64 TMEM columns).  The runtime's occupancy query
// answers 1 for kernels that allocate tensor memory; a grid of one CTA per
// SM leaves 3/4 of the warp slots empty while the encoder waits on its
// gathers.  A grid sized from this count is safe either way: CTAs beyond
// those resident wait for a free slot, and no CTA waits on another.
template <class K>
inline int resident_ctas(K kernel, int smem) {
  cudaFuncAttributes fa;
  if (cudaFuncGetAttributes(&fa, kernel) != cudaSuccess) return 1;
  int dev = 0, smem_sm = 0, regs_sm = 0, reserved = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&smem_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev);
  cudaDeviceGetAttribute(&regs_sm, cudaDevAttrMaxRegistersPerMultiprocessor, dev);
  cudaDeviceGetAttribute(&reserved, cudaDevAttrReservedSharedMemoryPerBlock, dev);
  int n = 8;
  const int cta_smem = smem + (int)fa.sharedSizeBytes + reserved;
  if (cta_smem > 0 && smem_sm / cta_smem < n) n = smem_sm / cta_smem;
  const int cta_regs = ((fa.numRegs + 7) / 8) * 8 * 128;  // 256-register warp granules
  if (cta_regs > 0 && regs_sm / cta_regs < n) n = regs_sm / cta_regs;
  return n < 1 ? 1 : n;
}

// Operand formats: 0 = FP16, 1 = BF16, 2 = FP8 E4M3.
template <int FMT>
struct Fmt {
  static constexpr int bytes = FMT == 2 ? 1 : 2;
  static constexpr uint32_t code = FMT == 1 ? 1u : 0u;  // instruction-descriptor A/B format
};

// K of an operand in bytes, padded to the 32-byte MMA step.
template <int FMT>
__host__ __device__ constexpr int kbytes(int K) {
  return ((K * Fmt<FMT>::bytes + 31) / 32) * 32;
}

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

// Bounded wait for the phase with the given parity; false on timeout.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity, uint32_t limit = kWaitLimit) {
  const uint32_t a = smem_u32(bar);
  for (uint32_t i = 0; i < limit; ++i) {
    uint32_t done;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(done)
        : "r"(a), "r"(parity)
        : "memory");
    if (done) return true;
  }
  return false;
}

// Warp-wide (all 32 lanes of one warp).
__device__ __forceinline__ void tmem_alloc(uint32_t* dst, uint32_t ncols) {
  asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(dst)),
               "r"(ncols)
               : "memory");
  asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}

__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols) {
  asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols) : "memory");
}

__device__ __forceinline__ void fence_before() {
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void fence_after() {
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}
// Makes this thread's generic-proxy shared-memory writes visible to the
// tensor core (async proxy).
__device__ __forceinline__ void fence_proxy_async() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

// Shared-memory matrix descriptor: start address, leading (K) and stride
// (M/N) byte offsets, descriptor version 1, no swizzle.
__device__ __forceinline__ uint64_t sdesc(uint32_t addr, uint32_t lbo, uint32_t sbo) {
  uint64_t d = 0;
  d |= (uint64_t)((addr & 0x3FFFFu) >> 4);
  d |= (uint64_t)((lbo >> 4) & 0x3FFFu) << 16;
  d |= (uint64_t)((sbo >> 4) & 0x3FFFu) << 32;
  d |= (uint64_t)1u << 46;
  return d;
}

// Instruction descriptor: D F32, A and B of one format, K-major, N and M.
__host__ __device__ constexpr uint32_t idesc_f16(int M, int N, int fmt) {
  return (1u << 4) | ((uint32_t)fmt << 7) | ((uint32_t)fmt << 10) | ((uint32_t)(N >> 3) << 17) |
         ((uint32_t)(M >> 4) << 24);
}

template <int FMT>
__device__ __forceinline__ void mma(uint32_t dtmem, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                    uint32_t accumulate) {
  if (FMT == 2) {
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f8f6f4 [%0], %1, %2, %3, p;\n\t}" ::"r"(dtmem),
        "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
        : "memory");
  } else {
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(dtmem),
        "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
        : "memory");
  }
}

__device__ __forceinline__ void mma_f16(uint32_t dtmem, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                        uint32_t accumulate) {
  mma<0>(dtmem, adesc, bdesc, idesc, accumulate);
}

__device__ __forceinline__ void commit(uint64_t* bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                   smem_u32(bar))
               : "memory");
}

// 16 consecutive FP32 columns of this thread's TMEM lane.
__device__ __forceinline__ void ld16(uint32_t taddr, float* v) {
  uint32_t r[16];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, "
      "[%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr)
      : "memory");
#pragma unroll
  for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

__device__ __forceinline__ void wait_ld() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }

// Byte offset of byte kb of row r in a K-major operand of Kb bytes per row.
__device__ __forceinline__ uint32_t core_off_b(int r, int kb, int Kb) {
  return (uint32_t)((((r >> 3) * (Kb >> 4) + (kb >> 4)) << 7) + ((r & 7) << 4) + (kb & 15));
}

// Byte offset of 16-bit element (r, k) of a K-major operand with K columns.
__device__ __forceinline__ uint32_t core_off(int r, int k, int K) { return core_off_b(r, k * 2, K * 2); }

template <bool BF16>
__device__ __forceinline__ uint16_t to16(float x) {
  if (BF16) {
    __nv_bfloat16 b = __float2bfloat16_rn(x);
    return *reinterpret_cast<uint16_t*>(&b);
  }
  __half h = __float2half_rn(x);
  return *reinterpret_cast<uint16_t*>(&h);
}

__device__ __forceinline__ uint32_t to8(float x) {
  return (uint32_t)__nv_cvt_float_to_fp8(x, __NV_SATFINITE, __NV_E4M3);
}

// Row r (8 values at k0..k0+7) of a 16-bit K-major operand, one 16-byte store.
template <bool BF16>
__device__ __forceinline__ void store8(unsigned char* base, int r, int k0, int K, const float* v) {
  uint4 q;
  q.x = (uint32_t)to16<BF16>(v[0]) | ((uint32_t)to16<BF16>(v[1]) << 16);
  q.y = (uint32_t)to16<BF16>(v[2]) | ((uint32_t)to16<BF16>(v[3]) << 16);
  q.z = (uint32_t)to16<BF16>(v[4]) | ((uint32_t)to16<BF16>(v[5]) << 16);
  q.w = (uint32_t)to16<BF16>(v[6]) | ((uint32_t)to16<BF16>(v[7]) << 16);
  *reinterpret_cast<uint4*>(base + core_off(r, k0, K)) = q;
}

// Row r of an operand in format FMT: n values (a multiple of 8), zero-padded
// to the padded K; 16-byte stores.
template <int FMT, int N>
__device__ __forceinline__ void store_row(unsigned char* base, int r, const float* v) {
  constexpr int Kb = kbytes<FMT>(N);
  if (FMT == 2) {
#pragma unroll
    for (int k0 = 0; k0 < Kb; k0 += 16) {
      uint32_t w[4];
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        uint32_t x = 0;
#pragma unroll
        for (int b = 0; b < 4; ++b) {
          const int k = k0 + q * 4 + b;
          x |= (k < N ? to8(v[k]) : 0u) << (8 * b);
        }
        w[q] = x;
      }
      *reinterpret_cast<uint4*>(base + core_off_b(r, k0, Kb)) = make_uint4(w[0], w[1], w[2], w[3]);
    }
  } else {
#pragma unroll
    for (int k0 = 0; k0 < N; k0 += 8) store8<FMT == 1>(base, r, k0, N, v + k0);
  }
}

// Shared memory of one CTA's tensor-core MLP (sized for 16-bit operands,
// which also holds the zero-padded FP8 operands).
template <int IN, int H>
struct TcSmem {
  alignas(128) unsigned char a[kM * IN * 2];   // features
  alignas(128) unsigned char a2[kM * H * 2];   // hidden layer 1
  alignas(128) unsigned char w1[H * IN * 2];   // W1 [H][IN]
  alignas(128) unsigned char w2[H * H * 2];    // W2 [H][H]
  float w3[H];
  uint64_t bar;
  uint32_t tmem;
};

// Stage the weights into the core-matrix layout of format FMT and W3 (FP32)
// into shared memory: 16-bit formats from the half-precision copy w16
// (row-major [out][in]), FP8 converted from the FP32 weights.  All threads.
template <int IN, int H, int FMT>
__device__ __forceinline__ void load_tc_weights(TcSmem<IN, H>& s, const uint16_t* w16, const float* w32) {
  if (FMT == 2) {
    constexpr int K1 = kbytes<2>(IN), K2 = kbytes<2>(H);
    for (int e = threadIdx.x; e < H * K1; e += blockDim.x) {
      const int r = e / K1, k = e % K1;
      s.w1[core_off_b(r, k, K1)] = (unsigned char)(k < IN ? to8(__ldg(w32 + r * IN + k)) : 0u);
    }
    for (int e = threadIdx.x; e < H * K2; e += blockDim.x) {
      const int r = e / K2, k = e % K2;
      s.w2[core_off_b(r, k, K2)] = (unsigned char)(k < H ? to8(__ldg(w32 + H * IN + r * H + k)) : 0u);
    }
  } else {
    for (int e = threadIdx.x; e < H * IN; e += blockDim.x) {
      const int r = e / IN, k = e % IN;
      *reinterpret_cast<uint16_t*>(s.w1 + core_off(r, k, IN)) = __ldg(w16 + e);
    }
    for (int e = threadIdx.x; e < H * H; e += blockDim.x) {
      const int r = e / H, k = e % H;
      *reinterpret_cast<uint16_t*>(s.w2 + core_off(r, k, H)) = __ldg(w16 + H * IN + e);
    }
  }
  for (int e = threadIdx.x; e < H; e += blockDim.x) s.w3[e] = __ldg(w32 + H * IN + H * H + e);
}

// CTA set-up: mbarrier and TMEM allocation (warp 0).  Call after
// load_tc_weights, before the first tile, by all threads.
template <int IN, int H>
__device__ __forceinline__ void tc_setup(TcSmem<IN, H>& s) {
  if (threadIdx.x == 0) mbar_init(&s.bar, 1);
  if (threadIdx.x < 32) tmem_alloc(&s.tmem, kTmemCols);
  fence_proxy_async();
  fence_before();
  __syncthreads();
  fence_after();
}

template <int IN, int H>
__device__ __forceinline__ void tc_teardown(TcSmem<IN, H>& s) {
  fence_before();
  __syncthreads();
  fence_after();
  if (threadIdx.x < 32) tmem_dealloc(s.tmem, kTmemCols);
}

// One 128-query tile.  Thread t supplies row t's features (IN floats; zeros
// when !valid) and gets the raw network output of row t.  All 128 threads
// of the CTA (4 warps) must call it together.  `phase` is the mbarrier
// parity this CTA waits for next (starts at 0); *err is set on a timeout.
template <int IN, int H, int FMT>
__device__ __forceinline__ float mlp_tile(TcSmem<IN, H>& s, const float* feat, bool valid, uint32_t& phase,
                                          int* err) {
  const int t = threadIdx.x;
  const int warp = t >> 5;
  constexpr int K1 = kbytes<FMT>(IN), K2 = kbytes<FMT>(H);
  {
    float z[IN];
#pragma unroll
    for (int i = 0; i < IN; ++i) z[i] = valid ? feat[i] : 0.0f;
    store_row<FMT, IN>(s.a, t, z);
  }
  fence_proxy_async();
  __syncthreads();
  constexpr uint32_t idesc = idesc_f16(kM, H, Fmt<FMT>::code);
  const uint32_t dt = s.tmem;
  if (t == 0) {
    fence_after();
    const uint32_t a0 = smem_u32(s.a), b0 = smem_u32(s.w1);
#pragma unroll
    for (int kk = 0; kk < K1 / 32; ++kk)
      mma<FMT>(dt, sdesc(a0 + kk * 256, 128, (K1 / 16) * 128), sdesc(b0 + kk * 256, 128, (K1 / 16) * 128), idesc,
               kk > 0 ? 1u : 0u);
    commit(&s.bar);
  }
  bool ok = mbar_wait(&s.bar, phase);
  phase ^= 1u;
  fence_after();
  const uint32_t lane_addr = dt + ((uint32_t)(warp * 32) << 16);
  {
    if (FMT == 2) {
      float h[H];
#pragma unroll
      for (int c0 = 0; c0 < H; c0 += 16) {
        ld16(lane_addr + c0, h + c0);
        wait_ld();
      }
#pragma unroll
      for (int i = 0; i < H; ++i) h[i] = fmaxf(h[i], 0.0f);
      store_row<FMT, H>(s.a2, t, h);
    } else {
      // 16-bit operands: ReLU and rounding in one paired conversion (a
      // negative value rounds to a non-positive one, which becomes +0, as
      // rounding the ReLU's +0 does), 16 bytes per store
#pragma unroll
      for (int c0 = 0; c0 < H; c0 += 16) {
        float v[16];
        ld16(lane_addr + c0, v);
        wait_ld();
#pragma unroll
        for (int h8 = 0; h8 < 16; h8 += 8) {
          uint32_t w[4];
#pragma unroll
          for (int p = 0; p < 4; ++p) {
            const float lo = v[h8 + 2 * p], hi = v[h8 + 2 * p + 1];
            if (FMT == 1)
              asm("cvt.rn.relu.bf16x2.f32 %0, %1, %2;" : "=r"(w[p]) : "f"(hi), "f"(lo));
            else
              asm("cvt.rn.relu.f16x2.f32 %0, %1, %2;" : "=r"(w[p]) : "f"(hi), "f"(lo));
          }
          *reinterpret_cast<uint4*>(s.a2 + core_off(t, c0 + h8, H)) = make_uint4(w[0], w[1], w[2], w[3]);
        }
      }
    }
  }
  fence_before();
  fence_proxy_async();
  __syncthreads();
  if (t == 0) {
    fence_after();
    const uint32_t a0 = smem_u32(s.a2), b0 = smem_u32(s.w2);
#pragma unroll
    for (int kk = 0; kk < K2 / 32; ++kk)
      mma<FMT>(dt, sdesc(a0 + kk * 256, 128, (K2 / 16) * 128), sdesc(b0 + kk * 256, 128, (K2 / 16) * 128), idesc,
               kk > 0 ? 1u : 0u);
    commit(&s.bar);
  }
  ok = mbar_wait(&s.bar, phase) && ok;
  phase ^= 1u;
  fence_after();
  float y = 0.0f;
#pragma unroll
  for (int c0 = 0; c0 < H; c0 += 16) {
    float v[16];
    ld16(lane_addr + c0, v);
    wait_ld();
#pragma unroll
    for (int i = 0; i < 16; i += 4) {  // the output weights four at a time, the sum in order
      const float4 w3 = *reinterpret_cast<const float4*>(s.w3 + c0 + i);
      y = fmaf(w3.x, fmaxf(v[i], 0.0f), y);
      y = fmaf(w3.y, fmaxf(v[i + 1], 0.0f), y);
      y = fmaf(w3.z, fmaxf(v[i + 2], 0.0f), y);
      y = fmaf(w3.w, fmaxf(v[i + 3], 0.0f), y);
    }
  }
  fence_before();
  if (!ok && err) atomicOr(err, kErrTimeout);
  return y;
}

}  // namespace tc
}  // namespace cinr
