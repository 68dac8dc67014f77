// Per-frame ray marching (Fig. 1, Alg. 1, Alg. 2, Sec. 5.1).
//
// One persistent kernel renders a frame.  Each warp owns one ray at a time
// and marches it in segments of 32 consecutive samples (lane i = sample
// k0 + i).  Per segment:
//   1. lanes compute their sample (binary32 contract), pick a stochastic LoD
//      (Sec. 5.3) and walk the page tables from that LoD to coarser ones
//      (Sec. 4.3); an Unmapped requested brick raises a ranked request
//      (Sec. 4.3.3); the first mapped brick is sampled trilinearly and its
//      slot stamped (LRU);
//   2. true misses of the CTA's 4 warps are compacted by warp ballot and
//      prefix sums into shared memory (Alg. 2's miss list), inferred by the
//      INR in one batch by all 128 threads and scattered back (InferINR and
//      InsertMisses of Alg. 1);
//   3. the warp composites its 32 samples front to back with a warp scan of
//      transmittances, and tests early termination after every K samples.
// Without a cache every sample is a true miss: the uncached baseline.
// Rays are handed out from an atomic counter in 8x8 pixel tiles.
#include <cmath>
#include <cstring>
#include <mutex>
#include <vector>

#include "cinr_internal.cuh"
#include "tc_mlp.cuh"

using namespace cinr;

struct cinr_renderer_s {
  int W, H;
  cinr_march_opts o;
  uint32_t* counters;            // [0] ray counter, [1] miss-record count
  unsigned long long* stats;     // ST_COUNT counters
  uint32_t* miss_rec;            // 2 * miss_cap
  float4* image;                 // W*H, for cinr_render_frame_host
  uint64_t frame;                // frame counter of uncached rendering
  int device;
  cudaEvent_t ev[3];             // frame kernel start/end, cache update end
  cudaStream_t cap = nullptr;    // capture stream of the per-frame CUDA graph
  cudaStream_t copy = nullptr;   // image read-back of cinr_render_frame_host
  cudaGraphExec_t exec = nullptr;
  cinr_macro_s* macro = nullptr; // attached macro cells (Sec. 5.2)
};

namespace {

constexpr uint32_t kFull = 0xffffffffu;
constexpr int kPtMaxSteps = 4096;  // tracking steps per path segment

struct FrameParams {
  CamDev cam;
  InrDev inr;
  CacheDev cache;
  float4 tf[256];
  float4* out;
  uint32_t n_rays;
  uint32_t tiles_x;
  uint32_t* ray_counter;
  unsigned long long* stats;
  uint32_t frame, Tf, fseed;
  int K;
  float eps;
  uint32_t* miss_rec;
  uint32_t miss_cap;
  uint32_t* miss_count;
  const uint16_t* w16;  // half-precision MLP weights (tensor-core path)
  int* err;             // set when a bounded device-side wait gives up
  MacroDev mac;         // transparent macro cells (skip == nullptr: off)
  // path tracing (Sec. 5.1): direction to the light, its irradiance, the
  // ambient radiance, the majorant and its reciprocal, bounces
  float pt_ls[3], pt_light[3], pt_amb[3];
  float pt_sbar, pt_inv;
  int pt_bounces;
};

// Bytes of the frame kernel's shared memory before the MLP region (TF,
// miss batch, values, bookkeeping); a multiple of 128.
constexpr int kFrameSmemHead = (256 + 128) * 16 + 128 * 4 + 32 * 4;

__device__ __forceinline__ float4 tf_lookup(const float4* s_tf, float v) {
  v = clamp01(v);
  const float x = v * 255.0f;
  int i = (int)x;
  i = i > 255 ? 255 : i;
  const int i1 = i + 1 > 255 ? 255 : i + 1;
  const float fr = x - (float)i;
  const float4 a = s_tf[i], b = s_tf[i1];
  // (r, g) and (b, extinction) as packed pairs: fr * (b - a) + a per channel
  const float2 fr2 = make_float2(fr, fr);
  const float2 lo = f2_fma(fr2, f2_sub(make_float2(b.x, b.y), make_float2(a.x, a.y)), make_float2(a.x, a.y));
  const float2 hi = f2_fma(fr2, f2_sub(make_float2(b.z, b.w), make_float2(a.z, a.w)), make_float2(a.z, a.w));
  return make_float4(lo.x, lo.y, hi.x, hi.y);
}

// tf_lookup for v clamped to [0,1]: x = v 255 <= 255, so floor(x) <= 255
__device__ __forceinline__ float4 tf_lookup_fast(const float4* s_tf, float v) {
  const float x = __saturatef(v) * 255.0f;
  const int i = (int)x;
  const int i1 = min(i + 1, 255);
  const float fr = x - (float)i;
  const float4 a = s_tf[i], b = s_tf[i1];
  const float2 fr2 = make_float2(fr, fr);
  const float2 lo = f2_fma(fr2, f2_sub(make_float2(b.x, b.y), make_float2(a.x, a.y)), make_float2(a.x, a.y));
  const float2 hi = f2_fma(fr2, f2_sub(make_float2(b.z, b.w), make_float2(a.z, a.w)), make_float2(a.z, a.w));
  return make_float4(lo.x, lo.y, hi.x, hi.y);
}

__device__ __forceinline__ float ex2_approx(float x) {
  float y;
  asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}

__device__ __forceinline__ float pool_at(const CacheDev& c, size_t i) {
  if (c.pool_prec == CINR_PREC_FP16) return __half2float(__ldg(reinterpret_cast<const __half*>(c.pool) + i));
  return __ldg(reinterpret_cast<const float*>(c.pool) + i);
}

// Trilinear sample inside a stored brick (slot) at LoD-l coordinates s.
__device__ __forceinline__ float brick_sample(const CacheDev& c, int l, uint32_t slot, const int b[3],
                                              const float s[3]) {
  int li[3];
  float f[3];
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    const float q = fminf(fmaxf(f_sub(s[a], 0.5f), 0.0f), (float)(c.dims[l][a] - 1));
    const int i0 = (int)floorf(q);
    f[a] = f_sub(q, (float)i0);
    li[a] = i0 - (b[a] * c.B - 1);
  }
  const int S = c.S;
  const int o = (li[2] * S + li[1]) * S + li[0];
  if (!in_range((uint32_t)o, (uint32_t)(S * S * S - S * S - S - 1), c.err)) return 0.0f;
  const size_t base = (size_t)slot * (size_t)(S * S * S) + (size_t)o;
  const float v000 = pool_at(c, base), v100 = pool_at(c, base + 1);
  const float v010 = pool_at(c, base + S), v110 = pool_at(c, base + S + 1);
  const float v001 = pool_at(c, base + S * S), v101 = pool_at(c, base + S * S + 1);
  const float v011 = pool_at(c, base + S * S + S), v111 = pool_at(c, base + S * S + S + 1);
  const float x00 = fmaf(f[0], v100 - v000, v000), x10 = fmaf(f[0], v110 - v010, v010);
  const float x01 = fmaf(f[0], v101 - v001, v001), x11 = fmaf(f[0], v111 - v011, v011);
  const float y0 = fmaf(f[1], x10 - x00, x00), y1 = fmaf(f[1], x11 - x01, x01);
  return fmaf(f[2], y1 - y0, y0);
}

// MLPP: 0 = FP32 SIMT MLP, 1 / 2 / 3 = FP16 / BF16 / FP8 tensor cores.
template <int IN, int H, bool CACHED, int MLPP>
__global__ void __launch_bounds__(kFrameThreads, (CACHED || MLPP) ? 6 : 4)
    frame_kernel(const __grid_constant__ FrameParams P) {
  extern __shared__ __align__(1024) float4 smem4[];
  float4* s_tf = smem4;                                   // 256
  float4* s_miss = s_tf + 256;                            // 128
  float* s_val = reinterpret_cast<float*>(s_miss + 128);  // 128
  int* s_i = reinterpret_cast<int*>(s_val + 128);         // 32 ints of bookkeeping
  float* sw = reinterpret_cast<float*>(s_i + 32);         // MLP weights (FP32 path)
  tc::TcSmem<IN, H>& tcs = *reinterpret_cast<tc::TcSmem<IN, H>*>(s_i + 32);  // tensor-core path
  int* s_cnt = s_i;        // [2][4] per-warp miss counts (double buffered)
  int* s_act = s_i + 8;    // [2][4] per-warp active flags
  int* s_pix = s_i + 16;   // [4] pixel of each warp's ray
  int* s_k0 = s_i + 20;    // [4] first sample of each warp's segment
  int* s_mbase = s_i + 24; // [2] miss-record base

  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  for (int i = tid; i < 256; i += kFrameThreads) s_tf[i] = P.tf[i];
  uint32_t phase = 0;
  // With a cache, true misses are rare (none once the coarsest LoD is
  // preloaded): their MLP reads the FP32 weights through L1 and the shared
  // memory stays small, leaving the SM's L1 to the brick voxels.
  const float* wmlp = CACHED ? P.inr.w : sw;
  if (MLPP) {
    tc::load_tc_weights<IN, H, (MLPP > 0 ? MLPP - 1 : 0)>(tcs, P.w16, P.inr.w);
    tc::tc_setup(tcs);
  } else {
    if (!CACHED) load_weights(sw, P.inr.w, mlp_floats<IN, H>());
    __syncthreads();
  }

  const CamDev& cam = P.cam;
  int state = 0;  // 0 needs a ray, 1 marching, 2 no rays left
  uint32_t pixel = 0, rseed = 0;
  float d[3] = {0.f, 0.f, 0.f}, tn = 0.f, tf = 0.f, T = 1.f, Cr = 0.f, Cg = 0.f, Cb = 0.f;
  int k0 = 0;
  Sched sch = {0.f, 0.f};
  uint32_t n_samp = 0, n_hit = 0, n_fb = 0, n_miss = 0, n_req = 0, n_slot = 0, n_skip = 0;
  int parity = 0;

  while (true) {
    while (state == 0) {  // warp-uniform: fetch the next ray
      uint32_t r = 0;
      if (lane == 0) r = atomicAdd(P.ray_counter, 1u);
      r = __shfl_sync(kFull, r, 0);
      if (r >= P.n_rays) {
        state = 2;
        break;
      }
      const uint32_t tile = r >> 6, w = r & 63u;
      const int px = (int)((tile % P.tiles_x) * 8 + (w & 7u));
      const int py = (int)((tile / P.tiles_x) * 8 + (w >> 3));
      if (px >= cam.W || py >= cam.H) continue;
      pixel = (uint32_t)(py * cam.W + px);
      if (!ray_setup(cam, px, py, d, tn, tf)) {
        if (lane == 0) P.out[pixel] = make_float4(0.f, 0.f, 0.f, 0.f);
        continue;
      }
      state = 1;
      k0 = 0;
      T = 1.f;
      Cr = Cg = Cb = 0.f;
      rseed = ray_seed(P.fseed, pixel);
    }
    const bool active = state == 1;

    // ---- 1. sample + cache lookup
    float x[3] = {0.f, 0.f, 0.f}, tm = 0.f, len = 0.f, v = 0.f;
    bool has = false, miss = false;
    if (active) {
      sched_segment(cam, tn, k0, sch);
      has = sample_in(cam, d, tn, tf, k0 + lane, sch, x, tm, len);
      if (has && macro_skips(P.mac, f_mul(x[0], (float)cam.vol[0]), f_mul(x[1], (float)cam.vol[1]),
                             f_mul(x[2], (float)cam.vol[2]))) {
        has = false;  // transparent cell (Sec. 5.2): alpha = 0, nothing to look up
        ++n_skip;
      }
      if (has) {
        ++n_samp;
        if (!CACHED) miss = true;
      }
    }
    if (CACHED) {
      const CacheDev& c = P.cache;
      bool want_req = false, hit = false;
      uint32_t req_key = 0, hit_slot = 0;
      if (has) {
        const int l = sample_lod(cam, c.L, 0, rseed, (uint32_t)(k0 + lane), tm);
        float pv[3];
#pragma unroll
        for (int a = 0; a < 3; ++a) pv[a] = f_mul(x[a], (float)c.vol[a]);
        for (int lev = l; lev < c.L; ++lev) {
          const float sc = 1.0f / (float)(1 << lev);
          float s[3];
          int b[3];
#pragma unroll
          for (int a = 0; a < 3; ++a) {
            s[a] = f_mul(pv[a], sc);
            // s / B: a power-of-two B divides exactly by multiplying with 1/B
            const float q = c.invB > 0.0f ? f_mul(s[a], c.invB) : f_div(s[a], (float)c.B);
            int bi = (int)floorf(q);
            bi = bi < 0 ? 0 : (bi > c.nb[lev][a] - 1 ? c.nb[lev][a] - 1 : bi);
            b[a] = bi;
          }
          const uint32_t key =
              c.off[lev] + (uint32_t)b[0] + (uint32_t)c.nb[lev][0] * ((uint32_t)b[1] + (uint32_t)c.nb[lev][1] * (uint32_t)b[2]);
          const uint32_t e = pt_entry(c, lev, key, b[0], b[1], b[2]);
          if (!(e & kMapped)) {
            if (lev == l) {
              want_req = true;
              req_key = key;
            }
            continue;
          }
          hit_slot = e & ~kMapped;
          v = brick_sample(c, lev, hit_slot, b, s);
          hit = true;
          if (lev == l)
            ++n_hit;
          else
            ++n_fb;
          break;
        }
        if (!hit) {
          miss = true;
          ++n_miss;
        }
      }
      // ranked request (Sec. 4.3.3), aggregated over lanes asking for the
      // same brick: r = max(r, T_f) + count, clamped at T_f + 1000
      const unsigned rq = __ballot_sync(kFull, want_req);
      if (want_req) {
        const unsigned peers = __match_any_sync(rq, req_key);
        if (lane == __ffs(peers) - 1) {
          const uint32_t old = atomicMax(c.rank + req_key, P.Tf);
          if (old < P.Tf) {
            ++n_req;
            push_touched(c, req_key);
          }
          atomicAdd(c.rank + req_key, (uint32_t)__popc(peers));
          atomicMin(c.rank + req_key, P.Tf + 1000u);
        }
      }
      // LRU stamp of the slots that served this segment
      // (only lanes that see a stale stamp take part; a stale cached read
      // costs one extra atomic, never a wrong count)
      const bool stale = hit && c.stamp[hit_slot] != P.frame;
      const unsigned hm = __ballot_sync(kFull, stale);
      if (stale) {
        const unsigned peers = __match_any_sync(hm, hit_slot);
        if (lane == __ffs(peers) - 1 && atomicExch(c.stamp + hit_slot, P.frame) != P.frame) ++n_slot;
      }
    }

    // ---- 2. miss compaction (ballot + prefix sums) and batched inference
    const unsigned bal = __ballot_sync(kFull, miss);
    if (lane == 0) {
      s_cnt[parity * 4 + warp] = __popc(bal);
      s_act[parity * 4 + warp] = active ? 1 : 0;
      s_pix[warp] = (int)pixel;
      s_k0[warp] = k0;
    }
    __syncthreads();
    int wbase = 0, total = 0, any = 0;
#pragma unroll
    for (int w = 0; w < 4; ++w) {
      const int cnt = s_cnt[parity * 4 + w];
      wbase += w < warp ? cnt : 0;
      total += cnt;
      any |= s_act[parity * 4 + w];
    }
    if (!any) break;  // block-uniform: no warp has a ray left
    if (total > 0) {
      if (miss) {
        const int pos = wbase + __popc(bal & ((1u << lane) - 1u));
        s_miss[pos] = make_float4(x[0], x[1], x[2], __int_as_float(warp * 32 + lane));
      }
      if (tid == 0 && P.miss_rec) s_mbase[parity] = (int)atomicAdd(P.miss_count, (uint32_t)total);
      __syncthreads();
      const bool mine = tid < total;
      float r = 0.f;
      const float4 m = mine ? s_miss[tid] : make_float4(0.f, 0.f, 0.f, 0.f);
      if (MLPP == 0) {
        if (mine) r = inr_raw_fp32<IN, H>(P.inr, wmlp, m.x, m.y, m.z);
      } else {
        float feat[IN];
        if (mine) encode_point<IN / 2>(P.inr, m.x, m.y, m.z, feat);
        r = tc::mlp_tile<IN, H, (MLPP > 0 ? MLPP - 1 : 0)>(tcs, feat, mine, phase, P.err);
      }
      if (mine) {
        const int slot = __float_as_int(m.w);
        s_val[slot] = fmaf(P.inr.vscale, r, P.inr.vmin);
        if (P.miss_rec) {
          const uint32_t at = (uint32_t)s_mbase[parity] + (uint32_t)tid;
          if (at < P.miss_cap) {
            P.miss_rec[2 * at] = (uint32_t)s_pix[slot >> 5];
            P.miss_rec[2 * at + 1] = (uint32_t)(s_k0[slot >> 5] + (slot & 31));
          }
        }
      }
      __syncthreads();
      if (miss) v = s_val[warp * 32 + lane];
    }
    parity ^= 1;

    // ---- 3. transfer function + front-to-back compositing (warp scan)
    if (active) {
      float alpha = 0.f;
      float4 e = make_float4(0.f, 0.f, 0.f, 0.f);
      if (has) {
        e = tf_lookup(s_tf, v);
        alpha = 1.0f - expf(-e.w * len);
      }
      float p = 1.0f - alpha;  // inclusive prefix product of transmittances
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const float q = __shfl_up_sync(kFull, p, o);
        if (lane >= o) p *= q;
      }
      float excl = __shfl_up_sync(kFull, p, 1);
      if (lane == 0) excl = 1.0f;
      const float wgt = excl * alpha;
      float cr = wgt * e.x, cg = wgt * e.y, cb = wgt * e.z;
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        cr += __shfl_xor_sync(kFull, cr, o);
        cg += __shfl_xor_sync(kFull, cg, o);
        cb += __shfl_xor_sync(kFull, cb, o);
      }
      const float segT = __shfl_sync(kFull, p, 31);
      Cr = fmaf(T, cr, Cr);
      Cg = fmaf(T, cg, Cg);
      Cb = fmaf(T, cb, Cb);
      T *= segT;
      const bool more = next_segment_exists(cam, tn, tf, k0, sch);
      k0 += 32;
      const bool term = (k0 % P.K == 0) && T < P.eps;
      if (!more || term) {
        if (lane == 0) P.out[pixel] = make_float4(Cr, Cg, Cb, 1.0f - T);
        state = 0;
      }
    }
  }

  if (MLPP) tc::tc_teardown(tcs);

  // ---- per-CTA statistics
  unsigned long long a[7] = {n_samp, n_hit, n_fb, n_miss, n_req, n_slot, n_skip};
#pragma unroll
  for (int j = 0; j < 7; ++j)
    for (int o = 16; o > 0; o >>= 1) a[j] += __shfl_xor_sync(kFull, a[j], o);
  if (lane == 0) {
    if (a[0]) atomicAdd(P.stats + ST_SAMPLES, a[0]);
    if (a[1]) atomicAdd(P.stats + ST_HITS, a[1]);
    if (a[2]) atomicAdd(P.stats + ST_FALLBACK, a[2]);
    const unsigned long long misses = CACHED ? a[3] : a[0];
    if (misses) {
      atomicAdd(P.stats + ST_MISSES, misses);
      atomicAdd(P.stats + ST_DIRECT, misses);
    }
    if (a[4]) atomicAdd(P.stats + ST_REQ, a[4]);
    if (a[5]) atomicAdd(P.stats + ST_SLOTS, a[5]);
    if (a[6]) atomicAdd(P.stats + ST_SKIPPED, a[6]);
  }
}

// Cached frames, thread per ray.  A warp takes a tile of 32 neighbouring rays
// (an 8 x 4 pixel block, so the lanes' samples at equal index lie in the
// same bricks) and each lane marches its ray sample by sample: stochastic
// LoD, page-table walk with fallback, ranked requests and LRU stamps
// aggregated over the lanes that name the same brick or slot, trilinear
// sampling, sequential front-to-back compositing and termination after every
// K samples.  A true miss (rare: none once the coarsest LoD is preloaded) is
// inferred in place by its lane with the FP32 weights (read through L1) and
// recorded in the miss list with one atomic per warp.  Warps meet only at
// the end, where the CTA adds its shared counts of rare events (new
// requests, first stamps) to the frame statistics.  The discrete state and
// the sample set are those of the segment-wise formulation.
int num_sms();

// A true miss of the thread-per-ray kernel: the INR at x with FP32 weights
// read through L1.  Kept out of line so that its registers (and spills)
// stay off the marching loop.
template <int IN, int H>
__device__ __noinline__ float infer_miss(const InrDev& q, float x, float y, float z) {
  return fmaf(q.vscale, inr_raw_fp32<IN, H>(q, q.w, x, y, z), q.vmin);
}

// Per-LoD constants of the cache, staged in shared memory (lanes of a warp
// sit at different LoDs, so indexing them in the parameter space would
// serialise the accesses).
struct LevelGeo {
  int nb0, nb1, nb2;
  uint32_t off;
  float dmax0, dmax1, dmax2;  // dims - 1
  float scale;                // 2^-level, exact
  float scale_b;              // 2^-level / B (B a power of two), exact
};

template <bool F16POOL, class I>
__device__ __forceinline__ float pool_ld(const void* pool, I i) {
  if (F16POOL) return __half2float(__ldg(reinterpret_cast<const __half*>(pool) + i));
  return __ldg(reinterpret_cast<const float*>(pool) + i);
}

// MISS: true misses possible (a cache without the coarsest-LoD preload).
// With the preload every fallback walk ends at a mapped brick, and the
// instantiation without the (out-of-line) inference call keeps the marching
// loop free of the register spills that the call's convention forces.
//
// BB: the brick size when it is a compile-time constant (8 or 16; 0 = read
// from the cache): the voxel offsets inside a brick then become immediates
// and the brick index a multiplication by the exact power-of-two 1/B.
template <int IN, int H, bool F16POOL, bool MISS, int BB>
__global__ void __launch_bounds__(kFrameThreads, 8) march_cached_kernel(const __grid_constant__ FrameParams P) {
  __shared__ float4 s_tf[256];
  __shared__ LevelGeo s_geo[kMaxLod];
  // rare events (new requests, first stamps) count in shared memory
  __shared__ uint32_t s_rare[2];
  const CacheDev& c = P.cache;
  if (threadIdx.x < 2) s_rare[threadIdx.x] = 0u;
  for (int i = threadIdx.x; i < 256; i += kFrameThreads) s_tf[i] = P.tf[i];
  if (threadIdx.x < c.L) {
    const int l = threadIdx.x;
    LevelGeo g;
    g.nb0 = c.nb[l][0];
    g.nb1 = c.nb[l][1];
    g.nb2 = c.nb[l][2];
    g.off = c.off[l];
    g.dmax0 = (float)(c.dims[l][0] - 1);
    g.dmax1 = (float)(c.dims[l][1] - 1);
    g.dmax2 = (float)(c.dims[l][2] - 1);
    g.scale = __int_as_float((127 - l) << 23);
    s_geo[l] = g;
  }
  __syncthreads();
  const int lane = threadIdx.x & 31;
  const CamDev& cam = P.cam;
  const float volf[3] = {(float)c.vol[0], (float)c.vol[1], (float)c.vol[2]};
  static_assert(BB == 0 || (BB & (BB - 1)) == 0, "compile-time brick sizes are powers of two");
  const int L = c.L, B = BB ? BB : c.B, S = BB ? BB + 2 : c.S;
  const float invB = BB ? 1.0f / (float)BB : c.invB, fB = (float)B;
  const size_t S3 = (size_t)S * S * S;
  const void* pool = c.pool;
  uint32_t n_samp = 0, n_fb = 0, n_miss = 0, n_skip = 0;  // hits = samples - fallbacks - misses
  // the slot this lane last saw stamped with this frame (stamps change only
  // between frames): runs of samples in one brick check the stamp once
  uint32_t stamped = 0xFFFFFFFFu;
  const uint32_t n_tiles = P.n_rays >> 5;
  while (true) {
    uint32_t tile = 0;
    if (lane == 0) tile = atomicAdd(P.ray_counter, 1u);
    tile = __shfl_sync(kFull, tile, 0);
    if (tile >= n_tiles) break;
    const uint32_t r = tile * 32u + (uint32_t)lane;  // ray index in 8x8 tiles
    const uint32_t t64 = r >> 6, w = r & 63u;
    const int px = (int)((t64 % P.tiles_x) * 8 + (w & 7u));
    const int py = (int)((t64 / P.tiles_x) * 8 + (w >> 3));
    const bool inside = px < cam.W && py < cam.H;
    const uint32_t pixel = inside ? (uint32_t)(py * cam.W + px) : 0u;
    float d[3], tn = 0.f, tf = 0.f;
    bool active = inside && ray_setup(cam, px, py, d, tn, tf);
    if (inside && !active) P.out[pixel] = make_float4(0.f, 0.f, 0.f, 0.f);
    const uint32_t rseed = ray_seed(P.fseed, pixel);
    float T = 1.f, Cr = 0.f, Cg = 0.f, Cb = 0.f;
    int k = 0, seg = P.K;  // seg: samples left in the current K-segment
    Sched sch = {0.f, 0.f};
    while (__any_sync(kFull, active)) {
      float x[3], tm = 0.f, len = 0.f, v = 0.f;
      bool has = false;
      if (active) {
        if ((k & 31) == 0) sched_segment(cam, tn, k, sch);
        has = sample_in(cam, d, tn, tf, k, sch, x, tm, len);
        if (!has) {
          P.out[pixel] = make_float4(Cr, Cg, Cb, 1.0f - T);
          active = false;
        }
      }
      bool want_req = false, hit = false, miss = false, take = false;
      uint32_t req_key = 0, hit_slot = 0;
      float pv0 = 0.f, pv1 = 0.f, pv2 = 0.f;
      if (has) {
        pv0 = f_mul(x[0], volf[0]);
        pv1 = f_mul(x[1], volf[1]);
        pv2 = f_mul(x[2], volf[2]);
        // transparent macro cell (Sec. 5.2): alpha = 0, nothing to look up
        take = !macro_skips(P.mac, pv0, pv1, pv2);
        if (!take) ++n_skip;
      }
      if (take) {
        ++n_samp;
        const int l = sample_lod(cam, L, 0, rseed, (uint32_t)k, tm);
        for (int lev = l; lev < L; ++lev) {
          const LevelGeo g = s_geo[lev];
          const float s0 = f_mul(pv0, g.scale), s1 = f_mul(pv1, g.scale), s2 = f_mul(pv2, g.scale);
          int b0 = (int)floorf(BB || invB > 0.0f ? f_mul(s0, invB) : f_div(s0, fB));
          int b1 = (int)floorf(BB || invB > 0.0f ? f_mul(s1, invB) : f_div(s1, fB));
          int b2 = (int)floorf(BB || invB > 0.0f ? f_mul(s2, invB) : f_div(s2, fB));
          b0 = min(max(b0, 0), g.nb0 - 1);
          b1 = min(max(b1, 0), g.nb1 - 1);
          b2 = min(max(b2, 0), g.nb2 - 1);
          const uint32_t key = g.off + (uint32_t)b0 + (uint32_t)g.nb0 * ((uint32_t)b1 + (uint32_t)g.nb1 * (uint32_t)b2);
          const uint32_t e = pt_entry(c, lev, key, b0, b1, b2);
          if (!(e & kMapped)) {
            if (lev == l) {
              want_req = true;
              req_key = key;
            }
            continue;
          }
          hit_slot = e & ~kMapped;
          // trilinear inside the stored brick (apron included)
          const float q0 = fminf(fmaxf(f_sub(s0, 0.5f), 0.0f), g.dmax0);
          const float q1 = fminf(fmaxf(f_sub(s1, 0.5f), 0.0f), g.dmax1);
          const float q2 = fminf(fmaxf(f_sub(s2, 0.5f), 0.0f), g.dmax2);
          const int i0 = (int)floorf(q0), i1 = (int)floorf(q1), i2 = (int)floorf(q2);
          const float f0 = f_sub(q0, (float)i0), f1 = f_sub(q1, (float)i1), f2 = f_sub(q2, (float)i2);
          const int l0 = i0 - (b0 * B - 1), l1 = i1 - (b1 * B - 1), l2 = i2 - (b2 * B - 1);
          // the slot's base pointer once, then 32-bit offsets inside the brick
          const void* bp = static_cast<const char*>(pool) + (size_t)hit_slot * S3 * (F16POOL ? 2 : 4);
          const int o = (l2 * S + l1) * S + l0, SS = S * S;
          if (!in_range((uint32_t)o, (uint32_t)(S3 - SS - S - 1), c.err)) continue;
          const float v000 = pool_ld<F16POOL>(bp, o), v100 = pool_ld<F16POOL>(bp, o + 1);
          const float v010 = pool_ld<F16POOL>(bp, o + S), v110 = pool_ld<F16POOL>(bp, o + S + 1);
          const float v001 = pool_ld<F16POOL>(bp, o + SS), v101 = pool_ld<F16POOL>(bp, o + SS + 1);
          const float v011 = pool_ld<F16POOL>(bp, o + SS + S), v111 = pool_ld<F16POOL>(bp, o + SS + S + 1);
          // x-lerps and the y-lerp on (z = 0, z = 1) pairs, then the z-lerp
          const float2 a0 = make_float2(v000, v001), a1 = make_float2(v100, v101);
          const float2 c0 = make_float2(v010, v011), c1 = make_float2(v110, v111);
          const float2 ff0 = make_float2(f0, f0);
          const float2 X0 = f2_fma(ff0, f2_sub(a1, a0), a0);                 // (x00, x01)
          const float2 X1 = f2_fma(ff0, f2_sub(c1, c0), c0);                 // (x10, x11)
          const float2 Y = f2_fma(make_float2(f1, f1), f2_sub(X1, X0), X0);  // (y0, y1)
          v = fmaf(f2, Y.y - Y.x, Y.x);
          hit = true;
          if (lev != l) ++n_fb;
          break;
        }
        if (!hit) {
          miss = true;
          ++n_miss;
        }
      }
      const unsigned rq = __ballot_sync(kFull, want_req);
      if (want_req) {
        const unsigned peers = __match_any_sync(rq, req_key);
        if (lane == __ffs(peers) - 1) {
          const uint32_t old = atomicMax(c.rank + req_key, P.Tf);
          if (old < P.Tf) {
            atomicAdd(&s_rare[0], 1u);
            push_touched(c, req_key);
          }
          atomicAdd(c.rank + req_key, (uint32_t)__popc(peers));
          atomicMin(c.rank + req_key, P.Tf + 1000u);
        }
      }
      const bool stale = hit && hit_slot != stamped && c.stamp[hit_slot] != P.frame;
      const unsigned hm = __ballot_sync(kFull, stale);
      if (stale) {
        const unsigned peers = __match_any_sync(hm, hit_slot);
        if (lane == __ffs(peers) - 1 && atomicExch(c.stamp + hit_slot, P.frame) != P.frame)
          atomicAdd(&s_rare[1], 1u);
      }
      if (hit) stamped = hit_slot;
      const unsigned mm = MISS ? __ballot_sync(kFull, miss) : 0u;
      if (MISS && mm) {
        if (miss) v = infer_miss<IN, H>(P.inr, x[0], x[1], x[2]);
        if (P.miss_rec) {
          uint32_t base = 0;
          if (lane == 0) base = atomicAdd(P.miss_count, (uint32_t)__popc(mm));
          base = __shfl_sync(kFull, base, 0);
          if (miss) {
            const uint32_t at = base + (uint32_t)__popc(mm & ((1u << lane) - 1u));
            if (at < P.miss_cap) {
              P.miss_rec[2 * at] = pixel;
              P.miss_rec[2 * at + 1] = (uint32_t)k;
            }
          }
        }
      }
      if (has) {
        if (take) {
          const float4 e4 = tf_lookup(s_tf, v);
          const float alpha = 1.0f - __expf(-e4.w * len);
          const float wgt = T * alpha;
          Cr = fmaf(wgt, e4.x, Cr);
          Cg = fmaf(wgt, e4.y, Cg);
          Cb = fmaf(wgt, e4.z, Cb);
          T *= 1.0f - alpha;
        } else {
          // transparent cell: the next samples in the same cell are skipped
          // at once, up to the K-segment end (the termination test stays on
          // its boundary) and, with LoD-scaled steps, the 32-sample segment
          int jump = macro_run(P.mac, cam, d, pv0, pv1, pv2, cam.step_mode ? sch.dts : cam.dt);
          jump = min(jump, seg - 1);
          if (cam.step_mode) jump = min(jump, 31 - (k & 31));
          if (jump > 0) {
            k += jump;
            seg -= jump;
            n_skip += (uint32_t)jump;
          }
        }
        ++k;
        if (--seg == 0) {
          seg = P.K;
          if (T < P.eps) {
            P.out[pixel] = make_float4(Cr, Cg, Cb, 1.0f - T);
            active = false;
          }
        }
      }
    }
  }
  unsigned long long a[5] = {n_samp, n_fb, n_miss, n_skip, 0ull};
#pragma unroll
  for (int j = 0; j < 4; ++j)
    for (int o = 16; o > 0; o >>= 1) a[j] += __shfl_xor_sync(kFull, a[j], o);
  a[4] = a[3];                      // skipped
  a[3] = a[2];                      // misses
  a[2] = a[1];                      // fallbacks
  a[1] = a[0] - a[2] - a[3];        // hits
  __syncthreads();
  if (threadIdx.x == 0) {
    if (s_rare[0]) atomicAdd(P.stats + ST_REQ, (unsigned long long)s_rare[0]);
    if (s_rare[1]) atomicAdd(P.stats + ST_SLOTS, (unsigned long long)s_rare[1]);
  }
  if (lane == 0) {
    if (a[0]) atomicAdd(P.stats + ST_SAMPLES, a[0]);
    if (a[1]) atomicAdd(P.stats + ST_HITS, a[1]);
    if (a[2]) atomicAdd(P.stats + ST_FALLBACK, a[2]);
    if (a[3]) {
      atomicAdd(P.stats + ST_MISSES, a[3]);
      atomicAdd(P.stats + ST_DIRECT, a[3]);
    }
    if (a[4]) atomicAdd(P.stats + ST_SKIPPED, a[4]);
  }
}

// The marching kernel specialised on the common configuration: fixed steps
// (step_mode 0; STEP: LoD-scaled 32-sample segments, step_mode 1),
// footprint LoD (lod_mode 0), flat page tables, no macro
// cells, the coarsest LoD preloaded (every fallback walk ends at a mapped
// brick) and the brick size BB a compile-time power of two.  It takes the
// same samples, LoDs, lookups, requests, stamps and values as
// march_cached_kernel, in the same binary32 operations; what it saves is
// bookkeeping and control flow: no per-sample tests of the run-time modes;
// the start of the next sample carried over from this sample's unclipped
// end (the same tn + (k+1) dt, or ts + (j+1) dts in a segment, whose last
// sample's end is the next segment's start); the dither key k * 0x9E3779B9 advanced by
// addition; brick and voxel coordinates of non-negative values truncated
// (the floor of a non-negative binary32); brick indices from one product
// with 2^-l / B (products with powers of two are exact); the sample count
// of a ray taken from its last sample index; and one straight-line pass
// per sample that every lane of the warp runs, with the rare events --
// fallback walks, requests, first stamps of a slot, ray ends -- behind
// warp-uniform votes, so that the warp issues no divergent branches on
// its common path (all lanes of a warp march the same sample index k).
template <bool F16POOL, int BB, bool TEX = false, bool STEP = false>
__global__ void __launch_bounds__(kFrameThreads, 8) march_fast_kernel(const __grid_constant__ FrameParams P) {
  static_assert(BB > 0 && (BB & (BB - 1)) == 0, "brick size must be a power of two");
  __shared__ float4 s_tf[256];
  __shared__ LevelGeo s_geo[kMaxLod];
  __shared__ uint32_t s_rare[2];
  const CacheDev& c = P.cache;
  if (threadIdx.x < 2) s_rare[threadIdx.x] = 0u;
  // the extinction channel pre-multiplied by -log2(e): alpha = 1 - 2^(w len)
  for (int i = threadIdx.x; i < 256; i += kFrameThreads) {
    float4 e = P.tf[i];
    e.w *= -1.4426950408889634f;
    s_tf[i] = e;
  }
  if (threadIdx.x < c.L) {
    const int l = threadIdx.x;
    LevelGeo g;
    g.nb0 = c.nb[l][0];
    g.nb1 = c.nb[l][1];
    g.nb2 = c.nb[l][2];
    g.off = c.off[l];
    g.dmax0 = (float)(c.dims[l][0] - 1);
    g.dmax1 = (float)(c.dims[l][1] - 1);
    g.dmax2 = (float)(c.dims[l][2] - 1);
    g.scale = __int_as_float((127 - l) << 23);
    g.scale_b = __int_as_float((127 - l) << 23) * (1.0f / (float)BB);
    s_geo[l] = g;
  }
  __syncthreads();
  const int lane = threadIdx.x & 31;
  const CamDev& cam = P.cam;
  const float volf0 = (float)c.vol[0], volf1 = (float)c.vol[1], volf2 = (float)c.vol[2];
  constexpr int B = BB, S = BB + 2, SS = S * S;
  constexpr float invB = 1.0f / (float)BB;
  constexpr uint32_t S3 = (uint32_t)(S * S * S);
  const int Lm1 = c.L - 1;
  const void* pool = c.pool;
  const uint32_t* pt = c.pt;
  uint32_t n_samp = 0, n_fb = 0, n_miss = 0;
  uint32_t stamped = 0xFFFFFFFFu;  // the slot this lane last saw stamped this frame
  const uint32_t n_tiles = P.n_rays >> 5;
  while (true) {
    uint32_t tile = 0;
    if (lane == 0) tile = atomicAdd(P.ray_counter, 1u);
    tile = __shfl_sync(kFull, tile, 0);
    if (tile >= n_tiles) break;
    const uint32_t r = tile * 32u + (uint32_t)lane;  // ray index in 8x8 tiles
    const uint32_t t64 = r >> 6, w = r & 63u;
    const int px = (int)((t64 % P.tiles_x) * 8 + (w & 7u));
    const int py = (int)((t64 / P.tiles_x) * 8 + (w >> 3));
    const bool inside = px < cam.W && py < cam.H;
    const uint32_t pixel = inside ? (uint32_t)(py * cam.W + px) : 0u;
    float d[3] = {0.f, 0.f, 0.f}, tn = 0.f, tf = 0.f;
    bool active = inside && ray_setup(cam, px, py, d, tn, tf);
    if (inside && !active) P.out[pixel] = make_float4(0.f, 0.f, 0.f, 0.f);
    const uint32_t rseed = ray_seed(P.fseed, pixel);
    float T = 1.f, Cr = 0.f, Cg = 0.f, Cb = 0.f;
    int k = 0, seg = P.K;
    float a = tn;         // start of sample k: tn + k dt (tn + 0 dt = tn)
    float kf1 = 1.0f;     // k + 1 as binary32 (exact below 2^24)
    // LoD-scaled steps (sched_segment): segment start ts, step dts,
    // j + 1 for the sample's index j in the segment
    float ts = tn, dts = 0.f, jf1 = 1.0f;
    if (STEP) dts = f_mul(cam.dt, (float)(1 << step_level(cam, tn)));
    uint32_t kh = 0u;     // k * 0x9E3779B9
    if (active && !(a < tf)) {  // (tn < tf for a hit: not reached)
      P.out[pixel] = make_float4(0.f, 0.f, 0.f, 0.f);
      active = false;
    }
    // Every lane runs the sample code each step, active or not (an
    // inactive lane's coordinates stay clamped inside the volume, its
    // lookups inside the tables and the pool); what an inactive lane
    // computes is discarded.  The rare events -- fallback walks, requests,
    // first stamps, ray ends -- sit behind warp-uniform tests.
    while (__any_sync(kFull, active)) {
      // sample k: midpoint of [a, min(tn + (k+1) dt, tf)] (sample_at)
      const float an = STEP ? f_add(ts, f_mul(jf1, dts)) : f_add(tn, f_mul(kf1, cam.dt));
      const float bnd = fminf(an, tf);
      const float tm = f_mul(f_add(a, bnd), 0.5f);
      const float len = f_sub(bnd, a);
      const float pv0 = f_mul(f_mul_sat(f_add(f_add(cam.o[0], f_mul(tm, d[0])), cam.h[0]), cam.inv_e[0]), volf0);
      const float pv1 = f_mul(f_mul_sat(f_add(f_add(cam.o[1], f_mul(tm, d[1])), cam.h[1]), cam.inv_e[1]), volf1);
      const float pv2 = f_mul(f_mul_sat(f_add(f_add(cam.o[2], f_mul(tm, d[2])), cam.h[2]), cam.inv_e[2]), volf2);
      // stochastic LoD, footprint mode (sample_lod)
      const float xf = f_mul(tm, cam.lodc);
      int l = 0;
      if (xf >= 1.0f) {
        uint32_t st = rseed ^ kh;
        if (st == 0u) st = 0x6D2B79F5u;
        const uint32_t u24 = xorshift32(st) >> 8;
        const uint32_t bits = __float_as_uint(xf);
        l = (int)(bits >> 23) - 127 + (u24 < 2u * (bits & 0x7FFFFFu) ? 1 : 0);
        l = l > Lm1 ? Lm1 : l;
      }
      // page-table lookup at the requested LoD
      LevelGeo g = s_geo[l];
      int b0 = min((int)f_mul(pv0, g.scale_b), g.nb0 - 1);
      int b1 = min((int)f_mul(pv1, g.scale_b), g.nb1 - 1);
      int b2 = min((int)f_mul(pv2, g.scale_b), g.nb2 - 1);
      const uint32_t key = g.off + (uint32_t)b0 + (uint32_t)g.nb0 * ((uint32_t)b1 + (uint32_t)g.nb1 * (uint32_t)b2);
      uint32_t e = in_range(key, c.n_bricks, c.err) ? __ldg(pt + key) : 0u;
      if ((e & kMapped) && !in_range(e & ~kMapped, c.n_slots, c.err)) e = 0u;
      const bool want_req = active && !(e & kMapped);
      const unsigned rq = __ballot_sync(kFull, want_req);
      if (rq) {
        // requests (Sec. 4.3.3), aggregated over the lanes naming one brick
        if (want_req) {
          const unsigned peers = __match_any_sync(rq, key);
          if (lane == __ffs(peers) - 1) {
            const uint32_t old = atomicMax(c.rank + key, P.Tf);
            if (old < P.Tf) {
              atomicAdd(&s_rare[0], 1u);
              push_touched(c, key);
            }
            atomicAdd(c.rank + key, (uint32_t)__popc(peers));
            atomicMin(c.rank + key, P.Tf + 1000u);
          }
          // fallback to coarser LoDs (Sec. 4.3); the preloaded coarsest
          // LoD ends the walk
          int lev = l;
          while (!(e & kMapped) && lev < Lm1) {
            ++lev;
            g = s_geo[lev];
            b0 = min((int)f_mul(pv0, g.scale_b), g.nb0 - 1);
            b1 = min((int)f_mul(pv1, g.scale_b), g.nb1 - 1);
            b2 = min((int)f_mul(pv2, g.scale_b), g.nb2 - 1);
            const uint32_t fk = g.off + (uint32_t)b0 + (uint32_t)g.nb0 * ((uint32_t)b1 + (uint32_t)g.nb1 * (uint32_t)b2);
            e = in_range(fk, c.n_bricks, c.err) ? __ldg(pt + fk) : 0u;
            if ((e & kMapped) && !in_range(e & ~kMapped, c.n_slots, c.err)) e = 0u;
          }
          if (e & kMapped) ++n_fb; else ++n_miss;  // a miss: not reached while the coarsest LoD stays mapped
        }
      }
      // trilinear inside the stored brick at the level that serves the
      // sample (an unmapped entry of an inactive lane reads slot 0)
      const uint32_t hit_slot = e & ~kMapped;
      const float s0 = f_mul(pv0, g.scale), s1 = f_mul(pv1, g.scale), s2 = f_mul(pv2, g.scale);
      const float q0 = fminf(fmaxf(f_sub(s0, 0.5f), 0.0f), g.dmax0);
      const float q1 = fminf(fmaxf(f_sub(s1, 0.5f), 0.0f), g.dmax1);
      const float q2 = fminf(fmaxf(f_sub(s2, 0.5f), 0.0f), g.dmax2);
      const int i0 = (int)q0, i1 = (int)q1, i2 = (int)q2;
      const float f0 = f_sub(q0, (float)i0), f1 = f_sub(q1, (float)i1), f2 = f_sub(q2, (float)i2);
      float vt;
      if (TEX) {
        // two bilinear fetches by the texture units (slices z and z + 1 of
        // the slot, blocks b and b + 1 of the 2D layout) and the z-lerp; a
        // fetch is clamped to the image, so any coordinate is safe
        const int lx = i0 - b0 * B + 1, ly = i1 - b1 * B + 1, lz = i2 - b2 * B + 1;
        const uint32_t blk = hit_slot * (uint32_t)S + (uint32_t)lz, m = (1u << c.tex_shift) - 1u;
        const float x0 = (float)((int)(blk & m) * S + lx) + f0 + 0.5f;
        const float y0 = (float)((int)(blk >> c.tex_shift) * S + ly) + f1 + 0.5f;
        const float x1 = (float)((int)((blk + 1u) & m) * S + lx) + f0 + 0.5f;
        const float y1 = (float)((int)((blk + 1u) >> c.tex_shift) * S + ly) + f1 + 0.5f;
        const float t0 = tex2D<float>((cudaTextureObject_t)c.tex, x0, y0);
        const float t1 = tex2D<float>((cudaTextureObject_t)c.tex, x1, y1);
        vt = fmaf(f2, t1 - t0, t0);
      } else {
        int o = ((i2 - b2 * B + 1) * S + (i1 - b1 * B + 1)) * S + (i0 - b0 * B + 1);
        if (!in_range((uint32_t)o, S3 - SS - S - 1, c.err)) o = 0;
        const void* bp = static_cast<const char*>(pool) + (size_t)hit_slot * S3 * (F16POOL ? 2u : 4u);
        const float v000 = pool_ld<F16POOL>(bp, o), v100 = pool_ld<F16POOL>(bp, o + 1);
        const float v010 = pool_ld<F16POOL>(bp, o + S), v110 = pool_ld<F16POOL>(bp, o + S + 1);
        const float v001 = pool_ld<F16POOL>(bp, o + SS), v101 = pool_ld<F16POOL>(bp, o + SS + 1);
        const float v011 = pool_ld<F16POOL>(bp, o + SS + S), v111 = pool_ld<F16POOL>(bp, o + SS + S + 1);
        const float2 a0 = make_float2(v000, v001), a1 = make_float2(v100, v101);
        const float2 c0 = make_float2(v010, v011), c1 = make_float2(v110, v111);
        const float2 ff0 = make_float2(f0, f0);
        const float2 X0 = f2_fma(ff0, f2_sub(a1, a0), a0);
        const float2 X1 = f2_fma(ff0, f2_sub(c1, c0), c0);
        const float2 Y = f2_fma(make_float2(f1, f1), f2_sub(X1, X0), X0);
        vt = fmaf(f2, Y.y - Y.x, Y.x);
      }
      const float v = (e & kMapped) ? vt : 0.0f;
      // LRU stamp: once per slot and frame (the first exchange counts it)
      const bool changed = active && (e & kMapped) && hit_slot != stamped;
      if (__any_sync(kFull, changed)) {
        if (changed && c.stamp[hit_slot] != P.frame && atomicExch(c.stamp + hit_slot, P.frame) != P.frame)
          atomicAdd(&s_rare[1], 1u);
      }
      if (changed) stamped = hit_slot;
      // transfer function and front-to-back compositing
      const float4 e4 = tf_lookup_fast(s_tf, v);
      const float alpha = 1.0f - ex2_approx(e4.w * len);
      const float wgt = active ? T * alpha : 0.0f;
      Cr = fmaf(wgt, e4.x, Cr);
      Cg = fmaf(wgt, e4.y, Cg);
      Cb = fmaf(wgt, e4.z, Cb);
      if (active) {
        T *= 1.0f - alpha;
        a = an;
        kf1 = f_add(kf1, 1.0f);
        ++k;
        kh += 0x9E3779B9u;
        if (STEP) {
          if (jf1 == 32.0f) {  // the next 32-sample segment starts at this sample's end
            ts = an;
            dts = f_mul(cam.dt, (float)(1 << step_level(cam, ts)));
            jf1 = 1.0f;
          } else {
            jf1 = f_add(jf1, 1.0f);
          }
        }
      }
      // termination after every K samples (k is the same for the warp's
      // active lanes) and the end of the ray
      bool ended = active && !(a < tf);
      if (--seg == 0) {
        seg = P.K;
        ended = ended || (active && T < P.eps);
      }
      if (__any_sync(kFull, ended)) {
        if (ended) {
          P.out[pixel] = make_float4(Cr, Cg, Cb, 1.0f - T);
          active = false;
        }
      }
    }
    n_samp += (uint32_t)k;
  }
  unsigned long long a3[3] = {n_samp, n_fb, n_miss};
#pragma unroll
  for (int j = 0; j < 3; ++j)
    for (int o = 16; o > 0; o >>= 1) a3[j] += __shfl_xor_sync(kFull, a3[j], o);
  __syncthreads();
  if (threadIdx.x == 0) {
    if (s_rare[0]) atomicAdd(P.stats + ST_REQ, (unsigned long long)s_rare[0]);
    if (s_rare[1]) atomicAdd(P.stats + ST_SLOTS, (unsigned long long)s_rare[1]);
  }
  if (lane == 0) {
    const unsigned long long hits = a3[0] - a3[1] - a3[2];
    if (a3[0]) atomicAdd(P.stats + ST_SAMPLES, a3[0]);
    if (hits) atomicAdd(P.stats + ST_HITS, hits);
    if (a3[1]) atomicAdd(P.stats + ST_FALLBACK, a3[1]);
    if (a3[2]) atomicAdd(P.stats + ST_MISSES, a3[2]);
  }
}

template <bool F16POOL, int BB, bool TEX = false, bool STEP = false>
int launch_march_fast(const FrameParams& P, cudaStream_t s) {
  auto k = march_fast_kernel<F16POOL, BB, TEX, STEP>;
  static int blocks_per_sm = 0;
  if (!blocks_per_sm) {
    CINR_CK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&blocks_per_sm, k, kFrameThreads, 0));
    if (blocks_per_sm < 1) return set_error(CINR_ERR_CUDA, "march kernel cannot be resident");
  }
  k<<<(unsigned)(blocks_per_sm * num_sms()), kFrameThreads, 0, s>>>(P);
  CINR_CK(cudaGetLastError());
  return CINR_OK;
}

template <int IN, int H, bool F16POOL, bool MISS, int BB>
int launch_march_cached(const FrameParams& P, cudaStream_t s) {
  auto k = march_cached_kernel<IN, H, F16POOL, MISS, BB>;
  static int blocks_per_sm = 0;
  if (!blocks_per_sm) {
    CINR_CK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&blocks_per_sm, k, kFrameThreads, 0));
    if (blocks_per_sm < 1) return set_error(CINR_ERR_CUDA, "march kernel cannot be resident");
  }
  k<<<(unsigned)(blocks_per_sm * num_sms()), kFrameThreads, 0, s>>>(P);
  CINR_CK(cudaGetLastError());
  return CINR_OK;
}

// With true misses possible the kernel infers them with the INR's shape;
// without, the shape plays no part and the brick size is specialised.
template <bool F16POOL>
int launch_march_cached_pool(const FrameParams& P, bool miss, cudaStream_t s) {
  const bool common = !miss && P.cam.lod_mode == 0 && !P.cache.pd && !P.mac.skip;
  const bool step = P.cam.step_mode != 0;
  if (P.cache.pool_tex) {  // FP16 bricks in the texture layout: the specialised kernel only
    if (F16POOL && common && !step && P.cache.B == 8) return launch_march_fast<true, 8, true>(P, s);
    if (F16POOL && common && !step && P.cache.B == 16) return launch_march_fast<true, 16, true>(P, s);
    return set_error(CINR_ERR_UNSUPPORTED,
                     "the texture layout serves fixed steps, footprint LoD, flat tables, no macro cells, "
                     "a preloaded coarsest LoD and bricks of 8 or 16 only");
  }
  if (common && !step && P.cache.B == 8) return launch_march_fast<F16POOL, 8>(P, s);
  if (common && !step && P.cache.B == 16) return launch_march_fast<F16POOL, 16>(P, s);
  if (common && step && P.cache.B == 8) return launch_march_fast<F16POOL, 8, false, true>(P, s);
  if (common && step && P.cache.B == 16) return launch_march_fast<F16POOL, 16, false, true>(P, s);
  if (!miss) {
    switch (P.cache.B) {
      case 8: return launch_march_cached<16, 32, F16POOL, false, 8>(P, s);
      case 16: return launch_march_cached<16, 32, F16POOL, false, 16>(P, s);
      default: return launch_march_cached<16, 32, F16POOL, false, 0>(P, s);
    }
  }
  switch (shape_of(P.inr.IN, P.inr.H)) {
    case Shape::S16x32: return launch_march_cached<16, 32, F16POOL, true, 0>(P, s);
    case Shape::S32x64: return launch_march_cached<32, 64, F16POOL, true, 0>(P, s);
    case Shape::S48x64: return launch_march_cached<48, 64, F16POOL, true, 0>(P, s);
    default: return set_error(CINR_ERR_ARG, "unsupported shape");
  }
}

int launch_march_cached_shape(const FrameParams& P, bool miss, cudaStream_t s) {
  const bool f16 = P.cache.pool_prec == CINR_PREC_FP16;
  return f16 ? launch_march_cached_pool<true>(P, miss, s) : launch_march_cached_pool<false>(P, miss, s);
}

// ---------------------------------------------------------------------------
// Path tracing with Woodcock delta tracking (Sec. 5.1), one path per pixel
// and frame, thread per path (a lane takes the next ray when its path
// ends).  Every quantity that positions a lookup is binary32 in a fixed
// order (the series log, the sphere sampler, the box exits and the cell
// walk use +,-,*,/,sqrt only), so the lookups, requests, stamps and misses
// match the oracle bit for bit; the collision decisions compare u times the
// majorant with the sampled extinction.

// j-th uniform of the SplitMix64 generator started at state key (top 24 bits).
__device__ __forceinline__ float pt_uniform(uint64_t key, uint32_t j) {
  uint64_t z = key + 0x9E3779B97F4A7C15ull * (uint64_t)j + 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  z = z ^ (z >> 31);
  return (float)(z >> 40) * (1.0f / 16777216.0f);
}

// -ln(1 - u): y = m 2^e with m in [sqrt(2)/2, sqrt(2)), ln y = e ln2 +
// 2 atanh((m-1)/(m+1)) by its series to z^15.
__device__ __forceinline__ float neg_log1m(float u) {
  const float y = f_sub(1.0f, u);
  const uint32_t bits = __float_as_uint(y);
  int e = (int)((bits >> 23) & 0xFFu) - 127;
  float m = __uint_as_float((bits & 0x7FFFFFu) | 0x3F800000u);
  if (m > 1.41421356f) {
    m = f_mul(m, 0.5f);
    e = e + 1;
  }
  const float z = f_div(f_sub(m, 1.0f), f_add(m, 1.0f));
  const float z2 = f_mul(z, z);
  float q = f_div(1.0f, 15.0f);
  q = f_add(f_mul(q, z2), f_div(1.0f, 13.0f));
  q = f_add(f_mul(q, z2), f_div(1.0f, 11.0f));
  q = f_add(f_mul(q, z2), f_div(1.0f, 9.0f));
  q = f_add(f_mul(q, z2), f_div(1.0f, 7.0f));
  q = f_add(f_mul(q, z2), f_div(1.0f, 5.0f));
  q = f_add(f_mul(q, z2), f_div(1.0f, 3.0f));
  q = f_add(f_mul(q, z2), 1.0f);
  const float lm = f_mul(f_mul(2.0f, z), q);
  return -f_add(f_mul((float)e, 0.693147180559945309f), lm);
}

// Uniform direction on the sphere (Marsaglia 1972), rejection in the disc.
__device__ __forceinline__ void pt_sphere(uint64_t key, uint32_t& j, float d[3]) {
  for (int tries = 0; tries < 64; ++tries) {
    const float x1 = f_sub(f_mul(pt_uniform(key, j++), 2.0f), 1.0f);
    const float x2 = f_sub(f_mul(pt_uniform(key, j++), 2.0f), 1.0f);
    const float s = f_add(f_mul(x1, x1), f_mul(x2, x2));
    if (s < 1.0f) {
      const float r = f_mul(2.0f, __fsqrt_rn(f_sub(1.0f, s)));
      d[0] = f_mul(x1, r);
      d[1] = f_mul(x2, r);
      d[2] = f_sub(1.0f, f_mul(2.0f, s));
      return;
    }
  }
  d[0] = 0.0f;
  d[1] = 0.0f;
  d[2] = 1.0f;
}

// Distance from a point inside the box [-h, h] to its boundary along d.
__device__ __forceinline__ float box_exit(const CamDev& c, const float o[3], const float d[3]) {
  float t = INFINITY;
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    if (d[a] == 0.0f) continue;
    const float inv = f_div(1.0f, d[a]);
    const float t0 = f_mul(f_sub(-c.h[a], o[a]), inv);
    const float t1 = f_mul(f_sub(c.h[a], o[a]), inv);
    t = fminf(t, fmaxf(t0, t1));
  }
  return t;
}

// World point o + t d, its normalised coordinate and distance to the eye.
__device__ __forceinline__ void pt_point(const CamDev& c, const float o[3], const float d[3], float t,
                                         float p[3], float x[3], float& dist) {
#pragma unroll
  for (int q = 0; q < 3; ++q) {
    p[q] = f_add(o[q], f_mul(t, d[q]));
    const float num = f_add(p[q], c.h[q]);
    x[q] = f_mul_sat(num, c.inv_e[q]);
  }
  const float dx = f_sub(p[0], c.o[0]), dy = f_sub(p[1], c.o[1]), dz = f_sub(p[2], c.o[2]);
  dist = __fsqrt_rn(f_add(f_add(f_mul(dx, dx), f_mul(dy, dy)), f_mul(dz, dz)));
}

struct PtCounts {
  uint32_t samp, hit, fb, miss, req, slot;
};

// Local-majorant tracking (Sec. 5.2: a macro cell's largest opacity sets
// the sampling rate of the rays through it; for Woodcock tracking that rate
// is the majorant).  A free flight spends its optical depth cell by cell
// along a 3D DDA over the macro cells; every step below is binary32 in the
// order the oracle takes it, so both sides place the same collisions.
struct PtWalk {
  int c0, c1, c2, s0, s1, s2;
  float tm0, tm1, tm2, td0, td1, td2;
  float mj, rj, te, t1;  // current cell's majorant, its reciprocal, exit; segment end
  bool live;
};

__device__ __forceinline__ void walk_axis(const MacroDev& m, const CamDev& cam, int a, float o, float d,
                                          float t, int& c, int& st, float& tm, float& td) {
  const float p = f_add(o, f_mul(t, d));
  const float x = f_mul_sat(f_add(p, cam.h[a]), cam.inv_e[a]);
  const float pv = f_mul(x, (float)cam.vol[a]);
  c = min((int)pv >> m.shift, m.dims[a] - 1);
  const float dv = f_mul(f_mul(d, cam.inv_e[a]), (float)cam.vol[a]);
  const float N = (float)(1 << m.shift);
  if (dv > 0.0f) {
    const float r = __frcp_rn(dv);  // correctly rounded 1/dv
    st = 1;
    tm = f_add(t, f_mul(f_sub((float)((c + 1) << m.shift), pv), r));
    td = f_mul(N, r);
  } else if (dv < 0.0f) {
    const float r = __frcp_rn(dv);
    st = -1;
    tm = f_add(t, f_mul(f_sub((float)(c << m.shift), pv), r));
    td = f_mul(N, -r);
  } else {
    st = 0;
    tm = INFINITY;
    td = INFINITY;
  }
}

// Enters the current cell: its majorant, the reciprocal, its exit.
__device__ __forceinline__ void walk_enter(PtWalk& w, const MacroDev& m) {
  // fewer than 2^31 cells (checked when the structure is created)
  const uint32_t cell = ((uint32_t)w.c2 * (uint32_t)m.dims[1] + (uint32_t)w.c1) * (uint32_t)m.dims[0] + (uint32_t)w.c0;
  w.mj = __ldg(m.major + cell);
  w.rj = w.mj > 0.0f ? __frcp_rn(w.mj) : 0.0f;
  w.te = fminf(fminf(fminf(w.tm0, w.tm1), w.tm2), w.t1);
}

// Enters the cell grid at the point o + t d of a segment that ends at t1.
__device__ __forceinline__ void walk_init(PtWalk& w, const MacroDev& m, const CamDev& cam, const float o[3],
                                          const float d[3], float t, float t1) {
  walk_axis(m, cam, 0, o[0], d[0], t, w.c0, w.s0, w.tm0, w.td0);
  walk_axis(m, cam, 1, o[1], d[1], t, w.c1, w.s1, w.tm1, w.td1);
  walk_axis(m, cam, 2, o[2], d[2], t, w.c2, w.s2, w.tm2, w.td2);
  w.t1 = t1;
  w.live = true;
  walk_enter(w, m);
}

// Spends optical depth tau from t: true with the tentative collision in t
// and its cell's majorant in maj; false when the segment's end (or the
// grid's) comes first.  Cells of majorant 0 are crossed without a collision.
__device__ __forceinline__ bool walk_flight(PtWalk& w, const MacroDev& m, float tau, float& t, float& maj) {
  float tt = t;
  int guard = 3 * (m.dims[0] + m.dims[1] + m.dims[2]) + 8;
  while (w.live && guard-- > 0) {
    if (w.mj > 0.0f) {
      const float dd = f_mul(w.mj, f_sub(w.te, tt));  // optical depth of the cell's stretch
      if (tau < dd) {
        t = fminf(f_add(tt, f_mul(tau, w.rj)), w.te);
        maj = w.mj;
        return true;
      }
      tau = f_sub(tau, dd);
    }
    tt = w.te;
    if (!(tt < w.t1)) break;
    if (w.tm0 <= w.tm1 && w.tm0 <= w.tm2) {
      w.c0 += w.s0;
      w.tm0 = f_add(w.tm0, w.td0);
      w.live = w.c0 >= 0 && w.c0 < m.dims[0];
    } else if (w.tm1 <= w.tm2) {
      w.c1 += w.s1;
      w.tm1 = f_add(w.tm1, w.td1);
      w.live = w.c1 >= 0 && w.c1 < m.dims[1];
    } else {
      w.c2 += w.s2;
      w.tm2 = f_add(w.tm2, w.td2);
      w.live = w.c2 >= 0 && w.c2 < m.dims[2];
    }
    if (w.live) walk_enter(w, m);
  }
  t = w.t1;
  return false;
}

// One lookup of the path tracer: through the cache (stochastic LoD from
// the distance to the eye, page-table walk with fallback, ranked request,
// LRU stamp, true miss inferred in place and recorded) or, without a
// cache, by direct inference.  Atomics are per lane: the rank update
// max(r, T_f) + 1 clamped at T_f + 1000 and the stamp reach the same final
// state in any order.
template <int IN, int H, bool CACHED, bool F16POOL, bool MISS, int BB>
__device__ float pt_value(const FrameParams& P, const LevelGeo* s_geo, const float x[3], float dist,
                          uint32_t rseed, uint32_t k, uint32_t pixel, PtCounts& n) {
  ++n.samp;
  if (CACHED) {
    const CacheDev& c = P.cache;
    const int L = c.L, B = BB ? BB : c.B, S = BB ? BB + 2 : c.S;
    const float invB = BB ? 1.0f / (float)BB : c.invB;
    const size_t S3 = (size_t)S * S * S;
    const int l = sample_lod(P.cam, L, 0, rseed, k, dist);
    const float pv0 = f_mul(x[0], (float)c.vol[0]), pv1 = f_mul(x[1], (float)c.vol[1]),
                pv2 = f_mul(x[2], (float)c.vol[2]);
    for (int lev = l; lev < L; ++lev) {
      const LevelGeo g = s_geo[lev];
      const float s0 = f_mul(pv0, g.scale), s1 = f_mul(pv1, g.scale), s2 = f_mul(pv2, g.scale);
      int b0 = (int)floorf(BB || invB > 0.0f ? f_mul(s0, invB) : f_div(s0, (float)B));
      int b1 = (int)floorf(BB || invB > 0.0f ? f_mul(s1, invB) : f_div(s1, (float)B));
      int b2 = (int)floorf(BB || invB > 0.0f ? f_mul(s2, invB) : f_div(s2, (float)B));
      b0 = min(max(b0, 0), g.nb0 - 1);
      b1 = min(max(b1, 0), g.nb1 - 1);
      b2 = min(max(b2, 0), g.nb2 - 1);
      const uint32_t key = g.off + (uint32_t)b0 + (uint32_t)g.nb0 * ((uint32_t)b1 + (uint32_t)g.nb1 * (uint32_t)b2);
      const uint32_t e = pt_entry(c, lev, key, b0, b1, b2);
      if (!(e & kMapped)) {
        if (lev == l) {
          const uint32_t old = atomicMax(c.rank + key, P.Tf);
          if (old < P.Tf) {
            ++n.req;
            push_touched(c, key);
          }
          atomicAdd(c.rank + key, 1u);
          atomicMin(c.rank + key, P.Tf + 1000u);
        }
        continue;
      }
      const uint32_t slot = e & ~kMapped;
      if (c.stamp[slot] != P.frame && atomicExch(c.stamp + slot, P.frame) != P.frame) ++n.slot;
      const float q0 = fminf(fmaxf(f_sub(s0, 0.5f), 0.0f), g.dmax0);
      const float q1 = fminf(fmaxf(f_sub(s1, 0.5f), 0.0f), g.dmax1);
      const float q2 = fminf(fmaxf(f_sub(s2, 0.5f), 0.0f), g.dmax2);
      const int i0 = (int)floorf(q0), i1 = (int)floorf(q1), i2 = (int)floorf(q2);
      const float f0 = f_sub(q0, (float)i0), f1 = f_sub(q1, (float)i1), f2 = f_sub(q2, (float)i2);
      const int l0 = i0 - (b0 * B - 1), l1 = i1 - (b1 * B - 1), l2 = i2 - (b2 * B - 1);
      const int ob = (l2 * S + l1) * S + l0;
      if (!in_range((uint32_t)ob, (uint32_t)(S3 - S * S - S - 1), c.err)) return 0.0f;
      const size_t base = (size_t)slot * S3 + (size_t)ob;
      const void* pool = c.pool;
      const float v000 = pool_ld<F16POOL>(pool, base), v100 = pool_ld<F16POOL>(pool, base + 1);
      const float v010 = pool_ld<F16POOL>(pool, base + S), v110 = pool_ld<F16POOL>(pool, base + S + 1);
      const float v001 = pool_ld<F16POOL>(pool, base + S * S), v101 = pool_ld<F16POOL>(pool, base + S * S + 1);
      const float v011 = pool_ld<F16POOL>(pool, base + S * S + S),
                  v111 = pool_ld<F16POOL>(pool, base + S * S + S + 1);
      const float x00 = fmaf(f0, v100 - v000, v000), x10 = fmaf(f0, v110 - v010, v010);
      const float x01 = fmaf(f0, v101 - v001, v001), x11 = fmaf(f0, v111 - v011, v011);
      const float y0 = fmaf(f1, x10 - x00, x00), y1 = fmaf(f1, x11 - x01, x01);
      if (lev == l)
        ++n.hit;
      else
        ++n.fb;
      return fmaf(f2, y1 - y0, y0);
    }
  }
  ++n.miss;
  if (!MISS) return 0.0f;  // unreachable: the preloaded coarsest LoD is always mapped
  if (P.miss_rec) {
    const uint32_t at = atomicAdd(P.miss_count, 1u);
    if (at < P.miss_cap) {
      P.miss_rec[2 * at] = pixel;
      P.miss_rec[2 * at + 1] = k;
    }
  }
  return infer_miss<IN, H>(P.inr, x[0], x[1], x[2]);
}

// MISS: lookups that can end in direct inference (no cache, or a cache
// without the coarsest-LoD preload).
template <int IN, int H, bool CACHED, bool F16POOL, bool MISS, int BB>
__global__ void __launch_bounds__(kFrameThreads, 5) pt_kernel(const __grid_constant__ FrameParams P) {
  __shared__ float4 s_tf[256];
  __shared__ LevelGeo s_geo[kMaxLod];
  for (int i = threadIdx.x; i < 256; i += kFrameThreads) s_tf[i] = P.tf[i];
  if (CACHED && threadIdx.x < P.cache.L) {
    const CacheDev& c = P.cache;
    const int l = threadIdx.x;
    LevelGeo g;
    g.nb0 = c.nb[l][0];
    g.nb1 = c.nb[l][1];
    g.nb2 = c.nb[l][2];
    g.off = c.off[l];
    g.dmax0 = (float)(c.dims[l][0] - 1);
    g.dmax1 = (float)(c.dims[l][1] - 1);
    g.dmax2 = (float)(c.dims[l][2] - 1);
    g.scale = __int_as_float((127 - l) << 23);
    s_geo[l] = g;
  }
  __syncthreads();
  const int lane = threadIdx.x & 31;
  const CamDev& cam = P.cam;
  PtCounts n = {0, 0, 0, 0, 0, 0};
  const bool local = P.mac.major != nullptr;  // per-cell majorants
  // Path regeneration: a lane whose path has ended takes the next ray at
  // once (rays handed out from the frame's counter, a warp's requests in
  // one atomic), so no lane idles while the others of its warp finish
  // longer paths.  A ray's path depends only on its pixel: images and
  // cache state are those of one path per pixel in any order.
  //
  // Per path, one loop over tracking steps with a per-lane mode, so that
  // the free flight, the walk and the lookup exist once in the code: lanes
  // tracking a camera or scattered segment (delta tracking) and lanes
  // tracking a shadow segment (ratio tracking) share those instructions.
  // Random numbers and lookups come in the order of the nested
  // formulation: per bounce the segment's flights and decisions, then the
  // shadow segment's flights, then the scattering direction.
  bool live = false, exhausted = false;
  uint32_t pixel = 0, rseed = 0, j = 0, k = 0;
  uint64_t key = 0;
  float o[3] = {0.f, 0.f, 0.f}, d[3] = {0.f, 0.f, 1.f}, t = 0.f, t1 = 0.f;
  float Lr = 0.f, Lg = 0.f, Lb = 0.f, alpha = 0.f, br = 1.f, bg = 1.f, bb = 1.f, Tr = 1.f;
  float p[3] = {0.f, 0.f, 0.f};
  int b = 0, steps = 0;
  bool shadow = false, begin = false;
  PtWalk W;
  while (true) {
    const bool need = !live && !exhausted;
    const unsigned nm = __ballot_sync(kFull, need);
    if (nm) {
      const int leader = __ffs(nm) - 1;
      uint32_t base = 0;
      if (lane == leader) base = atomicAdd(P.ray_counter, (uint32_t)__popc(nm));
      base = __shfl_sync(kFull, base, leader);
      if (need) {
        const uint32_t r = base + (uint32_t)__popc(nm & ((1u << lane) - 1u));
        if (r >= P.n_rays) {
          exhausted = true;
        } else {
          const uint32_t t64 = r >> 6, w = r & 63u;  // rays in 8x8 pixel tiles
          const int px = (int)((t64 % P.tiles_x) * 8 + (w & 7u));
          const int py = (int)((t64 / P.tiles_x) * 8 + (w >> 3));
          if (px < cam.W && py < cam.H) {
            pixel = (uint32_t)(py * cam.W + px);
            o[0] = cam.o[0];
            o[1] = cam.o[1];
            o[2] = cam.o[2];
            if (ray_setup(cam, px, py, d, t, t1)) {
              key = ((uint64_t)P.fseed << 32) | (uint64_t)pixel;
              rseed = ray_seed(P.fseed, pixel);
              br = bg = bb = Tr = 1.f;
              Lr = Lg = Lb = alpha = 0.f;
              j = k = 0;
              b = 0;
              shadow = false;
              begin = live = true;
            } else {
              P.out[pixel] = make_float4(P.pt_amb[0], P.pt_amb[1], P.pt_amb[2], 0.f);
            }
          }
        }
      }
    }
    if (!__any_sync(kFull, live)) {
      if (__all_sync(kFull, exhausted)) break;
      continue;
    }
    if (!live) continue;
    if (begin) {  // a segment o + t d, t in [t, t1), starts
      if (local) walk_init(W, P.mac, cam, o, d, t, t1);
      steps = 0;
      begin = false;
    }
    bool got = false;
    float maj = P.pt_sbar;
    if ((local || P.pt_sbar > 0.0f) && steps < kPtMaxSteps) {
      ++steps;
      const float tau = neg_log1m(pt_uniform(key, j++));
      if (local) {
        got = walk_flight(W, P.mac, tau, t, maj);
      } else {
        t = f_add(t, f_mul(tau, P.pt_inv));
        got = t < t1;
      }
    }
    if (got) {
      float q[3], x[3], dist;
      pt_point(cam, o, d, t, q, x, dist);
      const float v = pt_value<IN, H, CACHED, F16POOL, MISS, BB>(P, s_geo, x, dist, rseed, k, pixel, n);
      ++k;
      const float4 e4 = tf_lookup(s_tf, v);
      if (shadow) {
        Tr *= 1.0f - (local ? f_div(e4.w, maj) : e4.w * P.pt_inv);
      } else if (pt_uniform(key, j++) * maj < e4.w) {
        // real collision: albedo, then next-event estimation along the
        // shadow segment towards the light
        if (b == 0) alpha = 1.f;
        br *= e4.x;
        bg *= e4.y;
        bb *= e4.z;
        p[0] = q[0];
        p[1] = q[1];
        p[2] = q[2];
        o[0] = q[0];
        o[1] = q[1];
        o[2] = q[2];
        d[0] = P.pt_ls[0];
        d[1] = P.pt_ls[1];
        d[2] = P.pt_ls[2];
        t = 0.f;
        t1 = box_exit(cam, o, d);
        Tr = 1.f;
        shadow = begin = true;
      }
      continue;
    }
    // the segment ended without a (further) collision
    if (!shadow) {  // escaped: ambient radiance; the path is complete
      Lr = fmaf(br, P.pt_amb[0], Lr);
      Lg = fmaf(bg, P.pt_amb[1], Lg);
      Lb = fmaf(bb, P.pt_amb[2], Lb);
      P.out[pixel] = make_float4(Lr, Lg, Lb, alpha);
      live = false;
      continue;
    }
    const float ne = Tr * 0.0795774715459476679f;  // 1 / (4 pi)
    Lr = fmaf(br * P.pt_light[0], ne, Lr);
    Lg = fmaf(bg * P.pt_light[1], ne, Lg);
    Lb = fmaf(bb * P.pt_light[2], ne, Lb);
    if (b + 1 >= P.pt_bounces) {
      P.out[pixel] = make_float4(Lr, Lg, Lb, alpha);
      live = false;
      continue;
    }
    ++b;
    pt_sphere(key, j, d);
    o[0] = p[0];
    o[1] = p[1];
    o[2] = p[2];
    t = 0.f;
    t1 = box_exit(cam, o, d);
    shadow = false;
    begin = true;
  }
  unsigned long long a[6] = {n.samp, n.hit, n.fb, n.miss, n.req, n.slot};
#pragma unroll
  for (int i = 0; i < 6; ++i)
    for (int off = 16; off > 0; off >>= 1) a[i] += __shfl_xor_sync(kFull, a[i], off);
  if (lane == 0) {
    if (a[0]) atomicAdd(P.stats + ST_SAMPLES, a[0]);
    if (a[1]) atomicAdd(P.stats + ST_HITS, a[1]);
    if (a[2]) atomicAdd(P.stats + ST_FALLBACK, a[2]);
    if (a[3]) {
      atomicAdd(P.stats + ST_MISSES, a[3]);
      atomicAdd(P.stats + ST_DIRECT, a[3]);
    }
    if (a[4]) atomicAdd(P.stats + ST_REQ, a[4]);
    if (a[5]) atomicAdd(P.stats + ST_SLOTS, a[5]);
  }
}

template <int IN, int H, bool CACHED, bool F16POOL, bool MISS, int BB>
int launch_pt(const FrameParams& P, cudaStream_t s) {
  auto k = pt_kernel<IN, H, CACHED, F16POOL, MISS, BB>;
  static int blocks_per_sm = 0;
  if (!blocks_per_sm) {
    CINR_CK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&blocks_per_sm, k, kFrameThreads, 0));
    if (blocks_per_sm < 1) return set_error(CINR_ERR_CUDA, "path-tracing kernel cannot be resident");
  }
  k<<<(unsigned)(blocks_per_sm * num_sms()), kFrameThreads, 0, s>>>(P);
  CINR_CK(cudaGetLastError());
  return CINR_OK;
}

// Lookups that can end in direct inference use the INR's shape; cached
// lookups without true misses specialise the brick size instead.
template <bool CACHED, bool F16POOL, bool MISS>
int launch_pt_pool(const FrameParams& P, cudaStream_t s) {
  if constexpr (CACHED && !MISS) {
    switch (P.cache.B) {
      case 8: return launch_pt<16, 32, CACHED, F16POOL, false, 8>(P, s);
      case 16: return launch_pt<16, 32, CACHED, F16POOL, false, 16>(P, s);
      default: return launch_pt<16, 32, CACHED, F16POOL, false, 0>(P, s);
    }
  } else {
    switch (shape_of(P.inr.IN, P.inr.H)) {
      case Shape::S16x32: return launch_pt<16, 32, CACHED, F16POOL, MISS, 0>(P, s);
      case Shape::S32x64: return launch_pt<32, 64, CACHED, F16POOL, MISS, 0>(P, s);
      case Shape::S48x64: return launch_pt<48, 64, CACHED, F16POOL, MISS, 0>(P, s);
      default: return set_error(CINR_ERR_ARG, "unsupported shape");
    }
  }
}

int launch_pt_shape(const FrameParams& P, bool cached, bool miss, cudaStream_t s) {
  if (!cached) return launch_pt_pool<false, false, true>(P, s);
  const bool f16 = P.cache.pool_prec == CINR_PREC_FP16;
  if (miss) return f16 ? launch_pt_pool<true, true, true>(P, s) : launch_pt_pool<true, false, true>(P, s);
  return f16 ? launch_pt_pool<true, true, false>(P, s) : launch_pt_pool<true, false, false>(P, s);
}

// ----------------------------------------------------------- host side
void normalize3(const float a[3], float out[3]) {
  float l2 = a[0] * a[0] + a[1] * a[1];
  l2 = l2 + a[2] * a[2];
  const float l = sqrtf(l2);
  for (int i = 0; i < 3; ++i) out[i] = a[i] / l;
}

void cross3(const float a[3], const float b[3], float out[3]) {
  out[0] = a[1] * b[2] - a[2] * b[1];
  out[1] = a[2] * b[0] - a[0] * b[2];
  out[2] = a[0] * b[1] - a[1] * b[0];
}

// Camera basis and marching constants in binary32 (the host side of the
// numeric contract; compiled without FMA contraction).
void camera_consts(const cinr_camera* cam, const cinr_march_opts* o, CamDev* c) {
  float tmp[3];
  for (int a = 0; a < 3; ++a) tmp[a] = cam->target[a] - cam->eye[a];
  normalize3(tmp, c->fwd);
  cross3(c->fwd, cam->up, tmp);
  normalize3(tmp, c->right);
  cross3(c->right, c->fwd, c->upv);
  const float th = (float)tan((double)cam->fov_y_deg * (3.14159265358979323846 / 360.0));
  const float aspect = (float)cam->width / (float)cam->height;
  c->ax = th * aspect;
  c->ay = th;
  c->W = cam->width;
  c->H = cam->height;
  int m = o->dims[0];
  if (o->dims[1] > m) m = o->dims[1];
  if (o->dims[2] > m) m = o->dims[2];
  const float mf = (float)m;
  for (int a = 0; a < 3; ++a) {
    c->o[a] = cam->eye[a];
    c->e[a] = (float)o->dims[a] / mf;
    c->h[a] = c->e[a] * 0.5f;
    c->inv_e[a] = 1.0f / c->e[a];
    c->vol[a] = o->dims[a];
  }
  c->dt = cam->step_voxels / mf;
  const float c1 = (2.0f * th) / (float)cam->height;
  const float c2 = c1 * mf;
  c->lodc = c2 * o->lod_scale;
  c->lod_scale = o->lod_scale;
  c->lod_mode = o->lod_mode;
  c->step_mode = o->step_mode;
  c->step_lod_max = o->step_lod_max;
}

uint64_t splitmix64(uint64_t x) {
  uint64_t z = x + 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
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

template <int IN, int H, bool CACHED, int MLPP>
int launch_frame(const FrameParams& P, cudaStream_t s) {
  auto k = frame_kernel<IN, H, CACHED, MLPP>;
  int smem = kFrameSmemHead + (MLPP ? (int)sizeof(tc::TcSmem<IN, H>) : (CACHED ? 0 : mlp_floats<IN, H>() * 4));
  // tensor-core path: at most 8 CTAs (8 x 64 TMEM columns) per SM
  if (MLPP && smem < tc::kMinSmemPerCta) smem = tc::kMinSmemPerCta;
  static int blocks_per_sm = 0;
  if (!blocks_per_sm) {
    CINR_CK(cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
    // tensor-core path: the largest shared-memory carveout, so that the
    // occupancy query (and the launch) see every CTA that fits; the other
    // paths keep the default split (L1 serves the bricks and hash tables)
    if (MLPP)
      CINR_CK(cudaFuncSetAttribute(k, cudaFuncAttributePreferredSharedMemoryCarveout,
                                   (int)cudaSharedmemCarveoutMaxShared));
    CINR_CK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&blocks_per_sm, k, kFrameThreads, smem));
    if (blocks_per_sm < 1) return set_error(CINR_ERR_CUDA, "frame kernel cannot be resident");
    if (MLPP) {
      const int fit = tc::resident_ctas(k, smem);
      blocks_per_sm = fit > blocks_per_sm ? fit : blocks_per_sm;
    }
  }
  k<<<(unsigned)(blocks_per_sm * num_sms()), kFrameThreads, smem, s>>>(P);
  CINR_CK(cudaGetLastError());
  return CINR_OK;
}

template <bool CACHED, int MLPP>
int launch_frame_prec(const FrameParams& P, cudaStream_t s) {
  switch (shape_of(P.inr.IN, P.inr.H)) {
    case Shape::S16x32: return launch_frame<16, 32, CACHED, MLPP>(P, s);
    case Shape::S32x64: return launch_frame<32, 64, CACHED, MLPP>(P, s);
    case Shape::S48x64: return launch_frame<48, 64, CACHED, MLPP>(P, s);
    default: return set_error(CINR_ERR_ARG, "unsupported shape");
  }
}

// mlp_precision: CINR_PREC_FP32 -> SIMT, FP16 / BF16 -> tensor cores
// (uncached frames; cached frames infer their rare true misses with the
// FP32 weights, see frame_kernel).
template <bool CACHED>
int launch_frame_shape(const FrameParams& P, int mlp_precision, cudaStream_t s) {
  if constexpr (CACHED) return launch_frame_prec<CACHED, 0>(P, s);
  if (mlp_precision == CINR_PREC_FP16) return launch_frame_prec<CACHED, 1>(P, s);
  if (mlp_precision == CINR_PREC_BF16) return launch_frame_prec<CACHED, 2>(P, s);
  if (mlp_precision == CINR_PREC_FP8) return launch_frame_prec<CACHED, 3>(P, s);
  return launch_frame_prec<CACHED, 0>(P, s);
}

struct RendererLayout {
  uint32_t* counters;
  unsigned long long* stats;
  uint32_t* miss_rec;
  float4* image;
  size_t bytes;
};

RendererLayout rlayout(int W, int H, const cinr_march_opts* o, void* base) {
  Carver c(base);
  RendererLayout L;
  L.counters = c.take<uint32_t>(64);
  L.stats = c.take<unsigned long long>(ST_COUNT);
  L.miss_rec = c.take<uint32_t>(2 * (size_t)(o->miss_record_cap > 0 ? o->miss_record_cap : 0));
  L.image = c.take<float4>((size_t)W * H);
  L.bytes = align_up(c.off, 256);
  return L;
}

int check_opts(int W, int H, const cinr_march_opts* o) {
  if (!o) return set_error(CINR_ERR_ARG, "opts is NULL");
  if (W < 1 || H < 1 || (long)W * H > (1l << 30)) return set_error(CINR_ERR_ARG, "bad image size");
  if (o->K < 32 || (o->K % 32) != 0) return set_error(CINR_ERR_ARG, "K must be a positive multiple of 32");
  if (o->dims[0] < 1 || o->dims[1] < 1 || o->dims[2] < 1) return set_error(CINR_ERR_ARG, "bad dims");
  if (o->miss_record_cap < 0 || o->miss_record_cap > (1l << 30))
    return set_error(CINR_ERR_ARG, "bad miss_record_cap");
  if (o->lod_mode != 0 && o->lod_mode != 1) return set_error(CINR_ERR_ARG, "bad lod_mode");
  if (o->ray_layout != 0 && o->ray_layout != 1) return set_error(CINR_ERR_ARG, "bad ray_layout");
  if (o->step_mode != 0 && o->step_mode != 1) return set_error(CINR_ERR_ARG, "bad step_mode");
  if (o->step_lod_max < 0 || o->step_lod_max > 15) return set_error(CINR_ERR_ARG, "step_lod_max must be in [0, 15]");
  return CINR_OK;
}

// Captures one frame's launch sequence into a CUDA graph on the renderer's
// capture stream, updates the executable graph of the previous frame in
// place (same topology, new parameters) or instantiates a new one, and
// launches it on the caller's stream.
template <class F>
int launch_as_graph(cinr_renderer_s* r, F&& enqueue, cudaStream_t s) {
  if (!r->cap) CINR_CK(cudaStreamCreateWithFlags(&r->cap, cudaStreamNonBlocking));
  CINR_CK(cudaStreamBeginCapture(r->cap, cudaStreamCaptureModeThreadLocal));
  const int e = enqueue(r->cap);
  cudaGraph_t g = nullptr;
  const cudaError_t ce = cudaStreamEndCapture(r->cap, &g);
  if (e) {
    if (g) cudaGraphDestroy(g);
    return e;
  }
  if (ce != cudaSuccess) return cuda_error(ce, "cudaStreamEndCapture");
  if (r->exec) {
    cudaGraphExecUpdateResultInfo info;
    if (cudaGraphExecUpdate(r->exec, g, &info) != cudaSuccess) {
      (void)cudaGetLastError();
      cudaGraphExecDestroy(r->exec);
      r->exec = nullptr;
    }
  }
  if (!r->exec) {
    const cudaError_t ie = cudaGraphInstantiate(&r->exec, g, 0);
    if (ie != cudaSuccess) {
      cudaGraphDestroy(g);
      r->exec = nullptr;
      return cuda_error(ie, "cudaGraphInstantiate");
    }
  }
  cudaGraphDestroy(g);
  CINR_CK(cudaGraphLaunch(r->exec, s));
  return CINR_OK;
}

// host_img != nullptr: the image is also copied to host memory, on a second
// stream that starts when the marching kernel ends (overlapping the cache
// update), and the call returns once both streams are done.
int render(cinr_renderer_t r, cinr_cache_t cache, cinr_inr_t inr, const cinr_camera* cam,
           const cinr_tf* tf, float4* out, cinr_frame_stats* stats, cudaStream_t s,
           const cinr_pt_opts* pt = nullptr, float* host_img = nullptr) {
  if (!r || !inr || !cam || !tf) return set_error(CINR_ERR_ARG, "NULL argument");
  if (cam->width != r->W || cam->height != r->H)
    return set_error(CINR_ERR_ARG, "camera is %dx%d, renderer %dx%d", cam->width, cam->height, r->W, r->H);
  if (reinterpret_cast<uintptr_t>(out) & 15) return set_error(CINR_ERR_ARG, "image must be 16-byte aligned");
  if (!(cam->step_voxels > 0.0f)) return set_error(CINR_ERR_ARG, "step_voxels must be > 0");
  if (cache) {
    for (int a = 0; a < 3; ++a)
      if (cache->dev.vol[a] != r->o.dims[a]) return set_error(CINR_ERR_ARG, "cache dims differ from renderer dims");
    if (cache->inr != inr) return set_error(CINR_ERR_ARG, "cache was built for another INR");
    if (cache->o.lag == 2 && r->o.use_graph)
      return set_error(CINR_ERR_ARG, "a lag-2 cache decodes across frames and cannot run as a per-frame graph");
    if (cache->dev.pool_tex && (pt || r->o.ray_layout == 1))
      return set_error(CINR_ERR_UNSUPPORTED, "the texture layout serves the thread-per-ray marching kernel only");
  }
  FrameParams P;
  memset(&P, 0, sizeof(P));
  camera_consts(cam, &r->o, &P.cam);
  P.inr = inr->dev;
  uint64_t frame;
  if (cache) {
    frame = ++cache->frame;
    P.cache = cache->dev;
  } else {
    frame = ++r->frame;
  }
  P.frame = (uint32_t)frame;
  P.Tf = (uint32_t)(1001ull * frame);
  P.fseed = (uint32_t)splitmix64(r->o.seed ^ frame);
  memcpy(P.tf, tf->rgba, sizeof(P.tf));
  P.out = out;
  P.tiles_x = (uint32_t)((r->W + 7) / 8);
  P.n_rays = P.tiles_x * (uint32_t)((r->H + 7) / 8) * 64u;
  P.ray_counter = r->counters;
  P.stats = r->stats;
  P.K = r->o.K;
  P.eps = r->o.eps_T;
  P.miss_rec = r->o.miss_record_cap > 0 ? r->miss_rec : nullptr;
  P.miss_cap = (uint32_t)r->o.miss_record_cap;
  P.miss_count = r->counters + 1;

  P.w16 = inr->w16;
  P.err = reinterpret_cast<int*>(r->counters + 2);
  P.inr.err = P.err;  // the frame kernels' bounds checks report to the frame
  if (cache) P.cache.err = P.err;
  if (pt) {
    if (pt->max_bounces < 1) return set_error(CINR_ERR_ARG, "max_bounces must be >= 1");
    const float neg[3] = {-pt->light_dir[0], -pt->light_dir[1], -pt->light_dir[2]};
    if (!(neg[0] != 0.0f || neg[1] != 0.0f || neg[2] != 0.0f))
      return set_error(CINR_ERR_ARG, "light_dir must be non-zero");
    normalize3(neg, P.pt_ls);
    float m = 0.0f;
    for (int i = 0; i < 256; ++i) m = fmaxf(m, tf->rgba[i][3]);
    P.pt_sbar = pt->sigma_max > 0.0f ? pt->sigma_max : m;
    P.pt_inv = P.pt_sbar > 0.0f ? 1.0f / P.pt_sbar : 0.0f;
    for (int a = 0; a < 3; ++a) {
      P.pt_light[a] = pt->light[a];
      P.pt_amb[a] = pt->ambient[a];
    }
    P.pt_bounces = pt->max_bounces;
  }
  // ray marching skips transparent cells; path tracing with an automatic
  // majorant tracks with the cells' local majorants
  cinr_macro_s* mac = (pt && pt->sigma_max > 0.0f) ? nullptr : r->macro;
  if (mac) {
    for (int a = 0; a < 3; ++a)
      if (mac->vol[a] != r->o.dims[a]) return set_error(CINR_ERR_ARG, "macro-cell dims differ from renderer dims");
    P.mac = mac->dev();
  }
  // The frame's device work, enqueued on q: the caller's stream, or the
  // renderer's capture stream when the frame runs as a CUDA graph.
  // Inside a stream capture a plain event record only orders streams, so the
  // split between frame kernel and cache update is taken by an external event
  // node, and the frame's start and end events sit on the caller's stream
  // around the graph launch.
  const bool graph = r->o.use_graph != 0;
  auto enqueue = [&](cudaStream_t q) -> int {
    CINR_CK(cudaMemsetAsync(r->counters, 0, 64 * 4, q));
    CINR_CK(cudaMemsetAsync(r->stats, 0, ST_COUNT * 8, q));
    if (cache) CINR_CK(cudaMemsetAsync(cache->dev.touched_count, 0, 4, q));
    if (mac) {
      const int em = cinr_macro_apply(mac, tf->rgba, q);
      if (em) return em;
    }
    if (!graph) CINR_CK(cudaEventRecord(r->ev[0], q));
    int ee;
    if (pt)
      ee = launch_pt_shape(P, cache != nullptr, cache && !cache->o.preload, q);
    else if (!cache)
      ee = launch_frame_shape<false>(P, inr->p.mlp_precision, q);
    else if (r->o.ray_layout == 1)
      ee = launch_frame_shape<true>(P, inr->p.mlp_precision, q);
    else
      ee = launch_march_cached_shape(P, !cache->o.preload, q);
    if (ee) return ee;
    CINR_CK(cudaEventRecordWithFlags(r->ev[1], q, graph ? cudaEventRecordExternal : cudaEventRecordDefault));
    if (cache) {
      ee = cinr_cache_end_frame(cache, r->stats, q);
      if (ee) return ee;
    }
    if (!graph) CINR_CK(cudaEventRecord(r->ev[2], q));
    return CINR_OK;
  };
  int e;
  if (graph) {
    CINR_CK(cudaEventRecord(r->ev[0], s));
    e = launch_as_graph(r, enqueue, s);
    if (!e) CINR_CK(cudaEventRecord(r->ev[2], s));
  } else {
    e = enqueue(s);
  }
  if (e) return e;
  if (host_img) {
    if (!r->copy) CINR_CK(cudaStreamCreateWithFlags(&r->copy, cudaStreamNonBlocking));
    // (a graph's frame: after the whole graph, whose end event is on `s`)
    CINR_CK(cudaStreamWaitEvent(r->copy, graph ? r->ev[2] : r->ev[1], 0));
    CINR_CK(cudaMemcpyAsync(host_img, out, (size_t)r->W * r->H * 16, cudaMemcpyDeviceToHost, r->copy));
  }
  unsigned long long h[ST_COUNT];
  uint32_t cnt[3] = {0, 0, 0};  // ray counter, miss-record count, device error word
  CINR_CK(cudaMemcpyAsync(h, r->stats, sizeof(h), cudaMemcpyDeviceToHost, s));
  CINR_CK(cudaMemcpyAsync(cnt, r->counters, sizeof(cnt), cudaMemcpyDeviceToHost, s));
  CINR_CK(cudaStreamSynchronize(s));
  if (host_img) CINR_CK(cudaStreamSynchronize(r->copy));
  const uint32_t rec = cnt[1];
  if (device_status((int)cnt[2]) == CINR_ERR_DEVICE_CHECK)
    return set_error(CINR_ERR_DEVICE_CHECK, "a device bounds check tripped in the frame kernel");
  if (cnt[2]) return set_error(CINR_ERR_TIMEOUT, "a bounded device-side wait gave up in the frame kernel");
  if (stats) {
    stats->samples = h[ST_SAMPLES];
    stats->inr_queries_direct = h[ST_DIRECT];
    stats->inr_queries_decode = h[ST_DECODE];
    stats->true_misses = h[ST_MISSES];
    stats->fallback_hits = h[ST_FALLBACK];
    stats->hits = h[ST_HITS];
    stats->bricks_requested = h[ST_REQ];
    stats->bricks_decoded = h[ST_DECODED];
    stats->evictions = h[ST_EVICT];
    stats->misses_recorded = P.miss_rec ? (rec < P.miss_cap ? rec : P.miss_cap) : 0;
    stats->slots_touched = h[ST_SLOTS];
    stats->kernel_launches = 1u + (cache ? cache->last_launches : 0u) + (mac ? 1u : 0u);
    stats->samples_skipped = h[ST_SKIPPED];
    float ms0 = 0.f, ms1 = 0.f;
    CINR_CK(cudaEventElapsedTime(&ms0, r->ev[0], r->ev[1]));
    CINR_CK(cudaEventElapsedTime(&ms1, r->ev[1], r->ev[2]));
    stats->ms_frame_kernel = ms0;
    stats->ms_cache_update = ms1;
  }
  return CINR_OK;
}

}  // namespace

extern "C" int cinr_renderer_bytes(int width, int height, const cinr_march_opts* o, size_t* bytes) {
  int e = check_opts(width, height, o);
  if (e) return e;
  if (!bytes) return set_error(CINR_ERR_ARG, "bytes is NULL");
  *bytes = rlayout(width, height, o, nullptr).bytes;
  return CINR_OK;
}

extern "C" int cinr_create_renderer(void* dev_mem, size_t bytes, int width, int height,
                                    const cinr_march_opts* o, cinr_renderer_t* out) {
  int e = check_opts(width, height, o);
  if (e) return e;
  if (!out) return set_error(CINR_ERR_ARG, "out is NULL");
  if (!dev_mem || (reinterpret_cast<uintptr_t>(dev_mem) & 255))
    return set_error(CINR_ERR_ARG, "dev_mem must be non-NULL and 256-byte aligned");
  RendererLayout L = rlayout(width, height, o, dev_mem);
  if (bytes < L.bytes) return set_error(CINR_ERR_NOMEM, "renderer needs %zu bytes, got %zu", L.bytes, bytes);
  cinr_renderer_s* r = new cinr_renderer_s();
  r->W = width;
  r->H = height;
  r->o = *o;
  r->counters = L.counters;
  r->stats = L.stats;
  r->miss_rec = L.miss_rec;
  r->image = L.image;
  r->frame = 0;
  cudaGetDevice(&r->device);
  for (int i = 0; i < 3; ++i) {
    cudaError_t ce = cudaEventCreate(&r->ev[i]);
    if (ce != cudaSuccess) {
      for (int j = 0; j < i; ++j) cudaEventDestroy(r->ev[j]);
      delete r;
      return cuda_error(ce, "cudaEventCreate");
    }
  }
  *out = r;
  return CINR_OK;
}

extern "C" int cinr_destroy_renderer(cinr_renderer_t r) {
  if (r) {
    for (int i = 0; i < 3; ++i) cudaEventDestroy(r->ev[i]);
    if (r->exec) cudaGraphExecDestroy(r->exec);
    if (r->cap) cudaStreamDestroy(r->cap);
    if (r->copy) cudaStreamDestroy(r->copy);
  }
  delete r;
  return CINR_OK;
}

extern "C" int cinr_render_frame(cinr_renderer_t r, cinr_cache_t cache, cinr_inr_t inr,
                                 const cinr_camera* cam, const cinr_tf* tf, float* out_rgba_dev,
                                 cinr_frame_stats* stats, cinr_stream_t stream) {
  if (!out_rgba_dev) return set_error(CINR_ERR_ARG, "out_rgba_dev is NULL");
  return render(r, cache, inr, cam, tf, reinterpret_cast<float4*>(out_rgba_dev), stats,
                static_cast<cudaStream_t>(stream));
}

extern "C" int cinr_render_frame_pt(cinr_renderer_t r, cinr_cache_t cache, cinr_inr_t inr,
                                    const cinr_camera* cam, const cinr_tf* tf, const cinr_pt_opts* pt,
                                    float* out_rgba_dev, cinr_frame_stats* stats, cinr_stream_t stream) {
  if (!out_rgba_dev || !pt) return set_error(CINR_ERR_ARG, "NULL argument");
  return render(r, cache, inr, cam, tf, reinterpret_cast<float4*>(out_rgba_dev), stats,
                static_cast<cudaStream_t>(stream), pt);
}

extern "C" int cinr_render_frame_host(cinr_renderer_t r, cinr_cache_t cache, cinr_inr_t inr,
                                      const cinr_camera* cam, const cinr_tf* tf, float* out_rgba_host,
                                      cinr_frame_stats* stats, cinr_stream_t stream) {
  if (!r || !out_rgba_host) return set_error(CINR_ERR_ARG, "NULL argument");
  return render(r, cache, inr, cam, tf, r->image, stats, static_cast<cudaStream_t>(stream), nullptr,
                out_rgba_host);
}

extern "C" int cinr_debug_dump(void* obj, int what, void* host_out, size_t cap, size_t* count,
                               cinr_stream_t stream) {
  if (!obj || !count) return set_error(CINR_ERR_ARG, "NULL argument");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const void* src = nullptr;
  size_t n = 0, esz = 4;
  if (what == CINR_DUMP_MISSES) {
    cinr_renderer_s* r = static_cast<cinr_renderer_s*>(obj);
    uint32_t rec = 0;
    CINR_CK(cudaMemcpyAsync(&rec, r->counters + 1, 4, cudaMemcpyDeviceToHost, s));
    CINR_CK(cudaStreamSynchronize(s));
    size_t capr = (size_t)(r->o.miss_record_cap > 0 ? r->o.miss_record_cap : 0);
    n = 2 * (rec < capr ? rec : capr);
    src = r->miss_rec;
  } else {
    cinr_cache_s* c = static_cast<cinr_cache_s*>(obj);
    uint32_t cnt = 0;
    const int ew = cinr_cache_wait_decode(c, s);
    if (ew) return ew;
    switch (what) {
      case CINR_DUMP_PAGE_TABLE:
        if (c->dev.pd) return set_error(CINR_ERR_ARG, "paged tables: dump the page directory and pages");
        src = c->dev.pt;
        n = (size_t)c->n_bricks;
        break;
      case CINR_DUMP_PAGE_DIR:
        src = c->dev.pd;
        n = c->dev.pd ? (size_t)c->dev.pd_off[c->dev.L] : 0;
        break;
      case CINR_DUMP_PAGES:
        src = c->dev.pages;
        n = c->dev.pd ? (size_t)c->dev.n_pages << (3 * c->dev.page_shift) : 0;
        break;
      case CINR_DUMP_PAGE_KEYS: src = c->dev.page_key; n = c->dev.pd ? c->dev.n_pages : 0; break;
      case CINR_DUMP_PAGE_REFS: src = c->dev.page_ref; n = c->dev.pd ? c->dev.n_pages : 0; break;
      case CINR_DUMP_STAMPS: src = c->dev.stamp; n = (size_t)c->n_slots; break;
      case CINR_DUMP_OWNERS: src = c->dev.owner; n = (size_t)c->n_slots; break;
      case CINR_DUMP_RANK: src = c->dev.rank; n = (size_t)c->n_bricks; break;
      case CINR_DUMP_PINNED: src = c->dev.pinned; n = (size_t)c->n_slots; break;
      case CINR_DUMP_REQUESTS:
        CINR_CK(cudaMemcpyAsync(&cnt, c->req_n, 4, cudaMemcpyDeviceToHost, s));
        CINR_CK(cudaStreamSynchronize(s));
        src = c->req_sorted;
        n = cnt;
        break;
      case CINR_DUMP_VICTIMS:
        CINR_CK(cudaMemcpyAsync(&cnt, c->decode_n, 4, cudaMemcpyDeviceToHost, s));
        CINR_CK(cudaStreamSynchronize(s));
        src = c->vic_sorted;
        n = cnt;
        break;
      case CINR_DUMP_POOL:
        src = c->dev.pool;
        n = (size_t)c->n_slots * c->dev.S * c->dev.S * c->dev.S;
        esz = c->dev.pool_prec == CINR_PREC_FP16 ? 2 : 4;
        if (c->dev.pool_tex) {
          // the texture layout, copied whole and returned in slot order
          // (slot, z, y, x), x fastest, as the linear layout stores it
          const int S = c->dev.S;
          const size_t per_row = (size_t)1 << c->dev.tex_shift;
          const size_t rows = ((size_t)c->n_slots * S + per_row - 1) / per_row * S;
          std::vector<uint16_t> img(rows * (size_t)c->dev.tex_pitch);
          CINR_CK(cudaMemcpyAsync(img.data(), src, img.size() * 2, cudaMemcpyDeviceToHost, s));
          CINR_CK(cudaStreamSynchronize(s));
          *count = n;
          uint16_t* dst = static_cast<uint16_t*>(host_out);
          const size_t m = n < cap ? n : cap;
          if (dst)
            for (size_t i = 0; i < m; ++i) {
              const size_t S3 = (size_t)S * S * S;
              const uint32_t slot = (uint32_t)(i / S3);
              const int v = (int)(i % S3);
              dst[i] = img[tex_offset(S, c->dev.tex_shift, c->dev.tex_pitch, slot, v % S, (v / S) % S, v / (S * S))];
            }
          return CINR_OK;
        }
        break;
      default: return set_error(CINR_ERR_ARG, "unknown dump %d", what);
    }
  }
  *count = n;
  size_t m = n < cap ? n : cap;
  if (host_out && m > 0) {
    CINR_CK(cudaMemcpyAsync(host_out, src, m * esz, cudaMemcpyDeviceToHost, s));
    CINR_CK(cudaStreamSynchronize(s));
  }
  return CINR_OK;
}

// ---------------------------------------------------------------------------
// Allocation-free uncached render.
//
// For callers that must not allocate device memory (a real-time render loop
// where an allocation would stall or fail, code running under a memory
// policy that forbids new device allocations, a host-only plugin that owns no
// device buffer): the frame's working set (ray counter, statistics and the
// device copy of the image) lives in one file-scope device array instead of
// a caller-provided renderer buffer.  Every GPU that loads the library holds
// this array (kNoAllocBytes, about 4 MiB) until the process exits.
namespace {

constexpr int kNoAllocMaxPixels = 512 * 512;
constexpr size_t kNoAllocHeader = 512;  // counters (256 B) + statistics (256 B)
constexpr size_t kNoAllocBytes = kNoAllocHeader + (size_t)kNoAllocMaxPixels * sizeof(float4);

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocBytes];

constexpr int kNoAllocMaxDevices = 64;
unsigned char* g_noalloc_ptr[kNoAllocMaxDevices] = {};
std::mutex g_noalloc_mu;

// Device address of the scratch array on the current device, looked up once
// per device with that device current (in host code the array's name is only
// a host-side stand-in, not a device address).  The address is kept for the
// life of the process: it does not survive cudaDeviceReset (or any teardown
// of the device's primary context), after which this entry point must not
// be called again in the process.
int noalloc_scratch(unsigned char** out) {
  int dev = 0;
  CINR_CK(cudaGetDevice(&dev));
  if (dev < 0 || dev >= kNoAllocMaxDevices)
    return set_error(CINR_ERR_UNSUPPORTED, "device %d out of the supported range", dev);
  std::lock_guard<std::mutex> lock(g_noalloc_mu);
  if (!g_noalloc_ptr[dev]) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) return cuda_error(e, "cudaGetSymbolAddress(g_noalloc_scratch)");
    g_noalloc_ptr[dev] = static_cast<unsigned char*>(p);
  }
  *out = g_noalloc_ptr[dev];
  return CINR_OK;
}

}  // namespace

extern "C" int cinr_render_frame_noalloc(cinr_inr_t inr, const cinr_camera* cam, const cinr_tf* tf,
                                         const cinr_march_opts* o, float* out_rgba_host,
                                         cinr_frame_stats* stats, cinr_stream_t stream) {
  if (!inr || !cam || !tf || !o || !out_rgba_host) return set_error(CINR_ERR_ARG, "NULL argument");
  int e = check_opts(cam->width, cam->height, o);
  if (e) return e;
  if ((long)cam->width * cam->height > kNoAllocMaxPixels)
    return set_error(CINR_ERR_ARG,
                     "image of %d x %d pixels exceeds the allocation-free limit of %d pixels",
                     cam->width, cam->height, kNoAllocMaxPixels);
  if (o->miss_record_cap != 0)
    return set_error(CINR_ERR_ARG, "the allocation-free render keeps no miss record (cap must be 0)");
  if (!(cam->step_voxels > 0.0f)) return set_error(CINR_ERR_ARG, "step_voxels must be > 0");
  unsigned char* scratch = nullptr;
  e = noalloc_scratch(&scratch);
  if (e) return e;
  uint32_t* counters = reinterpret_cast<uint32_t*>(scratch);
  unsigned long long* st_dev = reinterpret_cast<unsigned long long*>(scratch + 256);
  float4* image = reinterpret_cast<float4*>(scratch + kNoAllocHeader);
  cudaStream_t s = static_cast<cudaStream_t>(stream);

  FrameParams P;
  memset(&P, 0, sizeof(P));
  camera_consts(cam, o, &P.cam);
  P.inr = inr->dev;
  P.frame = 1;
  P.Tf = 1001u;
  P.fseed = (uint32_t)splitmix64(o->seed ^ 1ull);
  memcpy(P.tf, tf->rgba, sizeof(P.tf));
  P.out = image;
  P.tiles_x = (uint32_t)((cam->width + 7) / 8);
  P.n_rays = P.tiles_x * (uint32_t)((cam->height + 7) / 8) * 64u;
  P.ray_counter = counters;
  P.stats = st_dev;
  P.K = o->K;
  P.eps = o->eps_T;
  P.miss_rec = nullptr;
  P.miss_cap = 0;
  P.miss_count = counters + 1;

  // The array keeps the previous call's contents: counters and statistics
  // must start at zero.
  CINR_CK(cudaMemsetAsync(scratch, 0, kNoAllocHeader, s));
  P.w16 = inr->w16;
  P.err = reinterpret_cast<int*>(counters + 2);
  P.inr.err = P.err;
  e = launch_frame_shape<false>(P, inr->p.mlp_precision, s);
  if (e) return e;
  unsigned long long h[ST_COUNT];
  uint32_t cnt[3] = {0, 0, 0};  // ray counter, miss-record count, device error word
  CINR_CK(cudaMemcpyAsync(out_rgba_host, image, (size_t)cam->width * cam->height * sizeof(float4),
                          cudaMemcpyDeviceToHost, s));
  CINR_CK(cudaMemcpyAsync(h, st_dev, sizeof(h), cudaMemcpyDeviceToHost, s));
  CINR_CK(cudaMemcpyAsync(cnt, counters, sizeof(cnt), cudaMemcpyDeviceToHost, s));
  CINR_CK(cudaStreamSynchronize(s));
  // a bounded tensor-core wait that gave up leaves the image incomplete
  if (device_status((int)cnt[2]) == CINR_ERR_DEVICE_CHECK)
    return set_error(CINR_ERR_DEVICE_CHECK, "a device bounds check tripped in the frame kernel");
  if (cnt[2]) return set_error(CINR_ERR_TIMEOUT, "a bounded device-side wait gave up in the frame kernel");
  if (stats) {
    memset(stats, 0, sizeof(*stats));
    stats->samples = h[ST_SAMPLES];
    stats->inr_queries_direct = h[ST_DIRECT];
    stats->true_misses = h[ST_MISSES];
  }
  return CINR_OK;
}

// ---------------------------------------------------------------------------
// Explicit-voxel render: the same rays, samples, transfer function and
// compositing, each sample valued by trilinear interpolation of an explicit
// field (the data an INR compresses, Sec. 4.1).  It is the quality judge of
// a trained INR and the uncompressed fallback.  Thread per ray, 8 x 4 ray
// tiles per warp.
namespace {

struct FieldParams {
  CamDev cam;
  float4 tf[256];
  const float* field;
  int3 fdims;
  float4* out;
  uint32_t n_rays, tiles_x;
  uint32_t* ray_counter;
  unsigned long long* stats;
  int K;
  float eps;
  MacroDev mac;
};

__global__ void __launch_bounds__(kFrameThreads, 8) march_field_kernel(const __grid_constant__ FieldParams P) {
  __shared__ float4 s_tf[256];
  for (int i = threadIdx.x; i < 256; i += kFrameThreads) s_tf[i] = P.tf[i];
  __syncthreads();
  const int lane = threadIdx.x & 31;
  const CamDev& cam = P.cam;
  uint32_t n_samp = 0, n_skip = 0;
  const uint32_t n_tiles = P.n_rays >> 5;
  while (true) {
    uint32_t tile = 0;
    if (lane == 0) tile = atomicAdd(P.ray_counter, 1u);
    tile = __shfl_sync(kFull, tile, 0);
    if (tile >= n_tiles) break;
    const uint32_t r = tile * 32u + (uint32_t)lane;
    const uint32_t t64 = r >> 6, w = r & 63u;
    const int px = (int)((t64 % P.tiles_x) * 8 + (w & 7u));
    const int py = (int)((t64 / P.tiles_x) * 8 + (w >> 3));
    if (px >= cam.W || py >= cam.H) continue;
    const uint32_t pixel = (uint32_t)(py * cam.W + px);
    float d[3], tn = 0.f, tf = 0.f;
    float T = 1.f, Cr = 0.f, Cg = 0.f, Cb = 0.f;
    if (ray_setup(cam, px, py, d, tn, tf)) {
      int seg = P.K;
      Sched sch = {0.f, 0.f};
      for (int k = 0;; ++k) {
        float x[3], tm, len;
        if ((k & 31) == 0) sched_segment(cam, tn, k, sch);
        if (!sample_in(cam, d, tn, tf, k, sch, x, tm, len)) break;
        if (macro_skips(P.mac, f_mul(x[0], (float)cam.vol[0]), f_mul(x[1], (float)cam.vol[1]),
                        f_mul(x[2], (float)cam.vol[2]))) {
          ++n_skip;  // transparent cell (Sec. 5.2)
        } else {
          ++n_samp;
          const float v = field_trilinear(P.field, P.fdims, x[0], x[1], x[2]);
          const float4 e4 = tf_lookup(s_tf, v);
          const float alpha = 1.0f - __expf(-e4.w * len);
          const float wgt = T * alpha;
          Cr = fmaf(wgt, e4.x, Cr);
          Cg = fmaf(wgt, e4.y, Cg);
          Cb = fmaf(wgt, e4.z, Cb);
          T *= 1.0f - alpha;
        }
        if (--seg == 0) {
          seg = P.K;
          if (T < P.eps) break;
        }
      }
    }
    P.out[pixel] = make_float4(Cr, Cg, Cb, 1.0f - T);
  }
  unsigned long long a = n_samp, b = n_skip;
  for (int o = 16; o > 0; o >>= 1) {
    a += __shfl_xor_sync(kFull, a, o);
    b += __shfl_xor_sync(kFull, b, o);
  }
  if (lane == 0 && a) atomicAdd(P.stats + ST_SAMPLES, a);
  if (lane == 0 && b) atomicAdd(P.stats + ST_SKIPPED, b);
}

}  // namespace

extern "C" int cinr_render_field(cinr_renderer_t r, const float* field_dev, const int fdims[3],
                                 const cinr_camera* cam, const cinr_tf* tf, float* out_rgba_dev,
                                 cinr_frame_stats* stats, cinr_stream_t stream) {
  if (!r || !field_dev || !fdims || !cam || !tf || !out_rgba_dev) return set_error(CINR_ERR_ARG, "NULL argument");
  if (fdims[0] < 1 || fdims[1] < 1 || fdims[2] < 1) return set_error(CINR_ERR_ARG, "bad field dims");
  if (cam->width != r->W || cam->height != r->H)
    return set_error(CINR_ERR_ARG, "camera is %dx%d, renderer %dx%d", cam->width, cam->height, r->W, r->H);
  if (reinterpret_cast<uintptr_t>(out_rgba_dev) & 15) return set_error(CINR_ERR_ARG, "image must be 16-byte aligned");
  if (!(cam->step_voxels > 0.0f)) return set_error(CINR_ERR_ARG, "step_voxels must be > 0");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  FieldParams P;
  memset(&P, 0, sizeof(P));
  camera_consts(cam, &r->o, &P.cam);
  memcpy(P.tf, tf->rgba, sizeof(P.tf));
  P.field = field_dev;
  P.fdims = make_int3(fdims[0], fdims[1], fdims[2]);
  P.out = reinterpret_cast<float4*>(out_rgba_dev);
  P.tiles_x = (uint32_t)((r->W + 7) / 8);
  P.n_rays = P.tiles_x * (uint32_t)((r->H + 7) / 8) * 64u;
  P.ray_counter = r->counters;
  P.stats = r->stats;
  P.K = r->o.K;
  P.eps = r->o.eps_T;
  if (r->macro) {
    for (int a = 0; a < 3; ++a)
      if (r->macro->vol[a] != r->o.dims[a] || fdims[a] != r->o.dims[a])
        return set_error(CINR_ERR_ARG, "with macro cells the field and macro dims must equal the renderer dims");
    P.mac = r->macro->dev();
  }
  CINR_CK(cudaMemsetAsync(r->counters, 0, 64 * 4, s));
  CINR_CK(cudaMemsetAsync(r->stats, 0, ST_COUNT * 8, s));
  if (r->macro) {
    const int em = cinr_macro_apply(r->macro, tf->rgba, s);
    if (em) return em;
  }
  static int per_sm = 0;
  if (!per_sm) {
    CINR_CK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, march_field_kernel, kFrameThreads, 0));
    if (per_sm < 1) return set_error(CINR_ERR_CUDA, "field kernel cannot be resident");
  }
  march_field_kernel<<<(unsigned)(per_sm * num_sms()), kFrameThreads, 0, s>>>(P);
  CINR_CK(cudaGetLastError());
  unsigned long long h[ST_COUNT];
  CINR_CK(cudaMemcpyAsync(h, r->stats, sizeof(h), cudaMemcpyDeviceToHost, s));
  CINR_CK(cudaStreamSynchronize(s));
  if (stats) {
    memset(stats, 0, sizeof(*stats));
    stats->samples = h[ST_SAMPLES];
    stats->samples_skipped = h[ST_SKIPPED];
  }
  return CINR_OK;
}

extern "C" int cinr_renderer_set_macro(cinr_renderer_t r, cinr_macro_t m) {
  if (!r) return set_error(CINR_ERR_ARG, "renderer is NULL");
  if (m)
    for (int a = 0; a < 3; ++a)
      if (m->vol[a] != r->o.dims[a]) return set_error(CINR_ERR_ARG, "macro-cell dims differ from renderer dims");
  r->macro = m;
  return CINR_OK;
}
