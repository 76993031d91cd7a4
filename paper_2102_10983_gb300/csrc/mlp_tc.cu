// Inference of the sub-cycle-count predictor on the 5th-generation tensor
// cores: tcgen05.mma with operands in shared memory and FP32 accumulators in
// tensor memory (TMEM).  Not part of the paper: the network only predicts the
// exponent k the criterion of Sec. IV will pick next, for binning; the
// criterion still decides every sub-step.
//
// Per CTA (128 threads, one warpgroup) and tile of 128 particles:
//   features: each thread forms one particle's phi (6 values, BF16, zero-
//     padded to K = 16) and stores it as row r of A1 [128 x 16], which shares
//     its bytes with the start of A2 (layer 1 has read A1 before epilogue 1
//     writes A2, and the next tile's features are stored after layer 3 has
//     read A2);
//   layer 1: one tcgen05.mma M=128 N=64 K=16, A1 x W1^T -> D1 (TMEM cols 0..63);
//   epilogue 1: each warp reads its 32 TMEM lanes (rows) with tcgen05.ld, adds
//     b1, applies ReLU, rounds to BF16 and writes A2 [128 x 64];
//   layer 2: four MMAs (K = 16 each) A2 x W2^T -> D2, in the same columns (the
//     epilogue has read D1);
//   epilogue 2: b2, ReLU, BF16 -> A2 again (layer 2 has read it);
//   layer 3: four MMAs A2 x W3^T (N = 16, rows 8..15 of W3 zero) -> D3 (cols 0..15);
//   epilogue 3: b3, argmax over the 8 classes (ties: the smaller k).
// A CTA holds 64 TMEM columns and ~30 KB of shared memory, so seven CTAs (28
// warps, seven tiles in flight) share an SM: the chain of a tile (features,
// three MMA round trips, three epilogues) is latency-bound, the SM is kept
// busy by the other tiles.
// One thread issues the MMAs, commits them to an mbarrier and waits on it (a
// bounded wait: on a give-up the CTA records it, marks its remaining
// predictions 0xFF, an invalid class, frees its TMEM and returns); the other
// threads wait at a CTA barrier, which takes no issue slots.
//
// Shared-memory operands use the no-swizzle K-major layout of 8 x 16-byte
// core matrices: element (r, k) of an R x K tile sits at
// (r / 8) * (K / 8) * 128 + (k / 8) * 128 + (r % 8) * 16 + (k % 8) * 2 bytes;
// the descriptors give the step between core matrices along K (128 B) and
// along R ((K / 8) * 128 B).
#include <cuda_bf16.h>
#include <math.h>

#include "pic_internal.h"
#include "push_device.cuh"

namespace pic {
namespace {

constexpr int kTcRows = 128;  // particles per tile (MMA M)
constexpr int kTcTiles = 1;   // tiles per CTA
constexpr int kTcThreads = kTcRows * kTcTiles;
constexpr int kTcH = 64, kTcIn = 6, kTcOut = 8;
constexpr uint32_t kTileCols = 64;  // TMEM columns per tile: D1, then D2, then D3
constexpr uint32_t kTmemCols = kTileCols * kTcTiles;

struct TcSmem {
  __align__(1024) unsigned char W1[kTcH * 16 * 2];    // [64 x 16]
  __align__(1024) unsigned char W2[kTcH * kTcH * 2];  // [64 x 64]
  __align__(1024) unsigned char W3[16 * kTcH * 2];    // [16 x 64], rows 8..15 zero
  // [128 x 64] per tile; its first 4 KB are also A1 [128 x 16] (layer 1's input)
  __align__(1024) unsigned char A2[kTcTiles][kTcRows * kTcH * 2];
  float b1[kTcH], b2[kTcH], b3[kTcOut];
  __align__(8) uint64_t bar;
  uint32_t tmem;
  int failed;
};
// Reserved per CTA (with the slack for aligning the buffers to 1 KB): seven
// CTAs fit an SM's 228 KB of shared memory and no more, and seven 64-column
// TMEM allocations fit its 512 columns, so an allocation never waits.
constexpr int kTcCtasPerSm = 7;
constexpr size_t kTcSmemBytes = sizeof(TcSmem) + 1024;
static_assert(kTcCtasPerSm * (kTcSmemBytes + 1024) <= 228 * 1024, "seven CTAs fit shared memory");
static_assert(8 * (kTcSmemBytes + 1024) > 228 * 1024, "an eighth CTA does not: TMEM stays within 512 columns");
static_assert(kTcCtasPerSm * kTmemCols <= 512, "TMEM columns of the resident CTAs");

__device__ __forceinline__ uint32_t saddr(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ uint32_t cm_off(int r, int k, int K) {
  return (uint32_t)(r >> 3) * (uint32_t)(K / 8) * 128u + (uint32_t)(k >> 3) * 128u +
         (uint32_t)(r & 7) * 16u + (uint32_t)(k & 7) * 2u;
}

// Shared-memory matrix descriptor (no swizzle): start address, the byte step
// between core matrices along K (leading) and along the rows (stride), and the
// descriptor version of this architecture.
__device__ __forceinline__ uint64_t sdesc(uint32_t addr, uint32_t k_step, uint32_t r_step) {
  uint64_t d = 0;
  d |= (uint64_t)((addr >> 4) & 0x3FFFu);
  d |= (uint64_t)((k_step >> 4) & 0x3FFFu) << 16;
  d |= (uint64_t)((r_step >> 4) & 0x3FFFu) << 32;
  d |= (uint64_t)1 << 46;
  return d;
}

// Instruction descriptor of kind::f16: FP32 accumulator, BF16 A and B, both
// K-major, N and M.
__host__ __device__ constexpr uint32_t idesc_bf16(int M, int N) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ void mma_bf16(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t idesc,
                                         int accumulate) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(d_tmem),
      "l"(a), "l"(b), "r"(idesc), "r"(accumulate));
}
__device__ __forceinline__ void mma_commit(uint64_t* bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(saddr(bar))
               : "memory");
}
__device__ __forceinline__ void fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

// Bounded wait for phase `parity` of the barrier: false = gave up.
__device__ __forceinline__ bool bar_wait(uint64_t* bar, uint32_t parity) {
  for (uint32_t it = 0; it < (1u << 22); ++it) {
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
        " selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(saddr(bar)), "r"(parity)
        : "memory");
    if (ok) return true;
  }
  return false;
}

// 16 consecutive FP32 accumulator columns of this thread's TMEM lane.
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float (&v)[16]) {
  uint32_t r[16];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int q = 0; q < 16; ++q) v[q] = __uint_as_float(r[q]);
}

__device__ __forceinline__ uint32_t bf2(float lo, float hi) {
  __nv_bfloat162 v = __floats2bfloat162_rn(lo, hi);
  return *reinterpret_cast<uint32_t*>(&v);
}

// max(lo, 0), max(hi, 0) rounded to BF16 and packed (lo in the low half): the
// conversion's relu clamps a negative value to zero, in one instruction.
__device__ __forceinline__ uint32_t bf2_relu(float lo, float hi) {
  uint32_t d;
  asm("cvt.rn.relu.bf16x2.f32 %0, %1, %2;" : "=r"(d) : "f"(hi), "f"(lo));
  return d;
}

// Packed FP32 master parameters (W1[64][6] b1[64] W2[64][64] b2[64] W3[8][64]
// b3[8]) to BF16 operand tiles and FP32 biases.
__device__ void tc_load_weights(TcSmem& s, const float* P) {
  const float* W1 = P;
  const float* b1 = W1 + kTcH * kTcIn;
  const float* W2 = b1 + kTcH;
  const float* b2 = W2 + kTcH * kTcH;
  const float* W3 = b2 + kTcH;
  const float* b3 = W3 + kTcOut * kTcH;
  for (int e = threadIdx.x; e < kTcH * 16; e += blockDim.x) {
    const int o = e / 16, i = e % 16;
    *reinterpret_cast<__nv_bfloat16*>(s.W1 + cm_off(o, i, 16)) =
        __float2bfloat16_rn(i < kTcIn ? W1[o * kTcIn + i] : 0.0f);
  }
  for (int e = threadIdx.x; e < kTcH * kTcH; e += blockDim.x) {
    const int o = e / kTcH, i = e % kTcH;
    *reinterpret_cast<__nv_bfloat16*>(s.W2 + cm_off(o, i, kTcH)) = __float2bfloat16_rn(W2[e]);
  }
  for (int e = threadIdx.x; e < 16 * kTcH; e += blockDim.x) {
    const int o = e / kTcH, i = e % kTcH;
    *reinterpret_cast<__nv_bfloat16*>(s.W3 + cm_off(o, i, kTcH)) =
        __float2bfloat16_rn(o < kTcOut ? W3[o * kTcH + i] : 0.0f);
  }
  for (int e = threadIdx.x; e < kTcH; e += blockDim.x) {
    s.b1[e] = b1[e];
    s.b2[e] = b2[e];
  }
  if (threadIdx.x < kTcOut) s.b3[threadIdx.x] = b3[threadIdx.x];
}

// Row r of tile q's A1 (the start of A2) from this thread's features (BF16,
// columns 6..15 zero).
__device__ __forceinline__ void put_features(TcSmem& s, int q, int r, const float (&f)[6]) {
  uint4 lo, hi;
  lo.x = bf2(f[0], f[1]);
  lo.y = bf2(f[2], f[3]);
  lo.z = bf2(f[4], f[5]);
  lo.w = 0u;
  hi = make_uint4(0u, 0u, 0u, 0u);
  *reinterpret_cast<uint4*>(s.A2[q] + cm_off(r, 0, 16)) = lo;
  *reinterpret_cast<uint4*>(s.A2[q] + cm_off(r, 8, 16)) = hi;
}

// Hidden layer epilogue: accumulator columns [c0, c0 + 64) of row r, plus
// bias, ReLU, BF16, into row r of tile q's A2.
__device__ __forceinline__ void hidden_epilogue(TcSmem& s, uint32_t lane_addr, int c0,
                                                const float* bias, int q, int r) {
#pragma unroll
  for (int blk = 0; blk < 4; ++blk) {
    float v[16];
    tmem_ld16(lane_addr + (uint32_t)(c0 + 16 * blk), v);
    const float2* b2 = reinterpret_cast<const float2*>(bias + 16 * blk);
    uint32_t w[8];
#pragma unroll
    for (int q = 0; q < 8; ++q) {  // bias in paired FP32 adds, ReLU in the BF16 conversion
      const float2 t = add2(make_float2(v[2 * q], v[2 * q + 1]), b2[q]);
      w[q] = bf2_relu(t.x, t.y);
    }
    uint4 w0 = make_uint4(w[0], w[1], w[2], w[3]);
    uint4 w1 = make_uint4(w[4], w[5], w[6], w[7]);
    *reinterpret_cast<uint4*>(s.A2[q] + cm_off(r, 16 * blk, kTcH)) = w0;
    *reinterpret_cast<uint4*>(s.A2[q] + cm_off(r, 16 * blk + 8, kTcH)) = w1;
  }
}

// The network on the CTA's two tiles; this thread carries the features f of
// row r of tile q (thread t: q = t / 128, r = t % 128), which is also the row
// its warp reads back (warp w: TMEM lanes 32 (w % 4) .. + 31 of tile w / 4).
// Returns the class (argmax, ties to the smaller k) or 0xFF after a give-up.
// Collective over the CTA.  `ph` is the mbarrier phase, advanced per commit.
__device__ __forceinline__ int tc_tiles(TcSmem& s, const float (&f)[6], uint32_t& ph) {
  const int q = threadIdx.x >> 7, r = threadIdx.x & 127;
  const int warp = threadIdx.x >> 5;
  put_features(s, q, r, f);
  fence_async_smem();
  fence_before();
  __syncthreads();
  fence_after();
  const uint32_t col0 = kTileCols * (uint32_t)q;
  const uint32_t lane_addr = s.tmem + ((uint32_t)(32 * (warp & 3)) << 16) + col0;
  bool ok = !s.failed;
  // layer 1
  if (ok && threadIdx.x == 0) {
#pragma unroll
    for (int t = 0; t < kTcTiles; ++t)
      mma_bf16(s.tmem + kTileCols * t, sdesc(saddr(s.A2[t]), 128, 256), sdesc(saddr(s.W1), 128, 256),
               idesc_bf16(kTcRows, kTcH), 0);
    mma_commit(&s.bar);
    if (!bar_wait(&s.bar, ph) && !bar_wait(&s.bar, ph)) s.failed = 1;  // gives up after two waits
  }
  ph ^= 1u;
  __syncthreads();  // the MMAs have completed (or the wait gave up) for every thread
  fence_after();
  ok = !s.failed;
  if (ok) hidden_epilogue(s, lane_addr, 0, s.b1, q, r);
  fence_async_smem();
  fence_before();
  if (!ok) s.failed = 1;
  __syncthreads();
  fence_after();
  ok = !s.failed;
  // layer 2
  if (ok && threadIdx.x == 0) {
#pragma unroll
    for (int t = 0; t < kTcTiles; ++t)
#pragma unroll
      for (int k = 0; k < 4; ++k)
        mma_bf16(s.tmem + kTileCols * t, sdesc(saddr(s.A2[t]) + 256u * k, 128, 1024),
                 sdesc(saddr(s.W2) + 256u * k, 128, 1024), idesc_bf16(kTcRows, kTcH), k > 0);
    mma_commit(&s.bar);
    if (!bar_wait(&s.bar, ph) && !bar_wait(&s.bar, ph)) s.failed = 1;  // gives up after two waits
  }
  ph ^= 1u;
  __syncthreads();
  fence_after();
  ok = !s.failed;
  if (ok) hidden_epilogue(s, lane_addr, 0, s.b2, q, r);
  fence_async_smem();
  fence_before();
  if (!ok) s.failed = 1;
  __syncthreads();
  fence_after();
  ok = !s.failed;
  // layer 3
  if (ok && threadIdx.x == 0) {
#pragma unroll
    for (int t = 0; t < kTcTiles; ++t)
#pragma unroll
      for (int k = 0; k < 4; ++k)
        mma_bf16(s.tmem + kTileCols * t, sdesc(saddr(s.A2[t]) + 256u * k, 128, 1024),
                 sdesc(saddr(s.W3) + 256u * k, 128, 1024), idesc_bf16(kTcRows, 16), k > 0);
    mma_commit(&s.bar);
    if (!bar_wait(&s.bar, ph) && !bar_wait(&s.bar, ph)) s.failed = 1;  // gives up after two waits
  }
  ph ^= 1u;
  __syncthreads();
  fence_after();
  ok = !s.failed;
  int cls = 0xFF;
  if (ok) {
    float z[16];
    tmem_ld16(lane_addr, z);
    float best = z[0] + s.b3[0];
    cls = 0;
#pragma unroll
    for (int c = 1; c < kTcOut; ++c) {
      const float v = z[c] + s.b3[c];
      if (v > best) { best = v; cls = c; }
    }
  }
  fence_before();
  if (!ok) s.failed = 1;
  __syncthreads();  // A1, A2 and the TMEM columns are reused by the next tiles
  fence_after();
  return s.failed ? 0xFF : cls;
}

__device__ __forceinline__ void tc_begin(TcSmem& s, const float* P) {
  tc_load_weights(s, P);
  if (threadIdx.x < 32) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(saddr(&s.tmem)),
                 "r"(kTmemCols));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  if (threadIdx.x == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(saddr(&s.bar)));
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    s.failed = 0;
  }
  fence_async_smem();
  fence_before();
  __syncthreads();
  fence_after();
}

__device__ __forceinline__ void tc_end(TcSmem& s) {
  fence_before();
  __syncthreads();
  fence_after();
  if (threadIdx.x < 32)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(s.tmem), "r"(kTmemCols));
}

}  // namespace

// pic_predict: features of every particle after step a (a.halfE / a.halfB: its
// feature nodes; the same code as the features kernel) and the network's
// class, in one pass.
template <int P>
__global__ void __launch_bounds__(kTcThreads) predict_tc_kernel(PushArgsMixed a, const float* Pm, uint8_t* pred,
                                                                int fieldless_zero) {
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  TcSmem& s = *reinterpret_cast<TcSmem*>(smem_raw + ((1024 - (saddr(smem_raw) & 1023)) & 1023));
  tc_begin(s, Pm);
  uint32_t ph = 0;
  const int64_t n_groups = (a.n + kTcThreads - 1) / kTcThreads;
  // each tile's particle loads are issued before the previous tile's network
  // runs, so their DRAM latency overlaps the MMA round trips
  int64_t t = blockIdx.x;
  FeatureInput cur = feature_input(a, t * kTcThreads + threadIdx.x);
  for (; t < n_groups; t += gridDim.x) {
    const int64_t i = t * kTcThreads + threadIdx.x;
    const int64_t tn = t + gridDim.x;
    const FeatureInput nxt = feature_input(a, tn < n_groups ? tn * kTcThreads + threadIdx.x : a.n);
    float f[6];
    features_of(a, a.halfE, a.halfB, a.lo, a.hi, cur, f);
    // no field at the particle: no rotation, the criterion takes k = 0
    const bool fieldless = fieldless_zero && f[0] == 0.f && f[1] == 0.f;
    int c = 0;
    if (__syncthreads_or(!fieldless)) c = tc_tiles(s, f, ph);  // uniform over the CTA
    if (fieldless && c != 0xFF) c = 0;
    if (i < a.n) pred[i] = (uint8_t)c;
    if (s.failed) break;
    cur = nxt;
  }
  if (s.failed && threadIdx.x == 0 && a.stats) atomicExch(&a.stats->error, 2);
  tc_end(s);
}

// pic_mlp_infer: the network's class of n feature rows phi[n][6].
__global__ void __launch_bounds__(kTcThreads) mlp_infer_tc_kernel(const float* Pm, const float* phi,
                                                                  int64_t n, uint8_t* pred) {
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  TcSmem& s = *reinterpret_cast<TcSmem*>(smem_raw + ((1024 - (saddr(smem_raw) & 1023)) & 1023));
  tc_begin(s, Pm);
  uint32_t ph = 0;
  const int64_t n_groups = (n + kTcThreads - 1) / kTcThreads;
  for (int64_t t = blockIdx.x; t < n_groups; t += gridDim.x) {
    const int64_t i = t * kTcThreads + threadIdx.x;
    float f[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
    if (i < n) {
#pragma unroll
      for (int q = 0; q < 6; ++q) f[q] = phi[i * 6 + q];
    }
    const int c = tc_tiles(s, f, ph);
    if (i < n) pred[i] = (uint8_t)c;
    if (s.failed) break;
  }
  tc_end(s);
}

static int tc_grid(int64_t n, int sm_count) {
  const int64_t groups = (n + kTcThreads - 1) / kTcThreads;
  const int64_t cap = (int64_t)(sm_count > 0 ? sm_count : 152) * kTcCtasPerSm;
  return (int)(groups < cap ? groups : cap);
}

template <class K>
static cudaError_t tc_configure(K kernel) {
  return cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kTcSmemBytes);
}

cudaError_t launch_predict_fused(const PushArgsMixed& a, int order, const float* P, uint8_t* pred,
                                 int sm_count, cudaStream_t st, bool fieldless_zero) {
  const int fz = fieldless_zero ? 1 : 0;
  if (a.n <= 0) return cudaSuccess;
  const int blocks = tc_grid(a.n, sm_count);
  cudaError_t e = cudaSuccess;
  switch (order) {
    case 1: e = tc_configure(predict_tc_kernel<1>); if (e == cudaSuccess) predict_tc_kernel<1><<<blocks, kTcThreads, kTcSmemBytes, st>>>(a, P, pred, fz); break;
    case 2: e = tc_configure(predict_tc_kernel<2>); if (e == cudaSuccess) predict_tc_kernel<2><<<blocks, kTcThreads, kTcSmemBytes, st>>>(a, P, pred, fz); break;
    case 3: e = tc_configure(predict_tc_kernel<3>); if (e == cudaSuccess) predict_tc_kernel<3><<<blocks, kTcThreads, kTcSmemBytes, st>>>(a, P, pred, fz); break;
    case 4: e = tc_configure(predict_tc_kernel<4>); if (e == cudaSuccess) predict_tc_kernel<4><<<blocks, kTcThreads, kTcSmemBytes, st>>>(a, P, pred, fz); break;
    case 5: e = tc_configure(predict_tc_kernel<5>); if (e == cudaSuccess) predict_tc_kernel<5><<<blocks, kTcThreads, kTcSmemBytes, st>>>(a, P, pred, fz); break;
    default: return cudaErrorInvalidValue;
  }
  if (e != cudaSuccess) return e;
  return cudaGetLastError();
}

cudaError_t launch_mlp_infer(const float* P, const float* phi, int64_t n, uint8_t* pred,
                             int sm_count, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  cudaError_t e = tc_configure(mlp_infer_tc_kernel);
  if (e != cudaSuccess) return e;
  mlp_infer_tc_kernel<<<tc_grid(n, sm_count), kTcThreads, kTcSmemBytes, s>>>(P, phi, n, pred);
  return cudaGetLastError();
}

}  // namespace pic
