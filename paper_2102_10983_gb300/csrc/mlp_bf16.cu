// Learned sub-cycle-count predictor: MLP 6 -> 64 -> 64 -> 8 (ReLU, softmax
// cross-entropy over k = 0..7), BF16 operands with FP32 accumulation.
//
// Not part of the paper: it only predicts, per particle, the exponent k the
// criterion of Sec. IV will choose at the next macro step, so that the push can
// bin work before launch.  The criterion still decides every sub-step.
//
// Row-vector convention: h1 = relu(phi W1^T + b1), h2 = relu(h1 W2^T + b2),
// z = h2 W3^T + b3; W_l is (out, in).  phi = (asinh|E|, asinh|B|, asinh p_x,
// asinh p_y, asinh p_z, log gamma).
//
// Training (this file): warp-level mma.sync m16n8k16 (BF16 in, FP32
// accumulate), 16 samples per warp tile.  A layer's accumulator fragments are,
// after bias and ReLU, exactly the next layer's A fragments, so hidden
// activations never leave registers in the forward pass.  Backward: dz on the
// CUDA cores, dh2 = dz W3 and dh1 = da2 W2 on the tensor cores, weight
// gradients (batch reductions) from BF16-rounded operands with FP32
// accumulation in shared memory.  Inference (mlp_tc.cu) runs on tcgen05 with
// TMEM accumulators.
#include <cuda_bf16.h>
#include <math.h>

#include "pic_internal.h"
#include "push_device.cuh"

namespace pic {

namespace {

constexpr int kH = 64, kIn = 6, kOut = 8, kK1 = 16;
// Row strides (BF16 elements) of the weight tiles in shared memory, padded so
// that the eight rows a warp's B-fragment loads touch at once fall in distinct
// banks (a 64-element row is 128 bytes: unpadded, those eight loads conflict).
constexpr int kS1 = 24, kS2 = 72;

__device__ __forceinline__ uint32_t pack2(float lo, float hi) {
  __nv_bfloat162 v = __floats2bfloat162_rn(lo, hi);
  return *reinterpret_cast<uint32_t*>(&v);
}
__device__ __forceinline__ float bf(float x) { return __bfloat162float(__float2bfloat16_rn(x)); }

__device__ __forceinline__ void mma16816(float (&d)[4], const uint32_t (&a)[4], uint32_t b0,
                                         uint32_t b1) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, "
      "{%8,%9}, {%0,%1,%2,%3};\n"
      : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

// Weights as the kernels read them from shared memory (BF16):
//   W1p [64][16] (cols 6..15 zero), W2 [64][64], W2T [64][64], W3 [8][64] (rows at the
//   padded strides kS1, kS2), W3T [64][8],
// and the FP32 biases.
struct SmemW {
  __nv_bfloat16 W1p[kH * kS1];
  __nv_bfloat16 W2[kH * kS2];
  __nv_bfloat16 W2T[kH * kS2];
  __nv_bfloat16 W3[kOut * kS2];
  __nv_bfloat16 W3T[kH * kOut];
  float b1[kH], b2[kH], b3[kOut];
};

__device__ void load_weights(SmemW& s, const float* P) {
  // packed FP32 master: W1[64][6] b1[64] W2[64][64] b2[64] W3[8][64] b3[8]
  const float* W1 = P;
  const float* b1 = W1 + kH * kIn;
  const float* W2 = b1 + kH;
  const float* b2 = W2 + kH * kH;
  const float* W3 = b2 + kH;
  const float* b3 = W3 + kOut * kH;
  for (int e = threadIdx.x; e < kH * kK1; e += blockDim.x) {
    const int o = e / kK1, i = e % kK1;
    s.W1p[o * kS1 + i] = __float2bfloat16_rn(i < kIn ? W1[o * kIn + i] : 0.0f);
  }
  for (int e = threadIdx.x; e < kH * kH; e += blockDim.x) {
    const int o = e / kH, i = e % kH;
    s.W2[o * kS2 + i] = __float2bfloat16_rn(W2[e]);
    s.W2T[i * kS2 + o] = __float2bfloat16_rn(W2[e]);
  }
  for (int e = threadIdx.x; e < kOut * kH; e += blockDim.x) {
    const int o = e / kH, i = e % kH;
    s.W3[o * kS2 + i] = __float2bfloat16_rn(W3[e]);
    s.W3T[i * kOut + o] = __float2bfloat16_rn(W3[e]);
  }
  for (int e = threadIdx.x; e < kH; e += blockDim.x) {
    s.b1[e] = b1[e];
    s.b2[e] = b2[e];
  }
  if (threadIdx.x < kOut) s.b3[threadIdx.x] = b3[threadIdx.x];
}

__device__ __forceinline__ uint32_t ld32(const __nv_bfloat16* p) {
  return *reinterpret_cast<const uint32_t*>(p);
}
// Forward of one 16-row tile.  a1: layer-1 input fragment.  Outputs the
// pre-activations (kept for the backward pass) and the logits.
struct Fwd {
  float acc1[8][4];  // a1 = phi W1^T + b1 (pre-ReLU)
  float acc2[8][4];  // a2
  float z[4];        // logits, rows (g, g+8), cols 2t, 2t+1
};

__device__ __forceinline__ void forward_tile(const SmemW& s, const uint32_t (&a1)[4], Fwd& f) {
  const int lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
#pragma unroll
  for (int nt = 0; nt < 8; ++nt) {
    const float bl = s.b1[8 * nt + 2 * t], bh = s.b1[8 * nt + 2 * t + 1];
    f.acc1[nt][0] = bl; f.acc1[nt][1] = bh; f.acc1[nt][2] = bl; f.acc1[nt][3] = bh;
    const __nv_bfloat16* w = s.W1p + (8 * nt + g) * kS1;
    mma16816(f.acc1[nt], a1, ld32(w + 2 * t), ld32(w + 2 * t + 8));
  }
  uint32_t a2[4][4];
#pragma unroll
  for (int kc = 0; kc < 4; ++kc) {
    a2[kc][0] = pack2(fmaxf(f.acc1[2 * kc][0], 0.f), fmaxf(f.acc1[2 * kc][1], 0.f));
    a2[kc][1] = pack2(fmaxf(f.acc1[2 * kc][2], 0.f), fmaxf(f.acc1[2 * kc][3], 0.f));
    a2[kc][2] = pack2(fmaxf(f.acc1[2 * kc + 1][0], 0.f), fmaxf(f.acc1[2 * kc + 1][1], 0.f));
    a2[kc][3] = pack2(fmaxf(f.acc1[2 * kc + 1][2], 0.f), fmaxf(f.acc1[2 * kc + 1][3], 0.f));
  }
#pragma unroll
  for (int nt = 0; nt < 8; ++nt) {
    const float bl = s.b2[8 * nt + 2 * t], bh = s.b2[8 * nt + 2 * t + 1];
    f.acc2[nt][0] = bl; f.acc2[nt][1] = bh; f.acc2[nt][2] = bl; f.acc2[nt][3] = bh;
    const __nv_bfloat16* w = s.W2 + (8 * nt + g) * kS2;
#pragma unroll
    for (int kc = 0; kc < 4; ++kc)
      mma16816(f.acc2[nt], a2[kc], ld32(w + 16 * kc + 2 * t), ld32(w + 16 * kc + 2 * t + 8));
  }
  uint32_t a3[4][4];
#pragma unroll
  for (int kc = 0; kc < 4; ++kc) {
    a3[kc][0] = pack2(fmaxf(f.acc2[2 * kc][0], 0.f), fmaxf(f.acc2[2 * kc][1], 0.f));
    a3[kc][1] = pack2(fmaxf(f.acc2[2 * kc][2], 0.f), fmaxf(f.acc2[2 * kc][3], 0.f));
    a3[kc][2] = pack2(fmaxf(f.acc2[2 * kc + 1][0], 0.f), fmaxf(f.acc2[2 * kc + 1][1], 0.f));
    a3[kc][3] = pack2(fmaxf(f.acc2[2 * kc + 1][2], 0.f), fmaxf(f.acc2[2 * kc + 1][3], 0.f));
  }
  const float bl = s.b3[2 * t], bh = s.b3[2 * t + 1];
  f.z[0] = bl; f.z[1] = bh; f.z[2] = bl; f.z[3] = bh;
  const __nv_bfloat16* w = s.W3 + g * kS2;
#pragma unroll
  for (int kc = 0; kc < 4; ++kc)
    mma16816(f.z, a3[kc], ld32(w + 16 * kc + 2 * t), ld32(w + 16 * kc + 2 * t + 8));
}

// Layer-1 fragment from an FP32 feature array phi[n][6] (rows >= n are zero).
__device__ __forceinline__ void phi_fragment(const float* phi, int64_t n, int64_t base,
                                             uint32_t (&a1)[4]) {
  const int lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
  float v[4] = {0.f, 0.f, 0.f, 0.f};
  if (t < 3) {
    if (base + g < n) { v[0] = phi[(base + g) * kIn + 2 * t]; v[1] = phi[(base + g) * kIn + 2 * t + 1]; }
    if (base + g + 8 < n) { v[2] = phi[(base + g + 8) * kIn + 2 * t]; v[3] = phi[(base + g + 8) * kIn + 2 * t + 1]; }
  }
  a1[0] = pack2(v[0], v[1]);
  a1[1] = pack2(v[2], v[3]);
  a1[2] = 0u;
  a1[3] = 0u;
}

}  // namespace

// ---------------------------------------------------------------- training (gradients)

struct WarpStage {
  float X[16][8];
  float h1[16][kH];
  float h2[16][kH];
  float dz[16][kOut];
  float da2[16][kH];
  float da1[16][kH];
};

// Per-block gradient accumulator, same packed order as the parameters.
constexpr int kNParams = kH * kIn + kH + kH * kH + kH + kOut * kH + kOut;

__global__ void __launch_bounds__(128) mlp_grad_kernel(const float* P, const float* phi,
                                                       const uint8_t* label, int64_t n,
                                                       float inv_batch, float* grad, float* loss) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  SmemW& s = *reinterpret_cast<SmemW*>(smem_raw);
  WarpStage* stage = reinterpret_cast<WarpStage*>(smem_raw + ((sizeof(SmemW) + 15) & ~(size_t)15));
  float* acc = reinterpret_cast<float*>(stage + (blockDim.x >> 5));  // kNParams floats
  load_weights(s, P);
  for (int e = threadIdx.x; e < kNParams; e += blockDim.x) acc[e] = 0.f;
  __syncthreads();
  const int lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3, warp = threadIdx.x >> 5;
  WarpStage& S = stage[warp];
  float* gW1 = acc;
  float* gb1 = gW1 + kH * kIn;
  float* gW2 = gb1 + kH;
  float* gb2 = gW2 + kH * kH;
  float* gW3 = gb2 + kH;
  float* gb3 = gW3 + kOut * kH;
  float my_loss = 0.f;
  const int64_t warps = (int64_t)gridDim.x * (blockDim.x >> 5);
  for (int64_t tile = blockIdx.x * (int64_t)(blockDim.x >> 5) + warp; tile * 16 < n; tile += warps) {
    const int64_t base = tile * 16;
    uint32_t a1[4];
    phi_fragment(phi, n, base, a1);
    Fwd f;
    forward_tile(s, a1, f);
    const bool r0 = base + g < n, r1 = base + g + 8 < n;
    // softmax cross-entropy; dz = (softmax - onehot) / batch
    float m0 = fmaxf(f.z[0], f.z[1]), m1 = fmaxf(f.z[2], f.z[3]);
    for (int o = 1; o <= 2; o <<= 1) {
      m0 = fmaxf(m0, __shfl_xor_sync(0xffffffffu, m0, o));
      m1 = fmaxf(m1, __shfl_xor_sync(0xffffffffu, m1, o));
    }
    const float e0 = __expf(f.z[0] - m0), e1 = __expf(f.z[1] - m0);
    const float e2 = __expf(f.z[2] - m1), e3 = __expf(f.z[3] - m1);
    float s0 = e0 + e1, s1 = e2 + e3;
    for (int o = 1; o <= 2; o <<= 1) {
      s0 += __shfl_xor_sync(0xffffffffu, s0, o);
      s1 += __shfl_xor_sync(0xffffffffu, s1, o);
    }
    const int y0 = r0 ? label[base + g] : -1, y1 = r1 ? label[base + g + 8] : -1;
    float dz[4];
    dz[0] = r0 ? (e0 / s0 - (y0 == 2 * t ? 1.f : 0.f)) * inv_batch : 0.f;
    dz[1] = r0 ? (e1 / s0 - (y0 == 2 * t + 1 ? 1.f : 0.f)) * inv_batch : 0.f;
    dz[2] = r1 ? (e2 / s1 - (y1 == 2 * t ? 1.f : 0.f)) * inv_batch : 0.f;
    dz[3] = r1 ? (e3 / s1 - (y1 == 2 * t + 1 ? 1.f : 0.f)) * inv_batch : 0.f;
    if (r0 && (y0 >> 1) == t) my_loss += logf(s0) - (f.z[y0 & 1] - m0);
    if (r1 && (y1 >> 1) == t) my_loss += logf(s1) - (f.z[2 + (y1 & 1)] - m1);
    // dh2 = dz W3 (K = 8 classes, padded to 16): B[k][n] = W3[k][n] = W3T[n][k]
    uint32_t adz[4] = {pack2(dz[0], dz[1]), pack2(dz[2], dz[3]), 0u, 0u};
    float dh2[8][4];
#pragma unroll
    for (int nt = 0; nt < 8; ++nt) {
      dh2[nt][0] = dh2[nt][1] = dh2[nt][2] = dh2[nt][3] = 0.f;
      mma16816(dh2[nt], adz, ld32(s.W3T + (8 * nt + g) * kOut + 2 * t), 0u);
    }
    // da2 = dh2 * (a2 > 0); dh1 = da2 W2: B[k][n] = W2[k][n] = W2T[n][k]
    float da2[8][4];
#pragma unroll
    for (int nt = 0; nt < 8; ++nt)
#pragma unroll
      for (int q = 0; q < 4; ++q) da2[nt][q] = f.acc2[nt][q] > 0.f ? dh2[nt][q] : 0.f;
    uint32_t ada2[4][4];
#pragma unroll
    for (int kc = 0; kc < 4; ++kc) {
      ada2[kc][0] = pack2(da2[2 * kc][0], da2[2 * kc][1]);
      ada2[kc][1] = pack2(da2[2 * kc][2], da2[2 * kc][3]);
      ada2[kc][2] = pack2(da2[2 * kc + 1][0], da2[2 * kc + 1][1]);
      ada2[kc][3] = pack2(da2[2 * kc + 1][2], da2[2 * kc + 1][3]);
    }
    float dh1[8][4];
#pragma unroll
    for (int nt = 0; nt < 8; ++nt) {
      dh1[nt][0] = dh1[nt][1] = dh1[nt][2] = dh1[nt][3] = 0.f;
      const __nv_bfloat16* w = s.W2T + (8 * nt + g) * kS2;
#pragma unroll
      for (int kc = 0; kc < 4; ++kc)
        mma16816(dh1[nt], ada2[kc], ld32(w + 16 * kc + 2 * t), ld32(w + 16 * kc + 2 * t + 8));
    }
    // stage the tile (BF16-rounded operands) for the weight-gradient reductions
#pragma unroll
    for (int nt = 0; nt < 8; ++nt) {
      const int c = 8 * nt + 2 * t;
      S.h1[g][c] = bf(fmaxf(f.acc1[nt][0], 0.f));
      S.h1[g][c + 1] = bf(fmaxf(f.acc1[nt][1], 0.f));
      S.h1[g + 8][c] = bf(fmaxf(f.acc1[nt][2], 0.f));
      S.h1[g + 8][c + 1] = bf(fmaxf(f.acc1[nt][3], 0.f));
      S.h2[g][c] = bf(fmaxf(f.acc2[nt][0], 0.f));
      S.h2[g][c + 1] = bf(fmaxf(f.acc2[nt][1], 0.f));
      S.h2[g + 8][c] = bf(fmaxf(f.acc2[nt][2], 0.f));
      S.h2[g + 8][c + 1] = bf(fmaxf(f.acc2[nt][3], 0.f));
      S.da2[g][c] = bf(da2[nt][0]);
      S.da2[g][c + 1] = bf(da2[nt][1]);
      S.da2[g + 8][c] = bf(da2[nt][2]);
      S.da2[g + 8][c + 1] = bf(da2[nt][3]);
      S.da1[g][c] = bf(f.acc1[nt][0] > 0.f ? dh1[nt][0] : 0.f);
      S.da1[g][c + 1] = bf(f.acc1[nt][1] > 0.f ? dh1[nt][1] : 0.f);
      S.da1[g + 8][c] = bf(f.acc1[nt][2] > 0.f ? dh1[nt][2] : 0.f);
      S.da1[g + 8][c + 1] = bf(f.acc1[nt][3] > 0.f ? dh1[nt][3] : 0.f);
    }
    S.dz[g][2 * t] = bf(dz[0]);
    S.dz[g][2 * t + 1] = bf(dz[1]);
    S.dz[g + 8][2 * t] = bf(dz[2]);
    S.dz[g + 8][2 * t + 1] = bf(dz[3]);
    {
      const __nv_bfloat162 x0 = *reinterpret_cast<const __nv_bfloat162*>(&a1[0]);
      const __nv_bfloat162 x1 = *reinterpret_cast<const __nv_bfloat162*>(&a1[1]);
      S.X[g][2 * t] = __bfloat162float(x0.x);
      S.X[g][2 * t + 1] = __bfloat162float(x0.y);
      S.X[g + 8][2 * t] = __bfloat162float(x1.x);
      S.X[g + 8][2 * t + 1] = __bfloat162float(x1.y);
    }
    __syncwarp();
    // weight gradients: sum over the 16 rows, FP32 accumulation (shared atomics
    // because the block's warps share one accumulator)
    for (int e = lane; e < kOut * kH; e += 32) {
      const int o = e / kH, i = e % kH;
      float a = 0.f;
#pragma unroll
      for (int m = 0; m < 16; ++m) a = fmaf(S.dz[m][o], S.h2[m][i], a);
      atomicAdd(&gW3[e], a);
    }
    if (lane < kOut) {
      float a = 0.f;
      for (int m = 0; m < 16; ++m) a += S.dz[m][lane];
      atomicAdd(&gb3[lane], a);
    }
    for (int e = lane; e < kH * kH; e += 32) {
      const int o = e / kH, i = e % kH;
      float a = 0.f;
#pragma unroll
      for (int m = 0; m < 16; ++m) a = fmaf(S.da2[m][o], S.h1[m][i], a);
      atomicAdd(&gW2[e], a);
    }
    for (int e = lane; e < kH * kIn; e += 32) {
      const int o = e / kIn, i = e % kIn;
      float a = 0.f;
#pragma unroll
      for (int m = 0; m < 16; ++m) a = fmaf(S.da1[m][o], S.X[m][i], a);
      atomicAdd(&gW1[e], a);
    }
    for (int o = lane; o < kH; o += 32) {
      float a = 0.f, b = 0.f;
      for (int m = 0; m < 16; ++m) {
        a += S.da2[m][o];
        b += S.da1[m][o];
      }
      atomicAdd(&gb2[o], a);
      atomicAdd(&gb1[o], b);
    }
    __syncwarp();
  }
  for (int o = 16; o > 0; o >>= 1) my_loss += __shfl_xor_sync(0xffffffffu, my_loss, o);
  if (lane == 0 && my_loss != 0.f) atomicAdd(loss, my_loss * inv_batch);
  __syncthreads();
  for (int e = threadIdx.x; e < kNParams; e += blockDim.x)
    if (acc[e] != 0.f) atomicAdd(&grad[e], acc[e]);
}

// Adam on the FP32 master parameters.
__global__ void mlp_adam_kernel(float* P, const float* grad, float* m1, float* m2, float lr,
                                float beta1, float beta2, float eps, float bc1, float bc2) {
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < kNParams; e += gridDim.x * blockDim.x) {
    const float gr = grad[e];
    const float a = beta1 * m1[e] + (1.f - beta1) * gr;
    const float b = beta2 * m2[e] + (1.f - beta2) * gr * gr;
    m1[e] = a;
    m2[e] = b;
    P[e] -= lr * (a / bc1) / (sqrtf(b / bc2) + eps);
  }
}

int mlp_param_count() { return kNParams; }

size_t mlp_grad_smem(int warps) {
  return ((sizeof(SmemW) + 15) & ~(size_t)15) + (size_t)warps * sizeof(WarpStage) +
         (size_t)kNParams * sizeof(float);
}

cudaError_t launch_mlp_grad(const float* P, const float* phi, const uint8_t* label, int64_t n,
                            float* grad, float* loss, int sm_count, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  const size_t smem = mlp_grad_smem(4);
  static bool configured = false;
  if (!configured) {
    cudaError_t e = cudaFuncSetAttribute(mlp_grad_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem);
    if (e != cudaSuccess) return e;
    configured = true;
  }
  const int64_t tiles = (n + 15) / 16;
  int64_t blocks = (tiles + 3) / 4;
  const int64_t cap = (int64_t)(sm_count > 0 ? sm_count : 152);
  if (blocks > cap) blocks = cap;
  mlp_grad_kernel<<<(int)blocks, 128, smem, s>>>(P, phi, label, n, 1.0f / (float)n, grad, loss);
  return cudaGetLastError();
}

cudaError_t launch_mlp_adam(float* P, const float* grad, float* m1, float* m2, float lr,
                            int step, cudaStream_t s) {
  const float b1 = 0.9f, b2 = 0.999f;
  const float bc1 = 1.f - powf(b1, (float)step), bc2 = 1.f - powf(b2, (float)step);
  mlp_adam_kernel<<<(kNParams + 255) / 256, 256, 0, s>>>(P, grad, m1, m2, lr, b1, b2, 1e-8f, bc1, bc2);
  return cudaGetLastError();
}

}  // namespace pic
