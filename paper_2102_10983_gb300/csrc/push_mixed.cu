// Mixed-precision form of the adaptive sub-cycling push (arXiv 2102.10983).
//
// Same method as push_f64.cu (Algorithm 1 of Sec. IV, order-p temporal
// Lagrange interpolation of Sec. VI, tent gather of Eqs. eq:Enp/eq:Bnp, Boris
// of Eqs. eq:p - eq:x) with a GB300-shaped arithmetic split:
//  - fields, Lagrange weights, the criterion and the Boris rotation are FP32
//    (GB300 issues ~60x more FP32 than FP64 per clock);
//  - the position is an exact int32 node index `cell` plus an FP32 offset
//    `frac` (x = (cell + frac) dx).  Sub-step displacements go into the
//    offset; the integer part is carried into `cell` once per macro step, so
//    the position keeps ~1e-7 of a cell absolute resolution anywhere on the
//    grid and over any drift, with no FP64 instruction in the loop.
// Particle state is 21 bytes: cell i32, frac f32, p 3 x f32, status u8.
//
// Every operation is an explicit round-to-nearest intrinsic, so the two
// schedules below (which call the same per-particle functions in different
// kernels) produce identical bits.
//
// Schedules:
//  PLAIN:  one thread per particle; a warp runs as long as its largest 4^k.
//  BINNED: one persistent kernel per macro step with an atomic work cursor.
//          The bulk streams every particle with 128-bit loads; a particle whose
//          criterion gives k = 0 is pushed at once, one with k > 0 is compacted
//          (warp match + one atomic per k) into the queue of its k and its
//          sub-cycling is deferred.  The first work items of the next step's
//          kernel drain those queues, largest k first, in warps of equal k:
//          each deferred particle finishes its previous step and then takes its
//          own criterion for the current one.  So the long sub-cycled pushes
//          run concurrently with the HBM stream of the next step instead of
//          after it.  A closing kernel finishes what the last step deferred.
//
// Status byte inside a binned call: bits 0-2 = k_prev, bit 3 = step parity
// (the bulk of step j only takes particles whose parity equals j & 1 and flips
// it), bits 4-6 = deferred k (0 = none), bit 7 = lost.  Outside a call the
// byte is in the public form (bits 0-6 = k).
#include <limits.h>
#include <math.h>

#include "pic_internal.h"

namespace pic {

__global__ void wtab_f32_kernel(float* out, const double* in, int64_t count) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < count;
       i += (int64_t)gridDim.x * blockDim.x)
    out[i] = (float)in[i];
}

cudaError_t build_wtab_f32(float* wtab, const double* wtab64, int64_t count, cudaStream_t s) {
  int blocks = (int)((count + 255) / 256);
  wtab_f32_kernel<<<blocks, 256, 0, s>>>(wtab, wtab64, count);
  return cudaGetLastError();
}

// ---------------------------------------------------------------- per-particle math

// Temporal sums at the two tent nodes jn, jn+1, then the tent weight wt.
template <int P>
__device__ __forceinline__ float gather_f32(const float* const* lv, const float* w, int32_t jn,
                                            float wt, int32_t mask) {
  const int32_t a0 = jn & mask, a1 = (jn + 1) & mask;
  float f0 = __fmul_rn(w[0], __ldg(lv[0] + a0));
  float f1 = __fmul_rn(w[0], __ldg(lv[0] + a1));
#pragma unroll
  for (int l = 1; l <= P; ++l) {
    f0 = __fmaf_rn(w[l], __ldg(lv[l] + a0), f0);
    f1 = __fmaf_rn(w[l], __ldg(lv[l] + a1), f1);
  }
  return __fmaf_rn(wt, __fsub_rn(f1, f0), f0);
}

struct MixedState {
  int32_t cell;
  float frac, ux, uy, uz;
};

// Tent coordinates of offset f from node `cell`: E grid nodes at i dx, B grid
// nodes at (i + 1/2) dx.  False if a node is outside [lo, hi].
__device__ __forceinline__ bool tent_coords(int32_t cell, float f, int32_t lo, int32_t hi,
                                            int32_t& je, float& we, int32_t& jb, float& wb) {
  const float fe = floorf(f);
  const float fbm = __fsub_rn(f, 0.5f);
  const float fb = floorf(fbm);
  je = cell + (int32_t)fe;
  we = __fsub_rn(f, fe);
  jb = cell + (int32_t)fb;
  wb = __fsub_rn(fbm, fb);
  return je >= lo && je < hi && jb >= lo && jb < hi;
}

__device__ __forceinline__ float norm2(float a, float b, float c) {
  return __fmaf_rn(c, c, __fmaf_rn(b, b, __fmul_rn(a, a)));
}

// Criterion (Sec. IV) in FP32: Psi0 = |q/m| |B| dt / (2 gamma); smallest k with
// Psi0 / 4^k <= Psi_max, capped at k_max.
template <int P>
__device__ __forceinline__ int criterion_f32(const float* const* B, const float* wcrit, int32_t jb,
                                             float wb, int32_t mask, const MixedState& s,
                                             float qm_abs, float dt, float psi_max, int k_max,
                                             bool& capped) {
  const float b0 = gather_f32<P>(B, wcrit, jb, wb, mask);
  const float g0 = __fsqrt_rn(__fadd_rn(1.0f, norm2(s.ux, s.uy, s.uz)));
  float psi = __fdiv_rn(__fmul_rn(__fmul_rn(qm_abs, fabsf(b0)), dt), __fmul_rn(2.0f, g0));
  int k = 0;
  while (psi > psi_max && k < k_max) {
    psi = __fmul_rn(psi, 0.25f);
    ++k;
  }
  capped = psi > psi_max;
  return k;
}

// Field view of one macro step.
template <int P>
struct StepFields {
  const float* E[P + 1];
  const float* B[P + 1];
  int32_t lo, hi;
};

// One Boris sub-step (Eqs. eq:p - eq:gamman) and the position update (Eq. eq:x)
// in the fields ey, bz, with momentum step hp and offset step hx (cells per
// unit velocity).
__device__ __forceinline__ void boris_f32(float ey, float bz, float hp, float hx, float qm,
                                          MixedState& s) {
  const float half = __fmul_rn(0.5f, hp);
  const float dpy = __fmul_rn(__fmul_rn(qm, ey), half);
  const float mx = s.ux, my = __fadd_rn(s.uy, dpy), mz = s.uz;
  const float inv_gn = rsqrtf(__fadd_rn(1.0f, norm2(mx, my, mz)));
  const float tz = __fmul_rn(__fmul_rn(__fmul_rn(qm, bz), half), inv_gn);
  const float ppx = __fmaf_rn(my, tz, mx);
  const float ppy = __fmaf_rn(-mx, tz, my);
  const float sz = __fdividef(__fmul_rn(2.0f, tz), __fmaf_rn(tz, tz, 1.0f));
  s.ux = __fmaf_rn(ppy, sz, mx);
  s.uy = __fadd_rn(__fmaf_rn(-ppx, sz, my), dpy);
  s.uz = mz;
  const float inv_g = rsqrtf(__fadd_rn(1.0f, norm2(s.ux, s.uy, s.uz)));
  s.frac = __fmaf_rn(hx, __fmul_rn(s.ux, inv_g), s.frac);
}

// Reciprocal of prod_{k != j} (j - k), the denominator of L_{p,j} (Sec. VI).
__host__ __device__ constexpr float lagrange_inv_den(int p, int j) {
  float d = 1.f;
  for (int k = 0; k <= p; ++k)
    if (k != j) d *= (float)(j - k);
  return 1.f / d;
}

// Weights of Eqs. eq:lagrange2-3 (E) and eq:lagrange2-2 (B) at theta, in FP32:
// prod_{k != j} (c_k + theta) times the reciprocal denominator, c_k = p-k-1/2
// (E) or p-k-1 (B).  Depends on the sub-step index only, so these FP32 ops run
// alongside the serial chain of the push instead of on it.
template <int P>
__device__ __forceinline__ void lagrange_f32(float theta, float* w) {
#pragma unroll
  for (int j = 0; j <= P; ++j) {
    float ne = 1.f, nb = 1.f;
#pragma unroll
    for (int k = 0; k <= P; ++k) {
      if (k == j) continue;
      ne = __fmul_rn(ne, __fadd_rn((float)(P - k) - 0.5f, theta));
      nb = __fmul_rn(nb, __fadd_rn((float)(P - k) - 1.0f, theta));
    }
    w[j] = __fmul_rn(ne, lagrange_inv_den(P, j));
    w[P + 1 + j] = __fmul_rn(nb, lagrange_inv_den(P, j));
  }
}

// Temporal sum over the levels' values v at one node, then nothing else: the
// same operation order as gather_f32.
template <int P>
__device__ __forceinline__ float tsum(const float* w, const float* v) {
  float f = __fmul_rn(w[0], v[0]);
#pragma unroll
  for (int l = 1; l <= P; ++l) f = __fmaf_rn(w[l], v[l], f);
  return f;
}

// The m = 4^k sub-steps of one macro step (Algorithm 1).  False if the particle
// left the window (state kept as reached).
//
// m = 1 takes a straight path with the tabulated weights.  For m > 1 the level
// values at the two tent nodes of each grid stay in registers while the node
// index is unchanged (an electron moves a small fraction of a cell per
// sub-step), and the weights of each sub-step are computed from theta_j on the
// spot: nothing on the serial chain of a long sub-cycle waits on memory.
template <int P>
__device__ __forceinline__ bool subcycle_f32(const StepFields<P>& F, const float* wtab,
                                             int32_t mask, float dt, float inv_dx, float qm,
                                             int field_time, int k, int k_prev, MixedState& s) {
  constexpr int stride = 2 * (P + 1);
  const float h = ldexpf(dt, -2 * k);
  const float h_old = ldexpf(dt, -2 * k_prev);
  const float hx = __fmul_rn(h, inv_dx);
  float hp = __fmul_rn(0.5f, __fadd_rn(h_old, h));
  if (k == 0) {
    const float* wr = wtab + wrow(0, 1) * stride;
    int32_t je, jb;
    float we, wb;
    if (!tent_coords(s.cell, s.frac, F.lo, F.hi, je, we, jb, wb)) return false;
    const float ey = gather_f32<P>(F.E, wr, je, we, mask);
    const float bz = gather_f32<P>(F.B, wr + (P + 1), jb, wb, mask);
    boris_f32(ey, bz, hp, hx, qm, s);
    return true;
  }
  const int m = 1 << (2 * k);
  const float inv_m = ldexpf(1.0f, -2 * k);
  int32_t ce = INT_MIN, cb = INT_MIN;
  float e0[P + 1], e1[P + 1], b0[P + 1], b1[P + 1];
  for (int j = 1; j <= m; ++j) {
    // theta_j = 1/2 + (j-1)/m (position time) or (j - 1/2)/m; exact in FP32 for m <= 4^7
    const float jm1 = (float)(j - 1);
    const float theta = field_time == 0 ? __fadd_rn(0.5f, __fmul_rn(jm1, inv_m))
                                        : __fmul_rn(__fadd_rn(jm1, 0.5f), inv_m);
    float w[stride];
    lagrange_f32<P>(theta, w);
    int32_t je, jb;
    float we, wb;
    if (!tent_coords(s.cell, s.frac, F.lo, F.hi, je, we, jb, wb)) return false;
    if (je != ce) {
      ce = je;
      const int32_t a0 = je & mask, a1 = (je + 1) & mask;
#pragma unroll
      for (int l = 0; l <= P; ++l) {
        e0[l] = __ldg(F.E[l] + a0);
        e1[l] = __ldg(F.E[l] + a1);
      }
    }
    if (jb != cb) {
      cb = jb;
      const int32_t a0 = jb & mask, a1 = (jb + 1) & mask;
#pragma unroll
      for (int l = 0; l <= P; ++l) {
        b0[l] = __ldg(F.B[l] + a0);
        b1[l] = __ldg(F.B[l] + a1);
      }
    }
    const float fe0 = tsum<P>(w, e0), fe1 = tsum<P>(w, e1);
    const float fb0 = tsum<P>(w + (P + 1), b0), fb1 = tsum<P>(w + (P + 1), b1);
    const float ey = __fmaf_rn(we, __fsub_rn(fe1, fe0), fe0);
    const float bz = __fmaf_rn(wb, __fsub_rn(fb1, fb0), fb0);
    boris_f32(ey, bz, hp, hx, qm, s);
    hp = h;
  }
  return true;
}

__device__ __forceinline__ void normalize(MixedState& s) {
  const float fl = floorf(s.frac);
  s.cell += (int32_t)fl;
  s.frac = __fsub_rn(s.frac, fl);
}

// ---------------------------------------------------------------- counters

// Per-thread counters: k = 0 steps and sub-step sums in registers; rare events
// (k > 0, caps, losses) straight into shared memory.
struct ThreadCounters {
  unsigned long long k0 = 0, sub = 0, star = 0;
};

__device__ __forceinline__ void count_step(ThreadCounters& tc, unsigned long long* sh, int k,
                                           bool capped) {
  const unsigned long long m = 1ull << (2 * k);
  tc.sub += m;
  if (k == 0) {
    ++tc.k0;
  } else {
    tc.star += m;
    atomicAdd(&sh[k], 1ull);
  }
  if (capped) atomicAdd(&sh[10], 1ull);
}

__device__ __forceinline__ unsigned long long warp_sum(unsigned long long v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// All threads of the block must call this.
__device__ __forceinline__ void flush_counters(const ThreadCounters& tc, unsigned long long* sh,
                                               DevStats* st) {
  const unsigned long long k0 = warp_sum(tc.k0), sub = warp_sum(tc.sub), star = warp_sum(tc.star);
  if ((threadIdx.x & 31) == 0) {
    if (k0) atomicAdd(&sh[0], k0);
    if (sub) atomicAdd(&sh[8], sub);
    if (star) atomicAdd(&sh[9], star);
  }
  __syncthreads();
  if (threadIdx.x < 12) {
    const unsigned long long v = sh[threadIdx.x];
    if (v) {
      unsigned long long* dst = threadIdx.x < 8 ? &st->k_hist[threadIdx.x]
                                : threadIdx.x == 8 ? &st->substeps
                                : threadIdx.x == 9 ? &st->n_star
                                : threadIdx.x == 10 ? &st->clamped
                                                    : &st->lost;
      atomicAdd(dst, v);
    }
  }
}

__device__ __forceinline__ MixedState load_state(const PushArgsMixed& a, int64_t i) {
  MixedState s;
  s.cell = a.cell[i];
  s.frac = a.frac[i];
  s.ux = a.px[i];
  s.uy = a.py[i];
  s.uz = a.pz[i];
  return s;
}

__device__ __forceinline__ void store_state(const PushArgsMixed& a, int64_t i, const MixedState& s) {
  a.cell[i] = s.cell;
  a.frac[i] = s.frac;
  a.px[i] = s.ux;
  a.py[i] = s.uy;
  a.pz[i] = s.uz;
}

template <int P>
__device__ __forceinline__ void load_fields(StepFields<P>& F, const float* const* E,
                                            const float* const* B, int32_t lo, int32_t hi) {
#pragma unroll
  for (int l = 0; l <= P; ++l) {
    F.E[l] = E[l];
    F.B[l] = B[l];
  }
  F.lo = lo;
  F.hi = hi;
}

// ---------------------------------------------------------------- PLAIN schedule

template <int P>
__global__ void __launch_bounds__(256) push_mixed_plain_kernel(PushArgsMixed a) {
  __shared__ unsigned long long sh[12];
  if (threadIdx.x < 12) sh[threadIdx.x] = 0ull;
  __syncthreads();
  constexpr int stride = 2 * (P + 1);
  const float* wcrit = a.wtab + a.crit_row * stride + (P + 1);
  StepFields<P> F;
  load_fields<P>(F, a.E, a.B, a.lo, a.hi);
  ThreadCounters tc;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < a.n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const uint8_t st = a.status[i];
    if (st & PIC_STATUS_LOST) continue;
    MixedState s = load_state(a, i);
    int32_t je, jb;
    float we, wb;
    if (!tent_coords(s.cell, s.frac, F.lo, F.hi, je, we, jb, wb)) {
      a.status[i] = (uint8_t)(st | PIC_STATUS_LOST);
      atomicAdd(&sh[11], 1ull);
      continue;
    }
    bool capped;
    const int k = criterion_f32<P>(F.B, wcrit, jb, wb, a.mask, s, a.qm_abs, a.dt, a.psi_max,
                                   a.k_max, capped);
    count_step(tc, sh, k, capped);
    const bool ok = subcycle_f32<P>(F, a.wtab, a.mask, a.dt, a.inv_dx, a.qm, a.field_time, k, st & 0x7f, s);
    normalize(s);
    store_state(a, i, s);
    a.status[i] = ok ? (uint8_t)k : (uint8_t)(k | PIC_STATUS_LOST);
    if (!ok) atomicAdd(&sh[11], 1ull);
  }
  flush_counters(tc, sh, a.stats);
}

// ---------------------------------------------------------------- BINNED schedule

constexpr int kV = 4;                 // particles per lane in the bulk (128-bit loads)
constexpr int kChunk = 32 * kV;       // particles per bulk work item
constexpr uint8_t kParity = 0x08;
constexpr uint8_t kDeferMask = 0x70;

__device__ __forceinline__ int deferred_k(uint8_t st) { return (st >> 4) & 7; }

// Enqueue particle i into the queue of its k (1..7); warp-aggregated: one
// atomic per distinct k in the warp.  All 32 lanes call this; key 0 = nothing.
__device__ __forceinline__ void enqueue(const PushArgsMixed& a, int key, int32_t i) {
  const unsigned peers = __match_any_sync(0xffffffffu, key);
  const int lane = threadIdx.x & 31;
  const int leader = __ffs(peers) - 1;
  int base = 0;
  if (key != 0 && lane == leader) base = atomicAdd(&a.qcount_out[key], __popc(peers));
  base = __shfl_sync(0xffffffffu, base, leader);
  if (key != 0) {
    const int rank = __popc(peers & ((1u << lane) - 1u));
    a.queue_out[(int64_t)(key - 1) * a.qcap + base + rank] = i;
  }
}

// Heavy item: finish the deferred previous step of particle i, then take its
// criterion for the current step (push at once if k = 0, else defer again).
// finalize: only finish the deferred step and write the public status.
template <int P>
__device__ __forceinline__ void heavy_particle(const PushArgsMixed& a, const StepFields<P>& Fp,
                                               const StepFields<P>& Fc, const float* wcrit,
                                               int64_t i, ThreadCounters& tc,
                                               unsigned long long* sh, int& defer_key) {
  defer_key = 0;
  const uint8_t st = a.status[i];
  const int k = deferred_k(st);
  const int k_prev = st & 7;
  MixedState s = load_state(a, i);
  const bool ok = subcycle_f32<P>(Fp, a.wtab, a.mask, a.dt, a.inv_dx, a.qm, a.field_time, k, k_prev, s);
  normalize(s);
  if (!ok) {
    store_state(a, i, s);
    a.status[i] = (uint8_t)(k | PIC_STATUS_LOST);
    atomicAdd(&sh[11], 1ull);
    return;
  }
  if (a.finalize) {
    store_state(a, i, s);
    a.status[i] = (uint8_t)k;
    return;
  }
  int32_t je, jb;
  float we, wb;
  if (!tent_coords(s.cell, s.frac, Fc.lo, Fc.hi, je, we, jb, wb)) {
    store_state(a, i, s);
    a.status[i] = (uint8_t)(k | PIC_STATUS_LOST);
    atomicAdd(&sh[11], 1ull);
    return;
  }
  bool capped;
  const int kn = criterion_f32<P>(Fc.B, wcrit, jb, wb, a.mask, s, a.qm_abs, a.dt, a.psi_max,
                                  a.k_max, capped);
  count_step(tc, sh, kn, capped);
  if (kn == 0) {
    const bool ok2 = subcycle_f32<P>(Fc, a.wtab, a.mask, a.dt, a.inv_dx, a.qm, a.field_time, 0, k, s);
    normalize(s);
    store_state(a, i, s);
    a.status[i] = ok2 ? (uint8_t)(a.parity_next ? kParity : 0) : (uint8_t)PIC_STATUS_LOST;
    if (!ok2) atomicAdd(&sh[11], 1ull);
  } else {
    store_state(a, i, s);
    a.status[i] = (uint8_t)(k | (kn << 4));
    defer_key = kn;
  }
}

template <int P>
__global__ void __launch_bounds__(256) push_mixed_binned_kernel(PushArgsMixed a) {
  __shared__ unsigned long long sh[12];
  __shared__ int s_task[8];
  __shared__ long long heavy_end[8];  // heavy items: ceil(count/32) per k, largest k first
  if (threadIdx.x < 12) sh[threadIdx.x] = 0ull;
  if (threadIdx.x == 0) {
    long long acc = 0;
    heavy_end[0] = 0;
    for (int k = 7; k >= 1; --k) {
      const long long c = (k <= a.k_max) ? a.qcount_in[k] : 0;
      acc += (c + 31) / 32;
      heavy_end[k] = acc;
    }
  }
  __syncthreads();
  constexpr int stride = 2 * (P + 1);
  const float* wcrit = a.wtab + a.crit_row * stride + (P + 1);
  StepFields<P> Fc, Fp;
  load_fields<P>(Fc, a.E, a.B, a.lo, a.hi);
  load_fields<P>(Fp, a.Ep, a.Bp, a.lo_p, a.hi_p);
  ThreadCounters tc;
  const int lane = threadIdx.x & 31;
  const int warp = threadIdx.x >> 5;

  const int64_t n_heavy = heavy_end[1];
  const int64_t n_bulk = a.finalize ? (a.n + kChunk - 1) / kChunk : (a.n + kChunk - 1) / kChunk;
  const int64_t n_items = n_heavy + n_bulk;

  for (;;) {
    if (lane == 0) s_task[warp] = atomicAdd(a.cursor, 1);
    __syncwarp();
    const int64_t t = s_task[warp];
    __syncwarp();
    if (t >= n_items) break;
    if (t < n_heavy) {
      int k = 7;
      while (k > 1 && t >= heavy_end[k]) --k;
      const int64_t first = (k == 7 ? 0 : heavy_end[k + 1]);
      const int64_t e = (t - first) * 32 + lane;
      int key = 0;
      if (e < a.qcount_in[k]) {
        const int32_t i = a.queue_in[(int64_t)(k - 1) * a.qcap + e];
        heavy_particle<P>(a, Fp, Fc, wcrit, i, tc, sh, key);
        enqueue(a, key, i);
      } else {
        enqueue(a, 0, 0);
      }
      continue;
    }
    // bulk item
    const int64_t base = (t - n_heavy) * kChunk + (int64_t)lane * kV;
    if (a.finalize) {
      // return every byte to the public form (deferred ones are written by
      // their heavy item)
#pragma unroll
      for (int v = 0; v < kV; ++v) {
        const int64_t i = base + v;
        if (i < a.n) {
          const uint8_t st = a.status[i];
          if ((st & kDeferMask) == 0) a.status[i] = (uint8_t)(st & (PIC_STATUS_LOST | 7));
        }
      }
      continue;
    }
    const uint8_t want = a.parity_cur ? kParity : 0;
    const bool full = base + kV <= a.n;
    MixedState s[kV];
    uint8_t st[kV];
    if (full) {
      const int4 c4 = *reinterpret_cast<const int4*>(a.cell + base);
      const float4 f4 = *reinterpret_cast<const float4*>(a.frac + base);
      const float4 x4 = *reinterpret_cast<const float4*>(a.px + base);
      const float4 y4 = *reinterpret_cast<const float4*>(a.py + base);
      const float4 z4 = *reinterpret_cast<const float4*>(a.pz + base);
      const uint32_t s4 = *reinterpret_cast<const uint32_t*>(a.status + base);
      s[0] = {c4.x, f4.x, x4.x, y4.x, z4.x};
      s[1] = {c4.y, f4.y, x4.y, y4.y, z4.y};
      s[2] = {c4.z, f4.z, x4.z, y4.z, z4.z};
      s[3] = {c4.w, f4.w, x4.w, y4.w, z4.w};
#pragma unroll
      for (int v = 0; v < kV; ++v) st[v] = (uint8_t)(s4 >> (8 * v));
    } else {
#pragma unroll
      for (int v = 0; v < kV; ++v) {
        if (base + v < a.n) {
          s[v] = load_state(a, base + v);
          st[v] = a.status[base + v];
        } else {
          st[v] = PIC_STATUS_LOST;
        }
      }
    }
    bool owned_elsewhere = false;  // a lane particle belongs to the heavy items
    bool touched[kV];
#pragma unroll
    for (int v = 0; v < kV; ++v) {
      const bool valid = base + v < a.n;
      const bool mine = valid && !(st[v] & PIC_STATUS_LOST) && !(st[v] & kDeferMask) &&
                        ((st[v] & kParity) == want);
      if (valid && !(st[v] & PIC_STATUS_LOST) && !mine) owned_elsewhere = true;
      touched[v] = mine;
      int key = 0;
      if (mine) {
        int32_t je, jb;
        float we, wb;
        if (!tent_coords(s[v].cell, s[v].frac, Fc.lo, Fc.hi, je, we, jb, wb)) {
          st[v] = (uint8_t)(st[v] | PIC_STATUS_LOST);
          atomicAdd(&sh[11], 1ull);
        } else {
          bool capped;
          const int k = criterion_f32<P>(Fc.B, wcrit, jb, wb, a.mask, s[v], a.qm_abs, a.dt,
                                         a.psi_max, a.k_max, capped);
          count_step(tc, sh, k, capped);
          const int k_prev = st[v] & 7;
          if (k == 0) {
            const bool ok = subcycle_f32<P>(Fc, a.wtab, a.mask, a.dt, a.inv_dx, a.qm,
                                            a.field_time, 0, k_prev, s[v]);
            normalize(s[v]);
            st[v] = ok ? (uint8_t)(a.parity_next ? kParity : 0) : (uint8_t)PIC_STATUS_LOST;
            if (!ok) atomicAdd(&sh[11], 1ull);
          } else {
            st[v] = (uint8_t)(k_prev | (k << 4));
            key = k;
          }
        }
      }
      enqueue(a, key, (int32_t)(base + v));
    }
    if (full && !owned_elsewhere) {
      *reinterpret_cast<int4*>(a.cell + base) = make_int4(s[0].cell, s[1].cell, s[2].cell, s[3].cell);
      *reinterpret_cast<float4*>(a.frac + base) = make_float4(s[0].frac, s[1].frac, s[2].frac, s[3].frac);
      *reinterpret_cast<float4*>(a.px + base) = make_float4(s[0].ux, s[1].ux, s[2].ux, s[3].ux);
      *reinterpret_cast<float4*>(a.py + base) = make_float4(s[0].uy, s[1].uy, s[2].uy, s[3].uy);
      *reinterpret_cast<float4*>(a.pz + base) = make_float4(s[0].uz, s[1].uz, s[2].uz, s[3].uz);
      *reinterpret_cast<uint32_t*>(a.status + base) =
          (uint32_t)st[0] | ((uint32_t)st[1] << 8) | ((uint32_t)st[2] << 16) | ((uint32_t)st[3] << 24);
    } else {
#pragma unroll
      for (int v = 0; v < kV; ++v) {
        if (touched[v]) {
          store_state(a, base + v, s[v]);
          a.status[base + v] = st[v];
        }
      }
    }
  }
  flush_counters(tc, sh, a.stats);

  // the last block to finish resets the cursor and the consumed queue counts
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    const unsigned done = atomicAdd(a.blocks_done, 1u);
    if (done == gridDim.x - 1) {
      __threadfence();
      *a.cursor = 0;
      *a.blocks_done = 0;
      for (int k = 0; k < 8; ++k) a.qcount_in[k] = 0;
      __threadfence();
    }
  }
}

// ---------------------------------------------------------------- predictor features

// phi = (asinh|E|, asinh|B|, asinh p_x, asinh p_y, asinh p_z, log gamma) of each
// particle after macro step n, with E and B at its position extrapolated to
// t_{n+1} (theta = 3/2) from step n's levels: everything known before level
// n+1 arrives.  Lost particles get zeros.
template <int P>
__global__ void features_kernel(PushArgsMixed a, float* phi) {
  StepFields<P> F;
  load_fields<P>(F, a.E, a.B, a.lo, a.hi);
  float w[2 * (P + 1)];
  lagrange_f32<P>(1.5f, w);
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < a.n;
       i += (int64_t)gridDim.x * blockDim.x) {
    float f[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
    const uint8_t st = a.status[i];
    if (!(st & PIC_STATUS_LOST)) {
      const MixedState s = load_state(a, i);
      int32_t je, jb;
      float we, wb;
      if (tent_coords(s.cell, s.frac, F.lo, F.hi, je, we, jb, wb)) {
        const float ey = gather_f32<P>(F.E, w, je, we, a.mask);
        const float bz = gather_f32<P>(F.B, w + (P + 1), jb, wb, a.mask);
        f[0] = asinhf(fabsf(ey));
        f[1] = asinhf(fabsf(bz));
      }
      f[2] = asinhf(s.ux);
      f[3] = asinhf(s.uy);
      f[4] = asinhf(s.uz);
      f[5] = 0.5f * log1pf(norm2(s.ux, s.uy, s.uz));
    }
#pragma unroll
    for (int q = 0; q < 6; ++q) phi[i * 6 + q] = f[q];
  }
}

cudaError_t launch_features_mixed(const PushArgsMixed& a, int order, float* phi, cudaStream_t s) {
  if (a.n <= 0) return cudaSuccess;
  const int64_t want = (a.n + 255) / 256;
  const int blocks = (int)(want < 152 * 16 ? want : 152 * 16);
  switch (order) {
    case 1: features_kernel<1><<<blocks, 256, 0, s>>>(a, phi); break;
    case 2: features_kernel<2><<<blocks, 256, 0, s>>>(a, phi); break;
    case 3: features_kernel<3><<<blocks, 256, 0, s>>>(a, phi); break;
    case 4: features_kernel<4><<<blocks, 256, 0, s>>>(a, phi); break;
    case 5: features_kernel<5><<<blocks, 256, 0, s>>>(a, phi); break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

// ---------------------------------------------------------------- launch

template <int P>
static cudaError_t launch_p(const PushArgsMixed& a, int schedule, int sm_count, cudaStream_t s) {
  const int sms = sm_count > 0 ? sm_count : 152;
  if (schedule == PIC_SCHED_BINNED) {
    static int occ = 0;
    if (occ == 0) {
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, push_mixed_binned_kernel<P>, 256, 0);
      if (occ < 1) occ = 1;
    }
    const int64_t items = (a.n + kChunk - 1) / kChunk;
    int64_t blocks = (int64_t)sms * occ;
    const int64_t need = (items + 7) / 8 + 1;
    if (blocks > need) blocks = need;
    push_mixed_binned_kernel<P><<<(int)blocks, 256, 0, s>>>(a);
  } else {
    const int64_t want = (a.n + 255) / 256;
    const int64_t cap = (int64_t)sms * 8;
    push_mixed_plain_kernel<P><<<(int)(want < cap ? want : cap), 256, 0, s>>>(a);
  }
  return cudaGetLastError();
}

cudaError_t launch_push_mixed(const PushArgsMixed& a, int order, int schedule, int sm_count,
                              cudaStream_t s, int* launches) {
  if (a.n <= 0) return cudaSuccess;
  cudaError_t e;
  switch (order) {
    case 1: e = launch_p<1>(a, schedule, sm_count, s); break;
    case 2: e = launch_p<2>(a, schedule, sm_count, s); break;
    case 3: e = launch_p<3>(a, schedule, sm_count, s); break;
    case 4: e = launch_p<4>(a, schedule, sm_count, s); break;
    case 5: e = launch_p<5>(a, schedule, sm_count, s); break;
    default: return cudaErrorInvalidValue;
  }
  if (launches) ++*launches;
  return e;
}

}  // namespace pic
