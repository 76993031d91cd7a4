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
__device__ __forceinline__ int psi_to_k(float b0, const MixedState& s, float qm_abs, float dt,
                                        float psi_max, int k_max, bool& capped) {
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

// b0 is B_z at the particle and t_n: with m = 1 it is also the first (and only)
// sub-step's B_z, since both use the theta = 1/2 weights at the same nodes.
template <int P>
__device__ __forceinline__ int criterion_f32(const float* const* B, const float* wcrit, int32_t jb,
                                             float wb, int32_t mask, const MixedState& s,
                                             float qm_abs, float dt, float psi_max, int k_max,
                                             bool& capped, float& b0) {
  b0 = gather_f32<P>(B, wcrit, jb, wb, mask);
  return psi_to_k(b0, s, qm_abs, dt, psi_max, k_max, capped);
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

// Lagrange basis polynomials of Sec. VI in monomial form around theta = 1:
// the nodes in u = theta - 1 are l - p - 1/2 (E) and l - p (B); multiply out
// prod_{k != l} (u - u_k) / (u_l - u_k) in FP64.
void lagrange_monomials(int p, float (&mono)[2][kMaxOrder + 1][kMaxOrder + 1]) {
  for (int grid = 0; grid < 2; ++grid) {
    const double off = grid == 0 ? -0.5 : 0.0;
    for (int l = 0; l <= kMaxOrder; ++l)
      for (int q = 0; q <= kMaxOrder; ++q) mono[grid][l][q] = 0.f;
    for (int l = 0; l <= p; ++l) {
      double c[kMaxOrder + 2] = {1.0};
      int deg = 0;
      double den = 1.0;
      const double ul = (double)(l - p) + off;
      for (int k = 0; k <= p; ++k) {
        if (k == l) continue;
        const double uk = (double)(k - p) + off;
        for (int q = deg + 1; q >= 0; --q) c[q] = (q > 0 ? c[q - 1] : 0.0) - uk * c[q];
        ++deg;
        den *= ul - uk;
      }
      for (int q = 0; q <= p; ++q) mono[grid][l][q] = (float)(c[q] / den);
    }
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
// Coefficients of the interpolating polynomial in u at two nodes a0, a1 of the
// given levels: c_q = sum_l v_l M[l][q].
template <int P>
__device__ __forceinline__ void to_monomial(const float* const* lv, int32_t a0, int32_t a1,
                                            const float (&M)[kMaxOrder + 1][kMaxOrder + 1],
                                            float* c0, float* c1) {
  float v0[P + 1], v1[P + 1];
#pragma unroll
  for (int l = 0; l <= P; ++l) {
    v0[l] = __ldg(lv[l] + a0);
    v1[l] = __ldg(lv[l] + a1);
  }
#pragma unroll
  for (int q = 0; q <= P; ++q) {
    float x0 = __fmul_rn(v0[0], M[0][q]), x1 = __fmul_rn(v1[0], M[0][q]);
#pragma unroll
    for (int l = 1; l <= P; ++l) {
      x0 = __fmaf_rn(v0[l], M[l][q], x0);
      x1 = __fmaf_rn(v1[l], M[l][q], x1);
    }
    c0[q] = x0;
    c1[q] = x1;
  }
}

template <int P>
__device__ __forceinline__ float horner(const float* c, float u) {
  float f = c[P];
#pragma unroll
  for (int q = P - 1; q >= 0; --q) f = __fmaf_rn(f, u, c[q]);
  return f;
}

// m = 1 takes a straight path with the tabulated weights and the criterion's
// B_z (b0; unused for m > 1).  For m > 1 the
// temporal interpolant at each tent node is a polynomial of degree p in
// u = theta - 1; its coefficients are formed when the node index changes (an
// electron moves a small fraction of a cell per sub-step) and each sub-step
// evaluates it by Horner's rule: p FMAs per node, nothing waits on memory.
template <int P>
__device__ __forceinline__ bool subcycle_f32(const StepFields<P>& F, const float* wtab,
                                             int32_t mask, float dt, float inv_dx, float qm,
                                             int field_time,
                                             const float (&mono)[2][kMaxOrder + 1][kMaxOrder + 1],
                                             int k, int k_prev, float b0, MixedState& s) {
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
    boris_f32(ey, b0, hp, hx, qm, s);  // b0: the criterion's B_z (same weights, same nodes)
    return true;
  }
  const int m = 1 << (2 * k);
  const float inv_m = ldexpf(1.0f, -2 * k);
  // u_j = theta_j - 1, exact in FP32 for m <= 4^7
  const float u1 = field_time == 0 ? -0.5f : __fsub_rn(__fmul_rn(0.5f, inv_m), 1.0f);
  int32_t ce = INT_MIN, cb = INT_MIN;
  float ce0[P + 1], ce1[P + 1], cb0[P + 1], cb1[P + 1];  // monomial coefficients per node
  for (int j = 1; j <= m; ++j) {
    const float u = __fmaf_rn((float)(j - 1), inv_m, u1);
    int32_t je, jb;
    float we, wb;
    if (!tent_coords(s.cell, s.frac, F.lo, F.hi, je, we, jb, wb)) return false;
    if (je != ce) {
      ce = je;
      to_monomial<P>(F.E, je & mask, (je + 1) & mask, mono[0], ce0, ce1);
    }
    if (jb != cb) {
      cb = jb;
      to_monomial<P>(F.B, jb & mask, (jb + 1) & mask, mono[1], cb0, cb1);
    }
    const float fe0 = horner<P>(ce0, u), fe1 = horner<P>(ce1, u);
    const float fb0 = horner<P>(cb0, u), fb1 = horner<P>(cb1, u);
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
    float b0;
    const int k = criterion_f32<P>(F.B, wcrit, jb, wb, a.mask, s, a.qm_abs, a.dt, a.psi_max,
                                   a.k_max, capped, b0);
    count_step(tc, sh, k, capped);
    const bool ok = subcycle_f32<P>(F, a.wtab, a.mask, a.dt, a.inv_dx, a.qm, a.field_time, a.mono,
                                    k, st & 0x7f, b0, s);
    normalize(s);
    store_state(a, i, s);
    a.status[i] = ok ? (uint8_t)k : (uint8_t)(k | PIC_STATUS_LOST);
    if (!ok) atomicAdd(&sh[11], 1ull);
  }
  flush_counters(tc, sh, a.stats);
}

// ---------------------------------------------------------------- BINNED schedule
//
// One persistent kernel per macro step; every warp takes work items from one
// atomic cursor, in this order:
//  1. deferred items (k >= kDeferMin, largest k first, 32 particles each): the
//     particles whose criterion picked a long sub-cycle in the previous step.
//     Each finishes that step, then takes its criterion for this one (pushed at
//     once unless k >= kDeferMin again).  Being first, the longest serial
//     chains start as the launch starts and run beside the stream below.
//  2. predicted items (predicted schedule only): particles binned before the
//     launch by the predictor's k, pushed fully, largest k first.
//  3. stream chunks of kChunk particles, one per thread, the next particle's
//     state loaded while the current one is pushed.  k = 0: pushed at once (the
//     criterion's B_z serves the push).  k = 1, 2: parked in the warp's stash
//     for that k (shared memory); whenever a stash holds 32 particles the warp
//     pushes them together, so short sub-cycles never diverge a warp and never
//     leave the chip.  k >= kDeferMin: compacted into the queue of its k (one
//     atomic per distinct k per warp) and deferred to the next launch.
// Status byte inside a binned call: bits 0-2 = k_prev, bit 3 = step parity
// (the stream of step j takes particles whose parity equals j & 1 and flips
// it), bits 4-6 = deferred k (0 = none), bit 7 = lost.

constexpr int kThreads = 256;
constexpr int kWarps = kThreads / 32;
constexpr int kChunk = 256;          // particles per stream item (8 per lane)
constexpr int kDeferMin = 3;         // smallest k that is deferred
constexpr int kStashK = kDeferMin - 1;
constexpr int kStashCap = 64;
constexpr uint8_t kParity = 0x08;
constexpr uint8_t kDeferMask = 0x70;

__device__ __forceinline__ int deferred_k(uint8_t st) { return (st >> 4) & 7; }

// Enqueue particle i into the queue of its k; warp-aggregated: one atomic per
// distinct k in the warp.  All 32 lanes call this; key 0 = nothing.
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

// A warp's stash of particles waiting for a short sub-cycle of one k.
struct Stash {
  int32_t idx[kStashCap];
  int32_t cell[kStashCap];
  float frac[kStashCap], ux[kStashCap], uy[kStashCap], uz[kStashCap];
  uint8_t kp[kStashCap];
};

// Push the first `cnt` (<= 32) stashed particles, one per lane, with 4^k
// sub-steps each; then move entries [cnt, n) to the front.  Warp-collective.
template <int P>
__device__ __forceinline__ void stash_drain(const PushArgsMixed& a, const StepFields<P>& F,
                                            Stash& S, int k, int& n, int cnt,
                                            unsigned long long* sh) {
  const int lane = threadIdx.x & 31;
  if (lane < cnt) {
    MixedState s = {S.cell[lane], S.frac[lane], S.ux[lane], S.uy[lane], S.uz[lane]};
    const int32_t i = S.idx[lane];
    const bool ok = subcycle_f32<P>(F, a.wtab, a.mask, a.dt, a.inv_dx, a.qm, a.field_time, a.mono,
                                    k, S.kp[lane], 0.f, s);
    normalize(s);
    store_state(a, i, s);
    a.status[i] = ok ? (uint8_t)(k | (a.parity_next ? kParity : 0)) : (uint8_t)(k | PIC_STATUS_LOST);
    if (!ok) atomicAdd(&sh[11], 1ull);
  }
  __syncwarp();
  const int rest = n - cnt;
  if (lane < rest) {
    const int q = cnt + lane;
    S.idx[lane] = S.idx[q];
    S.cell[lane] = S.cell[q];
    S.frac[lane] = S.frac[q];
    S.ux[lane] = S.ux[q];
    S.uy[lane] = S.uy[q];
    S.uz[lane] = S.uz[q];
    S.kp[lane] = S.kp[q];
  }
  __syncwarp();
  n = rest;
}

// Deferred item: finish the previous step of particle i, then take its
// criterion for the current step (pushed at once if k < kDeferMin, else
// deferred again).  finalize: only finish the deferred step (public status).
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
  const bool ok = subcycle_f32<P>(Fp, a.wtab, a.mask, a.dt, a.inv_dx, a.qm, a.field_time, a.mono,
                                  k, k_prev, 0.f, s);
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
  float b0;
  const int kn = criterion_f32<P>(Fc.B, wcrit, jb, wb, a.mask, s, a.qm_abs, a.dt, a.psi_max,
                                  a.k_max, capped, b0);
  count_step(tc, sh, kn, capped);
  if (kn < kDeferMin) {
    const bool ok2 = subcycle_f32<P>(Fc, a.wtab, a.mask, a.dt, a.inv_dx, a.qm, a.field_time,
                                     a.mono, kn, k, b0, s);
    normalize(s);
    store_state(a, i, s);
    a.status[i] = ok2 ? (uint8_t)(kn | (a.parity_next ? kParity : 0)) : (uint8_t)(kn | PIC_STATUS_LOST);
    if (!ok2) atomicAdd(&sh[11], 1ull);
  } else {
    store_state(a, i, s);
    a.status[i] = (uint8_t)(k | (kn << 4));
    defer_key = kn;
  }
}

// Predicted item: particle i was binned before the launch as likely to
// sub-cycle; take its exact criterion and all its sub-steps now.
template <int P>
__device__ __forceinline__ void predicted_particle(const PushArgsMixed& a, const StepFields<P>& Fc,
                                                   const float* wcrit, int64_t i, ThreadCounters& tc,
                                                   unsigned long long* sh) {
  const uint8_t st = a.status[i];
  const int k_prev = st & 7;
  MixedState s = load_state(a, i);
  int32_t je, jb;
  float we, wb;
  if (!tent_coords(s.cell, s.frac, Fc.lo, Fc.hi, je, we, jb, wb)) {
    a.status[i] = (uint8_t)(k_prev | PIC_STATUS_LOST);
    atomicAdd(&sh[11], 1ull);
    return;
  }
  bool capped;
  float b0;
  const int k = criterion_f32<P>(Fc.B, wcrit, jb, wb, a.mask, s, a.qm_abs, a.dt, a.psi_max,
                                 a.k_max, capped, b0);
  count_step(tc, sh, k, capped);
  const bool ok = subcycle_f32<P>(Fc, a.wtab, a.mask, a.dt, a.inv_dx, a.qm, a.field_time, a.mono,
                                  k, k_prev, b0, s);
  normalize(s);
  store_state(a, i, s);
  a.status[i] = ok ? (uint8_t)(k | (a.parity_next ? kParity : 0)) : (uint8_t)(k | PIC_STATUS_LOST);
  if (!ok) atomicAdd(&sh[11], 1ull);
}

// Before a predicted-schedule launch: particles the stream would take this
// step and whose predicted k is > 0 go into the queue of that k, and their
// parity bit is flipped so the stream leaves them to the predicted items.
__global__ void bin_predicted_kernel(const uint8_t* pred, uint8_t* status, int64_t n,
                                     int parity_cur, int32_t* pred_queue, int32_t* pred_count,
                                     int64_t qcap) {
  const uint8_t want = parity_cur ? kParity : 0;
  const int64_t n_round = (n + 31) & ~(int64_t)31;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n_round;
       i += (int64_t)gridDim.x * blockDim.x) {
    int key = 0;
    if (i < n) {
      const uint8_t st = status[i];
      const int kp = pred[i];
      if (!(st & PIC_STATUS_LOST) && !(st & kDeferMask) && ((st & kParity) == want) && kp > 0 &&
          kp <= 7) {
        status[i] = (uint8_t)(st ^ kParity);
        key = kp;
      }
    }
    const unsigned peers = __match_any_sync(0xffffffffu, key);
    const int lane = threadIdx.x & 31;
    const int leader = __ffs(peers) - 1;
    int base = 0;
    if (key != 0 && lane == leader) base = atomicAdd(&pred_count[key], __popc(peers));
    base = __shfl_sync(0xffffffffu, base, leader);
    if (key != 0)
      pred_queue[(int64_t)(key - 1) * qcap + base + __popc(peers & ((1u << lane) - 1u))] = (int32_t)i;
  }
}

cudaError_t launch_bin_predicted(const uint8_t* pred, uint8_t* status, int64_t n, int parity_cur,
                                 int32_t* pred_queue, int32_t* pred_count, int64_t qcap,
                                 cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  const int64_t want = (n + 255) / 256;
  const int blocks = (int)(want < 152 * 8 ? want : 152 * 8);
  bin_predicted_kernel<<<blocks, 256, 0, s>>>(pred, status, n, parity_cur, pred_queue, pred_count,
                                              qcap);
  return cudaGetLastError();
}

template <int P>
__global__ void __launch_bounds__(kThreads) push_binned_kernel(PushArgsMixed a) {
  extern __shared__ __align__(16) unsigned char smem[];
  Stash* stashes = reinterpret_cast<Stash*>(smem);  // [kWarps][kStashK]
  __shared__ unsigned long long sh[12];
  __shared__ int s_task[kWarps];
  __shared__ long long heavy_end[8];  // deferred items per k, largest k first (cumulative)
  __shared__ long long pred_end[8];   // then predicted items
  if (threadIdx.x < 12) sh[threadIdx.x] = 0ull;
  if (threadIdx.x == 0) {
    long long acc = 0;
    heavy_end[0] = 0;
    for (int k = 7; k >= 1; --k) {
      const long long c = (k <= a.k_max) ? a.qcount_in[k] : 0;
      acc += (c + 31) / 32;
      heavy_end[k] = acc;
    }
    pred_end[0] = acc;
    for (int k = 7; k >= 1; --k) {
      const long long c = a.pred_count ? a.pred_count[k] : 0;
      acc += (c + 31) / 32;
      pred_end[k] = acc;
    }
  }
  __syncthreads();
  constexpr int stride = 2 * (P + 1);
  const float* wcrit = a.wtab + a.crit_row * stride + (P + 1);
  const float* w0 = a.wtab + wrow(0, 1) * stride;  // theta = 1/2 weights of an m = 1 step
  StepFields<P> F, Fp;
  load_fields<P>(F, a.E, a.B, a.lo, a.hi);
  load_fields<P>(Fp, a.Ep, a.Bp, a.lo_p, a.hi_p);
  ThreadCounters tc;
  const int lane = threadIdx.x & 31;
  const int warp = threadIdx.x >> 5;
  Stash* my_stash = stashes + warp * kStashK;
  int stash_n[kStashK];
#pragma unroll
  for (int q = 0; q < kStashK; ++q) stash_n[q] = 0;
  const uint8_t want = a.parity_cur ? kParity : 0;
  const uint8_t done = a.parity_next ? kParity : 0;
  const float hx0 = __fmul_rn(a.dt, a.inv_dx);
  const int64_t n_heavy = heavy_end[1];
  const int64_t n_pred_end = pred_end[1];
  const int64_t n_chunks = a.finalize ? 0 : (a.n + kChunk - 1) / kChunk;
  const int64_t n_items = n_pred_end + n_chunks;

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
      int32_t i = 0;
      if (e < a.qcount_in[k]) {
        i = a.queue_in[(int64_t)(k - 1) * a.qcap + e];
        heavy_particle<P>(a, Fp, F, wcrit, i, tc, sh, key);
      }
      enqueue(a, key, i);
      continue;
    }
    if (t < n_pred_end) {
      int k = 7;
      while (k > 1 && t >= pred_end[k]) --k;
      const int64_t first = (k == 7 ? n_heavy : pred_end[k + 1]);
      const int64_t e = (t - first) * 32 + lane;
      if (e < a.pred_count[k])
        predicted_particle<P>(a, F, wcrit, a.pred_queue[(int64_t)(k - 1) * a.qcap + e], tc, sh);
      continue;
    }
    // stream chunk
    const int64_t c0 = (t - n_pred_end) * kChunk;
    int64_t i = c0 + lane;
    uint8_t st = PIC_STATUS_LOST;
    MixedState s = {0, 0.5f, 0.f, 0.f, 0.f};
    if (i < a.n) {
      st = a.status[i];
      s = load_state(a, i);
    }
#pragma unroll 1
    for (int r = 0; r < kChunk / 32; ++r, i += 32) {
      const int64_t inext = i + 32;
      uint8_t st_n = PIC_STATUS_LOST;
      MixedState s_n = {0, 0.5f, 0.f, 0.f, 0.f};
      if (r + 1 < kChunk / 32 && inext < a.n) {
        st_n = a.status[inext];
        s_n = load_state(a, inext);
      }
      const bool mine = i < a.n && !(st & PIC_STATUS_LOST) && !(st & kDeferMask) &&
                        ((st & kParity) == want);
      int key = 0, sk = 0;
      if (mine) {
        int32_t je, jb;
        float we, wb;
        const bool inwin = tent_coords(s.cell, s.frac, F.lo, F.hi, je, we, jb, wb);
        const float b0 = gather_f32<P>(F.B, wcrit, jb, wb, a.mask);
        const float ey = gather_f32<P>(F.E, w0, je, we, a.mask);
        if (!inwin) {
          a.status[i] = (uint8_t)(st | PIC_STATUS_LOST);
          atomicAdd(&sh[11], 1ull);
        } else {
          bool capped;
          const int k = psi_to_k(b0, s, a.qm_abs, a.dt, a.psi_max, a.k_max, capped);
          count_step(tc, sh, k, capped);
          const int k_prev = st & 7;
          if (k == 0) {
            const float h_old = ldexpf(a.dt, -2 * k_prev);
            const float hp = __fmul_rn(0.5f, __fadd_rn(h_old, a.dt));
            boris_f32(ey, b0, hp, hx0, a.qm, s);
            normalize(s);
            store_state(a, i, s);
            a.status[i] = done;
          } else if (k < kDeferMin) {
            sk = k;
          } else {
            a.status[i] = (uint8_t)(k_prev | (k << 4));
            key = k;
          }
        }
      }
      enqueue(a, key, (int32_t)i);
      // park k = 1, 2 in the warp's stashes; push a stash when it holds 32
#pragma unroll
      for (int q = 0; q < kStashK; ++q) {
        const unsigned m = __ballot_sync(0xffffffffu, sk == q + 1);
        if (m == 0u) continue;
        Stash& S = my_stash[q];
        if (sk == q + 1) {
          const int pos = stash_n[q] + __popc(m & ((1u << lane) - 1u));
          S.idx[pos] = (int32_t)i;
          S.cell[pos] = s.cell;
          S.frac[pos] = s.frac;
          S.ux[pos] = s.ux;
          S.uy[pos] = s.uy;
          S.uz[pos] = s.uz;
          S.kp[pos] = (uint8_t)(st & 7);
        }
        stash_n[q] += __popc(m);
        __syncwarp();
        if (stash_n[q] >= 32) stash_drain<P>(a, F, S, q + 1, stash_n[q], 32, sh);
      }
      st = st_n;
      s = s_n;
    }
  }
  // push what is left in the stashes
#pragma unroll
  for (int q = 0; q < kStashK; ++q)
    if (stash_n[q] > 0) stash_drain<P>(a, F, my_stash[q], q + 1, stash_n[q], stash_n[q], sh);
  flush_counters(tc, sh, a.stats);

  // the last block to finish resets the cursor and the consumed queue counts
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    const unsigned fin = atomicAdd(a.blocks_done, 1u);
    if (fin == gridDim.x - 1) {
      __threadfence();
      *a.cursor = 0;
      *a.blocks_done = 0;
      for (int k = 0; k < 8; ++k) a.qcount_in[k] = 0;
      if (a.pred_count)
        for (int k = 0; k < 8; ++k) a.pred_count[k] = 0;
      __threadfence();
    }
  }
}

// After the closing launch of a call: every status byte back to the public
// form (k | lost).  Deferred particles were written by that launch.
__global__ void reset_status_kernel(uint8_t* status, int64_t n) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const uint8_t st = status[i];
    const uint8_t pub = (uint8_t)(st & (PIC_STATUS_LOST | 7));
    if (pub != st) status[i] = pub;
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
static cudaError_t launch_p(const PushArgsMixed& a, int schedule, int sm_count, cudaStream_t s,
                            int* launches) {
  const int sms = sm_count > 0 ? sm_count : 152;
  if (schedule == PIC_SCHED_PLAIN) {
    const int64_t want = (a.n + 255) / 256;
    const int64_t cap = (int64_t)sms * 8;
    push_mixed_plain_kernel<P><<<(int)(want < cap ? want : cap), 256, 0, s>>>(a);
    if (launches) ++*launches;
  }
  return cudaGetLastError();
}

constexpr size_t kStashBytes = sizeof(Stash) * kWarps * kStashK;

template <int P>
static cudaError_t launch_binned_p(const PushArgsMixed& a, int sm_count, cudaStream_t main,
                                   int* launches) {
  const int sms = sm_count > 0 ? sm_count : 152;
  static int occ = 0;
  if (occ == 0) {
    cudaError_t e = cudaFuncSetAttribute(push_binned_kernel<P>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kStashBytes);
    if (e != cudaSuccess) return e;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, push_binned_kernel<P>, kThreads, kStashBytes);
    if (occ < 1) occ = 1;
  }
  int64_t blocks = (int64_t)sms * occ;
  const int64_t items = (a.n + kChunk - 1) / kChunk;
  if (!a.finalize && blocks > (items + kWarps - 1) / kWarps + sms) blocks = (items + kWarps - 1) / kWarps + sms;
  push_binned_kernel<P><<<(int)blocks, kThreads, kStashBytes, main>>>(a);
  int n = 1;
  if (a.finalize) {
    const int64_t want = (a.n + 255) / 256;
    reset_status_kernel<<<(int)(want < sms * 8 ? want : sms * 8), 256, 0, main>>>(a.status, a.n);
    ++n;
  }
  if (launches) *launches += n;
  return cudaGetLastError();
}

cudaError_t launch_push_mixed(const PushArgsMixed& a, int order, int schedule, int sm_count,
                              cudaStream_t s, int* launches) {
  if (a.n <= 0) return cudaSuccess;
  if (schedule != PIC_SCHED_PLAIN) return launch_binned_step(a, order, sm_count, s, launches);
  switch (order) {
    case 1: return launch_p<1>(a, schedule, sm_count, s, launches);
    case 2: return launch_p<2>(a, schedule, sm_count, s, launches);
    case 3: return launch_p<3>(a, schedule, sm_count, s, launches);
    case 4: return launch_p<4>(a, schedule, sm_count, s, launches);
    case 5: return launch_p<5>(a, schedule, sm_count, s, launches);
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t launch_binned_step(const PushArgsMixed& a, int order, int sm_count, cudaStream_t main,
                               int* launches) {
  if (a.n <= 0) return cudaSuccess;
  switch (order) {
    case 1: return launch_binned_p<1>(a, sm_count, main, launches);
    case 2: return launch_binned_p<2>(a, sm_count, main, launches);
    case 3: return launch_binned_p<3>(a, sm_count, main, launches);
    case 4: return launch_binned_p<4>(a, sm_count, main, launches);
    case 5: return launch_binned_p<5>(a, sm_count, main, launches);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace pic
