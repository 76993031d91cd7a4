// Batched ensembles: many independent problems (each its own dt, dx, Psi_max,
// q/m, k cap and sub-step field-time reading, and its own field ring; one
// Lagrange order and window size for all) advanced together, one persistent
// launch per macro step, the mixed-precision binned push of push_mixed.cu per
// particle.
//
// Work items, from one atomic cursor:
//  1. deferred items (k >= kDeferMin) of every ensemble, largest k first;
//  2. stream chunks; a chunk never spans two ensembles, so a warp streams one
//     ensemble's particles at a time (k = 1, 2 go to the warp stashes, whose
//     entries remember their ensemble).
// The chunk length and the grid are launch parameters (tuned by
// pic_batch_autotune).
#include <math.h>
#include <string.h>

#include "pic_internal.h"
#include "push_device.cuh"

namespace pic {

// Field view of ensemble e for the current (prev = false) or previous step.
template <int P>
__device__ __forceinline__ void ens_fields(const BatchArgs& a, const EnsDev& e, bool prev,
                                           StepFields<P, true>& F) {
  const int64_t start = prev ? a.start_prev : a.start_cur;
  F.E.base = e.ringE + start * a.lstride;
  F.B.base = e.ringB + start * a.lstride;
  F.E.lstride = (int32_t)a.lstride;
  F.B.lstride = (int32_t)a.lstride;
  int64_t lo = INT64_MIN, hi = INT64_MAX;
#pragma unroll
  for (int l = 0; l <= P; ++l) {
    const int64_t o = e.slot_i0[(start + l) % a.R];
    lo = o > lo ? o : lo;
    hi = o + a.lstride - 1 < hi ? o + a.lstride - 1 : hi;
  }
  // the step's node table of this ensemble (batch_halfstep_kernel)
  F.coef = (prev ? a.coef_p : a.coef) + (int64_t)(&e - a.ens) * a.lstride * (2 * (P + 1));
  F.lo = (int32_t)lo;
  F.hi = (int32_t)hi;
}

__device__ __forceinline__ int64_t queue_slot(const BatchArgs& a, const EnsDev& e, int k,
                                              int64_t entry) {
  return 7 * e.first + (int64_t)(k - 1) * e.count + entry;
}

// Warp-aggregated enqueue into ensemble ens's queue of k (key = ens * 8 + k;
// key < 0: nothing).  All 32 lanes call this.
__device__ __forceinline__ void batch_enqueue(const BatchArgs& a, int key, int32_t i) {
  if (!__any_sync(0xffffffffu, key >= 0)) return;
  const unsigned peers = __match_any_sync(0xffffffffu, key);
  const int lane = threadIdx.x & 31;
  const int leader = __ffs(peers) - 1;
  int base = 0;
  if (key >= 0 && lane == leader) base = atomicAdd(&a.qcount_out[key], __popc(peers));
  base = __shfl_sync(0xffffffffu, base, leader);
  if (key >= 0) {
    const EnsDev& e = a.ens[key >> 3];
    a.queue_out[queue_slot(a, e, key & 7, base + __popc(peers & ((1u << lane) - 1u)))] = i;
  }
}

struct BatchStash {
  int32_t idx[kStashCap];
  int32_t cell[kStashCap];
  float frac[kStashCap], ux[kStashCap], uy[kStashCap], uz[kStashCap];
  uint8_t kp[kStashCap];
  uint16_t ens[kStashCap];
};

template <int P>
__device__ __forceinline__ void batch_stash_drain(const BatchArgs& a, BatchStash& S, int k, int& n,
                                                  int cnt, unsigned long long* sh) {
  const int lane = threadIdx.x & 31;
  if (lane < cnt) {
    const EnsDev& e = a.ens[S.ens[lane]];
    StepFields<P, true> F;
    ens_fields<P>(a, e, false, F);
    MixedState s = {S.cell[lane], S.frac[lane], S.ux[lane], S.uy[lane], S.uz[lane]};
    const int32_t i = S.idx[lane];
    const bool ok = subcycle_f32<P, true, true>(F, a.wtab, a.mask, e.dt, e.inv_dx, e.qm, e.field_time, a.mono,
                                    k, S.kp[lane], 0.f, s);
    normalize(s);
    a.cell[i] = s.cell;
    a.frac[i] = s.frac;
    a.px[i] = s.ux;
    a.py[i] = s.uy;
    a.pz[i] = s.uz;
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
    S.ens[lane] = S.ens[q];
  }
  __syncwarp();
  n = rest;
}

// Field view of macro step s of ensemble e from its mirrored ring and the
// device copy of its slots' window origins: for a deferred particle that runs
// behind the stream (no node table).
template <int P>
__device__ __forceinline__ StepFields<P, true> ens_step_fields(const BatchArgs& a, const EnsDev& e,
                                                               int64_t s) {
  StepFields<P, true> F;
  const int64_t R = a.R;
  const int64_t start = ((s - P) % R + R) % R;
  F.E.base = e.ringE + start * a.lstride;
  F.B.base = e.ringB + start * a.lstride;
  F.E.lstride = (int32_t)a.lstride;
  F.B.lstride = (int32_t)a.lstride;
  F.coef = nullptr;
  int64_t lo = INT64_MIN, hi = INT64_MAX;
#pragma unroll
  for (int l = 0; l <= P; ++l) {
    const int64_t o = e.slot_i0[(start + l) % R];
    lo = o > lo ? o : lo;
    hi = o + a.lstride - 1 < hi ? o + a.lstride - 1 : hi;
  }
  F.lo = (int32_t)lo;
  F.hi = (int32_t)hi;
  return F;
}

__device__ __forceinline__ void batch_defer_mark(const BatchArgs& a, int64_t i, int k_prev, int k,
                                                 int64_t s, int j = 0) {
  a.status[i] = (uint8_t)(k_prev | (k << 4));
  a.lag_step[i] = (int32_t)(s - a.step0);
  a.lag_j[i] = (uint16_t)j;
}

// Deferred particle i of ensemble ens (the batched form of heavy_particle):
// it is in step step0 + lag_step[i] with lag_j[i] of its sub-steps done.
// Finish that step and, if it ran behind the stream, every step up to the
// previous one (taking each step's criterion), spending at most heavy_budget
// sub-steps of long sub-cycles; then take the current step's criterion:
// pushed at once if k < kDeferMin, else deferred again.  Out of budget: it
// stays deferred where it is and resumes in the next launch.  finalize: bring
// it to the end of the last step only (public status).  key: ens * 8 + k of
// a re-deferral, else -1.
template <int P>
__device__ __forceinline__ void batch_heavy(const BatchArgs& a, int ens, int64_t i,
                                            const float* wcrit, ThreadCounters& tc,
                                            unsigned long long* sh, int& key) {
  key = -1;
  const EnsDev& e = a.ens[ens];
  StepFields<P, true> Fp, Fc;
  ens_fields<P>(a, e, true, Fp);
  ens_fields<P>(a, e, false, Fc);
  const uint8_t st = a.status[i];
  int k = deferred_k(st);
  int k_prev = st & 7;
  MixedState s = {a.cell[i], a.frac[i], a.px[i], a.py[i], a.pz[i]};
  int64_t si = a.step0 + a.lag_step[i];
  int j0 = a.lag_j[i];
  int budget = !a.finalize && a.heavy_budget > 0 ? a.heavy_budget : INT_MAX;
  float b0 = 0.f;  // the criterion's B_z of step si (used when k = 0)
  auto store = [&]() {
    a.cell[i] = s.cell;
    a.frac[i] = s.frac;
    a.px[i] = s.ux;
    a.py[i] = s.uy;
    a.pz[i] = s.uz;
  };
  auto lose = [&]() {
    store();
    a.status[i] = (uint8_t)(k | PIC_STATUS_LOST);
    atomicAdd(&sh[11], 1ull);
  };
  for (;;) {
    // sub-steps j0+1 .. j1 of step si
    const int m = 1 << (2 * k);
    int j1 = m;
    if (k >= kDeferMin && m - j0 > budget) j1 = j0 + budget;
    bool ok;
    if (si >= a.step_cur - 1) {  // the previous or the current step: node tables
      const StepFields<P, true> Fs = si == a.step_cur ? Fc : Fp;
      ok = subcycle_f32<P, true, true>(Fs, a.wtab, a.mask, e.dt, e.inv_dx, e.qm, e.field_time, a.mono,
                                       k, k_prev, b0, s, j0, j1);
    } else {
      const StepFields<P, true> Fs = ens_step_fields<P>(a, e, si);
      ok = subcycle_f32<P, true, false>(Fs, a.wtab, a.mask, e.dt, e.inv_dx, e.qm, e.field_time,
                                        a.mono, k, k_prev, b0, s, j0, j1);
    }
    if (k >= kDeferMin) budget -= j1 - j0;
    if (!ok) {
      lose();
      return;
    }
    if (j1 < m) {  // out of budget inside the sub-cycle: resume here next launch
      store();
      batch_defer_mark(a, i, k_prev, k, si, j1);
      key = ens * 8 + k;
      return;
    }
    normalize(s);
    if (si == a.step_cur) {  // the current step's short sub-cycle is done
      store();
      a.status[i] = (uint8_t)(k | (a.parity_next ? kParity : 0));
      return;
    }
    if (si == a.step_cur - 1) {
      if (a.finalize) {
        store();
        a.status[i] = (uint8_t)k;
        return;
      }
      int32_t je, jb;
      float we, wb;
      if (!tent_coords(s.cell, s.frac, Fc.lo, Fc.hi, je, we, jb, wb)) {
        lose();
        return;
      }
      bool capped;
      const int kn = criterion_f32<P>(Fc.B, wcrit, jb, wb, a.mask, s, e.qm_abs, e.dt, e.psi_max,
                                      e.k_max, capped, b0);
      count_step(tc, sh, kn, capped);
      if (kn >= kDeferMin) {
        store();
        batch_defer_mark(a, i, k, kn, a.step_cur);
        key = ens * 8 + kn;
        return;
      }
      // a short sub-cycle of the current step: the next pass of the loop
      k_prev = k;
      k = kn;
      si = a.step_cur;
      j0 = 0;
      continue;
    }
    // behind the stream: the next step's criterion, then its sub-cycle
    si += 1;
    const StepFields<P, true> Fs = si == a.step_cur - 1 ? Fp : ens_step_fields<P>(a, e, si);
    int32_t je, jb;
    float we, wb;
    if (!tent_coords(s.cell, s.frac, Fs.lo, Fs.hi, je, we, jb, wb)) {
      lose();
      return;
    }
    bool capped;
    const int kn = criterion_f32<P>(Fs.B, wcrit, jb, wb, a.mask, s, e.qm_abs, e.dt, e.psi_max,
                                    e.k_max, capped, b0);
    count_step(tc, sh, kn, capped);
    k_prev = k;
    k = kn;
    j0 = 0;
    if (k >= kDeferMin && budget <= 0) {
      store();
      batch_defer_mark(a, i, k_prev, k, si);
      key = ens * 8 + k;
      return;
    }
  }
}

// Every ensemble's window nodes at t_n (theta = 1/2 weights): the same FMA
// chain as a full gather takes at one node (see halfstep_kernel); and every
// node's monomial coefficients of the temporal interpolant (to_monomial, the
// values the sub-cycles would form from the levels), so that a sub-cycle reads
// two 16-byte rows per grid instead of forming them.
template <int P>
__global__ void batch_halfstep_kernel(BatchArgs a) {
  constexpr int stride = 2 * (P + 1);
  const float* wB = a.wtab + a.crit_row * stride + (P + 1);
  const float* wE = a.wtab + wrow(0, 1) * stride;
  const int64_t W = a.lstride;
  const int64_t total = (int64_t)a.n_ens * W;
  for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < total;
       q += (int64_t)gridDim.x * blockDim.x) {
    const EnsDev& e = a.ens[q / W];
    const int64_t c = q % W;
    const float* E = e.ringE + a.start_cur * W + c;
    const float* B = e.ringB + a.start_cur * W + c;
    float fe = __fmul_rn(wE[0], __ldg(E));
    float fb = __fmul_rn(wB[0], __ldg(B));
#pragma unroll
    for (int l = 1; l <= P; ++l) {
      fe = __fmaf_rn(wE[l], __ldg(E + l * W), fe);
      fb = __fmaf_rn(wB[l], __ldg(B + l * W), fb);
    }
    a.half[q] = fe;
    a.half[total + q] = fb;
    StepFields<P, true> F;
    F.E.base = e.ringE + a.start_cur * W;
    F.B.base = e.ringB + a.start_cur * W;
    F.E.lstride = (int32_t)W;
    F.B.lstride = (int32_t)W;
    float e0[P + 1], e1[P + 1], b0[P + 1], b1[P + 1];
    to_monomial<P>(F.E, (int32_t)c, (int32_t)c, a.mono[0], e0, e1);
    to_monomial<P>(F.B, (int32_t)c, (int32_t)c, a.mono[1], b0, b1);
    float* r = a.coef + q * stride;
#pragma unroll
    for (int k = 0; k <= P; ++k) {
      r[k] = e0[k];
      r[P + 1 + k] = b0[k];
    }
  }
}

// Heavy-item prefix: items of (k, ensemble) in the order k = 7..1, ensemble
// ascending; prefix[q] = first item of entry q, prefix[7 * n_ens] = total.
__global__ void batch_prefix_kernel(const int32_t* qcount_in, int32_t n_ens, int32_t k_lo,
                                    int64_t* prefix) {
  __shared__ long long part[1024];
  const int n = 7 * n_ens;
  const int per = (n + blockDim.x - 1) / blockDim.x;
  const int q0 = threadIdx.x * per;
  long long sum = 0;
  for (int q = q0; q < q0 + per && q < n; ++q) {
    const int k = 7 - q / n_ens, e = q % n_ens;
    sum += k >= k_lo ? ((long long)qcount_in[e * 8 + k] + 31) / 32 : 0;
  }
  part[threadIdx.x] = sum;
  __syncthreads();
  if (threadIdx.x == 0) {
    long long acc = 0;
    for (int t = 0; t < (int)blockDim.x; ++t) {
      const long long v = part[t];
      part[t] = acc;
      acc += v;
    }
  }
  __syncthreads();
  long long acc = part[threadIdx.x];
  for (int q = q0; q < q0 + per && q < n; ++q) {
    prefix[q] = acc;
    const int k = 7 - q / n_ens, e = q % n_ens;
    acc += k >= k_lo ? ((long long)qcount_in[e * 8 + k] + 31) / 32 : 0;
  }
  if (threadIdx.x == blockDim.x - 1) prefix[n] = acc;
}

// Block shape of the batched kernel: four blocks of five warps per SM (20
// warps at <= 102 registers, 93 used), measured faster than two of eight
// (16 warps; 104 registers), three of six (18) and three of seven (21, with
// spills) on the 512-ensemble workload: its serial sub-cycle chains want warps.
#ifndef PIC_BATCH_THREADS
#define PIC_BATCH_THREADS 160
#endif
constexpr int kBatchThreads = PIC_BATCH_THREADS;
constexpr int kBatchWarps = kBatchThreads / 32;
#ifndef PIC_BATCH_MIN_BLOCKS
#define PIC_BATCH_MIN_BLOCKS 4
#endif

template <int P>
__global__ void __launch_bounds__(kBatchThreads, PIC_BATCH_MIN_BLOCKS) push_batch_kernel(BatchArgs a) {
  extern __shared__ __align__(16) unsigned char smem[];
  BatchStash* stashes = reinterpret_cast<BatchStash*>(smem);  // [kBatchWarps][kStashK]
  __shared__ unsigned long long sh[12];
  __shared__ int s_task[kBatchWarps];
  if (threadIdx.x < 12) sh[threadIdx.x] = 0ull;
  __syncthreads();
  constexpr int stride = 2 * (P + 1);
  const float* wcrit = a.wtab + a.crit_row * stride + (P + 1);
  const float* w0 = a.wtab + wrow(0, 1) * stride;
  ThreadCounters tc;
  const int lane = threadIdx.x & 31;
  const int warp = threadIdx.x >> 5;
  BatchStash* my_stash = stashes + warp * kStashK;
  int stash_n[kStashK];
#pragma unroll
  for (int q = 0; q < kStashK; ++q) stash_n[q] = 0;
  const uint8_t want = a.parity_cur ? kParity : 0;
  const uint8_t done = a.parity_next ? kParity : 0;
  const int64_t n_heavy = a.prefix[7 * a.n_ens];
  const int64_t n_items = n_heavy + (a.finalize ? 0 : a.n_chunks);
  const int per_lane = a.chunk / 32;

  for (;;) {
    if (lane == 0) s_task[warp] = atomicAdd(a.cursor, 1);
    __syncwarp();
    const int64_t t = s_task[warp];
    __syncwarp();
    if (t >= n_items) break;
    if (t < n_heavy) {
      int lo = 0, hi = 7 * a.n_ens - 1;  // last entry q with prefix[q] <= t
      while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (a.prefix[mid] <= t) lo = mid; else hi = mid - 1;
      }
      const int k = 7 - lo / a.n_ens, ens = lo % a.n_ens;
      const int64_t entry = (t - a.prefix[lo]) * 32 + lane;
      int key = -1;
      int32_t i = 0;
      if (entry < a.qcount_in[ens * 8 + k]) {
        i = a.queue_in[queue_slot(a, a.ens[ens], k, entry)];
        batch_heavy<P>(a, ens, i, wcrit, tc, sh, key);
      }
      batch_enqueue(a, key, i);
      continue;
    }
    // stream chunk: which ensemble, which particles
    const int64_t c = t - n_heavy;
    int lo = 0, hi = a.n_ens - 1;
    while (lo < hi) {
      const int mid = (lo + hi + 1) >> 1;
      if (a.ens[mid].chunk_first <= c) lo = mid; else hi = mid - 1;
    }
    const int ens = lo;
    const EnsDev& e = a.ens[ens];
    StepFields<P, true> F;
    ens_fields<P>(a, e, false, F);
    const float hx0 = __fmul_rn(e.dt, e.inv_dx);
    const int64_t first = e.first + (c - e.chunk_first) * a.chunk;
    const int64_t end = e.first + e.count;
    int64_t i = first + lane;
    uint8_t st = PIC_STATUS_LOST;
    MixedState s = {0, 0.5f, 0.f, 0.f, 0.f};
    if (i < end) {
      st = a.status[i];
      s = {a.cell[i], a.frac[i], a.px[i], a.py[i], a.pz[i]};
    }
#pragma unroll 1
    for (int r = 0; r < per_lane; ++r, i += 32) {
      const int64_t inext = i + 32;
      uint8_t st_n = PIC_STATUS_LOST;
      MixedState s_n = {0, 0.5f, 0.f, 0.f, 0.f};
      if (r + 1 < per_lane && inext < end) {
        st_n = a.status[inext];
        s_n = {a.cell[inext], a.frac[inext], a.px[inext], a.py[inext], a.pz[inext]};
      }
      const bool mine = i < end && !(st & PIC_STATUS_LOST) && !(st & kDeferMask) &&
                        ((st & kParity) == want);
      int key = -1, sk = 0;
      if (mine) {
        int32_t je, jb;
        float we, wb;
        const bool inwin = tent_coords(s.cell, s.frac, F.lo, F.hi, je, we, jb, wb);
        const float* hE = a.half + (int64_t)ens * a.lstride;
        const float* hB = hE + (int64_t)a.n_ens * a.lstride;
        const float f0b = __ldg(hB + (jb & a.mask)), f1b = __ldg(hB + ((jb + 1) & a.mask));
        const float f0e = __ldg(hE + (je & a.mask)), f1e = __ldg(hE + ((je + 1) & a.mask));
        const float b0 = __fmaf_rn(wb, __fsub_rn(f1b, f0b), f0b);
        const float ey = __fmaf_rn(we, __fsub_rn(f1e, f0e), f0e);
        if (!inwin) {
          a.status[i] = (uint8_t)(st | PIC_STATUS_LOST);
          atomicAdd(&sh[11], 1ull);
        } else {
          bool capped;
          const int k = psi_to_k(b0, s, e.qm_abs, e.dt, e.psi_max, e.k_max, capped);
          count_step(tc, sh, k, capped);
          const int k_prev = st & 7;
          if (k == 0) {
            const float h_old = pow4_down(e.dt, k_prev);
            const float hp = __fmul_rn(0.5f, __fadd_rn(h_old, e.dt));
            boris_f32(ey, b0, hp, hx0, e.qm, s);
            normalize(s);
            a.cell[i] = s.cell;
            a.frac[i] = s.frac;
            a.px[i] = s.ux;
            a.py[i] = s.uy;
            a.pz[i] = s.uz;
            a.status[i] = done;
          } else if (k < kDeferMin) {
            sk = k;
          } else {
            batch_defer_mark(a, i, k_prev, k, a.step_cur);
            key = ens * 8 + k;
          }
        }
      }
      batch_enqueue(a, key, (int32_t)i);
#pragma unroll
      for (int q = 0; q < kStashK; ++q) {
        const unsigned m = __ballot_sync(0xffffffffu, sk == q + 1);
        if (m == 0u) continue;
        BatchStash& S = my_stash[q];
        if (sk == q + 1) {
          const int pos = stash_n[q] + __popc(m & ((1u << lane) - 1u));
          S.idx[pos] = (int32_t)i;
          S.cell[pos] = s.cell;
          S.frac[pos] = s.frac;
          S.ux[pos] = s.ux;
          S.uy[pos] = s.uy;
          S.uz[pos] = s.uz;
          S.kp[pos] = (uint8_t)(st & 7);
          S.ens[pos] = (uint16_t)ens;
        }
        stash_n[q] += __popc(m);
        __syncwarp();
        if (stash_n[q] >= 32) batch_stash_drain<P>(a, S, q + 1, stash_n[q], 32, sh);
      }
      st = st_n;
      s = s_n;
    }
  }
#pragma unroll
  for (int q = 0; q < kStashK; ++q)
    if (stash_n[q] > 0) batch_stash_drain<P>(a, my_stash[q], q + 1, stash_n[q], stash_n[q], sh);
  flush_counters(tc, sh, a.stats);

  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    const unsigned fin = atomicAdd(a.blocks_done, 1u);
    if (fin == gridDim.x - 1) {
      __threadfence();
      *a.cursor = 0;
      *a.blocks_done = 0;
      for (int q = 0; q < 8 * a.n_ens; ++q) a.qcount_in[q] = 0;
      __threadfence();
    }
  }
}

__global__ void batch_reset_status_kernel(uint8_t* status, int64_t n) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const uint8_t st = status[i];
    const uint8_t pub = (uint8_t)(st & (PIC_STATUS_LOST | 7));
    if (pub != st) status[i] = pub;
  }
}

constexpr size_t kBatchStashBytes = sizeof(BatchStash) * kBatchWarps * kStashK;

static_assert(kBatchStashBytes <= 48 * 1024, "stashes must fit the default shared-memory limit");

template <int P>
static cudaError_t launch_batch_p(const BatchArgs& a, int blocks, cudaStream_t s, int* launches) {
  batch_prefix_kernel<<<1, 1024, 0, s>>>(a.qcount_in, a.n_ens, a.finalize ? 1 : kDeferMin,
                                         const_cast<int64_t*>(a.prefix));
  int n = 2;
  if (!a.finalize) {
    const int64_t total = (int64_t)a.n_ens * a.lstride;
    const int64_t want = (total + 255) / 256;
    batch_halfstep_kernel<P><<<(int)(want < 152 * 16 ? want : 152 * 16), 256, 0, s>>>(a);
    ++n;
  }
  push_batch_kernel<P><<<blocks, kBatchThreads, kBatchStashBytes, s>>>(a);
  if (a.finalize) {
    const int64_t want = (a.n_total + 255) / 256;
    batch_reset_status_kernel<<<(int)(want < 152 * 8 ? want : 152 * 8), 256, 0, s>>>(a.status,
                                                                                    a.n_total);
    ++n;
  }
  if (launches) *launches += n;
  return cudaGetLastError();
}

cudaError_t launch_batch_step(const BatchArgs& a, int order, int blocks, cudaStream_t s,
                              int* launches) {
  if (a.n_total <= 0) return cudaSuccess;
  switch (order) {
    case 1: return launch_batch_p<1>(a, blocks, s, launches);
    case 2: return launch_batch_p<2>(a, blocks, s, launches);
    case 3: return launch_batch_p<3>(a, blocks, s, launches);
    case 4: return launch_batch_p<4>(a, blocks, s, launches);
    case 5: return launch_batch_p<5>(a, blocks, s, launches);
    default: return cudaErrorInvalidValue;
  }
}

int batch_max_blocks_per_sm(int order) {
  int occ = 0;
  switch (order) {
    case 1: cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, push_batch_kernel<1>, kBatchThreads, kBatchStashBytes); break;
    case 2: cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, push_batch_kernel<2>, kBatchThreads, kBatchStashBytes); break;
    case 3: cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, push_batch_kernel<3>, kBatchThreads, kBatchStashBytes); break;
    case 4: cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, push_batch_kernel<4>, kBatchThreads, kBatchStashBytes); break;
    case 5: cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, push_batch_kernel<5>, kBatchThreads, kBatchStashBytes); break;
    default: break;
  }
  return occ > 0 ? occ : 1;
}

// Window of a level for every ensemble: Ey[e][c], Bz[e][c] -> ensemble e's
// mirrored ring, slot and slot + R; the slot's origin recorded on the device.
__global__ void batch_scatter_kernel(const EnsDev* ens, int32_t n_ens, int64_t slot, int64_t R,
                                     int64_t W, const double* Ey, const double* Bz,
                                     const int64_t* i0, int64_t* slot_i0_all) {
  const int64_t total = (int64_t)n_ens * W;
  for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < total;
       q += (int64_t)gridDim.x * blockDim.x) {
    const int e = (int)(q / W);
    const int64_t c = q % W;
    const int64_t pos = (i0[e] + c) & (W - 1);
    float* rE = const_cast<float*>(ens[e].ringE);
    float* rB = const_cast<float*>(ens[e].ringB);
    const float ev = (float)Ey[q], bv = (float)Bz[q];
    rE[slot * W + pos] = ev;
    rE[(slot + R) * W + pos] = ev;
    rB[slot * W + pos] = bv;
    rB[(slot + R) * W + pos] = bv;
    if (c == 0) slot_i0_all[(int64_t)e * R + slot] = i0[e];
  }
}

cudaError_t launch_batch_scatter(const EnsDev* ens, int32_t n_ens, int64_t slot, int64_t R,
                                 int64_t W, const double* Ey, const double* Bz, const int64_t* i0,
                                 int64_t* slot_i0_all, cudaStream_t s) {
  const int64_t total = (int64_t)n_ens * W;
  const int64_t want = (total + 255) / 256;
  batch_scatter_kernel<<<(int)(want < 152 * 16 ? want : 152 * 16), 256, 0, s>>>(
      ens, n_ens, slot, R, W, Ey, Bz, i0, slot_i0_all);
  return cudaGetLastError();
}

}  // namespace pic
