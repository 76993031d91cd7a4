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
//          The bulk streams every particle through tiles staged in shared
//          memory by bulk copies (two particles per lane per round); a particle
//          whose criterion gives k = 0 is pushed at once, one with k = 1, 2 is
//          parked in a per-warp stash and pushed with 31 others, one with
//          k >= 3 is compacted (warp match + one atomic per k) into the queue
//          of its k and its sub-cycling is deferred.  The first work items of
//          the next step's kernel drain those queues, largest k first, in warps
//          of equal k: each deferred particle finishes its previous step (at
//          most a budget of sub-steps per launch) and then takes its own
//          criterion for the current one.  So the long sub-cycled pushes run
//          concurrently with the HBM stream of the next step instead of after
//          it.  A closing kernel finishes what the last step deferred.
//
// Status byte inside a binned call: bits 0-2 = k_prev, bit 3 = step parity
// (the bulk of step j only takes particles whose parity equals j & 1 and flips
// it), bits 4-6 = deferred k (0 = none), bit 7 = lost.  Outside a call the
// byte is in the public form (bits 0-6 = k).
#include <limits.h>
#include <math.h>

#include "pic_internal.h"
#include "push_device.cuh"

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

// ---------------------------------------------------------------- half-step fields

// Every window node's E_y and B_z interpolated to t_n with the theta = 1/2
// weights: the same FMA chain over the same levels as gather_f32 takes at one
// node, so an m = 1 push (and the criterion) that reads these two nodes and
// applies the tent weight gets exactly the bits of the full gather, from two
// loads per grid instead of 2(p+1).
//
// With coef set, the same pass also writes each node's monomial coefficients
// (to_monomial over the same levels, so the same bits): E_y's p+1 then B_z's.
template <int P>
__global__ void halfstep_kernel(PushArgsMixed a, int64_t W, float* outE, float* outB, float* coef) {
  constexpr int stride = 2 * (P + 1);
  const float* wB = a.wtab + a.crit_row * stride + (P + 1);
  const float* wE = a.wtab + wrow(0, 1) * stride;
  StepFields<P, true> F;
  load_fields<P, true>(F, a, false);
  for (int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; c < W;
       c += (int64_t)gridDim.x * blockDim.x) {
    float fe = __fmul_rn(wE[0], __ldg(F.E.at(0) + c));
    float fb = __fmul_rn(wB[0], __ldg(F.B.at(0) + c));
#pragma unroll
    for (int l = 1; l <= P; ++l) {
      fe = __fmaf_rn(wE[l], __ldg(F.E.at(l) + c), fe);
      fb = __fmaf_rn(wB[l], __ldg(F.B.at(l) + c), fb);
    }
    outE[c] = fe;
    outB[c] = fb;
    if (c == 0) {  // padding node W: the circular successor of node W - 1
      outE[W] = fe;
      outB[W] = fb;
    }
    if (coef) {
      float e0[P + 1], e1[P + 1], b0[P + 1], b1[P + 1];
      to_monomial<P>(F.E, (int32_t)c, (int32_t)c, a.mono[0], e0, e1);
      to_monomial<P>(F.B, (int32_t)c, (int32_t)c, a.mono[1], b0, b1);
      float* r = coef + c * stride;
#pragma unroll
      for (int q = 0; q <= P; ++q) {
        r[q] = e0[q];
        r[P + 1 + q] = b0[q];
      }
    }
  }
}

cudaError_t launch_halfstep(const PushArgsMixed& a, int order, int64_t W, float* outE, float* outB,
                            float* coef, cudaStream_t s) {
  const int64_t want = (W + 255) / 256;
  const int blocks = (int)(want < 152 * 8 ? want : 152 * 8);
  switch (order) {
    case 1: halfstep_kernel<1><<<blocks, 256, 0, s>>>(a, W, outE, outB, coef); break;
    case 2: halfstep_kernel<2><<<blocks, 256, 0, s>>>(a, W, outE, outB, coef); break;
    case 3: halfstep_kernel<3><<<blocks, 256, 0, s>>>(a, W, outE, outB, coef); break;
    case 4: halfstep_kernel<4><<<blocks, 256, 0, s>>>(a, W, outE, outB, coef); break;
    case 5: halfstep_kernel<5><<<blocks, 256, 0, s>>>(a, W, outE, outB, coef); break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

// Tent interpolation of a half-step field between nodes j, j+1.  The array
// holds W + 1 nodes, node W repeating node 0, so the pair never wraps.
__device__ __forceinline__ float half_lerp(const float* f, int32_t j, float w, int32_t mask) {
  const float* q = f + (j & mask);
  const float f0 = __ldg(q);
  const float f1 = __ldg(q + 1);
  return __fmaf_rn(w, __fsub_rn(f1, f0), f0);
}

// ---------------------------------------------------------------- PLAIN schedule

template <int P, bool RING>
__global__ void __launch_bounds__(256) push_mixed_plain_kernel(PushArgsMixed a) {
  __shared__ unsigned long long sh[12];
  if (threadIdx.x < 12) sh[threadIdx.x] = 0ull;
  __syncthreads();
  constexpr int stride = 2 * (P + 1);
  const float* wcrit = a.wtab + a.crit_row * stride + (P + 1);
  StepFields<P, RING> F;
  load_fields<P, RING>(F, a, false);
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
    int k;
    if (a.halfE) {
      b0 = half_lerp(a.halfB, jb, wb, a.mask);
      k = psi_to_k(b0, s, a.qm_abs, a.dt, a.psi_max, a.k_max, capped);
    } else {
      k = criterion_f32<P>(F.B, wcrit, jb, wb, a.mask, s, a.qm_abs, a.dt, a.psi_max, a.k_max,
                           capped, b0);
    }
    count_step(tc, sh, k, capped);
    bool ok = true;
    if (k == 0 && a.halfE) {
      const float h_old = pow4_down(a.dt, st & 0x7f);
      const float hp = __fmul_rn(0.5f, __fadd_rn(h_old, a.dt));
      boris_f32(half_lerp(a.halfE, je, we, a.mask), b0, hp, __fmul_rn(a.dt, a.inv_dx), a.qm, s);
    } else {
      ok = subcycle_f32<P>(F, a.wtab, a.mask, a.dt, a.inv_dx, a.qm, a.field_time, a.mono, k,
                           st & 0x7f, b0, s);
    }
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
//  2. predicted items (predicted schedule only): particles binned at the last
//     refresh of the predictions by the predictor's k (k >= kPredMinK),
//     largest k first; the queue is kept, and its marked particles pushed by
//     every launch, until the next refresh.  Each takes its exact criterion;
//     k = 0 and a short k equal to the predicted one are pushed at once (so a
//     warp of right predictions is dense), another short k goes to the stash,
//     both staying in the queue; a long sub-cycle starts at once (resumable)
//     and leaves the queue; a wrong prediction costs one idle lane.
//  3. stream chunks of kChunk particles, staged into shared memory tile by
//     tile with bulk copies (one tile in flight while another is pushed),
//     two particles per lane per round.  k = 0: pushed at once (the
//     criterion's B_z serves the push).  k = 1, 2: parked in the warp's stash
//     for that k (shared memory); whenever a stash holds 32 particles the warp
//     pushes them together, so short sub-cycles never diverge a warp and never
//     leave the chip.  k >= kDeferMin: compacted into the queue of its k (one
//     atomic per distinct k per warp) and deferred to the next launch.
// Status byte inside a binned call: bits 0-2 = k_prev, bit 3 = step parity
// (the stream of step j takes particles whose parity equals j & 1 and flips
// it), bits 4-6 = deferred k (0 = none), bit 7 = lost.

// At a refresh of the predictions, before the step's launch: the predicted
// queue is rebuilt.  Every particle of the old queue leaves it (its mark is
// cleared); every particle the stream would take this step and whose predicted
// k is >= min_k joins the queue of that k and is marked (deferred-k field 1),
// so the streams leave it to the predicted items until the next refresh.
// pred_count must be zero on entry.
__global__ void bin_predicted_kernel(const uint8_t* pred, uint8_t* status, int64_t n,
                                     int parity_cur, int min_k, int32_t* pred_queue,
                                     int32_t* pred_count, int64_t qcap) {
  __shared__ int blk_cnt[8];   // this pass's binned particles per k (block-wide)
  __shared__ int blk_base[8];  // their start in the queue of k
  const uint8_t want = parity_cur ? kParity : 0;
  // Sixteen particles per thread per pass: one 16-byte load of each byte
  // array, so enough bytes are in flight.  Passes with a binned particle
  // (rare) reserve the block's queue slots with one global atomic per k.
  const int64_t n_vec = (n + 15) / 16;
  for (int64_t v0 = (int64_t)blockIdx.x * blockDim.x; v0 < n_vec;
       v0 += (int64_t)gridDim.x * blockDim.x) {
    const int64_t v = v0 + threadIdx.x;
    const int64_t i0 = 16 * v;
    uint32_t sw[4] = {0x80808080u, 0x80808080u, 0x80808080u, 0x80808080u};  // lost: skipped
    uint32_t pw[4] = {0u, 0u, 0u, 0u};
    if (i0 + 16 <= n) {
      const uint4 a4 = reinterpret_cast<const uint4*>(status)[v];
      const uint4 b4 = reinterpret_cast<const uint4*>(pred)[v];
      sw[0] = a4.x; sw[1] = a4.y; sw[2] = a4.z; sw[3] = a4.w;
      pw[0] = b4.x; pw[1] = b4.y; pw[2] = b4.z; pw[3] = b4.w;
    } else if (i0 < n) {
      for (int q = 0; q < 16 && i0 + q < n; ++q) {
        const int sh8 = 8 * (q & 3);
        sw[q >> 2] = (sw[q >> 2] & ~(0xffu << sh8)) | ((uint32_t)status[i0 + q] << sh8);
        pw[q >> 2] |= (uint32_t)pred[i0 + q] << sh8;
      }
    }
    int keys[16];
    bool any = false;
    uint32_t nw[4] = {sw[0], sw[1], sw[2], sw[3]};  // the bytes after this pass
#pragma unroll
    for (int q = 0; q < 16; ++q) {
      const int sh8 = 8 * (q & 3);
      uint8_t st = (uint8_t)(sw[q >> 2] >> sh8);
      const int kp = (int)((pw[q >> 2] >> sh8) & 0xffu);
      if ((st & kDeferMask) == kOwned) st = (uint8_t)(st & ~kDeferMask);  // leaves the old queue
      keys[q] = ((st & (PIC_STATUS_LOST | kDeferMask | kParity)) == want && kp >= min_k && kp <= 7)
                    ? kp
                    : 0;
      if (keys[q]) st = (uint8_t)(st | kOwned);
      nw[q >> 2] = (nw[q >> 2] & ~(0xffu << sh8)) | ((uint32_t)st << sh8);
      any |= keys[q] != 0;
    }
    if (__syncthreads_or(any)) {
      if (threadIdx.x < 8) blk_cnt[threadIdx.x] = 0;
      __syncthreads();
      int off[16];
#pragma unroll
      for (int q = 0; q < 16; ++q) off[q] = keys[q] ? atomicAdd(&blk_cnt[keys[q]], 1) : 0;
      __syncthreads();
      if (threadIdx.x > 0 && threadIdx.x < 8 && blk_cnt[threadIdx.x] > 0)
        blk_base[threadIdx.x] = atomicAdd(&pred_count[threadIdx.x], blk_cnt[threadIdx.x]);
      __syncthreads();
#pragma unroll
      for (int q = 0; q < 16; ++q)
        if (keys[q])
          pred_queue[(int64_t)(keys[q] - 1) * qcap + blk_base[keys[q]] + off[q]] = (int32_t)(i0 + q);
      __syncthreads();  // blk_cnt / blk_base are reused by the next pass
    }
    if ((nw[0] ^ sw[0]) | (nw[1] ^ sw[1]) | (nw[2] ^ sw[2]) | (nw[3] ^ sw[3])) {
      if (i0 + 16 <= n) {
        reinterpret_cast<uint4*>(status)[v] = make_uint4(nw[0], nw[1], nw[2], nw[3]);
      } else {
        for (int q = 0; q < 16 && i0 + q < n; ++q)
          if (((nw[q >> 2] ^ sw[q >> 2]) >> (8 * (q & 3))) & 0xffu)
            status[i0 + q] = (uint8_t)(nw[q >> 2] >> (8 * (q & 3)));
      }
    }
  }
}

cudaError_t launch_bin_predicted(const uint8_t* pred, uint8_t* status, int64_t n, int parity_cur,
                                 int min_k, int32_t* pred_queue, int32_t* pred_count, int64_t qcap,
                                 cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  const int64_t want = (n + 4095) / 4096;
  const int blocks = (int)(want < 152 * 8 ? want : 152 * 8);
  bin_predicted_kernel<<<blocks, 256, 0, s>>>(pred, status, n, parity_cur, min_k < 1 ? 1 : min_k,
                                              pred_queue, pred_count, qcap);
  return cudaGetLastError();
}

// Dynamic shared memory of the binned kernel: the warps' stashes, then their
// staged stream tiles.
constexpr size_t kStashBytes = sizeof(Stash) * kWarps * kStashK;
constexpr size_t kBinnedSmem = kStashBytes + sizeof(Tile) * kWarps * kStages;
static_assert(kStashBytes % 128 == 0, "tiles start on a 128-byte boundary");

// Two resident blocks per SM (of kThreads each): measured faster than three,
// whose register cap costs instructions and whose extra warps contend for the
// instruction cache across the kernel's stream, stash and deferred-particle
// code.
#ifndef PIC_BINNED_MIN_BLOCKS
#define PIC_BINNED_MIN_BLOCKS 2
#endif

template <int P, bool RING>
__global__ void __launch_bounds__(kThreads, PIC_BINNED_MIN_BLOCKS) push_binned_kernel(PushArgsMixed a) {
  extern __shared__ __align__(128) unsigned char smem[];
  Stash* stashes = reinterpret_cast<Stash*>(smem);  // [kWarps][kStashK]
  Tile* tiles = reinterpret_cast<Tile*>(smem + kStashBytes);  // [kWarps][kStages]
  __shared__ __align__(8) uint64_t bars[kWarps * kStages];
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
  StepFields<P, RING> F, Fp;
  load_fields<P, RING>(F, a, false);
  load_fields<P, RING>(Fp, a, true);
  ThreadCounters tc;
  const int lane = threadIdx.x & 31;
  const int warp = threadIdx.x >> 5;
  Stash* my_stash = stashes + warp * kStashK;
  Tile* my_tiles = tiles + warp * kStages;
  uint64_t* my_bars = bars + warp * kStages;
  uint32_t phase = 0;  // bit s: parity of stage s's next completion
  if (lane == 0) {
#pragma unroll
    for (int sidx = 0; sidx < kStages; ++sidx) mbar_init(my_bars + sidx);
    mbar_init_fence();
  }
  __syncwarp();
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

  // the stashes' fill counts, read and written at a run-time stash index
  auto stash_count = [&](int q) {
    int v = 0;
#pragma unroll
    for (int r = 0; r < kStashK; ++r)
      if (r == q) v = stash_n[r];
    return v;
  };
  auto stash_set = [&](int q, int v) {
#pragma unroll
    for (int r = 0; r < kStashK; ++r)
      if (r == q) stash_n[r] = v;
  };
  // push 32 particles of every stash that holds 32 or more (all = true: every
  // parked particle); one call site of the sub-cycle per call site of this
  auto drain = [&](bool all) {
#pragma unroll 1
    for (int q = 0; q < kStashK; ++q) {
      int n = stash_count(q);
      const int cnt = all ? n : (n >= 32 ? 32 : 0);
      if (cnt > 0) {
        stash_drain<P, RING>(a, F, my_stash[q], q + 1, n, cnt, sh);
        stash_set(q, n);
      }
    }
  };

  // park k = 1, 2 in the warp's stashes; push a stash when it holds 32
  // (warp-collective; sk = 0: nothing to park)
  auto park = [&](int sk, int32_t i, const MixedState& s, uint8_t kp) {
    bool full = false;
#pragma unroll
    for (int q = 0; q < kStashK; ++q) {
      const unsigned m = __ballot_sync(0xffffffffu, sk == q + 1);
      if (m == 0u) continue;
      Stash& S = my_stash[q];
      if (sk == q + 1) {
        const int pos = stash_n[q] + __popc(m & ((1u << lane) - 1u));
        S.idx[pos] = i;
#ifndef PIC_STASH_INDEX_ONLY
        S.cell[pos] = s.cell;
        S.frac[pos] = s.frac;
        S.ux[pos] = s.ux;
        S.uy[pos] = s.uy;
        S.uz[pos] = s.uz;
#endif
        S.kp[pos] = kp;
      }
      stash_n[q] += __popc(m);
      full |= stash_n[q] >= 32;
    }
    __syncwarp();
    if (full) drain(false);
  };

  constexpr uint8_t kStreamMask = PIC_STATUS_LOST | kDeferMask | kParity;
  // One stream round of 64 particles, two per lane (particles first+2q and
  // first+2q+1, q = 32 r + lane), from the staged tile or, for the array's
  // tail and unaligned arrays, from global memory: the criterion, then push
  // (k = 0), park (k = 1, 2) or defer (k >= kDeferMin).  The k = 0 arithmetic
  // runs on both particles at once with paired FP32 instructions (the bits of
  // boris_f32, so the same bits as the other schedules).  A round in which
  // every particle takes k = 0 (or is not the stream's) -- nearly all of them
  // -- skips the cap test, the queues and the stashes.  Warp-collective.
  const float qm_dt = __fmul_rn(a.qm_abs, a.dt);
  const float tp = __fmul_rn(2.0f, a.psi_max);
  const float tp2 = __fmul_rn(tp, tp);
  auto stream_pair = [&](const Tile& T, bool staged, int r, uint32_t first) {
    const int q = r * 32 + lane;
    const uint32_t i = first + 2u * (uint32_t)q;
    uint8_t st0, st1;
    MixedState2 s;
    if (staged) {
      const uint32_t st2 = reinterpret_cast<const uint16_t*>(T.st)[q];
      st0 = (uint8_t)st2;
      st1 = (uint8_t)(st2 >> 8);
      s.cell = reinterpret_cast<const int2*>(T.cell)[q];
      s.frac = reinterpret_cast<const float2*>(T.frac)[q];
      s.ux = reinterpret_cast<const float2*>(T.px)[q];
      s.uy = reinterpret_cast<const float2*>(T.py)[q];
      s.uz = reinterpret_cast<const float2*>(T.pz)[q];
    } else {
      MixedState u0, u1;
      fetch_stream(a, i, st0, u0);  // past the end: lost
      fetch_stream(a, i + 1, st1, u1);
      s.cell = make_int2(u0.cell, u1.cell);
      s.frac = make_float2(u0.frac, u1.frac);
      s.ux = make_float2(u0.ux, u1.ux);
      s.uy = make_float2(u0.uy, u1.uy);
      s.uz = make_float2(u0.uz, u1.uz);
    }
    const bool mine0 = (st0 & kStreamMask) == want, mine1 = (st1 & kStreamMask) == want;
    const float2 fe = floor2(s.frac);  // tent_coords of each
    const float2 fbm = add2(s.frac, bc2(-0.5f));
    const float2 fb = floor2(fbm);
    const float2 we = sub2(s.frac, fe), wb = sub2(fbm, fb);
    const int32_t je0 = s.cell.x + (int32_t)fe.x, je1 = s.cell.y + (int32_t)fe.y;
    const int32_t jb0 = s.cell.x + (int32_t)fb.x, jb1 = s.cell.y + (int32_t)fb.y;
    const bool in0 = jb0 >= F.lo && je0 < F.hi, in1 = jb1 >= F.lo && je1 < F.hi;
    float2 ey, bz;  // half_lerp of each, or gather_f32 without half-step fields
    if (a.halfE) {
      const float* e0 = a.halfE + (je0 & a.mask);
      const float* e1 = a.halfE + (je1 & a.mask);
      const float* b0 = a.halfB + (jb0 & a.mask);
      const float* b1 = a.halfB + (jb1 & a.mask);
      const float2 elo = make_float2(__ldg(e0), __ldg(e1));
      const float2 ehi = make_float2(__ldg(e0 + 1), __ldg(e1 + 1));
      const float2 blo = make_float2(__ldg(b0), __ldg(b1));
      const float2 bhi = make_float2(__ldg(b0 + 1), __ldg(b1 + 1));
      ey = fma2(we, sub2(ehi, elo), elo);
      bz = fma2(wb, sub2(bhi, blo), blo);
    } else {
      ey = make_float2(gather_f32<P>(F.E, w0, je0, we.x, a.mask),
                       gather_f32<P>(F.E, w0, je1, we.y, a.mask));
      bz = make_float2(gather_f32<P>(F.B, wcrit, jb0, wb.x, a.mask),
                       gather_f32<P>(F.B, wcrit, jb1, wb.y, a.mask));
    }
    const float2 av = mul2(bc2(qm_dt), bz);  // psi_terms of each
    const float2 a2 = mul2(av, av);
    const float2 rhs =
        mul2(bc2(tp2), add2(bc2(1.0f), fma2(s.uz, s.uz, fma2(s.uy, s.uy, mul2(s.ux, s.ux)))));
    bool push0 = mine0 && in0 && !(a2.x > rhs.x);
    bool push1 = mine1 && in1 && !(a2.y > rhs.y);
    tc.k0 += (push0 ? 1u : 0u) + (push1 ? 1u : 0u);
    const bool side = !__all_sync(0xffffffffu, (push0 || !mine0) && (push1 || !mine1));
    int key0 = 0, key1 = 0, sk0 = 0, sk1 = 0;
    if (side) {  // the rest of the criterion for the particles that do not take k = 0 at once
#pragma unroll 1
      for (int e = 0; e < 2; ++e) {
        const bool mine = e ? mine1 : mine0;
        bool& push = e ? push1 : push0;
        const bool inwin = e ? in1 : in0;
        const uint8_t st = e ? st1 : st0;
        const uint32_t ii = i + (uint32_t)e;
        int& key = e ? key1 : key0;
        int& sk = e ? sk1 : sk0;
        if (!mine || push) continue;
        if (!inwin) {
          a.status[ii] = (uint8_t)(st | PIC_STATUS_LOST);
          atomicAdd(&sh[11], 1ull);
          continue;
        }
        bool capped;
        const MixedState one = {0, 0.f, e ? s.ux.y : s.ux.x, e ? s.uy.y : s.uy.x, e ? s.uz.y : s.uz.x};
        const int k = psi_to_k(e ? bz.y : bz.x, one, a.qm_abs, a.dt, a.psi_max, a.k_max, capped);
        count_step(tc, sh, k, capped);
        if (k == 0) {
          push = true;  // capped at k_max = 0
        } else if (k >= kDeferMin) {
          defer_mark(a, ii, st & 7, k, a.step_cur);
          key = k;
        } else {
          sk = k;
        }
      }
    }
    const MixedState p0 = {s.cell.x, s.frac.x, s.ux.x, s.uy.x, s.uz.x};  // as loaded, for the stash
    const MixedState p1 = {s.cell.y, s.frac.y, s.ux.y, s.uy.y, s.uz.y};
    if (push0 || push1) {
      const float2 h_old = make_float2(pow4_down(a.dt, st0 & 7), pow4_down(a.dt, st1 & 7));
      const float2 hp = mul2(bc2(0.5f), add2(h_old, bc2(a.dt)));
      MixedState2 u = s;
      boris_f32x2(ey, bz, hp, hx0, a.qm, u);
      const float2 fl = floor2(u.frac);  // normalize each
      u.cell.x += (int32_t)fl.x;
      u.cell.y += (int32_t)fl.y;
      u.frac = sub2(u.frac, fl);
      if (push0 && push1 && a.tma) {  // 16-byte aligned arrays, i even: 8-byte stores
        __stcs(reinterpret_cast<int2*>(a.cell + i), u.cell);
        __stcs(reinterpret_cast<float2*>(a.frac + i), u.frac);
        __stcs(reinterpret_cast<float2*>(a.px + i), u.ux);
        __stcs(reinterpret_cast<float2*>(a.py + i), u.uy);
        __stcs(reinterpret_cast<float2*>(a.pz + i), u.uz);
        *reinterpret_cast<uint16_t*>(a.status + i) = (uint16_t)(done | (done << 8));
      } else {
        if (push0) {
          store_stream(a, i, MixedState{u.cell.x, u.frac.x, u.ux.x, u.uy.x, u.uz.x});
          a.status[i] = done;
        }
        if (push1) {
          store_stream(a, i + 1, MixedState{u.cell.y, u.frac.y, u.ux.y, u.uy.y, u.uz.y});
          a.status[i + 1] = done;
        }
      }
    }
    if (side) {
#pragma unroll 1
      for (int e = 0; e < 2; ++e) {
        enqueue(a, e ? key1 : key0, (int32_t)(i + (uint32_t)e));
        park(e ? sk1 : sk0, (int32_t)(i + (uint32_t)e), e ? p1 : p0, (uint8_t)((e ? st1 : st0) & 7));
      }
    }
  };

  // Work items: a warp's first item is its warp-major index (no atomic: the
  // heavy items, first in the order, spread over the SMs); later ones come
  // from the cursor, offset by the number of warps.  In the stream the next
  // claim is issued one item ahead (lane 0 holds it), so the atomic's round
  // trip overlaps the current item's work instead of stalling the warp.
  const int64_t n_warps = (int64_t)gridDim.x * kWarps;
  bool first_claim = true;
  auto claim = [&]() -> int64_t {
    if (first_claim) {
      first_claim = false;
      return (int64_t)warp * gridDim.x + blockIdx.x;
    }
    int v = 0;
    if (lane == 0) v = atomicAdd(a.cursor, 1);
    return n_warps + __shfl_sync(0xffffffffu, v, 0);
  };
  int ahead = 0;  // lane 0: the claim issued one item ahead
  auto claim_ahead = [&]() {
    if (lane == 0) ahead = atomicAdd(a.cursor, 1);
  };
  auto take_ahead = [&]() -> int64_t {
    const int64_t t = n_warps + __shfl_sync(0xffffffffu, ahead, 0);
    claim_ahead();
    return t;
  };

  // deferred and predicted items first (they come first in the cursor order);
  // one call site each of the deferred-particle code, enqueue and park
  int64_t t = claim();
  while (t < n_pred_end) {
    int key = 0, sk = 0;
    int32_t i = 0;
    MixedState s = {0, 0.5f, 0.f, 0.f, 0.f};
    uint8_t kp = 0;
    bool heavy = false;
    if (t < n_heavy) {
      int k = 7;
      while (k > 1 && t >= heavy_end[k]) --k;
      const int64_t first = (k == 7 ? 0 : heavy_end[k + 1]);
      const int64_t e = (t - first) * 32 + lane;
      if (e < a.qcount_in[k]) {
        i = a.queue_in[(int64_t)(k - 1) * a.qcap + e];
        heavy = true;
      }
    } else {
      int k = 7;
      while (k > 1 && t >= pred_end[k]) --k;
      const int64_t first = (k == 7 ? n_heavy : pred_end[k + 1]);
      const int64_t e = (t - first) * 32 + lane;
      if (e < a.pred_count[k]) {
        i = a.pred_queue[(int64_t)(k - 1) * a.qcap + e];
        predicted_particle<P, RING>(a, F, wcrit, i, k, tc, sh, key, sk, s, kp, heavy);
      }
    }
    if (heavy) heavy_particle<P, RING>(a, Fp, F, wcrit, i, tc, sh, key);
    enqueue(a, key, i);
    park(sk, i, s, kp);
    t = claim();
  }

  // The stream: every later claim is a stream item of kChunk particles, taken
  // as tiles of kTile.  Each warp keeps kStages tiles staged in shared memory:
  // while one is pushed the next is in flight, across item boundaries.  Tiles
  // that are not whole (the array's tail) or arrays that are not 16-byte
  // aligned are read with plain loads instead.
  if (t < n_items) {
    const int64_t n_tiles = (a.n + kTile - 1) / kTile;
    constexpr int64_t kTilesPerItem = kChunk / kTile;
    int64_t gen_next = (t - n_pred_end) * kTilesPerItem;
    int64_t gen_end = gen_next + kTilesPerItem < n_tiles ? gen_next + kTilesPerItem : n_tiles;
    bool gen_done = false;
    claim_ahead();
    auto gen = [&]() -> int64_t {  // next tile of this warp, -1 when the stream is exhausted
      if (gen_done) return -1;
      if (gen_next >= gen_end) {
        const int64_t it = take_ahead();
        if (it >= n_items) {
          gen_done = true;
          return -1;
        }
        gen_next = (it - n_pred_end) * kTilesPerItem;
        gen_end = gen_next + kTilesPerItem < n_tiles ? gen_next + kTilesPerItem : n_tiles;
      }
      return gen_next++;
    };
    auto whole = [&](int64_t tile) { return a.tma && (tile + 1) * kTile <= a.n; };
    const uint64_t policy = evict_first_policy();
    auto issue = [&](int sidx, int64_t tile) {
      if (tile >= 0 && whole(tile) && lane == 0)
        tile_issue(a, my_tiles + sidx, my_bars + sidx, tile * kTile, policy);
    };
    // q[o]: the tile staged in stage (stage + o) % kStages, o = 0 the next one
    // pushed.  The loop body -- the whole stream code -- exists once: the
    // stages rotate through registers instead of an unrolled loop per stage.
    int64_t q[kStages];
#pragma unroll
    for (int sidx = 0; sidx < kStages; ++sidx) {
      q[sidx] = gen();
      issue(sidx, q[sidx]);
    }
    int stage = 0;
#pragma unroll 1
    for (;;) {
      const int64_t tile = q[0];
      if (tile < 0) break;
      const int64_t first = tile * kTile;
      const bool staged = whole(tile);
      if (staged) {
        if (!mbar_wait(my_bars + stage, (phase >> stage) & 1u)) {
          // The copies never completed: flag it for the host (PIC_ETIMEOUT)
          // and leave the stream.  No instruction cancels a bulk copy, so
          // before the block may exit, every stage this warp has in flight --
          // this one included -- gets one more bounded wait: only a copy that
          // has not landed after two full waits (a memory system that no
          // longer answers) can outlive the block.
          if (lane == 0) atomicExch(&a.stats->error, 1);
#pragma unroll
          for (int o = 0; o < kStages; ++o) {
            const int so = (stage + o) % kStages;
            if (q[o] >= 0 && whole(q[o])) mbar_wait(my_bars + so, (phase >> so) & 1u);
          }
          break;
        }
        phase ^= 1u << stage;
      }
      // rounds of 64 particles (stream_pair's one call site): staged tiles from
      // shared memory, the rest (the array's tail, unaligned arrays) by plain loads
#pragma unroll 1
      for (int r = 0; r < kTile / 64; ++r) stream_pair(my_tiles[stage], staged, r, (uint32_t)first);
      __syncwarp();  // every lane is done with the stage before it is refilled
      const int64_t next = gen();
      issue(stage, next);
#pragma unroll
      for (int o = 0; o + 1 < kStages; ++o) q[o] = q[o + 1];
      q[kStages - 1] = next;
      stage = stage + 1 == kStages ? 0 : stage + 1;
    }
  }

  // the claim issued ahead must have been performed before the block reports
  // done (the last block resets the cursor): consuming its value waits for it
  if (lane == 0) s_task[warp] = ahead;
  // push what is left in the stashes
  drain(true);
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

// Every window node's E_y and B_z extrapolated to t_{n+1} (theta = 3/2) from
// step n's levels a: the temporal sum gather_f32 takes at a node, over the same
// levels in the same order; W + 1 nodes each, node W repeating node 0.
template <int P>
__global__ void feature_nodes_kernel(PushArgsMixed a, int64_t W, float* outE, float* outB) {
  StepFields<P, true> F;
  load_fields<P, true>(F, a, false);
  float w[2 * (P + 1)];
  lagrange_f32<P>(1.5f, w);
  for (int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; c < W;
       c += (int64_t)gridDim.x * blockDim.x) {
    float fe = __fmul_rn(w[0], __ldg(F.E.at(0) + c));
    float fb = __fmul_rn(w[P + 1], __ldg(F.B.at(0) + c));
#pragma unroll
    for (int l = 1; l <= P; ++l) {
      fe = __fmaf_rn(w[l], __ldg(F.E.at(l) + c), fe);
      fb = __fmaf_rn(w[P + 1 + l], __ldg(F.B.at(l) + c), fb);
    }
    outE[c] = fe;
    outB[c] = fb;
    if (c == 0) {
      outE[W] = fe;
      outB[W] = fb;
    }
  }
}

cudaError_t launch_feature_nodes(const PushArgsMixed& a, int order, int64_t W, float* outE,
                                 float* outB, cudaStream_t s) {
  const int64_t want = (W + 255) / 256;
  const int blocks = (int)(want < 152 * 8 ? want : 152 * 8);
  switch (order) {
    case 1: feature_nodes_kernel<1><<<blocks, 256, 0, s>>>(a, W, outE, outB); break;
    case 2: feature_nodes_kernel<2><<<blocks, 256, 0, s>>>(a, W, outE, outB); break;
    case 3: feature_nodes_kernel<3><<<blocks, 256, 0, s>>>(a, W, outE, outB); break;
    case 4: feature_nodes_kernel<4><<<blocks, 256, 0, s>>>(a, W, outE, outB); break;
    case 5: feature_nodes_kernel<5><<<blocks, 256, 0, s>>>(a, W, outE, outB); break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

// phi of every particle after macro step n (see particle_features; a.halfE,
// a.halfB: the feature nodes of step n).
__global__ void features_kernel(PushArgsMixed a, float* phi) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < a.n;
       i += (int64_t)gridDim.x * blockDim.x) {
    float f[6];
    particle_features(a, a.halfE, a.halfB, a.lo, a.hi, i, f);
#pragma unroll
    for (int q = 0; q < 6; ++q) phi[i * 6 + q] = f[q];
  }
}

cudaError_t launch_features_mixed(const PushArgsMixed& a, int order, float* phi, cudaStream_t s) {
  (void)order;
  if (a.n <= 0) return cudaSuccess;
  const int64_t want = (a.n + 255) / 256;
  const int blocks = (int)(want < 152 * 16 ? want : 152 * 16);
  features_kernel<<<blocks, 256, 0, s>>>(a, phi);
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
    push_mixed_plain_kernel<P, false><<<(int)(want < cap ? want : cap), 256, 0, s>>>(a);
    if (launches) ++*launches;
  }
  return cudaGetLastError();
}

template <int P, bool RING>
static cudaError_t launch_binned_p(const PushArgsMixed& a, int sm_count, cudaStream_t main,
                                   int* launches) {
  const int sms = sm_count > 0 ? sm_count : 152;
  static int occ = 0;
  if (occ == 0) {
    cudaError_t e = cudaFuncSetAttribute(push_binned_kernel<P, RING>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kBinnedSmem);
    if (e != cudaSuccess) return e;
#ifdef PIC_MIN_CARVEOUT
    {  // the smallest shared-memory carveout that holds the resident blocks: the rest is L1
      const int need = PIC_BINNED_MIN_BLOCKS * ((int)kBinnedSmem + 1024 + 512);
      int pct = (need * 100 + 228 * 1024 - 1) / (228 * 1024);
      if (pct > 100) pct = 100;
      e = cudaFuncSetAttribute(push_binned_kernel<P, RING>,
                               cudaFuncAttributePreferredSharedMemoryCarveout, pct);
      if (e != cudaSuccess) return e;
    }
#endif
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, push_binned_kernel<P, RING>, kThreads,
                                                  kBinnedSmem);
    if (occ < 1) occ = 1;
  }
  int64_t blocks = (int64_t)sms * occ;
  const int64_t items = (a.n + kChunk - 1) / kChunk;
  if (!a.finalize && blocks > (items + kWarps - 1) / kWarps + sms) blocks = (items + kWarps - 1) / kWarps + sms;
  push_binned_kernel<P, RING><<<(int)blocks, kThreads, kBinnedSmem, main>>>(a);
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
  if (a.ringE) {
    if (!a.coef || !a.coef_p) return cudaErrorInvalidValue;  // the ring form reads the node tables
    switch (order) {
      case 1: return launch_binned_p<1, true>(a, sm_count, main, launches);
      case 2: return launch_binned_p<2, true>(a, sm_count, main, launches);
      case 3: return launch_binned_p<3, true>(a, sm_count, main, launches);
      case 4: return launch_binned_p<4, true>(a, sm_count, main, launches);
      case 5: return launch_binned_p<5, true>(a, sm_count, main, launches);
      default: return cudaErrorInvalidValue;
    }
  }
  switch (order) {
    case 1: return launch_binned_p<1, false>(a, sm_count, main, launches);
    case 2: return launch_binned_p<2, false>(a, sm_count, main, launches);
    case 3: return launch_binned_p<3, false>(a, sm_count, main, launches);
    case 4: return launch_binned_p<4, false>(a, sm_count, main, launches);
    case 5: return launch_binned_p<5, false>(a, sm_count, main, launches);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace pic
