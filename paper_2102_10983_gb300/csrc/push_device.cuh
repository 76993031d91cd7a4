// Per-particle device arithmetic of the mixed-precision push, shared by the
// single-problem kernels (push_mixed.cu), the batched kernel (push_batch.cu)
// and the fused predictor kernel (mlp_bf16.cu).
#pragma once

#include <limits.h>
#include <math.h>

#include "pic_internal.h"

namespace pic {

// ---------------------------------------------------------------- per-particle math

// The p+1 levels of one grid used by one macro step (level 0 = oldest).
// Ring form: consecutive slots of the mirrored ring, level l at base + l*W.
// Pointer form: one pointer per level (levels owned by the caller).
template <int P, bool RING>
struct Levels;
template <int P>
struct Levels<P, true> {
  const float* base;
  int32_t lstride;  // l * lstride + node stays below 2^31 (window <= 2^28 nodes)
  __device__ __forceinline__ const float* at(int l) const { return base + (uint32_t)(l * lstride); }
};
template <int P>
struct Levels<P, false> {
  const float* ptr[P + 1];
  __device__ __forceinline__ const float* at(int l) const { return ptr[l]; }
};

// Temporal sums at the two tent nodes jn, jn+1, then the tent weight wt.
template <int P, class LV>
__device__ __forceinline__ float gather_f32(const LV& lv, const float* w, int32_t jn, float wt,
                                            int32_t mask) {
  const int32_t a0 = jn & mask, a1 = (jn + 1) & mask;
  float f0 = __fmul_rn(w[0], __ldg(lv.at(0) + a0));
  float f1 = __fmul_rn(w[0], __ldg(lv.at(0) + a1));
#pragma unroll
  for (int l = 1; l <= P; ++l) {
    f0 = __fmaf_rn(w[l], __ldg(lv.at(l) + a0), f0);
    f1 = __fmaf_rn(w[l], __ldg(lv.at(l) + a1), f1);
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
  return jb >= lo && je < hi;  // jb <= je: both nodes of both grids in [lo, hi)
}

__device__ __forceinline__ float norm2(float a, float b, float c) {
  return __fmaf_rn(c, c, __fmaf_rn(b, b, __fmul_rn(a, a)));
}

// Criterion (Sec. IV) in FP32: Psi0 = |q/m| |B| dt / (2 gamma); smallest k with
// Psi0 / 4^k <= Psi_max, capped at k_max.  Taken in squared form, with no
// square root and no division: Psi0 <= Psi_max 4^k  <=>
// (|q/m| dt B)^2 <= (2 Psi_max)^2 (1 + |p|^2) 16^k, and the right side is
// scaled by 16 (exactly) per step of k.
// The two sides of the k = 0 test: a2 = (|q/m| dt B)^2, rhs = (2 Psi_max)^2 (1 + |p|^2).
__device__ __forceinline__ void psi_terms(float b0, const MixedState& s, float qm_abs, float dt,
                                          float psi_max, float& a2, float& rhs) {
  const float a = __fmul_rn(__fmul_rn(qm_abs, dt), b0);
  a2 = __fmul_rn(a, a);
  const float tp = __fmul_rn(2.0f, psi_max);
  rhs = __fmul_rn(__fmul_rn(tp, tp), __fadd_rn(1.0f, norm2(s.ux, s.uy, s.uz)));
}

__device__ __forceinline__ int psi_to_k(float b0, const MixedState& s, float qm_abs, float dt,
                                        float psi_max, int k_max, bool& capped) {
  float a2, rhs;
  psi_terms(b0, s, qm_abs, dt, psi_max, a2, rhs);
  int k = 0;
  while (a2 > rhs && k < k_max) {
    rhs = __fmul_rn(rhs, 16.0f);
    ++k;
  }
  capped = a2 > rhs;
  return k;
}

// dt / 4^k for a normal dt whose quotient stays normal (checked by the host):
// the exponent field lowered by 2k, the same bits as ldexpf(dt, -2k).
__device__ __forceinline__ float pow4_down(float dt, int k) {
  return __int_as_float(__float_as_int(dt) - (k << 24));
}

// b0 is B_z at the particle and t_n: with m = 1 it is also the first (and only)
// sub-step's B_z, since both use the theta = 1/2 weights at the same nodes.
template <int P, class LV>
__device__ __forceinline__ int criterion_f32(const LV& B, const float* wcrit, int32_t jb,
                                             float wb, int32_t mask, const MixedState& s,
                                             float qm_abs, float dt, float psi_max, int k_max,
                                             bool& capped, float& b0) {
  b0 = gather_f32<P>(B, wcrit, jb, wb, mask);
  return psi_to_k(b0, s, qm_abs, dt, psi_max, k_max, capped);
}

// Field view of one macro step.  coef (optional): per window node, the
// monomial coefficients (to_monomial) of the temporal interpolant of E_y (P+1)
// then of B_z (P+1), written once per step by the half-step kernel, so a node
// change costs two contiguous loads per grid instead of 2(P+1) scattered ones.
template <int P, bool RING>
struct StepFields {
  Levels<P, RING> E, B;
  const float* coef;
  int32_t lo, hi;
};

// Single-instruction reciprocal and reciprocal square root (the SFU's
// approximations, ~2 ulp, subnormals flushed): every schedule of the mixed form
// calls these same two, so they agree bit for bit.  Their arguments here are
// 1 + |p|^2 >= 1 and 1 + t^2 >= 1.
__device__ __forceinline__ float rsqrt_sfu(float x) {
  float y;
  asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}
__device__ __forceinline__ float rcp_sfu(float x) {
  float y;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}

// One Boris sub-step (Eqs. eq:p - eq:gamman) and the position update (Eq. eq:x)
// in the fields ey, bz, with momentum step hp and offset step hx (cells per
// unit velocity).  The operations are ordered for the serial chain of a long
// sub-cycle: the terms of 1 + |p|^2 known early are summed first, so the
// component that arrives last costs a single FMA before each square root.
__device__ __forceinline__ void boris_f32(float ey, float bz, float hp, float hx, float qm,
                                          MixedState& s) {
  const float qmh = __fmul_rn(qm, __fmul_rn(0.5f, hp));  // q/m hp/2
  const float dpy = __fmul_rn(qmh, ey);
  const float mx = s.ux, mz = s.uz;
  const float g2xz = __fadd_rn(1.0f, __fmaf_rn(mz, mz, __fmul_rn(mx, mx)));
  const float my = __fadd_rn(s.uy, dpy);
  const float inv_gn = rsqrt_sfu(__fmaf_rn(my, my, g2xz));
  const float tz = __fmul_rn(__fmul_rn(qmh, bz), inv_gn);
  const float ppx = __fmaf_rn(my, tz, mx);
  const float ppy = __fmaf_rn(-mx, tz, my);
  const float sz = __fmul_rn(__fmul_rn(2.0f, tz), rcp_sfu(__fmaf_rn(tz, tz, 1.0f)));
  const float ux = __fmaf_rn(ppy, sz, mx);
  const float uy = __fadd_rn(__fmaf_rn(-ppx, sz, my), dpy);
  s.ux = ux;
  s.uy = uy;
  s.uz = mz;
  const float g2n = __fadd_rn(1.0f, __fmaf_rn(mz, mz, __fmul_rn(ux, ux)));
  const float inv_g = rsqrt_sfu(__fmaf_rn(uy, uy, g2n));
  s.frac = __fmaf_rn(hx, __fmul_rn(ux, inv_g), s.frac);
}

// ---------------------------------------------------------------- two particles per lane
//
// The same arithmetic on two particles at once with GB300's paired FP32
// instructions (mul/add/fma.rn.f32x2, written as PTX): each half rounds
// exactly as the scalar operation it replaces.  a - b is fma(b, -1, a).  A
// paired product that only paired sums consume can still be merged into them
// by the compiler, so such a product is kept scalar (see boris_f32x2).
__device__ __forceinline__ float2 bc2(float v) { return make_float2(v, v); }
__device__ __forceinline__ float2 mul2(float2 a, float2 b) {
  float2 d;
  asm("{\n .reg .b64 ra, rb, rd;\n mov.b64 ra, {%2, %3};\n mov.b64 rb, {%4, %5};\n"
      " mul.rn.f32x2 rd, ra, rb;\n mov.b64 {%0, %1}, rd;\n}"
      : "=f"(d.x), "=f"(d.y)
      : "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y));
  return d;
}
__device__ __forceinline__ float2 add2(float2 a, float2 b) {
  float2 d;
  asm("{\n .reg .b64 ra, rb, rd;\n mov.b64 ra, {%2, %3};\n mov.b64 rb, {%4, %5};\n"
      " add.rn.f32x2 rd, ra, rb;\n mov.b64 {%0, %1}, rd;\n}"
      : "=f"(d.x), "=f"(d.y)
      : "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y));
  return d;
}
__device__ __forceinline__ float2 fma2(float2 a, float2 b, float2 c) {
  float2 d;
  asm("{\n .reg .b64 ra, rb, rc, rd;\n mov.b64 ra, {%2, %3};\n mov.b64 rb, {%4, %5};\n"
      " mov.b64 rc, {%6, %7};\n fma.rn.f32x2 rd, ra, rb, rc;\n mov.b64 {%0, %1}, rd;\n}"
      : "=f"(d.x), "=f"(d.y)
      : "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y), "f"(c.x), "f"(c.y));
  return d;
}
__device__ __forceinline__ float2 sub2(float2 a, float2 b) { return fma2(b, bc2(-1.0f), a); }
__device__ __forceinline__ float2 floor2(float2 a) { return make_float2(floorf(a.x), floorf(a.y)); }

struct MixedState2 {
  int2 cell;
  float2 frac, ux, uy, uz;
};

// boris_f32 on two particles (same operation order, same bits).
__device__ __forceinline__ void boris_f32x2(float2 ey, float2 bz, float2 hp, float hx, float qm,
                                            MixedState2& s) {
  const float2 qmh = mul2(bc2(qm), mul2(bc2(0.5f), hp));
  const float2 dpy = make_float2(__fmul_rn(qmh.x, ey.x), __fmul_rn(qmh.y, ey.y));
  const float2 mx = s.ux, mz = s.uz;
  const float2 g2xz = add2(bc2(1.0f), fma2(mz, mz, mul2(mx, mx)));
  const float2 my = add2(s.uy, dpy);
  const float2 gn = fma2(my, my, g2xz);
  const float2 inv_gn = make_float2(rsqrt_sfu(gn.x), rsqrt_sfu(gn.y));
  const float2 tz = mul2(mul2(qmh, bz), inv_gn);
  const float2 ppx = fma2(my, tz, mx);
  const float2 ppy = fma2(make_float2(-mx.x, -mx.y), tz, my);
  const float2 tt = fma2(tz, tz, bc2(1.0f));
  const float2 sz = mul2(mul2(bc2(2.0f), tz), make_float2(rcp_sfu(tt.x), rcp_sfu(tt.y)));
  const float2 ux = fma2(ppy, sz, mx);
  const float2 uy = add2(fma2(make_float2(-ppx.x, -ppx.y), sz, my), dpy);
  s.ux = ux;
  s.uy = uy;
  s.uz = mz;
  const float2 g2n = add2(bc2(1.0f), fma2(mz, mz, mul2(ux, ux)));
  const float2 g = fma2(uy, uy, g2n);
  const float2 inv_g = make_float2(rsqrt_sfu(g.x), rsqrt_sfu(g.y));
  s.frac = fma2(bc2(hx), mul2(ux, inv_g), s.frac);
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
// Coefficients of the interpolating polynomial in u at two nodes a0, a1 of the
// given levels: c_q = sum_l v_l M[l][q].
template <int P, class LV>
__device__ __forceinline__ void to_monomial(const LV& lv, int32_t a0, int32_t a1,
                                            const float (&M)[kMaxOrder + 1][kMaxOrder + 1],
                                            float* c0, float* c1) {
  float v0[P + 1], v1[P + 1];
#pragma unroll
  for (int l = 0; l <= P; ++l) {
    v0[l] = __ldg(lv.at(l) + a0);
    v1[l] = __ldg(lv.at(l) + a1);
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

// Coefficients of nodes a0, a1 of one grid (g = 0: E, 1: B) from the step's
// table; the same values to_monomial computes from the levels.
template <int P>
__device__ __forceinline__ void table_coefs(const float* coef, int g, int32_t a0, int32_t a1,
                                            float* c0, float* c1) {
  constexpr int S = 2 * (P + 1);
  const float* r0 = coef + (int64_t)a0 * S + g * (P + 1);
  const float* r1 = coef + (int64_t)a1 * S + g * (P + 1);
  if constexpr (P == 3) {  // rows of 8 floats: each half is one aligned 16-byte load
    const float4 v0 = __ldg(reinterpret_cast<const float4*>(r0));
    const float4 v1 = __ldg(reinterpret_cast<const float4*>(r1));
    c0[0] = v0.x; c0[1] = v0.y; c0[2] = v0.z; c0[3] = v0.w;
    c1[0] = v1.x; c1[1] = v1.y; c1[2] = v1.z; c1[3] = v1.w;
  } else {
#pragma unroll
    for (int q = 0; q <= P; ++q) {
      c0[q] = __ldg(r0 + q);
      c1[q] = __ldg(r1 + q);
    }
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
// The floors of the offset on both grids are cached with the coefficients, so
// while the nodes stay the same a sub-step's tent weights are one subtraction
// each after the new offset (the same bits as a fresh floor).  The
// coefficients come from
// the step's node table (TABLE: F.coef, written by the half-step kernel), else
// from the levels.
//
// Sub-steps j0+1 .. j1 of the m (j1 = -1: all of them): a sub-cycle can stop
// after any sub-step and resume from the state it left (offset not yet
// normalised) with the same bits as an uninterrupted one.
template <int P, bool RING, bool TABLE = false>
__device__ __forceinline__ bool subcycle_f32(const StepFields<P, RING>& F, const float* wtab,
                                             int32_t mask, float dt, float inv_dx, float qm,
                                             int field_time,
                                             const float (&mono)[2][kMaxOrder + 1][kMaxOrder + 1],
                                             int k, int k_prev, float b0, MixedState& s,
                                             int j0 = 0, int j1 = -1) {
  constexpr int stride = 2 * (P + 1);
  const float h = pow4_down(dt, k);
  const float h_old = pow4_down(dt, k_prev);
  const float hx = __fmul_rn(h, inv_dx);
  float hp = j0 == 0 ? __fmul_rn(0.5f, __fadd_rn(h_old, h)) : h;
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
  const float inv_m = pow4_down(1.0f, k);
  // u_j = theta_j - 1, exact in FP32 for m <= 4^7
  const float u1 = field_time == 0 ? -0.5f : __fsub_rn(__fmul_rn(0.5f, inv_m), 1.0f);
  int32_t ce = INT_MIN, cb = INT_MIN;
  float ce0[P + 1], ce1[P + 1], cb0[P + 1], cb1[P + 1];  // monomial coefficients per node
#pragma unroll
  for (int q = 0; q <= P; ++q) ce0[q] = ce1[q] = cb0[q] = cb1[q] = 0.f;
  // floors of the offset on the two grids at the cached nodes (NaN: none yet)
  float fe = __int_as_float(0x7fc00000), fb = fe;
  const int j_end = j1 < 0 ? m : j1;
  // u_j = u_1 + (j-1)/m: every partial sum is a multiple of 1/m in [-1, 1],
  // exact in FP32, so the running sum has the bits of the direct formula
  float u = __fmaf_rn((float)j0, inv_m, u1);
  for (int j = j0 + 1; j <= j_end; ++j) {
    const float f = s.frac;
    const float fbm = __fsub_rn(f, 0.5f);
    float we = __fsub_rn(f, fe), wb = __fsub_rn(fbm, fb);
    // cached nodes still hold iff both rounded weights lie in [+0, 1): then
    // f - fe and fbm - fb are exact and fe, fb are the floors (a NaN or a
    // negative weight fails the unsigned test)
    if (!(__float_as_uint(we) < 0x3f800000u && __float_as_uint(wb) < 0x3f800000u)) {
      int32_t je, jb;
      if (!tent_coords(s.cell, f, F.lo, F.hi, je, we, jb, wb)) return false;
      fe = floorf(f);
      fb = floorf(fbm);
      if (je != ce) {
        ce = je;
        if constexpr (TABLE)
          table_coefs<P>(F.coef, 0, je & mask, (je + 1) & mask, ce0, ce1);
        else
          to_monomial<P>(F.E, je & mask, (je + 1) & mask, mono[0], ce0, ce1);
      }
      if (jb != cb) {
        cb = jb;
        if constexpr (TABLE)
          table_coefs<P>(F.coef, 1, jb & mask, (jb + 1) & mask, cb0, cb1);
        else
          to_monomial<P>(F.B, jb & mask, (jb + 1) & mask, mono[1], cb0, cb1);
      }
    }
    const float fe0 = horner<P>(ce0, u), fe1 = horner<P>(ce1, u);
    const float fb0 = horner<P>(cb0, u), fb1 = horner<P>(cb1, u);
    boris_f32(__fmaf_rn(we, __fsub_rn(fe1, fe0), fe0), __fmaf_rn(wb, __fsub_rn(fb1, fb0), fb0), hp,
              hx, qm, s);
    hp = h;
    u = __fadd_rn(u, inv_m);
  }
  return true;
}

// The node-table form of subcycle_f32 behind one call site.  With
// PIC_SUBCYCLE_NOINLINE defined, every caller in a kernel shares one copy of
// its code (a call per sub-cycle instead of a copy per caller: less for the
// instruction cache to hold); otherwise it is inlined at each caller.
struct SubOut {
  MixedState s;
  bool ok;
};
template <int P>
__device__ __noinline__ SubOut subcycle_table_call(StepFields<P, true> F, const float* wtab,
                                                   int32_t mask, float dt, float inv_dx, float qm,
                                                   int field_time, int k, int k_prev, float b0,
                                                   MixedState s, int j0, int j1) {
  float no_mono[2][kMaxOrder + 1][kMaxOrder + 1];  // the table form never reads it
  SubOut o;
  o.s = s;
  o.ok = subcycle_f32<P, true, true>(F, wtab, mask, dt, inv_dx, qm, field_time, no_mono, k, k_prev,
                                     b0, o.s, j0, j1);
  return o;
}
template <int P, bool RING, bool TABLE>
__device__ __forceinline__ bool subcycle_site(const StepFields<P, RING>& F, const float* wtab,
                                              int32_t mask, float dt, float inv_dx, float qm,
                                              int field_time,
                                              const float (&mono)[2][kMaxOrder + 1][kMaxOrder + 1],
                                              int k, int k_prev, float b0, MixedState& s,
                                              int j0 = 0, int j1 = -1) {
#ifdef PIC_SUBCYCLE_NOINLINE
  if constexpr (RING && TABLE) {
    const SubOut o = subcycle_table_call<P>(F, wtab, mask, dt, inv_dx, qm, field_time, k, k_prev, b0,
                                            s, j0, j1);
    s = o.s;
    return o.ok;
  }
#endif
  return subcycle_f32<P, RING, TABLE>(F, wtab, mask, dt, inv_dx, qm, field_time, mono, k, k_prev,
                                      b0, s, j0, j1);
}

__device__ __forceinline__ void normalize(MixedState& s) {
  const float fl = floorf(s.frac);
  s.cell += (int32_t)fl;
  s.frac = __fsub_rn(s.frac, fl);
}

// ---------------------------------------------------------------- counters

// Per-thread counters in registers: steps with k = 0, 1, 2 (the common ones)
// and caps.  Steps with k >= 3 are rare and go straight into the block's
// shared counters.  (Shared-memory atomics on one address for every
// sub-cycled particle serialised the warps at a front.)  The sub-step sums are
// not counted per particle: every counted step takes m = 4^k sub-steps, so
// they follow from the k histogram when the block flushes.
struct ThreadCounters {
  unsigned k0 = 0, k1 = 0, k2 = 0, capped = 0;
};

__device__ __forceinline__ void count_step(ThreadCounters& tc, unsigned long long* sh, int k,
                                           bool capped) {
  if (k == 0)
    ++tc.k0;
  else if (k == 1)
    ++tc.k1;
  else if (k == 2)
    ++tc.k2;
  else
    atomicAdd(&sh[k], 1ull);
  tc.capped += capped ? 1u : 0u;
}

__device__ __forceinline__ unsigned long long warp_sum(unsigned long long v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// All threads of the block must call this.  Block counters: sh[0..7] the k
// histogram, sh[10] caps, sh[11] particles lost; sh[8], sh[9] unused.
__device__ __forceinline__ void flush_counters(const ThreadCounters& tc, unsigned long long* sh,
                                               DevStats* st) {
  const unsigned long long k0 = warp_sum(tc.k0), k1 = warp_sum(tc.k1), k2 = warp_sum(tc.k2);
  const unsigned long long cap = warp_sum(tc.capped);
  if ((threadIdx.x & 31) == 0) {
    if (k0) atomicAdd(&sh[0], k0);
    if (k1) atomicAdd(&sh[1], k1);
    if (k2) atomicAdd(&sh[2], k2);
    if (cap) atomicAdd(&sh[10], cap);
  }
  __syncthreads();
  if (threadIdx.x < 12) {
    unsigned long long v = 0;
    if (threadIdx.x == 8 || threadIdx.x == 9) {  // sum of m = 4^k over the counted steps
#pragma unroll
      for (int k = threadIdx.x == 8 ? 0 : 1; k < 8; ++k) v += sh[k] << (2 * k);
    } else {
      v = sh[threadIdx.x];
    }
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

// The stream's loads and stores: each state word is touched once per step and
// the whole state is larger than L2, so these are marked evict-first to leave
// L2 to the field levels, half-step fields and queues.
// (Particle indices are below 2^31: 32-bit offsets address every array.)
__device__ __forceinline__ void fetch_stream(const PushArgsMixed& a, uint32_t i, uint8_t& st,
                                             MixedState& s) {
  st = PIC_STATUS_LOST;
  s = {0, 0.5f, 0.f, 0.f, 0.f};
  if ((int64_t)i < a.n) {
    st = __ldcs(a.status + i);
    s.cell = __ldcs(a.cell + i);
    s.frac = __ldcs(a.frac + i);
    s.ux = __ldcs(a.px + i);
    s.uy = __ldcs(a.py + i);
    s.uz = __ldcs(a.pz + i);
  }
}

__device__ __forceinline__ void store_stream(const PushArgsMixed& a, uint32_t i, const MixedState& s) {
  __stcs(a.cell + i, s.cell);
  __stcs(a.frac + i, s.frac);
  __stcs(a.px + i, s.ux);
  __stcs(a.py + i, s.uy);
  __stcs(a.pz + i, s.uz);
}

// ---------------------------------------------------------------- bulk-copy staging of particle tiles

// A tile of kTile consecutive particles' state as the stream reads it from
// shared memory; filled by six bulk copies (cp.async.bulk, the TMA engine's
// linear mode) that complete on one mbarrier.  Every member starts on a
// 128-byte boundary and the size is a multiple of 16 bytes.
#ifndef PIC_TILE
#define PIC_TILE 128
#endif
constexpr int kTile = PIC_TILE;
struct Tile {
  int32_t cell[kTile];
  float frac[kTile], px[kTile], py[kTile], pz[kTile];
  uint8_t st[kTile];
};
constexpr uint32_t kTileBytes = (uint32_t)sizeof(Tile);
static_assert(sizeof(Tile) % 16 == 0, "bulk copies move multiples of 16 bytes");

__device__ __forceinline__ uint32_t smem_addr(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void mbar_init(uint64_t* bar) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_addr(bar)) : "memory");
}
// Make the initialised barriers visible to the bulk-copy (async) proxy.
__device__ __forceinline__ void mbar_init_fence() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ __forceinline__ void mbar_expect(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)),
               "r"(bytes)
               : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
      " selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(smem_addr(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}
// Wait for phase `parity` of the barrier to complete, giving up after a bound
// (each try_wait itself blocks for a while): false = the copies never landed.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity) {
  for (uint32_t it = 0; it < (1u << 24); ++it)
    if (mbar_try_wait(bar, parity)) return true;
  return false;
}
// L2 policy for the particle stream: each word is used once per step and the
// whole state is larger than L2.
__device__ __forceinline__ uint64_t evict_first_policy() {
  uint64_t pol;
  asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(pol));
  return pol;
}
__device__ __forceinline__ void bulk_to_smem(void* dst, const void* src, uint32_t bytes,
                                             uint64_t* bar, uint64_t policy) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes.L2::cache_hint"
      " [%0], [%1], %2, [%3], %4;" ::"r"(smem_addr(dst)),
      "l"(src), "r"(bytes), "r"(smem_addr(bar)), "l"(policy)
      : "memory");
}
// One lane: stage particles [first, first + kTile) into t (all of them exist,
// the arrays are 16-byte aligned and first is a multiple of kTile).
__device__ __forceinline__ void tile_issue(const PushArgsMixed& a, Tile* t, uint64_t* bar,
                                           int64_t first, uint64_t policy) {
  mbar_expect(bar, kTileBytes);
  bulk_to_smem(t->cell, a.cell + first, kTile * 4, bar, policy);
  bulk_to_smem(t->frac, a.frac + first, kTile * 4, bar, policy);
  bulk_to_smem(t->px, a.px + first, kTile * 4, bar, policy);
  bulk_to_smem(t->py, a.py + first, kTile * 4, bar, policy);
  bulk_to_smem(t->pz, a.pz + first, kTile * 4, bar, policy);
  bulk_to_smem(t->st, a.status + first, kTile, bar, policy);
}

// The current (prev = false) or previous step's field view from the launch
// arguments: ring form from the mirrored ring's start slot, pointer form from
// the per-level pointers.
template <int P, bool RING>
__device__ __forceinline__ void load_fields(StepFields<P, RING>& F, const PushArgsMixed& a,
                                            bool prev) {
  if constexpr (RING) {
    const int64_t start = prev ? a.start_prev : a.start_cur;
    F.E.base = a.ringE + start * a.lstride;
    F.B.base = a.ringB + start * a.lstride;
    F.E.lstride = a.lstride;
    F.B.lstride = a.lstride;
  } else {
#pragma unroll
    for (int l = 0; l <= P; ++l) {
      F.E.ptr[l] = prev ? a.Ep[l] : a.E[l];
      F.B.ptr[l] = prev ? a.Bp[l] : a.B[l];
    }
  }
  F.coef = prev ? a.coef_p : a.coef;
  F.lo = prev ? a.lo_p : a.lo;
  F.hi = prev ? a.hi_p : a.hi;
}

// ---------------------------------------------------------------- predictor features

// phi = (asinh|E|, asinh|B|, asinh p_x, asinh p_y, asinh p_z, log gamma) of
// particle i after macro step n, with E and B at its position extrapolated to
// t_{n+1} (theta = 3/2) from step n's levels: everything known before level
// n+1 arrives.  The temporal extrapolation of every window node is done once
// (feature_nodes_kernel: nodeE, nodeB, W + 1 nodes each, node W repeating
// node 0), so a particle reads two nodes per grid and applies its tent weight:
// the same operations, in the same order, as gathering the levels at the
// particle.  lo, hi: step n's window.  Lost particles and i >= n get zeros;
// E and B are zero outside the window.
// The stored state particle_features reads (status LOST for i >= n), loaded
// apart from the arithmetic so that a caller can issue the loads of its next
// particle before working on the current one.
struct FeatureInput {
  uint8_t st;
  MixedState s;
};
__device__ __forceinline__ FeatureInput feature_input(const PushArgsMixed& a, int64_t i) {
  FeatureInput r;
  r.st = PIC_STATUS_LOST;
  r.s = {0, 0.f, 0.f, 0.f, 0.f};
  if (i < a.n) {
    r.st = a.status[i];
    r.s = load_state(a, i);
  }
  return r;
}

// asinh x = sign(x) ln(|x| + sqrt(x^2 + 1)), with the special-function unit's
// approximate reciprocal square root and logarithm (a few 1e-7 absolute, far
// below the BF16 resolution of the network's input); exactly 0 at 0 (a
// particle without field has zero field features).
__device__ __forceinline__ float asinh_sfu(float x) {
  const float a = fabsf(x);
  const float t = __fmaf_rn(a, a, 1.0f);
  const float r = copysignf(__logf(__fadd_rn(a, __fmul_rn(t, rsqrt_sfu(t)))), x);
  return x == 0.f ? x : r;
}

__device__ __forceinline__ void features_of(const PushArgsMixed& a, const float* nodeE,
                                            const float* nodeB, int32_t lo, int32_t hi,
                                            const FeatureInput& in, float (&f)[6]) {
#pragma unroll
  for (int q = 0; q < 6; ++q) f[q] = 0.f;
  if (in.st & PIC_STATUS_LOST) return;
  const MixedState& s = in.s;
  int32_t je, jb;
  float we, wb;
  if (tent_coords(s.cell, s.frac, lo, hi, je, we, jb, wb)) {
    const float* e = nodeE + (je & a.mask);
    const float* b = nodeB + (jb & a.mask);
    const float e0 = __ldg(e), e1 = __ldg(e + 1), b0 = __ldg(b), b1 = __ldg(b + 1);
    f[0] = asinh_sfu(fabsf(__fmaf_rn(we, __fsub_rn(e1, e0), e0)));
    f[1] = asinh_sfu(fabsf(__fmaf_rn(wb, __fsub_rn(b1, b0), b0)));
  }
  f[2] = asinh_sfu(s.ux);
  f[3] = asinh_sfu(s.uy);
  f[4] = asinh_sfu(s.uz);
  f[5] = 0.5f * __logf(__fadd_rn(1.0f, norm2(s.ux, s.uy, s.uz)));  // log gamma
}

__device__ __forceinline__ void particle_features(const PushArgsMixed& a, const float* nodeE,
                                                  const float* nodeB, int32_t lo, int32_t hi,
                                                  int64_t i, float (&f)[6]) {
  features_of(a, nodeE, nodeB, lo, hi, feature_input(a, i), f);
}

// Field view of macro step s from the mirrored ring and the device copy of
// the slots' window origins (the host's step_slots / fill_mixed, on the GPU):
// for a deferred particle that runs behind the stream.  No node table.
template <int P>
__device__ __forceinline__ StepFields<P, true> ring_step_fields(const PushArgsMixed& a, int64_t s) {
  StepFields<P, true> F;
  const int64_t R = a.ring_R;
  const int64_t start = ((s - P) % R + R) % R;
  F.E.base = a.ringE + start * a.lstride;
  F.B.base = a.ringB + start * a.lstride;
  F.E.lstride = (int32_t)a.lstride;
  F.B.lstride = (int32_t)a.lstride;
  F.coef = nullptr;
  int64_t lo = INT64_MIN, hi = INT64_MAX;
#pragma unroll
  for (int l = 0; l <= P; ++l) {
    const int64_t o = a.slot_i0[(start + l) % R];
    lo = o > lo ? o : lo;
    hi = o + a.lstride - 1 < hi ? o + a.lstride - 1 : hi;
  }
  F.lo = (int32_t)lo;
  F.hi = (int32_t)hi;
  return F;
}

// Marks particle i as deferred in step s with k (a long sub-cycle pending),
// j of its sub-steps done.
__device__ __forceinline__ void defer_mark(const PushArgsMixed& a, int64_t i, int k_prev, int k,
                                           int64_t s, int j = 0) {
  a.status[i] = (uint8_t)(k_prev | (k << 4));
  if (a.lag_step) {
    a.lag_step[i] = (int32_t)(s - a.step0);
    a.lag_j[i] = (uint16_t)j;
  }
}

// ---------------------------------------------------------------- binned schedule pieces

// Threads per block of the binned kernel: ten warps, two blocks per SM (20
// warps at <= 102 registers, 96 used); measured faster than eight (16 warps at
// <= 128) and twelve (24 at <= 85) on the 16.8M workload.
#ifndef PIC_THREADS
#define PIC_THREADS 320
#endif
constexpr int kThreads = PIC_THREADS;
constexpr int kWarps = kThreads / 32;
#ifndef PIC_CHUNK
#define PIC_CHUNK 512
#endif
#ifndef PIC_STAGES
#define PIC_STAGES 2
#endif
constexpr int kChunk = PIC_CHUNK;    // particles per stream item (kChunk / kTile tiles)
constexpr int kStages = PIC_STAGES;  // staged tiles per warp (one in flight while one is pushed)
static_assert(kChunk % kTile == 0 && kTile % 64 == 0, "a stream item is whole tiles of whole rounds");
constexpr int kStashK = kDeferMin - 1;
constexpr int kStashCap = 64;
constexpr uint8_t kParity = 0x08;
constexpr uint8_t kDeferMask = 0x70;
// Deferred-k field value 1 (a k no sub-cycle is deferred with): the particle
// belongs to the predicted queue, which pushes it every step until the next
// refresh of the predictions; the stream leaves it alone.
constexpr uint8_t kOwned = 0x10;
static_assert(kDeferMin > 1, "deferred-k value 1 marks predicted-queue particles");

__device__ __forceinline__ int deferred_k(uint8_t st) { return (st >> 4) & 7; }

// Enqueue particle i into the queue of its k; warp-aggregated: one atomic per
// distinct k in the warp.  All 32 lanes call this; key 0 = nothing.
__device__ __forceinline__ void enqueue(const PushArgsMixed& a, int key, int32_t i) {
  if (!__any_sync(0xffffffffu, key != 0)) return;
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
#ifdef PIC_STASH_INDEX_ONLY
// (index only: the drain reads the state back from global memory, leaving
// more of the SM's on-chip memory to the L1 cache)
struct Stash {
  int32_t idx[kStashCap];
  uint8_t kp[kStashCap];
};
#else
struct Stash {
  int32_t idx[kStashCap];
  int32_t cell[kStashCap];
  float frac[kStashCap], ux[kStashCap], uy[kStashCap], uz[kStashCap];
  uint8_t kp[kStashCap];
};
#endif

// Push the first `cnt` (<= 32) stashed particles, one per lane, with 4^k
// sub-steps each; then move entries [cnt, n) to the front.  Warp-collective.
// Stash entry kp: k_prev in bits 0-2, bit 3 set for a predicted-queue particle
// (which stays in that queue).
template <int P, bool RING>
__device__ __forceinline__ void stash_drain(const PushArgsMixed& a, const StepFields<P, RING>& F,
                                            Stash& S, int k, int& n, int cnt,
                                            unsigned long long* sh) {
  const int lane = threadIdx.x & 31;
  if (lane < cnt) {
    const int32_t i = S.idx[lane];
#ifdef PIC_STASH_INDEX_ONLY
    MixedState s = load_state(a, i);
#else
    MixedState s = {S.cell[lane], S.frac[lane], S.ux[lane], S.uy[lane], S.uz[lane]};
#endif
    const uint8_t kp = S.kp[lane];
    const bool ok = subcycle_site<P, RING, RING>(F, a.wtab, a.mask, a.dt, a.inv_dx, a.qm,
                                                 a.field_time, a.mono, k, kp & 7, 0.f, s);
    normalize(s);
    store_state(a, i, s);
    a.status[i] = ok ? (uint8_t)(k | (kp & 8 ? kOwned : 0) | (a.parity_next ? kParity : 0))
                     : (uint8_t)(k | PIC_STATUS_LOST);
    if (!ok) atomicAdd(&sh[11], 1ull);
  }
  __syncwarp();
  const int rest = n - cnt;
  if (lane < rest) {
    const int q = cnt + lane;
    S.idx[lane] = S.idx[q];
#ifndef PIC_STASH_INDEX_ONLY
    S.cell[lane] = S.cell[q];
    S.frac[lane] = S.frac[q];
    S.ux[lane] = S.ux[q];
    S.uy[lane] = S.uy[q];
    S.uz[lane] = S.uz[q];
#endif
    S.kp[lane] = S.kp[q];
  }
  __syncwarp();
  n = rest;
}

// Deferred item: particle i is in a step before this launch's (a long
// sub-cycle, possibly partly done), or -- a predicted particle -- starts the
// long sub-cycle of this launch's step.  Finish it -- and, if it ran behind the
// stream, every step up to the previous one, taking each step's criterion --
// spending at most heavy_budget sub-steps of long sub-cycles; then take the
// criterion of the current step: pushed at once if k < kDeferMin, else
// deferred again.  Out of budget: the particle stays deferred where it is
// (offset not normalised) and resumes in the next launch -- but not in a step
// before keep_step (the last launch of a call that carries its deferred work
// into the next call: the steps whose levels the ring must keep), which it
// finishes regardless of the budget.  finalize: bring it
// to the end of the last step only (public status).
template <int P, bool RING>
__device__ __forceinline__ void heavy_particle(const PushArgsMixed& a, const StepFields<P, RING>& Fp,
                                            const StepFields<P, RING>& Fc, const float* wcrit,
                                            int64_t i, ThreadCounters& tc,
                                            unsigned long long* sh, int& defer_key) {
  defer_key = 0;
  const uint8_t st = a.status[i];
  int k = deferred_k(st);
  int k_prev = st & 7;
  MixedState s = load_state(a, i);
  int64_t si = a.step_cur - 1;  // the step the particle is in
  int j0 = 0;                    // its sub-steps already done
  bool lag = false;
  if constexpr (RING) {
    if (a.lag_step) {
      si = a.step0 + a.lag_step[i];
      j0 = a.lag_j[i];
      lag = true;
    }
  }
  int budget = lag && !a.finalize && a.heavy_budget > 0 ? a.heavy_budget : INT_MAX;
  float b0 = 0.f;  // the criterion's B_z of step si (used when k = 0)
  for (;;) {
    // sub-steps j0+1 .. j1 of step si
    const int m = 1 << (2 * k);
    int j1 = m;
    if (k >= kDeferMin && m - j0 > budget && si >= a.keep_step) j1 = j0 + budget;
    bool ok;
    if (si >= a.step_cur - 1) {  // the previous or the current step: node tables
      const StepFields<P, RING> Fs = si == a.step_cur ? Fc : Fp;
      ok = subcycle_site<P, RING, RING>(Fs, a.wtab, a.mask, a.dt, a.inv_dx, a.qm, a.field_time,
                                        a.mono, k, k_prev, b0, s, j0, j1);
    } else {
      if constexpr (RING) {
        const StepFields<P, true> Fs = ring_step_fields<P>(a, si);
        ok = subcycle_f32<P, true, false>(Fs, a.wtab, a.mask, a.dt, a.inv_dx, a.qm, a.field_time,
                                          a.mono, k, k_prev, b0, s, j0, j1);
      } else {
        ok = false;  // unreachable: without the lag arrays si is always the previous step
      }
    }
    if (k >= kDeferMin) budget -= j1 - j0;
    if (!ok) {
      store_state(a, i, s);
      a.status[i] = (uint8_t)(k | PIC_STATUS_LOST);
      atomicAdd(&sh[11], 1ull);
      return;
    }
    if (j1 < m) {  // out of budget inside the sub-cycle: resume here next launch
      store_state(a, i, s);
      defer_mark(a, i, k_prev, k, si, j1);
      defer_key = k;
      return;
    }
    normalize(s);
    if (si == a.step_cur) {  // the current step's short sub-cycle is done
      store_state(a, i, s);
      a.status[i] = (uint8_t)(k | (a.parity_next ? kParity : 0));
      return;
    }
    if (si == a.step_cur - 1) {
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
                                      a.k_max, capped, b0);
      count_step(tc, sh, kn, capped);
      if (kn >= kDeferMin) {
        store_state(a, i, s);
        defer_mark(a, i, k, kn, a.step_cur);
        defer_key = kn;
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
    if constexpr (RING) {
      si += 1;
      const StepFields<P, true> Fs = si == a.step_cur - 1 ? Fp : ring_step_fields<P>(a, si);
      int32_t je, jb;
      float we, wb;
      if (!tent_coords(s.cell, s.frac, Fs.lo, Fs.hi, je, we, jb, wb)) {
        store_state(a, i, s);
        a.status[i] = (uint8_t)(k | PIC_STATUS_LOST);
        atomicAdd(&sh[11], 1ull);
        return;
      }
      bool capped;
      const int kn = criterion_f32<P>(Fs.B, wcrit, jb, wb, a.mask, s, a.qm_abs, a.dt, a.psi_max,
                                      a.k_max, capped, b0);
      count_step(tc, sh, kn, capped);
      k_prev = k;
      k = kn;
      j0 = 0;
      if (k >= kDeferMin && budget <= 0 && si >= a.keep_step) {
        store_state(a, i, s);
        defer_mark(a, i, k_prev, k, si);
        defer_key = k;
        return;
      }
    }
  }
}

// Predicted item: particle i was binned at the last refresh of the
// predictions as likely to take k_pred.  Skipped unless it still belongs to
// the predicted queue (a particle deferred since then is the deferred items'
// and then the stream's).  Takes its exact criterion: k = 0, and a short k
// equal to the predicted one, are pushed at once (a warp of right predictions
// runs dense); another short k goes to the caller's stash (sk, with its state
// s and stash byte kp); both stay in the queue.  A long sub-cycle leaves the
// queue and, with
// resumable sub-cycles (run_heavy), starts at once in the caller's deferred-
// particle code, at most heavy_budget sub-steps in this launch -- so a warp of
// right predictions runs dense from the start of the launch -- else it is
// deferred to the next launch (key), as the stream would.
template <int P, bool RING>
__device__ __forceinline__ void predicted_particle(const PushArgsMixed& a, const StepFields<P, RING>& Fc,
                                                   const float* wcrit, int64_t i, int k_pred,
                                                   ThreadCounters& tc, unsigned long long* sh,
                                                   int& key, int& sk, MixedState& s, uint8_t& kp,
                                                   bool& run_heavy) {
  const uint8_t st = a.status[i];
  if ((st & (PIC_STATUS_LOST | kDeferMask)) != kOwned) return;
  const int k_prev = st & 7;
  kp = (uint8_t)(k_prev | 8);
  s = load_state(a, i);
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
  if (k == 0 || (k == k_pred && k < kDeferMin)) {
    const bool ok = subcycle_site<P, RING, RING>(Fc, a.wtab, a.mask, a.dt, a.inv_dx, a.qm,
                                                 a.field_time, a.mono, k, k_prev, b0, s);
    normalize(s);
    store_state(a, i, s);
    a.status[i] = ok ? (uint8_t)(k | kOwned | (a.parity_next ? kParity : 0))
                     : (uint8_t)(k | PIC_STATUS_LOST);
    if (!ok) atomicAdd(&sh[11], 1ull);
  } else if (k < kDeferMin) {
    sk = k;
  } else {
    defer_mark(a, i, k_prev, k, a.step_cur);  // in this step, none of its sub-steps done
    if (RING && a.lag_step)
      run_heavy = true;
    else
      key = k;
  }
}

}  // namespace pic
