// Self-consistent 1D3V PIC loop around the adaptive sub-cycling integrator
// (arXiv 2102.10983): push + deposit, Yee field solve, Gauss check.
//
// Compiled with -fmad=false: every FP64 multiply and add rounds separately in
// the order written, so the loop reproduces a serial FP64 evaluation of the
// same definitions bit for bit.  The current deposit is exact fixed point
// (int64 units of 2^-44 n_c e, two's-complement atomics), so the order in
// which threads add their contributions does not change a bit either.
//
// Per macro step n (state: x at t_n, p at t_n - h_old/2):
//   push_deposit_kernel<P>: one thread per electron.  Criterion of Sec. IV
//     (|B_z| at x_n, t_n, gamma of the stored momentum; smallest k with
//     Psi0/4^k <= Psi_max); m = 4^k sub-steps of h = dt/4^k, the first with
//     (h_old + h)/2; each sub-step gathers E_x, E_y, B_z with the order-p
//     weights of Sec. VI (tabulated per (k, j)) and the tent (Eqs. eq:Enp,
//     eq:Bnp), takes the Boris push with E = (E_x, E_y, 0) (Eqs. eq:p -
//     eq:gamman) and moves x by h v_x (Eq. eq:x).  It adds (h/dt) v_y S(x_mid)
//     of every sub-step to per-node FP64 sums in registers, and at the end of
//     the macro step one rounded fixed-point value per node to J_y, and the
//     charge flux of its move (start -> end or frozen position) to J_x.
//   field_kernel: E_y^{n+1} (Eq. eq:Ey with -dt J_y; Mur at both ends),
//     E_x^{n+1} = E_x^n - dt J_x, B_z^{n+3/2} (Eq. eq:Bz); also clears the
//     other parity's accumulators for the next step.
//   rho_kernel + gauss_kernel (on request): node charges from the positions
//     and max_k |(E_x_{k+1/2} - E_x_{k-1/2})/dx - rho_k|.
#include <math.h>
#include <stdio.h>
#include <string.h>

#include <vector>

#include "pic_internal.h"
#include "pic_sc1d.h"

namespace pic {
namespace {

constexpr double kUnit = 0x1p-44;  // fixed-point charge unit

struct Sc1dArgs {
  int64_t n;
  double *x, *px, *py, *pz;
  uint8_t* status;
  const int64_t* Q;
  const double* Ex[kMaxOrder + 1];  // levels n-p .. n
  const double* Ey[kMaxOrder + 1];
  const double* Bz[kMaxOrder + 1];  // levels n+1/2-p .. n+1/2
  unsigned long long* F;            // J_x face fluxes (int64 two's complement)
  unsigned long long* D;            // J_y node sums
  int64_t M;                        // entries of every grid array (n_cells + 5)
  int32_t n_cells;
  double dt, inv_dx, psi_max, qm, qm_abs;
  int k_max;
  const double* wtab;
  int64_t crit_row;
  DevStats* stats;
};

// Field of one grid at coordinate u (node units of that grid), weights w over
// the P+1 levels in ascending time: temporal sums at the two tent nodes, then
// the tent weight.
template <int P>
__device__ __forceinline__ double gather(const double* const* lv, const double* w, double u) {
  const double fl = floor(u);
  const int64_t j = (int64_t)fl + 2;
  const double frac = u - fl;
  double f0 = w[0] * lv[0][j];
  double f1 = w[0] * lv[0][j + 1];
#pragma unroll
  for (int l = 1; l <= P; ++l) {
    f0 = f0 + w[l] * lv[l][j];
    f1 = f1 + w[l] * lv[l][j + 1];
  }
  return f0 + frac * (f1 - f0);
}

__device__ __forceinline__ bool inside(double s, int32_t n_cells) {
  return s >= 0.5 && s < (double)n_cells - 0.5;
}

// Node charges of Q at s: r0 at node floor(s), r1 at floor(s)+1, r0 + r1 = Q.
__device__ __forceinline__ void split(int64_t Q, double s, int64_t& i, int64_t& r0, int64_t& r1) {
  const double fl = floor(s);
  i = (int64_t)fl;
  r1 = __double2ll_rn((double)Q * (s - fl));
  r0 = Q - r1;
}

// a[idx] += v; an index outside [0, M) (only a non-finite position could
// make one) is dropped instead of written
__device__ __forceinline__ void add_i64(unsigned long long* a, int64_t idx, int64_t M, int64_t v) {
  if (idx >= 0 && idx < M) atomicAdd(a + idx, (unsigned long long)v);
}

template <int P>
__global__ void __launch_bounds__(256) push_deposit_kernel(Sc1dArgs a) {
  __shared__ unsigned long long sh[12];
  if (threadIdx.x < 12) sh[threadIdx.x] = 0ull;
  __syncthreads();
  constexpr int stride = 2 * (P + 1);
  const double* wcrit = a.wtab + a.crit_row * stride + (P + 1);
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < a.n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const uint8_t st = a.status[i];
    if (st & PIC_STATUS_LOST) continue;
    const int k_prev = st & 0x7f;
    double pv0 = a.px[i], pv1 = a.py[i], pv2 = a.pz[i];
    double xi = a.x[i];
    const double s_a = xi * a.inv_dx;
    if (!inside(s_a, a.n_cells)) {
      a.status[i] = (uint8_t)(st | PIC_STATUS_LOST);
      atomicAdd(&sh[11], 1ull);
      continue;
    }
    const double b0 = gather<P>(a.Bz, wcrit, s_a - 0.5);
    const double g0 = sqrt(1.0 + (pv0 * pv0 + pv1 * pv1 + pv2 * pv2));
    double psi = (a.qm_abs * fabs(b0) * a.dt) / (2.0 * g0);
    int k = 0;
    while (psi > a.psi_max && k < a.k_max) {
      psi = psi * 0.25;
      ++k;
    }
    const bool capped = psi > a.psi_max;
    const int64_t m = (int64_t)1 << (2 * k);
    const double h = ldexp(a.dt, -2 * k);
    const double h_old = ldexp(a.dt, -2 * k_prev);
    const double inv_m = ldexp(1.0, -2 * k);
    atomicAdd(&sh[k], 1ull);
    atomicAdd(&sh[8], (unsigned long long)m);
    if (k > 0) atomicAdd(&sh[9], (unsigned long long)m);
    if (capped) atomicAdd(&sh[10], 1ull);

    // J_y sums of nodes base .. base+4, base = floor(s_a) - 2 (a macro step
    // moves an electron less than one cell: c dt < dx)
    const int64_t base = (int64_t)floor(s_a) - 2;
    double acc[5] = {0.0, 0.0, 0.0, 0.0, 0.0};
    const double* wr = a.wtab + wrow(k, 1) * stride;
    bool frozen = false;
    for (int64_t j = 1; j <= m; ++j, wr += stride) {
      const double s = xi * a.inv_dx;
      if (!inside(s, a.n_cells)) {
        frozen = true;
        break;
      }
      const double ex = gather<P>(a.Ex, wr, s - 0.5);
      const double ey = gather<P>(a.Ey, wr, s);
      const double bz = gather<P>(a.Bz, wr + (P + 1), s - 0.5);
      const double hp = (j == 1) ? 0.5 * (h_old + h) : h;
      // Boris, E = (ex, ey, 0), B = (0, 0, bz)
      const double half = 0.5 * hp;
      const double dpx = (a.qm * ex) * half;
      const double dpy = (a.qm * ey) * half;
      const double mx = pv0 + dpx, my = pv1 + dpy, mz = pv2;
      const double gn = sqrt(1.0 + (mx * mx + my * my + mz * mz));
      const double tz = ((a.qm * bz) * half) / gn;
      const double ppx = mx + my * tz;
      const double ppy = my - mx * tz;
      const double sz = (2.0 * tz) / (1.0 + tz * tz);
      const double qx = mx + ppy * sz;
      const double qy = my - ppx * sz;
      pv0 = qx + dpx;
      pv1 = qy + dpy;
      pv2 = mz;
      const double g = sqrt(1.0 + (pv0 * pv0 + pv1 * pv1 + pv2 * pv2));
      const double vx = pv0 / g, vy = pv1 / g;
      const double s_mid = (xi + 0.5 * (h * vx)) * a.inv_dx;
      xi = xi + h * vx;
      const double fl = floor(s_mid);
      const int c = (int)((int64_t)fl - base);
      const double cw = vy * inv_m;  // (h/dt) v_y
      const double t = cw * (s_mid - fl);
#pragma unroll
      for (int q = 0; q < 4; ++q) {  // acc[c] += cw - t; acc[c+1] += t (registers)
        if (q == c) {
          acc[q] = acc[q] + (cw - t);
          acc[q + 1] = acc[q + 1] + t;
        }
      }
    }
    a.x[i] = xi;
    a.px[i] = pv0;
    a.py[i] = pv1;
    a.pz[i] = pv2;
    if (frozen) {
      a.status[i] = (uint8_t)(k | PIC_STATUS_LOST);
      atomicAdd(&sh[11], 1ull);
    } else {
      a.status[i] = (uint8_t)k;
    }
    const int64_t Q = a.Q[i];
#pragma unroll
    for (int c = 0; c < 5; ++c)
      if (acc[c] != 0.0) add_i64(a.D, base + c + 2, a.M, -__double2ll_rn(acc[c] * (double)Q));
    // J_x: the charge flux of the move s_a -> s_b through the faces
    const double s_b = xi * a.inv_dx;
    int64_t ia, ib, ra0, ra1, rb0, rb1;
    split(Q, s_a, ia, ra0, ra1);
    split(Q, s_b, ib, rb0, rb1);
    const int64_t lo = (ia < ib ? ia : ib) - 1;
    int64_t dC[6] = {0, 0, 0, 0, 0, 0};
#pragma unroll
    for (int c = 0; c < 6; ++c) {
      if (lo + c == ia) dC[c] += ra0;      // the electron's charge -r leaves s_a
      if (lo + c == ia + 1) dC[c] += ra1;
      if (lo + c == ib) dC[c] -= rb0;      // and arrives at s_b
      if (lo + c == ib + 1) dC[c] -= rb1;
    }
    int64_t flux = 0;
#pragma unroll
    for (int c = 0; c < 6; ++c) {
      flux -= dC[c];
      if (flux != 0) add_i64(a.F, lo + c + 2, a.M, flux);
    }
  }
  __syncthreads();
  if (threadIdx.x < 12) {
    const unsigned long long v = sh[threadIdx.x];
    if (v) {
      unsigned long long* dst = threadIdx.x < 8 ? &a.stats->k_hist[threadIdx.x]
                                : threadIdx.x == 8 ? &a.stats->substeps
                                : threadIdx.x == 9 ? &a.stats->n_star
                                : threadIdx.x == 10 ? &a.stats->clamped
                                                    : &a.stats->lost;
      atomicAdd(dst, v);
    }
  }
}

struct FieldArgs {
  const double *Ex0, *Ey0, *Bz0;
  double *Ex1, *Ey1, *Bz1;
  unsigned long long* F;  // this step's accumulators (read)
  unsigned long long* D;
  unsigned long long* F_next;  // the next step's (cleared)
  unsigned long long* D_next;
  int64_t N;
  double dt, dx, r, kappa;
};

// E_y^{n+1} at array index q (node q - 2): interior Yee update with -dt J_y,
// Mur at the two ends, zero in the padding.
__device__ __forceinline__ double ey_next(const FieldArgs& a, int64_t q) {
  auto interior = [&](int64_t u) {
    return (a.Ey0[u] - a.r * (a.Bz0[u] - a.Bz0[u - 1])) - a.dt * ((double)(long long)a.D[u] * kUnit);
  };
  const int64_t k = q - 2;
  if (k >= 1 && k <= a.N - 1) return interior(q);
  if (k == 0) return a.Ey0[3] + a.kappa * (interior(3) - a.Ey0[2]);
  if (k == a.N) return a.Ey0[a.N + 1] + a.kappa * (interior(a.N + 1) - a.Ey0[a.N + 2]);
  return 0.0;
}

__global__ void field_kernel(FieldArgs a) {
  const int64_t M = a.N + 5;
  for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < M;
       q += (int64_t)gridDim.x * blockDim.x) {
    a.Ex1[q] = a.Ex0[q] - ((double)(long long)a.F[q] * kUnit) * a.dx;
    const double e = ey_next(a, q);
    a.Ey1[q] = e;
    const int64_t k = q - 2;
    a.Bz1[q] = (k >= 0 && k <= a.N - 1) ? a.Bz0[q] - a.r * (ey_next(a, q + 1) - e) : 0.0;
    a.F_next[q] = 0ull;
    a.D_next[q] = 0ull;
  }
}

__global__ void rho_kernel(const double* x, const int64_t* Q, int64_t n, double inv_dx,
                           unsigned long long* C, int64_t M, int negate) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    int64_t ii, r0, r1;
    split(Q[i], x[i] * inv_dx, ii, r0, r1);
    add_i64(C, ii + 2, M, negate ? r0 : -r0);
    add_i64(C, ii + 3, M, negate ? r1 : -r1);
  }
}

// max over nodes k = -1 .. N+1 of |(E_x_{k+1/2} - E_x_{k-1/2})/dx - rho_k| and
// of |rho^e_k| (non-negative doubles compare like their bit patterns)
__global__ void gauss_kernel(const double* Ex, const unsigned long long* C,
                             const unsigned long long* C_ion, int64_t N, double inv_dx,
                             unsigned long long* out) {
  for (int64_t k = -1 + blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k <= N + 1;
       k += (int64_t)gridDim.x * blockDim.x) {
    const int64_t q = k + 2;
    const double rho = (double)((long long)C[q] + (long long)C_ion[q]) * kUnit;
    const double g = fabs((Ex[q] - Ex[q - 1]) * inv_dx - rho);
    const double re = fabs((double)(long long)C[q] * kUnit);
    atomicMax(&out[0], (unsigned long long)__double_as_longlong(g));
    atomicMax(&out[1], (unsigned long long)__double_as_longlong(re));
  }
}

__global__ void charge_units_kernel(const double* w, int64_t* Q, int64_t n) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    Q[i] = __double2ll_rn(w[i] * 0x1p44);
}

}  // namespace
}  // namespace pic

using namespace pic;

struct pic_sc1d {
  pic_sc1d_params prm;
  int64_t capacity = 0, n = 0, M = 0;
  int R = 0;  // ring slots (order + 1)
  cudaStream_t stream = nullptr;
  int sm_count = 0;
  double *x = nullptr, *px = nullptr, *py = nullptr, *pz = nullptr, *w_stage = nullptr;
  uint8_t* status = nullptr;
  int64_t* Q = nullptr;
  double* ring = nullptr;  // R slots x 3 fields x M
  std::vector<int64_t> slot_level;
  unsigned long long* acc = nullptr;  // [2 parities][F, D][M], then C, C_ion [M] each, gauss [2]
  double* wtab = nullptr;
  DevStats* dstats = nullptr;
  double* staging = nullptr;  // 3 M host-upload staging
  int64_t launches = 0;
  double gauss_res = 0.0, rho_max = 0.0;
  int32_t checks = 0;
  cudaEvent_t ev0 = nullptr, ev1 = nullptr;
  bool timing = false, timed = false;
  double timed_ms = 0.0;
  int64_t timed_steps = 0;
  char err[256] = {0};
};

static thread_local char g_sc_err[256];

static int sc_fail(pic_sc1d* c, int code, const char* msg, const char* detail = "") {
  char* dst = c ? c->err : g_sc_err;
  snprintf(dst, 256, "%s%s", msg, detail);
  return code;
}

#define SC_TRY(c, call)                                                           \
  do {                                                                            \
    cudaError_t e_ = (call);                                                      \
    if (e_ != cudaSuccess) return sc_fail((c), PIC_ECUDA, #call ": ", cudaGetErrorString(e_)); \
  } while (0)

static double* slot_field(pic_sc1d* c, int slot, int f) {
  return c->ring + ((int64_t)slot * 3 + f) * c->M;
}
static unsigned long long* accF(pic_sc1d* c, int par) { return c->acc + (int64_t)(2 * par) * c->M; }
static unsigned long long* accD(pic_sc1d* c, int par) { return c->acc + (int64_t)(2 * par + 1) * c->M; }
static unsigned long long* accC(pic_sc1d* c) { return c->acc + 4 * c->M; }
static unsigned long long* accCion(pic_sc1d* c) { return c->acc + 5 * c->M; }
static unsigned long long* accGauss(pic_sc1d* c) { return c->acc + 6 * c->M; }
static int grid_for(const pic_sc1d* c, int64_t n) {
  const int64_t want = (n + 255) / 256;
  const int64_t cap = (int64_t)(c->sm_count > 0 ? c->sm_count : 152) * 8;
  return (int)(want < 1 ? 1 : (want < cap ? want : cap));
}

extern "C" int pic_sc1d_create(const pic_sc1d_params* prm, int64_t capacity, void* stream,
                               pic_sc1d** out) {
  if (!prm || !out) return sc_fail(nullptr, PIC_EINVAL, "pic_sc1d_create: NULL argument");
  *out = nullptr;
  if (!(prm->dt > 0) || !(prm->dx > 0) || !(prm->psi_max > 0) || !isfinite(prm->qm) || prm->qm == 0.0)
    return sc_fail(nullptr, PIC_EINVAL, "pic_sc1d_create: dt, dx, psi_max must be > 0, qm != 0");
  if (!(prm->dt < prm->dx))
    return sc_fail(nullptr, PIC_EINVAL, "pic_sc1d_create: the Yee scheme needs c dt < dx");
  if (prm->order < 1 || prm->order > kMaxOrder || prm->k_max < 0 || prm->k_max > kMaxK ||
      (prm->field_time != 0 && prm->field_time != 1) || prm->n_cells < 16 ||
      prm->n_cells > (1 << 26) || prm->gauss_every < 0 || capacity < 0)
    return sc_fail(nullptr, PIC_EINVAL, "pic_sc1d_create: parameter out of range");
  pic_sc1d* c = new pic_sc1d();
  c->prm = *prm;
  c->capacity = capacity;
  c->M = (int64_t)prm->n_cells + 5;
  c->R = prm->order + 1;
  c->stream = (cudaStream_t)stream;
  c->slot_level.assign(c->R, INT64_MIN);
  int dev = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&c->sm_count, cudaDevAttrMultiProcessorCount, dev);
  const int64_t cap = capacity > 0 ? capacity : 1;
  bool ok = true;
  ok &= cudaMalloc(&c->x, cap * 8) == cudaSuccess;
  ok &= cudaMalloc(&c->px, cap * 8) == cudaSuccess;
  ok &= cudaMalloc(&c->py, cap * 8) == cudaSuccess;
  ok &= cudaMalloc(&c->pz, cap * 8) == cudaSuccess;
  ok &= cudaMalloc(&c->w_stage, cap * 8) == cudaSuccess;
  ok &= cudaMalloc(&c->status, cap) == cudaSuccess;
  ok &= cudaMalloc(&c->Q, cap * 8) == cudaSuccess;
  ok &= cudaMalloc(&c->ring, (int64_t)c->R * 3 * c->M * 8) == cudaSuccess;
  ok &= cudaMalloc(&c->acc, (6 * c->M + 2) * 8) == cudaSuccess;
  const int64_t wcount = wrows_total(prm->k_max) * 2 * (prm->order + 1);
  ok &= cudaMalloc(&c->wtab, wcount * 8) == cudaSuccess;
  ok &= cudaMalloc(&c->dstats, sizeof(DevStats)) == cudaSuccess;
  ok &= cudaMalloc(&c->staging, 3 * c->M * 8) == cudaSuccess;
  if (!ok) {
    pic_sc1d_destroy(c);
    return sc_fail(nullptr, PIC_ENOMEM, "pic_sc1d_create: device allocation failed");
  }
  cudaError_t e = cudaMemsetAsync(c->ring, 0, (int64_t)c->R * 3 * c->M * 8, c->stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(c->acc, 0, (6 * c->M + 2) * 8, c->stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(c->dstats, 0, sizeof(DevStats), c->stream);
  if (e == cudaSuccess) e = build_wtab_f64(c->wtab, prm->order, prm->k_max, prm->field_time, c->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
  if (e != cudaSuccess) {
    pic_sc1d_destroy(c);
    return sc_fail(nullptr, PIC_ECUDA, "pic_sc1d_create: ", cudaGetErrorString(e));
  }
  c->launches = 1;
  *out = c;
  return PIC_OK;
}

extern "C" int pic_sc1d_destroy(pic_sc1d* c) {
  if (!c) return PIC_OK;
  cudaFree(c->x); cudaFree(c->px); cudaFree(c->py); cudaFree(c->pz); cudaFree(c->w_stage);
  cudaFree(c->status); cudaFree(c->Q); cudaFree(c->ring); cudaFree(c->acc); cudaFree(c->wtab);
  cudaFree(c->dstats); cudaFree(c->staging);
  if (c->ev0) cudaEventDestroy(c->ev0);
  if (c->ev1) cudaEventDestroy(c->ev1);
  delete c;
  return PIC_OK;
}

static cudaMemcpyKind kind_to_dev(int where) {
  return where == PIC_HOST ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice;
}
static cudaMemcpyKind kind_from_dev(int where) {
  return where == PIC_HOST ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice;
}

extern "C" int pic_sc1d_particles_write(pic_sc1d* c, const double* x, const double* px,
                                        const double* py, const double* pz, const double* w,
                                        int64_t n, int32_t where) {
  if (!c) return PIC_EINVAL;
  if (n < 0 || n > c->capacity) return sc_fail(c, PIC_EINVAL, "pic_sc1d_particles_write: n out of range");
  if (where != PIC_HOST && where != PIC_DEVICE) return sc_fail(c, PIC_EINVAL, "bad where");
  if (n > 0 && (!x || !px || !py || !pz || !w)) return sc_fail(c, PIC_EINVAL, "NULL particle array");
  const cudaMemcpyKind k = kind_to_dev(where);
  if (n > 0) {
    SC_TRY(c, cudaMemcpyAsync(c->x, x, n * 8, k, c->stream));
    SC_TRY(c, cudaMemcpyAsync(c->px, px, n * 8, k, c->stream));
    SC_TRY(c, cudaMemcpyAsync(c->py, py, n * 8, k, c->stream));
    SC_TRY(c, cudaMemcpyAsync(c->pz, pz, n * 8, k, c->stream));
    SC_TRY(c, cudaMemcpyAsync(c->w_stage, w, n * 8, k, c->stream));
  }
  SC_TRY(c, cudaMemsetAsync(c->status, 0, n > 0 ? n : 1, c->stream));
  c->n = n;
  // fixed-point charges, then the ion background: minus the electrons' charge
  SC_TRY(c, cudaMemsetAsync(accCion(c), 0, c->M * 8, c->stream));
  if (n > 0) {
    charge_units_kernel<<<grid_for(c, n), 256, 0, c->stream>>>(c->w_stage, c->Q, n);
    rho_kernel<<<grid_for(c, n), 256, 0, c->stream>>>(c->x, c->Q, n, 1.0 / c->prm.dx, accCion(c), c->M, 1);
    c->launches += 2;
  }
  SC_TRY(c, cudaGetLastError());
  if (where == PIC_HOST) SC_TRY(c, cudaStreamSynchronize(c->stream));
  return PIC_OK;
}

extern "C" int pic_sc1d_particles_read(pic_sc1d* c, double* x, double* px, double* py, double* pz,
                                       uint8_t* status, int64_t n, int32_t where) {
  if (!c) return PIC_EINVAL;
  if (n < 0 || n > c->n) return sc_fail(c, PIC_EINVAL, "pic_sc1d_particles_read: n out of range");
  if (where != PIC_HOST && where != PIC_DEVICE) return sc_fail(c, PIC_EINVAL, "bad where");
  const cudaMemcpyKind k = kind_from_dev(where);
  if (n > 0) {
    if (x) SC_TRY(c, cudaMemcpyAsync(x, c->x, n * 8, k, c->stream));
    if (px) SC_TRY(c, cudaMemcpyAsync(px, c->px, n * 8, k, c->stream));
    if (py) SC_TRY(c, cudaMemcpyAsync(py, c->py, n * 8, k, c->stream));
    if (pz) SC_TRY(c, cudaMemcpyAsync(pz, c->pz, n * 8, k, c->stream));
    if (status) SC_TRY(c, cudaMemcpyAsync(status, c->status, n, k, c->stream));
  }
  if (where == PIC_HOST) SC_TRY(c, cudaStreamSynchronize(c->stream));
  return PIC_OK;
}

static int slot_of(const pic_sc1d* c, int64_t level) {
  return (int)(((level % c->R) + c->R) % c->R);
}

extern "C" int pic_sc1d_fields_write(pic_sc1d* c, int64_t level, const double* Ex, const double* Ey,
                                     const double* Bz, int32_t where) {
  if (!c) return PIC_EINVAL;
  if (!Ex || !Ey || !Bz) return sc_fail(c, PIC_EINVAL, "pic_sc1d_fields_write: NULL field");
  if (where != PIC_HOST && where != PIC_DEVICE) return sc_fail(c, PIC_EINVAL, "bad where");
  const int s = slot_of(c, level);
  const cudaMemcpyKind k = kind_to_dev(where);
  SC_TRY(c, cudaMemcpyAsync(slot_field(c, s, 0), Ex, c->M * 8, k, c->stream));
  SC_TRY(c, cudaMemcpyAsync(slot_field(c, s, 1), Ey, c->M * 8, k, c->stream));
  SC_TRY(c, cudaMemcpyAsync(slot_field(c, s, 2), Bz, c->M * 8, k, c->stream));
  if (where == PIC_HOST) SC_TRY(c, cudaStreamSynchronize(c->stream));
  c->slot_level[s] = level;
  return PIC_OK;
}

extern "C" int pic_sc1d_fields_read(pic_sc1d* c, int64_t level, double* Ex, double* Ey, double* Bz,
                                    int32_t where) {
  if (!c) return PIC_EINVAL;
  if (where != PIC_HOST && where != PIC_DEVICE) return sc_fail(c, PIC_EINVAL, "bad where");
  const int s = slot_of(c, level);
  if (c->slot_level[s] != level) return sc_fail(c, PIC_EINVAL, "pic_sc1d_fields_read: level not stored");
  const cudaMemcpyKind k = kind_from_dev(where);
  if (Ex) SC_TRY(c, cudaMemcpyAsync(Ex, slot_field(c, s, 0), c->M * 8, k, c->stream));
  if (Ey) SC_TRY(c, cudaMemcpyAsync(Ey, slot_field(c, s, 1), c->M * 8, k, c->stream));
  if (Bz) SC_TRY(c, cudaMemcpyAsync(Bz, slot_field(c, s, 2), c->M * 8, k, c->stream));
  if (where == PIC_HOST) SC_TRY(c, cudaStreamSynchronize(c->stream));
  return PIC_OK;
}

static int sc_gauss(pic_sc1d* c) {
  SC_TRY(c, cudaMemsetAsync(accC(c), 0, c->M * 8, c->stream));
  if (c->n > 0) {
    rho_kernel<<<grid_for(c, c->n), 256, 0, c->stream>>>(c->x, c->Q, c->n, 1.0 / c->prm.dx, accC(c), c->M, 0);
    ++c->launches;
  }
  return PIC_OK;
}

template <int P>
static void launch_push(const Sc1dArgs& a, int blocks, cudaStream_t s) {
  push_deposit_kernel<P><<<blocks, 256, 0, s>>>(a);
}

extern "C" int pic_sc1d_step(pic_sc1d* c, int64_t n0, int64_t n_steps, pic_sc1d_stats* stats) {
  if (!c) return PIC_EINVAL;
  if (n_steps < 1) return sc_fail(c, PIC_EINVAL, "pic_sc1d_step: n_steps must be >= 1");
  const int p = c->prm.order;
  for (int l = 0; l <= p; ++l)
    if (c->slot_level[slot_of(c, n0 - p + l)] != n0 - p + l)
      return sc_fail(c, PIC_EINVAL, "pic_sc1d_step: levels n0-p .. n0 must be stored");
  if (c->timing && !c->ev0) {
    SC_TRY(c, cudaEventCreate(&c->ev0));
    SC_TRY(c, cudaEventCreate(&c->ev1));
  }
  if (c->timing) SC_TRY(c, cudaEventRecord(c->ev0, c->stream));
  const double r = c->prm.dt / c->prm.dx;
  for (int64_t j = 0; j < n_steps; ++j) {
    const int64_t s = n0 + j;
    const int par = (int)(s & 1);
    Sc1dArgs a;
    memset(&a, 0, sizeof(a));
    a.n = c->n;
    a.x = c->x; a.px = c->px; a.py = c->py; a.pz = c->pz;
    a.status = c->status;
    a.Q = c->Q;
    for (int l = 0; l <= p; ++l) {
      const int se = slot_of(c, s - p + l);
      a.Ex[l] = slot_field(c, se, 0);
      a.Ey[l] = slot_field(c, se, 1);
      a.Bz[l] = slot_field(c, se, 2);
    }
    a.F = accF(c, par);
    a.D = accD(c, par);
    a.M = c->M;
    a.n_cells = c->prm.n_cells;
    a.dt = c->prm.dt;
    a.inv_dx = 1.0 / c->prm.dx;
    a.psi_max = c->prm.psi_max;
    a.qm = c->prm.qm;
    a.qm_abs = fabs(c->prm.qm);
    a.k_max = c->prm.k_max;
    a.wtab = c->wtab;
    a.crit_row = wrows_total(c->prm.k_max) - 1;
    a.stats = c->dstats;
    if (c->n > 0) {
      const int blocks = grid_for(c, c->n);
      switch (p) {
        case 1: launch_push<1>(a, blocks, c->stream); break;
        case 2: launch_push<2>(a, blocks, c->stream); break;
        case 3: launch_push<3>(a, blocks, c->stream); break;
        case 4: launch_push<4>(a, blocks, c->stream); break;
        case 5: launch_push<5>(a, blocks, c->stream); break;
      }
      ++c->launches;
    }
    FieldArgs f;
    const int s0 = slot_of(c, s), s1 = slot_of(c, s + 1);
    f.Ex0 = slot_field(c, s0, 0); f.Ey0 = slot_field(c, s0, 1); f.Bz0 = slot_field(c, s0, 2);
    f.Ex1 = slot_field(c, s1, 0); f.Ey1 = slot_field(c, s1, 1); f.Bz1 = slot_field(c, s1, 2);
    f.F = accF(c, par); f.D = accD(c, par);
    f.F_next = accF(c, par ^ 1); f.D_next = accD(c, par ^ 1);
    f.N = c->prm.n_cells;
    f.dt = c->prm.dt;
    f.dx = c->prm.dx;
    f.r = r;
    f.kappa = (r - 1.0) / (r + 1.0);
    field_kernel<<<grid_for(c, c->M), 256, 0, c->stream>>>(f);
    ++c->launches;
    SC_TRY(c, cudaGetLastError());
    c->slot_level[s1] = s + 1;
    const int ge = c->prm.gauss_every;
    if (ge > 0 && (((s + 1) % ge) + ge) % ge == 0) {  // after steps s + 1 = multiples of ge
      int rc = sc_gauss(c);
      if (rc != PIC_OK) return rc;
      gauss_kernel<<<grid_for(c, c->M), 256, 0, c->stream>>>(slot_field(c, s1, 0), accC(c), accCion(c),
                                                             c->prm.n_cells, 1.0 / c->prm.dx,
                                                             accGauss(c));
      ++c->launches;
      ++c->checks;  // the maxima accumulate on the device until stats are read
    }
  }
  if (c->timing) {
    SC_TRY(c, cudaEventRecord(c->ev1, c->stream));
    SC_TRY(c, cudaEventSynchronize(c->ev1));
    float ms = 0.f;
    SC_TRY(c, cudaEventElapsedTime(&ms, c->ev0, c->ev1));
    c->timed_ms += ms;
    c->timed_steps += n_steps;
  }
  if (!stats) return PIC_OK;
  DevStats h;
  unsigned long long g[2];
  SC_TRY(c, cudaMemcpyAsync(&h, c->dstats, sizeof(DevStats), cudaMemcpyDeviceToHost, c->stream));
  SC_TRY(c, cudaMemcpyAsync(g, accGauss(c), 16, cudaMemcpyDeviceToHost, c->stream));
  SC_TRY(c, cudaMemsetAsync(c->dstats, 0, sizeof(DevStats), c->stream));
  SC_TRY(c, cudaMemsetAsync(accGauss(c), 0, 16, c->stream));
  SC_TRY(c, cudaStreamSynchronize(c->stream));
  memcpy(&c->gauss_res, &g[0], 8);
  memcpy(&c->rho_max, &g[1], 8);
  memset(stats, 0, sizeof(*stats));
  for (int k = 0; k < 8; ++k) stats->k_hist[k] = (int64_t)h.k_hist[k];
  stats->substeps = (int64_t)h.substeps;
  stats->n_star = (int64_t)h.n_star;
  stats->clamped = (int64_t)h.clamped;
  stats->frozen = (int64_t)h.lost;
  stats->gauss_residual = c->gauss_res;
  stats->rho_max = c->rho_max;
  stats->checks = c->checks;
  c->gauss_res = 0.0;
  c->checks = 0;
  if (stats->clamped) return sc_fail(c, PIC_EKMAX, "criterion capped at k_max");
  return PIC_OK;
}

extern "C" int pic_sc1d_timing(pic_sc1d* c, double* total_ms, int64_t* steps) {
  if (!c) return PIC_EINVAL;
  c->timing = true;
  if (total_ms) *total_ms = c->timed_ms;
  if (steps) *steps = c->timed_steps;
  c->timed_ms = 0.0;
  c->timed_steps = 0;
  return PIC_OK;
}

extern "C" int64_t pic_sc1d_launch_count(const pic_sc1d* c) { return c ? c->launches : 0; }

extern "C" const char* pic_sc1d_last_error(const pic_sc1d* c) { return c ? c->err : g_sc_err; }
