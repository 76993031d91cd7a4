// Single-electron studies of Secs. IV-VII on the GPU: electrons from rest
// through the Gaussian-enveloped plane wave of Eqs. laser5 - laser3
// (a = a0 exp(-(xi - xi0)^2 / (2 sigma^2)) sin xi, E_y = B_z = -da/dxi) with
// the field sampled on the grid (the "perfectly propagating PIC" of Sec. III):
// E_y at nodes i dx and times n dt, B_z at (i + 1/2) dx and (n + 1/2) dt.
//
// One thread per electron of a case (a0, dt, dx, Psi_max, order, ...), one
// warp per CTA, x0 = j lambda / n_electrons; each thread integrates its whole
// trajectory with the method (Algorithm 1 of Sec. IV, order-p Lagrange in
// time of Sec. VI, tent in space, Boris), in FP64 compiled with -fmad=false in
// the order of a serial evaluation.  The field values a gather needs are
// computed from the formula (the device's exp, sin, cos) and cached per grid
// for the current node pair and level window: a macro step that keeps the
// nodes computes only the newest level, a sub-step none.
//
// Per electron and macro step (Sec. IV, Eqs. R error, gamma error): R = gamma
// - p_x, the energy error |gamma - gamma_th| / gamma_th with gamma_th = 1 +
// a(xi_p)^2 / 2 at the momentum's phase xi_p = t_p - x_p (t_p = t_{n+1} - h/2,
// x_p = x - (h/2) v_x); per case the maxima over steps and electrons, electron
// 0's own values, N and N* (Sec. VII).
#include <math.h>
#include <stdint.h>
#include <string.h>

#include <vector>

#include "pic_internal.h"

namespace pic {
namespace {

__device__ __forceinline__ double a_of(const pic_study_case& q, double xi) {
  const double d = xi - q.xi0;
  return q.a0 * exp(-(d * d) / (2.0 * q.sigma * q.sigma)) * sin(xi);
}

// E_y = B_z = -da/dxi (Eq. laser5)
__device__ __forceinline__ double field_of(const pic_study_case& q, double xi) {
  const double d = xi - q.xi0;
  const double env = exp(-(d * d) / (2.0 * q.sigma * q.sigma));
  double sn, cs;
  sincos(xi, &sn, &cs);  // one argument reduction for both
  return -(q.a0 * env * (cs - (d / (q.sigma * q.sigma)) * sn));
}

// The rounded reciprocals of the integer denominators prod_{k != j} (j - k),
// formed once per electron (the same values the weights' definition rounds).
__device__ void lagrange_inv_den(int p, double* inv_den) {
  for (int j = 0; j <= p; ++j) {
    long long den = 1;
    for (int k = 0; k <= p; ++k)
      if (k != j) den *= (long long)(j - k);
    inv_den[j] = 1.0 / (double)den;
  }
}

__device__ void lagrange(int p, bool is_e, double theta, const double* inv_den, double* w) {
  const double c_off = is_e ? -0.5 : -1.0;
  for (int j = 0; j <= p; ++j) {
    double num = 1.0;
    bool first = true;
    for (int k = 0; k <= p; ++k) {
      if (k == j) continue;
      const double factor = ((double)(p - k) + c_off) + theta;
      if (first) {
        num = factor;
        first = false;
      } else {
        num = num * factor;
      }
    }
    w[j] = num * inv_den[j];
  }
}

// The field values of one grid at its current node pair (j, j + 1) for the
// levels n - p .. n (E: times (n - p + l) dt; B: + dt/2), computed on demand.
template <int P>
struct GridCache {
  double v0[P + 1], v1[P + 1];
  double j = -1e300;  // node of v0 (a node index, held as a double)
  int64_t n = INT64_MIN;

  __device__ void ensure(const pic_study_case& q, bool is_b, double j_new, int64_t n_new) {
    if (j_new == j && n_new == n) return;
    const double off = is_b ? 0.5 : 0.0;
    const double x0 = (j_new + off) * q.dx, x1 = ((j_new + 1.0) + off) * q.dx;
    if (j_new == j && n_new == n + 1) {  // same nodes, the window moves up one level
#pragma unroll
      for (int l = 0; l < P; ++l) {
        v0[l] = v0[l + 1];
        v1[l] = v1[l + 1];
      }
      const double t = ((double)n_new + off) * q.dt;
      v0[P] = field_of(q, t - x0);
      v1[P] = field_of(q, t - x1);
    } else {
#pragma unroll
      for (int l = 0; l <= P; ++l) {
        const double t = ((double)(n_new - P + l) + off) * q.dt;
        v0[l] = field_of(q, t - x0);
        v1[l] = field_of(q, t - x1);
      }
    }
    j = j_new;
    n = n_new;
  }
};

// Temporal sums at the two tent nodes (ascending level), then the tent weight.
template <int P>
__device__ __forceinline__ double gather(GridCache<P>& c, const pic_study_case& q, bool is_b,
                                         int64_t n, const double* w, double u) {
  const double fl = floor(u);
  const double frac = u - fl;
  c.ensure(q, is_b, fl, n);
  double f0 = w[0] * c.v0[0];
  double f1 = w[0] * c.v1[0];
#pragma unroll
  for (int l = 1; l <= P; ++l) {
    f0 = f0 + w[l] * c.v0[l];
    f1 = f1 + w[l] * c.v1[l];
  }
  return f0 + frac * (f1 - f0);
}

__device__ __forceinline__ void atomic_max_pos(unsigned long long* a, double v) {
  atomicMax(a, (unsigned long long)__double_as_longlong(v));  // v >= 0
}

template <int P>
__device__ void study_electron(const pic_study_case& q, double x0, double* out_eps_r,
                               double* out_eps_e, double* out_gmax, int64_t* n_star,
                               int64_t* substeps, int64_t* k_hist) {
  const double dt = q.dt, inv_dx = 1.0 / q.dx;
  double wB_half[P + 1], wE[P + 1], wB[P + 1], inv_den[P + 1];
  lagrange_inv_den(P, inv_den);
  lagrange(P, false, 0.5, inv_den, wB_half);
  GridCache<P> cE, cB;
  double pv0 = 0.0, pv1 = 0.0, pv2 = 0.0;
  double xi = x0;
  int k_prev = 0;
  double eps_r = 0.0, eps_e = 0.0, gmax = 1.0;
  int64_t ns = 0, sub = 0;
  for (int64_t n = 0; n < q.n_steps; ++n) {
    double s = xi * inv_dx;
    const double b0 = gather<P>(cB, q, true, n, wB_half, s - 0.5);
    const double g0 = sqrt(1.0 + (pv0 * pv0 + pv1 * pv1 + pv2 * pv2));
    double psi = (fabs(q.qm) * fabs(b0) * dt) / (2.0 * g0);
    int k = 0;
    while (psi > q.psi_max && k < q.k_max) {
      psi = psi * 0.25;
      ++k;
    }
    const int64_t m = (int64_t)1 << (2 * k);
    const double h = ldexp(dt, -2 * k);
    const double h_old = ldexp(dt, -2 * k_prev);
    const double inv_m = ldexp(1.0, -2 * k);
    k_hist[k] += 1;
    sub += m;
    if (k > 0) ns += m;
    double g = g0;
    for (int64_t j = 1; j <= m; ++j) {
      const double theta = (q.field_time == 0) ? 0.5 + (double)(j - 1) * inv_m
                                                : ((double)(j - 1) + 0.5) * inv_m;
      lagrange(P, true, theta, inv_den, wE);
      lagrange(P, false, theta, inv_den, wB);
      s = xi * inv_dx;
      const double ey = gather<P>(cE, q, false, n, wE, s);
      const double bz = gather<P>(cB, q, true, n, wB, s - 0.5);
      const double hp = (j == 1) ? 0.5 * (h_old + h) : h;
      // Boris, E = (0, ey, 0), B = (0, 0, bz)
      const double half = 0.5 * hp;
      const double dpy = (q.qm * ey) * half;
      const double mx = pv0, my = pv1 + dpy, mz = pv2;
      const double gn = sqrt(1.0 + (mx * mx + my * my + mz * mz));
      const double tz = ((q.qm * bz) * half) / gn;
      const double ppx = mx + my * tz;
      const double ppy = my - mx * tz;
      const double sz = (2.0 * tz) / (1.0 + tz * tz);
      const double qx = mx + ppy * sz;
      const double qy = my - ppx * sz;
      pv0 = qx;
      pv1 = qy + dpy;
      pv2 = mz;
      g = sqrt(1.0 + (pv0 * pv0 + pv1 * pv1 + pv2 * pv2));
      xi = xi + h * (pv0 / g);
    }
    k_prev = k;
    const double R = g - pv0;
    const double dR = fabs(R - 1.0);
    if (dR > eps_r) eps_r = dR;
    const double t_p = (double)(n + 1) * dt - 0.5 * h;
    const double x_p = xi - 0.5 * h * (pv0 / g);
    const double a = a_of(q, t_p - x_p);
    const double g_th = 1.0 + 0.5 * a * a;
    const double de = fabs(g - g_th) / g_th;
    if (de > eps_e) eps_e = de;
    if (g > gmax) gmax = g;
  }
  *out_eps_r = eps_r;
  *out_eps_e = eps_e;
  *out_gmax = gmax;
  *n_star = ns;
  *substeps = sub;
}

struct StudyAcc {
  unsigned long long eps_r, eps_e, gmax;  // doubles >= 0 as bits
  unsigned long long n_star_sum, substeps_sum;
  unsigned long long k_hist[8];
};

// One warp per CTA: block b runs electrons 32 (b % per_case) .. + 31 of case
// b / per_case, so a case of 64 electrons spreads over two SMs (the FP64 pipe
// of one SM is the bound: ~2 DFMA per clock); every order in one launch, so
// the cases of all orders run at once.
__global__ void __launch_bounds__(32) study_kernel(const pic_study_case* cases, pic_study_result* out,
                                                   StudyAcc* acc, int per_case) {
  const int c = blockIdx.x / per_case;
  const pic_study_case q = cases[c];
  const int e = (blockIdx.x % per_case) * 32 + (int)threadIdx.x;
  if (e >= q.n_electrons) return;
  const double x0 = (2.0 * M_PI) * (double)e / (double)q.n_electrons;
  double er, ee, gm;
  int64_t ns, sub;
  int64_t kh[8] = {0, 0, 0, 0, 0, 0, 0, 0};
  switch (q.order) {
    case 1: study_electron<1>(q, x0, &er, &ee, &gm, &ns, &sub, kh); break;
    case 2: study_electron<2>(q, x0, &er, &ee, &gm, &ns, &sub, kh); break;
    case 3: study_electron<3>(q, x0, &er, &ee, &gm, &ns, &sub, kh); break;
    case 4: study_electron<4>(q, x0, &er, &ee, &gm, &ns, &sub, kh); break;
    default: study_electron<5>(q, x0, &er, &ee, &gm, &ns, &sub, kh); break;
  }
  StudyAcc& A = acc[c];
  atomic_max_pos(&A.eps_r, er);
  atomic_max_pos(&A.eps_e, ee);
  atomic_max_pos(&A.gmax, gm);
  atomicAdd(&A.n_star_sum, (unsigned long long)ns);
  atomicAdd(&A.substeps_sum, (unsigned long long)sub);
  for (int k = 0; k < 8; ++k)
    if (kh[k]) atomicAdd(&A.k_hist[k], (unsigned long long)kh[k]);
  if (e == 0) {
    pic_study_result& r = out[c];
    r.eps_dephasing_first = er;
    r.eps_energy_first = ee;
    r.gamma_max_first = gm;
    r.n_star_first = ns;
  }
}

}  // namespace
}  // namespace pic

using namespace pic;

extern "C" int pic_study_run(const pic_study_case* cases, int32_t n_cases, pic_study_result* out,
                             void* stream) {
  if (!cases || !out || n_cases < 1 || n_cases > 65535) {
    set_global_error("pic_study_run: bad arguments");
    return PIC_EINVAL;
  }
  for (int32_t i = 0; i < n_cases; ++i) {
    const pic_study_case& q = cases[i];
    if (!(q.dt > 0) || !(q.dx > 0) || !(q.psi_max > 0) || !(q.sigma > 0) || q.order < 1 ||
        q.order > kMaxOrder || q.k_max < 0 || q.k_max > kMaxK || q.n_electrons < 1 ||
        q.n_electrons > 256 || q.n_steps < 0 || (q.field_time != 0 && q.field_time != 1)) {
      set_global_error("pic_study_run: case parameter out of range");
      return PIC_EINVAL;
    }
  }
  cudaStream_t st = (cudaStream_t)stream;
  pic_study_case* dcases = nullptr;
  pic_study_result* dout = nullptr;
  StudyAcc* dacc = nullptr;
  auto cleanup = [&]() {
    cudaFree(dcases);
    cudaFree(dout);
    cudaFree(dacc);
  };
  cudaError_t e = cudaMalloc(&dcases, sizeof(pic_study_case) * n_cases);
  if (e == cudaSuccess) e = cudaMalloc(&dout, sizeof(pic_study_result) * n_cases);
  if (e == cudaSuccess) e = cudaMalloc(&dacc, sizeof(StudyAcc) * n_cases);
  if (e != cudaSuccess) {
    cleanup();
    set_global_error("pic_study_run: device allocation failed");
    return PIC_ENOMEM;
  }
  e = cudaMemcpyAsync(dcases, cases, sizeof(pic_study_case) * n_cases, cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) e = cudaMemsetAsync(dacc, 0, sizeof(StudyAcc) * n_cases, st);
  if (e == cudaSuccess) e = cudaMemsetAsync(dout, 0, sizeof(pic_study_result) * n_cases, st);
  int per_case = 1;
  for (int32_t i = 0; i < n_cases; ++i) {
    const int w = (cases[i].n_electrons + 31) / 32;
    per_case = w > per_case ? w : per_case;
  }
  if (e == cudaSuccess) {
    study_kernel<<<(unsigned)(n_cases * per_case), 32, 0, st>>>(dcases, dout, dacc, per_case);
    e = cudaGetLastError();
  }
  std::vector<StudyAcc> acc(n_cases);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(out, dout, sizeof(pic_study_result) * n_cases, cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(acc.data(), dacc, sizeof(StudyAcc) * n_cases, cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  cleanup();
  if (e != cudaSuccess) {
    set_global_error(cudaGetErrorString(e));
    return PIC_ECUDA;
  }
  for (int32_t i = 0; i < n_cases; ++i) {
    pic_study_result& r = out[i];
    memcpy(&r.eps_dephasing, &acc[i].eps_r, 8);
    memcpy(&r.eps_energy, &acc[i].eps_e, 8);
    memcpy(&r.gamma_max, &acc[i].gmax, 8);
    r.n_steps = cases[i].n_steps;
    r.n_star_mean = (double)acc[i].n_star_sum / (double)cases[i].n_electrons;
    r.substeps = (int64_t)acc[i].substeps_sum;
    for (int k = 0; k < 8; ++k) r.k_hist[k] = (int64_t)acc[i].k_hist[k];
  }
  return PIC_OK;
}
