// FP64 form of the adaptive sub-cycling push (arXiv 2102.10983).
//
// This translation unit is compiled with -fmad=false: every multiply and add
// below rounds separately, in exactly the order written, so that the result
// matches a serial FP64 evaluation of the same formulas bit for bit.  sqrt and
// division are the IEEE correctly rounded double operations.
//
// One thread per particle, grid-stride.  Per macro step (Algorithm 1, Sec. IV):
//   criterion: Psi0 = |q/m| |B(x_n, t_n)| dt / (2 gamma), gamma of the stored
//              momentum, B interpolated with the order-p weights at t_n;
//              k = smallest k with Psi0/4^k <= Psi_max (capped at k_max);
//   m = 4^k sub-steps of h = dt/4^k; the first uses (h_old + h)/2 (the
//   transitional step), each: order-p Lagrange in time (Sec. VI), tent in space
//   (Eqs. eq:Enp, eq:Bnp), Boris (Eqs. eq:p - eq:gamman), x += h v_x (Eq. eq:x).
#include <math.h>

#include "pic_internal.h"

namespace pic {

// Weights of Eqs. eq:lagrange2-2 (B) and eq:lagrange2-3 (E):
//   L_j(theta) = prod_{k != j} (c_k + theta) / (j - k),
// c_k = p-k-1 (B) or p-k-1/2 (E); numerator over ascending k, times the
// correctly rounded reciprocal of the integer denominator.
__device__ void lagrange_f64(int p, bool is_e, double theta, double* w) {
  const double c_off = is_e ? -0.5 : -1.0;
  for (int j = 0; j <= p; ++j) {
    double num = 1.0;
    bool first = true;
    long long den = 1;
    for (int k = 0; k <= p; ++k) {
      if (k == j) continue;
      double factor = ((double)(p - k) + c_off) + theta;
      if (first) {
        num = factor;
        first = false;
      } else {
        num = num * factor;
      }
      den *= (long long)(j - k);
    }
    w[j] = num * (1.0 / (double)den);
  }
}

// One row per (k, j) sub-step plus a last row for the criterion (theta = 1/2).
__global__ void wtab_f64_kernel(double* wtab, int p, int k_max, int field_time, int64_t rows) {
  const int stride = 2 * (p + 1);
  for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < rows;
       r += (int64_t)gridDim.x * blockDim.x) {
    double theta;
    if (r == rows - 1) {
      theta = 0.5;
    } else {
      int k = 0;
      while (k < k_max && wrow(k + 1, 1) <= r) ++k;
      int64_t j = r - wrow(k, 1) + 1;
      double inv_m = ldexp(1.0, -2 * k);
      theta = (field_time == 0) ? 0.5 + (double)(j - 1) * inv_m : ((double)(j - 1) + 0.5) * inv_m;
    }
    lagrange_f64(p, true, theta, wtab + r * stride);
    lagrange_f64(p, false, theta, wtab + r * stride + (p + 1));
  }
}

cudaError_t build_wtab_f64(double* wtab, int order, int k_max, int field_time, cudaStream_t s) {
  int64_t rows = wrows_total(k_max);
  int blocks = (int)((rows + 255) / 256);
  wtab_f64_kernel<<<blocks, 256, 0, s>>>(wtab, order, k_max, field_time, rows);
  return cudaGetLastError();
}

// Temporal sum at the two tent nodes (ascending level), then the tent weight.
template <int P>
__device__ __forceinline__ double gather_f64(const double* const* lv, const double* w, double s,
                                             int64_t mask) {
  double fl = floor(s);
  int64_t j = (int64_t)fl;
  double frac = s - fl;
  int64_t a0 = j & mask, a1 = (j + 1) & mask;
  double f0 = w[0] * __ldg(lv[0] + a0);
  double f1 = w[0] * __ldg(lv[0] + a1);
#pragma unroll
  for (int l = 1; l <= P; ++l) {
    f0 = f0 + w[l] * __ldg(lv[l] + a0);
    f1 = f1 + w[l] * __ldg(lv[l] + a1);
  }
  return f0 + frac * (f1 - f0);
}

template <int P>
__global__ void __launch_bounds__(256) push_f64_kernel(PushArgsF64 a) {
  __shared__ unsigned long long sh[12];
  if (threadIdx.x < 12) sh[threadIdx.x] = 0ull;
  __syncthreads();
  const int stride = 2 * (P + 1);
  const double* wcrit = a.wtab + a.crit_row * stride + (P + 1);
  const double* E[P + 1];
  const double* B[P + 1];
#pragma unroll
  for (int l = 0; l <= P; ++l) {
    E[l] = a.E[l];
    B[l] = a.B[l];
  }
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < a.n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const uint8_t st = a.status[i];
    if (st & PIC_STATUS_LOST) continue;
    const int k_prev = st & 0x7f;
    double pv0 = a.px[i], pv1 = a.py[i], pv2 = a.pz[i];
    double xi = a.x[i];

    double s = xi * a.inv_dx;
    double sb = s - 0.5;
    if (!(s >= a.lo && s < a.hi) || !(sb >= a.lo && sb < a.hi)) {
      a.status[i] = (uint8_t)(st | PIC_STATUS_LOST);
      atomicAdd(&sh[11], 1ull);
      continue;
    }
    double b0 = gather_f64<P>(B, wcrit, sb, a.mask);
    double g0 = sqrt(1.0 + (pv0 * pv0 + pv1 * pv1 + pv2 * pv2));
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
    atomicAdd(&sh[k], 1ull);
    atomicAdd(&sh[8], (unsigned long long)m);
    if (k > 0) atomicAdd(&sh[9], (unsigned long long)m);
    if (capped) atomicAdd(&sh[10], 1ull);

    const double* wr = a.wtab + wrow(k, 1) * stride;
    bool frozen = false;
    double work = a.work ? a.work[i] : 0.0;
    for (int64_t j = 1; j <= m; ++j, wr += stride) {
      s = xi * a.inv_dx;
      sb = s - 0.5;
      if (!(s >= a.lo && s < a.hi) || !(sb >= a.lo && sb < a.hi)) {
        frozen = true;
        break;
      }
      const double ey = gather_f64<P>(E, wr, s, a.mask);
      const double bz = gather_f64<P>(B, wr + (P + 1), sb, a.mask);
      const double hp = (j == 1) ? 0.5 * (h_old + h) : h;
      double vy_before = 0.0;
      if (a.work) vy_before = pv1 / sqrt(1.0 + (pv0 * pv0 + pv1 * pv1 + pv2 * pv2));
      // Boris, E = (0, ey, 0), B = (0, 0, bz)
      const double half = 0.5 * hp;
      const double dpy = (a.qm * ey) * half;
      const double mx = pv0, my = pv1 + dpy, mz = pv2;
      const double gn = sqrt(1.0 + (mx * mx + my * my + mz * mz));
      const double tz = ((a.qm * bz) * half) / gn;
      const double ppx = mx + my * tz;
      const double ppy = my - mx * tz;
      const double sz = (2.0 * tz) / (1.0 + tz * tz);
      const double qx = mx + ppy * sz;
      const double qy = my - ppx * sz;
      pv0 = qx;
      pv1 = qy + dpy;
      pv2 = mz;
      const double g = sqrt(1.0 + (pv0 * pv0 + pv1 * pv1 + pv2 * pv2));
      // the work of E over this push (App. B): (q hp / 2) E . (v_before + v_after)
      if (a.work) work = work + ((a.qm * hp) * 0.5) * (ey * (vy_before + pv1 / g));
      xi = xi + h * (pv0 / g);
    }
    if (a.work) a.work[i] = work;
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
  }
  __syncthreads();
  if (threadIdx.x < 12) {
    unsigned long long v = sh[threadIdx.x];
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

cudaError_t launch_push_f64(const PushArgsF64& a, int order, cudaStream_t s, int* launches) {
  if (a.n <= 0) return cudaSuccess;
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  int64_t want = (a.n + 255) / 256;
  int64_t cap = (int64_t)sms * 8;
  int blocks = (int)(want < cap ? want : cap);
  switch (order) {
    case 1: push_f64_kernel<1><<<blocks, 256, 0, s>>>(a); break;
    case 2: push_f64_kernel<2><<<blocks, 256, 0, s>>>(a); break;
    case 3: push_f64_kernel<3><<<blocks, 256, 0, s>>>(a); break;
    case 4: push_f64_kernel<4><<<blocks, 256, 0, s>>>(a); break;
    case 5: push_f64_kernel<5><<<blocks, 256, 0, s>>>(a); break;
    default: return cudaErrorInvalidValue;
  }
  if (launches) ++*launches;
  return cudaGetLastError();
}

}  // namespace pic
