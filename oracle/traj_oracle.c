/*
 * Oracle of the single-electron studies of Secs. IV-VII: one electron from
 * rest through the Gaussian-enveloped plane wave of Eqs. laser5 - laser3
 * (a = a0 exp(-(xi - xi0)^2 / (2 sigma^2)) sin xi, E_y = B_z = -da/dxi), with
 * the field sampled on the grid ("perfectly propagating PIC", Sec. III): E_y
 * at nodes i dx and times n dt, B_z at (i + 1/2) dx and (n + 1/2) dt, each
 * value computed from the formula when the gather needs it.  The push is the
 * method of orc_push_step (Algorithm 1, order-p Lagrange in time, tent in
 * space, Boris), written out again here for on-demand fields.
 *
 * TEST INFRASTRUCTURE ONLY.  Shares no code with the CUDA path.  Build with
 * -ffp-contract=off.
 *
 * Reported per run (Sec. IV, Eqs. R error and gamma error; Sec. VII):
 *   eps_dephasing = max over macro steps of |R - 1|, R = gamma - p_x;
 *   eps_energy    = max over macro steps of |gamma - gamma_th| / gamma_th with
 *                   gamma_th = 1 + a(xi_p)^2 / 2 at the momentum's phase
 *                   xi_p = t_p - x_p, t_p = t_{n+1} - h/2, x_p = x - (h/2) v_x;
 *   gamma_max, N (macro steps), N* (sub-steps of macro steps with k > 0), the
 *   k histogram, and the final position and momentum.
 */
#include <math.h>
#include <stdint.h>
#include <string.h>

typedef struct {
  double a0, xi0, sigma;
  double dt, dx, psi_max, qm;
  int32_t order, k_max, field_time, pad;
  int64_t n_steps;
  double x0;
  double field_scale; /* multiplies every field sample (1: the pulse as given;
                         tests move it by a few ulps to measure sensitivity) */
} trj_params;

typedef struct {
  double eps_dephasing, eps_energy, gamma_max;
  int64_t n_steps, n_star, substeps;
  int64_t k_hist[8];
  double x, px, py, pz; /* the state after the last macro step */
} trj_result;

static double trj_a(const trj_params* q, double xi) {
  const double d = xi - q->xi0;
  return q->a0 * exp(-(d * d) / (2.0 * q->sigma * q->sigma)) * sin(xi);
}

/* E_y = B_z = -da/dxi (Eq. laser5) */
static double trj_field(const trj_params* q, double xi) {
  const double d = xi - q->xi0;
  const double env = exp(-(d * d) / (2.0 * q->sigma * q->sigma));
  return -(q->a0 * env * (cos(xi) - (d / (q->sigma * q->sigma)) * sin(xi))) * q->field_scale;
}

static void trj_lagrange(int p, int is_e, double theta, double* w) {
  const double c_off = is_e ? -0.5 : -1.0;
  for (int j = 0; j <= p; ++j) {
    double num = 1.0;
    int first = 1;
    long den = 1;
    for (int k = 0; k <= p; ++k) {
      if (k == j) continue;
      double factor = ((double)(p - k) + c_off) + theta;
      if (first) { num = factor; first = 0; } else { num = num * factor; }
      den *= (long)(j - k);
    }
    w[j] = num * (1.0 / (double)den);
  }
}

/* Field of grid g (0: E_y on nodes at level times n - p + l; 1: B_z on
 * half nodes at n + 1/2 - p + l) at coordinate u (node units of the grid),
 * weights w over the p + 1 levels ascending: temporal sums at the two tent
 * nodes, then the tent weight (Eqs. eq:Enp, eq:Bnp). */
static double trj_gather(const trj_params* q, int g, int64_t n, const double* w, double u) {
  const int p = q->order;
  const double fl = floor(u);
  const double j = fl;
  const double frac = u - fl;
  double f0 = 0.0, f1 = 0.0;
  for (int l = 0; l <= p; ++l) {
    const double t = ((double)(n - p + l) + (g ? 0.5 : 0.0)) * q->dt;
    const double x0 = (j + (g ? 0.5 : 0.0)) * q->dx;
    const double x1 = ((j + 1.0) + (g ? 0.5 : 0.0)) * q->dx;
    const double v0 = trj_field(q, t - x0), v1 = trj_field(q, t - x1);
    if (l == 0) { f0 = w[0] * v0; f1 = w[0] * v1; }
    else { f0 = f0 + w[l] * v0; f1 = f1 + w[l] * v1; }
  }
  return f0 + frac * (f1 - f0);
}

static void trj_boris(double* p, double ey, double bz, double hp, double qm) {
  double half = 0.5 * hp;
  double dpy = (qm * ey) * half;
  double mx = p[0], my = p[1] + dpy, mz = p[2];
  double gn = sqrt(1.0 + (mx * mx + my * my + mz * mz));
  double tz = ((qm * bz) * half) / gn;
  double ppx = mx + my * tz;
  double ppy = my - mx * tz;
  double sz = (2.0 * tz) / (1.0 + tz * tz);
  double qx = mx + ppy * sz;
  double qy = my - ppx * sz;
  p[0] = qx;
  p[1] = qy + dpy;
  p[2] = mz;
}

void trj_run(const trj_params* q, trj_result* r) {
  const int p = q->order;
  const double dt = q->dt, inv_dx = 1.0 / q->dx;
  double wB_half[8], wE[8], wB[8];
  trj_lagrange(p, 0, 0.5, wB_half);
  memset(r, 0, sizeof(*r));
  double pv[3] = {0.0, 0.0, 0.0};
  double xi = q->x0;
  int k_prev = 0;
  r->gamma_max = 1.0;
  for (int64_t n = 0; n < q->n_steps; ++n) {
    double s = xi * inv_dx;
    double b0 = trj_gather(q, 1, n, wB_half, s - 0.5);
    double g0 = sqrt(1.0 + (pv[0] * pv[0] + pv[1] * pv[1] + pv[2] * pv[2]));
    double psi = (fabs(q->qm) * fabs(b0) * dt) / (2.0 * g0);
    int k = 0;
    while (psi > q->psi_max && k < q->k_max) { psi = psi * 0.25; ++k; }
    const int64_t m = (int64_t)1 << (2 * k);
    const double h = ldexp(dt, -2 * k);
    const double h_old = ldexp(dt, -2 * k_prev);
    const double inv_m = ldexp(1.0, -2 * k);
    r->k_hist[k] += 1;
    r->substeps += m;
    if (k > 0) r->n_star += m;
    double g = g0;
    for (int64_t j = 1; j <= m; ++j) {
      double theta = (q->field_time == 0) ? 0.5 + (double)(j - 1) * inv_m
                                          : ((double)(j - 1) + 0.5) * inv_m;
      trj_lagrange(p, 1, theta, wE);
      trj_lagrange(p, 0, theta, wB);
      s = xi * inv_dx;
      double ey = trj_gather(q, 0, n, wE, s);
      double bz = trj_gather(q, 1, n, wB, s - 0.5);
      double hp = (j == 1) ? 0.5 * (h_old + h) : h;
      trj_boris(pv, ey, bz, hp, q->qm);
      g = sqrt(1.0 + (pv[0] * pv[0] + pv[1] * pv[1] + pv[2] * pv[2]));
      xi = xi + h * (pv[0] / g);
    }
    k_prev = k;
    /* diagnostics after the macro step */
    const double R = g - pv[0];
    const double dR = fabs(R - 1.0);
    if (dR > r->eps_dephasing) r->eps_dephasing = dR;
    const double t_p = (double)(n + 1) * dt - 0.5 * h;
    const double x_p = xi - 0.5 * h * (pv[0] / g);
    const double a = trj_a(q, t_p - x_p);
    const double g_th = 1.0 + 0.5 * a * a;
    const double de = fabs(g - g_th) / g_th;
    if (de > r->eps_energy) r->eps_energy = de;
    if (g > r->gamma_max) r->gamma_max = g;
  }
  r->n_steps = q->n_steps;
  r->x = xi;
  r->px = pv[0];
  r->py = pv[1];
  r->pz = pv[2];
}
