/*
 * Oracle: plain, serial, FP64 CPU implementation of the adaptive electron
 * sub-cycling particle integrator of Tangtartharakul, Chen and Arefiev,
 * "Particle integrator for particle-in-cell simulations of ultra-high
 * intensity laser-plasma interactions" (arXiv 2102.10983).
 *
 * TEST INFRASTRUCTURE ONLY.  Only tests, the smoke check and the CPU baseline
 * leg of the benchmark may load this library.  It shares no code with the
 * CUDA path.  Build with -ffp-contract=off so that no multiply-add is fused.
 *
 * Normalized units: omega = c = m = |e| = 1.  Time in 1/omega, length in c/omega,
 * momentum in m c, fields in m omega c / |e|.  1D3V with E = (0, E_y, 0) and
 * B = (0, 0, B_z), the only components of the model problem (Sec. III).
 *
 * Grid (Sec. III, Eqs. eq:Ey/eq:Bz, relabelled by half a cell): E_y at nodes
 * x = i dx and integer times n dt; B_z at nodes x = (i + 1/2) dx and half-integer
 * times (n + 1/2) dt.  A field "level" is one time level sampled on W
 * consecutive nodes starting at global node index i0.
 *
 * Particle state: x at t_n, momentum at t_n - h_old/2, and a status byte whose
 * low 7 bits hold k_prev (the previous macro step's exponent, h_old = dt/4^k_prev)
 * and whose bit 7 marks a particle that left the field window (frozen).
 *
 * Readings of the paper taken here (each listed with its reason in the design
 * notes of the repository):
 *  - Algorithm 1: the loop count is dt/dt*_new = 4^k (the printed ratio
 *    dt*_old/dt*_new is read as a slip); the loop accepts |Psi| <= Psi_max; Psi is
 *    first evaluated with dt.
 *  - The criterion uses |B| interpolated (order p) to the particle at t_n and
 *    gamma of the stored momentum.
 *  - Sub-step field time: position time t_n + (j-1) h  (theta = 1/2 + (j-1)/m),
 *    or, as a switch, the middle of the j-th sub-interval of [t_n - dt/2, t_n + dt/2]
 *    (theta = (j - 1/2)/m).
 *  - k is capped at k_max (default 7); a capped step is counted.
 */
#include <math.h>
#include <stdint.h>
#include <string.h>

#define ORC_MAX_ORDER 7

typedef struct {
  double dt;        /* macro time step                                     */
  double dx;        /* cell size                                           */
  double psi_max;   /* rotation-angle threshold, Sec. IV                   */
  double qm;        /* charge / mass; -1 for the electron                  */
  int32_t order;    /* Lagrange order p of the temporal interpolation      */
  int32_t k_max;    /* cap on the sub-cycling exponent                     */
  int32_t field_time; /* 0: position time (default), 1: sub-interval middle */
  int32_t pad;
} orc_params;

typedef struct {
  int64_t k_hist[16];     /* macro steps taken with each k                   */
  int64_t substeps;       /* sum over particles of m = 4^k                   */
  int64_t n_star;         /* sum of m over macro steps with k > 0 (Sec. VII) */
  int64_t clamped;        /* macro steps whose k was capped at k_max         */
  int64_t out_of_window;  /* particles frozen this step (left the window)    */
} orc_stats;

/*
 * Lagrange weights of Eqs. eq:lagrange2-2 (B) and eq:lagrange2-3 (E), Sec. VI:
 *   L_j(theta) = prod_{k != j} (c_k + theta) / (j - k),  j = 0..p,
 * with c_k = p - k - 1 for B and c_k = p - k - 1/2 for E, theta = dt'/dt.
 * Evaluation order: the numerator product over ascending k, times the
 * correctly rounded reciprocal of the integer denominator.
 */
void orc_lagrange(int32_t p, int32_t is_e, double theta, double* w) {
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

/* One Boris push (Sec. III, Eqs. eq:p - eq:gamman) with step hp, in the 1D3V
 * field geometry E = (0, ey, 0), B = (0, 0, bz).  p[3] is updated in place. */
void orc_boris(double* p, double ey, double bz, double hp, double qm) {
  double half = 0.5 * hp;
  double dpy = (qm * ey) * half;                 /* q E hp / 2, y only      */
  double mx = p[0], my = p[1] + dpy, mz = p[2];  /* p^-                     */
  double gn = sqrt(1.0 + (mx * mx + my * my + mz * mz));
  double tz = ((qm * bz) * half) / gn;           /* Psi_z                   */
  double ppx = mx + my * tz;                     /* p' = p^- + p^- x Psi    */
  double ppy = my - mx * tz;
  double sz = (2.0 * tz) / (1.0 + tz * tz);      /* s = 2 Psi / (1 + Psi^2) */
  double qx = mx + ppy * sz;                     /* p^+ = p^- + p' x s      */
  double qy = my - ppx * sz;
  p[0] = qx;
  p[1] = qy + dpy;                               /* p_{n+1/2}               */
  p[2] = mz;
}

/* Field of one grid (E or B) at global coordinate s (in node units), from the
 * p+1 levels, with temporal weights w: temporal sum at the two tent nodes in
 * ascending level order, then the tent (linear) weight in space, Eqs. eq:Enp
 * and eq:Bnp.  Returns 0 if a node lies outside any level's window. */
static int orc_gather(const double* levels, const int64_t* i0, int64_t W, int32_t p,
                      const double* w, double s, double* out) {
  double fl = floor(s);
  int64_t j = (int64_t)fl;
  double frac = s - fl;
  double f0 = 0.0, f1 = 0.0;
  for (int l = 0; l <= p; ++l) {
    int64_t a = j - i0[l];
    if (a < 0 || a + 1 >= W) return 0;
    const double* lev = levels + (int64_t)l * W;
    if (l == 0) { f0 = w[0] * lev[a]; f1 = w[0] * lev[a + 1]; }
    else { f0 = f0 + w[l] * lev[a]; f1 = f1 + w[l] * lev[a + 1]; }
  }
  *out = f0 + frac * (f1 - f0);
  return 1;
}

/* Is s = x/dx a coordinate whose two tent nodes exist in every level?  Done on
 * the double before any conversion so that a NaN or huge x is caught. */
static int orc_in_window(double s, const int64_t* i0, int64_t W, int32_t p) {
  double lo = -1e300, hi = 1e300;
  for (int l = 0; l <= p; ++l) {
    double a = (double)i0[l], b = (double)(i0[l] + W - 1);
    if (a > lo) lo = a;
    if (b < hi) hi = b;
  }
  return (s >= lo) && (s < hi);
}

/*
 * One macro step dt of Algorithm 1 (Sec. IV) for the n particles, with the order-p
 * temporal interpolation of Sec. VI.
 *   E_lv: (p+1) x W, E levels n-p .. n (ascending), origins E_i0[p+1]
 *   B_lv: (p+1) x W, B levels n+1/2-p .. n+1/2,       origins B_i0[p+1]
 *   work: NULL, or per particle the work of the electric field accumulated
 *         over every Boris push (App. B, Eq. eq:work_nosub, taken per sub-step):
 *         w = (q hp / 2) E' . (v_before + v_after), v = p / gamma of the
 *         momentum before and after the push, hp its step.
 * Returns the number of particles that left the window during this step.
 */
int64_t orc_push_step(const orc_params* prm, int64_t n,
                      double* x, double* px, double* py, double* pz, uint8_t* status,
                      const double* E_lv, const int64_t* E_i0,
                      const double* B_lv, const int64_t* B_i0, int64_t W,
                      orc_stats* st, double* work) {
  const int32_t p = prm->order;
  const double dt = prm->dt;
  const double inv_dx = 1.0 / prm->dx;
  double wB_half[ORC_MAX_ORDER + 1];
  double wE[ORC_MAX_ORDER + 1], wB[ORC_MAX_ORDER + 1];
  orc_lagrange(p, 0, 0.5, wB_half);
  int64_t lost = 0;

  for (int64_t i = 0; i < n; ++i) {
    if (status[i] & 0x80) continue;
    int k_prev = status[i] & 0x7f;
    double pv[3] = {px[i], py[i], pz[i]};
    double xi = x[i];

    /* Criterion (Sec. IV): Psi with dt, B at t_n and x_n, gamma of stored p. */
    double s = xi * inv_dx;
    double sb = s - 0.5;
    if (!orc_in_window(s, E_i0, W, p) || !orc_in_window(sb, B_i0, W, p)) {
      status[i] = (uint8_t)(status[i] | 0x80);
      ++lost;
      continue;
    }
    double b0;
    orc_gather(B_lv, B_i0, W, p, wB_half, sb, &b0);
    double g0 = sqrt(1.0 + (pv[0] * pv[0] + pv[1] * pv[1] + pv[2] * pv[2]));
    double psi = (fabs(prm->qm) * fabs(b0) * dt) / (2.0 * g0);
    int k = 0;
    while (psi > prm->psi_max && k < prm->k_max) { psi = psi * 0.25; ++k; }
    if (psi > prm->psi_max) st->clamped += 1;
    int64_t m = (int64_t)1 << (2 * k);
    double h = ldexp(dt, -2 * k);
    double h_old = ldexp(dt, -2 * k_prev);
    double inv_m = ldexp(1.0, -2 * k);
    st->k_hist[k] += 1;
    st->substeps += m;
    if (k > 0) st->n_star += m;

    int frozen = 0;
    for (int64_t j = 1; j <= m; ++j) {
      double theta = (prm->field_time == 0) ? 0.5 + (double)(j - 1) * inv_m
                                            : ((double)(j - 1) + 0.5) * inv_m;
      orc_lagrange(p, 1, theta, wE);
      orc_lagrange(p, 0, theta, wB);
      s = xi * inv_dx;
      sb = s - 0.5;
      if (!orc_in_window(s, E_i0, W, p) || !orc_in_window(sb, B_i0, W, p)) { frozen = 1; break; }
      double ey, bz;
      orc_gather(E_lv, E_i0, W, p, wE, s, &ey);
      orc_gather(B_lv, B_i0, W, p, wB, sb, &bz);
      double hp = (j == 1) ? 0.5 * (h_old + h) : h;
      double vy_before = 0.0;
      if (work) {
        double gb = sqrt(1.0 + (pv[0] * pv[0] + pv[1] * pv[1] + pv[2] * pv[2]));
        vy_before = pv[1] / gb;
      }
      orc_boris(pv, ey, bz, hp, prm->qm);
      double g = sqrt(1.0 + (pv[0] * pv[0] + pv[1] * pv[1] + pv[2] * pv[2]));
      if (work) work[i] = work[i] + ((prm->qm * hp) * 0.5) * (ey * (vy_before + pv[1] / g));
      xi = xi + h * (pv[0] / g);                     /* Eqs. eq:gamma - eq:x */
    }
    x[i] = xi; px[i] = pv[0]; py[i] = pv[1]; pz[i] = pv[2];
    if (frozen) { status[i] = (uint8_t)(k | 0x80); ++lost; }
    else status[i] = (uint8_t)k;
  }
  st->out_of_window += lost;
  return lost;
}

/*
 * n_steps consecutive macro steps.  E_all / B_all hold n_steps + p levels
 * (rows), row r being level n0 - p + r; step s reads rows s .. s+p.  The
 * dephasing diagnostic of Eq. R error (Sec. IV) is accumulated per particle:
 * r_dev[i] = max over steps of |(gamma - p_x) - r_ref[i]| evaluated on the
 * momentum after each macro step (r_ref = 1 for an electron starting at rest;
 * for another start, gamma_0 - p_x0, App. A).  r_ref / r_dev may be NULL;
 * work as for orc_push_step.
 */
int64_t orc_run(const orc_params* prm, int64_t n_steps, int64_t n,
                double* x, double* px, double* py, double* pz, uint8_t* status,
                const double* E_all, const int64_t* E_i0_all,
                const double* B_all, const int64_t* B_i0_all, int64_t W,
                const double* r_ref, double* r_dev, orc_stats* st, double* work) {
  int64_t lost = 0;
  for (int64_t s = 0; s < n_steps; ++s) {
    lost += orc_push_step(prm, n, x, px, py, pz, status, E_all + s * W, E_i0_all + s,
                          B_all + s * W, B_i0_all + s, W, st, work);
    if (r_ref && r_dev) {
      for (int64_t i = 0; i < n; ++i) {
        double g = sqrt(1.0 + (px[i] * px[i] + py[i] * py[i] + pz[i] * pz[i]));
        double d = fabs((g - px[i]) - r_ref[i]);
        if (d > r_dev[i]) r_dev[i] = d;
      }
    }
  }
  return lost;
}
