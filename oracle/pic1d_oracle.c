/*
 * Oracle of the self-consistent 1D3V particle-in-cell step: the Yee field
 * solver of Sec. III (Eqs. eq:Ey, eq:Bz) with the plasma current and the
 * longitudinal field added, the adaptive sub-cycling electron push of Sec. IV
 * (Algorithm 1) with the order-p temporal interpolation of Sec. VI, and a
 * charge-conserving current deposit.
 *
 * TEST INFRASTRUCTURE ONLY.  Only tests, the smoke check and the CPU baseline
 * leg of the benchmark may load this library.  It shares no code with the
 * CUDA path.  Build with -ffp-contract=off.
 *
 * Units: omega = c = m = |e| = 1, densities in units of the critical density
 * n_c, so that dE/dt = curl B - J and div E = rho.  Electrons (q/m = qm, -1)
 * move; ions are an immobile background.
 *
 * Grid (N cells, the paper's staggering shifted by half a cell):
 *   nodes k dx:       E_y (level n at t = n dt), J_y (t = (n+1/2) dt), rho;
 *   faces (k+1/2) dx: E_x (t = n dt), B_z (t = (n+1/2) dt), J_x (t = (n+1/2) dt).
 * Arrays cover nodes k = -2 .. N+2 (index k + 2, length N + 5) and faces
 * k + 1/2, k = -2 .. N+2 (index k + 2, length N + 5), so that a particle frozen
 * one sub-step outside the interior can still be deposited.
 *
 * Interior of the push: s = x/dx in [1/2, N - 1/2), where both tent nodes of
 * the node grid lie in [0, N] and both of the face grid in [0, N-1] (faces
 * 1/2 .. N-1/2).  A particle whose s leaves it at the start of a sub-step is
 * frozen where it stands (status bit 7) and keeps its charge there.
 *
 * Field solve of one macro step n -> n+1 (r = dt/dx):
 *   E_y^{n+1}_k = E_y^n_k - r (B_z^{n+1/2}_{k+1/2} - B_z^{n+1/2}_{k-1/2}) - dt J_y_k,  k = 1..N-1
 *   E_y^{n+1}_0 = E_y^n_1 + kappa (E_y^{n+1}_1 - E_y^n_0),     kappa = (r - 1)/(r + 1)
 *   E_y^{n+1}_N = E_y^n_{N-1} + kappa (E_y^{n+1}_{N-1} - E_y^n_N)   (first-order Mur)
 *   E_x^{n+1}_{k+1/2} = E_x^n_{k+1/2} - dt J_x_{k+1/2},       every face
 *   B_z^{n+3/2}_{k+1/2} = B_z^{n+1/2}_{k+1/2} - r (E_y^{n+1}_{k+1} - E_y^{n+1}_k),  k = 0..N-1
 * Other entries of E_y and B_z stay zero.
 *
 * Deposit (fixed point, so that every summation is exact and any order of
 * accumulation gives the same bits).  A particle of density weight w carries
 * Q = rint(w 2^44) charge units (electron charge -Q).  At s = x/dx, i =
 * floor(s), f = s - i, its node charges are R_{i+1} = rint(Q f), R_i = Q -
 * R_{i+1} (their sum is exactly Q).
 *   J_x: for the move s_a -> s_b of one macro step (the start and the end or
 *        frozen position), dC_k = -(R_k(s_b) - R_k(s_a)), and the charge flux
 *        through face k+1/2 is F_{k+1/2} = -sum_{j <= k} dC_j (integer).
 *        Then dt J_x = F 2^-44 dx, so rho^{n+1} - rho^n = -(F_{k+1/2} -
 *        F_{k-1/2}) 2^-44 exactly: discrete charge conservation.
 *   J_y: time average over the macro step.  Sub-step j (step h = dt/4^k)
 *        contributes (h/dt) v_y^{(j)} S_k(s_mid) to node k, s_mid the middle
 *        of the sub-step's displacement, v_y = p_y/gamma after its Boris push,
 *        S the tent; the contributions of the macro step are summed per node
 *        in FP64 in sub-step order (a_k), and the node gets -rint(a_k Q)
 *        units (J_y = sum 2^-44).
 * Gauss's law: rho_k = (C^e_k + C^ion_k) 2^-44 with C^ion = -C^e at t = 0
 * (a neutral start, E_x = 0); residual g_k = (E_x_{k+1/2} - E_x_{k-1/2})/dx - rho_k.
 */
#include <math.h>
#include <stdint.h>
#include <string.h>

#define P1_MAX_ORDER 7
#define P1_SHIFT 44

typedef struct {
  double dt, dx, psi_max, qm;
  int32_t order, k_max, field_time, n_cells;
} p1_params;

typedef struct {
  int64_t k_hist[16];
  int64_t substeps, n_star, clamped, frozen;
} p1_stats;

/* Lagrange weights of Sec. VI (same definition as orc_lagrange). */
static void p1_lagrange(int p, int is_e, double theta, double* w) {
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

/* Boris push with E = (ex, ey, 0), B = (0, 0, bz) (Eqs. eq:p - eq:gamman). */
void p1_boris(double* p, double ex, double ey, double bz, double hp, double qm) {
  double half = 0.5 * hp;
  double dpx = (qm * ex) * half;
  double dpy = (qm * ey) * half;
  double mx = p[0] + dpx, my = p[1] + dpy, mz = p[2];
  double gn = sqrt(1.0 + (mx * mx + my * my + mz * mz));
  double tz = ((qm * bz) * half) / gn;
  double ppx = mx + my * tz;
  double ppy = my - mx * tz;
  double sz = (2.0 * tz) / (1.0 + tz * tz);
  double qx = mx + ppy * sz;
  double qy = my - ppx * sz;
  p[0] = qx + dpx;
  p[1] = qy + dpy;
  p[2] = mz;
}

/* Field of one grid at coordinate u (node units of that grid: u = s for the
 * node grid, s - 1/2 for the face grid), order-p weights w over the p+1
 * levels (ascending time), level l at lv[l] (array index = node + 2). */
static double p1_gather(const double* const* lv, int p, const double* w, double u) {
  double fl = floor(u);
  int64_t j = (int64_t)fl + 2;
  double frac = u - fl;
  double f0 = w[0] * lv[0][j], f1 = w[0] * lv[0][j + 1];
  for (int l = 1; l <= p; ++l) {
    f0 = f0 + w[l] * lv[l][j];
    f1 = f1 + w[l] * lv[l][j + 1];
  }
  return f0 + frac * (f1 - f0);
}

static int p1_inside(double s, int32_t n_cells) { return s >= 0.5 && s < (double)n_cells - 0.5; }

/* Node charges of Q at s: R[0] at node floor(s), R[1] at node floor(s)+1. */
static void p1_split(int64_t Q, double s, int64_t* i, int64_t* R) {
  double fl = floor(s);
  *i = (int64_t)fl;
  R[1] = (int64_t)rint((double)Q * (s - fl));
  R[0] = Q - R[1];
}

int64_t p1_charge_units(double w) { return (int64_t)rint(w * 0x1p44); }

/*
 * Push and deposit of macro step n for n particles.
 *   Ex[l], Ey[l]: E levels n-p+l (l = 0..p), Bz[l]: B levels n+1/2-p+l;
 *   each an array of N + 5 values (index = node or face + 2).
 *   F (faces) and D (nodes): int64 accumulators, N + 5 entries, added to.
 */
void p1_push_deposit(const p1_params* prm, int64_t n, double* x, double* px, double* py,
                     double* pz, uint8_t* status, const int64_t* Q,
                     const double* const* Ex, const double* const* Ey, const double* const* Bz,
                     int64_t* F, int64_t* D, p1_stats* st) {
  const int p = prm->order;
  const double dt = prm->dt;
  const double inv_dx = 1.0 / prm->dx;
  double wB_half[P1_MAX_ORDER + 1], wE[P1_MAX_ORDER + 1], wB[P1_MAX_ORDER + 1];
  p1_lagrange(p, 0, 0.5, wB_half);
  for (int64_t i = 0; i < n; ++i) {
    if (status[i] & 0x80) continue;
    const int k_prev = status[i] & 0x7f;
    double pv[3] = {px[i], py[i], pz[i]};
    double xi = x[i];
    const double s_a = xi * inv_dx;
    if (!p1_inside(s_a, prm->n_cells)) {
      status[i] = (uint8_t)(status[i] | 0x80);
      st->frozen += 1;
      continue;
    }
    /* criterion (Sec. IV): |B_z| at x_n, t_n; gamma of the stored momentum */
    double b0 = p1_gather(Bz, p, wB_half, s_a - 0.5);
    double g0 = sqrt(1.0 + (pv[0] * pv[0] + pv[1] * pv[1] + pv[2] * pv[2]));
    double psi = (fabs(prm->qm) * fabs(b0) * dt) / (2.0 * g0);
    int k = 0;
    while (psi > prm->psi_max && k < prm->k_max) { psi = psi * 0.25; ++k; }
    if (psi > prm->psi_max) st->clamped += 1;
    const int64_t m = (int64_t)1 << (2 * k);
    const double h = ldexp(dt, -2 * k);
    const double h_old = ldexp(dt, -2 * k_prev);
    const double inv_m = ldexp(1.0, -2 * k);
    st->k_hist[k] += 1;
    st->substeps += m;
    if (k > 0) st->n_star += m;
    /* J_y sums of this macro step: nodes floor(s_a) - 2 .. floor(s_a) + 2 */
    const int64_t base = (int64_t)floor(s_a) - 2;
    double a[5] = {0.0, 0.0, 0.0, 0.0, 0.0};
    int frozen = 0;
    for (int64_t j = 1; j <= m; ++j) {
      double theta = (prm->field_time == 0) ? 0.5 + (double)(j - 1) * inv_m
                                            : ((double)(j - 1) + 0.5) * inv_m;
      p1_lagrange(p, 1, theta, wE);
      p1_lagrange(p, 0, theta, wB);
      double s = xi * inv_dx;
      if (!p1_inside(s, prm->n_cells)) { frozen = 1; break; }
      double ex = p1_gather(Ex, p, wE, s - 0.5);
      double ey = p1_gather(Ey, p, wE, s);
      double bz = p1_gather(Bz, p, wB, s - 0.5);
      double hp = (j == 1) ? 0.5 * (h_old + h) : h;
      p1_boris(pv, ex, ey, bz, hp, prm->qm);
      double g = sqrt(1.0 + (pv[0] * pv[0] + pv[1] * pv[1] + pv[2] * pv[2]));
      double vx = pv[0] / g, vy = pv[1] / g;
      double s_mid = (xi + 0.5 * (h * vx)) * inv_dx;
      xi = xi + h * vx;
      double fl = floor(s_mid);
      int64_t c = (int64_t)fl - base;
      double cw = vy * inv_m;          /* (h/dt) v_y */
      double t = cw * (s_mid - fl);
      a[c] = a[c] + (cw - t);
      a[c + 1] = a[c + 1] + t;
    }
    x[i] = xi; px[i] = pv[0]; py[i] = pv[1]; pz[i] = pv[2];
    if (frozen) { status[i] = (uint8_t)(k | 0x80); st->frozen += 1; }
    else status[i] = (uint8_t)k;
    /* J_y: one rounding per node */
    for (int c = 0; c < 5; ++c)
      if (a[c] != 0.0) D[base + c + 2] += -(int64_t)rint(a[c] * (double)Q[i]);
    /* J_x: charge flux of the move s_a -> s_b */
    const double s_b = xi * inv_dx;
    int64_t ia, ib, Ra[2], Rb[2];
    p1_split(Q[i], s_a, &ia, Ra);
    p1_split(Q[i], s_b, &ib, Rb);
    int64_t dC[6] = {0, 0, 0, 0, 0, 0};  /* nodes lo .. lo+5 */
    const int64_t lo = (ia < ib ? ia : ib) - 1;
    dC[ia - lo] -= -Ra[0]; dC[ia + 1 - lo] -= -Ra[1];   /* electron charge -R, removed at s_a */
    dC[ib - lo] += -Rb[0]; dC[ib + 1 - lo] += -Rb[1];   /* and added at s_b */
    int64_t flux = 0;
    for (int c = 0; c < 6; ++c) {
      flux -= dC[c];
      if (flux != 0) F[lo + c + 2] += flux;             /* face (lo + c) + 1/2 */
    }
  }
}

/* The field solve of one macro step.  In: E levels n (Ex0, Ey0), B level
 * n+1/2 (Bz0), the accumulators F, D of step n.  Out: Ex1, Ey1 (level n+1),
 * Bz1 (level n+3/2).  Arrays of N + 5 entries. */
void p1_field_step(const p1_params* prm, const double* Ex0, const double* Ey0, const double* Bz0,
                   const int64_t* F, const int64_t* D, double* Ex1, double* Ey1, double* Bz1) {
  const int64_t N = prm->n_cells;
  const double dt = prm->dt, dx = prm->dx;
  const double r = dt / dx;
  const double kappa = (r - 1.0) / (r + 1.0);
  for (int64_t q = 0; q < N + 5; ++q) { Ex1[q] = 0.0; Ey1[q] = 0.0; Bz1[q] = 0.0; }
  for (int64_t k = 1; k <= N - 1; ++k) {
    const int64_t q = k + 2;
    Ey1[q] = (Ey0[q] - r * (Bz0[q] - Bz0[q - 1])) - dt * ((double)D[q] * 0x1p-44);
  }
  Ey1[2] = Ey0[3] + kappa * (Ey1[3] - Ey0[2]);
  Ey1[N + 2] = Ey0[N + 1] + kappa * (Ey1[N + 1] - Ey0[N + 2]);
  for (int64_t q = 0; q < N + 5; ++q) Ex1[q] = Ex0[q] - ((double)F[q] * 0x1p-44) * dx;
  for (int64_t k = 0; k <= N - 1; ++k) {
    const int64_t q = k + 2;
    Bz1[q] = Bz0[q] - r * (Ey1[q + 1] - Ey1[q]);
  }
}

/* Electron node charges C^e (units 2^-44) of n particles, added to C. */
void p1_rho(const p1_params* prm, int64_t n, const double* x, const int64_t* Q, int64_t* C) {
  const double inv_dx = 1.0 / prm->dx;
  for (int64_t i = 0; i < n; ++i) {
    int64_t ii, R[2];
    p1_split(Q[i], x[i] * inv_dx, &ii, R);
    C[ii + 2] += -R[0];
    C[ii + 3] += -R[1];
  }
}

/* Gauss's law residual max_k |(E_x_{k+1/2} - E_x_{k-1/2})/dx - rho_k| over
 * nodes k = -1 .. N+1, rho = (C + C_ion) 2^-44; also max |rho^e| in *rho_max. */
double p1_gauss(const p1_params* prm, const double* Ex, const int64_t* C, const int64_t* C_ion,
                double* rho_max) {
  const int64_t N = prm->n_cells;
  const double inv_dx = 1.0 / prm->dx;
  double worst = 0.0, rmax = 0.0;
  for (int64_t k = -1; k <= N + 1; ++k) {
    const int64_t q = k + 2;
    double rho = (double)(C[q] + C_ion[q]) * 0x1p-44;
    double g = (Ex[q] - Ex[q - 1]) * inv_dx - rho;
    if (fabs(g) > worst) worst = fabs(g);
    double re = fabs((double)C[q] * 0x1p-44);
    if (re > rmax) rmax = re;
  }
  if (rho_max) *rho_max = rmax;
  return worst;
}
