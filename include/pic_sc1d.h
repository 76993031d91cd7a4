/*
 * pic_sc1d.h -- C ABI of the self-consistent 1D3V particle-in-cell loop built
 * around the adaptive electron sub-cycling integrator (arXiv 2102.10983).
 *
 * One macro step dt of the loop (the "standard PIC" of Sec. III with the
 * integrator of Secs. IV and VI):
 *   1. push: every electron takes Algorithm 1 of Sec. IV (criterion
 *      |Psi| <= Psi_max, m = 4^k Boris sub-steps, transitional first step),
 *      the Boris push of Eqs. eq:p - eq:x with E = (E_x, E_y, 0) and
 *      B = (0, 0, B_z), each field interpolated in time with the order-p
 *      Lagrange weights of Sec. VI over the stored levels and in space with
 *      the tent shape (Eqs. eq:Enp, eq:Bnp);
 *   2. deposit (not in the paper; this library's definition): the charge-
 *      conserving longitudinal current from each electron's start and end
 *      positions, and the transverse current averaged over its sub-steps
 *      (each sub-step weighted h/dt), both summed in exact fixed point
 *      (units of 2^-44 n_c e), so that the sums do not depend on order;
 *   3. fields: the Yee scheme of Eqs. eq:Ey, eq:Bz with the current J_y,
 *      dE_x/dt = -J_x, first-order Mur boundaries for E_y at both ends.
 * Gauss's law div E_x = rho (immobile ions neutralizing the initial
 * electrons) is checked on the device on request; the check keeps running
 * maxima on the device, so it adds no synchronization.
 *
 * Units and grid: omega = c = m = |e| = 1, densities in n_c.  N cells; E_y on
 * nodes k dx (time levels n dt), E_x on faces (k + 1/2) dx (levels n dt), B_z
 * on faces (levels (n + 1/2) dt).  Every field array has N + 5 FP64 entries,
 * index = node or face + 2 (two padding entries on each side).  Electrons are
 * pushed while s = x/dx lies in [1/2, N - 1/2); one that leaves it is frozen
 * where it stands (status bit 7) and keeps its charge.
 *
 * Conventions as in pic_gb300.h: int status (PIC_OK or PIC_E*), borrowed
 * pointers in PIC_HOST or PIC_DEVICE memory, all work queued on the context's
 * stream, calls with host destinations or stats synchronize.
 */
#ifndef PIC_SC1D_H
#define PIC_SC1D_H

#include <stdint.h>

#include "pic_gb300.h"

#ifdef __cplusplus
extern "C" {
#endif

typedef struct {
  double dt;          /* macro step, > 0                                       */
  double dx;          /* cell size, > 0 (c dt / dx < 1 for the Yee scheme)      */
  double psi_max;     /* Psi_max of the criterion (Sec. IV), > 0                */
  double qm;          /* electron charge / mass, -1                              */
  int32_t order;      /* Lagrange order p, 1..5 (Sec. VI)                        */
  int32_t k_max;      /* cap on k, 0..7                                          */
  int32_t field_time; /* 0: sub-step fields at the position time t_n + (j-1)h;
                         1: the middle of the j-th sub-interval                  */
  int32_t n_cells;    /* N, 16 .. 2^26                                           */
  int32_t gauss_every; /* pic_sc1d_step checks Gauss's law after every macro
                          step s with s + 1 a multiple of this (0: never)         */
  int32_t reserved[3];
} pic_sc1d_params;

typedef struct {
  int64_t k_hist[8];       /* macro steps taken with each k                       */
  int64_t substeps;        /* Boris sub-steps (sum of m)                           */
  int64_t n_star;          /* sub-steps of macro steps with k > 0 (Sec. VII)       */
  int64_t clamped;         /* macro steps whose k was capped at k_max              */
  int64_t frozen;          /* electrons frozen (left the interior)                 */
  double gauss_residual;   /* max over the checks of max_k |div E_x - rho|_k        */
  double rho_max;          /* max over the checks of max_k |rho_e|_k                */
  int32_t checks;          /* Gauss checks made                                     */
  int32_t reserved;
} pic_sc1d_stats;

typedef struct pic_sc1d pic_sc1d;

/* Create a loop for up to `capacity` electrons.  Errors: PIC_EINVAL,
 * PIC_ENOMEM, PIC_ECUDA. */
int pic_sc1d_create(const pic_sc1d_params* prm, int64_t capacity, void* stream, pic_sc1d** out);
int pic_sc1d_destroy(pic_sc1d* c);

/* Load n electrons: position x, momentum (px, py, pz) at t - dt/2 (status
 * k_prev = 0), density weight w (units of n_c; charge rint(w 2^44) fixed-point
 * units).  The ion background is set to minus the electrons' charge at these
 * positions (a neutral start).  FP64 arrays of n entries in `where` memory.
 * Errors: PIC_EINVAL, PIC_ECUDA. */
int pic_sc1d_particles_write(pic_sc1d* c, const double* x, const double* px, const double* py,
                             const double* pz, const double* w, int64_t n, int32_t where);

/* Copy the first n electrons out (any pointer may be NULL).  status: k of the
 * last step | bit 7 frozen.  Errors: PIC_EINVAL, PIC_ECUDA. */
int pic_sc1d_particles_read(pic_sc1d* c, double* x, double* px, double* py, double* pz,
                            uint8_t* status, int64_t n, int32_t where);

/* Store field level `level`: E_x and E_y at t = level dt and B_z at
 * t = (level + 1/2) dt, N + 5 FP64 each.  Before the first step n0 the levels
 * n0 - p .. n0 must be stored (the history the interpolation needs); later
 * levels are made by pic_sc1d_step.  Errors: PIC_EINVAL, PIC_ECUDA. */
int pic_sc1d_fields_write(pic_sc1d* c, int64_t level, const double* Ex, const double* Ey,
                          const double* Bz, int32_t where);

/* Read level `level` (one of the newest p + 1).  Errors: PIC_EINVAL, PIC_ECUDA. */
int pic_sc1d_fields_read(pic_sc1d* c, int64_t level, double* Ex, double* Ey, double* Bz,
                         int32_t where);

/* Macro steps n0 .. n0 + n_steps - 1 (push, deposit, field solve; Gauss check
 * after the steps s with s + 1 a multiple of gauss_every).  Level n0 must be the newest
 * stored.  With stats: synchronizes, returns and resets the counters and the
 * Gauss maxima accumulated since the last stats (PIC_EKMAX if k was capped).
 * Errors: PIC_EINVAL, PIC_ECUDA, PIC_EKMAX. */
int pic_sc1d_step(pic_sc1d* c, int64_t n0, int64_t n_steps, pic_sc1d_stats* stats);

/* CUDA-event time of the steps since the last call (ms) and their count;
 * turns timing on at the first call.  Synchronizes. */
int pic_sc1d_timing(pic_sc1d* c, double* total_ms, int64_t* steps);

/* Kernel launches queued so far. */
int64_t pic_sc1d_launch_count(const pic_sc1d* c);

const char* pic_sc1d_last_error(const pic_sc1d* c);

#ifdef __cplusplus
}
#endif
#endif /* PIC_SC1D_H */
