// Internal declarations shared by the translation units of libpic_gb300.so.
// Nothing here is part of the public ABI (include/pic_gb300.h is).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "pic_gb300.h"

namespace pic {

constexpr int kMaxOrder = 5;
constexpr int kMaxK = 7;
// Binned schedule: smallest k whose sub-cycle is deferred to the next launch's
// first work items (shorter ones are compacted inside the warp); also the
// smallest predicted k the predicted schedule bins before a launch.
#ifndef PIC_DEFER_MIN
#define PIC_DEFER_MIN 3
#endif
constexpr int kDeferMin = PIC_DEFER_MIN;
// Predicted schedule: smallest predicted k that puts a particle in the
// predicted queue.  The long sub-cycles only: binning the short ones too (1)
// took them out of the stream's stashes but measured slower, the network
// over-predicting k = 2 and a predicted item costing more than a stream slot.
#ifndef PIC_PRED_MIN_K
#define PIC_PRED_MIN_K 3
#endif
constexpr int kPredMinK = PIC_PRED_MIN_K;

// Device counters of one context (accumulated by every push launch).
struct DevStats {
  unsigned long long k_hist[8];
  unsigned long long substeps;
  unsigned long long n_star;
  unsigned long long clamped;
  unsigned long long lost;
  int error;
  int pad;
};

// Row of the weight table for sub-step j (1-based) of a macro step with
// exponent k: rows are grouped by k, 4^k rows per k.
__host__ __device__ inline int64_t wrow(int k, int64_t j) {
  return (((int64_t)1 << (2 * k)) - 1) / 3 + (j - 1);
}
inline int64_t wrows_total(int k_max) { return wrow(k_max + 1, 1) + 1; }  // + criterion row

// Arguments of the FP64 push (one macro step).
struct PushArgsF64 {
  int64_t n;
  double* x;
  double* px;
  double* py;
  double* pz;
  uint8_t* status;
  const double* E[kMaxOrder + 1];  // ring slot of level n-p+l, l = 0..p
  const double* B[kMaxOrder + 1];
  double lo, hi;  // s = x/dx must satisfy lo <= s < hi (and s - 1/2 too)
  int64_t mask;   // W - 1
  double dt, inv_dx, psi_max, qm, qm_abs;
  int k_max;
  const double* wtab;  // rows of [E weights p+1 | B weights p+1]
  int64_t crit_row;
  DevStats* stats;
  double* work;  // nullptr, or per particle the accumulated work of E (App. B)
};

// Arguments of the mixed-precision push.  Position = (cell + frac) * dx with
// an exact int32 cell and an FP32 offset.
struct PushArgsMixed {
  int64_t n;
  int32_t* cell;
  float* frac;
  float* px;
  float* py;
  float* pz;
  uint8_t* status;
  // fields, ring form (ringE != nullptr): a mirrored ring of 2R slots of lstride
  // floats, every level stored in slot (level mod R) and in that slot + R, so a
  // step's p+1 levels are consecutive from slot start_cur (previous step:
  // start_prev).  Pointer form (ringE == nullptr): one pointer per level.
  const float* ringE;
  const float* ringB;
  int64_t lstride;
  int64_t start_cur, start_prev;
  const float* E[kMaxOrder + 1];   // this step's levels n-p .. n
  const float* B[kMaxOrder + 1];
  const float* Ep[kMaxOrder + 1];  // previous step's levels (binned: deferred work)
  const float* Bp[kMaxOrder + 1];
  // E_y and B_z of every window node interpolated to t_n (theta = 1/2), written
  // by the step's half-step kernel, W + 1 nodes each (node W repeats node 0);
  // nullptr = not provided (gather the levels)
  const float* halfE;
  const float* halfB;
  // per window node, the monomial coefficients of the temporal interpolant of
  // E_y (p+1) then B_z (p+1) for this step (coef) and the previous one
  // (coef_p); nullptr = form them from the levels
  const float* coef;
  const float* coef_p;
  int32_t lo, hi;      // tent node j must satisfy lo <= j and j+1 <= hi
  int32_t lo_p, hi_p;  // same for the previous step
  int32_t mask;
  float dt, psi_max, qm, qm_abs;
  float inv_dx;
  int k_max;
  int field_time;  // 0: theta_j = 1/2 + (j-1)/m; 1: theta_j = (j - 1/2)/m
  // monomial coefficients, in u = theta - 1, of the Lagrange basis polynomials:
  // L^E_{p,l}(theta) = sum_q mono[0][l][q] u^q, L^B likewise with mono[1]
  float mono[2][kMaxOrder + 1][kMaxOrder + 1];
  const float* wtab;
  int64_t crit_row;
  DevStats* stats;
  // binned schedule: per-k queues (k = 1..7, qcap entries each), double-buffered
  const int32_t* queue_in;
  int32_t* queue_out;
  int32_t* qcount_in;   // [8], consumed by this launch, zeroed by its last block
  int32_t* qcount_out;  // [8], filled by this launch
  int64_t qcap;
  int* cursor;            // work cursor of the launch
  unsigned* blocks_done;  // blocks finished
  int parity_cur, parity_next;
  int finalize;
  int tma;  // 1: the six particle arrays are 16-byte aligned (stream tiles by bulk copy)
  // resumable long sub-cycles (ring form; lag_step == nullptr: every deferred
  // step is finished by the next launch).  A deferred particle is in macro
  // step step0 + lag_step[i] with lag_j[i] of its sub-steps done; a deferred
  // item spends at most heavy_budget sub-steps of long (k >= kDeferMin)
  // sub-cycles per launch and catches a lagging particle up with the stream.
  int32_t* lag_step;
  uint16_t* lag_j;
  int64_t step0;          // base of lag_step: the first step of the call (of the
                          // first call of a run of carried calls)
  int64_t step_cur;       // this launch's stream step (closing launch: last step + 1)
  int64_t keep_step;      // a particle may be left out of budget only in a step
                          // >= keep_step (INT64_MIN: any); below it the budget
                          // does not apply
  int32_t heavy_budget;   // <= 0: no limit
  int32_t ring_R;         // ring slots (levels at slot level mod R, mirrored at + R)
  const int64_t* slot_i0; // device copy of each slot's window origin
  // predicted schedule: electrons binned by predicted k at the last refresh of
  // the predictions (per-k queues, qcap entries each), marked in their status
  // byte; every launch until the next refresh pushes those still marked
  const int32_t* pred_queue;
  int32_t* pred_count;  // [8], set by the refresh's binning pass
};

// Fills PushArgsMixed::mono for order p (host side, FP64 expansion).
void lagrange_monomials(int p, float (&mono)[2][kMaxOrder + 1][kMaxOrder + 1]);

// Sets the reason pic_last_error(NULL) reports.
void set_global_error(const char* msg);

// One ensemble of a batch, as the batched kernel reads it.
struct EnsDev {
  float dt, psi_max, qm, qm_abs, inv_dx;
  int32_t k_max, field_time, pad;
  const float* ringE;  // mirrored ring of this ensemble (2R slots x W)
  const float* ringB;
  const int64_t* slot_i0;  // [R] window origin of each ring slot
  int64_t first, count;    // particle range in the concatenated store
  int64_t chunk_first;     // index of its first stream chunk
};

// Arguments of one batched macro step.
struct BatchArgs {
  int32_t n_ens;
  const EnsDev* ens;
  int64_t n_total, n_chunks;
  int32_t chunk;  // particles per stream chunk (multiple of 32)
  int32_t* cell;
  float* frac;
  float* px;
  float* py;
  float* pz;
  uint8_t* status;
  int64_t R, lstride;  // ring slots, W
  int32_t mask;
  int64_t start_cur, start_prev;
  const float* wtab;
  int64_t crit_row;
  float mono[2][kMaxOrder + 1][kMaxOrder + 1];
  DevStats* stats;
  const int32_t* queue_in;  // ensemble e, k: entries from 7*first_e + (k-1)*count_e
  int32_t* queue_out;
  int32_t* qcount_in;   // [n_ens][8]
  int32_t* qcount_out;
  const int64_t* prefix;  // [7*n_ens + 1] heavy-item prefix (filled per launch)
  float* half;            // [2][n_ens][W]: E_y, B_z of every node at t_n (filled per launch)
  // [n_ens][W][2(p+1)]: every node's monomial coefficients of the temporal
  // interpolant (E_y then B_z) of this step (coef, filled per launch) and of
  // the previous one (coef_p); two such tables, by step parity
  float* coef;
  const float* coef_p;
  int* cursor;
  unsigned* blocks_done;
  int parity_cur, parity_next, finalize;
  // resumable long sub-cycles, as in PushArgsMixed: a deferred particle is in
  // step step0 + lag_step[i] with lag_j[i] of its sub-steps done; a deferred
  // item spends at most heavy_budget sub-steps of long sub-cycles per launch
  int32_t* lag_step;
  uint16_t* lag_j;
  int64_t step0, step_cur;
  int32_t heavy_budget;  // <= 0: no limit
};

cudaError_t launch_batch_step(const BatchArgs& a, int order, int blocks, cudaStream_t s,
                              int* launches);
int batch_max_blocks_per_sm(int order);
cudaError_t launch_batch_scatter(const EnsDev* ens, int32_t n_ens, int64_t slot, int64_t R,
                                 int64_t W, const double* Ey, const double* Bz, const int64_t* i0,
                                 int64_t* slot_i0_all, cudaStream_t s);
cudaError_t launch_to_mixed(const double* x, const double* px, const double* py, const double* pz,
                            int32_t* cell, float* frac, float* fpx, float* fpy, float* fpz,
                            double inv_dx, int64_t n, cudaStream_t s);
cudaError_t launch_from_mixed(const int32_t* cell, const float* frac, const float* fpx,
                              const float* fpy, const float* fpz, double* x, double* px, double* py,
                              double* pz, double dx, int64_t n, cudaStream_t s);

// Launchers (return cudaError_t of the launch).
cudaError_t build_wtab_f64(double* wtab, int order, int k_max, int field_time, cudaStream_t s);
cudaError_t build_wtab_f32(float* wtab, const double* wtab64, int64_t count, cudaStream_t s);
cudaError_t launch_push_f64(const PushArgsF64& a, int order, cudaStream_t s, int* launches);
cudaError_t launch_push_mixed(const PushArgsMixed& a, int order, int schedule, int sm_count,
                              cudaStream_t s, int* launches);
// One binned step (one launch); with a.finalize set, the closing launch of a
// call (the last step's deferred particles, then public status bytes).
cudaError_t launch_binned_step(const PushArgsMixed& a, int order, int sm_count, cudaStream_t main,
                               int* launches);
// E_y, B_z of every window node at t_n (the theta = 1/2 weights of a's step),
// and (coef != nullptr) every node's monomial coefficients, 2(p+1) floats.
cudaError_t launch_halfstep(const PushArgsMixed& a, int order, int64_t W, float* outE, float* outB,
                            float* coef, cudaStream_t s);
// E_y, B_z of every window node extrapolated to t_{n+1} (theta = 3/2) from step
// a's levels, W + 1 nodes each: the predictor's field features.
cudaError_t launch_feature_nodes(const PushArgsMixed& a, int order, int64_t W, float* outE,
                                 float* outB, cudaStream_t s);
// Features of every particle (a.halfE / a.halfB: the feature nodes of a's step).
cudaError_t launch_features_mixed(const PushArgsMixed& a, int order, float* phi, cudaStream_t s);

// Rebuilds the predicted queue: clears the old queue's marks, then bins and
// marks the particles whose predicted k is >= min_k (and that the stream would
// take this step) into per-k queues; pred_count must be zero on entry.
cudaError_t launch_bin_predicted(const uint8_t* pred, uint8_t* status, int64_t n, int parity_cur,
                                 int min_k, int32_t* pred_queue, int32_t* pred_count, int64_t qcap,
                                 cudaStream_t s);

// predictor (mlp_bf16.cu, mlp_api.cu)
const float* mlp_device_params(const struct ::pic_mlp* m);
int mlp_param_count();
cudaError_t launch_mlp_infer(const float* P, const float* phi, int64_t n, uint8_t* pred,
                             int sm_count, cudaStream_t s);
// Features of step a's levels (theta = 3/2; a.halfE / a.halfB: the feature
// nodes) and the predicted class of every particle in one pass (the same
// predictions as features + launch_mlp_infer).  fieldless_zero: a particle
// that sees no field (E_y = B_z = 0 at its position) gets class 0 without the
// network, and a tile of such particles skips the network.
cudaError_t launch_predict_fused(const PushArgsMixed& a, int order, const float* P, uint8_t* pred,
                                 int sm_count, cudaStream_t s, bool fieldless_zero = false);
cudaError_t launch_mlp_grad(const float* P, const float* phi, const uint8_t* label, int64_t n,
                            float* grad, float* loss, int sm_count, cudaStream_t s);
cudaError_t launch_mlp_adam(float* P, const float* grad, float* m1, float* m2, float lr, int step,
                            cudaStream_t s);

}  // namespace pic
