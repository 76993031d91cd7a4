// C ABI of the integrator (include/pic_gb300.h): the context, its particle
// store, its field ring and the step driver.  The arithmetic of the method
// lives in push_f64.cu and push_mixed.cu.
#include <math.h>
#include <stdio.h>
#include <string.h>

#include <new>
#include <vector>

#include "pic_internal.h"

using namespace pic;

struct pic_ctx {
  pic_params prm;
  int64_t capacity = 0;
  int64_t n = 0;  // particles loaded
  int64_t W = 0;
  int32_t R = 0;
  cudaStream_t stream = nullptr;
  int sm_count = 0;
  // FP64 particle store
  double *x = nullptr, *px = nullptr, *py = nullptr, *pz = nullptr;
  // mixed particle store
  int32_t* cell = nullptr;
  float *frac = nullptr, *fpx = nullptr, *fpy = nullptr, *fpz = nullptr;
  uint8_t* status = nullptr;
  // field ring: R slots of W values (double or float)
  void* ringE = nullptr;
  void* ringB = nullptr;
  std::vector<int64_t> slot_level, slot_i0;
  double* staging = nullptr;  // host-upload / conversion staging
  int64_t staging_len = 0;
  double* wtab64 = nullptr;
  float* wtab32 = nullptr;
  DevStats* dstats = nullptr;
  // binned schedule scratch
  int32_t* queue = nullptr;
  int32_t* qcount = nullptr;  // [0,16) deferred counts, 16 cursor, 18 blocks done, [32,40) predicted counts
  // predicted schedule
  uint8_t* pred = nullptr;
  float* half = nullptr;  // mixed form: E_y, B_z of every window node at the step's t_n
  float* coef = nullptr;  // mixed form: per node monomial coefficients, two steps (parity of s)
  float* feat = nullptr;  // mixed form: the predictor's feature nodes (E_y, B_z at t_{n+1}), W + 1 each
  // binned mixed form: resumable long sub-cycles (per particle: the step it is
  // in and the sub-steps done), and a device copy of slot_i0 for the kernel
  int32_t* lag_step = nullptr;
  uint16_t* lag_j = nullptr;
  int64_t* dslot_i0 = nullptr;
  int32_t heavy_budget = 256;
  double* work = nullptr;  // FP64 form with PIC_DIAG_WORK: per-particle work of E
  int32_t* pred_queue = nullptr;
  const pic_mlp* mlp = nullptr;
  int32_t predict_every = 1;
  // pic_params.carry: long sub-cycles left by the last call for the next one
  bool open = false;       // some may be carried (the particle store is mid-step)
  int64_t open_last = 0;   // the last step pushed
  int64_t open_step0 = 0;  // base of lag_step for the run of carried calls
  int64_t open_keep = 0;   // the oldest step a carried particle may be in
  int64_t run_j = 0;       // binned launches of the run: parities, queue buffers, refresh cadence

  int64_t launches = 0;
  // optional CUDA-event timing of push steps
  bool timing = false;
  std::vector<cudaEvent_t> ev;  // pairs (start, end)
  size_t ev_used = 0;           // pairs in use
  char err[256] = {0};
};

static thread_local char g_create_err[256];

void pic::set_global_error(const char* msg) {
  strncpy(g_create_err, msg, sizeof(g_create_err) - 1);
  g_create_err[sizeof(g_create_err) - 1] = 0;
}

static int fail(pic_ctx* c, int code, const char* fmt, const char* detail = "") {
  char* dst = c ? c->err : g_create_err;
  snprintf(dst, 256, fmt, detail);
  return code;
}

#define CUDA_TRY(ctx, call)                                                 \
  do {                                                                      \
    cudaError_t e_ = (call);                                                \
    if (e_ != cudaSuccess) return fail((ctx), PIC_ECUDA, "CUDA: %s", cudaGetErrorString(e_)); \
  } while (0)

static bool is_pow2(int64_t v) { return v > 0 && (v & (v - 1)) == 0; }

static int close_open(pic_ctx* c);

static void free_events(pic_ctx* c) {
  for (cudaEvent_t e : c->ev) cudaEventDestroy(e);
  c->ev.clear();
  c->ev_used = 0;
}

static void free_all(pic_ctx* c) {
  free_events(c);

  void* ptrs[] = {c->x, c->px, c->py, c->pz, c->cell, c->frac, c->fpx, c->fpy, c->fpz,
                  c->status, c->ringE, c->ringB, c->staging, c->wtab64, c->wtab32,
                  c->dstats, c->queue, c->qcount, c->pred, c->pred_queue, c->half,
                  c->coef, c->lag_step, c->lag_j, c->dslot_i0, c->work, c->feat};
  for (void* p : ptrs)
    if (p) cudaFree(p);
}

// ---------------------------------------------------------------- small kernels

// Write a window of W nodes starting at global node i0 into a ring slot,
// circularly: node i goes to position i & (W-1).  dslot_i0 (optional): the
// device copy of the slots' window origins, updated in stream order.
template <typename T>
__global__ void scatter_level_kernel(T* slotE, T* slotB, const double* Ey, const double* Bz,
                                     int64_t i0, int64_t W, int64_t* dslot_i0, int32_t slot) {
  if (dslot_i0 && blockIdx.x == 0 && threadIdx.x == 0) dslot_i0[slot] = i0;
  for (int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; c < W;
       c += (int64_t)gridDim.x * blockDim.x) {
    int64_t pos = (i0 + c) & (W - 1);
    slotE[pos] = (T)Ey[c];
    slotB[pos] = (T)Bz[c];
  }
}

// x -> (cell, frac) with x = (cell + frac) dx, frac in [0, 1); p rounded to FP32.
__global__ void to_mixed_kernel(const double* x, const double* px, const double* py,
                                const double* pz, int32_t* cell, float* frac, float* fpx,
                                float* fpy, float* fpz, double inv_dx, int64_t n) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    double s = x[i] * inv_dx;
    double fl = floor(s);
    double fr = s - fl;
    float f = (float)fr;
    if (f >= 1.0f) { f = 0.0f; fl += 1.0; }
    cell[i] = (int32_t)fl;
    frac[i] = f;
    fpx[i] = (float)px[i];
    fpy[i] = (float)py[i];
    fpz[i] = (float)pz[i];
  }
}

__global__ void from_mixed_kernel(const int32_t* cell, const float* frac, const float* fpx,
                                  const float* fpy, const float* fpz, double* x, double* px,
                                  double* py, double* pz, double dx, int64_t n) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    if (x) x[i] = ((double)cell[i] + (double)frac[i]) * dx;
    if (px) px[i] = (double)fpx[i];
    if (py) py[i] = (double)fpy[i];
    if (pz) pz[i] = (double)fpz[i];
  }
}

cudaError_t pic::launch_to_mixed(const double* x, const double* px, const double* py,
                                 const double* pz, int32_t* cell, float* frac, float* fpx,
                                 float* fpy, float* fpz, double inv_dx, int64_t n, cudaStream_t s) {
  const int64_t want = (n + 255) / 256;
  to_mixed_kernel<<<(int)(want < 152 * 16 ? (want > 0 ? want : 1) : 152 * 16), 256, 0, s>>>(
      x, px, py, pz, cell, frac, fpx, fpy, fpz, inv_dx, n);
  return cudaGetLastError();
}

cudaError_t pic::launch_from_mixed(const int32_t* cell, const float* frac, const float* fpx,
                                   const float* fpy, const float* fpz, double* x, double* px,
                                   double* py, double* pz, double dx, int64_t n, cudaStream_t s) {
  const int64_t want = (n + 255) / 256;
  from_mixed_kernel<<<(int)(want < 152 * 16 ? (want > 0 ? want : 1) : 152 * 16), 256, 0, s>>>(
      cell, frac, fpx, fpy, fpz, x, px, py, pz, dx, n);
  return cudaGetLastError();
}

static int grid_for(const pic_ctx* c, int64_t n) {
  int64_t b = (n + 255) / 256;
  int64_t cap = (int64_t)(c->sm_count > 0 ? c->sm_count : 152) * 16;
  if (b < 1) b = 1;
  return (int)(b < cap ? b : cap);
}

// ---------------------------------------------------------------- ABI

extern "C" int pic_create(const pic_params* prm, int64_t capacity, int64_t window_cells,
                          int32_t ring_levels, void* stream, pic_ctx** out) {
  if (!prm || !out) return fail(nullptr, PIC_EINVAL, "pic_create: NULL argument%s");
  *out = nullptr;
  if (!(prm->dt > 0) || !(prm->dx > 0) || !(prm->psi_max > 0) || !isfinite(prm->qm) ||
      prm->qm == 0.0)
    return fail(nullptr, PIC_EINVAL, "pic_create: dt, dx, psi_max must be > 0 and qm != 0%s");
  if (prm->order < 1 || prm->order > kMaxOrder)
    return fail(nullptr, PIC_EINVAL, "pic_create: order must be 1..5%s");
  if (prm->k_max < 0 || prm->k_max > kMaxK)
    return fail(nullptr, PIC_EINVAL, "pic_create: k_max must be 0..7%s");
  if (prm->precision != PIC_FP64 && prm->precision != PIC_MIXED)
    return fail(nullptr, PIC_EINVAL, "pic_create: precision must be PIC_FP64 or PIC_MIXED%s");
  if (prm->field_time != 0 && prm->field_time != 1)
    return fail(nullptr, PIC_EINVAL, "pic_create: field_time must be 0 or 1%s");
  if (prm->schedule != PIC_SCHED_PLAIN && prm->schedule != PIC_SCHED_BINNED &&
      prm->schedule != PIC_SCHED_PREDICTED)
    return fail(nullptr, PIC_EINVAL, "pic_create: unknown schedule%s");
  if (prm->precision == PIC_MIXED && !((float)prm->dt >= 0x1p-100f && (float)prm->dt < 0x1p100f))
    return fail(nullptr, PIC_EINVAL, "pic_create: the mixed form needs 2^-100 <= dt < 2^100%s");
  if (prm->schedule != PIC_SCHED_PLAIN && prm->precision != PIC_MIXED)
    return fail(nullptr, PIC_EINVAL, "pic_create: the binned schedules need PIC_MIXED%s");
  if (prm->diagnostics != 0 && (prm->diagnostics != PIC_DIAG_WORK || prm->precision != PIC_FP64))
    return fail(nullptr, PIC_EINVAL, "pic_create: PIC_DIAG_WORK is the only diagnostic (FP64 form)%s");
  if (prm->carry < 0 || prm->carry > (1 << 16) || (prm->carry > 0 && prm->schedule == PIC_SCHED_PLAIN))
    return fail(nullptr, PIC_EINVAL, "pic_create: carry must be 0, or 1..65536 with a binned schedule%s");
  if (prm->carry > 0 && (int64_t)ring_levels < (int64_t)prm->order + 1 + prm->carry)
    return fail(nullptr, PIC_EINVAL, "pic_create: carry = c needs ring_levels >= order + 1 + c%s");
  if (capacity < 0 || capacity > ((int64_t)1 << 31) - 1)
    return fail(nullptr, PIC_EINVAL, "pic_create: capacity must be 0..2^31-1%s");
  if (!is_pow2(window_cells) || window_cells < 16 || window_cells > ((int64_t)1 << 30))
    return fail(nullptr, PIC_EINVAL, "pic_create: window_cells must be a power of two >= 16%s");
  if (prm->precision == PIC_MIXED && window_cells > ((int64_t)1 << 28))
    return fail(nullptr, PIC_EINVAL, "pic_create: the mixed form takes window_cells <= 2^28%s");
  if (ring_levels < prm->order + 1 || ring_levels > (1 << 20))
    return fail(nullptr, PIC_EINVAL, "pic_create: ring_levels must be >= order + 1%s");
  if (prm->schedule != PIC_SCHED_PLAIN && ring_levels < prm->order + 2)
    return fail(nullptr, PIC_EINVAL, "pic_create: the binned schedule needs ring_levels >= order + 2%s");

  pic_ctx* c = new (std::nothrow) pic_ctx();
  if (!c) return fail(nullptr, PIC_ENOMEM, "pic_create: host allocation failed%s");
  c->prm = *prm;
  c->capacity = capacity;
  c->W = window_cells;
  c->R = ring_levels;
  c->stream = (cudaStream_t)stream;
  c->slot_level.assign(ring_levels, INT64_MIN);
  c->slot_i0.assign(ring_levels, 0);
  int dev = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&c->sm_count, cudaDevAttrMultiProcessorCount, dev);

  const bool mixed = prm->precision == PIC_MIXED;
  const size_t fsz = mixed ? sizeof(float) : sizeof(double);
  const size_t cap = (size_t)(capacity > 0 ? capacity : 1);
  cudaError_t e = cudaSuccess;
  auto A = [&](void** p, size_t bytes) {
    if (e == cudaSuccess) e = cudaMalloc(p, bytes);
  };
  if (mixed) {
    A((void**)&c->half, 2 * ((size_t)window_cells + 1) * 4);  // E_y, B_z: W + 1 nodes each
    A((void**)&c->coef, 2 * (size_t)window_cells * 2 * (prm->order + 1) * 4);
    A((void**)&c->feat, 2 * ((size_t)window_cells + 1) * 4);
    A((void**)&c->cell, cap * 4);
    A((void**)&c->frac, cap * 4);
    A((void**)&c->fpx, cap * 4);
    A((void**)&c->fpy, cap * 4);
    A((void**)&c->fpz, cap * 4);
    if (prm->schedule != PIC_SCHED_PLAIN) {
      A((void**)&c->queue, 2 * 7 * cap * 4);
      A((void**)&c->qcount, 64 * 4);
      A((void**)&c->lag_step, cap * 4);
      A((void**)&c->lag_j, cap * 2);
      A((void**)&c->dslot_i0, (size_t)c->R * 8);
      c->heavy_budget = prm->heavy_budget == 0 ? 256 : prm->heavy_budget;
    }
    if (prm->schedule == PIC_SCHED_PREDICTED) {
      A((void**)&c->pred, cap);
      A((void**)&c->pred_queue, 7 * cap * 4);
    }
  } else {
    A((void**)&c->x, cap * 8);
    A((void**)&c->px, cap * 8);
    A((void**)&c->py, cap * 8);
    A((void**)&c->pz, cap * 8);
    if (prm->diagnostics == PIC_DIAG_WORK) A((void**)&c->work, cap * 8);
  }
  A((void**)&c->status, cap);
  // the mixed form's ring is mirrored (2R slots, see PushArgsMixed)
  const size_t ring_slots = (size_t)ring_levels * (mixed ? 2 : 1);
  A(&c->ringE, ring_slots * window_cells * fsz);
  A(&c->ringB, ring_slots * window_cells * fsz);
  c->staging_len = 2 * window_cells;
  if (c->staging_len < ((int64_t)1 << 22)) c->staging_len = (int64_t)1 << 22;
  A((void**)&c->staging, (size_t)c->staging_len * 8);
  const int64_t rows = wrows_total(prm->k_max);
  const int64_t wcount = rows * 2 * (prm->order + 1);
  A((void**)&c->wtab64, (size_t)wcount * 8);
  if (mixed) A((void**)&c->wtab32, (size_t)wcount * 4);
  A((void**)&c->dstats, sizeof(DevStats));
  if (e != cudaSuccess) {
    free_all(c);
    delete c;
    cudaGetLastError();
    return fail(nullptr, e == cudaErrorMemoryAllocation ? PIC_ENOMEM : PIC_ECUDA,
                "pic_create: device allocation failed: %s", cudaGetErrorString(e));
  }
  e = cudaMemsetAsync(c->dstats, 0, sizeof(DevStats), c->stream);
  if (e == cudaSuccess && c->qcount) e = cudaMemsetAsync(c->qcount, 0, 64 * 4, c->stream);
  if (e == cudaSuccess && c->pred) e = cudaMemsetAsync(c->pred, 0, cap, c->stream);

  if (e == cudaSuccess) e = cudaMemsetAsync(c->status, 0, cap, c->stream);
  if (e == cudaSuccess) e = build_wtab_f64(c->wtab64, prm->order, prm->k_max, prm->field_time, c->stream);
  if (e == cudaSuccess) ++c->launches;
  if (e == cudaSuccess && mixed) {
    e = build_wtab_f32(c->wtab32, c->wtab64, wcount, c->stream);
    ++c->launches;
  }
  if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
  if (e != cudaSuccess) {
    free_all(c);
    delete c;
    return fail(nullptr, PIC_ECUDA, "pic_create: %s", cudaGetErrorString(e));
  }
  *out = c;
  return PIC_OK;
}

extern "C" int pic_destroy(pic_ctx* c) {
  if (!c) return PIC_OK;
  cudaStreamSynchronize(c->stream);
  free_all(c);
  delete c;
  return PIC_OK;
}

extern "C" int pic_set_stream(pic_ctx* c, void* stream) {
  if (!c) return PIC_EINVAL;
  // carried sub-cycles continue on the new stream: what the old one holds first
  if (c->open && (cudaStream_t)stream != c->stream) CUDA_TRY(c, cudaStreamSynchronize(c->stream));
  c->stream = (cudaStream_t)stream;
  return PIC_OK;
}

extern "C" int pic_timing_enable(pic_ctx* c, int32_t on) {
  if (!c) return PIC_EINVAL;
  c->timing = on != 0;
  return PIC_OK;
}

extern "C" int pic_timing_read(pic_ctx* c, double* total_ms, int64_t* steps, int32_t reset) {
  if (!c || !total_ms || !steps) return PIC_EINVAL;
  CUDA_TRY(c, cudaStreamSynchronize(c->stream));
  double tot = 0.0;
  for (size_t q = 0; q < c->ev_used; ++q) {
    float ms = 0.f;
    CUDA_TRY(c, cudaEventElapsedTime(&ms, c->ev[2 * q], c->ev[2 * q + 1]));
    tot += ms;
  }
  *total_ms = tot;
  *steps = (int64_t)c->ev_used;
  if (reset) c->ev_used = 0;
  return PIC_OK;
}

// Next (start, end) event pair of the timing pool, created on demand.
static int timing_pair(pic_ctx* c, cudaEvent_t* a, cudaEvent_t* b) {
  if (2 * (c->ev_used + 1) > c->ev.size()) {
    for (int q = 0; q < 2; ++q) {
      cudaEvent_t e;
      CUDA_TRY(c, cudaEventCreate(&e));
      c->ev.push_back(e);
    }
  }
  *a = c->ev[2 * c->ev_used];
  *b = c->ev[2 * c->ev_used + 1];
  ++c->ev_used;
  return PIC_OK;
}

extern "C" int64_t pic_launch_count(const pic_ctx* c) { return c ? c->launches : 0; }

extern "C" const char* pic_last_error(const pic_ctx* c) { return c ? c->err : g_create_err; }

static cudaMemcpyKind kind_in(int where) {
  return where == PIC_HOST ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice;
}
static cudaMemcpyKind kind_out(int where) {
  return where == PIC_HOST ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice;
}

extern "C" int pic_particles_write(pic_ctx* c, const double* x, const double* px,
                                   const double* py, const double* pz, const uint8_t* status,
                                   int64_t n, int32_t where) {
  if (!c) return PIC_EINVAL;
  if (n < 0 || n > c->capacity) return fail(c, PIC_EINVAL, "pic_particles_write: n out of range%s");
  if (where != PIC_HOST && where != PIC_DEVICE) return fail(c, PIC_EINVAL, "bad where%s");
  if (n > 0 && (!x || !px || !py || !pz)) return fail(c, PIC_EINVAL, "pic_particles_write: NULL array%s");
  if (c->open) {  // new particles replace any carried sub-cycles: drop their queues
    c->open = false;
    c->run_j = 0;
    CUDA_TRY(c, cudaMemsetAsync(c->qcount, 0, 64 * 4, c->stream));
  }
  c->n = n;
  if (n == 0) return PIC_OK;
  if (status)
    CUDA_TRY(c, cudaMemcpyAsync(c->status, status, (size_t)n, kind_in(where), c->stream));
  else
    CUDA_TRY(c, cudaMemsetAsync(c->status, 0, (size_t)n, c->stream));
  if (c->prm.precision == PIC_FP64) {
    if (c->work) CUDA_TRY(c, cudaMemsetAsync(c->work, 0, (size_t)n * 8, c->stream));
    CUDA_TRY(c, cudaMemcpyAsync(c->x, x, (size_t)n * 8, kind_in(where), c->stream));
    CUDA_TRY(c, cudaMemcpyAsync(c->px, px, (size_t)n * 8, kind_in(where), c->stream));
    CUDA_TRY(c, cudaMemcpyAsync(c->py, py, (size_t)n * 8, kind_in(where), c->stream));
    CUDA_TRY(c, cudaMemcpyAsync(c->pz, pz, (size_t)n * 8, kind_in(where), c->stream));
    return PIC_OK;
  }
  const double inv_dx = 1.0 / c->prm.dx;
  if (where == PIC_DEVICE) {
    to_mixed_kernel<<<grid_for(c, n), 256, 0, c->stream>>>(x, px, py, pz, c->cell, c->frac, c->fpx,
                                                            c->fpy, c->fpz, inv_dx, n);
    ++c->launches;
    CUDA_TRY(c, cudaGetLastError());
    return PIC_OK;
  }
  const int64_t chunk = c->staging_len / 4;
  for (int64_t off = 0; off < n; off += chunk) {
    const int64_t cnt = (n - off < chunk) ? n - off : chunk;
    double* s = c->staging;
    CUDA_TRY(c, cudaMemcpyAsync(s, x + off, cnt * 8, cudaMemcpyHostToDevice, c->stream));
    CUDA_TRY(c, cudaMemcpyAsync(s + chunk, px + off, cnt * 8, cudaMemcpyHostToDevice, c->stream));
    CUDA_TRY(c, cudaMemcpyAsync(s + 2 * chunk, py + off, cnt * 8, cudaMemcpyHostToDevice, c->stream));
    CUDA_TRY(c, cudaMemcpyAsync(s + 3 * chunk, pz + off, cnt * 8, cudaMemcpyHostToDevice, c->stream));
    to_mixed_kernel<<<grid_for(c, cnt), 256, 0, c->stream>>>(
        s, s + chunk, s + 2 * chunk, s + 3 * chunk, c->cell + off, c->frac + off, c->fpx + off,
        c->fpy + off, c->fpz + off, inv_dx, cnt);
    ++c->launches;
    CUDA_TRY(c, cudaGetLastError());
  }
  CUDA_TRY(c, cudaStreamSynchronize(c->stream));
  return PIC_OK;
}

extern "C" int pic_particles_read(pic_ctx* c, double* x, double* px, double* py, double* pz,
                                  uint8_t* status, int64_t n, int32_t where) {
  if (!c) return PIC_EINVAL;
  if (n < 0 || n > c->n) return fail(c, PIC_EINVAL, "pic_particles_read: n exceeds the loaded count%s");
  if (where != PIC_HOST && where != PIC_DEVICE) return fail(c, PIC_EINVAL, "bad where%s");
  int rc = close_open(c);  // carried sub-cycles first: the store is then whole
  if (rc != PIC_OK) return rc;
  if (n == 0) return PIC_OK;
  if (status)
    CUDA_TRY(c, cudaMemcpyAsync(status, c->status, (size_t)n, kind_out(where), c->stream));
  if (c->prm.precision == PIC_FP64) {
    double* src[4] = {c->x, c->px, c->py, c->pz};
    double* dst[4] = {x, px, py, pz};
    for (int q = 0; q < 4; ++q)
      if (dst[q])
        CUDA_TRY(c, cudaMemcpyAsync(dst[q], src[q], (size_t)n * 8, kind_out(where), c->stream));
  } else if (where == PIC_DEVICE) {
    from_mixed_kernel<<<grid_for(c, n), 256, 0, c->stream>>>(c->cell, c->frac, c->fpx, c->fpy,
                                                              c->fpz, x, px, py, pz, c->prm.dx, n);
    ++c->launches;
    CUDA_TRY(c, cudaGetLastError());
  } else {
    const int64_t chunk = c->staging_len / 4;
    double* s = c->staging;
    for (int64_t off = 0; off < n; off += chunk) {
      const int64_t cnt = (n - off < chunk) ? n - off : chunk;
      from_mixed_kernel<<<grid_for(c, cnt), 256, 0, c->stream>>>(
          c->cell + off, c->frac + off, c->fpx + off, c->fpy + off, c->fpz + off, s, s + chunk,
          s + 2 * chunk, s + 3 * chunk, c->prm.dx, cnt);
      ++c->launches;
      CUDA_TRY(c, cudaGetLastError());
      double* dst[4] = {x, px, py, pz};
      for (int q = 0; q < 4; ++q)
        if (dst[q])
          CUDA_TRY(c, cudaMemcpyAsync(dst[q] + off, s + q * chunk, cnt * 8, cudaMemcpyDeviceToHost,
                                      c->stream));
    }
  }
  if (where == PIC_HOST) CUDA_TRY(c, cudaStreamSynchronize(c->stream));
  return PIC_OK;
}

extern "C" int pic_fields_upload(pic_ctx* c, int64_t level, int64_t i0, const double* Ey,
                                 const double* Bz, int32_t where) {
  if (!c) return PIC_EINVAL;
  if (!Ey || !Bz) return fail(c, PIC_EINVAL, "pic_fields_upload: NULL field%s");
  if (where != PIC_HOST && where != PIC_DEVICE) return fail(c, PIC_EINVAL, "bad where%s");
  if (i0 < -((int64_t)1 << 40) || i0 > ((int64_t)1 << 40))
    return fail(c, PIC_EINVAL, "pic_fields_upload: window origin out of range%s");
  const int64_t W = c->W;
  const int32_t slot = (int32_t)(((level % c->R) + c->R) % c->R);
  if (c->open) {
    const int64_t old = c->slot_level[slot];
    if (old != INT64_MIN && old >= c->open_keep - c->prm.order && old <= c->open_last)
      return fail(c, PIC_EINVAL,
                  "pic_fields_upload: the slot holds a level that carried sub-cycles still need "
                  "(push the next step or call pic_finish first)%s");
  }
  const double* e = Ey;
  const double* b = Bz;
  if (where == PIC_HOST) {
    CUDA_TRY(c, cudaMemcpyAsync(c->staging, Ey, W * 8, cudaMemcpyHostToDevice, c->stream));
    CUDA_TRY(c, cudaMemcpyAsync(c->staging + W, Bz, W * 8, cudaMemcpyHostToDevice, c->stream));
    e = c->staging;
    b = c->staging + W;
  }
  const int blocks = grid_for(c, W);
  if (c->prm.precision == PIC_FP64) {
    double* sE = (double*)c->ringE + (int64_t)slot * W;
    double* sB = (double*)c->ringB + (int64_t)slot * W;
    scatter_level_kernel<double><<<blocks, 256, 0, c->stream>>>(sE, sB, e, b, i0, W, nullptr, 0);
  } else {
    for (int copy = 0; copy < 2; ++copy) {
      float* sE = (float*)c->ringE + ((int64_t)slot + (int64_t)copy * c->R) * W;
      float* sB = (float*)c->ringB + ((int64_t)slot + (int64_t)copy * c->R) * W;
      scatter_level_kernel<float><<<blocks, 256, 0, c->stream>>>(
          sE, sB, e, b, i0, W, copy == 0 ? c->dslot_i0 : nullptr, slot);
      ++c->launches;
    }
    CUDA_TRY(c, cudaGetLastError());
    c->slot_level[slot] = level;
    c->slot_i0[slot] = i0;
    return PIC_OK;
  }
  ++c->launches;
  CUDA_TRY(c, cudaGetLastError());
  c->slot_level[slot] = level;
  c->slot_i0[slot] = i0;
  return PIC_OK;
}

static int collect_stats(pic_ctx* c, pic_step_stats* out, bool reset) {
  DevStats h;
  CUDA_TRY(c, cudaMemcpyAsync(&h, c->dstats, sizeof(DevStats), cudaMemcpyDeviceToHost, c->stream));
  if (reset) CUDA_TRY(c, cudaMemsetAsync(c->dstats, 0, sizeof(DevStats), c->stream));
  CUDA_TRY(c, cudaStreamSynchronize(c->stream));
  memset(out, 0, sizeof(*out));
  for (int k = 0; k < 8; ++k) out->k_hist[k] = (int64_t)h.k_hist[k];
  out->substeps = (int64_t)h.substeps;
  out->n_star = (int64_t)h.n_star;
  out->clamped = (int64_t)h.clamped;
  out->out_of_window = (int64_t)h.lost;
  out->error = h.error;
  if (h.error) return fail(c, PIC_ETIMEOUT, "device error word set%s");
  if (out->out_of_window) return fail(c, PIC_ERANGE, "particles left the field window%s");
  if (out->clamped) return fail(c, PIC_EKMAX, "criterion capped at k_max%s");
  return PIC_OK;
}

extern "C" int pic_work_read(pic_ctx* c, double* work, int64_t n, int32_t where) {
  if (!c) return PIC_EINVAL;
  if (!c->work) return fail(c, PIC_EINVAL, "pic_work_read: create the context with PIC_DIAG_WORK%s");
  if (!work || n < 0 || n > c->n) return fail(c, PIC_EINVAL, "pic_work_read: bad buffer or count%s");
  if (where != PIC_HOST && where != PIC_DEVICE) return fail(c, PIC_EINVAL, "bad where%s");
  if (n > 0) CUDA_TRY(c, cudaMemcpyAsync(work, c->work, (size_t)n * 8, kind_out(where), c->stream));
  if (where == PIC_HOST) CUDA_TRY(c, cudaStreamSynchronize(c->stream));
  return PIC_OK;
}

extern "C" int pic_inject_error(pic_ctx* c, int32_t word) {
  if (!c) return PIC_EINVAL;
  // pageable source: the copy is staged before cudaMemcpyAsync returns
  CUDA_TRY(c, cudaMemcpyAsync(&c->dstats->error, &word, sizeof(int32_t), cudaMemcpyHostToDevice,
                              c->stream));
  return PIC_OK;
}

extern "C" int pic_stats_read(pic_ctx* c, pic_step_stats* stats, int32_t reset) {
  if (!c || !stats) return PIC_EINVAL;
  int rc = collect_stats(c, stats, reset != 0);
  return rc == PIC_ECUDA ? rc : PIC_OK;
}

// Ring slots of the levels step s needs (s-p .. s), and the intersection of
// their windows as node indices [lo, hi].
static int step_slots(pic_ctx* c, int64_t s, int* slots, int64_t* lo, int64_t* hi) {
  const int p = c->prm.order;
  *lo = INT64_MIN;
  *hi = INT64_MAX;
  for (int l = 0; l <= p; ++l) {
    const int64_t lev = s - p + l;
    const int slot = (int)(((lev % c->R) + c->R) % c->R);
    if (c->slot_level[slot] != lev)
      return fail(c, PIC_EINVAL, "pic_push_step: a field level the step needs is not in the ring%s");
    slots[l] = slot;
    const int64_t a = c->slot_i0[slot], b = c->slot_i0[slot] + c->W - 1;
    if (a > *lo) *lo = a;
    if (b < *hi) *hi = b;
  }
  return PIC_OK;
}

// Field arguments of step s (prev: as the previous step's fields) for the mixed
// form: the start slot of its p+1 consecutive levels in the mirrored ring.
static void fill_mixed(pic_ctx* c, PushArgsMixed& a, int64_t s, int64_t lo, int64_t hi, bool prev) {
  const int p = c->prm.order;
  const int64_t start = (((s - p) % c->R) + c->R) % c->R;
  a.ringE = (const float*)c->ringE;
  a.ringB = (const float*)c->ringB;
  a.lstride = c->W;
  for (int l = 0; l <= p; ++l) {  // the same levels as per-level pointers
    const float* e = (const float*)c->ringE + (start + l) * c->W;
    const float* b = (const float*)c->ringB + (start + l) * c->W;
    if (prev) {
      a.Ep[l] = e;
      a.Bp[l] = b;
    } else {
      a.E[l] = e;
      a.B[l] = b;
    }
  }
  if (prev) {
    a.start_prev = start;
    a.lo_p = (int32_t)lo;
    a.hi_p = (int32_t)hi;
  } else {
    a.start_cur = start;
    a.lo = (int32_t)lo;
    a.hi = (int32_t)hi;
  }
}

// Launch arguments of the mixed form common to every launch of a call.
static void mixed_base(pic_ctx* c, PushArgsMixed& base) {
  memset(&base, 0, sizeof(base));
  base.n = c->n;
  base.cell = c->cell; base.frac = c->frac; base.px = c->fpx; base.py = c->fpy; base.pz = c->fpz;
  base.status = c->status;
  base.tma = (((uintptr_t)c->cell | (uintptr_t)c->frac | (uintptr_t)c->fpx | (uintptr_t)c->fpy |
               (uintptr_t)c->fpz | (uintptr_t)c->status) & 15) == 0;
  base.mask = (int32_t)(c->W - 1);
  base.dt = (float)c->prm.dt;
  base.psi_max = (float)c->prm.psi_max;
  base.qm = (float)c->prm.qm;
  base.qm_abs = fabsf((float)c->prm.qm);
  base.inv_dx = (float)(1.0 / c->prm.dx);
  base.k_max = c->prm.k_max;
  base.field_time = c->prm.field_time;
  lagrange_monomials(c->prm.order, base.mono);
  base.wtab = c->wtab32;
  base.crit_row = wrows_total(c->prm.k_max) - 1;
  base.stats = c->dstats;
  base.qcap = c->capacity;
  base.keep_step = INT64_MIN;
  if (c->prm.schedule != PIC_SCHED_PLAIN) {
    base.cursor = (int*)(c->qcount + 16);
    base.blocks_done = (unsigned*)(c->qcount + 18);
    // deferred particles may run behind the stream: the kernel finds any
    // step's levels in the ring from the slots' origins
    base.lag_step = c->lag_step;
    base.lag_j = c->lag_j;
    base.heavy_budget = c->heavy_budget;
    base.ring_R = c->R;
    base.slot_i0 = c->dslot_i0;  // kept current by pic_fields_upload, in stream order
  }
}

// The closing launch after step s (a: that step's launch arguments, J its
// index in the run, coef_s its node table): every deferred particle is brought
// to the end of step s and the status bytes return to the public form.
static cudaError_t closing_launch(pic_ctx* c, const PushArgsMixed& a, int64_t s, int64_t lo,
                                  int64_t hi, int64_t J, const float* coef_s, int* launches) {
  const int64_t qsz = 7 * c->capacity;
  PushArgsMixed f = a;
  fill_mixed(c, f, s, lo, hi, true);
  f.queue_in = c->queue + ((J + 1) & 1) * qsz;
  f.qcount_in = c->qcount + ((J + 1) & 1) * 8;
  f.queue_out = c->queue + (J & 1) * qsz;
  f.qcount_out = c->qcount + (J & 1) * 8;
  f.finalize = 1;
  f.step_cur = s + 1;
  f.coef_p = coef_s;  // the deferred work finishes step s
  f.keep_step = INT64_MIN;
  f.pred_queue = nullptr;
  f.pred_count = nullptr;
  return launch_binned_step(f, c->prm.order, c->sm_count, c->stream, launches);
}

// Finish what carried calls left (pic_params.carry): the closing launch of the
// last step pushed.
static int close_open(pic_ctx* c) {
  if (!c->open) return PIC_OK;
  const int64_t S = c->open_last;
  int slots[kMaxOrder + 1];
  int64_t lo, hi;
  // the levels of the carried steps are kept by pic_fields_upload
  int rc = step_slots(c, S, slots, &lo, &hi);
  if (rc != PIC_OK) return rc;
  PushArgsMixed a;
  mixed_base(c, a);
  a.step0 = c->open_step0;
  a.step_cur = S;
  fill_mixed(c, a, S, lo, hi, false);
  const int64_t coef_stride = c->W * 2 * (c->prm.order + 1);
  const float* coef_s = c->coef + (S & 1) * coef_stride;
  a.coef = coef_s;
  a.halfE = c->half;
  a.halfB = c->half + c->W + 1;
  const int64_t J = c->run_j - 1;
  a.parity_cur = (int)(J & 1);
  a.parity_next = (int)((J + 1) & 1);
  int launches = 0;
  cudaError_t e = closing_launch(c, a, S, lo, hi, J, coef_s, &launches);
  c->launches += launches;
  c->open = false;
  c->run_j = 0;
  if (e != cudaSuccess) return fail(c, PIC_ECUDA, "closing launch: %s", cudaGetErrorString(e));
  return PIC_OK;
}

extern "C" int pic_finish(pic_ctx* c) {
  if (!c) return PIC_EINVAL;
  return close_open(c);
}

extern "C" int pic_push_step(pic_ctx* c, int64_t n, int64_t n_steps, pic_step_stats* stats) {
  if (!c) return PIC_EINVAL;
  if (n_steps < 1) return fail(c, PIC_EINVAL, "pic_push_step: n_steps must be >= 1%s");
  const int p = c->prm.order;
  const int64_t W = c->W;
  const bool binned = c->prm.schedule != PIC_SCHED_PLAIN;
  const bool predicted = c->prm.schedule == PIC_SCHED_PREDICTED && c->mlp != nullptr;
  const bool carry = binned && c->prm.carry > 0;
  // validate every step's levels before queuing anything
  for (int64_t s = n; s < n + n_steps; ++s) {
    int slots[kMaxOrder + 1];
    int64_t lo, hi;
    int rc = step_slots(c, s, slots, &lo, &hi);
    if (rc != PIC_OK) return rc;
    if (c->prm.precision == PIC_MIXED && (lo < -((int64_t)1 << 30) || hi > ((int64_t)1 << 30)))
      return fail(c, PIC_EINVAL, "pic_push_step: mixed form needs node indices within +-2^30%s");
  }
  // carried work continues only into the step after the last one pushed (and
  // while lag_step, relative to the run's first step, fits its 32 bits)
  if (c->open && (n != c->open_last + 1 || n + n_steps - c->open_step0 > ((int64_t)1 << 30))) {
    int rc = close_open(c);
    if (rc != PIC_OK) return rc;
  }
  const bool cont = c->open;  // this call's first launch takes over carried work
  const int64_t J0 = cont ? c->run_j : 0;
  PushArgsMixed base;
  if (c->prm.precision == PIC_MIXED) {
    mixed_base(c, base);
    base.step0 = cont ? c->open_step0 : n;
  } else {
    memset(&base, 0, sizeof(base));
  }
  for (int64_t j = 0; j < n_steps; ++j) {
    const int64_t s = n + j;
    const int64_t J = J0 + j;  // the launch's index in the run
    int slots[kMaxOrder + 1];
    int64_t lo, hi;
    step_slots(c, s, slots, &lo, &hi);
    if (c->n == 0) continue;
    int launches = 0;
    cudaError_t e;
    // with timing on, two events bracket the push kernel launch(es) of the step
    cudaEvent_t ev0 = nullptr, ev1 = nullptr;
    if (c->timing) {
      int rc = timing_pair(c, &ev0, &ev1);
      if (rc != PIC_OK) return rc;
    }
    auto mark = [&](cudaEvent_t ev) { return ev ? cudaEventRecord(ev, c->stream) : cudaSuccess; };
    if (c->prm.precision == PIC_FP64) {
      PushArgsF64 a;
      memset(&a, 0, sizeof(a));
      a.n = c->n;
      a.x = c->x; a.px = c->px; a.py = c->py; a.pz = c->pz; a.status = c->status;
      for (int l = 0; l <= p; ++l) {
        a.E[l] = (const double*)c->ringE + (int64_t)slots[l] * W;
        a.B[l] = (const double*)c->ringB + (int64_t)slots[l] * W;
      }
      a.lo = (double)lo;
      a.hi = (double)hi;
      a.mask = W - 1;
      a.dt = c->prm.dt;
      a.inv_dx = 1.0 / c->prm.dx;
      a.psi_max = c->prm.psi_max;
      a.qm = c->prm.qm;
      a.qm_abs = fabs(c->prm.qm);
      a.k_max = c->prm.k_max;
      a.wtab = c->wtab64;
      a.crit_row = wrows_total(c->prm.k_max) - 1;
      a.stats = c->dstats;
      a.work = c->work;
      e = mark(ev0);
      if (e == cudaSuccess) e = launch_push_f64(a, p, c->stream, &launches);
    } else {
      PushArgsMixed a = base;
      a.step_cur = s;
      fill_mixed(c, a, s, lo, hi, false);
      // this step's fields at t_n on every window node (the m = 1 pushes) and
      // its node coefficient table (the sub-cycles); the previous step's table
      // is the other half of c->coef
      const int64_t coef_stride = W * 2 * (p + 1);
      float* coef_cur = c->coef + (s & 1) * coef_stride;
      float* coef_prev = c->coef + ((s - 1) & 1) * coef_stride;
      e = launch_halfstep(a, p, W, c->half, c->half + W + 1, coef_cur, c->stream);
      ++launches;
      if (e != cudaSuccess) return fail(c, PIC_ECUDA, "half-step launch: %s", cudaGetErrorString(e));
      a.halfE = c->half;
      a.halfB = c->half + W + 1;
      a.coef = coef_cur;
      // deferred work of the previous step: from this call's last launch, or
      // carried from the last call
      const bool has_prev = j > 0 || cont;
      a.coef_p = has_prev ? coef_prev : coef_cur;
      if (binned) {
        const int64_t qsz = 7 * c->capacity;
        if (has_prev) {
          int ps[kMaxOrder + 1];
          int64_t plo, phi;
          int rc = step_slots(c, s - 1, ps, &plo, &phi);
          if (rc != PIC_OK) return rc;
          fill_mixed(c, a, s - 1, plo, phi, true);
        } else {
          fill_mixed(c, a, s, lo, hi, true);  // no deferred work on the first step
        }
        a.queue_in = c->queue + (J & 1) * qsz;
        a.queue_out = c->queue + ((J + 1) & 1) * qsz;
        a.qcount_in = c->qcount + (J & 1) * 8;
        a.qcount_out = c->qcount + ((J + 1) & 1) * 8;
        a.parity_cur = (int)(J & 1);
        a.parity_next = (int)((J + 1) & 1);
        a.finalize = 0;
        e = cudaSuccess;
        if (predicted && J % c->predict_every == 0) {
          // refresh the predictions from the state after the previous step and
          // rebuild the predicted queue, which the next predict_every steps
          // push (a run starts with a refresh: its status bytes carry no
          // queue marks)
          e = cudaMemsetAsync(c->qcount + 32, 0, 8 * sizeof(int32_t), c->stream);
          int ps[kMaxOrder + 1];
          int64_t plo, phi;
          if (e == cudaSuccess && step_slots(c, s - 1, ps, &plo, &phi) == PIC_OK) {
            PushArgsMixed fa = a;
            fill_mixed(c, fa, s - 1, plo, phi, false);
            fa.coef = fa.coef_p = nullptr;
            fa.halfE = c->feat;
            fa.halfB = c->feat + W + 1;
            e = launch_feature_nodes(fa, p, W, c->feat, c->feat + W + 1, c->stream);
            ++launches;
            if (e == cudaSuccess)
              e = launch_predict_fused(fa, p, mlp_device_params(c->mlp), c->pred, c->sm_count,
                                       c->stream, /*fieldless_zero=*/true);
            ++launches;
            if (e == cudaSuccess)
              e = launch_bin_predicted(c->pred, c->status, c->n, a.parity_cur, kPredMinK,
                                       c->pred_queue, c->qcount + 32, c->capacity, c->stream);
            ++launches;
          }
        }
        if (predicted) {
          a.pred_queue = c->pred_queue;
          a.pred_count = c->qcount + 32;
        }
        // the last launch of a carrying call leaves no particle further behind
        // than the steps whose levels the ring keeps for the next call
        if (carry && j == n_steps - 1) a.keep_step = s - (c->prm.carry - 1);
        if (e == cudaSuccess) e = mark(ev0);
        if (e == cudaSuccess)
          e = launch_binned_step(a, p, c->sm_count, c->stream, &launches);
        if (e == cudaSuccess && !carry && j == n_steps - 1)
          e = closing_launch(c, a, s, lo, hi, J, coef_cur, &launches);
      } else {
        e = mark(ev0);
        if (e == cudaSuccess)
          e = launch_push_mixed(a, p, c->prm.schedule, c->sm_count, c->stream, &launches);
      }
    }
    c->launches += launches;
    if (e != cudaSuccess) return fail(c, PIC_ECUDA, "push launch: %s", cudaGetErrorString(e));
    if (c->timing) CUDA_TRY(c, cudaEventRecord(ev1, c->stream));
  }
  if (carry && c->n > 0) {
    c->open = true;
    if (!cont) c->open_step0 = n;
    c->open_last = n + n_steps - 1;
    c->open_keep = c->open_last - (c->prm.carry - 1);
    c->run_j = J0 + n_steps;
  }
  if (stats) return collect_stats(c, stats, true);
  return PIC_OK;
}

extern "C" int pic_features(pic_ctx* c, int64_t n, float* phi) {
  if (!c || !phi) return PIC_EINVAL;
  if (c->prm.precision != PIC_MIXED) return fail(c, PIC_EINVAL, "pic_features: needs the mixed form%s");
  int rc = close_open(c);  // features of whole steps: carried sub-cycles first
  if (rc != PIC_OK) return rc;
  int slots[kMaxOrder + 1];
  int64_t lo, hi;
  rc = step_slots(c, n, slots, &lo, &hi);
  if (rc != PIC_OK) return rc;
  PushArgsMixed a;
  memset(&a, 0, sizeof(a));
  a.n = c->n;
  a.cell = c->cell; a.frac = c->frac; a.px = c->fpx; a.py = c->fpy; a.pz = c->fpz;
  a.status = c->status;
  a.mask = (int32_t)(c->W - 1);
  fill_mixed(c, a, n, lo, hi, false);
  a.halfE = c->feat;
  a.halfB = c->feat + c->W + 1;
  CUDA_TRY(c, launch_feature_nodes(a, c->prm.order, c->W, c->feat, c->feat + c->W + 1, c->stream));
  CUDA_TRY(c, launch_features_mixed(a, c->prm.order, phi, c->stream));
  c->launches += 2;
  return PIC_OK;
}

extern "C" int pic_predict(pic_ctx* c, const pic_mlp* mlp, int64_t n, uint8_t* pred) {
  if (!c || !mlp || (!pred && c->n > 0)) return PIC_EINVAL;
  if (c->prm.precision != PIC_MIXED) return fail(c, PIC_EINVAL, "pic_predict: needs the mixed form%s");
  int rc = close_open(c);  // features of whole steps: carried sub-cycles first
  if (rc != PIC_OK) return rc;
  int slots[kMaxOrder + 1];
  int64_t lo, hi;
  rc = step_slots(c, n, slots, &lo, &hi);
  if (rc != PIC_OK) return rc;
  PushArgsMixed a;
  memset(&a, 0, sizeof(a));
  a.n = c->n;
  a.cell = c->cell; a.frac = c->frac; a.px = c->fpx; a.py = c->fpy; a.pz = c->fpz;
  a.status = c->status;
  a.mask = (int32_t)(c->W - 1);
  fill_mixed(c, a, n, lo, hi, false);
  a.halfE = c->feat;
  a.halfB = c->feat + c->W + 1;
  CUDA_TRY(c, launch_feature_nodes(a, c->prm.order, c->W, c->feat, c->feat + c->W + 1, c->stream));
  CUDA_TRY(c, launch_predict_fused(a, c->prm.order, mlp_device_params(mlp), pred, c->sm_count,
                                   c->stream));
  c->launches += 2;
  return PIC_OK;
}

extern "C" int pic_attach_predictor(pic_ctx* c, pic_mlp* mlp, int32_t every) {
  if (!c) return PIC_EINVAL;
  if (c->prm.schedule != PIC_SCHED_PREDICTED)
    return fail(c, PIC_EINVAL, "pic_attach_predictor: the context's schedule is not PIC_SCHED_PREDICTED%s");
  if (every < 1) return fail(c, PIC_EINVAL, "pic_attach_predictor: every must be >= 1%s");
  // the predicted queue of a carried run belongs to the old predictor
  int rc = close_open(c);
  if (rc != PIC_OK) return rc;
  c->mlp = mlp;
  c->predict_every = every;
  return PIC_OK;
}
