// C ABI of batched ensembles (pic_batch_*): many independent problems in one
// particle store and one launch per macro step (push_batch.cu), optional
// CUDA-graph capture of multi-step calls, and an autotuner for the stream
// chunk length and the grid.
#include <math.h>
#include <stdio.h>
#include <string.h>

#include <new>
#include <vector>

#include "pic_internal.h"

using namespace pic;

struct pic_batch {
  int32_t n_ens = 0, order = 3;
  int64_t W = 0;
  int32_t R = 0;
  cudaStream_t stream = nullptr;
  int sm_count = 152;
  std::vector<pic_ensemble> ens_h;
  std::vector<EnsDev> ens_dev_h;
  EnsDev* ens_dev = nullptr;
  int64_t n_total = 0, n_chunks = 0;
  int32_t chunk = 256, blocks_per_sm = 2;
  bool use_graph = false;
  int32_t* cell = nullptr;
  float *frac = nullptr, *px = nullptr, *py = nullptr, *pz = nullptr;
  uint8_t* status = nullptr;
  float* ring = nullptr;
  int64_t* slot_i0 = nullptr;  // [n_ens][R]
  int64_t* i0_dev = nullptr;   // [n_ens]
  double* staging = nullptr;   // 2 x n_ens x W
  double* wtab64 = nullptr;
  float* wtab32 = nullptr;
  DevStats* dstats = nullptr;
  int32_t* queue = nullptr;   // 2 x 7 x n_total
  int32_t* qcount = nullptr;  // 2 x n_ens x 8, then cursor, blocks done
  int64_t* prefix = nullptr;  // 7 n_ens + 1
  float* half = nullptr;      // 2 x n_ens x W
  float* coef = nullptr;      // 2 (step parity) x n_ens x W x 2(p+1): node coefficient tables
  int32_t* lag_step = nullptr;  // per particle: the step a deferred particle is in (call-relative)
  uint16_t* lag_j = nullptr;    // and the sub-steps of it done
  int32_t heavy_budget = 1024;  // sub-steps of long sub-cycles per particle and launch
  std::vector<int64_t> slot_level;
  cudaGraphExec_t graph = nullptr;
  bool timing = false;
  std::vector<cudaEvent_t> ev;
  size_t ev_used = 0;
  int64_t launches = 0;
  char err[256] = {0};
};

static int bfail(pic_batch* b, int code, const char* msg) {
  if (b) {
    strncpy(b->err, msg, sizeof(b->err) - 1);
    b->err[sizeof(b->err) - 1] = 0;
  }
  set_global_error(msg);
  return code;
}

#define BATCH_TRY(b, call)                                               \
  do {                                                                   \
    cudaError_t e_ = (call);                                             \
    if (e_ != cudaSuccess) return bfail((b), PIC_ECUDA, cudaGetErrorString(e_)); \
  } while (0)

static void batch_free(pic_batch* b) {
  if (b->graph) cudaGraphExecDestroy(b->graph);
  for (cudaEvent_t e : b->ev) cudaEventDestroy(e);
  void* ptrs[] = {b->ens_dev, b->cell, b->frac, b->px, b->py, b->pz, b->status, b->ring,
                  b->slot_i0, b->i0_dev, b->staging, b->wtab64, b->wtab32, b->dstats,
                  b->queue, b->qcount, b->prefix, b->half, b->coef, b->lag_step, b->lag_j};
  for (void* p : ptrs)
    if (p) cudaFree(p);
}

extern "C" int pic_batch_create(const pic_ensemble* ens, int32_t n_ens, int32_t order,
                                int64_t window_cells, int32_t ring_levels, void* stream,
                                pic_batch** out) {
  if (!ens || !out || n_ens < 1 || n_ens > 65535)
    return bfail(nullptr, PIC_EINVAL, "pic_batch_create: 1..65535 ensembles required");
  *out = nullptr;
  if (order < 1 || order > kMaxOrder) return bfail(nullptr, PIC_EINVAL, "pic_batch_create: order must be 1..5");
  if (window_cells < 16 || window_cells > ((int64_t)1 << 28) || (window_cells & (window_cells - 1)))
    return bfail(nullptr, PIC_EINVAL, "pic_batch_create: window_cells must be a power of two in [16, 2^28]");
  if (ring_levels < order + 2 || ring_levels > (1 << 20))
    return bfail(nullptr, PIC_EINVAL, "pic_batch_create: ring_levels must be >= order + 2");
  int64_t total = 0;
  for (int e = 0; e < n_ens; ++e) {
    const pic_ensemble& q = ens[e];
    if (!(q.dt > 0) || !(q.dx > 0) || !(q.psi_max > 0) || !isfinite(q.qm) || q.qm == 0.0 ||
        q.k_max < 0 || q.k_max > kMaxK || (q.field_time != 0 && q.field_time != 1) ||
        q.n_particles < 0 || !((float)q.dt >= 0x1p-100f && (float)q.dt < 0x1p100f))
      return bfail(nullptr, PIC_EINVAL, "pic_batch_create: an ensemble's parameters are out of range");
    total += q.n_particles;
  }
  if (total > ((int64_t)1 << 31) - 1) return bfail(nullptr, PIC_EINVAL, "pic_batch_create: too many particles");
  pic_batch* b = new (std::nothrow) pic_batch();
  if (!b) return bfail(nullptr, PIC_ENOMEM, "pic_batch_create: host allocation failed");
  b->n_ens = n_ens;
  b->order = order;
  b->W = window_cells;
  b->R = ring_levels;
  b->stream = (cudaStream_t)stream;
  b->ens_h.assign(ens, ens + n_ens);
  b->n_total = total;
  b->slot_level.assign(ring_levels, INT64_MIN);
  int dev = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&b->sm_count, cudaDevAttrMultiProcessorCount, dev);
  const size_t cap = (size_t)(total > 0 ? total : 1);
  const int64_t rows = wrows_total(kMaxK);
  const int64_t wcount = rows * 2 * (order + 1);
  cudaError_t e = cudaSuccess;
  auto A = [&](void** p, size_t bytes) {
    if (e == cudaSuccess) e = cudaMalloc(p, bytes);
  };
  A((void**)&b->ens_dev, sizeof(EnsDev) * n_ens);
  A((void**)&b->cell, cap * 4);
  A((void**)&b->frac, cap * 4);
  A((void**)&b->px, cap * 4);
  A((void**)&b->py, cap * 4);
  A((void**)&b->pz, cap * 4);
  A((void**)&b->status, cap);
  const size_t ring_floats = (size_t)n_ens * 2 * (2 * (size_t)ring_levels) * (size_t)window_cells;
  A((void**)&b->ring, ring_floats * 4);
  A((void**)&b->slot_i0, sizeof(int64_t) * n_ens * ring_levels);
  A((void**)&b->i0_dev, sizeof(int64_t) * n_ens);
  A((void**)&b->staging, sizeof(double) * 2 * n_ens * window_cells);
  A((void**)&b->wtab64, (size_t)wcount * 8);
  A((void**)&b->wtab32, (size_t)wcount * 4);
  A((void**)&b->dstats, sizeof(DevStats));
  A((void**)&b->queue, 2 * 7 * cap * 4);
  A((void**)&b->qcount, sizeof(int32_t) * (2 * 8 * (size_t)n_ens + 8));
  A((void**)&b->prefix, sizeof(int64_t) * (7 * (size_t)n_ens + 1));
  A((void**)&b->half, sizeof(float) * 2 * (size_t)n_ens * window_cells);
  A((void**)&b->coef, sizeof(float) * 2 * (size_t)n_ens * window_cells * 2 * (size_t)(order + 1));
  A((void**)&b->lag_step, cap * 4);
  A((void**)&b->lag_j, cap * 2);
  if (e != cudaSuccess) {
    batch_free(b);
    delete b;
    cudaGetLastError();
    return bfail(nullptr, PIC_ENOMEM, "pic_batch_create: device allocation failed");
  }
  // ensemble table
  int64_t first = 0, chunk_first = 0;
  b->ens_dev_h.resize(n_ens);
  for (int q = 0; q < n_ens; ++q) {
    const pic_ensemble& s = ens[q];
    EnsDev& d = b->ens_dev_h[q];
    memset(&d, 0, sizeof(d));
    d.dt = (float)s.dt;
    d.psi_max = (float)s.psi_max;
    d.qm = (float)s.qm;
    d.qm_abs = fabsf((float)s.qm);
    d.inv_dx = (float)(1.0 / s.dx);
    d.k_max = s.k_max;
    d.field_time = s.field_time;
    d.ringE = b->ring + (size_t)q * 2 * (2 * (size_t)ring_levels) * window_cells;
    d.ringB = d.ringE + (2 * (size_t)ring_levels) * window_cells;
    d.slot_i0 = b->slot_i0 + (size_t)q * ring_levels;
    d.first = first;
    d.count = s.n_particles;
    d.chunk_first = chunk_first;
    first += s.n_particles;
    chunk_first += (s.n_particles + b->chunk - 1) / b->chunk;
  }
  b->n_chunks = chunk_first;
  e = cudaMemcpy(b->ens_dev, b->ens_dev_h.data(), sizeof(EnsDev) * n_ens, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemset(b->qcount, 0, sizeof(int32_t) * (2 * 8 * (size_t)n_ens + 8));
  if (e == cudaSuccess) e = cudaMemset(b->dstats, 0, sizeof(DevStats));
  if (e == cudaSuccess) e = cudaMemset(b->status, 0, cap);
  if (e == cudaSuccess) e = build_wtab_f64(b->wtab64, order, kMaxK, 0, b->stream);
  if (e == cudaSuccess) e = build_wtab_f32(b->wtab32, b->wtab64, wcount, b->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
  b->blocks_per_sm = batch_max_blocks_per_sm(order);
  if (e != cudaSuccess) {
    batch_free(b);
    delete b;
    return bfail(nullptr, PIC_ECUDA, "pic_batch_create: initialisation failed");
  }
  b->launches = 2;
  *out = b;
  return PIC_OK;
}

extern "C" int pic_batch_destroy(pic_batch* b) {
  if (!b) return PIC_OK;
  cudaStreamSynchronize(b->stream);
  batch_free(b);
  delete b;
  return PIC_OK;
}

// Re-chunk the ensembles (the chunk boundaries depend on the chunk length).
static int set_chunk(pic_batch* b, int32_t chunk) {
  b->chunk = chunk;
  int64_t chunk_first = 0;
  for (int q = 0; q < b->n_ens; ++q) {
    b->ens_dev_h[q].chunk_first = chunk_first;
    chunk_first += (b->ens_dev_h[q].count + chunk - 1) / chunk;
  }
  b->n_chunks = chunk_first;
  BATCH_TRY(b, cudaMemcpyAsync(b->ens_dev, b->ens_dev_h.data(), sizeof(EnsDev) * b->n_ens,
                               cudaMemcpyHostToDevice, b->stream));
  BATCH_TRY(b, cudaStreamSynchronize(b->stream));
  return PIC_OK;
}

extern "C" int pic_batch_config(pic_batch* b, int32_t chunk, int32_t blocks_per_sm,
                                int32_t use_graph) {
  if (!b) return PIC_EINVAL;
  if (chunk < 32 || chunk > 8192 || (chunk % 32))
    return bfail(b, PIC_EINVAL, "pic_batch_config: chunk must be a multiple of 32 in [32, 8192]");
  const int maxb = batch_max_blocks_per_sm(b->order);
  if (blocks_per_sm < 1 || blocks_per_sm > maxb)
    return bfail(b, PIC_EINVAL, "pic_batch_config: blocks_per_sm out of the kernel's occupancy");
  b->blocks_per_sm = blocks_per_sm;
  b->use_graph = use_graph != 0;
  return set_chunk(b, chunk);
}

extern "C" int pic_batch_particles_write(pic_batch* b, const double* x, const double* px,
                                         const double* py, const double* pz, const uint8_t* status,
                                         int32_t where) {
  if (!b || !x || !px || !py || !pz) return PIC_EINVAL;
  if (where != PIC_HOST && where != PIC_DEVICE) return PIC_EINVAL;
  const cudaMemcpyKind kin = where == PIC_HOST ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice;
  if (status)
    BATCH_TRY(b, cudaMemcpyAsync(b->status, status, (size_t)b->n_total, kin, b->stream));
  else
    BATCH_TRY(b, cudaMemsetAsync(b->status, 0, (size_t)b->n_total, b->stream));
  // staged per ensemble (each its own dx)
  double* st = nullptr;
  const int64_t biggest = [&] {
    int64_t m = 0;
    for (auto& q : b->ens_h) m = q.n_particles > m ? q.n_particles : m;
    return m;
  }();
  if (where == PIC_HOST && biggest > 0) BATCH_TRY(b, cudaMalloc((void**)&st, sizeof(double) * 4 * biggest));
  for (int q = 0; q < b->n_ens; ++q) {
    const EnsDev& d = b->ens_dev_h[q];
    if (d.count == 0) continue;
    const double* src[4] = {x + d.first, px + d.first, py + d.first, pz + d.first};
    if (where == PIC_HOST) {
      for (int c = 0; c < 4; ++c)
        BATCH_TRY(b, cudaMemcpyAsync(st + c * d.count, src[c], sizeof(double) * d.count,
                                     cudaMemcpyHostToDevice, b->stream));
      for (int c = 0; c < 4; ++c) src[c] = st + c * d.count;
    }
    BATCH_TRY(b, launch_to_mixed(src[0], src[1], src[2], src[3], b->cell + d.first, b->frac + d.first,
                                 b->px + d.first, b->py + d.first, b->pz + d.first,
                                 1.0 / b->ens_h[q].dx, d.count, b->stream));
    ++b->launches;
    if (where == PIC_HOST) BATCH_TRY(b, cudaStreamSynchronize(b->stream));
  }
  if (st) cudaFree(st);
  BATCH_TRY(b, cudaStreamSynchronize(b->stream));
  return PIC_OK;
}

extern "C" int pic_batch_particles_read(pic_batch* b, double* x, double* px, double* py, double* pz,
                                        uint8_t* status, int32_t where) {
  if (!b) return PIC_EINVAL;
  if (where != PIC_HOST && where != PIC_DEVICE) return PIC_EINVAL;
  const cudaMemcpyKind kout = where == PIC_HOST ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice;
  if (status) BATCH_TRY(b, cudaMemcpyAsync(status, b->status, (size_t)b->n_total, kout, b->stream));
  double* st = nullptr;
  if (where == PIC_HOST && b->n_total > 0)
    BATCH_TRY(b, cudaMalloc((void**)&st, sizeof(double) * 4 * b->n_total));
  for (int q = 0; q < b->n_ens; ++q) {
    const EnsDev& d = b->ens_dev_h[q];
    if (d.count == 0) continue;
    double* dst[4] = {x ? x + d.first : nullptr, px ? px + d.first : nullptr,
                      py ? py + d.first : nullptr, pz ? pz + d.first : nullptr};
    if (where == PIC_HOST)
      for (int c = 0; c < 4; ++c) dst[c] = st + c * b->n_total + d.first;
    BATCH_TRY(b, launch_from_mixed(b->cell + d.first, b->frac + d.first, b->px + d.first,
                                   b->py + d.first, b->pz + d.first, dst[0], dst[1], dst[2], dst[3],
                                   b->ens_h[q].dx, d.count, b->stream));
    ++b->launches;
  }
  if (where == PIC_HOST) {
    double* outs[4] = {x, px, py, pz};
    for (int c = 0; c < 4; ++c)
      if (outs[c])
        BATCH_TRY(b, cudaMemcpyAsync(outs[c], st + c * b->n_total, sizeof(double) * b->n_total,
                                     cudaMemcpyDeviceToHost, b->stream));
  }
  BATCH_TRY(b, cudaStreamSynchronize(b->stream));
  if (st) cudaFree(st);
  return PIC_OK;
}

extern "C" int pic_batch_fields_upload(pic_batch* b, int64_t level, const int64_t* i0,
                                       const double* Ey, const double* Bz, int32_t where) {
  if (!b || !i0 || !Ey || !Bz) return PIC_EINVAL;
  if (where != PIC_HOST && where != PIC_DEVICE) return PIC_EINVAL;
  for (int q = 0; q < b->n_ens; ++q)
    if (i0[q] < -((int64_t)1 << 30) || i0[q] + b->W > ((int64_t)1 << 30))
      return bfail(b, PIC_EINVAL, "pic_batch_fields_upload: window origin out of range");
  const int64_t slot = ((level % b->R) + b->R) % b->R;
  const double* e = Ey;
  const double* bb = Bz;
  const size_t bytes = sizeof(double) * b->n_ens * b->W;
  if (where == PIC_HOST) {
    BATCH_TRY(b, cudaMemcpyAsync(b->staging, Ey, bytes, cudaMemcpyHostToDevice, b->stream));
    BATCH_TRY(b, cudaMemcpyAsync(b->staging + b->n_ens * b->W, Bz, bytes, cudaMemcpyHostToDevice,
                                 b->stream));
    e = b->staging;
    bb = b->staging + b->n_ens * b->W;
  }
  BATCH_TRY(b, cudaMemcpyAsync(b->i0_dev, i0, sizeof(int64_t) * b->n_ens, cudaMemcpyHostToDevice,
                               b->stream));
  BATCH_TRY(b, launch_batch_scatter(b->ens_dev, b->n_ens, slot, b->R, b->W, e, bb, b->i0_dev,
                                    b->slot_i0, b->stream));
  ++b->launches;
  if (where == PIC_HOST) BATCH_TRY(b, cudaStreamSynchronize(b->stream));
  b->slot_level[slot] = level;
  return PIC_OK;
}

static int batch_timing_pair(pic_batch* b, cudaEvent_t* a, cudaEvent_t* c) {
  if (2 * (b->ev_used + 1) > b->ev.size()) {
    for (int q = 0; q < 2; ++q) {
      cudaEvent_t e;
      BATCH_TRY(b, cudaEventCreate(&e));
      b->ev.push_back(e);
    }
  }
  *a = b->ev[2 * b->ev_used];
  *c = b->ev[2 * b->ev_used + 1];
  ++b->ev_used;
  return PIC_OK;
}

static int queue_steps(pic_batch* b, int64_t n, int64_t n_steps) {
  const int p = b->order;
  BatchArgs base;
  memset(&base, 0, sizeof(base));
  base.n_ens = b->n_ens;
  base.ens = b->ens_dev;
  base.n_total = b->n_total;
  base.n_chunks = b->n_chunks;
  base.chunk = b->chunk;
  base.cell = b->cell; base.frac = b->frac; base.px = b->px; base.py = b->py; base.pz = b->pz;
  base.status = b->status;
  base.R = b->R;
  base.lstride = b->W;
  base.mask = (int32_t)(b->W - 1);
  base.wtab = b->wtab32;
  base.crit_row = wrows_total(kMaxK) - 1;
  lagrange_monomials(p, base.mono);
  base.stats = b->dstats;
  base.prefix = b->prefix;
  base.half = b->half;
  base.cursor = (int*)(b->qcount + 16 * b->n_ens);
  base.blocks_done = (unsigned*)(b->qcount + 16 * b->n_ens + 2);
  const int64_t qsz = 7 * b->n_total;
  const int blocks = b->sm_count * b->blocks_per_sm;
  for (int64_t j = 0; j <= n_steps; ++j) {
    const bool fin = j == n_steps;
    const int64_t s = fin ? n + n_steps - 1 : n + j;
    BatchArgs a = base;
    a.start_cur = (((s - p) % b->R) + b->R) % b->R;
    a.start_prev = (j > 0 && !fin) ? ((((s - 1 - p) % b->R) + b->R) % b->R) : a.start_cur;
    if (fin) a.start_prev = a.start_cur;  // the closing launch finishes step s with its own fields
    a.queue_in = b->queue + (j & 1) * qsz;
    a.queue_out = b->queue + ((j + 1) & 1) * qsz;
    a.qcount_in = b->qcount + (j & 1) * 8 * b->n_ens;
    a.qcount_out = b->qcount + ((j + 1) & 1) * 8 * b->n_ens;
    a.parity_cur = (int)(j & 1);
    a.parity_next = (int)((j + 1) & 1);
    a.finalize = fin ? 1 : 0;
    a.lag_step = b->lag_step;
    a.lag_j = b->lag_j;
    a.step0 = n;
    a.step_cur = fin ? s + 1 : s;  // the closing launch brings every particle to the end of s
    a.heavy_budget = b->heavy_budget;
    // node tables by step parity; the closing launch finishes step s with its own
    const int64_t table = b->n_ens * b->W * 2 * (p + 1);
    a.coef = b->coef + (s & 1) * table;
    a.coef_p = (j > 0 && !fin) ? b->coef + ((s - 1) & 1) * table : a.coef;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (b->timing && !fin) {
      int rc = batch_timing_pair(b, &e0, &e1);
      if (rc != PIC_OK) return rc;
      BATCH_TRY(b, cudaEventRecord(e0, b->stream));
    }
    int launches = 0;
    BATCH_TRY(b, launch_batch_step(a, p, blocks, b->stream, &launches));
    b->launches += launches;
    if (b->timing && !fin) BATCH_TRY(b, cudaEventRecord(e1, b->stream));
  }
  return PIC_OK;
}

extern "C" int pic_batch_push_step(pic_batch* b, int64_t n, int64_t n_steps, pic_step_stats* stats) {
  if (!b) return PIC_EINVAL;
  if (n_steps < 1) return bfail(b, PIC_EINVAL, "pic_batch_push_step: n_steps must be >= 1");
  const int p = b->order;
  for (int64_t lev = n - p; lev < n + n_steps; ++lev) {
    const int64_t slot = ((lev % b->R) + b->R) % b->R;
    if (b->slot_level[slot] != lev)
      return bfail(b, PIC_EINVAL, "pic_batch_push_step: a field level the steps need is not in the ring");
  }
  if (n_steps + p > b->R)
    return bfail(b, PIC_EINVAL, "pic_batch_push_step: more steps per call than the ring holds levels for");
  if (b->use_graph && b->stream && n_steps > 1) {
    if (b->graph) {
      BATCH_TRY(b, cudaStreamSynchronize(b->stream));
      cudaGraphExecDestroy(b->graph);
      b->graph = nullptr;
    }
    cudaGraph_t g = nullptr;
    BATCH_TRY(b, cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeThreadLocal));
    const int64_t before = b->launches;
    int rc = queue_steps(b, n, n_steps);
    cudaError_t e = cudaStreamEndCapture(b->stream, &g);
    if (rc != PIC_OK) {
      if (g) cudaGraphDestroy(g);
      return rc;
    }
    if (e != cudaSuccess) return bfail(b, PIC_ECUDA, cudaGetErrorString(e));
    e = cudaGraphInstantiate(&b->graph, g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) return bfail(b, PIC_ECUDA, cudaGetErrorString(e));
    BATCH_TRY(b, cudaGraphLaunch(b->graph, b->stream));
    b->launches = before + (b->launches - before);
  } else {
    int rc = queue_steps(b, n, n_steps);
    if (rc != PIC_OK) return rc;
  }
  if (!stats) return PIC_OK;
  DevStats h;
  BATCH_TRY(b, cudaMemcpyAsync(&h, b->dstats, sizeof(DevStats), cudaMemcpyDeviceToHost, b->stream));
  BATCH_TRY(b, cudaMemsetAsync(b->dstats, 0, sizeof(DevStats), b->stream));
  BATCH_TRY(b, cudaStreamSynchronize(b->stream));
  memset(stats, 0, sizeof(*stats));
  for (int k = 0; k < 8; ++k) stats->k_hist[k] = (int64_t)h.k_hist[k];
  stats->substeps = (int64_t)h.substeps;
  stats->n_star = (int64_t)h.n_star;
  stats->clamped = (int64_t)h.clamped;
  stats->out_of_window = (int64_t)h.lost;
  stats->error = h.error;
  if (stats->out_of_window) return bfail(b, PIC_ERANGE, "particles left the field window");
  if (stats->clamped) return bfail(b, PIC_EKMAX, "criterion capped at k_max");
  return PIC_OK;
}

extern "C" int pic_batch_timing(pic_batch* b, int32_t on, double* total_ms, int64_t* steps) {
  if (!b) return PIC_EINVAL;
  if (total_ms && steps) {
    BATCH_TRY(b, cudaStreamSynchronize(b->stream));
    double tot = 0.0;
    for (size_t q = 0; q < b->ev_used; ++q) {
      float ms = 0.f;
      BATCH_TRY(b, cudaEventElapsedTime(&ms, b->ev[2 * q], b->ev[2 * q + 1]));
      tot += ms;
    }
    *total_ms = tot;
    *steps = (int64_t)b->ev_used;
    b->ev_used = 0;
  }
  b->timing = on != 0;
  return PIC_OK;
}

extern "C" int64_t pic_batch_launch_count(const pic_batch* b) { return b ? b->launches : 0; }

// Autotuner: time `steps` macro steps from step n for each (chunk, blocks per
// SM) candidate, each from the same saved particle state; keep the fastest and
// put the state back.  The levels of steps n-1 .. n+steps-1 must be in the ring.
extern "C" int pic_batch_autotune(pic_batch* b, int64_t n, int32_t steps, int32_t* chunk_out,
                                  int32_t* blocks_out, double* ms_out) {
  if (!b || steps < 1) return PIC_EINVAL;
  const size_t N = (size_t)(b->n_total > 0 ? b->n_total : 1);
  char* save = nullptr;
  BATCH_TRY(b, cudaMalloc((void**)&save, N * 21));
  auto copy_state = [&](bool to_save) -> cudaError_t {
    void* arr[6] = {b->cell, b->frac, b->px, b->py, b->pz, b->status};
    const size_t sz[6] = {4, 4, 4, 4, 4, 1};
    size_t off = 0;
    for (int q = 0; q < 6; ++q) {
      cudaError_t e = to_save ? cudaMemcpyAsync(save + off, arr[q], N * sz[q], cudaMemcpyDeviceToDevice, b->stream)
                              : cudaMemcpyAsync(arr[q], save + off, N * sz[q], cudaMemcpyDeviceToDevice, b->stream);
      if (e != cudaSuccess) return e;
      off += N * sz[q];
    }
    return cudaSuccess;
  };
  cudaError_t e = copy_state(true);
  const int32_t chunks[4] = {128, 256, 512, 1024};
  const int maxb = batch_max_blocks_per_sm(b->order);
  double best = 1e300;
  int32_t best_c = b->chunk, best_b = b->blocks_per_sm;
  const bool graph = b->use_graph, timing = b->timing;
  b->use_graph = false;
  cudaEvent_t t0 = nullptr, t1 = nullptr;
  if (e == cudaSuccess) e = cudaEventCreate(&t0);
  if (e == cudaSuccess) e = cudaEventCreate(&t1);
  for (int ci = 0; ci < 4 && e == cudaSuccess; ++ci) {
    for (int bp = 1; bp <= maxb && e == cudaSuccess; ++bp) {
      if (set_chunk(b, chunks[ci]) != PIC_OK) { e = cudaErrorUnknown; break; }
      b->blocks_per_sm = bp;
      e = copy_state(false);
      if (e != cudaSuccess) break;
      b->timing = false;
      e = cudaEventRecord(t0, b->stream);
      if (e != cudaSuccess) break;
      if (queue_steps(b, n, steps) != PIC_OK) { e = cudaErrorUnknown; break; }
      e = cudaEventRecord(t1, b->stream);
      if (e == cudaSuccess) e = cudaEventSynchronize(t1);
      float ms = 0.f;
      if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, t0, t1);
      if (e == cudaSuccess && ms < best) {
        best = ms;
        best_c = chunks[ci];
        best_b = bp;
      }
    }
  }
  if (e == cudaSuccess) e = copy_state(false);
  if (e == cudaSuccess) e = cudaMemsetAsync(b->dstats, 0, sizeof(DevStats), b->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
  if (t0) cudaEventDestroy(t0);
  if (t1) cudaEventDestroy(t1);
  cudaFree(save);
  b->use_graph = graph;
  b->timing = timing;
  if (e != cudaSuccess) return bfail(b, PIC_ECUDA, "pic_batch_autotune: a trial failed");
  b->blocks_per_sm = best_b;
  int rc = set_chunk(b, best_c);
  if (rc != PIC_OK) return rc;
  if (chunk_out) *chunk_out = best_c;
  if (blocks_out) *blocks_out = best_b;
  if (ms_out) *ms_out = best / steps;
  return PIC_OK;
}

extern "C" const char* pic_batch_last_error(const pic_batch* b) { return b ? b->err : ""; }

extern "C" int pic_batch_heavy_budget(pic_batch* b, int32_t budget) {
  if (!b) return PIC_EINVAL;
  b->heavy_budget = budget == 0 ? 1024 : budget;
  return PIC_OK;
}
