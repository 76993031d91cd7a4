// pic_push_mixed_noalloc: the binned mixed-precision push for callers that
// cannot allocate device memory.
//
// Some host programs are not allowed to call cudaMalloc at the point where
// they push particles: an application whose device memory is owned and carved
// up by another framework, a real-time loop that must not hit the allocator or
// its implicit synchronisation, or a plugin whose host forbids allocations
// after start-up.  They can still hand over their own particle and field
// arrays.  This entry point takes those arrays and keeps everything else it
// needs (weight table, per-k queues, counters, work cursor) in one file-scope
// __device__ array of fixed size, so it never allocates.
//
// Cost of that choice: the array below (~12.8 MB) exists on every GPU that
// loads the library, from load until process exit, and all calls share it.
#include <math.h>
#include <stddef.h>
#include <string.h>

#include <mutex>

#include "pic_internal.h"

namespace pic {
namespace {

constexpr int64_t kNoAllocMaxParticles = 65536;
constexpr int64_t kRows = (((int64_t)1 << (2 * (kMaxK + 1))) - 1) / 3 + 1;  // wrows_total(7)
constexpr int64_t kMaxStride = 2 * (kMaxOrder + 1);
// FP32 weight tables, one per (order p, field-time reading), each with the rows
// of every k <= 7 (the rows of a smaller cap are a prefix of them) and a last
// row holding the theta = 1/2 weights every cap's criterion uses.  A table is
// built on the first call with its key and never rewritten, so work queued
// with one key never reads another key's weights.  Table (p, ft) starts at
// float ft * kRows * kSumStride + kRows * (p - 1)(p + 2).
constexpr int64_t kSumStride = 2 * (2 + 3 + 4 + 5 + 6);  // sum over p = 1..5 of 2(p + 1)
constexpr int64_t table_offset(int p, int ft) {
  return ft * kRows * kSumStride + kRows * (int64_t)(p - 1) * (p + 2);
}

struct NoAllocScratch {
  double wtab64[kRows * kMaxStride];  // build buffer of one table
  float wtab32[2 * kRows * kSumStride];
  int32_t queue[2 * 7 * kNoAllocMaxParticles];
  int32_t qcount[64];  // [0,16): per-k counts of both queue sets; 16: cursor; 18: blocks done
  DevStats stats;      // counters of the current call; the error word is kept until reported
};

// The scratch.  Host code must not use this name as an address: its device
// address comes from cudaGetSymbolAddress (see scratch_on_current_device).
__device__ __align__(256) unsigned char g_noalloc_scratch[sizeof(NoAllocScratch)];

constexpr int kMaxDevices = 64;
struct DeviceSlot {
  NoAllocScratch* ptr = nullptr;  // device address of g_noalloc_scratch
  int sm_count = 0;
  bool built[2][kMaxOrder + 1] = {};  // weight table (field_time, order) is in place
};
DeviceSlot g_slots[kMaxDevices];
std::mutex g_mutex;  // guards g_slots

thread_local char g_err[256];

int fail(int code, const char* msg) {
  strncpy(g_err, msg, sizeof(g_err) - 1);
  set_global_error(g_err);
  return code;
}

// With the device current and g_mutex held: the device address of the
// scratch array (looked up once per device).
int scratch_on_current_device(int dev, DeviceSlot** out) {
  DeviceSlot& s = g_slots[dev];
  if (!s.ptr) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess || !p) return fail(PIC_ECUDA, "pic_push_mixed_noalloc: cudaGetSymbolAddress failed");
    if (cudaDeviceGetAttribute(&s.sm_count, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
      return fail(PIC_ECUDA, "pic_push_mixed_noalloc: cannot query the device");
    s.ptr = (NoAllocScratch*)p;
  }
  *out = &s;
  return PIC_OK;
}

// With g_mutex held: the FP32 weight table of (p, ft), built on stream st and
// waited for the first time it is asked for (so a build failure is seen here
// and the table is complete before any later call can read it).
int table_on_device(DeviceSlot& s, int p, int ft, cudaStream_t st, const float** out) {
  NoAllocScratch* S = s.ptr;
  float* t = S->wtab32 + table_offset(p, ft);
  if (!s.built[ft][p]) {
    cudaError_t e = build_wtab_f64(S->wtab64, p, kMaxK, ft, st);
    if (e == cudaSuccess) e = build_wtab_f32(t, S->wtab64, kRows * 2 * (p + 1), st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return fail(PIC_ECUDA, cudaGetErrorString(e));
    s.built[ft][p] = true;
  }
  *out = t;
  return PIC_OK;
}

}  // namespace
}  // namespace pic

using namespace pic;

extern "C" int pic_push_mixed_noalloc(const pic_params* prm, int64_t n_particles, int32_t* cell,
                                      float* frac, float* px, float* py, float* pz,
                                      uint8_t* status, const float* const* Ey_levels,
                                      const float* const* Bz_levels, const int64_t* level_i0,
                                      int64_t window_cells, int64_t n0, int64_t n_steps,
                                      void* stream, pic_step_stats* stats) {
  if (!prm || !Ey_levels || !Bz_levels || !level_i0)
    return fail(PIC_EINVAL, "pic_push_mixed_noalloc: NULL argument");
  if (!(prm->dt > 0) || !(prm->dx > 0) || !(prm->psi_max > 0) || !isfinite(prm->qm) || prm->qm == 0.0)
    return fail(PIC_EINVAL, "pic_push_mixed_noalloc: dt, dx, psi_max must be > 0 and qm != 0");
  if (!((float)prm->dt >= 0x1p-100f && (float)prm->dt < 0x1p100f))
    return fail(PIC_EINVAL, "pic_push_mixed_noalloc: the mixed form needs 2^-100 <= dt < 2^100");
  if (prm->order < 1 || prm->order > kMaxOrder || prm->k_max < 0 || prm->k_max > kMaxK ||
      (prm->field_time != 0 && prm->field_time != 1))
    return fail(PIC_EINVAL, "pic_push_mixed_noalloc: order 1..5, k_max 0..7, field_time 0/1");
  if (prm->precision != PIC_MIXED || prm->schedule != PIC_SCHED_BINNED || prm->diagnostics != 0 ||
      prm->carry != 0)
    return fail(PIC_EINVAL, "pic_push_mixed_noalloc: needs precision PIC_MIXED, schedule PIC_SCHED_BINNED, no diagnostics, carry 0");
  if (n_particles < 0 || n_particles > kNoAllocMaxParticles)
    return fail(PIC_EINVAL, "pic_push_mixed_noalloc: n_particles exceeds the 65,536 the static scratch holds");
  if (n_particles > 0 && (!cell || !frac || !px || !py || !pz || !status))
    return fail(PIC_EINVAL, "pic_push_mixed_noalloc: NULL particle array");
  if (window_cells < 16 || window_cells > ((int64_t)1 << 30) || (window_cells & (window_cells - 1)))
    return fail(PIC_EINVAL, "pic_push_mixed_noalloc: window_cells must be a power of two >= 16");
  if (n_steps < 1) return fail(PIC_EINVAL, "pic_push_mixed_noalloc: n_steps must be >= 1");
  const int p = prm->order;
  for (int64_t r = 0; r < p + n_steps; ++r) {
    if (!Ey_levels[r] || !Bz_levels[r]) return fail(PIC_EINVAL, "pic_push_mixed_noalloc: NULL level");
    if (level_i0[r] < -((int64_t)1 << 30) || level_i0[r] + window_cells > ((int64_t)1 << 30))
      return fail(PIC_EINVAL, "pic_push_mixed_noalloc: level window outside +-2^30 nodes");
  }

  cudaStream_t st = (cudaStream_t)stream;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices)
    return fail(PIC_ECUDA, "pic_push_mixed_noalloc: no usable current CUDA device");
  DeviceSlot* slot = nullptr;
  const float* wtab = nullptr;
  {
    std::lock_guard<std::mutex> lock(g_mutex);
    int rc = scratch_on_current_device(dev, &slot);
    if (rc == PIC_OK) rc = table_on_device(*slot, p, prm->field_time, st, &wtab);
    if (rc != PIC_OK) return rc;
  }
  NoAllocScratch* S = slot->ptr;
  auto cuda_fail = [](cudaError_t e) {
    return fail(PIC_ECUDA, cudaGetErrorString(e));
  };
  cudaError_t e;
  // what must start at zero: queue counts, cursor, block counter, counters
  // (not the error word: an asynchronous call's give-up stays set until a
  // call with stats reports it)
  if ((e = cudaMemsetAsync(S->qcount, 0, sizeof(S->qcount), st)) != cudaSuccess) return cuda_fail(e);
  if ((e = cudaMemsetAsync(&S->stats, 0, offsetof(DevStats, error), st)) != cudaSuccess) return cuda_fail(e);

  const int64_t W = window_cells;
  auto window_of = [&](int64_t step, int64_t* lo, int64_t* hi) {
    *lo = INT64_MIN;
    *hi = INT64_MAX;
    for (int l = 0; l <= p; ++l) {
      const int64_t r = step - n0 + l;  // entry of level step - p + l
      if (level_i0[r] > *lo) *lo = level_i0[r];
      if (level_i0[r] + W - 1 < *hi) *hi = level_i0[r] + W - 1;
    }
  };
  PushArgsMixed base;
  memset(&base, 0, sizeof(base));
  base.keep_step = INT64_MIN;
  base.n = n_particles;
  base.cell = cell; base.frac = frac; base.px = px; base.py = py; base.pz = pz;
  base.status = status;
  base.tma = (((uintptr_t)cell | (uintptr_t)frac | (uintptr_t)px | (uintptr_t)py | (uintptr_t)pz |
               (uintptr_t)status) & 15) == 0;
  base.mask = (int32_t)(W - 1);
  base.dt = (float)prm->dt;
  base.psi_max = (float)prm->psi_max;
  base.qm = (float)prm->qm;
  base.qm_abs = fabsf((float)prm->qm);
  base.inv_dx = (float)(1.0 / prm->dx);
  base.k_max = prm->k_max;
  base.field_time = prm->field_time;
  lagrange_monomials(p, base.mono);
  base.wtab = wtab;
  base.crit_row = kRows - 1;  // theta = 1/2, the same weights as the cap's own criterion row
  base.stats = &S->stats;
  base.qcap = kNoAllocMaxParticles;
  base.cursor = (int*)(S->qcount + 16);
  base.blocks_done = (unsigned*)(S->qcount + 18);
  const int64_t qsz = 7 * kNoAllocMaxParticles;

  if (n_particles > 0) {
    for (int64_t j = 0; j < n_steps; ++j) {
      const int64_t s = n0 + j;
      PushArgsMixed a = base;
      int64_t lo, hi, plo, phi;
      window_of(s, &lo, &hi);
      const int64_t prev = j > 0 ? s - 1 : s;
      window_of(prev, &plo, &phi);
      for (int l = 0; l <= p; ++l) {
        a.E[l] = Ey_levels[s - n0 + l];
        a.B[l] = Bz_levels[s - n0 + l];
        a.Ep[l] = Ey_levels[prev - n0 + l];
        a.Bp[l] = Bz_levels[prev - n0 + l];
      }
      a.lo = (int32_t)lo; a.hi = (int32_t)hi;
      a.lo_p = (int32_t)plo; a.hi_p = (int32_t)phi;
      a.queue_in = S->queue + (j & 1) * qsz;
      a.queue_out = S->queue + ((j + 1) & 1) * qsz;
      a.qcount_in = S->qcount + (j & 1) * 8;
      a.qcount_out = S->qcount + ((j + 1) & 1) * 8;
      a.parity_cur = (int)(j & 1);
      a.parity_next = (int)((j + 1) & 1);
      if ((e = launch_push_mixed(a, p, PIC_SCHED_BINNED, slot->sm_count, st, nullptr)) != cudaSuccess)
        return cuda_fail(e);
      if (j == n_steps - 1) {
        PushArgsMixed f = a;
        for (int l = 0; l <= p; ++l) {
          f.Ep[l] = a.E[l];
          f.Bp[l] = a.B[l];
        }
        f.lo_p = a.lo; f.hi_p = a.hi;
        f.queue_in = S->queue + (n_steps & 1) * qsz;
        f.qcount_in = S->qcount + (n_steps & 1) * 8;
        f.queue_out = S->queue + ((n_steps + 1) & 1) * qsz;
        f.qcount_out = S->qcount + ((n_steps + 1) & 1) * 8;
        f.finalize = 1;
        if ((e = launch_push_mixed(f, p, PIC_SCHED_BINNED, slot->sm_count, st, nullptr)) != cudaSuccess)
          return cuda_fail(e);
      }
    }
  }
  if (!stats) return PIC_OK;
  DevStats h;
  if ((e = cudaMemcpyAsync(&h, &S->stats, sizeof(DevStats), cudaMemcpyDeviceToHost, st)) != cudaSuccess)
    return cuda_fail(e);
  if ((e = cudaStreamSynchronize(st)) != cudaSuccess) return cuda_fail(e);
  memset(stats, 0, sizeof(*stats));
  for (int k = 0; k < 8; ++k) stats->k_hist[k] = (int64_t)h.k_hist[k];
  stats->substeps = (int64_t)h.substeps;
  stats->n_star = (int64_t)h.n_star;
  stats->clamped = (int64_t)h.clamped;
  stats->out_of_window = (int64_t)h.lost;
  stats->error = h.error;
  if (h.error) {
    if ((e = cudaMemsetAsync(&S->stats.error, 0, sizeof(int), st)) != cudaSuccess) return cuda_fail(e);
    if ((e = cudaStreamSynchronize(st)) != cudaSuccess) return cuda_fail(e);
    return fail(PIC_ETIMEOUT, "pic_push_mixed_noalloc: a bounded device wait gave up (this call or an "
                              "earlier one without stats); particle state is not trustworthy");
  }
  if (stats->out_of_window) return fail(PIC_ERANGE, "particles left the field window");
  if (stats->clamped) return fail(PIC_EKMAX, "criterion capped at k_max");
  return PIC_OK;
}

extern "C" int pic_noalloc_inject_error(int32_t word, void* stream) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices)
    return fail(PIC_ECUDA, "pic_noalloc_inject_error: no usable current CUDA device");
  DeviceSlot* slot = nullptr;
  {
    std::lock_guard<std::mutex> lock(g_mutex);
    int rc = scratch_on_current_device(dev, &slot);
    if (rc != PIC_OK) return rc;
  }
  // pageable source: the copy is staged before cudaMemcpyAsync returns
  cudaError_t e = cudaMemcpyAsync(&slot->ptr->stats.error, &word, sizeof(int32_t),
                                  cudaMemcpyHostToDevice, (cudaStream_t)stream);
  if (e != cudaSuccess) return fail(PIC_ECUDA, cudaGetErrorString(e));
  return PIC_OK;
}
