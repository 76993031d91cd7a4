// C ABI of the learned sub-cycle-count predictor (pic_mlp_*): owns the FP32
// master parameters, the Adam moments and the gradient buffer on the device.
#include <math.h>
#include <stdio.h>
#include <string.h>

#include <new>
#include <vector>

#include "pic_internal.h"

using namespace pic;

struct pic_mlp {
  float* P = nullptr;     // packed FP32 parameters
  float* G = nullptr;     // gradient
  float* M1 = nullptr;    // Adam first moment
  float* M2 = nullptr;    // Adam second moment
  float* loss = nullptr;  // device scalar
  int step = 0;
  int sm_count = 0;
  cudaStream_t stream = nullptr;
};

static int mlp_fail(int code, const char* msg) {
  set_global_error(msg);
  return code;
}

#define MLP_TRY(call)                                                    \
  do {                                                                   \
    cudaError_t e_ = (call);                                             \
    if (e_ != cudaSuccess) return mlp_fail(PIC_ECUDA, cudaGetErrorString(e_)); \
  } while (0)

extern "C" int pic_mlp_param_count(void) { return mlp_param_count(); }

// He-uniform initial weights from a splitmix64 stream; zero biases.
extern "C" int pic_mlp_create(uint64_t seed, void* stream, pic_mlp** out) {
  if (!out) return mlp_fail(PIC_EINVAL, "pic_mlp_create: NULL out");
  *out = nullptr;
  pic_mlp* m = new (std::nothrow) pic_mlp();
  if (!m) return mlp_fail(PIC_ENOMEM, "pic_mlp_create: host allocation failed");
  m->stream = (cudaStream_t)stream;
  const int np = mlp_param_count();
  cudaError_t e = cudaSuccess;
  float** bufs[] = {&m->P, &m->G, &m->M1, &m->M2};
  for (float** b : bufs)
    if (e == cudaSuccess) e = cudaMalloc((void**)b, (size_t)np * sizeof(float));
  if (e == cudaSuccess) e = cudaMalloc((void**)&m->loss, sizeof(float));
  if (e != cudaSuccess) {
    for (float** b : bufs)
      if (*b) cudaFree(*b);
    if (m->loss) cudaFree(m->loss);
    delete m;
    return mlp_fail(PIC_ENOMEM, "pic_mlp_create: device allocation failed");
  }
  int dev = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&m->sm_count, cudaDevAttrMultiProcessorCount, dev);
  std::vector<float> h(np, 0.f);
  uint64_t x = seed;
  auto next = [&]() {
    x += 0x9E3779B97F4A7C15ull;
    uint64_t z = x;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    z ^= z >> 31;
    return (double)(z >> 11) * (1.0 / 9007199254740992.0);
  };
  const int sizes[4] = {6, 64, 64, 8};
  size_t off = 0;
  for (int l = 0; l < 3; ++l) {
    const int fi = sizes[l], fo = sizes[l + 1];
    const double bound = sqrt(6.0 / fi);
    for (int q = 0; q < fi * fo; ++q) h[off + q] = (float)((2.0 * next() - 1.0) * bound);
    off += (size_t)fi * fo + fo;  // biases stay zero
  }
  e = cudaMemcpy(m->P, h.data(), (size_t)np * sizeof(float), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemset(m->M1, 0, (size_t)np * sizeof(float));
  if (e == cudaSuccess) e = cudaMemset(m->M2, 0, (size_t)np * sizeof(float));
  if (e != cudaSuccess) {
    for (float** b : bufs) cudaFree(*b);
    cudaFree(m->loss);
    delete m;
    return mlp_fail(PIC_ECUDA, "pic_mlp_create: initialisation failed");
  }
  *out = m;
  return PIC_OK;
}

extern "C" int pic_mlp_destroy(pic_mlp* m) {
  if (!m) return PIC_OK;
  cudaStreamSynchronize(m->stream);
  cudaFree(m->P);
  cudaFree(m->G);
  cudaFree(m->M1);
  cudaFree(m->M2);
  cudaFree(m->loss);
  delete m;
  return PIC_OK;
}

extern "C" int pic_mlp_params(pic_mlp* m, float* buf, int32_t set, int32_t where) {
  if (!m || !buf) return mlp_fail(PIC_EINVAL, "pic_mlp_params: NULL argument");
  const size_t bytes = (size_t)mlp_param_count() * sizeof(float);
  const cudaMemcpyKind kin = where == PIC_HOST ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice;
  const cudaMemcpyKind kout = where == PIC_HOST ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice;
  if (set) {
    MLP_TRY(cudaMemcpyAsync(m->P, buf, bytes, kin, m->stream));
    MLP_TRY(cudaMemsetAsync(m->M1, 0, bytes, m->stream));
    MLP_TRY(cudaMemsetAsync(m->M2, 0, bytes, m->stream));
    m->step = 0;
  } else {
    MLP_TRY(cudaMemcpyAsync(buf, m->P, bytes, kout, m->stream));
  }
  if (where == PIC_HOST) MLP_TRY(cudaStreamSynchronize(m->stream));
  return PIC_OK;
}

static int grad_into(pic_mlp* m, const float* phi, const uint8_t* label, int64_t n) {
  MLP_TRY(cudaMemsetAsync(m->G, 0, (size_t)mlp_param_count() * sizeof(float), m->stream));
  MLP_TRY(cudaMemsetAsync(m->loss, 0, sizeof(float), m->stream));
  MLP_TRY(launch_mlp_grad(m->P, phi, label, n, m->G, m->loss, m->sm_count, m->stream));
  return PIC_OK;
}

extern "C" int pic_mlp_grad(pic_mlp* m, const float* phi, const uint8_t* label, int64_t n,
                            float* grad_out, float* loss_out) {
  if (!m || !phi || !label || n <= 0) return mlp_fail(PIC_EINVAL, "pic_mlp_grad: bad argument");
  int rc = grad_into(m, phi, label, n);
  if (rc != PIC_OK) return rc;
  if (grad_out)
    MLP_TRY(cudaMemcpyAsync(grad_out, m->G, (size_t)mlp_param_count() * sizeof(float),
                            cudaMemcpyDeviceToHost, m->stream));
  if (loss_out) MLP_TRY(cudaMemcpyAsync(loss_out, m->loss, sizeof(float), cudaMemcpyDeviceToHost, m->stream));
  MLP_TRY(cudaStreamSynchronize(m->stream));
  return PIC_OK;
}

extern "C" int pic_mlp_train_step(pic_mlp* m, const float* phi, const uint8_t* label, int64_t n,
                                  float lr, float* loss_out) {
  if (!m || !phi || !label || n <= 0 || !(lr > 0))
    return mlp_fail(PIC_EINVAL, "pic_mlp_train_step: bad argument");
  int rc = grad_into(m, phi, label, n);
  if (rc != PIC_OK) return rc;
  m->step += 1;
  MLP_TRY(launch_mlp_adam(m->P, m->G, m->M1, m->M2, lr, m->step, m->stream));
  if (loss_out) {
    MLP_TRY(cudaMemcpyAsync(loss_out, m->loss, sizeof(float), cudaMemcpyDeviceToHost, m->stream));
    MLP_TRY(cudaStreamSynchronize(m->stream));
  }
  return PIC_OK;
}

extern "C" int pic_mlp_infer(pic_mlp* m, const float* phi, int64_t n, uint8_t* pred) {
  if (!m || !phi || !pred || n < 0) return mlp_fail(PIC_EINVAL, "pic_mlp_infer: bad argument");
  MLP_TRY(launch_mlp_infer(m->P, phi, n, pred, m->sm_count, m->stream));
  return PIC_OK;
}

const float* pic::mlp_device_params(const pic_mlp* m) { return m ? m->P : nullptr; }
