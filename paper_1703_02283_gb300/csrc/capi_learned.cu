// The MLP object of the learned initial guess (include/pthroot.h, pr_mlp_*): parameters, Adam moments and
// batch work areas on the device; every operation runs in the kernels of k_learned.cu.
#include "pr_internal.h"

#include <math.h>
#include <string>

struct pr_mlp_s {
  int max_batch = 0;
  cudaStream_t stream = nullptr;
  int device = 0;
  int steps = 0;  // Adam steps taken
  float *theta = nullptr, *m = nullptr, *v = nullptr, *grad = nullptr;
  float *X = nullptr, *T = nullptr, *Y = nullptr, *H1 = nullptr, *H2 = nullptr;
  float *gpart = nullptr, *lpart = nullptr, *loss = nullptr;
};

namespace {

pr_status mfail(pr_status code, const std::string& msg) {
  pr::set_handleless_error(msg.c_str());
  return code;
}

#define PM_CK(call)                                                                                        \
  do {                                                                                                     \
    cudaError_t _e = (call);                                                                               \
    if (_e != cudaSuccess) return mfail(_e == cudaErrorMemoryAllocation ? PR_ENOMEM : PR_ECUDA,            \
                                        std::string(#call) + ": " + cudaGetErrorName(_e));                 \
  } while (0)

pr_status run_backward(pr_mlp mm, const float* X, const float* T, int B, bool adam, float lr, float* loss_out,
                       float* grad_out) {
  if (!mm) return mfail(PR_ESTATE, "pr_mlp: NULL model");
  if (!X || !T || B < 1 || B > mm->max_batch) return mfail(PR_EINVAL, "pr_mlp: bad batch");
  cudaSetDevice(mm->device);
  PM_CK(cudaMemcpyAsync(mm->X, X, sizeof(float) * 8 * (size_t)B, cudaMemcpyDefault, mm->stream));
  PM_CK(cudaMemcpyAsync(mm->T, T, sizeof(float) * 4 * (size_t)B, cudaMemcpyDefault, mm->stream));
  PM_CK(pr::mlp_forward(mm->theta, mm->X, B, mm->Y, mm->H1, mm->H2, mm->stream));
  float c1 = 1.0f, c2 = 1.0f;
  if (adam) {
    mm->steps += 1;
    c1 = 1.0f - powf(0.9f, (float)mm->steps);
    c2 = 1.0f - powf(0.999f, (float)mm->steps);
  }
  PM_CK(pr::mlp_backward(mm->theta, mm->X, mm->T, mm->Y, mm->H1, mm->H2, B, mm->gpart, mm->lpart, mm->grad, mm->loss,
                         mm->m, mm->v, mm->theta, lr, c1, c2, adam, mm->stream));
  float l = 0.0f;
  PM_CK(cudaMemcpyAsync(&l, mm->loss, sizeof(float), cudaMemcpyDeviceToHost, mm->stream));
  if (grad_out)
    PM_CK(cudaMemcpyAsync(grad_out, mm->grad, sizeof(float) * pr::mlp_params(), cudaMemcpyDefault, mm->stream));
  PM_CK(cudaStreamSynchronize(mm->stream));
  if (loss_out) *loss_out = l;
  return PR_OK;
}

}  // namespace

extern "C" {

pr_status pr_mlp_destroy(pr_mlp m) {
  if (!m) return PR_OK;
  cudaSetDevice(m->device);
  if (m->stream) cudaStreamSynchronize(m->stream);
  for (float* q : {m->theta, m->m, m->v, m->grad, m->X, m->T, m->Y, m->H1, m->H2, m->gpart, m->lpart, m->loss})
    if (q) cudaFree(q);
  delete m;
  return PR_OK;
}

pr_status pr_mlp_create(pr_mlp* out, const float* params, int max_batch, void* stream) {
  if (!out) return mfail(PR_EINVAL, "pr_mlp_create: m is NULL");
  *out = nullptr;
  if (!params || max_batch < 1 || max_batch > (1 << 24)) return mfail(PR_EINVAL, "pr_mlp_create: bad arguments");
  pr_mlp m = new pr_mlp_s();
  m->max_batch = max_batch;
  m->stream = (cudaStream_t)stream;
  cudaGetDevice(&m->device);
  const size_t P = (size_t)pr::mlp_params(), B = (size_t)max_batch, nb = (size_t)pr::mlp_backward_blocks(max_batch);
  struct {
    float** p;
    size_t n;
  } bufs[] = {{&m->theta, P}, {&m->m, P},      {&m->v, P},      {&m->grad, P},       {&m->X, 8 * B},
              {&m->T, 4 * B}, {&m->Y, 4 * B}, {&m->H1, 64 * B}, {&m->H2, 64 * B}, {&m->gpart, nb * P},
              {&m->lpart, nb}, {&m->loss, 1}};
  for (auto& b : bufs) {
    cudaError_t e = cudaMalloc((void**)b.p, sizeof(float) * b.n);
    if (e != cudaSuccess) {
      pr_mlp_destroy(m);
      return mfail(PR_ENOMEM, "pr_mlp_create: cudaMalloc failed");
    }
  }
  cudaError_t e = cudaMemcpyAsync(m->theta, params, sizeof(float) * P, cudaMemcpyDefault, m->stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(m->m, 0, sizeof(float) * P, m->stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(m->v, 0, sizeof(float) * P, m->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(m->stream);
  if (e != cudaSuccess) {
    pr_mlp_destroy(m);
    return mfail(PR_ECUDA, std::string("pr_mlp_create: ") + cudaGetErrorName(e));
  }
  *out = m;
  return PR_OK;
}

pr_status pr_mlp_forward(pr_mlp m, const float* X, int B, float* Y) {
  if (!m) return mfail(PR_ESTATE, "pr_mlp_forward: NULL model");
  if (!X || !Y || B < 1 || B > m->max_batch) return mfail(PR_EINVAL, "pr_mlp_forward: bad batch");
  cudaSetDevice(m->device);
  PM_CK(cudaMemcpyAsync(m->X, X, sizeof(float) * 8 * (size_t)B, cudaMemcpyDefault, m->stream));
  PM_CK(pr::mlp_forward(m->theta, m->X, B, m->Y, nullptr, nullptr, m->stream));
  PM_CK(cudaMemcpyAsync(Y, m->Y, sizeof(float) * 4 * (size_t)B, cudaMemcpyDefault, m->stream));
  PM_CK(cudaStreamSynchronize(m->stream));
  return PR_OK;
}

pr_status pr_mlp_loss_grad(pr_mlp m, const float* X, const float* T, int B, float* loss, float* grad) {
  return run_backward(m, X, T, B, false, 0.0f, loss, grad);
}

pr_status pr_mlp_adam_step(pr_mlp m, const float* X, const float* T, int B, float lr, float* loss) {
  if (!(lr > 0.0f)) return mfail(PR_EINVAL, "pr_mlp_adam_step: lr must be positive");
  return run_backward(m, X, T, B, true, lr, loss, nullptr);
}

pr_status pr_mlp_get_params(pr_mlp m, float* params) {
  if (!m) return mfail(PR_ESTATE, "pr_mlp_get_params: NULL model");
  if (!params) return mfail(PR_EINVAL, "pr_mlp_get_params: NULL output");
  cudaSetDevice(m->device);
  PM_CK(cudaMemcpyAsync(params, m->theta, sizeof(float) * pr::mlp_params(), cudaMemcpyDefault, m->stream));
  PM_CK(cudaStreamSynchronize(m->stream));
  return PR_OK;
}

}  // extern "C"
