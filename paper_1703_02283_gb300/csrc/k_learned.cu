// Kernels of the learned polynomial initial guess: trace features of A, the polynomial C_0, the power
// iteration that checks Eq. 2 for it, and the small MLP (8 -> 64 -> 64 -> 4, ReLU, FP32) that predicts the
// polynomial's coefficients, with its backward pass and Adam update. All reductions run in a fixed order.
#include "pr_internal.h"

#include <math.h>

namespace pr {
namespace {

constexpr int kThreads = 256;

__device__ __forceinline__ double warp_sum_d(double v) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

int blocks_for(int64_t total) {
  int64_t g = (total + kThreads - 1) / kThreads;
  if (g > 152 * 8) g = 152 * 8;
  return g < 1 ? 1 : (int)g;
}

// partial[block] = sum over the block's grid-stride share of X_ij Y_ij (fixed order within the block).
__global__ void k_dot_partial(const double* __restrict__ X, const double* __restrict__ Y, int64_t total,
                              double* __restrict__ partial) {
  __shared__ double sh[kThreads / 32];
  double s = 0.0;
  for (int64_t e = (int64_t)blockIdx.x * kThreads + threadIdx.x; e < total; e += (int64_t)gridDim.x * kThreads)
    s = fma(X[e], Y[e], s);
  s = warp_sum_d(s);
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < kThreads / 32; ++w) t += sh[w];
    partial[blockIdx.x] = t;
  }
}

__global__ void k_trace_partial(const double* __restrict__ X, int n, double* __restrict__ partial) {
  __shared__ double sh[kThreads / 32];
  double s = 0.0;
  for (int i = blockIdx.x * kThreads + threadIdx.x; i < n; i += gridDim.x * kThreads) s += X[(int64_t)i * n + i];
  s = warp_sum_d(s);
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < kThreads / 32; ++w) t += sh[w];
    partial[blockIdx.x] = t;
  }
}

__global__ void k_sum(const double* __restrict__ partial, int count, double* __restrict__ out) {
  __shared__ double sh[kThreads];
  double s = 0.0;
  for (int i = threadIdx.x; i < count; i += kThreads) s += partial[i];
  sh[threadIdx.x] = s;
  __syncthreads();
  for (int w = kThreads / 2; w > 0; w >>= 1) {
    if (threadIdx.x < w) sh[threadIdx.x] += sh[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) *out = sh[0];
}

// X = a0 I + a1 A + a2 P2 + a3 P3.
__global__ void k_poly(const double* __restrict__ A, const double* __restrict__ P2, const double* __restrict__ P3, int n,
                       double a0, double a1, double a2, double a3, double* __restrict__ X) {
  const int64_t total = (int64_t)n * n;
  for (int64_t e = (int64_t)blockIdx.x * kThreads + threadIdx.x; e < total; e += (int64_t)gridDim.x * kThreads) {
    double v = fma(a3, P3[e], fma(a2, P2[e], a1 * A[e]));
    if (e / n == e % n) v += a0;
    X[e] = v;
  }
}

// y = M x for a row-major n x n M: one warp per row.
__global__ void k_gemv(const double* __restrict__ M, int n, const double* __restrict__ x, double* __restrict__ y) {
  const int row = (blockIdx.x * kThreads + threadIdx.x) >> 5, lane = threadIdx.x & 31;
  if (row >= n) return;
  const double* r = M + (int64_t)row * n;
  double s = 0.0;
  for (int j = lane; j < n; j += 32) s = fma(r[j], x[j], s);
  s = warp_sum_d(s);
  if (lane == 0) y[row] = s;
}

// w = v - u; partial sums of w^2 (block-level, fixed order).
__global__ void k_sub_norm(const double* __restrict__ v, const double* __restrict__ u, int n, double* __restrict__ w,
                           double* __restrict__ partial) {
  __shared__ double sh[kThreads / 32];
  double s = 0.0;
  for (int i = blockIdx.x * kThreads + threadIdx.x; i < n; i += gridDim.x * kThreads) {
    const double d = v[i] - u[i];
    w[i] = d;
    s = fma(d, d, s);
  }
  s = warp_sum_d(s);
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int q = 0; q < kThreads / 32; ++q) t += sh[q];
    partial[blockIdx.x] = t;
  }
}

// v = w / sqrt(*ss); the estimate est = sqrt(*ss) (the norm of B v for the previous unit v).
__global__ void k_normalize(const double* __restrict__ w, int n, const double* __restrict__ ss, double* __restrict__ v,
                            double* __restrict__ est) {
  const double nrm = sqrt(*ss);
  const double inv = nrm > 0.0 ? 1.0 / nrm : 0.0;
  for (int i = blockIdx.x * kThreads + threadIdx.x; i < n; i += gridDim.x * kThreads) v[i] = w[i] * inv;
  if (blockIdx.x == 0 && threadIdx.x == 0) *est = nrm;
}

__global__ void k_start_vector(int n, double* __restrict__ v) {
  const double scale = 1.0 / sqrt((double)n * 1.125);
  for (int i = blockIdx.x * kThreads + threadIdx.x; i < n; i += gridDim.x * kThreads)
    v[i] = (1.0 + 0.5 * sin(1.0 + (double)i)) * scale;  // deterministic, touches every eigenvector
}

// ------------------------------------------------------------------------------------------------ MLP
// Flat FP32 parameters: W1 (64 x 8), b1 (64), W2 (64 x 64), b2 (64), W3 (4 x 64), b3 (4).
constexpr int IN = 8, H = 64, OUT = 4;
constexpr int OW1 = 0, OB1 = OW1 + H * IN, OW2 = OB1 + H, OB2 = OW2 + H * H, OW3 = OB2 + H, OB3 = OW3 + OUT * H;
constexpr int NPARAM = OB3 + OUT;
constexpr int SB = 64;  // samples per block in the backward pass

// One thread per sample; parameters staged in shared memory. H1, H2 may be null (inference).
__global__ void k_mlp_forward(const float* __restrict__ theta, const float* __restrict__ X, int B, float* __restrict__ Y,
                              float* __restrict__ H1, float* __restrict__ H2) {
  __shared__ float th[NPARAM];
  for (int i = threadIdx.x; i < NPARAM; i += blockDim.x) th[i] = theta[i];
  __syncthreads();
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= B) return;
  float x[IN], h1[H];
  for (int i = 0; i < IN; ++i) x[i] = X[(int64_t)b * IN + i];
  for (int j = 0; j < H; ++j) {
    float a = th[OB1 + j];
    for (int i = 0; i < IN; ++i) a = fmaf(th[OW1 + j * IN + i], x[i], a);
    h1[j] = fmaxf(a, 0.0f);
    if (H1) H1[(int64_t)b * H + j] = h1[j];
  }
  float y[OUT];
  for (int k = 0; k < OUT; ++k) y[k] = th[OB3 + k];
  for (int j = 0; j < H; ++j) {
    float a = th[OB2 + j];
    for (int i = 0; i < H; ++i) a = fmaf(th[OW2 + j * H + i], h1[i], a);
    const float h2 = fmaxf(a, 0.0f);
    if (H2) H2[(int64_t)b * H + j] = h2;
    for (int k = 0; k < OUT; ++k) y[k] = fmaf(th[OW3 + k * H + j], h2, y[k]);
  }
  for (int k = 0; k < OUT; ++k) Y[(int64_t)b * OUT + k] = y[k];
}

// Per block of SB samples: loss partial and the block's gradient partial (every parameter summed over the
// block's samples in order). scale = 2 / (B * OUT) (the mean squared error's derivative).
__global__ void k_mlp_backward(const float* __restrict__ theta, const float* __restrict__ X, const float* __restrict__ T,
                               const float* __restrict__ Y, const float* __restrict__ H1, const float* __restrict__ H2,
                               int B, float scale, float* __restrict__ gpart, float* __restrict__ lpart) {
  extern __shared__ float sm[];
  float* x = sm;                 // SB x IN
  float* h1 = x + SB * IN;       // SB x H
  float* h2 = h1 + SB * H;       // SB x H
  float* d2 = h2 + SB * H;       // SB x H  (dL/dA2)
  float* d1 = d2 + SB * H;       // SB x H  (dL/dA1)
  float* dy = d1 + SB * H;       // SB x OUT
  float* w2 = dy + SB * OUT;     // H x H
  float* w3 = w2 + H * H;        // OUT x H
  float* red = w3 + OUT * H;     // blockDim
  const int b0 = blockIdx.x * SB, nb = min(SB, B - b0);
  for (int i = threadIdx.x; i < H * H; i += blockDim.x) w2[i] = theta[OW2 + i];
  for (int i = threadIdx.x; i < OUT * H; i += blockDim.x) w3[i] = theta[OW3 + i];
  for (int i = threadIdx.x; i < SB * IN; i += blockDim.x) x[i] = i < nb * IN ? X[(int64_t)b0 * IN + i] : 0.0f;
  for (int i = threadIdx.x; i < SB * H; i += blockDim.x) {
    h1[i] = i < nb * H ? H1[(int64_t)b0 * H + i] : 0.0f;
    h2[i] = i < nb * H ? H2[(int64_t)b0 * H + i] : 0.0f;
  }
  float lsum = 0.0f;
  for (int i = threadIdx.x; i < SB * OUT; i += blockDim.x) {
    float d = 0.0f;
    if (i < nb * OUT) {
      d = Y[(int64_t)b0 * OUT + i] - T[(int64_t)b0 * OUT + i];
      lsum = fmaf(d, d, lsum);
    }
    dy[i] = scale * d;
  }
  red[threadIdx.x] = lsum;
  __syncthreads();
  for (int i = threadIdx.x; i < SB * H; i += blockDim.x) {  // dA2 = (dY W3) * [A2 > 0]
    const int b = i / H, j = i % H;
    float a = 0.0f;
    for (int k = 0; k < OUT; ++k) a = fmaf(dy[b * OUT + k], w3[k * H + j], a);
    d2[i] = h2[i] > 0.0f ? a : 0.0f;
  }
  __syncthreads();
  for (int i = threadIdx.x; i < SB * H; i += blockDim.x) {  // dA1 = (dA2 W2) * [A1 > 0]
    const int b = i / H, j = i % H;
    float a = 0.0f;
    for (int k = 0; k < H; ++k) a = fmaf(d2[b * H + k], w2[k * H + j], a);
    d1[i] = h1[i] > 0.0f ? a : 0.0f;
  }
  __syncthreads();
  float* g = gpart + (int64_t)blockIdx.x * NPARAM;
  for (int q = threadIdx.x; q < NPARAM; q += blockDim.x) {
    float a = 0.0f;
    if (q < OB1) {
      const int j = q / IN, i = q % IN;
      for (int b = 0; b < SB; ++b) a = fmaf(d1[b * H + j], x[b * IN + i], a);
    } else if (q < OW2) {
      const int j = q - OB1;
      for (int b = 0; b < SB; ++b) a += d1[b * H + j];
    } else if (q < OB2) {
      const int j = (q - OW2) / H, i = (q - OW2) % H;
      for (int b = 0; b < SB; ++b) a = fmaf(d2[b * H + j], h1[b * H + i], a);
    } else if (q < OW3) {
      const int j = q - OB2;
      for (int b = 0; b < SB; ++b) a += d2[b * H + j];
    } else if (q < OB3) {
      const int k = (q - OW3) / H, j = (q - OW3) % H;
      for (int b = 0; b < SB; ++b) a = fmaf(dy[b * OUT + k], h2[b * H + j], a);
    } else {
      const int k = q - OB3;
      for (int b = 0; b < SB; ++b) a += dy[b * OUT + k];
    }
    g[q] = a;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    float t = 0.0f;
    for (int i = 0; i < (int)blockDim.x; ++i) t += red[i];
    lpart[blockIdx.x] = t;
  }
}

// grad[q] = sum over blocks (in order) of gpart; loss = sum lpart / (B OUT); optional Adam update.
__global__ void k_mlp_reduce_adam(const float* __restrict__ gpart, const float* __restrict__ lpart, int nblocks, int B,
                                  float* __restrict__ grad, float* __restrict__ loss, float* __restrict__ theta,
                                  float* __restrict__ m, float* __restrict__ v, float lr, float c1, float c2, int adam) {
  const int q = blockIdx.x * blockDim.x + threadIdx.x;
  if (q == 0) {
    float t = 0.0f;
    for (int b = 0; b < nblocks; ++b) t += lpart[b];
    *loss = t / (float)(B * OUT);
  }
  if (q >= NPARAM) return;
  float gq = 0.0f;
  for (int b = 0; b < nblocks; ++b) gq += gpart[(int64_t)b * NPARAM + q];
  grad[q] = gq;
  if (adam) {
    const float beta1 = 0.9f, beta2 = 0.999f, eps = 1e-8f;
    const float mq = beta1 * m[q] + (1.0f - beta1) * gq;
    const float vq = beta2 * v[q] + (1.0f - beta2) * gq * gq;
    m[q] = mq;
    v[q] = vq;
    theta[q] -= lr * (mq / c1) / (sqrtf(vq / c2) + eps);
  }
}

}  // namespace

int mlp_params() { return NPARAM; }

cudaError_t frobenius_dot(const double* X, const double* Y, int64_t total, double* work, double* out, cudaStream_t s) {
  const int nb = blocks_for(total);
  k_dot_partial<<<nb, kThreads, 0, s>>>(X, Y, total, work);
  k_sum<<<1, kThreads, 0, s>>>(work, nb, out);
  return cudaGetLastError();
}

cudaError_t trace(const double* X, int n, double* work, double* out, cudaStream_t s) {
  const int nb = blocks_for(n);
  k_trace_partial<<<nb, kThreads, 0, s>>>(X, n, work);
  k_sum<<<1, kThreads, 0, s>>>(work, nb, out);
  return cudaGetLastError();
}

cudaError_t poly_combine(const double* A, const double* P2, const double* P3, int n, const double a[4], double* X,
                         cudaStream_t s) {
  k_poly<<<blocks_for((int64_t)n * n), kThreads, 0, s>>>(A, P2, P3, n, a[0], a[1], a[2], a[3], X);
  return cudaGetLastError();
}

cudaError_t gemv(const double* M, int n, const double* x, double* y, cudaStream_t s) {
  k_gemv<<<(n * 32 + kThreads - 1) / kThreads, kThreads, 0, s>>>(M, n, x, y);
  return cudaGetLastError();
}

cudaError_t power_start(int n, double* v, cudaStream_t s) {
  k_start_vector<<<blocks_for(n), kThreads, 0, s>>>(n, v);
  return cudaGetLastError();
}

cudaError_t power_finish_step(const double* v, const double* u, int n, double* w, double* work, double* ss, double* vout,
                              double* est, cudaStream_t s) {
  const int nb = blocks_for(n);
  k_sub_norm<<<nb, kThreads, 0, s>>>(v, u, n, w, work);
  k_sum<<<1, kThreads, 0, s>>>(work, nb, ss);
  k_normalize<<<nb, kThreads, 0, s>>>(w, n, ss, vout, est);
  return cudaGetLastError();
}

int mlp_backward_blocks(int B) { return (B + SB - 1) / SB; }

cudaError_t mlp_forward(const float* theta, const float* X, int B, float* Y, float* H1, float* H2, cudaStream_t s) {
  if (B < 1) return cudaSuccess;
  k_mlp_forward<<<(B + 127) / 128, 128, 0, s>>>(theta, X, B, Y, H1, H2);
  return cudaGetLastError();
}

cudaError_t mlp_backward(const float* theta, const float* X, const float* T, const float* Y, const float* H1,
                         const float* H2, int B, float* gpart, float* lpart, float* grad, float* loss, float* m,
                         float* v, float* theta_rw, float lr, float c1, float c2, bool adam, cudaStream_t s) {
  const int nb = mlp_backward_blocks(B);
  const size_t smem = sizeof(float) * (SB * IN + 4 * SB * H + SB * OUT + H * H + OUT * H + 256);
  static bool attr = false;
  if (!attr) {
    cudaError_t e = cudaFuncSetAttribute(k_mlp_backward, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    attr = true;
  }
  k_mlp_backward<<<nb, 256, smem, s>>>(theta, X, T, Y, H1, H2, B, 2.0f / (float)(B * OUT), gpart, lpart);
  k_mlp_reduce_adam<<<(NPARAM + 255) / 256, 256, 0, s>>>(gpart, lpart, nb, B, grad, loss, theta_rw, m, v, lr, c1, c2,
                                                          adam ? 1 : 0);
  return cudaGetLastError();
}

}  // namespace pr
