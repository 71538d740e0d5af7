// The paper's custom-precision experiment on the GPU (Sec. 4.2, 4.3; Fig. 2): floating-point numbers with m
// stored mantissa bits (m + 1 significant bits) and FP64's exponent range, rounded to nearest with ties to
// even, used either for every arithmetic operation of the iteration ("arithmetic") or only for the input and
// the stored iterates ("storage"). An operation in the custom type is the FP64 operation followed by the
// rounding. The kernels here are FP64-ALU work: the experiment measures what the number format does to the
// iteration, and no tensor-core format offers an arbitrary mantissa width.
#include "pr_internal.h"

namespace pr {
namespace {

constexpr int kQT = 16;  // the rounded product: 16 x 16 outputs per block, one per thread

// x rounded to m stored mantissa bits (1 <= m <= 52), ties to even, on the FP64 bit pattern: the dropped
// 52 - m bits decide, a carry out of the mantissa moves into the exponent. Inf and NaN pass unchanged.
__device__ __forceinline__ double round_m(double x, int m) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(x);
  if (((b >> 52) & 0x7ffull) == 0x7ffull || m >= 52) return x;
  const int drop = 52 - m;
  const unsigned long long unit = 1ull << drop, rest = b & (unit - 1), half = unit >> 1;
  unsigned long long r = b & ~(unit - 1);
  if (rest > half || (rest == half && (r & unit))) r += unit;
  return __longlong_as_double((long long)r);
}

// P = X Y (n x n, row-major) in the m-bit arithmetic: P_ij = (((x_i0 y_0j) + x_i1 y_1j) + ...) with every
// product and every partial sum rounded, in the order k = 0, 1, ..., n - 1 (the shared-memory tiles keep it).
__global__ void __launch_bounds__(kQT * kQT) k_gemm_round(const double* __restrict__ X, const double* __restrict__ Y,
                                                         int n, int m, double* __restrict__ P) {
  __shared__ double xs[kQT][kQT + 1], ys[kQT][kQT + 1];
  const int tx = threadIdx.x, ty = threadIdx.y;
  const int i = blockIdx.y * kQT + ty, j = blockIdx.x * kQT + tx;
  double s = 0.0;
  for (int k0 = 0; k0 < n; k0 += kQT) {
    xs[ty][tx] = (i < n && k0 + tx < n) ? X[(int64_t)i * n + k0 + tx] : 0.0;
    ys[ty][tx] = (k0 + ty < n && j < n) ? Y[(int64_t)(k0 + ty) * n + j] : 0.0;
    __syncthreads();
    const int kend = min(kQT, n - k0);
    for (int kk = 0; kk < kend; ++kk) s = round_m(__dadd_rn(s, round_m(__dmul_rn(xs[ty][kk], ys[kk][tx]), m)), m);
    __syncthreads();
  }
  if (i < n && j < n) P[(int64_t)i * n + j] = s;
}

// W = (((p + 1) C - T) / p) one rounded operation at a time (out may be T).
__global__ void k_quant_update(const double* __restrict__ C, const double* T, int64_t total, int p, int m,
                               double* out) {
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    const double u = round_m(__dmul_rn((double)(p + 1), C[e]), m);
    const double v = round_m(__dsub_rn(u, T[e]), m);
    out[e] = round_m(__ddiv_rn(v, (double)p), m);
  }
}

// out = (W + W^T) / 2 with the sum rounded (the halving is exact); out != W.
__global__ void k_quant_sym(const double* __restrict__ W, int n, int m, double* __restrict__ out) {
  const int64_t total = (int64_t)n * n;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = e / n, j = e % n;
    out[e] = 0.5 * round_m(__dadd_rn(W[e], W[j * n + i]), m);
  }
}

__global__ void k_round(const double* x, int64_t total, int m, double* out) {
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x)
    out[e] = round_m(x[e], m);
}

// partial[b] = sum over rows 8 b .. 8 b + 7 of sum_j (delta_ij - T_ij)^2 (FP64; one warp per row, fixed order).
__global__ void k_resid_rows(const double* __restrict__ T, int n, double* __restrict__ partial) {
  __shared__ double w[8];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, i = blockIdx.x * 8 + wid;
  double s = 0.0;
  if (i < n)
    for (int j = lane; j < n; j += 32) {
      const double d = (i == j ? 1.0 : 0.0) - T[(int64_t)i * n + j];
      s = fma(d, d, s);
    }
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if (lane == 0) w[wid] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int q = 0; q < 8; ++q) t += w[q];
    partial[blockIdx.x] = t;
  }
}

int grid_for(int64_t total) {
  int64_t g = (total + 255) / 256;
  return (int)(g < 1 ? 1 : (g > 152 * 16 ? 152 * 16 : g));
}

}  // namespace

cudaError_t gemm_round(const double* X, const double* Y, int n, int m, double* P, cudaStream_t s) {
  if (m < 1 || m > 52) return cudaErrorInvalidValue;
  dim3 grid((n + kQT - 1) / kQT, (n + kQT - 1) / kQT), block(kQT, kQT);
  k_gemm_round<<<grid, block, 0, s>>>(X, Y, n, m, P);
  return cudaGetLastError();
}

cudaError_t quant_update(const double* C, const double* T, int n, int p, int m, double* out, cudaStream_t s) {
  const int64_t total = (int64_t)n * n;
  k_quant_update<<<grid_for(total), 256, 0, s>>>(C, T, total, p, m, out);
  return cudaGetLastError();
}

cudaError_t quant_sym(const double* W, int n, int m, double* out, cudaStream_t s) {
  k_quant_sym<<<grid_for((int64_t)n * n), 256, 0, s>>>(W, n, m, out);
  return cudaGetLastError();
}

cudaError_t round_values(const double* x, int64_t total, int m, double* out, cudaStream_t s) {
  if (m < 1 || m > 52) return cudaErrorInvalidValue;
  k_round<<<grid_for(total), 256, 0, s>>>(x, total, m, out);
  return cudaGetLastError();
}

int resid_row_partials(int n) { return (n + 7) / 8; }

cudaError_t resid_rows(const double* T, int n, double* partial, cudaStream_t s) {
  k_resid_rows<<<resid_row_partials(n), 256, 0, s>>>(T, n, partial);
  return cudaGetLastError();
}

}  // namespace pr
