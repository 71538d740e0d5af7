// Bandwidth-bound kernels of the iteration: input checks, the norms and initial guess of Eq. 3,
// identity shifts, symmetrisation, low-precision copies and the deterministic residual reduction.
#include "pr_internal.h"

#include <math.h>

namespace pr {
namespace {

constexpr int kThreads = 256;

__device__ __forceinline__ double warp_sum(double v) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}
// The larger of a and b, NaN if either is NaN (fmax would drop a NaN and hide a non-finite input).
__device__ __forceinline__ double nan_max(double a, double b) { return (a > b || a != a) ? a : b; }

__device__ __forceinline__ double warp_max(double v) {
  for (int o = 16; o > 0; o >>= 1) v = nan_max(v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;
}

// Non-negative doubles order like their bit patterns, so an integer atomicMax is an exact max.
__device__ __forceinline__ void atomic_max_nonneg(double* addr, double v) {
  atomicMax(reinterpret_cast<unsigned long long*>(addr), static_cast<unsigned long long>(__double_as_longlong(v)));
}

__global__ void k_validate(const double* __restrict__ A, int n, double* __restrict__ scal) {
  // scal[0] max|a|, scal[1] max|a_ij - a_ji|, scal[2] #non-finite, scal[3] #non-positive diagonal
  const int64_t total = (int64_t)n * n;
  double amax = 0.0, asym = 0.0, bad = 0.0, nonpos = 0.0;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    const int i = (int)(e / n), j = (int)(e % n);
    const double a = A[e];
    if (!isfinite(a)) { bad += 1.0; continue; }
    amax = fmax(amax, fabs(a));
    if (j > i) {
      const double t = A[(int64_t)j * n + i];
      if (isfinite(t)) asym = fmax(asym, fabs(a - t));
    }
    if (i == j && !(a > 0.0)) nonpos += 1.0;
  }
  amax = warp_max(amax);
  asym = warp_max(asym);
  bad = warp_sum(bad);
  nonpos = warp_sum(nonpos);
  if ((threadIdx.x & 31) == 0) {
    atomic_max_nonneg(scal + 0, amax);
    atomic_max_nonneg(scal + 1, asym);
    if (bad > 0) atomicAdd(scal + 2, bad);      // integer-valued counts: exact in any order
    if (nonpos > 0) atomicAdd(scal + 3, nonpos);
  }
}

// One warp per row: row abs-sums.
__global__ void k_abs_rowsum(const double* __restrict__ A, int n, double* __restrict__ rows) {
  const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
  if (warp >= n) return;
  const double* r = A + (int64_t)warp * n;
  double s = 0.0;
  for (int j = lane; j < n; j += 32) s += fabs(r[j]);
  s = warp_sum(s);
  if (lane == 0) rows[warp] = s;
}

// Column abs-sums: a 32-column stripe per block, 8 row groups, combined in a fixed order.
__global__ void k_abs_colsum(const double* __restrict__ A, int n, double* __restrict__ cols) {
  __shared__ double part[8][33];
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
  const int j = blockIdx.x * 32 + tx;
  double s = 0.0;
  if (j < n)
    for (int i = ty; i < n; i += 8) s += fabs(A[(int64_t)i * n + j]);
  part[ty][tx] = s;
  __syncthreads();
  if (ty == 0 && j < n) {
    double t = 0.0;
    for (int q = 0; q < 8; ++q) t += part[q][tx];
    cols[j] = t;
  }
}

// out[0] = max(cols), out[1] = max(rows); one block. A NaN sum (from a NaN entry of A) gives a NaN maximum.
__global__ void k_max2(const double* __restrict__ cols, const double* __restrict__ rows, int n, double* __restrict__ out) {
  __shared__ double sc[kThreads / 32], sr[kThreads / 32];
  double mc = 0.0, mr = 0.0;
  for (int i = threadIdx.x; i < n; i += blockDim.x) { mc = nan_max(mc, cols[i]); mr = nan_max(mr, rows[i]); }
  mc = warp_max(mc);
  mr = warp_max(mr);
  if ((threadIdx.x & 31) == 0) { sc[threadIdx.x >> 5] = mc; sr[threadIdx.x >> 5] = mr; }
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int w = 1; w < kThreads / 32; ++w) { mc = nan_max(mc, sc[w]); mr = nan_max(mr, sr[w]); }
    out[0] = nan_max(mc, sc[0]);
    out[1] = nan_max(mr, sr[0]);
  }
}

// Cholesky factorisation of every diagonal block of order 64 (the last one smaller), one block of 64
// threads each, in shared memory: a principal submatrix of an SPD matrix is SPD, so a pivot that is not
// positive shows that A is not. Right-looking, thread t owns row t of the lower triangle. Adds the number
// of failing blocks to *bad.
constexpr int kCholB = 64;
__global__ void __launch_bounds__(kCholB) k_diag_cholesky(const double* __restrict__ A, int n, double* __restrict__ bad) {
  __shared__ double L[kCholB][kCholB + 1];
  __shared__ int fail;
  const int b0 = blockIdx.x * kCholB, m = min(kCholB, n - b0), t = threadIdx.x;
  for (int i = 0; i < m; ++i)
    if (t < m) L[i][t] = A[(int64_t)(b0 + i) * n + b0 + t];
  if (t == 0) fail = 0;
  __syncthreads();
  for (int j = 0; j < m; ++j) {
    if (t == 0) {
      const double d = L[j][j];
      if (d > 0.0) L[j][j] = sqrt(d);
      else fail = 1;
    }
    __syncthreads();
    if (fail) break;  // uniform: read after the barrier
    if (t > j && t < m) L[t][j] /= L[j][j];
    __syncthreads();
    if (t > j && t < m) {
      const double lt = L[t][j];
      for (int k = j + 1; k <= t; ++k) L[t][k] -= lt * L[k][j];
    }
    __syncthreads();
  }
  if (t == 0 && fail) atomicAdd(bad, 1.0);
}

// X = A^T * inv_s through a 32 x 32 shared-memory transpose (coalesced on both sides).
__global__ void k_c0_eq3(const double* __restrict__ A, int n, double inv_s, double* __restrict__ X) {
  __shared__ double tile[32][33];
  const int bx = blockIdx.x * 32, by = blockIdx.y * 32;
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;  // 32 x 8 threads
  for (int r = ty; r < 32; r += 8) {
    const int i = by + r, j = bx + tx;  // read A[i][j]
    if (i < n && j < n) tile[r][tx] = A[(int64_t)i * n + j];
  }
  __syncthreads();
  for (int r = ty; r < 32; r += 8) {
    const int i = bx + r, j = by + tx;  // write X[i][j] = A[j][i]
    if (i < n && j < n) X[(int64_t)i * n + j] = tile[tx][r] * inv_s;
  }
}

__global__ void k_scaled_identity(double* __restrict__ X, int n, double c) {
  const int64_t total = (int64_t)n * n;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x)
    X[e] = (e / n == e % n) ? c : 0.0;
}

__global__ void k_axpby_identity(const double* __restrict__ in, int n, double a, double b, double* __restrict__ out) {
  const int64_t total = (int64_t)n * n;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x)
    out[e] = ((e / n == e % n) ? a : 0.0) + b * in[e];
}

// out = a x + b y element by element, as fma(a, x, b y) (one rounding when b y is exact). out may be x or y.
__global__ void k_lincomb(const double* x, const double* y, int64_t total, double a, double b, double* out) {
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x)
    out[e] = fma(a, x[e], b * y[e]);
}

// One warp per row: the first and last column with a non-zero entry (n and -1 for a zero row).
__global__ void k_row_spans(const double* __restrict__ A, int n, int* __restrict__ first, int* __restrict__ last) {
  const int i = blockIdx.x * 8 + (threadIdx.x >> 5), lane = threadIdx.x & 31;
  if (i >= n) return;
  int lo = n, hi = -1;
  for (int j = lane; j < n; j += 32)
    if (A[(int64_t)i * n + j] != 0.0) {
      lo = min(lo, j);
      hi = max(hi, j);
    }
  for (int o = 16; o > 0; o >>= 1) {
    lo = min(lo, __shfl_xor_sync(0xffffffffu, lo, o));
    hi = max(hi, __shfl_xor_sync(0xffffffffu, hi, o));
  }
  if (lane == 0) {
    first[i] = lo;
    last[i] = hi;
  }
}

__global__ void k_symmetrize(const double* __restrict__ in, int n, double* __restrict__ out) {
  __shared__ double tile[32][33];
  const int bx = blockIdx.x * 32, by = blockIdx.y * 32;
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
  for (int r = ty; r < 32; r += 8) {  // tile = in[bx.., by..] read as rows bx+r
    const int i = bx + r, j = by + tx;
    if (i < n && j < n) tile[r][tx] = in[(int64_t)i * n + j];
  }
  __syncthreads();
  for (int r = ty; r < 32; r += 8) {  // out[by + r][bx + tx] = (in[by+r][bx+tx] + in[bx+tx][by+r]) / 2
    const int i = by + r, j = bx + tx;
    if (i < n && j < n) out[(int64_t)i * n + j] = 0.5 * (in[(int64_t)i * n + j] + tile[tx][r]);
  }
}

__global__ void k_reduce_sqrt(const double* __restrict__ partial, int count, double* __restrict__ result) {
  __shared__ double sh[kReduceThreads];
  const double r = block_sum_sqrt(partial, count, sh);
  if (threadIdx.x == 0) *result = r;
}

// One block per segment: out[m] = sqrt(sum partial[begin[m]..end[m])) in a fixed order.
__global__ void k_seg_reduce_sqrt(const double* __restrict__ partial, const int* __restrict__ begin,
                                  const int* __restrict__ end, double* __restrict__ out) {
  __shared__ double sh[kReduceThreads];
  const int m = blockIdx.x;
  const double r = block_sum_sqrt(partial + begin[m], end[m] - begin[m], sh);
  if (threadIdx.x == 0) out[m] = r;
}

__global__ void k_to_bf16(const double* __restrict__ src, int n, int ldl, __nv_bfloat16* __restrict__ dst) {
  const int64_t total = (int64_t)n * n;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x)
    dst[(e / n) * ldl + (e % n)] = bf16_rne(src[e]);
}

int grid_for(int64_t total) {
  int64_t g = (total + kThreads - 1) / kThreads;
  if (g > 152 * 16) g = 152 * 16;
  if (g < 1) g = 1;
  return (int)g;
}

}  // namespace

cudaError_t validate(const double* A, int n, double* scal4, cudaStream_t s) {
  cudaError_t err = cudaMemsetAsync(scal4, 0, 4 * sizeof(double), s);
  if (err != cudaSuccess) return err;
  k_validate<<<grid_for((int64_t)n * n), kThreads, 0, s>>>(A, n, scal4);
  k_diag_cholesky<<<(n + kCholB - 1) / kCholB, kCholB, 0, s>>>(A, n, scal4 + 3);
  return cudaGetLastError();
}

cudaError_t abs_norms(const double* A, int n, double* work, double* out2, cudaStream_t s) {
  double* cols = work;
  double* rows = work + n;
  k_abs_colsum<<<(n + 31) / 32, 256, 0, s>>>(A, n, cols);
  k_abs_rowsum<<<(n * 32 + kThreads - 1) / kThreads, kThreads, 0, s>>>(A, n, rows);
  k_max2<<<1, kThreads, 0, s>>>(cols, rows, n, out2);
  return cudaGetLastError();
}

cudaError_t init_c0_eq3(const double* A, int n, double inv_s, double* X, cudaStream_t s) {
  dim3 grid((n + 31) / 32, (n + 31) / 32);
  k_c0_eq3<<<grid, 256, 0, s>>>(A, n, inv_s, X);
  return cudaGetLastError();
}

cudaError_t set_scaled_identity(double* X, int n, double c, cudaStream_t s) {
  k_scaled_identity<<<grid_for((int64_t)n * n), kThreads, 0, s>>>(X, n, c);
  return cudaGetLastError();
}

cudaError_t axpby_identity(const double* in, int n, double a, double b, double* out, cudaStream_t s) {
  k_axpby_identity<<<grid_for((int64_t)n * n), kThreads, 0, s>>>(in, n, a, b, out);
  return cudaGetLastError();
}

cudaError_t lincomb(const double* x, const double* y, int64_t total, double a, double b, double* out, cudaStream_t s) {
  k_lincomb<<<grid_for(total), kThreads, 0, s>>>(x, y, total, a, b, out);
  return cudaGetLastError();
}

cudaError_t row_spans(const double* A, int n, int* first, int* last, cudaStream_t s) {
  k_row_spans<<<(n + 7) / 8, 256, 0, s>>>(A, n, first, last);
  return cudaGetLastError();
}

cudaError_t symmetrize(const double* in, int n, double* out, cudaStream_t s) {
  dim3 grid((n + 31) / 32, (n + 31) / 32);
  k_symmetrize<<<grid, 256, 0, s>>>(in, n, out);
  return cudaGetLastError();
}

cudaError_t reduce_partials_sqrt(const double* partial, int count, double* result, cudaStream_t s) {
  k_reduce_sqrt<<<1, kReduceThreads, 0, s>>>(partial, count, result);
  return cudaGetLastError();
}

cudaError_t segmented_reduce_sqrt(const double* partial, const int* begin, const int* end, int count, double* out,
                                  cudaStream_t s) {
  if (count < 1) return cudaSuccess;
  k_seg_reduce_sqrt<<<count, kReduceThreads, 0, s>>>(partial, begin, end, out);
  return cudaGetLastError();
}

cudaError_t to_bf16(const double* src, int n, int ldl, __nv_bfloat16* dst, cudaStream_t s) {
  k_to_bf16<<<grid_for((int64_t)n * n), kThreads, 0, s>>>(src, n, ldl, dst);
  return cudaGetLastError();
}

}  // namespace pr
