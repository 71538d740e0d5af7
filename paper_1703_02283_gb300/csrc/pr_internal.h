// Internal declarations shared by the library's translation units (not part of the ABI).
#pragma once

#include <cuda_runtime.h>
#include <cuda_bf16.h>
#include <stdint.h>

#include "../../include/pthroot.h"

namespace pr {

// Fused epilogue of one matrix product P = X Y, applied to every computed element (i, j). In symmetric
// mode only elements with i <= j are computed and each is also stored at (j, i).
//   out [i, j]  = P_ij                                    (if out != nullptr)
//   out2[i, j]  = a * delta_ij + b * P_ij + c * cin[i, j]  (if out2 != nullptr)
//   partial[t] += w_ij * (delta_ij - P_ij)^2 over the tile t (if partial != nullptr), w_ij = 2 for a mirrored
//                 off-diagonal element, 1 otherwise, so that the partials sum to ||I - P||_F^2.
//   out_lp / out2_lp: BF16 copies of out / out2 (operands of the next low-precision product).
struct Epilogue {
  double* out = nullptr;
  double* out2 = nullptr;
  const double* cin = nullptr;
  double a = 0.0, b = 0.0, c = 0.0;
  double* partial = nullptr;
  __nv_bfloat16* out_lp = nullptr;
  __nv_bfloat16* out2_lp = nullptr;
};

enum class Mode { Sym, Full };

// Round-to-nearest-even conversion of a double to BF16 through round-to-odd FP32 (Boldo and Melquiond,
// "Emulation of FMA and correctly rounded sums: proved algorithms using rounding to odd", IEEE TC 2008):
// rounding to odd at 24 bits and then to nearest at 8 bits equals rounding to nearest at 8 bits directly.
__device__ __forceinline__ __nv_bfloat16 bf16_rne(double x) {
  float f = __double2float_rz(x);
  unsigned int u = __float_as_uint(f);
  if ((double)f != x && (u & 0x7f800000u) != 0x7f800000u) u |= 1u;  // sticky bit: round to odd
  if ((u & 0x7f800000u) == 0x7f800000u) {                               // Inf / NaN: keep, quiet NaN
    const unsigned short h = (unsigned short)(u >> 16) | ((u & 0x007fffffu) ? 0x40u : 0u);
    return __ushort_as_bfloat16(h);
  }
  u += 0x7fffu + ((u >> 16) & 1u);  // nearest even at 8 significant bits
  return __ushort_as_bfloat16((unsigned short)(u >> 16));
}
__device__ __forceinline__ __nv_bfloat16 bf16_rne(float x) { return bf16_rne((double)x); }

// ---- FP64 products (k_gemm_f64.cu): P = X Y for n x n row-major X, Y.
// Returns the number of tiles (= entries written to e.partial).
int gemm_f64_tiles(int n, Mode mode);
cudaError_t gemm_f64(const double* X, const double* Y, int n, Mode mode, const Epilogue& e, cudaStream_t s);

// ---- BF16 tensor-core products (k_gemm_tc.cu): P = X Y^T for BF16 X, Y (n x n, leading dimension ldl,
// a multiple of 8, 16-byte aligned), FP32 accumulation; transpose (full mode only) stores P^T.
// err: device word set to a non-zero code if a bounded wait expired.
int gemm_tc_tiles(int n, Mode mode);
int bf16_ld(int n);
cudaError_t gemm_bf16_tc(const __nv_bfloat16* X, const __nv_bfloat16* Y, int n, int ldl, Mode mode, bool transpose,
                         const Epilogue& e, int* err, cudaStream_t s);

// ---- elementwise and reductions (k_elementwise.cu)
// scal[0] = max |a_ij|, scal[1] = max |a_ij - a_ji|, scal[2] = #non-finite, scal[3] = #non-positive diagonal
cudaError_t validate(const double* A, int n, double* scal4, cudaStream_t s);
// out[0] = ||A||_1 (max column abs-sum), out[1] = ||A||_inf (max row abs-sum); work: 2n doubles
cudaError_t abs_norms(const double* A, int n, double* work, double* out2, cudaStream_t s);
// X = A^T * inv_s (Eq. 3)
cudaError_t init_c0_eq3(const double* A, int n, double inv_s, double* X, cudaStream_t s);
// X = c * I
cudaError_t set_scaled_identity(double* X, int n, double c, cudaStream_t s);
// out = a * I + b * in
cudaError_t axpby_identity(const double* in, int n, double a, double b, double* out, cudaStream_t s);
// out = (in + in^T) / 2 (out != in)
cudaError_t symmetrize(const double* in, int n, double* out, cudaStream_t s);
// *result = sqrt(sum of partial[0..count)) in a fixed order
cudaError_t reduce_partials_sqrt(const double* partial, int count, double* result, cudaStream_t s);
// dst[i * ldl + j] = bf16(src[i * n + j]) for an n x n matrix
cudaError_t to_bf16(const double* src, int n, int ldl, __nv_bfloat16* dst, cudaStream_t s);

// Records the text returned by pr_last_error(NULL) for a failing call that has no handle.
void set_handleless_error(const char* msg);

}  // namespace pr
