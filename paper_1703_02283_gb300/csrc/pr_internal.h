// Internal declarations shared by the library's translation units (not part of the ABI).
#pragma once

#include <cuda_runtime.h>
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <math.h>
#include <stdint.h>

#include <vector>

#include "../../include/pthroot.h"

#include <nvtx3/nvToolsExt.h>

namespace pr {

// An NVTX range for the scope of the object (tracing tools show the library's iterations, products and
// batch solves on the host timeline; without a tool attached a push/pop costs a few nanoseconds).
struct NvtxRange {
  explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
  ~NvtxRange() { nvtxRangePop(); }
  NvtxRange(const NvtxRange&) = delete;
  NvtxRange& operator=(const NvtxRange&) = delete;
};

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

// Round-to-nearest-even conversions to BF16 (8 significant bits), in integer arithmetic: the FP64 units of
// GB300 are far too slow to sit in an epilogue.
__device__ __forceinline__ __nv_bfloat16 bf16_rne(float x) {
  unsigned int u = __float_as_uint(x);
  if ((u & 0x7f800000u) == 0x7f800000u)  // Inf / NaN (NaN kept quiet)
    return __ushort_as_bfloat16((unsigned short)((u >> 16) | ((u & 0x007fffffu) ? 0x40u : 0u)));
  u += 0x7fffu + ((u >> 16) & 1u);  // ties to even on the 16 dropped bits; a carry moves into the exponent
  return __ushort_as_bfloat16((unsigned short)(u >> 16));
}

// From FP64 in one rounding: keep the top 7 of the 52 stored mantissa bits and round on the other 45.
// Values outside the normal FP32 exponent range (zero, subnormal, huge, Inf, NaN) go through round-to-odd
// FP32 (Boldo and Melquiond, IEEE TC 2008), which also rounds once.
__device__ __forceinline__ __nv_bfloat16 bf16_rne(double x) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(x);
  const int e = (int)((b >> 52) & 0x7ffu);
  if (e >= 1023 - 126 && e <= 1023 + 127) {
    const unsigned long long m = b & 0xfffffffffffffull;
    const unsigned long long rest = m & ((1ull << 45) - 1), half = 1ull << 44;
    unsigned int v = ((unsigned int)(e - 1023 + 127) << 7) | (unsigned int)(m >> 45);
    if (rest > half || (rest == half && (v & 1u))) v += 1u;  // a carry into the exponent is correct
    return __ushort_as_bfloat16((unsigned short)(((unsigned int)(b >> 63) << 15) | v));
  }
  float f = __double2float_rz(x);
  unsigned int u = __float_as_uint(f);
  if ((double)f != x && (u & 0x7f800000u) != 0x7f800000u) u |= 1u;
  return bf16_rne(__uint_as_float(u));
}

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
// ---- FP8 (E4M3) tensor-core products (k_gemm_tc.cu): X = 2^sx_i Q_X, Y = 2^sy_j Q_Y row by row, Q n x n bytes
// with leading dimension ldq = fp8_ld(n) (a multiple of 16); P = X Y^T with FP32 accumulation, FP64 outputs
// only (the epilogue's out / out2 / partial; out_lp / out2_lp must be null). to_fp8: Q and sx of an FP64
// matrix (per row: s_i = exponent of its largest |x| - 7, then E4M3 round-to-nearest-even of x 2^-s_i).
int fp8_ld(int n);
cudaError_t to_fp8(const double* X, int n, int ldq, uint8_t* Q, int* sx, cudaStream_t s);
cudaError_t gemm_fp8_tc(const uint8_t* X, const int* sx, const uint8_t* Y, const int* sy, int n, int ldq, Mode mode,
                        bool transpose, const Epilogue& e, int* err, cudaStream_t s);

// ---- FP64-accurate products from exact FP16 digit slices (k_gemm_emu.cu).
// slice(): X (n x n FP64) -> 8 digit planes D (layout [row][k / 16][plane][k % 16], n x 8 ldl FP16 with
// ldl = emu_ld(n); planes >= S zero) and row exponents ex.
// gemm_emu(): P = X Y^T from the slices of X and Y over the work items (emu_launch_list), FP64 epilogue
// (out / out2 / partial; no BF16 copies). One residual partial per epilogue warp and tile
// (emu_partials_per_item() per tile, in tile order, also when tiles are split).
// Tiles are 128 rows x bn columns, bn = 96 (the default) or 48 (emu_tile_width_ok); the work items of a
// launch must be built for the bn it runs with.
// emu_tile_list(): appends the work items (m, tile row, tile column, 0) of matrix m (order n) in the
// kernel's order; symmetric mode keeps the tiles reaching the upper triangle.
bool emu_tile_width_ok(int bn);
void emu_tile_list(int m, int n, Mode mode, std::vector<int4>& out, int bn = 96);
int emu_tile_count(int n, Mode mode, int bn = 96);
// The work list of one single-matrix product: emu_tile_list, with every tile split over K into two items
// (emu_split_slots tiles; 0: not split) when split > 0, never when split == 0, and when that shortens the
// launch (ceil(2T / G) < 2 ceil(T / G) on G SMs) when split < 0. A split launch needs
// emu_split_bytes(slots) bytes of exact half totals and emu_split_counters(slots) ints, zero before the
// first launch (the kernel leaves them zero).
void emu_launch_list(int n, Mode mode, std::vector<int4>& out, int bn = 96, int split = -1);
int emu_split_slots(int n, Mode mode, int bn = 96, int split = -1);
bool emu_split_useful(int n, Mode mode, int bn);  // at least 2 K steps and fewer than 4 waves of tiles
// An unsplit item (from emu_tile_list) restricted to the K steps [j0, j1), 0 <= j0 < j1 <= KS < 65536: the
// steps left out must hold zero digits in the operand rows of the tile (a block-sparse operand).
int4 emu_range_item(int4 item, int j0, int j1);
size_t emu_split_bytes(int slots);
size_t emu_split_counters(int slots);
int emu_tiles(int n, Mode mode, int bn = 96);  // residual partials of one product: tiles * emu_partials_per_item
int emu_partials_per_item();
int emu_max_slices();
int emu_ld(int K);  // the K extent of a digit-plane row: K rounded up to 16
size_t emu_scratch_bytes();  // device scratch each gemm_emu / gemm_emu_batched call needs (per stream)
cudaError_t emu_prepare();   // one-time kernel attributes and driver entry points (before a graph capture)
cudaError_t slice(const double* X, int n, int ldl, int S, __half* D, int* ex, cudaStream_t s);
// Slices R rows of an FP64 array with leading dimension ldx; row r has row_n[r] valid columns (n if null).
cudaError_t slice_rows(const double* X, int R, int n, int ldx, int ldl, int S, const int* row_n, __half* D, int* ex,
                       cudaStream_t s);
cudaError_t gemm_emu(const __half* DX, const int* ex, const __half* DY, const int* ey, int n, int ldl, int S, Mode mode,
                     bool transpose, const int4* items, int nitems, const Epilogue& e, long long* scratch,
                     long long* split, int* split_cnt, int* err, cudaStream_t s, int bn = 96);

// A batch of matrices packed row-wise in shared buffers (leading dimension ld for FP64, ldl for digit
// planes; R packed rows per plane; K the largest order). Work items from emu_tile_list per matrix;
// per-matrix record = {order, first packed row, epilogue a, b, c}. nitems_dev (if set): the number of
// items is read on the device (the launch is one persistent CTA per SM). tstamp (if set): the kernel
// folds its start and end times (ns, %globaltimer) into tstamp[0] (min) and tstamp[1] (max).
struct EmuBatchMat {
  int n, row0;
  double a, b, c;
};
cudaError_t gemm_emu_batched(const __half* DX, const int* ex, const __half* DY, const int* ey, int R, int K, int ldl,
                             int ld, int S, Mode mode, bool transpose, const int4* items, int nitems,
                             const int* nitems_dev, const EmuBatchMat* mats, const Epilogue& e, long long* scratch,
                             int* err, unsigned long long* tstamp, cudaStream_t s, int bn = 96);

// ---- the custom-precision experiment (k_quant.cu): m stored mantissa bits, round to nearest even
// gemm_round: P = X Y with every product and partial sum rounded (order k = 0, 1, ...); quant_update:
// out = (((p + 1) C - T) / p) one rounded operation at a time (out may be T); quant_sym: out = rnd(W + W^T) / 2;
// round_values: out = rnd(x) (out may be x); resid_rows: per 8 rows the FP64 sum of (delta_ij - T_ij)^2
// (resid_row_partials(n) values).
cudaError_t gemm_round(const double* X, const double* Y, int n, int m, double* P, cudaStream_t s);
cudaError_t quant_update(const double* C, const double* T, int n, int p, int m, double* out, cudaStream_t s);
cudaError_t quant_sym(const double* W, int n, int m, double* out, cudaStream_t s);
cudaError_t round_values(const double* x, int64_t total, int m, double* out, cudaStream_t s);
int resid_row_partials(int n);
cudaError_t resid_rows(const double* T, int n, double* partial, cudaStream_t s);

// ---- elementwise and reductions (k_elementwise.cu)
// scal[0] = max |a_ij|, scal[1] = max |a_ij - a_ji|, scal[2] = #non-finite, scal[3] = #non-positive diagonal
// entries + #diagonal blocks of order 64 without a Cholesky factorisation (A not positive definite if > 0)
cudaError_t validate(const double* A, int n, double* scal4, cudaStream_t s);
// out[0] = ||A||_1 (max column abs-sum), out[1] = ||A||_inf (max row abs-sum); work: 2n doubles
cudaError_t abs_norms(const double* A, int n, double* work, double* out2, cudaStream_t s);
// X = A^T * inv_s (Eq. 3)
cudaError_t init_c0_eq3(const double* A, int n, double inv_s, double* X, cudaStream_t s);
// X = c * I
cudaError_t set_scaled_identity(double* X, int n, double c, cudaStream_t s);
// out = a * I + b * in
cudaError_t axpby_identity(const double* in, int n, double a, double b, double* out, cudaStream_t s);
// out[e] = fma(a, x[e], b y[e]) for e < total (out may alias x or y)
cudaError_t lincomb(const double* x, const double* y, int64_t total, double a, double b, double* out, cudaStream_t s);
// first[i] / last[i] = the smallest / largest j with A_ij != 0 (n and -1 for a zero row)
cudaError_t row_spans(const double* A, int n, int* first, int* last, cudaStream_t s);
// out = (in + in^T) / 2 (out != in)
cudaError_t symmetrize(const double* in, int n, double* out, cudaStream_t s);
// *result = sqrt(sum of partial[0..count)) in a fixed order
cudaError_t reduce_partials_sqrt(const double* partial, int count, double* result, cudaStream_t s);
// dst[i * ldl + j] = bf16(src[i * n + j]) for an n x n matrix
cudaError_t to_bf16(const double* src, int n, int ldl, __nv_bfloat16* dst, cudaStream_t s);

// ---- learned initial guess (k_learned.cu)
int mlp_params();
int mlp_backward_blocks(int B);
cudaError_t frobenius_dot(const double* X, const double* Y, int64_t total, double* work, double* out, cudaStream_t s);
cudaError_t trace(const double* X, int n, double* work, double* out, cudaStream_t s);
cudaError_t poly_combine(const double* A, const double* P2, const double* P3, int n, const double a[4], double* X,
                         cudaStream_t s);
cudaError_t gemv(const double* M, int n, const double* x, double* y, cudaStream_t s);
cudaError_t power_start(int n, double* v, cudaStream_t s);
// w = v - u, *ss = |w|^2, vout = w / |w|, *est = |w|
cudaError_t power_finish_step(const double* v, const double* u, int n, double* w, double* work, double* ss, double* vout,
                              double* est, cudaStream_t s);
cudaError_t mlp_forward(const float* theta, const float* X, int B, float* Y, float* H1, float* H2, cudaStream_t s);
cudaError_t mlp_backward(const float* theta, const float* X, const float* T, const float* Y, const float* H1,
                         const float* H2, int B, float* gpart, float* lpart, float* grad, float* loss, float* m,
                         float* v, float* theta_rw, float lr, float c1, float c2, bool adam, cudaStream_t s);

// sqrt(sum of v[0 .. count)) on a block of kReduceThreads threads, in one fixed order: thread t adds v[t],
// v[t + T], ... and the T partial sums meet in a pairwise tree. Every reduction of residual partials uses
// it, so that a batched solve reproduces the single-matrix path bit for bit. sh: T doubles of shared memory.
constexpr int kReduceThreads = 256;
__device__ inline double block_sum_sqrt(const double* v, int count, double* sh) {
  double s = 0.0;
  for (int i = threadIdx.x; i < count; i += kReduceThreads) s += v[i];
  sh[threadIdx.x] = s;
  __syncthreads();
  for (int w = kReduceThreads / 2; w > 0; w >>= 1) {
    if ((int)threadIdx.x < w) sh[threadIdx.x] += sh[threadIdx.x + w];
    __syncthreads();
  }
  return sqrt(sh[0]);
}

// out[m] = sqrt(sum of partial[begin[m] .. end[m])) for m < count, each sum in a fixed order.
cudaError_t segmented_reduce_sqrt(const double* partial, const int* begin, const int* end, int count, double* out,
                                  cudaStream_t s);

// The stop rule of pr_iterate on the newest residual r of a history: prev says that the residual before it,
// q, was taken at the same precision; low that the precision is below FP64 accuracy (PR_FP8, PR_BF16,
// PR_FP32X). Returns a pr_status to stop with, or -1 to apply one more update. (Host and device: the batched
// solver decides on the GPU.)
__host__ __device__ inline int stop_rule_last(double r, bool prev, double q, bool low, double tol,
                                              const pr_options& o) {
  if (!isfinite(r)) return PR_EDIVERGED;
  if (r <= tol) return PR_OK;
  if (prev) {
    const double arm = low ? o.stag_below_lowp : o.stag_below;
    if (q < arm && r > o.stag_ratio * q) return PR_ESTAGNATED;
    if (low && r >= q) return PR_ESTAGNATED;  // a low-precision floor, or the iteration leaving its basin
  }
  return -1;
}
// The same rule on a whole history with its per-entry precisions (capi.cu).
int stop_rule(const double* hist, const int* prec, int len, double tol, const pr_options& o);

// ---- device-side control of batched solves (k_batch.cu)
// All state of a batch that the solve loop reads or changes lives on the device, so that the whole loop
// runs as one graph: the kernels below build each product stage's work list from the matrices' states,
// append residuals to the histories, apply every matrix's stop rule and set the loop condition.
struct BatchCtl {
  int count;  // matrices
  int hcap;   // history entries per matrix
  int per;    // residual partials per work item
  int ld;     // leading dimension of the packed FP64 buffers
  // static description
  const int* order;                      // matrices by decreasing order
  const int *n, *p, *form, *row0;        // per matrix
  const int *off_sym, *cnt_sym, *off_full, *cnt_full;  // per matrix: its items in items_sym / items_full
  const int4 *items_sym, *items_full;    // every matrix's work items (emu_tile_list), symmetric and full
  // state
  int *active, *status, *iters, *hlen;   // per matrix (status -1: running)
  int* loops;                            // passes of the solve loop in the current solve
  double* hist;                          // count x hcap residual histories
  double* tally;                         // [0] timed ns, [1] timed flops, [2] timed launches,
                                         // [3] non-empty product launches, [4] products, [5] product flops
  const double* params;                  // [0] tolerance
  // the current stage
  int4* items;                           // its work list
  int* nitems;
  EmuBatchMat* mats;                     // its per-matrix records
  int *seg_b, *seg_e, *member, *ofs;     // per matrix: residual partial range, membership, first item
  // timing slots of the product launches (2 timestamps and the flops of the last launch per slot)
  unsigned long long* tstamp;
  double* flops_pending;
  // results
  double* result;
  int* row_n;
  int* row_n2;     // if set: a second per-row order array (-1 for rows not sliced) that stops also clear
  const int* err;
  // verification after the solve loop: the true residual ||I - X^p A||_F of every coupled-form matrix that
  // stopped on tol, stagnation or max_iter (-1 for the others), and the per-row orders of those matrices
  double* truer;
  int* row_v;
};
// Membership of a product stage: matrices of one form that are still iterating, optionally with p == pj
// (pcmp 1) or p > pj (pcmp 2), optionally only those without a residual yet (fresh_only), and never those
// with p == pskip (0: none).
struct BatchStage {
  int full;         // 0: symmetric-mode work items, 1: full
  int form;         // PR_FORM_NS or PR_FORM_COUPLED
  int pcmp, pj;
  int fresh_only;
  int pskip;
  int slot;         // timing slot of the product launch
  double a, b, c;   // epilogue coefficients of the members
  int verify;       // 1: members are the stopped matrices being verified (batch_verify_rows), not iterating ones
};
cudaError_t batch_stage_list(const BatchCtl& c, const BatchStage& st, cudaStream_t s);
// Residual of every member of the last stage from its partials, appended to its history (to_true: stored
// as the member's true residual instead).
cudaError_t batch_residuals(const BatchCtl& c, const double* partial, int to_true, cudaStream_t s);
// Marks the matrices to verify after the solve loop (coupled form, stopped on tol, stagnation or max_iter):
// their rows get their order in row_v (-1 elsewhere); truer is reset to -1.
cudaError_t batch_verify_rows(const BatchCtl& c, cudaStream_t s);
// The stop rule for every iterating matrix; a stopping matrix's rows of X go to the results and leave
// the digit slicing (row order -1).
cudaError_t batch_decide(const BatchCtl& c, const double* X, const pr_options& o, cudaStream_t s);
// Counts one update for every iterating matrix; with set_cond, sets the loop condition of the solve graph:
// some matrix still iterating, no device wait expired and fewer than `limit` passes.
cudaError_t batch_advance(const BatchCtl& c, cudaGraphConditionalHandle h, int set_cond, int limit, cudaStream_t s);
// Adds the last launch of every timing slot to the tally.
cudaError_t batch_harvest(const BatchCtl& c, int nslots, cudaStream_t s);
// out = fma(a, x, b y) (as lincomb) on the rows and columns of every iterating matrix with root pj, in the
// packed layout (leading dimension c.ld); other elements are left as they are.
cudaError_t batch_lincomb(const BatchCtl& c, int pj, const double* x, const double* y, double a, double b,
                          double* out, cudaStream_t s);

// Records the text returned by pr_last_error(NULL) for a failing call that has no handle.
void set_handleless_error(const char* msg);

}  // namespace pr
