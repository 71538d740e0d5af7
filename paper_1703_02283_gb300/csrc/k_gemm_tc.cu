// BF16 and FP8 tensor-core products for the low-precision iterations of Eq. 1 (Sec. 3, approximate
// arithmetic).
//
// P[i][j] = sum_k X[i][k] Y[j][k] for operands stored row-major (K contiguous), i.e. P = X Y^T; for the
// symmetric iterates of Sec. 2 Y^T = Y, so this is X Y. Two operand types share one kernel:
//   BF16  kind::f16 MMAs, K = 16 per instruction, 64 elements per 128-byte row of a stage;
//   FP8   E4M3 with a power-of-two scale per row (X_ik = 2^sx_i q_ik, Y_jk = 2^sy_j r_jk), kind::f8f6f4 MMAs,
//         K = 32 per instruction, 128 elements per 128-byte row; the epilogue multiplies the FP32 sum by
//         2^(sx_i + sy_j). Row scales of a symmetric iterate are its column scales, so the tile (i, j) of P
//         gets the scale of its row block times that of its column block, element by element.
// Both move the same bytes per stage and advance 32 bytes along K per instruction, so the ring, the
// descriptors and the epilogue are shared. Persistent kernel, one CTA per SM, 128 x 256 output tiles
// (symmetric mode: only tiles that reach the upper triangle), 192 threads:
//   warp 0 (one lane)  TMA producer: 128 x 128-byte boxes of X and 256 x 128-byte boxes of Y, 128-byte
//                      swizzled, into a 4-stage ring (48 KB per stage), completing on the stage's "full"
//                      mbarrier;
//   warp 1 (one lane)  MMA issuer: 4 x tcgen05.mma (M = 128, N = 256) per stage into one of two
//                      256-column FP32 accumulators in TMEM; tcgen05.commit frees the ring stage and, after
//                      the last K block, hands the accumulator to the epilogue ("tfull");
//   warps 2-5          epilogue: warp w reads TMEM lanes 32 (w % 4) .. + 31 (tile rows) with tcgen05.ld,
//                      32 columns at a time. Stores that go to (j, i) (the mirrored half) are coalesced
//                      straight from registers (lanes hold consecutive i); stores to (i, j) go through a
//                      32 x 33 shared-memory transpose per warp so that lanes write consecutive j. Then the
//                      accumulator is released ("tempty") while the MMA warp already fills the other one.
// Every wait is bounded (2 s); on expiry the kernel records an error code, raises a CTA-wide abort flag
// that ends every role's loop, drains its own copies and MMAs (bounded), frees TMEM and returns.
#include "pr_internal.h"
#include "tc_ptx.h"

#include <cudaTypedefs.h>

namespace pr {
namespace {

constexpr int BM = 128, BN = 256, ROW_BYTES = 128, STAGES = 4;
constexpr int EPI_WARPS = 4, THREADS = 64 + 32 * EPI_WARPS;
constexpr int A_BYTES = BM * ROW_BYTES, B_BYTES = BN * ROW_BYTES, STAGE_BYTES = A_BYTES + B_BYTES;
constexpr int STG_FLOATS = 32 * 33;
constexpr int SMEM_BYTES = 1024 + STAGES * STAGE_BYTES + EPI_WARPS * STG_FLOATS * 4 + 256;
constexpr int TMEM_COLS = 2 * BN;

// Elements of one 128-byte row of a stage (the K block) for 2-byte (BF16) and 1-byte (E4M3) operands.
template <bool F8>
constexpr int block_k() { return F8 ? 128 : 64; }

struct TcArgs {
  int n, ldl;
  int Tm, Tn, ntiles;
  int transpose;  // full mode: store P^T
  Epilogue e;
  const int* sx;  // FP8: row scales (exponents) of X and Y
  const int* sy;
  int* err;
};

// Tile t -> (bi, bj) of 128-row x 256-column tiles, column-panel major so that concurrently running CTAs
// share the B panel. Symmetric mode keeps tiles with 128 bi <= 256 bj + 255, i.e. bi <= 2 bj + 1.
__device__ __forceinline__ void tile_coords(int t, int Tm, int Tn, bool sym, int& bi, int& bj) {
  if (!sym) {
    bi = t % Tm;
    bj = t / Tm;
    return;
  }
  for (int b = 0; b < Tn; ++b) {
    const int c = min(2 * b + 2, Tm);
    if (t < c) {
      bi = t;
      bj = b;
      return;
    }
    t -= c;
  }
  bi = bj = 0;
}

// Writes every requested output at (di, dj) for the product value P. Arithmetic in FP32: the operands
// carry BF16 precision and the accumulator FP32, and FP64 instructions are scarce on this part.
struct Emit {
  const Epilogue& e;
  int n, ldl;
  float a, b, c;
  __device__ __forceinline__ void operator()(int di, int dj, float P) const {
    const int64_t ij = (int64_t)di * n + dj, lij = (int64_t)di * ldl + dj;
    if (e.out) e.out[ij] = (double)P;
    if (e.out_lp) e.out_lp[lij] = bf16_rne(P);
    if (e.out2 || e.out2_lp) {
      float w = b * P;
      if (di == dj) w += a;
      if (c != 0.0f) w = fmaf(c, (float)e.cin[ij], w);  // cin is symmetric wherever it is used
      if (e.out2) e.out2[ij] = (double)w;
      if (e.out2_lp) e.out2_lp[lij] = bf16_rne(w);
    }
  }
};

template <bool SYM, bool F8>
__global__ void __launch_bounds__(THREADS, 1)
    k_gemm_lowp_tc(const __grid_constant__ CUtensorMap tmX, const __grid_constant__ CUtensorMap tmY, TcArgs args) {
  constexpr int BK = block_k<F8>();
  constexpr uint32_t kIdesc = F8 ? ptx::idesc_e4m3_f32(BM, BN) : ptx::idesc_bf16_f32(BM, BN);
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  uint8_t* ring = smem;
  float* stg = reinterpret_cast<float*>(smem + STAGES * STAGE_BYTES);
  uint64_t* bars = reinterpret_cast<uint64_t*>(stg + EPI_WARPS * STG_FLOATS);  // full[S] empty[S] tfull[2] tempty[2] drain
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(bars + 2 * STAGES + 5);
  volatile int* s_abort = reinterpret_cast<volatile int*>(tmem_slot + 1);

  const int n = args.n, warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int KB = (n + BK - 1) / BK;
  const uint32_t full0 = ptx::smem_u32(bars), empty0 = full0 + 8 * STAGES, tfull0 = empty0 + 8 * STAGES,
                 tempty0 = tfull0 + 16, drain = tempty0 + 16;

  if (threadIdx.x == 0) {
    for (int s = 0; s < STAGES; ++s) {
      ptx::mbar_init(full0 + 8 * s, 1);
      ptx::mbar_init(empty0 + 8 * s, 1);
    }
    for (int b = 0; b < 2; ++b) {
      ptx::mbar_init(tfull0 + 8 * b, 1);
      ptx::mbar_init(tempty0 + 8 * b, EPI_WARPS);
    }
    ptx::mbar_init(drain, 1);
    *s_abort = 0;
    ptx::fence_barrier_init();
    ptx::prefetch_tmap(&tmX);
    ptx::prefetch_tmap(&tmY);
  }
  if (warp == 0) {
    ptx::tmem_alloc(ptx::smem_u32(tmem_slot), TMEM_COLS);
    ptx::tmem_relinquish();
  }
  ptx::tc_fence_before();
  __syncthreads();
  ptx::tc_fence_after();
  const uint32_t tmem = *tmem_slot;

  if (warp == 0) {
    if (lane == 0) {
      // ---------------- TMA producer
      int it = 0;
      for (int t = blockIdx.x; t < args.ntiles && !*s_abort; t += gridDim.x) {
        int bi, bj;
        tile_coords(t, args.Tm, args.Tn, SYM, bi, bj);
        for (int kb = 0; kb < KB; ++kb, ++it) {
          const int s = it % STAGES;
          if (*s_abort || !ptx::mbar_wait(empty0 + 8 * s, ((it / STAGES) & 1) ^ 1, args.err, 1)) {
            *s_abort = 1;
            break;
          }
          uint8_t* st = ring + s * STAGE_BYTES;
          ptx::mbar_expect_tx(full0 + 8 * s, STAGE_BYTES);
          ptx::tma_load_2d(ptx::smem_u32(st), &tmX, full0 + 8 * s, kb * BK, bi * BM);
          ptx::tma_load_2d(ptx::smem_u32(st + A_BYTES), &tmY, full0 + 8 * s, kb * BK, bj * BN);
        }
      }
      if (*s_abort) {  // copies issued but perhaps never consumed: let them land (bounded)
        for (int k = (it > STAGES ? it - STAGES : 0); k < it; ++k)
          ptx::mbar_wait(full0 + 8 * (k % STAGES), (k / STAGES) & 1, nullptr, 0);
      }
    }
  } else if (warp == 1) {
    if (lane == 0) {
      // ---------------- MMA issuer
      int it = 0, lt = 0;
      for (int t = blockIdx.x; t < args.ntiles && !*s_abort; t += gridDim.x, ++lt) {
        const int b = lt & 1;
        if (!ptx::mbar_wait(tempty0 + 8 * b, ((lt >> 1) & 1) ^ 1, args.err, 2)) {
          *s_abort = 1;
          break;
        }
        ptx::tc_fence_after();
        const uint32_t d = tmem + (uint32_t)(b * BN);
        bool ok = true;
        for (int kb = 0; kb < KB; ++kb, ++it) {
          const int s = it % STAGES;
          if (*s_abort || !ptx::mbar_wait(full0 + 8 * s, (it / STAGES) & 1, args.err, 3)) {
            *s_abort = 1;
            ok = false;
            break;
          }
          ptx::tc_fence_after();
          const uint32_t sa = ptx::smem_u32(ring + s * STAGE_BYTES);
          const uint64_t da = ptx::desc_sw128_kmajor(sa), db = ptx::desc_sw128_kmajor(sa + A_BYTES);
#pragma unroll
          for (int kk = 0; kk < 4; ++kk) {  // +32 bytes along K: +2 in the encoded start address
            if constexpr (F8) ptx::mma_f8(d, da + 2 * kk, db + 2 * kk, kIdesc, (kb | kk) != 0);
            else ptx::mma_f16(d, da + 2 * kk, db + 2 * kk, kIdesc, (kb | kk) != 0);
          }
          ptx::mma_commit(empty0 + 8 * s);
        }
        if (!ok) break;
        ptx::mma_commit(tfull0 + 8 * b);
      }
      // Every MMA issued has completed before TMEM can be released.
      ptx::mma_commit(drain);
      ptx::mbar_wait(drain, 0, nullptr, 0);
    }
  } else {
    // ---------------- epilogue warps
    const int q = warp & 3;
    float* wst = stg + q * STG_FLOATS;
    const Emit emit{args.e, n, args.ldl, (float)args.e.a, (float)args.e.b, (float)args.e.c};
    const Epilogue& e = args.e;
    int lt = 0;
    for (int t = blockIdx.x; t < args.ntiles; t += gridDim.x, ++lt) {
      if (__shfl_sync(0xffffffffu, *s_abort, 0)) break;
      const int b = lt & 1;
      const bool ok = __all_sync(0xffffffffu, ptx::mbar_wait(tfull0 + 8 * b, (lt >> 1) & 1, args.err, 4));
      if (!ok) {
        *s_abort = 1;
        break;
      }
      ptx::tc_fence_after();
      int bi, bj;
      tile_coords(t, args.Tm, args.Tn, SYM, bi, bj);
      const int i0 = bi * BM, j0 = bj * BN;
      const int i = i0 + 32 * q + lane;
      int sxi = 0;
      if constexpr (F8) sxi = i < n ? args.sx[i] : 0;
      float part = 0.0f;
#pragma unroll 1
      for (int c0 = 0; c0 < BN; c0 += 32) {
        uint32_t v[32];
        ptx::tmem_ld_32x32b_x32(tmem + ((uint32_t)(32 * q) << 16) + (uint32_t)(b * BN + c0), v);
        ptx::tmem_ld_wait();
        if constexpr (F8) {
          // P_ij = 2^(sx_i + sy_j) x the FP32 sum of the E4M3 products (lane = row i; column c0 + c).
          const int jl = j0 + c0 + lane, syl = jl < n ? args.sy[jl] : 0;
#pragma unroll
          for (int c = 0; c < 32; ++c)
            v[c] = __float_as_uint(ldexpf(__uint_as_float(v[c]), sxi + __shfl_sync(0xffffffffu, syl, c)));
        }
        // Register layout: lane = row i. Residual partials, and the stores that land at (j, i).
        const bool colset = SYM || args.transpose;
#pragma unroll
        for (int c = 0; c < 32; ++c) {
          const int j = j0 + c0 + c;
          if (i >= n || j >= n || (SYM && i > j)) continue;
          const float P = __uint_as_float(v[c]);
          if (e.partial) {
            const float dd = (i == j ? 1.0f : 0.0f) - P;
            part = fmaf((SYM && i != j) ? 2.0f * dd : dd, dd, part);
          }
          if (colset && (!SYM || i != j)) emit(j, i, P);
        }
        // Staged layout: lane = column j. The stores that land at (i, j).
        if (SYM || !args.transpose) {
          __syncwarp();
#pragma unroll
          for (int c = 0; c < 32; ++c) wst[lane * 33 + c] = __uint_as_float(v[c]);
          __syncwarp();
          const int j2 = j0 + c0 + lane;
#pragma unroll 4
          for (int rr = 0; rr < 32; ++rr) {
            const int i2 = i0 + 32 * q + rr;
            if (i2 < n && j2 < n && (!SYM || i2 <= j2)) emit(i2, j2, wst[rr * 33 + lane]);
          }
          __syncwarp();
        }
      }
      // Release the accumulator to the MMA warp.
      ptx::tc_fence_before();
      __syncwarp();
      if (lane == 0) ptx::mbar_arrive(tempty0 + 8 * b);
      if (e.partial) {
        for (int o = 16; o > 0; o >>= 1) part += __shfl_xor_sync(0xffffffffu, part, o);
        if (lane == 0) e.partial[(int64_t)t * EPI_WARPS + q] = (double)part;
      }
    }
  }
  ptx::tc_fence_before();
  __syncthreads();
  ptx::tc_fence_after();
  if (warp == 0) ptx::tmem_dealloc(tmem, TMEM_COLS);
}

PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  if (!fn) {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
  }
  return fn;
}

// Tensor map of an n x n BF16 matrix with leading dimension ldl: boxes of 64 (K) x box_rows, 128B swizzle.
// Tensor map of an n x n matrix of `esize`-byte elements with leading dimension ld (elements): boxes of one
// 128-byte row (K) x box_rows, 128B swizzle.
cudaError_t make_map(CUtensorMap* map, const void* ptr, int n, int ld, int esize, int box_rows) {
  auto fn = encode_fn();
  if (!fn) return cudaErrorNotSupported;
  cuuint64_t dims[2] = {(cuuint64_t)n, (cuuint64_t)n};
  cuuint64_t strides[1] = {(cuuint64_t)ld * esize};
  cuuint32_t box[2] = {(cuuint32_t)(ROW_BYTES / esize), (cuuint32_t)box_rows};
  cuuint32_t estr[2] = {1, 1};
  CUresult r = fn(map, esize == 2 ? CU_TENSOR_MAP_DATA_TYPE_BFLOAT16 : CU_TENSOR_MAP_DATA_TYPE_UINT8, 2,
                  const_cast<void*>(ptr), dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                  CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS ? cudaSuccess : cudaErrorInvalidValue;
}

int sm_count() {
  static int count = 0;
  if (!count) {
    int dev = 0;
    cudaGetDevice(&dev);
    if (cudaDeviceGetAttribute(&count, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || count < 1) count = 1;
  }
  return count;
}

void tile_grid(int n, Mode mode, int& Tm, int& Tn, int& ntiles) {
  Tm = (n + BM - 1) / BM;
  Tn = (n + BN - 1) / BN;
  if (mode == Mode::Full) {
    ntiles = Tm * Tn;
  } else {
    ntiles = 0;
    for (int b = 0; b < Tn; ++b) ntiles += (2 * b + 2 < Tm ? 2 * b + 2 : Tm);
  }
}


cudaError_t set_attributes() {
  static bool attr_set = false;
  if (attr_set) return cudaSuccess;
  for (auto k : {k_gemm_lowp_tc<true, false>, k_gemm_lowp_tc<false, false>, k_gemm_lowp_tc<true, true>,
                 k_gemm_lowp_tc<false, true>}) {
    cudaError_t a = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, SMEM_BYTES);
    if (a != cudaSuccess) return a;
  }
  attr_set = true;
  return cudaSuccess;
}

template <bool F8>
cudaError_t launch(const void* X, const void* Y, const int* sx, const int* sy, int n, int ld, Mode mode,
                   bool transpose, const Epilogue& e, int* err, cudaStream_t s) {
  const int esize = F8 ? 1 : 2;
  if ((ld * esize) % 16 != 0 || ld < n) return cudaErrorInvalidValue;
  if ((reinterpret_cast<uintptr_t>(X) | reinterpret_cast<uintptr_t>(Y)) & 15) return cudaErrorMisalignedAddress;
  if (F8 && (!sx || !sy)) return cudaErrorInvalidValue;
  cudaError_t r = set_attributes();
  if (r != cudaSuccess) return r;
  CUtensorMap mx, my;
  r = make_map(&mx, X, n, ld, esize, BM);
  if (r != cudaSuccess) return r;
  r = make_map(&my, Y, n, ld, esize, BN);
  if (r != cudaSuccess) return r;
  TcArgs args;
  args.n = n;
  args.ldl = ld;
  tile_grid(n, mode, args.Tm, args.Tn, args.ntiles);
  args.transpose = transpose ? 1 : 0;
  args.e = e;
  args.sx = sx;
  args.sy = sy;
  args.err = err;
  const int grid = args.ntiles < sm_count() ? args.ntiles : sm_count();
  if (mode == Mode::Sym) {
    k_gemm_lowp_tc<true, F8><<<grid, THREADS, SMEM_BYTES, s>>>(mx, my, args);
  } else {
    k_gemm_lowp_tc<false, F8><<<grid, THREADS, SMEM_BYTES, s>>>(mx, my, args);
  }
  return cudaGetLastError();
}

// Exponent of the row's largest |x| (FP64 bits; 0 for a zero row) minus 7: the row, divided by 2^s, has its
// largest magnitude in [128, 256), below E4M3's largest finite 448.
__device__ __forceinline__ int fp8_row_scale(unsigned long long max_bits) {
  const int E = (int)(max_bits >> 52);
  return E == 0 ? 0 : E - 1023 - 7;
}

// Rounds the finite y to E4M3 (1 sign, 4 exponent bits of bias 7, 3 mantissa bits; subnormals m 2^-9; no
// infinities; largest finite 448, larger magnitudes saturate to it) to nearest, ties to even, in one
// rounding from FP64 (integer arithmetic on the bit pattern).
__device__ __forceinline__ uint8_t e4m3_rne(double y) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(y);
  const unsigned sign = (unsigned)(b >> 63) << 7;
  const int E = (int)((b >> 52) & 0x7ff);
  if (E == 0) return (uint8_t)sign;  // zero, or an FP64 subnormal: far below 2^-10
  const int e = E - 1023;
  const unsigned long long M = (b & 0xfffffffffffffull) | (1ull << 52);  // |y| = M 2^(e - 52)
  const int emin = e < -6 ? -6 : e;           // binade of the result's last bit: 2^(emin - 3)
  const int sh = 49 + (emin - e);             // bits of M below that last bit
  unsigned q = 0;
  if (sh < 54) {
    q = (unsigned)(M >> sh);
    const unsigned long long rest = M & ((1ull << sh) - 1), half = 1ull << (sh - 1);
    if (rest > half || (rest == half && (q & 1u))) ++q;
  }
  int ee = emin;
  if (q >= 16u) {  // rounded up into the next binade
    q >>= 1;
    ++ee;
  }
  if (q < 8u) return (uint8_t)(sign | q);  // subnormal (ee = -6), or zero
  if (ee > 8 || (ee == 8 && q > 14u)) return (uint8_t)(sign | 0x7e);  // saturate at 448
  return (uint8_t)(sign | ((unsigned)(ee + 7) << 3) | (q - 8u));
}

// One warp per row: s_i from the row maximum, then q_ij = E4M3(x_ij 2^-s_i) (exact scaling, one rounding).
// Columns n .. ld - 1 get 0.
__global__ void k_to_fp8(const double* __restrict__ X, int n, int ld, uint8_t* __restrict__ Q, int* __restrict__ sx) {
  const int lane = threadIdx.x & 31;
  for (int i = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; i < n; i += (gridDim.x * blockDim.x) >> 5) {
    const unsigned long long* row = reinterpret_cast<const unsigned long long*>(X + (int64_t)i * n);
    unsigned long long mb = 0;
    for (int k = lane; k < n; k += 32) {
      const unsigned long long u = row[k] & 0x7fffffffffffffffull;
      mb = u > mb ? u : mb;
    }
    for (int o = 16; o > 0; o >>= 1) {
      const unsigned long long w = __shfl_xor_sync(0xffffffffu, mb, o);
      mb = w > mb ? w : mb;
    }
    const int si = fp8_row_scale(mb);
    if (lane == 0) sx[i] = si;
    for (int k = lane; k < ld; k += 32)
      Q[(int64_t)i * ld + k] = k < n ? e4m3_rne(ldexp(__longlong_as_double((long long)row[k]), -si)) : (uint8_t)0;
  }
}

}  // namespace

int gemm_tc_tiles(int n, Mode mode) {
  int Tm, Tn, nt;
  tile_grid(n, mode, Tm, Tn, nt);
  return nt * EPI_WARPS;  // one residual partial per epilogue warp and tile
}

int bf16_ld(int n) { return (n + 7) / 8 * 8; }

cudaError_t gemm_bf16_tc(const __nv_bfloat16* X, const __nv_bfloat16* Y, int n, int ldl, Mode mode, bool transpose,
                         const Epilogue& e, int* err, cudaStream_t s) {
  return launch<false>(X, Y, nullptr, nullptr, n, ldl, mode, transpose, e, err, s);
}

cudaError_t gemm_fp8_tc(const uint8_t* X, const int* sx, const uint8_t* Y, const int* sy, int n, int ldq, Mode mode,
                        bool transpose, const Epilogue& e, int* err, cudaStream_t s) {
  if (e.out_lp || e.out2_lp) return cudaErrorInvalidValue;  // FP8 products write FP64 results only
  return launch<true>(X, Y, sx, sy, n, ldq, mode, transpose, e, err, s);
}

int fp8_ld(int n) { return (n + 15) / 16 * 16; }

cudaError_t to_fp8(const double* X, int n, int ldq, uint8_t* Q, int* sx, cudaStream_t s) {
  if (ldq < n || ldq % 16 != 0) return cudaErrorInvalidValue;
  int blocks = (n + 7) / 8;
  if (blocks > 152 * 8) blocks = 152 * 8;
  k_to_fp8<<<blocks, 256, 0, s>>>(X, n, ldq, Q, sx);
  return cudaGetLastError();
}

}  // namespace pr
