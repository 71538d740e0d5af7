// BF16 tensor-core products for the low-precision iterations of Eq. 1 (Sec. 3, approximate arithmetic).
//
// P[i][j] = sum_k X[i][k] Y[j][k] for BF16 operands stored row-major (K contiguous), i.e. P = X Y^T; for the
// symmetric iterates of Sec. 2 Y^T = Y, so this is X Y. Persistent kernel, one CTA per SM, 128 x 256
// output tiles (symmetric mode: only tiles that reach the upper triangle), 192 threads:
//   warp 0 (one lane)  TMA producer: 128 x 64 boxes of X and 256 x 64 boxes of Y, 128-byte swizzled, into a
//                      4-stage ring (48 KB per stage), completing on the stage's "full" mbarrier;
//   warp 1 (one lane)  MMA issuer: 4 x tcgen05.mma (M = 128, N = 256, K = 16) per stage into one of two
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

constexpr int BM = 128, BN = 256, BK = 64, STAGES = 4;
constexpr int EPI_WARPS = 4, THREADS = 64 + 32 * EPI_WARPS;
constexpr int A_BYTES = BM * BK * 2, B_BYTES = BN * BK * 2, STAGE_BYTES = A_BYTES + B_BYTES;
constexpr int STG_FLOATS = 32 * 33;
constexpr int SMEM_BYTES = 1024 + STAGES * STAGE_BYTES + EPI_WARPS * STG_FLOATS * 4 + 256;
constexpr int TMEM_COLS = 2 * BN;
constexpr uint32_t kIdesc = ptx::idesc_bf16_f32(BM, BN);

struct TcArgs {
  int n, ldl;
  int Tm, Tn, ntiles;
  int transpose;  // full mode: store P^T
  Epilogue e;
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

template <bool SYM>
__global__ void __launch_bounds__(THREADS, 1)
    k_gemm_bf16_tc(const __grid_constant__ CUtensorMap tmX, const __grid_constant__ CUtensorMap tmY, TcArgs args) {
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
          for (int kk = 0; kk < BK / 16; ++kk)  // +32 bytes along K: +2 in the encoded start address
            ptx::mma_f16(d, da + 2 * kk, db + 2 * kk, kIdesc, (kb | kk) != 0);
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
      float part = 0.0f;
#pragma unroll 1
      for (int c0 = 0; c0 < BN; c0 += 32) {
        uint32_t v[32];
        ptx::tmem_ld_32x32b_x32(tmem + ((uint32_t)(32 * q) << 16) + (uint32_t)(b * BN + c0), v);
        ptx::tmem_ld_wait();
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
cudaError_t make_map(CUtensorMap* map, const __nv_bfloat16* ptr, int n, int ldl, int box_rows) {
  auto fn = encode_fn();
  if (!fn) return cudaErrorNotSupported;
  cuuint64_t dims[2] = {(cuuint64_t)n, (cuuint64_t)n};
  cuuint64_t strides[1] = {(cuuint64_t)ldl * 2};
  cuuint32_t box[2] = {(cuuint32_t)BK, (cuuint32_t)box_rows};
  cuuint32_t estr[2] = {1, 1};
  CUresult r = fn(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<__nv_bfloat16*>(ptr), dims, strides, box, estr,
                  CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                  CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
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

}  // namespace

int gemm_tc_tiles(int n, Mode mode) {
  int Tm, Tn, nt;
  tile_grid(n, mode, Tm, Tn, nt);
  return nt * EPI_WARPS;  // one residual partial per epilogue warp and tile
}

int bf16_ld(int n) { return (n + 7) / 8 * 8; }

cudaError_t gemm_bf16_tc(const __nv_bfloat16* X, const __nv_bfloat16* Y, int n, int ldl, Mode mode, bool transpose,
                         const Epilogue& e, int* err, cudaStream_t s) {
  if (ldl % 8 != 0 || ldl < n) return cudaErrorInvalidValue;
  if ((reinterpret_cast<uintptr_t>(X) | reinterpret_cast<uintptr_t>(Y)) & 15) return cudaErrorMisalignedAddress;
  static bool attr_set = false;
  if (!attr_set) {
    cudaError_t a = cudaFuncSetAttribute(k_gemm_bf16_tc<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, SMEM_BYTES);
    if (a != cudaSuccess) return a;
    a = cudaFuncSetAttribute(k_gemm_bf16_tc<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, SMEM_BYTES);
    if (a != cudaSuccess) return a;
    attr_set = true;
  }
  CUtensorMap mx, my;
  cudaError_t r = make_map(&mx, X, n, ldl, BM);
  if (r != cudaSuccess) return r;
  r = make_map(&my, Y, n, ldl, BN);
  if (r != cudaSuccess) return r;
  TcArgs args;
  args.n = n;
  args.ldl = ldl;
  tile_grid(n, mode, args.Tm, args.Tn, args.ntiles);
  args.transpose = transpose ? 1 : 0;
  args.e = e;
  args.err = err;
  const int grid = args.ntiles < sm_count() ? args.ntiles : sm_count();
  if (mode == Mode::Sym) {
    k_gemm_bf16_tc<true><<<grid, THREADS, SMEM_BYTES, s>>>(mx, my, args);
  } else {
    k_gemm_bf16_tc<false><<<grid, THREADS, SMEM_BYTES, s>>>(mx, my, args);
  }
  return cudaGetLastError();
}

}  // namespace pr
