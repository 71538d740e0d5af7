// BF16 tensor-core products for the low-precision iterations of Eq. 1 (Sec. 3, approximate arithmetic).
//
// P[i][j] = sum_k X[i][k] Y[j][k] for BF16 operands stored row-major (K contiguous), i.e. P = X Y^T; for the
// symmetric iterates of Sec. 2 Y^T = Y, so this is X Y. One CTA computes a 128 x 128 output tile:
//   warp 0, lane 0  TMA producer: 128 x 64 boxes of X (rows i0..) and Y (rows j0..) into a 3-stage ring of
//                   128-byte-swizzled shared-memory tiles, completing on the stage's "full" mbarrier;
//   warp 1, lane 0  MMA issuer: 4 x tcgen05.mma (M = 128, N = 128, K = 16) per stage into a 128-column FP32
//                   accumulator in TMEM; tcgen05.commit frees the stage ("empty") and finally signals "done";
//   warps 0-3       epilogue: each warp reads its 32 TMEM lanes (tile rows) with tcgen05.ld, applies the fused
//                   epilogue of pr::Epilogue in FP32 -> FP64, and stores FP64 masters and BF16 operands.
// Two CTAs fit on an SM (about 97 KB of shared memory and 128 TMEM columns each), so one CTA's epilogue
// overlaps the other's main loop. Every mbarrier wait is bounded: after 2 s the kernel records an error
// code, skips the rest of its work, waits (bounded) for its own copies and MMAs, frees TMEM and returns.
#include "pr_internal.h"
#include "tc_ptx.h"

#include <cudaTypedefs.h>

namespace pr {
namespace {

constexpr int TBM = 128, TBN = 128, TBK = 64, TSTAGES = 3, TTHREADS = 128;
constexpr int TILE_BYTES = TBM * TBK * 2;  // one 128 x 64 BF16 box
constexpr int TSMEM_BYTES = 2 * TSTAGES * TILE_BYTES + 1024 /*alignment slack*/ + 256 /*barriers*/;
constexpr uint32_t kIdesc = ptx::idesc_bf16_f32(TBM, TBN);

struct TcArgs {
  int n;       // order
  int ldl;     // leading dimension (elements) of the BF16 buffers
  int T;       // tiles per side
  int transpose;  // full mode: store P^T
  Epilogue e;
  int* err;
};

__device__ __forceinline__ void tri_index_tc(int t, int T, int& bi, int& bj) {
  const double b = 2.0 * T + 1.0;
  int r = (int)floor((b - sqrt(b * b - 8.0 * (double)t)) * 0.5);
  if (r < 0) r = 0;
  if (r > T - 1) r = T - 1;
  auto start = [T](int q) { return q * T - (q * (q - 1)) / 2; };
  while (r > 0 && start(r) > t) --r;
  while (r + 1 < T && start(r + 1) <= t) ++r;
  bi = r;
  bj = r + (t - start(r));
}

template <bool SYM>
__global__ void __launch_bounds__(TTHREADS, 2)
    k_gemm_bf16_tc(const __grid_constant__ CUtensorMap tmX, const __grid_constant__ CUtensorMap tmY, TcArgs args) {
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  uint8_t* sA = smem;
  uint8_t* sB = smem + TSTAGES * TILE_BYTES;
  uint64_t* bars = reinterpret_cast<uint64_t*>(smem + 2 * TSTAGES * TILE_BYTES);  // full[S], empty[S], done
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(bars + 2 * TSTAGES + 1);
  __shared__ double red[TTHREADS / 32];

  const int n = args.n, T = args.T;
  int bi, bj, tile_id;
  if (SYM) {
    tile_id = blockIdx.x;
    tri_index_tc(tile_id, T, bi, bj);
  } else {
    bi = blockIdx.y;
    bj = blockIdx.x;
    tile_id = blockIdx.y * gridDim.x + blockIdx.x;
  }
  const int i0 = bi * TBM, j0 = bj * TBN;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int KB = (n + TBK - 1) / TBK;
  const uint32_t full0 = ptx::smem_u32(bars), empty0 = ptx::smem_u32(bars + TSTAGES),
                 done = ptx::smem_u32(bars + 2 * TSTAGES);

  if (threadIdx.x == 0) {
    for (int s = 0; s < TSTAGES; ++s) {
      ptx::mbar_init(full0 + 8 * s, 1);
      ptx::mbar_init(empty0 + 8 * s, 1);
    }
    ptx::mbar_init(done, 1);
    ptx::fence_barrier_init();
    ptx::prefetch_tmap(&tmX);
    ptx::prefetch_tmap(&tmY);
  }
  if (warp == 0) {
    ptx::tmem_alloc(ptx::smem_u32(tmem_slot), TBN);
    ptx::tmem_relinquish();
  }
  ptx::tc_fence_before();
  __syncthreads();
  ptx::tc_fence_after();
  const uint32_t tmem = *tmem_slot;

  if (warp == 0 && lane == 0) {
    // TMA producer.
    int issued = 0;
    for (int kb = 0; kb < KB; ++kb) {
      const int s = kb % TSTAGES, r = kb / TSTAGES;
      if (!ptx::mbar_wait(empty0 + 8 * s, (r & 1) ^ 1, args.err, 1)) break;
      ptx::mbar_expect_tx(full0 + 8 * s, 2 * TILE_BYTES);
      ptx::tma_load_2d(ptx::smem_u32(sA + s * TILE_BYTES), &tmX, full0 + 8 * s, kb * TBK, i0);
      ptx::tma_load_2d(ptx::smem_u32(sB + s * TILE_BYTES), &tmY, full0 + 8 * s, kb * TBK, j0);
      ++issued;
    }
    // Do not leave while copies into this CTA's shared memory may still be landing (bounded).
    for (int kb = (issued > TSTAGES ? issued - TSTAGES : 0); kb < issued; ++kb)
      ptx::mbar_wait(full0 + 8 * (kb % TSTAGES), (kb / TSTAGES) & 1, args.err, 4);
  } else if (warp == 1 && lane == 0) {
    // MMA issuer.
    for (int kb = 0; kb < KB; ++kb) {
      const int s = kb % TSTAGES, r = kb / TSTAGES;
      if (!ptx::mbar_wait(full0 + 8 * s, r & 1, args.err, 2)) break;
      ptx::tc_fence_after();
      const uint64_t da = ptx::desc_sw128_kmajor(ptx::smem_u32(sA + s * TILE_BYTES));
      const uint64_t db = ptx::desc_sw128_kmajor(ptx::smem_u32(sB + s * TILE_BYTES));
#pragma unroll
      for (int kk = 0; kk < TBK / 16; ++kk)  // +32 bytes along K per step: +2 in the encoded start address
        ptx::mma_f16(tmem, da + 2 * kk, db + 2 * kk, kIdesc, (kb | kk) != 0);
      ptx::mma_commit(empty0 + 8 * s);
    }
    ptx::mma_commit(done);
  }
  __syncwarp();

  // Epilogue: warp w owns TMEM lanes (tile rows) 32w .. 32w + 31.
  const bool ok = ptx::mbar_wait(done, 0, args.err, 3);
  ptx::tc_fence_after();
  const Epilogue& e = args.e;
  const int ldl = args.ldl;
  const int r = warp * 32 + lane;
  const int i = i0 + r;
  const bool diag = SYM && bi == bj;
  double part = 0.0;
  if (ok) {
#pragma unroll 1
    for (int c0 = 0; c0 < TBN; c0 += 32) {
      uint32_t v[32];
      ptx::tmem_ld_32x32b_x32(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)c0, v);
      ptx::tmem_ld_wait();
      if (i >= n) continue;
#pragma unroll
      for (int c = 0; c < 32; ++c) {
        const int j = j0 + c0 + c;
        if (j >= n) continue;
        if (diag && r > c0 + c) continue;  // diagonal tile: upper triangle only
        const double P = (double)__uint_as_float(v[c]);
        const bool mirror = SYM && i != j;
        // Destination of element (i, j): transposed in full mode when asked.
        const int di = (!SYM && args.transpose) ? j : i, dj = (!SYM && args.transpose) ? i : j;
        const int64_t ij = (int64_t)di * n + dj, ji = (int64_t)dj * n + di;
        const int64_t lij = (int64_t)di * ldl + dj, lji = (int64_t)dj * ldl + di;
        if (e.out) {
          e.out[ij] = P;
          if (mirror) e.out[ji] = P;
        }
        if (e.out_lp) {
          const __nv_bfloat16 b = bf16_rne(P);
          e.out_lp[lij] = b;
          if (mirror) e.out_lp[lji] = b;
        }
        if (e.out2 || e.out2_lp) {
          double w = e.b * P;
          if (i == j) w += e.a;
          if (e.c != 0.0) w += e.c * e.cin[(int64_t)i * n + j];
          if (e.out2) {
            e.out2[ij] = w;
            if (mirror) e.out2[ji] = w;
          }
          if (e.out2_lp) {
            const __nv_bfloat16 b = bf16_rne(w);
            e.out2_lp[lij] = b;
            if (mirror) e.out2_lp[lji] = b;
          }
        }
        if (e.partial) {
          const double d = (i == j ? 1.0 : 0.0) - P;
          part += (mirror ? 2.0 : 1.0) * d * d;
        }
      }
    }
  }
  if (e.partial) {
    for (int o = 16; o > 0; o >>= 1) part += __shfl_xor_sync(0xffffffffu, part, o);
    if (lane == 0) red[warp] = part;
  }
  ptx::tc_fence_before();
  __syncthreads();
  if (e.partial && threadIdx.x == 0) e.partial[tile_id] = ((red[0] + red[1]) + red[2]) + red[3];
  if (warp == 0) ptx::tmem_dealloc(tmem, TBN);
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

// Tensor map of an n x n BF16 matrix with leading dimension ldl, box 64 (K) x 128 (rows), 128B swizzle.
cudaError_t make_map(CUtensorMap* map, const __nv_bfloat16* ptr, int n, int ldl) {
  auto fn = encode_fn();
  if (!fn) return cudaErrorNotSupported;
  cuuint64_t dims[2] = {(cuuint64_t)n, (cuuint64_t)n};
  cuuint64_t strides[1] = {(cuuint64_t)ldl * 2};
  cuuint32_t box[2] = {TBK, TBM};
  cuuint32_t estr[2] = {1, 1};
  CUresult r = fn(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<__nv_bfloat16*>(ptr), dims, strides, box, estr,
                  CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                  CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS ? cudaSuccess : cudaErrorInvalidValue;
}

}  // namespace

int gemm_tc_tiles(int n, Mode mode) {
  const int T = (n + TBM - 1) / TBM;
  return mode == Mode::Sym ? T * (T + 1) / 2 : T * T;
}

int bf16_ld(int n) { return (n + 7) / 8 * 8; }

cudaError_t gemm_bf16_tc(const __nv_bfloat16* X, const __nv_bfloat16* Y, int n, int ldl, Mode mode, bool transpose,
                         const Epilogue& e, int* err, cudaStream_t s) {
  if (ldl % 8 != 0 || ldl < n) return cudaErrorInvalidValue;
  if ((reinterpret_cast<uintptr_t>(X) | reinterpret_cast<uintptr_t>(Y)) & 15) return cudaErrorMisalignedAddress;
  static bool attr_set = false;
  if (!attr_set) {
    cudaError_t a = cudaFuncSetAttribute(k_gemm_bf16_tc<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, TSMEM_BYTES);
    if (a != cudaSuccess) return a;
    a = cudaFuncSetAttribute(k_gemm_bf16_tc<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, TSMEM_BYTES);
    if (a != cudaSuccess) return a;
    attr_set = true;
  }
  CUtensorMap mx, my;
  cudaError_t r = make_map(&mx, X, n, ldl);
  if (r != cudaSuccess) return r;
  r = make_map(&my, Y, n, ldl);
  if (r != cudaSuccess) return r;
  TcArgs args;
  args.n = n;
  args.ldl = ldl;
  args.T = (n + TBM - 1) / TBM;
  args.transpose = transpose ? 1 : 0;
  args.e = e;
  args.err = err;
  if (mode == Mode::Sym) {
    k_gemm_bf16_tc<true><<<args.T * (args.T + 1) / 2, TTHREADS, TSMEM_BYTES, s>>>(mx, my, args);
  } else {
    k_gemm_bf16_tc<false><<<dim3(args.T, args.T), TTHREADS, TSMEM_BYTES, s>>>(mx, my, args);
  }
  return cudaGetLastError();
}

}  // namespace pr
