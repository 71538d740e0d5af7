// FP64-accurate matrix products from exact BF16 digit slices on the tcgen05 tensor cores (PR_EMU64).
//
// GB300 executes FP64 at about 1/1800 of its BF16 tensor rate, so the FP64-accurate iterations of Eq. 1
// (Sec. 3: precise refinement) are built from exact low-precision pieces, following the error-free
// splitting of Ozaki, Ogita, Oishi and Rump ("Error-free transformations of matrix multiplication by using
// fast routines of matrix multiplication and its applications", Numer. Algorithms 59, 2012):
//
//  * slicing (k_slice): for row i of X let e_i be the smallest integer with max_k |x_ik| < 2^(e_i - 1). The
//    integer F_ik = round(x_ik 2^(7S - e_i)) (|F| < 2^(7S - 1)) is written in balanced base 128,
//    F = sum_{s=1..S} d_s 128^(S-s) with |d_s| <= 64, so x_ik = 2^e_i sum_s d_s 2^(-7s) up to 2^(e_i - 7S - 1).
//    The digits are small integers, exact in BF16. Integer arithmetic only.
//  * products (k_gemm_emu): P_ij = 2^(e_i + f_j) sum_{s + t <= S + 1} 2^(-7(s + t)) sum_k dX_s,ik dY_t,jk. Each
//    inner sum over at most 4096 terms is an integer of magnitude <= 4096 * 64 * 64 = 2^24, so the FP32
//    accumulation of the tensor cores computes it exactly. Pairs are taken level by level (L = s + t); the
//    exact pair results of a level are summed in int32, and each level is added into an FP64 total.
//    Dropping the pairs with s + t > S + 1 and the digits beyond S leaves an error of about
//    (S + 1) 2^(-7S - 2) in units of 2^(e_i + f_j) per product term: S = 9 (the default) gives 2^-62. F must
//    fit in 64-bit integers, which limits S to 9.
//
// k_gemm_emu is a persistent kernel, one CTA per SM, 128 x 128 output tiles (symmetric mode: upper
// triangle only, mirrored), 320 threads: warp 0 TMA producer (6-stage ring of 128 x 64 digit boxes), warp 1
// MMA issuer (M = N = 128, K = 16, one pass over K per pair into one of two 128-column TMEM accumulators),
// warps 2-9 epilogue (two warps per TMEM lane quadrant, 64 columns each): per pair they convert the exact
// FP32 result to int32 and add it to the level sum while the MMA warp fills the other accumulator; at a
// level end they add the level into an FP64 total kept in TMEM columns 256..511; after the last level
// they scale by 2^(e_i + f_j) and apply the fused FP64 epilogue. Waits are bounded as in k_gemm_tc.cu.
#include "pr_internal.h"
#include "tc_ptx.h"

#include <cudaTypedefs.h>

namespace pr {
namespace {

constexpr int EBM = 128, EBN = 128, EBK = 64, ESTAGES = 6;
constexpr int EPI_WARPS = 8, THREADS = 64 + 32 * EPI_WARPS;
constexpr int BOX_BYTES = EBM * EBK * 2, STAGE_BYTES = 2 * BOX_BYTES;
constexpr int SMEM_BYTES = 1024 + ESTAGES * STAGE_BYTES + 256;
constexpr int KCHUNK_BLOCKS = 4096 / EBK;  // K blocks per exact pass: 4096 * 64 * 64 = 2^24
constexpr int TOTAL_COL = 2 * EBN;         // TMEM column of the FP64 totals (2 words per element)
// Levels summed exactly in int64 before one FP64 addition: a level sum is below S * n * 2^12 <= 2^31, and
// kGroup levels Horner-combined with 7-bit shifts stay below 2^(31 + 7 (kGroup - 1)) <= 2^59.
constexpr int kGroup = 5;
constexpr uint32_t kIdesc = ptx::idesc_bf16_f32(EBM, EBN);

// ------------------------------------------------------------------------------------------ slicing

__device__ __forceinline__ unsigned long long warp_max_u64(unsigned long long v) {
  for (int o = 16; o > 0; o >>= 1) {
    const unsigned long long w = __shfl_xor_sync(0xffffffffu, v, o);
    v = w > v ? w : v;
  }
  return v;
}

// F = round(x 2^(7S - e)) of one double as an integer (|F| < 2^(7S - 1) for |x| < 2^(e - 1)).
__device__ __forceinline__ long long fixed_point(unsigned long long u, int e, int S) {
  const int E = (int)((u >> 52) & 0x7ff);
  if (E == 0) return 0;  // zero, or a subnormal far below the last digit
  const unsigned long long M = (u & 0xfffffffffffffull) | (1ull << 52);
  const int sh = (E - 1023) - e + 7 * S - 52;  // F = M 2^sh, sh <= 7S - 54
  long long F = 0;
  if (sh >= 0) F = (long long)(M << sh);
  else if (sh > -64) F = (long long)((M + (1ull << (-sh - 1))) >> (-sh));
  return (u >> 63) ? -F : F;
}

// One warp per row r of an R-row FP64 array (leading dimension ldx): exponent e_r, then S digit planes
// D[s][r][k] (plane s at s R ldl; s = 0 is the most significant digit). Row r has row_n[r] valid columns
// (all rows n when row_n is null); the rest of the ldl columns get digit 0. Each lane handles two adjacent
// columns (ldl is even), so loads are 16 bytes and stores bf16x2.
__global__ void k_slice(const double* __restrict__ X, int R, int n, int ldx, int ldl, int S,
                        const int* __restrict__ row_n, __nv_bfloat16* __restrict__ D, int* __restrict__ ex) {
  const int lane = threadIdx.x & 31;
  const int64_t plane = (int64_t)R * ldl;
  for (int i = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; i < R; i += (gridDim.x * blockDim.x) >> 5) {
    const int nr = row_n ? row_n[i] : n;
    const unsigned long long* row = reinterpret_cast<const unsigned long long*>(X + (int64_t)i * ldx);
    unsigned long long mb = 0;  // largest |x| as a bit pattern (non-negative doubles order like integers)
    for (int k = lane; k < nr; k += 32) {
      const unsigned long long u = row[k] & 0x7fffffffffffffffull;
      mb = u > mb ? u : mb;
    }
    mb = warp_max_u64(mb);
    const int emax = (int)(mb >> 52);               // biased exponent of the row maximum
    const int e = emax == 0 ? 0 : emax - 1023 + 2;  // zero (or subnormal-only) rows get digits 0
    if (lane == 0) ex[i] = e;
    for (int k = 2 * lane; k < ldl; k += 64) {
      long long F0 = 0, F1 = 0;
      if (emax != 0) {
        if (k < nr) F0 = fixed_point(row[k], e, S);
        if (k + 1 < nr) F1 = fixed_point(row[k + 1], e, S);
      }
      __nv_bfloat162* dst = reinterpret_cast<__nv_bfloat162*>(D + (int64_t)i * ldl + k);
      // Balanced base-128 digits, least significant first; the last one takes the remainder (|.| <= 64).
      for (int s = S - 1; s >= 1; --s) {
        const int r0 = (int)(F0 & 127), r1 = (int)(F1 & 127);
        const int d0 = r0 >= 64 ? r0 - 128 : r0, d1 = r1 >= 64 ? r1 - 128 : r1;
        F0 = (F0 - d0) >> 7;
        F1 = (F1 - d1) >> 7;
        dst[(int64_t)s * (plane / 2)] = __floats2bfloat162_rn((float)d0, (float)d1);
      }
      dst[0] = __floats2bfloat162_rn((float)F0, (float)F1);
    }
  }
}

// ------------------------------------------------------------------------------------------ products

__device__ __forceinline__ void tri_index_emu(int t, int T, int& bi, int& bj) {
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

// One matrix of a work list: its order, its first row in the packed layout, its epilogue coefficients.
struct EmuMat {
  int n, row0;
  double a, b, c;
};

struct EmuArgs {
  int S;                 // digit planes per operand
  int R;                 // rows of one digit plane (the packed row count)
  int ld;                // leading dimension of the FP64 outputs and of cin
  int ntiles;            // work items
  int T;                 // one matrix: tiles per side (items enumerated implicitly)
  const int4* items;     // a batch: (matrix, bi, bj, -) per work item; null for one matrix
  const EmuMat* mats;    // a batch: per-matrix data
  EmuMat one;            // one matrix: its data
  int transpose;         // full mode: store P^T
  Epilogue e;            // output pointers are the bases of the (packed) FP64 buffers
  const int* ex;         // row exponents of X (indexed by packed row)
  const int* ey;         // row exponents of Y
  int* err;
};

template <bool SYM>
__device__ __forceinline__ const EmuMat& item_of(const EmuArgs& a, int t, int& bi, int& bj) {
  if (a.items) {
    const int4 it = a.items[t];
    bi = it.y;
    bj = it.z;
    return a.mats[it.x];
  }
  if (SYM) {
    tri_index_emu(t, a.T, bi, bj);
  } else {
    bi = t % a.T;
    bj = t / a.T;
  }
  return a.one;
}


// x * 2^E for a finite double, by adding to the exponent field when the result stays normal.
__device__ __forceinline__ double scale2(double x, int E) {
  if (x == 0.0) return 0.0;
  const long long u = __double_as_longlong(x);
  const int be = (int)((u >> 52) & 0x7ff) + E;
  if (be > 0 && be < 2047 && ((u >> 52) & 0x7ff) != 0) return __longlong_as_double(u + ((long long)E << 52));
  return ldexp(x, E);
}

template <bool SYM>
__global__ void __launch_bounds__(THREADS, 1)
    k_gemm_emu(const __grid_constant__ CUtensorMap tmX, const __grid_constant__ CUtensorMap tmY, EmuArgs args) {
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  uint8_t* ring = smem;
  uint64_t* bars = reinterpret_cast<uint64_t*>(smem + ESTAGES * STAGE_BYTES);
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(bars + 2 * ESTAGES + 5);
  volatile int* s_abort = reinterpret_cast<volatile int*>(tmem_slot + 1);

  const int S = args.S, R = args.R, ld = args.ld, warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const uint32_t full0 = ptx::smem_u32(bars), empty0 = full0 + 8 * ESTAGES, tfull0 = empty0 + 8 * ESTAGES,
                 tempty0 = tfull0 + 16, drain = tempty0 + 16;

  if (threadIdx.x == 0) {
    for (int s = 0; s < ESTAGES; ++s) {
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
    ptx::tmem_alloc(ptx::smem_u32(tmem_slot), 512);
    ptx::tmem_relinquish();
  }
  ptx::tc_fence_before();
  __syncthreads();
  ptx::tc_fence_after();
  const uint32_t tmem = *tmem_slot;

  if (warp == 0) {
    if (lane == 0) {
      // ---------------- TMA producer: for every tile, pair (by level) and K chunk, the K blocks of the chunk
      int it = 0;
      bool stop = false;
      for (int t = blockIdx.x; t < args.ntiles && !stop; t += gridDim.x) {
        int bi, bj;
        const EmuMat& mt = item_of<SYM>(args, t, bi, bj);
        const int KB = (mt.n + EBK - 1) / EBK;
        for (int L = 2; L <= S + 1 && !stop; ++L)
          for (int s = 1; s <= L - 1 && !stop; ++s) {
            const int ya = (s - 1) * R + mt.row0 + bi * EBM, yb = (L - s - 1) * R + mt.row0 + bj * EBN;
            for (int kb = 0; kb < KB; ++kb, ++it) {
              const int st = it % ESTAGES;
              if (*s_abort || !ptx::mbar_wait(empty0 + 8 * st, ((it / ESTAGES) & 1) ^ 1, args.err, 11)) {
                *s_abort = 1;
                stop = true;
                break;
              }
              uint8_t* sp = ring + st * STAGE_BYTES;
              ptx::mbar_expect_tx(full0 + 8 * st, STAGE_BYTES);
              ptx::tma_load_2d(ptx::smem_u32(sp), &tmX, full0 + 8 * st, kb * EBK, ya);
              ptx::tma_load_2d(ptx::smem_u32(sp + BOX_BYTES), &tmY, full0 + 8 * st, kb * EBK, yb);
            }
          }
      }
      if (*s_abort) {
        for (int k = (it > ESTAGES ? it - ESTAGES : 0); k < it; ++k)
          ptx::mbar_wait(full0 + 8 * (k % ESTAGES), (k / ESTAGES) & 1, nullptr, 0);
      }
    }
  } else if (warp == 1) {
    if (lane == 0) {
      // ---------------- MMA issuer: one "unit" = one pair over one K chunk, into TMEM buffer (unit & 1)
      int it = 0, u = 0;
      bool stop = false;
      for (int t = blockIdx.x; t < args.ntiles && !stop; t += gridDim.x) {
        int bi, bj;
        const EmuMat& mt = item_of<SYM>(args, t, bi, bj);
        const int KB = (mt.n + EBK - 1) / EBK, nchunks = (KB + KCHUNK_BLOCKS - 1) / KCHUNK_BLOCKS;
        for (int L = 2; L <= S + 1 && !stop; ++L)
          for (int s = 1; s <= L - 1 && !stop; ++s)
            for (int c = 0; c < nchunks && !stop; ++c, ++u) {
              const int b = u & 1;
              if (*s_abort || !ptx::mbar_wait(tempty0 + 8 * b, ((u >> 1) & 1) ^ 1, args.err, 12)) {
                *s_abort = 1;
                stop = true;
                break;
              }
              ptx::tc_fence_after();
              const uint32_t d = tmem + (uint32_t)(b * EBN);
              const int kb0 = c * KCHUNK_BLOCKS, kb1 = min(KB, kb0 + KCHUNK_BLOCKS);
              for (int kb = kb0; kb < kb1; ++kb) {
                const int cur = it + (kb - kb0);
                const int st = cur % ESTAGES;
                if (*s_abort || !ptx::mbar_wait(full0 + 8 * st, (cur / ESTAGES) & 1, args.err, 13)) {
                  *s_abort = 1;
                  stop = true;
                  break;
                }
                ptx::tc_fence_after();
                const uint32_t sa = ptx::smem_u32(ring + st * STAGE_BYTES);
                const uint64_t da = ptx::desc_sw128_kmajor(sa), db = ptx::desc_sw128_kmajor(sa + BOX_BYTES);
#pragma unroll
                for (int kk = 0; kk < EBK / 16; ++kk)
                  ptx::mma_f16(d, da + 2 * kk, db + 2 * kk, kIdesc, (kb != kb0 || kk != 0) ? 1u : 0u);
                ptx::mma_commit(empty0 + 8 * st);
              }
              it += kb1 - kb0;
              if (stop) break;
              ptx::mma_commit(tfull0 + 8 * b);
            }
      }
      ptx::mma_commit(drain);
      ptx::mbar_wait(drain, 0, nullptr, 0);
    }
  } else {
    // ---------------- epilogue warps: quadrant q (TMEM lanes 32q..), column half h (64 columns)
    // Levels are summed exactly in int64, Horner-style over groups of up to kGroup levels (a group's
    // sum stays below 2^63); only at a group end is the group added into the FP64 total in TMEM.
    const int q = warp & 3, h = (warp - 2) >> 2;
    const Epilogue& e = args.e;
    const uint32_t lane_off = (uint32_t)(32 * q) << 16;
    int u = 0;
    bool stop = false;
    for (int t = blockIdx.x; t < args.ntiles && !stop; t += gridDim.x) {
      int bi, bj;
      const EmuMat& mt = item_of<SYM>(args, t, bi, bj);
      const int n = mt.n, row0 = mt.row0;
      const int nchunks = ((n + EBK - 1) / EBK + KCHUNK_BLOCKS - 1) / KCHUNK_BLOCKS;
      bool first_group = true;
      for (int g0 = 2; g0 <= S + 1 && !stop; g0 += kGroup) {
        const int glast = min(g0 + kGroup - 1, S + 1);
        long long acc[64];
#pragma unroll
        for (int c = 0; c < 64; ++c) acc[c] = 0;
        for (int L = g0; L <= glast && !stop; ++L) {
          const int shift = 7 * (glast - L);
          for (int s = 1; s <= L - 1 && !stop; ++s)
            for (int c = 0; c < nchunks; ++c, ++u) {
              if (__shfl_sync(0xffffffffu, *s_abort, 0)) { stop = true; break; }
              const int b = u & 1;
              if (!__all_sync(0xffffffffu, ptx::mbar_wait(tfull0 + 8 * b, (u >> 1) & 1, args.err, 14))) {
                *s_abort = 1;
                stop = true;
                break;
              }
              ptx::tc_fence_after();
#pragma unroll
              for (int half = 0; half < 2; ++half) {
                uint32_t v[32];
                ptx::tmem_ld_32x32b_x32(tmem + lane_off + (uint32_t)(b * EBN + 64 * h + 32 * half), v);
                ptx::tmem_ld_wait();
#pragma unroll
                for (int c2 = 0; c2 < 32; ++c2)
                  acc[32 * half + c2] += (long long)__float2int_rn(__uint_as_float(v[c2])) << shift;
              }
              ptx::tc_fence_before();
              __syncwarp();
              if (lane == 0) ptx::mbar_arrive(tempty0 + 8 * b);
            }
        }
        if (stop) break;
        // Group end: total (+)= acc 2^(-7 glast); FP64 words in TMEM, 16 elements (32 words) per access.
#pragma unroll
        for (int g = 0; g < 4; ++g) {
          const uint32_t ta = tmem + lane_off + (uint32_t)(TOTAL_COL + 128 * h + 32 * g);
          uint32_t w[32];
          if (!first_group) {
            ptx::tmem_ld_32x32b_x32(ta, w);
            ptx::tmem_ld_wait();
          }
#pragma unroll
          for (int c2 = 0; c2 < 16; ++c2) {
            double tot = scale2((double)acc[16 * g + c2], -7 * glast);
            if (!first_group) tot += __hiloint2double((int)w[2 * c2 + 1], (int)w[2 * c2]);
            w[2 * c2] = (uint32_t)__double2loint(tot);
            w[2 * c2 + 1] = (uint32_t)__double2hiint(tot);
          }
          ptx::tmem_st_32x32b_x32(ta, w);
          ptx::tmem_st_wait();
        }
        first_group = false;
      }
      if (stop) break;
      // Tile end: P = 2^(e_i + f_j) total, then the fused epilogue (FP64 values, FP32 residual partials).
      const int i = bi * EBM + 32 * q + lane;
      const int ei = i < n ? args.ex[row0 + i] : 0;
      float part = 0.0f;
#pragma unroll 1
      for (int g = 0; g < 4; ++g) {
        uint32_t w[32];
        ptx::tmem_ld_32x32b_x32(tmem + lane_off + (uint32_t)(TOTAL_COL + 128 * h + 32 * g), w);
        ptx::tmem_ld_wait();
        if (i >= n) continue;
#pragma unroll 4
        for (int c2 = 0; c2 < 16; ++c2) {
          const int j = bj * EBN + 64 * h + 16 * g + c2;
          if (j >= n || (SYM && i > j)) continue;
          const double P = scale2(__hiloint2double((int)w[2 * c2 + 1], (int)w[2 * c2]), ei + args.ey[row0 + j]);
          if (e.partial) {
            const float dd = (float)((i == j ? 1.0 : 0.0) - P);
            part = fmaf((SYM && i != j) ? 2.0f * dd : dd, dd, part);
          }
          const int64_t ij = (int64_t)(row0 + i) * ld + j, ji = (int64_t)(row0 + j) * ld + i;
          double w2 = 0.0;
          if (e.out2) {
            w2 = i == j ? fma(mt.b, P, mt.a) : mt.b * P;
            if (mt.c != 0.0) w2 = fma(mt.c, e.cin[ij], w2);
          }
          const bool direct = SYM || !args.transpose, mirrored = SYM ? (i != j) : (bool)args.transpose;
          if (direct) {
            if (e.out) e.out[ij] = P;
            if (e.out2) e.out2[ij] = w2;
          }
          if (mirrored) {
            if (e.out) e.out[ji] = P;
            if (e.out2) e.out2[ji] = w2;
          }
        }
      }
      if (e.partial) {
        for (int o = 16; o > 0; o >>= 1) part += __shfl_xor_sync(0xffffffffu, part, o);
        if (lane == 0) e.partial[(int64_t)t * EPI_WARPS + (warp - 2)] = (double)part;
      }
    }
  }
  ptx::tc_fence_before();
  __syncthreads();
  ptx::tc_fence_after();
  if (warp == 0) ptx::tmem_dealloc(tmem, 512);
}

PFN_cuTensorMapEncodeTiled_v12000 encode_fn_emu() {
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

// The S digit planes of an operand stacked as an (S R) x K BF16 matrix (leading dimension ldl); boxes of
// 64 (K) x 128 rows. Columns k >= K are outside the tensor and read as zero.
cudaError_t make_slice_map(CUtensorMap* map, const __nv_bfloat16* ptr, int K, int R, int ldl, int S) {
  auto fn = encode_fn_emu();
  if (!fn) return cudaErrorNotSupported;
  cuuint64_t dims[2] = {(cuuint64_t)K, (cuuint64_t)S * (cuuint64_t)R};
  cuuint64_t strides[1] = {(cuuint64_t)ldl * 2};
  cuuint32_t box[2] = {(cuuint32_t)EBK, (cuuint32_t)EBM};
  cuuint32_t estr[2] = {1, 1};
  CUresult r = fn(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<__nv_bfloat16*>(ptr), dims, strides, box, estr,
                  CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                  CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS ? cudaSuccess : cudaErrorInvalidValue;
}

int sm_count_emu() {
  static int count = 0;
  if (!count) {
    int dev = 0;
    cudaGetDevice(&dev);
    if (cudaDeviceGetAttribute(&count, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || count < 1) count = 1;
  }
  return count;
}

cudaError_t launch_emu(const __nv_bfloat16* DX, const __nv_bfloat16* DY, int K, int ldl, Mode mode, EmuArgs& a,
                       cudaStream_t s) {
  if (a.S < 1 || a.S > 9 || ldl % 8 != 0 || ldl < K) return cudaErrorInvalidValue;
  if ((reinterpret_cast<uintptr_t>(DX) | reinterpret_cast<uintptr_t>(DY)) & 15) return cudaErrorMisalignedAddress;
  if ((int64_t)a.S * a.R > (int64_t)1 << 31) return cudaErrorInvalidValue;
  // The int32 level sums hold up to S pairs of K-sums of K terms, each term at most 64 * 64.
  if ((int64_t)a.S * K * 4096 >= (int64_t)1 << 31) return cudaErrorInvalidValue;
  static bool attr_set = false;
  if (!attr_set) {
    cudaError_t r = cudaFuncSetAttribute(k_gemm_emu<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, SMEM_BYTES);
    if (r != cudaSuccess) return r;
    r = cudaFuncSetAttribute(k_gemm_emu<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, SMEM_BYTES);
    if (r != cudaSuccess) return r;
    attr_set = true;
  }
  if (a.ntiles == 0) return cudaSuccess;
  CUtensorMap mx, my;
  cudaError_t r = make_slice_map(&mx, DX, K, a.R, ldl, a.S);
  if (r != cudaSuccess) return r;
  r = make_slice_map(&my, DY, K, a.R, ldl, a.S);
  if (r != cudaSuccess) return r;
  const int grid = a.ntiles < sm_count_emu() ? a.ntiles : sm_count_emu();
  if (mode == Mode::Sym) {
    k_gemm_emu<true><<<grid, THREADS, SMEM_BYTES, s>>>(mx, my, a);
  } else {
    k_gemm_emu<false><<<grid, THREADS, SMEM_BYTES, s>>>(mx, my, a);
  }
  return cudaGetLastError();
}

}  // namespace

int emu_tiles(int n, Mode mode) {
  const int T = (n + EBM - 1) / EBM;
  return (mode == Mode::Sym ? T * (T + 1) / 2 : T * T) * EPI_WARPS;  // one partial per epilogue warp and tile
}

int emu_partials_per_item() { return EPI_WARPS; }

cudaError_t slice(const double* X, int n, int ldl, int S, __nv_bfloat16* D, int* ex, cudaStream_t s) {
  return slice_rows(X, n, n, n, ldl, S, nullptr, D, ex, s);
}

cudaError_t slice_rows(const double* X, int R, int n, int ldx, int ldl, int S, const int* row_n, __nv_bfloat16* D,
                       int* ex, cudaStream_t s) {
  int blocks = (R + 7) / 8;  // 8 warps (rows) per block
  if (blocks > 152 * 8) blocks = 152 * 8;
  if (blocks < 1) return cudaSuccess;
  k_slice<<<blocks, 256, 0, s>>>(X, R, n, ldx, ldl, S, row_n, D, ex);
  return cudaGetLastError();
}

cudaError_t gemm_emu(const __nv_bfloat16* DX, const int* ex, const __nv_bfloat16* DY, const int* ey, int n, int ldl,
                     int S, Mode mode, bool transpose, const Epilogue& e, int* err, cudaStream_t s) {
  EmuArgs a{};
  a.S = S;
  a.R = n;
  a.ld = n;
  a.T = (n + EBM - 1) / EBM;
  a.ntiles = mode == Mode::Sym ? a.T * (a.T + 1) / 2 : a.T * a.T;
  a.items = nullptr;
  a.mats = nullptr;
  a.one = EmuMat{n, 0, e.a, e.b, e.c};
  a.transpose = transpose ? 1 : 0;
  a.e = e;
  a.ex = ex;
  a.ey = ey;
  a.err = err;
  return launch_emu(DX, DY, n, ldl, mode, a, s);
}

cudaError_t gemm_emu_batched(const __nv_bfloat16* DX, const int* ex, const __nv_bfloat16* DY, const int* ey, int R,
                             int K, int ldl, int ld, int S, Mode mode, bool transpose, const int4* items, int nitems,
                             const EmuBatchMat* mats, const Epilogue& e, int* err, cudaStream_t s) {
  static_assert(sizeof(EmuBatchMat) == sizeof(EmuMat), "batch matrix record");
  EmuArgs a{};
  a.S = S;
  a.R = R;
  a.ld = ld;
  a.T = 0;
  a.ntiles = nitems;
  a.items = items;
  a.mats = reinterpret_cast<const EmuMat*>(mats);
  a.transpose = transpose ? 1 : 0;
  a.e = e;
  a.ex = ex;
  a.ey = ey;
  a.err = err;
  return launch_emu(DX, DY, K, ldl, mode, a, s);
}

}  // namespace pr
