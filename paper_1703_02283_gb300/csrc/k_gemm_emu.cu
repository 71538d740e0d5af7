// FP64-accurate matrix products from exact FP16 digit slices on the tcgen05 tensor cores (PR_EMU64).
//
// GB300 executes FP64 at about 1/1800 of its half-precision tensor rate, so the FP64-accurate iterations
// of Eq. 1 (Sec. 3: precise refinement) are built from exact low-precision pieces, following the
// error-free splitting of Ozaki, Ogita, Oishi and Rump ("Error-free transformations of matrix
// multiplication by using fast routines of matrix multiplication and its applications", Numer.
// Algorithms 59, 2012):
//
//  * slicing (k_slice): for row i of X let e_i be the smallest integer with max_k |x_ik| < 2^(e_i - 1). The
//    integer F_ik = round(x_ik 2^(8S - e_i)) (|F| < 2^(8S - 1)) is written in balanced base 256,
//    F = sum_{s=1..S} d_s 256^(S-s) with |d_s| <= 128, so x_ik = 2^e_i sum_s d_s 2^(-8s) up to 2^(e_i - 8S - 1).
//    The digits are small integers, exact in FP16. Integer arithmetic only.
//  * products (k_gemm_emu): P_ij = 2^(e_i + f_j) sum_{L=2..S+1} 2^(-8L) V_L with the level sums
//    V_L = sum_{s + t = L} sum_k dX_s,ik dY_t,jk. Each digit product is at most 2^14 in magnitude, so a
//    level of m pairs summed over 16 P values of k with m P <= 64 stays within 2^24 and the FP32
//    accumulation of the tensor cores is exact (P = 8 steps for the 8-pair level, up to 64 for one pair). Dropping the pairs with s + t > S + 1 and the digits beyond S leaves an
//    error of about (S + 2) 2^(-8S - 2) in units of 2^(e_i + f_j) per product term: S = 8 (the default)
//    gives 2^-63. F must fit in 64-bit integers, which limits S to 8.
//
// Data movement. All digit planes of both operands for one 16-wide step of k sit in shared memory at
// once (one TMA box per operand and plane group), and every pair (s, t) of the step is issued from them:
// each plane is fetched once per step instead of once per pair. In memory the 16 digits of a step are
// stored for 4 planes side by side (layout [row][step][plane][16]), so a box row is 128 contiguous bytes
// (one request) and lands 128-byte swizzled in shared memory, where plane s is the 32-byte K slice s % 4
// of group s / 4. The planes of X are copied into tensor memory (tcgen05.cp) and the MMAs read them there;
// shared memory serves only the Y planes to the tensor cores (both operands from shared memory would cap
// the tensor cores at the 128 bytes per clock that shared memory delivers).
//
// k_gemm_emu is a persistent kernel, one CTA per SM, 128 x 96 output tiles taken from a work list
// (matrix, tile row, tile column). Tensor memory holds four FP32 level accumulators of 96 columns and two
// 64-column buffers of X planes, so a tile takes two passes over k: levels 2..5 (digits 1..4 only) and
// levels 6..9. 640 threads: warp 0 TMA producer (4-stage ring), warp 1 copies the X planes into TMEM,
// warps 2-3 issue the MMAs (warp w owns accumulators 3 - w and w: 5 and 13 pairs per step; all 32 lanes
// run the loop on warp-uniform values and one elected lane issues each instruction), warps 4-19 epilogue
// (four warps per TMEM lane quadrant, 24 columns each). An accumulator is drained every P steps (8 to 64,
// by its level's pair count), staggered: the epilogue warps load its columns, release it, convert the
// exact FP32 values to integers and add them, shifted, into an exact int64 total per element. The
// first pass's totals wait in a scratch buffer; at the tile's end the 128-bit total hi 2^32 + lo is
// rounded once to FP64 (integer arithmetic), scaled by 2^(e_i + f_j) and the fused epilogue applied.
// Every wait is bounded as in k_gemm_tc.cu.
//
// Split tiles (the SPLIT variant). A short single-matrix launch whose tiles fill the SMs for a fraction of
// a wave is given every tile as two items over halves of k (emu_launch_list). Each half ends with exact
// int64 totals; the epilogue warp of the half that finishes second (one atomic counter per tile and warp)
// adds the other half's totals to its own, which is exact and independent of the order, and applies the
// epilogue. No warp waits for another CTA. Residual partials are indexed by tile, as without splitting.
#include "pr_internal.h"
#include "tc_ptx.h"

#include <cuda_fp16.h>
#include <cudaTypedefs.h>

#include <algorithm>
#include <vector>

namespace pr {
namespace {

constexpr int EBM = 128, EBK = 16, SMAX = 8, BAND = 8, NSTAGE = 4;
constexpr int NACC = 4;                  // level accumulators in TMEM: levels 2..5 (pass 0), 6..9 (pass 1)
constexpr int MMA_WARPS = 2, EPI_WARPS = 16, THREADS = 32 * (2 + MMA_WARPS + EPI_WARPS);
constexpr int A_GROUP = EBM * 128;       // bytes of 4 planes of the X tile (one 128-byte row per row)
constexpr int A_BYTES = 2 * A_GROUP;
constexpr int NBARS = 2 * NSTAGE + 2 * NACC + 2 + 1;
constexpr int BN_WIDE = 96, BN_NARROW = 48;  // the two tile widths (output columns per tile)

// What depends on the tile width BN (the N of every MMA and the rows of Y per stage).
template <int BN>
struct EmuTile {
  static constexpr int EPI_COLS = BN / 4;     // columns per epilogue warp (four warps per TMEM lane quadrant)
  static constexpr int B_GROUP = BN * 128;    // bytes of 4 planes of the Y tile
  static constexpr int STAGE_BYTES = A_BYTES + 2 * B_GROUP;
  static constexpr int SMEM_BYTES = 1024 + NSTAGE * STAGE_BYTES + 8 * NBARS + 16;
  static constexpr int ACOL = NACC * BN;      // TMEM column of the first X-plane buffer (after the accumulators)
  static constexpr int SCRATCH_PER_CTA = 2 * EPI_WARPS * 32 * EPI_COLS;  // int64 totals: first pass, then lo
  static constexpr int SPLIT_PER_PART = 2 * EPI_WARPS * 32 * EPI_COLS;   // int64: (hi, lo) per tile element
  static constexpr uint32_t kIdesc = ptx::idesc_f16_f32(EBM, BN);
  static_assert(BN % 16 == 0 && BN <= 256, "MMA N for M = 128");
  static_assert(ACOL + 2 * SMAX * 8 <= 512, "tensor memory budget");
  static_assert(STAGE_BYTES % 1024 == 0 && B_GROUP % 1024 == 0, "1024-byte aligned swizzle atoms");
  static_assert(SMEM_BYTES <= 232448, "shared memory");
  static_assert(EPI_COLS == 24 || EPI_COLS == 12, "epilogue column split");
};

// ------------------------------------------------------------------------------------------ slicing

__device__ __forceinline__ unsigned long long warp_max_u64(unsigned long long v) {
  for (int o = 16; o > 0; o >>= 1) {
    const unsigned long long w = __shfl_xor_sync(0xffffffffu, v, o);
    v = w > v ? w : v;
  }
  return v;
}

// F = round(x 2^(8S - e)) of one double as an integer (|F| < 2^(8S - 1) for |x| < 2^(e - 1)).
__device__ __forceinline__ long long fixed_point(unsigned long long u, int e, int S) {
  const int E = (int)((u >> 52) & 0x7ff);
  if (E == 0) return 0;  // zero, or a subnormal far below the last digit
  const unsigned long long M = (u & 0xfffffffffffffull) | (1ull << 52);
  const int sh = (E - 1023) - e + 8 * S - 52;  // F = M 2^sh, sh <= 8S - 54
  long long F = 0;
  if (sh >= 0) F = (long long)(M << sh);
  else if (sh > -64) F = (long long)((M + (1ull << (-sh - 1))) >> (-sh));
  return (u >> 63) ? -F : F;
}

// One 128-thread block per row r of an R-row FP64 array (leading dimension ldx): exponent e_r, then 8
// digit planes in the layout D[r][k / 16][s][k % 16] (row length 8 ldl halves, ldl a multiple of 16; s = 0
// is the most significant digit, planes s >= S are zero). Row r has row_n[r] valid columns (all rows n when
// row_n is null); columns from there up to the next multiple of 16 (the last step the products read for that
// row's matrix) get digit 0, later columns are left as they are; rows with row_n[r] < 0 are skipped.
// Each thread takes 8 consecutive columns at a time: two 16-byte loads per pair of columns when the row is
// 16-byte aligned, and one 16-byte store per digit plane (half a step's plane).
constexpr int SLICE_THREADS = 128;

__device__ __forceinline__ void balanced_digits(long long F, int S, int (&d)[SMAX]) {
  if (S == SMAX) {
    // Balanced base-256 digits in 32-bit arithmetic: digit k (least significant first) is
    // v = byte_k(F) + c minus 256 c' with carry c' = (v >= 128); the top digit is (F >> 56) + c.
    // (The same digits as the 64-bit recurrence F <- (F - d) >> 8 below.)
    const unsigned lo = (unsigned)F, hu = (unsigned)(F >> 32);
    int c = 0;
#pragma unroll
    for (int k = 0; k < SMAX - 1; ++k) {
      const int v = (int)(((k < 4 ? lo >> (8 * k) : hu >> (8 * (k - 4)))) & 255u) + c;
      c = v >= 128 ? 1 : 0;
      d[SMAX - 1 - k] = v - 256 * c;
    }
    d[0] = ((int)hu >> 24) + c;
  } else {
    // Balanced base-256 digits, least significant first (digit S - 1 down to 1); the most significant one
    // takes the remainder (|.| <= 128); planes S .. 7 are zero.
#pragma unroll
    for (int s = SMAX - 1; s >= 1; --s) {
      if (s < S) {
        const int r = (int)(F & 255);
        const int dd = r >= 128 ? r - 256 : r;
        F = (F - dd) >> 8;
        d[s] = dd;
      } else {
        d[s] = 0;
      }
    }
    d[0] = (int)F;
  }
}

__global__ void __launch_bounds__(SLICE_THREADS) k_slice(const double* __restrict__ X, int R, int n, int ldx, int ldl,
                                                         int S, const int* __restrict__ row_n, __half* __restrict__ D,
                                                         int* __restrict__ ex) {
  __shared__ unsigned long long red[SLICE_THREADS / 32];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int i = blockIdx.x; i < R; i += gridDim.x) {
    const int nr = row_n ? row_n[i] : n;  // uniform over the block
    if (nr < 0) continue;
    const double* rowd = X + (int64_t)i * ldx;
    const unsigned long long* row = reinterpret_cast<const unsigned long long*>(rowd);
    const bool vec = (reinterpret_cast<uintptr_t>(rowd) & 15) == 0;
    unsigned long long mb = 0;  // largest |x| as a bit pattern (non-negative doubles order like integers)
    for (int k = 8 * threadIdx.x; k < nr; k += 8 * SLICE_THREADS) {
      if (vec && k + 8 <= nr) {
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          const ulonglong2 u = *reinterpret_cast<const ulonglong2*>(row + k + 2 * q);
          const unsigned long long a = u.x & 0x7fffffffffffffffull, b = u.y & 0x7fffffffffffffffull;
          mb = a > mb ? a : mb;
          mb = b > mb ? b : mb;
        }
      } else {
        for (int q = 0; q < 8 && k + q < nr; ++q) {
          const unsigned long long a = row[k + q] & 0x7fffffffffffffffull;
          mb = a > mb ? a : mb;
        }
      }
    }
    mb = warp_max_u64(mb);
    if (lane == 0) red[warp] = mb;
    __syncthreads();
    mb = red[0];
#pragma unroll
    for (int w = 1; w < SLICE_THREADS / 32; ++w) mb = red[w] > mb ? red[w] : mb;
    __syncthreads();  // red is reused by the next row
    const int emax = (int)(mb >> 52);               // biased exponent of the row maximum
    const int e = emax == 0 ? 0 : emax - 1023 + 2;  // zero (or subnormal-only) rows get digits 0
    if (threadIdx.x == 0) ex[i] = e;
    const int kend = min(ldl, (nr + 15) & ~15);
    for (int k = 8 * threadIdx.x; k < kend; k += 8 * SLICE_THREADS) {
      unsigned long long u[8];
      if (vec && k + 8 <= nr) {
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          const ulonglong2 w2 = *reinterpret_cast<const ulonglong2*>(row + k + 2 * q);
          u[2 * q] = w2.x;
          u[2 * q + 1] = w2.y;
        }
      } else {
#pragma unroll
        for (int q = 0; q < 8; ++q) u[q] = k + q < nr ? row[k + q] : 0ull;
      }
      uint32_t h2[SMAX][4];  // plane s, column pair c: two halves
#pragma unroll
      for (int c = 0; c < 4; ++c) {
        int d0[SMAX], d1[SMAX];
        balanced_digits(emax != 0 && k + 2 * c < nr ? fixed_point(u[2 * c], e, S) : 0ll, S, d0);
        balanced_digits(emax != 0 && k + 2 * c + 1 < nr ? fixed_point(u[2 * c + 1], e, S) : 0ll, S, d1);
#pragma unroll
        for (int s = 0; s < SMAX; ++s) {
          const __half2 v = __floats2half2_rn((float)d0[s], (float)d1[s]);
          h2[s][c] = *reinterpret_cast<const uint32_t*>(&v);
        }
      }
      uint4* dst = reinterpret_cast<uint4*>(D + (int64_t)i * 8 * ldl + (k >> 4) * 128 + (k & 15));
#pragma unroll
      for (int s = 0; s < SMAX; ++s) dst[2 * s] = make_uint4(h2[s][0], h2[s][1], h2[s][2], h2[s][3]);
    }
  }
}

// ------------------------------------------------------------------------------------------ products

// One matrix of a work list: its order, its first row in the packed layout, its epilogue coefficients.
struct EmuMat {
  int n, row0;
  double a, b, c;
};

struct EmuArgs {
  int S;                 // digit planes per operand
  int ld;                // leading dimension of the FP64 outputs and of cin
  int ntiles;            // work items
  const int* ntiles_dev; // if set, the number of work items is read here (written by an earlier kernel)
  const int4* items;     // (matrix, tile row, tile column, part) per work item (part 0: the whole tile)
  const EmuMat* mats;    // per-matrix data; null: every item belongs to `one`
  EmuMat one;
  int transpose;         // full mode: store P^T
  Epilogue e;            // output pointers are the bases of the (packed) FP64 buffers
  const int* ex;         // row exponents of X (indexed by packed row)
  const int* ey;         // row exponents of Y
  long long* scratch;    // EmuTile::SCRATCH_PER_CTA int64 per CTA: the first pass's exact totals
  int* err;
  unsigned long long* tstamp;  // if set: [0] min over CTAs of the start time, [1] max of the end time (ns)
  long long* split;      // split tiles: per slot, 2 parts x SPLIT_PER_PART exact totals (hi, lo pairs)
  int* split_cnt;        // split tiles: per slot and epilogue warp, the parts finished so far (reset to 0)
};

// Item t: its matrix, tile, and the K steps [j0, j1) it covers. kpart = 0 is the whole tile; a tile split in
// two has items with kpart = 1 + 2 slot + half, half 0 taking the first KS / 2 steps and half 1 the rest.
// Unsplit items with w > 0 cover only the steps [w >> 16, w & 0xffff) (block-sparse operands: the digits of
// every other step are zero for the rows of the tile, so those steps add exact zeros; emu_range_item).
template <bool SPLIT>
__device__ __forceinline__ const EmuMat& item_of(const EmuArgs& a, int t, int& bi, int& bj, int& kpart, int& j0,
                                                 int& j1) {
  const int4 it = a.items[t];
  bi = it.y;
  bj = it.z;
  const EmuMat& mt = a.mats ? a.mats[it.x] : a.one;
  const int KS = (mt.n + EBK - 1) / EBK;
  if constexpr (SPLIT) {
    const int h = KS >> 1;
    kpart = it.w;
    j0 = kpart == 0 || ((kpart - 1) & 1) == 0 ? 0 : h;
    j1 = kpart == 0 || ((kpart - 1) & 1) == 1 ? KS : h;
  } else {
    kpart = 0;
    j0 = it.w > 0 ? (it.w >> 16) : 0;
    j1 = it.w > 0 ? (it.w & 0xffff) : KS;
  }
  return mt;
}

// (H 2^64 + Lw) 2^E0 for a two's-complement 128-bit integer H:Lw, rounded once to the nearest double
// (ties to even), in integer arithmetic.
__device__ __noinline__ double wide_to_double(long long H, unsigned long long Lw, int E0) {
  const unsigned long long sign = (unsigned long long)H & 0x8000000000000000ull;
  unsigned long long mh = (unsigned long long)H, ml = Lw;
  if (sign) {
    ml = ~ml + 1ull;
    mh = ~mh + (ml == 0ull ? 1ull : 0ull);
  }
  if ((mh | ml) == 0ull) return 0.0;
  const int lz = mh ? __clzll((long long)mh) : 64 + __clzll((long long)ml);
  if (lz >= 64) {
    mh = ml << (lz - 64);
    ml = 0ull;
  } else if (lz > 0) {
    mh = (mh << lz) | (ml >> (64 - lz));
    ml <<= lz;
  }
  unsigned long long mant = mh >> 11;  // 53 bits, the leading one at bit 52
  const unsigned long long rest = mh & 0x7ffull;
  if (rest > 0x400ull || (rest == 0x400ull && (ml != 0ull || (mant & 1ull)))) ++mant;
  int ex = 127 - lz + E0;  // exponent of the leading one
  if (mant >> 53) {
    mant >>= 1;
    ++ex;
  }
  const int be = ex + 1023;
  if (be >= 1 && be <= 2046)
    return __longlong_as_double((long long)(sign | ((unsigned long long)be << 52) | (mant & 0xfffffffffffffull)));
  const double v = ldexp((double)mant, ex - 52);  // outside the normal range
  return sign ? -v : v;
}

// The MMAs of one level L for S = 8 (pairs s = 1 .. L - 1, t = L - s), unrolled: X plane s - 1 from TMEM
// buffer aT, Y plane t - 1 from the shared-memory stage whose first plane group has descriptor bdesc.
template <int BN, int L>
struct MmaLevel {
  __device__ __forceinline__ void operator()(uint32_t d, uint32_t aT, uint64_t bdesc, bool fresh) const {
    using T = EmuTile<BN>;
#pragma unroll
    for (int s = 1; s <= L - 1; ++s) {
      const int t = L - s - 1;
      ptx::mma_f16_ts_w(d, aT + 8 * (s - 1), bdesc + (uint64_t)(((t >> 2) * T::B_GROUP + (t & 3) * 32) >> 4),
                        T::kIdesc, (fresh && s == 1) ? 0u : 1u);
    }
  }
};

// Drain period of level L: the largest power of two P <= 64 with m P <= 64 for the level's m digit pairs
// (m pairs x P steps x 16 values of k x 2^14 <= 2^24 keeps the level's FP32 sum exact). Accumulator a of a
// pass is drained after step j when (j + 2a) % P == P - 1 (the offsets stagger the drains) and after the
// pass's last step.
// 16-wide K chunks per pipeline step. The first pass moves one plane group per chunk, so a stage (and an
// X-plane buffer in TMEM) holds two chunks: chunk c's planes take the slots of the second pass's group c.
__device__ __forceinline__ int chunks_per_step(int pass) { return pass == 0 ? 2 : 1; }

__device__ __forceinline__ int drain_period(int L, int S) {
  const int m = min(S, L - 1) - max(1, L - S) + 1;
  return m <= 1 ? 64 : m <= 2 ? 32 : m <= 4 ? 16 : 8;
}

template <int BN, bool SYM, bool SPLIT>
__global__ void __launch_bounds__(THREADS, 1)  // 20 warps: up to 96 registers (5 warps per sub-partition)
    k_gemm_emu(const __grid_constant__ CUtensorMap tmX, const __grid_constant__ CUtensorMap tmY, EmuArgs args) {
  using T = EmuTile<BN>;
  constexpr int EPI_COLS = T::EPI_COLS, B_GROUP = T::B_GROUP, STAGE_BYTES = T::STAGE_BYTES, ACOL = T::ACOL;
  constexpr int SCRATCH_PER_CTA = T::SCRATCH_PER_CTA, SPLIT_PER_PART = T::SPLIT_PER_PART;
  constexpr uint32_t kIdesc = T::kIdesc;
  const int ntiles = args.ntiles_dev ? *args.ntiles_dev : args.ntiles;
  if ((int)blockIdx.x >= ntiles) return;  // no work for this CTA (uniform over the block)
  if (args.tstamp && threadIdx.x == 0) atomicMin(&args.tstamp[0], (unsigned long long)ptx::globaltimer());
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  uint8_t* ring = smem;
  uint64_t* bars = reinterpret_cast<uint64_t*>(smem + NSTAGE * STAGE_BYTES);
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(bars + NBARS);
  volatile int* s_abort = reinterpret_cast<volatile int*>(tmem_slot + 1);

  const int S = args.S, warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const uint32_t full0 = ptx::smem_u32(bars), empty0 = full0 + 8 * NSTAGE, lfull0 = empty0 + 8 * NSTAGE,
                 lempty0 = lfull0 + 8 * NACC, aready0 = lempty0 + 8 * NACC, drain = aready0 + 16;

  if (threadIdx.x == 0) {
    for (int s = 0; s < NSTAGE; ++s) {
      ptx::mbar_init(full0 + 8 * s, 1);
      ptx::mbar_init(empty0 + 8 * s, MMA_WARPS + 1);  // the MMA warps and the copy thread read the stage
    }
    for (int a = 0; a < NACC; ++a) {
      ptx::mbar_init(lfull0 + 8 * a, 1);
      ptx::mbar_init(lempty0 + 8 * a, EPI_WARPS);
    }
    for (int b = 0; b < 2; ++b) ptx::mbar_init(aready0 + 8 * b, 1);
    ptx::mbar_init(drain, MMA_WARPS + 1);
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
  // Planes used by a pass: levels 2..5 need digits 1..4 only (one plane group), levels 6..9 all 8. With at
  // most 4 digits (S <= 4) every level is at most 5: the second pass has no work and is skipped.
  const int groups1 = S > 4 ? 2 : 1, npass = S > 4 ? 2 : 1;

  if (warp == 0) {
    if (lane == 0) {
      // ---------------- TMA producer: per step, the plane groups of X (128 rows) and of Y (96 rows)
      int it = 0;
      bool stop = false;
      for (int t = blockIdx.x; t < ntiles && !stop; t += gridDim.x) {
        int bi, bj, kpart, j0, j1;
        const EmuMat& mt = item_of<SPLIT>(args, t, bi, bj, kpart, j0, j1);
        const int ya = mt.row0 + bi * EBM, yb = mt.row0 + bj * BN;
        for (int pass = 0; pass < npass && !stop; ++pass) {
          const int ng = pass == 0 ? 1 : groups1, kc = chunks_per_step(pass);
          for (int j = j0; j < j1; j += kc, ++it) {
            const int st = it % NSTAGE, nc = min(kc, j1 - j);
            if (*s_abort || !ptx::mbar_wait(empty0 + 8 * st, ((it / NSTAGE) & 1) ^ 1, args.err, 11)) {
              *s_abort = 1;
              stop = true;
              break;
            }
            uint8_t* sp = ring + st * STAGE_BYTES;
            ptx::mbar_expect_tx(full0 + 8 * st, (uint32_t)(nc * ng) * (A_GROUP + B_GROUP));
            for (int c = 0; c < nc; ++c) {
              for (int g = 0; g < ng; ++g) {
                const int slot = c * ng + g;
                ptx::tma_load_3d(ptx::smem_u32(sp + slot * A_GROUP), &tmX, full0 + 8 * st, 0, 2 * (j + c) + g, ya);
                ptx::tma_load_3d(ptx::smem_u32(sp + A_BYTES + slot * B_GROUP), &tmY, full0 + 8 * st, 0,
                                 2 * (j + c) + g, yb);
              }
            }
          }
        }
      }
      if (*s_abort) {
        for (int k = (it > NSTAGE ? it - NSTAGE : 0); k < it; ++k)
          ptx::mbar_wait(full0 + 8 * (k % NSTAGE), (k / NSTAGE) & 1, nullptr, 0);
      }
    }
  } else if (warp == 1) {
    // ---------------- copy warp: per step, the X planes of the pass into TMEM buffer (step & 1), once the MMAs
    // of two steps back (the last readers of that buffer) have finished. All 32 lanes run the loop; one
    // elected lane issues.
    int it = 0;
    bool stop = false;
    const uint64_t xdesc0 = ptx::desc_sw128_kmajor(ptx::smem_u32(ring));
    const uint32_t aT0 = tmem + (uint32_t)ACOL;
    auto wait_all = [&](uint32_t bar, uint32_t parity, int code) {
      return __all_sync(0xffffffffu, ptx::mbar_wait(bar, parity, args.err, code));
    };
    // One pass over KS steps; copy(aT, xdesc) copies the pass's planes of the stage with descriptor xdesc.
    auto run_pass = [&](auto copy, int nsteps) -> bool {
      for (int q = 0; q < nsteps; ++q, ++it) {
        const int st = it % NSTAGE, b = it & 1;
        if (!wait_all(full0 + 8 * st, (it / NSTAGE) & 1, 12) ||
            (it >= 2 && !wait_all(empty0 + 8 * ((it - 2) % NSTAGE), ((it - 2) / NSTAGE) & 1, 13)))
          return false;
        ptx::tc_fence_after();
        copy(aT0 + (uint32_t)(64 * b), xdesc0 + (uint64_t)((st * STAGE_BYTES) >> 4));
        ptx::mma_commit_w(aready0 + 8 * b);
        ptx::mma_commit_w(empty0 + 8 * st);
      }
      return true;
    };
    auto planes = [](uint32_t aT, uint64_t xd, int s) {
      ptx::tmem_cp_128x256b_w(aT + 8 * s, xd + (uint64_t)(((s >> 2) * A_GROUP + (s & 3) * 32) >> 4));
    };
    for (int t = blockIdx.x; t < ntiles && !stop; t += gridDim.x) {
      int bi, bj, kpart, j0, j1;
      item_of<SPLIT>(args, t, bi, bj, kpart, j0, j1);
      for (int pass = 0; pass < npass && !stop; ++pass) {
        if (__any_sync(0xffffffffu, *s_abort != 0)) {
          stop = true;
          break;
        }
        // Buffer plane v: the second pass's digit plane v, or in the first pass plane v % 4 of chunk v / 4.
        const int kc = chunks_per_step(pass), np = pass == 0 ? min(S, 4) : S, nsteps = (j1 - j0 + kc - 1) / kc;
        bool ok;
        if (np == 8 || (pass == 0 && np == 4)) {
          ok = run_pass([&](uint32_t aT, uint64_t xd) {
#pragma unroll
            for (int v = 0; v < 8; ++v) planes(aT, xd, v);
          }, nsteps);
        } else {
          ok = run_pass([&](uint32_t aT, uint64_t xd) {
            for (int c = 0; c < kc; ++c)
              for (int s = 0; s < np; ++s) planes(aT, xd, 4 * c + s);
          }, nsteps);
        }
        if (!ok) {
          *s_abort = 1;
          stop = true;
        }
      }
    }
    ptx::mma_commit_w(drain);
    ptx::mbar_wait(drain, 0, nullptr, 0);
  } else if (warp < 2 + MMA_WARPS) {
    // ---------------- MMA warp w: accumulators aH = 3 - w and aL = w of each pass (levels 5 - w, 2 + w in the
    // first pass, 9 - w, 6 + w in the second: 5 and 13 pairs per step for S = 8, the same for both warps).
    // All 32 lanes run the loop on warp-uniform values; one elected lane issues each tcgen05 instruction.
    const int w = warp - 2;
    uint32_t drained = 0u, par = 0u;  // per own accumulator (bit 0: aH, bit 1: aL): drained once / drain parity
    int it = 0;
    bool stop = false;
    const uint64_t bdesc0 = ptx::desc_sw128_kmajor(ptx::smem_u32(ring) + A_BYTES);
    const uint32_t aT0 = tmem + (uint32_t)ACOL;
    auto wait_all = [&](uint32_t bar, uint32_t parity, int code) {
      return __all_sync(0xffffffffu, ptx::mbar_wait(bar, parity, args.err, code));
    };
    // One pass over KS steps with the level issuers iH, iL (iX(d, aT, bdesc, fresh) issues the level's MMAs).
    auto run_pass = [&](auto iH, auto iL, bool useH, bool useL, int pass, int KS) -> bool {
      const int aH = 3 - w, aL = w, LH = 2 + 4 * pass + aH, LL = 2 + 4 * pass + aL;
      const uint32_t dH = tmem + (uint32_t)(BN * aH), dL = tmem + (uint32_t)(BN * aL);
      const int kc = chunks_per_step(pass), nsteps = (KS + kc - 1) / kc;
      const int pmH = drain_period(LH, S) / kc - 1, pmL = drain_period(LL, S) / kc - 1;
      bool fH = true, fL = true;  // the next MMA into the accumulator starts it afresh
      for (int j = 0; j < nsteps; ++j, ++it) {
        const int st = it % NSTAGE, b = it & 1;
        // One wait per step: the copy warp waited for this stage's TMA load before it copied the X planes, so
        // the completion of its copy (aready) also orders the stage's Y planes before these MMAs.
        if (!wait_all(aready0 + 8 * b, (it >> 1) & 1, 15)) return false;
        ptx::tc_fence_after();
        const uint64_t bdesc = bdesc0 + (uint64_t)((st * STAGE_BYTES) >> 4);
        const uint32_t aT = aT0 + (uint32_t)(64 * b);
        const bool last = j == nsteps - 1, two = kc == 2 && kc * j + 1 < KS;  // two chunks in this step
        // A level restarting after a drain waits for the epilogue's release; it goes second.
        const bool waitH = useH && fH && (drained & 1u), waitL = useL && fL && (drained & 2u);
        auto doH = [&]() -> bool {
          if (!useH) return true;
          if (waitH) {
            if (!wait_all(lempty0 + 8 * aH, (par & 1u) ^ 1u, 16)) return false;
            ptx::tc_fence_after();
          }
          iH(dH, aT, bdesc, fH);
          if (two) iH(dH, aT + 32, bdesc + (uint64_t)(B_GROUP >> 4), false);  // chunk 1: planes 4 columns on
          fH = false;
          if (last || ((j + 2 * aH) & pmH) == pmH) {
            ptx::mma_commit_w(lfull0 + 8 * aH);
            par ^= 1u;
            drained |= 1u;
            fH = true;
          }
          return true;
        };
        auto doL = [&]() -> bool {
          if (!useL) return true;
          if (waitL) {
            if (!wait_all(lempty0 + 8 * aL, ((par >> 1) & 1u) ^ 1u, 16)) return false;
            ptx::tc_fence_after();
          }
          iL(dL, aT, bdesc, fL);
          if (two) iL(dL, aT + 32, bdesc + (uint64_t)(B_GROUP >> 4), false);
          fL = false;
          if (last || ((j + 2 * aL) & pmL) == pmL) {
            ptx::mma_commit_w(lfull0 + 8 * aL);
            par ^= 2u;
            drained |= 2u;
            fL = true;
          }
          return true;
        };
        if (waitH ? !(doL() && doH()) : !(doH() && doL())) return false;
        ptx::mma_commit_w(empty0 + 8 * st);
      }
      return true;
    };
    // Any S: the level's pairs s = max(1, L - S) .. min(S, L - 1), t = L - s, in a loop.
    auto level_loop = [&](int L) {
      return [=](uint32_t d, uint32_t aT, uint64_t bdesc, bool fr) {
        const int s0 = max(1, L - S), s1 = min(S, L - 1);
        for (int s = s0; s <= s1; ++s) {
          const int tt = L - s - 1;
          ptx::mma_f16_ts_w(d, aT + 8 * (s - 1), bdesc + (uint64_t)(((tt >> 2) * B_GROUP + (tt & 3) * 32) >> 4),
                            kIdesc, (fr && s == s0) ? 0u : 1u);
        }
      };
    };
    for (int t = blockIdx.x; t < ntiles && !stop; t += gridDim.x) {
      int bi, bj, kpart, j0, j1;
      item_of<SPLIT>(args, t, bi, bj, kpart, j0, j1);
      const int KS = j1 - j0;
      for (int pass = 0; pass < npass && !stop; ++pass) {
        if (__any_sync(0xffffffffu, *s_abort != 0)) {
          stop = true;
          break;
        }
        bool ok;
        // S = 8: the four (warp, pass) level pairs with every MMA unrolled at compile time.
        switch (S == SMAX ? 2 * pass + w : -1) {
          case 0: ok = run_pass(MmaLevel<BN, 5>{}, MmaLevel<BN, 2>{}, true, true, pass, KS); break;
          case 1: ok = run_pass(MmaLevel<BN, 4>{}, MmaLevel<BN, 3>{}, true, true, pass, KS); break;
          case 2: ok = run_pass(MmaLevel<BN, 9>{}, MmaLevel<BN, 6>{}, true, true, pass, KS); break;
          case 3: ok = run_pass(MmaLevel<BN, 8>{}, MmaLevel<BN, 7>{}, true, true, pass, KS); break;
          default: {
            const int LH = 5 - w + 4 * pass, LL = 2 + w + 4 * pass;
            ok = run_pass(level_loop(LH), level_loop(LL), LH <= S + 1, LL <= S + 1, pass, KS);
          }
        }
        if (!ok) {
          *s_abort = 1;
          stop = true;
        }
      }
    }
    ptx::mma_commit_w(drain);
    ptx::mbar_wait(drain, 0, nullptr, 0);
  } else {
    // ---------------- epilogue warps: quadrant q (TMEM lanes 32q..), column quarter h (24 columns)
    const int ew = warp - 2 - MMA_WARPS, q = warp & 3, h = ew >> 2;
    const Epilogue& e = args.e;
    const uint32_t lane_off = (uint32_t)(32 * q) << 16;
    long long* scr = args.scratch + (size_t)blockIdx.x * SCRATCH_PER_CTA + (size_t)(ew * 32 + lane);
    uint32_t epar = 0u;  // per accumulator: parity of the drains taken so far
    bool stop = false;
    for (int t = blockIdx.x; t < ntiles && !stop; t += gridDim.x) {
      int bi, bj, kpart, j0, j1;
      const EmuMat& mt = item_of<SPLIT>(args, t, bi, bj, kpart, j0, j1);
      const int n = mt.n, row0 = mt.row0, KS = j1 - j0;
      // Exact totals: the first pass gives hi = sum_{L<=5} V_L 2^(8(5-L)) (kept in scratch), the second
      // lo = sum_{L>=6} V_L 2^(8(9-L)); P = hi 2^-40 + lo 2^-72.
      long long acc[EPI_COLS];
#pragma unroll
      for (int c = 0; c < EPI_COLS; ++c) acc[c] = 0;
      for (int pass = 0; pass < npass && !stop; ++pass) {
        const int kc = chunks_per_step(pass), nsteps = (KS + kc - 1) / kc;
        int pm[NACC];  // drain period (in steps) - 1 of each accumulator's level; -1: the level is empty
#pragma unroll
        for (int a = 0; a < NACC; ++a) {
          const int L = 2 + 4 * pass + a;
          pm[a] = L > S + 1 ? -1 : drain_period(L, S) / kc - 1;
        }
        for (int j = 0; j < nsteps && !stop; ++j) {
          const bool lastj = j == nsteps - 1;
#pragma unroll
          for (int a = 0; a < NACC; ++a) {
            if (pm[a] < 0 || !(lastj || ((j + 2 * a) & pm[a]) == pm[a])) continue;
            if (__shfl_sync(0xffffffffu, *s_abort, 0)) {
              stop = true;
              break;
            }
            if (!__all_sync(0xffffffffu, ptx::mbar_wait(lfull0 + 8 * a, (epar >> a) & 1u, args.err, 17))) {
              *s_abort = 1;
              stop = true;
              break;
            }
            ptx::tc_fence_after();
            const int sh = 8 * (3 - a);  // 8 (5 - L) in the first pass, 8 (9 - L) in the second
            const uint32_t ta = tmem + lane_off + (uint32_t)(BN * a + EPI_COLS * h);
            // 24 columns as 16 + 8 (h even) or 8 + 16 (h odd), 12 as 8 + 4 or 4 + 8: every load starts on a
            // multiple of its width. Both loads, one wait, and the accumulator is released before any
            // integer work.
            uint32_t v[EPI_COLS];
            if constexpr (EPI_COLS == 24) {
              if ((h & 1) == 0) {
                ptx::tmem_ld_32x32b_x16(ta, v);
                ptx::tmem_ld_32x32b_x8(ta + 16, v + 16);
              } else {
                ptx::tmem_ld_32x32b_x8(ta, v);
                ptx::tmem_ld_32x32b_x16(ta + 8, v + 8);
              }
            } else {
              if ((h & 1) == 0) {
                ptx::tmem_ld_32x32b_x8(ta, v);
                ptx::tmem_ld_32x32b_x4(ta + 8, v + 8);
              } else {
                ptx::tmem_ld_32x32b_x4(ta, v);
                ptx::tmem_ld_32x32b_x8(ta + 4, v + 4);
              }
            }
            ptx::tmem_ld_wait();
            ptx::tc_fence_before();
            __syncwarp();
            if (lane == 0) ptx::mbar_arrive(lempty0 + 8 * a);
            epar ^= 1u << a;
#pragma unroll
            for (int c = 0; c < EPI_COLS; ++c) acc[c] += (long long)__float2int_rn(__uint_as_float(v[c])) << sh;
          }
        }
        if (stop) break;
        if (pass == 0) {
#pragma unroll
          for (int c = 0; c < EPI_COLS; ++c) {
            scr[(size_t)c * (EPI_WARPS * 32)] = acc[c];
            acc[c] = 0;
          }
        }
      }
      if (stop) break;
      const int tile = SPLIT && kpart != 0 ? (kpart - 1) >> 1 : t;  // residual partials are indexed by tile
      long long* scr_lo = scr + (size_t)EPI_COLS * (EPI_WARPS * 32);
      if constexpr (SPLIT) {
        // The second pass's totals join the first's in the scratch, so that nothing of the step loop stays
        // live through the tile end.
#pragma unroll
        for (int c = 0; c < EPI_COLS; ++c) scr_lo[(size_t)c * (EPI_WARPS * 32)] = acc[c];
        if (kpart != 0) {
          // A tile split over K: this warp publishes its half's exact totals. The same warp of the other
          // half covers the same elements; whichever of the two finishes second adds the other's totals to
          // its own (integers, so the sum is exact and independent of the order) and applies the epilogue.
          // Nobody waits: the first to finish just moves on.
          const int half = (kpart - 1) & 1;
          longlong2* pub = reinterpret_cast<longlong2*>(args.split) + ((size_t)tile * 2 + half) * (SPLIT_PER_PART / 2) +
                           (ew * 32 + lane);
          for (int c = 0; c < EPI_COLS; ++c)
            pub[c * (EPI_WARPS * 32)] =
                make_longlong2(scr[(size_t)c * (EPI_WARPS * 32)], scr_lo[(size_t)c * (EPI_WARPS * 32)]);
          __threadfence();
          __syncwarp();
          int last = 0;
          if (lane == 0) {
            int* cnt = args.split_cnt + (size_t)tile * EPI_WARPS + ew;
            last = atomicAdd(cnt, 1) == 1;
            if (last) *cnt = 0;  // ready for the next launch
          }
          if (!__shfl_sync(0xffffffffu, last, 0)) continue;
          __threadfence();
          const longlong2* oth = pub + (half ? -1 : 1) * (ptrdiff_t)(SPLIT_PER_PART / 2);
          for (int c = 0; c < EPI_COLS; ++c) {
            const longlong2 o = __ldcg(oth + c * (EPI_WARPS * 32));
            scr[(size_t)c * (EPI_WARPS * 32)] += o.x;
            scr_lo[(size_t)c * (EPI_WARPS * 32)] += o.y;
          }
        }
      }
      // Tile end: P = 2^(e_i + f_j - 72) (hi 2^32 + lo), then the fused epilogue (FP64 values, FP32 partials).
      const int i = bi * EBM + 32 * q + lane;
      const int ei = i < n ? args.ex[row0 + i] : 0;
      double part = 0.0;  // the tile's share of ||I - P||_F^2, accumulated in FP64
#pragma unroll
      for (int c = 0; c < EPI_COLS; ++c) {
        const int jc = bj * BN + EPI_COLS * h + c;
        const long long hi = scr[(size_t)c * (EPI_WARPS * 32)];
        const long long lo = SPLIT ? scr_lo[(size_t)c * (EPI_WARPS * 32)] : acc[c];
        if (i >= n || jc >= n || (SYM && i > jc)) continue;
        const unsigned long long lw0 = (unsigned long long)hi << 32, lw = lw0 + (unsigned long long)lo;
        const long long H = (hi >> 32) + (lo >> 63) + (lw < lw0 ? 1 : 0);
        const double P = wide_to_double(H, lw, ei + args.ey[row0 + jc] - 72);
        if (e.partial) {
          const double dd = (i == jc ? 1.0 : 0.0) - P;
          part = fma((SYM && i != jc) ? 2.0 * dd : dd, dd, part);
        }
        const int64_t ij = (int64_t)(row0 + i) * args.ld + jc, ji = (int64_t)(row0 + jc) * args.ld + i;
        double w2 = 0.0;
        if (e.out2) {
          w2 = i == jc ? fma(mt.b, P, mt.a) : mt.b * P;
          if (mt.c != 0.0) w2 = fma(mt.c, e.cin[ij], w2);
        }
        const bool direct = SYM || !args.transpose, mirrored = SYM ? (i != jc) : (bool)args.transpose;
        if (direct) {
          if (e.out) e.out[ij] = P;
          if (e.out2) e.out2[ij] = w2;
        }
        if (mirrored) {
          if (e.out) e.out[ji] = P;
          if (e.out2) e.out2[ji] = w2;
        }
      }
      if (e.partial) {
        for (int o = 16; o > 0; o >>= 1) part += __shfl_xor_sync(0xffffffffu, part, o);
        if (lane == 0) e.partial[(int64_t)tile * EPI_WARPS + ew] = part;
      }
    }
  }
  ptx::tc_fence_before();
  __syncthreads();
  ptx::tc_fence_after();
  if (warp == 0) ptx::tmem_dealloc(tmem, 512);
  if (args.tstamp && threadIdx.x == 0) atomicMax(&args.tstamp[1], (unsigned long long)ptx::globaltimer());
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

// The digit planes of an operand ([row][step][plane][16], ldl / 16 steps) as a 3-D FP16 tensor
// (64 halves of one group of 4 planes, group index 2 step + g, row) with byte strides (128, 16 ldl);
// boxes of 64 x 1 x rows with 128-byte swizzling: one step of 4 planes for `rows` rows. Rows >= R read
// as zero.
cudaError_t make_plane_map(CUtensorMap* map, const __half* ptr, int R, int ldl, int rows) {
  auto fn = encode_fn_emu();
  if (!fn) return cudaErrorNotSupported;
  cuuint64_t dims[3] = {64, (cuuint64_t)(ldl / 8), (cuuint64_t)R};
  cuuint64_t strides[2] = {128, (cuuint64_t)ldl * 16};
  cuuint32_t box[3] = {64, 1, (cuuint32_t)rows};
  cuuint32_t estr[3] = {1, 1, 1};
  CUresult r = fn(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT16, 3, const_cast<__half*>(ptr), dims, strides, box, estr,
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

template <int BN>
cudaError_t set_emu_attributes() {
  const int bytes = EmuTile<BN>::SMEM_BYTES;
  for (auto k : {k_gemm_emu<BN, true, false>, k_gemm_emu<BN, false, false>, k_gemm_emu<BN, true, true>,
                 k_gemm_emu<BN, false, true>}) {
    cudaError_t r = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
    if (r != cudaSuccess) return r;
  }
  return cudaSuccess;
}

cudaError_t prepare_emu() {
  static bool attr_set = false;
  if (!attr_set) {
    cudaError_t r = set_emu_attributes<BN_WIDE>();
    if (r == cudaSuccess) r = set_emu_attributes<BN_NARROW>();
    if (r != cudaSuccess) return r;
    attr_set = true;
  }
  if (!encode_fn_emu()) return cudaErrorNotSupported;
  sm_count_emu();
  return cudaSuccess;
}

template <int BN>
cudaError_t launch_emu_bn(const CUtensorMap& mx, const CUtensorMap& my, int grid, Mode mode, const EmuArgs& a,
                          cudaStream_t s) {
  const int bytes = EmuTile<BN>::SMEM_BYTES;
  if (mode == Mode::Sym) {
    if (a.split) k_gemm_emu<BN, true, true><<<grid, THREADS, bytes, s>>>(mx, my, a);
    else k_gemm_emu<BN, true, false><<<grid, THREADS, bytes, s>>>(mx, my, a);
  } else {
    if (a.split) k_gemm_emu<BN, false, true><<<grid, THREADS, bytes, s>>>(mx, my, a);
    else k_gemm_emu<BN, false, false><<<grid, THREADS, bytes, s>>>(mx, my, a);
  }
  return cudaGetLastError();
}

cudaError_t launch_emu(const __half* DX, const __half* DY, int R, int K, int ldl, Mode mode, int bn, EmuArgs& a,
                       cudaStream_t s) {
  if (bn != BN_WIDE && bn != BN_NARROW) return cudaErrorInvalidValue;
  if (a.S < 1 || a.S > SMAX || ldl % 16 != 0 || ldl < K || K < 1 || !a.items || !a.scratch) return cudaErrorInvalidValue;
  if ((reinterpret_cast<uintptr_t>(DX) | reinterpret_cast<uintptr_t>(DY)) & 15) return cudaErrorMisalignedAddress;
  cudaError_t pr_ = prepare_emu();
  if (pr_ != cudaSuccess) return pr_;
  if (a.ntiles == 0 && !a.ntiles_dev) return cudaSuccess;
  CUtensorMap mx, my;
  cudaError_t r = make_plane_map(&mx, DX, R, ldl, EBM);
  if (r != cudaSuccess) return r;
  r = make_plane_map(&my, DY, R, ldl, bn);
  if (r != cudaSuccess) return r;
  const int grid = a.ntiles_dev || a.ntiles >= sm_count_emu() ? sm_count_emu() : a.ntiles;
  return bn == BN_WIDE ? launch_emu_bn<BN_WIDE>(mx, my, grid, mode, a, s)
                       : launch_emu_bn<BN_NARROW>(mx, my, grid, mode, a, s);
}

}  // namespace

void emu_tile_list(int m, int n, Mode mode, std::vector<int4>& out, int bn) {
  const int TM = (n + EBM - 1) / EBM, TN = (n + bn - 1) / bn;
  for (int g = 0; g < TM; g += BAND)
    for (int bj = 0; bj < TN; ++bj)
      for (int bi = g; bi < std::min(g + BAND, TM); ++bi)
        if (mode != Mode::Sym || bn * bj + bn - 1 >= EBM * bi) out.push_back(make_int4(m, bi, bj, 0));
}

// One product of a single matrix: its tiles, each split over K into two halves when that shortens the
// launch. A launch of T tiles on G CTAs lasts ceil(T / G) tile times; split, ceil(2T / G) half-tile times.
// Halves of tile k are items (0, bi, bj, 1 + 2k) and (0, bi, bj, 2 + 2k), next to each other.
int emu_split_slots(int n, Mode mode, int bn, int split) {
  const int T = emu_tile_count(n, mode, bn), G = sm_count_emu(), KS = (n + EBK - 1) / EBK;
  if (KS < 2 || split == 0) return 0;
  if (split > 0) return T;
  return T < 4 * G && (2 * T + G - 1) / G < 2 * ((T + G - 1) / G) ? T : 0;
}

bool emu_split_useful(int n, Mode mode, int bn) {
  return (n + EBK - 1) / EBK >= 2 && emu_tile_count(n, mode, bn) < 4 * sm_count_emu();
}

int4 emu_range_item(int4 item, int j0, int j1) {
  item.w = (j0 << 16) | j1;
  return item;
}

void emu_launch_list(int n, Mode mode, std::vector<int4>& out, int bn, int split) {
  std::vector<int4> tiles;
  emu_tile_list(0, n, mode, tiles, bn);
  if (emu_split_slots(n, mode, bn, split) == 0) {
    out.insert(out.end(), tiles.begin(), tiles.end());
    return;
  }
  for (size_t k = 0; k < tiles.size(); ++k) {
    const int4 t = tiles[k];
    out.push_back(make_int4(t.x, t.y, t.z, 1 + 2 * (int)k));
    out.push_back(make_int4(t.x, t.y, t.z, 2 + 2 * (int)k));
  }
}

// Sized for the wider tile, so that one buffer serves either width.
size_t emu_split_bytes(int slots) {
  return (size_t)slots * 2 * EmuTile<BN_WIDE>::SPLIT_PER_PART * sizeof(long long);
}

size_t emu_split_counters(int slots) { return (size_t)slots * EPI_WARPS; }

int emu_tile_count(int n, Mode mode, int bn) {
  std::vector<int4> v;
  emu_tile_list(0, n, mode, v, bn);
  return (int)v.size();
}

int emu_tiles(int n, Mode mode, int bn) { return emu_tile_count(n, mode, bn) * EPI_WARPS; }

int emu_partials_per_item() { return EPI_WARPS; }

bool emu_tile_width_ok(int bn) { return bn == BN_WIDE || bn == BN_NARROW; }

int emu_max_slices() { return SMAX; }

int emu_ld(int K) { return (K + 15) / 16 * 16; }

cudaError_t slice(const double* X, int n, int ldl, int S, __half* D, int* ex, cudaStream_t s) {
  return slice_rows(X, n, n, n, ldl, S, nullptr, D, ex, s);
}

cudaError_t slice_rows(const double* X, int R, int n, int ldx, int ldl, int S, const int* row_n, __half* D, int* ex,
                       cudaStream_t s) {
  if (S < 1 || S > SMAX || ldl % 16 != 0) return cudaErrorInvalidValue;
  int blocks = R;  // one block per row, up to 16 resident blocks per SM
  if (blocks > sm_count_emu() * 16) blocks = sm_count_emu() * 16;
  if (blocks < 1) return cudaSuccess;
  k_slice<<<blocks, SLICE_THREADS, 0, s>>>(X, R, n, ldx, ldl, S, row_n, D, ex);
  return cudaGetLastError();
}

cudaError_t emu_prepare() { return prepare_emu(); }

size_t emu_scratch_bytes() {
  return (size_t)sm_count_emu() * EmuTile<BN_WIDE>::SCRATCH_PER_CTA * sizeof(long long);  // the wider tile's
}

cudaError_t gemm_emu(const __half* DX, const int* ex, const __half* DY, const int* ey, int n, int ldl, int S, Mode mode,
                     bool transpose, const int4* items, int nitems, const Epilogue& e, long long* scratch,
                     long long* split, int* split_cnt, int* err, cudaStream_t s, int bn) {
  EmuArgs a{};
  a.scratch = scratch;
  a.split = split;
  a.split_cnt = split_cnt;
  a.S = S;
  a.ld = n;
  a.ntiles = nitems;
  a.items = items;
  a.mats = nullptr;
  a.one = EmuMat{n, 0, e.a, e.b, e.c};
  a.transpose = transpose ? 1 : 0;
  a.e = e;
  a.ex = ex;
  a.ey = ey;
  a.err = err;
  return launch_emu(DX, DY, n, n, ldl, mode, bn, a, s);
}

cudaError_t gemm_emu_batched(const __half* DX, const int* ex, const __half* DY, const int* ey, int R, int K, int ldl,
                             int ld, int S, Mode mode, bool transpose, const int4* items, int nitems,
                             const int* nitems_dev, const EmuBatchMat* mats, const Epilogue& e, long long* scratch,
                             int* err, unsigned long long* tstamp, cudaStream_t s, int bn) {
  static_assert(sizeof(EmuBatchMat) == sizeof(EmuMat), "batch matrix record");
  EmuArgs a{};
  a.scratch = scratch;
  a.S = S;
  a.ld = ld;
  a.ntiles = nitems;
  a.ntiles_dev = nitems_dev;
  a.tstamp = tstamp;
  a.items = items;
  a.mats = reinterpret_cast<const EmuMat*>(mats);
  a.transpose = transpose ? 1 : 0;
  a.e = e;
  a.ex = ex;
  a.ey = ey;
  a.err = err;
  return launch_emu(DX, DY, R, K, ldl, mode, bn, a, s);
}

}  // namespace pr
