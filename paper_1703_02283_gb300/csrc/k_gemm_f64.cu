// Native FP64 matrix products for the iteration of Eq. 1 (the plain FP64 path).
//
// P = X Y for n x n row-major X, Y, computed on the FP64 tensor instructions (mma.sync m8n8k4 f64,
// DMMA). A 64 x 64 output tile per 128-thread block, each warp a 32 x 32 sub-tile of 4 x 4 DMMA
// fragments, K staged through shared memory 16 at a time with register prefetch of the next slice.
// FP64 issue rate, not memory, bounds this kernel on GB300, so the tile is sized for occupancy.
//
// Symmetric mode computes only the upper-triangle tiles (bi <= bj) and stores each element at (i, j)
// and (j, i): products of commuting symmetric matrices (every pair of iterates, Sec. 2) are symmetric,
// so this halves the work. In a diagonal tile only elements with i <= j are kept, so the stored matrix
// is exactly symmetric. The fused epilogue (see pr::Epilogue) forms the next operand and the per-tile
// residual partial sums in the same pass.
#include "pr_internal.h"

namespace pr {
namespace {

constexpr int BM = 64, BN = 64, BK = 16, kThreads = 128;

__device__ __forceinline__ void dmma(double& d0, double& d1, double a, double b) {
  asm volatile("mma.sync.aligned.m8n8k4.row.col.f64.f64.f64.f64 {%0,%1}, {%2}, {%3}, {%0,%1};\n"
               : "+d"(d0), "+d"(d1)
               : "d"(a), "d"(b));
}

// Row-major upper-triangle enumeration of a T x T tile grid: t -> (bi, bj), bi <= bj.
__device__ __forceinline__ void tri_index(int t, int T, int& bi, int& bj) {
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
__global__ void __launch_bounds__(kThreads) k_gemm_f64(const double* __restrict__ X, const double* __restrict__ Y, int n,
                                                       int T, Epilogue e) {
  __shared__ double As[2][BK][BM + 2];  // As[k][m]
  __shared__ double Bs[2][BK][BN + 2];  // Bs[k][n]
  __shared__ double red[kThreads / 32];

  int bi, bj, tile_id;
  if (SYM) {
    tile_id = blockIdx.x;
    tri_index(tile_id, T, bi, bj);
  } else {
    bi = blockIdx.y;
    bj = blockIdx.x;
    tile_id = blockIdx.y * gridDim.x + blockIdx.x;
  }
  const int i0 = bi * BM, j0 = bj * BN;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int g = lane >> 2, t4 = lane & 3;
  const int wm = warp >> 1, wn = warp & 1;

  double acc[4][4][2];
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int b = 0; b < 4; ++b) acc[a][b][0] = acc[a][b][1] = 0.0;

  double ra[8], rb[8];
  auto load = [&](int k0) {
#pragma unroll
    for (int q = 0; q < 8; ++q) {
      const int ea = tid + kThreads * q;  // A tile: 64 rows x 16 k, k fastest
      const int r = ea >> 4, k = ea & 15;
      const int gi = i0 + r, gk = k0 + k;
      ra[q] = (gi < n && gk < n) ? X[(int64_t)gi * n + gk] : 0.0;
      const int kr = ea >> 6, c = ea & 63;  // B tile: 16 k x 64 cols, cols fastest
      const int gkk = k0 + kr, gj = j0 + c;
      rb[q] = (gkk < n && gj < n) ? Y[(int64_t)gkk * n + gj] : 0.0;
    }
  };
  auto store = [&](int buf) {
#pragma unroll
    for (int q = 0; q < 8; ++q) {
      const int ea = tid + kThreads * q;
      As[buf][ea & 15][ea >> 4] = ra[q];
      Bs[buf][ea >> 6][ea & 63] = rb[q];
    }
  };

  const int KT = (n + BK - 1) / BK;
  load(0);
  store(0);
  __syncthreads();
  for (int kt = 0; kt < KT; ++kt) {
    const int cur = kt & 1;
    if (kt + 1 < KT) load((kt + 1) * BK);
#pragma unroll
    for (int kk = 0; kk < BK; kk += 4) {
      double fa[4], fb[4];
#pragma unroll
      for (int mi = 0; mi < 4; ++mi) fa[mi] = As[cur][kk + t4][wm * 32 + mi * 8 + g];
#pragma unroll
      for (int ni = 0; ni < 4; ++ni) fb[ni] = Bs[cur][kk + t4][wn * 32 + ni * 8 + g];
#pragma unroll
      for (int mi = 0; mi < 4; ++mi)
#pragma unroll
        for (int ni = 0; ni < 4; ++ni) dmma(acc[mi][ni][0], acc[mi][ni][1], fa[mi], fb[ni]);
    }
    if (kt + 1 < KT) store(cur ^ 1);
    __syncthreads();
  }

  // Epilogue. Fragment element (g, 2 t4 + r) of DMMA tile (mi, ni).
  double part = 0.0;
#pragma unroll
  for (int mi = 0; mi < 4; ++mi)
#pragma unroll
    for (int ni = 0; ni < 4; ++ni)
#pragma unroll
      for (int r = 0; r < 2; ++r) {
        const int i = i0 + wm * 32 + mi * 8 + g;
        const int j = j0 + wn * 32 + ni * 8 + 2 * t4 + r;
        if (i >= n || j >= n) continue;
        if (SYM && i > j) continue;  // the diagonal tile keeps its upper triangle only
        const double P = acc[mi][ni][r];
        const int64_t ij = (int64_t)i * n + j, ji = (int64_t)j * n + i;
        const bool mirror = SYM && i != j;
        if (e.out) {
          e.out[ij] = P;
          if (mirror) e.out[ji] = P;
          if (e.out_lp) {
            const __nv_bfloat16 v = bf16_rne(P);
            e.out_lp[ij] = v;
            if (mirror) e.out_lp[ji] = v;
          }
        }
        if (e.out2) {
          double v = e.b * P;
          if (i == j) v += e.a;
          if (e.c != 0.0) v += e.c * e.cin[ij];
          e.out2[ij] = v;
          if (mirror) e.out2[ji] = v;
          if (e.out2_lp) {
            const __nv_bfloat16 w = bf16_rne(v);
            e.out2_lp[ij] = w;
            if (mirror) e.out2_lp[ji] = w;
          }
        }
        if (e.partial) {
          const double d = (i == j ? 1.0 : 0.0) - P;
          part += (mirror ? 2.0 : 1.0) * d * d;
        }
      }
  if (e.partial) {
    for (int o = 16; o > 0; o >>= 1) part += __shfl_xor_sync(0xffffffffu, part, o);
    if (lane == 0) red[warp] = part;
    __syncthreads();
    if (tid == 0) e.partial[tile_id] = ((red[0] + red[1]) + red[2]) + red[3];
  }
}

}  // namespace

int gemm_f64_tiles(int n, Mode mode) {
  const int T = (n + BM - 1) / BM;
  return mode == Mode::Sym ? T * (T + 1) / 2 : T * T;
}

cudaError_t gemm_f64(const double* X, const double* Y, int n, Mode mode, const Epilogue& e, cudaStream_t s) {
  const int T = (n + BM - 1) / BM;
  if (mode == Mode::Sym) {
    k_gemm_f64<true><<<T * (T + 1) / 2, kThreads, 0, s>>>(X, Y, n, T, e);
  } else {
    k_gemm_f64<false><<<dim3(T, T), kThreads, 0, s>>>(X, Y, n, T, e);
  }
  return cudaGetLastError();
}

}  // namespace pr
