// Device-side control of batched solves. The solve loop of a batch is one CUDA graph (a device-side while
// loop); every decision the host used to take between launches is taken here, on the GPU:
//  * k_batch_stage: the work list of one product stage, from the states of the matrices (which are still
//    iterating, their form and root), their per-matrix epilogue records and residual partial ranges;
//  * k_batch_residuals: each member's residual ||I - P||_F from its partials (the fixed-order sum of the
//    single-matrix path), appended to its history;
//  * k_batch_decide: the stop rule of every iterating matrix (the rule of pr_iterate); a matrix that stops
//    has its iterate copied to the results and its rows dropped from the digit slicing;
//  * k_batch_advance: one more update counted per iterating matrix, and the loop condition;
//  * k_batch_verify_rows: after the loop, the coupled-form matrices whose true residual ||I - X^p A||_F the
//    verification stages evaluate (their partials go to a per-matrix true residual, not the history);
//  * timing: each product launch folds its first start and last end time into a slot (%globaltimer); the
//    next list build for the same slot, or k_batch_harvest, adds that span to the tally.
#include "pr_internal.h"

#include <climits>

namespace pr {
namespace {

constexpr int kCtlThreads = 1024;  // one block builds a stage's list

// A matrix stopped on tol, stagnation or max_iter (not diverged) whose true residual the verification
// after the solve loop evaluates: the coupled form tests ||I - M||_F, which rounding can separate from it.
__device__ __forceinline__ bool to_verify(const BatchCtl& c, int m) {
  const int s = c.status[m];
  return !c.active[m] && c.form[m] == PR_FORM_COUPLED && (s == PR_OK || s == PR_ESTAGNATED || s == PR_EMAXITER);
}

__device__ __forceinline__ bool stage_member(const BatchCtl& c, const BatchStage& st, int m) {
  if (st.verify) {
    if (!to_verify(c, m)) return false;
  } else if (!c.active[m] || c.form[m] != st.form) {
    return false;
  }
  const int p = c.p[m];
  if (st.pcmp == 1 && p != st.pj) return false;
  if (st.pcmp == 2 && p <= st.pj) return false;
  if (st.verify) return true;
  if (st.fresh_only && c.hlen[m] != 0) return false;
  if (st.pskip != 0 && p == st.pskip) return false;
  return true;
}

// Adds the span recorded in timing slot k (if its launch had work) to the tally and re-arms the slot.
__device__ void harvest_slot(const BatchCtl& c, int k) {
  unsigned long long* t = c.tstamp + 2 * k;
  if (t[0] != ULLONG_MAX && t[1] > t[0]) {
    c.tally[0] += (double)(t[1] - t[0]);
    c.tally[1] += c.flops_pending[k];
    c.tally[2] += 1.0;
  }
  t[0] = ULLONG_MAX;
  t[1] = 0ull;
  c.flops_pending[k] = 0.0;
}

__global__ void __launch_bounds__(kCtlThreads) k_batch_stage(BatchCtl c, BatchStage st) {
  __shared__ int warp_sum[32];
  __shared__ double warp_flops[32];
  __shared__ int carry;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (threadIdx.x == 0) {
    harvest_slot(c, st.slot);
    carry = 0;
  }
  __syncthreads();
  const int* cnt = st.full ? c.cnt_full : c.cnt_sym;
  double flops = 0.0;
  int members = 0;
  // Offsets of the members' items, in the order of c.order (exclusive scan over the member counts).
  for (int base = 0; base < c.count; base += kCtlThreads) {
    const int i = base + threadIdx.x;
    int m = -1, k = 0;
    if (i < c.count) {
      m = c.order[i];
      if (stage_member(c, st, m)) {
        k = cnt[m];
        const double nm = c.n[m];
        flops += st.full ? 2.0 * nm * nm * nm : nm * nm * (nm + 1.0);
        members += 1;
      }
    }
    int v = k;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int y = __shfl_up_sync(0xffffffffu, v, o);
      if (lane >= o) v += y;
    }
    if (lane == 31) warp_sum[warp] = v;
    __syncthreads();
    if (warp == 0) {
      int w = warp_sum[lane];
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(0xffffffffu, w, o);
        if (lane >= o) w += y;
      }
      warp_sum[lane] = w;
    }
    __syncthreads();
    if (m >= 0) {
      const int first = carry + (warp ? warp_sum[warp - 1] : 0) + v - k;
      c.ofs[m] = k ? first : -1;
      c.member[m] = k ? 1 : 0;
      c.seg_b[m] = k ? first * c.per : 0;
      c.seg_e[m] = k ? (first + k) * c.per : 0;
      if (k) c.mats[m] = EmuBatchMat{c.n[m], c.row0[m], st.a, st.b, st.c};
    }
    __syncthreads();
    if (threadIdx.x == 0) carry += warp_sum[31];
    __syncthreads();
  }
  // Copy every member's items (one warp per matrix).
  const int4* src = st.full ? c.items_full : c.items_sym;
  const int* off = st.full ? c.off_full : c.off_sym;
  for (int i = warp; i < c.count; i += kCtlThreads / 32) {
    const int m = c.order[i];
    const int first = c.ofs[m];
    if (first < 0) continue;
    const int k = cnt[m];
    for (int j = lane; j < k; j += 32) c.items[first + j] = src[off[m] + j];
  }
  // Flops and member count of the stage.
  for (int o = 16; o > 0; o >>= 1) {
    flops += __shfl_down_sync(0xffffffffu, flops, o);
    members += __shfl_down_sync(0xffffffffu, members, o);
  }
  __syncthreads();
  if (lane == 0) {
    warp_flops[warp] = flops;
    warp_sum[warp] = members;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double f = 0.0;
    int mm = 0;
    for (int w = 0; w < kCtlThreads / 32; ++w) {
      f += warp_flops[w];
      mm += warp_sum[w];
    }
    *c.nitems = carry;
    c.flops_pending[st.slot] = f;
    if (carry > 0) {
      c.tally[3] += 1.0;
      c.tally[4] += (double)mm;
      c.tally[5] += f;
    }
  }
}

__global__ void k_batch_residuals(BatchCtl c, const double* __restrict__ partial, int to_true) {
  __shared__ double sh[kReduceThreads];
  const int m = blockIdx.x;
  if (!c.member[m]) return;  // uniform over the block
  const double r = block_sum_sqrt(partial + c.seg_b[m], c.seg_e[m] - c.seg_b[m], sh);
  if (threadIdx.x == 0 && to_true) {
    c.truer[m] = r;
  } else if (threadIdx.x == 0) {
    const int len = c.hlen[m];
    if (len < c.hcap) {
      c.hist[(size_t)m * c.hcap + len] = r;
      c.hlen[m] = len + 1;
    }
  }
}

__global__ void k_batch_decide(BatchCtl c, const double* __restrict__ X, pr_options o) {
  __shared__ int stop;
  const int m = blockIdx.x;
  if (threadIdx.x == 0) {
    int s = -1;
    if (c.active[m]) {
      const int len = c.hlen[m];
      const double* h = c.hist + (size_t)m * c.hcap;
      if (len >= 1) s = stop_rule_last(h[len - 1], len >= 2, len >= 2 ? h[len - 2] : 0.0, false, c.params[0], o);
      if (s < 0 && c.iters[m] >= o.max_iter) s = PR_EMAXITER;
    }
    stop = s;
  }
  __syncthreads();
  if (stop < 0) return;
  const int n = c.n[m], r0 = c.row0[m];
  const size_t base = (size_t)r0 * c.ld, total = (size_t)n * c.ld;
  for (size_t e = threadIdx.x; e < total; e += blockDim.x) c.result[base + e] = X[base + e];
  for (int r = threadIdx.x; r < n; r += blockDim.x) {
    c.row_n[r0 + r] = -1;
    if (c.row_n2) c.row_n2[r0 + r] = -1;
  }
  if (threadIdx.x == 0) {
    c.status[m] = stop;
    c.active[m] = 0;
  }
}

__global__ void __launch_bounds__(kCtlThreads) k_batch_advance(BatchCtl c, cudaGraphConditionalHandle h, int set_cond,
                                                               int limit) {
  __shared__ int warp_sum[32];
  int live = 0;
  for (int m = threadIdx.x; m < c.count; m += kCtlThreads)
    if (c.active[m]) {
      c.iters[m] += 1;
      live += 1;
    }
  for (int o = 16; o > 0; o >>= 1) live += __shfl_down_sync(0xffffffffu, live, o);
  if ((threadIdx.x & 31) == 0) warp_sum[threadIdx.x >> 5] = live;
  __syncthreads();
  if (threadIdx.x == 0 && set_cond) {
    int total = 0;
    for (int w = 0; w < kCtlThreads / 32; ++w) total += warp_sum[w];
    const int loops = *c.loops + 1;
    *c.loops = loops;
    cudaGraphSetConditional(h, (total > 0 && *c.err == 0 && loops < limit) ? 1u : 0u);
  }
}

// Block (m, g): warps take the rows r = 8 g + w, 8 g + w + 8 G, ... of matrix m (G row groups), lanes the
// columns.
constexpr int kLincombGroups = 16;

__global__ void __launch_bounds__(256) k_batch_lincomb(BatchCtl c, int pj, const double* x, const double* y,
                                                       double a, double b, double* out) {
  const int m = blockIdx.x;
  if (!c.active[m] || c.p[m] != pj) return;  // uniform over the block
  const int n = c.n[m], lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const size_t base = (size_t)c.row0[m] * c.ld;
  for (int r = 8 * blockIdx.y + w; r < n; r += 8 * kLincombGroups)
    for (int k = lane; k < n; k += 32) {
      const size_t e = base + (size_t)r * c.ld + k;
      out[e] = fma(a, x[e], b * y[e]);
    }
}

// Block m: the rows of matrix m get its order if it is verified, else -1; its true residual is reset.
__global__ void k_batch_verify_rows(BatchCtl c) {
  const int m = blockIdx.x;
  const int v = to_verify(c, m) ? c.n[m] : -1, r0 = c.row0[m];
  for (int r = threadIdx.x; r < c.n[m]; r += blockDim.x) c.row_v[r0 + r] = v;
  if (threadIdx.x == 0) c.truer[m] = -1.0;
}

__global__ void k_batch_harvest(BatchCtl c, int nslots) {
  if (threadIdx.x == 0)
    for (int k = 0; k < nslots; ++k) harvest_slot(c, k);
}

}  // namespace

cudaError_t batch_stage_list(const BatchCtl& c, const BatchStage& st, cudaStream_t s) {
  k_batch_stage<<<1, kCtlThreads, 0, s>>>(c, st);
  return cudaGetLastError();
}

cudaError_t batch_residuals(const BatchCtl& c, const double* partial, int to_true, cudaStream_t s) {
  k_batch_residuals<<<c.count, kReduceThreads, 0, s>>>(c, partial, to_true);
  return cudaGetLastError();
}

cudaError_t batch_verify_rows(const BatchCtl& c, cudaStream_t s) {
  k_batch_verify_rows<<<c.count, 256, 0, s>>>(c);
  return cudaGetLastError();
}

cudaError_t batch_decide(const BatchCtl& c, const double* X, const pr_options& o, cudaStream_t s) {
  k_batch_decide<<<c.count, 256, 0, s>>>(c, X, o);
  return cudaGetLastError();
}

cudaError_t batch_advance(const BatchCtl& c, cudaGraphConditionalHandle h, int set_cond, int limit, cudaStream_t s) {
  k_batch_advance<<<1, kCtlThreads, 0, s>>>(c, h, set_cond, limit);
  return cudaGetLastError();
}

cudaError_t batch_lincomb(const BatchCtl& c, int pj, const double* x, const double* y, double a, double b,
                          double* out, cudaStream_t s) {
  k_batch_lincomb<<<dim3(c.count, kLincombGroups), 256, 0, s>>>(c, pj, x, y, a, b, out);
  return cudaGetLastError();
}

cudaError_t batch_harvest(const BatchCtl& c, int nslots, cudaStream_t s) {
  k_batch_harvest<<<1, 32, 0, s>>>(c, nslots);
  return cudaGetLastError();
}

}  // namespace pr
