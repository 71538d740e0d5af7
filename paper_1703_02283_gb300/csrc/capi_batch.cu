// Batched solves: many independent problems A_i^{-1/p_i} (SPD matrices of uneven orders and roots) iterated
// together. Every matrix product stage of an iteration is one launch of the digit-slice tensor-core kernel
// over the 128 x 128 tiles of all matrices taking part in that stage; the matrices are packed row-wise
// in shared device buffers with one leading dimension, so one TMA descriptor serves the whole batch.
//
// Per matrix the iteration, the forms (Newton-Schulz for p = 1, coupled for p >= 2, as in capi.cu), the
// initial guess of Eq. 3 and the stop rule are those of the single-matrix path. A matrix whose stop rule
// fires is copied to the result buffer and leaves the work lists.
#include "pr_internal.h"

#include <math.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <string>
#include <utility>
#include <vector>

using pr::EmuBatchMat;
using pr::Epilogue;
using pr::Mode;

namespace {
thread_local std::string g_batch_error;

struct Buf {  // a packed FP64 buffer and its digit planes
  double* f = nullptr;
  __half* sl = nullptr;
  int* ex = nullptr;
  bool sl_valid = false;
};
}  // namespace

struct pr_batch_s {
  int count = 0;
  int S = 8;
  int R = 0;   // packed rows (sum of the orders)
  int K = 0;   // largest order
  int ld = 0;  // leading dimension of the packed buffers (K rounded up to 8)
  cudaStream_t stream = nullptr;
  int device = 0;
  pr_options opt{};
  std::vector<int> n, p, row0, form;
  std::vector<int> order;  // matrices by decreasing order (load balance of the work lists)
  Buf A, X, Xn, M, Mn, N, Nn, T0, T1;
  double* result = nullptr;  // packed results
  int* row_n = nullptr;      // order of the matrix owning each packed row
  double* partial = nullptr;
  int partial_cap = 0;
  int4* items = nullptr;
  int items_cap = 0;
  std::vector<int4> items_host;
  EmuBatchMat* mats = nullptr;
  int* seg = nullptr;  // segment begin[count], end[count]
  double* res = nullptr;
  double* hres = nullptr;  // pinned
  int* err = nullptr;
  long long* scratch = nullptr;  // PR_EMU64 first-pass totals
  // per matrix
  std::vector<std::vector<double>> hist;
  std::vector<int> active, status, iterations;
  int64_t launches = 0;
  pr_batch_stats_t st{};
  bool timing = false;
  // Pinned staging of the per-stage work lists, a ring of slots: a slot is rewritten only after the copy
  // that read it has completed (its event), so stages need no stream synchronisation.
  static constexpr int kSlots = 4;
  int4* h_items[kSlots] = {};
  EmuBatchMat* h_mats[kSlots] = {};
  cudaEvent_t slot_ev[kSlots] = {};
  bool slot_used[kSlots] = {};
  int slot = 0;
  // Event pairs around product launches, read at the next synchronisation.
  std::vector<std::pair<cudaEvent_t, cudaEvent_t>> ev_pool;
  std::vector<double> ev_flops;
  size_t ev_pending = 0;
  std::string errmsg;
};

namespace {

pr_status bfail(pr_batch b, pr_status code, const std::string& msg) {
  if (b) b->errmsg = msg;
  else g_batch_error = msg;
  pr::set_handleless_error(msg.c_str());
  return code;
}

#define PB_CK(b, call)                                                                                   \
  do {                                                                                                   \
    cudaError_t _e = (call);                                                                             \
    if (_e != cudaSuccess)                                                                               \
      return bfail((b), _e == cudaErrorMemoryAllocation ? PR_ENOMEM : PR_ECUDA,                          \
                   std::string(#call) + ": " + cudaGetErrorName(_e) + " (" + cudaGetErrorString(_e) + ")"); \
  } while (0)

// Adds the times of the product launches bracketed since the last call (the stream has been synchronised).
pr_status harvest_timing(pr_batch b) {
  for (size_t k = 0; k < b->ev_pending; ++k) {
    float ms = 0.f;
    PB_CK(b, cudaEventElapsedTime(&ms, b->ev_pool[k].first, b->ev_pool[k].second));
    b->st.stages_timed += 1;
    b->st.stage_ms += ms;
    b->st.stage_flops_timed += b->ev_flops[k];
  }
  b->ev_pending = 0;
  return PR_OK;
}

pr_status ensure_slices(pr_batch b, Buf& x) {
  if (x.sl_valid) return PR_OK;
  PB_CK(b, pr::slice_rows(x.f, b->R, b->K, b->ld, pr::emu_ld(b->K), b->S, b->row_n, x.sl, x.ex, b->stream));
  b->launches += 1;
  x.sl_valid = true;
  return PR_OK;
}

// One stage: P = X Y for every matrix in `who` (indices), with per-matrix epilogue coefficients `coef`
// (a, b, c). Writes out / out2 (packed), residual partials (if `partial_base` >= 0) and returns, through
// seg_begin / seg_end (host), the partial range of each matrix.
struct StageOut {
  Buf* out = nullptr;
  Buf* out2 = nullptr;
  const double* cin = nullptr;
  bool partial = false;
  bool transpose = false;
};

pr_status stage(pr_batch b, Buf& Xb, Buf& Yb, Mode mode, const std::vector<int>& who,
                const std::vector<double3>& coef, const StageOut& so, std::vector<int>* seg_begin,
                std::vector<int>* seg_end) {
  if (who.empty()) return PR_OK;
  pr_status s = ensure_slices(b, Xb);
  if (s == PR_OK) s = ensure_slices(b, Yb);
  if (s != PR_OK) return s;
  std::vector<int> sorted = who;
  std::sort(sorted.begin(), sorted.end(), [&](int x, int y) { return b->n[x] > b->n[y]; });
  // The host staging slot: wait until the copy that last read it has completed.
  const int sl = b->slot;
  b->slot = (b->slot + 1) % pr_batch_s::kSlots;
  if (b->slot_used[sl]) PB_CK(b, cudaEventSynchronize(b->slot_ev[sl]));
  EmuBatchMat* mats = b->h_mats[sl];
  for (int m = 0; m < b->count; ++m) mats[m] = EmuBatchMat{b->n[m], b->row0[m], 0.0, 0.0, 0.0};
  const int per = pr::emu_partials_per_item();
  for (size_t w = 0; w < who.size(); ++w) mats[who[w]] = EmuBatchMat{b->n[who[w]], b->row0[who[w]], coef[w].x, coef[w].y,
                                                                    coef[w].z};
  std::vector<int4>& items = b->items_host;
  items.clear();
  for (int m : sorted) {
    if (seg_begin) (*seg_begin)[m] = (int)items.size() * per;
    pr::emu_tile_list(m, b->n[m], mode, items);
    if (seg_end) (*seg_end)[m] = (int)items.size() * per;
  }
  if ((int)items.size() > b->items_cap) return bfail(b, PR_ECUDA, "pr_batch: work list larger than allocated");
  std::copy(items.begin(), items.end(), b->h_items[sl]);
  PB_CK(b, cudaMemcpyAsync(b->items, b->h_items[sl], items.size() * sizeof(int4), cudaMemcpyHostToDevice, b->stream));
  PB_CK(b, cudaMemcpyAsync(b->mats, mats, (size_t)b->count * sizeof(EmuBatchMat), cudaMemcpyHostToDevice, b->stream));
  PB_CK(b, cudaEventRecord(b->slot_ev[sl], b->stream));
  b->slot_used[sl] = true;
  double flops = 0.0;
  for (int m : who) {
    const double nm = b->n[m];
    flops += mode == Mode::Sym ? nm * nm * (nm + 1.0) : 2.0 * nm * nm * nm;
  }
  Epilogue e;
  if (so.out) e.out = so.out->f;
  if (so.out2) e.out2 = so.out2->f;
  e.cin = so.cin;
  e.partial = so.partial ? b->partial : nullptr;
  if (b->timing) {
    if (b->ev_pending == b->ev_pool.size()) {
      cudaEvent_t e0, e1;
      PB_CK(b, cudaEventCreate(&e0));
      PB_CK(b, cudaEventCreate(&e1));
      b->ev_pool.emplace_back(e0, e1);
      b->ev_flops.push_back(0.0);
    }
    PB_CK(b, cudaEventRecord(b->ev_pool[b->ev_pending].first, b->stream));
  }
  PB_CK(b, pr::gemm_emu_batched(Xb.sl, Xb.ex, Yb.sl, Yb.ex, b->R, b->K, pr::emu_ld(b->K), b->ld, b->S, mode, so.transpose,
                                b->items, (int)items.size(), b->mats, e, b->scratch, b->err, b->stream));
  if (b->timing) {
    PB_CK(b, cudaEventRecord(b->ev_pool[b->ev_pending].second, b->stream));
    b->ev_flops[b->ev_pending] = flops;
    b->ev_pending += 1;
  }
  b->launches += 1;
  b->st.stages += 1;
  b->st.products += (int64_t)who.size();
  b->st.product_flops += flops;
  if (so.out) so.out->sl_valid = false;
  if (so.out2) so.out2->sl_valid = false;
  return PR_OK;
}

// Residuals of the matrices in `who` from the partial ranges of the last stage; appended to histories.
pr_status read_residuals(pr_batch b, const std::vector<int>& who, const std::vector<int>& sb,
                         const std::vector<int>& se) {
  if (who.empty()) return PR_OK;
  std::vector<int> seg(2 * who.size());
  for (size_t w = 0; w < who.size(); ++w) {
    seg[w] = sb[who[w]];
    seg[who.size() + w] = se[who[w]];
  }
  PB_CK(b, cudaMemcpyAsync(b->seg, seg.data(), seg.size() * sizeof(int), cudaMemcpyHostToDevice, b->stream));
  PB_CK(b, pr::segmented_reduce_sqrt(b->partial, b->seg, b->seg + who.size(), (int)who.size(), b->res, b->stream));
  b->launches += 1;
  PB_CK(b, cudaMemcpyAsync(b->hres, b->res, who.size() * sizeof(double), cudaMemcpyDeviceToHost, b->stream));
  int word = 0;
  PB_CK(b, cudaMemcpyAsync(&word, b->err, sizeof(int), cudaMemcpyDeviceToHost, b->stream));
  PB_CK(b, cudaStreamSynchronize(b->stream));
  if (word != 0) {
    cudaMemsetAsync(b->err, 0, sizeof(int), b->stream);
    return bfail(b, PR_ETIMEOUT, "pr_batch: a bounded device wait expired");
  }
  pr_status hs = harvest_timing(b);
  if (hs != PR_OK) return hs;
  for (size_t w = 0; w < who.size(); ++w) b->hist[who[w]].push_back(b->hres[w]);
  return PR_OK;
}

// Coupled chain for the matrices in `who`: Y_1 = F src0, Y_j = F Y_{j-1}, the p-th product written as
// (out, out2 = ((p+1) I - out)/p) with residual partials; intermediate products go to T0 / T1.
pr_status chain(pr_batch b, Buf& F, Buf& src0, Buf& outM, Buf& outN, const std::vector<int>& who,
                std::vector<int>& sb, std::vector<int>& se) {
  int pmax = 0;
  for (int m : who) pmax = std::max(pmax, b->p[m]);
  for (int j = 1; j <= pmax; ++j) {
    Buf& src = j == 1 ? src0 : ((j - 1) & 1 ? b->T0 : b->T1);
    std::vector<int> fin, mid;
    std::vector<double3> cf, cm;
    for (int m : who) {
      if (b->p[m] == j) {
        fin.push_back(m);
        cf.push_back(make_double3((double)(j + 1) / j, -1.0 / j, 0.0));
      } else if (b->p[m] > j) {
        mid.push_back(m);
        cm.push_back(make_double3(0.0, 0.0, 0.0));
      }
    }
    StageOut om;
    om.out = (j & 1) ? &b->T0 : &b->T1;
    pr_status s = stage(b, F, src, Mode::Sym, mid, cm, om, nullptr, nullptr);
    if (s != PR_OK) return s;
    StageOut of;
    of.out = &outM;
    of.out2 = &outN;
    of.partial = true;
    s = stage(b, F, src, Mode::Sym, fin, cf, of, &sb, &se);
    if (s != PR_OK) return s;
    s = read_residuals(b, fin, sb, se);
    if (s != PR_OK) return s;
  }
  return PR_OK;
}

}  // namespace

extern "C" {

pr_status pr_batch_destroy(pr_batch b) {
  if (!b) return PR_OK;
  cudaSetDevice(b->device);
  if (b->stream) cudaStreamSynchronize(b->stream);
  for (Buf* x : {&b->A, &b->X, &b->Xn, &b->M, &b->Mn, &b->N, &b->Nn, &b->T0, &b->T1}) {
    if (x->f) cudaFree(x->f);
    if (x->sl) cudaFree(x->sl);
    if (x->ex) cudaFree(x->ex);
  }
  for (void* q : {(void*)b->result, (void*)b->row_n, (void*)b->partial, (void*)b->items, (void*)b->mats, (void*)b->seg,
                  (void*)b->res, (void*)b->err, (void*)b->scratch})
    if (q) cudaFree(q);
  if (b->hres) cudaFreeHost(b->hres);
  for (int k = 0; k < pr_batch_s::kSlots; ++k) {
    if (b->h_items[k]) cudaFreeHost(b->h_items[k]);
    if (b->h_mats[k]) cudaFreeHost(b->h_mats[k]);
    if (b->slot_ev[k]) cudaEventDestroy(b->slot_ev[k]);
  }
  for (auto& pr_ : b->ev_pool) {
    cudaEventDestroy(pr_.first);
    cudaEventDestroy(pr_.second);
  }
  delete b;
  return PR_OK;
}

pr_status pr_batch_init(pr_batch* out, int count, const int64_t* n, const int* p, const double* const* A,
                        const pr_options* opt, void* stream) {
  if (!out) return bfail(nullptr, PR_EINVAL, "pr_batch_init: b is NULL");
  *out = nullptr;
  if (count < 1 || !n || !p || !A) return bfail(nullptr, PR_EINVAL, "pr_batch_init: empty batch or NULL array");
  pr_options o;
  if (opt) o = *opt;
  else pr_default_options(&o);
  if (o.form != PR_FORM_AUTO) return bfail(nullptr, PR_EINVAL, "pr_batch_init: batches run the automatic forms");
  if (o.c0 != PR_C0_EQ3 && o.c0 != PR_C0_SCALED_I) return bfail(nullptr, PR_EINVAL, "pr_batch_init: unknown c0");
  if (o.emu_slices < 0 || o.emu_slices > pr::emu_max_slices() || o.max_iter < 0)
    return bfail(nullptr, PR_EINVAL, "pr_batch_init: bad option value");
  int64_t R = 0, K = 0;
  for (int m = 0; m < count; ++m) {
    if (n[m] < 1 || n[m] > 16384) return bfail(nullptr, PR_EINVAL, "pr_batch_init: orders must be in [1, 16384]");
    if (p[m] < 1 || p[m] > 64) return bfail(nullptr, PR_EINVAL, "pr_batch_init: roots must be in [1, 64]");
    if (!A[m]) return bfail(nullptr, PR_EINVAL, "pr_batch_init: NULL matrix");
    R += n[m];
    K = std::max(K, n[m]);
  }
  if (R > (int64_t)1 << 26) return bfail(nullptr, PR_EINVAL, "pr_batch_init: batch too large");
  pr_batch b = new pr_batch_s();
  b->count = count;
  b->opt = o;
  b->S = o.emu_slices > 0 ? o.emu_slices : pr::emu_max_slices();
  b->R = (int)R;
  b->K = (int)K;
  b->ld = (int)((K + 7) / 8 * 8);
  b->stream = (cudaStream_t)stream;
  cudaGetDevice(&b->device);
  b->n.resize(count);
  b->p.resize(count);
  b->row0.resize(count);
  b->form.resize(count);
  b->hist.resize(count);
  b->active.assign(count, 1);
  b->status.assign(count, -1);
  b->iterations.assign(count, 0);
  int row = 0;
  for (int m = 0; m < count; ++m) {
    b->n[m] = (int)n[m];
    b->p[m] = p[m];
    b->row0[m] = row;
    b->form[m] = p[m] == 1 ? PR_FORM_NS : PR_FORM_COUPLED;
    row += (int)n[m];
  }
  auto bail = [&](pr_status code) {
    g_batch_error = b->errmsg;
    pr_batch_destroy(b);
    return code;
  };
#define PB_INIT_CK(call)                                                                             \
  do {                                                                                               \
    cudaError_t _e = (call);                                                                         \
    if (_e != cudaSuccess) {                                                                         \
      bfail(b, PR_ECUDA, std::string(#call) + ": " + cudaGetErrorName(_e));                          \
      return bail(_e == cudaErrorMemoryAllocation ? PR_ENOMEM : PR_ECUDA);                          \
    }                                                                                                \
  } while (0)
  const size_t fbytes = (size_t)b->R * b->ld * sizeof(double);
  const size_t sbytes = (size_t)8 * b->R * pr::emu_ld(b->K) * sizeof(__half);
  for (Buf* x : {&b->A, &b->X, &b->Xn, &b->M, &b->Mn, &b->N, &b->Nn, &b->T0, &b->T1}) {
    PB_INIT_CK(cudaMalloc((void**)&x->f, fbytes));
    PB_INIT_CK(cudaMemsetAsync(x->f, 0, fbytes, b->stream));
    PB_INIT_CK(cudaMalloc((void**)&x->sl, sbytes));
    PB_INIT_CK(cudaMalloc((void**)&x->ex, (size_t)b->R * sizeof(int)));
  }
  PB_INIT_CK(cudaMalloc((void**)&b->result, fbytes));
  PB_INIT_CK(cudaMalloc((void**)&b->row_n, (size_t)b->R * sizeof(int)));
  int64_t items = 0;
  for (int m = 0; m < count; ++m) items += pr::emu_tile_count((int)n[m], Mode::Full);
  b->items_cap = (int)items;
  b->partial_cap = (int)(items * pr::emu_partials_per_item());
  PB_INIT_CK(cudaMalloc((void**)&b->items, (size_t)items * sizeof(int4)));
  for (int k = 0; k < pr_batch_s::kSlots; ++k) {
    PB_INIT_CK(cudaMallocHost((void**)&b->h_items[k], (size_t)items * sizeof(int4)));
    PB_INIT_CK(cudaMallocHost((void**)&b->h_mats[k], (size_t)count * sizeof(EmuBatchMat)));
    PB_INIT_CK(cudaEventCreateWithFlags(&b->slot_ev[k], cudaEventDisableTiming));
  }
  PB_INIT_CK(cudaMalloc((void**)&b->partial, (size_t)b->partial_cap * sizeof(double)));
  PB_INIT_CK(cudaMalloc((void**)&b->mats, (size_t)count * sizeof(EmuBatchMat)));
  PB_INIT_CK(cudaMalloc((void**)&b->seg, (size_t)2 * count * sizeof(int)));
  PB_INIT_CK(cudaMalloc((void**)&b->res, (size_t)count * sizeof(double)));
  PB_INIT_CK(cudaMalloc((void**)&b->err, sizeof(int)));
  PB_INIT_CK(cudaMalloc((void**)&b->scratch, pr::emu_scratch_bytes()));
  PB_INIT_CK(cudaMemsetAsync(b->err, 0, sizeof(int), b->stream));
  PB_INIT_CK(cudaMallocHost((void**)&b->hres, (size_t)count * sizeof(double)));
  {
    std::vector<int> rn(b->R);
    for (int m = 0; m < count; ++m)
      for (int r = 0; r < b->n[m]; ++r) rn[b->row0[m] + r] = b->n[m];
    PB_INIT_CK(cudaMemcpyAsync(b->row_n, rn.data(), rn.size() * sizeof(int), cudaMemcpyHostToDevice, b->stream));
    PB_INIT_CK(cudaStreamSynchronize(b->stream));
  }
  // Per matrix: checks and the norms of Eq. 3 (all matrices queued, one read-back), then C_0; staged
  // through an n x n work area on the batch's stream, without waiting between matrices.
  double *tA = nullptr, *tC = nullptr, *scal = nullptr, *work = nullptr, *hs = nullptr;
  PB_INIT_CK(cudaMalloc((void**)&tA, (size_t)K * K * sizeof(double)));
  PB_INIT_CK(cudaMalloc((void**)&tC, (size_t)K * K * sizeof(double)));
  PB_INIT_CK(cudaMalloc((void**)&scal, 8 * (size_t)count * sizeof(double)));
  PB_INIT_CK(cudaMalloc((void**)&work, 2 * (size_t)K * sizeof(double)));
  PB_INIT_CK(cudaMallocHost((void**)&hs, 8 * (size_t)count * sizeof(double)));
  pr_status st = PR_OK;
  cudaError_t e = cudaSuccess;
  for (int m = 0; m < count && e == cudaSuccess; ++m) {
    const int nm = b->n[m];
    const size_t pitch = (size_t)b->ld * sizeof(double), w = (size_t)nm * sizeof(double);
    e = cudaMemcpyAsync(tA, A[m], (size_t)nm * nm * sizeof(double), cudaMemcpyDefault, b->stream);
    if (e == cudaSuccess) e = pr::validate(tA, nm, scal + 8 * m, b->stream);
    if (e == cudaSuccess) e = pr::abs_norms(tA, nm, work, scal + 8 * m + 4, b->stream);
    if (e == cudaSuccess)
      e = cudaMemcpy2DAsync(b->A.f + (size_t)b->row0[m] * b->ld, pitch, tA, w, w, nm, cudaMemcpyDeviceToDevice,
                            b->stream);
    b->launches += 4;
  }
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(hs, scal, 8 * (size_t)count * sizeof(double), cudaMemcpyDeviceToHost, b->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
  if (e != cudaSuccess) st = bfail(b, PR_ECUDA, std::string("pr_batch_init: ") + cudaGetErrorName(e));
  for (int m = 0; m < count && st == PR_OK; ++m) {
    const double* h = hs + 8 * m;
    if (h[2] > 0 || h[1] > o.sym_tol * h[0])
      st = bfail(b, PR_EINVAL, "pr_batch_init: matrix " + std::to_string(m) + " is not finite and symmetric");
    else if (h[3] > 0)
      st = bfail(b, PR_ENOTSPD, "pr_batch_init: matrix " + std::to_string(m) + " has a non-positive diagonal");
  }
  for (int m = 0; m < count && st == PR_OK && e == cudaSuccess; ++m) {
    const int nm = b->n[m];
    const double* h = hs + 8 * m;
    const size_t pitch = (size_t)b->ld * sizeof(double), w = (size_t)nm * sizeof(double);
    if (o.c0 == PR_C0_EQ3) {
      e = cudaMemcpy2DAsync(tA, w, b->A.f + (size_t)b->row0[m] * b->ld, pitch, w, nm, cudaMemcpyDeviceToDevice,
                            b->stream);
      if (e == cudaSuccess) e = pr::init_c0_eq3(tA, nm, 1.0 / (h[4] * h[5]), tC, b->stream);
    } else {
      e = pr::set_scaled_identity(tC, nm, pow(h[4], -1.0 / p[m]), b->stream);
    }
    if (e == cudaSuccess)
      e = cudaMemcpy2DAsync(b->X.f + (size_t)b->row0[m] * b->ld, pitch, tC, w, w, nm, cudaMemcpyDeviceToDevice,
                            b->stream);
    b->launches += 1;
  }
  if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
  if (st == PR_OK && e != cudaSuccess) st = bfail(b, PR_ECUDA, std::string("pr_batch_init: ") + cudaGetErrorName(e));
  cudaFree(tA);
  cudaFree(tC);
  cudaFree(scal);
  cudaFree(work);
  cudaFreeHost(hs);
#undef PB_INIT_CK
  if (st != PR_OK) return bail(st);
  *out = b;
  return PR_OK;
}

pr_status pr_batch_solve(pr_batch b, int precision, double tol, int* iterations, int* status) {
  if (!b) return bfail(nullptr, PR_ESTATE, "pr_batch_solve: NULL batch");
  if (precision != PR_EMU64) return bfail(b, PR_EUNSUPPORTED, "pr_batch_solve: batches run PR_EMU64 products");
  if (!(tol >= 0)) return bfail(b, PR_EINVAL, "pr_batch_solve: tol < 0");
  cudaSetDevice(b->device);
  const int count = b->count;
  std::vector<int> sb(count, 0), se(count, 0);
  std::vector<int> ns, cp;  // active Newton-Schulz and coupled matrices
  for (int m = 0; m < count; ++m)
    if (b->active[m]) (b->form[m] == PR_FORM_NS ? ns : cp).push_back(m);
  // Coupled start: M_0 = X_0^p A, N_0 and r_0 (once).
  pr_status s = PR_OK;
  bool fresh = true;
  for (int m : cp) fresh = fresh && b->hist[m].empty();
  if (!cp.empty() && fresh) {
    s = chain(b, b->X, b->A, b->M, b->N, cp, sb, se);
    if (s != PR_OK) return s;
  }
  std::vector<int> prec_hist;
  while (!ns.empty() || !cp.empty()) {
    // Newton-Schulz residual of the current iterate: T = A X (stored transposed), ||I - T||_F.
    if (!ns.empty()) {
      StageOut o;
      o.out = &b->T0;
      o.partial = true;
      o.transpose = true;
      s = stage(b, b->A, b->X, Mode::Full, ns, std::vector<double3>(ns.size(), make_double3(0, 0, 0)), o, &sb, &se);
      if (s == PR_OK) s = read_residuals(b, ns, sb, se);
      if (s != PR_OK) return s;
    }
    // Stop decisions; stopped matrices are copied out and leave the lists.
    std::vector<int> ns2, cp2;
    for (int pass = 0; pass < 2; ++pass) {
      const std::vector<int>& lst = pass == 0 ? ns : cp;
      for (int m : lst) {
        const std::vector<double>& h = b->hist[m];
        prec_hist.assign(h.size(), PR_EMU64);
        int stop = pr::stop_rule(h.data(), prec_hist.data(), (int)h.size(), tol, b->opt);
        if (stop < 0 && b->iterations[m] >= b->opt.max_iter) stop = PR_EMAXITER;
        if (stop >= 0) {
          b->status[m] = stop;
          b->active[m] = 0;
          const size_t off = (size_t)b->row0[m] * b->ld;
          PB_CK(b, cudaMemcpyAsync(b->result + off, b->X.f + off, (size_t)b->n[m] * b->ld * sizeof(double),
                                   cudaMemcpyDeviceToDevice, b->stream));
          // Its rows are no longer sliced (row order -1).
          PB_CK(b, cudaMemsetAsync(b->row_n + b->row0[m], 0xFF, (size_t)b->n[m] * sizeof(int), b->stream));
        } else {
          (pass == 0 ? ns2 : cp2).push_back(m);
        }
      }
    }
    ns.swap(ns2);
    cp.swap(cp2);
    if (ns.empty() && cp.empty()) break;
    // Updates. Newton-Schulz: X' = 2X - X T. Coupled: X' = X N; M' = N^p M with N' and r'.
    {
      StageOut o;
      o.out2 = &b->Xn;
      o.cin = b->X.f;
      s = stage(b, b->X, b->T0, Mode::Sym, ns, std::vector<double3>(ns.size(), make_double3(0.0, -1.0, 2.0)), o,
                nullptr, nullptr);
      if (s != PR_OK) return s;
    }
    {
      StageOut o;
      o.out = &b->Xn;
      s = stage(b, b->X, b->N, Mode::Sym, cp, std::vector<double3>(cp.size(), make_double3(0, 0, 0)), o, nullptr,
                nullptr);
      if (s == PR_OK && !cp.empty()) s = chain(b, b->N, b->M, b->Mn, b->Nn, cp, sb, se);
      if (s != PR_OK) return s;
    }
    // Every matrix still active advanced; buffers of stopped matrices are no longer read.
    std::swap(b->X, b->Xn);
    std::swap(b->M, b->Mn);
    std::swap(b->N, b->Nn);
    for (int m : ns) b->iterations[m] += 1;
    for (int m : cp) b->iterations[m] += 1;
  }
  PB_CK(b, cudaStreamSynchronize(b->stream));
  s = harvest_timing(b);
  if (s != PR_OK) return s;
  for (int m = 0; m < count; ++m) {
    if (iterations) iterations[m] = b->iterations[m];
    if (status) status[m] = b->status[m];
  }
  return PR_OK;
}

pr_status pr_batch_result(pr_batch b, int i, double* C_out) {
  if (!b) return bfail(nullptr, PR_ESTATE, "pr_batch_result: NULL batch");
  if (i < 0 || i >= b->count || !C_out) return bfail(b, PR_EINVAL, "pr_batch_result: bad index or NULL output");
  if (b->status[i] < 0) return bfail(b, PR_ESTATE, "pr_batch_result: matrix not solved yet");
  cudaSetDevice(b->device);
  const size_t w = (size_t)b->n[i] * sizeof(double);
  PB_CK(b, cudaMemcpy2DAsync(C_out, w, b->result + (size_t)b->row0[i] * b->ld, (size_t)b->ld * sizeof(double), w,
                             b->n[i], cudaMemcpyDefault, b->stream));
  PB_CK(b, cudaStreamSynchronize(b->stream));
  return PR_OK;
}

pr_status pr_batch_history(pr_batch b, int i, double* out, int cap, int* len) {
  if (!b) return bfail(nullptr, PR_ESTATE, "pr_batch_history: NULL batch");
  if (i < 0 || i >= b->count) return bfail(b, PR_EINVAL, "pr_batch_history: bad index");
  const std::vector<double>& h = b->hist[i];
  if (len) *len = (int)h.size();
  for (int k = 0; out && k < cap && k < (int)h.size(); ++k) out[k] = h[k];
  return PR_OK;
}

int64_t pr_batch_launches(pr_batch b) { return b ? b->launches : 0; }

pr_status pr_batch_stats(pr_batch b, pr_batch_stats_t* out) {
  if (!b) return bfail(nullptr, PR_ESTATE, "pr_batch_stats: NULL batch");
  if (!out) return bfail(b, PR_EINVAL, "pr_batch_stats: out is NULL");
  *out = b->st;
  out->launches = b->launches;
  out->emu_slices = b->S;
  return PR_OK;
}

pr_status pr_batch_set_timing(pr_batch b, int on) {
  if (!b) return bfail(nullptr, PR_ESTATE, "pr_batch_set_timing: NULL batch");
  cudaSetDevice(b->device);
  b->timing = on != 0;
  return PR_OK;
}

const char* pr_batch_last_error(pr_batch b) { return b ? b->errmsg.c_str() : g_batch_error.c_str(); }

}  // extern "C"
