// Batched solves: many independent problems A_i^{-1/p_i} (SPD matrices of uneven orders and roots) iterated
// together. Every matrix product stage of an iteration is one launch of the digit-slice tensor-core kernel
// over the 128 x 96 tiles of all matrices taking part in that stage; the matrices are packed row-wise in
// shared device buffers with one leading dimension, so one TMA descriptor serves the whole batch.
//
// Per matrix the iteration, the forms (Newton-Schulz for p = 1, coupled for p >= 2, as in capi.cu), the
// initial guess (Eq. 3 or the scaled identity) and the stop rule are those of the single-matrix path. A
// matrix whose stop rule fires is copied to the result buffer and leaves the work lists.
//
// The whole solve is one CUDA graph, launched once per pr_batch_solve: a prologue (the coupled start
// M_0 = X_0^p A), then a device-side while loop whose body is two iterations (the FP64 buffers alternate,
// so two iterations bring them back), then the verification (the true residual ||I - X^p A||_F of every
// coupled-form matrix that stopped, as pr_iterate evaluates it) and the timing harvest. Every decision between launches (which
// matrices take part in a stage, their residuals, their stop rules, the loop condition) is taken by the
// control kernels of k_batch.cu from state kept on the device, so the host neither waits nor builds work
// lists during the solve. The graph is captured on the first pr_batch_solve and reused.
#include "pr_internal.h"

#include <math.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <climits>
#include <numeric>
#include <string>
#include <utility>
#include <vector>

using pr::BatchCtl;
using pr::BatchStage;
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

constexpr int kMaxSlots = 64;  // timing slots: product launches per captured graph
}  // namespace

struct pr_batch_s {
  int count = 0;
  int S = 8;
  int R = 0;   // packed rows (sum of the orders)
  int K = 0;   // largest order
  int ld = 0;  // leading dimension of the packed buffers (K rounded up to 8)
  int pmax = 0;  // largest root of a coupled-form matrix
  bool has_p3 = false;  // some matrix has p = 3 (its update takes two products, update_p3)
  int hcap = 0;  // history entries per matrix (max_iter + 2)
  int bn = 96;   // tile width of the digit-slice products (pr_options.emu_tile, or tuned at init)
  double tune_ms = 0.0;
  cudaStream_t stream = nullptr;
  int device = 0;
  pr_options opt{};
  std::vector<int> n, p, row0, form;
  std::vector<int> pre;                    // per matrix: the batch iterates on 2^pre A (Eq. 2 scaling)
  std::vector<double> norm1, norminf;      // per matrix: norms of the matrix iterated on
  std::vector<double> true_res;            // per matrix: true residual at the stop (-1: none)
  Buf A, X, Xn, M, Mn, N, Nn, T0, T1;
  double* result = nullptr;  // packed results
  int* row_n = nullptr;      // order of the matrix owning each packed row (-1 once it stopped)
  int* row_n_p3 = nullptr;   // the same for rows of p = 3 matrices, -1 on every other row
  int* row_v = nullptr;      // the same for rows of matrices being verified after the loop
  const int* slice_rows = nullptr;  // the per-row orders the digit slicing follows (row_n, or row_v)
  double* truer = nullptr;   // per matrix: true residual from the verification (-1: not verified)
  double* partial = nullptr;
  int4* items = nullptr;     // the current stage's work list
  int* err = nullptr;
  long long* scratch = nullptr;  // PR_EMU64 first-pass totals
  // device-side control (k_batch.cu); one allocation per kind
  int* d_static = nullptr;   // order, n, p, form, row0, off_sym, cnt_sym, off_full, cnt_full
  int4* d_items_all = nullptr;  // every matrix's symmetric items, then every matrix's full items
  int* d_state = nullptr;    // active, status, iters, hlen, loops
  double* d_dstate = nullptr;  // hist (count x hcap), tally[8], params[8]
  int* d_stage = nullptr;    // nitems, member, ofs, seg_b, seg_e
  EmuBatchMat* mats = nullptr;
  unsigned long long* tstamp = nullptr;
  double* flops_pending = nullptr;
  BatchCtl ctl{};
  // loading: an n x n work area, per-matrix checks and norms (device and pinned host)
  double *tA = nullptr, *tC = nullptr, *scal = nullptr, *work = nullptr, *hs = nullptr;
  // host mirrors (pinned) of the state
  int* h_state = nullptr;
  double* h_dstate = nullptr;
  int h_err = 0;
  // the solve graph
  cudaStream_t cap = nullptr;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  cudaGraphConditionalHandle cond = 0;
  int nslots = 0;
  int64_t cnt = 0;  // launches recorded by the capture in progress
  int64_t launches_pro = 0, launches_body = 0, launches_epi = 0;
  double tally_seen[3] = {0.0, 0.0, 0.0};
  // per matrix (host)
  std::vector<std::vector<double>> hist;
  std::vector<int> status, iterations;
  int64_t launches = 0;
  pr_batch_stats_t st{};
  bool timing = false;
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

pr_status ensure_slices(pr_batch b, Buf& x) {
  if (x.sl_valid) return PR_OK;
  PB_CK(b, pr::slice_rows(x.f, b->R, b->K, b->ld, pr::emu_ld(b->K), b->S, b->slice_rows, x.sl, x.ex, b->stream));
  b->cnt += 1;
  x.sl_valid = true;
  return PR_OK;
}

// Digit planes of the rows of p = 3 matrices only; x counts as sliced until the caller says otherwise.
pr_status slice_p3_rows(pr_batch b, Buf& x) {
  PB_CK(b, pr::slice_rows(x.f, b->R, b->K, b->ld, pr::emu_ld(b->K), b->S, b->row_n_p3, x.sl, x.ex, b->stream));
  b->cnt += 1;
  x.sl_valid = true;
  return PR_OK;
}

// What one stage writes.
struct StageOut {
  Buf* out = nullptr;
  Buf* out2 = nullptr;
  const double* cin = nullptr;
  bool partial = false;
  bool transpose = false;
};

// One stage: P = X Y for every member of `sp` (decided on the device when the stage runs), with the
// members' epilogue coefficients; residual partials are reduced and appended to the members' histories.
pr_status stage(pr_batch b, Buf& Xb, Buf& Yb, const BatchStage& sp, const StageOut& so) {
  pr_status s = ensure_slices(b, Xb);
  if (s == PR_OK) s = ensure_slices(b, Yb);
  if (s != PR_OK) return s;
  if (b->nslots >= kMaxSlots) return bfail(b, PR_ECUDA, "pr_batch: too many product stages in one graph");
  BatchStage st = sp;
  st.slot = b->nslots++;
  PB_CK(b, pr::batch_stage_list(b->ctl, st, b->stream));
  Epilogue e;
  if (so.out) e.out = so.out->f;
  if (so.out2) e.out2 = so.out2->f;
  e.cin = so.cin;
  e.partial = so.partial ? b->partial : nullptr;
  PB_CK(b, pr::gemm_emu_batched(Xb.sl, Xb.ex, Yb.sl, Yb.ex, b->R, b->K, pr::emu_ld(b->K), b->ld, b->S,
                                st.full ? Mode::Full : Mode::Sym, so.transpose, b->items, 0, b->ctl.nitems, b->mats, e,
                                b->scratch, b->err, b->tstamp + 2 * st.slot, b->stream, b->bn));
  b->cnt += 2;
  if (so.partial) {
    PB_CK(b, pr::batch_residuals(b->ctl, b->partial, sp.verify, b->stream));
    b->cnt += 1;
  }
  if (so.out) so.out->sl_valid = false;
  if (so.out2) so.out2->sl_valid = false;
  return PR_OK;
}

BatchStage spec(int full, int form, int pcmp, int pj, int fresh, double a = 0.0, double bb = 0.0, double c = 0.0,
                int pskip = 0) {
  BatchStage st{};
  st.full = full;
  st.form = form;
  st.pcmp = pcmp;
  st.pj = pj;
  st.fresh_only = fresh;
  st.pskip = pskip;
  st.a = a;
  st.b = bb;
  st.c = c;
  return st;
}

// Coupled chain of the coupled-form members (except those with p == pskip): Y_1 = F src0, Y_j = F Y_{j-1};
// the p-th product is written as (out, out2 = ((p+1) I - out)/p) with its residual; intermediate products
// go to T0 / T1.
pr_status chain(pr_batch b, Buf& F, Buf& src0, Buf& outM, Buf& outN, int fresh, int pskip) {
  for (int j = 1; j <= b->pmax; ++j) {
    if (j == pskip && j == b->pmax) break;
    Buf& src = j == 1 ? src0 : ((j - 1) & 1 ? b->T0 : b->T1);
    StageOut om;
    om.out = (j & 1) ? &b->T0 : &b->T1;
    pr_status s = stage(b, F, src, spec(0, PR_FORM_COUPLED, 2, j, fresh, 0.0, 0.0, 0.0, pskip), om);
    if (s != PR_OK) return s;
    if (j == pskip) continue;
    StageOut of;
    of.out = &outM;
    of.out2 = &outN;
    of.partial = true;
    s = stage(b, F, src, spec(0, PR_FORM_COUPLED, 1, j, fresh, (double)(j + 1) / j, -1.0 / j, 0.0, pskip), of);
    if (s != PR_OK) return s;
  }
  return PR_OK;
}

// p = 3 members: M' = N^3 M = L R with L = 4M - M^2 and R = (16I - 8M + M^2) / 27, two products (as the
// single-matrix path does). L is formed, and L and R are sliced, on the rows of p = 3 matrices only.
pr_status update_p3(pr_batch b, Buf& outM, Buf& outN) {
  StageOut s1;
  s1.out = &b->T0;
  s1.out2 = &b->T1;
  s1.cin = b->M.f;
  pr_status s = stage(b, b->M, b->M, spec(0, PR_FORM_COUPLED, 1, 3, 0, 16.0 / 27.0, 1.0 / 27.0, -8.0 / 27.0), s1);
  if (s != PR_OK) return s;
  PB_CK(b, pr::batch_lincomb(b->ctl, 3, b->M.f, b->T0.f, 4.0, -1.0, b->T0.f, b->stream));
  b->cnt += 1;
  s = slice_p3_rows(b, b->T0);
  if (s == PR_OK) s = slice_p3_rows(b, b->T1);
  if (s != PR_OK) return s;
  StageOut s2;
  s2.out = &outM;
  s2.out2 = &outN;
  s2.partial = true;
  s = stage(b, b->T0, b->T1, spec(0, PR_FORM_COUPLED, 1, 3, 0, 4.0 / 3.0, -1.0 / 3.0, 0.0), s2);
  b->T0.sl_valid = b->T1.sl_valid = false;  // their planes cover p = 3 rows only
  return s;
}

// One iteration of every iterating matrix: the Newton-Schulz residuals, the stop rules, the updates
// (Newton-Schulz X' = 2X - X T; coupled X' = X N, M' = N^p M with N' and r'), then the buffer swap.
pr_status iteration(pr_batch b, bool last) {
  StageOut o;
  o.out = &b->T0;
  o.partial = true;
  o.transpose = true;
  pr_status s = stage(b, b->A, b->X, spec(1, PR_FORM_NS, 0, 0, 0), o);
  if (s != PR_OK) return s;
  PB_CK(b, pr::batch_decide(b->ctl, b->X.f, b->opt, b->stream));
  b->cnt += 1;
  StageOut u;
  u.out2 = &b->Xn;
  u.cin = b->X.f;
  s = stage(b, b->X, b->T0, spec(0, PR_FORM_NS, 0, 0, 0, 0.0, -1.0, 2.0), u);
  if (s != PR_OK) return s;
  StageOut x;
  x.out = &b->Xn;
  s = stage(b, b->X, b->N, spec(0, PR_FORM_COUPLED, 0, 0, 0), x);
  if (s == PR_OK && b->has_p3) s = update_p3(b, b->Mn, b->Nn);
  if (s == PR_OK) s = chain(b, b->N, b->M, b->Mn, b->Nn, 0, b->has_p3 ? 3 : 0);
  if (s != PR_OK) return s;
  std::swap(b->X, b->Xn);
  std::swap(b->M, b->Mn);
  std::swap(b->N, b->Nn);
  PB_CK(b, pr::batch_advance(b->ctl, b->cond, last ? 1 : 0, b->opt.max_iter + 4, b->stream));
  b->cnt += 1;
  return PR_OK;
}

void invalidate_slices(pr_batch b) {
  for (Buf* x : {&b->A, &b->X, &b->Xn, &b->M, &b->Mn, &b->N, &b->Nn, &b->T0, &b->T1}) x->sl_valid = false;
}

// After the solve loop: ||I - X^p A||_F of every coupled-form matrix that stopped on tol, stagnation or
// max_iter, in the order of pr_residual (P_j = X P_{j-1} symmetric for j = 2..p, then the full product
// P_p A), with X the stopped iterate in the results. Members of stage j are the verified matrices with
// p >= j; P_j lands in T0 (j even) or T1 (j odd), rows of different matrices never overlap, so P_p of a
// matrix with p = j survives later stages and its final product runs right after. The loop's state
// buffers are free by now: the results' digit planes go into Mn's.
pr_status verify(pr_batch b) {
  PB_CK(b, pr::batch_verify_rows(b->ctl, b->stream));
  b->cnt += 1;
  invalidate_slices(b);
  b->A.sl_valid = true;  // sliced on every row by the prologue and not changed since
  b->slice_rows = b->row_v;
  Buf R;
  R.f = b->result;
  R.sl = b->Mn.sl;
  R.ex = b->Mn.ex;
  Buf* P = &R;
  pr_status s = PR_OK;
  for (int j = 2; j <= b->pmax && s == PR_OK; ++j) {
    Buf& out = (j & 1) ? b->T1 : b->T0;
    StageOut o;
    o.out = &out;
    BatchStage st = spec(0, PR_FORM_COUPLED, 2, j - 1, 0);
    st.verify = 1;
    s = stage(b, R, *P, st, o);
    if (s != PR_OK) break;
    P = &out;
    StageOut f;
    f.partial = true;
    BatchStage sf = spec(1, PR_FORM_COUPLED, 1, j, 0);
    sf.verify = 1;
    s = stage(b, out, b->A, sf, f);
  }
  b->slice_rows = b->row_n;
  invalidate_slices(b);
  return s;
}

// Captures the solve graph (prologue, while loop of two iterations, harvest) on a private stream.
pr_status build_graph(pr_batch b) {
  PB_CK(b, pr::emu_prepare());
  if (!b->cap) PB_CK(b, cudaStreamCreateWithFlags(&b->cap, cudaStreamNonBlocking));
  PB_CK(b, cudaGraphCreate(&b->graph, 0));
  PB_CK(b, cudaGraphConditionalHandleCreate(&b->cond, b->graph, 1, cudaGraphCondAssignDefault));
  cudaStream_t user = b->stream;
  b->stream = b->cap;
  b->nslots = 0;
  auto capture = [&](cudaGraph_t g, const cudaGraphNode_t* dep, size_t ndep, auto&& body) -> pr_status {
    cudaError_t e = cudaStreamBeginCaptureToGraph(b->cap, g, dep, nullptr, ndep, cudaStreamCaptureModeRelaxed);
    if (e != cudaSuccess) return bfail(b, PR_ECUDA, std::string("pr_batch: capture: ") + cudaGetErrorName(e));
    b->cnt = 0;
    pr_status s = body();
    cudaGraph_t out = nullptr;
    e = cudaStreamEndCapture(b->cap, &out);
    if (s == PR_OK && e != cudaSuccess) s = bfail(b, PR_ECUDA, std::string("pr_batch: capture: ") + cudaGetErrorName(e));
    return s;
  };
  // Prologue: the coupled start M_0 = X_0^p A, N_0, r_0 of every matrix without a residual yet.
  invalidate_slices(b);
  pr_status s = capture(b->graph, nullptr, 0, [&]() {
    pr_status r = ensure_slices(b, b->A);
    return r == PR_OK ? chain(b, b->X, b->A, b->M, b->N, 1, 0) : r;
  });
  b->launches_pro = b->cnt;
  // The prologue is one chain of nodes: the while loop follows its last node.
  cudaGraphNode_t sink = nullptr;
  if (s == PR_OK) {
    size_t nn = 0;
    cudaError_t e = cudaGraphGetNodes(b->graph, nullptr, &nn);
    std::vector<cudaGraphNode_t> nodes(nn);
    if (e == cudaSuccess) e = cudaGraphGetNodes(b->graph, nodes.data(), &nn);
    for (size_t i = 0; e == cudaSuccess && i < nn; ++i) {
      size_t nd = 0;
      e = cudaGraphNodeGetDependentNodes(nodes[i], nullptr, nullptr, &nd);
      if (e == cudaSuccess && nd == 0) {
        if (sink) e = cudaErrorInvalidValue;  // more than one last node
        sink = nodes[i];
      }
    }
    if (e != cudaSuccess || !sink) s = bfail(b, PR_ECUDA, "pr_batch: prologue graph has no single last node");
  }
  cudaGraphNode_t loop = nullptr;
  cudaGraph_t body = nullptr;
  if (s == PR_OK) {
    cudaGraphNodeParams cp{};
    cp.type = cudaGraphNodeTypeConditional;
    cp.conditional.handle = b->cond;
    cp.conditional.type = cudaGraphCondTypeWhile;
    cp.conditional.size = 1;
    cudaError_t e = cudaGraphAddNode(&loop, b->graph, &sink, nullptr, 1, &cp);
    if (e != cudaSuccess) s = bfail(b, PR_ECUDA, std::string("pr_batch: loop node: ") + cudaGetErrorName(e));
    else body = cp.conditional.phGraph_out[0];
  }
  // Loop body: two iterations. At its entry only A's digit planes are known to be current.
  if (s == PR_OK) {
    invalidate_slices(b);
    b->A.sl_valid = true;
    s = capture(body, nullptr, 0, [&]() {
      pr_status r = iteration(b, false);
      return r == PR_OK ? iteration(b, true) : r;
    });
    b->launches_body = b->cnt;
  }
  if (s == PR_OK) {
    s = capture(b->graph, &loop, 1, [&]() -> pr_status {
      if (b->pmax >= 2 && b->opt.verify) {
        pr_status r = verify(b);
        if (r != PR_OK) return r;
      }
      PB_CK(b, pr::batch_harvest(b->ctl, b->nslots, b->stream));
      b->cnt += 1;
      return PR_OK;
    });
    b->launches_epi = b->cnt;
  }
  if (s == PR_OK) {
    cudaError_t e = cudaGraphInstantiate(&b->exec, b->graph, 0);
    if (e != cudaSuccess) s = bfail(b, PR_ECUDA, std::string("pr_batch: instantiate: ") + cudaGetErrorName(e));
  }
  b->stream = user;
  invalidate_slices(b);
  if (s != PR_OK) {
    if (b->exec) cudaGraphExecDestroy(b->exec);
    if (b->graph) cudaGraphDestroy(b->graph);
    b->exec = nullptr;
    b->graph = nullptr;
  }
  return s;
}

// Copies the matrices in (device or host), checks them as pr_init does, forms the norms of Eq. 3 and C_0,
// and resets every matrix to "iterating, no residual yet". The solve graph (if captured) stays valid.
pr_status load(pr_batch b, const double* const* A, const char* who) {
  const int count = b->count;
  for (int m = 0; m < count; ++m)
    if (!A[m]) return bfail(b, PR_EINVAL, std::string(who) + ": NULL matrix");
  {
    std::vector<int> rn(b->R), rn3(b->R);
    for (int m = 0; m < count; ++m)
      for (int r = 0; r < b->n[m]; ++r) {
        rn[b->row0[m] + r] = b->n[m];
        rn3[b->row0[m] + r] = b->p[m] == 3 ? b->n[m] : -1;
      }
    std::vector<int> st0(4 * (size_t)count, 0);
    std::fill(st0.begin(), st0.begin() + count, 1);               // active
    std::fill(st0.begin() + count, st0.begin() + 2 * count, -1);  // status
    PB_CK(b, cudaMemcpyAsync(b->row_n, rn.data(), rn.size() * sizeof(int), cudaMemcpyHostToDevice, b->stream));
    PB_CK(b, cudaMemcpyAsync(b->row_n_p3, rn3.data(), rn3.size() * sizeof(int), cudaMemcpyHostToDevice, b->stream));
    PB_CK(b, cudaMemcpyAsync(b->d_state, st0.data(), st0.size() * sizeof(int), cudaMemcpyHostToDevice, b->stream));
    PB_CK(b, cudaStreamSynchronize(b->stream));
  }
  for (int m = 0; m < count; ++m) {
    b->status[m] = -1;
    b->iterations[m] = 0;
    b->hist[m].clear();
    b->true_res[m] = -1.0;
  }
  // Per matrix: checks and the norms of Eq. 3 (all matrices queued, one read-back), then C_0; staged
  // through an n x n work area on the batch's stream, without waiting between matrices.
  cudaError_t e = cudaSuccess;
  for (int m = 0; m < count && e == cudaSuccess; ++m) {
    const int nm = b->n[m];
    const size_t pitch = (size_t)b->ld * sizeof(double), w = (size_t)nm * sizeof(double);
    e = cudaMemcpyAsync(b->tA, A[m], (size_t)nm * nm * sizeof(double), cudaMemcpyDefault, b->stream);
    if (e == cudaSuccess) e = pr::validate(b->tA, nm, b->scal + 8 * m, b->stream);
    if (e == cudaSuccess) e = pr::abs_norms(b->tA, nm, b->work, b->scal + 8 * m + 4, b->stream);
    if (e == cudaSuccess)
      e = cudaMemcpy2DAsync(b->A.f + (size_t)b->row0[m] * b->ld, pitch, b->tA, w, w, nm, cudaMemcpyDeviceToDevice,
                            b->stream);
    b->launches += 4;
  }
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(b->hs, b->scal, 8 * (size_t)count * sizeof(double), cudaMemcpyDeviceToHost, b->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
  if (e != cudaSuccess) return bfail(b, PR_ECUDA, std::string(who) + ": " + cudaGetErrorName(e));
  for (int m = 0; m < count; ++m) {
    const double* h = b->hs + 8 * m;
    if (h[2] > 0 || h[1] > b->opt.sym_tol * h[0])
      return bfail(b, PR_EINVAL, std::string(who) + ": matrix " + std::to_string(m) + " is not finite and symmetric");
    if (h[3] > 0)
      return bfail(b, PR_ENOTSPD, std::string(who) + ": matrix " + std::to_string(m) +
                                      " is not positive definite (a non-positive diagonal entry, or a diagonal block "
                                      "of order 64 without a Cholesky factorisation)");
  }
  // Eq. 2 for Eq. 3's C_0 with p > 1 needs ||A||_1 >= 1: such matrices are scaled by an exact power of two
  // into ||2^k A||_1 in [1, 2), as pr_load does; pr_batch_result scales the root back by 2^(k/p).
  for (int m = 0; m < count && e == cudaSuccess; ++m) {
    double* h = b->hs + 8 * m;
    b->pre[m] = 0;
    if (b->p[m] > 1 && h[4] * h[5] < 1.0) {
      const int nm = b->n[m];
      const size_t pitch = (size_t)b->ld * sizeof(double), w = (size_t)nm * sizeof(double);
      int ex = 0;
      frexp(h[4], &ex);
      const double c = ldexp(1.0, 1 - ex);
      double* rows = b->A.f + (size_t)b->row0[m] * b->ld;
      e = cudaMemcpy2DAsync(b->tA, w, rows, pitch, w, nm, cudaMemcpyDeviceToDevice, b->stream);
      if (e == cudaSuccess) e = pr::lincomb(b->tA, b->tA, (int64_t)nm * nm, c, 0.0, b->tA, b->stream);
      if (e == cudaSuccess) e = cudaMemcpy2DAsync(rows, pitch, b->tA, w, w, nm, cudaMemcpyDeviceToDevice, b->stream);
      b->launches += 1;
      h[4] *= c;
      h[5] *= c;
      b->pre[m] = 1 - ex;
    }
    b->norm1[m] = h[4];
    b->norminf[m] = h[5];
  }
  for (int m = 0; m < count && e == cudaSuccess; ++m) {
    const int nm = b->n[m];
    const double* h = b->hs + 8 * m;
    const size_t pitch = (size_t)b->ld * sizeof(double), w = (size_t)nm * sizeof(double);
    if (b->opt.c0 == PR_C0_EQ3) {
      e = cudaMemcpy2DAsync(b->tA, w, b->A.f + (size_t)b->row0[m] * b->ld, pitch, w, nm, cudaMemcpyDeviceToDevice,
                            b->stream);
      if (e == cudaSuccess) e = pr::init_c0_eq3(b->tA, nm, 1.0 / (h[4] * h[5]), b->tC, b->stream);
    } else {
      e = pr::set_scaled_identity(b->tC, nm, pow(h[4], -1.0 / b->p[m]), b->stream);
    }
    if (e == cudaSuccess)
      e = cudaMemcpy2DAsync(b->X.f + (size_t)b->row0[m] * b->ld, pitch, b->tC, w, w, nm, cudaMemcpyDeviceToDevice,
                            b->stream);
    b->launches += 1;
  }
  if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
  if (e != cudaSuccess) return bfail(b, PR_ECUDA, std::string(who) + ": " + cudaGetErrorName(e));
  return PR_OK;
}

// The tile width of the batch's products (pr_options.emu_tile = 0): the symmetric product A A of every
// matrix, as one launch over all their tiles, timed (best of two) with 128 x 96 and with 128 x 48 tiles on
// the batch's stream; the faster width is kept for every stage. (Small orders waste less of a narrower tile;
// large ones issue fewer, larger MMAs with the wider one.)
pr_status tune_batch(pr_batch b) {
  pr_status s = ensure_slices(b, b->A);
  if (s != PR_OK) return s;
  std::vector<EmuBatchMat> mats(b->count);
  for (int m = 0; m < b->count; ++m) mats[m] = EmuBatchMat{b->n[m], b->row0[m], 0.0, 0.0, 0.0};
  EmuBatchMat* dmats = nullptr;
  int4* ditems = nullptr;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  float best = 1e30f;
  int pick = 96;
  cudaError_t e = cudaMalloc((void**)&dmats, mats.size() * sizeof(EmuBatchMat));
  if (e == cudaSuccess) e = cudaMemcpy(dmats, mats.data(), mats.size() * sizeof(EmuBatchMat), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaEventCreate(&e0);
  if (e == cudaSuccess) e = cudaEventCreate(&e1);
  for (int bn : {96, 48}) {
    if (e != cudaSuccess) break;
    std::vector<int4> items;
    for (int m = 0; m < b->count; ++m) pr::emu_tile_list(m, b->n[m], Mode::Sym, items, bn);
    if (ditems) cudaFree(ditems);
    ditems = nullptr;
    e = cudaMalloc((void**)&ditems, items.size() * sizeof(int4));
    if (e == cudaSuccess) e = cudaMemcpy(ditems, items.data(), items.size() * sizeof(int4), cudaMemcpyHostToDevice);
    Epilogue ep;
    ep.out = b->T0.f;
    float t = 1e30f;
    for (int rep = 0; rep < 2 && e == cudaSuccess; ++rep) {
      e = cudaEventRecord(e0, b->stream);
      if (e == cudaSuccess)
        e = pr::gemm_emu_batched(b->A.sl, b->A.ex, b->A.sl, b->A.ex, b->R, b->K, pr::emu_ld(b->K), b->ld, b->S,
                                 Mode::Sym, false, ditems, (int)items.size(), nullptr, dmats, ep, b->scratch, b->err,
                                 nullptr, b->stream, bn);
      if (e == cudaSuccess) e = cudaEventRecord(e1, b->stream);
      if (e == cudaSuccess) e = cudaEventSynchronize(e1);
      float ms = 0.f;
      if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
      t = std::min(t, ms);
      b->launches += 1;
    }
    b->tune_ms += 2 * t;
    if (t < best) {
      best = t;
      pick = bn;
    }
  }
  if (ditems) cudaFree(ditems);
  if (dmats) cudaFree(dmats);
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  if (e != cudaSuccess) return bfail(b, PR_ECUDA, std::string("pr_batch_init: tile tuning: ") + cudaGetErrorName(e));
  int word = 0;
  PB_CK(b, cudaMemcpy(&word, b->err, sizeof(int), cudaMemcpyDeviceToHost));
  if (word != 0) return bfail(b, PR_ETIMEOUT, "pr_batch_init: a bounded device wait expired while tuning");
  b->bn = pick;
  return PR_OK;
}

}  // namespace

extern "C" {

pr_status pr_batch_destroy(pr_batch b) {
  if (!b) return PR_OK;
  cudaSetDevice(b->device);
  if (b->stream) cudaStreamSynchronize(b->stream);
  if (b->exec) cudaGraphExecDestroy(b->exec);
  if (b->graph) cudaGraphDestroy(b->graph);
  if (b->cap) cudaStreamDestroy(b->cap);
  for (Buf* x : {&b->A, &b->X, &b->Xn, &b->M, &b->Mn, &b->N, &b->Nn, &b->T0, &b->T1}) {
    if (x->f) cudaFree(x->f);
    if (x->sl) cudaFree(x->sl);
    if (x->ex) cudaFree(x->ex);
  }
  for (void* q : {(void*)b->result, (void*)b->row_n, (void*)b->row_n_p3, (void*)b->row_v, (void*)b->truer,
                  (void*)b->partial, (void*)b->items, (void*)b->err,
                  (void*)b->scratch, (void*)b->d_static, (void*)b->d_items_all, (void*)b->d_state, (void*)b->d_dstate,
                  (void*)b->d_stage, (void*)b->mats, (void*)b->tstamp, (void*)b->flops_pending, (void*)b->tA,
                  (void*)b->tC, (void*)b->scal, (void*)b->work})
    if (q) cudaFree(q);
  if (b->hs) cudaFreeHost(b->hs);
  if (b->h_state) cudaFreeHost(b->h_state);
  if (b->h_dstate) cudaFreeHost(b->h_dstate);
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
  if (o.emu_slices < 0 || o.emu_slices > pr::emu_max_slices() || o.max_iter < 0 ||
      (o.emu_tile != 0 && !pr::emu_tile_width_ok(o.emu_tile)))
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
  b->pre.assign(count, 0);
  b->norm1.assign(count, 0.0);
  b->norminf.assign(count, 0.0);
  b->true_res.assign(count, -1.0);
  b->status.assign(count, -1);
  b->iterations.assign(count, 0);
  b->hcap = o.max_iter + 2;
  b->bn = o.emu_tile != 0 ? o.emu_tile : 96;
  int row = 0;
  for (int m = 0; m < count; ++m) {
    b->n[m] = (int)n[m];
    b->p[m] = p[m];
    b->row0[m] = row;
    b->form[m] = p[m] == 1 ? PR_FORM_NS : PR_FORM_COUPLED;
    if (p[m] > 1) b->pmax = std::max(b->pmax, p[m]);
    if (p[m] == 3) b->has_p3 = true;
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
  PB_INIT_CK(cudaMalloc((void**)&b->row_n_p3, (size_t)b->R * sizeof(int)));
  PB_INIT_CK(cudaMalloc((void**)&b->row_v, (size_t)b->R * sizeof(int)));
  PB_INIT_CK(cudaMalloc((void**)&b->truer, (size_t)count * sizeof(double)));
  b->slice_rows = b->row_n;
  // Device-side control state (independent of the tile width) and the loading work areas.
  const size_t hist_len = (size_t)count * b->hcap;
  PB_INIT_CK(cudaMalloc((void**)&b->mats, (size_t)count * sizeof(EmuBatchMat)));
  PB_INIT_CK(cudaMalloc((void**)&b->err, sizeof(int)));
  PB_INIT_CK(cudaMalloc((void**)&b->scratch, pr::emu_scratch_bytes()));
  PB_INIT_CK(cudaMemsetAsync(b->err, 0, sizeof(int), b->stream));
  PB_INIT_CK(cudaMalloc((void**)&b->d_state, (4 * (size_t)count + 1) * sizeof(int)));
  PB_INIT_CK(cudaMalloc((void**)&b->d_dstate, (hist_len + 16) * sizeof(double)));
  PB_INIT_CK(cudaMalloc((void**)&b->d_stage, (1 + 4 * (size_t)count) * sizeof(int)));
  PB_INIT_CK(cudaMalloc((void**)&b->tstamp, 2 * kMaxSlots * sizeof(unsigned long long)));
  PB_INIT_CK(cudaMalloc((void**)&b->flops_pending, kMaxSlots * sizeof(double)));
  PB_INIT_CK(cudaMallocHost((void**)&b->h_state, (4 * (size_t)count + 1) * sizeof(int)));
  PB_INIT_CK(cudaMallocHost((void**)&b->h_dstate, (hist_len + 16) * sizeof(double)));
  {
    std::vector<int> st0(4 * (size_t)count + 1, 0);
    std::fill(st0.begin(), st0.begin() + count, 1);               // active
    std::fill(st0.begin() + count, st0.begin() + 2 * count, -1);  // status
    std::vector<unsigned long long> ts(2 * kMaxSlots);
    for (int k = 0; k < kMaxSlots; ++k) {
      ts[2 * k] = ULLONG_MAX;
      ts[2 * k + 1] = 0ull;
    }
    PB_INIT_CK(cudaMemcpy(b->d_state, st0.data(), st0.size() * sizeof(int), cudaMemcpyHostToDevice));
    PB_INIT_CK(cudaMemset(b->d_dstate, 0, (hist_len + 16) * sizeof(double)));
    PB_INIT_CK(cudaMemcpy(b->tstamp, ts.data(), ts.size() * sizeof(unsigned long long), cudaMemcpyHostToDevice));
    PB_INIT_CK(cudaMemset(b->flops_pending, 0, kMaxSlots * sizeof(double)));
  }
  PB_INIT_CK(cudaMalloc((void**)&b->tA, (size_t)K * K * sizeof(double)));
  PB_INIT_CK(cudaMalloc((void**)&b->tC, (size_t)K * K * sizeof(double)));
  PB_INIT_CK(cudaMalloc((void**)&b->scal, 8 * (size_t)count * sizeof(double)));
  PB_INIT_CK(cudaMalloc((void**)&b->work, 2 * (size_t)K * sizeof(double)));
  PB_INIT_CK(cudaMallocHost((void**)&b->hs, 8 * (size_t)count * sizeof(double)));
  pr_status st = load(b, A, "pr_batch_init");
  if (st == PR_OK && o.emu_tile == 0) st = tune_batch(b);
  if (st != PR_OK) return bail(st);
  // Every matrix's work items (symmetric and full) for the tile width in use, and the static description.
  std::vector<int4> isym, ifull;
  std::vector<int> stat(9 * (size_t)count);
  int* s_order = stat.data();
  std::iota(s_order, s_order + count, 0);
  std::stable_sort(s_order, s_order + count, [&](int x, int y) { return b->n[x] > b->n[y]; });
  for (int m = 0; m < count; ++m) {
    stat[count + m] = b->n[m];
    stat[2 * count + m] = b->p[m];
    stat[3 * count + m] = b->form[m];
    stat[4 * count + m] = b->row0[m];
    stat[5 * count + m] = (int)isym.size();
    pr::emu_tile_list(m, b->n[m], Mode::Sym, isym, b->bn);
    stat[6 * count + m] = (int)isym.size() - stat[5 * count + m];
    stat[7 * count + m] = (int)ifull.size();
    pr::emu_tile_list(m, b->n[m], Mode::Full, ifull, b->bn);
    stat[8 * count + m] = (int)ifull.size() - stat[7 * count + m];
  }
  const size_t items = ifull.size();  // no stage has more items than every matrix's full product
  PB_INIT_CK(cudaMalloc((void**)&b->items, items * sizeof(int4)));
  PB_INIT_CK(cudaMalloc((void**)&b->partial, items * pr::emu_partials_per_item() * sizeof(double)));
  PB_INIT_CK(cudaMalloc((void**)&b->d_static, stat.size() * sizeof(int)));
  PB_INIT_CK(cudaMalloc((void**)&b->d_items_all, (isym.size() + ifull.size()) * sizeof(int4)));
  PB_INIT_CK(cudaMemcpy(b->d_static, stat.data(), stat.size() * sizeof(int), cudaMemcpyHostToDevice));
  PB_INIT_CK(cudaMemcpy(b->d_items_all, isym.data(), isym.size() * sizeof(int4), cudaMemcpyHostToDevice));
  PB_INIT_CK(cudaMemcpy(b->d_items_all + isym.size(), ifull.data(), ifull.size() * sizeof(int4),
                        cudaMemcpyHostToDevice));
  {
    BatchCtl& c = b->ctl;
    const int* d = b->d_static;
    c.count = count;
    c.hcap = b->hcap;
    c.per = pr::emu_partials_per_item();
    c.ld = b->ld;
    c.order = d;
    c.n = d + count;
    c.p = d + 2 * count;
    c.form = d + 3 * count;
    c.row0 = d + 4 * count;
    c.off_sym = d + 5 * count;
    c.cnt_sym = d + 6 * count;
    c.off_full = d + 7 * count;
    c.cnt_full = d + 8 * count;
    c.items_sym = b->d_items_all;
    c.items_full = b->d_items_all + isym.size();
    c.active = b->d_state;
    c.status = b->d_state + count;
    c.iters = b->d_state + 2 * count;
    c.hlen = b->d_state + 3 * count;
    c.loops = b->d_state + 4 * count;
    c.hist = b->d_dstate;
    c.tally = b->d_dstate + hist_len;
    c.params = b->d_dstate + hist_len + 8;
    c.items = b->items;
    c.nitems = b->d_stage;
    c.mats = b->mats;
    c.member = b->d_stage + 1;
    c.ofs = b->d_stage + 1 + count;
    c.seg_b = b->d_stage + 1 + 2 * count;
    c.seg_e = b->d_stage + 1 + 3 * count;
    c.tstamp = b->tstamp;
    c.flops_pending = b->flops_pending;
    c.result = b->result;
    c.row_n = b->row_n;
    c.row_n2 = b->row_n_p3;
    c.err = b->err;
    c.truer = b->truer;
    c.row_v = b->row_v;
  }
#undef PB_INIT_CK
  *out = b;
  return PR_OK;
}

pr_status pr_batch_load(pr_batch b, const double* const* A) {
  if (!b) return bfail(nullptr, PR_ESTATE, "pr_batch_load: NULL batch");
  if (!A) return bfail(b, PR_EINVAL, "pr_batch_load: A is NULL");
  cudaSetDevice(b->device);
  return load(b, A, "pr_batch_load");
}

pr_status pr_batch_solve(pr_batch b, int precision, double tol, int* iterations, int* status) {
  if (!b) return bfail(nullptr, PR_ESTATE, "pr_batch_solve: NULL batch");
  if (precision != PR_EMU64) return bfail(b, PR_EUNSUPPORTED, "pr_batch_solve: batches run PR_EMU64 products");
  if (!(tol >= 0)) return bfail(b, PR_EINVAL, "pr_batch_solve: tol < 0");
  cudaSetDevice(b->device);
  if (!b->exec) {
    pr_status s = build_graph(b);
    if (s != PR_OK) return s;
  }
  const int count = b->count;
  const size_t hist_len = (size_t)count * b->hcap;
  b->h_dstate[hist_len + 8] = tol;
  PB_CK(b, cudaMemcpyAsync(b->d_dstate + hist_len + 8, b->h_dstate + hist_len + 8, sizeof(double),
                           cudaMemcpyHostToDevice, b->stream));
  PB_CK(b, cudaMemsetAsync(b->ctl.loops, 0, sizeof(int), b->stream));  // the pass limit is per solve
  const pr::NvtxRange trace("pr_batch_solve graph");
  PB_CK(b, cudaGraphLaunch(b->exec, b->stream));
  PB_CK(b, cudaMemcpyAsync(b->h_state, b->d_state, (4 * (size_t)count + 1) * sizeof(int), cudaMemcpyDeviceToHost,
                           b->stream));
  PB_CK(b, cudaMemcpyAsync(b->h_dstate, b->d_dstate, (hist_len + 8) * sizeof(double), cudaMemcpyDeviceToHost,
                           b->stream));
  PB_CK(b, cudaMemcpyAsync(&b->h_err, b->err, sizeof(int), cudaMemcpyDeviceToHost, b->stream));
  const bool verified = b->pmax >= 2 && b->opt.verify;
  if (verified)
    PB_CK(b, cudaMemcpyAsync(b->true_res.data(), b->truer, (size_t)count * sizeof(double), cudaMemcpyDeviceToHost,
                             b->stream));
  PB_CK(b, cudaStreamSynchronize(b->stream));
  // Launches: the prologue and the harvest once, the loop body once per pass.
  const int loops = b->h_state[4 * count];
  b->launches += b->launches_pro + (int64_t)loops * b->launches_body + b->launches_epi;
  const double* tally = b->h_dstate + hist_len;
  b->st.stages = (int64_t)tally[3];
  b->st.products = (int64_t)tally[4];
  b->st.product_flops = tally[5];
  if (b->timing) {
    b->st.stage_ms += (tally[0] - b->tally_seen[0]) * 1e-6;
    b->st.stage_flops_timed += tally[1] - b->tally_seen[1];
    b->st.stages_timed += (int64_t)(tally[2] - b->tally_seen[2]);
  }
  for (int k = 0; k < 3; ++k) b->tally_seen[k] = tally[k];
  for (int m = 0; m < count; ++m) {
    b->status[m] = b->h_state[count + m];
    b->iterations[m] = b->h_state[2 * count + m];
    const int len = b->h_state[3 * count + m];
    b->hist[m].assign(b->h_dstate + (size_t)m * b->hcap, b->h_dstate + (size_t)m * b->hcap + len);
    if (b->form[m] != PR_FORM_COUPLED) {
      b->true_res[m] = (b->status[m] >= 0 && b->status[m] != PR_EDIVERGED && len > 0) ? b->hist[m].back() : -1.0;
    } else if (!verified) {
      b->true_res[m] = -1.0;
    } else if (b->status[m] == PR_OK && !(b->true_res[m] <= tol)) {
      b->status[m] = PR_EINACCURATE;  // ||I - M||_F met tol, the true residual did not (see pr_iterate)
    }
    if (iterations) iterations[m] = b->iterations[m];
    if (status) status[m] = b->status[m];
  }
  if (b->h_err != 0) {
    cudaMemsetAsync(b->err, 0, sizeof(int), b->stream);
    return bfail(b, PR_ETIMEOUT,
                 "pr_batch: a bounded device wait expired (code " + std::to_string(b->h_err) + ")");
  }
  for (int m = 0; m < count; ++m)
    if (b->status[m] < 0)
      return bfail(b, PR_ECUDA, "pr_batch_solve: the solve loop ended with matrix " + std::to_string(m) + " iterating");
  return PR_OK;
}

pr_status pr_batch_result(pr_batch b, int i, double* C_out) {
  if (!b) return bfail(nullptr, PR_ESTATE, "pr_batch_result: NULL batch");
  if (i < 0 || i >= b->count || !C_out) return bfail(b, PR_EINVAL, "pr_batch_result: bad index or NULL output");
  if (b->status[i] < 0) return bfail(b, PR_ESTATE, "pr_batch_result: matrix not solved yet");
  cudaSetDevice(b->device);
  const size_t w = (size_t)b->n[i] * sizeof(double);
  const double* rows = b->result + (size_t)b->row0[i] * b->ld;
  if (b->pre[i] != 0) {
    // The batch iterated on 2^k A: the root of A is 2^(k/p) times the result.
    const int64_t nn = (int64_t)b->n[i] * b->n[i];
    PB_CK(b, cudaMemcpy2DAsync(b->tA, w, rows, (size_t)b->ld * sizeof(double), w, b->n[i], cudaMemcpyDeviceToDevice,
                               b->stream));
    PB_CK(b, pr::lincomb(b->tA, b->tA, nn, exp2((double)b->pre[i] / b->p[i]), 0.0, b->tA, b->stream));
    b->launches += 1;
    PB_CK(b, cudaMemcpyAsync(C_out, b->tA, (size_t)nn * sizeof(double), cudaMemcpyDefault, b->stream));
  } else {
    PB_CK(b, cudaMemcpy2DAsync(C_out, w, rows, (size_t)b->ld * sizeof(double), w, b->n[i], cudaMemcpyDefault,
                               b->stream));
  }
  PB_CK(b, cudaStreamSynchronize(b->stream));
  return PR_OK;
}

pr_status pr_batch_matrix(pr_batch b, int i, pr_batch_matrix_t* out) {
  if (!b) return bfail(nullptr, PR_ESTATE, "pr_batch_matrix: NULL batch");
  if (i < 0 || i >= b->count || !out) return bfail(b, PR_EINVAL, "pr_batch_matrix: bad index or NULL output");
  out->n = b->n[i];
  out->p = b->p[i];
  out->form = b->form[i];
  out->status = b->status[i];
  out->iterations = b->iterations[i];
  out->norm_1 = b->norm1[i];
  out->norm_inf = b->norminf[i];
  out->prescale_log2 = b->pre[i];
  out->true_residual = b->true_res[i];
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
  out->tile_n = b->bn;
  out->tune_ms = b->tune_ms;
  return PR_OK;
}

pr_status pr_batch_set_timing(pr_batch b, int on) {
  if (!b) return bfail(nullptr, PR_ESTATE, "pr_batch_set_timing: NULL batch");
  b->timing = on != 0;
  return PR_OK;
}

const char* pr_batch_last_error(pr_batch b) { return b ? b->errmsg.c_str() : g_batch_error.c_str(); }

}  // extern "C"
