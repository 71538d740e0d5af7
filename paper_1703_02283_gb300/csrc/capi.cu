// Host runtime behind the C ABI of include/pthroot.h: handle state, the three evaluation orders of
// Eq. 1 (coupled, Newton-Schulz, literal), the stop rule and the precision ladder (Sec. 3: low-precision
// arithmetic for most iterations, then precise refinement).
#include "pr_internal.h"

#include <math.h>
#include <stdio.h>
#include <string.h>

#include <map>
#include <mutex>
#include <string>
#include <tuple>
#include <utility>
#include <vector>

using pr::Epilogue;
using pr::Mode;

namespace {
thread_local std::string g_init_error;  // text of the last failing pr_init (no handle to hold it)

// Precision levels: a switch to a higher level re-forms the coupled product M at that level.
int precision_level(int prec) {
  switch (prec) {
    case PR_FP8: return 0;
    case PR_BF16: return 1;
    case PR_FP32X: return 2;
    default: return 3;  // PR_FP64, PR_EMU64
  }
}

// Digit planes a PR_FP32X product uses: 3 of the 8 base-256 digits (24 bits per row, the significand width
// of FP32), 6 exact digit-pair products.
constexpr int kFp32xSlices = 3;

// One matrix in the two representations the products use: FP64 (leading dimension n) and BF16
// (leading dimension ldl, the operand of the tensor-core products).
struct Mat {
  double* f = nullptr;
  __nv_bfloat16* b = nullptr;
  __half* sl = nullptr;         // PR_EMU64: S FP16 digit planes of f (allocated on first use)
  int* ex = nullptr;            // PR_EMU64: row exponents of the digit planes
  bool sl_valid = false;        // the digit planes describe the current f
  uint8_t* q = nullptr;         // PR_FP8: E4M3 copy of f / 2^qe (row by row), allocated on first use
  int* qe = nullptr;            // PR_FP8: row scales (exponents)
  bool q_valid = false;         // the E4M3 copy describes the current f
  bool b_valid = false;         // pr_refine: the BF16 copy describes the current f (read by lp_operand only)
  void changed() { sl_valid = q_valid = b_valid = false; }  // f was written
};

void swap(Mat& a, Mat& b) { std::swap(a, b); }

// What one product writes; product() maps it onto the kernel epilogue of the chosen precision.
struct Out {
  Mat* out = nullptr;        // P
  bool out_master = true;    // low precision: also keep the FP64 copy of P
  Mat* out2 = nullptr;       // a I + b P + c cin
  bool out2_master = true;
  const double* cin = nullptr;
  double a = 0.0, b = 0.0, c = 0.0;
  bool partial = false;      // per-tile sums of the residual ||I - P||_F^2
  bool transpose = false;    // full-mode products whose result is the B operand of a later product
  bool lp_copy = true;       // BF16: also write the BF16 copies of out / out2 (operands of later BF16 products)
};
}  // namespace

struct pr_handle_s {
  int64_t n = 0;
  int p = 1;
  int form = PR_FORM_COUPLED;
  pr_options opt{};
  cudaStream_t stream = nullptr;
  int device = 0;
  int ldl = 0;  // leading dimension of the BF16 copies
  int ldq = 0;  // leading dimension (bytes) of the E4M3 copies
  int eld = 0;  // K extent of a PR_EMU64 digit-plane row (n rounded up to 16)
  int S = 8;    // digit planes per operand for PR_EMU64
  // PR_EMU64 / PR_FP32X work lists per product mode (symmetric, full) and variant (kEmuVariants: tile width
  // 96 or 48, whole tiles or tiles split over K); a variant that does not apply has no list.
  int4* emu_items[2][4] = {};
  int emu_nitems[2][4] = {};
  int emu_nsplit[2][4] = {};                 // split tiles of each list (0: whole tiles)
  int emu_plan[2][2] = {{-1, -1}, {-1, -1}}; // [mode][0: PR_EMU64, 1: PR_FP32X] chosen variant, -1 not yet
  long long* emu_scratch = nullptr;          // PR_EMU64 first-pass totals (pr::emu_scratch_bytes())
  long long* emu_split = nullptr;            // PR_EMU64 half totals of tiles split over K (pr::emu_launch_list)
  int* emu_split_cnt = nullptr;
  // Block-sparse A (pr_options.block_sparse): per row of the loaded A the first and last non-zero column, and
  // work lists of the unsplit variants restricted to the K steps the rows of A in a tile can reach,
  // [mode][width 96 / 48][A the first operand, the second, both], rebuilt after each pr_load.
  int* span_dev = nullptr;                   // 2n ints
  std::vector<int> a_first, a_last;
  bool sp_on = false;
  int4* sp_items[2][2][3] = {};
  bool sp_built[2][2][3] = {};

  // The input, the iterate X, the carried product M and operand N of the coupled form, their next
  // values, and two scratch products.
  Mat A, X, Xn, M, Mn, N, Nn, T0, T1;
  bool lp_stale = true;       // BF16 copies of A, X, M, N are out of date
  double* partial = nullptr;  // per-tile residual partial sums
  double* work = nullptr;     // 2n doubles (column and row abs-sums)
  double* scal = nullptr;     // device scalars: [0..3] checks, [4..5] norms, [6] residual, [7] error word
  double* hpin = nullptr;     // pinned host mirror of scal
  double* vec = nullptr;      // PR_C0_POLY gate and features: 4n vectors + reduction partials + scalars
  double* xbest = nullptr;    // pr_solve_ladder: the iterate with the lowest true residual at a rung boundary
  double* xstart = nullptr;   // pr_solve_ladder: the starting iterate, for a rung that diverges
  Mat Ra, Rb, Rc;             // pr_refine: three more matrices, allocated on its first call
  double* rdev = nullptr;     // pr_refine: reduction work area and device scalars
  double* rpin = nullptr;     // pr_refine: pinned host mirror of its scalars
  bool powers_valid = false;  // T0 = A^2 and T1 = A^3 of the loaded A (features, polynomial guess)

  // CUDA-event timing of the product kernels (pr_set_timing).
  bool timing = false;
  std::vector<cudaEvent_t> ev;  // pairs: ev[2i] before, ev[2i + 1] after product i
  std::vector<double> ev_flops;
  std::vector<int> ev_prec;
  int ev_pending = 0;

  bool state_ready = false;  // (coupled) M, N and the residual of the current iterate are formed
  int state_level = 0;       // precision level at which M was last formed
  std::vector<double> hist;  // r_0 .. r_k
  std::vector<int> hist_prec;
  pr_stats_t st{};
  std::string err;

  int* err_word() { return reinterpret_cast<int*>(scal + 7); }
};

namespace {

pr_status fail(pr_handle h, pr_status code, const std::string& msg) {
  if (h) {
    h->err = msg;
    h->st.last_stop = code;
  } else {
    g_init_error = msg;
  }
  return code;
}

pr_status cuda_fail(pr_handle h, const char* what, cudaError_t e) {
  std::string msg = std::string(what) + ": " + cudaGetErrorName(e) + " (" + cudaGetErrorString(e) + ")";
  return fail(h, e == cudaErrorMemoryAllocation ? PR_ENOMEM : PR_ECUDA, msg);
}

#define PR_CK(h, call)                                      \
  do {                                                       \
    cudaError_t _e = (call);                                 \
    if (_e != cudaSuccess) return cuda_fail((h), #call, _e); \
  } while (0)

double sym_flops(int64_t n) { return (double)n * (double)(n + 1) * (double)n; }
double full_flops(int64_t n) { return 2.0 * (double)n * (double)n * (double)n; }

constexpr int kEventPairs = 64;

pr_status harvest_events(pr_handle h) {
  for (int i = 0; i < h->ev_pending; ++i) {
    float ms = 0.f;
    PR_CK(h, cudaEventElapsedTime(&ms, h->ev[2 * i], h->ev[2 * i + 1]));
    h->st.gemm_ms += ms;
    h->st.gemms_timed += 1;
    h->st.gemm_flops_timed += h->ev_flops[i];
    const int pq = h->ev_prec[i];
    h->st.gemm_ms_by_precision[pq] += ms;
    h->st.gemms_timed_by_precision[pq] += 1;
    h->st.gemm_flops_by_precision[pq] += h->ev_flops[i];
  }
  h->ev_pending = 0;
  return PR_OK;
}

// Synchronises the stream, collects event timings and checks the device error word.
pr_status sync(pr_handle h) {
  PR_CK(h, cudaStreamSynchronize(h->stream));
  pr_status s = harvest_events(h);
  if (s != PR_OK) return s;
  int word = 0;
  PR_CK(h, cudaMemcpy(&word, h->err_word(), sizeof(int), cudaMemcpyDeviceToHost));
  if (word != 0) {
    char buf[128];
    snprintf(buf, sizeof buf, "a bounded device wait expired (code %d); the product was abandoned", word);
    PR_CK(h, cudaMemset(h->err_word(), 0, sizeof(int)));
    return fail(h, PR_ETIMEOUT, buf);
  }
  return PR_OK;
}

// The work-list variants of the digit-slice products: tile width (output columns per tile) and whether every
// tile is split over K into two halves run by neighbouring CTAs. All give bit-identical products, and the
// same residual partials for one tile width.
struct EmuVariant {
  int bn, split;
};
constexpr EmuVariant kEmuVariants[4] = {{96, 0}, {96, 1}, {48, 0}, {48, 1}};

// Process-wide record of the variant the tuner chose per (order, mode, digit planes), so that later handles of
// the same order (and repeated pr_load) do not tune again.
std::mutex g_tune_mu;
std::map<std::tuple<int, int, int>, int>& tune_cache() {
  static std::map<std::tuple<int, int, int>, int> cache;
  return cache;
}

// The rungs below FP64 accuracy: their own stagnation threshold (stag_below_lowp), a stop at the first
// residual that does not fall, and the roll-back of that last step.
bool lowp(int prec) { return prec == PR_BF16 || prec == PR_FP8 || prec == PR_FP32X; }

// Digit planes of m for PR_EMU64 products (allocated on first use, recomputed when m changed).
// The E4M3 copy of m for PR_FP8 products (allocated on first use, recomputed when m changed).
pr_status ensure_fp8(pr_handle h, Mat& m) {
  const int n = (int)h->n;
  if (!m.q) {
    PR_CK(h, cudaMalloc((void**)&m.q, (size_t)n * (size_t)h->ldq));
    PR_CK(h, cudaMalloc((void**)&m.qe, (size_t)n * sizeof(int)));
    m.q_valid = false;
  }
  if (m.q_valid) return PR_OK;
  PR_CK(h, pr::to_fp8(m.f, n, h->ldq, m.q, m.qe, h->stream));
  h->st.launches += 1;
  m.q_valid = true;
  return PR_OK;
}

pr_status ensure_slices(pr_handle h, Mat& m) {
  const int n = (int)h->n;
  if (!m.sl) {
    PR_CK(h, cudaMalloc((void**)&m.sl, (size_t)8 * (size_t)n * (size_t)h->eld * sizeof(__half)));
    PR_CK(h, cudaMalloc((void**)&m.ex, (size_t)n * sizeof(int)));
    m.sl_valid = false;
  }
  if (m.sl_valid) return PR_OK;
  PR_CK(h, pr::slice(m.f, n, h->eld, h->S, m.sl, m.ex, h->stream));
  h->st.launches += 1;
  m.sl_valid = true;
  return PR_OK;
}

// The work-list variant of the digit-slice products of mode m (0 symmetric, 1 full) at precision class pc
// (0 PR_EMU64, 1 PR_FP32X): fixed by pr_options.emu_tile (96 or 48, tiles split by the wave rule), taken from
// the process-wide record, or tuned: every applicable variant runs the product about to be computed twice
// (its results are exact integer totals rounded once, the same for every variant; the last run, with the
// chosen variant, writes the residual partials), timed with CUDA events, and the fastest is kept.
template <class Launch>
pr_status choose_emu_variant(pr_handle h, int m, int pc, int S, Launch&& launch) {
  const int n = (int)h->n;
  const Mode mode = m == 0 ? Mode::Sym : Mode::Full;
  if (h->opt.emu_tile != 0) {
    const int base = h->opt.emu_tile == 96 ? 0 : 2;
    h->emu_plan[m][pc] = base + (pr::emu_split_slots(n, mode, kEmuVariants[base].bn, -1) > 0 ? 1 : 0);
  } else {
    const auto key = std::make_tuple(n, m, S);
    {
      std::lock_guard<std::mutex> lock(g_tune_mu);
      auto it = tune_cache().find(key);
      if (it != tune_cache().end()) h->emu_plan[m][pc] = it->second;
    }
    if (h->emu_plan[m][pc] < 0) {
      cudaEvent_t e0, e1;
      PR_CK(h, cudaEventCreate(&e0));
      PR_CK(h, cudaEventCreate(&e1));
      float best = 1e30f;
      int pick = 0;
      for (int v = 0; v < 4; ++v) {
        if (!h->emu_items[m][v]) continue;
        float t = 1e30f;
        for (int rep = 0; rep < 2; ++rep) {
          PR_CK(h, cudaEventRecord(e0, h->stream));
          PR_CK(h, launch(v));
          PR_CK(h, cudaEventRecord(e1, h->stream));
          PR_CK(h, cudaEventSynchronize(e1));
          float ms = 0.f;
          PR_CK(h, cudaEventElapsedTime(&ms, e0, e1));
          t = std::min(t, ms);
          h->st.launches += 1;
        }
        h->st.emu_tune_ms += t * 2;
        if (pc == 0) h->st.emu_variant_ms[m][v] = t;
        if (t < best) {
          best = t;
          pick = v;
        }
      }
      cudaEventDestroy(e0);
      cudaEventDestroy(e1);
      pr_status s = sync(h);  // a bounded wait that expired during a trial shows here
      if (s != PR_OK) return s;
      h->emu_plan[m][pc] = pick;
      std::lock_guard<std::mutex> lock(g_tune_mu);
      tune_cache()[key] = pick;
    }
  }
  if (pc == 0) {
    h->st.emu_tile_n[m] = kEmuVariants[h->emu_plan[m][pc]].bn;
    h->st.emu_tile_split[m] = kEmuVariants[h->emu_plan[m][pc]].split;
  }
  return PR_OK;
}

// One matrix product P = X Y (X, Y symmetric, or Y given transposed in its BF16 copy) at the requested
// precision, with the fused epilogue described by o.
pr_status product(pr_handle h, int prec, Mat& X, Mat& Y, Mode mode, const Out& o) {
  const bool sym = mode == Mode::Sym;
  const pr::NvtxRange trace(prec == PR_EMU64    ? (sym ? "product EMU64 sym" : "product EMU64 full")
                            : prec == PR_FP32X ? (sym ? "product FP32X sym" : "product FP32X full")
                            : prec == PR_BF16  ? (sym ? "product BF16 sym" : "product BF16 full")
                            : prec == PR_FP8   ? (sym ? "product FP8 sym" : "product FP8 full")
                                               : (sym ? "product FP64 sym" : "product FP64 full"));
  const int n = (int)h->n;
  const double flops = mode == Mode::Sym ? sym_flops(n) : full_flops(n);
  Epilogue e;
  e.cin = o.cin;
  e.a = o.a;
  e.b = o.b;
  e.c = o.c;
  e.partial = o.partial ? h->partial : nullptr;
  if (prec == PR_EMU64 || prec == PR_FP32X) {
    pr_status s = ensure_slices(h, X);
    if (s == PR_OK) s = ensure_slices(h, Y);
    if (s != PR_OK) return s;
    if (o.out) e.out = o.out->f;
    if (o.out2) e.out2 = o.out2->f;
  } else if (prec == PR_FP8) {
    pr_status s = ensure_fp8(h, X);
    if (s == PR_OK) s = ensure_fp8(h, Y);
    if (s != PR_OK) return s;
    if (o.out) e.out = o.out->f;  // FP8 results keep their FP64 copies: the next product re-quantises them
    if (o.out2) e.out2 = o.out2->f;
  } else if (prec == PR_BF16) {
    if (o.out) {
      if (o.lp_copy) e.out_lp = o.out->b;
      if (o.out_master || !o.lp_copy) e.out = o.out->f;
    }
    if (o.out2) {
      if (o.lp_copy) e.out2_lp = o.out2->b;
      if (o.out2_master || !o.lp_copy) e.out2 = o.out2->f;
    }
  } else {
    if (o.out) e.out = o.out->f;
    if (o.out2) e.out2 = o.out2->f;
  }
  for (const Mat* t : {o.out, o.out2})
    if (t == &h->T0 || t == &h->T1) h->powers_valid = false;  // the scratch products are overwritten
  h->st.gemms += 1;
  h->st.gemm_flops += flops;
  if (h->timing) {
    if (h->ev_pending == kEventPairs) {
      pr_status s = sync(h);
      if (s != PR_OK) return s;
    }
    PR_CK(h, cudaEventRecord(h->ev[2 * h->ev_pending], h->stream));
  }
  switch (prec) {
    case PR_FP64:
      PR_CK(h, pr::gemm_f64(X.f, Y.f, n, mode, e, h->stream));
      h->lp_stale = true;
      break;
    case PR_BF16:
      PR_CK(h, pr::gemm_bf16_tc(X.b, Y.b, n, h->ldl, mode, o.transpose, e, h->err_word(), h->stream));
      break;
    case PR_EMU64:
    case PR_FP32X: {
      const int m = mode == Mode::Sym ? 0 : 1, pc = prec == PR_FP32X ? 1 : 0;
      const int S = prec == PR_FP32X ? std::min(h->S, kFp32xSlices) : h->S;
      auto launch = [&](int v) {
        return pr::gemm_emu(X.sl, X.ex, Y.sl, Y.ex, n, h->eld, S, mode, o.transpose, h->emu_items[m][v],
                            h->emu_nitems[m][v], e, h->emu_scratch, h->emu_nsplit[m][v] ? h->emu_split : nullptr,
                            h->emu_split_cnt, h->err_word(), h->stream, kEmuVariants[v].bn);
      };
      if (h->emu_plan[m][pc] < 0) {
        pr_status ps = choose_emu_variant(h, m, pc, S, launch);
        if (ps != PR_OK) return ps;
      }
      const bool xa = &X == &h->A, ya = &Y == &h->A;
      if (h->sp_on && (xa || ya)) {
        // Block-sparse A: the unsplit list of the chosen width, each tile restricted to the K steps where the
        // rows of A it reads are non-zero (the other steps add exact zeros).
        const int wi = kEmuVariants[h->emu_plan[m][pc]].bn == 96 ? 0 : 1, side = xa && ya ? 2 : (xa ? 0 : 1);
        PR_CK(h, pr::gemm_emu(X.sl, X.ex, Y.sl, Y.ex, n, h->eld, S, mode, o.transpose, h->sp_items[m][wi][side],
                              h->emu_nitems[m][2 * wi], e, h->emu_scratch, nullptr, h->emu_split_cnt, h->err_word(),
                              h->stream, kEmuVariants[2 * wi].bn));
        h->st.sparse_products += 1;
      } else {
        PR_CK(h, launch(h->emu_plan[m][pc]));
      }
      h->lp_stale = true;
      break;
    }
    case PR_FP8:
      PR_CK(h, pr::gemm_fp8_tc(X.q, X.qe, Y.q, Y.qe, n, h->ldq, mode, o.transpose, e, h->err_word(), h->stream));
      h->lp_stale = true;
      break;
    default:
      return fail(h, PR_EUNSUPPORTED, "precision not available in this build");
  }
  h->st.launches += 1;
  if (o.out) o.out->changed();
  if (o.out2) o.out2->changed();
  if (h->timing) {
    PR_CK(h, cudaEventRecord(h->ev[2 * h->ev_pending + 1], h->stream));
    h->ev_flops[h->ev_pending] = flops;
    h->ev_prec[h->ev_pending] = prec;
    h->ev_pending += 1;
  }
  return PR_OK;
}

int tiles_for(pr_handle h, int prec, Mode mode) {
  if (prec == PR_EMU64 || prec == PR_FP32X) {
    const int v = h->emu_plan[mode == Mode::Sym ? 0 : 1][prec == PR_FP32X ? 1 : 0];
    return pr::emu_tiles((int)h->n, mode, kEmuVariants[v < 0 ? 0 : v].bn);
  }
  return lowp(prec) ? pr::gemm_tc_tiles((int)h->n, mode) : pr::gemm_f64_tiles((int)h->n, mode);
}

// Brings the BF16 copies of the state up to date before low-precision products.
pr_status refresh_lowp(pr_handle h) {
  if (!h->lp_stale) return PR_OK;
  const int n = (int)h->n;
  for (Mat* m : {&h->A, &h->X, &h->M, &h->N}) {
    PR_CK(h, pr::to_bf16(m->f, n, h->ldl, m->b, h->stream));
    h->st.launches += 1;
  }
  h->lp_stale = false;
  return PR_OK;
}

// Sum of the partials of the last product -> sqrt -> host.
pr_status read_residual(pr_handle h, int count, double* r) {
  PR_CK(h, pr::reduce_partials_sqrt(h->partial, count, h->scal + 6, h->stream));
  h->st.launches += 1;
  PR_CK(h, cudaMemcpyAsync(h->hpin + 6, h->scal + 6, sizeof(double), cudaMemcpyDeviceToHost, h->stream));
  pr_status s = sync(h);
  if (s != PR_OK) return s;
  *r = h->hpin[6];
  return PR_OK;
}

void push_residual(pr_handle h, double r, int prec, bool replace_last) {
  if (replace_last && !h->hist.empty()) {
    h->hist.back() = r;
    h->hist_prec.back() = prec;
  } else {
    h->hist.push_back(r);
    h->hist_prec.push_back(prec);
  }
  h->st.last_residual = r;
}

// Coupled form: M = X^p A by p symmetric products (X is a polynomial in A), the last epilogue writing
// N = ((p+1) I - M)/p and the partials of ||I - M||_F.
pr_status form_M_from_X(pr_handle h, int prec, bool replace_last) {
  const int p = h->p;
  Mat* src = &h->A;
  for (int j = 1; j <= p; ++j) {
    Out o;
    if (j < p) {
      o.out = (j & 1) ? &h->T0 : &h->T1;
      o.out_master = false;
    } else {
      o.out = &h->M;
      o.out2 = &h->N;
      o.a = (double)(p + 1) / p;
      o.b = -1.0 / p;
      o.partial = true;
    }
    pr_status s = product(h, prec, h->X, *src, Mode::Sym, o);
    if (s != PR_OK) return s;
    src = o.out;
  }
  double r;
  pr_status s = read_residual(h, tiles_for(h, prec, Mode::Sym), &r);
  if (s != PR_OK) return s;
  push_residual(h, r, prec, replace_last);
  h->state_level = precision_level(prec);
  return PR_OK;
}

// X_{k+1} = X_k N_k; M_{k+1} = N_k^p M_k (p symmetric products, 3 for p = 4); N_{k+1} and r_{k+1} fused.
pr_status coupled_update(pr_handle h, int prec) {
  const int p = h->p;
  Out ox;
  ox.out = &h->Xn;
  pr_status s = product(h, prec, h->X, h->N, Mode::Sym, ox);
  if (s != PR_OK) return s;
  Out last;
  last.out = &h->Mn;
  last.out2 = &h->Nn;
  last.a = (double)(p + 1) / p;
  last.b = -1.0 / p;
  last.partial = true;
  // At low precision the FP64 copies of M and N are only needed if a later switch to higher precision
  // carries them over instead of re-forming M from X.
  last.out_master = last.out2_master = !(prec == PR_BF16 && h->opt.reanchor);
  if (p == 3 && prec != PR_BF16) {
    // N^3 M = M (4I - M)^3 / 27 = L R with L = 4M - M^2 and R = (16I - 8M + M^2) / 27: two products
    // instead of three (every factor is a polynomial in M, hence in A). The first product gives M^2 and, in
    // its epilogue, R; L follows element by element. (Low precision keeps the plain chain: its FP64 copy of
    // M, which L needs, is not kept.)
    Out o;
    o.out = &h->T0;
    o.out2 = &h->T1;
    o.cin = h->M.f;
    o.a = 16.0 / 27.0;
    o.b = 1.0 / 27.0;
    o.c = -8.0 / 27.0;
    s = product(h, prec, h->M, h->M, Mode::Sym, o);
    if (s != PR_OK) return s;
    PR_CK(h, pr::lincomb(h->M.f, h->T0.f, h->n * h->n, 4.0, -1.0, h->T0.f, h->stream));
    h->st.launches += 1;
    h->T0.changed();
    s = product(h, prec, h->T0, h->T1, Mode::Sym, last);
    if (s != PR_OK) return s;
  } else if (p == 4) {
    // N^4 M = (N^2)^2 M: three products instead of four (every factor is a polynomial in A).
    Out o;
    o.out = &h->T0;
    o.out_master = false;
    s = product(h, prec, h->N, h->N, Mode::Sym, o);
    if (s != PR_OK) return s;
    o.out = &h->T1;
    s = product(h, prec, h->T0, h->T0, Mode::Sym, o);
    if (s == PR_OK) s = product(h, prec, h->T1, h->M, Mode::Sym, last);
    if (s != PR_OK) return s;
  } else {
    Mat* src = &h->M;
    for (int j = 1; j <= p; ++j) {
      Out o;
      if (j < p) {
        o.out = (j & 1) ? &h->T0 : &h->T1;
        o.out_master = false;
      } else {
        o = last;
      }
      s = product(h, prec, h->N, *src, Mode::Sym, o);
      if (s != PR_OK) return s;
      src = o.out;
    }
  }
  double r;
  s = read_residual(h, tiles_for(h, prec, Mode::Sym), &r);
  if (s != PR_OK) return s;
  swap(h->X, h->Xn);
  swap(h->M, h->Mn);
  swap(h->N, h->Nn);
  push_residual(h, r, prec, false);
  return PR_OK;
}

// Newton-Schulz (p = 1): T = A X (full product; its BF16 copy is stored transposed so that it can be
// the K-major B operand of X T), residual ||I - T||_F of the current X.
pr_status ns_residual(pr_handle h, int prec, double* r) {
  Out o;
  o.out = &h->T0;
  o.out_master = false;
  o.partial = true;
  o.transpose = true;
  pr_status s = product(h, prec, h->A, h->X, Mode::Full, o);
  if (s != PR_OK) return s;
  return read_residual(h, tiles_for(h, prec, Mode::Full), r);
}

// X' = 2X - X T with T = A X from ns_residual; X T = X A X is symmetric for every symmetric X.
pr_status ns_update(pr_handle h, int prec) {
  Out o;
  o.out2 = &h->Xn;
  o.b = -1.0;
  o.c = 2.0;
  o.cin = h->X.f;
  pr_status s = product(h, prec, h->X, h->T0, Mode::Sym, o);
  if (s != PR_OK) return s;
  swap(h->X, h->Xn);
  return PR_OK;
}

// Literal Eq. 1 (FP64 only): T_j = C T_{j-1}, T_0 = A (full products); the residual from T_p = C^p A.
// The custom-precision experiment (pr_options.quant_bits with quant_mode PR_QUANT_ARITH): every operation
// of the literal iteration in m-bit arithmetic (k_quant.cu).
bool quant_arith(pr_handle h) { return h->opt.quant_bits > 0 && h->opt.quant_mode == PR_QUANT_ARITH; }

pr_status literal_residual(pr_handle h, int prec, double* r) {
  if (quant_arith(h)) {
    // T_j = C T_{j-1} in the m-bit arithmetic; the residual ||I - T_p||_F (the stop test) in FP64.
    const int n = (int)h->n, m = h->opt.quant_bits;
    Mat* src = &h->A;
    for (int j = 1; j <= h->p; ++j) {
      Mat* dst = (j & 1) ? &h->T0 : &h->T1;
      PR_CK(h, pr::gemm_round(h->X.f, src->f, n, m, dst->f, h->stream));
      dst->changed();
      h->powers_valid = false;
      h->st.gemms += 1;
      h->st.gemm_flops += full_flops(n);
      src = dst;
    }
    PR_CK(h, pr::resid_rows(src->f, n, h->partial, h->stream));
    h->st.launches += h->p + 1;
    return read_residual(h, pr::resid_row_partials(n), r);
  }
  Mat* src = &h->A;
  for (int j = 1; j <= h->p; ++j) {
    Out o;
    o.out = (j & 1) ? &h->T0 : &h->T1;
    o.partial = j == h->p;
    pr_status s = product(h, prec, h->X, *src, Mode::Full, o);
    if (s != PR_OK) return s;
    src = o.out;
  }
  return read_residual(h, tiles_for(h, prec, Mode::Full), r);
}

// C' = sym(((p+1) C - C T_p) / p); with pr_options.quant_bits the stored iterate is rounded (storage) or
// every operation is (arithmetic).
pr_status literal_update(pr_handle h, int prec) {
  Mat& Tp = (h->p & 1) ? h->T0 : h->T1;
  const int n = (int)h->n, m = h->opt.quant_bits;
  if (quant_arith(h)) {
    PR_CK(h, pr::gemm_round(h->X.f, Tp.f, n, m, h->Mn.f, h->stream));
    PR_CK(h, pr::quant_update(h->X.f, h->Mn.f, n, h->p, m, h->Mn.f, h->stream));
    PR_CK(h, pr::quant_sym(h->Mn.f, n, m, h->Xn.f, h->stream));
    h->st.gemms += 1;
    h->st.gemm_flops += full_flops(n);
    h->st.launches += 3;
    h->Xn.changed();
    h->Mn.changed();
    swap(h->X, h->Xn);
    return PR_OK;
  }
  Out o;
  o.out2 = &h->Mn;
  o.b = -1.0 / h->p;
  o.c = (double)(h->p + 1) / h->p;
  o.cin = h->X.f;
  pr_status s = product(h, prec, h->X, Tp, Mode::Full, o);
  if (s != PR_OK) return s;
  PR_CK(h, pr::symmetrize(h->Mn.f, (int)h->n, h->Xn.f, h->stream));
  h->st.launches += 1;
  if (m > 0) {  // storage: the new iterate is stored with m mantissa bits
    PR_CK(h, pr::round_values(h->Xn.f, (int64_t)n * n, m, h->Xn.f, h->stream));
    h->st.launches += 1;
  }
  h->Xn.changed();
  swap(h->X, h->Xn);
  return PR_OK;
}

// True residual ||I - C^p A||_F of the current iterate: C^p by symmetric products (powers of a symmetric
// matrix are symmetric), then the full product with A, with products at the given precision.
pr_status true_residual(pr_handle h, int precision, double* res_fro) {
  if (precision == PR_BF16) {
    pr_status s = refresh_lowp(h);
    if (s != PR_OK) return s;
  }
  Mat* P = &h->X;
  for (int j = 2; j <= h->p; ++j) {
    Out o;
    o.out = (j & 1) ? &h->T1 : &h->T0;
    o.out_master = false;
    pr_status s = product(h, precision, h->X, *P, Mode::Sym, o);
    if (s != PR_OK) return s;
    P = o.out;
  }
  Out o;
  o.partial = true;
  pr_status s = product(h, precision, *P, h->A, Mode::Full, o);
  if (s != PR_OK) return s;
  return read_residual(h, tiles_for(h, precision, Mode::Full), res_fro);
}

}  // namespace

// The stop rule (see pr_stop_rule): returns a pr_status to stop with, or -1 to apply one more update.
int pr::stop_rule(const double* hist, const int* prec, int len, double tol, const pr_options& o) {
  const bool prev = len >= 2 && prec[len - 2] == prec[len - 1];
  return stop_rule_last(hist[len - 1], prev, prev ? hist[len - 2] : 0.0, lowp(prec[len - 1]), tol, o);
}

namespace {
using pr::stop_rule;

int decide(pr_handle h, double tol, int steps_this_call, int max_steps) {
  const int stop = stop_rule(h->hist.data(), h->hist_prec.data(), (int)h->hist.size(), tol, h->opt);
  if (stop >= 0) return stop;
  if (h->st.iterations >= h->opt.max_iter || steps_this_call >= max_steps) return PR_EMAXITER;
  return -1;
}

bool precision_known(int prec) { return prec >= PR_FP64 && prec <= PR_FP8; }

pr_status check_precision(pr_handle h, int prec) {
  if (!precision_known(prec)) return fail(h, PR_EINVAL, "unknown precision");
  if (h->form == PR_FORM_LITERAL && prec != PR_FP64)
    return fail(h, PR_EUNSUPPORTED, "the literal form runs in PR_FP64 only");
  return PR_OK;
}

pr_status ensure_state(pr_handle h, int prec) {
  if (prec == PR_BF16) {
    pr_status s = refresh_lowp(h);
    if (s != PR_OK) return s;
  }
  if (h->form != PR_FORM_COUPLED) return PR_OK;
  if (!h->state_ready) {
    pr_status s = form_M_from_X(h, prec, false);
    if (s != PR_OK) return s;
    h->state_ready = true;
  } else if (h->opt.reanchor && precision_level(prec) > h->state_level) {
    pr_status s = form_M_from_X(h, prec, true);
    if (s != PR_OK) return s;
  }
  return PR_OK;
}

}  // namespace

namespace {

constexpr int kVecBlocks = 152 * 8;  // upper bound on the reduction blocks of k_learned.cu

pr_status ensure_vec(pr_handle h) {
  if (!h->vec) PR_CK(h, cudaMalloc((void**)&h->vec, sizeof(double) * (4 * (size_t)h->n + kVecBlocks + 16)));
  return PR_OK;
}

// T0 = A A, T1 = A (A A) with FP64-accurate (PR_EMU64) symmetric products; kept until an iteration, a
// residual or a new A overwrites the scratch products.
pr_status powers_of_A(pr_handle h) {
  if (h->powers_valid) return PR_OK;
  Out o2;
  o2.out = &h->T0;
  pr_status s = product(h, PR_EMU64, h->A, h->A, Mode::Sym, o2);
  if (s != PR_OK) return s;
  Out o3;
  o3.out = &h->T1;
  s = product(h, PR_EMU64, h->A, h->T0, Mode::Sym, o3);
  h->powers_valid = s == PR_OK;
  return s;
}

// Power iteration for ||M||_2 of a symmetric n x n M (from below), `iters` steps.
pr_status power_norm(pr_handle h, const double* M, int iters, double* out) {
  const int n = (int)h->n;
  double *v = h->vec, *u = v + n, *zero = u + n, *w = zero + n, *work = w + n, *sc2 = work + kVecBlocks;
  PR_CK(h, cudaMemsetAsync(zero, 0, sizeof(double) * n, h->stream));
  PR_CK(h, pr::power_start(n, v, h->stream));
  for (int it = 0; it < iters; ++it) {
    PR_CK(h, pr::gemv(M, n, v, u, h->stream));
    PR_CK(h, pr::power_finish_step(zero, u, n, w, work, sc2, v, sc2 + 1, h->stream));  // v = -M v / |M v|
    h->st.launches += 4;
  }
  PR_CK(h, cudaMemcpyAsync(h->hpin + 6, sc2 + 1, sizeof(double), cudaMemcpyDeviceToHost, h->stream));
  pr_status st = sync(h);
  if (st == PR_OK) *out = h->hpin[6];
  return st;
}

// Power iteration for ||A||_2 (from below): the spectrum of A / ||A||_1 lies in (0, ||A||_2 / ||A||_1].
pr_status spectral_radius(pr_handle h, double* out) {
  const int n = (int)h->n;
  double *v = h->vec, *u = v + n, *zero = u + n, *w = zero + n, *work = w + n, *sc2 = work + kVecBlocks;
  PR_CK(h, cudaMemsetAsync(zero, 0, sizeof(double) * n, h->stream));
  PR_CK(h, pr::power_start(n, v, h->stream));
  for (int it = 0; it < h->opt.gate_iters; ++it) {
    PR_CK(h, pr::gemv(h->A.f, n, v, u, h->stream));
    PR_CK(h, pr::power_finish_step(zero, u, n, w, work, sc2, v, sc2 + 1, h->stream));  // v = -A v / |A v|
    h->st.launches += 4;
  }
  PR_CK(h, cudaMemcpyAsync(h->hpin + 6, sc2 + 1, sizeof(double), cudaMemcpyDeviceToHost, h->stream));
  pr_status st = sync(h);
  if (st == PR_OK) *out = h->hpin[6];
  return st;
}

// C_0 = ||A||_1^{-1/p} q(A / ||A||_1) with the gate of Eq. 2; falls back to Eq. 3. Sets st.c0, st.c0_gate.
pr_status poly_initial_guess(pr_handle h) {
  const int n = (int)h->n, p = h->p;
  const double* c = h->opt.c0_coef;
  const double s1 = h->st.norm_1;
  pr_status s = ensure_vec(h);
  if (s != PR_OK) return s;
  double rho = 0.0;
  s = spectral_radius(h, &rho);
  if (s != PR_OK) return s;
  // q > 0 on [0, 1.05 ||A||_2 / ||A||_1] (a 5 % margin over the estimate from below) keeps C_0 positive
  // definite; for even p the gate alone would not see a negative q.
  const double top = fmin(1.0, 1.05 * rho / s1);
  bool ok = true;
  for (int k = 0; k <= 1000 && ok; ++k) {
    const double x = top * k / 1000.0;
    ok = ((c[3] * x + c[2]) * x + c[1]) * x + c[0] > 0.0;
  }
  double gate = INFINITY;
  if (ok) {
    s = powers_of_A(h);
    if (s != PR_OK) return s;
    const double sc = pow(s1, -1.0 / p);
    const double a[4] = {sc * c[0], sc * c[1] / s1, sc * c[2] / (s1 * s1), sc * c[3] / (s1 * s1 * s1)};
    PR_CK(h, pr::poly_combine(h->A.f, h->T0.f, h->T1.f, n, a, h->X.f, h->stream));
    // Power iteration for ||B||_2, B = I - C_0^p A (symmetric: C_0 is a polynomial in A).
    double *v = h->vec, *u = v + n, *u2 = u + n, *w = u2 + n, *work = w + n, *sc2 = work + kVecBlocks;
    PR_CK(h, pr::power_start(n, v, h->stream));
    for (int it = 0; it < h->opt.gate_iters; ++it) {
      PR_CK(h, pr::gemv(h->A.f, n, v, u, h->stream));
      double *src = u, *dst = u2;
      for (int j = 0; j < p; ++j) {
        PR_CK(h, pr::gemv(h->X.f, n, src, dst, h->stream));
        std::swap(src, dst);
      }
      PR_CK(h, pr::power_finish_step(v, src, n, w, work, sc2, v, sc2 + 1, h->stream));
      h->st.launches += p + 4;
    }
    PR_CK(h, cudaMemcpyAsync(h->hpin + 6, sc2 + 1, sizeof(double), cudaMemcpyDeviceToHost, h->stream));
    pr_status st = sync(h);
    if (st != PR_OK) return st;
    gate = h->hpin[6];
    ok = gate < h->opt.gate_max;
  }
  h->st.c0_gate = gate;
  h->st.c0 = ok ? PR_C0_POLY : PR_C0_EQ3;
  if (!ok) PR_CK(h, pr::init_c0_eq3(h->A.f, n, 1.0 / (h->st.norm_1 * h->st.norm_inf), h->X.f, h->stream));
  h->X.changed();
  if (!ok && !h->opt.gate_fallback) {
    char buf[200];
    snprintf(buf, sizeof buf,
             "the polynomial initial guess failed its gate (estimate of ||I - C_0^p A||_2 = %.3g, limit %.3g, or q not "
             "positive on the spectrum); the handle holds Eq. 3's C_0",
             gate, h->opt.gate_max);
    return fail(h, PR_EGATE, buf);
  }
  return PR_OK;
}

// Back to "C_0 formed, no iteration yet" (the loaded A and its norms stay).
void reset_iteration(pr_handle h) {
  h->state_ready = false;
  h->state_level = 0;
  h->lp_stale = true;
  for (Mat* m : {&h->X, &h->Xn, &h->M, &h->Mn, &h->N, &h->Nn, &h->T0, &h->T1}) m->changed();
  h->hist.clear();
  h->hist_prec.clear();
  h->st.iterations = 0;
  for (int& c : h->st.iterations_by_precision) c = 0;
  h->st.switch_iteration = -1;
  h->st.last_precision = -1;
  h->st.last_residual = 0.0;
  h->st.true_residual = -1.0;
  h->st.ladder_restores = 0;
}

// C_0 of the loaded A (Eq. 3, the scaled identity, or the gated polynomial) into X.
pr_status form_initial_guess(pr_handle h) {
  const int n = (int)h->n;
  h->st.c0 = h->opt.c0;
  h->st.c0_gate = 0.0;
  if (h->opt.c0 == PR_C0_EQ3) {
    PR_CK(h, pr::init_c0_eq3(h->A.f, n, 1.0 / (h->st.norm_1 * h->st.norm_inf), h->X.f, h->stream));
  } else if (h->opt.c0 == PR_C0_SCALED_I) {
    PR_CK(h, pr::set_scaled_identity(h->X.f, n, pow(h->st.norm_1, -1.0 / h->p), h->stream));
  } else if (h->opt.c0 == PR_C0_POLY) {
    pr_status st = poly_initial_guess(h);
    if (st == PR_EGATE) {
      const pr_status s2 = sync(h);
      return s2 == PR_OK ? PR_EGATE : s2;
    }
    if (st != PR_OK) return st;
  }
  if (h->opt.quant_bits > 0)  // C_0, computed in FP64, is stored with m mantissa bits
    PR_CK(h, pr::round_values(h->X.f, (int64_t)n * n, h->opt.quant_bits, h->X.f, h->stream));
  h->X.changed();
  h->st.launches += 1;
  return sync(h);
}

}  // namespace

namespace pr {
void set_handleless_error(const char* msg) { g_init_error = msg; }
}  // namespace pr

namespace {

pr_status matmul(int precision, int S, const double* X, const double* Y, int64_t n, int sym, double* P,
                 void* stream, int bn = 96, int split_mode = -1) {
  if (!X || !Y || !P) return fail(nullptr, PR_EINVAL, "pr_matmul: NULL matrix");
  if (n < 1 || n > (int64_t)1 << 17) return fail(nullptr, PR_EINVAL, "pr_matmul: n must be in [1, 131072]");
  if (!precision_known(precision)) return fail(nullptr, PR_EINVAL, "pr_matmul: unknown precision");
  const bool emu = precision == PR_EMU64 || precision == PR_FP32X;
  cudaStream_t s = (cudaStream_t)stream;
  const int ni = (int)n, ldl = pr::bf16_ld(ni);
  const size_t bytes = (size_t)n * (size_t)n * sizeof(double);
  const int eld = pr::emu_ld(ni), ldq = pr::fp8_ld(ni);
  const size_t lbytes = emu                     ? (size_t)8 * (size_t)n * (size_t)eld * sizeof(__half)
                        : precision == PR_FP8 ? (size_t)n * (size_t)ldq
                                              : (size_t)n * (size_t)ldl * sizeof(__nv_bfloat16);
  const Mode mode = sym ? Mode::Sym : Mode::Full;
  double *dX = nullptr, *dY = nullptr, *dP = nullptr;
  __nv_bfloat16 *bX = nullptr, *bY = nullptr;
  int *err = nullptr, *eX = nullptr, *eY = nullptr;
  int4* items = nullptr;
  long long* scratch = nullptr;
  long long* split = nullptr;
  int* split_cnt = nullptr;
  std::vector<int4> hitems;
  cudaError_t e = cudaSuccess;
  int word = 0;
  auto step = [&](cudaError_t r) {
    if (e == cudaSuccess) e = r;
  };
  step(cudaMalloc((void**)&dX, bytes));
  step(cudaMalloc((void**)&dY, bytes));
  step(cudaMalloc((void**)&dP, bytes));
  step(cudaMalloc((void**)&err, sizeof(int)));
  if (precision != PR_FP64) {
    step(cudaMalloc((void**)&bX, lbytes));
    step(cudaMalloc((void**)&bY, lbytes));
    step(cudaMalloc((void**)&eX, (size_t)n * sizeof(int)));
    step(cudaMalloc((void**)&eY, (size_t)n * sizeof(int)));
  }
  if (e == cudaSuccess) {
    step(cudaMemsetAsync(err, 0, sizeof(int), s));
    step(cudaMemcpyAsync(dX, X, bytes, cudaMemcpyDefault, s));
    step(cudaMemcpyAsync(dY, Y, bytes, cudaMemcpyDefault, s));
    Epilogue ep;
    ep.out = dP;
    if (precision == PR_FP64) {
      step(pr::gemm_f64(dX, dY, ni, mode, ep, s));
    } else if (precision == PR_BF16) {
      step(pr::to_bf16(dX, ni, ldl, bX, s));
      step(pr::to_bf16(dY, ni, ldl, bY, s));
      step(pr::gemm_bf16_tc(bX, bY, ni, ldl, mode, false, ep, err, s));
    } else if (precision == PR_FP8) {
      uint8_t *qX = reinterpret_cast<uint8_t*>(bX), *qY = reinterpret_cast<uint8_t*>(bY);
      step(pr::to_fp8(dX, ni, ldq, qX, eX, s));
      step(pr::to_fp8(dY, ni, ldq, qY, eY, s));
      step(pr::gemm_fp8_tc(qX, eX, qY, eY, ni, ldq, mode, false, ep, err, s));
    } else {
      __half *hX = reinterpret_cast<__half*>(bX), *hY = reinterpret_cast<__half*>(bY);
      pr::emu_launch_list(ni, mode, hitems, bn, split_mode);
      const int slots = pr::emu_split_slots(ni, mode, bn, split_mode);
      step(cudaMalloc((void**)&items, hitems.size() * sizeof(int4)));
      step(cudaMalloc((void**)&scratch, pr::emu_scratch_bytes()));
      if (slots > 0) {
        step(cudaMalloc((void**)&split, pr::emu_split_bytes(slots)));
        step(cudaMalloc((void**)&split_cnt, pr::emu_split_counters(slots) * sizeof(int)));
        step(cudaMemsetAsync(split_cnt, 0, pr::emu_split_counters(slots) * sizeof(int), s));
      }
      step(cudaMemcpyAsync(items, hitems.data(), hitems.size() * sizeof(int4), cudaMemcpyHostToDevice, s));
      step(pr::slice(dX, ni, eld, S, hX, eX, s));
      step(pr::slice(dY, ni, eld, S, hY, eY, s));
      step(pr::gemm_emu(hX, eX, hY, eY, ni, eld, precision == PR_FP32X ? std::min(S, kFp32xSlices) : S, mode, false,
                        items, (int)hitems.size(), ep, scratch, split, split_cnt, err, s, bn));
    }
    step(cudaMemcpyAsync(P, dP, bytes, cudaMemcpyDefault, s));
    step(cudaMemcpyAsync(&word, err, sizeof(int), cudaMemcpyDeviceToHost, s));
    step(cudaStreamSynchronize(s));
  }
  for (void* q : {(void*)dX, (void*)dY, (void*)dP, (void*)bX, (void*)bY, (void*)err, (void*)eX, (void*)eY, (void*)items,
                  (void*)scratch, (void*)split, (void*)split_cnt})
    if (q) cudaFree(q);
  if (e != cudaSuccess) return cuda_fail(nullptr, "pr_matmul", e);
  if (word != 0)
    return fail(nullptr, PR_ETIMEOUT, "pr_matmul: a bounded device wait expired (code " + std::to_string(word) + ")");
  return PR_OK;
}

}  // namespace

namespace {

// ---- Block-sparse A (pr_options.block_sparse)
//
// From the first and last non-zero column of every row of A: the unsplit work lists of every product mode and
// tile width with each tile restricted to the K steps [j0, j1) that can hold non-zero digits of the rows of A
// the tile reads (A the first operand: the tile's 128 rows; the second: its bn columns, i.e. rows of A; both:
// the intersection). A tile whose rows of A are zero keeps one step (its digits are zero). Used when the full
// product A X keeps at most 7/8 of the steps; the lists are rebuilt at every pr_load.
pr_status build_sparse_lists(pr_handle h) {
  const int n = (int)h->n, KS = (n + 15) / 16;
  auto envelope = [&](int r0, int rows, int& lo, int& hi) {
    for (int r = r0; r < std::min(n, r0 + rows); ++r) {
      lo = std::min(lo, h->a_first[r]);
      hi = std::max(hi, h->a_last[r]);
    }
  };
  std::vector<int4> lists[2][2][3];
  double kept = 0.0, total = 0.0;
  for (int m = 0; m < 2; ++m)
    for (int wi = 0; wi < 2; ++wi) {
      if (!h->emu_items[m][2 * wi]) continue;  // width not in use (pr_options.emu_tile)
      const int bn = kEmuVariants[2 * wi].bn;
      std::vector<int4> base;
      pr::emu_launch_list(n, m == 0 ? Mode::Sym : Mode::Full, base, bn, 0);
      for (int side = 0; side < 3; ++side) {
        std::vector<int4>& out = lists[m][wi][side];
        out.reserve(base.size());
        for (const int4& it : base) {
          int lo1 = n, hi1 = -1, lo2 = n, hi2 = -1;
          if (side != 1) envelope(128 * it.y, 128, lo1, hi1);
          if (side != 0) envelope(bn * it.z, bn, lo2, hi2);
          const int lo = side == 0 ? lo1 : side == 1 ? lo2 : std::max(lo1, lo2);
          const int hi = side == 0 ? hi1 : side == 1 ? hi2 : std::min(hi1, hi2);
          const int j0 = hi < lo ? 0 : lo / 16, j1 = hi < lo ? 1 : hi / 16 + 1;
          out.push_back(j0 == 0 && j1 == KS ? it : pr::emu_range_item(it, j0, j1));
          if (m == 1 && wi == 0 && side == 0) {
            kept += j1 - j0;
            total += KS;
          }
        }
      }
    }
  h->st.sparse_keep = total > 0 ? kept / total : 1.0;
  h->sp_on = h->st.sparse_keep <= 0.875;
  if (!h->sp_on) return PR_OK;
  for (int m = 0; m < 2; ++m)
    for (int wi = 0; wi < 2; ++wi)
      for (int side = 0; side < 3; ++side) {
        const std::vector<int4>& v = lists[m][wi][side];
        if (v.empty()) continue;
        if (!h->sp_items[m][wi][side]) PR_CK(h, cudaMalloc((void**)&h->sp_items[m][wi][side], v.size() * sizeof(int4)));
        PR_CK(h, cudaMemcpy(h->sp_items[m][wi][side], v.data(), v.size() * sizeof(int4), cudaMemcpyHostToDevice));
      }
  return PR_OK;
}

// ---- Newton refinement of an approximate root (pr_refine)
//
// Newton's method on the balanced residual G(X) = I - sym(X^m A X^m'), m = floor(p/2), m' = p - m: each step
// solves sym(dP_m(D) A X^m' + X^m A dP_m'(D)) = G(X) for a symmetric D by preconditioned conjugate gradients
// and sets X <- X + D (see pr_refine in the header). With U = X^m, V = X^m', Y = V A and W = U A:
//   G(X) = I - sym(W V),   L(S) = sym(Y dP_m(S) + W dP_m'(S))   (the transpose of the first term of the
//   definition, D_m A V, is V A D_m = Y dP_m(S); sym() does not see the difference),
//   dP_1(S) = S, dP_2(S) = X S + S X = 2 sym(X S); for m = m' both terms are equal, L(S) = 2 sym(Y dP_m(S)).
// Every product below has a symmetric second operand, so X Y and X Y^T coincide and the product kernels of
// every precision apply. Buffers (the coupled form's state and the scratch products are free while a
// refinement runs; the next pr_iterate re-forms M and N from X): T0 = X^2, T1 = Y, Nn = W (p = 3; W = Y when
// m = m', W = A when p = 1), M = R (the solve's residual, first G), Mn = D (the correction), N = S (the search
// direction), Ra = Z (the preconditioned residual), Rb = L(S), Rc = dP_2(S), Xn = a product before its
// symmetrisation.

constexpr int kRefScalars = 8;

pr_status ensure_refine(pr_handle h) {
  const size_t nn = (size_t)h->n * (size_t)h->n;
  for (Mat* m : {&h->Ra, &h->Rb, &h->Rc}) {
    if (!m->f) PR_CK(h, cudaMalloc((void**)&m->f, nn * sizeof(double)));
    if (!m->b) PR_CK(h, cudaMalloc((void**)&m->b, (size_t)h->n * (size_t)h->ldl * sizeof(__nv_bfloat16)));
  }
  if (!h->xbest) PR_CK(h, cudaMalloc((void**)&h->xbest, nn * sizeof(double)));
  if (!h->rdev) PR_CK(h, cudaMalloc((void**)&h->rdev, sizeof(double) * (kVecBlocks + kRefScalars)));
  if (!h->rpin) PR_CK(h, cudaMallocHost((void**)&h->rpin, sizeof(double) * kRefScalars));
  return PR_OK;
}

// BF16 products read their operands' BF16 copies; refresh them from the FP64 values. (Digit planes and E4M3
// copies are refreshed by product() itself when the matrix changed.)
pr_status lp_operand(pr_handle h, int prec, Mat& m) {
  if (prec != PR_BF16 || m.b_valid) return PR_OK;
  PR_CK(h, pr::to_bf16(m.f, (int)h->n, h->ldl, m.b, h->stream));
  h->st.launches += 1;
  m.b_valid = true;
  return PR_OK;
}

// out = P = Xop Yop (Yop symmetric) in the given mode.
pr_status plain_product(pr_handle h, int prec, Mat& Xop, Mat& Yop, Mode mode, Mat& out) {
  pr_status s = lp_operand(h, prec, Xop);
  if (s == PR_OK) s = lp_operand(h, prec, Yop);
  if (s != PR_OK) return s;
  Out o;
  o.out = &out;
  o.lp_copy = false;
  return product(h, prec, Xop, Yop, mode, o);
}

// out = scale sym(Xop Yop) (Yop symmetric), the full product going through Xn.
pr_status sym_of_product(pr_handle h, int prec, Mat& Xop, Mat& Yop, double scale, Mat& out) {
  pr_status s = lp_operand(h, prec, Xop);
  if (s == PR_OK) s = lp_operand(h, prec, Yop);
  if (s != PR_OK) return s;
  Out o;
  o.out2 = &h->Xn;
  o.b = scale;
  o.lp_copy = false;
  s = product(h, prec, Xop, Yop, Mode::Full, o);
  if (s != PR_OK) return s;
  PR_CK(h, pr::symmetrize(h->Xn.f, (int)h->n, out.f, h->stream));
  h->st.launches += 1;
  out.changed();
  return PR_OK;
}

// Frobenius inner product <x, y> into device scalar k.
pr_status fdot(pr_handle h, const Mat& x, const Mat& y, int k) {
  PR_CK(h, pr::frobenius_dot(x.f, y.f, h->n * h->n, h->rdev, h->rdev + kVecBlocks + k, h->stream));
  h->st.launches += 2;
  return PR_OK;
}

// Device scalars 0 .. count-1 -> h->rpin (synchronises; a bounded wait that expired shows here).
pr_status read_scalars(pr_handle h, int count) {
  PR_CK(h, cudaMemcpyAsync(h->rpin, h->rdev + kVecBlocks, count * sizeof(double), cudaMemcpyDeviceToHost,
                           h->stream));
  return sync(h);
}

struct RefineOps {
  int m = 0, mq = 0;
  Mat *U = nullptr, *V = nullptr, *Y = nullptr, *W = nullptr;  // U = X^m (null: I), V = X^m', Y = V A, W = U A
};

// The products of one step that do not depend on the correction, at the residual's precision.
pr_status refine_setup(pr_handle h, int prec, RefineOps& o) {
  o.m = h->p / 2;
  o.mq = h->p - o.m;
  pr_status s = PR_OK;
  Mat* X2 = nullptr;
  if (o.mq == 2) {
    s = plain_product(h, prec, h->X, h->X, Mode::Sym, h->T0);
    if (s != PR_OK) return s;
    X2 = &h->T0;
  }
  o.V = o.mq == 1 ? &h->X : X2;
  o.U = o.m == 0 ? nullptr : (o.m == 1 ? &h->X : X2);
  if (o.m >= 1) {
    s = plain_product(h, prec, *o.V, h->A, Mode::Full, h->T1);
    if (s != PR_OK) return s;
    o.Y = &h->T1;
  }
  if (o.m == 0) {
    o.W = &h->A;
  } else if (o.m == o.mq) {
    o.W = o.Y;
  } else {
    s = plain_product(h, prec, *o.U, h->A, Mode::Full, h->Nn);
    if (s != PR_OK) return s;
    o.W = &h->Nn;
  }
  return PR_OK;
}

// R = G(X) = I - sym(W V); *g = ||G(X)||_F.
pr_status refine_residual(pr_handle h, int prec, const RefineOps& o, double* g) {
  pr_status s = lp_operand(h, prec, *o.W);
  if (s == PR_OK) s = lp_operand(h, prec, *o.V);
  if (s != PR_OK) return s;
  Out oo;
  oo.a = 1.0;
  oo.b = -1.0;
  oo.lp_copy = false;
  if (o.m == o.mq) {  // W V = X^m A X^m is symmetric: upper tiles, mirrored
    oo.out2 = &h->M;
    s = product(h, prec, *o.W, *o.V, Mode::Sym, oo);
    if (s != PR_OK) return s;
  } else {
    oo.out2 = &h->Xn;
    s = product(h, prec, *o.W, *o.V, Mode::Full, oo);
    if (s != PR_OK) return s;
    PR_CK(h, pr::symmetrize(h->Xn.f, (int)h->n, h->M.f, h->stream));
    h->st.launches += 1;
  }
  h->M.changed();
  s = fdot(h, h->M, h->M, 0);
  if (s == PR_OK) s = read_scalars(h, 1);
  if (s != PR_OK) return s;
  *g = sqrt(h->rpin[0]);
  return PR_OK;
}

// LS = L(S) at prec.
pr_status refine_apply(pr_handle h, int prec, const RefineOps& o, Mat& S, Mat& LS) {
  pr_status s = PR_OK;
  Mat* D2 = nullptr;
  if (o.m == 2 || o.mq == 2) {
    s = sym_of_product(h, prec, h->X, S, 2.0, h->Rc);  // dP_2(S) = X S + S X
    if (s != PR_OK) return s;
    D2 = &h->Rc;
  }
  Mat* Dm = o.m == 1 ? &S : D2;
  Mat* Dmq = o.mq == 1 ? &S : D2;
  if (o.m == o.mq) return sym_of_product(h, prec, *o.Y, *Dm, 2.0, LS);
  if (o.m == 0) return sym_of_product(h, prec, *o.W, *Dmq, 1.0, LS);
  // p = 3: sym(Y S + W dP_2(S)), the first product kept in LS until the second adds it in its epilogue
  s = plain_product(h, prec, *o.Y, *Dm, Mode::Full, LS);
  if (s == PR_OK) s = lp_operand(h, prec, *o.W);
  if (s == PR_OK) s = lp_operand(h, prec, *Dmq);
  if (s != PR_OK) return s;
  Out oo;
  oo.out2 = &h->Xn;
  oo.b = 1.0;
  oo.c = 1.0;
  oo.cin = LS.f;
  oo.lp_copy = false;
  s = product(h, prec, *o.W, *Dmq, Mode::Full, oo);
  if (s != PR_OK) return s;
  PR_CK(h, pr::symmetrize(h->Xn.f, (int)h->n, LS.f, h->stream));
  h->st.launches += 1;
  LS.changed();
  return PR_OK;
}

// D with L(D) = R (R = G on entry, overwritten) by conjugate gradients preconditioned with Z = sym(X R) / p,
// from D = 0, until ||R||_F <= cg_tol g0 or cg_max iterations, or a breakdown (a non-positive curvature
// <S, L(S)> or <R, Z>, possible only far from the root); *its: the iterations taken.
pr_status refine_solve(pr_handle h, int prec, const RefineOps& o, double g0, int cg_max, double cg_tol, int* its) {
  Mat &R = h->M, &D = h->Mn, &S = h->N, &Z = h->Ra, &LS = h->Rb;
  const int64_t total = h->n * h->n;
  const double inv_p = 1.0 / h->p;
  *its = 0;
  PR_CK(h, cudaMemsetAsync(D.f, 0, (size_t)total * sizeof(double), h->stream));
  D.changed();
  pr_status s = sym_of_product(h, prec, h->X, R, inv_p, Z);
  if (s != PR_OK) return s;
  PR_CK(h, cudaMemcpyAsync(S.f, Z.f, (size_t)total * sizeof(double), cudaMemcpyDeviceToDevice, h->stream));
  S.changed();
  s = fdot(h, R, Z, 0);
  if (s == PR_OK) s = read_scalars(h, 1);
  if (s != PR_OK) return s;
  double rz = h->rpin[0];
  int it = 0;
  while (it < cg_max && rz > 0.0 && std::isfinite(rz)) {
    const pr::NvtxRange trace("refine solve iteration");
    s = refine_apply(h, prec, o, S, LS);
    if (s == PR_OK) s = fdot(h, S, LS, 0);
    if (s == PR_OK) s = read_scalars(h, 1);
    if (s != PR_OK) return s;
    const double curv = h->rpin[0];
    if (!(curv > 0.0) || !std::isfinite(curv)) break;
    const double alpha = rz / curv;
    PR_CK(h, pr::lincomb(D.f, S.f, total, 1.0, alpha, D.f, h->stream));
    PR_CK(h, pr::lincomb(R.f, LS.f, total, 1.0, -alpha, R.f, h->stream));
    h->st.launches += 2;
    D.changed();
    R.changed();
    ++it;
    s = fdot(h, R, R, 0);
    if (s != PR_OK) return s;
    if (it < cg_max) {  // the next preconditioned residual, read back with ||R||^2 in one synchronisation
      s = sym_of_product(h, prec, h->X, R, inv_p, Z);
      if (s == PR_OK) s = fdot(h, R, Z, 1);
      if (s != PR_OK) return s;
    }
    s = read_scalars(h, it < cg_max ? 2 : 1);
    if (s != PR_OK) return s;
    if (sqrt(h->rpin[0]) <= cg_tol * g0 || it >= cg_max) break;
    const double rz_new = h->rpin[1];
    PR_CK(h, pr::lincomb(Z.f, S.f, total, 1.0, rz_new / rz, S.f, h->stream));
    h->st.launches += 1;
    S.changed();
    rz = rz_new;
  }
  *its = it;
  return PR_OK;
}

}  // namespace

extern "C" {

int pr_version(void) { return 100; }

void pr_default_options(pr_options* o) {
  if (!o) return;
  memset(o, 0, sizeof(*o));
  o->form = PR_FORM_AUTO;
  o->c0 = PR_C0_EQ3;
  o->max_iter = 100;
  o->stag_below = 1e-3;
  o->stag_ratio = 0.5;
  o->sym_tol = 1e-12;
  o->reanchor = 1;
  o->emu_slices = 0;
  o->stag_below_lowp = 0.5;
  o->c0_coef[0] = 1.0;
  o->c0_coef[1] = o->c0_coef[2] = o->c0_coef[3] = 0.0;
  o->gate_max = 0.9;
  o->gate_iters = 30;
  o->verify = 1;
  o->gate_fallback = 1;
  o->emu_tile = 0;
  o->quant_bits = 0;
  o->quant_mode = PR_QUANT_STORAGE;
  o->block_sparse = 1;
}

const char* pr_last_error(pr_handle h) { return h ? h->err.c_str() : g_init_error.c_str(); }

pr_status pr_destroy(pr_handle h) {
  if (!h) return PR_OK;
  cudaSetDevice(h->device);
  if (h->stream) cudaStreamSynchronize(h->stream);
  for (Mat* m : {&h->A, &h->X, &h->Xn, &h->M, &h->Mn, &h->N, &h->Nn, &h->T0, &h->T1, &h->Ra, &h->Rb, &h->Rc}) {
    if (m->f) cudaFree(m->f);
    if (m->b) cudaFree(m->b);
    if (m->sl) cudaFree(m->sl);
    if (m->ex) cudaFree(m->ex);
    if (m->q) cudaFree(m->q);
    if (m->qe) cudaFree(m->qe);
  }
  for (double* b : {h->partial, h->work, h->scal, h->vec, h->xbest, h->xstart, h->rdev})
    if (b) cudaFree(b);
  if (h->rpin) cudaFreeHost(h->rpin);
  for (auto& lists : h->emu_items)
    for (int4* it : lists)
      if (it) cudaFree(it);
  if (h->emu_scratch) cudaFree(h->emu_scratch);
  if (h->emu_split) cudaFree(h->emu_split);
  if (h->emu_split_cnt) cudaFree(h->emu_split_cnt);
  if (h->span_dev) cudaFree(h->span_dev);
  for (auto& a : h->sp_items)
    for (auto& b : a)
      for (int4* it : b)
        if (it) cudaFree(it);
  if (h->hpin) cudaFreeHost(h->hpin);
  for (cudaEvent_t e : h->ev) cudaEventDestroy(e);
  delete h;
  return PR_OK;
}

pr_status pr_init(pr_handle* out, const double* A, int64_t n, int p, const pr_options* opt, void* stream) {
  if (!out) return fail(nullptr, PR_EINVAL, "pr_init: h is NULL");
  *out = nullptr;
  if (!A) return fail(nullptr, PR_EINVAL, "pr_init: A is NULL");
  if (n < 1 || n > (int64_t)1 << 17) return fail(nullptr, PR_EINVAL, "pr_init: n must be in [1, 131072]");
  if (p < 1 || p > 64) return fail(nullptr, PR_EINVAL, "pr_init: p must be in [1, 64]");
  pr_options o;
  if (opt) o = *opt;
  else pr_default_options(&o);
  if (o.form < PR_FORM_AUTO || o.form > PR_FORM_LITERAL) return fail(nullptr, PR_EINVAL, "pr_init: unknown form");
  if (o.c0 != PR_C0_EQ3 && o.c0 != PR_C0_SCALED_I && o.c0 != PR_C0_POLY)
    return fail(nullptr, PR_EINVAL, "pr_init: unknown c0 kind");
  if (o.c0 == PR_C0_POLY && (!(o.gate_max > 0) || o.gate_iters < 1))
    return fail(nullptr, PR_EINVAL, "pr_init: bad gate options");
  if (o.form == PR_FORM_NS && p != 1) return fail(nullptr, PR_EINVAL, "pr_init: the Newton-Schulz form needs p = 1");
  if (o.quant_bits != 0 &&
      (o.quant_bits < 1 || o.quant_bits > 52 || (o.quant_mode != PR_QUANT_STORAGE && o.quant_mode != PR_QUANT_ARITH)))
    return fail(nullptr, PR_EINVAL, "pr_init: quant_bits must be in [1, 52] and quant_mode storage or arithmetic");
  if (o.quant_bits != 0 && (o.form != PR_FORM_LITERAL || o.c0 != PR_C0_EQ3))
    return fail(nullptr, PR_EUNSUPPORTED, "pr_init: the custom-precision experiment runs the literal form from Eq. 3");
  if (o.max_iter < 0 || !(o.stag_ratio > 0) || !(o.sym_tol >= 0) || !(o.stag_below_lowp >= 0) ||
      o.emu_slices < 0 || o.emu_slices > pr::emu_max_slices() || (o.emu_tile != 0 && !pr::emu_tile_width_ok(o.emu_tile)))
    return fail(nullptr, PR_EINVAL, "pr_init: bad option value");

  pr_handle h = new pr_handle_s();
  h->n = n;
  h->p = p;
  h->opt = o;
  h->form = o.form == PR_FORM_AUTO ? (p == 1 ? PR_FORM_NS : PR_FORM_COUPLED) : o.form;
  h->stream = (cudaStream_t)stream;
  h->ldl = pr::bf16_ld((int)n);
  h->ldq = pr::fp8_ld((int)n);
  h->eld = pr::emu_ld((int)n);
  h->S = o.emu_slices > 0 ? o.emu_slices : pr::emu_max_slices();
  h->st.emu_slices = h->S;
  h->st.n = n;
  h->st.p = p;
  h->st.form = h->form;
  h->st.c0 = o.c0;
  h->st.switch_iteration = -1;
  h->st.last_precision = -1;
  h->st.true_residual = -1.0;
  cudaGetDevice(&h->device);

  auto bail = [&](pr_status code) {
    g_init_error = h->err;
    pr_destroy(h);
    return code;
  };
#define PR_INIT_CK(call)                                         \
  do {                                                           \
    cudaError_t _e = (call);                                     \
    if (_e != cudaSuccess) return bail(cuda_fail(h, #call, _e)); \
  } while (0)

  const size_t bytes = (size_t)n * (size_t)n * sizeof(double);
  const size_t lbytes = (size_t)n * (size_t)h->ldl * sizeof(__nv_bfloat16);
  for (Mat* m : {&h->A, &h->X, &h->Xn, &h->M, &h->Mn, &h->N, &h->Nn, &h->T0, &h->T1}) {
    PR_INIT_CK(cudaMalloc((void**)&m->f, bytes));
    PR_INIT_CK(cudaMalloc((void**)&m->b, lbytes));
  }
  const int T64 = (int)((n + 63) / 64);
  size_t nparts = (size_t)T64 * T64;
  const size_t tc_parts = (size_t)pr::gemm_tc_tiles((int)n, Mode::Full);
  const size_t emu_parts = (size_t)pr::emu_tiles((int)n, Mode::Full, 48);  // the narrower tile has more
  if (tc_parts > nparts) nparts = tc_parts;
  if (emu_parts > nparts) nparts = emu_parts;
  PR_INIT_CK(cudaMalloc((void**)&h->partial, sizeof(double) * nparts));
  PR_INIT_CK(cudaMalloc((void**)&h->work, sizeof(double) * 2 * (size_t)n));
  PR_INIT_CK(cudaMalloc((void**)&h->scal, sizeof(double) * 8));
  PR_INIT_CK(cudaMemset(h->scal, 0, sizeof(double) * 8));
  PR_INIT_CK(cudaMallocHost((void**)&h->hpin, sizeof(double) * 8));
  // The digit-slice products' work lists of this order (symmetric, full) for every variant that applies:
  // whole tiles always; tiles split over K only for short launches (fewer than 4 waves of tiles) with at
  // least two K steps, and only for the width chosen by emu_tile if it is fixed.
  int slots = 0;
  for (int k = 0; k < 2; ++k) {
    const Mode mode = k == 0 ? Mode::Sym : Mode::Full;
    for (int v = 0; v < 4; ++v) {
      const EmuVariant var = kEmuVariants[v];
      if (o.emu_tile != 0 && var.bn != o.emu_tile) continue;
      if (var.split && !(o.emu_tile == 0 ? pr::emu_split_useful((int)n, mode, var.bn)
                                         : pr::emu_split_slots((int)n, mode, var.bn, -1) > 0))
        continue;
      std::vector<int4> items;
      pr::emu_launch_list((int)n, mode, items, var.bn, var.split);
      h->emu_nsplit[k][v] = pr::emu_split_slots((int)n, mode, var.bn, var.split);
      slots = std::max(slots, h->emu_nsplit[k][v]);
      h->emu_nitems[k][v] = (int)items.size();
      PR_INIT_CK(cudaMalloc((void**)&h->emu_items[k][v], items.size() * sizeof(int4)));
      PR_INIT_CK(cudaMemcpy(h->emu_items[k][v], items.data(), items.size() * sizeof(int4), cudaMemcpyHostToDevice));
    }
  }
  PR_INIT_CK(cudaMalloc((void**)&h->emu_scratch, pr::emu_scratch_bytes()));
  PR_INIT_CK(cudaMalloc((void**)&h->span_dev, 2 * (size_t)n * sizeof(int)));
  if (slots > 0) {
    PR_INIT_CK(cudaMalloc((void**)&h->emu_split, pr::emu_split_bytes(slots)));
    PR_INIT_CK(cudaMalloc((void**)&h->emu_split_cnt, pr::emu_split_counters(slots) * sizeof(int)));
    PR_INIT_CK(cudaMemset(h->emu_split_cnt, 0, pr::emu_split_counters(slots) * sizeof(int)));
  }
#undef PR_INIT_CK
  pr_status s = pr_load(h, A);
  if (s != PR_OK) return bail(s);
  *out = h;
  return PR_OK;
}

pr_status pr_load(pr_handle h, const double* A) {
  if (!h) return fail(nullptr, PR_ESTATE, "pr_load: NULL handle");
  if (!A) return fail(h, PR_EINVAL, "pr_load: A is NULL");
  cudaSetDevice(h->device);
  const int n = (int)h->n;
  const size_t bytes = (size_t)n * (size_t)n * sizeof(double);
  reset_iteration(h);
  h->powers_valid = false;
  h->A.changed();
  h->st.norm_1 = 0.0;
  PR_CK(h, cudaMemcpyAsync(h->A.f, A, bytes, cudaMemcpyDefault, h->stream));
  if (h->opt.quant_bits > 0) {  // the custom-precision experiment: the input is stored with m mantissa bits
    PR_CK(h, pr::round_values(h->A.f, (int64_t)n * n, h->opt.quant_bits, h->A.f, h->stream));
    h->st.launches += 1;
  }
  PR_CK(h, pr::validate(h->A.f, n, h->scal, h->stream));
  PR_CK(h, pr::abs_norms(h->A.f, n, h->work, h->scal + 4, h->stream));
  h->st.launches += 4;
  PR_CK(h, cudaMemcpyAsync(h->hpin, h->scal, 6 * sizeof(double), cudaMemcpyDeviceToHost, h->stream));
  h->sp_on = false;
  h->st.sparse_keep = 1.0;
  if (h->opt.block_sparse) {
    PR_CK(h, pr::row_spans(h->A.f, n, h->span_dev, h->span_dev + n, h->stream));
    h->st.launches += 1;
    h->a_first.resize(n);
    h->a_last.resize(n);
    PR_CK(h, cudaMemcpyAsync(h->a_first.data(), h->span_dev, n * sizeof(int), cudaMemcpyDeviceToHost, h->stream));
    PR_CK(h, cudaMemcpyAsync(h->a_last.data(), h->span_dev + n, n * sizeof(int), cudaMemcpyDeviceToHost, h->stream));
  }
  pr_status s = sync(h);
  if (s != PR_OK) return s;
  const double amax = h->hpin[0], asym = h->hpin[1], nonfinite = h->hpin[2], nonpos = h->hpin[3];
  if (nonfinite > 0) return fail(h, PR_EINVAL, "pr_load: A has non-finite entries");
  if (asym > h->opt.sym_tol * amax) {
    char buf[160];
    snprintf(buf, sizeof buf, "pr_load: A is not symmetric (max|a_ij - a_ji| = %.3e > %.1e * max|a_ij|)", asym,
             h->opt.sym_tol);
    return fail(h, PR_EINVAL, buf);
  }
  if (nonpos > 0)
    return fail(h, PR_ENOTSPD,
                "pr_load: A is not positive definite (a non-positive diagonal entry, or a diagonal block of order 64 "
                "without a Cholesky factorisation)");
  h->st.norm_1 = h->hpin[4];
  h->st.norm_inf = h->hpin[5];
  if (h->opt.block_sparse) {
    s = build_sparse_lists(h);
    if (s != PR_OK) return s;
  }
  h->st.prescale_log2 = 0;
  if (h->p > 1 && h->st.norm_1 * h->st.norm_inf < 1.0) {
    // Eq. 2 for Eq. 3's C_0 needs ||A||_1 >= 1 when p > 1 (eigenvalues of C_0^p A up to ||A||_1^(1-p)):
    // iterate on 2^k A with ||2^k A||_1 = 2 f in [1, 2) (||A||_1 = f 2^e, f in [0.5, 1)). A power of two
    // scales exactly; pr_result multiplies the root by 2^(k/p).
    int e = 0;
    frexp(h->st.norm_1, &e);
    const int k = 1 - e;
    const double c = ldexp(1.0, k);
    PR_CK(h, pr::lincomb(h->A.f, h->A.f, (int64_t)n * n, c, 0.0, h->A.f, h->stream));
    h->st.launches += 1;
    h->st.norm_1 *= c;
    h->st.norm_inf *= c;
    h->st.prescale_log2 = k;
  }
  return form_initial_guess(h);
}

namespace {

// Byte layout of an exported state (see pr_state_header).
struct StateLayout {
  size_t hist, prec, f, b, total;
  int n_mats;
};

StateLayout state_layout(pr_handle h, int hist_len, int n_mats) {
  const size_t nn = (size_t)h->n * (size_t)h->n, nb = (size_t)h->n * (size_t)h->ldl;
  StateLayout L;
  L.n_mats = n_mats;
  L.hist = sizeof(pr_state_header);
  L.prec = L.hist + (size_t)hist_len * sizeof(double);
  L.f = L.prec + ((size_t)hist_len * sizeof(int32_t) + 7) / 8 * 8;
  L.b = L.f + (size_t)n_mats * nn * sizeof(double);
  L.total = L.b + (size_t)n_mats * nb * sizeof(__nv_bfloat16);
  return L;
}

int state_mats(pr_handle h) { return h->form == PR_FORM_COUPLED && h->state_ready ? 3 : 1; }

}  // namespace

pr_status pr_state_size(pr_handle h, size_t* bytes) {
  if (!h) return fail(nullptr, PR_ESTATE, "pr_state_size: NULL handle");
  if (!bytes) return fail(h, PR_EINVAL, "pr_state_size: bytes is NULL");
  *bytes = state_layout(h, (int)h->hist.size(), state_mats(h)).total;
  return PR_OK;
}

pr_status pr_export_state(pr_handle h, void* buf, size_t bytes) {
  if (!h) return fail(nullptr, PR_ESTATE, "pr_export_state: NULL handle");
  const StateLayout L = state_layout(h, (int)h->hist.size(), state_mats(h));
  if (!buf || bytes < L.total) return fail(h, PR_EINVAL, "pr_export_state: buffer NULL or too small");
  cudaSetDevice(h->device);
  pr_state_header hd{};
  hd.magic = PR_STATE_MAGIC;
  hd.version = PR_STATE_VERSION;
  hd.n = h->n;
  hd.p = h->p;
  hd.form = h->form;
  hd.c0 = h->st.c0;
  hd.norm_1 = h->st.norm_1;
  hd.norm_inf = h->st.norm_inf;
  hd.state_ready = h->state_ready ? 1 : 0;
  hd.state_level = h->state_level;
  hd.lp_stale = h->lp_stale ? 1 : 0;
  hd.iterations = h->st.iterations;
  for (int k = 0; k < PR_NPREC; ++k) hd.iterations_by_precision[k] = h->st.iterations_by_precision[k];
  hd.switch_iteration = h->st.switch_iteration;
  hd.last_precision = h->st.last_precision;
  hd.hist_len = (int32_t)h->hist.size();
  hd.n_mats = L.n_mats;
  hd.ldl = h->ldl;
  hd.last_residual = h->st.last_residual;
  char* out = static_cast<char*>(buf);
  memcpy(out, &hd, sizeof hd);
  if (!h->hist.empty()) {
    memcpy(out + L.hist, h->hist.data(), h->hist.size() * sizeof(double));
    for (size_t k = 0; k < h->hist_prec.size(); ++k) {
      const int32_t v = h->hist_prec[k];
      memcpy(out + L.prec + k * sizeof(int32_t), &v, sizeof v);
    }
  }
  const size_t nn = (size_t)h->n * (size_t)h->n, nb = (size_t)h->n * (size_t)h->ldl;
  const Mat* mats[3] = {&h->X, &h->M, &h->N};
  for (int k = 0; k < L.n_mats; ++k) {
    PR_CK(h, cudaMemcpyAsync(out + L.f + k * nn * sizeof(double), mats[k]->f, nn * sizeof(double),
                             cudaMemcpyDeviceToHost, h->stream));
    PR_CK(h, cudaMemcpyAsync(out + L.b + k * nb * sizeof(__nv_bfloat16), mats[k]->b, nb * sizeof(__nv_bfloat16),
                             cudaMemcpyDeviceToHost, h->stream));
  }
  return sync(h);
}

pr_status pr_import_state(pr_handle h, const void* buf, size_t bytes) {
  if (!h) return fail(nullptr, PR_ESTATE, "pr_import_state: NULL handle");
  if (!buf || bytes < sizeof(pr_state_header)) return fail(h, PR_EINVAL, "pr_import_state: buffer NULL or too small");
  pr_state_header hd;
  memcpy(&hd, buf, sizeof hd);
  if (hd.magic != PR_STATE_MAGIC || hd.version != PR_STATE_VERSION) return fail(h, PR_EINVAL, "pr_import_state: not a state buffer");
  if (hd.n != h->n || hd.p != h->p || hd.form != h->form || hd.ldl != h->ldl)
    return fail(h, PR_EINVAL, "pr_import_state: the state belongs to another order, root or form");
  if (hd.norm_1 != h->st.norm_1 || hd.norm_inf != h->st.norm_inf)
    return fail(h, PR_EINVAL, "pr_import_state: the state belongs to another matrix (its norms differ)");
  if (hd.hist_len < 0 || hd.hist_len > h->opt.max_iter + 2 || (hd.n_mats != 1 && hd.n_mats != 3) ||
      (hd.n_mats == 3) != (hd.form == PR_FORM_COUPLED && hd.state_ready != 0))
    return fail(h, PR_EINVAL, "pr_import_state: inconsistent header");
  const StateLayout L = state_layout(h, hd.hist_len, hd.n_mats);
  if (bytes < L.total) return fail(h, PR_EINVAL, "pr_import_state: buffer shorter than its header says");
  cudaSetDevice(h->device);
  const char* in = static_cast<const char*>(buf);
  const size_t nn = (size_t)h->n * (size_t)h->n, nb = (size_t)h->n * (size_t)h->ldl;
  Mat* mats[3] = {&h->X, &h->M, &h->N};
  for (int k = 0; k < L.n_mats; ++k) {
    PR_CK(h, cudaMemcpyAsync(mats[k]->f, in + L.f + k * nn * sizeof(double), nn * sizeof(double),
                             cudaMemcpyHostToDevice, h->stream));
    PR_CK(h, cudaMemcpyAsync(mats[k]->b, in + L.b + k * nb * sizeof(__nv_bfloat16), nb * sizeof(__nv_bfloat16),
                             cudaMemcpyHostToDevice, h->stream));
  }
  if (hd.lp_stale == 0) {  // the BF16 copies are current: A's (not in the state) must be too
    PR_CK(h, pr::to_bf16(h->A.f, (int)h->n, h->ldl, h->A.b, h->stream));
    h->st.launches += 1;
  }
  pr_status s = sync(h);
  if (s != PR_OK) return s;
  reset_iteration(h);
  h->state_ready = hd.state_ready != 0;
  h->state_level = hd.state_level;
  h->lp_stale = hd.lp_stale != 0;
  h->st.c0 = hd.c0;
  h->st.iterations = hd.iterations;
  for (int k = 0; k < PR_NPREC; ++k) h->st.iterations_by_precision[k] = hd.iterations_by_precision[k];
  h->st.switch_iteration = hd.switch_iteration;
  h->st.last_precision = hd.last_precision;
  h->st.last_residual = hd.last_residual;
  h->hist.resize(hd.hist_len);
  h->hist_prec.resize(hd.hist_len);
  if (hd.hist_len > 0) memcpy(h->hist.data(), in + L.hist, (size_t)hd.hist_len * sizeof(double));
  for (int k = 0; k < hd.hist_len; ++k) {
    int32_t v;
    memcpy(&v, in + L.prec + (size_t)k * sizeof(int32_t), sizeof v);
    h->hist_prec[k] = v;
  }
  return PR_OK;
}

pr_status pr_set_initial_guess(pr_handle h, int kind, const double* coef) {
  if (!h) return fail(nullptr, PR_ESTATE, "pr_set_initial_guess: NULL handle");
  if (kind != PR_C0_EQ3 && kind != PR_C0_SCALED_I && kind != PR_C0_POLY)
    return fail(h, PR_EINVAL, "pr_set_initial_guess: unknown kind");
  if (kind == PR_C0_POLY && !coef) return fail(h, PR_EINVAL, "pr_set_initial_guess: PR_C0_POLY needs coef");
  if (h->st.norm_1 <= 0.0) return fail(h, PR_ESTATE, "pr_set_initial_guess: no matrix loaded");
  if (kind == PR_C0_POLY)
    for (int i = 0; i < 4; ++i)
      if (!std::isfinite(coef[i])) return fail(h, PR_EINVAL, "pr_set_initial_guess: non-finite coefficient");
  cudaSetDevice(h->device);
  reset_iteration(h);
  // A one-off choice: the handle's options (used by later pr_load calls) stay as they are.
  const pr_options keep = h->opt;
  h->opt.c0 = kind;
  if (kind == PR_C0_POLY)
    for (int i = 0; i < 4; ++i) h->opt.c0_coef[i] = coef[i];
  pr_status s = form_initial_guess(h);
  h->opt = keep;
  return s;
}

pr_status pr_set_timing(pr_handle h, int on) {
  if (!h) return fail(nullptr, PR_ESTATE, "pr_set_timing: NULL handle");
  cudaSetDevice(h->device);
  if (on && h->ev.empty()) {
    h->ev.resize(2 * kEventPairs);
    h->ev_flops.resize(kEventPairs);
    h->ev_prec.resize(kEventPairs);
    for (cudaEvent_t& e : h->ev) PR_CK(h, cudaEventCreate(&e));
  }
  if (!on) {
    pr_status s = sync(h);
    if (s != PR_OK) return s;
  }
  h->timing = on != 0;
  return PR_OK;
}

pr_status pr_iterate(pr_handle h, int max_steps, int precision, double tol, int* steps_done) {
  if (steps_done) *steps_done = 0;
  if (!h) return fail(nullptr, PR_ESTATE, "pr_iterate: NULL handle");
  if (max_steps < 0 || !(tol >= 0)) return fail(h, PR_EINVAL, "pr_iterate: max_steps < 0 or tol < 0 / NaN");
  pr_status s = check_precision(h, precision);
  if (s != PR_OK) return s;
  cudaSetDevice(h->device);
  s = ensure_state(h, precision);
  if (s != PR_OK) return s;

  const pr::NvtxRange trace_call("pr_iterate");
  int steps = 0;
  int stop = -1;
  while (true) {
    const pr::NvtxRange trace_it(precision == PR_EMU64 ? "iteration EMU64"
                                 : precision == PR_BF16 ? "iteration BF16" : "iteration FP64");
    if (h->form == PR_FORM_NS || h->form == PR_FORM_LITERAL) {
      double r;
      s = h->form == PR_FORM_NS ? ns_residual(h, precision, &r) : literal_residual(h, precision, &r);
      if (s != PR_OK) return s;
      // A repeated call re-evaluates the same iterate: replace its residual instead of appending.
      const bool same_iterate = !h->hist.empty() && (int)h->hist.size() == h->st.iterations + 1;
      push_residual(h, r, precision, same_iterate);
    }
    stop = decide(h, tol, steps, max_steps);
    const bool worse = h->hist.size() >= 2 && !(h->hist.back() < h->hist[h->hist.size() - 2]);  // or not finite
    if ((stop == PR_ESTAGNATED || stop == PR_EDIVERGED) && lowp(precision) && steps > 0 && worse &&
        h->form != PR_FORM_LITERAL) {
      // The last low-precision update made things worse (or overflowed): return to the previous iterate,
      // which the double-buffered state still holds, so that a more precise phase starts from the better
      // one. A low-precision rung that overflows has reached its floor, not diverged.
      stop = PR_ESTAGNATED;
      swap(h->X, h->Xn);
      if (h->form == PR_FORM_COUPLED) {
        swap(h->M, h->Mn);
        swap(h->N, h->Nn);
      }
      h->hist.pop_back();
      h->hist_prec.pop_back();
      h->st.last_residual = h->hist.back();
      h->st.iterations -= 1;
      h->st.iterations_by_precision[precision] -= 1;
      steps -= 1;
    }
    if (stop >= 0) break;
    if (h->st.last_precision >= 0 && h->st.last_precision != precision) h->st.switch_iteration = h->st.iterations;
    if (h->form == PR_FORM_COUPLED) s = coupled_update(h, precision);
    else if (h->form == PR_FORM_NS) s = ns_update(h, precision);
    else s = literal_update(h, precision);
    if (s != PR_OK) return s;
    h->st.iterations += 1;
    h->st.iterations_by_precision[precision] += 1;
    h->st.last_precision = precision;
    ++steps;
  }
  if (steps_done) *steps_done = steps;
  if (stop != PR_EDIVERGED) {
    if (h->form != PR_FORM_COUPLED) {
      h->st.true_residual = h->hist.back();  // the tested residual is the true one
    } else if (h->opt.verify) {
      // The coupled form tested ||I - M||_F; the true residual of the iterate can be far larger when
      // rounding errors carried in M let X drift (Eq. 3's M_0 spans kappa^(p+1)).
      double r = 0.0;
      s = true_residual(h, precision, &r);
      if (s != PR_OK) return s;
      h->st.true_residual = r;
      if (stop == PR_OK && !(r <= tol)) {
        char buf[200];
        snprintf(buf, sizeof buf,
                 "pr_iterate: ||I - M||_F = %.3e met tol = %.3e, but the true residual ||I - X^p A||_F = %.3e does not",
                 h->hist.back(), tol, r);
        h->err = buf;
        stop = PR_EINACCURATE;
      }
    }
  }
  h->st.last_stop = stop;
  if (stop == PR_EDIVERGED) h->err = "pr_iterate: the residual is not finite";
  return (pr_status)stop;
}

int pr_stop_rule(const double* hist, const int* prec, int len, double tol, const pr_options* opt) {
  if (!hist || !prec || len < 1) return PR_EINVAL;
  pr_options o;
  if (opt) o = *opt;
  else pr_default_options(&o);
  return stop_rule(hist, prec, len, tol, o);
}

pr_status pr_solve(pr_handle h, int bulk_precision, int bulk_steps, int final_precision, double tol, int* steps_done) {
  if (steps_done) *steps_done = 0;
  if (!h) return fail(nullptr, PR_ESTATE, "pr_solve: NULL handle");
  int d1 = 0, d2 = 0;
  if (bulk_steps > 0) {
    pr_status s = pr_iterate(h, bulk_steps, bulk_precision, tol, &d1);
    if (steps_done) *steps_done = d1;
    if (s != PR_ESTAGNATED && s != PR_EMAXITER && s != PR_EINACCURATE) return s;
  }
  pr_status s = pr_iterate(h, 1 << 30, final_precision, tol, &d2);
  if (steps_done) *steps_done = d1 + d2;
  return s;
}

pr_status pr_solve_ladder(pr_handle h, int count, const int* precisions, const int* max_steps, double tol,
                          int* steps_done) {
  if (steps_done) *steps_done = 0;
  if (!h) return fail(nullptr, PR_ESTATE, "pr_solve_ladder: NULL handle");
  if (count < 1 || !precisions) return fail(h, PR_EINVAL, "pr_solve_ladder: count < 1 or precisions NULL");
  for (int r = 0; r < count; ++r) {
    pr_status s = check_precision(h, precisions[r]);
    if (s != PR_OK) return s;
  }
  cudaSetDevice(h->device);
  const size_t bytes = (size_t)h->n * (size_t)h->n * sizeof(double);
  // Rung guard. In the coupled form a low-precision rung tests the carried ||I - M||_F, which can keep
  // falling while rounding errors let X drift from M. At each boundary after a rung below FP64 accuracy
  // that hands over to a higher level, the true residual ||I - X^p A||_F is evaluated with the next rung's
  // products; an iterate worse than the best one seen at such a boundary is replaced by that one, and the
  // next rung starts from it (M re-formed from X).
  double best = INFINITY;
  auto restore = [&](const double* from) -> pr_status {
    PR_CK(h, cudaMemcpyAsync(h->X.f, from, bytes, cudaMemcpyDeviceToDevice, h->stream));
    h->X.changed();
    h->lp_stale = true;
    h->state_ready = false;
    h->st.ladder_restores += 1;
    return sync(h);
  };
  auto guard = [&](int next_prec) -> pr_status {
    double r = 0.0;
    pr_status s = true_residual(h, next_prec, &r);
    if (s != PR_OK) return s;
    if (!h->xbest) PR_CK(h, cudaMalloc((void**)&h->xbest, bytes));
    if (r <= best) {  // NaN compares false: never kept
      best = r;
      PR_CK(h, cudaMemcpyAsync(h->xbest, h->X.f, bytes, cudaMemcpyDeviceToDevice, h->stream));
      return sync(h);
    }
    h->st.true_residual = best;  // the restored iterate's, evaluated when it was kept
    return restore(h->xbest);
  };
  // A rung after the first that diverges from the iterate the earlier rungs left (a low-precision rung can
  // leave X^p A indefinite while its Frobenius residual fell) runs once more from the starting iterate.
  bool any_lowp = false;
  for (int r = 0; r + 1 < count; ++r) any_lowp = any_lowp || lowp(precisions[r]);
  if (any_lowp) {
    if (!h->xstart) PR_CK(h, cudaMalloc((void**)&h->xstart, bytes));
    PR_CK(h, cudaMemcpyAsync(h->xstart, h->X.f, bytes, cudaMemcpyDeviceToDevice, h->stream));
  }
  int total = 0;
  pr_status s = PR_EINVAL;
  for (int r = 0; r < count; ++r) {
    // The last rung of a ladder of several is judged with FP64-accurate products.
    const int next = r + 1 < count ? precisions[r + 1] : PR_EMU64;
    const bool guarded = count > 1 && lowp(precisions[r]) && precision_level(next) > precision_level(precisions[r]);
    if (guarded && best == INFINITY) {
      s = guard(next);  // the starting iterate is the first candidate
      if (s != PR_OK) return s;
    }
    int d = 0;
    s = pr_iterate(h, max_steps ? max_steps[r] : (1 << 30), precisions[r], tol, &d);
    total += d;
    if (s == PR_EDIVERGED && r > 0 && any_lowp) {
      s = restore(h->xstart);
      if (s != PR_OK) return s;
      d = 0;
      s = pr_iterate(h, max_steps ? max_steps[r] : (1 << 30), precisions[r], tol, &d);
      total += d;
    }
    if (steps_done) *steps_done = total;
    if (s != PR_ESTAGNATED && s != PR_EMAXITER && s != PR_EINACCURATE) return s;
    if (guarded) {
      pr_status g = guard(next);
      if (g != PR_OK) return g;
    }
  }
  return s;
}

pr_status pr_residual(pr_handle h, int precision, double* res_fro) {
  if (!h) return fail(nullptr, PR_ESTATE, "pr_residual: NULL handle");
  if (!res_fro) return fail(h, PR_EINVAL, "pr_residual: res_fro is NULL");
  if (!precision_known(precision)) return fail(h, PR_EINVAL, "pr_residual: unknown precision");
  cudaSetDevice(h->device);
  return true_residual(h, precision, res_fro);
}

pr_status pr_result(pr_handle h, double* C_out) {
  if (!h) return fail(nullptr, PR_ESTATE, "pr_result: NULL handle");
  if (!C_out) return fail(h, PR_EINVAL, "pr_result: C_out is NULL");
  cudaSetDevice(h->device);
  const size_t bytes = (size_t)h->n * (size_t)h->n * sizeof(double);
  const double* src = h->X.f;
  if (h->st.prescale_log2 != 0) {
    // The handle iterates on 2^k A: A^{-1/p} = 2^(k/p) (2^k A)^{-1/p}, scaled into the scratch product T1.
    PR_CK(h, pr::lincomb(h->X.f, h->X.f, h->n * h->n, exp2((double)h->st.prescale_log2 / h->p), 0.0, h->T1.f,
                         h->stream));
    h->st.launches += 1;
    h->T1.changed();
    h->powers_valid = false;
    src = h->T1.f;
  }
  PR_CK(h, cudaMemcpyAsync(C_out, src, bytes, cudaMemcpyDefault, h->stream));
  return sync(h);
}

pr_status pr_matmul_emu(int slices, const double* X, const double* Y, int64_t n, int sym, double* P, void* stream) {
  if (slices < 1 || slices > pr::emu_max_slices())
    return fail(nullptr, PR_EINVAL, "pr_matmul_emu: slices must be in [1, 8]");
  return matmul(PR_EMU64, slices, X, Y, n, sym, P, stream);
}

pr_status pr_matmul_emu_tiled(int slices, int tile_n, int split, const double* X, const double* Y, int64_t n, int sym,
                              double* P, void* stream) {
  if (slices < 1 || slices > pr::emu_max_slices())
    return fail(nullptr, PR_EINVAL, "pr_matmul_emu_tiled: slices must be in [1, 8]");
  if (!pr::emu_tile_width_ok(tile_n) || split < -1 || split > 1)
    return fail(nullptr, PR_EINVAL, "pr_matmul_emu_tiled: tile_n must be 96 or 48 and split -1, 0 or 1");
  return matmul(PR_EMU64, slices, X, Y, n, sym, P, stream, tile_n, split);
}

pr_status pr_matmul(int precision, const double* X, const double* Y, int64_t n, int sym, double* P, void* stream) {
  return matmul(precision, pr::emu_max_slices(), X, Y, n, sym, P, stream);
}


pr_status pr_features(pr_handle h, double* out) {
  if (!h) return fail(nullptr, PR_ESTATE, "pr_features: NULL handle");
  if (!out) return fail(h, PR_EINVAL, "pr_features: out is NULL");
  cudaSetDevice(h->device);
  const int n = (int)h->n;
  pr_status s = powers_of_A(h);
  if (s == PR_OK) s = ensure_vec(h);
  if (s != PR_OK) return s;
  const int64_t nn = (int64_t)n * n;
  double *work = h->vec + 4 * (size_t)n, *r = work + kVecBlocks;  // r[0..5]: tr A, <A,A>, <A,P2>, ...
  PR_CK(h, pr::trace(h->A.f, n, work, r + 0, h->stream));
  PR_CK(h, pr::frobenius_dot(h->A.f, h->A.f, nn, work, r + 1, h->stream));
  PR_CK(h, pr::frobenius_dot(h->A.f, h->T0.f, nn, work, r + 2, h->stream));
  PR_CK(h, pr::frobenius_dot(h->T0.f, h->T0.f, nn, work, r + 3, h->stream));
  PR_CK(h, pr::frobenius_dot(h->T0.f, h->T1.f, nn, work, r + 4, h->stream));
  PR_CK(h, pr::frobenius_dot(h->T1.f, h->T1.f, nn, work, r + 5, h->stream));
  h->st.launches += 12;
  double t[6];
  PR_CK(h, cudaMemcpyAsync(t, r, sizeof t, cudaMemcpyDeviceToHost, h->stream));
  s = sync(h);
  if (s != PR_OK) return s;
  const double s1 = h->st.norm_1;
  double sk = 1.0;
  for (int k = 0; k < 6; ++k) {
    sk *= s1;
    out[k] = t[k] / sk / n;  // tr(A^{k+1}) / s^{k+1} / n
  }
  out[6] = ldexp(h->st.norm_1, -h->st.prescale_log2);  // the norms of the caller's A
  out[7] = ldexp(h->st.norm_inf, -h->st.prescale_log2);
  return PR_OK;
}

pr_status pr_spectral_bounds(pr_handle h, int iters, double* lam_min, double* lam_max) {
  if (!h) return fail(nullptr, PR_ESTATE, "pr_spectral_bounds: NULL handle");
  if (iters < 1 || !lam_min || !lam_max) return fail(h, PR_EINVAL, "pr_spectral_bounds: iters < 1 or NULL output");
  if (h->st.norm_1 <= 0.0) return fail(h, PR_ESTATE, "pr_spectral_bounds: no matrix loaded");
  cudaSetDevice(h->device);
  pr_status s = ensure_vec(h);
  double na = 0.0, nc = 0.0;
  if (s == PR_OK) s = power_norm(h, h->A.f, iters, &na);
  if (s == PR_OK) s = power_norm(h, h->X.f, iters, &nc);
  if (s != PR_OK) return s;
  // The handle holds 2^k A and its root: lambda_max(A) = ||2^k A||_2 2^-k; the root of A is 2^(k/p) X, so
  // lambda_min(A) = ||2^(k/p) X||_2^(-p) = ||X||_2^(-p) 2^-k.
  *lam_max = ldexp(na, -h->st.prescale_log2);
  *lam_min = ldexp(pow(nc, -(double)h->p), -h->st.prescale_log2);
  return PR_OK;
}

pr_status pr_stats(pr_handle h, pr_stats_t* out) {
  if (!h) return fail(nullptr, PR_ESTATE, "pr_stats: NULL handle");
  if (!out) return fail(h, PR_EINVAL, "pr_stats: out is NULL");
  *out = h->st;
  return PR_OK;
}

pr_status pr_refine(pr_handle h, int precision, int inner_precision, int max_steps, double tol, int cg_max,
                    double cg_tol, int* steps_done) {
  if (steps_done) *steps_done = 0;
  if (!h) return fail(nullptr, PR_ESTATE, "pr_refine: NULL handle");
  if (!precision_known(precision) || !precision_known(inner_precision))
    return fail(h, PR_EINVAL, "pr_refine: unknown precision");
  if (max_steps < 0 || max_steps > PR_REFINE_MAX_STEPS || !(tol >= 0) || cg_max < 1 || !(cg_tol >= 0))
    return fail(h, PR_EINVAL, "pr_refine: max_steps outside [0, PR_REFINE_MAX_STEPS], tol or cg_tol < 0, or cg_max < 1");
  if (h->st.norm_1 <= 0.0) return fail(h, PR_ESTATE, "pr_refine: no matrix loaded");
  if (h->opt.quant_bits > 0) return fail(h, PR_EUNSUPPORTED, "pr_refine: not part of the custom-precision experiment");
  if (h->p > 4) return fail(h, PR_EUNSUPPORTED, "pr_refine: p > 4");
  cudaSetDevice(h->device);
  pr_status s = ensure_refine(h);
  if (s != PR_OK) return s;
  const pr::NvtxRange trace("pr_refine");
  const size_t bytes = (size_t)h->n * (size_t)h->n * sizeof(double);
  // From here on the coupled form's M and N, the scratch products and the BF16 copies are overwritten.
  h->state_ready = false;
  h->lp_stale = true;
  h->powers_valid = false;
  // Only this call's own conversions vouch for a BF16 copy (other paths keep theirs by lp_stale).
  for (Mat* m : {&h->A, &h->X, &h->Xn, &h->M, &h->Mn, &h->N, &h->Nn, &h->T0, &h->T1, &h->Ra, &h->Rb, &h->Rc})
    m->b_valid = false;
  h->st.refine_len = 0;
  int k = 0;
  double gprev = 0.0;
  pr_status stop = PR_OK;
  while (true) {
    const pr::NvtxRange trace_step("refine step");
    RefineOps o;
    double g = 0.0;
    s = refine_setup(h, precision, o);
    if (s == PR_OK) s = refine_residual(h, precision, o, &g);
    if (s != PR_OK) return s;
    h->st.refine_residuals[h->st.refine_len++] = g;
    if (!std::isfinite(g) || (k >= 1 && !(g < gprev))) {
      // The last correction did not help (the precision floor) or overflowed: return to the previous iterate.
      stop = std::isfinite(g) ? PR_ESTAGNATED : PR_EDIVERGED;
      if (k >= 1) {
        PR_CK(h, cudaMemcpyAsync(h->X.f, h->xbest, bytes, cudaMemcpyDeviceToDevice, h->stream));
        h->X.changed();
        h->st.refine_len -= 1;
        k -= 1;
        h->st.refine_steps -= 1;
        h->st.refine_cg_iterations -= h->st.refine_cg[k];
        h->st.refine_cg[k] = 0;
      }
      break;
    }
    if (g <= tol) {
      stop = PR_OK;
      break;
    }
    if (k >= 1 && gprev < h->opt.stag_below && g > h->opt.stag_ratio * gprev) {
      stop = PR_ESTAGNATED;
      break;
    }
    if (k >= max_steps) {
      stop = PR_EMAXITER;
      break;
    }
    int its = 0;
    s = refine_solve(h, inner_precision, o, g, cg_max, cg_tol, &its);
    if (s != PR_OK) return s;
    PR_CK(h, cudaMemcpyAsync(h->xbest, h->X.f, bytes, cudaMemcpyDeviceToDevice, h->stream));
    PR_CK(h, pr::lincomb(h->X.f, h->Mn.f, h->n * h->n, 1.0, 1.0, h->X.f, h->stream));
    h->st.launches += 1;
    h->X.changed();
    h->st.refine_cg[k] = its;
    h->st.refine_steps += 1;
    h->st.refine_cg_iterations += its;
    gprev = g;
    ++k;
  }
  if (steps_done) *steps_done = k;
  for (Mat* m : {&h->X, &h->Xn, &h->M, &h->Mn, &h->N, &h->Nn, &h->T0, &h->T1}) m->changed();
  if (stop != PR_EDIVERGED) {
    double r = 0.0;
    s = true_residual(h, precision, &r);
    if (s != PR_OK) return s;
    h->st.true_residual = r;
    if (stop == PR_OK && !(r <= tol)) {
      char buf[200];
      snprintf(buf, sizeof buf,
               "pr_refine: ||G(X)||_F = %.3e met tol = %.3e, but the true residual ||I - X^p A||_F = %.3e does not",
               h->st.refine_residuals[h->st.refine_len - 1], tol, r);
      h->err = buf;
      stop = PR_EINACCURATE;
    }
  } else {
    h->err = "pr_refine: the residual is not finite";
  }
  h->st.last_stop = stop;
  return stop;
}

pr_status pr_set_iterate(pr_handle h, const double* X) {
  if (!h) return fail(nullptr, PR_ESTATE, "pr_set_iterate: NULL handle");
  if (!X) return fail(h, PR_EINVAL, "pr_set_iterate: X is NULL");
  if (h->st.norm_1 <= 0.0) return fail(h, PR_ESTATE, "pr_set_iterate: no matrix loaded");
  cudaSetDevice(h->device);
  const int n = (int)h->n;
  const size_t bytes = (size_t)n * (size_t)n * sizeof(double);
  PR_CK(h, cudaMemcpyAsync(h->Xn.f, X, bytes, cudaMemcpyDefault, h->stream));
  PR_CK(h, pr::validate(h->Xn.f, n, h->scal, h->stream));
  h->st.launches += 1;
  PR_CK(h, cudaMemcpyAsync(h->hpin, h->scal, 4 * sizeof(double), cudaMemcpyDeviceToHost, h->stream));
  pr_status s = sync(h);
  if (s != PR_OK) return s;
  const double amax = h->hpin[0], asym = h->hpin[1], nonfinite = h->hpin[2], nonpos = h->hpin[3];
  if (nonfinite > 0) return fail(h, PR_EINVAL, "pr_set_iterate: X has non-finite entries");
  if (asym > h->opt.sym_tol * amax) return fail(h, PR_EINVAL, "pr_set_iterate: X is not symmetric");
  if (nonpos > 0) return fail(h, PR_ENOTSPD, "pr_set_iterate: X is not positive definite");
  reset_iteration(h);
  // The handle iterates on 2^k A, whose root is 2^(-k/p) times the root of the caller's A.
  const double c = exp2(-(double)h->st.prescale_log2 / h->p);
  PR_CK(h, pr::lincomb(h->Xn.f, h->Xn.f, (int64_t)n * n, c, 0.0, h->X.f, h->stream));
  h->st.launches += 1;
  h->X.changed();
  h->Xn.changed();
  return sync(h);
}

pr_status pr_history(pr_handle h, double* out, int cap, int* len) {
  if (!h) return fail(nullptr, PR_ESTATE, "pr_history: NULL handle");
  if (len) *len = (int)h->hist.size();
  if (out && cap > 0) {
    const int m = cap < (int)h->hist.size() ? cap : (int)h->hist.size();
    for (int i = 0; i < m; ++i) out[i] = h->hist[i];
  }
  return PR_OK;
}

}  // extern "C"
