// C ABI of the FIRLS library: context, operator set-up and the solve
// orchestration (Alg. 2 FIRLS_OG / Alg. 3 FIRLS_TV).  One outer step (weights,
// preconditioner, PCG initialisation and J PCG steps) is captured once as a
// CUDA graph per (J, tolerances) and replayed K times.
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <algorithm>
#include <functional>
#include <cstring>
#include <string>
#include <vector>

#include "firls.h"
#include "launch.h"

using namespace firls;

struct firls_ctx {
  int n = 0, batch = 0;
  unsigned flags = 0;
  cudaStream_t stream = nullptr;
  int device = 0;
  bool op_set = false;
  unsigned psi = 0;
  int levels = 0, kind = 0;
  int n_groups = 0, gsize = 0, gtotal = 0;
  bool groups = false;
  // multi-contrast images (Sec. 5.6): C consecutive slices are the contrasts
  // of one image, with joint weights and one set of PCG scalars
  int channels = 1;
  // slot mode (firls_run_steps / firls_run): only slots [0, active_slots) are
  // launched (0: all); cur_batch is the batch the launch helpers use (0: all)
  int active_slots = 0;
  int cur_batch = 0;
  // device workspace
  uint8_t* mask = nullptr;
  int* counts = nullptr;
  float2* tw = nullptr;
  float2 *atb = nullptr, *x = nullptr, *r = nullptr, *z = nullptr, *d = nullptr, *q = nullptr;
  float2 *t = nullptr, *u = nullptr, *cw = nullptr, *dx = nullptr, *tmpA = nullptr, *tmpB = nullptr;
  // dx: the update of the current outer step, sum_j alpha_j d_j, accumulated
  // from zero by the PCG steps and added to x once at the end of the step
  float *ww = nullptr, *wtv = nullptr, *ia = nullptr, *wdiag = nullptr;
  float* wtv2 = nullptr;  // l1 TV: the vertical weights W2 (wtv then holds W1)
  float* wg = nullptr;
  int *gidx = nullptr, *goff = nullptr, *inv_off = nullptr, *inv_ids = nullptr;
  int *gcounts = nullptr, *gcursor = nullptr, *gerr = nullptr;
  float* sqtab = nullptr;
  int* sqlen = nullptr;
  // tile shapes (autotuned or defaults)
  int tune_rb = 0, tune_cmax = 0, tune_ilu = 0;  // 0: ILU ring shape chosen from n and batch
  int wait_test = 0;  // failure-detection test: the ILU's bounded waits run out (firls_set_wait_test)
  SliceState* st = nullptr;
  double* part = nullptr;
  float *lam_d = nullptr, *lamtv_d = nullptr;
  std::vector<void*> allocs;
  std::string err;
  // per-kernel timing marks of one outer step
  bool timing = false;
  struct Mark {
    int cls, launches;
    cudaEvent_t a, b;
  };
  std::vector<Mark> marks;
  std::vector<cudaEvent_t> evpool;
  size_t evnext = 0;
  bool marks_valid = false;
  // captured macro-step graphs, by schedule and number of macro steps
  struct CachedGraph {
    firls_params sched;
    int steps;
    int batch;  // slots launched
    cudaGraphExec_t exec;
  };
  std::vector<CachedGraph> graphs;
  bool use_graph = true;
  SliceState* stw = nullptr;  // per macro step: the state with only outer-step starts running
};

namespace {

firls_status fail(firls_ctx* c, firls_status s, const std::string& msg) {
  if (c) c->err = msg;
  return s;
}

firls_status cuda_check(firls_ctx* c, cudaError_t e, const char* what) {
  if (e == cudaSuccess) return FIRLS_OK;
  return fail(c, e == cudaErrorMemoryAllocation ? FIRLS_E_NOMEM : FIRLS_E_CUDA,
              std::string(what) + ": " + cudaGetErrorString(e));
}

template <typename T> firls_status dalloc(firls_ctx* c, T** p, size_t count) {
  void* v = nullptr;
  cudaError_t e = cudaMalloc(&v, count * sizeof(T) + 16);
  if (e != cudaSuccess) return cuda_check(c, e, "cudaMalloc");
  c->allocs.push_back(v);
  *p = static_cast<T*>(v);
  return FIRLS_OK;
}

#define TRY(expr)                        \
  do {                                   \
    firls_status _s = (expr);            \
    if (_s != FIRLS_OK) return _s;       \
  } while (0)
#define CU(expr) TRY(cuda_check(c, (expr), #expr))

// Squared 1-D level-l basis functions of the periodic pyramid (low: scaling
// cascade h*...*h, high: g after l-1 lowpass steps), folded modulo n.
void basis_tables(int n, int levels, int kind, std::vector<float>& tab, std::vector<int>& len) {
  std::vector<double> h, g;
  if (kind == FIRLS_PSI_HAAR) {
    const double r = 1.0 / std::sqrt(2.0);
    h = {r, r};
  } else {
    const double s3 = std::sqrt(3.0), den = 4.0 * std::sqrt(2.0);
    h = {(1 + s3) / den, (3 + s3) / den, (3 - s3) / den, (1 - s3) / den};
  }
  const int K = (int)h.size();
  for (int t = 0; t < K; ++t) g.push_back(((t & 1) ? -1.0 : 1.0) * h[K - 1 - t]);
  tab.assign((size_t)levels * 2 * n, 0.f);
  len.assign((size_t)levels * 2, 0);
  std::vector<double> low(h.begin(), h.end());
  std::vector<double> high(g.begin(), g.end());
  for (int l = 1; l <= levels; ++l) {
    if (l > 1) {
      const int sh = 1 << (l - 1);
      const size_t L = low.size() + (size_t)sh * (K - 1);
      std::vector<double> nl(L, 0.0), nh(L, 0.0);
      for (int t = 0; t < K; ++t)
        for (size_t i = 0; i < low.size(); ++i) {
          nl[i + (size_t)sh * t] += h[t] * low[i];
          nh[i + (size_t)sh * t] += g[t] * low[i];
        }
      low.swap(nl);
      high.swap(nh);
    }
    for (int ty = 0; ty < 2; ++ty) {
      const std::vector<double>& f = ty ? high : low;
      std::vector<double> fold(n, 0.0);
      for (size_t i = 0; i < f.size(); ++i) fold[i % n] += f[i];
      const int ln = (int)std::min<size_t>(f.size(), (size_t)n);
      for (int i = 0; i < n; ++i) tab[(size_t)((l - 1) * 2 + ty) * n + i] = (float)(fold[i] * fold[i]);
      len[(l - 1) * 2 + ty] = ln;
    }
  }
}

// The slots the macro-step launches cover: all of them, or in slot mode the
// first active_slots (the others hold no running slice).
int run_batch(const firls_ctx* c) { return c->cur_batch > 0 ? c->cur_batch : c->batch; }

WavArgs wav_args(firls_ctx* c, const SliceState* st) {
  WavArgs a;
  a.batch = run_batch(c);
  a.n = c->n;
  a.levels = c->levels;
  a.kind = c->kind;
  a.stream = c->stream;
  a.st = st;
  a.tmpA = c->tmpA;
  a.tmpB = c->tmpB;
  a.part = c->part;
  a.rb = c->tune_rb;
  a.coarse_max = c->tune_cmax;
  return a;
}

FftArgs fft_args(firls_ctx* c) {
  FftArgs a;
  a.batch = run_batch(c);
  a.stream = c->stream;
  a.tw = c->tw;
  a.st = c->st;
  a.part = c->part;
  a.real = (c->flags & FIRLS_REAL_X) ? 1 : 0;
  return a;
}

bool has_tv(const firls_ctx* c) { return (c->psi & (FIRLS_PSI_TV | FIRLS_PSI_TV_ANISO)) != 0; }
bool is_aniso(const firls_ctx* c) { return (c->psi & FIRLS_PSI_TV_ANISO) != 0; }
float* tv2_of(const firls_ctx* c) { return is_aniso(c) ? c->wtv2 : nullptr; }

// ---- timing marks: an event pair around each launch group of a class ----
cudaEvent_t next_event(firls_ctx* c) {
  if (c->evnext == c->evpool.size()) {
    cudaEvent_t e = nullptr;
    cudaEventCreate(&e);
    c->evpool.push_back(e);
  }
  return c->evpool[c->evnext++];
}

// Inside a stream capture the events become external event-record nodes of
// the graph (recorded at every replay); outside one they are plain records.
void record_mark(cudaEvent_t e, cudaStream_t s) {
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  if (s != nullptr) cudaStreamIsCapturing(s, &cs);
  if (cs == cudaStreamCaptureStatusActive)
    cudaEventRecordWithFlags(e, s, cudaEventRecordExternal);
  else
    cudaEventRecord(e, s);
}

struct TMark {
  firls_ctx* c;
  int cls, launches;
  cudaEvent_t b = nullptr;
  TMark(firls_ctx* c_, int cls_, int launches_) : c(c_), cls(cls_), launches(launches_) {
    if (!c->timing) return;
    b = next_event(c);
    record_mark(b, c->stream);
  }
  ~TMark() {
    if (!c->timing) return;
    cudaEvent_t e = next_event(c);
    record_mark(e, c->stream);
    c->marks.push_back({cls, launches, b, e});
  }
};

void marks_reset(firls_ctx* c) {
  c->marks.clear();
  c->evnext = 0;
}

// q = S d  (mode 0: d = z; 1: d = z + beta d; 2: d as given; -1: per slice,
// d = x^k for a slice starting its outer step, else z or z + beta d)
void enqueue_S(firls_ctx* c, int mode, const float2* zin, float2* din, float2* q) {
  FftArgs a = fft_args(c);
  a.z = zin;
  a.d = din;
  a.t = c->t;
  a.mode = mode;
  a.xs = c->x;
  { TMark m(c, FIRLS_K_ROW_FFT, 1); fft_row_fwd(c->n, a); }
  a.mask = c->mask;
  { TMark m(c, FIRLS_K_COL_FFT_MASK, 1); fft_col_mask(c->n, a); }
  if (c->kind) {
    WavArgs w = wav_args(c, c->st);
    TMark m(c, FIRLS_K_WAVELET_S, wavelet_apply_launches(c->n, c->levels, c->kind, c->tune_rb, c->tune_cmax));
    wavelet_apply(w, din, c->cw, c->ww, WAV_MUL_W, c->u, nullptr, a.real);
  }
  a.u = c->kind ? c->u : nullptr;
  a.wtv = has_tv(c) ? c->wtv : nullptr;
  a.wtv2 = tv2_of(c);
  a.q = q;
  { TMark m(c, FIRLS_K_ROW_IFFT, 1); fft_row_inv(c->n, a); }
}

// Update W^k and P from x (Alg. 2/3, first two lines of the loop body) for
// the slices that `view` shows running (its other slices read as done).
void enqueue_weights(firls_ctx* c, const float2* x, int precond, const SliceState* view) {
  const int B = run_batch(c), n = c->n;
  TMark mk(c, FIRLS_K_WEIGHTS, 0);
  if (c->kind) {
    WavArgs w = wav_args(c, view);
    if (c->channels > 1) {
      wavelet_forward(w, x, c->cw, nullptr, WAV_RAW);
      joint_wavelet_weights(B, n, c->channels, c->stream, view, c->cw, c->ww);
    } else if (!c->groups) {
      wavelet_forward(w, x, c->cw, c->ww, WAV_SINGLETON_W);
    } else {
      wavelet_forward(w, x, c->cw, nullptr, WAV_RAW);
      group_norms(B, n, c->n_groups, c->stream, view, c->gidx, c->goff, c->gsize, c->cw, c->wg, 0.f);
      group_gather(B, n, c->n_groups, c->stream, view, c->inv_off, c->inv_ids, c->wg, c->ww);
    }
  }
  if (has_tv(c)) {
    // with TV, 1/a of the penta-diagonal P is also 1/diag(S) (the Jacobi scale)
    tv_weights(B, n, c->stream, view, x, c->wtv, tv2_of(c), c->channels);
    if (c->kind) wavelet_diag(B, n, c->levels, c->stream, view, c->ww, c->wdiag, c->sqtab, c->sqlen);
    penta_setup(B, n, c->stream, view, c->wtv, tv2_of(c), c->kind ? c->wdiag : nullptr, c->ia);
    // ILU(0): the pivots of the incomplete factorisation replace 1/a
    if (precond == FIRLS_PRECOND_ILU0) ilu0_pivots(B, n, c->stream, view, c->wtv, tv2_of(c), c->ia);
  } else if (precond == FIRLS_PRECOND_JACOBI) {
    wavelet_diag(B, n, c->levels, c->stream, view, c->ww, c->wdiag, c->sqtab, c->sqlen);
    jacobi_wavelet_setup(B, n, c->stream, view, c->wdiag, c->ia);
  }
}

PcgSched pcg_sched(const firls_params& sc) {
  return PcgSched{sc.pcg_tol, sc.pcg_tol_kind, sc.pcg_iters, sc.pcg_iters_late, sc.outer_late};
}

// alpha inside the ILU kernel (one launch fewer per macro step): the TV
// preconditioners with one contrast per image
bool alpha_in_ilu(const firls_ctx* c, const firls_params& sc) {
  return has_tv(c) && c->channels == 1 &&
         (sc.precond == FIRLS_PRECOND_PAPER || sc.precond == FIRLS_PRECOND_ILU0);
}

// Residual update and z = P^{-1} r, then rho (first residual) or beta and the
// PCG stop.  mode ILU_INIT: the first residual r = A^H b - q for every
// running slice; ILU_PER_SLICE: each slice by its phase.  x updates go to dx.
void enqueue_precond(firls_ctx* c, int mode, const firls_params& sc) {
  const int B = run_batch(c), n = c->n;
  const int real = (c->flags & FIRLS_REAL_X) ? 1 : 0;
  const bool init = mode == ILU_INIT;
  const int am = init ? AXPY_INIT : AXPY_PER_SLICE, sm = init ? SCALARS_INIT : SCALARS_PER_SLICE;
  const PcgSched ps = pcg_sched(sc);
  if (sc.precond == FIRLS_PRECOND_JACOBI || sc.precond == FIRLS_PRECOND_NONE) {
    // Jacobi or none: one fused pass, then the FP64 scalars
    {
      TMark m(c, FIRLS_K_AXPY, 1);
      axpy_diag_step(B, n, c->stream, c->st, c->part, am, c->dx, c->d, c->r, c->q, c->atb,
                     sc.precond == FIRLS_PRECOND_JACOBI ? c->ia : nullptr, c->z);
    }
    TMark m(c, FIRLS_K_SCALARS, 1);
    pcg_scalars(B, c->stream, c->st, c->part, axpy_ctas(n), axpy_ctas(n), sm, ps, c->channels);
    return;
  }
  if (has_tv(c)) {
    // the ILU CTA finishes rho (and beta) from its own sums, unless they are
    // sums over the contrasts of an image
    const bool fuse = c->channels == 1;
    {
      TMark m(c, FIRLS_K_ILU, 1);
      // the tuned ring shape for the whole batch, the default one for the
      // fewer slots of a compacted launch (every shape gives the same sums)
      const int shape = (c->tune_ilu && B == c->batch) ? c->tune_ilu : ilu_default_shape(n, B, is_aniso(c));
      const int alpha_np = (mode == ILU_PER_SLICE && alpha_in_ilu(c, sc)) ? fft_row_ctas(n) : 0;
      ilu_step(B, n, c->stream, c->st, c->part, mode, c->dx, c->d, c->r, c->q, c->atb, c->u, c->z, c->ia, c->wtv,
               shape, fuse ? 1 : 0, ps, c->wait_test, tv2_of(c), alpha_np);
    }
    if (!fuse) {
      TMark m(c, FIRLS_K_SCALARS, 1);
      pcg_scalars(B, c->stream, c->st, c->part, 1, 1, sm, ps, c->channels);
    }
    return;
  }
  {
    TMark m(c, FIRLS_K_AXPY, 1);
    axpy_step(B, n, c->stream, c->st, c->part, am, c->dx, c->d, c->r, c->q, c->atb);
  }
  WavArgs w = wav_args(c, c->st);
  {
    TMark m(c, FIRLS_K_WAVELET_P, wavelet_apply_launches(n, c->levels, c->kind, c->tune_rb, c->tune_cmax));
    wavelet_apply(w, c->r, c->cw, c->ww, WAV_MUL_PINV, c->z, c->r, real);
  }
  TMark m(c, FIRLS_K_SCALARS, 1);
  const int np = wavelet_apply_ctas(n, c->levels, c->kind, c->tune_rb, c->tune_cmax);
  pcg_scalars(B, c->stream, c->st, c->part, np, axpy_ctas(n), sm, ps, c->channels);
}

// One macro step: every slice advances by one step of its own outer step.
// In a boundary stage, slices whose PCG ended (PH_END) add their update to
// x, measure the relative change and either stop or make their next outer
// step due, and slices whose outer step is due (PH_BOUNDARY) update W^k and
// P.  Then slices with W^k and P ready (PH_START) apply S to x^k and form
// r_0, z_0, rho, and the others take one PCG step (Alg. 2 / Alg. 3).  With a
// boundary stage in every macro step, an outer step with J PCG steps spans
// J + 1 macro steps; with one every P macro steps a slice waits at most
// P - 1 macro steps per outer step.
void enqueue_macro(firls_ctx* c, const firls_params& sc, bool boundary_stage = true) {
  const int B = run_batch(c), n = c->n;
  if (boundary_stage) {
    {
      TMark m(c, FIRLS_K_OTHER, 3);
      outer_apply(B, n, c->stream, c->st, c->x, c->dx, c->part);
      // the plateau stop needs a whole contraction window of nearly exact inner solves
      const int plateau_after = sc.pcg_iters_late > 0 ? sc.outer_late + MU_WINDOW : 1 << 30;
      outer_end(B, c->stream, c->st, c->part, axpy_ctas(n), sc.outer_tol, sc.outer_tol_kind, sc.outer_stall_tol,
                plateau_after, c->channels);
      boundary_view(B, c->stream, c->st, c->stw);
    }
    enqueue_weights(c, c->x, sc.precond, c->stw);
  }
  enqueue_S(c, -1, c->z, c->d, c->q);
  if (!alpha_in_ilu(c, sc)) {
    TMark m(c, FIRLS_K_SCALARS, 1);
    pcg_alpha(B, c->stream, c->st, c->part, fft_row_ctas(n), c->channels);
  }
  enqueue_precond(c, ILU_PER_SLICE, sc);
}

int period_of(const firls_params& sc) { return sc.boundary_period > 1 ? sc.boundary_period : 1; }

// Two parameter sets capture the same macro-step graph (everything but the
// outer count and the lambdas, which live in device memory).
bool same_schedule(const firls_params& a, const firls_params& b) {
  return a.pcg_iters == b.pcg_iters && a.pcg_tol == b.pcg_tol && a.outer_tol == b.outer_tol &&
         a.outer_tol_kind == b.outer_tol_kind && a.precond == b.precond && a.outer_stall_tol == b.outer_stall_tol &&
         a.pcg_tol_kind == b.pcg_tol_kind && a.pcg_iters_late == b.pcg_iters_late && a.outer_late == b.outer_late &&
         period_of(a) == period_of(b);
}

firls_status check_params(firls_ctx* c, const firls_params* p) {
  if (!p) return fail(c, FIRLS_E_INVALID_ARG, "params is null");
  if (p->outer_iters < 1 || p->pcg_iters < 1) return fail(c, FIRLS_E_INVALID_ARG, "iteration counts must be >= 1");
  if (!(p->pcg_tol >= 0.f) || !(p->outer_tol >= 0.f)) return fail(c, FIRLS_E_INVALID_ARG, "tolerances must be >= 0");
  if (p->outer_tol_kind != 0 && p->outer_tol_kind != 1) return fail(c, FIRLS_E_INVALID_ARG, "bad outer_tol_kind");
  if (p->precond < FIRLS_PRECOND_PAPER || p->precond > FIRLS_PRECOND_ILU0)
    return fail(c, FIRLS_E_INVALID_ARG, "bad precond");
  if (p->precond == FIRLS_PRECOND_ILU0 && !has_tv(c))
    return fail(c, FIRLS_E_INVALID_ARG, "ILU(0) factors the TV preconditioner: needs FIRLS_PSI_TV or TV_ANISO");
  if (!(p->outer_stall_tol >= 0.f)) return fail(c, FIRLS_E_INVALID_ARG, "outer_stall_tol must be >= 0");
  if (p->pcg_tol_kind != 0 && p->pcg_tol_kind != 1) return fail(c, FIRLS_E_INVALID_ARG, "bad pcg_tol_kind");
  if (p->pcg_iters_late < 0 || p->outer_late < 0) return fail(c, FIRLS_E_INVALID_ARG, "bad late inner schedule");
  if (p->boundary_period < 0 || p->boundary_period > 64) return fail(c, FIRLS_E_INVALID_ARG, "bad boundary_period");
  const int B = c->batch;
  for (int s = 0; s < B; ++s) {
    const float l = p->lambda_per_slice ? p->lambda_per_slice[s] : p->lambda;
    const float lt = p->lambda_tv_per_slice ? p->lambda_tv_per_slice[s] : p->lambda_tv;
    if (!(l >= 0.f) || !std::isfinite(l)) return fail(c, FIRLS_E_INVALID_ARG, "lambda must be finite and >= 0");
    if (!(lt >= 0.f) || !std::isfinite(lt)) return fail(c, FIRLS_E_INVALID_ARG, "lambda_tv must be finite and >= 0");
    const int s0 = s - s % c->channels;
    if (s != s0) {  // one regulariser per multi-contrast image
      const float l0 = p->lambda_per_slice ? p->lambda_per_slice[s0] : p->lambda;
      const float lt0 = p->lambda_tv_per_slice ? p->lambda_tv_per_slice[s0] : p->lambda_tv;
      if (l != l0 || lt != lt0)
        return fail(c, FIRLS_E_INVALID_ARG, "the contrasts of an image must share lambda and lambda_tv");
    }
  }
  return FIRLS_OK;
}

firls_status upload_params(firls_ctx* c, const firls_params* p) {
  const int B = c->batch;
  std::vector<float> l(B), lt(B);
  for (int s = 0; s < B; ++s) {
    l[s] = p->lambda_per_slice ? p->lambda_per_slice[s] : p->lambda;
    lt[s] = has_tv(c) ? (p->lambda_tv_per_slice ? p->lambda_tv_per_slice[s] : p->lambda_tv) : 0.f;
    if (!c->kind) l[s] = 0.f;
  }
  CU(cudaMemcpyAsync(c->lam_d, l.data(), sizeof(float) * B, cudaMemcpyHostToDevice, c->stream));
  CU(cudaMemcpyAsync(c->lamtv_d, lt.data(), sizeof(float) * B, cudaMemcpyHostToDevice, c->stream));
  // pageable copies: make sure the host vectors may go out of scope
  CU(cudaStreamSynchronize(c->stream));
  return FIRLS_OK;
}

float eps_of(const firls_params* p) { return p->eps > 0.f ? p->eps : 1e-10f; }

// A^H b into atb (and x when x0 is null), ||A^H b||^2 partials, state init
// (every slice at the start of its first outer step, at most outer_max outer
// steps), dx cleared.
firls_status enqueue_setup(firls_ctx* c, const void* b, const firls_params* p, const void* x0) {
  const int B = c->batch, n = c->n;
  TRY(upload_params(c, p));
  FftArgs a = fft_args(c);
  a.b = static_cast<const float2*>(b);
  a.mask = c->mask;
  a.t = c->t;
  fft_row_ahb(n, a);
  a.atb = c->atb;
  a.x = x0 ? nullptr : c->x;
  fft_col_inv(n, a);
  if (x0) {
    CU(cudaMemcpyAsync(c->x, x0, sizeof(float2) * (size_t)B * n * n, cudaMemcpyDeviceToDevice, c->stream));
  }
  CU(cudaMemsetAsync(c->dx, 0, sizeof(float2) * (size_t)B * n * n, c->stream));
  state_init(B, c->stream, c->st, c->part, fft_col_ctas(n), c->counts, n, c->lam_d, c->lamtv_d, eps_of(p),
             p->outer_iters, PH_BOUNDARY, c->channels);
  return cuda_check(c, cudaGetLastError(), "setup launch");
}

void graphs_clear(firls_ctx* c) {
  for (auto& g : c->graphs)
    if (g.exec) cudaGraphExecDestroy(g.exec);
  c->graphs.clear();
}

// The graph of `steps` macro steps for this schedule (captured on first use;
// with timing on, the marks of its last capture are the ones read back).
firls_status macro_graph(firls_ctx* c, const firls_params& sc, int steps, cudaGraphExec_t* out) {
  for (auto& g : c->graphs)
    if (g.steps == steps && g.batch == run_batch(c) && same_schedule(g.sched, sc)) {
      *out = g.exec;
      return FIRLS_OK;
    }
  if (c->timing) marks_reset(c);
  cudaGraph_t g = nullptr;
  CU(cudaStreamBeginCapture(c->stream, cudaStreamCaptureModeThreadLocal));
  for (int i = 0; i < steps; ++i) enqueue_macro(c, sc, i % period_of(sc) == 0);
  cudaError_t e = cudaStreamEndCapture(c->stream, &g);
  if (e != cudaSuccess) return cuda_check(c, e, "graph capture");
  cudaGraphExec_t ex = nullptr;
  e = cudaGraphInstantiate(&ex, g, 0);
  cudaGraphDestroy(g);
  if (e != cudaSuccess) return cuda_check(c, e, "graph instantiate");
  c->graphs.push_back({sc, steps, run_batch(c), ex});
  *out = ex;
  return FIRLS_OK;
}

// Every slice of c stopped?  Reads the state on `s` (default: c's stream).
bool all_done(firls_ctx* c, bool* ok, cudaStream_t s = nullptr) {
  if (!s) s = c->stream;
  std::vector<SliceState> hs(c->batch);
  *ok = cudaMemcpyAsync(hs.data(), c->st, sizeof(SliceState) * c->batch, cudaMemcpyDeviceToHost, s) ==
            cudaSuccess &&
        cudaStreamSynchronize(s) == cudaSuccess;
  for (const SliceState& v : hs)
    if (v.active && !v.done) return false;
  return true;
}

// Enqueue `total` macro steps as replays of a graph of `chunk` macro steps
// (then single-step replays for the remainder).  With poll, the per-slice
// done flags are read every kPoll chunks and the loop stops once every slice
// has stopped.
firls_status run_macro(firls_ctx* c, const firls_params& sc, long total, int chunk, bool poll) {
  const bool graph = c->use_graph && c->stream != nullptr;
  if (chunk < 1) chunk = 1;
  if (chunk > total) chunk = (int)(total > 0 ? total : 1);
  if (!graph) {  // marks of the first chunk only, as with the graphs
    const bool t = c->timing;
    if (t) marks_reset(c);
    for (long k = 0; k < total; ++k) {
      if (k == chunk) c->timing = false;
      enqueue_macro(c, sc, k % period_of(sc) == 0);
    }
    c->timing = t;
    c->marks_valid = t;
    return cuda_check(c, cudaGetLastError(), "macro step launch");
  }
  cudaGraphExec_t ex = nullptr, ex1 = nullptr;
  TRY(macro_graph(c, sc, chunk, &ex));
  const long full = total / chunk, rem = total % chunk;
  const int kPoll = 4;
  for (long k = 0; k < full; ++k) {
    CU(cudaGraphLaunch(ex, c->stream));
    if (poll && (k + 1) % kPoll == 0 && (k + 1 < full || rem)) {
      bool ok = true;
      const bool done = all_done(c, &ok);
      if (!ok) return fail(c, FIRLS_E_CUDA, "state read-back failed");
      if (done) return FIRLS_OK;
    }
  }
  if (rem) {
    const bool t = c->timing;
    c->timing = false;  // the marks stay those of the chunk graph
    firls_params one = sc;
    one.boundary_period = 1;  // single steps: each with its boundary stage
    const firls_status s = macro_graph(c, one, 1, &ex1);
    c->timing = t;
    TRY(s);
    for (long k = 0; k < rem; ++k) CU(cudaGraphLaunch(ex1, c->stream));
  }
  c->marks_valid = c->timing;
  return FIRLS_OK;
}

// Macro steps of params->outer_iters outer steps: (J_k + 1) for outer step k
// and one more that applies the last one; without tolerances every slice
// finishes exactly then.
long solve_steps(const firls_params* p) {
  const int P = period_of(*p);
  long n = P;  // the boundary stage that applies the last outer step comes within P steps
  for (int k = 0; k < p->outer_iters; ++k)
    n += P + ((p->pcg_iters_late > 0 && k >= p->outer_late) ? p->pcg_iters_late : p->pcg_iters);
  return n;
}
bool has_tolerances(const firls_params* p) {
  return p->pcg_tol > 0.f || p->outer_tol > 0.f || p->outer_stall_tol > 0.f || period_of(*p) > 1;
}

firls_status collect_stats(firls_ctx* c, firls_stats* stats, bool* breakdown) {
  std::vector<SliceState> hs(c->batch);
  CU(cudaMemcpyAsync(hs.data(), c->st, sizeof(SliceState) * c->batch, cudaMemcpyDeviceToHost, c->stream));
  CU(cudaStreamSynchronize(c->stream));
  firls_stats s{};
  int faults = 0;
  for (const SliceState& v : hs) {
    s.outer_done = v.outer_done > s.outer_done ? v.outer_done : s.outer_done;
    s.pcg_steps += v.pcg_steps;
    if (v.relchg > s.max_rel_change) s.max_rel_change = v.relchg;
    const double rr = v.rhs2 > 0 ? std::sqrt(v.rr / v.rhs2) : 0.0;
    if (rr > s.max_rel_residual) s.max_rel_residual = rr;
    s.n_breakdown += v.breakdown ? 1 : 0;
    faults += v.fault ? 1 : 0;
  }
  if (stats) *stats = s;
  *breakdown = s.n_breakdown > 0;
  if (faults) return fail(c, FIRLS_E_DEVICE_TIMEOUT, "a bounded device wait ran out in " + std::to_string(faults) +
                                                         " slice(s); their results are invalid");
  return FIRLS_OK;
}

void prepare_kernels(int n);

}  // namespace

// ======================================================================= ABI

struct MultiGraph {
  std::vector<firls_ctx*> ctxs;
  firls_params sched{};
  cudaGraphExec_t exec = nullptr;
};
static MultiGraph g_multi;  // last multi-context graph (per process)

static void multi_forget(firls_ctx* c) {
  if (std::find(g_multi.ctxs.begin(), g_multi.ctxs.end(), c) != g_multi.ctxs.end()) {
    if (g_multi.exec) cudaGraphExecDestroy(g_multi.exec);
    g_multi.exec = nullptr;
    g_multi.ctxs.clear();
  }
}

extern "C" int firls_size_supported(int n) { return fft_size_supported(n) ? 1 : 0; }

extern "C" firls_status firls_create(firls_ctx** out, int n_rows, int n_cols, int batch, unsigned flags,
                                     void* cuda_stream) {
  if (!out) return FIRLS_E_INVALID_ARG;
  *out = nullptr;
  if (n_rows != n_cols || !fft_size_supported(n_rows)) return FIRLS_E_SHAPE;
  if (batch < 1 || batch > 65535) return FIRLS_E_INVALID_ARG;
  firls_ctx* c = new firls_ctx();
  c->n = n_rows;
  c->batch = batch;
  c->flags = flags;
  c->stream = static_cast<cudaStream_t>(cuda_stream);
  c->use_graph = std::getenv("FIRLS_NO_GRAPH") == nullptr;
  cudaGetDevice(&c->device);
  const int n = c->n;
  const size_t N = (size_t)n * n, BN = N * batch, BH = (size_t)batch * (n / 2) * (n / 2);
  firls_status s = FIRLS_OK;
  auto A = [&](auto** p, size_t cnt) {
    if (s == FIRLS_OK) s = dalloc(c, p, cnt);
  };
  A(&c->mask, BN);
  A(&c->counts, (size_t)batch);
  A(&c->tw, (size_t)n);
  for (float2** p : {&c->atb, &c->x, &c->r, &c->z, &c->d, &c->q, &c->t, &c->u, &c->cw, &c->dx}) A(p, BN);
  A(&c->tmpA, BH);
  A(&c->tmpB, BH);
  for (float** p : {&c->ww, &c->wtv, &c->ia, &c->wdiag, &c->wtv2}) A(p, BN);
  A(&c->st, (size_t)batch);
  A(&c->stw, (size_t)batch);
  A(&c->part, (size_t)batch * NSLOT * MAXPART);
  A(&c->lam_d, (size_t)batch);
  A(&c->lamtv_d, (size_t)batch);
  if (s != FIRLS_OK) {
    firls_destroy(c);
    return s;
  }
  std::vector<float2> tw(n);
  for (int j = 0; j < n; ++j) {
    const double ang = -2.0 * 3.14159265358979323846 * (double)j / (double)n;
    tw[j] = make_float2((float)std::cos(ang), (float)std::sin(ang));
  }
  cudaMemcpy(c->tw, tw.data(), sizeof(float2) * n, cudaMemcpyHostToDevice);
  // d is read (times 0) nowhere, but keep the workspace finite
  cudaMemset(c->d, 0, sizeof(float2) * BN);
  cudaMemset(c->part, 0, sizeof(double) * batch * NSLOT * MAXPART);
  // slots that are never loaded read as idle: nothing running, no steps
  cudaMemset(c->st, 0, sizeof(SliceState) * batch);
  prepare_kernels(n);
  if (cudaDeviceSynchronize() != cudaSuccess || cudaGetLastError() != cudaSuccess) {
    firls_destroy(c);
    return FIRLS_E_CUDA;
  }
  *out = c;
  return FIRLS_OK;
}

extern "C" firls_status firls_set_operator(firls_ctx* c, const uint8_t* mask, unsigned psi_kind,
                                           int wavelet_levels, const int32_t* group_idx,
                                           const int32_t* group_off, int n_groups, int group_size) {
  if (!c) return FIRLS_E_INVALID_ARG;
  if (!mask) return fail(c, FIRLS_E_INVALID_ARG, "mask is null");
  const int n = c->n;
  const bool haar = psi_kind & FIRLS_PSI_HAAR, db4 = psi_kind & FIRLS_PSI_DB4;
  const bool both_tv = (psi_kind & FIRLS_PSI_TV) && (psi_kind & FIRLS_PSI_TV_ANISO);
  if ((psi_kind & ~15u) || (haar && db4) || both_tv || psi_kind == 0)
    return fail(c, FIRLS_E_INVALID_ARG,
                "psi_kind must be HAAR or DB4, optionally with TV or TV_ANISO, or one TV form alone");
  const int kind = haar ? 1 : (db4 ? 2 : 0);
  if (kind) {
    if (wavelet_levels < 1 || (n % (1 << wavelet_levels)) || (n >> (wavelet_levels - 1)) < 2)
      return fail(c, FIRLS_E_SHAPE, "n must be divisible by 2^levels, levels >= 1");
  }
  if (group_idx && !kind) return fail(c, FIRLS_E_INVALID_ARG, "groups need a wavelet");
  if (c->channels > 1 && (group_idx || (psi_kind & FIRLS_PSI_TV_ANISO)))
    return fail(c, FIRLS_E_INVALID_ARG, "multi-contrast images take singleton joint groups and isotropic joint TV");
  if (group_idx && (n_groups < 1 || (!group_off && group_size < 1)))
    return fail(c, FIRLS_E_INVALID_ARG, "bad group counts");
  const int B = c->batch;
  const size_t N = (size_t)n * n;
  c->op_set = false;  // until every check below has passed
  CU(cudaMemcpyAsync(c->mask, mask, N * B, cudaMemcpyDeviceToDevice, c->stream));
  CU(cudaMemsetAsync(c->counts, 0, sizeof(int) * B, c->stream));
  mask_popcount(B, n, c->stream, c->mask, c->counts);
  {  // an empty mask (abar = 0, A = 0) leaves nothing to reconstruct: rejected
    std::vector<int> hc(B);
    CU(cudaMemcpyAsync(hc.data(), c->counts, sizeof(int) * B, cudaMemcpyDeviceToHost, c->stream));
    CU(cudaStreamSynchronize(c->stream));
    for (int s = 0; s < B; ++s)
      if (hc[s] <= 0) return fail(c, FIRLS_E_INVALID_ARG, "empty mask in slice " + std::to_string(s));
  }
  c->groups = false;
  if (group_idx) {
    int total = 0;
    if (group_off) {
      CU(cudaMemcpyAsync(&total, group_off + n_groups, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
      CU(cudaStreamSynchronize(c->stream));
    } else {
      total = n_groups * group_size;
    }
    if (total < 0) return fail(c, FIRLS_E_GROUPMAP, "negative member count");
    // (re)allocate the map buffers
    auto rel = [&](void* p) {
      if (!p) return;
      cudaFree(p);
      for (auto& a : c->allocs)
        if (a == p) a = nullptr;
    };
    rel(c->gidx);
    rel(c->goff);
    rel(c->inv_off);
    rel(c->inv_ids);
    rel(c->gcounts);
    rel(c->gcursor);
    rel(c->gerr);
    rel(c->wg);
    c->gidx = c->goff = nullptr;
    TRY(dalloc(c, &c->gidx, (size_t)total));
    if (group_off) TRY(dalloc(c, &c->goff, (size_t)n_groups + 1));
    TRY(dalloc(c, &c->inv_off, N + 1));
    TRY(dalloc(c, &c->inv_ids, (size_t)total));
    TRY(dalloc(c, &c->gcounts, N));
    TRY(dalloc(c, &c->gcursor, N));
    TRY(dalloc(c, &c->gerr, 1));
    TRY(dalloc(c, &c->wg, (size_t)n_groups * B));
    CU(cudaMemcpyAsync(c->gidx, group_idx, sizeof(int) * total, cudaMemcpyDeviceToDevice, c->stream));
    if (group_off)
      CU(cudaMemcpyAsync(c->goff, group_off, sizeof(int) * (n_groups + 1), cudaMemcpyDeviceToDevice, c->stream));
    CU(cudaMemsetAsync(c->gcounts, 0, sizeof(int) * N, c->stream));
    CU(cudaMemsetAsync(c->gcursor, 0, sizeof(int) * N, c->stream));
    CU(cudaMemsetAsync(c->gerr, 0, sizeof(int), c->stream));
    group_inverse_build(n, n_groups, group_size, c->stream, c->gidx, c->goff, c->gcounts, c->inv_off,
                        c->inv_ids, c->gcursor, c->gerr);
    int herr = 0;
    CU(cudaMemcpyAsync(&herr, c->gerr, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
    CU(cudaStreamSynchronize(c->stream));
    if (herr) return fail(c, FIRLS_E_GROUPMAP, "group index outside [0, n*n) or decreasing offsets");
    c->groups = true;
    c->n_groups = n_groups;
    c->gsize = group_size;
    c->gtotal = total;
  }
  if (kind) {  // squared basis tables of diag(Phi^T W Phi) (TV preconditioner, Jacobi)
    std::vector<float> tab;
    std::vector<int> len;
    basis_tables(n, wavelet_levels, kind == 1 ? FIRLS_PSI_HAAR : FIRLS_PSI_DB4, tab, len);
    if (c->sqtab) {
      cudaFree(c->sqtab);
      cudaFree(c->sqlen);
      for (auto& a : c->allocs)
        if (a == c->sqtab || a == c->sqlen) a = nullptr;
    }
    TRY(dalloc(c, &c->sqtab, tab.size()));
    TRY(dalloc(c, &c->sqlen, len.size()));
    CU(cudaMemcpy(c->sqtab, tab.data(), sizeof(float) * tab.size(), cudaMemcpyHostToDevice));
    CU(cudaMemcpy(c->sqlen, len.data(), sizeof(int) * len.size(), cudaMemcpyHostToDevice));
  }
  c->psi = psi_kind;
  c->kind = kind;
  c->levels = kind ? wavelet_levels : 0;
  multi_forget(c);
  graphs_clear(c);
  CU(cudaStreamSynchronize(c->stream));
  CU(cudaGetLastError());
  c->op_set = true;
  return FIRLS_OK;
}

extern "C" firls_status firls_solve(firls_ctx* c, const void* b, const firls_params* p, const void* x0,
                                    void* x_out, firls_stats* stats) {
  if (!c) return FIRLS_E_INVALID_ARG;
  if (!c->op_set) return fail(c, FIRLS_E_STATE, "firls_set_operator has not been called");
  if (!b || !x_out) return fail(c, FIRLS_E_INVALID_ARG, "b and x_out must be non-null");
  TRY(check_params(c, p));
  TRY(enqueue_setup(c, b, p, x0));
  TRY(run_macro(c, *p, solve_steps(p), p->pcg_iters + 1, has_tolerances(p)));
  const size_t bytes = sizeof(float2) * (size_t)c->batch * c->n * c->n;
  CU(cudaMemcpyAsync(x_out, c->x, bytes, cudaMemcpyDeviceToDevice, c->stream));
  CU(cudaGetLastError());
  if (stats || p->pcg_tol > 0.f || p->outer_tol > 0.f) {
    bool bd = false;
    TRY(collect_stats(c, stats, &bd));
    if (bd) return fail(c, FIRLS_E_BREAKDOWN, "PCG breakdown in at least one slice");
  }
  return FIRLS_OK;
}

// Several contexts (different sizes) in one CUDA graph per outer step: the
// capture forks from ctxs[0]'s stream to every context's stream, each
// context enqueues its outer step on its own stream, and the streams join
// back.  Graph replays are launched on ctxs[0]'s stream.

extern "C" firls_status firls_solve_multi(firls_ctx* const* ctxs, int n_ctx, const void* const* b,
                                          const firls_params* pa, const void* const* x0, void* const* x_out,
                                          firls_stats* stats) {
  if (!ctxs || n_ctx < 1 || !b || !x_out || !pa) return FIRLS_E_INVALID_ARG;
  const firls_params* p = &pa[0];  // the schedule (counts, tolerances) shared by all contexts
  bool graphable = true;
  for (int i = 0; i < n_ctx; ++i) {
    firls_ctx* c = ctxs[i];
    if (!c || !c->op_set) return FIRLS_E_STATE;
    TRY(check_params(c, &pa[i]));
    if (pa[i].outer_iters != p->outer_iters || !same_schedule(pa[i], *p))
      return fail(c, FIRLS_E_INVALID_ARG, "solve_multi: contexts must share the schedule and tolerances");
    if (!c->stream || !c->use_graph) graphable = false;
    for (int j = 0; j < i; ++j)
      if (ctxs[j] == c || (ctxs[j]->stream == c->stream && c->stream)) graphable = false;
  }
  firls_ctx* c0 = ctxs[0];
  cudaEvent_t fork = nullptr;
  std::vector<cudaEvent_t> join(n_ctx, nullptr);
  cudaEventCreateWithFlags(&fork, cudaEventDisableTiming);
  for (auto& e : join) cudaEventCreateWithFlags(&e, cudaEventDisableTiming);
  auto cleanup = [&]() {
    cudaEventDestroy(fork);
    for (auto e : join) cudaEventDestroy(e);
  };
  // set-up of every context (A^H b, state), ordered after c0's prior work
  cudaEventRecord(fork, c0->stream);
  for (int i = 0; i < n_ctx; ++i) {
    firls_ctx* c = ctxs[i];
    if (i > 0) cudaStreamWaitEvent(c->stream, fork, 0);
    firls_status st = enqueue_setup(c, b[i], &pa[i], x0 ? x0[i] : nullptr);
    if (st != FIRLS_OK) {
      cleanup();
      return st;
    }
  }
  const int chunk = p->pcg_iters + 1;  // macro steps of one outer step
  if (!graphable) {
    const long total = solve_steps(p);
    for (long k = 0; k < total; ++k)
      for (int i = 0; i < n_ctx; ++i) enqueue_macro(ctxs[i], *p, k % period_of(*p) == 0);
  } else {
    const bool same = g_multi.exec && same_schedule(g_multi.sched, *p) && (int)g_multi.ctxs.size() == n_ctx &&
                      std::equal(g_multi.ctxs.begin(), g_multi.ctxs.end(), ctxs);
    // every context's set-up must precede the replays on c0's stream
    for (int i = 1; i < n_ctx; ++i) {
      cudaEventRecord(join[i], ctxs[i]->stream);
      cudaStreamWaitEvent(c0->stream, join[i], 0);
    }
    if (!same) {
      if (g_multi.exec) cudaGraphExecDestroy(g_multi.exec);
      g_multi.exec = nullptr;
      cudaGraph_t g = nullptr;
      cudaError_t e = cudaStreamBeginCapture(c0->stream, cudaStreamCaptureModeThreadLocal);
      if (e != cudaSuccess) {
        cleanup();
        return cuda_check(c0, e, "multi capture");
      }
      cudaEventRecord(fork, c0->stream);
      for (int i = 1; i < n_ctx; ++i) cudaStreamWaitEvent(ctxs[i]->stream, fork, 0);
      for (int i = 0; i < n_ctx; ++i) {
        if (ctxs[i]->timing) marks_reset(ctxs[i]);
        for (int k = 0; k < chunk; ++k) enqueue_macro(ctxs[i], *p, k % period_of(*p) == 0);
      }
      for (int i = 1; i < n_ctx; ++i) {
        cudaEventRecord(join[i], ctxs[i]->stream);
        cudaStreamWaitEvent(c0->stream, join[i], 0);
      }
      e = cudaStreamEndCapture(c0->stream, &g);
      if (e != cudaSuccess) {
        cleanup();
        return cuda_check(c0, e, "multi capture end");
      }
      e = cudaGraphInstantiate(&g_multi.exec, g, 0);
      cudaGraphDestroy(g);
      if (e != cudaSuccess) {
        g_multi.exec = nullptr;
        cleanup();
        return cuda_check(c0, e, "multi instantiate");
      }
      g_multi.ctxs.assign(ctxs, ctxs + n_ctx);
      g_multi.sched = *p;
    }
    // replays of one outer step's worth of macro steps, then the remaining
    // steps (the last one applies every context's last outer step); with
    // tolerances, stop once every slice of every context has stopped
    const long total = solve_steps(p), full = (total - 1) / chunk;
    long rem = total - full * chunk;
    const bool poll = has_tolerances(p);
    for (long k = 0; k < full; ++k) {
      cudaError_t e = cudaGraphLaunch(g_multi.exec, c0->stream);
      if (e != cudaSuccess) {
        cleanup();
        return cuda_check(c0, e, "multi graph launch");
      }
      if (poll && (k + 1) % 4 == 0) {
        bool all = true, ok = true;
        for (int i = 0; i < n_ctx && all; ++i) all = all_done(ctxs[i], &ok, c0->stream) && ok;
        if (!ok) {
          cleanup();
          return fail(c0, FIRLS_E_CUDA, "state read-back failed");
        }
        if (all) {
          rem = 0;
          break;
        }
      }
    }
    if (rem > 0) {
      cudaEventRecord(fork, c0->stream);
      for (int i = 0; i < n_ctx; ++i) {
        firls_ctx* c = ctxs[i];
        if (i > 0) cudaStreamWaitEvent(c->stream, fork, 0);
        const bool t = c->timing;
        c->timing = false;
        for (long k = 0; k < rem; ++k) enqueue_macro(c, *p);  // each with its boundary stage
        c->timing = t;
        c->marks_valid = t;
        if (i > 0) {
          cudaEventRecord(join[i], c->stream);
          cudaStreamWaitEvent(c0->stream, join[i], 0);
        }
      }
    }
  }
  // results, on c0's stream after the replays; other streams wait for them
  for (int i = 0; i < n_ctx; ++i) {
    firls_ctx* c = ctxs[i];
    const size_t bytes = sizeof(float2) * (size_t)c->batch * c->n * c->n;
    cudaStream_t s = graphable ? c0->stream : c->stream;
    cudaMemcpyAsync(x_out[i], c->x, bytes, cudaMemcpyDeviceToDevice, s);
  }
  if (!graphable)
    for (int i = 1; i < n_ctx; ++i) {
      cudaEventRecord(join[i], ctxs[i]->stream);
      cudaStreamWaitEvent(c0->stream, join[i], 0);
    }
  cudaEventRecord(fork, c0->stream);
  for (int i = 1; i < n_ctx; ++i) cudaStreamWaitEvent(ctxs[i]->stream, fork, 0);
  firls_status ret = cuda_check(c0, cudaGetLastError(), "solve_multi");
  if (ret == FIRLS_OK && (stats || p->pcg_tol > 0.f || p->outer_tol > 0.f)) {
    for (int i = 0; i < n_ctx; ++i) {
      bool bd = false;
      firls_status s = collect_stats(ctxs[i], stats ? &stats[i] : nullptr, &bd);
      if (s != FIRLS_OK) ret = s;
      if (bd && ret == FIRLS_OK) ret = FIRLS_E_BREAKDOWN;
    }
  }
  cleanup();
  return ret;
}

extern "C" const char* firls_last_error(const firls_ctx* c) { return c ? c->err.c_str() : "null context"; }

extern "C" firls_status firls_set_timing(firls_ctx* c, int enable) {
  if (!c) return FIRLS_E_INVALID_ARG;
  multi_forget(c);
  const bool on = enable != 0;
  if (on != c->timing) graphs_clear(c);  // the captured graphs change shape
  c->timing = on;
  c->marks_valid = false;
  return FIRLS_OK;
}

extern "C" firls_status firls_get_timing(firls_ctx* c, double* ms, int* launches, int* applications) {
  if (!c || !ms || !launches) return FIRLS_E_INVALID_ARG;
  if (!c->timing || !c->marks_valid) return fail(c, FIRLS_E_STATE, "timing is off or no macro step ran");
  CU(cudaStreamSynchronize(c->stream));
  for (int k = 0; k < FIRLS_NKCLASS; ++k) {
    ms[k] = 0.0;
    launches[k] = 0;
    if (applications) applications[k] = 0;
  }
  for (const auto& m : c->marks) {
    float t = 0.f;
    CU(cudaEventElapsedTime(&t, m.a, m.b));
    ms[m.cls] += t;
    launches[m.cls] += m.launches;
    if (applications) applications[m.cls] += 1;
  }
  return FIRLS_OK;
}

extern "C" void firls_destroy(firls_ctx* c) {
  if (!c) return;
  multi_forget(c);
  if (c->stream) cudaStreamSynchronize(c->stream);
  else cudaDeviceSynchronize();
  graphs_clear(c);
  for (cudaEvent_t e : c->evpool) cudaEventDestroy(e);
  for (void* p : c->allocs)
    if (p) cudaFree(p);
  delete c;
}

// ------------------------------------------------ operator-level entry points

extern "C" firls_status firls_apply_AHA(firls_ctx* c, const void* d, void* q) {
  if (!c || !d || !q) return FIRLS_E_INVALID_ARG;
  if (!c->op_set) return fail(c, FIRLS_E_STATE, "operator not set");
  // run with lambdas 0 and no regulariser terms: state must say "running"
  std::vector<float> zeros(c->batch, 0.f);
  firls_params p{};
  p.outer_iters = p.pcg_iters = 1;
  p.lambda_per_slice = zeros.data();
  p.lambda_tv_per_slice = zeros.data();
  TRY(upload_params(c, &p));
  state_init(c->batch, c->stream, c->st, c->part, 0, c->counts, c->n, c->lam_d, c->lamtv_d, 1e-10f, 1, PH_START);
  FftArgs a = fft_args(c);
  const size_t bytes = sizeof(float2) * (size_t)c->batch * c->n * c->n;
  CU(cudaMemcpyAsync(c->d, d, bytes, cudaMemcpyDeviceToDevice, c->stream));
  a.d = c->d;
  a.t = c->t;
  a.mode = 2;
  fft_row_fwd(c->n, a);
  a.mask = c->mask;
  fft_col_mask(c->n, a);
  a.q = static_cast<float2*>(q);
  fft_row_inv(c->n, a);
  return cuda_check(c, cudaGetLastError(), "apply_AHA");
}

extern "C" firls_status firls_apply_Phi(firls_ctx* c, const void* x, void* cc) {
  if (!c || !x || !cc) return FIRLS_E_INVALID_ARG;
  if (!c->op_set || !c->kind) return fail(c, FIRLS_E_STATE, "no wavelet set");
  WavArgs w = wav_args(c, nullptr);
  wavelet_forward(w, static_cast<const float2*>(x), static_cast<float2*>(cc), nullptr, WAV_RAW);
  return cuda_check(c, cudaGetLastError(), "apply_Phi");
}

extern "C" firls_status firls_apply_PhiT(firls_ctx* c, const void* cc, void* x) {
  if (!c || !x || !cc) return FIRLS_E_INVALID_ARG;
  if (!c->op_set || !c->kind) return fail(c, FIRLS_E_STATE, "no wavelet set");
  WavArgs w = wav_args(c, nullptr);
  wavelet_inverse(w, static_cast<const float2*>(cc), static_cast<float2*>(x), nullptr, 0);
  return cuda_check(c, cudaGetLastError(), "apply_PhiT");
}

extern "C" firls_status firls_apply_S_P(firls_ctx* c, const firls_params* p, const void* x, const void* d,
                                        void* q, const void* r, void* z) {
  if (!c || !p || !x || !d || !q || !r || !z) return FIRLS_E_INVALID_ARG;
  if (!c->op_set) return fail(c, FIRLS_E_STATE, "operator not set");
  TRY(check_params(c, p));
  TRY(upload_params(c, p));
  const int B = c->batch, n = c->n;
  const size_t bytes = sizeof(float2) * (size_t)B * n * n;
  state_init(B, c->stream, c->st, c->part, 0, c->counts, n, c->lam_d, c->lamtv_d, eps_of(p), 1, PH_START);
  CU(cudaMemcpyAsync(c->x, x, bytes, cudaMemcpyDeviceToDevice, c->stream));
  enqueue_weights(c, c->x, p->precond, c->st);  // every slice starts an outer step here
  // q = S d
  CU(cudaMemcpyAsync(c->d, d, bytes, cudaMemcpyDeviceToDevice, c->stream));
  enqueue_S(c, 2, nullptr, c->d, static_cast<float2*>(q));
  // z = P^{-1} r: feed r as "A^H b" with q = 0 through the INIT path
  CU(cudaMemcpyAsync(c->atb, r, bytes, cudaMemcpyDeviceToDevice, c->stream));
  CU(cudaMemsetAsync(c->q, 0, bytes, c->stream));
  firls_params one = *p;
  one.pcg_tol = 0.f;
  enqueue_precond(c, ILU_INIT, one);
  CU(cudaMemcpyAsync(z, c->z, bytes, cudaMemcpyDeviceToDevice, c->stream));
  return cuda_check(c, cudaGetLastError(), "apply_S_P");
}

// F_eps per slice (Eq. anapro / iso with the eps of Eq. gw / wi), host out[batch].
firls_status objective_parts(firls_ctx* c, const void* b, const firls_params* p, const float2* x) {
  const int B = c->batch, n = c->n;
  const float eps = eps_of(p);
  FftArgs a = fft_args(c);
  a.st = nullptr;
  a.d = const_cast<float2*>(x);
  a.t = c->t;
  a.mode = 2;
  // row FFT of x into t (state checks off: the kernel runs every slice)
  TRY(cuda_check(c, cudaMemsetAsync(c->st, 0, sizeof(SliceState) * B, c->stream), "memset"));
  state_init(B, c->stream, c->st, c->part, 0, c->counts, n, c->lam_d, c->lamtv_d, eps, 1, PH_START);
  a.st = c->st;
  fft_row_fwd(n, a);
  a.b = static_cast<const float2*>(b);
  a.mask = c->mask;
  a.mode = SLOT_DQ;
  fft_col_resid(n, a);
  if (c->kind) {
    WavArgs w = wav_args(c, nullptr);
    wavelet_forward(w, x, c->cw, nullptr, WAV_RAW);
    l21_sum(B, n, c->stream, c->cw, c->groups ? c->gidx : nullptr, c->goff, c->n_groups, c->gsize, eps, c->part,
            SLOT_RZ, c->channels);
  }
  if (has_tv(c)) tv_sum(B, n, c->stream, x, eps, c->part, SLOT_RR, is_aniso(c) ? 1 : 0, c->channels);
  return cuda_check(c, cudaGetLastError(), "objective");
}

firls_status objective_read(firls_ctx* c, const firls_params* p, double* out) {
  const int B = c->batch, n = c->n;
  std::vector<double> h((size_t)B * NSLOT * MAXPART);
  CU(cudaMemcpyAsync(h.data(), c->part, sizeof(double) * h.size(), cudaMemcpyDeviceToHost, c->stream));
  CU(cudaStreamSynchronize(c->stream));
  const int nd = fft_col_ctas(n), nr = axpy_ctas(n);
  for (int s = 0; s < B; ++s) {
    auto sum = [&](int slot, int np) {
      double a = 0.0;
      for (int i = 0; i < np; ++i) a += h[((size_t)s * NSLOT + slot) * MAXPART + i];
      return a;
    };
    const double lam = p->lambda_per_slice ? p->lambda_per_slice[s] : p->lambda;
    const double lt = p->lambda_tv_per_slice ? p->lambda_tv_per_slice[s] : p->lambda_tv;
    double f = 0.5 * sum(SLOT_DQ, nd);
    if (c->kind) f += lam * sum(SLOT_RZ, nr);
    if (has_tv(c)) f += lt * sum(SLOT_RR, nr);
    out[s] = f;
  }
  // multi-contrast: F_eps of the whole image (the joint regularisers sit in
  // its first slice's parts), the same value for each of its contrasts
  const int C = c->channels;
  for (int s0 = 0; C > 1 && s0 < B; s0 += C) {
    double f = 0.0;
    for (int t = 0; t < C; ++t) f += out[s0 + t];
    for (int t = 0; t < C; ++t) out[s0 + t] = f;
  }
  return FIRLS_OK;
}

// ---- continuous batching: per-slot load, run, status, read-out ----

// Retire a slot: it stops taking part in the outer steps until reloaded.
__global__ void k_slot_retire(SliceState* st) { st->done = 1; st->active = 0; }

extern "C" firls_status firls_slot_load(firls_ctx* c, int s, const uint8_t* mask, const void* b, const void* x0,
                                        float lambda, float lambda_tv, float eps) {
  if (!c || !mask || !b) return FIRLS_E_INVALID_ARG;
  if (!c->op_set) return fail(c, FIRLS_E_STATE, "operator not set");
  if (s < 0 || s >= c->batch) return fail(c, FIRLS_E_INVALID_ARG, "slot out of range");
  if (c->channels > 1) return fail(c, FIRLS_E_STATE, "slots hold single-contrast slices (channels is > 1)");
  if (!(lambda >= 0.f) || !(lambda_tv >= 0.f) || !std::isfinite(lambda) || !std::isfinite(lambda_tv))
    return fail(c, FIRLS_E_INVALID_ARG, "lambdas must be finite and >= 0");
  const int n = c->n;
  const size_t N = (size_t)n * n, off = (size_t)s * N;
  CU(cudaMemcpyAsync(c->mask + off, mask, N, cudaMemcpyDeviceToDevice, c->stream));
  CU(cudaMemsetAsync(c->counts + s, 0, sizeof(int), c->stream));
  mask_popcount(1, n, c->stream, c->mask + off, c->counts + s);
  {  // an empty mask is rejected; the slot is left retired
    int hc = 0;
    CU(cudaMemcpyAsync(&hc, c->counts + s, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
    CU(cudaStreamSynchronize(c->stream));
    if (hc <= 0) {
      k_slot_retire<<<1, 1, 0, c->stream>>>(c->st + s);
      CU(cudaGetLastError());
      return fail(c, FIRLS_E_INVALID_ARG, "empty mask");
    }
  }
  const float lam[2] = {c->kind ? lambda : 0.f, has_tv(c) ? lambda_tv : 0.f};
  CU(cudaMemcpyAsync(c->lam_d + s, &lam[0], sizeof(float), cudaMemcpyHostToDevice, c->stream));
  CU(cudaMemcpyAsync(c->lamtv_d + s, &lam[1], sizeof(float), cudaMemcpyHostToDevice, c->stream));
  double* part = c->part + (size_t)s * NSLOT * MAXPART;
  FftArgs a = fft_args(c);
  a.batch = 1;
  a.part = part;
  a.b = static_cast<const float2*>(b);
  a.mask = c->mask + off;
  a.t = c->t + off;
  fft_row_ahb(n, a);
  a.atb = c->atb + off;
  a.x = x0 ? nullptr : c->x + off;
  fft_col_inv(n, a);
  if (x0) CU(cudaMemcpyAsync(c->x + off, x0, N * sizeof(float2), cudaMemcpyDeviceToDevice, c->stream));
  CU(cudaMemsetAsync(c->dx + off, 0, N * sizeof(float2), c->stream));
  // no outer-step limit: the caller reads the slot out when it wants
  state_init(1, c->stream, c->st + s, part, fft_col_ctas(n), c->counts + s, n, c->lam_d + s, c->lamtv_d + s,
             eps > 0.f ? eps : 1e-10f, 1 << 30, PH_BOUNDARY);
  return cuda_check(c, cudaGetLastError(), "slot_load");
}

extern "C" firls_status firls_run_steps(firls_ctx* c, const firls_params* p, int macro_steps) {
  if (!c || !p) return FIRLS_E_INVALID_ARG;
  if (!c->op_set) return fail(c, FIRLS_E_STATE, "operator not set");
  if (macro_steps < 1) return fail(c, FIRLS_E_INVALID_ARG, "macro_steps must be >= 1");
  firls_params q = *p;
  q.outer_iters = 1;  // the per-slot limits come from firls_slot_load
  TRY(check_params(c, &q));
  // one graph of all the steps: the caller polls with firls_slot_status
  c->cur_batch = c->active_slots;
  const firls_status st = run_macro(c, q, macro_steps, macro_steps, false);
  c->cur_batch = 0;
  return st;
}

extern "C" firls_status firls_run(firls_ctx* c, const firls_params* p) {
  if (!c || !p) return FIRLS_E_INVALID_ARG;
  if (p->outer_iters < 1 || p->pcg_iters < 1) return fail(c, FIRLS_E_INVALID_ARG, "iteration counts must be >= 1");
  if (!c->op_set) return fail(c, FIRLS_E_STATE, "operator not set");
  firls_params q = *p;
  q.outer_iters = 1;
  TRY(check_params(c, &q));
  c->cur_batch = c->active_slots;
  const firls_status st = run_macro(c, q, solve_steps(p), p->pcg_iters + 1, false);
  c->cur_batch = 0;
  return st;
}

extern "C" firls_status firls_slot_status(firls_ctx* c, int* done, int* outer_done, double* rel_change,
                                          int* pcg_steps) {
  if (!c) return FIRLS_E_INVALID_ARG;
  std::vector<SliceState> hs(c->batch);
  CU(cudaMemcpyAsync(hs.data(), c->st, sizeof(SliceState) * c->batch, cudaMemcpyDeviceToHost, c->stream));
  CU(cudaStreamSynchronize(c->stream));
  for (int s = 0; s < c->batch; ++s) {
    if (done) done[s] = hs[s].done;
    if (outer_done) outer_done[s] = hs[s].outer_done;
    if (rel_change) rel_change[s] = hs[s].relchg;
    if (pcg_steps) pcg_steps[s] = hs[s].pcg_steps;
  }
  return FIRLS_OK;
}


extern "C" firls_status firls_slot_retire(firls_ctx* c, int s) {
  if (!c || s < 0 || s >= c->batch) return FIRLS_E_INVALID_ARG;
  k_slot_retire<<<1, 1, 0, c->stream>>>(c->st + s);
  return cuda_check(c, cudaGetLastError(), "slot_retire");
}

extern "C" firls_status firls_set_active_slots(firls_ctx* c, int k) {
  if (!c) return FIRLS_E_INVALID_ARG;
  if (k < 0 || k > c->batch) return fail(c, FIRLS_E_INVALID_ARG, "active slots out of range");
  c->active_slots = k == c->batch ? 0 : k;
  return FIRLS_OK;
}

extern "C" firls_status firls_slot_move(firls_ctx* c, int from, int to) {
  if (!c) return FIRLS_E_INVALID_ARG;
  if (from < 0 || from >= c->batch || to < 0 || to >= c->batch || from == to)
    return fail(c, FIRLS_E_INVALID_ARG, "bad slot pair");
  if (!c->op_set) return fail(c, FIRLS_E_STATE, "operator not set");
  const size_t N = (size_t)c->n * c->n;
  auto mv = [&](auto* base, size_t per) -> cudaError_t {
    return cudaMemcpyAsync(base + (size_t)to * per, base + (size_t)from * per, sizeof(*base) * per,
                           cudaMemcpyDeviceToDevice, c->stream);
  };
  CU(mv(c->mask, N));
  CU(mv(c->counts, 1));
  for (float2* v : {c->atb, c->x, c->r, c->z, c->d, c->q, c->t, c->u, c->cw, c->dx}) CU(mv(v, N));
  for (float* v : {c->ww, c->wtv, c->ia, c->wdiag, c->wtv2}) CU(mv(v, N));
  if (c->groups) CU(mv(c->wg, (size_t)c->n_groups));
  CU(mv(c->st, 1));
  CU(mv(c->stw, 1));
  CU(mv(c->part, (size_t)NSLOT * MAXPART));
  CU(mv(c->lam_d, 1));
  CU(mv(c->lamtv_d, 1));
  k_slot_retire<<<1, 1, 0, c->stream>>>(c->st + from);
  return cuda_check(c, cudaGetLastError(), "slot_move");
}

extern "C" firls_status firls_slot_get(firls_ctx* c, int s, void* x_out) {
  if (!c || !x_out || s < 0 || s >= c->batch) return FIRLS_E_INVALID_ARG;
  const size_t N = (size_t)c->n * c->n;
  CU(cudaMemcpyAsync(x_out, c->x + (size_t)s * N, N * sizeof(float2), cudaMemcpyDeviceToDevice, c->stream));
  return FIRLS_OK;
}

// ---- autotuner: tile shapes timed on the context's own buffers ----
namespace {
bool tune_cache_lookup(const char* path, const std::string& key, int* rb, int* cm, int* il) {
  if (!path || !*path) return false;
  FILE* f = std::fopen(path, "r");
  if (!f) return false;
  char line[256];
  bool found = false;
  while (std::fgets(line, sizeof line, f)) {
    char k[128];
    int a, b2, d;
    if (std::sscanf(line, "%127[^|]| %d %d %d", k, &a, &b2, &d) == 4 && key == k) {
      *rb = a;
      *cm = b2;
      *il = d;
      found = true;  // last entry wins
    }
  }
  std::fclose(f);
  return found;
}

float time_ms(firls_ctx* c, const std::function<void()>& fn, int reps) {
  cudaEvent_t a, b;
  cudaEventCreate(&a);
  cudaEventCreate(&b);
  fn();  // warm-up
  cudaEventRecord(a, c->stream);
  for (int i = 0; i < reps; ++i) fn();
  cudaEventRecord(b, c->stream);
  cudaEventSynchronize(b);
  float ms = 0.f;
  cudaEventElapsedTime(&ms, a, b);
  cudaEventDestroy(a);
  cudaEventDestroy(b);
  return ms / reps;
}
}  // namespace

extern "C" firls_status firls_autotune(firls_ctx* c, const char* cache_path) {
  if (!c) return FIRLS_E_INVALID_ARG;
  if (!c->op_set) return fail(c, FIRLS_E_STATE, "operator not set");
  const int B = c->batch, n = c->n;
  char keybuf[128];
  std::snprintf(keybuf, sizeof keybuf, "n=%d batch=%d psi=%u levels=%d ", n, B, c->psi, c->levels);
  const std::string key(keybuf);
  int rb = 0, cm = 0, il = 0;
  if (!tune_cache_lookup(cache_path, key, &rb, &cm, &il)) {
    // deterministic, finite contents for timing
    const size_t BN = (size_t)B * n * n;
    for (float2* v : {c->x, c->d, c->r, c->q, c->z, c->atb, c->u, c->cw}) cudaMemsetAsync(v, 0, BN * 8, c->stream);
    for (float* v : {c->ww, c->wtv, c->wdiag}) cudaMemsetAsync(v, 0, BN * 4, c->stream);
    firls_params p{};
    p.outer_iters = p.pcg_iters = 1;
    p.lambda = 1e-3f;
    p.lambda_tv = 1e-3f;
    TRY(upload_params(c, &p));
    state_init(B, c->stream, c->st, c->part, 0, c->counts, n, c->lam_d, c->lamtv_d, 1e-10f, 1, PH_START);
    if (has_tv(c)) penta_setup(B, n, c->stream, c->st, c->wtv, tv2_of(c), nullptr, c->ia);
    float best = 1e30f;
    if (c->kind) {
      for (int r : {1, 2, 4, 8, 16})
        for (int m : {32, 64}) {
          const bool cluster = r < 4;
          if (cluster && (m != 64 || !wavelet_cluster_ctas(n, c->levels, c->kind, r))) continue;
          WavArgs w = wav_args(c, c->st);
          w.rb = r;
          w.coarse_max = m;
          const float t = time_ms(c, [&]() { wavelet_apply(w, c->d, c->cw, c->ww, WAV_MUL_W, c->u, nullptr, 0); }, 5);
          if (t < best) {
            best = t;
            rb = r;
            cm = m;
          }
        }
    }
    if (has_tv(c)) {
      best = 1e30f;
      for (int shape : {42, 43, 44, 22, 23, 24}) {
        if (!ilu_shape_fits(n, shape, is_aniso(c))) continue;
        const float t = time_ms(c, [&]() {
          ilu_step(B, n, c->stream, c->st, c->part, ILU_STEP, c->x, c->d, c->r, c->q, c->atb, c->u, c->z, c->ia,
                   c->wtv, shape, 0, PcgSched{0.f, 0, 1 << 30, 0, 0}, 0, tv2_of(c));
        }, 5);
        if (t < best) {
          best = t;
          il = shape;
        }
      }
    }
    CU(cudaGetLastError());
    if (cache_path && *cache_path) {
      FILE* f = std::fopen(cache_path, "a");
      if (f) {
        std::fprintf(f, "%s| %d %d %d\n", key.c_str(), rb, cm, il);
        std::fclose(f);
      }
    }
  }
  c->tune_rb = rb;
  c->tune_cmax = cm;
  c->tune_ilu = il;
  multi_forget(c);
  graphs_clear(c);
  return FIRLS_OK;
}

extern "C" firls_status firls_set_tuning(firls_ctx* c, int rows_per_cta, int coarse_max, int ilu_shape) {
  if (!c) return FIRLS_E_INVALID_ARG;
  if (rows_per_cta < 0 || coarse_max < 0 || ilu_shape < 0)
    return fail(c, FIRLS_E_INVALID_ARG, "tile shapes must be >= 0 (0 = default)");
  if (ilu_shape > 0 && !ilu_shape_fits(c->n, ilu_shape, is_aniso(c)))
    return fail(c, FIRLS_E_INVALID_ARG, "ILU shape does not fit this size");
  if ((rows_per_cta == 1 || rows_per_cta == 2) && c->kind && !wavelet_cluster_ctas(c->n, c->levels, c->kind, rows_per_cta))
    return fail(c, FIRLS_E_INVALID_ARG, "the one-launch cluster wavelet form does not fit this size");
  if (rows_per_cta == 3 || (rows_per_cta > 4 && rows_per_cta != 8 && rows_per_cta != 16))
    return fail(c, FIRLS_E_INVALID_ARG, "wavelet rows per CTA must be 0, 1, 2, 4, 8 or 16");
  if (c->tune_rb != rows_per_cta || c->tune_cmax != coarse_max || c->tune_ilu != ilu_shape) {
    c->tune_rb = rows_per_cta;
    c->tune_cmax = coarse_max;
    c->tune_ilu = ilu_shape;
    multi_forget(c);
    graphs_clear(c);  // the captured macro steps change shape
  }
  return FIRLS_OK;
}

extern "C" firls_status firls_set_channels(firls_ctx* c, int channels) {
  if (!c) return FIRLS_E_INVALID_ARG;
  if (channels < 1 || c->batch % channels)
    return fail(c, FIRLS_E_INVALID_ARG, "channels must be >= 1 and divide the batch");
  if (channels > 1 && c->op_set && (c->groups || (c->psi & FIRLS_PSI_TV_ANISO)))
    return fail(c, FIRLS_E_INVALID_ARG, "multi-contrast images take singleton joint groups and isotropic joint TV");
  if (channels != c->channels) {
    c->channels = channels;
    multi_forget(c);
    graphs_clear(c);  // the captured macro steps change
  }
  return FIRLS_OK;
}

extern "C" firls_status firls_set_wait_test(firls_ctx* c, int enable) {
  if (!c) return FIRLS_E_INVALID_ARG;
  const int v = enable ? 1 : 0;
  if (v != c->wait_test) {
    c->wait_test = v;
    multi_forget(c);
    graphs_clear(c);  // the captured macro steps change
  }
  return FIRLS_OK;
}

extern "C" firls_status firls_get_tuning(const firls_ctx* c, int* rows_per_cta, int* coarse_max, int* ilu_depth) {
  if (!c) return FIRLS_E_INVALID_ARG;
  if (rows_per_cta) *rows_per_cta = c->tune_rb;
  if (coarse_max) *coarse_max = c->tune_cmax;
  if (ilu_depth) *ilu_depth = c->tune_ilu;
  return FIRLS_OK;
}

extern "C" firls_status firls_adjoint(firls_ctx* c, const void* b, void* atb) {
  if (!c || !b || !atb) return FIRLS_E_INVALID_ARG;
  if (!c->op_set) return fail(c, FIRLS_E_STATE, "operator not set");
  FftArgs a = fft_args(c);
  a.b = static_cast<const float2*>(b);
  a.mask = c->mask;
  a.t = c->t;
  fft_row_ahb(c->n, a);
  a.atb = static_cast<float2*>(atb);
  a.x = nullptr;
  fft_col_inv(c->n, a);
  return cuda_check(c, cudaGetLastError(), "adjoint");
}

extern "C" firls_status firls_data_consistency(firls_ctx* c, const void* b, const void* x, void* out) {
  if (!c || !b || !x || !out) return FIRLS_E_INVALID_ARG;
  if (!c->op_set) return fail(c, FIRLS_E_STATE, "operator not set");
  const int B = c->batch, n = c->n;
  // kernels check the slice state: lambdas 0, all running
  std::vector<float> zeros(B, 0.f);
  firls_params p{};
  p.outer_iters = p.pcg_iters = 1;
  p.lambda_per_slice = zeros.data();
  p.lambda_tv_per_slice = zeros.data();
  TRY(upload_params(c, &p));
  state_init(B, c->stream, c->st, c->part, 0, c->counts, n, c->lam_d, c->lamtv_d, 1e-10f, 1, PH_START);
  FftArgs a = fft_args(c);
  a.d = const_cast<float2*>(static_cast<const float2*>(x));
  a.t = c->t;
  a.mode = 2;
  fft_row_fwd(n, a);
  a.b = static_cast<const float2*>(b);
  a.mask = c->mask;
  fft_col_dc(n, a);
  a.d = c->t;  // only read for the (unused) dot product
  a.u = nullptr;
  a.wtv = nullptr;
  a.q = static_cast<float2*>(out);
  fft_row_inv(n, a);
  return cuda_check(c, cudaGetLastError(), "data_consistency");
}

extern "C" firls_status firls_objective(firls_ctx* c, const void* b, const firls_params* p, const void* x,
                                        double* out) {
  if (!c || !b || !p || !x || !out) return FIRLS_E_INVALID_ARG;
  if (!c->op_set) return fail(c, FIRLS_E_STATE, "operator not set");
  TRY(check_params(c, p));
  TRY(upload_params(c, p));
  TRY(objective_parts(c, b, p, static_cast<const float2*>(x)));
  return objective_read(c, p, out);
}

extern "C" firls_status firls_warm_start_guard(firls_ctx* c, const void* b, const firls_params* p, const void* x1,
                                               void* x0, int* chosen) {
  if (!c || !b || !p || !x1 || !x0) return FIRLS_E_INVALID_ARG;
  if (!c->op_set) return fail(c, FIRLS_E_STATE, "operator not set");
  TRY(check_params(c, p));
  TRY(upload_params(c, p));
  const int B = c->batch, n = c->n;
  const size_t slice = sizeof(float2) * (size_t)n * n;
  std::vector<double> f1(B), f0(B);
  TRY(objective_parts(c, b, p, static_cast<const float2*>(x1)));
  TRY(objective_read(c, p, f1.data()));
  // A^H b into the context's atb buffer
  FftArgs a = fft_args(c);
  a.b = static_cast<const float2*>(b);
  a.mask = c->mask;
  a.t = c->t;
  fft_row_ahb(n, a);
  a.atb = c->atb;
  a.x = nullptr;
  fft_col_inv(n, a);
  TRY(objective_parts(c, b, p, c->atb));
  TRY(objective_read(c, p, f0.data()));
  for (int s = 0; s < B; ++s) {
    const bool use = std::isfinite(f1[s]) && f1[s] <= f0[s];
    const void* src = use ? static_cast<const char*>(x1) + s * slice : static_cast<const void*>(c->atb + (size_t)s * n * n);
    CU(cudaMemcpyAsync(static_cast<char*>(x0) + s * slice, src, slice, cudaMemcpyDeviceToDevice, c->stream));
    if (chosen) chosen[s] = use ? 1 : 0;
  }
  return cuda_check(c, cudaGetLastError(), "warm_start_guard");
}

extern "C" firls_status firls_get_weights(firls_ctx* c, float* w_wavelet, float* w_tv, float* w_tv2) {
  if (!c) return FIRLS_E_INVALID_ARG;
  const size_t bytes = sizeof(float) * (size_t)c->batch * c->n * c->n;
  if (w_wavelet) CU(cudaMemcpyAsync(w_wavelet, c->ww, bytes, cudaMemcpyDeviceToDevice, c->stream));
  if (w_tv) CU(cudaMemcpyAsync(w_tv, c->wtv, bytes, cudaMemcpyDeviceToDevice, c->stream));
  if (w_tv2) {
    if (!is_aniso(c)) return fail(c, FIRLS_E_STATE, "W2 exists only with FIRLS_PSI_TV_ANISO");
    CU(cudaMemcpyAsync(w_tv2, c->wtv2, bytes, cudaMemcpyDeviceToDevice, c->stream));
  }
  return FIRLS_OK;
}

extern "C" firls_status firls_get_precond(firls_ctx* c, float* wavelet_diag, float* inv_a) {
  if (!c) return FIRLS_E_INVALID_ARG;
  if (!has_tv(c)) return fail(c, FIRLS_E_STATE, "the TV preconditioner exists only with FIRLS_PSI_TV");
  const size_t bytes = sizeof(float) * (size_t)c->batch * c->n * c->n;
  if (wavelet_diag) {
    if (!c->kind) return fail(c, FIRLS_E_STATE, "no wavelet term");
    CU(cudaMemcpyAsync(wavelet_diag, c->wdiag, bytes, cudaMemcpyDeviceToDevice, c->stream));
  }
  if (inv_a) CU(cudaMemcpyAsync(inv_a, c->ia, bytes, cudaMemcpyDeviceToDevice, c->stream));
  return FIRLS_OK;
}

extern "C" firls_status firls_get_inverse_map(firls_ctx* c, int32_t* offsets, int32_t* ids) {
  if (!c || !offsets || !ids) return FIRLS_E_INVALID_ARG;
  if (!c->groups) return fail(c, FIRLS_E_STATE, "no group map set");
  const size_t N = (size_t)c->n * c->n;
  CU(cudaMemcpyAsync(offsets, c->inv_off, sizeof(int) * (N + 1), cudaMemcpyDeviceToDevice, c->stream));
  CU(cudaMemcpyAsync(ids, c->inv_ids, sizeof(int) * c->gtotal, cudaMemcpyDeviceToDevice, c->stream));
  return FIRLS_OK;
}

extern "C" firls_status firls_get_popcounts(firls_ctx* c, int32_t* counts) {
  if (!c || !counts) return FIRLS_E_INVALID_ARG;
  CU(cudaMemcpyAsync(counts, c->counts, sizeof(int) * c->batch, cudaMemcpyDeviceToDevice, c->stream));
  return FIRLS_OK;
}

namespace {
// Sets the dynamic shared-memory limits of every kernel for this size
// outside any stream capture.
void prepare_kernels(int n) {
  fft_prepare(n);
  wav_prepare();
}
}  // namespace
