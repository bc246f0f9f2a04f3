// extern "C" entry points of tensorctl and the PCG driver (Appendix 2,
// Algorithm 1). Every entry point catches the library's internal errors and
// returns a status code; nothing throws across the ABI.
#include <algorithm>
#include <cstdlib>
#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <new>
#include <atomic>
#include <mutex>
#include <thread>

#include "tctl_internal.cuh"

using namespace tctl;

namespace {

thread_local std::string g_last_error;

constexpr int kCap = 64;

int handle(Ctx *c, const Error &e) {
  if (c) c->err = e.msg;
  g_last_error = e.msg;
  return e.code;
}

void check_cp(const Ctx &c, const tctl_cp *t, const char *name, bool need_terms) {
  if (!t) fail(TCTL_E_ARG, std::string(name) + " is NULL");
  for (int l = 0; l < 3; ++l)
    if (t->n[l] != c.n) fail(TCTL_E_ARG, std::string(name) + ": mode size differs from n");
  if (t->rank < 0 || t->cap < 0 || t->rank > t->cap)
    fail(TCTL_E_ARG, std::string(name) + ": invalid rank/cap");
  if (need_terms && t->rank > 0 && (!t->w || !t->U[0] || !t->U[1] || !t->U[2]))
    fail(TCTL_E_ARG, std::string(name) + ": NULL factor pointer");
  if (!need_terms && t->cap > 0 && (!t->w || !t->U[0] || !t->U[1] || !t->U[2]))
    fail(TCTL_E_ARG, std::string(name) + ": NULL factor pointer");
}

// Restores the workspace's bump pointer when an entry point leaves, also by an
// error, so that a failed call does not shrink the workspace of the next one.
struct WsGuard {
  Arena &a;
  size_t m;
  explicit WsGuard(Arena &ar) : a(ar), m(ar.mark()) {}
  ~WsGuard() { a.reset(m); }
};

struct Timer {
  cudaEvent_t a, b;
  cudaStream_t st;
  explicit Timer(cudaStream_t s) : st(s) {
    TCTL_CUDA(cudaEventCreate(&a));
    TCTL_CUDA(cudaEventCreate(&b));
    TCTL_CUDA(cudaEventRecord(a, st));
  }
  double stop_ms() {
    TCTL_CUDA(cudaEventRecord(b, st));
    TCTL_CUDA(cudaEventSynchronize(b));
    float ms = 0;
    TCTL_CUDA(cudaEventElapsedTime(&ms, a, b));
    return ms;
  }
  ~Timer() {
    cudaEventDestroy(a);
    cudaEventDestroy(b);
  }
};

// fun / precond of Algorithm 1 on Tucker vectors; in the paper form (basis 0)
// the vectors are in grid coordinates and every apply goes through V_l^T / V_l.
// The anisotropic-Laplacian preconditioner (pre_src 3) is diagonal in the sine
// basis: its factors move there (W_l = S^T V_l) and back around the Hadamard step.
void apply_sep(Ctx &c, const Sep &D, const Tucker &x, Tucker &y, Tucker &tmp, double eps) {
  const bool sine = (&D == &c.pre) && c.pre_used == 3;
  if (c.o.basis == 1 && !sine) {
    sep_apply_trunc(c, D, x, y, eps);
    return;
  }
  tucker_copy(c, x, tmp);
  if (c.o.basis == 0) tucker_basis_change(c, tmp, true);
  if (sine) tucker_factor_change(c, tmp, c.W, false);
  sep_apply_trunc(c, D, tmp, y, eps);
  if (sine) tucker_factor_change(c, y, c.W, true);
  if (c.o.basis == 0) tucker_basis_change(c, y, false);
}

}  // namespace

namespace tctl {

void set_noalloc_error(const std::string &msg) { g_last_error = msg; }

// Algorithm 1 on the Tucker right-hand side B (context coordinates): X from
// X0 = 0 until ||R_k|| <= tol (absolute) or max_iter; the work vectors are
// the caller's. Returns the iterations; *rel = the last ||R_k|| / ||B||.
int pcg_run(Ctx &c, const Tucker &B, double bnorm, double tol, Tucker &X, Tucker *w, double *rel,
            int *maxr) {
  const double eps = c.eps;
  const double eps_x = c.o.eps_final > 0 ? c.o.eps_final : 0.1 * eps;
  Tucker &R = w[0], &Z = w[1], &P = w[2], &S = w[3], &T1 = w[4], &T2 = w[5];
  auto track = [&](const Tucker &t) {
    for (int l = 0; l < 3; ++l) *maxr = std::max(*maxr, t.r[l]);
  };
  int iters = 0;
  X.r[0] = X.r[1] = X.r[2] = 0;
  *rel = 1.0;
  tucker_copy(c, B, R);                       // R0 = B - fun(X0), X0 = 0
  {
    TCTL_OUTER(c, "precond");
    apply_sep(c, c.pre, R, Z, T1, eps);       // Z0 = trunc(precond(R0))
  }
  tucker_copy(c, Z, P);                       // P0 = Z0
  double rz = tucker_inner(c, R, Z);
  while (iters < c.o.max_iter) {
    {
      TCTL_OUTER(c, "fun");
      apply_sep(c, c.op, P, S, T1, eps);      // S = trunc(fun(P))
    }
    track(S);
    const double pS = tucker_inner(c, P, S);
    if (!(pS > 0.0) || !std::isfinite(pS)) fail(TCTL_E_NUMERIC, "PCG breakdown: <P, S> <= 0");
    const double a = rz / pS;
    {
      TCTL_OUTER(c, "update_x");
      tucker_axpby_trunc(c, 1.0, X, a, P, T2, eps_x);  // X = trunc(X + a P)
    }
    std::swap(X, T2);
    // R = trunc(R - a S); the stopping test uses ||R - a S|| before the
    // truncation, and a converged residual is not truncated (not used again)
    double rnorm = 0.0;
    {
      TCTL_OUTER(c, "update_r");
      tucker_axpby_trunc(c, 1.0, R, -a, S, T2, eps, &rnorm, tol);
    }
    std::swap(R, T2);
    track(X);
    track(R);
    ++iters;
    *rel = rnorm / bnorm;
    if (!std::isfinite(*rel)) fail(TCTL_E_NAN, "non-finite residual");
    if (rnorm <= tol) break;
    {
      TCTL_OUTER(c, "precond");
      apply_sep(c, c.pre, R, Z, T1, eps);     // Z = trunc(precond(R))
    }
    const double rz_new = tucker_inner(c, R, Z);
    const double beta = rz_new / rz;
    rz = rz_new;
    {
      TCTL_OUTER(c, "update_p");
      tucker_axpby_trunc(c, 1.0, Z, beta, P, T2, eps);  // P = trunc(Z + beta P)
    }
    std::swap(P, T2);
    track(P);
  }
  return iters;
}

// Algorithm 1, optionally inside opts.refine steps of FP64 residual
// refinement: X_0 = PCG(B) with the contractions at opts.tc_digits digits;
// then, while ||B - fun(X_j)|| > pcg_rtol ||B|| (the residual formed with
// FP64 FMA contractions, truncated at eps_final), X_{j+1} = trunc(X_j +
// PCG(B - fun(X_j))) with the same low-precision inner solve.
int pcg_solve(Ctx &c, const tctl_cp *b, tctl_cp *x, tctl_stats *st) {
  Timer timer(c.st);
  const double eps_x = c.o.eps_final > 0 ? c.o.eps_final : 0.1 * c.eps;
  const bool eig = (c.o.basis == 1);
  size_t mk = c.ws.mark();
  Tucker B, X, D, Rt, T1, w[6];
  for (Tucker *t : {&B, &X}) tucker_alloc(c, *t, kCap);
  for (Tucker &t : w) tucker_alloc(c, t, kCap);
  if (c.o.refine > 0)
    for (Tucker *t : {&D, &Rt, &T1}) tucker_alloc(c, *t, kCap);
  cp_to_tucker(c, b->rank, b->w, b->U, eig, B, 1e-12);
  const double bnorm = std::sqrt(std::max(tucker_inner(c, B, B), 0.0));
  const double tol = c.o.pcg_rtol * bnorm;
  int status = TCTL_OK;
  int iters = 0, maxr = 0, refines = 0;
  double rel = 0.0, true_rel = -1.0;
  X.r[0] = X.r[1] = X.r[2] = 0;
  // the inner solves' digit count and the FP64 switch of the residual step are
  // put back on every exit (a failure throws)
  struct Restore {
    Ctx &c;
    int tc;
    ~Restore() {
      c.digits = 6;
      c.o.tc_gemm = tc;
    }
  } restore{c, c.o.tc_gemm};
  c.digits = c.o.tc_digits;
  if (bnorm == 0.0) {
    x->rank = 0;
  } else {
    iters = pcg_run(c, B, bnorm, tol, X, w, &rel, &maxr);
    bool converged = rel <= c.o.pcg_rtol;
    for (int j = 0; j < c.o.refine; ++j) {
      // Rt = trunc(B - fun(X)) with FP64 contractions
      c.o.tc_gemm = 0;
      double rn = 0.0;
      {
        TCTL_OUTER(c, "residual");
        apply_sep(c, c.op, X, w[3], T1, eps_x);
        tucker_axpby_trunc(c, 1.0, B, -1.0, w[3], Rt, eps_x, &rn);
      }
      c.o.tc_gemm = restore.tc;
      true_rel = rn / bnorm;
      if (!std::isfinite(true_rel)) fail(TCTL_E_NAN, "non-finite residual");
      if (rn <= tol) {
        converged = true;
        break;
      }
      double rel_d = 0.0;
      iters += pcg_run(c, Rt, bnorm, tol, D, w, &rel_d, &maxr);
      {
        TCTL_OUTER(c, "update_x");
        tucker_axpby_trunc(c, 1.0, X, 1.0, D, T1, eps_x);  // X = trunc(X + D)
      }
      std::swap(X, T1);
      ++refines;
      converged = rel_d <= c.o.pcg_rtol;
      rel = rel_d;
    }
    if (!converged) status = TCTL_E_NOT_CONVERGED;
    TCTL_OUTER(c, "to_cp");
    const int s2 = tucker_to_cp(c, X, eig, eps_x, x);
    tcg_check(c);
    if (status == TCTL_OK) status = s2;
  }
  c.stats.iters = iters;
  c.stats.rel_res = rel;
  c.stats.refines = refines;
  c.stats.true_rel_res = true_rel;
  for (int l = 0; l < 3; ++l) c.stats.rank_x[l] = X.r[l];
  c.stats.max_rank = maxr;
  c.stats.ws_peak_mb = (double)c.ws.peak / (1 << 20);
  c.stats.ws_size_mb = (double)c.ws.size / (1 << 20);
  c.ws.reset(mk);
  c.stats.t_solve_ms = timer.stop_ms();
  if (st) *st = c.stats;
  return status;
}

}  // namespace tctl

extern "C" {

// Contexts allocate from the device's default memory pool, stream-ordered, so
// that creating and destroying contexts on concurrent streams never
// synchronises the device; freed blocks stay in the pool (release threshold
// raised once per device and process) for the next context.
static void keep_pool_memory() {
  static std::mutex mu;
  static std::vector<int> done;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return;
  std::lock_guard<std::mutex> lk(mu);
  if (std::find(done.begin(), done.end(), dev) != done.end()) return;
  cudaMemPool_t pool;
  if (cudaDeviceGetDefaultMemPool(&pool, dev) == cudaSuccess) {
    uint64_t thr = UINT64_MAX;
    cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &thr);
  }
  done.push_back(dev);
}

// Automatic workspace: the set-up needs 6 n^2 doubles; a solve's peak grows
// about linearly in n (sketch and Khatri-Rao matrices of n x 64^2, their digit
// planes, the core-projection chunks capped at 48 Mi doubles).
static size_t auto_arena_bytes(int n) {
  const size_t setup = (size_t)6 * n * n * sizeof(double);
  const size_t solve = std::min<size_t>((size_t)3 << 30, ((size_t)512 << 20) + (size_t)n * (1280u << 10));
  return setup + solve;
}

int tctl_default_opts(tctl_opts *o) {
  if (!o) return TCTL_E_ARG;
  std::memset(o, 0, sizeof(*o));
  o->pcg_rtol = 1e-7;
  o->max_iter = 100;
  o->op_tol = 1e-8;
  o->r_pre = 24;
  o->rank_cap = kCap;
  o->precision = 0;
  o->basis = 1;
  o->expsum_src = 1;
  o->paper_end_rows = 0;
  o->eps_final = 0.0;
  o->seed = 1;
  o->range_tol = 0.03;
  o->tc_gemm = 1;
  o->pre_src = 0;
  o->pre_r = 12;
  o->pre_model = nullptr;
  o->pre_delta_max = 0.25;
  o->op_model = nullptr;
  o->op_r = 16;
  o->op_judge = 1e-7;
  o->tune = 0;
  o->tc_digits = 6;
  o->refine = 0;
  return TCTL_OK;
}

int tctl_setup(tctl_ctx **ctx, const double *coeffs, int n, double alpha, double beta,
               double eps_trunc, const tctl_opts *opts, void *cuda_stream) {
  Ctx *c = nullptr;
  try {
    if (!ctx) fail(TCTL_E_ARG, "ctx is NULL");
    *ctx = nullptr;
    if (!coeffs) fail(TCTL_E_ARG, "coeffs is NULL");
    if (n < 2 || n > 32768) fail(TCTL_E_ARG, "n must be in [2, 32768]");
    if (!(alpha > 0.0 && alpha <= 1.0)) fail(TCTL_E_ARG, "alpha must be in (0, 1]");
    if (!(beta > 0.0) || !std::isfinite(beta)) fail(TCTL_E_ARG, "beta must be positive");
    if (!(eps_trunc > 0.0 && eps_trunc < 1.0)) fail(TCTL_E_ARG, "eps_trunc must be in (0, 1)");
    for (long long i = 0; i < 3ll * (n + 1); ++i)
      if (!(coeffs[i] > 0.0) || !std::isfinite(coeffs[i]))
        fail(TCTL_E_COEFF, "coefficient a_l(x) must be positive and finite");
    c = new (std::nothrow) Ctx();
    if (!c) fail(TCTL_E_NOMEM, "host allocation failed");
    tctl_default_opts(&c->o);
    if (opts) c->o = *opts;
    if (c->o.precision != 0 && c->o.precision != 1)
      fail(TCTL_E_ARG, "precision must be 0 (FP64) or 1 (tensor-core digit split)");
    if (c->o.precision == 1 && !tc_fullgrid_supported(n))
      fail(TCTL_E_ARG, "precision 1 needs n a multiple of 128 and n <= 1024");
    if (c->o.expsum_src < 0 || c->o.expsum_src > 2)
      fail(TCTL_E_ARG, "expsum_src must be 0 (sinc), 1 (fitted) or 2 (learned)");
    if (c->o.expsum_src == 2 && !c->o.op_model) fail(TCTL_E_ARG, "expsum_src 2 needs op_model");
    if (c->o.expsum_src == 2 && (c->o.op_r < 2 || c->o.op_r > kPreRMax))
      fail(TCTL_E_ARG, "op_r must be in [2, 32]");
    if (c->o.expsum_src == 2 && !(c->o.op_judge > 0.0 && c->o.op_judge < 1.0))
      fail(TCTL_E_ARG, "op_judge must be in (0, 1)");
    if (c->o.basis != 0 && c->o.basis != 1) fail(TCTL_E_ARG, "basis must be 0 or 1");
    if (c->o.tc_gemm != 0 && c->o.tc_gemm != 1) fail(TCTL_E_ARG, "tc_gemm must be 0 or 1");
    if (c->o.tc_digits != 3 && c->o.tc_digits != 4 && c->o.tc_digits != 6)
      fail(TCTL_E_ARG, "tc_digits must be 3, 4 or 6");
    if (c->o.refine < 0 || c->o.refine > 8) fail(TCTL_E_ARG, "refine must be in [0, 8]");
    if (c->o.workspace_mb < 0) fail(TCTL_E_ARG, "workspace_mb must be >= 0");
    if (c->o.pre_src < 0 || c->o.pre_src > 3) fail(TCTL_E_ARG, "pre_src must be 0, 1, 2 or 3");
    if ((c->o.pre_src == 1 || c->o.pre_src == 2) && (c->o.pre_r < 2 || c->o.pre_r > kPreRMax))
      fail(TCTL_E_ARG, "pre_r must be in [2, 32]");
    if (c->o.pre_src == 2 && !c->o.pre_model) fail(TCTL_E_ARG, "pre_src 2 needs pre_model");
    if (!(c->o.range_tol >= 0.0 && c->o.range_tol <= 1.0))
      fail(TCTL_E_ARG, "range_tol must lie in [0, 1]");
    if (!(c->o.op_tol > 0 && c->o.op_tol < 1e-2)) fail(TCTL_E_ARG, "op_tol must be in (0, 1e-2)");
    if (c->o.r_pre < 1 || c->o.r_pre > 200) fail(TCTL_E_ARG, "r_pre must be in [1, 200]");
    if (c->o.max_iter < 1) fail(TCTL_E_ARG, "max_iter must be >= 1");
    if (!(c->o.pcg_rtol > 0)) fail(TCTL_E_ARG, "pcg_rtol must be positive");
    {
      const char *tr = std::getenv("TCTL_TRACE");
      c->trace = tr && tr[0] == '1';
    }
    c->n = n;
    c->alpha = alpha;
    c->beta = beta;
    c->eps = eps_trunc;
    c->st = static_cast<cudaStream_t>(cuda_stream);
    auto t0 = std::chrono::steady_clock::now();
    const size_t arena = c->o.workspace_mb > 0 ? ((size_t)c->o.workspace_mb << 20) : auto_arena_bytes(n);
    void *base = nullptr;
    keep_pool_memory();
    c->hstage = stage_acquire();
    check_cuda(cudaMallocAsync(&base, arena, c->st), "cudaMallocAsync(workspace)");
    c->owned.push_back(base);
    c->ws.base = static_cast<char *>(base);
    c->ws.size = arena;
    c->coef = c->dmalloc((size_t)3 * (n + 1));
    c->coef_host.assign(coeffs, coeffs + 3 * (size_t)(n + 1));
    to_dev(*c, c->coef, coeffs, (size_t)3 * (n + 1));
    setup_eigs(*c);
    auto t_eig = std::chrono::steady_clock::now();
    setup_spectral_fit(*c);
    auto t_fit = std::chrono::steady_clock::now();
    setup_spectral_build(*c);
    TCTL_CUDA(cudaStreamSynchronize(c->st));
    auto t1 = std::chrono::steady_clock::now();
    c->stats.t_setup_ms = std::chrono::duration<double, std::milli>(t1 - t0).count();
    auto dms = [](std::chrono::steady_clock::time_point a, std::chrono::steady_clock::time_point b) {
      return std::chrono::duration<double, std::milli>(b - a).count();
    };
    if (c->trace)
      std::fprintf(stderr, "[tctl] setup n=%d: eigenpairs %.1f ms, host fits %.1f ms, factors %.1f ms\n",
                   n, dms(t0, t_eig), dms(t_eig, t_fit), dms(t_fit, t1));
    c->stats.op_rank = c->op.R;
    c->stats.pre_rank = c->pre.R;
    for (int l = 0; l < 3; ++l) c->stats.op_basis[l] = c->op.rD[l];
    c->stats.op_rel_err = c->op_rel_err;
    c->stats.expsum_used = c->expsum_used;
    c->stats.pre_used = c->pre_used;
    c->stats.pre_delta = c->pre_delta;
    c->stats.op_learned_err = c->op_learned_err;
    c->stats.sinc24_err = c->sinc24_err;
    c->stats.s_min = c->s_min;
    c->stats.s_max = c->s_max;
    *ctx = reinterpret_cast<tctl_ctx *>(c);
    return TCTL_OK;
  } catch (const Error &e) {
    const int code = handle(c, e);
    if (c) tctl_destroy(reinterpret_cast<tctl_ctx *>(c));
    return code;
  }
}

// which: 0 = F2(A), 1 = the preconditioner, 2 = A^-alpha (state)
static int apply_common(tctl_ctx *ctx, const tctl_cp *x, tctl_cp *y, int which) {
  Ctx *c = reinterpret_cast<Ctx *>(ctx);
  if (!c) return TCTL_E_ARG;
  try {
    check_cp(*c, x, "x", true);
    check_cp(*c, y, "y", false);
    if (which == 2) ensure_state_sep(*c);
    WsGuard g(c->ws);
    size_t mk = c->ws.mark();
    Tucker tx, ty;
    tucker_alloc(*c, tx, kCap);
    tucker_alloc(*c, ty, kCap);
    const double e2 = c->eps / std::sqrt(2.0);
    cp_to_tucker(*c, x->rank, x->w, x->U, true, tx, 1e-12);
    sep_apply_trunc(*c, which == 0 ? c->op : which == 1 ? c->pre : c->state, tx, ty, e2);
    const int s = tucker_to_cp(*c, ty, true, e2, y);
    c->ws.reset(mk);
    return s;
  } catch (const Error &e) {
    return handle(c, e);
  }
}

int tctl_apply_op(tctl_ctx *ctx, const tctl_cp *x, tctl_cp *y) { return apply_common(ctx, x, y, 0); }

int tctl_apply_precond(tctl_ctx *ctx, const tctl_cp *x, tctl_cp *y) {
  return apply_common(ctx, x, y, 1);
}

int tctl_apply_state(tctl_ctx *ctx, const tctl_cp *u, tctl_cp *y) { return apply_common(ctx, u, y, 2); }

int tctl_map_constants(double beta_p, double gamma, double *beta, double *u_scale) {
  try {
    if (!(beta_p > 0.0) || !(gamma > 0.0) || !std::isfinite(beta_p) || !std::isfinite(gamma))
      fail(TCTL_E_ARG, "beta_p and gamma must be positive");
    if (!beta || !u_scale) fail(TCTL_E_ARG, "NULL output");
    // beta_p A^-alpha + (gamma / beta_p) A^alpha = beta_p (A^-alpha + (gamma / beta_p^2) A^alpha)
    *beta = gamma / (beta_p * beta_p);
    *u_scale = 1.0 / beta_p;
    return TCTL_OK;
  } catch (const Error &e) {
    return handle(nullptr, e);
  }
}

int tctl_truncate(tctl_ctx *ctx, const tctl_cp *x, tctl_cp *y, double eps) {
  Ctx *c = reinterpret_cast<Ctx *>(ctx);
  if (!c) return TCTL_E_ARG;
  try {
    check_cp(*c, x, "x", true);
    check_cp(*c, y, "y", false);
    if (!(eps >= TCTL_TRUNC_EPS_MIN && eps < 1.0))
      fail(TCTL_E_ARG, "eps must be in [1e-7, 1): smaller tolerances are below what the "
                       "Gram-based range finding resolves");
    WsGuard g(c->ws);
    size_t mk = c->ws.mark();
    Tucker t;
    tucker_alloc(*c, t, kCap);
    cp_to_tucker(*c, x->rank, x->w, x->U, false, t, eps / std::sqrt(2.0));
    const int s = tucker_to_cp(*c, t, false, eps / std::sqrt(2.0), y);
    c->ws.reset(mk);
    return s;
  } catch (const Error &e) {
    return handle(c, e);
  }
}

int tctl_pcg_solve(tctl_ctx *ctx, const tctl_cp *b, tctl_cp *x, tctl_stats *st) {
  Ctx *c = reinterpret_cast<Ctx *>(ctx);
  if (!c) return TCTL_E_ARG;
  try {
    check_cp(*c, b, "b", true);
    check_cp(*c, x, "x", false);
    WsGuard g(c->ws);
    try {
      return pcg_solve(*c, b, x, st);
    } catch (const Error &e) {
      // a tensor-core wait that ran out leaves unwritten outputs behind it;
      // report the timeout rather than whatever it caused downstream
      if (tcg_timed_out(*c))
        throw Error{TCTL_E_NUMERIC, "tensor-core GEMM: bounded mbarrier wait timed out"};
      throw;
    }
  } catch (const Error &e) {
    return handle(c, e);
  }
}

int tctl_fullgrid_solve(tctl_ctx *ctx, const double *y, double *u) {
  Ctx *c = reinterpret_cast<Ctx *>(ctx);
  if (!c) return TCTL_E_ARG;
  try {
    if (!y || !u || y == u) fail(TCTL_E_ARG, "y and u must be distinct device arrays");
    if (c->o.precision == 1) fullgrid_apply_tc(*c, y, u, 0);
    else fullgrid_apply(*c, y, u, 0);
    return TCTL_OK;
  } catch (const Error &e) {
    return handle(c, e);
  }
}

int tctl_fullgrid_state(tctl_ctx *ctx, const double *u, double *y) {
  Ctx *c = reinterpret_cast<Ctx *>(ctx);
  if (!c) return TCTL_E_ARG;
  try {
    if (!y || !u || y == u) fail(TCTL_E_ARG, "u and y must be distinct device arrays");
    if (c->o.precision == 1) fullgrid_apply_tc(*c, u, y, 1);
    else fullgrid_apply(*c, u, y, 1);
    return TCTL_OK;
  } catch (const Error &e) {
    return handle(c, e);
  }
}

int tctl_cp_alloc(tctl_ctx *ctx, int cap, tctl_cp *out) {
  Ctx *c = reinterpret_cast<Ctx *>(ctx);
  if (!c || !out || cap < 0) return TCTL_E_ARG;
  std::memset(out, 0, sizeof(*out));
  for (int l = 0; l < 3; ++l) out->n[l] = c->n;
  out->cap = cap;
  if (cap == 0) return TCTL_OK;
  if (cudaMallocAsync(&out->w, sizeof(double) * cap, c->st) != cudaSuccess) return TCTL_E_NOMEM;
  for (int l = 0; l < 3; ++l)
    if (cudaMallocAsync(&out->U[l], sizeof(double) * cap * (size_t)c->n, c->st) != cudaSuccess) {
      tctl_cp_free(ctx, out);
      return TCTL_E_NOMEM;
    }
  return TCTL_OK;
}

void tctl_cp_free(tctl_ctx *ctx, tctl_cp *cp) {
  if (!cp) return;
  // stream-ordered frees on the context's stream (no device-wide synchronisation)
  const cudaStream_t st = ctx ? reinterpret_cast<Ctx *>(ctx)->st : cudaStreamPerThread;
  if (cp->w) cudaFreeAsync(cp->w, st);
  for (int l = 0; l < 3; ++l)
    if (cp->U[l]) cudaFreeAsync(cp->U[l], st);
  cp->w = nullptr;
  cp->U[0] = cp->U[1] = cp->U[2] = nullptr;
  cp->rank = cp->cap = 0;
}

int tctl_get_eigs(tctl_ctx *ctx, int mode, double *lam, double *V) {
  Ctx *c = reinterpret_cast<Ctx *>(ctx);
  if (!c || mode < 0 || mode > 2) return TCTL_E_ARG;
  try {
    if (lam) to_host(*c, lam, c->lam[mode], c->n);
    if (V) to_host(*c, V, c->V[mode], (size_t)c->n * c->n);
    return TCTL_OK;
  } catch (const Error &e) {
    return handle(c, e);
  }
}

int tctl_get_stats(tctl_ctx *ctx, tctl_stats *st) {
  Ctx *c = reinterpret_cast<Ctx *>(ctx);
  if (!c || !st) return TCTL_E_ARG;
  c->stats.ws_peak_mb = (double)c->ws.peak / (1 << 20);
  c->stats.ws_size_mb = (double)c->ws.size / (1 << 20);
  *st = c->stats;
  return TCTL_OK;
}

long long tctl_launch_count(const tctl_ctx *ctx) {
  const Ctx *c = reinterpret_cast<const Ctx *>(ctx);
  return c ? c->launches : 0;
}

int tctl_solve_host(const double *coeffs, int n, double alpha, double beta, double eps_trunc,
                    const tctl_opts *opts, const double *yw, const double *yU, int S, double *uw,
                    double *uU, int cap, int *u_rank, tctl_stats *st) {
  if (!yw || !yU || S < 0 || !uw || !uU || cap < 0 || !u_rank) return TCTL_E_ARG;
  // a stream of its own (non-blocking): concurrent calls from several host
  // threads overlap on the GPU instead of serialising on the legacy default stream
  cudaStream_t hs = nullptr;
  if (cudaStreamCreateWithFlags(&hs, cudaStreamNonBlocking) != cudaSuccess) {
    set_noalloc_error("tctl_solve_host: cudaStreamCreateWithFlags failed");
    return TCTL_E_CUDA;
  }
  struct StreamGuard {
    cudaStream_t s;
    ~StreamGuard() {
      cudaStreamSynchronize(s);
      cudaStreamDestroy(s);
    }
  } guard{hs};
  tctl_ctx *ctx = nullptr;
  int s = tctl_setup(&ctx, coeffs, n, alpha, beta, eps_trunc, opts, hs);
  if (s != TCTL_OK) return s;
  Ctx *c = reinterpret_cast<Ctx *>(ctx);
  tctl_cp b{}, x{};
  try {
    s = tctl_cp_alloc(ctx, S, &b);
    if (s != TCTL_OK) fail(s, "allocation of y_Omega failed");
    s = tctl_cp_alloc(ctx, cap, &x);
    if (s != TCTL_OK) fail(s, "allocation of the solution failed");
    b.rank = S;
    to_dev(*c, b.w, yw, S);
    for (int l = 0; l < 3; ++l) to_dev(*c, b.U[l], yU + (size_t)l * n * S, (size_t)n * S);
    s = pcg_solve(*c, &b, &x, st);
    *u_rank = x.rank;
    to_host(*c, uw, x.w, x.rank);
    for (int l = 0; l < 3; ++l) to_host(*c, uU + (size_t)l * n * cap, x.U[l], (size_t)n * x.rank);
  } catch (const Error &e) {
    s = handle(c, e);
  }
  tctl_cp_free(ctx, &b);
  tctl_cp_free(ctx, &x);
  tctl_destroy(ctx);
  return s;
}

int tctl_solve_batch(tctl_batch_item *items, int count, double eps_trunc, const tctl_opts *opts,
                     int workers) {
  if (count < 0 || (count > 0 && !items) || workers < 1) return TCTL_E_ARG;
  // independent problems, dynamically scheduled over `workers` host threads; each
  // thread's launches go to its own per-thread default stream, so the problems
  // overlap on the device while every solve keeps its own host-side decisions
  std::atomic<int> next{0};
  auto run = [&]() {
    for (int i = next.fetch_add(1); i < count; i = next.fetch_add(1)) {
      tctl_batch_item &it = items[i];
      const auto t0 = std::chrono::steady_clock::now();
      it.status = tctl_solve_host(it.coeffs, it.n, it.alpha, it.beta, eps_trunc, opts, it.yw, it.yU,
                                  it.S, it.uw, it.uU, it.cap, &it.u_rank, it.st);
      const auto t1 = std::chrono::steady_clock::now();
      it.latency_ms = std::chrono::duration<double, std::milli>(t1 - t0).count();
    }
  };
  const int nt = std::min(workers, std::max(count, 1));
  std::vector<std::thread> pool;
  for (int t = 1; t < nt; ++t) pool.emplace_back(run);
  run();
  for (auto &th : pool) th.join();
  int worst = TCTL_OK;
  for (int i = 0; i < count; ++i)
    if (items[i].status != TCTL_OK && worst == TCTL_OK) worst = items[i].status;
  return worst;
}

int tctl_gemm(tctl_ctx *ctx, int digits, int trans_a, int trans_b, int m, int n, int k,
              double alpha, const double *A, int lda, const double *B, int ldb, double beta,
              double *C, int ldc) {
  Ctx *c = reinterpret_cast<Ctx *>(ctx);
  if (!c) return TCTL_E_ARG;
  try {
    if (m < 0 || n < 0 || k < 0) fail(TCTL_E_ARG, "negative dimension");
    if (digits != 0 && digits != 3 && digits != 4 && digits != 6)
      fail(TCTL_E_ARG, "digits must be 0, 3, 4 or 6");
    if ((m && n && k) && (!A || !B || !C)) fail(TCTL_E_ARG, "NULL matrix");
    if (lda < std::max(1, trans_a ? k : m) || ldb < std::max(1, trans_b ? n : k) || ldc < std::max(1, m))
      fail(TCTL_E_ARG, "leading dimension too small");
    if (m == 0 || n == 0) return TCTL_OK;
    WsGuard g(c->ws);
    if (digits == 0 || k == 0)
      gemm(*c, trans_a != 0, trans_b != 0, m, n, k, alpha, A, lda, 0, B, ldb, 0, beta, C, ldc, 0);
    else {
      gemm_tc_cm(*c, digits, trans_a != 0, trans_b != 0, m, n, k, alpha, A, lda, B, ldb, beta, C, ldc);
      tcg_check(*c);
    }
    return TCTL_OK;
  } catch (const Error &e) {
    return handle(c, e);
  }
}

int tctl_gemm_kr(tctl_ctx *ctx, int digits, int k, int ra, int rb, int n, double alpha,
                 const double *X, int ldx, const double *Y, int ldy, const double *B, int ldb,
                 double beta, double *C, int ldc) {
  Ctx *c = reinterpret_cast<Ctx *>(ctx);
  if (!c) return TCTL_E_ARG;
  try {
    if (k < 0 || ra < 0 || rb < 0 || n < 0) fail(TCTL_E_ARG, "negative dimension");
    if (digits != 0 && digits != 3 && digits != 4 && digits != 6)
      fail(TCTL_E_ARG, "digits must be 0, 3, 4 or 6");
    const long long m = (long long)ra * rb;
    if (m > (1 << 30)) fail(TCTL_E_ARG, "ra * rb too large");
    if ((m && n && k) && (!X || !Y || !B || !C)) fail(TCTL_E_ARG, "NULL matrix");
    if (ldx < std::max(1, k) || ldy < std::max(1, k) || ldb < std::max(1, k) ||
        ldc < std::max<long long>(1, m))
      fail(TCTL_E_ARG, "leading dimension too small");
    if (m == 0 || n == 0) return TCTL_OK;
    WsGuard g(c->ws);
    if (digits == 0 || k == 0) {
      size_t mk = c->ws.mark();
      double *KR = c->ws.dbl((size_t)std::max(k, 1) * m);
      if (k > 0) khatri_rao(*c, k, X, ldx, ra, Y, ldy, rb, KR, k);
      gemm(*c, true, false, (int)m, n, k, alpha, KR, std::max(k, 1), 0, B, ldb, 0, beta, C, ldc, 0);
      c->ws.reset(mk);
    } else {
      gemm_tc_kr(*c, digits, k, ra, rb, n, alpha, X, ldx, Y, ldy, B, ldb, beta, C, ldc);
      tcg_check(*c);
    }
    return TCTL_OK;
  } catch (const Error &e) {
    return handle(c, e);
  }
}

int tctl_tune_report(char *buf, int buflen) {
  if (!buf || buflen <= 0) return TCTL_E_ARG;
  const std::string js = tune_report();
  if ((int)js.size() + 1 > buflen) return TCTL_E_ARG;
  std::memcpy(buf, js.c_str(), js.size() + 1);
  return TCTL_OK;
}

int tctl_inject_wait_timeout(tctl_ctx *ctx, int count) {
  Ctx *c = reinterpret_cast<Ctx *>(ctx);
  if (!c || count < 0) return TCTL_E_ARG;
  c->withhold_copies = count;
  return TCTL_OK;
}

int tctl_expsum_fit(double alpha, double beta, double s_min, double s_max, double tol, double *t,
                    double *w, int cap, int *r, double *err) {
  try {
    if (!(alpha > 0.0 && alpha <= 1.0)) fail(TCTL_E_ARG, "alpha must be in (0, 1]");
    if (!(beta > 0.0) || !std::isfinite(beta)) fail(TCTL_E_ARG, "beta must be positive");
    if (!(s_min > 0.0 && s_max > s_min && std::isfinite(s_max)))
      fail(TCTL_E_ARG, "need 0 < s_min < s_max < inf");
    if (!(tol > 0.0 && tol < 1.0)) fail(TCTL_E_ARG, "tol must be in (0, 1)");
    if (cap < 0 || (cap > 0 && (!t || !w))) fail(TCTL_E_ARG, "NULL output buffer");
    const int s = expsum_fit_host(alpha, beta, s_min, s_max, tol, t, w, cap, r, err);
    if (s == TCTL_E_RANK_CAP) fail(s, "more terms than cap");
    if (s == TCTL_E_NUMERIC) fail(s, "fitted exponential sum misses the tolerance");
    return TCTL_OK;
  } catch (const Error &e) {
    return handle(nullptr, e);
  }
}

int tctl_precond_fit(double alpha, double beta, double s_min, double s_max, int r, double *theta,
                     double *p, double *delta) {
  try {
    if (!(alpha > 0.0 && alpha <= 1.0)) fail(TCTL_E_ARG, "alpha must be in (0, 1]");
    if (!(beta > 0.0) || !std::isfinite(beta)) fail(TCTL_E_ARG, "beta must be positive");
    if (!(s_min > 0.0 && s_max > s_min && std::isfinite(s_max)))
      fail(TCTL_E_ARG, "need 0 < s_min < s_max < inf");
    if (r < 2 || r > kPreRMax) fail(TCTL_E_ARG, "r must be in [2, 32]");
    if (!theta || !p) fail(TCTL_E_ARG, "NULL output buffer");
    std::vector<double> tau(r), q(r);
    const double d = pre_fit(alpha, beta, s_min, s_max, r, tau.data(), q.data());
    const double h0 = 1.0 / (s_min * (std::pow(s_min, -alpha) + beta * std::pow(s_min, alpha)));
    for (int k = 0; k < r; ++k) {
      theta[k] = tau[k] / s_min;
      p[k] = q[k] * h0;
    }
    if (delta) *delta = d;
    return TCTL_OK;
  } catch (const Error &e) {
    return handle(nullptr, e);
  }
}

int tctl_precond_dataset(int r, int n_samples, unsigned long long seed, int threads, float *X,
                         float *Y, double *delta) {
  try {
    if (r < 2 || r > kPreRMax) fail(TCTL_E_ARG, "r must be in [2, 32]");
    if (n_samples < 1 || !X || !Y) fail(TCTL_E_ARG, "need n_samples >= 1 and output buffers");
    precond_sample_inputs(n_samples, seed, X);
    expsum_dataset(FitTarget::Pre, r, n_samples, X, std::max(1, std::min(threads, 256)), Y, delta);
    return TCTL_OK;
  } catch (const Error &e) {
    return handle(nullptr, e);
  }
}

int tctl_expsum_dataset(int which, int r, int n_samples, unsigned long long seed, int threads,
                        float *X, float *Y, double *err) {
  try {
    if (which != 0 && which != 1) fail(TCTL_E_ARG, "which must be 0 (operator) or 1 (preconditioner)");
    if (r < 2 || r > kPreRMax) fail(TCTL_E_ARG, "r must be in [2, 32]");
    if (n_samples < 1 || !X || !Y) fail(TCTL_E_ARG, "need n_samples >= 1 and output buffers");
    precond_sample_inputs(n_samples, seed, X);
    expsum_dataset(which == 0 ? FitTarget::Op : FitTarget::Pre, r, n_samples, X,
                   std::max(1, std::min(threads, 256)), Y, err);
    return TCTL_OK;
  } catch (const Error &e) {
    return handle(nullptr, e);
  }
}

int tctl_mlp_model_size(int r) { return (r < 2 || r > kPreRMax) ? -1 : mlp_param_count(2 * r) + 8 + 4 * r; }

int tctl_mlp_train(int r, int n_samples, const float *X, const float *Y, int steps, int batch,
                   float lr, unsigned long long seed, float *model, float *loss) {
  try {
    if (r < 2 || r > kPreRMax) fail(TCTL_E_ARG, "r must be in [2, 32]");
    if (n_samples < 2 || !X || !Y || !model) fail(TCTL_E_ARG, "need data and a model buffer");
    if (steps < 1 || batch < 1 || batch > 4096 || !(lr > 0.0f)) fail(TCTL_E_ARG, "bad training parameters");
    mlp_train(r, n_samples, X, Y, steps, batch, lr, seed, model, loss);
    return TCTL_OK;
  } catch (const Error &e) {
    return handle(nullptr, e);
  }
}

int tctl_mlp_grad(int r, int batch, const float *params, const float *X, const float *T, float *grad,
                  float *loss) {
  try {
    if (r < 2 || r > kPreRMax) fail(TCTL_E_ARG, "r must be in [2, 32]");
    if (batch < 1 || !params || !X || !T || !grad || !loss) fail(TCTL_E_ARG, "NULL buffer");
    mlp_grad_host(r, batch, params, X, T, grad, loss);
    return TCTL_OK;
  } catch (const Error &e) {
    return handle(nullptr, e);
  }
}

int tctl_mlp_forward(int r, int n, const float *model, const float *X, float *Y) {
  try {
    if (r < 2 || r > kPreRMax) fail(TCTL_E_ARG, "r must be in [2, 32]");
    if (n < 1 || !model || !X || !Y) fail(TCTL_E_ARG, "NULL buffer");
    mlp_forward_host(r, n, model, X, Y, cudaStreamPerThread);
    return TCTL_OK;
  } catch (const Error &e) {
    return handle(nullptr, e);
  }
}

int tctl_get_expsum(tctl_ctx *ctx, int which, double *t, double *w, int *m, int cap, int *R) {
  Ctx *c = reinterpret_cast<Ctx *>(ctx);
  if (!c) return TCTL_E_ARG;
  try {
    if (which != 0 && which != 1) fail(TCTL_E_ARG, "which must be 0 (operator) or 1 (preconditioner)");
    if (cap < 0 || (cap > 0 && (!t || !w || !m))) fail(TCTL_E_ARG, "NULL output buffer");
    const std::vector<double> &tw = which == 0 ? c->op_terms_w : c->pre_terms_w;
    const std::vector<double> &tt = which == 0 ? c->op_terms_t : c->pre_terms_t;
    const std::vector<int> &tm = which == 0 ? c->op_terms_m : c->pre_terms_m;
    const int n = (int)tw.size();
    if (R) *R = n;
    const int k = std::min(n, cap);
    for (int i = 0; i < k; ++i) {
      t[i] = tt[i];
      w[i] = tw[i];
      m[i] = tm[i];
    }
    if (n > cap) fail(TCTL_E_RANK_CAP, "more terms than cap");
    return TCTL_OK;
  } catch (const Error &e) {
    return handle(c, e);
  }
}

int tctl_profile_enable(tctl_ctx *ctx, int on) {
  Ctx *c = reinterpret_cast<Ctx *>(ctx);
  if (!c) return TCTL_E_ARG;
  c->prof = (on != 0);
  c->prof_phases = (on == 2);
  c->prof_recs.clear();
  c->prof_used = 0;
  return TCTL_OK;
}

int tctl_profile_report(tctl_ctx *ctx, char *buf, int buflen) {
  Ctx *c = reinterpret_cast<Ctx *>(ctx);
  if (!c || !buf || buflen <= 0) return TCTL_E_ARG;
  try {
    TCTL_CUDA(cudaStreamSynchronize(c->st));
    struct Agg {
      std::string name;
      long long launches = 0;
      double ms = 0, flops = 0, mma = 0, bytes = 0;
    };
    std::vector<Agg> agg;
    for (const ProfRec &r : c->prof_recs) {
      std::string nm(r.name);
      nm.erase(std::remove(nm.begin(), nm.end(), '('), nm.end());
      const size_t lt = nm.find('<');
      if (lt != std::string::npos) nm = nm.substr(0, lt);
      if (c->prof_phases && r.phase) nm = std::string(r.phase) + "/" + nm;
      if (c->prof_phases && r.outer) nm = std::string(r.outer) + "/" + nm;
      float ms = 0;
      TCTL_CUDA(cudaEventElapsedTime(&ms, r.a, r.b));
      auto it = std::find_if(agg.begin(), agg.end(), [&](const Agg &a) { return a.name == nm; });
      if (it == agg.end()) {
        agg.push_back(Agg{nm});
        it = agg.end() - 1;
      }
      it->launches++;
      it->ms += ms;
      it->flops += r.flops;
      it->mma += r.mma_flops;
      it->bytes += r.bytes;
    }
    std::string js = "{";
    for (size_t i = 0; i < agg.size(); ++i) {
      char tmp[640];
      std::snprintf(tmp, sizeof(tmp),
                    "%s\"%s\": {\"launches\": %lld, \"ms\": %.6f, \"flops\": %.6e, \"mma_flops\": %.6e, "
                    "\"bytes\": %.6e}",
                    i ? ", " : "", agg[i].name.c_str(), agg[i].launches, agg[i].ms, agg[i].flops,
                    agg[i].mma, agg[i].bytes);
      js += tmp;
    }
    js += "}";
    if ((int)js.size() + 1 > buflen) fail(TCTL_E_ARG, "profile report buffer too small");
    std::memcpy(buf, js.c_str(), js.size() + 1);
    c->prof_recs.clear();
    c->prof_used = 0;
    return TCTL_OK;
  } catch (const Error &e) {
    return handle(c, e);
  }
}

void tctl_destroy(tctl_ctx *ctx) {
  Ctx *c = reinterpret_cast<Ctx *>(ctx);
  if (!c) return;
  // the library is built with per-thread default streams: a NULL stream is the
  // calling thread's, and nothing here synchronises the whole device
  cudaStreamSynchronize(c->st);
  for (cudaEvent_t e : c->prof_pool) cudaEventDestroy(e);
  for (void *p : c->owned) cudaFreeAsync(p, c->st);
  cudaStreamSynchronize(c->st);
  stage_release(c->hstage);
  delete c;
}

const char *tctl_last_error(const tctl_ctx *ctx) {
  const Ctx *c = reinterpret_cast<const Ctx *>(ctx);
  if (c && !c->err.empty()) return c->err.c_str();
  return g_last_error.c_str();
}

}  // extern "C"
