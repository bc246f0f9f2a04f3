// Internal declarations of the tensorctl library (not part of the C ABI).
#pragma once

#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <chrono>
#include <cstdint>
#include <cstdio>
#include <string>
#include <vector>

#include "../../include/tensorctl.h"

#if defined(__has_include)
#if __has_include(<nvtx3/nvToolsExt.h>)
#include <nvtx3/nvToolsExt.h>
#define TCTL_HAVE_NVTX 1
#endif
#endif
#ifndef TCTL_HAVE_NVTX
#define TCTL_HAVE_NVTX 0
#endif

namespace tctl {

// Errors are C++ exceptions inside the library; every extern "C" entry point
// catches them and turns them into a status code plus tctl_last_error().
struct Error {
  int code;
  std::string msg;
};

[[noreturn]] void fail(int code, const std::string &msg);
void check_cuda(cudaError_t e, const char *what);
#define TCTL_CUDA(call) ::tctl::check_cuda((call), #call)

// Bump allocator over one device buffer; mark()/reset() scope temporaries.
struct Arena {
  char *base = nullptr;
  size_t size = 0;
  size_t top = 0;
  size_t peak = 0;
  void *alloc(size_t bytes);
  double *dbl(size_t count) { return static_cast<double *>(alloc(count * sizeof(double))); }
  int *i32(size_t count) { return static_cast<int *>(alloc(count * sizeof(int))); }
  size_t mark() const { return top; }
  void reset(size_t m) { top = m; }
};

// Separable diagonal operator in the tensor eigenbasis:
//   D = sum_k w[k] diag(E_1[:,k]) x diag(E_2[:,k]) x diag(E_3[:,k]),
// plus a per-mode orthonormal basis B_l (n x rD_l) of span(E_l) with
// E_l = B_l Z_l (Z_l: rD_l x R), used to keep the cost of applications
// proportional to rD_l rather than R.
struct Sep {
  int R = 0;
  double *w = nullptr;
  double *E[3] = {nullptr, nullptr, nullptr};
  int rD[3] = {0, 0, 0};
  double *B[3] = {nullptr, nullptr, nullptr};
  double *Z[3] = {nullptr, nullptr, nullptr};
  std::vector<double> w_host;
};

// Tucker tensor in arena/context memory: Q[l] n x r[l] (ld n, orthonormal
// columns), core r0 x r1 x r2 (first index fastest).
struct Tucker {
  int r[3] = {0, 0, 0};
  double *Q[3] = {nullptr, nullptr, nullptr};
  double *core = nullptr;
  int cap = 0;
};

// One profiled launch (opt-in: events around every kernel of the context).
struct ProfRec {
  const char *name;
  const char *outer;
  const char *phase;
  cudaEvent_t a, b;
  double flops;      // algorithmic FP64-class flops (GEMMs)
  double mma_flops;  // BF16 tensor-core flops of the digit products (2 MNK per product)
  double bytes;      // algorithmic global-memory bytes (operands read once, results written once)
};

struct Ctx {
  int n = 0;
  double alpha = 0, beta = 0, eps = 0;
  tctl_opts o{};
  cudaStream_t st = nullptr;
  double *coef = nullptr;            // 3 x (n+1)
  double *d[3] = {}, *e[3] = {};     // tridiagonal A_(l)
  double *lam[3] = {}, *V[3] = {};   // eigenpairs
  std::vector<double> lam_host[3];
  double s_min = 0, s_max = 0;
  Sep op, pre;
  double op_rel_err = 0;
  int expsum_used = 0;                     // 0 sinc, 1 fitted, 2 learned
  double op_learned_err = 0;               // expsum_src 2: the learned sum's measured error
  double t_fit_ms = 0;                     // host time of the spectral fits (set-up trace)
  double sinc24_err = 0;                   // expsum_src 2: sinc with 24 terms per function
  Sep state;                               // A^-alpha (state equation), built on first use
  double state_rel_err = 0;
  int pre_used = 0;                        // preconditioner: 0 K-node NNLS, 1 fitted, 2 learned, 3 anisotropic
  double *W[3] = {nullptr, nullptr, nullptr};  // pre_src 3: W_l = S^T V_l (sine basis <- eigenbasis)
  double *lamB[3] = {nullptr, nullptr, nullptr};  // pre_src 3: b0_l mu_k
  double b0[3] = {0, 0, 0};
  std::vector<double> coef_host;          // 3 x (n + 1) coefficients
  double pre_delta = 0;                    // its measured max |P F2 - 1|
  std::vector<double> op_terms_w, op_terms_t, pre_terms_w, pre_terms_t;  // host copies
  std::vector<int> op_terms_m, pre_terms_m;
  Arena ws;
  // pinned host staging for small transfers: [0, kStageRead) receives
  // device-to-host reads, the rest is a ring of host-to-device uploads whose
  // space is reused once a read has synchronised the stream
  char *hstage = nullptr;
  size_t hstage_top = 0;
  double *full_tmp = nullptr;        // n^3 temporary of the FP64 full-grid solve
  // tensor-core full grid: digit planes of V_l^T / V_l, row exponents, two FP32
  // n^3 buffers, column exponents, error flag (allocated on first use)
  __nv_bfloat16 *tc_w[6] = {};
  int *tc_e[6] = {};
  float *tc_x[2] = {};
  int *tc_f = nullptr;
  __nv_bfloat16 *tc_xd = nullptr;    // X digit blocks of one mode product
  int *tc_err = nullptr;
  tctl_stats stats{};
  std::string err;
  long long launches = 0;
  uint64_t rng_counter = 0;
  std::vector<void *> owned;         // device allocations freed at destroy
  int *tcg_err = nullptr;            // tensor-core GEMM wait-timeout flag (device)
  int digits = 6;                    // digit count of the rank-structured tensor-core contractions
  int withhold_copies = 0;           // failure-detection test: GEMM launches left to starve
  // digit planes of constant tensor-core operands (the operator's factor
  // matrices), keyed by the operand's address, strides and split geometry
  struct TcKept {
    const double *p;
    long long s0, s1, sk;
    int d, R, K, D, TR;
    int *e;
    void *planes;
  };
  std::vector<TcKept> tc_keep;
  bool prof = false;                 // record events around every launch
  bool trace = false;                // TCTL_TRACE=1: per-step ranks on stderr
  std::vector<std::string> interned;  // stable storage of generated profile names
  const char *intern(const char *s) {
    for (const std::string &x : interned)
      if (x == s) return x.c_str();
    if (interned.size() >= 4096) return "dgemm[...]";
    interned.reserve(4096);  // no reallocation: returned pointers stay valid
    interned.emplace_back(s);
    return interned.back().c_str();
  }
  bool prof_phases = false;          // report "phase/kernel" names
  std::vector<ProfRec> prof_recs;
  std::vector<cudaEvent_t> prof_pool;
  size_t prof_used = 0;
  double next_flops = 0;             // algorithmic flops of the next launch (GEMMs)
  double next_mma = 0;               // BF16 tensor-core flops of the next launch
  double next_bytes = 0;             // algorithmic bytes of the next launch (memory-bound kernels)
  const char *next_tag = nullptr;    // profile name of the next launch (GEMM call site)
  const char *phase = nullptr;       // current algorithm phase (profile grouping)
  const char *outer = nullptr;       // current PCG step (profile grouping)
  double *dmalloc(size_t count);
  cudaEvent_t prof_event();
};

// ------------------------------------------------------------ launch wrapper
// Every kernel launch of the library goes through LAUNCH so the context can
// count them and check the launch status.
#define LAUNCH(ctx, kernel, grid, block, smem, ...)                                \
  do {                                                                            \
    cudaEvent_t tctl_ev_a = nullptr, tctl_ev_b = nullptr;                         \
    if ((ctx).prof) {                                                             \
      tctl_ev_a = (ctx).prof_event();                                             \
      tctl_ev_b = (ctx).prof_event();                                             \
      ::tctl::check_cuda(cudaEventRecord(tctl_ev_a, (ctx).st), "cudaEventRecord"); \
    }                                                                             \
    kernel<<<(grid), (block), (smem), (ctx).st>>>(__VA_ARGS__);                   \
    ::tctl::check_cuda(cudaGetLastError(), #kernel);                              \
    (ctx).launches++;                                                             \
    if ((ctx).prof) {                                                             \
      ::tctl::check_cuda(cudaEventRecord(tctl_ev_b, (ctx).st), "cudaEventRecord"); \
      (ctx).prof_recs.push_back({(ctx).next_tag ? (ctx).next_tag : #kernel, (ctx).outer, (ctx).phase, \
                                 tctl_ev_a, tctl_ev_b, (ctx).next_flops, (ctx).next_mma,         \
                                 (ctx).next_bytes});                              \
    }                                                                             \
    (ctx).next_flops = 0;                                                         \
    (ctx).next_mma = 0;                                                           \
    (ctx).next_bytes = 0;                                                         \
    (ctx).next_tag = nullptr;                                                     \
  } while (0)

// Scoped algorithm phase for the per-kernel trace (names must be literals).
// Each scope is also an NVTX range (no-op unless a profiler is attached), so
// ncu / nsys can filter kernels by PCG step and phase (ncu --nvtx).
struct PhaseScope {
  Ctx &c;
  const char *Ctx::*slot;
  const char *prev;
  PhaseScope(Ctx &cc, const char *Ctx::*s, const char *p) : c(cc), slot(s), prev(cc.*s) {
    c.*s = p;
#if TCTL_HAVE_NVTX
    nvtxRangePushA(p);
#endif
  }
  ~PhaseScope() {
#if TCTL_HAVE_NVTX
    nvtxRangePop();
#endif
    c.*slot = prev;
  }
};
#define TCTL_CAT2(a, b) a##b
#define TCTL_CAT(a, b) TCTL_CAT2(a, b)
#define TCTL_PHASE(ctx, name) \
  ::tctl::PhaseScope TCTL_CAT(tctl_phase_scope_, __LINE__)(ctx, &::tctl::Ctx::phase, name)
#define TCTL_OUTER(ctx, name) \
  ::tctl::PhaseScope TCTL_CAT(tctl_outer_scope_, __LINE__)(ctx, &::tctl::Ctx::outer, name)

// ------------------------------------------------------------ tc_gemm.cu
// Operand of the digit-split tensor-core GEMM: rows r (m of A, j of B),
// contracted index k, batch item i; element at
// p + i sb + (r % d) s0 + (r / d) s1 + k sk.
// With q set, the operand is a Khatri-Rao product formed on the fly (no batch):
// element (r, k) = p[(r % d) s0 + k sk] * q[(r / d) s1 + k sk], the value
// khatri_rao() would have stored, so both forms give identical results.
struct TcOpnd {
  const double *p;
  long long s0, s1, sk, sb;
  int d;
  const double *q = nullptr;
  // the operand is owned by the context and never changes: its digit planes
  // are cut on first use and kept (Ctx::tc_keep)
  bool keep = false;
};
// C[b sC' + (m % cd) cm0 + (m / cd) cm1 + j cj] = alpha sum_k A(m, k) B(j, k) + beta C,
// batch item b of A / B = b / divA, b / divB; digits 3 (21-bit), 4 (28-bit) or 6 (42-bit).
void gemm_tc(Ctx &c, int digits, int M, int N, int K, int batch, int divA, int divB,
             double alpha, const TcOpnd &A, const TcOpnd &B, double beta, double *C,
             long long cm0, long long cm1, int cd, long long cj, long long cb);
bool gemm_tc_fits(int M, int N, int K, int batch);
// One GEMM of a grouped tensor-core launch (no batch):
// C[(m % cd) cm0 + (m / cd) cm1 + j cj] = alpha sum_k A(m, k) B(j, k) + beta C.
struct TcItem {
  int M, N, K;
  TcOpnd A, B;
  double alpha, beta;
  double *C;
  long long cm0, cm1;
  int cd;
  long long cj;
};
// Independent digit-split GEMMs in one launch (up to 4 per launch) plus one
// grouped reduction of their K-chunk partial sums; digits as gemm_tc.
void gemm_tc_group(Ctx &c, int digits, int count, const TcItem *items);
// gemm() semantics; the tensor cores when opts.tc_gemm and the shape pays, FP64 otherwise
void gemm_x(Ctx &c, int digits, bool ta, bool tb, int m, int n, int k, double alpha,
            const double *A, int lda, long long sA, const double *B, int ldb, long long sB,
            double beta, double *C, int ldc, long long sC, int batch = 1, int divA = 1,
            int divB = 1, bool a_kept = false);
// C (ra rb x n) = alpha KR(X, Y)^T B + beta C on the tensor cores, the
// Khatri-Rao rows formed inside the digit split (X k x ra, Y k x rb, B k x n).
void gemm_tc_kr(Ctx &c, int digits, int k, int ra, int rb, int n, double alpha, const double *X,
                int ldx, const double *Y, int ldy, const double *B, int ldb, double beta, double *C,
                int ldc);
// Column-major C = alpha op(A) op(B) + beta C on the tensor cores whatever the shape.
void gemm_tc_cm(Ctx &c, int digits, bool ta, bool tb, int m, int n, int k, double alpha,
                const double *A, int lda, const double *B, int ldb, double beta, double *C, int ldc);
// Raises TCTL_E_NUMERIC if a tensor-core GEMM timed out on a wait (synchronizes).
void tcg_check(Ctx &c);
// Reads and clears the wait-timeout flag without raising (synchronizes).
bool tcg_timed_out(Ctx &c);
// JSON list of the tile autotuner's decisions so far (process-wide).
std::string tune_report();

// ------------------------------------------------------------ linalg.cu
// C = alpha op(A) op(B) + beta C, column-major, batched with element strides;
// batch item b uses A + (b / divA) * sA, B + (b / divB) * sB, C + b * sC.
void gemm(Ctx &c, bool ta, bool tb, int m, int n, int k, double alpha,
          const double *A, int lda, long long sA, const double *B, int ldb,
          long long sB, double beta, double *C, int ldc, long long sC,
          int batch = 1, int divA = 1, int divB = 1);
// One GEMM of a group: C = alpha op(A) op(B) + beta C, column-major.
struct GemmSpec {
  bool ta, tb;
  int m, n, k;
  double alpha;
  const double *A;
  int lda;
  const double *B;
  int ldb;
  double beta;
  double *C;
  int ldc;
};
// Independent GEMMs in as few launches as their transpositions allow (one
// launch plus one split-K reduction per transposition pair, up to 8 items).
void gemm_group(Ctx &c, int count, const GemmSpec *spec);
// out[:, a + ra*b] = A[:, a] .* B[:, b]   (n rows, Khatri-Rao of columns)
void khatri_rao(Ctx &c, int n, const double *A, int lda, int ra, const double *B,
                int ldb, int rb, double *out, int ldo);
// Symmetric eigendecomposition (one-sided cyclic Jacobi, parallel ordering) of
// `batch` m x m matrices (ld m, contiguous); eigenvalues descending in lam
// (batch x m), eigenvectors as columns in Vout (batch x m x m). m <= 64.
void sym_eig(Ctx &c, int m, int batch, const double *A, double *lam, double *Vout);
// Several symmetric eigenproblems of different sizes (<= 64) in one launch.
void sym_eig_multi(Ctx &c, int count, const int *m, const double *const *A, double *const *lam,
                   double *const *Vout);
// Orthonormal basis of span(Y) (n x m, m <= 64) by pivoted Cholesky of Y^T Y:
// columns whose residual norm falls below tol * (reference) are dropped, where
// reference = max column norm (relative=true) or 1 (relative=false). Writes Q
// (n x r, ld n) and returns r (r <= min(m, rcap)). Two passes (CholeskyQR2).
// orth for `count` independent matrices (batched launches, one read-back per pass).
void orth_multi(Ctx &c, int count, int n, const int *m, double *const *Y, const int *ldy, double tol,
                bool relative, const int *rcap, double *const *Q, int *r_out);
int orth(Ctx &c, int n, int m, const double *Y, int ldy, double tol, bool relative,
         int rcap, double *Q);
// Column 2-norms of an n x m matrix.
void col_norms(Ctx &c, int n, int m, const double *A, int lda, double *out);
void scale_cols(Ctx &c, int n, int m, double *A, int lda, const double *s, bool inverse);
void fill_gaussian(Ctx &c, double *x, size_t count, uint64_t seed);
// Up to three fills in one launch, each with the draws fill_gaussian gives its seed.
void fill_gaussian_multi(Ctx &c, int count, double *const *x, const size_t *n, const uint64_t *seed);
void fill_zero(Ctx &c, double *x, size_t count);
void copy_d(Ctx &c, double *dst, const double *src, size_t count);
// Several device-to-device copies (dst[i] <- src[i], n[i] doubles) in one launch.
void copy_multi(Ctx &c, int count, double *const *dst, const double *const *src, const size_t *n);
void axpby(Ctx &c, size_t count, double a, const double *x, double b, double *y);
// Host copies. to_host / read_host return once the data is on the host (the
// context stream is synchronised); to_dev / write_dev are stream-ordered and
// the caller's buffer may be reused at once.
constexpr size_t kStageBytes = 1 << 20, kStageRead = 256 << 10;
char *stage_acquire();
void stage_release(char *p);
void read_host(Ctx &c, void *dst, const void *src, size_t bytes);
void write_dev(Ctx &c, void *dst, const void *src, size_t bytes);
void to_host(Ctx &c, double *dst, const double *src, size_t count);
void to_dev(Ctx &c, double *dst, const double *src, size_t count);

// ------------------------------------------------------------ eig.cu
// Assemble A_(l) from coef and compute all three eigendecompositions in FP64.
void setup_eigs(Ctx &c);


// ------------------------------------------------------------ spectral.cu
int expsum_fit_host(double a, double b, double smin, double smax, double tol, double *t, double *w,
                    int cap, int *r, double *err);
double sinc_err_at_rank(double a, double b, double smin, double smax, int r);
// ------------------------------------------------------------ learned.cu
constexpr int kMlpIn = 4, kMlpH = 64, kPreRMax = 32;
// What an r-term exponential sum sum_k w_k exp(-t_k s) approximates: the
// preconditioner's h(s) = 1 / (s F2(s)) (P = s sum) or the operator's
// g(s) = F2(s) / s (F2 = s sum).
enum class FitTarget { Pre, Op };
// Levenberg-Marquardt r-term fit (free log-nodes and log-weights); tau in
// x = s / s_min units, q the weights of exp(-tau x) for target(s_min x) /
// target(s_min). Returns the measured max |sum / target - 1|.
double expsum_fit_r(FitTarget tg, double a, double b, double smin, double smax, int r, double *tau_out,
                    double *q_out);
double sum_rel_err(FitTarget tg, const double *t, const double *w, int r, double a, double b,
                   double smin, double smax);
std::vector<double> weights_nnls(FitTarget tg, const std::vector<double> &theta, double a, double b,
                                 double smin, double smax);
void expsum_dataset(FitTarget tg, int r, int N, const float *X, int threads, float *Y, double *delta);
double pre_fit(double a, double b, double smin, double smax, int r, double *tau_out, double *q_out);
double pre_delta(const double *theta, const double *p, int r, double a, double b, double smin,
                 double smax);
std::vector<double> pre_weights_nnls(const std::vector<double> &theta, double a, double b,
                                     double smin, double smax);
int mlp_param_count(int O);
void precond_sample_inputs(int N, uint64_t seed, float *X);

void mlp_train(int r, int N, const float *X, const float *Y, int steps, int B, float lr,
               uint64_t seed, float *model, float *loss_out);
void mlp_grad_host(int r, int B, const float *params, const float *X, const float *T, float *grad,
                   float *loss);
void mlp_forward_host(int r, int n, const float *model, const float *X, float *Yout, cudaStream_t st);
// Lawson-Hanson NNLS, A M x K column-major.
std::vector<double> nnls_solve(const std::vector<double> &A, int M, int K, const std::vector<double> &b);
void ensure_state_sep(Ctx &c);
void setup_spectral(Ctx &c);
// The same in two parts: host fits of the sums (needs s_min, s_max only) and
// the device factor matrices (needs the eigenpairs).
void setup_spectral_fit(Ctx &c);
void setup_spectral_build(Ctx &c);
void fullgrid_apply(Ctx &c, const double *y, double *u, int which);

// ------------------------------------------------------------ tc_modeprod.cu
bool tc_fullgrid_supported(int n);
void fullgrid_apply_tc(Ctx &c, const double *y, double *u, int which);

// ------------------------------------------------------------ tucker.cu
struct TuckerOps;
// canonical (device) -> Tucker in the tensor eigenbasis (to_eig=true: factors
// are first multiplied by V_l^T), lossless up to the pivoting tolerance.
void cp_to_tucker(Ctx &c, int m, const double *w, double *const U[3], bool to_eig,
                  Tucker &out, double eps_core);
// Tucker -> canonical (T2C, slice SVDs), optional back transform with V_l.
int tucker_to_cp(Ctx &c, const Tucker &x, bool from_eig, double eps, tctl_cp *y);
void tucker_alloc(Ctx &c, Tucker &t, int cap);
void tucker_copy(Ctx &c, const Tucker &src, Tucker &dst);
// y = trunc(D .* x) with D separable (eigenbasis), eps relative.
void sep_apply_trunc(Ctx &c, const Sep &D, const Tucker &x, Tucker &y, double eps);
// z = trunc(a x + b y). With norm_out, ||a x + b y|| (before truncation) is
// returned there, and the truncation is skipped when it is <= keep_below.
void tucker_axpby_trunc(Ctx &c, double a, const Tucker &x, double b, const Tucker &y,
                        Tucker &z, double eps, double *norm_out = nullptr,
                        double keep_below = -1.0);
double tucker_inner(Ctx &c, const Tucker &x, const Tucker &y);
// Truncate a Tucker tensor in place by HOSVD of its core (eps relative).
void tucker_hosvd_trunc(Ctx &c, Tucker &x, double eps);
// Apply V_l (from_eig) or V_l^T (to_eig) to the Tucker factors in place.
void tucker_basis_change(Ctx &c, Tucker &x, bool to_eig);
// Q_l <- M_l^T Q_l (transpose) or M_l Q_l for n x n matrices M_l.
void tucker_factor_change(Ctx &c, Tucker &x, double *const M[3], bool transpose);

// Records the message returned by tctl_last_error(NULL) (entry points without a context).
void set_noalloc_error(const std::string &msg);

// ------------------------------------------------------------ pcg.cu
int pcg_solve(Ctx &c, const tctl_cp *b, tctl_cp *x, tctl_stats *st);


// Thread-block cluster helpers: this CTA's rank, the shared::cluster address of
// a shared variable as held by another CTA of the cluster, remote stores and
// loads, and the cluster-wide barrier (release / acquire).
__device__ __forceinline__ uint32_t cl_rank() {
  uint32_t r;
  asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
  return r;
}
// shared::cluster address of this CTA's shared variable p as held by CTA `rank`
__device__ __forceinline__ uint32_t cl_map(const void *p, uint32_t rank) {
  const uint32_t a = (uint32_t)__cvta_generic_to_shared(p);
  uint32_t r;
  asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"(a), "r"(rank));
  return r;
}
__device__ __forceinline__ void cl_st(uint32_t addr, double v) {
  asm volatile("st.shared::cluster.f64 [%0], %1;" ::"r"(addr), "d"(v) : "memory");
}
__device__ __forceinline__ int cl_ld(uint32_t addr) {
  int v;
  asm volatile("ld.shared::cluster.s32 %0, [%1];" : "=r"(v) : "r"(addr) : "memory");
  return v;
}
__device__ __forceinline__ void cl_sync() {
  asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;" ::
                   : "memory");
}


}  // namespace tctl
