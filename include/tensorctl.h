/*
 * tensorctl — C ABI of the GPU solver for the control equation of the tensor
 * method for optimal control constrained by a fractional 3D elliptic operator
 * with separable variable coefficients (arXiv 2006.09314).
 *
 * The library solves, on one GPU, the discrete control equation
 *
 *     F2(A) u = y_Omega,   F2(A) = A^-alpha + beta A^alpha                  (1)
 *
 * (Section 3.1, eq. "Lagrange_cont", with the paper's beta_p = 1 and
 * gamma = beta; a general (beta_p, gamma) pair maps to beta = gamma/beta_p^2
 * and u_paper = u/beta_p), where A = A_1 (+) A_2 (+) A_3 is the Kronecker sum
 * of the 1D finite-difference Sturm-Liouville matrices of Section 3.2 on n
 * interior points per axis (h = 1/(n+1)), by rank-truncated preconditioned CG
 * (Appendix 2, Algorithm 1) in the eigenbasis of the three 1D operators
 * (Section 3.3, eqs. "DiagGen", "DiagKron3D").
 *
 * Conventions shared by every entry point
 *   - Return value: TCTL_OK (0) or a negative TCTL_E_* code. No exception
 *     crosses the ABI; the library never exits, aborts or traps on the device.
 *     tctl_last_error() returns a message for the last failing call.
 *   - All work of a context is ordered on the CUDA stream given at setup.
 *   - Canonical tensors (tctl_cp) live in DEVICE memory and are owned by the
 *     caller (tctl_cp_alloc/tctl_cp_free are conveniences). Factor matrices
 *     are column-major with leading dimension n: U[l][i + k*n] is entry i of
 *     the factor of term k in mode l. Used terms: 0..rank-1 <= cap.
 *   - Full-grid arrays are DEVICE n^3 arrays with x1 fastest:
 *     y[i1 + n*i2 + n*n*i3].
 *   - Inputs and outputs must not alias, except where stated.
 *   - The context owns everything it allocates and frees it in tctl_destroy.
 */
#ifndef TENSORCTL_H
#define TENSORCTL_H

#ifdef __cplusplus
extern "C" {
#endif

enum {
  TCTL_OK = 0,
  TCTL_E_ARG = -1,          /* invalid argument (sizes, pointers, ranges)        */
  TCTL_E_COEFF = -2,        /* a coefficient a_l(x) <= 0 or not finite           */
  TCTL_E_CUDA = -3,         /* a CUDA runtime call failed                        */
  TCTL_E_NOMEM = -4,        /* device allocation failed                          */
  TCTL_E_RANK_CAP = -5,     /* output rank exceeded a capacity; result is capped */
  TCTL_E_NOT_CONVERGED = -6,/* PCG reached max_iter; x holds the last iterate    */
  TCTL_E_NAN = -7,          /* a NaN/Inf appeared in a reduction                 */
  TCTL_E_NUMERIC = -8       /* a numerical kernel failed (e.g. no convergence)   */
};

typedef struct tctl_ctx tctl_ctx;

/* Canonical tensor T = sum_k w[k] U[0][:,k] x U[1][:,k] x U[2][:,k]
 * (Appendix 1, "CP_form"), DEVICE memory, caller-owned. */
typedef struct {
  int n[3];      /* mode sizes (all equal to the context's n)        */
  int rank;      /* number of terms in use                           */
  int cap;       /* allocated number of terms                        */
  double *w;     /* [cap] weights                                    */
  double *U[3];  /* U[l]: n[l] x cap, column-major, leading dim n[l] */
} tctl_cp;

typedef struct {
  double pcg_rtol;    /* stop when ||R_k|| <= pcg_rtol ||B|| (default 1e-7)          */
  int max_iter;       /* Algorithm 1's k_max (default 100)                            */
  double op_tol;      /* target max relative error of the separable F2 on the
                         spectral interval (default 1e-8)                              */
  int r_pre;          /* nodes of the preconditioner exp-sum (default 24)             */
  int rank_cap;       /* maximal Tucker rank per mode inside the solver (default and
                         maximum 64)                                                  */
  int precision;      /* full-grid mode products: 0 = FP64 FMA (default); 1 = tensor
                         cores, BF16 digit split (5 x 7-bit digits, shared row/column
                         exponents, 15 products, exact leading levels, FP32 storage
                         between products; ~1e-7 relative per solve; needs
                         n % 128 == 0, n <= 1024). The rank-structured solver's
                         contractions are chosen by tc_gemm.                          */
  int basis;          /* 1 = PCG vectors kept in eigenbasis coordinates (default);
                         0 = paper form, mode products with V_l in every apply         */
  int expsum_src;     /* separable F2: 0 = sinc quadrature (Section 3.4); 1 = fitted
                         exponential sum of F2(s)/s (default; falls back to sinc
                         when the fit misses op_tol); 2 = learned sum (op_model)      */
  int paper_end_rows; /* 1 = the paper's printed end rows of A_(l) (default 0)        */
  double eps_final;   /* truncation of the returned solution; <= 0 means eps/10       */
  unsigned long long seed; /* seed of the sketching random numbers (default 1)       */
  double range_tol;   /* range finder of the truncated Hadamard products F2 .* x and
                         P .* x: a direction of the mode-l sketch is kept while its
                         residual exceeds max(1e-8, range_tol * eps_trunc) of the
                         largest sketch column (default 0.03)                          */
  int tc_gemm;        /* rank-structured contractions (sketches, core projection of
                         the Hadamard products): 1 = tensor cores, BF16 digit split
                         (6 digits = 42 bits for sketches and core; FP32
                         accumulate with exact low levels, FP64 result; default);
                         0 = FP64 FMA. Gram matrices, orthonormalisation and HOSVD
                         always run in FP64.                                           */
  int pre_src;        /* preconditioner exp-sum P(s) = s sum_k p_k exp(-theta_k s) ~ 1/F2:
                         0 = r_pre geometric nodes, NNLS weights (default); 1 = pre_r free
                         nodes fitted at set-up (tctl_precond_fit); 2 = nodes predicted by a
                         trained network (pre_model, tctl_mlp_train), weights re-solved
                         by NNLS. 1 and 2 are used only if their measured
                         delta = max |P F2 - 1| <= pre_delta_max, else 0 is used.
                         3 = case (A) of Section 3.5: 1/F2 of the anisotropic
                         constant-coefficient Laplacian B0 = sum_l b0_l Delta_l,
                         b0_l = (max a_l + min a_l)/2, applied in its sine basis
                         (W_l = S^T V_l, 3 n^2 doubles); r_pre nodes, NNLS weights.    */
  int pre_r;          /* terms of pre_src 1 / 2 (default 12; the network's r)          */
  const float *pre_model; /* HOST model blob of tctl_mlp_train (pre_src 2)              */
  double pre_delta_max;   /* acceptance bound of pre_src 1 / 2 (default 0.25)           */
  int workspace_mb;   /* device workspace arena of the context in MiB; 0 = automatic
                         (sized from n); too small an arena fails with TCTL_E_NOMEM   */
  const float *op_model; /* HOST model blob of tctl_mlp_train for expsum_src 2: the
                         network's op_r nodes of g(s) = F2(s)/s, weights re-solved by
                         NNLS; used only if the measured max relative error of F2 on
                         [s_min, s_max] is <= op_judge, else the sinc quadrature
                         (at op_tol) is used; alpha = 1 always uses sinc          */
  int op_r;           /* terms of the learned operator sum (default 16)              */
  double op_judge;    /* acceptance bound of the learned operator sum (default 1e-7)  */
  int tune;           /* 1 = tile autotuner for the tensor-core GEMMs: the contracted
                         length per CTA (64, 128 or 256) of each shape class is timed
                         at its first use and kept for the process; 0 = fixed 256
                         (default: timed while other contexts share the GPU, the
                         choices were measured to slow the concurrent solves)         */
  int tc_digits;      /* digits of the rank-structured tensor-core contractions inside
                         tctl_pcg_solve (tc_gemm = 1): 6 (default, 42 bits, 21
                         products), 4 (28 bits, 10 products) or 3 (21 bits, 6
                         products: the three-term BF16 split with FP32
                         accumulation); the other entry points use 6              */
  int refine;         /* FP64 outer residual refinement steps of tctl_pcg_solve
                         (default 0, at most 8): after the PCG, while the residual
                         B - F2(A) X formed with FP64 FMA contractions (truncated at
                         eps_final) exceeds pcg_rtol ||B||, X += PCG(that residual),
                         the inner solves at tc_digits                             */
} tctl_opts;

typedef struct {
  int iters;             /* PCG iterations performed                                 */
  double rel_res;        /* final recursive ||R||/||B||                               */
  int rank_x[3];         /* Tucker ranks of the solution before the final T2C         */
  int max_rank;          /* largest Tucker rank met inside the iteration              */
  int op_rank;           /* canonical rank R of the separable F2                      */
  int op_basis[3];       /* per-mode compressed operator basis size (FP64 contractions,
                            tc_gemm = 0; with tc_gemm = 1 the factors are used as they
                            are and this equals op_rank)                              */
  int pre_rank;          /* canonical rank of the preconditioner                      */
  double op_rel_err;     /* measured max rel. error of the separable F2 (sample)      */
  double s_min, s_max;   /* spectral interval of A                                    */
  double t_setup_ms;     /* time of tctl_setup                                       */
  double t_solve_ms;     /* time of the last tctl_pcg_solve                          */
  int expsum_used;       /* representation of F2 in use: 0 sinc, 1 fitted, 2 learned  */
  int pre_used;          /* preconditioner in use: 0 NNLS nodes, 1 fitted, 2 learned,
                            3 anisotropic Laplacian (case (A))                         */
  double pre_delta;      /* its measured max |P(s) F2(s) - 1| on [s_min, s_max]       */
  double ws_peak_mb;     /* peak use of the context's workspace arena so far (MiB)    */
  double ws_size_mb;     /* size of the arena (MiB)                                    */
  double op_learned_err; /* expsum_src 2: measured max rel. error of F2 of the learned
                            sum (accepted when <= op_judge); 0 otherwise               */
  double sinc24_err;     /* expsum_src 2: the same error of the sinc quadrature with 24
                            terms per function (the judge's reference); 0 otherwise    */
  int refines;           /* refinement steps taken by the last tctl_pcg_solve         */
  double true_rel_res;   /* refine > 0: the last FP64 residual ||B - F2(A) X|| / ||B||
                            formed (-1 when none was)                                   */
} tctl_stats;

/* Fills *o with the defaults listed above. */
int tctl_default_opts(tctl_opts *o);

/* Builds the solver for one coefficient set (Sections 3.2-3.5):
 * assembles A_(l) from coeffs (HOST, 3 x (n+1) doubles, row l holds
 * a_l(x_{i-1/2}) for i = 1..n+1), computes the 1D eigenpairs on the GPU in
 * FP64, the spectral interval, the exponential sum of F2 (fitted by default,
 * the sinc quadrature of Section 3.4 with expsum_src = 0 or as fallback) and
 * the preconditioner sum (Section 3.5, case (B) by default, case (A) with
 * pre_src = 3), and their factor matrices.
 * n >= 2, 0 < alpha <= 1, beta > 0, eps_trunc in (0, 1). opts may be NULL.
 * cuda_stream: a cudaStream_t (NULL = the calling host thread's default
 * stream: the library is built with per-thread default streams; pass
 * cudaStreamLegacy for the legacy default stream). Synchronizes once.
 * Errors: TCTL_E_ARG, TCTL_E_COEFF, TCTL_E_NOMEM, TCTL_E_CUDA, TCTL_E_NUMERIC. */
int tctl_setup(tctl_ctx **ctx, const double *coeffs, int n, double alpha,
               double beta, double eps_trunc, const tctl_opts *opts,
               void *cuda_stream);

/* y = trunc(F2(A) x, eps_trunc) with the separable F2 (eq. "Gen3DtimesX").
 * x, y: canonical, physical (grid) coordinates. y->cap must hold the result
 * (TCTL_E_RANK_CAP otherwise, y then holds the first y->cap terms). */
int tctl_apply_op(tctl_ctx *ctx, const tctl_cp *x, tctl_cp *y);

/* y = trunc(P(A) x, eps_trunc), P ~ F2^-1 the preconditioner chosen by
 * opts.pre_src (Section 3.5: case (B) in the operators' eigenbasis by
 * default, case (A) in the sine basis with pre_src = 3). */
int tctl_apply_precond(tctl_ctx *ctx, const tctl_cp *x, tctl_cp *y);

/* State recovery (state equation "State" of Section 3.1 with beta_p = 1):
 * y = trunc(A^-alpha u, eps_trunc) with the fitted exponential sum of
 * s^-alpha (one Kronecker term per node; measured relative error <= op_tol,
 * built on the first call). u, y: canonical, physical coordinates; y->cap as
 * in tctl_apply_op. Errors: as tctl_apply_op, TCTL_E_NUMERIC if no sum meets
 * op_tol. */
int tctl_apply_state(tctl_ctx *ctx, const tctl_cp *u, tctl_cp *y);

/* The paper's general constants (Section 3.1): beta_p A^-alpha u +
 * (gamma / beta_p) A^alpha u = y_Omega equals beta_p (A^-alpha + beta A^alpha) u
 * = y_Omega with beta = gamma / beta_p^2, so u_paper = u_scale * u with
 * u_scale = 1 / beta_p, u the solution for tctl_setup's beta. Host only. */
int tctl_map_constants(double beta_p, double gamma, double *beta, double *u_scale);

/* y = trunc(x, eps) (Appendix 1: canonical-to-Tucker by reduced HOSVD, core
 * truncation, Tucker-to-canonical). ||x - y|| <= eps ||x||. y may equal x.
 * eps must lie in [TCTL_TRUNC_EPS_MIN, 1): the range of each mode is found
 * from FP64 Gram matrices, which resolve directions down to about 1e-8 of the
 * largest weighted column, so a smaller eps could not be guaranteed and is
 * rejected with TCTL_E_ARG. */
#define TCTL_TRUNC_EPS_MIN 1e-7
int tctl_truncate(tctl_ctx *ctx, const tctl_cp *x, tctl_cp *y, double eps);

/* Solves (1) for b = y_Omega by Algorithm 1 (Appendix 2). x: output
 * (canonical, physical coordinates; any input content is ignored, X0 = 0).
 * st may be NULL. Errors: TCTL_E_NOT_CONVERGED (x holds the last iterate),
 * TCTL_E_RANK_CAP, TCTL_E_NAN, TCTL_E_CUDA. */
int tctl_pcg_solve(tctl_ctx *ctx, const tctl_cp *b, tctl_cp *x, tctl_stats *st);

/* Exact full-grid solve u = (xV)[((xV^T) y) ./ F2(lambda_i+lambda_j+lambda_k)]
 * (Sections 3.3-3.4, "DiagFGen2D"), six dense mode products and the
 * pointwise spectral divide. y, u: DEVICE n^3 arrays (x1 fastest), must not
 * alias. opts.precision selects FP64 FMA GEMMs (one n^3 double temporary) or
 * the tensor-core digit-split GEMMs (two n^3 float temporaries, digit planes
 * of the six eigenvector matrices); workspace is allocated on first use. */
int tctl_fullgrid_solve(tctl_ctx *ctx, const double *y, double *u);

/* State equation ("State"): y = A^-alpha u on the full grid (DEVICE n^3). */
int tctl_fullgrid_state(tctl_ctx *ctx, const double *u, double *y);

/* One-shot solve from HOST buffers: setup, host-to-device copies, PCG,
 * device-to-host copy of the canonical solution, teardown. coeffs as in
 * tctl_setup; yw (S) and yU (3 x n x S, mode-major, column-major per mode)
 * the canonical y_Omega; uw (cap) and uU (3 x n x cap) receive the solution,
 * *u_rank its rank. Runs on a non-blocking stream of its own, so calls from
 * several host threads overlap on the GPU. Returns the same codes as
 * tctl_pcg_solve. */
int tctl_solve_host(const double *coeffs, int n, double alpha, double beta,
                    double eps_trunc, const tctl_opts *opts, const double *yw,
                    const double *yU, int S, double *uw, double *uU, int cap,
                    int *u_rank, tctl_stats *st);

/* One problem of tctl_solve_batch: inputs as tctl_solve_host (HOST buffers;
 * yU: 3 x n x S mode-major, uU: 3 x n x cap); outputs u_rank, status (a
 * TCTL_* code), latency_ms (wall time of this problem: set-up, copies, PCG,
 * copy back, teardown) and *st when st is not NULL. */
typedef struct {
  const double *coeffs;
  int n;
  double alpha, beta;
  const double *yw, *yU;
  int S;
  double *uw, *uU;
  int cap;
  tctl_stats *st;
  int u_rank;
  int status;
  double latency_ms;
} tctl_batch_item;

/* Batched solves: `count` independent problems of any n, rank,
 * alpha and beta, scheduled dynamically over `workers` host threads, each
 * issuing to its own stream so that the problems overlap on the GPU. Returns
 * TCTL_OK, or the first non-OK item status (every item is attempted). */
int tctl_solve_batch(tctl_batch_item *items, int count, double eps_trunc, const tctl_opts *opts,
                     int workers);

/* Allocates a canonical tensor with cap terms (device memory, zero rank). */
int tctl_cp_alloc(tctl_ctx *ctx, int cap, tctl_cp *out);
void tctl_cp_free(tctl_ctx *ctx, tctl_cp *cp);

/* Copies the 1D eigenpairs of mode l to HOST buffers lam (n) and V (n x n,
 * column-major, eigenvectors as columns; the sign of column v is fixed by
 * sum_i v_i g_i > 0, g_i = 2 frac(i * 0.6180339887498949) - 1, i = 1..n). */
int tctl_get_eigs(tctl_ctx *ctx, int mode, double *lam, double *V);

/* Copies the statistics of the context (setup data and last solve) to *st. */
int tctl_get_stats(tctl_ctx *ctx, tctl_stats *st);

/* C = alpha op(A) op(B) + beta C for DEVICE FP64 column-major matrices
 * (op(A) m x k, op(B) k x n, op = transpose when trans_* != 0), ordered on
 * the context's stream. digits = 0: FP64 FMA kernels; digits = 3, 4 or 6: the
 * tensor-core digit split of the rank-structured path (each operand as 3 / 4 / 6
 * signed 7-bit BF16 digits with one binary exponent per row of op(A) and per
 * column of op(B); FP32 accumulation with exact leading levels, 256-deep K
 * chunks summed in FP64). Error per entry ~2^-7d K max|A_i.| max|B_.j|.
 * Synchronizes (checks the kernels' bounded waits) when digits > 0.
 * Errors: TCTL_E_ARG, TCTL_E_CUDA, TCTL_E_NUMERIC (a wait timed out). */
int tctl_gemm(tctl_ctx *ctx, int digits, int trans_a, int trans_b, int m, int n, int k,
              double alpha, const double *A, int lda, const double *B, int ldb, double beta,
              double *C, int ldc);

/* C (ra rb x n) = alpha KR(X, Y)^T B + beta C for DEVICE FP64 column-major
 * matrices: X (k x ra, ld ldx), Y (k x rb, ld ldy), B (k x n, ld ldb), C (ld
 * ldc), where column a + ra b of the Khatri-Rao product KR(X, Y) is the
 * entrywise product X(:, a) .* Y(:, b) -- the contraction of the sketches and
 * core projections of Section 3.4's Hadamard products (probe factors and
 * factor-basis products), contracted over the grid index. digits = 0: the
 * product is formed in the context's workspace and multiplied by the FP64
 * kernels; digits = 3, 4 or 6: the tensor-core digit split of tctl_gemm forms
 * each product X(i, a) Y(i, b) while splitting (nothing k x ra rb is stored),
 * with the same result as tctl_gemm on the stored product. Ordered on the
 * context's stream; synchronizes when digits > 0. Errors: TCTL_E_ARG,
 * TCTL_E_NOMEM (workspace, digits = 0), TCTL_E_CUDA, TCTL_E_NUMERIC. */
int tctl_gemm_kr(tctl_ctx *ctx, int digits, int k, int ra, int rb, int n, double alpha,
                 const double *X, int ldx, const double *Y, int ldy, const double *B, int ldb,
                 double beta, double *C, int ldc);

/* The fitted exponential sum behind expsum_src = 1 (host only, no device
 * work, no context): g(s) ~ sum_k w_k exp(-t_k s) on [s_min, s_max], t_k >= 0
 * (t_0 = 0 is a constant term), w_k > 0, where g = F2(s)/s = s^(-1-alpha) +
 * beta s^(alpha-1) for alpha < 1 (F2 ~ s g) and g = 1/s for alpha = 1
 * (F2 ~ g + beta s, exact positive power). The node count is the smallest
 * (to within a few) for which the max relative error of F2, measured on 2000
 * log-spaced points of [s_min, s_max], is <= tol; *err receives it and *r
 * the number of terms. t, w: HOST buffers of cap entries. Errors: TCTL_E_ARG,
 * TCTL_E_RANK_CAP (r > cap, first cap copied), TCTL_E_NUMERIC (tol not met;
 * the buffers hold the best fit found). */
int tctl_expsum_fit(double alpha, double beta, double s_min, double s_max, double tol, double *t,
                    double *w, int cap, int *r, double *err);

/* Learned preconditioner sums (host buffers, no context).
 * tctl_precond_fit: r free nodes theta (ascending) and weights p > 0 of
 * P(s) = s sum_k p_k exp(-theta_k s) ~ 1/F2(s) on [s_min, s_max]
 * (Levenberg-Marquardt on log parameters, Lawson reweighting; started from
 * geometric nodes + NNLS); *delta = measured max |P F2 - 1| (2000 points).
 * tctl_precond_dataset: n_samples seeded inputs X (n x 4: alpha, log10 beta,
 * ln s_min, ln s_max; alpha in [0.1, 0.9], log10 beta in [-4, 0], s_min in
 * [15, 45], log10 s_max in [4.5, 8.5]) and fitted targets Y (n x 2r: ln tau_k
 * ascending, ln q_k with tau = theta s_min, q = p (s_min F2(s_min))) on
 * `threads` host threads; delta (n) may be NULL.
 * tctl_mlp_train: MLP 4 -> 64 -> 64 -> 2r (FP32, tanh) trained on the GPU by
 * the library's kernels (MSE on standardised targets, Adam, cosine decay, one
 * step captured in a CUDA graph); model: tctl_mlp_model_size(r) floats
 * (parameters + input / output standardisation); loss[0], loss[1] = dataset
 * MSE before / after training (may be NULL).
 * tctl_mlp_grad: loss and parameter gradient of one batch (standardised X
 * (batch x 4) and T (batch x 2r); params: the first mlp parameters of a model).
 * tctl_mlp_forward: raw (ln tau, ln q) for n raw inputs (GPU inference kernel).
 * Errors: TCTL_E_ARG, TCTL_E_CUDA. r in [2, 32]. */
int tctl_precond_fit(double alpha, double beta, double s_min, double s_max, int r, double *theta,
                     double *p, double *delta);
int tctl_precond_dataset(int r, int n_samples, unsigned long long seed, int threads, float *X,
                         float *Y, double *delta);
/* The same for either head: which = 0 fits r-term sums of the operator's
 * g(s) = F2(s)/s (F2 = s sum_k w_k exp(-t_k s), Section 3.4's exponential-sum
 * form with free nodes), which = 1 the preconditioner sums of
 * tctl_precond_dataset. Targets Y (n x 2r): ln tau_k ascending, ln q_k in
 * x = s / s_min units with the sum normalised by its target at s_min;
 * err (n, may be NULL): measured max relative error of F2 (which = 0) or
 * delta (which = 1). Inputs as tctl_precond_dataset (alpha < 1 throughout). */
int tctl_expsum_dataset(int which, int r, int n_samples, unsigned long long seed, int threads,
                        float *X, float *Y, double *err);
int tctl_mlp_model_size(int r);
int tctl_mlp_train(int r, int n_samples, const float *X, const float *Y, int steps, int batch,
                   float lr, unsigned long long seed, float *model, float *loss);
int tctl_mlp_grad(int r, int batch, const float *params, const float *X, const float *T,
                  float *grad, float *loss);
int tctl_mlp_forward(int r, int n, const float *model, const float *X, float *Y);

/* Copies the separable representation in use (Sections 3.4, 3.5): which = 0
 * the operator F2 (R terms), 1 the preconditioner. Term k is the Kronecker
 * product over the modes l of diag(f_lk(lambda^(l))) with f_lk(x) =
 * (m[k] == l ? x : 1) exp(-t[k] x), weighted by w[k]; on the eigenbasis grid
 * the sum is the approximation of F2(lambda_i + lambda_j + lambda_k) (resp.
 * of its inverse). t, w, m: HOST buffers of cap entries; *R receives the
 * number of terms. TCTL_E_RANK_CAP if R > cap (the first cap are copied). */
int tctl_get_expsum(tctl_ctx *ctx, int which, double *t, double *w, int *m, int cap, int *R);

/* Number of GPU kernel launches issued by the context since setup (counter
 * kept by the library's own launch wrappers). */
long long tctl_launch_count(const tctl_ctx *ctx);

/* Allocation-free 1D eigendecompositions, for callers that cannot allocate
 * device memory: code running where cudaMalloc is not allowed or not wanted,
 * e.g. inside another library's memory pool, a stream-ordered pipeline whose
 * owner controls every allocation, or an embedded runtime with a fixed memory
 * budget. The paper has no counterpart of this entry point. It returns the
 * same eigenpairs as tctl_setup / tctl_get_eigs for the same coefficients,
 * without creating a context.
 *   coeffs: DEVICE, 3 x (n+1) doubles (row l = a_l(x_{i-1/2}), i = 1..n+1).
 *   lam:    DEVICE, 3 x n doubles, ascending per mode (output).
 *   V:      DEVICE, 3 x n x n doubles; mode l at V + l*n*n, column-major,
 *           eigenvectors as columns, signs as in tctl_get_eigs (output).
 *   cuda_stream: cudaStream_t (NULL = the calling thread's default stream);
 *           the call synchronizes
 *           the stream once (coefficient check) and leaves the eigensolver
 *           kernels queued on it.
 * Scratch comes from a file-scope device array sized for n <=
 * TCTL_EIG_NOALLOC_MAX_N (about 3.2 MB, held by every device that loads the
 * library until the process exits); no cudaMalloc, cudaFree or allocating
 * library routine is called. The first call on a device looks up the array's
 * device address (one-time set-up). Every call synchronizes its stream (the
 * coefficient check reads a status word back to the host), so no call may be
 * made while the stream is being captured into a CUDA graph: the capture would
 * be invalidated and the call returns TCTL_E_CUDA. All calls on a device share
 * the array: calls whose GPU work
 * overlaps (different streams, or host threads without ordering) race and
 * corrupt each other's results; serialize them.
 * Errors: TCTL_E_ARG (NULL pointer, n < 2 or n > TCTL_EIG_NOALLOC_MAX_N),
 * TCTL_E_COEFF (a coefficient <= 0 or not finite), TCTL_E_CUDA.
 * tctl_last_error(NULL) describes the failure. */
#define TCTL_EIG_NOALLOC_MAX_N 256
int tctl_eig1d_noalloc(const double *coeffs, int n, int paper_end_rows, double *lam,
                       double *V, void *cuda_stream);

/* Failure-detection test hook (no counterpart in the paper): the next `count`
 * tensor-core GEMM launches of this context withhold their operand copies, so
 * the kernel's bounded wait for the first stage (a barrier nothing arrives on)
 * runs out after about 1 ms instead of the normal 1 s limit. Such a launch
 * leaves its output unwritten, frees its tensor memory and returns; the call
 * that issued it returns TCTL_E_NUMERIC ("bounded mbarrier wait timed out"),
 * and the context stays usable for the next call. Nothing faults, traps or
 * hangs. count = 0 cancels. Errors: TCTL_E_ARG (NULL context, count < 0). */
int tctl_inject_wait_timeout(tctl_ctx *ctx, int count);

/* The tile autotuner's table (process-wide, host only): a JSON list with one
 * object per shape class met so far (digits, k steps of 16, log2 of the tile
 * count, the chosen k per CTA and the timed candidates in ms). Errors:
 * TCTL_E_ARG (NULL buffer or too small). */
int tctl_tune_report(char *buf, int buflen);

/* Per-kernel timing (tracing): when enabled, the context records a pair of
 * CUDA events on its stream around every kernel it launches. The report is a
 * JSON object {kernel: {"launches", "ms", "flops"}} aggregated over the
 * launches since the last report (flops: algorithmic 2mnk for GEMMs, 0 for
 * other kernels); it synchronizes the stream and clears the records.
 * on = 2 additionally prefixes every name with the algorithm phase
 * ("apply_op/...", "truncate/...", ...).
 * Errors: TCTL_E_ARG (NULL, or buffer too small). */
int tctl_profile_enable(tctl_ctx *ctx, int on);
int tctl_profile_report(tctl_ctx *ctx, char *buf, int buflen);

void tctl_destroy(tctl_ctx *ctx);
const char *tctl_last_error(const tctl_ctx *ctx);

#ifdef __cplusplus
}
#endif
#endif /* TENSORCTL_H */
