// Separable spectral functions (Section 3.4, 3.5) and the full-grid solve.
//
// F2(s) = s^-alpha + beta s^alpha is written, as in Section 3.4, through the
// Laplace transform s^-g = 1/Gamma(g) int_R exp(g tau - e^tau s) dtau and a
// trapezoid (sinc) rule in tau, for g = alpha (the term s^-alpha) and for
// g = 1 - alpha (the term s^(alpha-1), multiplied pointwise by the rank-3
// tensor s = lambda_i + lambda_j + lambda_k: D^alpha = D .* D^(alpha-1)).
// Quadrature parameters (the paper gives none): step h = 2 pi d / ln(1/delta)
// with d = 1.2; the left end where the omitted tail exp(g tau_a)/(g Gamma(g))
// times max(m/F) is delta/4; the right end where the tail
// t^(g-1) e^(-t s)/(s Gamma(g)) times m/F is delta/4 at s = s_min.
//
// The preconditioner (Section 3.5, case (B), a direct low Kronecker-rank
// approximation of 1/F2 in the same eigenbasis) is P(s) = s sum_k p_k
// exp(-theta_k s) with p_k >= 0 from a non-negative least-squares fit of
// P(s) F2(s) = 1 on 256 geometric sample points of [s_min, s_max]; the K
// nodes theta_k are geometric in [0.05/s_max, 20/s_min].
//
// Fitted exponential sum (expsum_src = 1, the default; the paper gives only
// the sinc construction, with rank bounds). For alpha < 1, g(s) = F2(s)/s =
// s^(-1-alpha) + beta s^(alpha-1) is completely monotone (a sum of negative
// powers), so it has exponential sums with positive weights:
// g(s) ~ w_0 + sum_k w_k exp(-t_k s), t_k geometric in [lo/s_max, hi/s_min],
// w_0 a constant term. Then F2(s) = s g(s) needs 3 Kronecker terms per
// exponential (s = lambda_i + lambda_j + lambda_k): one function instead of
// the sinc form's two. For alpha = 1, beta s is exact (3 terms) and g = 1/s. The weights minimise the relative
// error of g on 400 log-spaced samples under w >= 0 (Lawson-Hanson NNLS,
// which adds one node at a time and so stays stable although the full
// exponential basis is nearly collinear). The number of nodes grows until the
// measured max relative error of F2 on [s_min, s_max] is <= op_tol; if no fit
// reaches it the sinc sum is used.
//
// Every exponential factorises over the modes, so each term is a Kronecker
// product of three diagonal matrices in the eigenbasis; the factor matrices
// E_l[i, k] = (lambda_i^(l) or 1) * exp(-t_k lambda_i^(l)) are built on the GPU.
#include <algorithm>
#include <chrono>
#include <cstdio>
#include <cmath>
#include <numeric>

#include "tctl_internal.cuh"

namespace tctl {

namespace {

constexpr double kSincD = 1.2;
constexpr int kPreSamples = 256;

double F2h(double s, double a, double b) { return std::pow(s, -a) + b * std::pow(s, a); }

double min_F2(double a, double b, double smin, double smax) {
  const double star = (a >= 1.0) ? 1.0 / std::sqrt(b) : std::pow(b, -1.0 / (2.0 * a));
  if (smin <= star && star <= smax) return 2.0 * std::sqrt(b);
  return std::min(F2h(smin, a, b), F2h(smax, a, b));
}

double right_end(double g, double q) {
  double x = std::max(1.0, -std::log(q));
  for (int i = 0; i < 60; ++i) x = std::max(1e-300, -std::log(q) + (g - 1.0) * std::log(x));
  return x;
}

struct SincRule {
  double tau_lo, h;
  int r;
};

SincRule sinc_rule(double g, double delta, double smin, double left_gain, double right_q) {
  SincRule s;
  s.h = 2.0 * M_PI * kSincD / std::log(1.0 / delta);
  const double tau_a = std::log(0.25 * delta * g * std::tgamma(g) / left_gain) / g;
  const double x = right_end(g, right_q);
  const double tau_b = std::log(x / smin);
  const double tau_lo = tau_a + 0.5 * s.h;
  const double tau_hi = tau_b - 0.5 * s.h;
  s.r = (int)std::ceil((tau_hi - tau_lo) / s.h) + 1;
  s.tau_lo = tau_hi - (s.r - 1) * s.h;
  return s;
}

void sinc_nodes(double g, const SincRule &s, std::vector<double> &t, std::vector<double> &w) {
  t.resize(s.r);
  w.resize(s.r);
  const double ig = 1.0 / std::tgamma(g);
  for (int k = 0; k < s.r; ++k) {
    const double tau = s.tau_lo + s.h * k;
    t[k] = std::exp(tau);
    w[k] = s.h * std::exp(g * tau) * ig;
  }
}

// Lawson-Hanson non-negative least squares min ||A x - b||, x >= 0.
// A: M x K column-major. The least-squares problem on the passive set is
// solved from a Householder QR that grows by one column at a time: a column
// entering the passive set is multiplied by the reflectors of the columns
// before it and contributes one new reflector (O(M P) work, P passive
// columns), and Q^T b is updated the same way. When coordinates leave the
// passive set the factorization is rebuilt from the remaining columns, in
// their order of entry: the reflectors of the columns ahead of the first one
// that left depend on those columns only, so they are kept (truncate) and
// only the columns after it are added again (the same operations as a
// rebuild from scratch, the same result).
class IncQR {
 public:
  IncQR(const std::vector<double> &A, int M, const std::vector<double> &b)
      : A_(A), M_(M), b_(b) { reset(); }

  void reset() {
    cols_.clear();
    R_.clear();
    V_.clear();
    vn_.clear();
    qb_ = b_;
  }

  // keeps the first P columns of the factorization (Q^T b re-formed from b
  // by their reflectors, in the order of a rebuild)
  void truncate(int P) {
    if (P >= (int)cols_.size()) return;
    cols_.resize(P);
    R_.resize(P);
    V_.resize(P);
    vn_.resize(P);
    qb_ = b_;
    for (int p = 0; p < P; ++p) reflect(p, qb_);
  }

  // appends column j of A to the factorization
  void add(int j) {
    std::vector<double> c(A_.begin() + (size_t)j * M_, A_.begin() + (size_t)(j + 1) * M_);
    for (int p = 0; p < (int)cols_.size(); ++p) reflect(p, c);
    append(j, c);
  }

  // appends columns js of A in order, as add(js[0]), add(js[1]), ... would:
  // the reflectors already present are applied to all of them together (each
  // column's operations in the same order, several independent sums at a
  // time), then each column in turn takes the reflectors of those before it
  void add_many(const std::vector<int> &js) {
    const int P0 = (int)cols_.size(), nq = (int)js.size();
    std::vector<std::vector<double>> C(nq);
    for (int q = 0; q < nq; ++q)
      C[q].assign(A_.begin() + (size_t)js[q] * M_, A_.begin() + (size_t)(js[q] + 1) * M_);
    for (int q0 = 0; q0 < nq; q0 += 4) {
      const int qn = std::min(4, nq - q0);
      for (int p = 0; p < P0; ++p) reflect4(p, C, q0, qn);
    }
    for (int q = 0; q < nq; ++q) {
      for (int p = P0; p < (int)cols_.size(); ++p) reflect(p, C[q]);
      append(js[q], C[q]);
    }
  }

 private:
  // the new reflector of column j (already reflected by those before it)
  void append(int j, const std::vector<double> &c) {
    const int P = (int)cols_.size();
    double nrm = 0;
    for (int i = P; i < M_; ++i) nrm += c[i] * c[i];
    nrm = std::sqrt(nrm);
    std::vector<double> v(M_, 0.0);
    double vn = 0.0, alpha = 0.0;
    if (nrm > 0) {
      alpha = c[P] > 0 ? -nrm : nrm;
      for (int i = P; i < M_; ++i) v[i] = c[i];
      v[P] -= alpha;
      for (int i = P; i < M_; ++i) vn += v[i] * v[i];
    }
    V_.push_back(v);
    vn_.push_back(vn);
    cols_.push_back(j);
    // R column: c[0..P) above the diagonal, alpha on it
    std::vector<double> rc(c.begin(), c.begin() + P);
    rc.push_back(vn == 0 ? c[P] : alpha);
    R_.push_back(rc);
    reflect(P, qb_);
  }

 public:
  // least-squares coefficients of the passive columns (in order of entry)
  std::vector<double> solve() const {
    const int P = (int)cols_.size();
    std::vector<double> x(P, 0.0);
    for (int j = P - 1; j >= 0; --j) {
      double s = qb_[j];
      for (int k = j + 1; k < P; ++k) s -= R_[k][j] * x[k];
      const double d = R_[j][j];
      x[j] = d != 0 ? s / d : 0.0;
    }
    return x;
  }

  const std::vector<int> &cols() const { return cols_; }

 private:
  void reflect(int p, std::vector<double> &y) const {
    if (vn_[p] == 0) return;
    const std::vector<double> &v = V_[p];
    double s = 0;
    for (int i = p; i < M_; ++i) s += v[i] * y[i];
    s = 2 * s / vn_[p];
    for (int i = p; i < M_; ++i) y[i] -= s * v[i];
  }

  // reflect(p, .) on columns C[q0 .. q0 + qn), qn <= 4, their sums interleaved
  void reflect4(int p, std::vector<std::vector<double>> &C, int q0, int qn) const {
    if (vn_[p] == 0) return;
    const std::vector<double> &v = V_[p];
    double *y[4];
    for (int q = 0; q < 4; ++q) y[q] = C[q0 + std::min(q, qn - 1)].data();
    double s[4] = {0, 0, 0, 0};
    for (int i = p; i < M_; ++i) {
      s[0] += v[i] * y[0][i];
      s[1] += v[i] * y[1][i];
      s[2] += v[i] * y[2][i];
      s[3] += v[i] * y[3][i];
    }
    for (int q = 0; q < qn; ++q) {
      const double sq = 2 * s[q] / vn_[p];
      double *yq = y[q];
      for (int i = p; i < M_; ++i) yq[i] -= sq * v[i];
    }
  }

  const std::vector<double> &A_;
  int M_;
  const std::vector<double> &b_;
  std::vector<int> cols_;
  std::vector<std::vector<double>> R_, V_;
  std::vector<double> vn_, qb_;
};

std::vector<double> nnls(const std::vector<double> &A, int M, int K, const std::vector<double> &b) {
  std::vector<double> x(K, 0.0);
  std::vector<char> passive(K, 0), blocked(K, 0);
  const double tol = 1e-15;  // the duals of this ill-conditioned basis are tiny
  IncQR qr(A, M, b);
  for (int outer = 0; outer < 3 * K; ++outer) {
    // dual w = A^T (b - A x); the most positive free, unblocked coordinate enters
    std::vector<double> res(b);
    for (int k = 0; k < K; ++k)
      if (x[k] != 0)
        for (int i = 0; i < M; ++i) res[i] -= A[i + (size_t)k * M] * x[k];
    // (four duals at a time, each summed in the order of i)
    int jmax = -1;
    double wmax = tol;
    for (int k0 = 0; k0 < K; k0 += 4) {
      const double *col[4];
      bool use[4], any = false;
      for (int q = 0; q < 4; ++q) {
        const int k = k0 + q;
        use[q] = k < K && !passive[k] && !blocked[k];
        any = any || use[q];
        col[q] = A.data() + (size_t)(use[q] ? k : k0) * M;
      }
      if (!any) continue;
      double w[4] = {0, 0, 0, 0};
      for (int i = 0; i < M; ++i) {
        w[0] += col[0][i] * res[i];
        w[1] += col[1][i] * res[i];
        w[2] += col[2][i] * res[i];
        w[3] += col[3][i] * res[i];
      }
      for (int q = 0; q < 4; ++q)
        if (use[q] && w[q] > wmax) { wmax = w[q]; jmax = k0 + q; }
    }
    if (jmax < 0) break;
    passive[jmax] = 1;
    qr.add(jmax);
    for (int inner = 0; inner < 3 * K; ++inner) {
      const std::vector<int> cols = qr.cols();
      const std::vector<double> z = qr.solve();
      bool allpos = true;
      for (double v : z) allpos = allpos && (v > 0);
      if (allpos) {
        std::fill(x.begin(), x.end(), 0.0);
        for (size_t j = 0; j < cols.size(); ++j) x[cols[j]] = z[j];
        std::fill(blocked.begin(), blocked.end(), 0);
        break;
      }
      // step from x toward z until the first passive coordinate reaches zero
      double amin = 1e300;
      int imin = -1;
      for (size_t j = 0; j < cols.size(); ++j)
        if (z[j] <= 0) {
          const double al = x[cols[j]] / (x[cols[j]] - z[j]);
          if (al < amin) { amin = al; imin = cols[j]; }
        }
      for (size_t j = 0; j < cols.size(); ++j) x[cols[j]] += amin * (z[j] - x[cols[j]]);
      x[imin] = 0.0;
      for (size_t j = 0; j < cols.size(); ++j)
        if (x[cols[j]] <= 0.0) { passive[cols[j]] = 0; x[cols[j]] = 0.0; }
      // rebuild the factorization from the columns still passive (order of
      // entry), keeping the part ahead of the first column that left
      size_t keep = 0;
      while (keep < cols.size() && passive[cols[keep]]) ++keep;
      qr.truncate((int)keep);
      std::vector<int> again;
      for (size_t q = keep; q < cols.size(); ++q)
        if (passive[cols[q]]) again.push_back(cols[q]);
      qr.add_many(again);
      // the entering coordinate left at once: it cannot improve the fit now
      if (imin == jmax && amin == 0.0) { blocked[jmax] = 1; break; }
    }
  }
  return x;
}

// The fitted function: g = F2/s for alpha < 1 (F2 ~ s g); for alpha = 1 the
// positive power is exactly beta s and g = 1/s (F2 ~ g + beta s).
// beta = kStateFn selects the state operator's symbol s^-alpha itself (no
// positive power, approximated without the factor s).
constexpr double kStateFn = -1.0;
double g_of_s(double s, double a, double b) {
  if (b == kStateFn) return std::pow(s, -a);
  return a >= 1.0 ? 1.0 / s : std::pow(s, -1.0 - a) + b * std::pow(s, a - 1.0);
}

struct ExpFit {
  std::vector<double> t, w;  // g(s) ~ sum_k w_k exp(-t_k s) (t_0 = 0: the constant)
  double err = 1e300;        // measured max relative error of F2 = s g
};

double measure_F2_fit(const ExpFit &f, double a, double b, double smin, double smax) {
  double emax = 0;
  const int M = 2000;
  for (int j = 0; j < M; ++j) {
    const double s = std::exp(std::log(smin) + (std::log(smax) - std::log(smin)) * j / (M - 1));
    double v = 0;
    for (size_t k = 0; k < f.t.size(); ++k) v += f.w[k] * std::exp(-f.t[k] * s);
    const double ex = b == kStateFn ? std::pow(s, -a) : F2h(s, a, b);
    const double ap = b == kStateFn ? v : (a >= 1.0 ? v + b * s : s * v);
    emax = std::max(emax, std::fabs(ap - ex) / ex);
  }
  return emax;
}

ExpFit fit_g(double a, double b, double smin, double smax, int r, double lo, double hi) {
  constexpr int M = 400;
  const double rho = smax / smin, g0 = g_of_s(smin, a, b);
  std::vector<double> x(M), G(M), tau(r);
  for (int j = 0; j < M; ++j) {
    x[j] = std::exp(std::log(rho) * j / (M - 1));
    G[j] = g_of_s(smin * x[j], a, b) / g0;
  }
  tau[0] = 0.0;
  for (int k = 1; k < r; ++k)
    tau[k] = std::exp(std::log(lo / rho) + (std::log(hi) - std::log(lo / rho)) * (k - 1) / std::max(1, r - 2));
  // relative residual sum_k c_k exp(-tau_k x_j) / G_j - 1, columns scaled to unit norm
  std::vector<double> A((size_t)M * r), cs(r), rhs(M, 1.0);
  for (int k = 0; k < r; ++k) {
    double nrm = 0;
    for (int j = 0; j < M; ++j) {
      const double v = std::exp(-tau[k] * x[j]) / G[j];
      A[j + (size_t)k * M] = v;
      nrm += v * v;
    }
    cs[k] = std::sqrt(nrm);
    for (int j = 0; j < M; ++j) A[j + (size_t)k * M] /= cs[k];
  }
  const std::vector<double> c = nnls(A, M, r, rhs);
  ExpFit out;
  for (int k = 0; k < r; ++k) {
    if (!(c[k] > 0)) continue;
    out.t.push_back(tau[k] / smin);
    out.w.push_back(c[k] / cs[k] * g0);
  }
  out.err = out.t.empty() ? 1e300 : measure_F2_fit(out, a, b, smin, smax);
  return out;
}

// Smallest fitted sum (to a few nodes) with measured error <= tol: nodes in
// [0.1/s_max, 20/s_min]; r starts at 2.5 ln(s_max / s_min) (16..40) and is then
// set from the observed rate of about a decade per 5 nodes, raised by 3 until
// the fit passes. (Starting low matters on short intervals: there, dense nodes
// make the basis so collinear that more nodes can fit worse.)
ExpFit fit_F2(double a, double b, double smin, double smax, double tol) {
  constexpr int rmax = 96;
  constexpr double lo = 0.1, hi = 20.0;
  const int r0 = std::max(16, std::min(40, (int)std::lround(2.5 * std::log(smax / smin))));
  ExpFit best = fit_g(a, b, smin, smax, r0, lo, hi);
  if (best.err <= tol) return best;
  int r = r0 + std::max(3, (int)std::ceil(5.0 * std::log10(best.err / tol)));
  for (int attempt = 0; attempt < 10 && r <= rmax; ++attempt, r += 3) {
    ExpFit f = fit_g(a, b, smin, smax, r, lo, hi);
    if (f.err <= tol) return f;
    if (f.err < best.err) best = f;
  }
  return best;
}

// Term descriptor of one canonical column: factor in mode l is
// (lambda if lam_mode == l else 1) * (t == 0 ? 1 : exp(-t lambda)).
struct TermDesc {
  double t;
  int lam_mode;  // -1: none
};

__global__ void factors_kernel(int n, int R, const double *__restrict__ lam,
                               const double *__restrict__ tk, const int *__restrict__ lm, int l,
                               double *E) {
  const long long total = (long long)n * R;
  for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < total;
       q += (long long)gridDim.x * blockDim.x) {
    const int i = (int)(q % n), k = (int)(q / n);
    const double x = lam[i];
    double v = (tk[k] == 0.0) ? 1.0 : exp(-tk[k] * x);
    if (lm[k] == l) v *= x;
    E[q] = v;
  }
}

void build_sep(Ctx &c, Sep &D, const std::vector<double> &w, const std::vector<TermDesc> &td,
               double *const *lam_override = nullptr) {
  const int n = c.n;
  D.R = (int)w.size();
  D.w_host = w;
  D.w = c.dmalloc(D.R);
  to_dev(c, D.w, w.data(), D.R);
  std::vector<double> t(D.R);
  std::vector<int> lm(D.R);
  for (int k = 0; k < D.R; ++k) {
    t[k] = td[k].t;
    lm[k] = td[k].lam_mode;
  }
  size_t mk = c.ws.mark();
  double *td_t = c.ws.dbl(D.R);
  int *td_m = c.ws.i32(D.R);
  to_dev(c, td_t, t.data(), D.R);
  write_dev(c, td_m, lm.data(), sizeof(int) * D.R);
  // Factor columns are stored with unit 2-norm and their norms moved into the
  // weights, w_k E_0k E_1k E_2k unchanged: every term then enters a contraction
  // at the scale of its contribution (the tensor-core GEMMs bound their error
  // by row / column maxima, so unbalanced factors would waste their digits).
  std::vector<double> wn(w);
  double *nrm = c.ws.dbl(D.R);
  std::vector<double> nh(D.R);
  for (int l = 0; l < 3; ++l) {
    D.E[l] = c.dmalloc((size_t)n * D.R);
    const int blocks = (int)std::min<long long>(((long long)n * D.R + 255) / 256, 4096);
    LAUNCH(c, factors_kernel, blocks, 256, 0, n, D.R, lam_override ? lam_override[l] : c.lam[l], td_t,
           td_m, l, D.E[l]);
    col_norms(c, n, D.R, D.E[l], n, nrm);
    to_host(c, nh.data(), nrm, D.R);
    for (int k = 0; k < D.R; ++k) {
      if (!(nh[k] > 0.0) || !std::isfinite(nh[k])) nh[k] = 1.0;  // an underflowed column stays
      wn[k] *= nh[k];
    }
    to_dev(c, nrm, nh.data(), D.R);
    scale_cols(c, n, D.R, D.E[l], n, nrm, true);
    D.B[l] = D.E[l];
    D.rD[l] = D.R;
    D.Z[l] = nullptr;  // identity: no compression
  }
  D.w_host = wn;
  to_dev(c, D.w, wn.data(), D.R);
  TCTL_CUDA(cudaStreamSynchronize(c.st));
  c.ws.reset(mk);
}

__global__ void term_scale_kernel(int R, const double *__restrict__ w, const double *__restrict__ n0,
                                  const double *__restrict__ n1, const double *__restrict__ n2,
                                  int l, double *__restrict__ s) {
  for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < R; k += gridDim.x * blockDim.x) {
    double v = fabs(w[k]);
    if (l != 0) v *= n0[k];
    if (l != 1) v *= n1[k];
    if (l != 2) v *= n2[k];
    s[k] = v;
  }
}

double frob2(Ctx &c, int n, int m, const double *A, double *tmp) {
  col_norms(c, n, m, A, n, tmp);
  std::vector<double> h(m);
  to_host(c, h.data(), tmp, m);
  double s = 0;
  for (double v : h) s += v * v;
  return s;
}

// Per-mode orthonormal basis B_l (n x rD_l) of the factor columns of D, weighted by the
// term weight and the other modes' column norms, found by randomized range finding with
// deflation (each round resolves ~1e-7 of what is left), until the weighted residual is
// below tol in relative Frobenius norm; then Z_l = B_l^T E_l. Falls back to the plain
// factors (Z = identity) if the basis would not be smaller than R/2.
void compress_sep(Ctx &c, Sep &D, double tol) {
  // the tensor-core contractions use the factor matrices themselves (their error
  // is relative to row / column maxima, which the recombination B_l Z_l would
  // spoil): the compressed basis serves only the FP64 path
  if (c.o.tc_gemm) return;
  const int n = c.n, R = D.R;
  const int capD = std::min(R / 2, 192);
  if (capD < 8) return;
  size_t mk = c.ws.mark();
  double *nrm[3];
  for (int l = 0; l < 3; ++l) {
    nrm[l] = c.ws.dbl(R);
    col_norms(c, n, R, D.E[l], n, nrm[l]);
  }
  double *sc = c.ws.dbl(R), *tmp = c.ws.dbl(R);
  double *W = c.ws.dbl((size_t)n * R);
  double *Om = c.ws.dbl((size_t)R * 64), *Y = c.ws.dbl((size_t)n * 64), *Qr = c.ws.dbl((size_t)n * 64);
  double *C = c.ws.dbl((size_t)64 * R), *C2 = c.ws.dbl((size_t)capD * 64);
  for (int l = 0; l < 3; ++l) {
    LAUNCH(c, term_scale_kernel, (R + 255) / 256, 256, 0, R, D.w, nrm[0], nrm[1], nrm[2], l, sc);
    copy_d(c, W, D.E[l], (size_t)n * R);
    scale_cols(c, n, R, W, n, sc, false);
    const double total2 = frob2(c, n, R, W, tmp);
    double *Bq = c.dmalloc((size_t)n * capD);
    int rD = 0;
    bool ok = false;
    for (int round = 0; round < 8 && rD < capD; ++round) {
      fill_gaussian(c, Om, (size_t)R * 64, 0xC0FFEEull * (l + 1) + round);
      gemm(c, false, false, n, 64, R, 1.0, W, n, 0, Om, R, 0, 0.0, Y, n, 0);
      for (int pass = 0; pass < 2 && rD > 0; ++pass) {
        gemm(c, true, false, rD, 64, n, 1.0, Bq, n, 0, Y, n, 0, 0.0, C2, rD, 0);
        gemm(c, false, false, n, 64, rD, -1.0, Bq, n, 0, C2, rD, 0, 1.0, Y, n, 0);
      }
      const int q = orth(c, n, 64, Y, n, 1e-7, true, std::min(64, capD - rD), Qr);
      if (q == 0) break;
      copy_d(c, Bq + (size_t)n * rD, Qr, (size_t)n * q);
      rD += q;
      // deflate: W -= Qr (Qr^T W)
      gemm(c, true, false, q, R, n, 1.0, Qr, n, 0, W, n, 0, 0.0, C, q, 0);
      gemm(c, false, false, n, R, q, -1.0, Qr, n, 0, C, q, 0, 1.0, W, n, 0);
      const double res2 = frob2(c, n, R, W, tmp);
      if (res2 <= tol * tol * total2) {
        ok = true;
        break;
      }
    }
    if (!ok) continue;  // keep the plain factors for this mode
    D.B[l] = Bq;
    D.rD[l] = rD;
    D.Z[l] = c.dmalloc((size_t)rD * R);
    gemm(c, true, false, rD, R, n, 1.0, Bq, n, 0, D.E[l], n, 0, 0.0, D.Z[l], rD, 0);
  }
  TCTL_CUDA(cudaStreamSynchronize(c.st));
  c.ws.reset(mk);
}

}  // namespace

// S[i + j n] = sqrt(2 / (n + 1)) sin((i + 1)(j + 1) pi / (n + 1)): the orthonormal
// eigenvectors of every constant-coefficient Dirichlet FD Laplacian (symmetric, S^2 = I)
__global__ void sine_basis_kernel(int n, double *S) {
  const long long total = (long long)n * n;
  const double c = sqrt(2.0 / (n + 1));
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < total;
       t += (long long)gridDim.x * blockDim.x) {
    const long long i = t % n, j = t / n;
    const long long m = ((i + 1) * (j + 1)) % (2 * (n + 1));  // exact argument reduction
    S[t] = c * sinpi((double)m / (double)(n + 1));
  }
}

__global__ void scaled_laplacian_eigs_kernel(int n, double b0, double *lam) {
  const double h = 1.0 / (n + 1);
  for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < n; k += gridDim.x * blockDim.x) {
    const double s = sinpi(0.5 * h * (k + 1));
    lam[k] = b0 * 4.0 * s * s / (h * h);
  }
}

std::vector<double> nnls_solve(const std::vector<double> &A, int M, int K, const std::vector<double> &b) {
  return nnls(A, M, K, b);
}

namespace {

// Sinc quadrature of s^-alpha (t1, w1) and, for alpha < 1, of s^(alpha-1) (t2, w2)
// for a target error delta of F2 = sum1 + beta s sum2 (the rule of the file header).
void sinc_sums(double a, double b, double smin, double smax, double delta, std::vector<double> &t1,
               std::vector<double> &w1, std::vector<double> &t2, std::vector<double> &w2) {
  const double F2min = min_F2(a, b, smin, smax), F2lo = F2h(smin, a, b), F2hi = F2h(smax, a, b);
  {
    const SincRule s = sinc_rule(a, 0.5 * delta, smin, 1.0 / F2min,
                                 0.25 * 0.5 * delta * std::tgamma(a) * F2lo * std::pow(smin, a));
    sinc_nodes(a, s, t1, w1);
  }
  t2.clear();
  w2.clear();
  if (a < 1.0) {
    const double g = 1.0 - a;
    const SincRule s = sinc_rule(g, 0.5 * delta, smin, b * smax / F2hi,
                                 0.25 * 0.5 * delta * std::tgamma(g) * F2lo * std::pow(smin, g) /
                                     (b * smin));
    sinc_nodes(g, s, t2, w2);
  }
}

// measured max relative error of the sinc form of F2 on 2000 log-spaced points
double sinc_rel_err(double a, double b, double smin, double smax, const std::vector<double> &t1,
                    const std::vector<double> &w1, const std::vector<double> &t2,
                    const std::vector<double> &w2) {
  double emax = 0;
  const int M = 2000;
  for (int j = 0; j < M; ++j) {
    const double s = std::exp(std::log(smin) + (std::log(smax) - std::log(smin)) * j / (M - 1));
    double v = 0;
    for (size_t k = 0; k < t1.size(); ++k) v += w1[k] * std::exp(-t1[k] * s);
    if (a >= 1.0) v += b * s;
    else {
      double v2 = 0;
      for (size_t k = 0; k < t2.size(); ++k) v2 += w2[k] * std::exp(-t2[k] * s);
      v += b * s * v2;
    }
    const double ex = F2h(s, a, b);
    emax = std::max(emax, std::fabs(v - ex) / ex);
  }
  return emax;
}

}  // namespace

// Error of the sinc form with at most r terms per function: the smallest
// target delta (on a 1.25x grid from 1e-14) whose rules fit in r terms.
double sinc_err_at_rank(double a, double b, double smin, double smax, int r) {
  std::vector<double> t1, w1, t2, w2;
  for (double delta = 1e-14; delta < 0.5; delta *= 1.25) {
    sinc_sums(a, b, smin, smax, delta, t1, w1, t2, w2);
    if ((int)t1.size() <= r && (int)t2.size() <= r) return sinc_rel_err(a, b, smin, smax, t1, w1, t2, w2);
  }
  return 1.0;
}

int expsum_fit_host(double a, double b, double smin, double smax, double tol, double *t, double *w,
                    int cap, int *r, double *err) {
  const ExpFit f = fit_F2(a, b, smin, smax, tol);
  const int n = (int)f.t.size();
  if (r) *r = n;
  if (err) *err = f.err;
  for (int k = 0; k < std::min(n, cap); ++k) {
    t[k] = f.t[k];
    w[k] = f.w[k];
  }
  if (n > cap) return TCTL_E_RANK_CAP;
  return f.err <= tol ? TCTL_OK : TCTL_E_NUMERIC;
}

// Host part of the spectral set-up (needs only s_min, s_max, alpha, beta and the
// host coefficients): the operator's exponential sum and the preconditioner's
// sum, kept as term lists in the context. It can run while the eigensolver
// is still computing the interior eigenpairs.
void setup_spectral_fit(Ctx &c) {
  const double a = c.alpha, b = c.beta, smin = c.s_min, smax = c.s_max;
  const auto t0 = std::chrono::steady_clock::now();
  const double delta = c.o.op_tol;
  // ---- operator F2 (term order as in the canonical factor layout)
  std::vector<double> w;
  std::vector<TermDesc> td;
  c.expsum_used = 0;
  if (c.o.expsum_src == 1) {
    const ExpFit f = fit_F2(a, b, smin, smax, delta);
    if (f.err <= delta) {
      if (a >= 1.0) {
        for (size_t k = 0; k < f.t.size(); ++k) {
          w.push_back(f.w[k]);
          td.push_back({f.t[k], -1});
        }
        for (int m = 0; m < 3; ++m) {
          w.push_back(b);
          td.push_back({0.0, m});
        }
      } else {
        for (size_t k = 0; k < f.t.size(); ++k)
          for (int m = 0; m < 3; ++m) {
            w.push_back(f.w[k]);
            td.push_back({f.t[k], m});
          }
      }
      c.op_rel_err = f.err;
      c.expsum_used = 1;
    }
  }
  if (c.o.expsum_src == 2) {
    // learned operator sum: the network's op_r nodes of g = F2/s (x = s / s_min
    // units), weights as predicted or re-solved by NNLS on those nodes (the
    // better of the two), judged on the measured relative error of F2; the
    // sinc quadrature with 24 terms per function is measured as the reference
    c.sinc24_err = sinc_err_at_rank(a, b, smin, smax, 24);
    if (a < 1.0) {
      const int r = c.o.op_r;
      const float xin[4] = {(float)a, (float)std::log10(b), (float)std::log(smin), (float)std::log(smax)};
      std::vector<float> y(2 * r);
      mlp_forward_host(r, 1, c.o.op_model, xin, y.data(), c.st);
      const double g0 = F2h(smin, a, b) / smin;
      std::vector<double> tt(r), wr(r);
      for (int k = 0; k < r; ++k) {
        tt[k] = std::exp((double)y[k]) / smin;
        wr[k] = std::exp((double)y[r + k]) * g0;
      }
      const double e_raw = sum_rel_err(FitTarget::Op, tt.data(), wr.data(), r, a, b, smin, smax);
      const std::vector<double> wn = weights_nnls(FitTarget::Op, tt, a, b, smin, smax);
      const double e_nn = sum_rel_err(FitTarget::Op, tt.data(), wn.data(), r, a, b, smin, smax);
      if (e_nn < e_raw) wr = wn;
      const double e = std::min(e_raw, e_nn);
      c.op_learned_err = e;
      if (std::isfinite(e) && e <= c.o.op_judge) {
        for (int k = 0; k < r; ++k) {
          if (!(wr[k] > 0)) continue;
          for (int m = 0; m < 3; ++m) {
            w.push_back(wr[k]);
            td.push_back({tt[k], m});
          }
        }
        c.op_rel_err = e;
        c.expsum_used = 2;
      }
    }
  }
  if (c.expsum_used == 0) {
    std::vector<double> t1, w1, t2, w2;
    sinc_sums(a, b, smin, smax, delta, t1, w1, t2, w2);
    const bool exact_linear = (a >= 1.0);
    for (size_t k = 0; k < t1.size(); ++k) {
      w.push_back(w1[k]);
      td.push_back({t1[k], -1});
    }
    if (exact_linear) {
      for (int m = 0; m < 3; ++m) {
        w.push_back(b);
        td.push_back({0.0, m});
      }
    } else {
      for (size_t k = 0; k < t2.size(); ++k)
        for (int m = 0; m < 3; ++m) {
          w.push_back(b * w2[k]);
          td.push_back({t2[k], m});
        }
    }
    c.op_rel_err = sinc_rel_err(a, b, smin, smax, t1, w1, t2, w2);
  }
  c.op_terms_w = w;
  c.op_terms_t.clear();
  c.op_terms_m.clear();
  for (const TermDesc &d : td) {
    c.op_terms_t.push_back(d.t);
    c.op_terms_m.push_back(d.lam_mode);
  }
  c.t_fit_ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();

  // ---- preconditioner P(s) = s sum_k p_k exp(-theta_k s), NNLS weights
  // pre_src 3 (case (A) of Section 3.5): the anisotropic constant-coefficient
  // Laplacian B0 = sum_l b0_l Delta_l, b0_l = (max a_l + min a_l) / 2, whose
  // eigenbasis is the sine basis: P ~ 1/F2 on its spectrum (b0_l mu_k), applied
  // there (the basis change is built with the factors, it needs V_l).
  double psmin = smin, psmax = smax;
  if (c.o.pre_src == 3) {
    const int n = c.n;
    double mu1 = 0, mun = 0;
    const double h = 1.0 / (n + 1);
    for (int l = 0; l < 3; ++l) {
      const double *al = c.coef_host.data() + (size_t)l * (n + 1);
      const double amax = *std::max_element(al, al + n + 1), amin = *std::min_element(al, al + n + 1);
      c.b0[l] = 0.5 * (amax + amin);
      mu1 += c.b0[l] * 4.0 * std::pow(std::sin(0.5 * M_PI * h), 2) / (h * h);
      mun += c.b0[l] * 4.0 * std::pow(std::sin(0.5 * M_PI * h * n), 2) / (h * h);
    }
    psmin = mu1;
    psmax = mun;
  }
  const int K = std::max(1, c.o.r_pre);
  std::vector<double> theta(K), smp(kPreSamples);
  for (int k = 0; k < K; ++k)
    theta[k] = std::exp(std::log(0.05 / psmax) +
                        (K == 1 ? 0.0 : (std::log(20.0 / psmin) - std::log(0.05 / psmax)) * k / (K - 1)));
  for (int j = 0; j < kPreSamples; ++j)
    smp[j] = std::exp(std::log(psmin) + (std::log(psmax) - std::log(psmin)) * j / (kPreSamples - 1));
  std::vector<double> A((size_t)kPreSamples * K), cs(K, 0.0), rhs(kPreSamples, 1.0);
  for (int k = 0; k < K; ++k) {
    double nrm = 0;
    for (int j = 0; j < kPreSamples; ++j) {
      const double v = std::exp(-smp[j] * theta[k]) * smp[j] * F2h(smp[j], a, b);
      A[j + (size_t)k * kPreSamples] = v;
      nrm += v * v;
    }
    cs[k] = std::sqrt(nrm);
    for (int j = 0; j < kPreSamples; ++j) A[j + (size_t)k * kPreSamples] /= cs[k];
  }
  std::vector<double> p = nnls(A, kPreSamples, K, rhs);
  for (int k = 0; k < K; ++k) p[k] /= cs[k];
  // alternatives with r free nodes: fitted at set-up (pre_src 1) or predicted by the
  // trained network (pre_src 2, weights re-solved on its nodes); each is measured and
  // replaces the K-node NNLS sum only if its delta = max |P F2 - 1| <= pre_delta_max
  c.pre_used = c.o.pre_src == 3 ? 3 : 0;
  c.pre_delta = pre_delta(theta.data(), p.data(), K, a, b, psmin, psmax);
  if (c.o.pre_src == 1 || c.o.pre_src == 2) {
    const int r = c.o.pre_r;
    std::vector<double> th(r), pr(r);
    double d = 1e300;
    if (c.o.pre_src == 1) {
      std::vector<double> tau(r), q(r);
      pre_fit(a, b, smin, smax, r, tau.data(), q.data());
      const double h0 = 1.0 / (smin * F2h(smin, a, b));
      for (int k = 0; k < r; ++k) {
        th[k] = tau[k] / smin;
        pr[k] = q[k] * h0;
      }
      d = pre_delta(th.data(), pr.data(), r, a, b, smin, smax);
    } else {
      const float xin[4] = {(float)a, (float)std::log10(b), (float)std::log(smin), (float)std::log(smax)};
      std::vector<float> y(2 * r);
      mlp_forward_host(r, 1, c.o.pre_model, xin, y.data(), c.st);
      const double h0 = 1.0 / (smin * F2h(smin, a, b));
      for (int k = 0; k < r; ++k) {
        th[k] = std::exp((double)y[k]) / smin;
        pr[k] = std::exp((double)y[r + k]) * h0;
      }
      const double d_raw = pre_delta(th.data(), pr.data(), r, a, b, smin, smax);
      std::vector<double> pn = pre_weights_nnls(th, a, b, smin, smax);
      const double d_nnls = pre_delta(th.data(), pn.data(), r, a, b, smin, smax);
      if (d_nnls < d_raw) pr = pn;
      d = std::min(d_raw, d_nnls);
    }
    if (std::isfinite(d) && d <= c.o.pre_delta_max) {
      theta = th;
      p = pr;
      c.pre_used = c.o.pre_src;
      c.pre_delta = d;
    }
  }
  std::vector<double> pw;
  std::vector<TermDesc> ptd;
  for (size_t k = 0; k < theta.size(); ++k) {
    if (p[k] <= 0) continue;
    for (int m = 0; m < 3; ++m) {
      pw.push_back(p[k]);
      ptd.push_back({theta[k], m});
    }
  }
  if (pw.empty()) fail(TCTL_E_NUMERIC, "preconditioner fit produced no positive weight");
  c.pre_terms_w = pw;
  c.pre_terms_t.clear();
  c.pre_terms_m.clear();
  for (const TermDesc &d : ptd) {
    c.pre_terms_t.push_back(d.t);
    c.pre_terms_m.push_back(d.lam_mode);
  }
}

// Device part: the factor matrices of both sums (they need the eigenvalues on
// the device) and, for pre_src 3, the sine-basis change W_l = S^T V_l.
void setup_spectral_build(Ctx &c) {
  const auto t0 = std::chrono::steady_clock::now();
  auto ms = [&]() {
    return std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
  };
  auto terms = [](const std::vector<double> &t, const std::vector<int> &m) {
    std::vector<TermDesc> td;
    for (size_t k = 0; k < t.size(); ++k) td.push_back({t[k], m[k]});
    return td;
  };
  build_sep(c, c.op, c.op_terms_w, terms(c.op_terms_t, c.op_terms_m));
  compress_sep(c, c.op, 1e-13);
  const double t_op = ms();
  if (c.o.pre_src == 3) {
    const int n = c.n;
    size_t mks = c.ws.mark();
    double *S = c.ws.dbl((size_t)n * n);
    const int blocks = (int)std::min<long long>(((long long)n * n + 255) / 256, 4096);
    LAUNCH(c, sine_basis_kernel, blocks, 256, 0, n, S);
    for (int l = 0; l < 3; ++l) {
      c.lamB[l] = c.dmalloc(n);
      LAUNCH(c, scaled_laplacian_eigs_kernel, (n + 255) / 256, 256, 0, n, c.b0[l], c.lamB[l]);
      c.W[l] = c.dmalloc((size_t)n * n);
      // W_l = S^T V_l (S symmetric): FP64 for the basis change of the preconditioner
      gemm(c, true, false, n, n, n, 1.0, S, n, 0, c.V[l], n, 0, 0.0, c.W[l], n, 0);
    }
    c.ws.reset(mks);
  }
  build_sep(c, c.pre, c.pre_terms_w, terms(c.pre_terms_t, c.pre_terms_m),
            c.o.pre_src == 3 ? c.lamB : nullptr);
  compress_sep(c, c.pre, 1e-13);
  if (c.trace)
    std::fprintf(stderr, "[tctl] spectral: sums fitted in %.1f ms; operator factors %.1f ms, "
                 "preconditioner %.1f ms\n", c.t_fit_ms, t_op, ms() - t_op);
}

void setup_spectral(Ctx &c) {
  setup_spectral_fit(c);
  setup_spectral_build(c);
}

// State operator A^-alpha (state equation of Section 3.1, y = A^-alpha u): the
// fitted exponential sum of s^-alpha (completely monotone), one Kronecker term
// per node; built on first use.
void ensure_state_sep(Ctx &c) {
  if (c.state.R > 0) return;
  const ExpFit f = fit_F2(c.alpha, kStateFn, c.s_min, c.s_max, c.o.op_tol);
  if (!(f.err <= c.o.op_tol)) fail(TCTL_E_NUMERIC, "state operator: exponential sum misses op_tol");
  std::vector<double> w(f.w);
  std::vector<TermDesc> td;
  for (double t : f.t) td.push_back({t, -1});
  build_sep(c, c.state, w, td);
  compress_sep(c, c.state, 1e-13);
  c.state_rel_err = f.err;
}

// ------------------------------------------------------------------ full grid
// u[i1 + n i2 + n^2 i3] /= F2(lam1[i1] + lam2[i2] + lam3[i3])  (which = 0)
// u *= (lam1+lam2+lam3)^-alpha                                  (which = 1)
__global__ void spectral_divide_kernel(int n, double *__restrict__ u, const double *__restrict__ l1,
                                       const double *__restrict__ l2, const double *__restrict__ l3,
                                       double alpha, double beta, int which) {
  const long long total = (long long)n * n * n;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < total;
       t += (long long)gridDim.x * blockDim.x) {
    const int i1 = (int)(t % n);
    const int i2 = (int)((t / n) % n);
    const int i3 = (int)(t / ((long long)n * n));
    const double s = l1[i1] + l2[i2] + l3[i3];
    const double p = pow(s, alpha);
    u[t] = (which == 0) ? u[t] / (1.0 / p + beta * p) : u[t] / p;
  }
}

void fullgrid_apply(Ctx &c, const double *y, double *u, int which) {
  const int n = c.n;
  const long long n2 = (long long)n * n, n3 = n2 * n;
  if (!c.full_tmp) c.full_tmp = c.dmalloc((size_t)n3);
  double *t = c.full_tmp;
  // forward: x (V1^T, V2^T, V3^T)
  gemm(c, true, false, n, (int)n2, n, 1.0, c.V[0], n, 0, y, n, 0, 0.0, t, n, 0);
  gemm(c, false, false, n, n, n, 1.0, t, n, n2, c.V[1], n, 0, 0.0, u, n, n2, n);
  gemm(c, false, false, (int)n2, n, n, 1.0, u, (int)n2, 0, c.V[2], n, 0, 0.0, t, (int)n2, 0);
  const int blocks = (int)std::min<long long>((n3 + 255) / 256, 152 * 32);
  LAUNCH(c, spectral_divide_kernel, blocks, 256, 0, n, t, c.lam[0], c.lam[1], c.lam[2], c.alpha,
         c.beta, which);
  // back: x (V1, V2, V3)
  gemm(c, false, false, n, (int)n2, n, 1.0, c.V[0], n, 0, t, n, 0, 0.0, u, n, 0);
  gemm(c, false, true, n, n, n, 1.0, u, n, n2, c.V[1], n, 0, 0.0, t, n, n2, n);
  gemm(c, false, true, (int)n2, n, n, 1.0, t, (int)n2, 0, c.V[2], n, 0, 0.0, u, (int)n2, 0);
}

}  // namespace tctl
