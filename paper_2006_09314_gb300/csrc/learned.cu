// Learned exponential sums for the preconditioner (Section 3.5, case (B)).
//
// The preconditioner P(s) = s sum_{k<r} p_k exp(-theta_k s) ~ 1/F2(s) with a
// few terms (r = 8..16) is what the eigenbasis PCG applies once per
// iteration; its quality is the spectral equivalence constant
//   delta = max_{s in [s_min, s_max]} |P(s) F2(s) - 1|,
// which bounds the condition number of the preconditioned operator by
// (1 + delta) / (1 - delta). This file holds
//   * the fitter: r free nodes and weights, log-parametrised (positive, so P
//     stays SPD), fitted by Levenberg-Marquardt on the relative residual
//     P F2 - 1 at 300 log-spaced points, with Lawson reweighting toward the
//     minimax fit, started from geometric nodes and NNLS weights;
//   * a multilayer perceptron 4 -> 64 -> 64 -> 2r (FP32, tanh) mapping
//     (alpha, log10 beta, ln s_min, ln s_max) to the fitted (ln tau, ln q)
//     in the scaled variable x = s / s_min, trained on the GPU by the kernels
//     below (forward, backward, Adam), one training step captured in a CUDA
//     graph and replayed;
//   * inference: the network's nodes, with the weights re-solved by NNLS on
//     those nodes (one small least-squares problem on the host).
// The same fitter and network serve the operator: an r-term sum
// g(s) = F2(s)/s ~ sum_k w_k exp(-t_k s) (F2 = s g, 3 Kronecker terms per
// node; Section 3.4's exponential-sum representation with free nodes), whose
// quality is the measured max relative error of F2 on [s_min, s_max].
#include <algorithm>
#include <cmath>
#include <numeric>
#include <thread>
#include <vector>

#include "tctl_internal.cuh"

namespace tctl {

namespace {

constexpr int kFitM = 300;      // fitting samples
constexpr int kCheckM = 2000;   // samples of the measured delta

double F2s(double s, double a, double b) { return std::pow(s, -a) + b * std::pow(s, a); }
// P(s)/s must approximate h(s) = 1 / (s F2(s)); the operator's sum approximates
// g(s) = F2(s) / s
double h_of(double s, double a, double b) { return 1.0 / (s * F2s(s, a, b)); }
double target_of(FitTarget t, double s, double a, double b) {
  return t == FitTarget::Pre ? h_of(s, a, b) : F2s(s, a, b) / s;
}

// Cholesky solve of the SPD system A x = b (n x n, row-major); false if not SPD.
bool chol_solve(std::vector<double> A, std::vector<double> &x, int n) {
  for (int j = 0; j < n; ++j) {
    double d = A[j * n + j];
    for (int k = 0; k < j; ++k) d -= A[j * n + k] * A[j * n + k];
    if (!(d > 0.0) || !std::isfinite(d)) return false;
    d = std::sqrt(d);
    A[j * n + j] = d;
    for (int i = j + 1; i < n; ++i) {
      double v = A[i * n + j];
      for (int k = 0; k < j; ++k) v -= A[i * n + k] * A[j * n + k];
      A[i * n + j] = v / d;
    }
  }
  for (int i = 0; i < n; ++i) {
    double v = x[i];
    for (int k = 0; k < i; ++k) v -= A[i * n + k] * x[k];
    x[i] = v / A[i * n + i];
  }
  for (int i = n - 1; i >= 0; --i) {
    double v = x[i];
    for (int k = i + 1; k < n; ++k) v -= A[k * n + i] * x[k];
    x[i] = v / A[i * n + i];
  }
  return true;
}

}  // namespace

// max over 2000 log-spaced s of |sum_k w_k exp(-t_k s) / target(s) - 1|: for the
// preconditioner delta = max |P F2 - 1|, for the operator the relative error of F2
double sum_rel_err(FitTarget tg, const double *t, const double *w, int r, double a, double b,
                   double smin, double smax) {
  double dmax = 0.0;
  for (int j = 0; j < kCheckM; ++j) {
    const double s = std::exp(std::log(smin) + (std::log(smax) - std::log(smin)) * j / (kCheckM - 1));
    double v = 0.0;
    for (int k = 0; k < r; ++k) v += w[k] * std::exp(-t[k] * s);
    dmax = std::max(dmax, std::fabs(v / target_of(tg, s, a, b) - 1.0));
  }
  return dmax;
}

double pre_delta(const double *theta, const double *p, int r, double a, double b, double smin,
                 double smax) {
  return sum_rel_err(FitTarget::Pre, theta, p, r, a, b, smin, smax);
}

// NNLS weights on fixed nodes (s units) minimising the relative residual
// sum_k w_k exp(-t_k s_j) / target(s_j) - 1 on kFitM samples; w >= 0.
std::vector<double> weights_nnls(FitTarget tg, const std::vector<double> &theta, double a, double b,
                                 double smin, double smax) {
  const int r = (int)theta.size(), M = kFitM;
  std::vector<double> A((size_t)M * r), cs(r), rhs(M, 1.0);
  for (int k = 0; k < r; ++k) {
    double nrm = 0;
    for (int j = 0; j < M; ++j) {
      const double s = std::exp(std::log(smin) + (std::log(smax) - std::log(smin)) * j / (M - 1));
      const double v = std::exp(-theta[k] * s) / target_of(tg, s, a, b);
      A[j + (size_t)k * M] = v;
      nrm += v * v;
    }
    cs[k] = nrm > 0 ? std::sqrt(nrm) : 1.0;
    for (int j = 0; j < M; ++j) A[j + (size_t)k * M] /= cs[k];
  }
  std::vector<double> q = nnls_solve(A, M, r, rhs);
  for (int k = 0; k < r; ++k) q[k] /= cs[k];
  return q;
}

std::vector<double> pre_weights_nnls(const std::vector<double> &theta, double a, double b, double smin,
                                     double smax) {
  return weights_nnls(FitTarget::Pre, theta, a, b, smin, smax);
}

// r-term fit. Outputs tau (ascending, x = s / s_min units) and q (weights of
// exp(-tau x) approximating h(s_min x) / h(s_min)); theta = tau / s_min,
// p = q h(s_min). Returns the measured delta.
namespace {

// One Levenberg-Marquardt run from geometric nodes over [lo / rho, hi] (x units).
double fit_from(FitTarget tg, double a, double b, double smin, double smax, int r, double lo,
                double hi, double *tau_out, double *q_out) {
  const int M = kFitM, P = 2 * r;
  const double rho = smax / smin, h0 = target_of(tg, smin, a, b);
  std::vector<double> x(M), H(M);
  for (int j = 0; j < M; ++j) {
    x[j] = std::exp(std::log(rho) * j / (M - 1));
    H[j] = target_of(tg, smin * x[j], a, b) / h0;
  }
  // start: geometric nodes in [0.05 / rho, 20], NNLS weights (zeros lifted)
  std::vector<double> th(P);
  {
    std::vector<double> theta(r);
    for (int k = 0; k < r; ++k)
      theta[k] = std::exp(std::log(lo / rho) + (std::log(hi) - std::log(lo / rho)) * k / std::max(1, r - 1)) / smin;
    std::vector<double> p = weights_nnls(tg, theta, a, b, smin, smax);
    double pmax = 0;
    for (double v : p) pmax = std::max(pmax, v);
    if (!(pmax > 0)) pmax = h0;
    for (int k = 0; k < r; ++k) {
      th[k] = std::log(theta[k] * smin);
      th[r + k] = std::log(std::max(p[k], 1e-6 * pmax) / h0);
    }
  }
  std::vector<double> f(M), J((size_t)M * P), u(M, 1.0), JtJ((size_t)P * P), g(P), d(P), th2(P), f2(M);
  auto residual = [&](const std::vector<double> &t, std::vector<double> &out, bool jac) {
    for (int j = 0; j < M; ++j) {
      double v = 0.0;
      for (int k = 0; k < r; ++k) {
        const double tk = std::exp(t[k]), qk = std::exp(t[r + k]);
        const double e = qk * std::exp(-tk * x[j]) / H[j];
        v += e;
        if (jac) {
          J[(size_t)j * P + k] = -e * tk * x[j];
          J[(size_t)j * P + r + k] = e;
        }
      }
      out[j] = v - 1.0;
    }
  };
  auto wcost = [&](const std::vector<double> &ff) {
    double c = 0;
    for (int j = 0; j < M; ++j) c += u[j] * ff[j] * ff[j];
    return c;
  };
  auto maxabs = [&](const std::vector<double> &ff) {
    double m = 0;
    for (double v : ff) m = std::max(m, std::fabs(v));
    return m;
  };
  residual(th, f, true);
  std::vector<double> best = th;
  double best_max = maxabs(f);
  double mu = 1e-3;
  for (int round = 0; round < 6; ++round) {
    for (int it = 0; it < 25; ++it) {
      std::fill(JtJ.begin(), JtJ.end(), 0.0);
      std::fill(g.begin(), g.end(), 0.0);
      for (int j = 0; j < M; ++j) {
        const double *Jj = &J[(size_t)j * P];
        for (int a1 = 0; a1 < P; ++a1) {
          g[a1] += u[j] * Jj[a1] * f[j];
          for (int a2 = 0; a2 <= a1; ++a2) JtJ[a1 * P + a2] += u[j] * Jj[a1] * Jj[a2];
        }
      }
      for (int a1 = 0; a1 < P; ++a1)
        for (int a2 = 0; a2 < a1; ++a2) JtJ[a2 * P + a1] = JtJ[a1 * P + a2];
      const double c0 = wcost(f);
      bool moved = false;
      for (int tries = 0; tries < 8 && !moved; ++tries) {
        std::vector<double> A = JtJ;
        for (int a1 = 0; a1 < P; ++a1) A[a1 * P + a1] += mu * (JtJ[a1 * P + a1] + 1e-12);
        for (int a1 = 0; a1 < P; ++a1) d[a1] = -g[a1];
        if (!chol_solve(A, d, P)) {
          mu *= 10;
          continue;
        }
        for (int a1 = 0; a1 < P; ++a1) th2[a1] = th[a1] + std::max(-2.0, std::min(2.0, d[a1]));
        residual(th2, f2, false);
        if (wcost(f2) < c0 && std::isfinite(wcost(f2))) {
          th = th2;
          mu = std::max(mu / 3.0, 1e-12);
          moved = true;
        } else {
          mu *= 4.0;
        }
      }
      residual(th, f, true);
      const double m = maxabs(f);
      if (m < best_max) {
        best_max = m;
        best = th;
      }
      if (!moved) break;
    }
    // Lawson: weight the samples where the fit is worst
    const double m = maxabs(f);
    double mean = 0;
    for (int j = 0; j < M; ++j) {
      u[j] *= std::fabs(f[j]) + 0.1 * m;
      mean += u[j];
    }
    mean /= M;
    if (!(mean > 0)) break;
    for (int j = 0; j < M; ++j) u[j] /= mean;
  }
  // ascending nodes
  std::vector<int> ord(r);
  std::iota(ord.begin(), ord.end(), 0);
  std::sort(ord.begin(), ord.end(), [&](int i, int j) { return best[i] < best[j]; });
  std::vector<double> theta(r), p(r);
  for (int k = 0; k < r; ++k) {
    tau_out[k] = std::exp(best[ord[k]]);
    q_out[k] = std::exp(best[r + ord[k]]);
    theta[k] = tau_out[k] / smin;
    p[k] = q_out[k] * h0;
  }
  return sum_rel_err(tg, theta.data(), p.data(), r, a, b, smin, smax);
}

}  // namespace

// r-term fit, best of up to three starts: the node range of the K-node default
// first, two more ranges when the first run gains less than 2x over its start.
double expsum_fit_r(FitTarget tg, double a, double b, double smin, double smax, int r, double *tau_out,
                    double *q_out) {
  std::vector<double> theta(r), tb(r), qb(r);
  const double rho = smax / smin;
  for (int k = 0; k < r; ++k)
    theta[k] = std::exp(std::log(0.05 / rho) + (std::log(20.0) - std::log(0.05 / rho)) * k / std::max(1, r - 1)) / smin;
  const std::vector<double> pg = weights_nnls(tg, theta, a, b, smin, smax);
  const double d_geo = sum_rel_err(tg, theta.data(), pg.data(), r, a, b, smin, smax);
  double best = fit_from(tg, a, b, smin, smax, r, 0.05, 20.0, tau_out, q_out);
  const double starts[2][2] = {{0.5, 5.0}, {0.005, 100.0}};
  for (int t = 0; t < 2 && best > 0.5 * d_geo; ++t) {
    const double d = fit_from(tg, a, b, smin, smax, r, starts[t][0], starts[t][1], tb.data(), qb.data());
    if (d < best) {
      best = d;
      std::copy(tb.begin(), tb.end(), tau_out);
      std::copy(qb.begin(), qb.end(), q_out);
    }
  }
  return best;
}

double pre_fit(double a, double b, double smin, double smax, int r, double *tau_out, double *q_out) {
  return expsum_fit_r(FitTarget::Pre, a, b, smin, smax, r, tau_out, q_out);
}

}  // namespace tctl

// =====================================================================
// Multilayer perceptron 4 -> 64 -> 64 -> O (O = 2r), FP32, tanh hidden
// layers. Parameters, contiguous: W1 (64 x 4, row = output), b1 (64),
// W2 (64 x 64), b2 (64), W3 (O x 64), b3 (O). A model blob appends the
// input mean and std (4 + 4) and the output mean and std (O + O).
// =====================================================================
namespace tctl {

int mlp_param_count(int O) { return kMlpH * kMlpIn + kMlpH + kMlpH * kMlpH + kMlpH + O * kMlpH + O; }

namespace {

struct MlpView {
  float *W1, *b1, *W2, *b2, *W3, *b3;
};

MlpView mlp_view(float *p, int O) {
  MlpView v;
  v.W1 = p;
  v.b1 = v.W1 + kMlpH * kMlpIn;
  v.W2 = v.b1 + kMlpH;
  v.b2 = v.W2 + kMlpH * kMlpH;
  v.W3 = v.b2 + kMlpH;
  v.b3 = v.W3 + O * kMlpH;
  return v;
}

// out[b, o] = act(sum_i in[b, i] W[o, i] + bias[o]); act: 1 tanh, 0 identity
__global__ void dense_fwd_kernel(int B, int I, int Oo, const float *__restrict__ in,
                                 const float *__restrict__ W, const float *__restrict__ bias, int act,
                                 float *__restrict__ out) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= B * Oo) return;
  const int b = t / Oo, o = t % Oo;
  float s = bias[o];
  for (int i = 0; i < I; ++i) s = fmaf(in[b * I + i], W[o * I + i], s);
  out[t] = act ? tanhf(s) : s;
}

// dY = 2 (Y - T) / (B O); loss += sum (Y - T)^2 / (B O)
__global__ void mse_grad_kernel(int B, int O, const float *__restrict__ Y, const float *__restrict__ T,
                                float *__restrict__ dY, float *loss) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  float l = 0.0f;
  if (t < B * O) {
    const float d = Y[t] - T[t];
    dY[t] = 2.0f * d / (float)(B * O);
    l = d * d / (float)(B * O);
  }
  for (int s = 16; s > 0; s >>= 1) l += __shfl_down_sync(0xffffffffu, l, s);
  if ((threadIdx.x & 31) == 0 && loss) atomicAdd(loss, l);
}

// dIn[b, i] = (sum_o dOut[b, o] W[o, i]) (1 - h[b, i]^2)   (h = tanh activations of the input)
__global__ void dense_bwd_in_kernel(int B, int I, int Oo, const float *__restrict__ dOut,
                                    const float *__restrict__ W, const float *__restrict__ h,
                                    float *__restrict__ dIn) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= B * I) return;
  const int b = t / I, i = t % I;
  float s = 0.0f;
  for (int o = 0; o < Oo; ++o) s = fmaf(dOut[b * Oo + o], W[o * I + i], s);
  const float hv = h[t];
  dIn[t] = s * (1.0f - hv * hv);
}

// dW[o, i] = sum_b dOut[b, o] in[b, i]; db[o] = sum_b dOut[b, o]
__global__ void dense_bwd_w_kernel(int B, int I, int Oo, const float *__restrict__ dOut,
                                   const float *__restrict__ in, float *__restrict__ dW,
                                   float *__restrict__ db) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= Oo * (I + 1)) return;
  const int o = t / (I + 1), i = t % (I + 1);
  float s = 0.0f;
  if (i < I)
    for (int b = 0; b < B; ++b) s = fmaf(dOut[b * Oo + o], in[b * I + i], s);
  else
    for (int b = 0; b < B; ++b) s += dOut[b * Oo + o];
  if (i < I) dW[o * I + i] = s;
  else db[o] = s;
}

// Adam with bias correction and a cosine learning-rate decay to lr/20 over
// `total` steps; the step counter is read from device memory (graph replay).
__global__ void adam_kernel(int P, float *__restrict__ w, const float *__restrict__ g,
                            float *__restrict__ m, float *__restrict__ v, const int *__restrict__ step,
                            float lr0, int total, float b1, float b2, float eps) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= P) return;
  const int k = *step + 1;
  const float frac = fminf(1.0f, (float)k / (float)max(total, 1));
  const float lr = lr0 * (0.05f + 0.95f * 0.5f * (1.0f + cospif(frac)));
  const float mt = b1 * m[t] + (1.0f - b1) * g[t];
  const float vt = b2 * v[t] + (1.0f - b2) * g[t] * g[t];
  m[t] = mt;
  v[t] = vt;
  const float mh = mt / (1.0f - powf(b1, (float)k)), vh = vt / (1.0f - powf(b2, (float)k));
  w[t] -= lr * mh / (sqrtf(vh) + eps);
}

// batch rows (step * B + i) mod N of a fixed permutation
__global__ void gather_batch_kernel(int B, int O, int N, const int *__restrict__ perm,
                                    const int *__restrict__ step, const float *__restrict__ X,
                                    const float *__restrict__ Yt, float *__restrict__ xb,
                                    float *__restrict__ tb) {
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= B) return;
  const int row = perm[(int)(((long long)(*step) * B + b) % N)];
  for (int i = 0; i < kMlpIn; ++i) xb[b * kMlpIn + i] = X[(long long)row * kMlpIn + i];
  for (int o = 0; o < O; ++o) tb[b * O + o] = Yt[(long long)row * O + o];
}

__global__ void step_inc_kernel(int *step) { *step += 1; }

// per-sample inference: y = W3 tanh(W2 tanh(W1 x + b1) + b2) + b3
__global__ void mlp_infer_kernel(int n, int O, const float *__restrict__ p, const float *__restrict__ X,
                                 float *__restrict__ Y) {
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= n) return;
  const float *W1 = p, *b1 = W1 + kMlpH * kMlpIn, *W2 = b1 + kMlpH, *b2 = W2 + kMlpH * kMlpH,
              *W3 = b2 + kMlpH, *b3 = W3 + O * kMlpH;
  float h1[kMlpH], h2[kMlpH];
  for (int o = 0; o < kMlpH; ++o) {
    float a = b1[o];
    for (int i = 0; i < kMlpIn; ++i) a = fmaf(X[s * kMlpIn + i], W1[o * kMlpIn + i], a);
    h1[o] = tanhf(a);
  }
  for (int o = 0; o < kMlpH; ++o) {
    float a = b2[o];
    for (int i = 0; i < kMlpH; ++i) a = fmaf(h1[i], W2[o * kMlpH + i], a);
    h2[o] = tanhf(a);
  }
  for (int o = 0; o < O; ++o) {
    float a = b3[o];
    for (int i = 0; i < kMlpH; ++i) a = fmaf(h2[i], W3[o * kMlpH + i], a);
    Y[s * O + o] = a;
  }
}

inline int nblk(long long n) { return (int)((n + 255) / 256); }

}  // namespace

// One forward + backward pass for a batch already on the device.
// Buffers: xb (B x 4), tb (B x O), h1, h2 (B x 64), y, dy (B x O), d2, d1 (B x 64), grads (P).
struct MlpBatchBufs {
  float *xb, *tb, *h1, *h2, *y, *dy, *d2, *d1, *grad, *loss;
};

void mlp_fwd_bwd(cudaStream_t st, int B, int O, float *params, const MlpBatchBufs &q) {
  MlpView w = mlp_view(params, O), g = mlp_view(q.grad, O);
  dense_fwd_kernel<<<nblk((long long)B * kMlpH), 256, 0, st>>>(B, kMlpIn, kMlpH, q.xb, w.W1, w.b1, 1, q.h1);
  dense_fwd_kernel<<<nblk((long long)B * kMlpH), 256, 0, st>>>(B, kMlpH, kMlpH, q.h1, w.W2, w.b2, 1, q.h2);
  dense_fwd_kernel<<<nblk((long long)B * O), 256, 0, st>>>(B, kMlpH, O, q.h2, w.W3, w.b3, 0, q.y);
  mse_grad_kernel<<<nblk((long long)B * O), 256, 0, st>>>(B, O, q.y, q.tb, q.dy, q.loss);
  dense_bwd_w_kernel<<<nblk((long long)O * (kMlpH + 1)), 256, 0, st>>>(B, kMlpH, O, q.dy, q.h2, g.W3, g.b3);
  dense_bwd_in_kernel<<<nblk((long long)B * kMlpH), 256, 0, st>>>(B, kMlpH, O, q.dy, w.W3, q.h2, q.d2);
  dense_bwd_w_kernel<<<nblk((long long)kMlpH * (kMlpH + 1)), 256, 0, st>>>(B, kMlpH, kMlpH, q.d2, q.h1, g.W2, g.b2);
  dense_bwd_in_kernel<<<nblk((long long)B * kMlpH), 256, 0, st>>>(B, kMlpH, kMlpH, q.d2, w.W2, q.h1, q.d1);
  dense_bwd_w_kernel<<<nblk((long long)kMlpH * (kMlpIn + 1)), 256, 0, st>>>(B, kMlpIn, kMlpH, q.d1, q.xb, g.W1, g.b1);
}

void mlp_adam_step(cudaStream_t st, int P, float *params, const float *grad, float *m, float *v,
                   const int *step, float lr, int total) {
  adam_kernel<<<nblk(P), 256, 0, st>>>(P, params, grad, m, v, step, lr, total, 0.9f, 0.999f, 1e-8f);
}

void mlp_gather(cudaStream_t st, int B, int O, int N, const int *perm, const int *step, const float *X,
                const float *Y, float *xb, float *tb) {
  gather_batch_kernel<<<nblk(B), 256, 0, st>>>(B, O, N, perm, step, X, Y, xb, tb);
}

void mlp_step_inc(cudaStream_t st, int *step) { step_inc_kernel<<<1, 1, 0, st>>>(step); }

void mlp_infer(cudaStream_t st, int n, int O, const float *params, const float *X, float *Y) {
  mlp_infer_kernel<<<nblk(n), 256, 0, st>>>(n, O, params, X, Y);
}

}  // namespace tctl

// =====================================================================
// Host entry points (C ABI) of the learned preconditioner sums
// =====================================================================
namespace tctl {
namespace {

uint64_t splitmix(uint64_t x) {
  x += 0x9E3779B97F4A7C15ull;
  x = (x ^ (x >> 30)) * 0xBF58476D1CE4E5B9ull;
  x = (x ^ (x >> 27)) * 0x94D049BB133111EBull;
  return x ^ (x >> 31);
}
double unit(uint64_t seed, uint64_t i, uint64_t j) {
  return (double)(splitmix(seed * 0x100000001B3ull + i * 16 + j) >> 11) * (1.0 / 9007199254740992.0);
}

struct DevBuf {
  void *p = nullptr;
  ~DevBuf() {
    if (p) cudaFree(p);
  }
  template <class T>
  T *alloc(size_t n) {
    check_cuda(cudaMalloc(&p, std::max<size_t>(n, 1) * sizeof(T)), "cudaMalloc(mlp)");
    return static_cast<T *>(p);
  }
};

struct StreamGuard {
  cudaStream_t s = nullptr;
  cudaGraph_t g = nullptr;
  cudaGraphExec_t e = nullptr;
  ~StreamGuard() {
    if (e) cudaGraphExecDestroy(e);
    if (g) cudaGraphDestroy(g);
    if (s) {
      cudaStreamSynchronize(s);
      cudaStreamDestroy(s);
    }
  }
};

}  // namespace

void precond_sample_inputs(int N, uint64_t seed, float *X) {
  for (int i = 0; i < N; ++i) {
    X[i * 4 + 0] = (float)(0.1 + 0.8 * unit(seed, i, 0));           // alpha
    X[i * 4 + 1] = (float)(-4.0 + 4.0 * unit(seed, i, 1));          // log10 beta
    X[i * 4 + 2] = (float)std::log(15.0 + 30.0 * unit(seed, i, 2));  // ln s_min
    X[i * 4 + 3] = (float)(std::log(10.0) * (4.5 + 4.0 * unit(seed, i, 3)));  // ln s_max
  }
}

void expsum_dataset(FitTarget tg, int r, int N, const float *X, int threads, float *Y, double *delta) {
  const int O = 2 * r;
  auto work = [&](int t0) {
    std::vector<double> tau(r), q(r);
    for (int i = t0; i < N; i += threads) {
      const double a = X[i * 4 + 0], b = std::pow(10.0, (double)X[i * 4 + 1]);
      const double smin = std::exp((double)X[i * 4 + 2]), smax = std::exp((double)X[i * 4 + 3]);
      const double d = expsum_fit_r(tg, a, b, smin, smax, r, tau.data(), q.data());
      for (int k = 0; k < r; ++k) {
        Y[(size_t)i * O + k] = (float)std::log(tau[k]);
        Y[(size_t)i * O + r + k] = (float)std::log(q[k]);
      }
      if (delta) delta[i] = d;
    }
  };
  std::vector<std::thread> pool;
  for (int t = 1; t < threads; ++t) pool.emplace_back(work, t);
  work(0);
  for (auto &th : pool) th.join();
}

void mlp_train(int r, int N, const float *X, const float *Y, int steps, int B, float lr,
               uint64_t seed, float *model, float *loss_out) {
  const int O = 2 * r, P = mlp_param_count(O);
  // normalisation of inputs and targets
  std::vector<float> mu_in(4, 0), sd_in(4, 0), mu_out(O, 0), sd_out(O, 0);
  for (int i = 0; i < N; ++i) {
    for (int j = 0; j < 4; ++j) mu_in[j] += X[i * 4 + j] / N;
    for (int j = 0; j < O; ++j) mu_out[j] += Y[(size_t)i * O + j] / N;
  }
  for (int i = 0; i < N; ++i) {
    for (int j = 0; j < 4; ++j) sd_in[j] += (X[i * 4 + j] - mu_in[j]) * (X[i * 4 + j] - mu_in[j]) / N;
    for (int j = 0; j < O; ++j)
      sd_out[j] += (Y[(size_t)i * O + j] - mu_out[j]) * (Y[(size_t)i * O + j] - mu_out[j]) / N;
  }
  for (float &v : sd_in) v = std::sqrt(std::max(v, 1e-12f));
  for (float &v : sd_out) v = std::sqrt(std::max(v, 1e-12f));
  std::vector<float> Xn((size_t)N * 4), Yn((size_t)N * O);
  for (int i = 0; i < N; ++i) {
    for (int j = 0; j < 4; ++j) Xn[i * 4 + j] = (X[i * 4 + j] - mu_in[j]) / sd_in[j];
    for (int j = 0; j < O; ++j) Yn[(size_t)i * O + j] = (Y[(size_t)i * O + j] - mu_out[j]) / sd_out[j];
  }
  // Glorot-uniform weights, zero biases
  std::vector<float> w(P, 0.0f);
  {
    auto fill = [&](float *Wp, int fo, int fi, uint64_t tag) {
      const double a = std::sqrt(6.0 / (fo + fi));
      for (int t = 0; t < fo * fi; ++t) Wp[t] = (float)(a * (2.0 * unit(seed + tag, t, 0) - 1.0));
    };
    MlpView v = mlp_view(w.data(), O);
    fill(v.W1, kMlpH, kMlpIn, 1);
    fill(v.W2, kMlpH, kMlpH, 2);
    fill(v.W3, O, kMlpH, 3);
  }
  std::vector<int> perm(N);
  std::iota(perm.begin(), perm.end(), 0);
  for (int i = N - 1; i > 0; --i) std::swap(perm[i], perm[(int)(unit(seed, i, 7) * (i + 1))]);
  StreamGuard sg;
  check_cuda(cudaStreamCreateWithFlags(&sg.s, cudaStreamNonBlocking), "cudaStreamCreate");
  DevBuf dX, dY, dperm, dw, dm, dv, dg, dstep, dxb, dtb, dh1, dh2, dy, ddy, dd2, dd1, dloss;
  float *Xd = dX.alloc<float>((size_t)N * 4), *Yd = dY.alloc<float>((size_t)N * O);
  int *permd = dperm.alloc<int>(N), *step = dstep.alloc<int>(1);
  float *wd = dw.alloc<float>(P), *md = dm.alloc<float>(P), *vd = dv.alloc<float>(P), *gd = dg.alloc<float>(P);
  const int Bfull = std::max(B, std::min(N, 4096));
  MlpBatchBufs q;
  q.xb = dxb.alloc<float>((size_t)Bfull * 4);
  q.tb = dtb.alloc<float>((size_t)Bfull * O);
  q.h1 = dh1.alloc<float>((size_t)Bfull * kMlpH);
  q.h2 = dh2.alloc<float>((size_t)Bfull * kMlpH);
  q.y = dy.alloc<float>((size_t)Bfull * O);
  q.dy = ddy.alloc<float>((size_t)Bfull * O);
  q.d2 = dd2.alloc<float>((size_t)Bfull * kMlpH);
  q.d1 = dd1.alloc<float>((size_t)Bfull * kMlpH);
  q.grad = gd;
  q.loss = dloss.alloc<float>(1);
  cudaStream_t st = sg.s;
  check_cuda(cudaMemcpyAsync(Xd, Xn.data(), sizeof(float) * Xn.size(), cudaMemcpyHostToDevice, st), "H2D");
  check_cuda(cudaMemcpyAsync(Yd, Yn.data(), sizeof(float) * Yn.size(), cudaMemcpyHostToDevice, st), "H2D");
  check_cuda(cudaMemcpyAsync(permd, perm.data(), sizeof(int) * N, cudaMemcpyHostToDevice, st), "H2D");
  check_cuda(cudaMemcpyAsync(wd, w.data(), sizeof(float) * P, cudaMemcpyHostToDevice, st), "H2D");
  check_cuda(cudaMemsetAsync(md, 0, sizeof(float) * P, st), "memset");
  check_cuda(cudaMemsetAsync(vd, 0, sizeof(float) * P, st), "memset");
  check_cuda(cudaMemsetAsync(step, 0, sizeof(int), st), "memset");
  // full-dataset loss (chunks of Bfull rows, in dataset order)
  std::vector<int> ident(N);
  std::iota(ident.begin(), ident.end(), 0);
  DevBuf did;
  int *identd = did.alloc<int>(N);
  check_cuda(cudaMemcpyAsync(identd, ident.data(), sizeof(int) * N, cudaMemcpyHostToDevice, st), "H2D");
  auto full_loss = [&]() {
    double tot = 0.0;
    DevBuf dz;
    int *zero_step = dz.alloc<int>(1);
    for (int r0 = 0; r0 < N; r0 += Bfull) {
      const int nb = std::min(Bfull, N - r0);
      check_cuda(cudaMemcpyAsync(q.xb, Xd + (size_t)r0 * 4, sizeof(float) * nb * 4, cudaMemcpyDeviceToDevice, st), "D2D");
      check_cuda(cudaMemcpyAsync(q.tb, Yd + (size_t)r0 * O, sizeof(float) * nb * O, cudaMemcpyDeviceToDevice, st), "D2D");
      check_cuda(cudaMemsetAsync(q.loss, 0, sizeof(float), st), "memset");
      mlp_fwd_bwd(st, nb, O, wd, q);
      float l = 0;
      check_cuda(cudaMemcpyAsync(&l, q.loss, sizeof(float), cudaMemcpyDeviceToHost, st), "D2H");
      check_cuda(cudaStreamSynchronize(st), "sync");
      tot += (double)l * nb;
    }
    (void)zero_step;
    return tot / N;
  };
  if (loss_out) loss_out[0] = (float)full_loss();
  // one training step, captured once and replayed
  check_cuda(cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal), "capture");
  mlp_gather(st, B, O, N, permd, step, Xd, Yd, q.xb, q.tb);
  mlp_fwd_bwd(st, B, O, wd, MlpBatchBufs{q.xb, q.tb, q.h1, q.h2, q.y, q.dy, q.d2, q.d1, q.grad, nullptr});
  mlp_adam_step(st, P, wd, gd, md, vd, step, lr, steps);
  mlp_step_inc(st, step);
  check_cuda(cudaStreamEndCapture(st, &sg.g), "end capture");
  check_cuda(cudaGraphInstantiate(&sg.e, sg.g, 0), "graph instantiate");
  for (int t = 0; t < steps; ++t) check_cuda(cudaGraphLaunch(sg.e, st), "graph launch");
  check_cuda(cudaStreamSynchronize(st), "sync");
  if (loss_out) loss_out[1] = (float)full_loss();
  check_cuda(cudaMemcpyAsync(model, wd, sizeof(float) * P, cudaMemcpyDeviceToHost, st), "D2H");
  check_cuda(cudaStreamSynchronize(st), "sync");
  for (int j = 0; j < 4; ++j) {
    model[P + j] = mu_in[j];
    model[P + 4 + j] = sd_in[j];
  }
  for (int j = 0; j < O; ++j) {
    model[P + 8 + j] = mu_out[j];
    model[P + 8 + O + j] = sd_out[j];
  }
}

void mlp_grad_host(int r, int B, const float *params, const float *X, const float *T, float *grad,
                   float *loss) {
  const int O = 2 * r, P = mlp_param_count(O);
  StreamGuard sg;
  check_cuda(cudaStreamCreateWithFlags(&sg.s, cudaStreamNonBlocking), "cudaStreamCreate");
  DevBuf dw, dg, dxb, dtb, dh1, dh2, dy, ddy, dd2, dd1, dloss;
  float *wd = dw.alloc<float>(P);
  MlpBatchBufs q;
  q.xb = dxb.alloc<float>((size_t)B * 4);
  q.tb = dtb.alloc<float>((size_t)B * O);
  q.h1 = dh1.alloc<float>((size_t)B * kMlpH);
  q.h2 = dh2.alloc<float>((size_t)B * kMlpH);
  q.y = dy.alloc<float>((size_t)B * O);
  q.dy = ddy.alloc<float>((size_t)B * O);
  q.d2 = dd2.alloc<float>((size_t)B * kMlpH);
  q.d1 = dd1.alloc<float>((size_t)B * kMlpH);
  q.grad = dg.alloc<float>(P);
  q.loss = dloss.alloc<float>(1);
  cudaStream_t st = sg.s;
  check_cuda(cudaMemcpyAsync(wd, params, sizeof(float) * P, cudaMemcpyHostToDevice, st), "H2D");
  check_cuda(cudaMemcpyAsync(q.xb, X, sizeof(float) * B * 4, cudaMemcpyHostToDevice, st), "H2D");
  check_cuda(cudaMemcpyAsync(q.tb, T, sizeof(float) * B * O, cudaMemcpyHostToDevice, st), "H2D");
  check_cuda(cudaMemsetAsync(q.loss, 0, sizeof(float), st), "memset");
  mlp_fwd_bwd(st, B, O, wd, q);
  check_cuda(cudaGetLastError(), "mlp kernels");
  check_cuda(cudaMemcpyAsync(grad, q.grad, sizeof(float) * P, cudaMemcpyDeviceToHost, st), "D2H");
  check_cuda(cudaMemcpyAsync(loss, q.loss, sizeof(float), cudaMemcpyDeviceToHost, st), "D2H");
  check_cuda(cudaStreamSynchronize(st), "sync");
}

// raw (ln tau, ln q) for raw inputs, on the device given by `st`
void mlp_forward_host(int r, int n, const float *model, const float *X, float *Yout, cudaStream_t st) {
  const int O = 2 * r, P = mlp_param_count(O);
  std::vector<float> Xn((size_t)n * 4);
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < 4; ++j) Xn[i * 4 + j] = (X[i * 4 + j] - model[P + j]) / model[P + 4 + j];
  DevBuf dw, dx, dyv;
  float *wd = dw.alloc<float>(P), *xd = dx.alloc<float>((size_t)n * 4), *yd = dyv.alloc<float>((size_t)n * O);
  check_cuda(cudaMemcpyAsync(wd, model, sizeof(float) * P, cudaMemcpyHostToDevice, st), "H2D");
  check_cuda(cudaMemcpyAsync(xd, Xn.data(), sizeof(float) * n * 4, cudaMemcpyHostToDevice, st), "H2D");
  mlp_infer(st, n, O, wd, xd, yd);
  check_cuda(cudaGetLastError(), "mlp_infer_kernel");
  check_cuda(cudaMemcpyAsync(Yout, yd, sizeof(float) * n * O, cudaMemcpyDeviceToHost, st), "D2H");
  check_cuda(cudaStreamSynchronize(st), "sync");
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < O; ++j) Yout[(size_t)i * O + j] = Yout[(size_t)i * O + j] * model[P + 8 + O + j] + model[P + 8 + j];
}

}  // namespace tctl
