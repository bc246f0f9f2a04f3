// 1D Sturm-Liouville operators and their eigenbasis on the GPU, FP64.
//
// Section 3.2: A_(l) is tridiagonal with diagonal (a_{i-1/2} + a_{i+1/2})/h^2
// and off-diagonal -a_{i+1/2}/h^2 (h = 1/(n+1)); with paper_end_rows the
// first and last diagonal entries are the printed 2 a_{3/2}/h^2 and
// 2 a_{n-1/2}/h^2.
// Section 3.3 ("eigs_1D"): A_(l) = V_l diag(lambda^(l)) V_l^T. The paper
// calls this cubic-cost step negligible; here it is done in parallel:
//   * eigenvalues: Sturm-sequence bisection, one thread per eigenvalue
//     (inertia counts of T - x I are monotone in x);
//   * eigenvectors: one twisted factorization of T - lambda I per
//     eigenvalue (forward and backward LDL-type recurrences, twist index at
//     the smallest |gamma_k|), which gives (T - lambda I) z = gamma_r e_r;
//     z is normalised and its sign fixed so that sum_i z_i g_i > 0 with the
//     Weyl weights g_i = 2 frac(i * 0.6180339887498949) - 1, i = 1..n (the
//     first entry of a localized high mode can underflow, so it cannot fix
//     the sign).
// Eigenvalues are ascending; V_l is column-major with eigenvectors as columns.
#include <algorithm>
#include <chrono>
#include <cstdio>
#include <cfloat>
#include <cmath>
#include <mutex>
#include <string>

#include "tctl_internal.cuh"

namespace tctl {

__global__ void assemble_kernel(int n, const double *__restrict__ coef, int paper_end_rows,
                                double *d0, double *d1, double *d2, double *e0, double *e1,
                                double *e2) {
  const int l = blockIdx.y;
  double *d = l == 0 ? d0 : (l == 1 ? d1 : d2);
  double *e = l == 0 ? e0 : (l == 1 ? e1 : e2);
  const double *a = coef + (long long)l * (n + 1);
  const double h = 1.0 / (n + 1);
  const double ih2 = 1.0 / (h * h);
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    double di = (a[i] + a[i + 1]) * ih2;
    if (paper_end_rows && i == 0) di = 2.0 * a[1] * ih2;
    if (paper_end_rows && i == n - 1) di = 2.0 * a[n - 1] * ih2;
    d[i] = di;
    if (i < n - 1) e[i] = -a[i + 1] * ih2;
  }
}

// Gershgorin interval and pivmin per mode (one block per mode).
__global__ void gersh_kernel(int n, const double *d0, const double *d1, const double *d2,
                             const double *e0, const double *e1, const double *e2,
                             double *bounds) {
  const int l = blockIdx.x;
  const double *d = l == 0 ? d0 : (l == 1 ? d1 : d2);
  const double *e = l == 0 ? e0 : (l == 1 ? e1 : e2);
  double lo = 1e300, hi = -1e300, emax = 0.0;
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    const double r = (i > 0 ? fabs(e[i - 1]) : 0.0) + (i < n - 1 ? fabs(e[i]) : 0.0);
    lo = fmin(lo, d[i] - r);
    hi = fmax(hi, d[i] + r);
    if (i < n - 1) emax = fmax(emax, e[i] * e[i]);
  }
  __shared__ double s_lo[256], s_hi[256], s_e[256];
  s_lo[threadIdx.x] = lo;
  s_hi[threadIdx.x] = hi;
  s_e[threadIdx.x] = emax;
  __syncthreads();
  for (int o = blockDim.x / 2; o > 0; o >>= 1) {
    if (threadIdx.x < o) {
      s_lo[threadIdx.x] = fmin(s_lo[threadIdx.x], s_lo[threadIdx.x + o]);
      s_hi[threadIdx.x] = fmax(s_hi[threadIdx.x], s_hi[threadIdx.x + o]);
      s_e[threadIdx.x] = fmax(s_e[threadIdx.x], s_e[threadIdx.x + o]);
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    const double span = s_hi[0] - s_lo[0];
    bounds[4 * l + 0] = s_lo[0] - 2.0 * DBL_EPSILON * span - DBL_MIN;
    bounds[4 * l + 1] = s_hi[0] + 2.0 * DBL_EPSILON * span + DBL_MIN;
    bounds[4 * l + 2] = DBL_MIN * fmax(1.0, s_e[0]);
  }
}

// number of eigenvalues of T strictly below x
__device__ __forceinline__ int sturm_count(int n, const double *__restrict__ d,
                                           const double *__restrict__ e, double x, double pivmin) {
  int cnt = 0;
  double q = d[0] - x;
  if (fabs(q) < pivmin) q = -pivmin;
  cnt += (q < 0.0);
  for (int i = 1; i < n; ++i) {
    q = (d[i] - x) - e[i - 1] * e[i - 1] / q;
    if (fabs(q) < pivmin) q = -pivmin;
    cnt += (q < 0.0);
  }
  return cnt;
}

// Bisection brackets: with T = D^T diag(a) D / h^2 (a at the n + 1 half points;
// the boundary ones recovered from the end rows of T), the Courant-Fischer
// theorem gives a_min mu_k <= lambda_k <= a_max mu_k, mu_k = 4/h^2 sin^2(k pi h / 2)
// the eigenvalues for a = 1. The bracket [0.99 a_min mu_k, 1.01 a_max mu_k] is
// checked by two inertia counts and replaced by the Gershgorin interval if it
// fails (or if a recovered coefficient is not positive); it saves the ~20
// halvings that separate a small eigenvalue from the width of the spectrum.
__global__ void bisect_kernel(int n, const double *d0, const double *d1, const double *d2,
                              const double *e0, const double *e1, const double *e2,
                              const double *bounds, double *l0, double *l1, double *l2) {
  const int l = blockIdx.y;
  const double *d = l == 0 ? d0 : (l == 1 ? d1 : d2);
  const double *e = l == 0 ? e0 : (l == 1 ? e1 : e2);
  double *lam = l == 0 ? l0 : (l == 1 ? l1 : l2);
  const double glo = bounds[4 * l], ghi = bounds[4 * l + 1], pivmin = bounds[4 * l + 2];
  const double h = 1.0 / (n + 1), h2 = h * h;
  __shared__ double s_min[64], s_max[64];
  double amin = 1e300, amax = -1e300;
  for (int i = threadIdx.x; i <= n; i += blockDim.x) {
    double ai;
    if (i == 0) ai = d[0] * h2 + (n > 1 ? e[0] * h2 : 0.0);
    else if (i == n) ai = d[n - 1] * h2 + (n > 1 ? e[n - 2] * h2 : 0.0);
    else ai = -e[i - 1] * h2;
    amin = fmin(amin, ai);
    amax = fmax(amax, ai);
  }
  s_min[threadIdx.x] = amin;
  s_max[threadIdx.x] = amax;
  __syncthreads();
  for (int o = blockDim.x / 2; o > 0; o >>= 1) {
    if (threadIdx.x < o) {
      s_min[threadIdx.x] = fmin(s_min[threadIdx.x], s_min[threadIdx.x + o]);
      s_max[threadIdx.x] = fmax(s_max[threadIdx.x], s_max[threadIdx.x + o]);
    }
    __syncthreads();
  }
  amin = s_min[0];
  amax = s_max[0];
  for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < n; k += gridDim.x * blockDim.x) {
    double lo = glo, hi = ghi;
    if (amin > 0.0 && n > 1) {
      const double sn = sin(0.5 * M_PI * h * (k + 1));
      const double mu = 4.0 * sn * sn / h2;
      const double blo = fmax(glo, 0.99 * amin * mu), bhi = fmin(ghi, 1.01 * amax * mu);
      if (blo < bhi && sturm_count(n, d, e, blo, pivmin) <= k && sturm_count(n, d, e, bhi, pivmin) > k) {
        lo = blo;
        hi = bhi;
      }
    }
    // invariant: count(lo) <= k < count(hi)
    for (int it = 0; it < 200; ++it) {
      const double mid = 0.5 * (lo + hi);
      if (mid <= lo || mid >= hi) break;
      if (hi - lo <= 2.0 * DBL_EPSILON * fmax(fabs(lo), fabs(hi)) + 4.0 * pivmin) break;
      if (sturm_count(n, d, e, mid, pivmin) > k) hi = mid; else lo = mid;
    }
    lam[k] = 0.5 * (lo + hi);
  }
}

// One thread per eigenvector. Scratch: Dp (n x n) holds D+ then nothing,
// Um (n x n) holds the backward multipliers; V's column first holds the
// forward multipliers, then the eigenvector.
__global__ void twisted_kernel(int n, const double *d0, const double *d1, const double *d2,
                               const double *e0, const double *e1, const double *e2,
                               const double *bounds, const double *l0, const double *l1,
                               const double *l2, double *V0, double *V1, double *V2, double *Dp,
                               double *Um) {
  const int l = blockIdx.y;
  const double *d = l == 0 ? d0 : (l == 1 ? d1 : d2);
  const double *e = l == 0 ? e0 : (l == 1 ? e1 : e2);
  const double *lam = l == 0 ? l0 : (l == 1 ? l1 : l2);
  double *V = l == 0 ? V0 : (l == 1 ? V1 : V2);
  const double pivmin = bounds[4 * l + 2];
  double *DpL = Dp + (long long)l * n * n;
  double *UmL = Um + (long long)l * n * n;
  for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < n; k += gridDim.x * blockDim.x) {
    const double lk = lam[k];
    double *z = V + (long long)k * n;
    double *dp = DpL + (long long)k * n;
    double *um = UmL + (long long)k * n;
    // forward: D+_0 = c_0; L_i = b_i / D+_i; D+_{i+1} = c_{i+1} - L_i b_i
    double dplus = d[0] - lk;
    if (fabs(dplus) < pivmin) dplus = pivmin;
    dp[0] = dplus;
    for (int i = 0; i < n - 1; ++i) {
      const double Li = e[i] / dplus;
      z[i] = Li;
      dplus = (d[i + 1] - lk) - Li * e[i];
      if (fabs(dplus) < pivmin) dplus = pivmin;
      dp[i + 1] = dplus;
    }
    // backward: D-_{n-1} = c_{n-1}; U_i = b_i / D-_{i+1}; D-_i = c_i - U_i b_i
    double dminus = d[n - 1] - lk;
    if (fabs(dminus) < pivmin) dminus = pivmin;
    int r = n - 1;
    double gbest = fabs(dp[n - 1]);  // gamma_{n-1} = D+_{n-1}
    for (int i = n - 2; i >= 0; --i) {
      const double Ui = e[i] / dminus;
      um[i] = Ui;
      const double ci = d[i] - lk;
      dminus = ci - Ui * e[i];
      if (fabs(dminus) < pivmin) dminus = pivmin;
      const double gam = dp[i] + dminus - ci;
      if (fabs(gam) < gbest) { gbest = fabs(gam); r = i; }
    }
    // solve: z_r = 1, z_i = -L_i z_{i+1} (i < r), z_{i+1} = -U_i z_i (i >= r)
    double zi = 1.0;
    double nrm2 = 1.0;
    for (int i = r - 1; i >= 0; --i) {
      zi = -z[i] * zi;
      z[i] = zi;
      nrm2 = fma(zi, zi, nrm2);
    }
    z[r] = 1.0;
    zi = 1.0;
    for (int i = r; i < n - 1; ++i) {
      zi = -um[i] * zi;
      z[i + 1] = zi;
      nrm2 = fma(zi, zi, nrm2);
    }
    double dot = 0.0;
    for (int i = 0; i < n; ++i) {
      const double x = (double)(i + 1) * 0.6180339887498949;
      dot = fma(z[i], 2.0 * (x - floor(x)) - 1.0, dot);
    }
    const double s = (dot < 0.0 ? -1.0 : 1.0) / sqrt(nrm2);
    for (int i = 0; i < n; ++i) z[i] *= s;
  }
}

// ------------------------------------------------------------------ set-up eigensolver
// The set-up path spends its FP64 work (GB300: 2 FP64 FMA per clock per SM)
// on few inertia counts: per eigenvalue,
//   1. an FP32 Sturm trisection inside the Courant-Fischer bracket (the two
//      lanes of the eigenpair count at the two inner points) gives a guess
//      (the FP32 pipe is ~64x the FP64 one; its counts are only a guess);
//   2. Rayleigh-quotient iteration on twisted factorizations in FP64: the
//      factorization of T - sigma I with twist r gives (T - sigma I) z = gamma_r e_r
//      (z_r = 1), so z^T (T - sigma I) z / z^T z = gamma_r / ||z||^2 and
//      sigma + gamma_r / ||z||^2 is the Rayleigh quotient of z (cubic
//      convergence); the inertia of the same factorization (signs of D+)
//      shrinks a safeguarding bracket, and a step leaving it is a bisection;
//   3. two FP64 inertia counts at lambda -+ tau (one per lane) confirm the index k; if they
//      do not (or the iteration does not settle), the eigenvalue is bisected
//      in FP64 from the Courant-Fischer bracket as before.
// The eigenvector is the normalised z of the last factorization.

#ifndef TCTL_EIG_BLOCK
#define TCTL_EIG_BLOCK 32
#endif
constexpr int kEigBlock = TCTL_EIG_BLOCK;  // threads per block (two per eigenpair), a power of two <= 64

// FP32 copies of d and e^2 (the guess phase), e^2 in FP64, the Weyl sign weights.
__global__ void eig_prep_kernel(int n, const double *d0, const double *d1, const double *d2,
                                const double *e0, const double *e1, const double *e2,
                                float *__restrict__ d32, float *__restrict__ ee32,
                                double *__restrict__ ee, double *__restrict__ g) {
  const int l = blockIdx.y;
  const double *d = l == 0 ? d0 : (l == 1 ? d1 : d2);
  const double *e = l == 0 ? e0 : (l == 1 ? e1 : e2);
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    d32[(size_t)l * n + i] = (float)d[i];
    const double q = i < n - 1 ? e[i] * e[i] : 0.0;
    ee[(size_t)l * n + i] = q;
    ee32[(size_t)l * n + i] = (float)q;
    if (l == 0) {
      const double x = (double)(i + 1) * 0.6180339887498949;
      g[i] = 2.0 * (x - floor(x)) - 1.0;
    }
  }
}

// On this part a warp scheduler issues one FP64 instruction per 64 cycles
// (FP64 compares included), so the recurrences below keep the FP64 pipe for
// their arithmetic: magnitude and sign tests are taken on the bit patterns
// (a non-negative double orders as its 64-bit pattern), exactly as the FP64
// compares would decide them.
__device__ __forceinline__ long long mag_bits(double x) {
  return __double_as_longlong(x) & 0x7fffffffffffffffll;
}
__device__ __forceinline__ bool neg_bit(double x) { return __double_as_longlong(x) < 0; }

// FP64 reciprocal: the hardware approximation (relative error below 2^-20)
// refined by one third-order step r <- r (1 + e + e^2), e = 1 - q r (error
// about e^3, below rounding). The inertia counts need a quotient with a
// relative error of a few units in the last place, not a correctly rounded one
// (Kahan's backward-error argument for Sturm counts holds for any operation
// with a small relative error). |q| >= pivmin > 0 is never subnormal here.
__device__ __forceinline__ double rcp_nr(double q) {
  double r;
  asm("rcp.approx.ftz.f64 %0, %1;" : "=d"(r) : "d"(q));
  const double t = fma(-q, r, 1.0);
  return fma(r, fma(t, t, t), r);
}

// number of eigenvalues below x, FP64 (ee = e^2); |q| < pivmin is replaced by
// -pivmin, so q is never -0 and its sign bit is the test q < 0
__device__ int count64(int n, const double *__restrict__ d, const double *__restrict__ ee, double x,
                       double pivmin) {
  const long long pm = mag_bits(pivmin);
  double q = d[0] - x;
  if (mag_bits(q) < pm) q = -pivmin;
  int cnt = neg_bit(q);
  for (int i = 1; i < n; ++i) {
    q = fma(-ee[i - 1], rcp_nr(q), d[i] - x);
    if (mag_bits(q) < pm) q = -pivmin;
    cnt += neg_bit(q);
  }
  return cnt;
}

// the same in FP32: a guess only, never trusted for the index
__device__ int count32(int n, const float *__restrict__ d, const float *__restrict__ ee, float x,
                       float pivmin) {
  float q = d[0] - x;
  if (fabsf(q) < pivmin) q = -pivmin;
  int cnt = q < 0.0f;
  for (int i = 1; i < n; ++i) {
    q = (d[i] - x) - __fdividef(ee[i - 1], q);
    if (fabsf(q) < pivmin) q = -pivmin;
    cnt += q < 0.0f;
  }
  return cnt;
}

struct Twist {
  int cnt;      // eigenvalues below sigma (negative D+ pivots)
  int r;        // twist index
  double gam;   // gamma_r
  double nrm2;  // ||z||^2 with z_r = 1
};

// The two lanes (2j, 2j + 1 of a warp) of one eigenpair run the same
// instructions on mirrored data: side 0 the forward recurrence of the twisted
// factorization over i = 0, 1, ..., side 1 the backward one over
// i = n - 1, n - 2, ... (the backward recurrence is the forward one of the
// reversed tridiagonal), so the warp does not diverge; values cross between the
// two lanes by shuffles. Each warp instruction of the FP64 pipe costs tens of
// cycles on this part, so the chain of one eigenpair, not the total work, sets
// the time: two lanes halve the sweeps' part of it.
struct Pair {
  unsigned mask;  // the pair's two lanes
  int side;       // 0: forward, 1: backward
};

__device__ __forceinline__ double xchg(const Pair &p, double v) { return __shfl_xor_sync(p.mask, v, 1); }
__device__ __forceinline__ int xchg(const Pair &p, int v) { return __shfl_xor_sync(p.mask, v, 1); }
__device__ __forceinline__ long long xchg(const Pair &p, long long v) {
  return __shfl_xor_sync(p.mask, v, 1);
}

// |q| < pivmin is replaced by pivmin (so a pivot is never -0: its sign bit is the test q < 0)
__device__ __forceinline__ double piv(double q, double pivmin) {
  return mag_bits(q) < mag_bits(pivmin) ? pivmin : q;
}

// Twisted factorization of T - sigma I by the pair: side 0 the forward
// multipliers L_i = e_i / D+_i (to L[i ld]) and the inertia count, side 1 the
// backward ones U_i = e_i / D-_{i+1} (to U[i ld]); then each side scans half of
// the twist candidates gamma_i = D+_i + D-_i - (d_i - sigma) (gamma_{n-1} =
// D+_{n-1}; both pivots re-formed from the stored multipliers by the sweeps'
// own operations; the smallest |gamma| wins, ties to the larger index) and sums
// ||z||^2 over its part of z (z_r = 1, z_i = -L_i z_{i+1} for i < r, z_{i+1} =
// -U_i z_i for i >= r). Both lanes return the same Twist.
__device__ Twist twisted_pair(const Pair &pr, int n, const double *__restrict__ d,
                              const double *__restrict__ e, double sigma, double pivmin,
                              double *__restrict__ L, double *__restrict__ U, int ld) {
  const int s = pr.side;
  double *Mo = s ? U : L;
  double p = piv(d[s ? n - 1 : 0] - sigma, pivmin);
  int cnt = neg_bit(p);
  for (int t = 0; t < n - 1; ++t) {
    const int ie = s ? n - 2 - t : t;
    const int id = s ? n - 2 - t : t + 1;
    const double m = e[ie] * rcp_nr(p);
    Mo[(size_t)ie * ld] = m;
    p = piv(fma(-m, e[ie], d[id] - sigma), pivmin);
    cnt += neg_bit(p);
  }
  __syncwarp(pr.mask);  // each lane reads the other's multipliers below
  Twist t;
  const int ocnt = xchg(pr, cnt);
  t.cnt = s ? ocnt : cnt;              // side 0's inertia count
  const double op = xchg(pr, p);
  const double dplus_last = s ? op : p;  // D+_{n-1}
  // candidates: side 0 takes i in [0, h), side 1 [h, n)
  const int h = n / 2;
  const int i0 = s ? h : 0, i1 = s ? n : h;
  // |gamma| compared on the bit patterns (exactly as fabs(gam) <= best)
  long long best = __double_as_longlong(1e308);
  double bgam = 0.0;
  int br = -1;
#pragma unroll 4
  for (int i = i0; i < i1; ++i) {
    const double ci = d[i] - sigma;
    double gam;
    if (i == n - 1) {
      gam = dplus_last;
    } else {
      const double dp = i == 0 ? piv(ci, pivmin) : piv(fma(-L[(size_t)(i - 1) * ld], e[i - 1], ci), pivmin);
      const double dm = piv(fma(-U[(size_t)i * ld], e[i], ci), pivmin);
      gam = dp + dm - ci;
    }
    if (mag_bits(gam) <= best) {
      best = mag_bits(gam);
      bgam = gam;
      br = i;
    }
  }
  {
    const long long ob = xchg(pr, best);
    const double og = xchg(pr, bgam);
    const int orr = xchg(pr, br);
    const long long b0 = s ? ob : best, b1 = s ? best : ob;
    const double g0 = s ? og : bgam, g1 = s ? bgam : og;
    const int r0 = s ? orr : br, r1 = s ? br : orr;
    if (r1 >= 0 && (r0 < 0 || b1 <= b0)) {
      t.r = r1;
      t.gam = g1;
    } else {
      t.r = r0;
      t.gam = g0;
    }
    if (t.r < 0) {  // no finite candidate: the last index, as an unscanned factorization would give
      t.r = n - 1;
      t.gam = dplus_last;
    }
  }
  // ||z||^2
  const int len = s ? n - 1 - t.r : t.r;
  double z = 1.0, acc = 0.0;
#pragma unroll 4
  for (int q = 0; q < len; ++q) {
    const int i = s ? t.r + q : t.r - 1 - q;
    z = -Mo[(size_t)i * ld] * z;
    acc = fma(z, z, acc);
  }
  const double other = xchg(pr, acc);
  const double left = s ? other : acc, right = s ? acc : other;
  t.nrm2 = (1.0 + left) + right;
  return t;
}

__global__ void eig_rqi_kernel(int n, const double *d0, const double *d1, const double *d2,
                               const double *e0, const double *e1, const double *e2,
                               const double *__restrict__ ee_all, const float *__restrict__ d32_all,
                               const float *__restrict__ ee32_all, const double *__restrict__ g,
                               const double *bounds, double *l0, double *l1, double *l2,
                               double *V0, double *V1, double *V2, double *Lscr, double *Uscr,
                               int *fallbacks) {
  const int l = blockIdx.y;
  const double *d = l == 0 ? d0 : (l == 1 ? d1 : d2);
  const double *e = l == 0 ? e0 : (l == 1 ? e1 : e2);
  const double *ee = ee_all + (size_t)l * n;
  const float *d32 = d32_all + (size_t)l * n, *ee32 = ee32_all + (size_t)l * n;
  double *lam = l == 0 ? l0 : (l == 1 ? l1 : l2);
  double *V = l == 0 ? V0 : (l == 1 ? V1 : V2);
  const double glo = bounds[4 * l], ghi = bounds[4 * l + 1], pivmin = bounds[4 * l + 2];
  const double gnorm = fmax(fabs(glo), fabs(ghi));
  const float pivmin32 = FLT_MIN * fmaxf(1.0f, (float)(pivmin / DBL_MIN));
  const double h = 1.0 / (n + 1), h2 = h * h;
  // coefficient range at the n + 1 half points (Courant-Fischer brackets)
  __shared__ double s_min[64], s_max[64];
  double amin = 1e300, amax = -1e300;
  for (int i = threadIdx.x; i <= n; i += blockDim.x) {
    double ai;
    if (i == 0) ai = d[0] * h2 + e[0] * h2;
    else if (i == n) ai = d[n - 1] * h2 + e[n - 2] * h2;
    else ai = -e[i - 1] * h2;
    amin = fmin(amin, ai);
    amax = fmax(amax, ai);
  }
  s_min[threadIdx.x] = amin;
  s_max[threadIdx.x] = amax;
  __syncthreads();
  for (int o = blockDim.x / 2; o > 0; o >>= 1) {
    if (threadIdx.x < o) {
      s_min[threadIdx.x] = fmin(s_min[threadIdx.x], s_min[threadIdx.x + o]);
      s_max[threadIdx.x] = fmax(s_max[threadIdx.x], s_max[threadIdx.x + o]);
    }
    __syncthreads();
  }
  amin = s_min[0];
  amax = s_max[0];
  // two lanes per eigenpair (see Pair); a pair's lanes return together
  const int gt = blockIdx.x * blockDim.x + threadIdx.x;
  const int k = gt >> 1;
  if (k >= n) return;
  const Pair pr{3u << (threadIdx.x & 30), (int)(threadIdx.x & 1)};
  const int side = pr.side;
  double blo = glo, bhi = ghi;
  if (amin > 0.0) {
    const double sn = sin(0.5 * M_PI * h * (k + 1));
    const double mu = 4.0 * sn * sn / h2;
    const double a = fmax(glo, 0.99 * amin * mu), b = fmin(ghi, 1.01 * amax * mu);
    if (a < b) {
      blo = a;
      bhi = b;
    }
  }
  double *Lk = Lscr + (size_t)l * n * n + k;
  double *Uk = Uscr + (size_t)l * n * n + k;
  // 1. FP32 guess by trisection: the two lanes count at the two inner points
  float flo = (float)blo, fhi = (float)bhi;
  for (int it = 0; it < 64; ++it) {
    if (fhi - flo <= 4.0f * FLT_EPSILON * fmaxf(fabsf(flo), fabsf(fhi))) break;
    const float w = fhi - flo;
    const float m1 = flo + w * (1.0f / 3.0f), m2 = flo + w * (2.0f / 3.0f);
    if (!(m1 > flo && m2 > m1 && m2 < fhi)) break;
    const int cmine = count32(n, d32, ee32, side ? m2 : m1, pivmin32);
    const int cother = xchg(pr, cmine);
    const int c1 = side ? cother : cmine, c2 = side ? cmine : cother;
    if (c1 > k) fhi = m1;
    else if (c2 > k) {
      flo = m1;
      fhi = m2;
    } else {
      flo = m2;
    }
  }
  // 2. Rayleigh-quotient iteration, safeguarded by [lo, hi] (shrunk by every inertia)
  double lo = blo, hi = bhi;
  double sigma = fmin(fmax(0.5 * ((double)flo + (double)fhi), blo), bhi);
  double lamk = 0.0;
  Twist t{};
  bool ok = false;
  for (int it = 0; it < 10; ++it) {
    t = twisted_pair(pr, n, d, e, sigma, pivmin, Lk, Uk, n);
    if (t.cnt <= k) lo = fmax(lo, sigma); else hi = fmin(hi, sigma);
    const double delta = t.gam / t.nrm2;
    if (fabs(delta) <= 2.0 * DBL_EPSILON * fabs(sigma) + 8.0 * DBL_EPSILON * gnorm) {
      lamk = sigma + delta;
      ok = true;
      break;
    }
    double sn = sigma + delta;
    if (!(sn > lo && sn < hi)) sn = 0.5 * (lo + hi);
    sigma = sn;
  }
  // 3. the index: exactly k eigenvalues below lambda - tau, k + 1 below lambda + tau
  //    (one count per lane)
  if (ok) {
    const double tau = 64.0 * DBL_EPSILON * gnorm + 4.0 * DBL_EPSILON * fabs(lamk);
    const int cm = count64(n, d, ee, side ? lamk + tau : lamk - tau, pivmin);
    const int co = xchg(pr, cm);
    const int cminus = side ? co : cm, cplus = side ? cm : co;
    ok = cminus <= k && cplus > k;
  }
  if (!ok) {
    // FP64 bisection from the Courant-Fischer bracket (Gershgorin if it fails);
    // both lanes take the same steps (a rare path)
    lo = blo;
    hi = bhi;
    if (!(count64(n, d, ee, lo, pivmin) <= k && count64(n, d, ee, hi, pivmin) > k)) {
      lo = glo;
      hi = ghi;
    }
    for (int it = 0; it < 200; ++it) {
      const double mid = 0.5 * (lo + hi);
      if (mid <= lo || mid >= hi) break;
      if (hi - lo <= 2.0 * DBL_EPSILON * fmax(fabs(lo), fabs(hi)) + 4.0 * pivmin) break;
      if (count64(n, d, ee, mid, pivmin) > k) hi = mid; else lo = mid;
    }
    lamk = 0.5 * (lo + hi);
    t = twisted_pair(pr, n, d, e, lamk, pivmin, Lk, Uk, n);
    if (side == 0) atomicAdd(fallbacks, 1);
  }
  if (side == 0) lam[k] = lamk;
  // eigenvector: z of the last factorization, unit norm, sum_i z_i g_i > 0;
  // side 0 forms z_i for i <= r (from L), side 1 for i > r (from U)
  const int len = side ? n - 1 - t.r : t.r;
  const double *Mk = side ? Uk : Lk;
  double dot = side ? 0.0 : g[t.r], zi = 1.0;
  for (int q = 0; q < len; ++q) {
    const int i = side ? t.r + q : t.r - 1 - q;
    zi = -Mk[(size_t)i * n] * zi;
    dot = fma(zi, g[side ? i + 1 : i], dot);
  }
  const double odot = xchg(pr, dot);
  const double tot = side ? odot + dot : dot + odot;
  const double sc = (tot < 0.0 ? -1.0 : 1.0) / sqrt(t.nrm2);
  double *z = V + (size_t)k * n;
  if (side == 0) z[t.r] = sc;
  zi = 1.0;
  for (int q = 0; q < len; ++q) {
    const int i = side ? t.r + q : t.r - 1 - q;
    zi = -Mk[(size_t)i * n] * zi;
    z[side ? i + 1 : i] = zi * sc;
  }
}

// Set-up eigenpairs: A_(l) assembled, all 3n eigenpairs by eig_rqi_kernel, the
// eigenvalues read back (s_min, s_max of the spectral sums).
void setup_eigs(Ctx &c) {
  const int n = c.n;
  for (int l = 0; l < 3; ++l) {
    c.d[l] = c.dmalloc(n);
    c.e[l] = c.dmalloc(std::max(n - 1, 1));
    c.lam[l] = c.dmalloc(n);
    c.V[l] = c.dmalloc((size_t)n * n);
  }
  dim3 ga((n + 255) / 256, 3);
  LAUNCH(c, assemble_kernel, ga, 256, 0, n, c.coef, c.o.paper_end_rows, c.d[0], c.d[1], c.d[2],
         c.e[0], c.e[1], c.e[2]);
  size_t mk = c.ws.mark();
  double *bounds = c.ws.dbl(12);
  LAUNCH(c, gersh_kernel, 3, 256, 0, n, c.d[0], c.d[1], c.d[2], c.e[0], c.e[1], c.e[2], bounds);
  double *ee = c.ws.dbl((size_t)3 * n), *g = c.ws.dbl(n);
  float *d32 = reinterpret_cast<float *>(c.ws.dbl(((size_t)3 * n + 1) / 2));
  float *ee32 = reinterpret_cast<float *>(c.ws.dbl(((size_t)3 * n + 1) / 2));
  int *fallbacks = c.ws.i32(1);
  TCTL_CUDA(cudaMemsetAsync(fallbacks, 0, sizeof(int), c.st));
  LAUNCH(c, eig_prep_kernel, ga, 256, 0, n, c.d[0], c.d[1], c.d[2], c.e[0], c.e[1], c.e[2], d32, ee32,
         ee, g);
  double *Lscr = c.ws.dbl((size_t)3 * n * n);
  double *Uscr = c.ws.dbl((size_t)3 * n * n);
  // kEigBlock / 2 eigenpairs per block (a warp or part of one) spread the 3n
  // eigenpairs over all SMs; each pair of lanes' time is its eigenpair's chain
  // of dependent FP64 recurrences
  dim3 geig((2 * n + kEigBlock - 1) / kEigBlock, 3);
  const auto tb0 = std::chrono::steady_clock::now();
  LAUNCH(c, eig_rqi_kernel, geig, kEigBlock, 0, n, c.d[0], c.d[1], c.d[2], c.e[0], c.e[1], c.e[2], ee, d32,
         ee32, g, bounds, c.lam[0], c.lam[1], c.lam[2], c.V[0], c.V[1], c.V[2], Lscr, Uscr,
         fallbacks);
  for (int l = 0; l < 3; ++l) {
    c.lam_host[l].resize(n);
    to_host(c, c.lam_host[l].data(), c.lam[l], n);
  }
  if (c.trace) {
    int nf = 0;
    read_host(c, &nf, fallbacks, sizeof(int));
    std::fprintf(stderr, "[tctl] eigenpairs %.1f ms (%d of %d by bisection)\n",
                 std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - tb0).count(),
                 nf, 3 * n);
  }
  c.ws.reset(mk);
  c.s_min = c.lam_host[0][0] + c.lam_host[1][0] + c.lam_host[2][0];
  c.s_max = c.lam_host[0][n - 1] + c.lam_host[1][n - 1] + c.lam_host[2][n - 1];
  if (!(c.s_min > 0.0) || !std::isfinite(c.s_max))
    fail(TCTL_E_NUMERIC, "eigensolver produced a non-positive or non-finite spectrum");
}

}  // namespace tctl

// ------------------------------------------------------------------ allocation-free entry point
// tctl_eig1d_noalloc runs the same assembly, bisection and twisted-factorization
// kernels as tctl_setup, but takes its scratch (tridiagonal entries, Gershgorin
// bounds, the per-eigenvector D+ and backward-multiplier arrays, an error flag)
// from the file-scope device array below instead of cudaMalloc. The array is
// sized for n <= TCTL_EIG_NOALLOC_MAX_N and is resident on every device that
// loads the library until the process exits.
namespace tctl {
namespace {

constexpr int kNoAllocMaxN = TCTL_EIG_NOALLOC_MAX_N;
constexpr size_t kNoAllocDoubles =
    (size_t)6 * kNoAllocMaxN * kNoAllocMaxN + (size_t)6 * kNoAllocMaxN + 16;

}  // namespace
}  // namespace tctl

static __device__ __align__(256) double g_eig_noalloc_scratch[tctl::kNoAllocDoubles];

namespace tctl {
namespace {

std::mutex g_noalloc_mu;
double *g_noalloc_ptr[256] = {};  // device address of the scratch, per device ordinal

__global__ void coeff_check_kernel(int count, const double *__restrict__ coef, int *flag) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < count; i += gridDim.x * blockDim.x) {
    const double v = coef[i];
    if (!(v > 0.0) || !isfinite(v)) atomicExch(flag, 1);
  }
}

}  // namespace
}  // namespace tctl

extern "C" int tctl_eig1d_noalloc(const double *coeffs, int n, int paper_end_rows, double *lam,
                                  double *V, void *cuda_stream) {
  using namespace tctl;
  if (!coeffs || !lam || !V) {
    set_noalloc_error("tctl_eig1d_noalloc: NULL pointer argument");
    return TCTL_E_ARG;
  }
  if (n < 2 || n > kNoAllocMaxN) {
    set_noalloc_error("tctl_eig1d_noalloc: n = " + std::to_string(n) +
                      " is outside [2, TCTL_EIG_NOALLOC_MAX_N = " + std::to_string(kNoAllocMaxN) +
                      "]; use tctl_setup for larger grids");
    return TCTL_E_ARG;
  }
  cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 256) {
    set_noalloc_error("tctl_eig1d_noalloc: cudaGetDevice failed");
    return TCTL_E_CUDA;
  }
  double *base = nullptr;
  {
    // one-time set-up per device: the host-side name of the array is not a
    // device address, so its address is looked up with the device current.
    std::lock_guard<std::mutex> lock(g_noalloc_mu);
    if (!g_noalloc_ptr[dev]) {
      void *p = nullptr;
      const cudaError_t e = cudaGetSymbolAddress(&p, g_eig_noalloc_scratch);
      if (e != cudaSuccess || !p) {
        set_noalloc_error(std::string("tctl_eig1d_noalloc: cudaGetSymbolAddress failed: ") +
                          cudaGetErrorString(e));
        return TCTL_E_CUDA;
      }
      g_noalloc_ptr[dev] = static_cast<double *>(p);
    }
    base = g_noalloc_ptr[dev];
  }
  const size_t nn = (size_t)n * n;
  double *d = base;                  // 3 n
  double *e = d + 3 * (size_t)n;     // 3 n (n-1 used per mode)
  double *bounds = e + 3 * (size_t)n;  // 12
  int *flag = reinterpret_cast<int *>(bounds + 12);  // 1 int (in a 4-double slot)
  double *Dp = bounds + 16;          // 3 n^2
  double *Um = Dp + 3 * nn;          // 3 n^2
  auto fail_cuda = [&](const char *what) {
    set_noalloc_error(std::string("tctl_eig1d_noalloc: ") + what + ": " +
                      cudaGetErrorString(cudaGetLastError()));
    return TCTL_E_CUDA;
  };
  // the coefficient flag must start at zero on every call
  if (cudaMemsetAsync(flag, 0, sizeof(int), st) != cudaSuccess) return fail_cuda("memset");
  coeff_check_kernel<<<(3 * (n + 1) + 255) / 256, 256, 0, st>>>(3 * (n + 1), coeffs, flag);
  int hflag = 0;
  if (cudaMemcpyAsync(&hflag, flag, sizeof(int), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
      cudaStreamSynchronize(st) != cudaSuccess)
    return fail_cuda("coefficient check");
  if (hflag) {
    set_noalloc_error("tctl_eig1d_noalloc: coefficient a_l(x) must be positive and finite");
    return TCTL_E_COEFF;
  }
  double *dm[3], *em[3], *lm[3], *Vm[3];
  for (int l = 0; l < 3; ++l) {
    dm[l] = d + (size_t)l * n;
    em[l] = e + (size_t)l * n;
    lm[l] = lam + (size_t)l * n;
    Vm[l] = V + (size_t)l * nn;
  }
  dim3 ga((n + 255) / 256, 3);
  assemble_kernel<<<ga, 256, 0, st>>>(n, coeffs, paper_end_rows, dm[0], dm[1], dm[2], em[0], em[1],
                                      em[2]);
  gersh_kernel<<<3, 256, 0, st>>>(n, dm[0], dm[1], dm[2], em[0], em[1], em[2], bounds);
  dim3 gb((n + 63) / 64, 3);
  bisect_kernel<<<gb, 64, 0, st>>>(n, dm[0], dm[1], dm[2], em[0], em[1], em[2], bounds, lm[0], lm[1],
                                   lm[2]);
  twisted_kernel<<<gb, 64, 0, st>>>(n, dm[0], dm[1], dm[2], em[0], em[1], em[2], bounds, lm[0],
                                    lm[1], lm[2], Vm[0], Vm[1], Vm[2], Dp, Um);
  if (cudaGetLastError() != cudaSuccess) return fail_cuda("kernel launch");
  return TCTL_OK;
}
