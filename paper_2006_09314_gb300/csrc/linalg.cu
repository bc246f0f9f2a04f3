// Dense FP64 building blocks: batched GEMM (mode products, Gram matrices,
// projections), Khatri-Rao columns, small symmetric eigensolver, orthonormal
// bases by pivoted Cholesky, and elementwise helpers.
//
// GB300 executes FP64 at a small fraction of its FP32 rate, so these kernels
// are arithmetic-bound: exact-work tiles (no FMA spent on padding), split-K for
// tall-skinny reductions (Gram matrices with K = n) so that every SM has work,
// and the small eigenproblems spread over thread-block clusters.
#include <algorithm>
#include <cstdio>
#include <cmath>
#include <cstring>
#include <mutex>
#include <string>
#include <vector>

#include "tctl_internal.cuh"

namespace tctl {

[[noreturn]] void fail(int code, const std::string &msg) { throw Error{code, msg}; }

void check_cuda(cudaError_t e, const char *what) {
  if (e != cudaSuccess) {
    fail(e == cudaErrorMemoryAllocation ? TCTL_E_NOMEM : TCTL_E_CUDA,
         std::string(what) + ": " + cudaGetErrorString(e));
  }
}

void *Arena::alloc(size_t bytes) {
  size_t off = (top + 255) & ~size_t(255);
  if (off + bytes > size) {
    fail(TCTL_E_NOMEM, "workspace arena exhausted (need " + std::to_string(off + bytes) +
                           " bytes of " + std::to_string(size) + ")");
  }
  top = off + bytes;
  peak = std::max(peak, top);
  return base + off;
}

double *Ctx::dmalloc(size_t count) {
  void *p = nullptr;
  check_cuda(cudaMallocAsync(&p, std::max<size_t>(count, 1) * sizeof(double), st), "cudaMallocAsync");
  owned.push_back(p);
  return static_cast<double *>(p);
}

cudaEvent_t Ctx::prof_event() {
  if (prof_used == prof_pool.size()) {
    cudaEvent_t e;
    check_cuda(cudaEventCreate(&e), "cudaEventCreate");
    prof_pool.push_back(e);
  }
  return prof_pool[prof_used++];
}

// ------------------------------------------------------------------ GEMM
constexpr int GEMM_BK = 16;
// CTAs a split-K FP64 GEMM aims at (the contracted dimension is split until the
// grid has about this many): two per SM fill the GPU for one solve alone; with
// many solves on concurrent streams fewer, longer CTAs spend less time in
// per-CTA prologues, partial-sum writes and reductions.
#ifndef TCTL_SPLIT_TARGET
#define TCTL_SPLIT_TARGET (2 * 152)
#endif
constexpr int kSplitTarget = TCTL_SPLIT_TARGET;

template <int BM, int BN, bool TA, bool TB>
__global__ void __launch_bounds__(256)
dgemm_kernel(int m, int n, int k, double alpha, const double *__restrict__ A, int lda,
             long long sA, int divA, const double *__restrict__ B, int ldb, long long sB,
             int divB, double beta, double *__restrict__ C, int ldc, long long sC, int splits,
             int kchunk, double *__restrict__ part) {
  constexpr int TM = BM / 16, TN = BN / 16;
  __shared__ double As[GEMM_BK][BM + 1];
  __shared__ double Bs[GEMM_BK][BN + 1];
  const int bz = blockIdx.z;
  const int b = bz / splits, split = bz % splits;
  A += (long long)(b / divA) * sA;
  B += (long long)(b / divB) * sB;
  const int k0 = split * kchunk;
  const int k1 = min(k, k0 + kchunk);
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  const int row0 = blockIdx.x * BM, col0 = blockIdx.y * BN;
  double acc[TM][TN];
#pragma unroll
  for (int i = 0; i < TM; ++i)
#pragma unroll
    for (int j = 0; j < TN; ++j) acc[i][j] = 0.0;

  for (int kb = k0; kb < k1; kb += GEMM_BK) {
    for (int e = threadIdx.x; e < BM * GEMM_BK; e += 256) {
      int i, kk;
      if (!TA) { i = e % BM; kk = e / BM; } else { kk = e % GEMM_BK; i = e / GEMM_BK; }
      const int gi = row0 + i, gk = kb + kk;
      double v = 0.0;
      if (gi < m && gk < k1) v = TA ? A[gk + (long long)gi * lda] : A[gi + (long long)gk * lda];
      As[kk][i] = v;
    }
    for (int e = threadIdx.x; e < BN * GEMM_BK; e += 256) {
      int j, kk;
      if (!TB) { kk = e % GEMM_BK; j = e / GEMM_BK; } else { j = e % BN; kk = e / BN; }
      const int gj = col0 + j, gk = kb + kk;
      double v = 0.0;
      if (gj < n && gk < k1) v = TB ? B[gj + (long long)gk * ldb] : B[gk + (long long)gj * ldb];
      Bs[kk][j] = v;
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < GEMM_BK; ++kk) {
      double a[TM], bb[TN];
#pragma unroll
      for (int i = 0; i < TM; ++i) a[i] = As[kk][ty + 16 * i];
#pragma unroll
      for (int j = 0; j < TN; ++j) bb[j] = Bs[kk][tx + 16 * j];
#pragma unroll
      for (int i = 0; i < TM; ++i)
#pragma unroll
        for (int j = 0; j < TN; ++j) acc[i][j] = fma(a[i], bb[j], acc[i][j]);
    }
    __syncthreads();
  }
  if (splits == 1) {
    double *Cb = C + (long long)b * sC;
#pragma unroll
    for (int i = 0; i < TM; ++i)
#pragma unroll
      for (int j = 0; j < TN; ++j) {
        const int gi = row0 + ty + 16 * i, gj = col0 + tx + 16 * j;
        if (gi < m && gj < n) {
          double *p = Cb + gi + (long long)gj * ldc;
          *p = (beta == 0.0) ? alpha * acc[i][j] : fma(alpha, acc[i][j], beta * *p);
        }
      }
  } else {
    double *P = part + (long long)bz * m * n;
#pragma unroll
    for (int i = 0; i < TM; ++i)
#pragma unroll
      for (int j = 0; j < TN; ++j) {
        const int gi = row0 + ty + 16 * i, gj = col0 + tx + 16 * j;
        if (gi < m && gj < n) P[gi + (long long)gj * m] = acc[i][j];
      }
  }
}

// C = alpha sum_q part_q + beta C. A block takes 32 consecutive outputs (x)
// and spreads the partial sums over 8 groups (y) that run concurrently, so a
// small output with many K-splits is not one long chain of loads per thread;
// the order of summation is fixed, so results are reproducible.
__global__ void __launch_bounds__(256) splitk_reduce(int m, int n, int splits, int batch, double alpha,
                                                     const double *__restrict__ part, double beta,
                                                     double *C, int ldc, long long sC) {
  __shared__ double red[8][33];
  const long long mn = (long long)m * n, total = mn * batch;
  const long long t = blockIdx.x * 32ll + threadIdx.x;
  double s = 0.0;
  int b = 0;
  long long r = 0;
  if (t < total) {
    b = (int)(t / mn);
    r = t - (long long)b * mn;
    const double *p = part + (long long)b * splits * mn + r;
#pragma unroll 4
    for (int q = threadIdx.y; q < splits; q += 8) s += p[q * mn];
  }
  red[threadIdx.y][threadIdx.x] = s;
  __syncthreads();
  if (threadIdx.y == 0 && t < total) {
    for (int g = 1; g < 8; ++g) s += red[g][threadIdx.x];
    const int i = (int)(r % m), j = (int)(r / m);
    double *out = C + (long long)b * sC + i + (long long)j * ldc;
    *out = (beta == 0.0) ? alpha * s : fma(alpha, s, beta * *out);
  }
}

// ------------------------------------------------------------------ skinny GEMM
// C = alpha op(A) op(B) + beta C with n <= 16 columns (basis changes of a few
// vectors, matrix-vector products): the 64 x 64 tile kernel would leave most
// of its FP64 lanes idle. op(B) tiles of SK_KT x NC sit in shared memory; the
// contracted dimension is split across blocks (partial sums, splitk_reduce).
constexpr int SK_KT = 128;

// op(A) = A, rows contiguous: one thread per row.
template <int NC, bool TB>
__global__ void __launch_bounds__(256) skinny_nn_kernel(int m, int n, int k, const double *__restrict__ A,
                                                        int lda, const double *__restrict__ B, int ldb,
                                                        int kchunk, double *__restrict__ part) {
  __shared__ double Bs[SK_KT][NC];
  const int i = blockIdx.x * 256 + threadIdx.x;
  const int q = blockIdx.y;
  const int k0 = q * kchunk, k1 = min(k, k0 + kchunk);
  double acc[NC];
#pragma unroll
  for (int j = 0; j < NC; ++j) acc[j] = 0.0;
  for (int kt = k0; kt < k1; kt += SK_KT) {
    const int kn = min(SK_KT, k1 - kt);
    __syncthreads();
    for (int t = threadIdx.x; t < SK_KT * NC; t += 256) {
      const int kk = t / NC, j = t % NC;
      Bs[kk][j] = (kk < kn && j < n)
                      ? (TB ? B[j + (long long)(kt + kk) * ldb] : B[(kt + kk) + (long long)j * ldb])
                      : 0.0;
    }
    __syncthreads();
    if (i < m) {
      for (int kk = 0; kk < kn; ++kk) {
        const double a = A[i + (long long)(kt + kk) * lda];
#pragma unroll
        for (int j = 0; j < NC; ++j) acc[j] = fma(a, Bs[kk][j], acc[j]);
      }
    }
  }
  if (i < m)
#pragma unroll
    for (int j = 0; j < NC; ++j)
      if (j < n) part[(long long)q * m * n + i + (long long)j * m] = acc[j];
}

// op(A) = A^T, each row of op(A) contiguous: one warp per row, lanes along k.
template <int NC, bool TB>
__global__ void __launch_bounds__(256) skinny_tn_kernel(int m, int n, int k, const double *__restrict__ A,
                                                        int lda, const double *__restrict__ B, int ldb,
                                                        int kchunk, double *__restrict__ part) {
  constexpr int RPW = NC >= 8 ? 2 : 4;  // rows per warp
  __shared__ double Bs[SK_KT][NC];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int q = blockIdx.y;
  const int k0 = q * kchunk, k1 = min(k, k0 + kchunk);
  double acc[RPW][NC];
#pragma unroll
  for (int rr = 0; rr < RPW; ++rr)
#pragma unroll
    for (int j = 0; j < NC; ++j) acc[rr][j] = 0.0;
  for (int kt = k0; kt < k1; kt += SK_KT) {
    const int kn = min(SK_KT, k1 - kt);
    __syncthreads();
    for (int t = threadIdx.x; t < SK_KT * NC; t += 256) {
      const int kk = t / NC, j = t % NC;
      Bs[kk][j] = (kk < kn && j < n)
                      ? (TB ? B[j + (long long)(kt + kk) * ldb] : B[(kt + kk) + (long long)j * ldb])
                      : 0.0;
    }
    __syncthreads();
#pragma unroll
    for (int rr = 0; rr < RPW; ++rr) {
      const int i = blockIdx.x * (8 * RPW) + warp + 8 * rr;
      if (i >= m) continue;
      const double *a = A + (long long)i * lda + kt;
      for (int kk = lane; kk < kn; kk += 32) {
        const double av = a[kk];
#pragma unroll
        for (int j = 0; j < NC; ++j) acc[rr][j] = fma(av, Bs[kk][j], acc[rr][j]);
      }
    }
  }
#pragma unroll
  for (int rr = 0; rr < RPW; ++rr) {
    const int i = blockIdx.x * (8 * RPW) + warp + 8 * rr;
#pragma unroll
    for (int j = 0; j < NC; ++j) {
      double v = acc[rr][j];
      for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
      if (lane == 0 && i < m && j < n) part[(long long)q * m * n + i + (long long)j * m] = v;
    }
  }
}

template <int NC>
static void skinny_launch(Ctx &c, bool ta, bool tb, int m, int n, int k, const double *A, int lda,
                          const double *B, int ldb, double *part, int splits, int kchunk, int rowblocks) {
  dim3 g(rowblocks, splits);
#define TCTL_SK(KER, TB_) LAUNCH(c, (KER<NC, TB_>), g, 256, 0, m, n, k, A, lda, B, ldb, kchunk, part)
  if (!ta) {
    if (tb) TCTL_SK(skinny_nn_kernel, true);
    else TCTL_SK(skinny_nn_kernel, false);
  } else {
    if (tb) TCTL_SK(skinny_tn_kernel, true);
    else TCTL_SK(skinny_tn_kernel, false);
  }
#undef TCTL_SK
}

static void gemm_skinny(Ctx &c, bool ta, bool tb, int m, int n, int k, double alpha, const double *A,
                        int lda, const double *B, int ldb, double beta, double *C, int ldc) {
  const int NC = n <= 1 ? 1 : n <= 4 ? 4 : n <= 8 ? 8 : 16;
  const int rows_per_block = ta ? 8 * (NC >= 8 ? 2 : 4) : 256;
  const int rowblocks = (m + rows_per_block - 1) / rows_per_block;
  int splits = std::max(1, std::min((kSplitTarget + rowblocks - 1) / rowblocks, (k + 63) / 64));
  splits = std::min(splits, 256);
  const int kchunk = (k + splits - 1) / splits;
  splits = (k + kchunk - 1) / kchunk;
  size_t mk = c.ws.mark();
  double *part = c.ws.dbl((size_t)m * n * splits);
  c.next_flops = 2.0 * m * (double)n * k;
  if (NC == 1) skinny_launch<1>(c, ta, tb, m, n, k, A, lda, B, ldb, part, splits, kchunk, rowblocks);
  else if (NC == 4) skinny_launch<4>(c, ta, tb, m, n, k, A, lda, B, ldb, part, splits, kchunk, rowblocks);
  else if (NC == 8) skinny_launch<8>(c, ta, tb, m, n, k, A, lda, B, ldb, part, splits, kchunk, rowblocks);
  else skinny_launch<16>(c, ta, tb, m, n, k, A, lda, B, ldb, part, splits, kchunk, rowblocks);
  const long long total = (long long)m * n;
  c.next_bytes = 8.0 * total * (splits + 1 + (beta != 0.0));
  LAUNCH(c, splitk_reduce, (unsigned)((total + 31) / 32), dim3(32, 8), 0, m, n, splits, 1, alpha, part,
         beta, C, ldc, 0ll);
  c.ws.reset(mk);
}

template <int BM, int BN>
static void gemm_launch(Ctx &c, bool ta, bool tb, dim3 grid, int m, int n, int k, double alpha,
                        const double *A, int lda, long long sA, int divA, const double *B,
                        int ldb, long long sB, int divB, double beta, double *C, int ldc,
                        long long sC, int splits, int kchunk, double *part) {
#define TCTL_G(TA_, TB_)                                                                   \
  LAUNCH(c, (dgemm_kernel<BM, BN, TA_, TB_>), grid, 256, 0, m, n, k, alpha, A, lda, sA,   \
         divA, B, ldb, sB, divB, beta, C, ldc, sC, splits, kchunk, part)
  if (!ta && !tb) TCTL_G(false, false);
  else if (!ta && tb) TCTL_G(false, true);
  else if (ta && !tb) TCTL_G(true, false);
  else TCTL_G(true, true);
#undef TCTL_G
}

void gemm(Ctx &c, bool ta, bool tb, int m, int n, int k, double alpha, const double *A, int lda,
          long long sA, const double *B, int ldb, long long sB, double beta, double *C, int ldc,
          long long sC, int batch, int divA, int divB) {
  if (m <= 0 || n <= 0 || batch <= 0) return;
  if (k <= 0) {
    // C = beta C (an empty contraction)
    if (beta != 1.0)
      for (int b = 0; b < batch; ++b)
        for (int j = 0; j < n; ++j) {
          double *col = C + b * sC + (long long)j * ldc;
          if (beta == 0.0) TCTL_CUDA(cudaMemsetAsync(col, 0, sizeof(double) * m, c.st));
          else axpby(c, (size_t)m, beta, col, 0.0, col);  // col = beta col
        }
    return;
  }
  if (batch == 1 && n <= 16 && m >= 64 && (long long)m * n * k >= (1 << 16)) {
    gemm_skinny(c, ta, tb, m, n, k, alpha, A, lda, B, ldb, beta, C, ldc);
    return;
  }
  if (batch == 1) {
    // one product: the exact-work kernel of the grouped GEMMs
    const GemmSpec g{ta, tb, m, n, k, alpha, A, lda, B, ldb, beta, C, ldc};
    gemm_group(c, 1, &g);
    return;
  }
  const bool small = (m <= 32 && n <= 32);
  const int BM = small ? 32 : 64, BN = small ? 32 : 64;
  const int gx = (m + BM - 1) / BM, gy = (n + BN - 1) / BN;
  const long long tiles = (long long)gx * gy * batch;
  int splits = 1;
  const int target = kSplitTarget;
  if (tiles < target && k >= 4 * GEMM_BK) {
    // tall-skinny products (Gram matrices, projections with K = n): split K so that
    // about two CTAs per SM run; chunks down to one 16-deep tile.
    splits = (int)std::min<long long>((target + tiles - 1) / tiles, (k + GEMM_BK - 1) / GEMM_BK);
    const long long cap = std::max<long long>(1, (16ll << 20) / ((long long)m * n * batch));
    splits = (int)std::max<long long>(1, std::min<long long>({(long long)splits, 256ll, cap}));
  }
  int kchunk = (k + splits - 1) / splits;
  kchunk = ((kchunk + GEMM_BK - 1) / GEMM_BK) * GEMM_BK;
  splits = (k + kchunk - 1) / kchunk;
  if (gy > 65535 || (long long)batch * splits > 65535) {
    // split the batch to respect grid limits
    if ((long long)batch * splits > 65535 && batch > 1) {
      const int q = std::max(divA, divB) % std::min(divA, divB) == 0
                        ? std::max(divA, divB)
                        : divA * divB;  // batch chunks must keep whole divisor groups
      int chunk = std::max(1, 65535 / splits);
      chunk = std::max(q, chunk - chunk % q);
      for (int b0 = 0; b0 < batch; b0 += chunk) {
        const int nb = std::min(chunk, batch - b0);
        // divisors: only valid if b0 is a multiple of the divisors
        gemm(c, ta, tb, m, n, k, alpha, A + (long long)(b0 / divA) * sA, lda, sA,
             B + (long long)(b0 / divB) * sB, ldb, sB, beta, C + (long long)b0 * sC, ldc, sC, nb,
             divA, divB);
      }
      return;
    }
    if (gy > 65535) {
      const int ncol = 65535 * BN;
      for (int j0 = 0; j0 < n; j0 += ncol) {
        const int nn = std::min(ncol, n - j0);
        gemm(c, ta, tb, m, nn, k, alpha, A, lda, sA,
             tb ? B + j0 : B + (long long)j0 * ldb, ldb, sB, beta, C + (long long)j0 * ldc, ldc,
             sC, batch, divA, divB);
      }
      return;
    }
  }
  double *part = nullptr;
  size_t mk = c.ws.mark();
  if (splits > 1) part = c.ws.dbl((size_t)m * n * batch * splits);
  dim3 grid(gx, gy, batch * splits);
  if (c.prof && c.trace) {
    // per-shape profile names (TCTL_TRACE=1 with profiling on)
    char nm[96];
    std::snprintf(nm, sizeof(nm), "dgemm[%s%s %dx%dx%d b%d s%d]", ta ? "T" : "N", tb ? "T" : "N", m, n,
                  k, batch, splits);
    c.next_tag = c.intern(nm);
  }
  c.next_flops = 2.0 * m * n * (double)k * batch;
  c.next_bytes = 8.0 * ((double)m * k * ((batch - 1) / divA + 1) + (double)k * n * ((batch - 1) / divB + 1) +
                        (double)m * n * batch * (1 + (beta != 0.0)));
  if (small)
    gemm_launch<32, 32>(c, ta, tb, grid, m, n, k, alpha, A, lda, sA, divA, B, ldb, sB, divB, beta,
                        C, ldc, sC, splits, kchunk, part);
  else
    gemm_launch<64, 64>(c, ta, tb, grid, m, n, k, alpha, A, lda, sA, divA, B, ldb, sB, divB, beta,
                        C, ldc, sC, splits, kchunk, part);
  if (splits > 1) {
    const long long total = (long long)m * n * batch;
    c.next_bytes = 8.0 * total * (splits + 1 + (beta != 0.0));
    LAUNCH(c, splitk_reduce, (unsigned)((total + 31) / 32), dim3(32, 8), 0, m, n, splits, batch, alpha,
           part, beta, C, ldc, sC);
  }
  c.ws.reset(mk);
}

// ------------------------------------------------------------------ grouped GEMM
// Up to kGroupMax independent GEMMs of the same transposition in one launch
// (the three modes' Gram matrices and projections of a Tucker step): each
// item keeps its own shape, pointers and K-split; the launch's CTAs are dealt
// out to the items in order (item i owns CTAs [cta0_i, cta0_{i+1})), and one
// grouped reduction adds the split-K partial sums of all items. Every single
// (unbatched) FP64 product of the library goes through it as a one-item group.
constexpr int kGroupMax = 8;

struct GItem {
  const double *A, *B;
  double *C, *part;
  double alpha, beta;
  int m, n, k, lda, ldb, ldc, splits, kchunk, gx, cta0;
  long long out0;  // first output of this item in the grouped reduction
};

struct GArgs {
  int count;
  GItem it[kGroupMax];
};

// Grouped FP64 GEMMs with exact work. An item's output is cut into tiles of
// at most GT x GT; in a tile of P = mt nt outputs thread t takes output t % P
// and, for P < 256, the k-lane t / P of S = 256 / P lanes that split the CTA's
// k range (summed in a fixed order at the end). Every FMA is one of the
// product's: the Grams of the orthonormalisations and truncations have m, n
// of 5..64 and K = n, where a padded 32 x 32 register tile spent 3-10 times
// the algorithmic FMAs. This part issues FP64 at 2 FMA/clk/SM, so shared
// memory (two loads per FMA) has headroom and no register reuse is needed.
// The next k block is fetched into registers while the current one is used.
constexpr int GT = 16, GBK = 32;

template <bool TA, bool TB>
__global__ void __launch_bounds__(256) dgemm_group_kernel(GArgs g) {
  __shared__ double As[GBK][GT + 1];
  __shared__ double Bs[GBK][GT + 1];
  __shared__ double red[256];
  int item = 0;
  while (item + 1 < g.count && (int)blockIdx.x >= g.it[item + 1].cta0) ++item;
  const GItem &it = g.it[item];
  const int local = blockIdx.x - it.cta0;
  const int split = local % it.splits, tile = local / it.splits;
  const int row0 = (tile % it.gx) * GT, col0 = (tile / it.gx) * GT;
  const int m = it.m, n = it.n, lda = it.lda, ldb = it.ldb;
  const double *__restrict__ A = it.A;
  const double *__restrict__ B = it.B;
  const int k0 = split * it.kchunk;
  const int k1 = min(it.k, k0 + it.kchunk);
  const int mt = min(GT, m - row0), nt = min(GT, n - col0), P = mt * nt;
  const int S = 256 / P;  // k-lanes per output (>= 1)
  const int t = threadIdx.x;
  const int o = t % P, s = t / P;
  const bool active = s < S;
  const int oi = o % mt, oj = o / mt;
  // staging: elements e = t and t + 256 of the A block (GT x GBK) and the B block
  double pa[2], pb[2];
  auto fetch = [&](int kb) {
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int e = t + 256 * h;
      int i, kk;
      if (!TA) { i = e % GT; kk = e / GT; } else { kk = e % GBK; i = e / GBK; }
      const int gi = row0 + i, gk = kb + kk;
      pa[h] = (gi < m && gk < k1) ? (TA ? A[gk + (long long)gi * lda] : A[gi + (long long)gk * lda])
                                  : 0.0;
      int j;
      if (!TB) { kk = e % GBK; j = e / GBK; } else { j = e % GT; kk = e / GT; }
      const int gj = col0 + j;
      const int gk2 = kb + kk;
      pb[h] = (gj < n && gk2 < k1) ? (TB ? B[gj + (long long)gk2 * ldb] : B[gk2 + (long long)gj * ldb])
                                   : 0.0;
    }
  };
  double a0 = 0.0, a1 = 0.0;
  if (k0 < k1) fetch(k0);
  for (int kb = k0; kb < k1; kb += GBK) {
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int e = t + 256 * h;
      if (!TA) As[e / GT][e % GT] = pa[h]; else As[e % GBK][e / GBK] = pa[h];
      if (!TB) Bs[e % GBK][e / GBK] = pb[h]; else Bs[e / GT][e % GT] = pb[h];
    }
    __syncthreads();
    if (kb + GBK < k1) fetch(kb + GBK);
    const int kn = min(GBK, k1 - kb);
    if (active) {
      int kk = s;
      for (; kk + S < kn; kk += 2 * S) {
        a0 = fma(As[kk][oi], Bs[kk][oj], a0);
        a1 = fma(As[kk + S][oi], Bs[kk + S][oj], a1);
      }
      if (kk < kn) a0 = fma(As[kk][oi], Bs[kk][oj], a0);
    }
    __syncthreads();
  }
  double v = a0 + a1;
  if (S > 1) {
    red[t] = active ? v : 0.0;
    __syncthreads();
    if (active && s == 0)
      for (int q = 1; q < S; ++q) v += red[o + q * P];
  }
  if (!active || s != 0) return;
  const int gi = row0 + oi, gj = col0 + oj;
  if (it.splits == 1) {
    double *p = it.C + gi + (long long)gj * it.ldc;
    *p = (it.beta == 0.0) ? it.alpha * v : fma(it.alpha, v, it.beta * *p);
  } else {
    it.part[(long long)split * m * n + gi + (long long)gj * m] = v;
  }
}

// C_i = alpha_i sum_q part_i,q + beta_i C_i for the items with split K, in the
// fixed order of splitk_reduce (8 groups of splits, then the groups in order).
__global__ void __launch_bounds__(256) splitk_reduce_group(GArgs g, long long total) {
  __shared__ double red[8][33];
  const long long t = blockIdx.x * 32ll + threadIdx.x;
  int item = 0;
  if (t < total)
    while (item + 1 < g.count && t >= g.it[item + 1].out0) ++item;
  const GItem &it = g.it[item];
  const long long mn = (long long)it.m * it.n;
  const long long r = t - it.out0;
  double s = 0.0;
  if (t < total && it.splits > 1) {
    const double *p = it.part + r;
#pragma unroll 4
    for (int q = threadIdx.y; q < it.splits; q += 8) s += p[q * mn];
  }
  red[threadIdx.y][threadIdx.x] = s;
  __syncthreads();
  if (threadIdx.y == 0 && t < total && it.splits > 1) {
    for (int q = 1; q < 8; ++q) s += red[q][threadIdx.x];
    const int i = (int)(r % it.m), j = (int)(r / it.m);
    double *out = it.C + i + (long long)j * it.ldc;
    *out = (it.beta == 0.0) ? it.alpha * s : fma(it.alpha, s, it.beta * *out);
  }
}

void gemm_group(Ctx &c, int count, const GemmSpec *spec) {
  // items of one transposition pair go together; empty products are done alone
  std::vector<int> todo;
  for (int i = 0; i < count; ++i) {
    const GemmSpec &q = spec[i];
    if (q.m <= 0 || q.n <= 0) continue;
    if (q.k <= 0) {
      gemm(c, q.ta, q.tb, q.m, q.n, q.k, q.alpha, q.A, q.lda, 0, q.B, q.ldb, 0, q.beta, q.C, q.ldc, 0);
      continue;
    }
    todo.push_back(i);
  }
  while (!todo.empty()) {
    const bool ta = spec[todo[0]].ta, tb = spec[todo[0]].tb;
    std::vector<int> grp, rest;
    for (int i : todo) {
      if (spec[i].ta == ta && spec[i].tb == tb && (int)grp.size() < kGroupMax) grp.push_back(i);
      else rest.push_back(i);
    }
    todo.swap(rest);
    GArgs g;
    std::memset(&g, 0, sizeof(g));
    g.count = (int)grp.size();
    int ctas = 0;
    long long outs = 0, part_total = 0;
    double flops = 0, bytes = 0;
    for (int t = 0; t < g.count; ++t) {
      const GemmSpec &q = spec[grp[t]];
      GItem &it = g.it[t];
      it.A = q.A;
      it.B = q.B;
      it.C = q.C;
      it.alpha = q.alpha;
      it.beta = q.beta;
      it.m = q.m;
      it.n = q.n;
      it.k = q.k;
      it.lda = q.lda;
      it.ldb = q.ldb;
      it.ldc = q.ldc;
      it.gx = (q.m + GT - 1) / GT;
      const long long tiles = (long long)it.gx * ((q.n + GT - 1) / GT);
      if (tiles > (1ll << 30)) fail(TCTL_E_ARG, "gemm_group: item too large");
      // the group as a whole aims at about two CTAs per SM; a CTA contracts at
      // least two k blocks of 32, so its fixed costs stay small against its work
      const int target = (kSplitTarget + g.count - 1) / g.count;
      int splits = 1;
      if (tiles < target && q.k >= 4 * GBK)
        splits = (int)std::min<long long>((target + tiles - 1) / tiles, q.k / (2 * GBK));
      splits = std::max(1, std::min(splits, 256));
      int kchunk = (q.k + splits - 1) / splits;
      kchunk = ((kchunk + GBK - 1) / GBK) * GBK;
      it.splits = (q.k + kchunk - 1) / kchunk;
      it.kchunk = kchunk;
      it.cta0 = ctas;
      if ((long long)ctas + tiles * it.splits > (1ll << 31) - 1) fail(TCTL_E_ARG, "gemm_group: grid too large");
      ctas += (int)(tiles * it.splits);
      it.out0 = outs;
      outs += (long long)q.m * q.n;
      if (it.splits > 1) part_total += (long long)it.splits * q.m * q.n;
      flops += 2.0 * q.m * q.n * (double)q.k;
      bytes += 8.0 * ((double)q.m * q.k + (double)q.k * q.n + (double)q.m * q.n * (1 + (q.beta != 0.0)));
    }
    size_t mk = c.ws.mark();
    double *part = part_total > 0 ? c.ws.dbl((size_t)part_total) : nullptr;
    long long off = 0;
    for (int t = 0; t < g.count; ++t)
      if (g.it[t].splits > 1) {
        g.it[t].part = part + off;
        off += (long long)g.it[t].splits * g.it[t].m * g.it[t].n;
      }
    c.next_flops = flops;
    c.next_bytes = bytes;
    if (c.prof && c.trace) {
      // per-shape profile names (TCTL_TRACE=1 with profiling on)
      std::string nm = std::string("dgroup[") + (ta ? "T" : "N") + (tb ? "T" : "N");
      for (int t = 0; t < g.count; ++t) {
        char b[64];
        std::snprintf(b, sizeof(b), " %dx%dx%d s%d", g.it[t].m, g.it[t].n, g.it[t].k, g.it[t].splits);
        nm += b;
      }
      c.next_tag = c.intern((nm + "]").c_str());
    }
#define TCTL_GG(TA_, TB_) LAUNCH(c, (dgemm_group_kernel<TA_, TB_>), ctas, 256, 0, g)
    if (!ta && !tb) TCTL_GG(false, false);
    else if (!ta && tb) TCTL_GG(false, true);
    else if (ta && !tb) TCTL_GG(true, false);
    else TCTL_GG(true, true);
#undef TCTL_GG
    if (part_total > 0) {
      c.next_bytes = 8.0 * (double)(part_total + outs);
      LAUNCH(c, splitk_reduce_group, (unsigned)((outs + 31) / 32), dim3(32, 8), 0, g, outs);
    }
    c.ws.reset(mk);
  }
}

// ------------------------------------------------------------------ elementwise
__global__ void khatri_rao_kernel(int n, const double *__restrict__ A, int lda, int ra,
                                  const double *__restrict__ B, int ldb, int rb, double *out,
                                  int ldo) {
  const long long total = (long long)n * ra * rb;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < total;
       t += (long long)gridDim.x * blockDim.x) {
    const int i = (int)(t % n);
    const long long col = t / n;
    const int a = (int)(col % ra), bcol = (int)(col / ra);
    out[i + col * ldo] = A[i + (long long)a * lda] * B[i + (long long)bcol * ldb];
  }
}

void khatri_rao(Ctx &c, int n, const double *A, int lda, int ra, const double *B, int ldb, int rb,
                double *out, int ldo) {
  const long long total = (long long)n * ra * rb;
  if (total == 0) return;
  const int blocks = (int)std::min<long long>((total + 255) / 256, 152 * 16);
  c.next_bytes = 8.0 * ((double)total + (double)n * (ra + rb));
  LAUNCH(c, khatri_rao_kernel, blocks, 256, 0, n, A, lda, ra, B, ldb, rb, out, ldo);
}

__global__ void col_norms_kernel(int n, int m, const double *__restrict__ A, int lda,
                                 double *out) {
  const int j = blockIdx.x;
  double s = 0.0;
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    const double v = A[i + (long long)j * lda];
    s = fma(v, v, s);
  }
  __shared__ double red[32];
  for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x < 32) {
    s = (threadIdx.x < (blockDim.x >> 5)) ? red[threadIdx.x] : 0.0;
    for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
    if (threadIdx.x == 0) out[j] = sqrt(s);
  }
}

void col_norms(Ctx &c, int n, int m, const double *A, int lda, double *out) {
  if (m <= 0) return;
  LAUNCH(c, col_norms_kernel, m, 256, 0, n, m, A, lda, out);
}

__global__ void scale_cols_kernel(int n, int m, double *A, int lda, const double *s, int inv) {
  const long long total = (long long)n * m;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < total;
       t += (long long)gridDim.x * blockDim.x) {
    const int i = (int)(t % n), j = (int)(t / n);
    const double f = s[j];
    A[i + (long long)j * lda] *= inv ? (f != 0.0 ? 1.0 / f : 0.0) : f;
  }
}

void scale_cols(Ctx &c, int n, int m, double *A, int lda, const double *s, bool inverse) {
  const long long total = (long long)n * m;
  if (total == 0) return;
  const int blocks = (int)std::min<long long>((total + 255) / 256, 4096);
  LAUNCH(c, scale_cols_kernel, blocks, 256, 0, n, m, A, lda, s, inverse ? 1 : 0);
}

// splitmix64 counter hash -> two uniforms -> Box-Muller normal (gauss_draw)
__device__ __forceinline__ uint64_t mix64(uint64_t z) {
  z += 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

// Draw r of stream `seed`. The probes of the randomized range finder need
// Gaussian directions, not FP64-accurate samples: the Box-Muller transform runs
// in FP32 (24-bit uniforms; FP64 log / sqrt / cospi would cost tens of FP64
// operations per draw on this part) and the result is widened to FP64.
__device__ __forceinline__ double gauss_draw(uint64_t seed, uint64_t r) {
  const uint64_t h1 = mix64(seed ^ mix64(2 * r));
  const uint64_t h2 = mix64(seed ^ mix64(2 * r + 1));
  const float u1 = ((float)(uint32_t)(h1 >> 40) + 1.0f) * (1.0f / 16777216.0f);  // (0, 1]
  const float u2 = (float)(uint32_t)(h2 >> 40) * (1.0f / 16777216.0f);           // [0, 1)
  return (double)(sqrtf(-2.0f * logf(u1)) * cospif(2.0f * u2));
}

__global__ void gaussian_kernel(double *x, size_t count, uint64_t seed) {
  for (size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x; t < count;
       t += (size_t)gridDim.x * blockDim.x)
    x[t] = gauss_draw(seed, t);
}

void fill_gaussian(Ctx &c, double *x, size_t count, uint64_t seed) {
  if (count == 0) return;
  const int blocks = (int)std::min<size_t>((count + 255) / 256, 4096);
  LAUNCH(c, gaussian_kernel, blocks, 256, 0, x, count, seed);
}

// Several Gaussian fills in one launch: fill i writes x[i][t] = the value
// gaussian_kernel would write with seed[i] (the same counter-based draws).
struct GaussArgs {
  int count;
  double *x[3];
  uint64_t seed[3];
  long long off[4];  // prefix of the element counts
};

__global__ void gaussian_multi_kernel(GaussArgs a) {
  const long long total = a.off[a.count];
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < total;
       t += (long long)gridDim.x * blockDim.x) {
    int i = 0;
    while (i + 1 < a.count && t >= a.off[i + 1]) ++i;
    const uint64_t r = (uint64_t)(t - a.off[i]);
    a.x[i][r] = gauss_draw(a.seed[i], r);
  }
}

void fill_gaussian_multi(Ctx &c, int count, double *const *x, const size_t *n, const uint64_t *seed) {
  GaussArgs a{};
  long long tot = 0;
  for (int i = 0; i < count && i < 3; ++i) {
    a.x[a.count] = x[i];
    a.seed[a.count] = seed[i];
    a.off[a.count] = tot;
    tot += (long long)n[i];
    ++a.count;
  }
  if (!tot) return;
  a.off[a.count] = tot;
  const int blocks = (int)std::min<long long>((tot + 255) / 256, 4096);
  LAUNCH(c, gaussian_multi_kernel, blocks, 256, 0, a);
}

void fill_zero(Ctx &c, double *x, size_t count) {
  if (count) TCTL_CUDA(cudaMemsetAsync(x, 0, count * sizeof(double), c.st));
}

void copy_d(Ctx &c, double *dst, const double *src, size_t count) {
  if (count && dst != src)
    TCTL_CUDA(cudaMemcpyAsync(dst, src, count * sizeof(double), cudaMemcpyDeviceToDevice, c.st));
}

// Up to kCopyMax device-to-device copies in one launch.
constexpr int kCopyMax = 8;
struct CopyArgs {
  int count;
  double *dst[kCopyMax];
  const double *src[kCopyMax];
  long long off[kCopyMax + 1];  // prefix of the element counts
};

__global__ void copy_multi_kernel(CopyArgs a) {
  const long long total = a.off[a.count];
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < total;
       t += (long long)gridDim.x * blockDim.x) {
    int i = 0;
    while (i + 1 < a.count && t >= a.off[i + 1]) ++i;
    const long long r = t - a.off[i];
    a.dst[i][r] = a.src[i][r];
  }
}

void copy_multi(Ctx &c, int count, double *const *dst, const double *const *src, const size_t *n) {
  for (int b = 0; b < count; b += kCopyMax) {
    CopyArgs a;
    std::memset(&a, 0, sizeof(a));
    long long tot = 0;
    for (int i = b; i < std::min(count, b + kCopyMax); ++i) {
      if (!n[i] || dst[i] == src[i]) continue;
      a.dst[a.count] = dst[i];
      a.src[a.count] = src[i];
      a.off[a.count] = tot;
      tot += (long long)n[i];
      ++a.count;
    }
    if (!a.count) continue;
    a.off[a.count] = tot;
    const int blocks = (int)std::min<long long>((tot + 255) / 256, 152 * 8);
    c.next_bytes = 16.0 * tot;
    LAUNCH(c, copy_multi_kernel, blocks, 256, 0, a);
  }
}

__global__ void axpby_kernel(size_t count, double a, const double *x, double b, double *y) {
  for (size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x; t < count;
       t += (size_t)gridDim.x * blockDim.x)
    y[t] = (b == 0.0) ? a * x[t] : fma(a, x[t], b * y[t]);
}

void axpby(Ctx &c, size_t count, double a, const double *x, double b, double *y) {
  if (count == 0) return;
  const int blocks = (int)std::min<size_t>((count + 255) / 256, 4096);
  LAUNCH(c, axpby_kernel, blocks, 256, 0, count, a, x, b, y);
}

// Pinned staging buffers are recycled through a process-wide free list rather
// than freed: releasing pinned memory may synchronise the device, which would
// stall the other contexts' streams.
static std::mutex g_stage_mu;
static std::vector<char *> g_stage_free;

char *stage_acquire() {
  {
    std::lock_guard<std::mutex> lk(g_stage_mu);
    if (!g_stage_free.empty()) {
      char *p = g_stage_free.back();
      g_stage_free.pop_back();
      return p;
    }
  }
  void *p = nullptr;
  if (cudaHostAlloc(&p, kStageBytes, cudaHostAllocDefault) != cudaSuccess) {
    cudaGetLastError();
    return nullptr;  // transfers then take the pageable path
  }
  return static_cast<char *>(p);
}

void stage_release(char *p) {
  if (!p) return;
  std::lock_guard<std::mutex> lk(g_stage_mu);
  g_stage_free.push_back(p);
}

// A copy between device and pageable host memory may wait inside the driver
// for the stream to drain, and with many contexts working on concurrent
// streams that wait costs far more than synchronising the stream and copying
// from pinned memory. Small transfers therefore go through the context's
// pinned staging buffer; large ones synchronise first and copy directly.
void read_host(Ctx &c, void *dst, const void *src, size_t bytes) {
  if (!bytes) return;
  if (c.hstage && bytes <= kStageRead) {
    TCTL_CUDA(cudaMemcpyAsync(c.hstage, src, bytes, cudaMemcpyDeviceToHost, c.st));
    TCTL_CUDA(cudaStreamSynchronize(c.st));
    std::memcpy(dst, c.hstage, bytes);
  } else {
    TCTL_CUDA(cudaStreamSynchronize(c.st));
    TCTL_CUDA(cudaMemcpyAsync(dst, src, bytes, cudaMemcpyDeviceToHost, c.st));
    TCTL_CUDA(cudaStreamSynchronize(c.st));
  }
  c.hstage_top = 0;  // the stream is idle: every staged upload has landed
}

void write_dev(Ctx &c, void *dst, const void *src, size_t bytes) {
  if (!bytes) return;
  constexpr size_t ring = kStageBytes - kStageRead;
  if (!c.hstage || bytes > ring) {
    TCTL_CUDA(cudaStreamSynchronize(c.st));
    TCTL_CUDA(cudaMemcpyAsync(dst, src, bytes, cudaMemcpyHostToDevice, c.st));
    return;
  }
  size_t off = (c.hstage_top + 15) & ~size_t(15);
  if (off + bytes > ring) {  // ring full: wait until the queued uploads have landed
    TCTL_CUDA(cudaStreamSynchronize(c.st));
    off = 0;
  }
  char *p = c.hstage + kStageRead + off;
  std::memcpy(p, src, bytes);
  TCTL_CUDA(cudaMemcpyAsync(dst, p, bytes, cudaMemcpyHostToDevice, c.st));
  c.hstage_top = off + bytes;
}

void to_host(Ctx &c, double *dst, const double *src, size_t count) {
  read_host(c, dst, src, count * sizeof(double));
}

void to_dev(Ctx &c, double *dst, const double *src, size_t count) {
  write_dev(c, dst, src, count * sizeof(double));
}

// ------------------------------------------------------------------ Jacobi
// Parallel cyclic Jacobi (round-robin pairing) for symmetric m x m, m <= 64.
// One CTA per matrix; A and V in shared memory (padded to even size mp).
// Matrix b of the launch has size ms[b] and lives at As[b] (ld ms[b]); its
// eigenvalues (descending) go to lams[b], eigenvectors (columns) to Vs[b].
//
// A step rotates the mp/2 disjoint pairs (p, q) of the round-robin schedule at
// once: A <- J^T A J, V <- V J, J the product of the plane rotations
// [[c, s], [-s, c]] on (p, q). Since the pairs are disjoint, J^T A J splits into
// 2 x 2 blocks (rows of pair a, columns of pair b) that transform
// independently, B <- R_a^T B R_b; the upper-triangle blocks are computed once
// and mirrored (A stays exactly symmetric), and the rotated diagonal blocks
// are set to their exact values (a_pp - t a_pq, a_qq + t a_pq, 0) instead of
// being recomputed from differences of large numbers, so that the off-diagonal
// mass goes to zero rather than to the rounding level of the diagonal. A pair
// is left unrotated when |a_pq| <= about 1e-15 sqrt(a_pp a_qq) (the relative
// accuracy threshold of one-sided and two-sided Jacobi, Demmel and Veselic)
// or |a_pq| <= 1e-16 ||A||_F (the rounding level of the FP64 Gram products
// the kernel is given); the sweeps stop after a sweep without rotations.
constexpr int JMAX = 64;

struct EigDesc {
  const double *A;
  double *lam;
  double *V;
  int m;
};

// On this part one warp scheduler issues an FP64 instruction (any number of
// active lanes) every 64 cycles, and a dependent FP64 operation takes as long,
// while integer and FP32 operations take a few cycles; the FP64 conversions
// are FP64-pipe operations too. The rotation parameters are one warp's chain
// per step, so they are built from as few FP64 instructions as possible: the
// rotation test is taken on integer words, signs and factors of two are set
// on the bit patterns, and divisions and square roots are the hardware
// approximations (relative error below 2^-20, measured over [1, 4) on this
// part) refined by one third-order step each:
//   1/q:       r <- r (1 + e + e^2),          e = 1 - q r
//   1/sqrt(q): y <- y (1 + e/2 + 3 e^2 / 8),  e = 1 - q y^2
// (error about e^3, below 2^-57, i.e. the result is good to rounding). The
// rotation stays orthogonal to rounding level (c = 1/sqrt(1 + t^2) to a few
// ulp, s = t c).
__device__ __forceinline__ double jac_rcp(double q) {
  double r;
  asm("rcp.approx.ftz.f64 %0, %1;" : "=d"(r) : "d"(q));
  const double e = fma(-q, r, 1.0);
  return fma(r, fma(e, e, e), r);
}

__device__ __forceinline__ double jac_rsqrt(double q) {
  double y;
  asm("rsqrt.approx.ftz.f64 %0, %1;" : "=d"(y) : "d"(q));
  const double e = fma(-q, y * y, 1.0);
  return fma(y, e * fma(0.375, e, 0.5), y);
}

// -x on the bit pattern (an integer operation)
__device__ __forceinline__ double jac_neg(double x) {
  return __hiloint2double(__double2hiint(x) ^ (int)0x80000000, __double2loint(x));
}

// |x| as an integer increasing with |x|: the high word without the sign bit.
// (mag - (1023 << 20)) / 2^20 is log2|x| to within 0.09 (piecewise linear in
// the mantissa).
__device__ __forceinline__ int jac_mag(double x) { return __double2hiint(x) & 0x7fffffff; }

// log2(1e-30) in the units of jac_mag
constexpr int kJacRelMag = -104498822;

// Rotate the pair when |a_pq| is above the absolute floor (given as its
// jac_mag) and a_pq^2 above about 1e-30 |a_pp a_qq|; both compared on the
// integer words (the relative test to within a factor 1.3 on a_pq^2).
__device__ __forceinline__ bool jac_rotates(double app, double aqq, double apq, int floor_mag) {
  const int g = jac_mag(apq);
  return g > floor_mag && 2ll * g > (long long)jac_mag(app) + jac_mag(aqq) + kJacRelMag;
}

// The rotation that annihilates a_pq: tau2 = (a_qq - a_pp) / a_pq (twice the
// usual tau), t = sign(tau2) 2 / (|tau2| + sqrt(tau2^2 + 4)) (the root of
// t^2 + tau2 t - 1 = 0 with |t| <= 1), c = 1 / sqrt(1 + t^2), s = t c. A pair
// that passes the rotation test has |a_pq| > 1e-16 ||A||_F while
// |a_qq - a_pp| <= sqrt(2) ||A||_F, so |tau2| < 1.5e16: tau2^2 + 4 neither
// overflows nor calls for another form. 2 / den is 1 / den with the exponent
// raised by one (den in [2, 2e16], so 1 / den is a normal number) and the sign
// of tau2 set on the bit pattern.
__device__ __forceinline__ void jac_rotation(double app, double aqq, double apq, double &t, double &c,
                                             double &s) {
  const double tau2 = (aqq - app) * jac_rcp(apq);
  const double q4 = fma(tau2, tau2, 4.0);
  const double r = jac_rcp(fabs(tau2) + q4 * jac_rsqrt(q4));
  const int hi = (__double2hiint(r) + (1 << 20)) | (__double2hiint(tau2) & (int)0x80000000);
  t = __hiloint2double(hi, __double2loint(r));
  c = jac_rsqrt(fma(t, t, 1.0));
  s = t * c;
}

// One symmetric eigenproblem per thread-block cluster of kJacCluster CTAs
// (parallel-order Jacobi with exact 2x2 block updates). Every CTA keeps a
// replica of A and computes all rotation parameters of a step from it (the
// same operations on the same values); the 2x2 block updates of the step are
// dealt out over the CTAs, each writing its blocks into all replicas through
// distributed shared memory; each CTA owns a quarter of V's rows, whose
// updates need nothing from the others. The diagonal blocks are rotated by
// every CTA in its own replica, so one cluster barrier per step (every replica
// complete before the next parameters) suffices. The step's cost is FP64
// instructions per warp scheduler: the parameter chain of one warp, then the
// block and V updates packed onto few warps.
// The sweep-exit tests are taken from rank 0's flags by every CTA, so all
// CTAs run the same sequence of barriers whatever their replicas hold.
#ifndef TCTL_JAC_CLUSTER
#define TCTL_JAC_CLUSTER 4
#endif
constexpr int kJacCluster = TCTL_JAC_CLUSTER;  // CTAs per eigenproblem (2, 4 or 8)
// off-diagonal blocks one CTA updates at most (m <= JMAX)
constexpr int kJacOwnMax = ((JMAX / 2) * (JMAX / 2 - 1) / 2 + kJacCluster - 1) / kJacCluster;
constexpr int kJacThreads = 256;
static_assert(kJacOwnMax <= kJacThreads, "one lane per block at least");

__global__ void __cluster_dims__(kJacCluster, 1, 1) __launch_bounds__(kJacThreads)
    jacobi_kernel(const EigDesc *__restrict__ desc) {
  extern __shared__ double sm[];
  const int crank = (int)cl_rank();
  const EigDesc dsc = desc[blockIdx.x / kJacCluster];
  const int m = dsc.m;
  const int mp = (m + 1) & ~1;
  const int ld = mp + 1;
  const int half = mp / 2;
  const int vr = (mp + kJacCluster - 1) / kJacCluster;  // rows of V per CTA
  const int v0 = crank * vr, v1 = min(mp, v0 + vr);
  double *A = sm;               // mp x ld, replica
  double *V = A + mp * ld;      // rows v0..v1 of V, row-major: V[(i - v0) * ld + j]
  double *rc = V + vr * ld;     // half: c
  double *rs = rc + half;       // half: s
  int *rp = reinterpret_cast<int *>(rs + half);  // half: p
  int *rq = rp + half;                           // half: q
  int *rf = rq + half;                           // half: 1 if the pair rotates
  __shared__ double red[8];
  __shared__ int nrot, more, flag;
  // The off-diagonal blocks (a, b), a < b, of pairs a and b this CTA updates:
  // triangular indices b (b - 1) / 2 + a = crank, crank + kJacCluster, ...,
  // as a | b << 8.
  __shared__ int own[kJacOwnMax];
  const int ntri = half * (half - 1) / 2;
  const int nown = ntri > crank ? (ntri - crank + kJacCluster - 1) / kJacCluster : 0;
  for (int k = threadIdx.x; k < nown; k += blockDim.x) {
    const int kk = crank + kJacCluster * k;
    int b = (int)((1.0f + sqrtf(1.0f + 8.0f * (float)kk)) * 0.5f);
    while (b * (b - 1) / 2 > kk) --b;
    while ((b + 1) * b / 2 <= kk) ++b;
    own[k] = (kk - b * (b - 1) / 2) | (b << 8);
  }
  const double *Ab = dsc.A;
  double ss = 0.0;
  for (int t = threadIdx.x; t < mp * mp; t += blockDim.x) {
    const int i = t % mp, j = t / mp;
    const double v = (i < m && j < m) ? Ab[i + j * m] : 0.0;
    A[i + j * ld] = v;
    ss = fma(v, v, ss);
  }
  for (int t = threadIdx.x; t < (v1 - v0) * mp; t += blockDim.x) {
    const int i = v0 + t / mp, j = t % mp;
    V[(i - v0) * ld + j] = (i == j) ? 1.0 : 0.0;
  }
  for (int o = 16; o > 0; o >>= 1) ss += __shfl_down_sync(0xffffffffu, ss, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = ss;
  __syncthreads();
  double tot = 0.0;
  for (int w = 0; w < (int)(blockDim.x >> 5); ++w) tot += red[w];
  // |a_pq| below this: no rotation. The inputs are FP64 Gram products,
  // whose entries already carry rounding errors of about 1e-16 ||A||_F, so
  // annihilating smaller entries adds no accuracy
  const int floor_mag = jac_mag(1e-16 * sqrt(tot));
  uint32_t abase[kJacCluster];
#pragma unroll
  for (int r = 0; r < kJacCluster; ++r) abase[r] = cl_map(A, (uint32_t)r);
  const uint32_t nrot0 = cl_map(&nrot, 0), more0 = cl_map(&more, 0);
  cl_sync();  // every replica is initialised before any remote write
  // Entries (i, j), j in [j0, j0 + nj), of row i of the block (a, b) of
  // B <- R_a^T B R_b (B = [b00 b01; b10 b11], read before any lane of the
  // block writes), written into every replica (both triangles).
  auto block_row = [&](int a, int b, int i, int j0, int nj, double b00, double b01, double b10,
                       double b11) {
    const int pa = rp[a], qa = rq[a], pb = rp[b], qb = rq[b];
    const double ca = rc[a], sa = rs[a], cb = rc[b], sb = rs[b];
    const double x = i ? sa : ca, z = i ? ca : jac_neg(sa);
    const double l0 = fma(z, b10, x * b00);
    const double l1 = fma(z, b11, x * b01);
    const int row = i ? qa : pa;
    for (int j = j0; j < j0 + nj; ++j) {
      const double y = j ? sb : cb, w = j ? cb : jac_neg(sb);
      const double n = fma(l1, w, l0 * y);
      const int col = j ? qb : pb;
#pragma unroll
      for (int r = 0; r < kJacCluster; ++r) {
        cl_st(abase[r] + 8u * (uint32_t)(row + col * ld), n);
        cl_st(abase[r] + 8u * (uint32_t)(col + row * ld), n);
      }
    }
  };
  // Lanes per block: the blocks are packed onto as few warps as possible
  // (an FP64 instruction costs a warp scheduler the same for 1 or 32 active
  // lanes): 4 lanes (one entry each, 6 FP64 operations) while the blocks fit
  // 32 to a warp, 2 lanes (one row, 8) while they fit 64, else 1 (16).
  const int lsh = nown <= 32 ? 2 : nown <= 64 ? 1 : 0, lpb = 1 << lsh;
  for (int sweep = 0; sweep < 40 && mp > 1; ++sweep) {
    if (threadIdx.x == 0) nrot = 0;
    __syncthreads();
    for (int step = 0; step < mp - 1; ++step) {
      if (threadIdx.x < half) {
        // round robin: position 0 fixed, the others rotate
        const int t = threadIdx.x;
        auto at = [&](int pos) { return pos == 0 ? 0 : 1 + (pos - 1 + step) % (mp - 1); };
        int p = at(t), q = at(mp - 1 - t);
        if (p > q) { const int tmp = p; p = q; q = tmp; }
        const double app = A[p + p * ld], aqq = A[q + q * ld], apq = A[p + q * ld];
        double cc = 1.0, sn = 0.0;
        const bool rot = jac_rotates(app, aqq, apq, floor_mag);
        if (rot) {
          double tt;
          jac_rotation(app, aqq, apq, tt, cc, sn);
          nrot = 1;
          // The diagonal block (p, q), the only entries the parameters read,
          // is rotated by every CTA in its own replica (identical operations
          // on identical values), so no remote write can meet another CTA
          // still reading its pivots.
          A[p + p * ld] = fma(-tt, apq, app);
          A[q + q * ld] = fma(tt, apq, aqq);
          A[p + q * ld] = 0.0;
          A[q + p * ld] = 0.0;
        }
        rc[t] = cc;
        rs[t] = sn;
        rf[t] = rot;
        rp[t] = p;
        rq[t] = q;
      }
      __syncthreads();
      // This CTA's off-diagonal blocks (nown * lpb <= blockDim.x lanes, the
      // lanes of a block in one warp), written into every replica; a block's
      // lanes read its four entries before any of them writes.
      {
        const int e = threadIdx.x;
        int a = 0, b = 0, j = 0;
        bool go = false;
        double b00 = 0.0, b01 = 0.0, b10 = 0.0, b11 = 0.0;
        if (e < nown * lpb) {
          const int k = e >> lsh;
          j = e & (lpb - 1);
          a = own[k] & 255;
          b = own[k] >> 8;
          go = rf[a] || rf[b];
          if (go) {
            const int pa = rp[a], qa = rq[a], pb = rp[b], qb = rq[b];
            b00 = A[pa + pb * ld];
            b01 = A[pa + qb * ld];
            b10 = A[qa + pb * ld];
            b11 = A[qa + qb * ld];
          }
        }
        __syncwarp();
        if (go) {
          if (lpb == 4) {
            block_row(a, b, j >> 1, j & 1, 1, b00, b01, b10, b11);
          } else if (lpb == 2) {
            block_row(a, b, j, 0, 2, b00, b01, b10, b11);
          } else {
            block_row(a, b, 0, 0, 2, b00, b01, b10, b11);
            block_row(a, b, 1, 0, 2, b00, b01, b10, b11);
          }
        }
      }
      // columns p, q of this CTA's rows of V
      const int nv = v1 - v0;
      for (int u = threadIdx.x; u < half * nv; u += blockDim.x) {
        const int a = u % half, i = u / half;
        if (!rf[a]) continue;
        const double cc = rc[a], sn = rs[a];
        const int p = rp[a], q = rq[a];
        double *row = V + i * ld;
        const double vp = row[p], vq = row[q];
        row[p] = cc * vp - sn * vq;
        row[q] = sn * vp + cc * vq;
      }
      cl_sync();  // every replica holds the step's blocks before the next parameters
    }
    // Rank 0's flags decide for the whole cluster. Would the next sweep rotate
    // anything? A pair's test reads only entries that nothing but rotations
    // change, so a sweep without rotations is exactly the case where no pair
    // passes the test now: checking every pair once replaces that confirming
    // sweep (same result, 1/(mp-1) of its work).
    if (threadIdx.x == 0) flag = cl_ld(nrot0);
    cl_sync();  // read by every CTA before rank 0 resets it
    if (flag == 0) break;
    if (threadIdx.x == 0) more = 0;
    __syncthreads();
    for (int u = threadIdx.x; u < m * m; u += blockDim.x) {
      const int i = u % m, j = u / m;
      if (i >= j) continue;
      if (jac_rotates(A[i + i * ld], A[j + j * ld], A[i + j * ld], floor_mag)) more = 1;
    }
    cl_sync();  // rank 0's flag is final
    if (threadIdx.x == 0) flag = cl_ld(more0);
    cl_sync();  // read by every CTA before the next sweep resets the flags
    if (flag == 0) break;
  }
  cl_sync();  // no remote access to this CTA's shared memory after here
  // sort eigenvalues descending (selection by rank, m <= 64); this CTA writes
  // its rows of each eigenvector
  for (int i = threadIdx.x; i < m; i += blockDim.x) {
    const double di = A[i + i * ld];
    int rank = 0;
    for (int j = 0; j < m; ++j) {
      const double dj = A[j + j * ld];
      rank += (dj > di) || (dj == di && j < i);
    }
    if (crank == 0) dsc.lam[rank] = di;
    for (int r = v0; r < min(v1, m); ++r) dsc.V[r + (long long)rank * m] = V[(r - v0) * ld + i];
  }
}

static void jacobi_launch(Ctx &c, const std::vector<EigDesc> &d) {
  if (d.empty()) return;
  int mmax = 0;
  for (const EigDesc &e : d) {
    if (e.m > JMAX) fail(TCTL_E_ARG, "sym_eig: m > 64");
    mmax = std::max(mmax, e.m);
  }
  if (mmax <= 0) return;
  const int mp = (mmax + 1) & ~1;
  const int vr = (mp + kJacCluster - 1) / kJacCluster;
  const size_t smem = sizeof(double) * ((size_t)(mp + vr) * (mp + 1) + 2 * (mp / 2)) + sizeof(int) * 3 * (mp / 2);
  // set once per process, thread-safely (function-local static initialisation)
  static const cudaError_t attr =
      cudaFuncSetAttribute(jacobi_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, 100 * 1024);
  TCTL_CUDA(attr);
  size_t mk = c.ws.mark();
  EigDesc *dd = static_cast<EigDesc *>(c.ws.alloc(sizeof(EigDesc) * d.size()));
  TCTL_CUDA(cudaMemcpyAsync(dd, d.data(), sizeof(EigDesc) * d.size(), cudaMemcpyHostToDevice, c.st));
  LAUNCH(c, jacobi_kernel, (int)d.size() * kJacCluster, kJacThreads, smem, dd);
  // the descriptor buffer must outlive the (asynchronous) launch
  TCTL_CUDA(cudaStreamSynchronize(c.st));
  c.ws.reset(mk);
}

void sym_eig(Ctx &c, int m, int batch, const double *A, double *lam, double *Vout) {
  if (m <= 0 || batch <= 0) return;
  std::vector<EigDesc> d(batch);
  for (int b = 0; b < batch; ++b)
    d[b] = EigDesc{A + (size_t)b * m * m, lam + (size_t)b * m, Vout + (size_t)b * m * m, m};
  jacobi_launch(c, d);
}

void sym_eig_multi(Ctx &c, int count, const int *m, const double *const *A, double *const *lam,
                   double *const *Vout) {
  std::vector<EigDesc> d;
  for (int b = 0; b < count; ++b)
    if (m[b] > 0) d.push_back(EigDesc{A[b], lam[b], Vout[b], m[b]});
  jacobi_launch(c, d);
}

// ------------------------------------------------------------------ orth
// Pivoted Cholesky of the Gram matrix G (m x m): P^T G P = L L^T on the first
// r pivots, stopping when the largest remaining Schur diagonal is <= thr.
// Writes perm[0..r) and L (r x r, lower, ld 64) and r to out_r.
// Pivoting is virtual: G stays in its original order and a used[] mask marks
// the chosen indices; column p_j of G is overwritten by column j of L (at the
// original rows), which no later update touches, so L(a, b) = G[p_a][p_b].
// Each step is a warp argmax of the remaining diagonal, the new column of L,
// and a rank-1 update of the remaining block (three barriers).
__device__ __forceinline__ void pivchol_body(int m, const double *__restrict__ Gin,
                                             double thr_rel_or_abs, int relative, int rcap,
                                             int *perm_out, double *L_out, int *out_r) {
  __shared__ double G[JMAX][JMAX + 1];
  __shared__ int used[JMAX], perm[JMAX], rem[JMAX];
  __shared__ int piv, nrem;
  __shared__ double thr, dpiv, ipiv;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  for (int t = tid; t < m * m; t += blockDim.x) G[t % m][t / m] = Gin[t];
  for (int t = tid; t < m; t += blockDim.x) used[t] = 0;
  __syncthreads();
  if (warp == 0) {
    double dmax = 0.0;
    for (int i = lane; i < m; i += 32) dmax = fmax(dmax, G[i][i]);
    for (int o = 16; o > 0; o >>= 1) dmax = fmax(dmax, __shfl_xor_sync(0xffffffffu, dmax, o));
    if (lane == 0) {
      thr = relative ? thr_rel_or_abs * thr_rel_or_abs * dmax : thr_rel_or_abs * thr_rel_or_abs;
      if (!(dmax > 0.0)) thr = 1e300;
    }
  }
  __syncthreads();
  int r = 0;
  const int rmax = min(m, rcap);
  // The pivot search compares bit patterns as integers: a non-negative double
  // orders as its bit pattern, a negative one (sign bit set) as a negative
  // integer, below every candidate; the FP64 pipe (one instruction per 64
  // cycles per warp scheduler on this part) is kept for the arithmetic.
  const long long thr_bits = __double_as_longlong(thr);
  constexpr long long kInfBits = 0x7ff0000000000000ll;
  const long long tiny_bits = __double_as_longlong(1e-300);
  for (int j = 0; j < rmax; ++j) {
    if (warp == 0) {
      long long bk = -1;
      int bi = m;
      for (int i = lane; i < m; i += 32) {
        if (used[i]) continue;
        const long long k = __double_as_longlong(G[i][i]);
        if (k > bk) { bk = k; bi = i; }  // lanes scan ascending i: ties keep the lower index
      }
      for (int o = 16; o > 0; o >>= 1) {
        const long long ok_ = __shfl_xor_sync(0xffffffffu, bk, o);
        const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
        if (ok_ > bk || (ok_ == bk && oi < bi)) { bk = ok_; bi = oi; }
      }
      // every lane holds the same (bk, bi) after the butterfly; the pivot is
      // above the threshold and finite
      const bool ok = bi < m && bk > thr_bits && bk < kInfBits;
      if (lane == 0) {
        piv = ok ? bi : -1;
        if (ok) {
          used[bi] = 1;
          perm[j] = bi;
          // 1 / sqrt(pivot) as the hardware approximation refined by one
          // third-order step (a few FP64 operations instead of a correctly
          // rounded square root and one division per column entry)
          const double bv = __longlong_as_double(bk);
          const double y = bk > tiny_bits ? jac_rsqrt(bv) : 1.0 / sqrt(bv);
          dpiv = bv * y;
          ipiv = y;
        }
      }
      if (ok) {
        // the indices still to eliminate, in ascending order (ballot compaction)
        int base = 0;
        for (int c0 = 0; c0 < m; c0 += 32) {
          const int i = c0 + lane;
          const bool u = i < m && i != bi && !used[i];
          const unsigned bal = __ballot_sync(0xffffffffu, u);
          if (u) rem[base + __popc(bal & ((1u << lane) - 1u))] = i;
          base += __popc(bal);
        }
        if (lane == 0) nrem = base;
      }
    }
    __syncthreads();
    const int p = piv;
    if (p < 0) break;
    const double dp = dpiv, ip = ipiv;
    const int nr = nrem;
    // The Schur complement is kept in the lower triangle only (entry {i, k}
    // at G[max][min]); column p of L is written whole into G[.][p] (its slots
    // above the diagonal belong to no pair, those below to pairs with p,
    // which are eliminated now).
    for (int i = tid; i < m; i += blockDim.x) {
      const double g = G[max(i, p)][min(i, p)];
      G[i][p] = (i == p) ? dp : (used[i] ? 0.0 : g * ip);
    }
    __syncthreads();
    // Schur complement on the remaining indices: the nr (nr + 1) / 2 pairs
    // a >= b of rem, t = a (a + 1) / 2 + b, dealt out over the threads
    const int ntri = nr * (nr + 1) / 2;
    for (int t = tid; t < ntri; t += blockDim.x) {
      int a = (int)((sqrtf(8.0f * (float)t + 1.0f) - 1.0f) * 0.5f);
      while (a * (a + 1) / 2 > t) --a;
      while ((a + 1) * (a + 2) / 2 <= t) ++a;
      const int i = rem[a], k = rem[t - a * (a + 1) / 2];
      const int hi = max(i, k), lo = min(i, k);
      G[hi][lo] = fma(-G[i][p], G[k][p], G[hi][lo]);
    }
    __syncthreads();
    r = j + 1;
  }
  for (int t = tid; t < r * r; t += blockDim.x) {
    const int a = t % r, b = t / r;
    L_out[a + b * JMAX] = (b <= a) ? G[perm[a]][perm[b]] : 0.0;
  }
  for (int t = tid; t < r; t += blockDim.x) perm_out[t] = perm[t];
  if (tid == 0) *out_r = r;
}

__global__ void __launch_bounds__(256) pivchol_kernel(int m, const double *__restrict__ Gin,
                                                      double thr_rel_or_abs, int relative, int rcap,
                                                      int *perm_out, double *L_out, int *out_r) {
  pivchol_body(m, Gin, thr_rel_or_abs, relative, rcap, perm_out, L_out, out_r);
}

// Several independent pivoted Cholesky factorizations, one CTA each.
struct PcDesc {
  const double *G;
  int m, rcap;
  int *perm;
  double *L;
  int *r;
};

constexpr int ORTH_BATCH = 8;
struct PcBatch {
  PcDesc d[ORTH_BATCH];
};

__global__ void __launch_bounds__(256) pivchol_multi_kernel(const __grid_constant__ PcBatch b,
                                                            double thr_rel_or_abs, int relative) {
  const PcDesc x = b.d[blockIdx.x];
  pivchol_body(x.m, x.G, thr_rel_or_abs, relative, x.rcap, x.perm, x.L, x.r);
}

// max_ij |G_ij - delta_ij| > tol  ->  *flag = 1 (G: r x r Gram of nearly orthonormal columns)
__global__ void orth_check_kernel(int r, const double *__restrict__ G, double tol, int *flag) {
  int bad = 0;
  for (int t = threadIdx.x; t < r * r; t += blockDim.x) {
    const int i = t % r, j = t / r;
    const double d = G[t] - (i == j ? 1.0 : 0.0);
    if (!(fabs(d) <= tol)) bad = 1;
  }
  bad = __syncthreads_or(bad);
  if (threadIdx.x == 0) *flag = bad;
}

// orth_check_kernel for up to ORTH_BATCH matrices, one CTA each (r = 0: skipped).
struct OcBatch {
  const double *G[8];
  int r[8];
  int *flag[8];
};

__global__ void orth_check_multi_kernel(OcBatch b, double tol) {
  const int q = blockIdx.x, r = b.r[q];
  if (r <= 0) return;
  const double *G = b.G[q];
  int bad = 0;
  for (int t = threadIdx.x; t < r * r; t += blockDim.x) {
    const int i = t % r, j = t / r;
    const double d = G[t] - (i == j ? 1.0 : 0.0);
    if (!(fabs(d) <= tol)) bad = 1;
  }
  bad = __syncthreads_or(bad);
  if (threadIdx.x == 0) *b.flag[q] = bad;
}

// Q[i, :] = Y[i, perm] L^{-T}: forward substitution per row (x L^T = y).
// Q[i, :] solves Q[i, :] L^T = Y[i, perm] (row i independent), four lanes per
// row (blockDim / 4 rows per block). Columns go in blocks of 8, two per lane:
// a lane sums the contributions of the solved columns to its two, then the 8
// x values of the block are formed one by one by their owner and broadcast to
// the other three lanes (each keeps a full copy of the row's x). The diagonal
// is applied through its reciprocal. Four lanes per row give the 3 x n rows of
// a batch enough warps to keep every SM sub-partition's FP64 unit busy (this
// part issues 2 FP64 FMA per clock per SM).
__device__ __forceinline__ void trsm_rows_body(int n, int r, const double *__restrict__ Y, int ldy,
                                               const int *__restrict__ perm,
                                               const double *__restrict__ Lg, double *__restrict__ Q,
                                               int ldq, int bx, int gx) {
  __shared__ double L[JMAX][JMAX + 1];
  __shared__ double inv[JMAX];
  __shared__ int pm[JMAX];
  for (int t = threadIdx.x; t < r * r; t += blockDim.x) L[t % r][t / r] = Lg[(t % r) + (t / r) * JMAX];
  for (int t = threadIdx.x; t < r; t += blockDim.x) {
    pm[t] = perm[t];
    inv[t] = 1.0 / Lg[t + t * JMAX];
  }
  __syncthreads();
  constexpr int JB = 8;
  const int lane = threadIdx.x & 31, cl = lane & 3, grp = lane & ~3;
  const int rows = blockDim.x >> 2;
  for (int base = bx * rows; base < n; base += gx * rows) {
    const int i = base + (threadIdx.x >> 2);
    const bool ok = i < n;
    double x[JMAX];
#pragma unroll 1
    for (int j0 = 0; j0 < r; j0 += JB) {
      const int nb = min(JB, r - j0);
      const int c0 = 2 * cl, c1 = 2 * cl + 1;  // this lane's columns j0 + c0, j0 + c1
      const int l0 = min(j0 + c0, r - 1), l1 = min(j0 + c1, r - 1);
      double s0 = (ok && c0 < nb) ? Y[i + (long long)pm[j0 + c0] * ldy] : 0.0;
      double s1 = (ok && c1 < nb) ? Y[i + (long long)pm[j0 + c1] * ldy] : 0.0;
#pragma unroll 4
      for (int k = 0; k < j0; ++k) {
        const double xk = x[k];
        s0 = fma(-xk, L[l0][k], s0);
        s1 = fma(-xk, L[l1][k], s1);
      }
#pragma unroll 1
      for (int q = 0; q < nb; ++q) {
        const double v = ((q & 1) ? s1 : s0) * inv[j0 + q];
        const double xq = __shfl_sync(0xffffffffu, v, grp + (q >> 1));
        x[j0 + q] = xq;
        if (c0 > q) s0 = fma(-xq, L[l0][j0 + q], s0);
        if (c1 > q) s1 = fma(-xq, L[l1][j0 + q], s1);
      }
    }
    if (ok)
#pragma unroll 1
      for (int j = cl; j < r; j += 4) Q[i + (long long)j * ldq] = x[j];
  }
}

__global__ void trsm_rows_kernel(int n, int r, const double *__restrict__ Y, int ldy,
                                 const int *__restrict__ perm, const double *__restrict__ Lg,
                                 double *__restrict__ Q, int ldq) {
  trsm_rows_body(n, r, Y, ldy, perm, Lg, Q, ldq, blockIdx.x, gridDim.x);
}

struct TrDesc {
  const double *Y;
  int ldy, r;
  const int *perm;
  const double *L;
  double *Q;
};

struct TrBatch {
  TrDesc d[ORTH_BATCH];
};

// blockIdx.y selects the problem; problems with r = 0 do nothing
__global__ void trsm_rows_multi_kernel(int n, const __grid_constant__ TrBatch b) {
  const TrDesc x = b.d[blockIdx.y];
  if (x.r <= 0) return;
  trsm_rows_body(n, x.r, x.Y, x.ldy, x.perm, x.L, x.Q, n, blockIdx.x, gridDim.x);
}

int orth(Ctx &c, int n, int m, const double *Y, int ldy, double tol, bool relative, int rcap,
         double *Q) {
  if (m <= 0) return 0;
  if (m > JMAX) fail(TCTL_E_ARG, "orth: more than 64 columns");
  size_t mk = c.ws.mark();
  double *G = c.ws.dbl((size_t)m * m);
  double *L = c.ws.dbl((size_t)JMAX * JMAX);
  int *perm = c.ws.i32(JMAX);
  int *rdev = c.ws.i32(4);
  double *Q2 = c.ws.dbl((size_t)n * std::min(m, rcap > 0 ? rcap : 1));
  // 32 rows per block of 128 threads (four lanes per row)
  const int blocks = std::min((n + 31) / 32, 4096);
  auto read_int = [&](const int *p) {
    int v = 0;
    read_host(c, &v, p, sizeof(int));
    return v;
  };
  // pass 1: pivoted Cholesky of Y^T Y picks the columns and the rank
  gemm(c, true, false, m, m, n, 1.0, Y, ldy, 0, Y, ldy, 0, 0.0, G, m, 0);
  LAUNCH(c, pivchol_kernel, 1, 256, 0, m, G, tol, relative ? 1 : 0, rcap, perm, L, rdev);
  int r = read_int(rdev);
  if (r > 0) {
    LAUNCH(c, trsm_rows_kernel, blocks, 128, 0, n, r, Y, ldy, perm, L, Q, n);
    // passes 2 and 3 (Cholesky QR on the result) restore orthogonality to rounding
    // level; a column whose residual has fallen to rounding noise (kept in pass 1 at
    // the edge of the tolerance) is dropped here instead of breaking the factorization.
    // Pass 3 runs only if pass 2 left Q^T Q further than 1e-13 from the identity.
    for (int pass = 0; pass < 2 && r > 0; ++pass) {
      gemm(c, true, false, r, r, n, 1.0, Q, n, 0, Q, n, 0, 0.0, G, r, 0);
      if (pass == 1) {
        LAUNCH(c, orth_check_kernel, 1, 256, 0, r, G, 1e-13, rdev + 1);
        if (!read_int(rdev + 1)) break;
      }
      LAUNCH(c, pivchol_kernel, 1, 256, 0, r, G, 1e-10, 1, r, perm, L, rdev);
      const int r2 = read_int(rdev);
      if (r2 > 0) {
        LAUNCH(c, trsm_rows_kernel, blocks, 128, 0, n, r2, Q, n, perm, L, Q2, n);
        copy_d(c, Q, Q2, (size_t)n * r2);
      }
      r = r2;
    }
  }
  c.ws.reset(mk);
  return r;
}

// Orthonormal bases of several independent matrices at once (same algorithm as
// orth: pivoted Cholesky QR, up to three passes): one pivoted Cholesky launch
// (one CTA per matrix), one rank read-back and one triangular-solve launch per
// pass instead of one per matrix.
void orth_multi(Ctx &c, int count, int n, const int *m, double *const *Y, const int *ldy, double tol,
                bool relative, const int *rcap, double *const *Q, int *r_out) {
  if (count <= 0) return;
  if (count > ORTH_BATCH) fail(TCTL_E_ARG, "orth_multi: more than 8 matrices");
  for (int i = 0; i < count; ++i)
    if (m[i] > JMAX) fail(TCTL_E_ARG, "orth: more than 64 columns");
  size_t mk = c.ws.mark();
  std::vector<double *> G(count), L(count), Q2(count);
  std::vector<int *> perm(count);
  int *rdev = c.ws.i32((size_t)2 * count + 2);
  for (int i = 0; i < count; ++i) {
    G[i] = c.ws.dbl((size_t)JMAX * JMAX);
    L[i] = c.ws.dbl((size_t)JMAX * JMAX);
    perm[i] = c.ws.i32(JMAX);
    Q2[i] = c.ws.dbl((size_t)n * std::max(1, std::min(m[i], rcap[i] > 0 ? rcap[i] : 1)));
  }
  PcBatch hp{};
  TrBatch ht{};
  std::vector<int> r(count, 0), rr(2 * count);
  const int blocks = std::min((n + 31) / 32, 4096);
  auto read_ints = [&](int k) {
    read_host(c, rr.data(), rdev, sizeof(int) * k);
  };
  auto pivchol_all = [&](const std::vector<int> &mm, const std::vector<int> &cap, double thr, int rel) {
    for (int i = 0; i < count; ++i) hp.d[i] = PcDesc{G[i], mm[i], cap[i], perm[i], L[i], rdev + i};
    LAUNCH(c, pivchol_multi_kernel, count, 256, 0, hp, thr, rel);
    read_ints(count);
  };
  auto trsm_all = [&](const std::vector<const double *> &src, const std::vector<int> &ld,
                      const std::vector<int> &rk, const std::vector<double *> &dst) {
    for (int i = 0; i < count; ++i) ht.d[i] = TrDesc{src[i], ld[i], rk[i], perm[i], L[i], dst[i]};
    LAUNCH(c, trsm_rows_multi_kernel, dim3(blocks, count), 128, 0, n, ht);
  };
  // pass 1: pivoted Cholesky of Y^T Y picks the columns and the ranks
  std::vector<int> mm(m, m + count), cap(count);
  {
    // the Gram matrices of all the matrices in one grouped launch
    std::vector<GemmSpec> g;
    for (int i = 0; i < count; ++i) {
      cap[i] = rcap[i];
      if (m[i] > 0) g.push_back(GemmSpec{true, false, m[i], m[i], n, 1.0, Y[i], ldy[i], Y[i], ldy[i], 0.0, G[i], m[i]});
    }
    gemm_group(c, (int)g.size(), g.data());
  }
  pivchol_all(mm, cap, tol, relative ? 1 : 0);
  for (int i = 0; i < count; ++i) r[i] = m[i] > 0 ? rr[i] : 0;
  {
    std::vector<const double *> src(Y, Y + count);
    std::vector<int> ld(ldy, ldy + count);
    std::vector<double *> dst(Q, Q + count);
    trsm_all(src, ld, r, dst);
  }
  // passes 2 and 3: Cholesky QR of the result (see orth); pass 3 only where pass 2
  // left Q^T Q further than 1e-13 from the identity
  std::vector<char> active(count);
  for (int i = 0; i < count; ++i) active[i] = r[i] > 0;
  for (int pass = 0; pass < 2; ++pass) {
    std::vector<GemmSpec> g;
    for (int i = 0; i < count; ++i)
      if (active[i]) g.push_back(GemmSpec{true, false, r[i], r[i], n, 1.0, Q[i], n, Q[i], n, 0.0, G[i], r[i]});
    if (g.empty()) break;
    gemm_group(c, (int)g.size(), g.data());
    if (pass == 1) {
      OcBatch ob{};
      for (int i = 0; i < count; ++i) {
        ob.G[i] = G[i];
        ob.r[i] = active[i] ? r[i] : 0;
        ob.flag[i] = rdev + count + i;
      }
      TCTL_CUDA(cudaMemsetAsync(rdev + count, 0, sizeof(int) * count, c.st));
      LAUNCH(c, orth_check_multi_kernel, count, 256, 0, ob, 1e-13);
      read_ints(2 * count);
      bool any = false;
      for (int i = 0; i < count; ++i) {
        if (active[i] && !rr[count + i]) active[i] = 0;
        any = any || active[i];
      }
      if (!any) break;
    }
    std::vector<int> m2(count, 0), c2(count, 0);
    for (int i = 0; i < count; ++i)
      if (active[i]) {
        m2[i] = r[i];
        c2[i] = r[i];
      }
    pivchol_all(m2, c2, 1e-10, 1);
    std::vector<int> r2(count, 0);
    for (int i = 0; i < count; ++i) r2[i] = active[i] ? rr[i] : 0;
    {
      std::vector<const double *> src(Q, Q + count);
      std::vector<int> ld(count, n);
      trsm_all(src, ld, r2, Q2);
    }
    {
      std::vector<double *> dst;
      std::vector<const double *> srcq;
      std::vector<size_t> cnt;
      for (int i = 0; i < count; ++i)
        if (active[i] && r2[i] > 0) {
          dst.push_back(Q[i]);
          srcq.push_back(Q2[i]);
          cnt.push_back((size_t)n * r2[i]);
        }
      copy_multi(c, (int)dst.size(), dst.data(), srcq.data(), cnt.data());
    }
    for (int i = 0; i < count; ++i)
      if (active[i]) {
        r[i] = r2[i];
        if (r[i] == 0) active[i] = 0;
      }
  }
  for (int i = 0; i < count; ++i) r_out[i] = r[i];
  c.ws.reset(mk);
}

}  // namespace tctl
