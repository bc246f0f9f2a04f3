// FP64-class GEMMs of the rank-structured solver on the 5th-generation tensor
// cores (tcgen05, TMEM), by splitting both operands into D signed 7-bit digits
// (the splitting of Ozaki et al.).
//
// GB300 executes FP64 at 2 FMA/clk/SM (1.26 TFLOP/s per GPU) but BF16 at
// ~2.25 PFLOP/s. The contractions of the truncated Hadamard product (the
// sketches of its mode unfoldings and the projection of its core onto the new
// bases, Section 3.4 / Appendix 1 steps of Algorithm 1's fun and precond) are
// GEMMs with K up to n; they are run here as sums of BF16 digit products:
//   A[m, k] ~ 2^(e_m - 7) sum_p a_p[m, k],   B[k, j] ~ 2^(f_j - 7) sum_q b_q[k, j],
// with e_m (f_j) the binary exponent bound of row m of A (column j of B),
// a_p, b_q integers |.| <= 127 scaled by 2^-7p (exact in BF16), and
//   C[m, j] = 2^(e_m + f_j - 14) sum_{p + q <= D - 1} (a_p b_q)[m, j].
// The 7D-bit fixed point of each element is truncated; the neglected digit
// products and the truncation are ~2^-7D of the row / column maxima (D = 6:
// 42 bits, ~2e-13 relative to max|A_m| max|B_j| K; D = 4: 28 bits; D = 3:
// 21 bits in six products, the three-term BF16 split with FP32 accumulation).
// Products go to four TMEM accumulators by digit level L = p + q: levels 0, 1
// and 2 separately (every partial sum is an integer multiple of 2^-7L below
// (L + 1) 127^2 KCHUNK 2^-7L, i.e. fewer than 2^24 units for KCHUNK = 256:
// exact in FP32 whatever the tensor core's accumulation rounding, which was
// measured to lose low bits), and levels >= 3 together (their FP32 rounding
// is ~2^-21 x 2^-20 below the result). Every CTA contracts at most 256 k
// (KCHUNK), and longer K is split across CTAs whose FP64 partial sums a second
// kernel adds. The epilogue forms the FP64 result from the four FP32
// accumulators in integer arithmetic: levels 0-2 as exact integers, levels >= 3
// in units of 2^-35, summed in 64 bits and rounded once to FP64 by assembling
// its fields (FP64 conversions and adds would run on this part's FP64 pipe, 2
// per clock per SM). The digit cuts likewise read exponents and significands
// from the IEEE-754 fields with integer instructions.
//
// Layout: the digit planes of A (B) are cut once per GEMM by split_kernel into
// blocks of TM (TN) rows x 16 k per digit in the K-major core-matrix layout
// (tc_common.cuh), contiguous per (row tile, k slice); the GEMM kernel's
// producer thread moves a stage (D planes of A and of B) with two bulk copies
// (cp.async.bulk, completion on an mbarrier), one thread issues the
// tcgen05.mma of the stage and commits them to the stage's empty barrier, and
// all eight warps read the accumulators back (tcgen05.ld) in the epilogue.
// Every wait is bounded; a timeout sets an error flag the host reads.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <string>

#include "tc_common.cuh"
#include "tctl_internal.cuh"

namespace tctl {

namespace {

using namespace tc;

constexpr int TM = 128, TN = 64, NTHREADS = 256;
constexpr int KCHUNK = 256;               // contracted indices per CTA (exact levels 0..2)
constexpr int TMEM_COLS = 256;            // 4 accumulators of TN columns
constexpr int E_NONFINITE = 1 << 30;      // exponent code of a row / column holding Inf or NaN

__device__ __forceinline__ long long row_off(const TcOpnd &o, int r) {
  return (long long)(r % o.d) * o.s0 + (long long)(r / o.d) * o.s1;
}

// Row r of an operand: its two factor rows for the Khatri-Rao form, else one
// strided row (y unused).
struct RowPtr {
  const double *x, *y;
  __device__ __forceinline__ double at(long long k, long long sk, bool kr) const {
    return kr ? x[k * sk] * y[k * sk] : x[k * sk];
  }
};
__device__ __forceinline__ RowPtr row_ptr(const TcOpnd &o, int item, int r) {
  if (o.q) return RowPtr{o.p + (long long)(r % o.d) * o.s0, o.q + (long long)(r / o.d) * o.s1};
  return RowPtr{o.p + (long long)item * o.sb + row_off(o, r), nullptr};
}

// Row exponents, stored biased: e_out[item * Rpad + r] = E_BIAS + (smallest e
// with |X(r, k)| < 2^e for all k); 0 for an all-zero row (the buffer is
// zeroed first), E_NONFINITE if the row holds Inf/NaN. A block covers 32 rows
// x RE_K contracted indices and folds its maximum in with atomicMax, so long
// rows are spread over many blocks. Lanes run along whichever index is
// contiguous in memory.
constexpr int E_BIAS = 2000, RE_K = 256;

// The digit cuts and the epilogue work on the IEEE-754 fields of the FP64
// values with integer instructions: this part issues FP64 arithmetic and
// FP64 conversions at 2 per clock per SM, so a frexp / ldexp / double-to-int
// per element would bound these kernels by the FP64 pipe.

// Biased exponent code of v: E_BIAS + e with |v| in [2^(e-1), 2^e); 0 for zero,
// E_NONFINITE for Inf / NaN.
__device__ __forceinline__ int exp_code(double v) {
  const unsigned long long bits = (unsigned long long)__double_as_longlong(v);
  const int E = (int)((bits >> 52) & 0x7FF);
  const unsigned long long man = bits & 0xFFFFFFFFFFFFFull;
  if (E == 0x7FF) return E_NONFINITE;
  if (E == 0) {
    if (man == 0) return 0;
    return (63 - __clzll((long long)man)) - 1073 + E_BIAS;  // subnormal: man 2^-1074
  }
  return E - 1022 + E_BIAS;
}

// floor(|v| 2^(7D - e)) for |v| < 2^e: the 7D-bit fixed point of |v| / 2^e
// (truncated), from |v| = m 2^x with m the significand as an integer.
template <int D>
__device__ __forceinline__ unsigned long long fixed_point(double v, int e) {
  const unsigned long long bits = (unsigned long long)__double_as_longlong(v);
  const int E = (int)((bits >> 52) & 0x7FF);
  const unsigned long long man = bits & 0xFFFFFFFFFFFFFull;
  const unsigned long long m = E ? (man | (1ull << 52)) : man;
  const int x = E ? E - 1075 : -1074;
  const int sh = e - 7 * D - x;  // right shift
  unsigned long long F;
  if (sh >= 64) F = 0;
  else if (sh >= 0) F = m >> sh;
  else F = m << (-sh);  // a subnormal row: m < 2^(e - x), no overflow
  const unsigned long long cap = (1ull << (7 * D)) - 1;
  return F < cap ? F : cap;
}

// BF16 bits of s dg 2^(-7p), dg in [0, 127] (exact: at most 7 significant bits).
__device__ __forceinline__ uint32_t bf16_digit(uint32_t dg, int p, uint32_t sign) {
  if (dg == 0) return 0u;
  const int q = 31 - __clz((int)dg);  // leading bit, 0..6
  const uint32_t man = (dg << (7 - q)) & 0x7Fu;
  const uint32_t ex = (uint32_t)(127 + q - 7 * p);
  return (sign << 15) | (ex << 7) | man;
}

// t 2^sc as an FP64 number (t rounded to 53 bits, to nearest, ties to even),
// assembled from its fields; results outside the normal range take the FP64 route.
__device__ __forceinline__ double scaled_to_double(long long t, int sc) {
  if (t == 0) return 0.0;
  const unsigned long long u = t < 0 ? (unsigned long long)(-t) : (unsigned long long)t;
  int msb = 63 - __clzll((long long)u);
  unsigned long long mant;  // in [2^52, 2^53)
  if (msb > 52) {
    const int drop = msb - 52;
    mant = u >> drop;
    const unsigned long long rem = u & ((1ull << drop) - 1), half = 1ull << (drop - 1);
    if (rem > half || (rem == half && (mant & 1ull))) {
      ++mant;
      if (mant >> 53) {
        mant >>= 1;
        ++msb;
      }
    }
  } else {
    mant = u << (52 - msb);
  }
  const int ef = 1023 + msb + sc;
  if (ef <= 0 || ef >= 2047) return ldexp((double)t, sc);
  const unsigned long long bits = ((unsigned long long)(t < 0) << 63) |
                                  ((unsigned long long)ef << 52) | (mant & 0xFFFFFFFFFFFFFull);
  return __longlong_as_double((long long)bits);
}

// h 2^35 truncated toward zero, for |h| < 2^20 (FP32 fields; |h| < 2^-126 gives 0).
__device__ __forceinline__ long long fixed35(uint32_t hb) {
  const int E = (int)((hb >> 23) & 0xFF);
  if (E == 0) return 0;
  const long long M = (long long)((hb & 0x7FFFFFu) | 0x800000u);
  const int sh = E - 115;  // h 2^35 = M 2^(E - 150 + 35)
  const long long v = sh >= 0 ? (M << sh) : (sh > -32 ? (M >> (-sh)) : 0);
  return (hb >> 31) ? -v : v;
}

__device__ __forceinline__ void row_exp_body(const TcOpnd &o, int R, int K, int Rpad,
                                             int *__restrict__ e_out, int bx, int by, int item) {
  const int r0 = bx * 32, k0 = by * RE_K;
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;  // 8 warps
  const bool kr = o.q != nullptr;
  const int kend = min(K, k0 + RE_K);
  if (o.sk == 1) {
    // k contiguous: warp w takes rows r0 + w, r0 + w + 8, ...; lanes along k
    for (int rr = w; rr < 32; rr += 8) {
      const int r = r0 + rr;
      int c = 0;
      if (r < R) {
        const RowPtr x = row_ptr(o, item, r);
        for (int k = k0 + lane; k < kend; k += 32) c = max(c, exp_code(x.at(k, 1, kr)));
      }
      for (int s = 16; s > 0; s >>= 1) c = max(c, __shfl_xor_sync(0xffffffffu, c, s));
      if (lane == 0 && r < R && c > 0) atomicMax(&e_out[(long long)item * Rpad + r], c);
    }
  } else {
    // rows contiguous (or strided): lane = row, warp w takes k = k0 + w, k0 + w + 8, ...
    const int r = r0 + lane;
    int c = 0;
    if (r < R) {
      const RowPtr x = row_ptr(o, item, r);
      for (int k = k0 + w; k < kend; k += 8) c = max(c, exp_code(x.at(k, o.sk, kr)));
    }
    __shared__ int red[8][32];
    red[w][lane] = c;
    __syncthreads();
    if (w == 0) {
      for (int i = 1; i < 8; ++i) c = max(c, red[i][lane]);
      if (r < R && c > 0) atomicMax(&e_out[(long long)item * Rpad + r], c);
    }
  }
}

__global__ void row_exp_kernel(TcOpnd o, int R, int K, int Rpad, int *__restrict__ e_out) {
  row_exp_body(o, R, K, Rpad, e_out, blockIdx.x, blockIdx.y, blockIdx.z);
}

// Digit planes of one (row tile, 16-k slice) block: 2 TR threads, each cuts the
// D digits of 8 consecutive k of one row (one 16-byte core-matrix row per plane).
template <int D, int TR>
__device__ __forceinline__ void split_body(const TcOpnd &o, int R, int K, int Rpad, int nks,
                                           const int *__restrict__ e_in,
                                           __nv_bfloat16 *__restrict__ planes, int rt, int ks,
                                           int item) {
  const int t = threadIdx.x;
  int rl, kh;
  if (o.sk == 1) {
    rl = t >> 1;
    kh = t & 1;
  } else {
    rl = t % TR;
    kh = t / TR;
  }
  const int r = rt * TR + rl;
  const int k0 = ks * BK + kh * 8;
  const int ec = e_in[(long long)item * Rpad + r];
  const int e = ec - E_BIAS;
  uint32_t w[D][4];
#pragma unroll
  for (int p = 0; p < D; ++p)
#pragma unroll
    for (int h = 0; h < 4; ++h) w[p][h] = 0;
  if (r < R && ec != 0 && ec != E_NONFINITE) {
    const RowPtr x = row_ptr(o, item, r);
    const bool kr = o.q != nullptr;
#pragma unroll
    for (int i = 0; i < 8; ++i) {
      const int k = k0 + i;
      const double v = (k < K) ? x.at(k, o.sk, kr) : 0.0;
      const unsigned long long F = fixed_point<D>(v, e);  // 7D-bit fixed point (0 for v = 0)
      const uint32_t sg = (uint32_t)((unsigned long long)__double_as_longlong(v) >> 63);
#pragma unroll
      for (int p = 0; p < D; ++p) {
        const uint32_t dg = (uint32_t)((F >> (7 * (D - 1 - p))) & 127);
        w[p][i >> 1] |= bf16_digit(dg, p, sg) << (16 * (i & 1));
      }
    }
  }
  const int Rt = Rpad / TR;
  __nv_bfloat16 *blk = planes + (((long long)item * Rt + rt) * nks + ks) * D * (TR * BK);
  const uint32_t off = core_off(rl, kh * 8) / 2;
#pragma unroll
  for (int p = 0; p < D; ++p)
    *reinterpret_cast<uint4 *>(blk + p * (TR * BK) + off) = make_uint4(w[p][0], w[p][1], w[p][2], w[p][3]);
}

template <int D, int TR>
__global__ void __launch_bounds__(2 * TR) split_kernel(TcOpnd o, int R, int K, int Rpad, int nks,
                                                       const int *__restrict__ e_in,
                                                       __nv_bfloat16 *__restrict__ planes) {
  split_body<D, TR>(o, R, K, Rpad, nks, e_in, planes, blockIdx.x, blockIdx.y, blockIdx.z);
}

// Several operands' exponents / digit planes in one launch: operand i owns the
// blocks [b0[i], b0[i + 1]) of a one-dimensional grid, in (x, y) order.
constexpr int kSplitGroupMax = 4;
struct SplitItem {
  TcOpnd o;
  int R, K, Rpad, nks;
  int *e;
  __nv_bfloat16 *planes;
};
struct SplitGroup {
  int count;
  int b0[kSplitGroupMax + 1];
  SplitItem it[kSplitGroupMax];
};

__global__ void row_exp_group_kernel(SplitGroup g) {
  int i = 0;
  while (i + 1 < g.count && (int)blockIdx.x >= g.b0[i + 1]) ++i;
  const SplitItem &q = g.it[i];
  const int local = blockIdx.x - g.b0[i], gx = (q.R + 31) / 32;
  row_exp_body(q.o, q.R, q.K, q.Rpad, q.e, local % gx, local / gx, 0);
}

template <int D, int TR>
__global__ void __launch_bounds__(2 * TR) split_group_kernel(SplitGroup g) {
  int i = 0;
  while (i + 1 < g.count && (int)blockIdx.x >= g.b0[i + 1]) ++i;
  const SplitItem &q = g.it[i];
  const int local = blockIdx.x - g.b0[i], gx = q.Rpad / TR;
  split_body<D, TR>(q.o, q.R, q.K, q.Rpad, q.nks, q.e, q.planes, local % gx, local / gx, 0);
}

struct TcgArgs {
  int M, N, nks, nchunk, kst, divA, divB, Mt, Nt, Mpad, Npad;  // kst: 16-deep k steps per CTA
  const __nv_bfloat16 *pa, *pb;
  const int *ea, *eb;
  double alpha, beta;
  double *C;
  long long cm0, cm1, cj, cb;
  int cd;
  double *part;  // nchunk > 1: FP64 partial sums, [(b * nchunk + ch) * N + j] * M + m
  int *err;
  // failure-detection test: the producer withholds every copy, so the MMA
  // thread's wait for the first stage runs out after wait_ns
  int withhold;
  unsigned long long wait_ns;
};

// One CTA of a digit-split GEMM: output tile (mt, jt) of batch item / K chunk bz.
template <int D, int NST>
__device__ __forceinline__ void tcg_body(const TcgArgs &a, int mt, int jt, int bz) {
  constexpr int PA = TM * BK, PB = TN * BK;          // elements of one digit plane
  constexpr int A_BYTES = D * PA * 2, B_BYTES = D * PB * 2, STAGE = A_BYTES + B_BYTES;
  extern __shared__ __align__(1024) uint8_t smem_raw[];
  uint8_t *smem = reinterpret_cast<uint8_t *>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) &
                                              ~uintptr_t(1023));
  uint64_t *empty = reinterpret_cast<uint64_t *>(smem + NST * STAGE);
  uint64_t *full = empty + NST;
  uint64_t *done_bar = full + NST;
  uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(done_bar + 1);
  int *abort_flag = reinterpret_cast<int *>(tmem_slot + 1);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int b = bz / a.nchunk, ch = bz % a.nchunk;
  const int ia = b / a.divA, ib = b / a.divB;
  const int ks0 = ch * a.kst;
  const int nst = min(a.nks, ks0 + a.kst) - ks0;
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_u32(tmem_slot)),
                 "r"(TMEM_COLS));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  if (tid == 0) {
    for (int s = 0; s < NST; ++s) {
      asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(&empty[s])), "r"(1));
      asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(&full[s])), "r"(1));
    }
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(done_bar)), "r"(1));
    *abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;");
  }
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;");
  const uint32_t tmem = *tmem_slot;
  int issued = 0;  // stages whose bulk copies the producer started
  if (warp == 0 && lane == 0) {
    // producer: one bulk copy of the A digit block and one of the B block per stage
    const __nv_bfloat16 *asrc = a.pa + (((long long)ia * a.Mt + mt) * a.nks + ks0) * D * PA;
    const __nv_bfloat16 *bsrc = a.pb + (((long long)ib * a.Nt + jt) * a.nks + ks0) * D * PB;
    for (int s = 0; s < (a.withhold ? 0 : nst); ++s) {
      const int st = s % NST;
      if (s >= NST) {
        if (!mbar_wait(smem_u32(&empty[st]), (uint32_t)(((s - NST) / NST) & 1), a.wait_ns)) {
          atomicExch(abort_flag, 1);
          break;
        }
      }
      const uint32_t bar = smem_u32(&full[st]);
      const uint32_t dst = smem_u32(smem + st * STAGE);
      asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(STAGE));
      asm volatile(
          "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::
              "r"(dst),
          "l"(asrc + (long long)s * D * PA), "r"(A_BYTES), "r"(bar)
          : "memory");
      asm volatile(
          "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::
              "r"(dst + A_BYTES),
          "l"(bsrc + (long long)s * D * PB), "r"(B_BYTES), "r"(bar)
          : "memory");
      issued = s + 1;
    }
  } else if (warp == 1 && lane == 0) {
    // MMA issuer: kind::f16, BF16 x BF16 -> FP32, M = 128, N = 64
    const uint32_t idesc = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(TN >> 3) << 17) |
                           ((uint32_t)(TM >> 4) << 24);
    for (int s = 0; s < nst; ++s) {
      const int st = s % NST;
      if (!mbar_wait(smem_u32(&full[st]), (uint32_t)((s / NST) & 1), a.wait_ns)) {
        atomicExch(abort_flag, 1);
        break;
      }
      asm volatile("tcgen05.fence::after_thread_sync;");
      const uint32_t ab = smem_u32(smem + st * STAGE), bb = ab + A_BYTES;
#pragma unroll
      for (int p = 0; p < D; ++p) {
#pragma unroll
        for (int q = 0; q < D - p; ++q) {
          const uint64_t ad = smem_desc(ab + p * PA * 2);
          const uint64_t bd = smem_desc(bb + q * PB * 2);
          const int lvl = p + q < 3 ? p + q : 3;
          const uint32_t dst = tmem + (uint32_t)(TN * lvl);
          // the first product into each accumulator overwrites it
          const bool first = (s == 0) && (p == 0) && (q <= 3);
          const uint32_t acc = first ? 0u : 1u;
          asm volatile(
              "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
              " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(dst),
              "l"(ad), "l"(bd), "r"(idesc), "r"(acc));
        }
      }
      asm volatile(
          "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
              smem_u32(&empty[st])));
    }
    asm volatile(
        "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
            smem_u32(done_bar)));
  }
  const bool fin = mbar_wait(smem_u32(done_bar), 0u);
  const bool ok = (__syncthreads_and(fin ? 1 : 0) != 0) && (*abort_flag == 0) && nst > 0;
  if (!ok && nst > 0 && tid == 0) atomicExch(a.err, 1);
  if (!ok && warp == 0 && lane == 0) {
    // after an abort, bulk copies into stages the MMA thread never consumed may
    // still be landing: wait (bounded) for the last NST issued stages before the
    // CTA releases its shared memory (earlier stages completed before their
    // buffers were reissued)
    for (int s = max(0, issued - NST); s < issued; ++s)
      mbar_wait(smem_u32(&full[s % NST]), (uint32_t)((s / NST) & 1));
  }
  asm volatile("tcgen05.fence::after_thread_sync;");
  if (ok) {
    // warp w: TMEM lanes 32 (w % 4) .. +31 (rows), columns 32 (w / 4) .. +31, 16 at a time
    const int row = (warp & 3) * 32 + lane;
    const int m = mt * TM + row;
    const int ec = a.ea[(long long)ia * a.Mpad + min(m, a.Mpad - 1)];
#pragma unroll 1
    for (int half = 0; half < 2; ++half) {
      const int cb = (warp >> 2) * 32 + half * 16;
      uint32_t h0[16], h1[16], h2[16], h3[16];
      const uint32_t t0 = tmem + ((uint32_t)((warp & 3) * 32) << 16) + cb;
#define TCTL_LD16(dst, addr)                                                                     \
  asm volatile(                                                                                  \
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,"   \
      "%14,%15}, [%16];"                                                                         \
      : "=r"(dst[0]), "=r"(dst[1]), "=r"(dst[2]), "=r"(dst[3]), "=r"(dst[4]), "=r"(dst[5]),      \
        "=r"(dst[6]), "=r"(dst[7]), "=r"(dst[8]), "=r"(dst[9]), "=r"(dst[10]), "=r"(dst[11]),    \
        "=r"(dst[12]), "=r"(dst[13]), "=r"(dst[14]), "=r"(dst[15])                              \
      : "r"(addr))
      TCTL_LD16(h0, t0);
      TCTL_LD16(h1, t0 + TN);
      TCTL_LD16(h2, t0 + 2 * TN);
      if constexpr (D > 3) {
        TCTL_LD16(h3, t0 + 3 * TN);
      } else {
#pragma unroll
        for (int i = 0; i < 16; ++i) h3[i] = 0u;  // no level >= 3 with three digits
      }
#undef TCTL_LD16
      asm volatile("tcgen05.wait::ld.sync.aligned;");
      if (m < a.M) {
#pragma unroll
        for (int i = 0; i < 16; ++i) {
          const int j = jt * TN + cb + i;
          if (j >= a.N) break;
          const int fc = a.eb[(long long)ib * a.Npad + j];
          double v;
          if (ec == E_NONFINITE || fc == E_NONFINITE) v = __longlong_as_double(0x7FF8000000000000ll);
          else if (ec == 0 || fc == 0) v = 0.0;
          else {
            // levels 0..2 are exact integers in units of 2^-7L (below 2^24 units); the
            // levels >= 3 (below 2^3 in value) are taken in units of 2^-35: the sum
            // t (below 2^60) is exact and rounded once to FP64
            const long long l0 = __float2int_rn(__uint_as_float(h0[i]));
            const long long l1 = __float2int_rn(__uint_as_float(h1[i]) * 128.0f);
            const long long l2 = __float2int_rn(__uint_as_float(h2[i]) * 16384.0f);
            const long long l3 = fixed35(h3[i]);
            const long long t = l0 * 34359738368ll + l1 * 268435456ll + l2 * 2097152ll + l3;
            v = scaled_to_double(t, ec + fc - 2 * E_BIAS - 14 - 35);
          }
          if (a.nchunk == 1) {
            double *out = a.C + (long long)b * a.cb + (long long)(m % a.cd) * a.cm0 +
                          (long long)(m / a.cd) * a.cm1 + (long long)j * a.cj;
            if (a.beta == 0.0) *out = (a.alpha == 1.0) ? v : a.alpha * v;
            else *out = fma(a.alpha, v, a.beta * *out);
          } else {
            a.part[((long long)(b * a.nchunk + ch) * a.N + j) * a.M + m] = v;
          }
        }
      }
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TMEM_COLS));
}

template <int D, int NST>
__global__ void __launch_bounds__(NTHREADS, 2) tcg_kernel(TcgArgs a) {
  tcg_body<D, NST>(a, blockIdx.x, blockIdx.y, blockIdx.z);
}

// Several independent digit-split GEMMs in one launch: item i owns the CTAs
// [cta0[i], cta0[i + 1]) of a one-dimensional grid, in (mt, jt, bz) order.
constexpr int kTcgGroupMax = 4;
struct TcgGroup {
  int count;
  int cta0[kTcgGroupMax + 1];
  TcgArgs it[kTcgGroupMax];
};

template <int D, int NST>
__global__ void __launch_bounds__(NTHREADS, 2) tcg_group_kernel(TcgGroup g) {
  int item = 0;
  while (item + 1 < g.count && (int)blockIdx.x >= g.cta0[item + 1]) ++item;
  const TcgArgs &a = g.it[item];
  const int local = blockIdx.x - g.cta0[item];
  const int mt = local % a.Mt, rest = local / a.Mt;
  tcg_body<D, NST>(a, mt, rest % a.Nt, rest / a.Nt);
}

__global__ void tcg_reduce_kernel(int M, int N, int batch, int nchunk, const double *__restrict__ part,
                                  double alpha, double beta, double *C, long long cm0, long long cm1,
                                  int cd, long long cj, long long cb) {
  const long long total = (long long)M * N * batch;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < total;
       t += (long long)gridDim.x * blockDim.x) {
    const int m = (int)(t % M);
    const int j = (int)((t / M) % N);
    const int b = (int)(t / ((long long)M * N));
    double s = 0.0;
#pragma unroll 8
    for (int ch = 0; ch < nchunk; ++ch) s += part[((long long)(b * nchunk + ch) * N + j) * M + m];
    double *out = C + (long long)b * cb + (long long)(m % cd) * cm0 + (long long)(m / cd) * cm1 +
                  (long long)j * cj;
    *out = (beta == 0.0) ? alpha * s : fma(alpha, s, beta * *out);
  }
}

// the partial sums of the items of a group with K chunks (nchunk > 1)
struct TcgRedGroup {
  int count;
  long long out0[kTcgGroupMax + 1];
  const TcgArgs *dummy;
  TcgArgs it[kTcgGroupMax];
};

__global__ void tcg_reduce_group_kernel(TcgRedGroup g) {
  const long long total = g.out0[g.count];
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < total;
       t += (long long)gridDim.x * blockDim.x) {
    int item = 0;
    while (item + 1 < g.count && t >= g.out0[item + 1]) ++item;
    const TcgArgs &a = g.it[item];
    const long long r = t - g.out0[item];
    const int m = (int)(r % a.M);
    const int j = (int)((r / a.M) % a.N);
    const int b = (int)(r / ((long long)a.M * a.N));
    double sum = 0.0;
#pragma unroll 8
    for (int ch = 0; ch < a.nchunk; ++ch) sum += a.part[((long long)(b * a.nchunk + ch) * a.N + j) * a.M + m];
    double *out = a.C + (long long)b * a.cb + (long long)(m % a.cd) * a.cm0 + (long long)(m / a.cd) * a.cm1 +
                  (long long)j * a.cj;
    *out = (a.beta == 0.0) ? a.alpha * sum : fma(a.alpha, sum, a.beta * *out);
  }
}

template <int D, int NST>
constexpr int tcg_smem() {
  return NST * D * (TM + TN) * BK * 2 + 2048;
}

template <int D, int TR>
void split_operand(Ctx &c, const TcOpnd &o, int R, int K, int items, int Rpad, int nks, int *e,
                   __nv_bfloat16 *planes) {
  TCTL_CUDA(cudaMemsetAsync(e, 0, sizeof(int) * (size_t)items * Rpad, c.st));
  // algorithmic bytes: the operand's distinct elements once (a Khatri-Rao
  // operand: its two factors), the exponents, and the digit planes written
  const double in_bytes = o.q ? 8.0 * K * ((double)o.d + (double)R / o.d)
                              : 8.0 * (double)R * K * items;
  dim3 ge((R + 31) / 32, (K + RE_K - 1) / RE_K, items);
  c.next_bytes = in_bytes + 4.0 * items * Rpad;
  LAUNCH(c, row_exp_kernel, ge, 256, 0, o, R, K, Rpad, e);
  dim3 g(Rpad / TR, nks, items);
  c.next_bytes = in_bytes + 4.0 * items * Rpad + 2.0 * D * (double)items * Rpad * nks * BK;
  LAUNCH(c, (split_kernel<D, TR>), g, 2 * TR, 0, o, R, K, Rpad, nks, e, planes);
}

// Digit planes and row exponents of one operand: in the workspace, or for a
// kept operand (context-owned, constant) from the context's store, cut on
// first use.
template <int D, int TR>
void operand_planes(Ctx &c, const TcOpnd &o, int R, int K, int items, int Rpad, int nks, int *&e,
                    __nv_bfloat16 *&planes) {
  const size_t nplane = (size_t)items * (Rpad / TR) * nks * D * TR * BK;
  if (o.keep && items == 1 && !o.q) {
    for (const Ctx::TcKept &k : c.tc_keep)
      if (k.p == o.p && k.s0 == o.s0 && k.s1 == o.s1 && k.sk == o.sk && k.d == o.d && k.R == R &&
          k.K == K && k.D == D && k.TR == TR) {
        e = k.e;
        planes = static_cast<__nv_bfloat16 *>(k.planes);
        return;
      }
    e = reinterpret_cast<int *>(c.dmalloc(((size_t)Rpad + 1) / 2));
    planes = reinterpret_cast<__nv_bfloat16 *>(c.dmalloc((nplane * 2 + 7) / 8));
    split_operand<D, TR>(c, o, R, K, 1, Rpad, nks, e, planes);
    c.tc_keep.push_back(Ctx::TcKept{o.p, o.s0, o.s1, o.sk, o.d, R, K, D, TR, e, planes});
    return;
  }
  e = c.ws.i32((size_t)items * Rpad);
  planes = reinterpret_cast<__nv_bfloat16 *>(c.ws.dbl((nplane * 2 + 7) / 8));
  split_operand<D, TR>(c, o, R, K, items, Rpad, nks, e, planes);
}

// ---------------------------------------------------------------- tile autotuner
// The contracted length a CTA takes (kst 16-deep k steps: 64, 128 or 256 k)
// trades CTAs (parallelism of a sub-wave grid) against partial sums and the
// pipeline fill of short chunks. The first GEMM of each shape class, keyed by
// (digits, k steps, tile count bucket), times every candidate on the calling
// context's stream (CUDA events, best of two launches each, writing partial
// sums to scratch) and keeps the fastest for the process; later GEMMs of the
// class use the table. opts.tune = 0 keeps the fixed 256-deep chunks.
struct TuneEntry {
  int D, nks, tiles_log2;
  int kst;
  float ms[3];
};
std::mutex g_tune_mu;
std::vector<TuneEntry> g_tune;
constexpr int kTuneKst[3] = {4, 8, 16};

int tiles_bucket(long long tiles) {
  int b = 0;
  while ((1ll << (b + 1)) <= tiles && b < 30) ++b;
  return b;
}

template <int D, int NST>
int tcg_choose_kst(Ctx &c, int Mt, int Nt, int nks, int batch, int M, int N, const __nv_bfloat16 *pa,
                   const __nv_bfloat16 *pb, const int *ea, const int *eb, int Mpad, int Npad) {
  const int kfixed = KCHUNK / BK;
  if (!c.o.tune) return kfixed;
  const long long tiles = (long long)Mt * Nt * batch;
  const int tb = tiles_bucket(tiles);
  {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    for (const TuneEntry &t : g_tune)
      if (t.D == D && t.nks == nks && t.tiles_log2 == tb) return t.kst;
  }
  // time the candidates on this GEMM's own planes (results go to scratch partials)
  TuneEntry te{D, nks, tb, kfixed, {0, 0, 0}};
  size_t mk = c.ws.mark();
  double *part = c.ws.dbl((size_t)batch * ((nks + 3) / 4) * M * N);
  if (!c.tcg_err) {
    c.tcg_err = reinterpret_cast<int *>(c.dmalloc(1));
    TCTL_CUDA(cudaMemsetAsync(c.tcg_err, 0, sizeof(int), c.st));
  }
  cudaEvent_t e0, e1;
  TCTL_CUDA(cudaEventCreate(&e0));
  TCTL_CUDA(cudaEventCreate(&e1));
  float best = 1e30f;
  for (int ci = 0; ci < 3; ++ci) {
    const int kst = kTuneKst[ci];
    const int nchunk = (nks + kst - 1) / kst;
    if ((long long)batch * nchunk > 65535) {
      te.ms[ci] = -1;
      continue;
    }
    TcgArgs ar{};
    ar.M = M;
    ar.N = N;
    ar.nks = nks;
    ar.nchunk = nchunk;
    ar.kst = kst;
    ar.divA = 1;
    ar.divB = 1;
    ar.Mt = Mt;
    ar.Nt = Nt;
    ar.Mpad = Mpad;
    ar.Npad = Npad;
    ar.pa = pa;
    ar.pb = pb;
    ar.ea = ea;
    ar.eb = eb;
    ar.alpha = 1.0;
    ar.beta = 0.0;
    ar.C = part;  // only written when nchunk == 1: contiguous M x N x batch
    ar.cm0 = 1;
    ar.cm1 = 0;
    ar.cd = 1 << 30;
    ar.cj = M;
    ar.cb = (long long)M * N;
    ar.part = part;
    ar.err = c.tcg_err;
    ar.withhold = 0;
    ar.wait_ns = kWaitNs;
    dim3 grid(Mt, Nt, batch * nchunk);
    float ms = 1e30f;
    for (int rep = 0; rep < 2; ++rep) {
      TCTL_CUDA(cudaEventRecord(e0, c.st));
      tcg_kernel<D, NST><<<grid, NTHREADS, tcg_smem<D, NST>(), c.st>>>(ar);
      TCTL_CUDA(cudaGetLastError());
      c.launches++;
      TCTL_CUDA(cudaEventRecord(e1, c.st));
      TCTL_CUDA(cudaEventSynchronize(e1));
      float t = 0;
      TCTL_CUDA(cudaEventElapsedTime(&t, e0, e1));
      ms = std::min(ms, t);
    }
    // the partial sums' reduction, charged at its algorithmic bytes over the HBM rate
    if (nchunk > 1) ms += 0.004f + (float)(8.0 * (nchunk + 1) * (double)M * N * batch / 6.0e9);
    te.ms[ci] = ms;
    if (ms < best) {
      best = ms;
      te.kst = kst;
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  c.ws.reset(mk);
  std::lock_guard<std::mutex> lk(g_tune_mu);
  for (const TuneEntry &t : g_tune)
    if (t.D == D && t.nks == nks && t.tiles_log2 == tb) return t.kst;  // another thread's result
  g_tune.push_back(te);
  return te.kst;
}

template <int D, int NST>
void run_tcg(Ctx &c, int M, int N, int K, int batch, int divA, int divB, double alpha,
             const TcOpnd &A, const TcOpnd &B, double beta, double *C, long long cm0, long long cm1,
             int cd, long long cj, long long cb) {
  const int Mt = (M + TM - 1) / TM, Nt = (N + TN - 1) / TN;
  const int Mpad = Mt * TM, Npad = Nt * TN;
  const int nks = (K + BK - 1) / BK;
  const int itemsA = (batch - 1) / divA + 1, itemsB = (batch - 1) / divB + 1;
  size_t mk = c.ws.mark();
  int *ea = nullptr, *eb = nullptr;
  __nv_bfloat16 *pa = nullptr, *pb = nullptr;
  operand_planes<D, TM>(c, A, M, K, itemsA, Mpad, nks, ea, pa);
  operand_planes<D, TN>(c, B, N, K, itemsB, Npad, nks, eb, pb);
  // the attribute belongs to the function; a function-local static is set once, thread-safely
  static const cudaError_t attr = cudaFuncSetAttribute(
      tcg_kernel<D, NST>, cudaFuncAttributeMaxDynamicSharedMemorySize, tcg_smem<D, NST>());
  TCTL_CUDA(attr);
  const int kst = tcg_choose_kst<D, NST>(c, Mt, Nt, nks, batch, M, N, pa, pb, ea, eb, Mpad, Npad);
  const int nchunk = (nks + kst - 1) / kst;
  double *part = nchunk > 1 ? c.ws.dbl((size_t)batch * nchunk * M * N) : nullptr;
  if (!c.tcg_err) {
    c.tcg_err = reinterpret_cast<int *>(c.dmalloc(1));
    TCTL_CUDA(cudaMemsetAsync(c.tcg_err, 0, sizeof(int), c.st));
  }
  TcgArgs ar;
  ar.M = M;
  ar.N = N;
  ar.nks = nks;
  ar.nchunk = nchunk;
  ar.kst = kst;
  ar.divA = divA;
  ar.divB = divB;
  ar.Mt = Mt;
  ar.Nt = Nt;
  ar.Mpad = Mpad;
  ar.Npad = Npad;
  ar.pa = pa;
  ar.pb = pb;
  ar.ea = ea;
  ar.eb = eb;
  ar.alpha = alpha;
  ar.beta = beta;
  ar.C = C;
  ar.cm0 = cm0;
  ar.cm1 = cm1;
  ar.cj = cj;
  ar.cb = cb;
  ar.cd = cd;
  ar.part = part;
  ar.err = c.tcg_err;
  ar.withhold = 0;
  ar.wait_ns = kWaitNs;
  if (c.withhold_copies > 0) {
    // host-injected failure (tctl_inject_wait_timeout): a 1 ms limit on a
    // barrier nothing arrives on
    ar.withhold = 1;
    ar.wait_ns = 1000000ull;
    --c.withhold_copies;
  }
  dim3 grid(Mt, Nt, batch * nchunk);
  c.next_flops = 2.0 * M * (double)N * K * batch;
  c.next_mma = (D * (D + 1) / 2) * c.next_flops;  // digit products with p + q <= D - 1
  if (c.prof && c.trace) {
    // per-shape profile names (TCTL_TRACE=1 with profiling on)
    char nm[96];
    std::snprintf(nm, sizeof(nm), "tcg[%dx%dx%d b%d c%d]", M, N, K, batch, nchunk);
    c.next_tag = c.intern(nm);
  }
  constexpr int smem_bytes = tcg_smem<D, NST>();
  LAUNCH(c, (tcg_kernel<D, NST>), grid, NTHREADS, smem_bytes, ar);
  if (nchunk > 1) {
    const long long total = (long long)M * N * batch;
    const int blocks = (int)std::min<long long>((total + 255) / 256, 4096);
    c.next_bytes = 8.0 * total * (nchunk + 1 + (beta != 0.0));
    LAUNCH(c, tcg_reduce_kernel, blocks, 256, 0, M, N, batch, nchunk, part, alpha, beta, C, cm0, cm1,
           cd, cj, cb);
  }
  c.ws.reset(mk);
}

template <int D, int NST>
void run_tcg_group(Ctx &c, int count, const TcItem *items) {
  static const cudaError_t attr = cudaFuncSetAttribute(
      tcg_group_kernel<D, NST>, cudaFuncAttributeMaxDynamicSharedMemorySize, tcg_smem<D, NST>());
  TCTL_CUDA(attr);
  static const cudaError_t attr1 = cudaFuncSetAttribute(
      tcg_kernel<D, NST>, cudaFuncAttributeMaxDynamicSharedMemorySize, tcg_smem<D, NST>());
  TCTL_CUDA(attr1);
  if (!c.tcg_err) {
    c.tcg_err = reinterpret_cast<int *>(c.dmalloc(1));
    TCTL_CUDA(cudaMemsetAsync(c.tcg_err, 0, sizeof(int), c.st));
  }
  size_t mk = c.ws.mark();
  TcgGroup g;
  std::memset(&g, 0, sizeof(g));
  TcgRedGroup rg;
  std::memset(&rg, 0, sizeof(rg));
  g.count = count;
  int ctas = 0;
  double flops = 0;
  // digit planes: kept operands from the context's store (cut alone on first use),
  // the others collected and cut together: exponents zeroed by one memset, one
  // row-exponent launch, one split launch per tile height
  int *ea_[kTcgGroupMax], *eb_[kTcgGroupMax];
  __nv_bfloat16 *pa_[kTcgGroupMax], *pb_[kTcgGroupMax];
  std::vector<SplitItem> pend[2];  // [0]: TM-row tiles (A), [1]: TN-row tiles (B)
  auto prep = [&](const TcOpnd &o, int R, int K, int Rpad, int nks, bool isA, int *&e,
                  __nv_bfloat16 *&pl) {
    if (o.keep && !o.q) {
      if (isA) operand_planes<D, TM>(c, o, R, K, 1, Rpad, nks, e, pl);
      else operand_planes<D, TN>(c, o, R, K, 1, Rpad, nks, e, pl);
      return;
    }
    const size_t nplane = (size_t)Rpad * nks * D * BK;
    pl = reinterpret_cast<__nv_bfloat16 *>(c.ws.dbl((nplane * 2 + 7) / 8));
    e = nullptr;  // assigned below from one zeroed block
    pend[isA ? 0 : 1].push_back(SplitItem{o, R, K, Rpad, nks, nullptr, pl});
  };
  auto cut_pending = [&]() {
    size_t etot = 0;
    for (auto &v : pend)
      for (const SplitItem &q : v) etot += (size_t)q.Rpad;
    if (!etot) return;
    int *eblk = c.ws.i32(etot);
    TCTL_CUDA(cudaMemsetAsync(eblk, 0, sizeof(int) * etot, c.st));
    size_t off = 0;
    for (auto &v : pend)
      for (SplitItem &q : v) {
        q.e = eblk + off;
        off += (size_t)q.Rpad;
      }
    // hand the exponent arrays back to the items (matched by their plane buffers)
    for (int i = 0; i < count; ++i)
      for (auto &v : pend)
        for (const SplitItem &q : v) {
          if (q.planes == pa_[i]) ea_[i] = q.e;
          if (q.planes == pb_[i]) eb_[i] = q.e;
        }
    std::vector<SplitItem> all(pend[0]);
    all.insert(all.end(), pend[1].begin(), pend[1].end());
    for (size_t b = 0; b < all.size(); b += kSplitGroupMax) {
      SplitGroup sg;
      std::memset(&sg, 0, sizeof(sg));
      int blocks = 0;
      double bytes = 0;
      for (size_t i = b; i < std::min(all.size(), b + kSplitGroupMax); ++i) {
        const SplitItem &q = all[i];
        sg.it[sg.count] = q;
        sg.b0[sg.count] = blocks;
        blocks += ((q.R + 31) / 32) * ((q.K + RE_K - 1) / RE_K);
        bytes += (q.o.q ? 8.0 * q.K * ((double)q.o.d + (double)q.R / q.o.d) : 8.0 * (double)q.R * q.K) +
                 4.0 * q.Rpad;
        ++sg.count;
      }
      sg.b0[sg.count] = blocks;
      c.next_bytes = bytes;
      LAUNCH(c, row_exp_group_kernel, blocks, 256, 0, sg);
    }
    for (int h = 0; h < 2; ++h)
      for (size_t b = 0; b < pend[h].size(); b += kSplitGroupMax) {
        SplitGroup sg;
        std::memset(&sg, 0, sizeof(sg));
        int blocks = 0;
        double bytes = 0;
        const int TR = h == 0 ? TM : TN;
        for (size_t i = b; i < std::min(pend[h].size(), b + kSplitGroupMax); ++i) {
          const SplitItem &q = pend[h][i];
          sg.it[sg.count] = q;
          sg.b0[sg.count] = blocks;
          blocks += (q.Rpad / TR) * q.nks;
          bytes += (q.o.q ? 8.0 * q.K * ((double)q.o.d + (double)q.R / q.o.d) : 8.0 * (double)q.R * q.K) +
                   4.0 * q.Rpad + 2.0 * D * (double)q.Rpad * q.nks * BK;
          ++sg.count;
        }
        sg.b0[sg.count] = blocks;
        c.next_bytes = bytes;
        if (h == 0) LAUNCH(c, (split_group_kernel<D, TM>), blocks, 2 * TM, 0, sg);
        else LAUNCH(c, (split_group_kernel<D, TN>), blocks, 2 * TN, 0, sg);
      }
  };
  for (int i = 0; i < count; ++i) {
    const TcItem &q = items[i];
    const int Mt = (q.M + TM - 1) / TM, Nt = (q.N + TN - 1) / TN;
    const int Mpad = Mt * TM, Npad = Nt * TN, nks = (q.K + BK - 1) / BK;
    int *ea = nullptr, *eb = nullptr;
    __nv_bfloat16 *pa = nullptr, *pb = nullptr;
    prep(q.A, q.M, q.K, Mpad, nks, true, ea, pa);
    prep(q.B, q.N, q.K, Npad, nks, false, eb, pb);
    ea_[i] = ea;
    eb_[i] = eb;
    pa_[i] = pa;
    pb_[i] = pb;
  }
  cut_pending();
  for (int i = 0; i < count; ++i) {
    const TcItem &q = items[i];
    TcgArgs &ar = g.it[i];
    const int Mt = (q.M + TM - 1) / TM, Nt = (q.N + TN - 1) / TN;
    const int Mpad = Mt * TM, Npad = Nt * TN, nks = (q.K + BK - 1) / BK;
    int *ea = ea_[i], *eb = eb_[i];
    __nv_bfloat16 *pa = pa_[i], *pb = pb_[i];
    const int kst = tcg_choose_kst<D, NST>(c, Mt, Nt, nks, 1, q.M, q.N, pa, pb, ea, eb, Mpad, Npad);
    ar.M = q.M;
    ar.N = q.N;
    ar.nks = nks;
    ar.kst = kst;
    ar.nchunk = (nks + kst - 1) / kst;
    ar.divA = ar.divB = 1;
    ar.Mt = Mt;
    ar.Nt = Nt;
    ar.Mpad = Mpad;
    ar.Npad = Npad;
    ar.pa = pa;
    ar.pb = pb;
    ar.ea = ea;
    ar.eb = eb;
    ar.alpha = q.alpha;
    ar.beta = q.beta;
    ar.C = q.C;
    ar.cm0 = q.cm0;
    ar.cm1 = q.cm1;
    ar.cd = q.cd;
    ar.cj = q.cj;
    ar.cb = 0;
    ar.part = ar.nchunk > 1 ? c.ws.dbl((size_t)ar.nchunk * q.M * q.N) : nullptr;
    ar.err = c.tcg_err;
    ar.withhold = 0;
    ar.wait_ns = kWaitNs;
    if (c.withhold_copies > 0) {
      ar.withhold = 1;
      ar.wait_ns = 1000000ull;
      --c.withhold_copies;
    }
    g.cta0[i] = ctas;
    ctas += Mt * Nt * ar.nchunk;
    flops += 2.0 * q.M * (double)q.N * q.K;
  }
  g.cta0[count] = ctas;
  c.next_flops = flops;
  c.next_mma = (D * (D + 1) / 2) * flops;
  if (c.prof && c.trace) {
    std::string nm = "tcgroup[";
    for (int i = 0; i < count; ++i) {
      char b[64];
      std::snprintf(b, sizeof(b), "%s%dx%dx%d c%d", i ? " " : "", items[i].M, items[i].N, items[i].K,
                    g.it[i].nchunk);
      nm += b;
    }
    c.next_tag = c.intern((nm + "]").c_str());
  }
  constexpr int smem_bytes = tcg_smem<D, NST>();
  LAUNCH(c, (tcg_group_kernel<D, NST>), ctas, NTHREADS, smem_bytes, g);
  long long outs = 0;
  for (int i = 0; i < count; ++i)
    if (g.it[i].nchunk > 1) {
      rg.it[rg.count] = g.it[i];
      rg.out0[rg.count] = outs;
      outs += (long long)g.it[i].M * g.it[i].N;
      ++rg.count;
    }
  if (rg.count > 0) {
    rg.out0[rg.count] = outs;
    double bytes = 0;
    for (int i = 0; i < rg.count; ++i)
      bytes += 8.0 * rg.it[i].M * (double)rg.it[i].N * (rg.it[i].nchunk + 1 + (rg.it[i].beta != 0.0));
    c.next_bytes = bytes;
    const int blocks = (int)std::min<long long>((outs + 255) / 256, 4096);
    LAUNCH(c, tcg_reduce_group_kernel, blocks, 256, 0, rg);
  }
  c.ws.reset(mk);
}

}  // namespace

void gemm_tc_group(Ctx &c, int digits, int count, const TcItem *items) {
  for (int b = 0; b < count; b += kTcgGroupMax) {
    const int cnt = std::min(kTcgGroupMax, count - b);
    for (int i = b; i < b + cnt; ++i) {
      const TcItem &q = items[i];
      if (q.M <= 0 || q.N <= 0 || q.K <= 0) fail(TCTL_E_ARG, "gemm_tc_group: empty item");
      if ((q.M + TM - 1) / TM > 65535 || (q.N + TN - 1) / TN > 65535)
        fail(TCTL_E_ARG, "gemm_tc_group: item too large");
    }
    if (digits <= 3) run_tcg_group<3, 5>(c, cnt, items + b);
    else if (digits <= 4) run_tcg_group<4, 4>(c, cnt, items + b);
    else run_tcg_group<6, 3>(c, cnt, items + b);
  }
}

bool gemm_tc_fits(int M, int N, int K, int batch) {
  if (M <= 0 || N <= 0 || K <= 0 || batch <= 0) return false;
  const int Mt = (M + TM - 1) / TM, Nt = (N + TN - 1) / TN, nks = (K + BK - 1) / BK;
  const int nchunk = (nks + kTuneKst[0] - 1) / kTuneKst[0];  // the finest candidate chunking
  if (Nt > 65535 || (long long)batch * nchunk > 65535 || Mt > 65535) return false;
  // enough work to pay for the digit split, and tiles not mostly padding
  const double flops = 2.0 * M * (double)N * K * batch;
  const double padded = (double)Mt * TM * Nt * TN * nks * BK;
  return flops >= 2e7 && padded <= 4.0 * M * (double)N * K;
}

void gemm_tc(Ctx &c, int digits, int M, int N, int K, int batch, int divA, int divB, double alpha,
             const TcOpnd &A, const TcOpnd &B, double beta, double *C, long long cm0, long long cm1,
             int cd, long long cj, long long cb) {
  if (M <= 0 || N <= 0 || batch <= 0) return;
  if (K <= 0) fail(TCTL_E_ARG, "gemm_tc: K must be positive");
  if ((A.q || B.q) && batch != 1) fail(TCTL_E_ARG, "gemm_tc: a Khatri-Rao operand takes no batch");
  static_assert(TMEM_COLS >= 4 * TN, "four accumulators");
  if (digits <= 3)
    run_tcg<3, 5>(c, M, N, K, batch, divA, divB, alpha, A, B, beta, C, cm0, cm1, cd, cj, cb);
  else if (digits <= 4)
    run_tcg<4, 4>(c, M, N, K, batch, divA, divB, alpha, A, B, beta, C, cm0, cm1, cd, cj, cb);
  else
    run_tcg<6, 3>(c, M, N, K, batch, divA, divB, alpha, A, B, beta, C, cm0, cm1, cd, cj, cb);
}

void gemm_x(Ctx &c, int digits, bool ta, bool tb, int m, int n, int k, double alpha, const double *A,
            int lda, long long sA, const double *B, int ldb, long long sB, double beta, double *C,
            int ldc, long long sC, int batch, int divA, int divB, bool a_kept) {
  const bool use = digits > 0 && c.o.tc_gemm != 0;
  // a batch that reuses one operand (stride 0) splits it once
  if (sA == 0) divA = batch;
  if (sB == 0) divB = batch;
  // the larger of m, n goes to the 128-row side of the tile
  const bool swap = n > m;
  const int M = swap ? n : m, N = swap ? m : n;
  if (!use || !gemm_tc_fits(M, N, k, batch)) {
    gemm(c, ta, tb, m, n, k, alpha, A, lda, sA, B, ldb, sB, beta, C, ldc, sC, batch, divA, divB);
    return;
  }
  // op(A)(i, kk) = ta ? A[kk + i lda] : A[i + kk lda];  op(B)(kk, j) = tb ? B[j + kk ldb] : B[kk + j ldb]
  TcOpnd opA{A, ta ? (long long)lda : 1ll, 0ll, ta ? 1ll : (long long)lda, sA, 1 << 30};
  TcOpnd opB{B, tb ? 1ll : (long long)ldb, 0ll, tb ? (long long)ldb : 1ll, sB, 1 << 30};
  opA.keep = a_kept && batch == 1;
  if (!swap)
    gemm_tc(c, digits, m, n, k, batch, divA, divB, alpha, opA, opB, beta, C, 1, 0, 1 << 30, ldc, sC);
  else  // C^T = op(B)^T op(A)^T: rows j of op(B) become the 128-row operand
    gemm_tc(c, digits, n, m, k, batch, divB, divA, alpha, opB, opA, beta, C, ldc, 0, 1 << 30, 1, sC);
}

void gemm_tc_cm(Ctx &c, int digits, bool ta, bool tb, int m, int n, int k, double alpha,
                const double *A, int lda, const double *B, int ldb, double beta, double *C, int ldc) {
  if (m <= 0 || n <= 0) return;
  if (k <= 0) fail(TCTL_E_ARG, "k must be positive");
  if ((m + TM - 1) / TM > 65535 || (n + TN - 1) / TN > 65535)
    fail(TCTL_E_ARG, "matrix too large for one tensor-core GEMM launch");
  const TcOpnd opA{A, ta ? (long long)lda : 1ll, 0ll, ta ? 1ll : (long long)lda, 0, 1 << 30};
  const TcOpnd opB{B, tb ? 1ll : (long long)ldb, 0ll, tb ? (long long)ldb : 1ll, 0, 1 << 30};
  gemm_tc(c, digits, m, n, k, 1, 1, 1, alpha, opA, opB, beta, C, 1, 0, 1 << 30, ldc, 0);
}

void gemm_tc_kr(Ctx &c, int digits, int k, int ra, int rb, int n, double alpha, const double *X,
                int ldx, const double *Y, int ldy, const double *B, int ldb, double beta, double *C,
                int ldc) {
  const int m = ra * rb;
  if (m <= 0 || n <= 0) return;
  if (k <= 0) fail(TCTL_E_ARG, "k must be positive");
  if ((m + TM - 1) / TM > 65535 || (n + TN - 1) / TN > 65535)
    fail(TCTL_E_ARG, "matrix too large for one tensor-core GEMM launch");
  const TcOpnd kr{X, (long long)ldx, (long long)ldy, 1ll, 0, ra, Y};
  const TcOpnd opB{B, (long long)ldb, 0ll, 1ll, 0, 1 << 30};
  gemm_tc(c, digits, m, n, k, 1, 1, 1, alpha, kr, opB, beta, C, 1, 0, 1 << 30, ldc, 0);
}

std::string tune_report() {
  std::lock_guard<std::mutex> lk(g_tune_mu);
  std::string js = "[";
  for (size_t i = 0; i < g_tune.size(); ++i) {
    const TuneEntry &t = g_tune[i];
    char b[256];
    std::snprintf(b, sizeof(b),
                  "%s{\"digits\": %d, \"k_steps\": %d, \"tiles_log2\": %d, \"k_per_cta\": %d, "
                  "\"ms\": [%.5f, %.5f, %.5f]}",
                  i ? ", " : "", t.D, t.nks, t.tiles_log2, t.kst * BK, t.ms[0], t.ms[1], t.ms[2]);
    js += b;
  }
  return js + "]";
}

bool tcg_timed_out(Ctx &c) {
  if (!c.tcg_err) return false;
  int herr = 0;
  read_host(c, &herr, c.tcg_err, sizeof(int));
  if (herr) TCTL_CUDA(cudaMemsetAsync(c.tcg_err, 0, sizeof(int), c.st));
  return herr != 0;
}

void tcg_check(Ctx &c) {
  if (tcg_timed_out(c)) fail(TCTL_E_NUMERIC, "tensor-core GEMM: bounded mbarrier wait timed out");
}

}  // namespace tctl
