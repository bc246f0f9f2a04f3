// Full-grid mode products on the 5th-generation tensor cores (tcgen05, TMEM).
//
// A mode product of the n^3 grid tensor with an n x n matrix W (V_l^T forward,
// V_l back; Section 3.3, "DiagGen", "DiagFGen2D") is the GEMM
//     C[m, j] = sum_k W[m, k] X(k, j),   j = (j0, j1) the two other grid indices,
// with K = n. It is run in BF16 on the tensor cores with FP64-class accuracy by
// splitting the operands into five 7-bit signed digits that share one exponent
// per row of W (e_m) and per column of X (f_j) (the
// splitting of Ozaki et al.): W ~ 2^e_m sum_p t_p 2^-7p, X ~ 2^f_j sum_q s_q
// 2^-7q, |t_p|, |s_q| <= 127. Digit q is stored as the BF16 value s_q 2^-7(q-1)
// (exact: at most 7 significant bits). Products with p + q <= 6 (1-based) are
// kept (15 MMAs per 16-deep k-step) in three TMEM accumulators by digit level:
// level 0 (product of the leading digits: every partial sum is an integer
// below 127^2 K <= 2^24, K <= 1024, hence exact in FP32), level 1 (multiples
// of 2^-7 below 2^17: exact as well), and levels >= 2, whose FP32 rounding is
// 2^-14 below the result. Keeping the first two levels exact makes the result
// independent of how the tensor core rounds its FP32 accumulation.
// C = 2^(e_m + f_j - 14) (ACC_0 + ACC_1 + ACC_2). Truncation and the
// neglected digit products are of relative size ~2^-35 of the row / column
// maxima (an element far below its row or column maximum keeps fewer digits;
// the bound on the error of a product is 2^-35 n relative, 1.5e-8 at n = 512).
//
// Kernel structure: one CTA (8 warps) per SM computes a 128 x 128 tile of C
// (M = rows of W, N = 128 consecutive j) with K in 16-deep stages, four
// shared-memory stages of 40 KB. The digit planes of W (built once per
// context) and of X (cut once per mode product by x_digits_kernel) are stored
// in the tile layout, so one stage is two bulk copies (cp.async.bulk, completion
// counted on the stage's mbarrier) issued by one producer thread. One thread
// issues the 15 tcgen05.mma of a stage (M = 128, N = 128, K = 16, BF16 -> FP32,
// SWIZZLE_NONE K-major core matrices: 8 rows x 16 bytes, 128 B between K
// cores, 256 B between 8-row groups) into three TMEM accumulators of 128
// columns and commits them to the stage's empty barrier, which gates the next
// copy into it. At N = 128 an MMA reads 8 KB of shared memory per 128 x 128 x
// 16 product (N = 64 tiles were limited by shared-memory bandwidth: 52% vs
// 58% tensor-pipe activity measured). A persistent variant with two TMEM
// buffers (epilogue overlapped with the next tile) needs 6 x 128 columns for
// three accumulators, more than the 512 of an SM; with two accumulators the
// FP32 accumulation error reached 1e-6 at n = 512, and at N = 64 it ran slower.
// The epilogue reads the accumulators with tcgen05.ld, scales, optionally
// divides by F2(lambda_i + lambda_j + lambda_k) (the spectral divide of the
// last forward product), and stores FP32. Every mbarrier wait is bounded; on
// timeout the CTA records an error flag, skips its stores and frees TMEM.
#include <cuda_bf16.h>

#include <algorithm>
#include <cmath>

#include "tctl_internal.cuh"

namespace tctl {

namespace {

constexpr int TM = 128, TN = 128, BK = 16, NSTAGE = 4;
constexpr int NPLANE = 5;                                    // digits of W
constexpr int XPLANE = 5;                                    // digits of X
constexpr int NTHREADS = 256;  // 8 warps: producer, MMA issuer, all in the epilogue
constexpr int PLANE_ELEMS = TM * BK;                         // W plane: 2048 bf16 = 4 KB
constexpr int XPLANE_ELEMS = TN * BK;                        // X plane: 2048 bf16 = 4 KB
constexpr int W_BYTES = NPLANE * PLANE_ELEMS * 2;            // 20 KB per stage
constexpr int X_BYTES = XPLANE * XPLANE_ELEMS * 2;           // 20 KB per stage
constexpr int STAGE_BYTES = W_BYTES + X_BYTES;               // 40 KB
constexpr int SMEM_BYTES = NSTAGE * STAGE_BYTES + 2048;      // 162 KB: one CTA per SM
constexpr int TMEM_COLS = 512;                               // 3 accumulators of TN columns
constexpr int XD_KS = 2;                                     // K slices per x_digits block
constexpr uint32_t LBO = 128, SBO = (BK / 8) * 128;          // bytes

__device__ __forceinline__ uint32_t smem_u32(const void *p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ uint64_t smem_desc(uint32_t saddr) {
  uint64_t d = 0;
  d |= (uint64_t)((saddr & 0x3FFFF) >> 4);
  d |= (uint64_t)((LBO >> 4) & 0x3FFF) << 16;
  d |= (uint64_t)((SBO >> 4) & 0x3FFF) << 32;
  d |= (uint64_t)1 << 46;  // descriptor version for tcgen05; SWIZZLE_NONE, base offset 0
  return d;
}

// byte offset of element (r, k) of a 128 x 32 K-major tile in the core-matrix layout
__device__ __forceinline__ uint32_t core_off(int r, int k) {
  return (uint32_t)((r >> 3) * SBO + (k >> 3) * LBO + (r & 7) * 16 + (k & 7) * 2);
}

// Bounded wait on an mbarrier phase: false after 1 s (global timer) or 2^24
// polls without the phase completing; the caller records an error instead of
// hanging.
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity) {
  constexpr unsigned long long kLimitNs = 1000000000ull;
  unsigned long long t0, t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t0));
  for (uint32_t it = 0; it < (1u << 24); ++it) {
    uint32_t done;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
        " selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(done)
        : "r"(bar), "r"(parity));
    if (done) return true;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    if (t - t0 > kLimitNs) return false;
  }
  return false;
}

// Five 7-bit digits (35-bit fixed point, truncated) of |x| / 2^f for |x| < 2^f,
// x given as FP32 bits; all digits carry the sign of x.
__device__ __forceinline__ void digits_f32(uint32_t bits, int f, int d[XPLANE], float &sgn) {
  const int E = (int)((bits >> 23) & 0xFF);
  sgn = (bits >> 31) ? -1.0f : 1.0f;
#pragma unroll
  for (int q = 0; q < XPLANE; ++q) d[q] = 0;
  if (E == 0) return;  // zero or subnormal
  const uint64_t M = (uint64_t)((bits & 0x7FFFFFu) | 0x800000u);  // 24-bit significand
  // |x| / 2^f = M 2^(E - 150 - f); F = |x| 2^(35 - f) = (M << 11) >> (f - 1 - (E - 127))
  const int sh = f - 1 - (E - 127);
  if (sh >= 35 || sh < 0) return;
  const uint64_t F = (M << 11) >> sh;
  d[0] = (int)((F >> 28) & 127);
  d[1] = (int)((F >> 21) & 127);
  d[2] = (int)((F >> 14) & 127);
  d[3] = (int)((F >> 7) & 127);
  d[4] = (int)(F & 127);
}

__device__ __forceinline__ float pow2i(int e) {
  // 2^e for -126 <= e <= 127, 0 below (exact)
  return e < -126 ? 0.0f : __int_as_float((e + 127) << 23);
}

// ---------------------------------------------------------------- W digits
// W[m, k] = trans ? V[k + m n] : V[m + k n] (V column-major FP64). Row exponent
// e_m with max_k |W[m, k]| < 2^e_m; five digit planes stored per (M tile, K
// slice) block in the core-matrix layout so that a stage copies 4 x 8 KB.
__global__ void w_digits_kernel(int n, const double *__restrict__ V, int trans,
                                __nv_bfloat16 *__restrict__ planes, int *__restrict__ e_row) {
  const int m = blockIdx.x;
  __shared__ int s_e;
  int emax = -1000;
  for (int k = threadIdx.x; k < n; k += blockDim.x) {
    const double w = trans ? V[k + (long long)m * n] : V[m + (long long)k * n];
    if (w != 0.0) {
      int e;
      frexp(w, &e);  // |w| < 2^e
      emax = max(emax, e);
    }
  }
  for (int o = 16; o > 0; o >>= 1) emax = max(emax, __shfl_xor_sync(0xffffffffu, emax, o));
  if (threadIdx.x == 0) s_e = -1000;
  __syncthreads();
  if ((threadIdx.x & 31) == 0) atomicMax(&s_e, emax);
  __syncthreads();
  const int e = s_e;
  if (threadIdx.x == 0) e_row[m] = e;
  const int mt = m / TM, ml = m % TM, nks = n / BK;
  for (int k = threadIdx.x; k < n; k += blockDim.x) {
    const double w = trans ? V[k + (long long)m * n] : V[m + (long long)k * n];
    // 35-bit fixed point of |w| / 2^e (truncation), five 7-bit digits
    const double a = ldexp(fabs(w), 35 - e);
    const uint64_t F = (uint64_t)fmin(a, 34359738367.0);
    const float sg = w < 0.0 ? -1.0f : 1.0f;
    const int ks = k / BK, kl = k % BK;
    const long long blk = ((long long)mt * nks + ks) * NPLANE;
    const uint32_t off = core_off(ml, kl) / 2;  // in elements
    for (int p = 0; p < NPLANE; ++p) {
      const int dg = (int)((F >> (7 * (NPLANE - 1 - p))) & 127);
      const float v = sg * (float)dg * exp2f(-7.0f * p);
      planes[(blk + p) * PLANE_ELEMS + off] = __float2bfloat16_rn(v);
    }
  }
}

// ---------------------------------------------------------------- column exponents
// f_j with max_k |X(k, j)| < 2^f_j; X(k, j) at k sk + j0 sj0 + j1 sj1, j = j0 + n j1.
__global__ void col_exp_kernel(int n, const float *__restrict__ X, long long sk, long long sj0,
                               long long sj1, int *__restrict__ f) {
  const long long nj = (long long)n * n;
  if (sk == 1) {
    // contiguous along k: one warp per column
    const int lane = threadIdx.x & 31;
    for (long long j = (blockIdx.x * (long long)blockDim.x + threadIdx.x) / 32; j < nj;
         j += (long long)gridDim.x * blockDim.x / 32) {
      const long long base = (j % n) * sj0 + (j / n) * sj1;
      uint32_t mx = 0;
      for (int k = lane; k < n; k += 32) mx = max(mx, __float_as_uint(X[base + k]) & 0x7FFFFFFFu);
      for (int o = 16; o > 0; o >>= 1) mx = max(mx, __shfl_xor_sync(0xffffffffu, mx, o));
      if (lane == 0) f[j] = mx ? (int)((mx >> 23) & 0xFF) - 127 + 1 : -200;
    }
  } else {
    for (long long j = blockIdx.x * (long long)blockDim.x + threadIdx.x; j < nj;
         j += (long long)gridDim.x * blockDim.x) {
      const long long base = (j % n) * sj0 + (j / n) * sj1;
      uint32_t mx = 0;
      for (int k = 0; k < n; ++k) mx = max(mx, __float_as_uint(X[base + k * sk]) & 0x7FFFFFFFu);
      f[j] = mx ? (int)((mx >> 23) & 0xFF) - 127 + 1 : -200;
    }
  }
}

// ---------------------------------------------------------------- the GEMM
struct TcArgs {
  int n;
  const __nv_bfloat16 *wplanes;
  const int *e_row;
  const __nv_bfloat16 *xplanes;  // X digit blocks (x_digits_kernel)
  long long sk, sj0, sj1;  // input strides
  long long sm;            // output stride of m (j strides as the input)
  const int *f_col;
  float *C;
  // optional spectral factor at s = l_m[m] + l_0[j0] + l_1[j1]:
  // divide = 1: C /= s^-alpha + beta s^alpha;  divide = 2: C *= s^-alpha
  int divide;
  const double *lm, *l0, *l1;
  float alpha, beta;
  int *err;
};

// ---------------------------------------------------------------- X digits
// Cuts the five digit planes of X once per mode product, in the tile layout
// of the GEMM: block (jt, ks) holds, for the TN columns j of tile jt and the
// BK contracted indices of slice ks, five TN x BK BF16 planes in the K-major
// core-matrix layout (10 KB, contiguous). One CTA handles XD_KS consecutive
// slices of one tile; the column exponents f_j come from col_exp_kernel. Each
// thread owns one column j and 8 consecutive k (one 16-byte core-matrix row per
// plane), so the shared staging stores are 16-byte and conflict-free; the
// blocks are then copied out with coalesced 16-byte stores.
__global__ void __launch_bounds__(512) x_digits_kernel(int n, const float *__restrict__ X,
                                                       long long sk, long long sj0, long long sj1,
                                                       const int *__restrict__ f_col,
                                                       __nv_bfloat16 *__restrict__ planes) {
  __shared__ __align__(16) uint8_t st[XD_KS * X_BYTES];
  const int ksg = blockIdx.x, jt = blockIdx.y;
  const long long jbase = (long long)jt * TN;
  const int j1 = (int)(jbase / n), j0s = (int)(jbase % n);
  // work item: (jl, kg) with kg the group of 8 consecutive k within XD_KS slices
  constexpr int KG = XD_KS * BK / 8;  // 8
  const int t = threadIdx.x;
  int jl, kg;
  if (sk == 1) { kg = t % KG; jl = t / KG; } else { jl = t % TN; kg = t / TN; }
  const int f = f_col[jbase + jl];
  uint32_t w[XPLANE][4];
#pragma unroll
  for (int q = 0; q < XPLANE; ++q)
#pragma unroll
    for (int h = 0; h < 4; ++h) w[q][h] = 0;
  const long long base = (long long)(j0s + jl) * sj0 + (long long)j1 * sj1;
#pragma unroll
  for (int e = 0; e < 8; ++e) {
    const int k = ksg * XD_KS * BK + kg * 8 + e;
    const float x = X[base + (long long)k * sk];
    int d[XPLANE];
    float sg;
    digits_f32(__float_as_uint(x), f, d, sg);
#pragma unroll
    for (int q = 0; q < XPLANE; ++q) {
      const __nv_bfloat16 b = __float2bfloat16_rn(sg * (float)d[q] * pow2i(-7 * q));
      const uint32_t bits = (uint32_t)__bfloat16_as_ushort(b);
      w[q][e >> 1] |= bits << (16 * (e & 1));
    }
  }
  const int ksl = kg / (BK / 8), kin = (kg % (BK / 8)) * 8;
  const uint32_t off = core_off(jl, kin);
#pragma unroll
  for (int q = 0; q < XPLANE; ++q)
    *reinterpret_cast<uint4 *>(st + ksl * X_BYTES + q * XPLANE_ELEMS * 2 + off) =
        make_uint4(w[q][0], w[q][1], w[q][2], w[q][3]);
  __syncthreads();
  const int nks = n / BK;
  uint4 *dst = reinterpret_cast<uint4 *>(
      planes + ((long long)jt * nks + (long long)ksg * XD_KS) * XPLANE * XPLANE_ELEMS);
  const uint4 *src = reinterpret_cast<const uint4 *>(st);
  for (int e = threadIdx.x; e < XD_KS * X_BYTES / 16; e += blockDim.x) dst[e] = src[e];
}

// ---------------------------------------------------------------- the GEMM
// Pure tensor-core stage loop: every stage's W and X digit blocks (40 KB each,
// contiguous in global memory) are brought into shared memory by the
// bulk-copy engine (thread 0 of warp 0, completion counted on full[b]); one
// thread of warp 1 waits for them, issues the 30 tcgen05.mma of the stage and
// commits them to empty[b], which gates the next copy into the buffer.
__global__ void __launch_bounds__(NTHREADS, 1) tc_modeprod_kernel(TcArgs a) {
  extern __shared__ __align__(1024) uint8_t smem_raw[];
  uint8_t *smem = reinterpret_cast<uint8_t *>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) &
                                              ~uintptr_t(1023));
  uint64_t *empty = reinterpret_cast<uint64_t *>(smem + NSTAGE * STAGE_BYTES);
  uint64_t *full = empty + NSTAGE;
  uint64_t *done_bar = full + NSTAGE;
  uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(done_bar + 1);
  int *abort_flag = reinterpret_cast<int *>(tmem_slot + 1);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int n = a.n;
  const int mt = blockIdx.x;
  const int jt = blockIdx.y;
  const long long jbase = (long long)jt * TN;
  const int j1 = (int)(jbase / n);
  const int nks = n / BK;
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_u32(tmem_slot)),
                 "r"(TMEM_COLS));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  if (tid == 0) {
    for (int s = 0; s < NSTAGE; ++s) {
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
    // producer: bulk copies of the W and X digit blocks of each stage
    const __nv_bfloat16 *wsrc = a.wplanes + (long long)mt * nks * NPLANE * PLANE_ELEMS;
    const __nv_bfloat16 *xsrc = a.xplanes + (long long)jt * nks * XPLANE * XPLANE_ELEMS;
    for (int s = 0; s < nks; ++s) {
      const int b = s % NSTAGE;
      if (s >= NSTAGE) {
        const int t = s - NSTAGE;
        if (!mbar_wait(smem_u32(&empty[b]), (uint32_t)((t / NSTAGE) & 1))) {
          atomicExch(abort_flag, 1);
          break;
        }
      }
      const uint32_t bar = smem_u32(&full[b]);
      const uint32_t dst = smem_u32(smem + b * STAGE_BYTES);
      asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar),
                   "r"(STAGE_BYTES));
      asm volatile(
          "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::
              "r"(dst),
          "l"(wsrc + (long long)s * NPLANE * PLANE_ELEMS), "r"(W_BYTES), "r"(bar)
          : "memory");
      asm volatile(
          "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::
              "r"(dst + W_BYTES),
          "l"(xsrc + (long long)s * XPLANE * XPLANE_ELEMS), "r"(X_BYTES), "r"(bar)
          : "memory");
      issued = s + 1;
    }
  } else if (warp == 1 && lane == 0) {
    // MMA issuer
    const uint32_t idesc = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(TN >> 3) << 17) |
                           ((uint32_t)(TM >> 4) << 24);
    int s = 0;
    for (; s < nks; ++s) {
      const int b = s % NSTAGE;
      if (!mbar_wait(smem_u32(&full[b]), (uint32_t)((s / NSTAGE) & 1))) {
        atomicExch(abort_flag, 1);
        break;
      }
      asm volatile("tcgen05.fence::after_thread_sync;");
      const uint32_t wb = smem_u32(smem + b * STAGE_BYTES), xb = wb + W_BYTES;
      for (int t = 0; t < BK / 16; ++t) {
        for (int p = 0; p < NPLANE; ++p) {
          for (int q = 0; q < XPLANE; ++q) {
            if (p + q > 4) continue;  // digit pairs with p + q <= 4 (0-based): 15 products
            const uint64_t ad = smem_desc(wb + p * PLANE_ELEMS * 2 + t * 2 * LBO);
            const uint64_t bd = smem_desc(xb + q * XPLANE_ELEMS * 2 + t * 2 * LBO);
            // accumulator by digit level: 0 (exact integers), 1 (exact multiples of
            // 2^-7 below 2^17), >= 2 (FP32 rounding 2^-14 below the result)
            const int lvl = p + q < 2 ? p + q : 2;
            const uint32_t dst = tmem + (uint32_t)(TN * lvl);
            // the first product into each accumulator overwrites it
            const bool first = (s == 0 && t == 0) &&
                               ((p == 0 && q == 0) || (p == 0 && q == 1) || (p == 0 && q == 2));
            const uint32_t acc = first ? 0u : 1u;
            asm volatile(
                "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
                " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(dst),
                "l"(ad), "l"(bd), "r"(idesc), "r"(acc));
          }
        }
      }
      asm volatile(
          "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
              smem_u32(&empty[b])));
    }
    // completion of every MMA issued above (also after an abort, so that TMEM can be freed)
    asm volatile(
        "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
            smem_u32(done_bar)));
  }
  // everyone waits for the final commit (bounded)
  const bool fin = mbar_wait(smem_u32(done_bar), 0u);
  const bool ok = (__syncthreads_and(fin ? 1 : 0) != 0) && (*abort_flag == 0);
  if (!ok && tid == 0) atomicExch(a.err, 1);
  if (!ok && warp == 0 && lane == 0) {
    // after an abort, wait (bounded) for the bulk copies of the last NSTAGE
    // issued stages before the CTA releases its shared memory
    for (int s = max(0, issued - NSTAGE); s < issued; ++s)
      mbar_wait(smem_u32(&full[s % NSTAGE]), (uint32_t)((s / NSTAGE) & 1));
  }
  asm volatile("tcgen05.fence::after_thread_sync;");
  if (ok) {
    // warp w reads TMEM lanes 32 (w % 4) .. +31 (rows m), columns (TN / 2) (w / 4) .. +
    // TN / 2 - 1, 16 at a time
    const int row = (warp & 3) * 32 + lane;
    const int m = mt * TM + row;
    const int em = a.e_row[m];
#pragma unroll 1
    for (int half = 0; half < TN / 32; ++half) {
      const int cb = (warp >> 2) * (TN / 2) + half * 16;
      uint32_t hi[16], l1[16], rs[16];
      const uint32_t t0 = tmem + ((uint32_t)((warp & 3) * 32) << 16) + cb;
#define TCTL_LD16(dst, addr)                                                                     \
  asm volatile(                                                                                  \
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,"   \
      "%14,%15}, [%16];"                                                                         \
      : "=r"(dst[0]), "=r"(dst[1]), "=r"(dst[2]), "=r"(dst[3]), "=r"(dst[4]), "=r"(dst[5]),      \
        "=r"(dst[6]), "=r"(dst[7]), "=r"(dst[8]), "=r"(dst[9]), "=r"(dst[10]), "=r"(dst[11]),    \
        "=r"(dst[12]), "=r"(dst[13]), "=r"(dst[14]), "=r"(dst[15])                              \
      : "r"(addr))
      TCTL_LD16(hi, t0);
      TCTL_LD16(l1, t0 + TN);
      TCTL_LD16(rs, t0 + 2 * TN);
#undef TCTL_LD16
      asm volatile("tcgen05.wait::ld.sync.aligned;");
      const long long jb = jbase + cb;
      const int jj0 = (int)(jb % n);
      float *out = a.C + (long long)m * a.sm + (long long)jj0 * a.sj0 + (long long)j1 * a.sj1;
      const double lmj = a.divide ? a.lm[m] + a.l1[j1] : 0.0;
      float v[16];
#pragma unroll
      for (int i = 0; i < 16; ++i) {
        const int fj = a.f_col[jb + i];
        v[i] = ((__uint_as_float(hi[i]) + __uint_as_float(l1[i])) + __uint_as_float(rs[i])) *
               pow2i(em + fj - 14);
        if (a.divide) {
          const float pw = powf((float)(lmj + a.l0[jj0 + i]), a.alpha);
          v[i] = (a.divide == 1) ? v[i] / (1.0f / pw + a.beta * pw) : v[i] / pw;
        }
      }
      if (a.sj0 == 1) {
        // 16 contiguous floats: 16-byte stores
#pragma unroll
        for (int i = 0; i < 16; i += 4)
          *reinterpret_cast<float4 *>(out + i) = make_float4(v[i], v[i + 1], v[i + 2], v[i + 3]);
      } else {
#pragma unroll
        for (int i = 0; i < 16; ++i) out[(long long)i * a.sj0] = v[i];
      }
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem),
                 "r"(TMEM_COLS));
}

__global__ void f64_to_f32_kernel(long long count, const double *__restrict__ x, float *__restrict__ y) {
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < count;
       t += (long long)gridDim.x * blockDim.x)
    y[t] = (float)x[t];
}

__global__ void f32_to_f64_kernel(long long count, const float *__restrict__ x, double *__restrict__ y) {
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < count;
       t += (long long)gridDim.x * blockDim.x)
    y[t] = (double)x[t];
}

}  // namespace

bool tc_fullgrid_supported(int n) { return n >= 128 && n <= 1024 && n % 128 == 0; }  // (BK * XD_KS) | n

// u = (x V) [ ((x V^T) y) ./ F2(S) ] with all six mode products on the tensor cores.
void fullgrid_apply_tc(Ctx &c, const double *y, double *u, int which) {
  const int n = c.n;
  if (!tc_fullgrid_supported(n)) fail(TCTL_E_ARG, "tensor-core full grid needs n % 128 == 0, n <= 1024");
  const long long n2 = (long long)n * n, n3 = n2 * n;
  // digit planes of V_l^T (forward) and V_l (back), per mode, built once per context
  if (!c.tc_w[0]) {
    for (int l = 0; l < 3; ++l)
      for (int dir = 0; dir < 2; ++dir) {
        const int idx = 2 * l + dir;
        c.tc_w[idx] = reinterpret_cast<__nv_bfloat16 *>(c.dmalloc((n2 * NPLANE + 3) / 4));
        c.tc_e[idx] = reinterpret_cast<int *>(c.dmalloc((n + 1) / 2));
        LAUNCH(c, w_digits_kernel, n, 256, 0, n, c.V[l], dir == 0 ? 1 : 0, c.tc_w[idx],
               c.tc_e[idx]);
      }
    c.tc_x[0] = reinterpret_cast<float *>(c.dmalloc((size_t)(n3 + 1) / 2));
    c.tc_x[1] = reinterpret_cast<float *>(c.dmalloc((size_t)(n3 + 1) / 2));
    c.tc_f = reinterpret_cast<int *>(c.dmalloc((size_t)(n2 + 1) / 2));
    c.tc_xd = reinterpret_cast<__nv_bfloat16 *>(c.dmalloc((size_t)(n3 * XPLANE + 3) / 4));
    static_assert(XD_KS * X_BYTES <= 48 * 1024, "x_digits staging exceeds static shared memory");
    static_assert((TN * (XD_KS * BK / 8)) == 512, "x_digits work items must match its block");
    c.tc_err = reinterpret_cast<int *>(c.dmalloc(1));
    TCTL_CUDA(cudaFuncSetAttribute(tc_modeprod_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                   SMEM_BYTES));
  }
  TCTL_CUDA(cudaMemsetAsync(c.tc_err, 0, sizeof(int), c.st));
  float *A = c.tc_x[0], *B = c.tc_x[1];
  {
    const int blocks = (int)std::min<long long>((n3 + 255) / 256, 152 * 64);
    c.next_bytes = 12.0 * n3;
    LAUNCH(c, f64_to_f32_kernel, blocks, 256, 0, n3, y, A);
  }
  // strides of the three mode products (k = contracted index; j0, j1 the others)
  const long long sk[3] = {1, n, n2};
  const long long sj0[3] = {n, 1, 1};
  const long long sj1[3] = {n2, n2, n};
  auto pass = [&](int l, int dir, const float *X, float *C, int divide) {
    const int idx = 2 * l + dir;
    const int cblocks = (sk[l] == 1) ? (int)std::min<long long>(n2 * 32 / 256, 152 * 64)
                                     : (int)std::min<long long>((n2 + 255) / 256, 152 * 64);
    c.next_bytes = 4.0 * n3 + 4.0 * n2;
    LAUNCH(c, col_exp_kernel, cblocks, 256, 0, n, X, sk[l], sj0[l], sj1[l], c.tc_f);
    {
      dim3 g(n / (BK * XD_KS), (unsigned)(n2 / TN));
      c.next_bytes = 4.0 * n3 + 4.0 * n2 + 2.0 * XPLANE * n3;  // FP32 in, 5 BF16 digit planes out
      LAUNCH(c, x_digits_kernel, g, 512, 0, n, X, sk[l], sj0[l], sj1[l], c.tc_f, c.tc_xd);
    }
    TcArgs ar;
    ar.n = n;
    ar.wplanes = c.tc_w[idx];
    ar.e_row = c.tc_e[idx];
    ar.xplanes = c.tc_xd;
    ar.sk = sk[l];
    ar.sj0 = sj0[l];
    ar.sj1 = sj1[l];
    ar.sm = sk[l];
    ar.f_col = c.tc_f;
    ar.C = C;
    ar.divide = divide;
    // the divide happens after the mode-3 product: m = i3, j0 = i1, j1 = i2
    ar.lm = c.lam[2];
    ar.l0 = c.lam[0];
    ar.l1 = c.lam[1];
    ar.alpha = (float)c.alpha;
    ar.beta = (float)c.beta;
    ar.err = c.tc_err;
    dim3 grid(n / TM, (unsigned)(n2 / TN));
    c.next_flops = 2.0 * (double)n * (double)n2 * (double)n;  // one logical FP64-class GEMM
    c.next_mma = 15.0 * c.next_flops;                         // digit pairs with p + q <= 4
    LAUNCH(c, tc_modeprod_kernel, grid, NTHREADS, SMEM_BYTES, ar);
  };
  pass(0, 0, A, B, 0);
  pass(1, 0, B, A, 0);
  pass(2, 0, A, B, which == 0 ? 1 : 2);
  pass(0, 1, B, A, 0);
  pass(1, 1, A, B, 0);
  pass(2, 1, B, A, 0);
  {
    const int blocks = (int)std::min<long long>((n3 + 255) / 256, 152 * 64);
    c.next_bytes = 12.0 * n3;
    LAUNCH(c, f32_to_f64_kernel, blocks, 256, 0, n3, A, u);
  }
  int herr = 0;
  read_host(c, &herr, c.tc_err, sizeof(int));
  if (herr) fail(TCTL_E_NUMERIC, "tensor-core mode product: bounded mbarrier wait timed out");
}

}  // namespace tctl
