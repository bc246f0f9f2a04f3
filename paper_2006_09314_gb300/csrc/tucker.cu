// Rank-structured tensor algebra on the GPU (Appendix 1 of the paper):
// canonical-to-Tucker by reduced HOSVD of the side matrices, Tucker core
// truncation (HOSVD of the core), Tucker-to-canonical by slice SVDs, the
// Euclidean inner product, sums, and the Hadamard product with a separable
// diagonal operator followed by truncation (the fun/precond + trunc lines of
// Algorithm 1).
//
// Inside the solver a rank-truncated vector is kept in Tucker form
// (orthonormal Q_l, small dense core): the canonical form returned by
// Tucker-to-canonical has rank up to r^2, which would multiply the cost of
// the next Hadamard product; the Tucker form carries the same truncated
// tensor. Canonical tensors are converted at the API boundary.
//
// The Hadamard product D .* X of a rank-R separable diagonal D and a Tucker
// X has per-mode span inside span{e_k .* q_a}; its dominant mode-l subspace
// is found by a randomized range finder on the mode-l unfolding with
// Khatri-Rao-structured Gaussian probes (w_m x w_n per sample), which never
// forms the R*r columns; the core of D .* X in the new bases is then
// sum_k w_k core x_1 M_1k x_2 M_2k x_3 M_3k with M_lk = Q'_l^T diag(e_lk) Q_l,
// and the HOSVD of that core performs the eps truncation exactly (the bases
// are orthonormal, so Frobenius norms of the core are norms of the tensor).
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <numeric>

#include "tctl_internal.cuh"

namespace tctl {

namespace {

constexpr int kMaxRank = 64;
// The tensor-core GEMMs take c.digits digits (opts.tc_digits, default 6 = 42
// bits: the sketches must resolve directions down to the range tolerance, and
// the core feeds the eps truncation).

// The mode-2 and mode-3 unfoldings of a core in one pass (and, with o0, a copy):
// for in[a, b, c] (dims r0 x r1 x r2, first index fastest), o1[b, a, c] and
// o2[c, a, b] (dims r1 x r0 x r2 and r2 x r0 x r1).
__global__ void unfold3_kernel(int r0, int r1, int r2, const double *__restrict__ in,
                               double *__restrict__ o0, double *__restrict__ o1,
                               double *__restrict__ o2) {
  const long long total = (long long)r0 * r1 * r2;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < total;
       t += (long long)gridDim.x * blockDim.x) {
    const int a = (int)(t % r0), b = (int)((t / r0) % r1), cc = (int)(t / ((long long)r0 * r1));
    const double v = in[t];
    if (o0) o0[t] = v;
    o1[b + (long long)r1 * (a + (long long)r0 * cc)] = v;
    o2[cc + (long long)r2 * (a + (long long)r0 * b)] = v;
  }
}

void unfold3(Ctx &c, const int r[3], const double *in, double *o0, double *o1, double *o2) {
  const long long total = (long long)r[0] * r[1] * r[2];
  if (!total) return;
  const int blocks = (int)std::min<long long>((total + 255) / 256, 2048);
  c.next_bytes = 8.0 * total * (o0 ? 4 : 3);
  LAUNCH(c, unfold3_kernel, blocks, 256, 0, r[0], r[1], r[2], in, o0, o1, o2);
}

// out[a + ra*(s + ls*k)] = w[k] * sum_b F[(a + ra*b) + ra*rb*(s + ls*k)] * P[(b + rb*s) + rb*ls*k]
__global__ void contract_b_kernel(int ra, int rb, int ls, int K, const double *__restrict__ F,
                                  const double *__restrict__ P, const double *__restrict__ w,
                                  double *__restrict__ out) {
  const long long total = (long long)ra * ls * K;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < total;
       t += (long long)gridDim.x * blockDim.x) {
    const int a = (int)(t % ra);
    const long long sk = t / ra;  // s + ls*k
    const int k = (int)(sk / ls);
    const int s = (int)(sk % ls);
    const double *Fc = F + (long long)ra * rb * sk + a;
    const double *Pc = P + (long long)rb * ls * k + (long long)rb * s;
    double acc = 0.0;
    for (int b = 0; b < rb; ++b) acc = fma(Fc[(long long)ra * b], Pc[b], acc);
    out[t] = w[k] * acc;
  }
}

// Y[i, s] = sum_a Q[i, a] W[i, a + ra s] for s < ns: the Khatri-Rao
// contraction of W = B_l U^T with the factor Q (one thread per (i, s)).
__global__ void rowdot_kernel(int n, int ra, int ns, const double *__restrict__ Q, int ldq,
                              const double *__restrict__ W, int ldw, double *__restrict__ Y, int ldy) {
  const long long total = (long long)n * ns;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < total;
       t += (long long)gridDim.x * blockDim.x) {
    const int i = (int)(t % n), s = (int)(t / n);
    const double *w = W + i + (long long)ra * s * ldw;
    double acc = 0.0;
    for (int a = 0; a < ra; ++a) acc = fma(Q[i + (long long)a * ldq], w[(long long)a * ldw], acc);
    Y[i + (long long)s * ldy] = acc;
  }
}

// rowdot_kernel for the three modes of a sketch in one launch (ld = n throughout).
struct RowdotGroup {
  int count;
  int ra[3];
  const double *Q[3];
  const double *W[3];
  double *Y[3];
};

__global__ void rowdot_group_kernel(int n, int ns, RowdotGroup g) {
  const long long per = (long long)n * ns, total = per * g.count;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < total;
       t += (long long)gridDim.x * blockDim.x) {
    const int m = (int)(t / per);
    const long long u = t - per * m;
    const int i = (int)(u % n), s = (int)(u / n);
    const int ra = g.ra[m];
    const double *w = g.W[m] + i + (long long)ra * s * n;
    const double *q = g.Q[m] + i;
    double acc = 0.0;
    for (int a = 0; a < ra; ++a) acc = fma(q[(long long)a * n], w[(long long)a * n], acc);
    g.Y[m][i + (long long)s * n] = acc;
  }
}

__global__ void embed3_kernel(int a0, int a1, int a2, const double *__restrict__ in, int b0, int b1,
                              int b2, double scale, double *__restrict__ out) {
  // out (b0,b1,b2) zero-padded copy of scale*in (a0,a1,a2)
  const long long total = (long long)b0 * b1 * b2;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < total;
       t += (long long)gridDim.x * blockDim.x) {
    const int i = (int)(t % b0), j = (int)((t / b0) % b1), k = (int)(t / ((long long)b0 * b1));
    out[t] = (i < a0 && j < a1 && k < a2) ? scale * in[i + (long long)a0 * (j + (long long)a1 * k)]
                                          : 0.0;
  }
}

__global__ void dot_kernel(long long n, const double *__restrict__ x, const double *__restrict__ y,
                           double *out) {
  double s = 0.0;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < n;
       t += (long long)gridDim.x * blockDim.x)
    s = fma(x[t], y[t], s);
  __shared__ double red[32];
  for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x < 32) {
    s = (threadIdx.x < (blockDim.x >> 5)) ? red[threadIdx.x] : 0.0;
    for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
    if (threadIdx.x == 0) out[blockIdx.x] = s;
  }
}

double dot_host(Ctx &c, long long n, const double *x, const double *y) {
  if (n <= 0) return 0.0;
  const int blocks = (int)std::min<long long>((n + 255) / 256, 64);
  size_t mk = c.ws.mark();
  double *part = c.ws.dbl(blocks);
  LAUNCH(c, dot_kernel, blocks, 256, 0, n, x, y, part);
  std::vector<double> h(blocks);
  to_host(c, h.data(), part, blocks);
  c.ws.reset(mk);
  double s = 0.0;
  for (double v : h) s += v;
  if (!std::isfinite(s)) fail(TCTL_E_NAN, "non-finite inner product");
  return s;
}

__global__ void side_scale_kernel(int m, const double *__restrict__ w, const double *__restrict__ n0,
                                  const double *__restrict__ n1, const double *__restrict__ n2,
                                  int l, double *__restrict__ s) {
  for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < m; k += gridDim.x * blockDim.x) {
    const double nn[3] = {n0[k], n1[k], n2[k]};
    double v = fabs(w[k]);
    for (int q = 0; q < 3; ++q) {
      if (q != l) v *= nn[q];
    }
    s[k] = v;
  }
}

__global__ void gather_cols_kernel(int rows, const double *__restrict__ src, int lds,
                                   const int *__restrict__ idx, int count, double *__restrict__ dst,
                                   int ldd) {
  const long long total = (long long)rows * count;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < total;
       t += (long long)gridDim.x * blockDim.x) {
    const int i = (int)(t % rows), j = (int)(t / rows);
    dst[i + (long long)j * ldd] = src[i + (long long)idx[j] * lds];
  }
}

void gather_cols(Ctx &c, int rows, const double *src, int lds, const int *idx_dev, int count,
                 double *dst, int ldd) {
  const long long total = (long long)rows * count;
  if (!total) return;
  const int blocks = (int)std::min<long long>((total + 255) / 256, 4096);
  LAUNCH(c, gather_cols_kernel, blocks, 256, 0, rows, src, lds, idx_dev, count, dst, ldd);
}

// ttm along `mode`: out = core x_mode op(M), op(M) is p x r[mode]. If mt, M is stored as
// r[mode] x p (leading dim ldm) and op(M) = M^T; otherwise M is p x r[mode] (leading dim ldm).
void ttm(Ctx &c, const int r[3], const double *core, const double *M, int ldm, bool mt, int p,
         int mode, double *out) {
  if (mode == 0) {
    gemm(c, mt, false, p, r[1] * r[2], r[0], 1.0, M, ldm, 0, core, r[0], 0, 0.0, out, p, 0);
  } else if (mode == 1) {
    gemm(c, false, !mt, r[0], p, r[1], 1.0, core, r[0], (long long)r[0] * r[1], M, ldm, 0, 0.0,
         out, r[0], (long long)r[0] * p, r[2]);
  } else {
    gemm(c, false, !mt, r[0] * r[1], p, r[2], 1.0, core, r[0] * r[1], 0, M, ldm, 0, 0.0, out,
         r[0] * r[1], 0);
  }
}

// out[i, j, k] = sum_{a,b,c} A0(i, a) A1(j, b) A2(k, c) core[a, b, c] (the
// three mode products of a Tucker core in one launch): CTA k forms
// S = sum_c A2(k, c) core[:, :, c] (r0 x r1), then A0 S A1^T, in shared
// memory. A_l(x, y) = M_l[y + x ld_l] if transposed, else M_l[x + y ld_l].
struct Ttm3Args {
  const double *core;
  int r0, r1, r2;
  const double *M[3];
  int ld[3], tr[3];
  int p0, p1, p2;
  double *out;
};

// One output slab k per 4-CTA thread-block cluster. CTA c of the cluster takes
// the columns b in [b0, b1) of S = sum_c M2(k, c) core[:, :, c] (r0 x r1) and
// of T = A0 S (p0 x r1), and writes its columns of T into every CTA's copy
// through distributed shared memory; after one cluster barrier it forms the
// output rows j in [j0, j1) of out = T A1^T (p0 x p1). No work is repeated
// across the cluster, and a slab's FP64 work runs on four SMs.
constexpr int kTtmCluster = 4;

__global__ void __cluster_dims__(kTtmCluster, 1, 1) __launch_bounds__(256) ttm3_kernel(Ttm3Args g) {
  extern __shared__ double sm3[];
  const int crank = (int)cl_rank();
  const int k = blockIdx.x / kTtmCluster;
  const int r0 = g.r0, r1 = g.r1, r2 = g.r2, p0 = g.p0, p1 = g.p1;
  const int nbq = (r1 + kTtmCluster - 1) / kTtmCluster;
  const int b0 = min(r1, crank * nbq), b1 = min(r1, b0 + nbq), nb = b1 - b0;
  const int njq = (p1 + kTtmCluster - 1) / kTtmCluster;
  const int j0 = min(p1, crank * njq), j1 = min(p1, j0 + njq), nj = j1 - j0;
  double *T = sm3;                 // p0 x r1 (every CTA: the whole T)
  double *S = T + p0 * r1;         // r0 x nbq (this CTA's columns)
  double *A0 = S + r0 * nbq;       // p0 x r0
  double *A1 = A0 + p0 * r0;       // nj x r1 (this CTA's rows of op(M1))
  auto at = [&](int l, int x, int y) {
    return g.tr[l] ? g.M[l][y + (long long)x * g.ld[l]] : g.M[l][x + (long long)y * g.ld[l]];
  };
  for (int t = threadIdx.x; t < p0 * r0; t += blockDim.x) A0[t] = at(0, t % p0, t / p0);
  for (int t = threadIdx.x; t < nj * r1; t += blockDim.x) A1[t] = at(1, j0 + t % nj, t / nj);
  const long long slab = (long long)r0 * r1;
  for (int t = threadIdx.x; t < r0 * nb; t += blockDim.x) {
    const int a = t % r0, b = b0 + t / r0;
    double s = 0.0;
    for (int c = 0; c < r2; ++c) s = fma(at(2, k, c), g.core[a + (long long)r0 * b + c * slab], s);
    S[t] = s;
  }
  uint32_t tb[kTtmCluster];
#pragma unroll
  for (int q = 0; q < kTtmCluster; ++q) tb[q] = cl_map(T, (uint32_t)q);
  __syncthreads();
  for (int t = threadIdx.x; t < p0 * nb; t += blockDim.x) {
    const int i = t % p0, bl = t / p0;
    double s = 0.0;
    for (int a = 0; a < r0; ++a) s = fma(A0[i + a * p0], S[a + bl * r0], s);
    const uint32_t off = 8u * (uint32_t)(i + p0 * (b0 + bl));
#pragma unroll
    for (int q = 0; q < kTtmCluster; ++q) cl_st(tb[q] + off, s);
  }
  cl_sync();  // every CTA holds the whole T; no remote access after this
  double *o = g.out + (long long)p0 * p1 * k;
  for (int t = threadIdx.x; t < p0 * nj; t += blockDim.x) {
    const int i = t % p0, jl = t / p0;
    double s = 0.0;
    for (int b = 0; b < r1; ++b) s = fma(T[i + b * p0], A1[jl + b * nj], s);
    o[i + (long long)p0 * (j0 + jl)] = s;
  }
}

// core x_0 op(M0) x_1 op(M1) x_2 op(M2) -> out (p0 x p1 x p2); op(M_l) is p_l x r_l,
// stored transposed (r_l x p_l, ld) when tr_l. One fused launch while the
// shared-memory tiles fit, else three GEMM launches (ttm). t1, t2: scratch of
// the GEMM route (p0 r1 r2 and p0 p1 r2 doubles).
void ttm3(Ctx &c, const int r[3], const double *core, double *const M[3], const int ld[3],
          const bool tr[3], const int p[3], double *out, double *t1, double *t2) {
  const size_t nbq = (size_t)(r[1] + kTtmCluster - 1) / kTtmCluster;
  const size_t njq = (size_t)(p[1] + kTtmCluster - 1) / kTtmCluster;
  const size_t smem = sizeof(double) * ((size_t)p[0] * r[1] + (size_t)r[0] * nbq + (size_t)p[0] * r[0] +
                                        njq * r[1]);
  if (smem <= 96 * 1024 && p[2] > 0 && r[1] > 0) {
    static const cudaError_t attr =
        cudaFuncSetAttribute(ttm3_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, 96 * 1024);
    TCTL_CUDA(attr);
    Ttm3Args g{core, r[0], r[1], r[2], {M[0], M[1], M[2]}, {ld[0], ld[1], ld[2]},
               {tr[0] ? 1 : 0, tr[1] ? 1 : 0, tr[2] ? 1 : 0}, p[0], p[1], p[2], out};
    c.next_flops = 2.0 * p[2] * ((double)r[0] * r[1] * r[2] + (double)p[0] * r[0] * r[1] +
                                 (double)p[0] * p[1] * r[1]);
    c.next_bytes = 8.0 * ((double)r[0] * r[1] * r[2] + (double)p[0] * p[1] * p[2]);
    LAUNCH(c, ttm3_kernel, p[2] * kTtmCluster, 256, smem, g);
    return;
  }
  int rc[3] = {r[0], r[1], r[2]};
  ttm(c, rc, core, M[0], ld[0], tr[0], p[0], 0, t1);
  rc[0] = p[0];
  ttm(c, rc, t1, M[1], ld[1], tr[1], p[1], 1, t2);
  rc[1] = p[1];
  ttm(c, rc, t2, M[2], ld[2], tr[2], p[2], 2, out);
}

// Core of the truncated Hadamard product in the new bases, fused:
// out[a', b', c'] = sum_k w_k sum_{a,b,c} M0k(a', a) M1k(b', b) M2k(c', c) core[a, b, c],
// M_lk(x, y) = M_l[x + p_l y + p_l r_l k] (p_l x r_l per operator term k).
// CTA (c', q) sums the terms of k chunk q in shared memory (per term the
// mode-3 contraction first, then modes 1 and 2, as ttm3_kernel) and writes
// its partial sum; core_proj_reduce adds the chunks in a fixed order.
struct CoreProjArgs {
  const double *core;
  int r0, r1, r2, p0, p1, p2;
  const double *M[3];
  const double *w;
  int R, kchunk;
  double *part;  // [(q p2 + c') p0 p1 + a' + p0 b']
};

__global__ void __launch_bounds__(256) core_proj_kernel(CoreProjArgs g) {
  extern __shared__ double smc[];
  const int cp = blockIdx.x, q = blockIdx.y;
  const int r0 = g.r0, r1 = g.r1, r2 = g.r2, p0 = g.p0, p1 = g.p1, p2 = g.p2;
  double *S = smc;            // r0 x r1
  double *T = S + r0 * r1;    // p0 x r1
  double *acc = T + p0 * r1;  // p0 x p1
  for (int t = threadIdx.x; t < p0 * p1; t += blockDim.x) acc[t] = 0.0;
  const long long slab = (long long)r0 * r1;
  const int k0 = q * g.kchunk, k1 = min(g.R, k0 + g.kchunk);
  for (int k = k0; k < k1; ++k) {
    const double *M0 = g.M[0] + (long long)p0 * r0 * k;
    const double *M1 = g.M[1] + (long long)p1 * r1 * k;
    const double *M2 = g.M[2] + (long long)p2 * r2 * k;
    __syncthreads();  // acc / T of the previous term are complete
    for (int t = threadIdx.x; t < r0 * r1; t += blockDim.x) {
      double sacc = 0.0;
      for (int c = 0; c < r2; ++c) sacc = fma(M2[cp + (long long)p2 * c], g.core[t + c * slab], sacc);
      S[t] = sacc;
    }
    __syncthreads();
    for (int t = threadIdx.x; t < p0 * r1; t += blockDim.x) {
      const int i = t % p0, b = t / p0;
      double sacc = 0.0;
      for (int a = 0; a < r0; ++a) sacc = fma(M0[i + (long long)p0 * a], S[a + r0 * b], sacc);
      T[t] = sacc;
    }
    __syncthreads();
    const double wk = g.w[k];
    for (int t = threadIdx.x; t < p0 * p1; t += blockDim.x) {
      const int i = t % p0, j = t / p0;
      double sacc = 0.0;
      for (int b = 0; b < r1; ++b) sacc = fma(T[i + p0 * b], M1[j + (long long)p1 * b], sacc);
      acc[t] = fma(wk, sacc, acc[t]);
    }
  }
  __syncthreads();
  double *o = g.part + ((long long)q * p2 + cp) * p0 * p1;
  for (int t = threadIdx.x; t < p0 * p1; t += blockDim.x) o[t] = acc[t];
}

__global__ void core_proj_reduce(long long slab3, int chunks, const double *__restrict__ part,
                                 double *__restrict__ out) {
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < slab3;
       t += (long long)gridDim.x * blockDim.x) {
    double sacc = 0.0;
    for (int q = 0; q < chunks; ++q) sacc += part[t + q * slab3];
    out[t] = sacc;
  }
}

// The fused core projection for small ranks: its FP64 work per operator term,
// r0 r1 r2 + p0 r0 r1 + p0 p1 r1 FMAs, stays below 40k (ranks around 20, as in
// the PCG iterates); larger cores take the GEMM chain, whose last product runs
// on the tensor cores. False if the caller must use the chain.
bool core_proj(Ctx &c, const int r[3], const int p[3], const double *core, double *const M[3],
               const double *w, int R, double *out) {
  const size_t smem = sizeof(double) * ((size_t)r[0] * r[1] + (size_t)p[0] * r[1] + (size_t)p[0] * p[1]);
  const double per_term = (double)r[0] * r[1] * r[2] + (double)p[0] * r[0] * r[1] + (double)p[0] * p[1] * r[1];
  if (smem > 48 * 1024 || R <= 0 || per_term > 40000.0) return false;
  // the terms of one output slab in chunks so that the grid has about two CTAs per SM
  const int chunks = std::max(1, std::min(R, (2 * 152 + p[2] - 1) / p[2]));
  const int kchunk = (R + chunks - 1) / chunks;
  const int nq = (R + kchunk - 1) / kchunk;
  const long long slab3 = (long long)p[0] * p[1] * p[2];
  size_t mk = c.ws.mark();
  double *part = c.ws.dbl((size_t)slab3 * nq);
  CoreProjArgs g{core, r[0], r[1], r[2], p[0], p[1], p[2], {M[0], M[1], M[2]}, w, R, kchunk, part};
  c.next_flops = 2.0 * R * p[2] * ((double)r[0] * r[1] * r[2] + (double)p[0] * r[0] * r[1] +
                                   (double)p[0] * p[1] * r[1]);
  c.next_bytes = 8.0 * ((double)r[0] * r[1] * r[2] + (double)R * (p[0] * r[0] + p[1] * r[1] + p[2] * r[2]) +
                        (double)slab3 * nq);
  LAUNCH(c, core_proj_kernel, dim3(p[2], nq), 256, smem, g);
  const int blocks = (int)std::min<long long>((slab3 + 255) / 256, 4096);
  c.next_bytes = 8.0 * (double)slab3 * (nq + 1);
  LAUNCH(c, core_proj_reduce, blocks, 256, 0, slab3, nq, part, out);
  c.ws.reset(mk);
  return true;
}

int rank_from_tail(const std::vector<double> &lam_desc, double thr2) {
  // smallest r such that sum_{i >= r} max(lam_i, 0) <= thr2
  const int m = (int)lam_desc.size();
  double tail = 0.0;
  int r = m;
  for (int i = m - 1; i >= 0; --i) {
    const double v = std::max(lam_desc[i], 0.0);
    if (tail + v > thr2) break;
    tail += v;
    r = i;
  }
  return std::max(r, 1);
}

}  // namespace

void tucker_alloc(Ctx &c, Tucker &t, int cap) {
  t.cap = cap;
  for (int l = 0; l < 3; ++l) {
    t.Q[l] = c.ws.dbl((size_t)c.n * cap);
    t.r[l] = 0;
  }
  t.core = c.ws.dbl((size_t)cap * cap * cap);
}

void tucker_copy(Ctx &c, const Tucker &src, Tucker &dst) {
  for (int l = 0; l < 3; ++l) {
    dst.r[l] = src.r[l];
    copy_d(c, dst.Q[l], src.Q[l], (size_t)c.n * src.r[l]);
  }
  copy_d(c, dst.core, src.core, (size_t)src.r[0] * src.r[1] * src.r[2]);
}

static bool tucker_empty(const Tucker &x) { return x.r[0] == 0 || x.r[1] == 0 || x.r[2] == 0; }

void tucker_hosvd_trunc(Ctx &c, Tucker &x, double eps) {
  if (tucker_empty(x)) return;
  TCTL_PHASE(c, "hosvd");
  const int n = c.n;
  size_t mk = c.ws.mark();
  const int r[3] = {x.r[0], x.r[1], x.r[2]};
  const long long sz = (long long)r[0] * r[1] * r[2];
  double *perm1 = c.ws.dbl(sz), *perm2 = c.ws.dbl(sz);
  double *G[3], *lam[3], *U[3];
  std::vector<double> lh[3];
  double *lam_all = c.ws.dbl((size_t)r[0] + r[1] + r[2]);  // one read-back for the three modes
  unfold3(c, r, x.core, nullptr, perm1, perm2);
  {
    // Gram matrices of the three mode-l unfoldings (r_l x rest, ld r_l) in one launch
    const double *src[3] = {x.core, perm1, perm2};
    GemmSpec g[3];
    for (int l = 0; l < 3; ++l) {
      G[l] = c.ws.dbl((size_t)r[l] * r[l]);
      lam[l] = lam_all + (l == 0 ? 0 : l == 1 ? r[0] : r[0] + r[1]);
      U[l] = c.ws.dbl((size_t)r[l] * r[l]);
      g[l] = {false, true, r[l], r[l], (int)(sz / r[l]), 1.0, src[l], r[l], src[l], r[l], 0.0, G[l], r[l]};
    }
    gemm_group(c, 3, g);
  }
  sym_eig_multi(c, 3, r, G, lam, U);
  double tot = 0.0;
  {
    std::vector<double> all((size_t)r[0] + r[1] + r[2]);
    to_host(c, all.data(), lam_all, all.size());
    size_t o = 0;
    for (int l = 0; l < 3; ++l) {
      lh[l].assign(all.begin() + o, all.begin() + o + r[l]);
      o += r[l];
    }
  }
  for (double v : lh[0]) tot += std::max(v, 0.0);
  if (!std::isfinite(tot)) fail(TCTL_E_NAN, "non-finite core in truncation");
  if (tot == 0.0) {
    x.r[0] = x.r[1] = x.r[2] = 0;
    c.ws.reset(mk);
    return;
  }
  int rn[3];
  for (int l = 0; l < 3; ++l) rn[l] = rank_from_tail(lh[l], eps * eps * tot / 3.0);
  if (c.trace)
    std::fprintf(stderr, "[tctl] hosvd %s (%d,%d,%d) -> (%d,%d,%d)\n", c.outer ? c.outer : "-", r[0],
                 r[1], r[2], rn[0], rn[1], rn[2]);
  // new core = core x_l U_l[:, :rn]^T
  double *t1 = c.ws.dbl(sz), *t2 = c.ws.dbl(sz);
  {
    // the new core is written in place of the old one: through a separate buffer
    double *nc = c.ws.dbl((size_t)rn[0] * rn[1] * rn[2]);
    const int ldu[3] = {r[0], r[1], r[2]};
    const bool tr[3] = {true, true, true};
    ttm3(c, r, x.core, U, ldu, tr, rn, nc, t1, t2);
    copy_d(c, x.core, nc, (size_t)rn[0] * rn[1] * rn[2]);
  }
  // new factors Q_l U_l[:, :rn], the three modes in one launch
  {
    GemmSpec g[3];
    double *dst[3];
    const double *srcq[3];
    size_t cnt[3];
    for (int l = 0; l < 3; ++l) {
      double *Qt = c.ws.dbl((size_t)n * rn[l]);
      g[l] = {false, false, n, rn[l], r[l], 1.0, x.Q[l], n, U[l], r[l], 0.0, Qt, n};
      dst[l] = x.Q[l];
      srcq[l] = Qt;
      cnt[l] = (size_t)n * rn[l];
    }
    gemm_group(c, 3, g);
    copy_multi(c, 3, dst, srcq, cnt);
    for (int l = 0; l < 3; ++l) x.r[l] = rn[l];
  }
  c.ws.reset(mk);
}

double tucker_inner(Ctx &c, const Tucker &x, const Tucker &y) {
  if (tucker_empty(x) || tucker_empty(y)) return 0.0;
  TCTL_PHASE(c, "inner");
  const int n = c.n;
  size_t mk = c.ws.mark();
  double *M[3];
  {
    GemmSpec g[3];
    for (int l = 0; l < 3; ++l) {
      M[l] = c.ws.dbl((size_t)x.r[l] * y.r[l]);
      g[l] = {true, false, x.r[l], y.r[l], n, 1.0, x.Q[l], n, y.Q[l], n, 0.0, M[l], x.r[l]};
    }
    gemm_group(c, 3, g);
  }
  const long long big = (long long)std::max(x.r[0], y.r[0]) * std::max(x.r[1], y.r[1]) *
                        std::max(x.r[2], y.r[2]);
  double *t1 = c.ws.dbl(big), *t2 = c.ws.dbl(big), *t3 = c.ws.dbl(big);
  {
    const int ldm[3] = {x.r[0], x.r[1], x.r[2]};
    const bool tr[3] = {false, false, false};
    ttm3(c, y.r, y.core, M, ldm, tr, x.r, t3, t1, t2);
  }
  const double v = dot_host(c, (long long)x.r[0] * x.r[1] * x.r[2], x.core, t3);
  c.ws.reset(mk);
  return v;
}

void tucker_axpby_trunc(Ctx &c, double a, const Tucker &x, double b, const Tucker &y, Tucker &z,
                        double eps, double *norm_out, double keep_below) {
  // orthonormal bases throughout: the norm of the sum is the norm of its core
  auto finish = [&]() {
    if (norm_out) {
      const long long sz = (long long)z.r[0] * z.r[1] * z.r[2];
      *norm_out = std::sqrt(std::max(dot_host(c, sz, z.core, z.core), 0.0));
      if (*norm_out <= keep_below) return;
    }
    tucker_hosvd_trunc(c, z, eps);
  };
  const int n = c.n;
  if (tucker_empty(x) || a == 0.0) {
    tucker_copy(c, y, z);
    axpby(c, (size_t)y.r[0] * y.r[1] * y.r[2], b, y.core, 0.0, z.core);
    finish();
    return;
  }
  if (tucker_empty(y) || b == 0.0) {
    tucker_copy(c, x, z);
    axpby(c, (size_t)x.r[0] * x.r[1] * x.r[2], a, x.core, 0.0, z.core);
    finish();
    return;
  }
  TCTL_PHASE(c, "axpy");
  size_t mk = c.ws.mark();
  double *My[3];
  int rz[3];
  double *Qz[3], *Wl[3], *C1[3], *C2[3];
  for (int l = 0; l < 3; ++l) {
    C1[l] = c.ws.dbl((size_t)x.r[l] * y.r[l]);
    C2[l] = c.ws.dbl((size_t)x.r[l] * y.r[l]);
    Wl[l] = c.ws.dbl((size_t)n * y.r[l]);
    Qz[l] = c.ws.dbl((size_t)n * kMaxRank);
  }
  // W = Q_y - Q_x (Q_x^T Q_y), twice (block classical Gram-Schmidt with
  // reorthogonalisation), the three modes in one launch per step
  {
    GemmSpec g[3];
    double *dst[6];
    const double *src[6];
    size_t cnt[6];
    for (int l = 0; l < 3; ++l) {
      g[l] = {true, false, x.r[l], y.r[l], n, 1.0, x.Q[l], n, y.Q[l], n, 0.0, C1[l], x.r[l]};
      dst[l] = Wl[l];
      src[l] = y.Q[l];
      cnt[l] = (size_t)n * y.r[l];
      dst[3 + l] = Qz[l];
      src[3 + l] = x.Q[l];
      cnt[3 + l] = (size_t)n * x.r[l];
    }
    gemm_group(c, 3, g);
    copy_multi(c, 6, dst, src, cnt);
    for (int l = 0; l < 3; ++l)
      g[l] = {false, false, n, y.r[l], x.r[l], -1.0, x.Q[l], n, C1[l], x.r[l], 1.0, Wl[l], n};
    gemm_group(c, 3, g);
    for (int l = 0; l < 3; ++l)
      g[l] = {true, false, x.r[l], y.r[l], n, 1.0, x.Q[l], n, Wl[l], n, 0.0, C2[l], x.r[l]};
    gemm_group(c, 3, g);
    for (int l = 0; l < 3; ++l)
      g[l] = {false, false, n, y.r[l], x.r[l], -1.0, x.Q[l], n, C2[l], x.r[l], 1.0, Wl[l], n};
    gemm_group(c, 3, g);
  }
  // orthonormal complements of the three modes in one batched call
  {
    int ms[3], lds[3], caps[3], rw[3];
    double *Qw[3];
    for (int l = 0; l < 3; ++l) {
      ms[l] = y.r[l];
      lds[l] = n;
      caps[l] = std::max(0, kMaxRank - x.r[l]);
      Qw[l] = Qz[l] + (size_t)n * x.r[l];
    }
    orth_multi(c, 3, n, ms, Wl, lds, 1e-8, false, caps, Qw, rw);
    for (int l = 0; l < 3; ++l) rz[l] = x.r[l] + rw[l];
  }
  {
    // coordinates of Q_y in [Q_x | Q_w]: [C1 + C2 ; Q_w^T Q_y]
    GemmSpec g[3];
    for (int l = 0; l < 3; ++l) {
      My[l] = c.ws.dbl((size_t)rz[l] * y.r[l]);
      g[l] = {true, false, rz[l], y.r[l], n, 1.0, Qz[l], n, y.Q[l], n, 0.0, My[l], rz[l]};
    }
    gemm_group(c, 3, g);
  }
  const long long szz = (long long)rz[0] * rz[1] * rz[2];
  double *core = c.ws.dbl(szz);
  {
    const int blocks = (int)std::min<long long>((szz + 255) / 256, 2048);
    LAUNCH(c, embed3_kernel, blocks, 256, 0, x.r[0], x.r[1], x.r[2], x.core, rz[0], rz[1], rz[2], a,
           core);
  }
  double *t1 = c.ws.dbl(szz), *t2 = c.ws.dbl(szz), *t3 = c.ws.dbl(szz);
  {
    const int ldm[3] = {rz[0], rz[1], rz[2]};
    const bool tr[3] = {false, false, false};
    ttm3(c, y.r, y.core, My, ldm, tr, rz, t3, t1, t2);
  }
  axpby(c, (size_t)szz, b, t3, 1.0, core);
  {
    double *dst[4] = {z.Q[0], z.Q[1], z.Q[2], z.core};
    const double *src[4] = {Qz[0], Qz[1], Qz[2], core};
    size_t cnt[4] = {(size_t)n * rz[0], (size_t)n * rz[1], (size_t)n * rz[2], (size_t)szz};
    for (int l = 0; l < 3; ++l) z.r[l] = rz[l];
    copy_multi(c, 4, dst, src, cnt);
  }
  c.ws.reset(mk);
  finish();
}

void tucker_basis_change(Ctx &c, Tucker &x, bool to_eig) {
  tucker_factor_change(c, x, c.V, to_eig);
}

// Q_l <- M_l^T Q_l (transpose) or M_l Q_l; orthogonal M_l keep Q_l orthonormal.
void tucker_factor_change(Ctx &c, Tucker &x, double *const M[3], bool transpose) {
  const int n = c.n;
  size_t mk = c.ws.mark();
  double *t = c.ws.dbl((size_t)n * kMaxRank);
  for (int l = 0; l < 3; ++l) {
    if (!x.r[l]) continue;
    gemm(c, transpose, false, n, x.r[l], n, 1.0, M[l], n, 0, x.Q[l], n, 0, 0.0, t, n, 0);
    copy_d(c, x.Q[l], t, (size_t)n * x.r[l]);
  }
  c.ws.reset(mk);
}

// Y_l = op(V_l) X_l (n x m_l, contracted over the grid index) for the three
// modes: the boundary basis changes into and out of the eigenbasis (Section
// 3.3). With the tensor-core contractions they run as one grouped digit-split
// launch (6 digits; V_l's planes cut once per orientation and kept by the
// context) however narrow X_l is: the padded 128 x 64 tiles cost far less than
// the FP64 product on this part. FP64 otherwise.
static void basis_change3(Ctx &c, bool transpose_v, const int m[3], double *const X[3],
                          double *const Y[3]) {
  const int n = c.n;
  bool tc = c.o.tc_gemm != 0;
  for (int l = 0; l < 3 && tc; ++l) tc = m[l] <= 0 || ((n + 127) / 128 <= 65535 && m[l] <= 65535 * 64);
  if (!tc) {
    for (int l = 0; l < 3; ++l)
      if (m[l] > 0)
        gemm(c, transpose_v, false, n, m[l], n, 1.0, c.V[l], n, 0, X[l], n, 0, 0.0, Y[l], n, 0);
    return;
  }
  std::vector<TcItem> items;
  for (int l = 0; l < 3; ++l) {
    if (m[l] <= 0) continue;
    // op(V)(i, k) = transpose_v ? V[k + i n] : V[i + k n];  op(X)(k, j) = X[k + j n]
    TcOpnd v{c.V[l], transpose_v ? (long long)n : 1ll, 0, transpose_v ? 1ll : (long long)n, 0, 1 << 30};
    v.keep = true;
    const TcOpnd x{X[l], (long long)n, 0, 1, 0, 1 << 30};
    items.push_back(TcItem{n, m[l], n, v, x, 1.0, 0.0, Y[l], 1, 0, 1 << 30, (long long)n});
  }
  gemm_tc_group(c, 6, (int)items.size(), items.data());
}

void cp_to_tucker(Ctx &c, int m, const double *w, double *const U[3], bool to_eig, Tucker &out,
                  double eps_core) {
  const int n = c.n;
  if (m == 0) {
    out.r[0] = out.r[1] = out.r[2] = 0;
    return;
  }
  TCTL_PHASE(c, "c2t");
  size_t mk = c.ws.mark();
  double *X[3], *nu[3];
  for (int l = 0; l < 3; ++l) {
    X[l] = c.ws.dbl((size_t)n * m);
    if (!to_eig) copy_d(c, X[l], U[l], (size_t)n * m);
  }
  if (to_eig) {
    const int mm[3] = {m, m, m};
    basis_change3(c, true, mm, U, X);
  }
  for (int l = 0; l < 3; ++l) {
    nu[l] = c.ws.dbl(m);
    col_norms(c, n, m, X[l], n, nu[l]);
  }
  double *s = c.ws.dbl(m);
  double *Y = c.ws.dbl((size_t)n * std::max(m, kMaxRank));
  double *Ct[3];
  for (int l = 0; l < 3; ++l) {
    LAUNCH(c, side_scale_kernel, (m + 255) / 256, 256, 0, m, w, nu[0], nu[1], nu[2], l, s);
    // weighted side matrix: column k of X_l times |w_k| prod_{q != l} ||x_qk||
    copy_d(c, Y, X[l], (size_t)n * m);
    scale_cols(c, n, m, Y, n, s, false);
    int r;
    if (m <= kMaxRank) {
      r = orth(c, n, m, Y, n, 1e-8, true, kMaxRank, out.Q[l]);
    } else {
      double *Om = c.ws.dbl((size_t)m * kMaxRank);
      double *Ys = c.ws.dbl((size_t)n * kMaxRank);
      fill_gaussian(c, Om, (size_t)m * kMaxRank, c.o.seed * 0x9E3779B97F4A7C15ull + (c.rng_counter++));
      gemm(c, false, false, n, kMaxRank, m, 1.0, Y, n, 0, Om, m, 0, 0.0, Ys, n, 0);
      r = orth(c, n, kMaxRank, Ys, n, 1e-8, true, kMaxRank, out.Q[l]);
    }
    out.r[l] = r;
    // C_l^T = X_l^T Q_l (m x r)
    Ct[l] = c.ws.dbl((size_t)m * r);
    gemm(c, true, false, m, r, n, 1.0, X[l], n, 0, out.Q[l], n, 0, 0.0, Ct[l], m, 0);
  }
  // core_(1) = (diag(w) C_1^T)^T KR(C_2^T, C_3^T) : (r0 x m) (m x r1 r2)
  double *KR = c.ws.dbl((size_t)m * out.r[1] * out.r[2]);
  khatri_rao(c, m, Ct[1], m, out.r[1], Ct[2], m, out.r[2], KR, m);
  double *WC = c.ws.dbl((size_t)m * out.r[0]);
  copy_d(c, WC, Ct[0], (size_t)m * out.r[0]);
  // scale rows of WC by w: use scale_cols on the transpose view is not possible; do a gemm with
  // diag via khatri_rao of (w as n=m x 1) and WC
  khatri_rao(c, m, WC, m, out.r[0], w, m, 1, WC, m);
  gemm(c, true, false, out.r[0], out.r[1] * out.r[2], m, 1.0, WC, m, 0, KR, m, 0, 0.0, out.core,
       out.r[0], 0);
  c.ws.reset(mk);
  if (eps_core > 0) tucker_hosvd_trunc(c, out, eps_core);
}

// out (ra rb x N, ld ldo) = KR(X, Y)^T E, i.e.
// out[a + ra b, j] = sum_i X[i, a] Y[i, b] E[i, j], contracted over i < n.
// The tensor-core path forms the Khatri-Rao rows inside its digit split; the
// FP64 path materialises KR(X, Y) (n x ra rb) first.
static void kr_t_gemm(Ctx &c, int n, const double *X, int ldx, int ra, const double *Y, int ldy,
                      int rb, const double *E, int lde, int N, double *out, int ldo) {
  const int M = ra * rb;
  if (M <= 0 || N <= 0) return;
  if (c.o.tc_gemm && gemm_tc_fits(std::max(M, N), std::min(M, N), n, 1)) {
    const TcOpnd kr{X, (long long)ldx, (long long)ldy, 1, 0, ra, Y};
    TcOpnd e{E, (long long)lde, 0, 1, 0, 1 << 30};
    e.keep = true;  // E is a factor matrix of the context's operator
    // the larger dimension takes the 128-row side of the tile
    if (M >= N)
      gemm_tc(c, c.digits, M, N, n, 1, 1, 1, 1.0, kr, e, 0.0, out, 1, 0, 1 << 30, ldo, 0);
    else
      gemm_tc(c, c.digits, N, M, n, 1, 1, 1, 1.0, e, kr, 0.0, out, ldo, 0, 1 << 30, 1, 0);
    return;
  }
  size_t mk = c.ws.mark();
  double *KR = c.ws.dbl((size_t)n * M);
  khatri_rao(c, n, X, ldx, ra, Y, ldy, rb, KR, n);
  gemm_x(c, c.digits, true, false, M, N, n, 1.0, KR, n, 0, E, lde, 0, 0.0, out, ldo, 0);
  c.ws.reset(mk);
}

// The same for several independent products (the three modes of one step):
// on the tensor cores in one grouped launch when every item fits, else one by one.
struct KrSpec {
  const double *X;
  int ldx, ra;
  const double *Y;
  int ldy, rb;
  const double *E;
  int lde, N;
  double *out;
  int ldo;
};

static void kr_t_gemm_group(Ctx &c, int n, int count, const KrSpec *sp) {
  bool tc = c.o.tc_gemm != 0;
  for (int i = 0; i < count && tc; ++i) {
    const int M = sp[i].ra * sp[i].rb;
    tc = M > 0 && sp[i].N > 0 && gemm_tc_fits(std::max(M, sp[i].N), std::min(M, sp[i].N), n, 1);
  }
  if (!tc) {
    for (int i = 0; i < count; ++i)
      kr_t_gemm(c, n, sp[i].X, sp[i].ldx, sp[i].ra, sp[i].Y, sp[i].ldy, sp[i].rb, sp[i].E, sp[i].lde,
                sp[i].N, sp[i].out, sp[i].ldo);
    return;
  }
  std::vector<TcItem> items(count);
  for (int i = 0; i < count; ++i) {
    const KrSpec &q = sp[i];
    const int M = q.ra * q.rb;
    const TcOpnd kr{q.X, (long long)q.ldx, (long long)q.ldy, 1, 0, q.ra, q.Y};
    TcOpnd e{q.E, (long long)q.lde, 0, 1, 0, 1 << 30};
    e.keep = true;  // a factor matrix of the context's operator
    if (M >= q.N)
      items[i] = TcItem{M, q.N, n, kr, e, 1.0, 0.0, q.out, 1, 0, 1 << 30, (long long)q.ldo};
    else
      items[i] = TcItem{q.N, M, n, e, kr, 1.0, 0.0, q.out, (long long)q.ldo, 0, 1 << 30, 1};
  }
  gemm_tc_group(c, c.digits, count, items.data());
}

// Probe factor of mode m for the Khatri-Rao sketches: with Om (n x ls) a fresh
// Gaussian matrix, P_m[(a,s),k] = sum_i Q_m[i,a] Om[i,s] E_m[i,k]
// = (KR(Q_m, Om)^T B_m) Z_m, an (r_m ls) x R matrix in the workspace. The same
// P_m serves the sketches of both other modes (each sketch still draws
// independent Gaussian vectors in each of its two probe modes).
static double *sketch_factor(Ctx &c, const Sep &D, const Tucker &x, int m, int ls) {
  const int n = c.n, R = D.R;
  const int rm = x.r[m];
  double *P = c.ws.dbl((size_t)rm * ls * R);
  size_t mk = c.ws.mark();
  double *Om = c.ws.dbl((size_t)n * ls);
  fill_gaussian(c, Om, (size_t)n * ls, c.o.seed * 0x9E3779B97F4A7C15ull + (c.rng_counter++));
  if (D.Z[m]) {
    double *T = c.ws.dbl((size_t)rm * ls * D.rD[m]);
    kr_t_gemm(c, n, x.Q[m], n, rm, Om, n, ls, D.B[m], n, D.rD[m], T, rm * ls);
    gemm_x(c, c.digits, false, false, rm * ls, R, D.rD[m], 1.0, T, rm * ls, 0, D.Z[m], D.rD[m], 0,
           0.0, P, rm * ls, 0);
  } else {
    // uncompressed operator: B_m holds the R factor columns themselves
    kr_t_gemm(c, n, x.Q[m], n, rm, Om, n, ls, D.B[m], n, D.rD[m], P, rm * ls);
  }
  c.ws.reset(mk);
  return P;
}

// Y (n x ls) = mode-l unfolding of D .* X times ls Khatri-Rao Gaussian probes
// (one Gaussian vector per other mode per probe, from the probe factors P).
// Cl: core permuted so mode l is first.
// uT (r_l ls x rD_l, in the workspace) of the mode-l sketch:
// v[a,(s,k)] = w_k sum_{b,c} Cl[a,b,c] P_m1[(b,s),k] P_m2[(c,s),k], in chunks of k;
// uT[(a,s),p] = sum_k v[(a,s),k] Z_l[p,k] (uT = v for an uncompressed operator)
static double *sketch_uT(Ctx &c, const Sep &D, const Tucker &x, const double *Cl, int l, int ls,
                         double *const P[3]) {
  const int R = D.R;
  const int r[3] = {x.r[0], x.r[1], x.r[2]};
  const int oth[3][2] = {{1, 2}, {0, 2}, {0, 1}};
  const int m1 = oth[l][0], m2 = oth[l][1];
  double *uT = c.ws.dbl((size_t)r[l] * ls * D.rD[l]);
  size_t mk = c.ws.mark();
  const long long per_k = (long long)r[l] * r[m1] * ls;
  const int kc = (int)std::max<long long>(1, std::min<long long>(R, (32ll << 20) / std::max(per_k, 1ll)));
  double *F = c.ws.dbl((size_t)per_k * kc);
  double *v = c.ws.dbl((size_t)r[l] * ls * kc);
  for (int k0 = 0; k0 < R; k0 += kc) {
    const int nk = std::min(kc, R - k0);
    gemm_x(c, c.digits, false, false, r[l] * r[m1], ls * nk, r[m2], 1.0, Cl, r[l] * r[m1], 0,
           P[m2] + (size_t)r[m2] * ls * k0, r[m2], 0, 0.0, F, r[l] * r[m1], 0);
    const long long tot = (long long)r[l] * ls * nk;
    const int blocks = (int)std::min<long long>((tot + 255) / 256, 4096);
    LAUNCH(c, contract_b_kernel, blocks, 256, 0, r[l], r[m1], ls, nk, F,
           P[m1] + (size_t)r[m1] * ls * k0, D.w + k0, v);
    if (D.Z[l]) {
      gemm_x(c, c.digits, false, true, r[l] * ls, D.rD[l], nk, 1.0, v, r[l] * ls, 0,
             D.Z[l] + (size_t)D.rD[l] * k0, D.rD[l], 0, k0 == 0 ? 0.0 : 1.0, uT, r[l] * ls, 0);
    } else {
      copy_d(c, uT + (size_t)r[l] * ls * k0, v, (size_t)r[l] * ls * nk);
    }
  }
  c.ws.reset(mk);
  return uT;
}

// Y[i, s] = sum_{a,p} Q_l[i, a] B_l[i, p] uT[(a,s), p], contracted over p
// first: W[i, a + r_l s] = (B_l uT^T)[i, (a,s)] (n x r_l ls, in slices of s),
// then over a row by row. The Khatri-Rao product KR(Q_l, B_l) (n x r_l rD)
// is never formed.
static int sketch_slice(const Ctx &c, const Tucker &x, int l, int ls) {
  return std::max(1, std::min(ls, (int)((64ll << 20) / ((long long)c.n * x.r[l] * 8))));
}

static void sketch_rows(Ctx &c, const Sep &D, const Tucker &x, int l, int ls, const double *uT, double *Y) {
  const int n = c.n, rl = x.r[l];
  size_t mk = c.ws.mark();
  const int sc = sketch_slice(c, x, l, ls);
  double *W = c.ws.dbl((size_t)n * rl * sc);
  for (int s0 = 0; s0 < ls; s0 += sc) {
    const int ns = std::min(sc, ls - s0);
    gemm_x(c, c.digits, false, true, n, rl * ns, D.rD[l], 1.0, D.B[l], n, 0, uT + (size_t)rl * s0, rl * ls,
           0, 0.0, W, n, 0, 1, 1, 1, true);
    const long long tot = (long long)n * ns;
    const int blocks = (int)std::min<long long>((tot + 255) / 256, 4096);
    c.next_bytes = 8.0 * n * ((double)rl * ns + rl + ns);
    LAUNCH(c, rowdot_kernel, blocks, 256, 0, n, rl, ns, x.Q[l], n, W, n, Y + (size_t)n * s0, n);
  }
  c.ws.reset(mk);
}

// Y_l (n x ls) = mode-l unfolding of D .* X times ls Khatri-Rao Gaussian probes
// (one Gaussian vector per other mode per probe, from the probe factors P), for
// the modes in `modes`; Cl[l]: core permuted so mode l is first. With the
// tensor-core contractions the W products of all the modes run in one grouped
// launch when each needs a single slice.
static void sketch_modes(Ctx &c, const Sep &D, const Tucker &x, double *const Cl[3], const int *modes,
                         int count, int ls, double *const P[3], double *const Y[3]) {
  const int n = c.n;
  size_t mk = c.ws.mark();
  double *uT[3] = {nullptr, nullptr, nullptr};
  for (int t = 0; t < count; ++t) uT[modes[t]] = sketch_uT(c, D, x, Cl[modes[t]], modes[t], ls, P);
  bool group = c.o.tc_gemm != 0 && count > 1;
  for (int t = 0; t < count && group; ++t) {
    const int l = modes[t], N = x.r[l] * ls;
    group = !D.Z[l] && sketch_slice(c, x, l, ls) >= ls &&
            gemm_tc_fits(std::max(n, N), std::min(n, N), D.rD[l], 1);
  }
  if (!group) {
    for (int t = 0; t < count; ++t) sketch_rows(c, D, x, modes[t], ls, uT[modes[t]], Y[modes[t]]);
    c.ws.reset(mk);
    return;
  }
  double *W[3] = {nullptr, nullptr, nullptr};
  std::vector<TcItem> items;
  for (int t = 0; t < count; ++t) {
    const int l = modes[t], N = x.r[l] * ls, K = D.rD[l];
    W[l] = c.ws.dbl((size_t)n * N);
    // op(B_l)(i, p) = B_l[i + p n] (kept factor planes); op(uT^T)(j, p) = uT[j + p N]
    TcOpnd b{D.B[l], 1, 0, (long long)n, 0, 1 << 30};
    b.keep = true;
    const TcOpnd u{uT[l], 1, 0, (long long)N, 0, 1 << 30};
    if (n >= N)
      items.push_back(TcItem{n, N, K, b, u, 1.0, 0.0, W[l], 1, 0, 1 << 30, (long long)n});
    else  // W^T = uT B_l^T: the larger dimension on the 128-row side
      items.push_back(TcItem{N, n, K, u, b, 1.0, 0.0, W[l], (long long)n, 0, 1 << 30, 1});
  }
  gemm_tc_group(c, c.digits, (int)items.size(), items.data());
  RowdotGroup rg{};
  double bytes = 0;
  for (int t = 0; t < count; ++t) {
    const int l = modes[t];
    rg.ra[t] = x.r[l];
    rg.Q[t] = x.Q[l];
    rg.W[t] = W[l];
    rg.Y[t] = Y[l];
    bytes += 8.0 * n * ((double)x.r[l] * ls + x.r[l] + ls);
  }
  rg.count = count;
  const long long tot = (long long)n * ls * count;
  const int blocks = (int)std::min<long long>((tot + 255) / 256, 4096);
  c.next_bytes = bytes;
  LAUNCH(c, rowdot_group_kernel, blocks, 256, 0, n, ls, rg);
  c.ws.reset(mk);
}

void sep_apply_trunc(Ctx &c, const Sep &Dc, const Tucker &x, Tucker &y, double eps) {
  const int n = c.n;
  if (tucker_empty(x)) {
    y.r[0] = y.r[1] = y.r[2] = 0;
    return;
  }
  // The tensor-core contractions use the factor matrices E_l themselves: their
  // error is relative to the row / column maxima of the operands, and the
  // compressed form E_l = B_l Z_l recombines basis coefficients with
  // cancellation (entries of E_l span many orders of magnitude across i), which
  // would amplify that error. FP64 uses the compressed basis (rD_l < R columns).
  Sep Du;
  if (c.o.tc_gemm) {
    Du.R = Dc.R;
    Du.w = Dc.w;
    for (int l = 0; l < 3; ++l) {
      Du.E[l] = Du.B[l] = Dc.E[l];
      Du.rD[l] = Dc.R;
      Du.Z[l] = nullptr;
    }
  }
  const Sep &D = c.o.tc_gemm ? Du : Dc;
  const int R = D.R;
  size_t mk = c.ws.mark();
  const int r[3] = {x.r[0], x.r[1], x.r[2]};
  int rmax = std::max(r[0], std::max(r[1], r[2]));
  double *Qn[3];
  int rn[3];
  // permuted cores with mode l first: Cl[l] dims (r_l, r_m1, r_m2), m1 < m2 the other modes
  double *Cl[3];
  for (int l = 0; l < 3; ++l) Cl[l] = c.ws.dbl((size_t)r[0] * r[1] * r[2]);
  unfold3(c, r, x.core, Cl[0], Cl[1], Cl[2]);
  // ---------------- range finding per mode
  int ls = std::min(kMaxRank, rmax + 24);
  const double rtol = std::max(1e-8, c.o.range_tol * eps);
  TCTL_PHASE(c, "sep_sketch");
  for (int l = 0; l < 3; ++l) {
    Qn[l] = c.ws.dbl((size_t)n * kMaxRank);
    rn[l] = 0;
  }
  {
    // the three mode sketches first, then their bases in one batched orthonormalisation;
    // a saturated sketch (rank = width) is redone at width 64
    size_t mks = c.ws.mark();
    double *P[3] = {nullptr, nullptr, nullptr};
    double *Y[3];
    for (int l = 0; l < 3; ++l) Y[l] = c.ws.dbl((size_t)n * kMaxRank);
    bool todo[3] = {true, true, true};
    for (int attempt = 0; attempt < 2; ++attempt) {
      size_t mkp = c.ws.mark();
      if (!D.Z[0] && !D.Z[1] && !D.Z[2]) {
        // uncompressed operator (tensor-core path): P_m = KR(Q_m, Om_m)^T E_m, the
        // three modes in one grouped launch (probes drawn in mode order as below)
        double *Om[3];
        KrSpec sp[3];
        for (int m = 0; m < 3; ++m) P[m] = c.ws.dbl((size_t)x.r[m] * ls * R);
        size_t cnt[3];
        uint64_t seeds[3];
        for (int m = 0; m < 3; ++m) {
          Om[m] = c.ws.dbl((size_t)n * ls);
          cnt[m] = (size_t)n * ls;
          seeds[m] = c.o.seed * 0x9E3779B97F4A7C15ull + (c.rng_counter++);
          sp[m] = KrSpec{x.Q[m], n, x.r[m], Om[m], n, ls, D.B[m], n, D.rD[m], P[m], x.r[m] * ls};
        }
        fill_gaussian_multi(c, 3, Om, cnt, seeds);
        kr_t_gemm_group(c, n, 3, sp);
      } else {
        for (int m = 0; m < 3; ++m) P[m] = sketch_factor(c, D, x, m, ls);
      }
      int cnt = 0, ms[3], lds[3], caps[3], rr[3], idx[3];
      double *Ys[3], *Qs[3];
      {
        int modes[3], nm = 0;
        for (int l = 0; l < 3; ++l)
          if (todo[l]) modes[nm++] = l;
        sketch_modes(c, D, x, Cl, modes, nm, ls, P, Y);
      }
      for (int l = 0; l < 3; ++l) {
        if (!todo[l]) continue;
        idx[cnt] = l;
        ms[cnt] = ls;
        lds[cnt] = n;
        caps[cnt] = kMaxRank;
        Ys[cnt] = Y[l];
        Qs[cnt] = Qn[l];
        ++cnt;
      }
      orth_multi(c, cnt, n, ms, Ys, lds, rtol, true, caps, Qs, rr);
      bool again = false;
      for (int t = 0; t < cnt; ++t) {
        rn[idx[t]] = rr[t];
        todo[idx[t]] = (rr[t] >= ls && ls < kMaxRank);
        again = again || todo[idx[t]];
      }
      c.ws.reset(mkp);
      if (!again) break;
      ls = kMaxRank;
    }
    c.ws.reset(mks);
  }
  // ---------------- core of D .* X in the new bases
  TCTL_PHASE(c, "sep_core");
  double *M[3];
  {
    // N_l[(a',b), p] = sum_i Qn[i,a'] Q[i,b] B[i,p], the three modes grouped;
    // M_l = N_l Z_l : (rn r) x R for a compressed operator
    double *Nl[3];
    KrSpec sp[3];
    for (int l = 0; l < 3; ++l) {
      Nl[l] = c.ws.dbl((size_t)rn[l] * r[l] * D.rD[l]);
      sp[l] = KrSpec{Qn[l], n, rn[l], x.Q[l], n, r[l], D.B[l], n, D.rD[l], Nl[l], rn[l] * r[l]};
    }
    kr_t_gemm_group(c, n, 3, sp);
    for (int l = 0; l < 3; ++l) {
      if (D.Z[l]) {
        M[l] = c.ws.dbl((size_t)rn[l] * r[l] * R);
        gemm_x(c, c.digits, false, false, rn[l] * r[l], R, D.rD[l], 1.0, Nl[l], rn[l] * r[l], 0, D.Z[l],
               D.rD[l], 0, 0.0, M[l], rn[l] * r[l], 0);
      } else {
        M[l] = Nl[l];
      }
    }
  }
  const long long szo = (long long)rn[0] * rn[1] * rn[2];
  double *nc = c.ws.dbl(szo);
  if (!core_proj(c, r, rn, x.core, M, D.w, R, nc)) {
    const long long s1 = (long long)rn[0] * r[1] * r[2];
    const long long s2 = (long long)rn[0] * r[1] * rn[2];
    const long long s3 = szo;
    const long long per = s1 + s2 + s3;
    const int kc = (int)std::max<long long>(1, std::min<long long>(R, (48ll << 20) / per));
    double *T1 = c.ws.dbl((size_t)s1 * kc), *T2 = c.ws.dbl((size_t)s2 * kc),
           *T3 = c.ws.dbl((size_t)s3 * kc);
    // On the tensor cores T2 is written with the term next to the contracted
    // index, T2'[(a, c'), (b, k)], so that T3 and the weighted sum over the terms
    // are one GEMM contracted over (b, k) (K = r1 nk instead of r1), with the
    // weights folded into a scaled copy of M_1: nc[a, b', c'] += sum_(b,k)
    // T2'[(a, c'), (b, k)] w_k M_1k[b', b].
    // Only with 6 digits: one row of the merged GEMM's operands spans every
    // operator term, whose magnitudes differ by orders, and the digit split
    // keeps 7D bits below the row's largest; 42 bits hold the small terms'
    // contributions, the 21 of the three-term split do not (the per-term chain
    // below splits each term on its own).
    const bool fused = c.o.tc_gemm && c.digits >= 6 && gemm_tc_fits(rn[0] * r[1], rn[2], r[2], kc) &&
                       gemm_tc_fits(rn[0] * rn[2], rn[1], r[1] * kc, 1);
    double *M1w = nullptr;
    if (fused) {
      M1w = c.ws.dbl((size_t)rn[1] * r[1] * R);
      copy_d(c, M1w, M[1], (size_t)rn[1] * r[1] * R);
      scale_cols(c, rn[1] * r[1], R, M1w, rn[1] * r[1], D.w, false);
    }
    for (int k0 = 0; k0 < R; k0 += kc) {
      const int nk = std::min(kc, R - k0);
      // T1[k] = M_0k (rn0 x r0) * core (r0 x r1 r2)
      gemm_x(c, c.digits, false, false, rn[0], r[1] * r[2], r[0], 1.0,
             M[0] + (size_t)rn[0] * r[0] * k0, rn[0], (long long)rn[0] * r[0], x.core, r[0], 0, 0.0,
             T1, rn[0], s1, nk);
      if (fused) {
        // T2'[(a + rn0 c') + rn0 rn2 (b + r1 k)] = sum_c T1[k](a, b, c) M_2k(c', c)
        const TcOpnd A{T1, 1, 0, (long long)rn[0] * r[1], s1, 1 << 30};
        const TcOpnd B{M[2] + (size_t)rn[2] * r[2] * k0, 1, 0, (long long)rn[2], (long long)rn[2] * r[2],
                       1 << 30};
        gemm_tc(c, c.digits, rn[0] * r[1], rn[2], r[2], nk, 1, 1, 1.0, A, B, 0.0, T2, 1,
                (long long)rn[0] * rn[2], rn[0], rn[0], s2);
        // nc[a + rn0 b' + rn0 rn1 c'] (+)= sum_(b,k) T2'[(a, c'), (b, k)] M1w[b' + rn1 (b + r1 k)]
        const TcOpnd A3{T2, 1, 0, (long long)rn[0] * rn[2], 0, 1 << 30};
        const TcOpnd B3{M1w + (size_t)rn[1] * r[1] * k0, 1, 0, (long long)rn[1], 0, 1 << 30};
        gemm_tc(c, c.digits, rn[0] * rn[2], rn[1], r[1] * nk, 1, 1, 1, 1.0, A3, B3, k0 == 0 ? 0.0 : 1.0,
                nc, 1, (long long)rn[0] * rn[1], rn[0], rn[0], 0);
        continue;
      }
      // T2[k] = T1[k] (rn0 r1 x r2) * M_2k^T (r2 x rn2)
      gemm_x(c, c.digits, false, true, rn[0] * r[1], rn[2], r[2], 1.0, T1, rn[0] * r[1], s1,
             M[2] + (size_t)rn[2] * r[2] * k0, rn[2], (long long)rn[2] * r[2], 0.0, T2, rn[0] * r[1],
             s2, nk);
      // T3[k](a, b', c') = sum_b T2[k](a, b, c') M_1k(b', b)
      if (c.o.tc_gemm && gemm_tc_fits(rn[0] * rn[2], rn[1], r[1], nk)) {
        // one GEMM per k with rows (a, c'): T2[k] (rn0 rn2 x r1) * M_1k^T
        const TcOpnd A{T2, 1, (long long)rn[0] * r[1], (long long)rn[0], s2, rn[0]};
        const TcOpnd B{M[1] + (size_t)rn[1] * r[1] * k0, 1, 0, (long long)rn[1],
                       (long long)rn[1] * r[1], 1 << 30};
        gemm_tc(c, c.digits, rn[0] * rn[2], rn[1], r[1], nk, 1, 1, 1.0, A, B, 0.0, T3, 1,
                (long long)rn[0] * rn[1], rn[0], rn[0], s3);
      } else {
        // batch over (k, c'): T2[k][:,:,c'] (rn0 x r1) * M_1k^T (r1 x rn1)
        gemm(c, false, true, rn[0], rn[1], r[1], 1.0, T2, rn[0], (long long)rn[0] * r[1],
             M[1] + (size_t)rn[1] * r[1] * k0, rn[1], (long long)rn[1] * r[1], 0.0, T3, rn[0],
             (long long)rn[0] * rn[1], nk * rn[2], 1, rn[2]);
      }
      // nc += T3 w
      gemm(c, false, false, (int)szo, 1, nk, 1.0, T3, (int)szo, 0, D.w + k0, nk, 0,
           k0 == 0 ? 0.0 : 1.0, nc, (int)szo, 0);
    }
  }
  for (int l = 0; l < 3; ++l) {
    y.r[l] = rn[l];
    copy_d(c, y.Q[l], Qn[l], (size_t)n * rn[l]);
  }
  copy_d(c, y.core, nc, (size_t)szo);
  c.ws.reset(mk);
  tucker_hosvd_trunc(c, y, eps);
  if (c.trace)
    std::fprintf(stderr, "[tctl] %s R=%d x=(%d,%d,%d) ls=%d range=(%d,%d,%d) out=(%d,%d,%d)\n",
                 c.outer ? c.outer : "apply", R, r[0], r[1], r[2], ls, rn[0], rn[1], rn[2], y.r[0],
                 y.r[1], y.r[2]);
}

int tucker_to_cp(Ctx &c, const Tucker &x, bool from_eig, double eps, tctl_cp *y) {
  const int n = c.n;
  if (tucker_empty(x)) {
    y->rank = 0;
    return TCTL_OK;
  }
  TCTL_PHASE(c, "t2c");
  size_t mk = c.ws.mark();
  const int r0 = x.r[0], r1 = x.r[1], r2 = x.r[2];
  double *Qp[3];
  for (int l = 0; l < 3; ++l) {
    Qp[l] = c.ws.dbl((size_t)n * x.r[l]);
    if (!from_eig) copy_d(c, Qp[l], x.Q[l], (size_t)n * x.r[l]);
  }
  if (from_eig) basis_change3(c, false, x.r, x.Q, Qp);
  // slice Grams S_c^T S_c (r1 x r1), batch r2
  double *G = c.ws.dbl((size_t)r1 * r1 * r2);
  gemm(c, true, false, r1, r1, r0, 1.0, x.core, r0, (long long)r0 * r1, x.core, r0,
       (long long)r0 * r1, 0.0, G, r1, (long long)r1 * r1, r2, 1, 1);
  double *lam = c.ws.dbl((size_t)r1 * r2), *Bv = c.ws.dbl((size_t)r1 * r1 * r2);
  sym_eig(c, r1, r2, G, lam, Bv);
  // A_c = S_c Bv_c (r0 x r1); columns later divided by sigma
  double *Av = c.ws.dbl((size_t)r0 * r1 * r2);
  gemm(c, false, false, r0, r1, r1, 1.0, x.core, r0, (long long)r0 * r1, Bv, r1, (long long)r1 * r1,
       0.0, Av, r0, (long long)r0 * r1, r2, 1, 1);
  std::vector<double> lh((size_t)r1 * r2);
  to_host(c, lh.data(), lam, lh.size());
  double tot = 0.0;
  for (double v : lh) tot += std::max(v, 0.0);
  struct Trip {
    double s2;
    int c, i;
  };
  std::vector<Trip> trips;
  for (int cc = 0; cc < r2; ++cc)
    for (int i = 0; i < std::min(r0, r1); ++i) trips.push_back({std::max(lh[i + (size_t)cc * r1], 0.0), cc, i});
  std::vector<int> order(trips.size());
  std::iota(order.begin(), order.end(), 0);
  std::sort(order.begin(), order.end(), [&](int a, int b) { return trips[a].s2 < trips[b].s2; });
  std::vector<char> drop(trips.size(), 0);
  double acc = 0.0;
  for (int j : order) {
    if (acc + trips[j].s2 > eps * eps * tot) break;
    acc += trips[j].s2;
    drop[j] = 1;
  }
  std::vector<int> ia, ib, ic;
  std::vector<double> wv, inv;
  for (size_t j = 0; j < trips.size(); ++j) {
    if (drop[j] || trips[j].s2 <= 0.0) continue;
    const double sg = std::sqrt(trips[j].s2);
    ia.push_back(trips[j].i + trips[j].c * r1);  // column of Av / Bv (slice-major)
    ic.push_back(trips[j].c);
    wv.push_back(sg);
    inv.push_back(1.0 / sg);
  }
  const int rank = (int)wv.size();
  int status = TCTL_OK;
  int keep = rank;
  if (rank > y->cap) {
    status = TCTL_E_RANK_CAP;
    keep = y->cap;
  }
  if (keep > 0) {
    int *idx = c.ws.i32(keep), *idc = c.ws.i32(keep);
    write_dev(c, idx, ia.data(), sizeof(int) * keep);
    write_dev(c, idc, ic.data(), sizeof(int) * keep);
    double *Asel = c.ws.dbl((size_t)r0 * keep), *Bsel = c.ws.dbl((size_t)r1 * keep);
    double *invd = c.ws.dbl(keep);
    to_dev(c, invd, inv.data(), keep);
    gather_cols(c, r0, Av, r0, idx, keep, Asel, r0);
    scale_cols(c, r0, keep, Asel, r0, invd, false);
    gather_cols(c, r1, Bv, r1, idx, keep, Bsel, r1);
    gemm(c, false, false, n, keep, r0, 1.0, Qp[0], n, 0, Asel, r0, 0, 0.0, y->U[0], n, 0);
    gemm(c, false, false, n, keep, r1, 1.0, Qp[1], n, 0, Bsel, r1, 0, 0.0, y->U[1], n, 0);
    gather_cols(c, n, Qp[2], n, idc, keep, y->U[2], n);
    to_dev(c, y->w, wv.data(), keep);
  }
  y->rank = keep;
  c.ws.reset(mk);
  return status;
}

}  // namespace tctl
