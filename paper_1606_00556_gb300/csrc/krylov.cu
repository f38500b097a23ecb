// Restarted flexible GMRES(m) in FP64 (paper Sec. 3.3 solver list; GMRES(30)
// in Sec. 4), right preconditioned by CPR-FPF of the decoupled system, with
// the paper's stopping rule ||b - A x|| <= tol ||b|| (Alg. 1) tested on the
// recomputed FP64 residual of the original system.
//
// The Krylov space is that of D_QI^{-1} A preconditioned by CPR: with
// M^{-1} = CPR o D_QI^{-1}, (A M^{-1})^k b = D_QI ((D_QI^{-1} A) CPR)^k D_QI^{-1} b,
// so the iterates are those of the decoupled system and the minimised norm
// is the original residual.
//
// Orthogonalisation: classical Gram-Schmidt applied twice (CGS2) for every
// column: a multi-dot pass h1 = V^T w, an update pass w -= V h1, then the
// same again, the second update also reducing ||w||^2 and applying the
// Givens step; the first update and the second multi-dot share one pass over
// the basis, so a column takes three passes.  A second pass is necessary here: with a strong CPR
// preconditioner A M^{-1} is close to the identity, so the new direction
// cancels to 1e-6 of ||w|| and one classical pass alone loses all
// orthogonality.  The basis vectors are stored unnormalised with their
// scale 1/||v|| kept on the device; every reader applies it, so no pass is
// spent normalising.
//
// The basis is stored as split pairs (per vector a plane of high floats,
// then a plane of low floats: 48 significant bits, the same 8 bytes per
// entry as FP64), and the second coefficient pass and both updates compute
// in split arithmetic (df below): GB300 issues about 64 times more FP32
// than FP64 operations per clock, so these passes are bound by HBM instead
// of by the FP64 pipe (in FP64 they ran at 51-67% of HBM).  A split
// multiply-add keeps about 2^-46 of each term, so the Arnoldi relation
// A z_j = V h_j + w holds to about 1e-14 and the twice-orthogonalised
// vector is orthogonal to V to that level: far below the 1e-8 residual
// target, which is decided on the FP64 true residual.  The first
// coefficient pass reads only the high plane and sums in FP32: the second
// pass removes whatever it left in span(V), and the updates subtract
// exactly the coefficients they are given.
//
// The Arnoldi product w = A z_j reads a split copy of A (each value as an
// unevaluated sum hi + lo of two floats, 48 significant bits; see df in
// bo_internal.cuh) in a tiled layout, and the preconditioned vectors Z are
// stored as split pairs too (a hi plane, then a lo plane; exact for the FP32
// preconditioner's output).  The product is formed with FP32 instructions,
// so it is bound by HBM rather than by GB300's FP64 rate; w is written in
// FP64.  The true residual b - A x, which decides convergence, is FP64 on
// the original FP64 matrix.
//
// Every reduction is two-stage with a fixed order (per-block partial sums,
// then the last block to finish sums the partials), so results are bitwise
// repeatable.  The Givens rotations run in that last block; a flag in device
// memory makes the rest of a cycle's kernels return at once after
// convergence, so the host only polls with a lag of one iteration.
#include <chrono>
#include <cmath>
#include <algorithm>
#include <cstring>
#include <vector>
#include <mutex>

#include "bo_internal.cuh"

namespace bo {
namespace {

constexpr int kRedBlocks = 4 * 152;  // blocks of single reductions
constexpr int kMaxM = 64;
constexpr int kHistCap = 4096;
constexpr int kDotBlocks = 4 * 152;  // most chunks of a coefficient pass (partials per column)

// The split basis: vector k at k * ldv floats, ldv = 2 np, its high plane
// at [0, n) and its low plane at [np, np + n), np = n rounded up to a
// multiple of 4 so that every plane starts on a 16-byte boundary.  The
// Gram-Schmidt kernels below read and write four consecutive entries per
// thread with 16-byte accesses: with 4-byte ones a warp request carries
// too few bytes to keep enough of them in flight to stream at HBM rate.
// The last group of four of a plane may reach into the padding: its lanes
// at or beyond n are neither used nor stored.
__host__ __device__ __forceinline__ int64_t split_pad(int64_t n) { return (n + 3) & ~(int64_t)3; }

__device__ __forceinline__ float4 ld4(const float* p) { return *reinterpret_cast<const float4*>(p); }
// 16-byte loads with L1 eviction priorities: the fused Gram-Schmidt pass
// reads each column twice per thread, and asks L1 to keep the first read
// (evict_last) and to drop the second (evict_first)
__device__ __forceinline__ float4 ld4_keep(const float* p) {
  float4 v;
  asm volatile("ld.global.L1::evict_last.v4.f32 {%0,%1,%2,%3}, [%4];" : "=f"(v.x), "=f"(v.y), "=f"(v.z), "=f"(v.w) : "l"(p));
  return v;
}
__device__ __forceinline__ float4 ld4_last(const float* p) {
  float4 v;
  asm volatile("ld.global.L1::evict_first.v4.f32 {%0,%1,%2,%3}, [%4];" : "=f"(v.x), "=f"(v.y), "=f"(v.z), "=f"(v.w) : "l"(p));
  return v;
}
__device__ __forceinline__ void st4(float* p, float4 v) { *reinterpret_cast<float4*>(p) = v; }
__device__ __forceinline__ float lane4(const float4& v, int e) { return e == 0 ? v.x : e == 1 ? v.y : e == 2 ? v.z : v.w; }
// v with the lanes at or beyond `valid` (0..4) set to zero
__device__ __forceinline__ float4 mask4(float4 v, int valid) {
  if (valid < 4) {
    v.w = 0.f;
    if (valid < 3) v.z = 0.f;
    if (valid < 2) v.y = 0.f;
    if (valid < 1) v.x = 0.f;
  }
  return v;
}

// acc + a0 x0 + a1 x1 + a2 x2 in split arithmetic (low parts collected lazily)
__device__ __forceinline__ df dfma3(df acc, float2 a0, df x0, float2 a1, df x1, float2 a2, df x2) {
  acc = df_fma_acc(acc, df{a0.x, a0.y}, x0);
  acc = df_fma_acc(acc, df{a1.x, a1.y}, x1);
  return df_fma_acc(acc, df{a2.x, a2.y}, x2);
}

// w = A z on internal vectors: z split pairs (planes of n = 3N); w split
// pairs (W = float: an FGMRES basis vector) or FP64 (W = double: the
// BiCGSTAB recurrences).  A2 is the split copy of A; where it could not
// hold every value (*range) the product is formed in FP64 from A instead.
template <typename W>
__global__ void __launch_bounds__(kThreads) k_arnoldi_spmv(Geom g, const float2* __restrict__ A2,
                                                          const double* __restrict__ A, const int* __restrict__ range,
                                                          const float* __restrict__ z, W* __restrict__ w,
                                                          const DevState* st) {
  wait_prior_grid();
  const int64_t wlo = split_pad(3 * g.N);  // low plane of a split w (the basis layout)
  if (st->done) return;
  const int64_t n = 3 * g.N;
  const bool fp64 = *range != 0;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < g.N; t += (int64_t)gridDim.x * blockDim.x) {
    const int color = (int)(t / g.Nh);
    const int64_t q = t - color * g.Nh;
    const Cell c = decode(g, color, q);
    const size_t P = (size_t)g.Nh;
    df n0, n1, n2;
    if (!fp64) {
      df a0{0.f, 0.f}, a1{0.f, 0.f}, a2{0.f, 0.f};
#pragma unroll
      for (int sl = 0; sl < 7; ++sl) {
        const int64_t nq = nbr(g, c, q, sl);
        if (nq < 0) continue;
        const int xc = (sl == kDiag) ? color : (color ^ 1);
        const size_t i0 = vidx(g, 0, xc, nq), i1 = vidx(g, 1, xc, nq), i2 = vidx(g, 2, xc, nq);
        const df x0{z[i0], z[n + i0]}, x1{z[i1], z[n + i1]}, x2{z[i2], z[n + i2]};
        const float2* a = A2 + a2_index(g, color, sl * 9, q);
        a0 = dfma3(a0, __ldcs(a), x0, __ldcs(a + 32), x1, __ldcs(a + 64), x2);
        a1 = dfma3(a1, __ldcs(a + 96), x0, __ldcs(a + 128), x1, __ldcs(a + 160), x2);
        a2 = dfma3(a2, __ldcs(a + 192), x0, __ldcs(a + 224), x1, __ldcs(a + 256), x2);
      }
      n0 = df_renorm(a0);
      n1 = df_renorm(a1);
      n2 = df_renorm(a2);
    } else {
      double a0 = 0.0, a1 = 0.0, a2 = 0.0;
      for (int sl = 0; sl < 7; ++sl) {
        const int64_t nq = nbr(g, c, q, sl);
        if (nq < 0) continue;
        const int xc = (sl == kDiag) ? color : (color ^ 1);
        const size_t i0 = vidx(g, 0, xc, nq), i1 = vidx(g, 1, xc, nq), i2 = vidx(g, 2, xc, nq);
        const double x0 = (double)z[i0] + (double)z[n + i0], x1 = (double)z[i1] + (double)z[n + i1],
                     x2 = (double)z[i2] + (double)z[n + i2];
        const double* a = A + plane(g, color, sl, 0) + q;
        a0 = fma3(a0, a[0], x0, a[P], x1, a[2 * P], x2);
        a1 = fma3(a1, a[3 * P], x0, a[4 * P], x1, a[5 * P], x2);
        a2 = fma3(a2, a[6 * P], x0, a[7 * P], x1, a[8 * P], x2);
      }
      if constexpr (sizeof(W) == 8) {
        w[t] = a0;
        w[g.N + t] = a1;
        w[2 * g.N + t] = a2;
        continue;
      }
      n0 = df_from(a0);
      n1 = df_from(a1);
      n2 = df_from(a2);
    }
    if constexpr (sizeof(W) == 4) {
      w[t] = n0.hi;
      w[g.N + t] = n1.hi;
      w[2 * g.N + t] = n2.hi;
      w[wlo + t] = n0.lo;
      w[wlo + g.N + t] = n1.lo;
      w[wlo + 2 * g.N + t] = n2.lo;
    } else {
      w[t] = df_to_double(n0);
      w[g.N + t] = df_to_double(n1);
      w[2 * g.N + t] = df_to_double(n2);
    }
  }
}

// sum of partials[0..np) in a fixed order by one block
__device__ double reduce_partials(const double* partials, int np, double* sh) {
  double s = 0.0;
  for (int i = threadIdx.x; i < np; i += blockDim.x) s += __ldcg(partials + i);
  return block_sum(s, sh);
}

// r = b - A x (FP64), ||r|| -> st->beta
__global__ void __launch_bounds__(kThreads) k_true_residual(Geom g, const double* __restrict__ A,
                                                           const double* __restrict__ b, const double* __restrict__ x,
                                                           double* __restrict__ r, double* partials, DevState* st) {
  wait_prior_grid();
  __shared__ double sh[32];
  double acc = 0.0;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < g.N; t += (int64_t)gridDim.x * blockDim.x) {
    const int color = (int)(t / g.Nh);
    const int64_t q = t - color * g.Nh;
    const Cell c = decode(g, color, q);
    double a0 = 0.0, a1 = 0.0, a2 = 0.0;
#pragma unroll
    for (int sl = 0; sl < 7; ++sl) {
      const int64_t nq = nbr(g, c, q, sl);
      if (nq < 0) continue;
      const int xc = (sl == kDiag) ? color : (color ^ 1);
      const double x0 = x[vidx(g, 0, xc, nq)], x1 = x[vidx(g, 1, xc, nq)], x2 = x[vidx(g, 2, xc, nq)];
      const double* a = A + plane(g, color, sl, 0) + q;
      const size_t P = (size_t)g.Nh;
      a0 = fma3(a0, ld_stream(a), x0, ld_stream(a + P), x1, ld_stream(a + 2 * P), x2);
      a1 = fma3(a1, ld_stream(a + 3 * P), x0, ld_stream(a + 4 * P), x1, ld_stream(a + 5 * P), x2);
      a2 = fma3(a2, ld_stream(a + 6 * P), x0, ld_stream(a + 7 * P), x1, ld_stream(a + 8 * P), x2);
    }
    const double r0 = b[t] - a0, r1 = b[g.N + t] - a1, r2 = b[2 * g.N + t] - a2;
    r[t] = r0;
    r[g.N + t] = r1;
    r[2 * g.N + t] = r2;
    acc += r0 * r0 + r1 * r1 + r2 * r2;
  }
  acc = block_sum(acc, sh);
  if (threadIdx.x == 0) partials[blockIdx.x] = acc;
  if (last_block(&st->counter[1], gridDim.x)) {
    const double s = reduce_partials(partials, gridDim.x, sh);
    if (threadIdx.x == 0) {
      st->beta = sqrt(s);
      st->counter[1] = 0;
    }
  }
}

// ||v|| -> st->bnorm
__global__ void k_norm(int64_t n, const double* __restrict__ v, double* partials, DevState* st) {
  wait_prior_grid();
  __shared__ double sh[32];
  double acc = 0.0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    acc += v[i] * v[i];
  acc = block_sum(acc, sh);
  if (threadIdx.x == 0) partials[blockIdx.x] = acc;
  if (last_block(&st->counter[2], gridDim.x)) {
    const double s = reduce_partials(partials, gridDim.x, sh);
    if (threadIdx.x == 0) {
      st->bnorm = sqrt(s);
      st->counter[2] = 0;
    }
  }
}

// zero initial guess: r0 = b, so ||r0|| = ||b||
__global__ void k_beta_is_bnorm(DevState* st) {
  wait_prior_grid();
  st->beta = st->bnorm;
}

__global__ void k_set_target(DevState* st, double tol) {
  wait_prior_grid();
  st->target = tol * st->bnorm;
  st->err = 0;
  st->counter[5] = 0;  // the AMG grid barrier's word (its low 31 bits must start at 0)
  st->k = 0;
  st->hist_base = 0;
}

// start of a cycle: g = (beta, 0, ...), flags cleared
__global__ void k_cycle_start(DevState* st, double* gv, int m) {
  wait_prior_grid();
  for (int i = threadIdx.x; i <= m; i += blockDim.x) gv[i] = (i == 0) ? st->beta : 0.0;
  if (threadIdx.x == 0) {
    st->done = 0;
    st->hist_base += st->k;
    st->k = 0;
    st->happy = 0;
    st->est = st->beta;
    st->vscale[0] = 1.0;
  }
}

// v = src / beta as split pairs in the basis layout
__global__ void k_scale_beta(int64_t n, const double* __restrict__ src, float* __restrict__ v, const DevState* st) {
  wait_prior_grid();
  const double s = st->beta > 0.0 ? 1.0 / st->beta : 0.0;
  const int64_t np = split_pad(n);
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const df t = df_from(src[i] * s);
    v[i] = t.hi;
    v[np + i] = t.lo;
  }
}

// Hessenberg column j from the coefficients col[0..j] and h_{j+1,j} = hn:
// previous rotations, a new one, the residual estimate and the stop flag.
// Runs in one thread.
__device__ void givens_step(DevState* st, double* col, double hn, double* H, double* cs, double* sn, double* gv, int j,
                            int m, int ldh, double* hist) {
  double nrm2 = 0.0;
  for (int i = 0; i <= j; ++i) nrm2 += col[i] * col[i];
  const double wn0 = sqrt(nrm2 + hn * hn);
  for (int i = 0; i < j; ++i) {
    const double a = col[i], b = col[i + 1];
    col[i] = cs[i] * a + sn[i] * b;
    col[i + 1] = -sn[i] * a + cs[i] * b;
  }
  const double a = col[j];
  const double d = hypot(a, hn);
  const double c = d > 0.0 ? a / d : 1.0, s = d > 0.0 ? hn / d : 0.0;
  cs[j] = c;
  sn[j] = s;
  col[j] = d;
  for (int i = 0; i <= j; ++i) H[(size_t)i * ldh + j] = col[i];
  gv[j + 1] = -s * gv[j];
  gv[j] = c * gv[j];
  st->k = j + 1;
  st->est = fabs(gv[j + 1]);
  st->happy = hn <= 1e-14 * wn0;
  st->hn = hn;
  st->scale = hn > 0.0 ? 1.0 / hn : 0.0;
  const int hist_at = st->hist_base + j;
  if (hist && hist_at < kHistCap) hist[hist_at] = st->est;
  const bool bad = !isfinite(st->est) || !isfinite(d) || d == 0.0;
  if (bad) atomicOr(&st->err, kErrNonfinite);
  if (bad || (st->err & kErrTimeout) || st->est <= st->target || st->happy || j + 1 == m) st->done = 1;
}

struct ArnoldiArgs {
  double* H;
  double* cs;
  double* sn;
  double* gv;
  int j, m, ldh;
  double* hist;
};

// Gram-Schmidt coefficient passes: h[off + u] = vscale[u] <V_u, w> for
// u <= j.  Grid (chunks, j + 1): block (c, u) sums column u over chunk c of
// the groups of four entries, B groups per thread at a time with all their
// loads issued first (2 B, or 4 B, 16-byte loads in flight per thread); the
// block that finishes last reduces each column's partials (FP64) with one
// warp per column.  A block streams one contiguous stretch of one column
// (w, read once per column, stays in L2), and the chunk count makes the
// grid about one wave of resident blocks: measured at 3.1M entries, this
// reads the basis at 64-85% of HBM bandwidth for 2-30 columns, against
// 34-36% when every thread reads every column.
//   SPLIT = false: the first pass, on the high planes only (FP32 products
//     and per-thread sums), off = 0, B = 8;
//   SPLIT = true: the second pass of the four-pass form, in split
//     arithmetic (each thread's products and sums as split pairs),
//     off = kMaxM, B = 4.
// The block and chunk sums are FP64 in both.
template <bool SPLIT>
__host__ __device__ constexpr int dot_groups() { return SPLIT ? 4 : 8; }

template <bool SPLIT>
__global__ void __launch_bounds__(kThreads) k_gs_dots(int64_t n, const float* __restrict__ V, int64_t ldv,
                                                     const float* __restrict__ w, double* partials, DevState* st) {
  wait_prior_grid();
  constexpr int kDotB = dot_groups<SPLIT>();
  __shared__ double sh[32];
  if (st->done) return;
  const int nv = gridDim.y;
  const int nchunk = gridDim.x;
  const int u = blockIdx.y;
  const int64_t np = split_pad(n);
  const int64_t ng = (n + 3) >> 2;
  const int64_t len = (ng + nchunk - 1) / nchunk;
  const int64_t g0 = blockIdx.x * len;
  const int64_t g1 = min(ng, g0 + len);
  const float* a = V + (size_t)u * ldv;
  float acc32 = 0.f;
  df acc{0.f, 0.f};
  for (int64_t q0 = g0 + threadIdx.x; q0 < g1; q0 += (int64_t)kDotB * blockDim.x) {
    float4 ah[kDotB], al[kDotB], wh[kDotB], wl[kDotB];
#pragma unroll
    for (int b = 0; b < kDotB; ++b) {
      const int64_t q = q0 + (int64_t)b * blockDim.x;
      const int valid = q < g1 ? (int)min((int64_t)4, n - 4 * q) : 0;
      const int64_t qq = q < g1 ? q : g0;  // an in-range group for the masked lanes
      ah[b] = mask4(ld4(a + 4 * qq), valid);
      wh[b] = mask4(ld4(w + 4 * qq), valid);
      if (SPLIT) {
        al[b] = mask4(ld4(a + np + 4 * qq), valid);
        wl[b] = mask4(ld4(w + np + 4 * qq), valid);
      }
    }
#pragma unroll
    for (int b = 0; b < kDotB; ++b) {
      if (SPLIT) {
        acc = df_fma_acc(acc, df{ah[b].x, al[b].x}, df{wh[b].x, wl[b].x});
        acc = df_fma_acc(acc, df{ah[b].y, al[b].y}, df{wh[b].y, wl[b].y});
        acc = df_fma_acc(acc, df{ah[b].z, al[b].z}, df{wh[b].z, wl[b].z});
        acc = df_fma_acc(acc, df{ah[b].w, al[b].w}, df{wh[b].w, wl[b].w});
      } else {
        acc32 = fmaf(ah[b].w, wh[b].w, fmaf(ah[b].z, wh[b].z, fmaf(ah[b].y, wh[b].y, fmaf(ah[b].x, wh[b].x, acc32))));
      }
    }
  }
  const double sum = block_sum(SPLIT ? df_to_double(df_renorm(acc)) : (double)acc32, sh);
  if (threadIdx.x == 0) partials[(size_t)u * nchunk + blockIdx.x] = sum;
  if (!last_block(&st->counter[0], nchunk * nv)) return;
  const int off = SPLIT ? kMaxM : 0;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int r = warp; r < nv; r += kThreads / 32) {
    double t = 0.0;
    for (int b = lane; b < nchunk; b += 32) t += __ldcg(partials + (size_t)r * nchunk + b);
    t = warp_sum(t);
    if (lane == 0) st->h[off + r] = t * st->vscale[r];
  }
  if (threadIdx.x == 0) st->counter[0] = 0;
}

// CGS2's first update and second coefficient pass in one pass over the
// basis: each thread forms w1 = w - sum_k h[k] vscale[k] V_k for its group of
// four entries (as k_gs_update does), stores it, and sums <V_u, w1> in split
// arithmetic into per-thread accumulators for every column (NVMAX of them,
// the column count rounded up to a bucket), so h[kMaxM + u] needs no second
// pass over w1.  Each V_u is read twice by the thread, the second time from
// cache, so DRAM sees one pass over the basis where the separate update and
// coefficient passes made two.  Both loops take the columns in batches of
// kGsBatch, all of a batch's loads issued before its arithmetic (with a
// conditional load per column the loads of successive columns were not in
// flight together: 40-45% of HBM against 50-56% batched, at 3.1M entries).
// The sums are reduced once, at the end: over the warp by shuffles, over
// the block in shared memory (fixed order), one partial per column and
// block, and the block that finishes last reduces each column's partials.
// Grid: as many blocks as the partials hold for the bucket's columns.
// This form serves up to 16 and more than 32 columns; from 17 to 32,
// k_gs_pass_reg below holds each entry's columns in registers and reads the
// basis once (launch_gs_pass gives the measurements behind the split).
constexpr int kGsBatch = 4;

template <int NVMAX>
__global__ void __launch_bounds__(kThreads) k_gs_pass(int64_t n, const float* __restrict__ V, int64_t ldv,
                                                     float* __restrict__ w, double* partials, DevState* st, int nv) {
  wait_prior_grid();
  constexpr int B = kGsBatch;
  __shared__ df c[kMaxM + 1];
  __shared__ double wacc[kThreads / 32][NVMAX];
  if (st->done) return;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int64_t np = split_pad(n);
  const int64_t ng = (n + 3) >> 2;
  for (int k = threadIdx.x; k < nv; k += blockDim.x) c[k] = df_neg(df_from(st->h[k] * st->vscale[k]));
  __syncthreads();
  df acc[NVMAX];
#pragma unroll
  for (int u = 0; u < NVMAX; ++u) acc[u] = df{0.f, 0.f};
  for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < ng; q += (int64_t)gridDim.x * blockDim.x) {
    const int valid = (int)min((int64_t)4, n - 4 * q);
    const float* a = V + 4 * q;
    const float4 wh = ld4(w + 4 * q), wl = ld4(w + np + 4 * q);
    df s0{wh.x, wl.x}, s1{wh.y, wl.y}, s2{wh.z, wl.z}, s3{wh.w, wl.w};
    for (int k0 = 0; k0 < nv; k0 += B) {
      float4 ah[B], al[B];
#pragma unroll
      for (int b = 0; b < B; ++b) {
        const int k = k0 + b < nv ? k0 + b : nv - 1;  // past the last column: a repeat, not used
        ah[b] = ld4_keep(a + (size_t)k * ldv);
        al[b] = ld4_keep(a + (size_t)k * ldv + np);
      }
#pragma unroll
      for (int b = 0; b < B; ++b) {
        if (k0 + b < nv) {
          const df ck = c[k0 + b];
          s0 = df_fma_acc(s0, ck, df{ah[b].x, al[b].x});
          s1 = df_fma_acc(s1, ck, df{ah[b].y, al[b].y});
          s2 = df_fma_acc(s2, ck, df{ah[b].z, al[b].z});
          s3 = df_fma_acc(s3, ck, df{ah[b].w, al[b].w});
        }
      }
    }
    s0 = df_renorm(s0);
    s1 = df_renorm(s1);
    s2 = df_renorm(s2);
    s3 = df_renorm(s3);
    if (valid == 4) {
      st4(w + 4 * q, make_float4(s0.hi, s1.hi, s2.hi, s3.hi));
      st4(w + np + 4 * q, make_float4(s0.lo, s1.lo, s2.lo, s3.lo));
    } else {
      const df sv[4] = {s0, s1, s2, s3};
      for (int e = 0; e < valid; ++e) {
        w[4 * q + e] = sv[e].hi;
        w[np + 4 * q + e] = sv[e].lo;
      }
    }
    const float4 xh = mask4(make_float4(s0.hi, s1.hi, s2.hi, s3.hi), valid);
    const float4 xl = mask4(make_float4(s0.lo, s1.lo, s2.lo, s3.lo), valid);
#pragma unroll
    for (int k0 = 0; k0 < NVMAX; k0 += B) {
      if (k0 < nv) {
        float4 ah[B], al[B];
#pragma unroll
        for (int b = 0; b < B; ++b) {
          const int k = k0 + b < nv ? k0 + b : nv - 1;
          ah[b] = ld4_last(a + (size_t)k * ldv);
          al[b] = ld4_last(a + (size_t)k * ldv + np);
        }
#pragma unroll
        for (int b = 0; b < B; ++b) {
          const int u = k0 + b;
          if (u < nv) {
            acc[u] = df_fma_acc(acc[u], df{ah[b].x, al[b].x}, df{xh.x, xl.x});
            acc[u] = df_fma_acc(acc[u], df{ah[b].y, al[b].y}, df{xh.y, xl.y});
            acc[u] = df_fma_acc(acc[u], df{ah[b].z, al[b].z}, df{xh.z, xl.z});
            acc[u] = df_fma_acc(acc[u], df{ah[b].w, al[b].w}, df{xh.w, xl.w});
          }
        }
      }
    }
  }
#pragma unroll
  for (int u = 0; u < NVMAX; ++u) {
    if (u < nv) {
      const double p = warp_sum(df_to_double(df_renorm(acc[u])));
      if (lane == 0) wacc[warp][u] = p;
    }
  }
  __syncthreads();
  const int nblk = gridDim.x;
  for (int u = threadIdx.x; u < nv; u += blockDim.x) {
    double t = 0.0;
    for (int r = 0; r < kThreads / 32; ++r) t += wacc[r][u];
    partials[(size_t)u * nblk + blockIdx.x] = t;
  }
  if (!last_block(&st->counter[0], nblk)) return;
  for (int r = warp; r < nv; r += kThreads / 32) {
    double t = 0.0;
    for (int b = lane; b < nblk; b += 32) t += __ldcg(partials + (size_t)r * nblk + b);
    t = warp_sum(t);
    if (lane == 0) st->h[kMaxM + r] = t * st->vscale[r];
  }
  if (threadIdx.x == 0) st->counter[0] = 0;
}

// The same fused pass with each thread's columns held in registers: a
// thread takes one entry at a time, loads that entry of every column
// (high and low planes, all 2 nv loads issued before any arithmetic),
// forms w1, and sums its products with the same registers, so the basis is
// read once and nothing is re-read from cache.  NVMAX is the column count
// rounded up to a multiple of four (loads past the last column repeat it
// and go unused); the registers this takes (two per column for the entries
// and two for the sums) limit it to NVMAX <= 32.  Blocks of kGsRegThreads
// threads, at most 127 registers a thread up to 24 columns (four blocks per
// SM) and 168 above (three).
constexpr int kGsRegThreads = 128;

// a coefficient read from shared memory where it is used: a volatile load
// is not hoisted out of the loop over entries, which would hold every
// coefficient in two registers for the whole kernel (p 8-byte aligned)
__device__ __forceinline__ df ld_shared_df(const df* p) {
  df v;
  asm volatile("ld.shared.v2.f32 {%0,%1}, [%2];" : "=f"(v.hi), "=f"(v.lo) : "r"((unsigned)__cvta_generic_to_shared(p)));
  return v;
}

template <int NVMAX>
__global__ void __launch_bounds__(kGsRegThreads, NVMAX <= 24 ? 4 : 3)
    k_gs_pass_reg(int64_t n, const float* __restrict__ V, int64_t ldv, float* __restrict__ w, double* partials,
                  DevState* st, int nv) {
  wait_prior_grid();
  __shared__ __align__(8) df c[NVMAX];  // 8-byte aligned for ld_shared_df
  __shared__ double wacc[kGsRegThreads / 32][NVMAX];
  if (st->done) return;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int64_t np = split_pad(n);
  for (int k = threadIdx.x; k < nv; k += blockDim.x) c[k] = df_neg(df_from(st->h[k] * st->vscale[k]));
  __syncthreads();
  df acc[NVMAX];
#pragma unroll
  for (int u = 0; u < NVMAX; ++u) acc[u] = df{0.f, 0.f};
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    float vh[NVMAX], vl[NVMAX];
    // one pointer stepped from column to column (past the last column it
    // stays there: a repeat, not used), rather than a 64-bit offset per
    // column that the compiler would keep in registers across entries
    const float* a = V + i;
#pragma unroll
    for (int k = 0; k < NVMAX; ++k) {
      vh[k] = a[0];
      vl[k] = a[np];
      if (k + 1 < nv) a += ldv;
    }
    df s{w[i], w[np + i]};
#pragma unroll
    for (int k = 0; k < NVMAX; ++k)
      if (k < nv) s = df_fma_acc(s, ld_shared_df(&c[k]), df{vh[k], vl[k]});
    s = df_renorm(s);
    w[i] = s.hi;
    w[np + i] = s.lo;
#pragma unroll
    for (int u = 0; u < NVMAX; ++u)
      if (u < nv) acc[u] = df_fma_acc(acc[u], df{vh[u], vl[u]}, s);
  }
#pragma unroll
  for (int u = 0; u < NVMAX; ++u) {
    if (u < nv) {
      const double p = warp_sum(df_to_double(df_renorm(acc[u])));
      if (lane == 0) wacc[warp][u] = p;
    }
  }
  __syncthreads();
  const int nblk = gridDim.x;
  for (int u = threadIdx.x; u < nv; u += blockDim.x) {
    double t = 0.0;
    for (int r = 0; r < kGsRegThreads / 32; ++r) t += wacc[r][u];
    partials[(size_t)u * nblk + blockIdx.x] = t;
  }
  if (!last_block(&st->counter[0], nblk)) return;
  for (int r = warp; r < nv; r += kGsRegThreads / 32) {
    double t = 0.0;
    for (int b = lane; b < nblk; b += 32) t += __ldcg(partials + (size_t)r * nblk + b);
    t = warp_sum(t);
    if (lane == 0) st->h[kMaxM + r] = t * st->vscale[r];
  }
  if (threadIdx.x == 0) st->counter[0] = 0;
}

// launch of the fused pass for nv columns.  The register form serves 17 to
// 32 columns (its bucket rounded up to a multiple of four); up to 16 the
// cached form with four entries per thread is faster (measured at 3.1M
// entries: 322 and 755 us for the columns 1-8 and 9-16 of a 20-iteration
// solve, against 359 and 821 us in registers, whose single dependent chain
// per entry leaves the loads idle), and from 17 on the registers are
// (140 us against 157 us a launch at 17-20 columns, where the cached
// re-reads fall out of L1).  Past 32 columns the registers run out.
void launch_gs_pass(int64_t n, const float* V, int64_t ldv, float* w, double* partials, DevState* st, int nv,
                    cudaStream_t s) {
  const int64_t ng = (n + 3) >> 2;
  // the partials hold (kMaxM + 2) kDotBlocks values: as many blocks per
  // column as fit for the bucket's column count
  auto cached = [&](const void* k, auto kern, int nvmax) {
    const int g = std::min(occ_grid(k, ng), (kMaxM + 2) * kDotBlocks / nvmax);
    (launch_pdl(kern, g, kThreads, 0, s, n, V, ldv, w, partials, st, nv), note_launch());
  };
  auto reg = [&](const void* k, auto kern, int nvmax) {
    const int g = std::min(occ_grid(k, n, kGsRegThreads), (kMaxM + 2) * kDotBlocks / nvmax);
    (launch_pdl(kern, g, kGsRegThreads, 0, s, n, V, ldv, w, partials, st, nv), note_launch());
  };
  if (nv <= 8) cached((const void*)k_gs_pass<8>, k_gs_pass<8>, 8);
  else if (nv <= 16) cached((const void*)k_gs_pass<16>, k_gs_pass<16>, 16);
  else if (nv <= 20) reg((const void*)k_gs_pass_reg<20>, k_gs_pass_reg<20>, 20);
  else if (nv <= 24) reg((const void*)k_gs_pass_reg<24>, k_gs_pass_reg<24>, 24);
  else if (nv <= 28) reg((const void*)k_gs_pass_reg<28>, k_gs_pass_reg<28>, 28);
  else if (nv <= 32) reg((const void*)k_gs_pass_reg<32>, k_gs_pass_reg<32>, 32);
  else cached((const void*)k_gs_pass<kMaxM + 1>, k_gs_pass<kMaxM + 1>, kMaxM + 1);
}

// Gram-Schmidt update pass: w -= sum_u h[off + u] vscale[u] V_u in split
// arithmetic (the coefficients rounded to split pairs once per block, each
// entry's sum carried as a split pair and renormalised once), four entries
// per thread, the columns in batches of kGsBatch with all of a batch's loads
// issued first (78-95% of HBM for 10-30 columns at 3.1M entries, against
// 70-79% two columns at a time).  In the final pass (LAST) ||w||^2 is
// reduced in FP64 and the last block applies the Givens step to h1 + h2 and
// stores 1/||w|| as the new column's scale (w itself stays unnormalised).
// The squares are summed in split arithmetic (FP32 instructions only; GB300's
// FP64 pipe is narrow and this pass runs for every column) for groups whose
// high parts all lie in [2^-50, 2^56] (or are zero), so every square and its
// rounding error stay normal FP32 numbers and a thread's sum of up to 2^15
// of them stays in range, and in FP64 for any other group; both keep about
// 2^-46 of each term.  (A squared norm summed from the high parts
// alone in FP32 has stalled ill-conditioned solves.)
template <bool LAST>
__global__ void __launch_bounds__(kThreads) k_gs_update(int64_t n, const float* __restrict__ V, int64_t ldv,
                                                       float* __restrict__ w, double* partials, DevState* st,
                                                       ArnoldiArgs aa) {
  wait_prior_grid();
  constexpr int B = kGsBatch;
  __shared__ df c[kMaxM + 1];
  __shared__ double sh[32];
  if (st->done) return;
  const int nv = aa.j + 1;
  const int off = LAST ? kMaxM : 0;
  const int64_t np = split_pad(n);
  const int64_t ng = (n + 3) >> 2;
  for (int k = threadIdx.x; k < nv; k += blockDim.x) c[k] = df_neg(df_from(st->h[off + k] * st->vscale[k]));
  __syncthreads();
  double acc = 0.0;  // squares of the groups outside the split range
  df accs{0.f, 0.f};  // squares in split arithmetic
  for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < ng; q += (int64_t)gridDim.x * blockDim.x) {
    const float4 wh = ld4(w + 4 * q), wl = ld4(w + np + 4 * q);
    df s0{wh.x, wl.x}, s1{wh.y, wl.y}, s2{wh.z, wl.z}, s3{wh.w, wl.w};
    const float* a = V + 4 * q;
    for (int k0 = 0; k0 < nv; k0 += B) {
      float4 ah[B], al[B];
#pragma unroll
      for (int b = 0; b < B; ++b) {
        const int k = k0 + b < nv ? k0 + b : nv - 1;  // past the last column: a repeat, not used
        ah[b] = ld4(a + (size_t)k * ldv);
        al[b] = ld4(a + (size_t)k * ldv + np);
      }
#pragma unroll
      for (int b = 0; b < B; ++b) {
        if (k0 + b < nv) {
          const df ck = c[k0 + b];
          s0 = df_fma_acc(s0, ck, df{ah[b].x, al[b].x});
          s1 = df_fma_acc(s1, ck, df{ah[b].y, al[b].y});
          s2 = df_fma_acc(s2, ck, df{ah[b].z, al[b].z});
          s3 = df_fma_acc(s3, ck, df{ah[b].w, al[b].w});
        }
      }
    }
    s0 = df_renorm(s0);
    s1 = df_renorm(s1);
    s2 = df_renorm(s2);
    s3 = df_renorm(s3);
    const int valid = (int)min((int64_t)4, n - 4 * q);
    if (valid == 4) {
      st4(w + 4 * q, make_float4(s0.hi, s1.hi, s2.hi, s3.hi));
      st4(w + np + 4 * q, make_float4(s0.lo, s1.lo, s2.lo, s3.lo));
    } else {
      const df sv[4] = {s0, s1, s2, s3};
      for (int e = 0; e < valid; ++e) {
        w[4 * q + e] = sv[e].hi;
        w[np + 4 * q + e] = sv[e].lo;
      }
    }
    if (LAST) {
      const float4 xh = mask4(make_float4(s0.hi, s1.hi, s2.hi, s3.hi), valid);
      const float4 xl = mask4(make_float4(s0.lo, s1.lo, s2.lo, s3.lo), valid);
      const df e[4] = {{xh.x, xl.x}, {xh.y, xl.y}, {xh.z, xl.z}, {xh.w, xl.w}};
      bool safe = true;
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        const float m = fabsf(e[i].hi);
        safe = safe && (m == 0.f || (m >= 0x1p-50f && m <= 0x1p56f));
      }
      if (safe) {
#pragma unroll
        for (int i = 0; i < 4; ++i) accs = df_fma_acc(accs, e[i], e[i]);
      } else {
#pragma unroll
        for (int i = 0; i < 4; ++i) {
          const double d = df_to_double(e[i]);
          acc = fma(d, d, acc);
        }
      }
    }
  }
  if (!LAST) return;
  acc = block_sum(acc + df_to_double(df_renorm(accs)), sh);
  if (threadIdx.x == 0) partials[blockIdx.x] = acc;
  if (!last_block(&st->counter[3], gridDim.x)) return;
  const double hn2 = reduce_partials(partials, gridDim.x, sh);
  if (threadIdx.x != 0) return;
  st->counter[3] = 0;
  double col[kMaxM + 1];
  for (int u = 0; u < nv; ++u) col[u] = st->h[u] + st->h[kMaxM + u];
  const double hn = sqrt(hn2);
  givens_step(st, col, hn, aa.H, aa.cs, aa.sn, aa.gv, aa.j, aa.m, aa.ldh, aa.hist);
  st->vscale[aa.j + 1] = hn > 0.0 ? 1.0 / hn : 0.0;
}

// chunks per column of a coefficient pass over nv columns: about one wave of
// resident blocks in all, at most kDotBlocks per column (the partials' room)
template <bool SPLIT>
int gs_chunks(int64_t n, int nv) {
  const int64_t ng = (n + 3) >> 2;
  int64_t c = occ_grid((const void*)k_gs_dots<SPLIT>, ng) / nv;
  const int64_t most = (ng + (int64_t)dot_groups<SPLIT>() * kThreads - 1) / ((int64_t)dot_groups<SPLIT>() * kThreads);
  if (c > most) c = most;
  if (c > kDotBlocks) c = kDotBlocks;
  if (c < 1) c = 1;
  return (int)c;
}

// The device state copied into its pinned host mirror by a kernel: the
// host reads the mirror after an event behind this kernel.  A copy engine
// transfer in the stream between two kernels costs about 7.5 us of stream
// time on GB300 against about 1.2 us for this kernel, and it would also end
// the chain of programmatically dependent launches.
static_assert(sizeof(DevState) % 8 == 0, "DevState is copied as 8-byte words");
__global__ void k_publish(const DevState* st, DevState* host) {
  wait_prior_grid();
  const unsigned long long* src = reinterpret_cast<const unsigned long long*>(st);
  unsigned long long* dst = reinterpret_cast<unsigned long long*>(host);
  for (int i = threadIdx.x; i < (int)(sizeof(DevState) / 8); i += blockDim.x) dst[i] = src[i];
  __threadfence_system();
}

// the device state into host slot `slot` (the kernel above where the
// mirror has a device address, else a copy)
void publish_state(bo_prec* P, const DevState* st, int slot, cudaStream_t s) {
  if (P->h_st_dev) (launch_pdl(k_publish, 1, 128, 0, s, st, P->h_st_dev + slot), note_launch());
  else cudaMemcpyAsync(&P->h_st[slot], st, sizeof(DevState), cudaMemcpyDeviceToHost, s);
}

// y = H(0:k, 0:k)^{-1} g (upper triangular after the rotations)
__global__ void k_trisolve(DevState* st, const double* H, const double* gv, double* y, int ldh) {
  wait_prior_grid();
  if (threadIdx.x != 0) return;
  if (st->err & kErrNonfinite) { st->k = 0; return; }
  const int k = st->k;
  for (int i = k - 1; i >= 0; --i) {
    double s = gv[i];
    for (int t = i + 1; t < k; ++t) s -= H[(size_t)i * ldh + t] * y[t];
    y[i] = s / H[(size_t)i * ldh + i];
  }
}

// sum_{k < nv} c_k V_k[i] in split arithmetic (nv <= NU), in batches of B
// columns: each batch's 2 B loads are unconditional (past the last column
// they repeat it, unused), so all of them are in flight at once; only the
// arithmetic carries the bound
template <int NU, int B = NU>
__device__ __forceinline__ df lincomb(const df* c, const float* __restrict__ V, int64_t ldv, int64_t n, int64_t i,
                                      int nv) {
  df s{0.f, 0.f};
#pragma unroll 1
  for (int k0 = 0; k0 < NU; k0 += B) {
    if (k0 >= nv) break;
    float vh[B], vl[B];
#pragma unroll
    for (int k = 0; k < B; ++k) {
      const float* a = V + (size_t)(k0 + k < nv ? k0 + k : nv - 1) * ldv;
      vh[k] = a[i];
      vl[k] = a[n + i];
    }
#pragma unroll
    for (int k = 0; k < B; ++k)
      if (k0 + k < nv) s = df_fma_acc(s, c[k0 + k], df{vh[k], vl[k]});
  }
  return df_norm(s);
}

// x += sum_{l < k} y_l Z_l: the sum in split arithmetic (Z split pairs,
// ldz floats apart), added to the FP64 iterate
template <int NU>
__global__ void __launch_bounds__(kThreads, 2) k_xupdate(int64_t n, double* __restrict__ x, const float* __restrict__ Z, int64_t ldz,
                          const double* __restrict__ y, const DevState* st) {
  wait_prior_grid();
  __shared__ df ys[kMaxM];
  const int k = st->k;
  for (int l = threadIdx.x; l < k; l += blockDim.x) ys[l] = df_from(y[l]);
  __syncthreads();
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    x[i] += df_to_double(lincomb<NU, 16>(ys, Z, ldz, n, i, k));
}

}  // namespace

// process-wide source of graph generations: a preconditioner created at the
// address of a freed one never matches graphs recorded for the old one
std::atomic<unsigned long long> g_graph_gen{0};

void graphs_reset(bo_prec* P) {
  P->graph_gen = ++g_graph_gen;  // batch graphs recorded with this preconditioner are stale
  for (int j = 0; j < 64; ++j)
    if (P->col_exec[j]) {
      cudaGraphExecDestroy(P->col_exec[j]);
      P->col_exec[j] = nullptr;
    }
  P->graph_m = 0;
}

int krylov_alloc(bo_prec* P, int m) {
  if (P->mcap >= m && P->V) return BO_OK;
  graphs_reset(P);
  const Geom& g = P->mat->g;
  const int64_t n = 3 * g.N;
  auto fr = [](void* p) { if (p) cudaFree(p); };
  fr(P->V); fr(P->Vs); fr(P->Z); fr(P->H); fr(P->cs); fr(P->sn); fr(P->gvec); fr(P->y);
  P->V = nullptr; P->Vs = nullptr; P->Z = nullptr;
  bool ok = true;
  auto al = [&](size_t bytes) -> void* {
    void* p = nullptr;
    if (ok && cudaMalloc(&p, bytes) != cudaSuccess) { ok = false; return nullptr; }
    return p;
  };
  P->V = (double*)al((size_t)(m + 1) * split_pad(n) * sizeof(double));  // split pairs (FGMRES) or FP64 (BiCGSTAB)
  P->Vs = nullptr;
  P->Z = (double*)al((size_t)m * n * sizeof(double));
  P->H = (double*)al((size_t)(m + 1) * m * sizeof(double));
  P->cs = (double*)al((size_t)m * sizeof(double));
  P->sn = (double*)al((size_t)m * sizeof(double));
  P->gvec = (double*)al((size_t)(m + 1) * sizeof(double));
  P->y = (double*)al((size_t)m * sizeof(double));
  if (!P->xi) {
    P->xi = (double*)al((size_t)n * sizeof(double));
    P->bi = (double*)al((size_t)n * sizeof(double));
    P->rk = (double*)al((size_t)n * sizeof(double));
    P->npartials = (int64_t)(kMaxM + 2) * kDotBlocks + kHistCap;
    P->partials = (double*)al((size_t)P->npartials * sizeof(double));
    P->hostio = (double*)al((size_t)2 * n * sizeof(double));
    if (ok && cudaMallocHost(&P->h_st, 4 * sizeof(DevState)) != cudaSuccess) ok = false;
    if (ok && cudaHostGetDevicePointer((void**)&P->h_st_dev, P->h_st, 0) != cudaSuccess) {
      P->h_st_dev = nullptr;  // not mapped: copies instead
      cudaGetLastError();
    }
    if (ok)
      for (int e = 0; e < 4; ++e) cudaEventCreateWithFlags(&P->ev[e], cudaEventDisableTiming);
    P->hist_cap = kHistCap;
    P->hist = new double[kHistCap];
  }
  P->mcap = ok ? m : 0;
  return ok ? BO_OK : BO_ERR_OOM;
}

// One FGMRES solve as a resumable state machine.  advance() enqueues the
// next piece of work on the preconditioner's stream and checks the events
// of earlier pieces; with block = false it never waits, so many jobs on
// different streams can be driven round-robin by one host thread
// (bo_solve_batched); with block = true it waits on the oldest event it
// needs, which gives the single-solve path its one-column polling lag.
namespace {

constexpr int kRing = 3;        // status slots / events for columns
constexpr int kPhaseSlot = 3;   // status slot / event for the other phases

struct Job {
  enum Phase { kStart, kInitWait, kColumns, kCycleWait, kFinalWait, kDone };
  bo_prec* P = nullptr;
  const double* b_in = nullptr;
  double* x_in = nullptr;
  bo_solve_opts o;
  bo_solve_info* info = nullptr;
  const double* b_d = nullptr;
  double* x_d = nullptr;
  Phase phase = kStart;
  double bnorm = 0, beta = 0, est = 0, target = 0;
  int status = BO_OK, its = 0, restarts = 0;
  int j_enq = 0, j_polled = 0;
  bool cycle_stop = false, profile = false;
  std::vector<std::pair<cudaEvent_t, cudaEvent_t>> prof;
  std::chrono::steady_clock::time_point t0;

  cudaStream_t stream() const { return P->stream; }
  const Geom& geom() const { return P->mat->g; }
  int64_t n() const { return 3 * P->mat->g.N; }

  bool ready(cudaEvent_t e, bool block) {
    const cudaError_t r = block ? cudaEventSynchronize(e) : cudaEventQuery(e);
    if (r == cudaSuccess) return true;
    if (r != cudaErrorNotReady) fail(BO_ERR_CUDA);
    return false;
  }

  void fail(int st) {
    status = st;
    phase = kDone;
  }

  void mark(int slot) {
    publish_state(P, P->st, slot, stream());
    cudaEventRecord(P->ev[slot], stream());
  }

  void start() {
    t0 = std::chrono::steady_clock::now();
    cudaStream_t s = stream();
    if (!P->mat->a2_valid) launch_split_matrix(P->mat, s);
    const Geom& g = geom();
    const int64_t nn = n();
    DevState* st = P->st;
    b_d = b_in;
    x_d = x_in;
    if (o.mem == BO_MEM_HOST) {
      cudaMemcpyAsync(P->hostio, b_in, nn * sizeof(double), cudaMemcpyHostToDevice, s);
      b_d = P->hostio;
      x_d = P->hostio + nn;
      if (!o.x0_is_zero) cudaMemcpyAsync(x_d, x_in, nn * sizeof(double), cudaMemcpyHostToDevice, s);
    }
    launch_gather(g, b_d, P->bi, s);
    if (o.x0_is_zero) cudaMemsetAsync(P->xi, 0, nn * sizeof(double), s);
    else launch_gather(g, x_d, P->xi, s);
    (launch_pdl(k_norm, kRedBlocks, kThreads, 0, s, nn, P->bi, P->partials, st), note_launch());
    (launch_pdl(k_set_target, 1, 1, 0, s, st, o.tol), note_launch());
    if (o.x0_is_zero) {  // r0 = b: no pass over the matrix
      cudaMemcpyAsync(P->rk, P->bi, nn * sizeof(double), cudaMemcpyDeviceToDevice, s);
      (launch_pdl(k_beta_is_bnorm, 1, 1, 0, s, st), note_launch());
    } else {
      (launch_pdl(k_true_residual, kRedBlocks, kThreads, 0, s, g, P->mat->A, P->bi, P->xi, P->rk, P->partials, st),
       note_launch());
      if (P->wl) wells_after_residual(P);
    }
    mark(kPhaseSlot);
    P->nhist = 0;
    phase = kInitWait;
  }

  void start_cycle() {
    cudaStream_t s = stream();
    (launch_pdl(k_cycle_start, 1, 64, 0, s, P->st, P->gvec, o.restart), note_launch());
    (launch_pdl(k_scale_beta, grid_for(n()), kThreads, 0, s, n(), P->rk, (float*)P->V, P->st), note_launch());
    j_enq = j_polled = 0;
    cycle_stop = false;
    phase = kColumns;
  }

  // the kernels of Arnoldi column j on the preconditioner's stream
  void enqueue_column_kernels(int j, bool timed) {
    cudaStream_t s = stream();
    const Geom& g = geom();
    const int64_t nn = n(), ldv = 2 * split_pad(nn);  // basis vectors as split pairs (split_pad)
    const int m = o.restart;
    DevState* st = P->st;
    float* V = (float*)P->V;
    const float* vj = V + (size_t)j * ldv;
    float* w = V + (size_t)(j + 1) * ldv;
    float* zj = (float*)P->Z + (size_t)j * 2 * nn;  // split pairs: hi plane, lo plane
    double* dhist = P->partials + (P->npartials - kHistCap);
    launch_cpr_split_in(P, vj, zj, st, &st->vscale[j]);
    if (P->wl) wells_after_prec(P, zj, nn);
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (timed && prof.size() < 512) {
      e0 = P->prof_ev[2 * prof.size()];
      e1 = P->prof_ev[2 * prof.size() + 1];
      cudaEventRecord(e0, s);
    }
    (launch_pdl(k_arnoldi_spmv<float>, occ_grid((const void*)k_arnoldi_spmv<float>, g.N), kThreads, 0, s, 
         g, P->mat->A2, P->mat->A, P->mat->a2_range, zj, w, st),
     note_launch());
    if (e1) {
      cudaEventRecord(e1, s);
      prof.push_back({e0, e1});
    }
    if (P->wl) wells_after_product(P, w, split_pad(nn));
    const ArnoldiArgs aa{P->H, P->cs, P->sn, P->gvec, j, m, m, dhist};
    const int nv = j + 1;
    const int gu = occ_grid((const void*)k_gs_update<true>, nn);
    if (g_gs_fused.load()) {
      // CGS2 in three passes over the basis: the first coefficients, the
      // first update fused with the second coefficients, the final update
      (launch_pdl(k_gs_dots<false>, dim3(gs_chunks<false>(nn, nv), nv), kThreads, 0, s, nn, V, ldv, w, P->partials, st),
       note_launch());
      launch_gs_pass(nn, V, ldv, w, P->partials, st, nv, s);
    } else {
      (launch_pdl(k_gs_dots<false>, dim3(gs_chunks<false>(nn, nv), nv), kThreads, 0, s, nn, V, ldv, w, P->partials, st),
       note_launch());
      (launch_pdl(k_gs_update<false>, gu, kThreads, 0, s, nn, V, ldv, w, P->partials, st, aa), note_launch());
      (launch_pdl(k_gs_dots<true>, dim3(gs_chunks<true>(nn, nv), nv), kThreads, 0, s, nn, V, ldv, w, P->partials, st),
       note_launch());
    }
    (launch_pdl(k_gs_update<true>, gu, kThreads, 0, s, nn, V, ldv, w, P->partials, st, aa), note_launch());
  }

  // Column j's kernels captured once into a CUDA graph (on a private stream,
  // since the preconditioner's stream may be the legacy default stream) and
  // instantiated; valid while the workspace and restart length stay put.
  bool ensure_graph(int j) {
    const int m = o.restart;
    if (P->graph_m != m || P->graph_wl != P->wl) {
      graphs_reset(P);
      P->graph_m = m;
      P->graph_wl = P->wl;
    }
    if (P->col_exec[j]) return true;
    if (!P->cap_stream && cudaStreamCreateWithFlags(&P->cap_stream, cudaStreamNonBlocking) != cudaSuccess) return false;
    cudaStream_t saved = P->stream;
    P->stream = P->cap_stream;
    const long long l0 = g_launches.load();
    if (cudaStreamBeginCapture(P->cap_stream, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
      P->stream = saved;
      return false;
    }
    enqueue_column_kernels(j, false);
    cudaGraph_t gr = nullptr;
    const cudaError_t e = cudaStreamEndCapture(P->cap_stream, &gr);
    P->stream = saved;
    const long long nodes = g_launches.load() - l0;
    g_launches.fetch_sub(nodes);  // captured, not run: counted at each replay instead
    if (e != cudaSuccess || !gr) return false;
    const cudaError_t ei = cudaGraphInstantiate(&P->col_exec[j], gr, 0);
    cudaGraphDestroy(gr);
    if (ei != cudaSuccess) {
      P->col_exec[j] = nullptr;
      return false;
    }
    P->col_nodes[j] = nodes;
    return true;
  }

  void enqueue_column(int j) {
    if (P->launch_mode == BO_LAUNCH_GRAPH && !profile) {
      if (!ensure_graph(j)) {
        fail(BO_ERR_CUDA);
        return;
      }
      if (cudaGraphLaunch(P->col_exec[j], stream()) != cudaSuccess) {
        fail(BO_ERR_CUDA);
        return;
      }
      g_launches.fetch_add(P->col_nodes[j]);
    } else {
      enqueue_column_kernels(j, profile);
    }
    mark(j % kRing);
  }

  void end_cycle() {
    cudaStream_t s = stream();
    const int64_t nn = n();
    const int gn = grid_for(nn);
    (launch_pdl(k_trisolve, 1, 32, 0, s, P->st, P->H, P->gvec, P->y, o.restart), note_launch());
    const float* Z = (const float*)P->Z;
    if (o.restart <= 16) (launch_pdl(k_xupdate<16>, gn, kThreads, 0, s, nn, P->xi, Z, 2 * nn, P->y, P->st), note_launch());
    else if (o.restart <= 32) (launch_pdl(k_xupdate<32>, gn, kThreads, 0, s, nn, P->xi, Z, 2 * nn, P->y, P->st), note_launch());
    else (launch_pdl(k_xupdate<kMaxM>, gn, kThreads, 0, s, nn, P->xi, Z, 2 * nn, P->y, P->st), note_launch());
    (launch_pdl(k_true_residual, kRedBlocks, kThreads, 0, s, geom(), P->mat->A, P->bi, P->xi, P->rk, P->partials, P->st),
     note_launch());
    if (P->wl) wells_after_residual(P);
    mark(kPhaseSlot);
    phase = kCycleWait;
  }

  void finish() {
    cudaStream_t s = stream();
    if (status == BO_OK && bnorm > 0 && beta > target) status = BO_ERR_NOT_CONVERGED;
    launch_scatter(geom(), P->xi, x_d, s);
    if (o.mem == BO_MEM_HOST) cudaMemcpyAsync(x_in, x_d, n() * sizeof(double), cudaMemcpyDeviceToHost, s);
    cudaEventRecord(P->ev[kPhaseSlot], s);
    phase = kFinalWait;
  }

  void done() {
    const int nh = its < kHistCap ? its : kHistCap;
    if (nh > 0 && bnorm > 0) {
      cudaMemcpy(P->hist, P->partials + (P->npartials - kHistCap), nh * sizeof(double), cudaMemcpyDeviceToHost);
      for (int i = 0; i < nh; ++i) P->hist[i] /= bnorm;
    }
    P->nhist = nh > 0 ? nh : 0;
    if (info) {
      info->status = status;
      info->iters = its;
      info->restarts = restarts;
      info->true_rel_res = bnorm > 0 ? beta / bnorm : beta;
      info->est_rel_res = bnorm > 0 ? est / bnorm : est;
      info->spmv_launches = 0;
      info->spmv_ms = 0.0;
      for (size_t i = 0; i < prof.size(); ++i) {
        if ((int)i < its) {
          float ms = 0.f;
          cudaEventElapsedTime(&ms, prof[i].first, prof[i].second);
          info->spmv_ms += ms;
          info->spmv_launches++;
        }
      }
      info->solve_ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
    }
    phase = kDone;
  }

  // one step of progress; returns whether anything happened
  bool advance(bool block) {
    switch (phase) {
      case kStart:
        start();
        return true;
      case kInitWait: {
        if (!ready(P->ev[kPhaseSlot], block)) return false;
        const DevState& h = P->h_st[kPhaseSlot];
        bnorm = h.bnorm;
        beta = est = h.beta;
        if (!std::isfinite(bnorm) || !std::isfinite(beta)) {
          status = BO_ERR_NONFINITE;
          finish();
        } else if (bnorm == 0.0) {
          cudaMemsetAsync(P->xi, 0, n() * sizeof(double), stream());
          beta = 0.0;
          finish();
        } else {
          target = o.tol * bnorm;
          if (beta <= target || its >= o.maxit) finish();
          else start_cycle();
        }
        return true;
      }
      case kColumns: {
        bool moved = false;
        const int m = o.restart;
        while (!cycle_stop && j_enq < m && its + j_enq < o.maxit && j_enq - j_polled < 2) {
          enqueue_column(j_enq++);
          moved = true;
        }
        while (j_polled < j_enq && !cycle_stop) {
          // the single-solve path waits only for the column before the newest
          const bool may_block = block && (j_enq - j_polled >= 2 || j_enq == m || its + j_enq >= o.maxit);
          if (!ready(P->ev[j_polled % kRing], may_block)) break;
          if (P->h_st[j_polled % kRing].done) cycle_stop = true;
          ++j_polled;
          moved = true;
        }
        if (phase == kDone) return true;
        if (cycle_stop || j_enq == m || its + j_enq >= o.maxit) {
          end_cycle();
          moved = true;
        }
        return moved;
      }
      case kCycleWait: {
        if (!ready(P->ev[kPhaseSlot], block)) return false;
        const DevState& h = P->h_st[kPhaseSlot];
        ++restarts;
        its += h.k;
        const double prev = beta;
        beta = h.beta;
        est = h.est;
        if (h.err & kErrTimeout) {
          status = BO_ERR_TIMEOUT;
          finish();
        } else if (h.err & kErrNonfinite) {
          status = BO_ERR_BREAKDOWN;
          finish();
        } else if (h.k == 0 || beta <= target || its >= o.maxit) {
          finish();
        } else if (h.k == o.restart && beta > 0.99 * prev) {
          finish();  // a full cycle gained under 1%: stagnation, report NOT_CONVERGED
        } else {
          start_cycle();
        }
        return true;
      }
      case kFinalWait:
        if (!ready(P->ev[kPhaseSlot], block)) return false;
        done();
        return true;
      case kDone:
        return false;
    }
    return false;
  }
};

}  // namespace

namespace {
// v (FP64, internal order) -> split pairs: hi plane z[0..n), lo plane z[n..2n)
__global__ void k_split_vec(int64_t n, const double* __restrict__ v, float* __restrict__ z) {
  wait_prior_grid();
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    int bad = 0;
    const float2 p = df_split_bits(v[i], &bad);
    z[i] = p.x;
    z[n + i] = p.y;
  }
}
// w = hi + lo (exact in FP64) of a vector in the basis layout
__global__ void k_join_vec(int64_t n, const float* __restrict__ z, double* __restrict__ w) {
  wait_prior_grid();
  const int64_t np = split_pad(n);
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    w[i] = (double)z[i] + (double)z[np + i];
}
}  // namespace

// w = A v on internal vectors by the solver's own Arnoldi product: v split
// into pairs, the kernel every FGMRES iteration runs, its split result
// joined exactly into FP64 w
void launch_arnoldi_product(bo_prec* P, const double* v, double* w) {
  cudaStream_t s = P->stream;
  bo_mat* m = P->mat;
  const Geom& g = m->g;
  const int64_t n = 3 * g.N;
  if (!m->a2_valid) launch_split_matrix(m, s);
  float* z = (float*)P->Z;  // the first preconditioned vector's split planes as scratch
  float* ws = (float*)P->V;  // the first basis vector's split planes as scratch
  (launch_pdl(k_split_vec, grid_for(n), kThreads, 0, s, n, v, z), note_launch());
  (launch_pdl(k_arnoldi_spmv<float>, occ_grid((const void*)k_arnoldi_spmv<float>, g.N), kThreads, 0, s, 
       g, m->A2, m->A, m->a2_range, z, ws, P->st),
   note_launch());
  (launch_pdl(k_join_vec, grid_for(n), kThreads, 0, s, n, ws, w), note_launch());
}

int fgmres(bo_prec* P, const double* b_in, double* x_in, const bo_solve_opts* o, bo_solve_info* info) {
  int rc = krylov_alloc(P, o->restart);
  if (rc != BO_OK) return rc;
  if (o->profile && !P->prof_ready) {
    for (int i = 0; i < 2 * 512; ++i) cudaEventCreate(&P->prof_ev[i]);
    P->prof_ready = true;
  }
  Job job;
  job.P = P;
  job.b_in = b_in;
  job.x_in = x_in;
  job.o = *o;
  job.info = info;
  job.profile = o->profile != 0;
  while (job.phase != Job::kDone) job.advance(true);
  if (job.status == BO_ERR_CUDA && info) info->status = BO_ERR_CUDA;
  return job.status;
}

// ---------------------------------------------------------------- BiCGSTAB
// Right-preconditioned BiCGSTAB (van der Vorst, SIAM J. Sci. Stat. Comput.
// 13, 1992) with the same CPR preconditioner: the solver of the paper's
// scalability experiments (Sec. 4).  Each iteration takes the BiCG step
// p -> v = A M^{-1} p with alpha = rho / (rt, v) and the minimal-residual
// step s -> t = A M^{-1} s with omega = (t, s) / (t, t).  The recurrence
// vectors and scalars are FP64; the preconditioned vectors are the CPR's
// split-pair output and the products use the Arnoldi SpMV.  The scalars
// live in the device state and the host polls one iteration behind, as in
// FGMRES.  When the recursive residual meets tol ||b||, or a scalar of the
// recurrence vanishes, the cycle ends: the true FP64 residual is recomputed
// and, if it is above the target, the iteration restarts from it with a new
// shadow vector.
namespace {

// scalar slots of DevState::h used by BiCGSTAB
enum : int { kBcRho = 0, kBcRhoPrev, kBcAlpha, kBcOmega, kBcBeta, kBcRtv, kBcSs, kBcTs, kBcTt, kBcRr, kBcReason };
// why a cycle stopped (h[kBcReason])
enum : int { kBcGoing = 0, kBcSDone = 1, kBcRDone = 2, kBcBroke = 3 };

// h[o1] = a . b and, with c, h[o2] = c . d; per-block partials reduced in a
// fixed order by the block that finishes last
__global__ void __launch_bounds__(kThreads) k_bc_dots(int64_t n, const double* __restrict__ a,
                                                     const double* __restrict__ b, const double* __restrict__ c,
                                                     const double* __restrict__ d, double* partials, DevState* st,
                                                     int o1, int o2) {
  wait_prior_grid();
  __shared__ double sh[32];
  if (st->done) return;
  double s1 = 0.0, s2 = 0.0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    s1 = fma(a[i], b[i], s1);
    if (c) s2 = fma(c[i], d[i], s2);
  }
  s1 = block_sum(s1, sh);
  s2 = block_sum(s2, sh);
  if (threadIdx.x == 0) {
    partials[blockIdx.x] = s1;
    partials[gridDim.x + blockIdx.x] = s2;
  }
  if (!last_block(&st->counter[4], gridDim.x)) return;
  const double t1 = reduce_partials(partials, gridDim.x, sh);
  const double t2 = reduce_partials(partials + gridDim.x, gridDim.x, sh);
  if (threadIdx.x == 0) {
    st->h[o1] = t1;
    if (o2 >= 0) st->h[o2] = t2;
    st->counter[4] = 0;
  }
}

// the scalar steps of an iteration (one thread)
template <int PHASE>
__global__ void k_bc_scalar(DevState* st) {
  wait_prior_grid();
  if (st->done) return;
  double* h = st->h;
  auto stop = [&](int why) {
    h[kBcReason] = why;
    st->done = 1;
  };
  if (PHASE == 0) {  // rho = (rt, r) -> beta
    if (h[kBcRho] == 0.0 || !isfinite(h[kBcRho])) return stop(kBcBroke);
    h[kBcBeta] = (h[kBcRho] / h[kBcRhoPrev]) * (h[kBcAlpha] / h[kBcOmega]);
  } else if (PHASE == 1) {  // (rt, v) -> alpha
    if (h[kBcRtv] == 0.0 || !isfinite(h[kBcRtv])) return stop(kBcBroke);
    h[kBcAlpha] = h[kBcRho] / h[kBcRtv];
  } else if (PHASE == 2) {  // ||s||: the BiCG half step counts as the iteration
    st->k += 1;
    if (!isfinite(h[kBcSs])) return stop(kBcBroke);
    if (sqrt(h[kBcSs]) <= st->target) return stop(kBcSDone);
  } else if (PHASE == 3) {  // omega = (t, s) / (t, t)
    if (h[kBcTt] == 0.0 || !isfinite(h[kBcTt])) return stop(kBcSDone);  // t = 0: keep the half step
    h[kBcOmega] = h[kBcTs] / h[kBcTt];
  } else {  // ||r||
    h[kBcRhoPrev] = h[kBcRho];
    if (!isfinite(h[kBcRr])) return stop(kBcBroke);
    if (sqrt(h[kBcRr]) <= st->target || h[kBcOmega] == 0.0) return stop(kBcRDone);
  }
}

// p = r + beta (p - omega v)
__global__ void k_bc_p(int64_t n, const double* __restrict__ r, double* __restrict__ p, const double* __restrict__ v,
                       const DevState* st) {
  wait_prior_grid();
  if (st->done) return;
  const double beta = st->h[kBcBeta], omega = st->h[kBcOmega];
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    p[i] = r[i] + beta * (p[i] - omega * v[i]);
}

// s = r - alpha v and h[kBcSs] = ||s||^2
__global__ void __launch_bounds__(kThreads) k_bc_s(int64_t n, const double* __restrict__ r,
                                                  const double* __restrict__ v, double* __restrict__ s,
                                                  double* partials, DevState* st) {
  wait_prior_grid();
  __shared__ double sh[32];
  if (st->done) return;
  const double alpha = st->h[kBcAlpha];
  double acc = 0.0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const double t = r[i] - alpha * v[i];
    s[i] = t;
    acc = fma(t, t, acc);
  }
  acc = block_sum(acc, sh);
  if (threadIdx.x == 0) partials[blockIdx.x] = acc;
  if (!last_block(&st->counter[4], gridDim.x)) return;
  const double tot = reduce_partials(partials, gridDim.x, sh);
  if (threadIdx.x == 0) {
    st->h[kBcSs] = tot;
    st->counter[4] = 0;
  }
}

__device__ __forceinline__ double split_at(const float* z, int64_t n, int64_t i) {
  return (double)z[i] + (double)z[n + i];
}

// x += alpha p^ + omega s^, r = s - omega t and h[kBcRr] = ||r||^2 (p^, s^
// split pairs)
__global__ void __launch_bounds__(kThreads) k_bc_xr(int64_t n, double* __restrict__ x, const float* __restrict__ ph,
                                                   const float* __restrict__ shs, const double* __restrict__ s,
                                                   const double* __restrict__ t, double* __restrict__ r,
                                                   double* partials, DevState* st) {
  wait_prior_grid();
  __shared__ double sh[32];
  if (st->done) return;
  const double alpha = st->h[kBcAlpha], omega = st->h[kBcOmega];
  double acc = 0.0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    x[i] += alpha * split_at(ph, n, i) + omega * split_at(shs, n, i);
    const double ri = s[i] - omega * t[i];
    r[i] = ri;
    acc = fma(ri, ri, acc);
  }
  acc = block_sum(acc, sh);
  if (threadIdx.x == 0) partials[blockIdx.x] = acc;
  if (!last_block(&st->counter[4], gridDim.x)) return;
  const double tot = reduce_partials(partials, gridDim.x, sh);
  if (threadIdx.x == 0) {
    st->h[kBcRr] = tot;
    st->counter[4] = 0;
  }
}

// the cycle stopped after a BiCG half step whose residual met the target:
// x += alpha p^ (runs after the stop, so not gated by it)
__global__ void k_bc_xs(int64_t n, double* __restrict__ x, const float* __restrict__ ph, const DevState* st) {
  wait_prior_grid();
  if (st->h[kBcReason] != kBcSDone) return;
  const double alpha = st->h[kBcAlpha];
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    x[i] += alpha * split_at(ph, n, i);
}

// start of a cycle from the true residual rk: r = rt = rk, p = v = 0
__global__ void k_bc_start_vec(int64_t n, const double* __restrict__ rk, double* __restrict__ r,
                               double* __restrict__ rt, double* __restrict__ p, double* __restrict__ v) {
  wait_prior_grid();
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    r[i] = rk[i];
    rt[i] = rk[i];
    p[i] = 0.0;
    v[i] = 0.0;
  }
}

__global__ void k_bc_start(DevState* st) {
  wait_prior_grid();
  st->h[kBcRhoPrev] = st->h[kBcAlpha] = st->h[kBcOmega] = 1.0;
  st->h[kBcReason] = kBcGoing;
  st->done = 0;
  st->k = 0;
}

}  // namespace

int bicgstab(bo_prec* P, const double* b_in, double* x_in, const bo_solve_opts* o, bo_solve_info* info) {
  int rc = krylov_alloc(P, std::max(o->restart, 8));  // six FP64 recurrence vectors, two split ones
  if (rc != BO_OK) return rc;
  const auto t0 = std::chrono::steady_clock::now();
  cudaStream_t s = P->stream;
  const Geom& g = P->mat->g;
  const int64_t nn = 3 * g.N;
  DevState* st = P->st;
  if (!P->mat->a2_valid) launch_split_matrix(P->mat, s);
  const double* b_d = b_in;
  double* x_d = x_in;
  if (o->mem == BO_MEM_HOST) {
    cudaMemcpyAsync(P->hostio, b_in, nn * sizeof(double), cudaMemcpyHostToDevice, s);
    b_d = P->hostio;
    x_d = P->hostio + nn;
    if (!o->x0_is_zero) cudaMemcpyAsync(x_d, x_in, nn * sizeof(double), cudaMemcpyHostToDevice, s);
  }
  launch_gather(g, b_d, P->bi, s);
  if (o->x0_is_zero) cudaMemsetAsync(P->xi, 0, nn * sizeof(double), s);
  else launch_gather(g, x_d, P->xi, s);
  (launch_pdl(k_norm, kRedBlocks, kThreads, 0, s, nn, P->bi, P->partials, st), note_launch());
  (launch_pdl(k_set_target, 1, 1, 0, s, st, o->tol), note_launch());
  if (o->x0_is_zero) {
    cudaMemcpyAsync(P->rk, P->bi, nn * sizeof(double), cudaMemcpyDeviceToDevice, s);
    (launch_pdl(k_beta_is_bnorm, 1, 1, 0, s, st), note_launch());
  } else {
    (launch_pdl(k_true_residual, kRedBlocks, kThreads, 0, s, g, P->mat->A, P->bi, P->xi, P->rk, P->partials, st),
     note_launch());
  }
  auto read_state = [&](int slot) -> bool {
    publish_state(P, st, slot, s);
    cudaEventRecord(P->ev[slot], s);
    return cudaEventSynchronize(P->ev[slot]) == cudaSuccess;
  };
  int status = BO_OK;
  if (!read_state(3)) return BO_ERR_CUDA;
  const double bnorm = P->h_st[3].bnorm;
  double beta = P->h_st[3].beta;
  const double target = o->tol * bnorm;
  int its = 0, restarts = 0;
  if (!std::isfinite(bnorm) || !std::isfinite(beta)) status = BO_ERR_NONFINITE;
  // recurrence vectors in the Krylov workspace
  double* r = P->V;
  double* rt = P->V + nn;
  double* p = P->V + 2 * nn;
  double* v = P->V + 3 * nn;
  double* sv = P->V + 4 * nn;
  double* tv = P->V + 5 * nn;
  float* ph = (float*)P->Z;             // M^{-1} p as split pairs
  float* shs = (float*)P->Z + 2 * nn;   // M^{-1} s as split pairs
  const int gn = grid_for(nn);
  const int gs = occ_grid((const void*)k_arnoldi_spmv<double>, g.N);
  auto enqueue_iteration = [&]() {
    (launch_pdl(k_bc_dots, kRedBlocks, kThreads, 0, s, nn, rt, r, nullptr, nullptr, P->partials, st, kBcRho, -1),
     note_launch());
    (launch_pdl(k_bc_scalar<0>, 1, 1, 0, s, st), note_launch());
    (launch_pdl(k_bc_p, gn, kThreads, 0, s, nn, r, p, v, st), note_launch());
    launch_cpr_split(P, p, ph, st, nullptr);
    (launch_pdl(k_arnoldi_spmv<double>, gs, kThreads, 0, s, g, P->mat->A2, P->mat->A, P->mat->a2_range, ph, v, st),
     note_launch());
    (launch_pdl(k_bc_dots, kRedBlocks, kThreads, 0, s, nn, rt, v, nullptr, nullptr, P->partials, st, kBcRtv, -1),
     note_launch());
    (launch_pdl(k_bc_scalar<1>, 1, 1, 0, s, st), note_launch());
    (launch_pdl(k_bc_s, kRedBlocks, kThreads, 0, s, nn, r, v, sv, P->partials, st), note_launch());
    (launch_pdl(k_bc_scalar<2>, 1, 1, 0, s, st), note_launch());
    launch_cpr_split(P, sv, shs, st, nullptr);
    (launch_pdl(k_arnoldi_spmv<double>, gs, kThreads, 0, s, g, P->mat->A2, P->mat->A, P->mat->a2_range, shs, tv, st),
     note_launch());
    (launch_pdl(k_bc_dots, kRedBlocks, kThreads, 0, s, nn, tv, sv, tv, tv, P->partials, st, kBcTs, kBcTt), note_launch());
    (launch_pdl(k_bc_scalar<3>, 1, 1, 0, s, st), note_launch());
    (launch_pdl(k_bc_xr, kRedBlocks, kThreads, 0, s, nn, P->xi, ph, shs, sv, tv, r, P->partials, st), note_launch());
    (launch_pdl(k_bc_scalar<4>, 1, 1, 0, s, st), note_launch());
  };
  while (status == BO_OK && bnorm > 0.0 && beta > target && its < o->maxit) {
    (launch_pdl(k_bc_start_vec, gn, kThreads, 0, s, nn, P->rk, r, rt, p, v), note_launch());
    (launch_pdl(k_bc_start, 1, 1, 0, s, st), note_launch());
    // iterations, polled one behind: a stop leaves the queued iteration's kernels idle
    int enq = 0, polled = 0;
    bool stop = false;
    while (!stop && polled < enq + 1) {
      while (!stop && its + enq < o->maxit && enq - polled < 2) {
        enqueue_iteration();
        publish_state(P, st, enq % 2, s);
        cudaEventRecord(P->ev[enq % 2], s);
        ++enq;
      }
      if (polled == enq) break;
      if (cudaEventSynchronize(P->ev[polled % 2]) != cudaSuccess) return BO_ERR_CUDA;
      if (P->h_st[polled % 2].done) stop = true;
      ++polled;
    }
    (launch_pdl(k_bc_xs, gn, kThreads, 0, s, nn, P->xi, ph, st), note_launch());
    (launch_pdl(k_true_residual, kRedBlocks, kThreads, 0, s, g, P->mat->A, P->bi, P->xi, P->rk, P->partials, st),
     note_launch());
    if (!read_state(3)) return BO_ERR_CUDA;
    const DevState& h = P->h_st[3];
    its += h.k;
    ++restarts;
    beta = h.beta;
    if (!std::isfinite(beta)) {
      status = BO_ERR_BREAKDOWN;
    } else if ((int)h.h[kBcReason] == kBcBroke && h.k == 0) {
      status = BO_ERR_BREAKDOWN;  // the recurrence cannot start from this residual
    }
  }
  if (status == BO_OK && bnorm > 0.0 && beta > target) status = BO_ERR_NOT_CONVERGED;
  if (bnorm == 0.0) {
    cudaMemsetAsync(P->xi, 0, nn * sizeof(double), s);
    beta = 0.0;
  }
  launch_scatter(g, P->xi, x_d, s);
  if (o->mem == BO_MEM_HOST) cudaMemcpyAsync(x_in, x_d, nn * sizeof(double), cudaMemcpyDeviceToHost, s);
  if (cudaStreamSynchronize(s) != cudaSuccess) return BO_ERR_CUDA;
  P->nhist = 0;
  if (info) {
    info->status = status;
    info->iters = its;
    info->restarts = restarts;
    info->true_rel_res = bnorm > 0 ? beta / bnorm : beta;
    info->est_rel_res = info->true_rel_res;
    info->spmv_launches = 0;
    info->spmv_ms = 0.0;
    info->solve_ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
  }
  return status;
}

namespace {

// ---- lockstep batched solve (BO_LAUNCH_BATCH_GRAPH)
// Every realisation of the batch runs its FGMRES cycle in step with the
// others: Arnoldi column j of all of them is one CUDA graph (captured once,
// one branch per stream of the capture pool, the realisations spread over
// the branches), so one graph launch advances the whole batch by a column
// and the host reads every realisation's published state once per column.
// A realisation whose cycle has stopped has its column kernels return at
// once (its device state's done flag).  The cycle's start and end run on
// each realisation's own stream, as in the stream-pool form.
struct BatchGraphs {
  std::vector<bo_prec*> P;
  std::vector<unsigned long long> gen;
  int m = 0, width = 0;
  std::vector<cudaGraphExec_t> col;
  std::vector<long long> nodes;
  void release() {
    for (auto& e : col)
      if (e) cudaGraphExecDestroy(e);
    col.clear();
  }
};

constexpr int kBranchesPerStream = 4;
std::mutex g_bg_mu;
std::vector<BatchGraphs> g_bg;  // the two most recent batches' graphs
cudaStream_t g_bg_drv = nullptr;
std::vector<cudaStream_t> g_bg_cap;
std::vector<cudaEvent_t> g_bg_ev;  // fork, one join per capture stream, three column events

bool batch_streams(int width) {
  if (!g_bg_drv && cudaStreamCreateWithFlags(&g_bg_drv, cudaStreamNonBlocking) != cudaSuccess) return false;
  while ((int)g_bg_cap.size() < width) {
    cudaStream_t c;
    if (cudaStreamCreateWithFlags(&c, cudaStreamNonBlocking) != cudaSuccess) return false;
    g_bg_cap.push_back(c);
  }
  while ((int)g_bg_ev.size() < kBranchesPerStream * kMaxPoolStreams + 4) {
    cudaEvent_t e;
    if (cudaEventCreateWithFlags(&e, cudaEventDisableTiming) != cudaSuccess) return false;
    g_bg_ev.push_back(e);
  }
  return true;
}

BatchGraphs& batch_graphs(const std::vector<Job*>& act, int m, int width) {
  std::vector<bo_prec*> P;
  std::vector<unsigned long long> gen;
  for (Job* jb : act) {
    P.push_back(jb->P);
    gen.push_back(jb->P->graph_gen);
  }
  for (auto& c : g_bg)
    if (c.P == P && c.gen == gen && c.m == m && c.width == width) return c;
  if (g_bg.size() >= 2) {
    g_bg.front().release();
    g_bg.erase(g_bg.begin());
  }
  g_bg.emplace_back();
  BatchGraphs& c = g_bg.back();
  c.P = P;
  c.gen = gen;
  c.m = m;
  c.width = width;
  c.col.assign(m, nullptr);
  c.nodes.assign(m, 0);
  return c;
}

// capture column j of every realisation of `act` into one graph
bool capture_batch_column(BatchGraphs& c, const std::vector<Job*>& act, int j) {
  const int W = std::min(c.width, (int)act.size());
  cudaStream_t drv = g_bg_drv;
  const long long l0 = g_launches.load();
  if (cudaStreamBeginCapture(drv, cudaStreamCaptureModeThreadLocal) != cudaSuccess) return false;
  cudaEvent_t fork = g_bg_ev[0];
  cudaEventRecord(fork, drv);
  for (int w = 0; w < W; ++w) cudaStreamWaitEvent(g_bg_cap[w], fork, 0);
  for (size_t r = 0; r < act.size(); ++r) {
    Job* jb = act[r];
    cudaStream_t saved = jb->P->stream;
    jb->P->stream = g_bg_cap[r % W];
    jb->enqueue_column_kernels(j, false);
    publish_state(jb->P, jb->P->st, j % kRing, jb->P->stream);
    jb->P->stream = saved;
  }
  for (int w = 0; w < W; ++w) {
    cudaEventRecord(g_bg_ev[1 + w], g_bg_cap[w]);
    cudaStreamWaitEvent(drv, g_bg_ev[1 + w], 0);
  }
  cudaGraph_t gr = nullptr;
  const cudaError_t e = cudaStreamEndCapture(drv, &gr);
  const long long nodes = g_launches.load() - l0;
  g_launches.fetch_sub(nodes);  // captured, not run: counted at each replay instead
  if (e != cudaSuccess || !gr) return false;
  const cudaError_t ei = cudaGraphInstantiate(&c.col[j], gr, 0);
  cudaGraphDestroy(gr);
  if (ei != cudaSuccess) {
    c.col[j] = nullptr;
    return false;
  }
  c.nodes[j] = nodes;
  return true;
}

// returns BO_OK or BO_ERR_CUDA; per-realisation results are in the jobs
int fgmres_lockstep(std::vector<Job>& jobs) {
  // branches of a column graph: four per pool stream of the tuned width
  const int width = kBranchesPerStream * std::min(kMaxPoolStreams, std::max(1, g_pool_width.load()));
  std::lock_guard<std::mutex> lk(g_bg_mu);
  if (!batch_streams(width)) return BO_ERR_CUDA;
  cudaStream_t drv = g_bg_drv;
  for (auto& jb : jobs) jb.start();
  for (auto& jb : jobs)
    while (jb.phase == Job::kInitWait) jb.advance(true);
  for (;;) {
    std::vector<Job*> act;
    for (auto& jb : jobs)
      if (jb.phase == Job::kColumns) act.push_back(&jb);
    if (act.empty()) break;
    const int m = act[0]->o.restart;
    int L = m;  // columns this cycle: no realisation passes its iteration limit
    for (Job* jb : act) L = std::min(L, jb->o.maxit - jb->its);
    // the drive stream after every realisation's cycle start
    for (Job* jb : act) {
      cudaEventRecord(jb->P->ev[kPhaseSlot], jb->P->stream);
      cudaStreamWaitEvent(drv, jb->P->ev[kPhaseSlot], 0);
    }
    BatchGraphs& c = batch_graphs(act, m, width);
    cudaEvent_t* colev = &g_bg_ev[1 + kBranchesPerStream * kMaxPoolStreams];
    int launched = 0;
    bool stop = false;
    while (!stop && launched < L) {
      const int j = launched;
      if (!c.col[j] && !capture_batch_column(c, act, j)) return BO_ERR_CUDA;
      if (cudaGraphLaunch(c.col[j], drv) != cudaSuccess) return BO_ERR_CUDA;
      g_launches.fetch_add(c.nodes[j]);
      cudaEventRecord(colev[j % 3], drv);
      ++launched;
      if (j >= 1) {  // one column of lag: the states of column j - 1
        if (cudaEventSynchronize(colev[(j - 1) % 3]) != cudaSuccess) return BO_ERR_CUDA;
        bool all = true;
        for (Job* jb : act) all = all && jb->P->h_st[(j - 1) % kRing].done;
        stop = all;
      }
    }
    // every realisation's stream after the drive stream, then its cycle end
    cudaEventRecord(colev[0], drv);
    for (Job* jb : act) {
      cudaStreamWaitEvent(jb->P->stream, colev[0], 0);
      jb->j_enq = launched;
      jb->end_cycle();
    }
    for (Job* jb : act)
      while (jb->phase == Job::kCycleWait) jb->advance(true);
  }
  for (auto& jb : jobs)
    while (jb.phase != Job::kDone) jb.advance(true);
  return BO_OK;
}

}  // namespace

int fgmres_batched(bo_prec* const* P, int nreal, const double* const* b, double* const* x, const bo_solve_opts* o,
                   bo_solve_info* infos, const double* tols) {
  for (int r = 0; r < nreal; ++r) {
    const int rc = krylov_alloc(P[r], o->restart);
    if (rc != BO_OK) return rc;
  }
  std::vector<Job> jobs(nreal);
  for (int r = 0; r < nreal; ++r) {
    jobs[r].P = P[r];
    jobs[r].b_in = b[r];
    jobs[r].x_in = x[r];
    jobs[r].o = *o;
    if (tols) jobs[r].o.tol = tols[r];
    jobs[r].info = infos ? &infos[r] : nullptr;
  }
  bool lockstep = true;
  for (int r = 0; r < nreal; ++r) lockstep = lockstep && P[r]->launch_mode == BO_LAUNCH_BATCH_GRAPH && !P[r]->wl;
  if (lockstep) {
    const int rc = fgmres_lockstep(jobs);
    if (rc != BO_OK) return rc;
  }
  int remaining = lockstep ? 0 : nreal;
  while (remaining > 0) {
    bool moved = false;
    remaining = 0;
    for (auto& jb : jobs) {
      if (jb.phase == Job::kDone) continue;
      moved |= jb.advance(false);
      if (jb.phase != Job::kDone) ++remaining;
    }
    if (!moved && remaining > 0) {  // nothing ready: wait on the first pending job
      for (auto& jb : jobs)
        if (jb.phase != Job::kDone) {
          jb.advance(true);
          break;
        }
    }
  }
  int status = BO_OK;
  for (auto& jb : jobs)
    if (jb.status != BO_OK && status == BO_OK) status = jb.status;
  return status;
}

}  // namespace bo
