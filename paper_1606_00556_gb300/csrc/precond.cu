// CPR-FPF preconditioner (paper Sec. 3.2, Alg. 2) on the colour-split
// layout: Quasi-IMPES decoupling, red-black block ILU(0) as the local solver
// R, an aggregation AMG V-cycle on the pressure block A_pp, and their
// composition.
//
// Red-black block ILU(0).  With the red cells ordered first, red rows have
// no lower part and black-black blocks lie off the pattern except on the
// diagonal, so ILU(0) reduces to
//     D_b' = D_b - sum_{r ~ b} A_br D_r^{-1} A_rb     (pivot blocks of black cells)
// and (L U)^{-1} f is three stencil passes:
//     t_r = D_r^{-1} f_r;   z_b = D_b'^{-1} (f_b - sum A_br t_r);
//     z_r = t_r - D_r^{-1} sum A_rb z_b.
//
// AMG.  Level 0 is the (0,0) entry of every block of D_QI^{-1} A on the
// colour-split grid; level l+1 aggregates the 2x2x2 boxes of level l
// (piecewise-constant P, Galerkin P^T A P, still 7-point); coarsening stops
// at <= coarse_max cells, whose dense inverse is formed once per setup.
// V(nu1, nu2) with red-black Gauss-Seidel: red then black before the coarse
// correction, black then red after it.  After a black half sweep only red
// cells carry a residual, so restriction sums red residuals.  Levels of at
// most kTailCells cells run inside one thread block (kernel k_tail).
#include <atomic>
#include <cstdio>

#include "bo_internal.cuh"

namespace bo {
namespace {

constexpr int kTailThreads = 1024;
constexpr int64_t kTailCells = 4096;
constexpr int kCoarseMax = 128;
constexpr size_t kTailSmemMax = 200 * 1024;  // stage the tail levels in shared memory up to this size

// ---------------------------------------------------------------- 3x3 blocks
// inverse by Gauss-Jordan elimination with partial pivoting; false if a
// pivot is zero or the result is not finite.  Each pivot row is scaled by
// one reciprocal: on GB300 an FP64 division is a long sequence of FP64
// instructions, and six of them per pivot made the ILU setup FP64-bound.
template <typename T>
__device__ bool inv3(const T a[9], T out[9]) {
  T m[3][6];
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) {
      m[i][j] = a[3 * i + j];
      m[i][3 + j] = (i == j) ? T(1) : T(0);
    }
  for (int k = 0; k < 3; ++k) {
    int p = k;
    for (int i = k + 1; i < 3; ++i)
      if (fabs(m[i][k]) > fabs(m[p][k])) p = i;
    if (m[p][k] == T(0)) return false;
    if (p != k)
      for (int j = 0; j < 6; ++j) { const T t = m[k][j]; m[k][j] = m[p][j]; m[p][j] = t; }
    const T rp = T(1) / m[k][k];
    for (int j = 0; j < 6; ++j) m[k][j] *= rp;
    for (int i = 0; i < 3; ++i) {
      if (i == k) continue;
      const T f = m[i][k];
      for (int j = 0; j < 6; ++j) m[i][j] -= f * m[k][j];
    }
  }
  bool ok = true;
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) {
      out[3 * i + j] = m[i][3 + j];
      ok &= isfinite(out[3 * i + j]);
    }
  return ok;
}

// decoupled block (colour, slot) of the cell at half index q: row 0 becomes
// g0 row0 + g1 row1 + g2 row2 with the cell's weights (paper Sec. 3.2,
// D_QI^{-1} A), FP64
__device__ __forceinline__ void dec_block(const Geom& g, const double* __restrict__ A, const double* __restrict__ w,
                                          int color, int slot, int64_t q, double b[9]) {
  const double g0 = w[vidx(g, 0, color, q)], g1 = w[vidx(g, 1, color, q)], g2 = w[vidx(g, 2, color, q)];
  double a[9];
#pragma unroll
  for (int rc = 0; rc < 9; ++rc) a[rc] = A[plane(g, color, slot, rc) + q];
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    b[c] = g0 * a[c] + g1 * a[3 + c] + g2 * a[6 + c];
    b[3 + c] = a[3 + c];
    b[6 + c] = a[6 + c];
  }
}

template <typename T>
__device__ __forceinline__ void mul3(const T a[9], const T b[9], T c[9]) {
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j) c[3 * i + j] = a[3 * i] * b[j] + a[3 * i + 1] * b[3 + j] + a[3 * i + 2] * b[6 + j];
}

// Storage and arithmetic types.  S is the storage type of the matrix-like
// arrays (decoupled matrix, ILU pivot inverses, AMG coefficients, coarse
// inverse): double, float or BF16; vectors and arithmetic use T (double for
// S = double, float otherwise).  cv converts a stored value to T, to_store
// an FP64 value to S.
template <typename T, typename S>
__device__ __forceinline__ T cv(S v) { return (T)v; }
template <>
__device__ __forceinline__ float cv<float, __nv_bfloat16>(__nv_bfloat16 v) { return __bfloat162float(v); }
template <typename S>
__device__ __forceinline__ S to_store(double v) { return (S)v; }
template <>
__device__ __forceinline__ __nv_bfloat16 to_store<__nv_bfloat16>(double v) { return __float2bfloat16_rn((float)v); }

// ---------------------------------------------------------------- setup kernels
// Quasi-IMPES decoupling (paper Sec. 3.2): row 0 of each cell becomes
// g . (row0, row1, row2) with g = (1, -a01/a11, -a02/a22) from the cell's
// diagonal block.  Where that pressure pivot is not positive (injector cells
// flooded to residual oil: the oil row carries no pressure information and
// the water pivot is negative), the cell takes the exact local decoupling,
// g = row 0 of A_ii^{-1} (pivot 1), which keeps the AMG operator's diagonal
// positive for the Gauss-Seidel smoother.  With abf set every cell takes
// that row: the ABF decoupling (D = block diagonal of A) restricted to the
// pressure row, which is all of it the CPR needs (block ILU(0) is invariant
// under a block-diagonal left scaling).  Writes the weights [3][N] and the
// decoupled blocks in storage type S.  The weights are formed in FP64; for
// FP32 or BF16 storage the decoupled rows are formed from the split copy of
// A in split FP32 pairs (FP32 instructions; the result rounded once to S),
// unless the split copy could not hold every value (*range).
template <typename S>
__device__ __forceinline__ S store_split(df v) {
  return to_store<S>((double)__fadd_rn(v.hi, v.lo));
}
template <>
__device__ __forceinline__ float store_split<float>(df v) { return __fadd_rn(v.hi, v.lo); }
template <>
__device__ __forceinline__ __nv_bfloat16 store_split<__nv_bfloat16>(df v) {
  return __float2bfloat16_rn(__fadd_rn(v.hi, v.lo));
}

template <typename S>
__global__ void k_decouple(Geom g, const double* __restrict__ A, const float2* __restrict__ A2,
                           const int* __restrict__ range, S* __restrict__ At, double* __restrict__ w,
                           float* __restrict__ wf, int abf, DevState* st) {
  wait_prior_grid();
  const bool split = sizeof(S) < sizeof(double) && A2 && !*range;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < g.N; t += (int64_t)gridDim.x * blockDim.x) {
    const int color = (int)(t / g.Nh);
    const int64_t q = t - color * g.Nh;
    double D[9];
#pragma unroll
    for (int rc = 0; rc < 9; ++rc) D[rc] = A[plane(g, color, kDiag, rc) + q];
    double g0 = 1.0, g1 = 0.0, g2 = 0.0;
    if (D[4] == 0.0 || D[8] == 0.0 || !isfinite(D[4]) || !isfinite(D[8])) {
      atomicOr(&st->err, kErrBreakdown);
    } else {
      g1 = -D[1] / D[4];
      g2 = -D[2] / D[8];
      if (abf || !(g0 * D[0] + g1 * D[3] + g2 * D[6] > 0.0)) {
        double inv[9];
        if (inv3(D, inv)) {
          g0 = inv[0];
          g1 = inv[1];
          g2 = inv[2];
        } else {
          atomicOr(&st->err, kErrBreakdown);
        }
      }
    }
    w[vidx(g, 0, color, q)] = g0;
    w[vidx(g, 1, color, q)] = g1;
    w[vidx(g, 2, color, q)] = g2;
    if (wf) {
      wf[vidx(g, 0, color, q)] = (float)g0;
      wf[vidx(g, 1, color, q)] = (float)g1;
      wf[vidx(g, 2, color, q)] = (float)g2;
    }
    if (split) {
      int bad = 0;
      const float2 g0p = df_split_bits(g0, &bad), g1p = df_split_bits(g1, &bad), g2p = df_split_bits(g2, &bad);
      const df gs0{g0p.x, g0p.y}, gs1{g1p.x, g1p.y}, gs2{g2p.x, g2p.y};
#pragma unroll
      for (int s = 0; s < 7; ++s) {
        df a[9];
#pragma unroll
        for (int rc = 0; rc < 9; ++rc) {
          const float2 v = A2[a2_index(g, color, s * 9 + rc, q)];
          a[rc] = df{v.x, v.y};
        }
#pragma unroll
        for (int c = 0; c < 3; ++c) {
          df r = df_fma_acc(df{0.f, 0.f}, gs0, a[c]);
          r = df_fma_acc(r, gs1, a[3 + c]);
          r = df_norm(df_fma_acc(r, gs2, a[6 + c]));
          At[at_index(g, color, s * 9 + c, q)] = store_split<S>(r);
          At[at_index(g, color, s * 9 + 3 + c, q)] = store_split<S>(a[3 + c]);
          At[at_index(g, color, s * 9 + 6 + c, q)] = store_split<S>(a[6 + c]);
          if (s == kDiag && c == 0 && (r.hi == 0.f || !isfinite(r.hi))) atomicOr(&st->err, kErrBreakdown);
        }
      }
      continue;
    }
#pragma unroll
    for (int s = 0; s < 7; ++s) {
      double a[9];
#pragma unroll
      for (int rc = 0; rc < 9; ++rc) a[rc] = A[plane(g, color, s, rc) + q];
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        At[at_index(g, color, s * 9 + c, q)] = to_store<S>(g0 * a[c] + g1 * a[3 + c] + g2 * a[6 + c]);
        At[at_index(g, color, s * 9 + 3 + c, q)] = to_store<S>(a[3 + c]);
        At[at_index(g, color, s * 9 + 6 + c, q)] = to_store<S>(a[6 + c]);
      }
      if (s == kDiag) {
        const double app = g0 * a[0] + g1 * a[3] + g2 * a[6];
        if (app == 0.0 || !isfinite(app)) atomicOr(&st->err, kErrBreakdown);
      }
    }
  }
}

// Pivots are always factored in FP64 from the FP64 matrix and the
// Quasi-IMPES weights, whatever precision they are stored in: the black
// pivots are Schur complements D_b - sum A_br D_r^{-1} A_rb that cancel
// strongly where the permeability contrast is high, and FP32 arithmetic there
// can leave the local solver unstable.

// red pivots: D_r^{-1} of the decoupled diagonal blocks, stored in type S
// and, for the black pass, in FP64 in `red64` ([rc][N/2]); with SPLIT the
// black pass takes them as split pairs instead (red64 read as float2)
template <typename S, bool SPLIT>
__global__ void k_ilu_red(Geom g, const double* __restrict__ A, const double* __restrict__ w, S* __restrict__ Dinv,
                          double* __restrict__ red64, DevState* st) {
  wait_prior_grid();
  for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < g.Nh; q += (int64_t)gridDim.x * blockDim.x) {
    double d[9], inv[9];
    dec_block(g, A, w, 0, kDiag, q, d);
    if (!inv3(d, inv)) {
      atomicOr(&st->err, kErrBreakdown);
      for (int rc = 0; rc < 9; ++rc) inv[rc] = 0.0;
    }
    int bad = 0;
    for (int rc = 0; rc < 9; ++rc) {
      Dinv[(size_t)rc * g.N + q] = to_store<S>(inv[rc]);
      if (SPLIT) reinterpret_cast<float2*>(red64)[(size_t)rc * g.Nh + q] = df_split_bits(inv[rc], &bad);
      else red64[(size_t)rc * g.Nh + q] = inv[rc];
    }
  }
}

// The black pivots of a preconditioner stored in FP32 or BF16, formed in
// split FP32 pairs (48 significant bits, FP32 instructions) instead of FP64:
// the six products L D_r^{-1} U per cell are 324 multiply-adds, which on
// GB300's FP64 rate made this the slowest setup kernel.  The decoupled blocks
// come from the split copy of A and split weights; the Schur complement is
// summed in split pairs and inverted in FP64.  (An FP64-stored
// preconditioner keeps the FP64 kernel below.)
__device__ __forceinline__ void dec_block_split(const Geom& g, const float2* __restrict__ A2, const df wq[3],
                                                int color, int slot, int64_t q, df b[9]) {
  df a[9];
#pragma unroll
  for (int rc = 0; rc < 9; ++rc) {
    const float2 v = A2[a2_index(g, color, slot * 9 + rc, q)];
    a[rc] = df{v.x, v.y};
  }
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    df r = df_fma_acc(df{0.f, 0.f}, wq[0], a[c]);
    r = df_fma_acc(r, wq[1], a[3 + c]);
    r = df_fma_acc(r, wq[2], a[6 + c]);
    b[c] = df_norm(r);
    b[3 + c] = a[3 + c];
    b[6 + c] = a[6 + c];
  }
}

__device__ __forceinline__ void weights_split(const Geom& g, const double* __restrict__ w, int color, int64_t q,
                                              df wq[3]) {
  int bad = 0;
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    const float2 v = df_split_bits(w[vidx(g, k, color, q)], &bad);
    wq[k] = df{v.x, v.y};
  }
}

__device__ __forceinline__ void mul3_split(const df a[9], const df b[9], df c[9]) {
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j) {
      df r = df_fma_acc(df{0.f, 0.f}, a[3 * i], b[j]);
      r = df_fma_acc(r, a[3 * i + 1], b[3 + j]);
      r = df_fma_acc(r, a[3 * i + 2], b[6 + j]);
      c[3 * i + j] = df_norm(r);
    }
}

template <typename S>
__global__ void k_ilu_black_split(Geom g, const float2* __restrict__ A2, const double* __restrict__ A,
                                  const int* __restrict__ range, const double* __restrict__ w,
                                  const float2* __restrict__ red2, S* __restrict__ Dinv, DevState* st) {
  wait_prior_grid();
  if (*range) {  // a value outside the split form's range: the FP64 products, from A
    for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < g.Nh; q += (int64_t)gridDim.x * blockDim.x) {
      const Cell c = decode(g, 1, q);
      double Sc[9], inv[9];
      dec_block(g, A, w, 1, kDiag, q, Sc);
      for (int s = 0; s < 7; ++s) {
        if (s == kDiag) continue;
        const int64_t nq = nbr(g, c, q, s);
        if (nq < 0) continue;
        double L[9], U[9], Dr[9], T1[9], T2[9];
        dec_block(g, A, w, 1, s, q, L);
        dec_block(g, A, w, 0, opposite(s), nq, U);
        for (int rc = 0; rc < 9; ++rc) {
          const float2 v = red2[(size_t)rc * g.Nh + nq];
          Dr[rc] = (double)v.x + (double)v.y;
        }
        mul3(L, Dr, T1);
        mul3(T1, U, T2);
        for (int rc = 0; rc < 9; ++rc) Sc[rc] -= T2[rc];
      }
      if (!inv3(Sc, inv)) {
        atomicOr(&st->err, kErrBreakdown);
        for (int rc = 0; rc < 9; ++rc) inv[rc] = 0.0;
      }
      for (int rc = 0; rc < 9; ++rc) Dinv[(size_t)rc * g.N + g.Nh + q] = to_store<S>(inv[rc]);
    }
    return;
  }
  for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < g.Nh; q += (int64_t)gridDim.x * blockDim.x) {
    const Cell c = decode(g, 1, q);
    df wb[3], Sc[9];
    weights_split(g, w, 1, q, wb);
    dec_block_split(g, A2, wb, 1, kDiag, q, Sc);
#pragma unroll 1
    for (int s = 0; s < 7; ++s) {
      if (s == kDiag) continue;
      const int64_t nq = nbr(g, c, q, s);
      if (nq < 0) continue;
      df wr[3], L[9], U[9], Dr[9], T1[9], T2[9];
      weights_split(g, w, 0, nq, wr);
      dec_block_split(g, A2, wb, 1, s, q, L);
      dec_block_split(g, A2, wr, 0, opposite(s), nq, U);
#pragma unroll
      for (int rc = 0; rc < 9; ++rc) {
        const float2 v = red2[(size_t)rc * g.Nh + nq];
        Dr[rc] = df{v.x, v.y};
      }
      mul3_split(L, Dr, T1);
      mul3_split(T1, U, T2);
#pragma unroll
      for (int rc = 0; rc < 9; ++rc) Sc[rc] = df_add(Sc[rc], df_neg(T2[rc]));
    }
    double S64[9], inv[9];
#pragma unroll
    for (int rc = 0; rc < 9; ++rc) S64[rc] = df_to_double(Sc[rc]);
    if (!inv3(S64, inv)) {
      atomicOr(&st->err, kErrBreakdown);
      for (int rc = 0; rc < 9; ++rc) inv[rc] = 0.0;
    }
    for (int rc = 0; rc < 9; ++rc) Dinv[(size_t)rc * g.N + g.Nh + q] = to_store<S>(inv[rc]);
  }
}

// black pivots: D_b' = D_b - sum_r A_br D_r^{-1} A_rb with the FP64 red
// inverses, stored inverted in type S
template <typename S>
__global__ void k_ilu_black(Geom g, const double* __restrict__ A, const double* __restrict__ w,
                            const double* __restrict__ red64, S* __restrict__ Dinv, DevState* st) {
  wait_prior_grid();
  for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < g.Nh; q += (int64_t)gridDim.x * blockDim.x) {
    const Cell c = decode(g, 1, q);
    double Sc[9], inv[9];
    dec_block(g, A, w, 1, kDiag, q, Sc);
#pragma unroll
    for (int s = 0; s < 7; ++s) {
      if (s == kDiag) continue;
      const int64_t nq = nbr(g, c, q, s);
      if (nq < 0) continue;
      double L[9], U[9], Dr[9], T1[9], T2[9];
      dec_block(g, A, w, 1, s, q, L);
      dec_block(g, A, w, 0, opposite(s), nq, U);
      for (int rc = 0; rc < 9; ++rc) Dr[rc] = red64[(size_t)rc * g.Nh + nq];
      mul3(L, Dr, T1);
      mul3(T1, U, T2);
      for (int rc = 0; rc < 9; ++rc) Sc[rc] -= T2[rc];
    }
    if (!inv3(Sc, inv)) {
      atomicOr(&st->err, kErrBreakdown);
      for (int rc = 0; rc < 9; ++rc) inv[rc] = 0.0;
    }
    for (int rc = 0; rc < 9; ++rc) Dinv[(size_t)rc * g.N + g.Nh + q] = to_store<S>(inv[rc]);
  }
}

template <typename S>
__global__ void k_convert(const double* __restrict__ src, S* __restrict__ dst, size_t n) {
  wait_prior_grid();
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
    dst[i] = to_store<S>(src[i]);
}

// ------------------------------------------------------------ AMG setup
struct LevelDims {
  int32_t nx, ny, nz;
  int64_t n;
};

// (i, j, k) of natural index c of a level (c < 2^31), by 32-bit division
struct Ijk {
  int i, j, k;
};
__device__ __forceinline__ Ijk ijk_of(const LevelDims& L, int64_t c) {
  const uint32_t cu = (uint32_t)c, nx = (uint32_t)L.nx, ny = (uint32_t)L.ny;
  const uint32_t r = cu / nx;
  return Ijk{(int)(cu - r * nx), (int)(r % ny), (int)(r / ny)};
}

__device__ __forceinline__ int64_t nat_index(const LevelDims& L, int i, int j, int k) {
  return i + (int64_t)L.nx * (j + (int64_t)L.ny * k);
}

// direction slot of the coarse neighbour (di, dj, dk), or kDiag
__device__ __forceinline__ int dir_slot(int di, int dj, int dk) {
  if (dk < 0) return kZm;
  if (dk > 0) return kZp;
  if (dj < 0) return kYm;
  if (dj > 0) return kYp;
  if (di < 0) return kXm;
  if (di > 0) return kXp;
  return kDiag;
}

// Galerkin level 1 from level 0 (the decoupled pressure block, FP64 from A
// and the weights): coarse entry (I, J) = sum of fine a_ij, i in I, j in J.
__global__ void k_galerkin0(Geom g, const double* __restrict__ A, const double* __restrict__ w, LevelDims C,
                            double* __restrict__ c64, DevState* st) {
  wait_prior_grid();
  for (int64_t I = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; I < C.n; I += (int64_t)gridDim.x * blockDim.x) {
    const Ijk cc = ijk_of(C, I);
  const int ci = cc.i, cj = cc.j, ck = cc.k;
    double acc[7] = {0, 0, 0, 0, 0, 0, 0};
    for (int dk = 0; dk < 2; ++dk)
      for (int dj = 0; dj < 2; ++dj)
        for (int di = 0; di < 2; ++di) {
          const int i = 2 * ci + di, j = 2 * cj + dj, k = 2 * ck + dk;
          if (i >= g.nx || j >= g.ny || k >= g.nz) continue;
          const int color = (i + j + k) & 1;
          const int64_t q = (i + (int64_t)g.nx * (j + (int64_t)g.ny * k)) >> 1;
          const double g0 = w[vidx(g, 0, color, q)], g1 = w[vidx(g, 1, color, q)], g2 = w[vidx(g, 2, color, q)];
          const int ni[7] = {i, i, i - 1, i, i + 1, i, i};
          const int nj[7] = {j, j - 1, j, j, j, j + 1, j};
          const int nk[7] = {k - 1, k, k, k, k, k, k + 1};
          for (int s = 0; s < 7; ++s) {
            if (ni[s] < 0 || ni[s] >= g.nx || nj[s] < 0 || nj[s] >= g.ny || nk[s] < 0 || nk[s] >= g.nz) continue;
            const double a = g0 * A[plane(g, color, s, 0) + q] + g1 * A[plane(g, color, s, 3) + q] +
                             g2 * A[plane(g, color, s, 6) + q];
            const int cs = dir_slot(ni[s] / 2 - ci, nj[s] / 2 - cj, nk[s] / 2 - ck);
            acc[cs] += a;
          }
        }
    for (int s = 0; s < 7; ++s) c64[(size_t)s * C.n + I] = acc[s];
    if (acc[kDiag] == 0.0 || !isfinite(acc[kDiag])) atomicOr(&st->err, kErrBreakdown);
  }
}

// Galerkin level l+1 from natural-order level l
__global__ void k_galerkinn(LevelDims F, const double* __restrict__ f64, LevelDims C, double* __restrict__ c64,
                            DevState* st) {
  wait_prior_grid();
  for (int64_t I = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; I < C.n; I += (int64_t)gridDim.x * blockDim.x) {
    const Ijk cc = ijk_of(C, I);
  const int ci = cc.i, cj = cc.j, ck = cc.k;
    double acc[7] = {0, 0, 0, 0, 0, 0, 0};
    for (int dk = 0; dk < 2; ++dk)
      for (int dj = 0; dj < 2; ++dj)
        for (int di = 0; di < 2; ++di) {
          const int i = 2 * ci + di, j = 2 * cj + dj, k = 2 * ck + dk;
          if (i >= F.nx || j >= F.ny || k >= F.nz) continue;
          const int64_t c = nat_index(F, i, j, k);
          const int ni[7] = {i, i, i - 1, i, i + 1, i, i};
          const int nj[7] = {j, j - 1, j, j, j, j + 1, j};
          const int nk[7] = {k - 1, k, k, k, k, k, k + 1};
          for (int s = 0; s < 7; ++s) {
            if (ni[s] < 0 || ni[s] >= F.nx || nj[s] < 0 || nj[s] >= F.ny || nk[s] < 0 || nk[s] >= F.nz) continue;
            acc[dir_slot(ni[s] / 2 - ci, nj[s] / 2 - cj, nk[s] / 2 - ck)] += f64[(size_t)s * F.n + c];
          }
        }
    for (int s = 0; s < 7; ++s) c64[(size_t)s * C.n + I] = acc[s];
    if (acc[kDiag] == 0.0 || !isfinite(acc[kDiag])) atomicOr(&st->err, kErrBreakdown);
  }
}

// dense coarsest matrix: natural level (c64 given) or level 0 in the
// colour-split index order (index = colour * N/2 + q)
__global__ void k_dense_from_level(LevelDims L, const double* __restrict__ c64, Geom g, const double* __restrict__ A,
                                   const double* __restrict__ w, int level0, double* __restrict__ M) {
  wait_prior_grid();
  const int64_t n = L.n;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < n * n; t += (int64_t)gridDim.x * blockDim.x)
    M[t] = 0.0;
  __syncthreads();
  if (blockIdx.x != 0) return;
  // one block fills the stencil entries (grid of at most 128 cells)
  for (int64_t row = threadIdx.x; row < n; row += blockDim.x) {
    int i, j, k;
    if (level0) {
      const int color = (int)(row / g.Nh);
      const int64_t q = row - color * g.Nh;
      const Cell c = decode(g, color, q);
      i = c.i; j = c.j; k = c.k;
    } else {
      i = (int)(row % L.nx); j = (int)((row / L.nx) % L.ny); k = (int)(row / ((int64_t)L.nx * L.ny));
    }
    const int ni[7] = {i, i, i - 1, i, i + 1, i, i};
    const int nj[7] = {j, j - 1, j, j, j, j + 1, j};
    const int nk[7] = {k - 1, k, k, k, k, k, k + 1};
    for (int s = 0; s < 7; ++s) {
      if (ni[s] < 0 || ni[s] >= L.nx || nj[s] < 0 || nj[s] >= L.ny || nk[s] < 0 || nk[s] >= L.nz) continue;
      double a;
      int64_t colidx;
      if (level0) {
        const int color = (i + j + k) & 1;
        const int64_t q = (i + (int64_t)g.nx * (j + (int64_t)g.ny * k)) >> 1;
        a = w[vidx(g, 0, color, q)] * A[plane(g, color, s, 0) + q] + w[vidx(g, 1, color, q)] * A[plane(g, color, s, 3) + q] +
            w[vidx(g, 2, color, q)] * A[plane(g, color, s, 6) + q];
        const int ncol = (ni[s] + nj[s] + nk[s]) & 1;
        colidx = ncol * g.Nh + ((ni[s] + (int64_t)g.nx * (nj[s] + (int64_t)g.ny * nk[s])) >> 1);
      } else {
        a = c64[(size_t)s * n + row];
        colidx = nat_index(L, ni[s], nj[s], nk[s]);
      }
      M[row * n + colidx] += a;
    }
  }
}

// In-place Gauss-Jordan inversion with partial pivoting of an n x n matrix
// (n <= kCoarseMax) in shared memory by one thread block; the inverse is
// written to Minv in type S.
template <typename S>
__global__ void __launch_bounds__(1024) k_gj_inverse(int n, const double* __restrict__ M, S* __restrict__ Minv, DevState* st) {
  wait_prior_grid();
  extern __shared__ double sm[];
  double* a = sm;                 // n * n
  int* perm = (int*)(a + n * n);  // n
  __shared__ int piv;
  __shared__ int fail;
  __shared__ double fac[kCoarseMax];
  for (int t = threadIdx.x; t < n * n; t += blockDim.x) a[t] = M[t];
  if (threadIdx.x == 0) fail = 0;
  __syncthreads();
  for (int k = 0; k < n; ++k) {
    if (threadIdx.x == 0) {
      int p = k;
      for (int i = k + 1; i < n; ++i)
        if (fabs(a[i * n + k]) > fabs(a[p * n + k])) p = i;
      piv = p;
      perm[k] = p;
      if (a[p * n + k] == 0.0) fail = 1;
    }
    __syncthreads();
    if (fail) break;
    if (piv != k)
      for (int j = threadIdx.x; j < n; j += blockDim.x) {
        const double t = a[k * n + j];
        a[k * n + j] = a[piv * n + j];
        a[piv * n + j] = t;
      }
    __syncthreads();
    // the pivot row scaled by one reciprocal (an FP64 division is a long
    // sequence on GB300's narrow FP64 pipe; one per row instead of n)
    const double rp = 1.0 / a[k * n + k];
    __syncthreads();
    for (int j = threadIdx.x; j < n; j += blockDim.x) a[k * n + j] = (j == k ? 1.0 : a[k * n + j]) * rp;
    __syncthreads();
    // eliminate column k from every other row; factors first, so that the
    // row updates below read unmodified values
    for (int i = threadIdx.x; i < n; i += blockDim.x) fac[i] = a[i * n + k];
    __syncthreads();
    for (int t = threadIdx.x; t < n * n; t += blockDim.x) {
      const int i = t / n, j = t - (t / n) * n;
      if (i == k) continue;
      const double base = (j == k) ? 0.0 : a[i * n + j];
      a[i * n + j] = base - fac[i] * a[k * n + j];
    }
    __syncthreads();
  }
  if (fail) {
    if (threadIdx.x == 0) atomicOr(&st->err, kErrBreakdown);
    return;
  }
  // undo the row interchanges as column interchanges, last first
  for (int k = n - 1; k >= 0; --k) {
    const int p = perm[k];
    if (p != k)
      for (int i = threadIdx.x; i < n; i += blockDim.x) {
        const double t = a[i * n + k];
        a[i * n + k] = a[i * n + p];
        a[i * n + p] = t;
      }
    __syncthreads();
  }
  for (int t = threadIdx.x; t < n * n; t += blockDim.x) {
    Minv[t] = to_store<S>(a[t]);
    if (!isfinite(a[t])) atomicOr(&st->err, kErrBreakdown);
  }
}

// ------------------------------------------------------------ apply kernels
// Entry of the preconditioner: f = D_QI^{-1} v (DEC) or f = v, in precision
// T, fused with the first ILU pass on the red cells, t_r = D_r^{-1} f_r.
// v is FP64 or split pairs; sc the scale of an unnormalised Krylov vector.
// FP32 arithmetic reads the split input's high part (the low part lies
// below FP32's rounding) and the FP32 copy of the weights, so the FP32
// preconditioner issues no FP64 instruction here.
template <typename T>
__device__ __forceinline__ T in_get(const InV& v, size_t i, double sc) {
  if (v.f) {
    if constexpr (sizeof(T) == 4) return (float)sc * v.f[i];
    else return sc * ((double)v.f[i] + (double)v.f[v.n + i]);
  }
  return (T)(sc * v.d[i]);
}

template <typename T, typename S, bool DEC>
__global__ void k_cpr_entry(Geom g, InV v, const double* __restrict__ vs, const double* __restrict__ w,
                            const float* __restrict__ wf, const S* __restrict__ Dinv, T* __restrict__ f,
                            T* __restrict__ tv, const DevState* st) {
  wait_prior_grid();
  if (st->done) return;
  const double sc = vs ? *vs : 1.0;  // scale of an unnormalised Krylov vector
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < g.N; t += (int64_t)gridDim.x * blockDim.x) {
    const T v0 = in_get<T>(v, t, sc), v1 = in_get<T>(v, g.N + t, sc), v2 = in_get<T>(v, 2 * g.N + t, sc);
    T f0 = v0;
    if (DEC) {
      if constexpr (sizeof(T) == 4) f0 = fma3(0.f, wf[t], v0, wf[g.N + t], v1, wf[2 * g.N + t], v2);
      else f0 = fma3(0.0, w[t], v0, w[g.N + t], v1, w[2 * g.N + t], v2);
    }
    const T f1 = v1, f2 = v2;
    f[t] = f0;
    f[g.N + t] = f1;
    f[2 * g.N + t] = f2;
    if (t < g.Nh) {
      T d[9];
#pragma unroll
      for (int rc = 0; rc < 9; ++rc) d[rc] = cv<T>(Dinv[(size_t)rc * g.N + t]);
      tv[t] = d[0] * f0 + d[1] * f1 + d[2] * f2;
      tv[g.N + t] = d[3] * f0 + d[4] * f1 + d[5] * f2;
      tv[2 * g.N + t] = d[6] * f0 + d[7] * f1 + d[8] * f2;
    }
  }
}

// preconditioner output: FP64, or split pairs (exact for FP32 values)
template <typename T>
__device__ __forceinline__ void out_put(const OutV& o, size_t i, T v) {
  if (o.f) {
    if constexpr (sizeof(T) == 4) {
      o.f[i] = v;
      o.f[o.n + i] = 0.f;
    } else {
      const df d = df_from(v);
      o.f[i] = d.hi;
      o.f[o.n + i] = d.lo;
    }
  } else {
    o.d[i] = (double)v;
  }
}

template <typename T>
__global__ void k_widen_t(int64_t n, const T* __restrict__ a, double* __restrict__ b, const DevState* st) {
  wait_prior_grid();
  if (st->done) return;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    b[i] = (double)a[i];
}

template <typename T>
__global__ void k_copy_vec(int64_t n, const double* __restrict__ v, T* __restrict__ f, const DevState* st) {
  wait_prior_grid();
  if (st->done) return;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < n; t += (int64_t)gridDim.x * blockDim.x)
    f[t] = (T)v[t];
}

// sum over the six off-diagonal blocks of a row of At times the other
// colour's vector u: s = sum_s At[color][s] u[nbr]
template <typename T, typename S>
__device__ __forceinline__ void offdiag_sum(const Geom& g, const S* __restrict__ At, int color, int64_t q,
                                            const Cell& c, const T* __restrict__ u, T s[3]) {
  const int oc = color ^ 1;
  s[0] = s[1] = s[2] = T(0);
  // (every slot's loads are issued; a missing neighbour reads this cell's
  // own entries and is masked to zero, so all loads can be in flight)
#pragma unroll
  for (int sl = 0; sl < 7; ++sl) {
    if (sl == kDiag) continue;
    const int64_t nb = nbr(g, c, q, sl);
    const bool ok = nb >= 0;
    const int64_t nq = ok ? nb : q;
    T u0 = u[vidx(g, 0, oc, nq)], u1 = u[vidx(g, 1, oc, nq)], u2 = u[vidx(g, 2, oc, nq)];
    if (!ok) u0 = u1 = u2 = T(0);
    const S* a = At + at_index(g, color, sl * 9, q);
    constexpr size_t P = 32;  // entries (rc) of a block lie 32 apart in a tile
    s[0] = fma3(s[0], cv<T>(ld_stream(a)), u0, cv<T>(ld_stream(a + P)), u1, cv<T>(ld_stream(a + 2 * P)), u2);
    s[1] = fma3(s[1], cv<T>(ld_stream(a + 3 * P)), u0, cv<T>(ld_stream(a + 4 * P)), u1, cv<T>(ld_stream(a + 5 * P)), u2);
    s[2] = fma3(s[2], cv<T>(ld_stream(a + 6 * P)), u0, cv<T>(ld_stream(a + 7 * P)), u1, cv<T>(ld_stream(a + 8 * P)), u2);
  }
}

// ILU pass 2 (black): u_b = D_b'^{-1} (src_b - sum A_br t_r).
// OUT = false: z_b = u_b (precision T).
// OUT = true: t_b = u_b and the preconditioner's result on black cells,
//   zo_b = z1_b + Pi_p e_b + u_b, in FP64.
// blocks per SM the register budget is tuned for: the FP32 passes are
// memory-latency bound and want more warps; the FP64 ones are FP64-bound
template <typename T>
constexpr int ilu_min_blocks() { return sizeof(T) == 4 ? 4 : 3; }
template <typename T, int ROWS>
constexpr int res_min_blocks() { return (sizeof(T) == 4 && ROWS == 1) ? 5 : 4; }

template <typename T, typename S, bool OUT>
__global__ void __launch_bounds__(kThreads, ilu_min_blocks<T>()) k_ilu_b(Geom g, const S* __restrict__ At, const S* __restrict__ Dinv, const T* __restrict__ src,
                        T* __restrict__ tv, T* __restrict__ z, const T* __restrict__ e, OutV zo,
                        const DevState* st) {
  wait_prior_grid();
  if (st->done) return;
  for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < g.Nh; q += (int64_t)gridDim.x * blockDim.x) {
    const Cell c = decode(g, 1, q);
    T s[3];
    offdiag_sum(g, At, 1, q, c, tv, s);
    const T r0 = src[vidx(g, 0, 1, q)] - s[0], r1 = src[vidx(g, 1, 1, q)] - s[1], r2 = src[vidx(g, 2, 1, q)] - s[2];
    T d[9];
#pragma unroll
    for (int rc = 0; rc < 9; ++rc) d[rc] = cv<T>(Dinv[(size_t)rc * g.N + g.Nh + q]);
    const T u0 = d[0] * r0 + d[1] * r1 + d[2] * r2;
    const T u1 = d[3] * r0 + d[4] * r1 + d[5] * r2;
    const T u2 = d[6] * r0 + d[7] * r1 + d[8] * r2;
    if (OUT) {
      tv[vidx(g, 0, 1, q)] = u0;
      tv[vidx(g, 1, 1, q)] = u1;
      tv[vidx(g, 2, 1, q)] = u2;
      out_put<T>(zo, vidx(g, 0, 1, q), z[vidx(g, 0, 1, q)] + e[g.Nh + q] + u0);
      out_put<T>(zo, vidx(g, 1, 1, q), z[vidx(g, 1, 1, q)] + u1);
      out_put<T>(zo, vidx(g, 2, 1, q), z[vidx(g, 2, 1, q)] + u2);
    } else {
      z[vidx(g, 0, 1, q)] = u0;
      z[vidx(g, 1, 1, q)] = u1;
      z[vidx(g, 2, 1, q)] = u2;
    }
  }
}

// ILU pass 3 (red): corr = D_r^{-1} sum A_rb u_b, with u_b in `ub` (black half).
// OUT = false: z_r = t_r - corr (precision T).
// OUT = true: zo_r = z1_r + Pi_p e_r + t_r - corr, in FP64.
template <typename T, typename S, bool OUT>
__global__ void __launch_bounds__(kThreads, ilu_min_blocks<T>()) k_ilu_r2(Geom g, const S* __restrict__ At, const S* __restrict__ Dinv, const T* __restrict__ tv,
                         const T* __restrict__ ub, T* __restrict__ z, const T* __restrict__ e, OutV zo,
                         const DevState* st) {
  wait_prior_grid();
  if (st->done) return;
  for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < g.Nh; q += (int64_t)gridDim.x * blockDim.x) {
    const Cell c = decode(g, 0, q);
    T s[3];
    offdiag_sum(g, At, 0, q, c, ub, s);
    T d[9];
#pragma unroll
    for (int rc = 0; rc < 9; ++rc) d[rc] = cv<T>(Dinv[(size_t)rc * g.N + q]);
    const T c0 = d[0] * s[0] + d[1] * s[1] + d[2] * s[2];
    const T c1 = d[3] * s[0] + d[4] * s[1] + d[5] * s[2];
    const T c2 = d[6] * s[0] + d[7] * s[1] + d[8] * s[2];
    const T t0 = tv[vidx(g, 0, 0, q)] - c0, t1 = tv[vidx(g, 1, 0, q)] - c1, t2 = tv[vidx(g, 2, 0, q)] - c2;
    if (OUT) {
      out_put<T>(zo, vidx(g, 0, 0, q), z[vidx(g, 0, 0, q)] + e[q] + t0);
      out_put<T>(zo, vidx(g, 1, 0, q), z[vidx(g, 1, 0, q)] + t1);
      out_put<T>(zo, vidx(g, 2, 0, q), z[vidx(g, 2, 0, q)] + t2);
    } else {
      z[vidx(g, 0, 0, q)] = t0;
      z[vidx(g, 1, 0, q)] = t1;
      z[vidx(g, 2, 0, q)] = t2;
    }
  }
}

// Residuals of the decoupled system in precision T.
// ROWS = 1: out[t] = f_p - (At z)_p for all cells (the AMG right-hand side).
// ROWS = 3: out = f - At (z + Pi_p e), all components, fused with the first
//   ILU pass of the second local solve on red cells: tv_r = D_r^{-1} out_r.
template <typename T, typename S, int ROWS>
__global__ void __launch_bounds__(kThreads, res_min_blocks<T, ROWS>()) k_cpr_residual(Geom g, const S* __restrict__ At, const T* __restrict__ f, const T* __restrict__ z,
                               const T* __restrict__ e, T* __restrict__ out, const S* __restrict__ Dinv,
                               T* __restrict__ tv, const DevState* st) {
  wait_prior_grid();
  if (st->done) return;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < g.N; t += (int64_t)gridDim.x * blockDim.x) {
    const int color = (int)(t / g.Nh);
    const int64_t q = t - color * g.Nh;
    const Cell c = decode(g, color, q);
    T acc[ROWS];
#pragma unroll
    for (int r = 0; r < ROWS; ++r) acc[r] = T(0);
    // every slot's loads are issued whether or not its neighbour exists
    // (a missing one reads the cell's own entries and is masked to zero),
    // so all of a cell's loads can be in flight at once
#pragma unroll
    for (int sl = 0; sl < 7; ++sl) {
      const int64_t nb = nbr(g, c, q, sl);
      const bool ok = nb >= 0;
      const int64_t nq = ok ? nb : q;
      const int xc = (sl == kDiag || !ok) ? color : (color ^ 1);
      T x0 = z[vidx(g, 0, xc, nq)];
      if (ROWS == 3) x0 += e[(size_t)xc * g.Nh + nq];
      T x1 = z[vidx(g, 1, xc, nq)], x2 = z[vidx(g, 2, xc, nq)];
      if (!ok) x0 = x1 = x2 = T(0);
      const S* a = At + at_index(g, color, sl * 9, q);
      constexpr size_t P = 32;  // entries (rc) of a block lie 32 apart in a tile
#pragma unroll
      for (int r = 0; r < ROWS; ++r)
        acc[r] = fma3(acc[r], cv<T>(ld_stream(a + 3 * r * P)), x0, cv<T>(ld_stream(a + (3 * r + 1) * P)), x1,
                      cv<T>(ld_stream(a + (3 * r + 2) * P)), x2);
    }
    T res[ROWS];
#pragma unroll
    for (int r = 0; r < ROWS; ++r) {
      res[r] = f[(size_t)r * g.N + t] - acc[r];
      out[(size_t)r * g.N + t] = res[r];
    }
    if (ROWS == 3 && color == 0) {
      T d[9];
#pragma unroll
      for (int rc = 0; rc < 9; ++rc) d[rc] = cv<T>(Dinv[(size_t)rc * g.N + q]);
      tv[t] = d[0] * res[0] + d[1] * res[1 % ROWS] + d[2] * res[2 % ROWS];
      tv[g.N + t] = d[3] * res[0] + d[4] * res[1 % ROWS] + d[5] * res[2 % ROWS];
      tv[2 * g.N + t] = d[6] * res[0] + d[7] * res[1 % ROWS] + d[8] * res[2 % ROWS];
    }
  }
}

// ---- AMG level 0 (colour-split, coefficients = plane (colour, slot, 0) of At)
// One cell of a level-0 Gauss-Seidel half sweep.
template <typename T, typename S>
__device__ __forceinline__ T gs0_value(const Geom& g, const S* __restrict__ At, const T* __restrict__ f,
                                      const T* __restrict__ x, int color, int zero_guess, int64_t q) {
  const int oc = color ^ 1;
  T s = f[(size_t)color * g.Nh + q];
  if (!zero_guess) {
    const Cell c = decode(g, color, q);
#pragma unroll
    for (int sl = 0; sl < 7; ++sl) {
      if (sl == kDiag) continue;
      const int64_t nb = nbr(g, c, q, sl);
      const T xv = x[(size_t)oc * g.Nh + (nb >= 0 ? nb : q)];
      s -= cv<T>(At[at_index(g, color, sl * 9, q)]) * (nb >= 0 ? xv : T(0));
    }
  }
  return s / cv<T>(At[at_index(g, color, kDiag * 9, q)]);
}

// A level-0 half sweep over a grid-stride range, B cells per thread at a
// time: the loads of all B cells are issued before any store (the stores go
// to this colour's half of x, which no cell of the sweep reads), so a
// thread's cells overlap their memory latency instead of queueing it.
template <int B, typename T, typename F>
__device__ __forceinline__ void sweep_batched(int64_t t0, int64_t nt, int64_t n, T* __restrict__ out, F value) {
  for (int64_t q0 = t0; q0 < n; q0 += (int64_t)B * nt) {
    T v[B];
#pragma unroll
    for (int b = 0; b < B; ++b) {
      const int64_t q = q0 + b * nt;
      v[b] = q < n ? value(q) : T(0);
    }
#pragma unroll
    for (int b = 0; b < B; ++b) {
      const int64_t q = q0 + b * nt;
      if (q < n) out[q] = v[b];
    }
  }
}

// (B cells per thread at a time, their loads issued before their stores:
// a tile parameter of the per-kernel form that the batch autotuner sets)
template <typename T, typename S, int B>
__global__ void k_gs0(Geom g, const S* __restrict__ At, const T* __restrict__ f, T* __restrict__ x, int color,
                      int zero_guess, const DevState* st) {
  wait_prior_grid();
  if (st->done) return;
  sweep_batched<B>(blockIdx.x * (int64_t)blockDim.x + threadIdx.x, (int64_t)gridDim.x * blockDim.x, g.Nh,
                   x + (size_t)color * g.Nh, [&](int64_t q) { return gs0_value<T, S>(g, At, f, x, color, zero_guess, q); });
}

// First post-smoothing half sweep (black cells) with the coarse correction
// folded in: the red neighbours are read as x_r + s x_c(aggregate).  This
// equals prolongating x += s P x_c on every cell and then sweeping the black
// cells, because the black sweep overwrites x_b and the red sweep that
// follows overwrites x_r without reading its old value.
template <typename T, typename S>
__device__ __forceinline__ T gs0_prolong_value(const Geom& g, const S* __restrict__ At, const T* __restrict__ f,
                                              const T* __restrict__ x, const LevelDims& C, const T* __restrict__ xc,
                                              T sc, int64_t q) {
  const int di[7] = {0, 0, -1, 0, 1, 0, 0}, dj[7] = {0, -1, 0, 0, 0, 1, 0}, dk[7] = {-1, 0, 0, 0, 0, 0, 1};
  const Cell c = decode(g, 1, q);
  T s = f[(size_t)g.Nh + q];
#pragma unroll
  for (int sl = 0; sl < 7; ++sl) {
    if (sl == kDiag) continue;
    const int64_t nb = nbr(g, c, q, sl);
    const bool ok = nb >= 0;
    const int64_t cn = ok ? nat_index(C, (c.i + di[sl]) / 2, (c.j + dj[sl]) / 2, (c.k + dk[sl]) / 2) : 0;
    const T xv = x[ok ? nb : q] + sc * xc[cn];
    s -= cv<T>(At[at_index(g, 1, sl * 9, q)]) * (ok ? xv : T(0));
  }
  return s / cv<T>(At[at_index(g, 1, kDiag * 9, q)]);
}

template <typename T, typename S, int B>
__global__ void k_gs0_prolong(Geom g, const S* __restrict__ At, const T* __restrict__ f, T* __restrict__ x,
                              LevelDims C, const T* __restrict__ xc, T sc, const DevState* st) {
  wait_prior_grid();
  if (st->done) return;
  sweep_batched<B>(blockIdx.x * (int64_t)blockDim.x + threadIdx.x, (int64_t)gridDim.x * blockDim.x, g.Nh, x + g.Nh,
                   [&](int64_t q) { return gs0_prolong_value<T, S>(g, At, f, x, C, xc, sc, q); });
}

// Sum of level-0 residuals over aggregate I (red cells only when the last
// half sweep was black)
template <typename T, typename S>
__device__ __forceinline__ T restrict0_cell(const Geom& g, const S* __restrict__ At, const T* __restrict__ f,
                                            const T* __restrict__ x, const LevelDims& C, int64_t I, int red_only) {
  const Ijk cc = ijk_of(C, I);
  const int ci = cc.i, cj = cc.j, ck = cc.k;
  T acc = T(0);
  for (int dk = 0; dk < 2; ++dk)
    for (int dj = 0; dj < 2; ++dj)
      for (int di = 0; di < 2; ++di) {
        const int i = 2 * ci + di, j = 2 * cj + dj, k = 2 * ck + dk;
        if (i >= g.nx || j >= g.ny || k >= g.nz) continue;
        const int color = (i + j + k) & 1;
        if (red_only && color == 1) continue;
        const int64_t q = (i + (int64_t)g.nx * (j + (int64_t)g.ny * k)) >> 1;
        const Cell c{i, j, k, i & 1};
        T r = f[(size_t)color * g.Nh + q];
#pragma unroll
        for (int sl = 0; sl < 7; ++sl) {
          const int64_t nq = nbr(g, c, q, sl);
          if (nq < 0) continue;
          const int xc = (sl == kDiag) ? color : (color ^ 1);
          r -= cv<T>(At[at_index(g, color, sl * 9, q)]) * x[(size_t)xc * g.Nh + nq];
        }
        acc += r;
      }
  return acc;
}

template <typename T, typename S>
__global__ void k_restrict0(Geom g, const S* __restrict__ At, const T* __restrict__ f, const T* __restrict__ x,
                            LevelDims C, T* __restrict__ fc, int red_only, const DevState* st) {
  wait_prior_grid();
  if (st->done) return;
  for (int64_t I = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; I < C.n; I += (int64_t)gridDim.x * blockDim.x)
    fc[I] = restrict0_cell<T, S>(g, At, f, x, C, I, red_only);
}

template <typename T>
__device__ __forceinline__ void prolong0_cell(const Geom& g, T* __restrict__ x, const LevelDims& C,
                                              const T* __restrict__ xc, T s, int64_t t) {
  const int color = (int)(t / g.Nh);
  const int64_t q = t - color * g.Nh;
  const Cell c = decode(g, color, q);
  x[t] += s * xc[nat_index(C, c.i / 2, c.j / 2, c.k / 2)];
}

template <typename T>
__global__ void k_prolong0(Geom g, T* __restrict__ x, LevelDims C, const T* __restrict__ xc, T s, const DevState* st) {
  wait_prior_grid();
  if (st->done) return;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < g.N; t += (int64_t)gridDim.x * blockDim.x)
    prolong0_cell<T>(g, x, C, xc, s, t);
}

// ---- natural-order levels (device functions shared by the multi-block
// kernels and the single-block tail)
template <typename T, typename S = T>
struct LevelView {
  LevelDims d;
  const S* c;  // 7 n coefficients (storage type)
  T* f;
  T* x;
  __device__ __forceinline__ T cc(int slot, int64_t cidx) const { return cv<T>(c[slot * d.n + cidx]); }
};

// Loads of iterates and right-hand sides.  CG = true: through L2 only, for
// values that other thread blocks of the same launch wrote before a barrier
// (the cluster form of the coarse levels); false: ordinary loads.
template <bool CG, typename T>
__device__ __forceinline__ T ldv(const T* p) {
  if (CG) return __ldcg(p);
  return *p;
}

template <bool CG = false, typename T, typename S>
__device__ __forceinline__ void gs_cell(const LevelView<T, S>& L, int64_t cidx, int color, int zero_guess) {
  const Ijk p = ijk_of(L.d, cidx);
  const int i = p.i, j = p.j, k = p.k;
  if (((i + j + k) & 1) != color) return;
  T s = ldv<CG>(L.f + cidx);
  if (!zero_guess) {
    // every neighbour's loads are issued; a missing one reads the cell
    // itself and the value read is replaced by zero
    const int64_t nxy = (int64_t)L.d.nx * L.d.ny;
    const bool ok[6] = {k > 0, j > 0, i > 0, i < L.d.nx - 1, j < L.d.ny - 1, k < L.d.nz - 1};
    const int slot[6] = {kZm, kYm, kXm, kXp, kYp, kZp};
    const int64_t off[6] = {-nxy, -(int64_t)L.d.nx, -1, 1, (int64_t)L.d.nx, nxy};
#pragma unroll
    for (int d = 0; d < 6; ++d) {
      const T xv = ldv<CG>(L.x + (ok[d] ? cidx + off[d] : cidx));
      s -= L.cc(slot[d], cidx) * (ok[d] ? xv : T(0));
    }
  }
  L.x[cidx] = s / L.cc(kDiag, cidx);
}

template <bool CG = false, typename T, typename S>
__device__ __forceinline__ T residual_cell(const LevelView<T, S>& L, int i, int j, int k) {
  const int64_t cidx = nat_index(L.d, i, j, k);
  const int64_t nxy = (int64_t)L.d.nx * L.d.ny;
  T r = ldv<CG>(L.f + cidx) - L.cc(kDiag, cidx) * ldv<CG>(L.x + cidx);
  if (k > 0) r -= L.cc(kZm, cidx) * ldv<CG>(L.x + cidx - nxy);
  if (j > 0) r -= L.cc(kYm, cidx) * ldv<CG>(L.x + cidx - L.d.nx);
  if (i > 0) r -= L.cc(kXm, cidx) * ldv<CG>(L.x + cidx - 1);
  if (i < L.d.nx - 1) r -= L.cc(kXp, cidx) * ldv<CG>(L.x + cidx + 1);
  if (j < L.d.ny - 1) r -= L.cc(kYp, cidx) * ldv<CG>(L.x + cidx + L.d.nx);
  if (k < L.d.nz - 1) r -= L.cc(kZp, cidx) * ldv<CG>(L.x + cidx + nxy);
  return r;
}

template <bool CG = false, typename T, typename S>
__device__ __forceinline__ T restrict_cell(const LevelView<T, S>& F, const LevelDims& C, int64_t I, int red_only) {
  const Ijk cc = ijk_of(C, I);
  const int ci = cc.i, cj = cc.j, ck = cc.k;
  T acc = T(0);
  for (int dk = 0; dk < 2; ++dk)
    for (int dj = 0; dj < 2; ++dj)
      for (int di = 0; di < 2; ++di) {
        const int i = 2 * ci + di, j = 2 * cj + dj, k = 2 * ck + dk;
        if (i >= F.d.nx || j >= F.d.ny || k >= F.d.nz) continue;
        if (red_only && ((i + j + k) & 1)) continue;
        acc += residual_cell<CG>(F, i, j, k);
      }
  return acc;
}

template <bool CG = false, typename T, typename S>
__device__ __forceinline__ void prolong_cell(const LevelView<T, S>& F, const LevelView<T, S>& C, int64_t cidx, T s) {
  const Ijk p = ijk_of(F.d, cidx);
  const int i = p.i, j = p.j, k = p.k;
  F.x[cidx] = ldv<CG>(F.x + cidx) + s * ldv<CG>(C.x + nat_index(C.d, i / 2, j / 2, k / 2));
}

// black half sweep with the coarse correction of the red neighbours folded in
// (the natural-order counterpart of k_gs0_prolong)
template <bool CG = false, typename T, typename S>
__device__ __forceinline__ void gs_cell_prolong(const LevelView<T, S>& L, const LevelView<T, S>& C, int64_t cidx, T sc) {
  const Ijk p = ijk_of(L.d, cidx);
  const int i = p.i, j = p.j, k = p.k;
  if (((i + j + k) & 1) != 1) return;
  const int64_t nxy = (int64_t)L.d.nx * L.d.ny;
  T s = ldv<CG>(L.f + cidx);
  const bool ok[6] = {k > 0, j > 0, i > 0, i < L.d.nx - 1, j < L.d.ny - 1, k < L.d.nz - 1};
  const int slot[6] = {kZm, kYm, kXm, kXp, kYp, kZp};
  const int64_t off[6] = {-nxy, -(int64_t)L.d.nx, -1, 1, (int64_t)L.d.nx, nxy};
  const int ci[6] = {i / 2, i / 2, (i - 1) / 2, (i + 1) / 2, i / 2, i / 2};
  const int cj[6] = {j / 2, (j - 1) / 2, j / 2, j / 2, (j + 1) / 2, j / 2};
  const int ck[6] = {(k - 1) / 2, k / 2, k / 2, k / 2, k / 2, (k + 1) / 2};
#pragma unroll
  for (int d = 0; d < 6; ++d) {
    const int64_t fi = ok[d] ? cidx + off[d] : cidx;
    const int64_t cn = ok[d] ? nat_index(C.d, ci[d], cj[d], ck[d]) : nat_index(C.d, i / 2, j / 2, k / 2);
    const T xv = ldv<CG>(L.x + fi) + sc * ldv<CG>(C.x + cn);
    s -= L.cc(slot[d], cidx) * (ok[d] ? xv : T(0));
  }
  L.x[cidx] = s / L.cc(kDiag, cidx);
}

template <typename T, typename S>
__global__ void k_gsn_prolong(LevelView<T, S> L, LevelView<T, S> C, T sc, const DevState* st) {
  wait_prior_grid();
  if (st->done) return;
  for (int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; c < L.d.n; c += (int64_t)gridDim.x * blockDim.x)
    gs_cell_prolong(L, C, c, sc);
}

template <typename T, typename S>
__global__ void k_gsn(LevelView<T, S> L, int color, int zero_guess, const DevState* st) {
  wait_prior_grid();
  if (st->done) return;
  for (int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; c < L.d.n; c += (int64_t)gridDim.x * blockDim.x)
    gs_cell(L, c, color, zero_guess);
}

template <typename T, typename S>
__global__ void k_restrictn(LevelView<T, S> F, LevelView<T, S> C, int red_only, const DevState* st) {
  wait_prior_grid();
  if (st->done) return;
  for (int64_t I = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; I < C.d.n; I += (int64_t)gridDim.x * blockDim.x)
    C.f[I] = restrict_cell(F, C.d, I, red_only);
}

template <typename T, typename S>
__global__ void k_prolongn(LevelView<T, S> F, LevelView<T, S> C, T s, const DevState* st) {
  wait_prior_grid();
  if (st->done) return;
  for (int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; c < F.d.n; c += (int64_t)gridDim.x * blockDim.x)
    prolong_cell(F, C, c, s);
}

template <typename T, typename S>
struct TailArgs {
  int first, last;  // levels first..last (last = coarsest)
  int nu1, nu2;
  T s;
  LevelView<T, S> lv[24];
  const S* inv;     // dense inverse of level `last`
};

// Dynamic shared memory of the single-block tail (one symbol for the whole
// translation unit).
extern __shared__ __align__(16) uint8_t g_tail_smem[];

// Views of the tail levels: in global memory (the kernel's arguments), or
// staged in the tail's shared memory.  The shared-memory views are rebuilt
// from offsets into g_tail_smem at each use, so the compiler sees shared
// addresses and issues shared-memory loads (pointers read back from a
// shared struct would be generic and take the slower generic path).
template <typename T, typename S>
struct TailGlobalViews {
  const TailArgs<T, S>* a;
  __device__ LevelView<T, S> lv(int l) const { return a->lv[l]; }
  __device__ const S* inv() const { return a->inv; }
};
template <typename T, typename S>
struct TailSharedViews {
  const TailArgs<T, S>* a;
  const uint32_t* off;  // per level: coefficient, right-hand side and iterate offsets; the inverse at off[72]
  __device__ LevelView<T, S> lv(int l) const {
    LevelView<T, S> v = a->lv[l];
    v.c = reinterpret_cast<const S*>(g_tail_smem + off[3 * l]);
    v.f = reinterpret_cast<T*>(g_tail_smem + off[3 * l + 1]);
    v.x = reinterpret_cast<T*>(g_tail_smem + off[3 * l + 2]);
    return v;
  }
  __device__ const S* inv() const { return reinterpret_cast<const S*>(g_tail_smem + off[72]); }
};

// x_first = V-cycle(f_first) over levels first..last by one thread block
template <typename T, typename S, typename Views>
__device__ void tail_cycle(const TailArgs<T, S>& a, const Views& vw) {
  const int nt = blockDim.x;
  for (int l = a.first; l < a.last; ++l) {
    const LevelView<T, S> L = vw.lv(l);
    if (a.nu1 == 0) {
      for (int64_t c = threadIdx.x; c < L.d.n; c += nt) L.x[c] = T(0);
      __syncthreads();
    }
    for (int sw = 0; sw < a.nu1; ++sw)
      for (int color = 0; color < 2; ++color) {
        for (int64_t c = threadIdx.x; c < L.d.n; c += nt) gs_cell(L, c, color, sw == 0 && color == 0);
        __syncthreads();
      }
    const LevelView<T, S> C = vw.lv(l + 1);
    for (int64_t I = threadIdx.x; I < C.d.n; I += nt) C.f[I] = restrict_cell(L, C.d, I, a.nu1 > 0);
    __syncthreads();
  }
  {
    const LevelView<T, S> C = vw.lv(a.last);
    const S* inv = vw.inv();
    const int64_t n = C.d.n;
    for (int64_t i = threadIdx.x; i < n; i += nt) {
      T s = T(0);
      for (int64_t j = 0; j < n; ++j) s += cv<T>(inv[i * n + j]) * C.f[j];
      C.x[i] = s;
    }
    __syncthreads();
  }
  for (int l = a.last - 1; l >= a.first; --l) {
    const LevelView<T, S> L = vw.lv(l);
    const LevelView<T, S> C = vw.lv(l + 1);
    if (a.nu2 == 0) {
      for (int64_t c = threadIdx.x; c < L.d.n; c += nt) prolong_cell(L, C, c, a.s);
      __syncthreads();
    }
    for (int sw = 0; sw < a.nu2; ++sw)
      for (int color = 1; color >= 0; --color) {
        for (int64_t c = threadIdx.x; c < L.d.n; c += nt) {
          if (sw == 0 && color == 1) gs_cell_prolong(L, C, c, a.s);
          else gs_cell(L, c, color, 0);
        }
        __syncthreads();
      }
  }
}

template <typename T, typename S>
__global__ void __launch_bounds__(kTailThreads) k_tail(TailArgs<T, S> a, const DevState* st) {
  wait_prior_grid();
  if (st->done) return;
  tail_cycle(a, TailGlobalViews<T, S>{&a});
}

__host__ __device__ constexpr size_t align16(size_t b) { return (b + 15) & ~size_t(15); }

// shared-memory bytes that k_tail_smem needs for levels first..last
template <typename T, typename S>
__host__ __device__ size_t tail_smem_bytes(const TailArgs<T, S>& a) {
  size_t b = 0;
  for (int l = a.first; l <= a.last; ++l)
    b += align16(7 * a.lv[l].d.n * sizeof(S)) + 2 * align16(a.lv[l].d.n * sizeof(T));
  return b + align16((size_t)a.lv[a.last].d.n * a.lv[a.last].d.n * sizeof(S));
}

// The same V-cycle with the tail levels staged in shared memory: their
// coefficients, right-hand sides and iterates, and the coarse inverse, are
// copied in once, every sweep then reads shared memory instead of L2, and
// only the first tail level's iterate (read by the next finer level's
// prolongation) is copied back.
// Offsets of the tail levels in the dynamic shared memory (per level: the
// coefficients, the right-hand side and the iterate; the coarse inverse at
// off[72]), computed by thread 0.
template <typename T, typename S>
__device__ void tail_offsets(const TailArgs<T, S>& a, uint32_t* off) {
  if (threadIdx.x == 0) {
    uint32_t o = 0;
    for (int l = a.first; l <= a.last; ++l) {
      const uint32_t n = (uint32_t)a.lv[l].d.n;
      off[3 * l] = o;
      o += (uint32_t)align16(7 * n * sizeof(S));
      off[3 * l + 1] = o;
      o += (uint32_t)align16(n * sizeof(T));
      off[3 * l + 2] = o;
      o += (uint32_t)align16(n * sizeof(T));
    }
    off[72] = o;
  }
}

// Copies the tail levels' coefficients and the coarse inverse into shared
// memory (they do not change during a V-cycle; the caller synchronises).
template <typename T, typename S>
__device__ void tail_stage_coefficients(const TailArgs<T, S>& a, const TailSharedViews<T, S>& vw) {
  for (int l = a.first; l <= a.last; ++l) {
    const int64_t n = a.lv[l].d.n;
    S* c = const_cast<S*>(vw.lv(l).c);
    const S* src = a.lv[l].c;
#pragma unroll 8
    for (int64_t i = threadIdx.x; i < 7 * n; i += blockDim.x) c[i] = src[i];
  }
  const int64_t nc = a.lv[a.last].d.n;
  S* inv = const_cast<S*>(vw.inv());
#pragma unroll 8
  for (int64_t i = threadIdx.x; i < nc * nc; i += blockDim.x) inv[i] = a.inv[i];
}

// The same staging with asynchronous copies (cp.async, 16 bytes each; a
// remainder below 16 bytes is copied directly), so the block can go on with
// other work while they land; the caller waits (cp.async.wait_all) and
// synchronises before the staged values are read.  The sources are device
// allocations and the shared-memory offsets multiples of 16 bytes.
__device__ __forceinline__ void copy_to_shared_async(void* dst, const void* src, size_t bytes) {
  const size_t n16 = bytes / 16;
  const uint32_t d0 = (uint32_t)__cvta_generic_to_shared(dst);
  for (size_t i = threadIdx.x; i < n16; i += blockDim.x)
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(d0 + (uint32_t)(16 * i)),
                 "l"(reinterpret_cast<const char*>(src) + 16 * i)
                 : "memory");
  for (size_t b = 16 * n16 + threadIdx.x; b < bytes; b += blockDim.x)
    reinterpret_cast<char*>(dst)[b] = reinterpret_cast<const char*>(src)[b];
}

template <typename T, typename S>
__device__ void tail_stage_coefficients_async(const TailArgs<T, S>& a, const TailSharedViews<T, S>& vw) {
  for (int l = a.first; l <= a.last; ++l)
    copy_to_shared_async(const_cast<S*>(vw.lv(l).c), a.lv[l].c, (size_t)7 * a.lv[l].d.n * sizeof(S));
  const int64_t nc = a.lv[a.last].d.n;
  copy_to_shared_async(const_cast<S*>(vw.inv()), a.inv, (size_t)nc * nc * sizeof(S));
  asm volatile("cp.async.commit_group;" ::: "memory");
}

// The tail V-cycle on staged coefficients: the first tail level's
// right-hand side comes in from global memory (through L2: other blocks of
// a cooperative launch wrote it), and only its iterate goes back.
template <typename T, typename S>
__device__ void tail_run_staged(const TailArgs<T, S>& a, const TailSharedViews<T, S>& vw) {
  const int64_t n = a.lv[a.first].d.n;
  T* f = vw.lv(a.first).f;
  for (int64_t i = threadIdx.x; i < n; i += blockDim.x) f[i] = __ldcg(a.lv[a.first].f + i);
  __syncthreads();
  tail_cycle(a, vw);
  const T* x = vw.lv(a.first).x;
  for (int64_t i = threadIdx.x; i < n; i += blockDim.x) a.lv[a.first].x[i] = x[i];
}

template <typename T, typename S>
__global__ void __launch_bounds__(kTailThreads) k_tail_smem(TailArgs<T, S> a, const DevState* st) {
  wait_prior_grid();
  if (st->done) return;
  __shared__ uint32_t off[73];
  tail_offsets(a, off);
  __syncthreads();
  const TailSharedViews<T, S> vw{&a, off};
  tail_stage_coefficients(a, vw);
  tail_run_staged(a, vw);
}

// ---- the multi-block AMG levels in two cooperative launches
// Grid-wide barrier of a cooperative launch (all blocks resident): one
// arrival counter and one generation word in the device state.  The wait is
// bounded; if it runs out (which needs a block that never arrives) the
// barrier records kErrTimeout, and every later barrier of the launch fails
// at once, so the kernel returns and the solve reports BO_ERR_TIMEOUT.
// (the limit is a launch argument: bo_set_amg_barrier_spins lowers it)
// one block of 1024 threads per SM: a quarter of the arrivals at each
// barrier of four 256-thread blocks, for the same threads
constexpr int kCoopThreads = 1024;

__device__ __forceinline__ unsigned atom_add_release(unsigned* p, unsigned v) {
  unsigned old;
  asm volatile("atom.add.release.gpu.u32 %0, [%1], %2;" : "=r"(old) : "l"(p), "r"(v) : "memory");
  return old;
}
__device__ __forceinline__ unsigned ld_acquire(const unsigned* p) {
  unsigned v;
  asm volatile("ld.acquire.gpu.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

// The arrival is a release (every write the block made before the barrier,
// ordered by the block barrier ahead of it, is visible to whoever acquires
// the flipped word) and the polls are acquires; no separate fences.
__device__ __forceinline__ bool grid_barrier(DevState* st, unsigned spins) {
  __shared__ int ok;
  __syncthreads();
  if (threadIdx.x == 0) {
    volatile int* err = &st->err;
    int good = !(*err & kErrTimeout);
    if (good) {
      // One word per barrier round: block 0 adds 2^31 - (blocks - 1) and
      // every other block adds 1, so the round's arrivals sum to 2^31 and
      // the last one flips the word's top bit; a block has passed when the
      // top bit differs from the one its own addition saw.
      const unsigned inc = blockIdx.x == 0 ? 0x80000000u - (gridDim.x - 1) : 1u;
      const unsigned old = atom_add_release(&st->counter[5], inc);
      unsigned it = 0;
      while (((ld_acquire(&st->counter[5]) ^ old) & 0x80000000u) == 0) {
        if (++it > spins || (*err & kErrTimeout)) {
          atomicOr(&st->err, kErrTimeout);
          good = 0;
          break;
        }
        __nanosleep(32);
      }
    }
    ok = good;
  }
  __syncthreads();
  return ok;
}

// (i + j + k) even at a natural-order level
__device__ __forceinline__ bool red_cell(const LevelDims& L, int64_t c) {
  const Ijk p = ijk_of(L, c);
  return ((p.i + p.j + p.k) & 1) == 0;
}

template <typename T, typename S>
struct CycleArgs {
  Geom g;
  const S* At;
  T* f0;
  T* x0;
  int tail_from;  // first level of the single-block tail
  int legs_to;    // the down and up legs smooth levels 0 .. legs_to - 1 (the rest: the cluster kernel)
  int nu1, nu2;
  T s;
  unsigned spins;  // polls of a grid barrier before it gives up (BO_ERR_TIMEOUT)
  LevelView<T, S> lv[24];
};

// Down leg: level-0 pre-smoothing and restriction, then the same for the
// natural-order levels 1 .. tail_from - 1, a grid barrier after every half
// sweep (the kernel-per-half-sweep form launches each separately).
template <typename T, typename S>
__device__ bool amg_down(const CycleArgs<T, S>& a, DevState* st) {
  const int64_t t0 = blockIdx.x * (int64_t)blockDim.x + threadIdx.x, nt = (int64_t)gridDim.x * blockDim.x;
  const Geom& g = a.g;
  for (int sw = 0; sw < a.nu1; ++sw)
    for (int color = 0; color < 2; ++color) {
      const int zero = sw == 0 && color == 0;
      sweep_batched<4>(t0, nt, g.Nh, a.x0 + (size_t)color * g.Nh,
                       [&](int64_t q) { return gs0_value<T, S>(g, a.At, a.f0, a.x0, color, zero, q); });
      if (!grid_barrier(st, a.spins)) return false;
    }
  if (a.nu1 == 0) {
    for (int64_t t = t0; t < g.N; t += nt) a.x0[t] = T(0);
    if (!grid_barrier(st, a.spins)) return false;
  }
  // The first pre-smoothing half sweep of a multi-block level starts from
  // zero, x_r = f_r / a_rr: the thread that restricts a red cell's
  // right-hand side computes it at once, which saves that sweep's barrier.
  {
    const LevelView<T, S>& C = a.lv[1];
    const bool fold = a.nu1 > 0 && 1 < a.tail_from;
    for (int64_t I = t0; I < C.d.n; I += nt) {
      const T fI = restrict0_cell<T, S>(g, a.At, a.f0, a.x0, C.d, I, a.nu1 > 0);
      C.f[I] = fI;
      if (fold && red_cell(C.d, I)) C.x[I] = fI / C.cc(kDiag, I);
    }
  }
  for (int l = 1; l < a.legs_to; ++l) {
    if (!grid_barrier(st, a.spins)) return false;
    const LevelView<T, S>& L = a.lv[l];
    for (int sw = 0; sw < a.nu1; ++sw)
      for (int color = 0; color < 2; ++color) {
        if (sw == 0 && color == 0) continue;  // done with the restriction
        for (int64_t c = t0; c < L.d.n; c += nt) gs_cell(L, c, color, 0);
        if (!grid_barrier(st, a.spins)) return false;
      }
    if (a.nu1 == 0) {
      for (int64_t c = t0; c < L.d.n; c += nt) L.x[c] = T(0);
      if (!grid_barrier(st, a.spins)) return false;
    }
    const LevelView<T, S>& C = a.lv[l + 1];
    const bool fold = a.nu1 > 0 && l + 1 < a.tail_from;
    for (int64_t I = t0; I < C.d.n; I += nt) {
      const T fI = restrict_cell(L, C.d, I, a.nu1 > 0);
      C.f[I] = fI;
      if (fold && red_cell(C.d, I)) C.x[I] = fI / C.cc(kDiag, I);
    }
  }
  return true;
}

// Up leg: post-smoothing of levels tail_from - 1 .. 1 and then level 0, the
// first (black) half sweep of each level reading the coarse correction
template <typename T, typename S>
__device__ bool amg_up(const CycleArgs<T, S>& a, DevState* st) {
  const int64_t t0 = blockIdx.x * (int64_t)blockDim.x + threadIdx.x, nt = (int64_t)gridDim.x * blockDim.x;
  const Geom& g = a.g;
  for (int l = a.legs_to - 1; l >= 1; --l) {
    const LevelView<T, S>& L = a.lv[l];
    const LevelView<T, S>& C = a.lv[l + 1];
    if (a.nu2 == 0) {
      for (int64_t c = t0; c < L.d.n; c += nt) prolong_cell(L, C, c, a.s);
      if (!grid_barrier(st, a.spins)) return false;
    }
    for (int sw = 0; sw < a.nu2; ++sw)
      for (int color = 1; color >= 0; --color) {
        for (int64_t c = t0; c < L.d.n; c += nt) {
          if (sw == 0 && color == 1) gs_cell_prolong(L, C, c, a.s);
          else gs_cell(L, c, color, 0);
        }
        if (!grid_barrier(st, a.spins)) return false;
      }
  }
  const LevelView<T, S>& C1 = a.lv[1];
  if (a.nu2 == 0) {
    for (int64_t t = t0; t < g.N; t += nt) prolong0_cell<T>(g, a.x0, C1.d, C1.x, a.s, t);
    return true;
  }
  for (int sw = 0; sw < a.nu2; ++sw) {
    if (sw == 0)
      sweep_batched<4>(t0, nt, g.Nh, a.x0 + g.Nh, [&](int64_t q) {
        return gs0_prolong_value<T, S>(g, a.At, a.f0, a.x0, C1.d, C1.x, a.s, q);
      });
    else
      sweep_batched<4>(t0, nt, g.Nh, a.x0 + g.Nh,
                       [&](int64_t q) { return gs0_value<T, S>(g, a.At, a.f0, a.x0, 1, 0, q); });
    if (!grid_barrier(st, a.spins)) return false;
    sweep_batched<4>(t0, nt, g.Nh, a.x0, [&](int64_t q) { return gs0_value<T, S>(g, a.At, a.f0, a.x0, 0, 0, q); });
    if (sw + 1 < a.nu2 && !grid_barrier(st, a.spins)) return false;
  }
  return true;
}

template <typename T, typename S>
__global__ void __launch_bounds__(kCoopThreads, 1) k_amg_down(CycleArgs<T, S> a, DevState* st) {
  wait_prior_grid();
  if (st->done) return;
  amg_down(a, st);
}

template <typename T, typename S>
__global__ void __launch_bounds__(kCoopThreads, 1) k_amg_up(CycleArgs<T, S> a, DevState* st) {
  wait_prior_grid();
  if (st->done) return;
  amg_up(a, st);
}

// ---- the coarse levels (1 .. coarsest) in one thread-block cluster
// Hardware barrier of all threads of the cluster, with release / acquire
// semantics at cluster scope: every global-memory write of the cluster's
// thread blocks before it is visible to their reads after it (those reads
// also go through L2, ldv<true>).  It is not a spin on a flag: every thread
// of the cluster reaches every barrier (the control flow is uniform).
__device__ __forceinline__ void cluster_sync_all() {
  asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;" ::: "memory");
}

// The levels from a.legs_to (level 2; level 1, 131k cells at 128x128x64,
// stays in the cooperative legs, which give it the whole GPU) down to the
// coarsest, launched as a single cluster of up to 16 blocks (one per SM)
// after the down leg has restricted onto level a.legs_to: pre-smoothing and
// restriction of the multi-block levels, the tail V-cycle (levels of at
// most kTailCells cells) in the last block, in shared memory when it fits,
// then post-smoothing back up to level a.legs_to.
// The same sweeps as the down and up legs, with a cluster barrier (a few
// hundred nanoseconds) where they need a grid-wide one (several
// microseconds), on the L2-resident coarse data.
template <typename T, typename S>
__global__ void __launch_bounds__(kCoopThreads, 1) k_amg_coarse(CycleArgs<T, S> a, TailArgs<T, S> ta, int tail_smem,
                                                               const DevState* st) {
  wait_prior_grid();
  if (st->done) return;  // uniform: every block reads the same flag
  const int64_t t0 = blockIdx.x * (int64_t)blockDim.x + threadIdx.x, nt = (int64_t)gridDim.x * blockDim.x;
  // the last block runs the tail; it stages the tail's coefficients and
  // coarse inverse asynchronously at the start, under the multi-block levels
  const bool tail_block = blockIdx.x == gridDim.x - 1;
  __shared__ uint32_t off[73];
  const TailSharedViews<T, S> vw{&ta, off};
  if (tail_smem && tail_block) {
    tail_offsets(ta, off);
    __syncthreads();
    tail_stage_coefficients_async(ta, vw);
  }
  for (int l = a.legs_to; l < a.tail_from; ++l) {
    const LevelView<T, S>& L = a.lv[l];
    for (int sw = 0; sw < a.nu1; ++sw)
      for (int color = 0; color < 2; ++color) {
        if (sw == 0 && color == 0) continue;  // done with the restriction
        for (int64_t c = t0; c < L.d.n; c += nt) gs_cell<true>(L, c, color, 0);
        cluster_sync_all();
      }
    if (a.nu1 == 0) {
      for (int64_t c = t0; c < L.d.n; c += nt) L.x[c] = T(0);
      cluster_sync_all();
    }
    const LevelView<T, S>& C = a.lv[l + 1];
    const bool fold = a.nu1 > 0 && l + 1 < a.tail_from;
    for (int64_t I = t0; I < C.d.n; I += nt) {
      const T fI = restrict_cell<true>(L, C.d, I, a.nu1 > 0);
      C.f[I] = fI;
      if (fold && red_cell(C.d, I)) C.x[I] = fI / C.cc(kDiag, I);
    }
    cluster_sync_all();
  }
  if (tail_block) {
    if (tail_smem) {
      asm volatile("cp.async.wait_all;" ::: "memory");
      __syncthreads();
      tail_run_staged(ta, vw);
    } else {
      tail_cycle(ta, TailGlobalViews<T, S>{&ta});
    }
  }
  cluster_sync_all();
  for (int l = a.tail_from - 1; l >= a.legs_to; --l) {
    const LevelView<T, S>& L = a.lv[l];
    const LevelView<T, S>& C = a.lv[l + 1];
    if (a.nu2 == 0) {
      for (int64_t c = t0; c < L.d.n; c += nt) prolong_cell<true>(L, C, c, a.s);
      cluster_sync_all();
    }
    for (int sw = 0; sw < a.nu2; ++sw)
      for (int color = 1; color >= 0; --color) {
        for (int64_t c = t0; c < L.d.n; c += nt) {
          if (sw == 0 && color == 1) gs_cell_prolong<true>(L, C, c, a.s);
          else gs_cell<true>(L, c, color, 0);
        }
        cluster_sync_all();
      }
  }
}

// dense solve on level 0 when level 0 is the coarsest: x = inv f
template <typename T, typename S>
__global__ void k_dense0(int64_t n, const S* __restrict__ inv, const T* __restrict__ f, T* __restrict__ x,
                         const DevState* st) {
  wait_prior_grid();
  if (st->done) return;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    T s = T(0);
    for (int64_t j = 0; j < n; ++j) s += cv<T>(inv[i * n + j]) * f[j];
    x[i] = s;
  }
}

template <typename T>
__global__ void k_zero(int64_t n, T* __restrict__ x, const DevState* st) {
  wait_prior_grid();
  if (st->done) return;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    x[i] = T(0);
}

// z = Pi_p e (stage AMG alone), FP64 output
template <typename T>
__global__ void k_place_p(Geom g, const T* __restrict__ e, double* __restrict__ z, const DevState* st) {
  wait_prior_grid();
  if (st->done) return;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < g.N; t += (int64_t)gridDim.x * blockDim.x) {
    z[t] = (double)e[t];
    z[g.N + t] = 0.0;
    z[2 * g.N + t] = 0.0;
  }
}

// y = At x with At rebuilt in FP64 from A and the weights (parity checks)
__global__ void k_spmv_dec64(Geom g, const double* __restrict__ A, const double* __restrict__ w,
                             const double* __restrict__ x, double* __restrict__ y) {
  wait_prior_grid();
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < g.N; t += (int64_t)gridDim.x * blockDim.x) {
    const int color = (int)(t / g.Nh);
    const int64_t q = t - color * g.Nh;
    const Cell c = decode(g, color, q);
    double acc[3] = {0, 0, 0};
    for (int sl = 0; sl < 7; ++sl) {
      const int64_t nq = nbr(g, c, q, sl);
      if (nq < 0) continue;
      const int xc = (sl == kDiag) ? color : (color ^ 1);
      double b[9];
      dec_block(g, A, w, color, sl, q, b);
      for (int r = 0; r < 3; ++r)
        for (int k = 0; k < 3; ++k) acc[r] += b[3 * r + k] * x[vidx(g, k, xc, nq)];
    }
    for (int r = 0; r < 3; ++r) y[vidx(g, r, color, q)] = acc[r];
  }
}

// ---------------------------------------------------------------- host side
template <typename T, typename S>
LevelView<T, S> view(bo_prec* P, int l) {
  const Level& L = P->lev[l];
  return LevelView<T, S>{LevelDims{L.nx, L.ny, L.nz, L.n}, (const S*)L.c, (T*)L.f, (T*)L.x};
}

LevelDims dims_of(const Level& L) { return LevelDims{L.nx, L.ny, L.nz, L.n}; }

// Blocks of the cluster that runs the coarse AMG levels: 16 (a
// non-portable cluster size) where the device can co-schedule them with
// the tail's shared memory, else 8, else 0 (no cluster form).  Queried once
// per instantiation.
template <typename T, typename S>
int coarse_cluster_size() {
  static std::atomic<int> cached{-1};
  int cs = cached.load();
  if (cs >= 0) return cs;
  cs = 0;
  const void* k = (const void*)k_amg_coarse<T, S>;
  if (cudaFuncSetAttribute(k_amg_coarse<T, S>, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) == cudaSuccess &&
      cudaFuncSetAttribute(k_amg_coarse<T, S>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kTailSmemMax) ==
          cudaSuccess) {
    for (int c : {16, 8}) {
      cudaLaunchConfig_t cfg = {};
      cfg.gridDim = dim3(c, 1, 1);
      cfg.blockDim = dim3(kCoopThreads, 1, 1);
      cfg.dynamicSmemBytes = kTailSmemMax;
      cudaLaunchAttribute at[1];
      at[0].id = cudaLaunchAttributeClusterDimension;
      at[0].val.clusterDim.x = c;
      at[0].val.clusterDim.y = 1;
      at[0].val.clusterDim.z = 1;
      cfg.attrs = at;
      cfg.numAttrs = 1;
      int n = 0;
      if (cudaOccupancyMaxActiveClusters(&n, k, &cfg) == cudaSuccess && n >= 1) {
        cs = c;
        break;
      }
    }
  }
  cudaGetLastError();
  cached.store(cs);
  return cs;
}

template <typename T, typename S>
void amg_vcycle(bo_prec* P, const DevState* st) {
  cudaStream_t s = P->stream;
  const Geom& g = P->mat->g;
  const S* At = (const S*)P->At;
  T* f0 = (T*)P->f0;
  T* x0 = (T*)P->e0;
  const int nu1 = P->opts.amg_nu1, nu2 = P->opts.amg_nu2;
  const T sc = (T)P->opts.amg_overcorr;
  if (P->nlev == 1) {
    (launch_pdl(k_dense0<T, S>, grid_for(g.N), kThreads, 0, s, g.N, (const S*)P->coarse_inv, f0, x0, st), note_launch());
    return;
  }
  // tile parameters of the per-kernel form (set by the batch autotuner):
  // threads per block and level-0 cells per thread
  const int TB = P->amg_threads;
  const int CB = P->amg_cells;
  const int ghalf = grid_for((g.Nh + CB - 1) / CB, TB);
  auto gs0 = [&](int color, int zero) {
    if (CB == 4) (launch_pdl(k_gs0<T, S, 4>, ghalf, TB, 0, s, g, At, f0, x0, color, zero, st), note_launch());
    else if (CB == 2) (launch_pdl(k_gs0<T, S, 2>, ghalf, TB, 0, s, g, At, f0, x0, color, zero, st), note_launch());
    else (launch_pdl(k_gs0<T, S, 1>, ghalf, TB, 0, s, g, At, f0, x0, color, zero, st), note_launch());
  };
  auto gs0_prolong = [&]() {
    const LevelDims C1 = dims_of(P->lev[1]);
    const T* xc = (const T*)P->lev[1].x;
    if (CB == 4) (launch_pdl(k_gs0_prolong<T, S, 4>, ghalf, TB, 0, s, g, At, f0, x0, C1, xc, sc, st), note_launch());
    else if (CB == 2) (launch_pdl(k_gs0_prolong<T, S, 2>, ghalf, TB, 0, s, g, At, f0, x0, C1, xc, sc, st), note_launch());
    else (launch_pdl(k_gs0_prolong<T, S, 1>, ghalf, TB, 0, s, g, At, f0, x0, C1, xc, sc, st), note_launch());
  };
  const int last = P->nlev - 1;
  // Launch forms (all compute the same V-cycle):
  //  mode 2: levels 0 and 1 in two cooperative launches (down leg, up leg,
  //          grid barriers between half sweeps) around one cluster launch
  //          for every coarser level (cluster barriers);
  //  mode 1: the cooperative legs also smooth the multi-block natural
  //          levels, the tail levels in one block;
  //  mode 0, or inside stream capture, or when a launch form is refused:
  //          one kernel per half sweep, restriction and prolongation.
  const int mode = g_amg_coop.load();
  cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
  cudaStreamIsCapturing(s, &cap);
  const bool coop = mode != 0 && cap == cudaStreamCaptureStatusNone;
  const int cs = (coop && mode == 2) ? coarse_cluster_size<T, S>() : 0;
  CycleArgs<T, S> ca;
  ca.g = g;
  ca.At = At;
  ca.f0 = f0;
  ca.x0 = x0;
  ca.tail_from = P->tail_from;
  ca.legs_to = cs ? (P->tail_from < 2 ? P->tail_from : 2) : P->tail_from;
  ca.nu1 = nu1;
  ca.nu2 = nu2;
  ca.s = sc;
  ca.spins = g_amg_spins.load();
  for (int l = 1; l <= last; ++l) ca.lv[l] = view<T, S>(P, l);
  TailArgs<T, S> ta;
  ta.first = P->tail_from;
  ta.last = last;
  ta.nu1 = nu1;
  ta.nu2 = nu2;
  ta.s = sc;
  for (int l = 1; l <= last; ++l) ta.lv[l] = view<T, S>(P, l);
  ta.inv = (const S*)P->coarse_inv;
  const size_t tb = tail_smem_bytes(ta);
  DevState* stw = const_cast<DevState*>(st);

  // per-kernel pre- and post-smoothing of the multi-block natural levels
  auto natural_down = [&]() {
    for (int l = 1; l < P->tail_from; ++l) {
      LevelView<T, S> L = view<T, S>(P, l), C = view<T, S>(P, l + 1);
      const int gl = grid_for(L.d.n, TB);
      for (int sw = 0; sw < nu1; ++sw) {
        (launch_pdl(k_gsn<T, S>, gl, TB, 0, s, L, 0, sw == 0, st), note_launch());
        (launch_pdl(k_gsn<T, S>, gl, TB, 0, s, L, 1, 0, st), note_launch());
      }
      if (nu1 == 0) (launch_pdl(k_zero<T>, gl, TB, 0, s, L.d.n, L.x, st), note_launch());
      (launch_pdl(k_restrictn<T, S>, grid_for(C.d.n, TB), TB, 0, s, L, C, nu1 > 0, st), note_launch());
    }
  };
  auto natural_up = [&]() {
    for (int l = P->tail_from - 1; l >= 1; --l) {
      LevelView<T, S> L = view<T, S>(P, l), C = view<T, S>(P, l + 1);
      const int gl = grid_for(L.d.n, TB);
      if (nu2 == 0) (launch_pdl(k_prolongn<T, S>, gl, TB, 0, s, L, C, sc, st), note_launch());
      for (int sw = 0; sw < nu2; ++sw) {
        if (sw == 0) (launch_pdl(k_gsn_prolong<T, S>, gl, TB, 0, s, L, C, sc, st), note_launch());
        else (launch_pdl(k_gsn<T, S>, gl, TB, 0, s, L, 1, 0, st), note_launch());
        (launch_pdl(k_gsn<T, S>, gl, TB, 0, s, L, 0, 0, st), note_launch());
      }
    }
  };
  auto tail = [&]() {
    if (tb <= kTailSmemMax) {
      cudaFuncSetAttribute(k_tail_smem<T, S>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)tb);
      (launch_pdl(k_tail_smem<T, S>, 1, kTailThreads, tb, s, ta, st), note_launch());
    } else {
      (launch_pdl(k_tail<T, S>, 1, kTailThreads, 0, s, ta, st), note_launch());
    }
  };

  // a cooperative launch that may also start as soon as the previous
  // kernel's blocks have finished (programmatic dependent launch)
  auto launch_coop = [&](auto kern, int grid) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(grid, 1, 1);
    cfg.blockDim = dim3(kCoopThreads, 1, 1);
    cfg.stream = s;
    cudaLaunchAttribute at[2];
    at[0].id = cudaLaunchAttributeCooperative;
    at[0].val.cooperative = 1;
    at[1].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at[1].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = at;
    cfg.numAttrs = 2;
    return cudaLaunchKernelEx(&cfg, kern, ca, stw) == cudaSuccess;
  };

  // down leg
  bool down_done = false;
  if (coop) {
    const int gd = occ_grid((const void*)k_amg_down<T, S>, g.Nh, kCoopThreads);
    down_done = launch_coop(k_amg_down<T, S>, gd);
    if (down_done) note_launch();
    else cudaGetLastError();
  }
  if (!down_done) {
    for (int sw = 0; sw < nu1; ++sw) {
      gs0(0, sw == 0);
      gs0(1, 0);
    }
    if (nu1 == 0) (launch_pdl(k_zero<T>, grid_for(g.N, TB), TB, 0, s, g.N, x0, st), note_launch());
    (launch_pdl(k_restrict0<T, S>, grid_for(P->lev[1].n, TB), TB, 0, s, g, At, f0, x0, dims_of(P->lev[1]),
        (T*)P->lev[1].f, nu1 > 0, st), note_launch());
    natural_down();
    tail();
  } else if (cs > 0) {
    // every coarser level in one cluster launch (or per kernel if refused)
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(cs, 1, 1);
    cfg.blockDim = dim3(kCoopThreads, 1, 1);
    cfg.dynamicSmemBytes = tb <= kTailSmemMax ? tb : 0;
    cfg.stream = s;
    cudaLaunchAttribute at[2];
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = cs;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    at[1].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at[1].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = at;
    cfg.numAttrs = 2;
    if (cudaLaunchKernelEx(&cfg, k_amg_coarse<T, S>, ca, ta, tb <= kTailSmemMax ? 1 : 0, st) == cudaSuccess) {
      note_launch();
    } else {
      cudaGetLastError();
      natural_down();
      tail();
      natural_up();
    }
  } else {
    tail();
  }

  // up leg
  if (down_done) {
    const int gu = occ_grid((const void*)k_amg_up<T, S>, g.Nh, kCoopThreads);
    if (launch_coop(k_amg_up<T, S>, gu)) {
      note_launch();
      return;
    }
    cudaGetLastError();
    if (cs == 0) natural_up();
  } else {
    natural_up();
  }
  if (nu2 == 0)
    (launch_pdl(k_prolong0<T>, grid_for(g.N, TB), TB, 0, s, g, x0, dims_of(P->lev[1]), (const T*)P->lev[1].x, sc, st),
     note_launch());
  for (int sw = 0; sw < nu2; ++sw) {
    if (sw == 0) gs0_prolong();
    else gs0(1, 0);
    gs0(0, 0);
  }
}

// z = CPR stage applied to v (FP64, internal order); result FP64 in zo
template <typename T, typename S>
void cpr_apply(bo_prec* P, InV v, OutV zo, int stage, const DevState* st, const double* vs) {
  cudaStream_t s = P->stream;
  const Geom& g = P->mat->g;
  const int gN = grid_for(g.N), gh = grid_for(g.Nh);
  const S* At = (const S*)P->At;
  const S* D = (const S*)P->Dinv;
  T* f = (T*)P->f;
  T* tv = (T*)P->t;
  T* r = (T*)P->r;
  T* e0 = (T*)P->e0;
  T* f0 = (T*)P->f0;
  T* z1 = (T*)P->z1;
  if (stage == BO_STAGE_AMG) {  // (v is a caller's FP64 vector here: vs is NULL)
    (launch_pdl(k_copy_vec<T>, gN, kThreads, 0, s, g.N, v.d, f0, st), note_launch());
    amg_vcycle<T, S>(P, st);
    learned_coarse_apply(P, st);
    (launch_pdl(k_place_p<T>, gN, kThreads, 0, s, g, e0, zo.d, st), note_launch());
    return;
  }
  // x1 = R^{-1} f with f = D_QI^{-1} v (stage CPR) or f = v
  if (stage == BO_STAGE_CPR)
    (launch_pdl(k_cpr_entry<T, S, true>, occ_grid((const void*)k_cpr_entry<T, S, true>, g.N), kThreads, 0, s, g, v, vs, P->w, P->wf,
        D, f, tv, st),
     note_launch());
  else
    (launch_pdl(k_cpr_entry<T, S, false>, occ_grid((const void*)k_cpr_entry<T, S, false>, g.N), kThreads, 0, s, g, v, vs, P->w, P->wf,
        D, f, tv, st),
     note_launch());
  (launch_pdl(k_ilu_b<T, S, false>, occ_grid((const void*)k_ilu_b<T, S, false>, g.Nh), kThreads, 0, s, g, At, D, f, tv, z1, nullptr,
      OutV{}, st),
   note_launch());
  // (ub and z are both z1: the pass reads its black half and writes its red half)
  (launch_pdl(k_ilu_r2<T, S, false>, occ_grid((const void*)k_ilu_r2<T, S, false>, g.Nh), kThreads, 0, s, g, At, D, tv, z1, z1,
      nullptr, OutV{}, st),
   note_launch());
  if (stage == BO_STAGE_ILU) {
    (launch_pdl(k_widen_t<T>, grid_for(3 * g.N), kThreads, 0, s, 3 * g.N, z1, zo.d, st), note_launch());
    return;
  }
  // x2 = x1 + Pi_p AMG(A_pp)^{-1} Pi_r (f - At x1)
  (launch_pdl(k_cpr_residual<T, S, 1>, occ_grid((const void*)k_cpr_residual<T, S, 1>, g.N), kThreads, 0, s, 
       g, At, f, z1, nullptr, f0, nullptr, nullptr, st),
   note_launch());
  amg_vcycle<T, S>(P, st);
  learned_coarse_apply(P, st);
  // r = f - At x2 (with the red pass of R^{-1} r fused);  x3 = x2 + R^{-1} r
  (launch_pdl(k_cpr_residual<T, S, 3>, occ_grid((const void*)k_cpr_residual<T, S, 3>, g.N), kThreads, 0, s, g, At, f, z1, e0, r,
      D, tv, st),
   note_launch());
  (launch_pdl(k_ilu_b<T, S, true>, occ_grid((const void*)k_ilu_b<T, S, true>, g.Nh), kThreads, 0, s, g, At, D, r, tv, z1, e0, zo,
      st),
   note_launch());
  (launch_pdl(k_ilu_r2<T, S, true>, occ_grid((const void*)k_ilu_r2<T, S, true>, g.Nh), kThreads, 0, s, g, At, D, tv, tv, z1, e0,
      zo, st),
   note_launch());
}

template <typename S>
int values_impl(bo_prec* P) {
  bo_mat* m = P->mat;
  cudaStream_t s = P->stream;
  const Geom& g = m->g;
  const int gN = grid_for(g.N), gh = grid_for(g.Nh);
  (launch_pdl(k_decouple<S>, gN, kThreads, 0, s, g, m->A, m->a2_valid ? m->A2 : nullptr, m->a2_range, (S*)P->At, P->w, P->wf,
      P->opts.decoupling == BO_DECOUPLE_ABF, P->st), note_launch());
  // FP64 red inverses for the black pass: the Krylov basis is idle during setup
  double* red64 = P->V;
  if (sizeof(S) < sizeof(double) && m->a2_valid) {
    // black pivots in split arithmetic (the kernel takes the FP64 products
    // itself where the split copy of A could not hold every value)
    (launch_pdl(k_ilu_red<S, true>, gh, kThreads, 0, s, g, m->A, P->w, (S*)P->Dinv, red64, P->st), note_launch());
    (launch_pdl(k_ilu_black_split<S>, gh, kThreads, 0, s, g, m->A2, m->A, m->a2_range, P->w,
        reinterpret_cast<const float2*>(red64), (S*)P->Dinv, P->st),
     note_launch());
  } else {
    (launch_pdl(k_ilu_red<S, false>, gh, kThreads, 0, s, g, m->A, P->w, (S*)P->Dinv, red64, P->st), note_launch());
    (launch_pdl(k_ilu_black<S>, gh, kThreads, 0, s, g, m->A, P->w, red64, (S*)P->Dinv, P->st), note_launch());
  }
  // AMG hierarchy values
  for (int l = 1; l < P->nlev; ++l) {
    Level& C = P->lev[l];
    if (l == 1)
      (launch_pdl(k_galerkin0, grid_for(C.n), kThreads, 0, s, g, m->A, P->w, dims_of(C), C.c64, P->st), note_launch());
    else
      (launch_pdl(k_galerkinn, grid_for(C.n), kThreads, 0, s, dims_of(P->lev[l - 1]), P->lev[l - 1].c64, dims_of(C), C.c64,
          P->st), note_launch());
    (launch_pdl(k_convert<S>, grid_for(7 * C.n), kThreads, 0, s, C.c64, (S*)C.c, (size_t)7 * C.n), note_launch());
  }
  const int last = P->nlev - 1;
  LevelDims cd = last == 0 ? LevelDims{g.nx, g.ny, g.nz, g.N} : dims_of(P->lev[last]);
  (launch_pdl(k_dense_from_level, 1, kThreads, 0, s, cd, last == 0 ? nullptr : P->lev[last].c64, g, m->A, P->w, last == 0,
      P->coarse64), note_launch());
  const int n = (int)P->ncoarse;
  const size_t smem = (size_t)n * n * sizeof(double) + (size_t)n * sizeof(int);
  cudaFuncSetAttribute(k_gj_inverse<S>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  (launch_pdl(k_gj_inverse<S>, 1, 1024, smem, s, n, P->coarse64, (S*)P->coarse_inv, P->st), note_launch());
  if (cudaGetLastError() != cudaSuccess) return BO_ERR_CUDA;
  return learned_coarse_values(P);
}

}  // namespace

int prec_alloc(bo_prec* P) {
  const Geom& g = P->mat->g;
  const size_t ts = P->tsize;
  bool ok = true;
  auto al = [&](size_t bytes) -> void* {
    void* p = nullptr;
    if (ok && cudaMalloc(&p, bytes) != cudaSuccess) { ok = false; return nullptr; }
    return p;
  };
  const size_t ss = P->ssize;  // storage of the matrix-like arrays
  P->At = al(a2_size(g) * ss);  // tiled like the split copy of A (at_index)
  P->w = (double*)al((size_t)3 * g.N * sizeof(double));
  P->wf = ts == sizeof(float) ? (float*)al((size_t)3 * g.N * sizeof(float)) : nullptr;
  P->Dinv = al((size_t)9 * g.N * ss);
  P->f = al((size_t)3 * g.N * ts);
  P->t = al((size_t)3 * g.N * ts);
  P->r = al((size_t)3 * g.N * ts);
  P->z1 = al((size_t)3 * g.N * ts);
  P->e0 = al((size_t)g.N * ts);
  P->f0 = al((size_t)g.N * ts);
  // AMG hierarchy shape
  int coarse_max = P->opts.amg_coarse_max;
  if (coarse_max <= 0 || coarse_max > kCoarseMax) coarse_max = kCoarseMax;
  P->nlev = 1;
  int nx = g.nx, ny = g.ny, nz = g.nz;
  int64_t n = g.N;
  while (n > coarse_max && P->nlev < 24) {
    nx = (nx + 1) / 2; ny = (ny + 1) / 2; nz = (nz + 1) / 2;
    n = (int64_t)nx * ny * nz;
    Level& L = P->lev[P->nlev];
    L.nx = nx; L.ny = ny; L.nz = nz; L.n = n;
    L.c64 = (double*)al((size_t)7 * n * sizeof(double));
    L.c = al((size_t)7 * n * ss);
    L.f = al((size_t)n * ts);
    L.x = al((size_t)n * ts);
    P->nlev++;
  }
  if (n > kCoarseMax) return BO_ERR_ARG;
  P->ncoarse = n;
  P->tail_from = P->nlev - 1;
  for (int l = 1; l < P->nlev; ++l)
    if (P->lev[l].n <= kTailCells) { P->tail_from = l; break; }
  if (P->tail_from < 1) P->tail_from = 1;
  P->coarse64 = (double*)al((size_t)n * n * sizeof(double));
  P->coarse_inv = al((size_t)n * n * ss);
  if (ok && cudaMalloc(&P->st, sizeof(DevState)) != cudaSuccess) ok = false;
  if (ok) cudaMemsetAsync(P->st, 0, sizeof(DevState), P->stream);
  return ok ? BO_OK : BO_ERR_OOM;
}

void prec_free(bo_prec* P) {
  auto fr = [](void* p) { if (p) cudaFree(p); };
  fr(P->At); fr(P->w); fr(P->wf); fr(P->Dinv);
  fr(P->f); fr(P->t); fr(P->r); fr(P->z1); fr(P->e0); fr(P->f0);
  for (int l = 1; l < P->nlev; ++l) { fr(P->lev[l].c64); fr(P->lev[l].c); fr(P->lev[l].f); fr(P->lev[l].x); }
  fr(P->coarse64); fr(P->coarse_inv); fr(P->st);
  learned_coarse_free(P);
  graphs_reset(P);
  if (P->cap_stream) cudaStreamDestroy(P->cap_stream);
  P->cap_stream = nullptr;
}

int prec_values(bo_prec* P) {
  if (P->bf16) return values_impl<__nv_bfloat16>(P);
  return P->fp32 ? values_impl<float>(P) : values_impl<double>(P);
}

int launch_dense_inverse64(int n, const double* M, double* Minv, DevState* st, cudaStream_t s) {
  if (n < 1 || n > kCoarseMax) return BO_ERR_ARG;
  const size_t smem = (size_t)n * n * sizeof(double) + (size_t)n * sizeof(int);
  cudaFuncSetAttribute(k_gj_inverse<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  (launch_pdl(k_gj_inverse<double>, 1, 1024, smem, s, n, M, Minv, st), note_launch());
  return cudaGetLastError() == cudaSuccess ? BO_OK : BO_ERR_CUDA;
}

void launch_cpr(bo_prec* P, const double* v, double* z, int stage, const DevState* st, const double* vs) {
  const int64_t n = 3 * P->mat->g.N;
  const InV in{v, nullptr, n};
  const OutV out{z, nullptr, n};
  if (P->bf16) cpr_apply<float, __nv_bfloat16>(P, in, out, stage, st, vs);
  else if (P->fp32) cpr_apply<float, float>(P, in, out, stage, st, vs);
  else cpr_apply<double, double>(P, in, out, stage, st, vs);
}

void launch_cpr_split(bo_prec* P, const double* v, float* z, const DevState* st, const double* vs) {
  const int64_t n = 3 * P->mat->g.N;
  const InV in{v, nullptr, n};
  const OutV out{nullptr, z, n};
  if (P->bf16) cpr_apply<float, __nv_bfloat16>(P, in, out, BO_STAGE_CPR, st, vs);
  else if (P->fp32) cpr_apply<float, float>(P, in, out, BO_STAGE_CPR, st, vs);
  else cpr_apply<double, double>(P, in, out, BO_STAGE_CPR, st, vs);
}

void launch_cpr_split_in(bo_prec* P, const float* v, float* z, const DevState* st, const double* vs) {
  const int64_t n = 3 * P->mat->g.N;
  const InV in{nullptr, v, (n + 3) & ~(int64_t)3};  // the basis layout: low plane at n rounded up to 4
  const OutV out{nullptr, z, n};
  if (P->bf16) cpr_apply<float, __nv_bfloat16>(P, in, out, BO_STAGE_CPR, st, vs);
  else if (P->fp32) cpr_apply<float, float>(P, in, out, BO_STAGE_CPR, st, vs);
  else cpr_apply<double, double>(P, in, out, BO_STAGE_CPR, st, vs);
}

void launch_spmv_decoupled_internal(bo_prec* P, const double* x, double* y) {
  const Geom& g = P->mat->g;
  (launch_pdl(k_spmv_dec64, grid_for(g.N), kThreads, 0, P->stream, g, P->mat->A, P->w, x, y), note_launch());
}

}  // namespace bo
