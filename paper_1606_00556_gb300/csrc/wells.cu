// Rate-controlled wells: the bordered Newton system of paper Sec. 2.3 (a
// well under a fixed water, oil or liquid rate has its bottom-hole pressure
// p_h as an unknown and one constraint row) in the block form of Sec. 3.2,
//
//     [ A     A_pw ] [x  ]   [b  ]
//     [ A_wp  A_ww ] [x_w] = [b_w],
//
// with A the reservoir BSR matrix, A_pw the well columns (three entries in
// the rows of each perforated cell), A_wp the well rows (three entries per
// perforation) and A_ww diagonal (a constraint involves only its own p_h).
//
// The solve eliminates the wells exactly.  With U = A_pw A_ww^{-1} and
// V^T = A_wp, x solves the reservoir system S x = g with the Schur
// complement S = A - U V^T and g = b - U b_w, and x_w = A_ww^{-1}(b_w - A_wp x).
// FGMRES runs on S: each Arnoldi product is the solver's own product A z
// followed by a rank-W correction on the perforated rows.  The
// preconditioner is the CPR M of A with the well coupling folded in by the
// Woodbury identity,
//
//     P = (M^{-1} - U V^T)^{-1} = M + (M U) C^{-1} V^T M,   C = I - V^T M U,
//
// so P S is as close to the identity as M A is, whatever the wells do to
// the perforated rows.  M U (W vectors of 3N) and C^{-1} (W x W) are formed
// once per preconditioner and well values (W applications of M); each
// iteration then adds one pass over M U to the preconditioned vector.
// Because V^T applied to the corrected vector equals C^{-1} V^T M r, both
// corrections of an iteration come from the W numbers V^T M r.
//
// Layout: the perforations are grouped by well (perf_well non-decreasing);
// a cell is perforated at most once, so the corrections touch disjoint
// rows.  Internal vectors use the solver's colour-split order; the caller's
// vectors are natural order, 3N cell unknowns followed by the W well
// unknowns.
#include <cmath>
#include <cstring>
#include <new>
#include <vector>

#include "bo_internal.cuh"

using namespace bo;

struct bo_wells {
  bo_mat* mat;
  int32_t W, P;
  int32_t* wstart;     // W + 1 perforation offsets per well
  int32_t* perf_cell;  // natural cell of each perforation
  int32_t* perf_t;     // its position in a colour-split plane
  int32_t* perf_well;
  double* apw;         // 3P: d(cell equations)/d p_h
  double* awp;         // 3P: d(well constraint)/d(cell unknowns)
  double* aww;         // W
  bool values_set;
  unsigned long long version;
  int coupling;        // 1: Woodbury correction of the preconditioner, 0: none
  // preconditioner-dependent state (valid for prep_prec at prep_setups / prep_version)
  const bo_prec* prep_prec;
  unsigned long long prep_setups, prep_version;
  float* MU;           // W x 3N: M applied to each column of U, internal order
  double* Cinv;        // W x W
  double* t;           // 2W: per-column coefficients (t1, t2)
  // natural-order scratch of the solve
  double* g;           // 3N Schur right-hand side
  double* rfull;       // 3N + W residual of a nonzero initial guess
  double* dx;          // 3N + W correction
  double* partials;
  double* norms;       // device: squared norms
  double* h_norms;     // pinned mirror
};

namespace bo {
void mat_release_ref(bo_mat* m);
}

namespace {

constexpr int kMaxWells = 128;
constexpr int kRed = 4 * 152;

// s_v = sum over the perforations of well v of awp . z; one warp per well,
// lanes over the perforations, a fixed summation order.  z: FP64 internal
// vector (Z = double) or split planes (Z = float, low plane at z + n).
template <typename Z>
__device__ void perf_dots(int W, const int32_t* wstart, const int32_t* perf_t, int64_t N, const double* awp,
                          const Z* z, int64_t n, double* s) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
  for (int v = warp; v < W; v += nw) {
    double acc = 0.0;
    for (int e = wstart[v] + lane; e < wstart[v + 1]; e += 32) {
      const int64_t t0 = perf_t[e];
#pragma unroll
      for (int u = 0; u < 3; ++u) {
        const int64_t i = u * N + t0;
        double zi;
        if constexpr (sizeof(Z) == 4) zi = (double)z[i] + (double)z[n + i];
        else zi = z[i];
        acc = fma(awp[3 * e + u], zi, acc);
      }
    }
    acc = warp_sum(acc);
    if (lane == 0) s[v] = acc;
  }
}

// After the preconditioner: s = A_wp z, t1 = C^{-1} s (coupling) or s,
// t2 = A_ww^{-1} t1.  One block.
__global__ void k_wl_coeffs(int W, const int32_t* wstart, const int32_t* perf_t, int64_t N, const double* awp,
                            const float* z, int64_t n, const double* Cinv, const double* aww, int coupling,
                            double* t, const DevState* st) {
  wait_prior_grid();
  if (st->done) return;
  __shared__ double s[kMaxWells];
  perf_dots<float>(W, wstart, perf_t, N, awp, z, n, s);
  __syncthreads();
  for (int v = threadIdx.x; v < W; v += blockDim.x) {
    double t1 = s[v];
    if (coupling) {
      t1 = 0.0;
      for (int u = 0; u < W; ++u) t1 = fma(Cinv[(size_t)v * W + u], s[u], t1);
    }
    t[v] = t1;
    t[W + v] = t1 / aww[v];
  }
}

// z += (M U) t1 on the split planes of a preconditioned vector, in split
// arithmetic (FP32 M U columns, coefficients split once per block)
__global__ void __launch_bounds__(kThreads) k_wl_woodbury(int64_t n, int W, const float* __restrict__ MU,
                                                          const double* __restrict__ t, float* __restrict__ z,
                                                          const DevState* st) {
  wait_prior_grid();
  if (st->done) return;
  __shared__ df ts[kMaxWells];
  for (int v = threadIdx.x; v < W; v += blockDim.x) ts[v] = df_from(t[v]);
  __syncthreads();
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    df acc{z[i], z[n + i]};
    for (int v = 0; v < W; ++v) acc = df_fma_acc(acc, df{__ldcs(MU + (size_t)v * n + i), 0.f}, ts[v]);
    acc = df_renorm(acc);
    z[i] = acc.hi;
    z[n + i] = acc.lo;
  }
}

// After the Arnoldi product w = A z: w -= A_pw t2 on the perforated rows
// (split planes, low plane at w + np).  One block.
__global__ void k_wl_product(int P, int W, const int32_t* perf_t, const int32_t* perf_well, int64_t N,
                             const double* apw, const double* t, float* w, int64_t np, const DevState* st) {
  wait_prior_grid();
  if (st->done) return;
  for (int e = threadIdx.x; e < P; e += blockDim.x) {
    const double tv = t[W + perf_well[e]];
    const int64_t t0 = perf_t[e];
#pragma unroll
    for (int u = 0; u < 3; ++u) {
      const int64_t i = u * N + t0;
      const df d = df_from((double)w[i] + (double)w[np + i] - apw[3 * e + u] * tv);
      w[i] = d.hi;
      w[np + i] = d.lo;
    }
  }
}

// The true residual of S: r = (g - A x) + A_pw A_ww^{-1} A_wp x on the
// perforated rows (x, r FP64 internal).  One block.
__global__ void k_wl_residual(int W, const int32_t* wstart, const int32_t* perf_t, int64_t N, const double* awp,
                              const double* apw, const double* aww, const double* x, double* r) {
  wait_prior_grid();
  __shared__ double s[kMaxWells];
  perf_dots<double>(W, wstart, perf_t, N, awp, x, 0, s);
  __syncthreads();
  for (int v = 0; v < W; ++v) {
    const double tv = s[v] / aww[v];
    for (int e = wstart[v] + threadIdx.x; e < wstart[v + 1]; e += blockDim.x) {
      const int64_t t0 = perf_t[e];
#pragma unroll
      for (int u = 0; u < 3; ++u) r[u * N + t0] = fma(apw[3 * e + u], tv, r[u * N + t0]);
    }
  }
}

// ||r|| -> st->beta (the solver's reduction pattern; counter[1] is free
// once the true-residual kernel before it has finished)
__global__ void k_wl_beta(int64_t n, const double* __restrict__ r, double* partials, DevState* st) {
  wait_prior_grid();
  __shared__ double sh[32];
  double acc = 0.0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    acc = fma(r[i], r[i], acc);
  acc = block_sum(acc, sh);
  if (threadIdx.x == 0) partials[blockIdx.x] = acc;
  if (last_block(&st->counter[1], gridDim.x)) {
    double s = 0.0;
    for (int i = threadIdx.x; i < (int)gridDim.x; i += blockDim.x) s += __ldcg(partials + i);
    s = block_sum(s, sh);
    if (threadIdx.x == 0) {
      st->beta = sqrt(s);
      st->counter[1] = 0;
    }
  }
}

// out[slot] = sum of squares of v[0..n), deterministic two-phase reduction
__global__ void k_wl_sumsq(int64_t n, const double* __restrict__ v, double* partials) {
  wait_prior_grid();
  __shared__ double sh[32];
  double acc = 0.0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    acc = fma(v[i], v[i], acc);
  acc = block_sum(acc, sh);
  if (threadIdx.x == 0) partials[blockIdx.x] = acc;
}
__global__ void k_wl_sumsq_finish(int np, const double* partials, double* out) {
  wait_prior_grid();
  __shared__ double sh[32];
  double s = 0.0;
  for (int i = threadIdx.x; i < np; i += blockDim.x) s += partials[i];
  s = block_sum(s, sh);
  if (threadIdx.x == 0) *out = s;
}

// g = b - A_pw A_ww^{-1} b_w on the perforated rows of a copy of b (natural order)
__global__ void k_wl_rhs(int P, int64_t N, const int32_t* perf_cell, const int32_t* perf_well, const double* apw,
                         const double* aww, const double* b, double* g) {
  wait_prior_grid();
  for (int e = threadIdx.x; e < P; e += blockDim.x) {
    const int v = perf_well[e];
    const double tv = b[3 * N + v] / aww[v];
    const int64_t c = perf_cell[e];
#pragma unroll
    for (int u = 0; u < 3; ++u) g[3 * c + u] = fma(-apw[3 * e + u], tv, g[3 * c + u]);
  }
}

// x_w = A_ww^{-1} (b_w - A_wp x) (natural order; x_w at x + 3N)
__global__ void k_wl_recover(int W, const int32_t* wstart, const int32_t* perf_cell, int64_t N, const double* awp,
                             const double* aww, const double* b, double* x) {
  wait_prior_grid();
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
  for (int v = warp; v < W; v += nw) {
    double acc = 0.0;
    for (int e = wstart[v] + lane; e < wstart[v + 1]; e += 32) {
      const int64_t c = perf_cell[e];
#pragma unroll
      for (int u = 0; u < 3; ++u) acc = fma(awp[3 * e + u], x[3 * c + u], acc);
    }
    acc = warp_sum(acc);
    if (lane == 0) x[3 * N + v] = (b[3 * N + v] - acc) / aww[v];
  }
}

// The border's part of y = alpha A_b x + beta y once y's cell rows hold
// alpha A x + beta y: y_cells += alpha A_pw x_w, y_w = alpha (A_wp x + A_ww x_w) + beta y_w
__global__ void k_wl_border_product(int W, const int32_t* wstart, const int32_t* perf_cell, int64_t N,
                                    const double* apw, const double* awp, const double* aww, double alpha,
                                    const double* x, double beta, double* y) {
  wait_prior_grid();
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
  for (int v = warp; v < W; v += nw) {
    double acc = 0.0;
    const double xw = x[3 * N + v];
    for (int e = wstart[v] + lane; e < wstart[v + 1]; e += 32) {
      const int64_t c = perf_cell[e];
#pragma unroll
      for (int u = 0; u < 3; ++u) {
        acc = fma(awp[3 * e + u], x[3 * c + u], acc);
        y[3 * c + u] = fma(alpha * apw[3 * e + u], xw, y[3 * c + u]);
      }
    }
    acc = warp_sum(acc);
    if (lane == 0) {
      const double yw = beta == 0.0 ? 0.0 : beta * y[3 * N + v];
      y[3 * N + v] = fma(alpha, fma(aww[v], xw, acc), yw);
    }
  }
}

// u = U column v = A_pw[:, v] / A_ww[v] on the perforated rows (internal
// order; the rest of u is zero)
__global__ void k_wl_unit(int v, const int32_t* wstart, const int32_t* perf_t, int64_t N, const double* apw,
                          const double* aww, double* u) {
  wait_prior_grid();
  for (int e = wstart[v] + threadIdx.x; e < wstart[v + 1]; e += blockDim.x) {
    const int64_t t0 = perf_t[e];
#pragma unroll
    for (int r = 0; r < 3; ++r) u[r * N + t0] = apw[3 * e + r] / aww[v];
  }
}

// C = I - A_wp (M U): block u forms column u, one warp per row v
__global__ void k_wl_cmat(int W, const int32_t* wstart, const int32_t* perf_t, int64_t N, const double* awp,
                          const float* MU, double* C) {
  wait_prior_grid();
  const int u = blockIdx.x;
  const float* mu = MU + (size_t)u * 3 * N;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
  for (int v = warp; v < W; v += nw) {
    double acc = 0.0;
    for (int e = wstart[v] + lane; e < wstart[v + 1]; e += 32) {
      const int64_t t0 = perf_t[e];
#pragma unroll
      for (int r = 0; r < 3; ++r) acc = fma(awp[3 * e + r], (double)mu[r * N + t0], acc);
    }
    acc = warp_sum(acc);
    if (lane == 0) C[(size_t)v * W + u] = (v == u ? 1.0 : 0.0) - acc;
  }
}

// inverse of a small dense matrix by Gauss-Jordan elimination with partial
// pivoting (row-major, n x n); false if a pivot vanishes
bool invert_small(std::vector<double> a, int n, std::vector<double>& inv) {
  inv.assign((size_t)n * n, 0.0);
  for (int i = 0; i < n; ++i) inv[(size_t)i * n + i] = 1.0;
  for (int k = 0; k < n; ++k) {
    int p = k;
    for (int i = k + 1; i < n; ++i)
      if (std::fabs(a[(size_t)i * n + k]) > std::fabs(a[(size_t)p * n + k])) p = i;
    const double piv = a[(size_t)p * n + k];
    if (!(std::fabs(piv) > 0.0) || !std::isfinite(piv)) return false;
    if (p != k)
      for (int j = 0; j < n; ++j) {
        std::swap(a[(size_t)p * n + j], a[(size_t)k * n + j]);
        std::swap(inv[(size_t)p * n + j], inv[(size_t)k * n + j]);
      }
    const double d = 1.0 / piv;
    for (int j = 0; j < n; ++j) {
      a[(size_t)k * n + j] *= d;
      inv[(size_t)k * n + j] *= d;
    }
    for (int i = 0; i < n; ++i) {
      if (i == k) continue;
      const double f = a[(size_t)i * n + k];
      if (f == 0.0) continue;
      for (int j = 0; j < n; ++j) {
        a[(size_t)i * n + j] -= f * a[(size_t)k * n + j];
        inv[(size_t)i * n + j] -= f * inv[(size_t)k * n + j];
      }
    }
  }
  return true;
}

int status_of(cudaError_t e) {
  if (e == cudaSuccess) return BO_OK;
  if (e == cudaErrorMemoryAllocation) return BO_ERR_OOM;
  return BO_ERR_CUDA;
}

void wells_free(bo_wells* w) {
  cudaFree(w->wstart);
  cudaFree(w->perf_cell);
  cudaFree(w->perf_t);
  cudaFree(w->perf_well);
  cudaFree(w->apw);
  cudaFree(w->awp);
  cudaFree(w->aww);
  cudaFree(w->MU);
  cudaFree(w->Cinv);
  cudaFree(w->t);
  cudaFree(w->g);
  cudaFree(w->rfull);
  cudaFree(w->dx);
  cudaFree(w->partials);
  cudaFree(w->norms);
  cudaFreeHost(w->h_norms);
}

}  // namespace

// ------------------------------------------------------------ solver hooks
namespace bo {

// after the preconditioner wrote z (split planes of n entries)
void wells_after_prec(bo_prec* P, float* z, int64_t n) {
  bo_wells* wl = P->wl;
  cudaStream_t s = P->stream;
  const int64_t N = P->mat->g.N;
  (launch_pdl(k_wl_coeffs, 1, kThreads, 0, s, wl->W, wl->wstart, wl->perf_t, N, wl->awp, z, n, wl->Cinv, wl->aww,
                                      wl->coupling, wl->t, P->st),
   note_launch());
  if (wl->coupling)
    (launch_pdl(k_wl_woodbury, occ_grid((const void*)k_wl_woodbury, n), kThreads, 0, s, n, wl->W, wl->MU, wl->t, z, P->st),
     note_launch());
}

// after the Arnoldi product wrote w (split planes, low plane at w + np)
void wells_after_product(bo_prec* P, float* w, int64_t np) {
  bo_wells* wl = P->wl;
  if (wl->P == 0) return;
  (launch_pdl(k_wl_product, 1, kThreads, 0, P->stream, wl->P, wl->W, wl->perf_t, wl->perf_well, P->mat->g.N, wl->apw, wl->t,
      w, np, P->st),
   note_launch());
}

// after the true residual rk = bi - A xi and its norm: the Schur complement's
void wells_after_residual(bo_prec* P) {
  bo_wells* wl = P->wl;
  if (wl->P == 0) return;
  cudaStream_t s = P->stream;
  const int64_t N = P->mat->g.N;
  (launch_pdl(k_wl_residual, 1, kThreads, 0, s, wl->W, wl->wstart, wl->perf_t, N, wl->awp, wl->apw, wl->aww, P->xi, P->rk),
   note_launch());
  (launch_pdl(k_wl_beta, kRed, kThreads, 0, s, 3 * N, P->rk, P->partials, P->st), note_launch());
}

}  // namespace bo

namespace {

// M U and C^{-1} for preconditioner P (W applications of M); synchronises
int wells_prepare(bo_wells* wl, bo_prec* P) {
  cudaStream_t s = P->stream;
  const Geom& g = P->mat->g;
  const int64_t n = 3 * g.N;
  const int W = wl->W;
  double* u = P->rk;  // the solver's vectors are idle before a solve
  double* z = P->xi;
  for (int v = 0; v < W; ++v) {
    cudaMemsetAsync(u, 0, n * sizeof(double), s);
    (launch_pdl(k_wl_unit, 1, kThreads, 0, s, v, wl->wstart, wl->perf_t, g.N, wl->apw, wl->aww, u), note_launch());
    cudaMemsetAsync(&P->st->done, 0, sizeof(int), s);
    launch_cpr(P, u, z, BO_STAGE_CPR, P->st);
    launch_to_f32(z, wl->MU + (size_t)v * n, (size_t)n, s);
  }
  double* C = wl->rfull;  // scratch of W x W doubles (rfull holds 3N + W >= W^2)
  (launch_pdl(k_wl_cmat, W, kThreads, 0, s, W, wl->wstart, wl->perf_t, g.N, wl->awp, wl->MU, C), note_launch());
  std::vector<double> hc((size_t)W * W), hinv;
  int err = 0;
  cudaError_t e = cudaMemcpyAsync(hc.data(), C, hc.size() * sizeof(double), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(P->mat->h_flags, &P->st->err, sizeof(int), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return status_of(e);
  err = *P->mat->h_flags;
  if (err & kErrTimeout) return BO_ERR_TIMEOUT;
  if (err & (kErrNonfinite | kErrBreakdown)) return BO_ERR_BREAKDOWN;
  for (double c : hc)
    if (!std::isfinite(c)) return BO_ERR_NONFINITE;
  if (!invert_small(hc, W, hinv)) return BO_ERR_BREAKDOWN;
  e = cudaMemcpyAsync(wl->Cinv, hinv.data(), hinv.size() * sizeof(double), cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return status_of(e);
  wl->prep_prec = P;
  wl->prep_setups = P->setups;
  wl->prep_version = wl->version;
  return BO_OK;
}

// squared norm of v[0..n) into wl->norms[slot]
void sumsq(bo_wells* wl, const double* v, int64_t n, int slot, cudaStream_t s) {
  (launch_pdl(k_wl_sumsq, kRed, kThreads, 0, s, n, v, wl->partials), note_launch());
  (launch_pdl(k_wl_sumsq_finish, 1, kThreads, 0, s, kRed, wl->partials, wl->norms + slot), note_launch());
}

}  // namespace

extern "C" {

int bo_wells_create(bo_mat* A, int32_t nwells, int32_t nperf, const int32_t* perf_cell, const int32_t* perf_well,
                    bo_wells** out) {
  if (!A || !out || nwells < 1 || nwells > kMaxWells || nperf < 0 || nperf > (1 << 22)) return BO_ERR_ARG;
  if (nperf > 0 && (!perf_cell || !perf_well)) return BO_ERR_ARG;
  const Geom& g = A->g;
  // structure checks on the host: cells in range and perforated once, wells grouped
  std::vector<int32_t> wstart(nwells + 1, 0), pt(nperf);
  std::vector<char> seen((size_t)g.N, 0);
  for (int32_t e = 0; e < nperf; ++e) {
    const int64_t c = perf_cell[e];
    const int32_t v = perf_well[e];
    if (c < 0 || c >= g.N || v < 0 || v >= nwells) return BO_ERR_ARG;
    if (e > 0 && v < perf_well[e - 1]) return BO_ERR_ARG;
    if (seen[c]) return BO_ERR_ARG;
    seen[c] = 1;
    wstart[v + 1]++;
    const int64_t r = c / g.nx;
    const int i = (int)(c - r * g.nx), j = (int)(r % g.ny), k = (int)(r / g.ny);
    pt[e] = (int32_t)(((i + j + k) & 1) * g.Nh + (c >> 1));
  }
  for (int v = 0; v < nwells; ++v) wstart[v + 1] += wstart[v];
  if (cudaSetDevice(A->ctx->device) != cudaSuccess) return BO_ERR_CUDA;
  bo_wells* w = new (std::nothrow) bo_wells();
  if (!w) return BO_ERR_OOM;
  w->mat = A;
  w->W = nwells;
  w->P = nperf;
  w->coupling = 1;
  const int64_t n = 3 * g.N;
  const size_t pe = (size_t)(nperf > 0 ? nperf : 1);
  cudaError_t e = cudaSuccess;
  auto dev = [&](void** p, size_t bytes) {
    if (e == cudaSuccess) e = cudaMalloc(p, bytes);
  };
  dev((void**)&w->wstart, (nwells + 1) * sizeof(int32_t));
  dev((void**)&w->perf_cell, pe * sizeof(int32_t));
  dev((void**)&w->perf_t, pe * sizeof(int32_t));
  dev((void**)&w->perf_well, pe * sizeof(int32_t));
  dev((void**)&w->apw, 3 * pe * sizeof(double));
  dev((void**)&w->awp, 3 * pe * sizeof(double));
  dev((void**)&w->aww, nwells * sizeof(double));
  dev((void**)&w->MU, (size_t)nwells * n * sizeof(float));
  dev((void**)&w->Cinv, (size_t)nwells * nwells * sizeof(double));
  dev((void**)&w->t, 2 * nwells * sizeof(double));
  dev((void**)&w->g, n * sizeof(double));
  dev((void**)&w->rfull, (size_t)(n + nwells > (int64_t)nwells * nwells ? n + nwells : (int64_t)nwells * nwells) *
                             sizeof(double));
  dev((void**)&w->dx, (n + nwells) * sizeof(double));
  dev((void**)&w->partials, kRed * sizeof(double));
  dev((void**)&w->norms, 4 * sizeof(double));
  if (e == cudaSuccess) e = cudaMallocHost((void**)&w->h_norms, 4 * sizeof(double));
  cudaStream_t s = A->ctx->stream;
  if (e == cudaSuccess) e = cudaMemcpyAsync(w->wstart, wstart.data(), wstart.size() * 4, cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess && nperf > 0) {
    e = cudaMemcpyAsync(w->perf_cell, perf_cell, nperf * 4, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(w->perf_t, pt.data(), nperf * 4, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(w->perf_well, perf_well, nperf * 4, cudaMemcpyHostToDevice, s);
  }
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) {
    wells_free(w);
    delete w;
    return status_of(e);
  }
  A->refs++;
  *out = w;
  return BO_OK;
}

int bo_wells_update_values(bo_wells* w, const double* apw, const double* awp, const double* aww, int mem) {
  if (!w || !aww || (w->P > 0 && (!apw || !awp))) return BO_ERR_ARG;
  if (mem != BO_MEM_HOST && mem != BO_MEM_DEVICE) return BO_ERR_ARG;
  if (cudaSetDevice(w->mat->ctx->device) != cudaSuccess) return BO_ERR_CUDA;
  // the border is small: checked on the host, then stored on the device
  const size_t p3 = 3 * (size_t)w->P;
  std::vector<double> h(2 * p3 + w->W);
  const cudaMemcpyKind k = mem == BO_MEM_HOST ? cudaMemcpyHostToHost : cudaMemcpyDeviceToHost;
  cudaError_t e = cudaSuccess;
  if (p3) e = cudaMemcpy(h.data(), apw, p3 * sizeof(double), k);
  if (e == cudaSuccess && p3) e = cudaMemcpy(h.data() + p3, awp, p3 * sizeof(double), k);
  if (e == cudaSuccess) e = cudaMemcpy(h.data() + 2 * p3, aww, w->W * sizeof(double), k);
  if (e != cudaSuccess) return status_of(e);
  for (double v : h)
    if (!std::isfinite(v)) return BO_ERR_NONFINITE;
  for (int v = 0; v < w->W; ++v)
    if (h[2 * p3 + v] == 0.0) return BO_ERR_BREAKDOWN;  // a constraint that does not involve its p_h
  cudaStream_t s = w->mat->ctx->stream;
  if (p3) e = cudaMemcpyAsync(w->apw, h.data(), p3 * sizeof(double), cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess && p3) e = cudaMemcpyAsync(w->awp, h.data() + p3, p3 * sizeof(double), cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(w->aww, h.data() + 2 * p3, w->W * sizeof(double), cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return status_of(e);
  w->values_set = true;
  w->version++;
  return BO_OK;
}

int bo_wells_set_coupling(bo_wells* w, int mode) {
  if (!w || (mode != 0 && mode != 1)) return BO_ERR_ARG;
  w->coupling = mode;
  w->prep_prec = nullptr;
  return BO_OK;
}

int bo_wells_spmv(bo_wells* w, double alpha, const double* x, double beta, double* y) {
  if (!w || !x || !y || !w->values_set) return BO_ERR_ARG;
  bo_mat* m = w->mat;
  if (cudaSetDevice(m->ctx->device) != cudaSuccess) return BO_ERR_CUDA;
  launch_spmv_nat(m, alpha, x, beta, y, BO_PREC_FP64);
  (launch_pdl(k_wl_border_product, 1, kThreads, 0, m->ctx->stream, w->W, w->wstart, w->perf_cell, m->g.N, w->apw, w->awp,
      w->aww, alpha, x, beta, y),
   note_launch());
  return status_of(cudaStreamSynchronize(m->ctx->stream));
}

int bo_solve_bordered(bo_prec* P, bo_wells* w, const double* b, double* x, const bo_solve_opts* opts,
                      bo_solve_info* info) {
  if (!P || !w || !b || !x || w->mat != P->mat || !w->values_set) return BO_ERR_ARG;
  bo_solve_opts o;
  bo_solve_opts_default(&o);
  if (opts) o = *opts;
  if (!(o.tol > 0.0) || o.restart < 1 || o.restart > 64 || o.maxit < 0 || o.mem != BO_MEM_DEVICE) return BO_ERR_ARG;
  bo_mat* m = P->mat;
  if (cudaSetDevice(m->ctx->device) != cudaSuccess) return BO_ERR_CUDA;
  if (P->stream != m->ctx->stream) return BO_ERR_ARG;
  cudaStream_t s = P->stream;
  const int64_t N = m->g.N, n = 3 * N, nf = n + w->W;
  int rc = BO_OK;
  if (w->coupling && (w->prep_prec != P || w->prep_setups != P->setups || w->prep_version != w->version)) {
    rc = wells_prepare(w, P);
    if (rc != BO_OK) return rc;
  }
  // the system solved: A_b d = rb with rb = b (zero guess) or b - A_b x0
  const double* rb = b;
  double* d = x;
  if (!o.x0_is_zero) {
    cudaMemcpyAsync(w->rfull, b, nf * sizeof(double), cudaMemcpyDeviceToDevice, s);
    launch_spmv_nat(m, -1.0, x, 1.0, w->rfull, BO_PREC_FP64);
    (launch_pdl(k_wl_border_product, 1, kThreads, 0, s, w->W, w->wstart, w->perf_cell, N, w->apw, w->awp, w->aww, -1.0, x,
        1.0, w->rfull),
     note_launch());
    rb = w->rfull;
    d = w->dx;
  }
  cudaMemcpyAsync(w->g, rb, n * sizeof(double), cudaMemcpyDeviceToDevice, s);
  if (w->P > 0)
    (launch_pdl(k_wl_rhs, 1, kThreads, 0, s, w->P, N, w->perf_cell, w->perf_well, w->apw, w->aww, rb, w->g), note_launch());
  sumsq(w, b, nf, 0, s);
  sumsq(w, w->g, n, 1, s);
  cudaError_t e = cudaMemcpyAsync(w->h_norms, w->norms, 2 * sizeof(double), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return status_of(e);
  const double bnorm = std::sqrt(w->h_norms[0]), gnorm = std::sqrt(w->h_norms[1]);
  if (!std::isfinite(bnorm) || !std::isfinite(gnorm)) return BO_ERR_NONFINITE;
  bo_solve_info inf;
  std::memset(&inf, 0, sizeof(inf));
  if (bnorm == 0.0) {
    cudaMemsetAsync(x, 0, nf * sizeof(double), s);
    rc = status_of(cudaStreamSynchronize(s));
    if (info) *info = inf;
    return rc;
  }
  if (gnorm == 0.0) {
    cudaMemsetAsync(d, 0, n * sizeof(double), s);
  } else {
    bo_solve_opts o2 = o;
    o2.tol = o.tol * bnorm / gnorm;  // ||g - S d|| <= tol ||b||
    o2.x0_is_zero = 1;
    P->wl = w;
    rc = fgmres(P, w->g, d, &o2, &inf);
    P->wl = nullptr;
    if (rc != BO_OK && rc != BO_ERR_NOT_CONVERGED) {
      if (info) *info = inf;
      return rc;
    }
    // reported relative to ||b|| of the bordered system
    inf.true_rel_res *= gnorm / bnorm;
    inf.est_rel_res *= gnorm / bnorm;
    for (int i = 0; i < P->nhist; ++i) P->hist[i] *= gnorm / bnorm;
  }
  (launch_pdl(k_wl_recover, 1, kThreads, 0, s, w->W, w->wstart, w->perf_cell, N, w->awp, w->aww, rb, d), note_launch());
  if (!o.x0_is_zero) launch_newton_update(x, w->dx, nf, s);
  e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return status_of(e);
  if (info) *info = inf;
  return rc;
}

int bo_wells_destroy(bo_wells* w) {
  if (!w) return BO_ERR_ARG;
  cudaSetDevice(w->mat->ctx->device);
  cudaStreamSynchronize(w->mat->ctx->stream);
  wells_free(w);
  bo_mat* m = w->mat;
  delete w;
  bo::mat_release_ref(m);
  return BO_OK;
}

}  // extern "C"
