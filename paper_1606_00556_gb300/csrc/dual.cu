// Dual-porosity systems (paper Sec. 2.1's dual-porosity model): every cell
// has a fracture node (7-point flow among fracture nodes, wells) and a
// matrix node coupled only to its own fracture node.  In block form, with F
// the fracture and M the matrix unknowns,
//   [A_ff  A_fm] [x_f]   [b_f]
//   [A_mf  A_mm] [x_m] = [b_m],   A_fm, A_mf, A_mm block diagonal (3x3 per cell).
// The matrix unknowns are eliminated exactly, cell by cell:
//   S = A_ff - A_fm A_mm^{-1} A_mf   (7-point: only the diagonal blocks change),
//   S x_f = b_f - A_fm A_mm^{-1} b_m,   x_m = A_mm^{-1} (b_m - A_mf x_f),
// so the fracture system goes through the single-porosity CPR-FGMRES path
// unchanged.  Because x_m is recovered exactly, the full system's residual
// equals S's residual in the fracture rows and vanishes in the matrix rows;
// the solve asks S for tol ||b|| / ||b_hat|| and then checks the full
// system's FP64 residual itself, refining if rounding left it short.
//
// Input: a BSR matrix of 2N block rows, row c < N the fracture node of cell
// c (its 7-point fracture neighbours and column N + c), row N + c the
// matrix node (columns c and N + c); vectors of 6N doubles, the fracture
// nodes' (p, Sw, Sg) first.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <new>
#include <vector>

#include "bo_internal.cuh"

struct bo_dp {
  bo_ctx* ctx;
  bo_mat* S;            // condensed fracture system (owned)
  bo::Geom g;
  int64_t N, nnzb;
  int32_t* rowptr;      // device copy of the full pattern (2N + 1)
  int32_t* col;
  double* val;          // device copy of the full values (9 nnzb)
  int32_t* fmap;        // per cell: positions of the 7 slot blocks (-1: none), then of A_fm
  int32_t* mmap;        // per cell: positions of A_mf and A_mm
  double* minv;         // A_mm^{-1}, 9 per cell
  double* bhat;         // condensed right-hand side (3N)
  double* r;            // full residual / correction right-hand side (6N)
  double* dx;           // correction (6N)
  double* part;         // reduction partials
  double* norms;        // device: ||b||^2, ||b_hat||^2, ||r||^2
  double* h_norms;      // pinned mirror
  int* flags;
  int* h_flags;
};

namespace bo {
namespace {

constexpr int kRedGrid = 1024;

__device__ bool inv3d(const double a[9], double out[9]) {
  double m[3][6];
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) {
      m[i][j] = a[3 * i + j];
      m[i][3 + j] = (i == j) ? 1.0 : 0.0;
    }
  for (int k = 0; k < 3; ++k) {
    int p = k;
    for (int i = k + 1; i < 3; ++i)
      if (fabs(m[i][k]) > fabs(m[p][k])) p = i;
    if (m[p][k] == 0.0) return false;
    if (p != k)
      for (int j = 0; j < 6; ++j) { const double t = m[k][j]; m[k][j] = m[p][j]; m[p][j] = t; }
    const double rp = 1.0 / m[k][k];  // one FP64 division per pivot
    for (int j = 0; j < 6; ++j) m[k][j] *= rp;
    for (int i = 0; i < 3; ++i) {
      if (i == k) continue;
      const double f = m[i][k];
      for (int j = 0; j < 6; ++j) m[i][j] -= f * m[k][j];
    }
  }
  bool ok = true;
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) {
      out[3 * i + j] = m[i][3 + j];
      ok = ok && isfinite(out[3 * i + j]);
    }
  return ok;
}

__device__ __forceinline__ void mm3(const double a[9], const double b[9], double c[9]) {
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j) c[3 * i + j] = a[3 * i] * b[j] + a[3 * i + 1] * b[3 + j] + a[3 * i + 2] * b[6 + j];
}

__device__ __forceinline__ void mv3(const double a[9], const double x[3], double y[3]) {
#pragma unroll
  for (int i = 0; i < 3; ++i) y[i] = a[3 * i] * x[0] + a[3 * i + 1] * x[1] + a[3 * i + 2] * x[2];
}

// S's colour-split planes and A_mm^{-1} from the full values
__global__ void k_dp_condense(Geom g, const double* __restrict__ val, const int32_t* __restrict__ fmap,
                              const int32_t* __restrict__ mmap, double* __restrict__ A, double* __restrict__ minv,
                              int* flags) {
  wait_prior_grid();
  for (int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; c < g.N; c += (int64_t)gridDim.x * blockDim.x) {
    const int i = (int)(c % g.nx), j = (int)((c / g.nx) % g.ny), k = (int)(c / ((int64_t)g.nx * g.ny));
    const int color = (i + j + k) & 1;
    const int64_t q = c >> 1;
    double M[9], Mi[9], Af[9], Am[9], T1[9], T[9];
    const int64_t pmf = mmap[2 * c], pmm = mmap[2 * c + 1], pfm = fmap[8 * c + 7];
    bool fin = true;
    for (int e = 0; e < 9; ++e) {
      M[e] = val[9 * pmm + e];
      Af[e] = val[9 * pfm + e];
      Am[e] = val[9 * pmf + e];
      fin = fin && isfinite(M[e]) && isfinite(Af[e]) && isfinite(Am[e]);
    }
    if (!fin) atomicOr(flags, kErrNonfinite);
    if (!inv3d(M, Mi)) {
      atomicOr(flags, kErrBreakdown);
      for (int e = 0; e < 9; ++e) Mi[e] = 0.0;
    }
    mm3(Af, Mi, T1);
    mm3(T1, Am, T);
    for (int e = 0; e < 9; ++e) minv[9 * c + e] = Mi[e];
    for (int s = 0; s < 7; ++s) {
      const int64_t p = fmap[8 * c + s];
      for (int rc = 0; rc < 9; ++rc) {
        double v = p >= 0 ? val[9 * p + rc] : 0.0;
        if (s == kDiag) v -= T[rc];
        if (p >= 0 && !isfinite(val[9 * p + rc])) atomicOr(flags, kErrNonfinite);
        A[plane(g, color, s, rc) + q] = v;
      }
    }
  }
}

// b_hat = b_f - A_fm A_mm^{-1} b_m
__global__ void k_dp_rhs(int64_t N, const double* __restrict__ val, const int32_t* __restrict__ fmap,
                         const double* __restrict__ minv, const double* __restrict__ b, double* __restrict__ bhat) {
  wait_prior_grid();
  for (int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; c < N; c += (int64_t)gridDim.x * blockDim.x) {
    double Mi[9], Af[9], bm[3], t[3], u[3];
    for (int e = 0; e < 9; ++e) {
      Mi[e] = minv[9 * c + e];
      Af[e] = val[9 * (int64_t)fmap[8 * c + 7] + e];
    }
    for (int r = 0; r < 3; ++r) bm[r] = b[3 * (N + c) + r];
    mv3(Mi, bm, t);
    mv3(Af, t, u);
    for (int r = 0; r < 3; ++r) bhat[3 * c + r] = b[3 * c + r] - u[r];
  }
}

// x_m = A_mm^{-1} (b_m - A_mf x_f)
__global__ void k_dp_recover(int64_t N, const double* __restrict__ val, const int32_t* __restrict__ mmap,
                             const double* __restrict__ minv, const double* __restrict__ b, double* __restrict__ x) {
  wait_prior_grid();
  for (int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; c < N; c += (int64_t)gridDim.x * blockDim.x) {
    double Mi[9], Am[9], xf[3], t[3], y[3];
    for (int e = 0; e < 9; ++e) {
      Mi[e] = minv[9 * c + e];
      Am[e] = val[9 * (int64_t)mmap[2 * c] + e];
    }
    for (int r = 0; r < 3; ++r) xf[r] = x[3 * c + r];
    mv3(Am, xf, t);
    for (int r = 0; r < 3; ++r) t[r] = b[3 * (N + c) + r] - t[r];
    mv3(Mi, t, y);
    for (int r = 0; r < 3; ++r) x[3 * (N + c) + r] = y[r];
  }
}

// r = b - A x over the full 2N-row BSR (FP64), one block row per thread
__global__ void k_dp_residual(int64_t nb, const int32_t* __restrict__ rowptr, const int32_t* __restrict__ col,
                              const double* __restrict__ val, const double* __restrict__ b,
                              const double* __restrict__ x, double* __restrict__ r) {
  wait_prior_grid();
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < nb; i += (int64_t)gridDim.x * blockDim.x) {
    double s[3] = {b[3 * i], b[3 * i + 1], b[3 * i + 2]};
    for (int32_t e = rowptr[i]; e < rowptr[i + 1]; ++e) {
      const int64_t cj = col[e];
      const double x0 = x[3 * cj], x1 = x[3 * cj + 1], x2 = x[3 * cj + 2];
      const double* a = val + 9 * (int64_t)e;
      for (int rr = 0; rr < 3; ++rr) s[rr] -= a[3 * rr] * x0 + a[3 * rr + 1] * x1 + a[3 * rr + 2] * x2;
    }
    r[3 * i] = s[0];
    r[3 * i + 1] = s[1];
    r[3 * i + 2] = s[2];
  }
}

// fixed-order sum of squares: per-block partials, then one block sums them
__global__ void k_sq_partials(const double* __restrict__ x, int64_t n, double* __restrict__ part) {
  wait_prior_grid();
  __shared__ double sh[32];
  double s = 0.0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    s += x[i] * x[i];
  s = block_sum(s, sh);
  if (threadIdx.x == 0) part[blockIdx.x] = s;
}

__global__ void k_sum_final(const double* __restrict__ part, int nb, double* __restrict__ out) {
  wait_prior_grid();
  __shared__ double sh[32];
  double s = 0.0;
  for (int i = threadIdx.x; i < nb; i += blockDim.x) s += part[i];
  s = block_sum(s, sh);
  if (threadIdx.x == 0) *out = s;
}

__global__ void k_add(int64_t n, double* __restrict__ x, const double* __restrict__ dx) {
  wait_prior_grid();
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    x[i] += dx[i];
}

void sq_norm(const double* x, int64_t n, double* part, double* out, cudaStream_t s) {
  const int gb = grid_for(n, kThreads, kRedGrid);
  (launch_pdl(k_sq_partials, gb, kThreads, 0, s, x, n, part), note_launch());
  (launch_pdl(k_sum_final, 1, kThreads, 0, s, part, gb, out), note_launch());
}

void dp_free(bo_dp* d) {
  auto fr = [](void* p) { if (p) cudaFree(p); };
  fr(d->rowptr); fr(d->col); fr(d->val); fr(d->fmap); fr(d->mmap); fr(d->minv); fr(d->bhat); fr(d->r);
  fr(d->dx); fr(d->part); fr(d->norms); fr(d->flags);
  if (d->h_norms) cudaFreeHost(d->h_norms);
  if (d->h_flags) cudaFreeHost(d->h_flags);
  if (d->S) bo_mat_destroy(d->S);
}

// values -> S planes, A_mm^{-1}; reads the error bits back
int dp_condense(bo_dp* d) {
  cudaStream_t s = d->ctx->stream;
  cudaMemsetAsync(d->flags, 0, sizeof(int), s);
  (launch_pdl(k_dp_condense, grid_for(d->N), kThreads, 0, s, d->g, d->val, d->fmap, d->mmap, d->S->A, d->minv, d->flags),
   note_launch());
  d->S->a32_valid = false;
  d->S->a16_valid = false;
  launch_split_matrix(d->S, s);
  cudaMemcpyAsync(d->h_flags, d->flags, sizeof(int), cudaMemcpyDeviceToHost, s);
  if (cudaStreamSynchronize(s) != cudaSuccess) return BO_ERR_CUDA;
  if (*d->h_flags & kErrNonfinite) return BO_ERR_NONFINITE;
  if (*d->h_flags & kErrBreakdown) return BO_ERR_BREAKDOWN;
  return BO_OK;
}

}  // namespace
}  // namespace bo

extern "C" {

int bo_dp_create(bo_ctx* ctx, const bo_grid* grid, int32_t nbrows, int64_t nnzb, const int32_t* rowptr,
                 const int32_t* col, const double* val, int mem, bo_dp** out) {
  if (!ctx || !grid || !rowptr || !col || !val || !out || grid->ncontinua != 2) return BO_ERR_ARG;
  if (mem != BO_MEM_HOST && mem != BO_MEM_DEVICE) return BO_ERR_ARG;
  if (grid->nx < 2 || (grid->nx % 2) != 0 || grid->ny < 1 || grid->nz < 1) return BO_ERR_ARG;
  const int64_t nx = grid->nx, ny = grid->ny, nz = grid->nz, N = nx * ny * nz;
  if (N > ((int64_t)1 << 27) || nbrows != 2 * N || nnzb <= 0 || nnzb > INT32_MAX) return BO_ERR_ARG;
  if (cudaSetDevice(ctx->device) != cudaSuccess) return BO_ERR_CUDA;
  // the pattern on the host (copied back if it lives on the device)
  std::vector<int32_t> hrp(2 * N + 1), hcol(nnzb);
  const cudaMemcpyKind kd = mem == BO_MEM_HOST ? cudaMemcpyHostToHost : cudaMemcpyDeviceToHost;
  if (cudaMemcpy(hrp.data(), rowptr, hrp.size() * sizeof(int32_t), kd) != cudaSuccess ||
      cudaMemcpy(hcol.data(), col, hcol.size() * sizeof(int32_t), kd) != cudaSuccess)
    return BO_ERR_CUDA;
  if (hrp[0] != 0 || hrp[2 * N] != nnzb) return BO_ERR_PATTERN;
  for (int64_t r = 0; r < 2 * N; ++r)
    if (hrp[r + 1] < hrp[r]) return BO_ERR_PATTERN;
  // position maps; every expected block exactly once and nothing else
  std::vector<int32_t> fmap(8 * N, -1), mmap(2 * N, -1);
  std::vector<int32_t> rp7(N + 1, 0), col7;
  col7.reserve(7 * N);
  for (int64_t c = 0; c < N; ++c) {
    const int64_t i = c % nx, j = (c / nx) % ny, k = c / (nx * ny);
    const int64_t nb7[7] = {k > 0 ? c - nx * ny : -1, j > 0 ? c - nx : -1, i > 0 ? c - 1 : -1, c,
                            i < nx - 1 ? c + 1 : -1, j < ny - 1 ? c + nx : -1, k < nz - 1 ? c + nx * ny : -1};
    int expect = 1;
    for (int s = 0; s < 7; ++s) expect += nb7[s] >= 0;
    if (hrp[c + 1] - hrp[c] != expect) return BO_ERR_PATTERN;
    for (int32_t e = hrp[c]; e < hrp[c + 1]; ++e) {
      const int64_t cj = hcol[e];
      int slot = -1;
      for (int s = 0; s < 7; ++s)
        if (nb7[s] == cj) slot = s;
      if (slot >= 0) {
        if (fmap[8 * c + slot] >= 0) return BO_ERR_PATTERN;
        fmap[8 * c + slot] = e;
      } else if (cj == N + c) {
        if (fmap[8 * c + 7] >= 0) return BO_ERR_PATTERN;
        fmap[8 * c + 7] = e;
      } else {
        return BO_ERR_PATTERN;
      }
    }
    for (int s = 0; s < 7; ++s)
      if (nb7[s] >= 0) col7.push_back((int32_t)nb7[s]);
    rp7[c + 1] = (int32_t)col7.size();
    const int64_t r = N + c;
    if (hrp[r + 1] - hrp[r] != 2) return BO_ERR_PATTERN;
    for (int32_t e = hrp[r]; e < hrp[r + 1]; ++e) {
      if (hcol[e] == c && mmap[2 * c] < 0) mmap[2 * c] = e;
      else if (hcol[e] == N + c && mmap[2 * c + 1] < 0) mmap[2 * c + 1] = e;
      else return BO_ERR_PATTERN;
    }
  }
  bo_dp* d = new (std::nothrow) bo_dp();
  if (!d) return BO_ERR_OOM;
  std::memset(d, 0, sizeof(*d));
  d->ctx = ctx;
  d->N = N;
  d->nnzb = nnzb;
  d->g = bo::Geom{grid->nx, grid->ny, grid->nz, grid->nx / 2, N, N / 2};
  // the condensed system's matrix object, created on the 7-point pattern
  bo_grid g1 = *grid;
  g1.ncontinua = 1;
  {
    std::vector<double> zeros((size_t)9 * col7.size(), 0.0);
    int rc = bo_mat_create_bsr(ctx, &g1, (int32_t)N, (int64_t)col7.size(), rp7.data(), col7.data(), zeros.data(),
                               BO_MEM_HOST, &d->S);
    if (rc != BO_OK) {
      delete d;
      return rc;
    }
  }
  bool ok = true;
  auto al = [&](void** p, size_t bytes) {
    if (ok && cudaMalloc(p, bytes) != cudaSuccess) ok = false;
  };
  al((void**)&d->rowptr, (2 * N + 1) * sizeof(int32_t));
  al((void**)&d->col, nnzb * sizeof(int32_t));
  al((void**)&d->val, (size_t)9 * nnzb * sizeof(double));
  al((void**)&d->fmap, 8 * N * sizeof(int32_t));
  al((void**)&d->mmap, 2 * N * sizeof(int32_t));
  al((void**)&d->minv, 9 * N * sizeof(double));
  al((void**)&d->bhat, 3 * N * sizeof(double));
  al((void**)&d->r, 6 * N * sizeof(double));
  al((void**)&d->dx, 6 * N * sizeof(double));
  al((void**)&d->part, bo::kRedGrid * sizeof(double));
  al((void**)&d->norms, 4 * sizeof(double));
  al((void**)&d->flags, sizeof(int));
  if (ok && cudaMallocHost((void**)&d->h_norms, 4 * sizeof(double)) != cudaSuccess) ok = false;
  if (ok && cudaMallocHost((void**)&d->h_flags, sizeof(int)) != cudaSuccess) ok = false;
  if (!ok) {
    bo::dp_free(d);
    delete d;
    return BO_ERR_OOM;
  }
  ctx->refs++;
  cudaStream_t s = ctx->stream;
  cudaMemcpyAsync(d->rowptr, hrp.data(), hrp.size() * sizeof(int32_t), cudaMemcpyHostToDevice, s);
  cudaMemcpyAsync(d->col, hcol.data(), hcol.size() * sizeof(int32_t), cudaMemcpyHostToDevice, s);
  cudaMemcpyAsync(d->fmap, fmap.data(), fmap.size() * sizeof(int32_t), cudaMemcpyHostToDevice, s);
  cudaMemcpyAsync(d->mmap, mmap.data(), mmap.size() * sizeof(int32_t), cudaMemcpyHostToDevice, s);
  int rc = bo_dp_update_values(d, val, mem);
  if (rc != BO_OK) {
    bo_dp_destroy(d);
    return rc;
  }
  *out = d;
  return BO_OK;
}

int bo_dp_update_values(bo_dp* d, const double* val, int mem) {
  if (!d || !val || (mem != BO_MEM_HOST && mem != BO_MEM_DEVICE)) return BO_ERR_ARG;
  if (cudaSetDevice(d->ctx->device) != cudaSuccess) return BO_ERR_CUDA;
  const cudaMemcpyKind kd = mem == BO_MEM_HOST ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice;
  if (cudaMemcpyAsync(d->val, val, (size_t)9 * d->nnzb * sizeof(double), kd, d->ctx->stream) != cudaSuccess)
    return BO_ERR_CUDA;
  return bo::dp_condense(d);
}

bo_mat* bo_dp_fracture_matrix(bo_dp* d) { return d ? d->S : nullptr; }

int bo_dp_solve(bo_dp* d, bo_prec* P, const double* b, double* x, const bo_solve_opts* opts, bo_solve_info* info) {
  if (!d || !P || !b || !x || !opts) return BO_ERR_ARG;
  if (P->mat != d->S) return BO_ERR_ARG;
  if (cudaSetDevice(d->ctx->device) != cudaSuccess) return BO_ERR_CUDA;
  cudaStream_t s = d->ctx->stream;
  const int64_t N = d->N;
  const int gN = bo::grid_for(N);
  bo_solve_info acc;
  std::memset(&acc, 0, sizeof(acc));
  // ||b||
  bo::sq_norm(b, 6 * N, d->part, d->norms, s);
  const double* rhs = b;   // right-hand side of the current pass
  double* xs = x;          // where the current pass writes its solution
  int rc = BO_OK;
  const int kPasses = 3;   // the solve plus up to two refinement passes
  for (int pass = 0; pass < kPasses; ++pass) {
    (bo::launch_pdl(bo::k_dp_rhs, gN, bo::kThreads, 0, s, N, d->val, d->fmap, d->minv, rhs, d->bhat), bo::note_launch());
    bo::sq_norm(d->bhat, 3 * N, d->part, d->norms + 1, s);
    cudaMemcpyAsync(d->h_norms, d->norms, 2 * sizeof(double), cudaMemcpyDeviceToHost, s);
    if (cudaStreamSynchronize(s) != cudaSuccess) return BO_ERR_CUDA;
    const double nb = std::sqrt(d->h_norms[0]), nbh = std::sqrt(d->h_norms[1]);
    bo_solve_opts o = *opts;
    o.mem = BO_MEM_DEVICE;
    if (pass > 0) o.x0_is_zero = 1;
    if (!(nbh > 0.0)) {  // nothing to solve for the fracture unknowns
      cudaMemsetAsync(xs, 0, 3 * N * sizeof(double), s);
    } else {
      // S's residual equals the full residual: ask for tol ||b|| relative to ||b_hat||
      o.tol = opts->tol * std::sqrt(d->h_norms[0]) / nbh;
      if (pass > 0) o.tol = std::min(0.5, o.tol);
      bo_solve_info si;
      rc = bo_solve(P, d->bhat, xs, &o, &si);
      acc.iters += si.iters;
      acc.restarts += si.restarts;
      acc.solve_ms += si.solve_ms;
      acc.spmv_launches += si.spmv_launches;
      acc.spmv_ms += si.spmv_ms;
      acc.est_rel_res = si.est_rel_res;
      if (rc != BO_OK && rc != BO_ERR_NOT_CONVERGED) return rc;
    }
    (bo::launch_pdl(bo::k_dp_recover, gN, bo::kThreads, 0, s, N, d->val, d->mmap, d->minv, rhs, xs), bo::note_launch());
    if (pass > 0) (bo::launch_pdl(bo::k_add, bo::grid_for(6 * N), bo::kThreads, 0, s, 6 * N, x, xs), bo::note_launch());
    // the full system's FP64 residual
    (bo::launch_pdl(bo::k_dp_residual, bo::grid_for(2 * N), bo::kThreads, 0, s, 2 * N, d->rowptr, d->col, d->val, b, x, d->r),
     bo::note_launch());
    bo::sq_norm(d->r, 6 * N, d->part, d->norms + 2, s);
    cudaMemcpyAsync(d->h_norms + 2, d->norms + 2, sizeof(double), cudaMemcpyDeviceToHost, s);
    if (cudaStreamSynchronize(s) != cudaSuccess) return BO_ERR_CUDA;
    const double rel = nb > 0 ? std::sqrt(d->h_norms[2]) / nb : std::sqrt(d->h_norms[2]);
    acc.true_rel_res = rel;
    if (rel <= opts->tol || !(rel == rel)) break;
    // refine: solve A dx = r and add it
    rhs = d->r;
    xs = d->dx;
  }
  acc.status = acc.true_rel_res <= opts->tol ? BO_OK : BO_ERR_NOT_CONVERGED;
  if (info) *info = acc;
  return acc.status;
}

int bo_dp_solve_batched(bo_dp* const* dps, bo_prec* const* P, int nreal, const double* const* b, double* const* x,
                        const bo_solve_opts* opts, bo_solve_info* infos) {
  if (!dps || !P || !b || !x || !opts || nreal < 1) return BO_ERR_ARG;
  if (!(opts->tol > 0.0) || opts->restart < 1 || opts->restart > 64 || opts->maxit < 0) return BO_ERR_ARG;
  const int dev = dps[0] ? dps[0]->ctx->device : -1;
  for (int r = 0; r < nreal; ++r) {
    if (!dps[r] || !P[r] || !b[r] || !x[r] || P[r]->mat != dps[r]->S || dps[r]->ctx->device != dev) return BO_ERR_ARG;
    for (int q = 0; q < r; ++q)
      if (P[q] == P[r] || dps[q] == dps[r]) return BO_ERR_ARG;
  }
  if (cudaSetDevice(dev) != cudaSuccess) return BO_ERR_CUDA;
  // condensed right-hand sides and the norms that set each fracture solve's
  // tolerance (as in bo_dp_solve's first pass)
  for (int r = 0; r < nreal; ++r) {
    bo_dp* d = dps[r];
    cudaStream_t s = d->ctx->stream;
    bo::sq_norm(b[r], 6 * d->N, d->part, d->norms, s);
    (bo::launch_pdl(bo::k_dp_rhs, bo::grid_for(d->N), bo::kThreads, 0, s, d->N, d->val, d->fmap, d->minv, b[r], d->bhat),
     bo::note_launch());
    bo::sq_norm(d->bhat, 3 * d->N, d->part, d->norms + 1, s);
    cudaMemcpyAsync(d->h_norms, d->norms, 2 * sizeof(double), cudaMemcpyDeviceToHost, s);
  }
  std::vector<const double*> bh(nreal);
  std::vector<double*> xs(nreal);
  std::vector<double> tols(nreal);
  std::vector<int> zero(nreal, 0);
  for (int r = 0; r < nreal; ++r) {
    bo_dp* d = dps[r];
    if (cudaStreamSynchronize(d->ctx->stream) != cudaSuccess) return BO_ERR_CUDA;
    const double nb = std::sqrt(d->h_norms[0]), nbh = std::sqrt(d->h_norms[1]);
    bh[r] = d->bhat;
    xs[r] = x[r];  // the fracture unknowns come first in x
    tols[r] = nbh > 0.0 ? opts->tol * nb / nbh : opts->tol;
    zero[r] = !(nbh > 0.0);
  }
  bo_solve_opts o = *opts;
  o.mem = BO_MEM_DEVICE;
  std::vector<bo_solve_info> si(nreal);
  int rc = bo::solve_batched(P, nreal, bh.data(), xs.data(), o, si.data(), tols.data());
  if (rc != BO_OK && rc != BO_ERR_NOT_CONVERGED) return rc;
  // matrix unknowns and the full FP64 residual of every system
  for (int r = 0; r < nreal; ++r) {
    bo_dp* d = dps[r];
    cudaStream_t s = d->ctx->stream;
    if (zero[r]) cudaMemsetAsync(x[r], 0, 3 * d->N * sizeof(double), s);
    (bo::launch_pdl(bo::k_dp_recover, bo::grid_for(d->N), bo::kThreads, 0, s, d->N, d->val, d->mmap, d->minv, b[r], x[r]),
     bo::note_launch());
    (bo::launch_pdl(bo::k_dp_residual, bo::grid_for(2 * d->N), bo::kThreads, 0, s, 2 * d->N, d->rowptr, d->col, d->val, b[r],
        x[r], d->r),
     bo::note_launch());
    bo::sq_norm(d->r, 6 * d->N, d->part, d->norms + 2, s);
    cudaMemcpyAsync(d->h_norms + 2, d->norms + 2, sizeof(double), cudaMemcpyDeviceToHost, s);
  }
  int status = BO_OK;
  for (int r = 0; r < nreal; ++r) {
    bo_dp* d = dps[r];
    if (cudaStreamSynchronize(d->ctx->stream) != cudaSuccess) return BO_ERR_CUDA;
    const double nb = std::sqrt(d->h_norms[0]);
    const double rel = nb > 0 ? std::sqrt(d->h_norms[2]) / nb : std::sqrt(d->h_norms[2]);
    bo_solve_info inf = si[r];
    inf.true_rel_res = rel;
    inf.status = rel <= opts->tol ? BO_OK : BO_ERR_NOT_CONVERGED;
    if (inf.status != BO_OK) {
      // rounding left this one above tol (or its solve stopped short): the
      // single solve with its refinement passes, from zero
      bo_solve_opts o1 = *opts;
      o1.mem = BO_MEM_DEVICE;
      o1.x0_is_zero = 1;
      bo_solve_info i1{};
      bo_dp_solve(d, P[r], b[r], x[r], &o1, &i1);
      i1.iters += inf.iters;
      inf = i1;
    }
    if (infos) infos[r] = inf;
    if (inf.status != BO_OK && status == BO_OK) status = inf.status;
  }
  return status;
}

int bo_dp_destroy(bo_dp* d) {
  if (!d) return BO_ERR_ARG;
  cudaStreamSynchronize(d->ctx->stream);
  bo::dp_free(d);
  bo_ctx* c = d->ctx;
  delete d;
  return bo_ctx_destroy(c);
}

}  // extern "C"
