// Learned coarse space inside CPR and the learned initial guess.  No
// counterpart in the paper: an addition that hands the preconditioner of
// Sec. 3.3 (Alg. 2) a predicted pressure field and the Krylov solve of
// Sec. 3 a predicted starting point.
//
// Coarse space.  The grid is cut into tiles of tx x ty x tz cells; column t
// of Z holds the predicted pressure update dp on the cells of tile t and
// zero elsewhere.  With A~_pp the decoupled pressure block (row 0 of
// D_QI^{-1} A against the pressure unknowns, the matrix the AMG V-cycle
// solves), E = Z^T A~_pp Z is a dense nt x nt matrix, inverted once per
// matrix in FP64.  After each V-cycle on the pressure residual f,
//   e += Z E^{-1} Z^T f,
// an additive two-level correction.  Flexible GMRES accepts the changed
// preconditioner as it accepts any other.
//
// Layout: dp is held in the solver's colour-split order (colour (i+j+k) & 1,
// half index q = c >> 1), like the pressure vectors it multiplies.
#include <cmath>

#include "bo_internal.cuh"

namespace bo {
namespace {

constexpr int kMaxTiles = 128;

struct Tiles {
  int tx, ty, tz;  // tile size in cells
  int nx, ny, nz;  // tiles per axis
};

__device__ __forceinline__ int tile_of(const Tiles& T, int i, int j, int k) {
  return i / T.tx + T.nx * (j / T.ty + T.ny * (k / T.tz));
}

// z[colour-split] = dp[natural]
// z (colour-split order) = scale * dp[c * stride] (natural order): an FP64
// field (stride 1) or channel 0 of a network prediction [N][4] (stride 4)
template <typename T>
__global__ void k_lc_perm(Geom g, const T* __restrict__ dp, int stride, double scale, double* __restrict__ z) {
  wait_prior_grid();
  for (int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; c < g.N; c += (int64_t)gridDim.x * blockDim.x) {
    const int i = (int)(c % g.nx), j = (int)((c / g.nx) % g.ny), k = (int)(c / ((int64_t)g.nx * g.ny));
    z[((i + j + k) & 1) * g.Nh + (c >> 1)] = scale * (double)dp[c * stride];
  }
}

// Row s of E = Z^T A~_pp Z, one block per tile s.  A cell couples only to
// its 6 neighbours, so row s has at most 7 nonzeros (its own tile and the 6
// adjacent tiles); every thread sums its cells' contributions to those 7 in
// registers, then one block reduction per entry.  E is zeroed first; a tile
// whose column of Z is zero gets E_ss = 1 so that E stays invertible (the
// correction on it is zero either way).
__global__ void k_lc_galerkin(Geom g, Tiles T, const double* __restrict__ A, const double* __restrict__ w,
                              const double* __restrict__ z, double* __restrict__ E, int nt) {
  wait_prior_grid();
  __shared__ double sh[32];
  const int s = blockIdx.x;
  const int a = s % T.nx, b = (s / T.nx) % T.ny, c = s / (T.nx * T.ny);
  const int i0 = a * T.tx, j0 = b * T.ty, k0 = c * T.tz;
  const int i1 = min(i0 + T.tx, g.nx), j1 = min(j0 + T.ty, g.ny), k1 = min(k0 + T.tz, g.nz);
  const int li = i1 - i0, lj = j1 - j0, lk = k1 - k0;
  const int cnt = li * lj * lk;
  double acc[7] = {0, 0, 0, 0, 0, 0, 0};  // by the neighbour tile's direction (slot order)
  double zz = 0.0;
  for (int t = threadIdx.x; t < cnt; t += blockDim.x) {
    const int i = i0 + t % li, j = j0 + (t / li) % lj, k = k0 + t / (li * lj);
    const int color = (i + j + k) & 1;
    const int64_t q = (i + (int64_t)g.nx * (j + (int64_t)g.ny * k)) >> 1;
    const double zc = z[color * g.Nh + q];
    zz += zc * zc;
    if (zc == 0.0) continue;
    const double g0 = w[vidx(g, 0, color, q)], g1 = w[vidx(g, 1, color, q)], g2 = w[vidx(g, 2, color, q)];
    const int ni[7] = {i, i, i - 1, i, i + 1, i, i};
    const int nj[7] = {j, j - 1, j, j, j, j + 1, j};
    const int nk[7] = {k - 1, k, k, k, k, k, k + 1};
#pragma unroll
    for (int sl = 0; sl < 7; ++sl) {
      if (ni[sl] < 0 || ni[sl] >= g.nx || nj[sl] < 0 || nj[sl] >= g.ny || nk[sl] < 0 || nk[sl] >= g.nz) continue;
      const double app = g0 * A[plane(g, color, sl, 0) + q] + g1 * A[plane(g, color, sl, 3) + q] +
                         g2 * A[plane(g, color, sl, 6) + q];
      const int ncol = (ni[sl] + nj[sl] + nk[sl]) & 1;
      const int64_t nq = (ni[sl] + (int64_t)g.nx * (nj[sl] + (int64_t)g.ny * nk[sl])) >> 1;
      const double zd = z[ncol * g.Nh + nq];
      // which tile the neighbour is in: own, or the adjacent one across that face
      const bool own = ni[sl] / T.tx == a && nj[sl] / T.ty == b && nk[sl] / T.tz == c;
      acc[own ? kDiag : sl] += zc * app * zd;
    }
  }
  zz = block_sum(zz, sh);
  double row[7];
#pragma unroll
  for (int sl = 0; sl < 7; ++sl) row[sl] = block_sum(acc[sl], sh);
  if (threadIdx.x == 0) {
    const int da[7] = {0, 0, -1, 0, 1, 0, 0}, db[7] = {0, -1, 0, 0, 0, 1, 0}, dc[7] = {-1, 0, 0, 0, 0, 0, 1};
    for (int sl = 0; sl < 7; ++sl) {
      const int aa = a + da[sl], bb = b + db[sl], cc = c + dc[sl];
      if (aa < 0 || aa >= T.nx || bb < 0 || bb >= T.ny || cc < 0 || cc >= T.nz) continue;
      E[(size_t)s * nt + aa + T.nx * (bb + T.ny * cc)] = row[sl];
    }
    if (zz == 0.0) E[(size_t)s * nt + s] = 1.0;
  }
}

// y[t] = (Z^T f)_t, one block per tile
template <typename T>
__global__ void k_lc_restrict(Geom g, Tiles Tl, const double* __restrict__ z, const T* __restrict__ f,
                              double* __restrict__ y, const DevState* st) {
  wait_prior_grid();
  __shared__ double sh[32];
  if (st->done) return;
  const int s = blockIdx.x;
  const int a = s % Tl.nx, b = (s / Tl.nx) % Tl.ny, c = s / (Tl.nx * Tl.ny);
  const int i0 = a * Tl.tx, j0 = b * Tl.ty, k0 = c * Tl.tz;
  const int li = min(i0 + Tl.tx, g.nx) - i0, lj = min(j0 + Tl.ty, g.ny) - j0, lk = min(k0 + Tl.tz, g.nz) - k0;
  double acc = 0.0;
  for (int t = threadIdx.x; t < li * lj * lk; t += blockDim.x) {
    const int i = i0 + t % li, j = j0 + (t / li) % lj, k = k0 + t / (li * lj);
    const int64_t idx = ((i + j + k) & 1) * g.Nh + ((i + (int64_t)g.nx * (j + (int64_t)g.ny * k)) >> 1);
    acc += z[idx] * (double)f[idx];
  }
  acc = block_sum(acc, sh);
  if (threadIdx.x == 0) y[s] = acc;
}

// u = E^{-1} y (one block)
__global__ void k_lc_solve(int nt, const double* __restrict__ Einv, const double* __restrict__ y,
                           double* __restrict__ u, const DevState* st) {
  wait_prior_grid();
  if (st->done) return;
  for (int r = threadIdx.x; r < nt; r += blockDim.x) {
    double s = 0.0;
    for (int c = 0; c < nt; ++c) s += Einv[(size_t)r * nt + c] * y[c];
    u[r] = s;
  }
}

// e += Z u
template <typename T>
__global__ void k_lc_prolong(Geom g, Tiles Tl, const double* __restrict__ z, const double* __restrict__ u,
                             T* __restrict__ e, const DevState* st) {
  wait_prior_grid();
  if (st->done) return;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < g.N; t += (int64_t)gridDim.x * blockDim.x) {
    const int color = t >= g.Nh;
    const Cell c = decode(g, color, t - color * g.Nh);
    e[t] = (T)((double)e[t] + z[t] * u[tile_of(Tl, c.i, c.j, c.k)]);
  }
}

// x0[3 c + k] = scale[k] pred[c][k] for k < ncomp, else 0 (natural order)
__global__ void k_guess(int64_t N, const float* __restrict__ pred, double s0, double s1, double s2, int ncomp,
                        double* __restrict__ x0) {
  wait_prior_grid();
  for (int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; c < N; c += (int64_t)gridDim.x * blockDim.x) {
    x0[3 * c] = s0 * (double)pred[4 * c];
    x0[3 * c + 1] = ncomp > 1 ? s1 * (double)pred[4 * c + 1] : 0.0;
    x0[3 * c + 2] = ncomp > 2 ? s2 * (double)pred[4 * c + 2] : 0.0;
  }
}

// ||b - A x0||^2 and ||b||^2 on natural-order vectors (FP64), into out[0..1]:
// per-block partials in the preconditioner's reduction memory, summed in a
// fixed order by the block that finishes last (counter 6 of the device state)
__global__ void __launch_bounds__(kThreads) k_guess_norms(Geom g, const double* __restrict__ A,
                                                         const double* __restrict__ b,
                                                         const double* __restrict__ x, double* partials,
                                                         DevState* st, double* __restrict__ out) {
  wait_prior_grid();
  __shared__ double sh[32];
  double rr = 0.0, bb = 0.0;
  for (int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; c < g.N; c += (int64_t)gridDim.x * blockDim.x) {
    const Nat n = decode_nat(g, c);
    const unsigned valid = valid_slots(g, n);
    double a0 = 0.0, a1 = 0.0, a2 = 0.0;
#pragma unroll
    for (int s = 0; s < 7; ++s) {
      if (!((valid >> s) & 1u)) continue;
      const int64_t nc = c + nat_offset(g, s);
      const double* a = A + plane(g, n.color, s, 0) + n.q;
      const size_t P = (size_t)g.Nh;
      a0 = fma3(a0, a[0], x[3 * nc], a[P], x[3 * nc + 1], a[2 * P], x[3 * nc + 2]);
      a1 = fma3(a1, a[3 * P], x[3 * nc], a[4 * P], x[3 * nc + 1], a[5 * P], x[3 * nc + 2]);
      a2 = fma3(a2, a[6 * P], x[3 * nc], a[7 * P], x[3 * nc + 1], a[8 * P], x[3 * nc + 2]);
    }
    const double b0 = b[3 * c], b1 = b[3 * c + 1], b2 = b[3 * c + 2];
    const double r0 = b0 - a0, r1 = b1 - a1, r2 = b2 - a2;
    rr += r0 * r0 + r1 * r1 + r2 * r2;
    bb += b0 * b0 + b1 * b1 + b2 * b2;
  }
  rr = block_sum(rr, sh);
  bb = block_sum(bb, sh);
  if (threadIdx.x == 0) {
    partials[2 * blockIdx.x] = rr;
    partials[2 * blockIdx.x + 1] = bb;
  }
  if (!last_block(&st->counter[6], gridDim.x)) return;
  double sr = 0.0, sb = 0.0;
  for (int i = threadIdx.x; i < (int)gridDim.x; i += blockDim.x) {
    sr += __ldcg(partials + 2 * i);
    sb += __ldcg(partials + 2 * i + 1);
  }
  sr = block_sum(sr, sh);
  sb = block_sum(sb, sh);
  if (threadIdx.x == 0) {
    out[0] = sqrt(sr);
    out[1] = sqrt(sb);
    st->counter[6] = 0;
  }
}

__global__ void k_zero64(int64_t n, double* __restrict__ x) {
  wait_prior_grid();
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    x[i] = 0.0;
}

Tiles tiles_of(const bo_prec* P) {
  return Tiles{P->lc_tile[0], P->lc_tile[1], P->lc_tile[2], P->lc_ntile[0], P->lc_ntile[1], P->lc_ntile[2]};
}

}  // namespace

int learned_coarse_values(bo_prec* P) {
  if (P->lc_nt == 0) return BO_OK;
  const Geom& g = P->mat->g;
  cudaStream_t s = P->stream;
  const int nt = P->lc_nt;
  cudaMemsetAsync(P->lc_E, 0, (size_t)nt * nt * sizeof(double), s);
  (launch_pdl(k_lc_galerkin, nt, kThreads, 0, s, g, tiles_of(P), P->mat->A, P->w, P->lc_z, P->lc_E, nt), note_launch());
  return launch_dense_inverse64(nt, P->lc_E, P->lc_Einv, P->st, s);
}

void learned_coarse_apply(bo_prec* P, const DevState* st) {
  if (P->lc_nt == 0) return;
  const Geom& g = P->mat->g;
  cudaStream_t s = P->stream;
  const Tiles T = tiles_of(P);
  if (P->fp32) {
    (launch_pdl(k_lc_restrict<float>, P->lc_nt, kThreads, 0, s, g, T, P->lc_z, (const float*)P->f0, P->lc_y, st),
     note_launch());
    (launch_pdl(k_lc_solve, 1, kThreads, 0, s, P->lc_nt, P->lc_Einv, P->lc_y, P->lc_u, st), note_launch());
    (launch_pdl(k_lc_prolong<float>, grid_for(g.N), kThreads, 0, s, g, T, P->lc_z, P->lc_u, (float*)P->e0, st),
     note_launch());
  } else {
    (launch_pdl(k_lc_restrict<double>, P->lc_nt, kThreads, 0, s, g, T, P->lc_z, (const double*)P->f0, P->lc_y, st),
     note_launch());
    (launch_pdl(k_lc_solve, 1, kThreads, 0, s, P->lc_nt, P->lc_Einv, P->lc_y, P->lc_u, st), note_launch());
    (launch_pdl(k_lc_prolong<double>, grid_for(g.N), kThreads, 0, s, g, T, P->lc_z, P->lc_u, (double*)P->e0, st),
     note_launch());
  }
}

void learned_coarse_free(bo_prec* P) {
  auto fr = [](void* p) { if (p) cudaFree(p); };
  fr(P->lc_z); fr(P->lc_E); fr(P->lc_Einv); fr(P->lc_y); fr(P->lc_u);
  P->lc_z = P->lc_E = P->lc_Einv = P->lc_y = P->lc_u = nullptr;
  P->lc_nt = 0;
  P->setups++;
}

}  // namespace bo

namespace bo {
namespace {

// the coarse space from dp (FP64, stride 1) or a prediction (FP32, stride 4)
template <typename T>
int set_coarse_space(bo_prec* P, const T* dp, int stride, double scale, int tx, int ty, int tz) {
  if (!P) return BO_ERR_ARG;
  if (cudaSetDevice(P->mat->ctx->device) != cudaSuccess) return BO_ERR_CUDA;
  cudaStreamSynchronize(P->stream);
  learned_coarse_free(P);
  graphs_reset(P);  // captured columns hold the old preconditioner sequence
  if (!dp) return BO_OK;
  const Geom& g = P->mat->g;
  if (tx < 1 || ty < 1 || tz < 1 || !std::isfinite(scale)) return BO_ERR_ARG;
  const int ntx = (g.nx + tx - 1) / tx, nty = (g.ny + ty - 1) / ty, ntz = (g.nz + tz - 1) / tz;
  const int64_t nt = (int64_t)ntx * nty * ntz;
  if (nt > kMaxTiles) return BO_ERR_ARG;
  bool ok = cudaMalloc(&P->lc_z, g.N * sizeof(double)) == cudaSuccess &&
            cudaMalloc(&P->lc_E, nt * nt * sizeof(double)) == cudaSuccess &&
            cudaMalloc(&P->lc_Einv, nt * nt * sizeof(double)) == cudaSuccess &&
            cudaMalloc(&P->lc_y, nt * sizeof(double)) == cudaSuccess &&
            cudaMalloc(&P->lc_u, nt * sizeof(double)) == cudaSuccess;
  if (!ok) {
    learned_coarse_free(P);
    return BO_ERR_OOM;
  }
  P->lc_tile[0] = tx; P->lc_tile[1] = ty; P->lc_tile[2] = tz;
  P->lc_ntile[0] = ntx; P->lc_ntile[1] = nty; P->lc_ntile[2] = ntz;
  P->lc_nt = (int)nt;
  P->setups++;
  cudaStream_t s = P->stream;
  cudaMemsetAsync(&P->st->err, 0, sizeof(P->st->err), s);
  (launch_pdl(k_lc_perm<T>, grid_for(g.N), kThreads, 0, s, g, dp, stride, scale, P->lc_z), note_launch());
  int rc = learned_coarse_values(P);
  DevState h;
  if (cudaMemcpyAsync(&h, P->st, sizeof(h), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
      cudaStreamSynchronize(s) != cudaSuccess)
    rc = BO_ERR_CUDA;
  if (rc == BO_OK && h.err) rc = BO_ERR_BREAKDOWN;
  if (rc != BO_OK) learned_coarse_free(P);
  return rc;
}

}  // namespace
}  // namespace bo

extern "C" {

int bo_prec_set_coarse_space(bo_prec* P, const double* dp, int tx, int ty, int tz) {
  return bo::set_coarse_space<double>(P, dp, 1, 1.0, tx, ty, tz);
}

int bo_learned_coarse_space(bo_prec* P, const float* pred, double scale, int tx, int ty, int tz) {
  return bo::set_coarse_space<float>(P, pred, 4, scale, tx, ty, tz);
}

int bo_learned_guess(bo_prec* P, const double* b, const float* pred, const double* scale, int ncomp, double* x0,
                     int* used) {
  if (!P || !b || !pred || !scale || !x0 || ncomp < 1 || ncomp > 3) return BO_ERR_ARG;
  if (cudaSetDevice(P->mat->ctx->device) != cudaSuccess) return BO_ERR_CUDA;
  const bo::Geom& g = P->mat->g;
  cudaStream_t s = P->mat->ctx->stream;
  (bo::launch_pdl(bo::k_guess, bo::grid_for(g.N), bo::kThreads, 0, s, g.N, pred, scale[0], scale[1], scale[2], ncomp, x0),
   bo::note_launch());
  // ||b - A x0|| against ||b||: partial sums in the preconditioner's own
  // reduction memory, the two norms at the start of the idle Krylov basis
  double* norms = P->V;
  (bo::launch_pdl(bo::k_guess_norms, bo::grid_for(g.N), bo::kThreads, 0, s, g, P->mat->A, b, x0, P->partials, P->st, norms),
   bo::note_launch());
  double h[2];
  if (cudaMemcpyAsync(h, norms, sizeof(h), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
      cudaStreamSynchronize(s) != cudaSuccess)
    return BO_ERR_CUDA;
  const int keep = std::isfinite(h[0]) && h[0] < h[1];
  if (!keep) (bo::launch_pdl(bo::k_zero64, bo::grid_for(3 * g.N), bo::kThreads, 0, s, 3 * g.N, x0), bo::note_launch());
  if (used) *used = keep;
  return cudaGetLastError() == cudaSuccess ? BO_OK : BO_ERR_CUDA;
}

}  // extern "C"
