// Two-phase oil-water systems (paper Sec. 2.2: unknowns p_o and S_w per
// cell, oil and water conservation equations): 2x2 BSR on the 7-point
// pattern.
//
// The system is solved on the three-unknown layout: each 2x2 block becomes
// the upper-left part of a 3x3 block, the third unknown of a cell has a unit
// diagonal and no other coupling, and vectors carry a zero third component.
// Every stage of the CPR is then the 2x2 one: the Quasi-IMPES weight of the
// third row is -0/1 = 0 and the ABF inverse is block diagonal with a unit
// third entry, the block ILU(0) factors of the padded matrix are the 2x2
// factors with a unit third pivot, the AMG acts on the pressure block only,
// and a zero third component stays zero through every Krylov vector.  The
// price is bandwidth: the padded blocks hold 9 values where 4 carry
// information (2.25x the matrix bytes of a native 2x2 layout), accepted to
// run the same tuned kernels.
#include <new>
#include <vector>

#include "bo_internal.cuh"

using namespace bo;

struct bo_ow {
  bo_ctx* ctx;
  bo_mat* m;        // the padded 3x3 matrix (owned)
  int64_t N, nnzb;
  int32_t* rowptr;  // device copy of the pattern
  int32_t* col;
  double* val4;     // device staging of 2x2 values passed from the host
  double* val9;     // padded values
  double* b3;       // padded vectors (3N)
  double* x3;
};

namespace {

// 2x2 blocks -> 3x3 blocks with a unit (2,2) entry on the diagonal block
__global__ void k_ow_pad_matrix(int64_t N, const int32_t* __restrict__ rowptr, const int32_t* __restrict__ col,
                                const double* __restrict__ v4, double* __restrict__ v9) {
  wait_prior_grid();
  for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < N; r += (int64_t)gridDim.x * blockDim.x) {
    for (int32_t e = rowptr[r]; e < rowptr[r + 1]; ++e) {
      const double* a = v4 + 4 * (size_t)e;
      double* o = v9 + 9 * (size_t)e;
      o[0] = a[0];
      o[1] = a[1];
      o[2] = 0.0;
      o[3] = a[2];
      o[4] = a[3];
      o[5] = 0.0;
      o[6] = 0.0;
      o[7] = 0.0;
      o[8] = col[e] == r ? 1.0 : 0.0;
    }
  }
}

// (p, Sw) per cell -> (p, Sw, 0)
__global__ void k_ow_pad_vec(int64_t N, const double* __restrict__ v2, double* __restrict__ v3) {
  wait_prior_grid();
  for (int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; c < N; c += (int64_t)gridDim.x * blockDim.x) {
    v3[3 * c] = v2[2 * c];
    v3[3 * c + 1] = v2[2 * c + 1];
    v3[3 * c + 2] = 0.0;
  }
}

__global__ void k_ow_unpad_vec(int64_t N, const double* __restrict__ v3, double* __restrict__ v2) {
  wait_prior_grid();
  for (int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; c < N; c += (int64_t)gridDim.x * blockDim.x) {
    v2[2 * c] = v3[3 * c];
    v2[2 * c + 1] = v3[3 * c + 1];
  }
}

int ow_status(cudaError_t e) {
  if (e == cudaSuccess) return BO_OK;
  if (e == cudaErrorMemoryAllocation) return BO_ERR_OOM;
  return BO_ERR_CUDA;
}

void ow_free(bo_ow* w) {
  cudaFree(w->rowptr);
  cudaFree(w->col);
  cudaFree(w->val4);
  cudaFree(w->val9);
  cudaFree(w->b3);
  cudaFree(w->x3);
}

// values (host or device) -> padded device values
int ow_pad(bo_ow* w, const double* val, int mem) {
  cudaStream_t s = w->ctx->stream;
  const double* v4 = val;
  if (mem == BO_MEM_HOST) {
    const cudaError_t e = cudaMemcpyAsync(w->val4, val, 4 * (size_t)w->nnzb * sizeof(double), cudaMemcpyHostToDevice, s);
    if (e != cudaSuccess) return ow_status(e);
    v4 = w->val4;
  }
  (launch_pdl(k_ow_pad_matrix, grid_for(w->N), kThreads, 0, s, w->N, w->rowptr, w->col, v4, w->val9), note_launch());
  return BO_OK;
}

}  // namespace

extern "C" {

int bo_ow_create(bo_ctx* ctx, const bo_grid* grid, int32_t nbrows, int64_t nnzb, const int32_t* rowptr,
                 const int32_t* col, const double* val, int mem, bo_ow** out) {
  if (!ctx || !grid || !rowptr || !col || !val || !out) return BO_ERR_ARG;
  if (mem != BO_MEM_HOST && mem != BO_MEM_DEVICE) return BO_ERR_ARG;
  if (grid->nx < 2 || grid->ny < 1 || grid->nz < 1 || grid->ncontinua != 1) return BO_ERR_ARG;
  const int64_t N = (int64_t)grid->nx * grid->ny * grid->nz;
  if (nbrows != N || nnzb <= 0 || nnzb > INT32_MAX || N > ((int64_t)1 << 28)) return BO_ERR_ARG;
  if (cudaSetDevice(ctx->device) != cudaSuccess) return BO_ERR_CUDA;
  // the padding kernel walks the rows: check the row pointers on the host
  // (the matrix ingest checks the pattern itself)
  std::vector<int32_t> hrp(N + 1);
  const cudaMemcpyKind kd = mem == BO_MEM_HOST ? cudaMemcpyHostToHost : cudaMemcpyDeviceToHost;
  if (cudaMemcpy(hrp.data(), rowptr, hrp.size() * sizeof(int32_t), kd) != cudaSuccess) return BO_ERR_CUDA;
  if (hrp[0] != 0 || hrp[N] != nnzb) return BO_ERR_PATTERN;
  for (int64_t r = 0; r < N; ++r)
    if (hrp[r + 1] < hrp[r]) return BO_ERR_PATTERN;
  bo_ow* w = new (std::nothrow) bo_ow();
  if (!w) return BO_ERR_OOM;
  w->ctx = ctx;
  w->N = N;
  w->nnzb = nnzb;
  cudaError_t e = cudaSuccess;
  auto dev = [&](void** p, size_t bytes) {
    if (e == cudaSuccess) e = cudaMalloc(p, bytes);
  };
  dev((void**)&w->rowptr, (N + 1) * sizeof(int32_t));
  dev((void**)&w->col, nnzb * sizeof(int32_t));
  dev((void**)&w->val4, 4 * nnzb * sizeof(double));
  dev((void**)&w->val9, 9 * nnzb * sizeof(double));
  dev((void**)&w->b3, 3 * N * sizeof(double));
  dev((void**)&w->x3, 3 * N * sizeof(double));
  cudaStream_t s = ctx->stream;
  const cudaMemcpyKind k2 = mem == BO_MEM_HOST ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice;
  if (e == cudaSuccess) e = cudaMemcpyAsync(w->rowptr, rowptr, (N + 1) * sizeof(int32_t), k2, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(w->col, col, nnzb * sizeof(int32_t), k2, s);
  int rc = ow_status(e);
  if (rc == BO_OK) rc = ow_pad(w, val, mem);
  if (rc == BO_OK)
    rc = bo_mat_create_bsr(ctx, grid, (int32_t)N, nnzb, w->rowptr, w->col, w->val9, BO_MEM_DEVICE, &w->m);
  if (rc != BO_OK) {
    cudaStreamSynchronize(s);
    ow_free(w);
    delete w;
    return rc;
  }
  ctx->refs++;
  *out = w;
  return BO_OK;
}

int bo_ow_update_values(bo_ow* w, const double* val, int mem) {
  if (!w || !val || (mem != BO_MEM_HOST && mem != BO_MEM_DEVICE)) return BO_ERR_ARG;
  if (cudaSetDevice(w->ctx->device) != cudaSuccess) return BO_ERR_CUDA;
  const int rc = ow_pad(w, val, mem);
  if (rc != BO_OK) return rc;
  return bo_mat_update_values(w->m, w->val9, BO_MEM_DEVICE);
}

bo_mat* bo_ow_matrix(bo_ow* w) { return w ? w->m : nullptr; }

int bo_ow_spmv(bo_ow* w, double alpha, const double* x, double beta, double* y) {
  if (!w || !x || !y) return BO_ERR_ARG;
  if (cudaSetDevice(w->ctx->device) != cudaSuccess) return BO_ERR_CUDA;
  cudaStream_t s = w->ctx->stream;
  const int gN = grid_for(w->N);
  (launch_pdl(k_ow_pad_vec, gN, kThreads, 0, s, w->N, x, w->x3), note_launch());
  if (beta != 0.0) (launch_pdl(k_ow_pad_vec, gN, kThreads, 0, s, w->N, y, w->b3), note_launch());
  launch_spmv_nat(w->m, alpha, w->x3, beta, w->b3, BO_PREC_FP64);
  (launch_pdl(k_ow_unpad_vec, gN, kThreads, 0, s, w->N, w->b3, y), note_launch());
  return ow_status(cudaStreamSynchronize(s));
}

// solver 0: FGMRES, 1: BiCGSTAB
static int ow_solve(bo_ow* w, bo_prec* P, const double* b, double* x, const bo_solve_opts* opts, bo_solve_info* info,
                    int solver) {
  if (!w || !P || !b || !x || P->mat != w->m) return BO_ERR_ARG;
  bo_solve_opts o;
  bo_solve_opts_default(&o);
  if (opts) o = *opts;
  if (!(o.tol > 0.0) || o.maxit < 0 || o.mem != BO_MEM_DEVICE) return BO_ERR_ARG;
  if (solver == 0 && (o.restart < 1 || o.restart > 64)) return BO_ERR_ARG;
  if (solver == 1 && (o.restart < 1 || o.restart > 64)) o.restart = 30;
  if (cudaSetDevice(w->ctx->device) != cudaSuccess) return BO_ERR_CUDA;
  cudaStream_t s = P->stream;
  const int gN = grid_for(w->N);
  (launch_pdl(k_ow_pad_vec, gN, kThreads, 0, s, w->N, b, w->b3), note_launch());
  if (!o.x0_is_zero) (launch_pdl(k_ow_pad_vec, gN, kThreads, 0, s, w->N, x, w->x3), note_launch());
  const int rc = solver == 0 ? fgmres(P, w->b3, w->x3, &o, info) : bicgstab(P, w->b3, w->x3, &o, info);
  (launch_pdl(k_ow_unpad_vec, gN, kThreads, 0, s, w->N, w->x3, x), note_launch());
  const int rs = ow_status(cudaStreamSynchronize(s));
  return rc != BO_OK ? rc : rs;
}

int bo_ow_solve(bo_ow* w, bo_prec* P, const double* b, double* x, const bo_solve_opts* opts, bo_solve_info* info) {
  return ow_solve(w, P, b, x, opts, info, 0);
}

int bo_ow_solve_bicgstab(bo_ow* w, bo_prec* P, const double* b, double* x, const bo_solve_opts* opts,
                         bo_solve_info* info) {
  return ow_solve(w, P, b, x, opts, info, 1);
}

int bo_ow_destroy(bo_ow* w) {
  if (!w) return BO_ERR_ARG;
  cudaSetDevice(w->ctx->device);
  cudaStreamSynchronize(w->ctx->stream);
  bo_mat_destroy(w->m);
  ow_free(w);
  bo_ctx* c = w->ctx;
  delete w;
  return bo_ctx_destroy(c);
}

}  // extern "C"
