// C ABI entry points (declared in bosolve.h): argument checks, object
// lifetimes, host <-> device staging and error mapping.  All arithmetic runs
// in the kernels of layout.cu, precond.cu and krylov.cu.
#include <algorithm>
#include <cstdlib>
#include <cstring>
#include <mutex>
#include <new>
#include <unordered_map>
#include <vector>

#include "bo_internal.cuh"

using namespace bo;

namespace bo {
std::atomic<long long> g_launches{0};
std::atomic<int> g_pool_width{kMaxPoolStreams};
std::atomic<int> g_conv_engine{1};
std::atomic<int> g_amg_coop{2};
std::atomic<unsigned> g_amg_spins{kAmgSpinsDefault};
std::atomic<int> g_gs_fused{1};

int occ_grid(const void* kernel, int64_t n, int threads, size_t smem) {
  static std::mutex mu;
  static std::unordered_map<const void*, int> cache;
  int dev = 0;
  cudaGetDevice(&dev);
  int per_sm = 0;
  {
    std::lock_guard<std::mutex> lk(mu);
    auto it = cache.find(kernel);
    if (it != cache.end()) per_sm = it->second;
  }
  if (per_sm == 0) {
    int sms = 0, b = 0;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, kernel, threads, smem);
    per_sm = (b > 0 ? b : 1) * (sms > 0 ? sms : 1);
    std::lock_guard<std::mutex> lk(mu);
    cache[kernel] = per_sm;
  }
  const int64_t need = (n + threads - 1) / threads;
  return (int)(need < 1 ? 1 : (need < per_sm ? need : per_sm));
}
}

namespace {

void ctx_release(bo_ctx* c) {
  if (--c->refs > 0) return;
  cudaStreamSynchronize(c->stream);
  if (c->own_stream) cudaStreamDestroy(c->stream);
  delete c;
}

int cuda_status(cudaError_t e) {
  if (e == cudaSuccess) return BO_OK;
  if (e == cudaErrorMemoryAllocation) return BO_ERR_OOM;
  return BO_ERR_CUDA;
}

bool grid_ok(const bo_grid* g) {
  return g && g->nx >= 2 && g->ny >= 1 && g->nz >= 1 && (g->nx % 2) == 0 && g->ncontinua == 1 &&
         (int64_t)g->nx * g->ny * g->nz <= ((int64_t)1 << 28);
}

int64_t nnzb_of(const bo_grid* g) {
  const int64_t nx = g->nx, ny = g->ny, nz = g->nz;
  return nx * ny * nz + 2 * ((nx - 1) * ny * nz + nx * (ny - 1) * nz + nx * ny * (nz - 1));
}

// read back and clear the matrix error flags; map to a status
int mat_flags(bo_mat* m) {
  cudaMemcpyAsync(m->h_flags, m->flags, sizeof(int), cudaMemcpyDeviceToHost, m->ctx->stream);
  cudaError_t e = cudaStreamSynchronize(m->ctx->stream);
  if (e != cudaSuccess) return cuda_status(e);
  const int f = *m->h_flags;
  cudaMemsetAsync(m->flags, 0, sizeof(int), m->ctx->stream);
  if (f & kErrPattern) return BO_ERR_PATTERN;
  if (f & kErrNonfinite) return BO_ERR_NONFINITE;
  return BO_OK;
}

int load_values(bo_mat* m, const double* val, int mem) {
  const size_t bytes = (m->kind == 0 ? 9 * (size_t)m->nnz : (size_t)m->nnz) * sizeof(double);
  const double* dval = val;
  if (mem == BO_MEM_HOST) {
    cudaError_t e = cudaMemcpyAsync(m->stage, val, bytes, cudaMemcpyHostToDevice, m->ctx->stream);
    if (e != cudaSuccess) return cuda_status(e);
    dval = m->stage;
  }
  int rc = m->kind == 0 ? ingest_bsr(m, dval, m->ctx->stream) : ingest_csr(m, dval, m->ctx->stream);
  if (rc != BO_OK) return rc;
  m->a32_valid = false;
  m->a16_valid = false;
  return mat_flags(m);
}

void mat_free(bo_mat* m) {
  if (!m) return;
  cudaStreamSynchronize(m->ctx->stream);
  cudaFree(m->rowptr);
  cudaFree(m->col);
  cudaFree(m->stage);
  cudaFree(m->A);
  cudaFree(m->A32);
  cudaFree(m->A16);
  cudaFree(m->A2);
  cudaFree(m->a2_range);
  cudaFree(m->flags);
  cudaFreeHost(m->h_flags);
  bo_ctx* c = m->ctx;
  delete m;
  ctx_release(c);
}

void mat_release(bo_mat* m) {
  if (--m->refs == 0) mat_free(m);
}

}  // namespace

namespace bo {
void ctx_release_ref(bo_ctx* c) { ctx_release(c); }
void mat_release_ref(bo_mat* m) { mat_release(m); }
}  // namespace bo

namespace {

int mat_create(bo_ctx* ctx, const bo_grid* grid, int kind, int64_t nrows, int64_t nnz, const int32_t* rowptr,
               const int32_t* col, const double* val, int mem, bo_mat** out) {
  if (!ctx || !out || !rowptr || !col || !val || !grid_ok(grid) || nnz <= 0 || nnz > INT32_MAX) return BO_ERR_ARG;
  if (mem != BO_MEM_HOST && mem != BO_MEM_DEVICE) return BO_ERR_ARG;
  const int64_t N = (int64_t)grid->nx * grid->ny * grid->nz;
  if (nrows != (kind == 0 ? N : 3 * N)) return BO_ERR_ARG;
  if (kind == 0 && nnz != nnzb_of(grid)) return BO_ERR_PATTERN;
  if (cudaSetDevice(ctx->device) != cudaSuccess) return BO_ERR_CUDA;
  if (mem == BO_MEM_HOST) {  // cheap host-side checks of the row pointers
    if (rowptr[0] != 0 || rowptr[nrows] != nnz) return BO_ERR_PATTERN;
    for (int64_t i = 0; i < nrows; ++i)
      if (rowptr[i + 1] < rowptr[i]) return BO_ERR_PATTERN;
  }
  bo_mat* m = new (std::nothrow) bo_mat();
  if (!m) return BO_ERR_OOM;
  std::memset(m, 0, sizeof(*m));
  m->ctx = ctx;
  m->refs = 1;
  ctx->refs++;
  m->grid = *grid;
  m->g = Geom{grid->nx, grid->ny, grid->nz, grid->nx / 2, N, N / 2};
  m->kind = kind;
  m->nnz = nnz;
  cudaStream_t s = ctx->stream;
  const size_t vbytes = (kind == 0 ? 9 * (size_t)nnz : (size_t)nnz) * sizeof(double);
  cudaError_t e = cudaSuccess;
  if (e == cudaSuccess) e = cudaMalloc(&m->rowptr, (nrows + 1) * sizeof(int32_t));
  if (e == cudaSuccess) e = cudaMalloc(&m->col, nnz * sizeof(int32_t));
  if (e == cudaSuccess) e = cudaMalloc(&m->stage, vbytes);
  if (e == cudaSuccess) e = cudaMalloc(&m->A, (size_t)63 * N * sizeof(double));
  if (e == cudaSuccess) e = cudaMalloc(&m->A2, a2_size(m->g) * sizeof(float2));
  if (e == cudaSuccess) e = cudaMalloc(&m->a2_range, sizeof(int));
  if (e == cudaSuccess) e = cudaMalloc(&m->flags, sizeof(int));
  if (e == cudaSuccess) e = cudaMallocHost(&m->h_flags, sizeof(int));
  if (e != cudaSuccess) {
    mat_free(m);
    return cuda_status(e);
  }
  const cudaMemcpyKind kd = mem == BO_MEM_HOST ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice;
  cudaMemcpyAsync(m->rowptr, rowptr, (nrows + 1) * sizeof(int32_t), kd, s);
  cudaMemcpyAsync(m->col, col, nnz * sizeof(int32_t), kd, s);
  cudaMemsetAsync(m->flags, 0, sizeof(int), s);
  int rc = load_values(m, val, mem);
  if (rc != BO_OK) {
    mat_free(m);
    return rc;
  }
  *out = m;
  return BO_OK;
}

// a pool of streams per device, created once and kept for the process;
// batched calls use the first g_pool_width of them
bool stream_pool(int dev, std::vector<cudaStream_t>& pool) {
  static std::mutex mu;
  static std::unordered_map<int, std::vector<cudaStream_t>> pools;
  std::lock_guard<std::mutex> lk(mu);
  auto& pl = pools[dev];
  if (pl.empty())
    for (int i = 0; i < kMaxPoolStreams; ++i) {
      cudaStream_t st;
      if (cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess) return false;
      pl.push_back(st);
    }
  pool = pl;
  return true;
}

void prec_opts_fill(const bo_prec_opts* in, bo_prec_opts* o) {
  bo_prec_opts_default(o);
  if (in) *o = *in;
}

// set up values and read the error bits back
int prec_refresh(bo_prec* P) {
  cudaStream_t s = P->stream;
  cudaMemsetAsync(&P->st->err, 0, sizeof(int), s);
  int rc = prec_values(P);
  if (rc != BO_OK) return rc;
  int err = 0;
  cudaError_t e = cudaMemcpyAsync(P->mat->h_flags, &P->st->err, sizeof(int), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return cuda_status(e);
  err = *P->mat->h_flags;
  cudaMemsetAsync(&P->st->err, 0, sizeof(int), s);
  cudaMemsetAsync(&P->st->done, 0, sizeof(int), s);
  P->setups++;
  if (err & kErrBreakdown) return BO_ERR_BREAKDOWN;
  if (err & kErrNonfinite) return BO_ERR_NONFINITE;
  return BO_OK;
}

}  // namespace

namespace bo {
int solve_batched(bo_prec* const* P, int nreal, const double* const* b, double* const* x, const bo_solve_opts& o,
                  bo_solve_info* infos, const double* tols) {
  const int dev = P[0]->mat->ctx->device;
  if (cudaSetDevice(dev) != cudaSuccess) return BO_ERR_CUDA;
  std::vector<cudaStream_t> pool;
  if (!stream_pool(dev, pool)) return BO_ERR_CUDA;
  constexpr int kPool = kMaxPoolStreams;
  // order the batch after everything already queued on the contexts' streams,
  // and the contexts' streams after the batch
  std::vector<cudaEvent_t> evs;
  auto join = [&](cudaStream_t from, cudaStream_t to) {
    cudaEvent_t e;
    cudaEventCreateWithFlags(&e, cudaEventDisableTiming);
    cudaEventRecord(e, from);
    cudaStreamWaitEvent(to, e, 0);
    evs.push_back(e);
  };
  const int width = std::min(kPool, std::max(1, g_pool_width.load()));
  const int S = nreal < width ? nreal : width;
  for (int r = 0; r < nreal; ++r) join(P[r]->mat->ctx->stream, pool[r % S]);
  for (int r = 0; r < nreal; ++r) P[r]->stream = pool[r % S];
  const int rc = fgmres_batched(P, nreal, b, x, &o, infos, tols);
  for (int r = 0; r < nreal; ++r) {
    join(pool[r % S], P[r]->mat->ctx->stream);
    P[r]->stream = P[r]->mat->ctx->stream;
  }
  for (int r = 0; r < S; ++r) cudaStreamSynchronize(pool[r]);
  for (auto e : evs) cudaEventDestroy(e);
  return rc;
}
}  // namespace bo

extern "C" {

const char* bo_status_str(int s) {
  switch (s) {
    case BO_OK: return "ok";
    case BO_ERR_ARG: return "invalid argument";
    case BO_ERR_CUDA: return "CUDA error";
    case BO_ERR_OOM: return "out of device memory";
    case BO_ERR_PATTERN: return "pattern is not the grid's 7-point stencil";
    case BO_ERR_NONFINITE: return "non-finite value in input";
    case BO_ERR_BREAKDOWN: return "singular pivot (decoupling, ILU or AMG)";
    case BO_ERR_NOT_CONVERGED: return "iteration limit reached";
    case BO_ERR_TIMEOUT: return "device loop cap reached";
    default: return "unknown status";
  }
}

void bo_prec_opts_default(bo_prec_opts* o) {
  if (!o) return;
  o->precision = BO_PREC_FP64;
  o->amg_nu1 = 2;
  o->amg_nu2 = 2;
  o->amg_overcorr = 1.3;
  o->amg_coarse_max = 128;
  o->decoupling = BO_DECOUPLE_QI;
}

void bo_solve_opts_default(bo_solve_opts* o) {
  if (!o) return;
  o->tol = 1e-8;
  o->restart = 30;
  o->maxit = 500;
  o->x0_is_zero = 0;
  o->mem = BO_MEM_DEVICE;
  o->profile = 0;
}

int bo_ctx_create(int device, void* cuda_stream, bo_ctx** out) {
  if (!out) return BO_ERR_ARG;
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev) return BO_ERR_ARG;
  if (cudaSetDevice(device) != cudaSuccess) return BO_ERR_CUDA;
  bo_ctx* c = new (std::nothrow) bo_ctx();
  if (!c) return BO_ERR_OOM;
  c->device = device;
  c->refs = 1;
  if (cuda_stream) {
    c->stream = (cudaStream_t)cuda_stream;
    c->own_stream = false;
  } else {
    if (cudaStreamCreateWithFlags(&c->stream, cudaStreamNonBlocking) != cudaSuccess) {
      delete c;
      return BO_ERR_CUDA;
    }
    c->own_stream = true;
  }
  *out = c;
  return BO_OK;
}

int bo_ctx_destroy(bo_ctx* c) {
  if (!c) return BO_ERR_ARG;
  ctx_release(c);
  return BO_OK;
}

int bo_mat_create_bsr(bo_ctx* ctx, const bo_grid* grid, int32_t nbrows, int64_t nnzb, const int32_t* rowptr,
                      const int32_t* col, const double* val, int mem, bo_mat** out) {
  return mat_create(ctx, grid, 0, nbrows, nnzb, rowptr, col, val, mem, out);
}

int bo_mat_create_csr(bo_ctx* ctx, const bo_grid* grid, int32_t nrows, int64_t nnz, const int32_t* rowptr,
                      const int32_t* col, const double* val, int mem, bo_mat** out) {
  return mat_create(ctx, grid, 1, nrows, nnz, rowptr, col, val, mem, out);
}

int bo_mat_update_values(bo_mat* m, const double* val, int mem) {
  if (!m || !val || (mem != BO_MEM_HOST && mem != BO_MEM_DEVICE)) return BO_ERR_ARG;
  return load_values(m, val, mem);
}

int bo_mat_spmv(bo_mat* m, double alpha, const double* x, double beta, double* y, int precision) {
  if (!m || !x || !y) return BO_ERR_ARG;
  if (precision != BO_PREC_FP64 && precision != BO_PREC_FP32 && precision != BO_PREC_BF16) return BO_ERR_ARG;
  // the reduced-precision copies, in the split copy's tiled layout
  if (precision == BO_PREC_FP32 && !m->a32_valid) {
    if (!m->A32 && cudaMalloc(&m->A32, a2_size(m->g) * sizeof(float)) != cudaSuccess) return BO_ERR_OOM;
    launch_to_tiled_f32(m, m->A32, m->ctx->stream);
    m->a32_valid = true;
  }
  if (precision == BO_PREC_BF16 && !m->a16_valid) {
    if (!m->A16 && cudaMalloc(&m->A16, a2_size(m->g) * sizeof(__nv_bfloat16)) != cudaSuccess) return BO_ERR_OOM;
    launch_to_tiled_bf16(m, m->A16, m->ctx->stream);
    m->a16_valid = true;
  }
  launch_spmv_nat(m, alpha, x, beta, y, precision);
  return cuda_status(cudaGetLastError());
}

int bo_mat_destroy(bo_mat* m) {
  if (!m) return BO_ERR_ARG;
  mat_release(m);
  return BO_OK;
}

int bo_prec_setup(bo_mat* m, const bo_prec_opts* opts, bo_prec** out) {
  if (!m || !out) return BO_ERR_ARG;
  bo_prec_opts o;
  prec_opts_fill(opts, &o);
  if ((o.precision != BO_PREC_FP64 && o.precision != BO_PREC_FP32 && o.precision != BO_PREC_BF16) ||
      o.amg_nu1 < 0 || o.amg_nu2 < 0 ||
      o.amg_nu1 > 8 || o.amg_nu2 > 8 || o.amg_coarse_max < 1 || o.amg_coarse_max > 128 ||
      (o.decoupling != BO_DECOUPLE_QI && o.decoupling != BO_DECOUPLE_ABF) ||
      !(o.amg_overcorr > 0.0 && o.amg_overcorr < 4.0))
    return BO_ERR_ARG;
  if (cudaSetDevice(m->ctx->device) != cudaSuccess) return BO_ERR_CUDA;
  bo_prec* P = new (std::nothrow) bo_prec();  // value-initialised: every member zero or its default
  if (!P) return BO_ERR_OOM;
  P->mat = m;
  P->stream = m->ctx->stream;
  m->refs++;
  P->opts = o;
  P->fp32 = o.precision != BO_PREC_FP64;
  P->bf16 = o.precision == BO_PREC_BF16;
  P->tsize = P->fp32 ? sizeof(float) : sizeof(double);
  P->ssize = P->bf16 ? sizeof(__nv_bfloat16) : P->tsize;
  int rc = prec_alloc(P);
  if (rc == BO_OK) rc = krylov_alloc(P, 30);
  if (rc == BO_OK) rc = prec_refresh(P);
  if (rc != BO_OK) {
    bo_prec_destroy(P);
    return rc;
  }
  *out = P;
  return BO_OK;
}

int bo_prec_update(bo_prec* P) {
  if (!P) return BO_ERR_ARG;
  return prec_refresh(P);
}

int bo_prec_apply(bo_prec* P, int stage, const double* r, double* z) {
  if (!P || !r || !z || stage < BO_STAGE_CPR || stage > BO_STAGE_ARNOLDI_SPMV) return BO_ERR_ARG;
  cudaStream_t s = P->stream;
  const Geom& g = P->mat->g;
  cudaMemsetAsync(&P->st->done, 0, sizeof(int), s);
  launch_gather(g, r, P->bi, s);
  if (stage == BO_STAGE_ARNOLDI_SPMV) {
    launch_arnoldi_product(P, P->bi, P->xi);
    launch_scatter(g, P->xi, z, s);
    return cuda_status(cudaStreamSynchronize(s));
  }
  // r -> internal (bi), apply, z (precision T) -> FP64 internal -> natural
  launch_cpr(P, P->bi, P->Z, stage, P->st);
  launch_scatter(g, P->Z, z, s);
  return cuda_status(cudaStreamSynchronize(s));
}

int bo_prec_spmv_decoupled(bo_prec* P, const double* x, double* y) {
  if (!P || !x || !y) return BO_ERR_ARG;
  cudaStream_t s = P->stream;
  const Geom& g = P->mat->g;
  launch_gather(g, x, P->bi, s);
  launch_spmv_decoupled_internal(P, P->bi, P->xi);
  launch_scatter(g, P->xi, y, s);
  return cuda_status(cudaStreamSynchronize(s));
}

int bo_prec_amg_levels(bo_prec* P, int32_t* dims, int cap) {
  if (!P) return BO_ERR_ARG;
  for (int l = 0; l < P->nlev && l < cap && dims; ++l) {
    if (l == 0) {
      dims[0] = P->mat->g.nx; dims[1] = P->mat->g.ny; dims[2] = P->mat->g.nz;
    } else {
      dims[3 * l] = P->lev[l].nx; dims[3 * l + 1] = P->lev[l].ny; dims[3 * l + 2] = P->lev[l].nz;
    }
  }
  return P->nlev;
}

int bo_prec_destroy(bo_prec* P) {
  if (!P) return BO_ERR_ARG;
  cudaStreamSynchronize(P->stream);
  prec_free(P);
  auto fr = [](void* p) { if (p) cudaFree(p); };
  fr(P->V); fr(P->Vs); fr(P->Z); fr(P->H); fr(P->cs); fr(P->sn); fr(P->gvec); fr(P->y);
  fr(P->xi); fr(P->bi); fr(P->rk); fr(P->partials); fr(P->hostio);
  if (P->h_st) cudaFreeHost(P->h_st);
  for (int e = 0; e < 4; ++e)
    if (P->ev[e]) cudaEventDestroy(P->ev[e]);
  if (P->prof_ready)
    for (int i = 0; i < 2 * 512; ++i) cudaEventDestroy(P->prof_ev[i]);
  delete[] P->hist;
  bo_mat* m = P->mat;
  delete P;
  mat_release(m);
  return BO_OK;
}

int bo_solve(bo_prec* P, const double* b, double* x, const bo_solve_opts* opts, bo_solve_info* info) {
  if (!P || !b || !x) return BO_ERR_ARG;
  bo_solve_opts o;
  bo_solve_opts_default(&o);
  if (opts) o = *opts;
  if (!(o.tol > 0.0) || o.restart < 1 || o.restart > 64 || o.maxit < 0 ||
      (o.mem != BO_MEM_HOST && o.mem != BO_MEM_DEVICE))
    return BO_ERR_ARG;
  if (cudaSetDevice(P->mat->ctx->device) != cudaSuccess) return BO_ERR_CUDA;
  return fgmres(P, b, x, &o, info);
}

int bo_solve_bicgstab(bo_prec* P, const double* b, double* x, const bo_solve_opts* opts, bo_solve_info* info) {
  if (!P || !b || !x) return BO_ERR_ARG;
  bo_solve_opts o;
  bo_solve_opts_default(&o);
  if (opts) o = *opts;
  if (!(o.tol > 0.0) || o.maxit < 0 || (o.mem != BO_MEM_HOST && o.mem != BO_MEM_DEVICE)) return BO_ERR_ARG;
  if (o.restart < 1 || o.restart > 64) o.restart = 30;  // sizes the shared workspace only
  if (cudaSetDevice(P->mat->ctx->device) != cudaSuccess) return BO_ERR_CUDA;
  return bicgstab(P, b, x, &o, info);
}

int bo_solve_batched(bo_prec* const* P, int nreal, const double* const* b, double* const* x,
                     const bo_solve_opts* opts, bo_solve_info* infos) {
  if (!P || !b || !x || nreal < 1) return BO_ERR_ARG;
  bo_solve_opts o;
  bo_solve_opts_default(&o);
  if (opts) o = *opts;
  if (!(o.tol > 0.0) || o.restart < 1 || o.restart > 64 || o.maxit < 0 ||
      (o.mem != BO_MEM_HOST && o.mem != BO_MEM_DEVICE))
    return BO_ERR_ARG;
  const int dev = P[0] ? P[0]->mat->ctx->device : -1;
  for (int r = 0; r < nreal; ++r) {
    if (!P[r] || !b[r] || !x[r] || P[r]->mat->ctx->device != dev) return BO_ERR_ARG;
    for (int q = 0; q < r; ++q)
      if (P[q] == P[r]) return BO_ERR_ARG;  // each solve needs its own workspace
  }
  return bo::solve_batched(P, nreal, b, x, o, infos, nullptr);
}

int bo_update_batched(bo_prec* const* P, int nreal, const double* const* val, int mem) {
  if (!P || nreal < 1 || (mem != BO_MEM_HOST && mem != BO_MEM_DEVICE)) return BO_ERR_ARG;
  const int dev = P[0] ? P[0]->mat->ctx->device : -1;
  for (int r = 0; r < nreal; ++r) {
    if (!P[r] || P[r]->mat->ctx->device != dev) return BO_ERR_ARG;
    for (int q = 0; q < r; ++q)
      if (P[q] == P[r] || P[q]->mat == P[r]->mat) return BO_ERR_ARG;
  }
  if (cudaSetDevice(dev) != cudaSuccess) return BO_ERR_CUDA;
  std::vector<cudaStream_t> pool;
  if (!stream_pool(dev, pool)) return BO_ERR_CUDA;
  const int width = std::min(kMaxPoolStreams, std::max(1, g_pool_width.load()));
  const int S = nreal < width ? nreal : width;
  int* hflags = nullptr;
  if (cudaMallocHost(&hflags, 2 * (size_t)nreal * sizeof(int)) != cudaSuccess) return BO_ERR_OOM;
  std::vector<cudaEvent_t> evs;
  auto join = [&](cudaStream_t from, cudaStream_t to) {
    cudaEvent_t e;
    cudaEventCreateWithFlags(&e, cudaEventDisableTiming);
    cudaEventRecord(e, from);
    cudaStreamWaitEvent(to, e, 0);
    evs.push_back(e);
  };
  int rc = BO_OK;
  for (int r = 0; r < nreal && rc == BO_OK; ++r) {
    bo_prec* p = P[r];
    bo_mat* m = p->mat;
    cudaStream_t s = pool[r % S];
    join(m->ctx->stream, s);
    p->stream = s;
    cudaMemsetAsync(&p->st->err, 0, sizeof(int), s);
    if (val && val[r]) {
      const double* dval = val[r];
      const size_t bytes = (m->kind == 0 ? 9 * (size_t)m->nnz : (size_t)m->nnz) * sizeof(double);
      if (mem == BO_MEM_HOST) {
        if (cudaMemcpyAsync(m->stage, val[r], bytes, cudaMemcpyHostToDevice, s) != cudaSuccess) rc = BO_ERR_CUDA;
        dval = m->stage;
      }
      if (rc == BO_OK) rc = m->kind == 0 ? ingest_bsr(m, dval, s) : ingest_csr(m, dval, s);
      m->a32_valid = false;
      m->a16_valid = false;
    }
    if (rc == BO_OK) rc = prec_values(p);
    cudaMemcpyAsync(&hflags[2 * r], m->flags, sizeof(int), cudaMemcpyDeviceToHost, s);
    cudaMemcpyAsync(&hflags[2 * r + 1], &p->st->err, sizeof(int), cudaMemcpyDeviceToHost, s);
    cudaMemsetAsync(m->flags, 0, sizeof(int), s);
    cudaMemsetAsync(&p->st->err, 0, sizeof(int), s);
    cudaMemsetAsync(&p->st->done, 0, sizeof(int), s);
  }
  for (int r = 0; r < nreal; ++r) {
    join(P[r]->stream, P[r]->mat->ctx->stream);
    P[r]->stream = P[r]->mat->ctx->stream;
  }
  for (int r = 0; r < S; ++r)
    if (cudaStreamSynchronize(pool[r]) != cudaSuccess) rc = BO_ERR_CUDA;
  for (auto e : evs) cudaEventDestroy(e);
  for (int r = 0; r < nreal && rc == BO_OK; ++r) {
    const int f = hflags[2 * r] | hflags[2 * r + 1];
    if (f & kErrPattern) rc = BO_ERR_PATTERN;
    else if (f & kErrNonfinite) rc = BO_ERR_NONFINITE;
    else if (f & kErrBreakdown) rc = BO_ERR_BREAKDOWN;
  }
  cudaFreeHost(hflags);
  return rc;
}

int bo_prec_residual_history(bo_prec* P, double* buf, int cap) {
  if (!P || (!buf && cap > 0)) return BO_ERR_ARG;
  const int n = P->nhist < cap ? P->nhist : cap;
  for (int i = 0; i < n; ++i) buf[i] = P->hist[i];
  return n;
}

int64_t bo_kernel_launches(void) { return g_launches.load(); }

int bo_set_amg_cooperative(int on) {
  if (on < 0 || on > 2) return BO_ERR_ARG;
  g_amg_coop.store(on);
  return BO_OK;
}

int bo_set_amg_barrier_spins(uint32_t spins) {
  g_amg_spins.store(spins == 0 ? kAmgSpinsDefault : spins);
  return BO_OK;
}

int bo_set_gs_fused(int on) {
  if (on != 0 && on != 1) return BO_ERR_ARG;
  g_gs_fused.store(on);
  return BO_OK;
}

int bo_set_conv_engine(int engine) {
  if (engine != 0 && engine != 1) return BO_ERR_ARG;
  g_conv_engine.store(engine);
  return BO_OK;
}

int bo_prec_set_launch_mode(bo_prec* P, int mode) {
  if (!P || (mode != BO_LAUNCH_STREAM && mode != BO_LAUNCH_GRAPH && mode != BO_LAUNCH_BATCH_GRAPH)) return BO_ERR_ARG;
  P->launch_mode = mode;
  return BO_OK;
}

int bo_prec_set_amg_tile(bo_prec* P, int cells, int threads) {
  if (!P || (cells != 1 && cells != 2 && cells != 4) || (threads != 128 && threads != 256 && threads != 512))
    return BO_ERR_ARG;
  if (P->amg_cells != cells || P->amg_threads != threads) {
    P->amg_cells = cells;
    P->amg_threads = threads;
    graphs_reset(P);  // captured columns hold the old launch shapes
  }
  return BO_OK;
}

int bo_newton_update(bo_ctx* ctx, double* state, const double* dx, int64_t n) {
  if (!ctx || !state || !dx || n < 0) return BO_ERR_ARG;
  launch_newton_update(state, dx, n, ctx->stream);
  return cuda_status(cudaGetLastError());
}

}  // extern "C"
