// bo_mat_residual_noalloc: the residual r = b - A x and the norms
// ||r||_2, ||b||_2 of a matrix the caller already created, computed without
// allocating any device memory during the call.
//
// Who needs this: code that must not call cudaMalloc at the point where it
// checks a residual.  A framework's caching allocator may already hold
// nearly all device memory, so a raw cudaMalloc fails there; cudaMalloc and
// cudaFree also synchronise the whole device, which a serving loop or a
// real-time caller that only allocates at start-up cannot afford.  The
// solver's own reductions keep their partial sums in memory owned by a
// preconditioner; this entry point keeps them in a fixed array compiled into
// the library instead.
//
// The scratch array below is a file-scope __device__ variable: every GPU
// that loads the library holds it (256 KB plus a counter) until the process
// exits, and all calls on one device share it.  Its size fixes the largest
// grid a call accepts: one block of 256 cells per partial sum pair, at most
// kNaMaxBlocks blocks, i.e. 4,194,304 cells; larger matrices get BO_ERR_ARG.
// Calls that overlap on the GPU (on different streams at the same time)
// race on the shared array and give wrong sums; the ticket counter is
// cleared on the caller's stream at the start of every call.
#include <mutex>

#include "bo_internal.cuh"

namespace bo {
namespace {

constexpr int kNaThreads = 256;
constexpr int kNaMaxBlocks = 16384;
constexpr int kNaMaxDevices = 64;

// two partial sums per block (||r||^2, ||b||^2), then the ticket counter
static __device__ __align__(256) double g_na_scratch[2 * kNaMaxBlocks + 32];

double* g_na_ptr[kNaMaxDevices];
cudaError_t g_na_rc[kNaMaxDevices];
std::once_flag g_na_once[kNaMaxDevices];

// One thread per cell (natural order); one pair of partial sums per block,
// summed in a fixed order by the block that finishes last.
__global__ void __launch_bounds__(kNaThreads) k_residual_noalloc(Geom g, const double* __restrict__ A,
                                                                const double* __restrict__ b,
                                                                const double* __restrict__ x,
                                                                double* __restrict__ r, double* scratch,
                                                                double* __restrict__ out) {
  __shared__ double sh[32];
  const int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  double rr = 0.0, bb = 0.0;
  if (c < g.N) {
    const Nat n = decode_nat(g, c);
    const unsigned valid = valid_slots(g, n);
    double a0 = 0.0, a1 = 0.0, a2 = 0.0;
#pragma unroll
    for (int s = 0; s < 7; ++s) {
      if (!((valid >> s) & 1u)) continue;
      const int64_t nc = c + nat_offset(g, s);
      const double x0 = x[3 * nc], x1 = x[3 * nc + 1], x2 = x[3 * nc + 2];
      const double* a = A + plane(g, n.color, s, 0) + n.q;
      const size_t P = (size_t)g.Nh;
      a0 += a[0] * x0 + a[P] * x1 + a[2 * P] * x2;
      a1 += a[3 * P] * x0 + a[4 * P] * x1 + a[5 * P] * x2;
      a2 += a[6 * P] * x0 + a[7 * P] * x1 + a[8 * P] * x2;
    }
    const double b0 = b[3 * c], b1 = b[3 * c + 1], b2 = b[3 * c + 2];
    const double r0 = b0 - a0, r1 = b1 - a1, r2 = b2 - a2;
    r[3 * c] = r0;
    r[3 * c + 1] = r1;
    r[3 * c + 2] = r2;
    rr = r0 * r0 + r1 * r1 + r2 * r2;
    bb = b0 * b0 + b1 * b1 + b2 * b2;
  }
  rr = block_sum(rr, sh);
  bb = block_sum(bb, sh);
  if (threadIdx.x == 0) {
    scratch[2 * blockIdx.x] = rr;
    scratch[2 * blockIdx.x + 1] = bb;
  }
  unsigned* counter = reinterpret_cast<unsigned*>(scratch + 2 * kNaMaxBlocks);
  if (last_block(counter, gridDim.x)) {
    double sr = 0.0, sb = 0.0;
    for (int i = threadIdx.x; i < (int)gridDim.x; i += blockDim.x) {
      sr += __ldcg(scratch + 2 * i);
      sb += __ldcg(scratch + 2 * i + 1);
    }
    sr = block_sum(sr, sh);
    sb = block_sum(sb, sh);
    if (threadIdx.x == 0) {
      out[0] = sqrt(sr);
      out[1] = sqrt(sb);
      *counter = 0u;
    }
  }
}

}  // namespace
}  // namespace bo

extern "C" int bo_mat_residual_noalloc(bo_mat* m, const double* b, const double* x, double* r, double* norms) {
  using namespace bo;
  if (!m || !b || !x || !r || !norms) return BO_ERR_ARG;
  // r is written while other threads still read b and x (x at six
  // neighbours): it must not overlap either of them
  const size_t bytes = (size_t)3 * (size_t)m->g.N * sizeof(double);
  auto overlap = [bytes](const void* p, const void* q) {
    const char* a = (const char*)p;
    const char* c = (const char*)q;
    return a < c + bytes && c < a + bytes;
  };
  if (overlap(r, x) || overlap(r, b)) return BO_ERR_ARG;
  const int64_t blocks = (m->g.N + kNaThreads - 1) / kNaThreads;
  if (blocks > kNaMaxBlocks) return BO_ERR_ARG;  // more than 4,194,304 cells
  const int dev = m->ctx->device;
  if (dev < 0 || dev >= kNaMaxDevices) return BO_ERR_ARG;
  // once per device, with that device current: the device address of the
  // scratch array (a host-side reference to the symbol is not a device address)
  std::call_once(g_na_once[dev], [dev]() {
    int prev = 0;
    cudaGetDevice(&prev);
    cudaError_t e = cudaSetDevice(dev);
    if (e == cudaSuccess) e = cudaGetSymbolAddress((void**)&g_na_ptr[dev], g_na_scratch);
    g_na_rc[dev] = e;
    cudaSetDevice(prev);
  });
  if (g_na_rc[dev] != cudaSuccess || !g_na_ptr[dev]) return BO_ERR_CUDA;
  if (cudaSetDevice(dev) != cudaSuccess) return BO_ERR_CUDA;
  cudaStream_t s = m->ctx->stream;
  double* scratch = g_na_ptr[dev];
  // the ticket counter must start at zero
  if (cudaMemsetAsync(scratch + 2 * kNaMaxBlocks, 0, sizeof(unsigned), s) != cudaSuccess) return BO_ERR_CUDA;
  (k_residual_noalloc<<<(unsigned)blocks, kNaThreads, 0, s>>>(m->g, m->A, b, x, r, scratch, norms), note_launch());
  return cudaGetLastError() == cudaSuccess ? BO_OK : BO_ERR_CUDA;
}
