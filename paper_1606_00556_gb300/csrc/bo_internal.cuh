// Internal declarations shared by the solver's translation units.
//
// Data layout in HBM ("colour-split structured BSR").  Cells are split into
// the two colours of the 7-point graph, red ((i + j + k) even) and black.
// With nx even, cell c has half index q = c >> 1 inside its colour, and the
// half indices of each colour run over [0, N/2).  All six neighbours of a
// cell have the other colour, so every operation that the red-black block
// ILU(0) and the Gauss-Seidel smoother run on one colour touches contiguous
// memory.
//   matrix values: plane (colour, slot, rc) is an array of N/2 scalars,
//       offset ((colour * 7 + slot) * 9 + rc) * N/2; slot is the stencil
//       position (-z, -y, -x, diag, +x, +y, +z), rc = 3 * row + column of
//       the 3x3 block.  Blocks whose neighbour lies outside the grid hold 0.
//   vectors (internal): entry (component, colour, q) at
//       component * N + colour * N/2 + q, i.e. the pressure component of
//       all cells first (red half, black half), then Sw, then Sg.
// Column indices are implied by the stencil and never stored.
#pragma once

#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <cstdint>
#include <cstddef>
#include <atomic>
#include <vector>

#include "bosolve.h"

namespace bo {

constexpr int kThreads = 256;

enum Slot { kZm = 0, kYm = 1, kXm = 2, kDiag = 3, kXp = 4, kYp = 5, kZp = 6 };

// error bits written by device kernels
enum : int { kErrPattern = 1, kErrNonfinite = 2, kErrBreakdown = 4, kErrTimeout = 8 };

struct Geom {
  int32_t nx, ny, nz, hx;
  int64_t N, Nh;
};

struct Cell {
  int32_t i, j, k, s;  // s: parity of i (the position of the cell inside its half-index pair)
};

__host__ __device__ __forceinline__ int opposite(int slot) { return 6 - slot; }

// (half indices are below 2^31 for any grid that fits one GPU: 32-bit
// division is several times cheaper than 64-bit)
__device__ __forceinline__ Cell decode(const Geom& g, int color, int64_t q) {
  const uint32_t qu = (uint32_t)q, hx = (uint32_t)g.hx, ny = (uint32_t)g.ny;
  const uint32_t r = qu / hx;
  const int32_t ih = (int32_t)(qu - r * hx);
  const int32_t j = (int32_t)(r % ny);
  const int32_t k = (int32_t)(r / ny);
  const int32_t s = (color ^ j ^ k) & 1;
  return Cell{2 * ih + s, j, k, s};
}

// Half index (in the neighbour's colour) of the neighbour at `slot`, or -1
// when it lies outside the grid.  slot is a compile-time constant after
// unrolling, so the switch folds away.
__device__ __forceinline__ int64_t nbr(const Geom& g, const Cell& c, int64_t q, int slot) {
  switch (slot) {
    case kZm: return c.k > 0 ? q - (int64_t)g.hx * g.ny : -1;
    case kYm: return c.j > 0 ? q - g.hx : -1;
    case kXm: return c.i > 0 ? q - 1 + c.s : -1;
    case kDiag: return q;
    case kXp: return c.i < g.nx - 1 ? q + c.s : -1;
    case kYp: return c.j < g.ny - 1 ? q + g.hx : -1;
    default: return c.k < g.nz - 1 ? q + (int64_t)g.hx * g.ny : -1;
  }
}

// A cell in natural order c = i + nx (j + ny k): its coordinates, colour
// and half index.  Kernels that read or write the caller's natural-order
// vectors (ingest, the public SpMV, the allocation-free residual) decode
// cells with these helpers, so the natural-to-colour-plane mapping is
// written once.
struct Nat {
  int32_t i, j, k;
  int color;
  int64_t q;
};

__device__ __forceinline__ Nat decode_nat(const Geom& g, int64_t c) {
  const int64_t r = c / g.nx;
  Nat n;
  n.i = (int32_t)(c - r * g.nx);
  n.j = (int32_t)(r % g.ny);
  n.k = (int32_t)(r / g.ny);
  n.color = (n.i + n.j + n.k) & 1;
  n.q = c >> 1;
  return n;
}

// stencil slot of column offset d for a cell at (i, j, k), or -1
__device__ __forceinline__ int slot_of(const Geom& g, const Nat& n, int64_t d) {
  const int64_t nxy = (int64_t)g.nx * g.ny;
  if (d == 0) return kDiag;
  if (d == -1 && n.i > 0) return kXm;
  if (d == 1 && n.i < g.nx - 1) return kXp;
  if (d == -nxy && n.k > 0) return kZm;
  if (d == nxy && n.k < g.nz - 1) return kZp;
  if (d == -(int64_t)g.nx && n.j > 0) return kYm;
  if (d == (int64_t)g.nx && n.j < g.ny - 1) return kYp;
  return -1;
}

__device__ __forceinline__ unsigned valid_slots(const Geom& g, const Nat& n) {
  unsigned m = 1u << kDiag;
  if (n.k > 0) m |= 1u << kZm;
  if (n.j > 0) m |= 1u << kYm;
  if (n.i > 0) m |= 1u << kXm;
  if (n.i < g.nx - 1) m |= 1u << kXp;
  if (n.j < g.ny - 1) m |= 1u << kYp;
  if (n.k < g.nz - 1) m |= 1u << kZp;
  return m;
}

// natural-order offset c' - c of the neighbour at `slot`
__device__ __forceinline__ int64_t nat_offset(const Geom& g, int slot) {
  const int64_t nxy = (int64_t)g.nx * g.ny;
  switch (slot) {
    case kZm: return -nxy;
    case kYm: return -(int64_t)g.nx;
    case kXm: return -1;
    case kDiag: return 0;
    case kXp: return 1;
    case kYp: return (int64_t)g.nx;
    default: return nxy;
  }
}

__host__ __device__ __forceinline__ size_t plane(const Geom& g, int color, int slot, int rc) {
  return ((size_t)(color * 7 + slot) * 9 + rc) * (size_t)g.Nh;
}

__host__ __device__ __forceinline__ size_t vidx(const Geom& g, int comp, int color, int64_t q) {
  return (size_t)comp * (size_t)g.N + (size_t)color * (size_t)g.Nh + (size_t)q;
}

// Split copy of the matrix (A2, read by the Arnoldi product) in a tiled
// layout: the 63 values of 32 consecutive half indices of one colour form a
// contiguous 16 KB tile, [colour][q / 32][slot * 9 + rc][q % 32], so the 63
// loads of a warp stream one contiguous region instead of 63 planes.
__host__ __device__ __forceinline__ int64_t a2_tiles(const Geom& g) { return (g.Nh + 31) / 32; }
__host__ __device__ __forceinline__ size_t a2_size(const Geom& g) { return (size_t)2 * a2_tiles(g) * 63 * 32; }
__host__ __device__ __forceinline__ size_t a2_index(const Geom& g, int color, int v, int64_t q) {
  return (((size_t)color * a2_tiles(g) + (size_t)(q >> 5)) * 63 + (size_t)v) * 32 + (size_t)(q & 31);
}

// The decoupled matrix of the preconditioner uses the same tiles (its
// kernels read a block's entries 32 apart).
__host__ __device__ __forceinline__ size_t at_index(const Geom& g, int color, int v, int64_t q) {
  return a2_index(g, color, v, q);
}

// streaming (evict-first) loads for matrix values that are read once per pass
__device__ __forceinline__ double ld_stream(const double* p) { return __ldcs(p); }
__device__ __forceinline__ float ld_stream(const float* p) { return __ldcs(p); }
__device__ __forceinline__ __nv_bfloat16 ld_stream(const __nv_bfloat16* p) {
  return __ushort_as_bfloat16(__ldcs(reinterpret_cast<const unsigned short*>(p)));
}

// acc + a0 x0 + a1 x1 + a2 x2 as a chain of three fused multiply-adds (one
// FP64 instruction per product: the FP64 kernels are bound by FP64 issue)
__device__ __forceinline__ double fma3(double acc, double a0, double x0, double a1, double x1, double a2, double x2) {
  return fma(a2, x2, fma(a1, x1, fma(a0, x0, acc)));
}
__device__ __forceinline__ float fma3(float acc, float a0, float x0, float a1, float x1, float a2, float x2) {
  return fmaf(a2, x2, fmaf(a1, x1, fmaf(a0, x0, acc)));
}

// ---- split FP32 pairs for the Krylov vectors and the Arnoldi product
// A value is the unevaluated sum hi + lo of two floats with |lo| below one
// ulp of hi (Dekker's double-length arithmetic, Numer. Math. 18, 1971):
// about 48 significant bits (2^-46 relative) with FP32's exponent range.
// The error-free transformations are Knuth's TwoSum and the FMA form of
// Dekker's TwoProduct.  GB300 issues 128 FP32 operations per clock per SM
// against about 2 FP64 FMAs, so a split multiply-add (about 12 FP32
// operations) is several times cheaper than one FP64 FMA, and the kernels
// built from it (the Arnoldi product, the black ILU pivots of a
// reduced-precision preconditioner) are bound by memory instead of the FP64
// pipe.  The _rn intrinsics are never contracted into FMAs, which the
// transformations rely on.
struct df {
  float hi, lo;
};

__device__ __forceinline__ df df_two_sum(float a, float b) {
  const float s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  const float e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
  return df{s, e};
}
// |a| >= |b| (or a == 0)
__device__ __forceinline__ df df_fast_two_sum(float a, float b) {
  const float s = __fadd_rn(a, b);
  return df{s, __fsub_rn(b, __fsub_rn(s, a))};
}
__device__ __forceinline__ df df_add(df a, df b) {
  const df s = df_two_sum(a.hi, b.hi);
  return df_fast_two_sum(s.hi, __fadd_rn(s.lo, __fadd_rn(a.lo, b.lo)));
}
__device__ __forceinline__ df df_neg(df a) { return df{-a.hi, -a.lo}; }
// acc + a b for a long sum: the low parts of the products and of the
// running sum collect in acc.lo without renormalising each step (the sum is
// renormalised once, by df_norm, before it is used)
__device__ __forceinline__ df df_fma_acc(df acc, df a, df b) {
  const float p = __fmul_rn(a.hi, b.hi);
  float pe = __fmaf_rn(a.hi, b.hi, -p);
  pe = __fmaf_rn(a.hi, b.lo, __fmaf_rn(a.lo, b.hi, pe));
  const df s = df_two_sum(acc.hi, p);
  return df{s.hi, __fadd_rn(acc.lo, __fadd_rn(s.lo, pe))};
}
__device__ __forceinline__ df df_norm(df a) { return df_fast_two_sum(a.hi, a.lo); }
// the same with no assumption on the magnitudes (after a sum whose high
// parts cancelled below the accumulated low parts)
__device__ __forceinline__ df df_renorm(df a) { return df_two_sum(a.hi, a.lo); }
__device__ __forceinline__ df df_from(double v) {
  const float h = __double2float_rn(v);
  return df{h, __double2float_rn(v - (double)h)};
}
__device__ __forceinline__ double df_to_double(df a) { return (double)a.hi + (double)a.lo; }
// The leading 24 significant bits of a as a float (truncated), by integer
// operations on the bit pattern: no FP64 instruction.  Magnitudes beyond
// FP32's normal range go to 0 or +-FLT_MAX.
__device__ __forceinline__ float df_hi_bits(double a) {
  const unsigned long long u = (unsigned long long)__double_as_longlong(a);
  const unsigned sign = (unsigned)(u >> 32) & 0x80000000u;
  const int e = (int)((u >> 52) & 0x7ff) - 1023;
  if (e < -126) return __uint_as_float(sign);
  if (e > 127) return __uint_as_float(sign | 0x7f7fffffu);
  return __uint_as_float(sign | ((unsigned)(e + 127) << 23) | (unsigned)((u >> 29) & 0x7fffffu));
}

// The same split by integer operations on the bit pattern (no FP64
// instruction): hi keeps the leading 24 significant bits, lo the next 24
// (both truncated), so |a - hi - lo| < 2^-46 |a|.  Below 2^-74 the low part
// would be subnormal and is dropped; *bad is set where |a| > 2^126 or
// 0 < |a| < 2^-120 (outside what the split form represents) or a is not
// finite.
__device__ __forceinline__ float2 df_split_bits(double a, int* bad) {
  const unsigned long long u = (unsigned long long)__double_as_longlong(a);
  const unsigned sign = (unsigned)(u >> 32) & 0x80000000u;
  const int E = (int)((u >> 52) & 0x7ff);
  const unsigned long long M = u & 0xFFFFFFFFFFFFFull;
  if (E == 0) {
    *bad |= (M != 0);
    return make_float2(__uint_as_float(sign), __uint_as_float(sign));
  }
  const int e = E - 1023;
  if (e > 126 || e < -120) {
    *bad = 1;
    return make_float2(__double2float_rn(a), 0.f);
  }
  const float hi = __uint_as_float(sign | ((unsigned)(e + 127) << 23) | (unsigned)(M >> 29));
  const unsigned R = (unsigned)(M & 0x1FFFFFFFu);
  const int lz = __clz(R);
  const int fe = e - 52 + (31 - lz) + 127;
  if (R == 0 || fe < 1) return make_float2(hi, __uint_as_float(sign));
  const unsigned mant = (unsigned)((((unsigned long long)R) << (lz + 1)) & 0xFFFFFFFFull) >> 9;
  return make_float2(hi, __uint_as_float(sign | ((unsigned)fe << 23) | mant));
}

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Sum over the thread block in a fixed order; the result is valid in every
// thread.  `sh` must hold 32 doubles of shared memory.
__device__ __forceinline__ double block_sum(double v, double* sh) {
  v = warp_sum(v);
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  __syncthreads();
  if (l == 0) sh[w] = v;
  __syncthreads();
  const int nw = (blockDim.x + 31) >> 5;
  v = l < nw ? sh[l] : 0.0;
  return warp_sum(v);
}

// A preconditioner input or output vector of 3N entries in internal order:
// FP64 (d) or split pairs (f: hi plane, then the lo plane at f + n).
struct InV {
  const double* d;
  const float* f;
  int64_t n;
};
struct OutV {
  double* d;
  float* f;
  int64_t n;
};

// Ticket of the "last block done" pattern: true in the block that finished
// last among `total`.  Partials written before the call are visible to it.
__device__ __forceinline__ bool last_block(unsigned* counter, unsigned total) {
  __shared__ unsigned ticket;
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) ticket = atomicAdd(counter, 1u);
  __syncthreads();
  return ticket == total - 1;
}

// Device-side state of one preconditioner / solve.  Lives in device memory.
struct DevState {
  int done;        // stop the current FGMRES cycle (device side early exit)
  int k;           // Arnoldi steps completed in the current cycle
  int happy;       // happy breakdown in the current cycle
  int err;         // kErr* bits from setup and apply kernels
  int hist_base;   // Arnoldi steps of the finished cycles of this solve (residual-history offset)
  unsigned counter[8];
  double est;      // Arnoldi estimate of ||b - A x|| after k steps
  double target;   // tol * ||b||
  double beta;     // ||r|| from the last true residual
  double bnorm;    // ||b||
  double wn0;      // ||w|| before orthogonalisation
  double hn;       // ||w|| after orthogonalisation
  double scale;    // 1 / h_{j+1,j}: normalisation of the new basis vector
  double vscale[72];  // 1 / ||V_k|| of the unnormalised basis vectors
  double h[136];   // Gram-Schmidt coefficients of the column under construction: pass 1 at 0, pass 2 at 64
};

// Number of kernels this library has launched (reported by bo_kernel_launches).
extern std::atomic<long long> g_launches;
// streams of the batched solve's pool in use (1..kMaxPoolStreams)
constexpr int kMaxPoolStreams = 16;
extern std::atomic<int> g_pool_width;
// convolution engine of the 32 -> 32 layers: 0 mma.sync, 1 tcgen05 (conv_tc.cu)
extern std::atomic<int> g_conv_engine;
// AMG launch form: 2 (default) cooperative legs for levels 0-1 around a cluster
// launch for the coarser levels, 1 cooperative legs for every multi-block
// level around a one-block tail, 0 one kernel per sweep
extern std::atomic<int> g_amg_coop;
// polls of an AMG grid barrier before it gives up (default 2^22, about 0.1 s)
constexpr unsigned kAmgSpinsDefault = 1u << 22;
extern std::atomic<unsigned> g_amg_spins;
// Gram-Schmidt form: 1 (default) three passes (first update fused with the
// second coefficients), 0 four separate passes
extern std::atomic<int> g_gs_fused;
inline void note_launch() { g_launches.fetch_add(1, std::memory_order_relaxed); }

// Programmatic dependent launch.  The solver's kernels are launched with
// launch_pdl, which lets a kernel be scheduled as soon as every block of the
// kernel before it on the stream has finished, without waiting for that
// kernel's completion to be processed (about 1.5-2.7 us saved per kernel
// boundary, measured on GB300 for 16 MB streaming kernels).  Every such
// kernel calls wait_prior_grid() before its first memory access: it returns
// once the previous kernel has completed and its writes are visible (at
// once when the kernel was launched without the attribute).  No kernel
// triggers its dependents early, so a dependent never occupies an SM while
// its predecessor still runs.
__device__ __forceinline__ void wait_prior_grid() { asm volatile("griddepcontrol.wait;" ::: "memory"); }

template <typename... KArgs, typename... Args>
inline cudaError_t launch_pdl(void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t s,
                              Args&&... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  at[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, kernel, static_cast<KArgs>(args)...);
}

// grid size for a grid-stride loop over n items
inline int grid_for(int64_t n, int threads = kThreads, int max_blocks = 152 * 16) {
  int64_t b = (n + threads - 1) / threads;
  if (b < 1) b = 1;
  if (b > max_blocks) b = max_blocks;
  return (int)b;
}

// Grid for a grid-stride loop over n items of a kernel launched with
// kThreads threads: every SM gets as many blocks as can be resident at once
// (one full wave, no partial last wave), capped by the work available.
int occ_grid(const void* kernel, int64_t n, int threads = kThreads, size_t smem = 0);

}  // namespace bo

// ----------------------------------------------------------------- objects
// Contexts and matrices are reference counted: a matrix holds its context
// and a preconditioner holds its matrix, so destroying them in any order is
// safe (the object is freed when its last holder lets go).
struct bo_ctx {
  int device;
  cudaStream_t stream;
  bool own_stream;
  int refs;
};

struct bo_mat {
  bo_ctx* ctx;
  int refs;
  bo_grid grid;
  bo::Geom g;
  int kind;            // 0 BSR, 1 CSR
  int64_t nnz;         // blocks (BSR) or scalars (CSR)
  int32_t* rowptr;     // device copy of the pattern
  int32_t* col;
  double* stage;       // device staging of values passed from the host
  double* A;           // 63 N FP64 values, colour-split planes
  float* A32;          // FP32 copy for bo_mat_spmv(..., BO_PREC_FP32), tiled (a2_index)
  bool a32_valid;
  __nv_bfloat16* A16;  // BF16 copy for bo_mat_spmv(..., BO_PREC_BF16), tiled (a2_index)
  bool a16_valid;
  float2* A2;          // split (hi, lo) copy of A for the Arnoldi product, tiled (a2_index)
  bool a2_valid;
  int* a2_range;       // device flag: a value lies outside the split form's range
  int* flags;          // device error bits
  int* h_flags;        // pinned host copy
};

namespace bo {

// one AMG level stored in natural cell order (levels >= 1)
struct Level {
  int32_t nx, ny, nz;
  int64_t n;
  double* c64;   // 7 n FP64 coefficients [slot][cell] (setup master)
  void* c;       // 7 n coefficients in the preconditioner precision
  void* f;       // n right-hand side
  void* x;       // n iterate
};

}  // namespace bo

struct bo_wells;

struct bo_prec {
  bo_mat* mat;
  cudaStream_t stream;     // stream of all preconditioner work (the context's, or a batch stream)
  bo_prec_opts opts;
  bool fp32;               // preconditioner arithmetic FP32 (else FP64)
  size_t tsize;            // sizeof(preconditioner vector scalar / arithmetic)
  size_t ssize;            // sizeof(stored matrix, pivot and AMG coefficient)
  bool bf16;               // BF16 storage of those (arithmetic FP32)
  void* At;                // 63 N decoupled values (preconditioner precision), tiled (at_index)
  double* w;               // 3 N decoupling weights (g0, g1, g2) of row 0, [3][N] internal order
  float* wf;               // the same weights rounded to FP32 (FP32 arithmetic), else NULL
  void* Dinv;              // 9 N inverted ILU pivot blocks [rc][N], preconditioner precision
  // AMG: level 0 = the pressure block of At (colour-split), levels 1.. natural order
  int nlev;
  bo::Level lev[24];
  int tail_from;           // first level handled by the single-block tail kernel
  double* coarse64;        // dense coarsest matrix / inverse workspace (FP64)
  void* coarse_inv;        // dense inverse of the coarsest level (precision T)
  int64_t ncoarse;
  // CPR work vectors (precision T, internal order)
  void* f;                 // 3N decoupled input
  void* t;                 // 3N ILU intermediates
  void* r;                 // 3N residual
  void* z1;                // 3N first local solve x1 = R^{-1} f
  void* e0;                // N level-0 AMG correction
  void* f0;                // N level-0 AMG right-hand side
  // Krylov workspace (FP64 unless noted)
  int mcap;                // restart length the workspace was sized for
  double* V;               // (mcap+1) 3N basis as split pairs (FGMRES; 8 bytes per entry), FP64 scratch otherwise
  float* Vs;               // unused (kept NULL)
  double* Z;               // mcap 3N preconditioned vectors as split pairs: per vector a hi plane, then a lo plane
  double* H;               // (mcap+1) mcap
  double* cs;
  double* sn;
  double* gvec;            // mcap+1
  double* y;               // mcap
  double* xi;              // 3N internal iterate
  double* bi;              // 3N internal right-hand side
  double* rk;              // 3N true residual
  double* partials;        // reduction partials
  int64_t npartials;
  double* hostio;          // device staging of host b / x
  bo::DevState* st;        // device state
  bo::DevState* h_st;      // pinned host mirror (three column slots, one phase slot)
  bo::DevState* h_st_dev;  // its device address (written by a kernel), or NULL
  cudaEvent_t ev[4];
  cudaEvent_t prof_ev[2 * 512];
  bool prof_ready;
  // learned coarse space (Z = tile restriction of a predicted dp)
  int lc_nt = 0;           // tiles (columns of Z); 0: off
  int lc_tile[3] = {0, 0, 0};
  int lc_ntile[3] = {0, 0, 0};
  double* lc_z = nullptr;  // dp, colour-split order
  double* lc_E = nullptr;  // Z^T A~_pp Z, nt x nt
  double* lc_Einv = nullptr;
  double* lc_y = nullptr;  // Z^T f
  double* lc_u = nullptr;  // E^{-1} Z^T f
  // CUDA-graph launch of the Arnoldi columns (BO_LAUNCH_GRAPH): one
  // instantiated graph per column index, captured for restart length graph_m
  int launch_mode = 0;
  int graph_m = 0;
  cudaStream_t cap_stream = nullptr;
  cudaGraphExec_t col_exec[64] = {};
  unsigned long long graph_gen = 0;  // bumped whenever captured graphs go stale
  // tile parameters of the per-kernel AMG form (the form inside captured
  // graphs): threads per block and level-0 Gauss-Seidel cells per thread
  int amg_threads = 256;
  int amg_cells = 1;
  long long col_nodes[64] = {};
  double* hist;            // host residual history of the last solve
  int nhist;
  int hist_cap;
  // preconditioner setups so far (values refreshed or coarse space changed):
  // state derived from this preconditioner checks it before reuse
  unsigned long long setups = 0;
  // rate-controlled wells of the bordered solve in progress (NULL otherwise),
  // and those the captured Arnoldi-column graphs were recorded with
  bo_wells* wl = nullptr;
  const bo_wells* graph_wl = nullptr;
};

// ----------------------------------------------------------------- launchers
namespace bo {

// layout.cu
int ingest_bsr(bo_mat* m, const double* dval, cudaStream_t s);
int ingest_csr(bo_mat* m, const double* dval, cudaStream_t s);
void launch_to_f32(const double* src, float* dst, size_t n, cudaStream_t s);
void launch_widen(const float* src, double* dst, size_t n, cudaStream_t s);
void launch_spmv_nat(const bo_mat* m, double alpha, const double* x, double beta, double* y, int precision);
// FP32 / BF16 copies of A in the tiled layout of the split copy (a2_size entries)
void launch_to_tiled_f32(const bo_mat* m, float* dst, cudaStream_t s);
void launch_to_tiled_bf16(const bo_mat* m, __nv_bfloat16* dst, cudaStream_t s);
void launch_to_bf16(const double* src, __nv_bfloat16* dst, size_t n, cudaStream_t s);
void launch_gather(const Geom& g, const double* nat, double* in, cudaStream_t s);
void launch_scatter(const Geom& g, const double* in, double* nat, cudaStream_t s);
void launch_newton_update(double* state, const double* dx, int64_t n, cudaStream_t s);

// precond.cu
int prec_values(bo_prec* P);   // decoupling + ILU + AMG values (stream-ordered, flags in st->err)
int prec_alloc(bo_prec* P);
void prec_free(bo_prec* P);
// z = stage(v * vs[0]) in internal order, FP64 in and out (vs may be NULL: scale 1)
void launch_cpr(bo_prec* P, const double* v, double* z, int stage, const DevState* st, const double* vs = nullptr);
// the CPR stage with its output as split pairs (FP64 basis vector in, preconditioned vector out)
void launch_cpr_split(bo_prec* P, const double* v, float* z, const DevState* st, const double* vs);
// the same with a split-pair input vector (an FGMRES basis vector)
void launch_cpr_split_in(bo_prec* P, const float* v, float* z, const DevState* st, const double* vs);
// A2 = split copy of A, flagging values outside FP32's normal range
void launch_split_matrix(bo_mat* m, cudaStream_t s);
void launch_spmv_decoupled_internal(bo_prec* P, const double* x, double* y);  // FP64 values of At rebuilt on the fly

// capi.cu: drop a reference on a context (frees it with the last one)
void ctx_release_ref(bo_ctx* c);

// krylov.cu
int fgmres(bo_prec* P, const double* b_nat, double* x_nat, const bo_solve_opts* o, bo_solve_info* info);
// wells.cu: the bordered solve's corrections inside FGMRES (P->wl set):
// after the preconditioner wrote z (split planes of n entries), after the
// Arnoldi product wrote w (split planes, low plane at w + np), and after the
// true residual of the iterate
void wells_after_prec(bo_prec* P, float* z, int64_t n);
void wells_after_product(bo_prec* P, float* w, int64_t np);
void wells_after_residual(bo_prec* P);
// capi.cu: drop a reference to a matrix
void mat_release_ref(bo_mat* m);
int bicgstab(bo_prec* P, const double* b_nat, double* x_nat, const bo_solve_opts* o, bo_solve_info* info);
// tols: per-system tolerances replacing o->tol (NULL: o->tol for all)
int fgmres_batched(bo_prec* const* P, int nreal, const double* const* b, double* const* x, const bo_solve_opts* o,
                   bo_solve_info* infos, const double* tols = nullptr);
// capi.cu: the batched solve on the stream pool (argument checks done)
int solve_batched(bo_prec* const* P, int nreal, const double* const* b, double* const* x, const bo_solve_opts& o,
                  bo_solve_info* infos, const double* tols);
int krylov_alloc(bo_prec* P, int m);
// w = A v (internal order, FP64 in and out) by the FGMRES Arnoldi product
// (split copy of A, v split into pairs; the FP64 planes where the split copy
// is out of range); uses P's first preconditioned vector and the first FP32
// shadow as scratch
void launch_arnoldi_product(bo_prec* P, const double* v, double* w);
void graphs_reset(bo_prec* P);
// tcgen05 convolution for 32 -> 32 layers; mode 0 ReLU, 1 ReLU + residual,
// 2 linear FP32 output.  BO_ERR_ARG where it does not apply.
int launch_conv_tc(int nx, int ny, int nz, int B, const __nv_bfloat16* X, const __nv_bfloat16* W, const float* bias,
                   const __nv_bfloat16* R, __nv_bfloat16* Y, float* Yf, int mode, cudaStream_t s);
// dense FP64 inverse of an n x n matrix (n <= 128) by one block; sets
// st->err on a zero pivot
int launch_dense_inverse64(int n, const double* M, double* Minv, DevState* st, cudaStream_t s);
int learned_coarse_values(bo_prec* P);
void learned_coarse_apply(bo_prec* P, const DevState* st);
void learned_coarse_free(bo_prec* P);

}  // namespace bo
