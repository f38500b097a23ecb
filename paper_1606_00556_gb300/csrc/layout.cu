// Matrix ingest (BSR / CSR -> colour-split planes), the public BSR SpMV
// (paper Sec. 3.3: y = alpha A x + beta y), natural <-> internal vector
// permutations and the Newton update (paper Alg. 1: x^l = x^{l-1} + dx).
#include <cstdint>

#include "bo_internal.cuh"

namespace bo {
namespace {

// One thread per cell: check the block row's pattern against the stencil
// and scatter its 3x3 blocks into the colour-split planes, in FP64 (A) and
// as split pairs (A2, read by the Arnoldi product).  A warp takes 32
// consecutive cells at a time: their blocks are one contiguous stretch of
// val (rowptr[c0] .. rowptr[c0 + 32]), which the warp copies into shared
// memory with coalesced 8-byte asynchronous copies before each thread reads
// its own cell's blocks from there.  (Each thread reading its 504 bytes
// straight from global memory made every warp load touch 32 lines, which
// left L1 before their reuse: 61% of HBM.)  A stretch that is not a
// plausible pattern (rowptr out of range or decreasing, more than seven
// blocks a cell on average) is read from global memory, where the checks
// below flag it.
constexpr int kIngestWarps = 2;
constexpr int kIngestSpan = 32 * 7 * 9;  // doubles staged per warp

__global__ void __launch_bounds__(32 * kIngestWarps) k_ingest_bsr(Geom g, const int32_t* __restrict__ rowptr,
                                                                  const int32_t* __restrict__ col,
                                                                  const double* __restrict__ val, int64_t nnz,
                                                                  double* __restrict__ A, float2* __restrict__ A2,
                                                                  int* flags, int* range) {
  wait_prior_grid();
  __shared__ double stage[kIngestWarps][kIngestSpan];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const double* sm = stage[warp];
  const uint32_t sm0 = (uint32_t)__cvta_generic_to_shared(sm);
  int split_bad = 0;
  const int64_t nchunk = (g.N + 31) / 32;
  // the loop is uniform over the warp: every lane takes part in the copies
  // and the shuffles
  for (int64_t ch = (int64_t)blockIdx.x * kIngestWarps + warp; ch < nchunk; ch += (int64_t)gridDim.x * kIngestWarps) {
    const int64_t c = ch * 32 + lane;
    const bool live = c < g.N;
    const int32_t e0 = live ? rowptr[c] : 0, e1 = live ? rowptr[c + 1] : 0;
    const int last = (int)min((int64_t)31, g.N - 1 - ch * 32);
    const int32_t E0 = __shfl_sync(0xffffffffu, e0, 0), E1 = __shfl_sync(0xffffffffu, e1, last);
    const bool staged = E0 >= 0 && E1 >= E0 && E1 <= nnz && E1 - E0 <= 32 * 7;
    if (staged) {
      const double* src = val + 9 * (size_t)E0;
      const int cnt = 9 * (E1 - E0);
      for (int t = lane; t < cnt; t += 32)
        asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(sm0 + 8u * (uint32_t)t), "l"(src + t) : "memory");
      asm volatile("cp.async.commit_group;\n\tcp.async.wait_group 0;" ::: "memory");
    }
    __syncwarp();
    if (live) {
      const Nat n = decode_nat(g, c);
      const unsigned valid = valid_slots(g, n);
      unsigned seen = 0;
      int bad = e0 < 0 || e1 < e0 || e1 > nnz || (e1 - e0) != __popc(valid);
      const bool here = staged && e0 >= E0 && e1 <= E1;  // the cell's blocks are in the stage
      int nonfinite = 0;
      for (int32_t e = e0; e < e1 && !bad; ++e) {
        const int s = slot_of(g, n, (int64_t)col[e] - c);
        if (s < 0 || ((seen >> s) & 1u)) { bad = 1; break; }
        seen |= 1u << s;
        const double* v = here ? sm + 9 * (size_t)(e - E0) : val + 9 * (size_t)e;
#pragma unroll
        for (int rc = 0; rc < 9; ++rc) {
          const double a = v[rc];
          nonfinite |= !isfinite(a);
          A[plane(g, n.color, s, rc) + n.q] = a;
          A2[a2_index(g, n.color, s * 9 + rc, n.q)] = df_split_bits(a, &split_bad);
        }
      }
      for (int s = 0; s < 7; ++s)
        if (!((valid >> s) & 1u))
          for (int rc = 0; rc < 9; ++rc) {
            A[plane(g, n.color, s, rc) + n.q] = 0.0;
            A2[a2_index(g, n.color, s * 9 + rc, n.q)] = make_float2(0.f, 0.f);
          }
      if (bad) atomicOr(flags, kErrPattern);
      if (nonfinite) atomicOr(flags, kErrNonfinite);
    }
    __syncwarp();  // the stage is refilled for the warp's next cells
  }
  if (__any_sync(0xffffffffu, split_bad) && lane == 0) atomicOr(range, 1);
}

// One thread per cell: zero the cell's blocks, then add every scalar entry
// of its three CSR rows (row 3c+r, column 3c'+k) into block (c, c').
__global__ void k_ingest_csr(Geom g, const int32_t* __restrict__ rowptr, const int32_t* __restrict__ col,
                             const double* __restrict__ val, int64_t nnz, double* __restrict__ A,
                             float2* __restrict__ A2, int* flags, int* range) {
  wait_prior_grid();
  int split_bad = 0;
  for (int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; c < g.N; c += (int64_t)gridDim.x * blockDim.x) {
    const Nat n = decode_nat(g, c);
    for (int s = 0; s < 7; ++s)
      for (int rc = 0; rc < 9; ++rc) A[plane(g, n.color, s, rc) + n.q] = 0.0;
    int bad = 0, nonfinite = 0;
    for (int r = 0; r < 3; ++r) {
      const int64_t row = 3 * c + r;
      const int32_t e0 = rowptr[row], e1 = rowptr[row + 1];
      if (e0 < 0 || e1 < e0 || e1 > nnz) { bad = 1; continue; }
      for (int32_t e = e0; e < e1; ++e) {
        if (col[e] < 0) { bad = 1; continue; }
        const int64_t cc = col[e] / 3;
        const int k = col[e] - 3 * (int32_t)cc;
        const int s = slot_of(g, n, cc - c);
        if (s < 0) { bad = 1; continue; }
        const double a = val[e];
        nonfinite |= !isfinite(a);
        A[plane(g, n.color, s, 3 * r + k) + n.q] += a;
      }
    }
    for (int s = 0; s < 7; ++s)
      for (int rc = 0; rc < 9; ++rc)
        A2[a2_index(g, n.color, s * 9 + rc, n.q)] = df_split_bits(A[plane(g, n.color, s, rc) + n.q], &split_bad);
    if (bad) atomicOr(flags, kErrPattern);
    if (nonfinite) atomicOr(flags, kErrNonfinite);
  }
  if (__any_sync(0xffffffffu, split_bad) && (threadIdx.x & 31) == 0) atomicOr(range, 1);
}

__global__ void k_to_f32(const double* __restrict__ src, float* __restrict__ dst, size_t n) {
  wait_prior_grid();
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
    dst[i] = (float)src[i];
}

// y = alpha A x + beta y on natural-order interleaved vectors.
// FP64 values: one thread per pair of cells (2q, 2q+1) of a grid row (nx is
// even); the two cells have the two colours and the same half index q, so a
// warp reads 32 consecutive values of each plane of each colour per load
// instruction, and writes the pair's six consecutive outputs.  FP32 and BF16
// values: one thread per cell; neighbouring lanes alternate colours, and the
// warp's gathers of x stay within fewer lines, which matters more once the
// matrix bytes are halved or quartered.
template <typename TM>
__device__ __forceinline__ float to_f(TM v) { return (float)v; }
template <>
__device__ __forceinline__ float to_f<__nv_bfloat16>(__nv_bfloat16 v) { return __bfloat162float(v); }

// TA: accumulation type.  FP64 values accumulate in FP64; FP32 and BF16
// values (the reduced-precision copies) multiply and accumulate in FP32, so
// they are bound by the bytes they move rather than by the FP64 rate.
template <typename TM, typename TA>
__global__ void __launch_bounds__(kThreads) k_spmv_nat(Geom g, const TM* __restrict__ A, const double* __restrict__ x,
                                                      double* __restrict__ y, double alpha, double beta) {
  wait_prior_grid();
  constexpr int H = sizeof(TA) == 8 ? 2 : 1;  // cells per thread
  const int64_t nxy = (int64_t)g.nx * g.ny;
  const int64_t off[7] = {-nxy, -(int64_t)g.nx, -1, 0, 1, (int64_t)g.nx, nxy};
  const int64_t nu = g.N / H;
  for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < nu; q += (int64_t)gridDim.x * blockDim.x) {
    TA acc[H][3];
#pragma unroll
    for (int h = 0; h < H; ++h) {
      const int64_t c = H * q + h;
      const Nat n = decode_nat(g, c);
      const unsigned valid = valid_slots(g, n);
      TA acc0 = 0, acc1 = 0, acc2 = 0;
#pragma unroll
      for (int s = 0; s < 7; ++s) {
        if ((valid >> s) & 1u) {
          const int64_t nc = c + off[s];
          const TA x0 = (TA)__ldg(x + 3 * nc), x1 = (TA)__ldg(x + 3 * nc + 1), x2 = (TA)__ldg(x + 3 * nc + 2);
          const TM* a = A + plane(g, n.color, s, 0) + n.q;
          const size_t P = (size_t)g.Nh;
          if constexpr (sizeof(TA) == 8) {
            acc0 = fma3(acc0, (TA)ld_stream(a), x0, (TA)ld_stream(a + P), x1, (TA)ld_stream(a + 2 * P), x2);
            acc1 = fma3(acc1, (TA)ld_stream(a + 3 * P), x0, (TA)ld_stream(a + 4 * P), x1, (TA)ld_stream(a + 5 * P), x2);
            acc2 = fma3(acc2, (TA)ld_stream(a + 6 * P), x0, (TA)ld_stream(a + 7 * P), x1, (TA)ld_stream(a + 8 * P), x2);
          } else {
            acc0 = fma3(acc0, to_f(ld_stream(a)), x0, to_f(ld_stream(a + P)), x1, to_f(ld_stream(a + 2 * P)), x2);
            acc1 = fma3(acc1, to_f(ld_stream(a + 3 * P)), x0, to_f(ld_stream(a + 4 * P)), x1,
                        to_f(ld_stream(a + 5 * P)), x2);
            acc2 = fma3(acc2, to_f(ld_stream(a + 6 * P)), x0, to_f(ld_stream(a + 7 * P)), x1,
                        to_f(ld_stream(a + 8 * P)), x2);
          }
        }
      }
      acc[h][0] = acc0;
      acc[h][1] = acc1;
      acc[h][2] = acc2;
    }
    double* yo = y + 3 * H * q;
#pragma unroll
    for (int r = 0; r < 3 * H; ++r) {
      const double v = alpha * (double)acc[r / 3][r % 3];
      yo[r] = beta == 0.0 ? v : v + beta * yo[r];
    }
  }
}

// y = alpha A x + beta y on natural-order vectors from a tiled copy of the
// values (the layout of the split copy: the 63 values of 32 consecutive half
// indices of one colour in one 16 KB tile).  V = float2: the split copy
// itself, products and sums in split FP32 pairs (48 significant bits, x split
// on load by integer operations), bound by HBM rather than by GB300's FP64
// rate; V = float or __nv_bfloat16: the reduced-precision copies, FP32
// products and sums.  A thread takes the 2Q cells of Q consecutive half
// indices q0 .. q0 + Q - 1 of one grid row (cells 2 q0 .. 2 q0 + 2Q - 1; the
// two cells of a half index have the two colours), so each of its value
// loads is 8 bytes wide: Q = 1 split pair, 2 floats or 4 BF16 values.  Needs
// hx % Q == 0 (then every group lies in one row and Nh % Q == 0).  x is read
// as contiguous 16-byte pieces of each neighbouring row (the cells' own row
// with one cell on each side, and the rows at -z, -y, +y, +z), y written
// the same way.

// the 3 entries of cell e of a row segment held in registers
template <int M>
__device__ __forceinline__ void seg3(const double (&s)[M], int e, double& x0, double& x1, double& x2) {
  x0 = s[3 * e];
  x1 = s[3 * e + 1];
  x2 = s[3 * e + 2];
}

template <typename V, int Q>
__device__ __forceinline__ void load_vals(const V* a, float (&av)[9][Q], df (&dv)[9]) {
  // one load of Q consecutive entries per block entry: q0 is a multiple of
  // Q, and Q divides the 32 entries of a tile row, so the load is aligned to
  // its own width
#pragma unroll
  for (int rc = 0; rc < 9; ++rc) {
    if constexpr (sizeof(V) == 8) {
      const float2 v2 = __ldcs(reinterpret_cast<const float2*>(a) + 32 * rc);
      dv[rc] = df{v2.x, v2.y};
    } else if constexpr (sizeof(V) == 4 && Q == 2) {
      const float2 v2 = __ldcs(reinterpret_cast<const float2*>(reinterpret_cast<const float*>(a) + 32 * rc));
      av[rc][0] = v2.x;
      av[rc][Q - 1] = v2.y;
    } else if constexpr (sizeof(V) == 4) {
      av[rc][0] = __ldcs(reinterpret_cast<const float*>(a) + 32 * rc);
    } else if constexpr (Q == 4) {
      const uint2 u = __ldcs(reinterpret_cast<const uint2*>(reinterpret_cast<const __nv_bfloat16*>(a) + 32 * rc));
      av[rc][0] = __uint_as_float(u.x << 16);
      av[rc][Q > 1 ? 1 : 0] = __uint_as_float(u.x & 0xffff0000u);
      av[rc][Q > 2 ? 2 : 0] = __uint_as_float(u.y << 16);
      av[rc][Q > 3 ? 3 : 0] = __uint_as_float(u.y & 0xffff0000u);
    } else if constexpr (Q == 2) {
      const unsigned u = __ldcs(reinterpret_cast<const unsigned*>(reinterpret_cast<const __nv_bfloat16*>(a) + 32 * rc));
      av[rc][0] = __uint_as_float(u << 16);
      av[rc][Q - 1] = __uint_as_float(u & 0xffff0000u);
    } else {
      const unsigned short u = __ldcs(reinterpret_cast<const unsigned short*>(a) + 32 * rc);
      av[rc][0] = __uint_as_float((unsigned)u << 16);
    }
  }
}

template <typename V, int Q>
__global__ void __launch_bounds__(kThreads) k_spmv_tiled(Geom g, const V* __restrict__ A, const double* __restrict__ x,
                                                        double* __restrict__ y, double alpha, double beta,
                                                        const double* __restrict__ A64, const int* __restrict__ range) {
  wait_prior_grid();
  constexpr bool SPLIT = sizeof(V) == 8;
  constexpr int C = 2 * Q;  // cells of a group
  // a split copy that could not hold every value: the FP64 planes instead
  const bool fp64 = SPLIT && *range != 0;
  const int64_t ng = g.Nh / Q;
  const int64_t nxy = (int64_t)g.nx * g.ny;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < ng; t += (int64_t)gridDim.x * blockDim.x) {
    const int64_t q0 = Q * t;
    const uint32_t row = (uint32_t)q0 / (uint32_t)g.hx;
    const int i0 = 2 * (int)((uint32_t)q0 - row * (uint32_t)g.hx);
    const int j = (int)(row % (uint32_t)g.ny), k = (int)(row / (uint32_t)g.ny);
    const int cA = (j + k) & 1;  // colour of the even cells of the group
    const int64_t c0 = 2 * q0;
    float acc[C][3];
    df dacc[C][3];
#pragma unroll
    for (int e = 0; e < C; ++e)
#pragma unroll
      for (int r = 0; r < 3; ++r) {
        acc[e][r] = 0.f;
        dacc[e][r] = df{0.f, 0.f};
      }
    // add the block of slot sl (colour of cell e) times (x0, x1, x2) to cell e
    auto add = [&](int e, const float (&av)[9][Q], const df (&dv)[9], int sl, int col, double x0, double x1,
                   double x2) {
      if (fp64) {
        const double* a64 = A64 + plane(g, col, sl, 0) + q0 + e / 2;
        const size_t P = (size_t)g.Nh;
#pragma unroll
        for (int r = 0; r < 3; ++r)
          dacc[e][r] = df_add(dacc[e][r], df_from(fma3(0.0, a64[3 * r * P], x0, a64[(3 * r + 1) * P], x1,
                                                       a64[(3 * r + 2) * P], x2)));
      } else if constexpr (SPLIT) {
        int bad = 0;
        const float2 s0 = df_split_bits(x0, &bad), s1 = df_split_bits(x1, &bad), s2 = df_split_bits(x2, &bad);
        const df d0{s0.x, s0.y}, d1{s1.x, s1.y}, d2{s2.x, s2.y};
#pragma unroll
        for (int r = 0; r < 3; ++r) {
          dacc[e][r] = df_fma_acc(dacc[e][r], dv[3 * r], d0);
          dacc[e][r] = df_fma_acc(dacc[e][r], dv[3 * r + 1], d1);
          dacc[e][r] = df_fma_acc(dacc[e][r], dv[3 * r + 2], d2);
        }
      } else {
        const int p = e / 2;
        const float f0 = (float)x0, f1 = (float)x1, f2 = (float)x2;
#pragma unroll
        for (int r = 0; r < 3; ++r)
          acc[e][r] = fma3(acc[e][r], av[3 * r][p], f0, av[3 * r + 1][p], f1, av[3 * r + 2][p], f2);
      }
    };
    float av[2][9][Q];
    df dv[2][9];
    // rows at -z, -y, +y, +z: the C cells directly across, 3 C contiguous
    // doubles starting at an even index (16-byte aligned)
#pragma unroll
    for (int which = 0; which < 4; ++which) {
      const int sl = which == 0 ? kZm : which == 1 ? kYm : which == 2 ? kYp : kZp;
      const bool ok = which == 0 ? k > 0 : which == 1 ? j > 0 : which == 2 ? j < g.ny - 1 : k < g.nz - 1;
      // BF16 and split values: a missing row is read as the cells' own row
      // (every load issued, so all of a thread's loads can be in flight) and
      // its x replaced by zero (measured faster: BF16 53 -> 48 us at
      // 128x128x64); FP32 values skip it (the masked form measured slower)
      if (sizeof(V) == 4 && !ok) continue;
      const int64_t off =
          !ok ? 0 : which == 0 ? -nxy : which == 1 ? -(int64_t)g.nx : which == 2 ? (int64_t)g.nx : nxy;
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        const int col = h ? 1 - cA : cA;
        load_vals<V, Q>(A + a2_index(g, col, sl * 9, q0), av[h], dv[h]);
      }
      double xs[3 * C];
      const double2* xp = reinterpret_cast<const double2*>(x + 3 * (c0 + off));
#pragma unroll
      for (int u = 0; u < 3 * C / 2; ++u) {
        const double2 v = __ldg(xp + u);
        xs[2 * u] = ok ? v.x : 0.0;
        xs[2 * u + 1] = ok ? v.y : 0.0;
      }
#pragma unroll
      for (int e = 0; e < C; ++e) {
        double x0, x1, x2;
        seg3(xs, e, x0, x1, x2);
        add(e, av[e & 1], dv[e & 1], sl, (e & 1) ? 1 - cA : cA, x0, x1, x2);
      }
    }
    // the cells' own row: -x, diag, +x from the C cells and one on each side
    {
      double xs[3 * (C + 2)];  // cells c0 - 1 .. c0 + C
      const double2* xp = reinterpret_cast<const double2*>(x + 3 * c0);
#pragma unroll
      for (int u = 0; u < 3 * C / 2; ++u) {
        const double2 v = __ldg(xp + u);
        xs[3 + 2 * u] = v.x;
        xs[3 + 2 * u + 1] = v.y;
      }
      const bool has_l = i0 > 0, has_r = i0 + C < g.nx;
#pragma unroll
      for (int m = 0; m < 3; ++m) {
        xs[m] = has_l ? __ldg(x + 3 * (c0 - 1) + m) : 0.0;
        xs[3 * (C + 1) + m] = has_r ? __ldg(x + 3 * (c0 + C) + m) : 0.0;
      }
#pragma unroll
      for (int which = 0; which < 3; ++which) {
        const int sl = which == 0 ? kXm : which == 1 ? kDiag : kXp;
#pragma unroll
        for (int h = 0; h < 2; ++h) {
          const int col = h ? 1 - cA : cA;
          load_vals<V, Q>(A + a2_index(g, col, sl * 9, q0), av[h], dv[h]);
        }
#pragma unroll
        for (int e = 0; e < C; ++e) {
          const int nb = e + (which == 0 ? -1 : which == 1 ? 0 : 1);  // neighbour within the segment
          if (which == 0 && e == 0 && !has_l) continue;
          if (which == 2 && e == C - 1 && !has_r) continue;
          double x0, x1, x2;
          seg3(xs, nb + 1, x0, x1, x2);
          add(e, av[e & 1], dv[e & 1], sl, (e & 1) ? 1 - cA : cA, x0, x1, x2);
        }
      }
    }
    // y: 3 C contiguous doubles from an even index
    double ys[3 * C];
#pragma unroll
    for (int e = 0; e < C; ++e)
#pragma unroll
      for (int r = 0; r < 3; ++r)
        ys[3 * e + r] = alpha * (SPLIT ? df_to_double(df_renorm(dacc[e][r])) : (double)acc[e][r]);
    double2* yp = reinterpret_cast<double2*>(y + 3 * c0);
#pragma unroll
    for (int u = 0; u < 3 * C / 2; ++u) {
      double2 v = make_double2(ys[2 * u], ys[2 * u + 1]);
      if (beta != 0.0) {
        const double2 o = yp[u];
        v.x += beta * o.x;
        v.y += beta * o.y;
      }
      yp[u] = v;
    }
  }
}

// the FP64 planes rounded to T in the tiled layout (the reduced-precision
// copies the public SpMV reads)
template <typename T>
__global__ void k_to_tiled(Geom g, const double* __restrict__ src, T* __restrict__ dst) {
  wait_prior_grid();
  const size_t n = (size_t)126 * g.Nh;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
    const int p = (int)(i / g.Nh);  // plane: colour * 63 + slot * 9 + rc
    const int64_t q = (int64_t)(i - (size_t)p * g.Nh);
    const double v = src[i];
    T o;
    if constexpr (sizeof(T) == 2) o = __float2bfloat16_rn((float)v);
    else o = (T)v;
    dst[a2_index(g, p / 63, p % 63, q)] = o;
  }
}

__global__ void k_to_bf16(const double* __restrict__ src, __nv_bfloat16* __restrict__ dst, size_t n) {
  wait_prior_grid();
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
    dst[i] = __float2bfloat16_rn((float)src[i]);
}

// split (hi, lo) copy of the matrix values for the Arnoldi product, in the
// tiled layout; *range flags values the split form cannot hold
__global__ void k_split_matrix(Geom g, const double* __restrict__ src, float2* __restrict__ dst, int* range) {
  wait_prior_grid();
  int bad = 0;
  const size_t n = (size_t)126 * g.Nh;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
    const int p = (int)(i / g.Nh);  // plane: colour * 63 + slot * 9 + rc
    const int64_t q = (int64_t)(i - (size_t)p * g.Nh);
    dst[a2_index(g, p / 63, p % 63, q)] = df_split_bits(src[i], &bad);
  }
  if (__any_sync(0xffffffffu, bad) && (threadIdx.x & 31) == 0) atomicOr(range, 1);
}

__global__ void k_widen(const float* __restrict__ src, double* __restrict__ dst, size_t n) {
  wait_prior_grid();
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
    dst[i] = (double)src[i];
}

__global__ void k_gather(Geom g, const double* __restrict__ nat, double* __restrict__ in) {
  wait_prior_grid();
  for (int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; c < g.N; c += (int64_t)gridDim.x * blockDim.x) {
    const Nat n = decode_nat(g, c);
    for (int k = 0; k < 3; ++k) in[vidx(g, k, n.color, n.q)] = nat[3 * c + k];
  }
}

__global__ void k_scatter(Geom g, const double* __restrict__ in, double* __restrict__ nat) {
  wait_prior_grid();
  for (int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; c < g.N; c += (int64_t)gridDim.x * blockDim.x) {
    const Nat n = decode_nat(g, c);
    for (int k = 0; k < 3; ++k) nat[3 * c + k] = in[vidx(g, k, n.color, n.q)];
  }
}

__global__ void k_axpy1(double* __restrict__ s, const double* __restrict__ d, int64_t n) {
  wait_prior_grid();
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    s[i] += d[i];
}

}  // namespace

int ingest_bsr(bo_mat* m, const double* dval, cudaStream_t s) {
  cudaMemsetAsync(m->a2_range, 0, sizeof(int), s);
  const int threads = 32 * kIngestWarps;  // one cell per thread and step
  (launch_pdl(k_ingest_bsr, occ_grid((const void*)k_ingest_bsr, m->g.N, threads), threads, 0, s, m->g, m->rowptr, m->col,
      dval, m->nnz, m->A, m->A2, m->flags, m->a2_range), note_launch());
  m->a2_valid = true;
  return cudaGetLastError() == cudaSuccess ? BO_OK : BO_ERR_CUDA;
}

int ingest_csr(bo_mat* m, const double* dval, cudaStream_t s) {
  cudaMemsetAsync(m->a2_range, 0, sizeof(int), s);
  (launch_pdl(k_ingest_csr, grid_for(m->g.N), kThreads, 0, s, m->g, m->rowptr, m->col, dval, m->nnz, m->A, m->A2, m->flags,
      m->a2_range), note_launch());
  m->a2_valid = true;
  return cudaGetLastError() == cudaSuccess ? BO_OK : BO_ERR_CUDA;
}

void launch_to_f32(const double* src, float* dst, size_t n, cudaStream_t s) {
  (launch_pdl(k_to_f32, grid_for((int64_t)n), kThreads, 0, s, src, dst, n), note_launch());
}

void launch_spmv_nat(const bo_mat* m, double alpha, const double* x, double beta, double* y, int precision) {
  const Geom& g = m->g;
  cudaStream_t s = m->ctx->stream;
  if ((((uintptr_t)x) | ((uintptr_t)y)) & 15) {
    // vectors off a 16-byte boundary: the tiled kernels read and write them
    // 16 bytes at a time, so the FP64 planes with scalar accesses instead
    (launch_pdl(k_spmv_nat<double, double>, grid_for(g.Nh, kThreads, 152 * 64), kThreads, 0, s, g, m->A, x, y, alpha, beta),
     note_launch());
    return;
  }
  if (precision == BO_PREC_FP32) {
    const int Q = g.hx % 2 == 0 ? 2 : 1;
    if (Q == 2)
      (launch_pdl(k_spmv_tiled<float, 2>, grid_for((g.Nh + 1) / 2), kThreads, 0, s, g, m->A32, x, y, alpha, beta, nullptr,
          nullptr),
       note_launch());
    else
      (launch_pdl(k_spmv_tiled<float, 1>, grid_for(g.Nh), kThreads, 0, s, g, m->A32, x, y, alpha, beta, nullptr, nullptr),
       note_launch());
  } else if (precision == BO_PREC_BF16) {
    if (g.hx % 2 == 0)
      (launch_pdl(k_spmv_tiled<__nv_bfloat16, 2>, grid_for((g.Nh + 1) / 2), kThreads, 0, s, g, m->A16, x, y, alpha, beta,
          nullptr, nullptr),
       note_launch());
    else
      (launch_pdl(k_spmv_tiled<__nv_bfloat16, 1>, grid_for(g.Nh), kThreads, 0, s, g, m->A16, x, y, alpha, beta, nullptr,
          nullptr),
       note_launch());
  } else {
    bo_mat* mm = const_cast<bo_mat*>(m);
    if (!mm->a2_valid) launch_split_matrix(mm, s);
    (launch_pdl(k_spmv_tiled<float2, 1>, grid_for(g.Nh), kThreads, 0, s, g, m->A2, x, y, alpha, beta, m->A, m->a2_range),
     note_launch());
  }
}

void launch_to_tiled_f32(const bo_mat* m, float* dst, cudaStream_t s) {
  (launch_pdl(k_to_tiled<float>, grid_for((int64_t)63 * m->g.N), kThreads, 0, s, m->g, m->A, dst), note_launch());
}

void launch_to_tiled_bf16(const bo_mat* m, __nv_bfloat16* dst, cudaStream_t s) {
  (launch_pdl(k_to_tiled<__nv_bfloat16>, grid_for((int64_t)63 * m->g.N), kThreads, 0, s, m->g, m->A, dst), note_launch());
}

void launch_split_matrix(bo_mat* m, cudaStream_t s) {
  cudaMemsetAsync(m->a2_range, 0, sizeof(int), s);
  (launch_pdl(k_split_matrix, grid_for((int64_t)63 * m->g.N), kThreads, 0, s, m->g, m->A, m->A2, m->a2_range), note_launch());
  m->a2_valid = true;
}

void launch_to_bf16(const double* src, __nv_bfloat16* dst, size_t n, cudaStream_t s) {
  (launch_pdl(k_to_bf16, grid_for((int64_t)n), kThreads, 0, s, src, dst, n), note_launch());
}

void launch_widen(const float* src, double* dst, size_t n, cudaStream_t s) {
  (launch_pdl(k_widen, grid_for((int64_t)n), kThreads, 0, s, src, dst, n), note_launch());
}

void launch_gather(const Geom& g, const double* nat, double* in, cudaStream_t s) {
  (launch_pdl(k_gather, grid_for(g.N), kThreads, 0, s, g, nat, in), note_launch());
}

void launch_scatter(const Geom& g, const double* in, double* nat, cudaStream_t s) {
  (launch_pdl(k_scatter, grid_for(g.N), kThreads, 0, s, g, in, nat), note_launch());
}

void launch_newton_update(double* state, const double* dx, int64_t n, cudaStream_t s) {
  (launch_pdl(k_axpy1, grid_for(n), kThreads, 0, s, state, dx, n), note_launch());
}

}  // namespace bo
