// 3D convolutional network for the learned Newton pressure update: BF16
// tensor-core convolution kernels (forward, data gradient, weight gradient)
// with FP32 accumulation, the elementwise pieces of training (ReLU masks,
// residual adds, MSE loss, Adam with FP32 master weights) and the network
// that strings them together.  No counterpart in the paper: an addition
// that gives the Krylov solve of Sec. 3 a predicted initial guess and coarse
// space.
//
// Layout.  Activations are NDHWC BF16: [batch][nz][ny][nx][C], voxel
// v = x + nx (y + ny z) (the solver's cell index), C = 16 for the input
// (6 features padded) or 32.  Weights are [27 taps][Cout][Cin] BF16 with tap
// t = 9 (dz+1) + 3 (dy+1) + (dx+1); 'same' zero padding.
//
// Convolution as an implicit GEMM on mma.sync.m16n8k16 (BF16 in, FP32
// accumulate): M = voxels (16 per warp), N = Cout, K = 27 taps x Cin.  A
// fragments come straight from global memory (each voxel's channels are
// contiguous; the neighbours of a warp's voxels stay in L1), B fragments
// from the layer's weights staged once per block in shared memory (row
// stride padded to avoid bank conflicts).  The data gradient is the forward
// kernel run on dY with flipped, transposed weights; the weight gradient is a
// GEMM over voxels on channel-major copies of X and dY, split over blocks
// with per-block partials summed in a fixed order.
#include <cuda_bf16.h>

#include <cmath>
#include <cstring>
#include <new>
#include <random>
#include <vector>

#include "bo_internal.cuh"

namespace bo {
namespace {

using bf16 = __nv_bfloat16;
constexpr int kConvThreads = 256;
constexpr int kVoxPerBlock = 128;   // 8 warps x 16 voxels
constexpr int kOutF32 = 4;          // FP32 prediction channels (dp, then optionally dSw, dSg)

__device__ __forceinline__ void mma_bf16(float d[4], const uint32_t a[4], uint32_t b0, uint32_t b1) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
      "{%0,%1,%2,%3};\n"
      : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

__device__ __forceinline__ uint32_t ld_pair(const bf16* p) { return *reinterpret_cast<const uint32_t*>(p); }

__device__ __forceinline__ uint32_t pack2(float lo, float hi) {
  const bf16 l = __float2bfloat16_rn(lo), h = __float2bfloat16_rn(hi);
  return (uint32_t)__bfloat16_as_ushort(l) | ((uint32_t)__bfloat16_as_ushort(h) << 16);
}

__device__ __forceinline__ void tap_offset(int tap, int& dx, int& dy, int& dz) {
  dz = tap / 9 - 1;
  dy = (tap / 3) % 3 - 1;
  dx = tap % 3 - 1;
}

// Y[v][co] = act(bias[co] + sum_tap,ci X[v + off(tap)][ci] W[tap][co][ci] (+ R[v][co]))
// RELU: clamp at 0 after the residual add.  RES: add R.  F32: 0 BF16 output
// only; 1 BF16 output and channels 0..3 in FP32 (Yf[v][0..3]); 2 FP32 output
// of all channels only (Yf[v][co]).
template <int CIN, int COUT, bool RELU, bool RES, int F32>
__global__ void __launch_bounds__(kConvThreads) k_conv3d_fwd(int nx, int ny, int nz, const bf16* __restrict__ X,
                                                            const bf16* __restrict__ W, const float* __restrict__ bias,
                                                            const bf16* __restrict__ R, bf16* __restrict__ Y,
                                                            float* __restrict__ Yf) {
  constexpr int WS = CIN / 2 + 4;  // padded row stride (32-bit words) of one (tap, co) weight row
  extern __shared__ __align__(16) uint32_t ws[];
  for (int i = threadIdx.x; i < 27 * COUT * (CIN / 2); i += blockDim.x) {
    const int row = i / (CIN / 2), col = i - row * (CIN / 2);
    ws[row * WS + col] = reinterpret_cast<const uint32_t*>(W)[i];
  }
  __syncthreads();
  const int V = nx * ny * nz;
  const int b = blockIdx.y;
  const bf16* Xb = X + (size_t)b * V * CIN;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, g = lane >> 2, c = lane & 3;
  const int v0 = blockIdx.x * kVoxPerBlock + warp * 16;
  int vr[2], xr[2], yr[2], zr[2];
  bool ok[2];
#pragma unroll
  for (int r = 0; r < 2; ++r) {
    vr[r] = v0 + g + 8 * r;
    ok[r] = vr[r] < V;
    xr[r] = vr[r] % nx;
    yr[r] = (vr[r] / nx) % ny;
    zr[r] = vr[r] / (nx * ny);
  }
  float acc[COUT / 8][4];
#pragma unroll
  for (int j = 0; j < COUT / 8; ++j) acc[j][0] = acc[j][1] = acc[j][2] = acc[j][3] = 0.f;
  for (int tap = 0; tap < 27; ++tap) {
    int dx, dy, dz;
    tap_offset(tap, dx, dy, dz);
    const bf16* src[2];
    bool in[2];
#pragma unroll
    for (int r = 0; r < 2; ++r) {
      in[r] = ok[r] && xr[r] + dx >= 0 && xr[r] + dx < nx && yr[r] + dy >= 0 && yr[r] + dy < ny && zr[r] + dz >= 0 &&
              zr[r] + dz < nz;
      src[r] = Xb + (size_t)(in[r] ? vr[r] + dx + nx * (dy + ny * dz) : 0) * CIN;
    }
#pragma unroll
    for (int kc = 0; kc < CIN / 16; ++kc) {
      uint32_t a[4];
      a[0] = in[0] ? ld_pair(src[0] + kc * 16 + 2 * c) : 0u;
      a[1] = in[1] ? ld_pair(src[1] + kc * 16 + 2 * c) : 0u;
      a[2] = in[0] ? ld_pair(src[0] + kc * 16 + 2 * c + 8) : 0u;
      a[3] = in[1] ? ld_pair(src[1] + kc * 16 + 2 * c + 8) : 0u;
#pragma unroll
      for (int j = 0; j < COUT / 8; ++j) {
        const uint32_t* wrow = ws + (tap * COUT + j * 8 + g) * WS + kc * 8;
        mma_bf16(acc[j], a, wrow[c], wrow[c + 4]);
      }
    }
  }
#pragma unroll
  for (int j = 0; j < COUT / 8; ++j) {
    const int co = j * 8 + 2 * c;
#pragma unroll
    for (int r = 0; r < 2; ++r) {
      if (!ok[r]) continue;
      const size_t o = ((size_t)b * V + vr[r]) * COUT + co;
      float y0 = acc[j][2 * r] + bias[co], y1 = acc[j][2 * r + 1] + bias[co + 1];
      if (RES) {
        const uint32_t rp = ld_pair(R + o);
        y0 += __bfloat162float(__ushort_as_bfloat16((unsigned short)(rp & 0xffffu)));
        y1 += __bfloat162float(__ushort_as_bfloat16((unsigned short)(rp >> 16)));
      }
      if (RELU) {
        y0 = fmaxf(y0, 0.f);
        y1 = fmaxf(y1, 0.f);
      }
      if (F32 == 2) {
        Yf[o] = y0;
        Yf[o + 1] = y1;
      } else {
        *reinterpret_cast<uint32_t*>(Y + o) = pack2(y0, y1);
        if (F32 == 1 && co < kOutF32) {
          Yf[((size_t)b * V + vr[r]) * kOutF32 + co] = y0;
          Yf[((size_t)b * V + vr[r]) * kOutF32 + co + 1] = y1;
        }
      }
    }
  }
}

// data-gradient weights: Wd[t][ci][co] = W[26 - t][co][ci]
__global__ void k_flip_transpose(const bf16* __restrict__ W, bf16* __restrict__ Wd, int cin, int cout) {
  const int n = 27 * cin * cout;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    const int t = i / (cin * cout), rem = i - t * cin * cout, ci = rem / cout, co = rem - ci * cout;
    Wd[i] = W[((26 - t) * cout + co) * cin + ci];
  }
}

// ldmatrix of four 8x8 b16 blocks, transposed: lanes 8i..8i+7 give the 16-byte
// rows of block i; register i receives block i in the mma fragment layout
__device__ __forceinline__ void ldsm_x4_t(uint32_t r[4], const void* p) {
  const uint32_t a = (uint32_t)__cvta_generic_to_shared(p);
  asm volatile("ldmatrix.sync.aligned.m8n8.x4.trans.shared.b16 {%0,%1,%2,%3}, [%4];\n"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])
               : "r"(a));
}

// Weight gradient dW[t][co][ci] = sum_v dY[v][co] X[v + off(t)][ci] as a
// persistent implicit GEMM (M = co, N = ci, K = voxels) over bricks of
// 8 x 8 x 4 voxels.  Per brick the block stages dY (256 voxels) and X with
// a one-voxel halo (10 x 10 x 6) in shared memory, rows padded by 16 bytes so
// that the 8 rows of an ldmatrix fall in distinct banks; ldmatrix.trans
// turns the voxel-major tiles into the K-major mma fragments, for every tap
// (the tap only moves the X row addresses).  Warps own (tap, 16-row co tile)
// units and keep their accumulators in registers across all bricks of the
// block; at the end each block writes its partial sums
// part[block][tap][co][ci], summed in a fixed order by k_wgrad_reduce.
// Voxels of a brick outside the grid have dY = 0, so they add nothing.
constexpr int kBrickX = 8, kBrickY = 8, kBrickZ = 4, kBrick = 256;
constexpr int kHaloX = 10, kHaloY = 10, kHalo = 600;
constexpr int kWgMaxBlocks = 304;

template <int CIN, int COUT>
constexpr size_t wgrad_smem() {
  return (size_t)(kHalo * (CIN + 8) + kBrick * (COUT + 8)) * sizeof(bf16);
}

template <int CIN, int COUT>
__global__ void __launch_bounds__(kConvThreads, 1) k_conv3d_wgrad(int nx, int ny, int nz, int B,
                                                                 const bf16* __restrict__ X,
                                                                 const bf16* __restrict__ D, float* __restrict__ part) {
  constexpr int XS = CIN + 8, DS = COUT + 8;  // shared row strides (bf16)
  constexpr int MT = COUT / 16, NT = CIN / 8;
  constexpr int kUnits = (27 * MT + 7) / 8;   // (tap, co tile) units per warp
  extern __shared__ __align__(16) bf16 sm[];
  bf16* xs = sm;                // [kHalo][XS]
  bf16* ds = sm + kHalo * XS;   // [kBrick][DS]
  const int V = nx * ny * nz;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, g = lane >> 2, c = lane & 3;
  const int mi = lane >> 3, r = lane & 7;
  const int bxn = (nx + kBrickX - 1) / kBrickX, byn = (ny + kBrickY - 1) / kBrickY,
            bzn = (nz + kBrickZ - 1) / kBrickZ;
  const int nbricks = bxn * byn * bzn * B;
  float acc[kUnits][NT][4];
#pragma unroll
  for (int u = 0; u < kUnits; ++u)
#pragma unroll
    for (int n = 0; n < NT; ++n) acc[u][n][0] = acc[u][n][1] = acc[u][n][2] = acc[u][n][3] = 0.f;
  for (int br = blockIdx.x; br < nbricks; br += gridDim.x) {
    int t = br;
    const int bx = t % bxn; t /= bxn;
    const int by = t % byn; t /= byn;
    const int bz = t % bzn;
    const int b = t / bzn;
    const int x0 = bx * kBrickX, y0 = by * kBrickY, z0 = bz * kBrickZ;
    const bf16* Xb = X + (size_t)b * V * CIN;
    const bf16* Db = D + (size_t)b * V * COUT;
    __syncthreads();  // the previous brick's fragments are read
    for (int i = threadIdx.x; i < kHalo * (CIN / 8); i += blockDim.x) {
      const int row = i / (CIN / 8), ch = i - row * (CIN / 8);
      const int gx = x0 + row % kHaloX - 1, gy = y0 + (row / kHaloX) % kHaloY - 1, gz = z0 + row / (kHaloX * kHaloY) - 1;
      uint4 v = make_uint4(0u, 0u, 0u, 0u);
      if (gx >= 0 && gx < nx && gy >= 0 && gy < ny && gz >= 0 && gz < nz)
        v = *reinterpret_cast<const uint4*>(Xb + (size_t)(gx + nx * (gy + ny * gz)) * CIN + ch * 8);
      *reinterpret_cast<uint4*>(xs + row * XS + ch * 8) = v;
    }
    for (int i = threadIdx.x; i < kBrick * (COUT / 8); i += blockDim.x) {
      const int row = i / (COUT / 8), ch = i - row * (COUT / 8);
      const int gx = x0 + row % kBrickX, gy = y0 + (row / kBrickX) % kBrickY, gz = z0 + row / (kBrickX * kBrickY);
      uint4 v = make_uint4(0u, 0u, 0u, 0u);
      if (gx < nx && gy < ny && gz < nz)
        v = *reinterpret_cast<const uint4*>(Db + (size_t)(gx + nx * (gy + ny * gz)) * COUT + ch * 8);
      *reinterpret_cast<uint4*>(ds + row * DS + ch * 8) = v;
    }
    __syncthreads();
#pragma unroll
    for (int u = 0; u < kUnits; ++u) {
      const int unit = warp + 8 * u;
      if (unit >= 27 * MT) break;  // warp-uniform
      const int tap = unit / MT, mt = unit - tap * MT;
      int dx, dy, dz;
      tap_offset(tap, dx, dy, dz);
#pragma unroll 2
      for (int ks = 0; ks < kBrick; ks += 16) {
        uint32_t a[4];
        ldsm_x4_t(a, ds + (ks + r + ((mi >> 1) << 3)) * DS + mt * 16 + ((mi & 1) << 3));
        const int v = ks + r + ((mi & 1) << 3);
        const int hrow = ((v & 7) + 1 + dx) + kHaloX * ((((v >> 3) & 7) + 1 + dy) + kHaloY * ((v >> 6) + 1 + dz));
#pragma unroll
        for (int np = 0; np < NT / 2; ++np) {
          uint32_t bq[4];
          ldsm_x4_t(bq, xs + hrow * XS + (2 * np + (mi >> 1)) * 8);
          mma_bf16(acc[u][2 * np], a, bq[0], bq[1]);
          mma_bf16(acc[u][2 * np + 1], a, bq[2], bq[3]);
        }
      }
    }
  }
#pragma unroll
  for (int u = 0; u < kUnits; ++u) {
    const int unit = warp + 8 * u;
    if (unit >= 27 * MT) break;
    const int tap = unit / MT, mt = unit - tap * MT;
    float* P = part + ((size_t)blockIdx.x * 27 + tap) * COUT * CIN;
#pragma unroll
    for (int n = 0; n < NT; ++n)
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        const int co = mt * 16 + g + 8 * h, ci = n * 8 + 2 * c;
        P[co * CIN + ci] = acc[u][n][2 * h];
        P[co * CIN + ci + 1] = acc[u][n][2 * h + 1];
      }
  }
}

// out[i] = sum over k < chunks of part[k n + i] (fixed order, FP64 sum)
__global__ void k_wgrad_reduce(const float* __restrict__ part, float* __restrict__ out, int n, int chunks) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    double s = 0.0;
    for (int k = 0; k < chunks; ++k) s += part[(size_t)k * n + i];
    out[i] = (float)s;
  }
}

// Per-block bias-gradient partials: part[block][co] = sum over this block's
// voxels of dY[v][co] (FP64).  Threads take consecutive (voxel, channel)
// pairs, so the loads are coalesced; C divides the block size.
__global__ void k_bias_partial(const float* __restrict__ dY, double* __restrict__ part, int64_t nvox, int C) {
  __shared__ double sh[kThreads];
  const int per = blockDim.x / C;
  const int co = threadIdx.x % C, sub = threadIdx.x / C;
  double s = 0.0;
  for (int64_t v = blockIdx.x * (int64_t)per + sub; v < nvox; v += (int64_t)gridDim.x * per) s += dY[v * C + co];
  sh[threadIdx.x] = s;
  __syncthreads();
  if (threadIdx.x < C) {
    double t = 0.0;
    for (int k = 0; k < per; ++k) t += sh[k * C + threadIdx.x];
    part[(size_t)blockIdx.x * C + threadIdx.x] = t;
  }
}

__global__ void k_bias_reduce(const double* __restrict__ part, float* __restrict__ db, int C, int chunks) {
  const int co = threadIdx.x;
  if (co >= C) return;
  double s = 0.0;
  for (int k = 0; k < chunks; ++k) s += part[(size_t)k * C + co];
  db[co] = (float)s;
}

// dpre = dpost * (post > 0); also the BF16 copy used as the next mma input
__global__ void k_relu_bwd(const float* __restrict__ dpost, const bf16* __restrict__ post, float* __restrict__ dpre,
                           bf16* __restrict__ dpre16, int64_t n) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const float d = __bfloat162float(post[i]) > 0.f ? dpost[i] : 0.f;
    dpre[i] = d;
    dpre16[i] = __float2bfloat16_rn(d);
  }
}

__global__ void k_add_f32(float* __restrict__ a, const float* __restrict__ b, int64_t n) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    a[i] += b[i];
}

// Masked mean squared error over the first nout prediction channels:
// loss = inv_count sum_v mask_v sum_k<nout (pred[v][k] - target[v][k])^2 with
// pred/target [v][kOutF32]; dY[v][0..C) is its gradient (zero past nout).
__global__ void k_mse(const float* __restrict__ pred, const float* __restrict__ target, const float* __restrict__ mask,
                      float* __restrict__ dY, int C, int nout, int64_t n, double inv_count, double* partials) {
  __shared__ double sh[32];
  double s = 0.0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const double m = mask ? mask[i] : 1.0;
    for (int k = 0; k < C; ++k) {
      float g = 0.f;
      if (k < nout) {
        const double d = (double)pred[i * kOutF32 + k] - (double)target[i * kOutF32 + k];
        s += m * d * d;
        g = (float)(2.0 * m * d * inv_count);
      }
      dY[i * C + k] = g;
    }
  }
  s = block_sum(s, sh);
  if (threadIdx.x == 0) partials[blockIdx.x] = s * inv_count;
}

// Adam (Kingma & Ba) on FP32 master weights; writes the BF16 copy
__global__ void k_adam(float* __restrict__ p, const float* __restrict__ gr, float* __restrict__ m, float* __restrict__ v,
                       bf16* __restrict__ p16, int64_t n, float lr, float b1, float b2, float eps, float c1, float c2) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const float gi = gr[i];
    const float mi = b1 * m[i] + (1.f - b1) * gi;
    const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    const float w = p[i] - lr * (mi / c1) / (sqrtf(vi / c2) + eps);
    p[i] = w;
    if (p16) p16[i] = __float2bfloat16_rn(w);
  }
}

__global__ void k_f32_to_bf16(const float* __restrict__ a, bf16* __restrict__ b, int64_t n) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    b[i] = __float2bfloat16_rn(a[i]);
}

// ------------------------------------------------------------ dispatch
template <int CIN, int COUT, bool RELU, bool RES, int F32>
int launch_fwd_t(int nx, int ny, int nz, int B, const bf16* X, const bf16* W, const float* bias, const bf16* R, bf16* Y,
                 float* Yf, cudaStream_t s) {
  const int V = nx * ny * nz;
  const size_t smem = (size_t)27 * COUT * (CIN / 2 + 4) * sizeof(uint32_t);
  auto k = k_conv3d_fwd<CIN, COUT, RELU, RES, F32>;
  if (cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess)
    return BO_ERR_CUDA;
  const dim3 grid((V + kVoxPerBlock - 1) / kVoxPerBlock, B);
  (k<<<grid, kConvThreads, smem, s>>>(nx, ny, nz, X, W, bias, R, Y, Yf), note_launch());
  return cudaGetLastError() == cudaSuccess ? BO_OK : BO_ERR_CUDA;
}

// the (channels, mode) combinations the network and its gradients use
enum FwdMode { kReluBf16, kReluResBf16, kLinearOut, kLinearF32All };

int launch_fwd(int cin, int cout, FwdMode mode, int nx, int ny, int nz, int B, const bf16* X, const bf16* W,
               const float* bias, const bf16* R, bf16* Y, float* Yf, cudaStream_t s) {
  if (g_conv_engine.load() == 1 && cin == 32 && cout == 32 &&
      (mode == kReluBf16 || mode == kReluResBf16 || mode == kLinearF32All)) {
    const int tm = mode == kReluBf16 ? 0 : mode == kReluResBf16 ? 1 : 2;
    const int rc = launch_conv_tc(nx, ny, nz, B, X, W, bias, R, Y, Yf, tm, s);
    if (rc != BO_ERR_ARG) return rc;  // else: the mma.sync kernel below
  }
  if (mode == kReluBf16 && cin == 16 && cout == 32)
    return launch_fwd_t<16, 32, true, false, 0>(nx, ny, nz, B, X, W, bias, R, Y, Yf, s);
  if (mode == kReluBf16 && cin == 32 && cout == 32)
    return launch_fwd_t<32, 32, true, false, 0>(nx, ny, nz, B, X, W, bias, R, Y, Yf, s);
  if (mode == kReluResBf16 && cin == 32 && cout == 32)
    return launch_fwd_t<32, 32, true, true, 0>(nx, ny, nz, B, X, W, bias, R, Y, Yf, s);
  if (mode == kLinearOut && cin == 32 && cout == 16)
    return launch_fwd_t<32, 16, false, false, 1>(nx, ny, nz, B, X, W, bias, R, Y, Yf, s);
  if (mode == kLinearF32All && cin == 32 && cout == 32)
    return launch_fwd_t<32, 32, false, false, 2>(nx, ny, nz, B, X, W, bias, R, Y, Yf, s);
  if (mode == kLinearF32All && cin == 16 && cout == 32)
    return launch_fwd_t<16, 32, false, false, 2>(nx, ny, nz, B, X, W, bias, R, Y, Yf, s);
  if (mode == kLinearF32All && cin == 32 && cout == 16)
    return launch_fwd_t<32, 16, false, false, 2>(nx, ny, nz, B, X, W, bias, R, Y, Yf, s);
  return BO_ERR_ARG;
}

template <int CIN, int COUT>
int launch_wgrad_t(int nx, int ny, int nz, int B, const bf16* X, const bf16* D, float* part, float* dW,
                   cudaStream_t s) {
  auto k = k_conv3d_wgrad<CIN, COUT>;
  constexpr size_t smem = wgrad_smem<CIN, COUT>();
  if (cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess)
    return BO_ERR_CUDA;
  const int64_t nbricks = (int64_t)((nx + kBrickX - 1) / kBrickX) * ((ny + kBrickY - 1) / kBrickY) *
                          ((nz + kBrickZ - 1) / kBrickZ) * B;
  int grid = occ_grid((const void*)k, nbricks * kConvThreads, kConvThreads, smem);
  if (grid > kWgMaxBlocks) grid = kWgMaxBlocks;
  (k<<<grid, kConvThreads, smem, s>>>(nx, ny, nz, B, X, D, part), note_launch());
  const int n = 27 * CIN * COUT;
  (k_wgrad_reduce<<<grid_for(n), kThreads, 0, s>>>(part, dW, n, grid), note_launch());
  return cudaGetLastError() == cudaSuccess ? BO_OK : BO_ERR_CUDA;
}

int launch_wgrad(int cin, int cout, int nx, int ny, int nz, int B, const bf16* X, const bf16* D, float* part,
                 float* dW, cudaStream_t s) {
  if (cin == 16 && cout == 32) return launch_wgrad_t<16, 32>(nx, ny, nz, B, X, D, part, dW, s);
  if (cin == 32 && cout == 32) return launch_wgrad_t<32, 32>(nx, ny, nz, B, X, D, part, dW, s);
  if (cin == 32 && cout == 16) return launch_wgrad_t<32, 16>(nx, ny, nz, B, X, D, part, dW, s);
  return BO_ERR_ARG;
}

// Data gradient of a layer: dX (FP32, cin channels) from dY (BF16, cout
// channels): the forward kernel on dY with the flipped, transposed weights.
int launch_dgrad(int cin, int cout, int nx, int ny, int nz, int B, const bf16* dY, const bf16* W, bf16* wd,
                 const float* zero_bias, float* dX, cudaStream_t s) {
  (k_flip_transpose<<<grid_for(27 * cin * cout), kThreads, 0, s>>>(W, wd, cin, cout), note_launch());
  return launch_fwd(cout, cin, kLinearF32All, nx, ny, nz, B, dY, wd, zero_bias, nullptr, nullptr, dX, s);
}

// Weight and bias gradients of a layer from its input X (BF16) and dY
// (FP32; its BF16 copy dY16 is made here unless have16)
int launch_layer_wgrad(int cin, int cout, int nx, int ny, int nz, int B, const bf16* X, const float* dY, bf16* dY16,
                       bool have16, float* part, double* bpart, float* dW, float* db, cudaStream_t s) {
  const int64_t V = (int64_t)nx * ny * nz, BV = B * V;
  if (!have16) (k_f32_to_bf16<<<grid_for(BV * cout), kThreads, 0, s>>>(dY, dY16, BV * cout), note_launch());
  const int rc = launch_wgrad(cin, cout, nx, ny, nz, B, X, dY16, part, dW, s);
  if (rc != BO_OK) return rc;
  const int gb = grid_for(BV * cout, kThreads, kWgMaxBlocks);
  (k_bias_partial<<<gb, kThreads, 0, s>>>(dY, bpart, BV, cout), note_launch());
  (k_bias_reduce<<<1, 32, 0, s>>>(bpart, db, cout, gb), note_launch());
  return cudaGetLastError() == cudaSuccess ? BO_OK : BO_ERR_CUDA;
}

}  // namespace
}  // namespace bo

// ====================================================================== network
// Input conv (16 -> 32, ReLU); 6 residual blocks of two 32 -> 32 convs
// (ReLU, then + block input and ReLU); output conv (32 -> 16, linear;
// channel 0 is the predicted Newton pressure update, 1..2 optionally the
// saturation updates; channels 0..3 are kept in FP32).
namespace {

using bo::bf16;

struct Layer {
  int cin, cout;
  bo::FwdMode mode;
  int64_t woff, boff;  // offsets into the flat parameter vector
};

}  // namespace

struct bo_cnn {
  bo_ctx* ctx;
  int nx, ny, nz, bmax;
  int64_t V;
  std::vector<Layer> layers;
  int64_t nparam;
  float* p = nullptr;       // FP32 master parameters
  float* gr = nullptr;      // gradients of the last backward pass
  float* m = nullptr;       // Adam moments
  float* v = nullptr;
  bf16* p16 = nullptr;      // BF16 copy used by the kernels
  bf16* wd = nullptr;       // flipped/transposed weights (data gradient)
  float* zero_bias = nullptr;
  float* part = nullptr;    // weight-gradient partials
  double* loss_part = nullptr;
  double* h_loss = nullptr;
  std::vector<bf16*> act;   // act[0] input, act[l+1] output of layer l
  float* outf = nullptr;    // FP32 prediction [B][V][4]
  float* gA = nullptr;      // FP32 activation gradients (32 channels)
  float* gB = nullptr;
  float* gC = nullptr;
  bf16* g16 = nullptr;
  double* bpart = nullptr;  // bias-gradient partials
  int64_t step = 0;
};

namespace {

void cnn_free(bo_cnn* n) {
  auto fr = [](void* q) { if (q) cudaFree(q); };
  fr(n->p); fr(n->gr); fr(n->m); fr(n->v); fr(n->p16); fr(n->wd); fr(n->zero_bias); fr(n->part); fr(n->loss_part);
  for (auto a : n->act) fr(a);
  fr(n->outf); fr(n->gA); fr(n->gB); fr(n->gC); fr(n->g16); fr(n->bpart);
  if (n->h_loss) cudaFreeHost(n->h_loss);
}

int cnn_alloc(bo_cnn* n) {
  bool ok = true;
  auto al = [&](size_t bytes) -> void* {
    void* q = nullptr;
    if (ok && cudaMalloc(&q, bytes) != cudaSuccess) { ok = false; return nullptr; }
    return q;
  };
  const int64_t BV = (int64_t)n->bmax * n->V;
  n->p = (float*)al(n->nparam * 4);
  n->gr = (float*)al(n->nparam * 4);
  n->m = (float*)al(n->nparam * 4);
  n->v = (float*)al(n->nparam * 4);
  n->p16 = (bf16*)al(n->nparam * 2);
  n->wd = (bf16*)al((size_t)27 * 32 * 32 * 2);
  n->zero_bias = (float*)al(32 * 4);
  n->part = (float*)al((size_t)bo::kWgMaxBlocks * 27 * 32 * 32 * 4);
  n->loss_part = (double*)al(4096 * sizeof(double));
  if (ok && cudaMallocHost(&n->h_loss, sizeof(double)) != cudaSuccess) ok = false;
  n->act.assign(n->layers.size() + 1, nullptr);
  n->act[0] = (bf16*)al(BV * 16 * 2);
  for (size_t l = 0; l < n->layers.size(); ++l) n->act[l + 1] = (bf16*)al(BV * n->layers[l].cout * 2);
  n->outf = (float*)al(BV * bo::kOutF32 * 4);
  n->gA = (float*)al(BV * 32 * 4);
  n->gB = (float*)al(BV * 32 * 4);
  n->gC = (float*)al(BV * 32 * 4);
  n->g16 = (bf16*)al(BV * 32 * 2);
  n->bpart = (double*)al((size_t)bo::kWgMaxBlocks * 32 * sizeof(double));
  if (!ok) return BO_ERR_OOM;
  cudaStream_t s = n->ctx->stream;
  cudaMemsetAsync(n->m, 0, n->nparam * 4, s);
  cudaMemsetAsync(n->v, 0, n->nparam * 4, s);
  cudaMemsetAsync(n->gr, 0, n->nparam * 4, s);
  cudaMemsetAsync(n->zero_bias, 0, 32 * 4, s);
  return BO_OK;
}

void sync_p16(bo_cnn* n) {
  (bo::k_f32_to_bf16<<<bo::grid_for(n->nparam), bo::kThreads, 0, n->ctx->stream>>>(n->p, n->p16, n->nparam),
   bo::note_launch());
}

int cnn_forward(bo_cnn* n, const bf16* x, int B) {
  cudaStream_t s = n->ctx->stream;
  if (cudaMemcpyAsync(n->act[0], x, (size_t)B * n->V * 16 * 2, cudaMemcpyDeviceToDevice, s) != cudaSuccess)
    return BO_ERR_CUDA;
  for (size_t l = 0; l < n->layers.size(); ++l) {
    const Layer& L = n->layers[l];
    const bf16* R = L.mode == bo::kReluResBf16 ? n->act[l - 1] : nullptr;  // the block's input
    const int rc = bo::launch_fwd(L.cin, L.cout, L.mode, n->nx, n->ny, n->nz, B, n->act[l], n->p16 + L.woff,
                                  n->p + L.boff, R, n->act[l + 1], L.mode == bo::kLinearOut ? n->outf : nullptr, s);
    if (rc != BO_OK) return rc;
  }
  return BO_OK;
}

// Forward, masked MSE loss against target and backward pass into gr.
int cnn_backward(bo_cnn* n, const bf16* x, const float* target, const float* mask, int nout, int B, double* loss) {
  int rc = cnn_forward(n, x, B);
  if (rc != BO_OK) return rc;
  cudaStream_t s = n->ctx->stream;
  const int64_t BV = (int64_t)B * n->V;
  const int nl = (int)n->layers.size();
  const int lgrid = bo::grid_for(BV, bo::kThreads, 1024);
  // d loss / d output (16 channels, only channel 0 nonzero) into gA
  (bo::k_mse<<<lgrid, bo::kThreads, 0, s>>>(n->outf, target, mask, n->gA, 16, nout, BV, 1.0 / (double)BV,
                                             n->loss_part),
   bo::note_launch());
  // output layer (linear)
  const Layer& Lo = n->layers[nl - 1];
  rc = bo::launch_layer_wgrad(Lo.cin, Lo.cout, n->nx, n->ny, n->nz, B, n->act[nl - 1], n->gA, n->g16, false,
                              n->part, n->bpart, n->gr + Lo.woff, n->gr + Lo.boff, s);
  if (rc != BO_OK) return rc;
  rc = bo::launch_dgrad(Lo.cin, Lo.cout, n->nx, n->ny, n->nz, B, n->g16, n->p16 + Lo.woff, n->wd, n->zero_bias,
                        n->gB, s);  // gB = d act[nl-1] (output of the last block)
  if (rc != BO_OK) return rc;
  // residual blocks, last to first: layer a = l - 1, layer b = l
  for (int l = nl - 2; l >= 2; l -= 2) {
    const Layer& Lb = n->layers[l];
    const Layer& La = n->layers[l - 1];
    const int64_t cnt = BV * 32;
    // dpre_b = d out * (out > 0) -> gA
    (bo::k_relu_bwd<<<bo::grid_for(cnt), bo::kThreads, 0, s>>>(n->gB, n->act[l + 1], n->gA, n->g16, cnt),
     bo::note_launch());
    rc = bo::launch_layer_wgrad(Lb.cin, Lb.cout, n->nx, n->ny, n->nz, B, n->act[l], n->gA, n->g16, true,
                                n->part, n->bpart, n->gr + Lb.woff, n->gr + Lb.boff, s);
    if (rc != BO_OK) return rc;
    rc = bo::launch_dgrad(Lb.cin, Lb.cout, n->nx, n->ny, n->nz, B, n->g16, n->p16 + Lb.woff, n->wd, n->zero_bias,
                          n->gC, s);  // gC = d act[l] (output of conv a)
    if (rc != BO_OK) return rc;
    // the residual path: d block input starts as dpre_b (gA); keep it in gB
    cudaMemcpyAsync(n->gB, n->gA, cnt * 4, cudaMemcpyDeviceToDevice, s);
    (bo::k_relu_bwd<<<bo::grid_for(cnt), bo::kThreads, 0, s>>>(n->gC, n->act[l], n->gA, n->g16, cnt),
     bo::note_launch());
    rc = bo::launch_layer_wgrad(La.cin, La.cout, n->nx, n->ny, n->nz, B, n->act[l - 1], n->gA, n->g16, true,
                                n->part, n->bpart, n->gr + La.woff, n->gr + La.boff, s);
    if (rc != BO_OK) return rc;
    rc = bo::launch_dgrad(La.cin, La.cout, n->nx, n->ny, n->nz, B, n->g16, n->p16 + La.woff, n->wd, n->zero_bias,
                          n->gC, s);
    if (rc != BO_OK) return rc;
    (bo::k_add_f32<<<bo::grid_for(cnt), bo::kThreads, 0, s>>>(n->gB, n->gC, cnt), bo::note_launch());
  }
  // input layer: dpre_0 = d act[1] * (act[1] > 0)
  const Layer& Li = n->layers[0];
  (bo::k_relu_bwd<<<bo::grid_for(BV * 32), bo::kThreads, 0, s>>>(n->gB, n->act[1], n->gA, n->g16, BV * 32),
   bo::note_launch());
  rc = bo::launch_layer_wgrad(Li.cin, Li.cout, n->nx, n->ny, n->nz, B, n->act[0], n->gA, n->g16, true,
                              n->part, n->bpart, n->gr + Li.woff, n->gr + Li.boff, s);
  if (rc != BO_OK) return rc;
  if (loss) {
    std::vector<double> lp(lgrid);
    cudaMemcpyAsync(lp.data(), n->loss_part, lgrid * sizeof(double), cudaMemcpyDeviceToHost, s);
    if (cudaStreamSynchronize(s) != cudaSuccess) return BO_ERR_CUDA;
    double t = 0.0;
    for (double q : lp) t += q;
    *loss = t;
  }
  return cudaGetLastError() == cudaSuccess ? BO_OK : BO_ERR_CUDA;
}

}  // namespace

extern "C" {

int bo_cnn_create(bo_ctx* ctx, int nx, int ny, int nz, int max_batch, uint64_t seed, bo_cnn** out) {
  if (!ctx || !out || nx < 1 || ny < 1 || nz < 1 || max_batch < 1 || (int64_t)nx * ny * nz * max_batch > (1ll << 31))
    return BO_ERR_ARG;
  if (cudaSetDevice(ctx->device) != cudaSuccess) return BO_ERR_CUDA;
  bo_cnn* n = new (std::nothrow) bo_cnn();
  if (!n) return BO_ERR_OOM;
  n->ctx = ctx;
  n->nx = nx; n->ny = ny; n->nz = nz; n->bmax = max_batch;
  n->V = (int64_t)nx * ny * nz;
  int64_t off = 0;
  auto add = [&](int cin, int cout, bo::FwdMode mode) {
    Layer L{cin, cout, mode, off, off + 27 * cin * cout};
    off += 27 * cin * cout + cout;
    n->layers.push_back(L);
  };
  add(16, 32, bo::kReluBf16);
  for (int blk = 0; blk < 6; ++blk) {
    add(32, 32, bo::kReluBf16);
    add(32, 32, bo::kReluResBf16);
  }
  add(32, 16, bo::kLinearOut);
  n->nparam = off;
  int rc = cnn_alloc(n);
  if (rc != BO_OK) {
    cnn_free(n);
    delete n;
    return rc;
  }
  // He-normal weights; the second conv of each block and the output conv
  // start small so the untrained network is close to the identity map
  std::vector<float> h(n->nparam, 0.f);
  std::mt19937_64 rng(seed);
  std::normal_distribution<float> nd(0.f, 1.f);
  for (size_t l = 0; l < n->layers.size(); ++l) {
    const Layer& L = n->layers[l];
    float sd = std::sqrt(2.f / (27.f * L.cin));
    if (L.mode == bo::kReluResBf16 || L.mode == bo::kLinearOut) sd *= 0.1f;
    for (int64_t i = 0; i < 27 * L.cin * L.cout; ++i) h[L.woff + i] = sd * nd(rng);
  }
  cudaMemcpyAsync(n->p, h.data(), n->nparam * 4, cudaMemcpyHostToDevice, ctx->stream);
  sync_p16(n);
  if (cudaStreamSynchronize(ctx->stream) != cudaSuccess) {
    cnn_free(n);
    delete n;
    return BO_ERR_CUDA;
  }
  ctx->refs++;
  *out = n;
  return BO_OK;
}

int bo_cnn_destroy(bo_cnn* n) {
  if (!n) return BO_ERR_ARG;
  cudaStreamSynchronize(n->ctx->stream);
  cnn_free(n);
  bo_ctx* c = n->ctx;
  delete n;
  return bo_ctx_destroy(c);
}

int64_t bo_cnn_param_count(const bo_cnn* n) { return n ? n->nparam : -1; }

int bo_cnn_get_params(bo_cnn* n, float* host, int64_t cap) {
  if (!n || !host || cap < n->nparam) return BO_ERR_ARG;
  cudaMemcpyAsync(host, n->p, n->nparam * 4, cudaMemcpyDeviceToHost, n->ctx->stream);
  return cudaStreamSynchronize(n->ctx->stream) == cudaSuccess ? BO_OK : BO_ERR_CUDA;
}

int bo_cnn_set_params(bo_cnn* n, const float* host, int64_t count) {
  if (!n || !host || count != n->nparam) return BO_ERR_ARG;
  cudaMemcpyAsync(n->p, host, n->nparam * 4, cudaMemcpyHostToDevice, n->ctx->stream);
  sync_p16(n);
  return cudaStreamSynchronize(n->ctx->stream) == cudaSuccess ? BO_OK : BO_ERR_CUDA;
}

int bo_cnn_get_grads(bo_cnn* n, float* host, int64_t cap) {
  if (!n || !host || cap < n->nparam) return BO_ERR_ARG;
  cudaMemcpyAsync(host, n->gr, n->nparam * 4, cudaMemcpyDeviceToHost, n->ctx->stream);
  return cudaStreamSynchronize(n->ctx->stream) == cudaSuccess ? BO_OK : BO_ERR_CUDA;
}

int bo_cnn_forward(bo_cnn* n, const uint16_t* x, int batch, float* pred) {
  if (!n || !x || !pred || batch < 1 || batch > n->bmax) return BO_ERR_ARG;
  int rc = cnn_forward(n, reinterpret_cast<const bf16*>(x), batch);
  if (rc != BO_OK) return rc;
  cudaMemcpyAsync(pred, n->outf, (size_t)batch * n->V * bo::kOutF32 * 4, cudaMemcpyDeviceToDevice, n->ctx->stream);
  return cudaGetLastError() == cudaSuccess ? BO_OK : BO_ERR_CUDA;
}

int bo_cnn_backward(bo_cnn* n, const uint16_t* x, const float* target, const float* mask, int nout, int batch,
                    double* loss) {
  if (!n || !x || !target || batch < 1 || batch > n->bmax || nout < 1 || nout > bo::kOutF32) return BO_ERR_ARG;
  return cnn_backward(n, reinterpret_cast<const bf16*>(x), target, mask, nout, batch, loss);
}

int bo_cnn_adam_step(bo_cnn* n, float lr) {
  if (!n || !(lr > 0.f)) return BO_ERR_ARG;
  n->step++;
  const float b1 = 0.9f, b2 = 0.999f;
  const float c1 = 1.f - std::pow(b1, (float)n->step), c2 = 1.f - std::pow(b2, (float)n->step);
  (bo::k_adam<<<bo::grid_for(n->nparam), bo::kThreads, 0, n->ctx->stream>>>(n->p, n->gr, n->m, n->v, n->p16,
                                                                            n->nparam, lr, b1, b2, 1e-8f, c1, c2),
   bo::note_launch());
  return cudaGetLastError() == cudaSuccess ? BO_OK : BO_ERR_CUDA;
}

// ---- single-layer primitives (parity checks and other callers)
int bo_conv3d_forward(bo_ctx* ctx, int nx, int ny, int nz, int batch, int cin, int cout, const uint16_t* x,
                      const uint16_t* w, const float* bias, const uint16_t* residual, int relu, uint16_t* y,
                      float* yf) {
  if (!ctx || !x || !w || !bias || batch < 1 || nx < 1 || ny < 1 || nz < 1 ||
      (int64_t)nx * ny * nz * batch > (1ll << 31))
    return BO_ERR_ARG;
  bo::FwdMode mode;
  if (yf && !y && !relu && !residual) mode = bo::kLinearF32All;
  else if (relu && residual && y) mode = bo::kReluResBf16;
  else if (relu && y) mode = bo::kReluBf16;
  else if (y && yf && !relu && !residual) mode = bo::kLinearOut;
  else return BO_ERR_ARG;
  return bo::launch_fwd(cin, cout, mode, nx, ny, nz, batch, reinterpret_cast<const bf16*>(x),
                        reinterpret_cast<const bf16*>(w), bias, reinterpret_cast<const bf16*>(residual),
                        reinterpret_cast<bf16*>(y), yf, ctx->stream);
}

int bo_conv3d_backward_data(bo_ctx* ctx, int nx, int ny, int nz, int batch, int cin, int cout, const uint16_t* dy,
                            const uint16_t* w, float* dx) {
  if (!ctx || !dy || !w || !dx || batch < 1 || nx < 1 || ny < 1 || nz < 1 ||
      (int64_t)nx * ny * nz * batch > (1ll << 31))
    return BO_ERR_ARG;
  bf16* wd = nullptr;
  float* zb = nullptr;
  if (cudaMalloc(&wd, (size_t)27 * cin * cout * 2) != cudaSuccess) return BO_ERR_OOM;
  if (cudaMalloc(&zb, 64 * 4) != cudaSuccess) { cudaFree(wd); return BO_ERR_OOM; }
  cudaMemsetAsync(zb, 0, 64 * 4, ctx->stream);
  const int rc = bo::launch_dgrad(cin, cout, nx, ny, nz, batch, reinterpret_cast<const bf16*>(dy),
                                  reinterpret_cast<const bf16*>(w), wd, zb, dx, ctx->stream);
  cudaStreamSynchronize(ctx->stream);
  cudaFree(wd);
  cudaFree(zb);
  return rc;
}

int bo_conv3d_backward_weights(bo_ctx* ctx, int nx, int ny, int nz, int batch, int cin, int cout, const uint16_t* x,
                               const float* dy, float* dw, float* db) {
  if (!ctx || !x || !dy || !dw || !db || batch < 1 || nx < 1 || ny < 1 || nz < 1 ||
      (int64_t)nx * ny * nz * batch > (1ll << 31))
    return BO_ERR_ARG;
  if (!((cin == 16 && cout == 32) || (cin == 32 && cout == 32) || (cin == 32 && cout == 16))) return BO_ERR_ARG;
  const int64_t BV = (int64_t)batch * nx * ny * nz;
  bf16* d16 = nullptr;
  float* part = nullptr;
  double* bpart = nullptr;
  bool ok = cudaMalloc(&d16, BV * cout * 2) == cudaSuccess &&
            cudaMalloc(&part, (size_t)bo::kWgMaxBlocks * 27 * cin * cout * 4) == cudaSuccess &&
            cudaMalloc(&bpart, (size_t)bo::kWgMaxBlocks * cout * sizeof(double)) == cudaSuccess;
  int rc = ok ? bo::launch_layer_wgrad(cin, cout, nx, ny, nz, batch, reinterpret_cast<const bf16*>(x), dy, d16, false,
                                       part, bpart, dw, db, ctx->stream)
              : BO_ERR_OOM;
  cudaStreamSynchronize(ctx->stream);
  cudaFree(d16); cudaFree(part); cudaFree(bpart);
  return rc;
}

}  // extern "C"
