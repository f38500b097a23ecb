// 3x3x3 convolution, 32 -> 32 channels, on the fifth-generation tensor
// cores: tcgen05.mma with the accumulator in tensor memory, operands in
// shared memory, input tiles fetched by TMA.  Computes the same as the
// mma.sync forward kernel in cnn.cu for the network's 32 -> 32 layers
// (BF16 in, FP32 accumulate):
//   Y[v][co] = act(bias[co] + sum_t,ci X[v + off(t)][ci] W[t][co][ci] (+ R[v][co]))
// with 'same' zero padding.
//
// Tile = 8 x 16 voxels of one z plane (M = 128 rows of the MMA, row
// m = x + 8 y).  Its input with a one-voxel halo, 10 x 18 x 3 voxels, comes
// in as four TMA boxes of 8 channels each (box {8, 10, 18, 3, 1} over the
// tensor {C, X, Y, Z, batch}; coordinates outside the volume read as zero),
// so shared memory holds it channel-chunk-major: chunk kc is a plane of
// 540 rows of 16 bytes.  In that layout the 128 rows a tap needs are, for
// each 8-voxel run along x, 8 consecutive 16-byte rows: exactly a core
// matrix of the no-swizzle K-major operand layout, with the next run
// (y + 1) 10 rows further on.  So every tap is a shared-memory descriptor
// on the same halo (start address moved by the tap's offset; K-direction
// core-matrix stride = one chunk plane, M-direction stride = 160 bytes),
// and a tile is 27 taps x 2 K-steps = 54 MMAs of 128 x 32 x 16 into one
// 32-column TMEM accumulator.  The weights (N = 32 rows, K = 27 x 32) sit
// in shared memory for the whole persistent CTA.
//
// One CTA of 288 threads (nine warps) per SM, persistent over tiles.  Warp
// 0 issues the TMA copies and the MMAs (one elected thread); three halo
// buffers let the copies of the next tiles overlap the MMAs of the current
// one, and two 32-column TMEM accumulators let the MMAs of one tile overlap
// the epilogue of the previous one.  Warps 1-8 form the epilogue: warp w
// reads TMEM lane quarter w % 4 (the 32 lanes its warp may access) for
// output channels 16 ((w - 1) / 4) .. + 15 with tcgen05.ld, then applies
// bias, residual and ReLU and stores BF16 or FP32.  Every wait on an
// mbarrier is bounded: on expiry the CTA records an error, waits (bounded)
// for its copies in flight, frees its TMEM and returns.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_bf16.h>

#include <cstring>
#include <mutex>

#include "bo_internal.cuh"

namespace bo {
namespace {

using bf16 = __nv_bfloat16;

constexpr int kTcThreads = 288;  // warp 0: TMA + MMA issue; warps 1-8: epilogue
constexpr int kTileX = 8, kTileY = 16;
constexpr int kHX = 10, kHY = 18, kHZ = 3;
constexpr int kHaloRows = kHX * kHY * kHZ;                       // 540
constexpr int kChunkStride = ((kHaloRows * 16 + 127) / 128) * 128;  // 8704: one 8-channel plane, 128-B aligned
constexpr int kChunkBytes = kHaloRows * 16;                       // 8640 written by one TMA box
constexpr int kHaloBuf = 4 * kChunkStride;                        // 34816
constexpr int kWBytes = 27 * 2048;                                // weights, 27 taps x (32 x 32 bf16)
constexpr int kOffW = 0;
constexpr int kOffHalo = kWBytes;                                 // 55296 (128-B aligned)
constexpr int kStages = 3;                                        // halo buffers
constexpr int kOffBar = kOffHalo + kStages * kHaloBuf;            // 159744
constexpr int kSmemBytes = kOffBar + 256 + 1024;                  // barriers, TMEM slot, flag, bias; base-alignment slack
constexpr long kSpinLimit = 1l << 26;
constexpr uint32_t kTxBytes = 4 * kChunkBytes;

__device__ int g_tc_err;  // set by a CTA whose wait expired (read and cleared by bo_tc_status)

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

// shared-memory matrix descriptor: no swizzle, K-major, version 1
__device__ __forceinline__ uint64_t smem_desc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
  return (uint64_t)((saddr >> 4) & 0x3FFF) | ((uint64_t)((lbo >> 4) & 0x3FFF) << 16) |
         ((uint64_t)((sbo >> 4) & 0x3FFF) << 32) | ((uint64_t)1 << 46);
}

// instruction descriptor, kind::f16: D FP32, A and B BF16, both K-major, M = 128, N = 32
constexpr uint32_t kIdesc = (1u << 4) | (1u << 7) | (1u << 10) | ((32u >> 3) << 17) | ((128u >> 4) << 24);

__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity) {
  uint32_t done = 0;
  for (long it = 0; it < kSpinLimit; ++it) {
    asm volatile(
        "{\n.reg .pred p;\nmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\nselp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(done)
        : "r"(bar), "r"(parity)
        : "memory");
    if (done) return true;
  }
  return false;
}

__device__ __forceinline__ void tma_halo(const CUtensorMap* map, uint32_t dst, uint32_t bar, int x0, int y0, int z,
                                         int b) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(bar), "r"(kTxBytes) : "memory");
#pragma unroll
  for (int kc = 0; kc < 4; ++kc) {
    asm volatile(
        "cp.async.bulk.tensor.5d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4, %5, "
        "%6}], [%7];\n" ::"r"(dst + kc * kChunkStride),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(8 * kc), "r"(x0 - 1), "r"(y0 - 1), "r"(z - 1), "r"(b), "r"(bar)
        : "memory");
  }
}

__device__ __forceinline__ void mbar_arrive(uint32_t bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];\n" ::"r"(bar) : "memory");
}

__device__ __forceinline__ void umma_commit(uint32_t bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(bar) : "memory");
}

__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float v[16]) {
  uint32_t r[16];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];\n"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
        "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;\n" ::: "memory");
#pragma unroll
  for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

// OUT 0: Y = ReLU(conv + bias (+ R)) in BF16;  OUT 1: Yf = conv + bias in FP32.
// Warp 0 (one elected thread) feeds TMA and issues the MMAs of tile k into
// TMEM accumulator k & 1 while warps 1-8 drain the other accumulator
// (warp w reads TMEM lanes 32 (w % 4) .. and output channels 16 ((w - 1) / 4) ..).  Tile k's halo sits in buffer
// k % 3: the TMA for tile k + 2 goes out right after tile k's MMAs are
// queued, once tile k - 1's MMAs (queued earlier) have released its buffer,
// so the tensor pipe never drains while waiting for a copy.  mbarriers:
//   full[b]     TMA bytes of halo buffer b landed          (TMA -> MMA)
//   empty[b]    the MMAs reading halo buffer b finished     (MMA -> TMA)
//   accfull[a]  the MMAs into accumulator a finished        (MMA -> epilogue)
//   accempty[a] the epilogue finished reading accumulator a (epilogue -> MMA, 8 arrivals)
// The n-th completion of a barrier has parity n & 1; each side counts the
// completions it has waited for.
template <bool RES, int OUT>
__global__ void __launch_bounds__(kTcThreads, 1) k_conv3d_tc(const __grid_constant__ CUtensorMap xmap, int nx, int ny,
                                                           int nz, int B, const bf16* __restrict__ W,
                                                           const float* __restrict__ bias, const bf16* __restrict__ R,
                                                           bf16* __restrict__ Y, float* __restrict__ Yf) {
  extern __shared__ uint8_t smraw[];
  uint8_t* sm = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smraw) + 1023) & ~uintptr_t(1023));
  uint64_t* bars = reinterpret_cast<uint64_t*>(sm + kOffBar);  // full[3], empty[3], accfull[2], accempty[2]
  uint32_t* tslot = reinterpret_cast<uint32_t*>(sm + kOffBar + 80);
  volatile int* sfail = reinterpret_cast<volatile int*>(sm + kOffBar + 84);
  float* sbias = reinterpret_cast<float*>(sm + kOffBar + 128);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int V = nx * ny * nz;
  const int ntx = (nx + kTileX - 1) / kTileX, nty = (ny + kTileY - 1) / kTileY;
  const int ntiles = ntx * nty * nz * B;
  // weights -> core-matrix layout: tap t, chunk kc = ci / 8, row co: t*2048 + kc*512 + co*16
  for (int i = tid; i < 27 * 32 * 4; i += kTcThreads) {
    const int t = i / 128, rem = i - t * 128, co = rem >> 2, kc = rem & 3;
    const uint4 w = *reinterpret_cast<const uint4*>(W + ((size_t)(t * 32 + co) * 32 + kc * 8));
    *reinterpret_cast<uint4*>(sm + kOffW + t * 2048 + kc * 512 + co * 16) = w;
  }
  if (tid < 32) sbias[tid] = bias[tid];
  uint32_t full[kStages], empty[kStages], accfull[2], accempty[2];
  for (int i = 0; i < kStages; ++i) {
    full[i] = smem_u32(&bars[i]);
    empty[i] = smem_u32(&bars[kStages + i]);
  }
  for (int i = 0; i < 2; ++i) {
    accfull[i] = smem_u32(&bars[2 * kStages + i]);
    accempty[i] = smem_u32(&bars[2 * kStages + 2 + i]);
  }
  if (tid == 0) {
    for (int i = 0; i < kStages; ++i) {
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(full[i]));
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(empty[i]));
    }
    for (int i = 0; i < 2; ++i) {
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(accfull[i]));
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 8;\n" ::"r"(accempty[i]));
    }
    *sfail = 0;
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
  }
  asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
  __syncthreads();
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], 64;\n" ::"r"(smem_u32(tslot)));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n");
  }
  asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
  const uint32_t tmem = *tslot;
  const uint32_t wbase = smem_u32(sm + kOffW);
  const uint32_t hbase = smem_u32(sm + kOffHalo);
  auto tile_xyzb = [&](int t, int& x0, int& y0, int& z, int& b) {
    const int tx = t % ntx;
    t /= ntx;
    const int ty = t % nty;
    t /= nty;
    z = t % nz;
    b = t / nz;
    x0 = tx * kTileX;
    y0 = ty * kTileY;
  };
  const int first = blockIdx.x, step = gridDim.x;
  const int mine = first < ntiles ? (ntiles - 1 - first) / step + 1 : 0;  // tiles of this CTA
  if (warp == 0) {
    if (lane == 0) {
      int fills[kStages] = {0, 0, 0}, uses[kStages] = {0, 0, 0}, commits[kStages] = {0, 0, 0},
          freed[kStages] = {0, 0, 0};
      int acc_waits[2] = {0, 0};
      bool ok = true;
      for (int s = 0; s < 2 && s < mine; ++s) {
        int x0, y0, z, b;
        tile_xyzb(first + s * step, x0, y0, z, b);
        tma_halo(&xmap, hbase + s * kHaloBuf, full[s], x0, y0, z, b);
        ++fills[s];
      }
      for (int k = 0; k < mine && ok; ++k) {
        const int bf = k % kStages, a = k & 1;
        if (*sfail) { ok = false; break; }
        ok = mbar_wait(full[bf], uses[bf] & 1);
        if (!ok) break;
        ++uses[bf];
        if (k >= 2) {  // tile k - 2's epilogue is done with accumulator a
          ok = mbar_wait(accempty[a], acc_waits[a] & 1);
          if (!ok) break;
          ++acc_waits[a];
        }
        asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
        const uint32_t hb = hbase + bf * kHaloBuf;
        const uint32_t dacc = tmem + (uint32_t)(a * 32);
        // The 54 descriptors differ from the buffer's first ones only in
        // their start-address field (address / 16 in the low 14 bits), by
        // offsets that are compile-time constants once the loops are
        // unrolled: one add per MMA instead of building each descriptor
        // (the single issuing thread otherwise spent most of a tile on it).
        const uint64_t da0 = smem_desc(hb, kChunkStride, kHX * 16);
        const uint64_t db0 = smem_desc(wbase, 512, 128);
#pragma unroll
        for (int tap = 0; tap < 27; ++tap) {
          const int dz = tap / 9 - 1, dy = (tap / 3) % 3 - 1, dx = tap % 3 - 1;
          const uint32_t rowoff = ((1 + dz) * kHY + (1 + dy)) * kHX + (1 + dx);
#pragma unroll
          for (int ks = 0; ks < 2; ++ks) {
            const uint64_t da = da0 + (uint64_t)((2 * ks * kChunkStride + rowoff * 16) >> 4);
            const uint64_t db = db0 + (uint64_t)((tap * 2048 + 2 * ks * 512) >> 4);
            const uint32_t acc = (tap | ks) ? 1u : 0u;
            asm volatile(
                "{\n.reg .pred p;\nsetp.ne.u32 p, %4, 0;\n"
                "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(dacc),
                "l"(da), "l"(db), "r"(kIdesc), "r"(acc)
                : "memory");
          }
        }
        umma_commit(empty[bf]);
        umma_commit(accfull[a]);
        ++commits[bf];
        // tile k + 2 goes into the buffer tile k - 1 used, once its MMAs are done
        if (k + 2 < mine) {
          const int nb = (k + 2) % kStages;
          if (commits[nb] > freed[nb]) {
            ok = mbar_wait(empty[nb], freed[nb] & 1);
            if (!ok) break;
            ++freed[nb];
          }
          int x0, y0, z, b;
          tile_xyzb(first + (k + 2) * step, x0, y0, z, b);
          tma_halo(&xmap, hbase + nb * kHaloBuf, full[nb], x0, y0, z, b);
          ++fills[nb];
        }
      }
      if (!ok) {
        *sfail = 1;
        atomicExch(&g_tc_err, 1);
        // copies and MMAs in flight finish before shared and tensor memory go away
        for (int i = 0; i < kStages; ++i) {
          if (fills[i] > uses[i]) mbar_wait(full[i], uses[i] & 1);
          while (commits[i] > freed[i] && mbar_wait(empty[i], freed[i] & 1)) ++freed[i];
        }
      }
    }
    __syncwarp();
  } else {
    // epilogue warps: TMEM lane quarter w % 4, output channels 16 ((w - 1) / 4) .. + 15
    const int quarter = warp & 3, ch0 = 16 * ((warp - 1) >> 2);
    for (int k = 0; k < mine; ++k) {
      const int a = k & 1;
      if (!mbar_wait(accfull[a], (k >> 1) & 1)) {
        *sfail = 1;
        atomicExch(&g_tc_err, 1);
        break;
      }
      asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
      float acc[16];
      tmem_ld16(tmem + ((uint32_t)(quarter * 32) << 16) + (uint32_t)(a * 32 + ch0), acc);
      asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
      __syncwarp();
      if (lane == 0) mbar_arrive(accempty[a]);
      int x0, y0, z, b;
      tile_xyzb(first + k * step, x0, y0, z, b);
      const int m = quarter * 32 + lane;
      const int x = x0 + (m & 7), y = y0 + (m >> 3);
      if (x < nx && y < ny) {
        const size_t o = ((size_t)b * V + x + (size_t)nx * (y + (size_t)ny * z)) * 32 + ch0;
        if (OUT == 0) {
          float rr[16];
          if (RES) {
#pragma unroll
            for (int q = 0; q < 2; ++q) {
              const uint4 u = *reinterpret_cast<const uint4*>(R + o + 8 * q);
              const uint32_t wv[4] = {u.x, u.y, u.z, u.w};
#pragma unroll
              for (int e = 0; e < 4; ++e) {
                rr[8 * q + 2 * e] = __bfloat162float(__ushort_as_bfloat16((unsigned short)(wv[e] & 0xffffu)));
                rr[8 * q + 2 * e + 1] = __bfloat162float(__ushort_as_bfloat16((unsigned short)(wv[e] >> 16)));
              }
            }
          }
#pragma unroll
          for (int q = 0; q < 2; ++q) {
            uint32_t pk[4];
#pragma unroll
            for (int e = 0; e < 4; ++e) {
              const int c0 = 8 * q + 2 * e;
              float y0v = acc[c0] + sbias[ch0 + c0], y1v = acc[c0 + 1] + sbias[ch0 + c0 + 1];
              if (RES) {
                y0v += rr[c0];
                y1v += rr[c0 + 1];
              }
              y0v = fmaxf(y0v, 0.f);
              y1v = fmaxf(y1v, 0.f);
              pk[e] = (uint32_t)__bfloat16_as_ushort(__float2bfloat16_rn(y0v)) |
                      ((uint32_t)__bfloat16_as_ushort(__float2bfloat16_rn(y1v)) << 16);
            }
            *reinterpret_cast<uint4*>(Y + o + 8 * q) = make_uint4(pk[0], pk[1], pk[2], pk[3]);
          }
        } else {
#pragma unroll
          for (int q = 0; q < 4; ++q)
            *reinterpret_cast<float4*>(Yf + o + 4 * q) =
                make_float4(acc[4 * q] + sbias[ch0 + 4 * q], acc[4 * q + 1] + sbias[ch0 + 4 * q + 1],
                            acc[4 * q + 2] + sbias[ch0 + 4 * q + 2], acc[4 * q + 3] + sbias[ch0 + 4 * q + 3]);
        }
      }
      if (*sfail) break;
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
  if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, 64;\n" ::"r"(tmem));
}

PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  static std::once_flag once;
  std::call_once(once, [] {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
  });
  return fn;
}

}  // namespace

// The tensor-core path for a 32 -> 32 layer; BO_ERR_ARG where it does not
// apply (the caller then uses the mma.sync kernel).
//   relu_res: 0 ReLU, 1 ReLU with residual, 2 linear FP32 output (Yf)
int launch_conv_tc(int nx, int ny, int nz, int B, const __nv_bfloat16* X, const __nv_bfloat16* W, const float* bias,
                   const __nv_bfloat16* R, __nv_bfloat16* Y, float* Yf, int mode, cudaStream_t s) {
  if ((reinterpret_cast<uintptr_t>(X) & 15) || (reinterpret_cast<uintptr_t>(W) & 15) ||
      (Y && (reinterpret_cast<uintptr_t>(Y) & 15)) || (R && (reinterpret_cast<uintptr_t>(R) & 15)) ||
      (Yf && (reinterpret_cast<uintptr_t>(Yf) & 15)))
    return BO_ERR_ARG;
  PFN_cuTensorMapEncodeTiled_v12000 enc = encode_fn();
  if (!enc) return BO_ERR_ARG;
  CUtensorMap map;
  const cuuint64_t dims[5] = {32, (cuuint64_t)nx, (cuuint64_t)ny, (cuuint64_t)nz, (cuuint64_t)B};
  const cuuint64_t strides[4] = {64, 64ull * nx, 64ull * nx * ny, 64ull * nx * ny * nz};
  const cuuint32_t box[5] = {8, kHX, kHY, kHZ, 1};
  const cuuint32_t estr[5] = {1, 1, 1, 1, 1};
  if (enc(&map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 5, const_cast<__nv_bfloat16*>(X), dims, strides, box, estr,
          CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
          CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
    return BO_ERR_ARG;
  const int ntiles = ((nx + kTileX - 1) / kTileX) * ((ny + kTileY - 1) / kTileY) * nz * B;
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const int grid = ntiles < sms ? ntiles : sms;
  auto run = [&](auto kern) {
    if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, kSmemBytes) != cudaSuccess)
      return BO_ERR_CUDA;
    (kern<<<grid, kTcThreads, kSmemBytes, s>>>(map, nx, ny, nz, B, W, bias, R, Y, Yf), note_launch());
    return cudaGetLastError() == cudaSuccess ? BO_OK : BO_ERR_CUDA;
  };
  if (mode == 0) return run(k_conv3d_tc<false, 0>);
  if (mode == 1) return run(k_conv3d_tc<true, 0>);
  if (mode == 2) return run(k_conv3d_tc<false, 1>);
  return BO_ERR_ARG;
}

}  // namespace bo

extern "C" int bo_tc_status(void) {
  int h = 0;
  if (cudaMemcpyFromSymbol(&h, bo::g_tc_err, sizeof(int)) != cudaSuccess) return BO_ERR_CUDA;
  if (h) {
    const int z = 0;
    cudaMemcpyToSymbol(bo::g_tc_err, &z, sizeof(int));
    return BO_ERR_TIMEOUT;
  }
  return BO_OK;
}
