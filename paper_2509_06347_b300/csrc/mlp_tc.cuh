// Forward pass of the per-cell network on the fifth-generation tensor cores:
// layers 1 and 2 (76 -> 64 -> 64, GELU) as tcgen05.mma (kind::f16, BF16 x
// BF16 -> FP32) with the accumulators in tensor memory, layer 3 (64 -> 4) on
// the CUDA cores.  One CTA of 4 warps takes 128 rows (cells), the M of one
// MMA; warp w reads back tensor-memory lanes 32w..32w+31, i.e. rows
// 32w..32w+31, one row per thread.
//
// Operands sit in shared memory in the canonical K-major layout without
// swizzling: the tile is cut into 8 x 8 "core matrices" (8 rows of 16 bytes),
// each stored as 128 contiguous bytes; core (r8, k8) of a tile of R rows sits
// at byte ((k8 * R / 8) + r8) * 128.  Cores adjacent along M/N are therefore
// 128 bytes apart (the descriptor's stride byte offset) and cores adjacent
// along K R/8 * 128 bytes apart (its leading byte offset).  One MMA consumes
// K = 16, two cores along K.
#pragma once
#include <cuda_bf16.h>
#include <cstdint>

#include "mlp.cuh"

namespace cgks {
namespace mlp {

constexpr int kTcRows = 128;                      // rows per CTA = MMA M
constexpr int kTcK1 = 80;                         // layer-1 K: 76 inputs zero-padded to 5 x 16
static_assert(kIn <= kTcK1 && kTcK1 % 16 == 0, "layer-1 K tile");
constexpr int kTcCols = 64;                       // tensor-memory columns: one 128 x 64 FP32 accumulator
constexpr int kTcThreads = 128;
// dynamic shared memory: A1 [128 x 80], A2 [128 x 64], B1 [64 x 80], B2 [64 x 64] (bf16)
constexpr int kTcOffA1 = 0;
constexpr int kTcOffA2 = kTcOffA1 + kTcRows * kTcK1 * 2;   // 20,480
constexpr int kTcOffB1 = kTcOffA2 + kTcRows * kH * 2;      // 36,864
constexpr int kTcOffB2 = kTcOffB1 + kH * kTcK1 * 2;        // 47,104
constexpr int kTcOffF = kTcOffB2 + kH * kH * 2;            // 55,296: fp32 b1, b2 [64 + 64], W3 [4 x 64], b3 [4]
constexpr int kTcOffBar = kTcOffF + (2 * kH + kOut * kH + kOut) * 4;  // 56,848: mbarrier, tensor-memory slot
// The allocation is rounded up to 64 KB: the farthest byte any operand read of
// the MMAs can reach, under either assignment of the two descriptor offsets
// to the K and M/N directions, is 63,743, so every read stays inside it.
constexpr int kTcSmem = 65536;
static_assert(kTcOffBar + 32 <= kTcSmem, "shared-memory layout");
// mbarrier waits give up after this many polls (each poll may suspend for a
// while); the kernel then records an error and returns without hanging
constexpr long long kTcMaxPolls = 1ll << 26;

// byte offset of element (r, k) of a K-major tile of R rows in the core layout
__device__ __forceinline__ uint32_t tc_core_off(int r, int k, int R) {
  return (uint32_t)((((k >> 3) * (R >> 3)) + (r >> 3)) * 128 + (r & 7) * 16 + (k & 7) * 2);
}

// shared-memory matrix descriptor: start, leading (K) and stride (M/N) byte
// offsets in 16-byte units, descriptor version 1 (bits 46-47), no swizzle
__device__ __forceinline__ uint64_t tc_sdesc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
  uint64_t d = (uint64_t)((saddr >> 4) & 0x3FFFu);
  d |= (uint64_t)((lbo >> 4) & 0x3FFFu) << 16;
  d |= (uint64_t)((sbo >> 4) & 0x3FFFu) << 32;
  d |= (uint64_t)1 << 46;
  return d;
}

// instruction descriptor of kind::f16: FP32 accumulator (bits 4-5 = 1), BF16 A
// and B (bits 7-9 = 1, 10-12 = 1), both K-major (bits 15, 16 = 0), N >> 3 at
// bits 17-22, M >> 4 at bits 24-28
__host__ __device__ constexpr uint32_t tc_idesc(int M, int N) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void tc_mma(uint32_t tmem_d, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                       uint32_t accumulate) {
  asm volatile(
      "{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem_d),
      "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
      : "memory");
}

__device__ __forceinline__ void tc_commit(uint32_t mbar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(mbar)
               : "memory");
}

__device__ __forceinline__ bool tc_wait(uint32_t mbar, uint32_t parity) {
  for (long long i = 0; i < kTcMaxPolls; ++i) {
    uint32_t done;
    asm volatile(
        "{\n.reg .pred p;\nmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\nselp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(done)
        : "r"(mbar), "r"(parity)
        : "memory");
    if (done) return true;
  }
  return false;
}

// 16 consecutive FP32 columns of this thread's tensor-memory lane
__device__ __forceinline__ void tc_ld16(uint32_t taddr, float* v) {
  uint32_t r[16];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];\n"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

// Issue the MMAs of one layer (thread 0 only) and commit them to the mbarrier:
// D[128 x 64] = A[128 x K] B[64 x K]^T over K / 16 steps.
__device__ __forceinline__ void tc_layer(uint32_t tmem, uint32_t a_base, uint32_t b_base, int K, uint32_t mbar) {
  constexpr uint32_t idesc = tc_idesc(kTcRows, kH);
  const uint32_t a_lbo = (kTcRows / 8) * 128, b_lbo = (kH / 8) * 128;
  for (int s = 0; s < K / 16; ++s) {
    const uint64_t ad = tc_sdesc(a_base + 2 * s * a_lbo, a_lbo, 128);
    const uint64_t bd = tc_sdesc(b_base + 2 * s * b_lbo, b_lbo, 128);
    tc_mma(tmem, ad, bd, idesc, s > 0 ? 1u : 0u);
  }
  tc_commit(mbar);
}

// Bias + GELU epilogue of one layer for this thread's row (tensor-memory lane
// = row of the tile): Z (fp32, nullable) and A (bf16, nullable) rows in global
// memory, the bf16 activations into the next operand tile (smem, nullable),
// 8 at a time as 16-byte stores, and into act[64] (rounded to bf16).
__device__ __forceinline__ void tc_epilogue(uint32_t taddr, const float* bias, int r, int64_t row, bool valid,
                                            float* Z, __nv_bfloat16* A, unsigned char* next_tile, float* act) {
#pragma unroll
  for (int c0 = 0; c0 < kH; c0 += 16) {
    float v[16];
    tc_ld16(taddr + (uint32_t)c0, v);
    __align__(16) __nv_bfloat16 a[16];
    float z[16];
#pragma unroll
    for (int i = 0; i < 16; ++i) {
      z[i] = v[i] + bias[c0 + i];
      a[i] = __float2bfloat16(gelu(z[i]));
      act[c0 + i] = __bfloat162float(a[i]);
    }
    if (valid && Z) {
      float4* zo = reinterpret_cast<float4*>(Z + row * kH + c0);
#pragma unroll
      for (int i = 0; i < 4; ++i) zo[i] = make_float4(z[4 * i], z[4 * i + 1], z[4 * i + 2], z[4 * i + 3]);
    }
    const uint4* ap = reinterpret_cast<const uint4*>(a);
    if (valid && A) {
      uint4* ao = reinterpret_cast<uint4*>(A + row * kH + c0);
      ao[0] = ap[0];
      ao[1] = ap[1];
    }
    if (next_tile) {
      *reinterpret_cast<uint4*>(next_tile + tc_core_off(r, c0, kTcRows)) = ap[0];
      *reinterpret_cast<uint4*>(next_tile + tc_core_off(r, c0 + 8, kTcRows)) = ap[1];
    }
  }
}

// Persistent: each CTA stages the weights once, then takes 128-row tiles
// t = blockIdx.x, blockIdx.x + gridDim.x, ...  X bf16 [M][76] (rows of 152
// bytes, read as 8-byte words that never straddle a row); Wbf the bf16
// parameter copy, theta the fp32 masters (biases); outputs (each nullable
// except P): Z1, Z2 fp32 [M][64], A1, A2 bf16 [M][64], P fp32 [M][4].  err
// (device int) is set to 1 if an mbarrier wait gives up.
__global__ void __launch_bounds__(kTcThreads) k_mlp_forward_tc(int M, const __nv_bfloat16* __restrict__ X,
                                                               const __nv_bfloat16* __restrict__ Wbf,
                                                               const float* __restrict__ theta,
                                                               float* __restrict__ Z1, __nv_bfloat16* __restrict__ A1,
                                                               float* __restrict__ Z2, __nv_bfloat16* __restrict__ A2,
                                                               float* __restrict__ P, int* __restrict__ err) {
  static_assert(kIn % 4 == 0 && kTcK1 - kIn == 4, "rows of 4-element words, one word of padding");
  constexpr int kW = kIn / 4;  // 8-byte words per row
  extern __shared__ __align__(1024) unsigned char smem[];
  unsigned char* sA1 = smem + kTcOffA1;
  unsigned char* sB1 = smem + kTcOffB1;
  unsigned char* sA2 = smem + kTcOffA2;
  unsigned char* sB2 = smem + kTcOffB2;
  float* sF = reinterpret_cast<float*>(smem + kTcOffF);  // b1 [64], b2 [64], W3 [4][64], b3 [4]
  uint64_t* mbar = reinterpret_cast<uint64_t*>(smem + kTcOffBar);
  uint32_t* tslot = reinterpret_cast<uint32_t*>(smem + kTcOffBar + 16);
  const int tid = threadIdx.x, warp = tid >> 5;
  const int ntiles = (M + kTcRows - 1) / kTcRows;
  const uint2 zero2 = make_uint2(0u, 0u);

  // tensor memory: one accumulator of 64 columns, allocated by warp 0
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tslot)),
                 "r"(kTcCols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  if (tid == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(mbar)) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  // weights once per CTA: W1 [64][76] as 8-byte words (+ one zero word of
  // K padding per row), W2 [64][64] as 16-byte words; biases and layer 3
  for (int j = tid; j < kH * (kW + 1); j += kTcThreads) {
    const int n = j / (kW + 1), q = j - n * (kW + 1);
    const uint2 v = q < kW ? reinterpret_cast<const uint2*>(Wbf + oW1 + n * kIn)[q] : zero2;
    *reinterpret_cast<uint2*>(sB1 + tc_core_off(n, 4 * q, kH)) = v;
  }
  for (int j = tid; j < kH * (kH / 8); j += kTcThreads) {
    const int n = j / (kH / 8), q = j - n * (kH / 8);
    *reinterpret_cast<uint4*>(sB2 + tc_core_off(n, 8 * q, kH)) =
        reinterpret_cast<const uint4*>(Wbf + oW2 + n * kH)[q];
  }
  for (int e = tid; e < 2 * kH + kOut * kH + kOut; e += kTcThreads) {
    float v;
    if (e < kH) v = theta[ob1 + e];
    else if (e < 2 * kH) v = theta[ob2 + e - kH];
    else if (e < 2 * kH + kOut * kH) v = __bfloat162float(Wbf[oW3 + e - 2 * kH]);
    else v = theta[ob3 + e - 2 * kH - kOut * kH];
    sF[e] = v;
  }
  // the K padding word of every input row stays zero for all tiles
  for (int r = tid; r < kTcRows; r += kTcThreads)
    *reinterpret_cast<uint2*>(sA1 + tc_core_off(r, kIn, kTcRows)) = zero2;
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tslot;
  const uint32_t mb = smem_u32(mbar);
  const uint32_t taddr = tmem + ((uint32_t)(warp * 32) << 16);  // this warp's 32 lanes
  const int r = tid;                                            // row within the tile
  float act[kH];
  uint32_t phase = 0;    // completed MMA batches (mbarrier phases)
  uint32_t pending = 0;  // 1 + parity of a batch still in flight after a failed wait
  for (int tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
    const int64_t row0 = (int64_t)tile * kTcRows;
    // the input tile: 8-byte words, consecutive threads on consecutive words
    for (int j = tid; j < kTcRows * kW; j += kTcThreads) {
      const int rr = j / kW, q = j - rr * kW;
      const int64_t g = row0 + rr;
      const uint2 v = g < M ? reinterpret_cast<const uint2*>(X + g * kIn)[q] : zero2;
      *reinterpret_cast<uint2*>(sA1 + tc_core_off(rr, 4 * q, kTcRows)) = v;
    }
    fence_async_smem();  // the operand stores must be visible to the tensor cores
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const int64_t row = row0 + r;
    const bool valid = row < M;
    // layer 1: D = X W1^T (K = 80)
    if (tid == 0) tc_layer(tmem, smem_u32(sA1), smem_u32(sB1), kTcK1, mb);
    if (!__syncthreads_and(tc_wait(mb, phase & 1u))) { pending = 1 + (phase & 1u); break; }
    ++phase;
    tc_fence_after();
    tc_epilogue(taddr, sF, r, row, valid, Z1, A1, sA2, act);
    fence_async_smem();
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    // layer 2: D = A1 W2^T (K = 64), into the same tensor-memory columns
    if (tid == 0) tc_layer(tmem, smem_u32(sA2), smem_u32(sB2), kH, mb);
    if (!__syncthreads_and(tc_wait(mb, phase & 1u))) { pending = 1 + (phase & 1u); break; }
    ++phase;
    tc_fence_after();
    tc_epilogue(taddr, sF + kH, r, row, valid, Z2, A2, nullptr, act);
    // layer 3 on the CUDA cores from the bf16 activations, FP32 sums in k order
    if (valid) {
      float o[kOut];
#pragma unroll
      for (int c = 0; c < kOut; ++c) {
        float s = 0.f;
        const float* w3 = sF + 2 * kH + c * kH;
#pragma unroll
        for (int k = 0; k < kH; ++k) s = fmaf(act[k], w3[k], s);
        o[c] = s + sF[2 * kH + kOut * kH + c];
      }
      *reinterpret_cast<float4*>(P + row * kOut) = make_float4(o[0], o[1], o[2], o[3]);
    }
    // every lane's tensor-memory reads and the tiles are done before the next tile
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
  }
  if (pending) {
    // an mbarrier wait gave up: record it, and wait (bounded) for the MMAs in
    // flight before the tensor memory is freed
    if (tid == 0) atomicExch(err, 1);
    tc_wait(mb, pending - 1);
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 0) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kTcCols) : "memory");
  }
}

}  // namespace mlp
}  // namespace cgks
