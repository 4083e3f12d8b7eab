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

// Bias + GELU epilogue of one layer for this thread's row: Z (fp32, nullable),
// A (bf16 global, nullable) and the bf16 activations into the next operand
// tile (smem, nullable) and into act[64] (registers, rounded to bf16).
__device__ __forceinline__ void tc_epilogue(uint32_t taddr, const float* bias, int row, bool valid, float* Z,
                                            __nv_bfloat16* A, unsigned char* next_tile, float* act) {
#pragma unroll
  for (int c0 = 0; c0 < kH; c0 += 16) {
    float v[16];
    tc_ld16(taddr + (uint32_t)c0, v);
#pragma unroll
    for (int i = 0; i < 16; ++i) {
      const float z = v[i] + bias[c0 + i];
      const __nv_bfloat16 a = __float2bfloat16(gelu(z));
      act[c0 + i] = __bfloat162float(a);
      if (valid && Z) Z[(size_t)row * kH + c0 + i] = z;
      if (valid && A) A[(size_t)row * kH + c0 + i] = a;
      if (next_tile)
        *reinterpret_cast<__nv_bfloat16*>(next_tile + tc_core_off(row & (kTcRows - 1), c0 + i, kTcRows)) = a;
    }
  }
}

// X bf16 [M][76]; Wbf the bf16 parameter copy, theta the fp32 masters (biases);
// outputs (each nullable except P): Z1, Z2 fp32 [M][64], A1, A2 bf16 [M][64],
// P fp32 [M][4].  err (device int) is set to 1 if an mbarrier wait gives up.
__global__ void __launch_bounds__(kTcThreads) k_mlp_forward_tc(int M, const __nv_bfloat16* __restrict__ X,
                                                               const __nv_bfloat16* __restrict__ Wbf,
                                                               const float* __restrict__ theta,
                                                               float* __restrict__ Z1, __nv_bfloat16* __restrict__ A1,
                                                               float* __restrict__ Z2, __nv_bfloat16* __restrict__ A2,
                                                               float* __restrict__ P, int* __restrict__ err) {
  extern __shared__ __align__(1024) unsigned char smem[];
  unsigned char* sA1 = smem + kTcOffA1;
  unsigned char* sB1 = smem + kTcOffB1;
  unsigned char* sA2 = smem + kTcOffA2;
  unsigned char* sB2 = smem + kTcOffB2;
  float* sF = reinterpret_cast<float*>(smem + kTcOffF);  // b1 [64], b2 [64], W3 [4][64], b3 [4]
  uint64_t* mbar = reinterpret_cast<uint64_t*>(smem + kTcOffBar);
  uint32_t* tslot = reinterpret_cast<uint32_t*>(smem + kTcOffBar + 16);
  const int tid = threadIdx.x, warp = tid >> 5;
  const int row0 = blockIdx.x * kTcRows;
  const __nv_bfloat16 zero = __float2bfloat16(0.f);

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
  // operands: the X tile (zero rows past M, zero columns 68..79), W1, W2,
  // biases and layer 3 into shared memory
  for (int e = tid; e < kTcRows * kTcK1; e += kTcThreads) {
    const int r = e / kTcK1, k = e - r * kTcK1;
    __nv_bfloat16 v = zero;
    if (k < kIn && row0 + r < M) v = X[(size_t)(row0 + r) * kIn + k];
    *reinterpret_cast<__nv_bfloat16*>(sA1 + tc_core_off(r, k, kTcRows)) = v;
  }
  for (int e = tid; e < kH * kTcK1; e += kTcThreads) {
    const int n = e / kTcK1, k = e - n * kTcK1;
    const __nv_bfloat16 v = k < kIn ? Wbf[oW1 + n * kIn + k] : zero;
    *reinterpret_cast<__nv_bfloat16*>(sB1 + tc_core_off(n, k, kH)) = v;
  }
  for (int e = tid; e < kH * kH; e += kTcThreads) {
    const int n = e / kH, k = e - n * kH;
    *reinterpret_cast<__nv_bfloat16*>(sB2 + tc_core_off(n, k, kH)) = Wbf[oW2 + n * kH + k];
  }
  for (int e = tid; e < 2 * kH + kOut * kH + kOut; e += kTcThreads) {
    float v;
    if (e < kH) v = theta[ob1 + e];
    else if (e < 2 * kH) v = theta[ob2 + e - kH];
    else if (e < 2 * kH + kOut * kH) v = __bfloat162float(Wbf[oW3 + e - 2 * kH]);
    else v = theta[ob3 + e - 2 * kH - kOut * kH];
    sF[e] = v;
  }
  fence_async_smem();  // the operand stores must be visible to the tensor cores
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tslot;
  const uint32_t mb = smem_u32(mbar);
  const uint32_t taddr = tmem + ((uint32_t)(warp * 32) << 16);  // this warp's 32 lanes
  const int r = tid;                                            // row within the tile
  const int row = row0 + r;
  const bool valid = row < M;
  float act[kH];
  bool ok = true;

  // layer 1: D = X W1^T (K = 80)
  if (tid == 0) tc_layer(tmem, smem_u32(sA1), smem_u32(sB1), kTcK1, mb);
  ok = tc_wait(mb, 0);
  uint32_t pending = 0;  // parity of an MMA batch still to be waited for on the error path
  if (__syncthreads_and(ok)) {
    tc_fence_after();
    // Z1, A1 and the layer-2 operand tile (rows past M are computed and not stored)
    tc_epilogue(taddr, sF, row, valid, Z1, A1, sA2, act);
    fence_async_smem();
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    // layer 2: D = A1 W2^T (K = 64), into the same tensor-memory columns
    if (tid == 0) tc_layer(tmem, smem_u32(sA2), smem_u32(sB2), kH, mb);
    ok = tc_wait(mb, 1);
    if (__syncthreads_and(ok)) {
      tc_fence_after();
      tc_epilogue(taddr, sF + kH, row, valid, Z2, A2, nullptr, act);
      // layer 3 on the CUDA cores from the bf16 activations, FP32 sums in k order
      if (valid) {
#pragma unroll
        for (int o = 0; o < kOut; ++o) {
          float s = 0.f;
          const float* w3 = sF + 2 * kH + o * kH;
#pragma unroll
          for (int k = 0; k < kH; ++k) s = fmaf(act[k], w3[k], s);
          P[(size_t)row * kOut + o] = s + sF[2 * kH + kOut * kH + o];
        }
      }
    } else {
      pending = 2;  // layer 2's batch (parity 1)
    }
  } else {
    pending = 1;  // layer 1's batch (parity 0)
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
