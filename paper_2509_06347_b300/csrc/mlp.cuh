// Learned coarse-grid correction: per-cell MLP 76 -> 64 -> 64 -> 4 (GELU),
// BF16 operands on the tensor cores with FP32 accumulation, trained on the GPU
// (forward, backward, Adam on FP32 master weights with BF16 copies).
//
// The dense layers are small (N <= 76, K <= 76) over many rows (cells), so one
// tiled GEMM kernel serves inference, back-propagation and (split over K)
// the weight gradients: 64 x 64 block tiles, 4 warps of 32 x 32, each warp
// issuing mma.sync.m16n8k16 (bf16 x bf16 -> f32) per 16-wide K step.
#pragma once
#include <cuda_bf16.h>
#include <cstdint>

namespace cgks {
namespace mlp {

constexpr int kIn = 76, kH = 64, kOut = 4;
constexpr int kParams = kH * kIn + kH + kH * kH + kH + kOut * kH + kOut;  // 9348
// offsets in the flat parameter vector
constexpr int oW1 = 0, ob1 = oW1 + kH * kIn, oW2 = ob1 + kH, ob2 = oW2 + kH * kH, oW3 = ob2 + kH,
              ob3 = oW3 + kOut * kH;

__device__ __forceinline__ float gelu(float x) { return 0.5f * x * (1.0f + erff(x * 0.70710678118654752f)); }
__device__ __forceinline__ float gelu_grad(float x) {
  const float cdf = 0.5f * (1.0f + erff(x * 0.70710678118654752f));
  return cdf + x * 0.39894228040143268f * __expf(-0.5f * x * x);
}

// epilogue modes
enum : int {
  kEpiStore = 0,      // C (fp32) = acc + bias
  kEpiGeluBf16 = 1,   // C (fp32) = acc + bias, and Abf = bf16(gelu(C))
  kEpiGeluGrad = 2,   // Abf = bf16(acc * gelu'(Z)), Z given (fp32, same shape)
  kEpiPartial = 3     // split-K partial: C[slice] (fp32) = acc
};

struct GemmArgs {
  int M, N, K;
  const __nv_bfloat16* A;  // op(A) is M x K
  int lda, ta;             // ta: A stored K x M
  const __nv_bfloat16* B;  // op(B) is K x N
  int ldb, tb;             // tb: B stored N x K
  float* C;                // M x N (ldc = N), or [slices][M][N] partials
  const float* bias;       // [N] or null
  __nv_bfloat16* Abf;      // M x N bf16 output (epilogues 1, 2)
  const float* Z;          // M x N pre-activation (epilogue 2)
  int epi;
  int k_per_slice;         // split-K (epilogue 3): slice z covers [z*kps, (z+1)*kps)
};

__device__ __forceinline__ void mma_bf16(float* d, const uint32_t* a, const uint32_t* b) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
      "{%0,%1,%2,%3};\n"
      : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
}

// 64 x 64 block tile, K step 16, 128 threads (2 x 2 warps of 32 x 32)
__global__ void __launch_bounds__(128) k_gemm_bf16(GemmArgs g) {
  constexpr int BM = 64, BN = 64, BK = 16, PAD = 8;
  __shared__ __align__(16) __nv_bfloat16 As[BM][BK + PAD];
  __shared__ __align__(16) __nv_bfloat16 Bs[BN][BK + PAD];  // [n][k]
  const int m0 = blockIdx.y * BM, n0 = blockIdx.x * BN;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int wm = (warp >> 1) * 32, wn = (warp & 1) * 32;
  const int gid = lane >> 2, tig = lane & 3;
  int kbeg = 0, kend = g.K;
  if (g.epi == kEpiPartial) {
    kbeg = blockIdx.z * g.k_per_slice;
    kend = min(g.K, kbeg + g.k_per_slice);
  }
  float acc[2][4][4];
#pragma unroll
  for (int i = 0; i < 2; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j)
#pragma unroll
      for (int r = 0; r < 4; ++r) acc[i][j][r] = 0.f;
  const __nv_bfloat16 zero = __float2bfloat16(0.f);
  for (int k0 = kbeg; k0 < kend; k0 += BK) {
    // stage the A and B tiles (bounds-checked, zero fill)
    for (int e = tid; e < BM * BK; e += 128) {
      const int r = e / BK, c = e % BK;
      const int m = m0 + r, k = k0 + c;
      __nv_bfloat16 v = zero;
      if (m < g.M && k < kend) v = g.ta ? g.A[(size_t)k * g.lda + m] : g.A[(size_t)m * g.lda + k];
      As[r][c] = v;
    }
    for (int e = tid; e < BN * BK; e += 128) {
      const int r = e / BK, c = e % BK;
      const int n = n0 + r, k = k0 + c;
      __nv_bfloat16 v = zero;
      if (n < g.N && k < kend) v = g.tb ? g.B[(size_t)n * g.ldb + k] : g.B[(size_t)k * g.ldb + n];
      Bs[r][c] = v;
    }
    __syncthreads();
    uint32_t af[2][4], bfr[4][2];
#pragma unroll
    for (int i = 0; i < 2; ++i) {
      const int r = wm + i * 16 + gid;
      af[i][0] = *reinterpret_cast<const uint32_t*>(&As[r][tig * 2]);
      af[i][1] = *reinterpret_cast<const uint32_t*>(&As[r + 8][tig * 2]);
      af[i][2] = *reinterpret_cast<const uint32_t*>(&As[r][tig * 2 + 8]);
      af[i][3] = *reinterpret_cast<const uint32_t*>(&As[r + 8][tig * 2 + 8]);
    }
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int n = wn + j * 8 + gid;
      bfr[j][0] = *reinterpret_cast<const uint32_t*>(&Bs[n][tig * 2]);
      bfr[j][1] = *reinterpret_cast<const uint32_t*>(&Bs[n][tig * 2 + 8]);
    }
#pragma unroll
    for (int i = 0; i < 2; ++i)
#pragma unroll
      for (int j = 0; j < 4; ++j) mma_bf16(acc[i][j], af[i], bfr[j]);
    __syncthreads();
  }
  // epilogue: accumulator element r of tile (i, j) sits at row gid (+8 for
  // r >= 2), column 2 tig + (r & 1)
#pragma unroll
  for (int i = 0; i < 2; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j)
#pragma unroll
      for (int r = 0; r < 4; ++r) {
        const int m = m0 + wm + i * 16 + gid + (r >= 2 ? 8 : 0);
        const int n = n0 + wn + j * 8 + tig * 2 + (r & 1);
        if (m >= g.M || n >= g.N) continue;
        float v = acc[i][j][r];
        const size_t o = (size_t)m * g.N + n;
        if (g.epi == kEpiPartial) {
          g.C[(size_t)blockIdx.z * g.M * g.N + o] = v;
          continue;
        }
        if (g.epi == kEpiGeluGrad) {
          g.Abf[o] = __float2bfloat16(v * gelu_grad(g.Z[o]));
          continue;
        }
        if (g.bias) v += g.bias[n];
        if (g.C) g.C[o] = v;
        if (g.epi == kEpiGeluBf16) g.Abf[o] = __float2bfloat16(gelu(v));
      }
}

// sum of split-K partials in slice order (deterministic): out[i] = sum_z part[z][i]
__global__ void k_reduce_slices(const float* __restrict__ part, int slices, int n, float* __restrict__ out) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  float s = 0.f;
  for (int z = 0; z < slices; ++z) s += part[(size_t)z * n + i];
  out[i] = s;
}

// column sums of a [rows][cols] fp32 or bf16 matrix, fixed order, one block per column
template <typename T>
__global__ void k_colsum(const T* __restrict__ X, int rows, int cols, float* __restrict__ out) {
  __shared__ float sh[256];
  const int c = blockIdx.x;
  float s = 0.f;
  for (int r = threadIdx.x; r < rows; r += blockDim.x) s += (float)X[(size_t)r * cols + c];
  sh[threadIdx.x] = s;
  __syncthreads();
  for (int st = blockDim.x / 2; st > 0; st >>= 1) {
    if (threadIdx.x < st) sh[threadIdx.x] += sh[threadIdx.x + st];
    __syncthreads();
  }
  if (threadIdx.x == 0) out[c] = sh[0];
}

// dP = 2 (P - Y) / (rows * cols) (fp32 and bf16 copies); per-block squared-error partials
__global__ void k_mse_grad(const float* __restrict__ P, const float* __restrict__ Y, int n, float scale,
                           float* __restrict__ dP, __nv_bfloat16* __restrict__ dPb, float* __restrict__ part) {
  __shared__ float sh[256];
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  float e2 = 0.f;
  if (i < n) {
    // a NaN target marks a row excluded from training (k_mark_nonfinite_rows):
    // it contributes neither loss nor gradient
    const float y = Y[i];
    const float d = y == y ? P[i] - y : 0.f;
    e2 = d * d;
    const float gdp = 2.f * d * scale;
    dP[i] = gdp;
    dPb[i] = __float2bfloat16(gdp);
  }
  sh[threadIdx.x] = e2;
  __syncthreads();
  for (int st = blockDim.x / 2; st > 0; st >>= 1) {
    if (threadIdx.x < st) sh[threadIdx.x] += sh[threadIdx.x + st];
    __syncthreads();
  }
  if (threadIdx.x == 0) part[blockIdx.x] = sh[0];
}

__global__ void k_sum_fixed(const float* __restrict__ part, int n, float scale, float* __restrict__ out) {
  __shared__ float sh[256];
  float s = 0.f;
  for (int i = threadIdx.x; i < n; i += blockDim.x) s += part[i];
  sh[threadIdx.x] = s;
  __syncthreads();
  for (int st = blockDim.x / 2; st > 0; st >>= 1) {
    if (threadIdx.x < st) sh[threadIdx.x] += sh[threadIdx.x + st];
    __syncthreads();
  }
  if (threadIdx.x == 0) *out = sh[0] * scale;
}

// Adam on the FP32 master parameters, refreshing the BF16 compute copies
__global__ void k_adam(int n, const float* __restrict__ g, float* __restrict__ theta, float* __restrict__ m,
                       float* __restrict__ v, __nv_bfloat16* __restrict__ theta_bf, float lr, float b1, float b2,
                       float eps, float bc1, float bc2) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const float gi = g[i];
  const float mi = b1 * m[i] + (1.f - b1) * gi;
  const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
  m[i] = mi;
  v[i] = vi;
  const float t = theta[i] - lr * (mi / bc1) / (sqrtf(vi / bc2) + eps);
  theta[i] = t;
  theta_bf[i] = __float2bfloat16(t);
}

__global__ void k_f32_to_bf16(int n, const float* __restrict__ x, __nv_bfloat16* __restrict__ y) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) y[i] = __float2bfloat16(x[i]);
}

// rows [0, n) of an appended block: a row with a non-finite input or target
// gets zero inputs (a finite forward pass) and NaN targets (no loss, no
// gradient in k_mse_grad)
__global__ void k_mark_nonfinite_rows(int64_t n, __nv_bfloat16* __restrict__ X, float* __restrict__ Y) {
  const int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= n) return;
  bool ok = true;
  for (int c = 0; c < kIn; ++c) ok = ok && isfinite(__bfloat162float(X[r * kIn + c]));
  for (int c = 0; c < kOut; ++c) ok = ok && isfinite(Y[r * kOut + c]);
  if (ok) return;
  for (int c = 0; c < kIn; ++c) X[r * kIn + c] = __float2bfloat16(0.f);
  for (int c = 0; c < kOut; ++c) Y[r * kOut + c] = __int_as_float(0x7fc00000);
}

// gather rows (mini-batch) of the training set
__global__ void k_gather_batch(int b, const int* __restrict__ idx, const __nv_bfloat16* __restrict__ X,
                               const float* __restrict__ Y, __nv_bfloat16* __restrict__ Xb, float* __restrict__ Yb) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= b * kIn) return;
  const int r = t / kIn, c = t % kIn;
  const size_t src = idx[r];
  Xb[t] = X[src * kIn + c];
  if (c < kOut) Yb[(size_t)r * kOut + c] = Y[src * kOut + c];
}

}  // namespace mlp
}  // namespace cgks
