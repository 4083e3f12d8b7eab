// CUDA kernels of one GMG-CGKS V-cycle (sm_103a).
//
// Layout: cells are renumbered colour-major on the host, so every LU-SGS
// colour is a contiguous range [lo, hi) and "neighbour j has a lower colour"
// is simply j < lo.  Per-cell state W, slopes G and polynomial coefficients
// are cell-major (a cell's values contiguous) because they are gathered by
// neighbours and faces; per-cell geometry that only its own thread reads
// (reconstruction operator, moments) is variable-major so warps read it
// coalesced.  Every face flux is evaluated once, by ngp adjacent lanes (one
// per Gauss point) whose results are combined with warp shuffles; cells then
// gather their faces in a fixed order, so residual sums are deterministic and
// need no atomics.
#pragma once
#include <cuda_bf16.h>

#include <cstdint>
#include <type_traits>

#include "physics.cuh"

namespace cgks {

constexpr int kBlock = 256;
constexpr int kClusterBlock = 512;  // threads per block of the cluster kernels

// all threads of the thread-block cluster: arrive with release and wait with
// acquire semantics at cluster scope (the PTX defaults), so that the global
// writes of every block before the barrier are visible to every block after it
__device__ __forceinline__ void cluster_barrier() {
  asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;" ::: "memory");
}

// Row access.  The N values of one cell or face are contiguous, and every
// array is its own cudaMalloc allocation (256-byte aligned), so a row of four
// doubles (2-D states, residuals, face fluxes) starts on a 16-byte boundary
// and moves as two 16-byte vectors, a row of eight doubles (2-D slopes) as
// four, and a row of four floats (FP32 increments) as one.  Rows of five
// (3-D) stay scalar.
template <int N, typename T>
__device__ __forceinline__ void ld_row(const T* __restrict__ p, size_t i, T* x) {
  if constexpr (sizeof(T) == 8 && (N == 4 || N == 8)) {
    const double2* q = reinterpret_cast<const double2*>(p) + i * (N / 2);
#pragma unroll
    for (int k = 0; k < N / 2; ++k) {
      const double2 a = q[k];
      x[2 * k] = a.x;
      x[2 * k + 1] = a.y;
    }
  } else if constexpr (sizeof(T) == 4 && N == 4) {
    const float4 a = reinterpret_cast<const float4*>(p)[i];
    x[0] = a.x;
    x[1] = a.y;
    x[2] = a.z;
    x[3] = a.w;
  } else {
#pragma unroll
    for (int k = 0; k < N; ++k) x[k] = p[i * N + k];
  }
}
template <int N, typename T>
__device__ __forceinline__ void st_row(T* __restrict__ p, size_t i, const T* x) {
  if constexpr (sizeof(T) == 8 && (N == 4 || N == 8)) {
    double2* q = reinterpret_cast<double2*>(p) + i * (N / 2);
#pragma unroll
    for (int k = 0; k < N / 2; ++k) q[k] = make_double2(x[2 * k], x[2 * k + 1]);
  } else if constexpr (sizeof(T) == 4 && N == 4) {
    reinterpret_cast<float4*>(p)[i] = make_float4(x[0], x[1], x[2], x[3]);
  } else {
#pragma unroll
    for (int k = 0; k < N; ++k) p[i * N + k] = x[k];
  }
}

// VAR = 0: simplices (triangles, tetrahedra), every cell with dim + 1 faces
// and every face with the same Gauss points; VAR = 1: 3-D mixed elements
// (tetrahedra, pyramids, prisms, hexahedra), up to 6 faces per cell and 3
// (triangle) or 4 (quadrilateral) Gauss points per face, the counts read per
// cell and per face and the arrays padded to these maxima.
template <int DIM, int VAR = 0>
struct Dims {
  static constexpr int NV = DIM + 2;
  static constexpr int NFC = VAR ? 6 : DIM + 1;             // faces per cell (at most)
  static constexpr int NGP = VAR ? 4 : (DIM == 2 ? 2 : 3);  // Gauss points per face (at most)
  static constexpr int NK = DIM == 2 ? 5 : 9;   // quadratic basis size
  static constexpr int NC = NK + 1;             // polynomial coefficients
  static constexpr int NQ = DIM == 2 ? 3 : 6;   // quadratic monomials
  static constexpr int NCOL = NFC + NFC * DIM;  // operator columns
};

// Fine-level mesh on the device (colour-major cell ids)
struct DevFine {
  int n, nf;
  const int* fL;
  const int* fR;
  const int* ftag;
  const double* fn;   // [nf][dim]
  const double* fS;   // [nf]
  const double* XL;   // [nf][ngp][dim]
  const double* XR;
  const int* cface;          // [n][nfc]
  const signed char* cside;  // [n][nfc]
  const int* cnbr;           // [n][nfc]
  const double* op;          // [nk*ncol][n]  variable-major
  const unsigned char* op_ok;
  const double* avg0;   // [nk][n]
  const double* gg;     // [nfc*dim][n]
  const double* m2;     // [dim*dim][n]
  const double* vol;    // [n]
  const double* bsc;    // [n] |Omega|^(2/dim)
  const double* gpmax;  // [nk][n] max over the cell's face Gauss points of |X^k| (monomials of X = x - centroid)
  const int* grp;       // [n] batch group of each cell (free stream index), or null
  // mixed-element meshes only (null for simplices):
  const signed char* cnf;   // [n] faces of each cell
  const signed char* fngp;  // [nf] Gauss points of each face (3 or 4)
  const double* gw;         // [nf][ngp] their weights (sum 1)
};

// Cell -> face entries for the sweeps and cell-based coarse fluxes (CSR).
struct Topo {
  int n;
  const int* off;            // [n+1]
  const int* nbr;            // neighbour id or -1
  const int* tag;            // boundary tag (0 interior)
  const signed char* side;   // +1 if the cell is the face's left cell
  const double* S;           // face measure
  const double* nrm;         // [e][dim] outward unit normal from the cell
  const double* vol;         // [n]
  const int* face;           // face index of the entry in the level's face list
};

// A level's faces (unique, L -> R orientation; R = -1 on boundary faces)
struct FaceSet {
  int nf;
  const int* fL;
  const int* fR;
  const int* ftag;
  const double* fn;  // [nf][dim]
  const double* fS;  // [nf]
  const int* grp;    // batch group of each cell of the level, or null
};

struct Counters {
  unsigned long long recon_fallback;
  unsigned long long update_halved;
  unsigned long long update_zeroed;
  unsigned long long nonfinite;
};

// ---------------------------------------------------------------------------
// K1: reconstruction (Sec 3) + local time steps, one thread per cell
// ---------------------------------------------------------------------------
template <int DIM>
__device__ __forceinline__ void quad_pq(int q, int& a, int& b) {
  if constexpr (DIM == 2) {
    a = q == 2 ? 1 : 0;
    b = q == 0 ? 0 : 1;
  } else {
    const int pa[6] = {0, 0, 0, 1, 1, 2}, pb[6] = {0, 1, 2, 1, 2, 2};
    a = pa[q];
    b = pb[q];
  }
}

template <int DIM, typename S = double>
__device__ __forceinline__ S eval_poly(const S* c, const S* X) {
  using D = Dims<DIM>;
  S s = c[0];
#pragma unroll
  for (int d = 0; d < DIM; ++d) s += c[1 + d] * X[d];
#pragma unroll
  for (int q = 0; q < D::NQ; ++q) {
    int a, b;
    quad_pq<DIM>(q, a, b);
    s += c[1 + DIM + q] * (X[a] * X[b]);  // the monomial is shared by every variable at X
  }
  return s;
}
template <int DIM, typename S = double>
__device__ __forceinline__ void grad_poly(const S* c, const S* X, S* g) {
  using D = Dims<DIM>;
#pragma unroll
  for (int d = 0; d < DIM; ++d) g[d] = c[1 + d];
#pragma unroll
  for (int q = 0; q < D::NQ; ++q) {
    int a, b;
    quad_pq<DIM>(q, a, b);
    g[a] += c[1 + DIM + q] * X[b];
    g[b] += c[1 + DIM + q] * X[a];
  }
}

template <int DIM, int VAR = 0>
__device__ __forceinline__ void recon_cell(DevFine M, const double* __restrict__ W,
                                           const double* __restrict__ Gr, const double* __restrict__ alpha_prev,
                                           const double* __restrict__ winf, double gamma, double cfl_exp,
                                           double cfl_imp, double gam_hi, double weps, double* __restrict__ coef,
                                           double* __restrict__ dte, double* __restrict__ dti,
                                           Counters* __restrict__ cnt, dword* __restrict__ coef_dw, int c) {
  using D = Dims<DIM, VAR>;
  constexpr int NV = D::NV, NFC = D::NFC, NK = D::NK, NC = D::NC, NCOL = D::NCOL;
  if (c >= M.n) return;
  const int n = M.n;
  const int nf = VAR ? (int)M.cnf[c] : NFC;  // faces of this cell
  double W0[NV];
#pragma unroll
  for (int v = 0; v < NV; ++v) W0[v] = W[(size_t)c * NV + v];
  // neighbour means and slopes (ghosts across boundary faces)
  double Qm[NFC][NV], Dm[NFC][NV][DIM], nrm[NFC][DIM], Sf[NFC];
  int fid[NFC];
  signed char sd[NFC];
#pragma unroll
  for (int m = 0; m < NFC; ++m) {
    if (VAR && m >= nf) {  // padding of a cell with fewer faces: contributes nothing
      fid[m] = 0;
      sd[m] = 0;
      Sf[m] = 0.0;
#pragma unroll
      for (int d = 0; d < DIM; ++d) nrm[m][d] = 0.0;
#pragma unroll
      for (int v = 0; v < NV; ++v) {
        Qm[m][v] = W0[v];
#pragma unroll
        for (int d = 0; d < DIM; ++d) Dm[m][v][d] = 0.0;
      }
      continue;
    }
    const int f = M.cface[(size_t)c * NFC + m];
    fid[m] = f;
    sd[m] = M.cside[(size_t)c * NFC + m];
    Sf[m] = M.fS[f];
#pragma unroll
    for (int d = 0; d < DIM; ++d) nrm[m][d] = sd[m] * M.fn[(size_t)f * DIM + d];
    const int j = M.cnbr[(size_t)c * NFC + m];
    if (j >= 0) {
#pragma unroll
      for (int v = 0; v < NV; ++v) {
        Qm[m][v] = W[(size_t)j * NV + v];
#pragma unroll
        for (int d = 0; d < DIM; ++d) Dm[m][v][d] = Gr[((size_t)j * NV + v) * DIM + d];
      }
    } else {
      const int tag = M.ftag[f];
      double g0[NV][DIM];
#pragma unroll
      for (int v = 0; v < NV; ++v)
#pragma unroll
        for (int d = 0; d < DIM; ++d) g0[v][d] = Gr[((size_t)c * NV + v) * DIM + d];
      const double* wi = winf + NV * (M.grp ? M.grp[c] : 0);
      ghost_state<DIM>(tag, wi, nrm[m], W0, Qm[m], gamma);
      ghost_grad<DIM>(tag, wi, nrm[m], g0, Dm[m]);
    }
  }
  // local time steps: dt = CFL V / sum_f S_f (|u.n| + c)
  {
    double ke = 0.0;
#pragma unroll
    for (int d = 0; d < DIM; ++d) ke += W0[1 + d] * W0[1 + d];
    const double ir = 1.0 / W0[0];
    const double cs = sqrt(gamma * (gamma - 1.0) * (W0[NV - 1] - 0.5 * ke * ir) * ir);
    double sum = 0.0;
#pragma unroll
    for (int m = 0; m < NFC; ++m) {
      double un = 0.0;
#pragma unroll
      for (int d = 0; d < DIM; ++d) un += W0[1 + d] * nrm[m][d];
      sum += Sf[m] * (fabs(un * ir) + cs);
    }
    const double q = M.vol[c] / sum;
    dte[c] = cfl_exp * q;
    dti[c] = cfl_imp * q;
  }
  const bool ok = M.op_ok[c] != 0;
  const double ap = alpha_prev[c];
  // |Omega|^(2|l|/dim - 1) times int over Omega of (D^l p)^2 = |Omega|^(2|l|/dim) <(D^l p)^2>
  const double b1s = M.bsc[c];
  const double b2s = b1s * M.bsc[c];
  double mom[DIM][DIM];
#pragma unroll
  for (int a = 0; a < DIM; ++a)
#pragma unroll
    for (int b = 0; b < DIM; ++b) mom[a][b] = M.m2[(size_t)(a * DIM + b) * n + c];
  double P[NV][NC];
#pragma unroll
  for (int v = 0; v < NV; ++v) {
    double e[NFC];
#pragma unroll
    for (int m = 0; m < NFC; ++m) e[m] = Qm[m][v] - W0[v];
    // p1: Green-Gauss in difference form, scaled by the previous DF
    double g1[DIM];
#pragma unroll
    for (int d = 0; d < DIM; ++d) {
      double s = 0.0;
#pragma unroll
      for (int m = 0; m < NFC; ++m) s += e[m] * M.gg[(size_t)(m * DIM + d) * n + c];
      g1[d] = ap * s;
    }
    if (!ok) {
      P[v][0] = W0[v];
#pragma unroll
      for (int d = 0; d < DIM; ++d) P[v][1 + d] = g1[d];
#pragma unroll
      for (int q = 0; q < D::NQ; ++q) P[v][1 + DIM + q] = 0.0;
      continue;
    }
    // p2: a = Op [e; d]
    double a[NK];
#pragma unroll
    for (int k = 0; k < NK; ++k) {
      const double* o = M.op + (size_t)(k * NCOL) * n + c;
      double s = 0.0;
#pragma unroll
      for (int m = 0; m < NFC; ++m) s += o[(size_t)m * n] * e[m];
#pragma unroll
      for (int m = 0; m < NFC; ++m)
#pragma unroll
        for (int d = 0; d < DIM; ++d) s += o[(size_t)(NFC + m * DIM + d) * n] * Dm[m][v][d];
      a[k] = s;
    }
    double c2[NC];
    double c0 = W0[v];
#pragma unroll
    for (int k = 0; k < NK; ++k) c0 -= a[k] * M.avg0[(size_t)k * n + c];
    c2[0] = c0;
#pragma unroll
    for (int k = 0; k < NK; ++k) c2[1 + k] = a[k];
    // smoothness indicators (sum over |l| of |Omega|^(2|l|/dim - 1) int (D^l p)^2)
    double b1 = 0.0;
#pragma unroll
    for (int d = 0; d < DIM; ++d) b1 += g1[d] * g1[d];
    b1 *= b1s;
    double H[DIM][DIM];
#pragma unroll
    for (int q = 0; q < D::NQ; ++q) {
      int pa, pb;
      quad_pq<DIM>(q, pa, pb);
      H[pa][pb] = (pa == pb ? 2.0 : 1.0) * a[DIM + q];
      H[pb][pa] = H[pa][pb];
    }
    double b2 = 0.0, b2q = 0.0;
#pragma unroll
    for (int d = 0; d < DIM; ++d) {
      double s = a[d] * a[d];
#pragma unroll
      for (int x = 0; x < DIM; ++x)
#pragma unroll
        for (int y = 0; y < DIM; ++y) s += H[d][x] * mom[x][y] * H[d][y];
      b2 += s;
#pragma unroll
      for (int x = d; x < DIM; ++x) b2q += H[d][x] * H[d][x];
    }
    b2 = b1s * b2 + b2s * b2q;
    // w_H ~ gam_hi (1 + tz / (b2 + eps)), w_L ~ gl (1 + tz / (b1 + eps)), normalised;
    // both multiplied by (b1 + eps)(b2 + eps) so that one reciprocal remains;
    // fh = w_H / gam_hi
    const double gl = 1.0 - gam_hi;
    const double tz = fabs(b2 - b1);
    const double e1 = b1 + weps, e2 = b2 + weps;
    const double xh = (e2 + tz) * e1;
    double wl = gl * (e1 + tz) * e2;
    const double iw = 1.0 / (gam_hi * xh + wl);
    wl *= iw;
    const double fh = xh * iw;
    P[v][0] = fh * (c2[0] - gl * W0[v]) + wl * W0[v];
#pragma unroll
    for (int d = 0; d < DIM; ++d) P[v][1 + d] = fh * (c2[1 + d] - gl * g1[d]) + wl * g1[d];
#pragma unroll
    for (int q = 0; q < D::NQ; ++q) P[v][1 + DIM + q] = fh * c2[1 + DIM + q];
  }
  // positivity at the cell's face Gauss points (reading: first-order fallback).
  // A sufficient condition first: with |X^k| <= gpmax_k at those points,
  // |P_v - c0_v| <= B_v = sum_k |c_k| gpmax_k, so rho >= c0_rho - B_rho and
  // p > 0 follows from E_min - |m|_max^2 / (2 rho_min) > 0; only the cells it
  // does not clear evaluate every Gauss point (same outcome, less FP64 work).
  bool sure = false;
  {
    double B[NV];
#pragma unroll
    for (int v = 0; v < NV; ++v) {
      double b = 0.0;
#pragma unroll
      for (int k = 0; k < NK; ++k) b += fabs(P[v][1 + k]) * M.gpmax[(size_t)k * n + c];
      B[v] = b;
    }
    const double rmin = P[0][0] - B[0];
    if (rmin > 1e-12 * fabs(P[0][0])) {
      double mm = 0.0;
#pragma unroll
      for (int d = 0; d < DIM; ++d) {
        const double t = fabs(P[1 + d][0]) + B[1 + d];
        mm += t * t;
      }
      const double emin = P[NV - 1][0] - B[NV - 1];
      sure = emin * rmin - 0.5 * mm > 1e-12 * fabs(P[NV - 1][0]) * rmin;  // rmin > 0 here
    }
  }
  bool bad = false;
#pragma unroll 1
  for (int m = 0; m < nf && !bad && !sure; ++m) {
    const double* X = (sd[m] > 0 ? M.XL : M.XR) + (size_t)fid[m] * D::NGP * DIM;
    const int ng = VAR ? (int)M.fngp[fid[m]] : D::NGP;
#pragma unroll
    for (int g = 0; g < D::NGP; ++g) {
      if (VAR && g >= ng) break;
      double Wp[NV];
#pragma unroll
      for (int v = 0; v < NV; ++v) Wp[v] = eval_poly<DIM>(P[v], X + g * DIM);
      double ke = 0.0;
#pragma unroll
      for (int d = 0; d < DIM; ++d) ke += Wp[1 + d] * Wp[1 + d];
      // p > 0 as rho E - |rho u|^2 / 2 > 0 once rho > 0 (no division)
      if (!(Wp[0] > 0.0) || !(Wp[NV - 1] * Wp[0] - 0.5 * ke > 0.0)) bad = true;
    }
  }
  if (bad) {
    atomicAdd(&cnt->recon_fallback, 1ull);
#pragma unroll
    for (int v = 0; v < NV; ++v) {
      P[v][0] = W0[v];
#pragma unroll
      for (int k = 1; k < NC; ++k) P[v][k] = 0.0;
    }
  }
  double* out = coef + (size_t)c * NV * NC;
#pragma unroll
  for (int v = 0; v < NV; ++v)
#pragma unroll
    for (int k = 0; k < NC; ++k) out[v * NC + k] = P[v][k];
  if (coef_dw) {  // the same coefficients as double-words for the FP32-pipe flux
    dword* od = coef_dw + (size_t)c * NV * NC;
#pragma unroll
    for (int v = 0; v < NV; ++v)
#pragma unroll
      for (int k = 0; k < NC; ++k) od[v * NC + k] = dword(P[v][k]);
  }
}

// One thread per cell.  In 2-D the grid holds only the resident blocks and
// warps loop over tasks of 32 cells, task t in block t mod gridDim.x, so that
// every SM gets the same number of cells to within one task (a grid of one
// thread per cell leaves a partial last wave on a few SMs).  3-D meshes span
// hundreds of waves, and the loop would cost the 3-D kernel spills: there the
// grid has one thread per cell.
template <int DIM, int VAR = 0>
__global__ void __launch_bounds__(kBlock) k_recon(DevFine M, const double* __restrict__ W,
                                                  const double* __restrict__ Gr, const double* __restrict__ alpha_prev,
                                                  const double* __restrict__ winf, double gamma, double cfl_exp,
                                                  double cfl_imp, double gam_hi, double weps, double* __restrict__ coef,
                                                  double* __restrict__ dte, double* __restrict__ dti,
                                                  Counters* __restrict__ cnt, dword* __restrict__ coef_dw) {
  if constexpr (DIM == 3) {
    recon_cell<DIM, VAR>(M, W, Gr, alpha_prev, winf, gamma, cfl_exp, cfl_imp, gam_hi, weps, coef, dte, dti, cnt,
                         coef_dw, blockIdx.x * blockDim.x + threadIdx.x);
  } else {
    const int lane = threadIdx.x & 31;
    const int ntask = (M.n + 31) / 32;
    const int nwarp = gridDim.x * (blockDim.x >> 5);
    for (int task = (threadIdx.x >> 5) * gridDim.x + blockIdx.x; task < ntask; task += nwarp)
      recon_cell<DIM>(M, W, Gr, alpha_prev, winf, gamma, cfl_exp, cfl_imp, gam_hi, weps, coef, dte, dti, cnt, coef_dw,
                      task * 32 + lane);
  }
}

// double-word arithmetic check: a, b split into double-words, then
// out[i] = (a + b, a - b, a * b, a / b, sqrt(a), exp(-a), erfc(b)) returned in FP64
__global__ void k_dword_selftest(int n, const double* __restrict__ a, const double* __restrict__ b,
                                 double* __restrict__ out) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const dword x(a[i]), y(b[i]);
  double* o = out + (size_t)i * 7;
  o[0] = static_cast<double>(x + y);
  o[1] = static_cast<double>(x - y);
  o[2] = static_cast<double>(x * y);
  o[3] = static_cast<double>(x / y);
  o[4] = static_cast<double>(sqrt(x));
  o[5] = static_cast<double>(exp(-x));
  o[6] = static_cast<double>(erfc(y));
}

// out[i] = (erfc(x) as the flux computes it, erfcx(|x|), exp(-|x|), and the
// CUDA library's erfc(x) and exp(-|x|)) for the check of special.cuh
__global__ void k_special_selftest(int n, const double* __restrict__ x, double* __restrict__ out) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const double v = x[i];
  double* o = out + (size_t)i * 5;
  o[0] = erfc_with_exp(v, exp_neg(-v * v));
  o[1] = erfcx_pos(fabs(v));
  o[2] = exp_neg(-fabs(v));
  o[3] = erfc(v);
  o[4] = exp(-fabs(v));
}

// ---------------------------------------------------------------------------
// K2: gas-kinetic flux, one lane per (face, Gauss point)
// ---------------------------------------------------------------------------
// value and gradient of one variable's polynomial at a Gauss point; a shared
// call in the double-word flux (see OutOfLine)
template <int DIM, typename S>
__device__ __forceinline__ void eval_grad(const S* c, const S* x, S& W, S* g) {
  using D = Dims<DIM>;
  S cc[D::NC];
  if constexpr (std::is_same<S, double>::value && D::NC % 2 == 0) {
    // 16-byte loads: every variable's coefficient row starts on a 16-byte
    // boundary (rows of NV * NC doubles, NC even, from 256-byte aligned buffers)
    const double2* c2 = reinterpret_cast<const double2*>(c);
#pragma unroll
    for (int k = 0; k < D::NC / 2; ++k) {
      const double2 t = __ldg(c2 + k);
      cc[2 * k] = t.x;
      cc[2 * k + 1] = t.y;
    }
  } else {
#pragma unroll
    for (int k = 0; k < D::NC; ++k) cc[k] = c[k];
  }
  W = eval_poly<DIM, S>(cc, x);
  grad_poly<DIM, S>(cc, x, g);
}
template <int DIM, typename S>
__device__ __noinline__ void eval_grad_ool(const S* c, const S* x, S& W, S* g) {
  eval_grad<DIM, S>(c, x, W, g);
}
template <int DIM, typename S>
__device__ __forceinline__ void eval_grad_c(const S* c, const S* x, S& W, S* g) {
  if constexpr (OutOfLine<S>::value) eval_grad_ool<DIM, S>(c, x, W, g);
  else eval_grad<DIM, S>(c, x, W, g);
}

// warp shuffle of a flux-code scalar
__device__ __forceinline__ double shfl_s(double x, int src) { return __shfl_sync(0xffffffffu, x, src); }
__device__ __forceinline__ dword shfl_s(dword x, int src) {
  return dword(__shfl_sync(0xffffffffu, x.hi, src), __shfl_sync(0xffffffffu, x.lo, src));
}

// One task of the gas-kinetic face flux: FPW faces, NGP lanes per face.
template <int DIM, bool POINT, typename S>
__device__ __forceinline__ void flux_task(const DevFine& M, const S* __restrict__ coef, const double* __restrict__ dte,
                                          const double* __restrict__ winf, const PhysT<S>& P, double gamma,
                                          double* __restrict__ Fface, double* __restrict__ Wface,
                                          double* __restrict__ aface, const double* __restrict__ Wc,
                                          double* __restrict__ rface, int task, int lane) {
  using D = Dims<DIM>;
  constexpr int NV = D::NV, NC = D::NC, NGP = D::NGP;
  constexpr int FPW = 32 / NGP;  // faces per warp
  const int g = lane % NGP;
  const int f = task * FPW + lane / NGP;
  const bool active = lane < FPW * NGP && f < M.nf;
  S Fs[NV], Ws[NV], af = S(1.0);
#pragma unroll
  for (int v = 0; v < NV; ++v) { Fs[v] = S(0.0); Ws[v] = S(0.0); }
  if (active) {
    const int L = M.fL[f], R = M.fR[f];
    S n[DIM];
#pragma unroll
    for (int d = 0; d < DIM; ++d) n[d] = S(M.fn[(size_t)f * DIM + d]);
    const Frame<DIM, S> fr = make_frame<DIM, S>(n);
    S Wl[NV], gl[NV][DIM], Wr[NV], gr[NV][DIM];
    {
      const double* X = M.XL + ((size_t)f * NGP + g) * DIM;
      S x[DIM];
#pragma unroll
      for (int d = 0; d < DIM; ++d) x[d] = S(X[d]);
      const S* c = coef + (size_t)L * NV * NC;
#pragma unroll
      for (int v = 0; v < NV; ++v) eval_grad_c<DIM, S>(c + v * NC, x, Wl[v], gl[v]);
    }
    double dt = dte[L];
    if (R >= 0) {
      const double* X = M.XR + ((size_t)f * NGP + g) * DIM;
      S x[DIM];
#pragma unroll
      for (int d = 0; d < DIM; ++d) x[d] = S(X[d]);
      const S* c = coef + (size_t)R * NV * NC;
#pragma unroll
      for (int v = 0; v < NV; ++v) eval_grad_c<DIM, S>(c + v * NC, x, Wr[v], gr[v]);
      dt = fmin(dt, dte[R]);
    } else {
      const int tag = M.ftag[f];
      const double* wd = winf + NV * (M.grp ? M.grp[L] : 0);
      S wi[NV];
#pragma unroll
      for (int v = 0; v < NV; ++v) wi[v] = S(wd[v]);
      ghost_state<DIM, S>(tag, wi, n, Wl, Wr, P.gamma);
      ghost_grad<DIM, S>(tag, wi, n, gl, gr);
    }
    S wl[NV], wr[NV], Gl[DIM][NV], Gr[DIM][NV], Fl[NV], Wt[NV];
    to_local<DIM, S>(fr, Wl, wl);
    to_local<DIM, S>(fr, Wr, wr);
    grad_to_local<DIM, S>(fr, gl, Gl);
    grad_to_local<DIM, S>(fr, gr, Gr);
    af = gks_flux<DIM, POINT, S>(P, wl, Gl, wr, Gr, S(dt), Fl, Wt);
    S Fg[NV], Wg[NV];
    to_global<DIM, S>(fr, Fl, Fg);
    to_global<DIM, S>(fr, Wt, Wg);
    const S w = S(M.fS[f] * (1.0 / NGP));  // equal Gauss weights on every face
#pragma unroll
    for (int v = 0; v < NV; ++v) { Fs[v] = w * Fg[v]; Ws[v] = w * Wg[v]; }
  }
  // combine the NGP lanes of a face (group leader = lane with g == 0)
  const int leader = lane - g;
#pragma unroll
  for (int k = 1; k < NGP; ++k) {
    const int src = leader + k;
#pragma unroll
    for (int v = 0; v < NV; ++v) {
      const S fo = shfl_s(Fs[v], src < 32 ? src : lane);
      const S wo = shfl_s(Ws[v], src < 32 ? src : lane);
      if (g == 0) { Fs[v] += fo; Ws[v] += wo; }
    }
    const S ao = shfl_s(af, src < 32 ? src : lane);
    if (g == 0) af *= ao;
  }
  if (active && g == 0) {
#pragma unroll
    for (int v = 0; v < NV; ++v) {
      Fface[(size_t)f * NV + v] = static_cast<double>(Fs[v]);
      if (POINT) Wface[(size_t)f * NV + v] = static_cast<double>(Ws[v]);
    }
    aface[f] = static_cast<double>(af);
  }
  if (rface && active && g == 0) {
    // spectral radius of the LU-SGS splitting at the mean of the cell means
    const int L = M.fL[f], R = M.fR[f];
    double n[DIM], WL[NV], WR[NV];
#pragma unroll
    for (int d = 0; d < DIM; ++d) n[d] = M.fn[(size_t)f * DIM + d];
#pragma unroll
    for (int v = 0; v < NV; ++v) WL[v] = Wc[(size_t)L * NV + v];
    if (R >= 0) {
#pragma unroll
      for (int v = 0; v < NV; ++v) WR[v] = Wc[(size_t)R * NV + v];
    } else {
      ghost_state<DIM>(M.ftag[f], winf + NV * (M.grp ? M.grp[L] : 0), n, WL, WR, gamma);
    }
    rface[f] = spectral_radius<DIM, double>(gamma, WL, WR, n);
  }
}

// All NGP Gauss points of face f in one lane, summed in the order the lane
// groups of flux_task use.  For the 3-point faces of 3-D meshes: 32 faces per
// warp use every lane, where 3 lanes per face leave 2 of 32 idle, and the
// per-face work (indices, frame, spectral radius) runs on every lane.
template <int DIM, bool POINT, typename S, int VAR = 0>
__device__ __forceinline__ void flux_face(const DevFine& M, const S* __restrict__ coef, const double* __restrict__ dte,
                                          const double* __restrict__ winf, const PhysT<S>& P, double gamma,
                                          double* __restrict__ Fface, double* __restrict__ Wface,
                                          double* __restrict__ aface, const double* __restrict__ Wc,
                                          double* __restrict__ rface, int f) {
  using D = Dims<DIM, VAR>;
  constexpr int NV = D::NV, NC = D::NC, NGP = D::NGP;
  if (f >= M.nf) return;
  const int L = M.fL[f], R = M.fR[f];
  const int ng = VAR ? (int)M.fngp[f] : NGP;  // Gauss points of this face
  S n[DIM];
#pragma unroll
  for (int d = 0; d < DIM; ++d) n[d] = S(M.fn[(size_t)f * DIM + d]);
  const Frame<DIM, S> fr = make_frame<DIM, S>(n);
  double dt = dte[L];
  if (R >= 0) dt = fmin(dt, dte[R]);
  // equal Gauss weights on every simplex face; per-point weights on mixed meshes
  const S w0 = S(M.fS[f] * (1.0 / NGP));
  S Fs[NV], Ws[NV], af = S(1.0);
#pragma unroll
  for (int v = 0; v < NV; ++v) { Fs[v] = S(0.0); Ws[v] = S(0.0); }
#pragma unroll 1
  for (int g = 0; g < ng; ++g) {
    const S w = VAR ? S(M.fS[f] * M.gw[(size_t)f * NGP + g]) : w0;
    S Wl[NV], gl[NV][DIM], Wr[NV], gr[NV][DIM];
    {
      const double* X = M.XL + ((size_t)f * NGP + g) * DIM;
      S x[DIM];
#pragma unroll
      for (int d = 0; d < DIM; ++d) x[d] = S(X[d]);
      const S* c = coef + (size_t)L * NV * NC;
#pragma unroll
      for (int v = 0; v < NV; ++v) eval_grad_c<DIM, S>(c + v * NC, x, Wl[v], gl[v]);
    }
    if (R >= 0) {
      const double* X = M.XR + ((size_t)f * NGP + g) * DIM;
      S x[DIM];
#pragma unroll
      for (int d = 0; d < DIM; ++d) x[d] = S(X[d]);
      const S* c = coef + (size_t)R * NV * NC;
#pragma unroll
      for (int v = 0; v < NV; ++v) eval_grad_c<DIM, S>(c + v * NC, x, Wr[v], gr[v]);
    } else {
      const int tag = M.ftag[f];
      const double* wd = winf + NV * (M.grp ? M.grp[L] : 0);
      S wi[NV];
#pragma unroll
      for (int v = 0; v < NV; ++v) wi[v] = S(wd[v]);
      ghost_state<DIM, S>(tag, wi, n, Wl, Wr, P.gamma);
      ghost_grad<DIM, S>(tag, wi, n, gl, gr);
    }
    S wl[NV], wr[NV], Gl[DIM][NV], Gr[DIM][NV], Fl[NV], Wt[NV];
    to_local<DIM, S>(fr, Wl, wl);
    to_local<DIM, S>(fr, Wr, wr);
    grad_to_local<DIM, S>(fr, gl, Gl);
    grad_to_local<DIM, S>(fr, gr, Gr);
    af *= gks_flux<DIM, POINT, S>(P, wl, Gl, wr, Gr, S(dt), Fl, Wt);
    S Fg[NV], Wg[NV];
    to_global<DIM, S>(fr, Fl, Fg);
    to_global<DIM, S>(fr, Wt, Wg);
#pragma unroll
    for (int v = 0; v < NV; ++v) {
      Fs[v] += w * Fg[v];
      if (POINT) Ws[v] += w * Wg[v];
    }
  }
#pragma unroll
  for (int v = 0; v < NV; ++v) {
    Fface[(size_t)f * NV + v] = static_cast<double>(Fs[v]);
    if (POINT) Wface[(size_t)f * NV + v] = static_cast<double>(Ws[v]);
  }
  aface[f] = static_cast<double>(af);
  if (rface) {
    // spectral radius of the LU-SGS splitting at the mean of the cell means
    double nd[DIM], WL[NV], WR[NV];
#pragma unroll
    for (int d = 0; d < DIM; ++d) nd[d] = M.fn[(size_t)f * DIM + d];
#pragma unroll
    for (int v = 0; v < NV; ++v) WL[v] = Wc[(size_t)L * NV + v];
    if (R >= 0) {
#pragma unroll
      for (int v = 0; v < NV; ++v) WR[v] = Wc[(size_t)R * NV + v];
    } else {
      ghost_state<DIM>(M.ftag[f], winf + NV * (M.grp ? M.grp[L] : 0), nd, WL, WR, gamma);
    }
    rface[f] = spectral_radius<DIM, double>(gamma, WL, WR, nd);
  }
}

// Gas-kinetic face flux.  S = double: FP64; S = dword: the same arithmetic in
// double-word on the FP32 pipes (coefficients read as double-word, geometry and
// time step converted once per Gauss point, results returned in FP64).
// In FP64 each warp loops over tasks of FPW faces.  The grid holds only the
// blocks that are resident at once, and task t goes to block t mod gridDim.x,
// so every SM gets the same number of tasks to within one (a grid of one block
// per face group leaves a partial last wave on a few SMs).  The double-word
// variant, whose registers are capped for two blocks per SM, keeps one task
// per warp: the loop costs it stack space and spills.
template <int DIM, bool POINT, typename S = double, int VAR = 0>
__global__ void __launch_bounds__(kBlock, OutOfLine<S>::value ? 2 : 1) k_flux(DevFine M, const S* __restrict__ coef,
                                                 const double* __restrict__ dte, const double* __restrict__ winf,
                                                 PhysT<S> P, double gamma, double* __restrict__ Fface,
                                                 double* __restrict__ Wface, double* __restrict__ aface,
                                                 const double* __restrict__ Wc, double* __restrict__ rface) {
  static_assert(VAR == 0 || (DIM == 3 && !OutOfLine<S>::value), "mixed elements: 3-D, FP64 flux");
  constexpr int FPW = 32 / Dims<DIM>::NGP;
  const int lane = threadIdx.x & 31;
  const int ntask = (M.nf + FPW - 1) / FPW;
  if constexpr (OutOfLine<S>::value) {
    const int task = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (task < ntask) flux_task<DIM, POINT, S>(M, coef, dte, winf, P, gamma, Fface, Wface, aface, Wc, rface, task, lane);
  } else if constexpr (DIM == 3) {
    // one face per lane, tasks of 32 faces
    const int nwarp = gridDim.x * (blockDim.x >> 5);
    const int nt = (M.nf + 31) / 32;
    for (int task = (threadIdx.x >> 5) * gridDim.x + blockIdx.x; task < nt; task += nwarp)
      flux_face<DIM, POINT, S, VAR>(M, coef, dte, winf, P, gamma, Fface, Wface, aface, Wc, rface, task * 32 + lane);
  } else {
    const int nwarp = gridDim.x * (blockDim.x >> 5);
    for (int task = (threadIdx.x >> 5) * gridDim.x + blockIdx.x; task < ntask; task += nwarp)
      flux_task<DIM, POINT, S>(M, coef, dte, winf, P, gamma, Fface, Wface, aface, Wc, rface, task, lane);
  }
}

// ---------------------------------------------------------------------------
// LU-SGS diagonal with DF relaxation (Sec 4.3):
// D_i = alpha (V/dt_imp + 1/2 sum S r) + (1 - alpha) V/dt_exp
// ---------------------------------------------------------------------------
template <int DIM>
__device__ __forceinline__ double lusgs_diag(const Topo& T, int c, const double* rface, double alpha, double dte,
                                             double dti) {
  double sr = 0.0;
  for (int e = T.off[c]; e < T.off[c + 1]; ++e) sr += T.S[e] * rface[T.face[e]];
  const double V = T.vol[c];
  return alpha * (V / dti + 0.5 * sr) + (1.0 - alpha) * V / dte;
}
// The same diagonal from the time-step denominator sum = sum_f S_f (|u.n| + c),
// with dt_exp = cfl_exp V / sum and dt_imp = cfl_imp V / sum:
// D_i = sum (alpha cfl_exp + (1 - alpha) cfl_imp) / (cfl_imp cfl_exp) + alpha / 2 sum S r,
// one division where the form above takes four.
template <int DIM>
__device__ __forceinline__ double lusgs_diag_sum(const Topo& T, int c, const double* rface, double alpha, double sum,
                                                 double cfl_exp, double cfl_imp) {
  double sr = 0.0;
  for (int e = T.off[c]; e < T.off[c + 1]; ++e) sr += T.S[e] * rface[T.face[e]];
  return sum * (alpha * cfl_exp + (1.0 - alpha) * cfl_imp) / (cfl_imp * cfl_exp) + 0.5 * alpha * sr;
}

// The forward LU-SGS step of the first colour, fused into the kernel that
// forms R~ and D: colour 0 has no lower-coloured neighbours, so its step is
// dW* = -R~ / D, written exactly as k_sweep<MODE 0> would (and to dW as well
// when colour 0 is the only colour, as k_sweep<MODE 2> would).
template <int NV, typename T>
__device__ __forceinline__ void colour0_forward(int c, const double* __restrict__ R, double alpha, double D,
                                                T* __restrict__ dWs, T* __restrict__ dW) {
  const T ha = (T)(0.5 * alpha);
  const T iD = T(1) / (T)D;  // in the sweep precision: an FP32 reciprocal in the mixed mode
  double rc[NV];
  T x[NV];
  ld_row<NV>(R, c, rc);
#pragma unroll
  for (int v = 0; v < NV; ++v) {
    const double rhs = -(rc[v] + 0.0);
    x[v] = ((T)rhs - ha * (T)0) * iD;
  }
  st_row<NV>(dWs, c, x);
  if (dW) st_row<NV>(dW, c, x);
}

// ---------------------------------------------------------------------------
// K3: per-cell gather of residual, new slopes (Sec 2.4) and DF (Sec 3.3)
// ---------------------------------------------------------------------------
template <int DIM, typename TS = double, int VAR = 0>
__global__ void __launch_bounds__(kBlock) k_gather(DevFine M, Topo T, const double* __restrict__ Fface,
                                                   const double* __restrict__ Wface, const double* __restrict__ aface,
                                                   const double* __restrict__ W, const double* __restrict__ winf,
                                                   double gamma, const double* __restrict__ dte,
                                                   const double* __restrict__ dti, double* __restrict__ R,
                                                   double* __restrict__ Gout, double* __restrict__ alpha,
                                                   double* __restrict__ Dg, double* __restrict__ gradnew_out,
                                                   double* __restrict__ norm_part, double relax_fixed,
                                                   double om_alpha, double om_slope,
                                                   const double* __restrict__ rface, double* __restrict__ qcell,
                                                   const int* __restrict__ active, TS* __restrict__ dWs0 = nullptr,
                                                   TS* __restrict__ dW0 = nullptr, int c0_end = 0) {
  using Dm = Dims<DIM, VAR>;
  constexpr int NV = Dm::NV, NFC = Dm::NFC;
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  double rl2[NV], rmax[NV];
#pragma unroll
  for (int v = 0; v < NV; ++v) { rl2[v] = 0.0; rmax[v] = 0.0; }
  if (c < M.n) {
    double r[NV], gn[NV][DIM], a = 1.0;
#pragma unroll
    for (int v = 0; v < NV; ++v) {
      r[v] = 0.0;
#pragma unroll
      for (int d = 0; d < DIM; ++d) gn[v][d] = 0.0;
    }
    const int nf = VAR ? (int)M.cnf[c] : NFC;
#pragma unroll
    for (int m = 0; m < NFC; ++m) {
      if (VAR && m >= nf) break;
      const int f = M.cface[(size_t)c * NFC + m];
      const double s = M.cside[(size_t)c * NFC + m];
      double nn[DIM], ff[NV], wf[NV];
#pragma unroll
      for (int d = 0; d < DIM; ++d) nn[d] = s * M.fn[(size_t)f * DIM + d];
      ld_row<NV>(Fface, f, ff);
      ld_row<NV>(Wface, f, wf);
#pragma unroll
      for (int v = 0; v < NV; ++v) {
        r[v] += s * ff[v];
#pragma unroll
        for (int d = 0; d < DIM; ++d) gn[v][d] += wf[v] * nn[d];
      }
      a *= aface[f];
    }
    const double iV = 1.0 / M.vol[c];
    const bool live = !active || active[M.grp[c]];  // frozen (converged) batch members keep their state
    // stored DF: the product itself, or, where it rises, under-relaxed towards
    // it (a fall takes effect at once; same fixed points)
    const double as = (om_alpha < 1.0 && a > alpha[c]) ? alpha[c] + om_alpha * (a - alpha[c]) : a;
    st_row<NV>(R, c, r);
    double qc[2 * NV], gv[NV * DIM], go[NV * DIM];
    if (Gout && live && om_slope < 1.0) ld_row<NV * DIM>(Gout, c, go);
#pragma unroll
    for (int v = 0; v < NV; ++v) {
      const double q = r[v] * iV;
      rl2[v] = q * q;
      rmax[v] = fabs(q);
      qc[2 * v] = q * q;
      qc[2 * v + 1] = fabs(q);
#pragma unroll
      for (int d = 0; d < DIM; ++d) {
        const double g = gn[v][d] * iV;
        gv[v * DIM + d] = g;
        // slope update with DF, replaced or under-relaxed
        go[v * DIM + d] = om_slope < 1.0 ? go[v * DIM + d] + om_slope * (as * g - go[v * DIM + d]) : as * g;
      }
    }
    if (qcell) st_row<2 * NV>(qcell, c, qc);
    if (gradnew_out) st_row<NV * DIM>(gradnew_out, c, gv);
    if (Gout && live) st_row<NV * DIM>(Gout, c, go);
    if (live) alpha[c] = as;
    // LU-SGS diagonal with DF, or with the constant of the fixed-factor schemes (relax_fixed >= 0)
    if (Dg) {
      const double rel = relax_fixed < 0.0 ? as : relax_fixed;
      const double D = lusgs_diag<DIM>(T, c, rface, rel, dte[c], dti[c]);
      Dg[c] = D;
      if (dWs0 && c < c0_end) colour0_forward<NV, TS>(c, R, rel, D, dWs0, dW0);
    }
  }
  if (norm_part) {
    // block reduction in a fixed order: warp shuffles then warp 0
    __shared__ double sh[2 * NV][kBlock / 32];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
    for (int v = 0; v < NV; ++v) {
      double s = rl2[v], mx = rmax[v];
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        s += __shfl_down_sync(0xffffffffu, s, o);
        mx = fmax(mx, __shfl_down_sync(0xffffffffu, mx, o));
      }
      if (lane == 0) { sh[2 * v][wid] = s; sh[2 * v + 1][wid] = mx; }
    }
    __syncthreads();
    if (threadIdx.x == 0) {
#pragma unroll
      for (int v = 0; v < NV; ++v) {
        double s = 0.0, mx = 0.0;
        for (int w = 0; w < kBlock / 32; ++w) { s += sh[2 * v][w]; mx = fmax(mx, sh[2 * v + 1][w]); }
        norm_part[(size_t)blockIdx.x * 2 * NV + 2 * v] = s;
        norm_part[(size_t)blockIdx.x * 2 * NV + 2 * v + 1] = mx;
      }
    }
  }
}

// final norm reduction (one block, fixed order) -> out[nv][2] = RMS, max
template <int NV>
__global__ void k_norm_final(const double* __restrict__ part, int nblocks, int ncells, double* __restrict__ hist,
                             int* __restrict__ cycle, int max_hist, double* __restrict__ last) {
  __shared__ double s[2 * NV][kBlock];
  for (int i = 0; i < 2 * NV; ++i) {
    double acc = (i & 1) ? 0.0 : 0.0;
    for (int b = threadIdx.x; b < nblocks; b += blockDim.x) {
      const double x = part[(size_t)b * 2 * NV + i];
      acc = (i & 1) ? fmax(acc, x) : acc + x;
    }
    s[i][threadIdx.x] = acc;
  }
  __syncthreads();
  for (int st = blockDim.x / 2; st > 0; st >>= 1) {
    if (threadIdx.x < st)
      for (int i = 0; i < 2 * NV; ++i)
        s[i][threadIdx.x] = (i & 1) ? fmax(s[i][threadIdx.x], s[i][threadIdx.x + st])
                                    : s[i][threadIdx.x] + s[i][threadIdx.x + st];
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    double out[2 * NV];
    for (int v = 0; v < NV; ++v) {
      out[2 * v] = sqrt(s[2 * v][0] / ncells);
      out[2 * v + 1] = s[2 * v + 1][0];
    }
    if (last)
      for (int i = 0; i < 2 * NV; ++i) last[i] = out[i];
    if (hist && cycle) {
      const int k = *cycle;
      if (k < max_hist)
        for (int i = 0; i < 2 * NV; ++i) hist[(size_t)k * 2 * NV + i] = out[i];
      *cycle = k + 1;
    }
  }
}

// per-group norms (batched meshes): one block per group, fixed order
template <int NV>
__global__ void k_group_norm(const double* __restrict__ qcell, const int* __restrict__ goff,
                             const int* __restrict__ gidx, double* __restrict__ hist, const int* __restrict__ cycle,
                             int max_hist, int n_groups, double* __restrict__ last) {
  __shared__ double s[2 * NV][kBlock];
  const int g = blockIdx.x;
  const int lo = goff[g], hi = goff[g + 1];
  for (int i = 0; i < 2 * NV; ++i) {
    double acc = 0.0;
    for (int k = lo + threadIdx.x; k < hi; k += blockDim.x) {
      const double x = qcell[(size_t)gidx[k] * 2 * NV + i];
      acc = (i & 1) ? fmax(acc, x) : acc + x;
    }
    s[i][threadIdx.x] = acc;
  }
  __syncthreads();
  for (int st = blockDim.x / 2; st > 0; st >>= 1) {
    if (threadIdx.x < st)
      for (int i = 0; i < 2 * NV; ++i)
        s[i][threadIdx.x] = (i & 1) ? fmax(s[i][threadIdx.x], s[i][threadIdx.x + st])
                                    : s[i][threadIdx.x] + s[i][threadIdx.x + st];
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    const int k = *cycle;
    for (int v = 0; v < NV; ++v) {
      const double rms = sqrt(s[2 * v][0] / (double)(hi - lo)), mx = s[2 * v + 1][0];
      if (hist && k < max_hist) {
        hist[((size_t)k * n_groups + g) * 2 * NV + 2 * v] = rms;
        hist[((size_t)k * n_groups + g) * 2 * NV + 2 * v + 1] = mx;
      }
      last[(size_t)g * 2 * NV + 2 * v] = rms;
      last[(size_t)g * 2 * NV + 2 * v + 1] = mx;
    }
  }
}
__global__ void k_bump(int* __restrict__ cycle) { *cycle += 1; }

// Packs what the host needs after a chunk of recorded V-cycles, so that one
// small device-to-host copy serves the convergence test and the norms:
// out[0] = cycles recorded so far, out[1] / out[2] = density RMS of the first
// and of the latest recorded cycle, then the rows of the last `chunk` cycles
// (nv2 values each; -1 where a row lies outside the history).
__global__ void k_pack_hist(const double* __restrict__ hist, const int* __restrict__ cycle, int max_hist, int nv2,
                            int chunk, double* __restrict__ out) {
  const int k = *cycle;
  const int upto = min(k, max_hist);
  if (threadIdx.x == 0) {
    out[0] = k;
    out[1] = upto > 0 ? hist[0] : 0.0;
    out[2] = upto > 0 ? hist[(size_t)(upto - 1) * nv2] : 0.0;
  }
  for (int t = threadIdx.x; t < chunk * nv2; t += blockDim.x) {
    const int idx = k - chunk + t / nv2;
    out[3 + t] = (idx >= 0 && idx < max_hist) ? hist[(size_t)idx * nv2 + t % nv2] : -1.0;
  }
}

// ---------------------------------------------------------------------------
// K4 / K5: multi-colour LU-SGS sweeps (Eqs. gpu-forward-relaxation and
// gpu-backward-relaxation), one launch per colour over cells [lo, hi).
// T is the sweep precision (double, or float in the mixed mode).
// rhs = -(R + P) with P the coarse forcing (nullptr on the fine level).
// ---------------------------------------------------------------------------
template <int DIM, typename T>
__device__ __forceinline__ void offdiag_term(const Topo& Tp, int e, const double* W, const T* dWsrc,
                                             const double* rface, double gamma, T* acc) {
  constexpr int NV = DIM + 2;
  const int j = Tp.nbr[e];
  T nn[DIM], Wj[NV], dj[NV], dF[NV];
#pragma unroll
  for (int d = 0; d < DIM; ++d) nn[d] = (T)Tp.nrm[(size_t)e * DIM + d];
  double wj[NV];
  ld_row<NV>(W, j, wj);
  ld_row<NV>(dWsrc, j, dj);
#pragma unroll
  for (int v = 0; v < NV; ++v) Wj[v] = (T)wj[v];
  const T r = (T)rface[Tp.face[e]];
  if constexpr (sizeof(T) == 8) {
    // plain difference of Euler fluxes in FP64
    T F1[NV], F0[NV], Wp[NV];
#pragma unroll
    for (int v = 0; v < NV; ++v) Wp[v] = Wj[v] + dj[v];
    euler_flux<DIM, T>((T)gamma, Wp, nn, F1);
    euler_flux<DIM, T>((T)gamma, Wj, nn, F0);
#pragma unroll
    for (int v = 0; v < NV; ++v) dF[v] = F1[v] - F0[v];
  } else {
    euler_flux_increment<DIM, T>((T)gamma, Wj, dj, nn, dF);
  }
  const T S = (T)Tp.S[e];
#pragma unroll
  for (int v = 0; v < NV; ++v) acc[v] += S * (dF[v] - r * dj[v]);
}

// mode 0: forward (neighbours j < lo); mode 1: backward (j >= hi);
// mode 2: the top colour, forward then dW = dW*.
// state update with the positivity guard (reading): halve up to 10 times, else drop
template <int DIM>
__device__ __forceinline__ int guarded_add(double gamma, double* W, const double* dW) {
  constexpr int NV = DIM + 2;
  double s = 1.0;
  for (int it = 0; it <= 10; ++it) {
    double Wn[NV], ke = 0.0;
#pragma unroll
    for (int v = 0; v < NV; ++v) Wn[v] = W[v] + s * dW[v];
#pragma unroll
    for (int d = 0; d < DIM; ++d) ke += Wn[1 + d] * Wn[1 + d];
    if (Wn[0] > 0.0 && (Wn[NV - 1] - 0.5 * ke / Wn[0]) > 0.0) {
#pragma unroll
      for (int v = 0; v < NV; ++v) W[v] = Wn[v];
      return it;
    }
    s *= 0.5;
  }
  return -1;
}

// the guarded update of cell c into Wout (the state's other buffer), as k_update
template <int DIM, typename T>
__device__ __forceinline__ void update_into(int c, double gamma, const double* __restrict__ W, const T* d_c,
                                            double* __restrict__ Wout, Counters* __restrict__ cnt) {
  constexpr int NV = DIM + 2;
  double w[NV], d[NV];
  bool finite = true;
  ld_row<NV>(W, c, w);
#pragma unroll
  for (int v = 0; v < NV; ++v) {
    d[v] = (double)d_c[v];
    finite = finite && isfinite(d[v]);
  }
  if (!finite) {
    atomicAdd(&cnt->nonfinite, 1ull);
  } else {
    const int r = guarded_add<DIM>(gamma, w, d);
    if (r > 0) atomicAdd(&cnt->update_halved, 1ull);
    if (r < 0) atomicAdd(&cnt->update_zeroed, 1ull);
  }
  st_row<NV>(Wout, c, w);
}

// Wout (nullable): the state's other buffer.  Where this launch finalises the
// increments of its colour (MODE 2: the last colour; MODE 1: backward), it
// also writes the guarded update W + dW there, so that no separate update
// launch is needed (the sweeps keep reading W).
// the LU-SGS step of cell c of the colour [lo, hi) (k_sweep's per-cell work)
template <int DIM, typename T, int MODE>
__device__ __forceinline__ void sweep_cell(const Topo& Tp, int c, int lo, int hi, const double* __restrict__ W,
                                           const double* __restrict__ R, const double* __restrict__ Pf,
                                           const double* __restrict__ alpha, const double* __restrict__ Dg,
                                           const double* __restrict__ rface, double gamma, T* __restrict__ dWs,
                                           T* __restrict__ dW, double* __restrict__ Wout,
                                           Counters* __restrict__ cnt) {
  constexpr int NV = DIM + 2;
  T acc[NV];
#pragma unroll
  for (int v = 0; v < NV; ++v) acc[v] = 0;
  const T* src = MODE == 1 ? dW : dWs;
  for (int e = Tp.off[c]; e < Tp.off[c + 1]; ++e) {
    const int j = Tp.nbr[e];
    if (j < 0) continue;  // ghost increments are zero
    if (MODE == 1 ? (j < hi) : (j >= lo)) continue;
    offdiag_term<DIM, T>(Tp, e, W, src, rface, gamma, acc);
  }
  const T ha = (T)(0.5 * alpha[c]);
  const T iD = T(1) / (T)Dg[c];  // as in colour0_forward
  T fin[NV];  // the final increment (MODE 1, 2)
  if (MODE == 1) {
    T ds[NV];
    ld_row<NV>(dWs, c, ds);
#pragma unroll
    for (int v = 0; v < NV; ++v) fin[v] = ds[v] - ha * acc[v] * iD;
    st_row<NV>(dW, c, fin);
  } else {
    double rc[NV], pc[NV];
    ld_row<NV>(R, c, rc);
    if (Pf) ld_row<NV>(Pf, c, pc);
#pragma unroll
    for (int v = 0; v < NV; ++v) {
      const double rhs = -(rc[v] + (Pf ? pc[v] : 0.0));
      fin[v] = ((T)rhs - ha * acc[v]) * iD;
    }
    st_row<NV>(dWs, c, fin);
    if (MODE == 2) st_row<NV>(dW, c, fin);
  }
  if (MODE != 0 && Wout) update_into<DIM, T>(c, gamma, W, fin, Wout, cnt);
}

template <int DIM, typename T, int MODE>
__global__ void __launch_bounds__(kBlock) k_sweep(Topo Tp, int lo, int hi, const double* __restrict__ W,
                                                  const double* __restrict__ R, const double* __restrict__ Pf,
                                                  const double* __restrict__ alpha, const double* __restrict__ Dg,
                                                  const double* __restrict__ rface, double gamma,
                                                  T* __restrict__ dWs, T* __restrict__ dW,
                                                  double* __restrict__ Wout = nullptr,
                                                  Counters* __restrict__ cnt = nullptr) {
  const int c = lo + blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= hi) return;
  sweep_cell<DIM, T, MODE>(Tp, c, lo, hi, W, R, Pf, alpha, Dg, rface, gamma, dWs, dW, Wout, cnt);
}

template <int DIM, typename T>
__global__ void __launch_bounds__(kBlock) k_update(int n, double gamma, double* __restrict__ W,
                                                   const T* __restrict__ dW, Counters* __restrict__ cnt,
                                                   const int* __restrict__ grp, const int* __restrict__ active) {
  constexpr int NV = DIM + 2;
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= n) return;
  if (active && !active[grp[c]]) return;
  double w[NV], d[NV];
  T dc[NV];
  bool finite = true;
  ld_row<NV>(W, c, w);
  ld_row<NV>(dW, c, dc);
#pragma unroll
  for (int v = 0; v < NV; ++v) {
    d[v] = (double)dc[v];
    finite = finite && isfinite(d[v]);
  }
  if (!finite) {
    atomicAdd(&cnt->nonfinite, 1ull);
    return;
  }
  const int r = guarded_add<DIM>(gamma, w, d);
  if (r > 0) atomicAdd(&cnt->update_halved, 1ull);
  if (r < 0) atomicAdd(&cnt->update_zeroed, 1ull);
  st_row<NV>(W, c, w);
}

// explicit local-time-step update W -= dt_exp R / V (Eq. smo, fine smoother option)
template <int DIM>
__global__ void __launch_bounds__(kBlock) k_explicit(int n, double gamma, const double* __restrict__ R,
                                                     const double* __restrict__ dte, const double* __restrict__ vol,
                                                     double* __restrict__ W, Counters* __restrict__ cnt,
                                                     const int* __restrict__ grp, const int* __restrict__ active) {
  constexpr int NV = DIM + 2;
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= n) return;
  if (active && !active[grp[c]]) return;
  const double s = -dte[c] / vol[c];
  double w[NV], d[NV];
#pragma unroll
  for (int v = 0; v < NV; ++v) {
    w[v] = W[(size_t)c * NV + v];
    d[v] = s * R[(size_t)c * NV + v];
  }
  const int r = guarded_add<DIM>(gamma, w, d);
  if (r > 0) atomicAdd(&cnt->update_halved, 1ull);
  if (r < 0) atomicAdd(&cnt->update_zeroed, 1ull);
#pragma unroll
  for (int v = 0; v < NV; ++v) W[(size_t)c * NV + v] = w[v];
}

// ---------------------------------------------------------------------------
// K6: coarse levels: first-order KFVS face flux (S-weighted, global frame) and
// the spectral radius of the LU-SGS splitting, once per face ...
// ---------------------------------------------------------------------------
template <int DIM>
__global__ void __launch_bounds__(kBlock) k_face_kfvs(FaceSet Fs, const double* __restrict__ W,
                                                      const double* __restrict__ winf, PhysParams P,
                                                      double* __restrict__ Fout, double* __restrict__ rout) {
  constexpr int NV = DIM + 2;
  const int f = blockIdx.x * blockDim.x + threadIdx.x;
  if (f >= Fs.nf) return;
  const int L = Fs.fL[f], R = Fs.fR[f];
  double n[DIM], WL[NV], WR[NV];
#pragma unroll
  for (int d = 0; d < DIM; ++d) n[d] = Fs.fn[(size_t)f * DIM + d];
  ld_row<NV>(W, L, WL);
  if (R >= 0) {
    ld_row<NV>(W, R, WR);
  } else {
    ghost_state<DIM>(Fs.ftag[f], winf + NV * (Fs.grp ? Fs.grp[L] : 0), n, WL, WR, P.gamma);
  }
  if (Fout) {
    const Frame<DIM> fr = make_frame<DIM>(n);
    double wl[NV], wr[NV], Fl[NV], Fg[NV];
    to_local<DIM>(fr, WL, wl);
    to_local<DIM>(fr, WR, wr);
    kfvs_flux<DIM>(P, wl, wr, Fl);
    to_global<DIM>(fr, Fl, Fg);
    const double S = Fs.fS[f];
#pragma unroll
    for (int v = 0; v < NV; ++v) Fg[v] *= S;
    st_row<NV>(Fout, f, Fg);
  }
  if (rout) rout[f] = spectral_radius<DIM, double>(P.gamma, WL, WR, n);
}

// ... then per cell: R~ = sum_f +-S F + P (or, with Rstar, the forcing
// P = R* - R), local time steps and the DF-relaxed LU-SGS diagonal.
template <int DIM, typename T>
__device__ __forceinline__ void coarse_cell(const Topo& Tp, int c, const double* __restrict__ W,
                                            const double* __restrict__ Fface, const double* __restrict__ rface,
                                            const double* __restrict__ Pf, const double* __restrict__ Rstar,
                                            const double* __restrict__ alpha, double gamma, double cfl_exp,
                                            double cfl_imp, double* __restrict__ out, double* __restrict__ Dg,
                                            T* __restrict__ dWs0, T* __restrict__ dW0, int c0_end) {
  constexpr int NV = DIM + 2;
  double r[NV];
#pragma unroll
  for (int v = 0; v < NV; ++v) r[v] = 0.0;
  for (int e = Tp.off[c]; e < Tp.off[c + 1]; ++e) {
    const int f = Tp.face[e];
    const double sd = Tp.side[e];
    double ff[NV];
    ld_row<NV>(Fface, f, ff);
#pragma unroll
    for (int v = 0; v < NV; ++v) r[v] += sd * ff[v];
  }
  {
    double o[NV], q[NV];
    if (Rstar) ld_row<NV>(Rstar, c, q);
    else if (Pf) ld_row<NV>(Pf, c, q);
#pragma unroll
    for (int v = 0; v < NV; ++v) o[v] = Rstar ? q[v] - r[v] : r[v] + (Pf ? q[v] : 0.0);
    st_row<NV>(out, c, o);
  }
  if (Dg) {
    double Wi[NV], ke = 0.0;
    ld_row<NV>(W, c, Wi);
#pragma unroll
    for (int d = 0; d < DIM; ++d) ke += Wi[1 + d] * Wi[1 + d];
    const double ir = 1.0 / Wi[0];
    const double cs = sqrt(gamma * (gamma - 1.0) * (Wi[NV - 1] - 0.5 * ke * ir) * ir);
    double sum = 0.0;
    for (int e = Tp.off[c]; e < Tp.off[c + 1]; ++e) {
      double un = 0.0;
#pragma unroll
      for (int d = 0; d < DIM; ++d) un += Wi[1 + d] * Tp.nrm[(size_t)e * DIM + d];
      sum += Tp.S[e] * (fabs(un * ir) + cs);
    }
    const double D = lusgs_diag_sum<DIM>(Tp, c, rface, alpha[c], sum, cfl_exp, cfl_imp);
    Dg[c] = D;
    if (dWs0 && c < c0_end) colour0_forward<NV, T>(c, out, alpha[c], D, dWs0, dW0);
  }
}

template <int DIM, typename T = double>
__global__ void __launch_bounds__(kBlock) k_coarse_cell(Topo Tp, const double* __restrict__ W,
                                                        const double* __restrict__ Fface,
                                                        const double* __restrict__ rface,
                                                        const double* __restrict__ Pf,
                                                        const double* __restrict__ Rstar,
                                                        const double* __restrict__ alpha, double gamma,
                                                        double cfl_exp, double cfl_imp, double* __restrict__ out,
                                                        double* __restrict__ Dg, T* __restrict__ dWs0,
                                                        T* __restrict__ dW0, int c0_end) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= Tp.n) return;
  coarse_cell<DIM, T>(Tp, c, W, Fface, rface, Pf, Rstar, alpha, gamma, cfl_exp, cfl_imp, out, Dg, dWs0, dW0, c0_end);
}

// One smoothing step of a small two-colour coarse level after its face fluxes
// (k_face_kfvs): R~ and D of every cell with the forward step of colour 0
// (k_coarse_cell), then colour 1 forward and backward with its guarded update
// (k_sweep mode 2), then colour 0 backward with its update (k_sweep mode 1).
// One thread-block cluster runs the three phases, separated by cluster
// barriers (release / acquire at cluster scope) instead of kernel boundaries;
// every cell does exactly the work, in the same order, of the three kernels.
template <int DIM, typename T>
__global__ void __launch_bounds__(kClusterBlock) k_coarse_step_cluster(
    Topo Tp, const double* __restrict__ W, const double* __restrict__ Fface, const double* __restrict__ rface,
    const double* __restrict__ Pf, const double* __restrict__ alpha, double gamma, double cfl_exp, double cfl_imp,
    double* __restrict__ R, double* __restrict__ Dg, T* __restrict__ dWs, T* __restrict__ dW, int c1,
    double* __restrict__ Wout, Counters* __restrict__ cnt) {
  const int n = Tp.n;
  const int stride = gridDim.x * blockDim.x;
  const int t0 = blockIdx.x * blockDim.x + threadIdx.x;
  for (int c = t0; c < n; c += stride)
    coarse_cell<DIM, T>(Tp, c, W, Fface, rface, Pf, nullptr, alpha, gamma, cfl_exp, cfl_imp, R, Dg, dWs, nullptr, c1);
  cluster_barrier();
  for (int c = c1 + t0; c < n; c += stride)
    sweep_cell<DIM, T, 2>(Tp, c, c1, n, W, R, nullptr, alpha, Dg, rface, gamma, dWs, dW, Wout, cnt);
  cluster_barrier();
  for (int c = t0; c < c1; c += stride)
    sweep_cell<DIM, T, 1>(Tp, c, 0, c1, W, R, nullptr, alpha, Dg, rface, gamma, dWs, dW, Wout, cnt);
}

// ---------------------------------------------------------------------------
// K7: restriction (Sec 5.2): volume-weighted state, summed residual, min DF
// ---------------------------------------------------------------------------
template <int DIM>
__global__ void __launch_bounds__(kBlock) k_restrict(int nc, const int* __restrict__ ch_off,
                                                     const int* __restrict__ ch_idx, const double* __restrict__ vol_f,
                                                     const double* __restrict__ vol_c, const double* __restrict__ Wf,
                                                     const double* __restrict__ af, const double* __restrict__ Rf,
                                                     double* __restrict__ W0, double* __restrict__ Wc,
                                                     double* __restrict__ ac, double* __restrict__ Rstar) {
  constexpr int NV = DIM + 2;
  const int I = blockIdx.x * blockDim.x + threadIdx.x;
  if (I >= nc) return;
  double w[NV], r[NV], a = 1.0;
#pragma unroll
  for (int v = 0; v < NV; ++v) { w[v] = 0.0; r[v] = 0.0; }
  for (int k = ch_off[I]; k < ch_off[I + 1]; ++k) {
    const int i = ch_idx[k];
    const double V = vol_f[i];
    double wi[NV], ri[NV];
    ld_row<NV>(Wf, i, wi);
    ld_row<NV>(Rf, i, ri);
#pragma unroll
    for (int v = 0; v < NV; ++v) {
      w[v] += V * wi[v];
      r[v] += ri[v];
    }
    a = fmin(a, af[i]);
  }
  const double iV = 1.0 / vol_c[I];
#pragma unroll
  for (int v = 0; v < NV; ++v) w[v] *= iV;
  st_row<NV>(W0, I, w);
  st_row<NV>(Wc, I, w);
  st_row<NV>(Rstar, I, r);
  ac[I] = a;
}

// ---------------------------------------------------------------------------
// K8: DF-limited injection prolongation (Eq. prolongation)
// ---------------------------------------------------------------------------
template <int DIM>
__global__ void __launch_bounds__(kBlock) k_prolong(int nf, const int* __restrict__ parent,
                                                    const double* __restrict__ af, const double* __restrict__ Wc,
                                                    const double* __restrict__ Wc0, double gamma, double* __restrict__ Wf,
                                                    Counters* __restrict__ cnt, const int* __restrict__ grp,
                                                    const int* __restrict__ active) {
  constexpr int NV = DIM + 2;
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= nf) return;
  if (active && !active[grp[i]]) return;
  const int I = parent[i];
  double w[NV], d[NV], wc[NV], wc0[NV];
  const double a = af[i];
  ld_row<NV>(Wf, i, w);
  ld_row<NV>(Wc, I, wc);
  ld_row<NV>(Wc0, I, wc0);
#pragma unroll
  for (int v = 0; v < NV; ++v) d[v] = a * (wc[v] - wc0[v]);
  const int r = guarded_add<DIM>(gamma, w, d);
  if (r > 0) atomicAdd(&cnt->update_halved, 1ull);
  if (r < 0) atomicAdd(&cnt->update_zeroed, 1ull);
  st_row<NV>(Wf, i, w);
}

// ---------------------------------------------------------------------------
// helpers: permutation scatter / gather of per-cell rows
// ---------------------------------------------------------------------------
// out[orig[c]] = in[c] (rows of width w): device colour order -> original order
__global__ void k_scatter_rows(int n, int w, const int* __restrict__ iperm, const double* __restrict__ in,
                               double* __restrict__ out) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (int64_t)n * w) return;
  const int c = (int)(t / w), k = (int)(t % w);
  out[(size_t)iperm[c] * w + k] = in[t];
}
// out[c] = in[orig[c]]: original order -> device colour order
__global__ void k_gather_rows(int n, int w, const int* __restrict__ iperm, const double* __restrict__ in,
                              double* __restrict__ out) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (int64_t)n * w) return;
  const int c = (int)(t / w), k = (int)(t % w);
  out[t] = in[(size_t)iperm[c] * w + k];
}
__global__ void k_fill(int64_t n, double v, double* __restrict__ x) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t < n) x[t] = v;
}


__global__ void k_scale(int64_t n, double a, double* __restrict__ x) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t < n) x[t] *= a;
}
__global__ void k_f2d(int64_t n, const float* __restrict__ x, double* __restrict__ y) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t < n) y[t] = (double)x[t];
}
// LU-SGS diagonal from given time steps and DF factors
template <int DIM>
__global__ void __launch_bounds__(kBlock) k_diag(Topo Tp, const double* __restrict__ rface,
                                                 const double* __restrict__ alpha, const double* __restrict__ dte,
                                                 const double* __restrict__ dti, double* __restrict__ Dg) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= Tp.n) return;
  Dg[c] = lusgs_diag<DIM>(Tp, c, rface, alpha[c], dte[c], dti[c]);
}

// ---------------------------------------------------------------------------
// Learned coarse-grid correction (2-D): per-cell features, training targets,
// gated application and the judge error.
// Features of a cell (17, scaled by the free stream's rho, rho c, rho c^2):
// W, slopes times h = |Omega|^(1/2), R dt_imp / |Omega|, DF; the network input
// is the cell's 17 followed by its three face neighbours' (ghosts across
// boundary faces: mirrored / free-stream state, zero residual, own DF and h).
// ---------------------------------------------------------------------------
__device__ __forceinline__ void fs_scales(const double* w, double gamma, double* sc) {
  const double rho = w[0];
  const double ke = 0.5 * (w[1] * w[1] + w[2] * w[2]) / rho;
  const double p = (gamma - 1.0) * (w[3] - ke);
  const double c = sqrt(gamma * p / rho);
  sc[0] = rho;
  sc[1] = rho * c;
  sc[2] = rho * c;
  sc[3] = rho * c * c;
}

__device__ __forceinline__ void cell_features(const double* W, const double (*g)[2], double rterm_scale,
                                              const double* R, double a, double h, const double* sc,
                                              __nv_bfloat16* out) {
#pragma unroll
  for (int v = 0; v < 4; ++v) out[v] = __float2bfloat16((float)(W[v] / sc[v]));
#pragma unroll
  for (int v = 0; v < 4; ++v)
#pragma unroll
    for (int d = 0; d < 2; ++d) out[4 + 2 * v + d] = __float2bfloat16((float)(g[v][d] * h / sc[v]));
#pragma unroll
  for (int v = 0; v < 4; ++v) out[12 + v] = __float2bfloat16((float)(R ? R[v] * rterm_scale / sc[v] : 0.0));
  out[16] = __float2bfloat16((float)a);
}

// Inputs per cell: 17 for the cell and each of its 3 face neighbours (68),
// then the restricted residuals of its level-1 parent and level-2 grandparent
// (8): the coarse-grid defects that drive the correction the network predicts.
constexpr int kFeat = 76;

// Rc[I] = sum of Rf over the children of coarse cell I (4 variables, in the
// children's stored order)
__global__ void k_sum_children(int nc, const int* __restrict__ ch_off, const int* __restrict__ ch_idx,
                               const double* __restrict__ Rf, double* __restrict__ Rc) {
  const int I = blockIdx.x * blockDim.x + threadIdx.x;
  if (I >= nc) return;
  double s[4] = {0.0, 0.0, 0.0, 0.0};
  for (int e = ch_off[I]; e < ch_off[I + 1]; ++e) {
    const int i = ch_idx[e];
#pragma unroll
    for (int v = 0; v < 4; ++v) s[v] += Rf[(size_t)i * 4 + v];
  }
#pragma unroll
  for (int v = 0; v < 4; ++v) Rc[(size_t)I * 4 + v] = s[v];
}

// parent1/parent2: level-1 parent of each fine cell and level-2 parent of each
// level-1 cell (stored order); R1, R2 the restricted residuals and vol1, vol2
// the volumes of those levels (all null on a mesh of fewer than 3 levels: the
// 8 inputs are then zero).  Each coarse residual enters as an increment: times
// the cell's implicit time step scaled by the length ratio to the coarse
// cell, sqrt(V_I / V_c), over V_I.  With S non-null the 24 residual-type
// inputs are further divided by the cell's defect scale s (its implicit time
// step times the size of the residual over the whole mesh, from the norms
// gnorm [groups][4][rms, max]), stored in S: the network then sees the
// defect relative to the current stage of the solve, and its output is
// multiplied by s (a correction proportional to the size of the defect).
__global__ void __launch_bounds__(kBlock) k_features2(DevFine M, const double* __restrict__ W,
                                                      const double* __restrict__ G, const double* __restrict__ R,
                                                      const double* __restrict__ dti, const double* __restrict__ alpha,
                                                      const double* __restrict__ winf, double gamma,
                                                      const int* __restrict__ parent1, const int* __restrict__ parent2,
                                                      const double* __restrict__ R1, const double* __restrict__ R2,
                                                      const double* __restrict__ vol1, const double* __restrict__ vol2,
                                                      const double* __restrict__ gnorm, __nv_bfloat16* __restrict__ X,
                                                      float* __restrict__ S) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= M.n) return;
  const double* wi = winf + 4 * (M.grp ? M.grp[c] : 0);
  double sc[4];
  fs_scales(wi, gamma, sc);
  __nv_bfloat16* out = X + (size_t)c * kFeat;
  double inv_s = 1.0;
  {
    double f1[4] = {0.0, 0.0, 0.0, 0.0}, f2[4] = {0.0, 0.0, 0.0, 0.0};
    if (parent1 && parent2) {
      const int I = parent1[c], J = parent2[I];
      const double k1 = dti[c] * sqrt(vol1[I] / M.vol[c]) / vol1[I];
      const double k2 = dti[c] * sqrt(vol2[J] / M.vol[c]) / vol2[J];
#pragma unroll
      for (int v = 0; v < 4; ++v) {
        f1[v] = R1[(size_t)I * 4 + v] * k1 / sc[v];
        f2[v] = R2[(size_t)J * 4 + v] * k2 / sc[v];
      }
    }
    if (S) {
      // defect scale of the cell: its implicit time step times the RMS over
      // the variables of the mesh's (group's) last residual norms, RMS of
      // R_v / |Omega| over the cells, in free-stream units
      const double* q = gnorm + 8 * (M.grp ? M.grp[c] : 0);
      double ss = 0.0;
#pragma unroll
      for (int v = 0; v < 4; ++v) {
        const double t = q[2 * v] / sc[v];
        ss += t * t;
      }
      double s = dti[c] * sqrt(0.25 * ss);
      if (!(s > 0.0)) s = 1.0;
      inv_s = 1.0 / s;
      S[c] = (float)s;
    }
#pragma unroll
    for (int v = 0; v < 4; ++v) {
      out[68 + v] = __float2bfloat16((float)(f1[v] * inv_s));
      out[72 + v] = __float2bfloat16((float)(f2[v] * inv_s));
    }
  }
  double Wc[4], gc[4][2];
#pragma unroll
  for (int v = 0; v < 4; ++v) {
    Wc[v] = W[(size_t)c * 4 + v];
#pragma unroll
    for (int d = 0; d < 2; ++d) gc[v][d] = G[((size_t)c * 4 + v) * 2 + d];
  }
  const double hc = sqrt(M.vol[c]);
  cell_features(Wc, gc, dti[c] / M.vol[c] * inv_s, R + (size_t)c * 4, alpha[c], hc, sc, out);
#pragma unroll
  for (int m = 0; m < 3; ++m) {
    const int j = M.cnbr[(size_t)c * 3 + m];
    __nv_bfloat16* o = out + 17 * (m + 1);
    if (j >= 0) {
      double Wj[4], gj[4][2];
#pragma unroll
      for (int v = 0; v < 4; ++v) {
        Wj[v] = W[(size_t)j * 4 + v];
#pragma unroll
        for (int d = 0; d < 2; ++d) gj[v][d] = G[((size_t)j * 4 + v) * 2 + d];
      }
      cell_features(Wj, gj, dti[j] / M.vol[j] * inv_s, R + (size_t)j * 4, alpha[j], sqrt(M.vol[j]), sc, o);
    } else {
      const int f = M.cface[(size_t)c * 3 + m];
      const double sd = M.cside[(size_t)c * 3 + m];
      double n[2] = {sd * M.fn[(size_t)f * 2], sd * M.fn[(size_t)f * 2 + 1]};
      double Wg[4], gg[4][2];
      ghost_state<2>(M.ftag[f], wi, n, Wc, Wg, gamma);
      ghost_grad<2>(M.ftag[f], wi, n, gc, gg);
      cell_features(Wg, gg, 0.0, nullptr, alpha[c], hc, sc, o);
    }
  }
}

// training target: the applied fine correction, scaled like W (and divided by
// the defect scale S where given)
__global__ void k_target2(int n, const double* __restrict__ W, const double* __restrict__ Wsave,
                          const int* __restrict__ grp, const double* __restrict__ winf, double gamma,
                          const float* __restrict__ S, float* __restrict__ Y) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= n) return;
  double sc[4];
  fs_scales(winf + 4 * (grp ? grp[c] : 0), gamma, sc);
  const double is = S ? 1.0 / (double)S[c] : 1.0;
#pragma unroll
  for (int v = 0; v < 4; ++v)
    Y[(size_t)c * 4 + v] = (float)((W[(size_t)c * 4 + v] - Wsave[(size_t)c * 4 + v]) / sc[v] * is);
}

// learned correction applied where the DF factor is at least the gate
__global__ void __launch_bounds__(kBlock) k_apply_learned2(int n, const float* __restrict__ P,
                                                           const double* __restrict__ alpha, double gate,
                                                           const int* __restrict__ grp, const double* __restrict__ winf,
                                                           const int* __restrict__ active, double gamma,
                                                           const float* __restrict__ S, double* __restrict__ W,
                                                           Counters* __restrict__ cnt) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= n) return;
  if (active && !active[grp[c]]) return;
  if (!(alpha[c] >= gate)) return;
  double sc[4], w[4], d[4];
  fs_scales(winf + 4 * (grp ? grp[c] : 0), gamma, sc);
  const double s = S ? (double)S[c] : 1.0;
#pragma unroll
  for (int v = 0; v < 4; ++v) {
    w[v] = W[(size_t)c * 4 + v];
    d[v] = (double)P[(size_t)c * 4 + v] * s * sc[v];
  }
  const int r = guarded_add<2>(gamma, w, d);
  if (r > 0) atomicAdd(&cnt->update_halved, 1ull);
  if (r < 0) atomicAdd(&cnt->update_zeroed, 1ull);
#pragma unroll
  for (int v = 0; v < 4; ++v) W[(size_t)c * 4 + v] = w[v];
}

// judge: per variable, the squared error of the prediction against the
// applied plain correction and the squared size of that correction, over gated
// cells (free-stream units; per-block partials, 8 per block)
__global__ void __launch_bounds__(kBlock) k_judge2(int n, const float* __restrict__ P, const double* __restrict__ W,
                                                   const double* __restrict__ Wsave, const double* __restrict__ alpha,
                                                   double gate, const int* __restrict__ grp,
                                                   const double* __restrict__ winf, double gamma,
                                                   const float* __restrict__ S, double* __restrict__ part) {
  __shared__ double sw[kBlock / 32][8];
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  double q[8] = {0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0};
  if (c < n && alpha[c] >= gate) {
    double sc[4];
    fs_scales(winf + 4 * (grp ? grp[c] : 0), gamma, sc);
    const double s = S ? (double)S[c] : 1.0;
#pragma unroll
    for (int v = 0; v < 4; ++v) {
      const double t = (W[(size_t)c * 4 + v] - Wsave[(size_t)c * 4 + v]) / sc[v];
      const double d = (double)P[(size_t)c * 4 + v] * s - t;
      q[v] = d * d;
      q[4 + v] = t * t;
    }
  }
#pragma unroll
  for (int k = 0; k < 8; ++k)
    for (int o = 16; o > 0; o >>= 1) q[k] += __shfl_down_sync(0xffffffffu, q[k], o);
  const int lane = threadIdx.x & 31, wp = threadIdx.x >> 5;
  if (lane == 0)
#pragma unroll
    for (int k = 0; k < 8; ++k) sw[wp][k] = q[k];
  __syncthreads();
  if (threadIdx.x < 8) {
    double a = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) a += sw[w][threadIdx.x];
    part[8 * (size_t)blockIdx.x + threadIdx.x] = a;
  }
}

// out[0..3] squared errors, out[4..7] squared corrections, per variable
// (blocks summed in order)
__global__ void k_judge_final(const double* __restrict__ part, int nb, double* __restrict__ out) {
  if (blockIdx.x != 0 || threadIdx.x >= 8) return;
  double a = 0.0;
  for (int b = 0; b < nb; ++b) a += part[8 * (size_t)b + threadIdx.x];
  out[threadIdx.x] = a;
}

// FMA-throughput probe: CH independent chains per thread
template <typename T, int CH>
__global__ void k_fma_probe(T* __restrict__ out, int iters, T a, T b) {
  T x[CH];
#pragma unroll
  for (int c = 0; c < CH; ++c) x[c] = (T)(threadIdx.x + c) * (T)1e-3;
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int c = 0; c < CH; ++c) x[c] = fma(x[c], a, b);
  }
  T s = 0;
#pragma unroll
  for (int c = 0; c < CH; ++c) s += x[c];
  out[(size_t)blockIdx.x * blockDim.x + threadIdx.x] = s;
}

// pointwise gas-kinetic flux for parity checks (local frame inputs)
template <int DIM>
__global__ void k_gks_points(int n, PhysParams P, const double* __restrict__ Wl, const double* __restrict__ Gl,
                             const double* __restrict__ Wr, const double* __restrict__ Gr,
                             const double* __restrict__ dt, double* __restrict__ F, double* __restrict__ Wt,
                             double* __restrict__ alpha) {
  constexpr int NV = DIM + 2;
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  double wl[NV], wr[NV], gl[DIM][NV], gr[DIM][NV], f[NV], w[NV];
#pragma unroll
  for (int v = 0; v < NV; ++v) { wl[v] = Wl[(size_t)i * NV + v]; wr[v] = Wr[(size_t)i * NV + v]; }
#pragma unroll
  for (int d = 0; d < DIM; ++d)
#pragma unroll
    for (int v = 0; v < NV; ++v) {
      gl[d][v] = Gl[((size_t)i * DIM + d) * NV + v];
      gr[d][v] = Gr[((size_t)i * DIM + d) * NV + v];
    }
  const double a = gks_flux<DIM>(P, wl, gl, wr, gr, dt[i], f, w);
#pragma unroll
  for (int v = 0; v < NV; ++v) { F[(size_t)i * NV + v] = f[v]; Wt[(size_t)i * NV + v] = w[v]; }
  alpha[i] = a;
}

template <int DIM>
__global__ void k_kfvs_points(int n, PhysParams P, const double* __restrict__ Wl, const double* __restrict__ Wr,
                              double* __restrict__ F) {
  constexpr int NV = DIM + 2;
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  double wl[NV], wr[NV], f[NV];
#pragma unroll
  for (int v = 0; v < NV; ++v) { wl[v] = Wl[(size_t)i * NV + v]; wr[v] = Wr[(size_t)i * NV + v]; }
  kfvs_flux<DIM>(P, wl, wr, f);
#pragma unroll
  for (int v = 0; v < NV; ++v) F[(size_t)i * NV + v] = f[v];
}

}  // namespace cgks
