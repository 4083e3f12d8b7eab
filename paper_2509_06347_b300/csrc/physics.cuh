// Device physics of the compact gas-kinetic scheme: Maxwellian moments,
// the time-accurate gas-kinetic interface flux and point value, the KFVS
// flux, the Euler flux and its increments, local frames and boundary ghosts.
//
// Paper (arXiv 2509.06347) references:
//   Sec 2.1  BGK model, Maxwellian, K internal degrees of freedom
//   Sec 2.3  Eqs. integral1, flux-3d-1, flux-3d-2, dis1, equli,
//            compatibility2, dis2, co, co-moment (gas-kinetic solver)
//   Sec 2.4  point value W(x, t^{n+1}) from the same distribution
//   Sec 3.3  discontinuity feedback factor
//   Sec 4.2  Euler flux T(W).n used by the LU-SGS flux splitting
//   Sec 5.2  first-order KFVS flux on the coarse levels
// Readings (the paper defers them): numerical collision time
// tau = C1 dt + C2 |pl - pr| / (pl + pr) dt; interface-equilibrium slopes are
// the mean of both sides; KFVS = collisionless split of constant states;
// slip wall = mirror ghost; supersonic far field = free stream on inflow faces,
// interior copy on outflow faces.
#pragma once
#include <cuda_runtime.h>
#include <math.h>

#include "dword.cuh"
#include "special.cuh"

namespace cgks {

// Parameters of the gas-kinetic flux in the scalar type S of the flux code
// (double, or double-word for the FP32-pipe variant).
template <typename S>
struct PhysT {
  S gamma;   // ratio of specific heats
  S K;       // internal degrees of freedom
  S c1, c2;  // collision-time coefficients
  S mu;      // dynamic viscosity (Navier-Stokes, tau = mu / p); 0 for the Euler equations
  // derived on the host: N = K + dim, 2/N, 4/N, 2/gamma
  S N, twoOverN, fourOverN, twoOverGamma;
};
using PhysParams = PhysT<double>;

inline PhysParams make_phys(double gamma, int dim, double c1, double c2, double mu = 0.0) {
  PhysParams p;
  p.gamma = gamma;
  p.mu = mu;
  p.K = dim == 2 ? (4.0 - 2.0 * gamma) / (gamma - 1.0) : (5.0 - 3.0 * gamma) / (gamma - 1.0);
  p.c1 = c1;
  p.c2 = c2;
  p.N = p.K + dim;
  p.twoOverN = 2.0 / p.N;
  p.fourOverN = 4.0 / p.N;
  p.twoOverGamma = 2.0 / gamma;
  return p;
}

inline PhysT<dword> phys_dword(const PhysParams& p) {
  PhysT<dword> q;
  q.gamma = dword(p.gamma);
  q.K = dword(p.K);
  q.mu = dword(p.mu);
  q.c1 = dword(p.c1);
  q.c2 = dword(p.c2);
  q.N = dword(p.N);
  q.twoOverN = dword(p.twoOverN);
  q.fourOverN = dword(p.fourOverN);
  q.twoOverGamma = dword(p.twoOverGamma);
  return q;
}

// Moments of a (half-)Maxwellian normalised by density: mu[n] = <u^n> in the
// normal direction over the chosen half line (or full line), mv/mw over the
// tangential lines, xi2/xi4 the internal-energy moments.
template <int DIM, typename S = double>
struct Mom {
  S mu[7];
  S mv[6];
  S mw[6];
  S xi2, xi4;
};

// primitive: rho, U[DIM], lambda = rho / (2 p)
template <int DIM, typename S = double>
struct Prim {
  S rho, irho, lam, h;  // h = 1 / (2 lambda) = p / rho
  S sl;                 // sqrt(lambda)
  S U[DIM];
};

// With A = rho E - |rho U|^2 / 2 = rho (E - rho |U|^2 / 2) and
// E - rho |U|^2 / 2 = N rho h / 2 (N = K + DIM), one reciprocal r = 1 / (rho A)
// gives both 1 / rho = A r and lambda = N rho^2 / (4 A) = (N / 4) rho^3 r.
template <int DIM, typename S>
__device__ __forceinline__ Prim<DIM, S> to_prim(const S* W, const PhysT<S>& P) {
  Prim<DIM, S> p;
  p.rho = W[0];
  S m2 = S(0.0);
#pragma unroll
  for (int d = 0; d < DIM; ++d) m2 += W[1 + d] * W[1 + d];
  const S A = p.rho * W[DIM + 1] - S(0.5) * m2;
  const S r = S(1.0) / (p.rho * A);
  p.irho = A * r;
#pragma unroll
  for (int d = 0; d < DIM; ++d) p.U[d] = W[1 + d] * p.irho;
  p.h = A * p.irho * p.irho * P.twoOverN;
  p.lam = S(0.25) * P.N * (p.rho * p.rho) * (p.rho * r);
  p.sl = sqrt(p.lam);
  return p;
}

// tangential and internal-energy moments (shared by full and half spaces)
template <int DIM, typename S>
__device__ __forceinline__ void tang_moments(const Prim<DIM, S>& p, S K, Mom<DIM, S>& m) {
  const S h = p.h;
  const S V = p.U[1];
  m.mv[0] = S(1.0);
  m.mv[1] = V;
#pragma unroll
  for (int n = 0; n < 4; ++n) m.mv[n + 2] = V * m.mv[n + 1] + (n + 1) * h * m.mv[n];
  if constexpr (DIM == 3) {
    const S Wv = p.U[DIM - 1];
    m.mw[0] = S(1.0);
    m.mw[1] = Wv;
#pragma unroll
    for (int n = 0; n < 4; ++n) m.mw[n + 2] = Wv * m.mw[n + 1] + (n + 1) * h * m.mw[n];
  } else {
#pragma unroll
    for (int n = 0; n < 6; ++n) m.mw[n] = n == 0 ? S(1.0) : S(0.0);
  }
  m.xi2 = K * h;
  m.xi4 = (K * K + S(2.0) * K) * h * h;
}

// normal moments: half = 0 full line, +1 u > 0, -1 u < 0
template <int DIM, typename S>
__device__ __forceinline__ void normal_moments(const Prim<DIM, S>& p, int half, Mom<DIM, S>& m) {
  const S U = p.U[0];
  const S h = p.h;
  if (half == 0) {
    m.mu[0] = S(1.0);
    m.mu[1] = U;
  } else {
    const S sl = p.sl;
    const S E = exp_neg(-p.lam * U * U);
    const S te = E * S(0.5 * M_2_SQRTPI) * (sl * h);  // e^{-lam U^2} / (2 sqrt(pi lam))
    const S hs = S(0.5) * erfc_with_exp(S(-half) * sl * U, E);  // erfc(x) from E = e^{-x^2}
    m.mu[0] = hs;
    m.mu[1] = U * hs + half * te;
  }
#pragma unroll
  for (int n = 0; n < 5; ++n) m.mu[n + 2] = U * m.mu[n + 1] + (n + 1) * h * m.mu[n];
}

// G(a, b, c) = <u^a v^b w^c>
template <int DIM, int A, int B, int C, typename S>
__device__ __forceinline__ S G(const Mom<DIM, S>& m) {
  if constexpr (DIM == 2 && C > 0) return S(0.0);
  if constexpr (DIM == 3) return m.mu[A] * m.mv[B] * m.mw[C];
  else return m.mu[A] * m.mv[B];
}

// <u^a v^b w^c psi>
template <int DIM, int A, int B, int C, typename S>
__device__ __forceinline__ void psi_mom(const Mom<DIM, S>& m, S* out) {
  out[0] = G<DIM, A, B, C>(m);
  out[1] = G<DIM, A + 1, B, C>(m);
  out[2] = G<DIM, A, B + 1, C>(m);
  if constexpr (DIM == 3) {
    out[3] = G<DIM, A, B, C + 1>(m);
    out[DIM + 1] = S(0.5) * (G<DIM, A + 2, B, C>(m) + G<DIM, A, B + 2, C>(m) + G<DIM, A, B, C + 2>(m) +
                             m.xi2 * G<DIM, A, B, C>(m));
  } else {
    out[DIM + 1] = S(0.5) * (G<DIM, A + 2, B, C>(m) + G<DIM, A, B + 2, C>(m) + m.xi2 * G<DIM, A, B, C>(m));
  }
}

// Solve <psi (a . psi)> = sc b for a (sc b normalised by density): explicit
// inverse of the Maxwellian moment matrix.  The scale sc (1 / rho, or -1 / rho
// for the time slopes) enters through the per-side factors 2 lambda and
// 4 lambda^2 / N, so b itself is never scaled.
template <int DIM, typename S>
__device__ __forceinline__ void slope_solve(const Prim<DIM, S>& p, const PhysT<S>& P, const S* b, S sc, S* a) {
  S q2 = S(0.0), ub = S(0.0), bd[DIM];
#pragma unroll
  for (int d = 0; d < DIM; ++d) {
    q2 += p.U[d] * p.U[d];
    bd[d] = b[1 + d] - p.U[d] * b[0];
    ub += p.U[d] * bd[d];
  }
  const S e = q2 + P.N * p.h;
  const S aE = ((P.fourOverN * p.lam * p.lam) * sc) * (S(2.0) * b[DIM + 1] - e * b[0] - S(2.0) * ub);
  const S tl = (S(2.0) * p.lam) * sc;
  S s = S(0.0);
#pragma unroll
  for (int d = 0; d < DIM; ++d) {
    a[1 + d] = tl * bd[d] - p.U[d] * aE;
    s += p.U[d] * a[1 + d];
  }
  a[DIM + 1] = aE;
  a[0] = sc * b[0] - s - S(0.5) * aE * e;
}

// The part of the distribution that multiplies a Maxwellian in the flux and
// point-value integrals is a polynomial in the velocity x = (u, v[, w]) and
// xi^2:  c0 + cA sum_d (a_d . psi) x_d + cT (A . psi), with psi = (1, x,
// (|x|^2 + xi^2) / 2).  Expanded once per side it reads
//   P = p0 + pl.x + x^T pq x + h xi^2 + sum_d qc_d x_d (|x|^2 + xi^2),
// so every moment <x^alpha psi P> is a short sum of products of the 1-D
// moments instead of one matrix-vector product per slope vector.
template <int DIM, typename S = double>
struct Poly {
  S p0, h;
  S pl[DIM], qc[DIM];
  S pq[DIM][DIM];  // upper triangle used
};

// A == nullptr: no time-slope term
template <int DIM, typename S>
__device__ __forceinline__ Poly<DIM, S> make_poly(S c0, S cA, S cT, const S (*a)[DIM + 2], const S* A) {
  constexpr int E = DIM + 1;
  Poly<DIM, S> P;
  const S hT = A ? S(0.5) * cT * A[E] : S(0.0);
  P.p0 = A ? c0 + cT * A[0] : c0;
  P.h = hT;
#pragma unroll
  for (int d = 0; d < DIM; ++d) {
    P.pl[d] = A ? cA * a[d][0] + cT * A[1 + d] : cA * a[d][0];
    P.qc[d] = S(0.5) * cA * a[d][E];
    P.pq[d][d] = cA * a[d][1 + d] + hT;
#pragma unroll
    for (int e = d + 1; e < DIM; ++e) P.pq[d][e] = cA * (a[d][1 + e] + a[e][1 + d]);
  }
  return P;
}

// 2-D form of <u^A0 psi P>.  Grouped by powers of v, P reads
//   sum_j v^j (sum_i c_ij u^i) + xi^2 (e_00 + e_10 u + e_01 v),
// with c_i0 = (p0, pl0, pq00, qc0), c_i1 = (pl1, pq01, qc1), c_i2 = (pq11, qc0),
// c_03 = qc1 and e = (h, qc0, qc1).  With D_j(a) = sum_i c_ij mu[a+i],
// E_0(a) = h mu[a] + qc0 mu[a+1] and E_1(a) = qc1 mu[a] = D_3(a):
//   <u^a v^b P>      = sum_j mv[b+j] D_j(a) + xi2 (mv[b] E_0(a) + mv[b+1] E_1(a))
//   <u^a xi^2 P>     = xi2 sum_j mv[j] D_j(a) + xi4 (mv[0] E_0(a) + mv[1] E_1(a)).
// Each 1-D moment product is formed once instead of once per output.
template <int A0, typename S>
__device__ __forceinline__ void poly_psi_mom_2d(const Mom<2, S>& m, const Poly<2, S>& P, S* out) {
  const S* mu = m.mu;
  const S* mv = m.mv;
  S F0[3], F1[3], D2[3], D3[3], D0a = S(0.0), D1a = S(0.0), E0a = S(0.0);
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    const int a = A0 + k;
    const S d0 = P.p0 * mu[a] + P.pl[0] * mu[a + 1] + P.pq[0][0] * mu[a + 2] + P.qc[0] * mu[a + 3];
    const S d1 = P.pl[1] * mu[a] + P.pq[0][1] * mu[a + 1] + P.qc[1] * mu[a + 2];
    const S e0 = P.h * mu[a] + P.qc[0] * mu[a + 1];
    D2[k] = P.pq[1][1] * mu[a] + P.qc[0] * mu[a + 1];
    D3[k] = P.qc[1] * mu[a];
    F0[k] = d0 + m.xi2 * e0;
    F1[k] = d1 + m.xi2 * D3[k];
    if (k == 0) { D0a = d0; D1a = d1; E0a = e0; }
  }
  // <u^(A0+k) v^b P>; mv[0] = 1.  Macc adds it to acc (one chain of
  // multiply-adds, no separate sum)
  auto M = [&](int k, int b) { return mv[b] * F0[k] + mv[b + 1] * F1[k] + mv[b + 2] * D2[k] + mv[b + 3] * D3[k]; };
  auto Macc = [&](S acc, int k, int b) {
    return acc + mv[b] * F0[k] + mv[b + 1] * F1[k] + mv[b + 2] * D2[k] + mv[b + 3] * D3[k];
  };
  out[0] = M(0, 0);
  out[1] = M(1, 0);
  out[2] = M(0, 1);
  const S sv = D0a * mv[0] + D1a * mv[1] + D2[0] * mv[2] + D3[0] * mv[3];
  const S se = E0a * mv[0] + D3[0] * mv[1];
  const S sE = Macc(M(2, 0), 0, 2) + m.xi2 * sv + m.xi4 * se;
  out[3] = S(0.5) * sE;
}

// 3-D form of <u^A0 psi P>, grouped by the powers (j, k) of v and w:
//   D_00(a) = p0 mu[a] + pl0 mu[a+1] + pq00 mu[a+2] + qc0 mu[a+3]
//   D_10(a) = pl1 mu[a] + pq01 mu[a+1] + qc1 mu[a+2]
//   D_01(a) = pl2 mu[a] + pq02 mu[a+1] + qc2 mu[a+2]
//   D_20(a) = pq11 mu[a] + qc0 mu[a+1],  D_02(a) = pq22 mu[a] + qc0 mu[a+1]
//   D_11(a) = pq12 mu[a],  D_30 = D_12 = Q1(a) = qc1 mu[a],  D_21 = D_03 = Q2(a) = qc2 mu[a]
// and the xi^2 part E_00(a) = h mu[a] + qc0 mu[a+1], E_10 = Q1, E_01 = Q2, so
//   <u^a v^b w^c P> = sum_jk mv[b+j] mw[c+k] (D_jk(a) + xi2 E_jk(a))
//   <u^a xi^2 P>    = xi2 sum_jk mv[j] mw[k] D_jk(a) + xi4 sum_jk mv[j] mw[k] E_jk(a).
template <int A0, typename S>
__device__ __forceinline__ void poly_psi_mom_3d(const Mom<3, S>& m, const Poly<3, S>& P, S* out) {
  const S* mu = m.mu;
  const S* mv = m.mv;
  const S* mw = m.mw;
  struct Grp { S F00, F10, F01, D20, D02, D11, Q1, Q2; };
  Grp g[3];
  S D00a = S(0.0), D10a = S(0.0), D01a = S(0.0), E00a = S(0.0);
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    const int a = A0 + k;
    const S d00 = P.p0 * mu[a] + P.pl[0] * mu[a + 1] + P.pq[0][0] * mu[a + 2] + P.qc[0] * mu[a + 3];
    const S d10 = P.pl[1] * mu[a] + P.pq[0][1] * mu[a + 1] + P.qc[1] * mu[a + 2];
    const S d01 = P.pl[2] * mu[a] + P.pq[0][2] * mu[a + 1] + P.qc[2] * mu[a + 2];
    const S e00 = P.h * mu[a] + P.qc[0] * mu[a + 1];
    g[k].D20 = P.pq[1][1] * mu[a] + P.qc[0] * mu[a + 1];
    g[k].D02 = P.pq[2][2] * mu[a] + P.qc[0] * mu[a + 1];
    g[k].D11 = P.pq[1][2] * mu[a];
    g[k].Q1 = P.qc[1] * mu[a];
    g[k].Q2 = P.qc[2] * mu[a];
    g[k].F00 = d00 + m.xi2 * e00;
    g[k].F10 = d10 + m.xi2 * g[k].Q1;
    g[k].F01 = d01 + m.xi2 * g[k].Q2;
    if (k == 0) { D00a = d00; D10a = d10; D01a = d01; E00a = e00; }
  }
  // <u^(A0+k) v^b w^c P>, summed by powers of w; mv[0] = mw[0] = 1
  auto Macc = [&](S acc, int k, int b, int c) {
    const Grp& q = g[k];
    return acc + mw[c] * (mv[b] * q.F00 + mv[b + 1] * q.F10 + mv[b + 2] * q.D20 + mv[b + 3] * q.Q1) +
           mw[c + 1] * (mv[b] * q.F01 + mv[b + 1] * q.D11 + mv[b + 2] * q.Q2) +
           mw[c + 2] * (mv[b] * q.D02 + mv[b + 1] * q.Q1) + mw[c + 3] * (mv[b] * q.Q2);
  };
  auto M = [&](int k, int b, int c) {
    const Grp& q = g[k];
    return mw[c] * (mv[b] * q.F00 + mv[b + 1] * q.F10 + mv[b + 2] * q.D20 + mv[b + 3] * q.Q1) +
           mw[c + 1] * (mv[b] * q.F01 + mv[b + 1] * q.D11 + mv[b + 2] * q.Q2) +
           mw[c + 2] * (mv[b] * q.D02 + mv[b + 1] * q.Q1) + mw[c + 3] * (mv[b] * q.Q2);
  };
  out[0] = M(0, 0, 0);
  out[1] = M(1, 0, 0);
  out[2] = M(0, 1, 0);
  out[3] = M(0, 0, 1);
  const Grp& q = g[0];
  const S sv = (D00a + mv[1] * D10a + mv[2] * q.D20 + mv[3] * q.Q1) +
               mw[1] * (D01a + mv[1] * q.D11 + mv[2] * q.Q2) + mw[2] * (q.D02 + mv[1] * q.Q1) + mw[3] * q.Q2;
  const S se = E00a + mv[1] * q.Q1 + mw[1] * q.Q2;
  const S sE = Macc(Macc(M(2, 0, 0), 0, 2, 0), 0, 0, 2) + m.xi2 * sv + m.xi4 * se;
  out[4] = S(0.5) * sE;
}

// out = <u^A0 psi P>
template <int DIM, int A0, typename S>
__device__ __forceinline__ void poly_psi_mom(const Mom<DIM, S>& m, const Poly<DIM, S>& P, S* out) {
  if constexpr (DIM == 2) {
    poly_psi_mom_2d<A0, S>(m, P, out);
  } else {
    poly_psi_mom_3d<A0, S>(m, P, out);
  }
}

// Sum over directions d of (dF_d/dW) . dW_d for the Euler fluxes F_d along the
// local axes: for a Maxwellian g(W(x)), int u_d psi dg/dx_d = d/dx_d F_d(W), so
// this equals <psi (a.u)> of the full-space Maxwellian (times rho) without
// forming the velocity moments.  ir = 1 / W[0], which every caller already holds.
// Only the first ND directions are summed (the others are taken as zero).
// Every accumulation is written as acc + a b + c d, which FP64 code issues as
// fused multiply-adds into the accumulator.
template <int DIM, typename S, int ND = DIM>
__device__ __forceinline__ void euler_flux_divergence(S gamma, const S* W, S ir, const S (*dW)[DIM + 2], S* out) {
  constexpr int NV = DIM + 2;
  S u[DIM], q2 = S(0.0);
#pragma unroll
  for (int i = 0; i < DIM; ++i) {
    u[i] = W[1 + i] * ir;
    q2 += u[i] * u[i];
  }
  const S gm1 = gamma - S(1.0), hq2 = S(0.5) * q2;
  const S p = gm1 * (W[NV - 1] - W[0] * hq2);
  const S H = (W[NV - 1] + p) * ir;  // total enthalpy
#pragma unroll
  for (int d = 0; d < ND; ++d) {
    const S* g = dW[d];
    // derivatives of primitive quantities along this direction
    S du[DIM], udu = S(0.0);
#pragma unroll
    for (int i = 0; i < DIM; ++i) {
      du[i] = (g[1 + i] - u[i] * g[0]) * ir;
      udu += u[i] * du[i];
    }
    const S dp = gm1 * (g[NV - 1] - g[0] * hq2 - W[0] * udu);
    out[0] = d == 0 ? g[1] : out[0] + g[1 + d];
#pragma unroll
    for (int i = 0; i < DIM; ++i)
      out[1 + i] = d == 0 ? g[1 + d] * u[i] + W[1 + d] * du[i] : out[1 + i] + g[1 + d] * u[i] + W[1 + d] * du[i];
    out[1 + d] += dp;
    const S dH = (g[NV - 1] + dp - H * g[0]) * ir;
    out[NV - 1] = d == 0 ? g[1 + d] * H + W[1 + d] * dH : out[NV - 1] + g[1 + d] * H + W[1 + d] * dH;
  }
}

// Sum over directions d of (dQ_d/dW) . dW_d, with Q_d(W) = rho <u_0 u_d psi g_W>
// the second velocity moments of the full-space Maxwellian of W (u_0 along the
// local normal).  For the slopes a_d of that Maxwellian (<psi (a_d . psi)> = dW_d
// / rho) this equals rho <u_0 psi (a . u)>, the part of the equilibrium flux
// that the time integral T2 multiplies, in closed form.  With theta = p / rho,
// D velocity components and K internal degrees of freedom,
//   Q_d^rho = rho U_0 U_d + p delta_0d
//   Q_d^i   = rho U_0 U_d U_i + p (U_0 delta_di + U_d delta_0i + U_i delta_0d)
//   Q_d^E   = U_0 U_d (rho |U|^2 + (D + 4 + K) p) / 2
//             + delta_0d (p |U|^2 + (D + 2 + K) p theta) / 2.
// ir = 1 / W[0].  Accumulations as in euler_flux_divergence.
template <int DIM, typename S>
__device__ __forceinline__ void second_moment_divergence(S gamma, S K, const S* W, S ir, const S (*dW)[DIM + 2],
                                                         S* out) {
  constexpr int NV = DIM + 2;
  S U[DIM], q2 = S(0.0);
#pragma unroll
  for (int i = 0; i < DIM; ++i) {
    U[i] = W[1 + i] * ir;
    q2 += U[i] * U[i];
  }
  const S gm1 = gamma - S(1.0), hq2 = S(0.5) * q2;
  const S p = gm1 * (W[NV - 1] - W[0] * hq2);
  const S th = p * ir;
  const S cA = S(double(DIM + 4)) + K, cB = S(double(DIM + 2)) + K;
  const S hcA = S(0.5) * cA, hcB = S(0.5) * cB;
  const S hA = W[0] * hq2 + hcA * p;  // (rho |U|^2 + cA p) / 2
#pragma unroll
  for (int d = 0; d < DIM; ++d) {
    const S* g = dW[d];
    S du[DIM], udu = S(0.0);
#pragma unroll
    for (int i = 0; i < DIM; ++i) {
      du[i] = (g[1 + i] - U[i] * g[0]) * ir;
      udu += U[i] * du[i];
    }
    const S dp = gm1 * (g[NV - 1] - g[0] * hq2 - W[0] * udu);
    const S u0d = U[0] * U[d];
    const S du0d = du[0] * U[d] + U[0] * du[d];  // d(U_0 U_d)
    out[0] = (d == 0 ? dp : out[0]) + g[0] * u0d + W[0] * du0d;
    // d(rho U_0 U_d U_i) = (g0 u0d + rho du0d) U_i + rho u0d du_i
    const S gw = g[0] * u0d + W[0] * du0d, wu = W[0] * u0d;
#pragma unroll
    for (int i = 0; i < DIM; ++i) {
      S t = d == 0 ? gw * U[i] + wu * du[i] : out[1 + i] + gw * U[i] + wu * du[i];
      if (i == d) t = t + dp * U[0] + p * du[0];
      if (i == 0) t = t + dp * U[d] + p * du[d];
      if (d == 0) t = t + dp * U[i] + p * du[i];
      out[1 + i] = t;
    }
    // d(A) / 2 with A = rho |U|^2 + cA p
    const S hdA = g[0] * hq2 + W[0] * udu + hcA * dp;
    out[NV - 1] = d == 0 ? du0d * hA + u0d * hdA : out[NV - 1] + du0d * hA + u0d * hdA;
    if (d == 0) {
      const S dth = (dp - th * g[0]) * ir;
      out[NV - 1] = out[NV - 1] + dp * hq2 + p * udu + hcB * (dp * th + p * dth);
    }
  }
}

// (dF_n/dW) . v for the Euler flux through the local normal (first axis)
template <int DIM, typename S>
__device__ __forceinline__ void euler_flux_jvp_normal(S gamma, const S* W, S ir, const S* v, S* out) {
  constexpr int NV = DIM + 2;
  S g[DIM][NV];
#pragma unroll
  for (int d = 0; d < DIM; ++d)
#pragma unroll
    for (int i = 0; i < NV; ++i) g[d][i] = d == 0 ? v[i] : S(0.0);
  euler_flux_divergence<DIM, S, 1>(gamma, W, ir, g, out);
}

// Out-of-line variants for the double-word flux.  Its code, fully inlined, is
// several times larger than the FP64 code and overflows the instruction cache,
// so the helpers called several times per Gauss point become shared calls
// there; the FP64 instantiation keeps them inline.
template <typename S>
struct OutOfLine { static constexpr bool value = false; };
template <>
struct OutOfLine<dword> { static constexpr bool value = true; };

template <int DIM, typename S>
__device__ __noinline__ void slope_solve_ool(const Prim<DIM, S>& p, const PhysT<S>& P, const S* b, S sc, S* a) {
  slope_solve<DIM, S>(p, P, b, sc, a);
}
template <int DIM, typename S>
__device__ __forceinline__ void slope_solve_c(const Prim<DIM, S>& p, const PhysT<S>& P, const S* b, S sc, S* a) {
  if constexpr (OutOfLine<S>::value) slope_solve_ool<DIM, S>(p, P, b, sc, a);
  else slope_solve<DIM, S>(p, P, b, sc, a);
}
template <int DIM, typename S>
__device__ __noinline__ void euler_flux_divergence_ool(S gamma, const S* W, S ir, const S (*dW)[DIM + 2], S* out) {
  euler_flux_divergence<DIM, S>(gamma, W, ir, dW, out);
}
template <int DIM, typename S>
__device__ __forceinline__ void euler_flux_divergence_c(S gamma, const S* W, S ir, const S (*dW)[DIM + 2], S* out) {
  if constexpr (OutOfLine<S>::value) euler_flux_divergence_ool<DIM, S>(gamma, W, ir, dW, out);
  else euler_flux_divergence<DIM, S>(gamma, W, ir, dW, out);
}
template <int DIM, typename S>
__device__ __noinline__ void second_moment_divergence_ool(S gamma, S K, const S* W, S ir, const S (*dW)[DIM + 2],
                                                         S* out) {
  second_moment_divergence<DIM, S>(gamma, K, W, ir, dW, out);
}
template <int DIM, typename S>
__device__ __forceinline__ void second_moment_divergence_c(S gamma, S K, const S* W, S ir, const S (*dW)[DIM + 2],
                                                           S* out) {
  if constexpr (OutOfLine<S>::value) second_moment_divergence_ool<DIM, S>(gamma, K, W, ir, dW, out);
  else second_moment_divergence<DIM, S>(gamma, K, W, ir, dW, out);
}
template <int DIM, typename S>
__device__ __noinline__ void moments_ool(const Prim<DIM, S>& p, S K, int half, Mom<DIM, S>& m) {
  tang_moments<DIM, S>(p, K, m);
  normal_moments<DIM, S>(p, half, m);
}
template <int DIM, typename S>
__device__ __forceinline__ void moments_c(const Prim<DIM, S>& p, S K, int half, Mom<DIM, S>& m) {
  if constexpr (OutOfLine<S>::value) {
    moments_ool<DIM, S>(p, K, half, m);
  } else {
    tang_moments<DIM, S>(p, K, m);
    normal_moments<DIM, S>(p, half, m);
  }
}
// <u^A0 psi (c0 + cA (a . u) + cT (A . psi))>
template <int DIM, int A0, typename S>
__device__ __forceinline__ void kin_moments(const Mom<DIM, S>& m, S c0, S cA, S cT, const S (*a)[DIM + 2],
                                            const S* A, S* out) {
  poly_psi_mom<DIM, A0, S>(m, make_poly<DIM, S>(c0, cA, cT, a, A), out);
}
template <int DIM, int A0, typename S>
__device__ __noinline__ void kin_moments_ool(const Mom<DIM, S>& m, S c0, S cA, S cT, const S (*a)[DIM + 2],
                                             const S* A, S* out) {
  kin_moments<DIM, A0, S>(m, c0, cA, cT, a, A, out);
}
template <int DIM, int A0, typename S>
__device__ __forceinline__ void kin_moments_c(const Mom<DIM, S>& m, S c0, S cA, S cT, const S (*a)[DIM + 2],
                                              const S* A, S* out) {
  if constexpr (OutOfLine<S>::value) kin_moments_ool<DIM, A0, S>(m, c0, cA, cT, a, A, out);
  else kin_moments<DIM, A0, S>(m, c0, cA, cT, a, A, out);
}

// Gas-kinetic flux (time average over [0, dt]) and point value at t = dt in
// the local frame (u normal).  G?[d][v] = derivative along local direction d.
// Returns the DF point factor 1 / (1 + D^2) of Sec 3.3, formed from the same
// primitives: 1 / p = 2 lambda / rho and 1 / c = sqrt(rho / (gamma p)) =
// sqrt(2 lambda / gamma), so D = |pl - pr| (1/pl + 1/pr) + |Ul/cl - Ur/cr|^2
// needs no division beyond the final one.
template <int DIM, bool POINT = true, typename S = double>
__device__ S gks_flux(const PhysT<S>& P, const S* Wl, const S (*Gl)[DIM + 2], const S* Wr, const S (*Gr)[DIM + 2],
                      S dt, S* F, S* Wt) {
  constexpr int NV = DIM + 2;
  const S K = P.K;
  const Prim<DIM, S> pl = to_prim<DIM, S>(Wl, P), pr = to_prim<DIM, S>(Wr, P);
  const S pL = pl.rho * pl.h, pR = pr.rho * pr.h;
  S alpha;
  {
    S dm2 = S(0.0);
#pragma unroll
    for (int d = 0; d < DIM; ++d) {
      const S dm = pl.U[d] * pl.sl - pr.U[d] * pr.sl;
      dm2 += dm * dm;
    }
    const S D = S(2.0) * fabs(pL - pR) * (pl.lam * pl.irho + pr.lam * pr.irho) + P.twoOverGamma * dm2;
    alpha = S(1.0) / (S(1.0) + D * D);
  }
  // half-space moments for the kinetic part
  Mom<DIM, S> ml, mr;
  moments_c<DIM, S>(pl, K, +1, ml);
  moments_c<DIM, S>(pr, K, -1, mr);
  // interface equilibrium from half-space moments (Eq. compatibility2)
  S Wc[NV], t[NV];
  psi_mom<DIM, 0, 0, 0>(ml, Wc);
  psi_mom<DIM, 0, 0, 0>(mr, t);
#pragma unroll
  for (int i = 0; i < NV; ++i) Wc[i] = pl.rho * Wc[i] + pr.rho * t[i];
  // pressure of the interface equilibrium
  const S irc = S(1.0) / Wc[0];
  S pwc;
  {
    S kc = S(0.0);
#pragma unroll
    for (int d = 0; d < DIM; ++d) kc += Wc[1 + d] * Wc[1 + d];
    pwc = (P.gamma - S(1.0)) * (Wc[DIM + 1] - S(0.5) * kc * irc);
  }
  {
    // vacuum (both sides moving apart): no admissible interface equilibrium;
    // take the collisionless limit, i.e. the KFVS flux, point value W^c
    if (!(Wc[0] > S(1e-10) * (pl.rho + pr.rho)) || !(pwc > S(1e-10) * (pL + pR))) {
      S a[NV], b[NV];
      psi_mom<DIM, 1, 0, 0>(ml, a);
      psi_mom<DIM, 1, 0, 0>(mr, b);
#pragma unroll
      for (int i = 0; i < NV; ++i) {
        F[i] = pl.rho * a[i] + pr.rho * b[i];
        Wt[i] = Wc[i];
      }
      return alpha;
    }
  }
  // spatial slopes of the two kinetic Maxwellians (Eq. co); the interface
  // Maxwellian's slopes enter only through closed-form moments below
  S al[DIM][NV], ar[DIM][NV];
#pragma unroll
  for (int d = 0; d < DIM; ++d) {
    slope_solve_c<DIM, S>(pl, P, Gl[d], pl.irho, al[d]);
    slope_solve_c<DIM, S>(pr, P, Gr[d], pr.irho, ar[d]);
  }
  // time slopes from <A + a.u> = 0, with <psi (a.u)> of a full-space
  // Maxwellian given by the Euler-flux divergence of its slopes
  S Al[NV], Ar[NV];
  {
    S s[NV];
    euler_flux_divergence_c<DIM, S>(P.gamma, Wl, pl.irho, Gl, s);
    slope_solve_c<DIM, S>(pl, P, s, -pl.irho, Al);
    euler_flux_divergence_c<DIM, S>(P.gamma, Wr, pr.irho, Gr, s);
    slope_solve_c<DIM, S>(pr, P, s, -pr.irho, Ar);
  }
  // interface Maxwellian with the mean slopes g_c = (G_l + G_r) / 2: with the
  // Euler-flux divergence D(g) (linear in g), rho_c <psi (a_c.u)> = D(g_c);
  // its time slope gives rho_c <psi (A_c.psi)> = -D(g_c) and
  // rho_c <u psi (A_c.psi)> = -J_n D(g_c) (J_n the Jacobian of the Euler flux
  // through the normal); rho_c <u psi (a_c.u)> is the
  // divergence of the second moments Q(g_c); <u psi> is the Euler flux.  They
  // are formed here from the sum G_l + G_r = 2 g_c, and the factor 1/2 joins
  // the time integrals below.
  S PAc[NV], UAc[NV], QAc[NV], Fc[NV];  // D(2 g_c), J_n D(2 g_c), Q(2 g_c)
  {
    S gs[DIM][NV];
#pragma unroll
    for (int d = 0; d < DIM; ++d)
#pragma unroll
      for (int i = 0; i < NV; ++i) gs[d][i] = Gl[d][i] + Gr[d][i];
    euler_flux_divergence_c<DIM, S>(P.gamma, Wc, irc, gs, PAc);
    second_moment_divergence_c<DIM, S>(P.gamma, K, Wc, irc, gs, QAc);
    euler_flux_jvp_normal<DIM, S>(P.gamma, Wc, irc, PAc, UAc);
    // Euler flux of W^c through the local normal
    const S un = Wc[1] * irc;
#pragma unroll
    for (int i = 0; i < NV; ++i) Fc[i] = un * Wc[i];
    Fc[1] += pwc;
    Fc[NV - 1] += un * pwc;
  }
  // Collision time.  Euler: tau = C1 dt + C2 |dp| / (pl + pr) dt; Navier-Stokes
  // (Sec 2.1): the physical mu / p of the interface equilibrium in place of
  // C1 dt.  Either way tau / dt = a / b, and one reciprocal r = 1 / (a b) gives
  // s = tau / dt = a^2 r and dt / tau = b^2 r.
  const S sp = pL + pR, cdp = P.c2 * fabs(pL - pR);
  S ta, tb;
  if (P.mu > S(0.0)) {
    tb = pwc * dt * sp;
    ta = P.mu * sp + cdp * pwc * dt;
  } else {
    tb = sp;
    ta = P.c1 * sp + cdp;
  }
  const S tr = S(1.0) / (ta * tb);
  const S s = ta * ta * tr;
  const S tau = s * dt;
  const S e = exp_neg(-(tb * tb * tr));
  // the time integrals T1..T5 of the flux divided by dt, so that the flux
  // needs no final division; the point-value coefficients C1..C3 as they are
  const S T1 = S(1.0) - s * (S(1.0) - e);
  const S T2 = tau * (S(2.0) * s - S(1.0) - (S(1.0) + S(2.0) * s) * e);
  const S T3 = S(0.5) * dt - tau + tau * s * (S(1.0) - e);
  const S T4 = s * (S(1.0) - e);
  const S T5 = tau * (s - (S(1.0) + s) * e);
  const S C1 = S(1.0) - e, C2 = (dt + tau) * e - tau, C3 = dt - tau + tau * e;
  // --- equilibrium part (g^c, full space): T1 <u psi> + T2 <u psi (a_c . u)>
  // + T3 <u psi (A_c . psi)>; point value C1 <psi> + (C2 - C3) <psi (A_c . psi)>
  // (times rho_c; the slope terms from the doubled-slope quantities above)
  S fx[NV], wx[NV];
  const S hT2 = S(0.5) * T2, hT3 = S(0.5) * T3, hC23 = S(0.5) * (C2 - C3);
#pragma unroll
  for (int i = 0; i < NV; ++i) {
    F[i] = T1 * Fc[i] + hT2 * QAc[i] - hT3 * UAc[i];
    Wt[i] = POINT ? C1 * Wc[i] + hC23 * PAc[i] : S(0.0);
  }
  // --- kinetic part (g^l on u > 0, g^r on u < 0)
#pragma unroll
  for (int side = 0; side < 2; ++side) {
    const Mom<DIM, S>& m = side == 0 ? ml : mr;
    const S(*a)[NV] = side == 0 ? al : ar;
    const S* Ak = side == 0 ? Al : Ar;
    const S rho = side == 0 ? pl.rho : pr.rho;
    // flux: T4 - (tau T4 + T5) (a . u) - tau T4 (A . psi); point value at dt:
    // e - e (tau + dt) (a . u) - e tau (A . psi)
    kin_moments_c<DIM, 1, S>(m, T4, -(tau * T4 + T5), -tau * T4, a, Ak, fx);
    if (POINT) kin_moments_c<DIM, 0, S>(m, e, -e * (tau + dt), -e * tau, a, Ak, wx);
#pragma unroll
    for (int i = 0; i < NV; ++i) {
      F[i] += rho * fx[i];
      if (POINT) Wt[i] += rho * wx[i];
    }
  }
  return alpha;
}

// KFVS flux of constant states, local frame
template <int DIM>
__device__ __forceinline__ void kfvs_flux(const PhysParams& P, const double* Wl, const double* Wr, double* F) {
  constexpr int NV = DIM + 2;
  const double K = P.K;
  const Prim<DIM> pl = to_prim<DIM>(Wl, P), pr = to_prim<DIM>(Wr, P);
  Mom<DIM> ml, mr;
  tang_moments<DIM>(pl, K, ml);
  tang_moments<DIM>(pr, K, mr);
  normal_moments<DIM>(pl, +1, ml);
  normal_moments<DIM>(pr, -1, mr);
  double a[NV], b[NV];
  psi_mom<DIM, 1, 0, 0>(ml, a);
  psi_mom<DIM, 1, 0, 0>(mr, b);
#pragma unroll
  for (int i = 0; i < NV; ++i) F[i] = pl.rho * a[i] + pr.rho * b[i];
}


// ---------------------------------------------------------------------------
// frames: rows n, t1, t2
template <int DIM, typename S = double>
struct Frame {
  S r[DIM][DIM];
};
template <int DIM, typename S>
__device__ __forceinline__ Frame<DIM, S> make_frame(const S* n) {
  Frame<DIM, S> f;
  if constexpr (DIM == 2) {
    f.r[0][0] = n[0]; f.r[0][1] = n[1];
    f.r[1][0] = -n[1]; f.r[1][1] = n[0];
  } else {
    int a = 0;
    if (fabs(n[1]) < fabs(n[a])) a = 1;
    if (fabs(n[DIM - 1]) < fabs(n[a])) a = 2;
    S e[3] = {S(0.0), S(0.0), S(0.0)};
    e[a] = S(1.0);
    S t1[3] = {n[1] * e[2] - n[2] * e[1], n[2] * e[0] - n[0] * e[2], n[0] * e[1] - n[1] * e[0]};
    const S il = S(1.0) / sqrt(t1[0] * t1[0] + t1[1] * t1[1] + t1[2] * t1[2]);
    for (int i = 0; i < 3; ++i) t1[i] *= il;
    const S t2[3] = {n[1] * t1[2] - n[2] * t1[1], n[2] * t1[0] - n[0] * t1[2], n[0] * t1[1] - n[1] * t1[0]};
    for (int i = 0; i < DIM; ++i) { f.r[0][i] = n[i]; f.r[1][i] = t1[i]; f.r[DIM - 1][i] = t2[i]; }
  }
  return f;
}
template <int DIM, typename S>
__device__ __forceinline__ void to_local(const Frame<DIM, S>& f, const S* W, S* Wl) {
  Wl[0] = W[0];
#pragma unroll
  for (int a = 0; a < DIM; ++a) {
    S s = S(0.0);
#pragma unroll
    for (int d = 0; d < DIM; ++d) s += f.r[a][d] * W[1 + d];
    Wl[1 + a] = s;
  }
  Wl[DIM + 1] = W[DIM + 1];
}
template <int DIM, typename S>
__device__ __forceinline__ void to_global(const Frame<DIM, S>& f, const S* Wl, S* W) {
  W[0] = Wl[0];
#pragma unroll
  for (int d = 0; d < DIM; ++d) {
    S s = S(0.0);
#pragma unroll
    for (int a = 0; a < DIM; ++a) s += f.r[a][d] * Wl[1 + a];
    W[1 + d] = s;
  }
  W[DIM + 1] = Wl[DIM + 1];
}
// global gradient g[v][d] -> local derivatives Gl[a][v'] (direction a, rotated variable v')
template <int DIM, typename S>
__device__ __forceinline__ void grad_to_local(const Frame<DIM, S>& f, const S (*g)[DIM], S (*Gl)[DIM + 2]) {
  constexpr int NV = DIM + 2;
#pragma unroll
  for (int a = 0; a < DIM; ++a) {
    S dir[NV];
#pragma unroll
    for (int v = 0; v < NV; ++v) {
      S s = S(0.0);
#pragma unroll
      for (int d = 0; d < DIM; ++d) s += f.r[a][d] * g[v][d];
      dir[v] = s;
    }
    to_local<DIM, S>(f, dir, Gl[a]);
  }
}

// ---------------------------------------------------------------------------
// Euler flux T(W).n and its increment T(W + dW).n - T(W).n
template <int DIM, typename T>
__device__ __forceinline__ void euler_flux(T gamma, const T* W, const T* n, T* F) {
  T ke = 0, un = 0;
  const T ir = T(1) / W[0];
#pragma unroll
  for (int d = 0; d < DIM; ++d) { ke += W[1 + d] * W[1 + d]; un += W[1 + d] * n[d]; }
  un *= ir;
  const T p = (gamma - T(1)) * (W[DIM + 1] - T(0.5) * ke * ir);
  F[0] = W[0] * un;
#pragma unroll
  for (int d = 0; d < DIM; ++d) F[1 + d] = W[1 + d] * un + p * n[d];
  F[DIM + 1] = (W[DIM + 1] + p) * un;
}

// cancellation-free increment: with u' = (m + dm)/(rho + drho), du = u' - u
// computed from (dm - u drho)/(rho + drho), every term is a product with an
// increment, so the result carries relative (not absolute) rounding.
template <int DIM, typename T>
__device__ __forceinline__ void euler_flux_increment(T gamma, const T* W, const T* dW, const T* n, T* dF) {
  const T rho = W[0], rho1 = W[0] + dW[0];
  const T ir = T(1) / rho, ir1 = T(1) / rho1;
  T u[DIM], du[DIM], u1[DIM];
  T un = 0, dun = 0, u1n = 0, ke_d = 0;
#pragma unroll
  for (int d = 0; d < DIM; ++d) {
    u[d] = W[1 + d] * ir;
    du[d] = (dW[1 + d] - u[d] * dW[0]) * ir1;
    u1[d] = u[d] + du[d];
    un += u[d] * n[d];
    dun += du[d] * n[d];
  }
  u1n = un + dun;
  // d(rho |u|^2 / 2) = drho |u'|^2 / 2 + rho (u + u') . du / 2
  T u1sq = 0, sdu = 0;
#pragma unroll
  for (int d = 0; d < DIM; ++d) { u1sq += u1[d] * u1[d]; sdu += (u[d] + u1[d]) * du[d]; }
  ke_d = T(0.5) * dW[0] * u1sq + T(0.5) * rho * sdu;
  T q2 = 0;
#pragma unroll
  for (int d = 0; d < DIM; ++d) q2 += u[d] * u[d];
  const T p = (gamma - T(1)) * (W[DIM + 1] - T(0.5) * rho * q2);
  const T dp = (gamma - T(1)) * (dW[DIM + 1] - ke_d);
  dF[0] = dW[0] * u1n + rho * dun;  // d(rho u_n)
#pragma unroll
  for (int d = 0; d < DIM; ++d)
    dF[1 + d] = dW[0] * u1[d] * u1n + rho * (du[d] * u1n + u[d] * dun) + dp * n[d];
  dF[DIM + 1] = (dW[DIM + 1] + dp) * u1n + (W[DIM + 1] + p) * dun;
}

// spectral radius |u.n| + c at the arithmetic mean of two states
template <int DIM, typename T>
__device__ __forceinline__ T spectral_radius(T gamma, const T* Wa, const T* Wb, const T* n) {
  T m[DIM + 2];
#pragma unroll
  for (int i = 0; i < DIM + 2; ++i) m[i] = T(0.5) * (Wa[i] + Wb[i]);
  T ke = 0, un = 0;
#pragma unroll
  for (int d = 0; d < DIM; ++d) { ke += m[1 + d] * m[1 + d]; un += m[1 + d] * n[d]; }
  const T ir = T(1) / m[0];
  const T p = (gamma - T(1)) * (m[DIM + 1] - T(0.5) * ke * ir);
  return fabs(un * ir) + sqrt(gamma * p * ir);
}

// ---------------------------------------------------------------------------
// boundary ghosts, global frame
enum : int { kTagWall = 1, kTagFarfield = 2, kTagNoSlipWall = 3, kTagFarfieldRiemann = 4 };

template <int DIM, typename S = double>
__device__ __forceinline__ bool inflow(const S* winf, const S* n) {
  S un = S(0.0);
#pragma unroll
  for (int d = 0; d < DIM; ++d) un += winf[1 + d] * n[d];
  return un < S(0.0);
}
// Far-field state from the Riemann invariants along the outward normal n:
// R+ = u_n + 2c/(gamma-1) from the interior, R- = u_n - 2c/(gamma-1) from the
// free stream (each the invariant carried into the face by its characteristic);
// their sum and difference give u_n and c on the face, and the tangential
// velocity and the entropy p/rho^gamma come from upstream (the free stream on
// inflow, the interior on outflow).  Supersonic faces take the upwind state.
template <int DIM, typename S = double>
__device__ __forceinline__ void riemann_farfield(S gamma, const S* winf, const S* n, const S* W, S* Wb) {
  constexpr int NV = DIM + 2;
  const S gm1 = gamma - S(1.0);
  const S ri = S(1.0) / W[0], rf = S(1.0) / winf[0];
  S uni = S(0.0), unf = S(0.0), qi = S(0.0), qf = S(0.0);
#pragma unroll
  for (int d = 0; d < DIM; ++d) {
    uni += W[1 + d] * n[d];
    unf += winf[1 + d] * n[d];
    qi += W[1 + d] * W[1 + d];
    qf += winf[1 + d] * winf[1 + d];
  }
  uni *= ri;
  unf *= rf;
  const S pi = gm1 * (W[NV - 1] - S(0.5) * qi * ri), pf = gm1 * (winf[NV - 1] - S(0.5) * qf * rf);
  const S ci = sqrt(gamma * pi * ri), cf = sqrt(gamma * pf * rf);
  if (!(fabs(unf) < cf)) {  // supersonic normal flow
    const S* src = unf < S(0.0) ? winf : W;
#pragma unroll
    for (int i = 0; i < NV; ++i) Wb[i] = src[i];
    return;
  }
  const S rp = uni + S(2.0) * ci / gm1, rm = unf - S(2.0) * cf / gm1;
  const S un = S(0.5) * (rp + rm), cb = S(0.25) * gm1 * (rp - rm);
  const bool in = un < S(0.0);
  const S* up = in ? winf : W;
  const S ir = in ? rf : ri;
  const S ent = (in ? pf : pi) / pow(up[0], gamma);  // p / rho^gamma upstream
  const S rho = pow(cb * cb / (gamma * ent), S(1.0) / gm1);
  const S p = rho * cb * cb / gamma;
  S upn = S(0.0);
#pragma unroll
  for (int d = 0; d < DIM; ++d) upn += up[1 + d] * n[d];
  upn *= ir;
  S q = S(0.0);
  Wb[0] = rho;
#pragma unroll
  for (int d = 0; d < DIM; ++d) {
    const S u = up[1 + d] * ir + (un - upn) * n[d];  // upstream tangential part, face normal part
    Wb[1 + d] = rho * u;
    q += u * u;
  }
  Wb[NV - 1] = p / gm1 + S(0.5) * rho * q;
}

template <int DIM, typename S = double>
__device__ __forceinline__ void ghost_state(int tag, const S* winf, const S* n, const S* W, S* Wg, S gamma) {
  constexpr int NV = DIM + 2;
  if (tag == kTagFarfieldRiemann) {
    riemann_farfield<DIM, S>(gamma, winf, n, W, Wg);
  } else if (tag == kTagWall) {
    S mn = S(0.0);
#pragma unroll
    for (int d = 0; d < DIM; ++d) mn += W[1 + d] * n[d];
#pragma unroll
    for (int i = 0; i < NV; ++i) Wg[i] = W[i];
#pragma unroll
    for (int d = 0; d < DIM; ++d) Wg[1 + d] = W[1 + d] - S(2.0) * mn * n[d];
  } else if (tag == kTagNoSlipWall) {
    // no-slip adiabatic wall: every velocity component reversed, density and energy kept
#pragma unroll
    for (int i = 0; i < NV; ++i) Wg[i] = W[i];
#pragma unroll
    for (int d = 0; d < DIM; ++d) Wg[1 + d] = -W[1 + d];
  } else if (inflow<DIM, S>(winf, n)) {
#pragma unroll
    for (int i = 0; i < NV; ++i) Wg[i] = winf[i];
  } else {
#pragma unroll
    for (int i = 0; i < NV; ++i) Wg[i] = W[i];
  }
}
// gradient g[v][d] of the ghost field
template <int DIM, typename S = double>
__device__ __forceinline__ void ghost_grad(int tag, const S* winf, const S* n, const S (*g)[DIM],
                                           S (*gg)[DIM]) {
  constexpr int NV = DIM + 2;
  if (tag == kTagWall || tag == kTagNoSlipWall) {
    // mirror image q(H x), H = I - 2nn^T: scalars H grad;  momentum: slip
    // H (dm/dx) H (reflected), no-slip -(dm/dx) H (reversed)
    S t[NV][DIM];
#pragma unroll
    for (int v = 0; v < NV; ++v) {
      S s = S(0.0);
#pragma unroll
      for (int d = 0; d < DIM; ++d) s += g[v][d] * n[d];
#pragma unroll
      for (int d = 0; d < DIM; ++d) t[v][d] = g[v][d] - S(2.0) * s * n[d];
    }
    if (tag == kTagWall) {
#pragma unroll
      for (int d = 0; d < DIM; ++d) {
        S s = S(0.0);
#pragma unroll
        for (int e = 0; e < DIM; ++e) s += n[e] * t[1 + e][d];
#pragma unroll
        for (int e = 0; e < DIM; ++e) t[1 + e][d] -= S(2.0) * n[e] * s;
      }
    } else {
#pragma unroll
      for (int e = 0; e < DIM; ++e)
#pragma unroll
        for (int d = 0; d < DIM; ++d) t[1 + e][d] = -t[1 + e][d];
    }
#pragma unroll
    for (int v = 0; v < NV; ++v)
#pragma unroll
      for (int d = 0; d < DIM; ++d) gg[v][d] = t[v][d];
  } else if (tag == kTagFarfieldRiemann || inflow<DIM, S>(winf, n)) {
#pragma unroll
    for (int v = 0; v < NV; ++v)
#pragma unroll
      for (int d = 0; d < DIM; ++d) gg[v][d] = S(0.0);
  } else {
#pragma unroll
    for (int v = 0; v < NV; ++v)
#pragma unroll
      for (int d = 0; d < DIM; ++d) gg[v][d] = g[v][d];
  }
}

}  // namespace cgks
