/*
 * cgks_oracle.c -- plain, slow, FP64 CPU oracle of the GMG-CGKS V-cycle.
 *
 * TEST INFRASTRUCTURE ONLY.  Only the tests, the smoke check and the CPU
 * baseline leg of the benchmark load this library.  It shares no code with the
 * CUDA path: geometry, faces, colouring, reconstruction, the gas-kinetic flux,
 * KFVS, LU-SGS and the multigrid cycle are all written here from the paper
 * (arXiv 2509.06347) in its order and notation, without blocking or fusion.
 * Loops over independent cells and faces may run on OpenMP threads; every sum
 * over cells or faces is still formed serially in a fixed order, so results
 * are the same for any thread count.
 *
 * The gas-kinetic moments are taken the long way: the distribution function is
 * held as a polynomial in (u, v, w, xi^2) times a (half-)Maxwellian and every
 * moment is integrated term by term from the 1-D Maxwellian moment recursion.
 *
 * Paper sections followed:
 *   Sec 2.1  BGK model, Maxwellian, internal degrees of freedom K    (Eq. bgk)
 *   Sec 2.2  finite-volume residual with face Gauss quadrature
 *   Sec 2.3  gas-kinetic flux: Eqs. integral1, flux-3d-1/2, dis1, equli,
 *            compatibility2, dis2, co, co-moment
 *   Sec 2.4  direct evolution of cell-averaged slopes (divergence theorem)
 *   Sec 3.1  constrained least-squares quadratic p2 (Eqs. self-/neighbor-constrain)
 *   Sec 3.2  Green-Gauss sub-stencil p1;  Sec 3.3 discontinuity feedback (DF)
 *   Sec 4.1  colouring algorithm;  Sec 4.2-4.3 LU-SGS with DF relaxation
 *            (Eqs. gpu-forward-relaxation, gpu-backward-relaxation)
 *   Sec 5.1  coarse-cell volume and centre;  Sec 5.2 restriction, forcing term,
 *            prolongation (Eq. prolongation), three-level V-cycle
 * Readings where the paper is silent or garbled are marked "reading:".
 */
#include <math.h>
#include <stdint.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define MAXD 3
#define MAXV 5
#define MAXF 6   /* faces per cell (a hexahedron has 6) */
#define MAXG 4   /* Gauss points per face (4 on a quadrilateral) */
#define MAXK 9   /* quadratic basis size (3-D) */

/* ------------------------------------------------------------------------ */
/* configuration (flat double array, order fixed by the Python wrapper)      */
/* ------------------------------------------------------------------------ */
typedef struct {
  double gamma, cfl_imp, cfl_exp, tau_c1, tau_c2, weno_gh, weno_eps, r_safety;
  int n_sweep;            /* LU-SGS sweeps per coarse level */
  double winf[MAXV];      /* free stream (conservative) for far-field ghosts */
  double relax;           /* V-cycle LU-SGS relaxation factor: < 0 the DF of each cell
                             (Sec 4.3); otherwise this constant in place of DF (1: fully
                             implicit; in (0,1): the fixed-factor scheme of the remark) */
  int df_prolong;         /* 1: prolongation scaled by DF; 0: plain injection */
  int fine_smoother;      /* 0: DF-relaxed LU-SGS step; 1: explicit update (Eq. smo) */
  double mu;              /* dynamic viscosity: 0 Euler; > 0 Navier-Stokes, Pr = 1 */
  double slope_relax;     /* reading: pseudo-time slope update G <- G + w (DF Gnew - G); 1 replaces */
  double alpha_relax;     /* reading: a rise of the stored DF is under-relaxed by this factor;
                             a fall takes effect at once; 1 takes the product itself */
} OCfg;

static void cfg_from(const double* c, int nv, OCfg* o) {
  o->gamma = c[0]; o->cfl_imp = c[1]; o->cfl_exp = c[2]; o->tau_c1 = c[3];
  o->tau_c2 = c[4]; o->weno_gh = c[5]; o->weno_eps = c[6]; o->r_safety = c[7];
  o->n_sweep = (int)c[8];
  for (int v = 0; v < nv; ++v) o->winf[v] = c[9 + v];
  o->relax = c[9 + nv];
  o->df_prolong = (int)c[10 + nv];
  o->fine_smoother = (int)c[11 + nv];
  o->mu = c[12 + nv];
  o->slope_relax = c[13 + nv];
  o->alpha_relax = c[14 + nv];
}

/* ------------------------------------------------------------------------ */
/* mesh levels                                                               */
/* ------------------------------------------------------------------------ */
typedef struct {
  int n_cells, n_faces, n_bfaces;
  double* vol;     /* [n] */
  double* cen;     /* [n*dim] */
  double* mom2;    /* [n*dim*dim] central second moments divided by volume */
  /* faces: interior faces first then boundary faces */
  int* fL;         /* [nf] */
  int* fR;         /* [nf] right cell, or -1 for boundary */
  int* ftag;       /* [nf] boundary tag (0 for interior) */
  double* fn;      /* [nf*dim] unit normal from L to R (outward for boundary) */
  double* fS;      /* [nf] area */
  double* fshift;  /* [nf*dim] x_in_L_frame = x_in_R_frame + shift */
  double* fgp;     /* [nf*MAXG*dim] Gauss points in L's frame (fine level only) */
  /* mixed-element meshes only (NULL on simplex meshes, where every face has
     M->ngp points of equal weight and fgp[0] lies on the face plane): */
  int* fngp;       /* [nf] Gauss points of the face (3 triangle, 4 quadrilateral) */
  double* fgw;     /* [nf*MAXG] their weights, summing to 1 */
  double* fpt;     /* [nf*dim] the face's node mean, the point the ghost mirror plane passes through */
  /* cell -> faces in stored order; sign +1 if the cell is L */
  int* cnf;        /* [n] number of faces */
  int* cface;      /* [n*maxnf] */
  int* cside;      /* [n*maxnf] */
  int maxnf;
  int* parent;     /* [n] parent in the next level (NULL on the coarsest) */
  int* color;      /* [n] colours 1..nc */
  int n_colors;
} OLevel;

typedef struct {
  int dim, nv, ngp, nlev;
  OLevel lev[8];
} OMesh;

/* ------------------------------------------------------------------------ */
/* small dense linear algebra                                                */
/* ------------------------------------------------------------------------ */
/* Solve A x = B (n x n, nrhs columns, row-major, in place) by Gaussian
 * elimination with partial pivoting.  Returns 0, or -1 if a pivot falls below
 * tol * (largest |A_ij|). */
static int gauss_solve(double* A, double* B, int n, int nrhs, double tol) {
  double amax = 0.0;
  for (int i = 0; i < n * n; ++i) if (fabs(A[i]) > amax) amax = fabs(A[i]);
  for (int k = 0; k < n; ++k) {
    int p = k;
    for (int i = k + 1; i < n; ++i) if (fabs(A[i * n + k]) > fabs(A[p * n + k])) p = i;
    if (!(fabs(A[p * n + k]) > tol * amax)) return -1;
    if (p != k) {
      for (int j = 0; j < n; ++j) { double t = A[k * n + j]; A[k * n + j] = A[p * n + j]; A[p * n + j] = t; }
      for (int j = 0; j < nrhs; ++j) { double t = B[k * nrhs + j]; B[k * nrhs + j] = B[p * nrhs + j]; B[p * nrhs + j] = t; }
    }
    for (int i = k + 1; i < n; ++i) {
      double f = A[i * n + k] / A[k * n + k];
      if (f == 0.0) continue;
      for (int j = k; j < n; ++j) A[i * n + j] -= f * A[k * n + j];
      for (int j = 0; j < nrhs; ++j) B[i * nrhs + j] -= f * B[k * nrhs + j];
    }
  }
  for (int k = n - 1; k >= 0; --k) {
    for (int j = 0; j < nrhs; ++j) {
      double s = B[k * nrhs + j];
      for (int i = k + 1; i < n; ++i) s -= A[k * n + i] * B[i * nrhs + j];
      B[k * nrhs + j] = s / A[k * n + k];
    }
  }
  return 0;
}

/* ------------------------------------------------------------------------ */
/* Maxwellian moments (Sec 2.1, Eq. co-moment)                               */
/* g = rho (lambda/pi)^((D+K)/2) exp(-lambda(|u-U|^2 + xi^2))                */
/* ------------------------------------------------------------------------ */
#define MU 8
typedef struct {
  double rho, lam, U[MAXD];
  double mu[MU];        /* <u^n> over the chosen half (or full) space in u   */
  double mv[MU], mw[MU];/* <v^n>, <w^n> full space                           */
  double mxi[3];        /* <(xi^2)^n>, n = 0, 1, 2                           */
} Maxw;

/* half: 0 full space, +1 u > 0, -1 u < 0 (u = first local velocity) */
static void maxw_init(Maxw* g, int dim, double K, const double* prim, int half) {
  /* prim = rho, U[dim], lambda */
  g->rho = prim[0];
  for (int d = 0; d < MAXD; ++d) g->U[d] = d < dim ? prim[1 + d] : 0.0;
  g->lam = prim[1 + dim];
  double lam = g->lam, U = g->U[0];
  if (half == 0) { g->mu[0] = 1.0; g->mu[1] = U; }
  else {
    double sl = sqrt(lam);
    double ex = exp(-lam * U * U) / (2.0 * sqrt(M_PI * lam));
    if (half > 0) { g->mu[0] = 0.5 * erfc(-sl * U); g->mu[1] = U * g->mu[0] + ex; }
    else          { g->mu[0] = 0.5 * erfc(sl * U);  g->mu[1] = U * g->mu[0] - ex; }
  }
  for (int n = 0; n + 2 < MU; ++n) g->mu[n + 2] = U * g->mu[n + 1] + (n + 1) / (2.0 * lam) * g->mu[n];
  double V = g->U[1], W = g->U[2];
  g->mv[0] = 1.0; g->mv[1] = V; g->mw[0] = 1.0; g->mw[1] = W;
  for (int n = 0; n + 2 < MU; ++n) {
    g->mv[n + 2] = V * g->mv[n + 1] + (n + 1) / (2.0 * lam) * g->mv[n];
    g->mw[n + 2] = W * g->mw[n + 1] + (n + 1) / (2.0 * lam) * g->mw[n];
  }
  g->mxi[0] = 1.0;
  g->mxi[1] = K / (2.0 * lam);
  g->mxi[2] = (K * K + 2.0 * K) / (4.0 * lam * lam);
}

/* sparse polynomial in (u, v, w, xi^2) */
#define MAXT 96
typedef struct { int n; unsigned char e[MAXT][4]; double c[MAXT]; } Poly;

static void poly_zero(Poly* p) { p->n = 0; }
static void poly_term(Poly* p, int eu, int ev, int ew, int ex, double c) {
  if (c == 0.0) return;
  for (int i = 0; i < p->n; ++i)
    if (p->e[i][0] == eu && p->e[i][1] == ev && p->e[i][2] == ew && p->e[i][3] == ex) { p->c[i] += c; return; }
  if (p->n >= MAXT) { fprintf(stderr, "oracle: polynomial overflow\n"); abort(); }
  p->e[p->n][0] = (unsigned char)eu; p->e[p->n][1] = (unsigned char)ev;
  p->e[p->n][2] = (unsigned char)ew; p->e[p->n][3] = (unsigned char)ex;
  p->c[p->n] = c; p->n++;
}
static void poly_axpy(Poly* y, double a, const Poly* x) {
  for (int i = 0; i < x->n; ++i) poly_term(y, x->e[i][0], x->e[i][1], x->e[i][2], x->e[i][3], a * x->c[i]);
}
static void poly_mul(Poly* out, const Poly* a, const Poly* b) {
  poly_zero(out);
  for (int i = 0; i < a->n; ++i)
    for (int j = 0; j < b->n; ++j)
      poly_term(out, a->e[i][0] + b->e[j][0], a->e[i][1] + b->e[j][1], a->e[i][2] + b->e[j][2],
                a->e[i][3] + b->e[j][3], a->c[i] * b->c[j]);
}
/* psi_i: 1, u, v, (w), 1/2 (u^2 + v^2 + w^2 + xi^2) */
static void poly_psi(Poly* p, int dim, int i) {
  poly_zero(p);
  if (i == 0) poly_term(p, 0, 0, 0, 0, 1.0);
  else if (i <= dim) poly_term(p, i == 1, i == 2, i == 3, 0, 1.0);
  else {
    poly_term(p, 2, 0, 0, 0, 0.5);
    poly_term(p, 0, 2, 0, 0, 0.5);
    if (dim == 3) poly_term(p, 0, 0, 2, 0, 0.5);
    poly_term(p, 0, 0, 0, 1, 0.5);
  }
}
/* a . psi for a coefficient vector a[nv] */
static void poly_lin(Poly* p, int dim, const double* a) {
  Poly t; poly_zero(p);
  for (int i = 0; i < dim + 2; ++i) { poly_psi(&t, dim, i); poly_axpy(p, a[i], &t); }
}
/* velocity component u_d (d = 0 normal, 1, 2 tangential) */
static void poly_vel(Poly* p, int d) { poly_zero(p); poly_term(p, d == 0, d == 1, d == 2, 0, 1.0); }

static double mono_mom(const Maxw* g, const unsigned char* e) {
  return g->rho * g->mu[e[0]] * g->mv[e[1]] * g->mw[e[2]] * g->mxi[e[3]];
}
static double poly_mom(const Maxw* g, const Poly* p) {
  double s = 0.0;
  for (int i = 0; i < p->n; ++i) s += p->c[i] * mono_mom(g, p->e[i]);
  return s;
}
/* integral of (extra * P) g over the Maxwellian's space, extra a polynomial */
static double poly_mom2(const Maxw* g, const Poly* extra, const Poly* P) {
  Poly t; poly_mul(&t, extra, P);
  return poly_mom(g, &t);
}

/* ------------------------------------------------------------------------ */
/* primitive / conservative conversions (Sec 2.1)                            */
/* ------------------------------------------------------------------------ */
static double K_of(int dim, double gamma) {
  /* reading: K = (4-2g)/(g-1) in 2-D (the paper states the 3-D formula only) */
  return dim == 2 ? (4.0 - 2.0 * gamma) / (gamma - 1.0) : (5.0 - 3.0 * gamma) / (gamma - 1.0);
}
static double pressure(int dim, double gamma, const double* W) {
  double ke = 0.0;
  for (int d = 0; d < dim; ++d) ke += W[1 + d] * W[1 + d];
  return (gamma - 1.0) * (W[dim + 1] - 0.5 * ke / W[0]);
}
/* prim = rho, U, lambda  with lambda = rho / (2 p) */
static void to_prim(int dim, double gamma, const double* W, double* prim) {
  prim[0] = W[0];
  for (int d = 0; d < dim; ++d) prim[1 + d] = W[1 + d] / W[0];
  prim[1 + dim] = W[0] / (2.0 * pressure(dim, gamma, W));
}

/* moment matrix M_ij = int psi_i psi_j g and the solve M a = b (Eq. co) */
static void solve_slope(const Maxw* g, int dim, const double* b, double* a) {
  int nv = dim + 2;
  double M[MAXV * MAXV], B[MAXV];
  Poly pi, pj;
  for (int i = 0; i < nv; ++i) {
    poly_psi(&pi, dim, i);
    for (int j = 0; j < nv; ++j) { poly_psi(&pj, dim, j); M[i * nv + j] = poly_mom2(g, &pi, &pj); }
    B[i] = b[i];
  }
  if (gauss_solve(M, B, nv, 1, 1e-300) != 0) { fprintf(stderr, "oracle: singular moment matrix\n"); abort(); }
  for (int i = 0; i < nv; ++i) a[i] = B[i];
}

static void kfvs_point(int dim, double gamma, const double* Wl, const double* Wr, double* F);

/* ------------------------------------------------------------------------ */
/* gas-kinetic interface flux at one Gauss point, local frame (Sec 2.3)      */
/* ------------------------------------------------------------------------ */
typedef struct {
  double al[MAXD][MAXV], Al[MAXV], ar[MAXD][MAXV], Ar[MAXV];
  double Wc[MAXV], ac[MAXD][MAXV], Ac[MAXV], tau;
} GksDebug;

/* Wl, Wr: conservative states (rho, rho u_n, rho u_t1, [rho u_t2], rho E);
 * dWl, dWr: derivatives [dim][nv] along (n, t1, t2);  dt: flux time step.
 * Outputs: Fbar (time-averaged flux over [0, dt]), Wt (point value at t = dt). */
static void gks_point(int dim, double gamma, double c1, double c2, double mu, const double* Wl,
                      const double* dWl, const double* Wr, const double* dWr, double dt,
                      double* Fbar, double* Wt, GksDebug* dbg) {
  int nv = dim + 2;
  double K = K_of(dim, gamma);
  double pl[MAXV], pr[MAXV];
  to_prim(dim, gamma, Wl, pl);
  to_prim(dim, gamma, Wr, pr);
  Maxw gl, gr, glp, grm;
  maxw_init(&gl, dim, K, pl, 0);
  maxw_init(&gr, dim, K, pr, 0);
  maxw_init(&glp, dim, K, pl, +1);
  maxw_init(&grm, dim, K, pr, -1);
  Poly psi[MAXV], ud[MAXD], t, t2;
  for (int i = 0; i < nv; ++i) poly_psi(&psi[i], dim, i);
  for (int d = 0; d < dim; ++d) poly_vel(&ud[d], d);

  /* slopes of the initial states: <a_{x_d}> = dW/dx_d (Eq. co) */
  double al[MAXD][MAXV], ar[MAXD][MAXV], Al[MAXV], Ar[MAXV];
  for (int d = 0; d < dim; ++d) {
    solve_slope(&gl, dim, dWl + d * nv, al[d]);
    solve_slope(&gr, dim, dWr + d * nv, ar[d]);
  }
  /* a.u = sum_d (a_d . psi) u_d as polynomials */
  Poly aul, aur, auc;
  poly_zero(&aul); poly_zero(&aur);
  for (int d = 0; d < dim; ++d) {
    poly_lin(&t, dim, al[d]); poly_mul(&t2, &t, &ud[d]); poly_axpy(&aul, 1.0, &t2);
    poly_lin(&t, dim, ar[d]); poly_mul(&t2, &t, &ud[d]); poly_axpy(&aur, 1.0, &t2);
  }
  /* time derivative: <A + a.u> = 0 */
  double bl[MAXV], br[MAXV];
  for (int i = 0; i < nv; ++i) { bl[i] = -poly_mom2(&gl, &psi[i], &aul); br[i] = -poly_mom2(&gr, &psi[i], &aur); }
  solve_slope(&gl, dim, bl, Al);
  solve_slope(&gr, dim, br, Ar);

  /* equilibrium state at the interface from half-space moments (Eq. compatibility2) */
  double Wc[MAXV], pc[MAXV];
  for (int i = 0; i < nv; ++i) Wc[i] = poly_mom(&glp, &psi[i]) + poly_mom(&grm, &psi[i]);
  const double p_eq = pressure(dim, gamma, Wc);
  {
    /* reading (vacuum, not treated by the paper): when both sides move apart so
     * fast that the half-space moments give no admissible equilibrium, the
     * point takes the collisionless limit: KFVS flux, point value W^c */
    double pwl = pressure(dim, gamma, Wl), pwr = pressure(dim, gamma, Wr);
    double pwc = pressure(dim, gamma, Wc);
    if (!(Wc[0] > 1e-10 * (Wl[0] + Wr[0])) || !(pwc > 1e-10 * (pwl + pwr))) {
      kfvs_point(dim, gamma, Wl, Wr, Fbar);
      for (int i = 0; i < nv; ++i) Wt[i] = Wc[i];
      if (dbg) memset(dbg, 0, sizeof(*dbg));
      return;
    }
  }
  to_prim(dim, gamma, Wc, pc);
  Maxw gc;
  maxw_init(&gc, dim, K, pc, 0);
  /* reading: derivatives of the interface equilibrium = mean of both sides */
  double ac[MAXD][MAXV], Ac[MAXV], bc[MAXV];
  for (int d = 0; d < dim; ++d) {
    double dc[MAXV];
    for (int i = 0; i < nv; ++i) dc[i] = 0.5 * (dWl[d * nv + i] + dWr[d * nv + i]);
    solve_slope(&gc, dim, dc, ac[d]);
  }
  poly_zero(&auc);
  for (int d = 0; d < dim; ++d) { poly_lin(&t, dim, ac[d]); poly_mul(&t2, &t, &ud[d]); poly_axpy(&auc, 1.0, &t2); }
  for (int i = 0; i < nv; ++i) bc[i] = -poly_mom2(&gc, &psi[i], &auc);
  solve_slope(&gc, dim, bc, Ac);

  /* reading: numerical collision time C1 dt + C2 |dp| / (pl + pr) dt for the
   * Euler equations; for the Navier-Stokes equations (Sec 2.1: tau = mu / p,
   * Pr = 1) mu / p of the interface equilibrium replaces C1 dt */
  double pL = 1.0 / (2.0 * pl[1 + dim]) * pl[0], pR = 1.0 / (2.0 * pr[1 + dim]) * pr[0];
  double tau = (mu > 0.0 ? mu / p_eq : c1 * dt) + c2 * fabs(pL - pR) / (pL + pR) * dt;

  Poly Alp, Arp, Acp;
  poly_lin(&Alp, dim, Al);
  poly_lin(&Arp, dim, Ar);
  poly_lin(&Acp, dim, Ac);

  /* time integrals over [0, dt] of the coefficients of Eqs. dis1 and dis2 */
  double e = exp(-dt / tau);
  double T1 = dt - tau * (1.0 - e);                                    /* int C1 */
  double T2 = -tau * dt + 2.0 * tau * tau - tau * (dt + 2.0 * tau) * e;  /* int C2 */
  double T3 = 0.5 * dt * dt - tau * dt + tau * tau * (1.0 - e);         /* int C3 */
  double T4 = tau * (1.0 - e);                                         /* int e^{-t/tau} */
  double T5 = tau * tau - tau * (dt + tau) * e;                        /* int t e^{-t/tau} */

  /* time-integrated distribution: polynomial factors per Maxwellian */
  Poly Pc, Pl, Pr;
  poly_zero(&Pc);
  poly_term(&Pc, 0, 0, 0, 0, T1);
  poly_axpy(&Pc, T2, &auc);
  poly_axpy(&Pc, T3, &Acp);
  poly_zero(&Pl);
  poly_term(&Pl, 0, 0, 0, 0, T4);
  poly_axpy(&Pl, -tau * T4 - T5, &aul);
  poly_axpy(&Pl, -tau * T4, &Alp);
  poly_zero(&Pr);
  poly_term(&Pr, 0, 0, 0, 0, T4);
  poly_axpy(&Pr, -tau * T4 - T5, &aur);
  poly_axpy(&Pr, -tau * T4, &Arp);
  for (int i = 0; i < nv; ++i) {
    Poly upsi;
    poly_mul(&upsi, &ud[0], &psi[i]);
    double F = poly_mom2(&gc, &upsi, &Pc) + poly_mom2(&glp, &upsi, &Pl) + poly_mom2(&grm, &upsi, &Pr);
    Fbar[i] = F / dt;
  }
  /* point value at t = dt (Eq. point with f from Eqs. dis1 + dis2) */
  double C1 = 1.0 - e, C2 = (dt + tau) * e - tau, C3 = dt - tau + tau * e;
  poly_zero(&Pc);
  poly_term(&Pc, 0, 0, 0, 0, C1);
  poly_axpy(&Pc, C2, &auc);
  poly_axpy(&Pc, C3, &Acp);
  poly_zero(&Pl);
  poly_term(&Pl, 0, 0, 0, 0, e);
  poly_axpy(&Pl, -e * (tau + dt), &aul);
  poly_axpy(&Pl, -e * tau, &Alp);
  poly_zero(&Pr);
  poly_term(&Pr, 0, 0, 0, 0, e);
  poly_axpy(&Pr, -e * (tau + dt), &aur);
  poly_axpy(&Pr, -e * tau, &Arp);
  for (int i = 0; i < nv; ++i)
    Wt[i] = poly_mom2(&gc, &psi[i], &Pc) + poly_mom2(&glp, &psi[i], &Pl) + poly_mom2(&grm, &psi[i], &Pr);

  if (dbg) {
    for (int d = 0; d < MAXD; ++d)
      for (int i = 0; i < MAXV; ++i) {
        dbg->al[d][i] = (d < dim && i < nv) ? al[d][i] : 0.0;
        dbg->ar[d][i] = (d < dim && i < nv) ? ar[d][i] : 0.0;
        dbg->ac[d][i] = (d < dim && i < nv) ? ac[d][i] : 0.0;
      }
    for (int i = 0; i < MAXV; ++i) {
      dbg->Al[i] = i < nv ? Al[i] : 0.0; dbg->Ar[i] = i < nv ? Ar[i] : 0.0;
      dbg->Ac[i] = i < nv ? Ac[i] : 0.0; dbg->Wc[i] = i < nv ? Wc[i] : 0.0;
    }
    dbg->tau = tau;
  }
}

/* first-order KFVS flux, local frame (Sec 5.2; reading: collisionless split) */
static void kfvs_point(int dim, double gamma, const double* Wl, const double* Wr, double* F) {
  int nv = dim + 2;
  double K = K_of(dim, gamma);
  double pl[MAXV], pr[MAXV];
  to_prim(dim, gamma, Wl, pl);
  to_prim(dim, gamma, Wr, pr);
  Maxw glp, grm;
  maxw_init(&glp, dim, K, pl, +1);
  maxw_init(&grm, dim, K, pr, -1);
  Poly psi, u, up;
  poly_vel(&u, 0);
  for (int i = 0; i < nv; ++i) {
    poly_psi(&psi, dim, i);
    poly_mul(&up, &u, &psi);
    F[i] = poly_mom(&glp, &up) + poly_mom(&grm, &up);
  }
}

/* discontinuity feedback at a Gauss point (Sec 3.3), local frame */
static double df_point(int dim, double gamma, const double* Wl, const double* Wr) {
  double pl = pressure(dim, gamma, Wl), pr = pressure(dim, gamma, Wr);
  double cl = sqrt(gamma * pl / Wl[0]), cr = sqrt(gamma * pr / Wr[0]);
  double D = fabs(pl - pr) / pl + fabs(pl - pr) / pr;
  double dn = Wl[1] / Wl[0] / cl - Wr[1] / Wr[0] / cr;
  D += dn * dn;
  for (int d = 1; d < dim; ++d) {
    double dt = Wl[1 + d] / Wl[0] / cl - Wr[1 + d] / Wr[0] / cr;
    D += dt * dt;  /* reading: squared norm of the tangential Mach difference */
  }
  return 1.0 / (1.0 + D * D);
}

/* Euler flux T(W).n in the global frame (Sec 4.2) */
static void euler_flux(int dim, double gamma, const double* W, const double* n, double* T) {
  double p = pressure(dim, gamma, W);
  double un = 0.0;
  for (int d = 0; d < dim; ++d) un += W[1 + d] / W[0] * n[d];
  T[0] = W[0] * un;
  for (int d = 0; d < dim; ++d) T[1 + d] = W[1 + d] * un + p * n[d];
  T[dim + 1] = (W[dim + 1] + p) * un;
}

/* ------------------------------------------------------------------------ */
/* local frames                                                              */
/* ------------------------------------------------------------------------ */
static void frame(int dim, const double* n, double* R /* rows n, t1, t2 */) {
  if (dim == 2) { R[0] = n[0]; R[1] = n[1]; R[2] = -n[1]; R[3] = n[0]; return; }
  int a = 0;
  if (fabs(n[1]) < fabs(n[a])) a = 1;
  if (fabs(n[2]) < fabs(n[a])) a = 2;
  double e[3] = {0, 0, 0};
  e[a] = 1.0;
  double t1[3] = {n[1] * e[2] - n[2] * e[1], n[2] * e[0] - n[0] * e[2], n[0] * e[1] - n[1] * e[0]};
  double l = sqrt(t1[0] * t1[0] + t1[1] * t1[1] + t1[2] * t1[2]);
  for (int i = 0; i < 3; ++i) t1[i] /= l;
  double t2[3] = {n[1] * t1[2] - n[2] * t1[1], n[2] * t1[0] - n[0] * t1[2], n[0] * t1[1] - n[1] * t1[0]};
  for (int i = 0; i < 3; ++i) { R[i] = n[i]; R[3 + i] = t1[i]; R[6 + i] = t2[i]; }
}
/* rotate conservative vector to local frame (Wloc[1+a] = sum_d R[a][d] W[1+d]) */
static void rot_to(int dim, const double* R, const double* W, double* Wl) {
  Wl[0] = W[0];
  for (int a = 0; a < dim; ++a) { double s = 0; for (int d = 0; d < dim; ++d) s += R[a * dim + d] * W[1 + d]; Wl[1 + a] = s; }
  Wl[dim + 1] = W[dim + 1];
}
static void rot_from(int dim, const double* R, const double* Wl, double* W) {
  W[0] = Wl[0];
  for (int d = 0; d < dim; ++d) { double s = 0; for (int a = 0; a < dim; ++a) s += R[a * dim + d] * Wl[1 + a]; W[1 + d] = s; }
  W[dim + 1] = Wl[dim + 1];
}
/* gradient G[d][v] (global) -> local derivatives along frame directions with
 * rotated momentum components: Gl[a][v'] */
static void rot_grad(int dim, const double* R, const double* G, double* Gl) {
  int nv = dim + 2;
  double tmp[MAXD * MAXV];
  for (int a = 0; a < dim; ++a)
    for (int v = 0; v < nv; ++v) {
      double s = 0; for (int d = 0; d < dim; ++d) s += R[a * dim + d] * G[d * nv + v];
      tmp[a * nv + v] = s;
    }
  for (int a = 0; a < dim; ++a) rot_to(dim, R, tmp + a * nv, Gl + a * nv);
}

/* ------------------------------------------------------------------------ */
/* geometry (Sec 2.2, Sec 5.1)                                               */
/* ------------------------------------------------------------------------ */
static double simplex_geom(int dim, const double* x, double* cen, double* m2) {
  int nvert = dim + 1;
  for (int d = 0; d < dim; ++d) { cen[d] = 0; for (int v = 0; v < nvert; ++v) cen[d] += x[v * dim + d]; cen[d] /= nvert; }
  double vol;
  if (dim == 2) {
    double ax = x[2] - x[0], ay = x[3] - x[1], bx = x[4] - x[0], by = x[5] - x[1];
    vol = 0.5 * fabs(ax * by - ay * bx);
  } else {
    double a[3], b[3], c[3];
    for (int d = 0; d < 3; ++d) { a[d] = x[3 + d] - x[d]; b[d] = x[6 + d] - x[d]; c[d] = x[9 + d] - x[d]; }
    double det = a[0] * (b[1] * c[2] - b[2] * c[1]) - a[1] * (b[0] * c[2] - b[2] * c[0]) + a[2] * (b[0] * c[1] - b[1] * c[0]);
    vol = fabs(det) / 6.0;
  }
  /* second central moment of a simplex: sum_v (x_v - c)(x_v - c)^T / ((n+1)(n+2)) */
  for (int d = 0; d < dim; ++d)
    for (int e = 0; e < dim; ++e) {
      double s = 0;
      for (int v = 0; v < nvert; ++v) s += (x[v * dim + d] - cen[d]) * (x[v * dim + e] - cen[e]);
      m2[d * dim + e] = s / ((dim + 1) * (dim + 2));
    }
  return vol;
}

typedef struct { int key[3]; int cell, k; } FKey;
static int fkey_cmp(const void* a, const void* b) {
  const FKey* x = (const FKey*)a; const FKey* y = (const FKey*)b;
  for (int i = 0; i < 3; ++i) { if (x->key[i] != y->key[i]) return x->key[i] < y->key[i] ? -1 : 1; }
  if (x->cell != y->cell) return x->cell < y->cell ? -1 : 1;
  return x->k - y->k;
}
static void sort_key(int n, int* k) {
  for (int i = 0; i < n; ++i) for (int j = i + 1; j < n; ++j) if (k[j] < k[i]) { int t = k[i]; k[i] = k[j]; k[j] = t; }
}

static void level_alloc_cells(OLevel* L, int n, int dim, int maxnf) {
  L->n_cells = n; L->maxnf = maxnf;
  L->vol = calloc(n, sizeof(double)); L->cen = calloc((size_t)n * dim, sizeof(double));
  L->mom2 = calloc((size_t)n * dim * dim, sizeof(double));
  L->cnf = calloc(n, sizeof(int)); L->cface = calloc((size_t)n * maxnf, sizeof(int));
  L->cside = calloc((size_t)n * maxnf, sizeof(int));
  L->color = calloc(n, sizeof(int));
  L->parent = NULL;
}
static void level_alloc_faces(OLevel* L, int nf, int dim, int with_gp) {
  L->n_faces = nf;
  L->fL = calloc(nf, sizeof(int)); L->fR = calloc(nf, sizeof(int)); L->ftag = calloc(nf, sizeof(int));
  L->fn = calloc((size_t)nf * dim, sizeof(double)); L->fS = calloc(nf, sizeof(double));
  L->fshift = calloc((size_t)nf * dim, sizeof(double));
  L->fgp = with_gp ? calloc((size_t)nf * MAXG * dim, sizeof(double)) : NULL;
  L->fngp = NULL; L->fgw = NULL; L->fpt = NULL;
}

/* Build the fine level from simplices.  Face k of a cell is the face opposite
 * its k-th vertex (the stored face order).  Returns 0 or a negative code. */
static int build_fine(OMesh* M, int dim, int n, const int* cn, const double* cx, int nbf,
                      const int* bfn, const int* bft, char* err) {
  int nvert = dim + 1, nf_c = dim + 1;
  M->dim = dim; M->nv = dim + 2; M->ngp = dim == 2 ? 2 : 3; M->nlev = 1;
  OLevel* L = &M->lev[0];
  level_alloc_cells(L, n, dim, nf_c);
  for (int c = 0; c < n; ++c) L->vol[c] = simplex_geom(dim, cx + (size_t)c * nvert * dim, L->cen + (size_t)c * dim, L->mom2 + (size_t)c * dim * dim);
  size_t ns = (size_t)n * nf_c;
  FKey* keys = malloc(ns * sizeof(FKey));
  for (int c = 0; c < n; ++c)
    for (int k = 0; k < nf_c; ++k) {
      FKey* f = &keys[(size_t)c * nf_c + k];
      int m = 0; f->key[2] = -1;
      for (int v = 0; v < nvert; ++v) if (v != k) f->key[m++] = cn[(size_t)c * nvert + v];
      sort_key(dim, f->key);
      f->cell = c; f->k = k;
    }
  qsort(keys, ns, sizeof(FKey), fkey_cmp);
  FKey* bk = malloc((size_t)(nbf > 0 ? nbf : 1) * sizeof(FKey));
  for (int b = 0; b < nbf; ++b) {
    bk[b].key[2] = -1;
    for (int v = 0; v < dim; ++v) bk[b].key[v] = bfn[(size_t)b * dim + v];
    sort_key(dim, bk[b].key);
    bk[b].cell = b; bk[b].k = 0;
  }
  qsort(bk, nbf, sizeof(FKey), fkey_cmp);
  /* count */
  int n_int = 0, n_bnd = 0;
  for (size_t i = 0; i < ns;) {
    size_t j = i + 1;
    while (j < ns && memcmp(keys[j].key, keys[i].key, sizeof(keys[i].key)) == 0) ++j;
    if (j - i == 2) n_int++;
    else if (j - i == 1) n_bnd++;
    else { snprintf(err, 256, "face shared by %d cells", (int)(j - i)); free(keys); free(bk); return -3; }
    i = j;
  }
  if (n_bnd != nbf) { snprintf(err, 256, "%d open faces but %d boundary faces given", n_bnd, nbf); free(keys); free(bk); return -3; }
  level_alloc_faces(L, n_int + n_bnd, dim, 1);
  L->n_bfaces = n_bnd;
  int fi = 0, fb = n_int;
  for (size_t i = 0; i < ns;) {
    size_t j = i + 1;
    while (j < ns && memcmp(keys[j].key, keys[i].key, sizeof(keys[i].key)) == 0) ++j;
    int f;
    if (j - i == 2) {
      f = fi++;
      L->fL[f] = keys[i].cell; L->fR[f] = keys[i + 1].cell; L->ftag[f] = 0;
      L->cface[keys[i].cell * nf_c + keys[i].k] = f; L->cside[keys[i].cell * nf_c + keys[i].k] = +1;
      L->cface[keys[i + 1].cell * nf_c + keys[i + 1].k] = f; L->cside[keys[i + 1].cell * nf_c + keys[i + 1].k] = -1;
    } else {
      FKey q = keys[i]; q.cell = -1; q.k = 0;
      int lo = 0, hi = nbf - 1, found = -1;
      while (lo <= hi) {
        int mid = (lo + hi) / 2;
        int c = memcmp(bk[mid].key, q.key, sizeof(q.key));
        int cmp = 0;
        for (int t = 0; t < 3; ++t) if (bk[mid].key[t] != q.key[t]) { cmp = bk[mid].key[t] < q.key[t] ? -1 : 1; break; }
        (void)c;
        if (cmp == 0) { found = mid; break; }
        if (cmp < 0) lo = mid + 1; else hi = mid - 1;
      }
      if (found < 0) { snprintf(err, 256, "open face of cell %d not in the boundary list", keys[i].cell); free(keys); free(bk); return -3; }
      f = fb++;
      L->fL[f] = keys[i].cell; L->fR[f] = -1; L->ftag[f] = bft[bk[found].cell];
      L->cface[keys[i].cell * nf_c + keys[i].k] = f; L->cside[keys[i].cell * nf_c + keys[i].k] = +1;
    }
    /* geometry from L's vertex coordinates; shift from R's copy of the same face */
    int cl = L->fL[f], kl = keys[i].k, cr = L->fR[f], kr = cr >= 0 ? keys[i + 1].k : -1;
    double fv[MAXD][MAXD], fc[MAXD] = {0, 0, 0};
    int m = 0;
    for (int v = 0; v < nvert; ++v) if (v != kl) { for (int d = 0; d < dim; ++d) fv[m][d] = cx[((size_t)cl * nvert + v) * dim + d]; ++m; }
    for (int v = 0; v < dim; ++v) for (int d = 0; d < dim; ++d) fc[d] += fv[v][d] / dim;
    double nrm[3], S;
    if (dim == 2) {
      double ex = fv[1][0] - fv[0][0], ey = fv[1][1] - fv[0][1];
      S = sqrt(ex * ex + ey * ey); nrm[0] = ey / S; nrm[1] = -ex / S;
    } else {
      double a[3], b[3];
      for (int d = 0; d < 3; ++d) { a[d] = fv[1][d] - fv[0][d]; b[d] = fv[2][d] - fv[0][d]; }
      double cr3[3] = {a[1] * b[2] - a[2] * b[1], a[2] * b[0] - a[0] * b[2], a[0] * b[1] - a[1] * b[0]};
      double l = sqrt(cr3[0] * cr3[0] + cr3[1] * cr3[1] + cr3[2] * cr3[2]);
      S = 0.5 * l; for (int d = 0; d < 3; ++d) nrm[d] = cr3[d] / l;
    }
    double dot = 0; for (int d = 0; d < dim; ++d) dot += (fc[d] - L->cen[cl * dim + d]) * nrm[d];
    if (dot < 0) for (int d = 0; d < dim; ++d) nrm[d] = -nrm[d];
    for (int d = 0; d < dim; ++d) L->fn[f * dim + d] = nrm[d];
    L->fS[f] = S;
    if (cr >= 0) {
      double fcr[MAXD] = {0, 0, 0};
      for (int v = 0; v < nvert; ++v) if (v != kr) for (int d = 0; d < dim; ++d) fcr[d] += cx[((size_t)cr * nvert + v) * dim + d] / dim;
      for (int d = 0; d < dim; ++d) L->fshift[f * dim + d] = fc[d] - fcr[d];
    }
    /* Gauss points: reading: 2-point Gauss-Legendre per 2-D edge; 3-point
     * degree-2 rule (barycentric 2/3, 1/6, 1/6) per triangle (Sec 2.2) */
    if (dim == 2) {
      double s = 0.5 / sqrt(3.0);
      for (int d = 0; d < 2; ++d) {
        L->fgp[(f * MAXG + 0) * dim + d] = fc[d] - s * (fv[1][d] - fv[0][d]);
        L->fgp[(f * MAXG + 1) * dim + d] = fc[d] + s * (fv[1][d] - fv[0][d]);
      }
    } else {
      for (int g = 0; g < 3; ++g)
        for (int d = 0; d < 3; ++d) {
          double s = 0;
          for (int v = 0; v < 3; ++v) s += (v == g ? 2.0 / 3.0 : 1.0 / 6.0) * fv[v][d];
          L->fgp[(f * MAXG + g) * dim + d] = s;
        }
    }
    i = j;
  }
  for (int c = 0; c < n; ++c) L->cnf[c] = nf_c;
  free(keys); free(bk);
  return 0;
}

/* ------------------------------------------------------------------------ */
/* mixed-element fine level (tetrahedra, pyramids, prisms, hexahedra)        */
/* ------------------------------------------------------------------------ */
/* Local faces of each cell type (node count 4, 5, 6, 8), cyclic; the stored
 * face order of a cell is this order.  Quadrilateral faces end at index 3,
 * triangles have -1 there. */
static const int MF_TET[4][4] = {{1, 2, 3, -1}, {0, 2, 3, -1}, {0, 1, 3, -1}, {0, 1, 2, -1}};
static const int MF_PYR[5][4] = {{0, 1, 2, 3}, {0, 1, 4, -1}, {1, 2, 4, -1}, {2, 3, 4, -1}, {3, 0, 4, -1}};
static const int MF_PRI[5][4] = {{0, 1, 2, -1}, {3, 4, 5, -1}, {0, 1, 4, 3}, {1, 2, 5, 4}, {2, 0, 3, 5}};
static const int MF_HEX[6][4] = {{0, 1, 2, 3}, {4, 5, 6, 7}, {0, 1, 5, 4}, {1, 2, 6, 5}, {2, 3, 7, 6}, {3, 0, 4, 7}};
static int mixed_faces(int type, const int (**tab)[4]) {
  switch (type) {
    case 4: *tab = MF_TET; return 4;
    case 5: *tab = MF_PYR; return 5;
    case 6: *tab = MF_PRI; return 5;
    case 8: *tab = MF_HEX; return 6;
    default: return -1;
  }
}

static void cross3(const double* a, const double* b, double* c) {
  c[0] = a[1] * b[2] - a[2] * b[1]; c[1] = a[2] * b[0] - a[0] * b[2]; c[2] = a[0] * b[1] - a[1] * b[0];
}

/* Volume, centroid and central second moments / V of a cell given by its
 * nodes x [nn][3]: the union of the tetrahedra (node mean, face triangle),
 * each quadrilateral face cut into the 4 triangles around its node mean (the
 * cells are star-shaped about their node mean).  A tetrahedron with vertices
 * p_i (about the node mean) has int x x^T = V/20 (sum p_i p_i^T + s s^T),
 * s = sum p_i. */
static double mixed_geom(int type, int nn, const double* x, double* cen, double* m2) {
  const int (*tab)[4];
  int nf = mixed_faces(type, &tab);
  double xm[3] = {0, 0, 0};
  for (int v = 0; v < nn; ++v) for (int d = 0; d < 3; ++d) xm[d] += x[v * 3 + d] / nn;
  double V = 0, S1[3] = {0, 0, 0}, S2[9] = {0};
  for (int k = 0; k < nf; ++k) {
    int q = tab[k][3] >= 0 ? 4 : 3;
    double tri[4][3][3];  /* up to 4 triangles, vertices about xm */
    int nt = 0;
    if (q == 3) {
      for (int i = 0; i < 3; ++i) for (int d = 0; d < 3; ++d) tri[0][i][d] = x[tab[k][i] * 3 + d] - xm[d];
      nt = 1;
    } else {
      double fc[3] = {0, 0, 0};
      for (int i = 0; i < 4; ++i) for (int d = 0; d < 3; ++d) fc[d] += (x[tab[k][i] * 3 + d] - xm[d]) / 4.0;
      for (int i = 0; i < 4; ++i) {
        for (int d = 0; d < 3; ++d) {
          tri[i][0][d] = fc[d];
          tri[i][1][d] = x[tab[k][i] * 3 + d] - xm[d];
          tri[i][2][d] = x[tab[k][(i + 1) % 4] * 3 + d] - xm[d];
        }
      }
      nt = 4;
    }
    for (int t = 0; t < nt; ++t) {
      /* tetrahedron (0, a, b, c) about the node mean */
      double c3[3];
      cross3(tri[t][1], tri[t][2], c3);
      double vt = fabs(tri[t][0][0] * c3[0] + tri[t][0][1] * c3[1] + tri[t][0][2] * c3[2]) / 6.0;
      double s[3];
      for (int d = 0; d < 3; ++d) s[d] = tri[t][0][d] + tri[t][1][d] + tri[t][2][d];
      V += vt;
      for (int d = 0; d < 3; ++d) S1[d] += vt * s[d] / 4.0;
      for (int a = 0; a < 3; ++a)
        for (int b = 0; b < 3; ++b) {
          double pp = 0;
          for (int i = 0; i < 3; ++i) pp += tri[t][i][a] * tri[t][i][b];
          S2[a * 3 + b] += vt / 20.0 * (pp + s[a] * s[b]);
        }
    }
  }
  for (int d = 0; d < 3; ++d) cen[d] = xm[d] + S1[d] / V;
  for (int a = 0; a < 3; ++a)
    for (int b = 0; b < 3; ++b) m2[a * 3 + b] = S2[a * 3 + b] / V - (S1[a] / V) * (S1[b] / V);
  return V;
}

typedef struct { int key[4]; int cell, k; } MKey;
static int mkey_cmp(const void* a, const void* b) {
  const MKey* x = (const MKey*)a; const MKey* y = (const MKey*)b;
  for (int i = 0; i < 4; ++i) { if (x->key[i] != y->key[i]) return x->key[i] < y->key[i] ? -1 : 1; }
  if (x->cell != y->cell) return x->cell < y->cell ? -1 : 1;
  return x->k - y->k;
}
static int mkey_same(const MKey* x, const MKey* y) {
  for (int i = 0; i < 4; ++i) if (x->key[i] != y->key[i]) return 0;
  return 1;
}
/* sorted node ids of a face, -1 last for a triangle */
static void mkey_make(int q, const int* ids, int* key) {
  int t[4] = {ids[0], ids[1], ids[2], q == 4 ? ids[3] : 0};
  sort_key(q, t);
  for (int i = 0; i < 4; ++i) key[i] = i < q ? t[i] : -1;
}

/* Face geometry from the owning (L) cell's cyclic vertices fv [q][3]:
 * triangle: area vector 1/2 (v1-v0) x (v2-v0), the degree-2 rule of the
 * simplex meshes (barycentric 2/3, 1/6, 1/6), equal weights; quadrilateral:
 * area vector 1/2 (v2-v0) x (v3-v1) (that of the 4 triangles around its node
 * mean), points of the 2 x 2 Gauss-Legendre rule on the bilinear surface
 * x(s, t) = sum N_i(s, t) v_i, weights proportional to |x_s x x_t| there
 * (Sec 2.2: four points per quadrilateral face). */
static void mixed_face_geom(int q, const double (*fv)[3], const double* cell_cen, double* nrm, double* S,
                            double* fc, double* gp, double* gw) {
  double A[3];
  for (int d = 0; d < 3; ++d) { fc[d] = 0; for (int i = 0; i < q; ++i) fc[d] += fv[i][d] / q; }
  if (q == 3) {
    double a[3], b[3];
    for (int d = 0; d < 3; ++d) { a[d] = fv[1][d] - fv[0][d]; b[d] = fv[2][d] - fv[0][d]; }
    cross3(a, b, A);
  } else {
    double a[3], b[3];
    for (int d = 0; d < 3; ++d) { a[d] = fv[2][d] - fv[0][d]; b[d] = fv[3][d] - fv[1][d]; }
    cross3(a, b, A);
  }
  for (int d = 0; d < 3; ++d) A[d] *= 0.5;
  double l = sqrt(A[0] * A[0] + A[1] * A[1] + A[2] * A[2]);
  *S = l;
  for (int d = 0; d < 3; ++d) nrm[d] = A[d] / l;
  double dot = 0; for (int d = 0; d < 3; ++d) dot += (fc[d] - cell_cen[d]) * nrm[d];
  if (dot < 0) for (int d = 0; d < 3; ++d) nrm[d] = -nrm[d];
  if (q == 3) {
    for (int g = 0; g < 3; ++g) {
      for (int d = 0; d < 3; ++d) {
        double s = 0;
        for (int v = 0; v < 3; ++v) s += (v == g ? 2.0 / 3.0 : 1.0 / 6.0) * fv[v][d];
        gp[g * 3 + d] = s;
      }
      gw[g] = 1.0 / 3.0;
    }
    return;
  }
  const double r = 1.0 / sqrt(3.0);
  const double ss[4] = {-r, r, r, -r}, tt[4] = {-r, -r, r, r};
  double wsum = 0;
  for (int g = 0; g < 4; ++g) {
    double s = ss[g], t = tt[g];
    double N[4] = {(1 - s) * (1 - t) / 4, (1 + s) * (1 - t) / 4, (1 + s) * (1 + t) / 4, (1 - s) * (1 + t) / 4};
    double Ns[4] = {-(1 - t) / 4, (1 - t) / 4, (1 + t) / 4, -(1 + t) / 4};
    double Nt[4] = {-(1 - s) / 4, -(1 + s) / 4, (1 + s) / 4, (1 - s) / 4};
    double xs[3] = {0, 0, 0}, xt[3] = {0, 0, 0};
    for (int d = 0; d < 3; ++d) {
      double p = 0;
      for (int i = 0; i < 4; ++i) { p += N[i] * fv[i][d]; xs[d] += Ns[i] * fv[i][d]; xt[d] += Nt[i] * fv[i][d]; }
      gp[g * 3 + d] = p;
    }
    double j3[3];
    cross3(xs, xt, j3);
    gw[g] = sqrt(j3[0] * j3[0] + j3[1] * j3[1] + j3[2] * j3[2]);
    wsum += gw[g];
  }
  for (int g = 0; g < 4; ++g) gw[g] /= wsum;
}

/* Build the fine level of a mixed mesh: cell_type [n] (node count 4, 5, 6 or
 * 8), cell_node_off [n+1], cell_nodes and cell_xyz [sum][3] in the node order
 * of each type; boundary faces by bface_node_off [nb+1], bface_nodes (3 or 4
 * ids) and tags.  Faces match by their sorted node ids.  Returns 0 or a
 * negative code. */
static int build_fine_mixed(OMesh* M, int n, const int* types, const long long* off, const int* cn,
                            const double* cx, int nbf, const long long* boff, const int* bfn, const int* bft,
                            char* err) {
  const int dim = 3;
  M->dim = 3; M->nv = 5; M->ngp = 3; M->nlev = 1;
  OLevel* L = &M->lev[0];
  level_alloc_cells(L, n, dim, MAXF);
  size_t ns = 0;
  for (int c = 0; c < n; ++c) {
    const int (*tab)[4];
    int nf = mixed_faces(types[c], &tab);
    int nn = (int)(off[c + 1] - off[c]);
    if (nf < 0 || nn != types[c]) { snprintf(err, 256, "cell %d: unknown type %d or %d nodes", c, types[c], nn); return -1; }
    L->cnf[c] = nf;
    ns += nf;
    L->vol[c] = types[c] == 4 ? simplex_geom(3, cx + off[c] * 3, L->cen + c * 3, L->mom2 + c * 9)
                              : mixed_geom(types[c], nn, cx + off[c] * 3, L->cen + c * 3, L->mom2 + c * 9);
    if (!(L->vol[c] > 0)) { snprintf(err, 256, "degenerate cell %d", c); return -3; }
  }
  MKey* keys = malloc(ns * sizeof(MKey));
  size_t e = 0;
  for (int c = 0; c < n; ++c) {
    const int (*tab)[4];
    int nf = mixed_faces(types[c], &tab);
    for (int k = 0; k < nf; ++k, ++e) {
      int q = tab[k][3] >= 0 ? 4 : 3, ids[4];
      for (int i = 0; i < q; ++i) ids[i] = cn[off[c] + tab[k][i]];
      mkey_make(q, ids, keys[e].key);
      keys[e].cell = c; keys[e].k = k;
    }
  }
  qsort(keys, ns, sizeof(MKey), mkey_cmp);
  MKey* bk = malloc((size_t)(nbf > 0 ? nbf : 1) * sizeof(MKey));
  for (int b = 0; b < nbf; ++b) {
    int q = (int)(boff[b + 1] - boff[b]);
    if (q != 3 && q != 4) { snprintf(err, 256, "boundary face %d has %d nodes", b, q); free(keys); free(bk); return -1; }
    mkey_make(q, bfn + boff[b], bk[b].key);
    bk[b].cell = b; bk[b].k = 0;
  }
  qsort(bk, nbf, sizeof(MKey), mkey_cmp);
  int n_int = 0, n_bnd = 0;
  for (size_t i = 0; i < ns;) {
    size_t j = i + 1;
    while (j < ns && mkey_same(&keys[j], &keys[i])) ++j;
    if (j - i == 2) n_int++;
    else if (j - i == 1) n_bnd++;
    else { snprintf(err, 256, "face shared by %d cells", (int)(j - i)); free(keys); free(bk); return -3; }
    i = j;
  }
  if (n_bnd != nbf) { snprintf(err, 256, "%d open faces but %d boundary faces given", n_bnd, nbf); free(keys); free(bk); return -3; }
  level_alloc_faces(L, n_int + n_bnd, dim, 1);
  L->n_bfaces = n_bnd;
  L->fngp = calloc((size_t)(n_int + n_bnd), sizeof(int));
  L->fgw = calloc((size_t)(n_int + n_bnd) * MAXG, sizeof(double));
  L->fpt = calloc((size_t)(n_int + n_bnd) * dim, sizeof(double));
  int fi = 0, fb = n_int;
  for (size_t i = 0; i < ns;) {
    size_t j = i + 1;
    while (j < ns && mkey_same(&keys[j], &keys[i])) ++j;
    int f;
    if (j - i == 2) {
      f = fi++;
      L->fL[f] = keys[i].cell; L->fR[f] = keys[i + 1].cell; L->ftag[f] = 0;
      L->cface[keys[i].cell * MAXF + keys[i].k] = f; L->cside[keys[i].cell * MAXF + keys[i].k] = +1;
      L->cface[keys[i + 1].cell * MAXF + keys[i + 1].k] = f; L->cside[keys[i + 1].cell * MAXF + keys[i + 1].k] = -1;
    } else {
      int lo = 0, hi = nbf - 1, found = -1;
      while (lo <= hi) {
        int mid = (lo + hi) / 2, cmp = 0;
        for (int t = 0; t < 4; ++t) if (bk[mid].key[t] != keys[i].key[t]) { cmp = bk[mid].key[t] < keys[i].key[t] ? -1 : 1; break; }
        if (cmp == 0) { found = mid; break; }
        if (cmp < 0) lo = mid + 1; else hi = mid - 1;
      }
      if (found < 0) { snprintf(err, 256, "open face of cell %d not in the boundary list", keys[i].cell); free(keys); free(bk); return -3; }
      f = fb++;
      L->fL[f] = keys[i].cell; L->fR[f] = -1; L->ftag[f] = bft[bk[found].cell];
      L->cface[keys[i].cell * MAXF + keys[i].k] = f; L->cside[keys[i].cell * MAXF + keys[i].k] = +1;
    }
    /* geometry from the L cell's cyclic vertices */
    int cl = L->fL[f], kl = keys[i].k;
    const int (*tab)[4] = MF_TET;
    mixed_faces(types[cl], &tab);
    int q = tab[kl][3] >= 0 ? 4 : 3;
    double fv[4][3];
    for (int v = 0; v < q; ++v) for (int d = 0; d < 3; ++d) fv[v][d] = cx[(off[cl] + tab[kl][v]) * 3 + d];
    double gp[MAXG * 3], gw[MAXG];
    mixed_face_geom(q, (const double (*)[3])fv, L->cen + cl * 3, L->fn + f * 3, &L->fS[f], L->fpt + f * 3, gp, gw);
    L->fngp[f] = q == 4 ? 4 : 3;
    for (int g = 0; g < L->fngp[f]; ++g) {
      L->fgw[(size_t)f * MAXG + g] = gw[g];
      for (int d = 0; d < 3; ++d) L->fgp[((size_t)f * MAXG + g) * 3 + d] = gp[g * 3 + d];
    }
    i = j;
  }
  free(keys); free(bk);
  return 0;
}

/* coarse level from parent map (Sec 5.1: V_c = sum V_i, C_c = sum V_i C_i / V_c).
 * Coarse faces: one per unordered pair (I, J) of distinct parents, with the
 * summed area vector; boundary faces merged per (I, tag).  A coarse cell's
 * faces are stored in ascending order of (neighbour, tag) (reading). */
typedef struct { int I, J, tag; double sn[MAXD]; } CFace;
static int cface_cmp(const void* a, const void* b) {
  const CFace* x = (const CFace*)a; const CFace* y = (const CFace*)b;
  if (x->I != y->I) return x->I < y->I ? -1 : 1;
  if (x->J != y->J) return x->J < y->J ? -1 : 1;
  return x->tag - y->tag;
}
static int build_coarse(OMesh* M, const int* parent, char* err) {
  int dim = M->dim;
  OLevel* F = &M->lev[M->nlev - 1];
  int nc = 0;
  for (int i = 0; i < F->n_cells; ++i) { if (parent[i] < 0) { snprintf(err, 256, "negative parent"); return -1; } if (parent[i] + 1 > nc) nc = parent[i] + 1; }
  F->parent = malloc(F->n_cells * sizeof(int));
  memcpy(F->parent, parent, F->n_cells * sizeof(int));
  /* faces: two half-records per interior coarse face (one per side) */
  CFace* rec = malloc((size_t)(2 * F->n_faces + 1) * sizeof(CFace));
  int nr = 0;
  for (int f = 0; f < F->n_faces; ++f) {
    int I = parent[F->fL[f]];
    if (F->fR[f] < 0) {
      rec[nr].I = I; rec[nr].J = -1; rec[nr].tag = F->ftag[f];
      for (int d = 0; d < dim; ++d) rec[nr].sn[d] = F->fS[f] * F->fn[f * dim + d];
      nr++;
      continue;
    }
    int J = parent[F->fR[f]];
    if (I == J) continue;
    int a = I < J ? I : J, b = I < J ? J : I;
    double sg = (I < J) ? 1.0 : -1.0;
    rec[nr].I = a; rec[nr].J = b; rec[nr].tag = 0;
    for (int d = 0; d < dim; ++d) rec[nr].sn[d] = sg * F->fS[f] * F->fn[f * dim + d];
    nr++;
  }
  qsort(rec, nr, sizeof(CFace), cface_cmp);
  int nu = 0;
  for (int i = 0; i < nr;) {
    int j = i + 1;
    while (j < nr && rec[j].I == rec[i].I && rec[j].J == rec[i].J && rec[j].tag == rec[i].tag) {
      for (int d = 0; d < dim; ++d) rec[i].sn[d] += rec[j].sn[d];
      ++j;
    }
    rec[nu++] = rec[i];
    i = j;
  }
  int n_int = 0, n_bnd = 0;
  for (int i = 0; i < nu; ++i) { if (rec[i].J >= 0) n_int++; else n_bnd++; }
  OLevel* C = &M->lev[M->nlev];
  /* count faces per coarse cell */
  int* cnt = calloc(nc, sizeof(int));
  for (int i = 0; i < nu; ++i) { cnt[rec[i].I]++; if (rec[i].J >= 0) cnt[rec[i].J]++; }
  int maxnf = 0;
  for (int c = 0; c < nc; ++c) if (cnt[c] > maxnf) maxnf = cnt[c];
  level_alloc_cells(C, nc, dim, maxnf);
  level_alloc_faces(C, nu, dim, 0);
  C->n_bfaces = n_bnd;
  int fi = 0, fb = n_int;
  for (int i = 0; i < nu; ++i) {
    int f = rec[i].J >= 0 ? fi++ : fb++;
    C->fL[f] = rec[i].I; C->fR[f] = rec[i].J; C->ftag[f] = rec[i].tag;
    double S = 0; for (int d = 0; d < dim; ++d) S += rec[i].sn[d] * rec[i].sn[d];
    S = sqrt(S);
    C->fS[f] = S;
    for (int d = 0; d < dim; ++d) C->fn[f * dim + d] = rec[i].sn[d] / S;
  }
  /* cell -> face lists, ascending by (neighbour, tag): interior neighbours
   * first in ascending order, then boundary faces by tag */
  for (int c = 0; c < nc; ++c) C->cnf[c] = 0;
  typedef struct { int nb, tag, f, side; } Ent;
  Ent* ent = malloc((size_t)nc * maxnf * sizeof(Ent));
  for (int f = 0; f < nu; ++f) {
    int I = C->fL[f], J = C->fR[f];
    Ent e1 = {J >= 0 ? J : (1 << 30), C->ftag[f], f, +1};
    ent[(size_t)I * maxnf + C->cnf[I]++] = e1;
    if (J >= 0) { Ent e2 = {I, 0, f, -1}; ent[(size_t)J * maxnf + C->cnf[J]++] = e2; }
  }
  for (int c = 0; c < nc; ++c) {
    Ent* e = ent + (size_t)c * maxnf;
    int m = C->cnf[c];
    for (int i = 0; i < m; ++i) for (int j = i + 1; j < m; ++j)
      if (e[j].nb < e[i].nb || (e[j].nb == e[i].nb && e[j].tag < e[i].tag)) { Ent t = e[i]; e[i] = e[j]; e[j] = t; }
    for (int i = 0; i < m; ++i) { C->cface[c * maxnf + i] = e[i].f; C->cside[c * maxnf + i] = e[i].side; }
  }
  free(ent); free(cnt);
  /* volumes and centres */
  for (int i = 0; i < F->n_cells; ++i) {
    int I = parent[i];
    C->vol[I] += F->vol[i];
    for (int d = 0; d < dim; ++d) C->cen[I * dim + d] += F->vol[i] * F->cen[i * dim + d];
  }
  for (int I = 0; I < nc; ++I) {
    if (!(C->vol[I] > 0)) { snprintf(err, 256, "empty coarse cell %d", I); free(rec); return -1; }
    for (int d = 0; d < dim; ++d) C->cen[I * dim + d] /= C->vol[I];
  }
  free(rec);
  M->nlev++;
  return 0;
}

/* ------------------------------------------------------------------------ */
/* colouring (Sec 4.1, Algorithm "coloring")                                 */
/* reading: breadth-first from cell 0 in stored face order, FIFO in painting */
/* order, restart at the lowest unpainted cell                               */
/* ------------------------------------------------------------------------ */
static int nbr_of(const OLevel* L, int c, int k) {
  int f = L->cface[c * L->maxnf + k];
  return L->cside[c * L->maxnf + k] > 0 ? L->fR[f] : L->fL[f];
}
static void color_level(OLevel* L) {
  int n = L->n_cells;
  int* q = malloc(n * sizeof(int));
  int qh = 0, qt = 0, nc = 0;
  for (int i = 0; i < n; ++i) L->color[i] = 0;
  int next = 0;
  int painted = 0;
  while (painted < n) {
    while (next < n && L->color[next] != 0) ++next;
    if (qh == qt) {
      /* (re)start: paint the lowest unpainted cell */
      int v0 = next;
      int used[64] = {0};
      for (int k = 0; k < L->cnf[v0]; ++k) { int w = nbr_of(L, v0, k); if (w >= 0 && L->color[w] > 0 && L->color[w] < 64) used[L->color[w]] = 1; }
      int col = 1; while (used[col]) ++col;
      L->color[v0] = col; if (col > nc) nc = col;
      q[qt++] = v0; painted++;
    }
    while (qh < qt) {
      int v = q[qh++];
      for (int k = 0; k < L->cnf[v]; ++k) {
        int w = nbr_of(L, v, k);
        if (w < 0 || L->color[w] != 0) continue;
        int used[64] = {0};
        for (int kk = 0; kk < L->cnf[w]; ++kk) { int j = nbr_of(L, w, kk); if (j >= 0 && L->color[j] > 0 && L->color[j] < 64) used[L->color[j]] = 1; }
        int col = 1; while (used[col]) ++col;
        L->color[w] = col; if (col > nc) nc = col;
        q[qt++] = w; painted++;
      }
    }
  }
  L->n_colors = nc;
  free(q);
}

/* ------------------------------------------------------------------------ */
/* boundary ghosts (reading: slip wall = mirror; supersonic far field =      */
/* free stream on inflow faces, copy on outflow faces)                       */
/* ------------------------------------------------------------------------ */
static int is_inflow(const OCfg* cfg, int dim, const double* n) {
  double un = 0; for (int d = 0; d < dim; ++d) un += cfg->winf[1 + d] * n[d];
  return un < 0.0;
}
/* ghost mean state across a boundary face with outward unit normal n */
/* far field by the characteristic (Riemann-invariant) boundary state: with
 * the outward normal n, J+ = u_n + 2c/(gamma-1) leaves the domain (interior
 * values) and J- = u_n - 2c/(gamma-1) enters it (free-stream values); on the
 * face u_n = (J+ + J-)/2 and c = (gamma-1)(J+ - J-)/4, while the entropy
 * p/rho^gamma and the tangential velocity are those of the upstream side.  A
 * supersonic normal free stream takes the free stream on inflow and the
 * interior on outflow. */
static void riemann_state(const OCfg* cfg, int dim, const double* n, const double* W, double* Wb) {
  int nv = dim + 2;
  double g = cfg->gamma;
  double ui[MAXD], uf[MAXD], uin = 0, ufn = 0;
  for (int d = 0; d < dim; ++d) {
    ui[d] = W[1 + d] / W[0]; uf[d] = cfg->winf[1 + d] / cfg->winf[0];
    uin += ui[d] * n[d]; ufn += uf[d] * n[d];
  }
  double p_i = pressure(dim, g, W), p_f = pressure(dim, g, cfg->winf);
  double c_i = sqrt(g * p_i / W[0]), c_f = sqrt(g * p_f / cfg->winf[0]);
  if (fabs(ufn) >= c_f) {
    const double* src = ufn < 0.0 ? cfg->winf : W;
    for (int v = 0; v < nv; ++v) Wb[v] = src[v];
    return;
  }
  double jp = uin + 2.0 * c_i / (g - 1.0), jm = ufn - 2.0 * c_f / (g - 1.0);
  double un = 0.5 * (jp + jm), c = 0.25 * (g - 1.0) * (jp - jm);
  int inflow = un < 0.0;
  double s = inflow ? p_f / pow(cfg->winf[0], g) : p_i / pow(W[0], g);
  const double* ut = inflow ? uf : ui;
  double utn = inflow ? ufn : uin;
  double rho = pow(c * c / (g * s), 1.0 / (g - 1.0));
  double p = rho * c * c / g, q2 = 0.0;
  Wb[0] = rho;
  for (int d = 0; d < dim; ++d) {
    double u = ut[d] - utn * n[d] + un * n[d];
    Wb[1 + d] = rho * u;
    q2 += u * u;
  }
  Wb[nv - 1] = p / (g - 1.0) + 0.5 * rho * q2;
}

static void ghost_mean(const OCfg* cfg, int dim, int tag, const double* n, const double* W, double* Wg) {
  int nv = dim + 2;
  if (tag == 4) {
    riemann_state(cfg, dim, n, W, Wg);
  } else if (tag == 1) {
    double mn = 0; for (int d = 0; d < dim; ++d) mn += W[1 + d] * n[d];
    for (int v = 0; v < nv; ++v) Wg[v] = W[v];
    for (int d = 0; d < dim; ++d) Wg[1 + d] = W[1 + d] - 2.0 * mn * n[d];
  } else if (tag == 3) {
    /* no-slip adiabatic wall: the velocity reversed, density and energy kept */
    for (int v = 0; v < nv; ++v) Wg[v] = W[v];
    for (int d = 0; d < dim; ++d) Wg[1 + d] = -W[1 + d];
  } else if (is_inflow(cfg, dim, n)) {
    for (int v = 0; v < nv; ++v) Wg[v] = cfg->winf[v];
  } else {
    for (int v = 0; v < nv; ++v) Wg[v] = W[v];
  }
}
/* ghost gradient G[d][v] (global) */
static void ghost_grad(const OCfg* cfg, int dim, int tag, const double* n, const double* G, double* Gg) {
  int nv = dim + 2;
  if (tag == 1 || tag == 3) {
    /* the ghost field is the mirror image q(H x), H = I - 2 n n^T: scalar fields
     * get H grad; the momentum is reflected at a slip wall, H (dm/dx) H, and
     * reversed at a no-slip wall, -(dm/dx) H */
    double tmp[MAXD * MAXV];
    for (int v = 0; v < nv; ++v) {
      double s = 0; for (int d = 0; d < dim; ++d) s += n[d] * G[d * nv + v];
      for (int d = 0; d < dim; ++d) tmp[d * nv + v] = G[d * nv + v] - 2.0 * n[d] * s;
    }
    for (int d = 0; d < dim; ++d) {
      double s = 0; for (int e = 0; e < dim; ++e) s += n[e] * tmp[d * nv + 1 + e];
      for (int v = 0; v < nv; ++v) Gg[d * nv + v] = tmp[d * nv + v];
      for (int e = 0; e < dim; ++e)
        Gg[d * nv + 1 + e] = tag == 1 ? tmp[d * nv + 1 + e] - 2.0 * n[e] * s : -tmp[d * nv + 1 + e];
    }
  } else if (tag == 4 || is_inflow(cfg, dim, n)) {
    for (int i = 0; i < dim * nv; ++i) Gg[i] = 0.0;
  } else {
    for (int i = 0; i < dim * nv; ++i) Gg[i] = G[i];
  }
}

/* ------------------------------------------------------------------------ */
/* reconstruction (Sec 3.1-3.3)                                              */
/* polynomial per variable: P(X) = c0 + sum_d c_d X_d + sum_{d<=e} c_de X_d X_e */
/* with X = x - x0 (cell centroid)                                           */
/* ------------------------------------------------------------------------ */
#define NCOEF(dim) ((dim) == 2 ? 6 : 10)
static int quad_index(int dim, int d, int e) {
  /* index of X_d X_e (d <= e) among quadratic terms */
  if (d > e) { int t = d; d = e; e = t; }
  if (dim == 2) return d == 0 ? (e == 0 ? 0 : 1) : 2;
  static const int idx[3][3] = {{0, 1, 2}, {1, 3, 4}, {2, 4, 5}};
  return idx[d][e];
}
static double poly_eval(int dim, const double* c, const double* X) {
  double s = c[0];
  for (int d = 0; d < dim; ++d) s += c[1 + d] * X[d];
  for (int d = 0; d < dim; ++d) for (int e = d; e < dim; ++e) s += c[1 + dim + quad_index(dim, d, e)] * X[d] * X[e];
  return s;
}
static void poly_grad(int dim, const double* c, const double* X, double* g) {
  for (int d = 0; d < dim; ++d) {
    double s = c[1 + d];
    for (int e = 0; e < dim; ++e) {
      int q = quad_index(dim, d, e);
      s += (d == e ? 2.0 : 1.0) * c[1 + dim + q] * X[e];
    }
    g[d] = s;
  }
}

/* neighbour record in cell 0's frame */
typedef struct {
  double vol, cen[MAXD], m2[MAXD * MAXD], n[MAXD], S;
  double W[MAXV], G[MAXD * MAXV];
} Nbr;

static void gather_stencil(const OMesh* M, const OCfg* cfg, const double* W, const double* G, int c, Nbr* nb) {
  const OLevel* L = &M->lev[0];
  int dim = M->dim, nv = M->nv;
  for (int k = 0; k < L->cnf[c]; ++k) {
    int f = L->cface[c * L->maxnf + k], side = L->cside[c * L->maxnf + k];
    Nbr* b = &nb[k];
    b->S = L->fS[f];
    for (int d = 0; d < dim; ++d) b->n[d] = side * L->fn[f * dim + d];
    int j = side > 0 ? L->fR[f] : L->fL[f];
    if (j >= 0) {
      b->vol = L->vol[j];
      for (int d = 0; d < dim; ++d) b->cen[d] = L->cen[j * dim + d] + side * L->fshift[f * dim + d];
      for (int i = 0; i < dim * dim; ++i) b->m2[i] = L->mom2[j * dim * dim + i];
      for (int v = 0; v < nv; ++v) b->W[v] = W[j * nv + v];
      for (int i = 0; i < dim * nv; ++i) b->G[i] = G[(size_t)j * dim * nv + i];
    } else {
      /* ghost: mirror image of cell c across the face plane */
      const double* n = b->n;
      const double* x0 = L->cen + c * dim;
      const double* xf = L->fpt ? L->fpt + (size_t)f * dim : L->fgp + (size_t)f * MAXG * dim; /* on the face plane */
      double h = 0; for (int d = 0; d < dim; ++d) h += (xf[d] - x0[d]) * n[d];
      b->vol = L->vol[c];
      for (int d = 0; d < dim; ++d) b->cen[d] = x0[d] + 2.0 * h * n[d];
      const double* m = L->mom2 + c * dim * dim;
      double Hm[MAXD * MAXD];
      for (int a = 0; a < dim; ++a) for (int e = 0; e < dim; ++e) {
        double s = 0; for (int q = 0; q < dim; ++q) s += ((a == q) - 2.0 * n[a] * n[q]) * m[q * dim + e];
        Hm[a * dim + e] = s;
      }
      for (int a = 0; a < dim; ++a) for (int e = 0; e < dim; ++e) {
        double s = 0; for (int q = 0; q < dim; ++q) s += Hm[a * dim + q] * ((q == e) - 2.0 * n[q] * n[e]);
        b->m2[a * dim + e] = s;
      }
      ghost_mean(cfg, dim, L->ftag[f], n, W + c * nv, b->W);
      ghost_grad(cfg, dim, L->ftag[f], n, G + (size_t)c * dim * nv, b->G);
    }
  }
}

/* the cell's face Gauss points in its own frame */
static int cell_gauss_points(const OMesh* M, int c, double* pts) {
  const OLevel* L = &M->lev[0];
  int dim = M->dim, m = 0;
  for (int k = 0; k < L->cnf[c]; ++k) {
    int f = L->cface[c * L->maxnf + k], side = L->cside[c * L->maxnf + k];
    int ng = L->fngp ? L->fngp[f] : M->ngp;
    for (int g = 0; g < ng; ++g, ++m)
      for (int d = 0; d < dim; ++d)
        pts[m * dim + d] = L->fgp[((size_t)f * MAXG + g) * dim + d] - (side > 0 ? 0.0 : L->fshift[f * dim + d]);
  }
  return m;
}

/* multi-index list for 1 <= |k| <= 2: first the dim linear ones, then the
 * quadratic ones in quad_index order */
static void kmulti(int dim, int idx, int* p, int* q) {
  if (idx < dim) { *p = idx; *q = -1; return; }
  int r = idx - dim;
  for (int d = 0; d < dim; ++d) for (int e = d; e < dim; ++e) if (quad_index(dim, d, e) == r) { *p = d; *q = e; return; }
}

/* reconstruct cell c: coefficients out[nv][ncoef]; returns 1 if the positivity
 * fallback was taken */
/* Nonlinear combination of the large-stencil quadratic p2 (coefficients c2)
 * and the Green-Gauss linear p1 (c1), Sec 3.3 with the weights deferred by the
 * paper (reading: WENO-Z type with one large and one sub stencil):
 *   tau = |b2 - b1|,  w~H = gH (1 + tau/(b2+eps)),  w~L = gL (1 + tau/(b1+eps)),
 *   (wH, wL) = (w~H, w~L) / (w~H + w~L),  P = (wH/gH)(p2 - gL p1) + wL p1,
 * with gL = 1 - gH and b1, b2 the smoothness indicators of p1 and p2. */
static void hweno_combine(int nco, double b1, double b2, double gh, double eps, const double* c1,
                          const double* c2, double* out) {
  double gl = 1.0 - gh;
  double tz = fabs(b2 - b1);
  double wh = gh * (1.0 + tz / (b2 + eps)), wl = gl * (1.0 + tz / (b1 + eps));
  double ws = wh + wl;
  wh /= ws; wl /= ws;
  for (int i = 0; i < nco; ++i) out[i] = wh / gh * (c2[i] - gl * c1[i]) + wl * c1[i];
}

static int reconstruct_cell(const OMesh* M, const OCfg* cfg, const double* W, const double* G,
                            const double* alpha_prev, int c, double* out, int* rank_fallback) {
  const OLevel* L = &M->lev[0];
  int dim = M->dim, nv = M->nv, nf = L->cnf[c], nk = dim == 2 ? 5 : 9, nco = NCOEF(dim);
  Nbr nb[MAXF];
  gather_stencil(M, cfg, W, G, c, nb);
  const double* x0 = L->cen + c * dim;
  const double* m0 = L->mom2 + c * dim * dim;
  double V0 = L->vol[c];
  double h = pow(V0, 1.0 / dim);
  /* average of X^k over cell 0 and over each neighbour (in 0's frame) */
  double avg0[MAXK], avgm[MAXF][MAXK], davg[MAXF][MAXD][MAXK];
  for (int k = 0; k < nk; ++k) {
    int p, q; kmulti(dim, k, &p, &q);
    avg0[k] = q < 0 ? 0.0 : m0[p * dim + q];
    for (int m = 0; m < nf; ++m) {
      double dx[MAXD];
      for (int d = 0; d < dim; ++d) dx[d] = nb[m].cen[d] - x0[d];
      avgm[m][k] = q < 0 ? dx[p] : nb[m].m2[p * dim + q] + dx[p] * dx[q];
      for (int d = 0; d < dim; ++d) {
        /* average over Omega_m of d/dx_d of X^k */
        if (q < 0) davg[m][d][k] = (d == p) ? 1.0 : 0.0;
        else davg[m][d][k] = (d == p ? dx[q] : 0.0) + (d == q ? dx[p] : 0.0);
      }
    }
  }
  /* constrained least squares per variable, unknowns scaled by h^|k|:
   * minimise |B a - d|^2 subject to C a = e  via the KKT system */
  int ne = nf, nl = nf * dim, n = nk + ne;
  double A[(MAXK + MAXF) * (MAXK + MAXF)], R[(MAXK + MAXF) * MAXV];
  double Bm[MAXF * MAXD][MAXK], Cm[MAXF][MAXK];
  for (int k = 0; k < nk; ++k) {
    int p, q; kmulti(dim, k, &p, &q);
    double sc = q < 0 ? h : h * h;
    for (int m = 0; m < nf; ++m) {
      Cm[m][k] = (avgm[m][k] - avg0[k]) / sc;
      for (int d = 0; d < dim; ++d) Bm[m * dim + d][k] = davg[m][d][k] / sc;
    }
  }
  for (int i = 0; i < n * n; ++i) A[i] = 0.0;
  for (int i = 0; i < nk; ++i) for (int j = 0; j < nk; ++j) {
    double s = 0; for (int r = 0; r < nl; ++r) s += Bm[r][i] * Bm[r][j];
    A[i * n + j] = s;
  }
  for (int m = 0; m < ne; ++m) for (int k = 0; k < nk; ++k) { A[(nk + m) * n + k] = Cm[m][k]; A[k * n + nk + m] = Cm[m][k]; }
  for (int v = 0; v < nv; ++v) {
    for (int i = 0; i < nk; ++i) {
      double s = 0;
      for (int m = 0; m < nf; ++m) for (int d = 0; d < dim; ++d) s += Bm[m * dim + d][i] * nb[m].G[d * nv + v];
      R[i * nv + v] = s;
    }
    for (int m = 0; m < ne; ++m) R[(nk + m) * nv + v] = nb[m].W[v] - W[c * nv + v];
  }
  int ok = gauss_solve(A, R, n, nv, 1e-12) == 0;
  if (!ok && rank_fallback) (*rank_fallback)++;
  double ap = alpha_prev[c];
  double beta_scale1 = pow(V0, 2.0 / dim - 1.0), beta_scale2 = pow(V0, 4.0 / dim - 1.0);
  for (int v = 0; v < nv; ++v) {
    double W0 = W[c * nv + v];
    /* p1: Green-Gauss in difference form, scaled by the previous DF (Sec 3.2-3.3) */
    double g1[MAXD] = {0, 0, 0};
    for (int m = 0; m < nf; ++m) for (int d = 0; d < dim; ++d) g1[d] += (nb[m].W[v] - W0) * nb[m].S * nb[m].n[d] / (2.0 * V0);
    for (int d = 0; d < dim; ++d) g1[d] *= ap;
    double c1[10] = {0};
    c1[0] = W0;
    for (int d = 0; d < dim; ++d) c1[1 + d] = g1[d];
    /* p2 in monomial form about x0 */
    double c2[10] = {0};
    if (ok) {
      double a[MAXK];
      for (int k = 0; k < nk; ++k) { int p, q; kmulti(dim, k, &p, &q); a[k] = R[k * nv + v] / (q < 0 ? h : h * h); }
      double cst = W0;
      for (int k = 0; k < nk; ++k) cst -= a[k] * avg0[k];
      c2[0] = cst;
      for (int k = 0; k < nk; ++k) {
        int p, q; kmulti(dim, k, &p, &q);
        if (q < 0) c2[1 + p] = a[k]; else c2[1 + dim + quad_index(dim, p, q)] = a[k];
      }
    }
    if (!ok) { for (int i = 0; i < nco; ++i) out[v * nco + i] = c1[i]; continue; }
    /* smoothness indicators (reading: sum_l |Omega|^(2|l|/dim - 1) int (D^l p)^2) */
    double b1 = beta_scale1 * V0 * (g1[0] * g1[0] + g1[1] * g1[1] + (dim == 3 ? g1[2] * g1[2] : 0.0));
    double b2 = 0.0;
    {
      double Hs[MAXD][MAXD];
      for (int d = 0; d < dim; ++d) for (int e = 0; e < dim; ++e)
        Hs[d][e] = (d == e ? 2.0 : 1.0) * c2[1 + dim + quad_index(dim, d, e)];
      for (int d = 0; d < dim; ++d) {
        /* int (c_d + H_d . X)^2 = V (c_d^2 + H_d M H_d) since <X> = 0 */
        double s = 0;
        for (int a = 0; a < dim; ++a) for (int e = 0; e < dim; ++e) s += Hs[d][a] * m0[a * dim + e] * Hs[d][e];
        b2 += beta_scale1 * V0 * (c2[1 + d] * c2[1 + d] + s);
      }
      for (int d = 0; d < dim; ++d) for (int e = d; e < dim; ++e) b2 += beta_scale2 * V0 * Hs[d][e] * Hs[d][e];
    }
    hweno_combine(nco, b1, b2, cfg->weno_gh, cfg->weno_eps, c1, c2, out + v * nco);
  }
  /* positivity: density and pressure at every face Gauss point of the cell */
  double pts[MAXF * MAXG * MAXD];
  int np = cell_gauss_points(M, c, pts);
  int bad = 0;
  for (int g = 0; g < np && !bad; ++g) {
    double X[MAXD], Wp[MAXV];
    for (int d = 0; d < dim; ++d) X[d] = pts[g * dim + d] - x0[d];
    for (int v = 0; v < nv; ++v) Wp[v] = poly_eval(dim, out + v * nco, X);
    if (!(Wp[0] > 0.0) || !(pressure(dim, cfg->gamma, Wp) > 0.0)) bad = 1;
  }
  if (bad) {
    for (int v = 0; v < nv; ++v) { for (int i = 0; i < nco; ++i) out[v * nco + i] = 0.0; out[v * nco] = W[c * nv + v]; }
  }
  return bad;
}

/* ------------------------------------------------------------------------ */
/* local time steps (reading: dt_i = CFL V_i / sum_f S_f (|u_i.n_f| + c_i))  */
/* ------------------------------------------------------------------------ */
static void time_steps(const OMesh* M, int lev, const OCfg* cfg, const double* W, double* dte, double* dti) {
  const OLevel* L = &M->lev[lev];
  int dim = M->dim, nv = M->nv;
#pragma omp parallel for schedule(static)
  for (int c = 0; c < L->n_cells; ++c) {
    const double* w = W + c * nv;
    double cs = sqrt(cfg->gamma * pressure(dim, cfg->gamma, w) / w[0]);
    double sum = 0;
    for (int k = 0; k < L->cnf[c]; ++k) {
      int f = L->cface[c * L->maxnf + k];
      double un = 0; for (int d = 0; d < dim; ++d) un += w[1 + d] / w[0] * L->fn[f * dim + d];
      sum += L->fS[f] * (fabs(un) + cs);
    }
    if (dte) dte[c] = cfg->cfl_exp * L->vol[c] / sum;
    if (dti) dti[c] = cfg->cfl_imp * L->vol[c] / sum;
  }
}

/* ------------------------------------------------------------------------ */
/* third-order residual on the fine level (Sec 2.2-2.4, Sec 3)               */
/* ------------------------------------------------------------------------ */
typedef struct { long long recon_fallback, rank_fallback, update_halved, update_zeroed; } OStats;

static void fine_residual(const OMesh* M, const OCfg* cfg, const double* W, const double* G,
                          const double* alpha_prev, double* R, double* Gnew, double* alpha,
                          double* dte, double* dti, OStats* st) {
  const OLevel* L = &M->lev[0];
  int dim = M->dim, nv = M->nv, n = L->n_cells, nco = NCOEF(dim);
  double* dtl = malloc(n * sizeof(double));
  time_steps(M, 0, cfg, W, dtl, dti);
  if (dte) memcpy(dte, dtl, n * sizeof(double));
  double* P = malloc((size_t)n * nv * nco * sizeof(double));
  int* bad = calloc(n, sizeof(int));
  int* rf = calloc(n, sizeof(int));
  /* cells are independent: OpenMP threads may share them out */
#pragma omp parallel for schedule(dynamic, 16)
  for (int c = 0; c < n; ++c) bad[c] = reconstruct_cell(M, cfg, W, G, alpha_prev, c, P + (size_t)c * nv * nco, &rf[c]);
  if (st) for (int c = 0; c < n; ++c) { st->recon_fallback += bad[c]; st->rank_fallback += rf[c]; }
  free(bad); free(rf);
  for (int i = 0; i < n * nv; ++i) R[i] = 0.0;
  for (int i = 0; i < n * nv * dim; ++i) Gnew[i] = 0.0;
  for (int c = 0; c < n; ++c) alpha[c] = 1.0;
  double wq = 1.0 / M->ngp;
  /* per-face results (faces are independent), then summed into the cells in
     face order, so the sums do not depend on the thread count */
  int nf = L->n_faces;
  double* FsA = malloc((size_t)nf * nv * sizeof(double));
  double* WsA = malloc((size_t)nf * nv * sizeof(double));
  double* afA = malloc((size_t)nf * sizeof(double));
#pragma omp parallel for schedule(dynamic, 16)
  for (int f = 0; f < nf; ++f) {
    int cl = L->fL[f], cr = L->fR[f], tag = L->ftag[f];
    const double* n_ = L->fn + f * dim;
    double Rm[MAXD * MAXD];
    frame(dim, n_, Rm);
    double dt = dtl[cl];
    if (cr >= 0 && dtl[cr] < dt) dt = dtl[cr];
    double Fs[MAXV] = {0}, Ws[MAXV] = {0}, af = 1.0;
    int ng = L->fngp ? L->fngp[f] : M->ngp;
    for (int g = 0; g < ng; ++g) {
      double wg = L->fgw ? L->fgw[(size_t)f * MAXG + g] : wq;
      const double* xg = L->fgp + ((size_t)f * MAXG + g) * dim;
      double Xl[MAXD], Wl[MAXV], Gl[MAXD * MAXV], Wr[MAXV], Gr[MAXD * MAXV], gg[MAXD];
      for (int d = 0; d < dim; ++d) Xl[d] = xg[d] - L->cen[cl * dim + d];
      for (int v = 0; v < nv; ++v) {
        const double* pc = P + ((size_t)cl * nv + v) * nco;
        Wl[v] = poly_eval(dim, pc, Xl);
        poly_grad(dim, pc, Xl, gg);
        for (int d = 0; d < dim; ++d) Gl[d * nv + v] = gg[d];
      }
      if (cr >= 0) {
        double Xr[MAXD];
        for (int d = 0; d < dim; ++d) Xr[d] = xg[d] - L->fshift[f * dim + d] - L->cen[cr * dim + d];
        for (int v = 0; v < nv; ++v) {
          const double* pc = P + ((size_t)cr * nv + v) * nco;
          Wr[v] = poly_eval(dim, pc, Xr);
          poly_grad(dim, pc, Xr, gg);
          for (int d = 0; d < dim; ++d) Gr[d * nv + v] = gg[d];
        }
      } else {
        ghost_mean(cfg, dim, tag, n_, Wl, Wr);
        ghost_grad(cfg, dim, tag, n_, Gl, Gr);
      }
      double wl[MAXV], wr[MAXV], gl[MAXD * MAXV], gr[MAXD * MAXV], Floc[MAXV], Wtl[MAXV], Fg[MAXV], Wg[MAXV];
      rot_to(dim, Rm, Wl, wl);
      rot_to(dim, Rm, Wr, wr);
      rot_grad(dim, Rm, Gl, gl);
      rot_grad(dim, Rm, Gr, gr);
      gks_point(dim, cfg->gamma, cfg->tau_c1, cfg->tau_c2, cfg->mu, wl, gl, wr, gr, dt, Floc, Wtl, NULL);
      rot_from(dim, Rm, Floc, Fg);
      rot_from(dim, Rm, Wtl, Wg);
      for (int v = 0; v < nv; ++v) { Fs[v] += wg * Fg[v]; Ws[v] += wg * Wg[v]; }
      af *= df_point(dim, cfg->gamma, wl, wr);
    }
    for (int v = 0; v < nv; ++v) { FsA[(size_t)f * nv + v] = Fs[v]; WsA[(size_t)f * nv + v] = Ws[v]; }
    afA[f] = af;
  }
  for (int f = 0; f < nf; ++f) {
    int cl = L->fL[f], cr = L->fR[f];
    const double* n_ = L->fn + f * dim;
    const double* Fs = FsA + (size_t)f * nv;
    const double* Ws = WsA + (size_t)f * nv;
    double af = afA[f];
    double S = L->fS[f];
    for (int v = 0; v < nv; ++v) {
      R[cl * nv + v] += S * Fs[v];
      for (int d = 0; d < dim; ++d) Gnew[((size_t)cl * dim + d) * nv + v] += S * Ws[v] * n_[d] / L->vol[cl];
    }
    alpha[cl] *= af;
    if (cr >= 0) {
      for (int v = 0; v < nv; ++v) {
        R[cr * nv + v] -= S * Fs[v];
        for (int d = 0; d < dim; ++d) Gnew[((size_t)cr * dim + d) * nv + v] -= S * Ws[v] * n_[d] / L->vol[cr];
      }
      alpha[cr] *= af;
    }
  }
  free(FsA); free(WsA); free(afA);
  free(P); free(dtl);
}

/* first-order KFVS residual on a coarse level (Sec 5.2) */
static void kfvs_residual(const OMesh* M, int lev, const OCfg* cfg, const double* W, double* R) {
  const OLevel* L = &M->lev[lev];
  int dim = M->dim, nv = M->nv;
  for (int i = 0; i < L->n_cells * nv; ++i) R[i] = 0.0;
  /* face fluxes (independent), then summed into the cells in face order */
  double* FgA = malloc((size_t)L->n_faces * nv * sizeof(double));
#pragma omp parallel for schedule(static)
  for (int f = 0; f < L->n_faces; ++f) {
    int cl = L->fL[f], cr = L->fR[f];
    const double* n_ = L->fn + f * dim;
    double Rm[MAXD * MAXD], Wr[MAXV], wl[MAXV], wr[MAXV], Fl[MAXV];
    frame(dim, n_, Rm);
    if (cr >= 0) memcpy(Wr, W + cr * nv, nv * sizeof(double));
    else ghost_mean(cfg, dim, L->ftag[f], n_, W + cl * nv, Wr);
    rot_to(dim, Rm, W + cl * nv, wl);
    rot_to(dim, Rm, Wr, wr);
    kfvs_point(dim, cfg->gamma, wl, wr, Fl);
    rot_from(dim, Rm, Fl, FgA + (size_t)f * nv);
  }
  for (int f = 0; f < L->n_faces; ++f) {
    int cl = L->fL[f], cr = L->fR[f];
    const double* Fg = FgA + (size_t)f * nv;
    for (int v = 0; v < nv; ++v) {
      R[cl * nv + v] += L->fS[f] * Fg[v];
      if (cr >= 0) R[cr * nv + v] -= L->fS[f] * Fg[v];
    }
  }
  free(FgA);
}

/* ------------------------------------------------------------------------ */
/* multi-colour LU-SGS with DF relaxation (Sec 4.2-4.3)                      */
/* ------------------------------------------------------------------------ */
static double spectral_radius(int dim, double gamma, double rs, const double* Wi, const double* Wj, const double* n) {
  int nv = dim + 2;
  double m[MAXV];
  for (int v = 0; v < nv; ++v) m[v] = 0.5 * (Wi[v] + Wj[v]);
  double un = 0; for (int d = 0; d < dim; ++d) un += m[1 + d] / m[0] * n[d];
  double c = sqrt(gamma * pressure(dim, gamma, m) / m[0]);
  return rs * (fabs(un) + c);
}

/* positivity guard on an update (reading): halve up to 10 times, else drop */
static void apply_update(int dim, double gamma, double* W, const double* dW, OStats* st) {
  int nv = dim + 2;
  double s = 1.0, Wn[MAXV];
  for (int it = 0; it <= 10; ++it) {
    for (int v = 0; v < nv; ++v) Wn[v] = W[v] + s * dW[v];
    if (Wn[0] > 0.0 && pressure(dim, gamma, Wn) > 0.0) {
      if (it > 0 && st) {
#pragma omp atomic update
        st->update_halved++;
      }
      for (int v = 0; v < nv; ++v) W[v] = Wn[v];
      return;
    }
    s *= 0.5;
  }
  if (st) {
#pragma omp atomic update
    st->update_zeroed++;
  }
}

/* One forward + backward sweep for  D dW + 1/2 alpha sum S [dT - r dW] = rhs
 * and the state update.  rhs = -R (fine) or -(R + P) (coarse). */
static void lusgs(const OMesh* M, int lev, const OCfg* cfg, double* W, const double* rhs,
                  const double* alpha, const double* dte, const double* dti, double* dW_out, OStats* st) {
  const OLevel* L = &M->lev[lev];
  int dim = M->dim, nv = M->nv, n = L->n_cells;
  double* D = malloc(n * sizeof(double));
  double* dWs = calloc((size_t)n * nv, sizeof(double));
  double* dW = calloc((size_t)n * nv, sizeof(double));
  double* r = malloc(L->n_faces * sizeof(double));
#pragma omp parallel for schedule(static)
  for (int f = 0; f < L->n_faces; ++f) {
    int cl = L->fL[f], cr = L->fR[f];
    double Wg[MAXV];
    const double* Wj;
    if (cr >= 0) Wj = W + cr * nv;
    else { ghost_mean(cfg, dim, L->ftag[f], L->fn + f * dim, W + cl * nv, Wg); Wj = Wg; }
    r[f] = spectral_radius(dim, cfg->gamma, cfg->r_safety, W + cl * nv, Wj, L->fn + f * dim);
  }
#pragma omp parallel for schedule(static)
  for (int c = 0; c < n; ++c) {
    double s = 0;
    for (int k = 0; k < L->cnf[c]; ++k) { int f = L->cface[c * L->maxnf + k]; s += L->fS[f] * r[f]; }
    double a = alpha[c];
    /* reading: implicit time step in the alpha term, explicit one in the (1-alpha) term */
    D[c] = a * (L->vol[c] / dti[c] + 0.5 * s) + (1.0 - a) * L->vol[c] / dte[c];
  }
  /* off-diagonal sum over neighbours j selected by colour */
  for (int pass = 0; pass < 2; ++pass) {
    int nc = L->n_colors;
    for (int ci = 0; ci < nc; ++ci) {
      int col = pass == 0 ? ci + 1 : nc - ci;
      /* the cells of one colour are independent of each other */
#pragma omp parallel for schedule(static)
      for (int c = 0; c < n; ++c) {
        if (L->color[c] != col) continue;
        double sum[MAXV] = {0};
        for (int k = 0; k < L->cnf[c]; ++k) {
          int f = L->cface[c * L->maxnf + k], side = L->cside[c * L->maxnf + k];
          int j = side > 0 ? L->fR[f] : L->fL[f];
          if (j < 0) continue;  /* reading: ghost dW = 0 */
          if (pass == 0 ? !(L->color[j] < col) : !(L->color[j] > col)) continue;
          const double* dj = (pass == 0 ? dWs : dW) + j * nv;
          double nn[MAXD], Wp[MAXV], T1[MAXV], T0[MAXV];
          for (int d = 0; d < dim; ++d) nn[d] = side * L->fn[f * dim + d];
          for (int v = 0; v < nv; ++v) Wp[v] = W[j * nv + v] + dj[v];
          euler_flux(dim, cfg->gamma, Wp, nn, T1);
          euler_flux(dim, cfg->gamma, W + j * nv, nn, T0);
          for (int v = 0; v < nv; ++v) sum[v] += L->fS[f] * ((T1[v] - T0[v]) - r[f] * dj[v]);
        }
        for (int v = 0; v < nv; ++v) {
          if (pass == 0) dWs[c * nv + v] = (rhs[c * nv + v] - 0.5 * alpha[c] * sum[v]) / D[c];
          else dW[c * nv + v] = dWs[c * nv + v] - 0.5 * alpha[c] * sum[v] / D[c];
        }
      }
    }
  }
#pragma omp parallel for schedule(static)
  for (int c = 0; c < n; ++c) apply_update(dim, cfg->gamma, W + c * nv, dW + c * nv, st);
  if (dW_out) memcpy(dW_out, dW, (size_t)n * nv * sizeof(double));
  free(D); free(dWs); free(dW); free(r);
}

/* ------------------------------------------------------------------------ */
/* multigrid (Sec 5.2)                                                       */
/* ------------------------------------------------------------------------ */
static void restrict_state(const OMesh* M, int lev, const double* Wf, const double* af,
                           double* Wc, double* ac) {
  const OLevel* F = &M->lev[lev];
  const OLevel* C = &M->lev[lev + 1];
  int nv = M->nv;
  for (int i = 0; i < C->n_cells * nv; ++i) Wc[i] = 0.0;
  for (int i = 0; i < C->n_cells; ++i) ac[i] = 1.0;
  for (int i = 0; i < F->n_cells; ++i) {
    int I = F->parent[i];
    for (int v = 0; v < nv; ++v) Wc[I * nv + v] += F->vol[i] * Wf[i * nv + v];
    if (af[i] < ac[I]) ac[I] = af[i];  /* reading: coarse DF = min over children */
  }
  for (int I = 0; I < C->n_cells; ++I) for (int v = 0; v < nv; ++v) Wc[I * nv + v] /= C->vol[I];
}
static void restrict_sum(const OMesh* M, int lev, const double* Rf, double* Rc) {
  const OLevel* F = &M->lev[lev];
  const OLevel* C = &M->lev[lev + 1];
  int nv = M->nv;
  for (int i = 0; i < C->n_cells * nv; ++i) Rc[i] = 0.0;
  for (int i = 0; i < F->n_cells; ++i) for (int v = 0; v < nv; ++v) Rc[F->parent[i] * nv + v] += Rf[i * nv + v];
}

/* n_sweep FAS smoothing steps on coarse level `lev` given the forcing P:
 * each step: Rt = R^lev(W) + P, LU-SGS on -Rt, update */
static void coarse_smooth(const OMesh* M, int lev, const OCfg* cfg, double* W, const double* Pf,
                          const double* alpha, int nsw, OStats* st) {
  const OLevel* L = &M->lev[lev];
  int nv = M->nv, n = L->n_cells;
  double* R = malloc((size_t)n * nv * sizeof(double));
  double* rhs = malloc((size_t)n * nv * sizeof(double));
  double* dte = malloc(n * sizeof(double));
  double* dti = malloc(n * sizeof(double));
  for (int s = 0; s < nsw; ++s) {
    kfvs_residual(M, lev, cfg, W, R);
    for (int i = 0; i < n * nv; ++i) rhs[i] = -(R[i] + Pf[i]);
    time_steps(M, lev, cfg, W, dte, dti);
    lusgs(M, lev, cfg, W, rhs, alpha, dte, dti, NULL, st);
  }
  free(R); free(rhs); free(dte); free(dti);
}

/* injection prolongation limited by DF: W_f += alpha_f (W_c - W_c0)[parent] */
static void prolong(const OMesh* M, int lev, const OCfg* cfg, double* Wf, const double* af,
                    const double* Wc, const double* Wc0, OStats* st) {
  const OLevel* F = &M->lev[lev];
  int nv = M->nv;
#pragma omp parallel for schedule(static)
  for (int i = 0; i < F->n_cells; ++i) {
    int I = F->parent[i];
    double d[MAXV];
    for (int v = 0; v < nv; ++v) d[v] = af[i] * (Wc[I * nv + v] - Wc0[I * nv + v]);
    apply_update(M->dim, cfg->gamma, Wf + i * nv, d, st);
  }
}

static void norms_of(const OMesh* M, int lev, const double* R, double* out /* [nv*2] */) {
  const OLevel* L = &M->lev[lev];
  int nv = M->nv;
  for (int v = 0; v < nv; ++v) {
    double s = 0, mx = 0;
    for (int c = 0; c < L->n_cells; ++c) { double q = R[c * nv + v] / L->vol[c]; s += q * q; if (fabs(q) > mx) mx = fabs(q); }
    out[v * 2] = sqrt(s / L->n_cells);
    out[v * 2 + 1] = mx;
  }
}

/* ------------------------------------------------------------------------ */
/* exported API (ctypes)                                                     */
/* ------------------------------------------------------------------------ */
static char g_err[256];
const char* om_last_error(void) { return g_err; }
/* threads of the OpenMP loops over independent cells and faces (results do not
 * depend on it: every sum over cells or faces is formed in a fixed order) */
void om_set_threads(int n) {
#ifdef _OPENMP
  if (n > 0) omp_set_num_threads(n);
#else
  (void)n;
#endif
}
int om_get_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}

void* om_create(int dim, int n_cells, const int* cell_nodes, const double* cell_xyz, int n_bf,
                const int* bface_nodes, const int* bface_tag) {
  if (dim != 2 && dim != 3) { snprintf(g_err, 256, "dim must be 2 or 3"); return NULL; }
  OMesh* M = calloc(1, sizeof(OMesh));
  if (build_fine(M, dim, n_cells, cell_nodes, cell_xyz, n_bf, bface_nodes, bface_tag, g_err) != 0) { free(M); return NULL; }
  color_level(&M->lev[0]);
  return M;
}
void* om_create_mixed(int n_cells, const int* cell_type, const long long* cell_node_off, const int* cell_nodes,
                      const double* cell_xyz, int n_bf, const long long* bface_node_off, const int* bface_nodes,
                      const int* bface_tag) {
  OMesh* M = calloc(1, sizeof(OMesh));
  if (build_fine_mixed(M, n_cells, cell_type, cell_node_off, cell_nodes, cell_xyz, n_bf, bface_node_off, bface_nodes,
                       bface_tag, g_err) != 0) { free(M); return NULL; }
  color_level(&M->lev[0]);
  return M;
}
/* Gauss points per face and their weights (mixed meshes; 0 / -1 elsewhere) */
void om_get_face_gauss(void* h, int lev, int* ngp, double* w) {
  OLevel* L = &((OMesh*)h)->lev[lev];
  for (int f = 0; f < L->n_faces; ++f) {
    ngp[f] = L->fngp ? L->fngp[f] : 0;
    for (int g = 0; g < MAXG; ++g) w[f * MAXG + g] = L->fgw ? L->fgw[f * MAXG + g] : -1.0;
  }
}
int om_add_level(void* h, const int* parent) {
  OMesh* M = (OMesh*)h;
  if (M->nlev >= 8) { snprintf(g_err, 256, "too many levels"); return -1; }
  if (build_coarse(M, parent, g_err) != 0) return -1;
  color_level(&M->lev[M->nlev - 1]);
  return 0;
}
void om_destroy(void* h) {
  OMesh* M = (OMesh*)h;
  if (!M) return;
  for (int l = 0; l < M->nlev; ++l) {
    OLevel* L = &M->lev[l];
    free(L->vol); free(L->cen); free(L->mom2); free(L->fL); free(L->fR); free(L->ftag); free(L->fn);
    free(L->fS); free(L->fshift); free(L->fgp); free(L->cnf); free(L->cface); free(L->cside);
    free(L->parent); free(L->color); free(L->fngp); free(L->fgw); free(L->fpt);
  }
  free(M);
}
int om_num_levels(void* h) { return ((OMesh*)h)->nlev; }
int om_num_cells(void* h, int lev) { return ((OMesh*)h)->lev[lev].n_cells; }
int om_num_faces(void* h, int lev) { return ((OMesh*)h)->lev[lev].n_faces; }
int om_num_bfaces(void* h, int lev) { return ((OMesh*)h)->lev[lev].n_bfaces; }
int om_num_colors(void* h, int lev) { return ((OMesh*)h)->lev[lev].n_colors; }
int om_max_faces_per_cell(void* h, int lev) { return ((OMesh*)h)->lev[lev].maxnf; }
void om_get_colors(void* h, int lev, int* out) { OLevel* L = &((OMesh*)h)->lev[lev]; memcpy(out, L->color, L->n_cells * sizeof(int)); }
void om_get_cells(void* h, int lev, double* vol, double* cen, double* m2) {
  OMesh* M = (OMesh*)h; OLevel* L = &M->lev[lev]; int dim = M->dim;
  if (vol) memcpy(vol, L->vol, L->n_cells * sizeof(double));
  if (cen) memcpy(cen, L->cen, (size_t)L->n_cells * dim * sizeof(double));
  if (m2 && L->mom2) memcpy(m2, L->mom2, (size_t)L->n_cells * dim * dim * sizeof(double));
}
/* faces: L, R (-1 boundary), tag, normal[dim], S, shift[dim], gauss points [MAXG*dim] (fine only) */
void om_get_faces(void* h, int lev, int* fl, int* fr, int* tag, double* n, double* S, double* shift, double* gp) {
  OMesh* M = (OMesh*)h; OLevel* L = &M->lev[lev]; int dim = M->dim, nf = L->n_faces;
  memcpy(fl, L->fL, nf * sizeof(int)); memcpy(fr, L->fR, nf * sizeof(int)); memcpy(tag, L->ftag, nf * sizeof(int));
  memcpy(n, L->fn, (size_t)nf * dim * sizeof(double)); memcpy(S, L->fS, nf * sizeof(double));
  memcpy(shift, L->fshift, (size_t)nf * dim * sizeof(double));
  if (gp && L->fgp) memcpy(gp, L->fgp, (size_t)nf * MAXG * dim * sizeof(double));
}
/* cell -> neighbour list in stored order (-1 for boundary), [n*maxnf], count per cell */
void om_get_neighbors(void* h, int lev, int* cnt, int* nb) {
  OMesh* M = (OMesh*)h; OLevel* L = &M->lev[lev];
  for (int c = 0; c < L->n_cells; ++c) {
    cnt[c] = L->cnf[c];
    for (int k = 0; k < L->maxnf; ++k) nb[c * L->maxnf + k] = k < L->cnf[c] ? nbr_of(L, c, k) : -2;
  }
}

void om_gks_point(int dim, const double* cfgv, const double* Wl, const double* dWl, const double* Wr,
                  const double* dWr, double dt, double* F, double* Wt, double* dbg /* 2*15+5+15+5+1+5 */) {
  OCfg cfg; cfg_from(cfgv, dim + 2, &cfg);
  GksDebug d;
  gks_point(dim, cfg.gamma, cfg.tau_c1, cfg.tau_c2, cfg.mu, Wl, dWl, Wr, dWr, dt, F, Wt, &d);
  if (dbg) {
    int o = 0;
    for (int a = 0; a < MAXD; ++a) for (int i = 0; i < MAXV; ++i) dbg[o++] = d.al[a][i];
    for (int i = 0; i < MAXV; ++i) dbg[o++] = d.Al[i];
    for (int a = 0; a < MAXD; ++a) for (int i = 0; i < MAXV; ++i) dbg[o++] = d.ar[a][i];
    for (int i = 0; i < MAXV; ++i) dbg[o++] = d.Ar[i];
    for (int i = 0; i < MAXV; ++i) dbg[o++] = d.Wc[i];
    for (int a = 0; a < MAXD; ++a) for (int i = 0; i < MAXV; ++i) dbg[o++] = d.ac[a][i];
    for (int i = 0; i < MAXV; ++i) dbg[o++] = d.Ac[i];
    dbg[o++] = d.tau;
  }
}
void om_kfvs_point(int dim, double gamma, const double* Wl, const double* Wr, double* F) { kfvs_point(dim, gamma, Wl, Wr, F); }
void om_hweno_combine(int nco, double b1, double b2, double gh, double eps, const double* c1, const double* c2,
                      double* out) { hweno_combine(nco, b1, b2, gh, eps, c1, c2, out); }
double om_df_point(int dim, double gamma, const double* Wl, const double* Wr) { return df_point(dim, gamma, Wl, Wr); }
void om_euler_flux(int dim, double gamma, const double* W, const double* n, double* T) { euler_flux(dim, gamma, W, n, T); }

/* reconstruction polynomials of every fine cell: out[n][nv][ncoef] */
long long om_reconstruct(void* h, const double* cfgv, const double* W, const double* G, const double* alpha_prev, double* out) {
  OMesh* M = (OMesh*)h; OCfg cfg; cfg_from(cfgv, M->nv, &cfg);
  long long nb = 0;
  int nco = NCOEF(M->dim);
  for (int c = 0; c < M->lev[0].n_cells; ++c) nb += reconstruct_cell(M, &cfg, W, G, alpha_prev, c, out + (size_t)c * M->nv * nco, NULL);
  return nb;
}
void om_time_steps(void* h, int lev, const double* cfgv, const double* W, double* dte, double* dti) {
  OMesh* M = (OMesh*)h; OCfg cfg; cfg_from(cfgv, M->nv, &cfg);
  time_steps(M, lev, &cfg, W, dte, dti);
}
void om_residual(void* h, const double* cfgv, const double* W, const double* G, const double* alpha_prev,
                 double* R, double* Gnew, double* alpha, double* dte, double* dti) {
  OMesh* M = (OMesh*)h; OCfg cfg; cfg_from(cfgv, M->nv, &cfg);
  fine_residual(M, &cfg, W, G, alpha_prev, R, Gnew, alpha, dte, dti, NULL);
}
void om_kfvs_residual(void* h, int lev, const double* cfgv, const double* W, double* R) {
  OMesh* M = (OMesh*)h; OCfg cfg; cfg_from(cfgv, M->nv, &cfg);
  kfvs_residual(M, lev, &cfg, W, R);
}
/* one LU-SGS step on level lev with rhs; W updated in place; dW returned */
void om_lusgs(void* h, int lev, const double* cfgv, double* W, const double* rhs, const double* alpha,
              const double* dte, const double* dti, double* dW) {
  OMesh* M = (OMesh*)h; OCfg cfg; cfg_from(cfgv, M->nv, &cfg);
  lusgs(M, lev, &cfg, W, rhs, alpha, dte, dti, dW, NULL);
}
void om_restrict(void* h, int lev, const double* Wf, const double* af, const double* Rf, double* Wc, double* ac, double* Rc) {
  OMesh* M = (OMesh*)h;
  restrict_state(M, lev, Wf, af, Wc, ac);
  if (Rf && Rc) restrict_sum(M, lev, Rf, Rc);
}
/* coarse correction on level lev: forcing P = Rstar - R^lev(W0), n_sweep
 * smoothing steps from W0; returns the smoothed state in W */
void om_coarse_solve(void* h, int lev, const double* cfgv, const double* W0, const double* Rstar, const double* alpha, double* W) {
  OMesh* M = (OMesh*)h; OCfg cfg; cfg_from(cfgv, M->nv, &cfg);
  int n = M->lev[lev].n_cells, nv = M->nv;
  double* P = malloc((size_t)n * nv * sizeof(double));
  kfvs_residual(M, lev, &cfg, W0, P);
  for (int i = 0; i < n * nv; ++i) P[i] = Rstar[i] - P[i];
  memcpy(W, W0, (size_t)n * nv * sizeof(double));
  coarse_smooth(M, lev, &cfg, W, P, alpha, cfg.n_sweep, NULL);
  free(P);
}
void om_norms(void* h, int lev, const double* R, double* out) { norms_of((OMesh*)h, lev, R, out); }

/* The DF factor a cell keeps for the next reconstruction, the LU-SGS
 * relaxation and the prolongation: the product of its Gauss-point factors
 * (Sec 3.3), or, where that product exceeds the kept value, a step of
 * alpha_relax towards it (reading: a pseudo-time under-relaxation; a steady
 * state is a fixed point either way). */
static double stored_df(const OCfg* cfg, double kept, double product) {
  if (cfg->alpha_relax < 1.0 && product > kept) return kept + cfg->alpha_relax * (product - kept);
  return product;
}

/* V-cycles (Sec 5.2, pre-smooth 1, post-smooth 0).  State (W, G, alpha) is
 * updated in place.  norms[c*nv*2 ...] receives the fine-level residual norms
 * (RMS and max of R/V per variable) measured at the start of cycle c.
 * stats[4]: reconstruction fallbacks, rank fallbacks, halved and zeroed updates. */
int om_vcycle(void* h, const double* cfgv, double* W, double* G, double* alpha, int n_cycles,
              double* norms, long long* stats) {
  OMesh* M = (OMesh*)h; OCfg cfg; cfg_from(cfgv, M->nv, &cfg);
  int nv = M->nv, dim = M->dim, n0 = M->lev[0].n_cells, nl = M->nlev;
  OStats st = {0, 0, 0, 0};
  double* R = malloc((size_t)n0 * nv * sizeof(double));
  double* Gn = malloc((size_t)n0 * nv * dim * sizeof(double));
  double* an = malloc(n0 * sizeof(double));
  double* dte = malloc(n0 * sizeof(double));
  double* dti = malloc(n0 * sizeof(double));
  double* rhs = malloc((size_t)n0 * nv * sizeof(double));
  double *Wl[8], *Wl0[8], *al[8], *Rs[8], *Pl[8], *kl[8], *one[8];
  /* kl: the constant relaxation factor of each level; one: plain injection */
  for (int l = 0; l < nl; ++l) {
    int n = M->lev[l].n_cells;
    kl[l] = malloc(n * sizeof(double)); one[l] = malloc(n * sizeof(double));
    for (int c = 0; c < n; ++c) { kl[l][c] = cfg.relax; one[l][c] = 1.0; }
    if (l == 0) continue;
    Wl[l] = malloc((size_t)n * nv * sizeof(double)); Wl0[l] = malloc((size_t)n * nv * sizeof(double));
    al[l] = malloc(n * sizeof(double)); Rs[l] = malloc((size_t)n * nv * sizeof(double));
    Pl[l] = malloc((size_t)n * nv * sizeof(double));
  }
  const int use_df = cfg.relax < 0.0;
  for (int cyc = 0; cyc < n_cycles; ++cyc) {
    /* 1. residual, DF and slopes; slope update with DF */
    fine_residual(M, &cfg, W, G, alpha, R, Gn, an, dte, dti, &st);
    if (norms) norms_of(M, 0, R, norms + (size_t)cyc * nv * 2);
    for (int c = 0; c < n0; ++c) {
      alpha[c] = stored_df(&cfg, alpha[c], an[c]);
      for (int i = 0; i < nv * dim; ++i) {
        double* g = &G[(size_t)c * nv * dim + i];
        double target = alpha[c] * Gn[(size_t)c * nv * dim + i];
        *g = cfg.slope_relax < 1.0 ? *g + cfg.slope_relax * (target - *g) : target;
      }
    }
    /* 2. fine pre-smoothing: one DF-relaxed LU-SGS step driven by -R, or the
       explicit local-time-step update W -= dt R / V (Eq. smo) */
    if (cfg.fine_smoother == 1) {
      for (int c = 0; c < n0; ++c) {
        double d[MAXV];
        for (int v = 0; v < nv; ++v) d[v] = -dte[c] * R[(size_t)c * nv + v] / M->lev[0].vol[c];
        apply_update(dim, cfg.gamma, W + (size_t)c * nv, d, &st);
      }
    } else {
      for (int i = 0; i < n0 * nv; ++i) rhs[i] = -R[i];
      lusgs(M, 0, &cfg, W, rhs, use_df ? alpha : kl[0], dte, dti, NULL, &st);
    }
    if (nl == 1) continue;
    /* 3. residual at the smoothed state (slopes not updated); its DF is kept */
    fine_residual(M, &cfg, W, G, alpha, R, Gn, an, NULL, NULL, &st);
    for (int c = 0; c < n0; ++c) alpha[c] = stored_df(&cfg, alpha[c], an[c]);
    /* 4-7. restriction, forcing and coarse smoothing, level by level */
    const double* Wf = W; const double* af = alpha; const double* Rf = R;
    for (int l = 1; l < nl; ++l) {
      int n = M->lev[l].n_cells;
      restrict_state(M, l - 1, Wf, af, Wl0[l], al[l]);
      restrict_sum(M, l - 1, Rf, Rs[l]);
      /* forcing: reading: P = R* - R(W0) and coarse rhs = -(R(W) + P) */
      kfvs_residual(M, l, &cfg, Wl0[l], Pl[l]);
      for (int i = 0; i < n * nv; ++i) Pl[l][i] = Rs[l][i] - Pl[l][i];
      memcpy(Wl[l], Wl0[l], (size_t)n * nv * sizeof(double));
      coarse_smooth(M, l, &cfg, Wl[l], Pl[l], use_df ? al[l] : kl[l], cfg.n_sweep, &st);
      if (l + 1 < nl) {
        /* residual to restrict: R^l(W) + P at the smoothed state */
        kfvs_residual(M, l, &cfg, Wl[l], Rs[l]);
        for (int i = 0; i < n * nv; ++i) Rs[l][i] += Pl[l][i];
      }
      Wf = Wl[l]; af = al[l]; Rf = Rs[l];
    }
    /* 8. DF-limited prolongation, coarse to fine */
    for (int l = nl - 1; l >= 1; --l) {
      if (l - 1 >= 1) prolong(M, l - 1, &cfg, Wl[l - 1], cfg.df_prolong ? al[l - 1] : one[l - 1], Wl[l], Wl0[l], &st);
      else prolong(M, 0, &cfg, W, cfg.df_prolong ? alpha : one[0], Wl[l], Wl0[l], &st);
    }
  }
  if (stats) { stats[0] = st.recon_fallback; stats[1] = st.rank_fallback; stats[2] = st.update_halved; stats[3] = st.update_zeroed; }
  free(R); free(Gn); free(an); free(dte); free(dti); free(rhs);
  for (int l = 0; l < nl; ++l) {
    free(kl[l]); free(one[l]);
    if (l > 0) { free(Wl[l]); free(Wl0[l]); free(al[l]); free(Rs[l]); free(Pl[l]); }
  }
  return 0;
}
/* ghost state of a boundary face (tag, outward unit normal n) for the interior W */
void om_ghost_state(int dim, const double* cfgv, int tag, const double* n, const double* W, double* Wg) {
  OCfg cfg; cfg_from(cfgv, dim + 2, &cfg);
  ghost_mean(&cfg, dim, tag, n, W, Wg);
}
/* DF-limited injection prolongation from level lev+1 into level lev */
void om_prolong(void* h, int lev, const double* cfgv, double* Wf, const double* af, const double* Wc, const double* Wc0) {
  OMesh* M = (OMesh*)h; OCfg cfg; cfg_from(cfgv, M->nv, &cfg);
  prolong(M, lev, &cfg, Wf, af, Wc, Wc0, NULL);
}
