"""FP64 CPU oracle of the GMG-CGKS V-cycle (arXiv 2509.06347).

TEST INFRASTRUCTURE ONLY: imported by tests/, by the smoke check and by the
CPU-baseline leg of bench.py, never by the product path.  It shares no code
with the CUDA library; see cgks_oracle.c for the paper sections it follows.

Parity status per function (pins live in tests/test_oracle_*.py):
  geometry, colouring, coarse agglomeration ........ pinned (closed forms, invariants)
  gas-kinetic point flux and point value ........... pinned (Euler flux, brute-force
                                                     velocity/time quadrature, symmetry)
  KFVS flux, DF factor, Euler flux ................. pinned (closed forms, limits)
  reconstruction (p2, p1, weights) ................. pinned (quadratic exactness,
                                                     constants; weights: equal-beta
                                                     limit P = p2, hand-worked cases,
                                                     indicators by independent quadrature)
  fine residual .................................... pinned (free stream, conservation)
  LU-SGS ........................................... pinned (dense block factorisation,
                                                     alpha = 0 explicit limit)
  FAS forcing / prolongation ....................... pinned (zero-forcing, alpha = 0)
  agglomeration coarsening (agglomerate.py) ......... pinned (hand-worked hashes, closed-form
                                                     skewness in 2D and 3D, a hash-decided
                                                     strip, partition invariants)
  V-cycle histories ................................ parity unpinned beyond the above
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "cgks_oracle.c")
_LIB = os.path.join(_HERE, "_build", "libcgks_oracle.so")

DEFAULTS = dict(gamma=1.4, cfl_imp=10.0, cfl_exp=0.5, tau_c1=0.01, tau_c2=1.0,
                weno_gamma_high=0.95, weno_eps=1e-15, r_safety=1.0, n_sweep=6,
                relax=-1.0, df_prolong=1, fine_smoother=0, mu=0.0, slope_relax=1.0, alpha_relax=1.0)


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (plain -O2, no fast-math, no FMA contraction;
    OpenMP over independent cells and faces, with every sum in a fixed order so
    that results do not depend on the thread count)."""
    os.makedirs(os.path.dirname(_LIB), exist_ok=True)
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-D_GNU_SOURCE", "-fPIC", "-shared", "-fopenmp",
                               "-ffp-contract=off", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


_lib = None


def lib():
    global _lib
    if _lib is None:
        _lib = C.CDLL(build())
        P, I, D, LL = C.c_void_p, C.c_int, C.c_double, C.c_longlong
        dp = np.ctypeslib.ndpointer(np.float64, flags="C_CONTIGUOUS")
        ip = np.ctypeslib.ndpointer(np.int32, flags="C_CONTIGUOUS")
        lp = np.ctypeslib.ndpointer(np.int64, flags="C_CONTIGUOUS")
        sig = {
            "om_last_error": (C.c_char_p, []),
            "om_create": (P, [I, I, ip, dp, I, ip, ip]),
            "om_create_mixed": (P, [I, ip, lp, ip, dp, I, lp, ip, ip]),
            "om_get_face_gauss": (None, [P, I, ip, dp]),
            "om_add_level": (I, [P, ip]),
            "om_destroy": (None, [P]),
            "om_num_levels": (I, [P]),
            "om_num_cells": (I, [P, I]),
            "om_num_faces": (I, [P, I]),
            "om_num_bfaces": (I, [P, I]),
            "om_num_colors": (I, [P, I]),
            "om_max_faces_per_cell": (I, [P, I]),
            "om_get_colors": (None, [P, I, ip]),
            "om_get_cells": (None, [P, I, dp, dp, dp]),
            "om_get_faces": (None, [P, I, ip, ip, ip, dp, dp, dp, dp]),
            "om_get_neighbors": (None, [P, I, ip, ip]),
            "om_gks_point": (None, [I, dp, dp, dp, dp, dp, D, dp, dp, dp]),
            "om_kfvs_point": (None, [I, D, dp, dp, dp]),
            "om_hweno_combine": (None, [I, D, D, D, D, dp, dp, dp]),
            "om_df_point": (D, [I, D, dp, dp]),
            "om_euler_flux": (None, [I, D, dp, dp, dp]),
            "om_reconstruct": (LL, [P, dp, dp, dp, dp, dp]),
            "om_time_steps": (None, [P, I, dp, dp, dp, dp]),
            "om_residual": (None, [P, dp, dp, dp, dp, dp, dp, dp, dp, dp]),
            "om_kfvs_residual": (None, [P, I, dp, dp, dp]),
            "om_lusgs": (None, [P, I, dp, dp, dp, dp, dp, dp, dp]),
            "om_restrict": (None, [P, I, dp, dp, dp, dp, dp, dp]),
            "om_coarse_solve": (None, [P, I, dp, dp, dp, dp, dp]),
            "om_norms": (None, [P, I, dp, dp]),
            "om_vcycle": (I, [P, dp, dp, dp, dp, I, dp, lp]),
            "om_prolong": (None, [P, I, dp, dp, dp, dp, dp]),
            "om_ghost_state": (None, [I, dp, I, dp, dp, dp]),
            "om_set_threads": (None, [I]),
            "om_get_threads": (I, []),
        }
        for name, (res, args) in sig.items():
            fn = getattr(_lib, name)
            fn.restype = res
            fn.argtypes = args
    return _lib


def set_threads(n: int) -> int:
    """Threads of the oracle's OpenMP loops (results are the same for any
    count); returns the count now in effect."""
    lib().om_set_threads(int(n))
    return int(lib().om_get_threads())


def get_threads() -> int:
    return int(lib().om_get_threads())


def cfg_vector(dim: int, winf=None, **over) -> np.ndarray:
    """Flat configuration: gamma, cfl_imp, cfl_exp, tau_c1, tau_c2, weno_gamma_high,
    weno_eps, r_safety, n_sweep, then the free-stream state (nv values), then the
    V-cycle switches: relax (negative: DF relaxes LU-SGS; else this constant
    stands for DF), df_prolong (1: DF-scaled prolongation; 0: plain injection)
    and fine_smoother (0: LU-SGS step; 1: explicit update), then mu (dynamic
    viscosity; 0 for the Euler equations), then slope_relax and alpha_relax
    (pseudo-time under-relaxation of the slope update and of a rise of the
    stored DF factor; 1 replaces them)."""
    c = dict(DEFAULTS)
    c.update(over)
    nv = dim + 2
    w = np.zeros(nv) if winf is None else np.asarray(winf, float)
    if winf is None:
        w[0] = 1.0
        w[-1] = 1.0 / (c["gamma"] * (c["gamma"] - 1.0))
    return np.ascontiguousarray(np.concatenate([[c["gamma"], c["cfl_imp"], c["cfl_exp"], c["tau_c1"],
                                                 c["tau_c2"], c["weno_gamma_high"], c["weno_eps"],
                                                 c["r_safety"], float(c["n_sweep"])], w,
                                                [c["relax"], float(c["df_prolong"]), float(c["fine_smoother"]),
                                                 c["mu"], c["slope_relax"], c["alpha_relax"]]]))


def _c(a, dt=np.float64):
    return np.ascontiguousarray(a, dtype=dt)


class OracleMesh:
    """Mesh hierarchy held by the oracle (original cell numbering throughout)."""

    def __init__(self, mesh: dict, levels: int | None = None):
        L = lib()
        self.dim = int(mesh["dim"])
        self.nv = self.dim + 2
        self.mixed = bool(mesh.get("mixed", False))
        cn = _c(mesh["cell_nodes"], np.int32)
        cx = _c(mesh["cell_xyz"])
        bn = _c(mesh["bface_nodes"], np.int32).reshape(-1)
        bt = _c(mesh["bface_tag"], np.int32)
        if bn.size == 0:
            bn = np.zeros(1, np.int32)
            bt_arg = np.zeros(1, np.int32)
        else:
            bt_arg = bt
        if self.mixed:
            # tetrahedra, pyramids, prisms and hexahedra (cell type = node count)
            ct = _c(mesh["cell_type"], np.int32)
            self.h = L.om_create_mixed(ct.size, ct, _c(mesh["cell_node_off"], np.int64), cn.reshape(-1),
                                       cx.reshape(-1), int(bt.size), _c(mesh["bface_node_off"], np.int64),
                                       bn, bt_arg)
        else:
            self.h = L.om_create(self.dim, cn.shape[0], cn.reshape(-1), cx.reshape(-1),
                                 int(bt.size), bn, bt_arg)
        if not self.h:
            raise RuntimeError("oracle mesh: " + L.om_last_error().decode())
        parents = mesh.get("parents", [])
        if levels is not None:
            parents = parents[: levels - 1]
        for p in parents:
            if L.om_add_level(self.h, _c(p, np.int32)) != 0:
                raise RuntimeError("oracle hierarchy: " + L.om_last_error().decode())

    def __del__(self):
        if getattr(self, "h", None):
            lib().om_destroy(self.h)
            self.h = None

    # --- topology and geometry -------------------------------------------
    @property
    def n_levels(self):
        return lib().om_num_levels(self.h)

    def n_cells(self, lev=0):
        return lib().om_num_cells(self.h, lev)

    def colors(self, lev=0):
        out = np.zeros(self.n_cells(lev), np.int32)
        lib().om_get_colors(self.h, lev, out)
        return out

    def n_colors(self, lev=0):
        return lib().om_num_colors(self.h, lev)

    def cells(self, lev=0):
        n, d = self.n_cells(lev), self.dim
        vol, cen, m2 = np.zeros(n), np.zeros((n, d)), np.zeros((n, d, d))
        lib().om_get_cells(self.h, lev, vol, cen.reshape(-1), m2.reshape(-1))
        return vol, cen, m2

    def faces(self, lev=0):
        nf, d = lib().om_num_faces(self.h, lev), self.dim
        fl, fr, tag = (np.zeros(nf, np.int32) for _ in range(3))
        n, S, sh, gp = np.zeros((nf, d)), np.zeros(nf), np.zeros((nf, d)), np.zeros((nf, 4, d))
        lib().om_get_faces(self.h, lev, fl, fr, tag, n.reshape(-1), S, sh.reshape(-1), gp.reshape(-1))
        out = dict(L=fl, R=fr, tag=tag, n=n, S=S, shift=sh, gp=gp)
        if self.mixed and lev == 0:
            ngp, w = np.zeros(nf, np.int32), np.zeros((nf, 4))
            lib().om_get_face_gauss(self.h, lev, ngp, w.reshape(-1))
            out.update(ngp=ngp, gw=w)
        return out

    def neighbors(self, lev=0):
        n = self.n_cells(lev)
        m = lib().om_max_faces_per_cell(self.h, lev)
        cnt = np.zeros(n, np.int32)
        nb = np.zeros(n * m, np.int32)
        lib().om_get_neighbors(self.h, lev, cnt, nb)
        return cnt, nb.reshape(n, m)

    # --- the scheme --------------------------------------------------------
    def reconstruct(self, cfg, W, G, alpha_prev):
        n, nv, d = self.n_cells(), self.nv, self.dim
        nco = 6 if d == 2 else 10
        out = np.zeros((n, nv, nco))
        Gi = np.ascontiguousarray(np.transpose(np.asarray(G, float), (0, 2, 1)))  # -> [n, dim, nv]
        nb = lib().om_reconstruct(self.h, _c(cfg), _c(W), Gi.reshape(-1), _c(alpha_prev),
                                  out.reshape(-1))
        return out, int(nb)

    def time_steps(self, cfg, W, lev=0):
        n = self.n_cells(lev)
        dte, dti = np.zeros(n), np.zeros(n)
        lib().om_time_steps(self.h, lev, _c(cfg), _c(W), dte, dti)
        return dte, dti

    def residual(self, cfg, W, G, alpha_prev):
        """Fine third-order residual.  G is [n, nv, dim] (d/dx_d of variable v)."""
        n, nv, d = self.n_cells(), self.nv, self.dim
        Gi = np.ascontiguousarray(np.transpose(np.asarray(G, float), (0, 2, 1)))  # -> [n, dim, nv]
        R, Gn = np.zeros((n, nv)), np.zeros((n, d, nv))
        al, dte, dti = np.zeros(n), np.zeros(n), np.zeros(n)
        lib().om_residual(self.h, _c(cfg), _c(W), Gi.reshape(-1), _c(alpha_prev), R.reshape(-1),
                          Gn.reshape(-1), al, dte, dti)
        return dict(R=R, grad=np.transpose(Gn, (0, 2, 1)).copy(), alpha=al, dt_exp=dte, dt_imp=dti)

    def kfvs_residual(self, cfg, W, lev):
        R = np.zeros((self.n_cells(lev), self.nv))
        lib().om_kfvs_residual(self.h, lev, _c(cfg), _c(W), R.reshape(-1))
        return R

    def lusgs(self, cfg, W, rhs, alpha, dte, dti, lev=0):
        Wn = _c(W).copy()
        dW = np.zeros_like(Wn)
        lib().om_lusgs(self.h, lev, _c(cfg), Wn.reshape(-1), _c(rhs), _c(alpha), _c(dte), _c(dti),
                       dW.reshape(-1))
        return Wn, dW

    def restrict(self, lev, Wf, af, Rf=None):
        nc = self.n_cells(lev + 1)
        Wc, ac, Rc = np.zeros((nc, self.nv)), np.zeros(nc), np.zeros((nc, self.nv))
        Rfa = _c(Rf) if Rf is not None else np.zeros((self.n_cells(lev), self.nv))
        lib().om_restrict(self.h, lev, _c(Wf), _c(af), Rfa, Wc, ac, Rc)
        return Wc, ac, Rc

    def coarse_solve(self, cfg, lev, W0, Rstar, alpha):
        W = np.zeros((self.n_cells(lev), self.nv))
        lib().om_coarse_solve(self.h, lev, _c(cfg), _c(W0), _c(Rstar), _c(alpha), W)
        return W

    def prolong(self, cfg, lev, Wf, af, Wc, Wc0):
        W = _c(Wf).copy()
        lib().om_prolong(self.h, lev, _c(cfg), W, _c(af), _c(Wc), _c(Wc0))
        return W

    def norms(self, R, lev=0):
        out = np.zeros((self.nv, 2))
        lib().om_norms(self.h, lev, _c(R), out.reshape(-1))
        return out

    def vcycle(self, cfg, W, G, alpha, n_cycles):
        """Run n_cycles V-cycles from (W, G, alpha); returns the new state,
        per-cycle fine norms [n_cycles, nv, 2] and fallback counters."""
        n, nv, d = self.n_cells(), self.nv, self.dim
        Ws = _c(W).copy()
        Gs = np.ascontiguousarray(np.transpose(np.asarray(G, float), (0, 2, 1))).copy()
        al = _c(alpha).copy()
        norms = np.zeros((n_cycles, nv, 2))
        stats = np.zeros(4, np.int64)
        lib().om_vcycle(self.h, _c(cfg), Ws.reshape(-1), Gs.reshape(-1), al, n_cycles,
                        norms.reshape(-1), stats)
        return dict(W=Ws, grad=np.transpose(Gs, (0, 2, 1)).copy(), alpha=al, norms=norms,
                    stats=stats)


def ghost_state(dim, cfg, tag, n, W):
    """Ghost state across a boundary face with outward unit normal n."""
    Wg = np.zeros(dim + 2)
    lib().om_ghost_state(dim, _c(cfg), int(tag), _c(n), _c(W), Wg)
    return Wg


def gks_point(dim, cfg, Wl, dWl, Wr, dWr, dt):
    """Gas-kinetic flux at one Gauss point in the local frame.

    dWl/dWr are [dim, nv]: derivative along (n, t1, t2) of each conservative
    variable.  Returns (Fbar, W(dt), debug dict of the expansion coefficients)."""
    nv = dim + 2
    F, Wt, dbg = np.zeros(nv), np.zeros(nv), np.zeros(66)
    lib().om_gks_point(dim, _c(cfg), _c(Wl), _c(dWl).reshape(-1), _c(Wr), _c(dWr).reshape(-1),
                       float(dt), F, Wt, dbg)
    o = 0

    def take(k):
        nonlocal o
        v = dbg[o:o + k]
        o += k
        return v
    d = dict(al=take(15).reshape(3, 5)[:dim, :nv], Al=take(5)[:nv], ar=take(15).reshape(3, 5)[:dim, :nv],
             Ar=take(5)[:nv], Wc=take(5)[:nv], ac=take(15).reshape(3, 5)[:dim, :nv], Ac=take(5)[:nv],
             tau=take(1)[0])
    return F, Wt, d


def hweno_combine(b1, b2, gamma_high, eps, c1, c2):
    """Nonlinear HWENO combination of the sub-stencil linear polynomial c1 and
    the large-stencil quadratic c2 (coefficient vectors of equal length) with
    smoothness indicators b1, b2 (Sec 3.3, reading R9)."""
    c1, c2 = _c(c1), _c(c2)
    out = np.zeros_like(c1)
    lib().om_hweno_combine(c1.size, float(b1), float(b2), float(gamma_high), float(eps), c1, c2, out)
    return out


def kfvs_point(dim, gamma, Wl, Wr):
    F = np.zeros(dim + 2)
    lib().om_kfvs_point(dim, gamma, _c(Wl), _c(Wr), F)
    return F


def df_point(dim, gamma, Wl, Wr):
    return lib().om_df_point(dim, gamma, _c(Wl), _c(Wr))


def euler_flux(dim, gamma, W, n):
    T = np.zeros(dim + 2)
    lib().om_euler_flux(dim, gamma, _c(W), _c(n), T)
    return T
