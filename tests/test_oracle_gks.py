"""Pins of the oracle's gas-kinetic machinery (Sec 2.1, 2.3, 3.3, 5.2 of the paper).

The oracle integrates polynomial x Maxwellian moments through the 1-D moment
recursion.  These tests integrate the same distribution functions by brute-force
quadrature in velocity space (Gauss-Legendre in u on each half line, in v, w and
in the radial internal-energy variable) and in time, and check closed forms:
the Euler flux of a uniform state, mirror symmetry, the KFVS upwind limit and
the DF factor of equal states.
"""
import math

import numpy as np
import pytest

import oracle

GAMMA = 1.4


def K_of(dim, gamma=GAMMA):
    return (4 - 2 * gamma) / (gamma - 1) if dim == 2 else (5 - 3 * gamma) / (gamma - 1)


def euler_flux_local(dim, W, gamma=GAMMA):
    """Closed-form Euler flux through a face with normal e_1."""
    rho = W[0]
    u = W[1:1 + dim] / rho
    p = (gamma - 1) * (W[-1] - 0.5 * rho * np.dot(u, u))
    F = np.zeros(dim + 2)
    F[0] = rho * u[0]
    F[1:1 + dim] = rho * u[0] * u
    F[1] += p
    F[-1] = (W[-1] + p) * u[0]
    return F


def random_state(rng, dim):
    rho = rng.uniform(0.6, 1.8)
    u = rng.uniform(-0.9, 0.9, dim)
    p = rng.uniform(0.5, 1.6)
    E = p / (GAMMA - 1) + 0.5 * rho * np.dot(u, u)
    return np.concatenate([[rho], rho * u, [E]])


class BruteMaxwellian:
    """Quadrature nodes over (u, v, [w], xi) for brute-force velocity integrals.

    u: composite Gauss-Legendre on each half line (the half-space split is what
    the erfc moments encode); v, w: Gauss-Hermite about the mean velocity;
    internal energy: generalised Gauss-Laguerre in y = |xi|^2 over R^K."""

    def __init__(self, dim, nu=96, nh=12, nl=8, span=7.5):
        self.dim = dim
        self.K = K_of(dim)
        self.nu, self.nh, self.nl, self.span = nu, nh, nl, span

    def nodes(self, W):
        from scipy.special import roots_genlaguerre
        dim, K = self.dim, self.K
        rho = W[0]
        U = W[1:1 + dim] / rho
        p = (GAMMA - 1) * (W[-1] - 0.5 * rho * np.dot(U, U))
        lam = rho / (2 * p)
        sig = 1.0 / math.sqrt(lam)
        x, w = np.polynomial.legendre.leggauss(self.nu)
        L = abs(U[0]) + self.span * sig
        un = np.concatenate([-L * 0.5 * (x + 1), L * 0.5 * (x + 1)])
        uw = np.concatenate([L * 0.5 * w, L * 0.5 * w]) * np.exp(-lam * (un - U[0]) ** 2)
        axes, wts = [un], [uw]
        xh, wh = np.polynomial.hermite.hermgauss(self.nh)
        for d in range(1, dim):
            axes.append(U[d] + xh * sig)
            wts.append(wh * sig)
        y, wy = roots_genlaguerre(self.nl, K / 2 - 1)
        area = 2 * math.pi ** (K / 2) / math.gamma(K / 2)
        axes.append(y / lam)  # |xi|^2
        wts.append(0.5 * area * lam ** (-K / 2) * wy)
        grids = np.meshgrid(*axes, indexing="ij")
        wgrid = np.ones_like(grids[0])
        for i, wt in enumerate(wts):
            shape = [1] * len(wts)
            shape[i] = -1
            wgrid = wgrid * wt.reshape(shape)
        vel = grids[:dim]
        xi2 = grids[dim]
        return vel, xi2, rho * (lam / math.pi) ** ((dim + K) / 2) * wgrid

    def psi(self, vel, xi2):
        dim = self.dim
        out = [np.ones_like(vel[0])] + [vel[d] for d in range(dim)]
        out.append(0.5 * (sum(vel[d] ** 2 for d in range(dim)) + xi2))
        return out


def lin(a, psi):
    return sum(a[j] * psi[j] for j in range(len(psi)))


@pytest.mark.parametrize("dim", [2, 3])
def test_uniform_state_gives_euler_flux(dim):
    """A uniform state with zero slopes must give exactly the Euler flux, and the
    point value must equal the state, for any tau and dt (Sec 2.3)."""
    rng = np.random.default_rng(7 + dim)
    cfg = oracle.cfg_vector(dim)
    for _ in range(5):
        W = random_state(rng, dim)
        G = np.zeros((dim, dim + 2))
        for dt in (1e-3, 0.37, 5.0):
            F, Wt, dbg = oracle.gks_point(dim, cfg, W, G, W, G, dt)
            np.testing.assert_allclose(F, euler_flux_local(dim, W), rtol=1e-13, atol=1e-13)
            np.testing.assert_allclose(Wt, W, rtol=1e-13, atol=1e-13)
            np.testing.assert_allclose(dbg["Wc"], W, rtol=1e-14)


@pytest.mark.parametrize("dim", [2, 3])
def test_gks_against_brute_force_quadrature(dim):
    """Every coefficient and both outputs of the flux against direct quadrature
    of Eqs. dis1 + dis2 over velocity space and time."""
    rng = np.random.default_rng(11 + dim)
    nv = dim + 2
    bm = BruteMaxwellian(dim)
    c1, c2 = 0.01, 1.0
    cfg = oracle.cfg_vector(dim, tau_c1=c1, tau_c2=c2)
    for trial in range(2):
        Wl, Wr = random_state(rng, dim), random_state(rng, dim)
        Gl = 0.3 * rng.standard_normal((dim, nv))
        Gr = 0.3 * rng.standard_normal((dim, nv))
        dt = [0.05, 0.8][trial]
        F, Wt, d = oracle.gks_point(dim, cfg, Wl, Gl, Wr, Gr, dt)
        (vl, xl, gl), (vr, xr, gr) = bm.nodes(Wl), bm.nodes(Wr)
        psl, psr = bm.psi(vl, xl), bm.psi(vr, xr)
        # slopes: <psi (a_d . psi)> = dW/dx_d ; compatibility <psi (A + a.u)> = 0
        for side, (vel, ps, g, G, a, A) in enumerate(((vl, psl, gl, Gl, d["al"], d["Al"]),
                                                      (vr, psr, gr, Gr, d["ar"], d["Ar"]))):
            for dd in range(dim):
                mom = np.array([np.sum(ps[i] * lin(a[dd], ps) * g) for i in range(nv)])
                np.testing.assert_allclose(mom, G[dd], rtol=1e-10, atol=1e-10)
            au = sum(lin(a[dd], ps) * vel[dd] for dd in range(dim))
            comp = np.array([np.sum(ps[i] * (lin(A, ps) + au) * g) for i in range(nv)])
            np.testing.assert_allclose(comp, 0.0, atol=1e-10)
        # interface equilibrium from half-space moments (Eq. compatibility2)
        Hl = (vl[0] > 0).astype(float)
        Hr = (vr[0] < 0).astype(float)
        Wc = np.array([np.sum(psl[i] * Hl * gl) + np.sum(psr[i] * Hr * gr) for i in range(nv)])
        np.testing.assert_allclose(d["Wc"], Wc, rtol=1e-11)
        vc, xc, gc = bm.nodes(d["Wc"])
        psc = bm.psi(vc, xc)
        for dd in range(dim):
            mom = np.array([np.sum(psc[i] * lin(d["ac"][dd], psc) * gc) for i in range(nv)])
            np.testing.assert_allclose(mom, 0.5 * (Gl[dd] + Gr[dd]), rtol=1e-10, atol=1e-10)
        auc = sum(lin(d["ac"][dd], psc) * vc[dd] for dd in range(dim))
        comp = np.array([np.sum(psc[i] * (lin(d["Ac"], psc) + auc) * gc) for i in range(nv)])
        np.testing.assert_allclose(comp, 0.0, atol=1e-10)
        pl = (GAMMA - 1) * (Wl[-1] - 0.5 * np.dot(Wl[1:1 + dim], Wl[1:1 + dim]) / Wl[0])
        pr = (GAMMA - 1) * (Wr[-1] - 0.5 * np.dot(Wr[1:1 + dim], Wr[1:1 + dim]) / Wr[0])
        tau = c1 * dt + c2 * abs(pl - pr) / (pl + pr) * dt
        assert abs(d["tau"] - tau) <= 1e-15 * tau
        # velocity integrals of each term of f, then the time behaviour by quadrature
        aul = sum(lin(d["al"][dd], psl) * vl[dd] for dd in range(dim))
        aur = sum(lin(d["ar"][dd], psr) * vr[dd] for dd in range(dim))

        def terms(weight_l, weight_r, weight_c):
            V1 = np.array([np.sum(weight_c * psc[i] * gc) for i in range(nv)])
            V2 = np.array([np.sum(weight_c * psc[i] * auc * gc) for i in range(nv)])
            V3 = np.array([np.sum(weight_c * psc[i] * lin(d["Ac"], psc) * gc) for i in range(nv)])
            K0 = np.array([np.sum(weight_l * psl[i] * Hl * gl * (1 - tau * (aul + lin(d["Al"], psl))))
                           + np.sum(weight_r * psr[i] * Hr * gr * (1 - tau * (aur + lin(d["Ar"], psr))))
                           for i in range(nv)])
            K1 = np.array([-np.sum(weight_l * psl[i] * Hl * gl * aul) - np.sum(weight_r * psr[i] * Hr * gr * aur)
                           for i in range(nv)])
            return V1, V2, V3, K0, K1

        def coeffs(t):
            e = np.exp(-t / tau)
            return 1 - e, (t + tau) * e - tau, t - tau + tau * e, e, t * e

        # flux: time average of F(t) by composite Gauss-Legendre
        V1, V2, V3, K0, K1 = terms(vl[0], vr[0], vc[0])
        xt, wt = np.polynomial.legendre.leggauss(64)
        cut = min(60 * tau, dt)
        Fb = np.zeros(nv)
        for a, b in ((0.0, cut), (cut, dt)):
            if b <= a:
                continue
            t = a + (b - a) * 0.5 * (xt + 1)
            w = (b - a) * 0.5 * wt
            C1, C2, C3, E0, E1 = coeffs(t)
            Fb += (np.sum(w * C1) * V1 + np.sum(w * C2) * V2 + np.sum(w * C3) * V3
                   + np.sum(w * E0) * K0 + np.sum(w * E1) * K1)
        Fb /= dt
        np.testing.assert_allclose(F, Fb, rtol=1e-9, atol=1e-10 * np.max(np.abs(Fb)))
        # point value at t = dt
        V1, V2, V3, K0, K1 = terms(1.0, 1.0, 1.0)
        C1, C2, C3, E0, E1 = coeffs(dt)
        Wb = C1 * V1 + C2 * V2 + C3 * V3 + E0 * K0 + E1 * K1
        np.testing.assert_allclose(Wt, Wb, rtol=1e-9, atol=1e-10 * np.max(np.abs(Wb)))


def mirror(dim, W):
    M = W.copy()
    M[1] = -M[1]
    return M


def mirror_grad(dim, G):
    """Derivatives of the mirrored field x_n -> -x_n with u_n -> -u_n."""
    M = G.copy()
    M[0] = -M[0]       # normal derivative flips
    M[:, 1] = -M[:, 1]  # normal momentum flips
    return M


@pytest.mark.parametrize("dim", [2, 3])
def test_gks_mirror_symmetry(dim):
    """Reflecting the problem through the face plane (l <-> r, x_n -> -x_n)
    negates mass, tangential momentum and energy fluxes and keeps the normal
    momentum flux; the point value is the mirror image."""
    rng = np.random.default_rng(3 + dim)
    cfg = oracle.cfg_vector(dim)
    nv = dim + 2
    for _ in range(4):
        Wl, Wr = random_state(rng, dim), random_state(rng, dim)
        Gl, Gr = 0.2 * rng.standard_normal((dim, nv)), 0.2 * rng.standard_normal((dim, nv))
        F, Wt, _ = oracle.gks_point(dim, cfg, Wl, Gl, Wr, Gr, 0.3)
        F2, Wt2, _ = oracle.gks_point(dim, cfg, mirror(dim, Wr), mirror_grad(dim, Gr),
                                      mirror(dim, Wl), mirror_grad(dim, Gl), 0.3)
        expect = -F.copy()
        expect[1] = F[1]
        np.testing.assert_allclose(F2, expect, rtol=1e-12, atol=1e-13)
        np.testing.assert_allclose(Wt2, mirror(dim, Wt), rtol=1e-12, atol=1e-13)


@pytest.mark.parametrize("dim", [2, 3])
def test_kfvs_limits(dim):
    """KFVS: a uniform state gives the Euler flux; when both sides move right
    with u_n sqrt(lambda) >> 1 the flux is the Euler flux of the left state."""
    rng = np.random.default_rng(5 + dim)
    for _ in range(4):
        W = random_state(rng, dim)
        np.testing.assert_allclose(oracle.kfvs_point(dim, GAMMA, W, W), euler_flux_local(dim, W),
                                   rtol=1e-13, atol=1e-13)
    rho, p = 1.0, 1.0
    u = np.zeros(dim)
    u[0] = 30.0
    Wl = np.concatenate([[rho], rho * u, [p / (GAMMA - 1) + 0.5 * rho * 900.0]])
    # the right state moves right just as fast: nothing crosses the face leftwards
    Wr = np.concatenate([[0.7], 0.7 * u, [1.3 / (GAMMA - 1) + 0.5 * 0.7 * 900.0]])
    np.testing.assert_allclose(oracle.kfvs_point(dim, GAMMA, Wl, Wr), euler_flux_local(dim, Wl),
                               rtol=1e-12)


@pytest.mark.parametrize("dim", [2, 3])
def test_df_closed_form(dim):
    """DF point factor 1/(1+D^2) with D from pressure jumps and Mach jumps (Sec 3.3)."""
    rng = np.random.default_rng(9)
    W = random_state(rng, dim)
    assert oracle.df_point(dim, GAMMA, W, W) == 1.0
    Wl, Wr = random_state(rng, dim), random_state(rng, dim)

    def prim(W):
        rho = W[0]
        u = W[1:1 + dim] / rho
        p = (GAMMA - 1) * (W[-1] - 0.5 * rho * u @ u)
        return p, u / math.sqrt(GAMMA * p / rho)
    pl, ml = prim(Wl)
    pr, mr = prim(Wr)
    D = abs(pl - pr) / pl + abs(pl - pr) / pr + (ml[0] - mr[0]) ** 2 + np.sum((ml[1:] - mr[1:]) ** 2)
    assert abs(oracle.df_point(dim, GAMMA, Wl, Wr) - 1 / (1 + D * D)) < 1e-15


@pytest.mark.parametrize("dim", [2, 3])
def test_vacuum_interface_takes_collisionless_limit(dim):
    """Two states rushing apart (|u_n| sqrt(lambda) ~ 12): the half-space
    moments leave no admissible interface equilibrium, and the point falls back
    to the collisionless limit: finite, equal to the KFVS flux, and nearly zero
    (nothing crosses the face)."""
    nv = dim + 2
    rho, p = 1e-3, 1e-4
    u = np.zeros(dim)
    u[0] = -4.0
    Wl = np.concatenate([[rho], rho * u, [p / (GAMMA - 1) + 0.5 * rho * 16.0]])
    Wr = Wl.copy()
    Wr[1] = -Wl[1]
    G = np.zeros((dim, nv))
    F, Wt, _ = oracle.gks_point(dim, oracle.cfg_vector(dim), Wl, G, Wr, G, 0.1)
    assert np.all(np.isfinite(F)) and np.all(np.isfinite(Wt))
    np.testing.assert_allclose(F, oracle.kfvs_point(dim, GAMMA, Wl, Wr), rtol=0, atol=1e-30)
    assert np.max(np.abs(F)) < 1e-30
