"""Pins of the oracle's Navier-Stokes gas-kinetic flux (Sec 2.1: first-order
Chapman-Enskog truncation with tau = mu / p, Pr = 1) and of its no-slip
adiabatic wall.

For continuous data (the same state and slopes on both sides) of a steady
inviscid field, the time-averaged gas-kinetic flux is exactly the Euler flux
minus tau times the moments of u psi (a . u) g: with tau = mu / p that is the
Navier-Stokes flux of a BGK gas, whatever the time step.  Two such fields have
closed forms from continuum mechanics:
  * plane Couette shear, u_t = U0 + gamma_dot n at uniform rho, p: the shear
    stress mu gamma_dot and its work U0 mu gamma_dot;
  * heat conduction in a gas at rest, rho(n) at uniform p: Fourier's law with
    kappa = mu c_p (Pr = 1), c_p = gamma / (gamma - 1).
The no-slip wall reverses the velocity in its ghost: the face flux is then odd
in velocity for mass and energy, so a cell closed by such walls keeps its mass
and energy exactly, for any state and slopes.  The characteristic far field is
pinned by the invariants that define it.
"""
import numpy as np
import pytest

import oracle
from paper_2509_06347_b300 import synth

GAMMA = 1.4


def _cfg(dim, mu, c1=0.01, c2=1.0):
    return oracle.cfg_vector(dim, mu=mu, tau_c1=c1, tau_c2=c2)


@pytest.mark.parametrize("dim", [2, 3])
@pytest.mark.parametrize("dt", [1e-3, 0.3])
def test_couette_shear_stress(dim, dt):
    rho, p, U0, gd, mu = 1.2, 0.8, 0.35, 0.7, 0.013
    nv = dim + 2
    W = np.zeros(nv)
    W[0], W[2] = rho, rho * U0
    W[-1] = p / (GAMMA - 1) + 0.5 * rho * U0 * U0
    dW = np.zeros((dim, nv))
    dW[0, 2] = rho * gd            # d(rho u_t)/dn
    dW[0, -1] = rho * U0 * gd      # dE/dn at uniform p
    F, _, _ = oracle.gks_point(dim, _cfg(dim, mu), W, dW, W, dW, dt)
    expect = np.zeros(nv)
    expect[1] = p
    expect[2] = -mu * gd
    expect[-1] = -mu * gd * U0
    np.testing.assert_allclose(F, expect, rtol=0, atol=1e-13)
    # the Euler collision time C1 dt takes mu / p's place when mu = 0
    F0, _, _ = oracle.gks_point(dim, _cfg(dim, 0.0, c1=0.05), W, dW, W, dW, dt)
    np.testing.assert_allclose(F0[2], -0.05 * dt * p * gd, rtol=1e-12)


@pytest.mark.parametrize("dim", [2, 3])
def test_fourier_heat_flux_pr1(dim):
    rho, p, drho, mu = 0.9, 1.1, 0.4, 0.02
    nv = dim + 2
    W = np.zeros(nv)
    W[0], W[-1] = rho, p / (GAMMA - 1)
    dW = np.zeros((dim, nv))
    dW[0, 0] = drho
    F, _, _ = oracle.gks_point(dim, _cfg(dim, mu), W, dW, W, dW, 0.01)
    kappa = mu * GAMMA / (GAMMA - 1)
    dT = -p * drho / rho ** 2      # T = p / rho
    expect = np.zeros(nv)
    expect[1] = p
    expect[-1] = -kappa * dT
    np.testing.assert_allclose(F, expect, rtol=0, atol=1e-13)


@pytest.mark.parametrize("dim", [2, 3])
def test_noslip_cell_keeps_mass_and_energy(dim):
    """One simplex closed by no-slip walls: zero mass and energy residual for a
    random state and random slopes; the momentum residual is not zero (the
    walls exert a force).  The same cell closed by slip walls keeps its
    tangential momentum balance different: the two walls differ."""
    rng = np.random.default_rng(17 + dim)
    if dim == 2:
        xyz = np.array([[[0.0, 0.0], [1.0, 0.1], [0.2, 0.9]]])
        bn = np.array([[1, 2], [2, 0], [0, 1]], np.int32)
    else:
        xyz = np.array([[[0.0, 0.0, 0.0], [1.0, 0.1, 0.0], [0.2, 0.9, 0.1], [0.1, 0.2, 0.8]]])
        bn = np.array([[1, 2, 3], [0, 2, 3], [0, 1, 3], [0, 1, 2]], np.int32)
    nv = dim + 2
    cn = np.arange(dim + 1, dtype=np.int32)[None, :]
    out = {}
    for tag in (synth.TAG_NOSLIP_WALL, synth.TAG_WALL):
        m = dict(dim=dim, cell_nodes=cn, cell_xyz=xyz, bface_nodes=bn,
                 bface_tag=np.full(len(bn), tag, np.int32), parents=[])
        om = oracle.OracleMesh(m, levels=1)
        u = rng.uniform(-0.4, 0.4, dim) if tag == synth.TAG_NOSLIP_WALL else out["u"]
        out["u"] = u
        W = np.zeros((1, nv))
        W[0, 0] = 1.1
        W[0, 1:1 + dim] = 1.1 * u
        W[0, -1] = 0.9 / (GAMMA - 1) + 0.5 * 1.1 * u @ u
        G = 0.3 * np.random.default_rng(5).standard_normal((1, nv, dim))
        cfg = oracle.cfg_vector(dim, mu=0.02)
        R = om.residual(cfg, W, G, np.ones(1))["R"][0]
        scale = np.max(np.abs(W))
        if tag == synth.TAG_NOSLIP_WALL:
            assert abs(R[0]) < 1e-14 * scale and abs(R[-1]) < 1e-14 * scale, R
            assert np.max(np.abs(R[1:1 + dim])) > 1e-6
        out[tag] = R
    assert np.max(np.abs(out[synth.TAG_NOSLIP_WALL][1:1 + dim] - out[synth.TAG_WALL][1:1 + dim])) > 1e-6


def _riemann(W, n, dim):
    rho = W[0]
    u = W[1:1 + dim] / rho
    p = (GAMMA - 1) * (W[-1] - 0.5 * rho * u @ u)
    c = np.sqrt(GAMMA * p / rho)
    un = u @ n
    return un + 2 * c / (GAMMA - 1), un - 2 * c / (GAMMA - 1), p / rho ** GAMMA, u - un * n, un, c


@pytest.mark.parametrize("dim", [2, 3])
def test_characteristic_farfield(dim):
    """The far-field state of tag 4 is defined by its invariants: on a subsonic
    face it carries the outgoing invariant J+ = u_n + 2c/(gamma-1) of the
    interior and the incoming J- = u_n - 2c/(gamma-1) of the free stream, with
    the entropy p/rho^gamma and tangential velocity of the upstream side; a
    supersonic normal free stream gives the upwind state; an interior equal to
    the free stream is returned unchanged."""
    rng = np.random.default_rng(40 + dim)
    nv = dim + 2
    n = rng.standard_normal(dim)
    n /= np.linalg.norm(n)
    for mach in (0.3, 0.8):
        d = rng.standard_normal(dim)
        d -= (d @ n) * n
        d /= np.linalg.norm(d)
        for sgn in (-1.0, 1.0):  # inflow / outflow
            uf = mach * (sgn * 0.6 * n + 0.8 * d)
            wf = np.concatenate([[1.0], uf, [1 / (GAMMA * (GAMMA - 1)) + 0.5 * uf @ uf]])
            cfg = oracle.cfg_vector(dim, winf=wf)
            np.testing.assert_allclose(oracle.ghost_state(dim, cfg, 4, n, wf), wf, rtol=1e-14, atol=1e-15)
            ui = uf + 0.05 * rng.standard_normal(dim)
            Wi = np.concatenate([[0.95], 0.95 * ui, [1.05 / (GAMMA - 1) + 0.5 * 0.95 * ui @ ui]])
            Wb = oracle.ghost_state(dim, cfg, 4, n, Wi)
            jp_b, jm_b, s_b, ut_b, un_b, _ = _riemann(Wb, n, dim)
            jp_i, _, s_i, ut_i, _, _ = _riemann(Wi, n, dim)
            _, jm_f, s_f, ut_f, _, _ = _riemann(wf, n, dim)
            assert abs(jp_b - jp_i) < 1e-13 and abs(jm_b - jm_f) < 1e-13
            up_s, up_t = (s_f, ut_f) if un_b < 0 else (s_i, ut_i)
            assert abs(s_b - up_s) < 1e-13 * up_s
            np.testing.assert_allclose(ut_b, up_t, rtol=0, atol=1e-13)
    # supersonic normal flow: upwind state
    uf = 2.0 * n
    wf = np.concatenate([[1.0], uf, [1 / (GAMMA * (GAMMA - 1)) + 0.5 * uf @ uf]])
    Wi = wf * 1.01
    cfg = oracle.cfg_vector(dim, winf=wf)
    np.testing.assert_array_equal(oracle.ghost_state(dim, cfg, 4, n, Wi), Wi)      # outflow
    np.testing.assert_array_equal(oracle.ghost_state(dim, cfg, 4, -n, Wi), wf)     # inflow


def test_characteristic_farfield_preserves_free_stream():
    """A uniform free stream on the cylinder with every boundary a tag-4 far
    field has zero residual."""
    m = dict(synth.cylinder_mesh(16, 8, n_refine=1))
    m["bface_tag"] = np.full_like(m["bface_tag"], 4)
    w = synth.freestream(0.4, angle_deg=15.0)
    om = oracle.OracleMesh(m, levels=1)
    W = synth.uniform_state(m, w)
    n = len(W)
    R = om.residual(oracle.cfg_vector(2, winf=w, mu=0.01), W, np.zeros((n, 4, 2)), np.ones(n))["R"]
    assert np.max(np.abs(R)) < 1e-13
