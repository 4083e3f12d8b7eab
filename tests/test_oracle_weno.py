"""Pins of the oracle's nonlinear HWENO combination (Sec 3.3; the paper defers
the weights, read here as WENO-Z-type weights of one large and one sub
stencil): the equal-indicator limit, two hand-worked cases, and the
smoothness indicators recomputed on real cells by independent quadrature."""
import numpy as np
import pytest

import oracle
from paper_2509_06347_b300 import synth
from helpers import _TET2, _TRI2, physical_quadratic_state


@pytest.mark.parametrize("beta", [0.0, 1e-30, 0.37, 2.5e6])
@pytest.mark.parametrize("gh", [0.95, 0.6])
def test_equal_indicators_give_p2(beta, gh):
    """beta_1 = beta_2 makes tau_Z = 0, the weights fall back to the linear
    weights, and P = (1/gamma_H)(p2 - gamma_L p1) gamma_H + gamma_L p1 = p2
    exactly, for any p1.  (A combination w_H p2 + w_L p1 would give
    gamma_H p2 + gamma_L p1 here.)"""
    rng = np.random.default_rng(3)
    c1, c2 = rng.standard_normal(10), rng.standard_normal(10)
    P = oracle.hweno_combine(beta, beta, gh, 1e-15, c1, c2)
    np.testing.assert_allclose(P, c2, rtol=0, atol=1e-14 * np.max(np.abs(c2)))


def test_hand_worked_weights():
    """beta_1 = 1, beta_2 = 3, gamma_H = 19/20, eps -> 0: tau = 2,
    w~H = 19/20 * 5/3 = 19/12, w~L = 1/20 * 3 = 3/20, so (w_H, w_L) =
    (95/104, 9/104) and P = (100/104)(p2 - p1/20) + (9/104) p1 = (25 p2 + p1)/26.
    Swapped (beta_1 = 3, beta_2 = 1): w~H = 57/20, w~L = 1/12, (w_H, w_L) =
    (171/176, 5/176) and P = (45 p2 - p1)/44.  A squared ratio (tau/beta)^2
    would give (w_H, w_L) = (247/292, 45/292) in the first case."""
    c1 = np.array([1.0, -2.0, 0.5, 3.0])
    c2 = np.array([4.0, 1.0, -1.5, 0.25])
    P = oracle.hweno_combine(1.0, 3.0, 0.95, 1e-300, c1, c2)
    np.testing.assert_allclose(P, (25 * c2 + c1) / 26, rtol=1e-14, atol=1e-14)
    P = oracle.hweno_combine(3.0, 1.0, 0.95, 1e-300, c1, c2)
    np.testing.assert_allclose(P, (45 * c2 - c1) / 44, rtol=1e-14, atol=1e-14)


def test_smooth_sub_stencil_dominates():
    """beta_1 = 0 < beta_2: w~L = gamma_L (1 + beta_2/eps) dominates and P -> p1
    with an error of relative order eps / beta_2."""
    c1 = np.array([1.0, 0.2, -0.1])
    c2 = np.array([1.3, -0.4, 0.7])
    P = oracle.hweno_combine(0.0, 1.0, 0.95, 1e-15, c1, c2)
    np.testing.assert_allclose(P, c1, rtol=0, atol=1e-13)


def _quad_grad(dim, c, X):
    """Gradient at X [..., dim] of c0 + c_d X_d + sum_{d<=e} c_de X_d X_e."""
    g = np.broadcast_to(c[1:1 + dim], X.shape[:-1] + (dim,)).copy()
    k = 1 + dim
    for d in range(dim):
        for e in range(d, dim):
            if d == e:
                g[..., d] += 2 * c[k] * X[..., d]
            else:
                g[..., d] += c[k] * X[..., e]
                g[..., e] += c[k] * X[..., d]
            k += 1
    return g


def _second_derivatives(dim, c):
    """D^l p for the multi-indices |l| = 2, each once: d_dd = 2 c_dd, d_de = c_de."""
    out, k = [], 1 + dim
    for d in range(dim):
        for e in range(d, dim):
            out.append(2 * c[k] if d == e else c[k])
            k += 1
    return np.array(out)


@pytest.mark.parametrize("name", ["vortex", "sphere"])
def test_indicators_on_mesh(name):
    """On real cells: p2 is taken from the reconstruction with gamma_H = 1, p1
    is the Green-Gauss gradient (difference form) of the cell averages, and
    beta_q = sum_{1<=|l|<=deg} |Omega|^(2|l|/dim - 1) int (D^l p_q)^2 is
    integrated here with an exact degree-2 simplex rule.  The reconstruction at
    gamma_H = 0.95 must equal the pinned combination of p1 and p2 with these
    indicators."""
    m = synth.vortex_mesh(n_coarse=4, n_refine=2) if name == "vortex" else synth.sphere_mesh(n_panel=4, n_r=4)
    dim, nv = m["dim"], m["dim"] + 2
    nco = 6 if dim == 2 else 10
    om = oracle.OracleMesh(m, levels=1)
    rng = np.random.default_rng(17)
    xyz = m["cell_xyz"]
    W, G, _, _ = physical_quadratic_state(rng, dim, xyz, scale=0.2)
    n = len(W)
    ones = np.ones(n)
    P2, nb = om.reconstruct(oracle.cfg_vector(dim, weno_gamma_high=1.0), W, G, ones)
    P, nb2 = om.reconstruct(oracle.cfg_vector(dim), W, G, ones)
    assert nb == 0 and nb2 == 0
    vol, cen, _ = om.cells(0)
    F = om.faces(0)
    interior = F["R"] >= 0
    fl, fr, S, nrm = F["L"][interior], F["R"][interior], F["S"][interior], F["n"][interior]
    g1 = np.zeros((n, nv, dim))
    dW = (W[fr] - W[fl])[:, :, None] * (S[:, None] * nrm)[:, None, :]
    np.add.at(g1, fl, dW / (2 * vol[fl])[:, None, None])
    np.add.at(g1, fr, dW / (2 * vol[fr])[:, None, None])
    closed = np.ones(n, bool)
    closed[F["L"][~interior]] = False
    cells = np.nonzero(closed)[0]
    assert cells.size > n // 4
    bary, wq = (_TRI2 if dim == 2 else _TET2)
    s1, s2 = vol ** (2.0 / dim - 1.0), vol ** (4.0 / dim - 1.0)
    worst = 0.0
    for c in cells:
        X = bary @ xyz[c] - cen[c]  # quadrature points about the centroid
        for v in range(nv):
            c1 = np.zeros(nco)
            c1[0] = W[c, v]
            c1[1:1 + dim] = g1[c, v]
            c2 = P2[c, v]
            b1 = s1[c] * vol[c] * np.sum(g1[c, v] ** 2)
            gq = _quad_grad(dim, c2, X)
            b2 = s1[c] * vol[c] * np.sum(wq[:, None] * gq ** 2) + s2[c] * vol[c] * np.sum(_second_derivatives(dim, c2) ** 2)
            want = oracle.hweno_combine(b1, b2, 0.95, 1e-15, c1, c2)
            scale = np.max(np.abs(c2)) + np.max(np.abs(c1))
            worst = max(worst, float(np.max(np.abs(P[c, v] - want)) / scale))
    assert worst < 1e-12, worst
